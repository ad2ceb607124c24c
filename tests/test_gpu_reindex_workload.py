"""Steps interleaved with row-set changes (the re-index workload): every 100
steps an MCMC-style event prunes 5 % of the rows, appends clones of 5 % with
fresh state, and relocates 2 % (destination state reset).  The library
re-indexes its state (gs_reindex_state) and gathers the attributes
(gs_gather_attrs); the oracle does the same by its reindex and by indexing
the attribute rows (Sec. 2: new and relocated primitives start from zero
moments, App. "Scaling in RSR" item (1)).

Visibility: where the GPU's FP32 decision differs from the oracle's on the
oracle's own positions, the row must sit within the FP32 rounding band of a
frustum plane, and the oracle adopts the GPU's decision for it, so both
trajectories stay comparable on every row."""
import numpy as np
import pytest

from harness import check_trajectory_masks, GpuScene, OracleRun, assert_close, group_errors
from paper_2601_16736_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def G():
    from paper_2601_16736_gb300 import build
    build.build()
    from paper_2601_16736_gb300 import gsopt
    return gsopt


def _gather_attrs(G, run, attr_src):
    out = {k: torch.empty_like(v) for k, v in run.attrs.items()}
    src = torch.from_numpy(attr_src).cuda()
    G.gs_gather_attrs(run.h, G.make_attrs(run.attrs), run.n, G.make_attrs(out), src, attr_src.size)
    run.attrs = out
    run.grads = {k: torch.zeros_like(v) for k, v in out.items()}


@pytest.mark.parametrize("prec", ["FP32", "BF16_HYBRID", "FP16_BLOCK"])
def test_steps_with_reindex_events(G, orc, prec):
    n, steps, every, seed = 40_000, 350, 100, 1705
    groups = synth.scene_blobs(n, seed, 12.5)
    cams = synth.ring_cameras(20, (-15.0, 0.0, 15.0))
    order = synth.view_order(len(cams), steps, seed)
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    ref = OracleRun(orc, synth.to_rows(groups))
    adopted = 0
    for k in range(1, steps + 1):
        g = synth.grads_rows(n, seed, k)
        run.set_grads(g)
        cam = cams[order[k - 1]]
        lr = synth.lr_for_step(k, steps)
        rs = k % every == 0
        gxyz = run.attrs["xyz"].cpu().numpy()                  # the means this step decides on
        run.step_camera(cam, G.make_params(lr, k, restate=rs, restate_ratio=0.2, seed=seed))
        gmask = run.mask[:n].cpu().numpy()
        omask = ref.visible(cam)
        adopted += check_trajectory_masks(orc, gmask, omask, ref.st.theta[:, 0:3], gxyz, cam)
        ref.step(g, gmask, lr, True, True, k, restate=rs, ratio=0.2, seed=seed)
        if rs:
            src, reset, attr_src = synth.reindex_event(n, seed, k // every)
            assert src.size == n                    # prune and clone fractions match
            G.gs_reindex_state(run.h, torch.from_numpy(src).cuda(), torch.from_numpy(reset).cuda(), src.size)
            _gather_attrs(G, run, attr_src)
            theta = ref.st.theta[attr_src].copy()
            ref.st = orc.reindex(ref.st, src, reset)
            ref.st.theta[:] = theta
            assert G.gs_opt_rows(run.h) == n
    torch.cuda.synchronize()
    assert G.gs_opt_sync_errors(run.h) == 0
    got = run.rows()
    m, v, t = run.state()
    assert np.array_equal(t, ref.st.t), "step counters after re-index events"
    print(prec, "rows whose decision was adopted from the GPU:", adopted)
    if prec == "FP32":
        assert_close(got, ref.st.theta, 1e-4, what="after 350 steps and 3 re-index events")
        assert_close(m, ref.st.m, 1e-4, what="m")
        assert_close(v, ref.st.v, 1e-4, what="v")
    else:
        cols = {"xyz": slice(0, 3), "scale": slice(3, 6), "rot": slice(6, 10), "opacity": slice(10, 11),
                "sh": slice(11, 59)}
        for gname, sl in cols.items():
            e = np.linalg.norm(got[:, sl] - ref.st.theta[:, sl]) / np.linalg.norm(ref.st.theta[:, sl])
            assert e <= 1e-3, f"{prec} group {gname}: {e:.2e}"
        if prec == "BF16_HYBRID":        # the non-SH columns keep FP32 moments: as close as the FP32 path
            errs = group_errors(got, ref.st.theta)
            for gname in ("xyz", "scale", "rot", "opacity"):
                assert errs[gname][0] <= 1e-4, f"{gname}: {errs[gname][0]:.2e}"
    run.close()


@pytest.mark.parametrize("prec", ["FP32", "BF16_HYBRID", "FP16_BLOCK"])
def test_reindex_6m_sampled(G, orc, prec):
    """One event at 6 M rows (the size the re-index bench times), checked
    bit-exactly on 50 000 sampled output rows against the oracle's re-index
    of their source rows."""
    n = 6_000_000
    rng = np.random.default_rng(1706)
    h = G.gs_opt_init(G.make_config(prec=getattr(G, "GS_MOM_" + prec)), n)
    gen = torch.Generator(device="cuda").manual_seed(1706)
    m = torch.randn((n, 59), generator=gen, device="cuda")
    v = torch.rand((n, 59), generator=gen, device="cuda")
    t = torch.randint(0, 5000, (n,), generator=gen, device="cuda", dtype=torch.int32)
    G.gs_opt_import_state(h, m, v, t)
    m0 = torch.empty_like(m)
    v0 = torch.empty_like(v)
    t0 = torch.empty_like(t)
    G.gs_opt_export_state(h, m0, v0, t0)          # the stored (rounded) state
    src, reset, _ = synth.reindex_event(n, 1707, 0)
    G.gs_reindex_state(h, torch.from_numpy(src).cuda(), torch.from_numpy(reset).cuda(), src.size)
    m1 = torch.empty((src.size, 59), device="cuda")
    v1 = torch.empty_like(m1)
    t1 = torch.empty(src.size, dtype=torch.int32, device="cuda")
    G.gs_opt_export_state(h, m1, v1, t1)
    torch.cuda.synchronize()
    assert G.gs_opt_sync_errors(h) == 0
    sample = np.sort(rng.choice(src.size, 50_000, replace=False))
    # the oracle re-indexes a state made of exactly the sampled rows' sources
    s_src = src[sample]
    used = np.unique(s_src[s_src >= 0])
    pos = np.full(n, -1, np.int64)
    pos[used] = np.arange(used.size)
    ids = torch.from_numpy(used).cuda()
    st_in = orc.State(np.zeros((used.size, 59)), m0[ids].cpu().numpy(), v0[ids].cpu().numpy(),
                      t0[ids].cpu().numpy().view(np.uint32))
    local_src = np.where(s_src >= 0, pos[np.maximum(s_src, 0)], -1).astype(np.int32)
    out = orc.reindex(st_in, local_src, reset[sample])
    sid = torch.from_numpy(sample).cuda()
    assert np.array_equal(m1[sid].cpu().numpy().astype(np.float64), out.m)
    assert np.array_equal(v1[sid].cpu().numpy().astype(np.float64), out.v)
    assert np.array_equal(t1[sid].cpu().numpy().view(np.uint32), out.t)
    G.gs_opt_destroy(h)
