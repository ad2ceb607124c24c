"""Batched step (gs_batch_*): one persistent launch over several scenes.

Every scene's result must be bit-identical to gs_step_camera on that scene
alone — through the autotuning phase (each candidate launch configuration in
turn) and through the captured graph — and match the FP64 oracle."""
import numpy as np
import pytest

from harness import GpuScene, OracleRun, assert_close
from paper_2601_16736_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

SIZES = [1, 257, 5_003, 40_000, 123_457]


@pytest.fixture(scope="module")
def G():
    from paper_2601_16736_gb300 import build
    build.build()
    from paper_2601_16736_gb300 import gsopt
    return gsopt


def _scenes(prec_name, G):
    runs_b, runs_s, cams = [], [], []
    for i, n in enumerate(SIZES):
        groups = synth.scene_blobs(n, 1200 + i, [6.0, 12.5, 22.0, 40.0, 75.0][i])
        rb = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec_name))
        rs = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec_name))
        g = synth.grads_rows(n, 1300 + i)
        rb.set_grads(g)
        rs.set_grads(g)
        runs_b.append(rb)
        runs_s.append(rs)
        cams.append(synth.ring_cameras(10, (0.0, 30.0)))
    return runs_b, runs_s, cams


def _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph):
    for s, (rb, rs) in enumerate(zip(runs_b, runs_s)):
        p = G.make_params(synth.lr_for_step(k, total), k, restate=(k % 5 == 0), restate_ratio=0.3, seed=s)
        cam = cams[s][(k * 7 + s) % len(cams[s])]
        b.set(s, G.make_attrs(rb.attrs), G.make_attrs(rb.grads), G.make_camera(cam), p)
        rs.step_camera(cam, p, mask_out=False)
        nvis[s] -= rs.nvis[0]
    G.gs_batch_step(b, nvis, graph=graph)


def _assert_same(runs_b, runs_s, nvis):
    torch.cuda.synchronize()
    assert int(nvis.abs().sum().item()) == 0          # same visible counts
    for rb, rs in zip(runs_b, runs_s):
        assert rb.rows().tobytes() == rs.rows().tobytes()
        mb, vb, tb = rb.state()
        ms, vs, ts = rs.state()
        assert mb.tobytes() == ms.tobytes() and vb.tobytes() == vs.tobytes() and tb.tobytes() == ts.tobytes()


@pytest.mark.parametrize("prec", ["FP32", "BF16_HYBRID", "FP16_BLOCK"])
def test_batch_equals_single_scene_steps(G, prec):
    """Eager calls until the tuner has run every candidate (each candidate in
    turn), then tuned eager calls, then graph replays."""
    runs_b, runs_s, cams = _scenes(prec, G)
    b = G.gs_batch_create([r.h for r in runs_b])
    nvis = torch.zeros(len(SIZES), dtype=torch.int64, device="cuda")
    total, k = 60, 0
    while not G.gs_batch_config(b)["tuned"]:
        k += 1
        assert k <= 40, "tuning did not finish"
        _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph=False)
    for _ in range(3):
        k += 1
        _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph=False)
    for _ in range(3):
        k += 1
        _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph=True)
    _assert_same(runs_b, runs_s, nvis)
    b.close()
    for r in runs_b + runs_s:
        r.close()


def _grow(G, run, n_add, seed):
    """Re-index a scene to n + n_add rows: the old rows keep their state, the
    new ones start fresh and copy the attributes of random old rows."""
    n = run.n
    rng = np.random.default_rng(seed)
    src = np.concatenate([np.arange(n), np.full(n_add, -1)]).astype(np.int32)
    attr_src = np.concatenate([np.arange(n), rng.integers(0, n, n_add)]).astype(np.int32)
    G.gs_reindex_state(run.h, torch.from_numpy(src).cuda(), None, src.size)
    out = {k: torch.empty((src.size,) + tuple(v.shape[1:]), dtype=v.dtype, device="cuda") for k, v in run.attrs.items()}
    G.gs_gather_attrs(run.h, G.make_attrs(run.attrs), n, G.make_attrs(out), torch.from_numpy(attr_src).cuda(), src.size)
    grads = {k: torch.zeros_like(v) for k, v in out.items()}
    for k, v in run.grads.items():
        grads[k][:n].copy_(v)
        grads[k][n:].copy_(v[torch.from_numpy(attr_src[n:]).cuda().long()])
    run.attrs, run.grads, run.n = out, grads, src.size


def test_batch_graph_follows_scene_sizes(G):
    """Graph replays, then one scene grows by a re-index (its tile count
    changes, and with it the batch's tile table and, for the one-CTA-per-tile
    form, the grid of the graph's kernel), then more graph replays: still
    bit-identical to single-scene steps."""
    runs_b, runs_s, cams = _scenes("FP32", G)
    b = G.gs_batch_create([r.h for r in runs_b])
    nvis = torch.zeros(len(SIZES), dtype=torch.int64, device="cuda")
    total, k = 60, 0
    while not G.gs_batch_config(b)["tuned"]:
        k += 1
        assert k <= 40, "tuning did not finish"
        _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph=False)
    for _ in range(3):
        k += 1
        _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph=True)
    for run in (runs_b[3], runs_s[3]):
        _grow(G, run, 20_011, 1250)
    for _ in range(4):
        k += 1
        _step_both(G, b, runs_b, runs_s, cams, nvis, k, total, graph=True)
    _assert_same(runs_b, runs_s, nvis)
    assert runs_b[3].n == SIZES[3] + 20_011
    b.close()
    for r in runs_b + runs_s:
        r.close()


def test_batch_matches_oracle(G, orc):
    """Two scenes in one batched launch against the oracle: 1e-5 after the
    first step, 1e-4 after 300 steps with RSR every 100.  Rows whose mean
    came within 1e-5 of a frustum plane at some step are left out of the
    300-step comparison: there the GPU (deciding on its FP32 means) and the
    oracle (on its FP64 means rounded to FP32) may see different sides."""
    sizes = [3_001, 20_011]
    runs, refs, cams = [], [], []
    for i, n in enumerate(sizes):
        groups = synth.scene_blobs(n, 1400 + i, 12.5)
        runs.append(GpuScene(groups))
        refs.append(OracleRun(orc, synth.to_rows(groups)))
        cams.append(synth.ring_cameras(6, (0.0, 30.0)))
    near = [np.zeros(n, bool) for n in sizes]
    b = G.gs_batch_create([r.h for r in runs])
    steps = 300
    for k in range(1, steps + 1):
        for s, (r, ref) in enumerate(zip(runs, refs)):
            g = synth.grads_rows(sizes[s], 1500 + s, k % 7)
            r.set_grads(g)
            lr = synth.lr_for_step(k, steps)
            cam = cams[s][k % len(cams[s])]
            rs = k % 100 == 0
            b.set(s, G.make_attrs(r.attrs), G.make_attrs(r.grads), G.make_camera(cam),
                  G.make_params(lr, k, restate=rs, restate_ratio=0.5, seed=7))
            margin, vis = orc.frustum_margin_f64(ref.st.theta[:, 0:3].astype(np.float32), cam)
            near[s] |= np.abs(margin) < 1e-5
            ref.step(g, vis, lr, True, True, k, restate=rs, ratio=0.5, seed=7)
        G.gs_batch_step(b)
        torch.cuda.synchronize()
        if k == 1:
            for r, ref in zip(runs, refs):
                assert_close(r.rows(), ref.st.theta, 1e-5, 1e-5, what="batched scene, step 1")
    for s, (r, ref) in enumerate(zip(runs, refs)):
        keep = ~near[s]
        assert keep.mean() > 0.99
        assert_close(r.rows(), ref.st.theta, 1e-4, rows=keep, what=f"batched scene, {steps} steps")
        _, _, t = r.state()
        assert np.array_equal(t[keep], ref.st.t[keep])
    b.close()
    for r in runs:
        r.close()


def test_batch_rejects_bad_sets(G):
    a = GpuScene(synth.scene_uniform(100, 1600))
    c = GpuScene(synth.scene_uniform(100, 1601), prec=G.GS_MOM_BF16)
    with pytest.raises(G.GsError):                 # mixed moment precisions
        G.gs_batch_create([a.h, c.h])
    with pytest.raises(G.GsError):                 # more than GS_MAX_BATCH scenes
        G.gs_batch_create([a.h] * (G.GS_MAX_BATCH + 1))
    a.close()
    c.close()
