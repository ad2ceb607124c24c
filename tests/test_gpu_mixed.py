"""Low-precision moment storage (GS_MOM_BF16, GS_MOM_BF16_HYBRID,
GS_MOM_FP16_BLOCK; GS_MOM_FP8E4M3 in the 1000-step run, the rest of its
tests in test_gpu_fp8.py) against the FP64 oracle.

Bounds, from the arithmetic: the step computes every moment in FP32 and only
rounds the stored copy, so after one step from zero state the attributes are
as accurate as the FP32 path and each stored moment is within BF16's rounding
of the oracle's: half an ulp (2^-8 relative) when rounded to nearest, one ulp
(2^-7) when rounded stochastically (the second moments of BF16 columns).  For
FP16 blocks the ulp is 2^-10 relative for every value within 2^29 of its
group's largest magnitude; below that FP16 subnormals space values 2^-24
apart in the group's scaled units.  Over
many steps the rounded moments feed back; after 1000 steps of the 3 M
workload the metric's gate, group relative L2 ||d|| / ||theta_ref|| <= 1e-3,
is asserted for FP16 block and the hybrid.  All-BF16 and FP8 miss it (8 and 4
significant bits cannot carry a second moment that moves ~0.1 % per step, nor
the first moments of the opacity and SH-DC columns); they are held to a
recorded regression bound and reported as failing the gate.
"""
import numpy as np
import pytest

from harness import GpuScene, OracleRun, assert_close, group_errors
from paper_2601_16736_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

LR = synth.lr_for_step(1, 10)
BF16_HALF_ULP = 2.0 ** -8
FP16_HALF_ULP = 2.0 ** -11
# FP16-block groups in canonical columns: 6 x 8 SH, rotation, xyz + scale + opacity
F16B_GROUPS = [list(range(11 + 8 * g, 19 + 8 * g)) for g in range(6)] + [[6, 7, 8, 9], [0, 1, 2, 3, 4, 5, 10]]
LOWP = ["BF16", "BF16_HYBRID", "FP16_BLOCK"]
GROUP_COLS = {"xyz": slice(0, 3), "scale": slice(3, 6), "rot": slice(6, 10), "opacity": slice(10, 11),
              "sh": slice(11, 59)}


@pytest.fixture(scope="module")
def G():
    from paper_2601_16736_gb300 import build
    build.build()
    from paper_2601_16736_gb300 import gsopt
    return gsopt


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _group_exponent(blk):
    e = ((np.ascontiguousarray(blk, np.float32).view(np.uint32) >> 23) & 0xFF).max(axis=1).astype(np.int64)
    return np.where(e < 15, 0, e)


def _f16b(x, second_moment=False):
    """The FP16-block encoding restated: per row and group, the largest biased
    FP32 exponent e; values stored as FP16 (nearest) of x * 2^(141 - e); a
    positive second moment keeps at least the smallest FP16 subnormal."""
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros_like(x)
    for cols in F16B_GROUPS:
        blk = x[:, cols].astype(np.float64)
        e = _group_exponent(x[:, cols])
        sc = np.where(e > 0, np.ldexp(1.0, 141 - e), 0.0)
        h = (blk * sc[:, None]).astype(np.float32).astype(np.float16)
        if second_moment:
            h = np.where((h == 0) & (blk > 0) & (e[:, None] > 0), np.float16(2.0 ** -24), h)
        dec = np.where(e > 0, np.ldexp(1.0, e - 141), 0.0)
        out[:, cols] = (h.astype(np.float64) * dec[:, None]).astype(np.float32)
    return out


def _group_max(x):
    """Per element, the largest magnitude of its FP16-block group."""
    out = np.zeros(x.shape, np.float64)
    for cols in F16B_GROUPS:
        out[:, cols] = np.abs(x[:, cols]).max(axis=1, keepdims=True)
    return out


def group_rel_l2(got, ref, rows=None):
    out = {}
    for g, sl in GROUP_COLS.items():
        a = np.asarray(got[:, sl], np.float64)
        b = np.asarray(ref[:, sl], np.float64)
        if rows is not None:
            a, b = a[rows], b[rows]
        out[g] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return out


@pytest.mark.parametrize("prec", LOWP)
def test_one_step(G, orc, prec):
    n = 60_013
    groups = synth.scene_blobs(n, 901, 12.5)
    grads = synth.grads_rows(n, 902)
    cam = synth.ring_cameras(8)[2]
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    run.set_grads(grads)
    run.step_camera(cam, G.make_params(LR, 100, restate=True, restate_ratio=0.3, seed=9))
    got = run.rows()
    m, v, t = run.state()
    ref = OracleRun(orc, synth.to_rows(groups))
    vis = ref.visible(cam)
    ref.step(grads, vis, LR, True, True, 100, restate=True, ratio=0.3, seed=9)
    assert_close(got, ref.st.theta, 1e-5, 1e-5, what="theta")
    v_ulps = 2.0                                         # stochastic rounding: within one ulp
    half = FP16_HALF_ULP if prec == "FP16_BLOCK" else BF16_HALF_ULP
    for name, a, b, ulps in [("m", m, ref.st.m, 1.0), ("v", v, ref.st.v, v_ulps)]:
        d = np.abs(a - b)
        floor = 2.0 ** -37 * _group_max(b) if prec == "FP16_BLOCK" else 0.0     # FP16 subnormal spacing
        assert np.all(d <= ulps * half * np.abs(b) * (1 + 1e-5) + floor + 1e-30), f"{name} beyond {prec} rounding"
    if prec == "BF16_HYBRID":      # columns 0-13 (all but the SH rest) stay FP32
        assert_close(m[:, :14], ref.st.m[:, :14], 1e-5)
        assert_close(v[:, :14], ref.st.v[:, :14], 1e-5)
    assert np.array_equal(t, ref.st.t)
    run.close()


@pytest.mark.parametrize("prec", LOWP)
@pytest.mark.parametrize("n", [1, 33, 257, 513])
def test_edge_sizes(G, orc, prec, n):
    groups = synth.scene_uniform(n, 910 + n)
    rng = np.random.default_rng(n)
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    ref = OracleRun(orc, synth.to_rows(groups))
    for k in (1, 2, 3, 100):
        grads = synth.grads_rows(n, 911, k)
        mask_np = (rng.random(n) < 0.6).astype(np.uint8)
        run.set_grads(grads)
        p = G.make_params(LR, k, restate=(k == 100), restate_ratio=0.5, seed=3)
        run.step_mask(torch.from_numpy(mask_np).cuda(), p)
        ref.step(grads, mask_np, LR, True, True, k, restate=(k == 100), ratio=0.5, seed=3)
    # 4 steps with rounded moments fed back: a few BF16 ulps of lr-sized steps
    assert_close(run.rows(), ref.st.theta, 2e-3, what=prec)
    _, _, t = run.state()
    assert np.array_equal(t, ref.st.t)
    run.close()


@pytest.mark.parametrize("prec", LOWP)
def test_export_import_and_reindex(G, orc, prec):
    n = 20_001
    run = GpuScene(synth.scene_uniform(n, 920), prec=getattr(G, "GS_MOM_" + prec))
    rng = np.random.default_rng(921)
    m = rng.normal(size=(n, 59)).astype(np.float32)
    v = rng.random((n, 59)).astype(np.float32)
    t = rng.integers(0, 1000, n).astype(np.uint32)
    G.gs_opt_import_state(run.h, torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(),
                          torch.from_numpy(t.view(np.int32)).cuda())
    m2, v2, t2 = run.state()
    if prec == "FP16_BLOCK":
        em, ev = _f16b(m), _f16b(v, second_moment=True)
    else:
        em, ev = _bf16(m), _bf16(v)
    if prec == "BF16_HYBRID":
        em[:, :14], ev[:, :14] = m[:, :14], v[:, :14]
    assert m2.tobytes() == em.tobytes() and v2.tobytes() == ev.tobytes() and t2.tobytes() == t.tobytes()
    src, reset, _ = synth.reindex_event(n, 922, 0)
    G.gs_reindex_state(run.h, torch.from_numpy(src).cuda(), torch.from_numpy(reset).cuda(), src.size)
    run.n = src.size
    m3, v3, t3 = run.state()
    out = orc.reindex(orc.State(np.zeros((n, 59)), m2, v2, t2), src, reset)
    assert np.array_equal(m3.astype(np.float64), out.m) and np.array_equal(v3.astype(np.float64), out.v)
    assert np.array_equal(t3, out.t)
    run.close()


def _run_sampled(G, orc, wl, prec, sample):
    groups = wl.scene_groups()
    cams = wl.cameras()
    order = synth.view_order(len(cams), wl.steps, wl.seed)
    grads_host = [synth.grads_rows(wl.n, wl.seed, b) for b in range(wl.grad_buffers)]
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    gdev = [{k: torch.from_numpy(v).cuda() for k, v in synth.from_rows(gh).items()} for gh in grads_host]
    ids_t = torch.from_numpy(sample).cuda()
    ref = OracleRun(orc, synth.to_rows(groups)[sample], row_ids=sample)
    diverged = np.zeros(sample.size, bool)
    for k in range(1, wl.steps + 1):
        cam = cams[order[k - 1]]
        b = (k - 1) % len(gdev)
        lr = synth.lr_for_step(k, wl.steps)
        rs = k % wl.restate_every == 0
        p = G.make_params(lr, k, restate=rs, restate_ratio=wl.restate_ratio, seed=wl.seed)
        G.gs_step_camera(run.h, G.make_attrs(run.attrs), G.make_attrs(gdev[b]), G.make_camera(cam), p,
                         mask_out=run.mask)
        gmask = run.mask[ids_t].cpu().numpy()
        omask = ref.visible(cam)
        diverged |= gmask != omask
        ref.step(grads_host[b][sample], omask, lr, True, True, k, restate=rs, ratio=wl.restate_ratio,
                 seed=wl.seed)
    got = run.rows()[sample]
    run.close()
    return got, ref.st.theta, ~diverged


# (format, meets the 1e-3 gate, regression bound on the largest group error)
MIXED_3M = [("FP32", True, 1e-4), ("FP16_BLOCK", True, 1e-3), ("BF16_HYBRID", True, 1e-3), ("BF16", False, 3e-2),
            ("FP8E4M3", False, 0.1)]


@pytest.mark.parametrize("prec,meets_gate,bound", MIXED_3M)
def test_3m_1000_steps_sampled(G, orc, prec, meets_gate, bound):
    """The 3 M-primitive, 1000-step workload (about 20 % visible per view),
    followed by the oracle on 2000 sampled primitives.  FP32 moments are held
    to the FP32 parity bound after 1000 steps (1e-4); the formats that
    meet the 1e-3 gate are asserted against it; the others are held to a
    recorded regression bound and then marked as failing the gate (xfail,
    with the measured error), which is not a pass."""
    wl = synth.WORKLOADS["c3_3m"]
    sample = np.sort(np.random.default_rng(17).choice(wl.n, 2000, replace=False))
    got, ref, keep = _run_sampled(G, orc, wl, prec, sample)
    assert keep.mean() > (0.998 if meets_gate else 0.9)
    errs = group_rel_l2(got, ref, rows=keep)
    worst = max(errs.values())
    print(prec, "group relative L2 after 1000 steps:", errs)
    for g, e in errs.items():
        assert np.isfinite(e) and e <= bound, f"{prec} group {g}: {e:.2e} > {bound:.0e}"
    if not meets_gate:
        pytest.xfail(f"{prec}: largest group error {worst:.2e} after 1000 steps, above the 1e-3 gate")


def test_fp16_block_with_optional_terms(G, orc):
    """Noise on every row, AIU, RSR and the active count with FP16-block
    moments: attributes follow the oracle to the mixed-precision bound, and
    the count equals the classification of the GPU's own logits."""
    n = 20_011
    groups = synth.scene_uniform(n, 930)
    run = GpuScene(groups, prec=G.GS_MOM_FP16_BLOCK)
    st = orc.State(synth.to_rows(groups))
    cfg = orc.Config(n_i=orc.dar_normaliser(800 * 800))
    rng = np.random.default_rng(931)
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    for k in range(1, 7):
        g = synth.grads_rows(n, 932, k)
        mask = (rng.random(n) < 0.4).astype(np.uint8)
        kw = dict(noise=2, noise_lr=50.0, noise_k=3.0, noise_t=0.5, aiu=k > 2, aiu_prob=0.3, aiu_scale=0.5)
        ext = orc.Ext(noise_mode=2, aiu=k > 2, noise_lr=50.0, noise_k=3.0, noise_t=0.5, aiu_prob=0.3,
                      aiu_scale=0.5, seed=13)
        rs = k == 4
        run.set_grads(g)
        na.zero_()
        run.step_mask(torch.from_numpy(mask).cuda(),
                      G.make_params(LR, k, restate=rs, restate_ratio=0.4, seed=13, n_active=na, **kw))
        orc.step_ext(cfg, st, g, mask, LR, True, True, k, ext)
        if rs:
            orc.restate(cfg, st, 13, k, 0.4)
        assert int(na.item()) == orc.active_rows(run.attrs["opacity"].cpu().numpy().ravel()).size
    assert_close(run.rows(), st.theta, 2e-3, what="FP16 block with noise, AIU, RSR")
    _, _, t = run.state()
    assert np.array_equal(t, st.t)
    run.close()
