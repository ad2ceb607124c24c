"""Position noise (App. Eq. disentangled_mu), AIU (Sec. 3.2) and the active
count / prune list (Sec. 4, opacity > 1/255) through the C ABI, against the
FP64 oracle.

Steps take the caller's mask here, so both sides update exactly the same
rows while the noise moves the means.  Tolerances: the noise is formed in
FP32 (Box-Muller and the covariance product, a few ulp of the noise term),
so positions follow the oracle to the FP32 bound used for the plain step.
The active decision is an integer decided by floating point: the GPU's count
must equal the oracle's classification of the GPU's own FP32 logits."""
import numpy as np
import pytest

from harness import GpuScene, assert_close
from paper_2601_16736_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

LR = synth.lr_for_step(1, 10)


@pytest.fixture(scope="module")
def G():
    from paper_2601_16736_gb300 import build
    build.build()
    from paper_2601_16736_gb300 import gsopt
    return gsopt


def _noisy_scene(n, seed):
    """Large, half-transparent primitives so the noise gate and Sigma are
    far from zero; opacity logits straddle the 1/255 threshold."""
    g = synth.scene_uniform(n, seed)
    rng = np.random.default_rng(seed + 1)
    g["scale"] = rng.normal(-1.2, 0.3, (n, 3)).astype(np.float32)
    op = rng.normal(0.0, 1.0, (n, 1))
    op[::3] = rng.normal(-5.537, 0.05, (len(op[::3]), 1))     # near -ln 254
    g["opacity"] = op.astype(np.float32)
    return g


def _ext(G, orc, **kw):
    o = dict(noise=0, noise_lr=5e5, noise_k=100.0, noise_t=0.005, aiu=False, aiu_prob=0.0, aiu_scale=1.0)
    o.update(kw)
    return o, orc.Ext(noise_mode=o["noise"], aiu=o["aiu"], noise_lr=o["noise_lr"], noise_k=o["noise_k"],
                      noise_t=o["noise_t"], aiu_prob=o["aiu_prob"], aiu_scale=o["aiu_scale"])


@pytest.mark.parametrize("prec", ["FP32", "BF16_HYBRID", "FP16_BLOCK"])
def test_term_kernels_without_terms_are_the_plain_step(G, prec):
    """The terms form of the step kernel (active count only) and the extended
    kernel (noise on every row with eta_Ro = 0, so the noise is exactly zero,
    plus the count) must give the plain kernel's results bit for bit: the
    same per-element arithmetic.  Their counts must agree."""
    n = 20_011
    groups = synth.scene_uniform(n, 1900)
    pr = getattr(G, "GS_MOM_" + prec)
    a, b, c = GpuScene(groups, prec=pr), GpuScene(groups, prec=pr), GpuScene(groups, prec=pr)
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    nc = torch.zeros(1, dtype=torch.int64, device="cuda")
    rng = np.random.default_rng(1901)
    for k in range(1, 6):
        g = synth.grads_rows(n, 1902, k)
        mask = torch.from_numpy((rng.random(n) < 0.5).astype(np.uint8)).cuda()
        for r in (a, b, c):
            r.set_grads(g)
        kw = dict(restate=(k == 3), restate_ratio=0.4, seed=5)
        nb.zero_()
        nc.zero_()
        a.step_mask(mask, G.make_params(LR, k, **kw))
        b.step_mask(mask, G.make_params(LR, k, n_active=nb, **kw))
        c.step_mask(mask, G.make_params(LR, k, n_active=nc, noise=2, noise_lr=0.0, **kw))
        torch.cuda.synchronize()
        assert nb.item() == nc.item() > 0
    ra = a.rows().tobytes()
    assert b.rows().tobytes() == ra and c.rows().tobytes() == ra
    for x, y, z in zip(a.state(), b.state(), c.state()):
        assert x.tobytes() == y.tobytes() == z.tobytes()
    for r in (a, b, c):
        r.close()


@pytest.mark.parametrize("prec", ["FP32", "BF16_HYBRID", "FP16_BLOCK"])
@pytest.mark.parametrize("mode", [1, 2])
def test_noise_matches_oracle(G, orc, prec, mode):
    n = 30_007
    groups = _noisy_scene(n, 1910)
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    st = orc.State(synth.to_rows(groups))
    cfg = orc.Config(n_i=orc.dar_normaliser(800 * 800))
    rng = np.random.default_rng(1911)
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    for k in range(1, 9):
        g = synth.grads_rows(n, 1912, k)
        mask = (rng.random(n) < 0.4).astype(np.uint8)
        lr = synth.lr_for_step(k, 8)
        o, ext = _ext(G, orc, noise=mode, noise_lr=400.0, noise_k=3.0, noise_t=0.5)
        ext.seed = 77
        rs = k == 4
        run.set_grads(g)
        na.zero_()
        run.step_mask(torch.from_numpy(mask).cuda(),
                      G.make_params(lr, k, restate=rs, restate_ratio=0.3, seed=77, n_active=na, **o))
        orc.step_ext(cfg, st, g, mask, lr, True, True, k, ext)
        if rs:
            orc.restate(cfg, st, 77, k, 0.3)
        got_tau = run.attrs["opacity"].cpu().numpy().ravel()
        assert int(na.item()) == orc.active_rows(got_tau).size
    got = run.rows()
    moved = np.abs(got[:, 0:3] - synth.to_rows(groups)[:, 0:3]).max()
    assert moved > 1e-3                               # the noise is far above FP32 rounding
    tol = 1e-5 if prec == "FP32" else 2e-3
    assert_close(got, st.theta, tol, what=f"noise mode {mode}")
    run.close()


@pytest.mark.parametrize("prec", ["FP32", "FP16_BLOCK"])
@pytest.mark.parametrize("n", [1, 255, 257, 513, 1537])
def test_terms_form_edge_sizes(G, orc, prec, n):
    """The terms form (active count and noise on visible rows, RSR on one
    step) at sizes around the 256-row tiles, with all-visible, none-visible
    and random masks: rows against the oracle, the count against the
    classification of the GPU's own logits, step counters exact."""
    groups = _noisy_scene(n, 1960 + n)
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    st = orc.State(synth.to_rows(groups))
    cfg = orc.Config(n_i=orc.dar_normaliser(800 * 800))
    rng = np.random.default_rng(1961 + n)
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    masks = [np.ones(n, np.uint8), np.zeros(n, np.uint8)] + [(rng.random(n) < 0.4).astype(np.uint8) for _ in range(4)]
    for k, mask in enumerate(masks, start=1):
        g = synth.grads_rows(n, 1962 + n, k)
        lr = synth.lr_for_step(k, len(masks))
        o, ext = _ext(G, orc, noise=1, noise_lr=400.0, noise_k=3.0, noise_t=0.5)
        ext.seed = 78
        rs = k == 3
        run.set_grads(g)
        na.zero_()
        run.step_mask(torch.from_numpy(mask).cuda(),
                      G.make_params(lr, k, restate=rs, restate_ratio=0.5, seed=78, n_active=na, **o))
        orc.step_ext(cfg, st, g, mask, lr, True, True, k, ext)
        if rs:
            orc.restate(cfg, st, 78, k, 0.5)
        got_tau = run.attrs["opacity"].cpu().numpy().ravel()
        assert int(na.item()) == orc.active_rows(got_tau).size
    tol = 1e-5 if prec == "FP32" else 2e-3
    assert_close(run.rows(), st.theta, tol, what=f"terms form, {n} rows")
    _, _, t = run.state()
    assert np.array_equal(t, st.t)
    run.close()


def test_noise_only_rows_move_by_the_noise_term(G, orc):
    """First step, g = 0, DAR off: the Adam direction is 0 and the position
    change is exactly the noise term (visible and, in mode 2, invisible)."""
    n = 5_003
    groups = _noisy_scene(n, 1920)
    run = GpuScene(groups)
    mask = (np.arange(n) % 2).astype(np.uint8)
    o, ext = _ext(G, orc, noise=2, noise_lr=100.0, noise_k=3.0, noise_t=0.5)
    run.step_mask(torch.from_numpy(mask).cuda(), G.make_params(LR, 1, dar_opacity=False, dar_scale=False, seed=3,
                                                               **o))
    got = run.rows()
    rows = synth.to_rows(groups).astype(np.float64)
    for i in range(0, n, 97):
        d = orc.noise_term(rows[i], 100.0, LR[0], 3.0, 0.5, orc.gauss3(3, 1, i))
        np.testing.assert_allclose(got[i, 0:3], rows[i, 0:3] - d, rtol=0, atol=2e-6 * (1 + np.abs(d).max()))
    run.close()


@pytest.mark.parametrize("prec", ["FP32", "BF16_HYBRID", "FP16_BLOCK"])
@pytest.mark.parametrize("bias_mode", [0, 1])
def test_aiu_matches_oracle(G, orc, prec, bias_mode):
    n = 25_013
    groups = synth.scene_uniform(n, 1930)
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec), bias_mode=bias_mode)
    st = orc.State(synth.to_rows(groups))
    cfg = orc.Config(n_i=orc.dar_normaliser(800 * 800), bias_mode=bias_mode)
    rng = np.random.default_rng(1931)
    for k in range(1, 11):
        g = synth.grads_rows(n, 1932, k)
        mask = (rng.random(n) < 0.3).astype(np.uint8)
        lr = synth.lr_for_step(k, 10)
        on = k >= 3
        o, ext = _ext(G, orc, aiu=on, aiu_prob=0.35, aiu_scale=0.5)
        ext.seed = 11
        rs = k in (5, 8)
        run.set_grads(g)
        run.step_mask(torch.from_numpy(mask).cuda(),
                      G.make_params(lr, k, restate=rs, restate_ratio=0.5, seed=11, **o))
        orc.step_ext(cfg, st, g, mask, lr, True, True, k, ext)
        if rs:
            orc.restate(cfg, st, 11, k, 0.5)
    got = run.rows()
    m, v, t = run.state()
    assert np.array_equal(t, st.t)
    if prec == "FP32":
        assert_close(got, st.theta, 1e-5, what="AIU")
        assert_close(m, st.m, 1e-5, what="m")
        assert_close(v, st.v, 1e-5, what="v")
    else:
        assert_close(got, st.theta, 2e-3, what="AIU hybrid")
    run.close()


def test_active_count_all_paths(G, orc):
    """Noise on every row, AIU and RSR together: the count comes from phase A
    (untouched and noise-only rows) and from the row items (visible and AIU
    rows); it must equal the classification of the GPU's own logits."""
    n = 40_009
    groups = _noisy_scene(n, 1940)
    run = GpuScene(groups)
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    rng = np.random.default_rng(1941)
    for k in range(1, 7):
        run.set_grads(synth.grads_rows(n, 1942, k))
        mask = torch.from_numpy((rng.random(n) < 0.3).astype(np.uint8)).cuda()
        na.zero_()
        run.step_mask(mask, G.make_params(LR, k, restate=(k % 2 == 0), restate_ratio=0.3, seed=9, noise=2,
                                          noise_lr=10.0, noise_k=3.0, noise_t=0.5, aiu=k > 1, aiu_prob=0.5,
                                          aiu_scale=1.0, n_active=na))
        tau = run.attrs["opacity"].cpu().numpy().ravel()
        want = orc.active_rows(tau).size
        assert int(na.item()) == want
        assert 0 < want < n
    run.close()


@pytest.mark.parametrize("n", [0, 1, 1023, 1024, 1025, 4095, 4096, 4097, 300_001, 2_000_003])
def test_active_rows_matches_oracle(G, orc, n):
    rng = np.random.default_rng(1950 + n)
    tau = rng.normal(-5.5, 1.0, n).astype(np.float32)
    if n >= 100:     # the FP32 neighbours of -ln 254
        t0 = np.float32(-np.log(254.0))
        near = [t0]
        for _ in range(20):
            near.append(np.nextafter(near[-1], np.float32(np.inf)))
            near.insert(0, np.nextafter(near[0], np.float32(-np.inf)))
        tau[:len(near)] = np.array(near, np.float32)
    h = G.gs_opt_init(G.make_config(), n)
    t_dev = torch.from_numpy(tau).cuda() if n else torch.zeros(1, device="cuda")
    rows = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -5, dtype=torch.int64, device="cuda")
    G.gs_active_rows(h, t_dev if n else None, rows if n else None, cnt)
    torch.cuda.synchronize()
    want = orc.active_rows(tau)
    assert int(cnt.item()) == want.size
    assert np.array_equal(rows.cpu().numpy()[:want.size], want)
    if n:
        cnt2 = torch.zeros(1, dtype=torch.int64, device="cuda")
        G.gs_active_rows(h, t_dev, None, cnt2)               # count only
        torch.cuda.synchronize()
        assert int(cnt2.item()) == want.size
        # repeated calls on one context (each call a new epoch of the scan's
        # status words), with different data in between
        for rep in range(3):
            tau2 = rng.normal(-5.5 + rep, 1.5, n).astype(np.float32)
            t2 = torch.from_numpy(tau2).cuda()
            rows.fill_(-1)
            G.gs_active_rows(h, t2, rows, cnt)
            torch.cuda.synchronize()
            want2 = orc.active_rows(tau2)
            assert int(cnt.item()) == want2.size
            assert np.array_equal(rows.cpu().numpy()[:want2.size], want2)
        assert G.gs_opt_sync_errors(h) == G.GS_OK
    G.gs_opt_destroy(h)


def test_prune_dead_rows_through_reindex(G, orc):
    """The active list is the source list of a prune: re-index the state and
    gather the attributes with it, then compare with the oracle."""
    n = 50_021
    groups = _noisy_scene(n, 1960)
    run = GpuScene(groups)
    run.set_grads(synth.grads_rows(n, 1961))
    run.step_mask(torch.ones(n, dtype=torch.uint8, device="cuda"), G.make_params(LR, 1))
    m0, v0, t0 = run.state()
    rows = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.gs_active_rows(run.h, run.attrs["opacity"], rows, cnt)
    torch.cuda.synchronize()
    keep = int(cnt.item())
    before = run.rows()
    want = orc.active_rows(before[:, 10].astype(np.float32))
    assert keep == want.size and 0 < keep < n
    src = rows[:keep].clone()
    G.gs_reindex_state(run.h, src, None, keep)
    out = {k: torch.empty((keep, v.shape[1]), device="cuda") for k, v in run.attrs.items()}
    G.gs_gather_attrs(run.h, G.make_attrs(run.attrs), n, G.make_attrs(out), src, keep)
    run.attrs = out
    run.n = keep
    assert G.gs_opt_rows(run.h) == keep
    after = run.rows()
    assert np.array_equal(after, before[want])
    m1, v1, t1 = run.state()
    ref = orc.reindex(orc.State(np.zeros((n, 59)), m0, v0, t0), want)
    assert np.array_equal(m1.astype(np.float64), ref.m) and np.array_equal(t1, ref.t)
    assert G.gs_opt_sync_errors(run.h) == 0
    run.close()


def test_batch_rejects_extended_terms(G):
    a = GpuScene(synth.scene_uniform(100, 1970))
    b = G.gs_batch_create([a.h])
    for kw in (dict(noise=1), dict(aiu=True, aiu_prob=0.1),
               dict(n_active=torch.zeros(1, dtype=torch.int64, device="cuda"))):
        b.set(0, G.make_attrs(a.attrs), G.make_attrs(a.grads), G.make_camera(synth.ring_cameras(4)[0]),
              G.make_params(LR, 1, **kw))
        with pytest.raises(G.GsError) as e:
            G.gs_batch_step(b)
        assert e.value.status == G.GS_ERR_UNSUPPORTED
    b.close()
    a.close()


def test_extended_params_validated(G):
    a = GpuScene(synth.scene_uniform(10, 1980))
    bad = [dict(noise=3), dict(noise=1, noise_lr=float("nan")), dict(aiu=True, aiu_prob=1.5),
           dict(aiu=True, aiu_prob=0.5, aiu_scale=float("inf"))]
    for kw in bad:
        with pytest.raises(G.GsError) as e:
            a.step_mask(torch.ones(10, dtype=torch.uint8, device="cuda"), G.make_params(LR, 1, **kw))
        assert e.value.status == G.GS_ERR_INVALID_ARG
    with pytest.raises(G.GsError):
        a.step_mask(torch.ones(10, dtype=torch.uint8, device="cuda"), G.make_params(LR, 1 << 30))
    a.close()
