"""Pins of the oracle's position noise (App. Eq. disentangled_mu), AIU
(Sec. 3.2) and active/dead classification (Sec. 4, opacity > 1/255), each
against something other than the oracle itself: a distribution test, a
library rotation, closed forms, and high-precision arithmetic."""
import numpy as np
import pytest

from paper_2601_16736_gb300 import synth

scipy_stats = pytest.importorskip("scipy.stats")
Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


# ------------------------------------------------------------------ gamma

def test_gauss3_is_standard_normal(orc):
    g = np.array([orc.gauss3(77, 5, r) for r in range(60_000)])
    for j in range(3):
        assert abs(g[:, j].mean()) < 0.02
        assert abs(g[:, j].var() - 1.0) < 0.03
        assert scipy_stats.kstest(g[:, j], "norm").pvalue > 1e-3
    c = np.corrcoef(g.T)
    assert np.all(np.abs(c - np.eye(3)) < 0.02)
    # another iteration is a fresh draw
    h = np.array([orc.gauss3(77, 6, r) for r in range(20_000)])
    assert abs(np.corrcoef(g[:20_000, 0], h[:, 0])[0, 1]) < 0.03
    assert np.all(np.abs(g) < 5.8)            # 24-bit uniforms: |gamma| <= sqrt(-2 ln 2^-24)


def test_gauss3_is_a_function_of_seed_iteration_row(orc):
    a = orc.gauss3(123, 9, 4567)
    assert np.array_equal(a, orc.gauss3(123, 9, 4567))
    assert not np.array_equal(a, orc.gauss3(124, 9, 4567))
    assert not np.array_equal(a, orc.gauss3(123, 9, 4568))


# ------------------------------------------------------------- covariance

def test_covariance_matches_library_rotation(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        q = rng.normal(size=4) * rng.uniform(0.1, 5.0)
        kappa = rng.normal(-2.0, 1.0, size=3)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()       # scipy: (x, y, z, w)
        want = R @ np.diag(np.exp(2 * kappa)) @ R.T
        np.testing.assert_allclose(orc.covariance(q, kappa), want, rtol=1e-12, atol=1e-15)
        ev = np.sort(np.linalg.eigvalsh(orc.covariance(q, kappa)))
        np.testing.assert_allclose(ev, np.sort(np.exp(2 * kappa)), rtol=1e-10)


def test_covariance_special_cases(orc):
    k = np.log([2.0, 3.0, 5.0])
    np.testing.assert_allclose(orc.covariance([1, 0, 0, 0], k), np.diag([4.0, 9.0, 25.0]), atol=1e-14)
    # 90 degrees about z swaps the x and y variances
    c = np.cos(np.pi / 4)
    np.testing.assert_allclose(orc.covariance([c, 0, 0, c], k), np.diag([9.0, 4.0, 25.0]), atol=1e-12)
    # a zero quaternion normalises to zero: R = I
    np.testing.assert_allclose(orc.covariance([0, 0, 0, 0], k), np.diag([4.0, 9.0, 25.0]), atol=1e-14)


# ------------------------------------------------------------- noise term

def _row(tau, kappa, q):
    r = np.zeros(59)
    r[3:6] = kappa
    r[6:10] = q
    r[10] = tau
    return r


def test_noise_term_closed_forms(orc):
    gamma = np.array([0.3, -1.2, 2.0])
    lam_mu, lam_t = 100.0, 0.005
    # o = lambda_t: the gate is sigmoid(0) = 1/2; identity rotation, s = 1
    tau = np.log(lam_t / (1 - lam_t))
    out = orc.noise_term(_row(tau, [0, 0, 0], [1, 0, 0, 0]), 5e5, 1.6e-4, lam_mu, lam_t, gamma)
    np.testing.assert_allclose(out, 5e5 * 1.6e-4 * 0.5 * gamma, rtol=1e-12)
    # scales enter squared
    out = orc.noise_term(_row(tau, np.log([0.1, 0.2, 0.3]), [1, 0, 0, 0]), 2.0, 3.0, lam_mu, lam_t, gamma)
    np.testing.assert_allclose(out, 2.0 * 3.0 * 0.5 * np.array([0.01, 0.04, 0.09]) * gamma, rtol=1e-12)
    # an opaque primitive gets (almost) no noise: gate = 1/(1 + exp(100 (sigmoid(8) - 0.005)))
    o = 1 / (1 + np.exp(-8.0))
    gate = 1 / (1 + np.exp(lam_mu * (o - lam_t)))
    out = orc.noise_term(_row(8.0, [0, 0, 0], [1, 0, 0, 0]), 1.0, 1.0, lam_mu, lam_t, gamma)
    np.testing.assert_allclose(out, gate * gamma, rtol=1e-10)
    assert np.all(np.abs(out) < 1e-40)
    # rotated: Sigma gamma with the library rotation
    q = np.array([0.9, 0.1, -0.3, 0.2])
    kap = np.array([-1.0, -2.0, -0.5])
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    want = 4.0 * 0.5 * (R @ np.diag(np.exp(2 * kap)) @ R.T @ gamma)
    out = orc.noise_term(_row(tau, kap, q), 4.0, 1.0, lam_mu, lam_t, gamma)
    np.testing.assert_allclose(out, want, rtol=1e-11)


def test_step_ext_noise_moves_only_mu(orc):
    """g = 0, DAR off, first step: the Adam direction is 0/(0 + eps) = 0, so
    the visible rows move by exactly the noise term; noise_mode 1 leaves
    invisible rows alone, noise_mode 2 moves them too."""
    n = 400
    groups = synth.scene_uniform(n, 1800)
    rows = synth.to_rows(groups).astype(np.float64)
    rows[:, 10] = np.log(0.3 / 0.7)                 # o = 0.3
    mask = (np.arange(n) % 3 != 0).astype(np.uint8)
    lr = np.array([1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4])
    ext = orc.Ext(noise_mode=1, noise_lr=5e5, noise_k=2.0, noise_t=0.5, seed=99)
    for mode in (1, 2):
        ext.noise_mode = mode
        st = orc.State(rows)
        orc.step_ext(orc.Config(), st, np.zeros((n, 59), np.float32), mask, lr, False, False, 1, ext)
        for i in range(n):
            moved = mode == 2 or mask[i]
            want = rows[i, 0:3].copy()
            if moved:
                g = orc.gauss3(99, 1, i)
                R = Rotation.from_quat([rows[i, 7], rows[i, 8], rows[i, 9], rows[i, 6]]).as_matrix()
                sig = R @ np.diag(np.exp(2 * rows[i, 3:6])) @ R.T
                gate = 1 / (1 + np.exp(2.0 * (0.3 - 0.5)))
                want -= 5e5 * lr[0] * gate * sig @ g
            np.testing.assert_allclose(st.theta[i, 0:3], want, rtol=1e-12, atol=1e-15)
            np.testing.assert_array_equal(st.theta[i, 3:], rows[i, 3:])


# -------------------------------------------------------------------- AIU

def test_aiu_sampling_frequency_and_independence(orc):
    rows = np.arange(100_000)
    a = orc.aiu_sampled(3, 11, rows, 0.3).astype(bool)
    assert abs(a.mean() - 0.3) < 4 * np.sqrt(0.3 * 0.7 / rows.size)
    s = orc.stss_sampled(3, 11, rows, 0.5).astype(bool)     # same seed and k, other stream
    assert abs(np.corrcoef(a, s)[0, 1]) < 0.02
    assert orc.aiu_sampled(3, 11, rows[:1000], 0.0).sum() == 0
    assert orc.aiu_sampled(3, 11, rows[:1000], 1.0).sum() == 1000


def test_aiu_step_after_one_visible_step_is_sign(orc):
    """After one visible step from zero state with gradient g, m^ = g and
    v^ = g^2, so the AIU direction is g/(|g| + eps) = sign(g): a sampled
    invisible row moves by -lr * eta_AIU * sign(g), keeps m, v and t, and a
    row never seen (t = 0) does not move."""
    n = 300
    rows = synth.to_rows(synth.scene_uniform(n, 1801))
    g = synth.grads_rows(n, 1802)
    lr = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3])
    cfg = orc.Config(eps=1e-30)
    st = orc.State(rows)
    seen = (np.arange(n) % 4 != 0).astype(np.uint8)
    orc.step(cfg, st, g, seen, lr, False, False, 1)
    after1 = st.copy()
    ext = orc.Ext(aiu=True, aiu_prob=1.0, aiu_scale=0.5, seed=1)
    orc.step_ext(cfg, st, np.zeros((n, 59), np.float32), np.zeros(n, np.uint8), lr, False, False, 2, ext)
    for i in range(n):
        if seen[i]:
            want = after1.theta[i] - lr[orc.LR_GROUP] * 0.5 * np.sign(g[i].astype(np.float64))
            np.testing.assert_allclose(st.theta[i], want, rtol=1e-12, atol=1e-18)
        else:
            np.testing.assert_array_equal(st.theta[i], after1.theta[i])
    np.testing.assert_array_equal(st.m, after1.m)
    np.testing.assert_array_equal(st.v, after1.v)
    np.testing.assert_array_equal(st.t, after1.t)


def test_aiu_touches_only_sampled_invisible_rows(orc):
    n = 2000
    rows = synth.to_rows(synth.scene_uniform(n, 1803))
    lr = np.full(6, 1e-3)
    st = orc.State(rows)
    orc.step(orc.Config(), st, synth.grads_rows(n, 1804), None, lr, False, False, 1)
    before = st.copy()
    mask = (np.arange(n) % 2).astype(np.uint8)
    g2 = synth.grads_rows(n, 1805)
    ext = orc.Ext(aiu=True, aiu_prob=0.25, aiu_scale=1.0, seed=42)
    orc.step_ext(orc.Config(), st, g2, mask, lr, False, False, 2, ext)
    ref = before.copy()
    orc.step(orc.Config(), ref, g2, mask, lr, False, False, 2)
    sampled = orc.aiu_sampled(42, 2, np.arange(n), 0.25).astype(bool) & (mask == 0)
    assert 0.2 < sampled.sum() / (n / 2) < 0.3
    same = ~sampled
    np.testing.assert_array_equal(st.theta[same], ref.theta[same])     # visible rows: the plain step
    assert np.all(np.any(st.theta[sampled] != before.theta[sampled], axis=1))
    np.testing.assert_array_equal(st.m, ref.m)
    np.testing.assert_array_equal(st.t, ref.t)


# ------------------------------------------------------------ active rows

def test_active_threshold_is_exact(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    T = -mp.log(254)                                   # sigmoid(tau) > 1/255  <=>  tau > -ln 254
    t0 = np.float32(float(T))
    taus = [t0]
    for _ in range(40):
        taus.append(np.nextafter(taus[-1], np.float32(np.inf)))
    lo = [t0]
    for _ in range(40):
        lo.append(np.nextafter(lo[-1], np.float32(-np.inf)))
    taus = np.array(sorted(set(lo + taus)), np.float32)
    for tau in taus:
        exact = 1 / (1 + mp.exp(-mp.mpf(float(tau)))) > mp.mpf(1) / 255
        assert orc.is_active(float(tau)) == bool(exact), float(tau)
    assert orc.active_rows(taus).tolist() == [i for i, x in enumerate(taus) if mp.mpf(float(x)) > T]


def test_active_rows_ascending_and_counts(orc):
    rng = np.random.default_rng(7)
    tau = rng.normal(-5.0, 2.0, 100_000).astype(np.float32)
    rows = orc.active_rows(tau)
    assert np.all(np.diff(rows) > 0)
    assert np.array_equal(rows, np.nonzero(tau.astype(np.float64) > -np.log(254.0))[0])
    assert orc.active_rows(np.zeros(0, np.float32)).size == 0


def test_step_ext_returns_active_count(orc):
    n = 1000
    rows = synth.to_rows(synth.scene_uniform(n, 1806))
    rows[:, 10] = np.linspace(-8, -3, n)
    st = orc.State(rows)
    mask = (np.arange(n) % 2).astype(np.uint8)
    na = orc.step_ext(orc.Config(), st, synth.grads_rows(n, 1807), mask, np.full(6, 1e-2), True, True, 1,
                      orc.Ext())
    assert na == int((1 / (1 + np.exp(-st.theta[:, 10])) > 1 / 255).sum())
    assert 0 < na < n
