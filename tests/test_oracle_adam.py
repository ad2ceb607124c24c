"""Pins of the oracle's Sparse Adam core against things other than itself.

* dense case (all-true mask, no regulariser) = torch.optim.Adam in FP64
  (Eq. meth::first_grad / meth::adam_update with bias correction);
* each primitive's own trajectory under a random visibility sequence = a
  plain Adam run over only the steps where it was visible (per-primitive t,
  Sec. 3.2 "asynchronous indexing");
* global-t mode = torch.optim.SparseAdam (global step, skipped rows);
* all-false mask leaves everything bit-identical (Eq. meth::sparse_beta);
* closed forms: first step from zero state, zero-gradient decay.
"""
import numpy as np
import pytest
import torch

from paper_2601_16736_gb300 import synth

NCOL = 59
GROUP_COLS = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, 59)]


def _rows(n, seed):
    return synth.to_rows(synth.scene_uniform(n, seed)).astype(np.float64)


def _torch_adam_run(theta0, grads, lr, beta1, beta2, eps, visible_steps=None):
    """Reference: torch.optim.Adam, one parameter tensor per lr group."""
    params = [torch.tensor(theta0[:, sl], dtype=torch.float64, requires_grad=True) for sl in GROUP_COLS]
    opt = torch.optim.Adam([{"params": [p], "lr": float(l)} for p, l in zip(params, lr)],
                           betas=(beta1, beta2), eps=eps)
    for kk, g in enumerate(grads):
        if visible_steps is not None and not visible_steps[kk]:
            continue
        for p, sl in zip(params, GROUP_COLS):
            p.grad = torch.tensor(g[:, sl].astype(np.float64))
        opt.step()
    return np.concatenate([p.detach().numpy() for p in params], axis=1)


@pytest.mark.parametrize("eps", [1e-15, 1e-3])
def test_dense_equals_torch_adam(orc, eps):
    n, steps = 64, 25
    theta0 = _rows(n, 11)
    grads = [synth.grads_rows(n, 12, b) * (1.0 + b) for b in range(steps)]
    lr = np.array([1e-2, 2e-2, 3e-3, 5e-2, 7e-3, 1e-4])
    cfg = orc.Config(beta1=0.9, beta2=0.999, eps=eps)
    st = orc.State(theta0)
    for k, g in enumerate(grads, start=1):
        orc.step(cfg, st, g, None, lr, False, False, k)
    ref = _torch_adam_run(theta0, grads, lr, 0.9, 0.999, eps)
    np.testing.assert_allclose(st.theta, ref, rtol=1e-12, atol=1e-14)
    assert np.all(st.t == steps)


def test_sparse_is_adam_on_visible_subsequence(orc):
    """Sparse Adam with per-primitive t: every row evolves exactly like a
    dense Adam that only ever sees the steps on which the row was visible."""
    n, steps = 12, 30
    theta0 = _rows(n, 21)
    rng = np.random.default_rng(22)
    masks = (rng.random((steps, n)) < 0.4).astype(np.uint8)
    masks[:, 0] = 0                      # a row that is never visible
    masks[:, 1] = 1                      # a row that is always visible
    grads = [synth.grads_rows(n, 23, b) for b in range(steps)]
    lr = np.array([1e-2, 2e-2, 3e-3, 5e-2, 7e-3, 1e-4])
    cfg = orc.Config(beta1=0.8, beta2=0.99, eps=1e-6)
    st = orc.State(theta0)
    for k in range(steps):
        orc.step(cfg, st, grads[k], masks[k], lr, False, False, k + 1)
    for i in range(n):
        ref = _torch_adam_run(theta0[i:i + 1], [g[i:i + 1] for g in grads], lr, 0.8, 0.99, 1e-6,
                              visible_steps=masks[:, i])
        np.testing.assert_allclose(st.theta[i:i + 1], ref, rtol=1e-12, atol=1e-14)
        assert st.t[i] == masks[:, i].sum()
    np.testing.assert_array_equal(st.theta[0], theta0[0])


def test_global_t_mode_equals_torch_sparse_adam(orc):
    """bias_mode=1 (one global step count) with a visibility mask is what
    torch.optim.SparseAdam does with the visible rows as sparse indices.
    SparseAdam adds eps before the bias correction (eps / sqrt(1 - b2^k) in
    Adam's terms), so eps is negligible here: the test pins the masking and
    the global step count."""
    n, steps = 40, 20
    theta0 = _rows(n, 31)
    rng = np.random.default_rng(32)
    masks = (rng.random((steps, n)) < 0.5).astype(np.uint8)
    grads = [synth.grads_rows(n, 33, b) for b in range(steps)]
    lr = 3e-2
    cfg = orc.Config(beta1=0.9, beta2=0.999, eps=1e-30, bias_mode=1)
    st = orc.State(theta0)
    p = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.SparseAdam([p], lr=lr, betas=(0.9, 0.999), eps=1e-30)
    for k in range(steps):
        orc.step(cfg, st, grads[k], masks[k], np.full(6, lr), False, False, k + 1)
        idx = np.nonzero(masks[k])[0]
        vals = torch.tensor(grads[k][idx].astype(np.float64))
        p.grad = torch.sparse_coo_tensor(torch.tensor(idx)[None, :], vals, (n, NCOL),
                                         check_invariants=True)
        opt.step()
    np.testing.assert_allclose(st.theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_all_false_mask_is_bit_identical(orc):
    n = 50
    theta0 = _rows(n, 41)
    rng = np.random.default_rng(42)
    st = orc.State(theta0, rng.normal(size=(n, NCOL)), rng.random((n, NCOL)), rng.integers(0, 9, n))
    before = st.copy()
    cfg = orc.Config()
    orc.step(cfg, st, synth.grads_rows(n, 43), np.zeros(n, np.uint8), np.full(6, 0.1), True, True, 7)
    for a, b in [(st.theta, before.theta), (st.m, before.m), (st.v, before.v), (st.t, before.t)]:
        assert a.tobytes() == b.tobytes()


def test_first_step_closed_form(orc):
    """From zero state, m^ = g and v^ = g^2, so theta_1 = theta_0 - lr g/(|g|+eps)."""
    n = 200
    theta0 = _rows(n, 51)
    g = synth.grads_rows(n, 52)
    lr = np.array([1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4])
    cfg = orc.Config(eps=1e-15)
    st = orc.State(theta0)
    orc.step(cfg, st, g, None, lr, False, False, 1)
    gd = g.astype(np.float64)
    lr_col = np.concatenate([np.full(sl.stop - sl.start, l) for sl, l in zip(GROUP_COLS, lr)])
    expect = theta0 - lr_col * gd / (np.abs(gd) + 1e-15)
    np.testing.assert_allclose(st.theta, expect, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(st.m, 0.1 * gd, rtol=1e-13)
    np.testing.assert_allclose(st.v, 0.001 * gd * gd, rtol=1e-12)


def test_zero_gradient_decay_closed_form(orc):
    """k visible zero-gradient steps: m_k = b1^k m_0, v_k = b2^k v_0."""
    n, k = 30, 17
    rng = np.random.default_rng(61)
    m0 = rng.normal(size=(n, NCOL))
    v0 = rng.random((n, NCOL)) + 0.1
    st = orc.State(_rows(n, 62), m0, v0, np.zeros(n))
    cfg = orc.Config(beta1=0.85, beta2=0.995)
    zero = np.zeros((n, NCOL), np.float32)
    for kk in range(1, k + 1):
        orc.step(cfg, st, zero, None, np.full(6, 1e-3), False, False, kk)
    np.testing.assert_allclose(st.m, 0.85 ** k * m0, rtol=1e-13)
    np.testing.assert_allclose(st.v, 0.995 ** k * v0, rtol=1e-13)


def test_bias_denominators_closed_form(orc):
    d1 = orc.bias_denominators(0.9, 6)
    np.testing.assert_allclose(d1, [0.0, 0.1, 0.19, 0.271, 0.3439, 0.40951], rtol=1e-14, atol=1e-16)
    d2 = orc.bias_denominators(0.999, 3)
    np.testing.assert_allclose(d2, [0.0, 0.001, 0.001999], rtol=1e-12, atol=1e-18)
