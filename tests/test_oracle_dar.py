"""Pins of the oracle's Decoupled Attribute Regularization (Sec. 3.3,
Eq. disentangled_adam; App. Eqs. disentangled_opacity / disentangled_scaling)
and of the ablation regularisers (Eqs. meth::undisentangled_mom,
disentangled_adam2, disentangled_adamwithcliping).

Expected values are hand-derived closed forms: from zero state the first
step has m^ = g and sqrt(v^) = |g|, the logistic derivative at 0 is exactly
1/4, exp(0) = 1, and the paper's constants are lambda_o = 1e-3,
lambda_s = 1e-5, C_t = 10, N_I = 60000 for an 800 x 800 image.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

NCOL = 59
TAU, KAPPA0 = 10, 3
LR = np.array([1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4])
GOLD = json.loads((Path(__file__).parent / "golden" / "paper_hyperparameters.json").read_text())


def _cfg(orc, **kw):
    base = dict(lambda_o=GOLD["lambda_o"]["value"], lambda_s=GOLD["lambda_s"]["value"],
                clip_o=GOLD["clip_o"]["value"], clip_s=GOLD["clip_s"]["value"], n_i=60000.0, eps=1e-15)
    base.update(kw)
    return orc.Config(**base)


def _one_row(theta_vals: dict, grad_vals: dict):
    th = np.zeros((1, NCOL))
    g = np.zeros((1, NCOL), np.float32)
    for c, x in theta_vals.items():
        th[0, c] = x
    for c, x in grad_vals.items():
        g[0, c] = x
    return th, g


@pytest.mark.parametrize("g, expect_dar", [
    (2.0 ** -30, 1e-3 * 0.25 / 60000.0 / (2.0 ** -30 + 1e-15)),   # active, unclipped (~4.47)
    (-(2.0 ** -30), 1e-3 * 0.25 / 60000.0 / (2.0 ** -30 + 1e-15)),
    (2.0 ** -34, 10.0),                                            # ~71.6 -> clipped at C_t
])
def test_opacity_first_step(orc, g, expect_dar):
    th, gr = _one_row({TAU: 0.0}, {TAU: g})
    st = orc.State(th)
    orc.step(_cfg(orc), st, gr, None, LR, True, False, 1)
    adam = g / (abs(g) + 1e-15)
    assert st.theta[0, TAU] == pytest.approx(0.0 - 2.5e-2 * (adam + expect_dar), rel=1e-13)
    # with DAR off the same step is plain Adam
    st2 = orc.State(th)
    orc.step(_cfg(orc), st2, gr, None, LR, False, False, 1)
    assert st2.theta[0, TAU] == pytest.approx(-2.5e-2 * adam, rel=1e-13)


@pytest.mark.parametrize("g, expect_dar", [
    (2.0 ** -34, 1e-5 * 1.0 / 60000.0 / (2.0 ** -34 + 1e-15)),    # ~2.86, unclipped
    (2.0 ** -37, 10.0),                                            # ~22.9 -> clipped
])
def test_scale_first_step(orc, g, expect_dar):
    th, gr = _one_row({KAPPA0: 0.0, KAPPA0 + 1: 0.0, KAPPA0 + 2: 0.0}, {KAPPA0: g, KAPPA0 + 1: g, KAPPA0 + 2: -g})
    st = orc.State(th)
    orc.step(_cfg(orc), st, gr, None, LR, False, True, 1)
    adam = g / (abs(g) + 1e-15)
    for c, s in [(KAPPA0, 1), (KAPPA0 + 1, 1), (KAPPA0 + 2, -1)]:
        assert st.theta[0, c] == pytest.approx(-5e-3 * (s * adam + expect_dar), rel=1e-13)


def test_clip_regime_closed_form(orc):
    """Zero gradients and zero state: v^ = 0, d = eps, so the DAR term is
    min(huge, C) = C every step and theta_k = theta_0 - k lr C."""
    k = 9
    th, gr = _one_row({TAU: 0.7, KAPPA0: -4.0, KAPPA0 + 1: -3.0, KAPPA0 + 2: -5.0, 0: 1.0, 20: 0.3}, {})
    st = orc.State(th)
    for kk in range(1, k + 1):
        orc.step(_cfg(orc), st, gr, None, LR, True, True, kk)
    assert st.theta[0, TAU] == pytest.approx(0.7 - k * 2.5e-2 * 10.0, rel=1e-13)
    for c, x0 in [(KAPPA0, -4.0), (KAPPA0 + 1, -3.0), (KAPPA0 + 2, -5.0)]:
        assert st.theta[0, c] == pytest.approx(x0 - k * 5e-3 * 10.0, rel=1e-13)
    # attributes without a regulariser do not move (u = 0 / eps = 0)
    assert st.theta[0, 0] == 1.0 and st.theta[0, 20] == 0.3


def test_unclipped_tail_uses_logistic_derivative(orc):
    """Far in the tail (tau = 20) the zero-state DAR term is below C:
    lambda_o sig'(tau) / (N_I eps), with sig'(tau) = 1 / (4 cosh^2(tau/2))."""
    tau0 = 20.0
    th, gr = _one_row({TAU: tau0}, {})
    st = orc.State(th)
    orc.step(_cfg(orc), st, gr, None, LR, True, False, 1)
    dsig = 1.0 / (4.0 * math.cosh(tau0 / 2.0) ** 2)
    term = 1e-3 * dsig / 60000.0 / 1e-15
    assert term < 10.0
    assert st.theta[0, TAU] == pytest.approx(tau0 - 2.5e-2 * term, rel=1e-12)


def test_regularizer_sees_pre_update_theta_and_post_update_v(orc):
    """Second step from a known state: the DAR term uses the v^ of this step
    (after the moment update) and the opacity before this step's update."""
    tau0, m0, v0, g = 1.5, 2e-9, 1e-17, 4e-9
    th, gr = _one_row({TAU: tau0}, {TAU: g})
    m = np.zeros((1, NCOL)); m[0, TAU] = m0
    v = np.zeros((1, NCOL)); v[0, TAU] = v0
    st = orc.State(th, m, v, np.array([1]))
    orc.step(_cfg(orc), st, gr, None, LR, True, False, 2)
    g32 = float(np.float32(g))
    m1 = 0.9 * m0 + 0.1 * g32
    v1 = 0.999 * v0 + 0.001 * g32 * g32
    d = math.sqrt(v1 / (1 - 0.999 ** 2)) + 1e-15
    s = 1.0 / (1.0 + math.exp(-tau0))
    expect = tau0 - 2.5e-2 * (m1 / (1 - 0.81) / d + min(1e-3 * s * (1 - s) / 60000.0 / d, 10.0))
    assert st.theta[0, TAU] == pytest.approx(expect, rel=1e-12)


def test_adamw_style_variants(orc):
    """Eq. disentangled_adam2 adds lambda grad R unpreconditioned; Eq.
    disentangled_adamwithcliping clips it at C_t.  At tau = 0, grad R = 1/4."""
    th, gr = _one_row({TAU: 0.0}, {TAU: 1e-3})
    g32 = float(np.float32(1e-3))
    adam = g32 / (g32 + 1e-15)
    st = orc.State(th)
    orc.step(_cfg(orc, reg_mode=2, lambda_o=1e-3), st, gr, None, LR, True, False, 1)
    assert st.theta[0, TAU] == pytest.approx(-2.5e-2 * (adam + 1e-3 * 0.25), rel=1e-12)
    st = orc.State(th)
    orc.step(_cfg(orc, reg_mode=3, lambda_o=100.0), st, gr, None, LR, True, False, 1)
    assert st.theta[0, TAU] == pytest.approx(-2.5e-2 * (adam + 10.0), rel=1e-12)


def test_coupled_variant_enters_moments(orc):
    """Eq. meth::undisentangled_mom: the regulariser gradient lambda grad R / N_v
    joins the photometric gradient inside the moments; first step from zero
    state is then lr * sign(g + lambda grad R / N_v)."""
    n_v = 1000
    for g in (1e-9, -1e-9):
        th, gr = _one_row({TAU: 0.0}, {TAU: g})
        st = orc.State(th)
        orc.step(_cfg(orc, reg_mode=1), st, gr, None, LR, True, False, 1, n_visible=n_v)
        geff = float(np.float32(g)) + 1e-3 * 0.25 / n_v
        assert st.theta[0, TAU] == pytest.approx(-2.5e-2 * geff / (abs(geff) + 1e-15), rel=1e-12)
        assert st.m[0, TAU] == pytest.approx(0.1 * geff, rel=1e-12)


def test_n_i_rule(orc):
    """App. 'DAR': keep the most significant digit of N_I, then divide by ten."""
    assert orc.dar_normaliser(800 * 800) == 60000.0        # 640000 -> 600000 -> 60000
    assert orc.dar_normaliser(1920 * 1080) == 200000.0     # 2073600 -> 2000000 -> 200000
    assert orc.dar_normaliser(1000) == 100.0
    assert orc.dar_normaliser(999) == 90.0
    assert orc.dar_normaliser(7) == 0.7
