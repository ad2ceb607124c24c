"""Pins of the oracle's Re-State Regularization (Eq. meth::restate), its
StSS sampler (SplitMix64, Steele et al. 2014) and the state re-index across
densify / prune / relocate (App. 'Scaling in RSR' item 1)."""
import json
from pathlib import Path

import numpy as np

from paper_2601_16736_gb300 import synth

NCOL = 59
GOLD = Path(__file__).parent / "golden"


def test_splitmix64_published_vector(orc):
    expect = [int(x) for x in (GOLD / "splitmix64_seed1234567.txt").read_text().split()
              if not x.startswith("#") and x.strip().isdigit()]
    assert len(expect) == 5
    assert [orc.splitmix64_at(1234567, c) for c in range(5)] == expect


def test_paper_rsr_defaults():
    h = json.loads((GOLD / "paper_hyperparameters.json").read_text())
    a1, a2 = h["alpha1"]["value"], h["alpha2"]["value"]
    assert 0 <= a1 < 1 and 0 <= a2 < 1          # Eq. meth::restate bounds
    assert abs(a2 - a1 * a1) < 1e-15           # App. 'Scaling in RSR' item (2)


def _state(orc, n, seed):
    rng = np.random.default_rng(seed)
    return orc.State(synth.to_rows(synth.scene_uniform(n, seed)), rng.normal(size=(n, NCOL)),
                     rng.random((n, NCOL)), rng.integers(0, 50, n))


def test_restate_scales_sampled_rows_only(orc):
    n = 4000
    st = _state(orc, n, 71)
    before = st.copy()
    cfg = orc.Config(alpha1=0.2, alpha2=0.04)
    cnt = orc.restate(cfg, st, seed=99, k=300, ratio=0.25)
    sampled = orc.stss_sampled(99, 300, range(n), 0.25).astype(bool)
    assert cnt == sampled.sum()
    # binomial(4000, 0.25): mean 1000, sd ~27
    assert abs(cnt - 1000) < 6 * 27.4
    np.testing.assert_array_equal(st.m[sampled], 0.2 * before.m[sampled])
    np.testing.assert_array_equal(st.v[sampled], 0.04 * before.v[sampled])
    assert st.m[~sampled].tobytes() == before.m[~sampled].tobytes()
    assert st.v[~sampled].tobytes() == before.v[~sampled].tobytes()
    assert st.t.tobytes() == before.t.tobytes() and st.theta.tobytes() == before.theta.tobytes()


def test_restate_ratio_limits_and_row_ids(orc):
    n = 500
    cfg = orc.Config()
    st = _state(orc, n, 72)
    assert orc.restate(cfg, st, 5, 100, 0.0) == 0
    assert orc.restate(cfg, st, 5, 100, 1.0) == n
    # a subset of rows with their global ids draws exactly what the full set draws
    full = _state(orc, n, 73)
    ids = np.arange(100, 160)
    sub = orc.State(full.theta[ids], full.m[ids], full.v[ids], full.t[ids])
    orc.restate(cfg, full, 6, 200, 0.3)
    orc.restate(cfg, sub, 6, 200, 0.3, row_ids=ids)
    assert sub.m.tobytes() == full.m[ids].tobytes()


def test_stss_draws_are_uniform_and_independent(orc):
    """Different sampling events pick (nearly) independent subsets."""
    n = 20000
    a = orc.stss_sampled(1, 100, range(n), 0.5).astype(bool)
    b = orc.stss_sampled(1, 200, range(n), 0.5).astype(bool)
    assert abs(a.mean() - 0.5) < 0.02 and abs(b.mean() - 0.5) < 0.02
    assert abs((a & b).mean() - 0.25) < 0.02


def test_restate_with_zero_alpha_is_reset(orc):
    """App. 'Scaling in RSR' (1): new / reallocated primitives are an RSR
    with alpha1 = alpha2 = 0 -- moments zero, exactly as a re-index reset."""
    n = 300
    st = _state(orc, n, 74)
    orc.restate(orc.Config(alpha1=0.0, alpha2=0.0), st, 3, 100, 1.0)
    src = np.arange(n, dtype=np.int32)
    re = orc.reindex(_state(orc, n, 74), src, np.ones(n, np.uint8))
    # equal as values (0 * negative m is -0.0, a reset writes +0.0)
    assert np.array_equal(st.m, re.m) and np.array_equal(st.v, re.v)
    assert np.all(st.m == 0)


def test_reindex_identity_and_inverse(orc):
    n = 1000
    st = _state(orc, n, 75)
    ident = orc.reindex(st, np.arange(n, dtype=np.int32))
    assert ident.m.tobytes() == st.m.tobytes() and ident.t.tobytes() == st.t.tobytes()
    perm = np.random.default_rng(76).permutation(n).astype(np.int32)
    fwd = orc.reindex(st, perm)
    inv = np.empty(n, np.int32)
    inv[perm] = np.arange(n, dtype=np.int32)
    back = orc.reindex(fwd, inv)
    assert back.m.tobytes() == st.m.tobytes() and back.v.tobytes() == st.v.tobytes()
    assert back.t.tobytes() == st.t.tobytes()


def test_reindex_event_semantics(orc):
    n = 2000
    st = _state(orc, n, 77)
    src, reset, attr_src = synth.reindex_event(n, 78, 0)
    out = orc.reindex(st, src, reset)
    assert out.n == src.size == n          # prune 5 % and clone 5 % keep the count
    fresh = (src < 0) | (reset != 0)
    assert np.all(out.m[fresh] == 0) and np.all(out.v[fresh] == 0) and np.all(out.t[fresh] == 0)
    kept = ~fresh
    np.testing.assert_array_equal(out.m[kept], st.m[src[kept]])
    np.testing.assert_array_equal(out.t[kept], st.t[src[kept]])
    assert fresh.sum() == int(round(0.05 * n)) + int(round(0.02 * n))


def test_reindex_rejects_out_of_range(orc):
    import pytest
    st = _state(orc, 10, 79)
    with pytest.raises(IndexError):
        orc.reindex(st, np.array([0, 10], np.int32))
