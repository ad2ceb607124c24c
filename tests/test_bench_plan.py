"""Host-side arithmetic of bench.py (no GPU): the steps a run indexes stay
inside the scene it builds, and the timed window always holds an RSR step
(Eq. meth::restate, every 100 iterations), whatever --steps and --warmup."""
import importlib.util
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("steps,warmup,e2e", [(20, 5, None), (1, 3, None), (3, 3, 50), (99, 3, None),
                                              (100, 10, None), (1000, 10, 50), (7, 250, 0)])
def test_timed_window_holds_an_rsr_step(bench, steps, warmup, e2e):
    every = 100
    e2e_steps = steps if e2e is None else e2e
    k0, n = bench.headline_plan(warmup, steps, e2e_steps, every)
    assert 0 <= k0 < every
    timed = [k0 + i + 1 for i in range(warmup, warmup + steps)]       # iteration of each timed step
    assert any(k % every == 0 for k in timed)
    # every step index the device-timed run and the end-to-end leg touch exists
    assert warmup + steps <= n
    assert 3 + e2e_steps <= n


def test_driver_command_plan(bench):
    """--steps 20 --warmup 5: iterations 91-110 are timed, RSR at 100."""
    k0, n = bench.headline_plan(5, 20, 20, 100)
    assert (k0 + 6, k0 + 25) == (91, 110)
    assert n == 25


def test_camera_order_index_wraps(bench):
    from paper_2601_16736_gb300 import synth
    wl = synth.WORKLOADS["c2_1m"]
    order = synth.view_order(len(wl.cameras()), 25, wl.seed)
    k0, _ = bench.headline_plan(5, 20, 20, 100)
    # Scene.cam(i) indexes order[(k - 1) % len(order)]; k goes past len(order) here
    assert all(0 <= (k0 + i) % len(order) < len(order) for i in range(25))
    assert len(order) >= 25


def test_launch_bytes_per_row():
    """Algorithmic bytes of a launch from the per-row counts: a visible FP32
    row reads attributes, gradients, m, v (4 x 236 B) and writes attributes,
    m, v (3 x 236 B), and reads and writes its 4-B step counter; its 12-B
    mean is counted once, with every row's frustum test.  An invisible
    StSS-sampled row has its m and v read and written."""
    import bench
    assert bench.launch_bytes("fp32", 1, 1, 0) == 7 * 236 + 8
    assert bench.launch_bytes("fp32", 1_000_000, 0, 0) == 12_000_000
    assert bench.launch_bytes("fp32", 10, 3, 2) == 3 * 1648 + 10 * 12 + 2 * 4 * 236
    # FP16 block: 2 x 126 B of moments and a 2-B counter per moment row, read and written
    assert bench.bytes_visible("fp16_block") == 3 * 236 + 4 * 126 + 4 - 12
    assert bench.launch_bytes("fp16_block", 1_000_000, 268_093, 0) == 334_783_972
    assert bench.launch_bytes("fp32", 1_000_000, 268_093, 0) == 453_817_264
