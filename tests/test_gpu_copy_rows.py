"""gs_copy_rows: the step's memory traffic without the update leaves every
attribute, gradient and moment bit-identical, for every moment format, and
reports an out-of-range row through the context's error word."""
import numpy as np
import pytest

from harness import GpuScene
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


def _snapshot(run):
    torch.cuda.synchronize()
    a = {k: v.clone() for k, v in run.attrs.items()}
    g = {k: v.clone() for k, v in run.grads.items()}
    return a, g, run.state()


def _same(run, snap):
    a, g, (m, v, t) = snap
    for k in a:
        assert torch.equal(run.attrs[k].view(torch.int32), a[k].view(torch.int32)), k
        assert torch.equal(run.grads[k].view(torch.int32), g[k].view(torch.int32)), k
    m2, v2, t2 = run.state()
    assert np.array_equal(m2.view(np.uint32), m.view(np.uint32))
    assert np.array_equal(v2.view(np.uint32), v.view(np.uint32))
    assert np.array_equal(t2, t)


@pytest.mark.parametrize("prec", ["FP32", "BF16", "BF16_HYBRID", "FP16_BLOCK", "FP8E4M3"])
def test_copy_rows_changes_nothing(G, prec):
    n = 60_007
    groups = synth.scene_blobs(n, 131, 12.5)
    run = GpuScene(groups, prec=getattr(G, "GS_MOM_" + prec))
    run.set_grads(synth.grads_rows(n, 132))
    cams = synth.ring_cameras(6)
    for k in range(1, 4):
        run.step_camera(cams[k], G.make_params(synth.lr_for_step(k, 10), k))
    rows = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.gs_visibility(run.h, run.attrs["xyz"], G.make_camera(cams[4]), run.mask, rows, cnt)
    torch.cuda.synchronize()
    nv = int(cnt.item())
    assert 0 < nv < n
    snap = _snapshot(run)
    A, GR = G.make_attrs(run.attrs), G.make_attrs(run.grads)
    G.gs_copy_rows(run.h, A, GR, rows, nv)
    G.gs_copy_rows(run.h, A, GR, rows, 0)
    all_rows = torch.arange(n, dtype=torch.int32, device="cuda")
    G.gs_copy_rows(run.h, A, GR, all_rows, n)
    assert G.gs_opt_sync_errors(run.h) == G.GS_OK
    _same(run, snap)
    run.close()


def test_copy_rows_out_of_range_is_recorded(G):
    n = 10_000
    run = GpuScene(synth.scene_uniform(n, 133))
    run.set_grads(synth.grads_rows(n, 134))
    snap = _snapshot(run)
    rows = torch.tensor([0, 5, n, 7, -1, n - 1], dtype=torch.int32, device="cuda")
    G.gs_copy_rows(run.h, G.make_attrs(run.attrs), G.make_attrs(run.grads), rows, rows.numel())
    assert G.gs_opt_sync_errors(run.h) == G.GS_ERR_INVALID_ARG
    _same(run, snap)
    with pytest.raises(G.GsError):
        G.gs_copy_rows(run.h, G.make_attrs(run.attrs), G.make_attrs(run.grads), rows, n + 1)
    run.close()
