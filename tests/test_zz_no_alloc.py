"""gs_step_host_noalloc: the host-gradient step for callers that cannot
allocate device memory when they step (a fixed device-memory budget committed
up front, latency-critical threads, runtimes that own the allocator).  It
stages the gradients in the library's fixed device array instead of a buffer
created on first use, and must give the same result as gs_step_host.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
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


@pytest.mark.parametrize("prec", ["FP32", "FP16_BLOCK", "FP8E4M3"])
def test_noalloc_step_matches_allocating_step(G, prec):
    """Both calls run the same step kernel on the same gradient values (the
    allocating one reads pinned memory in place, this one stages it), so
    attributes, moments and step counters must be bit-identical."""
    n = 50_001                       # ~195 tiles of 256 rows and a ragged tail
    groups = synth.scene_blobs(n, 880, 12.5)
    cams = synth.ring_cameras(8, (0.0, 30.0))
    p_enum = getattr(G, "GS_MOM_" + prec)
    ref, new = GpuScene(groups, prec=p_enum), GpuScene(groups, prec=p_enum)
    for call in range(2):            # two calls in a row: the array keeps the first call's contents
        k = call + 1
        grads = synth.grads_rows(n, 881, call)
        gh = {g: torch.from_numpy(v).pin_memory() for g, v in synth.from_rows(grads).items()}
        p = G.make_params(synth.lr_for_step(k, 10), k, restate=(call == 1), restate_ratio=0.5, seed=5)
        cam = G.make_camera(cams[3 * call])
        nv_ref = G.gs_step_host(ref.h, G.make_attrs(ref.attrs), G.make_attrs(gh), cam, p)
        nv_new = G.gs_step_host_noalloc(new.h, G.make_attrs(new.attrs), G.make_attrs(gh), cam, p)
        assert nv_new == nv_ref > 0
        assert new.rows().tobytes() == ref.rows().tobytes(), f"attributes after call {k}"
        m_r, v_r, t_r = ref.state()
        m_n, v_n, t_n = new.state()
        assert m_n.tobytes() == m_r.tobytes() and v_n.tobytes() == v_r.tobytes(), f"moments after call {k}"
        assert np.array_equal(t_n, t_r)
    ref.close()
    new.close()


def test_noalloc_rejects_more_rows_than_the_array_holds(G):
    n = G.GS_NOALLOC_MAX_ROWS + 1
    run = GpuScene(synth.scene_uniform(n, 882))
    gh = {g: torch.zeros(v.shape, dtype=torch.float32).pin_memory() for g, v in run.attrs.items()}
    with pytest.raises(G.GsError) as e:
        G.gs_step_host_noalloc(run.h, G.make_attrs(run.attrs), G.make_attrs(gh),
                               G.make_camera(synth.ring_cameras(4)[0]), G.make_params(np.ones(6) * 1e-3, 1))
    assert e.value.status == G.GS_ERR_INVALID_ARG
    run.close()
