"""Python binding of libgsopt.so: argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/gsopt.h for semantics, layouts and ownership) and does no arithmetic
of its own: tensors are passed as raw device pointers, the CUDA stream as its
handle (default: torch's current stream).  The library is loaded from this
package directory on first use; if it has not been built the call raises —
there is no fallback path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "libgsopt.so"
_lib = None

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_UNSUPPORTED, GS_ERR_TIMEOUT, GS_ERR_STATE = range(7)
GS_MOM_FP32, GS_MOM_BF16, GS_MOM_FP8E4M3, GS_MOM_BF16_HYBRID, GS_MOM_FP16_BLOCK = range(5)
GS_REG_DAR, GS_REG_COUPLED, GS_REG_ADAMW, GS_REG_ADAMW_CLIP = range(4)
GS_NOISE_OFF, GS_NOISE_VISIBLE, GS_NOISE_ALL = range(3)
GROUPS = (("xyz", 3), ("scale", 3), ("rot", 4), ("opacity", 1), ("sh", 48))
GS_NOALLOC_MAX_ROWS = 65536
GS_MAX_BATCH = 64


class GsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_name(status)}")


class gs_opt_config(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_float),
                ("lambda_o", ctypes.c_float), ("lambda_s", ctypes.c_float), ("clip_o", ctypes.c_float),
                ("clip_s", ctypes.c_float), ("alpha1", ctypes.c_float), ("alpha2", ctypes.c_float),
                ("prec", ctypes.c_int32), ("bias_mode", ctypes.c_int32), ("reg_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n_pixels", ctypes.c_int64)]


class gs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("tan_half_fovx", ctypes.c_float),
                ("tan_half_fovy", ctypes.c_float), ("znear", ctypes.c_float), ("zfar", ctypes.c_float)]


class gs_step_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 6), ("dar_opacity", ctypes.c_int32), ("dar_scale", ctypes.c_int32),
                ("restate", ctypes.c_int32), ("reserved", ctypes.c_int32), ("restate_ratio", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("iteration", ctypes.c_int64), ("n_visible", ctypes.c_int64),
                ("noise", ctypes.c_int32), ("aiu", ctypes.c_int32), ("noise_lr", ctypes.c_float),
                ("noise_k", ctypes.c_float), ("noise_t", ctypes.c_float), ("aiu_prob", ctypes.c_float),
                ("aiu_scale", ctypes.c_float), ("reserved2", ctypes.c_int32), ("n_active", ctypes.c_void_p)]


class gs_attrs(ctypes.Structure):
    _fields_ = [(g, ctypes.c_void_p) for g, _ in GROUPS]


gs_grads = gs_attrs   # same five pointers (const in C)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"{_LIB_PATH} is not built; run __graft_entry__.build() "
                           "(the optimizer has no CPU fallback)")
    L = ctypes.CDLL(str(_LIB_PATH))
    P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "gs_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "gs_abi_version": ([], i32),
        "gs_dar_normaliser": ([i64], f64),
        "gs_opt_init": ([ctypes.POINTER(P), ctypes.POINTER(gs_opt_config), i64, P], ctypes.c_int),
        "gs_opt_destroy": ([P], None),
        "gs_opt_rows": ([P], i64),
        "gs_visibility": ([P, P, ctypes.POINTER(gs_camera), P, P, P, P], ctypes.c_int),
        "gs_step": ([P, ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_attrs), P, ctypes.POINTER(gs_step_params), P],
                    ctypes.c_int),
        "gs_step_camera": ([P, ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_camera), P, P,
                            ctypes.POINTER(gs_step_params), P], ctypes.c_int),
        "gs_step_host": ([P, ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_camera),
                          ctypes.POINTER(gs_step_params), ctypes.POINTER(i64), P], ctypes.c_int),
        "gs_step_host_noalloc": ([P, ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_camera),
                                  ctypes.POINTER(gs_step_params), ctypes.POINTER(i64), P], ctypes.c_int),
        "gs_reindex_state": ([P, P, P, i64, P], ctypes.c_int),
        "gs_gather_attrs": ([P, ctypes.POINTER(gs_attrs), i64, ctypes.POINTER(gs_attrs), P, i64, P], ctypes.c_int),
        "gs_active_rows": ([P, P, P, P, P], ctypes.c_int),
        "gs_copy_rows": ([P, ctypes.POINTER(gs_attrs), ctypes.POINTER(gs_attrs), P, i64, P], ctypes.c_int),
        "gs_opt_export_state": ([P, P, P, P, P], ctypes.c_int),
        "gs_opt_import_state": ([P, P, P, P, P], ctypes.c_int),
        "gs_bias_table_len": ([P], i64),
        "gs_bias_table": ([P, P, P, i64, P], ctypes.c_int),
        "gs_opt_sync_errors": ([P, P], ctypes.c_int),
        "gs_batch_create": ([ctypes.POINTER(P), P, i32], ctypes.c_int),
        "gs_batch_destroy": ([P], None),
        "gs_batch_step": ([P, P, P, P, P, P, P], ctypes.c_int),
        "gs_batch_graph_step": ([P, P, P, P, P, P, P], ctypes.c_int),
        "gs_batch_config": ([P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)],
                            ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def lib():
    return _load()


def status_name(s: int) -> str:
    return _load().gs_status_string(int(s)).decode()


def _check(s: int, what: str) -> None:
    if s != GS_OK:
        raise GsError(s, what)


def _ptr(t):
    """Device pointer of a tensor (None -> NULL)."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_attrs(groups: dict) -> gs_attrs:
    return gs_attrs(*[None if groups.get(g) is None else groups[g].data_ptr() for g, _ in GROUPS])


def make_camera(cam16) -> gs_camera:
    c = [float(x) for x in cam16]
    return gs_camera((ctypes.c_float * 9)(*c[:9]), (ctypes.c_float * 3)(*c[9:12]), *c[12:16])


def make_config(beta1=0.9, beta2=0.999, eps=1e-15, lambda_o=1e-3, lambda_s=1e-5, clip_o=10.0, clip_s=10.0,
                alpha1=0.2, alpha2=0.04, prec=GS_MOM_FP32, bias_mode=0, reg_mode=GS_REG_DAR,
                n_pixels=800 * 800) -> gs_opt_config:
    return gs_opt_config(beta1, beta2, eps, lambda_o, lambda_s, clip_o, clip_s, alpha1, alpha2, prec, bias_mode,
                         reg_mode, 0, n_pixels)


def make_params(lr, iteration, dar_opacity=True, dar_scale=True, restate=False, restate_ratio=0.0, seed=0,
                n_visible=0, noise=0, noise_lr=5e5, noise_k=100.0, noise_t=0.005, aiu=False, aiu_prob=0.0,
                aiu_scale=1.0, n_active=None) -> gs_step_params:
    """Per-step parameters.  noise: GS_NOISE_OFF / _VISIBLE / _ALL (position
    noise of App. Eq. disentangled_mu; noise_lr, noise_k, noise_t are
    eta_Ro, lambda_mu, lambda_t, not given by the paper: the defaults are
    3DGS-MCMC's).  aiu: the Artificial Implicit Update with probability
    aiu_prob and step scale aiu_scale.  n_active: optional device int64
    tensor that receives the active count (opacity > 1/255)."""
    return gs_step_params((ctypes.c_float * 6)(*[float(x) for x in lr]), int(bool(dar_opacity)),
                          int(bool(dar_scale)), int(bool(restate)), 0, float(restate_ratio),
                          int(seed) & (2 ** 64 - 1), int(iteration), int(n_visible), int(noise), int(bool(aiu)),
                          float(noise_lr), float(noise_k), float(noise_t), float(aiu_prob), float(aiu_scale), 0,
                          None if n_active is None else n_active.data_ptr())


# ------------------------------------------------------------- entry points

def gs_abi_version() -> int:
    return _load().gs_abi_version()


def gs_dar_normaliser(n_pixels: int) -> float:
    return _load().gs_dar_normaliser(int(n_pixels))


def gs_opt_init(cfg: gs_opt_config, n_rows: int, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_load().gs_opt_init(ctypes.byref(h), ctypes.byref(cfg), int(n_rows), _stream(stream)), "gs_opt_init")
    return h


def gs_opt_destroy(h) -> None:
    _load().gs_opt_destroy(h)


def gs_opt_rows(h) -> int:
    return _load().gs_opt_rows(h)


def gs_visibility(h, xyz, cam: gs_camera, mask, visible_rows=None, n_visible=None, stream=None) -> None:
    _check(_load().gs_visibility(h, _ptr(xyz), ctypes.byref(cam), _ptr(mask), _ptr(visible_rows), _ptr(n_visible),
                                 _stream(stream)), "gs_visibility")


def gs_copy_rows(h, attrs: gs_attrs, grads: gs_attrs, rows, n_listed: int, stream=None) -> None:
    _check(_load().gs_copy_rows(h, ctypes.byref(attrs), ctypes.byref(grads), _ptr(rows), n_listed, _stream(stream)),
           "gs_copy_rows")


def gs_step(h, attrs: gs_attrs, grads: gs_attrs, mask, params: gs_step_params, stream=None) -> None:
    _check(_load().gs_step(h, ctypes.byref(attrs), ctypes.byref(grads), _ptr(mask), ctypes.byref(params),
                           _stream(stream)), "gs_step")


def gs_step_camera(h, attrs: gs_attrs, grads: gs_attrs, cam: gs_camera, params: gs_step_params, mask_out=None,
                   n_visible=None, stream=None) -> None:
    _check(_load().gs_step_camera(h, ctypes.byref(attrs), ctypes.byref(grads), ctypes.byref(cam), _ptr(mask_out),
                                  _ptr(n_visible), ctypes.byref(params), _stream(stream)), "gs_step_camera")


def gs_step_host(h, attrs: gs_attrs, grads_host: gs_attrs, cam: gs_camera, params: gs_step_params,
                 stream=None) -> int:
    nv = ctypes.c_int64(0)
    _check(_load().gs_step_host(h, ctypes.byref(attrs), ctypes.byref(grads_host), ctypes.byref(cam),
                                ctypes.byref(params), ctypes.byref(nv), _stream(stream)), "gs_step_host")
    return nv.value


def gs_step_host_noalloc(h, attrs: gs_attrs, grads_host: gs_attrs, cam: gs_camera, params: gs_step_params,
                         stream=None) -> int:
    nv = ctypes.c_int64(0)
    _check(_load().gs_step_host_noalloc(h, ctypes.byref(attrs), ctypes.byref(grads_host), ctypes.byref(cam),
                                        ctypes.byref(params), ctypes.byref(nv), _stream(stream)),
           "gs_step_host_noalloc")
    return nv.value


def gs_reindex_state(h, src_rows, reset, n_new: int, stream=None) -> None:
    _check(_load().gs_reindex_state(h, _ptr(src_rows), _ptr(reset), int(n_new), _stream(stream)),
           "gs_reindex_state")


def gs_gather_attrs(h, attrs_in: gs_attrs, n_in: int, attrs_out: gs_attrs, src_rows, n_new: int,
                    stream=None) -> None:
    _check(_load().gs_gather_attrs(h, ctypes.byref(attrs_in), int(n_in), ctypes.byref(attrs_out), _ptr(src_rows),
                                   int(n_new), _stream(stream)), "gs_gather_attrs")


def gs_active_rows(h, opacity, rows, n_active, stream=None) -> None:
    """Ascending rows with opacity > 1/255 into `rows` (optional) and their
    count into the device int64 `n_active`."""
    _check(_load().gs_active_rows(h, _ptr(opacity), _ptr(rows), _ptr(n_active), _stream(stream)), "gs_active_rows")


def gs_opt_export_state(h, m=None, v=None, t=None, stream=None) -> None:
    _check(_load().gs_opt_export_state(h, _ptr(m), _ptr(v), _ptr(t), _stream(stream)), "gs_opt_export_state")


def gs_opt_import_state(h, m=None, v=None, t=None, stream=None) -> None:
    _check(_load().gs_opt_import_state(h, _ptr(m), _ptr(v), _ptr(t), _stream(stream)), "gs_opt_import_state")


def gs_bias_table_len(h) -> int:
    return _load().gs_bias_table_len(h)


def gs_bias_table(h, b1, b2, length: int, stream=None) -> None:
    _check(_load().gs_bias_table(h, _ptr(b1), _ptr(b2), int(length), _stream(stream)), "gs_bias_table")


def gs_opt_sync_errors(h, stream=None) -> int:
    return _load().gs_opt_sync_errors(h, _stream(stream))


# ------------------------------------------------------------------ batches

class Batch:
    """Host arrays for gs_batch_* (attrs, grads, cameras, params of every
    scene), built once from per-scene structs and reused across calls."""

    def __init__(self, handles):
        n = len(handles)
        self.n = n
        arr = (ctypes.c_void_p * n)(*[h.value for h in handles])
        self.h = ctypes.c_void_p()
        _check(_load().gs_batch_create(ctypes.byref(self.h), arr, n), "gs_batch_create")
        self.attrs = (gs_attrs * n)()
        self.grads = (gs_attrs * n)()
        self.cams = (gs_camera * n)()
        self.params = (gs_step_params * n)()

    def set(self, s, attrs=None, grads=None, cam=None, params=None):
        if attrs is not None:
            self.attrs[s] = attrs
        if grads is not None:
            self.grads[s] = grads
        if cam is not None:
            self.cams[s] = cam
        if params is not None:
            self.params[s] = params

    def close(self):
        if self.h is not None and self.h.value:
            _load().gs_batch_destroy(self.h)
            self.h = None


def gs_batch_step(b: Batch, n_visible=None, stream=None, graph: bool = False) -> None:
    fn = _load().gs_batch_graph_step if graph else _load().gs_batch_step
    _check(fn(b.h, ctypes.cast(b.attrs, ctypes.c_void_p), ctypes.cast(b.grads, ctypes.c_void_p),
              ctypes.cast(b.cams, ctypes.c_void_p), ctypes.cast(b.params, ctypes.c_void_p), _ptr(n_visible),
              _stream(stream)), "gs_batch_graph_step" if graph else "gs_batch_step")


def gs_batch_graph_step(b: Batch, n_visible=None, stream=None) -> None:
    gs_batch_step(b, n_visible, stream, graph=True)


def gs_batch_config(b: Batch) -> dict:
    t, w, m, tuned = (ctypes.c_int32() for _ in range(4))
    _check(_load().gs_batch_config(b.h, ctypes.byref(t), ctypes.byref(w), ctypes.byref(m), ctypes.byref(tuned)),
           "gs_batch_config")
    return dict(tile_rows=t.value, sh_width=w.value, blocks_per_sm=m.value, tuned=bool(tuned.value))


def gs_batch_create(handles) -> Batch:
    return Batch(handles)


def gs_batch_destroy(b: Batch) -> None:
    b.close()
