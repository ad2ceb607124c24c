"""FP64 CPU oracle for the AdamW-GS optimizer step (arXiv 2601.16736).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2601_16736_gb300``) never imports it and
shares no code with it: the arithmetic lives in ``oracle/oracle.c``, compiled
with gcc (``-ffp-contract=off``) into ``oracle/liboracle.so``.

Arrays follow the canonical 59-column row of ``oracle.c``: xyz 0-2, log-scale
3-5, quaternion 6-9, opacity logit 10, SH 11-58 (DC 11-13).  Attributes and
moments are float64; gradients and positions enter as float32, as the GPU path
receives them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

NCOL = 59
_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB_PATH = _HERE / "liboracle.so"
_lib = None

# column -> learning-rate group (xyz, scale, rotation, opacity, SH DC, SH rest)
LR_GROUP = np.array([0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * 45, dtype=np.int64)


def build(force: bool = False) -> Path:
    """Compile oracle.c into liboracle.so (plain gcc, no CUDA)."""
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".so.{os.getpid()}")
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             str(_SRC), "-o", str(tmp), "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(ctypes.Structure):
    _fields_ = [
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
        ("lambda_o", ctypes.c_double), ("lambda_s", ctypes.c_double),
        ("clip_o", ctypes.c_double), ("clip_s", ctypes.c_double),
        ("n_i", ctypes.c_double), ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double),
        ("bias_mode", ctypes.c_int32), ("reg_mode", ctypes.c_int32),
    ]


class _Ext(ctypes.Structure):
    _fields_ = [
        ("noise_mode", ctypes.c_int32), ("aiu", ctypes.c_int32),
        ("noise_lr", ctypes.c_double), ("noise_k", ctypes.c_double), ("noise_t", ctypes.c_double),
        ("aiu_prob", ctypes.c_double), ("aiu_scale", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


@dataclass
class Ext:
    """Position noise (App. Eq. disentangled_mu) and AIU (Sec. 3.2) switches
    of one iteration.  noise_mode: 0 off, 1 visible primitives, 2 all."""
    noise_mode: int = 0
    aiu: bool = False
    noise_lr: float = 5e5
    noise_k: float = 100.0
    noise_t: float = 0.005
    aiu_prob: float = 0.0
    aiu_scale: float = 1.0
    seed: int = 0

    def _c(self) -> _Ext:
        return _Ext(int(self.noise_mode), int(bool(self.aiu)), self.noise_lr, self.noise_k, self.noise_t,
                    self.aiu_prob, self.aiu_scale, self.seed & (2**64 - 1))


@dataclass
class Config:
    """Static hyper-parameters; defaults are the paper's (App. "Hyperparameter
    Selection": lambda_o 1e-3, lambda_s 1e-5, C_t 10, alpha 0.2 / 0.04)."""
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    lambda_o: float = 1e-3
    lambda_s: float = 1e-5
    clip_o: float = 10.0
    clip_s: float = 10.0
    n_i: float = 60000.0
    alpha1: float = 0.2
    alpha2: float = 0.04
    bias_mode: int = 0
    reg_mode: int = 0

    def _c(self) -> _Config:
        return _Config(self.beta1, self.beta2, self.eps, self.lambda_o, self.lambda_s,
                       self.clip_o, self.clip_s, self.n_i, self.alpha1, self.alpha2,
                       self.bias_mode, self.reg_mode)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB_PATH))
        P = ctypes.c_void_p
        i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        L.orc_dar_normaliser.argtypes = [i64]
        L.orc_dar_normaliser.restype = f64
        L.orc_splitmix64_at.argtypes = [u64, u64]
        L.orc_splitmix64_at.restype = u64
        L.orc_stss_sampled.argtypes = [u64, i64, i64, f64]
        L.orc_stss_sampled.restype = i32
        L.orc_visibility_f32.argtypes = [P, i64, P, P]
        L.orc_visibility_f32.restype = None
        L.orc_frustum_margin_f64.argtypes = [P, i64, P, P, P]
        L.orc_frustum_margin_f64.restype = None
        L.orc_step.argtypes = [ctypes.POINTER(_Config), i64, P, P, P, P, P, P, P, i32, i32, i64, i64]
        L.orc_step.restype = None
        L.orc_restate.argtypes = [ctypes.POINTER(_Config), i64, P, P, P, u64, i64, f64]
        L.orc_restate.restype = i64
        L.orc_reindex.argtypes = [i64, P, P, P, i64, P, P, P, P, P]
        L.orc_reindex.restype = i32
        L.orc_bias_denominators.argtypes = [f64, i64, P]
        L.orc_bias_denominators.restype = None
        L.orc_aiu_sampled.argtypes = [u64, i64, i64, f64]
        L.orc_aiu_sampled.restype = i32
        L.orc_gauss3.argtypes = [u64, i64, i64, P]
        L.orc_gauss3.restype = None
        L.orc_covariance.argtypes = [P, P, P]
        L.orc_covariance.restype = None
        L.orc_noise_term.argtypes = [P, f64, f64, f64, f64, P, P]
        L.orc_noise_term.restype = None
        L.orc_is_active.argtypes = [f64]
        L.orc_is_active.restype = i32
        L.orc_active_rows.argtypes = [P, i64, P]
        L.orc_active_rows.restype = i64
        L.orc_step_ext.argtypes = [ctypes.POINTER(_Config), i64, P, P, P, P, P, P, P, i32, i32, i64, i64,
                                   ctypes.POINTER(_Ext), P]
        L.orc_step_ext.restype = i64
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _req(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def dar_normaliser(n_pixels: int) -> float:
    return lib().orc_dar_normaliser(int(n_pixels))


def splitmix64_at(seed: int, counter: int) -> int:
    return lib().orc_splitmix64_at(seed & (2**64 - 1), counter & (2**64 - 1))


def stss_sampled(seed: int, k: int, rows, ratio: float) -> np.ndarray:
    L = lib()
    return np.array([L.orc_stss_sampled(seed & (2**64 - 1), int(k), int(r), float(ratio)) for r in rows],
                    dtype=np.uint8)


def visibility_f32(xyz, cam) -> np.ndarray:
    xyz = _req(xyz, np.float32)
    n = xyz.size // 3
    cam = _req(cam, np.float32, (16,))
    mask = np.zeros(n, np.uint8)
    lib().orc_visibility_f32(_ptr(xyz), n, _ptr(cam), _ptr(mask))
    return mask


def visibility(xyz, cam) -> np.ndarray:
    """The visibility filter V of Eq. meth::sparse_beta, read as the frustum
    test of the mean, decided in FP64: 1 where the signed distance to every
    frustum plane (``frustum_margin_f64``) is >= 0."""
    return frustum_margin_f64(xyz, cam)[1]


def frustum_margin_f64(xyz, cam):
    xyz = _req(xyz, np.float32)
    n = xyz.size // 3
    cam = _req(cam, np.float32, (16,))
    margin = np.zeros(n, np.float64)
    mask64 = np.zeros(n, np.uint8)
    lib().orc_frustum_margin_f64(_ptr(xyz), n, _ptr(cam), _ptr(margin), _ptr(mask64))
    return margin, mask64


def frustum_fp32_band(xyz, cam) -> np.ndarray:
    """Per-row bound on |FP64 frustum margin| wherever the FP32 decision of
    ``visibility_f32`` can differ from the exact (FP64) one.

    The FP32 test evaluates each camera coordinate p_r = sum_j R_rj mu_j + t_r
    with rounded products summed left to right.  By the inner-product bound
    (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1) the
    computed value is within gamma_4 * S_r of the exact one, S_r =
    sum_j |R_rj mu_j| + |t_r|, gamma_4 = 4u / (1 - 4u), u = 2^-24.  The side
    test |p_x| <= fl(p_z tan_x) also rounds the product once (u |p_z tan_x|).
    A decision can flip only where the exact quantity lies within the sum of
    these errors of zero; divided by the plane normal's length (the margin is
    a Euclidean distance) that gives, per plane,
        side x:  (e_x + tan_x e_z + u tan_x (|p_z| + e_z)) / sqrt(1 + tan_x^2)
        side y:  the same with y
        near, far:  e_z
    and the band is the largest of them (plus 1e-12 (1 + S) for the FP64
    margin's own rounding)."""
    x = np.asarray(xyz, np.float32).reshape(-1, 3).astype(np.float64)
    c = np.asarray(cam, np.float32).reshape(16).astype(np.float64)
    u = 2.0 ** -24
    g4 = 4 * u / (1 - 4 * u)
    R = c[:9].reshape(3, 3)
    t = c[9:12]
    S = np.abs(x[:, None, :] * R[None, :, :]).sum(axis=2) + np.abs(t)[None, :]
    e = g4 * S
    pz = x @ R[2] + t[2]
    tx, ty = c[12], c[13]
    bx = (e[:, 0] + tx * e[:, 2] + u * tx * (np.abs(pz) + e[:, 2])) / np.sqrt(1 + tx * tx)
    by = (e[:, 1] + ty * e[:, 2] + u * ty * (np.abs(pz) + e[:, 2])) / np.sqrt(1 + ty * ty)
    return np.maximum(np.maximum(bx, by), e[:, 2]) + 1e-12 * (1 + S.max(axis=1))


class State:
    """Oracle copy of the primitives: FP64 attributes, FP64 moments, u32 t."""

    def __init__(self, theta, m=None, v=None, t=None):
        self.theta = np.array(theta, dtype=np.float64, order="C").reshape(-1, NCOL)
        n = self.theta.shape[0]
        self.m = np.zeros((n, NCOL)) if m is None else np.array(m, np.float64).reshape(n, NCOL)
        self.v = np.zeros((n, NCOL)) if v is None else np.array(v, np.float64).reshape(n, NCOL)
        self.t = np.zeros(n, np.uint32) if t is None else np.array(t, np.uint32).reshape(n)

    @property
    def n(self) -> int:
        return self.theta.shape[0]

    def copy(self) -> "State":
        return State(self.theta.copy(), self.m.copy(), self.v.copy(), self.t.copy())


def step(cfg: Config, st: State, grad, mask, lr, dar_o: bool, dar_s: bool, k: int,
         n_visible: int = 0) -> None:
    """One optimizer step in place (see orc_step in oracle.c)."""
    grad = _req(grad, np.float32, (st.n, NCOL))
    mask_a = None if mask is None else _req(mask, np.uint8, (st.n,))
    lr = _req(lr, np.float64, (6,))
    c = cfg._c()
    lib().orc_step(ctypes.byref(c), st.n, _ptr(st.theta), _ptr(grad), _ptr(st.m), _ptr(st.v),
                   _ptr(st.t), _ptr(mask_a), _ptr(lr), int(bool(dar_o)), int(bool(dar_s)), int(k),
                   int(n_visible))


def restate(cfg: Config, st: State, seed: int, k: int, ratio: float, row_ids=None) -> int:
    """Re-State Regularization on the StSS-sampled rows, in place."""
    ids = None if row_ids is None else _req(row_ids, np.int64, (st.n,))
    c = cfg._c()
    return lib().orc_restate(ctypes.byref(c), st.n, _ptr(st.m), _ptr(st.v), _ptr(ids),
                             seed & (2**64 - 1), int(k), float(ratio))


def reindex(st: State, src, reset=None) -> State:
    """State gather for a new row set; returns a new State (theta left zero:
    attribute re-indexing belongs to the caller)."""
    src = _req(src, np.int32)
    n_new = src.size
    rs = None if reset is None else _req(reset, np.uint8, (n_new,))
    out = State(np.zeros((n_new, NCOL)))
    rc = lib().orc_reindex(st.n, _ptr(st.m), _ptr(st.v), _ptr(st.t), n_new, _ptr(src), _ptr(rs),
                           _ptr(out.m), _ptr(out.v), _ptr(out.t))
    if rc != 0:
        raise IndexError("reindex source row out of range")
    return out


def bias_denominators(beta: float, length: int) -> np.ndarray:
    out = np.zeros(length, np.float64)
    lib().orc_bias_denominators(float(beta), int(length), _ptr(out))
    return out


# ------------------------------------------- position noise, AIU, N_a / N_d

def aiu_sampled(seed: int, k: int, rows, prob: float) -> np.ndarray:
    """AIU membership of each row (stream tag 1)."""
    L = lib()
    return np.array([L.orc_aiu_sampled(seed & (2**64 - 1), int(k), int(r), float(prob)) for r in rows], np.uint8)


def gauss3(seed: int, k: int, row: int) -> np.ndarray:
    """The noise draw gamma ~ N(0, I_3) of one row and iteration."""
    g = np.zeros(3, np.float64)
    lib().orc_gauss3(seed & (2**64 - 1), int(k), int(row), _ptr(g))
    return g


def covariance(q, kappa) -> np.ndarray:
    q = _req(q, np.float64, (4,))
    kappa = _req(kappa, np.float64, (3,))
    out = np.zeros(9, np.float64)
    lib().orc_covariance(_ptr(q), _ptr(kappa), _ptr(out))
    return out.reshape(3, 3)


def noise_term(row, eta_ro: float, eta_mu: float, lam_mu: float, lam_t: float, gamma) -> np.ndarray:
    row = _req(row, np.float64, (NCOL,))
    gamma = _req(gamma, np.float64, (3,))
    out = np.zeros(3, np.float64)
    lib().orc_noise_term(_ptr(row), float(eta_ro), float(eta_mu), float(lam_mu), float(lam_t), _ptr(gamma),
                         _ptr(out))
    return out


def is_active(tau: float) -> bool:
    return bool(lib().orc_is_active(float(tau)))


def active_rows(tau) -> np.ndarray:
    """Ascending indices of the active rows (opacity > 1/255) of FP32 logits."""
    tau = _req(tau, np.float32)
    out = np.zeros(max(tau.size, 1), np.int32)
    c = lib().orc_active_rows(_ptr(tau), tau.size, _ptr(out))
    return out[:c].copy()


def step_ext(cfg: Config, st: State, grad, mask, lr, dar_o: bool, dar_s: bool, k: int, ext: Ext,
             row_ids=None, n_visible: int = 0) -> int:
    """orc_step with the position noise and AIU; returns N_a after the step."""
    grad = _req(grad, np.float32, (st.n, NCOL))
    mask_a = None if mask is None else _req(mask, np.uint8, (st.n,))
    lr = _req(lr, np.float64, (6,))
    ids = None if row_ids is None else _req(row_ids, np.int64, (st.n,))
    c = cfg._c()
    x = ext._c()
    return lib().orc_step_ext(ctypes.byref(c), st.n, _ptr(st.theta), _ptr(grad), _ptr(st.m), _ptr(st.v),
                              _ptr(st.t), _ptr(mask_a), _ptr(lr), int(bool(dar_o)), int(bool(dar_s)), int(k),
                              int(n_visible), ctypes.byref(x), _ptr(ids))
