"""Test harness: drives the CUDA path through the C ABI and the FP64 oracle
side by side on the same seeded inputs, and compares them per attribute
group.  Test infrastructure only."""
from __future__ import annotations

import numpy as np

from paper_2601_16736_gb300 import synth

GROUP_COLS = {"xyz": slice(0, 3), "scale": slice(3, 6), "rot": slice(6, 10), "opacity": slice(10, 11),
              "sh": slice(11, 59)}


def group_errors(got_rows: np.ndarray, ref_rows: np.ndarray, rows=None) -> dict:
    """Per group: max|d| / max|ref| (the relative error gate) and the largest
    elementwise |d| / (|ref| + 1e-3)."""
    out = {}
    for g, sl in GROUP_COLS.items():
        a = np.asarray(got_rows[:, sl], np.float64)
        b = np.asarray(ref_rows[:, sl], np.float64)
        if rows is not None:
            a, b = a[rows], b[rows]
        if a.size == 0:
            out[g] = (0.0, 0.0)
            continue
        d = np.abs(a - b)
        out[g] = (float(d.max() / max(np.abs(b).max(), 1e-30)), float((d / (np.abs(b) + 1e-3)).max()))
    return out


def assert_close(got_rows, ref_rows, rel: float, elem: float | None = None, rows=None, what: str = ""):
    errs = group_errors(got_rows, ref_rows, rows)
    for g, (r, e) in errs.items():
        assert r <= rel, f"{what} group {g}: max|d|/max|ref| = {r:.3e} > {rel:.1e}"
        if elem is not None:
            assert e <= elem, f"{what} group {g}: elementwise {e:.3e} > {elem:.1e}"
    return errs


class GpuScene:
    """Attributes, gradients and an optimizer context on cuda:0."""

    def __init__(self, groups: dict, cfg=None, **cfg_kw):
        import torch
        from paper_2601_16736_gb300 import gsopt as G
        self.G, self.torch = G, torch
        self.n = groups["xyz"].shape[0]
        self.attrs = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in groups.items()}
        self.grads = {k: torch.zeros_like(v) for k, v in self.attrs.items()}
        self.cfg = cfg if cfg is not None else G.make_config(**cfg_kw)
        self.h = G.gs_opt_init(self.cfg, self.n)
        self.mask = torch.zeros(max(self.n, 1), dtype=torch.uint8, device="cuda")
        self.nvis = torch.zeros(1, dtype=torch.int64, device="cuda")

    def close(self):
        if self.h is not None:
            self.G.gs_opt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_grads(self, grad_rows: np.ndarray):
        for k, v in synth.from_rows(grad_rows).items():
            self.grads[k].copy_(self.torch.from_numpy(v))

    def step_camera(self, cam16, params, mask_out=True):
        G = self.G
        self.nvis.zero_()
        G.gs_step_camera(self.h, G.make_attrs(self.attrs), G.make_attrs(self.grads), G.make_camera(cam16), params,
                         mask_out=self.mask if mask_out else None, n_visible=self.nvis)

    def step_mask(self, mask, params):
        G = self.G
        G.gs_step(self.h, G.make_attrs(self.attrs), G.make_attrs(self.grads), mask, params)

    def rows(self) -> np.ndarray:
        self.torch.cuda.synchronize()
        return synth.to_rows({k: v.cpu().numpy() for k, v in self.attrs.items()})

    def state(self):
        torch = self.torch
        m = torch.zeros((self.n, 59), dtype=torch.float32, device="cuda")
        v = torch.zeros_like(m)
        t = torch.zeros(self.n, dtype=torch.int32, device="cuda")
        self.G.gs_opt_export_state(self.h, m, v, t)
        torch.cuda.synchronize()
        return m.cpu().numpy(), v.cpu().numpy(), t.cpu().numpy().view(np.uint32)


class OracleRun:
    """The oracle on (a subset of) the same primitives; `row_ids` are their
    global ids (for the StSS draw)."""

    def __init__(self, orc, rows: np.ndarray, row_ids=None, **cfg_kw):
        self.orc = orc
        self.st = orc.State(rows)
        kw = dict(n_i=orc.dar_normaliser(800 * 800))
        kw.update(cfg_kw)
        self.cfg = orc.Config(**kw)
        self.row_ids = None if row_ids is None else np.asarray(row_ids, np.int64)

    def visible(self, cam16) -> np.ndarray:
        """The oracle's (FP64) frustum decision on its own positions rounded
        to FP32."""
        xyz32 = self.st.theta[:, 0:3].astype(np.float32)
        return self.orc.visibility(xyz32, cam16)

    def step(self, grad_rows, mask, lr, dar_o, dar_s, k, restate=False, ratio=0.0, seed=0, n_visible=0):
        self.orc.step(self.cfg, self.st, grad_rows, mask, lr, dar_o, dar_s, k, n_visible)
        if restate:
            self.orc.restate(self.cfg, self.st, seed, k, ratio, row_ids=self.row_ids)


# Rows within this distance of a frustum plane may be decided either way
# (the tolerance the visibility parity is stated with).
PLANE_TOL = 1e-6


def check_mask(orc, got, xyz, cam16) -> dict:
    """The GPU mask `got` against the oracle's FP64 decision on the same FP32
    means: every disagreement must lie within PLANE_TOL of a plane.  Returns
    the rows within PLANE_TOL of a plane and the disagreements among them."""
    margin, ref = orc.frustum_margin_f64(xyz, cam16)
    differ = np.asarray(got, np.uint8) != ref
    near = np.abs(margin) <= PLANE_TOL
    bad = differ & ~near
    assert not bad.any(), (f"{int(bad.sum())} visibility decisions differ from the FP64 definition away from "
                           f"the planes (largest |margin| {np.abs(margin[bad]).max():.3e})")
    return {"near_plane": int(near.sum()), "differ": int(differ.sum())}


def check_trajectory_masks(orc, gmask, omask, orc_xyz, gpu_xyz, cam16) -> int:
    """Masks of the same step taken on the GPU's and the oracle's positions,
    which differ by the FP32 rounding of earlier steps.  The GPU decides
    exactly, so a decision may differ only where the oracle's mean is within
    |mu_gpu - mu_oracle| + PLANE_TOL of a plane (R is a rotation, so moving a
    mean by d moves its plane distances by at most |d|).  Returns the count."""
    differ = np.asarray(gmask, np.uint8) != np.asarray(omask, np.uint8)
    if differ.any():
        margin, _ = orc.frustum_margin_f64(np.asarray(orc_xyz, np.float32)[differ], cam16)
        d = np.linalg.norm(np.asarray(gpu_xyz, np.float64)[differ] - np.asarray(orc_xyz, np.float64)[differ], axis=1)
        assert np.all(np.abs(margin) <= d + PLANE_TOL), "decision differs farther from a plane than the means do"
    return int(differ.sum())
