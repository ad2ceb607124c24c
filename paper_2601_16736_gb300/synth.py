"""Seeded synthetic inputs shaped like the paper's 3DGS / 3DGS-MCMC scenes.

This module only draws inputs: primitive attributes, cameras, gradients,
per-step hyper-parameters and re-index events.  It holds none of the
optimizer's arithmetic, so the CUDA path and the FP64 oracle can both consume
it without sharing method code.  All randomness is numpy ``default_rng`` with
explicit seeds, drawn on the host.

Attribute groups (structure of arrays, float32, row-major per group):
    xyz [N,3]  position mu
    scale [N,3] log-scale kappa (s = exp(kappa))
    rot [N,4]  quaternion
    opacity [N,1] opacity logit tau (o = sigmoid(tau))
    sh [N,48]  16 SH coefficients x RGB, columns 0-2 = DC
The canonical 59-column row concatenates them in that order.

The Mip-NeRF360 / Tanks&Temples / Deep Blending scenes of the paper are not
available; these generators stand in for them with the primitive counts
(0.1 M - 6 M), attribute distributions and visible fractions stated per
workload below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GROUPS = (("xyz", 3), ("scale", 3), ("rot", 4), ("opacity", 1), ("sh", 48))
NCOL = 59
GROUP_SLICES = {}
_c = 0
for _name, _w in GROUPS:
    GROUP_SLICES[_name] = slice(_c, _c + _w)
    _c += _w
del _c, _name, _w

# 3DGS reference-implementation defaults (publicly documented), used as
# workload configuration: xyz 1.6e-4 -> 1.6e-6 log-linear, SH DC 2.5e-3,
# SH rest 2.5e-3 / 20, opacity 2.5e-2, scale 5e-3, rotation 1e-3.
LR_DEFAULT = dict(xyz=1.6e-4, xyz_final=1.6e-6, scale=5e-3, rot=1e-3, opacity=2.5e-2,
                  sh_dc=2.5e-3, sh_rest=2.5e-3 / 20.0)


# ----------------------------------------------------------------- scenes

def _attrs_common(rng, n):
    scale = rng.normal(-4.0, 0.5, size=(n, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rot = q.astype(np.float32)
    opacity = rng.normal(0.0, 1.0, size=(n, 1)).astype(np.float32)
    sh = rng.normal(0.0, 0.2, size=(n, 48)).astype(np.float32)
    return scale, rot, opacity, sh


def scene_uniform(n: int, seed: int, half_extent: float = 5.0) -> dict:
    """Means uniform in [-5, 5]^3; other attributes as in every workload."""
    rng = np.random.default_rng([seed, 1])
    xyz = rng.uniform(-half_extent, half_extent, size=(n, 3)).astype(np.float32)
    scale, rot, opacity, sh = _attrs_common(rng, n)
    return dict(xyz=xyz, scale=scale, rot=rot, opacity=opacity, sh=sh)


def scene_blobs(n: int, seed: int, extent: float, n_blobs: int = 64, sigma: float = 0.5,
                shuffle: bool = True) -> dict:
    """Means in `n_blobs` isotropic Gaussian blobs (std `sigma`) whose centres
    are uniform in [-extent, extent]^3.  Rows are in random order when
    `shuffle` (the worst case for row locality), else grouped by blob."""
    rng = np.random.default_rng([seed, 2])
    centres = rng.uniform(-extent, extent, size=(n_blobs, 3))
    which = rng.integers(0, n_blobs, size=n)
    if not shuffle:
        which = np.sort(which)
    xyz = (centres[which] + rng.normal(0.0, sigma, size=(n, 3))).astype(np.float32)
    scale, rot, opacity, sh = _attrs_common(rng, n)
    return dict(xyz=xyz, scale=scale, rot=rot, opacity=opacity, sh=sh)


def to_rows(groups: dict) -> np.ndarray:
    """Concatenate the five groups into the canonical [N, 59] float32 rows."""
    return np.concatenate([np.asarray(groups[g], np.float32).reshape(-1, w) for g, w in GROUPS], axis=1)


def from_rows(rows: np.ndarray) -> dict:
    rows = np.asarray(rows)
    return {g: np.ascontiguousarray(rows[:, GROUP_SLICES[g]]) for g, _ in GROUPS}


# ---------------------------------------------------------------- cameras

def look_at_camera(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), fov_x_deg: float = 60.0,
                   fov_y_deg: float = 60.0, znear: float = 0.01, zfar: float = 100.0) -> np.ndarray:
    """Pinhole camera as float32[16] = {R row-major (world->camera), t, tan(fov_x/2),
    tan(fov_y/2), z_near, z_far}; OpenCV axes (x right, y down, z forward)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    cam = np.concatenate([R.reshape(-1), t, [math.tan(math.radians(fov_x_deg) / 2),
                                             math.tan(math.radians(fov_y_deg) / 2), znear, zfar]])
    return cam.astype(np.float32)


def ring_cameras(n_azimuth: int, elevations_deg=(0.0,), radius: float = 10.0,
                 fov_deg: float = 60.0) -> list:
    """Cameras on circles of `radius` around the origin, looking at it: every
    elevation x `n_azimuth` evenly spaced azimuths (800x800, 60 deg FOV)."""
    cams = []
    for el in elevations_deg:
        e = math.radians(el)
        for a in range(n_azimuth):
            az = 2 * math.pi * a / n_azimuth
            eye = (radius * math.cos(e) * math.cos(az), radius * math.cos(e) * math.sin(az),
                   radius * math.sin(e))
            cams.append(look_at_camera(eye, fov_x_deg=fov_deg, fov_y_deg=fov_deg))
    return cams


def view_order(n_views: int, n_steps: int, seed: int) -> np.ndarray:
    """View index for steps 1..n_steps: a fresh random permutation each epoch."""
    out = np.empty(n_steps, np.int64)
    for e in range((n_steps + n_views - 1) // n_views):
        perm = np.random.default_rng([seed, 3, e]).permutation(n_views)
        lo = e * n_views
        hi = min(lo + n_views, n_steps)
        out[lo:hi] = perm[: hi - lo]
    return out


# -------------------------------------------------------------- gradients

def grads_rows(n: int, seed: int, buffer: int = 0, sigma_xyz: float = 1e-4,
               sigma_other: float = 1e-3) -> np.ndarray:
    """Photometric gradients as [N, 59] float32: N(0, 1e-4) on xyz, N(0, 1e-3)
    elsewhere.  Values on invisible rows are never read by the step."""
    rng = np.random.default_rng([seed, 4, buffer])
    g = rng.standard_normal(size=(n, NCOL), dtype=np.float32)
    g[:, 0:3] *= np.float32(sigma_xyz)
    g[:, 3:] *= np.float32(sigma_other)
    return g


# ------------------------------------------------- per-step hyper-params

def lr_for_step(k: int, n_steps: int, lrs: dict = LR_DEFAULT) -> np.ndarray:
    """Per-group learning rates at iteration k (1-based): xyz log-linear from
    its initial to its final value over the run, others constant.  Order:
    xyz, scale, rot, opacity, SH DC, SH rest."""
    s = 0.0 if n_steps <= 1 else min(max((k - 1) / (n_steps - 1), 0.0), 1.0)
    lr_xyz = math.exp((1 - s) * math.log(lrs["xyz"]) + s * math.log(lrs["xyz_final"]))
    return np.array([lr_xyz, lrs["scale"], lrs["rot"], lrs["opacity"], lrs["sh_dc"], lrs["sh_rest"]],
                    dtype=np.float64)


# --------------------------------------------------------- re-index events

def reindex_event(n: int, seed: int, event: int, prune: float = 0.05, clone: float = 0.05,
                  relocate: float = 0.02):
    """An MCMC-style row-set change: prune a random `prune` fraction, append
    clones of a random `clone` fraction (new state), and relocate a random
    `relocate` fraction (destination keeps its slot, state reset).

    Returns (src int32[N'], reset uint8[N'], attr_src int32[N']): src[j] is the
    old row whose optimizer state row j inherits (-1 = fresh), reset[j] marks
    rows whose state restarts at zero, attr_src[j] the old row whose
    attributes the caller copies into row j."""
    rng = np.random.default_rng([seed, 5, event])
    n_prune = int(round(prune * n))
    n_clone = int(round(clone * n))
    keep = np.sort(rng.permutation(n)[n_prune:]).astype(np.int32)
    n_keep = keep.size
    reloc_dst = rng.choice(n_keep, size=int(round(relocate * n)), replace=False)
    reloc_src = keep[rng.integers(0, n_keep, size=reloc_dst.size)]
    clone_src = keep[rng.integers(0, n_keep, size=n_clone)]
    src = np.concatenate([keep, np.full(n_clone, -1, np.int32)]).astype(np.int32)
    reset = np.zeros(src.size, np.uint8)
    reset[reloc_dst] = 1
    attr_src = np.concatenate([keep, clone_src]).astype(np.int32)
    attr_src[reloc_dst] = reloc_src
    return src, reset, attr_src


# -------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    n: int
    steps: int
    seed: int
    scene: str                      # "uniform" or "blobs"
    extent: float = 5.0             # blob-centre half extent (blobs only)
    elevations: tuple = (0.0,)
    n_azimuth: int = 200
    dar: bool = True                # DAR on opacity and scale every step
    restate_every: int = 100        # RSR interval (App. "StSS in RSR")
    restate_ratio: float = 0.1      # StSS ratio (schedule only in a figure; our choice)
    grad_buffers: int = 8
    n_pixels: int = 800 * 800
    extra: dict = field(default_factory=dict)

    def scene_groups(self) -> dict:
        if self.scene == "uniform":
            return scene_uniform(self.n, self.seed)
        return scene_blobs(self.n, self.seed, self.extent)

    def cameras(self) -> list:
        return ring_cameras(self.n_azimuth, self.elevations)


# Blob extents chosen so the mean visible fraction over the 200 views is near
# the target (0.30 at 1 M, 0.20 at 3 M, 0.10 at 6 M); the bench reports the
# fraction it measures.
WORKLOADS = {
    "c1_100k": Workload("c1_100k", 100_000, 50, 1001, "uniform", n_azimuth=50),
    "c2_1m": Workload("c2_1m", 1_000_000, 1000, 1002, "blobs", extent=12.5,
                      elevations=(-30.0, -15.0, 0.0, 15.0, 30.0), n_azimuth=40),
    "c3_3m": Workload("c3_3m", 3_000_000, 1000, 1003, "blobs", extent=22.0,
                      elevations=(-30.0, -15.0, 0.0, 15.0, 30.0), n_azimuth=40),
    "c5_6m": Workload("c5_6m", 6_000_000, 3000, 1005, "blobs", extent=75.0,
                      elevations=(-30.0, -15.0, 0.0, 15.0, 30.0), n_azimuth=40, grad_buffers=4),
}
