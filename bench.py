"""Throughput of the fused AdamW-GS step (visibility + Sparse Adam + DAR + RSR).

Headline (``value``): the 1 M-primitive workload — 59 FP32 attributes per
primitive (xyz 3, log-scale 3, quaternion 4, opacity logit 1, SH degree 3 48),
means in 64 Gaussian blobs, 200 ring/elevation views in random order (about
30 % of the primitives visible per view), DAR on opacity and scale every step,
RSR every 100 steps (StSS ratio 0.1, an RSR step inside every timed window),
FP32 moments.  One step = one launch of the fused step kernel over all rows;
the timed steps run back to back between two region events.

Beside it in the same line: ``roofline`` (algorithmic bytes per step against
the measured copy bandwidth; DRAM traffic from the committed ncu capture of
this kernel build), ``e2e`` (the host-gradient call), per-launch percentiles
from a second instrumented pass, the blob-sorted row order, the 100 k
(L2-resident) workload, mixed-precision moments on the 1 M and 3 M workloads
with their error against the FP32 step, the optional terms, the access
ceiling, the re-index and batched workloads, the GPU's frustum decisions
against the FP64 oracle, and the oracle itself on the host cores.

Prints one JSON line.  Multi-GPU (torchrun): every rank runs an independent
replica on its own scene (rows are independent; no data exchange); value =
visible updates of all ranks / the slowest rank's time.

--impl reference times the FP64 CPU oracle (the method's plain restatement)
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import json
import os
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "visible Gaussians updated/s & HBM GB/s: mixed-prec vs FP32 step at ≤1e-3 err"
UNIT = "visible Gaussians/s"
WORKLOAD = "c2_1m"
MIXED_WORKLOAD = "c3_3m"
# Algorithmic bytes per visible row: theta read + write and g read (59 FP32
# values each), m and v read + write in the storage format, t read + write;
# minus the row's 12-B mean, whose read is already counted by the frustum test.
# FP32 moments 4 * 236 B; hybrid 4 * (45 * 2 + 14 * 4) B; BF16 4 * 59 * 2 B.
# FP16-block: 4 * (59 FP16 values + 8 group exponent bytes); its t is a uint16.
STATE_RW = {"fp32": 4 * 236, "bf16_hybrid": 4 * (45 * 2 + 14 * 4), "bf16": 4 * 118, "fp16_block": 4 * (118 + 8),
            "fp8_e4m3": 4 * 59}
T_RW = {"fp32": 8, "bf16_hybrid": 8, "bf16": 8, "fp16_block": 4, "fp8_e4m3": 8}
PREC_ENUM = {"fp32": 0, "bf16": 1, "fp8_e4m3": 2, "bf16_hybrid": 3, "fp16_block": 4}
BYTES_ROW_VIS = 12          # every row: the mean read by the frustum test
# The sources of the step kernel; the DRAM traffic of an ncu capture is
# reported only while they match the capture's record of them.
KERNEL_SOURCES = ("paper_2601_16736_gb300/csrc/step_kernels.cu", "paper_2601_16736_gb300/csrc/step_common.cuh",
                  "paper_2601_16736_gb300/csrc/gs_internal.cuh")


def bytes_visible(prec: str) -> int:
    return 3 * 236 + STATE_RW[prec] + T_RW[prec] - 12


def launch_bytes(prec: str, n_rows: int, n_visible: int, rsr_rows: int) -> int:
    """Algorithmic bytes of one fused step launch: every row's mean for the
    frustum test, each visible row's attributes, gradients, moments and step
    counter (its mean already counted), and the moments of each invisible
    StSS-sampled row that RSR scales."""
    return n_visible * bytes_visible(prec) + n_rows * BYTES_ROW_VIS + rsr_rows * STATE_RW[prec]


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "20"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
                for nm, val in zip(names, r[4:8]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(base: int, rank: int) -> int:
    """Each rank steps its own independent scene (weak scaling)."""
    return base + 1000 * rank


def reduce_over_ranks(dist, elapsed: float, units: int, device: str):
    """Whole-job figures: the slowest rank's time and the units of all ranks."""
    if dist is None:
        return elapsed, float(units)
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def rsr_offset(warmup: int, steps: int, every: int) -> int:
    """Iteration offset k0 (step i of a run is iteration k0 + i + 1) that puts
    an RSR event (k = 0 mod `every`, Eq. meth::restate with the StSS interval
    of the appendix) inside the timed steps warmup+1 .. warmup+steps, near
    their middle, whatever `steps` is."""
    return (-(warmup + (steps + 1) // 2)) % every


def headline_plan(warmup: int, steps: int, e2e_steps: int, every: int, e2e_warmup: int = 3):
    """(k0, n): the iteration offset of the headline run and the number of
    steps its scene must hold: the device-timed run uses steps 0 .. warmup +
    steps - 1 and the end-to-end leg steps 0 .. e2e_warmup + e2e_steps - 1."""
    return rsr_offset(warmup, steps, every), max(warmup + steps, e2e_warmup + e2e_steps)


class Scene:
    """One workload resident on the GPU: attributes, a pool of gradient
    buffers, cameras and the per-step parameters of `total_steps` steps.
    Step i (0-based) of a run is iteration k0 + i + 1; the learning-rate
    schedule spans the workload's own run length."""

    def __init__(self, G, synth, wl, seed, total_steps, k0=0, shuffle=True):
        import torch
        self.G, self.synth, self.wl, self.seed, self.k0 = G, synth, wl, seed, k0
        if wl.scene == "blobs":
            groups = synth.scene_blobs(wl.n, seed, wl.extent, shuffle=shuffle)
        else:
            groups = synth.scene_uniform(wl.n, seed)
        self.host_groups = groups
        self.attrs0 = {k: torch.from_numpy(v).cuda() for k, v in groups.items()}
        self.attrs = {k: v.clone() for k, v in self.attrs0.items()}
        gen = torch.Generator(device="cuda").manual_seed(seed)
        self.gbufs = []
        for _ in range(wl.grad_buffers):
            self.gbufs.append({name: torch.randn((wl.n, w), generator=gen, device="cuda", dtype=torch.float32)
                               * (1e-4 if name == "xyz" else 1e-3) for name, w in synth.GROUPS})
        self.cams = wl.cameras()
        self.order = synth.view_order(len(self.cams), max(k0 + total_steps, len(self.cams)), seed)
        self.total = total_steps
        self.A = G.make_attrs(self.attrs)
        self.GB = [G.make_attrs(g) for g in self.gbufs]
        self.CAMS = [G.make_camera(c) for c in self.cams]
        self.P = [self.params(self.k(i)) for i in range(total_steps)]

    def k(self, i: int) -> int:
        """Iteration number of step i of a run."""
        return self.k0 + i + 1

    def cam(self, i: int):
        """Camera of step i: the random view order, indexed by iteration."""
        return self.CAMS[self.order[(self.k(i) - 1) % len(self.order)]]

    def params(self, k, **extra):
        wl = self.wl
        rs = k % wl.restate_every == 0
        return self.G.make_params(self.synth.lr_for_step(k, wl.steps), k, dar_opacity=wl.dar, dar_scale=wl.dar,
                                  restate=rs, restate_ratio=wl.restate_ratio, seed=self.seed, **extra)

    def reset(self):
        for k, v in self.attrs.items():
            v.copy_(self.attrs0[k])


def timed_run(G, sc, prec, steps, warmup, clocks_device=None, dist=None, extra=None, instrument=False):
    """Warm-up then `steps` timed launches of gs_step_camera on a fresh
    context, back to back, with CUDA events on the launching stream around
    the whole region only (events between launches would serialise them and
    cost ~3.5 % here).  With `instrument`, the same steps run again on a fresh
    context with events around every launch, for the per-launch percentiles
    and the isolated kernel time.  `extra`: make_params keywords added to
    every step (the optional terms).  Step i of the run is iteration sc.k(i)."""
    import torch
    L = G.lib()
    if warmup + steps > len(sc.P):
        raise ValueError(f"scene holds {len(sc.P)} steps, the run needs {warmup + steps}")
    P = sc.P
    if extra:
        P = [sc.params(sc.k(i), **extra) for i in range(warmup + steps)]
    stream = torch.cuda.current_stream()
    sh = ctypes.c_void_p(stream.cuda_stream)

    def run(per_launch, sampler=None):
        sc.reset()
        h = G.gs_opt_init(G.make_config(n_pixels=sc.wl.n_pixels, prec=PREC_ENUM[prec]), sc.wl.n)
        counts = torch.zeros(warmup + steps, dtype=torch.int64, device="cuda")
        cnt = counts.data_ptr()

        def launch(i):
            s = L.gs_step_camera(h, ctypes.byref(sc.A), ctypes.byref(sc.GB[i % len(sc.GB)]),
                                 ctypes.byref(sc.cam(i)), None, ctypes.c_void_p(cnt + 8 * i),
                                 ctypes.byref(P[i]), sh)
            if s != 0:
                raise G.GsError(s, "gs_step_camera")

        for i in range(warmup):
            launch(i)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)] if per_launch else None
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        if sampler:
            sampler.start()
            time.sleep(0.3)
        torch.cuda.synchronize()
        if not per_launch:                     # lets a profiler restrict its launch list to the timed region
            torch.cuda.nvtx.range_push("timed")
        t0.record(stream)
        for j in range(steps):
            if per_launch:
                ev[j][0].record(stream)
            launch(warmup + j)
            if per_launch:
                ev[j][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        if not per_launch:
            torch.cuda.nvtx.range_pop()
        if dist is not None:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        G.gs_opt_destroy(h)
        per = np.array([x.elapsed_time(y) for x, y in ev]) / 1e3 if per_launch else None
        return t0.elapsed_time(t1) / 1e3, counts.cpu().numpy(), per, clocks

    sampler = ClockSampler(clocks_device) if clocks_device is not None else None
    elapsed, nv, _, clocks = run(False, sampler)
    timed_nv = int(nv[warmup:].sum())
    rsr, rsr_steps = 0, []
    for j in range(steps):
        k = sc.k(warmup + j)
        if k % sc.wl.restate_every == 0:
            rsr_steps.append(k)
            rsr += int(round(sc.wl.restate_ratio * (sc.wl.n - int(nv[warmup + j]))))
    byt = launch_bytes(prec, steps * sc.wl.n, timed_nv, rsr) / steps
    # the first timed launch: the one an ncu capture skipping the warm-up launches (-s warmup -c 1) takes
    k1, nv1 = sc.k(warmup), int(nv[warmup])
    rsr1 = int(round(sc.wl.restate_ratio * (sc.wl.n - nv1))) if k1 % sc.wl.restate_every == 0 else 0
    first = dict(iteration=k1, visible_rows=nv1, rsr_rows=rsr1,
                 algorithmic_bytes=launch_bytes(prec, sc.wl.n, nv1, rsr1))
    out = dict(elapsed=elapsed, step_s=elapsed / steps, nv=timed_nv, bytes_per_launch=byt, clocks=clocks,
               steps=steps, rsr_steps=rsr_steps, rsr_rows=rsr, first_timed=first)
    if instrument:
        _, _, per, _ = run(True)
        out["kern"] = float(per.mean())
        out.update({f"p{q}_ms": float(np.percentile(per, q) * 1e3) for q in (10, 50, 90)})
    return out


def error_vs_fp32(G, sc, prec, steps=1000):
    """Group relative L2 distance ||theta_prec - theta_fp32|| / ||theta_fp32||
    after `steps` steps of the same workload with `prec` moments and with FP32
    moments (both on the GPU, same gradients, cameras and parameters), over
    every row whose visibility decision was the same in both runs at every
    step."""
    import torch
    wl = sc.wl
    sc.reset()
    other = {k: v.clone() for k, v in sc.attrs0.items()}
    A2 = G.make_attrs(other)
    h32 = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels, prec=PREC_ENUM["fp32"]), wl.n)
    hp = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels, prec=PREC_ENUM[prec]), wl.n)
    m32 = torch.zeros(wl.n, dtype=torch.uint8, device="cuda")
    mp = torch.zeros_like(m32)
    diverged = torch.zeros(wl.n, dtype=torch.bool, device="cuda")
    for k in range(1, steps + 1):
        i = k - 1
        p = sc.params(k)
        cam = sc.CAMS[sc.order[i % len(sc.order)]]
        G.gs_step_camera(h32, sc.A, sc.GB[i % len(sc.GB)], cam, p, mask_out=m32)
        G.gs_step_camera(hp, A2, sc.GB[i % len(sc.GB)], cam, p, mask_out=mp)
        diverged |= m32 != mp
    torch.cuda.synchronize()
    G.gs_opt_destroy(h32)
    G.gs_opt_destroy(hp)
    keep = ~diverged
    errs = {}
    for g in ("xyz", "scale", "rot", "opacity", "sh"):
        ref = sc.attrs[g][keep].double()
        got = other[g][keep].double()
        errs[g] = float((got - ref).norm() / ref.norm().clamp_min(1e-30))
    return {"group_rel_l2_vs_fp32": errs, "max": max(errs.values()), "rows": int(keep.sum().item()),
            "steps": steps}


def kernel_source_sha() -> str:
    """Hash of the sources that define the step kernel: a DRAM traffic figure
    taken from an ncu capture applies only while these are unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update((ROOT / f).read_bytes())
    return h.hexdigest()[:16]


def captured_traffic(workload: str, prec: str):
    """DRAM bytes (read + write) of one step-kernel launch and the algorithmic
    bytes of that same launch, from the `bench-traffic:` lines of the ncu
    summaries under profiles/.  Returns (dram, algorithmic, note); dram is
    None when no capture matches or the kernel sources changed since."""
    sha = kernel_source_sha()
    found = None
    for f in sorted((ROOT / "profiles").glob("*.md")):
        for line in f.read_text().splitlines():
            if not line.startswith("bench-traffic:"):
                continue
            kv = dict(x.split("=", 1) for x in line.split()[1:] if "=" in x)
            if kv.get("workload") == workload and kv.get("prec") == prec:
                found = (kv, f.name)
    if found is None:
        return None, None, f"no ncu capture of the {workload} {prec} step kernel"
    kv, name = found
    if kv.get("kernel_src_sha") != sha:
        return None, None, (f"ncu capture in profiles/{name} was taken from kernel sources {kv.get('kernel_src_sha')}, "
                            f"this build is {sha}: not applicable")
    return (float(kv["dram_bytes"]), float(kv["algorithmic_bytes"]),
            f"ncu capture of this kernel build (sources {sha}), profiles/{name}, taken {kv.get('captured')}")


def e2e_leg(G, sc, prec, steps, warmup=3):
    """End to end through the public host-gradient call: every step hands the
    library FP32 gradients of all rows in pinned host memory (two buffers,
    alternating) and gets the step's visible count back.  The step kernel
    reads the visible rows' gradients in place over the CPU-GPU link; the
    attributes and the optimizer state stay resident on the device.  Timed
    on the host clock around synchronous calls."""
    import torch
    wl = sc.wl
    gh = [{k: v.cpu().pin_memory() for k, v in g.items()} for g in sc.gbufs[:2]]
    GH = [G.make_attrs(g) for g in gh]
    sc.reset()
    h = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels, prec=PREC_ENUM[prec]), wl.n)
    for i in range(warmup):
        G.gs_step_host(h, sc.A, GH[i % 2], sc.cam(i), sc.P[i])
    torch.cuda.synchronize()
    nvs = []
    tt = time.perf_counter()
    for j in range(steps):
        i = warmup + j
        nvs.append(G.gs_step_host(h, sc.A, GH[i % 2], sc.cam(i), sc.P[i]))
    dt = time.perf_counter() - tt
    G.gs_opt_destroy(h)
    tot = sum(nvs)
    return {"value": tot / dt, "unit": UNIT, "steps": steps, "ms_per_step": dt / steps * 1e3,
            "h2d_bytes_per_step": 236 * tot / steps, "d2h_bytes_per_step": 8,
            "path": ("gs_step_host, one synchronous call per step: all rows' FP32 gradients (236 B per row) sit in "
                     "pinned host memory, and the step kernel reads the visible rows' gradients in place over the "
                     "CPU-GPU link (h2d_bytes_per_step = 236 B x the visible rows of each step, counted from the "
                     "visible counts the calls return); the visible count (8 B) comes back to the host; attributes "
                     "and optimizer state stay resident on the device"),
            "host_gradient_bytes_resident": sum(v.numel() * 4 for v in gh[0].values())}


def run_ours(args):
    import torch
    from paper_2601_16736_gb300 import build as B
    B.build()
    from paper_2601_16736_gb300 import gsopt as G
    from paper_2601_16736_gb300 import synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = synth.WORKLOADS[args.workload]
    if args.grad_buffers:
        wl = dataclasses.replace(wl, grad_buffers=args.grad_buffers)
    seed = replica_seed(wl.seed, rank)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else args.steps
    k0, n_scene = headline_plan(args.warmup, args.steps, e2e_steps, wl.restate_every)
    sc = Scene(G, synth, wl, seed, n_scene, k0=k0)
    r = timed_run(G, sc, args.prec, args.steps, args.warmup, clocks_device=local, dist=dist, instrument=True)
    elapsed, timed_nv = r["elapsed"], r["nv"]
    elapsed_all, nv_all = reduce_over_ranks(dist, elapsed, timed_nv, "cuda")

    peak, peak_kind = _peaks()
    traffic, t_alg, traffic_note = captured_traffic(wl.name, args.prec)
    achieved = r["bytes_per_launch"] / r["step_s"] / 1e9
    out = {
        "metric": METRIC, "value": nv_all / elapsed_all, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_all / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{wl.name}: {wl.n} Gaussians, SH3 (59 fp32 attrs), 64 blobs, 200 views in random "
                               f"order, DAR+RSR(0.1/100), {args.prec} moments, fused visibility+step",
                   "n_rows": wl.n, "visible_fraction": timed_nv / args.steps / wl.n, "moments": args.prec,
                   "row_order": "random (shuffled)",
                   "iterations": f"{sc.k(args.warmup)}-{sc.k(args.warmup + args.steps - 1)} timed "
                                 f"(warm-up from {sc.k(0)})",
                   "rsr_steps_timed": r["rsr_steps"],
                   "l2": "inputs larger than L2: 0.94 GB of attributes/grads/state, ~0.5 GB touched per step; "
                         "no flush",
                   "parallelism": f"replicas x{ws}"},
        "p10_ms": r["p10_ms"], "p50_ms": r["p50_ms"], "p90_ms": r["p90_ms"],
        "hbm_gbs": achieved,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
                                    if peak_kind == "measured" else "fallback 6800 GB/s",
                     "traffic": traffic,
                     "traffic_over_algorithmic": traffic / t_alg if traffic else None,
                     "traffic_source": traffic_note,
                     "bytes_per_launch": r["bytes_per_launch"],
                     "duration": "mean launch time in the timed region (region events / launches, back to back)",
                     "step_ms": r["step_s"] * 1e3, "kernel_ms_isolated": r["kern"] * 1e3,
                     "first_timed_launch": r["first_timed"]},
        "gpu_launches": args.steps,
        "clocks": r["clocks"],
    }

    if rank == 0 and args.mixed:
        # the gate-passing 16-bit format on the headline workload itself
        rf = timed_run(G, sc, "fp16_block", args.steps, args.warmup, instrument=True)
        t16, a16, n16 = captured_traffic(wl.name, "fp16_block")
        out["mixed_precision_headline"] = {
            "workload": f"{wl.name} (this line's workload), {args.steps} timed steps",
            "fp16_block": {"value": rf["nv"] / rf["elapsed"], "ms_per_step": rf["elapsed"] / args.steps * 1e3,
                           "p50_ms": rf["p50_ms"], "hbm_gbs": rf["bytes_per_launch"] / rf["step_s"] / 1e9,
                           "traffic": t16, "traffic_over_algorithmic": t16 / a16 if t16 else None,
                           "traffic_source": n16,
                           "speedup_vs_fp32": (rf["nv"] / rf["elapsed"]) / (r["nv"] / r["elapsed"]),
                           "error": error_vs_fp32(G, sc, "fp16_block") if args.mixed_error else None}}
    if rank == 0 and e2e_steps > 0:
        out["e2e"] = e2e_leg(G, sc, args.prec, e2e_steps)
    del sc
    torch.cuda.empty_cache()

    if rank == 0 and args.secondary:
        out["row_order_sorted"] = sorted_order_leg(G, synth, wl, args, r)
        out["c1_100k"] = c1_leg(G, synth, max(args.steps, 200), args.warmup)
    if rank == 0 and args.mixed:
        mwl = synth.WORKLOADS[MIXED_WORKLOAD]
        msc = Scene(G, synth, mwl, mwl.seed, max(1000, args.mixed_steps + 10))
        legs = {}
        for prec in ("fp32", "fp16_block", "bf16_hybrid", "bf16", "fp8_e4m3"):
            rr = timed_run(G, msc, prec, args.mixed_steps, 10)
            tb, ta, _ = captured_traffic(mwl.name, prec)
            legs[prec] = {"value": rr["nv"] / rr["elapsed"], "hbm_gbs": rr["bytes_per_launch"] / rr["step_s"] / 1e9,
                          "ms_per_step": rr["elapsed"] / args.mixed_steps * 1e3,
                          "bytes_per_launch": rr["bytes_per_launch"],
                          "traffic_over_algorithmic": tb / ta if tb else None}
            if args.mixed_error and prec != "fp32":
                legs[prec]["error"] = error_vs_fp32(G, msc, prec)
        for prec in ("fp16_block", "bf16_hybrid", "bf16", "fp8_e4m3"):
            legs[prec]["speedup_vs_fp32"] = legs[prec]["value"] / legs["fp32"]["value"]
        legs["fp8_e4m3"]["bytes"] = ("algorithmic: 59 B per moment per visible row; the kernel also re-encodes a "
                                     "block's other rows in a column whose scale grows, and reads every row's codes "
                                     "on the block's full pass (one step in 128)")
        out["mixed_precision"] = {"workload": f"{mwl.name}: {mwl.n} Gaussians, ~20% visible, {args.mixed_steps} "
                                              f"timed steps per format", "gate": "group relative L2 vs the FP32 step <= 1e-3",
                                  **legs}
    if rank == 0 and args.next_rows:
        out["next_rows"] = next_rows_leg(G, synth, args.next_steps)
    if rank == 0 and args.ceiling:
        out["access_ceiling"] = access_ceiling_leg(G, synth)
    if rank == 0 and args.reindex:
        out["reindex"] = reindex_leg(G, synth, args.reindex_steps)
    if rank == 0 and args.batched:
        out["batched"] = batched_leg(G, synth, args.batched_steps)
    if rank == 0 and args.cpu_baseline and args.visibility_band:
        out["visibility_vs_oracle"] = visibility_leg(G, synth, wl)
    if rank == 0 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def sorted_order_leg(G, synth, wl, args, headline):
    """The headline workload with its rows grouped by blob instead of shuffled
    (the same means, attributes and views; rows of one blob are contiguous,
    so a view's visible rows form long runs): the best case for row locality,
    beside the random-order headline."""
    import torch
    sc = Scene(G, synth, wl, wl.seed, args.warmup + args.steps,
               k0=rsr_offset(args.warmup, args.steps, wl.restate_every), shuffle=False)
    r = timed_run(G, sc, args.prec, args.steps, args.warmup, instrument=True)
    del sc
    torch.cuda.empty_cache()
    peak, _ = _peaks()
    gbs = r["bytes_per_launch"] / r["step_s"] / 1e9
    return {"workload": f"{wl.name} with rows grouped by blob (not shuffled), {args.prec} moments, "
                        f"{args.steps} timed steps",
            "value": r["nv"] / r["elapsed"], "ms_per_step": r["elapsed"] / args.steps * 1e3,
            "p10_ms": r["p10_ms"], "p50_ms": r["p50_ms"], "p90_ms": r["p90_ms"], "hbm_gbs": gbs,
            "frac": gbs / peak, "visible_fraction": r["nv"] / args.steps / wl.n,
            "speedup_vs_random_order": (r["nv"] / r["elapsed"]) / (headline["nv"] / headline["elapsed"])}


def c1_leg(G, synth, steps, warmup):
    """The 100 k workload (uniform means, 50 ring views; most rows visible).
    Its whole working set (about 95 MB of attributes, gradients and FP32
    state) fits the 129 MB L2, and nothing is flushed between steps, so this
    is an L2-resident figure, not an HBM one."""
    import torch
    wl = synth.WORKLOADS["c1_100k"]
    sc = Scene(G, synth, wl, wl.seed, warmup + steps, k0=rsr_offset(warmup, steps, wl.restate_every))
    r = timed_run(G, sc, "fp32", steps, warmup, instrument=True)
    del sc
    torch.cuda.empty_cache()
    return {"workload": f"{wl.name}: {wl.n} Gaussians, uniform means, {wl.n_azimuth} ring views, fp32 moments, "
                        f"{steps} timed steps",
            "residency": "L2-resident (working set < 129 MB L2, no flush between steps)",
            "value": r["nv"] / r["elapsed"], "ms_per_step": r["elapsed"] / steps * 1e3,
            "p10_ms": r["p10_ms"], "p50_ms": r["p50_ms"], "p90_ms": r["p90_ms"],
            "gbs_algorithmic": r["bytes_per_launch"] / r["step_s"] / 1e9,
            "visible_fraction": r["nv"] / steps / wl.n}


def access_ceiling_leg(G, synth, reps=320, n_views=16):
    """The FP32 step beside gs_copy_rows on the same visible rows.  The copy
    reads every attribute, gradient, moment and step-counter byte the step
    reads for those rows and writes back every byte it writes (the same
    1648 B per row), with no arithmetic, at full parallelism: the cost of
    the scattered row accesses alone.  step_over_copy is what the update,
    the frustum test over every row (12 B each, not in the copy) and the
    in-kernel compaction add to it.  n_views views of each workload, cycled;
    no RSR steps."""
    import torch
    out = {}
    for wname in (WORKLOAD, MIXED_WORKLOAD):
        wl = synth.WORKLOADS[wname]
        sc = Scene(G, synth, wl, wl.seed, n_views)
        h = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels), wl.n)
        masks = torch.zeros((n_views, wl.n), dtype=torch.uint8, device="cuda")
        lists = torch.zeros((n_views, wl.n), dtype=torch.int32, device="cuda")
        cnts = torch.zeros(n_views, dtype=torch.int64, device="cuda")
        for i in range(n_views):
            G.gs_visibility(h, sc.attrs["xyz"], sc.CAMS[sc.order[i]], masks[i], lists[i], cnts[i:i + 1])
        nvs = cnts.cpu().tolist()
        P = [G.make_params(synth.lr_for_step(k, 1000), k, dar_opacity=wl.dar, dar_scale=wl.dar)
             for k in range(1, n_views + 1)]
        ng = len(sc.GB)

        def timed(launch):
            for i in range(3 * n_views):
                launch(i % n_views)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(reps):
                launch(i % n_views)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        copy_ms = timed(lambda i: G.gs_copy_rows(h, sc.A, sc.GB[i % ng], lists[i], nvs[i]))
        mask_ms = timed(lambda i: G.gs_step(h, sc.A, sc.GB[i % ng], masks[i], P[i]))
        cam_ms = timed(lambda i: G.gs_step_camera(h, sc.A, sc.GB[i % ng], sc.CAMS[sc.order[i]], P[i]))
        G.gs_opt_destroy(h)
        nv = sum(nvs[i % n_views] for i in range(reps)) / reps
        row_bytes = 3 * 236 + STATE_RW["fp32"] + T_RW["fp32"] + 4       # + the list entry
        out[wname] = {"visible_rows_mean": nv, "copy_rows_ms": copy_ms,
                      "copy_rows_gbs": nv * row_bytes / copy_ms / 1e6,
                      "copy_rows_frac": nv * row_bytes / copy_ms / 1e6 / _peaks()[0],
                      "step_mask_ms": mask_ms, "step_camera_ms": cam_ms,
                      "step_over_copy": cam_ms / copy_ms}
        del sc, masks, lists
        torch.cuda.empty_cache()
    out["bytes"] = ("copy: 1664 B per listed row (attributes and moments read and written, gradients read, "
                    "t read and written, the list entry read)")
    return out


def next_rows_leg(G, synth, steps, warmup=10, aiu_prob=0.1):
    """The optional terms on the 1 M workload (FP32 moments), each timed as a
    whole run like the headline: the active count alone, position noise on
    the visible or on every primitive (App. Eq. disentangled_mu; eta_Ro 5e5,
    lambda_mu 100, lambda_t 0.005 as in 3DGS-MCMC), AIU with probability
    0.1 (Sec. 3.2), and gs_active_rows over 6 M logits.  Extra algorithmic
    bytes over the plain step: 4 B per invisible row for the count (its
    opacity), 44 B per invisible row for noise on every row (rotation,
    scale, opacity read, xyz written), and per AIU row its attributes read
    and written plus m, v and t read (948 B), counted at the expected number
    of AIU rows aiu_prob * (N - N_v)."""
    import torch
    wl = synth.WORKLOADS[WORKLOAD]
    sc = Scene(G, synth, wl, wl.seed, warmup + steps)
    na = torch.zeros(1, dtype=torch.int64, device="cuda")
    base = timed_run(G, sc, "fp32", steps, warmup)
    variants = {
        "active_count": (dict(n_active=na), 4, 0.0),
        "noise_visible": (dict(noise=1, n_active=na), 4, 0.0),
        "noise_all": (dict(noise=2, n_active=na), 4 + 44, 0.0),
        "aiu_p0.1": (dict(aiu=True, aiu_prob=aiu_prob, aiu_scale=1.0), 0, aiu_prob * 948),
    }
    out = {"workload": f"{wl.name}: {wl.n} Gaussians, fp32 moments, {steps} timed steps per variant",
           "plain": {"value": base["nv"] / base["elapsed"], "ms_per_step": base["elapsed"] / steps * 1e3,
                     "hbm_gbs": base["bytes_per_launch"] / base["step_s"] / 1e9}}
    for name, (extra, b_inv, b_aiu) in variants.items():
        r = timed_run(G, sc, "fp32", steps, warmup, extra=extra)
        inv = wl.n - r["nv"] / steps
        byt = r["bytes_per_launch"] + inv * (b_inv + b_aiu)
        gbs = byt / r["step_s"] / 1e9
        out[name] = {"value": r["nv"] / r["elapsed"], "ms_per_step": r["elapsed"] / steps * 1e3,
                     "hbm_gbs": gbs, "slowdown_vs_plain": r["step_s"] / base["step_s"],
                     # time per algorithmic byte against the plain step: the terms that read
                     # invisible rows (noise on every row, AIU) move more bytes per step
                     "slowdown_per_byte_vs_plain": out["plain"]["hbm_gbs"] / gbs}
    del sc
    torch.cuda.empty_cache()
    # prune list over 6 M logits
    n = 6_000_000
    gen = torch.Generator(device="cuda").manual_seed(1005)
    tau = torch.randn(n, generator=gen, device="cuda") * 2.0 - 4.0
    rows = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    h = G.gs_opt_init(G.make_config(), n)
    for _ in range(3):
        G.gs_active_rows(h, tau, rows, cnt)
    torch.cuda.synchronize()
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        G.gs_active_rows(h, tau, rows, cnt)
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / reps
    na_rows = int(cnt.item())
    # the standalone visibility filter over the 6 M scene's means: mask,
    # compacted visible list and count
    wl6 = synth.WORKLOADS["c5_6m"]
    xyz = torch.from_numpy(synth.scene_blobs(wl6.n, wl6.seed, wl6.extent)["xyz"]).cuda()
    cam = G.make_camera(wl6.cameras()[3])
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        G.gs_visibility(h, xyz, cam, mask, rows, cnt)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        G.gs_visibility(h, xyz, cam, mask, rows, cnt)
    e1.record()
    torch.cuda.synchronize()
    dv = e0.elapsed_time(e1) / 1e3 / reps
    nvis = int(cnt.item())
    G.gs_opt_destroy(h)
    out["active_rows_6m"] = {"ms": dt * 1e3, "n_active": na_rows,
                             "hbm_gbs": (4 * n + 4 * na_rows) / dt / 1e9,
                             "bytes": "4 B read per logit + 4 B written per active row (algorithmic)"}
    out["visibility_6m"] = {"ms": dv * 1e3, "n_visible": nvis, "hbm_gbs": (13 * n + 4 * nvis) / dv / 1e9,
                            "bytes": "12 B mean read + 1 B mask written per row, 4 B per visible row (algorithmic)"}
    return out


def density_sweep(G, synth, densities=(1.0, 0.6, 0.3, 0.1, 0.05), steps=200, warmup=20, prec="fp32"):
    """The plain step (moments in `prec`) on the 1 M scene with caller masks
    of random rows at each density: how the achieved bandwidth depends on how
    scattered the visible rows are.  Each density also reports the time per
    step, so formats compare directly."""
    import torch
    wl = synth.WORKLOADS[WORKLOAD]
    n = wl.n
    groups = synth.scene_blobs(n, wl.seed, wl.extent)
    attrs = {k: torch.from_numpy(v).cuda() for k, v in groups.items()}
    gen = torch.Generator(device="cuda").manual_seed(1)
    gb = [{nm: torch.randn((n, w), generator=gen, device="cuda") * 1e-3 for nm, w in synth.GROUPS} for _ in range(4)]
    A, GB = G.make_attrs(attrs), [G.make_attrs(g) for g in gb]
    h = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels, prec=PREC_ENUM[prec]), n)
    rng = np.random.default_rng(0)
    peak, _ = _peaks()
    out = {"workload": f"{wl.name} scene, random-row masks, {prec} moments, {steps} steps per density"}
    for dens in densities:
        masks = [torch.from_numpy((rng.random(n) < dens).astype(np.uint8)).cuda() for _ in range(4)]
        nvis = [int(m.sum().item()) for m in masks]
        P = [G.make_params(synth.lr_for_step(k, 1000), k) for k in range(1, warmup + steps + 1)]
        for i in range(warmup):
            G.gs_step(h, A, GB[i % 4], masks[i % 4], P[i])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(warmup, warmup + steps):
            G.gs_step(h, A, GB[i % 4], masks[i % 4], P[i])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        nv = sum(nvis[i % 4] for i in range(warmup, warmup + steps)) / steps
        gbs = (nv * (3 * 236 + STATE_RW[prec] + T_RW[prec]) + n) / ms / 1e6    # visible rows' bytes, mask
        out[str(dens)] = {"ms": ms, "hbm_gbs": gbs, "frac": gbs / peak}
    G.gs_opt_destroy(h)
    return out


# m, v and t of one row as the re-index moves them (B): hybrid (14 FP32 and 45
# BF16 columns per moment, t inside), FP16 block (59 FP16 values and 8
# exponent bytes per moment, uint16 t)
REINDEX_STATE = {"bf16_hybrid": 2 * (14 * 4 + 45 * 2) + 4, "fp16_block": 2 * (59 * 2 + 8) + 2}


def reindex_leg(G, synth, steps, precs=("fp16_block", "bf16_hybrid"), n_events=3):
    """The 6 M workload (about 10 % visible) with mixed-precision moments and a
    row-set change every 100 steps: prune 5 %, clone 5 % (fresh state),
    relocate 2 % (destination state reset).  Each event re-indexes the
    library's state (gs_reindex_state) and gathers the attributes into the
    second attribute buffer (gs_gather_attrs); both run inside the timed
    region.  The events' index arrays are resident on the device.  One run per
    moment format in `precs`, from the same scene."""
    import torch
    wl = synth.WORKLOADS["c5_6m"]
    warm = wl.restate_every                   # the first event (spare state allocation) is a warm-up
    sc = Scene(G, synth, wl, wl.seed, warm + steps)
    other = {k: torch.empty_like(v) for k, v in sc.attrs.items()}
    events = []
    for e in range(n_events):
        src, reset, attr_src = synth.reindex_event(wl.n, wl.seed, e)
        assert src.size == wl.n
        events.append(dict(src=torch.from_numpy(src).cuda(), reset=torch.from_numpy(reset).cuda(),
                           attr_src=torch.from_numpy(attr_src).cuda(),
                           n_copy=int(((src >= 0) & (reset == 0)).sum())))
    out = {}
    for prec in precs:
        sc.reset()
        bufs = [(sc.attrs, sc.A), (other, G.make_attrs(other))]
        state = REINDEX_STATE[prec]
        h = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels, prec=PREC_ENUM[prec]), wl.n)
        counts = torch.zeros(warm + steps, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        cur = [0]
        ev_pairs = []
        moved = [0.0]

        def step(i, timed):
            k = i + 1
            A = bufs[cur[0]][1]
            G.gs_step_camera(h, A, sc.GB[i % len(sc.GB)], sc.CAMS[sc.order[i]], sc.P[i],
                             n_visible=counts[i:i + 1], stream=stream)
            if k % wl.restate_every == 0:
                ev = events[(k // wl.restate_every) % n_events]
                if timed:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                G.gs_reindex_state(h, ev["src"], ev["reset"], wl.n, stream=stream)
                G.gs_gather_attrs(h, A, wl.n, bufs[1 - cur[0]][1], ev["attr_src"], wl.n, stream=stream)
                cur[0] = 1 - cur[0]
                if timed:
                    e1.record(stream)
                    ev_pairs.append((e0, e1))
                    moved[0] += ev["n_copy"] * state + wl.n * (state + 5) + wl.n * (2 * 236 + 4)

        for i in range(warm):
            step(i, False)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(warm, warm + steps):
            step(i, True)
        t1.record(stream)
        torch.cuda.synchronize()
        assert G.gs_opt_sync_errors(h) == 0
        G.gs_opt_destroy(h)
        if cur[0]:                            # leave the scene's attributes in their own buffer
            for k in sc.attrs:
                sc.attrs[k].copy_(other[k])
        elapsed = t0.elapsed_time(t1) / 1e3
        nv = int(counts[warm:].sum().item())
        re_s = sum(a.elapsed_time(b) for a, b in ev_pairs) / 1e3
        out[prec] = {"workload": f"{wl.name}: {wl.n} Gaussians, ~{nv / steps / wl.n:.0%} visible, {prec} moments, "
                                 f"re-index every {wl.restate_every} steps (prune 5 %, clone 5 %, relocate 2 %)",
                     "value": nv / elapsed, "unit": UNIT, "steps": steps, "ms_per_step": elapsed / steps * 1e3,
                     "events": len(ev_pairs), "reindex_ms_per_event": re_s / max(len(ev_pairs), 1) * 1e3,
                     "reindex_share_of_time": re_s / elapsed,
                     "reindex_gbs": moved[0] / re_s / 1e9 if re_s > 0 else None,
                     "reindex_bytes_per_event": moved[0] / max(len(ev_pairs), 1)}
    del sc
    torch.cuda.empty_cache()
    return out


def batched_leg(G, synth, steps, n_scenes=16, seed=1004, prec="fp32"):
    """16 independent scenes, primitive counts log-uniform in [50k, 2M] and
    blob extents log-uniform in [6, 75] (10-60 % visible), each with its own
    camera sequence and step counters: 16 separate FP32 launches per step vs
    one batched persistent launch (eager, and replayed as a CUDA graph)."""
    import torch
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(50_000), np.log(2_000_000), n_scenes)).astype(int)
    extents = np.exp(rng.uniform(np.log(6.0), np.log(75.0), n_scenes))
    scenes = []
    for s in range(n_scenes):
        groups = synth.scene_blobs(int(sizes[s]), seed + s, float(extents[s]))
        attrs = {k: torch.from_numpy(v).cuda() for k, v in groups.items()}
        gen = torch.Generator(device="cuda").manual_seed(seed + s)
        grads = {n: torch.randn((int(sizes[s]), w), generator=gen, device="cuda") * (1e-4 if n == "xyz" else 1e-3)
                 for n, w in synth.GROUPS}
        cams = synth.ring_cameras(40, (-30.0, -15.0, 0.0, 15.0, 30.0))
        order = synth.view_order(len(cams), 10_000, seed + s)
        scenes.append(dict(n=int(sizes[s]), attrs=attrs, grads=grads, A=G.make_attrs(attrs), GR=G.make_attrs(grads),
                           cams=[G.make_camera(c) for c in cams], order=order))
    total = int(sizes.sum())

    def params(k, s):
        return G.make_params(synth.lr_for_step(k, 10_000), k, restate=(k % 100 == 0), restate_ratio=0.1, seed=s)

    def timed(fn, nsteps, k0):
        counts = torch.zeros(n_scenes, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for j in range(nsteps):
            fn(k0 + j, counts)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, int(counts.sum().item())

    def tune_until_done(b, fn, k0):
        """Eager calls until the autotuner has timed every candidate, then 3 more."""
        k = k0
        while not G.gs_batch_config(b)["tuned"]:
            timed(fn, 1, k)
            k += 1
            if k - k0 > 200:
                raise RuntimeError("batched launch did not finish tuning")
        timed(fn, 3, k)

    res = {"workload": f"{n_scenes} scenes, {total} Gaussians in total (sizes log-uniform 50k-2M)",
           "sizes": sizes.tolist()}
    # 16 separate FP32 launches per step
    hs = [G.gs_opt_init(G.make_config(), sc["n"]) for sc in scenes]

    def sep(k, counts):
        for s, sc in enumerate(scenes):
            G.gs_step_camera(hs[s], sc["A"], sc["GR"], sc["cams"][sc["order"][k]], params(k, s),
                             n_visible=counts[s:s + 1])
    timed(sep, 5, 1)
    dt, nv = timed(sep, steps, 6)
    res["separate_launches"] = {"value": nv / dt, "ms_per_step": dt / steps * 1e3, "launches_per_step": n_scenes}
    # one batched launch per step (tuning happens over the first calls)
    b = G.gs_batch_create(hs)

    def bat(k, counts, graph=False):
        for s, sc in enumerate(scenes):
            b.set(s, sc["A"], sc["GR"], sc["cams"][sc["order"][k]], params(k, s))
        G.gs_batch_step(b, counts, graph=graph)
    tune_until_done(b, bat, 1000)
    dt, nv = timed(bat, steps, 2000)
    res["batched_persistent"] = {"value": nv / dt, "ms_per_step": dt / steps * 1e3, "launches_per_step": 1,
                                 "tuned": G.gs_batch_config(b)}
    timed(lambda k, c: bat(k, c, True), 3, 3000)
    dt, nv = timed(lambda k, c: bat(k, c, True), steps, 4000)
    res["batched_graph"] = {"value": nv / dt, "ms_per_step": dt / steps * 1e3, "launches_per_step": 1}
    res["speedup_batched_vs_separate"] = res["batched_persistent"]["value"] / res["separate_launches"]["value"]
    res["speedup_graph_vs_separate"] = res["batched_graph"]["value"] / res["separate_launches"]["value"]
    b.close()
    for h in hs:
        G.gs_opt_destroy(h)
    # the same batch with FP16-block moments (passes the 1e-3 gate), graph replay
    hs = [G.gs_opt_init(G.make_config(prec=PREC_ENUM["fp16_block"]), sc["n"]) for sc in scenes]
    b = G.gs_batch_create(hs)
    tune_until_done(b, bat, 5000)
    timed(lambda k, c: bat(k, c, True), 3, 6000)
    dt, nv = timed(lambda k, c: bat(k, c, True), steps, 7000)
    res["batched_graph_fp16_block"] = {"value": nv / dt, "ms_per_step": dt / steps * 1e3, "launches_per_step": 1,
                                       "tuned": G.gs_batch_config(b),
                                       "speedup_vs_separate_fp32": (nv / dt) / res["separate_launches"]["value"]}
    b.close()
    for h in hs:
        G.gs_opt_destroy(h)
    return res


def visibility_leg(G, synth, wl, n_views=40):
    """The GPU's frustum decisions on the headline scene against the FP64
    oracle (part of the oracle leg): for `n_views` of its views, the means
    within 1e-6 of a frustum plane, the decisions that differ from the
    oracle's, and those differing farther than 1e-6 from a plane (must be 0)."""
    import oracle
    import torch
    oracle.build()
    groups = synth.scene_blobs(wl.n, wl.seed, wl.extent)
    xyz = torch.from_numpy(groups["xyz"]).cuda()
    h = G.gs_opt_init(G.make_config(n_pixels=wl.n_pixels), wl.n)
    mask = torch.empty(wl.n, dtype=torch.uint8, device="cuda")
    cams = wl.cameras()
    near = differ = far = 0
    for c in cams[:n_views]:
        G.gs_visibility(h, xyz, G.make_camera(c), mask)
        got = mask.cpu().numpy()
        margin, ref = oracle.frustum_margin_f64(groups["xyz"], c)
        d = got != ref
        near += int((np.abs(margin) <= 1e-6).sum())
        differ += int(d.sum())
        far += int((d & (np.abs(margin) > 1e-6)).sum())
    G.gs_opt_destroy(h)
    return {"workload": f"{wl.name} means, {n_views} views x {wl.n} rows", "means_within_1e-6_of_a_plane": near,
            "decisions_differing_from_fp64": differ, "differing_beyond_1e-6": far}


class OracleSample:
    """The FP64 oracle (single-threaded C) on a bounded sample of the
    workload: the first `rows` primitives of the same scene, stepping through
    the same view schedule (visibility + step + RSR every 100 steps)."""

    def __init__(self, rows: int, workload: str = WORKLOAD, offset: int = 0):
        import oracle
        from paper_2601_16736_gb300 import synth
        oracle.build()
        self.oracle, self.synth = oracle, synth
        self.wl = wl = synth.WORKLOADS[workload]
        groups = (synth.scene_blobs(wl.n, wl.seed, wl.extent) if wl.scene == "blobs"
                  else synth.scene_uniform(wl.n, wl.seed))
        self.rows, self.offset = rows, offset
        self.ids = np.arange(offset, offset + rows, dtype=np.int64)     # global ids for the StSS draw
        self.st = oracle.State(synth.to_rows(groups)[offset:offset + rows])
        self.grads = [synth.grads_rows(rows, wl.seed + offset, b) for b in range(2)]
        self.cams = wl.cameras()
        self.order = synth.view_order(len(self.cams), 200_000, wl.seed)
        self.cfg = oracle.Config(n_i=oracle.dar_normaliser(wl.n_pixels))
        self.k = 0

    def step(self) -> int:
        o, wl = self.oracle, self.wl
        self.k += 1
        k = self.k
        cam = self.cams[self.order[k - 1]]
        mask = o.visibility(self.st.theta[:, 0:3].astype(np.float32), cam)
        o.step(self.cfg, self.st, self.grads[k % 2], mask, self.synth.lr_for_step(k, wl.steps), wl.dar, wl.dar, k)
        if k % wl.restate_every == 0:
            o.restate(self.cfg, self.st, wl.seed, k, wl.restate_ratio, row_ids=self.ids)
        return int(mask.sum())

    def describe(self, steps: int, seconds: float) -> str:
        return (f"primitives {self.offset}-{self.offset + self.rows - 1} of {self.wl.name}, {steps} steps in "
                f"{seconds:.1f} s, single-threaded FP64 C oracle")


def _oracle_shard(job):
    """One host core: the oracle on one row shard for `budget` seconds."""
    offset, rows, budget = job
    ob = OracleSample(rows, offset=offset)
    done, n, t0 = 0, 0, time.perf_counter()
    while time.perf_counter() - t0 < budget:
        done += ob.step()
        n += 1
    return done, n, time.perf_counter() - t0


def cpu_baseline(budget_s: float) -> dict:
    """The oracle on the host cores: one process per core (spawned), each
    stepping its own shard of the 1 M scene through the same view schedule;
    the rate is the sum of the shards' rates.  One core alone is reported
    beside it."""
    import multiprocessing as mp
    single = _oracle_shard((0, 100_000, budget_s))
    cores = max(1, os.cpu_count() or 1)
    n_rows = 1_000_000
    shard = n_rows // cores
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_shard, [(i * shard, shard, budget_s) for i in range(cores)])
    value = sum(d / t for d, _, t in res)
    steps = min(n for _, n, _ in res)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each the single-threaded FP64 C oracle on {shard} primitives of "
                      f"{WORKLOAD} (together all {shard * cores}), {budget_s:.0f} s each, at least {steps} steps",
            "single_core": {"value": single[0] / single[2], "cores": 1,
                            "sample": f"primitives 0-99999 of {WORKLOAD}, {single[1]} steps in {single[2]:.1f} s"}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    # about 30 ms per oracle step at 100 000 rows: size the sample so the
    # whole run stays near two minutes
    per_step_100k, budget = 0.03, 120.0
    rows = int(min(100_000, max(2_000, 100_000 * budget / (per_step_100k * (args.steps + args.warmup)))))
    ob = OracleSample(rows)
    for _ in range(args.warmup):
        ob.step()
    done, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        done += ob.step()
    dt = time.perf_counter() - t0
    value = done / dt
    cb = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": ob.describe(args.steps, dt)}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD}: bounded sample of {rows} primitives on the host cores"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--prec", choices=list(PREC_ENUM), default="fp32")
    ap.add_argument("--e2e-steps", type=int, default=None, help="default: --steps")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--mixed-steps", type=int, default=300)
    ap.add_argument("--no-mixed-error", dest="mixed_error", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-reindex", dest="reindex", action="store_false")
    ap.add_argument("--no-next-rows", dest="next_rows", action="store_false")
    ap.add_argument("--no-ceiling", dest="ceiling", action="store_false")
    ap.add_argument("--density-sweep", action="store_true",
                    help="only time the plain step at several visible densities (random-row masks)")
    ap.add_argument("--next-steps", type=int, default=300)
    ap.add_argument("--reindex-steps", type=int, default=1000)
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the blob-sorted row order and the 100 k (L2-resident) legs")
    ap.add_argument("--no-visibility-band", dest="visibility_band", action="store_false")
    ap.add_argument("--only", choices=["mixed", "batched", "reindex", "next_rows", "ceiling"], default=None,
                    help="run the headline and this one leg only (for profiling)")
    ap.add_argument("--grad-buffers", type=int, default=None,
                    help="gradient buffers per scene (default: the workload's pool); fewer keeps profiled runs small")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only:
        for leg in ("mixed", "batched", "reindex", "next_rows", "ceiling", "secondary", "cpu_baseline"):
            setattr(args, leg, leg == args.only)
        args.e2e_steps = 0
    if args.impl == "reference":
        run_reference(args)
    elif args.density_sweep:
        from paper_2601_16736_gb300 import build as B
        B.build()
        from paper_2601_16736_gb300 import gsopt as G
        from paper_2601_16736_gb300 import synth
        print(json.dumps({"density_sweep": density_sweep(G, synth, prec=args.prec)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
