"""Benchmark of the Kirchhoff migration hot path (Eq. 1) on GB300.

One step = one full migration call through the C ABI: offset binning and sort of the
traces, then the migration kernel over every (image tile, offset bin).  The metric is
G image-point x trace contributions per second (Eq. 2: one contribution is one image point
and one in-aperture trace; the count is exact, computed on the device).

Default workload: 3D survey with v(z) = 1500 + 0.5 z (analytic linear-gradient
traveltimes), 100 000 traces x 1500 FP32 samples at 4 ms, 256^3 image at 12.5 m, 16 offset
bins of 100 m, 2 km aperture, obliquity x spreading weight.  Synthetic data: 20 Hz Ricker
reflections from 4 seeded dipping planes (sheets of point scatterers every 100 m) and 40
diffractors, arrival times from the library's traveltime kernel.

Workload ``batch64-3d-vz``: 64 independent 3D v(z) migrations of uneven size (per job,
seeded: n^3 image with n ~ U{64..192}, 1k-50k traces, 750-2000 samples), tiles chosen by the
autotuner, run as one graph-captured persistent launch; the line also reports a loop of
per-job kirchhoff_migrate calls on the same stream with the same tiles.

``--trace-dtype f16|bf16`` stores the traces in 16 bits (FP32 arithmetic).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (bounded
samples of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1204_1225_gb300 import survey as sv  # noqa: E402

# ALU roofline (GB300): thread instructions each SM can issue or execute per clock, per pipe
# (dispatch: 4 sub-partitions x 32 lanes; FP32 FMA pipe 128; integer/logic ALU 64; MUFU
# special-function unit 16, the rate a throughput probe of back-to-back MUFU instructions
# measured on this GPU; shared-memory load/store unit 32).  The migration kernel is a gather
# with no HBM bound (about 1.1e-3 algorithmic bytes per contribution: traces and image once), so
# its roofline is the smallest of N_SM x clock x lanes_p / n_p over these pipes, n_p = the
# kernel's executed thread instructions per contribution on pipe p (ncu
# sm__inst_executed_pipe_*.sum x 32 and smsp__thread_inst_executed.sum, divided by the
# contribution count of the captured launch).
N_SM = 152
LANES_PER_SM_CLK = {"issue": 128, "fma": 128, "alu": 64, "xu": 16, "lsu": 32}
# n_p per workload's kernel variant, from one ncu capture of the kernel per variant (the
# 100k-trace 256^3 workload runs the variant measured on its 10k-trace case: same grid, tile
# and 5-term per-leg fit).
PIPE_MIX = {
    "3d-vz-100k-256cube": {"issue": 33.30, "fma": 21.37, "alu": 3.77, "xu": 3.15, "lsu": 3.37},
    "3d-vz-10k-256cube": {"issue": 33.30, "fma": 21.37, "alu": 3.77, "xu": 3.15, "lsu": 3.37},
    "3d-vz-40k-128cube": {"issue": 34.71, "fma": 22.81, "alu": 3.68, "xu": 3.20, "lsu": 3.42},
    "25d-vz-20k-512x400": {"issue": 36.09, "fma": 23.96, "alu": 4.25, "xu": 2.37, "lsu": 3.75},
    # gridded v(x, z): per-location first-arrival tables read from L2 (k_migrate<grid, one, fast, sample pairs, M=4>)
    "25d-vxz-20k-512x400": {"issue": 20.63, "fma": 11.31, "alu": 3.82, "xu": 0.004, "lsu": 3.31},
    # mixed precision: 16-bit radial tables + FP16 traces (k_migrate<table, obliquity, FP16, M=2, table type>)
    "3d-vz-100k-256cube-table-u16-f16": {"issue": 30.67, "fma": 16.37, "alu": 5.16, "xu": 2.20, "lsu": 5.40},
    "3d-vz-10k-256cube-table-u16-f16": {"issue": 30.67, "fma": 16.37, "alu": 5.16, "xu": 2.20, "lsu": 5.40},
    "3d-vz-100k-256cube-table-f16-f16": {"issue": 33.10, "fma": 19.69, "alu": 4.07, "xu": 2.20, "lsu": 5.53},
    "3d-vz-10k-256cube-table-f16-f16": {"issue": 33.10, "fma": 19.69, "alu": 4.07, "xu": 2.20, "lsu": 5.53},
    # adjoint (k_demigrate) and gradient (k_vgrad), headline variants measured on the 10k case
    "3d-vz-100k-256cube-demigrate": {"issue": 68.11, "fma": 32.78, "alu": 12.33, "xu": 3.98, "lsu": 10.36},
    "3d-vz-10k-256cube-demigrate": {"issue": 68.11, "fma": 32.78, "alu": 12.33, "xu": 3.98, "lsu": 10.36},
    "3d-vz-100k-256cube-vgrad": {"issue": 54.58, "fma": 34.94, "alu": 8.32, "xu": 3.15, "lsu": 5.49},
    "3d-vz-10k-256cube-vgrad": {"issue": 54.58, "fma": 34.94, "alu": 8.32, "xu": 3.15, "lsu": 5.49},
    # prestack time migration (k_migrate<time migration, obliquity, fast, sample pairs>)
    "3d-pstm-100k-256cube": {"issue": 23.43, "fma": 13.39, "alu": 3.19, "xu": 2.08, "lsu": 3.36},
    "3d-pstm-10k-256cube": {"issue": 23.43, "fma": 13.39, "alu": 3.19, "xu": 2.08, "lsu": 3.36},
    # true-amplitude weight, constant velocity (k_migrate<const, true amplitude, fast, sample pairs>,
    # tile-relative legs, source leg cached), measured on the 10k-trace case
    "3d-ta-100k-256cube": {"issue": 33.17, "fma": 17.81, "alu": 6.05, "xu": 4.15, "lsu": 3.36},
    "3d-ta-10k-256cube": {"issue": 33.17, "fma": 17.81, "alu": 6.05, "xu": 4.15, "lsu": 3.36},
    # the same with operator anti-aliasing (25 m spacing): per in-aperture pair, including the pairs
    # whose weight the warp's bounds prove 0 and that are skipped
    "3d-ta-aa-100k-256cube": {"issue": 19.03, "fma": 8.82, "alu": 5.03, "xu": 1.61, "lsu": 0.88},
    "3d-ta-aa-10k-256cube": {"issue": 19.03, "fma": 8.82, "alu": 5.03, "xu": 1.61, "lsu": 0.88},
    # the headline survey with operator anti-aliasing (25 m spacing), per in-aperture pair
    "3d-vz-aa-100k-256cube": {"issue": 24.51, "fma": 13.66, "alu": 5.21, "xu": 1.78, "lsu": 1.19},
    "3d-vz-aa-10k-256cube": {"issue": 24.51, "fma": 13.66, "alu": 5.21, "xu": 1.78, "lsu": 1.19},
    # persistent batched kernel, constant velocity, sample pairs (measured on the 8-job small batch)
    "batch64-3d-vz-f32": {"issue": 23.35, "fma": 13.83, "alu": 3.46, "xu": 2.38, "lsu": 2.54},
}


# DRAM bytes (read + write) of one launch of the variant's main kernel, ncu
# dram__bytes_{read,write}.sum from the same captures (10k-trace cases); None where not captured.
TRAFFIC = {
    "3d-vz-10k-256cube": 86816256 + 1025687552,
    "3d-vz-40k-128cube": 281054208 + 111904000,
    "25d-vz-20k-512x400": 91543808 + 2981376,
    "25d-vxz-20k-512x400": 138770944 + 5204480,
    "3d-vz-10k-256cube-demigrate": 5606103296 + 8223564800,
    "3d-vz-10k-256cube-vgrad": 1127874560 + 15597568,
    "3d-vz-10k-256cube-table-u16-f16": 37533696 + 1023990784,
    "3d-vz-10k-256cube-table-f16-f16": 35020800 + 1024065536,
    "3d-pstm-10k-256cube": 87162880 + 1023754240,
    "3d-ta-10k-256cube": 93872128 + 1025078272,
    "3d-ta-aa-10k-256cube": 96422400 + 1025947136,
    "3d-vz-aa-10k-256cube": 89446400 + 1035280384,
}

# Parity bars against the FP64 oracle (relative L2 over the sampled outputs): FP32 forms, and the
# mixed-precision form (16-bit traces and traveltime table, FP32 arithmetic).
BAR_FP32 = 1e-5
BAR_MIXED = 3e-3
# The velocity gradient is a sum of signed terms that cancel; its bar is relative to the sum of
# their absolute values (the FP32 rounding of the individual terms).
BAR_GRAD_ABS = 1e-4


# The velocity model and weight each workload is defined with (the kernel variant its mix is of).
WORKLOAD_MODEL = {
    "3d-vz-100k-256cube": ("linear", "obliq"),
    "3d-vz-40k-128cube": ("linear", "obliq"),
    "3d-vz-10k-256cube": ("linear", "obliq"),
    "25d-vz-20k-512x400": ("linear", "one"),
    "3d-ta-100k-256cube": ("const", "ta"),
    "3d-ta-10k-256cube": ("const", "ta"),
    "3d-ta-aa-100k-256cube": ("const", "ta"),
    "3d-ta-aa-10k-256cube": ("const", "ta"),
    "3d-vz-aa-100k-256cube": ("linear", "obliq"),
    "3d-vz-aa-10k-256cube": ("linear", "obliq"),
}


def pipe_roofline(mix, clk_mhz: float):
    """(bound name, contributions/s bound in G/s, all pipe bounds) for an instruction mix."""
    bounds = {p: N_SM * LANES_PER_SM_CLK[p] * clk_mhz * 1e6 / n / 1e9 for p, n in mix.items()}
    p = min(bounds, key=bounds.get)
    return p, bounds[p], bounds


def workloads():
    return {
        "3d-vz-100k-256cube": lambda: sv.survey_3d_gradient(),
        "3d-vz-40k-128cube": lambda: sv.survey_3d_gradient(ntr=40_000, n=128),
        "3d-vz-10k-256cube": lambda: sv.survey_3d_gradient(ntr=10_000, n=256),
        "2d-const-1024tr-128x128": lambda: sv.survey_2d_const(),
        "25d-vz-20k-512x400": lambda: sv.survey_25d_lsm(),
        "25d-vxz-20k-512x400": lambda: sv.survey_25d_vxz(),
        "3d-ta-100k-256cube": lambda: sv.survey_3d_gradient().replace(
            vel="const", v0=2000.0, k=0.0, weight="ta", name="3d-const2000-ta-100000tr-256cube"),
        "3d-ta-10k-256cube": lambda: sv.survey_3d_gradient(ntr=10_000, n=256).replace(
            vel="const", v0=2000.0, k=0.0, weight="ta", name="3d-const2000-ta-10000tr-256cube"),
        # the same with operator anti-aliasing for the 25 m receiver spacing
        "3d-ta-aa-100k-256cube": lambda: sv.survey_3d_gradient().replace(
            vel="const", v0=2000.0, k=0.0, weight="ta", aa_spacing=25.0, name="3d-const2000-ta-aa25-100000tr-256cube"),
        "3d-ta-aa-10k-256cube": lambda: sv.survey_3d_gradient(ntr=10_000, n=256).replace(
            vel="const", v0=2000.0, k=0.0, weight="ta", aa_spacing=25.0, name="3d-const2000-ta-aa25-10000tr-256cube"),
        # the headline survey with operator anti-aliasing for the 25 m receiver spacing
        "3d-vz-aa-100k-256cube": lambda: sv.survey_3d_gradient().replace(
            aa_spacing=25.0, name="3d-vz-aa25-100000tr-256cube"),
        "3d-vz-aa-10k-256cube": lambda: sv.survey_3d_gradient(ntr=10_000, n=256).replace(
            aa_spacing=25.0, name="3d-vz-aa25-10000tr-256cube"),
        "25d-velan-4608tr-128x100": lambda: sv.survey_25d_velan(),
        "3d-pstm-100k-256cube": lambda: sv.survey_3d_gradient().replace(
            vel="pstm", oz=0.0, dz=0.012, name="3d-pstm-100000tr-256x256x256t"),
        "3d-pstm-10k-256cube": lambda: sv.survey_3d_gradient(ntr=10_000, n=256).replace(
            vel="pstm", oz=0.0, dz=0.012, name="3d-pstm-10000tr-256x256x256t"),
        "batch64-3d-vz": lambda: sv.survey_batch_3d(64),
        "batch8-3d-vz-small": lambda: sv.survey_batch_3d(8, n_range=(64, 96), ntr_range=(1000, 5000)),
    }


_TDT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def sum_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        ident = str(self.dev)
        try:
            uuid = torch.cuda.get_device_properties(self.dev).uuid
            ident = "GPU-" + str(uuid)
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            if vis:
                ident = vis.split(",")[self.dev]
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", ident, "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def synth_traces(s, plan, device):
    from paper_1204_1225_gb300 import kirchhoff as kh
    rng = np.random.default_rng(sv.BASE_SEED)
    if s.dim == 3:
        if s.vel == "pstm":   # the time image: depth scatterers, depths read as two-way times (1 km/s)
            sc = sv.reflectors_3d(rng, s.replace(vel="linear", oz=0.0, dz=12.5), spacing=100.0)
            sc[:, 2] *= 1e-3
        else:
            sc = sv.reflectors_3d(rng, s, spacing=100.0)
        freq = 20.0
    else:
        sc = sv.point_scatterers_2d(rng, xr=(0.1 * s.nx * s.dx, 0.9 * s.nx * s.dx),
                                    zr=(0.2 * s.nz * s.dz, 0.9 * s.nz * s.dz))
        freq = 25.0
    return sv.synthesize(s, sc, kh.arrival_times_fn(plan), freq, noise_sigma=0.0,
                         device=device, chunk=1 << 23)


def synth_batch_job(s, plan, j: int, device):
    """Job j of the batch: 25 Hz Ricker arrivals from 3 seeded point scatterers inside the
    job's volume (amplitude 1) plus white noise of sigma 0.1 drawn on the device."""
    from paper_1204_1225_gb300 import kirchhoff as kh
    rng = np.random.default_rng(sv.BASE_SEED + 1000 + j)
    w = s.nx * s.dx
    sc = np.stack([rng.uniform(0.1 * w, 0.9 * w, 3), rng.uniform(0.1 * w, 0.9 * w, 3),
                   rng.uniform(0.2 * w, 0.9 * w, 3), np.ones(3)], axis=1)
    d = sv.synthesize(s, sc, kh.arrival_times_fn(plan), 25.0, noise_sigma=0.0, device=device,
                      chunk=1 << 23)
    g = torch.Generator(device=device).manual_seed(sv.BASE_SEED + j)
    return d.add_(torch.randn(d.shape, generator=g, device=device), alpha=0.1)


def cpu_baseline(s, traces_cpu, target_s: float, seed: int):
    """The FP64 oracle on a bounded sample of image points of the same workload."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    d64 = traces_cpu
    probe = sv.sample_points(s, 64, seed)
    t0 = time.perf_counter()
    oracle.migrate_points(s, d64, probe)
    t_probe = max(time.perf_counter() - t0, 1e-3)
    n = int(min(max(64, 64 * target_s / t_probe), np.prod(s.image_shape)))
    pts = sv.sample_points(s, n, seed + 1)
    t0 = time.perf_counter()
    _, ncontrib = oracle.migrate_points(s, d64, pts, return_count=True)
    el = time.perf_counter() - t0
    return {"value": ncontrib / el / 1e9, "unit": "Gcontrib/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} random image samples of {s.name} (all bins), {ncontrib} contributions, "
                      f"FP64 brute force, {el:.1f} s"}


def run_reference(args, s):
    """Reference arm: the FP64 CPU oracle, each step a bounded sample of the workload."""
    import oracle
    oracle.build()
    rng_traces = sv.random_traces(s, sv.BASE_SEED, smooth=0) if s.ntr * s.nt < 2e8 else None
    if rng_traces is None:
        rng_traces = np.random.default_rng(sv.BASE_SEED).standard_normal((s.ntr, s.nt)).astype(np.float32)
    d64 = rng_traces.astype(np.float64)
    del rng_traces
    probe = sv.sample_points(s, 32, 7)
    t0 = time.perf_counter()
    oracle.migrate_points(s, d64, probe)
    t_probe = max(time.perf_counter() - t0, 1e-3)
    per_step = float(os.environ.get("KH_REF_STEP_S", "8"))
    n = int(min(max(32, 32 * per_step / t_probe), np.prod(s.image_shape)))
    for w in range(args.warmup):
        oracle.migrate_points(s, d64, sv.sample_points(s, max(8, n // 8), 100 + w))
    tot_c, tot_t = 0, 0.0
    for k in range(args.steps):
        pts = sv.sample_points(s, n, 1000 + k)
        t0 = time.perf_counter()
        _, c = oracle.migrate_points(s, d64, pts, return_count=True)
        tot_t += time.perf_counter() - t0
        tot_c += c
    v = tot_c / tot_t / 1e9
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": "G image-point x trace contributions/s", "value": v,
            "unit": "Gcontrib/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": s.name, "sample_points_per_step": n},
            "cpu_baseline": {"value": v, "unit": "Gcontrib/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} random image samples per step of {s.name}"},
            "e2e": {"value": v, "unit": "Gcontrib/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d-vz-100k-256cube", choices=sorted(workloads()))
    ap.add_argument("--fast-math", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--trace-dtype", default="f32", choices=sorted(_TDT))
    ap.add_argument("--vel", default="analytic", choices=["analytic", "table"],
                    help="traveltimes: analytic v(z) formulas or the radial traveltime table")
    ap.add_argument("--table-dtype", default="u16", choices=["f32", "f16", "u16"])
    ap.add_argument("--no-tune", action="store_true", help="batch: default tiles, no autotuning")
    ap.add_argument("--tile-cache", default=None, help="batch: autotuner JSON cache path")
    ap.add_argument("--no-loop", action="store_true", help="batch: skip the per-job loop arm")
    ap.add_argument("--batch-mode", default="concurrent", choices=["persistent", "concurrent"],
                    help="batch: one persistent kernel, or each job's kernel on forked streams")
    ap.add_argument("--op", default="migrate", choices=["migrate", "demigrate", "vgrad", "cgls", "velan"],
                    help="operator timed: migration (Eq. 1), its adjoint, the (v0, k) gradient, a "
                         "least-squares migration (CGLS, --cg-iters iterations) per step, or a velocity "
                         "analysis (BFGS on the offset images' semblance, from a perturbed model) per step")
    ap.add_argument("--cg-iters", type=int, default=20, help="CGLS iterations of one --op cgls step")
    ap.add_argument("--aperture", type=float, default=None,
                    help="override the workload's aperture (metres)")
    ap.add_argument("--spatial-sort", type=int, default=1,
                    help="1: traces sorted by (bin, midpoint cell), each CTA examines the cells of "
                         "its aperture disc; 0: each CTA examines its whole bin")
    ap.add_argument("--forms", type=int, default=None,
                    help="1: add the other forms of the metric to the headline line (mixed precision, "
                         "batched vs loop, adjoint, gradient), each timed on its own; default: on for "
                         "the headline migration, off otherwise")
    ap.add_argument("--form-steps", type=int, default=3, help="timed steps of each added form")
    ap.add_argument("--parallelism", default="replicas", choices=["replicas", "image"],
                    help="N > 1: every rank migrates the whole workload (replicas, weak scaling), or "
                         "rank r migrates its slab of image columns with every trace (image, strong "
                         "scaling: the N slabs make the one image; no exchange of partial sums)")
    ap.add_argument("--parity-points", type=int, default=4096,
                    help="image samples compared with the FP64 oracle (0: no parity check)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    return args


def main():
    args = parse_args()
    ws, rank, local = dist_init()
    s = workloads()[args.workload]()
    if args.aperture is not None and not isinstance(s, list):
        s = s.replace(aperture=args.aperture, name=f"{s.name}-A{args.aperture:g}")
    args.image_partition = args.parallelism == "image" and ws > 1 and not isinstance(s, list)
    if args.image_partition:
        from paper_1204_1225_gb300 import partition
        s = partition.slab_survey(s, *partition.image_slabs(s, ws)[rank])
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, s[0] if isinstance(s, list) else s)
        return
    from paper_1204_1225_gb300 import build as khbuild
    khbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if isinstance(s, list):
        line = run_batched(args, s, ws, rank, local, dev)
    elif args.op == "cgls":
        line = run_cgls(args, s, ws, rank, local, dev)
    elif args.op == "velan":
        line = run_velan(args, s, ws, rank, local, dev)
    else:
        cache = {}
        line = run_single(args, s, ws, rank, local, dev, cache)
        headline = (args.workload == "3d-vz-100k-256cube" and args.op == "migrate" and args.vel == "analytic"
                    and args.trace_dtype == "f32" and args.aperture is None and args.spatial_sort
                    and not args.image_partition)
        forms = run_forms(args, s, ws, rank, local, dev, cache, line) \
            if (args.forms if args.forms is not None else headline) else None
        if line is not None and forms is not None:
            line["forms"] = forms
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


def _oracle():
    import oracle
    oracle.build()
    return oracle


def parity_image(s_oracle, traces64, image, npts, bar, what):
    """The GPU image at `npts` random samples against the FP64 oracle at the same samples."""
    if npts <= 0:
        return None
    oracle = _oracle()
    pts = sv.sample_points(s_oracle, npts, sv.BASE_SEED + 17)
    got = image.reshape(-1)[torch.as_tensor(pts, device=image.device)].double().cpu().numpy()
    t0 = time.perf_counter()
    want = oracle.migrate_points(s_oracle, traces64, pts)
    err = float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))
    return {"rel_l2": err, "bar": bar, "within_bar": (err <= bar) if bar else None,
            "points": int(pts.size), "vs": what, "oracle_s": round(time.perf_counter() - t0, 2)}


def run_single(args, s, ws, rank, local, dev, cache, *, op=None, trace_dtype=None, vel=None,
               table_dtype=None, steps=None, warmup=None, e2e=None, cpu=None, spatial_sort=None):
    """Times `steps` calls of one operator on one survey; returns the JSON line (rank 0)."""
    from paper_1204_1225_gb300 import kirchhoff as kh
    op = op or args.op
    trace_dtype = trace_dtype or args.trace_dtype
    vel = vel or args.vel
    table_dtype = table_dtype or args.table_dtype
    steps = steps or args.steps
    warmup = warmup or args.warmup
    e2e = (not args.no_e2e) if e2e is None else e2e
    cpu = (not args.no_cpu_baseline) if cpu is None else cpu
    spatial_sort = bool(args.spatial_sort) if spatial_sort is None else spatial_sort
    tdt = _TDT[trace_dtype]
    s_run = s.replace(vel="table") if vel == "table" else s
    grid_rec = None
    if s.vel == "grid":
        # gridded model: the per-location first-arrival tables are built once per model (timed
        # here on their own); the steps migrate with them
        plan = kh.Plan(s_run.replace(grid_v=None), fast_math=bool(args.fast_math), trace_dtype=tdt)
        grid_rec = time_grid_tables(plan, s, dev)
    else:
        plan = kh.Plan(s_run, fast_math=bool(args.fast_math), trace_dtype=tdt, table_dtype=table_dtype)
    plan.set_spatial_sort(spatial_sort)
    if "hdr" not in cache:
        cache["hdr"] = kh.Headers.of(s, device=dev)
        s_syn = s.replace(vel="linear", grid_v=None) if s.vel == "grid" else s   # data content: background model
        cache["traces"] = synth_traces(s_syn, kh.Plan(s_syn), dev).contiguous()
        cache["count"] = plan.count(cache["hdr"])
    hdr = cache["hdr"]
    traces = cache["traces"].to(tdt).contiguous()
    image = torch.empty(plan.image_shape, dtype=torch.float32, device=dev)
    contrib = cache["count"]
    stream = torch.cuda.current_stream(dev)
    if op != "migrate":
        if "image" not in cache:
            cache["image"] = torch.empty(plan.image_shape, dtype=torch.float32, device=dev)
            kh.Plan(s).migrate(hdr, cache["traces"], out=cache["image"])   # the adjoint and gradient read an image
        image = cache["image"]
        d_out = torch.empty((s.ntr, s.nt), dtype=torch.float32, device=dev)
        g_out = torch.empty(2, dtype=torch.float64, device=dev)

    def step():
        if op == "migrate":
            plan.migrate(hdr, traces, out=image)
        elif op == "demigrate":
            plan.demigrate(hdr, image, out=d_out)
        else:
            plan.velocity_grad(hdr, image, traces, out=g_out)

    for _ in range(warmup):
        step()
    plan.sync()
    plan.profile(True)
    plan.profile_read()
    plan.staging_stats()
    launches0 = plan.launches
    barrier(ws)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    plan.sync()
    launches = plan.launches - launches0
    kern_ms, kern_n = plan.profile_read()
    stage_stats = plan.staging_stats()
    plan.profile(False)
    t_ms = max_over_ranks(ws, e0.elapsed_time(e1))
    barrier(ws)
    # replicas: every rank did the whole workload; image partition: the ranks' slabs make one image
    image_part = getattr(args, "image_partition", False)
    units = sum_over_ranks(ws, contrib) if image_part else contrib * ws
    value = units * steps / (t_ms / 1e3) / 1e9
    clocks = clk.summary()

    # end to end through the public API: pinned host inputs in, image back to pinned host, every
    # step (kirchhoff_migrate_host: one step's copies overlap the next or previous step's migration)
    e2e_rec = None
    if e2e and op == "migrate":
        h_tr = traces.cpu().pin_memory()
        h_hdr = [t.cpu().pin_memory() for t in hdr.args()]
        h_img = torch.empty(plan.image_shape, dtype=torch.float32).pin_memory()
        h2d = h_tr.numel() * h_tr.element_size() + sum(t.numel() * 4 for t in h_hdr)
        d2h = h_img.numel() * 4
        for _ in range(2):   # the host slots' device buffers are allocated by the first calls
            plan.migrate_host(h_hdr, h_tr, h_img)
        plan.host_join(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
        with ClockSampler(local) as eclk:
            e0.record(stream)
            for _ in range(steps):
                plan.migrate_host(h_hdr, h_tr, h_img)
            plan.host_join(stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        plan.sync()
        te = max_over_ranks(ws, e0.elapsed_time(e1))
        e2e_rec = {"value": units * steps / (te / 1e3) / 1e9, "unit": "Gcontrib/s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "ms_per_step": te / steps, "clocks": eclk.summary(),
                   "api": "Plan.migrate_host (kirchhoff_migrate_host), pinned host buffers"}
        del h_tr, h_img

    if rank != 0:
        return None
    # pipe roofline of the main kernel at the median SM clock of the timed region
    clk_mhz = clocks.get("sm_mhz") or 2070.0
    achieved = contrib / (kern_ms / max(kern_n, 1) / 1e3) / 1e9 if kern_n else None
    kname = {"migrate": "k_migrate", "demigrate": "k_demigrate", "vgrad": "k_vgrad"}[op]
    workload = args.workload.replace("3d-vz", "3d-pstm") if s.vel == "pstm" else args.workload
    if vel == "table":
        mix_key = f"{workload}-table-{table_dtype}-{trace_dtype}"
    elif trace_dtype == "f32":
        mix_key = workload if op == "migrate" else f"{workload}-{op}"
    else:
        mix_key = None
    if args.aperture is not None or not spatial_sort:
        mix_key = None   # instruction mixes were measured on the workloads as defined
    if s.vel in ("const", "linear") and (s.vel, s.weight) != (WORKLOAD_MODEL.get(args.workload) or (s.vel, s.weight)):
        mix_key = None   # another velocity model or weight than the workload's own: another kernel
    mix = PIPE_MIX.get(mix_key) if (mix_key and args.fast_math) else None
    roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "unit": "Gcontrib/s",
            "kernel_ms_per_launch": kern_ms / max(kern_n, 1)}
    if mix:
        pipe, peak, bounds = pipe_roofline(mix, clk_mhz)
        roof.update({"peak": peak, "frac": (achieved / peak) if achieved else None,
                     "binding_pipe": pipe, "pipe_bounds": {k: round(v, 1) for k, v in bounds.items()},
                     "instructions_per_contribution": mix,
                     "peak_basis": f"min over pipes of {N_SM} SMs x lanes/clk x {clk_mhz:.0f} MHz / "
                                   f"executed instructions per contribution (ncu instruction mix of "
                                   f"{kname} on this variant)"})
    else:
        roof.update({"peak": None, "frac": None,
                     "peak_basis": "no measured instruction mix for this kernel variant"})
    roof["traffic"] = TRAFFIC.get(mix_key) if mix_key else None

    # parity with the FP64 oracle on sampled outputs of this very launch configuration
    parity = None
    npts = args.parity_points
    if npts > 0:
        if "traces64" not in cache:
            cache["traces64"] = cache["traces"].double().cpu().numpy()
        if op == "migrate" and vel == "table":
            parity = parity_image(s.replace(vel="table"), cache["traces64"], image, npts, BAR_MIXED,
                                  "FP64 oracle, same radial-table algorithm, on the FP32 traces "
                                  "(storage error of the 16-bit traces and table included)")
            parity["vs_exact_traveltimes"] = parity_image(s, cache["traces64"], image, npts, None,
                                                          "FP64 oracle, exact closed-form T")["rel_l2"]
        elif op == "migrate":
            bar = BAR_FP32 if trace_dtype == "f32" else BAR_MIXED
            parity = parity_image(s, cache["traces64"], image, npts, bar,
                                  "FP64 oracle on the FP32 traces" + (" (16-bit storage error included)"
                                                                      if trace_dtype != "f32" else ""))
        elif op == "demigrate":
            parity = parity_demigrate(s, image, d_out)
        else:
            parity = parity_vgrad(s, dev, cache)
    cpu_rec = None
    if cpu and ws == 1 and op == "migrate":
        if "traces64" not in cache:
            cache["traces64"] = cache["traces"].double().cpu().numpy()
        cpu_rec = cpu_baseline(s, cache["traces64"], args.cpu_seconds, sv.BASE_SEED)
    tbytes = traces.numel() * traces.element_size()
    return {
        "metric": "G image-point x trace contributions/s", "value": value, "unit": "Gcontrib/s",
        "n_gpus": ws, "steps": steps, "warmup": warmup,
        "ms_per_step": t_ms / steps, "higher_is_better": True, "scaling": "strong" if image_part else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": s.name, "operator": op, "image": list(plan.image_shape),
                   "ntr": s.ntr, "nt": s.nt,
                   "velocity": (f"{s.vel} v0={s.v0} k={s.k}" if s.vel != "grid" else
                                f"gridded v(x, z) on {s.grid_v.shape[0]}x{s.grid_v.shape[1]} nodes of "
                                f"{s.grid_h:g} m (v0 + k z = {s.v0} + {s.k} z with a low-velocity lens)"),
                   "weight": s.weight, "aa_spacing_m": float(getattr(s, "aa_spacing", 0.0)),
                   "aperture_m": s.aperture, "contributions_per_step": contrib,
                   "fast_math": bool(args.fast_math), "trace_storage": trace_dtype,
                   "traveltimes": ("per-location first-arrival tables (FP64 eikonal, FP32 storage)"
                                   if s.vel == "grid" else "analytic" if vel == "analytic" else
                                   f"table ({table_dtype}, {s.table_spacing:g} m)"),
                   "eikonal_tables": grid_rec,
                   "l2": "inputs larger than L2 (traces %.0f MB, image %.0f MB)" % (
                       tbytes / 1e6, image.numel() * 4 / 1e6),
                   "parallelism": (f"image slabs x{ws} (rank 0's slab shown)" if image_part else
                                   "replicas" if ws > 1 else "single"),
                   "trace_order": _trace_order(plan, spatial_sort),
                   "staging_per_cta": _staging(*stage_stats)},
        "roofline": roof, "parity": parity, "cpu_baseline": cpu_rec, "e2e": e2e_rec,
        "gpu_launches": launches, "clocks": clocks,
    }


def parity_demigrate(s, image, d_out, n_traces: int = 6):
    """Sampled trace rows of the adjoint against the oracle's transpose of Eq. 1 (whole rows)."""
    oracle = _oracle()
    rng = np.random.default_rng(sv.BASE_SEED + 23)
    idx = np.sort(rng.choice(s.ntr, size=n_traces, replace=False))
    got = d_out[torch.as_tensor(idx, device=d_out.device)].double().cpu().numpy()
    t0 = time.perf_counter()
    want = oracle.demigrate(s.subset(idx), image.double().cpu().numpy())
    err = float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))
    return {"rel_l2": err, "bar": BAR_FP32, "within_bar": err <= BAR_FP32, "traces": int(idx.size),
            "vs": "FP64 oracle transpose of Eq. 1, whole sampled trace rows",
            "oracle_s": round(time.perf_counter() - t0, 2)}


def parity_vgrad(s, dev, cache, block: int = 16):
    """The gradient on a sub-problem the oracle finishes in seconds: a block x block-column window
    of the image (all depths) and the traces of one offset bin."""
    from paper_1204_1225_gb300 import kirchhoff as kh
    oracle = _oracle()
    bins = oracle.bins(s)
    b = s.n_bins // 3
    idx = np.flatnonzero(bins == b)
    i0, j0 = (s.nx - block) // 2, (s.ny - block) // 2
    sub = s.subset(idx).replace(nx=block, ny=block, ox=s.ox + i0 * s.dx, oy=s.oy + j0 * s.dy)
    img = cache["image"][:, j0:j0 + block, i0:i0 + block, :].contiguous()
    tr = cache["traces"][torch.as_tensor(idx, device=dev)].contiguous()
    got = kh.Plan(sub).velocity_grad(kh.Headers.of(sub, device=dev), img, tr).cpu().numpy()
    t0 = time.perf_counter()
    want, absum = oracle.vgrad(sub, img.double().cpu().numpy(), tr.double().cpu().numpy(), return_abs=True)
    err = float(np.max(np.abs(got - want) / absum))
    return {"abs_err_over_sum_abs_terms": err, "bar": BAR_GRAD_ABS, "within_bar": err <= BAR_GRAD_ABS,
            "rel_err": [float(abs(g - w) / max(abs(w), 1e-300)) for g, w in zip(got, want)],
            "vs": f"FP64 oracle gradient on a {block}x{block}-column window of the image (all depths) "
                  f"and the {idx.size} traces of offset bin {b}",
            "oracle_s": round(time.perf_counter() - t0, 2)}


def run_cgls(args, s, ws, rank, local, dev):
    """Least-squares migration: each step is a full CGLS solve, min_m ||L^T m - d||^2 with
    --cg-iters iterations (one L for the start plus one L^T and one L per iteration), FP32
    vectors and FP64 inner products.  The metric counts the contributions of every operator
    apply of the step."""
    from paper_1204_1225_gb300 import kirchhoff as kh
    from paper_1204_1225_gb300 import lsm
    op = lsm.Operator(s, device=dev, fast_math=bool(args.fast_math))
    if s.dim == 2:
        sc = sv.reflectors_2d(np.random.default_rng(sv.BASE_SEED), s, spacing=5.0)
        d = sv.synthesize(s, sc, kh.arrival_times_fn(op.plan()), 25.0, device=dev, chunk=1 << 23)
    else:
        d = synth_traces(s, op.plan(), dev)
    d = d.contiguous()
    contrib = op.plan().count(op.hdr)
    applies = 1 + 2 * args.cg_iters
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(1, args.warmup // 3)):
        lsm.cgls(op, d, n_iter=args.cg_iters)
    torch.cuda.synchronize(dev)
    barrier(ws)
    launches0 = sum(p.launches for p in op._plans.values())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            m, rn, gn = lsm.cgls(op, d, n_iter=args.cg_iters)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    op.plan().sync()
    launches = sum(p.launches for p in op._plans.values()) - launches0
    t_ms = max_over_ranks(ws, e0.elapsed_time(e1))
    barrier(ws)
    if rank != 0:
        return None
    value = contrib * applies * args.steps * ws / (t_ms / 1e3) / 1e9
    rn = rn.numpy()
    return {
        "metric": "G image-point x trace contributions/s", "value": value, "unit": "Gcontrib/s",
        "n_gpus": ws, "steps": args.steps, "warmup": max(1, args.warmup // 3),
        "ms_per_step": t_ms / args.steps, "ms_per_cg_iteration": t_ms / args.steps / args.cg_iters,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": s.name, "operator": f"CGLS, {args.cg_iters} iterations "
                                                   f"({applies} operator applies per step)",
                   "image": list(op.image_shape), "ntr": s.ntr, "nt": s.nt,
                   "velocity": f"{s.vel} v0={s.v0} k={s.k}", "contributions_per_apply": contrib,
                   "inner_products": "FP64", "l2": "inputs larger than L2 (traces %.0f MB)" % (d.numel() * 4 / 1e6),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "cg": {"residual_norm_first": float(rn[0]), "residual_norm_last": float(rn[-1]),
               "normal_residual_first": float(gn[0]), "normal_residual_last": float(gn[-1]),
               "residual_monotone": bool(np.all(np.diff(rn) <= 1e-6 * rn[0]))},
        "roofline": {"bound": "alu", "kernel": "k_migrate + k_demigrate", "achieved": value, "peak": None,
                     "frac": None, "unit": "Gcontrib/s",
                     "peak_basis": "a sum of two kernels; see the migrate and demigrate lines"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
    }


def run_velan(args, s, ws, rank, local, dev):
    """Velocity analysis: each step migrates, measures the semblance of the offset images and its
    (v0, k) gradient, and updates (v0, k) by BFGS until it converges (at most 30 iterations),
    starting from v0 - 100 m/s, k - 0.1.  Noise-free 12 Hz diffractors.  The metric counts the
    contributions of every migration and gradient call of the step."""
    from paper_1204_1225_gb300.velan import VelocityAnalysis
    from paper_1204_1225_gb300 import kirchhoff as kh
    sc = sv.diffractors_2d(np.random.default_rng(3), s)
    d = sv.synthesize(s, sc, kh.arrival_times_fn(kh.Plan(s)), 12.0, device=dev)
    contrib = kh.Plan(s).count(kh.Headers.of(s, device=dev))
    va = VelocityAnalysis(s, d, fast_math=bool(args.fast_math), device=dev)
    start = (s.v0 - 100.0, s.k - 0.1)
    va.run(*start, n_iter=3)                      # warm-up
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    va.evaluations = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            r = va.run(*start, n_iter=30)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    t_ms = max_over_ranks(ws, e0.elapsed_time(e1))
    if rank != 0:
        return None
    evals = va.evaluations / args.steps
    zref = 700.0
    return {
        "metric": "G image-point x trace contributions/s",
        "value": 2 * contrib * evals * args.steps / (t_ms / 1e3) / 1e9, "unit": "Gcontrib/s",
        "n_gpus": ws, "steps": args.steps, "warmup": 1, "ms_per_step": t_ms / args.steps,
        "ms_per_evaluation": t_ms / args.steps / evals, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": s.name, "operator": "velocity analysis: BFGS on the semblance of the offset "
                                                   "images, gradient through the velocity-gradient kernel",
                   "start": {"v0": start[0], "k": start[1]}, "true": {"v0": s.v0, "k": s.k},
                   "contributions_per_migration": contrib, "evaluations_per_step": evals,
                   "parallelism": "replicas" if ws > 1 else "single"},
        "result": {"v0": r["v0"], "k": r["k"], "V": r["V"], "iterations": len(r["history"]) - 1,
                   "v_at_700m_rel_err": (r["v0"] + r["k"] * zref - (s.v0 + s.k * zref)) / (s.v0 + s.k * zref),
                   "k_err": r["k"] - s.k},
        "roofline": {"bound": "alu", "kernel": "k_migrate + k_vgrad", "achieved": None, "peak": None,
                     "frac": None, "unit": "Gcontrib/s",
                     "peak_basis": "a loop of two kernels; see the migrate and vgrad lines"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk.summary(),
    }


def time_grid_tables(plan, s, dev, reps: int = 3):
    """Builds the plan's first-arrival tables `reps` + 1 times (the first untimed) and reports the
    median wall time of kirchhoff_grid_tables (a synchronous setup call), with the work it did."""
    from paper_1204_1225_gb300 import kirchhoff as kh
    loc = kh.locations(s)
    times = []
    for i in range(reps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        plan.set_grid(s.grid_v, s.grid_ox, s.grid_h, loc)
        if i:
            times.append((time.perf_counter() - t0) * 1e3)
    _, rounds = plan.grid_tables()
    r = rounds.double()
    ms = statistics.median(times)
    nodes = int(s.grid_v.size)
    return {"ms": ms, "locations": int(loc.size), "nodes_per_location": nodes,
            "rounds_mean": float(r.mean()), "rounds_max": int(r.max()),
            "location_nodes_per_s": loc.size * nodes / (ms / 1e3),
            "what": "kirchhoff_grid_tables wall time: host checks of the model and locations, "
                    "one CTA per location sweeping in FP64, table store"}


def _form(line):
    """The fields of a form's own measurement kept in the headline line."""
    keep = ("value", "unit", "steps", "warmup", "ms_per_step", "roofline", "parity", "clocks",
            "gpu_launches", "loop", "speedup_vs_loop", "loop_tuned_tiles", "speedup_vs_loop_tuned_tiles")
    out = {k: line[k] for k in keep if k in line}
    out["config"] = {k: v for k, v in line["config"].items()
                     if k in ("workload", "operator", "trace_storage", "traveltimes", "contributions_per_step",
                              "batch_mode", "work_items", "staging_per_cta", "eikonal_tables", "velocity", "weight",
                              "aa_spacing_m")}
    return out


def run_forms(args, s, ws, rank, local, dev, cache, head):
    """The metric's other forms on the same GPU, each timed on its own: mixed precision (16-bit
    traces and traveltime table) on the headline survey, the adjoint and the (v0, k) gradient on
    the headline survey, prestack time migration of the same traces, gridded v(x, z) tables on the
    2.5D line, the true-amplitude weight at constant velocity (without and with operator anti-aliasing), and the 64-job batch as one graph
    replay against a loop of per-job calls (FP32 and FP16 traces)."""
    k = dict(steps=args.form_steps, warmup=3, e2e=False, cpu=False)
    forms = {}
    mixed = run_single(args, s, ws, rank, local, dev, cache, trace_dtype="f16", vel="table",
                       table_dtype="u16", **k)
    if rank == 0:
        forms["mixed_u16_table_f16_traces"] = _form(mixed)
        forms["mixed_u16_table_f16_traces"]["speedup_vs_fp32"] = mixed["value"] / head["value"]
    for op in ("demigrate", "vgrad"):
        r = run_single(args, s, ws, rank, local, dev, cache, op=op, **k)
        if rank == 0:
            forms[op] = _form(r)
    # prestack time migration of the same traces on a two-way-time axis (256 samples of 12 ms):
    # the same (column, trace) pairs, so the same contribution count
    s_t = s.replace(vel="pstm", oz=0.0, dz=0.012, name="3d-pstm-100000tr-256x256x256t")
    tcache = {key: cache[key] for key in ("hdr", "traces", "count", "traces64") if key in cache}
    r = run_single(args, s_t, ws, rank, local, dev, tcache, **k)
    if rank == 0:
        forms["time_migration"] = _form(r)
    # a laterally varying model on the 2.5D line: migration with the per-location first-arrival
    # tables of the eikonal solver, against the analytic v(z) path on the same geometry
    for wl, name in (("25d-vxz-20k-512x400", "gridded_vxz_tables"), ("25d-vz-20k-512x400", "gridded_vxz_background")):
        gargs = argparse.Namespace(**vars(args))
        gargs.workload = wl
        r = run_single(gargs, workloads()[wl](), ws, rank, local, dev, {}, **k)
        if rank == 0:
            forms[name] = _form(r)
    if rank == 0:
        forms["gridded_vxz_tables"]["speedup_vs_analytic_vz"] = (forms["gridded_vxz_tables"]["value"] /
                                                                 forms["gridded_vxz_background"]["value"])
    # the true-amplitude weight (constant velocity 2000 m/s) on the headline geometry and traces
    targs = argparse.Namespace(**vars(args))
    targs.workload = "3d-ta-100k-256cube"
    ccache = {key: cache[key] for key in ("hdr", "traces", "count", "traces64") if key in cache}
    r = run_single(targs, workloads()[targs.workload](), ws, rank, local, dev, ccache, **k)
    if rank == 0:
        forms["true_amplitude_const_v"] = _form(r)
    # and with operator anti-aliasing (the dip limitation for the 25 m receiver spacing)
    targs.workload = "3d-ta-aa-100k-256cube"
    r = run_single(targs, workloads()[targs.workload](), ws, rank, local, dev, ccache, **k)
    if rank == 0:
        forms["true_amplitude_anti_aliased_const_v"] = _form(r)
    # the headline v(z) survey and traces with operator anti-aliasing
    targs.workload = "3d-vz-aa-100k-256cube"
    r = run_single(targs, workloads()[targs.workload](), ws, rank, local, dev, ccache, **k)
    if rank == 0:
        forms["anti_aliased_vz"] = _form(r)
    cache.clear()
    torch.cuda.empty_cache()
    surveys = workloads()["batch64-3d-vz"]()
    bargs = parse_args(["--steps", str(args.form_steps), "--warmup", "3", "--no-tune",
                        "--batch-mode", args.batch_mode, "--no-cpu-baseline",
                        "--parity-points", str(min(args.parity_points, 1024))])
    bargs.workload = "batch64-3d-vz"
    jobs_cache = {}
    for tdt in ("f32", "f16"):
        bargs.trace_dtype = tdt
        r = run_batched(bargs, surveys, ws, rank, local, dev, jobs_cache)
        if rank == 0:
            forms[f"batch64_{tdt}"] = _form(r)
    # the persistent kernel over the FP32 batch, against the same per-job loop
    bargs.trace_dtype, bargs.batch_mode, bargs.no_loop = "f32", "persistent", True
    r = run_batched(bargs, surveys, ws, rank, local, dev, jobs_cache)
    if rank == 0:
        f = _form(r)
        loop = forms["batch64_f32"].get("loop")
        f["speedup_vs_loop"] = (r["value"] / loop["value"]) if loop else None
        forms["batch64_f32_persistent"] = f
    return forms


def _trace_order(plan, spatial_sort):
    from paper_1204_1225_gb300 import kirchhoff as kh
    g = kh.kirchhoff_cell_grid(plan.desc, spatial_sort)
    if g["ncx"] * g["ncy"] > 1:
        return f"offset bin, then midpoint cell of a {g['ncx']}x{g['ncy']} grid, then shot order"
    return "offset bin, then shot order (one midpoint cell)"


def _staging(examined, staged, ctas):
    """Traces the staging warps examined and staged per CTA (migration and gradient kernels)."""
    if not ctas:
        return None
    return {"examined": round(examined / ctas, 1), "staged": round(staged / ctas, 1), "ctas": ctas}


def run_batched(args, surveys, ws, rank, local, dev, jobs_cache=None):
    """64 uneven jobs: one graph-captured launch sequence per step vs a per-job loop."""
    from paper_1204_1225_gb300 import kirchhoff as kh
    from paper_1204_1225_gb300.autotune import TileTuner
    stream = torch.cuda.current_stream(dev)
    tdt = _TDT[args.trace_dtype]
    jobs_cache = {} if jobs_cache is None else jobs_cache
    if "traces" not in jobs_cache:
        jobs_cache["traces"] = [synth_batch_job(s, kh.Plan(s), j, dev) for j, s in enumerate(surveys)]
        jobs_cache["hdr"] = [kh.Headers.of(s, device=dev) for s in surveys]
    jobs = []
    for j, s in enumerate(surveys):
        p = kh.Plan(s, fast_math=bool(args.fast_math), trace_dtype=tdt)
        d = jobs_cache["traces"][j].to(tdt).contiguous()
        jobs.append((p, jobs_cache["hdr"][j], d, torch.empty(p.image_shape, dtype=torch.float32, device=dev)))
    contrib = sum(p.count(h) for (p, h, _, _) in jobs)
    t_tune = time.perf_counter()
    tiles = {}
    if not args.no_tune:
        tuner = TileTuner(path=args.tile_cache or os.path.join(ROOT, ".tile_cache", "tiles.json"))
        for (p, h, d, _) in jobs:
            t = tuner.choose(p, h, d)
            tiles[f"{t[0]}x{t[1]}x{t[2]}"] = tiles.get(f"{t[0]}x{t[1]}x{t[2]}", 0) + 1
    t_tune = time.perf_counter() - t_tune
    batch = kh.Batch(jobs, mode=args.batch_mode)
    graph = batch.capture()
    info = batch.info()
    launches_per_step = info["launches"]   # the capture ran the launch sequence once
    for _ in range(args.warmup):
        graph.replay()
    batch.sync()
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    batch.sync()
    t_ms = max_over_ranks(ws, e0.elapsed_time(e1))
    value = contrib * args.steps * ws / (t_ms / 1e3) / 1e9
    clocks = clk.summary()
    # a few jobs' batched images, kept for the bit-for-bit comparison with the per-job calls
    check = [0, len(jobs) // 2, len(jobs) - 1]
    kept = {j: jobs[j][3].clone() for j in check}

    def loop_arm(what):
        for _ in range(args.warmup):
            for (p, h, d, m) in jobs:
                p.migrate(h, d, out=m)
        torch.cuda.synchronize(dev)
        l0 = sum(p.launches for (p, _, _, _) in jobs)
        for (p, _, _, _) in jobs:   # events around each job's migration kernel
            p.profile(True)
            p.profile_read()
        e0.record(stream)
        for _ in range(args.steps):
            for (p, h, d, m) in jobs:
                p.migrate(h, d, out=m)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        for (p, _, _, _) in jobs:
            p.sync()
        kern = sum(p.profile_read()[0] for (p, _, _, _) in jobs) / args.steps
        for (p, _, _, _) in jobs:
            p.profile(False)
        tl = max_over_ranks(ws, e0.elapsed_time(e1))
        # what a single launch over all jobs could recover at most: the time of the step outside
        # the 64 migration kernels (binning, pair staging, launch gaps) plus the tails inside them
        return {"value": contrib * args.steps * ws / (tl / 1e3) / 1e9, "unit": "Gcontrib/s",
                "ms_per_step": tl / args.steps, "migration_kernels_ms_per_step": kern,
                "outside_kernels_frac": max(0.0, 1.0 - kern / (tl / args.steps)),
                "launches_per_step": (sum(p.launches for (p, _, _, _) in jobs) - l0) // args.steps,
                "what": what}

    loop = loop_tuned = None
    if not args.no_loop:
        if tiles:   # the batch's tuned tiles, then the plain path's default tiles
            loop_tuned = loop_arm("per-job kirchhoff_migrate calls on the same stream, the batch's tuned "
                                  "tiles, same precision")
            for (p, _, _, _) in jobs:
                p.set_tile(None)
        loop = loop_arm("per-job kirchhoff_migrate calls on the same stream, default tiles, same precision")
    barrier(ws)
    line = None
    if rank == 0:
        parity = None
        if not args.no_loop and not tiles:
            same = all(torch.equal(kept[j], jobs[j][3]) for j in check)
            parity = {"bitwise_equal_to_per_job_calls": same, "jobs_compared": check}
            if args.parity_points > 0:
                j = check[0]
                parity["oracle"] = parity_image(
                    surveys[j], jobs_cache["traces"][j].to(tdt).double().cpu().numpy(), kept[j],
                    args.parity_points, BAR_FP32, f"FP64 oracle on job {j}'s {args.trace_dtype} traces")
        clk_mhz = clocks.get("sm_mhz") or 2070.0
        mix = PIPE_MIX.get(f"{args.workload}-{args.trace_dtype}") if args.batch_mode == "persistent" else None
        roof = {"bound": "alu", "kernel": "k_migrate_batched" if args.batch_mode == "persistent" else "k_migrate",
                "achieved": value, "unit": "Gcontrib/s", "traffic": None}
        if mix:
            pipe, peak, bounds = pipe_roofline(mix, clk_mhz)
            roof.update({"peak": peak, "frac": value / peak, "binding_pipe": pipe,
                         "pipe_bounds": {k: round(v, 1) for k, v in bounds.items()},
                         "peak_basis": "min over pipes of the batched kernel's ncu-measured instruction "
                                       "mix; achieved over the whole graph replay"})
        else:
            roof.update({"peak": None, "frac": None,
                         "peak_basis": "no measured instruction mix for this kernel variant"})
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            s0, d0 = surveys[0], jobs[0][2]
            cpu = cpu_baseline(s0, d0.double().cpu().numpy(), args.cpu_seconds, sv.BASE_SEED)
        tb = sum(d.numel() * d.element_size() for (_, _, d, _) in jobs)
        ib = sum(m.numel() * 4 for (_, _, _, m) in jobs)
        line = {
            "metric": "G image-point x trace contributions/s", "value": value, "unit": "Gcontrib/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch64-3d-vz: {len(surveys)} jobs, n^3 at 10 m, n~U{{64..192}}, "
                                   "N_tr~U{1000..50000}, nt~U{750..2000}, constant v 2000 m/s, W=1, full "
                                   "aperture, 8 bins, 3 Ricker scatterers + noise per job",
                       "contributions_per_step": contrib, "trace_storage": args.trace_dtype,
                       "batch_mode": args.batch_mode, "work_items": info["items"], "ctas": info["ctas"],
                       "tiles": tiles,
                       "autotune_s": round(t_tune, 2),
                       "l2": "inputs larger than L2 (traces %.1f GB, images %.1f GB)" % (tb / 1e9, ib / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "loop": loop, "speedup_vs_loop": (value / loop["value"]) if loop else None,
            "loop_tuned_tiles": loop_tuned,
            "speedup_vs_loop_tuned_tiles": (value / loop_tuned["value"]) if loop_tuned else None,
            "roofline": roof, "parity": parity, "cpu_baseline": cpu, "e2e": None,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
        }
    batch.close()
    for (p, _, _, _) in jobs:
        p.close()
    return line


if __name__ == "__main__":
    main()
