"""Throughput benchmark of the Lagrange-flux hot path on one GB300 (or N replicas).

A "step" is one full Heun/RK2 time step (Sec. 4, steps 1-11: CFL dt from the
device-side wave-speed maximum, fused predictor, fused corrector) over the
whole mesh.  Default workload: the 8192 x 8192 periodic Kelvin-Helmholtz
shear layer (gamma 1.4, van Leer MUSCL, CFL 0.45) in FP32, the mesh of the
FP32-vs-FP64 precision study.  The state (1.07 GB in FP32) is far larger than
the 129 MB L2, so no L2 flush is needed between steps.

Printed: one JSON line (rank 0) with cell-updates/s, the per-kernel HBM
roofline of the dominant kernel (timed live with CUDA events on the solver's
stream), the FP64 path on the same workload, the FP32-vs-FP64 error after the
FP64 steps, an end-to-end number through the host-buffer API, SM clocks
sampled during the timed region, and the CPU oracle timed on a bounded sample
(the CPU baseline).  `--impl reference` times the CPU oracle alone.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s"
# The paper's own multicore-CPU throughput for the Lagrange-flux scheme (Sec. 5, performance
# table): context only, another machine; it states neither precision nor mesh size.
PAPER_CPU_CONTEXT = {
    "value": 81.0e6, "unit": METRIC, "note": "context only (other hardware, precision and mesh not stated)",
    "hardware": "2x Intel Xeon E5-2670 (Sandy Bridge, 16 cores, AVX, OpenMP)",
    "single_core": {"scalar": 2.6e6, "avx": 5.8e6}, "source": "arXiv:1607.08710, Sec. 5, performance table",
}
BYTES_PER_CELL = {  # algorithmic bytes per cell per launch: words read + written x word size
    ("stage0", "fp32"): 8 * 4, ("stage1", "fp32"): 12 * 4,
    ("stage0", "fp64"): 8 * 8, ("stage1", "fp64"): 12 * 8,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-run-steps", type=int, default=100)
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--ref-size", type=int, default=0,
                    help="mesh side of the --impl reference arm (0: --size, the benchmark's own mesh)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the measured FMA peaks (and the ALU rooflines)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-rk3", action="store_true")
    ap.add_argument("--rk3-steps", type=int, default=100)
    ap.add_argument("--no-species", action="store_true")
    ap.add_argument("--species-steps", type=int, default=100)
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--size3d", type=int, default=384)
    ap.add_argument("--steps3d", type=int, default=50)
    ap.add_argument("--batch-problems", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=300)
    ap.add_argument("--tile-rows", type=int, default=0,
                    help="rows per tile of the 2D stage kernels on the main mesh (0: chosen by lf_init)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-size", type=int, default=512)
    ap.add_argument("--adjoint-steps", type=int, default=256)
    return ap.parse_args()


def workload_config(args, n=None):
    n = n or args.size
    return {"workload": f"periodic Kelvin-Helmholtz shear layer {n}x{n}",
            "nx": n, "ny": n, "gamma": 1.4, "limiter": "van Leer", "cfl": 0.45,
            "bc": "periodic", "riemann": "eqs. 13-14, a = max(c_L, c_R)", "seed": 0,
            "l2_policy": "inputs larger than L2 (state %.2f GB vs 129 MB L2), no flush" %
                         (4 * n * n * (4 if args.precision == "fp32" else 8) / 1e9)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="lf_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and self.uuid not in f[1]:
                continue
            rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[4]) for r in rows if r[4].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
KERNEL_SOURCES = ("lf_device.cuh", "lf_stage.cuh", "lf_internal.h", "lf_kernels_f32.cu", "lf_kernels_f64.cu",
                  "lf_device3d.cuh", "lf_stage3d.cuh", "lf_internal3d.h", "lf_kernels3d_f32.cu",
                  "lf_batch_stage.cuh", "lf_batch.cu")


def code_text(src: str) -> str:
    """C++/CUDA source without comments and with whitespace collapsed: the
    part of a file that decides what the compiler builds."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash(root: str = ROOT) -> str:
    """Hash of the device code that the stage kernels are compiled from
    (comments and layout excluded, so a counter capture stays tied to the
    code it measured)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(code_text(open(os.path.join(root, "paper_1607_08710_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, cells: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to `cells`; None when absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d["kernels"][kernel]
        if d.get("source_hash") != kernel_source_hash():
            return None
        return e["dram_bytes_per_launch"] * cells / e["cells"]
    except (KeyError, ValueError, ZeroDivisionError):
        return None


def algorithmic_flops(workload: str = "kh2d"):
    """The method's flops per cell (predictor, corrector, step) from the
    oracle's op count stored in profiles/algorithmic_flops.json (written by
    oracle/count_flops.py); None when absent."""
    path = os.path.join(ROOT, "profiles", "algorithmic_flops.json")
    if not os.path.exists(path):
        return None
    try:
        return json.load(open(path))["workloads"][workload]["flops_per_cell"]
    except (KeyError, ValueError):
        return None


def alu_peaks(device: int):
    """Measured FMA throughput (lf_measure_peak) of FP64, FP32 and paired FP32,
    with the SM clock sampled while the chains run."""
    from paper_1607_08710_gb300.lagflux import measure_peak

    clocks = ClockSampler(None)
    clocks.start()
    res = {k: measure_peak(k, device, 50.0) for k in ("fp64", "fp32", "fp32_paired")}
    res["clocks"] = clocks.stop()
    res["unit"] = "TFLOP/s"
    res["how"] = "lf_measure_peak: 8 independent FMA chains per thread, 8 CTAs x 256 threads per SM, best of 3 launches"
    return res


def fp64_alu_roofline(stage_ms, cells, alu):
    """FP64 ALU roofline of the FP64 corrector: the method's algorithmic flops
    per cell (oracle op count) x cells / live kernel time, against the measured
    FP64 FMA peak; beside it the FP64 flops the kernel executes (ncu count of
    the committed capture, when it matches the current kernel sources), which
    include the Newton sequences of the divisions and square roots."""
    k = "stage2d_kernel<double, VANLEER, corrector>"
    alg = algorithmic_flops()
    if alg is None or not alu:
        return None
    t = stage_ms[1] / 1e3
    peak = alu["fp64"]
    achieved = alg["corrector"] * cells / t / 1e12
    sm = alu.get("clocks", {}).get("sm_mhz")
    roof = {"bound": "alu", "kernel": k, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flops_per_cell": alg["corrector"],
            "flops_kind": "algorithmic: oracle op count of the method, each add, multiply, divide and root one flop "
                          f"({alg['div_sqrt']['corrector']:.1f} of them divisions or roots; "
                          "profiles/algorithmic_flops.json)",
            "peak_kind": f"measured: lf_measure_peak DFMA chains (SM clock {sm} MHz)"}
    path = os.path.join(ROOT, "profiles", "fp64_flops.json")
    if os.path.exists(path):
        d = json.load(open(path))
        if d.get("source_hash") == kernel_source_hash():
            ex = d["kernels"][k]["fp64_flops_per_cell"]
            roof["executed"] = {"flops_per_cell": ex, "achieved": ex * cells / t / 1e12,
                                "frac": ex * cells / t / 1e12 / peak,
                                "source": "ncu dadd + dmul + 2 dfma per cell (" + d["capture"] + ")"}
    return roof


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


CPU_SAMPLES = {  # the oracle's timing samples: (generator, bc, mesh side, steps)
    "C1": ("four-quadrant Riemann problem (seed 0)", "transmissive", 2048, 10),
    "C2": ("periodic Kelvin-Helmholtz shear layer (seed 0)", "periodic", 1024, 20),
}


def time_oracle(O, key, n=None, steps=None):
    """Seconds and steps of one oracle run of sample `key` (the loaded build)."""
    from paper_1607_08710_gb300 import inputs

    what, bc, n0, s0 = CPU_SAMPLES[key]
    n, steps = n or n0, steps or s0
    oc = O.OracleConfig(nx=n, ny=n, limiter="vanleer", bc=bc, cfl=0.45)
    q = inputs.quadrant(n, n, seed=0) if key == "C1" else inputs.kelvin_helmholtz(n, n, seed=0)
    U0 = O.prim_to_cons(oc, q.stack())
    t0 = time.perf_counter()
    r = O.run(oc, U0, steps)
    return time.perf_counter() - t0, r.steps, n


def cpu_baseline(args):
    """The CPU oracle as it stands on bounded samples of the workloads: C1
    (2048^2 four-quadrant problem, 10 steps) and C2 (1024^2 periodic shear
    layer, 20 steps), each single-threaded (the plain build) and on all host
    cores (the same source built with OpenMP, same bits).  The headline is C2
    (the benchmark's generator on a smaller mesh) on all cores."""
    from oracle import oracle as O

    cores = host_cores()
    runs = []
    for key in ("C1", "C2"):
        el, steps, n = time_oracle(O, key)
        runs.append({"sample": key, "mesh": f"{n}x{n}", "steps": steps, "threads": 1, "seconds": el,
                     "value": n * n * steps / el})
    with O.use_library(O.build_omp()):
        threads = O.threads(cores)
        for key in ("C1", "C2"):
            time_oracle(O, key, n=256, steps=1)  # start the thread pool
            el, steps, n = time_oracle(O, key)
            runs.append({"sample": key, "mesh": f"{n}x{n}", "steps": steps, "threads": threads, "seconds": el,
                         "value": n * n * steps / el})
    head = runs[-1]
    return {"value": head["value"], "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle (OpenMP build, {threads} threads), periodic Kelvin-Helmholtz "
                      f"{head['mesh']}, {head['steps']} steps ({head['seconds']:.1f} s)",
            "single_thread": runs[1]["value"], "runs": runs,
            "samples": {k: f"{v[0]}, {v[2]}x{v[2]}, {v[3]} steps, {v[1]}" for k, v in CPU_SAMPLES.items()}}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args, dist):
    """The CPU oracle (OpenMP build, all host cores) on the benchmark's own
    workload: W warm-up steps, then K timed Heun steps of the 8192^2 periodic
    shear layer (about 4 s per step on 16 Grace cores).  --ref-size runs a
    smaller mesh of the same generator, and the config line then names it."""
    if dist.rank != 0:
        return
    from oracle import oracle as O
    from paper_1607_08710_gb300 import inputs

    n = args.ref_size or args.size
    oc = O.OracleConfig(nx=n, ny=n, limiter="vanleer", bc="periodic", cfl=0.45)
    U = O.prim_to_cons(oc, inputs.kelvin_helmholtz(n, n, seed=0).stack())
    with O.use_library(O.build_omp()):
        threads = O.threads(host_cores())
        if args.warmup > 0:
            U = O.run(oc, U, args.warmup).U
        t0 = time.perf_counter()
        r = O.run(oc, U, args.steps)
        el = time.perf_counter() - t0
    v = n * n * r.steps / el
    cfg = workload_config(args, n)
    sample = (f"FP64 oracle (OpenMP build, {threads} threads), {r.steps} Heun steps of the periodic "
              f"Kelvin-Helmholtz shear layer on {n}x{n} cells after {args.warmup} warm-up steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
        "steps": r.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(r.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_batched(args, dist, dev):
    """Independent four-quadrant problems with sides log-uniform in [64, 1024]
    (seeded), FP32, van Leer, CFL 0.45, transmissive; tile height autotuned;
    the loop of --batch-steps steps recorded as one CUDA graph, replayed once
    as warm-up and once timed."""
    import torch

    from paper_1607_08710_gb300 import inputs
    from paper_1607_08710_gb300.lagflux import Config, LagrangeFluxBatch

    sizes = [tuple(int(v) for v in s) for s in inputs.batched_sizes(args.batch_problems, seed=0)]
    cfgs = [Config(nx=nx, ny=ny, precision="fp32", limiter="vanleer", bc="transmissive", cfl=0.45,
                   device=dist.local_rank) for nx, ny in sizes]
    b = LagrangeFluxBatch(cfgs)
    for p, (nx, ny) in enumerate(sizes):
        q = torch.from_numpy(inputs.quadrant(nx, ny, seed=p).stack()).to(dev, torch.float32)
        b.set_primitive(p, q[0], q[1], q[2], q[3])
    rows = b.autotune(3)
    b.run(args.batch_steps)  # records the graph and runs it once (warm-up)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    e0.record()
    b.run(args.batch_steps)
    e1.record()
    torch.cuda.synchronize()
    t = dist.max(e0.elapsed_time(e1) / 1e3)
    _, steps = b.times()  # raises on a device error flag
    # per-stage device time, a separate pass of direct launches bracketed by events
    pm0, pm1 = b.profile(10)
    b.close()
    cells = sum(nx * ny for nx, ny in sizes)
    # columns the warp strips compute (64 per strip of 60 outputs in FP32) over the mesh's columns
    strips = sum(-(-nx // 60) * 64 * ny for nx, ny in sizes)
    edge = sum((2 if nx > 60 else 1) * 64 * ny for nx, ny in sizes)
    tile_halo = sum(nx * (ny + 4 * -(-ny // rows)) for nx, ny in sizes)
    peak, peak_kind = peaks()
    st = {"stage0": pm0 / 10, "stage1": pm1 / 10}
    gbs = {k: BYTES_PER_CELL[(k, "fp32")] * cells / (v / 1e3) / 1e9 for k, v in st.items()}
    dom = max(st, key=st.get)
    kb = "batch_stage_kernel<float, VANLEER, %s>" % ("predictor" if dom == "stage0" else "corrector")
    traffic = measured_traffic(kb, cells)
    return {"value": dist.world * cells * args.batch_steps / t, "unit": METRIC, "problems": len(sizes),
            "cells": cells, "steps": args.batch_steps, "ms_per_step": 1e3 * t / args.batch_steps,
            "tile_rows": rows, "graph": True, "launches_per_step": 4,
            "stage_ms": [st["stage0"], st["stage1"]],
            "roofline": {"bound": "hbm", "kernel": kb,
                         "achieved": gbs[dom], "peak": peak, "unit": "GB/s", "frac": gbs[dom] / peak,
                         "traffic": traffic,
                         "traffic_frac": None if traffic is None else traffic / (st[dom] / 1e3) / 1e9 / peak,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "algorithmic_bytes_per_cell": BYTES_PER_CELL[(dom, "fp32")],
                         "step_frac": 80 * cells * args.batch_steps / t / 1e9 / peak},
            "work_shape": {"strip_columns_over_cells": strips / cells, "edge_strip_share": edge / strips,
                           "rows_read_over_rows": tile_halo / cells},
            "workload": "four-quadrant Riemann problems, sides log-uniform in [64, 1024], seeds 0..P-1"}


def fd_at_literal_state(s, q, gq, dts, rho_target, n, ndir=4):
    """Central finite differences of J along seeded smooth directions in
    (rho0, p0) at the literal shear layer, replaying the frozen dt sequence,
    against <grad, d> of the adjoint.  The layer is piecewise constant, so
    every slope starts on the limiter's kink and every max(c_L, c_R) inside a
    layer is a tie: J is only directionally differentiable there (a
    non-smooth point), and the two need not agree.  Reported, not a check."""
    import torch

    from paper_1607_08710_gb300 import inputs

    def J(qq):
        s.set_primitive(qq[0], qq[1], qq[2], qq[3])
        for dt in dts:
            s.step_fixed(float(dt))
        U = torch.empty_like(qq)
        s.get_state(U)
        return float(((U[0] - rho_target) ** 2).sum())

    errs = {}
    for h in (1e-6, 1e-7):
        e = []
        for k in range(ndir):
            d = torch.zeros_like(q)
            d[0] = torch.from_numpy(inputs.smooth_perturbation(n, n, seed=1000 + 2 * k)).to(q)
            d[3] = torch.from_numpy(inputs.smooth_perturbation(n, n, seed=1001 + 2 * k)).to(q)
            ad = float((gq * d).sum())
            fd = (J(q + h * d) - J(q - h * d)) / (2 * h)
            e.append(abs(fd - ad) / abs(ad))
        errs[f"h={h:g}"] = e
    return {"label": "non-smooth point (literal shear layer, no background)", "directions": ndir,
            "relative_error_per_direction": errs}


def run_adjoint(args, dev):
    """Gradient of J = sum (rho(T) - rho_target)^2 with respect to the initial
    (rho, u, v, p), 512 x 512 periodic Kelvin-Helmholtz layer, 256 steps at
    CFL 0.4, van Leer, FP64 and FP32: the checkpointed forward sweep
    (lf_adjoint_forward) and the reverse sweep (lf_adjoint_backward), each
    timed with CUDA events, against a plain forward run of the same steps.
    rho_target is rho(T) of a run from the same layer with a seeded smooth
    density perturbation (not timed)."""
    import torch

    from paper_1607_08710_gb300 import inputs
    from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux

    n, nsteps = args.adjoint_size, args.adjoint_steps
    cells = n * n
    q0 = inputs.kelvin_helmholtz(n, n, seed=0).stack()
    qt = q0.copy()
    qt[0] += 1e-2 * inputs.smooth_perturbation(n, n, seed=98)
    res = {"workload": f"periodic Kelvin-Helmholtz shear layer {n}x{n}, {nsteps} steps at CFL 0.4, "
                       "J = sum (rho(T) - rho_target)^2, gradient in (rho, u, v, p)(0)",
           "unit": METRIC, "steps": nsteps, "checkpoints": "every ceil(sqrt(N)) steps, segments recomputed once"}
    for prec, tdt in (("fp64", torch.float64), ("fp32", torch.float32)):
        kw = dict(nx=n, ny=n, precision=prec, limiter="vanleer", bc="periodic", cfl=0.4)
        s = LagrangeFlux(Config(**kw))
        q = torch.from_numpy(qt).to(dev, tdt)
        s.set_primitive(q[0], q[1], q[2], q[3])
        s.run(max_steps=nsteps)
        UT = torch.empty((4, n, n), dtype=tdt, device=dev)
        s.get_state(UT)
        rho_target = UT[0].clone()
        q = torch.from_numpy(q0).to(dev, tdt)
        lam = torch.zeros((4, n, n), dtype=tdt, device=dev)
        gq = torch.empty((4, n, n), dtype=tdt, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        for rep in range(2):  # the first pass warms up; the second is timed
            s.set_primitive(q[0], q[1], q[2], q[3])
            torch.cuda.synchronize()
            ev[0].record()
            s.run(max_steps=nsteps)
            ev[1].record()
            s.set_primitive(q[0], q[1], q[2], q[3])
            torch.cuda.synchronize()
            ev[2].record()
            dts = s.adjoint_forward(nsteps)
            ev[3].record()
            s.get_state(UT)
            lam[0] = 2.0 * (UT[0] - rho_target)
            torch.cuda.synchronize()
            e_b0 = torch.cuda.Event(enable_timing=True)
            e_b0.record()
            s.adjoint_backward(lam, grad_q0=gq)
            ev[4].record()
            torch.cuda.synchronize()
        t_plain = ev[0].elapsed_time(ev[1]) / 1e3
        t_fwd = ev[2].elapsed_time(ev[3]) / 1e3
        t_bwd = e_b0.elapsed_time(ev[4]) / 1e3
        assert bool(torch.isfinite(gq).all())
        res[prec] = {"value": cells * nsteps / (t_fwd + t_bwd), "forward_ms": 1e3 * t_fwd,
                     "backward_ms": 1e3 * t_bwd, "plain_forward_ms": 1e3 * t_plain,
                     "gradient_over_forward": (t_fwd + t_bwd) / t_plain}
        if prec == "fp64":
            res[prec]["fd_nonsmooth_point"] = fd_at_literal_state(s, q, gq, dts, rho_target, n)
        s.close()
        del q, UT, lam, gq
        torch.cuda.empty_cache()
    return res


def run_ours(args, dist):
    import torch

    from paper_1607_08710_gb300 import inputs
    from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux

    torch.cuda.set_device(dist.local_rank)
    dev = torch.device("cuda", dist.local_rank)
    n = args.size
    cells = n * n
    prec = args.precision
    tdt = torch.float32 if prec == "fp32" else torch.float64
    prim = inputs.kelvin_helmholtz(n, n, seed=0).stack()
    kw = dict(nx=n, ny=n, limiter="vanleer", bc="periodic", cfl=0.45, device=dist.local_rank,
              tile_rows=args.tile_rows)

    solver = LagrangeFlux(Config(precision=prec, **kw))
    tile_used = solver.tile_rows
    q = torch.from_numpy(prim).to(dev, tdt)
    solver.set_primitive(q[0], q[1], q[2], q[3])
    del q
    for _ in range(args.warmup):
        solver.step()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    start.record()
    for _ in range(args.steps):
        solver.step()
    stop.record()
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    t_local = start.elapsed_time(stop) / 1e3
    solver.sync()  # raises on a device-side error flag
    t = dist.max(t_local)
    value = dist.world * cells * args.steps / t

    # per-kernel device time (separate pass, so the tracing events do not touch the timed number)
    solver.profile(True)
    for _ in range(args.profile_steps):
        solver.step()
    (ms0, ms1), (n0, n1) = solver.profile_read()
    solver.profile(False)
    kernels = {}
    for name, ms, cnt in (("stage0", ms0, n0), ("stage1", ms1, n1)):
        avg = ms / cnt / 1e3
        b = BYTES_PER_CELL[(name, prec)] * cells
        kernels[name] = {"avg_ms": avg * 1e3, "launches": cnt, "algorithmic_bytes": b, "gbs": b / avg / 1e9}
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"])
    peak, peak_kind = peaks()
    kname = {"stage0": "stage2d_kernel<%s, VANLEER, predictor>", "stage1": "stage2d_kernel<%s, VANLEER, corrector>"}
    kname = {k: v % ("float" if prec == "fp32" else "double") for k, v in kname.items()}
    traffic = measured_traffic(kname[dom], cells)
    roofline = {"bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kernels[dom]["gbs"] / peak, "traffic": traffic,
                # ncu-measured DRAM bytes of a launch over its live duration
                "traffic_frac": None if traffic is None else traffic / (kernels[dom]["avg_ms"] / 1e3) / 1e9 / peak,
                "kernel": kname[dom],
                "peak_kind": f"{peak_kind} copy bandwidth",
                "step_frac": (sum(BYTES_PER_CELL[(k, prec)] for k in ("stage0", "stage1")) * cells * args.steps / t_local
                              / 1e9) / peak}

    out = {}
    alu = None
    if not args.no_peaks and dist.rank == 0:
        alu = alu_peaks(dist.local_rank)
        out["alu_peaks"] = alu
        alg = algorithmic_flops()
        if alg is not None:  # the FP32 step's arithmetic against the paired-FP32 peak (context: it is HBM-bound)
            roofline["alu_context"] = {
                "flops_per_cell_step": alg["step"],
                "achieved": alg["step"] * cells * args.steps / t_local / 1e12, "unit": "TFLOP/s",
                "peak": alu["fp32_paired"],
                "frac": alg["step"] * cells * args.steps / t_local / 1e12 / alu["fp32_paired"]}
    # FP64 path on the same workload, and the FP32-vs-FP64 error after those steps
    if prec == "fp32" and not args.no_fp64 and dist.rank == 0:
        s64 = LagrangeFlux(Config(precision="fp64", **kw))
        q = torch.from_numpy(prim).to(dev, torch.float64)
        s64.set_primitive(q[0], q[1], q[2], q[3])
        s64.step()  # warm-up
        s64.set_primitive(q[0], q[1], q[2], q[3])
        del q
        dts = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.fp64_steps):
            s64.step()
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        s64.profile(True)
        s64.step()
        (m0, m1), _ = s64.profile_read()
        s64.profile(False)
        # replay the FP64 dt sequence in FP32 from the same initial state
        s64.set_primitive(*torch.from_numpy(prim).to(dev, torch.float64))
        for _ in range(args.fp64_steps):
            dts.append(s64.step(return_dt=True))
        ref = torch.empty((4, n, n), dtype=torch.float64, device=dev)
        s64.get_state(ref)
        s64.close()
        s32 = LagrangeFlux(Config(precision="fp32", **kw))
        s32.set_primitive(*torch.from_numpy(prim).to(dev, torch.float32))
        for dt in dts:
            s32.step_fixed(dt)
        got = torch.empty((4, n, n), dtype=torch.float32, device=dev)
        s32.get_state(got)
        s32.close()
        l1 = [float((got[l].double() - ref[l]).abs().sum() / ref[l].abs().sum()) for l in range(4)]
        del ref, got
        v64 = cells * args.fp64_steps / t64
        out["fp64"] = {"value": v64, "unit": METRIC, "steps": args.fp64_steps, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                       "stage_ms": [m0, m1], "roofline": fp64_alu_roofline([m0, m1], cells, alu)}
        out["fp32_over_fp64"] = value / dist.world / v64
        out["l1_error"] = {"fp32_vs_fp64_relative_l1": dict(zip(["rho", "rhou", "rhov", "rhoE"], l1)),
                           "after_steps": args.fp64_steps}
        torch.cuda.empty_cache()

    # the same workload with the third-order SSP Runge-Kutta integrator (three fused stages per step)
    if not args.no_rk3 and dist.rank == 0:
        s3 = LagrangeFlux(Config(precision=prec, time_order=3, **kw))
        q = torch.from_numpy(prim).to(dev, tdt)
        s3.set_primitive(q[0], q[1], q[2], q[3])
        del q
        for _ in range(args.warmup):
            s3.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.rk3_steps):
            s3.step()
        e1.record()
        torch.cuda.synchronize()
        t3 = e0.elapsed_time(e1) / 1e3
        s3.sync()
        s3.profile(True)
        for _ in range(5):
            s3.step()
        (a0, a1), (c0, c1) = s3.profile_read()
        s3.close()
        out["rk3"] = {"value": cells * args.rk3_steps / t3, "unit": METRIC, "steps": args.rk3_steps,
                      "ms_per_step": 1e3 * t3 / args.rk3_steps, "first_stage_ms": a0 / c0,
                      "later_stage_ms": a1 / c1, "integrator": "SSP-RK3 (Shu-Osher), 3 fused stages per step"}
        torch.cuda.empty_cache()

    # the same shear layer carrying two transported mass fractions (Sec. 5): 6 fields per cell
    if not args.no_species and dist.rank == 0:
        ns = 2
        ps = inputs.shear_layer_tracers(n, n, seed=0, nspecies=ns).stack()
        ssp = LagrangeFlux(Config(precision=prec, nspecies=ns, **kw))
        q = torch.from_numpy(ps).to(dev, tdt)
        del ps
        ssp.set_primitive(q[0], q[1], q[2], q[3])
        ssp.set_mass_fractions(q[4:].contiguous())
        del q
        for _ in range(args.warmup):
            ssp.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.species_steps):
            ssp.step()
        e1.record()
        torch.cuda.synchronize()
        tsp = e0.elapsed_time(e1) / 1e3
        ssp.sync()
        ssp.profile(True)
        for _ in range(args.profile_steps):
            ssp.step()
        (a0, a1), (c0, c1) = ssp.profile_read()
        ssp.close()
        word = 4 if prec == "fp32" else 8
        nf = 4 + ns
        ms = {"stage0": a0 / c0, "stage1": a1 / c1}
        byts = {"stage0": 2 * nf * word * cells, "stage1": 3 * nf * word * cells}
        peak, peak_kind = peaks()
        sk = max(ms, key=ms.get)
        gbs = byts[sk] / (ms[sk] / 1e3) / 1e9
        out["species"] = {
            "value": cells * args.species_steps / tsp, "unit": METRIC, "steps": args.species_steps,
            "ms_per_step": 1e3 * tsp / args.species_steps, "nspecies": ns, "stage_ms": [ms["stage0"], ms["stage1"]],
            "roofline": {"bound": "hbm", "kernel": f"stage2d_kernel<{'float' if prec == 'fp32' else 'double'}, "
                         f"VANLEER, {'predictor' if sk == 'stage0' else 'corrector'}, NF={nf}>",
                         "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "algorithmic_bytes_per_cell": byts[sk] // cells},
            "workload": f"periodic shear layer {n}x{n} with tracers y_1 = layer indicator, y_2 = 1 - y_1"}
        torch.cuda.empty_cache()

    # the 3D step (faces normal to x, y and z) on a periodic 3D shear layer
    if not args.no_3d and dist.rank == 0:
        n3 = args.size3d
        cells3 = n3 ** 3
        s3d = LagrangeFlux(Config(nx=n3, ny=n3, nz=n3, dim=3, precision=prec, limiter="vanleer", bc="periodic",
                                  cfl=0.45, device=dist.local_rank))
        q = torch.from_numpy(inputs.shear_layer_3d(n3, seed=0).stack()).to(dev, tdt)
        s3d.set_primitives(q)
        del q
        for _ in range(args.warmup):
            s3d.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps3d):
            s3d.step()
        e1.record()
        torch.cuda.synchronize()
        t3d = e0.elapsed_time(e1) / 1e3
        s3d.sync()
        s3d.profile(True)
        for _ in range(args.profile_steps):
            s3d.step()
        (a0, a1), (c0, c1) = s3d.profile_read()
        s3d.close()
        word = 4 if prec == "fp32" else 8
        ms = {"stage0": a0 / c0, "stage1": a1 / c1}
        byts = {"stage0": 2 * 5 * word * cells3, "stage1": 3 * 5 * word * cells3}
        peak, peak_kind = peaks()
        sk = max(ms, key=ms.get)
        gbs = byts[sk] / (ms[sk] / 1e3) / 1e9
        k3 = (f"stage3d_kernel<{'float' if prec == 'fp32' else 'double'}, "
              f"VANLEER, {'predictor' if sk == 'stage0' else 'corrector'}>")
        traffic3 = measured_traffic(k3, cells3)
        out["3d"] = {
            "value": cells3 * args.steps3d / t3d, "unit": METRIC, "steps": args.steps3d,
            "ms_per_step": 1e3 * t3d / args.steps3d, "stage_ms": [ms["stage0"], ms["stage1"]],
            "roofline": {"bound": "hbm", "kernel": k3,
                         "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "traffic": traffic3,
                         "traffic_frac": None if traffic3 is None else traffic3 / (ms[sk] / 1e3) / 1e9 / peak,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "algorithmic_bytes_per_cell": byts[sk] // cells3},
            "workload": f"periodic 3D shear layer {n3}^3 (Kelvin-Helmholtz layer, perturbation x cos(2 pi z))"}
        torch.cuda.empty_cache()

    # discrete adjoint: gradient of a final-time objective through the checkpointed step loop
    if not args.no_adjoint and dist.rank == 0:
        out["adjoint"] = run_adjoint(args, dev)

    # batched: 512 seeded uneven meshes, one persistent launch per stage, graph of the step loop
    if not args.no_batch:
        out["batched"] = run_batched(args, dist, dev)

    # end to end through the host-buffer API: pinned host state in, one step, state out
    if not args.no_e2e:
        hin = torch.from_numpy(prim).to(dev, tdt)
        solver.set_primitive(hin[0], hin[1], hin[2], hin[3])
        U = torch.empty((4, n, n), dtype=tdt, device=dev)
        solver.get_state(U)
        h_in = U.cpu().pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        del U, hin
        solver.set_state(h_in[0], h_in[1], h_in[2], h_in[3])
        for _ in range(2):  # warm-up: first touch of the pinned pages, graph-free step path
            solver.step()
            solver.get_state(h_out)
            solver.set_state(h_out[0], h_out[1], h_out[2], h_out[3])
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            solver.set_state(h_out[0], h_out[1], h_out[2], h_out[3])
            solver.step()
            solver.get_state(h_out)
        torch.cuda.synchronize()
        te = dist.max(time.perf_counter() - t0)
        nbytes = h_in.numel() * h_in.element_size()
        out["e2e"] = {"value": dist.world * cells * args.e2e_steps / te, "unit": METRIC,
                      "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                      "how": "per step: lf_set_state from pinned host planes, lf_step, lf_get_state to pinned host"}
        # a simulation run through the same host-buffer API: the state goes in
        # once, lf_run advances it, the final state comes out once
        kr = args.e2e_run_steps
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        solver.set_state(h_in[0], h_in[1], h_in[2], h_in[3])
        solver.run(max_steps=kr)
        solver.get_state(h_out)
        torch.cuda.synchronize()
        tr = dist.max(time.perf_counter() - t0)
        out["e2e_run"] = {"value": dist.world * cells * kr / tr, "unit": METRIC, "steps": kr,
                          "h2d_bytes": nbytes, "d2h_bytes": nbytes,
                          "how": f"lf_set_state from pinned host planes, lf_run of {kr} steps, lf_get_state to pinned "
                                 "host, all in the timed region"}
        del h_in, h_out
    solver.close()

    if dist.rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": dict(workload_config(args), tile_rows=tile_used,
                       parallelism=f"replicas x{dist.world}" if dist.world > 1 else "single GPU"),
        "roofline": roofline, "kernels": kernels, "gpu_launches": 4 * args.steps, "clocks": clk,
    }
    line.update(out)
    line["paper_cpu_context"] = PAPER_CPU_CONTEXT
    if not args.no_cpu_baseline and dist.world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
