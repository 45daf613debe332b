"""Benchmark of the spin-F BEC hot path on one (or N replicated) GB300.

Default workload: spin-3, 3D, 256^3 on [-10,10]^3, V = |x|^2/2 + 10 sum sin^2(pi x_i/2),
beta = (1000, -5, 10, 2), M = 0 (7 components, 1.88 GB per FP64 field; synthetic:
seeded Gaussian-times-noise states put on the constraint manifold by the library's own
projective retraction), in the FP64 form.  `--workload` selects the other synthetic
workloads: spin1_1d (n = 256), spin2_2d (256^2), spin3_3d_128 (the finest level of the
32^3 -> 64^3 -> 128^3 cascadic workload), batch512 (512 spin-1 2D instances on
64^2 / 128^2 / 256^2 grids with their own beta1 and M); `--precision mixed` the mixed form.

One step = one pass of the hot path as a Newton/BB iteration uses it:
  sbec_grad     energy, Euclidean and Riemannian gradient, ||grad E|| (Eq. 3.7, 3.12, Lemma 4.1)
  sbec_hessvec  Riemannian Hessian-vector product along the gradient (Eq. 3.13, Lemma 4.2)
  sbec_retract  projective retraction of a trial step (Lemma 5.1)
  sbec_energy   energy of the trial point
Each step works on a resident state larger than the 129 MB L2 (or cycles through
enough states to exceed it), so no step reads its inputs from L2 left by the previous one.

metric value = energy+grad evaluations per second (one per step and instance) over all ranks.
`--impl reference` times the CPU FP64 oracle doing the same step on a bounded sample
of the workload, on all host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from dataclasses import replace

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1907_01194_gb300 import workloads as W  # noqa: E402

METRIC = "energy+grad evals/s and time-to-ground-state (|Rgrad|<1e-8), % HBM roofline"
UNIT = "evals/s"
T_TRIAL = 1e-3
SIGMA = 0.5
L2_BYTES = 129e6

# FP64 ALU peak, nominal: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz.  The roofline uses
# the rate the library's FMA probe (sbec_probe_fma_peak) measures in the same run; the
# nominal figure is the fallback when the probe is skipped.
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.07


def _measured_hbm_gbs():
    # the measured copy bandwidth of this GPU type (read + write bytes), written next to
    # the repository by the measurement run; 6.8 TB/s when that file is absent
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _measured_hbm_gbs()
# pointwise FLOPs per grid point of the epilogues (counted from Eq. 3.7, 3.12, 3.13 in the
# ladder / pair form the kernels use: densities, then each output component's terms)
PW_FLOPS = {"grad": {1: 170, 2: 375, 3: 760}, "hess": {1: 300, 2: 640, 3: 1400},
            "energy": {1: 70, 2: 140, 3: 290}}
# the share of those counts that forms the densities (rho, F_z, F_+, A00, A_{2l}): the
# energy count less its energy-density terms.  The FP64 Hessian epilogue of a 2D / 3D
# product at the state of the latest gradient (every product of the bench's step and of
# the solvers) reads the densities that gradient stored instead of forming them
DENS_FLOPS = {1: 45, 2: 100, 3: 225}
# DRAM traffic per launch from ncu captures of the unchanged kernels (bytes), by
# (kernel, workload, form); profiles/ holds the summaries
NCU_TRAFFIC = {
    # full capture of the 256^2 FP64 workload (the state stays in L2: one read per field)
    ("s_k2", "spin2_2d_256x256", "fp64"): 5328128.0,
    # 128^3 capture of the same kernel (mean over its 8 launches, both forms) scaled by the
    # 8x larger fields (writes partly held in L2 at 128^3, so this is a lower bound at 256^3)
    ("proj_apply", "spin3_3d_256cubed", "mixed"): 8 * (234989280.0 + 81436448.0),
    # 128^3 capture of the FP64 spin-3 Hessian epilogue that reads the stored densities
    # (reads 994.2 MB, writes 241.7 MB per launch: 4 S + S_V + 16 density doubles per point)
    # scaled by the 8x larger fields
    ("x_inv_hess", "spin3_3d_256cubed", "fp64"): 8 * (994229760.0 + 241698048.0),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spin3_3d_256",
                    choices=["spin1_1d", "spin2_2d", "spin3_3d_128", "spin3_3d_256", "batch512"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paper-table", action="store_true",
                    help="only the paper's ARNT/RGBB x R1/R2/R3 comparison on its spin-2 2D case")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-ground-state solves")
    ap.add_argument("--solve-maxit", type=int, default=10000,
                    help="outer-iteration cap of each level of the time-to-ground-state solves")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--tiles", default=None,
                    help="launch shapes as JSON (keys of sbec_tune) instead of autotuning, e.g. for profiling")
    ap.add_argument("--grid", default=None,
                    help="the workload's problem on another grid, e.g. 128,128,256: a small case of the same "
                         "kernels for profiling (evaluation rate only: no solves, no CPU baseline)")
    args = ap.parse_args()
    if args.grid:
        if args.workload == "batch512":
            ap.error("--grid applies to the single-problem workloads")
        args.no_solve = args.no_cpu_baseline = True
    return args


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(name):
    if name == "spin1_1d":
        return W.spin1_1d()
    if name == "spin2_2d":
        return W.spin2_2d()
    if name == "spin3_3d_128":
        return W.spin3_3d_cascadic()
    if name == "spin3_3d_256":
        return W.spin3_3d_256()
    raise ValueError(name)


def solve_tol(name):
    return 1e-10 if name == "spin1_1d" else 1e-8


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle doing the same step
# ---------------------------------------------------------------------------
def oracle_step_runner(w):
    from oracle import sbec_oracle as O
    P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)
    u = O.psi_R1(P, O.to_u(P, O.to_matrix(P, W.initial_fields(w))))

    def step():
        g = O.egrad_u(P, u)
        E = O.E_u(P, u)
        rg = O.project(P, u, g)
        O.rhess(P, u, rg, g=g, sigma=SIGMA)
        z = O.retract(P, u, -T_TRIAL, 1)
        O.E_u(P, z)
        return E
    return step


# The CPU oracle's step on a grid of more than 2^21 points takes minutes: it is sampled
# on a z-slab of 2^20 points of the same workload (same x-y grid, grid spacing, spin,
# beta, M and potential values; the slab's z extent is cut to its points), and the
# rate is scaled by the slab's share of the grid.  Its pointwise work (most of the
# oracle's time) scales exactly with the points; its z transforms are shorter than the
# workload's (a small share of the time), so the scaled rate slightly favours the CPU.
SLAB_POINTS = 1 << 20


def cpu_workload_sample(w):
    """(workload the oracle steps on, its share of w's grid points, description)."""
    if w.dim < 3 or w.G <= 2 * SLAB_POINTS:
        return w, 1.0, f"full steps of the {w.name} workload"
    nz = max(2, SLAB_POINTS // (w.n[0] * w.n[1]))
    hz = (w.hi[2] - w.lo[2]) / w.n[2]
    j0 = w.n[2] // 2 - nz // 2
    lo = (w.lo[0], w.lo[1], w.lo[2] + j0 * hz)
    hi = (w.hi[0], w.hi[1], lo[2] + nz * hz)
    from dataclasses import replace
    ws = replace(w, name=f"{w.name}_zslab{nz}", n=(w.n[0], w.n[1], nz), lo=lo, hi=hi, levels=())
    return ws, ws.G / w.G, (f"steps on a {w.n[0]}x{w.n[1]}x{nz} z-slab (grid points z{j0}..z{j0 + nz - 1}) "
                            f"of the {w.name} workload, rate scaled by the slab's share {ws.G}/{w.G} of the points")


def host_cores():
    try:
        aff = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = os.cpu_count() or 1
    return aff, os.cpu_count() or aff


def cpu_sample(w, budget=15.0, max_steps=50, warmup=1):
    """The oracle as it stands on the host's cores: scipy.fft with one worker per core
    of the process's affinity mask, numpy's own threading for the rest.  `warmup`
    untimed steps (at least one, at most `budget` seconds of them), then up to max_steps
    timed steps within `budget` seconds (at least one).  Returns (evals/s of the full
    workload, timed steps, seconds, description, cores)."""
    import scipy.fft as sfft
    ws, share, desc = cpu_workload_sample(w)
    cores, _ = host_cores()
    with sfft.set_workers(cores):
        step = oracle_step_runner(ws)
        t0 = time.perf_counter()
        for i in range(max(1, warmup)):
            step()
            if time.perf_counter() - t0 > budget:
                break
        t0 = time.perf_counter()
        n = 0
        while n < max_steps and (n == 0 or time.perf_counter() - t0 < budget):
            step()
            n += 1
        dt = time.perf_counter() - t0
    return share * n / dt, n, dt, desc, cores


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    w = W.batched_spin1_2d()[2] if args.workload == "batch512" else workload(args.workload)
    val, n, dt, desc, cores = cpu_sample(w, budget=120.0, max_steps=args.steps, warmup=args.warmup)
    aff, total = host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "F": w.F, "grid": list(w.n), "components": w.C,
                       "parallelism": "replicas" if args.gpus > 1 else "single"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} {desc} (numpy/scipy FP64; scipy.fft workers = {cores} "
                                       f"cores of the affinity mask, {total} on the host)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 8:
                    rows.append(f)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def flops_model(w, kname, B=1):
    """Algorithmic FLOPs of one launch kind (per launch) for the workload (B instances)."""
    C, n = w.C, w.n
    G = int(np.prod(n))
    fft = lambda m: 5.0 * m * math.log2(m)
    d = len(n)
    if kname == "s_k2":
        m = n[-1]
        return B * C * (G // m) * (2 * fft(m) + 4 * m)
    if kname in ("s_fwd", "s_inv", "s_parseval") and d > 1:
        m = n[1] if kname != "s_parseval" else n[-1]
        return B * C * (G // m) * fft(m)
    if kname in ("x_fwd", "x_inv"):
        return B * C * (G // n[0]) * fft(n[0])
    if kname == "x_fwd_energy":
        return B * (C * (G // n[0]) * fft(n[0]) + G * PW_FLOPS["energy"][w.F])
    # 2D/3D: the gradient and Hessian epilogues are pointwise kernels of their own
    # (the inverse x transform before them is the x_inv launch)
    if kname == "x_inv_grad":
        return B * G * PW_FLOPS["grad"][w.F]
    if kname == "x_inv_hess":
        return B * G * (PW_FLOPS["hess"][w.F] - DENS_FLOPS[w.F])
    if kname == "x_full_grad":
        return B * (C * (2 * fft(n[0]) + 4 * n[0]) + G * PW_FLOPS["grad"][w.F])
    if kname == "x_full_hess":
        return B * (C * (2 * fft(n[0]) + 4 * n[0]) + G * PW_FLOPS["hess"][w.F])
    return None


def bytes_model(w, kname, elem, B=1):
    """Compulsory DRAM bytes of one launch (reads + writes), elem = bytes per complex value."""
    C, G = w.C, int(np.prod(w.n))
    S = B * C * G * elem
    SV = B * G * elem // 2
    return {"x_fwd": 2 * S, "x_inv": 2 * S, "x_fwd_energy": 2 * S + SV, "s_k2": 2 * S, "s_fwd": 2 * S, "s_inv": 2 * S,
            "s_parseval": S, "x_inv_grad": 3 * S + SV, "x_inv_hess": 4 * S + SV, "x_full_grad": 3 * S + SV,
            "x_full_hess": 4 * S + SV, "proj_apply": 3 * S, "dot_reduce": 2 * S, "retract_w": 3 * S,
            "scale": 2 * S, "lincomb": 3 * S}.get(kname)


def roofline_of(prof, w, precision, B, wname, fp64_peak=None):
    # the dominant kernel among those with an algorithmic model (the one-block finalize
    # kernels have none: they are launch-latency work)
    total = sum(v[0] for v in prof.values())
    modelled = {k: v for k, v in prof.items()
                if (flops_model(w, k, B) if precision == "fp64" else bytes_model(w, k, 8, B))}
    kname, (kms, kcnt) = max((modelled or prof).items(), key=lambda kv: kv[1][0])
    per_launch_s = kms / kcnt * 1e-3
    if precision == "fp64":
        fl = flops_model(w, kname, B)
        ach = fl / per_launch_s / 1e9 if fl else None
        peak = fp64_peak or FP64_NOMINAL_GFLOPS
        src = ("measured: FP64 FMA probe of this run (sbec_probe_fma_peak)" if fp64_peak else
               "FP64 nominal: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz")
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "GFLOP/s",
                "frac": ach / peak if ach else None,
                "traffic": NCU_TRAFFIC.get((kname, wname, "fp64")), "kernel": kname, "kernel_share": kms / total,
                "peak_source": src, "frac_of_nominal": ach / FP64_NOMINAL_GFLOPS if ach else None}
    by = bytes_model(w, kname, 8, B)
    ach = by / per_launch_s / 1e9 if by else None
    return {"bound": "hbm", "achieved": ach, "peak": HBM_PEAK_GBS, "unit": "GB/s",
            "frac": ach / HBM_PEAK_GBS if ach else None, "traffic": NCU_TRAFFIC.get((kname, wname, "mixed")),
            "kernel": kname, "kernel_share": kms / total, "peak_source": HBM_PEAK_SOURCE + " copy bandwidth (read + write bytes)"}


def aggregate(dist, elapsed_s, units_per_rank, device=None):
    """Whole-job rate over replicas: the slowest rank's time bounds the job, so
    value = units on all ranks / max over ranks of the elapsed time."""
    import torch
    world = dist.get_world_size() if dist is not None else 1
    t = elapsed_s
    if dist is not None:
        x = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t


def run_ours(args, world, rank, local):
    import torch
    from paper_1907_01194_gb300 import sbec

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return aggregate(pg, x, 1.0, dev)[1]

    stream = torch.cuda.current_stream()
    # measured FMA rates of this GPU (the FP64 form's roofline denominator)
    peaks = {"fp64_gflops": sbec.probe_fma_peak("fp64"), "fp32_gflops": sbec.probe_fma_peak("fp32")}
    cdt = torch.complex128 if args.precision == "fp64" else torch.complex64
    elem = 16 if args.precision == "fp64" else 8

    # ---- handles and resident states ----
    if args.workload == "batch512":
        insts = W.batched_spin1_2d()
        groups = []
        for n in (64, 128, 256):
            ws = [w for w in insts if w.n[0] == n]
            h = sbec.Handle.batch(ws, precision=args.precision, stream=stream.cuda_stream)
            X = torch.from_numpy(np.stack([W.initial_fields(w) for w in ws])).to(dev).to(cdt)
            h.retract(X, torch.zeros_like(X), 0.0, 1, X)
            groups.append((h, [X], ws))
        wname = "batch512_spin1_2d_64_128_256"
        w_main = insts[2]
        n_inst = len(insts)
        nstates = 1
    else:
        w_main = workload(args.workload)
        if args.grid:
            w_main = w_main.at(tuple(int(v) for v in args.grid.split(",")))
            w_main = replace(w_main, name=f"{w_main.name}_on_{'x'.join(str(v) for v in w_main.n)}")
        wname = w_main.name
        h = sbec.Handle.from_workload(w_main, precision=args.precision, stream=stream.cuda_stream)
        sbytes = w_main.C * w_main.G * elem
        nstates = int(min(32, max(1, math.ceil(2 * L2_BYTES / sbytes))))
        states = []
        for i in range(nstates):
            X = torch.from_numpy(W.initial_fields(w_main, seed=w_main.seed + 97 * i)).to(dev).to(cdt)
            h.retract(X, torch.zeros_like(X), 0.0, 1, X)     # put it on the manifold (R1 of u)
            states.append(X)
        groups = [(h, states, [w_main])]
        n_inst = 1
    for h, st, _ in groups:
        h.sync()
    # launch shapes: measured by the library's autotuner on each handle (not timed)
    if args.tiles:
        for h, _, _ in groups:
            h.set_tune(json.loads(args.tiles))
        tiles = [h.get_tune() for h, _, _ in groups]
    else:
        tiles = [h.get_tune() if args.no_autotune else h.autotune(st[0]) for h, st, _ in groups]
    bufs = [tuple(torch.empty_like(st[0]) for _ in range(3)) for _, st, _ in groups]

    def step(k):
        for (hh, st, _), (rg, hz, xt) in zip(groups, bufs):
            X = st[k % len(st)]
            hh.grad(X, G_riem=rg, sync=False)
            hh.hessvec(X, rg, hz, sigma=SIGMA, riemannian=True)
            hh.retract(X, rg, -T_TRIAL, 1, xt)
            hh.energy(xt, sync=False)

    for k in range(args.warmup):
        step(k)
    for h, _, _ in groups:
        h.sync()
    barrier()
    n0 = sum(h.launch_count() for h, _, _ in groups)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            step(k)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    launches = sum(h.launch_count() for h, _, _ in groups) - n0
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    status = max(h.sync_status() for h, _, _ in groups)
    value = world * n_inst * args.steps / (ms * 1e-3)
    clocks = clk.summary()

    # per-kernel device times (separate pass with event timing around every launch)
    for h, _, _ in groups:
        h.profile(True)
    for k in range(args.steps):
        step(k)
    prof = {}
    for h, _, _ in groups:
        for kname, (kms, kcnt) in h.profile_read().items():
            a = prof.get(kname, (0.0, 0))
            prof[kname] = (a[0] + kms, a[1] + kcnt)
        h.profile(False)
    if args.workload == "batch512":
        # roofline of the largest size class (170 instances of 256^2), profiled alone
        hh, st, _ = groups[-1]
        rg, hz, xt = bufs[-1]
        hh.profile(True)
        for k in range(args.steps):
            hh.grad(st[0], G_riem=rg, sync=False)
            hh.hessvec(st[0], rg, hz, sigma=SIGMA, riemannian=True)
            hh.retract(st[0], rg, -T_TRIAL, 1, xt)
            hh.energy(xt, sync=False)
        prof_last = hh.profile_read()
        hh.profile(False)
        roofline = roofline_of(prof_last, w_main, args.precision, hh.B, wname, peaks["fp64_gflops"])
    else:
        roofline = roofline_of(prof, w_main, args.precision, 1, wname, peaks["fp64_gflops"])

    # end-to-end through the C ABI with pinned host buffers: every call takes host
    # arrays, so the library copies inputs in and results out on its stream
    hh, st, _ = groups[-1]
    hostX = [torch.empty(st[0].shape, dtype=st[0].dtype).pin_memory() for _ in range(min(4, len(st)))]
    for i, hx in enumerate(hostX):
        hx.copy_(st[i].cpu())
    hRG, hHZ, hXT = (torch.empty_like(hostX[0]).pin_memory() for _ in range(3))

    def e2e_step(k):
        hx = hostX[k % len(hostX)]
        hh.grad(hx, G_riem=hRG)                           # H2D X; D2H grad, |grad|, E
        hh.hessvec(hx, hRG, hHZ, sigma=SIGMA, riemannian=True)   # H2D X, Z; D2H HZ
        hh.retract(hx, hRG, -T_TRIAL, 1, hXT)             # H2D U, Xi; D2H trial point
        return hh.energy(hXT)                             # H2D trial point; D2H E

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(3, args.steps // 2)
    for k in range(ne):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_dt = max_over_ranks(time.perf_counter() - t0)
    nbytes = hostX[0].numel() * hostX[0].element_size()
    e2e = {"value": world * hh.B * ne / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": 6 * nbytes, "d2h_bytes_per_step": 3 * nbytes + 3 * 16 * hh.B,
           "scope": "largest size class" if args.workload == "batch512" else "workload"}

    # mixed form on the same step (when the headline is FP64)
    mixed_value = None
    if args.precision == "fp64" and args.workload != "batch512":
        hm = sbec.Handle.from_workload(w_main, precision="mixed", stream=stream.cuda_stream)
        mst = [x.to(torch.complex64) for x in groups[0][1]]
        if not args.no_autotune:
            hm.autotune(mst[0])
        mb = tuple(torch.empty_like(mst[0]) for _ in range(3))
        save = groups[:], bufs[:]
        groups[:] = [(hm, mst, [w_main])]
        bufs[:] = [mb]
        for k in range(args.warmup):
            step(k)
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.steps):
            step(k)
        ev1.record(stream)
        ev1.synchronize()
        mixed_value = world * args.steps / (ev0.elapsed_time(ev1) * 1e-3)
        groups[:], bufs[:] = save
        hm.close()

    # time to ground state from the seeded initial state
    tts = None
    if not args.no_solve:
        tts = time_to_ground_state(args, sbec, torch, dev, stream, groups, w_main)
    paper = None
    if not args.no_solve and args.workload == "spin2_2d" and args.precision == "fp64":
        paper = paper_case(args, sbec, torch, dev, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        val, n, dt, desc, cores = cpu_sample(w_main)
        aff, total = host_cores()
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} {desc} (numpy/scipy FP64; scipy.fft workers = {cores} cores of the affinity "
                         f"mask, {total} on the host)"
                         + (" (one 256^2 instance of the batch)" if args.workload == "batch512" else ""),
               "seconds": dt}

    for h, _, _ in groups:
        h.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32 (FFT, pointwise) + f64 (reductions)",
                "data": "synthetic",
                "config": {"workload": wname, "F": w_main.F, "grid": list(w_main.n), "components": w_main.C,
                           "instances": n_inst,
                           "step": "grad + riemannian hessvec + R1 retract + energy",
                           "l2": f"inputs larger than L2: {nstates} resident state(s) per size class, "
                                 f"{sum(st[0].numel() * elem * len(st) for _, st, _ in groups) / 1e6:.0f} MB",
                           "parallelism": "replicas" if world > 1 else "single",
                           "tiles": {"autotuned": not (args.no_autotune or args.tiles),
                                     "shapes": [{k: v for k, v in t.items() if k != "ms"} for t in tiles]}},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "status": status, "alu_peaks_measured": peaks,
                "mixed_fp32_value": mixed_value,
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof.items())},
                "time_to_ground_state_s": (tts or {}).get("fp64", {}).get("seconds"),
                "time_to_ground_state": tts,
                "paper_case": paper}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def golden_ground_state(name):
    """The CPU oracle's ground-state energy of a workload, from the fixture the oracle's
    own script writes (tests/golden/baseline_ground_states.txt), or None."""
    path = os.path.join(ROOT, "tests", "golden", "baseline_ground_states.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if parts and not parts[0].startswith("#") and parts[0] == name:
                    return float(parts[1])
    except OSError:
        pass
    return None


def gold_report(gold, energies):
    if gold is None:
        return {"energy": None, "note": "no stored oracle ground state for this workload"}
    return {"energy": gold, **{f"{k}_rel_err": abs(v - gold) / abs(gold) for k, v in energies.items()}}


def time_to_ground_state(args, sbec, torch, dev, stream, groups, w):
    tol = solve_tol(args.workload)

    def tuned(hh, wl):
        # launch shapes of a new handle by the autotuner, from the workload's initial data
        if not args.no_autotune:
            cdt = torch.complex128 if hh.precision == "fp64" else torch.complex64
            hh.autotune(torch.from_numpy(W.initial_fields(wl)).to(dev).to(cdt))
        return hh
    if args.workload == "batch512":
        out = {"tol": tol, "classes": []}
        t_all = 0.0
        t_mix = 0.0
        for h, _, ws in groups:
            X0 = torch.from_numpy(np.stack([W.initial_fields(x) for x in ws])).to(dev).to(
                torch.complex128 if args.precision == "fp64" else torch.complex64)
            X = X0.clone()
            nb = 10 * X.numel() * X.element_size()
            ws_buf = torch.empty(nb, dtype=torch.uint8, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sts = sbec.solve_batch(h, X, tol=tol, workspace=ws_buf)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            t_all += dt
            cls = {"grid": list(ws[0].n), "instances": len(ws), "seconds": dt,
                   "converged": int(sum(s["converged"] for s in sts)),
                   "max_outer": int(max(s["outer_iters"] for s in sts)),
                   "max_inner": int(max(s["inner_iters"] for s in sts)),
                   "energies_head": [s["energy"] for s in sts[:3]]}
            # the instances of the class whose oracle ground state is stored (a seeded sample)
            gold = {x.name: golden_ground_state(x.name) for x in ws}
            cls["oracle_sample_fp64_rel_err"] = {x.name: abs(s["energy"] - gold[x.name]) / abs(gold[x.name])
                                                 for x, s in zip(ws, sts) if gold[x.name] is not None}
            del ws_buf
            if args.precision == "fp64":
                # mixed form of the same class: FP32 lock-step solve, FP64 refinement
                h32 = sbec.Handle.batch(ws, precision="mixed", stream=stream.cuda_stream)
                if not args.no_autotune:
                    h32.autotune(X0.to(torch.complex64))
                Xm = X0.clone()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sm, sf = sbec.solve_mixed(h, h32, Xm, tol=tol, tol_mixed=1e-3)
                torch.cuda.synchronize()
                dm = time.perf_counter() - t0
                t_mix += dm
                h32.close()
                cls["mixed_refined"] = {
                    "seconds": dm, "converged": int(sum(s["converged"] for s in sf)),
                    "max_energy_rel_diff": max(abs(a["energy"] - b["energy"]) / abs(b["energy"])
                                               for a, b in zip(sf, sts)),
                    "oracle_sample_rel_err": {x.name: abs(s["energy"] - gold[x.name]) / abs(gold[x.name])
                                              for x, s in zip(ws, sf) if gold[x.name] is not None}}
            out["classes"].append(cls)
        out["fp64" if args.precision == "fp64" else "mixed"] = {"seconds": t_all}
        # the same solves as ONE device-driven graph launch over the three size classes
        Xs = [torch.from_numpy(np.stack([W.initial_fields(x) for x in ws])).to(dev).to(
            torch.complex128 if args.precision == "fp64" else torch.complex64) for _, _, ws in groups]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, gst = sbec.solve_graph([h for h, _, _ in groups], Xs, tol=tol)
        torch.cuda.synchronize()
        tg = time.perf_counter() - t0
        out["graph"] = {"seconds": tg, "status": rc, "launches": 1,
                        "converged": int(sum(s["converged"] for st in gst for s in st)),
                        "max_outer": int(max(s["outer_iters"] for st in gst for s in st)),
                        "energies_head": [st[0]["energy"] for st in gst]}
        del Xs
        if args.precision == "fp64":
            out["mixed_refined"] = {"seconds": t_mix}
            out["speedup_mixed_over_fp64"] = t_all / t_mix if t_mix > 0 else None
        return out
    h = groups[0][0]
    X0 = torch.from_numpy(W.initial_fields(w)).to(dev)
    def cascade(lv):
        # cascadic multigrid (Algorithm 1), coarse levels to 1e-5 (Sec. 7.1): the FP64 form
        # and the mixed form (each level: FP32 solve, FP64 refinement with FP32 Newton CG)
        hf = h if args.precision == "fp64" else tuned(sbec.Handle.from_workload(w, stream=stream.cuda_stream), w)
        hs = [tuned(sbec.Handle.from_workload(x, stream=stream.cuda_stream), x) for x in lv[:-1]] + [hf]
        hm = [tuned(sbec.Handle.from_workload(x, precision="mixed", stream=stream.cuda_stream), x) for x in lv]

        def states():
            return [torch.from_numpy(W.initial_fields(lv[0])).to(dev)] + [
                torch.empty((x.C,) + x.shape, dtype=torch.complex128, device=dev) for x in lv[1:]]
        ws = torch.empty(10 * w.C * w.G * 16 + 11 * w.C * w.G * 8, dtype=torch.uint8, device=dev)
        st64 = states()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64 = sbec.solve_cascadic(hs, st64, tol=tol, workspace=ws, maxit=args.solve_maxit)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        stm = states()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sm, sf = sbec.solve_cascadic_mixed(hs, hm, stm, tol=tol, workspace=ws, maxit=args.solve_maxit)
        torch.cuda.synchronize()
        tmx = time.perf_counter() - t0
        for x in hs[:-1] + hm:
            x.close()
        if hf is not h:
            hf.close()
        gold = golden_ground_state(w.name)
        return {"tol": tol, "levels": [list(x.n) for x in lv], "maxit": args.solve_maxit,
                "fp64": {"seconds": t64, "energy": s64["energy"], "grad_norm": s64["grad_norm"],
                         "outer": s64["outer_iters"], "inner": s64["inner_iters"], "rgbb": s64["rgbb_iters"],
                         "n_hvp": s64["n_hvp"], "converged": bool(s64["converged"])},
                "mixed_refined": {"seconds": tmx, "energy": sf["energy"], "grad_norm": sf["grad_norm"],
                                  "finest_mixed_phase": {k: sm[k] for k in ("outer_iters", "inner_iters",
                                                                            "rgbb_iters", "n_hvp")},
                                  "finest_fp64_phase": {k: sf[k] for k in ("outer_iters", "inner_iters",
                                                                           "rgbb_iters", "n_hvp")},
                                  "converged": bool(sf["converged"])},
                "speedup_mixed_over_fp64": t64 / tmx if tmx > 0 else None,
                "energy_rel_diff": abs(sf["energy"] - s64["energy"]) / abs(s64["energy"]),
                "oracle": gold_report(gold, {"fp64": s64["energy"], "mixed_refined": sf["energy"]})}

    if w.levels:
        return cascade([w.at(n) for n in w.levels] + [w])
    nb64 = 10 * X0.numel() * 16
    ws = torch.empty(nb64 + 11 * X0.numel() * 8, dtype=torch.uint8, device=dev)
    hf = h if args.precision == "fp64" else tuned(sbec.Handle.from_workload(w, stream=stream.cuda_stream), w)
    hm2 = tuned(sbec.Handle.from_workload(w, precision="mixed", stream=stream.cuda_stream), w)
    X = X0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s64 = hf.solve(X, tol=tol, workspace=ws)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    Xm = X0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sm, sf = sbec.solve_mixed(hf, hm2, Xm, tol=tol, tol_mixed=1e-3, workspace=ws)
    torch.cuda.synchronize()
    tmx = time.perf_counter() - t0
    hm2.close()
    if hf is not h:
        hf.close()
    out = {"tol": tol,
            "fp64": {"seconds": t64, "energy": s64["energy"], "grad_norm": s64["grad_norm"],
                     "outer": s64["outer_iters"], "inner": s64["inner_iters"], "rgbb": s64["rgbb_iters"],
                     "n_grad": s64["n_grad"], "n_hvp": s64["n_hvp"], "n_energy": s64["n_energy"],
                     "converged": bool(s64["converged"])},
            "mixed_refined": {"seconds": tmx, "energy": sf["energy"], "grad_norm": sf["grad_norm"],
                              "mixed_phase": {k: sm[k] for k in ("outer_iters", "inner_iters", "rgbb_iters",
                                                                 "n_hvp")},
                              "fp64_phase": {k: sf[k] for k in ("outer_iters", "inner_iters", "rgbb_iters",
                                                                "n_hvp")},
                              "converged": bool(sf["converged"])},
            "speedup_mixed_over_fp64": t64 / tmx if tmx > 0 else None,
            "energy_rel_diff": abs(sf["energy"] - s64["energy"]) / abs(s64["energy"]),
            "oracle": gold_report(golden_ground_state(w.name), {"fp64": s64["energy"], "mixed_refined": sf["energy"]})}
    if w.dim >= 2:
        # the same ground state by Algorithm 1 itself: the single-mesh solve above spends
        # most of its Newton iterations where the modified CG stops at its cap; from the
        # cascadic levels n/4, n/2 the finest level starts close to the minimiser
        out["cascadic"] = cascade([w.at(tuple(v // c for v in w.n)) for c in (4, 2)] + [w])
    return out


# The paper's spin-2 2D case (Sec. 7.1, table of spin-2 results in 2D, ARNT with R1):
# printed energy f and time in seconds (MATLAB R2018b on 12 Xeon E5-2680 v3 cores)
PAPER_SPIN2_2D = {0.0: (14.3386, 8.3), 0.5: (14.3730, 13.5), 1.5: (14.6754, 13.5)}
# and its spin-1 2D case (table of spin-1 results in 2D, ARNT with R1)
PAPER_SPIN1_2D = {0.0: (15.1032, 17.0), 0.2: (15.1411, 19.9), 0.5: (15.3436, 27.2), 0.9: (15.9621, 23.8)}


def paper_case(args, sbec, torch, dev, stream):
    """Context: the paper's spin-2 and spin-1 2D solves (cascadic from n/4 and n/2, R1,
    the paper's tolerances 1e-5 / 1e-6 and initial spinors) timed on this GPU next to
    the paper's printed energies and CPU times."""
    runs = []
    cases = [("spin-2 2D 256^2", W.paper_spin2_2d, (64, 128, 256), M, e, t) for M, (e, t) in PAPER_SPIN2_2D.items()]
    cases += [("spin-1 2D 512^2", W.paper_spin1_2d, (128, 256, 512), M, e, t) for M, (e, t) in PAPER_SPIN1_2D.items()]
    for name, make, levels, M, e_printed, t_paper in cases:
        ws = [make(M, n) for n in levels]
        hs = [sbec.Handle.from_workload(w, stream=stream.cuda_stream) for w in ws]
        for h, w in zip(hs, ws):
            if not args.no_autotune:
                h.autotune(torch.from_numpy(W.paper_initial(w)).to(dev))
        states = [torch.from_numpy(W.paper_initial(ws[0])).to(dev)] + [
            torch.empty((ws[0].C,) + w.shape, dtype=torch.complex128, device=dev) for w in ws[1:]]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sbec.solve_cascadic(hs, states, tol=1e-6, tol_coarse=1e-5)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for h in hs:
            h.close()
        runs.append({"case": name, "M": M, "seconds": dt, "energy": st["energy"], "grad_norm": st["grad_norm"],
                     "paper_energy": e_printed, "paper_seconds": t_paper,
                     "speedup_vs_paper": t_paper / dt if dt > 0 else None})
    return {"cases": "paper Sec. 7.1: spin-2 2D 256^2 x 5, beta = (243, 12.1, -13), [-8,8]^2; "
                     "spin-1 2D 512^2 x 3, beta = (300, 100), [-16,16]^2",
            "paper_hardware": "MATLAB R2018b, 12 x Intel Xeon E5-2680 v3 (context, not the target)",
            "runs": runs}


# The paper's algorithm comparison (Sec. 7.1, tables of ARNT / RGBB with the retractions
# R1 / R2 / R3, the comparison system RTR left out): its spin-2 2D case, columns f, nrmG,
# iter, time; for ARNT "iter" is outer iterations (average inner CG iterations) on the
# finest mesh, for RGBB the RGBB iterations there.
PAPER_TABLE_M = (0.0, 0.5, 1.5)


def paper_table(args):
    """ARNT and RGBB with R1, R2, R3 on the paper's spin-2 2D case (cascadic 64^2 ->
    128^2 -> 256^2, tolerances 1e-5 / 1e-6, the paper's nematic initial spinor), timed
    on this GPU; one JSON line with every row."""
    import torch
    from paper_1907_01194_gb300 import sbec
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    rows = []
    for M in PAPER_TABLE_M:
        ws = [W.paper_spin2_2d(M, n) for n in (64, 128, 256)]
        hs = [sbec.Handle.from_workload(w, stream=stream.cuda_stream) for w in ws]
        for h, w in zip(hs, ws):
            h.autotune(torch.from_numpy(W.paper_initial(w)).to(dev))
        for method in ("arnt", "rgbb"):
            for retr in (1, 2, 3):
                states = [torch.from_numpy(W.paper_initial(ws[0])).to(dev)] + [
                    torch.empty((w.C,) + w.shape, dtype=torch.complex128, device=dev) for w in ws[1:]]
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = sbec.solve_cascadic(hs, states, tol=1e-6, tol_coarse=1e-5, method=method, retraction=retr)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if method == "arnt":
                    it = f"{st['outer_iters']} ({st['inner_iters'] / max(1, st['outer_iters']):.0f})"
                else:
                    it = f"{st['rgbb_iters']}"
                rows.append({"M": M, "method": method.upper(), "retr": f"R{retr}", "f": st["energy"],
                             "nrmG": st["grad_norm"], "iter": it, "seconds": dt, "converged": bool(st["converged"])})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        for h in hs:
            h.close()
    print(json.dumps({"paper_table": "spin-2 2D 256^2 x 5, beta = (243, 12.1, -13), [-8,8]^2 (Sec. 7.1)",
                      "rows": rows}), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.paper_table:
        return paper_table(args)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
