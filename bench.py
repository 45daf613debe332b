"""Benchmark of the spin-F BEC hot path on one (or N replicated) GB300.

Workload: spin-2, 2D, 256 x 256 on [-12,12]^2, V = |x|^2/2 + 20 sum sin^2(pi x_i/2),
beta = (200, 10, -5), M = 0.3 (synthetic; seeded Gaussian-times-noise states put on
the constraint manifold by the library's own projective retraction).

One step = one pass of the hot path as a Newton/BB iteration uses it:
  sbec_grad     energy, Euclidean and Riemannian gradient, ||grad E|| (Eq. 3.7, 3.12, Lemma 4.1)
  sbec_hessvec  Riemannian Hessian-vector product along the gradient (Eq. 3.13, Lemma 4.2)
  sbec_retract  projective retraction of a trial step (Lemma 5.1)
  sbec_energy   energy of the trial point
Each step works on a different one of 32 resident states (168 MB > the 129 MB L2),
so no step reads its inputs from L2 left by the previous one.

metric value = energy+grad evaluations per second (one per step) over all ranks.
`--impl reference` times the CPU FP64 oracle doing the same step.
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

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1907_01194_gb300 import workloads as W  # noqa: E402

METRIC = "energy+grad evals/s and time-to-ground-state (|Rgrad|<1e-8), % HBM roofline"
UNIT = "evals/s"
NSTATES = 32
T_TRIAL = 1e-3
SIGMA = 0.5

# FP64 ALU peak: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (the recipe's unit counts and
# maximum SM clock); the FMA probe measured 1.195 TFLOP/s on this machine's GB300.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# pointwise FLOPs per grid point of the epilogues (counted from Eq. 3.7, 3.12, 3.13 in the
# ladder / pair form the kernels use; the derivation is in the design doc)
PW_FLOPS = {"grad": {1: 170, 2: 375, 3: 760}, "hess": {1: 300, 2: 640, 3: 1400},
            "energy": {1: 70, 2: 140, 3: 290}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-ground-state solves")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload():
    return W.spin2_2d()


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
        z = O.retract(P, u, -T_TRIAL * rg, 1)
        O.E_u(P, z)
        return E
    return step


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    w = workload()
    step = oracle_step_runner(w)
    for _ in range(max(1, min(args.warmup, 1))):
        step()
    t0 = time.perf_counter()
    n = 0
    budget = 120.0
    while n < args.steps:
        step()
        n += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    val = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * dt / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "F": w.F, "grid": list(w.n), "components": w.C,
                       "parallelism": "replicas" if args.gpus > 1 else "single"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n} full steps of the {w.name} workload (numpy/scipy FP64, "
                                       "one thread)"},
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


def flops_model(w, kname, launches):
    """Algorithmic FLOPs of one launch kind (per launch) for the workload."""
    C, n = w.C, w.n
    G = int(np.prod(n))
    fft = lambda m: 5.0 * m * math.log2(m)
    if kname == "s_k2":
        m = n[-1]
        return C * (G // m) * (2 * fft(m) + 4 * m)
    if kname in ("s_fwd", "s_inv", "s_parseval"):
        m = n[1]
        return C * (G // m) * fft(m)
    if kname == "x_fwd":
        return C * (G // n[0]) * fft(n[0])
    if kname == "x_fwd_energy":
        return C * (G // n[0]) * fft(n[0]) + G * PW_FLOPS["energy"][w.F]
    if kname == "x_inv_grad":
        return C * (G // n[0]) * fft(n[0]) + G * PW_FLOPS["grad"][w.F]
    if kname == "x_inv_hess":
        return C * (G // n[0]) * fft(n[0]) + G * PW_FLOPS["hess"][w.F]
    return None


def bytes_model(w, kname, elem):
    """Algorithmic DRAM bytes of one launch (compulsory reads + writes)."""
    C, G = w.C, int(np.prod(w.n))
    S = C * G * elem
    SV = G * elem // 2
    return {"x_fwd": 2 * S, "x_fwd_energy": 2 * S + SV, "s_k2": 2 * S, "s_fwd": 2 * S, "s_inv": 2 * S,
            "s_parseval": S, "x_inv_grad": 3 * S + SV, "x_inv_hess": 4 * S + SV,
            "proj_apply": 3 * S, "dot_reduce": 2 * S, "retract_w": 3 * S, "scale": 2 * S}.get(kname)


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

    w = workload()
    stream = torch.cuda.current_stream()
    h = sbec.Handle.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    states = []
    for i in range(NSTATES):
        X = torch.from_numpy(W.initial_fields(w, seed=w.seed + 97 * i)).to(dev)
        h.retract(X, torch.zeros_like(X), 0.0, 1, X)     # put it on the manifold (R1 of u)
        states.append(X)
    h.sync()
    RG = torch.empty_like(states[0])
    HZ = torch.empty_like(states[0])
    XT = torch.empty_like(states[0])

    def step(k, hh=h, st=states, rg=RG, hz=HZ, xt=XT):
        X = st[k % len(st)]
        hh.grad(X, G_riem=rg, sync=False)
        hh.hessvec(X, rg, hz, sigma=SIGMA, riemannian=True)
        hh.retract(X, rg, -T_TRIAL, 1, xt)
        hh.energy(xt, sync=False)

    for k in range(args.warmup):
        step(k)
    h.sync()
    barrier()
    n0 = h.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            step(k)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    launches = h.launch_count() - n0
    ms = ev0.elapsed_time(ev1)
    status = h.sync_status()
    if pg:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.steps / (ms * 1e-3)
    clocks = clk.summary()

    # per-kernel device times (separate pass with event timing around every launch)
    h.profile(True)
    for k in range(args.steps):
        step(k)
    prof = h.profile_read()
    h.profile(False)
    total = sum(v[0] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][0])
    kname, (kms, kcnt) = top
    per_launch_s = kms / kcnt * 1e-3
    fl = flops_model(w, kname, kcnt)
    roofline = {"bound": "alu", "achieved": fl / per_launch_s / 1e9 if fl else None,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": (fl / per_launch_s / 1e9) / FP64_PEAK_GFLOPS if fl else None,
                "traffic": None, "kernel": kname, "kernel_share": kms / total,
                "peak_source": "FP64 nominal: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz"}

    # end-to-end through the C ABI with pinned host buffers: every call takes host
    # arrays, so the library copies inputs in and results out on its stream
    hostX = [torch.empty(states[0].shape, dtype=states[0].dtype).pin_memory() for _ in range(4)]
    for i, hx in enumerate(hostX):
        hx.copy_(states[i].cpu())
    hRG, hHZ, hXT = (torch.empty_like(hostX[0]).pin_memory() for _ in range(3))

    def e2e_step(k):
        hx = hostX[k % 4]
        h.grad(hx, G_riem=hRG)                            # H2D X; D2H grad E, |grad|, E
        h.hessvec(hx, hRG, hHZ, sigma=SIGMA, riemannian=True)   # H2D X, Z; D2H HZ
        h.retract(hx, hRG, -T_TRIAL, 1, hXT)              # H2D U, Xi; D2H trial point
        return h.energy(hXT)                              # H2D trial point; D2H E

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(3, args.steps // 2)
    for k in range(ne):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    if pg:
        t = torch.tensor([e2e_dt], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_dt = float(t.item())
    nbytes = hostX[0].numel() * hostX[0].element_size()
    e2e = {"value": world * ne / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": 6 * nbytes, "d2h_bytes_per_step": 3 * nbytes + 3 * 16}

    # mixed form (FP32 FFT and pointwise, FP64 reductions) on the same step
    hm = sbec.Handle.from_workload(w, precision="mixed", stream=stream.cuda_stream)
    mstates = [s.to(torch.complex64) for s in states]
    mRG, mHZ, mXT = (torch.empty_like(mstates[0]) for _ in range(3))
    for k in range(args.warmup):
        step(k, hm, mstates, mRG, mHZ, mXT)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(args.steps):
        step(k, hm, mstates, mRG, mHZ, mXT)
    ev1.record(stream)
    ev1.synchronize()
    mixed_value = world * args.steps / (ev0.elapsed_time(ev1) * 1e-3)
    hm.close()

    # time to ground state (|Rgrad| < 1e-8) from the seeded initial state: FP64 ARNT, and
    # the mixed form (FP32 FFT / pointwise to 1e-3) followed by FP64 refinement
    tts = None
    if not args.no_solve:
        X0 = torch.from_numpy(W.initial_fields(w)).to(dev)
        nb64 = 10 * X0.numel() * 16
        ws = torch.empty(nb64 + 11 * X0.numel() * 8, dtype=torch.uint8, device=dev)
        hm2 = sbec.Handle.from_workload(w, precision="mixed", stream=stream.cuda_stream)
        X = X0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64 = h.solve(X, tol=1e-8, workspace=ws)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        Xm = X0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sm, sf = sbec.solve_mixed(h, hm2, Xm, tol=1e-8, tol_mixed=1e-3, workspace=ws)
        torch.cuda.synchronize()
        tmx = time.perf_counter() - t0
        hm2.close()
        tts = {"fp64": {"seconds": t64, "energy": s64["energy"], "grad_norm": s64["grad_norm"],
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
               "energy_rel_diff": abs(sf["energy"] - s64["energy"]) / abs(s64["energy"])}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ostep = oracle_step_runner(w)
        ostep()
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < 15.0 and n < 50:
            ostep()
            n += 1
        dt = time.perf_counter() - t0
        cpu = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} full steps of the {w.name} workload on one host thread"}

    h.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": w.name, "F": w.F, "grid": list(w.n), "components": w.C,
                           "step": "grad + riemannian hessvec + R1 retract + energy",
                           "l2": f"inputs larger than L2: {NSTATES} resident states, "
                                 f"{NSTATES * states[0].numel() * 16 / 1e6:.0f} MB",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "status": status,
                "mixed_fp32_value": mixed_value,
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof.items())},
                "time_to_ground_state_s": tts["fp64"]["seconds"] if tts else None,
                "time_to_ground_state": tts}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
