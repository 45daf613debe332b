"""Write tests/golden/baseline_ground_states.txt: the CPU oracle's ground-state
energies of the benchmark workloads (test infrastructure: this script calls
only the oracle and the seeded input generators).

Each case is solved by the oracle's own Algorithm 1 (RGBB warm start, ARNT) to
the workload's tolerance (1e-8 on ||grad||; 1e-10 for the spin-1 1D case), from
the seeded initial data of the workload, cascadically where the workload lists
coarse levels (the spin-2 2D workload also cascadically from n/4 and n/2, as a
second case).  The batched spin-1 sweep is represented by a seeded stratified
sample of three instances per grid size.  The 256^3 spin-3 workload is not
solved here: the oracle's step on it takes minutes, its solve days.

Usage: python oracle/make_ground_states.py [case ...] [--jobs J]
Cases run in parallel worker processes (spawned); each line records the host,
core count, commit and the seconds the solve took.
"""
from __future__ import annotations

import argparse
import datetime
import multiprocessing as mp
import os
import platform
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "golden", "baseline_ground_states.txt")


def batch_sample(count_per_class=3):
    """Seeded stratified sample of the 512-instance sweep: count_per_class instance
    indices of each grid size, drawn from PCG64(190701194 + 4 + 100)."""
    import numpy as np
    from paper_1907_01194_gb300 import workloads as W
    insts = W.batched_spin1_2d()
    rng = np.random.Generator(np.random.PCG64(W.SEED_BASE + 4 + 100))
    out = []
    for n in (64, 128, 256):
        idx = [i for i, w in enumerate(insts) if w.n[0] == n]
        out += sorted(int(i) for i in rng.choice(idx, size=count_per_class, replace=False))
    return out


def cases():
    from paper_1907_01194_gb300 import workloads as W
    from dataclasses import replace
    cs = {"spin1_1d_n256": (W.spin1_1d(), 1e-10),
          "spin2_2d_256x256": (W.spin2_2d(), 1e-8),
          # the same problem by Algorithm 1's cascade from the levels n/4, n/2
          "spin2_2d_256x256_cascadic": (replace(W.spin2_2d(), levels=((64, 64), (128, 128))), 1e-8),
          "spin3_3d_128cubed": (W.spin3_3d_cascadic(), 1e-8)}
    insts = W.batched_spin1_2d()
    for i in batch_sample():
        cs[insts[i].name] = (insts[i], 1e-8)
    return cs


def solve_case(name, workers):
    import numpy as np
    import scipy.fft as sfft
    from oracle import sbec_oracle as O
    from paper_1907_01194_gb300 import workloads as W
    w, tol = cases()[name]
    lv = [w.at(n) for n in w.levels] + [w]
    probs = [O.Problem(F=x.F, n=x.n, lo=x.lo, hi=x.hi, beta=x.beta, V=W.potential(x), p=x.p, q=x.q, M=x.M)
             for x in lv]
    X0 = O.to_matrix(probs[0], W.initial_fields(lv[0]))
    t0 = time.perf_counter()
    with sfft.set_workers(workers):
        X, st, _ = O.solve(probs, X0, O.SolveOptions(tol=tol))
    dt = time.perf_counter() - t0
    return (name, float(st.energy), float(st.grad_norm), int(st.outer_iters), int(st.inner_iters),
            bool(st.converged), dt, [list(x.n) for x in lv], float(np.log10(tol)))


def _solve_star(a):
    return solve_case(*a)


def _commit():
    try:
        return subprocess.run(["git", "-C", ROOT, "rev-parse", "--short", "HEAD"], capture_output=True,
                              text=True).stdout.strip() or "unknown"
    except OSError:
        return "unknown"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*")
    ap.add_argument("--jobs", type=int, default=4)
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    names = args.names or list(cases())
    workers = max(1, (os.cpu_count() or 1) // args.jobs)
    rows = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                rows[line.split()[0]] = line.rstrip("\n")
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        for r in pool.imap_unordered(_solve_star, [(n, workers) for n in names]):
            name, E, gn, outer, inner, conv, dt, levels, ltol = r
            lv = "->".join("x".join(str(v) for v in n) for n in levels)
            rows[name] = (f"{name} {E:.15f} {gn:.3e} tol=1e{ltol:.0f} converged={int(conv)} outer={outer} "
                          f"inner={inner} levels={lv} seconds={dt:.0f} host={platform.machine()} "
                          f"cores={workers} commit={_commit()} date={datetime.date.today().isoformat()}")
            print(rows[name], flush=True)
            with open(OUT, "w") as f:
                f.write("# CPU oracle ground states of the benchmark workloads (oracle/make_ground_states.py):\n"
                        "# name  E_h  ||grad||  tolerance  converged  outer/inner iterations of the finest level\n"
                        "#   levels (cascadic coarse-to-fine)  seconds  host  scipy.fft workers  commit  date\n")
                for k in sorted(rows):
                    f.write(rows[k] + "\n")


if __name__ == "__main__":
    main()
