"""Shared test helpers: oracle problems built from the seeded workloads and the
paper's Sec. 7 cases."""
import math

import numpy as np

from oracle import sbec_oracle as O
from paper_1907_01194_gb300 import workloads as W


def oracle_problem(w: W.Workload) -> O.Problem:
    return O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w),
                     p=w.p, q=w.q, M=w.M)


def small_workload(F, n, L=8.0, beta=None, M=0.3, lattice=0.0, seed=7, p=0.0, q=0.0):
    d = len(n)
    if beta is None:
        beta = (50.0, -2.0, 3.0, -1.0)
    return W.Workload(f"small_F{F}_{'x'.join(map(str, n))}", F=F, n=tuple(n), lo=(-L,) * d,
                      hi=(L,) * d, beta=tuple(beta), M=M, p=p, q=q, lattice_amp=lattice,
                      lattice_k=math.pi / 2, seed=seed)


def on_manifold(P: O.Problem, w: W.Workload, seed=None):
    """Seeded raw initial data put on M with the oracle's projective retraction."""
    X = O.to_matrix(P, W.initial_fields(w, seed))
    return O.psi_R1(P, O.to_u(P, X))


def random_tangent(P: O.Problem, u, seed, smooth_w=None):
    if smooth_w is not None:
        Z = O.to_matrix(P, W.smooth_random_fields(smooth_w, seed))
    else:
        Z = O.to_matrix(P, W.random_fields((P.C,) + P.shape, seed))
    xi = O.project(P, u, O.to_u(P, Z))
    return xi / np.linalg.norm(xi)


def paper_spin2_1d(case, M):
    """Sec. 7.2 spin-2 1D cases with the paper's initial data (Sec. 7)."""
    beta = {1: (130.6, -25.4, -125.3, 0.0), 2: (243.0, 12.1, -13.0, 0.0),
            3: (183.9, 26.8, 134.7, 0.0)}[case]
    n, L = (256, 8.0) if case == 1 else (512, 16.0)
    x = -L + 2 * L / n * np.arange(n)
    V = 0.5 * x ** 2 + 25.0 * np.sin(np.pi * x / 4) ** 2
    P = O.Problem(F=2, n=(n,), lo=(-L,), hi=(L,), beta=beta, V=V, M=M)
    m1, m2 = math.sqrt(2 + M), math.sqrt(2 - M)
    if case == 1:      # ferromagnetic spinor
        U = np.array([m1 ** 4 / 16, m1 ** 3 * m2 / 8, math.sqrt(6) * m1 ** 2 * m2 ** 2 / 16,
                      m1 * m2 ** 3 / 8, m2 ** 4 / 16])
    elif case == 2:    # nematic spinor
        U = np.array([math.sqrt(2 + M) / 2, 0, 0, 0, math.sqrt(2 - M) / 2])
    else:              # cyclic spinor
        U = np.array([math.sqrt((M + 1) / 3), 0, 0, math.sqrt((2 - M) / 3), 0])
    phi0 = np.pi ** -0.25 * np.exp(-x ** 2 / 2)
    X = math.sqrt(P.dV) * phi0[:, None] * U[None, :]
    return P, X.astype(complex)


def paper_spin3_1d(case, M, seed=0):
    """Sec. 7.3 spin-3 1D cases; the random spinor U is drawn from PCG64(seed)."""
    beta = (100.0, 1.0, -10.0, -1.0) if case == 1 else (100.0, 1.0, 10.0, 1.0)
    n, L = 256, 8.0
    x = -L + 2 * L / n * np.arange(n)
    V = 0.5 * x ** 2 + 25.0 * np.sin(np.pi * x / 4) ** 2
    P = O.Problem(F=3, n=(n,), lo=(-L,), hi=(L,), beta=beta, V=V, M=M)
    U = np.random.default_rng(seed).uniform(0, 1, 7)
    phi0 = np.pi ** -0.25 * np.exp(-x ** 2 / 2)
    X = math.sqrt(P.dV) * phi0[:, None] * U[None, :]
    return P, X.astype(complex)
