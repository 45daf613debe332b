"""Helpers of the GPU parity tests: seeded inputs on the manifold, oracle
references, normwise relative errors."""
import numpy as np

from oracle import sbec_oracle as O
from paper_1907_01194_gb300 import workloads as W


def case_inputs(w, seed_z=5):
    """(P, u on M, X fields, Z fields): X from the seeded raw data projected with the
    oracle's R1, Z a smooth random direction."""
    P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), p=w.p, q=w.q,
                  M=w.M)
    u = O.psi_R1(P, O.to_u(P, O.to_matrix(P, W.initial_fields(w))))
    Xf = O.to_fields(P, O.from_u(P, u))
    Zf = W.smooth_random_fields(w, seed_z)
    return P, u, Xf, Zf


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
