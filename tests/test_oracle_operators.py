"""Pins of the oracle's discrete operators against things other than itself:
printed explicit formulas, commutation relations, dense DFT matrices, closed
forms of Gaussian integrals and finite differences."""
import math

import numpy as np
import pytest

from oracle import sbec_oracle as O
from paper_1907_01194_gb300 import workloads as W
from tests.oracle_helpers import oracle_problem, small_workload

rng = np.random.default_rng(1234)


def crandn(*shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- Sec. 2 matrices

@pytest.mark.parametrize("F", [1, 2, 3, 4, 5])
def test_spin_algebra(F):
    fx, fy, fz = O.spin_matrices(F)
    for f in (fx, fy, fz):
        assert np.allclose(f, f.conj().T, atol=1e-15)
    assert np.allclose(fx @ fy - fy @ fx, 1j * fz, atol=1e-14)
    assert np.allclose(fy @ fz - fz @ fy, 1j * fx, atol=1e-14)
    assert np.allclose(fx @ fx + fy @ fy + fz @ fz, F * (F + 1) * np.eye(2 * F + 1), atol=1e-13)


@pytest.mark.parametrize("F", [1, 2, 3])
def test_general_spin_matrices_are_the_printed_ones(F):
    # the construction used for F >= 4 reproduces the matrices printed in Sec. 2
    for a, b in zip(O.spin_matrices_general(F), O.spin_matrices(F)):
        assert np.allclose(a, b, atol=1e-15)


def _rotation(F, theta, axis):
    # exp(-i theta f_axis) of the printed / general spin matrices
    f = O.spin_matrices(F)[axis]
    w, V = np.linalg.eigh(f)
    return V @ np.diag(np.exp(-1j * theta * w)) @ V.conj().T


@pytest.mark.parametrize("F", [2, 3, 4, 5])
def test_singlet_pair_is_rotation_invariant(F):
    # A00 = Phi^T A Phi is the amplitude of the total-spin-0 pair: a spin rotation
    # R = exp(-i theta f) leaves it unchanged (R^T A R = A), and the matrices of
    # F = 2, 3 are the printed ones
    A = O.singlet_matrix(F)
    for axis, th in ((0, 0.7), (1, -1.3), (2, 2.1)):
        R = _rotation(F, th, axis)
        assert np.allclose(R.T @ A @ R, A, atol=1e-12)
    assert abs(np.linalg.norm(A) - 1.0) < 1e-14


def test_spin1_explicit_F():
    # Eq. (2.3): explicit F_x, F_y, F_z of a spin-1 spinor
    fx, fy, fz = O.spin_matrices(1)
    p1, p0, pm = crandn(3)
    Phi = np.array([p1, p0, pm])
    Fx = (np.conj(p1) * p0 + np.conj(p0) * (p1 + pm) + np.conj(pm) * p0) / math.sqrt(2)
    Fy = 1j / math.sqrt(2) * (-np.conj(p1) * p0 + np.conj(p0) * (p1 - pm) + np.conj(pm) * p0)
    Fz = abs(p1) ** 2 - abs(pm) ** 2
    for f, ref in ((fx, Fx), (fy, Fy), (fz, Fz)):
        assert abs(np.conj(Phi) @ f @ Phi - ref) < 1e-14


def test_spin2_explicit_F_and_A00():
    fx, fy, fz = O.spin_matrices(2)
    p2, p1, p0, pm1, pm2 = crandn(5)
    Phi = np.array([p2, p1, p0, pm1, pm2])
    c = np.conj
    s = math.sqrt(6) / 2
    Fx = (c(p2) * p1 + c(p1) * p2 + c(pm1) * pm2 + c(pm2) * pm1
          + s * (c(p1) * p0 + c(p0) * p1 + c(p0) * pm1 + c(pm1) * p0))
    Fy = 1j * (c(p1) * p2 - c(p2) * p1 + c(pm2) * pm1 - c(pm1) * pm2
               + s * (c(p0) * p1 - c(p1) * p0 + c(pm1) * p0 - c(p0) * pm1))
    Fz = 2 * abs(p2) ** 2 + abs(p1) ** 2 - abs(pm1) ** 2 - 2 * abs(pm2) ** 2
    for f, ref in ((fx, Fx), (fy, Fy), (fz, Fz)):
        assert abs(c(Phi) @ f @ Phi - ref) < 1e-13
    A00 = (2 * p2 * pm2 - 2 * p1 * pm1 + p0 ** 2) / math.sqrt(5)
    assert abs(Phi @ O.singlet_matrix(2) @ Phi - A00) < 1e-14


def test_spin3_explicit_F_A00_A2l():
    fx, fy, fz = O.spin_matrices(3)
    psi = crandn(7)
    p = {l: psi[3 - l] for l in range(-3, 4)}
    c = np.conj
    Fp = (math.sqrt(6) * c(p[3]) * p[2] + math.sqrt(10) * c(p[2]) * p[1]
          + 2 * math.sqrt(3) * c(p[1]) * p[0] + 2 * math.sqrt(3) * c(p[0]) * p[-1]
          + math.sqrt(10) * c(p[-1]) * p[-2] + math.sqrt(6) * c(p[-2]) * p[-3])
    Fz = sum(l * abs(p[l]) ** 2 for l in range(-3, 4))
    assert abs(c(psi) @ (fx + 1j * fy) @ psi - Fp) < 1e-13
    assert abs(c(psi) @ fz @ psi - Fz) < 1e-13
    r7, r21 = math.sqrt(7), math.sqrt(21)
    A00 = (2 * p[3] * p[-3] - 2 * p[2] * p[-2] + 2 * p[1] * p[-1] - p[0] ** 2) / r7
    assert abs(psi @ O.singlet_matrix(3) @ psi - A00) < 1e-14
    Aq = O.quintet_matrices(3)
    A20 = (5 * p[3] * p[-3] - 3 * p[1] * p[-1] + math.sqrt(2) * p[0] ** 2) / r21
    assert abs(psi @ Aq[0] @ psi - A20) < 1e-14
    for s in (1, -1):
        A21 = (5 * p[3 * s] * p[-2 * s] - math.sqrt(15) * p[2 * s] * p[-s]
               + math.sqrt(2) * p[s] * p[0]) / r21
        assert abs(psi @ Aq[s] @ psi - A21) < 1e-14
        # A_{2,+-2}: explicit formula with the psi_{+-1}^2 coefficient of the printed
        # unit vector a_{+-2} (sqrt6/sqrt21); the explicit formula prints sqrt2/sqrt21.
        A22 = (math.sqrt(10) * p[3 * s] * p[-s] - math.sqrt(20) * p[2 * s] * p[0]
               + math.sqrt(6) * p[s] ** 2) / r21
        assert abs(psi @ Aq[2 * s] @ psi - A22) < 1e-14


def test_spin3_quintet_vectors_unit_norm():
    # the printed vectors a_{+-1}, a_{+-2} have unit norm (the reading for A_{+-2} keeps it)
    Aq = O.quintet_matrices(3)
    for l in (1, 2, -1, -2):
        assert abs(np.sum(Aq[l] ** 2) - 1.0) < 1e-14
        assert np.allclose(Aq[l], Aq[l].T)
    # every pair matrix couples only m + m' = l (indices j + k = 8 - l, 1-based)
    for l, A in Aq.items():
        j, k = np.nonzero(A)
        assert np.all((j + 1) + (k + 1) == 8 - l)


# ---------------------------------------------------------------- Sec. 3 Laplacian

@pytest.mark.parametrize("n,lo,hi", [((8,), (-2.0,), (3.0,)), ((16,), (-8.0,), (8.0,)),
                                     ((8, 16), (-1.0, -4.0), (2.0, 4.0)),
                                     ((8, 8, 16), (-2.0, -3.0, -1.0), (2.0, 1.0, 4.0))])
def test_laplacian_matches_dense_dft(n, lo, hi):
    G = int(np.prod(n))
    P = O.Problem(F=1, n=n, lo=lo, hi=hi, beta=(0,), V=np.zeros(G))
    X = crandn(G, 3)
    L = O.dense_laplacian(P)
    assert np.allclose(L, L.conj().T, atol=1e-12)
    ref = L @ X
    got = O.laplacian(P, X)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_laplacian_at_matches_dense_rows():
    # the point-sampled Laplacian against rows of the brute-force dense matrix
    n, lo, hi = (8, 4, 16), (-2.0, -3.0, -1.0), (2.0, 1.0, 4.0)
    G = int(np.prod(n))
    P = O.Problem(F=1, n=n, lo=lo, hi=hi, beta=(0,), V=np.zeros(G))
    X = crandn(G, 3)
    idx = np.array([0, 5, 77, 130, G - 1, 311])
    ref = (O.dense_laplacian(P) @ X)[idx]
    got = O.laplacian_at(P, X, idx)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("F", [1, 2, 3])
def test_gradient_and_hessvec_at_points_match_full(F):
    # rows of the full Eq. (3.12)/(3.13) results (pinned by finite differences below)
    n = (8, 4, 16)
    G = int(np.prod(n))
    P = O.Problem(F=F, n=n, lo=(-3.0, -2.0, -4.0), hi=(3.0, 2.0, 4.0), beta=(30.0, -2.0, 5.0, 1.5),
                  V=rng.uniform(0, 3, G), p=0.3, q=0.2, M=0.1)
    X = crandn(G, P.C) * 0.1
    Z = crandn(G, P.C)
    idx = np.array([3, 64, 100, 257, G - 2])
    g, H = O.gradient(P, X), O.hessvec(P, X, Z)
    assert np.max(np.abs(O.gradient_at(P, X, idx) - g[idx])) <= 1e-12 * np.max(np.abs(g))
    assert np.max(np.abs(O.hessvec_at(P, X, Z, idx) - H[idx])) <= 1e-12 * np.max(np.abs(H))


def test_laplacian_plane_wave_eigenvalue():
    # -d^2/dx^2 of e^{i lambda_p (x - a)} is lambda_p^2 exactly, the Nyquist mode included
    n, a, b = 16, -3.0, 5.0
    P = O.Problem(F=1, n=(n,), lo=(a,), hi=(b,), beta=(0,), V=np.zeros(n))
    x = P.grid_axes()[0]
    for p in range(-n // 2, n // 2):
        lam = 2 * math.pi * p / (b - a)
        col = np.exp(1j * lam * (x - a))
        out = O.laplacian(P, np.stack([col] * 3, axis=1))
        assert np.allclose(out[:, 0], lam ** 2 * col, atol=1e-11)


# ---------------------------------------------------------------- Sec. 3 energy

def _gaussian_energy_closed_form(F, d, U, beta, p, q, lattice_amp, lattice_k):
    """E of Phi = U pi^{-d/4} exp(-|x|^2/2) with |U| = 1, V = |x|^2/2 + A sum sin^2(k x_i),
    from the explicit spin / pair formulas (not the oracle's matrices)."""
    ls = np.arange(F, -F - 1, -1)
    E = d / 2.0
    E += np.sum((-p * ls + q * ls ** 2) * np.abs(U) ** 2)
    E += d * lattice_amp * (1 - math.exp(-lattice_k ** 2)) / 2
    c = np.conj
    u = {l: U[F - l] for l in ls}
    if F == 1:
        Fx = (c(u[1]) * u[0] + c(u[0]) * (u[1] + u[-1]) + c(u[-1]) * u[0]) / math.sqrt(2)
        Fy = 1j / math.sqrt(2) * (-c(u[1]) * u[0] + c(u[0]) * (u[1] - u[-1]) + c(u[-1]) * u[0])
        F2 = abs(Fx) ** 2 + abs(Fy) ** 2 + (abs(u[1]) ** 2 - abs(u[-1]) ** 2) ** 2
        A2 = 0.0
        Q2 = 0.0
    else:
        cm = lambda m: math.sqrt(F * (F + 1) - m * (m + 1))
        Fp = sum(cm(m) * c(u[m + 1]) * u[m] for m in range(-F, F))
        Fz = sum(l * abs(u[l]) ** 2 for l in ls)
        F2 = abs(Fp) ** 2 + Fz ** 2
        if F == 2:
            A2 = abs((2 * u[2] * u[-2] - 2 * u[1] * u[-1] + u[0] ** 2) / math.sqrt(5)) ** 2
            Q2 = 0.0
        elif F >= 4:
            # singlet pair amplitude sum_l (-1)^(F-l) u_l u_-l / sqrt(2F+1); no quintet term
            A2 = abs(sum((-1) ** (F - l) * u[l] * u[-l] for l in ls) / math.sqrt(2 * F + 1)) ** 2
            Q2 = 0.0
        else:
            r21 = math.sqrt(21)
            A2 = abs((2 * u[3] * u[-3] - 2 * u[2] * u[-2] + 2 * u[1] * u[-1] - u[0] ** 2)
                     / math.sqrt(7)) ** 2
            Q2 = abs((5 * u[3] * u[-3] - 3 * u[1] * u[-1] + math.sqrt(2) * u[0] ** 2) / r21) ** 2
            for s in (1, -1):
                Q2 += abs((5 * u[3 * s] * u[-2 * s] - math.sqrt(15) * u[2 * s] * u[-s]
                           + math.sqrt(2) * u[s] * u[0]) / r21) ** 2
                Q2 += abs((math.sqrt(10) * u[3 * s] * u[-s] - math.sqrt(20) * u[2 * s] * u[0]
                           + math.sqrt(6) * u[s] ** 2) / r21) ** 2
    b0, b1, b2, b3 = beta
    E += (2 * math.pi) ** (-d / 2) * (b0 / 2 + b1 / 2 * F2 + b2 / 2 * A2 + b3 / 2 * Q2)
    return float(np.real(E))


@pytest.mark.parametrize("F,n,L", [(1, (128,), 16.0), (2, (64, 64), 8.0), (3, (128,), 16.0),
                                   (3, (64, 64, 64), 8.0), (4, (64, 64), 8.0), (5, (128,), 16.0)])
def test_energy_gaussian_closed_form(F, n, L):
    d = len(n)
    beta = (37.0, -3.0, 5.0, 2.5)
    p, q, A, k = 0.3, 0.7, 4.0, math.pi / 2
    w = W.Workload("g", F=F, n=n, lo=(-L,) * d, hi=(L,) * d, beta=beta, M=0.0, p=p, q=q,
                   lattice_amp=A, lattice_k=k)
    P = oracle_problem(w)
    U = crandn(2 * F + 1)
    U /= np.linalg.norm(U)
    r2 = sum(np.meshgrid(*[x ** 2 for x in reversed(P.grid_axes())], indexing="ij"))
    phi = np.pi ** (-d / 4) * np.exp(-r2 / 2)
    X = math.sqrt(P.dV) * phi.reshape(-1)[:, None] * U[None, :]
    ref = _gaussian_energy_closed_form(F, d, U, beta, p, q, A, k)
    assert abs(O.energy(P, X) - ref) <= 1e-12 * abs(ref)
    assert abs(O.constraints(P, X)[0] - 1.0) < 1e-13


def _fd_case(F, n, beta, seed):
    w = small_workload(F, n, beta=beta, lattice=3.0, p=0.2, q=-0.1)
    P = oracle_problem(w)
    X = O.to_matrix(P, W.initial_fields(w, seed))
    D = O.to_matrix(P, W.smooth_random_fields(w, seed + 1))
    return P, X, D


@pytest.mark.parametrize("F", [1, 2, 3, 4])
@pytest.mark.parametrize("term", [0, 1, 2, 3, None])
def test_gradient_central_fd(F, term):
    beta = (40.0, -3.0, 6.0, -2.0) if term is None else tuple(25.0 * (i == term) for i in range(4))
    P, X, D = _fd_case(F, (24, 16), beta, 11)
    eps = 1e-6
    fd = (O.energy(P, X + eps * D) - O.energy(P, X - eps * D)) / (2 * eps)
    an = np.real(np.sum(O.gradient(P, X) * np.conj(D)))
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


@pytest.mark.parametrize("F", [1, 2, 3, 4])
@pytest.mark.parametrize("term", [0, 1, 2, 3, None])
def test_hessvec_central_fd_and_symmetry(F, term):
    beta = (40.0, -3.0, 6.0, -2.0) if term is None else tuple(25.0 * (i == term) for i in range(4))
    P, X, Z = _fd_case(F, (16, 24), beta, 21)
    eps = 1e-6
    fd = (O.gradient(P, X + eps * Z) - O.gradient(P, X - eps * Z)) / (2 * eps)
    H = O.hessvec(P, X, Z)
    assert np.linalg.norm(fd - H) <= 1e-7 * np.linalg.norm(H)
    Z2 = O.to_matrix(P, W.random_fields((P.C,) + P.shape, 99))
    lhs = np.real(np.vdot(Z2, H))            # Re<H[Z], Z2> (conjugate-symmetric form)
    rhs = np.real(np.vdot(O.hessvec(P, X, Z2), Z))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_energy_symmetry_flip_components():
    # Sec. 4: with p = 0, E is invariant under phi_l <-> phi_{-l}
    for F in (1, 2, 3, 4):
        w = small_workload(F, (32,), beta=(30.0, -2.0, 4.0, 1.5), q=0.4)
        P = oracle_problem(w)
        X = O.to_matrix(P, W.random_fields((P.C,) + P.shape, 5, 0.1))
        assert abs(O.energy(P, X) - O.energy(P, X[:, ::-1])) < 1e-12 * abs(O.energy(P, X))
