"""Pins of the oracle's manifold geometry (Sec. 4) and retractions (Sec. 6):
tangency and idempotence, the Riemannian Hessian against its definition by
finite differences along a curve on M, the constraints after retraction, the
retraction axioms, the spin-1 special cases of Lemma 5.2 and the spin-1
quadratic form of R2."""
import math

import numpy as np
import pytest

from oracle import sbec_oracle as O
from tests.oracle_helpers import oracle_problem, on_manifold, random_tangent, small_workload


def _case(F, n=(32,), M=0.3, seed=3):
    w = small_workload(F, n, beta=(40.0, -2.0, 5.0, -1.5), M=M, lattice=2.0, seed=seed)
    P = oracle_problem(w)
    u = on_manifold(P, w)
    return w, P, u


@pytest.mark.parametrize("F,M", [(1, 0.3), (2, 0.0), (2, 1.2), (3, 0.7), (4, 2.2)])
def test_projection_tangent_idempotent(F, M):
    w, P, u = _case(F, M=M)
    Gm = O.gamma_weights(P)
    assert abs(u @ u - 1) < 1e-13 and abs(u @ (Gm * u) - M) < 1e-13
    rng = np.random.default_rng(0)
    v = rng.standard_normal(u.size)
    pv = O.project(P, u, v)
    assert abs(u @ pv) < 1e-13 * np.linalg.norm(v)
    assert abs(u @ (Gm * pv)) < 1e-13 * np.linalg.norm(v)
    assert np.linalg.norm(O.project(P, u, pv) - pv) < 1e-13 * np.linalg.norm(v)
    # the removed part lies in span{u, Gamma u} (the normal space)
    B = np.stack([u, Gm * u], axis=1)
    coef, *_ = np.linalg.lstsq(B, v - pv, rcond=None)
    assert np.linalg.norm(B @ coef - (v - pv)) < 1e-12 * np.linalg.norm(v)


@pytest.mark.parametrize("F,M", [(1, 0.4), (2, 0.5), (3, 1.1)])
def test_riemannian_hessian_matches_connection(F, M):
    # Hess f(u)[xi] = P_u(d/dt grad f(gamma(t)) at t = 0) for a curve gamma on M with
    # gamma(0) = u, gamma'(0) = xi (Eq. hess2); here gamma(t) = R1_u(t xi).
    w, P, u = _case(F, n=(24, 16), M=M)
    xi = random_tangent(P, u, 17, smooth_w=w)
    eps = 1e-5
    gp = O.rgrad(P, O.retract(P, u, eps * xi, 1))
    gm = O.rgrad(P, O.retract(P, u, -eps * xi, 1))
    fd = O.project(P, u, (gp - gm) / (2 * eps))
    H = O.rhess(P, u, xi)
    assert np.linalg.norm(H - fd) <= 1e-6 * np.linalg.norm(H)
    Gm = O.gamma_weights(P)
    assert abs(u @ H) < 1e-11 * np.linalg.norm(H) and abs(u @ (Gm * H)) < 1e-11 * np.linalg.norm(H)
    # symmetric on the tangent space
    eta = random_tangent(P, u, 18, smooth_w=w)
    a, b = eta @ O.rhess(P, u, xi), xi @ O.rhess(P, u, eta)
    assert abs(a - b) < 1e-11 * max(1.0, abs(a))


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("F,M", [(1, 0.5), (2, 0.0), (2, 1.3), (3, 0.2), (3, 2.5), (4, 0.4)])
def test_retraction_constraints_and_axioms(kind, F, M):
    w, P, u = _case(F, n=(32,), M=M)
    Gm = O.gamma_weights(P)
    xi = random_tangent(P, u, 5, smooth_w=w)
    for t in (0.3, 0.05):
        z = O.retract(P, u, t * xi, kind)
        assert abs(z @ z - 1) < 1e-12
        assert abs(z @ (Gm * z) - M) < 1e-12
    assert np.linalg.norm(O.retract(P, u, 0 * xi, kind) - u) < 1e-13      # R_u(0) = u
    # local rigidity: R_u(t xi) - (u + t xi) = O(t^2)
    e1 = np.linalg.norm(O.retract(P, u, 1e-2 * xi, kind) - (u + 1e-2 * xi))
    e2 = np.linalg.norm(O.retract(P, u, 5e-3 * xi, kind) - (u + 5e-3 * xi))
    assert 3.5 < e1 / e2 < 4.5


@pytest.mark.parametrize("F,M", [(1, 0.5), (2, 0.3), (3, 1.7)])
def test_R1_is_the_nearest_point(F, M):
    # KKT of the projection (Lemma 5.1 proof): w - z lies in the normal space
    # span{z, Gamma z}, z on M, and the multipliers give 1 - mu - l lambda > 0.
    w_, P, u = _case(F, M=M)
    rng = np.random.default_rng(3)
    w = u + 0.2 * rng.standard_normal(u.size) / math.sqrt(u.size)
    z = O.psi_R1(P, w)
    Gm = O.gamma_weights(P)
    B = np.stack([z, Gm * z], axis=1)
    coef, *_ = np.linalg.lstsq(B, w - z, rcond=None)
    assert np.linalg.norm(B @ coef - (w - z)) < 1e-11
    # z is closer to w than nearby points on M
    d0 = np.linalg.norm(z - w)
    for s in range(5):
        xi = O.project(P, z, rng.standard_normal(z.size))
        zz = O.psi_R3(P, z + 1e-3 * xi / np.linalg.norm(xi))
        assert np.linalg.norm(zz - w) >= d0 - 1e-14


def _spin1_norms(P, z):
    G = P.G
    return [np.linalg.norm(z[2 * G * c: 2 * G * (c + 1)]) for c in range(3)]


def test_R1_spin1_cases_of_lemma_5_2():
    rng = np.random.default_rng(8)
    # case (1): M = 0
    w_, P, u = _case(1, M=0.0)
    w = u + 0.1 * rng.standard_normal(u.size) / 8
    n1, n0, nm = _spin1_norms(P, w)
    t = math.sqrt(n0 ** 2 + (n1 + nm) ** 2 / 2)
    z = O.psi_R1(P, w)
    G = P.G
    ref = w.copy()
    ref[2 * G: 4 * G] = w[2 * G: 4 * G] / t
    ref[0: 2 * G] = (n1 + nm) / (2 * t * n1) * w[0: 2 * G]
    ref[4 * G: 6 * G] = (n1 + nm) / (2 * t * nm) * w[4 * G: 6 * G]
    assert np.linalg.norm(z - ref) < 1e-13
    # case (2): M > 0, w_0 = 0
    M = 0.35
    w_, P, u = _case(1, M=M)
    w = u + 0.1 * rng.standard_normal(u.size) / 8
    w[2 * G: 4 * G] = 0
    n1, n0, nm = _spin1_norms(P, w)
    z = O.psi_R1(P, w)
    ref = w.copy()
    ref[0: 2 * G] *= math.sqrt(1 + M) / (math.sqrt(2) * n1)
    ref[4 * G: 6 * G] *= math.sqrt(1 - M) / (math.sqrt(2) * nm)
    assert np.linalg.norm(z - ref) < 1e-13
    # case (3): M > 0, w_{-1} = 0
    w = u + 0.1 * rng.standard_normal(u.size) / 8
    w[4 * G: 6 * G] = 0
    n1, n0, nm = _spin1_norms(P, w)
    z = O.psi_R1(P, w)
    ref = w.copy()
    ref[2 * G: 4 * G] *= math.sqrt(1 - M) / n0
    ref[0: 2 * G] *= math.sqrt(M) / n1
    assert np.linalg.norm(z - ref) < 1e-13


def test_R2_spin1_quadratic_closed_form():
    # for F = 1, h2(t) = -(1+M) m_{-1} - M m_0 t + (1-M) m_1 t^2 (Lemma 5.3 remark)
    M = 0.45
    w_, P, u = _case(1, M=M)
    rng = np.random.default_rng(2)
    w = u + 0.3 * rng.standard_normal(u.size) / 8
    n1, n0, nm = _spin1_norms(P, w)
    m1, m0, mm = n1 ** 2, n0 ** 2, nm ** 2
    a, b, c = (1 - M) * m1, -M * m0, -(1 + M) * mm
    r = (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)
    s0 = 1 / math.sqrt(mm / r + m0 + m1 * r)
    z, r_or = O.psi_R2(P, w, return_r=True)
    assert abs(r_or - r) < 1e-13 * r
    G = P.G
    ref = w.copy()
    ref[0: 2 * G] *= s0 * math.sqrt(r)
    ref[2 * G: 4 * G] *= s0
    ref[4 * G: 6 * G] *= s0 / math.sqrt(r)
    assert np.linalg.norm(z - ref) < 1e-13
    # Bao-Lim condition sigma_1 sigma_{-1} = sigma_0^2 holds by construction


@pytest.mark.parametrize("F", [2, 3])
def test_R2_geometric_scales(F):
    # Eq. (orth): sigma_{l-1} sigma_{l+1} = sigma_l^2 and sigma_l sigma_{-l} = sigma_0^2
    w_, P, u = _case(F, M=0.6)
    rng = np.random.default_rng(4)
    w = u + 0.2 * rng.standard_normal(u.size) / 8
    z = O.psi_R2(P, w)
    G = P.G
    sig = np.array([(z[2 * G * c: 2 * G * (c + 1)] @ w[2 * G * c: 2 * G * (c + 1)])
                    / (w[2 * G * c: 2 * G * (c + 1)] @ w[2 * G * c: 2 * G * (c + 1)])
                    for c in range(P.C)])
    s = {int(l): sig[F - int(l)] for l in P.ls}
    for l in range(1, F):
        assert abs(s[l - 1] * s[l + 1] - s[l] ** 2) < 1e-13
    for l in range(1, F + 1):
        assert abs(s[l] * s[-l] - s[0] ** 2) < 1e-13


def test_R3_agrees_with_R1_to_higher_order():
    # the closed-form retraction approximates the projective one (Sec. 6.3): their
    # difference is of higher order than the O(t^2) correction of either
    w_, P, u = _case(2, M=0.4)
    xi = random_tangent(P, u, 9)
    d1 = np.linalg.norm(O.retract(P, u, 0.02 * xi, 3) - O.retract(P, u, 0.02 * xi, 1))
    d2 = np.linalg.norm(O.retract(P, u, 0.01 * xi, 3) - O.retract(P, u, 0.01 * xi, 1))
    assert d1 / d2 > 7.0


def test_outside_domain_raises():
    w_, P, u = _case(1, M=0.3)
    G = P.G
    w = u.copy()
    w[4 * G:] = 0     # only l >= 0 left: f1 = 0 < M but with w_1, w_0 ... still in Omega
    O.psi_R1(P, w)
    w[2 * G: 4 * G] = 0   # only l = 1 left: f1 = f2 = 1 > M, outside Omega
    with pytest.raises(FloatingPointError):
        O.psi_R1(P, w)
    with pytest.raises(FloatingPointError):
        O.psi_R2(P, w)
    with pytest.raises(FloatingPointError):
        O.psi_R3(P, w)
