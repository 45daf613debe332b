"""Batch handles (many instances of one shape with their own beta, M and V in
one launch per pass) against the oracle instance by instance: energy,
Euclidean and Riemannian gradient, Hessian-vector products and retractions;
FP64 bar 1e-12 relative as for single instances."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sbec_oracle as O  # noqa: E402
from paper_1907_01194_gb300 import workloads as W  # noqa: E402
from tests.gpu_helpers import case_inputs, rel  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _batch(F, n, L, count, seed=11):
    rng = np.random.default_rng(seed)
    d = len(n)
    out = []
    for i in range(count):
        b1 = float(rng.uniform(-2, 2))
        M = float(rng.uniform(0.05, 0.9))
        lat = float(rng.uniform(0, 5))
        out.append(W.Workload(f"b{i}", F=F, n=n, lo=(-L,) * d, hi=(L,) * d,
                              beta=(float(rng.uniform(20, 120)), b1, float(rng.uniform(-3, 3)), 1.0), M=M,
                              lattice_amp=lat, lattice_k=math.pi / 2, seed=1000 + i))
    return out


@pytest.mark.parametrize("F,n,L,count", [(1, (64, 32), 8.0, 5), (2, (128,), 10.0, 3), (3, (16, 8, 8), 5.0, 4)])
def test_batch_matches_oracle_per_instance(F, n, L, count, dev):
    from paper_1907_01194_gb300 import sbec
    ws = _batch(F, n, L, count)
    cases = [case_inputs(w, seed_z=20 + i) for i, w in enumerate(ws)]
    X = torch.from_numpy(np.stack([c[2] for c in cases])).to(dev)
    Z = torch.from_numpy(np.stack([c[3] for c in cases])).to(dev)
    Ge, Gr, H1, H2, R = (torch.empty_like(X) for _ in range(5))
    with sbec.Handle.batch(ws) as h:
        assert h.B == count
        E1 = h.energy(X)
        E2, rn = h.grad(X, G_euc=Ge, G_riem=Gr)
        h.hessvec(X, Z, H1, sigma=0.3, riemannian=False)
        h.hessvec(X, Z, H2, sigma=0.3, riemannian=True)
        h.retract(X, Gr, -1e-2, 1, R)
        h.sync()
    for i, (P, u, Xf, Zf) in enumerate(cases):
        Xm = O.from_u(P, u)
        E_ref = O.energy(P, Xm)
        assert abs(E1[i] - E_ref) <= 1e-12 * abs(E_ref)
        assert abs(E2[i] - E_ref) <= 1e-12 * abs(E_ref)
        g = O.gradient(P, Xm)
        assert rel(Ge[i].cpu().numpy(), O.to_fields(P, g)) <= 1e-12
        rg = O.rgrad(P, u, O.to_u(P, g))
        assert abs(rn[i] - np.linalg.norm(rg)) <= 1e-11 * np.linalg.norm(O.to_u(P, g))
        Zm = O.to_matrix(P, Zf)
        assert rel(H1[i].cpu().numpy(), O.to_fields(P, O.hessvec(P, Xm, Zm) + 0.3 * Zm)) <= 1e-12
        Hr = O.rhess(P, u, O.to_u(P, Zm), g=O.to_u(P, g), sigma=0.3)
        assert rel(H2[i].cpu().numpy(), O.to_fields(P, O.from_u(P, Hr))) <= 1e-11
        ref = O.retract(P, u, -1e-2 * rg, 1)
        assert rel(R[i].cpu().numpy(), O.to_fields(P, O.from_u(P, ref))) <= 1e-12


def test_batch_of_one_equals_single_handle(dev):
    from paper_1907_01194_gb300 import sbec
    w = _batch(2, (32, 16), 6.0, 1)[0]
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    G1, G2 = torch.empty_like(X), torch.empty_like(X)
    with sbec.Handle.from_workload(w) as h1, sbec.Handle.batch([w]) as hb:
        a = h1.grad(X, G_riem=G1)
        b = hb.grad(X, G_riem=G2)
    assert a == b
    assert torch.equal(G1, G2)


@pytest.mark.parametrize("F,n,L,count", [(1, (64,), 8.0, 4), (1, (16, 16), 6.0, 3)])
def test_batch_solve_matches_oracle_per_instance(F, n, L, count, dev):
    # a14: many instances with their own beta and M solved together (lock step)
    from paper_1907_01194_gb300 import sbec
    ws = _batch(F, n, L, count, seed=5)
    X0 = np.stack([W.initial_fields(w) for w in ws])
    X = torch.from_numpy(X0).to(dev)
    with sbec.Handle.batch(ws) as h:
        sts = sbec.solve_batch(h, X, tol=1e-9)
    for i, w in enumerate(ws):
        P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)
        Xs, ost, _ = O.solve(P, O.to_matrix(P, X0[i]), O.SolveOptions(tol=1e-9))
        assert sts[i]["converged"] and ost.converged
        assert abs(sts[i]["energy"] - ost.energy) <= 1e-10 * abs(ost.energy)
        m = np.sum(np.abs(X[i].cpu().numpy().reshape(w.C, -1)) ** 2, axis=1)
        assert abs(m.sum() - 1) < 1e-12 and abs(m @ np.arange(w.F, -w.F - 1, -1) - w.M) < 1e-12


def test_batch_mixed_solve_with_fp64_refinement(dev):
    # a13 x a14: FP32 lock-step batch solve, then FP64 refinement of every instance;
    # refined energies meet the FP64 oracle's to 1e-10 relative
    from paper_1907_01194_gb300 import sbec
    ws = _batch(1, (32, 32), 7.0, 4, seed=8)
    X0 = np.stack([W.initial_fields(w) for w in ws])
    X = torch.from_numpy(X0).to(dev)
    with sbec.Handle.batch(ws) as h64, sbec.Handle.batch(ws, precision="mixed") as h32:
        sm, sf = sbec.solve_mixed(h64, h32, X, tol=1e-9, tol_mixed=1e-3)
    assert len(sm) == len(sf) == len(ws)
    for i, w in enumerate(ws):
        P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)
        Xs, ost, _ = O.solve(P, O.to_matrix(P, X0[i]), O.SolveOptions(tol=1e-9))
        assert sf[i]["converged"] and ost.converged
        assert abs(sf[i]["energy"] - ost.energy) <= 1e-10 * abs(ost.energy)
