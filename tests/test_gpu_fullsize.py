"""Parity at the benchmark workloads' full sizes, with the launch shapes the
autotuner picks (the configuration bench.py times).

* spin-2 2D 256^2 (FP64): energy, Euclidean and Riemannian gradient and both
  Hessian-vector products element by element against the oracle.
* spin-3 3D 128^3 (FP64): energy and the Euclidean and Riemannian gradient on
  the whole grid, the Hessian-vector product on sampled grid points.
* spin-3 3D 256^3 (mixed form): energy against the oracle's, gradient and
  Hessian-vector product on sampled grid points.  A row of L X needs only one
  row of each 1D operator of Eq. (3.5) and the grid lines through the point,
  so the oracle evaluates sampled rows of Eq. (3.12)/(3.13) exactly.
* the 512-instance spin-1 sweep (three batch handles, one per grid size):
  energies and gradient norms of sampled instances against the oracle.

Bars as in the parity tests: FP64 1e-12 relative (normwise for fields, over
the sample where sampled); mixed 2e-6 for energies and 2e-5 normwise for fields.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sbec_oracle as O  # noqa: E402
from paper_1907_01194_gb300 import workloads as W  # noqa: E402
from tests.gpu_helpers import rel  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _problem(w):
    return O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), p=w.p, q=w.q, M=w.M)


def _on_manifold(P, Xf):
    # the oracle's own R1 (Lemma 5.1) puts the seeded raw data on M
    u = O.psi_R1(P, O.to_u(P, O.to_matrix(P, Xf)))
    return u, O.from_u(P, u)


def _sample(G, k=160, seed=7):
    rng = np.random.default_rng(seed)
    idx = rng.choice(G, size=k, replace=False)
    return np.unique(np.concatenate([idx, [0, G // 2, G - 1]]))


def test_spin2_2d_256_fp64_elementwise(dev):
    from paper_1907_01194_gb300 import sbec
    w = W.spin2_2d()
    P = _problem(w)
    u, Xm = _on_manifold(P, W.initial_fields(w))
    Xf = O.to_fields(P, Xm)
    Zf = W.smooth_random_fields(w, 5)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Ge, Gr, H1, H2 = (torch.empty_like(X) for _ in range(4))
    with sbec.Handle.from_workload(w) as h:
        h.autotune(X)
        E, rn = h.grad(X, G_euc=Ge, G_riem=Gr)
        h.hessvec(X, Z, H1, sigma=0.3, riemannian=False)
        h.hessvec(X, Z, H2, sigma=0.3, riemannian=True)
        h.sync()
    Zm = O.to_matrix(P, Zf)
    E_ref = O.energy(P, Xm)
    g = O.gradient(P, Xm)
    assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
    assert rel(Ge.cpu().numpy(), O.to_fields(P, g)) <= 1e-12
    rg = O.rgrad(P, u, O.to_u(P, g))
    assert rel(Gr.cpu().numpy(), O.to_fields(P, O.from_u(P, rg))) <= 1e-11
    assert abs(rn - np.linalg.norm(rg)) <= 1e-11 * np.linalg.norm(rg)
    H_ref = O.hessvec(P, Xm, Zm) + 0.3 * Zm
    assert rel(H1.cpu().numpy(), O.to_fields(P, H_ref)) <= 1e-12
    Hr = O.rhess(P, u, O.to_u(P, Zm), g=O.to_u(P, g), sigma=0.3)
    assert rel(H2.cpu().numpy(), O.to_fields(P, O.from_u(P, Hr))) <= 1e-11


def test_spin3_3d_128_fp64(dev):
    from paper_1907_01194_gb300 import sbec
    w = W.spin3_3d_cascadic()                 # finest level: 128^3
    P = _problem(w)
    u, Xm = _on_manifold(P, W.initial_fields(w))
    Xf = O.to_fields(P, Xm)
    Zf = W.smooth_random_fields(w, 5)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Ge, Gr, H = (torch.empty_like(X) for _ in range(3))
    with sbec.Handle.from_workload(w) as h:
        h.autotune(X)
        E, rn = h.grad(X, G_euc=Ge, G_riem=Gr)
        h.hessvec(X, Z, H, sigma=0.0, riemannian=False)
        h.sync()
    Zm = O.to_matrix(P, Zf)
    E_ref = O.energy(P, Xm)
    assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
    g = O.gradient(P, Xm)
    assert rel(Ge.cpu().numpy(), O.to_fields(P, g)) <= 1e-12
    rg = O.rgrad(P, u, O.to_u(P, g))
    assert rel(Gr.cpu().numpy(), O.to_fields(P, O.from_u(P, rg))) <= 1e-11
    idx = _sample(P.G)
    H_ref = O.hessvec_at(P, Xm, Zm, idx)
    assert rel(O.to_matrix(P, H.cpu().numpy())[idx], H_ref) <= 1e-12


def test_spin3_3d_256_mixed_sampled(dev):
    from paper_1907_01194_gb300 import sbec
    w = W.spin3_3d_256()
    P = _problem(w)
    Xf = W.initial_fields(w).astype(np.complex64)
    Zf = W.smooth_random_fields(w, 5).astype(np.complex64)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Ge, H = torch.empty_like(X), torch.empty_like(X)
    with sbec.Handle.from_workload(w, precision="mixed") as h:
        h.autotune(X)
        E, _ = h.grad(X, G_euc=Ge)
        h.hessvec(X, Z, H, sigma=0.0, riemannian=False)
        h.sync()
    Ge_s = O.to_matrix(P, Ge.cpu().numpy())
    H_s = O.to_matrix(P, H.cpu().numpy())
    del Ge, H
    Xm = O.to_matrix(P, Xf.astype(np.complex128))
    Zm = O.to_matrix(P, Zf.astype(np.complex128))
    idx = _sample(P.G)
    assert rel(Ge_s[idx], O.gradient_at(P, Xm, idx)) <= 2e-5
    assert rel(H_s[idx], O.hessvec_at(P, Xm, Zm, idx)) <= 2e-5
    E_ref = O.energy(P, Xm)
    assert abs(E - E_ref) <= 2e-6 * abs(E_ref)


def test_batched_sweep_sampled_instances(dev):
    from paper_1907_01194_gb300 import sbec
    insts = W.batched_spin1_2d()
    for n in (64, 128, 256):
        ws = [w for w in insts if w.n[0] == n]
        picks = (0, len(ws) // 2, len(ws) - 1)
        Xs = [W.initial_fields(w) for w in ws]
        ref = {}
        for i in picks:                      # sampled instances on M by the oracle's R1
            P = _problem(ws[i])
            u, Xm = _on_manifold(P, Xs[i])
            Xs[i] = O.to_fields(P, Xm)
            ref[i] = (O.energy(P, Xm), np.linalg.norm(O.rgrad(P, u)))
        X = torch.from_numpy(np.stack(Xs)).to(dev)
        with sbec.Handle.batch(ws) as h:
            h.autotune(X)
            E, rn = h.grad(X)
        for i in picks:
            E_ref, rn_ref = ref[i]
            assert abs(E[i] - E_ref) <= 1e-12 * abs(E_ref)
            assert abs(rn[i] - rn_ref) <= 1e-11 * rn_ref
