"""The autograd wrappers (adjoint kernels behind torch.autograd.Function) against
central finite differences in FP64 and against the oracle's gradient and
Hessian-vector product; includes the finite-difference check on the 32^3 level
of the spin-3 cascadic workload (h = 1e-6)."""
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


def test_energy_backward_is_oracle_gradient(dev):
    from paper_1907_01194_gb300 import autograd as A, sbec
    w = W.Workload("ag_s2", F=2, n=(32, 16), lo=(-6.0, -5.0), hi=(6.0, 5.0), beta=(60.0, 2.0, -3.0, 0.0),
                   M=0.4, lattice_amp=3.0, lattice_k=math.pi / 2)
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev).requires_grad_(True)
    with sbec.Handle.from_workload(w) as h:
        E = A.energy(X, h)
        E.backward()
    assert abs(E.item() - O.energy(P, O.from_u(P, u))) <= 1e-12 * abs(E.item())
    G_ref = O.to_fields(P, O.gradient(P, O.from_u(P, u)))
    assert rel(X.grad.cpu().numpy(), G_ref) <= 1e-12


def test_gradient_backward_is_oracle_hessvec(dev):
    from paper_1907_01194_gb300 import autograd as A, sbec
    w = W.Workload("ag_s3", F=3, n=(64,), lo=(-8.0,), hi=(8.0,), beta=(80.0, -1.0, 4.0, 1.0), M=0.6)
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev).requires_grad_(True)
    V = torch.from_numpy(Zf).to(dev)
    with sbec.Handle.from_workload(w) as h:
        G = A.gradient(X, h)
        # L = Re<G, V> = sum Re(G) Re(V) + Im(G) Im(V): its gradient is H[V]
        L = (G.real * V.real + G.imag * V.imag).sum()
        L.backward()
    H_ref = O.to_fields(P, O.hessvec(P, O.from_u(P, u), O.to_matrix(P, Zf)))
    assert rel(X.grad.cpu().numpy(), H_ref) <= 1e-12


def test_torch_gradcheck_small(dev):
    from paper_1907_01194_gb300 import autograd as A, sbec
    w = W.Workload("ag_gc", F=1, n=(16,), lo=(-4.0,), hi=(4.0,), beta=(20.0, -1.0, 0, 0), M=0.2)
    X = torch.from_numpy(W.initial_fields(w)).to(dev).requires_grad_(True)
    with sbec.Handle.from_workload(w) as h:
        assert torch.autograd.gradcheck(lambda x: A.energy(x, h), (X,), eps=1e-6, atol=1e-7, rtol=1e-6)
        assert torch.autograd.gradcheck(lambda x: A.gradient(x, h), (X,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_central_fd_on_spin3_32cubed_level(dev):
    # the 32^3 level of the spin-3 cascadic workload: E(X + h D) - E(X - h D) / 2h against
    # Re<grad, D>, and grad(X + h D) - grad(X - h D) / 2h against H[D], h = 1e-6, FP64
    from paper_1907_01194_gb300 import autograd as A, sbec
    w = W.spin3_3d_cascadic().at((32, 32, 32))
    X = torch.from_numpy(W.initial_fields(w)).to(dev)
    D = torch.from_numpy(W.smooth_random_fields(w, 3)).to(dev)
    hstep = 1e-6
    with sbec.Handle.from_workload(w) as h:
        Xr = X.clone().requires_grad_(True)
        E = A.energy(Xr, h)
        E.backward()
        g = Xr.grad
        fd = (h.energy(X + hstep * D) - h.energy(X - hstep * D)) / (2 * hstep)
        an = float((g.real * D.real + g.imag * D.imag).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        Gp, Gm, HD = torch.empty_like(X), torch.empty_like(X), torch.empty_like(X)
        h.grad(X + hstep * D, G_euc=Gp)
        h.grad(X - hstep * D, G_euc=Gm)
        h.hessvec(X, D, HD)
        fdg = (Gp - Gm) / (2 * hstep)
        assert float(torch.linalg.norm(fdg - HD) / torch.linalg.norm(HD)) <= 1e-6
