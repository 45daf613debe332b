"""Cascadic multigrid on the GPU: the spectral prolongation (sbec_prolongate)
against the oracle's, and the cascadic solve (sbec_solve_cascadic) against the
oracle's cascadic driver (Algorithm 1), including a reduced spin-3 3D case with
the parameters of the 32^3 -> 64^3 -> 128^3 workload."""
import math

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


def _P(w):
    return O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)


@pytest.mark.parametrize("F,nc,nf", [(1, (16,), (32,)), (2, (8, 16), (16, 32)), (3, (8, 8, 8), (16, 16, 16)),
                                     (1, (16, 16), (16, 64))])
def test_prolongation_matches_oracle(F, nc, nf, dev):
    from paper_1907_01194_gb300 import sbec
    d = len(nc)
    base = W.Workload("pro", F=F, n=nc, lo=(-6.0,) * d, hi=(6.0,) * d, beta=(20.0, 1.0, 1.0, 1.0), M=0.3)
    wc, wf = base, base.at(nf)
    Pc, Pf = _P(wc), _P(wf)
    uc = O.psi_R1(Pc, O.to_u(Pc, O.to_matrix(Pc, W.initial_fields(wc))))
    Xc = O.to_fields(Pc, O.from_u(Pc, uc))
    ref = O.to_fields(Pf, O.prolongate(Pc, Pf, O.from_u(Pc, uc)))
    Xcd = torch.from_numpy(Xc).to(dev)
    Xfd = torch.empty(ref.shape, dtype=torch.complex128, device=dev)
    with sbec.Handle.from_workload(wc) as hc, sbec.Handle.from_workload(wf) as hf:
        sbec.prolongate(hc, Xcd, hf, Xfd)
        hf.sync()
    assert rel(Xfd.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("w,levels", [
    (W.Workload("casc1d", F=1, n=(64,), lo=(-8.0,), hi=(8.0,), beta=(40.0, -1.0, 0, 0), M=0.25), ((16,), (32,))),
    (W.Workload("casc3d", F=3, n=(16, 16, 16), lo=(-8.0,) * 3, hi=(8.0,) * 3, beta=(500.0, -2.0, 5.0, -1.0),
                M=0.2), ((8, 8, 8),)),
], ids=["spin1_1d", "spin3_3d_reduced"])
def test_cascadic_solve_matches_oracle(w, levels, dev):
    from paper_1907_01194_gb300 import sbec
    ws = [w.at(n) for n in levels] + [w]
    P = [_P(x) for x in ws]
    X0 = W.initial_fields(ws[0])
    Xs, ost, _ = O.solve(P, O.to_matrix(P[0], X0), O.SolveOptions(tol=1e-9))
    hs = [sbec.Handle.from_workload(x) for x in ws]
    states = [torch.from_numpy(X0).to(dev)] + [torch.empty((x.C,) + x.shape, dtype=torch.complex128, device=dev)
                                                 for x in ws[1:]]
    try:
        st = sbec.solve_cascadic(hs, states, tol=1e-9)
    finally:
        for h in hs:
            h.close()
    assert st["converged"] and ost.converged
    assert abs(st["energy"] - ost.energy) <= 1e-10 * abs(ost.energy)


def test_cascadic_mixed_solve_matches_oracle(dev):
    # sbec_solve_cascadic_mixed: every level a mixed solve with FP64 refinement (FP32
    # Newton CG); the finest energy meets the oracle's FP64 cascadic solve to 1e-10
    from paper_1907_01194_gb300 import sbec
    w = W.Workload("casc3d", F=3, n=(16, 16, 16), lo=(-8.0,) * 3, hi=(8.0,) * 3, beta=(500.0, -2.0, 5.0, -1.0),
                   M=0.2)
    ws = [w.at((8, 8, 8)), w]
    P = [_P(x) for x in ws]
    X0 = W.initial_fields(ws[0])
    Xs, ost, _ = O.solve(P, O.to_matrix(P[0], X0), O.SolveOptions(tol=1e-9))
    h64 = [sbec.Handle.from_workload(x) for x in ws]
    h32 = [sbec.Handle.from_workload(x, precision="mixed") for x in ws]
    states = [torch.from_numpy(X0).to(dev)] + [torch.empty((x.C,) + x.shape, dtype=torch.complex128, device=dev)
                                                 for x in ws[1:]]
    try:
        sm, sf = sbec.solve_cascadic_mixed(h64, h32, states, tol=1e-9)
        E, gn = h64[-1].grad(states[-1])
    finally:
        for h in h64 + h32:
            h.close()
    assert sf["converged"] and ost.converged and gn <= 1e-9
    assert abs(sf["energy"] - ost.energy) <= 1e-10 * abs(ost.energy)
    assert abs(E - ost.energy) <= 1e-10 * abs(ost.energy)
