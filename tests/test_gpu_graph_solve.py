"""The device-driven solve (sbec_solve_graph): Algorithm 1 for every instance of
one or several handles as one CUDA graph launch, its decisions taken by control
kernels on the device.  It takes the same decisions as the host-driven lock-step
batch solver, so each instance ends on the same iterate (same iteration counts,
energies equal to rounding); the instances of handles of different grid sizes
solve in one launch; the ground states match the CPU oracle's; and a loop cap
ends the launch with SBEC_ERR_TIMEOUT while the handles stay usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sbec_oracle as O  # noqa: E402
from paper_1907_01194_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _class(n, count=3, start=0):
    insts = [w for w in W.batched_spin1_2d(48) if w.n[0] == n]
    return insts[start:start + count]


def _X(ws, dev, dtype=torch.complex128):
    return torch.from_numpy(np.stack([W.initial_fields(w) for w in ws])).to(dev).to(dtype)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_solve_takes_the_batch_solvers_decisions(precision, dev):
    from paper_1907_01194_gb300 import sbec
    ws = _class(64, 4)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    tol = 1e-8 if precision == "fp64" else 1e-4
    X0 = _X(ws, dev, dt)
    with sbec.Handle.batch(ws, precision=precision) as h:
        Xa = X0.clone()
        sa = sbec.solve_batch(h, Xa, tol=tol)
        Xb = X0.clone()
        rc, sb = sbec.solve_graph([h], [Xb], tol=tol)
        E, gn = h.grad(Xb)
    assert rc == sbec.OK
    for a, b in zip(sa, sb[0]):
        assert a["converged"] and b["converged"]
        assert (a["outer_iters"], a["inner_iters"], a["rgbb_iters"]) == (b["outer_iters"], b["inner_iters"],
                                                                          b["rgbb_iters"])
        assert abs(a["energy"] - b["energy"]) <= 1e-13 * abs(a["energy"])
    assert torch.equal(Xa, Xb)


def test_graph_solve_of_uneven_sizes_in_one_launch_matches_oracle(dev):
    # three grid sizes as three parallel branches of one graph; each instance's
    # ground state against the oracle's solve of the same instance
    from paper_1907_01194_gb300 import sbec
    classes = [_class(64, 2), _class(128, 2), _class(256, 1)]
    hs = [sbec.Handle.batch(ws) for ws in classes]
    Xs = [_X(ws, dev) for ws in classes]
    try:
        rc, sts = sbec.solve_graph(hs, Xs, tol=1e-8)
    finally:
        for h in hs:
            h.close()
    assert rc == sbec.OK
    for ws, st, Xg in zip(classes, sts, Xs):
        for i, (w, s) in enumerate(zip(ws, st)):
            assert s["converged"] and s["grad_norm"] <= 1e-8
            if w.n[0] > 64:
                continue          # the oracle solves the 64^2 instances here (the others: sampled sweep test)
            P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)
            Xo, ost, _ = O.solve(P, O.to_matrix(P, W.initial_fields(w)), O.SolveOptions(tol=1e-8))
            assert abs(s["energy"] - ost.energy) <= 1e-10 * abs(ost.energy)
            m = np.sum(np.abs(Xg[i].cpu().numpy().reshape(w.C, -1)) ** 2, axis=1)
            assert abs(m.sum() - 1) < 1e-12 and abs(m @ np.arange(w.F, -w.F - 1, -1) - w.M) < 1e-12


def test_graph_solve_single_handle_matches_sbec_solve(dev):
    from paper_1907_01194_gb300 import sbec
    w = W.Workload("g2d", F=2, n=(32, 32), lo=(-6.0, -6.0), hi=(6.0, 6.0), beta=(60.0, 2.0, -3.0, 0.0), M=0.4,
                   lattice_amp=3.0, lattice_k=np.pi / 2)
    X0 = torch.from_numpy(W.initial_fields(w)).to(dev)
    with sbec.Handle.from_workload(w) as h:
        Xa = X0.clone()
        sa = h.solve(Xa, tol=1e-9)
        Xb = X0.clone()
        rc, sb = sbec.solve_graph([h], [Xb], tol=1e-9)
    assert rc == sbec.OK and sb[0][0]["converged"]
    assert abs(sa["energy"] - sb[0][0]["energy"]) <= 1e-12 * abs(sa["energy"])


def test_graph_solve_loop_cap_times_out_and_handle_stays_usable(dev):
    # a cap of three loop-body executions cannot finish the RGBB warm start: the
    # launch ends with SBEC_ERR_TIMEOUT (a bounded device-side loop, no hang), and
    # the handle and its stream keep working
    from paper_1907_01194_gb300 import sbec
    ws = _class(64, 2)
    X = _X(ws, dev)
    with sbec.Handle.batch(ws) as h:
        rc, st = sbec.solve_graph([h], [X.clone()], tol=1e-8, loop_cap=3)
        assert rc == sbec.ERR_TIMEOUT
        assert all(not s["converged"] for s in st[0])
        E = h.energy(X)
        assert np.all(np.isfinite(np.atleast_1d(E)))
        rc2, st2 = sbec.solve_graph([h], [X.clone()], tol=1e-8)
        assert rc2 == sbec.OK and all(s["converged"] for s in st2[0])
