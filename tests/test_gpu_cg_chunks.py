"""Device-driven modified CG (Sec. 5, Eq. prob-lsub): the CG coefficients and
stopping tests run on the device in chunks of cg_chunk iterations, each chunk
the replay of a CUDA graph.  An instance whose CG has ended inside a chunk
leaves the rest of it untouched, so the chunk length and the use of graphs
change nothing in the arithmetic: states, energies and iteration counts are
bit-identical across settings, and the per-launch count seen by the library is
the same with and without graphs."""
import math

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


CASES = [
    W.spin1_1d(),
    W.Workload("s2_2d_32", F=2, n=(32, 32), lo=(-6.0, -6.0), hi=(6.0, 6.0),
               beta=(60.0, 2.0, -3.0, 0.0), M=0.4, lattice_amp=3.0, lattice_k=math.pi / 2),
    W.Workload("s3_3d_16", F=3, n=(16, 16, 16), lo=(-5.0,) * 3, hi=(5.0,) * 3,
               beta=(40.0, -1.0, 2.0, -0.5), M=0.2),
]
SETTINGS = [(1, False), (4, True), (3, True), (4, False), (64, True)]
KEYS = ("energy", "grad_norm", "outer_iters", "inner_iters", "rgbb_iters", "n_grad", "n_energy", "n_hvp")


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_chunk_length_and_graphs_do_not_change_the_solve(w, dev):
    from paper_1907_01194_gb300 import sbec
    X0 = W.initial_fields(w)
    runs = []
    with sbec.Handle.from_workload(w) as h:
        for chunk, graphs in SETTINGS:
            X = torch.from_numpy(X0).to(dev)
            st = h.solve(X, tol=1e-9, cg_chunk=chunk, graphs=graphs)
            runs.append((st, X))
    st0, X0d = runs[0]
    assert st0["converged"] and st0["inner_iters"] > 0
    for st, X in runs[1:]:
        assert torch.equal(X, X0d)
        for k in KEYS:
            assert st[k] == st0[k], k


def test_launch_count_is_the_same_with_graphs(dev):
    from paper_1907_01194_gb300 import sbec
    w = CASES[1]
    X0 = W.initial_fields(w)
    counts = []
    with sbec.Handle.from_workload(w) as h:
        for graphs in (False, True, True):
            X = torch.from_numpy(X0).to(dev)
            c0 = h.launch_count()
            h.solve(X, tol=1e-9, cg_chunk=4, graphs=graphs)
            counts.append(h.launch_count() - c0)
    assert counts[0] > 0 and counts[0] == counts[1] == counts[2]


def test_handle_calls_after_a_solve_see_every_instance(dev):
    # the CG's per-instance switch (S_SKIP) is off again when sbec_solve returns:
    # the energy of the result by sbec_energy equals the oracle's
    from paper_1907_01194_gb300 import sbec
    w = CASES[1]
    X0 = W.initial_fields(w)
    X = torch.from_numpy(X0).to(dev)
    P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)
    with sbec.Handle.from_workload(w) as h:
        st = h.solve(X, tol=1e-9)
        E = h.energy(X)
    Eo = O.energy(P, O.to_matrix(P, X.cpu().numpy()))
    assert abs(E - Eo) <= 1e-12 * abs(Eo)
    assert abs(st["energy"] - Eo) <= 1e-12 * abs(Eo)


def test_batch_chunks_and_graphs_do_not_change_the_solve(dev):
    from paper_1907_01194_gb300 import sbec
    rng = np.random.default_rng(3)
    ws = [W.Workload(f"b{i}", F=1, n=(32, 32), lo=(-7.0, -7.0), hi=(7.0, 7.0),
                     beta=(float(rng.uniform(30, 90)), float(rng.uniform(-2, 2)), 0.0, 0.0),
                     M=float(rng.uniform(0.05, 0.8)), seed=200 + i) for i in range(5)]
    X0 = np.stack([W.initial_fields(w) for w in ws])
    out = []
    with sbec.Handle.batch(ws) as h:
        for chunk, graphs in ((1, False), (4, True), (5, True)):
            X = torch.from_numpy(X0).to(dev)
            sts = sbec.solve_batch(h, X, tol=1e-9, cg_chunk=chunk, graphs=graphs)
            out.append((sts, X))
    sts0, Xr = out[0]
    assert all(s["converged"] for s in sts0)
    for sts, X in out[1:]:
        assert torch.equal(X, Xr)
        for a, b in zip(sts, sts0):
            for k in KEYS:
                assert a[k] == b[k], k
