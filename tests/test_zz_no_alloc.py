"""The allocation-free energy entry point (sbec_energy_noalloc) against the
handle-based sbec_energy and against the CPU oracle.

sbec_energy_noalloc exists for callers that must not allocate device memory
where they need the energy (a framework owning all device memory through its
own pool, or a loop that cannot wait on cudaMalloc/cudaFree).  It keeps its
intermediates in one fixed device array inside the library, so this test calls
it several times in a row on different problems and checks that each result
matches the handle-based entry point and the oracle's E_h within the FP64
parity bar of the other GPU tests (1e-12 relative): a stale intermediate from
an earlier call would show up in a later one.  The cases cover 1D (the
single-pass energy kernel), 2D with a tabulated potential, 3D with the
harmonic trap, and the documented capacity edge (spin-3 on 256 x 256 with the
harmonic trap built inside the array).  The file is named to be collected
last."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sbec_oracle as O  # noqa: E402
from paper_1907_01194_gb300 import workloads as W  # noqa: E402


def _state(w, dev):
    return torch.from_numpy(W.initial_fields(w)).to(dev)


def _oracle_energy(w, Xf):
    P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), p=w.p, q=w.q, M=w.M)
    return O.energy(P, O.to_matrix(P, Xf))


def test_noalloc_energy_matches_handle_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_01194_gb300 import sbec
    dev = torch.device("cuda:0")
    line = W.Workload("na_line", F=1, n=(256,), lo=(-16.0,), hi=(16.0,), beta=(100.0, -0.5, 0.0, 0.0), M=0.5)
    lattice = W.Workload("na_lattice", F=2, n=(64, 32), lo=(-8.0, -6.0), hi=(8.0, 6.0),
                         beta=(200.0, 10.0, -5.0, 0.0), M=0.3, lattice_amp=20.0,
                         lattice_k=math.pi / 2)
    harmonic = W.Workload("na_harmonic", F=3, n=(16, 8, 32), lo=(-6.0,) * 3, hi=(6.0,) * 3,
                          beta=(500.0, -2.0, 5.0, -1.0), M=0.2)
    # the capacity edge: 2 C G + G + tables ~ 1.02M of the 1.048M doubles
    edge = W.Workload("na_edge", F=3, n=(256, 256), lo=(-10.0, -10.0), hi=(10.0, 10.0),
                      beta=(1000.0, -5.0, 10.0, 2.0), M=0.0)
    cases = [(line, None), (lattice, torch.from_numpy(W.potential(lattice)).to(dev)), (harmonic, None),
             (edge, None), (line, None)]
    for w, V in cases:
        Xf = W.initial_fields(w)
        X = torch.from_numpy(Xf).to(dev)
        E_na = sbec.energy_noalloc(w.F, w.n, w.lo, w.hi, w.beta, w.M, X, V=V)
        with sbec.Handle.from_workload(w, V=(W.potential(w) if V is not None else None)) as h:
            E_ref = h.energy(X)
        assert abs(E_na - E_ref) <= 1e-12 * abs(E_ref), (w.name, E_na, E_ref)
        E_or = _oracle_energy(w, Xf)
        assert abs(E_na - E_or) <= 1e-12 * abs(E_or), (w.name, E_na, E_or)
    # oversized problems are rejected, not truncated
    big = W.Workload("na_big", F=3, n=(512, 256), lo=(-8.0, -8.0), hi=(8.0, 8.0),
                     beta=(1.0, 0.0, 0.0, 0.0), M=0.0)
    Xb = torch.zeros((7, 256, 512), dtype=torch.complex128, device=dev)
    with pytest.raises(sbec.SbecError) as e:
        sbec.energy_noalloc(big.F, big.n, big.lo, big.hi, big.beta, big.M, Xb)
    assert e.value.status == sbec.ERR_ARG
    # host arrays never reach the kernels: the binding refuses them, and so does the
    # C entry point when handed a host pointer directly
    Xh = torch.from_numpy(W.initial_fields(line))
    with pytest.raises(ValueError):
        sbec.energy_noalloc(line.F, line.n, line.lo, line.hi, line.beta, line.M, Xh)
    assert sbec.energy_noalloc_raw(line.F, line.n, line.lo, line.hi, line.beta, line.M, Xh.data_ptr()) \
        == sbec.ERR_ARG
