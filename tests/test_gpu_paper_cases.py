"""The paper's own 2D and 3D cases (Sec. 7.2, 7.3) solved on the GPU from the
paper's initial data with the cascadic ARNT of Algorithm 1, against the
energies the paper prints (tests/golden/spin2_2d_3d_energies.txt,
tests/golden/spin3_2d_3d_energies.txt).

* Spin-2 2D, cases I-III at M = 0, 0.5, 1.5: the ten-digit values, to 1e-9,
  except the cyclic case III at M = 0, where the printed value is a stationary
  point above the minimum: there the GPU reaches the scalar-GPE energy with the
  same beta0, a lower bound of the energy for beta1, beta2 >= 0 that the cyclic
  spinor attains at M = 0 (checked by solving the beta1 = beta2 = 0 problem).
* Spin-2 3D, case III at M = 0: the same lower bound on the 256^3 mesh.
* Spin-3 2D, cases I and II, and spin-3 3D case I: the four-decimal values, to
  the printed precision (1e-4; the random initial spinor is drawn from a seeded
  generator, as the paper's is random).
* Spin-1 3D (ferromagnetic, 256^3) at M = 0 from a 128^3 level: the printed
  four-decimal value (tests/golden/spin1_3d_energies.txt) to half a unit of its
  last decimal."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01194_gb300 import workloads as W  # noqa: E402
from tests.conftest import golden  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _printed(name):
    return {(int(r[0]), int(r[1]), float(r[2])): float(r[3]) for r in golden(name)}


def _cascadic(make, n, dev, tol=1e-8, mixed=False, coarse=(4, 2), init=None):
    from paper_1907_01194_gb300 import sbec
    ws = [make(n // c) for c in coarse] + [make(n)]
    h64 = [sbec.Handle.from_workload(w) for w in ws]
    X0 = W.paper_initial(init(n // coarse[0]) if init else ws[0])
    states = [torch.from_numpy(X0).to(dev)] + [
        torch.empty((w.C,) + w.shape, dtype=torch.complex128, device=dev) for w in ws[1:]]
    try:
        if mixed:
            h32 = [sbec.Handle.from_workload(w, precision="mixed") for w in ws]
            try:
                _, st = sbec.solve_cascadic_mixed(h64, h32, states, tol=tol, maxit=300)
            finally:
                for h in h32:
                    h.close()
        else:
            st = sbec.solve_cascadic(h64, states, tol=tol, maxit=300)
    finally:
        for h in h64:
            h.close()
    return st


def _scalar_bound(make, n, dev, mixed=False, tol=1e-8):
    # the same problem with beta1 = beta2 = 0: its ground-state energy is the
    # scalar-GPE one (the reduction pinned by the oracle's tests).  Its minimisers
    # form a continuum (every spinor direction with the constraints), so ARNT's
    # last digits of ||grad|| come slowly; the energy, quadratic in the gradient,
    # is settled long before
    from dataclasses import replace

    def scalar(m):
        w = make(m)
        return replace(w, beta=(w.beta[0], 0.0, 0.0, 0.0))
    return _cascadic(scalar, n, dev, mixed=mixed, init=make, tol=tol)


@pytest.mark.parametrize("case", [1, 2, 3])
@pytest.mark.parametrize("M", [0.0, 0.5, 1.5])
def test_spin2_2d_ten_digit_energies(case, M, dev):
    printed = _printed("spin2_2d_3d_energies.txt")[(2, case, M)]
    make = lambda n: W.paper_spin2_2d_case(case, M, n)
    st = _cascadic(make, 256, dev)
    assert st["converged"]
    if case == 3 and M == 0.0:
        bound = _scalar_bound(make, 256, dev)
        assert bound["converged"]
        assert abs(st["energy"] - bound["energy"]) <= 1e-9 * bound["energy"]
        assert st["energy"] < printed - 0.4
    else:
        assert abs(st["energy"] - printed) <= 1e-9 * printed, (st["energy"], printed)


def test_spin2_3d_cyclic_reaches_the_scalar_bound(dev):
    printed = _printed("spin2_2d_3d_energies.txt")[(3, 3, 0.0)]
    make = lambda n: W.paper_spin2_3d_case(3, 0.0, n)
    st = _cascadic(make, 256, dev, mixed=True)
    bound = _scalar_bound(make, 256, dev, mixed=True, tol=1e-6)
    assert st["converged"] and bound["converged"]
    assert abs(st["energy"] - bound["energy"]) <= 1e-9 * bound["energy"]
    assert st["energy"] < printed - 0.5


@pytest.mark.parametrize("case", [1, 2])
@pytest.mark.parametrize("M", [0.0, 0.5, 1.5])
def test_spin3_2d_table_energies(case, M, dev):
    printed = _printed("spin3_2d_3d_energies.txt")[(2, case, M)]
    st = _cascadic(lambda n: W.paper_spin3_2d(case, M, n), 256, dev)
    assert st["converged"]
    assert abs(st["energy"] - printed) <= 5e-5 + 1e-9, (st["energy"], printed)


@pytest.mark.parametrize("M", [0.0, 0.5, 1.5])
def test_spin3_3d_case1_table_energies(M, dev):
    printed = _printed("spin3_2d_3d_energies.txt")[(3, 1, M)]
    st = _cascadic(lambda n: W.paper_spin3_3d(1, M, n), 128, dev)
    assert st["converged"]
    assert abs(st["energy"] - printed) <= 1e-4, (st["energy"], printed)


def test_spin1_3d_m0_table_energy(dev):
    # the 256^3 lattice (period 2 on [-16, 16]) has four points per period on a 64^3
    # level, too few to carry the lattice's ground state: the cascade starts at 128^3
    printed = {float(r[0]): float(r[1]) for r in golden("spin1_3d_energies.txt")}[0.0]
    st = _cascadic(lambda n: W.paper_spin1_3d(0.0, n), 256, dev, coarse=(2,))
    assert st["converged"]
    assert abs(st["energy"] - printed) <= 5e-5, (st["energy"], printed)
