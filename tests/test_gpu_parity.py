"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on the same seeded inputs: energy (Eq. 3.7), Euclidean gradient
(Eq. 3.12), Riemannian gradient (Lemma 4.1), Hessian-vector products
(Eq. 3.13, Lemma 4.2) and the three retractions (Lemmas 5.1, 5.3, 5.4).

Bars: FP64 form 1e-12 relative (normwise for fields); mixed form (FP32 FFT and
pointwise arithmetic, FP64 reductions) 2e-6 relative for energies and 2e-5
normwise for fields (derived from the float unit roundoff 6e-8 times the
log2(G) FFT depth and the conditioning of the nonlinear terms)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sbec_oracle as O  # noqa: E402
from paper_1907_01194_gb300 import workloads as W  # noqa: E402
from tests.gpu_helpers import case_inputs, rel  # noqa: E402


def _sbec():
    from paper_1907_01194_gb300 import sbec
    return sbec


def _wl(F, n, L, M, beta, lattice=0.0, p=0.0, q=0.0):
    d = len(n)
    return W.Workload(f"par_F{F}_{'x'.join(map(str, n))}", F=F, n=tuple(n), lo=(-L,) * d, hi=(L,) * d,
                      beta=beta, M=M, p=p, q=q, lattice_amp=lattice, lattice_k=math.pi / 2)


CASES = [
    _wl(1, (256,), 16.0, 0.5, (100.0, -0.5, 0, 0)),                      # 1D, spin-1
    _wl(3, (8,), 4.0, 0.7, (30.0, 1.0, 2.0, -1.0), p=0.2, q=0.1),       # tiny 1D
    _wl(2, (64, 32), 8.0, 0.3, (200.0, 10.0, -5.0, 0), lattice=20.0),     # 2D non-square
    _wl(3, (16, 64), 6.0, 1.1, (60.0, -2.0, 5.0, -1.0), lattice=3.0),     # 2D spin-3
    _wl(1, (2, 256), 5.0, 0.2, (50.0, 1.0, 0, 0)),                        # degenerate x axis
    _wl(3, (16, 8, 32), 6.0, 0.2, (500.0, -2.0, 5.0, -1.0)),              # 3D non-cubic
    _wl(2, (32, 32, 32), 8.0, 0.0, (100.0, 3.0, 4.0, 0), lattice=10.0),   # 3D, M = 0
    _wl(1, (1024,), 20.0, 0.4, (300.0, 2.0, 0, 0)),                       # longest axis
    _wl(2, (512, 4), 12.0, 0.3, (80.0, 2.0, -1.0, 0)),                     # long x rows in 2D
    _wl(1, (4, 8, 512), 6.0, 0.1, (40.0, 1.0, 0, 0)),                      # long strided axis
    _wl(4, (128,), 8.0, 1.3, (60.0, -1.5, 4.0, 0), p=0.1, q=0.05),        # spin-4, 1D
    _wl(4, (32, 16), 6.0, 2.1, (80.0, 1.0, -3.0, 0), lattice=5.0),        # spin-4, 2D
    _wl(4, (16, 8, 16), 6.0, 0.5, (120.0, -2.0, 6.0, 0)),                 # spin-4, 3D
]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_fp64_energy_grad_hess_parity(w, dev):
    sbec = _sbec()
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Ge, Gr, H1, H2 = (torch.empty_like(X) for _ in range(4))
    with sbec.Handle.from_workload(w) as h:
        E1 = h.energy(X)
        E2, rn = h.grad(X, G_euc=Ge, G_riem=Gr)
        h.hessvec(X, Z, H1, sigma=0.3, riemannian=False)
        h.hessvec(X, Z, H2, sigma=0.3, riemannian=True)
        h.sync()
    Xm = O.from_u(P, u)
    E_ref = O.energy(P, Xm)
    assert abs(E1 - E_ref) <= 1e-12 * abs(E_ref)
    assert abs(E2 - E_ref) <= 1e-12 * abs(E_ref)
    g = O.gradient(P, Xm)
    assert rel(Ge.cpu().numpy(), O.to_fields(P, g)) <= 1e-12
    rg = O.rgrad(P, u, O.to_u(P, g))
    assert rel(Gr.cpu().numpy(), O.to_fields(P, O.from_u(P, rg))) <= 1e-11 * max(1.0, np.linalg.norm(O.to_u(P, g)) / np.linalg.norm(rg))
    assert abs(rn - np.linalg.norm(rg)) <= 1e-11 * np.linalg.norm(O.to_u(P, g))
    Zm = O.to_matrix(P, Zf)
    H_ref = O.hessvec(P, Xm, Zm) + 0.3 * Zm
    assert rel(H1.cpu().numpy(), O.to_fields(P, H_ref)) <= 1e-12
    Hr_ref = O.rhess(P, u, O.to_u(P, Zm), g=O.to_u(P, g), sigma=0.3)
    assert rel(H2.cpu().numpy(), O.to_fields(P, O.from_u(P, Hr_ref))) <= 1e-11


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("w", [CASES[0], CASES[2], CASES[5], CASES[6], CASES[11]], ids=lambda w: w.name)
def test_fp64_retraction_parity(w, kind, dev):
    sbec = _sbec()
    P, u, Xf, Zf = case_inputs(w)
    xi = O.project(P, u, O.to_u(P, O.to_matrix(P, Zf)))
    xi /= np.linalg.norm(xi)
    Xi = O.to_fields(P, O.from_u(P, xi))
    U = torch.from_numpy(Xf).to(dev)
    XiD = torch.from_numpy(Xi).to(dev)
    out = torch.empty_like(U)
    with sbec.Handle.from_workload(w) as h:
        for t in (0.3, 1e-3):
            h.retract(U, XiD, t, kind, out)
            h.sync()
            ref = O.retract(P, u, t * xi, kind)
            assert rel(out.cpu().numpy(), O.to_fields(P, O.from_u(P, ref))) <= 1e-12
            got = O.to_u(P, O.to_matrix(P, out.cpu().numpy()))
            Gm = O.gamma_weights(P)
            assert abs(got @ got - 1) < 1e-12 and abs(got @ (Gm * got) - w.M) < 1e-12


# FP32 strided passes on TMA tiles: pass axes of 128 / 256 points, x a multiple of 16
TMA_CASES = [
    _wl(2, (32, 128, 128), 8.0, 0.3, (150.0, 4.0, -3.0, 0), lattice=6.0),     # 3D: y and z passes
    _wl(3, (16, 256), 8.0, 0.9, (90.0, -1.0, 4.0, 1.5), lattice=4.0),        # 2D: fused y pass
    _wl(1, (64, 32, 256), 8.0, 0.2, (60.0, 1.0, 0, 0)),                      # z on TMA, y (32) not
]


@pytest.mark.parametrize("w", [CASES[0], CASES[2], CASES[5], CASES[12]] + TMA_CASES, ids=lambda w: w.name)
def test_mixed_precision_bound(w, dev):
    sbec = _sbec()
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf.astype(np.complex64)).to(dev)
    Z = torch.from_numpy(Zf.astype(np.complex64)).to(dev)
    Ge, H1 = torch.empty_like(X), torch.empty_like(X)
    with sbec.Handle.from_workload(w, precision="mixed") as h:
        E = h.energy(X)
        E2, rn = h.grad(X, G_euc=Ge)
        h.hessvec(X, Z, H1, sigma=0.0, riemannian=False)
        h.sync()
    # the oracle sees the same float-rounded inputs
    Xm = O.to_matrix(P, Xf.astype(np.complex64).astype(np.complex128))
    Zm = O.to_matrix(P, Zf.astype(np.complex64).astype(np.complex128))
    E_ref = O.energy(P, Xm)
    assert abs(E - E_ref) <= 2e-6 * abs(E_ref)
    assert abs(E2 - E_ref) <= 2e-6 * abs(E_ref)
    assert rel(Ge.cpu().numpy(), O.to_fields(P, O.gradient(P, Xm))) <= 2e-5
    assert rel(H1.cpu().numpy(), O.to_fields(P, O.hessvec(P, Xm, Zm))) <= 2e-5


def _tma_tiles(w, width):
    # launch shapes with the TMA pass of the given tile width on every axis it runs on
    # (128 or 256 points), None when x is not a multiple of the width
    if w.n[0] % width:
        return None
    pen, spl = [0, 0, 0], [0, 0, 0]
    for ax in range(1, w.dim):
        if w.n[ax] in (128, 256):
            pen[ax], spl[ax] = width, 16
    return dict(s_pencils=pen, s_split=spl)


@pytest.mark.parametrize("width", [8, 16, 32])
@pytest.mark.parametrize("w", TMA_CASES, ids=lambda w: w.name)
def test_mixed_riemannian_and_repeatable_on_tma_passes(w, width, dev):
    # the Riemannian products through the TMA passes of each tile width (8, 16, 32
    # columns: 4, 2, 1 blocks per SM), and bitwise repeatability of the persistent
    # tile loop (fixed tile order per block, fixed reduction order)
    sbec = _sbec()
    tiles = _tma_tiles(w, width)
    if tiles is None:
        pytest.skip(f"n_x = {w.n[0]} is not a multiple of the tile width {width}")
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf.astype(np.complex64)).to(dev)
    Z = torch.from_numpy(Zf.astype(np.complex64)).to(dev)
    Gr, H1, H2 = (torch.empty_like(X) for _ in range(3))
    with sbec.Handle.from_workload(w, precision="mixed") as h:
        h.set_tune(tiles)
        got = h.get_tune()
        for ax in range(1, w.dim):
            if tiles["s_split"][ax]:
                assert (got["s_pencils"][ax], got["s_split"][ax]) == (width, 16), got
        E1 = h.energy(X)
        E2, rn = h.grad(X, G_riem=Gr)
        h.hessvec(X, Z, H1, sigma=0.2, riemannian=True)
        h.hessvec(X, Z, H2, sigma=0.2, riemannian=True)
        assert h.energy(X) == E1
        h.sync()
    assert torch.equal(H1, H2)
    Xm = O.to_matrix(P, Xf.astype(np.complex64).astype(np.complex128))
    Zm = O.to_matrix(P, Zf.astype(np.complex64).astype(np.complex128))
    uu = O.to_u(P, Xm)
    g = O.to_u(P, O.gradient(P, Xm))
    rg = O.rgrad(P, uu, g)
    assert abs(rn - np.linalg.norm(rg)) <= 2e-5 * np.linalg.norm(g)
    Hr = O.rhess(P, uu, O.to_u(P, Zm), g=g, sigma=0.2)
    assert rel(H1.cpu().numpy(), O.to_fields(P, O.from_u(P, Hr))) <= 2e-5


def test_host_pointers_match_device(dev):
    sbec = _sbec()
    w = CASES[2]
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    Gd = torch.empty_like(X)
    Gh = np.empty_like(Xf)
    with sbec.Handle.from_workload(w) as h:
        Ed, rd = h.grad(X, G_riem=Gd)
        Eh, rh = h.grad(np.ascontiguousarray(Xf), G_riem=Gh)
    assert Ed == Eh and rd == rh
    assert np.array_equal(Gd.cpu().numpy(), Gh)


def test_pinned_host_arrays_match_device(dev):
    # page-locked host arrays are read in place by the kernels; results equal the
    # device-array results bit for bit
    sbec = _sbec()
    w = CASES[5]
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Xp = torch.from_numpy(Xf).pin_memory()
    Zp = torch.from_numpy(Zf).pin_memory()
    Gd, Hd, Rd = (torch.empty_like(X) for _ in range(3))
    Gp, Hp, Rp = (torch.empty_like(Xp).pin_memory() for _ in range(3))
    with sbec.Handle.from_workload(w) as h:
        a = h.grad(X, G_riem=Gd)
        h.hessvec(X, Z, Hd, sigma=0.4, riemannian=True)
        h.retract(X, Gd, -1e-3, 1, Rd)
        Ed = h.energy(Rd)
        h.sync()
        b = h.grad(Xp, G_riem=Gp)
        h.hessvec(Xp, Zp, Hp, sigma=0.4, riemannian=True)
        h.retract(Xp, Gp, -1e-3, 1, Rp)
        Ep = h.energy(Rp)
    assert a == b and Ed == Ep
    for dv, hv in ((Gd, Gp), (Hd, Hp), (Rd, Rp)):
        assert torch.equal(dv.cpu(), hv)


def test_host_riemannian_hessvec_uses_the_gradient_at_the_same_pointer(dev):
    # the Lemma 4.2 coefficients come from the latest sbec_grad at the same X pointer,
    # host or device; a new pointer recomputes them
    sbec = _sbec()
    w = CASES[2]
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Hd = torch.empty_like(X)
    Xh = np.array(Xf, copy=True)
    Zh = np.array(Zf, copy=True)
    Hh1, Hh2 = np.empty_like(Xf), np.empty_like(Xf)
    with sbec.Handle.from_workload(w) as h:
        h.grad(X)
        h.hessvec(X, Z, Hd, sigma=0.2, riemannian=True)
        h.sync()
        h.grad(Xh)                                           # cached for the host pointer Xh
        h.hessvec(Xh, Zh, Hh1, sigma=0.2, riemannian=True)  # Xh's staged copy reused
        Xh2 = np.array(Xf, copy=True)                        # another pointer: recomputed
        h.hessvec(Xh2, Zh, Hh2, sigma=0.2, riemannian=True)
        h.grad(Xh)
        h.energy(np.array(Zf, copy=True))                    # another host array through the staging
        Hh3 = np.empty_like(Xf)
        h.hessvec(Xh, Zh, Hh3, sigma=0.2, riemannian=True)  # Xh staged again
    assert np.array_equal(Hd.cpu().numpy(), Hh1)
    assert np.array_equal(Hd.cpu().numpy(), Hh2)
    assert np.array_equal(Hd.cpu().numpy(), Hh3)


@pytest.mark.parametrize("w", [CASES[2], CASES[3], CASES[4], CASES[5], CASES[11]], ids=lambda w: w.name)
def test_hessian_reads_the_densities_of_the_gradient_at_the_same_state(w, dev):
    # FP64 handles in 2D / 3D: a Hessian-vector product at the X of the latest
    # gradient reads the densities that gradient stored; at any other X it forms them.
    # Both against the oracle, and the stored densities of another state are not used
    sbec = _sbec()
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    X2 = torch.from_numpy(W.initial_fields(w, seed=12345)).to(dev)
    Hf, Hc, Ho, Hr = (torch.empty_like(X) for _ in range(4))
    with sbec.Handle.from_workload(w) as h:
        h.hessvec(X, Z, Hf, sigma=0.1, riemannian=False)          # no gradient yet: formed
        h.grad(X2)                                                # densities of X2 stored
        h.hessvec(X, Z, Ho, sigma=0.1, riemannian=False)          # another state: formed
        h.grad(X)
        h.hessvec(X, Z, Hc, sigma=0.1, riemannian=False)          # read
        h.hessvec(X, Z, Hr, sigma=0.1, riemannian=True)           # read
        h.sync()
    Xm, Zm = O.from_u(P, u), O.to_matrix(P, Zf)
    H_ref = O.to_fields(P, O.hessvec(P, Xm, Zm) + 0.1 * Zm)
    for H in (Hf, Hc, Ho):
        assert rel(H.cpu().numpy(), H_ref) <= 1e-12
    assert torch.equal(Hf, Ho)
    assert rel(Hc.cpu().numpy(), Hf.cpu().numpy()) <= 1e-14
    g = O.to_u(P, O.gradient(P, Xm))
    Hr_ref = O.rhess(P, u, O.to_u(P, Zm), g=g, sigma=0.1)
    assert rel(Hr.cpu().numpy(), O.to_fields(P, O.from_u(P, Hr_ref))) <= 1e-11


def test_deterministic_repeat(dev):
    sbec = _sbec()
    w = CASES[5]
    P, u, Xf, Zf = case_inputs(w)
    X = torch.from_numpy(Xf).to(dev)
    with sbec.Handle.from_workload(w) as h:
        a = h.grad(X)
        b = h.grad(X)
    assert a == b


def test_error_codes(dev):
    sbec = _sbec()
    with pytest.raises(sbec.SbecError) as e:
        sbec.Handle(1, (64,), (-8,), (8,), (10.0, 1.0), M=1.0)        # |M| >= F
    assert e.value.status == sbec.ERR_ARG
    with pytest.raises(sbec.SbecError):
        sbec.Handle(1, (48,), (-8,), (8,), (10.0, 1.0), M=0.2)        # n not a power of two
    w = CASES[0]
    P, u, Xf, Zf = case_inputs(w)
    U = np.array(Xf, copy=True)
    U[1:] = 0                                                         # only l = 1 left: outside Omega
    Xi = np.zeros_like(U)
    out = np.empty_like(U)
    with sbec.Handle.from_workload(w) as h:
        for kind in (1, 2, 3):
            with pytest.raises(sbec.SbecError) as e:
                h.retract(U, Xi, 0.0, kind, out)
            assert e.value.status == sbec.ERR_DOMAIN
        bad = np.array(Xf, copy=True)
        bad[0, 3] = np.nan
        with pytest.raises(sbec.SbecError) as e:
            h.grad(bad)
        assert e.value.status == sbec.ERR_NONFINITE
        # the handle stays usable after an error
        E, rn = h.grad(np.array(Xf, copy=True))
        assert math.isfinite(E)
