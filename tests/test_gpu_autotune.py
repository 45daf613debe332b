"""Launch shapes chosen by the autotuner (sbec_autotune) or set explicitly
(sbec_set_tune): every accepted shape computes the same energy, gradient and
Hessian-vector product as the oracle (FP64 bar 1e-12 relative, as in the
parity tests), invalid shapes are rejected on the host, and the tuner leaves
the handle on the shapes it reports."""
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


def _wl(F, n, L, M, beta, lattice=0.0):
    d = len(n)
    return W.Workload(f"tune_F{F}_{'x'.join(map(str, n))}", F=F, n=tuple(n), lo=(-L,) * d, hi=(L,) * d,
                      beta=beta, M=M, lattice_amp=lattice, lattice_k=math.pi / 2)


W1 = _wl(1, (256,), 16.0, 0.5, (100.0, -0.5, 0, 0))
W2 = _wl(2, (64, 32), 8.0, 0.3, (200.0, 10.0, -5.0, 0), lattice=20.0)
W3 = _wl(3, (16, 8, 32), 6.0, 0.2, (500.0, -2.0, 5.0, -1.0))

# explicit shapes spanning the accepted range (small and large tiles, split
# butterflies, few and many elementwise blocks); tiles of more than 256 threads
# run the shared-memory Stockham kernels, smaller ones the two-level kernels
SHAPES = {
    W1.name: [dict(x_rows=1, elem_per_sm=1), dict(x_rows=1, elem_per_sm=32)],
    W2.name: [dict(x_rows=1, s_pencils=[0, 1, 0], s_split=[0, 4, 0], elem_per_sm=2),
              dict(x_rows=8, s_pencils=[0, 64, 0], s_split=[0, 1, 0], elem_per_sm=32),
              dict(x_rows=4, s_pencils=[0, 8, 0], s_split=[0, 8, 0])],
    W3.name: [dict(x_rows=1, s_pencils=[0, 1, 1], s_split=[0, 2, 4], elem_per_sm=3),
              dict(x_rows=16, s_pencils=[0, 16, 16], s_split=[0, 1, 8], elem_per_sm=32)],
}


def _check(h, P, u, Xf, Zf, dev):
    X = torch.from_numpy(Xf).to(dev)
    Z = torch.from_numpy(Zf).to(dev)
    Ge, Gr, H = (torch.empty_like(X) for _ in range(3))
    E1 = h.energy(X)
    E2, _ = h.grad(X, G_euc=Ge, G_riem=Gr)
    h.hessvec(X, Z, H, sigma=0.3, riemannian=True)
    h.sync()
    Xm = O.from_u(P, u)
    E_ref = O.energy(P, Xm)
    assert abs(E1 - E_ref) <= 1e-12 * abs(E_ref)
    assert abs(E2 - E_ref) <= 1e-12 * abs(E_ref)
    g = O.gradient(P, Xm)
    assert rel(Ge.cpu().numpy(), O.to_fields(P, g)) <= 1e-12
    Zm = O.to_matrix(P, Zf)
    Hr = O.rhess(P, u, O.to_u(P, Zm), g=O.to_u(P, g), sigma=0.3)
    assert rel(H.cpu().numpy(), O.to_fields(P, O.from_u(P, Hr))) <= 1e-11


@pytest.mark.parametrize("w", [W1, W2, W3], ids=lambda w: w.name)
def test_explicit_shapes_match_oracle(w, dev):
    from paper_1907_01194_gb300 import sbec
    P, u, Xf, Zf = case_inputs(w)
    with sbec.Handle.from_workload(w) as h:
        for shape in SHAPES[w.name]:
            h.set_tune(shape)
            got = h.get_tune()
            for k, v in shape.items():
                assert got[k] == v, (k, got)
            _check(h, P, u, Xf, Zf, dev)


@pytest.mark.parametrize("w", [W1, W2, W3], ids=lambda w: w.name)
def test_autotune_picks_valid_shapes_and_keeps_parity(w, dev):
    from paper_1907_01194_gb300 import sbec
    P, u, Xf, Zf = case_inputs(w)
    with sbec.Handle.from_workload(w) as h:
        X = torch.from_numpy(Xf).to(dev)
        t = h.autotune(X, reps=3)
        assert t["ms"] > 0
        got = h.get_tune()
        for k in ("x_rows", "s_pencils", "s_split", "elem_per_sm"):
            assert got[k] == t[k]
        _check(h, P, u, Xf, Zf, dev)


def test_invalid_shapes_are_rejected(dev):
    from paper_1907_01194_gb300 import sbec
    with sbec.Handle.from_workload(W2) as h:
        before = h.get_tune()
        for bad in (dict(x_rows=3), dict(x_rows=16), dict(s_pencils=[0, 128, 0]), dict(s_pencils=[0, 3, 0]),
                    dict(s_split=[0, 3, 0]), dict(s_pencils=[0, 0, 4]), dict(s_pencils=[2, 0, 0]),
                    dict(s_pencils=[0, 16, 0], s_split=[0, 16, 0]),     # the TMA pass: FP32 only
                    dict(elem_per_sm=33), dict(elem_per_sm=-1)):
            with pytest.raises(sbec.SbecError):
                h.set_tune(bad)
            assert h.get_tune() == before


def test_batch_autotune_matches_single_instances(dev):
    from paper_1907_01194_gb300 import sbec
    rng = np.random.default_rng(9)
    ws = [W.Workload(f"tb{i}", F=1, n=(64, 64), lo=(-8.0, -8.0), hi=(8.0, 8.0),
                     beta=(float(rng.uniform(30, 90)), float(rng.uniform(-2, 2)), 0.0, 0.0),
                     M=float(rng.uniform(0.05, 0.8)), seed=300 + i) for i in range(6)]
    X0 = np.stack([W.initial_fields(w) for w in ws])
    X = torch.from_numpy(X0).to(dev)
    with sbec.Handle.batch(ws) as hb:
        hb.autotune(X, reps=2)
        Eb = hb.energy(X)
    for i, w in enumerate(ws):
        P = O.Problem(F=w.F, n=w.n, lo=w.lo, hi=w.hi, beta=w.beta, V=W.potential(w), M=w.M)
        E_ref = O.energy(P, O.to_matrix(P, X0[i]))
        assert abs(Eb[i] - E_ref) <= 1e-12 * abs(E_ref)


def test_tma_pass_shapes_on_mixed_handles(dev):
    # FP32 passes along 128- or 256-point axes default to the TMA kernel with 16-column
    # tiles on the middle axis and 8-column tiles on the last (s_split = 16 marks the
    # TMA pass, s_pencils its width); widths other than
    # 8, 16, 32 are rejected, and the tuner may move between TMA widths and the
    # register kernels
    from paper_1907_01194_gb300 import sbec
    w = _wl(2, (32, 128, 128), 8.0, 0.3, (150.0, 4.0, -3.0, 0), lattice=6.0)
    with sbec.Handle.from_workload(w, precision="mixed") as h:
        t0 = h.get_tune()
        assert t0["s_pencils"][1:] == [16, 8] and t0["s_split"][1:] == [16, 16]
        for bad in (dict(s_pencils=[0, 4, 0], s_split=[0, 16, 0]), dict(s_pencils=[0, 64, 0], s_split=[0, 16, 0])):
            with pytest.raises(sbec.SbecError):
                h.set_tune(bad)
            assert h.get_tune() == t0
        X = torch.from_numpy(W.initial_fields(w).astype(np.complex64)).to(dev)
        t = h.autotune(X, reps=2)
        got = h.get_tune()
        for k in ("x_rows", "s_pencils", "s_split", "elem_per_sm"):
            assert got[k] == t[k]
        for ax in (1, 2):
            assert t["s_split"][ax] in (1, 2, 4, 16)
            if t["s_split"][ax] == 16:
                assert t["s_pencils"][ax] in (8, 16, 32)
