"""The bench's algorithmic work model (roofline numerators) against the counts
the design states: a length-m complex FFT is 5 m log2 m flops; the last-axis
pass is a forward and an inverse transform plus the |k|^2/G scaling (4 flops per
element); the 2D/3D gradient and Hessian epilogues are pointwise kernels of
their own (the inverse x transform before them is a separate launch), so their
flops are the per-point counts only; DRAM bytes are the compulsory reads and
writes of each launch in units of one field S and of the potential S_V."""
import math
import sys

import pytest

import bench
from paper_1907_01194_gb300 import workloads as W


def _fft(m):
    return 5.0 * m * math.log2(m)


@pytest.mark.parametrize("name", ["spin2_2d", "spin3_3d_128", "spin3_3d_256"])
def test_flop_model(name):
    w = bench.workload(name)
    C, n = w.C, w.n
    G = math.prod(n)
    rows_x = G // n[0]
    assert bench.flops_model(w, "x_fwd") == C * rows_x * _fft(n[0])
    assert bench.flops_model(w, "x_inv") == C * rows_x * _fft(n[0])
    assert bench.flops_model(w, "x_fwd_energy") == C * rows_x * _fft(n[0]) + G * bench.PW_FLOPS["energy"][w.F]
    # epilogues: pointwise only
    assert bench.flops_model(w, "x_inv_grad") == G * bench.PW_FLOPS["grad"][w.F]
    # the FP64 Hessian epilogue reads the densities the gradient stored
    assert bench.flops_model(w, "x_inv_hess") == G * (bench.PW_FLOPS["hess"][w.F] - bench.DENS_FLOPS[w.F])
    assert 0 < bench.DENS_FLOPS[w.F] < bench.PW_FLOPS["energy"][w.F]
    m = n[-1]
    assert bench.flops_model(w, "s_k2") == C * (G // m) * (2 * _fft(m) + 4 * m)
    # batches scale linearly
    assert bench.flops_model(w, "x_inv_hess", 3) == 3 * bench.flops_model(w, "x_inv_hess")


def test_flop_model_1d_full_passes():
    w = W.spin1_1d()
    n, C, G = w.n[0], w.C, w.n[0]
    assert bench.flops_model(w, "x_full_grad") == C * (2 * _fft(n) + 4 * n) + G * bench.PW_FLOPS["grad"][1]
    assert bench.flops_model(w, "x_full_hess") == C * (2 * _fft(n) + 4 * n) + G * bench.PW_FLOPS["hess"][1]


@pytest.mark.parametrize("elem", [8, 16])
def test_byte_model(elem):
    w = bench.workload("spin3_3d_256")
    G = math.prod(w.n)
    S = w.C * G * elem
    SV = G * elem // 2
    expect = {"x_fwd": 2 * S, "x_inv": 2 * S, "x_fwd_energy": 2 * S + SV, "s_fwd": 2 * S, "s_inv": 2 * S,
              "s_k2": 2 * S, "s_parseval": S, "x_inv_grad": 3 * S + SV, "x_inv_hess": 4 * S + SV,
              "proj_apply": 3 * S, "dot_reduce": 2 * S, "retract_w": 3 * S, "scale": 2 * S, "lincomb": 3 * S}
    for k, v in expect.items():
        assert bench.bytes_model(w, k, elem) == v, k
    assert bench.bytes_model(w, "finalize", elem) is None


def test_roofline_picks_the_longest_modelled_kernel():
    w = bench.workload("spin3_3d_128")
    prof = {"x_inv_hess": (4.0, 1), "s_k2": (2.5, 2), "finalize": (9.0, 3)}
    r = bench.roofline_of(prof, w, "fp64", 1, w.name)
    assert r["kernel"] == "x_inv_hess" and r["bound"] == "alu"
    fl = math.prod(w.n) * (bench.PW_FLOPS["hess"][w.F] - bench.DENS_FLOPS[w.F])
    assert r["achieved"] == pytest.approx(fl / 4.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_NOMINAL_GFLOPS)
    # with a measured FP64 rate the fraction is of that rate
    r = bench.roofline_of(prof, w, "fp64", 1, w.name, fp64_peak=1000.0)
    assert r["peak"] == 1000.0 and r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert r["peak_source"].startswith("measured")


def test_cpu_sample_slab_of_large_grids():
    # grids above 2^21 points are sampled on a z-slab of 2^20 points of the same
    # workload (same spacing and potential values), scaled by the slab's share
    import numpy as np
    from paper_1907_01194_gb300 import workloads as W
    w = bench.workload("spin3_3d_256")
    ws, share, desc = bench.cpu_workload_sample(w)
    assert ws.n == (256, 256, 16) and share == pytest.approx(1 / 16)
    assert ws.dV == pytest.approx(w.dV, rel=1e-15)
    assert np.array_equal(W.potential(ws), W.potential(w)[120:136])
    small = bench.workload("spin2_2d")
    assert bench.cpu_workload_sample(small)[0] is small


def test_grid_option_is_an_evaluation_rate_only_run(monkeypatch):
    # --grid runs the workload's problem on another grid (small profiling cases): no
    # solves and no CPU baseline; the batched sweep has no single grid to change
    monkeypatch.setattr(sys, "argv", ["bench.py", "--grid", "128,128,256", "--precision", "mixed"])
    a = bench.parse()
    assert a.grid == "128,128,256" and a.no_solve and a.no_cpu_baseline
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "batch512", "--grid", "64,64"])
    with pytest.raises(SystemExit):
        bench.parse()


def test_stored_oracle_ground_states_are_read_by_name():
    # the bench's time-to-ground-state entries compare with these stored energies
    assert bench.golden_ground_state("spin2_2d_256x256") == pytest.approx(19.227438467888131, rel=1e-15)
    assert bench.golden_ground_state("spin3_3d_128cubed") == pytest.approx(4.826029455710223, rel=1e-15)
    assert bench.golden_ground_state("no_such_workload") is None
    r = bench.gold_report(2.0, {"fp64": 2.0 + 2e-12})
    assert r["energy"] == 2.0 and r["fp64_rel_err"] == pytest.approx(1e-12)
