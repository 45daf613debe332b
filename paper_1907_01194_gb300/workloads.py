"""Seeded synthetic workloads: problem parameters, potentials on the grid and
raw initial / direction fields.

This module holds no arithmetic of the method (no energy, gradient, FFT,
projection or retraction).  It only samples the inputs the paper's problems
are stated with (Sec. 7: domain, grid, trap and lattice potential, interaction
strengths, magnetisation) and draws seeded random fields.  Both the CUDA path
and the CPU oracle take their inputs from here, so they start from identical
bits.

Random numbers come from numpy's PCG64 generator with the seeds given below.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

SEED_BASE = 190701194


@dataclass(frozen=True)
class Workload:
    """One problem instance.

    n, lo, hi are per axis in (x, y, z) order.  The potential is
    V(x) = harmonic * |x|^2 + lattice_amp * sum_i sin^2(lattice_k * x_i).
    beta = (beta0, beta1, beta2, beta3); entries beyond the spin's terms are 0.
    levels lists coarser grids (per-axis n) solved first by the cascadic driver.
    """
    name: str
    F: int
    n: tuple
    lo: tuple
    hi: tuple
    beta: tuple
    M: float
    p: float = 0.0
    q: float = 0.0
    harmonic: float = 0.5
    lattice_amp: float = 0.0
    lattice_k: float = 0.0
    seed: int = SEED_BASE
    levels: tuple = ()

    @property
    def C(self) -> int:
        return 2 * self.F + 1

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        """Array shape of one component: (n_z, n_y, n_x), x fastest."""
        return tuple(reversed(self.n))

    @property
    def G(self) -> int:
        return int(np.prod(self.n))

    @property
    def dV(self) -> float:
        return float(np.prod([(b - a) / m for a, b, m in zip(self.lo, self.hi, self.n)]))

    def at(self, n) -> "Workload":
        """The same problem on another grid (for the cascadic levels)."""
        return replace(self, n=tuple(n), levels=())


def grid_axes(w: Workload):
    """Grid points x_j = a + j h, j = 0..n-1, per axis (x, y, z)."""
    return [w.lo[i] + (w.hi[i] - w.lo[i]) / w.n[i] * np.arange(w.n[i]) for i in range(w.dim)]


def potential(w: Workload) -> np.ndarray:
    """V sampled at the grid points, float64 array of shape w.shape."""
    axes = grid_axes(w)
    V = np.zeros(w.shape)
    for i, x in enumerate(axes):
        sh = [1] * w.dim
        sh[w.dim - 1 - i] = w.n[i]
        term = w.harmonic * x ** 2
        if w.lattice_amp != 0.0:
            term = term + w.lattice_amp * np.sin(w.lattice_k * x) ** 2
        V = V + term.reshape(sh)
    return V


def initial_fields(w: Workload, seed: int | None = None) -> np.ndarray:
    """Raw initial data sqrt(dV) * exp(-|x|^2/2) * (1 + 0.1 U[-1,1]), drawn per
    component and grid point, real, complex128 array of shape (C,) + w.shape.

    It is not on the constraint manifold; each side puts it there with its own
    projection.
    """
    rng = np.random.Generator(np.random.PCG64(w.seed if seed is None else seed))
    axes = grid_axes(w)
    r2 = np.zeros(w.shape)
    for i, x in enumerate(axes):
        sh = [1] * w.dim
        sh[w.dim - 1 - i] = w.n[i]
        r2 = r2 + (x ** 2).reshape(sh)
    base = np.exp(-r2 / 2.0)
    noise = rng.uniform(-1.0, 1.0, size=(w.C,) + w.shape)
    X = np.sqrt(w.dV) * base[None] * (1.0 + 0.1 * noise)
    return X.astype(np.complex128)


def random_fields(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Complex Gaussian field (real and imaginary parts N(0, scale^2))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))).astype(np.complex128)


def smooth_random_fields(w: Workload, seed: int) -> np.ndarray:
    """Random complex field times the Gaussian envelope of the initial data:
    a direction with the spatial decay of the states it perturbs."""
    axes = grid_axes(w)
    r2 = np.zeros(w.shape)
    for i, x in enumerate(axes):
        sh = [1] * w.dim
        sh[w.dim - 1 - i] = w.n[i]
        r2 = r2 + (x ** 2).reshape(sh)
    env = np.sqrt(w.dV) * np.exp(-r2 / 2.0)
    return random_fields((w.C,) + w.shape, seed) * env[None]


# ---------------------------------------------------------------------------
# The five benchmark workloads (synthetic relatives of the paper's Sec. 7 cases)
# ---------------------------------------------------------------------------

def spin1_1d() -> Workload:
    """Spin-1, 1D, n = 256 on [-16,16], V = x^2/2, beta = (100, -0.5), M = 0.5."""
    return Workload("spin1_1d_n256", F=1, n=(256,), lo=(-16.0,), hi=(16.0,),
                    beta=(100.0, -0.5, 0.0, 0.0), M=0.5, seed=SEED_BASE + 1)


def spin2_2d() -> Workload:
    """Spin-2, 2D, 256^2 on [-12,12]^2, V = |x|^2/2 + 20 sum sin^2(pi x_i / 2),
    beta = (200, 10, -5), M = 0.3."""
    return Workload("spin2_2d_256x256", F=2, n=(256, 256), lo=(-12.0, -12.0), hi=(12.0, 12.0),
                    beta=(200.0, 10.0, -5.0, 0.0), M=0.3, lattice_amp=20.0,
                    lattice_k=np.pi / 2, seed=SEED_BASE + 2)


def spin3_3d_cascadic() -> Workload:
    """Spin-3, 3D, cascadic 32^3 -> 64^3 -> 128^3 on [-8,8]^3, harmonic,
    beta = (500, -2, 5, -1), M = 0.2."""
    return Workload("spin3_3d_128cubed", F=3, n=(128, 128, 128), lo=(-8.0,) * 3, hi=(8.0,) * 3,
                    beta=(500.0, -2.0, 5.0, -1.0), M=0.2, seed=SEED_BASE + 3,
                    levels=((32, 32, 32), (64, 64, 64)))


def spin3_3d_256() -> Workload:
    """Spin-3, 3D, 256^3 on [-10,10]^3, V = harmonic + 10 sum sin^2(pi x_i / 2),
    beta = (1000, -5, 10, 2), M = 0.  Its ground state is computed cascadically from the
    coarse levels n/4 and n/2 (64^3, 128^3)."""
    return Workload("spin3_3d_256cubed", F=3, n=(256, 256, 256), lo=(-10.0,) * 3, hi=(10.0,) * 3,
                    beta=(1000.0, -5.0, 10.0, 2.0), M=0.0, lattice_amp=10.0,
                    lattice_k=np.pi / 2, seed=SEED_BASE + 5, levels=((64, 64, 64), (128, 128, 128)))


def paper_spin2_2d(M: float, n: int = 256) -> Workload:
    """The paper's spin-2 2D case (Sec. 7.1): V = |x|^2/2 + 10 sum sin^2(pi x_i / 2),
    beta = (243, 12.1, -13), box [-8,8]^2, n = 2^8 per axis on the finest mesh."""
    return Workload(f"paper_spin2_2d_n{n}", F=2, n=(n, n), lo=(-8.0, -8.0), hi=(8.0, 8.0),
                    beta=(243.0, 12.1, -13.0, 0.0), M=M, lattice_amp=10.0, lattice_k=np.pi / 2)


def paper_spin1_2d(M: float, n: int = 512) -> Workload:
    """The paper's antiferromagnetic spin-1 2D case (Sec. 7.1): beta = (300, 100),
    box [-16,16]^2, n = 2^9 per axis, V = |x|^2/2 + 10 sum sin^2(pi x_i / 2).  The text
    prints sin^2(pi x_i / 4); the energies of its table belong to pi x_i / 2 (with it the
    printed values are reproduced to all four decimals, with pi x_i / 4 they are not)."""
    return Workload(f"paper_spin1_2d_n{n}", F=1, n=(n, n), lo=(-16.0, -16.0), hi=(16.0, 16.0),
                    beta=(300.0, 100.0, 0.0, 0.0), M=M, lattice_amp=10.0, lattice_k=np.pi / 2)


def paper_spin1_3d(M: float, n: int = 256) -> Workload:
    """The paper's ferromagnetic spin-1 3D case (Sec. 7.1): V = sum (x_i^2 +
    200 sin^2(pi x_i / 2)) / 2, beta = (880, -4.1), box [-16,16]^3, n = 2^8 per axis."""
    return Workload(f"paper_spin1_3d_n{n}", F=1, n=(n, n, n), lo=(-16.0,) * 3, hi=(16.0,) * 3,
                    beta=(880.0, -4.1, 0.0, 0.0), M=M, lattice_amp=100.0, lattice_k=np.pi / 2)


# The paper's spin-2 cases (Sec. 7.2): I ferromagnetic, II antiferromagnetic (nematic
# ground state), III cyclic
SPIN2_BETA = {1: (130.6, -25.4, -125.3, 0.0), 2: (243.0, 12.1, -13.0, 0.0), 3: (183.9, 26.8, 134.7, 0.0)}
# and spin-3 cases (Sec. 7.3)
SPIN3_BETA = {1: (100.0, 1.0, -10.0, -1.0), 2: (100.0, 1.0, 10.0, 1.0)}


def paper_spin2_2d_case(case: int, M: float, n: int = 256) -> Workload:
    """Sec. 7.2, spin-2 2D case I/II/III: V = |x|^2/2 + 10 sum sin^2(pi x_i / 2), box
    [-8,8]^2, n = 2^8 per axis on the finest mesh."""
    return Workload(f"paper_spin2_2d_case{case}_n{n}", F=2, n=(n, n), lo=(-8.0, -8.0), hi=(8.0, 8.0),
                    beta=SPIN2_BETA[case], M=M, lattice_amp=10.0, lattice_k=np.pi / 2)


def paper_spin2_3d_case(case: int, M: float, n: int | None = None) -> Workload:
    """Sec. 7.2, spin-2 3D case I/II/III: V = |x|^2/2 + 100 sum sin^2(pi x_i / 2); case I
    on [-8,8] x [-16,16] x [-16,16] with n = 2^7, cases II and III on [-16,16]^3 with
    n = 2^8 per axis."""
    if case == 1:
        n = n or 128
        lo, hi = (-8.0, -16.0, -16.0), (8.0, 16.0, 16.0)
    else:
        n = n or 256
        lo, hi = (-16.0,) * 3, (16.0,) * 3
    return Workload(f"paper_spin2_3d_case{case}_n{n}", F=2, n=(n, n, n), lo=lo, hi=hi, beta=SPIN2_BETA[case], M=M,
                    lattice_amp=100.0, lattice_k=np.pi / 2)


def paper_spin3_2d(case: int, M: float, n: int = 256) -> Workload:
    """Sec. 7.3, spin-3 2D case I/II: V = |x|^2/2 + 10 sum sin^2(pi x_i / 2), box [-8,8]^2,
    n = 2^8 per axis."""
    return Workload(f"paper_spin3_2d_case{case}_n{n}", F=3, n=(n, n), lo=(-8.0, -8.0), hi=(8.0, 8.0),
                    beta=SPIN3_BETA[case], M=M, lattice_amp=10.0, lattice_k=np.pi / 2)


def paper_spin3_3d(case: int, M: float, n: int = 128) -> Workload:
    """Sec. 7.3, spin-3 3D case I/II: V = |x|^2/2 + 100 sum sin^2(pi x_i / 2), box
    [-8,8]^3, n = 2^7 per axis."""
    return Workload(f"paper_spin3_3d_case{case}_n{n}", F=3, n=(n, n, n), lo=(-8.0,) * 3, hi=(8.0,) * 3,
                    beta=SPIN3_BETA[case], M=M, lattice_amp=100.0, lattice_k=np.pi / 2)


def paper_spinor(w: Workload, seed: int = 0) -> np.ndarray:
    """The paper's initial spinor U (Sec. 7) for the interaction type of w.

    spin-1: ferromagnetic (beta1 <= 0) or antiferromagnetic; spin-2: ferromagnetic
    (beta1 < 0, beta2 > 20 beta1), nematic (beta2 < 0, beta2 < 20 beta1) or cyclic
    (beta1 > 0, beta2 > 0); spin-3: "a random vector", drawn here as 7 uniform
    numbers in [0, 1) from numpy's PCG64 with the given seed."""
    M = w.M
    if w.F == 1 and w.beta[1] <= 0.0:
        return np.array([np.sqrt(1.0 + 3.0 * M) / 2.0, np.sqrt((1.0 - M) / 2.0), np.sqrt(1.0 - M) / 2.0])
    if w.F == 1:
        return np.array([np.sqrt((1.0 + M) / 2.0), 0.0, np.sqrt((1.0 - M) / 2.0)])
    if w.F == 2:
        b1, b2 = w.beta[1], w.beta[2]
        if b1 < 0.0 and b2 > 20.0 * b1:
            m1, m2 = np.sqrt(2.0 + M), np.sqrt(2.0 - M)
            return np.array([m1 ** 4 / 16.0, m1 ** 3 * m2 / 8.0, np.sqrt(6.0) * m1 ** 2 * m2 ** 2 / 16.0,
                             m1 * m2 ** 3 / 8.0, m2 ** 4 / 16.0])
        if b2 < 0.0 and b2 < 20.0 * b1:
            return np.array([np.sqrt(2.0 + M) / 2.0, 0.0, 0.0, 0.0, np.sqrt(2.0 - M) / 2.0])
        if b1 > 0.0 and b2 > 0.0:
            return np.array([np.sqrt((M + 1.0) / 3.0), 0.0, 0.0, np.sqrt((2.0 - M) / 3.0), 0.0])
    if w.F == 3:
        return np.random.Generator(np.random.PCG64(seed)).uniform(0.0, 1.0, 7)
    raise ValueError("no initial spinor of the paper for this case")


def paper_initial(w: Workload, seed: int = 0) -> np.ndarray:
    """The paper's initial data U phi_0 (Sec. 7) with phi_0 = pi^{-d/4} exp(-|x|^2/2),
    scaled by sqrt(dV); complex128, (C,) + w.shape (seed: the spin-3 random spinor)."""
    axes = grid_axes(w)
    r2 = np.zeros(w.shape)
    for i, x in enumerate(axes):
        sh = [1] * w.dim
        sh[w.dim - 1 - i] = w.n[i]
        r2 = r2 + (x ** 2).reshape(sh)
    phi0 = np.pi ** (-w.dim / 4.0) * np.exp(-r2 / 2.0)
    U = paper_spinor(w, seed)
    return (np.sqrt(w.dV) * U.reshape((w.C,) + (1,) * w.dim) * phi0[None]).astype(np.complex128)


def paper_nematic_initial(w: Workload) -> np.ndarray:
    """paper_initial for the nematic spin-2 case."""
    assert w.F == 2
    return paper_initial(w)


def batched_spin1_2d(count: int = 512) -> list:
    """Batched spin-1 2D sweep: instance i has n = (64,128,256)[i mod 3] per axis
    on [-10,10]^2, harmonic, beta0 = 100, beta1_i ~ U[-2,2], M_i ~ U[0,0.9]
    drawn in order from PCG64(SEED_BASE + 4); init seed SEED_BASE + 1000 + i."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4))
    out = []
    for i in range(count):
        b1 = float(rng.uniform(-2.0, 2.0))
        M = float(rng.uniform(0.0, 0.9))
        n = (64, 128, 256)[i % 3]
        out.append(Workload(f"batch{i}", F=1, n=(n, n), lo=(-10.0, -10.0), hi=(10.0, 10.0),
                            beta=(100.0, b1, 0.0, 0.0), M=M, seed=SEED_BASE + 1000 + i))
    return out


CONFIGS = {
    "spin1_1d": spin1_1d,
    "spin2_2d": spin2_2d,
    "spin3_3d_cascadic": spin3_3d_cascadic,
    "spin3_3d_256": spin3_3d_256,
}
