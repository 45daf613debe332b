"""Plain CPU FP64 oracle for the spin-F BEC ground-state computation of
Tian, Cai, Wu & Wen, "Ground states and their characterization of spin-F
Bose-Einstein condensates" (arXiv:1907.01194).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
restatement of the paper that the CUDA library is checked against.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may
import it.  The product path (the C-ABI library and its Python binding) never
imports, links or calls anything here, and nothing here calls the product.

Notation follows the paper:

* Sec. 3: the wavefunction is the matrix X = (sqrt(h) phi_{jl}) in C^{G x C},
  grid points j as rows, components l = F, ..., -F as columns; in d dimensions
  h becomes the cell volume dV = prod_i h_i (the paper leaves multi-D as
  "straightforward"; the reading is stated in the package's design notes).
  Grid points are x_j = a + j h, j = 0..n-1, on every axis.  The grid is held
  as a numpy array of shape (n_z, n_y, n_x) (x fastest), and the matrix row
  index is the C-order flattening of that array.
* Eq. (3.5)-(3.6): the discrete negative Laplacian L = C^* Lambda C with
  lambda_p = 2 pi p / (b - a), p = -n/2 .. n/2-1, acting on every axis.
* Eq. (3.7): E_h(X); the gradient (3.12) and the Hessian-vector product (3.13).
* Sec. 4: the real stacking u in R^N, Gamma, the projection of Lemma 4.1 and the
  Riemannian Hessian of Lemma 4.2.
* Sec. 5 and Algorithm 1: RGBB, ARNT with the modified CG, cascadic levels.
* Sec. 6: the retractions R1 (Lemma 5.1), R2 (Lemma 5.3), R3 (Lemma 5.4).

Where the paper is silent or inconsistent, the reading used is stated next to
the code that depends on it (spin-3 quintet constants, R2 denominator, the
modified-CG details, sigma update, prolongation).

Every routine is pinned by a test in tests/test_oracle_*.py against something
other than itself: brute-force dense DFT matrices, closed-form Gaussian
energies, finite differences, invariants of the projection and retractions,
the spin-1 special cases of Lemma 5.2, the spin-1 quadratic form of R2, the
harmonic ground-state energy d/2, the scalar-GPE reduction, the Zeeman shift,
and the ten-digit spin-2 energies printed in the paper's Sec. 7.2 tables.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft


# ---------------------------------------------------------------------------
# Sec. 2: spin matrices and singlet / quintet pair matrices, as printed.
# Basis order is l = F, F-1, ..., -F (first row/column is l = F).
# ---------------------------------------------------------------------------

def spin_matrices(F: int):
    """(f_x, f_y, f_z) for F = 1, 2, 3 exactly as printed in Sec. 2."""
    if F == 1:
        s = 1.0 / math.sqrt(2.0)
        fx = s * np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=complex)
        fy = 1j * s * np.array([[0, -1, 0], [1, 0, -1], [0, 1, 0]], dtype=complex)
        fz = np.diag([1.0, 0.0, -1.0]).astype(complex)
    elif F == 2:
        a = math.sqrt(1.5)
        fx = np.array([[0, 1, 0, 0, 0],
                       [1, 0, a, 0, 0],
                       [0, a, 0, a, 0],
                       [0, 0, a, 0, 1],
                       [0, 0, 0, 1, 0]], dtype=complex)
        fy = 1j * np.array([[0, -1, 0, 0, 0],
                            [1, 0, -a, 0, 0],
                            [0, a, 0, -a, 0],
                            [0, 0, a, 0, -1],
                            [0, 0, 0, 1, 0]], dtype=complex)
        fz = np.diag([2.0, 1.0, 0.0, -1.0, -2.0]).astype(complex)
    elif F == 3:
        a, b, c = math.sqrt(1.5), math.sqrt(2.5), math.sqrt(3.0)
        fx = np.array([[0, a, 0, 0, 0, 0, 0],
                       [a, 0, b, 0, 0, 0, 0],
                       [0, b, 0, c, 0, 0, 0],
                       [0, 0, c, 0, c, 0, 0],
                       [0, 0, 0, c, 0, b, 0],
                       [0, 0, 0, 0, b, 0, a],
                       [0, 0, 0, 0, 0, a, 0]], dtype=complex)
        fy = 1j * np.array([[0, -a, 0, 0, 0, 0, 0],
                            [a, 0, -b, 0, 0, 0, 0],
                            [0, b, 0, -c, 0, 0, 0],
                            [0, 0, c, 0, -c, 0, 0],
                            [0, 0, 0, c, 0, -b, 0],
                            [0, 0, 0, 0, b, 0, -a],
                            [0, 0, 0, 0, 0, a, 0]], dtype=complex)
        fz = np.diag([3.0, 2.0, 1.0, 0.0, -1.0, -2.0, -3.0]).astype(complex)
    else:
        return spin_matrices_general(F)
    return fx, fy, fz


def spin_matrices_general(F: int):
    """(f_x, f_y, f_z) for any integer spin F: the angular-momentum matrices the
    printed F = 1, 2, 3 ones are instances of (Sec. 2), in the basis l = F..-F.
    f_z = diag(l); the raising matrix has (f_+)_{l+1, l} = sqrt(F(F+1) - l(l+1));
    f_x = (f_+ + f_-)/2 and f_y = (f_+ - f_-)/(2i) with f_- = f_+^T.  The paper
    prints the matrices for F <= 3 only; for F >= 4 this is the reading of its
    claim that the method applies to any integer spin."""
    C = 2 * F + 1
    ls = np.arange(F, -F - 1, -1)
    fp = np.zeros((C, C))
    for j in range(1, C):                     # row j-1 holds l + 1, column j holds l
        l = ls[j]
        fp[j - 1, j] = math.sqrt(F * (F + 1) - l * (l + 1))
    fm = fp.T
    fx = (fp + fm).astype(complex) / 2.0
    fy = (fp - fm).astype(complex) / 2.0j
    fz = np.diag(ls.astype(float)).astype(complex)
    return fx, fy, fz


def singlet_matrix(F: int):
    """The singlet-pair matrix bold-A of Sec. 2 (F = 2: 1/sqrt5, F = 3: 1/sqrt7).
    For F >= 4 (reading): the same alternating anti-diagonal, A[j, 2F-j] =
    (-1)^j / sqrt(2F+1), the pattern of the printed F = 2, 3 matrices."""
    if F >= 4:
        A = np.zeros((2 * F + 1, 2 * F + 1))
        for j in range(2 * F + 1):
            A[j, 2 * F - j] = (-1.0) ** j
        return A / math.sqrt(2 * F + 1.0)
    if F == 2:
        A = np.zeros((5, 5))
        for j, s in enumerate([1, -1, 1, -1, 1]):
            A[j, 4 - j] = s
        return A / math.sqrt(5.0)
    if F == 3:
        A = np.zeros((7, 7))
        for j, s in enumerate([1, -1, 1, -1, 1, -1, 1]):
            A[j, 6 - j] = s
        return A / math.sqrt(7.0)
    return None


def quintet_matrices(F: int):
    """The spin-3 quintet matrices bold-A_l, l = 2, 1, 0, -1, -2 (Sec. 2).

    A_0 is the printed 7x7 matrix.  A_{+-1}, A_{+-2} are built from the printed
    vectors a_l: the only nonzero entries of A_l are at (1-based) j + k = 8 - l,
    listed by increasing row index j.  Reading (quintet constant): the printed
    vector a_{+-2} (its psi_{+-1}^2 entry sqrt2/sqrt7, unit norm) is used; the
    explicit A_{2,+-2} formula printed beside it gives sqrt2/sqrt21 instead,
    which is taken to be a misprint because the vectors define the matrices
    that enter E_h, its gradient and its Hessian.
    Returns a dict l -> 7x7 real symmetric matrix.
    """
    if F != 3:
        return {}
    r7 = math.sqrt(7.0)
    A0 = np.zeros((7, 7))
    A0[0, 6] = A0[6, 0] = 5.0 / (2.0 * math.sqrt(3.0))
    A0[2, 4] = A0[4, 2] = -math.sqrt(3.0) / 2.0
    A0[3, 3] = math.sqrt(2.0 / 3.0)
    A0 /= r7
    a1 = np.array([5.0 / (2.0 * math.sqrt(3.0)), -math.sqrt(5.0) / 2.0, 1.0 / math.sqrt(6.0),
                   1.0 / math.sqrt(6.0), -math.sqrt(5.0) / 2.0, 5.0 / (2.0 * math.sqrt(3.0))]) / r7
    a2 = np.array([math.sqrt(5.0 / 6.0), -math.sqrt(5.0 / 3.0), math.sqrt(2.0),
                   -math.sqrt(5.0 / 3.0), math.sqrt(5.0 / 6.0)]) / r7
    mats = {0: A0}
    for l, vec in ((1, a1), (2, a2), (-1, a1), (-2, a2)):
        A = np.zeros((7, 7))
        # rows j (1-based) with a partner k = 8 - l - j inside 1..7
        rows = [j for j in range(1, 8) if 1 <= 8 - l - j <= 7]
        assert len(rows) == len(vec)
        for i, j in enumerate(rows):
            A[j - 1, 8 - l - j - 1] = vec[i]
        mats[l] = A
    return mats


# ---------------------------------------------------------------------------
# Problem: grid, potential, Zeeman diagonal, Laplacian symbol (Sec. 3)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """A discretised spin-F problem.

    n, lo, hi are per axis in the order (x, y, z); V is the potential sampled
    at the grid points as an array of shape (n_z, n_y, n_x) (d entries).
    """
    F: int
    n: tuple
    lo: tuple
    hi: tuple
    beta: tuple            # (beta0, beta1, beta2, beta3); unused entries ignored
    V: np.ndarray
    p: float = 0.0
    q: float = 0.0
    M: float = 0.0
    # derived
    C: int = field(init=False)
    d: int = field(init=False)
    shape: tuple = field(init=False)
    G: int = field(init=False)
    h: tuple = field(init=False)
    dV: float = field(init=False)
    ls: np.ndarray = field(init=False)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.lo = tuple(float(v) for v in self.lo)
        self.hi = tuple(float(v) for v in self.hi)
        self.d = len(self.n)
        assert isinstance(self.F, int) and self.F >= 1
        assert len(self.lo) == self.d and len(self.hi) == self.d
        self.C = 2 * self.F + 1
        self.shape = tuple(reversed(self.n))          # (n_z, n_y, n_x)
        self.G = int(np.prod(self.n))
        self.h = tuple((b - a) / m for a, b, m in zip(self.lo, self.hi, self.n))
        self.dV = float(np.prod(self.h))
        self.V = np.asarray(self.V, dtype=np.float64).reshape(self.shape)
        self.ls = np.arange(self.F, -self.F - 1, -1).astype(np.float64)   # l = F..-F
        beta = tuple(self.beta) + (0.0,) * (4 - len(self.beta))
        self.beta = tuple(float(b) for b in beta[:4])
        # Zeeman diagonal b_l = -p l + q l^2 (Sec. 3, B = diag(b))
        self.bvec = -self.p * self.ls + self.q * self.ls ** 2
        self.fx, self.fy, self.fz = spin_matrices(self.F)
        self.A = singlet_matrix(self.F)
        self.Aq = quintet_matrices(self.F)
        self.k2 = self._laplacian_symbol()

    # lambda_p^2 summed over axes on the numpy FFT frequency ordering
    def _laplacian_symbol(self):
        k2 = np.zeros(self.shape)
        for i in range(self.d):
            n, L = self.n[i], self.hi[i] - self.lo[i]
            p = np.fft.fftfreq(n, d=1.0 / n)            # 0,1,..,n/2-1,-n/2,..,-1
            lam2 = (2.0 * math.pi * p / L) ** 2
            ax = self.d - 1 - i                          # numpy axis of problem axis i
            sh = [1] * self.d
            sh[ax] = n
            k2 = k2 + lam2.reshape(sh)
        return k2

    def grid_axes(self):
        """x_j = a + j h, j = 0..n-1 per axis (x, y, z)."""
        return [self.lo[i] + self.h[i] * np.arange(self.n[i]) for i in range(self.d)]


# ---------------------------------------------------------------------------
# Layout helpers: component fields (C, n_z, n_y, n_x) <-> the matrix X (G x C)
# ---------------------------------------------------------------------------

def to_matrix(P: Problem, fields):
    fields = np.asarray(fields)
    return fields.reshape(P.C, P.G).T.copy()


def to_fields(P: Problem, X):
    return np.asarray(X).T.reshape((P.C,) + P.shape).copy()


def to_u(P: Problem, X):
    """Real stacking of Sec. 4: (X_r; X_i) column by column, u in R^{2G(2F+1)}."""
    X = np.asarray(X)
    return np.concatenate([np.concatenate([X[:, c].real, X[:, c].imag]) for c in range(P.C)])


def from_u(P: Problem, u):
    u = np.asarray(u, dtype=np.float64)
    G = P.G
    X = np.empty((G, P.C), dtype=complex)
    for c in range(P.C):
        blk = u[2 * G * c: 2 * G * (c + 1)]
        X[:, c] = blk[:G] + 1j * blk[G:]
    return X


def gamma_weights(P: Problem):
    """Diagonal of Gamma = diag(F I_{2n}, ..., -F I_{2n}) as an N-vector."""
    return np.repeat(P.ls, 2 * P.G)


# ---------------------------------------------------------------------------
# Discrete operators (Sec. 3)
# ---------------------------------------------------------------------------

def laplacian(P: Problem, X):
    """L X with L the Fourier pseudospectral negative Laplacian, every column."""
    out = np.empty_like(X, dtype=complex)
    axes = tuple(range(P.d))
    for c in range(P.C):
        col = X[:, c].reshape(P.shape)
        hat = sfft.fftn(col, axes=axes)                       # unnormalised forward DFT
        out[:, c] = sfft.ifftn(P.k2 * hat, axes=axes).reshape(P.G)   # 1/G in the inverse
    return out


def dense_laplacian_1d(n: int, a: float, b: float):
    """L = (1/n) sum_p lambda_p^2 e^{i 2 pi (j-k) p / n}, written out (n small)."""
    j = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    L = np.zeros((n, n), dtype=complex)
    for p in range(-n // 2, n // 2):
        lam = 2.0 * math.pi * p / (b - a)
        L += lam * lam * np.exp(1j * 2.0 * math.pi * (j - k) * p / n)
    return L / n


def dense_laplacian(P: Problem):
    """Dense G x G matrix of L on the C-order flattened grid (tiny grids only)."""
    mats = [dense_laplacian_1d(P.n[i], P.lo[i], P.hi[i]) for i in range(P.d)]
    # numpy axis order is (z, y, x): Kronecker factors in that order
    order = list(reversed(range(P.d)))
    L = np.zeros((P.G, P.G), dtype=complex)
    for i in range(P.d):
        factors = [mats[i] if ax == i else np.eye(P.n[ax]) for ax in order]
        K = factors[0]
        for f in factors[1:]:
            K = np.kron(K, f)
        L += K
    return L


def densities(P: Problem, X):
    """rho, F_alpha (alpha = x, y, z), A00 and A2l as column vectors (Sec. 3)."""
    rho = np.sum(X * X.conj(), axis=1).real                     # diag(X X^*)
    Fa = [np.sum((X @ f.T) * X.conj(), axis=1).real for f in (P.fx, P.fy, P.fz)]
    A00 = np.sum((X @ P.A) * X, axis=1) if P.A is not None else None     # diag(X A X^T)
    A2 = {l: np.sum((X @ Al) * X, axis=1) for l, Al in P.Aq.items()}
    return rho, Fa, A00, A2


def energy(P: Problem, X):
    """E_h(X), Eq. (3.7) with h -> dV."""
    b0, b1, b2, b3 = P.beta
    h = P.dV
    LX = laplacian(P, X)
    E = 0.5 * np.real(np.sum(X.conj() * LX))                    # (1/2) tr(X^* L X)
    E += np.sum(P.V.reshape(P.G)[:, None] * np.abs(X) ** 2)     # tr(X^* V X)
    E += np.real(np.sum((X * P.bvec[None, :]) * X.conj()))      # tr(X B X^*)
    rho, Fa, A00, A2 = densities(P, X)
    E += b0 / (2 * h) * rho @ rho
    E += b1 / (2 * h) * sum(F @ F for F in Fa)
    if A00 is not None:
        E += b2 / (2 * h) * np.real(np.vdot(A00, A00))
    for l in A2:
        E += b3 / (2 * h) * np.real(np.vdot(A2[l], A2[l]))
    return float(E)


def _gradient_local(P: Problem, X, V):
    """The terms of Eq. (3.12) other than L X, for rows X of the matrix (grid points)
    with potential values V at those points: every one of them is pointwise."""
    b0, b1, b2, b3 = P.beta
    h = P.dV
    V = np.asarray(V)[:, None]
    rho, Fa, A00, A2 = densities(P, X)
    G = 2 * V * X + 2 * X * P.bvec[None, :]
    G += (2 * b0 / h) * rho[:, None] * X
    for F, f in zip(Fa, (P.fx, P.fy, P.fz)):
        G += (2 * b1 / h) * F[:, None] * (X @ f.T)
    if A00 is not None:
        G += (2 * b2 / h) * A00[:, None] * (X.conj() @ P.A)
    for l, Al in P.Aq.items():
        G += (2 * b3 / h) * A2[l][:, None] * (X.conj() @ Al)
    return G


def gradient(P: Problem, X):
    """Euclidean gradient nabla E_h(X) w.r.t. Re<.,.>, Eq. (3.12) with h -> dV."""
    return laplacian(P, X) + _gradient_local(P, X, P.V.reshape(P.G))


def _hessvec_local(P: Problem, X, Z, V):
    """The terms of Eq. (3.13) other than L Z, for rows X, Z (grid points) with
    potential values V there: every one of them is pointwise."""
    b0, b1, b2, b3 = P.beta
    h = P.dV
    V = np.asarray(V)[:, None]
    rho, Fa, A00, A2 = densities(P, X)
    H = 2 * V * Z + 2 * Z * P.bvec[None, :]
    reZX = np.sum(Z * X.conj(), axis=1).real                    # diag(Re(Z X^*))
    H += (2 * b0 / h) * (rho[:, None] * Z + 2 * reZX[:, None] * X)
    for F, f in zip(Fa, (P.fx, P.fy, P.fz)):
        reZfX = np.sum((Z @ f.T) * X.conj(), axis=1).real       # diag(Re(Z f^T X^*))
        H += (2 * b1 / h) * (F[:, None] * (Z @ f.T) + 2 * reZfX[:, None] * (X @ f.T))
    if A00 is not None:
        ZAX = np.sum((Z @ P.A) * X, axis=1)                     # diag(Z A X^T)
        H += (2 * b2 / h) * (A00[:, None] * (Z.conj() @ P.A) + 2 * ZAX[:, None] * (X.conj() @ P.A))
    for l, Al in P.Aq.items():
        ZAX = np.sum((Z @ Al) * X, axis=1)
        H += (2 * b3 / h) * (A2[l][:, None] * (Z.conj() @ Al) + 2 * ZAX[:, None] * (X.conj() @ Al))
    return H


def hessvec(P: Problem, X, Z):
    """Euclidean Hessian-vector product nabla^2 E_h(X)[Z], Eq. (3.13), h -> dV."""
    return laplacian(P, Z) + _hessvec_local(P, X, Z, P.V.reshape(P.G))


# ---------------------------------------------------------------------------
# The same quantities at a few grid points of a large grid: L is the sum over
# the axes of the 1D operator of Eq. (3.5) acting along that axis, so (L X)_j
# needs one row of each 1D matrix and the grid lines through x_j.
# ---------------------------------------------------------------------------

def laplacian_at(P: Problem, X, idx):
    """(L X)_j for the flat (C-order) grid indices idx."""
    idx = np.asarray(idx)
    Xg = np.asarray(X).reshape(P.shape + (P.C,))               # (n_z, n_y, n_x, C)
    coords = np.unravel_index(idx, P.shape)                    # numpy axis order (z, y, x)
    out = np.zeros((idx.size, P.C), dtype=complex)
    for i in range(P.d):
        ax = P.d - 1 - i                                       # numpy axis of problem axis i
        L1 = dense_laplacian_1d(P.n[i], P.lo[i], P.hi[i])
        for r in range(idx.size):
            at = [int(coords[k][r]) for k in range(P.d)]
            line = [slice(None) if k == ax else at[k] for k in range(P.d)]
            out[r] += L1[at[ax], :] @ Xg[tuple(line)]
    return out


def gradient_at(P: Problem, X, idx):
    """Rows idx of nabla E_h(X) (Eq. 3.12)."""
    X = np.asarray(X)
    return laplacian_at(P, X, idx) + _gradient_local(P, X[idx], P.V.reshape(P.G)[idx])


def hessvec_at(P: Problem, X, Z, idx):
    """Rows idx of nabla^2 E_h(X)[Z] (Eq. 3.13)."""
    X, Z = np.asarray(X), np.asarray(Z)
    return laplacian_at(P, Z, idx) + _hessvec_local(P, X[idx], Z[idx], P.V.reshape(P.G)[idx])


def constraints(P: Problem, X):
    """(tr(X^* X), tr(X^* X D)) of Sec. 3."""
    m = np.sum(np.abs(X) ** 2, axis=0)
    return float(m.sum()), float(m @ P.ls)


# ---------------------------------------------------------------------------
# Manifold geometry (Sec. 4) on the real stacking u in R^N
# ---------------------------------------------------------------------------

def E_u(P, u):
    return energy(P, from_u(P, u))


def egrad_u(P, u):
    return to_u(P, gradient(P, from_u(P, u)))


def ehess_u(P, u, xi):
    return to_u(P, hessvec(P, from_u(P, u), from_u(P, xi)))


def project(P: Problem, u, w):
    """Lemma 4.1: orthogonal projection of w onto T_u M."""
    Gm = gamma_weights(P)
    M = P.M
    uGGu = u @ (Gm * Gm * u)
    uw = u @ w
    uGw = u @ (Gm * w)
    den = uGGu - M * M
    if not den > 0:
        raise FloatingPointError("u^T Gamma^2 u - M^2 <= 0: outside the manifold's domain")
    return w - (uGGu * uw - M * uGw) / den * u + (M * uw - uGw) / den * (Gm * u)


def rgrad(P: Problem, u, g=None):
    """grad f(u) = P_u nabla f(u), Eq. (4.6)."""
    if g is None:
        g = egrad_u(P, u)
    return project(P, u, g)


def rhess(P: Problem, u, xi, g=None, sigma=0.0):
    """Lemma 4.2 (formula Hess0), for f with Euclidean Hessian H + sigma I.

    g is the Euclidean gradient of f at u (recomputed if None); sigma adds the
    regularisation of the ARNT model m_k (its Euclidean Hessian is H_k + sigma I
    and its Euclidean gradient at u_k is nabla E(u_k)).
    """
    Gm = gamma_weights(P)
    M = P.M
    if g is None:
        g = egrad_u(P, u)
    # The lemma holds for xi in T_u M; xi is projected there first so that the
    # rounding-level normal part of a tangent input (for instance a Riemannian
    # gradient formed by cancellation) is not amplified by the dropped terms.
    xi = project(P, u, xi)
    he = ehess_u(P, u, xi) + sigma * xi
    au = u @ (Gm * Gm * u) - M * M                         # alpha_u
    ug, uGg = u @ g, u @ (Gm * g)
    ag = (1 + M * M / au) * ug - M / au * uGg                # alpha_g
    bg = -M / au * ug + 1.0 / au * uGg                       # beta_g
    bu = u @ (Gm * he) - bg * (u @ (Gm * Gm * xi))           # beta_u
    uGGu = u @ (Gm * Gm * u)
    return (he - ag * xi - bg * (Gm * xi)
            - (uGGu * (u @ he) - M * bu) / au * u
            + (M * (u @ he) - bu) / au * (Gm * u))


# ---------------------------------------------------------------------------
# Retractions (Sec. 6): R_u(xi) = psi(u + xi)
# ---------------------------------------------------------------------------

def _component_norms2(P: Problem, w):
    return np.array([w[2 * P.G * c: 2 * P.G * (c + 1)] @ w[2 * P.G * c: 2 * P.G * (c + 1)]
                     for c in range(P.C)])


def _scale_components(P: Problem, w, sig):
    out = w.copy()
    for c in range(P.C):
        out[2 * P.G * c: 2 * P.G * (c + 1)] *= sig[c]
    return out


def _f1_f2(P: Problem, m):
    nz = [P.ls[c] for c in range(P.C) if m[c] > 0]
    if not nz:
        raise FloatingPointError("w = 0")
    return min(nz), max(nz)


def psi_R1(P: Problem, w, return_r=False):
    """Lemma 5.1: the projection P_M(w) (projective retraction R1).

    r is the unique zero of the increasing h1 on (1/(f1-M), 1/(f2-M)); it is
    bracketed by bisection to the resolution of doubles and polished by Newton
    steps on h1 (Eq. hderi gives h1').
    """
    M = P.M
    m = _component_norms2(P, w)
    f1, f2 = _f1_f2(P, m)
    if not (f1 < M < f2):
        raise FloatingPointError("w is outside Omega (needs f1(w) < M < f2(w))")
    act = [(P.ls[c], m[c]) for c in range(P.C) if P.ls[c] >= f1 and P.ls[c] <= f2]

    def h1(t):
        return sum((l - M) * mm / (1 - (l - M) * t) ** 2 for l, mm in act)

    def dh1(t):
        return sum(2 * (l - M) ** 2 * mm / (1 - (l - M) * t) ** 3 for l, mm in act)

    lo, hi = 1.0 / (f1 - M), 1.0 / (f2 - M)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if h1(mid) < 0:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    for _ in range(3):
        d = dh1(r)
        if d > 0:
            rn = r - h1(r) / d
            if 1.0 / (f1 - M) < rn < 1.0 / (f2 - M):
                r = rn
    s = sum(mm / (1 - (l - M) * r) ** 2 for l, mm in act)
    sig = np.zeros(P.C)
    for c in range(P.C):
        l = P.ls[c]
        if f1 <= l <= f2:
            sig[c] = 1.0 / (math.sqrt(s) * (1 - (l - M) * r))
    z = _scale_components(P, w, sig)
    return (z, r) if return_r else z


def psi_R2(P: Problem, w, return_r=False):
    """Lemma 5.3: the orthogonal retraction R2.

    r is the unique positive zero of h2(t) = sum_{l=0}^{2F} (l-F-M)||w_{l-F}||^2 t^l,
    found as the positive zero of h3 = h2 t^{-f1-F} (h3(0) < 0, increasing at its
    root) by bracketing, bisection and Newton polish.  Reading (R2 denominator):
    sigma_0^2 = 1 / sum_k ||w_k||^2 r^k as in the lemma's proof; the statement's
    ||w_l|| inside that sum is taken as a misprint.
    """
    M, F = P.M, P.F
    m = _component_norms2(P, w)
    f1, f2 = _f1_f2(P, m)
    if not (f1 < M < f2):
        raise FloatingPointError("w is outside Omega (needs f1(w) < M < f2(w))")
    # coefficients of h3 in powers t^j, j = 0..f2-f1, coefficient for l = j + f1
    coef = {}
    for c in range(P.C):
        l = P.ls[c]
        if f1 <= l <= f2:
            coef[int(round(l - f1))] = (l - M) * m[c]

    def h3(t):
        return sum(cf * t ** j for j, cf in coef.items())

    def dh3(t):
        return sum(j * cf * t ** (j - 1) for j, cf in coef.items() if j > 0)

    lo, hi = 0.0, 1.0
    while h3(hi) <= 0:
        lo, hi = hi, 2 * hi
        if hi > 1e300:
            raise FloatingPointError("no positive root of h2")
    for _ in range(2000):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if h3(mid) < 0:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    for _ in range(3):
        d = dh3(r)
        if d > 0:
            rn = r - h3(r) / d
            if rn > 0:
                r = rn
    ssum = sum(m[c] * r ** P.ls[c] for c in range(P.C))
    s0 = math.sqrt(1.0 / ssum)
    sig = np.array([s0 * r ** (P.ls[c] / 2.0) for c in range(P.C)])
    z = _scale_components(P, w, sig)
    return (z, r) if return_r else z


def psi_R3(P: Problem, w):
    """Lemma 5.4, Eq. (retract3): the closed-form retraction R3 (needs w in S)."""
    M = P.M
    Gm = gamma_weights(P)
    a = w @ w
    b = w @ (Gm * w)
    c = w @ (Gm * Gm * w)
    den = a * c - b * b
    sig = np.zeros(P.C)
    for i in range(P.C):
        l = P.ls[i]
        num = c - (M + l) * b + M * l * a
        if not (num > 0 and den > 0):
            raise FloatingPointError("w is outside S")
        sig[i] = math.sqrt(num / den)
    return _scale_components(P, w, sig)


PSI = {1: psi_R1, 2: psi_R2, 3: psi_R3}


def retract(P: Problem, u, xi, kind=1):
    """R_u(xi) = psi(u + xi), Eq. (oretr0)."""
    return PSI[kind](P, u + xi)


# ---------------------------------------------------------------------------
# Optimisers (Sec. 5, Algorithm 1)
# ---------------------------------------------------------------------------

@dataclass
class SolveOptions:
    retraction: int = 1
    tol: float = 1e-8               # finest-mesh stop on ||grad||_2
    tol_coarse: float = 1e-5        # coarse meshes (Sec. 7.1)
    rgbb_tol_in_arnt: float = 1e-2  # RGBB warm start inside ARNT (Sec. 7.1)
    rgbb_maxit_in_arnt: int = 2000
    maxit: int = 10000
    method: str = "arnt"            # "arnt" or "rgbb"
    # RGBB constants: rho, varrho, delta; first step gamma_0 (reading)
    rgbb_rho: float = 1e-4
    rgbb_varrho: float = 0.85
    rgbb_delta: float = 0.2
    rgbb_gamma0: float = 1e-3
    rgbb_max_backtracks: int = 10
    # ARNT constants (Sec. 7.1)
    eta1: float = 0.01
    eta2: float = 0.9
    gamma0: float = 0.2
    gamma1: float = 1.0
    gamma2: float = 10.0
    sigma_hat0: float = 1.0
    # curvilinear search (commented constants of Sec. 7.1): alpha0, delta, rho
    ls_alpha0: float = 1.0
    ls_delta: float = 0.2
    ls_rho: float = 1e-4
    ls_max_backtracks: int = 10
    # modified CG (reading): theta, T, negative-curvature threshold
    cg_theta: float = 1.0
    cg_T: float = 0.1
    cg_eps: float = 1e-12
    gamma_tilde: float = 0.0
    # rounding floor of E in units of eps |E|, and the stagnation cap on sigma_hat
    noise_factor: float = 100.0
    sigma_hat_max: float = 1e20


@dataclass
class SolveStats:
    energy: float = 0.0
    grad_norm: float = 0.0
    outer_iters: int = 0
    inner_iters: int = 0
    rgbb_iters: int = 0
    n_grad: int = 0
    n_energy: int = 0
    n_hvp: int = 0
    converged: bool = False
    history: list = field(default_factory=list)


def rgbb(P: Problem, u, opts: SolveOptions, tol, maxit, stats: SolveStats):
    """Riemannian gradient method with BB step and Zhang-Hager nonmonotone
    Armijo search (Sec. 5, Eq. NMN and the C_k, Q_k recursion).

    Readings: gamma_0 = opts.rgbb_gamma0 on the first step; the BB step is
    clamped to [1e-10, 1e10]; s and v are plain differences (no transport); at
    most opts.rgbb_max_backtracks reductions, after which the last trial is
    taken; a trial whose energy differs from the current one by no more than
    the rounding floor noise_factor * eps * max(1, |E|) passes the test (the
    floor the ARNT search uses).
    """
    kind = opts.retraction
    E = E_u(P, u)
    stats.n_energy += 1
    C, Q = E, 1.0
    u_prev = rg_prev = None
    for k in range(maxit + 1):
        g = egrad_u(P, u)
        stats.n_grad += 1
        rg = project(P, u, g)
        gn = float(np.linalg.norm(rg))
        stats.history.append(("rgbb", E, gn))
        if gn <= tol or k == maxit:
            return u, E, gn, k
        eta = -rg
        if u_prev is None:
            gam = opts.rgbb_gamma0
        else:
            s = u - u_prev
            v = rg - rg_prev
            vv = v @ v
            gam = abs(s @ v) / vv if vv > 0 else opts.rgbb_gamma0
            gam = min(max(gam, 1e-10), 1e10)
        slope = rg @ eta                                   # <grad, eta> = -||grad||^2
        t = gam
        noise = opts.noise_factor * np.finfo(float).eps * max(1.0, abs(E))
        for _ in range(opts.rgbb_max_backtracks + 1):
            z = retract(P, u, t * eta, kind)
            Ez = E_u(P, z)
            stats.n_energy += 1
            if Ez <= C + opts.rgbb_rho * t * slope or abs(Ez - E) <= noise:
                break
            t *= opts.rgbb_delta
        u_prev, rg_prev = u, rg
        u, E = z, Ez
        Qn = opts.rgbb_varrho * Q + 1.0
        C = (opts.rgbb_varrho * Q * C + E) / Qn
        Q = Qn
        stats.rgbb_iters += 1
    return u, E, gn, maxit


def modified_cg(P: Problem, u, g, rg, sigma, opts: SolveOptions, max_inner, stats: SolveStats):
    """Modified truncated CG on Hess m_k(u_k)[xi] = -grad m_k(u_k) (Eq. prob-lsub).

    Reading (the details live in the cited ARNT paper, not in this one):
    Steihaug-type CG from xi = 0 in T_u M; stop when ||r_j|| <=
    min(T, ||grad||^theta) ||grad||; the model is declared not positive along p
    when <p, Hp> <= eps ||p||^2: at j = 0 the output is s = -grad, d = 0,
    otherwise s = the current iterate, and d = p when the curvature is
    negative (<p, Hp> < -eps ||p||^2), else d = 0.  sigma_est = |<p,Hp>| / ||p||^2.
    Returns (s, d, Hd, sigma_est, iterations).
    """
    gn = float(np.linalg.norm(rg))
    stop = min(opts.cg_T, gn ** opts.cg_theta) * gn
    x = np.zeros_like(u)
    r = -rg.copy()
    p = r.copy()
    rr = r @ r
    if rr == 0.0:
        return x, None, None, None, 0
    for j in range(max_inner):
        Hp = rhess(P, u, p, g=g, sigma=sigma)
        stats.n_hvp += 1
        kap = p @ Hp
        pp = p @ p
        if kap <= opts.cg_eps * pp:
            sig_est = abs(kap) / pp
            if j == 0:
                return -rg.copy(), None, None, sig_est, j + 1
            if kap < -opts.cg_eps * pp:
                return x, p, Hp, sig_est, j + 1
            return x, None, None, sig_est, j + 1
        a = rr / kap
        x = x + a * p
        r = r - a * Hp
        rr_new = r @ r
        if math.sqrt(rr_new) <= stop:
            return x, None, None, None, j + 1
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, None, None, None, max_inner


def arnt(P: Problem, u, opts: SolveOptions, tol, maxit, stats: SolveStats):
    """ARNT part of Algorithm 1 with the curvilinear search (tp1)-(tp2), the ratio
    (ratio) and the sigma update of Sec. 7.1.

    Readings: sigma_k = sigma_hat_k ||grad||; sigma_hat <- gamma0 sigma_hat if
    rho_k >= eta2, unchanged if eta1 <= rho_k < eta2, gamma2 sigma_hat if the
    trial is rejected; after negative curvature sigma_{k+1} = max(sigma_{k+1},
    sigma_est + gamma_tilde).  m_k(z) is evaluated exactly with one Euclidean
    Hessian-vector product.  Inner CG cap: 100 while ||grad|| > 1e-3, else 300.
    """
    kind = opts.retraction
    E = E_u(P, u)
    stats.n_energy += 1
    sig_hat = opts.sigma_hat0
    sig_floor = 0.0
    g = egrad_u(P, u)
    stats.n_grad += 1
    rg = project(P, u, g)
    gn = float(np.linalg.norm(rg))
    k = 0
    for k in range(maxit + 1):
        stats.history.append(("arnt", E, gn))
        if gn <= tol or k == maxit:
            break
        sigma = max(sig_hat * gn, sig_floor)
        max_inner = 100 if gn > 1e-3 else 300
        s, d, Hd, sig_est, nin = modified_cg(P, u, g, rg, sigma, opts, max_inner, stats)
        stats.inner_iters += nin
        if d is not None:
            kd = d @ Hd
            tau = (d @ rg) / kd
            xi = s + tau * d
        else:
            xi = s
        slope = rg @ xi
        if not (slope < 0 and np.all(np.isfinite(xi))):
            xi = -rg
            slope = rg @ xi
        # Rounding floor of E and of m_k: below it neither the Armijo test nor
        # the ratio can be resolved, and the step is taken as it stands.
        noise = opts.noise_factor * np.finfo(float).eps * max(1.0, abs(E))
        t = opts.ls_alpha0
        for _ in range(opts.ls_max_backtracks + 1):
            z = retract(P, u, t * xi, kind)
            dz = z - u
            mz = g @ dz + 0.5 * dz @ ehess_u(P, u, dz) + 0.5 * sigma * dz @ dz
            stats.n_hvp += 1
            if mz <= opts.ls_rho * t * slope or abs(mz) <= noise:
                break
            t *= opts.ls_delta
        Ez = E_u(P, z)
        stats.n_energy += 1
        if abs(mz) <= noise and abs(Ez - E) <= noise:
            ratio = 1.0
        else:
            ratio = (Ez - E) / mz if mz < 0 else -1.0
        if ratio >= opts.eta1:
            u, E = z, Ez
            g = egrad_u(P, u)
            stats.n_grad += 1
            rg = project(P, u, g)
            gn = float(np.linalg.norm(rg))
            if ratio >= opts.eta2:
                sig_hat *= opts.gamma0
            else:
                sig_hat *= opts.gamma1
        else:
            sig_hat *= opts.gamma2
        sig_floor = (sig_est + opts.gamma_tilde) if sig_est is not None else 0.0
        stats.outer_iters += 1
        if sig_hat > opts.sigma_hat_max:
            break                                        # stagnation: report as not converged
    return u, E, gn, k


def solve_level(P: Problem, u, opts: SolveOptions, tol, stats: SolveStats):
    if opts.method == "rgbb":
        u, E, gn, _ = rgbb(P, u, opts, tol, opts.maxit, stats)
    else:
        u, E, gn, _ = rgbb(P, u, opts, max(tol, opts.rgbb_tol_in_arnt),
                           opts.rgbb_maxit_in_arnt, stats)
        if gn > tol:
            u, E, gn, _ = arnt(P, u, opts, tol, opts.maxit, stats)
    stats.energy, stats.grad_norm = E, gn
    stats.converged = gn <= tol
    return u


def prolongate(Pc: Problem, Pf: Problem, Xc):
    """Cascadic prolongation (Algorithm 1, 'refine uniformly').

    Reading: same domain, finer n; the trigonometric interpolant of each
    component is sampled on the finer grid by zero-padding the DFT (the
    coarse Nyquist coefficient is split evenly between +-n/2), X is rescaled
    by sqrt(dV_f / dV_c) * (G_f / G_c), and the result is put back on M with
    the projective retraction R1.
    """
    axes = tuple(range(Pc.d))
    Xf = np.empty((Pf.G, Pc.C), dtype=complex)
    for c in range(Pc.C):
        hat = sfft.fftn(Xc[:, c].reshape(Pc.shape), axes=axes)
        for ax in range(Pc.d):
            nc = hat.shape[ax]
            nf = Pf.shape[ax]
            if nf == nc:
                continue
            sh = list(hat.shape)
            sh[ax] = nf
            out = np.zeros(sh, dtype=complex)
            idx_c = [slice(None)] * Pc.d
            idx_f = [slice(None)] * Pc.d
            half = nc // 2
            # nonnegative frequencies 0..half-1
            idx_c[ax] = slice(0, half)
            idx_f[ax] = slice(0, half)
            out[tuple(idx_f)] = hat[tuple(idx_c)]
            # negative frequencies -half+1..-1
            idx_c[ax] = slice(nc - half + 1, nc)
            idx_f[ax] = slice(nf - half + 1, nf)
            out[tuple(idx_f)] = hat[tuple(idx_c)]
            # Nyquist -half split to +half and -half
            idx_c[ax] = slice(half, half + 1)
            nyq = hat[tuple(idx_c)]
            idx_f[ax] = slice(half, half + 1)
            out[tuple(idx_f)] = 0.5 * nyq
            idx_f[ax] = slice(nf - half, nf - half + 1)
            out[tuple(idx_f)] = 0.5 * nyq
            hat = out
        phi = sfft.ifftn(hat, axes=axes) * (Pf.G / Pc.G)
        Xf[:, c] = phi.reshape(Pf.G)
    Xf *= math.sqrt(Pf.dV / Pc.dV)
    uf = psi_R1(Pf, to_u(Pf, Xf))
    return from_u(Pf, uf)


def solve(problems, X0, opts: SolveOptions | None = None):
    """Cascadic driver of Algorithm 1 over a list of problems coarse -> fine.

    X0 is the initial matrix on the coarsest problem; it is put on M with R1.
    Returns (X on the finest mesh, SolveStats of the finest level, all stats).
    """
    if opts is None:
        opts = SolveOptions()
    if isinstance(problems, Problem):
        problems = [problems]
    u = psi_R1(problems[0], to_u(problems[0], X0))
    all_stats = []
    for j, P in enumerate(problems):
        if j > 0:
            u = to_u(P, prolongate(problems[j - 1], P, from_u(problems[j - 1], u)))
        st = SolveStats()
        tol = opts.tol if j == len(problems) - 1 else opts.tol_coarse
        u = solve_level(P, u, opts, tol, st)
        all_stats.append(st)
    return from_u(problems[-1], u), all_stats[-1], all_stats
