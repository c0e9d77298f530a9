"""Seeded generators for block tridiagonal systems ``tridiag(A_i, D_i, C_i)``.

Notation (Section 3, the block tridiagonal form of the 2D operator): block row
``i`` of the matrix holds ``A_i`` (sub-diagonal, couples to block ``i-1``),
``D_i`` (diagonal) and ``C_i`` (super-diagonal, couples to block ``i+1``).  The
paper writes these ``E_i, D_i, F_i``.  ``A_0`` and ``C_{n-1}`` do not exist and
are stored as zeros.

The 2D problems use an ``n x n`` interior grid of the unit square with
homogeneous Dirichlet conditions, ``h = 1/(n+1)``.  Unknown ``(p, q)`` (``p``
along x, ``q`` along y) is row ``p`` of block ``q``: a block is one grid line,
so ``D_i`` is tridiagonal (the x-couplings) and ``A_i``, ``C_i`` are diagonal
(the y-couplings), which is the exact structure stated in Section 3.  Every
operator is multiplied by ``h^2``.

Two storage forms are produced:

* *banded* (compact): ``Dl, Dd, Du`` -- sub-, main and super-diagonal of each
  ``D_i`` (``Dl[i, 0]`` and ``Du[i, b-1]`` are zero), and ``a, c`` -- the
  diagonals of ``A_i`` and ``C_i``.  Arrays are ``(nblk, b)`` float64.
* *dense*: ``A, D, C`` of shape ``(nblk, b, b)``; ``X[i]`` is block ``i`` as an
  ordinary (row, col) matrix.  ``dense_colmajor()`` gives the C-ABI layout
  (each block column-major, blocks contiguous).

Nothing in this module performs cyclic reduction or any other solver step.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class BlockTridiag:
    """Banded block tridiagonal system with ``nblk`` blocks of size ``b``."""

    nblk: int
    b: int
    Dl: np.ndarray  # (nblk, b)  D_i[r, r-1]
    Dd: np.ndarray  # (nblk, b)  D_i[r, r]
    Du: np.ndarray  # (nblk, b)  D_i[r, r+1]
    a: np.ndarray   # (nblk, b)  diag(A_i); a[0] == 0
    c: np.ndarray   # (nblk, b)  diag(C_i); c[-1] == 0
    name: str = ""

    @property
    def N(self) -> int:
        return self.nblk * self.b

    # ---- dense views -------------------------------------------------
    def dense_blocks(self):
        """Return ``(A, D, C)`` as ``(nblk, b, b)`` float64 row/col matrices."""
        n, b = self.nblk, self.b
        A = np.zeros((n, b, b))
        D = np.zeros((n, b, b))
        C = np.zeros((n, b, b))
        r = np.arange(b)
        D[:, r, r] = self.Dd
        D[:, r[1:], r[1:] - 1] = self.Dl[:, 1:]
        D[:, r[:-1], r[:-1] + 1] = self.Du[:, :-1]
        A[:, r, r] = self.a
        C[:, r, r] = self.c
        return A, D, C

    def dense_colmajor(self):
        """Blocks in the C-ABI layout: each block column-major, blocks contiguous.

        Returns three C-contiguous float64 arrays of shape ``(nblk, b, b)`` whose
        memory order is block-major then column-major (``arr[i, col, row]``).
        """
        A, D, C = self.dense_blocks()
        t = lambda X: np.ascontiguousarray(np.transpose(X, (0, 2, 1)))
        return t(A), t(D), t(C)

    def banded_abi(self):
        """Compact C-ABI layout: ``D`` as ``(nblk, 3, b)`` = [sub, main, super]
        per block, ``A`` and ``C`` as ``(nblk, b)`` diagonals."""
        D3 = np.ascontiguousarray(np.stack([self.Dl, self.Dd, self.Du], axis=1))
        return (np.ascontiguousarray(self.a), D3, np.ascontiguousarray(self.c))

    def assemble(self) -> np.ndarray:
        """The full ``N x N`` matrix (small sizes only)."""
        n, b = self.nblk, self.b
        A, D, C = self.dense_blocks()
        M = np.zeros((n * b, n * b))
        for i in range(n):
            s = slice(i * b, (i + 1) * b)
            M[s, s] = D[i]
            if i > 0:
                M[s, (i - 1) * b:i * b] = A[i]
            if i < n - 1:
                M[s, (i + 1) * b:(i + 2) * b] = C[i]
        return M

    def matvec(self, X: np.ndarray) -> np.ndarray:
        """``Y = M X`` for ``X`` of shape ``(N,)`` or ``(N, k)`` (banded form)."""
        n, b = self.nblk, self.b
        X2 = X.reshape(n, b, -1)
        Y = self.Dd[:, :, None] * X2
        Y[:, 1:] += self.Dl[:, 1:, None] * X2[:, :-1]
        Y[:, :-1] += self.Du[:, :-1, None] * X2[:, 1:]
        Y[1:] += self.a[1:, :, None] * X2[:-1]
        Y[:-1] += self.c[:-1, :, None] * X2[1:]
        return Y.reshape(X.shape)


# ---------------------------------------------------------------------------
# Gaussian random field
# ---------------------------------------------------------------------------

def gaussian_random_field(npts: int, seed: int, corr_len: float = 0.1) -> np.ndarray:
    """Smooth seeded field on an ``npts x npts`` node grid of the unit square.

    White noise is convolved (periodically, by FFT) with the kernel
    ``exp(-|x|^2 / corr_len^2)``, which gives the covariance
    ``exp(-|x|^2 / (2 corr_len^2))``; the result is shifted and scaled to zero
    mean and unit variance.  Returned as ``g[q, p]`` (y index first).
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((npts, npts))
    h = 1.0 / max(npts - 1, 1)
    k = np.fft.fftfreq(npts, d=h)  # cycles per unit length
    kx, ky = np.meshgrid(k, k, indexing="xy")
    # Fourier transform of exp(-|x|^2/L^2) is proportional to exp(-pi^2 L^2 |k|^2)
    filt = np.exp(-(math.pi ** 2) * corr_len ** 2 * (kx ** 2 + ky ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g /= sd
    return g


# ---------------------------------------------------------------------------
# Operators (all multiplied by h^2)
# ---------------------------------------------------------------------------

def _empty(n: int):
    z = lambda: np.zeros((n, n))
    return z(), z(), z(), z(), z()


def poisson(n: int) -> BlockTridiag:
    """Constant-coefficient 5-point Laplacian: ``D_i = tridiag(-1, 4, -1)``,
    ``A_i = C_i = -I`` (Section 3, Eq. for the block tridiagonal form)."""
    Dl, Dd, Du, a, c = _empty(n)
    Dd[:] = 4.0
    Dl[:, 1:] = -1.0
    Du[:, :-1] = -1.0
    a[1:] = -1.0
    c[:-1] = -1.0
    return BlockTridiag(n, n, Dl, Dd, Du, a, c, name=f"poisson{n}")


def variable_diffusion(n: int, seed: int, contrast: float = 1e4,
                       corr_len: float = 0.1) -> BlockTridiag:
    """``-div(a grad u) = f``, 5-point finite volume (Section 3's variable
    coefficient Poisson problem).

    Cell coefficient ``a = exp(sigma * g)`` with ``g`` a seeded Gaussian random
    field on the ``(n+2)^2`` node grid and ``sigma`` chosen so that
    ``max a / min a == contrast`` over that grid.  Interior faces take the
    harmonic mean of their two cells, boundary faces the cell's own value.
    Diagonal = sum of the four face coefficients, neighbours = -face.
    """
    g = gaussian_random_field(n + 2, seed, corr_len)
    sigma = math.log(contrast) / (g.max() - g.min())
    kap = np.exp(sigma * (g - g.min()))
    cell = kap[1:-1, 1:-1]  # [q, p]

    def hm(x, y):
        return 2.0 * x * y / (x + y)

    # faces in x (between p and p+1) and y (between q and q+1)
    fw = np.empty((n, n)); fe = np.empty((n, n)); fs = np.empty((n, n)); fn = np.empty((n, n))
    fw[:, 0] = cell[:, 0]
    fw[:, 1:] = hm(cell[:, 1:], cell[:, :-1])
    fe[:, -1] = cell[:, -1]
    fe[:, :-1] = hm(cell[:, :-1], cell[:, 1:])
    fs[0, :] = cell[0, :]
    fs[1:, :] = hm(cell[1:, :], cell[:-1, :])
    fn[-1, :] = cell[-1, :]
    fn[:-1, :] = hm(cell[:-1, :], cell[1:, :])

    Dl, Dd, Du, a, c = _empty(n)
    Dd[:] = fw + fe + fs + fn
    Dl[:, 1:] = -fw[:, 1:]
    Du[:, :-1] = -fe[:, :-1]
    a[1:] = -fs[1:]
    c[:-1] = -fn[:-1]
    return BlockTridiag(n, n, Dl, Dd, Du, a, c, name=f"diffusion{n}")


def convection_diffusion(n: int, seed: int, beta_mag: float = 1e3,
                         corr_len: float = 0.1) -> BlockTridiag:
    """``-Lap u + beta . grad u = f`` with first-order upwinding (Section 4's
    nonsymmetric test, here with a seeded recirculating field).

    ``beta = beta_mag (cos theta, sin theta)``, ``theta = pi * g`` with ``g`` a
    seeded Gaussian random field at the interior nodes.  Row coefficients
    (times ``h^2``): west ``-1 - h max(bx,0)``, east ``-1 + h min(bx,0)``,
    south ``-1 - h max(by,0)``, north ``-1 + h min(by,0)``, diagonal
    ``4 + h(|bx| + |by|)``.
    """
    h = 1.0 / (n + 1)
    g = gaussian_random_field(n + 2, seed, corr_len)[1:-1, 1:-1]
    theta = math.pi * g
    bx = beta_mag * np.cos(theta)
    by = beta_mag * np.sin(theta)
    Dl, Dd, Du, a, c = _empty(n)
    Dd[:] = 4.0 + h * (np.abs(bx) + np.abs(by))
    Dl[:, 1:] = (-1.0 - h * np.maximum(bx, 0.0))[:, 1:]
    Du[:, :-1] = (-1.0 + h * np.minimum(bx, 0.0))[:, :-1]
    a[1:] = (-1.0 - h * np.maximum(by, 0.0))[1:]
    c[:-1] = (-1.0 + h * np.minimum(by, 0.0))[:-1]
    return BlockTridiag(n, n, Dl, Dd, Du, a, c, name=f"convdiff{n}")


def helmholtz(n: int, seed: int, ppw: float = 16.0, variation: float = 0.2,
              corr_len: float = 0.1) -> BlockTridiag:
    """``-Lap u - kappa(x,y)^2 u = f`` (Section 4's Helmholtz test), 5-point.

    ``kappa = kappa0 (1 + variation * clip(g/3, -1, 1))`` with
    ``kappa0 = 2 pi / (ppw h)`` (``ppw`` points per wavelength) and ``g`` a
    seeded Gaussian random field at the interior nodes.  The matrix is real,
    symmetric and indefinite.
    """
    h = 1.0 / (n + 1)
    g = gaussian_random_field(n + 2, seed, corr_len)[1:-1, 1:-1]
    kappa0 = 2.0 * math.pi / (ppw * h)
    kappa = kappa0 * (1.0 + variation * np.clip(g / 3.0, -1.0, 1.0))
    Dl, Dd, Du, a, c = _empty(n)
    Dd[:] = 4.0 - (kappa * h) ** 2
    Dl[:, 1:] = -1.0
    Du[:, :-1] = -1.0
    a[1:] = -1.0
    c[:-1] = -1.0
    return BlockTridiag(n, n, Dl, Dd, Du, a, c, name=f"helmholtz{n}")


def random_blocks(nblk: int, b: int, seed: int, dominance: float = 2.0,
                  symmetric: bool = False):
    """Dense random block tridiagonal system (not a PDE): every block full.

    Returns ``(A, D, C)`` as ``(nblk, b, b)`` row/col matrices.  Entries are
    uniform[-1, 1]; ``D_i`` gets ``dominance * b`` added to its diagonal so the
    matrix is block diagonally dominant (and every reduced block invertible).
    """
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (nblk, b, b))
    D = rng.uniform(-1, 1, (nblk, b, b))
    C = rng.uniform(-1, 1, (nblk, b, b))
    if symmetric:
        D = 0.5 * (D + np.transpose(D, (0, 2, 1)))
        C[:-1] = np.transpose(A[1:], (0, 2, 1))
    D += dominance * b * np.eye(b)[None]
    A[0] = 0.0
    C[-1] = 0.0
    return A, D, C


def strip_kernel_blocks(nblk: int, b: int, width: int = 3, alpha: float = 1.0,
                        beta: float = 0.3, seed: int = 0):
    """Dense block tridiagonal system with mid-rank off-diagonal structure.

    ``D_i = alpha_i I + K`` with ``K[r, s] = 1 / (1 + |p_r - p_s|)`` over ``b``
    points ``p_r`` of a ``width``-wide strip of the integer lattice (point ``r``
    at ``(r mod width, r div width)``), and ``A_i = C_i = -beta I``.  ``K`` is
    symmetric positive definite (``1/(1+t)`` is a positive mixture of
    ``exp(-s t)``), so with ``beta < alpha / 2`` the whole matrix is symmetric
    positive definite.  ``alpha_i`` is ``alpha`` scaled by a seeded factor in
    ``[1, 1.1]``.  For ``width = 3``, the off-diagonal nodes of ``D_i^-1``
    and of the reduced blocks have numerical ranks between 13 and 28 at a
    relative threshold of 1e-6, at every tree level of a 1024-block.  Returns
    ``(A, D, C)`` as ``(nblk, b, b)`` row/col matrices.
    """
    rng = np.random.default_rng(seed)
    r = np.arange(b)
    px, py = r % width, r // width
    dist = np.hypot(px[:, None] - px[None, :], py[:, None] - py[None, :])
    K = 1.0 / (1.0 + dist)
    D = np.repeat(K[None], nblk, axis=0)
    D += (alpha * rng.uniform(1.0, 1.1, nblk))[:, None, None] * np.eye(b)[None]
    A = np.repeat((-beta * np.eye(b))[None], nblk, axis=0)
    C = A.copy()
    A[0] = 0.0
    C[-1] = 0.0
    return A, D, C


def rhs_uniform(N: int, nrhs: int, seed: int) -> np.ndarray:
    """Seeded uniform[-1, 1] right-hand sides, ``(N, nrhs)`` Fortran order."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, (N, nrhs)))


# ---------------------------------------------------------------------------
# The five workloads (sizes, tolerances, RHS counts)
# ---------------------------------------------------------------------------

CONFIGS = {
    0: dict(name="poisson64", n=64, leaf=16, tol=1e-10, nrhs=1),
    1: dict(name="diffusion256", n=256, leaf=32, tol=1e-6, nrhs=16),
    2: dict(name="convdiff512", n=512, leaf=64, tol=1e-6, nrhs=64),
    3: dict(name="helmholtz1024", n=1024, leaf=64, tol=1e-8, nrhs=8),
}


def make_config(idx: int, n: int | None = None) -> BlockTridiag:
    """Build workload ``idx`` (0..3), optionally at another grid size ``n``.

    Field seeds are ``1000 + idx``; RHS seeds (see ``rhs_uniform``) are
    ``2000 + idx``.
    """
    cfg = CONFIGS[idx]
    n = cfg["n"] if n is None else n
    if idx == 0:
        return poisson(n)
    if idx == 1:
        return variable_diffusion(n, seed=1000 + idx)
    if idx == 2:
        return convection_diffusion(n, seed=1000 + idx)
    if idx == 3:
        return helmholtz(n, seed=1000 + idx)
    raise ValueError(idx)
