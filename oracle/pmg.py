"""Geometric p-multigrid (paper Sec. 4): coarsening, spectral transfers,
block smoothers, the V-cycle (Algorithm 1), FMG (Algorithm 2) and the dense
coarsest-level solve.

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper:

* Coarsening (Sec. 4.1): the printed case condition is contradictory.  Going
  from fine to coarse: if Nx > Nz halve Nx (and Ny); if Nz > Nx set
  Nz <- max(2, ceil(Nz/2)); if equal do both.  Stop when the next level would
  have Nx < 4 or Nz < 2, or as soon as a level has at most ``coarsest_max``
  unknowns.  Coarse operators are rediscretised with Fourier-truncated h and
  eta.
* Transfers (Sec. 4.2): restriction = Fourier truncation (coarse Nyquist
  dropped) then Chebyshev truncation; prolongation = Chebyshev interpolation
  then Fourier zero-padding.  ``bc_transfer="paper"`` transfers the whole
  column, boundary-row residuals included, through the Chebyshev truncation
  (the paper's "same course of action").  ``bc_transfer="inject"`` (default)
  restricts the surface and bottom rows by Fourier truncation only and
  injects them into the coarse surface and bottom rows: the boundary-row
  residuals are residuals of different equations, and mixing them into the
  interior polynomial makes the V-cycle amplify the smooth, x-constant error
  mode by about 1.6 per cycle with the block-Jacobi smoother.
* Smoother (Sec. 4.3): one block per vertical column with the diagonal
  (Nz+1)^2 block of the operator.  ``block_gauss_seidel`` is the paper's
  forward sweep over columns; ``block_jacobi`` is the damped simultaneous
  variant the GPU runs.  Neither the damping nor the sweep counts are given
  by the paper (defaults omega = 0.4, nu1 = nu2 = 2).
* Nyquist split (``nyquist_split=True``, default): on the even Fourier grid
  the composite second derivative D_x(D_x .) annihilates the x-Nyquist mode
  (-1)^j, but the column block carries the mean x-diagonal
  -(1/Nx) sum kappa^2, so plain block-Jacobi leaves that mode unsmoothed and
  the Fourier truncation cannot correct it.  The residual's Nyquist part
  r_N = P_N r (P_N: projection on (-1)^j along x, and along y in 3D) is
  therefore solved with the column block whose x- (y-) diagonal term is
  zero, the rest with the ordinary block, both damped by omega.
"""

import math

import numpy as np

from . import spectral as sp
from .operator import Grid, Geometry, apply_A, assemble_A, column_blocks


def coarsen(Nx, Ny, Nz):
    """One coarsening step of the combined standard/semi strategy (Sec. 4.1)."""
    if Nx > Nz:
        return Nx // 2, (Ny // 2 if Ny > 1 else 1), Nz
    if Nz > Nx:
        return Nx, Ny, max(2, math.ceil(Nz / 2))
    return Nx // 2, (Ny // 2 if Ny > 1 else 1), max(2, math.ceil(Nz / 2))


def hierarchy(Nx, Ny, Nz, coarsest_max=256):
    """Level sizes (Sec. 4.1 coarsening), finest first, ending at the coarsest
    (direct-solve) level."""
    levels = [(Nx, Ny, Nz)]
    while True:
        nx, ny, nz = levels[-1]
        if nx * ny * (nz + 1) <= coarsest_max:
            break
        cx, cy, cz = coarsen(nx, ny, nz)
        if cx < 4 or cz < 2 or (Ny > 1 and cy < 4) or (cx, cy, cz) == (nx, ny, nz):
            break
        levels.append((cx, cy, cz))
    return levels


def restrict_surface(f, Nx_c, Ny_c):
    """Fourier truncation (Sec. 4.2) of a surface array (Ny, Nx) to (Ny_c, Nx_c)."""
    g = sp.fourier_resample(f, Nx_c, axis=1)
    if g.shape[0] > 1:
        g = sp.fourier_resample(g, Ny_c, axis=0)
    return g


class Level:
    """One grid of the hierarchy (Sec. 4.1) with its rediscretised operator A_{a,b}."""

    def __init__(self, Nx, Ny, Nz, L, h, eta_a, eta_b):
        self.grid = Grid(Nx, Ny, Nz, L)
        h = restrict_surface(h, Nx, Ny)              # fine (Ny_f, Nx_f) -> this level
        ea = restrict_surface(eta_a, Nx, Ny)
        eb = restrict_surface(eta_b, Nx, Ny)
        self.geo_a = Geometry(self.grid, h, ea)
        self.geo_b = Geometry(self.grid, h, eb)
        self._blocks = None
        self._dense = None

    def apply(self, p):
        return apply_A(self.grid, self.geo_a, self.geo_b, p)

    @property
    def blocks(self):
        if self._blocks is None:
            self._blocks = column_blocks(self.grid, self.geo_a, self.geo_b)
        return self._blocks

    @property
    def dense(self):
        if self._dense is None:
            self._dense = assemble_A(self.grid, self.geo_a, self.geo_b)
        return self._dense


def build_levels(Nx, Ny, Nz, L, h, eta_a, eta_b, coarsest_max=256):
    h = np.asarray(h, dtype=np.float64).reshape(Ny, Nx)
    eta_a = np.asarray(eta_a, dtype=np.float64).reshape(Ny, Nx)
    eta_b = np.asarray(eta_b, dtype=np.float64).reshape(Ny, Nx)
    return [Level(nx, ny, nz, L, h, eta_a, eta_b)
            for (nx, ny, nz) in hierarchy(Nx, Ny, Nz, coarsest_max)]


def restrict_sigma_matrix(Nz_f, Nz_c, bc_transfer="inject"):
    """Chebyshev part of the restriction, shape (Nz_c+1, Nz_f+1).

    "paper": plain truncation of the whole column; "inject": the same for the
    interior coarse rows, the surface and bottom rows copied unchanged."""
    R = sp.cheb_restrict_matrix(Nz_f, Nz_c)
    if bc_transfer == "inject":
        R = R.copy()
        R[0, :] = 0.0
        R[0, 0] = 1.0
        R[-1, :] = 0.0
        R[-1, -1] = 1.0
    return R


def restrict(fine, coarse, r, bc_transfer="inject"):
    """R (Sec. 4.2, Algorithm 1): fine residual -> coarse grid (Fourier
    truncation, then Chebyshev)."""
    g = sp.fourier_resample(r, coarse.Nx, axis=2)
    if fine.Ny > 1:
        g = sp.fourier_resample(g, coarse.Ny, axis=1)
    R = restrict_sigma_matrix(fine.Nz, coarse.Nz, bc_transfer)
    return np.tensordot(R, g, axes=(1, 0))


def prolong(coarse, fine, e):
    """P (Sec. 4.2, Algorithm 1): coarse correction -> fine grid (Chebyshev
    interpolation, then Fourier zero-pad)."""
    P = sp.cheb_prolong_matrix(coarse.Nz, fine.Nz)
    g = np.tensordot(P, e, axes=(1, 0))
    if fine.Ny > 1:
        g = sp.fourier_resample(g, fine.Ny, axis=1)
    return sp.fourier_resample(g, fine.Nx, axis=2)


def nyquist_parts(grid, r):
    """Split r into parts by x- and y-Nyquist content (for the Sec. 4.3 block
    smoother with the Nyquist reading): {(ix, iy): r_part}, where
    ix = 1 marks the projection on (-1)^jx along x (likewise iy along y)."""
    def proj(f, axis):
        N = f.shape[axis]
        shape = [1] * f.ndim
        shape[axis] = N
        s = ((-1.0) ** np.arange(N)).reshape(shape)
        return (f * s).mean(axis=axis, keepdims=True) * s
    parts = {}
    px = proj(r, 2)
    if grid.Ny > 1:
        pxy = proj(px, 1)
        py = proj(r, 1)
        parts[(1, 1)] = pxy
        parts[(1, 0)] = px - pxy
        parts[(0, 1)] = py - pxy
        parts[(0, 0)] = r - px - py + pxy
    else:
        parts[(1, 0)] = px
        parts[(0, 0)] = r - px
    return parts


def nyquist_blocks(level, ix, iy):
    """Column blocks (Sec. 4.3) with the x- (ix=1) and/or y- (iy=1) diagonal
    term removed."""
    g = level.grid
    def diag2(N):
        if N == 1:
            return 0.0
        k2 = sp.fourier_wavenumbers(N, g.L) ** 2
        k2[N // 2] = 0.0
        return -np.sum(k2) / N
    J = np.eye(g.M1)
    J[0, 0] = J[-1, -1] = 0.0
    c = (diag2(g.Nx) if ix else 0.0) + (diag2(g.Ny) if iy else 0.0)
    return level.blocks - c * J


def block_jacobi(level, x, f, omega, nyquist_split=True):
    """One damped block-Jacobi sweep (Sec. 4.3 block relaxation, Jacobi form):
    x <- x + omega A_rr^{-1} (f - A x)_r for all r
    (with ``nyquist_split`` the Nyquist parts use their own column blocks)."""
    r = f - level.apply(x)
    parts = nyquist_parts(level.grid, r) if nyquist_split else {(0, 0): r}
    dx = np.zeros_like(x)
    for (ix, iy), rp in parts.items():
        B = level.blocks if (ix, iy) == (0, 0) else nyquist_blocks(level, ix, iy)
        rc = np.moveaxis(rp, 0, -1)[..., None]         # (Ny, Nx, M1, 1)
        dx += np.moveaxis(np.linalg.solve(B, rc)[..., 0], -1, 0)
    return x + omega * dx


def block_gauss_seidel(level, x, f):
    """One forward block Gauss-Seidel sweep over the columns (Sec. 4.3).

    x_r <- A_rr^{-1} (f_r - sum_{s != r} A_rs x_s), columns taken in order,
    newest values used.  Uses the dense matrix: small levels only.
    """
    g = level.grid
    A = level.dense
    x = x.copy().reshape(g.shape)
    idx = np.arange(g.n).reshape(g.shape)
    for jy in range(g.Ny):
        for jx in range(g.Nx):
            rows = idx[:, jy, jx]
            xf = x.ravel()
            res = f.reshape(-1)[rows] - A[rows] @ xf + A[np.ix_(rows, rows)] @ xf[rows]
            x[:, jy, jx] = np.linalg.solve(A[np.ix_(rows, rows)], res)
    return x


def reference_column_matrix(grid, kappa2, dref):
    """Column matrix of the flat reference operator for one horizontal
    Fourier mode: the operator with eta = 0 and h = dref (so sigma_x =
    sigma_y = 0, sigma_z = 1/dref) acting on p(sigma) exp(i kappa . x):
    interior rows D D / dref^2 - kappa^2 I, surface row e_0 (Eq. bcpd),
    bottom row D[Nz, :] / dref (Eq. bcpdneu with n = (0, 0, 1)).  kappa^2
    is the discrete second-derivative symbol: the Nyquist mode, which the
    composite D_x(D_x .) annihilates, has kappa^2 = 0 along that axis."""
    D = grid.Ds
    A = (D @ D) / dref ** 2 - kappa2 * np.eye(grid.M1)
    A[0, :] = 0.0
    A[0, 0] = 1.0
    A[-1, :] = D[-1, :] / dref
    return A


def reference_kappa2(grid):
    """kappa_x^2 + kappa_y^2 (Sec. 3.4 wavenumbers) of every (y, x) Fourier mode,
    numpy FFT order,
    with the Nyquist wavenumber of each axis counted as 0."""
    def k2(N):
        if N == 1:
            return np.zeros(1)
        k = sp.fourier_wavenumbers(N, grid.L)
        k2 = k ** 2
        k2[N // 2] = 0.0
        return k2
    return k2(grid.Ny)[:, None] + k2(grid.Nx)[None, :]


def spectral_smooth(level, x, f, omega_s, dref, transpose=False):
    """One sweep of the mean-depth spectral smoother (the stronger smoother
    row of the build's plan; the paper's Sec. 4.3 leaves the smoother open
    beyond block relaxation): x <- x + omega_s S (f - A x), where S solves
    the flat reference problem of depth dref exactly, mode by mode: the
    residual is Fourier transformed along x (and y), each mode's column is
    solved with ``reference_column_matrix``, and the result transformed
    back.  ``transpose`` uses the transposed column matrices (the smoother
    of A^T; the modal transform is symmetric)."""
    g = level.grid
    r = f - (level.apply(x) if not transpose else level.dense.T @ x.ravel()).reshape(g.shape)
    R = np.fft.fft(r, axis=2)
    if g.Ny > 1:
        R = np.fft.fft(R, axis=1)
    K2 = reference_kappa2(g)
    out = np.zeros_like(R)
    for iy in range(g.Ny):
        for ix in range(g.Nx):
            A = reference_column_matrix(g, K2[iy, ix], dref)
            out[:, iy, ix] = np.linalg.solve(A.T if transpose else A, R[:, iy, ix])
    if g.Ny > 1:
        out = np.fft.ifft(out, axis=1)
    out = np.real(np.fft.ifft(out, axis=2))
    return x + omega_s * out


def smooth(level, x, f, sweeps, smoother, omega, omega_s=1.0, dref=None):
    """``sweeps`` sweeps of the chosen smoother (Sec. 4.3): "jacobi" (damped block-Jacobi
    with the Nyquist split), "jacobi-plain", "gs" (forward block
    Gauss-Seidel), "spectral" (mean-depth spectral smoother of depth dref),
    "jacobi+spectral" (a block-Jacobi sweep then a spectral sweep)."""
    for _ in range(sweeps):
        if smoother == "gs":
            x = block_gauss_seidel(level, x, f)
        elif smoother == "jacobi-plain":
            x = block_jacobi(level, x, f, omega, nyquist_split=False)
        elif smoother == "spectral":
            x = spectral_smooth(level, x, f, omega_s, dref)
        elif smoother == "jacobi+spectral":
            x = block_jacobi(level, x, f, omega)
            x = spectral_smooth(level, x, f, omega_s, dref)
        else:
            x = block_jacobi(level, x, f, omega)
    return x


def coarse_solve(level, f):
    """Direct solve u = A^{-1} f on the coarsest grid (Algorithm 1)."""
    return np.linalg.solve(level.dense, f.ravel()).reshape(level.grid.shape)


def vcycle(levels, l, x, f, nu1=2, nu2=2, smoother="jacobi", omega=0.4,
           bc_transfer="inject", omega_s=1.0, dref=None):
    """Recursive V-cycle (Algorithm 1), level index l = 0 is the finest.
    smoother: one kind for every level, or a list of kinds by level index
    (Algorithm 1 leaves the smoother of each level open)."""
    lev = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(lev, f)
    kind = smoother[l] if isinstance(smoother, (list, tuple)) else smoother
    x = smooth(lev, x, f, nu1, kind, omega, omega_s, dref)
    r = f - lev.apply(x)
    rc = restrict(lev.grid, levels[l + 1].grid, r, bc_transfer)
    ec = vcycle(levels, l + 1, np.zeros_like(rc), rc, nu1, nu2, smoother, omega, bc_transfer,
                omega_s, dref)
    x = x + prolong(levels[l + 1].grid, lev.grid, ec)
    x = smooth(lev, x, f, nu2, kind, omega, omega_s, dref)
    return x


def fmg(levels, f, nu1=2, nu2=2, smoother="jacobi", omega=0.4, bc_transfer="inject", omega_s=1.0,
        dref=None):
    """Full multigrid (Algorithm 2): V-cycles from the coarsest grid upwards,
    prolongating each result as the next level's initial state."""
    fs = [f]
    for l in range(len(levels) - 1):
        fs.append(restrict(levels[l].grid, levels[l + 1].grid, fs[-1], bc_transfer))
    P = len(levels)
    u = np.zeros_like(fs[-1])
    for l in range(P - 1, 0, -1):
        u = vcycle(levels, l, u, fs[l], nu1, nu2, smoother, omega, bc_transfer, omega_s, dref)
        u = prolong(levels[l].grid, levels[l - 1].grid, u)
    return vcycle(levels, 0, u, fs[0], nu1, nu2, smoother, omega, bc_transfer, omega_s, dref)
