"""sigma-transform metric, transformed gradient / divergence and the
mixed-stage Poisson operator with its boundary rows.

Test infrastructure only (see ``oracle/__init__.py``).

Fields are float64 arrays of shape (Nz+1, Ny, Nx); index 0 of the first axis
is the free surface (sigma = 1), index Nz the bottom (sigma = 0).  A 2D tank
has Ny = 1 (every y-derivative is then zero).  The domain is [0, L) x [0, L).

Definitions followed:

* sigma = (z + h) / d, d = h + eta                          (Eq. sigtrans)
* sigma_x = (h_x - sigma d_x) / d, sigma_y likewise, sigma_z = 1/d
                                                            (Eq. 1_Scoef)
* Grad f = (f_chi + sigma_x f_sigma, f_gamma + sigma_y f_sigma, sigma_z f_sigma)
  Div G  = dG_x/dchi + sigma_x dG_x/dsigma + dG_y/dgamma + sigma_y dG_y/dsigma
           + sigma_z dG_z/dsigma                            (Eq. 1_chain)
* Mixed-stage operator A_{a,b} p = Div_a(Grad_b p) on interior rows
  (Eq. poissonp: divergence at stage k = geometry a, gradient at stage k-1 =
  geometry b); the sigma = 1 rows are the Dirichlet condition p_D = 0
  (Eq. bcpd) and the sigma = 0 rows the Neumann condition
  n . Grad_b p (Eq. bcpdneu) with n = (h_x, h_y, 1).

Reading of the paper: the operator is the composite Div_a o Grad_b of the
discrete first derivatives, not the expanded transformed Laplacian; mixed
derivatives are derivatives applied one after the other (Sec. 3.5).  The
outward normal's sign and length cancel because the same n multiplies the
right-hand side row.
"""

import numpy as np

from . import spectral as sp


class Grid:
    """Tensor grid of one level (Sec. 3.4): Nx (x) by Ny (y) Fourier nodes,
    Nz+1 CGL nodes."""

    def __init__(self, Nx, Ny, Nz, L):
        self.Nx, self.Ny, self.Nz, self.L = int(Nx), int(Ny), int(Nz), float(L)
        self.M1 = self.Nz + 1
        self.x = sp.fourier_nodes(self.Nx, L)
        self.y = sp.fourier_nodes(self.Ny, L) if self.Ny > 1 else np.zeros(1)
        self.sigma = sp.cgl_sigma(self.Nz)
        self.Ds = sp.cheb_diff_matrix_sigma(self.Nz)

    @property
    def shape(self):
        return (self.M1, self.Ny, self.Nx)

    @property
    def n(self):
        return self.M1 * self.Ny * self.Nx

    # first derivatives of fields (M1, Ny, Nx) or surfaces (Ny, Nx)
    def dx(self, f):
        return sp.fourier_derivative(f, self.L, axis=f.ndim - 1)

    def dy(self, f):
        return sp.fourier_derivative(f, self.L, axis=f.ndim - 2)

    def ds(self, f):
        return np.tensordot(self.Ds, f, axes=(1, 0))


class Geometry:
    """Per-column metric of one free-surface elevation (Eq. 1_Scoef)."""

    def __init__(self, grid, h, eta):
        h = np.asarray(h, dtype=np.float64).reshape(grid.Ny, grid.Nx)
        eta = np.asarray(eta, dtype=np.float64).reshape(grid.Ny, grid.Nx)
        self.h, self.eta = h, eta
        self.d = h + eta
        self.hx, self.hy = grid.dx(h), grid.dy(h)
        self.dxd, self.dyd = grid.dx(self.d), grid.dy(self.d)
        s = grid.sigma[:, None, None]
        self.sx = (self.hx[None] - s * self.dxd[None]) / self.d[None]
        self.sy = (self.hy[None] - s * self.dyd[None]) / self.d[None]
        self.sz = 1.0 / self.d                       # (Ny, Nx)

    def z_nodes(self, grid):
        """Physical z of every node: z = sigma d - h (inverse of Eq. sigtrans)."""
        return grid.sigma[:, None, None] * self.d[None] - self.h[None]


def grad(grid, geo, f):
    """Transformed gradient (Eq. 1_chain) -> (G_x, G_y, G_z)."""
    fs = grid.ds(f)
    return (grid.dx(f) + geo.sx * fs,
            grid.dy(f) + geo.sy * fs,
            geo.sz[None] * fs)


def div(grid, geo, G):
    """Transformed divergence of a nodal vector field (Eq. 1_chain)."""
    Gx, Gy, Gz = G
    return (grid.dx(Gx) + geo.sx * grid.ds(Gx)
            + grid.dy(Gy) + geo.sy * grid.ds(Gy)
            + geo.sz[None] * grid.ds(Gz))


def apply_A(grid, geo_a, geo_b, p):
    """Mixed-stage Poisson operator A_{a,b} p with boundary rows.

    Interior rows: Div_a(Grad_b p) (Eq. poissonp); surface rows: p (Eq. bcpd);
    bottom rows: h_x G_x + h_y G_y + G_z with G = Grad_b p (Eq. bcpdneu).
    """
    p = np.asarray(p, dtype=np.float64).reshape(grid.shape)
    G = grad(grid, geo_b, p)
    out = div(grid, geo_a, G)
    out[0] = p[0]
    out[-1] = geo_b.hx * G[0][-1] + geo_b.hy * G[1][-1] + G[2][-1]
    return out


def assemble_A(grid, geo_a, geo_b):
    """Dense matrix of A_{a,b} (Eq. poissonp) by applying it to every unit
    vector (tiny sizes)."""
    n = grid.n
    A = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = apply_A(grid, geo_a, geo_b, e).ravel()
        e[j] = 0.0
    return A


def column_blocks(grid, geo_a, geo_b):
    """Diagonal (Nz+1)x(Nz+1) block A_rr of A_{a,b} for every vertical column r
    (the blocks of the Sec. 4.3 block relaxation).

    Written out from the composite operator: the x- and y-derivative matrices
    have a zero diagonal, so within one column only the second-derivative
    diagonal (D_x D_x)_rr = -(1/Nx) sum_{|n|<Nx/2} kappa_n^2 (Nyquist removed)
    and the sigma-derivative terms survive:
      A_rr = c_xx I + c_yy I + diag(sx_a) D diag(sx_b) D
             + diag(sy_a) D diag(sy_b) D + sz_a sz_b D D,
    the surface row is e_0^T and the bottom row
    (h_x sx_b + h_y sy_b + sz_b)|_bottom D[Nz, :].
    Returns an array (Ny, Nx, M1, M1).  Pinned against the rows/columns of
    ``assemble_A``.
    """
    D = grid.Ds
    M1 = grid.M1

    def diag2(N):
        if N == 1:
            return 0.0
        k = sp.fourier_wavenumbers(N, grid.L)
        k2 = k ** 2
        k2[N // 2] = 0.0
        return -np.sum(k2) / N

    cxx, cyy = diag2(grid.Nx), diag2(grid.Ny)
    B = np.zeros((grid.Ny, grid.Nx, M1, M1))
    DD = D @ D
    for jy in range(grid.Ny):
        for jx in range(grid.Nx):
            sxa, sxb = geo_a.sx[:, jy, jx], geo_b.sx[:, jy, jx]
            sya, syb = geo_a.sy[:, jy, jx], geo_b.sy[:, jy, jx]
            blk = (cxx + cyy) * np.eye(M1)
            blk += sxa[:, None] * (D @ (sxb[:, None] * D))
            blk += sya[:, None] * (D @ (syb[:, None] * D))
            blk += geo_a.sz[jy, jx] * geo_b.sz[jy, jx] * DD
            blk[0, :] = 0.0
            blk[0, 0] = 1.0
            coef = (geo_b.hx[jy, jx] * sxb[-1] + geo_b.hy[jy, jx] * syb[-1]
                    + geo_b.sz[jy, jx])
            blk[-1, :] = coef * D[-1, :]
            B[jy, jx] = blk
    return B


def poisson_rhs(grid, geo_a, geo_b, ustar, beta_dt):
    """Right-hand side of the projection form of Eq. poissonp / bcpdneu.

    With u* = u^(k-1) + beta_k (alpha_k K^(k-1) + dt F(q^(k-1))) (F without
    p_D), requiring Div_a u^(k) = 0 and n . u^(k) = 0 for
    u^(k) = u* - beta_k dt Grad_b p_D gives
      interior: Div_a u* / (beta_k dt), surface: 0,
      bottom:   (h_x u* + h_y v* + w*) / (beta_k dt).
    This equals the paper's right-hand side term by term (rho = 1).
    """
    b = div(grid, geo_a, ustar) / beta_dt
    b[0] = 0.0
    b[-1] = (geo_b.hx * ustar[0][-1] + geo_b.hy * ustar[1][-1] + ustar[2][-1]) / beta_dt
    return b
