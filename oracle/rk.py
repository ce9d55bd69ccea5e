"""Low-storage explicit Runge-Kutta time stepping with the pressure projection
at every stage (paper Sec. 3.1-3.3) and the kinematic free-surface update.

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper:

* Eq. (LSERK) gives the 2N-storage form but no coefficients; the "4th order"
  low-storage method is read as Carpenter & Kennedy's five-stage,
  fourth-order 2N-storage scheme (NASA TM-109112, 1994): alpha = A_k,
  beta = B_k.  ``butcher_from_2n`` and its test check the fourth-order
  conditions, which pins the constants independently of this table.
* Pressure split (Sec. 2): with p = p_D + g (eta - z) (rho = 1) the momentum
  forcing keeps -g (eta_x, eta_y, 0); the vertical hydrostatic part cancels
  gravity (Eq. sigmom1).
* Stage order: eta^(k) does not depend on p_D, so the free-surface update
  (Eq. kinematicFS) is done first; the Poisson problem then uses
  a = geometry of eta^(k) (divergence) and b = geometry of eta^(k-1)
  (gradient, forcing), Eq. poissonp.
* sigma_t = -sigma d_t / d with d_t = eta_t from the kinematic condition
  (Eq. 1_Scoef and the relation for d_t that follows it).
* Filter placement (Sec. 3.6 says "every stage"): on the stage input
  (eta^(k-1), u^(k-1)) before anything else, so the projected u^(k) stays
  discretely divergence-free.  Off unless ``filter=True``.
* Viscosity (nu > 0, Sec. 5.4): the forcing carries nu Div_b Grad_b q for
  every velocity component, the composite discrete Laplacian of the
  operator's interior rows, at every node.  No surface condition is
  printed; the reading is a stress-free surface: the vertical component of
  Grad_b q is zero on the surface nodes before the divergence (without a
  condition there the collocation Laplacian is not dissipative and the
  explicit stages blow up).  The bed is no-slip: after each stage the
  velocity and its registers K are set to zero on the bottom nodes.  The
  projection only zeroes the normal velocity there, so the tangential part
  is reset explicitly (the divergence invariant then holds up to that
  slip's size).
* ``linear=True`` is the linearised model of Sec. 5.3 (Eq. NSElin, linFS):
  no advection, d eta/dt = w~, and the sigma-map frozen at the still-water
  level (eta = 0 in every metric), since linearising about rest also
  linearises the moving domain (otherwise O(kA) geometry terms remain).
"""

import math
from fractions import Fraction

import numpy as np

from . import spectral as sp
from .operator import Grid, Geometry, grad, div, poisson_rhs
from . import krylov, pmg

# Carpenter-Kennedy RK4(3)5[2R+]C, 2N-storage (alpha_k, beta_k, c_k), k = 1..5
ALPHA = [Fraction(0), Fraction(-567301805773, 1357537059087),
         Fraction(-2404267990393, 2016746695238), Fraction(-3550918686646, 2091501179385),
         Fraction(-1275806237668, 842570457699)]
BETA = [Fraction(1432997174477, 9575080441755), Fraction(5161836677717, 13612068292357),
        Fraction(1720146321549, 2090206949498), Fraction(3134564353537, 4481467310338),
        Fraction(2277821191437, 14882151754819)]
CNODE = [Fraction(0), Fraction(1432997174477, 9575080441755),
         Fraction(2526269341429, 6820363183443), Fraction(2006345519317, 3224310063776),
         Fraction(2802321613138, 2924317926251)]
STAGES = 5


def butcher_from_2n(alpha, beta):
    """Butcher tableau (a_ij, b_j, c_i) implied by the 2N-storage recursion
    (Eq. LSERK).

    K^k = sum_{j<=k} (prod_{l=j+1..k} alpha_l) dt f_j and
    y^(k) = y^n + sum_{i<=k} beta_i K^i, so stage k (evaluated at y^(k-1)) has
    a_kj = sum_{i=j}^{k-1} beta_i prod_{l=j+1}^{i} alpha_l and the weights
    b_j = sum_{i=j}^{s} beta_i prod_{l=j+1}^{i} alpha_l.
    """
    s = len(alpha)

    def P(j, i):
        out = Fraction(1)
        for l in range(j + 1, i + 1):
            out *= alpha[l]
        return out

    A = [[Fraction(0)] * s for _ in range(s)]
    for k in range(s):
        for j in range(k):
            A[k][j] = sum((beta[i] * P(j, i) for i in range(j, k)), Fraction(0))
    b = [sum((beta[i] * P(j, i) for i in range(j, s)), Fraction(0)) for j in range(s)]
    c = [sum(A[k], Fraction(0)) for k in range(s)]
    return A, b, c


class State:
    """eta (Ny, Nx); u, v, w (Nz+1, Ny, Nx); the 2N registers K of Eq. LSERK; last p_D."""

    def __init__(self, grid, eta, u, v, w):
        self.eta = np.array(eta, dtype=np.float64).reshape(grid.Ny, grid.Nx)
        self.u = np.array(u, dtype=np.float64).reshape(grid.shape)
        self.v = np.array(v, dtype=np.float64).reshape(grid.shape)
        self.w = np.array(w, dtype=np.float64).reshape(grid.shape)
        self.Keta = np.zeros_like(self.eta)
        self.Ku = np.zeros_like(self.u)
        self.Kv = np.zeros_like(self.v)
        self.Kw = np.zeros_like(self.w)
        self.p = np.zeros(grid.shape)
        self.t = 0.0

    def copy(self):
        import copy
        return copy.deepcopy(self)


class Tank:
    """Problem definition (Sec. 2): grid, bathymetry h(x, y) > 0, gravity,
    viscosity, options."""

    def __init__(self, Nx, Ny, Nz, L, h, g=9.81, nu=0.0, linear=False, filter=False,
                 tol=1e-12, solver="pmg", coarsest_max=256, nu1=2, nu2=2, omega=0.4,
                 smoother="jacobi", restart=30):
        self.grid = Grid(Nx, Ny, Nz, L)
        self.h = np.asarray(h, dtype=np.float64).reshape(self.grid.Ny, self.grid.Nx)
        self.g, self.nu = float(g), float(nu)
        self.linear, self.filter = bool(linear), bool(filter)
        self.tol, self.solver = tol, solver
        self.opts = dict(coarsest_max=coarsest_max, nu1=nu1, nu2=nu2, omega=omega,
                         smoother=smoother, restart=restart)
        self.Fc = sp.cheb_filter_matrix(self.grid.Nz)
        self.last_info = []


def forcing(tank, geo_b, st):
    """f_eta (Eq. kinematicFS) and the momentum forcing without p_D (Eq. forc1).

    F_q = -(u dq/dchi + v dq/dgamma + w_sigma dq/dsigma) + nu Div_b Grad_b q
          - g (eta_x, eta_y, 0)_q,
    w_sigma = sigma_t + u sigma_x + v sigma_y + w sigma_z,
    sigma_t = -sigma f_eta / d.
    """
    gr = tank.grid
    ex, ey = gr.dx(st.eta), gr.dy(st.eta)
    ut, vt, wt = st.u[0], st.v[0], st.w[0]
    f_eta = wt if tank.linear else (-ut * ex - vt * ey + wt)
    F = [np.broadcast_to(-tank.g * ex[None], gr.shape).copy(),
         np.broadcast_to(-tank.g * ey[None], gr.shape).copy(),
         np.zeros(gr.shape)]
    if not tank.linear:
        sigt = -gr.sigma[:, None, None] * (f_eta / geo_b.d)[None]
        wsig = sigt + st.u * geo_b.sx + st.v * geo_b.sy + st.w * geo_b.sz[None]
        for i, q in enumerate((st.u, st.v, st.w)):
            F[i] -= st.u * gr.dx(q) + st.v * gr.dy(q) + wsig * gr.ds(q)
    if tank.nu != 0.0:
        for i, q in enumerate((st.u, st.v, st.w)):
            G = grad(gr, geo_b, q)
            G[2][0] = 0.0                     # stress-free surface: no vertical flux
            F[i] += tank.nu * div(gr, geo_b, G)
    return f_eta, F


def apply_filter(tank, st):
    """Exponential cut-off on Fourier (x, y) and Chebyshev (sigma) modes (Sec. 3.6)."""
    gr = tank.grid
    st.eta = sp.fourier_filter(st.eta, axis=1)
    if gr.Ny > 1:
        st.eta = sp.fourier_filter(st.eta, axis=0)
    for name in ("u", "v", "w"):
        q = getattr(st, name)
        q = sp.fourier_filter(q, axis=2)
        if gr.Ny > 1:
            q = sp.fourier_filter(q, axis=1)
        q = np.tensordot(tank.Fc, q, axes=(1, 0))
        setattr(st, name, q)


def solve_pressure(tank, eta_a, eta_b, rhs, x0):
    gr = tank.grid
    if tank.solver == "dense":
        lev = pmg.Level(gr.Nx, gr.Ny, gr.Nz, gr.L, tank.h, eta_a, eta_b)
        return krylov.solve_dense(lev, rhs), 0
    p, its, hist, _ = krylov.solve_pmg(gr.Nx, gr.Ny, gr.Nz, gr.L, tank.h, eta_a, eta_b, rhs,
                                       tol=tank.tol, x0=x0, **tank.opts)
    return p, its


def stage(tank, st, k, dt):
    """One LSERK stage k = 1..5 with the mixed-stage projection (Sec. 3.2)."""
    a = float(ALPHA[k - 1])
    b = float(BETA[k - 1])
    gr = tank.grid
    if tank.filter:
        apply_filter(tank, st)
    flat = np.zeros_like(st.eta)
    geo_b = Geometry(gr, tank.h, flat if tank.linear else st.eta)
    f_eta, F = forcing(tank, geo_b, st)
    st.Keta = a * st.Keta + dt * f_eta
    eta_new = st.eta + b * st.Keta
    geo_a = geo_b if tank.linear else Geometry(gr, tank.h, eta_new)
    ustar = [q + b * (a * K + dt * Fq)
             for q, K, Fq in zip((st.u, st.v, st.w), (st.Ku, st.Kv, st.Kw), F)]
    rhs = poisson_rhs(gr, geo_a, geo_b, ustar, b * dt)
    p, its = solve_pressure(tank, flat if tank.linear else eta_new,
                            flat if tank.linear else st.eta, rhs, st.p)
    tank.last_info.append(its)
    G = grad(gr, geo_b, p)
    st.Ku = a * st.Ku + dt * (F[0] - G[0])
    st.Kv = a * st.Kv + dt * (F[1] - G[1])
    st.Kw = a * st.Kw + dt * (F[2] - G[2])
    st.u = st.u + b * st.Ku
    st.v = st.v + b * st.Kv
    st.w = st.w + b * st.Kw
    if tank.nu != 0.0:                      # no-slip bed
        for q in (st.u, st.v, st.w, st.Ku, st.Kv, st.Kw):
            q[-1] = 0.0
    st.eta = eta_new
    st.p = p
    return st


def step(tank, st, dt):
    """One full step of Eq. LSERK (all five stages)."""
    for k in range(1, STAGES + 1):
        stage(tank, st, k, dt)
    st.t += dt
    return st


def relaxation_weight(x, x0, x1):
    """Target weight of a relaxation zone (Sec. 5.5, after Larsen & Dancy):
    with xi = (x - x0) / (x1 - x0), w = (exp(xi^3.5) - 1) / (e - 1) inside the
    zone (0 at its inner edge x0, 1 at x1), 0 outside."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = min(x0, x1), max(x0, x1)
    xi = np.clip((x - x0) / (x1 - x0), 0.0, 1.0)
    w = (np.exp(xi ** 3.5) - 1.0) / (math.e - 1.0)
    return np.where((x >= lo) & (x <= hi), w, 0.0)


def relax(tank, st, x0, x1, eta_t=None, u_t=None, v_t=None, w_t=None):
    """Relaxation zone (Sec. 5.5): q <- (1 - w) q + w q_target for the given
    targets (columns of the zone)."""
    wgt = relaxation_weight(tank.grid.x, x0, x1)[None, :]
    if eta_t is not None:
        st.eta = (1.0 - wgt) * st.eta + wgt * eta_t
    for name, tgt in (("u", u_t), ("v", v_t), ("w", w_t)):
        if tgt is not None and not (name == "v" and tank.grid.Ny == 1):
            q = getattr(st, name)
            setattr(st, name, (1.0 - wgt[None]) * q + wgt[None] * tgt)
    return st


def divergence_residual(tank, st):
    """Interior Div u and bottom n . u of the current state (geometry of st.eta):
    the incompressibility and bed conditions the projection of Eq. rkforc1 enforces."""
    gr = tank.grid
    geo = Geometry(gr, tank.h, np.zeros_like(st.eta) if tank.linear else st.eta)
    dv = div(gr, geo, (st.u, st.v, st.w))
    bot = geo.hx * st.u[-1] + geo.hy * st.v[-1] + st.w[-1]
    return dv[1:-1], bot
