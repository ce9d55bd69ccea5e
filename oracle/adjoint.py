"""Exact derivative of the discrete time step (the paper has no adjoint).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The forward map of one low-storage Runge-Kutta step with the pressure
projection at every stage (Sec. 3.1-3.3, Eq. kinematicFS, forc1, poissonp,
bcpd, bcpdneu, rkforc1) is restated here for 2D tanks with plain PyTorch CPU
float64 operations: dense derivative matrices (the same closed forms as
``spectral``), the dense operator A_{a,b} assembled column by column and a
dense LU solve.  ``torch.autograd`` then gives the exact derivative of that
map with respect to the bathymetry h(x) and the state, with no hand-derived
adjoint equation on this side; a GPU adjoint is compared with it.

Pins (tests/test_oracle_adjoint.py):
* the forward step equals ``rk.step`` with the dense solver (numpy, pinned by
  its own tests) to 1e-12 relative, with and without the filter and in the
  linearised model;
* directional derivatives of the gauge loss along random directions in h and
  in the initial elevation match central finite differences of ``rk.step``
  (step 1e-6) to 1e-6 relative;
* the dense transposed operator satisfies <A x, y> = <x, A^T y>.

Gauge loss of the gradient workload: J = 1/2 sum_n sum_g (eta_n(x_g) -
eta*_n(x_g))^2 dt over the states after steps n = 1..N at gauge nodes x_g.
"""

import numpy as np
import torch

from . import spectral as sp
from .rk import ALPHA, BETA, STAGES

F64 = torch.float64


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=F64)


class Grid2:
    """2D grid (Sec. 3.4): Nx Fourier nodes (x, last axis), Nz+1 CGL nodes (sigma, first axis)."""

    def __init__(self, Nx, Nz, L):
        self.Nx, self.Nz, self.L = int(Nx), int(Nz), float(L)
        self.M1 = self.Nz + 1
        self.Dx = _t(sp.fourier_diff_matrix(self.Nx, self.L))     # Nyquist coefficient -> 0
        self.Ds = _t(sp.cheb_diff_matrix_sigma(self.Nz))
        self.sigma = _t(sp.cgl_sigma(self.Nz))
        self.Fx = _t(sp.fourier_filter(np.eye(self.Nx), axis=0))  # filter as a matrix
        self.Fc = _t(sp.cheb_filter_matrix(self.Nz))

    def dx(self, f):
        return f @ self.Dx.T

    def ds(self, f):
        return torch.matmul(self.Ds, f)


def metric(g, h, e):
    """Per-column sigma metric of surface e over bathymetry h (Eq. 1_Scoef)."""
    d = h + e
    hx = g.dx(h)
    sx = (hx[None] - g.sigma[:, None] * g.dx(d)[None]) / d[None]
    return dict(d=d, hx=hx, sx=sx, sz=1.0 / d)


def grad(g, m, f):
    fs = g.ds(f)
    return g.dx(f) + m["sx"] * fs, m["sz"] * fs


def div(g, m, Gx, Gz):
    return g.dx(Gx) + m["sx"] * g.ds(Gx) + m["sz"] * g.ds(Gz)


def apply_A(g, ma, mb, p):
    """A_{a,b} p (Eq. poissonp, bcpd, bcpdneu; Eq. 1_chain) for p of shape
    (..., M1, Nx): interior Div_a Grad_b p, surface row p, bottom row
    h_x G_x + G_z."""
    Gx, Gz = grad(g, mb, p)
    out = div(g, ma, Gx, Gz)
    bot = (mb["hx"] * Gx[..., -1, :] + Gz[..., -1, :]).unsqueeze(-2)
    return torch.cat([p[..., :1, :], out[..., 1:-1, :], bot], dim=-2)


def assemble_A(g, ma, mb):
    """Dense A_{a,b} of Eq. poissonp (n x n, n = M1 Nx, row-major (m, x) ordering)."""
    n = g.M1 * g.Nx
    E = torch.eye(n, dtype=F64).reshape(n, g.M1, g.Nx)
    return apply_A(g, ma, mb, E).reshape(n, n).T


def apply_AT(g, ma, mb, lam):
    """A_{a,b}^T lam through the dense matrix (the plain definition; the paper
    has no adjoint, this is the transpose of the Eq. poissonp operator)."""
    return (assemble_A(g, ma, mb).T @ lam.reshape(-1)).reshape(g.M1, g.Nx)


def poisson_rhs(g, ma, mb, us, ws, bdt):
    b = div(g, ma, us, ws) / bdt
    bot = (mb["hx"] * us[-1] + ws[-1]) / bdt
    return torch.cat([torch.zeros_like(bot)[None], b[1:-1], bot[None]], dim=0)


def stage(g, h, st, k, dt, grav=9.81, linear=False, filt=False):
    """Stage k of Eq. LSERK with the projection: st = (eta, u, w, K_eta, K_u, K_w)."""
    a, b = float(ALPHA[k - 1]), float(BETA[k - 1])
    eta, u, w, Ke, Ku, Kw = st
    if filt:
        eta = eta @ g.Fx.T
        u = g.Fc @ (u @ g.Fx.T)
        w = g.Fc @ (w @ g.Fx.T)
    zero = torch.zeros_like(eta)
    mb = metric(g, h, zero if linear else eta)
    ex = g.dx(eta)
    fe = w[0] if linear else (-u[0] * ex + w[0])
    Fu = (-grav * ex)[None].expand(g.M1, g.Nx)
    Fw = torch.zeros_like(w)
    if not linear:
        wsig = -g.sigma[:, None] * (fe / mb["d"])[None] + u * mb["sx"] + w * mb["sz"][None]
        Fu = Fu - (u * g.dx(u) + wsig * g.ds(u))
        Fw = Fw - (u * g.dx(w) + wsig * g.ds(w))
    Ke = a * Ke + dt * fe
    eta_new = eta + b * Ke
    ma = mb if linear else metric(g, h, eta_new)
    Ku1 = a * Ku + dt * Fu
    Kw1 = a * Kw + dt * Fw
    rhs = poisson_rhs(g, ma, mb, u + b * Ku1, w + b * Kw1, b * dt)
    p = torch.linalg.solve(assemble_A(g, ma, mb), rhs.reshape(-1)).reshape(g.M1, g.Nx)
    Gx, Gz = grad(g, mb, p)
    Ku2 = Ku1 - dt * Gx
    Kw2 = Kw1 - dt * Gz
    return (eta_new, u + b * Ku2, w + b * Kw2, Ke, Ku2, Kw2)


def step(g, h, eta, u, w, dt, **kw):
    """One full step of Eq. LSERK from (eta, u, w); the 2N registers start at
    zero (alpha_1 = 0)."""
    st = (eta, u, w, torch.zeros_like(eta), torch.zeros_like(u), torch.zeros_like(w))
    for k in range(1, STAGES + 1):
        st = stage(g, h, st, k, dt, **kw)
    return st[0], st[1], st[2]


def run(g, h, eta, u, w, dt, nsteps, gauges, **kw):
    """Gauge series: eta after steps 1..nsteps (Eq. LSERK) at the gauge node indices."""
    out = []
    for _ in range(nsteps):
        eta, u, w = step(g, h, eta, u, w, dt, **kw)
        out.append(eta[gauges])
    return torch.stack(out), (eta, u, w)


def gauge_loss(series, target, dt):
    return 0.5 * torch.sum((series - target) ** 2) * dt


def loss_and_gradient(g, h, eta0, u0, w0, dt, nsteps, gauges, target, **kw):
    """J and dJ/dh, dJ/d(eta0, u0, w0) by reverse-mode differentiation of the
    discrete steps (the paper has no adjoint: the derivative of Sec. 3.1-3.3
    as discretised here)."""
    h = _t(h).requires_grad_(True)
    eta0 = _t(eta0).requires_grad_(True)
    u0 = _t(u0).requires_grad_(True)
    w0 = _t(w0).requires_grad_(True)
    series, _ = run(g, h, eta0, u0, w0, dt, nsteps, gauges, **kw)
    J = gauge_loss(series, _t(target), dt)
    gh, ge, gu, gw = torch.autograd.grad(J, (h, eta0, u0, w0))
    return J.item(), gh.numpy(), ge.numpy(), gu.numpy(), gw.numpy()


def step_vjp(g, h, eta, u, w, dt, lam_eta, lam_u, lam_w, **kw):
    """(d step / d(state, h))^T applied to (lam_eta, lam_u, lam_w) (no paper
    passage: the derivative of one Eq. LSERK step): the adjoint of one step, returning (lam_eta, lam_u, lam_w) at the step start
    and the contribution to dJ/dh."""
    h = _t(h).requires_grad_(True)
    s = [_t(a).requires_grad_(True) for a in (eta, u, w)]
    out = step(g, h, *s, dt, **kw)
    val = sum(torch.sum(o * _t(l)) for o, l in zip(out, (lam_eta, lam_u, lam_w)))
    grads = torch.autograd.grad(val, (*s, h))
    return tuple(x.numpy() for x in grads)
