"""Steady nonlinear periodic waves by the Fourier stream-function method
(Rienecker & Fenton 1981), the initial condition of the paper's nonlinear
accuracy study (Sec. 5.2) and of its bar case (Sec. 5.5).

Test infrastructure only (see ``oracle/__init__.py``).

The paper cites the method without printing it.  What is solved here, in a
frame moving with the wave speed c over a flat bed at y = 0 (still depth d):

* stream function psi(X, y) = -U y + sum_{j=1..N} B_j sinh(j k y) / cosh(j k d)
  cos(j k X), with X = x - c t; velocities u = psi_y, w = -psi_X (moving
  frame).  The bed psi = 0 is a streamline by construction and Laplace's
  equation holds exactly (irrotational, incompressible flow);
* at the N + 1 surface points X_m = m pi / (N k), m = 0..N (crest to trough;
  the wave is symmetric about its crest), with surface heights y = d + eta_m:
  the surface is a streamline, psi = -Q, and Bernoulli's condition holds,
  (u^2 + w^2) / 2 + g eta_m = R;
* eta is measured from the mean water level: its mean over the wavelength
  (trapezoidal rule on the N + 1 points, which is exact for the cosine
  series) is zero; the wave height is eta_0 - eta_N = H;
* no mean Eulerian current in the fixed frame: c = U.

Unknowns U, Q, R, eta_0..eta_N, B_1..B_N (2N + 4) against 2N + 4 equations,
solved by Newton's method with a central-difference Jacobian; the height is
raised in steps from a linear-theory start (continuation).  In the fixed
frame the fields are eta(x, t) = sum_j E_j cos(j k (x - c t)) (the cosine
interpolant of the eta_m) and, at height z above the still level,
u = sum_j j k B_j cosh(j k (z + d)) / cosh(j k d) cos(j k X),
w = sum_j j k B_j sinh(j k (z + d)) / cosh(j k d) sin(j k X).
"""

import math

import numpy as np


class Wave:
    """A solved stream-function wave (the Sec. 5.2 initial condition): k, d, H,
    g, c, U, Q, R, B (1..N), eta_m."""

    def __init__(self, k, d, H, g, N, U, Q, R, eta, B):
        self.k, self.d, self.H, self.g, self.N = k, d, H, g, N
        self.U, self.Q, self.R = U, Q, R
        self.c = U
        self.eta_nodes = np.asarray(eta, dtype=np.float64)
        self.B = np.asarray(B, dtype=np.float64)
        # cosine coefficients of the surface from its N + 1 node values
        m = np.arange(N + 1)
        w = np.ones(N + 1)
        w[0] = w[-1] = 0.5
        E = np.array([2.0 / N * np.sum(w * self.eta_nodes * np.cos(j * m * math.pi / N))
                      for j in range(N + 1)])
        E[0] *= 0.5
        E[N] *= 0.5
        self.E = E

    def eta(self, x, t=0.0):
        X = np.asarray(x, dtype=np.float64) - self.c * t
        j = np.arange(self.N + 1)
        return np.cos(np.multiply.outer(X, j * self.k)) @ self.E

    def velocity(self, x, z, t=0.0):
        """Fixed-frame (u, w) of the Sec. 5.2 wave at horizontal position x and
        height z above the still water level (broadcast together)."""
        X = np.asarray(x, dtype=np.float64) - self.c * t
        y = np.asarray(z, dtype=np.float64) + self.d
        X, y = np.broadcast_arrays(X, y)
        u = np.zeros(X.shape)
        w = np.zeros(X.shape)
        for j in range(1, self.N + 1):
            jk = j * self.k
            sh, ch = _sh_ch(jk, y, self.d)
            u += jk * self.B[j - 1] * ch * np.cos(jk * X)
            w += jk * self.B[j - 1] * sh * np.sin(jk * X)
        return u, w


def _sh_ch(jk, y, d):
    """sinh(jk y) / cosh(jk d) and cosh(jk y) / cosh(jk d) without overflow."""
    e1 = np.exp(jk * (y - d))
    e2 = np.exp(-jk * (y + d))
    e3 = math.exp(-2.0 * jk * d)
    return (e1 - e2) / (1.0 + e3), (e1 + e2) / (1.0 + e3)


def _residual(z, k, d, H, g, N):
    U, Q, R = z[0], z[1], z[2]
    eta = z[3:3 + N + 1]
    B = z[3 + N + 1:]
    Xm = np.arange(N + 1) * math.pi / (N * k)
    y = d + eta
    psi = -U * y
    u = -U * np.ones(N + 1)
    w = np.zeros(N + 1)
    for j in range(1, N + 1):
        jk = j * k
        sh, ch = _sh_ch(jk, y, d)
        psi += B[j - 1] * sh * np.cos(jk * Xm)
        u += B[j - 1] * jk * ch * np.cos(jk * Xm)
        w += B[j - 1] * jk * sh * np.sin(jk * Xm)
    kin = psi + Q
    dyn = 0.5 * (u * u + w * w) + g * eta - R
    wts = np.ones(N + 1)
    wts[0] = wts[-1] = 0.5
    mean = np.sum(wts * eta) / N
    height = eta[0] - eta[-1] - H
    return np.concatenate([kin, dyn, [mean, height]])


def solve(k, d, H, g=9.81, N=24, steps=None, tol=1e-13, maxit=60):
    """Stream-function wave (Sec. 5.2; Rienecker & Fenton, cited there) of
    wavenumber k, depth d, height H (Newton's method with continuation in H).
    Returns a ``Wave``."""
    if steps is None:
        steep = H * k / (2 * math.pi)
        steps = max(1, int(math.ceil(steep / 0.005)))
    c0 = math.sqrt(g / k * math.tanh(k * d))
    n = 2 * N + 4
    Xm = np.arange(N + 1) * math.pi / (N * k)
    sols = []
    for s in range(1, steps + 1):
        Hs = H * s / steps
        if not sols:                      # linear theory
            cur = np.zeros(n)
            cur[0] = c0
            cur[1] = c0 * d
            cur[2] = 0.5 * c0 * c0
            cur[3:3 + N + 1] = 0.5 * Hs * np.cos(k * Xm)
            cur[3 + N + 1] = c0 * Hs / (2.0 * math.tanh(k * d))
        elif len(sols) == 1:
            cur = sols[-1].copy()
        else:                             # linear extrapolation in H
            cur = 2.0 * sols[-1] - sols[-2]
        for _ in range(maxit):
            F = _residual(cur, k, d, Hs, g, N)
            J = np.zeros((n, n))
            for i in range(n):                     # central differences
                hstep = 1e-6 * max(1e-3, abs(cur[i]))
                zp = cur.copy()
                zm = cur.copy()
                zp[i] += hstep
                zm[i] -= hstep
                J[:, i] = (_residual(zp, k, d, Hs, g, N) - _residual(zm, k, d, Hs, g, N)) / (2 * hstep)
            dz = np.linalg.solve(J, -F)
            cur = cur + dz
            if np.abs(dz).max() < tol * max(1.0, np.abs(cur).max()):
                break
        sols.append(cur)
    z = sols[-1]
    F = _residual(z, k, d, H, g, N)
    if not np.all(np.isfinite(F)) or np.abs(F).max() > 1e-9 * max(1.0, g * H):
        raise RuntimeError("stream-function Newton iteration did not converge (max residual %.2e)"
                           % np.abs(F).max())
    return Wave(k, d, H, g, N, z[0], z[1], z[2], z[3:3 + N + 1], z[3 + N + 1:])
