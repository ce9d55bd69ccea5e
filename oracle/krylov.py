"""Krylov outer iteration (paper Sec. 4.4) and the solve entry points.

Test infrastructure only (see ``oracle/__init__.py``).

Reading of the paper: it names GMRES with one p-multigrid cycle as the
preconditioner but gives neither restart length nor orthogonalisation nor
side.  Used here: GMRES(m) with right preconditioning (so the monitored
residual is the true residual of the original system), modified
Gram-Schmidt, Givens rotations, stop when ||b - A x||_2 / ||b||_2 <= tol,
checked with the true residual at the end of every cycle.
"""

import numpy as np

from . import pmg


def gmres(apply_A, b, x0=None, precond=None, tol=1e-12, restart=30, maxit=1000):
    """Right-preconditioned restarted GMRES (Sec. 4.4); returns (x, iterations,
    relres_history)."""
    shape = b.shape
    bv = b.ravel()
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    if nb == 0.0:
        return np.zeros(shape), 0, [0.0]
    M = (lambda v: v) if precond is None else (lambda v: precond(v.reshape(shape)).ravel())
    A = lambda v: apply_A(v.reshape(shape)).ravel()
    hist = []
    its = 0
    while True:
        r = bv - A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta / nb <= tol or its >= maxit:
            return x.reshape(shape), its, hist
        m = restart
        V = np.zeros((m + 1, bv.size))
        Z = np.zeros((m, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            Z[k] = M(V[k])
            w = A(Z[k])
            for i in range(k + 1):                       # modified Gram-Schmidt
                H[i, k] = np.dot(w, V[i])
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                           # apply previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            k_used = k + 1
            if abs(g[k + 1]) / nb <= tol or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + Z[:k_used].T @ y


def solve_dense(level, b):
    """Plain definition of the discrete solution of Eq. poissonp: dense LU of
    A_{a,b} (tiny sizes)."""
    return np.linalg.solve(level.dense, b.ravel()).reshape(level.grid.shape)


def solve_pmg(Nx, Ny, Nz, L, h, eta_a, eta_b, b, tol=1e-12, x0=None, restart=30,
              maxit=500, cycle="v", nu1=2, nu2=2, smoother="jacobi", omega=0.4,
              coarsest_max=256, precondition=True, bc_transfer="inject", omega_s=1.0):
    """GMRES + one p-multigrid cycle per preconditioner application (Sec. 4.4).

    ``cycle`` is "v" (Algorithm 1) or "fmg" (Algorithm 2).  The spectral
    smoothers use the reference depth min(h) of the fine bathymetry.
    Returns (p, iterations, relres_history, levels).
    """
    levels = pmg.build_levels(Nx, Ny, Nz, L, h, eta_a, eta_b, coarsest_max)
    fine = levels[0]
    dref = float(np.min(h))
    if not precondition:
        pre = None
    elif cycle == "fmg":
        pre = lambda r: pmg.fmg(levels, r, nu1, nu2, smoother, omega, bc_transfer, omega_s, dref)
    else:
        pre = lambda r: pmg.vcycle(levels, 0, np.zeros_like(r), r, nu1, nu2, smoother, omega,
                                   bc_transfer, omega_s, dref)
    x, its, hist = gmres(fine.apply, np.asarray(b, dtype=np.float64).reshape(fine.grid.shape),
                         x0=x0, precond=pre, tol=tol, restart=restart, maxit=maxit)
    return x, its, hist, levels
