"""Pins of the oracle's metric, transformed gradient / divergence and the
mixed-stage Poisson operator (paper Eq. 1_chain, 1_Scoef, poissonp, bcpd,
bcpdneu) against closed forms and independent constructions.  CPU only."""

import math

import numpy as np
import pytest

from oracle import operator as op
from oracle import spectral as sp
import seeded_inputs as si


def curved_2d(Nx, Nz, L=2 * math.pi, amp=0.05):
    g = op.Grid(Nx, 1, Nz, L)
    x = g.x
    h = 1.0 + 0.2 * np.cos(2 * math.pi * x / L) + 0.1 * np.sin(4 * math.pi * x / L)
    eta = amp * np.cos(2 * math.pi * x / L + 0.3)
    return g, h, eta


def test_grad_matches_physical_gradient():
    # f(x, z) = sin(x) exp(z): Grad_b f at the nodes of geometry b = (cos x e^z, sin x e^z)
    errs = []
    for Nx, Nz in [(16, 8), (32, 14)]:
        g, h, eta = curved_2d(Nx, Nz)
        geo = op.Geometry(g, h, eta)
        z = geo.z_nodes(g)
        X = g.x[None, None, :]
        G = op.grad(g, geo, np.sin(X) * np.exp(z))
        errs.append(max(np.abs(G[0] - np.cos(X) * np.exp(z)).max(),
                        np.abs(G[2] - np.sin(X) * np.exp(z)).max()))
    assert errs[1] < 1e-11 and errs[1] < errs[0] * 1e-3      # spectral convergence


def test_div_matches_physical_divergence():
    # F = (cos(x) z^2, sin(2x) e^z):  div F = -sin(x) z^2 + sin(2x) e^z
    g, h, eta = curved_2d(32, 14)
    geo = op.Geometry(g, h, eta)
    z = geo.z_nodes(g)
    X = g.x[None, None, :]
    F = (np.cos(X) * z ** 2, np.zeros_like(z), np.sin(2 * X) * np.exp(z))
    ref = -np.sin(X) * z ** 2 + np.sin(2 * X) * np.exp(z)
    assert np.abs(op.div(g, geo, F) - ref).max() < 1e-10


@pytest.mark.parametrize("Nx,Nz", [(16, 8), (32, 12), (64, 16)])
def test_harmonic_function_has_zero_interior_residual(Nx, Nz):
    # p = cos(x) cosh(z + c) satisfies p_xx + p_zz = 0 for any surface / bottom
    g, h, eta = curved_2d(Nx, Nz)
    geo = op.Geometry(g, h, eta)
    z = geo.z_nodes(g)
    X = g.x[None, None, :]
    c = 1.3
    p = np.cos(X) * np.cosh(z + c)
    Ap = op.apply_A(g, geo, geo, p)
    px = -np.sin(X) * np.cosh(z + c)
    pz = np.cos(X) * np.sinh(z + c)
    tol = {16: 1e-3, 32: 1e-10, 64: 1e-9}[Nx]
    assert np.abs(Ap[1:-1]).max() < tol
    assert np.abs(Ap[0] - p[0]).max() == 0.0
    assert np.abs(Ap[-1] - (geo.hx * px[-1] + pz[-1])).max() < tol


def test_harmonic_3d():
    Nx, Nz, L = 32, 16, 2 * math.pi
    g = op.Grid(Nx, Nx, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 + 0.1 * np.cos(X) * np.sin(Y)
    eta = 0.03 * np.cos(X + 2 * Y)
    geo = op.Geometry(g, h, eta)
    z = geo.z_nodes(g)
    kx, ky = 1.0, 2.0
    k = math.hypot(kx, ky)
    p = np.cos(kx * X + ky * Y)[None] * np.cosh(k * (z + 1.5))
    Ap = op.apply_A(g, geo, geo, p)
    px = -kx * np.sin(kx * X + ky * Y)[None] * np.cosh(k * (z + 1.5))
    py = -ky * np.sin(kx * X + ky * Y)[None] * np.cosh(k * (z + 1.5))
    pz = k * np.cos(kx * X + ky * Y)[None] * np.sinh(k * (z + 1.5))
    assert np.abs(Ap[1:-1]).max() < 1e-8 * np.abs(p).max()
    bot = geo.hx * px[-1] + geo.hy * py[-1] + pz[-1]
    assert np.abs(Ap[-1] - bot).max() < 1e-8 * np.abs(p).max()


def test_flat_operator_equals_kronecker_assembly():
    # eta = 0, h = 1: A = D_x D_x (x) I + I (x) D_s D_s inside, identity on top,
    # D_s on the bottom row -- built from the 1D matrices independently.
    Nx, Nz, L = 8, 6, 3.0
    g = op.Grid(Nx, 1, Nz, L)
    geo = op.Geometry(g, np.ones(Nx), np.zeros(Nx))
    A = op.assemble_A(g, geo, geo)
    Dx = sp.fourier_diff_matrix(Nx, L)
    Ds = sp.cheb_diff_matrix_sigma(Nz)
    Ix, Is = np.eye(Nx), np.eye(Nz + 1)
    K = np.kron(Is, Dx @ Dx) + np.kron(Ds @ Ds, Ix)
    top = np.kron(Is[:1], Ix)
    bot = np.kron(Ds[-1:], Ix)
    K[:Nx] = top
    K[-Nx:] = bot
    assert np.abs(A - K).max() < 1e-11 * np.abs(K).max()


@pytest.mark.parametrize("Ny", [1, 4])
def test_column_blocks_equal_dense_diagonal_blocks(Ny):
    Nx, Nz, L = 8, 5, 4.0
    g = op.Grid(Nx, Ny, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 + 0.2 * np.cos(2 * np.pi * X / L) + (0.1 * np.sin(2 * np.pi * Y / L) if Ny > 1 else 0)
    ea = 0.05 * np.cos(2 * np.pi * (X + Y) / L)
    eb = 0.04 * np.sin(2 * np.pi * X / L)
    geo_a, geo_b = op.Geometry(g, h, ea), op.Geometry(g, h, eb)
    A = op.assemble_A(g, geo_a, geo_b)
    B = op.column_blocks(g, geo_a, geo_b)
    idx = np.arange(g.n).reshape(g.shape)
    for jy in range(Ny):
        for jx in range(Nx):
            rows = idx[:, jy, jx]
            assert np.abs(A[np.ix_(rows, rows)] - B[jy, jx]).max() < 1e-10 * np.abs(B).max()


def test_manufactured_solution_dense_solve():
    # 64 x 16 flat tank: q lies in the discrete space and cosh(z+1) is resolved
    # to rounding, so the discrete solution equals p_exact to rounding.
    Nx, Nz, L = 64, 16, 2 * math.pi
    g = op.Grid(Nx, 1, Nz, L)
    geo = op.Geometry(g, np.ones(Nx), np.zeros(Nx))
    z = geo.z_nodes(g)
    X = np.broadcast_to(g.x[None, None, :], g.shape)
    ms = si.Manufactured(seed=0)
    b = ms.laplacian(X, z)
    b[0] = ms.p(X[0], z[0])
    b[-1] = ms.dpdz(X[-1], z[-1])
    from oracle import pmg, krylov
    lev = pmg.Level(Nx, 1, Nz, L, np.ones((1, Nx)), np.zeros((1, Nx)), np.zeros((1, Nx)))
    p = krylov.solve_dense(lev, b)
    pe = ms.p(X, z)
    assert np.abs(p - pe).max() < 1e-11 * np.abs(pe).max()
    # and the residual of the exact solution in the oracle's operator is at rounding level
    r = b - op.apply_A(g, geo, geo, pe)
    assert np.linalg.norm(r) < 1e-11 * np.linalg.norm(b)


def test_poisson_rhs_projection_identity():
    # With b from poisson_rhs and the exact solve, u = u* - beta dt Grad_b p is
    # divergence-free (interior, geometry a) and satisfies n.u = 0 at the bottom.
    from oracle import pmg, krylov
    Nx, Nz, L = 16, 8, 2 * math.pi
    g, h, ea = curved_2d(Nx, Nz)
    eb = 0.9 * ea
    geo_a, geo_b = op.Geometry(g, h, ea), op.Geometry(g, h, eb)
    rng = np.random.default_rng(5)
    ustar = (rng.standard_normal(g.shape), np.zeros(g.shape), rng.standard_normal(g.shape))
    bdt = 0.013
    b = op.poisson_rhs(g, geo_a, geo_b, ustar, bdt)
    lev = pmg.Level(Nx, 1, Nz, g.L, h[None], ea[None], eb[None])
    p = krylov.solve_dense(lev, b)
    G = op.grad(g, geo_b, p)
    u = [ustar[i] - bdt * G[i] for i in range(3)]
    dv = op.div(g, geo_a, u)
    assert np.abs(dv[1:-1]).max() < 1e-9 * np.abs(op.div(g, geo_a, ustar)).max()
    bot = geo_b.hx * u[0][-1] + u[2][-1]
    assert np.abs(bot).max() < 1e-11
