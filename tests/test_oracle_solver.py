"""Pins of the oracle's p-multigrid / GMRES solve (paper Sec. 4, Algorithms 1-2)
against the dense LU solve of the same collocation system.  CPU only."""

import math

import numpy as np
import pytest

from oracle import krylov, pmg
from oracle import operator as op


def problem(Nx, Ny, Nz, L=2 * math.pi, seed=7):
    g = op.Grid(Nx, Ny, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - 0.3 * np.exp(-((X - L / 2) / (L / 8)) ** 2)
    if Ny > 1:
        h = h + 0.05 * np.cos(2 * np.pi * Y / L)
    ea = 0.06 * np.cos(2 * np.pi * X / L) + (0.02 * np.sin(2 * np.pi * Y / L) if Ny > 1 else 0)
    eb = 0.05 * np.cos(2 * np.pi * X / L + 0.1)
    b = np.random.default_rng(seed).standard_normal(g.shape)
    return g, h, ea, eb, b


def test_hierarchies_of_the_workloads():
    assert pmg.hierarchy(64, 1, 16) == [(64, 1, 16), (32, 1, 16), (16, 1, 16), (8, 1, 8)]
    assert pmg.hierarchy(1024, 1, 24)[-2:] == [(16, 1, 24), (16, 1, 12)]
    assert pmg.hierarchy(256, 256, 16)[-1] == (4, 4, 4)
    # coarsest-size option
    assert pmg.hierarchy(1024, 1, 24, coarsest_max=64)[-1] == (8, 1, 6)


@pytest.mark.parametrize("smoother,cycle", [("jacobi", "v"), ("gs", "v"), ("jacobi", "fmg")])
def test_pmg_gmres_equals_dense_lu_2d(smoother, cycle):
    g, h, ea, eb, b = problem(32, 1, 10)
    lev = pmg.Level(32, 1, 10, g.L, h, ea, eb)
    p_lu = krylov.solve_dense(lev, b)
    p, its, hist, levels = krylov.solve_pmg(32, 1, 10, g.L, h, ea, eb, b, tol=1e-13,
                                            smoother=smoother, cycle=cycle, coarsest_max=64)
    assert len(levels) >= 3
    assert np.abs(p - p_lu).max() < 1e-9 * np.abs(p_lu).max()
    r = b - lev.apply(p)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b) * 1.0001
    assert hist[-1] <= 1e-13


def test_pmg_gmres_equals_dense_lu_3d():
    g, h, ea, eb, b = problem(8, 8, 6)
    lev = pmg.Level(8, 8, 6, g.L, h, ea, eb)
    p_lu = krylov.solve_dense(lev, b)
    p, its, hist, levels = krylov.solve_pmg(8, 8, 6, g.L, h, ea, eb, b, tol=1e-12,
                                            coarsest_max=64)
    assert len(levels) >= 2
    assert np.abs(p - p_lu).max() < 1e-8 * np.abs(p_lu).max()


def test_preconditioner_cuts_iterations():
    # Table 1 finds the p-multigrid preconditioner reduces GMRES iterations by
    # orders of magnitude; check the same qualitative gap.
    g, h, ea, eb, b = problem(32, 1, 16)
    _, its_pmg, _, _ = krylov.solve_pmg(32, 1, 16, g.L, h, ea, eb, b, tol=1e-8)
    _, its_none, _, _ = krylov.solve_pmg(32, 1, 16, g.L, h, ea, eb, b, tol=1e-8,
                                         precondition=False, maxit=400)
    assert its_pmg * 10 < its_none


def test_vcycle_is_a_contraction():
    g, h, ea, eb, b = problem(32, 1, 12)
    levels = pmg.build_levels(32, 1, 12, g.L, h, ea, eb, coarsest_max=64)
    x = np.zeros(g.shape)
    r0 = np.linalg.norm(b)
    for _ in range(6):
        x = x + pmg.vcycle(levels, 0, np.zeros(g.shape), b - levels[0].apply(x))
    assert np.linalg.norm(b - levels[0].apply(x)) < 0.5 * r0


def test_sigma_transfers_between_equal_degrees_are_the_identity():
    # Truncating the degree-Nz Chebyshev interpolant of a column to degree Nz
    # and evaluating it at the same Gauss-Lobatto nodes returns the column,
    # and so does interpolating it there (Sec. 4.2 transfers): a coarsening
    # step in x only moves the residual and the correction through the
    # Fourier resampling alone.
    from oracle import spectral as sp
    for Nz in (4, 6, 8, 12, 16, 24, 32):
        for bc in ("inject", "paper"):
            R = pmg.restrict_sigma_matrix(Nz, Nz, bc)
            assert np.abs(R - np.eye(Nz + 1)).max() < 1e-12, (Nz, bc)
        P = sp.cheb_prolong_matrix(Nz, Nz)
        assert np.abs(P - np.eye(Nz + 1)).max() < 1e-12, Nz
    # between different degrees, restriction after interpolation is exact on
    # the coarse polynomials (R P = I) while P R is a projection, not I
    for Nf, Nc in ((24, 12), (16, 8), (12, 6)):
        P = sp.cheb_prolong_matrix(Nc, Nf)
        for bc in ("inject", "paper"):
            R = pmg.restrict_sigma_matrix(Nf, Nc, bc)
            assert np.abs(R @ P - np.eye(Nc + 1)).max() < 1e-12, (Nf, Nc, bc)
        PR = P @ pmg.restrict_sigma_matrix(Nf, Nc, "paper")
        assert np.abs(PR @ PR - PR).max() < 1e-10 and np.abs(PR - np.eye(Nf + 1)).max() > 0.1
    # the whole restriction of an x-only coarsening step is the Fourier truncation
    g, h, ea, eb, b = problem(32, 1, 8)
    lev = pmg.build_levels(32, 1, 8, 2 * math.pi, h, ea, eb, coarsest_max=64)
    fine, coarse = lev[0].grid, lev[1].grid
    assert (coarse.Nx, coarse.Nz) == (16, 8)
    r = pmg.restrict(fine, coarse, b)
    assert np.abs(r - sp.fourier_resample(b, 16, axis=2)).max() < 1e-12 * np.abs(b).max()
    e = np.random.default_rng(2).standard_normal(coarse.shape)
    assert np.abs(pmg.prolong(coarse, fine, e) - sp.fourier_resample(e, 32, axis=2)).max() < 1e-12 * np.abs(e).max()


def test_fmg_on_two_levels_is_a_vcycle_from_the_prolongated_coarse_solve():
    # Algorithm 2 with two grids: the coarse problem for the restricted
    # right-hand side solved exactly (dense LU), prolongated, and one V-cycle
    # on the fine grid from that state
    g, h, ea, eb, b = problem(16, 1, 8)
    levels = pmg.build_levels(16, 1, 8, g.L, h, ea, eb, coarsest_max=100)
    assert len(levels) == 2
    fc = pmg.restrict(levels[0].grid, levels[1].grid, b)
    uc = np.linalg.solve(levels[1].dense, fc.ravel()).reshape(levels[1].grid.shape)
    u0 = pmg.prolong(levels[1].grid, levels[0].grid, uc)
    want = pmg.vcycle(levels, 0, u0, b, 2, 2, "jacobi", 0.4, "inject")
    got = pmg.fmg(levels, b, 2, 2, "jacobi", 0.4, "inject")
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # with one level it is the direct solve
    one = pmg.build_levels(8, 1, 4, g.L, h[:, ::2], ea[:, ::2], eb[:, ::2], coarsest_max=64)
    assert len(one) == 1
    f1 = b[::2, :, ::2].copy()
    assert np.allclose(pmg.fmg(one, f1), np.linalg.solve(one[0].dense, f1.ravel()).reshape(f1.shape),
                       rtol=0, atol=1e-12 * np.abs(f1).max() * 1e3)


def test_fmg_is_linear_and_beats_one_vcycle():
    g, h, ea, eb, b = problem(64, 1, 12)
    levels = pmg.build_levels(64, 1, 12, g.L, h, ea, eb, coarsest_max=64)
    lev = levels[0]
    b2 = np.random.default_rng(11).standard_normal(g.shape)
    a = pmg.fmg(levels, 2.0 * b - 3.0 * b2)
    c = 2.0 * pmg.fmg(levels, b) - 3.0 * pmg.fmg(levels, b2)
    assert np.abs(a - c).max() <= 1e-11 * np.abs(c).max()
    # a smooth right-hand side: FMG's error is below one V-cycle's from zero
    X = np.broadcast_to(g.x[None, None, :], g.shape)
    S = np.broadcast_to(g.sigma[:, None, None], g.shape)
    f = np.cos(X) * (1 + S ** 2)
    exact = np.linalg.solve(lev.dense, f.ravel()).reshape(g.shape)
    e_fmg = np.linalg.norm(pmg.fmg(levels, f) - exact)
    e_v = np.linalg.norm(pmg.vcycle(levels, 0, np.zeros(g.shape), f) - exact)
    assert e_fmg < e_v


@pytest.mark.parametrize("Nx,Ny,Nz,dref", [(32, 1, 10, 1.0), (16, 1, 8, 0.7), (8, 8, 6, 1.3)])
def test_spectral_smoother_is_exact_on_the_flat_reference_tank(Nx, Ny, Nz, dref):
    # on a flat tank of depth dref at rest the reference operator is the
    # operator itself, so one undamped sweep from zero is the dense solve
    L = 2 * math.pi
    g = op.Grid(Nx, Ny, Nz, L)
    h = np.full((Ny, Nx), dref)
    z = np.zeros((Ny, Nx))
    lev = pmg.Level(Nx, Ny, Nz, L, h, z, z)
    b = np.random.default_rng(2).standard_normal(g.shape)
    want = np.linalg.solve(lev.dense, b.ravel()).reshape(g.shape)
    got = pmg.spectral_smooth(lev, np.zeros(g.shape), b, 1.0, dref)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    wantT = np.linalg.solve(lev.dense.T, b.ravel()).reshape(g.shape)
    gotT = pmg.spectral_smooth(lev, np.zeros(g.shape), b, 1.0, dref, transpose=True)
    assert np.abs(gotT - wantT).max() <= 1e-10 * np.abs(wantT).max()
    # a wrong reference depth is no longer exact
    off = pmg.spectral_smooth(lev, np.zeros(g.shape), b, 1.0, 1.1 * dref)
    assert np.abs(off - want).max() > 1e-3 * np.abs(want).max()


@pytest.mark.parametrize("smoother", ["spectral", "jacobi+spectral"])
def test_spectral_smoothers_solve_to_dense_lu(smoother):
    g, h, ea, eb, b = problem(32, 1, 10)
    lev = pmg.Level(32, 1, 10, g.L, h, ea, eb)
    p_lu = krylov.solve_dense(lev, b)
    p, its, hist, levels = krylov.solve_pmg(32, 1, 10, g.L, h, ea, eb, b, tol=1e-13, smoother=smoother,
                                            coarsest_max=64, nu1=1, nu2=1)
    assert np.abs(p - p_lu).max() < 1e-9 * np.abs(p_lu).max()
    _, its_bj, _, _ = krylov.solve_pmg(32, 1, 10, g.L, h, ea, eb, b, tol=1e-13, coarsest_max=64, nu1=1, nu2=1)
    if smoother == "jacobi+spectral":
        assert its < its_bj


def test_vcycle_smoother_by_level_list():
    # a list of smoother kinds by level: the same kind everywhere reproduces
    # the single-kind cycle, and a mixed list differs from both pure ones
    N, Nz, L = 16, 8, 2 * math.pi
    g = op.Grid(N, N, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - 0.2 * np.exp(-((X - 3) ** 2 + (Y - 3) ** 2))
    ea = 0.05 * np.cos(X)
    levels = pmg.build_levels(N, N, Nz, L, h, ea, ea, coarsest_max=64)
    r = np.random.default_rng(1).standard_normal(g.shape)
    nl = len(levels)
    dref = float(h.min())
    for kind in ("jacobi", "spectral"):
        a = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 1, 1, kind, 0.4, "inject", 1.0, dref)
        b = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 1, 1, [kind] * nl, 0.4, "inject", 1.0, dref)
        assert np.array_equal(a, b)
    mixed = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 1, 1, ["spectral"] + ["jacobi"] * (nl - 1), 0.4,
                       "inject", 1.0, dref)
    for kind in ("jacobi", "spectral"):
        pure = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 1, 1, kind, 0.4, "inject", 1.0, dref)
        assert np.abs(mixed - pure).max() > 1e-6 * np.abs(pure).max()
