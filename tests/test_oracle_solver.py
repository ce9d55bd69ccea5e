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
