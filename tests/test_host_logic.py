"""Host logic of the library, on the CPU (no GPU, no CUDA call): the
multigrid hierarchy wt_create builds (Sec. 4.1 coarsening, as read for the
oracle) and the stream-function wave solver behind wt_stream_function_wave
(Sec. 5.2 initial condition), through their host-only C-ABI entry points.

The hierarchy is compared with the oracle's coarsening over every grid the
library accepts, and with the level sizes of the benchmark's 1024 x 24 bar.
The stream-function solution is compared with the oracle's (a separate Newton
solve with a central-difference Jacobian) and checked on its own against the
conditions it must satisfy between the collocation nodes."""

import math

import numpy as np
import pytest

from oracle import pmg
from oracle import streamfunction as sf

G = 9.81


@pytest.fixture(scope="module")
def w():
    from paper_2406_00991_gb300 import build
    build.build()
    import paper_2406_00991_gb300 as pkg
    pkg._reload()
    return pkg


def test_levels_for_the_benchmark_bar(w):
    # 1024 x 24 with the default coarsest_max 64: x halves while Nx > Nz,
    # sigma halves while Nz > Nx, until a level has at most 64 unknowns:
    # ten levels down to 8 x 6 (56 unknowns)
    st, dims = w.wt_levels_for(1024, 1, 24, 64)
    assert st == w.WT_OK
    assert dims == [(1024, 1, 24), (512, 1, 24), (256, 1, 24), (128, 1, 24), (64, 1, 24), (32, 1, 24),
                    (16, 1, 24), (16, 1, 12), (8, 1, 12), (8, 1, 6)]
    # the 3D sea, 256 x 256 x 16: both halve at Nx = Nz = 16, then again
    st, dims = w.wt_levels_for(256, 256, 16, 64)
    assert st == w.WT_OK
    assert dims == [(256, 256, 16), (128, 128, 16), (64, 64, 16), (32, 32, 16), (16, 16, 16), (8, 8, 8),
                    (4, 4, 4)]


def test_levels_for_matches_the_oracle_coarsening(w):
    count = unsupported = 0
    for Nx in [2 ** e for e in range(2, 13)]:
        for Ny in (1, 4, 16, 64, 256, 1024):
            for Nz in (2, 3, 4, 5, 7, 8, 12, 16, 17, 20, 24, 31, 32):
                for cmax in (1, 32, 64, 128):
                    st, dims = w.wt_levels_for(Nx, Ny, Nz, cmax)
                    want = pmg.hierarchy(Nx, Ny, Nz, coarsest_max=cmax)
                    nx, ny, nz = want[-1]
                    # a coarsest level the dense FP64 solve cannot take (Ny
                    # far above Nx stops the coarsening early) is reported as
                    # wt_create reports it, with the levels still written
                    big = nx * ny * (nz + 1) > 128
                    assert st == (w.WT_ENOTSUP if big else w.WT_OK), (Nx, Ny, Nz, cmax, w.wt_last_error())
                    assert dims == [tuple(l) for l in want], (Nx, Ny, Nz, cmax)
                    count += 1
                    unsupported += big
    assert count == 11 * 6 * 13 * 4 and 0 < unsupported < count


def test_levels_for_rejects_what_wt_create_rejects(w):
    for args in ((100, 1, 16, 64), (2, 1, 16, 64), (8192, 1, 16, 64), (64, 2, 16, 64), (64, 2048, 16, 64),
                 (64, 1, 1, 64), (64, 1, 33, 64), (64, 1, 16, 0), (64, 1, 16, 129)):
        st, _ = w.wt_levels_for(*args)
        assert st == w.WT_EINVAL, args
    assert "coarsest_max" in w.wt_last_error()[1]


def _battjes_height(kh, frac, k):
    return frac * 0.1401 * math.tanh(0.8863 * kh) * 2 * math.pi / k


CASES = [(0.5, 0.5), (2.0, 0.5), (2 * math.pi, 0.5), (2.0, 0.7)]


@pytest.mark.parametrize("kh,frac", CASES)
def test_stream_function_solve_matches_oracle(w, kh, frac):
    d, N = 1.0, 32
    k = kh / d
    H = _battjes_height(kh, frac, k)
    st, (c, Q, R), B, E = w.wt_stream_function_solve(k, d, H, G, N)
    assert st == w.WT_OK, w.wt_last_error()
    W = sf.solve(k, d, H, g=G, N=N)
    # two Newton solutions (analytic and central-difference Jacobians) of a
    # system whose conditioning grows with the steepness: 1e-10 for moderate
    # waves, 1e-8 at 0.7 x Battjes
    bound = 1e-10 if frac <= 0.5 else 1e-8
    assert abs(c - W.c) <= bound * W.c
    assert abs(Q - W.Q) <= bound * abs(W.Q)
    assert abs(R - W.R) <= bound * abs(W.R)
    assert np.abs(E - W.E).max() <= bound * H
    assert np.abs(B - W.B).max() <= bound * np.abs(W.B).max()


@pytest.mark.parametrize("kh,frac", CASES)
def test_stream_function_solve_satisfies_the_surface_conditions(w, kh, frac):
    # the library's coefficients on their own: between the N + 1 collocation
    # nodes the surface is a streamline of the steady flow in the wave's
    # frame and Bernoulli's constant holds along it; zero mean level, height H
    d, N = 1.0, 32
    k = kh / d
    H = _battjes_height(kh, frac, k)
    st, (c, Q, R), B, E = w.wt_stream_function_solve(k, d, H, G, N)
    assert st == w.WT_OK
    X = (np.arange(200) + 0.37) * (2 * math.pi / k) / 200
    j = np.arange(N + 1)
    eta = np.cos(np.multiply.outer(X, j * k)) @ E
    eta_x = -(np.sin(np.multiply.outer(X, j * k)) * (j * k)) @ E
    y = d + eta
    u = np.zeros_like(X)
    ww = np.zeros_like(X)
    psi = -c * y
    for m in range(1, N + 1):
        jk = m * k
        e1, e2, e3 = np.exp(jk * (y - d)), np.exp(-jk * (y + d)), math.exp(-2 * jk * d)
        sh, ch = (e1 - e2) / (1 + e3), (e1 + e2) / (1 + e3)
        u += jk * B[m - 1] * ch * np.cos(jk * X)
        ww += jk * B[m - 1] * sh * np.sin(jk * X)
        psi += B[m - 1] * sh * np.cos(jk * X)
    scale = c * np.abs(eta_x).max()
    assert np.abs((u - c) * eta_x - ww).max() < 1e-8 * scale          # kinematic
    assert np.abs(psi + Q).max() < 1e-8 * c * d                         # the streamline psi = -Q
    bern = 0.5 * ((u - c) ** 2 + ww ** 2) + G * eta
    assert np.abs(bern - R).max() < 1e-8 * G * H                         # Bernoulli
    assert abs(eta.mean()) < 1e-12 * H
    assert abs(E @ np.ones(N + 1) - E @ np.cos(j * math.pi) - H) < 1e-12 * H


def test_stream_function_solve_linear_limit(w):
    for kh in (0.5, 2.0, 6.0):
        st, (c, _, _), _, E = w.wt_stream_function_solve(kh, 1.0, 1e-5, G, 16)
        assert st == w.WT_OK
        assert abs(c / math.sqrt(G / kh * math.tanh(kh)) - 1.0) < 1e-8
        assert abs(E[1] - 0.5e-5) < 1e-4 * 1e-5


def test_stream_function_solve_rejects(w):
    k = 2.0
    st, *_ = w.wt_stream_function_solve(k, 1.0, _battjes_height(2.0, 0.95, k), G, 32)
    assert st == w.WT_EINVAL and "Battjes" in w.wt_last_error()[1]
    for args in ((k, 1.0, 0.01, G, 1), (k, 1.0, 0.01, G, 129), (0.0, 1.0, 0.01, G, 16), (k, -1.0, 0.01, G, 16),
                 (k, 1.0, 0.0, G, 16), (k, 1.0, 0.01, 0.0, 16)):
        st, *_ = w.wt_stream_function_solve(*args)
        assert st == w.WT_EINVAL, args


SIGMA_CASES = [(Nz, Nzc) for Nz in (2, 3, 4, 6, 8, 12, 16, 17, 24, 32) for Nzc in sorted({2, (Nz + 1) // 2, Nz})
               if 2 <= Nzc <= Nz]


def test_sigma_matrices_match_the_oracle(w):
    from oracle import spectral as sp
    for Nz, Nzc in SIGMA_CASES:
        for bc in (0, 1):
            st, D, F, R, P = w.wt_sigma_matrices(Nz, Nzc, bc)
            assert st == w.WT_OK, w.wt_last_error()
            D0 = sp.cheb_diff_matrix_sigma(Nz)
            assert np.abs(D - D0).max() <= 1e-12 * np.abs(D0).max(), (Nz, "D")
            F0 = sp.cheb_filter_matrix(Nz)
            assert np.abs(F - F0).max() <= 1e-12, (Nz, "F")
            R0 = pmg.restrict_sigma_matrix(Nz, Nzc, "inject" if bc == 0 else "paper")
            assert np.abs(R - R0).max() <= 1e-12, (Nz, Nzc, bc, "R")
            P0 = sp.cheb_prolong_matrix(Nzc, Nz)
            assert np.abs(P - P0).max() <= 1e-12, (Nz, Nzc, "P")


def test_sigma_matrices_on_polynomials(w):
    # independent of the oracle: d/dsigma is exact on polynomials of degree
    # <= Nz; the filter keeps degrees <= floor(0.9 Nz); prolongation then
    # restriction is the identity on the coarse nodes (both forms); the
    # prolongation reproduces a coarse-degree polynomial at the fine nodes
    for Nz, Nzc in SIGMA_CASES:
        st, D, F, R, P = w.wt_sigma_matrices(Nz, Nzc, 0)
        st1, _, _, R1, _ = w.wt_sigma_matrices(Nz, Nzc, 1)
        assert st == st1 == w.WT_OK
        s = 0.5 * (np.cos(np.pi * np.arange(Nz + 1) / Nz) + 1.0)
        sc = 0.5 * (np.cos(np.pi * np.arange(Nzc + 1) / Nzc) + 1.0)
        for deg in range(Nz + 1):
            assert np.abs(D @ s ** deg - deg * s ** max(deg - 1, 0)).max() <= 1e-10 * max(1, deg * deg), (Nz, deg)
        for deg in range(int(np.floor(0.9 * Nz)) + 1):
            assert np.abs(F @ s ** deg - s ** deg).max() <= 1e-12, (Nz, deg)
        assert np.abs(R @ P - np.eye(Nzc + 1)).max() <= 1e-12, (Nz, Nzc)
        assert np.abs(R1 @ P - np.eye(Nzc + 1)).max() <= 1e-12, (Nz, Nzc)
        for deg in range(Nzc + 1):
            assert np.abs(P @ sc ** deg - s ** deg).max() <= 1e-12, (Nz, Nzc, deg)
    assert w.wt_sigma_matrices(33, 8)[0] == w.WT_EINVAL
    assert w.wt_sigma_matrices(16, 17)[0] == w.WT_EINVAL
    assert w.wt_sigma_matrices(16, 1)[0] == w.WT_EINVAL
    assert w.wt_sigma_matrices(16, 8, 2)[0] == w.WT_EINVAL
