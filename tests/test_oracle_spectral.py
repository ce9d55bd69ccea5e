"""Pins of the oracle's grids, derivatives, transfers and filter against closed
forms (paper Sec. 3.4-3.6, 4.2).  CPU only."""

import math

import numpy as np
import pytest

from oracle import spectral as sp


@pytest.mark.parametrize("N,L", [(8, 2 * math.pi), (32, 32.0), (64, 7.3)])
def test_fourier_derivative_exact_on_trig_polynomials(N, L):
    x = sp.fourier_nodes(N, L)
    rng = np.random.default_rng(1)
    f = np.zeros(N)
    df = np.zeros(N)
    for n in range(0, N // 2):                     # |n| < N/2: resolved exactly
        a, b = rng.standard_normal(2)
        k = 2 * math.pi * n / L
        f += a * np.cos(k * x) + b * np.sin(k * x)
        df += -a * k * np.sin(k * x) + b * k * np.cos(k * x)
    scale = max(1.0, np.abs(df).max())
    assert np.abs(sp.fourier_derivative(f, L, axis=0) - df).max() < 1e-12 * scale * N
    D = sp.fourier_diff_matrix(N, L)
    assert np.abs(D @ f - df).max() < 1e-12 * scale * N


def test_fourier_nyquist_is_annihilated():
    N, L = 16, 2 * math.pi
    nyq = (-1.0) ** np.arange(N)
    assert np.abs(sp.fourier_derivative(nyq, L, axis=0)).max() < 1e-13
    assert np.abs(sp.fourier_diff_matrix(N, L) @ nyq).max() < 1e-12
    # second derivative as D(D f): the Nyquist mode stays annihilated
    assert np.abs(sp.fourier_derivative(nyq, L, axis=0, order=2)).max() < 1e-13


def test_fourier_matrix_matches_fft_third_witness():
    N, L = 24, 5.0
    f = np.random.default_rng(2).standard_normal(N)
    k = 2 * math.pi * np.fft.fftfreq(N, 1.0 / N) / L
    k[N // 2] = 0
    ref = np.real(np.fft.ifft(1j * k * np.fft.fft(f)))
    assert np.abs(sp.fourier_diff_matrix(N, L) @ f - ref).max() < 1e-12


def test_cgl_nodes_endpoints_and_order():
    s = sp.cgl_sigma(16)
    assert s[0] == 1.0 and abs(s[-1]) < 1e-16
    assert np.all(np.diff(s) < 0)


@pytest.mark.parametrize("Nz", [2, 5, 16, 24])
def test_cheb_derivative_exact_on_polynomials(Nz):
    s = sp.cgl_sigma(Nz)
    D = sp.cheb_diff_matrix_sigma(Nz)
    for deg in range(Nz + 1):
        f = s ** deg
        df = deg * s ** (deg - 1) if deg > 0 else np.zeros_like(s)
        assert np.abs(D @ f - df).max() < 1e-11 * max(1, deg) ** 2 * Nz ** 2 / 16


def test_cheb_derivative_of_T_n_closed_form():
    # T_n'(xi) = n U_{n-1}(xi); at xi = 1: n^2, at xi = -1: (-1)^(n+1) n^2
    Nz = 12
    D = sp.cheb_diff_matrix_xi(Nz)
    xi = sp.cgl_xi(Nz)
    for n in range(Nz + 1):
        d = D @ sp.cheb_T(n, xi)
        assert abs(d[0] - n * n) < 1e-10
        assert abs(d[-1] - (-1) ** (n + 1) * n * n) < 1e-10


def test_modal_recursion_matches_nodal_matrix():
    # reading of Eq. (chebDeriv): standard backward recursion
    Nz = 20
    rng = np.random.default_rng(3)
    f = rng.standard_normal(Nz + 1)
    a = sp.cheb_nodal_to_modal(f)
    b = sp.cheb_modal_derivative(a)
    via_recursion = sp.cheb_modal_to_nodal(b)
    via_matrix = sp.cheb_diff_matrix_xi(Nz) @ f
    assert np.abs(via_recursion - via_matrix).max() < 1e-10 * np.abs(via_matrix).max()
    # T_2 -> 4 T_1 and T_3 -> 3 T_0 + 6 T_2 (textbook)
    assert np.allclose(sp.cheb_modal_derivative(np.array([0, 0, 1.0])), [0, 4, 0])
    assert np.allclose(sp.cheb_modal_derivative(np.array([0, 0, 0, 1.0])), [3, 0, 6, 0])


def test_fourier_resample_preserves_resolved_modes_and_drops_nyquist():
    L = 2 * math.pi
    xf, xc = sp.fourier_nodes(32, L), sp.fourier_nodes(16, L)
    f = lambda x: 1 + np.cos(3 * x) - 0.5 * np.sin(7 * x)
    assert np.abs(sp.fourier_resample(f(xf), 16, 0) - f(xc)).max() < 1e-13
    assert np.abs(sp.fourier_resample(f(xc), 32, 0) - f(xf)).max() < 1e-13
    # the coarse Nyquist (n = 8) and everything above are removed by restriction
    g = np.cos(8 * xf) + np.cos(11 * xf)
    assert np.abs(sp.fourier_resample(g, 16, 0)).max() < 1e-13
    # restriction after prolongation is the identity on the coarse space minus Nyquist
    c = np.random.default_rng(4).standard_normal(16)
    c_nonyq = sp.fourier_resample(sp.fourier_resample(c, 8, 0), 16, 0)  # some smooth vector
    assert np.abs(sp.fourier_resample(sp.fourier_resample(c_nonyq, 32, 0), 16, 0) - c_nonyq).max() < 1e-13


def test_chebyshev_transfers_preserve_polynomials():
    Nf, Nc = 24, 12
    R = sp.cheb_restrict_matrix(Nf, Nc)
    P = sp.cheb_prolong_matrix(Nc, Nf)
    sf, sc = sp.cgl_sigma(Nf), sp.cgl_sigma(Nc)
    for deg in range(Nc + 1):
        assert np.abs(R @ sf ** deg - sc ** deg).max() < 1e-12
        assert np.abs(P @ sc ** deg - sf ** deg).max() < 1e-12
    assert np.abs(R @ P - np.eye(Nc + 1)).max() < 1e-12
    # a mode above the coarse order is removed by restriction
    T = sp.cheb_T(Nc + 3, sp.cgl_xi(Nf))
    assert np.abs(R @ T).max() < 1e-12


def test_filter_response():
    N, Nc = 24, 21
    r = sp.filter_response(np.arange(N + 1), N, Nc)
    assert np.all(r[: Nc + 1] == 1.0)
    assert np.all(np.diff(r[Nc:]) < 0)
    assert abs(r[N] - math.exp(-36 * ((N - Nc) / (N + 1 - Nc)) ** 2)) < 1e-15
    # Chebyshev filter matrix leaves polynomials of degree <= Nc unchanged
    F = sp.cheb_filter_matrix(N)
    s = sp.cgl_sigma(N)
    assert np.abs(F @ s ** 7 - s ** 7).max() < 1e-12
    # Fourier filter: modes |n| <= Nx/4 untouched, Nyquist damped by exp(-36 (...)^2)
    Nx = 32
    x = sp.fourier_nodes(Nx, 2 * math.pi)
    assert np.abs(sp.fourier_filter(np.cos(8 * x), 0) - np.cos(8 * x)).max() < 1e-13
    damp = sp.fourier_filter(np.cos(16 * x), 0) / np.cos(16 * x)
    assert np.allclose(damp, math.exp(-36 * ((16 - 8) / (16 + 1 - 8)) ** 2))
