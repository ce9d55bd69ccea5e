"""Grids, differentiation and modal transforms (paper Sec. 3.4-3.6).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper used here:

* Fourier grid (Sec. 3.4): the printed nodes 2*pi*n/(N+1), n=0..N are read as
  the even-count periodic grid x_j = j*L/Nx, j=0..Nx-1, with wavenumbers
  kappa_n = 2*pi*n/L, n = -Nx/2+1..Nx/2.  The first derivative multiplies the
  Nyquist coefficient by zero, so every derivative maps real data to real data.
* CGL grid (Sec. 3.4): the printed cos(m*pi/(M+1)) is read as the standard
  Chebyshev-Gauss-Lobatto nodes xi_m = cos(m*pi/Nz), m=0..Nz; sigma = (xi+1)/2
  so m=0 is the free surface (sigma=1) and m=Nz the bottom (sigma=0).
* Chebyshev derivative recursion (Sec. 3.5, Eq. chebDeriv): the printed start
  index is off by one; the standard backward recursion b_{M}=b_{M+1}=0,
  b_{q-1} = (b_{q+1} + 2 q a_q)/c_{q-1}, q = M..1, c_0 = 2 is used.
* Exponential filter (Sec. 3.6): the printed exp(+alpha ...) with alpha=36
  would amplify; the damping sign exp(-alpha ((i-Nc)/(N+1-Nc))^s) is used.
  Chebyshev: i=m, N=Nz, Nc=floor(0.9 Nz).  Fourier: i=|n|, N=Nx/2,
  Nc=floor(Nx/4) (the printed Nc=0.5 Nx would filter nothing).
"""

import numpy as np


# ---------------------------------------------------------------- Fourier (x, y)

def fourier_nodes(N, L):
    """Periodic equispaced nodes x_j = j L / N (Sec. 3.4, even-N reading)."""
    return np.arange(N, dtype=np.float64) * (L / N)


def fourier_wavenumbers(N, L):
    """Wavenumbers kappa_n = 2 pi n / L (Sec. 3.4) in numpy FFT order (n = 0, 1, .., -1)."""
    return 2.0 * np.pi * np.fft.fftfreq(N, d=1.0 / N) / L


def fourier_derivative(f, L, axis, order=1):
    """D^order f along ``axis``: F^{-1}( (i kappa)^order F(f) ) (Sec. 3.5).

    The Nyquist coefficient is multiplied by zero at every application, so
    ``order=2`` equals two applications of the first derivative (that is how
    the second x-derivative arises inside the composite operator).
    """
    N = f.shape[axis]
    if N == 1:
        return np.zeros_like(f)
    kap = fourier_wavenumbers(N, L)
    mult = 1j * kap
    if N % 2 == 0:
        mult[N // 2] = 0.0
    mult = mult ** order
    shape = [1] * f.ndim
    shape[axis] = N
    fh = np.fft.fft(f, axis=axis)
    return np.real(np.fft.ifft(fh * mult.reshape(shape), axis=axis))


def fourier_diff_matrix(N, L):
    """Dense first-derivative matrix of the periodic grid (Sec. 3.5, closed form).

    D_ij = 1/2 (-1)^(i-j) cot((i-j) h / 2), D_ii = 0, h = 2 pi / N, scaled by
    2 pi / L.  For even N this is exactly the spectral derivative with the
    Nyquist coefficient set to zero.
    """
    h = 2.0 * np.pi / N
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    k = i - j
    D = np.zeros((N, N))
    off = k != 0
    D[off] = 0.5 * ((-1.0) ** k[off]) / np.tan(k[off] * h / 2.0)
    return D * (2.0 * np.pi / L)


def fourier_resample(f, Nout, axis):
    """Spectral transfer along a periodic axis (Sec. 4.2).

    Restriction (Nout < N): FFT, keep |n| < Nout/2 (the coarse Nyquist is
    dropped), inverse FFT on Nout points.  Prolongation (Nout > N): FFT, keep
    |n| < N/2 (the fine-side Nyquist of the coarse grid is dropped), zero-pad,
    inverse FFT on Nout points.  Values are interpolation-preserving: a trig
    polynomial with |n| < min(N, Nout)/2 keeps its nodal values.
    """
    N = f.shape[axis]
    if Nout == N:
        return f.copy()
    fh = np.fft.fft(f, axis=axis)
    n_in = np.fft.fftfreq(N, d=1.0 / N)
    keep = np.abs(n_in) < min(N, Nout) / 2.0
    n_out = np.fft.fftfreq(Nout, d=1.0 / Nout)
    shape_out = list(f.shape)
    shape_out[axis] = Nout
    gh = np.zeros(shape_out, dtype=np.complex128)
    # map each kept input mode n to the output slot with the same n
    src = np.nonzero(keep)[0]
    dst = np.array([int(np.nonzero(n_out == n_in[s])[0][0]) for s in src])
    sl_src = [slice(None)] * f.ndim
    sl_dst = [slice(None)] * f.ndim
    sl_src[axis] = src
    sl_dst[axis] = dst
    gh[tuple(sl_dst)] = fh[tuple(sl_src)]
    return np.real(np.fft.ifft(gh, axis=axis)) * (Nout / N)


def fourier_filter(f, axis, alpha=36.0, s=2):
    """Exponential cut-off filter on the Fourier modes along ``axis`` (Sec. 3.6)."""
    N = f.shape[axis]
    if N < 4:
        return f.copy()
    n = np.abs(np.fft.fftfreq(N, d=1.0 / N))
    resp = filter_response(n, N // 2, N // 4, alpha, s)
    shape = [1] * f.ndim
    shape[axis] = N
    return np.real(np.fft.ifft(np.fft.fft(f, axis=axis) * resp.reshape(shape), axis=axis))


def filter_response(i, N, Nc, alpha=36.0, s=2):
    """F_S(i, Nc, alpha, s) of Sec. 3.6 (damping sign): 1 for i <= Nc,
    exp(-alpha ((i-Nc)/(N+1-Nc))^s) above."""
    i = np.asarray(i, dtype=np.float64)
    out = np.ones_like(i)
    hi = i > Nc
    out[hi] = np.exp(-alpha * ((i[hi] - Nc) / (N + 1.0 - Nc)) ** s)
    return out


# ------------------------------------------------------------ Chebyshev (sigma)

def cgl_xi(Nz):
    """CGL nodes xi_m = cos(m pi / Nz), m = 0..Nz (xi_0 = 1) (Sec. 3.4, as read)."""
    return np.cos(np.pi * np.arange(Nz + 1) / Nz)


def cgl_sigma(Nz):
    """sigma_m = (xi_m + 1)/2 in [0, 1] (Sec. 3.4); m = 0 is the free surface."""
    return 0.5 * (cgl_xi(Nz) + 1.0)


def cheb_diff_matrix_xi(Nz):
    """Textbook CGL differentiation matrix on [-1, 1] (Sec. 3.5).

    D_ij = (c_i / c_j) (-1)^(i+j) / (xi_i - xi_j) for i != j, c_0 = c_Nz = 2,
    else 1; the diagonal is the negative row sum (exact on constants).
    """
    x = cgl_xi(Nz)
    c = np.ones(Nz + 1)
    c[0] = c[-1] = 2.0
    i = np.arange(Nz + 1)[:, None]
    j = np.arange(Nz + 1)[None, :]
    sign = (-1.0) ** (i + j)
    X = x[:, None] - x[None, :]
    D = np.zeros((Nz + 1, Nz + 1))
    off = i != j
    D[off] = ((c[:, None] / c[None, :]) * sign)[off] / X[off]
    D[np.diag_indices(Nz + 1)] = -D.sum(axis=1)
    return D


def cheb_diff_matrix_sigma(Nz):
    """d/dsigma on the CGL nodes (Sec. 3.5): sigma = (xi+1)/2, so D_sigma = 2 D_xi."""
    return 2.0 * cheb_diff_matrix_xi(Nz)


def cheb_T(m, xi):
    """T_m(xi) = cos(m arccos xi) (Sec. 3.4)."""
    return np.cos(m * np.arccos(np.clip(xi, -1.0, 1.0)))


def cheb_vandermonde(Nz, xi=None):
    """V[j, m] = T_m(xi_j) (Sec. 3.4 basis) on the given points (default: the CGL nodes)."""
    if xi is None:
        xi = cgl_xi(Nz)
    m = np.arange(Nz + 1)[None, :]
    return cheb_T(m, np.asarray(xi)[:, None])


def cheb_nodal_to_modal(f, axis=0):
    """Modal Chebyshev coefficients (Sec. 3.4) from CGL nodal values (V^{-1} f)."""
    Nz = f.shape[axis] - 1
    V = cheb_vandermonde(Nz)
    fm = np.moveaxis(f, axis, 0)
    a = np.linalg.solve(V, fm.reshape(Nz + 1, -1)).reshape(fm.shape)
    return np.moveaxis(a, 0, axis)


def cheb_modal_to_nodal(a, axis=0):
    Nz = a.shape[axis] - 1
    V = cheb_vandermonde(Nz)
    am = np.moveaxis(a, axis, 0)
    f = (V @ am.reshape(Nz + 1, -1)).reshape(am.shape)
    return np.moveaxis(f, 0, axis)


def cheb_modal_derivative(a):
    """d/dxi of a Chebyshev series by the backward recursion of Eq. (chebDeriv).

    b_M = b_{M+1} = 0;  for q = M..1:  b_{q-1} = (b_{q+1} + 2 q a_q) / c_{q-1},
    c_0 = 2, c_q = 1 otherwise.  ``a`` holds a_0..a_M along axis 0.
    """
    a = np.asarray(a, dtype=np.float64)
    M = a.shape[0] - 1
    b = np.zeros((M + 2,) + a.shape[1:])
    for q in range(M, 0, -1):
        c = 2.0 if q - 1 == 0 else 1.0
        b[q - 1] = (b[q + 1] + 2.0 * q * a[q]) / c
    return b[: M + 1]


def cheb_restrict_matrix(Nz_f, Nz_c):
    """Chebyshev truncation Nz_f -> Nz_c (Sec. 4.2): modes m <= Nz_c kept,
    evaluated on the coarse CGL nodes.  Shape (Nz_c+1, Nz_f+1)."""
    Vf_inv = np.linalg.inv(cheb_vandermonde(Nz_f))
    return cheb_vandermonde(Nz_f, cgl_xi(Nz_c))[:, : Nz_c + 1] @ Vf_inv[: Nz_c + 1, :]


def cheb_prolong_matrix(Nz_c, Nz_f):
    """Chebyshev zero-padding Nz_c -> Nz_f (Sec. 4.2): the coarse interpolant
    evaluated on the fine CGL nodes.  Shape (Nz_f+1, Nz_c+1)."""
    Vc_inv = np.linalg.inv(cheb_vandermonde(Nz_c))
    return cheb_vandermonde(Nz_c, cgl_xi(Nz_f)) @ Vc_inv


def cheb_filter_matrix(Nz, alpha=36.0, s=2):
    """Nodal matrix of the Chebyshev exponential filter (Sec. 3.6): V diag(F_S(m)) V^{-1}."""
    V = cheb_vandermonde(Nz)
    resp = filter_response(np.arange(Nz + 1), Nz, int(np.floor(0.9 * Nz)), alpha, s)
    return V @ np.diag(resp) @ np.linalg.inv(V)
