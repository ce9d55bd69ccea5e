"""Seeded synthetic wave-tank inputs shared by the oracle tests, the GPU tests
and the benchmark.

This module holds no arithmetic of the numerical method: it draws seeded
random numbers and evaluates closed-form initial data (linear / second-order
Stokes wave theory, a JONSWAP sea, Gaussian bumps) at coordinates that the
caller passes in.  Node coordinates (x, y, z) always come from the caller's
own grid.  Random streams are numpy ``Generator(PCG64(seed))``.

The paper's own workloads (stream-function waves, the Beji-Battjes bar and
its laboratory data) are not available; these recipes stand in for them:

* ``manufactured``  - flat 2D tank, L = 2 pi, p = cos(x) cosh(z+1) + q with q a
                      seeded 8 x 8 Fourier x Chebyshev series scaled by
                      2^-(n+m) (the Poisson pin of the 64 x 16 workload).
* ``airy``          - small-amplitude linear wave, eta = A cos(k x).
* ``stokes2``       - second-order Stokes surface with linear-theory velocity.
* ``bump``          - h(x) = 1 - A exp(-((x - x0)/w)^2).
* ``jonswap_sea``   - 3D directional sea on the periodic wavenumber lattice.
* ``batch_tanks``   - the 256 uneven 2D tanks of the batched workload.
* ``adjoint_bathymetry`` - random Fourier bathymetry of the gradient workload.
"""

import math

import numpy as np

G = 9.81


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def omega(k, h, g=G):
    """Linear dispersion relation omega^2 = g k tanh(k h) (paper Sec. 5.3)."""
    return math.sqrt(g * k * math.tanh(k * h))


# ----------------------------------------------------------------- manufactured

class Manufactured:
    """p(x, z) = cos(x) cosh(z + 1) + q(x, xi), xi = 2 z + 1 on the flat tank
    z in [-1, 0], L = 2 pi, with
    q = sum_{n,m=0..7} 2^-(n+m) (a_nm cos(n x) + b_nm sin(n x)) T_m(xi),
    a, b ~ N(0, 1) (b_0m = 0).  Laplacian, surface and bottom data in closed form."""

    def __init__(self, seed=0, modes=8):
        r = rng(seed)
        self.a = r.standard_normal((modes, modes))
        self.b = r.standard_normal((modes, modes))
        self.b[0, :] = 0.0
        self.modes = modes
        n = np.arange(modes)[:, None]
        m = np.arange(modes)[None, :]
        self.scale = 2.0 ** (-(n + m))

    def _series(self, x, z, dxo=0, dzo=0):
        from numpy.polynomial import chebyshev as C
        xi = 2.0 * z + 1.0
        out = np.zeros(np.broadcast(x, z).shape)
        for n in range(self.modes):
            if dxo == 0:
                cx, sx = np.cos(n * x), np.sin(n * x)
            elif dxo == 1:
                cx, sx = -n * np.sin(n * x), n * np.cos(n * x)
            else:
                cx, sx = -n * n * np.cos(n * x), -n * n * np.sin(n * x)
            ca = self.a[n] * self.scale[n]
            cb = self.b[n] * self.scale[n]
            if dzo:
                ca = C.chebder(ca, dzo) * (2.0 ** dzo)   # d/dz = 2 d/dxi
                cb = C.chebder(cb, dzo) * (2.0 ** dzo)
            out = out + cx * C.chebval(xi, ca) + sx * C.chebval(xi, cb)
        return out

    def p(self, x, z):
        return np.cos(x) * np.cosh(z + 1.0) + self._series(x, z)

    def laplacian(self, x, z):
        return self._series(x, z, dxo=2) + self._series(x, z, dzo=2)

    def dpdz(self, x, z):
        return np.cos(x) * np.sinh(z + 1.0) + self._series(x, z, dzo=1)


# ------------------------------------------------------------------ wave theory

def airy(x, z, A=0.005, k=1.0, h=1.0, g=G):
    """Linear (Airy) wave at t = 0: eta = A cos(kx), u, w from potential theory."""
    w_ = omega(k, h, g)
    eta = A * np.cos(k * x)
    if z is None:
        return eta
    u = A * w_ * np.cosh(k * (z + h)) / np.sinh(k * h) * np.cos(k * x)
    w = A * w_ * np.sinh(k * (z + h)) / np.sinh(k * h) * np.sin(k * x)
    return eta, u, w


def stokes2_eta(x, a, k, h):
    """Second-order Stokes surface a cos kx + (k a^2/4) cosh kh (2 + cosh 2kh)/sinh^3 kh cos 2kx."""
    c2 = k * a * a / 4.0 * math.cosh(k * h) * (2.0 + math.cosh(2 * k * h)) / math.sinh(k * h) ** 3
    return a * np.cos(k * x) + c2 * np.cos(2 * k * x)


def linear_velocity(x, z, a, k, h, g=G):
    w_ = omega(k, h, g)
    u = a * w_ * np.cosh(k * (z + h)) / np.sinh(k * h) * np.cos(k * x)
    w = a * w_ * np.sinh(k * (z + h)) / np.sinh(k * h) * np.sin(k * x)
    return u, w


def bump(x, L, A, width):
    return 1.0 - A * np.exp(-(((x - L / 2.0) / width) ** 2))


def nonlinear_2d_tank():
    """The 1024 x 24 nonlinear tank: L = 32, Stokes-2 wave with 5 wavelengths in
    the domain (kh = 0.982 at the deep end, the periodic wavenumber nearest
    kh = 1), H/L = 0.04, bump h = 1 - 0.5 exp(-((x-16)/2)^2), dt = 0.5 dx /
    sqrt(g h_max)."""
    L, Nx, Nz = 32.0, 1024, 24
    k = 2.0 * math.pi * 5 / L
    H = 0.04 * 2.0 * math.pi / k
    dt = 0.5 * (L / Nx) / math.sqrt(G * 1.0)
    return dict(L=L, Nx=Nx, Nz=Nz, k=k, a=H / 2.0, h0=1.0, bump_A=0.5, bump_w=2.0, dt=dt,
                steps=2000)


def nonlinear_2d_initial(x, z, p):
    """eta(x) and (u, w)(x, z) of ``nonlinear_2d_tank``; z = node depths from the caller."""
    eta = stokes2_eta(x, p["a"], p["k"], p["h0"])
    if z is None:
        return eta
    u, w = linear_velocity(x, z, p["a"], p["k"], p["h0"])
    return eta, u, w


# ---------------------------------------------------------------- 3D JONSWAP sea

def jonswap_sea(seed=2, L=64.0, ncomp=4096, kp=1.5, gamma=3.3, s=10, hs_over_lp=0.02,
                h=1.0, g=G):
    """Lattice components (kx, ky, amplitude, phase) of a directional JONSWAP sea.

    Lattice points kappa = 2 pi (n, m)/L with |kappa| in [0.5, 2.5] kp, seeded
    shuffle, first ``ncomp``; S = JONSWAP(omega(|kappa|)) cos^{2s}(theta/2)
    (mean direction +x); amplitudes sqrt(2 S dk^2) rescaled so that
    Hs = 4 sqrt(sum a^2 / 2) = hs_over_lp * 2 pi / kp; phases U[0, 2 pi).
    """
    r = rng(seed)
    dk = 2.0 * math.pi / L
    nmax = int(math.ceil(2.5 * kp / dk)) + 1
    n = np.arange(-nmax, nmax + 1)
    NX, NY = np.meshgrid(n, n, indexing="xy")
    KX, KY = NX * dk, NY * dk
    K = np.hypot(KX, KY)
    sel = (K >= 0.5 * kp) & (K <= 2.5 * kp)
    idx = np.nonzero(sel.ravel())[0]
    idx = idx[r.permutation(idx.size)][:ncomp]
    kx, ky, kk = KX.ravel()[idx], KY.ravel()[idx], K.ravel()[idx]
    om = np.sqrt(g * kk * np.tanh(kk * h))
    omp = math.sqrt(g * kp * math.tanh(kp * h))
    sig = np.where(om <= omp, 0.07, 0.09)
    rexp = np.exp(-((om - omp) ** 2) / (2.0 * sig ** 2 * omp ** 2))
    S = g ** 2 / om ** 5 * np.exp(-1.25 * (omp / om) ** 4) * gamma ** rexp
    theta = np.arctan2(ky, kx)
    S = S * np.cos(theta / 2.0) ** (2 * s)
    amp = np.sqrt(2.0 * S * dk * dk)
    hs = hs_over_lp * 2.0 * math.pi / kp
    amp *= hs / (4.0 * math.sqrt(np.sum(amp ** 2) / 2.0))
    phase = r.uniform(0.0, 2.0 * math.pi, size=kx.size)
    return dict(kx=kx, ky=ky, k=kk, amp=amp, phase=phase, omega=om, L=L, h=h)


def jonswap_fields(sea, Nx, sigma):
    """eta (N, N) and linear-theory u, v, w (len(sigma), N, N) on the N x N
    periodic grid, built by summing the lattice components with an inverse FFT.
    The vertical profile is evaluated at z + h = sigma h (still-water mapping)."""
    L, h = sea["L"], sea["h"]
    dk = 2.0 * math.pi / L
    ix = np.rint(sea["kx"] / dk).astype(int) % Nx
    iy = np.rint(sea["ky"] / dk).astype(int) % Nx
    c = sea["amp"] * np.exp(1j * sea["phase"])

    def synth(coef):
        spec = np.zeros((Nx, Nx), dtype=np.complex128)
        np.add.at(spec, (iy, ix), coef)
        return np.real(np.fft.ifft2(spec) * Nx * Nx)

    eta = synth(c)
    k, om = sea["k"], sea["omega"]
    u = np.empty((len(sigma), Nx, Nx))
    v = np.empty_like(u)
    w = np.empty_like(u)
    for m, s in enumerate(sigma):
        ch = np.cosh(k * s * h) / np.sinh(k * h)
        sh = np.sinh(k * s * h) / np.sinh(k * h)
        u[m] = synth(c * om * ch * sea["kx"] / k)
        v[m] = synth(c * om * ch * sea["ky"] / k)
        w[m] = synth(-1j * c * om * sh)
    return eta, u, v, w


# ------------------------------------------------------------ batched 2D tanks

def battjes_limit(kh):
    """Battjes breaking steepness (H/L)_max = 0.1401 tanh(0.8863 kh) (paper Sec. 5.2)."""
    return 0.1401 * math.tanh(0.8863 * kh)


def batch_tanks(n=256, seed=3, safety=0.8):
    """Tank table of the batched workload.  L = 8 wavelengths of k = kh (h = 1);
    a tank whose steepness exceeds ``safety`` x Battjes at the bump-crest depth
    1 - A is redrawn from the same stream (count returned)."""
    r = rng(seed)
    out, redrawn = [], 0
    while len(out) < n:
        Nx = int(r.choice([128, 256, 512, 1024, 2048]))
        Nz = int(r.choice([8, 12, 16, 24, 32]))
        kh = float(r.uniform(0.5, 3.0))
        steep = float(r.uniform(0.005, 0.05))
        A = float(r.uniform(0.0, 0.5))
        k = kh
        L = 8.0 * 2.0 * math.pi / k
        width = float(r.uniform(L / 20.0, L / 8.0))
        if steep > safety * battjes_limit(k * (1.0 - A)):
            redrawn += 1
            continue
        H = steep * 2.0 * math.pi / k
        dt = 0.5 * (L / Nx) / math.sqrt(G * 1.0)
        out.append(dict(Nx=Nx, Nz=Nz, L=L, k=k, a=H / 2.0, h0=1.0, bump_A=A, bump_w=width,
                        dt=dt, steps=500))
    return out, redrawn


# ------------------------------------------------------------ adjoint workload

def adjoint_bathymetry(seed, L=16.0, K=64):
    """b_k ~ N(0, (0.02/k)^2), phi_k ~ U[0, 2 pi), k = 1..K."""
    r = rng(seed)
    kk = np.arange(1, K + 1)
    b = r.standard_normal(K) * (0.02 / kk)
    phi = r.uniform(0.0, 2.0 * math.pi, size=K)
    return b, phi


def fourier_bathymetry(x, b, phi, L=16.0):
    kk = np.arange(1, len(b) + 1)
    return 1.0 + np.sum(b[:, None] * np.cos(2.0 * math.pi * kk[:, None] * x[None, :] / L
                                           + phi[:, None]), axis=0)
