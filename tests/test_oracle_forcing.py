"""Pin of the oracle's nonlinear momentum forcing (paper Eq. forc1, sigmom1,
1_Scoef, kinematicFS) against closed-form physical-coordinate advection.

For a velocity field given in physical coordinates, Q(x, y, z), sampled on the
sigma grid of a curved bottom h and a curved free surface eta, the sigma-frame
time derivative of the advection-only equation dQ/dt = -(u Q_x + v Q_y + w Q_z)
is

    q_t|sigma = -(u Q_x + v Q_y + w Q_z) - sigma_t q_sigma,

because z = sigma d - h moves with the surface: q_t|sigma = Q_t + Q_z sigma
eta_t and sigma_t = -sigma eta_t / d.  With eta_t = f_eta = -u~ eta_x - v~
eta_y + w~ (the surface values) and q_sigma = d Q_z, every term on the right
is closed form.  The oracle's forcing computes the same quantity through its
spectral derivatives and the metric (h_x - sigma d_x) / d, 1 / d, plus the
hydrostatic surface slope -g (eta_x, eta_y, 0).  The fields are entire
functions of (x, y, sigma) with band-limited h and eta, so the spectral
derivatives are exact to rounding at the sizes used.  CPU only.
"""

import math

import numpy as np
import pytest

from oracle import operator as op
from oracle import rk

KX, KY, A_U, A_W, A_V = 1.0, 1.0, 0.7, 0.5, 0.4


def _fields(X, Y, Z, three_d):
    """u, v, w and their physical x, y, z derivatives (closed form)."""
    e = np.exp(KX * Z)
    cy, sy = (np.cos(KY * Y), np.sin(KY * Y)) if three_d else (np.ones_like(Y), np.zeros_like(Y))
    u = A_U * np.sin(KX * X) * e * cy
    w = A_W * np.cos(KX * X) * e * cy + 0.3 * Z
    v = A_V * np.cos(KX * X) * e * sy if three_d else np.zeros_like(X)
    du = (A_U * KX * np.cos(KX * X) * e * cy,
          -A_U * np.sin(KX * X) * e * KY * sy if three_d else np.zeros_like(X),
          A_U * KX * np.sin(KX * X) * e * cy)
    dw = (-A_W * KX * np.sin(KX * X) * e * cy,
          -A_W * np.cos(KX * X) * e * KY * sy if three_d else np.zeros_like(X),
          A_W * KX * np.cos(KX * X) * e * cy + 0.3)
    if three_d:
        dv = (-A_V * KX * np.sin(KX * X) * e * sy,
              A_V * np.cos(KX * X) * e * KY * cy,
              A_V * KX * np.cos(KX * X) * e * sy)
    else:
        dv = (np.zeros_like(X),) * 3
    return (u, v, w), (du, dv, dw)


def _setup(Nx, Ny, Nz):
    L = 2 * math.pi
    g = op.Grid(Nx, Ny, Nz, L)
    X2, Y2 = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - 0.2 * np.cos(X2 + 0.4) + (0.1 * np.sin(Y2) if Ny > 1 else 0.0)
    eta = 0.15 * np.cos(2 * X2 + 0.3) + 0.05 * np.sin(X2) + (0.08 * np.cos(Y2 - 0.2) if Ny > 1 else 0.0)
    ex = -0.3 * np.sin(2 * X2 + 0.3) + 0.05 * np.cos(X2)
    ey = -0.08 * np.sin(Y2 - 0.2) if Ny > 1 else np.zeros_like(X2)
    d = h + eta
    s = g.sigma[:, None, None]
    Z = s * d[None] - h[None]
    X = np.broadcast_to(X2[None], g.shape)
    Y = np.broadcast_to(Y2[None], g.shape)
    return g, L, h, eta, ex, ey, d, s, X, Y, Z


def _closed_form(Nx, Ny, Nz, grav):
    g, L, h, eta, ex, ey, d, s, X, Y, Z = _setup(Nx, Ny, Nz)
    (u, v, w), derivs = _fields(X, Y, Z, Ny > 1)
    f_eta = -u[0] * ex - v[0] * ey + w[0]                      # Eq. kinematicFS
    sig_t = -s * (f_eta / d)[None]                             # Eq. 1_Scoef, d_t = eta_t
    F = []
    terms = {}
    for i, (q, (qx, qy, qz)) in enumerate(zip((u, v, w), derivs)):
        adv = -(u * qx + v * qy + w * qz)
        moving = -sig_t * (d[None] * qz)                       # -sigma_t q_sigma
        hyd = -grav * (ex if i == 0 else ey if i == 1 else np.zeros_like(ex))[None]
        F.append(adv + moving + hyd)
        terms[i] = (adv, moving, hyd)
    return g, h, eta, (u, v, w), f_eta, F, terms


@pytest.mark.parametrize("three_d", [False, True])
def test_forcing_matches_closed_form_advection(three_d):
    Ny = 16 if three_d else 1
    g, h, eta, (u, v, w), f_eta_ref, F_ref, terms = _closed_form(32, Ny, 20, 9.81)
    tank = rk.Tank(32, Ny, 20, 2 * math.pi, h, g=9.81)
    st = rk.State(g, eta, u, v, w)
    geo_b = op.Geometry(g, h, st.eta)
    f_eta, F = rk.forcing(tank, geo_b, st)
    assert np.abs(f_eta - f_eta_ref).max() <= 1e-12 * np.abs(f_eta_ref).max()
    comps = (0, 1, 2) if three_d else (0, 2)
    for i in comps:
        scale = np.abs(F_ref[i]).max()
        assert np.abs(F[i] - F_ref[i]).max() <= 1e-10 * scale, i
    # every term is large enough that flipping its sign, or dropping it,
    # moves F far outside the tolerance (the test is sensitive to each)
    for i in comps:
        scale = np.abs(F_ref[i]).max()
        for name, t in zip(("advection", "moving sigma", "hydrostatic"), terms[i]):
            if name == "hydrostatic" and i == 2:
                continue
            assert np.abs(t).max() > 1e-2 * scale, (i, name)


@pytest.mark.parametrize("mistake", ["sigma_t sign", "sigma_x sign", "drop v sigma_y", "sigma_z sign"])
def test_forcing_pin_detects_planted_mistakes(mistake):
    """A mistake planted in the oracle's forcing (on the CPU) fails the pin."""
    three_d = mistake == "drop v sigma_y"
    Ny = 8 if three_d else 1
    g, h, eta, (u, v, w), _, F_ref, _ = _closed_form(32, Ny, 16, 9.81)
    tank = rk.Tank(32, Ny, 16, 2 * math.pi, h, g=9.81)
    st = rk.State(g, eta, u, v, w)
    geo_b = op.Geometry(g, h, st.eta)
    if mistake == "sigma_t sign":
        geo_b.d = -geo_b.d            # only sigma_t reads d directly in the forcing
    elif mistake == "sigma_x sign":
        geo_b.sx = -geo_b.sx
    elif mistake == "drop v sigma_y":
        geo_b.sy = np.zeros_like(geo_b.sy)
    elif mistake == "sigma_z sign":
        geo_b.sz = -geo_b.sz
    _, F = rk.forcing(tank, geo_b, st)
    err = max(np.abs(F[i] - F_ref[i]).max() / np.abs(F_ref[i]).max() for i in (0, 2))
    assert err > 1e-4


def test_forcing_spectral_convergence_in_nz():
    """The pin is a limit, not a coincidence: the error decays spectrally in Nz."""
    errs = []
    for Nz in (4, 6, 8):
        g, h, eta, (u, v, w), _, F_ref, _ = _closed_form(32, 1, Nz, 9.81)
        tank = rk.Tank(32, 1, Nz, 2 * math.pi, h, g=9.81)
        st = rk.State(g, eta, u, v, w)
        _, F = rk.forcing(tank, op.Geometry(g, h, st.eta), st)
        errs.append(np.abs(F[0] - F_ref[0]).max())
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-2 * errs[1]


def test_viscous_term_is_the_physical_laplacian():
    # q = sin(x) z^2 with z = sigma d - h on a curved, moving geometry: the
    # composite Div_b Grad_b q must equal the physical Laplacian
    # (2 - z^2) sin(x) at every node (q is band-limited in x and quadratic in
    # sigma, so the discrete derivatives are exact to rounding)
    g, L, h, eta, ex, ey, d, s, X, Y, Z = _setup(32, 1, 12)
    q = np.sin(X) * Z ** 2
    geo = op.Geometry(g, h, eta)
    lap = op.div(g, geo, op.grad(g, geo, q))
    want = (2.0 - Z ** 2) * np.sin(X)
    assert np.abs(lap - want).max() <= 1e-10 * np.abs(want).max()
    # in the forcing it enters with the factor nu and the stress-free surface
    # (no vertical flux on the surface nodes): for q2 = sin(x) (z - eta)^2,
    # whose z-derivative vanishes at the surface, that is again the physical
    # Laplacian, -sin(x) s^2 - 4 cos(x) s eta_x + 2 sin(x) eta_x^2
    # - 2 sin(x) s eta_xx + 2 sin(x) with s = z - eta
    tank0 = rk.Tank(32, 1, 12, L, h, g=9.81)
    tank1 = rk.Tank(32, 1, 12, L, h, g=9.81, nu=0.3)
    S = Z - eta[None]
    exx = (-0.6 * np.cos(2 * X[0] + 0.3) - 0.05 * np.sin(X[0]))[None]
    q2 = np.sin(X) * S ** 2
    want2 = (-np.sin(X) * S ** 2 - 4 * np.cos(X) * S * ex[None] + 2 * np.sin(X) * ex[None] ** 2
             - 2 * np.sin(X) * S * exx + 2 * np.sin(X))
    st = rk.State(g, eta, q2, np.zeros_like(q2), np.zeros_like(q2))
    _, F0 = rk.forcing(tank0, geo, st)
    _, F1 = rk.forcing(tank1, geo, st)
    assert np.abs((F1[0] - F0[0]) - 0.3 * want2).max() <= 1e-10 * 0.3 * np.abs(want2).max()
    # the stress-free reading changes the term when the surface flux is not zero
    st = rk.State(g, eta, q, np.zeros_like(q), np.zeros_like(q))
    _, F0 = rk.forcing(tank0, geo, st)
    _, F1 = rk.forcing(tank1, geo, st)
    assert np.abs((F1[0] - F0[0]) - 0.3 * want).max() > 1e-3 * 0.3 * np.abs(want).max()


def test_viscous_stage_is_no_slip_and_relaxation_weights():
    Nx, Nz, L = 32, 10, 2 * math.pi
    g = op.Grid(Nx, 1, Nz, L)
    h = np.ones((1, Nx))
    eta = 0.01 * np.cos(g.x)[None]
    u = np.broadcast_to(0.05 * np.cos(g.x)[None, None, :], g.shape).copy()
    w = np.zeros(g.shape)
    tank = rk.Tank(Nx, 1, Nz, L, h, nu=1e-3, solver="dense")
    st = rk.State(g, eta, u, np.zeros_like(u), w)
    rk.stage(tank, st, 1, 1e-3)
    assert np.all(st.u[-1] == 0.0) and np.all(st.w[-1] == 0.0) and np.all(st.Ku[-1] == 0.0)
    assert np.abs(st.u[0]).max() > 0.04
    x = np.linspace(0.0, 4.0, 401)
    wg = rk.relaxation_weight(x, 1.0, 3.0)
    assert wg[x < 1.0].max() == 0.0 and wg[x > 3.0].max() == 0.0
    assert abs(wg[100]) < 1e-15 and abs(wg[300] - 1.0) < 1e-15
    inside = wg[(x >= 1.0) & (x <= 3.0)]
    assert np.all(np.diff(inside) >= 0.0)
    assert np.allclose(rk.relaxation_weight(x, 3.0, 1.0), rk.relaxation_weight(4.0 - x, 1.0, 3.0))
