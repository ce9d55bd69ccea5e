"""Pins of the oracle's exact step derivative (oracle/adjoint.py): its forward
map against the numpy oracle step, and its gradients against central finite
differences of the numpy oracle (the paper has no adjoint)."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as adj  # noqa: E402
from oracle import operator as op  # noqa: E402
from oracle import rk  # noqa: E402
import seeded_inputs as si  # noqa: E402


def small_tank(Nx=32, Nz=8, L=8.0, seed=1):
    x = np.arange(Nx) * L / Nx
    b, phi = si.adjoint_bathymetry(seed, L=L, K=6)
    h = si.fourier_bathymetry(x, 3 * b, phi, L=L)
    eta = 0.02 * np.cos(2 * math.pi * x / (L / 2)) + 0.01 * np.sin(2 * math.pi * x / L)
    g = op.Grid(Nx, 1, Nz, L)
    geo = op.Geometry(g, h, eta)
    k = 2 * math.pi / (L / 2)
    u, w = si.linear_velocity(x[None, None, :], geo.z_nodes(g), 0.02, k, 1.0)
    return x, h, eta, u[:, 0, :], w[:, 0, :]


def numpy_step(Nx, Nz, L, h, eta, u, w, dt, linear=False, filt=False, nsteps=1):
    T = rk.Tank(Nx, 1, Nz, L, h[None], solver="dense", linear=linear, filter=filt)
    st = rk.State(T.grid, eta[None], u[:, None], np.zeros_like(u)[:, None], w[:, None])
    for _ in range(nsteps):
        rk.step(T, st, dt)
    return st.eta[0], st.u[:, 0], st.w[:, 0]


@pytest.mark.parametrize("kw", [dict(), dict(filt=True), dict(linear=True)])
def test_forward_equals_numpy_oracle(kw):
    Nx, Nz, L = 32, 8, 8.0
    x, h, eta, u, w = small_tank(Nx, Nz, L)
    g = adj.Grid2(Nx, Nz, L)
    dt = 0.02
    e1, u1, w1 = adj.step(g, adj._t(h), adj._t(eta), adj._t(u), adj._t(w), dt, **kw)
    e2, u2, w2 = numpy_step(Nx, Nz, L, h, eta, u, w, dt, linear=kw.get("linear", False),
                            filt=kw.get("filt", False))
    for a, b in ((e1, e2), (u1, u2), (w1, w2)):
        assert np.abs(a.numpy() - b).max() <= 1e-12 * np.abs(b).max()


def test_transposed_operator_dot_product():
    Nx, Nz, L = 16, 6, 4.0
    x, h, eta, _, _ = small_tank(Nx, Nz, L)
    g = adj.Grid2(Nx, Nz, L)
    ma = adj.metric(g, adj._t(h), adj._t(eta))
    mb = adj.metric(g, adj._t(h), adj._t(0.5 * eta))
    r = np.random.default_rng(0)
    X = adj._t(r.standard_normal((Nz + 1, Nx)))
    Y = adj._t(r.standard_normal((Nz + 1, Nx)))
    lhs = torch.sum(adj.apply_A(g, ma, mb, X) * Y).item()
    rhs = torch.sum(X * adj.apply_AT(g, ma, mb, Y)).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the matrix-free torch operator is the numpy oracle's operator
    ref = op.apply_A(op.Grid(Nx, 1, Nz, L), op.Geometry(op.Grid(Nx, 1, Nz, L), h, eta),
                     op.Geometry(op.Grid(Nx, 1, Nz, L), h, 0.5 * eta), X.numpy()[:, None])
    assert np.abs(adj.apply_A(g, ma, mb, X).numpy() - ref[:, 0]).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("kw", [dict(), dict(filt=True), dict(linear=True)])
def test_gauge_loss_gradient_matches_finite_differences(kw):
    Nx, Nz, L = 32, 8, 8.0
    x, h, eta, u, w = small_tank(Nx, Nz, L)
    g = adj.Grid2(Nx, Nz, L)
    dt, nsteps = 0.02, 3
    gauges = np.arange(0, Nx, 8)
    target = 0.01 * np.random.default_rng(3).standard_normal((nsteps, len(gauges)))
    J, gh, ge, gu, gw = adj.loss_and_gradient(g, h, eta, u, w, dt, nsteps, gauges, target, **kw)

    def J_np(hh, ee):
        series = []
        e_, u_, w_ = ee, u, w
        for _ in range(nsteps):
            e_, u_, w_ = numpy_step(Nx, Nz, L, hh, e_, u_, w_, dt, linear=kw.get("linear", False),
                                    filt=kw.get("filt", False))
            series.append(e_[gauges])
        return 0.5 * np.sum((np.array(series) - target) ** 2) * dt

    assert abs(J - J_np(h, eta)) <= 1e-12 * J
    r = np.random.default_rng(5)
    # the h-derivative of a 3-step gauge loss is ~1e-4 of J / |h|: a step of
    # 1e-5 keeps the rounding noise of the differences below 1e-6 of it
    for which, eps in (("h", 1e-5), ("eta", 1e-6)):
        d = r.standard_normal(Nx)
        if which == "h":
            fd = (J_np(h + eps * d, eta) - J_np(h - eps * d, eta)) / (2 * eps)
            ad = np.dot(gh, d)
        else:
            fd = (J_np(h, eta + eps * d) - J_np(h, eta - eps * d)) / (2 * eps)
            ad = np.dot(ge, d)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (which, fd, ad)


def test_step_vjp_matches_finite_differences():
    Nx, Nz, L = 32, 8, 8.0
    x, h, eta, u, w = small_tank(Nx, Nz, L)
    g = adj.Grid2(Nx, Nz, L)
    dt = 0.02
    r = np.random.default_rng(9)
    lam = (r.standard_normal(Nx), r.standard_normal((Nz + 1, Nx)), r.standard_normal((Nz + 1, Nx)))
    le, lu, lw, lh = adj.step_vjp(g, h, eta, u, w, dt, *lam, filt=True)
    de, du, dw, dh = (r.standard_normal(Nx), r.standard_normal((Nz + 1, Nx)),
                      r.standard_normal((Nz + 1, Nx)), r.standard_normal(Nx))
    eps = 1e-6
    p = numpy_step(Nx, Nz, L, h + eps * dh, eta + eps * de, u + eps * du, w + eps * dw, dt, filt=True)
    m = numpy_step(Nx, Nz, L, h - eps * dh, eta - eps * de, u - eps * du, w - eps * dw, dt, filt=True)
    fd = sum(np.sum(l * (a - b)) for l, a, b in zip(lam, p, m)) / (2 * eps)
    ad = np.dot(le, de) + np.sum(lu * du) + np.sum(lw * dw) + np.dot(lh, dh)
    assert abs(fd - ad) <= 1e-6 * abs(ad)
