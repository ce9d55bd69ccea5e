"""Adjoint of the 2D step on the GPU (the paper has no adjoint): the
transposed operator against the oracle's dense A^T, the transposed solve,
one reversed step against the oracle's exact step derivative
(oracle/adjoint.py, torch.autograd of the restated step), the checkpointed
torch.autograd.Function against the oracle's gradient, and central finite
differences of the GPU forward run on the gradient workload's bathymetry."""

import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle import operator as op

torch = pytest.importorskip("torch")
from oracle import adjoint as adj  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_00991_gb300 as wt
    return wt


def curved2d(Nx, Nz, L, seed=0):
    r = np.random.default_rng(seed)
    x = np.arange(Nx) * L / Nx
    h = 1.0 - 0.3 * np.exp(-((x - L / 2) / (0.15 * L)) ** 2)
    ea = 0.05 * np.cos(2 * math.pi * x / L + r.uniform(0, 6)) + 0.02 * np.sin(4 * math.pi * x / L)
    eb = 0.9 * ea + 0.01 * np.cos(6 * math.pi * x / L)
    return x, h[None], ea[None], eb[None]


@pytest.mark.parametrize("prec,bound", [(0, 1e-11), (2, 2e-4)])
def test_transposed_operator_matches_dense_transpose(wt, prec, bound):
    Nx, Nz, L = 64, 12, 4.0
    x, h, ea, eb = curved2d(Nx, Nz, L)
    g = op.Grid(Nx, 1, Nz, L)
    A = op.assemble_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb))
    lam = np.random.default_rng(1).standard_normal(g.shape)
    ref = (A.T @ lam.ravel()).reshape(g.shape)
    T = wt.Tank(Nx, 1, Nz, L, h)
    out = T.apply_operator_transposed(ea, eb, lam, precision=prec)
    assert np.abs(out - ref).max() <= bound * np.abs(ref).max()


def test_transposed_dot_product_1024x24(wt):
    Nx, Nz, L = 1024, 24, 32.0
    x, h, ea, eb = curved2d(Nx, Nz, L)
    T = wt.Tank(Nx, 1, Nz, L, h)
    r = np.random.default_rng(2)
    X = r.standard_normal(T.shape)
    Y = r.standard_normal(T.shape)
    lhs = np.sum(T.apply_operator(ea, eb, X) * Y)
    rhs = np.sum(X * T.apply_operator_transposed(ea, eb, Y))
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(T.apply_operator(ea, eb, X) ** 2) * np.sum(Y ** 2))


@pytest.mark.parametrize("mode", [0, 1])
def test_transposed_solve(wt, mode):
    Nx, Nz, L = 64, 12, 4.0
    x, h, ea, eb = curved2d(Nx, Nz, L)
    g = op.Grid(Nx, 1, Nz, L)
    A = op.assemble_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb))
    b = np.random.default_rng(3).standard_normal(g.shape)
    ref = np.linalg.solve(A.T, b.ravel()).reshape(g.shape)
    T = wt.Tank(Nx, 1, Nz, L, h, mode=mode, tol=1e-12)
    lam, info = T.adjoint_solve(ea, eb, b)
    assert info.rel_residual <= 1e-12
    assert np.abs(lam - ref).max() <= 1e-8 * np.abs(ref).max()


def small_state(Nx, Nz, L, seed=1):
    x = np.arange(Nx) * L / Nx
    b, phi = si.adjoint_bathymetry(seed, L=L, K=6)
    h = si.fourier_bathymetry(x, 3 * b, phi, L=L)
    eta = 0.02 * np.cos(2 * math.pi * x / (L / 2)) + 0.01 * np.sin(2 * math.pi * x / L)
    g = op.Grid(Nx, 1, Nz, L)
    z = op.Geometry(g, h, eta).z_nodes(g)
    u, w = si.linear_velocity(x[None, None, :], z, 0.02, 2 * math.pi / (L / 2), 1.0)
    return h, eta, np.ascontiguousarray(u[:, 0, :]), np.ascontiguousarray(w[:, 0, :])


@pytest.mark.parametrize("kw,mode", [(dict(), 0), (dict(filt=True), 0), (dict(linear=True), 0),
                                     (dict(filt=True), 1)])
def test_adjoint_step_matches_oracle(wt, kw, mode):
    Nx, Nz, L, dt = 32, 8, 8.0, 0.02
    h, eta, u, w = small_state(Nx, Nz, L)
    g = adj.Grid2(Nx, Nz, L)
    r = np.random.default_rng(9)
    lam = (r.standard_normal(Nx), r.standard_normal((Nz + 1, Nx)), r.standard_normal((Nz + 1, Nx)))
    le_o, lu_o, lw_o, lh_o = adj.step_vjp(g, h, eta, u, w, dt, *lam, **kw)
    T = wt.Tank(Nx, 1, Nz, L, h[None], mode=mode, tol=1e-12, filter=int(kw.get("filt", False)),
                linear=int(kw.get("linear", False)))
    le = lam[0].copy()[None]
    lu = lam[1].copy()[:, None, :]
    lw = lam[2].copy()[:, None, :]
    dh = np.zeros((1, Nx))
    T.adjoint_step(dt, eta[None].copy(), u[:, None, :].copy(), w[:, None, :].copy(), le, lu, lw, dh)
    bound = 1e-8
    for a, b in ((le[0], le_o), (lu[:, 0], lu_o), (lw[:, 0], lw_o), (dh[0], lh_o)):
        assert np.abs(a - b).max() <= bound * np.abs(b).max()


def test_gauge_series_gradient_matches_oracle(wt):
    from paper_2406_00991_gb300.adjoint import gauge_series
    Nx, Nz, L, dt, nsteps = 32, 8, 8.0, 0.02, 6
    h, eta, u, w = small_state(Nx, Nz, L)
    gauges = np.arange(0, Nx, 8)
    target = 0.01 * np.random.default_rng(3).standard_normal((nsteps, len(gauges)))
    J_o, gh_o, ge_o, gu_o, gw_o = adj.loss_and_gradient(adj.Grid2(Nx, Nz, L), h, eta, u, w, dt, nsteps,
                                                        gauges, target, filt=True)
    dev = torch.device("cuda")
    T = wt.Tank(Nx, 1, Nz, L, h[None], mode=0, tol=1e-12, filter=1)
    ht = torch.tensor(h, device=dev, requires_grad=True)
    et = torch.tensor(eta, device=dev, requires_grad=True)
    ut = torch.tensor(u, device=dev, requires_grad=True)
    wt_ = torch.tensor(w, device=dev, requires_grad=True)
    series = gauge_series(T, ht, et, ut, wt_, dt, nsteps, gauges, every=4)
    J = 0.5 * torch.sum((series - torch.tensor(target, device=dev)) ** 2) * dt
    J.backward()
    assert abs(J.item() - J_o) <= 1e-10 * J_o
    for a, b in ((ht.grad, gh_o), (et.grad, ge_o), (ut.grad, gu_o), (wt_.grad, gw_o)):
        a = a.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()


def test_bathymetry_gradient_finite_differences(wt):
    # the gradient workload's tank (L = 16, Nx = 512, Nz = 20, 64-mode seeded
    # bathymetry, eta0 = 0.02 cos(2 pi x / 4), u0 = w0 = 0) over 40 steps
    # (0.2 s: long enough for the bathymetry to act on the gauges)
    from paper_2406_00991_gb300.adjoint import gauge_series
    Nx, Nz, L, nsteps = 512, 20, 16.0, 40
    dt = 0.5 * (L / Nx) / math.sqrt(9.81)
    x = np.arange(Nx) * L / Nx
    b0, phi = si.adjoint_bathymetry(5, L=L, K=64)
    kk = np.arange(1, 65)
    C = np.cos(2 * math.pi * kk[:, None] * x[None, :] / L + phi[:, None])      # (64, Nx)
    eta0 = 0.02 * np.cos(2 * math.pi * x / 4.0)
    gauges = np.arange(0, Nx, 32)
    dev = torch.device("cuda")
    T = wt.Tank(Nx, 1, Nz, L, (1.0 + b0 @ C)[None], mode=0, tol=1e-12, filter=1, max_it=400)
    Ct = torch.tensor(C, device=dev)
    zeros = torch.zeros((Nz + 1, Nx), dtype=torch.float64, device=dev)
    target = torch.zeros((nsteps, len(gauges)), dtype=torch.float64, device=dev)

    def J_of(b, e0, grad=False):
        bt = torch.tensor(b, device=dev, requires_grad=grad)
        et = torch.tensor(e0, device=dev, requires_grad=grad)
        series = gauge_series(T, 1.0 + bt @ Ct, et, zeros, zeros, dt, nsteps, gauges, every=10)
        J = 0.5 * torch.sum((series - target) ** 2) * dt
        if grad:
            J.backward()
            return J.item(), bt.grad.cpu().numpy(), et.grad.cpu().numpy()
        return J.item()

    J0, gb, ge = J_of(b0, eta0, grad=True)
    r = np.random.default_rng(11)
    db = r.standard_normal(64) * 0.02 / kk
    de = 0.02 * r.standard_normal(Nx)
    for d_b, d_e, eps in ((db, 0 * de, 1e-2), (0 * db, de, 1e-4)):
        fd = (J_of(b0 + eps * d_b, eta0 + eps * d_e) - J_of(b0 - eps * d_b, eta0 - eps * d_e)) / (2 * eps)
        ad = np.dot(gb, d_b) + np.dot(ge, d_e)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_gradient_workload_as_stated(wt):
    """The gradient workload as stated: L = 16, Nx = 512, Nz = 20, 64-mode
    seeded bathymetry, eta0 = 0.02 cos(2 pi x / 4), u0 = w0 = 0, 400 steps,
    checkpoints every 20 steps, 16 gauges, target from a forward run over a
    second seeded bathymetry.  The FP64 gradient (solves at 1e-12, the
    tightest relative residual the FP64 path reaches here) against central
    finite differences with step 1e-6 along a unit direction in the 64 b_k
    and one in eta0 (agreement to 1e-6 relative), and the mixed solver's
    gradient (1e-10 solves) against the FP64 one."""
    from paper_2406_00991_gb300.adjoint import gauge_series
    Nx, Nz, L, nsteps, every = 512, 20, 16.0, 400, 20
    dt = 0.5 * (L / Nx) / math.sqrt(9.81)
    x = np.arange(Nx) * L / Nx
    b0, phi = si.adjoint_bathymetry(5, L=L, K=64)
    b_star, _ = si.adjoint_bathymetry(6, L=L, K=64)
    kk = np.arange(1, 65)
    C = np.cos(2 * math.pi * kk[:, None] * x[None, :] / L + phi[:, None])
    eta0 = 0.02 * np.cos(2 * math.pi * x / 4.0)
    gauges = np.arange(0, Nx, 32)
    dev = torch.device("cuda")
    Ct = torch.tensor(C, device=dev)
    zeros = torch.zeros((Nz + 1, Nx), dtype=torch.float64, device=dev)
    T = wt.Tank(Nx, 1, Nz, L, (1.0 + b0 @ C)[None], mode=0, tol=1e-12, filter=1, max_it=600)
    with torch.no_grad():
        target = gauge_series(T, 1.0 + torch.tensor(b_star, device=dev) @ Ct, torch.tensor(eta0, device=dev),
                              zeros, zeros, dt, nsteps, gauges, every=every).clone()

    def J_of(b, e0, grad=False):
        bt = torch.tensor(b, device=dev, requires_grad=grad)
        et = torch.tensor(e0, device=dev, requires_grad=grad)
        series = gauge_series(T, 1.0 + bt @ Ct, et, zeros, zeros, dt, nsteps, gauges, every=every)
        J = 0.5 * torch.sum((series - target) ** 2) * dt
        if grad:
            J.backward()
            return J.item(), bt.grad.cpu().numpy(), et.grad.cpu().numpy()
        return J.item()

    J0, gb, ge = J_of(b0, eta0, grad=True)
    r = np.random.default_rng(11)
    db = r.standard_normal(64)
    db /= np.linalg.norm(db)
    de = r.standard_normal(Nx)
    de /= np.linalg.norm(de)
    eps = 1e-6
    for d_b, d_e in ((db, 0 * de), (0 * db, de)):
        fd = (J_of(b0 + eps * d_b, eta0 + eps * d_e) - J_of(b0 - eps * d_b, eta0 - eps * d_e)) / (2 * eps)
        ad = float(np.dot(gb, d_b) + np.dot(ge, d_e))
        print("gradient workload: finite difference %.12e, adjoint %.12e, relative %.2e"
              % (fd, ad, abs(fd - ad) / abs(ad)))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    # the mixed solver's gradient
    T.set_options(mode=1, tol=1e-10)
    J1, gb1, ge1 = J_of(b0, eta0, grad=True)
    rel_b = np.abs(gb1 - gb).max() / np.abs(gb).max()
    rel_e = np.abs(ge1 - ge).max() / np.abs(ge).max()
    print("mixed vs FP64 gradient: J %.2e, b %.2e, eta0 %.2e relative" % (abs(J1 - J0) / J0, rel_b, rel_e))
    assert abs(J1 - J0) <= 1e-8 * J0
    assert rel_b <= 1e-7 and rel_e <= 1e-7
    T.close()
