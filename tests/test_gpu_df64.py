"""FP64 derivative passes in double-float arithmetic (option df64): the FP64
operator and solve against the oracle (Eq. 1_chain / Sec. 3.5 derivatives,
Sec. 4.4 solve) at the FP64 bounds, and against the FP64-arithmetic passes
on the same tank; a band-limited derivative against its closed form."""

import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle import operator as op
from oracle import rk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    return w


def curved(Nx, Ny, Nz, L, seed=0, amp=0.05, bump=0.3):
    g = op.Grid(Nx, Ny, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - bump * np.exp(-((X - L / 2) / (L / 8)) ** 2) + 0.05 * np.cos(2 * np.pi * Y / L)
    r = np.random.default_rng(seed)
    ea = amp * np.cos(2 * np.pi * X / L) + 0.3 * amp * np.sin(2 * np.pi * Y / L)
    eb = ea + 0.01 * amp * r.standard_normal(ea.shape)
    return g, np.ascontiguousarray(h), np.ascontiguousarray(ea), np.ascontiguousarray(eb)


@pytest.mark.parametrize("N,Nz", [(64, 8), (128, 16), (256, 12)])
def test_df64_operator_parity(wt, N, Nz):
    L = 2 * math.pi
    g, h, ea, eb = curved(N, N, Nz, L)
    p = np.random.default_rng(2).standard_normal(g.shape)
    ref = op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    scale = np.abs(ref).max()
    T = wt.Tank(N, N, Nz, L, h, df64=1)
    got = T.apply_operator(ea, eb, p, wt.WT_FP64)
    T.set_options(df64=0)
    nat = T.apply_operator(ea, eb, p, wt.WT_FP64)
    err_df, err_nat = np.abs(got - ref).max() / scale, np.abs(nat - ref).max() / scale
    print("FP64 operator, max error / max |Ap|: double-float %.2e, FP64 %.2e" % (err_df, err_nat))
    assert err_df <= 1e-11
    assert np.abs(got - nat).max() <= 1e-12 * scale


def test_df64_derivative_closed_form(wt):
    # a band-limited field whose x- and y-derivatives are known exactly: the
    # operator on a flat tank at rest with p independent of sigma reduces to
    # the horizontal Laplacian (interior rows), so A p = -(kx^2 + ky^2) p
    N, Nz, L = 256, 8, 2 * math.pi
    g = op.Grid(N, N, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    f = np.cos(7 * X + 0.3) * np.sin(11 * Y) + 0.5 * np.sin(100 * X - 60 * Y)
    lap = -(49 + 121) * np.cos(7 * X + 0.3) * np.sin(11 * Y) - 0.5 * (100 ** 2 + 60 ** 2) * np.sin(100 * X - 60 * Y)
    p = np.broadcast_to(f, g.shape).copy()
    z = np.zeros((N, N))
    h = np.ones((N, N))
    out = {}
    for df in (1, 0):
        T = wt.Tank(N, N, Nz, L, h, df64=df)
        out[df] = T.apply_operator(z, z, p, wt.WT_FP64)
    scale = np.abs(lap).max()
    for df in (1, 0):
        err = np.abs(out[df][1:-1] - lap[None]).max() / scale
        print("interior Laplacian, df64=%d: max error / max |lap| %.2e" % (df, err))
        assert err <= 5e-13


def test_df64_solve_residual_in_oracle_operator(wt):
    N, Nz, L = 64, 12, 2 * math.pi
    g, h, ea, eb = curved(N, N, Nz, L)
    b = np.random.default_rng(4).standard_normal(g.shape)
    for mode in (0, 1, 3):
        T = wt.Tank(N, N, Nz, L, h, mode=mode, tol=1e-10, max_it=300, df64=1)
        p, info = T.poisson_solve(ea, eb, b)
        assert info.rel_residual <= 1e-10
        r = b - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
        bound = 1e-10 if mode == 0 else 1e-9
        assert np.linalg.norm(r) <= bound * np.linalg.norm(b) * 1.5


def test_df64_stages_parity(wt):
    # five RK stages of a small directional sea (16,384 columns, filter on)
    # with the FP64 derivative passes in double-float, against the oracle
    N, Nz, L = 128, 4, 2 * math.pi
    g = op.Grid(N, N, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - 0.1 * np.cos(X) * np.sin(Y)
    sea = si.jonswap_sea(seed=2, L=L, ncomp=48, kp=4.0, hs_over_lp=0.01)
    eta0, u0, v0, w0 = si.jonswap_fields(sea, N, g.sigma)
    tank_o = rk.Tank(N, N, Nz, L, h, tol=1e-13, coarsest_max=64, filter=True)
    st = rk.State(g, eta0, u0, v0, w0)
    dt = 0.005
    T = wt.Tank(N, N, Nz, L, h, mode=wt.WT_MIXED, tol=1e-12, max_it=400, filter=1, df64=1)
    T.set_state(*(np.ascontiguousarray(a) for a in (eta0, u0, v0, w0)))
    for k in range(1, 6):
        rk.stage(tank_o, st, k, dt)
        T.rk_stage(k, dt)
    eta, u, v, w, tm = T.get_state()
    for got, ref in ((eta, st.eta), (u, st.u), (v, st.v), (w, st.w)):
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(256, 1, 24), (64, 64, 12)])
def test_df64_attainable_residual(wt, shape):
    # the smallest relative residual an FP64 solve reaches (tolerance 1e-15,
    # stopped by the iteration cap): FP64 arithmetic; double-float kernels
    # with the true residuals' row passes in FP64 (df64 = 1, the default:
    # FP64's floor); double-float everywhere (df64 = 2); all well below the
    # method's 1e-10
    Nx, Ny, Nz = shape
    L = 8.0
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    if Ny == 1:
        h, ea, eb = (np.ascontiguousarray(a[:1]) for a in (h, ea, eb))
    b = np.random.default_rng(11).standard_normal(g.shape)
    floor = {}
    for df in (0, 1, 2):
        T = wt.Tank(Nx, Ny, Nz, L, h, mode=wt.WT_FP64, tol=1e-15, max_it=120, df64=df)
        p, info = T.poisson_solve(ea, eb, b, raise_noconv=False)
        floor[df] = info.rel_residual
        T.close()
    print("attainable FP64 relative residual %s: FP64 %.1e, df64=1 %.1e, df64=2 %.1e"
          % (shape, floor[0], floor[1], floor[2]))
    assert floor[0] <= 1e-12 and floor[1] <= 2e-12 and floor[2] <= 1e-11
