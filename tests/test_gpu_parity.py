"""GPU parity: the CUDA path (through the C ABI) against the oracle on the
same seeded inputs.  Tolerances follow from the arithmetic (unit roundoff u
times the accumulation depth of the FFT stages and sigma contractions times
the cancellation inside the composite operator, about 1e3 u with random-walk
growth): the operator within 1e-11 (FP64) and 2e-4 (FP32) of max |A p|; one
V-cycle within 1e-9 (FP64) and 5e-3 (FP32) of its largest value, where the
column-block inverses' condition numbers (up to ~1e5 for 33-point Chebyshev
blocks) multiply u; solves to the required relative residual, 1e-10 in FP64
and 1e-9 in the mixed modes, measured with the oracle's own operator."""

import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle import krylov, pmg, rk
from oracle import operator as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    return w


def curved(Nx, Ny, Nz, L, seed=0, amp=0.05, bump=0.3):
    g = op.Grid(Nx, Ny, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - bump * np.exp(-((X - L / 2) / (L / 8)) ** 2)
    if Ny > 1:
        h = h + 0.05 * np.cos(2 * np.pi * Y / L)
    r = np.random.default_rng(seed)
    ea = amp * np.cos(2 * np.pi * X / L) + (0.3 * amp * np.sin(2 * np.pi * Y / L) if Ny > 1 else 0)
    eb = ea + 0.01 * amp * r.standard_normal(ea.shape)
    return g, np.ascontiguousarray(h), np.ascontiguousarray(ea), np.ascontiguousarray(eb)


CASES_2D = [(8, 4, 2 * math.pi), (64, 16, 2 * math.pi), (256, 24, 32.0), (1024, 24, 32.0), (2048, 16, 64.0)]


@pytest.mark.parametrize("Nx,Nz,L", CASES_2D)
def test_operator_parity_2d(wt, Nx, Nz, L):
    g, h, ea, eb = curved(Nx, 1, Nz, L)
    p = np.random.default_rng(1).standard_normal(g.shape)
    ref = op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    T = wt.Tank(Nx, 1, Nz, L, h)
    got = T.apply_operator(ea, eb, p, wt.WT_FP64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-11 * scale
    got32 = T.apply_operator(ea, eb, p, wt.WT_FP32)
    assert np.abs(got32 - ref).max() <= 2e-4 * scale


# (128, 128, 8) and (128, 128, 16) have >= 8192 columns: the thread-per-column
# sigma kernel; the smaller ones the warp-per-column kernel
@pytest.mark.parametrize("Nx,Ny,Nz", [(8, 8, 4), (32, 32, 8), (64, 64, 16), (128, 128, 8), (128, 128, 16)])
def test_operator_parity_3d(wt, Nx, Ny, Nz):
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    p = np.random.default_rng(2).standard_normal(g.shape)
    ref = op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    T = wt.Tank(Nx, Ny, Nz, L, h)
    got = T.apply_operator(ea, eb, p, wt.WT_FP64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-11 * scale
    got32 = T.apply_operator(ea, eb, p, wt.WT_FP32)
    assert np.abs(got32 - ref).max() <= 2e-4 * scale


def test_levels_match_oracle_hierarchy(wt):
    for (Nx, Ny, Nz) in [(1024, 1, 24), (64, 1, 16), (256, 256, 16), (2048, 1, 32)]:
        T = wt.Tank(Nx, Ny, Nz, 1.0, np.ones((Ny, Nx)))
        assert T.levels() == pmg.hierarchy(Nx, Ny, Nz, coarsest_max=64)


@pytest.mark.parametrize("tail_max,grid,cluster", [(0, 0, 0), (8192, 0, 0), (100000, 0, 0), (0, 1, 0),
                                                   (8192, 0, 16), (100000, 0, 8), (2048, 0, 2)])
@pytest.mark.parametrize("Nx,Ny,Nz", [(64, 1, 16), (256, 1, 24), (1024, 1, 24), (16, 16, 8),
                                      (32, 32, 12), (64, 64, 16)])
def test_vcycle_parity(wt, Nx, Ny, Nz, tail_max, grid, cluster):
    # same algorithm on both sides (block Jacobi with Nyquist split, omega 0.4,
    # nu1 = nu2 = 2, injected boundary rows, coarsest <= 64 unknowns): the
    # preconditioned vectors agree to rounding.  tail_max selects how many
    # levels run in the single-launch tail of the V-cycle (0: none, 100000:
    # all), cluster the CTAs of the thread-block cluster that runs it (0: one
    # CTA); grid = 1 runs the whole cycle as one cooperative launch.
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    r = np.random.default_rng(3).standard_normal(g.shape)
    levels = pmg.build_levels(Nx, Ny, Nz, L, h, ea, eb, coarsest_max=64)
    ref = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 2, 2, "jacobi", 0.4, "inject")
    T = wt.Tank(Nx, Ny, Nz, L, h, tail_max=tail_max, vcycle_grid=grid, tail_cluster=cluster)
    got = T.precondition(ea, eb, r, wt.WT_FP64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-9 * scale
    got32 = T.precondition(ea, eb, r, wt.WT_FP32)
    assert np.abs(got32 - ref).max() <= 5e-3 * scale


def manufactured_rhs():
    Nx, Nz, L = 64, 16, 2 * math.pi
    g = op.Grid(Nx, 1, Nz, L)
    geo = op.Geometry(g, np.ones(Nx), np.zeros(Nx))
    z = geo.z_nodes(g)
    X = np.broadcast_to(g.x[None, None, :], g.shape)
    ms = si.Manufactured(seed=0)
    b = ms.laplacian(X, z)
    b[0] = ms.p(X[0], z[0])
    b[-1] = ms.dpdz(X[-1], z[-1])
    return g, np.ascontiguousarray(b), ms.p(X, z)


@pytest.mark.parametrize("mode,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-12, 1e-9), (3, 1e-12, 1e-9)])
def test_manufactured_solve(wt, mode, tol, bound):
    g, b, pe = manufactured_rhs()
    T = wt.Tank(64, 1, 16, 2 * math.pi, np.ones((1, 64)), mode=mode, tol=tol)
    z = np.zeros((1, 64))
    p, info = T.poisson_solve(z, z, b)
    assert info.rel_residual <= tol
    assert (info.refinements >= 1) == (mode == 3)
    assert np.abs(p - pe).max() <= bound * np.abs(pe).max()
    geo = op.Geometry(g, np.ones(64), np.zeros(64))
    r = b - op.apply_A(g, geo, geo, p)
    assert np.linalg.norm(r) <= max(tol, 1e-13) * 10 * np.linalg.norm(b)


@pytest.mark.parametrize("mode", [0, 1, 3])
@pytest.mark.parametrize("Nx,Ny,Nz,L", [(1024, 1, 24, 32.0), (128, 1, 12, 8.0), (32, 32, 8, 2 * math.pi),
                                        (128, 128, 16, 8.0)])
def test_curved_solve_residual_in_oracle_operator(wt, mode, Nx, Ny, Nz, L):
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    b = np.random.default_rng(4).standard_normal(g.shape)
    T = wt.Tank(Nx, Ny, Nz, L, h, mode=mode, tol=1e-10, max_it=300)
    p, info = T.poisson_solve(ea, eb, b)
    assert info.rel_residual <= 1e-10
    r = b - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    bound = 1e-10 if mode == 0 else 1e-9
    assert np.linalg.norm(r) <= bound * np.linalg.norm(b) * 1.5


SCHEDULES = [dict(vcycle_grid=1), dict(tail_max=8192, tail_cluster=16), dict(tail_max=2048, tail_cluster=8)]


@pytest.mark.parametrize("sched", range(len(SCHEDULES)))
@pytest.mark.parametrize("Nx,Ny,Nz,L", [(1024, 1, 24, 32.0), (32, 32, 12, 2 * math.pi)])
def test_grid_vcycle_matches_launch_per_phase(wt, Nx, Ny, Nz, L, sched):
    # the cooperative V-cycle and the cluster tail run the same bodies: a
    # mixed solve and (2D) a nonlinear step agree with the
    # one-launch-per-phase path to rounding
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    b = np.random.default_rng(6).standard_normal(g.shape)
    out = []
    opts = [dict(), SCHEDULES[sched]]
    for o in opts:
        T = wt.Tank(Nx, Ny, Nz, L, h, mode=1, tol=1e-10, max_it=300, **o)
        p, info = T.poisson_solve(ea, eb, b)
        assert info.rel_residual <= 1e-10
        out.append((p, info.iterations))
    assert out[0][1] == out[1][1]
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-9 * np.abs(out[0][0]).max()
    if Ny == 1:
        x = np.arange(Nx) * L / Nx
        eta = si.stokes2_eta(x, 0.1, 2 * math.pi * 5 / L, 1.0)[None]
        geo = op.Geometry(g, h, eta)
        u, w = si.linear_velocity(x[None, None, :], geo.z_nodes(g), 0.1, 2 * math.pi * 5 / L, 1.0)
        st = []
        for o in opts:
            T = wt.Tank(Nx, 1, Nz, L, h, tol=1e-10, filter=1, **o)
            T.set_state(np.ascontiguousarray(eta), np.ascontiguousarray(u), np.zeros_like(u),
                        np.ascontiguousarray(w))
            T.step(0.005, 2)
            st.append(T.get_state())
        for a, c in zip(st[0][:4], st[1][:4]):
            assert np.abs(a - c).max() <= 1e-9 * max(np.abs(c).max(), 1e-30)


def test_solve_matches_oracle_dense_lu(wt):
    Nx, Nz, L = 32, 10, 2 * math.pi
    g, h, ea, eb = curved(Nx, 1, Nz, L)
    b = np.random.default_rng(5).standard_normal(g.shape)
    lev = pmg.Level(Nx, 1, Nz, L, h, ea, eb)
    ref = krylov.solve_dense(lev, b)
    # the oracle's own GMRES + p-multigrid at 1e-12 lands 3e-13 from the LU
    # solution (cond(A) ~ 2e4 here), so the solve bounds of the method apply
    # directly: 1e-10 for the FP64 path, 1e-9 for the mixed paths
    for mode, bound in ((0, 1e-10), (1, 1e-9), (3, 1e-9)):
        T = wt.Tank(Nx, 1, Nz, L, h, mode=mode, tol=1e-12)
        p, info = T.poisson_solve(ea, eb, b)
        err = np.abs(p - ref).max() / np.abs(ref).max()
        print("dense LU parity, mode %d: %.2e (%d iterations)" % (mode, err, info.iterations))
        assert err <= bound


def test_zero_rhs_and_invalid_geometry(wt):
    Nx, Nz, L = 32, 8, 2 * math.pi
    h = np.ones((1, Nx))
    T = wt.Tank(Nx, 1, Nz, L, h)
    z = np.zeros((1, Nx))
    p, info = T.poisson_solve(z, z, np.zeros(T.shape), p=np.ones(T.shape))
    assert np.all(p == 0.0)
    bad = np.full((1, Nx), -2.0)                 # d = h + eta <= 0
    with pytest.raises(wt.WtError) as e:
        T.apply_operator(bad, z, np.ones(T.shape))
    assert e.value.code == wt.WT_EBREAK
    # the tank stays usable after the error
    T.apply_operator(z, z, np.ones(T.shape))


def _oracle_state(g, tank_o, eta, u, w):
    st = rk.State(g, eta, u, np.zeros_like(u), w)
    return st


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_rk_stages_parity(wt, mode):
    # five stages of a nonlinear wave over a bump: GPU vs oracle, both solving
    # each Poisson problem to 1e-12
    Nx, Nz, L = 64, 12, 2 * math.pi
    x = np.arange(Nx) * L / Nx
    h = (1.0 - 0.3 * np.exp(-((x - L / 2) / 1.0) ** 2))[None]
    g = op.Grid(Nx, 1, Nz, L)
    eta0 = si.stokes2_eta(x, 0.03, 1.0, 1.0)[None]
    geo = op.Geometry(g, h, eta0)
    u0, w0 = si.linear_velocity(x[None, None, :], geo.z_nodes(g), 0.03, 1.0, 1.0)
    tank_o = rk.Tank(Nx, 1, Nz, L, h, tol=1e-13, coarsest_max=64)
    st = rk.State(g, eta0, u0, np.zeros_like(u0), w0)
    dt = 0.01
    T = wt.Tank(Nx, 1, Nz, L, h, mode=mode, tol=1e-12)
    T.set_state(np.ascontiguousarray(eta0), np.ascontiguousarray(u0), np.zeros_like(u0),
                np.ascontiguousarray(w0))
    for k in range(1, 6):
        rk.stage(tank_o, st, k, dt)
        T.rk_stage(k, dt)
    eta, u, v, w, tm = T.get_state()
    assert abs(tm - dt) < 1e-15
    assert np.abs(eta - st.eta).max() <= 1e-10 * np.abs(st.eta).max()
    assert np.abs(u - st.u).max() <= 1e-8 * np.abs(st.u).max()
    assert np.abs(w - st.w).max() <= 1e-8 * np.abs(st.w).max()
    # the projected velocity is discretely divergence-free in the oracle's operator
    dv, bot = rk.divergence_residual(tank_o, rk.State(g, eta, u, v, w))
    assert np.abs(dv).max() < 1e-7 and np.abs(bot).max() < 1e-9


def test_airy_period_on_gpu(wt):
    # linear model, k = 1, h = 1: eta returns to A cos x after one period
    Nx, Nz, L = 64, 16, 2 * math.pi
    T = wt.Tank(Nx, 1, Nz, L, np.ones((1, Nx)), mode=0, tol=1e-12, linear=1)
    g = op.Grid(Nx, 1, Nz, L)
    A = 0.005
    eta0 = si.airy(g.x, None, A=A)[None]
    geo = op.Geometry(g, np.ones(Nx), np.zeros(Nx))
    _, u, w = si.airy(g.x[None, None, :], geo.z_nodes(g), A=A)
    T.set_state(np.ascontiguousarray(eta0), np.ascontiguousarray(u), np.zeros_like(u),
                np.ascontiguousarray(w))
    Tp = 2 * math.pi / si.omega(1.0, 1.0)
    T.step(Tp / 100, 100)
    eta = T.get_state()[0]
    assert np.abs(eta - eta0).max() / A < 2e-5
    assert abs(eta.mean()) < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_rk_stages_parity_3d(wt, mode):
    # five stages of a small directional sea in a 3D tank over a gentle bump
    N, Nz, L = 16, 8, 2 * math.pi
    g = op.Grid(N, N, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - 0.1 * np.cos(X) * np.sin(Y)
    sea = si.jonswap_sea(seed=2, L=L, ncomp=12, kp=2.0, hs_over_lp=0.01)
    eta0, u0, v0, w0 = si.jonswap_fields(sea, N, g.sigma)
    tank_o = rk.Tank(N, N, Nz, L, h, tol=1e-13, coarsest_max=64)
    st = rk.State(g, eta0, u0, v0, w0)
    dt = 0.01
    T = wt.Tank(N, N, Nz, L, h, mode=mode, tol=1e-12, max_it=400)
    T.set_state(*(np.ascontiguousarray(a) for a in (eta0, u0, v0, w0)))
    for k in range(1, 6):
        rk.stage(tank_o, st, k, dt)
        T.rk_stage(k, dt)
    eta, u, v, w, tm = T.get_state()
    for got, ref in ((eta, st.eta), (u, st.u), (v, st.v), (w, st.w)):
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    dv, bot = rk.divergence_residual(tank_o, rk.State(g, eta, u, v, w))
    assert np.abs(dv).max() < 1e-7 and np.abs(bot).max() < 1e-9


@pytest.mark.parametrize("N,Nz,stages", [(128, 4, 5), (128, 16, 1)])
def test_rk_stages_parity_3d_many_columns(wt, N, Nz, stages):
    # 16,384 columns: the FP64 sigma derivatives and the Chebyshev filter of
    # the stage run one thread per column (the column-matrix kernel for
    # levels of at least 8,192 columns), filter on, against the oracle
    L = 2 * math.pi
    g = op.Grid(N, N, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - 0.1 * np.cos(X) * np.sin(Y)
    sea = si.jonswap_sea(seed=2, L=L, ncomp=48, kp=4.0, hs_over_lp=0.01)
    eta0, u0, v0, w0 = si.jonswap_fields(sea, N, g.sigma)
    tank_o = rk.Tank(N, N, Nz, L, h, tol=1e-13, coarsest_max=64, filter=True)
    st = rk.State(g, eta0, u0, v0, w0)
    dt = 0.005
    T = wt.Tank(N, N, Nz, L, h, mode=wt.WT_MIXED, tol=1e-12, max_it=400, filter=1)
    T.set_state(*(np.ascontiguousarray(a) for a in (eta0, u0, v0, w0)))
    for k in range(1, stages + 1):
        rk.stage(tank_o, st, k, dt)
        T.rk_stage(k, dt)
    eta, u, v, w, tm = T.get_state()
    for got, ref in ((eta, st.eta), (u, st.u), (v, st.v), (w, st.w)):
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("Nx,Ny,Nz", [(64, 1, 16), (1024, 1, 24), (16, 16, 8), (32, 32, 12)])
def test_fmg_parity(wt, Nx, Ny, Nz):
    # one full-multigrid cycle (Algorithm 2) as the preconditioner: the GPU's
    # cycle against the oracle's on the same hierarchy and smoother
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    r = np.random.default_rng(4).standard_normal(g.shape)
    levels = pmg.build_levels(Nx, Ny, Nz, L, h, ea, eb, coarsest_max=64)
    ref = pmg.fmg(levels, r, 2, 2, "jacobi", 0.4, "inject")
    T = wt.Tank(Nx, Ny, Nz, L, h, cycle=1)
    got = T.precondition(ea, eb, r, wt.WT_FP64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-9 * scale
    got32 = T.precondition(ea, eb, r, wt.WT_FP32)
    assert np.abs(got32 - ref).max() <= 5e-3 * scale


@pytest.mark.parametrize("mode", [0, 1])
def test_fmg_solve_takes_no_more_iterations_than_vcycle(wt, mode):
    # Table 1: FMG + GMRES needs slightly fewer iterations than V-cycle +
    # GMRES for the same tolerance (and costs more per iteration)
    Nx, Nz, L = 256, 24, 8.0
    g, h, ea, eb = curved(Nx, 1, Nz, L)
    b = np.random.default_rng(9).standard_normal(g.shape)
    its = {}
    for cyc in (0, 1):
        T = wt.Tank(Nx, 1, Nz, L, h, mode=mode, tol=1e-10, cycle=cyc)
        p, info = T.poisson_solve(ea, eb, b)
        r = b - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
        its[cyc] = info.iterations
    print("iterations V-cycle %d, FMG %d (mode %d)" % (its[0], its[1], mode))
    assert its[1] <= its[0]


@pytest.mark.parametrize("Nx,Ny,Nz", [(256, 256, 12), (512, 512, 4), (1024, 1024, 2)])
def test_operator_parity_warp_passes(wt, Nx, Ny, Nz):
    # 3D levels with many lines run their FP32 x- and y-derivative passes one
    # warp per line pair (transform in registers; 256, 512 and 1024 points):
    # against the oracle, and against the CTA-per-line passes (warp_fft = 0)
    # on the same tank
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    p = np.random.default_rng(2).standard_normal(g.shape)
    ref = op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    scale = np.abs(ref).max()
    T = wt.Tank(Nx, Ny, Nz, L, h)
    got = T.apply_operator(ea, eb, p, wt.WT_FP64)
    got32 = T.apply_operator(ea, eb, p, wt.WT_FP32)
    assert np.abs(got - ref).max() <= 1e-11 * scale
    assert np.abs(got32 - ref).max() <= 2e-4 * scale
    T.set_options(warp_fft=0)
    old = T.apply_operator(ea, eb, p, wt.WT_FP64)
    old32 = T.apply_operator(ea, eb, p, wt.WT_FP32)
    assert np.abs(got - old).max() <= 1e-12 * scale
    assert np.abs(got32 - old32).max() <= 1e-4 * scale
