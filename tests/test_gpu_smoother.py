"""The mean-depth spectral smoother on the GPU (option smoother = 1, and 2 =
block-Jacobi then spectral) against the oracle's: one V-cycle (Algorithm 1)
with the same hierarchy, reference depth min(h) and damping, compared to
rounding (1e-9 FP64, 5e-3 FP32 of the largest value, the V-cycle parity
bounds); solves to the method's tolerance in the oracle's operator, with
fewer Krylov iterations than block-Jacobi alone; the transposed smoother
inside the adjoint solve."""

import math

import numpy as np
import pytest

from oracle import krylov, pmg
from oracle import operator as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    return w


def curved(Nx, Ny, Nz, L, bump=0.3, amp=0.05):
    g = op.Grid(Nx, Ny, Nz, L)
    X, Y = np.meshgrid(g.x, g.y, indexing="xy")
    h = 1.0 - bump * np.exp(-((X - L / 2) / (L / 8)) ** 2)
    if Ny > 1:
        h = h + 0.05 * np.cos(2 * np.pi * Y / L)
    ea = amp * np.cos(2 * np.pi * X / L) + (0.3 * amp * np.sin(2 * np.pi * Y / L) if Ny > 1 else 0)
    eb = 0.98 * ea
    return g, np.ascontiguousarray(h), np.ascontiguousarray(ea), np.ascontiguousarray(eb)


KINDS = {1: "spectral", 2: "jacobi+spectral"}


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("Nx,Ny,Nz", [(64, 1, 16), (1024, 1, 24), (16, 16, 8), (32, 32, 12), (64, 64, 16)])
def test_spectral_vcycle_parity(wt, Nx, Ny, Nz, kind):
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    r = np.random.default_rng(6).standard_normal(g.shape)
    levels = pmg.build_levels(Nx, Ny, Nz, L, h, ea, eb, coarsest_max=64)
    ref = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 2, 2, KINDS[kind], 0.4, "inject", 1.0, float(h.min()))
    T = wt.Tank(Nx, Ny, Nz, L, h, smoother=kind)
    scale = np.abs(ref).max()
    got = T.precondition(ea, eb, r, wt.WT_FP64)
    assert np.abs(got - ref).max() <= 1e-9 * scale
    got32 = T.precondition(ea, eb, r, wt.WT_FP32)
    assert np.abs(got32 - ref).max() <= 5e-3 * scale
    # damping omega_s reaches the device
    T.set_options(omega_s=0.7)
    ref7 = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 2, 2, KINDS[kind], 0.4, "inject", 0.7, float(h.min()))
    assert np.abs(T.precondition(ea, eb, r, wt.WT_FP64) - ref7).max() <= 1e-9 * np.abs(ref7).max()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("Nx,Ny,Nz,L,bump", [(256, 1, 24, 8.0, 0.5), (32, 32, 16, 16.0, 0.0)])
def test_spectral_smoother_cuts_iterations(wt, mode, Nx, Ny, Nz, L, bump):
    g, h, ea, eb = curved(Nx, Ny, Nz, L, bump=bump, amp=0.04)
    b = np.random.default_rng(8).standard_normal(g.shape)
    its = {}
    for kind, nu in ((0, 2), (2, 2), (1, 1)):
        T = wt.Tank(Nx, Ny, Nz, L, h, mode=mode, tol=1e-10, smoother=kind, nu1=nu, nu2=nu, omega=0.5,
                    max_it=300)
        p, info = T.poisson_solve(ea, eb, b)
        r = b - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b), (kind, info.iterations)
        its[kind] = info.iterations
        T.close()
    print("Krylov iterations (block-Jacobi V(2,2), BJ+spectral V(2,2), spectral V(1,1)):", its)
    assert its[2] < its[0]
    if Ny > 1:
        assert its[1] < its[0]


def test_spectral_smoother_transposed_solve(wt):
    Nx, Nz, L = 32, 10, 2 * math.pi
    g, h, ea, eb = curved(Nx, 1, Nz, L)
    b = np.random.default_rng(12).standard_normal(g.shape)
    lev = pmg.Level(Nx, 1, Nz, L, h, ea, eb)
    ref = np.linalg.solve(lev.dense.T, b.ravel()).reshape(g.shape)
    T = wt.Tank(Nx, 1, Nz, L, h, mode=0, tol=1e-12, smoother=2)
    lam, info = T.adjoint_solve(ea, eb, b)
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()


def test_spectral_tables_follow_the_bathymetry(wt):
    # the reference depth is min(h): a new bathymetry rebuilds the tables
    Nx, Nz, L = 64, 12, 2 * math.pi
    g, h, ea, eb = curved(Nx, 1, Nz, L)
    r = np.random.default_rng(1).standard_normal(g.shape)
    T = wt.Tank(Nx, 1, Nz, L, h, smoother=1)
    h2 = np.ascontiguousarray(h * 0.8 + 0.1)
    T.set_bathymetry(h2)
    levels = pmg.build_levels(Nx, 1, Nz, L, h2, ea, eb, coarsest_max=64)
    ref = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 2, 2, "spectral", 0.4, "inject", 1.0, float(h2.min()))
    got = T.precondition(ea, eb, r, wt.WT_FP64)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    with pytest.raises(wt.WtError) as e:
        T.set_options(smoother=3)
    assert e.value.code == wt.WT_EINVAL


@pytest.mark.parametrize("Nx,Ny,Nz,tail,cluster", [(64, 64, 16, 4352, 0), (64, 64, 16, 4352, 8),
                                                    (32, 32, 12, 1000, 0), (1024, 1, 24, 2048, 0)])
def test_spectral_vcycle_with_tail_parity(wt, Nx, Ny, Nz, tail, cluster):
    # spectral smoother on the levels above tail_max unknowns, the one-launch
    # tail (one CTA, or a cluster) with block-Jacobi sweeps on the rest:
    # against the oracle's V-cycle with the same smoother kind by level
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    r = np.random.default_rng(6).standard_normal(g.shape)
    levels = pmg.build_levels(Nx, Ny, Nz, L, h, ea, eb, coarsest_max=64)
    sizes = [lv.grid.Nx * lv.grid.Ny * (lv.grid.Nz + 1) for lv in levels]
    kinds = ["spectral" if n > tail else "jacobi" for n in sizes]
    assert "jacobi" in kinds[:-1] and kinds[0] == "spectral"
    ref = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 2, 2, kinds, 0.4, "inject", 1.0, float(h.min()))
    T = wt.Tank(Nx, Ny, Nz, L, h, smoother=1, tail_max=tail, tail_cluster=cluster)
    scale = np.abs(ref).max()
    got = T.precondition(ea, eb, r, wt.WT_FP64)
    assert np.abs(got - ref).max() <= 1e-9 * scale
    got32 = T.precondition(ea, eb, r, wt.WT_FP32)
    assert np.abs(got32 - ref).max() <= 5e-3 * scale
    # and a mixed solve to the method's tolerance in the oracle's operator
    T.set_options(mode=wt.WT_MIXED, tol=1e-10, max_it=300, nu1=1, nu2=1)
    p, info = T.poisson_solve(ea, eb, r)
    res = r - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    assert np.linalg.norm(res) <= 1.5e-9 * np.linalg.norm(r)


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("Nx,Ny,Nz,smin", [(64, 64, 16, 8192), (1024, 1, 24, 3000)])
def test_spectral_min_parity(wt, Nx, Ny, Nz, smin, kind):
    # spectral sweeps (kind 1, or block-Jacobi then spectral, kind 2) on the
    # levels of at least spectral_min unknowns, block-Jacobi below, launch
    # per phase: against the oracle's V-cycle with those kinds by level
    L = 2 * math.pi
    g, h, ea, eb = curved(Nx, Ny, Nz, L)
    r = np.random.default_rng(7).standard_normal(g.shape)
    levels = pmg.build_levels(Nx, Ny, Nz, L, h, ea, eb, coarsest_max=64)
    sizes = [lv.grid.Nx * lv.grid.Ny * (lv.grid.Nz + 1) for lv in levels]
    kinds = [KINDS[kind] if n >= smin else "jacobi" for n in sizes]
    assert "jacobi" in kinds[:-1] and kinds[0] == KINDS[kind]
    ref = pmg.vcycle(levels, 0, np.zeros(g.shape), r, 2, 2, kinds, 0.4, "inject", 1.0, float(h.min()))
    T = wt.Tank(Nx, Ny, Nz, L, h, smoother=kind, spectral_min=smin)
    scale = np.abs(ref).max()
    assert np.abs(T.precondition(ea, eb, r, wt.WT_FP64) - ref).max() <= 1e-9 * scale
    assert np.abs(T.precondition(ea, eb, r, wt.WT_FP32) - ref).max() <= 5e-3 * scale
