"""Failure paths of the C ABI (status codes WT_ENOCONV, WT_EBREAK, WT_ETIMEOUT,
WT_EINVAL), each made without a GPU fault: an iteration cap, a non-finite
host input, a grid-barrier wait bound of a few cycles (every wait in the
one-launch V-cycle is bounded and returns, so the kernel ends and the tank
stays usable).  After each failure the same tank must solve correctly."""

import numpy as np
import pytest

from oracle import operator as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    return w


def _problem(Nx=256, Nz=16, L=8.0, seed=3):
    g = op.Grid(Nx, 1, Nz, L)
    x = g.x
    h = (1.0 - 0.3 * np.exp(-((x - L / 2) / (L / 8)) ** 2))[None]
    ea = (0.05 * np.cos(2 * np.pi * x / L))[None]
    eb = ea * 0.99
    b = np.random.default_rng(seed).standard_normal(g.shape)
    return g, np.ascontiguousarray(h), np.ascontiguousarray(ea), np.ascontiguousarray(eb), b


def _residual(g, h, ea, eb, b, p):
    r = b - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_iteration_cap_gives_enoconv_and_best_iterate(wt, mode):
    g, h, ea, eb, b = _problem()
    T = wt.Tank(g.Nx, 1, g.Nz, g.L, h, mode=mode, tol=1e-11, max_it=1, max_ir=1)
    with pytest.raises(wt.WtError) as e:
        T.poisson_solve(ea, eb, b)
    assert e.value.code == wt.WT_ENOCONV
    p, info = T.poisson_solve(ea, eb, b, raise_noconv=False)
    assert info.status == wt.WT_ENOCONV and info.iterations == 1
    # the iterate written back is the one whose residual the call reports
    rel = _residual(g, h, ea, eb, b, p)
    assert rel < 1.0 and abs(rel - info.rel_residual) <= 1e-6 * rel
    T.set_options(max_it=200, max_ir=30)
    p, info = T.poisson_solve(ea, eb, b)
    assert _residual(g, h, ea, eb, b, p) <= 1.5e-11


def test_non_finite_host_inputs_give_ebreak(wt):
    g, h, ea, eb, b = _problem()
    T = wt.Tank(g.Nx, 1, g.Nz, g.L, h, mode=1, tol=1e-10)
    bad = b.copy()
    bad[3, 0, 17] = np.nan
    with pytest.raises(wt.WtError) as e:
        T.poisson_solve(ea, eb, bad)
    assert e.value.code == wt.WT_EBREAK
    inf_eta = ea.copy()
    inf_eta[0, 5] = np.inf
    with pytest.raises(wt.WtError) as e:
        T.poisson_solve(inf_eta, eb, b)
    assert e.value.code == wt.WT_EBREAK
    # a state with a NaN velocity breaks the next stage
    u = np.zeros(g.shape)
    u[4, 0, 9] = np.nan
    T.set_state(np.ascontiguousarray(ea), u, np.zeros(g.shape), np.zeros(g.shape))
    with pytest.raises(wt.WtError) as e:
        T.rk_stage(1, 1e-3)
    assert e.value.code == wt.WT_EBREAK
    # the tank stays usable
    p, info = T.poisson_solve(ea, eb, b)
    assert _residual(g, h, ea, eb, b, p) <= 1.5e-10
    T.set_state(np.ascontiguousarray(ea), np.zeros(g.shape), np.zeros(g.shape), np.zeros(g.shape))
    T.rk_stage(1, 1e-3)


def test_grid_barrier_bound_gives_etimeout_then_recovers(wt):
    # the cooperative one-launch V-cycle with a wait bound of a few cycles: the
    # first CTA to arrive at a grid barrier gives up, sets the abort word and
    # returns; every other CTA returns at its next barrier
    g, h, ea, eb, b = _problem(1024, 24, 32.0)
    T = wt.Tank(g.Nx, 1, g.Nz, g.L, h, mode=1, tol=1e-10, vcycle_grid=1, barrier_cycles=64, max_it=3)
    with pytest.raises(wt.WtError) as e:
        T.poisson_solve(ea, eb, b)
    assert e.value.code == wt.WT_ETIMEOUT
    assert "barrier" in str(e.value)
    # default bound again: the barrier state was reset, the same tank converges
    T.set_options(barrier_cycles=0, max_it=200)
    p, info = T.poisson_solve(ea, eb, b)
    assert info.rel_residual <= 1e-10
    assert _residual(g, h, ea, eb, b, p) <= 1.5e-10
    with pytest.raises(wt.WtError) as e:
        T.set_options(barrier_cycles=-1)
    assert e.value.code == wt.WT_EINVAL


def test_invalid_arguments(wt):
    h = np.ones((1, 64))
    for args in [(63, 1, 8), (64, 2, 8), (64, 1, 1), (64, 1, 33), (8192, 1, 8)]:
        Nx, Ny, Nz = args
        with pytest.raises(wt.WtError) as e:
            wt.Tank(Nx, Ny, Nz, 1.0, np.ones((Ny, Nx)))
        assert e.value.code == wt.WT_EINVAL, args
    with pytest.raises(wt.WtError) as e:
        wt.Tank(64, 1, 8, 1.0, -h)
    assert e.value.code == wt.WT_EINVAL
    T = wt.Tank(64, 1, 8, 1.0, h)
    for bad in [dict(tol=0.0), dict(restart=40), dict(omega=2.5), dict(nu1=0, nu2=0), dict(mode=9),
                dict(coarsest_max=500)]:
        with pytest.raises(wt.WtError) as e:
            T.set_options(**bad)
        assert e.value.code == wt.WT_EINVAL, bad
    with pytest.raises(wt.WtError) as e:
        T.rk_stage(1, 0.01)                      # no state yet
    assert e.value.code == wt.WT_EINVAL
    with pytest.raises(wt.WtError) as e:
        T.rk_stage(6, 0.01)
    assert e.value.code == wt.WT_EINVAL
