"""Batched uneven 2D tanks (one persistent launch, one CTA per tank) against
the host-driven single-tank path and against the oracle's Runge-Kutta step
(Sec. 4.1 low-storage RK4, Eq. kinematicFS, forc1, poissonp, rkforc1), in the
mixed form (FP32 V-cycle) and the plain FP64 form."""

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
        pytest.skip("no CUDA device")
    import paper_2406_00991_gb300 as wt
    return wt


def wave_tank(Nx, Nz, L, amp, m=1, bump=0.3, seed=0):
    """Bathymetry, eta, u, w of a second-order wave of m wavelengths over a bump."""
    rng = np.random.default_rng(seed)
    x = np.arange(Nx) * L / Nx
    x0 = L * (0.3 + 0.4 * rng.random())
    h = (1.0 - bump * np.exp(-((x - x0) / (0.1 * L)) ** 2))[None]
    k = 2 * math.pi * m / L
    g = op.Grid(Nx, 1, Nz, L)
    eta = si.stokes2_eta(x, amp, k, 1.0)[None]
    geo = op.Geometry(g, h, eta)
    u, w = si.linear_velocity(x[None, None, :], geo.z_nodes(g), amp, k, 1.0)
    return h, np.ascontiguousarray(eta), np.ascontiguousarray(u), np.ascontiguousarray(w)


def single(wt, Nx, Nz, L, h, eta, u, w, dt, nsteps, **opt):
    T = wt.Tank(Nx, 1, Nz, L, h, **opt)
    T.set_state(eta, u, np.zeros_like(u), w)
    T.step(dt, nsteps)
    e, uu, _, ww, tm = T.get_state()
    its = T.stats()
    T.close()
    return e, uu, ww, tm, its


def close(a, b, rel):
    return np.abs(a - b).max() <= rel * max(np.abs(b).max(), 1e-30)


SHAPES = [(64, 12, 2 * math.pi, 0.03, 1), (256, 24, 8.0, 0.05, 2), (128, 16, 4.0, 0.02, 1),
          (1024, 24, 32.0, 0.15, 5), (32, 8, 1.0, 0.004, 1)]


@pytest.mark.parametrize("opts", [dict(), dict(filter=1), dict(linear=1), dict(mode=0), dict(mode=0, filter=1),
                                  dict(mode=3, inner_tol=1e-4), dict(mode=3, filter=1)])
def test_batch_matches_single_tanks(wt, opts):
    # uneven tanks, including the 1024 x 24 tank and a 32 x 8 one; 1e-10 is the
    # method's solve tolerance (1e-12 lies below the FP64 rounding floor of the
    # larger tanks' residual, for the host-driven path as well)
    tanks = [wave_tank(Nx, Nz, L, a, m, seed=i) for i, (Nx, Nz, L, a, m) in enumerate(SHAPES)]
    dts = [0.2 * L / Nx / math.sqrt(9.81) for Nx, _, L, _, _ in SHAPES]
    B = wt.Batch([s[0] for s in SHAPES], [s[1] for s in SHAPES], [s[2] for s in SHAPES],
                 [t[0] for t in tanks], tol=1e-10, **opts)
    for i, (h, eta, u, w) in enumerate(tanks):
        B.set_state(i, eta, u, w)
    B.step(dts, 2)
    for i, ((Nx, Nz, L, _, _), (h, eta, u, w)) in enumerate(zip(SHAPES, tanks)):
        e1, u1, w1, t1 = B.get_state(i)
        o = dict(opts)
        o.setdefault("mode", 1)
        e2, u2, w2, t2, (solves, its) = single(wt, Nx, Nz, L, h, eta, u, w, dts[i], 2, tol=1e-10, **o)
        assert abs(t1 - 2 * dts[i]) < 1e-14 and abs(t2 - t1) < 1e-14
        assert close(e1, e2, 1e-10), (i, np.abs(e1 - e2).max())
        assert close(u1, u2, 1e-8), (i, np.abs(u1 - u2).max())
        assert close(w1, w2, 1e-8), (i, np.abs(w1 - w2).max())
        bs, bits, brel = B.stats(i)
        assert bs == 10 == solves
        assert brel <= 1e-10
        # same method, reductions in another order; the refinement form's FP32
        # inner solves react more to that order (they restart every refinement)
        assert abs(bits - its) <= (10 if o["mode"] != 3 else max(10, its // 2))
    B.close()


@pytest.mark.parametrize("mode", [1, 0, 3])
def test_batch_matches_oracle_step(wt, mode):
    Nx, Nz, L = 64, 12, 2 * math.pi
    h, eta, u, w = wave_tank(Nx, Nz, L, 0.03)
    dt = 0.01
    B = wt.Batch([Nx], [Nz], [L], [h], tol=1e-12, mode=mode)
    B.set_state(0, eta, u, w)
    B.step([dt], 1)
    e1, u1, w1, _ = B.get_state(0)
    g = op.Grid(Nx, 1, Nz, L)
    tank_o = rk.Tank(Nx, 1, Nz, L, h, tol=1e-13, coarsest_max=64)
    st = rk.State(g, eta.copy(), u.copy(), np.zeros_like(u), w.copy())
    rk.step(tank_o, st, dt)
    assert close(e1, st.eta, 1e-10)
    assert close(u1, st.u, 1e-8)
    assert close(w1, st.w, 1e-8)
    dv, bot = rk.divergence_residual(tank_o, rk.State(g, e1, u1, np.zeros_like(u1), w1))
    assert np.abs(dv).max() < 1e-7 and np.abs(bot).max() < 1e-9
    B.close()


def test_batch_more_tanks_than_sms(wt):
    # 200 tanks of 32 x 8 (more CTAs than SMs); each must equal its own batch of one
    n, Nx, Nz, L = 200, 32, 8, 2 * math.pi
    amps = 0.001 + 0.04 * np.arange(n) / n
    tanks = [wave_tank(Nx, Nz, L, a, seed=i) for i, a in enumerate(amps)]
    B = wt.Batch([Nx] * n, [Nz] * n, [L] * n, [t[0] for t in tanks], tol=1e-12)
    for i, (h, eta, u, w) in enumerate(tanks):
        B.set_state(i, eta, u, w)
    B.step(0.01, 1)
    for i in (0, 151, 152, 199):
        h, eta, u, w = tanks[i]
        one = wt.Batch([Nx], [Nz], [L], [h], tol=1e-12)
        one.set_state(0, eta, u, w)
        one.step(0.01, 1)
        a, b = B.get_state(i), one.get_state(0)
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y), i      # the same CTA code on the same data
        one.close()
    B.close()


def test_batch_errors(wt):
    h = np.ones((1, 64))
    with pytest.raises(wt.WtError) as e:
        wt.Batch([4096], [8], [1.0], [np.ones((1, 4096))])
    assert e.value.code == wt.WT_ENOTSUP
    B = wt.Batch([64], [8], [1.0], [h])
    with pytest.raises(wt.WtError) as e:
        B.step(0.01, 1)                                     # no state yet
    assert e.value.code == wt.WT_EINVAL
    eta = np.zeros((1, 64))
    u = np.zeros((9, 1, 64))
    B.set_state(0, eta, u, u)
    with pytest.raises(wt.WtError) as e:
        B.step(-0.01, 1)
    assert e.value.code == wt.WT_EINVAL
    with pytest.raises(wt.WtError) as e:
        B.set_options(smoother=1)
    assert e.value.code == wt.WT_ENOTSUP
    # still water stays still; zero right-hand sides take zero iterations
    B.step(0.01, 3)
    e1, u1, w1, tm = B.get_state(0)
    assert np.abs(e1).max() == 0 and np.abs(u1).max() == 0 and np.abs(w1).max() == 0
    assert abs(tm - 0.03) < 1e-15
    assert B.stats(0)[:2] == (15, 0)
    B.close()
