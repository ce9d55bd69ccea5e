"""The benchmark's own workloads against the oracle, in the launch
configuration the benchmark times.

* The 2D nonlinear bar (1024 x 24, L = 32, Stokes-2 wave, exponential filter
  on): two full Runge-Kutta steps (ten mixed-stage Poisson solves) from the
  same seeded state on the GPU and in the oracle, compared element by element.
  The oracle solves every stage to 1e-11; the GPU's FP64 solver also to 1e-11,
  the mixed solver to the benchmark's 1e-10.  Bounds: 1e-10 (eta) and 1e-8
  (velocities) relative to the field's maximum; the solve tolerance reaches
  the velocities through the projection's gradient of p (Eq. rkforc1).
* The 3D directional sea (256 x 256 x 16, 4096 components) and the 256
  uneven tanks of the batched workload: too large for the oracle's solver,
  so a full GPU step is checked through properties that hold at any size -
  the projected velocity is discretely divergence-free and has no bottom
  flux in the oracle's own operator (Sec. 3.2, Eq. poissonp, bcpdneu), the
  mean of eta is conserved (mass, Eq. kinematicFS) - plus, for the batch,
  the smallest tanks of the seeded table against the oracle step.
"""

import math
import os
import sys

import numpy as np
import pytest

import seeded_inputs as si
from oracle import operator as op
from oracle import rk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402  (the benchmark's workload recipe, no GPU code at import)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    return w


@pytest.fixture(scope="module")
def bar_oracle():
    """Initial state and the oracle's state after 1 and 2 steps (filter on)."""
    p, x, h = bench.workload()
    tank = rk.Tank(p["Nx"], 1, p["Nz"], p["L"], h, tol=1e-11, coarsest_max=64, filter=True,
                   nu1=1, nu2=1, omega=0.5)
    st = bench.oracle_state(p, x, h)
    init = st.copy()
    out = []
    for _ in range(2):
        rk.step(tank, st, p["dt"])
        out.append(st.copy())
    return p, x, h, tank, init, out


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("mode,tol", [(0, 1e-11), (1, 1e-10)])
def test_bar_workload_two_steps_match_oracle(wt, bar_oracle, mode, tol):
    p, x, h, tank_o, init, ref = bar_oracle
    T = wt.Tank(p["Nx"], 1, p["Nz"], p["L"], h, mode=mode, tol=tol, filter=1)
    T.set_state(np.ascontiguousarray(init.eta), np.ascontiguousarray(init.u), np.zeros_like(init.u),
                np.ascontiguousarray(init.w))
    errs = []
    for n in range(2):
        T.step(p["dt"], 1)
        eta, u, v, w, tm = T.get_state()
        assert abs(tm - (n + 1) * p["dt"]) < 1e-14
        e = (_rel(eta, ref[n].eta), _rel(u, ref[n].u), _rel(w, ref[n].w))
        errs.append(e)
        assert e[0] <= 1e-10, (n, e)
        assert e[1] <= 1e-8 and e[2] <= 1e-8, (n, e)
    print("bar workload, mode %d: relative errors after 1, 2 steps (eta, u, w):" % mode, errs)
    # invariants of the discrete method in the oracle's operator
    dv, bot = rk.divergence_residual(tank_o, rk.State(tank_o.grid, eta, u, v, w))
    assert np.abs(dv).max() < 1e-6 and np.abs(bot).max() < 1e-8
    assert abs(eta.mean() - init.eta.mean()) < 1e-12
    T.close()


def test_sea3d_full_step_invariants(wt):
    N, Nz, L = 256, 16, 64.0
    T = wt.Tank(N, N, Nz, L, np.ones((N, N)), mode=wt.WT_MIXED, tol=1e-10, filter=1, omega=0.6, max_it=400)
    _, _, sigma = T.grid()
    sea = si.jonswap_sea(seed=3, L=L, ncomp=4096, kp=1.5, hs_over_lp=0.02)
    eta0, u0, v0, w0 = si.jonswap_fields(sea, N, sigma)
    T.set_state(*(np.ascontiguousarray(a) for a in (eta0, u0, v0, w0)))
    dt = 0.5 * (L / N) / math.sqrt(9.81)
    T.step(dt, 1)
    eta, u, v, w, tm = T.get_state()
    T.close()
    tank_o = rk.Tank(N, N, Nz, L, np.ones((N, N)))
    dv, bot = rk.divergence_residual(tank_o, rk.State(tank_o.grid, eta, u, v, w))
    vel = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    # |Div u| <= beta dt tol |b| at the last stage; |b| ~ |u| / (beta dt) per node
    # times the derivative scale (kappa_max ~ 12.6, CGL ~ Nz^2): a few 1e-8 vel
    assert np.abs(dv).max() < 1e-6 * vel
    assert np.abs(bot).max() < 1e-8 * vel
    # mass: the mean of eta moves only by the surface flux that the solve
    # tolerance leaves, five stages of ~tol * |eta|
    assert abs(eta.mean() - eta0.mean()) < 1e-9 * np.abs(eta0).max()
    assert np.isfinite(eta).all() and np.abs(eta - eta0).max() < 0.1


def _batch_inputs(tanks):
    st, hs = [], []
    for q in tanks:
        xq = np.arange(q["Nx"]) * q["L"] / q["Nx"]
        hq = si.bump(xq, q["L"], q["bump_A"], q["bump_w"])
        sig = (np.cos(np.pi * np.arange(q["Nz"] + 1) / q["Nz"]) + 1.0) / 2.0
        e, u, _, ww = bench.initial_state(q, xq, hq[None], sig)
        st.append((e, u, ww))
        hs.append(hq[None])
    return st, hs


def test_batch_workload_full_step(wt):
    tanks, _ = si.batch_tanks()
    st, hs = _batch_inputs(tanks)
    B = wt.Batch([q["Nx"] for q in tanks], [q["Nz"] for q in tanks], [q["L"] for q in tanks], hs, tol=1e-10)
    for i, s in enumerate(st):
        B.set_state(i, *s)
    dts = [q["dt"] for q in tanks]
    B.step(dts, 1)
    order = np.argsort([q["Nx"] * (q["Nz"] + 1) for q in tanks])
    for i in range(len(tanks)):
        q = tanks[i]
        e1, u1, w1, tm = B.get_state(i)
        assert abs(tm - q["dt"]) < 1e-14
        assert B.stats(i)[2] <= 1e-10
        assert abs(e1.mean() - st[i][0].mean()) < 1e-9 * np.abs(st[i][0]).max()
        if i in order[:64:8]:
            tank_o = rk.Tank(q["Nx"], 1, q["Nz"], q["L"], hs[i], tol=1e-10, filter=False)
            dv, bot = rk.divergence_residual(tank_o, rk.State(tank_o.grid, e1, u1, np.zeros_like(u1), w1))
            vel = max(np.abs(u1).max(), np.abs(w1).max())
            assert np.abs(dv).max() < 1e-6 * vel and np.abs(bot).max() < 1e-8 * vel, i
    # the two smallest tanks of the table against the oracle's step
    for i in order[:2]:
        q = tanks[i]
        e1, u1, w1, _ = B.get_state(i)
        tank_o = rk.Tank(q["Nx"], 1, q["Nz"], q["L"], hs[i], tol=1e-11, coarsest_max=64)
        so = rk.State(tank_o.grid, st[i][0], st[i][1], np.zeros_like(st[i][1]), st[i][2])
        rk.step(tank_o, so, q["dt"])
        assert _rel(e1, so.eta) <= 1e-10, i
        assert _rel(u1, so.u) <= 1e-8 and _rel(w1, so.w) <= 1e-8, i
    B.close()
