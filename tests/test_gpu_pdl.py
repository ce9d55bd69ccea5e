"""Programmatic dependent launch (option `pdl`) changes when a kernel is made
resident, not what it computes: every kernel waits for its predecessor's
completion before it touches memory, so the step, the operator and the solve
give bit-identical results with the option on and off."""

import math

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    return w


def run_2d(wt, pdl, mode):
    Nx, Nz, L = 128, 16, 2 * math.pi
    x = np.arange(Nx) * L / Nx
    h = (1.0 - 0.3 * np.exp(-((x - L / 2) / 1.0) ** 2))[None]
    T = wt.Tank(Nx, 1, Nz, L, h, mode=mode, tol=1e-11, filter=1, pdl=pdl)
    _, _, sigma = T.grid()
    eta = si.stokes2_eta(x, 0.04, 1.0, 1.0)[None]
    d = h[0] + eta[0]
    z = sigma[:, None] * d[None, :] - h[0][None, :]
    u, w = si.linear_velocity(x[None, :], z, 0.04, 1.0, 1.0)
    T.set_state(np.ascontiguousarray(eta), np.ascontiguousarray(u[:, None, :]),
                np.zeros((Nz + 1, 1, Nx)), np.ascontiguousarray(w[:, None, :]))
    T.step(0.02, 3)
    out = T.get_state()[:4]
    its = T.stats()[1]
    T.close()
    return out, its


@pytest.mark.parametrize("mode", ["WT_MIXED", "WT_FP64", "WT_REFINE"])
def test_pdl_bit_identical_2d(wt, mode):
    a, ia = run_2d(wt, 1, getattr(wt, mode))
    b, ib = run_2d(wt, 0, getattr(wt, mode))
    assert ia == ib
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_pdl_bit_identical_3d(wt):
    N, Nz, L = 32, 8, 2 * math.pi
    x = np.arange(N) * L / N
    X, Y = np.meshgrid(x, x)
    h = 1.0 - 0.2 * np.exp(-((X - 3) ** 2 + (Y - 3.3) ** 2))
    ea = 0.05 * np.sin(X) * np.cos(2 * Y)
    rhs = np.random.default_rng(5).standard_normal((Nz + 1, N, N))
    res = []
    for pdl in (1, 0):
        T = wt.Tank(N, N, Nz, L, h, mode=wt.WT_MIXED, tol=1e-10, smoother=2, pdl=pdl)
        ap = T.apply_operator(ea, 0.9 * ea, rhs, wt.WT_FP32)
        p, info = T.poisson_solve(ea, 0.9 * ea, rhs)
        res.append((ap, p, info.iterations))
        T.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]
