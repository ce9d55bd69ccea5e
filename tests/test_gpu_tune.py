"""Solver autotuner (one of the batching / graph / tuning pieces of the hot
path): it must return a setting from its grid that reaches the tolerance, is
no slower than the options it started from, and is left active on the tank."""

import numpy as np
import pytest

from oracle import operator as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_00991_gb300 as wt
    return wt


@pytest.mark.parametrize("mode", [1, 0])
def test_autotune(wt, mode):
    from test_gpu_parity import curved
    Nx, Nz, L = 256, 16, 8.0
    g, h, ea, eb = curved(Nx, 1, Nz, L)
    b = np.random.default_rng(7).standard_normal(g.shape)
    T = wt.Tank(Nx, 1, Nz, L, h, mode=mode, tol=1e-10)
    opts, best, entry = T.autotune(ea, eb, b, reps=2)
    assert 0 < best <= entry
    assert opts["omega"] in (0.3, 0.4, 0.5, 0.6)
    assert (opts["nu1"], opts["nu2"]) in ((1, 1), (2, 2), (3, 3))
    assert opts["coarsest_max"] in (32, 64, 128)
    assert opts["mode"] in ((1, 3) if mode == 1 else (0,))
    assert opts["tol"] == 1e-10
    assert T.options() == opts
    p, info = T.poisson_solve(ea, eb, b)
    assert info.rel_residual <= 1e-10
    r = b - op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
    assert np.linalg.norm(r) <= 1.5e-9 * np.linalg.norm(b)
