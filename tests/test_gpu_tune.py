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


@pytest.mark.parametrize("mode", [1, 0])
def test_batch_autotune(wt, mode):
    # a small uneven batch: the tuner keeps the batch's mode, returns a grid
    # point no slower than the entry options, leaves it active and restores
    # every tank's state
    from test_gpu_batch import wave_tank
    shapes = [(64, 12, 2 * np.pi, 0.03, 1), (256, 24, 8.0, 0.05, 2), (128, 16, 4.0, 0.02, 1)]
    tanks = [wave_tank(Nx, Nz, L, a, m, seed=i) for i, (Nx, Nz, L, a, m) in enumerate(shapes)]
    B = wt.Batch([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], [t[0] for t in tanks],
                 tol=1e-10, mode=mode)
    for i, (h, eta, u, w) in enumerate(tanks):
        B.set_state(i, eta, u, w)
    dts = [0.2 * s[2] / s[0] / np.sqrt(9.81) for s in shapes]
    opts, best, entry = B.autotune(dts, reps=1)
    assert 0 < best <= entry
    assert opts["mode"] == mode and opts["omega"] in (0.3, 0.4, 0.5, 0.6)
    assert (opts["nu1"], opts["nu2"]) in ((1, 1), (2, 2))
    assert B.options() == opts
    for i, (h, eta, u, w) in enumerate(tanks):
        e1, u1, w1, tm = B.get_state(i)
        assert tm == 0.0 and np.array_equal(e1, eta) and np.array_equal(u1, u)
    B.step(dts, 1)
    for i in range(len(shapes)):
        assert B.stats(i)[2] <= 1e-10
    B.close()


def test_autotune_cache(wt, tmp_path):
    # a completed search is written to the file under its key; a second tank
    # of the same grid and settings takes the stored options without
    # measuring (no step runs: the solver statistics stay at zero)
    import json
    from test_gpu_parity import curved
    path = tmp_path / "tuned.jsonl"
    assert wt.wt_autotune_cache(str(path)) == wt.WT_OK
    try:
        Nx, Nz, L = 128, 12, 8.0
        g, h, ea, eb = curved(Nx, 1, Nz, L)
        z = np.zeros(g.shape)
        eta = np.ascontiguousarray(0.01 * np.cos(2 * np.pi * g.x / L)[None, :])

        def tank():
            T = wt.Tank(Nx, 1, Nz, L, h, mode=1, tol=1e-10, filter=1)
            T.set_state(eta, z, z, z)
            return T

        A = tank()
        opts, best, entry = A.autotune_step(0.01, reps=1)
        lines = path.read_text().splitlines()
        assert len(lines) == 1
        rec = json.loads(lines[0])
        assert rec["key"].startswith("step 128x1x12 fp64=0 filter=1 linear=0")
        assert (rec["omega"], rec["nu1"], rec["smoother"], rec["spectral_min"], rec["omega_s"]) == \
            (opts["omega"], opts["nu1"], opts["smoother"], opts["spectral_min"], opts["omega_s"])
        B = tank()
        opts2, best2, entry2 = B.autotune_step(0.01, reps=1)
        assert B.stats() == (0, 0)
        assert opts2 == opts and (best2, entry2) == (pytest.approx(best), pytest.approx(entry))
        # another grid is a different key: searched and appended
        C = wt.Tank(64, 1, 12, L, np.ascontiguousarray(h[:, ::2]), mode=1, tol=1e-10, filter=1)
        C.set_state(np.ascontiguousarray(eta[:, ::2]), np.zeros((13, 1, 64)), np.zeros((13, 1, 64)),
                    np.zeros((13, 1, 64)))
        C.autotune_step(0.01, reps=1)
        assert len(path.read_text().splitlines()) == 2
    finally:
        wt.wt_autotune_cache(None)
