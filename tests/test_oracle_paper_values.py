"""The constants the paper prints, read from tests/golden/paper_constants.json
(each with its section / table), and the Table 1 sanity band.  CPU only."""

import json
import math
import os

import numpy as np

from oracle import krylov, spectral as sp
import seeded_inputs as si

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_filter_uses_the_printed_parameters():
    f = GOLD["filter"]
    N = 40
    Nc = int(math.floor(f["Nc_chebyshev_fraction"] * N))
    resp = sp.filter_response(np.arange(N + 1), N, Nc)
    want = np.exp(-f["alpha"] * ((np.arange(N + 1) - Nc) / (N + 1 - Nc)) ** f["s"])
    want[: Nc + 1] = 1.0
    assert np.allclose(resp, want, rtol=0, atol=1e-15)


def test_battjes_limit_constants():
    b = GOLD["battjes"]
    for kh in (0.5, 2.0, 2 * math.pi):
        assert abs(si.battjes_limit(kh) - b["coefficient"] * math.tanh(b["kh_factor"] * kh)) < 1e-15


def test_gravity_of_the_inputs():
    assert si.G == GOLD["g"]


def test_table1_iteration_band():
    # Table 1: p-MG preconditioning cuts GMRES iterations from ~1e3 to a handful.
    # On a 40-node-class 2D tank (Nx = 32, Nz = 40 here: power-of-two Fourier grid)
    # the preconditioned count to 1e-8 must sit within 10x of the printed 4, and
    # unpreconditioned GMRES(30) must need more than 20x as many iterations.
    t = GOLD["table1"]
    Nx, Nz, L = 32, 40, 2 * math.pi
    x = sp.fourier_nodes(Nx, L)
    h = np.ones(Nx)
    eta = 0.05 * np.cos(x)
    rng = np.random.default_rng(11)
    b = rng.standard_normal((Nz + 1, 1, Nx))
    _, its, _, _ = krylov.solve_pmg(Nx, 1, Nz, L, h, eta, eta, b, tol=t["rel_error"][1])
    assert its <= 10 * t["vcycle_gmres_iterations"][1]
    _, its0, _, _ = krylov.solve_pmg(Nx, 1, Nz, L, h, eta, eta, b, tol=t["rel_error"][1],
                                     precondition=False, maxit=20 * its + 1)
    assert its0 > 20 * its
