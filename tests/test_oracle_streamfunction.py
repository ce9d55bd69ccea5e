"""Pins of the oracle's stream-function waves (Rienecker & Fenton's method, the
initial condition of the paper's Sec. 5.2 accuracy study), by properties the
exact steady wave must have and by classical limits, none of which restates
the solver's own equations at its collocation points:

* linear limit: speed sqrt(g/k tanh kh), surface (H/2) cos kx;
* Stokes' deep-water third-order speed c = sqrt(g/k) (1 + (ka)^2 / 2);
* Stokes' second-order harmonic k a^2 cosh kh (2 + cosh 2kh) / (4 sinh^3 kh);
* between the collocation points, the surface is a streamline of the flow
  seen in the wave's frame ((u - c) eta_x = w) and Bernoulli's constant is
  the same along it;
* zero mean level, crest-to-trough height H.
CPU only."""

import math

import numpy as np
import pytest

from oracle import streamfunction as sf

G = 9.81


def test_linear_limit():
    for kh in (0.5, 2.0, 6.0):
        k, d, H = kh, 1.0, 1e-5
        W = sf.solve(k, d, H, N=16)
        c0 = math.sqrt(G / k * math.tanh(kh))
        assert abs(W.c / c0 - 1.0) < 1e-8
        x = np.linspace(0, 2 * math.pi / k, 37)
        # the second harmonic is O(k H) relative to the first (below 1e-4 here)
        assert np.abs(W.eta(x) - 0.5 * H * np.cos(k * x)).max() < 1e-4 * H


def test_stokes_deep_water_speed():
    k, d = 1.0, 10.0                    # tanh(kh) = 1 - 4e-9
    for ka in (0.02, 0.05, 0.08):
        W = sf.solve(k, d, 2 * ka / k, N=24)
        c0 = math.sqrt(G / k)
        assert abs(W.c / c0 - (1.0 + 0.5 * ka ** 2)) < 3.0 * ka ** 4, ka


def test_stokes_second_harmonic():
    for kh in (0.8, 1.5):
        k, d = kh, 1.0
        a = 0.01
        W = sf.solve(k, d, 2 * a, N=24)
        want = k * a * a * math.cosh(kh) * (2 + math.cosh(2 * kh)) / (4 * math.sinh(kh) ** 3)
        assert abs(W.E[2] / want - 1.0) < 0.05, (kh, W.E[2], want)


@pytest.mark.parametrize("kh,frac", [(0.5, 0.5), (2.0, 0.5), (2 * math.pi, 0.5), (2.0, 0.7)])
def test_surface_conditions_between_the_nodes(kh, frac):
    d = 1.0
    k = kh / d
    H = frac * 0.1401 * math.tanh(0.8863 * kh) * 2 * math.pi / k
    W = sf.solve(k, d, H, N=32)
    # points between the N + 1 collocation points
    X = (np.arange(200) + 0.37) * (2 * math.pi / k) / 200
    j = np.arange(W.N + 1)
    eta = W.eta(X)
    eta_x = -(np.sin(np.multiply.outer(X, j * k)) * (j * k)) @ W.E
    u, w = W.velocity(X, eta)
    # kinematic: the surface is a streamline of the steady flow (frame of the wave)
    scale = W.c * np.abs(eta_x).max()
    assert np.abs((u - W.c) * eta_x - w).max() < 1e-8 * scale
    # dynamic: Bernoulli's constant along the surface
    B = 0.5 * ((u - W.c) ** 2 + w ** 2) + G * eta
    assert (B.max() - B.min()) < 1e-8 * G * H
    assert abs(eta.mean()) < 1e-12 * H
    assert abs(W.eta(0.0) - W.eta(math.pi / k) - H) < 1e-12 * H
    # the crest is higher above the mean than the trough is below (nonlinear)
    assert W.eta(0.0) > 0.5 * H
