"""Pins of the learned-guess oracle (oracle/guess.py): the scaled network
output of Sec. 2.2's x0 = N(b) followed by damped-Jacobi sweeps."""
import math

import numpy as np

from oracle import direct, guess
from oracle import nn as onn
from synthetic import lognormal_kappa


def test_diagonal_matches_dense_matrices():
    n = 5
    assert np.allclose(guess.diagonal(2, n), np.diag(direct.dense_laplacian_2d(n)), rtol=1e-14)
    kap = lognormal_kappa(n, 5001, smooth_sigma=1.0)
    d = guess.diagonal(3, n, kap)
    assert np.allclose(d, np.diag(direct.dense_laplacian_3d(n, kap)), rtol=1e-13)
    assert np.allclose(guess.diagonal(3, n), np.diag(direct.dense_laplacian_3d(n)), rtol=1e-14)


def test_sweep_on_an_eigenmode_error_is_a_scaling():
    """2D: D = 4/h^2 I, so one sweep maps the error e = x - x* of an eigenvector
    of A with eigenvalue lambda to (1 - omega lambda / d) e, exactly."""
    n, omega = 12, 0.8
    h = 2.0 / (n + 1)
    d = 4.0 / (h * h)
    phi, _, lam = direct.eigen_pair_2d(n, 3, 2)
    rng = np.random.default_rng(1)
    xstar = rng.standard_normal(n * n)
    b = direct.dense_laplacian_2d(n) @ xstar
    x0 = xstar + 0.3 * phi
    for k in (1, 2, 5):
        xk = guess.jacobi(2, n, b, x0, k, omega)
        expect = xstar + 0.3 * (1.0 - omega * lam / d) ** k * phi
        assert np.linalg.norm(xk - expect) <= 1e-12 * np.linalg.norm(expect), k


def test_exact_solution_is_a_fixed_point():
    n = 6
    kap = lognormal_kappa(n, 5001, smooth_sigma=1.0)
    rng = np.random.default_rng(2)
    xstar = rng.standard_normal(n ** 3)
    b = direct.dense_laplacian_3d(n, kap) @ xstar
    x = guess.jacobi(3, n, b, xstar, 4, 0.7, kap)
    assert np.linalg.norm(x - xstar) <= 1e-12 * np.linalg.norm(xstar)
    # and a sweep moves any other x towards it in the A-norm (A SPD, omega <= 1)
    A = direct.dense_laplacian_3d(n, kap)
    x0 = xstar + rng.standard_normal(n ** 3)
    x1 = guess.jacobi(3, n, b, x0, 1, 0.7, kap)
    en = lambda e: math.sqrt(e @ A @ e)  # noqa: E731
    assert en(x1 - xstar) < en(x0 - xstar)


def test_without_sweeps_the_guess_is_the_scaled_network_output():
    n = 16
    rng = np.random.default_rng(3)
    params = {}
    for name, shape in onn.param_shapes(n, C=4):
        params[name] = 0.2 * rng.standard_normal(shape)
    b = rng.standard_normal(n * n) * 7.0
    s = onn.rms(b)
    y = onn.forward(params, b / s, n)
    x = guess.learned_guess(params, b, n, 1.7, 0, 0.8)
    assert np.allclose(x, 1.7 * s * y, rtol=1e-14, atol=0.0)
