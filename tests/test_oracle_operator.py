"""Pins of the oracle's operators (Sec. 1.4 discrete Laplacian, zero Dirichlet)
and of the DST-I direct solver against dense LU and closed forms."""
import math

import numpy as np
import pytest

from oracle import native, direct


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16])
def test_apply_2d_matches_dense(n):
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n * n)
    A = direct.dense_laplacian_2d(n)
    assert np.allclose(native.apply_2d(n, u), A @ u, rtol=1e-13, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("n", [1, 2, 3, 5])
@pytest.mark.parametrize("var", [False, True])
def test_apply_3d_matches_dense(n, var):
    rng = np.random.default_rng(10 + n)
    u = rng.standard_normal(n ** 3)
    kap = np.exp(rng.standard_normal(n ** 3)) if var else None
    A = direct.dense_laplacian_3d(n, kap)
    got = native.apply_3d(n, u, kap)
    assert np.allclose(got, A @ u, rtol=1e-12, atol=1e-12 * np.abs(A).max())


def test_3d_symmetric_positive():
    n = 10
    rng = np.random.default_rng(3)
    kap = np.exp(rng.standard_normal(n ** 3))
    u, v = rng.standard_normal((2, n ** 3))
    Au = native.apply_3d(n, u, kap)
    Av = native.apply_3d(n, v, kap)
    assert abs(u @ Av - Au @ v) <= 1e-12 * abs(u @ Av)
    assert u @ Au > 0


@pytest.mark.parametrize("n,p,q", [(7, 1, 1), (16, 2, 5), (33, 4, 3)])
def test_2d_eigenmode_closed_form(n, p, q):
    b, x, lam = direct.eigen_pair_2d(n, p, q)
    # lambda_pq = (4/h^2)(sin^2(p pi/2(n+1)) + sin^2(q pi/2(n+1)))
    h = 2.0 / (n + 1)
    lam2 = 4.0 / h ** 2 * (math.sin(p * math.pi / (2 * (n + 1))) ** 2
                           + math.sin(q * math.pi / (2 * (n + 1))) ** 2)
    assert abs(lam - lam2) <= 1e-12 * lam2
    assert np.allclose(native.apply_2d(n, x), b, rtol=0, atol=1e-12)


def test_3d_constant_kappa_eigenmode():
    n = 9
    k = np.arange(1, n + 1)
    s = [np.sin(p * math.pi * k / (n + 1)) for p in (1, 2, 3)]
    u = (s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]).reshape(-1)
    h = 2.0 / (n + 1)
    lam = 4.0 / h ** 2 * sum(math.sin(p * math.pi / (2 * (n + 1))) ** 2 for p in (1, 2, 3))
    assert np.allclose(native.apply_3d(n, u), lam * u, atol=1e-11 * lam)
    assert np.allclose(native.apply_3d(n, u, np.full(n ** 3, 2.5)), 2.5 * lam * u, atol=1e-10 * lam)


@pytest.mark.parametrize("n", [1, 4, 9, 16])
def test_dst_2d_vs_dense_lu(n):
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n * n)
    x = np.linalg.solve(direct.dense_laplacian_2d(n), b)
    assert np.allclose(direct.dst_solve_2d(n, b), x, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("n", [2, 5, 7])
def test_dst_3d_vs_dense_lu(n):
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n ** 3)
    x = np.linalg.solve(direct.dense_laplacian_3d(n), b)
    assert np.allclose(direct.dst_solve_3d(n, b), x, rtol=1e-11, atol=1e-13)


def test_dst_large_residual():
    n = 256
    rng = np.random.default_rng(0)
    b = rng.standard_normal(n * n)
    x = direct.dst_solve_2d(n, b)
    r = b - native.apply_2d(n, x)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b)
