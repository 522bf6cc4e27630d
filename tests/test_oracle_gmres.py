"""Pins of the FP64 GMRES(m) oracle: restarted GMRES (Sec. 1.2) against dense
LU, closed-form eigenpairs, brute-force Krylov least squares, the Arnoldi
relation, orthonormality, residual monotonicity and full-GMRES termination."""
import math

import numpy as np
import pytest

from oracle import native, direct
from synthetic import MovingGaussians2D


def test_eigenmode_converges_in_one_iteration():
    n = 32
    b, x_exact, _ = direct.eigen_pair_2d(n, 3, 2)
    x, st, _ = native.gmres(2, n, b, m=20, rtol=1e-12)
    assert st["status"] == 0 and st["iters"] == 1
    assert np.linalg.norm(x - x_exact) <= 1e-12 * np.linalg.norm(x_exact)


@pytest.mark.parametrize("n,m", [(4, 3), (8, 5), (12, 10), (16, 20)])
def test_vs_dense_lu(n, m):
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n * n)
    x_lu = np.linalg.solve(direct.dense_laplacian_2d(n), b)
    x, st, _ = native.gmres(2, n, b, m=m, rtol=1e-12)
    assert st["status"] == 0 and st["relres_true"] <= 1e-12
    assert np.linalg.norm(x - x_lu) <= 1e-9 * np.linalg.norm(x_lu)


@pytest.mark.parametrize("n,k", [(5, 3), (6, 4), (8, 5)])
def test_first_cycle_is_krylov_minimiser(n, k):
    rng = np.random.default_rng(100 + n)
    A = direct.dense_laplacian_2d(n)
    b = rng.standard_normal(n * n)
    x0 = rng.standard_normal(n * n) * 0.01
    best = direct.krylov_min_residual(A, b, x0, k)
    _, st, _ = native.gmres(2, n, b, m=k, rtol=1e-15, max_iters=k, x0=x0)
    assert st["cycles"] == 1 and st["status"] == 1
    got = st["relres_first_cycle"] * st["bnorm"]
    assert abs(got - best) <= 1e-10 * best


def test_arnoldi_relation_and_orthonormality():
    n, m = 16, 20
    rng = np.random.default_rng(1)
    v0 = rng.standard_normal(n * n)
    V, H, steps = native.arnoldi(2, n, v0, m)
    assert steps == m
    A = direct.dense_laplacian_2d(n)
    lhs = A @ V[:m].T
    rhs = V.T @ H
    normA = np.linalg.norm(A, 2)
    assert np.linalg.norm(lhs - rhs, 2) <= 1e-12 * normA
    G = V @ V.T
    assert np.abs(G - np.eye(m + 1)).max() <= 1e-12
    # H is upper Hessenberg with a positive subdiagonal
    assert np.all(np.tril(H, -2) == 0) and np.all(np.diag(H, -1) > 0)


def test_arnoldi_3d_variable_kappa():
    n, m = 6, 12
    rng = np.random.default_rng(2)
    kap = np.exp(rng.standard_normal(n ** 3))
    v0 = rng.standard_normal(n ** 3)
    V, H, steps = native.arnoldi(3, n, v0, m, kappa=kap)
    A = direct.dense_laplacian_3d(n, kap)
    assert np.linalg.norm(A @ V[:steps].T - V[:steps + 1].T @ H[:steps + 1, :steps], 2) \
        <= 1e-12 * np.linalg.norm(A, 2)


def test_residuals_monotone():
    n, m = 32, 20
    b = MovingGaussians2D(n, 1001, 50).rhs(0)
    x, st, hist = native.gmres(2, n, b, m=m, rtol=1e-8, hist_cap=100000)
    assert st["status"] == 0 and st["relres_true"] <= 1e-8
    assert len(hist) == st["iters"]
    # within every cycle the least-squares residual never grows
    for c in range(0, len(hist), m):
        seg = hist[c:c + m]
        assert np.all(np.diff(seg) <= 1e-12 * seg[0])
    # across restarts the implicit residual keeps falling (small slack for rounding)
    starts = hist[m - 1::m]
    assert np.all(np.diff(starts) <= 1e-10)


def test_full_gmres_terminates_within_distinct_eigenvalues():
    n = 6
    lam1 = [4 * math.sin(p * math.pi / (2 * (n + 1))) ** 2 for p in range(1, n + 1)]
    distinct = len({round(a + b, 12) for a in lam1 for b in lam1})
    rng = np.random.default_rng(3)
    b = rng.standard_normal(n * n)
    _, st, _ = native.gmres(2, n, b, m=n * n, rtol=1e-10)
    assert st["status"] == 0 and st["iters"] <= distinct


def test_zero_rhs_and_iteration_cap():
    n = 16
    x, st, _ = native.gmres(2, n, np.zeros(n * n), m=10, rtol=1e-10, x0=np.ones(n * n))
    assert st["status"] == 0 and st["iters"] == 0 and np.all(x == 0)
    b = MovingGaussians2D(n, 5, 10).rhs(0)
    _, st, _ = native.gmres(2, n, b, m=5, rtol=1e-14, max_iters=12)
    assert st["status"] == 1 and st["iters"] == 12 and st["relres_true"] > 1e-14


def test_3d_vs_dst_and_dense():
    n = 8
    rng = np.random.default_rng(4)
    b = rng.standard_normal(n ** 3)
    x, st, _ = native.gmres(3, n, b, m=30, rtol=1e-12)
    assert np.linalg.norm(x - direct.dst_solve_3d(n, b)) <= 1e-9 * np.linalg.norm(x)
    n = 5
    kap = np.exp(rng.standard_normal(n ** 3))
    b = rng.standard_normal(n ** 3)
    x, st, _ = native.gmres(3, n, b, m=30, rtol=1e-12, kappa=kap)
    x_lu = np.linalg.solve(direct.dense_laplacian_3d(n, kap), b)
    assert np.linalg.norm(x - x_lu) <= 1e-9 * np.linalg.norm(x_lu)


def test_config1_against_dst():
    """32^2, GMRES(20), rtol 1e-8, moving Gaussian sources: the true-residual
    certificate and the error against the exact DST solution."""
    n = 32
    gen = MovingGaussians2D(n, 1001, 50)
    for t in (0, 25, 49):
        b = gen.rhs(t)
        x, st, _ = native.gmres(2, n, b, m=20, rtol=1e-8)
        assert st["status"] == 0 and st["relres_true"] <= 1e-8
        xe = direct.dst_solve_2d(n, b)
        assert np.linalg.norm(x - xe) <= 1e-5 * np.linalg.norm(xe)
        assert st["relres_first_cycle"] >= st["relres_true"]


def test_guess_warm_start():
    n = 32
    b = MovingGaussians2D(n, 1001, 50).rhs(3)
    xe = direct.dst_solve_2d(n, b)
    _, st0, _ = native.gmres(2, n, b, m=20, rtol=1e-8)
    _, st1, _ = native.gmres(2, n, b, m=20, rtol=1e-8, x0=xe * (1 + 1e-3))
    assert st1["iters"] < st0["iters"]
    assert abs(st1["relres_guess"] - 1e-3) < 1e-6
