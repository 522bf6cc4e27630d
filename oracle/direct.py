"""Direct FP64 solutions that pin the GMRES oracle from outside.

TEST INFRASTRUCTURE ONLY.

* ``dense_laplacian_2d/3d``: the operator matrix assembled entry by entry from
  the stencil definition (discrete Laplacian with zero-Dirichlet walls, Sec. 1.4
  and Sec. 3), for small grids.
* ``dst_solve_2d/3d``: the fast Poisson solver for constant coefficients.  The
  1D operator tridiag(-1, 2, -1) has eigenvectors sin(j k pi/(n+1)) and
  eigenvalues 4 sin^2(k pi/(2(n+1))), so A = (1/h^2) sum of Kronecker terms is
  diagonalised by the type-I sine transform in every axis.  scipy's DST-I is
  its own inverse up to the factor 2(n+1) per axis.
* ``eigen_pair_2d``: the closed-form eigenpair b = sin*sin, x = b / lambda_pq.
* ``krylov_min_residual``: brute-force min_y ||b - A(x0 + K y)|| over the
  explicit Krylov basis [r, Ar, ..., A^{k-1} r] by QR least squares, the value
  one GMRES cycle of k steps attains in exact arithmetic.
"""

import math

import numpy as np
import scipy.fft


def _scale(n):
    h = 2.0 / (n + 1)
    return 1.0 / (h * h)


def dense_laplacian_2d(n):
    N = n * n
    A = np.zeros((N, N))
    s = _scale(n)
    for iy in range(n):
        for ix in range(n):
            r = iy * n + ix
            A[r, r] = 4.0 * s
            if ix > 0:
                A[r, r - 1] = -s
            if ix < n - 1:
                A[r, r + 1] = -s
            if iy > 0:
                A[r, r - n] = -s
            if iy < n - 1:
                A[r, r + n] = -s
    return A


def dense_laplacian_3d(n, kappa=None):
    """-div(kappa grad) with harmonic-mean face coefficients; on a wall face the
    coefficient is the cell's own kappa and the outside value is 0."""
    N = n ** 3
    kap = np.ones(N) if kappa is None else np.asarray(kappa, dtype=np.float64)
    A = np.zeros((N, N))
    s = _scale(n)
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                r = (iz * n + iy) * n + ix
                for (d, ok) in (((0, 0, -1), ix > 0), ((0, 0, 1), ix < n - 1),
                                ((0, -1, 0), iy > 0), ((0, 1, 0), iy < n - 1),
                                ((-1, 0, 0), iz > 0), ((1, 0, 0), iz < n - 1)):
                    if ok:
                        c = ((iz + d[0]) * n + (iy + d[1])) * n + (ix + d[2])
                        kf = 2.0 * kap[r] * kap[c] / (kap[r] + kap[c])
                        A[r, r] += s * kf
                        A[r, c] -= s * kf
                    else:
                        A[r, r] += s * kap[r]
    return A


def _lam1d(n):
    k = np.arange(1, n + 1, dtype=np.float64)
    return 4.0 * np.sin(k * math.pi / (2.0 * (n + 1))) ** 2


def dst_solve_2d(n, b):
    B = np.asarray(b, dtype=np.float64).reshape(n, n)
    lam = _lam1d(n)
    Bh = scipy.fft.dst(scipy.fft.dst(B, type=1, axis=0), type=1, axis=1)
    Uh = Bh / (_scale(n) * (lam[:, None] + lam[None, :]))
    U = scipy.fft.dst(scipy.fft.dst(Uh, type=1, axis=0), type=1, axis=1) / (2.0 * (n + 1)) ** 2
    return U.reshape(-1)


def dst_solve_3d(n, b):
    B = np.asarray(b, dtype=np.float64).reshape(n, n, n)
    lam = _lam1d(n)
    Bh = B
    for ax in range(3):
        Bh = scipy.fft.dst(Bh, type=1, axis=ax)
    Uh = Bh / (_scale(n) * (lam[:, None, None] + lam[None, :, None] + lam[None, None, :]))
    U = Uh
    for ax in range(3):
        U = scipy.fft.dst(U, type=1, axis=ax)
    return (U / (2.0 * (n + 1)) ** 3).reshape(-1)


def eigen_pair_2d(n, p, q):
    """b = sin(p pi i/(n+1)) sin(q pi j/(n+1)), i = x index, j = y index, 1..n.
    Returns (b, x, lambda) with A x = b."""
    k = np.arange(1, n + 1, dtype=np.float64)
    sx = np.sin(p * math.pi * k / (n + 1))
    sy = np.sin(q * math.pi * k / (n + 1))
    b = np.outer(sy, sx).reshape(-1)
    lam = _scale(n) * 4.0 * (math.sin(p * math.pi / (2 * (n + 1))) ** 2
                             + math.sin(q * math.pi / (2 * (n + 1))) ** 2)
    return b, b / lam, lam


def krylov_min_residual(A, b, x0, k):
    """min over y of ||b - A (x0 + K y)||, K = [r0, A r0, ..., A^{k-1} r0]."""
    r0 = b - A @ x0
    K = np.empty((len(b), k))
    v = r0 / np.linalg.norm(r0)
    for i in range(k):
        K[:, i] = v
        v = A @ v
        v = v / np.linalg.norm(v)
    AK = A @ K
    Q, R = np.linalg.qr(AK)
    y = np.linalg.solve(R, Q.T @ r0)
    return np.linalg.norm(r0 - AK @ y)
