"""The learned initial guess as a whole, for parity with the library's
``mlgmres_guess``.

TEST INFRASTRUCTURE ONLY.

Sec. 2.2 forms the guess as x0 = N(b).  The library scales input and output
(a reading: the paper leaves scaling open) and smooths the result:

    s  = rms(b)                        (s = 1 when b = 0)
    x0 = c * s * N(b / s)              c = the training phase's target scale
    x0 <- x0 + omega * D^-1 (b - A x0)   repeated `sweeps` times

D is the diagonal of A.  The sweeps are damped Jacobi, the textbook smoother;
they are not in the paper (the library applies them to remove the white
BF16 rounding noise of the network output, which A amplifies).

Pins (tests/test_oracle_guess.py): the diagonal against the dense matrices of
``direct``; one sweep on an eigenmode error scales it by exactly
1 - omega * lambda / d (2D, constant d); the exact solution is a fixed point;
with sweeps = 0 the guess is c * s * N(b / s) of ``nn.forward``.
"""

import numpy as np

from . import native
from . import nn as onn


def diagonal(dim, n, kappa=None):
    """Diagonal of A: 4/h^2 in 2D; in 3D (1/h^2) * sum over the six faces of
    the face coefficient (harmonic mean of the two cells' kappa, the cell's own
    kappa on a wall face)."""
    h = 2.0 / (n + 1)
    if dim == 2:
        return np.full(n * n, 4.0 / (h * h))
    k = np.ones((n, n, n)) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(n, n, n)
    d = np.zeros((n, n, n))
    for axis in range(3):
        for shift in (-1, 1):
            nb = np.roll(k, shift, axis=axis)
            face = 2.0 * k * nb / (k + nb)
            # the rolled-in slab wraps around: there the face is a wall
            edge = [slice(None)] * 3
            edge[axis] = 0 if shift == 1 else n - 1
            face[tuple(edge)] = k[tuple(edge)]
            d += face
    return d.reshape(-1) / (h * h)


def jacobi(dim, n, b, x, sweeps, omega, kappa=None):
    """`sweeps` damped-Jacobi sweeps x <- x + omega D^-1 (b - A x)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    d = diagonal(dim, n, kappa)
    for _ in range(sweeps):
        x = x + omega * (b - native.apply(dim, n, x, kappa)) / d
    return x


def learned_guess(params, b, n, c, sweeps, omega, dim=2, kappa=None):
    """x0 = c s N(b/s) with s = rms(b), then the sweeps."""
    b = np.asarray(b, dtype=np.float64)
    s = onn.rms(b)
    if not s > 0.0:
        s = 1.0
    y = onn.forward(params, b / s, n, dim=dim)
    return jacobi(dim, n, b, c * s * y, sweeps, omega, kappa)
