"""Source-term generators for the Poisson time series.

Grid convention (shared by every workload): ``n`` interior points per axis on
[-1, 1], spacing h = 2/(n+1), coordinates x_i = -1 + (i+1) h for i = 0..n-1,
row-major with x fastest (2D index iy*n + ix, 3D index (iz*n + iy)*n + ix).

Every generator draws its parameters from one splitmix64 stream, in the order
listed in its docstring, so a seed fixes the whole time series.  The right-hand
side b_t is the source f_t sampled at the grid points.
"""

import math

import numpy as np

from .rng import SplitMix64, normal_stream

TWO_PI = 2.0 * math.pi


def grid_coords(n):
    h = 2.0 / (n + 1)
    return -1.0 + h * np.arange(1, n + 1, dtype=np.float64)


def _gauss1d(coords, centre, sigma):
    d = coords - centre
    return np.exp(-(d * d) / (2.0 * sigma * sigma))


class MovingGaussians2D:
    """Signed Gaussian bumps whose centres run on circles and whose amplitudes
    oscillate (the moving-charge benchmark of Sec. 3).

    Parameters drawn per source k, in this order:
    centre c_k ~ U[-0.5,0.5]^2 (x then y), radius rho_k ~ U[0.1,0.4],
    phase phi_k ~ U[0,2pi), angular rate omega_k ~ U[0.5,2], sign s_k = +-1,
    amplitude rate nu_k ~ U[0.5,2], amplitude phase psi_k ~ U[0,2pi).

    At step t of T: theta = phi + 2 pi omega t/T, centre = c + rho (cos, sin),
    amplitude a = s (1 + 0.5 sin(2 pi nu t/T + psi)).
    """

    def __init__(self, n, seed, T, n_sources=3, sigma=0.1):
        self.n = int(n)
        self.T = int(T)
        self.sigma = float(sigma)
        g = SplitMix64(seed)
        self.params = []
        for _ in range(n_sources):
            cx = g.uniform(-0.5, 0.5)
            cy = g.uniform(-0.5, 0.5)
            rho = g.uniform(0.1, 0.4)
            phi = g.uniform(0.0, TWO_PI)
            omega = g.uniform(0.5, 2.0)
            s = g.sign()
            nu = g.uniform(0.5, 2.0)
            psi = g.uniform(0.0, TWO_PI)
            self.params.append((cx, cy, rho, phi, omega, s, nu, psi))
        self.coords = grid_coords(self.n)

    def sources(self, t):
        out = []
        for (cx, cy, rho, phi, omega, s, nu, psi) in self.params:
            th = phi + TWO_PI * omega * t / self.T
            a = s * (1.0 + 0.5 * math.sin(TWO_PI * nu * t / self.T + psi))
            out.append((cx + rho * math.cos(th), cy + rho * math.sin(th), a))
        return out

    def rhs(self, t):
        x = self.coords
        b = np.zeros((self.n, self.n), dtype=np.float64)
        for (px, py, a) in self.sources(t):
            b += a * np.outer(_gauss1d(x, py, self.sigma), _gauss1d(x, px, self.sigma))
        return b.reshape(-1)


class Dipoles2D:
    """Asymmetric two-scale dipoles, drawn afresh at every step (the
    multi-scale workload of the network-architecture section: each pole is
    made of two scales, the poles are shifted on the domain and relative to
    each other, and every right-hand side has its own random overall scale).

    Step t draws from SplitMix64(seed + 7919 t), in this order:
    centre c ~ U[-0.5,0.5]^2 (x then y); separation r ~ U[0.15,0.5] at angle
    phi ~ U[0,2pi) (poles at c -+ r/2 (cos phi, sin phi)); then per pole (the
    positive one first): narrow width s1 ~ U[0.03,0.06], wide width
    s2 ~ U[0.1,0.2], weights w1, w2 ~ U[0.5,1.5], and the offset of the wide
    part from the narrow one, (dx, dy) ~ U[-0.1,0.1]^2; the negative pole's
    strength a ~ U[0.5,1.5] (so the dipole is not symmetric); finally the
    overall scale S = 10^u, u ~ U[-1,1].

    b_t = S (pole_+ - a pole_-), pole = w1 G(s1) + w2 G(s2, shifted).
    """

    def __init__(self, n, seed):
        self.n = int(n)
        self.seed = int(seed)
        self.coords = grid_coords(self.n)

    def params(self, t):
        g = SplitMix64(self.seed + 7919 * int(t))
        cx = g.uniform(-0.5, 0.5)
        cy = g.uniform(-0.5, 0.5)
        r = g.uniform(0.15, 0.5)
        phi = g.uniform(0.0, TWO_PI)
        poles = []
        for sgn in (1.0, -1.0):
            px = cx - sgn * 0.5 * r * math.cos(phi)
            py = cy - sgn * 0.5 * r * math.sin(phi)
            s1 = g.uniform(0.03, 0.06)
            s2 = g.uniform(0.1, 0.2)
            w1 = g.uniform(0.5, 1.5)
            w2 = g.uniform(0.5, 1.5)
            dx = g.uniform(-0.1, 0.1)
            dy = g.uniform(-0.1, 0.1)
            poles.append((px, py, s1, s2, w1, w2, dx, dy))
        a = g.uniform(0.5, 1.5)
        S = 10.0 ** g.uniform(-1.0, 1.0)
        return poles, a, S

    def rhs(self, t):
        x = self.coords
        poles, a, S = self.params(t)
        b = np.zeros((self.n, self.n), dtype=np.float64)
        for k, (px, py, s1, s2, w1, w2, dx, dy) in enumerate(poles):
            amp = 1.0 if k == 0 else -a
            b += amp * w1 * np.outer(_gauss1d(x, py, s1), _gauss1d(x, px, s1))
            b += amp * w2 * np.outer(_gauss1d(x, py + dy, s2), _gauss1d(x, px + dx, s2))
        return (S * b).reshape(-1)


class RandomWalkSources2D:
    """Sixteen signed Gaussians on a random walk plus one exact Laplacian
    eigenmode (the 2048^2 refinement workload).

    Drawn in order: per source k: centre ~ U[-0.8,0.8]^2, sign, magnitude
    ~ U[0.5,1.5]; then p, q ~ U{1,2,3}.  Each step t >= 1 then draws, per
    source, two normals and moves the centre by 0.02 * (normal, normal),
    clipped to [-0.9, 0.9].  b_t = sum_k gaussians + alpha sin(p pi i/(n+1))
    sin(q pi j/(n+1)) with alpha = 0.5 and i, j = 1..n.
    """

    def __init__(self, n, seed, n_sources=16, sigma=0.1, alpha=0.5, step=0.02):
        self.n = int(n)
        self.sigma = float(sigma)
        self.alpha = float(alpha)
        self.step = float(step)
        self.g = SplitMix64(seed)
        self.centres = []
        self.amps = []
        for _ in range(n_sources):
            cx = self.g.uniform(-0.8, 0.8)
            cy = self.g.uniform(-0.8, 0.8)
            s = self.g.sign()
            a = self.g.uniform(0.5, 1.5)
            self.centres.append([cx, cy])
            self.amps.append(s * a)
        self.p = self.g.randint(1, 3)
        self.q = self.g.randint(1, 3)
        self.path = [[tuple(c) for c in self.centres]]
        self.coords = grid_coords(self.n)

    def _advance_to(self, t):
        while len(self.path) <= t:
            for c in self.centres:
                c[0] = min(0.9, max(-0.9, c[0] + self.step * self.g.normal()))
                c[1] = min(0.9, max(-0.9, c[1] + self.step * self.g.normal()))
            self.path.append([tuple(c) for c in self.centres])

    def rhs(self, t):
        self._advance_to(t)
        x = self.coords
        b = np.zeros((self.n, self.n), dtype=np.float64)
        for (cx, cy), a in zip(self.path[t], self.amps):
            b += a * np.outer(_gauss1d(x, cy, self.sigma), _gauss1d(x, cx, self.sigma))
        b += self.alpha * mode_rhs_2d(self.n, self.p, self.q).reshape(self.n, self.n)
        return b.reshape(-1)


class MovingGaussians3D:
    """Three signed Gaussians moving on tilted circles in [-1,1]^3.

    Drawn per source, in order: centre ~ U[-0.5,0.5]^3 (x, y, z), rho ~
    U[0.1,0.4], phi ~ U[0,2pi), omega ~ U[0.5,2], tilt zeta ~ U[0,2pi),
    sign, nu ~ U[0.5,2], psi ~ U[0,2pi).  Position at step t:
    c + rho (cos th, sin th cos zeta, sin th sin zeta), th = phi + 2 pi omega t/T.
    """

    def __init__(self, n, seed, T, n_sources=3, sigma=0.1):
        self.n = int(n)
        self.T = int(T)
        self.sigma = float(sigma)
        g = SplitMix64(seed)
        self.params = []
        for _ in range(n_sources):
            c = (g.uniform(-0.5, 0.5), g.uniform(-0.5, 0.5), g.uniform(-0.5, 0.5))
            rho = g.uniform(0.1, 0.4)
            phi = g.uniform(0.0, TWO_PI)
            omega = g.uniform(0.5, 2.0)
            zeta = g.uniform(0.0, TWO_PI)
            s = g.sign()
            nu = g.uniform(0.5, 2.0)
            psi = g.uniform(0.0, TWO_PI)
            self.params.append((c, rho, phi, omega, zeta, s, nu, psi))
        self.coords = grid_coords(self.n)

    def rhs(self, t):
        x = self.coords
        n = self.n
        b = np.zeros((n, n, n), dtype=np.float64)
        for (c, rho, phi, omega, zeta, s, nu, psi) in self.params:
            th = phi + TWO_PI * omega * t / self.T
            px = c[0] + rho * math.cos(th)
            py = c[1] + rho * math.sin(th) * math.cos(zeta)
            pz = c[2] + rho * math.sin(th) * math.sin(zeta)
            a = s * (1.0 + 0.5 * math.sin(TWO_PI * nu * t / self.T + psi))
            gx = _gauss1d(x, px, self.sigma)
            gy = _gauss1d(x, py, self.sigma)
            gz = _gauss1d(x, pz, self.sigma)
            b += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        return b.reshape(-1)


def batched_sides(count, base_seed=4001, n_min=64, n_max=512):
    """The sides of batched_instances without building the right-hand sides."""
    return [SplitMix64(base_seed + i).randint(n_min, n_max) for i in range(count)]


def batched_instances(count, base_seed=4001, n_min=64, n_max=512):
    """Independent instances for the batched workload: instance i uses seed
    base_seed + i; its first draw is the side n_i ~ U{n_min..n_max}, the rest
    seeds a MovingGaussians2D at t = 0 (T = 1)."""
    out = []
    for i in range(count):
        g = SplitMix64(base_seed + i)
        n = g.randint(n_min, n_max)
        sub_seed = g.next_u64()
        src = MovingGaussians2D(n, sub_seed, T=1)
        out.append((n, src.rhs(0)))
    return out


def mode_rhs_2d(n, p, q):
    """sin(p pi i/(n+1)) sin(q pi j/(n+1)), i (x) and j (y) = 1..n."""
    k = np.arange(1, n + 1, dtype=np.float64)
    sx = np.sin(p * math.pi * k / (n + 1))
    sy = np.sin(q * math.pi * k / (n + 1))
    return np.outer(sy, sx).reshape(-1)


def lognormal_kappa(n, seed, smooth_sigma=4.0):
    """Cell coefficient kappa = exp(g) on an n^3 grid, where g is white N(0,1)
    noise (normal_stream order = linear index), Gaussian-filtered with
    sigma = smooth_sigma cells (zero padding) and rescaled to unit std."""
    from scipy.ndimage import gaussian_filter

    w = normal_stream(seed, n * n * n).reshape(n, n, n)
    g = gaussian_filter(w, sigma=smooth_sigma, mode="constant", cval=0.0)
    g = g / g.std()
    return np.exp(g).reshape(-1)
