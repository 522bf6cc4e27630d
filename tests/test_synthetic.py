"""Input generators: splitmix64 against its published test vector, the
vectorised stream against the scalar generator, and workload shapes."""
import math

import numpy as np

from synthetic import (SplitMix64, splitmix64_stream, uniform_stream, normal_stream,
                       MovingGaussians2D, RandomWalkSources2D, MovingGaussians3D,
                       batched_instances, lognormal_kappa, mode_rhs_2d)


def test_splitmix64_published_vector():
    # Test vector of the splitmix64 reference implementation, seed 1234567.
    g = SplitMix64(1234567)
    got = [g.next_u64() for _ in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_stream_matches_scalar():
    g = SplitMix64(99)
    scalar = [g.next_u64() for _ in range(1000)]
    assert [int(v) for v in splitmix64_stream(99, 1000)] == scalar
    g = SplitMix64(7)
    u = [g.uniform() for _ in range(100)]
    assert np.array_equal(np.array(u), uniform_stream(7, 100))


def test_normal_moments():
    z = normal_stream(5, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_moving_gaussians_deterministic():
    a = MovingGaussians2D(32, 1001, 50).rhs(7)
    b = MovingGaussians2D(32, 1001, 50).rhs(7)
    assert a.shape == (1024,) and np.array_equal(a, b)
    assert not np.array_equal(a, MovingGaussians2D(32, 1001, 50).rhs(8))


def test_other_generators_shapes():
    rw = RandomWalkSources2D(64, 3001)
    assert rw.rhs(3).shape == (4096,) and 1 <= rw.p <= 3 and 1 <= rw.q <= 3
    assert MovingGaussians3D(16, 5001, 200).rhs(0).shape == (4096,)
    inst = batched_instances(4)
    assert all(64 <= n <= 512 and b.shape == (n * n,) for n, b in inst)
    k = lognormal_kappa(16, 5001)
    assert k.shape == (4096,) and np.all(k > 0)
    assert abs(np.log(k).std() - 1.0) < 1e-12
    assert mode_rhs_2d(8, 1, 2).shape == (64,)


def test_dipoles_structure_and_determinism():
    from synthetic import Dipoles2D
    g = Dipoles2D(48, 6001)
    b1, b2 = g.rhs(3), Dipoles2D(48, 6001).rhs(3)
    assert np.array_equal(b1, b2)                       # random access by step
    assert not np.allclose(g.rhs(3), g.rhs(4))           # fresh draw every step
    scales = []
    for t in range(40):
        poles, a, S = g.params(t)
        assert 0.5 <= a <= 1.5 and 0.1 <= S <= 10.0
        (px, py, *_), (qx, qy, *_) = poles
        assert 0.15 - 1e-12 <= math.hypot(px - qx, py - qy) <= 0.5 + 1e-12
        b = g.rhs(t).reshape(48, 48)
        assert b.max() > 0 > b.min()                       # one pole of each sign
        scales.append(S)
    assert max(scales) / min(scales) > 10                  # overall scale varies
