"""GPU parity of the persistent GMRES(m) path against the FP64 oracle, the
DST-I exact solution and the closed forms (GMRES(k), Sec. 1.2; the Poisson
benchmark of Sec. 3).  Every call goes through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import native, direct  # noqa: E402
from synthetic import MovingGaussians2D, MovingGaussians3D, lognormal_kappa  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2103_10975_gb300 import MLGMRESError  # noqa: E402
    from paper_2103_10975_gb300 import Solver as _Solver  # noqa: E402


def Solver(*a, **k):
    """A handle with an iteration cap that bounds any test's run time."""
    k.setdefault("max_iters", 300000)
    return _Solver(*a, **k)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def iters_close(a, b):
    return abs(a - b) <= max(2, 0.01 * b)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 255])
def test_apply_2d(n):
    s = Solver(n, m=5)
    u = np.random.default_rng(n).standard_normal(n * n)
    got = s.apply(dev(u)).cpu().numpy()
    ref = native.apply_2d(n, u)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n", [1, 3, 8, 19])
@pytest.mark.parametrize("var", [False, True])
def test_apply_3d(n, var):
    rng = np.random.default_rng(n)
    kap = np.exp(rng.standard_normal(n ** 3)).astype(np.float32) if var else None
    s = Solver(n, dim=3, kappa=kap, m=5)
    u = rng.standard_normal(n ** 3)
    got = s.apply(dev(u)).cpu().numpy()
    ref = native.apply_3d(n, u, None if kap is None else kap.astype(np.float64))
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_config1_all_steps_fp64():
    """32^2, GMRES(20), rtol 1e-8, x0 = 0, 50 moving-Gaussian steps."""
    n, T = 32, 50
    gen = MovingGaussians2D(n, 1001, T)
    s = Solver(n, m=20, rtol=1e-8)
    for t in range(T):
        b = gen.rhs(t)
        x, r = s.solve(dev(b))
        xr, st, _ = native.gmres(2, n, b, m=20, rtol=1e-8)
        assert r["status"] == 0 and r["relres_true"] <= 1e-8
        assert iters_close(r["iters"], st["iters"]), (t, r["iters"], st["iters"])
        xg = x.cpu().numpy()
        assert rel(xg, xr) <= 1e-6
        assert rel(xg, direct.dst_solve_2d(n, b)) <= 1e-5
        # E_k: true residual after the first cycle
        assert abs(r["relres_first_cycle"] - st["relres_first_cycle"]) <= 1e-6 * st["relres_first_cycle"] + 1e-14


@pytest.mark.parametrize("n,m,prec", [(64, 30, "fp64"), (128, 30, "fp64"),
                                      (64, 30, "fp32_refine"), (128, 30, "fp32_refine"),
                                      (37, 20, "fp64"), (37, 20, "fp32_refine")])
def test_tol_1e10_vs_exact(n, m, prec):
    b = MovingGaussians2D(n, 2001, 500).rhs(17)
    s = Solver(n, m=m, rtol=1e-10, precision=prec)
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    xe = direct.dst_solve_2d(n, b)
    assert rel(x.cpu().numpy(), xe) <= 1e-7
    if prec == "fp64" and n <= 64:
        _, st, _ = native.gmres(2, n, b, m=m, rtol=1e-10)
        assert iters_close(r["iters"], st["iters"]), (r["iters"], st["iters"])


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_config2_size_one_step(prec):
    """256^2, GMRES(30), rtol 1e-10: certificate and error vs the exact solve."""
    n = 256
    b = MovingGaussians2D(n, 2001, 500).rhs(0)
    s = Solver(n, m=30, rtol=1e-10, precision=prec)
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    assert rel(x.cpu().numpy(), direct.dst_solve_2d(n, b)) <= 1e-7
    # check the certificate independently through the oracle's operator
    xr = x.cpu().numpy()
    assert np.linalg.norm(b - native.apply_2d(n, xr)) <= 1.0001e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("blocks", [1, 2, 7, 64])
def test_partitioning_does_not_change_result(blocks):
    n = 45
    b = MovingGaussians2D(n, 7, 10).rhs(3)
    s = Solver(n, m=20, rtol=1e-10, grid_blocks=blocks)
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    _, st, _ = native.gmres(2, n, b, m=20, rtol=1e-10)
    assert iters_close(r["iters"], st["iters"])
    assert rel(x.cpu().numpy(), direct.dst_solve_2d(n, b)) <= 1e-7


@pytest.mark.parametrize("n,blocks", [(250, 7), (256, 4), (129, 3)])
def test_fp32_basis_in_hbm(n, blocks):
    """Few CTAs, so each CTA's slice of V exceeds shared memory and the FP32
    passes stream V from HBM through the bulk-copy stages (ragged last tile
    for n = 250 and 129): same certificate, same solution, and the iteration
    count of the FP64 solver."""
    b = MovingGaussians2D(n, 2001, 500).rhs(5)
    s32 = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", grid_blocks=blocks)
    x, r = s32.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    assert rel(x.cpu().numpy(), direct.dst_solve_2d(n, b)) <= 1e-7
    s64 = Solver(n, m=30, rtol=1e-10, precision="fp64", grid_blocks=blocks)
    _, r64 = s64.solve(dev(b))
    assert abs(r["iters"] - r64["iters"]) <= max(5, r64["iters"] // 50), (r["iters"], r64["iters"])


@pytest.mark.parametrize("stages", [0, 2, 3, 16])
def test_fp32_basis_stage_counts(stages):
    """Every bulk-copy depth (and direct loads) gives the same solve."""
    n = 250
    b = MovingGaussians2D(n, 2001, 500).rhs(9)
    s = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", grid_blocks=5, v_stages=stages)
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    assert rel(x.cpu().numpy(), direct.dst_solve_2d(n, b)) <= 1e-7
    ref = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", grid_blocks=5, v_stages=0)
    _, r0 = ref.solve(dev(b))
    assert abs(r["iters"] - r0["iters"]) <= max(3, r0["iters"] // 100)


@pytest.mark.parametrize("n,blocks", [(256, 256), (250, 300), (512, 200)])
def test_compact_variant(n, blocks):
    """The two-CTAs-per-SM variants (128 registers, m <= 47), with V slices in
    shared memory (256^2, 250^2: slices fit next to the smaller state) and
    streamed by bulk copies (512^2): same certificate, solution and iteration
    count as the standard variant."""
    b = MovingGaussians2D(n, 2001, 500).rhs(11)
    s = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", grid_blocks=blocks, compact=1)
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    assert rel(x.cpu().numpy(), direct.dst_solve_2d(n, b)) <= 1e-7
    ref = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", compact=0)
    _, r0 = ref.solve(dev(b))
    assert abs(r["iters"] - r0["iters"]) <= max(3, r0["iters"] // 100), (r["iters"], r0["iters"])


@pytest.mark.parametrize("m,stages", [(40, -1), (50, 4), (50, 2), (55, -1)])
def test_compact_variant_3d(m, stages):
    """The 3D compact variant (two CTAs per SM; GMRES(50) with two stages per
    warp is the shape the autotuner picks at 192^3; m = 55 is its bucket limit)
    on variable kappa, through the face-coefficient stencil and its zero-padded
    windows, against the oracle's solution."""
    n = 24
    kap = lognormal_kappa(n, 5001, smooth_sigma=2.0).astype(np.float32)
    b = MovingGaussians3D(n, 5001, 200).rhs(7)
    xr, _, _ = native.gmres(3, n, b, m=50, rtol=1e-13, kappa=kap.astype(np.float64))
    s = Solver(n, dim=3, kappa=kap, m=m, rtol=1e-10, precision="fp32_refine", grid_blocks=60,
               compact=1, v_stages=stages)
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and r["relres_true"] <= 1e-10
    assert rel(x.cpu().numpy(), xr) <= 1e-7


def test_kappa_changed_between_solves():
    """kappa is read at the start of every solve: after the caller rewrites the
    device array in place, the next FP32-refined solve (face coefficients formed
    again) matches the oracle for the new coefficients."""
    n = 20
    k1 = lognormal_kappa(n, 5001, smooth_sigma=2.0).astype(np.float32)
    k2 = lognormal_kappa(n, 5002, smooth_sigma=2.0).astype(np.float32)
    b = MovingGaussians3D(n, 5001, 200).rhs(3)
    s = Solver(n, dim=3, kappa=k1, m=40, rtol=1e-10, precision="fp32_refine")
    x1, r1 = s.solve(dev(b))
    xr1, _, _ = native.gmres(3, n, b, m=50, rtol=1e-13, kappa=k1.astype(np.float64))
    assert r1["status"] == 0 and rel(x1.cpu().numpy(), xr1) <= 1e-7
    s.kappa.copy_(torch.as_tensor(k2).cuda())
    x2, r2 = s.solve(dev(b))
    xr2, _, _ = native.gmres(3, n, b, m=50, rtol=1e-13, kappa=k2.astype(np.float64))
    assert r2["status"] == 0 and rel(x2.cpu().numpy(), xr2) <= 1e-7


def test_autotune_picks_the_fastest_candidate_and_caches():
    n = 512
    b = MovingGaussians2D(n, 2001, 500).rhs(2)
    s = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", max_iters=4000)
    t = s.autotune(dev(b), steps=60, retune=True)
    assert t["from_cache"] == 0 and len(t["candidates"]) >= 2
    assert t["us_per_step"] == min(c[2] for c in t["candidates"])
    assert (t["grid_blocks"], t["v_stages"]) in [(c[0], c[1]) for c in t["candidates"]]
    # the tuned handle still solves correctly (capped: compare with the oracle's
    # operator on the returned iterate)
    x, r = s.solve(dev(b))
    xr = x.cpu().numpy()
    assert abs(np.linalg.norm(b - native.apply_2d(n, xr)) / np.linalg.norm(b)
               - r["relres_true"]) <= 1e-6 * r["relres_true"] + 1e-15
    s2 = Solver(n, m=30, rtol=1e-10, precision="fp32_refine")
    t2 = s2.autotune(dev(b))
    assert t2["from_cache"] == 1 and t2["grid_blocks"] == t["grid_blocks"]
    assert t2["v_stages"] == t["v_stages"]


def test_eigenmode_one_iteration():
    n = 64
    b, xe, _ = direct.eigen_pair_2d(n, 2, 3)
    for prec in ("fp64", "fp32_refine"):
        s = Solver(n, m=30, rtol=1e-12 if prec == "fp64" else 1e-10, precision=prec)
        x, r = s.solve(dev(b))
        assert r["status"] == 0
        if prec == "fp64":
            assert r["iters"] == 1
        assert rel(x.cpu().numpy(), xe) <= 1e-9


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_grids(n):
    b = np.random.default_rng(n).standard_normal(n * n)
    s = Solver(n, m=10, rtol=1e-12)
    x, r = s.solve(dev(b))
    assert r["status"] == 0
    assert rel(x.cpu().numpy(), np.linalg.solve(direct.dense_laplacian_2d(n), b)) <= 1e-10


def test_zero_rhs_and_cap():
    n = 32
    s = Solver(n, m=10, rtol=1e-10, guess="user")
    x0 = dev(np.ones(n * n))
    x, r = s.solve(dev(np.zeros(n * n)), x0)
    assert r["status"] == 0 and r["iters"] == 0 and float(x.abs().max()) == 0.0
    s = Solver(n, m=10, rtol=1e-14, max_iters=25)
    b = MovingGaussians2D(n, 3, 5).rhs(0)
    x, r = s.solve(dev(b))
    assert r["status"] == 1 and r["iters"] == 25
    _, st, _ = native.gmres(2, n, b, m=10, rtol=1e-14, max_iters=25)
    assert abs(r["relres_true"] - st["relres_true"]) <= 1e-6 * st["relres_true"]


def test_guess_modes_prev_and_user():
    n = 64
    gen = MovingGaussians2D(n, 2001, 500)
    b0, b1 = gen.rhs(0), gen.rhs(1)
    s = Solver(n, m=30, rtol=1e-10, guess="prev")
    _, r0 = s.solve(dev(b0))
    x1, r1 = s.solve(dev(b1))
    assert r0["guess_used"] == 0 and r1["guess_used"] == 1
    _, st, _ = native.gmres(2, n, b1, m=30, rtol=1e-10, x0=direct.dst_solve_2d(n, b0))
    assert r1["relres_true"] <= 1e-10
    assert abs(r1["relres_guess"] - st["relres_guess"]) <= 1e-6 * st["relres_guess"]
    su = Solver(n, m=30, rtol=1e-10, guess="user")
    xe = direct.dst_solve_2d(n, b1)
    x, r = su.solve(dev(b1), dev(xe * (1 + 1e-3)))
    assert r["guess_used"] == 3 and abs(r["relres_guess"] - 1e-3) < 1e-6
    assert r["relres_true"] <= 1e-10


def test_nonfinite_user_guess_reports_status():
    n = 16
    s = Solver(n, m=10, rtol=1e-10, guess="user")
    x0 = np.zeros(n * n)
    x0[5] = np.nan
    x, r = s.solve(dev(np.ones(n * n)), dev(x0), check=False)
    assert r["status"] == -5


def test_barrier_timeout_is_reported_and_context_survives():
    """The bounded group-barrier wait runs out (the barrier waits for one CTA
    that is never launched) and the solve returns ERR_TIMEOUT; the context
    stays usable afterwards."""
    n = 64
    s = Solver(n, m=10, rtol=1e-10, grid_blocks=4, fault_inject=1, barrier_timeout_s=0.2)
    b = dev(MovingGaussians2D(n, 1, 5).rhs(0))
    with pytest.raises(MLGMRESError) as e:
        s.solve(b)
    assert e.value.status == -4
    ok = Solver(n, m=30, rtol=1e-10)
    _, r = ok.solve(b)
    assert r["status"] == 0 and r["relres_true"] <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_arnoldi_invariants(prec):
    """A V_k = V_{k+1} H_k and V^T V = I for the CGS2 basis."""
    n, k = 64, 30
    s = Solver(n, m=k, precision=prec)
    v0 = np.random.default_rng(5).standard_normal(n * n)
    V, H, done = s.arnoldi(dev(v0), k)
    assert done == k
    V = V.cpu().numpy()
    AV = np.stack([native.apply_2d(n, V[j]) for j in range(k)])
    eps = 1e-12 if prec == "fp64" else 5e-6
    normA = 8.0 * ((n + 1) / 2.0) ** 2
    assert np.linalg.norm(AV.T - V.T @ H, 2) <= eps * normA * 10
    G = V @ V.T
    assert np.abs(G - np.eye(k + 1)).max() <= (1e-12 if prec == "fp64" else 1e-5)
    # H matches the oracle's MGS Hessenberg in exact arithmetic
    Vr, Hr, _ = native.arnoldi(2, n, v0, k)
    assert np.allclose(H, Hr, rtol=0, atol=(1e-9 if prec == "fp64" else 2e-3) * normA)


@pytest.mark.parametrize("n", [12, 20])
def test_3d_variable_kappa_vs_oracle(n):
    kap = lognormal_kappa(n, 5001, smooth_sigma=2.0).astype(np.float32)
    b = MovingGaussians3D(n, 5001, 200).rhs(3)
    kd = kap.astype(np.float64)
    xr, st, _ = native.gmres(3, n, b, m=50, rtol=1e-13, kappa=kd)
    for prec in ("fp64", "fp32_refine"):
        s = Solver(n, dim=3, kappa=kap, m=50, rtol=1e-10, precision=prec)
        x, r = s.solve(dev(b))
        assert r["status"] == 0 and r["relres_true"] <= 1e-10
        assert rel(x.cpu().numpy(), xr) <= 1e-7
        if prec == "fp64":
            _, st10, _ = native.gmres(3, n, b, m=50, rtol=1e-10, kappa=kd)
            assert iters_close(r["iters"], st10["iters"])


def test_3d_constant_kappa_vs_dst():
    n = 24
    b = MovingGaussians3D(n, 11, 20).rhs(0)
    s = Solver(n, dim=3, m=50, rtol=1e-10, precision="fp32_refine")
    x, r = s.solve(dev(b))
    assert r["status"] == 0 and rel(x.cpu().numpy(), direct.dst_solve_3d(n, b)) <= 1e-7


def test_batched_uneven_grids():
    """Many independent systems of uneven size in one persistent launch
    (one CTA group per list of systems), each against its exact solution and
    against a single solve of the same system."""
    from synthetic import batched_instances
    rng = np.random.default_rng(11)
    sides = [int(v) for v in rng.integers(5, 72, size=13)] + [1, 2, 72]
    bs, xs_exact = [], []
    for i, n in enumerate(sides):
        b = MovingGaussians2D(n, 4001 + i, 1).rhs(0) if n > 2 else rng.standard_normal(n * n)
        bs.append(dev(b))
        xs_exact.append(direct.dst_solve_2d(n, b))
    s = Solver(72, m=30, rtol=1e-10, precision="fp32_refine", batch_slots=5)
    xs, res = s.solve_batch(sides, bs)
    for i, n in enumerate(sides):
        assert res[i]["status"] == 0 and res[i]["relres_true"] <= 1e-10, (i, n, res[i])
        assert rel(xs[i].cpu().numpy(), xs_exact[i]) <= 1e-7, (i, n)
        single = Solver(n, m=30, rtol=1e-10, precision="fp32_refine")
        _, r1 = single.solve(bs[i])
        # a batched group may sum its partials over another number of CTAs
        # than the single solve (other FP32 rounding).  On the smallest grids
        # the last cycle starts near the FP32 floor of the inner Arnoldi
        # process, where the Givens estimate crosses the tolerance slowly, so
        # the stopping step inside that cycle moves (measured at n = 13: 73
        # against 63 steps, three cycles each); both solves must end in the
        # same cycle, and larger grids within max(2, 1%) steps
        assert res[i]["cycles"] == r1["cycles"], (n, res[i]["cycles"], r1["cycles"])
        assert abs(res[i]["iters"] - r1["iters"]) < 30, (n, res[i]["iters"], r1["iters"])
        if n >= 24:
            assert iters_close(res[i]["iters"], r1["iters"]), (n, res[i]["iters"], r1["iters"])
    # the c4 generator: sides drawn from U{64..512}; a few of the smaller ones
    inst = [(n, b) for n, b in batched_instances(40) if n <= 96][:4]
    if inst:
        s2 = Solver(96, m=30, rtol=1e-8, precision="fp32_refine", batch_slots=4)
        xs2, res2 = s2.solve_batch([n for n, _ in inst], [dev(b) for _, b in inst])
        for (n, b), x, r in zip(inst, xs2, res2):
            assert r["status"] == 0 and r["relres_true"] <= 1e-8
            assert rel(x.cpu().numpy(), direct.dst_solve_2d(n, b)) <= 1e-5


def test_batched_3d_with_own_kappa():
    sides = [6, 9, 12]
    kaps, bs, refs = [], [], []
    for i, n in enumerate(sides):
        k = lognormal_kappa(n, 77 + i, smooth_sigma=1.5).astype(np.float32)
        b = MovingGaussians3D(n, 5 + i, 10).rhs(0)
        kaps.append(torch.as_tensor(k).cuda())
        bs.append(dev(b))
        xr, _, _ = native.gmres(3, n, b, m=50, rtol=1e-13, kappa=k.astype(np.float64))
        refs.append(xr)
    s = Solver(12, dim=3, m=50, rtol=1e-10, precision="fp64", batch_slots=2)
    xs, res = s.solve_batch(sides, bs, kappas=kaps)
    for x, r, xr in zip(xs, res, refs):
        assert r["status"] == 0 and r["relres_true"] <= 1e-10
        assert rel(x.cpu().numpy(), xr) <= 1e-7


def test_batch_rejects_bad_arguments():
    s = Solver(16, m=10, batch_slots=2)
    b = dev(np.ones(17 * 17))
    with pytest.raises(MLGMRESError):
        s.solve_batch([17], [b])
    s0 = Solver(16, m=10)
    with pytest.raises(MLGMRESError):
        s0.solve_batch([16], [dev(np.ones(256))])


def test_exchange_floor_probe():
    """mlgmres_exchange_floor runs the solver's two group exchanges per step
    alone: a positive time per step, below the full Arnoldi step at the same
    CTA count (which adds the passes and the scalar work), and argument errors
    rejected before any launch."""
    import ctypes
    from paper_2103_10975_gb300 import binding, exchange_floor
    fl = exchange_floor(64, 30, 500)
    assert fl > 0.0
    b = torch.as_tensor(MovingGaussians2D(128, 2001, 500).rhs(0)).cuda()
    s = Solver(128, m=30, rtol=1e-10, precision="fp32_refine", grid_blocks=64, max_iters=300)
    s.solve(b)
    _, r = s.solve(b)
    full = 1e3 * r["tos_ms"] / r["iters"]
    assert fl < full, (fl, full)
    lib = binding.load_library()
    us = ctypes.c_float(0)
    for args in ((0, 30, 10), (64, 0, 10), (64, 65, 10), (64, 30, 0), (2000, 30, 10)):
        assert lib.mlgmres_exchange_floor(*args, ctypes.byref(us)) == binding.MLGMRES_ERR_ARG, args
    assert lib.mlgmres_exchange_floor(64, 30, 10, None) == binding.MLGMRES_ERR_ARG
