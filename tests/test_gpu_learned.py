"""What the trained network gains (Sec. 2, Algorithm 1, Sec. 2.3): the online
loop -- network guess, GMRES(k), gate, replay, training every 10 steps -- run
on a moving-Gaussian series against plain GMRES from x0 = 0 on the same
right-hand sides.  The training trajectory itself is stochastic (minibatch
sampling), so the claim checked is statistical: fewer iterations per step
after warm-up, with a bootstrap confidence interval that excludes zero."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synthetic import MovingGaussians2D  # noqa: E402

pytestmark = pytest.mark.gpu


def bootstrap_ci(gain, seed=0):
    rng = np.random.default_rng(seed)
    boots = [rng.choice(gain, size=len(gain)).mean() for _ in range(2000)]
    return np.percentile(boots, [2.5, 97.5])


def test_learned_guess_reduces_iterations():
    """Against x0 = 0 and against a control that gives x0 = 0 the same
    damped-Jacobi sweeps the learned guess gets (no network), so that the
    network's own share of the gain is seen."""
    from paper_2103_10975_gb300 import Solver
    n, T, tau0 = 128, 150, 50
    gen = MovingGaussians2D(n, 2001, 500)
    learned = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="learned",
                     fallback="zero", warmup_steps=tau0, train_iters=64, batch=8, lr=2e-3,
                     deterministic_tos=1, max_iters=300000, seed=3, overlap_train=0)
    plain = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="zero", max_iters=300000)
    ctrl = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="user", max_iters=300000)
    sweeps = learned.opt.guess_smooth
    it_l, it_z, it_s, used = [], [], [], []
    for t in range(T):
        b = torch.as_tensor(gen.rhs(t)).cuda()
        _, rl = learned.solve(b)
        _, rz = plain.solve(b)
        _, rs = ctrl.solve(b, ctrl.smooth(b, torch.zeros_like(b), sweeps))
        assert rl["status"] == 0 and rl["relres_true"] <= 1e-10
        if (t + 1) % 10 == 0:
            learned.train_step()
        if t >= tau0 + 10:
            it_l.append(rl["iters"])   # includes the discarded first cycle
            it_z.append(rz["iters"])
            it_s.append(rs["iters"])
            used.append(rl["guess_used"] == 2)
    it_l, it_z, it_s = (np.array(v, dtype=float) for v in (it_l, it_z, it_s))
    lo, hi = bootstrap_ci(it_z - it_l)
    slo, shi = bootstrap_ci(it_s - it_l, 1)
    print("mean iterations: learned %.1f, zero %.1f, smoothing only %.1f; gain over zero %.1f "
          "(95%% CI %.1f..%.1f), over smoothing only %.1f (95%% CI %.1f..%.1f); learned guess "
          "used in %.0f%% of steps" % (it_l.mean(), it_z.mean(), it_s.mean(),
                                       (it_z - it_l).mean(), lo, hi, (it_s - it_l).mean(), slo,
                                       shi, 100 * np.mean(used)))
    assert np.mean(used) > 0.5
    assert lo > 0.0


def test_learned_guess_3d_variable_kappa():
    """The online loop on the 3D variable-coefficient operator with the 3D
    network (3x3x3 kernels): after the warm-up the network's guess is formed,
    smoothed with kappa-weighted Jacobi sweeps and scored against x0 = 0 by
    one GMRES cycle; every step still reaches the tolerance and the oracle's
    solution."""
    from paper_2103_10975_gb300 import Solver
    from oracle import native
    from synthetic import MovingGaussians3D, lognormal_kappa
    n, T, tau0 = 16, 10, 4
    kap = lognormal_kappa(n, 5001, smooth_sigma=2.0).astype(np.float32)
    gen = MovingGaussians3D(n, 5001, 40)
    s = Solver(n, dim=3, kappa=kap, m=30, rtol=1e-10, precision="fp32_refine", guess="learned",
               fallback="zero", warmup_steps=tau0, train_iters=8, batch=2, lr=2e-3,
               deterministic_tos=1, max_iters=100000, seed=4)
    formed = 0
    for t in range(T):
        b = gen.rhs(t)
        x, r = s.solve(torch.as_tensor(b).cuda())
        assert r["status"] == 0 and r["relres_true"] <= 1e-10, (t, r)
        xr, _, _ = native.gmres(3, n, b, m=50, rtol=1e-13, kappa=kap.astype(np.float64))
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-7 * np.linalg.norm(xr)
        if t >= tau0:
            assert np.isfinite(r["relres_learned"]) and r["relres_learned"] >= 0.0
            assert r["guess_used"] in (0, 2)
            formed += 1
        if (t + 1) % 2 == 0:
            s.train_step()
    assert formed == T - tau0


def test_dipole_workload_fifth_iteration_error():
    """The two-scale dipole workload (a fresh asymmetric dipole with a random
    overall scale every step, so x_{t-1} carries no information): after the
    warm-up, five GMRES(30) iterations from the network's guess (mlgmres_guess)
    leave a smaller true residual than five from x0 = 0 (geometric mean over
    the last 40 steps; about 4x at 64^2 over 200 steps)."""
    import math
    from paper_2103_10975_gb300 import Solver
    from synthetic import Dipoles2D
    n, T, tau0 = 64, 120, 40
    gen = Dipoles2D(n, 6001)
    learned = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="learned",
                     fallback="zero", warmup_steps=tau0, train_iters=64, lr=2e-3, batch=8,
                     guess_smooth=32, deterministic_tos=1, max_iters=10 ** 6, seed=5)
    cap_user = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="user", max_iters=5)
    cap_zero = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", max_iters=5)
    logs, logs_s = [], []
    for t in range(T):
        b = torch.as_tensor(gen.rhs(t)).cuda()
        if t >= T - 40:
            _, ru = cap_user.solve(b, x=learned.guess(b))
            _, rz = cap_zero.solve(b)
            # control: the same 32 sweeps from x0 = 0, no network
            _, rs = cap_user.solve(b, x=cap_user.smooth(b, torch.zeros_like(b), 32))
            assert ru["iters"] == 5 and rz["iters"] == 5 and rs["iters"] == 5
            logs.append(math.log(rz["relres_true"] / ru["relres_true"]))
            logs_s.append(math.log(rs["relres_true"] / ru["relres_true"]))
        _, r = learned.solve(b)
        assert r["status"] == 0 and r["relres_true"] <= 1e-10
        if (t + 1) % 10 == 0:
            learned.train_step()
    gm = math.exp(sum(logs) / len(logs))
    gs = math.exp(sum(logs_s) / len(logs_s))
    print("fifth-iteration residual, x0 = 0 / learned: %.2f; smoothing only / learned: %.2f"
          % (gm, gs))
    assert gm > 1.5, gm


def test_adaptive_growth_appends_blocks_on_stagnation():
    """grow_tol = 1 counts every training phase after the first as stagnant,
    so one residual block is appended per phase until grow_blocks; the solves
    stay correct while the network deepens."""
    from paper_2103_10975_gb300 import Solver
    n = 32
    gen = MovingGaussians2D(n, 1001, 50)
    s = Solver(n, m=20, rtol=1e-8, guess="learned", fallback="zero", warmup_steps=5,
               train_iters=2, batch=4, grow_blocks=2, grow_tol=1.0, deterministic_tos=1, seed=9)
    depth = []
    for t in range(30):
        _, r = s.solve(torch.as_tensor(gen.rhs(t)).cuda())
        assert r["status"] == 0 and r["relres_true"] <= 1e-8
        if (t + 1) % 5 == 0:
            s.train_step()
            depth.append(s.nn_blocks())
    assert depth[:4] == [0, 1, 2, 2], depth
