"""Small, fixed cases of the library's kernels for profiling (ncu) and timing.

    python -m paper_2103_10975_gb300.profile_cases solve --n 256 --blocks 128 --max-iters 300
    python -m paper_2103_10975_gb300.profile_cases nn --n 256 --batch 8
    python -m paper_2103_10975_gb300.profile_cases batch --count 512 --nmax 512
    python -m paper_2103_10975_gb300.profile_cases cube --n 192 --max-iters 500
    python -m paper_2103_10975_gb300.profile_cases cube --n 192 --compact 1 --blocks 304 --stages 2

    python -m paper_2103_10975_gb300.profile_cases dipole --n 64 --T 200
    python -m paper_2103_10975_gb300.profile_cases floor --ctas 128 --m 30

--stages selects the bulk-copy depth for a basis in HBM (0 = direct loads,
-1 = automatic); --compact 1 forces the two-CTAs-per-SM variant; --autotune
runs mlgmres_autotune first.

`solve` runs the same capped solve twice on one moving-Gaussian right-hand
side (the second launch is the one to capture) and prints the device time
per Arnoldi step; `nn` runs the network's forward + backward seven times on
random inputs and prints the mean time; `floor` times the solver's two group
exchanges per Arnoldi step alone (mlgmres_exchange_floor), next to the full
step of the same shape on the 256^2 moving-Gaussian right-hand side.
"""

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def solve_case(n, blocks, max_iters, m, precision, source, stages=-1, autotune=False,
               compact=-1):
    import torch
    from paper_2103_10975_gb300 import Solver
    from synthetic import MovingGaussians2D, RandomWalkSources2D
    if source == "walk":
        b = RandomWalkSources2D(n, 3001).rhs(0)
    else:
        b = MovingGaussians2D(n, 2001, 500).rhs(0)
    bd = torch.as_tensor(b).cuda()
    s = Solver(n, m=m, rtol=1e-10, precision=precision, grid_blocks=blocks, max_iters=max_iters,
               v_stages=stages, compact=compact)
    if autotune:
        t = s.autotune(bd, retune=True)
        print("autotune:", t)
    s.solve(bd)
    _, r = s.solve(bd)
    print("n=%d m=%d %s blocks=%d stages=%d: %d steps, %.3f ms, %.2f us/step"
          % (n, m, precision, blocks, stages, r["iters"], r["tos_ms"],
             1e3 * r["tos_ms"] / r["iters"]))


def nn_case(n, batch, dim=2):
    import torch
    from paper_2103_10975_gb300 import Solver
    s = Solver(n, dim=dim, m=10, batch=batch)
    g = torch.Generator(device="cuda").manual_seed(0)
    u = torch.randn(batch, n ** dim, device="cuda", dtype=torch.float32, generator=g)
    t = torch.randn(batch, n ** dim, device="cuda", dtype=torch.float32, generator=g)
    times = []
    for _ in range(7):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.nn_loss_grad(u, t)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    print("network forward+backward %d^%d batch %d: %.2f ms" % (n, dim, batch,
                                                               1e3 * sum(times[2:]) / 5))


def batch_case(count, nmin, nmax, rtol, m, stages=-1, compact=-1):
    """Independent systems with sides drawn from U{nmin..nmax} (seed 4001 + i),
    FP32-refined GMRES(m), all in one persistent launch."""
    import torch
    from paper_2103_10975_gb300 import Solver
    from synthetic import batched_instances
    inst = batched_instances(count, n_min=nmin, n_max=nmax)
    ns = [n for n, _ in inst]
    bs = [torch.as_tensor(b).cuda() for _, b in inst]
    s = Solver(max(ns), m=m, rtol=rtol, precision="fp32_refine", batch_slots=4096,
               max_iters=10 ** 7, v_stages=stages, compact=compact)
    xs, res = s.solve_batch(ns, bs)
    worst = max(r["relres_true"] for r in res)
    iters = sum(r["iters"] for r in res)
    unknowns = sum(n * n for n in ns)
    print("batch of %d systems (sides %d..%d, %d unknowns): %.1f ms for the launch, "
          "%d Arnoldi steps in total, worst relres %.2e, status %s"
          % (count, min(ns), max(ns), unknowns, res[0]["tos_ms"], iters, worst,
             sorted(set(r["status"] for r in res))))


def cube_case(n, m, max_iters, stages=-1, autotune=False, blocks=0, compact=-1):
    """192^3 variable-coefficient Poisson (log-normal kappa, seed 5001), FP32-refined
    GMRES(m) capped at max_iters steps; prints the device time per step."""
    import torch
    from paper_2103_10975_gb300 import Solver
    from synthetic import MovingGaussians3D, lognormal_kappa
    kap = lognormal_kappa(n, 5001).astype("float32")
    b = torch.as_tensor(MovingGaussians3D(n, 5001, 200).rhs(0)).cuda()
    s = Solver(n, dim=3, kappa=kap, m=m, rtol=1e-10, precision="fp32_refine",
               max_iters=max_iters, v_stages=stages, grid_blocks=blocks, compact=compact)
    if autotune:
        print("autotune:", s.autotune(b, retune=True))
    s.solve(b)
    _, r = s.solve(b)
    print("n=%d^3 m=%d: %d steps, %.1f ms, %.1f us/step, relres %.3e"
          % (n, m, r["iters"], r["tos_ms"], 1e3 * r["tos_ms"] / r["iters"], r["relres_true"]))


def dipole_case(n, T, tau0, train_iters, lr, k):
    """The two-scale dipole workload (a fresh asymmetric dipole with a random
    overall scale every step): the online loop (learned guess with x0 = 0 as
    fallback, training every 10 steps) against GMRES from x0 = 0, reporting
    after the warm-up the true residual after k GMRES(30) iterations from the
    network's guess and from x0 = 0 (the paper's fifth-iteration error), and
    the iterations to rtol 1e-10 of both."""
    import math
    import torch
    from paper_2103_10975_gb300 import Solver
    from synthetic import Dipoles2D
    gen = Dipoles2D(n, 6001)
    learned = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="learned",
                     fallback="zero", warmup_steps=tau0, train_iters=train_iters, lr=lr,
                     batch=8, guess_smooth=32, max_iters=10 ** 6, seed=5)
    plain = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", max_iters=10 ** 6)
    cap_user = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", guess="user", max_iters=k)
    cap_zero = Solver(n, m=30, rtol=1e-10, precision="fp32_refine", max_iters=k)
    ratios, it_l, it_z, used = [], [], [], []
    for t in range(T):
        b = torch.as_tensor(gen.rhs(t)).cuda()
        if t >= tau0:
            x0 = learned.guess(b)
            _, ru = cap_user.solve(b, x=x0)
            _, rz = cap_zero.solve(b)
            ratios.append(rz["relres_true"] / ru["relres_true"])
        _, rl = learned.solve(b)
        _, rp = plain.solve(b)
        if t >= tau0:
            it_l.append(rl["iters"])
            it_z.append(rp["iters"])
            used.append(rl["guess_used"] == 2)
        if (t + 1) % 10 == 0:
            learned.train_step()
    lr_ = [math.log(r) for r in ratios]
    gm = math.exp(sum(lr_) / len(lr_))
    last = ratios[-20:]
    gm_last = math.exp(sum(math.log(r) for r in last) / len(last))
    print("dipoles %d^2, T=%d, tau0=%d: E_%d(x0=0)/E_%d(learned) geometric mean %.2f "
          "(last 20 steps %.2f); iterations learned %.0f vs x0=0 %.0f; learned used %.2f"
          % (n, T, tau0, k, k, gm, gm_last, sum(it_l) / len(it_l), sum(it_z) / len(it_z),
             sum(used) / len(used)))


def floor_case(ctas, m, steps, n):
    import torch
    from paper_2103_10975_gb300 import Solver, exchange_floor
    from synthetic import MovingGaussians2D
    fl = exchange_floor(ctas, m, steps)
    b = torch.as_tensor(MovingGaussians2D(n, 2001, 500).rhs(0)).cuda()
    s = Solver(n, m=m, rtol=1e-10, precision="fp32_refine", grid_blocks=ctas,
               max_iters=10 * m)
    s.solve(b)
    _, r = s.solve(b)
    full = 1e3 * r["tos_ms"] / r["iters"]
    print("exchange floor at %d CTAs, m=%d: %.2f us/step; full step at n=%d: %.2f us/step "
          "(%.2fx the floor)" % (ctas, m, fl, n, full, full / fl))


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="case", required=True)
    a = sub.add_parser("solve")
    a.add_argument("--n", type=int, default=256)
    a.add_argument("--blocks", type=int, default=0)
    a.add_argument("--max-iters", type=int, default=300)
    a.add_argument("--m", type=int, default=30)
    a.add_argument("--precision", default="fp32_refine")
    a.add_argument("--source", default="moving", choices=["moving", "walk"])
    a.add_argument("--stages", type=int, default=-1)
    a.add_argument("--autotune", action="store_true")
    a.add_argument("--compact", type=int, default=-1)
    b = sub.add_parser("nn")
    b.add_argument("--n", type=int, default=256)
    b.add_argument("--batch", type=int, default=8)
    b.add_argument("--dim", type=int, default=2)
    c = sub.add_parser("batch")
    c.add_argument("--count", type=int, default=512)
    c.add_argument("--nmin", type=int, default=64)
    c.add_argument("--nmax", type=int, default=512)
    c.add_argument("--rtol", type=float, default=1e-8)
    c.add_argument("--m", type=int, default=30)
    c.add_argument("--stages", type=int, default=-1)
    c.add_argument("--compact", type=int, default=-1)
    d = sub.add_parser("cube")
    d.add_argument("--n", type=int, default=192)
    d.add_argument("--m", type=int, default=50)
    d.add_argument("--max-iters", type=int, default=500)
    d.add_argument("--stages", type=int, default=-1)
    d.add_argument("--autotune", action="store_true")
    d.add_argument("--blocks", type=int, default=0)
    d.add_argument("--compact", type=int, default=-1)
    e = sub.add_parser("dipole")
    e.add_argument("--n", type=int, default=64)
    e.add_argument("--T", type=int, default=200)
    e.add_argument("--tau0", type=int, default=50)
    e.add_argument("--train-iters", type=int, default=64)
    e.add_argument("--lr", type=float, default=2e-3)
    e.add_argument("--k", type=int, default=5)
    f = sub.add_parser("floor")
    f.add_argument("--ctas", type=int, default=128)
    f.add_argument("--m", type=int, default=30)
    f.add_argument("--steps", type=int, default=3000)
    f.add_argument("--n", type=int, default=256)
    args = ap.parse_args(argv)
    if args.case == "solve":
        solve_case(args.n, args.blocks, args.max_iters, args.m, args.precision, args.source,
                   args.stages, args.autotune, args.compact)
    elif args.case == "nn":
        nn_case(args.n, args.batch, args.dim)
    elif args.case == "batch":
        batch_case(args.count, args.nmin, args.nmax, args.rtol, args.m, args.stages, args.compact)
    elif args.case == "floor":
        floor_case(args.ctas, args.m, args.steps, args.n)
    elif args.case == "dipole":
        dipole_case(args.n, args.T, args.tau0, args.train_iters, args.lr, args.k)
    else:
        cube_case(args.n, args.m, args.max_iters, args.stages, args.autotune, args.blocks,
                  args.compact)


if __name__ == "__main__":
    main()
