"""Small, fixed cases of the library's kernels for profiling (ncu) and timing.

    python -m paper_2103_10975_gb300.profile_cases solve --n 256 --blocks 128 --max-iters 300
    python -m paper_2103_10975_gb300.profile_cases nn --n 256 --batch 8

`solve` runs the same capped solve twice on one moving-Gaussian right-hand
side (the second launch is the one to capture) and prints the device time
per Arnoldi step; `nn` runs the network's forward + backward seven times on
random inputs and prints the mean time.
"""

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def solve_case(n, blocks, max_iters, m, precision, source):
    import torch
    from paper_2103_10975_gb300 import Solver
    from synthetic import MovingGaussians2D, RandomWalkSources2D
    if source == "walk":
        b = RandomWalkSources2D(n, 3001).rhs(0)
    else:
        b = MovingGaussians2D(n, 2001, 500).rhs(0)
    bd = torch.as_tensor(b).cuda()
    s = Solver(n, m=m, rtol=1e-10, precision=precision, grid_blocks=blocks, max_iters=max_iters)
    s.solve(bd)
    _, r = s.solve(bd)
    print("n=%d m=%d %s blocks=%d: %d steps, %.3f ms, %.2f us/step"
          % (n, m, precision, blocks, r["iters"], r["tos_ms"], 1e3 * r["tos_ms"] / r["iters"]))


def nn_case(n, batch):
    import torch
    from paper_2103_10975_gb300 import Solver
    s = Solver(n, m=10, batch=batch)
    g = torch.Generator(device="cuda").manual_seed(0)
    u = torch.randn(batch, n * n, device="cuda", dtype=torch.float32, generator=g)
    t = torch.randn(batch, n * n, device="cuda", dtype=torch.float32, generator=g)
    times = []
    for _ in range(7):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.nn_loss_grad(u, t)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    print("network forward+backward %dx%d batch %d: %.2f ms" % (n, n, batch,
                                                               1e3 * sum(times[2:]) / 5))


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
    b = sub.add_parser("nn")
    b.add_argument("--n", type=int, default=256)
    b.add_argument("--batch", type=int, default=8)
    args = ap.parse_args(argv)
    if args.case == "solve":
        solve_case(args.n, args.blocks, args.max_iters, args.m, args.precision, args.source)
    else:
        nn_case(args.n, args.batch)


if __name__ == "__main__":
    main()
