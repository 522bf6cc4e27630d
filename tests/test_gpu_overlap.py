"""Training beside the solves (Sec. 2.3: the network is trained in real time
while the simulation goes on).  With overlap_train = 1 a solve issued while a
training phase runs on another stream does not wait for it: it returns while
the phase is still running, with the fallback guess (the guess's inference
copy has no trained parameters yet), and its solution is still the oracle's.
Once the phase has completed, the next solve takes its parameters.  With
overlap_train = 0 the solve waits for the phase."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct  # noqa: E402
from synthetic import MovingGaussians2D  # noqa: E402

pytestmark = pytest.mark.gpu


def make(overlap):
    from paper_2103_10975_gb300 import Solver
    # 400 Adam steps of batch 8 at 128^2: a phase of a few hundred ms, against
    # a solve of some tens of ms
    return Solver(128, m=30, rtol=1e-10, precision="fp32_refine", guess="learned",
                  fallback="prev", warmup_steps=4, train_iters=400, batch=8, lr=2e-3,
                  deterministic_tos=1, overlap_train=overlap, seed=21)


@pytest.mark.parametrize("overlap", [1, 0])
def test_solve_during_a_training_phase(overlap):
    n = 128
    gen = MovingGaussians2D(n, 2001, 60)
    s = make(overlap)
    main = torch.cuda.Stream()
    side = torch.cuda.Stream()
    with torch.cuda.stream(main):
        for t in range(4):
            _, r = s.solve(torch.as_tensor(gen.rhs(t)).cuda())
            assert r["status"] == 0
        torch.cuda.synchronize()
        s.train_step(stream=side)
        phase_end = torch.cuda.Event()
        phase_end.record(side)
        b = gen.rhs(4)
        x, r = s.solve(torch.as_tensor(b).cuda())
        running_at_return = not phase_end.query()
        assert r["status"] == 0 and r["relres_true"] <= 1e-10
        xr = direct.dst_solve_2d(n, b)
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-7 * np.linalg.norm(xr)
        if overlap:
            assert running_at_return, "the solve waited for the training phase"
            assert r["relres_learned"] < 0.0     # no trained parameters yet: no learned guess
        else:
            assert not running_at_return
            assert r["relres_learned"] >= 0.0    # it waited and used the trained network
        side.synchronize()
        x, r = s.solve(torch.as_tensor(gen.rhs(5)).cuda())
        assert r["status"] == 0 and r["relres_learned"] >= 0.0
