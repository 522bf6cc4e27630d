"""GPU parity of Algorithm 1's gate (Sec. 2.2) and of its retraining trigger:
the library's admit decisions and training phases on an online loop are
replayed through the oracle's gate (oracle/gate.py) from the (E_k, TOS, x)
triples the library reported, with TOS the iteration count
(deterministic_tos = 1), and must agree on every step.

The spread check compares the new solution with the C_t members stored in the
FP32 replay ring (x/s), the oracle with the FP64 solutions; a |cos| within
1e-5 of theta could fall either way, so such a step (none is expected) follows
the library's decision and is counted."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.gate import GateRef, abs_cos  # noqa: E402
from synthetic import MovingGaussians2D  # noqa: E402

pytestmark = pytest.mark.gpu

TIE = 1e-5


class Replay:
    """GateRef driven step by step, following the library on near-ties."""

    def __init__(self, p, theta, warmup):
        self.g = GateRef(p=p, theta=theta, warmup=warmup)
        self.ties = 0

    def step(self, E, TOS, x, admitted_gpu):
        g = self.g
        near = any(abs(abs_cos(x, c) - g.theta) < TIE for c in g.C)
        decision = g.step(E, TOS, x)
        if near and decision != bool(admitted_gpu):
            self.ties += 1
            if admitted_gpu:
                g.C.append(np.asarray(x, dtype=np.float64))
            else:
                g.C.pop()
            decision = bool(admitted_gpu)
        return decision


def run_loop(T, tau0, p, theta, every=None, f_r=0, n=32, seed=5):
    from paper_2103_10975_gb300 import Solver
    gen = MovingGaussians2D(n, 1001, 100)
    s = Solver(n, m=20, rtol=1e-8, guess="learned", fallback="prev", warmup_steps=tau0,
               window_p=p, ortho_theta=theta, retrain_after=f_r, deterministic_tos=1,
               train_iters=4, batch=4, seed=seed)
    rows = []
    for t in range(T):
        x, r = s.solve(torch.as_tensor(gen.rhs(t)).cuda())
        assert r["status"] == 0 and r["relres_true"] <= 1e-8
        rows.append((r, x.cpu().numpy()))
        if every and (t + 1) % every == 0:
            s.train_step()
            rows[-1][0]["train_after"] = 1
    return s, rows


def test_gate_decisions_match_the_oracle_fixed_cadence():
    """tau0 = 10, p = 10, theta = 0.9, training every 10 steps, 90 steps."""
    T, tau0, p, theta = 90, 10, 10, 0.9
    s, rows = run_loop(T, tau0, p, theta, every=10)
    rep = Replay(p, theta, tau0)
    admitted_after = 0
    kinds = {"good": 0, "admitted": 0, "rejected": 0}
    for t, (r, x) in enumerate(rows):
        before = rep.g.N
        want = rep.step(r["relres_first_cycle"], r["iters"], x, r["admitted"])
        assert int(want) == r["admitted"], (t, r["relres_first_cycle"], r["iters"], r["admitted"])
        if t >= tau0:
            admitted_after += r["admitted"]
            if rep.g.N == before:
                kinds["good"] += 1
            else:
                kinds["admitted" if r["admitted"] else "rejected"] += 1
        if r.get("train_after"):
            rep.g.trained()
    assert rep.ties <= 1, rep.ties
    # every branch of the gate was taken
    assert min(kinds.values()) > 0, kinds
    ring = min(64, tau0 + admitted_after)
    assert s.replay_size() == ring
    print("post-warm-up steps retained: %d of %d (%s), ties %d"
          % (admitted_after, T - tau0, kinds, rep.ties))


def test_retraining_trigger_matches_algorithm_1():
    """retrain_after = f_r: the library starts a phase at tau0 and then exactly
    when Algorithm 1's counter N (under-performing steps since the previous
    phase, admitted or not) reaches f_r."""
    T, tau0, p, theta, f_r = 80, 10, 10, 0.9, 3
    s, rows = run_loop(T, tau0, p, theta, f_r=f_r)
    rep = Replay(p, theta, tau0)
    phases = 0
    for t, (r, x) in enumerate(rows):
        want = rep.step(r["relres_first_cycle"], r["iters"], x, r["admitted"])
        assert int(want) == r["admitted"], t
        due = t + 1 >= tau0 and (phases == 0 or rep.g.due(f_r))
        assert r["trained"] == int(due), (t, rep.g.N, phases, r["trained"])
        if due:
            phases += 1
            rep.g.trained()
    assert phases >= 3 and rep.ties <= 1
