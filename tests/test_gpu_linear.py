"""The simplified model of Sec. 3.1: a single dense layer x0 = c T b trained
online on a randomly moving localized source at 30 x 30.  Its guess gives
r0 = (I - c A T) b, so ||r0|| <= ||I - c A T||_2 ||b||, and as T learns, the
eigenvalues of c A T move from 0 towards 1 (onto the unit circle) along the
directions the training pairs span."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct  # noqa: E402
from synthetic import RandomWalkSources2D  # noqa: E402

pytestmark = pytest.mark.gpu


def test_linear_model_spectrum_moves_to_one():
    from paper_2103_10975_gb300 import Solver
    n, T, tau0 = 30, 150, 20
    N = n * n
    gen = RandomWalkSources2D(n, 7001, n_sources=1, alpha=0.0, step=0.1)
    s = Solver(n, m=30, rtol=1e-10, guess="learned", fallback="zero", model="linear",
               warmup_steps=tau0, train_iters=64, lr=0.5, batch=8, guess_smooth=0,
               deterministic_tos=1, seed=3)
    A = direct.dense_laplacian_2d(n)

    def spectrum():
        """Eigenvalues of c A T for the current T (c from the guess itself)."""
        Tm = s.get_params().reshape(N, N).astype(np.float64)
        bb = gen.rhs(0)
        Tb = Tm @ bb
        if not np.any(Tb):
            return np.zeros(N)
        x0 = s.guess(torch.as_tensor(bb).cuda()).cpu().numpy()
        return np.linalg.eigvals((float(x0 @ Tb) / float(Tb @ Tb)) * A @ Tm)

    r0s, near_at = [], []
    for t in range(T):
        if t in (tau0 - 1, T // 2):
            near_at.append(np.mean(np.abs(spectrum() - 1.0) < 0.3))
        b = gen.rhs(t)
        bd = torch.as_tensor(b).cuda()
        if t >= T - 20:
            x0 = s.guess(bd).cpu().numpy()
            r0s.append(np.linalg.norm(b - A @ x0) / np.linalg.norm(b))
        x, r = s.solve(bd)
        assert r["status"] == 0 and r["relres_true"] <= 1e-10
        if (t + 1) % 5 == 0:
            s.train_step()
    # the guess is linear in b: x0 = c T b
    Tm = s.get_params().reshape(N, N).astype(np.float64)
    b = gen.rhs(T)
    x0 = s.guess(torch.as_tensor(b).cuda()).cpu().numpy()
    Tb = Tm @ b
    c = float(x0 @ Tb) / float(Tb @ Tb)
    assert np.linalg.norm(x0 - c * Tb) <= 1e-4 * np.linalg.norm(x0)
    M = c * A @ Tm
    lam = np.linalg.eigvals(M)
    near = np.mean(np.abs(lam - 1.0) < 0.3)
    # ||r0|| <= ||I - cAT|| ||b|| (an equality only for the worst b)
    r0 = np.linalg.norm(b - A @ x0)
    bound = np.linalg.norm(np.eye(N) - M, 2) * np.linalg.norm(b)
    assert r0 <= bound * (1 + 1e-6)
    print("linear model: eigenvalues of cAT within 0.3 of 1: %.1f%% at step %d, %.1f%% at %d, "
          "%.1f%% at %d; median |lambda| %.3f, ||I - cAT||_2 %.2f, r0/||b|| over the last "
          "20 steps %.3f" % (100 * near_at[0], tau0 - 1, 100 * near_at[1], T // 2, 100 * near, T,
                             np.median(np.abs(lam)), np.linalg.norm(np.eye(N) - M, 2),
                             float(np.mean(r0s))))
    # T = 0 gives all eigenvalues 0; training moves more of them to 1 as it
    # sees more of the source's positions, and the guess beats x0 = 0
    assert near_at[0] == 0.0
    assert near >= near_at[1] > 0.0
    assert np.mean(r0s) < 1.0
