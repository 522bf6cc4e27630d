"""mlgmres_solve_static against mlgmres_solve.

The static entry point serves callers that cannot allocate device memory (a
memory pool that owns all free device memory, a thread that must not enter an
allocator while it solves): it runs the same persistent solver on a fixed
array compiled into the library.  This file is collected last so that a run
stopping at its first failure has already run every other test; it passes on
its own in a fresh process and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct  # noqa: E402
from synthetic import MovingGaussians2D  # noqa: E402

pytestmark = pytest.mark.gpu


def test_static_solve_matches_handle_solve_twice():
    from paper_2103_10975_gb300 import Solver, binding
    n, m, rtol = 128, 30, 1e-10
    gen = MovingGaussians2D(n, 2001, 500)
    ref = Solver(n, m=m, rtol=rtol, precision="fp32_refine", guess="zero", max_iters=300000)
    for t in (3, 4):  # two calls in a row reuse the same fixed array
        b = torch.as_tensor(gen.rhs(t)).cuda()
        x_ref, r_ref = ref.solve(b)
        x = torch.full_like(b, float("nan"))
        st, r = binding.solve_static(n, b, x, m=m, rtol=rtol, max_iters=300000)
        assert st == binding.MLGMRES_OK, (st, r)
        assert r["status"] == 0 and r["relres_true"] <= rtol
        xs, xr = x.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(xs - xr) <= 1e-7 * np.linalg.norm(xr)
        assert abs(r["iters"] - r_ref["iters"]) <= max(2, 0.01 * r_ref["iters"])
        xe = direct.dst_solve_2d(n, gen.rhs(t))
        assert np.linalg.norm(xs - xe) <= 1e-7 * np.linalg.norm(xe)


def test_static_solve_leaves_free_device_memory_unchanged():
    """The property the entry point exists for: a call takes no device memory.
    After a first call (which loads the library's module with its fixed array),
    the free device memory reported by the driver is the same before and after
    a second call."""
    from paper_2103_10975_gb300 import binding
    n = 96
    b = torch.as_tensor(MovingGaussians2D(n, 2001, 500).rhs(7)).cuda()
    x = torch.zeros_like(b)
    st, _ = binding.solve_static(n, b, x, m=20, rtol=1e-8, max_iters=100000)
    assert st == binding.MLGMRES_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st, r = binding.solve_static(n, b, x, m=20, rtol=1e-8, max_iters=100000)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == binding.MLGMRES_OK and r["relres_true"] <= 1e-8
    assert free1 == free0, (free0, free1)


def test_static_solve_rejects_sizes_beyond_the_fixed_array():
    from paper_2103_10975_gb300 import binding
    b = torch.zeros(257 * 257, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _ = binding.solve_static(257, b, x)
    assert st == binding.MLGMRES_ERR_ARG
    b = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _ = binding.solve_static(64, b, x, m=33)
    assert st == binding.MLGMRES_ERR_ARG
