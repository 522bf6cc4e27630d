"""The bulk-copy variants' stages carry the stencil's neighbour windows of w'
(and of kappa in 3D) besides the basis.  kappa's windows are staged only when
its copies can be 16-byte aligned (aligned base, N a multiple of 4); otherwise
the stencil reads kappa per point.  Each path is checked here against the FP64
oracle after one GMRES(m) cycle from x0 = 0 (E_k, Sec. 2.2): the FP64 variant's
true residual and iterate agree with the oracle's to rounding, and the
FP32-refined variant's reported residual is the one the oracle's operator
measures on the returned x (its certificate)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import native  # noqa: E402
from synthetic import MovingGaussians3D, lognormal_kappa  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2103_10975_gb300 import Solver  # noqa: E402

THREADS = max(1, min(16, os.cpu_count() or 1))


def _kappa_dev(kap, offset):
    """kappa on the device; offset 1 places it 4 bytes past a 16-byte boundary."""
    buf = torch.empty(kap.size + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.as_tensor(kap.ravel(), dtype=torch.float32)
    return buf[offset:]


@pytest.mark.parametrize("n,offset", [(40, 0), (40, 1), (37, 0)])
def test_3d_kappa_stage_paths(n, offset):
    m = 20
    kap = lognormal_kappa(n, 7001).astype(np.float32)
    kd = kap.astype(np.float64)
    b = MovingGaussians3D(n, 7001, 50).rhs(3)
    xr, st, _ = native.gmres(3, n, b, m=m, rtol=1e-12, max_iters=m, kappa=kd, nthreads=THREADS)
    nb = np.linalg.norm(b)
    e_orc = float(np.linalg.norm(b - native.apply(3, n, xr, kd)) / nb)
    kdev = _kappa_dev(kap, offset)
    assert (kdev.data_ptr() % 16 == 0) == (offset == 0)
    bd = torch.as_tensor(b).cuda()
    for prec in ("fp64", "fp32_refine"):
        s = Solver(n, dim=3, kappa=kdev, m=m, rtol=1e-12, precision=prec, max_iters=m,
                   v_stages=4)
        assert s.kappa.data_ptr() == kdev.data_ptr()  # the view itself, not a copy
        x, r = s.solve(bd)
        assert r["iters"] == m and r["cycles"] == 1, (prec, r)
        xg = x.cpu().numpy()
        e_chk = float(np.linalg.norm(b - native.apply(3, n, xg, kd)) / nb)
        assert abs(e_chk - r["relres_true"]) <= 1e-6 * e_chk, (prec, e_chk, r)
        if prec == "fp64":
            assert abs(r["relres_true"] - e_orc) <= 1e-6 * e_orc, (r["relres_true"], e_orc)
            assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)


@pytest.mark.parametrize("n", [64, 66])
def test_2d_stencil_rows_unaligned(n):
    """2D bulk variant (two CTAs: the slices exceed shared memory) with n % 4 = 0
    and 2: for n = 66 the +-n rows of w' start off a 16-byte boundary in FP32
    and are copied from the boundary below."""
    m = 20
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n * n)
    nb = np.linalg.norm(b)
    xr, st, _ = native.gmres(2, n, b, m=m, rtol=1e-12, max_iters=m, nthreads=THREADS)
    e_orc = float(np.linalg.norm(b - native.apply(2, n, xr, None)) / nb)
    for prec in ("fp64", "fp32_refine"):
        s = Solver(n, m=m, rtol=1e-12, precision=prec, max_iters=m, grid_blocks=2, v_stages=4)
        x, r = s.solve(torch.as_tensor(b).cuda())
        assert r["iters"] == m and r["cycles"] == 1, (prec, r)
        xg = x.cpu().numpy()
        e_chk = float(np.linalg.norm(b - native.apply(2, n, xg, None)) / nb)
        assert abs(e_chk - r["relres_true"]) <= 1e-6 * e_chk, (prec, e_chk, r)
        if prec == "fp64":
            assert abs(r["relres_true"] - e_orc) <= 1e-6 * e_orc, (r["relres_true"], e_orc)
            assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)
