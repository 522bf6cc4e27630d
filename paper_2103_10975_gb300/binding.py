"""ctypes binding of ``libmlgmres.so`` (see include/mlgmres.h).

Argument marshalling only: every step of the solve and of the network runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  The
library must have been built (``paper_2103_10975_gb300.build``); there is no
fallback of any kind when it is missing.
"""

import ctypes
import os

from . import build as _build

MLGMRES_OK = 0
MLGMRES_NOT_CONVERGED = 1
MLGMRES_ERR_ARG = -1
MLGMRES_ERR_CUDA = -2
MLGMRES_ERR_OOM = -3
MLGMRES_ERR_TIMEOUT = -4
MLGMRES_ERR_NONFINITE = -5
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM",
                -4: "ERR_TIMEOUT", -5: "ERR_NONFINITE"}

FP64 = 0
FP32_REFINE = 1
GUESS_ZERO, GUESS_PREV, GUESS_LEARNED, GUESS_USER = 0, 1, 2, 3
GUESS_NAMES = {"zero": GUESS_ZERO, "prev": GUESS_PREV, "learned": GUESS_LEARNED,
               "user": GUESS_USER}


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("kappa_dev", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int),
        ("rtol", ctypes.c_double),
        ("max_iters", ctypes.c_longlong),
        ("precision", ctypes.c_int),
        ("guess", ctypes.c_int),
        ("fallback", ctypes.c_int),
        ("replay_cap", ctypes.c_int),
        ("warmup_steps", ctypes.c_int),
        ("window_p", ctypes.c_int),
        ("ortho_theta", ctypes.c_double),
        ("deterministic_tos", ctypes.c_int),
        ("train_iters", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("lr", ctypes.c_float),
        ("seed", ctypes.c_ulonglong),
        ("grid_blocks", ctypes.c_int),
        ("batch_slots", ctypes.c_int),
        ("barrier_timeout_s", ctypes.c_double),
        ("guess_smooth", ctypes.c_int),
        ("guess_omega", ctypes.c_float),
        ("guess_select", ctypes.c_int),
        ("fault_inject", ctypes.c_int),
        ("v_stages", ctypes.c_int),
        ("retrain_after", ctypes.c_int),
        ("grow_blocks", ctypes.c_int),
        ("grow_tol", ctypes.c_double),
        ("compact", ctypes.c_int),
        ("model", ctypes.c_int),
        ("overlap_train", ctypes.c_int),
    ]


class Tuning(ctypes.Structure):
    _fields_ = [
        ("grid_blocks", ctypes.c_int),
        ("v_stages", ctypes.c_int),
        ("us_per_step", ctypes.c_float),
        ("candidates", ctypes.c_int),
        ("cand_blocks", ctypes.c_int * 32),
        ("cand_stages", ctypes.c_int * 32),
        ("cand_us_per_step", ctypes.c_float * 32),
        ("from_cache", ctypes.c_int),
        ("compact", ctypes.c_int),
        ("cand_compact", ctypes.c_int * 32),
    ]

    def as_dict(self):
        k = self.candidates
        return {"grid_blocks": self.grid_blocks, "v_stages": self.v_stages,
                "us_per_step": self.us_per_step, "from_cache": self.from_cache,
                "compact": self.compact,
                "candidates": [(self.cand_blocks[i], self.cand_stages[i],
                                self.cand_us_per_step[i], self.cand_compact[i])
                               for i in range(k)]}


class Result(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_longlong),
        ("cycles", ctypes.c_int),
        ("status", ctypes.c_int),
        ("guess_used", ctypes.c_int),
        ("admitted", ctypes.c_int),
        ("bnorm", ctypes.c_double),
        ("relres_true", ctypes.c_double),
        ("relres_first_cycle", ctypes.c_double),
        ("relres_guess", ctypes.c_double),
        ("relres_learned", ctypes.c_double),
        ("tos_ms", ctypes.c_float),
        ("guess_ms", ctypes.c_float),
        ("trained", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every exported entry point and its signature (checked against the header by
# the tests).
_vp = ctypes.c_void_p
_SIGS = {
    "mlgmres_default_options": (None, [ctypes.POINTER(Options)]),
    "mlgmres_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Options),
                                      ctypes.POINTER(_vp)]),
    "mlgmres_solve": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(Result)]),
    "mlgmres_solve_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(Grid),
                                           ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp,
                                           ctypes.POINTER(Result)]),
    "mlgmres_train_step": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_float)]),
    "mlgmres_last_error": (ctypes.c_char_p, [_vp]),
    "mlgmres_destroy": (None, [_vp]),
    "mlgmres_apply": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mlgmres_arnoldi": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       _vp, ctypes.POINTER(ctypes.c_int), _vp]),
    "mlgmres_nn_param_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "mlgmres_nn_get_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_longlong]),
    "mlgmres_nn_set_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_longlong]),
    "mlgmres_nn_forward": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "mlgmres_nn_loss_grad": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp,
                                            ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_float), _vp]),
    "mlgmres_replay_size": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "mlgmres_kernel_launches": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong)]),
    "mlgmres_solve_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_longlong, _vp, _vp, _vp,
                                            ctypes.POINTER(Result)]),
    "mlgmres_guess": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mlgmres_nn_blocks": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mlgmres_smooth": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "mlgmres_exchange_floor": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_float)]),
    "mlgmres_autotune": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp,
                                        ctypes.POINTER(Tuning)]),
    "mlgmres_batch_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
}

_lib = None


def library_path():
    return _build.LIB


def load_library(build_if_missing=True):
    """Loads libmlgmres.so (building it first if it is missing or stale and
    ``build_if_missing``).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libmlgmres.so is not built (%s); run "
                           "python -m paper_2103_10975_gb300.build" % path)
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def kernel_launches():
    c = ctypes.c_longlong(0)
    load_library().mlgmres_kernel_launches(ctypes.byref(c))
    return c.value


def exchange_floor(ctas, m, steps=2000):
    """mlgmres_exchange_floor: device microseconds per Arnoldi step of a
    persistent launch that does only the step's two group exchanges."""
    us = ctypes.c_float(0.0)
    st = load_library().mlgmres_exchange_floor(int(ctas), int(m), int(steps), ctypes.byref(us))
    if st != MLGMRES_OK:
        raise MLGMRESError(st, "exchange_floor failed")
    return us.value


def solve_static(n, b, x, m=30, rtol=1e-10, max_iters=10 ** 7, stream=None):
    """mlgmres_solve_static: the FP32-refined solve from x0 = 0 without any
    device allocation (n*n <= 65536, m <= 32).  Returns (status, result dict)."""
    r = Result()
    st = load_library().mlgmres_solve_static(int(n), int(m), float(rtol), int(max_iters),
                                             _ptr(b), _ptr(x), _stream_handle(stream),
                                             ctypes.byref(r))
    return st, r.as_dict()


def batch_plan(dim, sides, ctas):
    """mlgmres_batch_plan: the CTA groups a batched launch would use (host
    only).  Returns (group_ctas list, group_of list)."""
    count = len(sides)
    n = (ctypes.c_int * count)(*[int(v) for v in sides])
    G = ctypes.c_int(0)
    gc = (ctypes.c_int * max(1, int(ctas)))()
    go = (ctypes.c_int * count)()
    st = load_library().mlgmres_batch_plan(int(dim), count, n, int(ctas), ctypes.byref(G), gc, go)
    if st != MLGMRES_OK:
        raise MLGMRESError(st, "batch_plan: invalid arguments")
    return list(gc[:G.value]), list(go)


class MLGMRESError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def default_options(**kw):
    o = Options()
    load_library().mlgmres_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "guess" and isinstance(v, str):
            v = GUESS_NAMES[v]
        if k == "fallback" and isinstance(v, str):
            v = GUESS_NAMES[v]
        if k == "model" and isinstance(v, str):
            v = {"conv": 0, "linear": 1}[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "fp32_refine": FP32_REFINE}[v]
        setattr(o, k, v)
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Solver:
    """One MLGMRES handle: ``Solver(n, dim=2, kappa=None, **options)``.

    ``solve(b, x=None)`` takes a CUDA float64 tensor of n^dim values and
    returns (x, result dict)."""

    def __init__(self, n, dim=2, kappa=None, **opts):
        import torch
        self.lib = load_library()
        self.n = int(n)
        self.dim = int(dim)
        self.N = self.n ** self.dim
        self.kappa = None
        if kappa is not None:
            self.kappa = torch.as_tensor(kappa, dtype=torch.float32).cuda().contiguous()
        self.grid = Grid(self.dim, self.n, _ptr(self.kappa))
        self.opt = default_options(**opts)
        h = ctypes.c_void_p()
        st = self.lib.mlgmres_create(ctypes.byref(self.grid), ctypes.byref(self.opt),
                                     ctypes.byref(h))
        if st != MLGMRES_OK:
            raise MLGMRESError(st, "mlgmres_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mlgmres_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self):
        return self.lib.mlgmres_last_error(self.h).decode()

    def _check(self, st, what, allow=(MLGMRES_OK,)):
        if st not in allow:
            raise MLGMRESError(st, "%s: %s" % (what, self.error()))
        return st

    def solve(self, b, x=None, stream=None, check=True):
        import torch
        assert b.is_cuda and b.dtype == torch.float64 and b.numel() == self.N
        b = b.contiguous()
        if x is None:
            x = torch.empty_like(b)
        r = Result()
        st = self.lib.mlgmres_solve(self.h, _ptr(b), _ptr(x), _stream_handle(stream),
                                    ctypes.byref(r))
        if check:
            self._check(st, "solve", (MLGMRES_OK, MLGMRES_NOT_CONVERGED))
        d = r.as_dict()
        d["status_code"] = st
        return x, d

    def solve_batch(self, ns, bs, xs=None, stream=None, kappas=None):
        import torch
        count = len(ns)
        grids = (Grid * count)()
        for i, n in enumerate(ns):
            kp = None if kappas is None or kappas[i] is None else _ptr(kappas[i])
            grids[i] = Grid(self.dim, int(n), kp)
        if xs is None:
            xs = [torch.empty_like(b) for b in bs]
        bp = (ctypes.c_void_p * count)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * count)(*[x.data_ptr() for x in xs])
        res = (Result * count)()
        st = self.lib.mlgmres_solve_batch(self.h, count, grids, bp, xp, _stream_handle(stream),
                                          res)
        self._check(st, "solve_batch", (MLGMRES_OK, MLGMRES_NOT_CONVERGED))
        return xs, [r.as_dict() for r in res]

    def autotune(self, b, steps=0, retune=False, stream=None):
        """mlgmres_autotune: returns the tuning record as a dict."""
        t = Tuning()
        self._check(self.lib.mlgmres_autotune(self.h, _ptr(b), int(steps), int(bool(retune)),
                                              _stream_handle(stream), ctypes.byref(t)),
                    "autotune")
        return t.as_dict()

    def train_step(self, stream=None, want_loss=False):
        loss = ctypes.c_float(-1.0)
        st = self.lib.mlgmres_train_step(self.h, _stream_handle(stream),
                                         ctypes.byref(loss) if want_loss else None)
        self._check(st, "train_step")
        return loss.value if want_loss else None

    def apply(self, u, stream=None):
        import torch
        out = torch.empty_like(u)
        self._check(self.lib.mlgmres_apply(self.h, _ptr(u), _ptr(out), _stream_handle(stream)),
                    "apply")
        return out

    def arnoldi(self, v0, steps, stream=None):
        import numpy as np
        import torch
        H = np.zeros((steps, steps + 1))
        V = torch.zeros((steps + 1, self.N), dtype=torch.float64, device=v0.device)
        done = ctypes.c_int(0)
        st = self.lib.mlgmres_arnoldi(self.h, _ptr(v0), steps,
                                      H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      _ptr(V), ctypes.byref(done), _stream_handle(stream))
        self._check(st, "arnoldi")
        k = done.value
        Hm = H.T.copy()  # column-major (steps+1) x steps
        return V[: k + 1], Hm[: k + 1, :k], k

    def param_count(self):
        c = ctypes.c_longlong(0)
        self._check(self.lib.mlgmres_nn_param_count(self.h, ctypes.byref(c)), "param_count")
        return c.value

    def get_params(self):
        import numpy as np
        p = np.zeros(self.param_count(), dtype=np.float32)
        self._check(self.lib.mlgmres_nn_get_params(
            self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(p)), "get_params")
        return p

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.mlgmres_nn_set_params(
            self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(p)), "set_params")

    def nn_forward(self, u, stream=None):
        import torch
        B = u.shape[0]
        y = torch.empty_like(u)
        self._check(self.lib.mlgmres_nn_forward(self.h, B, _ptr(u), _ptr(y),
                                                _stream_handle(stream)), "nn_forward")
        return y

    def nn_loss_grad(self, u, t, stream=None):
        import numpy as np
        B = u.shape[0]
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = ctypes.c_float(0)
        self._check(self.lib.mlgmres_nn_loss_grad(
            self.h, B, _ptr(u), _ptr(t), ctypes.byref(loss),
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream_handle(stream)),
            "nn_loss_grad")
        return loss.value, g

    def guess(self, b, stream=None):
        """mlgmres_guess: the network's x0 for b (no solve)."""
        import torch
        x = torch.empty_like(b)
        self._check(self.lib.mlgmres_guess(self.h, _ptr(b), _ptr(x), _stream_handle(stream)),
                    "guess")
        return x

    def smooth(self, b, x, sweeps, stream=None):
        """mlgmres_smooth: `sweeps` damped-Jacobi sweeps of A x = b on x, in place."""
        self._check(self.lib.mlgmres_smooth(self.h, _ptr(b), _ptr(x), int(sweeps),
                                            _stream_handle(stream)), "smooth")
        return x

    def nn_blocks(self, set_to=-1):
        """mlgmres_nn_blocks: residual blocks appended so far (optionally set)."""
        c = ctypes.c_int(0)
        self._check(self.lib.mlgmres_nn_blocks(self.h, int(set_to), ctypes.byref(c)),
                    "nn_blocks")
        return c.value

    def replay_size(self):
        c = ctypes.c_int(0)
        self._check(self.lib.mlgmres_replay_size(self.h, ctypes.byref(c)), "replay_size")
        return c.value
