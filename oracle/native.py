"""Builds and loads the plain-C FP64 GMRES oracle (``gmres_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmres_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_long),
        ("cycles", ctypes.c_int),
        ("status", ctypes.c_int),
        ("bnorm", ctypes.c_double),
        ("relres_true", ctypes.c_double),
        ("relres_first_cycle", ctypes.c_double),
        ("relres_guess", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def build(force=False):
    """Compile the oracle with gcc (OpenMP for the optional threaded mode)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            L.oracle_apply_2d.argtypes = [ctypes.c_int, dp, dp]
            L.oracle_apply_2d.restype = None
            L.oracle_apply_3d.argtypes = [ctypes.c_int, dp, dp, dp]
            L.oracle_apply_3d.restype = None
            L.oracle_arnoldi.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp, dp,
                                         ctypes.c_int]
            L.oracle_arnoldi.restype = ctypes.c_int
            L.oracle_gmres.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_long, ctypes.c_int,
                                       ctypes.POINTER(OracleStats), dp, ctypes.c_long]
            L.oracle_gmres.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def apply_2d(n, u):
    u = _f64(u)
    out = np.empty(n * n)
    lib().oracle_apply_2d(n, _ptr(u), _ptr(out))
    return out


def apply_3d(n, u, kappa=None):
    u = _f64(u)
    out = np.empty(n ** 3)
    if kappa is not None:
        kap = _f64(kappa)
        lib().oracle_apply_3d(n, _ptr(kap), _ptr(u), _ptr(out))
    else:
        lib().oracle_apply_3d(n, None, _ptr(u), _ptr(out))
    return out


def apply(dim, n, u, kappa=None):
    return apply_2d(n, u) if dim == 2 else apply_3d(n, u, kappa)


def arnoldi(dim, n, v0, m, kappa=None, nthreads=1):
    """MGS Arnoldi: returns (V[(m+1), N], H[(m+1), m], steps)."""
    N = n ** dim
    v0 = _f64(v0)
    V = np.zeros((m + 1, N))
    Hf = np.zeros(m * (m + 1))
    kap = _f64(kappa) if kappa is not None else None
    steps = lib().oracle_arnoldi(dim, n, _ptr(kap) if kap is not None else None, _ptr(v0), m,
                                 _ptr(V), _ptr(Hf), nthreads)
    H = Hf.reshape(m, m + 1).T.copy()  # column-major storage -> (m+1, m)
    return V, H, steps


def gmres(dim, n, b, m, rtol, max_iters=10 ** 9, x0=None, kappa=None, nthreads=1,
          hist_cap=0):
    """FP64 restarted GMRES(m).  Returns (x, stats dict, hist) where hist holds
    the implicit relative residual |g_{j+1}|/||b|| after each iteration."""
    N = n ** dim
    b = _f64(b)
    x = np.zeros(N) if x0 is None else _f64(x0).copy()
    st = OracleStats()
    hist = np.zeros(max(hist_cap, 1))
    kap = _f64(kappa) if kappa is not None else None
    lib().oracle_gmres(dim, n, _ptr(kap) if kap is not None else None, _ptr(b), _ptr(x), m,
                       float(rtol), int(max_iters), int(nthreads), ctypes.byref(st), _ptr(hist),
                       int(hist_cap))
    d = st.as_dict()
    return x, d, hist[: min(hist_cap, d["iters"])]
