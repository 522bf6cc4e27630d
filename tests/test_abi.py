"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/mlgmres.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import paper_2103_10975_gb300 as pkg
from paper_2103_10975_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:mlgmres_status|void|const char\*)\s+(mlgmres_\w+)\s*\(",
                                src, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mlgmres_create", "mlgmres_solve", "mlgmres_solve_batch",
                     "mlgmres_train_step", "mlgmres_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = pkg.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding._SIGS, name


def test_struct_layouts_match_header():
    # sizes of the C structs as laid out by a C compiler on this ABI
    assert ctypes.sizeof(binding.Grid) == 16
    assert ctypes.sizeof(binding.Result) == 8 + 4 * 4 + 5 * 8 + 2 * 4 + 4 + 4  # + trained, pad
    o = binding.default_options()
    assert o.m == 30 and o.rtol == 1e-10 and o.replay_cap == 64 and o.warmup_steps == 50
    assert o.window_p == 10 and abs(o.ortho_theta - 0.9) < 1e-15 and o.batch == 8
    assert o.fault_inject == 0 and o.v_stages == -1 and o.retrain_after == 0
    assert o.grow_blocks == 0 and o.grow_tol == 0.02 and o.overlap_train == 1


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    lib = pkg.load_library()
    g = binding.Grid(2, 16, None)
    o = binding.default_options()
    h = ctypes.c_void_p()
    st = lib.mlgmres_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h))
    assert st in (binding.MLGMRES_ERR_CUDA, binding.MLGMRES_ERR_OOM) and not h.value
    # invalid arguments are rejected before any device call
    g = binding.Grid(4, 16, None)
    assert lib.mlgmres_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == \
        binding.MLGMRES_ERR_ARG
