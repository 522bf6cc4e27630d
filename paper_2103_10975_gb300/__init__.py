"""GB300 (sm_103a) MLGMRES: restarted GMRES(m) on time-stepped Poisson systems
with an online-trained initial-guess network (arXiv 2103.10975).

The compute path is the C-ABI library ``libmlgmres.so`` (CUDA kernels under
``csrc/``, declared in ``include/mlgmres.h``); ``binding`` is its ctypes
wrapper.  Importing this package does not load the library; the first use of
``Solver`` or ``load_library`` does, and raises if it is missing.
"""

from .binding import (Solver, Result, Options, Grid, default_options, load_library,  # noqa: F401
                      library_path, MLGMRESError, kernel_launches, batch_plan, exchange_floor, FP64, FP32_REFINE, GUESS_ZERO, GUESS_PREV,
                      GUESS_LEARNED, GUESS_USER)
