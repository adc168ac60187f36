"""GB300 (sm_103a) quasi-static projection multigrid (arXiv 1904.03808).

``binding`` is the thin ctypes face of the C ABI (include/qsmg.h) over the
CUDA library built by ``build``; ``inputs`` draws the seeded synthetic fields.
"""
from . import build, inputs  # noqa: F401
from .binding import (MG_FP64, MG_MIXED, Context, QSMGError, lib, make_state,  # noqa: F401
                      mg_stats, plastic_work, qs_state)
