"""Parareal with low-rank coarse solvers (Gander, Ohlberger, Rave, arXiv
2508.08873) on GB300: a C-ABI CUDA library (include/lrp.h) with a thin Python
binding.  The CUDA library is loaded lazily on first use."""
from .api import (Context, Operator, Coarse, Server, propagate, parareal_solve, fine_solution,
                  gaussian, PREC_F64, PREC_MIXED)

__all__ = ["Context", "Operator", "Coarse", "Server", "propagate", "parareal_solve",
           "fine_solution", "gaussian", "PREC_F64", "PREC_MIXED"]
