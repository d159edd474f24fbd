"""GB300 (sm_103a) shifted-Sternheimer solver: C-ABI library + thin Python binding."""
from .sgw import (EXPORTS, LIB_PATH, MLP, MLP_PARAMS, PAIR_BREAKDOWN, PAIR_CONVERGED, PAIR_MAXITER, PAIR_NONFINITE,
                  SgwError, System, aaa, load, screened_coulomb)

__all__ = ["EXPORTS", "LIB_PATH", "MLP", "MLP_PARAMS", "PAIR_BREAKDOWN", "PAIR_CONVERGED", "PAIR_MAXITER", "PAIR_NONFINITE",
           "SgwError", "System", "aaa", "load", "screened_coulomb"]
