"""GB300 (sm_103a) shifted-Sternheimer solver: C-ABI library + thin Python binding."""
from .sgw import (EXPORTS, LIB_PATH, MLP, MLP_PARAMS, PAIR_BREAKDOWN, PAIR_CONVERGED, PAIR_MAXITER, PAIR_NONFINITE,
                  SGW_EALIAS, SGW_ECUDA, SGW_EINVAL, SGW_ENOCONV, SGW_ENOMEM, SGW_ESTATE, SGW_EUNSUPPORTED, SGW_OK,
                  SgwError, System, aaa, load, screened_coulomb, solve_batched)

__all__ = ["EXPORTS", "LIB_PATH", "MLP", "MLP_PARAMS", "PAIR_BREAKDOWN", "PAIR_CONVERGED", "PAIR_MAXITER", "PAIR_NONFINITE",
           "SGW_EALIAS", "SGW_ECUDA", "SGW_EINVAL", "SGW_ENOCONV", "SGW_ENOMEM", "SGW_ESTATE", "SGW_EUNSUPPORTED", "SGW_OK",
           "SgwError", "System", "aaa", "load", "screened_coulomb",
           "solve_batched"]
