"""The ctypes binding refuses buffers whose shape or dtype does not match the sizes it passes
to the C ABI (the library sees pointers only, so a short buffer would be read or written past
its end on the device), and lets every well-formed call through to the library.

No GPU is needed: a handle-less System stands in for a real one.  A malformed call must fail
in the binding (ValueError / TypeError) before the library is reached; a well-formed call
reaches the library, which refuses the NULL handle with SGW_EINVAL."""
import ctypes

import numpy as np
import pytest

import paper_1812_03717_gb300 as P
from paper_1812_03717_gb300 import build as B
from paper_1812_03717_gb300 import sgw as S

NPW = 12


@pytest.fixture(scope="module")
def sys_():
    import os
    if not os.path.exists(B.LIB):
        B.build()
    s = S.System.__new__(S.System)
    s._h = ctypes.c_void_p()     # NULL: the library refuses it before touching a device
    s.n_pw = NPW
    s.nocc = 0
    return s


def _c(*shape):
    return np.zeros(shape, dtype=np.complex128)


def _reaches_library(call):
    with pytest.raises(S.SgwError) as e:
        call()
    assert e.value.status == S.SGW_EINVAL


def test_solve_shifted_shapes(sys_):
    om = np.linspace(0.0, 1.0, 4)
    with pytest.raises(ValueError):
        sys_.solve_shifted(_c(3, NPW - 1), np.zeros(3), om, 0.01)        # wrong n_pw
    with pytest.raises(ValueError):
        sys_.solve_shifted(_c(NPW), np.zeros(1), om, 0.01)               # one vector, not [rows][n_pw]
    with pytest.raises(ValueError):
        sys_.solve_shifted(_c(3, NPW), np.zeros(2), om, 0.01)            # e_ref shorter than rhs
    with pytest.raises(ValueError):
        sys_.solve_shifted(_c(3, NPW), np.zeros(3), om, 0.01, out=_c(3, 3, NPW))
    with pytest.raises(TypeError):
        sys_.solve_shifted(_c(3, NPW), np.zeros(3), om, 0.01, out=np.zeros((3, 4, NPW), np.complex64))
    with pytest.raises(ValueError):
        sys_.solve_shifted(_c(3, NPW), np.zeros(3), om, 0.01, x0=_c(3, 4, NPW - 1))
    _reaches_library(lambda: sys_.solve_shifted(_c(3, NPW), np.zeros(3), om, 0.01))
    _reaches_library(lambda: sys_.solve_shifted(_c(3, NPW), np.zeros(3), om, 0.01, out=_c(3, 4, NPW),
                                                x0=_c(3, 4, NPW)))


def test_apply_and_occupied_shapes(sys_):
    with pytest.raises(ValueError):
        sys_.apply_h(_c(2, NPW + 1))
    with pytest.raises(ValueError):
        sys_.apply_h(_c(2, NPW), out=_c(3, NPW))
    with pytest.raises(ValueError):
        sys_.apply_shifted(_c(2, 2, NPW), 0.1 + 0.01j)
    with pytest.raises(ValueError):
        sys_.set_occupied(_c(3, NPW), np.zeros(4))
    _reaches_library(lambda: sys_.apply_h(_c(2, NPW)))
    _reaches_library(lambda: sys_.apply_h(_c(NPW)))
    _reaches_library(lambda: sys_.apply_shifted(_c(2, NPW), [0.1 + 0.01j, 0.2 + 0.01j]))
    _reaches_library(lambda: sys_.set_occupied(_c(4, NPW), np.zeros(4)))


def test_make_rhs_shapes(sys_):
    sk = S.System.__new__(S.System)
    sk._h = ctypes.c_void_p()
    sk.n_pw = NPW + 3
    gp = np.zeros((2, 3), dtype=np.int32)
    with pytest.raises(ValueError):
        sys_.make_rhs(sk, _c(4, NPW), gp)                  # psi_k lives in the k basis (n_pw + 3)
    with pytest.raises(ValueError):
        sys_.make_rhs(sk, _c(4, NPW + 3), gp, out=_c(4, NPW))
    _reaches_library(lambda: sys_.make_rhs(sk, _c(4, NPW + 3), gp))


def test_residual_pershift_and_density_shapes(sys_):
    om = np.linspace(0.0, 1.0, 4)
    with pytest.raises(ValueError):
        sys_.residual(_c(3, NPW), np.zeros(3), om, 0.01, _c(3, 3, NPW))
    with pytest.raises(ValueError):
        sys_.solve_pershift(_c(3, NPW), np.zeros(3), np.zeros(2), 0.01)
    with pytest.raises(ValueError):
        sys_.solve_pershift(_c(3, NPW), np.zeros(3), np.zeros(3), 0.01, out=_c(2, NPW))
    with pytest.raises(ValueError):
        sys_.precond_diag(_c(3, NPW), np.zeros(1), np.zeros(3), 0.01)
    with pytest.raises(ValueError):
        sys_.density_response(_c(6, NPW - 2), np.zeros(2), om, 0.01)
    with pytest.raises(ValueError):
        sys_.density_response(_c(6, NPW), np.zeros(2), om, 0.01, out=_c(3, 3, 3))
    with pytest.raises(ValueError):
        sys_.solve_green([0, 1], [0.1 + 0.01j], out=_c(2, 2, NPW))
    _reaches_library(lambda: sys_.residual(_c(3, NPW), np.zeros(3), om, 0.01, _c(3, 4, NPW)))
    _reaches_library(lambda: sys_.solve_pershift(_c(3, NPW), np.zeros(3), np.zeros(3), 0.01))
    _reaches_library(lambda: sys_.precond_diag(_c(3, NPW), np.zeros(3), np.zeros(3), 0.01))
    _reaches_library(lambda: sys_.density_response(_c(6, NPW), np.zeros(2), om, 0.01, out=_c(3, 3, 4)))
    _reaches_library(lambda: sys_.solve_green([0, 1], [0.1 + 0.01j], out=_c(2, 1, NPW)))


def test_batched_item_shapes(sys_):
    om = np.linspace(0.0, 1.0, 4)
    with pytest.raises(ValueError):
        P.solve_batched([{"sys": sys_, "rhs": _c(3, NPW), "e_ref": np.zeros(2), "omega": om}], 0.01)
    with pytest.raises(ValueError):
        P.solve_batched([{"sys": sys_, "rhs": _c(3, NPW), "e_ref": np.zeros(3), "omega": om,
                          "out": _c(3, 4, NPW - 1)}], 0.01)
