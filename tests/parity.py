"""Shared comparison helper of the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def column_errors(a, ref, axis=0):
    """Relative 2-norm error of every column of `a` against `ref`, a column running along
    `axis` (e.g. over G for each (G', omega) of dn[G][G'][omega]).  Columns whose reference
    norm is below 1e-13 of the largest column norm are measured against that largest norm
    (a structurally zero column must stay at rounding level, but has no scale of its own)."""
    a = np.moveaxis(np.asarray(a), axis, 0).reshape(np.shape(a)[axis], -1)
    r = np.moveaxis(np.asarray(ref), axis, 0).reshape(np.shape(ref)[axis], -1)
    num = np.linalg.norm(a - r, axis=0)
    den = np.linalg.norm(r, axis=0)
    floor = 1e-13 * den.max()
    return num / np.where(den > floor, den, den.max())


def assert_columns_close(a, ref, rtol, axis=0):
    err = column_errors(a, ref, axis)
    assert err.max() <= rtol, f"worst column relative error {err.max():.3e} > {rtol:g} (column {int(err.argmax())})"
