"""Pins of the screening oracle (Sec. 2.4 and 2.6: truncated Coulomb potential, Eq. 4 dielectric
matrix, its inverse and W-bar of Eq. 9) against numerical quadrature, closed forms and
perturbation series.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


@pytest.mark.parametrize("q,r_cut", [(0.3, 5.0), (1.7, 3.2), (0.05, 8.0)])
def test_truncated_coulomb_by_quadrature(q, r_cut):
    """v(q) = integral over |r| < R_cut of exp(-i q.r) / |r|, done numerically in spherical
    coordinates (the imaginary part cancels)."""
    val, _ = integrate.dblquad(lambda th, r: 2.0 * math.pi * r * math.sin(th) * math.cos(q * r * math.cos(th)),
                               0.0, r_cut, 0.0, math.pi, epsabs=1e-12, epsrel=1e-11)
    v = O.coulomb_spherical([[q, 0.0, 0.0]], r_cut)[0]
    assert v == pytest.approx(val, rel=1e-9)


def test_truncated_coulomb_limits():
    r = 4.0
    # q -> 0: 2 pi R^2, continuous across the series / closed-form switch
    v = O.coulomb_spherical([[0.0, 0.0, 0.0], [1e-7, 0, 0], [2e-5, 0, 0], [3e-5, 0, 0]], r)
    assert v[0] == pytest.approx(2.0 * math.pi * r * r, rel=1e-15)
    assert np.all(np.abs(v - v[0]) <= 1e-8 * v[0])
    # direction-independent, bare potential when not truncated
    a = O.coulomb_spherical([[0.3, 0.4, 0.0], [0.0, 0.0, 0.5]], r)
    assert a[0] == pytest.approx(a[1], rel=1e-14)
    np.testing.assert_allclose(O.coulomb_spherical([[0.5, 0, 0]], 0.0), [4.0 * math.pi / 0.25], rtol=1e-15)
    with pytest.raises(ValueError):
        O.coulomb_spherical([[0.0, 0.0, 0.0]], 0.0)


def _qg(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.8, (n, 3)) + np.array([0.1, 0.0, 0.0])


def test_diagonal_response_closed_form():
    n, vol, r = 5, 270.0, 6.0
    qg = _qg(n)
    d = (-0.5 - 0.2j) * np.arange(1, n + 1)
    dn = np.zeros((n, n, 2), complex)
    dn[np.arange(n), np.arange(n), 0] = d
    dn[np.arange(n), np.arange(n), 1] = 2 * d
    einv, wbar = O.screened_coulomb(dn, qg, vol, r)
    v = O.coulomb_spherical(qg, r)
    for j, f in enumerate((1.0, 2.0)):
        e = 1.0 - f * d * v / vol
        np.testing.assert_allclose(np.diagonal(einv[:, :, j]), 1.0 / e, rtol=1e-14)
        np.testing.assert_allclose(np.diagonal(wbar[:, :, j]), v * (1.0 / e - 1.0), rtol=1e-13)
        off = einv[:, :, j] - np.diag(np.diagonal(einv[:, :, j]))
        assert np.abs(off).max() == 0.0


def test_perturbation_series_and_hermiticity():
    """W-bar = v chi v + v chi v chi v + O(chi^3) with chi = dn / Omega (v on the row, chi v the
    response to the Coulomb potential of a unit charge); a Hermitian static response gives a
    Hermitian W-bar."""
    n, vol, r = 6, 1080.0, 7.0
    qg = _qg(n, 3)
    rng = np.random.default_rng(4)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    herm = -(a @ a.conj().T)                      # negative definite like a static response
    scale = 1e-4
    dn = (scale * herm)[:, :, None]
    einv, wbar = O.screened_coulomb(dn, qg, vol, r)
    v = O.coulomb_spherical(qg, r)
    chi = dn[:, :, 0] / vol
    vm = np.diag(v)
    first = vm @ chi @ vm
    second = first + vm @ chi @ vm @ chi @ vm
    third = vm @ chi @ vm @ chi @ vm @ chi @ vm
    err1 = np.abs(wbar[:, :, 0] - first).max()
    err2 = np.abs(wbar[:, :, 0] - second).max()
    assert err2 < 2.0 * np.abs(third).max() + 1e-15 * np.abs(first).max()
    assert err2 < 1e-2 * err1
    np.testing.assert_allclose(wbar[:, :, 0], wbar[:, :, 0].conj().T, atol=1e-13 * np.abs(wbar).max())


def test_mutation_coulomb_on_the_row_is_caught():
    """The same series with v placed on the row of epsilon (eps = 1 - v chi) gives a different
    W-bar: the series pin distinguishes the two placements."""
    n, vol, r = 6, 1080.0, 7.0
    qg = _qg(n, 3)
    rng = np.random.default_rng(5)
    chi = 1e-4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    v = O.coulomb_spherical(qg, r)
    eps_row = np.eye(n) - v[:, None] * chi
    w_row = v[:, None] * (np.linalg.inv(eps_row) - np.eye(n))
    _, wbar = O.screened_coulomb((chi * vol)[:, :, None], qg, vol, r)
    assert np.abs(w_row - wbar[:, :, 0]).max() > 1e-3 * np.abs(wbar).max()


def test_zero_wavevector_keeps_only_the_diagonal():
    n, vol, r = 4, 500.0, 5.0
    qg = _qg(n, 6)
    qg[2] = 0.0
    rng = np.random.default_rng(7)
    dn = 0.3 * (rng.standard_normal((n, n, 1)) + 1j * rng.standard_normal((n, n, 1)))
    einv, wbar = O.screened_coulomb(dn, qg, vol, r)
    assert np.all(einv[2, [0, 1, 3], 0] == 0) and np.all(einv[[0, 1, 3], 2, 0] == 0)
    assert einv[2, 2, 0] != 0
