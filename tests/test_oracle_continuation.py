"""Pins of the imaginary-axis density response and of the AAA continuation oracle (Sec. 2.7):
the sum over states at imaginary frequencies with its symmetry and sign, exact recovery of
rational functions, interpolation at the support points, accuracy on an analytic function,
and a planted mistake.  CPU only."""
import math

import numpy as np
import pytest

import instances as I
import oracle as O


def test_imaginary_axis_response_is_hermitian_and_negative():
    """For w = i omega each pair of terms 1/(a + w) + 1/(a - w) = 2a / (a^2 + omega^2) is real, and
    negative when every unoccupied level at k+q lies above every occupied level at k: the
    response is Hermitian negative semidefinite and decays with omega."""
    inst = I.tiny_fcc(ecut_ry=5.0, dims=(16, 16, 16), n_occ=2, n_pert=4, n_omega=3)
    kp = inst.kpoints[0]
    hk, mk, _ = O.dense_h_inst(inst, kp.k_frac)
    hq, mq, _ = O.dense_h_inst(inst, kp.kq_frac)
    wk, vk = np.linalg.eigh(hk)
    wq, vq = np.linalg.eigh(hq)
    assert wq[2] > wk[1]
    w = 1j * np.array([0.05, 0.5, 2.0])
    dn = O.density_response_w(hq, vq[:, :2].T.copy(), vk[:, :2].T.copy(), mk, mq, wk[:2], inst.gp_miller, w,
                              inst.fft_dims, 1.0)
    sos = O.density_response_sos(hq, 2, vk[:, :2].T.copy(), mk, mq, wk[:2], inst.gp_miller, None, None, 1.0, w=w)
    assert np.abs(dn - sos).max() <= 1e-11 * np.abs(sos).max()
    norms = []
    for j in range(3):
        m = dn[:, :, j]
        np.testing.assert_allclose(m, m.conj().T, atol=1e-12 * np.abs(m).max())
        ev = np.linalg.eigvalsh(0.5 * (m + m.conj().T))
        assert ev.max() <= 1e-12 * np.abs(ev).max()
        norms.append(np.abs(ev).max())
    assert norms[0] > norms[1] > norms[2]


def _model(z):
    """A rational function of type (3, 3): three simple poles off the imaginary axis."""
    p = np.array([0.7 - 0.01j, -0.7 - 0.01j, 1.9 - 0.2j])
    a = np.array([0.3 + 0.1j, -0.3 + 0.1j, 0.8])
    return 1.0 + np.sum(a[None, :] / (np.asarray(z)[:, None] - p[None, :]), axis=1)


def test_aaa_recovers_a_rational_function_off_the_sample_line():
    zi = 1j * np.linspace(0.02, 6.0, 48)
    zs, fs, w = O.aaa(zi, _model(zi), tol=1e-13, mmax=20)
    assert len(zs) <= 5
    x = np.linspace(-3.0, 3.0, 41) + 0.02j           # the real axis, slightly above the poles
    ref = _model(x)
    assert np.abs(O.aaa_eval(zs, fs, w, x) - ref).max() <= 1e-8 * np.abs(ref).max()


def test_aaa_interpolates_its_support_points():
    zi = 1j * np.linspace(0.1, 4.0, 30)
    f = np.exp(zi) / (1.0 + zi ** 2 / 9.0)
    zs, fs, w = O.aaa(zi, f, tol=1e-12)
    np.testing.assert_array_equal(O.aaa_eval(zs, fs, w, zs), fs)
    rest = np.setdiff1d(np.arange(len(zi)), [int(np.nonzero(zi == s)[0][0]) for s in zs])
    assert np.abs(O.aaa_eval(zs, fs, w, zi[rest]) - f[rest]).max() <= 1e-12 * np.abs(f).max() * 10


def test_aaa_accuracy_on_an_analytic_function():
    """exp on [-1, 1] is approximated to 1e-13 by a low-degree rational (a textbook AAA case)."""
    x = np.linspace(-1.0, 1.0, 200).astype(complex)
    zs, fs, w = O.aaa(x, np.exp(x), tol=1e-13)
    assert len(zs) <= 12
    t = np.linspace(-1.0, 1.0, 777)
    assert np.abs(O.aaa_eval(zs, fs, w, t) - np.exp(t)).max() < 1e-12


def test_mutation_largest_singular_vector_is_caught():
    """Weights from the largest instead of the smallest singular vector do not reproduce the
    rational model: the recovery pin would fail."""
    zi = 1j * np.linspace(0.02, 6.0, 48)
    f = _model(zi)
    zs, fs, w = O.aaa(zi, f, tol=1e-13, mmax=20)
    idx = np.array([k for k in range(len(zi)) if zi[k] not in zs])
    loew = (f[idx][:, None] - fs[None, :]) / (zi[idx][:, None] - zs[None, :])
    _, _, vh = np.linalg.svd(loew)
    bad = vh[0].conj()
    x = np.linspace(-3.0, 3.0, 41) + 0.02j
    assert np.abs(O.aaa_eval(zs, fs, bad, x) - _model(x)).max() > 1e-3
    assert math.isfinite(float(np.abs(O.aaa_eval(zs, fs, w, x)).max()))
