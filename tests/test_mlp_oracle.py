"""Pins of the learned-preconditioner oracle (perceptron, Adam, scalings) by routes other
than its own formulas: finite differences, quadrature, closed-form Adam steps, exact
bfloat16 values, and the zero-output-layer identity."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def _theta(seed=0, scale_last=0.1):
    rng = np.random.default_rng(seed)
    th = M.init_params(rng).astype(np.float64)
    th[-(M.N_H + 1):] = scale_last * rng.standard_normal(M.N_H + 1)
    return th


def test_parameter_count():
    assert M.N_PARAMS == 4545


def test_gelu_by_quadrature():
    """x Phi(x) with Phi integrated numerically from the normal density."""
    for x in (-2.5, -0.7, 0.0, 0.3, 1.9):
        t = np.linspace(-12.0, x, 200001)
        phi = np.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)
        cdf = np.trapezoid(phi, t)
        assert M.gelu(np.array([x]))[0] == pytest.approx(x * cdf, abs=1e-9)
        h = 1e-5
        fd = (M.gelu(np.array([x + h]))[0] - M.gelu(np.array([x - h]))[0]) / (2 * h)
        assert M.gelu_grad(np.array([x]))[0] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_gradient_by_finite_differences():
    th = _theta()
    rng = np.random.default_rng(1)
    x = rng.standard_normal((40, 4))
    t = rng.standard_normal(40)
    _, g = M.loss_and_grad(th, x, t)
    for i in rng.choice(M.N_PARAMS, 60, replace=False):
        e = np.zeros(M.N_PARAMS)
        e[i] = 1e-5
        fd = (M.loss_and_grad(th + e, x, t)[0] - M.loss_and_grad(th - e, x, t)[0]) / 2e-5
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_adam_first_step_closed_form():
    """With zero moments the first bias-corrected step is lr * g / (|g| + eps)."""
    g = np.array([0.5, -3.0, 1e-3])
    th, m, v = M.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    th2, _, _ = M.adam_step(th, m, v, g, 2, 0.01)
    np.testing.assert_allclose(th2 - th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_bf16_rounding_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -(1 + 2 ** -7 + 2 ** -8), 65504.0], dtype=np.float32)
    np.testing.assert_array_equal(M.bf16_round(x), [1.0, 1.0, 1 + 2 ** -7, -(1 + 2 ** -6), 65536.0])


def test_untrained_network_is_the_plain_scaling():
    th = M.init_params(np.random.default_rng(0))
    x = np.random.default_rng(2).standard_normal((10, 4))
    assert np.all(M.forward(th, x) == 0.0)


def test_scalings_on_a_known_case():
    kin = np.array([0.1, 0.5, 2.0, 8.0])
    b = np.array([1.0, 1.0j, 0.0, 0.0])
    # e_prec = 1.35 * (0.1 + 0.5) / 2 = 0.405
    np.testing.assert_allclose(M.plain_scaling(kin, b), [1.0, 0.405 / 0.5, 0.405 / 2.0, 0.405 / 8.0])
    hd = M.h_diag(kin, -0.2, np.array([[1.0, 2.0, 0.0, 1j]]), np.array([0.5]))
    np.testing.assert_allclose(hd, [0.4, 2.3, 1.8, 8.3])
    j = M.jacobi_scaling(hd, 0.4 + 0.01j, 0.1)
    np.testing.assert_allclose(j, [10.0, 1 / abs(1.9 - 0.01j), 1 / abs(1.4 - 0.01j), 1 / abs(7.9 - 0.01j)])
    np.testing.assert_allclose(M.targets(np.array([1.0, 0.01]), np.array([math.e, 1.0])), [1.0, 3.0])


def test_features_on_a_hand_worked_row():
    """The feature normalisation: T_G / (E_cut / 2) is 1 on the sphere surface |k+G|^2 = E_cut[Ry]
    (T_G = |k+G|^2 / 2 Ha), the top of the 60 eV frequency window maps to 1 (60 eV = 2.20496 Ha),
    and e_ref, <V_loc> pass through in Ha.  A Ry/Ha slip in either scale fails this."""
    ha_ev = 27.211386245988
    f = M.features(np.array([0.0, 2.5, 5.0]), 10.0, 60.0 / ha_ev, -0.3, -0.7)
    np.testing.assert_allclose(f[:, 0], [0.0, 0.5, 1.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(f[:, 1], 1.0, rtol=0, atol=3e-5)
    assert np.all(f[:, 2] == -0.3) and np.all(f[:, 3] == -0.7)
    # on a real basis every kinetic feature lies in (0, 1], the largest close to 1
    import instances as I
    inst = I.config1()
    from instances.generate import sphere
    mil, n2 = sphere(inst.a, inst.kpoints[0].kq_frac, inst.ecut_ry)
    k = M.features(0.5 * n2, inst.ecut_ry, 0.0, 0.0, 0.0)[:, 0]
    assert k.max() <= 1.0 and k.max() > 0.9
