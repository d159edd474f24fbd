"""Pins of the Green's-function oracle (Eq. 2-3) against what the mathematics fixes: the
spectral representation, the free-electron closed form, the large-|z| expansion, the adjoint
relation, the sign of the spectral function, the Sternheimer solution it must reproduce, and
the residual certificate.  CPU only."""
import math

import numpy as np
import pytest

import instances as I
import oracle as O


@pytest.fixture(scope="module")
def tiny():
    inst = I.tiny_fcc(ecut_ry=5.0, dims=(12, 12, 12), n_occ=2, n_pert=3, n_omega=6)
    kp = inst.kpoints[0]
    h, mil, kin = O.dense_h_inst(inst, kp.kq_frac)
    w = np.linalg.eigvalsh(h)
    mu = 0.5 * (w[1] + w[2])
    omega = mu + np.linspace(-1.1, 1.1, 8)
    z = O.time_ordered_shifts(omega, mu, 0.02)
    return inst, h, kin, z, mu


def test_time_ordered_shift_signs():
    z = O.time_ordered_shifts([-1.0, 0.2, 0.3, 2.0], 0.25, 0.1)
    np.testing.assert_array_equal(z.imag, [-0.1, -0.1, 0.1, 0.1])
    np.testing.assert_array_equal(z.real, [-1.0, 0.2, 0.3, 2.0])
    with pytest.raises(ValueError):
        O.time_ordered_shifts([0.25], 0.25, 0.1)


def test_green_equals_spectral_representation(tiny):
    inst, h, kin, z, mu = tiny
    cols = np.arange(h.shape[0])
    g = O.green_columns(h, cols, z)
    s = O.green_sum_over_states(h, cols, z)
    assert np.abs(g - s).max() <= 1e-11 * np.abs(s).max()


def test_free_electron_closed_form(tiny):
    """V = 0, D = 0: H is diagonal and G_{G G'}(z) = delta_{G G'} / (z - |k+G|^2 / 2)."""
    inst, _, _, z, _ = tiny
    k = np.array([0.13, -0.07, 0.21])
    h, mil, kin = O.dense_h(inst.a, inst.tau, inst.ecut_ry, k, inst.fft_dims, np.zeros(inst.fft_dims),
                            inst.kb_atom, inst.kb_width, np.zeros(len(inst.kb_d)))
    cols = np.array([0, 3, len(kin) - 1])
    g = O.green_columns(h, cols, z)
    for c, gp in enumerate(cols):
        for j, zj in enumerate(z):
            ref = np.zeros(len(kin), dtype=complex)
            ref[gp] = 1.0 / (zj - kin[gp])
            np.testing.assert_allclose(g[c, j], ref, rtol=0, atol=1e-14 * abs(ref[gp]))


def test_large_z_expansion(tiny):
    """G(z) = (z - H)^-1 = z^-1 + H z^-2 + H^2 z^-3 + ...: fixes the sign of the right-hand
    side and of the operator."""
    inst, h, _, _, _ = tiny
    n = h.shape[0]
    cols = np.arange(n)
    hn = np.linalg.norm(h, 2)
    for zj in (400.0 + 300.0j, -500.0 - 100.0j):
        g = O.green_columns(h, cols, [zj])[:, 0, :].T          # G[:, c] as columns
        approx = np.eye(n) / zj + h / zj ** 2 + h @ h / zj ** 3
        assert np.linalg.norm(g - approx, 2) <= 2.0 * hn ** 3 / abs(zj) ** 4


def test_adjoint_and_spectral_sign(tiny):
    """G(z*) = G(z)^H, and -Im G_GG(z) / pi > 0 for Im z > 0 (a positive spectral weight)."""
    inst, h, _, z, _ = tiny
    n = h.shape[0]
    cols = np.arange(n)
    gz = O.green_columns(h, cols, z)
    gc = O.green_columns(h, cols, np.conj(z))
    for j in range(len(z)):
        a = gz[:, j, :].T
        b = gc[:, j, :].T
        np.testing.assert_allclose(b, a.conj().T, atol=1e-12 * np.abs(a).max())
        d = np.diagonal(a)
        assert np.all(np.sign(z[j].imag) * d.imag < 0)


def test_projected_green_reproduces_sternheimer(tiny):
    """With psi_v eigenvectors and b = -P_c rhs in range(P_c):
    (P_c H P_c - z)^-1 b = (H - z)^-1 b, so dpsi = G(z) P_c rhs."""
    inst, h, _, _, _ = tiny
    w, v = np.linalg.eigh(h)
    psi_v = v[:, :2].T.copy()
    kp = inst.kpoints[0]
    rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k[:2], inst.gp_miller)[:3]
    e_ref = np.full(3, kp.eps_k[0])
    x = O.solve_shifted(h, psi_v, rhs, e_ref, inst.omega[:3], inst.eta)
    pr = O.project_c(psi_v, rhs)
    cols = np.arange(h.shape[0])
    for j, om in enumerate(inst.omega[:3]):
        g = O.green_columns(h, cols, [e_ref[0] + om + 1j * inst.eta])[:, 0, :].T
        np.testing.assert_allclose(x[:, j, :], (g @ pr.T).T, atol=1e-11 * np.abs(x).max())


def test_green_residual_and_certificate(tiny):
    inst, h, _, z, _ = tiny
    cols = np.array([0, 5, 9])
    g = O.green_columns(h, cols, z)
    rel, cert = O.green_residual(h, cols, z, g)
    assert rel.max() < 1e-12
    rng = np.random.default_rng(2)
    gp = g + 1e-6 * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    _, cert2 = O.green_residual(h, cols, z, gp)
    err = np.linalg.norm(gp - g, axis=2) / np.linalg.norm(gp, axis=2)
    assert np.all(err <= cert2 * (1 + 1e-9))


def test_mutation_rhs_sign_is_caught(tiny, monkeypatch):
    """Plant +delta for -delta (a flipped sign): the large-z pin fails."""
    orig = O.sgw_oracle.unit_columns
    monkeypatch.setattr(O.sgw_oracle, "unit_columns", lambda n, c: -orig(n, c))
    with pytest.raises(AssertionError):
        test_large_z_expansion(tiny)


def test_mutation_dropped_potential_is_caught(tiny):
    """A Green's function built from the kinetic part alone fails the spectral pin."""
    inst, h, kin, z, _ = tiny
    cols = np.arange(h.shape[0])
    bad = O.green_columns(np.diag(np.diag(h)), cols, z)
    s = O.green_sum_over_states(h, cols, z)
    assert np.abs(bad - s).max() > 1e-3 * np.abs(s).max()
    assert math.isfinite(float(np.abs(bad).max()))
