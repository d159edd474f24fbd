"""Pins of the density-response oracle (Eq. 5): the paper's real-space route against the sum
over the eigenstates of H_{k+q}, the +-omega symmetry, the free-electron closed form, and a
planted mistake.  CPU only."""
import numpy as np
import pytest

import instances as I
import oracle as O


@pytest.fixture(scope="module")
def gapped():
    """Tiny fcc basis; the occupied states at k and k+q are the oracle's own eigenvectors, so
    P_c is the spectral projector of H_{k+q} and the sum over states is exact."""
    inst = I.tiny_fcc(ecut_ry=5.0, dims=(16, 16, 16), n_occ=2, n_pert=4, n_omega=5)
    kp = inst.kpoints[0]
    hk, mk, _ = O.dense_h_inst(inst, kp.k_frac)
    hq, mq, _ = O.dense_h_inst(inst, kp.kq_frac)
    wk, vk = np.linalg.eigh(hk)
    wq, vq = np.linalg.eigh(hq)
    assert wq[2] - wq[1] > 1e-3
    return inst, hq, mk, mq, vk[:, :2].T.copy(), wk[:2], vq[:, :2].T.copy()


def test_density_response_equals_sum_over_states(gapped):
    inst, hq, mk, mq, psi_k, eps_k, psi_q = gapped
    dn = O.density_response(hq, psi_q, psi_k, mk, mq, eps_k, inst.gp_miller, inst.omega, inst.eta,
                            inst.fft_dims, 0.5)
    sos = O.density_response_sos(hq, 2, psi_k, mk, mq, eps_k, inst.gp_miller, inst.omega, inst.eta, 0.5)
    assert np.abs(dn - sos).max() <= 1e-11 * np.abs(sos).max()
    assert np.abs(sos).max() > 1e-3


def test_minus_omega_gives_the_adjoint(gapped):
    """dn(-omega) = dn(omega)^H for real omega: each pair of terms 1/(a + w) + 1/(a - w),
    w = omega + i eta, turns into its complex conjugate when omega changes sign."""
    inst, hq, mk, mq, psi_k, eps_k, psi_q = gapped
    om = np.array([0.05, 0.4, 1.3])
    a = O.density_response(hq, psi_q, psi_k, mk, mq, eps_k, inst.gp_miller, om, inst.eta, inst.fft_dims, 1.0)
    b = O.density_response(hq, psi_q, psi_k, mk, mq, eps_k, inst.gp_miller, -om, inst.eta, inst.fft_dims, 1.0)
    for j in range(len(om)):
        np.testing.assert_allclose(b[:, :, j], a[:, :, j].conj().T, atol=1e-12 * np.abs(a).max())
    # the static response is Hermitian
    s = O.density_response(hq, psi_q, psi_k, mk, mq, eps_k, inst.gp_miller, [0.0], inst.eta, inst.fft_dims, 1.0)
    np.testing.assert_allclose(s[:, :, 0], s[:, :, 0].conj().T, atol=1e-12 * np.abs(s).max())


def test_free_electron_closed_form():
    """V = 0, D = 0, one occupied plane wave (G = 0) at k and at k+q: the response is
    diagonal in (G, G'), zero for G = 0 (projected out), and for G != 0
        dn[G][G] = w [1/(T_k(0) + omega + i eta - T_{k+q}(G)) + 1/(T_k(0) - omega - i eta - T_{k+q}(G))]."""
    inst = I.tiny_fcc(ecut_ry=5.0, dims=(16, 16, 16), n_occ=1, n_pert=4, n_omega=3)
    k = np.array([0.02, -0.01, 0.03])
    q = np.array([0.05, 0.0, 0.02])
    zero_v = np.zeros(inst.fft_dims)
    hk, mk, tk = O.dense_h(inst.a, inst.tau, inst.ecut_ry, k, inst.fft_dims, zero_v, inst.kb_atom,
                           inst.kb_width, np.zeros(len(inst.kb_d)))
    hq, mq, tq = O.dense_h(inst.a, inst.tau, inst.ecut_ry, k + q, inst.fft_dims, zero_v, inst.kb_atom,
                           inst.kb_width, np.zeros(len(inst.kb_d)))
    i0k = int(np.argmin(tk))
    i0q = int(np.argmin(tq))
    assert np.array_equal(mk[i0k], [0, 0, 0]) and np.array_equal(mq[i0q], [0, 0, 0])
    psi_k = np.zeros((1, len(tk)), complex)
    psi_k[0, i0k] = 1.0
    psi_q = np.zeros((1, len(tq)), complex)
    psi_q[0, i0q] = 1.0
    om = np.array([0.0, 0.3, 1.1])
    eta = inst.eta
    dn = O.density_response(hq, psi_q, psi_k, mk, mq, [tk[i0k]], inst.gp_miller, om, eta, inst.fft_dims, 0.5)
    lookup = {tuple(m): i for i, m in enumerate(mq)}
    for p, g in enumerate(inst.gp_miller):
        for p2 in range(len(inst.gp_miller)):
            if p2 != p:
                assert np.abs(dn[p, p2]).max() < 1e-14
        if not np.any(g):
            assert np.abs(dn[p, p]).max() < 1e-14
            continue
        tg = tq[lookup[tuple(g)]]
        w = om + 1j * eta
        ref = 0.5 * (1.0 / (tk[i0k] + w - tg) + 1.0 / (tk[i0k] - w - tg))
        np.testing.assert_allclose(dn[p, p], ref, rtol=1e-12)


def test_mutation_missing_conjugate_is_caught(gapped, monkeypatch):
    """Plant u(r) for conj(u(r)) in the product: the sum-over-states pin fails."""
    psi_k = gapped[4]
    orig = O.sgw_oracle.periodic_on_box

    def bad(coef, miller, dims):
        r = orig(coef, miller, dims)
        return np.conj(r) if np.shares_memory(coef, psi_k) else r    # only the unperturbed u
    monkeypatch.setattr(O.sgw_oracle, "periodic_on_box", bad)
    with pytest.raises(AssertionError):
        test_density_response_equals_sum_over_states(gapped)
