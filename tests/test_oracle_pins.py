"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle by a route other than its own formula: integer lattice
arithmetic, real-space quadrature, invariances, the sum over states of a full
diagonalisation, and independently built fixtures.  The mutation tests at the end plant
a plausible mistake in the oracle (on the CPU) and show that a pin catches it.
"""
import math

import numpy as np
import pytest

import instances as I
import oracle as O
from instances.generate import cubic8_cell, fcc_cell


# ------------------------------------------------------------------- Eq. 1: the basis

def _integer_sphere_fcc(alat, ecut_ry):
    """fcc: B rows are (2 pi / a)(-1,1,1), (1,-1,1), (1,1,-1); |m.B|^2 = (2pi/a)^2 * integer."""
    lim = int(math.sqrt(ecut_ry) * alat / (2 * math.pi)) + 2
    s = (alat / (2 * math.pi)) ** 2 * ecut_ry
    out = []
    for m1 in range(-lim, lim + 1):
        for m2 in range(-lim, lim + 1):
            for m3 in range(-lim, lim + 1):
                q = (-m1 + m2 + m3) ** 2 + (m1 - m2 + m3) ** 2 + (m1 + m2 - m3) ** 2
                if q <= s:
                    out.append((m1, m2, m3))
    return out


def _integer_sphere_cubic(alat, ecut_ry):
    lim = int(math.sqrt(ecut_ry) * alat / (2 * math.pi)) + 1
    s = (alat / (2 * math.pi)) ** 2 * ecut_ry
    return [(a, b, c) for a in range(-lim, lim + 1) for b in range(-lim, lim + 1)
            for c in range(-lim, lim + 1) if a * a + b * b + c * c <= s]


@pytest.mark.parametrize("cell,ecut,count", [("fcc", 10.0, 137), ("cubic", 20.0, 1647)])
def test_sphere_matches_integer_enumeration(cell, ecut, count):
    if cell == "fcc":
        a, _ = fcc_cell(10.26)
        ref = _integer_sphere_fcc(10.26, ecut)
    else:
        a, _ = cubic8_cell(10.26)
        ref = _integer_sphere_cubic(10.26, ecut)
    mil, kin = O.gsphere(a, (0, 0, 0), ecut)
    assert len(mil) == count == len(ref)
    assert [tuple(m) for m in mil] == sorted(ref)           # canonical = lexicographic
    # kinetic = |G|^2 / 2 from the integer metric
    if cell == "cubic":
        q = (mil.astype(np.int64) ** 2).sum(1)
        np.testing.assert_allclose(kin, 0.5 * (2 * math.pi / 10.26) ** 2 * q, rtol=1e-14)


def test_sphere_count_large_cell_and_continuum_limit():
    a = np.eye(3) * 20.52
    mil, _ = O.gsphere(a, (0, 0, 0), 25.0)
    assert len(mil) == 18277
    vol = 20.52 ** 3
    approx = vol * 25.0 ** 1.5 / (6 * math.pi ** 2)      # Omega E^{3/2} / (6 pi^2)
    assert abs(len(mil) - approx) / approx < 0.01


def test_sphere_reciprocal_translation():
    """k -> k + (1,0,0) relabels G -> G - b1: same set shifted by one Miller unit."""
    a, _ = cubic8_cell(10.26)
    k = np.array([0.13, -0.21, 0.34])
    m0, kin0 = O.gsphere(a, k, 20.0)
    m1, kin1 = O.gsphere(a, k + np.array([1.0, 0, 0]), 20.0)
    assert sorted(map(tuple, m0)) == sorted(tuple(m + np.array([1, 0, 0])) for m in m1)
    assert np.allclose(np.sort(kin0), np.sort(kin1), rtol=1e-13)


def test_sphere_agrees_with_generator_order():
    """The generator's basis (its own enumeration) equals the oracle's, in order."""
    inst = I.config1()
    kp = inst.kpoints[0]
    m, _ = O.gsphere(inst.a, kp.kq_frac, inst.ecut_ry)
    assert np.array_equal(m, kp.miller_kq)


def test_box_map_values_and_injective():
    mil = np.array([[-1, 0, 2], [0, 0, 0], [3, -2, -1]], dtype=np.int32)
    idx = O.box_map(mil, (8, 9, 10))
    assert idx.tolist() == [(7 * 9 + 0) * 10 + 2, 0, (3 * 9 + 7) * 10 + 9]
    a, _ = cubic8_cell(10.26)
    mil, _ = O.gsphere(a, (0.1, 0.2, -0.3), 20.0)
    assert len(set(O.box_map(mil, (36, 36, 36)).tolist())) == len(mil)


def test_min_box_values():
    a, _ = fcc_cell(10.26)
    assert O.min_box(a, 10.0) == (15, 15, 15)
    a, _ = cubic8_cell(10.26)
    assert O.min_box(a, 20.0) == (29, 29, 29)


# ----------------------------------------------------------- Sec. 2.1: the Hamiltonian

def _cell_inputs(inst, vloc=None, d=None):
    return (inst.a, inst.tau, inst.ecut_ry, None, inst.fft_dims,
            inst.vloc_r if vloc is None else vloc, inst.kb_atom, inst.kb_width,
            inst.kb_d if d is None else d)


@pytest.fixture(scope="module")
def tiny():
    return I.tiny_fcc(ecut_ry=4.0, dims=(12, 12, 12), n_occ=4, n_pert=3, n_omega=5)


def test_empty_lattice(tiny):
    """V = 0, D = 0: eigenvalues are exactly |k+G|^2 / 2 (free electrons)."""
    k = np.array([0.1, -0.2, 0.05])
    zeros = np.zeros(tiny.fft_dims)
    h, mil, _ = O.dense_h(tiny.a, tiny.tau, tiny.ecut_ry, k, tiny.fft_dims, zeros,
                          tiny.kb_atom, tiny.kb_width, np.zeros(2))
    w = np.linalg.eigvalsh(h)
    alat = 10.26
    # fcc integer metric with fractional k: |(m+k).B|^2 = (2pi/a)^2 sum of squares
    mk = mil + k
    q = (-mk[:, 0] + mk[:, 1] + mk[:, 2]) ** 2 + (mk[:, 0] - mk[:, 1] + mk[:, 2]) ** 2 \
        + (mk[:, 0] + mk[:, 1] - mk[:, 2]) ** 2
    ref = np.sort(0.5 * (2 * math.pi / alat) ** 2 * q)
    np.testing.assert_allclose(w, ref, rtol=1e-12, atol=1e-13)


def test_constant_potential_shift(tiny):
    k = np.array([0.1, 0.0, 0.0])
    v0 = -0.37
    h0, _, _ = O.dense_h(tiny.a, tiny.tau, tiny.ecut_ry, k, tiny.fft_dims, tiny.vloc_r,
                         tiny.kb_atom, tiny.kb_width, tiny.kb_d)
    h1, _, _ = O.dense_h(tiny.a, tiny.tau, tiny.ecut_ry, k, tiny.fft_dims, tiny.vloc_r + v0,
                         tiny.kb_atom, tiny.kb_width, tiny.kb_d)
    np.testing.assert_allclose(np.linalg.eigvalsh(h1), np.linalg.eigvalsh(h0) + v0, atol=1e-12)


def test_plane_wave_potential_index_direction(tiny):
    """V(r) = 2 sin(G0.r) has V(G0) = -i, V(-G0) = +i; H[G,G'] = V(G - G')."""
    n = tiny.fft_dims
    j = np.stack(np.meshgrid(*[np.arange(x) for x in n], indexing="ij"), -1)
    m0 = np.array([1, 0, -1])
    phase = 2 * math.pi * (j * (m0 / np.array(n))).sum(-1)           # G0 . r_j
    v = 2 * np.sin(phase)
    h, mil, kin = O.dense_h(tiny.a, tiny.tau, tiny.ecut_ry, np.zeros(3), n, v,
                            tiny.kb_atom, tiny.kb_width, np.zeros(2))
    h = h - np.diag(kin)
    lookup = {tuple(m): i for i, m in enumerate(mil)}
    checked = 0
    for i, m in enumerate(mil):
        jj = lookup.get(tuple(m - m0))
        if jj is not None:
            assert abs(h[i, jj] - (-1j)) < 1e-13          # m_G - m_G' = m0
            assert abs(h[jj, i] - (1j)) < 1e-13           # m_G - m_G' = -m0
            checked += 1
    assert checked > 5
    assert np.abs(h).sum() == pytest.approx(2 * checked, rel=1e-12)


def test_gaussian_potential_normalisation_by_quadrature():
    """Cell average of the sampled potential = (1/Omega) * sum_atoms of the Gaussian's
    integral, computed here by brute-force quadrature on a fine real-space grid."""
    inst = I.tiny_fcc(ecut_ry=4.0, dims=(12, 12, 12))
    hgrid = 0.06
    x = np.arange(-7.0, 7.0 + 1e-9, hgrid)
    g1 = np.exp(-x ** 2 / (2 * 0.9 ** 2))
    integral = -4.0 * (g1.sum() * hgrid) ** 3
    vhat0 = O.vloc_hat(inst.vloc_r)[0, 0, 0].real
    assert vhat0 == pytest.approx(2 * integral / inst.volume, rel=1e-10)


def test_kb_projector_by_quadrature(tiny):
    """<k+G|beta> = Omega^-1/2 int beta(r - tau) exp(-i(k+G).r) d^3r, brute-force quadrature."""
    k = np.array([0.1, -0.05, 0.2])
    mil, _ = O.gsphere(tiny.a, k, tiny.ecut_ry)
    beta = O.kb_beta(tiny.a, tiny.tau, k, mil, tiny.kb_atom, tiny.kb_width)
    b = O.reciprocal(tiny.a)
    w = 0.9
    hgrid = 0.09
    x = np.arange(-6.3, 6.3 + 1e-9, hgrid)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    g = (math.pi * w * w) ** -0.75 * np.exp(-(X * X + Y * Y + Z * Z) / (2 * w * w))
    for gi in [0, 5, len(mil) - 1]:
        kg = (mil[gi] + k) @ b
        for ia in range(2):
            t = tiny.tau[ia]
            ph = np.exp(-1j * (kg[0] * (X + t[0]) + kg[1] * (Y + t[1]) + kg[2] * (Z + t[2])))
            val = (g * ph).sum() * hgrid ** 3 / math.sqrt(tiny.volume)
            assert abs(val - beta[ia, gi]) < 1e-9 * abs(val) + 1e-12


def test_hamiltonian_hermitian(tiny):
    h, _, _ = O.dense_h_inst(tiny, tiny.kpoints[0].kq_frac)
    assert np.abs(h - h.conj().T).max() < 1e-15


def test_translation_invariance():
    """Moving every atom by t multiplies H by diagonal phases: H' = D H D^H, D = diag(e^{-iG.t})."""
    base = I.tiny_fcc(ecut_ry=4.0, dims=(12, 12, 12))
    t = np.array([0.31, -0.17, 0.52])
    moved = I.make_instance("moved", 0, base.a, base.tau + t, base.ecut_ry, base.fft_dims, 4,
                            [], base.gp_miller, base.omega, base.eta)
    k = np.array([0.05, 0.1, -0.15])
    h0, mil, _ = O.dense_h_inst(base, k)
    h1, _, _ = O.dense_h_inst(moved, k)
    gc = mil @ O.reciprocal(base.a)
    d = np.exp(-1j * (gc @ t))
    np.testing.assert_allclose(h1, d[:, None] * h0 * d.conj()[None, :], atol=1e-12)
    np.testing.assert_allclose(np.linalg.eigvalsh(h1), np.linalg.eigvalsh(h0), atol=1e-12)


def test_generator_ground_state_is_eigenbasis_of_oracle_h():
    """The generator diagonalises H built from closed-form V(G); the oracle builds H from the
    DFT of the sampled box.  Band-limited + alias-free box => the same operator."""
    inst = I.config1()
    kp = inst.kpoints[0]
    for kf, psi, eps in [(kp.k_frac, kp.psi_k, kp.eps_k), (kp.kq_frac, kp.psi_kq, kp.eps_kq)]:
        h, _, _ = O.dense_h_inst(inst, kf)
        res = h @ psi.T - psi.T * eps[None, :]
        assert np.abs(res).max() < 1e-10
        assert np.abs(psi.conj() @ psi.T - np.eye(len(eps))).max() < 1e-12


def test_fft_apply_equals_dense(tiny):
    """Sec. 2.1's split (kinetic/non-local in G space, V_loc via FFT) equals dense H x:
    the convolution theorem on the box."""
    k = tiny.kpoints[0].kq_frac
    h, mil, _ = O.dense_h_inst(tiny, k)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, len(mil))) + 1j * rng.standard_normal((3, len(mil)))
    y = O.apply_h_fft(tiny.a, tiny.tau, tiny.ecut_ry, k, tiny.fft_dims, tiny.vloc_r,
                      tiny.kb_atom, tiny.kb_width, tiny.kb_d, x)
    np.testing.assert_allclose(y, x @ h.T, atol=1e-12)


def test_alias_negative_control():
    """A box below 2 m_rho + 1 cannot hold the band-limited potential: the generator refuses,
    and folding the coefficients into it changes the matrix elements."""
    a, tau = fcc_cell(10.26)
    with pytest.raises(ValueError):
        I.generate.vloc_box(a, tau, 10.0, (12, 12, 12))
    good = I.generate.vloc_box(a, tau, 4.0, (12, 12, 12))
    # same potential folded into a 6^3 box (below 2 m_rho + 1 for 4 Ry)
    mil, _ = I.generate.sphere(a, (0, 0, 0), 16.0, check_margin=False)
    vg = I.generate.vloc_coeffs(a, tau, mil)
    box = np.zeros((6, 6, 6), complex)
    np.add.at(box, tuple(np.mod(mil[:, i], 6) for i in range(3)), vg)
    small = (np.fft.ifftn(box) * 216).real
    vh_good = O.vloc_hat(good)
    vh_small = O.vloc_hat(small)
    # coefficient at Miller (3,0,0) aliases with (-3,0,0)
    assert abs(vh_small[3, 0, 0] - vh_good[3, 0, 0]) > 1e-6


# ------------------------------------------------------------------ Eq. 8: the RHS

def test_rhs_gather_matches_real_space_product(tiny):
    """dV psi_v with dV = exp(i(q+G_p).r) computed on a real-space grid and projected back
    onto the k+q plane waves equals the coefficient gather."""
    kp = tiny.kpoints[0]
    rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, tiny.gp_miller)
    n = (24, 24, 24)
    ntot = np.prod(n)
    j = np.stack(np.meshgrid(*[np.arange(x) for x in n], indexing="ij"), -1).reshape(-1, 3)
    frac_r = j / np.array(n)
    b = O.reciprocal(tiny.a)
    for p, gp in enumerate(tiny.gp_miller):
        for v in range(tiny.n_occ):
            # psi_{v,k}(r) = sum_G c_G exp(i (k+G).r);  r.b_i = 2 pi frac_i
            phase_k = np.exp(2j * math.pi * frac_r @ (kp.miller_k + kp.k_frac).T)
            psi_r = phase_k @ kp.psi_k[v]
            dv = np.exp(2j * math.pi * frac_r @ (kp.kq_frac - kp.k_frac + gp))
            prod = psi_r * dv
            phase_kq = np.exp(-2j * math.pi * frac_r @ (kp.miller_kq + kp.kq_frac).T)
            coef = prod @ phase_kq / ntot
            np.testing.assert_allclose(coef, rhs[v * tiny.n_pert + p], atol=1e-12)
    assert b.shape == (3, 3)


# ------------------------------------------------------------- Eq. 6-7: the solution

@pytest.fixture(scope="module")
def tiny_gapped():
    """A tiny basis whose occupied/unoccupied cut falls in a gap, with the oracle's own
    eigenvectors as the occupied manifold (so P_c is the spectral projector)."""
    inst = I.tiny_fcc(ecut_ry=5.0, dims=(12, 12, 12), n_occ=2, n_pert=3, n_omega=6)
    kp = inst.kpoints[0]
    h, mil, _ = O.dense_h_inst(inst, kp.kq_frac)
    w, v = np.linalg.eigh(h)
    assert w[2] - w[1] > 1e-3
    return inst, h, v[:, :2].T.copy(), w


def test_sternheimer_equals_sum_over_states(tiny_gapped):
    inst, h, psi_v, w = tiny_gapped
    kp = inst.kpoints[0]
    rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k[:2], inst.gp_miller)
    e_ref = np.repeat(kp.eps_k[:2], inst.n_pert)
    x = O.solve_shifted(h, psi_v, rhs, e_ref, inst.omega, inst.eta)
    sos, _ = O.sum_over_states(h, 2, rhs, e_ref, inst.omega, inst.eta)
    err = np.abs(x - sos).max() / np.abs(sos).max()
    assert err < 1e-11


def test_solution_invariants(tiny_gapped):
    inst, h, psi_v, w = tiny_gapped
    kp = inst.kpoints[0]
    rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k[:2], inst.gp_miller)
    e_ref = np.repeat(kp.eps_k[:2], inst.n_pert)
    x = O.solve_shifted(h, psi_v, rhs, e_ref, inst.omega, inst.eta)
    # orthogonal to the occupied manifold
    assert np.abs(np.einsum("vg,rjg->rjv", psi_v.conj(), x)).max() < 1e-12
    # linear in the right-hand side
    x2 = O.solve_shifted(h, psi_v, 2.5j * rhs[:2] - rhs[1:3], e_ref[:2], inst.omega, inst.eta)
    np.testing.assert_allclose(x2, 2.5j * x[:2] - x[1:3], atol=1e-11)
    # adjoint relation: (A(z*))^-1 = (A(z)^-1)^H   <=>   <y, A(z)^-1 u> = <A(z*)^-1 y, u>
    z = e_ref[0] + inst.omega[3] + 1j * inst.eta
    a = O.shifted_operator(h, psi_v, z)
    ac = O.shifted_operator(h, psi_v, np.conj(z))
    rng = np.random.default_rng(0)
    u = rng.standard_normal(len(h)) + 1j * rng.standard_normal(len(h))
    y = rng.standard_normal(len(h)) + 1j * rng.standard_normal(len(h))
    lhs = np.vdot(y, np.linalg.solve(a, u))
    rhs_ = np.vdot(np.linalg.solve(ac, y), u)
    assert abs(lhs - rhs_) < 1e-10 * abs(lhs)


def test_residual_and_certificate_bound(tiny_gapped):
    inst, h, psi_v, w = tiny_gapped
    kp = inst.kpoints[0]
    rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k[:2], inst.gp_miller)
    e_ref = np.repeat(kp.eps_k[:2], inst.n_pert)
    x = O.solve_shifted(h, psi_v, rhs, e_ref, inst.omega, inst.eta)
    rel, cert = O.residual(h, psi_v, rhs, e_ref, inst.omega, inst.eta, x)
    assert rel.max() < 1e-12
    rng = np.random.default_rng(1)
    noise = 1e-6 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
    noise = noise - np.einsum("rjv,vg->rjg", np.einsum("vg,rjg->rjv", psi_v.conj(), noise), psi_v)
    xp = x + noise
    rel2, cert2 = O.residual(h, psi_v, rhs, e_ref, inst.omega, inst.eta, xp)
    err = np.linalg.norm(xp - x, axis=2) / np.linalg.norm(xp, axis=2)
    assert np.all(err <= cert2 * (1 + 1e-9))


def test_config1_ground_state_gap_recorded():
    """Config-1 cut (4 bands) falls inside the p-like triplet of the synthetic potential at
    Gamma; the generator reports it (parity is unaffected: psi_v is an input)."""
    inst = I.config1()
    assert inst.kpoints[0].gap_k < 1e-6


# --------------------------------------------------------------------- mutation tests

def test_mutation_vhat_conjugate_is_caught(tiny, monkeypatch):
    """Plant V(G'-G) for V(G-G') (a transposed operand): the index-direction pin fails."""
    orig = O.sgw_oracle.vloc_hat
    monkeypatch.setattr(O.sgw_oracle, "vloc_hat", lambda v: np.conj(orig(v)))
    with pytest.raises(AssertionError):
        test_plane_wave_potential_index_direction(tiny)


def test_mutation_kb_phase_sign_is_caught(tiny, monkeypatch):
    """Plant exp(+i(k+G).tau) in the projector: the quadrature pin fails."""
    orig = O.sgw_oracle.kb_beta

    def bad(a, tau, k, mil, atom, width):
        return orig(a, -np.asarray(tau), k, mil, atom, width)
    monkeypatch.setattr(O.sgw_oracle, "kb_beta", bad)
    monkeypatch.setattr(O, "kb_beta", bad)
    with pytest.raises(AssertionError):
        test_kb_projector_by_quadrature(tiny)


def test_mutation_dropped_projector_is_caught(tiny_gapped, monkeypatch):
    """Plant b = -rhs (P_c dropped from the right-hand side): the sum-over-states pin fails."""
    monkeypatch.setattr(O.sgw_oracle, "project_c", lambda psi, x: np.atleast_2d(x))
    with pytest.raises(AssertionError):
        test_solution_invariants(tiny_gapped)
