"""Parity of the Green's-function columns (Eq. 2-3) computed through the C ABI
(sgw_solve_green) with the FP64 oracle's dense LU, on time-ordered shifts
z_j = omega_j + i eta sgn(omega_j - mu).  Per (column, shift) pair the relative error must be
<= 1e-8 and the true residual <= 1e-10; the certificate |r| / (|Im z| |g|) bounds the error."""
import numpy as np
import pytest

import instances as I
import oracle as O

pytestmark = pytest.mark.gpu

HA_EV = 27.211386245988
TOL = 1e-10
TOL_G = 1e-8


@pytest.fixture(scope="module")
def sgw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    import paper_1812_03717_gb300 as P
    from paper_1812_03717_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    return P


def _shifts(inst, ik, nz, span_ev=25.0):
    kp = inst.kpoints[ik]
    mu = float(kp.eps_kq[-1]) + 0.5 * float(kp.gap_kq)     # inside the gap above the occupied states
    omega = mu + np.linspace(-span_ev, span_ev, nz) / HA_EV
    return O.time_ordered_shifts(omega, mu, inst.eta), mu


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.fixture(scope="module")
def cfg1():
    return I.config1()


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_green_config1_all_columns(sgw, cfg1, precision):
    """Every column of G(z) on the config-1 basis (137 plane waves), 16 shifts on both sides
    of the chemical potential, against one dense LU per shift."""
    kp = cfg1.kpoints[0]
    s = sgw.System.from_instance(cfg1, kp.kq_frac)     # no occupied states: Eq. 3 has no projector
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    z, _ = _shifts(cfg1, 0, 16)
    assert np.any(z.imag < 0) and np.any(z.imag > 0)
    cols = np.arange(s.n_pw)
    g, rep, ok = s.solve_green(cols, z, tol=TOL, precision=precision)
    assert ok, np.unique(rep["status"], return_counts=True)
    assert rep["rel_res"].max() <= TOL
    ref = O.green_columns(h, cols, z)
    err = _relerr(g, ref)
    assert err.max() <= TOL_G, err.max()
    assert np.all(err <= rep["cert"] * (1 + 1e-6) + 1e-13)
    # the oracle's own residual of the returned columns agrees with the library's
    rel, _ = O.green_residual(h, cols[:5], z, g[:5])
    assert rel.max() <= 2 * TOL


def test_green_config2_sampled_columns(sgw):
    """Sampled columns of G(z) on the 1647-plane-wave basis (k-point 0 of the 8-atom cell)
    with 64 time-ordered shifts; eight shifts are checked against the dense LU."""
    inst = I.config2(k_subset=[0])
    kp = inst.kpoints[0]
    s = sgw.System.from_instance(inst, kp.kq_frac)
    z, _ = _shifts(inst, 0, 64)
    rng = np.random.default_rng(5)
    cols = np.sort(rng.choice(s.n_pw, 6, replace=False))
    cols[0] = 0
    g, rep, ok = s.solve_green(cols, z, tol=TOL, precision="df32")
    assert ok
    assert rep["rel_res"].max() <= TOL
    h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
    js = np.array([0, 9, 21, 31, 32, 44, 55, 63])
    ref = O.green_columns(h, cols, z[js])
    err = _relerr(g[:, js], ref)
    assert err.max() <= TOL_G, err.max()


def test_green_matches_projected_sternheimer(sgw, cfg1):
    """G(z) P_c rhs equals the Sternheimer solution of sgw_solve_shifted when psi_v are
    eigenvectors (both computed on the GPU; an identity of the mathematics)."""
    kp = cfg1.kpoints[0]
    s = sgw.System.from_instance(cfg1, kp.kq_frac)
    sk = sgw.System.from_instance(cfg1, kp.k_frac)
    s.set_occupied(kp.psi_kq, kp.eps_kq)
    rhs = s.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[:3]
    e = float(kp.eps_k[0])
    om = cfg1.omega[[1, 7, 12]]
    x, rep, ok = s.solve_shifted(rhs, np.full(3, e), om, cfg1.eta, tol=TOL)
    assert ok
    g, rep2, ok2 = s.solve_green(np.arange(s.n_pw), e + om + 1j * cfg1.eta, tol=TOL)
    assert ok2
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)[:3]
    assert np.array_equal(rhs, rref)
    pr = O.project_c(kp.psi_kq, rref)
    for j in range(3):
        y = (g[:, j, :].T @ pr.T).T
        assert _relerr(x[:, j], y).max() <= 1e-8


def test_green_device_buffers(sgw, cfg1):
    import torch
    kp = cfg1.kpoints[0]
    s = sgw.System.from_instance(cfg1, kp.kq_frac)
    z, _ = _shifts(cfg1, 0, 8)
    cols = np.array([3, 17, 40])
    g_host, _, _ = s.solve_green(cols, z, tol=TOL)
    g_dev, rep, ok = s.solve_green(cols, z, tol=TOL, device="cuda")
    assert ok and isinstance(g_dev, torch.Tensor) and g_dev.is_cuda
    np.testing.assert_allclose(g_dev.cpu().numpy(), g_host, rtol=0, atol=1e-12 * np.abs(g_host).max())


def test_green_edge_cases(sgw, cfg1):
    kp = cfg1.kpoints[0]
    s = sgw.System.from_instance(cfg1, kp.kq_frac)
    z = np.array([0.1 + 0.01j, 0.2 - 0.01j])
    g, rep, ok = s.solve_green(np.zeros(0, dtype=np.int32), z)
    assert ok and g.shape == (0, 2, s.n_pw)
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        s.solve_green([s.n_pw], z)
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        s.solve_green([-1], z)
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        s.solve_green([0], [0.3 + 0.0j])
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        s.solve_green([0], [np.nan + 0.1j])
    with pytest.raises(sgw.SgwError, match="EUNSUPPORTED"):
        s.solve_green([0], np.full(513, 0.1 + 0.01j))
    # a single shift and a single column, far from the spectrum: G ~ 1/z e
    g, rep, ok = s.solve_green([5], [200.0 + 50.0j], tol=1e-12)
    assert ok
    assert abs(g[0, 0, 5] * (200.0 + 50.0j) - 1.0) < 0.1
