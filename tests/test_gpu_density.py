"""Parity of the density response of Eq. 5 computed through the C ABI
(sgw_density_response: Sternheimer solves at +-(omega + i eta) sharing one Krylov space, then
the reciprocal-space reduction) with the FP64 oracle, which takes the paper's route (dense LU
per shift, real-space product with conj(u_v), box Fourier transform back)."""
import numpy as np
import pytest

import instances as I
import oracle as O
from parity import assert_columns_close

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


@pytest.fixture(scope="module")
def cfg1():
    return I.config1()


def _setup(P, inst, ik=0):
    kp = inst.kpoints[ik]
    skq = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    return kp, skq, sk


def _oracle(inst, kp, v_rows, p_rows, omega, weight):
    h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
    return O.density_response(h, kp.psi_kq, kp.psi_k[v_rows], kp.miller_k, kp.miller_kq, kp.eps_k[v_rows],
                              inst.gp_miller[p_rows], omega, inst.eta, inst.fft_dims, weight)


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_density_config1_full(sgw, cfg1, precision):
    """Every (G, G', omega) of config 1: 4 bands x 8 perturbations x 16 frequencies."""
    kp, skq, sk = _setup(sgw, cfg1)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)
    dn, rep, ok = skq.density_response(rhs, kp.eps_k, cfg1.omega, cfg1.eta, weight=2.0, tol=TOL,
                                       precision=precision)
    assert ok and rep["rel_res"].max() <= TOL
    assert rep["status"].shape == (32, 32)
    ref = _oracle(cfg1, kp, np.arange(4), np.arange(8), cfg1.omega, 2.0)
    assert_columns_close(dn, ref, 1e-8)


def test_density_config2_sampled(sgw):
    """Two bands, four perturbations (G = 0 among them) and four frequencies of the
    1647-plane-wave k-point of config 2."""
    inst = I.config2(k_subset=[0])
    kp, skq, sk = _setup(sgw, inst)
    v_rows = np.array([0, 9])
    p_rows = np.array([0, 3, 17, 31])
    om = inst.omega[[0, 13, 40, 63]]
    gp = inst.gp_miller[p_rows]
    rhs_all = skq.make_rhs(sk, kp.psi_k[v_rows], gp)
    dn, rep, ok = skq.density_response(rhs_all, kp.eps_k[v_rows], om, inst.eta, weight=0.5, tol=TOL,
                                       precision="df32")
    assert ok
    ref = _oracle(inst, kp, v_rows, p_rows, om, 0.5)
    assert_columns_close(dn, ref, 1e-8)


def test_density_minus_omega_adjoint_and_accumulation(sgw, cfg1):
    """dn(-omega) = dn(omega)^H (both from the GPU), and a second call accumulates into a
    device buffer."""
    import torch
    kp, skq, sk = _setup(sgw, cfg1)
    rhs = skq.make_rhs(sk, torch.from_numpy(kp.psi_k).cuda(), cfg1.gp_miller)
    om = cfg1.omega[[2, 9]]
    a, _, ok1 = skq.density_response(rhs, kp.eps_k, om, cfg1.eta, tol=TOL)
    b, _, ok2 = skq.density_response(rhs, kp.eps_k, -om, cfg1.eta, tol=TOL)
    assert ok1 and ok2 and a.is_cuda
    a, b = a.cpu().numpy(), b.cpu().numpy()
    for j in range(2):
        np.testing.assert_allclose(b[:, :, j], a[:, :, j].conj().T, atol=1e-9 * np.abs(a).max())
    acc = torch.zeros((8, 8, 2), dtype=torch.complex128, device="cuda")
    skq.density_response(rhs, kp.eps_k, om, cfg1.eta, weight=0.25, tol=TOL, out=acc)
    skq.density_response(rhs, kp.eps_k, om, cfg1.eta, weight=0.75, tol=TOL, out=acc)
    np.testing.assert_allclose(acc.cpu().numpy(), a, atol=1e-12 * np.abs(a).max())


def test_density_edge_cases(sgw, cfg1):
    kp, skq, sk = _setup(sgw, cfg1)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        skq.density_response(rhs, kp.eps_k, cfg1.omega, 0.0)
    with pytest.raises(sgw.SgwError, match="EUNSUPPORTED"):
        skq.density_response(rhs, kp.eps_k, np.linspace(0, 1, 257), cfg1.eta)
    fresh = sgw.System.from_instance(cfg1, kp.kq_frac)
    with pytest.raises(sgw.SgwError, match="ESTATE"):
        fresh.density_response(rhs, kp.eps_k, cfg1.omega, cfg1.eta)
    # a zero right-hand side contributes nothing
    dn, rep, ok = skq.density_response(np.zeros_like(rhs), kp.eps_k, cfg1.omega[:2], cfg1.eta)
    assert ok and np.abs(dn).max() == 0.0
