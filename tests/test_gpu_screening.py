"""Parity of the screening step (Eq. 4 and 9 with the truncated Coulomb potential of Sec. 2.6)
computed through the C ABI (sgw_screened_coulomb) with the FP64 oracle: on seeded synthetic
responses of the config-2 shape (elementwise, 1e-10 relative to the largest entry: epsilon's
condition number reaches 1.1e3 on these inputs, so either inverse may carry kappa n u ~ 4e-12),
and along the whole chain
Sternheimer -> density response -> epsilon^-1 -> W-bar on config 1 (1e-8 relative, the
accuracy of the solves)."""
import numpy as np
import pytest

import instances as I
import oracle as O
from parity import assert_columns_close

pytestmark = pytest.mark.gpu


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
def cfg2():
    return I.config2(k_subset=[0], n_omega=4)       # cell, q and the 32 G_p of config 2


def _qg(inst, ik=0):
    """Cartesian q + G_p of the instance's perturbations (q = k+q - k, fractional in B)."""
    kp = inst.kpoints[ik]
    b = O.reciprocal(inst.a)
    q = np.asarray(kp.kq_frac) - np.asarray(kp.k_frac)
    return (q[None, :] + inst.gp_miller) @ b


def _synthetic_dn(n, nw, seed):
    """A seeded response with the structure of Eq. 5: a negative-definite Hermitian static part
    and frequency-dependent poles."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    m = rng.standard_normal((n, 3 * n)) + 1j * rng.standard_normal((n, 3 * n))
    poles = rng.uniform(0.2, 2.0, 3 * n)
    w = np.linspace(0.0, 2.2, nw) + 0.0037j
    dn = np.empty((n, n, nw), complex)
    for j in range(nw):
        f = 1.0 / (w[j] - poles) - 1.0 / (w[j] + poles)
        dn[:, :, j] = 0.05 * (m * f) @ m.conj().T - 0.01 * (a @ a.conj().T)
    return dn


@pytest.mark.parametrize("r_cut", [6.0, 0.0])
def test_screening_matches_oracle_config2_shape(sgw, cfg2, r_cut):
    inst = cfg2
    qg = _qg(inst)
    dn = _synthetic_dn(len(qg), 64, 1)
    einv, wbar = sgw.screened_coulomb(dn, qg, inst.volume, r_cut)
    re, rw = O.screened_coulomb(dn, qg, inst.volume, r_cut)
    assert_columns_close(einv, re, 1e-10)
    assert_columns_close(wbar, rw, 1e-10)


def test_screening_chain_config1(sgw):
    """Density response on the GPU and in the oracle (the paper's real-space route), each
    followed by its own screening step."""
    inst = I.config1()
    kp = inst.kpoints[0]
    skq = sgw.System.from_instance(inst, kp.kq_frac)
    sk = sgw.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    rhs = skq.make_rhs(sk, kp.psi_k, inst.gp_miller)
    dn, rep, ok = skq.density_response(rhs, kp.eps_k, inst.omega, inst.eta, weight=2.0, tol=1e-10)
    assert ok
    qg = _qg(inst)
    einv, wbar = sgw.screened_coulomb(dn, qg, inst.volume, 8.0)
    h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
    dref = O.density_response(h, kp.psi_kq, kp.psi_k, kp.miller_k, kp.miller_kq, kp.eps_k, inst.gp_miller,
                              inst.omega, inst.eta, inst.fft_dims, 2.0)
    re, rw = O.screened_coulomb(dref, qg, inst.volume, 8.0)
    assert_columns_close(einv, re, 1e-8)
    assert_columns_close(wbar, rw, 1e-8)


def test_screening_device_buffers_and_zero_wavevector(sgw, cfg2):
    import torch
    inst = cfg2
    qg = _qg(inst)[:8].copy()
    qg[3] = 0.0
    dn = _synthetic_dn(8, 5, 2)
    e_host, w_host = sgw.screened_coulomb(dn, qg, inst.volume, 5.0)
    e_dev, w_dev = sgw.screened_coulomb(torch.from_numpy(dn).cuda(), qg, inst.volume, 5.0)
    assert e_dev.is_cuda and w_dev.is_cuda
    np.testing.assert_allclose(w_dev.cpu().numpy(), w_host, rtol=0, atol=1e-13 * np.abs(w_host).max())
    assert np.all(e_host[3, [0, 1, 2, 4, 5, 6, 7]] == 0) and np.all(e_host[[0, 1, 2, 4, 5, 6, 7], 3] == 0)
    re, rw = O.screened_coulomb(dn, qg, inst.volume, 5.0)
    assert_columns_close(w_host, rw, 1e-10)


def test_screening_edge_cases(sgw, cfg2):
    inst = cfg2
    qg = _qg(inst)[:4].copy()
    dn = _synthetic_dn(4, 3, 3)
    e, w = sgw.screened_coulomb(dn[:0, :0], qg[:0], inst.volume, 5.0)
    assert w.shape == (0, 0, 3)
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        sgw.screened_coulomb(dn, qg, -1.0, 5.0)
    z = qg.copy()
    z[0] = 0.0
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        sgw.screened_coulomb(dn, z, inst.volume, 0.0)
    with pytest.raises(sgw.SgwError, match="EUNSUPPORTED"):
        sgw.screened_coulomb(np.zeros((65, 65, 1), complex), np.ones((65, 3)), inst.volume, 5.0)
    # a non-finite response at one frequency: no finite pivot there, ENOCONV reported (a
    # response that makes epsilon exactly singular cannot be built in floating point)
    bad = dn.copy()
    bad[2, 1, 1] = np.nan
    with pytest.raises(sgw.SgwError, match="ENOCONV"):
        sgw.screened_coulomb(bad, qg, inst.volume, 5.0)
