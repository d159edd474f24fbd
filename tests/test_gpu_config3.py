"""Parity at the size of the 64-atom supercell (18 277 plane waves, 72^3 box, 128 occupied
bands, 64 perturbations, 128 frequencies), where the on-chip box is shared by a
thread-block cluster: bit-exact sphere, map and Eq. 8 gather; H against the oracle's dense H;
the multishift solve of every perturbation of one band at all 128 frequencies, each pair's
FP64 residual and certificate, and dense-LU spot checks of three (band, frequency) pairs with
all 64 perturbations.  The oracle's dense H is 5.3 GB and each LU some 1.6e13 flops on the
host: this module takes minutes."""
import numpy as np
import pytest

import instances as I
import oracle as O

pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-8


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
def inst3():
    return I.config3()


@pytest.fixture(scope="module")
def sys3(sgw, inst3):
    kp = inst3.kpoints[0]
    s = sgw.System.from_instance(inst3, kp.kq_frac)
    s.set_occupied(kp.psi_kq, kp.eps_kq)
    return s


@pytest.fixture(scope="module")
def h3(inst3):
    h, _, _ = O.dense_h_inst(inst3, inst3.kpoints[0].kq_frac)
    return h


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def test_config3_sphere_map_and_split(sys3, inst3):
    mil, kin = sys3.gvectors
    ref_m, ref_k = O.gsphere(inst3.a, inst3.kpoints[0].kq_frac, inst3.ecut_ry)
    assert len(ref_m) == 18277
    assert np.array_equal(mil, ref_m)
    np.testing.assert_allclose(kin, ref_k, rtol=1e-14, atol=0)
    assert np.array_equal(sys3.box_map(), O.box_map(ref_m, inst3.fft_dims))
    c16, c8 = sys3.split()
    assert c16 > 1 and c8 >= 1        # the 72^3 box does not fit one CTA


def test_config3_apply_matches_dense(sys3, h3):
    rng = np.random.default_rng(31)
    x = rng.standard_normal((3, sys3.n_pw)) + 1j * rng.standard_normal((3, sys3.n_pw))
    ref = x @ h3.T
    assert _relerr(sys3.apply_h(x), ref).max() < 1e-12
    assert _relerr(sys3.apply_h(x, precision="df32"), ref).max() < 1e-11
    assert _relerr(sys3.apply_h(x, precision="fp32"), ref).max() < 3e-6


def test_config3_rhs_solve_and_lu_spot_checks(sgw, sys3, inst3, h3):
    """All 64 perturbations of one band at all 128 frequencies (the highest ones need some
    14 000 Lanczos steps): every pair's FP64 residual and certificate, and the dense LU of
    three (band, frequency) pairs with all 64 perturbations."""
    import torch
    kp = inst3.kpoints[0]
    npert = inst3.n_pert
    band = 37
    # Eq. 8 right-hand sides of the band for every perturbation, bit-exact against the oracle
    sk = sgw.System.from_instance(inst3, kp.k_frac)
    rhs = sys3.make_rhs(sk, torch.from_numpy(kp.psi_k[[band]]).cuda(), inst3.gp_miller)
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k[[band]], inst3.gp_miller)
    assert np.array_equal(rhs.cpu().numpy(), rref)
    e_ref = np.full(npert, kp.eps_k[band])
    d, rep, ok = sys3.solve_shifted(rhs, e_ref, inst3.omega, inst3.eta, tol=1e-10, precision="df32")
    torch.cuda.synchronize()
    assert ok, np.unique(rep["status"], return_counts=True)
    assert rep["rel_res"].max() <= 1e-10 and rep["cert"].max() <= 1e-8
    d = d.cpu().numpy()
    js = [0, 64, 127]
    ref = O.solve_shifted(h3, kp.psi_kq, rref, e_ref, inst3.omega[js], inst3.eta)
    assert _relerr(d[:, js], ref).max() < TOL_SOLVE
