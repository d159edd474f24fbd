"""Parity of the library's other execution modes with the FP64 oracle, through the C ABI:

* the cluster-split H application (the box shared by 2..8 CTAs through distributed shared
  memory) on boxes that also fit one CTA, so the dense oracle checks it at small sizes;
* the FP32 (complex64) inner solve inside FP64 iterative refinement;
* the certificate-aware stopping rule (every pair's |r| / (eta |x|) <= 1e-8);
* resuming from given solutions (x0) and preconditioned corrections with the learned
  diagonal, including the fall back to the plain diagonal;
* the BiCGstab(ell) kernel (multishift, per-shift and preconditioned corrections) on
  cluster-split boxes.
"""
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
def cfg1():
    return I.config1()


@pytest.fixture(scope="module")
def cfg2():
    return I.config2(k_subset=[0])


@pytest.fixture(scope="module")
def h2(cfg2):
    kp = cfg2.kpoints[0]
    h, _, _ = O.dense_h_inst(cfg2, kp.kq_frac)
    return h


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def _systems(P, inst, ik=0):
    kp = inst.kpoints[ik]
    skq = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    return skq, sk


# ----------------------------------------------------------------- cluster-split box

@pytest.mark.parametrize("csize", [2, 3, 4, 8])
def test_cluster_apply_matches_dense(sgw, cfg2, h2, csize):
    """H applied by a cluster of csize CTAs (sticks split by rank, xy-planes gathered through
    distributed shared memory) equals the oracle's dense H, in every precision."""
    kp = cfg2.kpoints[0]
    s = sgw.System.from_instance(cfg2, kp.kq_frac)
    assert s.split()[0] == 1          # config 2 fits one CTA by default
    assert s.set_split(csize)[0] == csize
    rng = np.random.default_rng(21)
    x = rng.standard_normal((6, s.n_pw)) + 1j * rng.standard_normal((6, s.n_pw))
    ref = x @ h2.T
    assert _relerr(s.apply_h(x), ref).max() < 1e-12
    assert _relerr(s.apply_h(x, precision="df32"), ref).max() < 1e-11
    if s.split()[1] == csize:
        assert _relerr(s.apply_h(x, precision="fp32"), ref).max() < 2e-6


@pytest.mark.parametrize("csize", [2, 4])
def test_cluster_shifted_operator_and_solve(sgw, cfg2, h2, csize):
    """The projected shifted operator and the multishift solve on a cluster split: the same
    answers as the LU, and the same answers as the one-CTA split."""
    kp = cfg2.kpoints[0]
    skq, sk = _systems(sgw, cfg2)
    rng = np.random.default_rng(22)
    x = rng.standard_normal((3, skq.n_pw)) + 1j * rng.standard_normal((3, skq.n_pw))
    z = np.array([0.2 + 0.0037j, -0.1 + 0.5j, 1.0 + 0.0037j])
    y1 = skq.apply_shifted(x, z)
    skq.set_split(csize)
    yc = skq.apply_shifted(x, z)
    ref = np.stack([O.shifted_operator(h2, kp.psi_kq, z[i]) @ x[i] for i in range(3)])
    assert _relerr(yc, ref).max() < 1e-12
    assert _relerr(yc, y1).max() < 1e-12
    npert = cfg2.n_pert
    rows = np.array([0, 5, npert + 3, 7 * npert + 31])
    rhs = skq.make_rhs(sk, kp.psi_k, cfg2.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg2.gp_miller)[rows]
    e_ref = cfg2.e_ref(0)[rows]
    om = cfg2.omega[[0, 20, 41, 63]]
    d, rep, ok = skq.solve_shifted(rhs, e_ref, om, cfg2.eta, tol=1e-10, precision="df32")
    assert ok, rep["status"]
    ref = O.solve_shifted(h2, kp.psi_kq, rref, e_ref, om, cfg2.eta)
    assert _relerr(d, ref).max() < TOL_SOLVE
    assert rep["cert"].max() <= 1e-8
    skq.set_split(0)
    assert skq.split()[0] == 1
    d1, _, ok1 = skq.solve_shifted(rhs, e_ref, om, cfg2.eta, tol=1e-10, precision="df32")
    assert ok1 and _relerr(d, d1).max() < 1e-8


def test_cluster_residual_and_green(sgw, cfg1):
    """The true-residual kernel and the Green's-function solve on a two-CTA split of config 1."""
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[:6]
    e_ref = cfg1.e_ref(0)[:6]
    d, _, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-6, cert_tol=-1, max_refine=-1)
    rel1, cert1 = skq.residual(rhs, e_ref, cfg1.omega, cfg1.eta, d)
    skq.set_split(2)
    rel2, cert2 = skq.residual(rhs, e_ref, cfg1.omega, cfg1.eta, d)
    # the cluster sums the same products in another order: equal to rounding
    np.testing.assert_allclose(rel2, rel1, rtol=1e-6, atol=1e-15)
    np.testing.assert_allclose(cert2, cert1, rtol=1e-6, atol=1e-15)
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    cols = np.array([0, 17, 100])
    z = np.array([0.3 + 0.0037j, -0.2 - 0.0037j])
    g, rep, ok = skq.solve_green(cols, z, tol=1e-10, precision="df32")
    assert ok
    ref = O.green_columns(h, cols, z)
    assert _relerr(g, ref).max() < TOL_SOLVE


def _theta(seed=3):
    """Perceptron parameters with a non-zero last layer (a learned diagonal that differs from
    the plain scaling)."""
    from oracle import mlp_oracle as M
    rng = np.random.default_rng(seed)
    th = M.init_params(rng)
    th[-(M.N_H + 1):] = (0.05 * rng.standard_normal(M.N_H + 1)).astype(np.float32)
    return th


def test_cluster_bicgstab_multishift(sgw, cfg1):
    """The shifted BiCGstab(ell) kernel on a two-CTA split of config 1: every pair converges to
    the LU's answer and to the one-CTA kernel's."""
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[:6]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)[:6]
    e_ref = cfg1.e_ref(0)[:6]
    d1, _, ok1 = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, method="bicgstab")
    assert skq.set_split(2)[0] == 2
    d2, rep2, ok2 = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, method="bicgstab")
    assert ok1 and ok2, rep2["status"]
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    ref = O.solve_shifted(h, kp.psi_kq, rref, e_ref, cfg1.omega, cfg1.eta)
    assert _relerr(d2, ref).max() < TOL_SOLVE
    assert _relerr(d2, d1).max() < 2 * TOL_SOLVE


@pytest.mark.parametrize("precond", ["none", "plain", "learned"])
def test_cluster_pershift_solves(sgw, cfg1, precond):
    """Per-shift right-preconditioned BiCGstab on a two-CTA split of config 1: the LU's answers
    (the diagonal changes the route, not the answer)."""
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    assert skq.set_split(2)[0] == 2
    rows = np.array([0, 5, 13, 20, 27, 31])
    cols = np.array([0, 3, 8, 11, 14, 15])
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)[rows]
    e = cfg1.e_ref(0)[rows]
    om = cfg1.omega[cols]
    mlp = sgw.MLP(_theta()) if precond == "learned" else None
    x, rep, ok = skq.solve_pershift(rhs, e, om, cfg1.eta, tol=1e-10, precond=precond, mlp=mlp)
    assert ok, rep["status"]
    assert rep["rel_res"].max() <= 1e-10
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    ref = np.stack([O.solve_shifted(h, kp.psi_kq, rref[i:i + 1], e[i:i + 1], om[i:i + 1], cfg1.eta)[0, 0]
                    for i in range(len(rows))])
    assert _relerr(x, ref).max() < TOL_SOLVE


def test_cluster_pershift_config2(sgw, cfg2, h2):
    """Per-shift solves with the plain diagonal on a four-CTA split of config 2 (1 647 plane
    waves, frequencies from the bottom to the top of the 0-60 eV window) against the LU."""
    kp = cfg2.kpoints[0]
    skq, sk = _systems(sgw, cfg2)
    assert skq.set_split(4)[0] == 4
    npert = cfg2.n_pert
    rows = np.array([0, 5, npert + 3, 7 * npert + 31])
    rhs = skq.make_rhs(sk, kp.psi_k, cfg2.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg2.gp_miller)[rows]
    e = cfg2.e_ref(0)[rows]
    om = cfg2.omega[[0, 20, 41, 63]]
    x, rep, ok = skq.solve_pershift(rhs, e, om, cfg2.eta, tol=1e-10, precond="plain")
    assert ok, rep["status"]
    ref = np.stack([O.solve_shifted(h2, kp.psi_kq, rref[i:i + 1], e[i:i + 1], om[i:i + 1], cfg2.eta)[0, 0]
                    for i in range(len(rows))])
    assert _relerr(x, ref).max() < TOL_SOLVE


def test_cluster_preconditioned_corrections(sgw, cfg1):
    """Resuming from a perturbed solution on a two-CTA split: corrections by the learned
    diagonal (untrained network: the plain scaling), the same with the fall back forced by a
    plain budget of one H application, and by the plain diagonal all reach the LU."""
    from oracle import mlp_oracle as M
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    assert skq.set_split(2)[0] == 2
    rows = np.arange(1, 32, 4)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)[rows]
    e_ref = cfg1.e_ref(0)[rows]
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    ref = O.solve_shifted(h, kp.psi_kq, rref, e_ref, cfg1.omega, cfg1.eta)
    x0 = ref * (1 + 1e-3 * np.random.default_rng(6).standard_normal(ref.shape))
    mlp = sgw.MLP(M.init_params(np.random.default_rng(0)))
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0, precond="learned", mlp=mlp)
    assert ok and _relerr(d, ref).max() < TOL_SOLVE
    assert rep["fallbacks"][0] == 0
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0, precond="learned", mlp=mlp,
                                   plain_budget=1)
    assert ok and _relerr(d, ref).max() < TOL_SOLVE
    assert rep["fallbacks"][0] > 0
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0, precond="plain")
    assert ok and _relerr(d, ref).max() < TOL_SOLVE


# ------------------------------------------------------------ FP32 inner + FP64 refinement

def test_apply_h_fp32_matches_dense(sgw, cfg2, h2):
    kp = cfg2.kpoints[0]
    s = sgw.System.from_instance(cfg2, kp.kq_frac)
    rng = np.random.default_rng(23)
    x = rng.standard_normal((4, s.n_pw)) + 1j * rng.standard_normal((4, s.n_pw))
    err = _relerr(s.apply_h(x, precision="fp32"), x @ h2.T).max()
    assert 1e-9 < err < 2e-6   # single precision: FP32 rounding, not FP64


def test_solve_fp32_config1_all_pairs(sgw, cfg1):
    """FP32 multishift pass + FP64 residual + float-float corrections: every pair of config 1
    meets the FP64 criteria and the LU to 1e-8."""
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)
    e_ref = cfg1.e_ref(0)
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, precision="fp32")
    assert ok, np.unique(rep["status"], return_counts=True)
    assert rep["rel_res"].max() <= 1e-10 and rep["cert"].max() <= 1e-8
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    ref = O.solve_shifted(h, kp.psi_kq, rref, e_ref, cfg1.omega, cfg1.eta)
    assert _relerr(d, ref).max() < TOL_SOLVE


def test_solve_fp32_config2_sampled(sgw, cfg2, h2):
    kp = cfg2.kpoints[0]
    skq, sk = _systems(sgw, cfg2)
    npert = cfg2.n_pert
    rows = np.concatenate([np.arange(v * npert, v * npert + 8) for v in (0, 15)])
    rhs = skq.make_rhs(sk, kp.psi_k, cfg2.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg2.gp_miller)[rows]
    e_ref = cfg2.e_ref(0)[rows]
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg2.omega, cfg2.eta, tol=1e-10, precision="fp32")
    assert ok, np.unique(rep["status"], return_counts=True)
    for j in (0, 33, 63):
        ref = O.solve_shifted(h2, kp.psi_kq, rref, e_ref, cfg2.omega[j:j + 1], cfg2.eta)[:, 0]
        assert _relerr(d[:, j], ref).max() < TOL_SOLVE


# ----------------------------------------------------------- certificate-aware stopping

def test_every_pair_certified(sgw, cfg2):
    """The default stopping rule: rel_res <= tol and cert <= 1e-8 on every pair; without the
    certificate rule (cert_tol < 0) some pairs stop with cert above 1e-8 (the rule matters)."""
    kp = cfg2.kpoints[0]
    skq, sk = _systems(sgw, cfg2)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg2.gp_miller)[::16].copy()
    e_ref = cfg2.e_ref(0)[::16]
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg2.omega, cfg2.eta, tol=1e-10, precision="df32")
    assert ok
    assert rep["rel_res"].max() <= 1e-10 and rep["cert"].max() <= 1e-8
    _, rep0, _ = skq.solve_shifted(rhs, e_ref, cfg2.omega, cfg2.eta, tol=1e-10, precision="df32", cert_tol=-1)
    assert rep0["cert"].max() > 1e-8
    assert rep["matvecs"].max(axis=1).sum() >= rep0["matvecs"].max(axis=1).sum()


# ------------------------------------------------------------- resume and preconditioning

def test_resume_from_x0(sgw, cfg1):
    """x0 = the oracle's solution perturbed by 1e-4: the library repairs every pair to the LU
    at 1e-8; x0 = an already converged solution costs no H application at all."""
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    rows = np.arange(0, 32, 3)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)[rows]
    e_ref = cfg1.e_ref(0)[rows]
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    ref = O.solve_shifted(h, kp.psi_kq, rref, e_ref, cfg1.omega, cfg1.eta)
    rng = np.random.default_rng(5)
    x0 = ref * (1 + 1e-4 * rng.standard_normal(ref.shape))
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0)
    assert ok
    assert _relerr(d, ref).max() < TOL_SOLVE
    assert rep["matvecs"].min() > 0
    d2, rep2, ok2 = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=d)
    assert ok2 and np.all(rep2["matvecs"] == 0)
    assert _relerr(d2, d).max() < 1e-14   # only re-projected onto range(P_c)


def test_learned_corrections_and_plain_fallback(sgw, cfg1):
    """Corrections preconditioned by the learned diagonal (an untrained network: exactly the
    plain scaling) reach the LU; with a plain budget of one H application the learned round
    stops at two, and its pairs restart with the plain diagonal (the fall back)."""
    from oracle import mlp_oracle as M
    kp = cfg1.kpoints[0]
    skq, sk = _systems(sgw, cfg1)
    rows = np.arange(1, 32, 4)
    rhs = skq.make_rhs(sk, kp.psi_k, cfg1.gp_miller)[rows]
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, cfg1.gp_miller)[rows]
    e_ref = cfg1.e_ref(0)[rows]
    h, _, _ = O.dense_h_inst(cfg1, kp.kq_frac)
    ref = O.solve_shifted(h, kp.psi_kq, rref, e_ref, cfg1.omega, cfg1.eta)
    x0 = ref * (1 + 1e-3 * np.random.default_rng(6).standard_normal(ref.shape))
    mlp = sgw.MLP(M.init_params(np.random.default_rng(0)))
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0, precond="learned", mlp=mlp)
    assert ok and _relerr(d, ref).max() < TOL_SOLVE
    assert rep["fallbacks"][0] == 0
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0, precond="learned", mlp=mlp,
                                   plain_budget=1)
    assert ok and _relerr(d, ref).max() < TOL_SOLVE
    assert rep["fallbacks"][0] > 0
    d, rep, ok = skq.solve_shifted(rhs, e_ref, cfg1.omega, cfg1.eta, tol=1e-10, x0=x0, precond="plain")
    assert ok and _relerr(d, ref).max() < TOL_SOLVE
