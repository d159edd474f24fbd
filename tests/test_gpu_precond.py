"""GPU parity of the per-shift preconditioned solves and the learned preconditioner's
kernels (perceptron forward, gradient, Adam step, diagonals, training rows) against the
FP64 oracles, through the C ABI."""
import numpy as np
import pytest

import instances as I
import oracle as O
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    import paper_1812_03717_gb300 as P
    from paper_1812_03717_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    inst = I.config1()
    kp = inst.kpoints[0]
    skq = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    rhs = skq.make_rhs(sk, kp.psi_k, inst.gp_miller)
    # the oracle's own right-hand sides and basis (bit-identical to the library's) feed the oracle
    rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, inst.gp_miller)
    assert np.array_equal(rhs, rref)
    return P, inst, skq, rhs, rref


def _theta(seed=3):
    rng = np.random.default_rng(seed)
    th = M.init_params(rng)
    th[-(M.N_H + 1):] = (0.05 * rng.standard_normal(M.N_H + 1)).astype(np.float32)
    return th


def _rows(n=3000, seed=4):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-0.4, 0, n),
                         rng.uniform(-0.5, -0.2, n)]).astype(np.float32)
    t = rng.normal(0, 0.5, n).astype(np.float32)
    return x, t


def test_mlp_forward_matches_oracle(env):
    import torch
    P = env[0]
    th = _theta()
    mlp = P.MLP(th)
    x, _ = _rows()
    y = mlp.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = M.forward(M.bf16_round(th), x.astype(np.float64))
    assert np.abs(y - ref).max() < 1e-4 * max(1.0, np.abs(ref).max())


def test_mlp_gradient_matches_oracle(env):
    """GPU backward (bf16 weights, FP32 accumulation) vs FP64 backpropagation with the same
    bf16-rounded weights: relative error <= 1e-3."""
    import torch
    P = env[0]
    th = _theta()
    mlp = P.MLP(th)
    x, t = _rows()
    loss, g = mlp.grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    rl, rg = M.loss_and_grad(M.bf16_round(th), x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(rl, rel=1e-4)
    assert np.linalg.norm(g - rg) <= 1e-3 * np.linalg.norm(rg)


def test_mlp_adam_step_matches_oracle(env):
    import torch
    P = env[0]
    th = _theta()
    mlp = P.MLP(th)
    x, t = _rows()
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, g = mlp.grad(xd, td)
    mlp.train_step(xd, td, lr=1e-3)
    ref, _, _ = M.adam_step(th.astype(np.float64), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS),
                            g.astype(np.float64), 1, 1e-3)
    np.testing.assert_allclose(mlp.params, ref, rtol=0, atol=2e-6)


def test_training_reduces_loss(env):
    import torch
    P = env[0]
    mlp = P.MLP(M.init_params(np.random.default_rng(0)))
    x, _ = _rows(4096)
    t = (np.sin(3 * x[:, 0]) - x[:, 1]).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = mlp.train_step(xd, td, lr=3e-3)
    for _ in range(150):
        last = mlp.train_step(xd, td, lr=3e-3)
    assert last < 0.2 * first


def test_diagonals_match_oracle(env):
    P, inst, skq, rhs, rref = env
    kp = inst.kpoints[0]
    mil, kin = O.gsphere(inst.a, kp.kq_frac, inst.ecut_ry)   # the oracle's basis
    rows = [0, 7, 19]
    e = inst.e_ref(0)[rows]
    om = inst.omega[[2, 9, 15]]
    d = skq.precond_diag(rhs[rows], e, om, inst.eta, "plain")
    for i, r in enumerate(rows):
        np.testing.assert_allclose(d[i], M.plain_scaling(kin, rref[r]), rtol=1e-13)
    beta = O.kb_beta(inst.a, inst.tau, kp.kq_frac, mil, inst.kb_atom, inst.kb_width)
    hd = M.h_diag(kin, inst.vloc_r.mean(), beta, inst.kb_d)
    dj = skq.precond_diag(rhs[rows], e, om, inst.eta, "jacobi", delta=[0.1, 0.3, 1.0])
    for i in range(3):
        np.testing.assert_allclose(dj[i], M.jacobi_scaling(hd, e[i] + om[i] + 1j * inst.eta, [0.1, 0.3, 1.0][i]),
                                   rtol=1e-12)
    th = _theta()
    mlp = P.MLP(th)
    dl = skq.precond_diag(rhs[rows], e, om, inst.eta, "learned", mlp=mlp)
    for i, r in enumerate(rows):
        f = M.features(kin, inst.ecut_ry, om[i], e[i], inst.vloc_r.mean())
        ref = M.plain_scaling(kin, rref[r]) * np.exp(M.forward(M.bf16_round(th), f))
        np.testing.assert_allclose(dl[i], ref, rtol=2e-4)


def test_training_rows_match_oracle(env):
    import torch
    P, inst, skq, rhs, rref = env
    kp = inst.kpoints[0]
    mil, kin = O.gsphere(inst.a, kp.kq_frac, inst.ecut_ry)   # the oracle's basis
    rows = [3, 11]
    e = inst.e_ref(0)[rows]
    om = inst.omega[[4, 12]]
    delta = np.array([0.3, 0.0])
    f, t = skq.training_rows(torch.from_numpy(rhs[rows]).cuda(), e, om, inst.eta, delta)
    f, t = f.cpu().numpy().reshape(2, -1, 4), t.cpu().numpy().reshape(2, -1)
    beta = O.kb_beta(inst.a, inst.tau, kp.kq_frac, mil, inst.kb_atom, inst.kb_width)
    hd = M.h_diag(kin, inst.vloc_r.mean(), beta, inst.kb_d)
    for i, r in enumerate(rows):
        np.testing.assert_allclose(f[i], M.features(kin, inst.ecut_ry, om[i], e[i], inst.vloc_r.mean()), rtol=1e-6)
        m = M.plain_scaling(kin, rref[r])
        j = M.jacobi_scaling(hd, e[i] + om[i] + 1j * inst.eta, delta[i]) if delta[i] > 0 else None
        np.testing.assert_allclose(t[i], M.targets(m, j), atol=1e-6)


@pytest.mark.parametrize("precond", ["none", "plain", "jacobi", "learned"])
def test_pershift_solve_matches_lu(env, precond):
    """Preconditioning changes the route, not the answer: per-shift solves vs the oracle LU."""
    P, inst, skq, rhs, rref = env
    kp = inst.kpoints[0]
    rows = np.array([0, 5, 13, 20, 27, 31])
    cols = np.array([0, 3, 8, 11, 14, 15])
    e = inst.e_ref(0)[rows]
    om = inst.omega[cols]
    mlp = P.MLP(_theta()) if precond == "learned" else None
    x, rep, ok = skq.solve_pershift(rhs[rows], e, om, inst.eta, tol=1e-10, precond=precond,
                                    delta=0.3 if precond == "jacobi" else None, mlp=mlp)
    assert ok, rep["status"]
    assert rep["rel_res"].max() <= 1e-10
    h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
    for i, (r, j) in enumerate(zip(rows, cols)):
        ref = O.solve_shifted(h, kp.psi_kq, rref[r:r + 1], e[i:i + 1], om[i:i + 1], inst.eta)[0, 0]
        assert np.linalg.norm(x[i] - ref) / np.linalg.norm(ref) < 1e-8
