"""Parity of the imaginary-axis route of Sec. 2.7 through the C ABI: the density response at
imaginary frequencies (sgw_density_response_w) against the oracle's real-space route, and the
batched AAA continuation (sgw_aaa) against the oracle's AAA on the same samples."""
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


def test_imaginary_axis_density_config1(sgw):
    inst = I.config1()
    kp = inst.kpoints[0]
    skq = sgw.System.from_instance(inst, kp.kq_frac)
    sk = sgw.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    rhs = skq.make_rhs(sk, kp.psi_k, inst.gp_miller)
    w = 1j * np.linspace(0.05, 3.0, 8)
    dn, rep, ok = skq.density_response_w(rhs, kp.eps_k, w, weight=2.0, tol=1e-10, precision="df32")
    assert ok and rep["rel_res"].max() <= 1e-10
    h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
    ref = O.density_response_w(h, kp.psi_kq, kp.psi_k, kp.miller_k, kp.miller_kq, kp.eps_k, inst.gp_miller, w,
                               inst.fft_dims, 2.0)
    assert_columns_close(dn, ref, 1e-8)
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        skq.density_response_w(rhs, kp.eps_k, [0.3 + 0.0j], tol=1e-10)


def _models(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        p = rng.uniform(0.3, 2.5, 3) * rng.choice([-1, 1], 3) - 1j * rng.uniform(0.005, 0.3, 3)
        a = rng.normal(0, 0.4, 3) + 1j * rng.normal(0, 0.1, 3)
        out.append((p, a, rng.normal()))
    return out


def _eval_model(mdl, z):
    p, a, c = mdl
    return c + np.sum(a[None, :] / (np.asarray(z)[:, None] - p[None, :]), axis=1)


def test_aaa_matches_oracle_on_rational_models(sgw):
    zi = 1j * np.linspace(0.02, 6.0, 48)
    x = np.linspace(-3.0, 3.0, 61) + 0.02j
    models = _models(40, 1)
    f = np.array([_eval_model(m, zi) for m in models])
    r, deg = sgw.aaa(zi, f, x, tol=1e-13, mmax=20)
    for i, mdl in enumerate(models):
        zs, fs, w = O.aaa(zi, f[i], tol=1e-13, mmax=20)
        ref = O.aaa_eval(zs, fs, w, x)
        exact = _eval_model(mdl, x)
        assert deg[i] == len(zs)
        assert np.abs(r[i] - ref).max() <= 1e-8 * np.abs(exact).max()
        assert np.abs(r[i] - exact).max() <= 1e-7 * np.abs(exact).max()


def test_aaa_analytic_function_and_device_buffers(sgw):
    import torch
    xs = np.linspace(-1.0, 1.0, 100).astype(complex)
    f = np.vstack([np.exp(xs), np.cos(3 * xs), 1.0 / (1.2 - xs)])
    t = np.linspace(-1.0, 1.0, 301).astype(complex)
    r, deg = sgw.aaa(xs, f, t, tol=1e-13)
    exact = np.vstack([np.exp(t), np.cos(3 * t), 1.0 / (1.2 - t)])
    assert np.abs(r - exact).max() < 1e-11 * np.abs(exact).max()
    rd, degd = sgw.aaa(xs, torch.from_numpy(f).cuda(), t, tol=1e-13)
    assert rd.is_cuda
    np.testing.assert_allclose(rd.cpu().numpy(), r, rtol=0, atol=1e-14 * np.abs(r).max())
    assert np.array_equal(deg, degd)
    # support points are reproduced exactly
    rs, _ = sgw.aaa(xs, f[:1], xs, tol=1e-13)
    zs, fs, w = O.aaa(xs, f[0], tol=1e-13)
    for s in zs:
        k = int(np.nonzero(xs == s)[0][0])
        assert rs[0, k] == f[0, k]


def test_aaa_edge_cases(sgw):
    z = 1j * np.linspace(0.1, 2.0, 10)
    f = np.vstack([1.0 / (z + 0.5), 2.0 + 0 * z])
    r, deg = sgw.aaa(z, f, [0.3 + 0.1j], tol=1e-13, mmax=1)
    assert list(deg) == [1, 1] and r[1, 0] == 2.0
    with pytest.raises(sgw.SgwError, match="EUNSUPPORTED"):
        sgw.aaa(1j * np.linspace(0.1, 2.0, 129), np.ones((1, 129)), [0.0])
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        sgw.aaa(np.array([0.1j, 0.1j, 0.2j]), np.ones((1, 3)), [0.0])
    bad = f.copy()
    bad[0, 3] = np.nan
    with pytest.raises(sgw.SgwError, match="EINVAL"):
        sgw.aaa(z, bad, [0.3 + 0.1j])
    r, deg = sgw.aaa(z, np.zeros((0, 10)), [0.3])
    assert r.shape == (0, 1)
