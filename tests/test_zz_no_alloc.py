"""The allocation-free residual check gives the same per-pair residuals and certificates as
sgw_residual, on two calls in a row, through the C ABI.

Some callers cannot let a library allocate device memory (a framework whose allocator owns
all device memory, or code that must not pay cudaFree's device-wide synchronisation); for
them sgw_residual_noalloc keeps its scratch in a built-in device array.  This file is
collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import instances as I

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_residual_twice():
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
    dev = torch.device("cuda", 0)
    rhs = skq.make_rhs(sk, torch.from_numpy(kp.psi_k).to(dev), inst.gp_miller)
    e_ref = inst.e_ref(0)
    # a loosely converged solution, so that residuals are well above rounding
    dpsi, _, _ = skq.solve_shifted(rhs, e_ref, inst.omega, inst.eta, tol=1e-6, max_refine=-1)
    rel_ref, cert_ref = skq.residual(rhs, e_ref, inst.omega, inst.eta, dpsi)

    e_ref_d = torch.from_numpy(np.ascontiguousarray(e_ref)).to(dev)
    omega_d = torch.from_numpy(np.ascontiguousarray(inst.omega)).to(dev)
    for _ in range(2):
        rel = torch.full((rhs.shape[0], len(inst.omega)), float("nan"), dtype=torch.float64, device=dev)
        cert = torch.full_like(rel, float("nan"))
        skq.residual_noalloc(rhs, e_ref_d, omega_d, inst.eta, dpsi, rel, cert)
        torch.cuda.synchronize()
        np.testing.assert_allclose(rel.cpu().numpy(), rel_ref, rtol=1e-12, atol=0)
        np.testing.assert_allclose(cert.cpu().numpy(), cert_ref, rtol=1e-12, atol=0)
    assert rel_ref.max() > 1e-9        # the comparison is not between zeros
