"""The allocation-free residual check gives the same per-pair residuals and certificates as
sgw_residual, on two calls in a row, through the C ABI.

Some callers cannot let a library allocate device memory: a framework whose caching allocator
or fixed arena owns every byte of the device, or code that must not pay the device-wide
synchronisation cudaFree can imply.  For them sgw_residual_noalloc keeps its scratch in a
built-in device array.  This file is collected last so that a run stopping at the first
failure has run every other test.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_noalloc_size_limit_matches_header():
    """The documented plane-wave limit is the built-in scratch divided by two complex128
    vectors per CTA (the kernel's per-CTA need): 4 MiB / 32 B = 131 072."""
    text = open(os.path.join(ROOT, "include", "sgw.h")).read()
    m = re.search(r"#define SGW_NOALLOC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", text)
    assert m, "SGW_NOALLOC_SCRATCH_BYTES not found"
    nbytes = int(m.group(1)) << int(m.group(2))
    assert nbytes // (2 * 16) == 131072
    assert "n_pw > SGW_NOALLOC_SCRATCH_BYTES / 32 gives" in text


@pytest.mark.gpu
def test_residual_noalloc_matches_residual_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
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
    dpsi, _, _ = skq.solve_shifted(rhs, e_ref, inst.omega, inst.eta, tol=1e-6, max_refine=-1, cert_tol=-1)
    rel_ref, cert_ref = skq.residual(rhs, e_ref, inst.omega, inst.eta, dpsi)

    e_ref_d = torch.from_numpy(np.ascontiguousarray(e_ref)).to(dev)
    omega_d = torch.from_numpy(np.ascontiguousarray(inst.omega)).to(dev)
    rel = torch.full((rhs.shape[0], len(inst.omega)), float("nan"), dtype=torch.float64, device=dev)
    cert = torch.full_like(rel, float("nan"))
    torch.cuda.synchronize()
    for call in range(2):
        rel.fill_(float("nan"))
        cert.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        alloc0 = torch.cuda.memory_allocated(dev)
        skq.residual_noalloc(rhs, e_ref_d, omega_d, inst.eta, dpsi, rel, cert)
        torch.cuda.synchronize()
        if call == 1:   # the first call may look up the scratch array; the second allocates nothing
            assert torch.cuda.mem_get_info(dev)[0] == free0
            assert torch.cuda.memory_allocated(dev) == alloc0
        np.testing.assert_allclose(rel.cpu().numpy(), rel_ref, rtol=1e-12, atol=0)
        np.testing.assert_allclose(cert.cpu().numpy(), cert_ref, rtol=1e-12, atol=0)
    assert rel_ref.max() > 1e-9        # the comparison is not between zeros

    # host memory is refused by the library itself (the binding's checks bypassed): nothing runs
    lib = P.load()
    e_host = np.ascontiguousarray(e_ref)
    st = lib.sgw_residual_noalloc(skq._h, rhs.shape[0], rhs.data_ptr(), e_host.ctypes.data, len(inst.omega),
                                  omega_d.data_ptr(), float(inst.eta), dpsi.data_ptr(), rel.data_ptr(),
                                  cert.data_ptr(), None)
    assert st == P.SGW_EINVAL
    assert "device memory" in lib.sgw_last_error().decode()
    # the binding refuses a wrong dtype or shape before calling the library
    with pytest.raises(TypeError):
        skq.residual_noalloc(rhs, e_ref_d.float(), omega_d, inst.eta, dpsi, rel, cert)
    with pytest.raises(ValueError):
        skq.residual_noalloc(rhs, e_ref_d, omega_d, inst.eta, dpsi[:, :-1].contiguous(), rel, cert)
    # the caller's current device is unchanged
    assert torch.cuda.current_device() == 0
