"""Thin ctypes binding of libsgw.so (include/sgw.h): argument marshalling only.

Vectors may be numpy arrays (host) or torch tensors (host or CUDA); the library detects
device pointers itself.  Outputs are allocated like the main input (numpy -> numpy,
CUDA tensor -> CUDA tensor).  Every compute step runs in the library's CUDA kernels; if
the library is missing this module raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsgw.so")

SGW_OK, SGW_EINVAL, SGW_ENOMEM, SGW_ECUDA, SGW_ENOCONV, SGW_EALIAS, SGW_ESTATE, SGW_EUNSUPPORTED = range(8)
PAIR_CONVERGED, PAIR_MAXITER, PAIR_BREAKDOWN, PAIR_NONFINITE = range(4)
METHOD_LANCZOS, METHOD_BICGSTAB = range(2)
PREC_FP64, PREC_DF32, PREC_FP32 = range(3)
_PREC = {"fp64": PREC_FP64, "df32": PREC_DF32, "fp32": PREC_FP32}
STATUS_NAMES = ["SGW_OK", "SGW_EINVAL", "SGW_ENOMEM", "SGW_ECUDA", "SGW_ENOCONV", "SGW_EALIAS", "SGW_ESTATE",
                "SGW_EUNSUPPORTED"]

EXPORTS = ["sgw_create_system", "sgw_get_gvectors", "sgw_get_box_map", "sgw_set_split", "sgw_get_split",
           "sgw_solve_capacity", "sgw_solve_batched",
           "sgw_set_occupied", "sgw_make_rhs",
           "sgw_apply_h", "sgw_apply_shifted", "sgw_solve_shifted", "sgw_solve_green", "sgw_density_response", "sgw_density_response_w", "sgw_aaa", "sgw_screened_coulomb", "sgw_residual", "sgw_residual_noalloc",
           "sgw_solve_pershift", "sgw_precond_diag", "sgw_training_rows", "sgw_mlp_create", "sgw_mlp_get_params",
           "sgw_mlp_forward", "sgw_mlp_grad", "sgw_mlp_train_step", "sgw_mlp_destroy", "sgw_destroy_system",
           "sgw_last_error"]
PRECOND_NONE, PRECOND_PLAIN, PRECOND_LEARNED, PRECOND_JACOBI = range(4)
_PRECOND = {"none": PRECOND_NONE, "plain": PRECOND_PLAIN, "learned": PRECOND_LEARNED, "jacobi": PRECOND_JACOBI}
MLP_PARAMS = 4545


class SgwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class _Cell(ctypes.Structure):
    _fields_ = [("a", (ctypes.c_double * 3) * 3), ("n_atoms", ctypes.c_int), ("tau", ctypes.c_void_p)]


class _KB(ctypes.Structure):
    _fields_ = [("n_proj", ctypes.c_int), ("atom", ctypes.c_void_p), ("width", ctypes.c_void_p),
                ("D", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("precision", ctypes.c_int), ("ell", ctypes.c_int),
                ("seed_index", ctypes.c_int), ("max_matvec", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("threads", ctypes.c_int), ("stream", ctypes.c_void_p), ("cert_tol", ctypes.c_double),
                ("x0", ctypes.c_void_p), ("precond", ctypes.c_int), ("mlp", ctypes.c_void_p),
                ("plain_budget", ctypes.c_int)]


def _opts(method=0, precision=0, ell=4, seed_index=-1, max_matvec=0, max_refine=0, threads=0, stream=None,
          cert_tol=0.0, x0=None, precond=0, mlp=None, plain_budget=0):
    return _Opts(method, precision, ell, seed_index, max_matvec, max_refine, threads, stream, cert_tol, x0,
                 precond, mlp, plain_budget)


_REPORT_KEYS = ("matvecs", "est_res", "rel_res", "cert", "status", "launches", "kernel_ms", "fallbacks")


class _Report(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in _REPORT_KEYS]


def _report(nr, nw):
    """Per-pair report arrays [nr][nw] (nw None: [nr]) and the ctypes struct pointing at them."""
    shp = (nr,) if nw is None else (nr, nw)
    rep = {"matvecs": np.zeros(shp, dtype=np.int32), "est_res": np.zeros(shp), "rel_res": np.zeros(shp),
           "cert": np.zeros(shp), "status": np.zeros(shp, dtype=np.int32), "launches": np.zeros(1, dtype=np.int32),
           "kernel_ms": np.zeros(1), "fallbacks": np.zeros(1, dtype=np.int32)}
    return rep, _Report(*(rep[k].ctypes.data for k in _REPORT_KEYS))


class _BatchItem(ctypes.Structure):
    _fields_ = [("sys", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("rhs", ctypes.c_void_p), ("e_ref", ctypes.c_void_p),
                ("nomega", ctypes.c_int), ("omega", ctypes.c_void_p), ("dpsi", ctypes.c_void_p),
                ("report", ctypes.c_void_p)]


def solve_batched(items, eta, tol=1e-10, precision="fp64", threads=0, max_matvec=0, max_refine=0, cert_tol=0.0,
                  stream=None, raise_on_noconv=False):
    """sgw_solve_batched: items is a list of dicts {sys, rhs, e_ref, omega[, out]} (systems of
    uneven sizes); returns (list of dpsi, list of report dicts, converged flag)."""
    keep, citems, outs, reps = [], [], [], []
    for it in items:
        rhs = _c128(it["rhs"])
        e_ref = np.ascontiguousarray(it["e_ref"], dtype=np.float64)
        om = np.ascontiguousarray(it["omega"], dtype=np.float64)
        nr, nw = _need_rows(rhs, it["sys"].n_pw, "rhs"), len(om)
        _need_shape(e_ref, (nr,), "e_ref")
        out = it.get("out")
        if out is None:
            out = _like(rhs, (nr, nw, it["sys"].n_pw))
        _need_out(out, (nr, nw, it["sys"].n_pw))
        rep, crep = _report(nr, nw)
        keep += [rhs, e_ref, om, out, crep]
        citems.append(_BatchItem(it["sys"]._h.value, nr, _ptr(rhs), e_ref.ctypes.data, nw, om.ctypes.data, _ptr(out),
                                 ctypes.addressof(crep)))
        outs.append(out)
        reps.append(rep)
    arr = (_BatchItem * len(citems))(*citems)
    st = stream if stream is not None else (_stream_of(outs[0], None) if outs else None)
    opts = _opts(METHOD_LANCZOS, _PREC[precision], 4, -1, int(max_matvec), int(max_refine), int(threads), st,
                 float(cert_tol))
    s = load().sgw_solve_batched(len(citems), ctypes.cast(arr, ctypes.c_void_p), float(eta), float(tol),
                                 ctypes.byref(opts))
    _check(s, allow=() if raise_on_noconv else (SGW_ENOCONV,))
    return outs, reps, s == SGW_OK


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1812_03717_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.sgw_create_system.argtypes = [ctypes.POINTER(_Cell), dp, vp, vp, vp, ctypes.POINTER(_KB), ctypes.POINTER(vp)]
    lib.sgw_get_gvectors.argtypes = [vp, vp, vp, vp]
    lib.sgw_get_box_map.argtypes = [vp, vp]
    lib.sgw_set_split.argtypes = [vp, ip]
    lib.sgw_get_split.argtypes = [vp, vp, vp]
    lib.sgw_solve_capacity.argtypes = [vp, ip, ip, ip, vp]
    lib.sgw_solve_batched.argtypes = [ip, vp, dp, dp, ctypes.POINTER(_Opts)]
    lib.sgw_set_occupied.argtypes = [vp, ip, vp, vp]
    lib.sgw_make_rhs.argtypes = [vp, vp, ip, vp, ip, vp, vp, vp]
    lib.sgw_apply_h.argtypes = [vp, ip, vp, vp, ip, vp]
    lib.sgw_apply_shifted.argtypes = [vp, ip, vp, vp, vp, ip, vp]
    lib.sgw_solve_shifted.argtypes = [vp, ip, vp, vp, ip, vp, dp, dp, ctypes.POINTER(_Opts), vp,
                                      ctypes.POINTER(_Report)]
    lib.sgw_solve_green.argtypes = [vp, ip, vp, ip, vp, dp, ctypes.POINTER(_Opts), vp, ctypes.POINTER(_Report)]
    lib.sgw_density_response.argtypes = [vp, ip, ip, vp, vp, ip, vp, dp, dp, dp, ctypes.POINTER(_Opts), vp,
                                         ctypes.POINTER(_Report)]
    lib.sgw_screened_coulomb.argtypes = [ip, ip, vp, vp, dp, dp, vp, vp, vp]
    lib.sgw_density_response_w.argtypes = [vp, ip, ip, vp, vp, ip, vp, dp, dp, ctypes.POINTER(_Opts), vp,
                                           ctypes.POINTER(_Report)]
    lib.sgw_aaa.argtypes = [ip, ip, vp, vp, dp, ip, ip, vp, vp, vp, vp]
    lib.sgw_residual.argtypes = [vp, ip, vp, vp, ip, vp, dp, vp, vp, vp, vp]
    lib.sgw_residual_noalloc.argtypes = [vp, ip, vp, vp, ip, vp, dp, vp, vp, vp, vp]
    lib.sgw_solve_pershift.argtypes = [vp, ip, vp, vp, vp, dp, dp, ip, vp, vp, ctypes.POINTER(_Opts), vp,
                                       ctypes.POINTER(_Report)]
    lib.sgw_precond_diag.argtypes = [vp, ip, vp, vp, vp, dp, ip, vp, vp, vp, vp]
    lib.sgw_training_rows.argtypes = [vp, ip, vp, vp, vp, dp, vp, vp, vp, vp]
    lib.sgw_mlp_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.sgw_mlp_get_params.argtypes = [vp, vp]
    lib.sgw_mlp_forward.argtypes = [vp, ip, vp, vp, vp]
    lib.sgw_mlp_grad.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp]
    lib.sgw_mlp_train_step.argtypes = [vp, ip, vp, vp, vp, ctypes.c_float, vp, vp]
    lib.sgw_mlp_destroy.argtypes = [vp]
    lib.sgw_mlp_destroy.restype = None
    lib.sgw_destroy_system.argtypes = [vp]
    lib.sgw_destroy_system.restype = None
    lib.sgw_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("sgw_destroy_system", "sgw_last_error", "sgw_mlp_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, allow=()):
    if status != SGW_OK and status not in allow:
        raise SgwError(status, load().sgw_last_error().decode())
    return status


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> int:
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data


def _c128(x):
    if _is_torch(x):
        import torch
        if x.dtype != torch.complex128:
            raise TypeError("complex128 tensor required")
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=np.complex128)


def _like(x, shape):
    if _is_torch(x):
        import torch
        return torch.empty(shape, dtype=torch.complex128, device=x.device)
    return np.empty(shape, dtype=np.complex128)


def _need_shape(x, shape, name):
    """The C ABI sees pointers only: every buffer it reads or writes must have exactly the
    shape the sizes passed beside it describe (a smaller one would be read or written past
    its end on the device)."""
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(x.shape)}")


def _need_out(out, shape, name="out"):
    """A caller's result buffer: complex128 of exactly `shape` (the library writes all of it)."""
    if _is_torch(out):
        import torch
        ok = out.dtype == torch.complex128
    else:
        ok = getattr(out, "dtype", None) == np.complex128
    if not ok:
        raise TypeError(f"{name} must be complex128")
    _need_shape(out, shape, name)


def _need_rows(x, ncols, name):
    """A [rows][ncols] complex128 buffer (already converted by _c128); returns rows."""
    if x.ndim != 2 or x.shape[1] != ncols:
        raise ValueError(f"{name} must be [rows][{ncols}], got shape {tuple(x.shape)}")
    return x.shape[0]


def _stream_of(x, stream):
    if stream is not None:
        return stream
    if _is_torch(x) and x.is_cuda:
        import torch
        return torch.cuda.current_stream(x.device).cuda_stream
    return None


def aaa(z, f, z_eval, tol=1e-13, mmax=32, stream=None):
    """sgw_aaa: AAA approximants of the rows of f (sampled at the points z), evaluated at
    z_eval.  Returns (r [nfun][n_eval] like f, degree [nfun])."""
    zc = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).ravel())
    ze = np.ascontiguousarray(np.asarray(z_eval, dtype=np.complex128).ravel())
    f = _c128(f)
    if f.ndim == 1:
        f = f.reshape(1, -1)
    nfun, m = f.shape
    if m != len(zc):
        raise ValueError("f must be [nfun][len(z)]")
    r = _like(f, (nfun, len(ze)))
    deg = np.zeros(nfun, dtype=np.int32)
    _check(load().sgw_aaa(nfun, m, zc.ctypes.data, _ptr(f), float(tol), int(mmax), len(ze), ze.ctypes.data, _ptr(r),
                          deg.ctypes.data, _stream_of(f, stream)))
    return r, deg


def screened_coulomb(dn, qg, volume, r_cut, want_eps_inv=True, stream=None):
    """sgw_screened_coulomb: (eps_inv or None, wbar), each [n_g][n_g][nomega] like dn (a CUDA
    tensor stays on the device).  qg: [n_g][3] Cartesian q + G (bohr^-1)."""
    dn = _c128(dn)
    qg = np.ascontiguousarray(qg, dtype=np.float64).reshape(-1, 3)
    n, nw = qg.shape[0], (dn.shape[2] if dn.ndim == 3 else 0)
    if tuple(dn.shape[:2]) != (n, n):
        raise ValueError("dn must be [n_g][n_g][nomega] with n_g = len(qg)")
    wbar = _like(dn, tuple(dn.shape))
    einv = _like(dn, tuple(dn.shape)) if want_eps_inv else None
    _check(load().sgw_screened_coulomb(n, nw, _ptr(dn), qg.ctypes.data, float(volume), float(r_cut),
                                       _ptr(einv) if einv is not None else None, _ptr(wbar),
                                       _stream_of(dn, stream)))
    return einv, wbar


class System:
    """One plane-wave basis with its Hamiltonian (sgw_create_system) and occupied states."""

    def __init__(self, a, tau, ecut_ry, k_frac, fft_dims, vloc_r, kb_atom=(), kb_width=(), kb_d=()):
        lib = load()
        cell = _Cell()
        a = np.asarray(a, dtype=np.float64)
        for i in range(3):
            for j in range(3):
                cell.a[i][j] = float(a[i, j])
        self._tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(-1, 3)
        cell.n_atoms = len(self._tau)
        cell.tau = self._tau.ctypes.data
        self._kb_atom = np.ascontiguousarray(kb_atom, dtype=np.int32)
        self._kb_width = np.ascontiguousarray(kb_width, dtype=np.float64)
        self._kb_d = np.ascontiguousarray(kb_d, dtype=np.float64)
        kb = _KB(len(self._kb_atom), self._kb_atom.ctypes.data, self._kb_width.ctypes.data, self._kb_d.ctypes.data)
        k = np.ascontiguousarray(k_frac, dtype=np.float64)
        dims = np.ascontiguousarray(fft_dims, dtype=np.int32)
        v = np.ascontiguousarray(vloc_r, dtype=np.float64)
        if v.size != int(np.prod(dims)):
            raise ValueError("vloc_r size does not match fft_dims")
        h = ctypes.c_void_p()
        _check(lib.sgw_create_system(ctypes.byref(cell), float(ecut_ry), k.ctypes.data, dims.ctypes.data,
                                     v.ctypes.data, ctypes.byref(kb), ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int()
        _check(lib.sgw_get_gvectors(self._h, ctypes.byref(n), None, None))
        self.n_pw = n.value
        self.nocc = 0

    @classmethod
    def from_instance(cls, inst, k_frac):
        return cls(inst.a, inst.tau, inst.ecut_ry, k_frac, inst.fft_dims, inst.vloc_r, inst.kb_atom,
                   inst.kb_width, inst.kb_d)

    def close(self):
        if getattr(self, "_h", None):
            load().sgw_destroy_system(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def gvectors(self):
        mil = np.empty((self.n_pw, 3), dtype=np.int32)
        kin = np.empty(self.n_pw, dtype=np.float64)
        _check(load().sgw_get_gvectors(self._h, None, mil.ctypes.data, kin.ctypes.data))
        return mil, kin

    def box_map(self):
        m = np.empty(self.n_pw, dtype=np.int32)
        _check(load().sgw_get_box_map(self._h, m.ctypes.data))
        return m

    def set_split(self, csize):
        """Forces the cluster size of the on-chip box (0: automatic); returns split()."""
        _check(load().sgw_set_split(self._h, int(csize)))
        return self.split()

    def split(self):
        """(CTAs per vector for FP64 / float-float, for FP32) of the current box split."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().sgw_get_split(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def lanczos_owners(self, nomega, precision="df32", threads=0):
        """Right-hand sides the multishift kernel holds at once (sgw_solve_capacity)."""
        n = ctypes.c_int()
        _check(load().sgw_solve_capacity(self._h, int(nomega), _PREC[precision], int(threads), ctypes.byref(n)))
        return n.value

    def set_occupied(self, psi_v, eps_v):
        psi = _c128(psi_v)
        eps = np.ascontiguousarray(eps_v, dtype=np.float64)
        _need_shape(psi, (len(eps), self.n_pw), "psi_v")
        _check(load().sgw_set_occupied(self._h, len(eps), _ptr(psi), eps.ctypes.data))
        self.nocc = len(eps)

    def make_rhs(self, sys_k, psi_k, gp_miller, out=None, stream=None):
        psi = _c128(psi_k)
        gp = np.ascontiguousarray(gp_miller, dtype=np.int32).reshape(-1, 3)
        n_v = _need_rows(psi, sys_k.n_pw, "psi_k")
        if out is None:
            out = _like(psi, (n_v * len(gp), self.n_pw))
        _need_out(out, (n_v * len(gp), self.n_pw))
        _check(load().sgw_make_rhs(self._h, sys_k._h, n_v, _ptr(psi), len(gp), gp.ctypes.data, _ptr(out),
                                   _stream_of(psi, stream)))
        return out

    def apply_h(self, x, out=None, precision="fp64", stream=None):
        x = _c128(x)
        if x.ndim not in (1, 2) or x.shape[-1] != self.n_pw:
            raise ValueError(f"x must be [nvec][{self.n_pw}] or [{self.n_pw}], got shape {tuple(x.shape)}")
        nvec = x.shape[0] if x.ndim == 2 else 1
        if out is None:
            out = _like(x, x.shape)
        _need_out(out, x.shape)
        _check(load().sgw_apply_h(self._h, nvec, _ptr(x), _ptr(out), _PREC[precision], _stream_of(x, stream)))
        return out

    def apply_shifted(self, x, z, out=None, precision="fp64", stream=None):
        x = _c128(x)
        if x.ndim not in (1, 2) or x.shape[-1] != self.n_pw:
            raise ValueError(f"x must be [nvec][{self.n_pw}] or [{self.n_pw}], got shape {tuple(x.shape)}")
        nvec = x.shape[0] if x.ndim == 2 else 1
        zz = np.ascontiguousarray(np.broadcast_to(np.asarray(z, dtype=np.complex128), (nvec,)))
        if out is None:
            out = _like(x, x.shape)
        _need_out(out, x.shape)
        _check(load().sgw_apply_shifted(self._h, nvec, _ptr(x), zz.ctypes.data, _ptr(out), _PREC[precision],
                                        _stream_of(x, stream)))
        return out

    def solve_shifted(self, rhs, e_ref, omega, eta, tol=1e-10, method="lanczos", precision="fp64", ell=4, seed_index=-1, max_matvec=0,
                      max_refine=0, threads=0, out=None, stream=None, raise_on_noconv=False, cert_tol=0.0, x0=None,
                      precond="none", mlp=None, plain_budget=0):
        """Returns (dpsi [nrhs][nomega][n_pw], report dict, converged flag).  cert_tol: certificate
        target (0: the library default 1e-8, negative: not checked); x0: initial solutions like
        dpsi (resume); precond: "none" / "plain" / "learned" for the per-shift corrections."""
        rhs = _c128(rhs)
        nrhs = _need_rows(rhs, self.n_pw, "rhs")
        e_ref = np.ascontiguousarray(e_ref, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        _need_shape(e_ref, (nrhs,), "e_ref")
        nw = len(omega)
        if out is None:
            out = _like(rhs, (nrhs, nw, self.n_pw))
        _need_out(out, (nrhs, nw, self.n_pw))
        if x0 is not None:
            x0 = _c128(x0)
            if tuple(x0.shape) != (nrhs, nw, self.n_pw):
                raise ValueError("x0 must be [nrhs][nomega][n_pw]")
        rep, crep = _report(nrhs, nw)
        m = {"lanczos": METHOD_LANCZOS, "bicgstab": METHOD_BICGSTAB}[method]
        opts = _opts(m, _PREC[precision], int(ell), int(seed_index), int(max_matvec), int(max_refine), int(threads),
                     _stream_of(rhs, stream), float(cert_tol), _ptr(x0) if x0 is not None else None,
                     _PRECOND[precond], mlp._h if mlp is not None else None, int(plain_budget))
        s = load().sgw_solve_shifted(self._h, nrhs, _ptr(rhs), e_ref.ctypes.data, nw, omega.ctypes.data,
                                     float(eta), float(tol), ctypes.byref(opts), _ptr(out), ctypes.byref(crep))
        _check(s, allow=() if raise_on_noconv else (SGW_ENOCONV,))
        return out, rep, s == SGW_OK

    def solve_green(self, cols, z, tol=1e-10, precision="fp64", max_matvec=0, max_refine=0, threads=0, out=None,
                    device=None, stream=None, raise_on_noconv=False, cert_tol=0.0):
        """Columns cols of G(z_j) = (z_j - H)^-1 (sgw_solve_green): returns (g [ncol][nz][n_pw], report
        dict, converged flag).  z: complex shifts with Im z != 0.  The result is a CUDA tensor when
        out is one or device is "cuda", else a numpy array."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        zc = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).ravel())
        zz = np.ascontiguousarray(np.column_stack([zc.real, zc.imag]))
        nc, nz = len(cols), len(zc)
        if out is None:
            if device is not None and str(device).startswith("cuda"):
                import torch
                out = torch.empty((nc, nz, self.n_pw), dtype=torch.complex128, device=device)
            else:
                out = np.empty((nc, nz, self.n_pw), dtype=np.complex128)
        _need_out(out, (nc, nz, self.n_pw))
        rep, crep = _report(nc, nz)
        opts = _opts(METHOD_LANCZOS, _PREC[precision], 4, -1, int(max_matvec), int(max_refine), int(threads),
                     _stream_of(out, stream), float(cert_tol))
        s = load().sgw_solve_green(self._h, nc, cols.ctypes.data, nz, zz.ctypes.data, float(tol), ctypes.byref(opts),
                                   _ptr(out), ctypes.byref(crep))
        _check(s, allow=() if raise_on_noconv else (SGW_ENOCONV,))
        return out, rep, s == SGW_OK

    def density_response(self, rhs, eps_v, omega, eta, weight=1.0, tol=1e-10, precision="fp64", max_matvec=0,
                         max_refine=0, threads=0, out=None, stream=None, raise_on_noconv=False, cert_tol=0.0):
        """One k-point's contribution to Eq. 5 (sgw_density_response): rhs [n_v * n_pert][n_pw] from
        make_rhs, eps_v [n_v].  Accumulates into out [n_pert][n_pert][nomega] (zeros when None; a
        CUDA tensor stays on the device) and returns (out, report [n_v * n_pert][2 nomega], converged)."""
        rhs = _c128(rhs)
        eps_v = np.ascontiguousarray(eps_v, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        n_v = len(eps_v)
        nr = _need_rows(rhs, self.n_pw, "rhs")
        if n_v == 0 or nr % n_v:
            raise ValueError("rhs rows must be n_v * n_pert")
        n_p, nw = nr // n_v, len(omega)
        if out is None:
            if _is_torch(rhs):
                import torch
                out = torch.zeros((n_p, n_p, nw), dtype=torch.complex128, device=rhs.device)
            else:
                out = np.zeros((n_p, n_p, nw), dtype=np.complex128)
        _need_out(out, (n_p, n_p, nw))
        rep, crep = _report(nr, 2 * nw)
        opts = _opts(METHOD_LANCZOS, _PREC[precision], 4, -1, int(max_matvec), int(max_refine), int(threads),
                     _stream_of(rhs, stream), float(cert_tol))
        s = load().sgw_density_response(self._h, n_v, n_p, _ptr(rhs), eps_v.ctypes.data, nw, omega.ctypes.data,
                                        float(eta), float(weight), float(tol), ctypes.byref(opts), _ptr(out),
                                        ctypes.byref(crep))
        _check(s, allow=() if raise_on_noconv else (SGW_ENOCONV,))
        return out, rep, s == SGW_OK

    def density_response_w(self, rhs, eps_v, w, weight=1.0, tol=1e-10, precision="fp64", max_matvec=0,
                           max_refine=0, threads=0, out=None, stream=None, raise_on_noconv=False, cert_tol=0.0):
        """sgw_density_response_w: as density_response at complex frequencies w (w = 1j * omega on
        the imaginary axis); returns (dn [n_pert][n_pert][nw], report, converged)."""
        rhs = _c128(rhs)
        eps_v = np.ascontiguousarray(eps_v, dtype=np.float64)
        wc = np.asarray(w, dtype=np.complex128).ravel()
        ww = np.ascontiguousarray(np.column_stack([wc.real, wc.imag]))
        n_v = len(eps_v)
        nr = _need_rows(rhs, self.n_pw, "rhs")
        if n_v == 0 or nr % n_v:
            raise ValueError("rhs rows must be n_v * n_pert")
        n_p, nw = nr // n_v, len(wc)
        if out is None:
            if _is_torch(rhs):
                import torch
                out = torch.zeros((n_p, n_p, nw), dtype=torch.complex128, device=rhs.device)
            else:
                out = np.zeros((n_p, n_p, nw), dtype=np.complex128)
        _need_out(out, (n_p, n_p, nw))
        rep, crep = _report(nr, 2 * nw)
        opts = _opts(METHOD_LANCZOS, _PREC[precision], 4, -1, int(max_matvec), int(max_refine), int(threads),
                     _stream_of(rhs, stream), float(cert_tol))
        s = load().sgw_density_response_w(self._h, n_v, n_p, _ptr(rhs), eps_v.ctypes.data, nw, ww.ctypes.data,
                                          float(weight), float(tol), ctypes.byref(opts), _ptr(out), ctypes.byref(crep))
        _check(s, allow=() if raise_on_noconv else (SGW_ENOCONV,))
        return out, rep, s == SGW_OK

    def residual(self, rhs, e_ref, omega, eta, dpsi, stream=None):
        rhs = _c128(rhs)
        dpsi = _c128(dpsi)
        e_ref = np.ascontiguousarray(e_ref, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        nrhs, nw = _need_rows(rhs, self.n_pw, "rhs"), len(omega)
        _need_shape(e_ref, (nrhs,), "e_ref")
        _need_shape(dpsi, (nrhs, nw, self.n_pw), "dpsi")
        rel = np.zeros((nrhs, nw))
        cert = np.zeros((nrhs, nw))
        _check(load().sgw_residual(self._h, nrhs, _ptr(rhs), e_ref.ctypes.data, nw, omega.ctypes.data, float(eta),
                                   _ptr(dpsi), rel.ctypes.data, cert.ctypes.data, _stream_of(rhs, stream)))
        return rel, cert

    def residual_noalloc(self, rhs, e_ref, omega, eta, dpsi, rel_res, cert, stream=None):
        """sgw_residual_noalloc: every argument a CUDA tensor (float64 e_ref / omega / rel_res /
        cert, complex128 rhs / dpsi); writes rel_res and cert on the device; allocates nothing."""
        import torch
        for t in (rhs, e_ref, omega, dpsi, rel_res, cert):
            if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
                raise ValueError("residual_noalloc takes contiguous CUDA tensors only")
        dev = rhs.device
        if any(t.device != dev for t in (e_ref, omega, dpsi, rel_res, cert)):
            raise ValueError("residual_noalloc: every tensor must be on the same device")
        for t, dt, name in ((rhs, torch.complex128, "rhs"), (dpsi, torch.complex128, "dpsi"),
                            (e_ref, torch.float64, "e_ref"), (omega, torch.float64, "omega"),
                            (rel_res, torch.float64, "rel_res"), (cert, torch.float64, "cert")):
            if t.dtype != dt:
                raise TypeError(f"residual_noalloc: {name} must be {dt}")
        if rhs.ndim != 2 or rhs.shape[1] != self.n_pw:
            raise ValueError("residual_noalloc: rhs must be [nrhs][n_pw]")
        nrhs, nw = rhs.shape[0], omega.numel()
        if omega.ndim != 1 or e_ref.shape != (nrhs,):
            raise ValueError("residual_noalloc: omega must be [nomega], e_ref [nrhs]")
        if tuple(dpsi.shape) != (nrhs, nw, self.n_pw):
            raise ValueError("residual_noalloc: dpsi must be [nrhs][nomega][n_pw]")
        if tuple(rel_res.shape) != (nrhs, nw) or tuple(cert.shape) != (nrhs, nw):
            raise ValueError("residual_noalloc: rel_res and cert must be [nrhs][nomega]")
        _check(load().sgw_residual_noalloc(self._h, nrhs, rhs.data_ptr(), e_ref.data_ptr(), nw, omega.data_ptr(),
                                           float(eta), dpsi.data_ptr(), rel_res.data_ptr(), cert.data_ptr(),
                                           _stream_of(rhs, stream)))

    def solve_pershift(self, rhs, e_ref, omega, eta, tol=1e-10, precond="plain", delta=None, mlp=None, ell=4,
                       max_matvec=0, out=None, stream=None):
        """Independent single-shift solves of pairs (rhs[i], z_i = e_ref[i] + omega[i] + i eta) with a
        diagonal preconditioner; returns (x [npairs][n_pw], report, converged)."""
        rhs = _c128(rhs)
        n = _need_rows(rhs, self.n_pw, "rhs")
        e_ref = np.ascontiguousarray(e_ref, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        _need_shape(e_ref, (n,), "e_ref")
        _need_shape(omega, (n,), "omega")
        dl = None if delta is None else np.ascontiguousarray(np.broadcast_to(delta, (n,)), dtype=np.float64)
        if out is None:
            out = _like(rhs, (n, self.n_pw))
        _need_out(out, (n, self.n_pw))
        rep, crep = _report(n, None)
        opts = _opts(METHOD_BICGSTAB, PREC_FP64, int(ell), -1, int(max_matvec), -1, 0, _stream_of(rhs, stream))
        st = load().sgw_solve_pershift(self._h, n, _ptr(rhs), e_ref.ctypes.data, omega.ctypes.data, float(eta),
                                       float(tol), _PRECOND[precond], dl.ctypes.data if dl is not None else None,
                                       mlp._h if mlp is not None else None, ctypes.byref(opts), _ptr(out),
                                       ctypes.byref(crep))
        _check(st, allow=(SGW_ENOCONV,))
        return out, rep, st == SGW_OK

    def precond_diag(self, rhs, e_ref, omega, eta, precond="plain", delta=None, mlp=None):
        rhs = _c128(rhs)
        n = _need_rows(rhs, self.n_pw, "rhs")
        d = np.empty((n, self.n_pw))
        e_ref = np.ascontiguousarray(e_ref, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        _need_shape(e_ref, (n,), "e_ref")
        _need_shape(omega, (n,), "omega")
        dl = None if delta is None else np.ascontiguousarray(np.broadcast_to(delta, (n,)), dtype=np.float64)
        _check(load().sgw_precond_diag(self._h, n, _ptr(rhs), e_ref.ctypes.data, omega.ctypes.data, float(eta),
                                       _PRECOND[precond], dl.ctypes.data if dl is not None else None,
                                       mlp._h if mlp is not None else None, d.ctypes.data, _stream_of(rhs, None)))
        return d

    def training_rows(self, rhs, e_ref, omega, eta, delta):
        """(feats [n*n_pw][4], targets [n*n_pw]) float32 CUDA tensors; rhs a CUDA tensor."""
        import torch
        if not (_is_torch(rhs) and rhs.is_cuda and rhs.is_contiguous() and rhs.dtype == torch.complex128):
            raise TypeError("training_rows takes a contiguous complex128 CUDA tensor rhs")
        n = _need_rows(rhs, self.n_pw, "rhs")
        rows = n * self.n_pw
        feats = torch.empty((rows, 4), dtype=torch.float32, device=rhs.device)
        targets = torch.empty(rows, dtype=torch.float32, device=rhs.device)
        e_ref = np.ascontiguousarray(e_ref, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        _need_shape(e_ref, (n,), "e_ref")
        _need_shape(omega, (n,), "omega")
        dl = np.ascontiguousarray(np.broadcast_to(delta, (n,)), dtype=np.float64)
        _check(load().sgw_training_rows(self._h, n, rhs.data_ptr(), e_ref.ctypes.data, omega.ctypes.data, float(eta),
                                        dl.ctypes.data, feats.data_ptr(), targets.data_ptr(), _stream_of(rhs, None)))
        return feats, targets


class MLP:
    """The learned preconditioner's perceptron (sgw_mlp); rows are float32 CUDA tensors."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_PARAMS:
            raise ValueError("expected 4545 parameters")
        h = ctypes.c_void_p()
        _check(load().sgw_mlp_create(p.ctypes.data, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().sgw_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self):
        p = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(load().sgw_mlp_get_params(self._h, p.ctypes.data))
        return p

    def forward(self, feats):
        import torch
        out = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
        _check(load().sgw_mlp_forward(self._h, feats.shape[0], feats.data_ptr(), out.data_ptr(),
                                      _stream_of(feats, None)))
        return out

    def grad(self, feats, targets, weight=None):
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(load().sgw_mlp_grad(self._h, feats.shape[0], feats.data_ptr(), targets.data_ptr(),
                                   weight.data_ptr() if weight is not None else None, g.ctypes.data,
                                   loss.ctypes.data, _stream_of(feats, None)))
        return float(loss[0]), g

    def train_step(self, feats, targets, weight=None, lr=1e-3):
        loss = np.zeros(1, dtype=np.float32)
        _check(load().sgw_mlp_train_step(self._h, feats.shape[0], feats.data_ptr(), targets.data_ptr(),
                                         weight.data_ptr() if weight is not None else None, float(lr),
                                         loss.ctypes.data, _stream_of(feats, None)))
        return float(loss[0])
