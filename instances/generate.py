"""Seeded synthetic instances of the shifted Sternheimer problem (SternheimerGW, Sec. 2.1-2.3).

This module is the one input generator that both the CUDA path and the CPU oracle consume.
It builds what the method takes as *given*:

* the crystal (lattice rows a_i in bohr, atom positions), the cutoff and the FFT box;
* the local potential sampled on the FFT box, V_loc(r_j) (a real array: what the
  library receives), made of one Gaussian v(r) = A exp(-r^2 / (2 sigma^2)) per atom with
  A = -4 Ha, sigma = 0.9 bohr, band-limited to |G|^2 <= 4 E_cut;
* one s-type Gaussian Kleinman-Bylander projector per atom (width 0.9 bohr, D = +1 Ha);
* k-points, q, the perturbation wave vectors G_p, the frequencies omega_j and eta;
* the Kohn-Sham ground state (occupied psi_v and eps_v at k and at k+q).  In the paper
  this comes from a DFT code (Sec. 2.1); here a dense FP64 diagonalisation of the
  synthetic Hamiltonian stands in for that code.  It uses the closed-form Fourier
  coefficients of the potential, not the sampled box, so it is a different numerical
  route from the one the oracle and the CUDA path take.

Units: Hartree atomic units (energy Ha, length bohr); E_cut is given in Ry, so the
plane-wave sphere is |k+G|^2 <= E_cut[Ry] in bohr^-2.  Random draws use numpy's PCG64
(``numpy.random.default_rng(seed)``); the draw order is documented at each config.

The G-sphere enumeration below follows the library's documented canonical order
(Miller triples lexicographic, m1 outermost, each ascending) and its documented FP64
membership test, so that coefficient arrays line up between producer and consumers.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.linalg

HA_EV = 27.211386245988          # eV per Hartree (CODATA 2018)
VLOC_DEPTH = -4.0                # Ha
VLOC_SIGMA = 0.9                 # bohr
KB_WIDTH = 0.9                   # bohr
KB_D = 1.0                       # Ha
BOUNDARY_MARGIN = 1e-10          # relative distance from the sphere surface no G may have


@dataclass
class KPointData:
    k_frac: np.ndarray                # Bloch vector of the unperturbed states (fractional, of B)
    kq_frac: np.ndarray               # k+q: basis the response lives in
    miller_k: np.ndarray              # int32 [npw_k][3]
    miller_kq: np.ndarray             # int32 [npw_kq][3]
    psi_k: np.ndarray                 # c128 [n_occ][npw_k]
    eps_k: np.ndarray                 # f64 [n_occ]
    psi_kq: np.ndarray                # c128 [n_occ][npw_kq]
    eps_kq: np.ndarray                # f64 [n_occ]
    gap_k: float = 0.0
    gap_kq: float = 0.0


@dataclass
class Instance:
    name: str
    seed: int
    a: np.ndarray                     # [3][3], rows = lattice vectors, bohr
    tau: np.ndarray                   # [n_atoms][3] cartesian bohr
    ecut_ry: float
    fft_dims: tuple
    vloc_r: np.ndarray                # f64 [N1][N2][N3] (C order), Ha
    kb_atom: np.ndarray               # int32 [n_proj]
    kb_width: np.ndarray              # f64 [n_proj]
    kb_d: np.ndarray                  # f64 [n_proj]
    n_occ: int
    gp_miller: np.ndarray             # int32 [n_pert][3]
    omega: np.ndarray                 # f64 [n_omega], Ha
    eta: float                        # Ha
    kpoints: list = field(default_factory=list)

    @property
    def n_pert(self) -> int:
        return len(self.gp_miller)

    @property
    def volume(self) -> float:
        return abs(float(np.linalg.det(self.a)))

    def e_ref(self, ik: int) -> np.ndarray:
        """eps_{v,k} for each right-hand side r = v * n_pert + p of k-point ik."""
        return np.repeat(self.kpoints[ik].eps_k, self.n_pert)


# ----------------------------------------------------------------------------- lattice

def recip(a: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(np.asarray(a, dtype=np.float64)).T


def _kcart(k_frac, b):
    k = np.asarray(k_frac, dtype=np.float64)
    return (k[0] * b[0] + k[1] * b[1]) + k[2] * b[2]


def sphere(a, k_frac, ecut_ry, check_margin=True):
    """Canonical plane-wave sphere {m : |k + m.B|^2 <= ecut}; returns (miller int32, |k+G|^2)."""
    b = recip(a)
    kc = _kcart(k_frac, b)
    amax = np.linalg.norm(a, axis=1)
    kf = np.abs(np.asarray(k_frac, dtype=np.float64))
    bound = [int(math.floor(math.sqrt(ecut_ry) * amax[i] / (2 * math.pi) + kf[i])) + 1 for i in range(3)]
    r = [np.arange(-bound[i], bound[i] + 1) for i in range(3)]
    m1, m2, m3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    m1 = m1.ravel().astype(np.float64)
    m2 = m2.ravel().astype(np.float64)
    m3 = m3.ravel().astype(np.float64)
    g = [((kc[x] + m1 * b[0, x]) + m2 * b[1, x]) + m3 * b[2, x] for x in range(3)]
    n2 = (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]
    near = np.abs(n2 - ecut_ry) < BOUNDARY_MARGIN * ecut_ry
    if check_margin and np.any(near):
        raise ValueError("a plane wave lies within the boundary margin of the cutoff sphere")
    keep = n2 <= ecut_ry
    mil = np.stack([m1[keep], m2[keep], m3[keep]], axis=1).astype(np.int32)
    return mil, n2[keep]


# ------------------------------------------------------------------ synthetic potential

def vloc_coeffs(a, tau, mil):
    """Closed-form Fourier coefficients V(G) of the periodic sum of atomic Gaussians."""
    b = recip(a)
    omega_cell = abs(np.linalg.det(a))
    g = mil.astype(np.float64) @ b
    g2 = np.einsum("ij,ij->i", g, g)
    pref = VLOC_DEPTH * (2 * math.pi * VLOC_SIGMA ** 2) ** 1.5 / omega_cell
    sf = np.exp(-1j * (g @ np.asarray(tau).T)).sum(axis=1)
    return pref * np.exp(-0.5 * VLOC_SIGMA ** 2 * g2) * sf


def vloc_box(a, tau, ecut_ry, dims):
    """V_loc(r_j) on the box, r_j = sum_i (j_i / N_i) a_i; V(G) kept for |G|^2 <= 4 E_cut."""
    mil, _ = sphere(a, (0.0, 0.0, 0.0), 4.0 * ecut_ry, check_margin=False)
    for i in range(3):
        if dims[i] < 2 * int(np.abs(mil[:, i]).max()) + 1:
            raise ValueError("FFT box too small for the band-limited potential")
    vg = vloc_coeffs(a, tau, mil)
    box = np.zeros(dims, dtype=np.complex128)
    idx = tuple(np.mod(mil[:, i], dims[i]) for i in range(3))
    box[idx] = vg
    vr = np.fft.ifftn(box) * (dims[0] * dims[1] * dims[2])
    if np.abs(vr.imag).max() > 1e-12 * max(1.0, np.abs(vr.real).max()):
        raise AssertionError("potential is not real")
    return np.ascontiguousarray(vr.real)


def kb_coeffs(a, tau, k_frac, mil, width):
    """<k+G|beta_a> for s-type Gaussian projectors, one per atom: [n_atoms][npw]."""
    b = recip(a)
    omega_cell = abs(np.linalg.det(a))
    kg = mil.astype(np.float64) @ b + _kcart(k_frac, b)
    kg2 = np.einsum("ij,ij->i", kg, kg)
    out = []
    for ia, t in enumerate(np.asarray(tau)):
        w = width[ia]
        amp = omega_cell ** -0.5 * (4 * math.pi * w * w) ** 0.75 * np.exp(-0.5 * w * w * kg2)
        out.append(amp * np.exp(-1j * (kg @ t)))
    return np.array(out)


def closed_form_h(inst: Instance, k_frac):
    """Dense H in the k sphere from the closed-form V(G - G') (kept for |G - G'|^2 <= 4 E_cut),
    T_G and the KB projectors: the generator's own route to the ground state.  V is tabulated
    once on the grid of Miller differences and gathered row block by row block."""
    mil, n2 = sphere(inst.a, k_frac, inst.ecut_ry)
    b = recip(inst.a)
    n = len(mil)
    lo = (mil.min(axis=0) - mil.max(axis=0)).astype(np.int64)      # smallest difference per axis
    ext = (2 * (mil.max(axis=0) - mil.min(axis=0)) + 1).astype(np.int64)
    grid = np.stack(np.meshgrid(*[np.arange(lo[i], lo[i] + ext[i]) for i in range(3)], indexing="ij"),
                    axis=-1).reshape(-1, 3)
    g2 = np.einsum("ij,ij->i", grid @ b, grid @ b)
    keep = g2 <= 4.0 * inst.ecut_ry * (1 + 1e-12)
    vtab = np.zeros(len(grid), dtype=np.complex128)
    vtab[keep] = vloc_coeffs(inst.a, inst.tau, grid[keep])
    m = mil.astype(np.int64) - lo[None, :]
    h = np.empty((n, n), dtype=np.complex128)
    for r0 in range(0, n, 1024):
        r1 = min(n, r0 + 1024)
        d = m[r0:r1, None, :] - mil.astype(np.int64)[None, :, :]
        h[r0:r1] = vtab[(d[..., 0] * ext[1] + d[..., 1]) * ext[2] + d[..., 2]]
    h[np.diag_indices(n)] += 0.5 * n2
    beta = kb_coeffs(inst.a, inst.tau, k_frac, mil, inst.kb_width)[inst.kb_atom]
    h += (beta.T * inst.kb_d[None, :]) @ beta.conj()
    h = 0.5 * (h + h.conj().T)
    return mil, h


def _lowest_eigenpairs(h, count):
    """The `count` lowest eigenpairs of the Hermitian h.  Large matrices go to the GPU's dense
    eigensolver (cuSOLVER through torch) when one is present, else LAPACK's subset driver; each
    eigenvector's phase is fixed (its largest component real and positive)."""
    w = v = None
    if h.shape[0] > 6000:
        try:
            import torch
            if torch.cuda.is_available():
                t = torch.from_numpy(h).cuda()
                wt, vt = torch.linalg.eigh(t)
                w = wt[:count].cpu().numpy()
                v = vt[:, :count].cpu().numpy()
                del t, wt, vt
                torch.cuda.empty_cache()
        except ImportError:
            pass
    if w is None:
        w, v = scipy.linalg.eigh(h, subset_by_index=[0, count - 1])
    big = np.argmax(np.abs(v), axis=0)
    ph = v[big, np.arange(v.shape[1])]
    v = v * (np.abs(ph) / ph)[None, :]
    return w, v


def ground_state(inst: Instance, k_frac, n_bands: int):
    """Lowest n_bands eigenpairs of the synthetic Hamiltonian at k (stand-in for the DFT input)."""
    mil, h = closed_form_h(inst, k_frac)
    w, v = _lowest_eigenpairs(h, n_bands + 1)
    del h
    return mil, np.ascontiguousarray(v[:, :n_bands].T), w[:n_bands], float(w[n_bands] - w[n_bands - 1])


# ------------------------------------------------------------------------ perturbations

def shortest_g(a, count, include_zero=True):
    """The `count` shortest G, ranked by |G|^2, ties broken by the Miller triple ascending."""
    b = recip(a)
    rng_m = 4
    while True:
        r = np.arange(-rng_m, rng_m + 1)
        m = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
        if not include_zero:
            m = m[np.any(m != 0, axis=1)]
        g = m.astype(np.float64) @ b
        g2 = np.round(np.einsum("ij,ij->i", g, g), 10)
        order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], g2))
        sel = m[order[:count]]
        if np.abs(sel).max() < rng_m:
            return sel.astype(np.int32)
        rng_m *= 2


# ------------------------------------------------------------------------------ configs

def fcc_cell(alat):
    a = np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]) * alat
    tau = np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]]) * alat
    return a, tau


DIAMOND_FRAC = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                         [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])


def cubic8_cell(alat):
    return np.eye(3) * alat, DIAMOND_FRAC * alat


def make_instance(name, seed, a, tau, ecut_ry, dims, n_occ, kq_pairs, gp, omega, eta, cache=False):
    if cache:
        inst = _cache_load(name, seed)
        if inst is not None:
            return inst
    n_at = len(tau)
    inst = Instance(name=name, seed=seed, a=np.asarray(a, float), tau=np.asarray(tau, float),
                    ecut_ry=float(ecut_ry), fft_dims=tuple(int(x) for x in dims),
                    vloc_r=vloc_box(a, tau, ecut_ry, dims),
                    kb_atom=np.arange(n_at, dtype=np.int32),
                    kb_width=np.full(n_at, KB_WIDTH), kb_d=np.full(n_at, KB_D),
                    n_occ=int(n_occ), gp_miller=np.asarray(gp, np.int32),
                    omega=np.asarray(omega, float), eta=float(eta))
    for k, kq in kq_pairs:
        mk, pk, ek, gk = ground_state(inst, k, n_occ)
        if np.array_equal(np.asarray(k, float), np.asarray(kq, float)):
            mq, pq, eq, gq = mk, pk, ek, gk          # q = 0: one basis
        else:
            mq, pq, eq, gq = ground_state(inst, kq, n_occ)
        inst.kpoints.append(KPointData(k_frac=np.asarray(k, float), kq_frac=np.asarray(kq, float),
                                       miller_k=mk, miller_kq=mq, psi_k=pk, eps_k=ek,
                                       psi_kq=pq, eps_kq=eq, gap_k=gk, gap_kq=gq))
    if cache:
        _cache_store(inst)
    return inst


# ---------------------------------------------------------------- on-disk instance cache
#
# The large instances take minutes to diagonalise; their arrays are kept in
# $SGW_INSTANCE_CACHE (default: <tmp>/sgw_instances) under the instance name and seed, so that
# the processes of one session (tests, benchmark) generate each only once.

_CACHE_VERSION = 1


def _cache_path(name, seed):
    import os
    import tempfile
    d = os.environ.get("SGW_INSTANCE_CACHE") or os.path.join(tempfile.gettempdir(), "sgw_instances")
    return os.path.join(d, f"{name}-seed{seed}-v{_CACHE_VERSION}.npz")


def _cache_store(inst):
    import os
    path = _cache_path(inst.name, inst.seed)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    arrays = {"a": inst.a, "tau": inst.tau, "ecut_ry": inst.ecut_ry, "fft_dims": np.asarray(inst.fft_dims),
              "vloc_r": inst.vloc_r, "kb_atom": inst.kb_atom, "kb_width": inst.kb_width, "kb_d": inst.kb_d,
              "n_occ": inst.n_occ, "gp_miller": inst.gp_miller, "omega": inst.omega, "eta": inst.eta,
              "nk": len(inst.kpoints)}
    for i, kp in enumerate(inst.kpoints):
        for f in ("k_frac", "kq_frac", "miller_k", "miller_kq", "psi_k", "eps_k", "psi_kq", "eps_kq", "gap_k",
                  "gap_kq"):
            arrays[f"k{i}_{f}"] = getattr(kp, f)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def _cache_load(name, seed):
    import os
    path = _cache_path(name, seed)
    if not os.path.exists(path):
        return None
    z = np.load(path)
    inst = Instance(name=name, seed=seed, a=z["a"], tau=z["tau"], ecut_ry=float(z["ecut_ry"]),
                    fft_dims=tuple(int(x) for x in z["fft_dims"]), vloc_r=z["vloc_r"], kb_atom=z["kb_atom"],
                    kb_width=z["kb_width"], kb_d=z["kb_d"], n_occ=int(z["n_occ"]), gp_miller=z["gp_miller"],
                    omega=z["omega"], eta=float(z["eta"]))
    for i in range(int(z["nk"])):
        g = lambda f: z[f"k{i}_{f}"]
        inst.kpoints.append(KPointData(k_frac=g("k_frac"), kq_frac=g("kq_frac"), miller_k=g("miller_k"),
                                       miller_kq=g("miller_kq"), psi_k=g("psi_k"), eps_k=g("eps_k"),
                                       psi_kq=g("psi_kq"), eps_kq=g("eps_kq"), gap_k=float(g("gap_k")),
                                       gap_kq=float(g("gap_kq"))))
    return inst


def _frac_of_cart(a, v_cart):
    """Fractional coordinates (of B) of a cartesian reciprocal-space vector."""
    return np.asarray(v_cart, float) @ np.asarray(a, float).T / (2 * math.pi)


def config1(seed: int = 0, ecut_ry: float = 10.0, dims=(16, 16, 16), n_occ: int = 4,
            n_pert: int = 8, n_omega: int = 16):
    """fcc Si-like cell a = 10.26 bohr, k = Gamma, q = (0.1,0,0) 2pi/a, 8 shortest G,
    omega = linspace(0, 50 eV, 16), eta = 0.1 eV.  No random draws (seed is recorded only)."""
    alat = 10.26
    a, tau = fcc_cell(alat)
    q = _frac_of_cart(a, np.array([0.1, 0.0, 0.0]) * 2 * math.pi / alat)
    k = np.zeros(3)
    omega = np.linspace(0.0, 50.0, n_omega) / HA_EV
    return make_instance("fcc2-ecut%g" % ecut_ry, seed, a, tau, ecut_ry, dims, n_occ,
                         [(k, k + q)], shortest_g(a, n_pert, True), omega, 0.1 / HA_EV)


def tiny_fcc(ecut_ry: float = 4.0, dims=(12, 12, 12), n_occ: int = 4, n_pert: int = 3,
             n_omega: int = 5, q_cart=(0.1, 0.0, 0.0)):
    """Small-basis variant of config1 for brute-force checks (tens of plane waves)."""
    alat = 10.26
    a, tau = fcc_cell(alat)
    q = _frac_of_cart(a, np.asarray(q_cart) * 2 * math.pi / alat)
    omega = np.linspace(0.0, 50.0, n_omega) / HA_EV
    return make_instance("tiny-fcc-ecut%g" % ecut_ry, 0, a, tau, ecut_ry, dims, n_occ,
                         [(np.zeros(3), q)], shortest_g(a, n_pert, True), omega, 0.1 / HA_EV)


def config2(seed: int = 0, n_k: int = 4, ecut_ry: float = 20.0, dims=(36, 36, 36),
            n_occ: int = 16, n_pert: int = 32, n_omega: int = 64, k_subset=None):
    """8-atom cubic diamond cell a = 10.26 bohr, ecut 20 Ry, 36^3 box, 16 occupied bands,
    32 shortest G, omega = linspace(0, 60 eV, 64), eta = 0.1 eV.
    Draws: rng = default_rng(seed); k = rng.uniform(-1/2, 1/2, (n_k, 3)) then
    q = rng.uniform(-1/2, 1/2, 3), all fractional coordinates of B."""
    alat = 10.26
    a, tau = cubic8_cell(alat)
    rng = np.random.default_rng(seed)
    ks = rng.uniform(-0.5, 0.5, size=(n_k, 3))
    q = rng.uniform(-0.5, 0.5, size=3)
    pairs = [(k, k + q) for k in ks]
    if k_subset is not None:
        pairs = [pairs[i] for i in k_subset]
    omega = np.linspace(0.0, 60.0, n_omega) / HA_EV
    return make_instance("cubic8-ecut%g" % ecut_ry, seed, a, tau, ecut_ry, dims, n_occ,
                         pairs, shortest_g(a, n_pert, True), omega, 0.1 / HA_EV)


def fcc_perturbed(seed: int, ecut_ry: float = 10.0, dims=(16, 16, 16), n_occ: int = 4, n_pert: int = 8,
                  n_omega: int = 16):
    """Config-1 cell with seeded disorder, for training the learned preconditioner.
    Draws: rng = default_rng(seed); atom displacements N(0, 0.05 bohr) (2 x 3), then k uniform
    in [-1/2, 1/2)^3 (fractional); q = (0.1, 0, 0) 2pi/a, 8 shortest G, omega in [0, 50] eV."""
    alat = 10.26
    a, tau = fcc_cell(alat)
    rng = np.random.default_rng(seed)
    tau = tau + rng.normal(0.0, 0.05, size=tau.shape)
    k = rng.uniform(-0.5, 0.5, size=3)
    q = _frac_of_cart(a, np.array([0.1, 0.0, 0.0]) * 2 * math.pi / alat)
    omega = np.linspace(0.0, 50.0, n_omega) / HA_EV
    return make_instance("fcc2-disordered-%d" % seed, seed, a, tau, ecut_ry, dims, n_occ,
                         [(k, k + q)], shortest_g(a, n_pert, True), omega, 0.1 / HA_EV)


def supercell64_cell(alat=10.26):
    """2 x 2 x 2 supercell of the 8-atom cubic diamond cell: cube of side 2 alat, 64 sites."""
    sites = np.array([(np.array([i, j, k]) + f) / 2.0 for i in (0, 1) for j in (0, 1) for k in (0, 1)
                      for f in DIAMOND_FRAC])
    return np.eye(3) * (2 * alat), sites * (2 * alat)


def config3(seed: int = 0, ecut_ry: float = 25.0, dims=(72, 72, 72), n_occ: int = 128, n_pert: int = 64,
            n_omega: int = 128, cache: bool = True):
    """64-atom 2 x 2 x 2 supercell of the cubic cell (a = 20.52 bohr), ecut 25 Ry (18 277 plane
    waves), 72^3 box, k = Gamma, q = 0, 128 occupied bands, the 64 shortest non-zero G,
    omega = linspace(0, 60 eV, 128), eta = 0.1 eV.
    Draws: rng = default_rng(seed); displacements rng.normal(0, 0.05, (64, 3)) bohr added to the
    diamond sites (site order: supercell offset (i, j, k) outermost, then the 8-atom cell's sites).
    With q = 0 the right-hand side of G_p = 0 would be zero after P_c (the bands are
    eigenvectors), hence the non-zero G."""
    alat = 10.26
    a, tau = supercell64_cell(alat)
    rng = np.random.default_rng(seed)
    tau = tau + rng.normal(0.0, 0.05, size=tau.shape)
    omega = np.linspace(0.0, 60.0, n_omega) / HA_EV
    k = np.zeros(3)
    return make_instance("supercell64-ecut%g" % ecut_ry, seed, a, tau, ecut_ry, dims, n_occ, [(k, k)],
                         shortest_g(a, n_pert, False), omega, 0.1 / HA_EV, cache=cache)


def smooth235(n: int) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5."""
    m = max(1, n)
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def config4_spec(seed: int):
    """The drawn parameters of instance `seed` of the batched uneven workload (48 seeded
    instances of uneven size): n atoms uniform in [2, 64], cubic cell L = 10.26 (n/8)^(1/3) bohr, the
    smallest c x c x c conventional supercell holding n diamond sites, a seeded choice of n of its
    sites (fractional coordinates kept), N(0, 0.05 bohr) noise, N_occ = 2n, E_cut uniform in
    [10, 25] Ry, n_omega uniform in [16, 256], N_pert uniform in [1, 16]; k = Gamma, q = 0 and the
    N_pert shortest non-zero G; the FFT box is the smallest 2-3-5 size >= 2 m_rho + 1.
    Draws: rng = default_rng(seed); n = rng.integers(2, 65); ecut = rng.uniform(10, 25);
    n_omega = rng.integers(16, 257); n_pert = rng.integers(1, 17); sites = rng.permutation(8 c^3);
    noise = rng.normal(0, 0.05, (n, 3))."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 65))
    ecut = float(rng.uniform(10.0, 25.0))
    n_omega = int(rng.integers(16, 257))
    n_pert = int(rng.integers(1, 17))
    c = 1
    while 8 * c ** 3 < n:
        c += 1
    perm = rng.permutation(8 * c ** 3)
    noise = rng.normal(0.0, 0.05, size=(n, 3))
    L = 10.26 * (n / 8.0) ** (1.0 / 3.0)
    sites = np.array([(np.array([i, j, k]) + f) / c for i in range(c) for j in range(c) for k in range(c)
                      for f in DIAMOND_FRAC])
    tau = sites[perm[:n]] * L + noise
    a = np.eye(3) * L
    mil, _ = sphere(a, (0.0, 0.0, 0.0), 4.0 * ecut, check_margin=False)
    dims = tuple(smooth235(2 * int(np.abs(mil[:, i]).max()) + 1) for i in range(3))
    npw = len(sphere(a, (0.0, 0.0, 0.0), ecut, check_margin=False)[0])
    return {"seed": seed, "n_atoms": n, "ecut_ry": ecut, "n_omega": n_omega, "n_pert": n_pert, "a": a, "tau": tau,
            "dims": dims, "n_pw": npw, "n_occ": 2 * n}


def config4(seed: int, cache: bool = True):
    """Instance `seed` (0..47) of the batched uneven workload (config4_spec), with its ground
    state; omega = linspace(0, 60 eV, n_omega), eta = 0.1 eV."""
    sp = config4_spec(seed)
    omega = np.linspace(0.0, 60.0, sp["n_omega"]) / HA_EV
    k = np.zeros(3)
    return make_instance("uneven%d-n%d-ecut%.3f" % (seed, sp["n_atoms"], sp["ecut_ry"]), seed, sp["a"], sp["tau"],
                         sp["ecut_ry"], sp["dims"], sp["n_occ"], [(k, k)],
                         shortest_g(sp["a"], sp["n_pert"], False), omega, 0.1 / HA_EV, cache=cache)
