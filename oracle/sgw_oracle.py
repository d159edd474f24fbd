"""Plain FP64 CPU oracle for the shifted Sternheimer solve (SternheimerGW, Sec. 2.1-2.3).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or run this module:
only the tests, the smoke check and the timed CPU-baseline leg of the benchmark use it.
It shares no code with the CUDA library; both consume the same seeded inputs.

What it computes, by plain definition (no blocking, fusion or reordering):

* the plane-wave basis of Eq. 1: the sphere {G : |k+G|^2 <= E_cut[Ry]} in canonical
  order (Miller triples lexicographic, m1 outermost), kinetic energies |k+G|^2 / 2;
* the sphere -> FFT-box map ((m1 mod N1) N2 + (m2 mod N2)) N3 + (m3 mod N3);
* the dense Hamiltonian of Sec. 2.1 in that basis: kinetic and non-local
  (Kleinman-Bylander) parts in reciprocal space, the local potential through the
  discrete Fourier transform of its samples on the box, i.e.
  H[G,G'] = T_G delta + Vhat((m_G - m_G') mod N) + sum_p D_p beta_p(k+G) conj(beta_p(k+G'));
* the right-hand side of Eq. 8 for the periodic perturbation exp(i(q+G_p).r): the
  occupied state at k re-expressed in the k+q basis (an exact gather of coefficients),
  then b = -P_c rhs with P_c = 1 - sum_v |psi_v><psi_v| (the sign follows the problem
  statement -P_c dV psi_v; Eq. 8 prints +(1 - P_occ), a global sign);
* the solution of the Sternheimer equation Eq. 6 with the Coulomb-response operator of
  Eq. 7 read as (P_c H P_c - z) dpsi = b, z = eps_v + omega + i eta, by one dense LU per
  shift;
* the sum over all unoccupied eigenstates of the finite basis, which equals that
  solution (used to pin it on tiny bases);
* the true residual and the a-posteriori error certificate |r| / (eta |dpsi|);
* columns of the Green's function of Eq. 2-3, G(z) = (z - H)^-1 (no projector), by dense
  LU per shift and by the spectral sum over all eigenstates, with their residual and
  certificate |r| / (|Im z| |g|);
* one k-point's contribution to the density response of Eq. 5 by the paper's route
  (Sternheimer solutions at +-(omega + i eta), real-space product with the unperturbed
  periodic part, Fourier transform back) and by the sum over the eigenstates of H_{k+q};
* the spherically truncated Coulomb potential of Sec. 2.6, the dielectric matrix of Eq. 4
  and its inverse, and the correlation part W-bar of the screened interaction (Eq. 9);
* the density response at imaginary frequencies and the AAA rational approximation used to
  continue such data to the real axis (Sec. 2.7).

Each function cites the passage of the paper it restates.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


# ------------------------------------------------------------------------- Eq. 1 basis

def reciprocal(a):
    """Reciprocal lattice rows b_i = 2 pi (a_j x a_k) / Omega (cyclic), Omega = a_1.(a_2 x a_3)."""
    a = np.asarray(a, dtype=np.float64)
    vol = float(np.dot(a[0], np.cross(a[1], a[2])))
    return np.array([np.cross(a[1], a[2]), np.cross(a[2], a[0]), np.cross(a[0], a[1])]) * (2 * math.pi / vol)


def cell_volume(a):
    a = np.asarray(a, dtype=np.float64)
    return abs(float(np.dot(a[0], np.cross(a[1], a[2]))))


def gsphere(a, k_frac, ecut_ry):
    """Plane waves of Eq. 1 kept by the cutoff: Miller triples m with |k + m.B|^2 <= E_cut[Ry].

    The membership test is evaluated in FP64 in a fixed order without fused multiply-add:
    k_x = (k1 b1x + k2 b2x) + k3 b3x;  g_x = ((k_x + m1 b1x) + m2 b2x) + m3 b3x;
    |g|^2 = (g_x g_x + g_y g_y) + g_z g_z.  Order: m1 outermost, m3 innermost, ascending.
    Returns (miller int32 [npw][3], kinetic f64 [npw] = |k+G|^2 / 2).
    """
    b = reciprocal(a)
    k = np.asarray(k_frac, dtype=np.float64)
    kc = [(k[0] * b[0, x] + k[1] * b[1, x]) + k[2] * b[2, x] for x in range(3)]
    lengths = [math.sqrt(float(np.dot(a[i], a[i]))) for i in range(3)]
    # |m_i + k_i| = |(k+G).a_i| / 2pi <= sqrt(E_cut) |a_i| / 2pi
    bound = [int(math.ceil(math.sqrt(ecut_ry) * lengths[i] / (2 * math.pi) + abs(k[i]))) for i in range(3)]
    m1, m2, m3 = np.meshgrid(np.arange(-bound[0], bound[0] + 1), np.arange(-bound[1], bound[1] + 1),
                             np.arange(-bound[2], bound[2] + 1), indexing="ij")
    m = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    mf = m.astype(np.float64)
    g = [((kc[x] + mf[:, 0] * b[0, x]) + mf[:, 1] * b[1, x]) + mf[:, 2] * b[2, x] for x in range(3)]
    n2 = (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]
    keep = n2 <= ecut_ry
    return m[keep].astype(np.int32), 0.5 * n2[keep]


def box_map(miller, dims):
    """Sphere -> box linear index, box stored C order [N1][N2][N3] (axis 3 fastest)."""
    m = np.asarray(miller, dtype=np.int64)
    n1, n2, n3 = dims
    return (((m[:, 0] % n1) * n2 + (m[:, 1] % n2)) * n3 + (m[:, 2] % n3)).astype(np.int32)


def min_box(a, ecut_ry):
    """Smallest alias-free box: N_i >= 2 max|m_i| + 1 over the potential's sphere |G|^2 <= 4 E_cut."""
    mil, _ = gsphere(a, (0.0, 0.0, 0.0), 4.0 * ecut_ry)
    return tuple(2 * int(np.abs(mil[:, i]).max()) + 1 for i in range(3))


# --------------------------------------------------------------- Sec. 2.1 Hamiltonian

def vloc_hat(vloc_r):
    """Vhat(n) = N^-3 sum_j V(r_j) exp(-2 pi i n.j / N): the potential's coefficients on the box."""
    v = np.asarray(vloc_r, dtype=np.float64)
    return np.fft.fftn(v) / v.size


def kb_beta(a, tau, k_frac, miller, kb_atom, kb_width):
    """<k+G|beta_p> for s-type Gaussian projectors beta(r) = (pi w^2)^(-3/4) exp(-r^2 / 2w^2)
    centred on atom tau_{atom[p]}: Omega^(-1/2) (4 pi w^2)^(3/4) exp(-w^2 |k+G|^2 / 2) exp(-i (k+G).tau).
    Returns [n_proj][npw] c128."""
    b = reciprocal(a)
    vol = cell_volume(a)
    kg = (np.asarray(miller, np.float64) + np.asarray(k_frac, np.float64)[None, :]) @ b
    kg2 = np.sum(kg * kg, axis=1)
    out = np.empty((len(kb_atom), len(miller)), dtype=np.complex128)
    for p, (ia, w) in enumerate(zip(kb_atom, kb_width)):
        t = np.asarray(tau, np.float64)[ia]
        out[p] = vol ** -0.5 * (4 * math.pi * w * w) ** 0.75 * np.exp(-0.5 * w * w * kg2) \
            * np.exp(-1j * (kg @ t))
    return out


def dense_h(a, tau, ecut_ry, k_frac, dims, vloc_r, kb_atom, kb_width, kb_d):
    """Dense H_k of Sec. 2.1 in the plane-wave basis of Eq. 1.  Returns (H, miller, kinetic)."""
    miller, kin = gsphere(a, k_frac, ecut_ry)
    vh = vloc_hat(vloc_r)
    n = len(miller)
    h = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        d = (miller[i][None, :] - miller) % np.asarray(dims)[None, :]
        h[i, :] = vh[d[:, 0], d[:, 1], d[:, 2]]
    h[np.diag_indices(n)] += kin
    beta = kb_beta(a, tau, k_frac, miller, kb_atom, kb_width)
    # sum_p D_p beta_p(G) conj(beta_p(G')) as one matrix product over p
    h += (beta.T * np.asarray(kb_d, np.float64)[None, :]) @ beta.conj()
    return h, miller, kin


def dense_h_inst(inst, k_frac):
    return dense_h(inst.a, inst.tau, inst.ecut_ry, k_frac, inst.fft_dims, inst.vloc_r,
                   inst.kb_atom, inst.kb_width, inst.kb_d)


def apply_h_fft(a, tau, ecut_ry, k_frac, dims, vloc_r, kb_atom, kb_width, kb_d, x):
    """Matrix-free H x as Sec. 2.1 describes it: kinetic and non-local in reciprocal
    space, V_loc in real space via FFT (numpy's).  x: [nvec][npw].  Used as the
    matrix-free CPU comparison; it must equal dense_h(...) @ x."""
    miller, kin = gsphere(a, k_frac, ecut_ry)
    idx = box_map(miller, dims)
    n_box = int(np.prod(dims))
    x = np.atleast_2d(np.asarray(x, np.complex128))
    beta = kb_beta(a, tau, k_frac, miller, kb_atom, kb_width)
    y = np.empty_like(x)
    for v in range(x.shape[0]):
        box = np.zeros(n_box, dtype=np.complex128)
        box[idx] = x[v]
        psi_r = np.fft.ifftn(box.reshape(dims)) * n_box          # sum_G c_G exp(+iG.r)
        w = np.fft.fftn(psi_r * vloc_r).ravel() / n_box           # back to coefficients
        y[v] = w[idx] + kin * x[v] + (np.asarray(kb_d)[:, None] * beta * (beta.conj() @ x[v])[:, None]).sum(0)
    return y


# -------------------------------------------------------------- Eq. 7-8 projector, RHS

def project_c(psi_v, x):
    """P_c x = x - sum_v psi_v <psi_v|x> for rows x ([nvec][npw]); psi_v [n_occ][npw]."""
    psi = np.asarray(psi_v, np.complex128)
    x = np.atleast_2d(np.asarray(x, np.complex128))
    return x - (x @ psi.conj().T) @ psi


def make_rhs(miller_kq, miller_k, psi_k, gp_miller):
    """dV psi_v expressed in the k+q basis for dV = exp(i(q+G_p).r) (Eq. 8 driving field):
    rhs[v*n_pert + p][G'] = psi_{v,k}(G' - G_p) when G' - G_p is in the k sphere, else 0."""
    lookup = {tuple(int(c) for c in m): i for i, m in enumerate(miller_k)}
    n_v, n_p = len(psi_k), len(gp_miller)
    out = np.zeros((n_v * n_p, len(miller_kq)), dtype=np.complex128)
    for p, gp in enumerate(gp_miller):
        for j, m in enumerate(miller_kq):
            src = lookup.get((int(m[0] - gp[0]), int(m[1] - gp[1]), int(m[2] - gp[2])))
            if src is not None:
                for v in range(n_v):
                    out[v * n_p + p, j] = psi_k[v][src]
    return out


# ------------------------------------------------------------------ Eq. 6-7 the solve

def projected_h(h, psi_v):
    """P_c H P_c with P_c = 1 - Q, Q = sum_v |psi_v><psi_v| (Eq. 7), expanded as
    H - Q H - H Q + Q H Q and each Q product taken through the n_occ states (the same matrix as
    forming P_c densely, at a cost linear in n_occ)."""
    psi = np.asarray(psi_v, np.complex128)
    a = psi.conj() @ h                 # <psi_v| H      [n_occ][n]
    b = h @ psi.T                      # H |psi_v>      [n][n_occ]
    c = a @ psi.T                      # <psi_v|H|psi_w>
    return h - psi.T @ a - b @ psi.conj() + psi.T @ (c @ psi.conj())


def shifted_operator(h, psi_v, z):
    """P_c H P_c - z on the full basis (on range(P_v) it acts as -z; z has Im z = eta > 0)."""
    n = h.shape[0]
    return projected_h(h, psi_v) - z * np.eye(n)


def solve_shifted(h, psi_v, rhs, e_ref, omega, eta):
    """dpsi[r][j] solving (P_c H P_c - z_rj) dpsi = -P_c rhs_r, z_rj = e_ref[r] + omega_j + i eta,
    by one dense LU per distinct shift (Eq. 6 with the operator of Eq. 7)."""
    rhs = np.atleast_2d(np.asarray(rhs, np.complex128))
    b = -project_c(psi_v, rhs)
    n = h.shape[0]
    pcp = projected_h(h, psi_v)
    e_ref = np.asarray(e_ref, np.float64)
    out = np.zeros((len(rhs), len(omega), n), dtype=np.complex128)
    for e in np.unique(e_ref):
        rows = np.nonzero(e_ref == e)[0]
        for j, w in enumerate(omega):
            z = e + w + 1j * eta
            lu = scipy.linalg.lu_factor(pcp - z * np.eye(n), check_finite=False)
            out[rows, j, :] = scipy.linalg.lu_solve(lu, b[rows].T, check_finite=False).T
    return out


def sum_over_states(h, n_occ, rhs, e_ref, omega, eta):
    """Sum over all unoccupied eigenstates of the finite basis:
    dpsi = sum_c psi_c <psi_c|dV psi_v> / (eps_v + omega - eps_c + i eta), with the occupied
    subspace spanned by the n_occ lowest eigenvectors of h."""
    w, v = np.linalg.eigh(h)
    vc = v[:, n_occ:]
    wc = w[n_occ:]
    rhs = np.atleast_2d(np.asarray(rhs, np.complex128))
    coef = rhs @ vc.conj()                       # <psi_c|rhs_r>
    out = np.zeros((len(rhs), len(omega), h.shape[0]), dtype=np.complex128)
    for r in range(len(rhs)):
        for j, om in enumerate(omega):
            out[r, j] = (coef[r] / (e_ref[r] + om - wc + 1j * eta)) @ vc.T
    return out, w


def residual(h, psi_v, rhs, e_ref, omega, eta, dpsi):
    """True residual of each pair: rel_res = |b - A x| / |b| and the certificate |r| / (eta |x|).
    A = P_c H P_c - z is normal with dist(z, spec(A + z)) >= eta, so |x - x*| / |x| <= cert."""
    rhs = np.atleast_2d(np.asarray(rhs, np.complex128))
    b = -project_c(psi_v, rhs)
    nr, nw = dpsi.shape[0], dpsi.shape[1]
    rel = np.zeros((nr, nw))
    cert = np.zeros((nr, nw))
    for r in range(nr):
        bn = np.linalg.norm(b[r])
        for j in range(nw):
            a = shifted_operator(h, psi_v, e_ref[r] + omega[j] + 1j * eta)
            res = b[r] - a @ dpsi[r, j]
            rn = np.linalg.norm(res)
            xn = np.linalg.norm(dpsi[r, j])
            rel[r, j] = rn / bn if bn > 0 else 0.0
            cert[r, j] = rn / (eta * xn) if xn > 0 else 0.0
    return rel, cert


# ------------------------------------------------------- Eq. 2-3: the Green's function

def unit_columns(n, cols):
    """e_{G'} for G' = cols, as rows [ncol][n]."""
    e = np.zeros((len(cols), n), dtype=np.complex128)
    e[np.arange(len(cols)), np.asarray(cols, dtype=np.int64)] = 1.0
    return e


def green_columns(h, cols, z):
    """g[c][j] = column cols[c] of G(z_j), i.e. the solution of (H - z_j) g = -delta_{G G'}
    (Eq. 2 with the operator of Eq. 3: no projector), by one dense LU per shift; z_j is
    complex with Im z_j != 0 (its sign is the caller's time-ordering choice)."""
    n = h.shape[0]
    e = unit_columns(n, cols)
    out = np.zeros((len(cols), len(z), n), dtype=np.complex128)
    for j, zj in enumerate(z):
        lu = scipy.linalg.lu_factor(h - zj * np.eye(n), check_finite=False)
        out[:, j, :] = scipy.linalg.lu_solve(lu, -e.T, check_finite=False).T
    return out


def green_sum_over_states(h, cols, z):
    """The spectral representation G(z) = sum_n psi_n psi_n^H / (z - eps_n) over every
    eigenstate of the finite basis (equal to green_columns by the spectral theorem)."""
    w, v = np.linalg.eigh(h)
    cols = np.asarray(cols, dtype=np.int64)
    out = np.zeros((len(cols), len(z), h.shape[0]), dtype=np.complex128)
    for j, zj in enumerate(z):
        out[:, j, :] = ((v / (zj - w)) @ v[cols].conj().T).T
    return out


def green_residual(h, cols, z, g):
    """rel_res = |-e - (H - z) g| / |e| and the certificate |r| / (|Im z| |g|): H - z is normal
    with every eigenvalue at distance >= |Im z| from 0, so |g - g*| / |g| <= cert."""
    n = h.shape[0]
    e = unit_columns(n, cols)
    rel = np.zeros((len(cols), len(z)))
    cert = np.zeros((len(cols), len(z)))
    for j, zj in enumerate(z):
        a = h - zj * np.eye(n)
        for c in range(len(cols)):
            res = -e[c] - a @ g[c, j]
            rn = np.linalg.norm(res)
            xn = np.linalg.norm(g[c, j])
            rel[c, j] = rn
            cert[c, j] = rn / (abs(zj.imag) * xn) if xn > 0 else 0.0
    return rel, cert


def time_ordered_shifts(omega, mu, eta):
    """z_j = omega_j + i eta sgn(omega_j - mu): the retarded side above the chemical potential
    mu and the advanced side below it (the reading of the time-ordering choice of Eq. 2)."""
    omega = np.asarray(omega, dtype=np.float64)
    if np.any(omega == mu):
        raise ValueError("omega_j = mu has no time-ordering sign")
    return omega + 1j * eta * np.sign(omega - mu)


# -------------------------------------------------------------- Eq. 5: density response

def solve_shifted_z(h, psi_v, rhs, z):
    """x[r][j] solving (P_c H P_c - z[r][j]) x = -P_c rhs_r for arbitrary complex z[r][j]
    (one dense LU per distinct shift)."""
    rhs = np.atleast_2d(np.asarray(rhs, np.complex128))
    z = np.asarray(z, np.complex128)
    b = -project_c(psi_v, rhs)
    n = h.shape[0]
    pc = np.eye(n, dtype=np.complex128) - np.asarray(psi_v).T @ np.asarray(psi_v).conj()
    pcp = pc @ h @ pc
    out = np.zeros((len(rhs), z.shape[1], n), dtype=np.complex128)
    for zz in np.unique(z):
        rows, cols = np.nonzero(z == zz)
        lu = scipy.linalg.lu_factor(pcp - zz * np.eye(n), check_finite=False)
        out[rows, cols, :] = scipy.linalg.lu_solve(lu, b[rows].T, check_finite=False).T
    return out


def periodic_on_box(coef, miller, dims):
    """u(r_j) = sum_G c_G exp(i G.r_j) on the box (the convention of the FFT apply)."""
    box = np.zeros(tuple(dims), dtype=np.complex128)
    m = np.asarray(miller, dtype=np.int64) % np.asarray(dims)
    box[m[:, 0], m[:, 1], m[:, 2]] = coef
    return np.fft.ifftn(box) * float(np.prod(dims))


def box_coefficient(f, g_miller, dims):
    """c_G = N^-3 sum_j f(r_j) exp(-i G.r_j) for the listed G."""
    c = np.fft.fftn(f) / float(np.prod(dims))
    m = np.asarray(g_miller, dtype=np.int64) % np.asarray(dims)
    return c[m[:, 0], m[:, 1], m[:, 2]]


def density_response(h_kq, psi_v_kq, psi_k, miller_k, miller_kq, eps_k, gp_miller, omega, eta, dims, weight):
    """One k-point's contribution to Eq. 5, by the paper's route:
        dn[G][G'][j] = weight * sum_v sum_{+-} FT_G[ conj(u_{v,k}(r)) du_{v,k+q,G'}(r; +-omega_j) ]
    where du(+-omega) solves the Sternheimer equation (P_c H P_c - z) du = -P_c dV_G' psi_v with
    the complex frequency omega_j + i eta taken with both signs, z = eps_v +- (omega_j + i eta);
    u and du are the periodic parts on the box (coefficients of Eq. 1 summed with exp(iG.r)),
    the product is formed in real space and Fourier transformed back (box DFT, N^-3); G and
    G' both run over the perturbation list gp_miller (weight = 2 / N_k for spin and the
    k-point average)."""
    w = np.asarray(omega, np.float64) + 1j * eta
    return density_response_w(h_kq, psi_v_kq, psi_k, miller_k, miller_kq, eps_k, gp_miller, w, dims, weight)


def density_response_w(h_kq, psi_v_kq, psi_k, miller_k, miller_kq, eps_k, gp_miller, w, dims, weight):
    """density_response at arbitrary complex frequencies w_j (z = eps_v +- w_j); w_j = i omega_j
    gives the response on the imaginary axis (Sec. 2.7)."""
    psi_k = np.atleast_2d(np.asarray(psi_k, np.complex128))
    w = np.asarray(w, np.complex128)
    n_v, n_p, n_w = len(psi_k), len(gp_miller), len(w)
    rhs = make_rhs(miller_kq, miller_k, psi_k, gp_miller)          # row v * n_p + p
    out = np.zeros((n_p, n_p, n_w), dtype=np.complex128)
    for v in range(n_v):
        u = periodic_on_box(psi_k[v], miller_k, dims)
        z = np.concatenate([eps_k[v] + w, eps_k[v] - w])[None, :].repeat(n_p, axis=0)
        x = solve_shifted_z(h_kq, psi_v_kq, rhs[v * n_p:(v + 1) * n_p], z)   # [n_p][2 n_w][npw]
        for p_in in range(n_p):
            for j in range(n_w):
                for s in (j, n_w + j):
                    du = periodic_on_box(x[p_in, s], miller_kq, dims)
                    out[:, p_in, j] += weight * box_coefficient(np.conj(u) * du, gp_miller, dims)
    return out


def density_response_sos(h_kq, n_occ_kq, psi_k, miller_k, miller_kq, eps_k, gp_miller, omega, eta, weight, w=None):
    """The same contribution from the eigenstates of H_{k+q} (an Adler-Wiser-type sum over the
    unoccupied states c, the n_occ_kq lowest being occupied):
        dn[G][G'][j] = weight sum_v sum_c conj(M_vc(G)) M_vc(G') [1/(eps_v + w_j - e_c)
                                                                 + 1/(eps_v - w_j - e_c)],
    w_j = omega_j + i eta (or the complex frequencies w when given),
    M_vc(G') = <psi_c | exp(i(q+G').r) psi_{v,k}>."""
    wv, vec = np.linalg.eigh(h_kq)
    vc, ec = vec[:, n_occ_kq:], wv[n_occ_kq:]
    psi_k = np.atleast_2d(np.asarray(psi_k, np.complex128))
    n_v, n_p = len(psi_k), len(gp_miller)
    freqs = (np.asarray(omega, np.float64) + 1j * eta) if w is None else np.asarray(w, np.complex128)
    rhs = make_rhs(miller_kq, miller_k, psi_k, gp_miller)
    out = np.zeros((n_p, n_p, len(freqs)), dtype=np.complex128)
    for v in range(n_v):
        m = rhs[v * n_p:(v + 1) * n_p] @ vc.conj()          # [p][c] = <psi_c|rhs_vp>
        for j, wc in enumerate(freqs):
            f = 1.0 / (eps_k[v] + wc - ec) + 1.0 / (eps_k[v] - wc - ec)
            out[:, :, j] += weight * (m.conj() * f) @ m.T
    return out


# --------------------------------------------- Eq. 4, 9 and Sec. 2.6: epsilon^-1 and W-bar

def coulomb_spherical(qg, r_cut):
    """v(q) = 4 pi / q^2 [1 - cos(q R_cut)] (Hartree units, e^2 / (4 pi eps0) = 1), the
    Coulomb potential cut off at distance R_cut (Sec. 2.6); its q -> 0 limit is 2 pi R_cut^2.
    r_cut <= 0 gives the bare 4 pi / q^2 (q = 0 is then an error)."""
    q = np.linalg.norm(np.atleast_2d(np.asarray(qg, np.float64)), axis=1)
    if r_cut <= 0:
        if np.any(q == 0):
            raise ValueError("q + G = 0 needs a truncated Coulomb potential")
        return 4.0 * math.pi / q ** 2
    out = np.empty_like(q)
    small = q * r_cut < 1e-4
    qs = q[~small]
    out[~small] = 4.0 * math.pi / qs ** 2 * (1.0 - np.cos(qs * r_cut))
    x = q[small] * r_cut                     # series of 4 pi R^2 (1 - cos x) / x^2
    out[small] = 4.0 * math.pi * r_cut ** 2 * (0.5 - x ** 2 / 24.0 + x ** 4 / 720.0)
    return out


def screened_coulomb(dn, qg, volume, r_cut):
    """From the accumulated density response dn[G][G'][w] (Eq. 5, weights included):
        eps[G][G'] = delta - dn[G][G'] v(q + G') / Omega        (Eq. 4, the response to the
                                                                  Coulomb potential of a unit
                                                                  plane-wave charge at q + G')
        W-bar[G][G'] = v(q + G) (eps^-1[G][G'] - delta)          (Eq. 9)
    per frequency by a dense inverse; rows and columns with q + G = 0 keep only their diagonal
    in eps^-1 (Sec. 2.4).  Returns (eps^-1, W-bar), each [G][G'][w]."""
    dn = np.asarray(dn, np.complex128)
    n, _, nw = dn.shape
    v = coulomb_spherical(qg, r_cut)
    zero = np.linalg.norm(np.atleast_2d(qg), axis=1) == 0
    einv = np.zeros_like(dn)
    wbar = np.zeros_like(dn)
    eye = np.eye(n)
    for j in range(nw):
        eps = eye - dn[:, :, j] * v[None, :] / volume
        inv = np.linalg.inv(eps)
        for g in np.nonzero(zero)[0]:
            d = inv[g, g]
            inv[g, :] = 0.0
            inv[:, g] = 0.0
            inv[g, g] = d
        einv[:, :, j] = inv
        wbar[:, :, j] = v[:, None] * (inv - eye)
    return einv, wbar



# ------------------------------------------ Sec. 2.7: analytic continuation by AAA

def aaa(z, f, tol=1e-13, mmax=32):
    """The adaptive Antoulas-Anderson rational approximation (Nakatsukasa, Sete and Trefethen,
    SIAM J. Sci. Comput. 40, A1494, 2018) of samples f at points z, as Sec. 2.7 uses it: greedy
    choice of support points (the sample where the current approximant errs most, the first
    on ties; the first approximant is the mean of f), barycentric weights from the right
    singular vector of the Loewner matrix for its smallest singular value, stop when the
    largest deviation on the remaining samples is <= tol * max|f| or at mmax support points.
    Returns (support points, support values, weights)."""
    z = np.asarray(z, np.complex128)
    f = np.asarray(f, np.complex128)
    m = len(z)
    fmax = np.abs(f).max()
    rest = np.ones(m, bool)
    sup = []
    r = np.full(m, f.mean())
    w = np.zeros(0, np.complex128)
    for _ in range(min(mmax, m)):
        err = np.where(rest, np.abs(f - r), -1.0)
        j = int(np.argmax(err))
        sup.append(j)
        rest[j] = False
        zs, fs = z[sup], f[sup]
        idx = np.nonzero(rest)[0]
        cauchy = 1.0 / (z[idx][:, None] - zs[None, :])
        loewner = (f[idx][:, None] - fs[None, :]) * cauchy
        if len(idx) == 0:
            w = np.ones(len(sup), np.complex128) / math.sqrt(len(sup))
            break
        _, _, vh = np.linalg.svd(loewner, full_matrices=True)
        w = vh[-1].conj()
        r = f.copy()
        r[idx] = (cauchy @ (w * fs)) / (cauchy @ w)
        if np.abs(f[idx] - r[idx]).max() <= tol * fmax:
            break
    return z[sup], f[sup], w


def aaa_eval(zs, fs, w, x):
    """r(x) = sum_j w_j f_j / (x - z_j) / sum_j w_j / (x - z_j), and f_j at x = z_j."""
    x = np.asarray(x, np.complex128)
    out = np.empty(x.shape, np.complex128)
    for i, xi in enumerate(x.ravel()):
        d = xi - zs
        hit = np.nonzero(d == 0)[0]
        if len(hit):
            out.ravel()[i] = fs[hit[0]]
        else:
            c = w / d
            out.ravel()[i] = np.sum(c * fs) / np.sum(c)
    return out
