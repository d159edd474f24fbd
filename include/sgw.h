/*
 * sgw.h -- C ABI of the GB300 shifted-Sternheimer library.
 *
 * The library solves, for every right-hand side r and frequency omega_j,
 *
 *     (P_c H P_c - z_rj) dpsi_rj = -P_c rhs_r,     z_rj = e_ref[r] + omega_j + i eta,
 *
 * the Sternheimer equation of SternheimerGW (arXiv:1812.03717, Sec. 2.3, Eq. 6) with the
 * Coulomb-response operator of Eq. 7 read as H restricted to the conduction subspace
 * (P_c = 1 - sum_v |psi_v><psi_v|; on b in range(P_c) this has the same solution as
 * H + alpha P_occ - z for any alpha > 0), and the driving field of Eq. 8 given by the
 * caller as rhs_r = dV psi_v expressed in this system's plane-wave basis.  All shifts
 * of one right-hand side share one Krylov space (Sec. 2.2): one seed system carries them.
 * The same machinery gives the columns of the Green's function of Eq. 2-3
 * (sgw_solve_green), the density response of Eq. 5 on the real or imaginary frequency axis
 * (sgw_density_response, sgw_density_response_w); sgw_screened_coulomb turns the response
 * into epsilon^-1 and W-bar (Eq. 4, 9) and sgw_aaa continues sampled functions by AAA
 * (Sec. 2.7).
 *
 * Units: Hartree atomic units (Ha, bohr).  E_cut is in Ry: the basis of Eq. 1 is the
 * sphere |k+G|^2 <= E_cut[Ry] (bohr^-2).  Complex numbers are interleaved FP64 pairs
 * (re, im) = C99 double complex / numpy complex128.
 *
 * Memory: every vector argument marked "host or device" may be a host pointer or a CUDA
 * device pointer of the current device; the library detects which.  The library copies
 * what it keeps (the system owns its device copies); the caller owns every buffer it
 * passes.  Work is ordered on the stream given (NULL = the legacy default stream); calls
 * that return results to host memory synchronise that stream before returning.  A call on a
 * system makes the system's device (the current device at sgw_create_system) current while
 * it runs and gives the caller's current device back before it returns.
 *
 * Errors: every call returns an sgw_status; nothing throws across the ABI and nothing
 * aborts.  sgw_last_error() returns a message for the last failing call of this host
 * thread.  A system handle must be used by one host thread at a time.
 */
#ifndef SGW_H
#define SGW_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgw_system sgw_system;   /* opaque, owned by the library */

typedef enum {
    SGW_OK = 0,
    SGW_EINVAL = 1,       /* invalid argument (sizes, NaN/Inf, eta <= 0, non-orthonormal psi_v, ...) */
    SGW_ENOMEM = 2,       /* device allocation failed */
    SGW_ECUDA = 3,        /* a CUDA call failed; the message names it */
    SGW_ENOCONV = 4,      /* some (rhs, omega) pair missed the tolerance; results and report still written */
    SGW_EALIAS = 5,       /* FFT box smaller than 2 m_rho + 1 along some axis */
    SGW_ESTATE = 6,       /* call out of order (e.g. solve before sgw_set_occupied) */
    SGW_EUNSUPPORTED = 7  /* a size this build does not handle (named in the message) */
} sgw_status;

/* Per-pair status codes written to sgw_report.status. */
enum {
    SGW_PAIR_CONVERGED = 0,
    SGW_PAIR_MAXITER = 1,    /* matrix-vector budget exhausted */
    SGW_PAIR_BREAKDOWN = 2,  /* a Krylov denominator vanished */
    SGW_PAIR_NONFINITE = 3   /* a NaN/Inf appeared in the recurrences */
};

typedef struct {
    double a[3][3];        /* rows = lattice vectors a1, a2, a3 (bohr) */
    int n_atoms;
    const double* tau;     /* [n_atoms][3] Cartesian positions (bohr), host */
} sgw_cell;

/* Kleinman-Bylander non-local part, one s-type Gaussian projector per entry:
 * beta_p(r) = (pi w_p^2)^(-3/4) exp(-|r - tau_{atom[p]}|^2 / (2 w_p^2)),
 * V_NL = sum_p |beta_p> D_p <beta_p|  (Sec. 2.1: non-local part applied in reciprocal space). */
typedef struct {
    int n_proj;
    const int* atom;       /* [n_proj] atom index of each projector, host */
    const double* width;   /* [n_proj] w_p (bohr), host */
    const double* D;       /* [n_proj] D_p (Ha), host */
} sgw_kb;

/* Builds the plane-wave basis of Eq. 1 at Bloch vector k (the basis the response lives
 * in: k+q in perturbation-theory terms) and uploads the Hamiltonian of Sec. 2.1.
 *   cell      lattice and atoms (host).
 *   ecut_ry   E_cut in Ry (> 0).
 *   k_frac    k in fractional coordinates of the reciprocal lattice (host, 3 doubles).
 *   fft_dims  box N1, N2, N3 (host); each must factor into 2, 3 and 5 and satisfy
 *             N_i >= 2 m_rho,i + 1 with m_rho the largest |Miller index| of |G|^2 <= 4 E_cut
 *             (else SGW_EALIAS).
 *   vloc_r    real local potential V(r_j) on the box, r_j = sum_i (j_i / N_i) a_i, C order
 *             [N1][N2][N3] (host), Ha.
 *   kb        projectors (host arrays; n_proj may be 0).
 *   out       receives the handle.
 * The sphere is built on the GPU with an FP64 test evaluated without fused multiply-add:
 *   k_x = (k1 b1x + k2 b2x) + k3 b3x,  g_x = ((k_x + m1 b1x) + m2 b2x) + m3 b3x,
 *   |k+G|^2 = (g_x^2 + g_y^2) + g_z^2 <= E_cut, Miller triples in lexicographic order
 *   (m1 outermost, each ascending): the canonical order of every coefficient array. */
sgw_status sgw_create_system(const sgw_cell* cell, double ecut_ry, const double k_frac[3],
                             const int fft_dims[3], const double* vloc_r, const sgw_kb* kb,
                             sgw_system** out);

/* The plane-wave basis of Eq. 1 (Sec. 2.1) built by sgw_create_system: the number of plane
 * waves and, optionally, the Miller triples [n_pw][3] and the kinetic energies |k+G|^2 / 2
 * (Ha) [n_pw] in canonical order (host buffers, or NULL).  SGW_EINVAL for a NULL sys. */
sgw_status sgw_get_gvectors(const sgw_system* sys, int* n_pw, int* miller, double* kin);

/* Sphere -> FFT box map of the H application by Fourier transforms (Sec. 2.1): entry
 * g = ((m1 mod N1) N2 + (m2 mod N2)) N3 + (m3 mod N3), written to the host int[n_pw]
 * `map`.  SGW_EINVAL for a NULL argument. */
sgw_status sgw_get_box_map(const sgw_system* sys, int* map);

/* Split of the on-chip FFT box (an implementation choice the paper has no counterpart for:
 * how the Sec. 2.1 H application is laid out on this GPU).  A box whose sticks and planes do
 * not fit one CTA's shared memory is shared by a thread-block cluster of csize CTAs, each
 * holding a contiguous range of sticks and owning their plane waves; the library picks csize
 * (1..16) at sgw_create_system / sgw_set_occupied as the size that keeps the most SMs busy.
 * sgw_set_split forces csize (0 restores the automatic choice; SGW_EUNSUPPORTED if the box
 * cannot be split that way) -- a test and tuning hook; it synchronises the device.
 * sgw_get_split reports the sizes in use for the 16-byte policies (FP64, float-float) and for
 * FP32 (0: FP32 does not fit). */
sgw_status sgw_set_split(sgw_system* sys, int csize);
sgw_status sgw_get_split(const sgw_system* sys, int* csize, int* csize_fp32);

/* Occupied manifold of this basis (Eq. 7-8: P_occ): psi_v complex [n_occ][n_pw] (host or
 * device) and eps_v [n_occ] (host, Ha).  Rejected with SGW_EINVAL unless
 * max |psi^H psi - I| <= 1e-10.  May be called again to replace the manifold. */
sgw_status sgw_set_occupied(sgw_system* sys, int n_occ, const void* psi_v, const double* eps_v);

/* Driving field of Eq. 8 for the periodic perturbations dV = exp(i (q + G_p).r):
 *   rhs[v * n_pert + p][G'] = psi_k[v][G' - G_p]  if G' - G_p is in sys_k's sphere, else 0,
 * for G' in sys_kq's sphere (sys_kq at k+q, sys_k at k).  psi_k complex [n_v][n_pw(sys_k)]
 * (host or device); gp_miller int [n_pert][3] (host); rhs complex [n_v*n_pert][n_pw(sys_kq)]
 * (host or device).  An exact gather: bit-identical to the definition. */
sgw_status sgw_make_rhs(const sgw_system* sys_kq, const sgw_system* sys_k, int n_v, const void* psi_k,
                        int n_pert, const int* gp_miller, void* rhs, void* stream);

/* Arithmetic of the H application and of the Krylov vectors of the multishift pass.  The
 * Krylov recurrence scalars, the right-hand side b = -P_c rhs, its norm and the true
 * residual judging every pair are FP64 in every mode (the problem statement's "FP64" and
 * "mixed" modes: FP64 is SGW_PREC_FP64; SGW_PREC_DF32 and SGW_PREC_FP32 are two mixed forms). */
enum {
    SGW_PREC_FP64 = 0,   /* FP64 throughout (the FP64 pipe) */
    SGW_PREC_DF32 = 1,   /* float-float: value = hi + lo in two FP32 numbers (~48-bit significand)
                            on the FP32 pipes; one multishift pass reaches FP64-level residuals */
    SGW_PREC_FP32 = 2    /* FP32 (complex64) inner solve with FP32 accumulation inside FP64
                            iterative refinement: the multishift pass runs in FP32, every pair's
                            true residual is formed in FP64 and the pairs above tolerance get
                            correction solves in float-float until the FP64 check passes */
};

/* y = H x for nvec vectors [nvec][n_pw] (host or device): kinetic + non-local in
 * reciprocal space, local through the FFT box (Sec. 2.1).  precision: SGW_PREC_*.  Test hook. */
sgw_status sgw_apply_h(sgw_system* sys, int nvec, const void* x, void* y, int precision, void* stream);

/* y_i = (P_c H P_c - z_i) x_i, z complex [nvec] as (re, im) pairs (host).  Requires
 * sgw_set_occupied.  Test hook for the operator the solver iterates with. */
sgw_status sgw_apply_shifted(sgw_system* sys, int nvec, const void* x, const double* z, void* y,
                             int precision, void* stream);

/* Multishift methods. */
enum {
    SGW_METHOD_LANCZOS = 0,   /* shifted Lanczos (FOM) on the Hermitian P_c H P_c: one H application per
                                 Krylov step, every shift's Galerkin solution from T_k - z_j (default) */
    SGW_METHOD_BICGSTAB = 1   /* shifted BiCGstab(ell) (Frommer 2003) */
};

typedef struct sgw_mlp sgw_mlp;   /* learned preconditioner (below) */

typedef struct {
    int method;       /* SGW_METHOD_* */
    int precision;    /* SGW_PREC_* of the multishift pass (Lanczos only; the true residual is
                         assembled in FP64, with H applied in FP64 for SGW_PREC_FP64 and in
                         float-float otherwise) */
    int ell;          /* BiCGstab(ell) degree 1..4 (0 -> 4); unused by Lanczos */
    int seed_index;   /* BiCGstab seed shift; -1 -> the largest omega; unused by Lanczos */
    int max_matvec;   /* H applications per right-hand side and per correction solve (0 -> 16384 for
                         Lanczos, whose basis it sizes, 40000 for BiCGstab); the Lanczos basis is also
                         capped by half the free device memory */
    int max_refine;   /* rounds of per-shift correction solves (0 -> 3, negative -> none) */
    int threads;      /* CTA size of the Lanczos kernel: 256, 384 or 512 (0 -> 384 FP64, else 512) */
    void* stream;     /* cudaStream_t, NULL = default stream */
    double cert_tol;  /* a pair is converged when rel_res <= tol and its error certificate
                         |r| / (|Im z| |x|) <= cert_tol (0 -> 1e-8; negative -> not checked) */
    const void* x0;   /* NULL, or initial solutions [nrhs][nomega][n_pw] (host or device; e.g. a
                         previous call's dpsi, to resume): the multishift pass is skipped, every
                         pair's true residual is checked from x0 and only the pairs above the
                         tolerances get per-shift correction solves */
    int precond;      /* SGW_PRECOND_* of the per-shift correction solves: NONE -> shifted Lanczos
                         (one shift), PLAIN / LEARNED -> right-preconditioned BiCGstab(ell)
                         (one CTA per vector, or one cluster when the box is split) */
    const sgw_mlp* mlp;  /* the perceptron of SGW_PRECOND_LEARNED */
    int plain_budget; /* SGW_PRECOND_LEARNED: the plain preconditioner's typical (median) H
                         applications for systems of this size; the learned round stops at twice
                         it and its unconverged pairs restart from their current x with the plain
                         preconditioner (0 -> no such cap: only max_matvec) */
} sgw_solve_opts;

/* Per-pair outputs, each [nrhs][nomega] host arrays (any may be NULL). */
typedef struct {
    int* matvecs;       /* H applications spent on the pair: the seed's count when the pair left the
                           multishift pass, plus its correction solves */
    double* est_res;    /* recursive residual estimate |r| / |b| when the multishift pass stopped */
    double* rel_res;    /* true FP64 residual |b - A x| / |b| of the returned solution */
    double* cert;       /* error certificate |b - A x| / (eta |x|) >= |x - x*| / |x| */
    int* status;        /* SGW_PAIR_*: CONVERGED iff rel_res <= tol and cert <= cert_tol */
    int* launches;      /* one int: library kernels launched by this call */
    double* kernel_ms;  /* one double: CUDA-event time of the multishift kernel launch on the stream */
    int* fallbacks;     /* one int: pairs that restarted with the plain preconditioner after the
                           learned round (SGW_PRECOND_LEARNED) */
} sgw_report;

/* Right-hand sides the multishift kernel works on at once (one per CTA, or per cluster when
 * the box is split) for nomega shifts in `precision` with `threads` per CTA (0: default):
 * batches of a multiple of it keep every owner busy.  Not in the paper: a sizing query. */
sgw_status sgw_solve_capacity(const sgw_system* sys, int nomega, int precision, int threads, int* owners);

/* Multishift solve (the hot path).  For every r < nrhs and j < nomega solves
 *   (P_c H P_c - z_rj) dpsi[r][j] = -P_c rhs[r],   z_rj = e_ref[r] + omega[j] + i eta.
 * 1. Multishift pass (Sec. 2.2: shifted systems share one Krylov space).  Default: the
 *    Lanczos process on the Hermitian P_c H P_c with b as start vector; each shift's
 *    Galerkin solution x_j = V_k (T_k - z_j)^{-1} |b| e_1 and its residual norm follow from
 *    the tridiagonal T_k alone, a shift is done when its residual reaches tol |b|, and the
 *    solutions are formed from the stored basis at the end.  Alternative: shifted
 *    BiCGstab(ell) (Frommer 2003, the solver the paper cites), one seed system carrying
 *    all shifts through scalar recurrences.
 * 2. True FP64 residual and certificate of every pair (as sgw_residual).
 * 3. Pairs whose true residual exceeds tol or whose certificate exceeds cert_tol, but whose
 *    relative residual is at most 1e-3 (near convergence: rounding of the pass, the
 *    recursive / true residual gap), get per-shift correction solves A_j d = r_j, x_j += d,
 *    then step 2 again; up to max_refine rounds.  The returned solutions are projected onto
 *    range(P_c), where the exact ones lie.
 *   rhs    complex [nrhs][n_pw] (host or device): dV psi_v in this basis.
 *   e_ref  [nrhs] host, Ha.   omega [nomega] host, Ha.   eta > 0 (Ha), else SGW_EINVAL.
 *   tol    relative residual target (e.g. 1e-10).
 *   dpsi   complex [nrhs][nomega][n_pw] (host or device), overwritten.
 *   report optional per-pair report.
 * A pair is converged when rel_res <= tol and cert <= opts.cert_tol (default 1e-8): the
 * multishift pass keeps a shift going until its estimated certificate also holds, and the
 * corrections of step 3 cover both targets.  With opts.x0 the pass is skipped (resume).
 * A zero right-hand side gives dpsi = 0 with status CONVERGED.  Returns SGW_ENOCONV if any
 * pair misses tol or the certificate (results and report are still written). */
sgw_status sgw_solve_shifted(sgw_system* sys, int nrhs, const void* rhs, const double* e_ref,
                             int nomega, const double* omega, double eta, double tol,
                             const sgw_solve_opts* opts, void* dpsi, sgw_report* report);

/* Batched multishift solves of several systems of uneven sizes (the paper has no counterpart:
 * this packs the right-hand sides, frequencies and k-points of different bases into few kernel
 * launches).  Every item is solved exactly as sgw_solve_shifted would (same eta, tol and opts;
 * each item has its own frequencies), but the multishift passes of all items whose on-chip box
 * uses the same cluster size run in ONE persistent launch: its work queue hands out (item,
 * right-hand side) pairs, the items with the most plane waves first, each owner re-reading the
 * item's plan and twiddles when it changes item; the Krylov workspace is sized for the largest
 * item.  Then each item's FP64 check and corrections run as in sgw_solve_shifted.
 *   items   [nitems] host array; item.sys distinct, all on one device, with occupied states;
 *           rhs / dpsi host or device as in sgw_solve_shifted; report optional (launches counts
 *           the shared launch in the first item of each group; kernel_ms is the shared launch's).
 *   opts    as sgw_solve_shifted; method Lanczos only, no x0 (else SGW_EUNSUPPORTED).
 * Returns SGW_ENOCONV if any pair of any item misses tol or the certificate. */
typedef struct {
    sgw_system* sys;
    int nrhs;
    const void* rhs;        /* complex [nrhs][n_pw(sys)] (host or device) */
    const double* e_ref;    /* [nrhs] host, Ha */
    int nomega;
    const double* omega;    /* [nomega] host, Ha */
    void* dpsi;             /* complex [nrhs][nomega][n_pw(sys)] (host or device), overwritten */
    sgw_report* report;     /* optional */
} sgw_batch_item;
sgw_status sgw_solve_batched(int nitems, const sgw_batch_item* items, double eta, double tol,
                             const sgw_solve_opts* opts);

/* Green's-function columns (Sec. 2.2, Eq. 2 with the operator of Eq. 3).  For every c < ncol
 * and j < nz solves
 *   (H - z_j) g[c][j] = -e_{G'},   G' = cols[c],
 * i.e. g[c][j] is column G' of G(z_j) = (z_j - H)^{-1} in this system's plane-wave basis.
 * There is no projector: the occupied states set by sgw_set_occupied are not used (and need
 * not be set).  All shifts of one column share one Krylov space (the Lanczos process on the
 * Hermitian H, as in sgw_solve_shifted), followed by the FP64 true residual and per-shift
 * corrections of pairs above tol.
 *   cols   [ncol] host, plane-wave indices in [0, n_pw) (else SGW_EINVAL).
 *   z      [nz][2] host, (Re z, Im z) in Ha; Im z != 0 (else SGW_EINVAL) and of either sign
 *          per shift: the caller chooses it (time ordering: Im z_j = eta sgn(Re z_j - mu)).
 *   tol    residual target |-e - (H - z) g| <= tol (|e| = 1).
 *   opts   as sgw_solve_shifted; only SGW_METHOD_LANCZOS (else SGW_EUNSUPPORTED).
 *   g      complex [ncol][nz][n_pw] (host or device), overwritten.
 *   report optional per-pair report [ncol][nz]; cert = |r| / (|Im z| |g|).
 * Returns SGW_ENOCONV if any pair's true residual stays above tol (results still written). */
sgw_status sgw_solve_green(sgw_system* sys, int ncol, const int* cols, int nz, const double* z, double tol,
                           const sgw_solve_opts* opts, void* g, sgw_report* report);

/* One k-point's contribution to the density response of Eq. 5 (Sec. 2.3):
 *   dn[G][G'][j] += weight * sum_v sum_{+-} FT_G[ conj(u_{v,k}(r)) du_{v,k+q,G'}(r; +-w_j) ],
 * w_j = omega[j] + i eta, with du(+-w) the Sternheimer solutions
 *   (P_c H P_c - z) du = -P_c rhs[v n_pert + p],   z = eps_v[v] +- w_j,
 * both signs sharing one Krylov space per right-hand side (2 nomega shifts, the -w branch
 * with Im z = -eta), followed by the FP64 true residual and corrections as in
 * sgw_solve_shifted.  u_{v,k}(r) = sum_G psi_{v,k}(G) e^{iG.r} and du likewise (periodic parts);
 * FT_G is the box coefficient N^-3 sum_r f(r) e^{-iG.r}.  The library evaluates it in
 * reciprocal space as <dV_G psi_v | du> (equal by the convolution theorem; dV_G psi_v is the
 * Eq. 8 right-hand side for G).  G and G' both run over the n_pert perturbations of rhs.
 *   rhs     complex [n_v * n_pert][n_pw] (host or device): sgw_make_rhs output, row v n_pert + p.
 *   eps_v   [n_v] host, Ha (the unperturbed energies eps_{v,k}).   omega [nomega] host, Ha;
 *           2 nomega <= 512 (else SGW_EUNSUPPORTED).   eta > 0 (else SGW_EINVAL).
 *   weight  e.g. 2 / N_k (spin, k-point average); dn is ACCUMULATED: call once per k-point.
 *   dn      complex [n_pert (G)][n_pert (G')][nomega] (host or device), read and updated.
 *   report  optional per-pair report [n_v * n_pert][2 nomega] (shift j < nomega at +w_j,
 *           nomega + j at -w_j); launches counts the density kernel too.
 * Returns SGW_ESTATE without occupied states, SGW_ENOCONV (dn still updated) if a pair's
 * true residual stays above tol. */
sgw_status sgw_density_response(sgw_system* sys, int n_v, int n_pert, const void* rhs, const double* eps_v,
                                int nomega, const double* omega, double eta, double weight, double tol,
                                const sgw_solve_opts* opts, void* dn, sgw_report* report);

/* sgw_density_response at arbitrary complex frequencies w_j (Sec. 2.7: the imaginary-axis
 * variant takes w_j = i omega_j): shifts z = eps_v + w_j and eps_v - w_j, everything else as
 * sgw_density_response.  w: [nw][2] host, (Re w, Im w) in Ha with Im w != 0 (else
 * SGW_EINVAL); 2 nw <= 512.  dn: [n_pert][n_pert][nw], accumulated. */
sgw_status sgw_density_response_w(sgw_system* sys, int n_v, int n_pert, const void* rhs, const double* eps_v,
                                  int nw, const double* w, double weight, double tol, const sgw_solve_opts* opts,
                                  void* dn, sgw_report* report);

/* AAA rational approximation (Sec. 2.7; Nakatsukasa, Sete and Trefethen 2018), batched over
 * nfun functions that share the m sample points, and its evaluation: the analytic
 * continuation of data on the imaginary axis to other complex frequencies.  Per function:
 * the first approximant is the mean of the samples; each step adds the sample with the
 * largest deviation (the first on ties) to the support set and takes the barycentric weights
 * from the right singular vector of the Loewner matrix for its smallest singular value
 * (one-sided Jacobi SVD in FP64); it stops when the largest deviation on the other samples
 * is <= tol max|f|, at mmax support points, or when no sample is left.
 *   z       complex [m] host, distinct finite sample points; m <= 128.
 *   f       complex [nfun][m] (host or device) samples.   mmax <= 32.
 *   z_eval  complex [n_eval] host; r_eval complex [nfun][n_eval] (host or device), the
 *           approximant there (the sample value where a point is a support point).
 *   degree  [nfun] (host or device) or NULL: support points used.
 * A function with a non-finite sample gets NaN outputs and the call returns SGW_EINVAL. */
sgw_status sgw_aaa(int nfun, int m, const void* z, const void* f, double tol, int mmax, int n_eval,
                   const void* z_eval, void* r_eval, int* degree, void* stream);

/* Screening from an accumulated density response (Sec. 2.4, Eq. 4 and 9, with the Coulomb
 * potential of Sec. 2.6).  Per frequency j:
 *   v(q)          = 4 pi / |q|^2 [1 - cos(|q| r_cut)]   (spherical truncation; its limit
 *                   2 pi r_cut^2 at q = 0; the bare 4 pi / |q|^2 when r_cut <= 0; Hartree units)
 *   eps[G][G']    = delta - dn[G][G'][j] v(q + G') / volume   (the response to the Coulomb
 *                   potential of a unit plane-wave charge at q + G')
 *   eps_inv       = eps^-1 by Gauss-Jordan elimination with partial pivoting in FP64; rows and
 *                   columns with q + G = 0 keep only their diagonal
 *   wbar[G][G'][j] = v(q + G) (eps_inv[G][G'] - delta)
 *   dn       complex [n_g][n_g][nomega] (host or device): sgw_density_response's output summed
 *            over k-points (weights included).
 *   qg       [n_g][3] host: the Cartesian vectors q + G (bohr^-1) of the perturbations, in the
 *            order of dn's rows.   volume: cell volume (bohr^3) > 0.
 *   eps_inv  complex [n_g][n_g][nomega] (host or device) or NULL; wbar likewise, required.
 * n_g <= 64 (else SGW_EUNSUPPORTED).  q + G = 0 with r_cut <= 0 is SGW_EINVAL.  A singular
 * eps at some frequency gives NaN outputs for it and SGW_ENOCONV. */
sgw_status sgw_screened_coulomb(int n_g, int nomega, const void* dn, const double* qg, double volume, double r_cut,
                                void* eps_inv, void* wbar, void* stream);

/* True FP64 residual of given solutions: for every pair
 *   r = -P_c rhs - (P_c H P_c - z) dpsi,  rel_res = |r| / |P_c rhs|,  cert = |r| / (eta |dpsi|).
 * Since P_c H P_c - z is normal with every eigenvalue at distance >= eta from 0, cert bounds
 * the relative error |dpsi - dpsi*| / |dpsi|.  rel_res, cert: host [nrhs][nomega] (either may be NULL). */
sgw_status sgw_residual(sgw_system* sys, int nrhs, const void* rhs, const double* e_ref, int nomega,
                        const double* omega, double eta, const void* dpsi, double* rel_res,
                        double* cert, void* stream);

/* Allocation-free variant of sgw_residual (the paper has no counterpart: this serves
 * callers that cannot let a library allocate device memory, e.g. a framework whose caching
 * allocator or fixed arena owns all device memory, or a code path that must not pay the
 * device-wide synchronisation cudaFree can imply).  Same results as sgw_residual, but:
 *   - every array argument (rhs, e_ref, omega, dpsi, rel_res, cert) must be device memory of
 *     the system's device, or managed memory (else SGW_EINVAL: host memory and other GPUs'
 *     memory are refused before anything is launched); rel_res and cert are written on the
 *     device; nrhs * nomega must not exceed INT_MAX (else SGW_EUNSUPPORTED);
 *   - the calling thread's current device is the same after the call as before it;
 *   - it calls no cudaMalloc / cudaFree: its scratch (2 * n_pw complex values per CTA) is a
 *     built-in device array of SGW_NOALLOC_SCRATCH_BYTES, held by every GPU that loads the
 *     library until the process exits; n_pw > SGW_NOALLOC_SCRATCH_BYTES / 32 gives
 *     SGW_EUNSUPPORTED;
 *   - the first call on a device looks up that array's device address, so make the first
 *     call on each device before any stream capture;
 *   - all calls share the array: calls that overlap on the GPU (other streams, other host
 *     threads) race and must be serialised by the caller;
 *   - it is asynchronous on `stream`: results are ready when the stream is. */
#define SGW_NOALLOC_SCRATCH_BYTES ((size_t)4 << 20)
sgw_status sgw_residual_noalloc(sgw_system* sys, int nrhs, const void* rhs, const double* e_ref, int nomega,
                                const double* omega, double eta, const void* dpsi, double* rel_res,
                                double* cert, void* stream);

/* ---------------------------------------------------------------------------------------
 * Per-shift solves with a diagonal preconditioner.  The paper does not say how its linear
 * systems are preconditioned; this part is an addition.  A preconditioner breaks the shift
 * invariance the multishift pass relies on, so it acts on single-shift systems: pairs that
 * are solved one by one (stragglers, correction equations).  Pair i solves
 * (P_c H P_c - z_i) x_i = -P_c rhs_i, z_i = e_ref[i] + omega[i] + i eta, by BiCGstab(ell)
 * right-preconditioned with a positive diagonal D:
 *   SGW_PRECOND_PLAIN    M_G = 1 / max(1, T_G / e_prec), e_prec = 1.35 <r|T|r> / <r|r> of the
 *                        pair's right-hand side r (a kinetic-energy scaling);
 *   SGW_PRECOND_JACOBI   J_G = 1 / max(|H_GG - z_i|, delta_i), H_GG = T_G + <V_loc> +
 *                        sum_p D_p |beta_p(G)|^2 (delta_i from the `delta` array);
 *   SGW_PRECOND_LEARNED  M_G exp(f(phi_G)), phi_G = (T_G / (E_cut / 2), omega / 2.205 Ha, e_ref,
 *                        <V_loc>), f the perceptron of an sgw_mlp trained to predict
 *                        log(J_G / M_G) at the floor that solved training pairs fastest.
 * The Krylov residual decides convergence, so D changes iteration counts, never the answer.
 * --------------------------------------------------------------------------------------- */
enum { SGW_PRECOND_NONE = 0, SGW_PRECOND_PLAIN = 1, SGW_PRECOND_LEARNED = 2, SGW_PRECOND_JACOBI = 3 };

/* The perceptron 4 -> 64 -> 64 -> 1 with erf-GELU activations (4545 FP32 master parameters,
 * packed w1[64][4], b1[64], w2[64][64], b2[64], w3[64], b3), evaluated with bfloat16 weights
 * and FP32 accumulation; trained with Adam (beta 0.9 / 0.999, eps 1e-8) on a mean squared
 * error.  Row arrays (feats [n][4], targets [n], weight [n], out [n]) are FP32 device buffers. */
#define SGW_MLP_PARAMS 4545
sgw_status sgw_mlp_create(const float* params /* host [4545] */, sgw_mlp** out);
sgw_status sgw_mlp_get_params(const sgw_mlp* mlp, float* params /* host [4545] */);
sgw_status sgw_mlp_forward(const sgw_mlp* mlp, int n, const float* feats, float* out, void* stream);
/* Loss mean_i weight_i (f_i - target_i)^2 (weight NULL -> 1) and its gradient (host [4545]). */
sgw_status sgw_mlp_grad(sgw_mlp* mlp, int n, const float* feats, const float* targets, const float* weight,
                        float* grad, float* loss, void* stream);
/* One Adam step on that loss; *loss receives the loss before the step. */
sgw_status sgw_mlp_train_step(sgw_mlp* mlp, int n, const float* feats, const float* targets,
                              const float* weight, float lr, float* loss, void* stream);
void sgw_mlp_destroy(sgw_mlp* mlp);

/* Per-shift preconditioned solves of npairs independent pairs.  rhs, x: complex
 * [npairs][n_pw] (host or device); e_ref, omega (and delta for JACOBI): host [npairs];
 * precond SGW_PRECOND_*; mlp required for SGW_PRECOND_LEARNED.  opts: ell, max_matvec and
 * stream are used.  report arrays are [npairs]; rel_res and cert are the FP64 true residual
 * and certificate. */
sgw_status sgw_solve_pershift(sgw_system* sys, int npairs, const void* rhs, const double* e_ref,
                              const double* omega, double eta, double tol, int precond, const double* delta,
                              const sgw_mlp* mlp, const sgw_solve_opts* opts, void* x, sgw_report* report);

/* The diagonal D of each pair (test hook): d [npairs][n_pw] FP64 (host or device). */
sgw_status sgw_precond_diag(sgw_system* sys, int npairs, const void* rhs, const double* e_ref,
                            const double* omega, double eta, int precond, const double* delta,
                            const sgw_mlp* mlp, double* d, void* stream);

/* Training rows of the learned preconditioner, one row per plane wave of each pair: features
 * phi_G and target log(clip(J_G / M_G, e^-3, e^3)) at the pair's best Jacobi floor delta[i]
 * (host [npairs]; delta <= 0 means the plain scaling was best: target 0).  rhs complex
 * [npairs][n_pw] device; feats [npairs * n_pw][4] and targets [npairs * n_pw] FP32 device. */
sgw_status sgw_training_rows(sgw_system* sys, int npairs, const void* rhs, const double* e_ref,
                             const double* omega, double eta, const double* delta, float* feats,
                             float* targets, void* stream);

/* Releases a system and every device buffer it owns (resource management of this ABI; the
 * paper has no counterpart).  NULL is a no-op.  It makes the system's device current and
 * synchronises it first, so work still in flight on the system finishes before its memory is
 * freed. */
void sgw_destroy_system(sgw_system* sys);

/* Message of the last failing call on this host thread ("" if none); the pointer stays
 * valid until the thread's next call into the library (error reporting of this ABI; the
 * paper has no counterpart). */
const char* sgw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGW_H */
