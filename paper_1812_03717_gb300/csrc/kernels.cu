// Hot kernels: the multishift BiCGstab(ell) solve of the Sternheimer equation (Eq. 6 with
// the operator of Eq. 7), the H application test hook and the true-residual certificate.
//
// Solver organisation.  One CTA owns one right-hand side at a time (a work queue hands
// them out) and runs its whole Krylov iteration: every H application, dot product,
// recurrence scalar and shift update of that right-hand side happens inside the CTA, so
// the iteration needs no grid-wide synchronisation and no host round trips.  Seed vectors
// live in a per-CTA slice of global memory (L2-resident), shift vectors x_j and u_j in
// the caller's output and in a per-CTA workspace.
//
// Method (shifted BiCGstab(ell) for families of shifted systems, the Krylov solver the
// paper cites for "all frequencies at the cost of one", Sec. 2.2).  The seed system is
// A_0 = P_c H P_c - z_s; shift j solves (A_0 + sigma_j) x_j = b with sigma_j = z_s - z_j.
// With phi_n the BiCG residual polynomials of the seed and zeta_n^j = phi_n(-sigma_j),
//   zeta_{n+1} = (1 + alpha_n beta_{n-1}/alpha_{n-1} + alpha_n sigma) zeta_n
//                - (alpha_n beta_{n-1}/alpha_{n-1}) zeta_{n-1},
//   alpha_n^j = alpha_n zeta_n / zeta_{n+1},   beta_{n-1}^j = beta_{n-1} (zeta_{n-1}/zeta_n)^2,
// and every minimal-residual polynomial q(l) = 1 - sum_i gamma_i l^i of the seed becomes
// q^j(mu) = q(mu - sigma_j) / q(-sigma_j) for shift j.  Residuals of all shifts stay
// collinear with the seed's, r^j = r / (Psi^j zeta^j) with Psi^j the product of the
// q(-sigma_j); each shift keeps only x_j and its direction u_j, and the powers
// A_j^t r^j, A_j^t u_j it needs are expanded binomially in the seed's R_t = A_0^t r and
// U_t = A_0^t u.
#include <cuda_runtime.h>

#include "mlp.cuh"
#include "setup.h"
#include "sgw_internal.cuh"

namespace sgw {

namespace {

// Per-shift state in shared memory.
struct ShiftSmem {
    int zp, zc, psi, zn, as, bs, cr, las, cx, ca, cb, sig, est, st, mv, act, end;
};

__host__ __device__ inline ShiftSmem shift_layout(int base, int ns) {
    ShiftSmem s;
    int off = base;
    s.zp = off;  off = align16(off + ns * 16);
    s.zc = off;  off = align16(off + ns * 16);
    s.psi = off; off = align16(off + ns * 16);
    s.zn = off;  off = align16(off + ns * 16);
    s.as = off;  off = align16(off + ns * 16);
    s.bs = off;  off = align16(off + ns * 16);
    s.cr = off;  off = align16(off + ns * 16);
    s.las = off; off = align16(off + ns * 16);
    s.cx = off;  off = align16(off + ns * kMaxEll * 16);
    s.ca = off;  off = align16(off + ns * kMaxEll * 16);
    s.cb = off;  off = align16(off + ns * kMaxEll * 16);
    s.sig = off; off = align16(off + ns * 8);
    s.est = off; off = align16(off + ns * 8);
    s.st = off;  off = align16(off + ns * 4);
    s.mv = off;  off = align16(off + ns * 4);
    s.act = off; off = align16(off + ns * 4);
    s.end = off;
    return s;
}

struct SeedScalars {
    double2 rho0, alpha, omega, alpha_prev, beta;
    double2 gam[kMaxEll];
    double bnorm, rnorm;
    int first, nact, fail;
};

__device__ __forceinline__ int binom(int n, int k) {
    // n <= 4
    const int t[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    return t[n][k];
}

// Solves the ell x ell Hermitian system M g = v (complex, FP64) by Gaussian elimination
// with partial pivoting.  Returns false on a zero pivot.
__device__ bool small_solve(double2 (&M)[kMaxEll][kMaxEll], double2 (&v)[kMaxEll], int n, double2 (&g)[kMaxEll]) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = cabs2(M[c][c]);
        for (int r = c + 1; r < n; ++r)
            if (cabs2(M[r][c]) > best) { best = cabs2(M[r][c]); piv = r; }
        if (!(best > 0.0)) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double2 t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
            double2 t = v[c]; v[c] = v[piv]; v[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double2 f = cdiv(M[r][c], M[c][c]);
            for (int k = c; k < n; ++k) M[r][k] = csub(M[r][k], cmul(f, M[c][k]));
            v[r] = csub(v[r], cmul(f, v[c]));
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double2 s = v[r];
        for (int k = r + 1; k < n; ++k) s = csub(s, cmul(M[r][k], g[k]));
        g[r] = cdiv(s, M[r][r]);
    }
    return true;
}

__device__ __forceinline__ double2 cpowr(double2 a, int e) {
    double2 r = make_double2(1.0, 0.0);
    for (int i = 0; i < e; ++i) r = cmul(r, a);
    return r;
}

}  // namespace

// Dots out[v] = sum_g conj(V[v ld + g]) x[g], v < nv, over the vector's owners: the CTA's
// block dots when one CTA holds the box, the warp-split dots and the rank-ordered cluster sum
// when the box is split over a cluster.
__device__ __forceinline__ void owner_dots(const Plan& P, const Part& q, Red& Rd, const double2* V, int nv, int ld,
                                           const double2* x, double2* out) {
    if (P.csize == 1) block_dots(V, nv, ld, x, P.npw, Rd.red, out);
    else part_dots_f64(P, q, Rd, V, nv, ld, x, out);
}

// out = A D in with A = P_c H P_c - z and D = diag(pre) (right preconditioning of a
// single-shift system): T1 = D in, T2 = P_c T1, out = P_c H T2 - z T1.  Without `pre` the
// Krylov vectors already lie in range(P_c) and out = P_c H in - z in.  Each rank of a
// cluster reads and writes its own plane waves [q.g0, q.g1) of every vector only.
static __device__ void apply_op(const Plan& P, unsigned char* smem, const Part& q, Red& Rd, const double2* in,
                                double2* out, double2 zs, const double* pre, double2* t1, double2* t2) {
    if (!pre) {
        apply_h_block<ArF64>(P, smem, q, Rd, in, out, zs, APPLY_PROJ_OUT | APPLY_SUB_Z);
        return;
    }
    const ApplySmem L = apply_smem_layout(P, 16);
    double2* coef = reinterpret_cast<double2*>(smem + L.coef);
    const int npw = P.npw, tid = threadIdx.x, nt = blockDim.x, g0 = q.g0, g1 = q.g1;
    for (int g = g0 + tid; g < g1; g += nt) t1[g] = cscal(in[g], pre[g]);
    __syncthreads();
    owner_dots(P, q, Rd, P.psi, P.nocc, npw, t1, coef);
    for (int g = g0 + tid; g < g1; g += nt) {
        double2 h = t1[g];
        for (int v = 0; v < P.nocc; ++v) h = csub(h, cmul(coef[v], P.psi[(size_t)v * npw + g]));
        t2[g] = h;
    }
    __syncthreads();
    apply_h_block<ArF64>(P, smem, q, Rd, t2, out, cz(), APPLY_PROJ_OUT);
    for (int g = g0 + tid; g < g1; g += nt) out[g] = csub(out[g], cmul(zs, t1[g]));
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) ms_solve_kernel(Plan P, SolveArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SeedScalars S;
    __shared__ double2 s_dot[kRedSlots];

    load_twiddles<ArF64>(P, smem);
    const ApplySmem L = apply_smem_layout(P, 16);
    Red Rd = make_red(P, smem, L);
    const Part q = make_part(P);
    double2* coef = reinterpret_cast<double2*>(smem + L.coef);
    const int ns = A.nshift, ell = A.ell, npw = P.npw;
    const int g0 = q.g0, g1 = q.g1;
    const ShiftSmem Q = shift_layout(L.end, ns);
    double2* zp = reinterpret_cast<double2*>(smem + Q.zp);
    double2* zc = reinterpret_cast<double2*>(smem + Q.zc);
    double2* Psi = reinterpret_cast<double2*>(smem + Q.psi);
    double2* zn = reinterpret_cast<double2*>(smem + Q.zn);
    double2* as = reinterpret_cast<double2*>(smem + Q.as);
    double2* bs = reinterpret_cast<double2*>(smem + Q.bs);
    double2* cr = reinterpret_cast<double2*>(smem + Q.cr);
    double2* las = reinterpret_cast<double2*>(smem + Q.las);
    double2* cx = reinterpret_cast<double2*>(smem + Q.cx);
    double2* ca = reinterpret_cast<double2*>(smem + Q.ca);
    double2* cb = reinterpret_cast<double2*>(smem + Q.cb);
    double* sig = reinterpret_cast<double*>(smem + Q.sig);
    double* est = reinterpret_cast<double*>(smem + Q.est);
    int* st = reinterpret_cast<int*>(smem + Q.st);
    int* mv = reinterpret_cast<int*>(smem + Q.mv);
    int* act = reinterpret_cast<int*>(smem + Q.act);

    const int tid = threadIdx.x, nt = blockDim.x;
    const int own = blockIdx.x / P.csize;   // the owner (CTA, or cluster) of the workspace slices
    double2* W = A.seedw + (size_t)own * (2 * ell + 3) * npw;
    double2* R[kMaxEll + 1];
    double2* U[kMaxEll + 1];
    for (int i = 0; i <= kMaxEll; ++i) {
        R[i] = W + (size_t)min(i, ell) * npw;
        U[i] = W + (size_t)(ell + 1 + min(i, ell)) * npw;
    }
    double2* RT = W + (size_t)(2 * ell + 2) * npw;
    double2* UW = A.uw + (size_t)own * ns * npw;
    double2* T1 = A.pscr ? A.pscr + (size_t)own * 2 * npw : nullptr;
    double2* T2 = T1 ? T1 + npw : nullptr;
    for (int j = tid; j < ns; j += nt) sig[j] = A.sig[j];

    for (;;) {
        const int r = next_item(P, A.counter);
        if (r >= A.nrhs) break;
        const double2* rhs = A.rhs + (size_t)r * npw;
        double2* X = A.x + (size_t)r * ns * npw;
        const double2 zs = make_double2(A.e_ref[r] + A.omega_seed, A.eta);
        const double* pre = A.pre ? A.pre + (size_t)r * npw : nullptr;   // single-shift systems only

        // b = -P_c rhs (Eq. 8 with the sign of the problem statement)
        owner_dots(P, q, Rd, P.psi, P.nocc, npw, rhs, coef);
        {
            double2 acc[1] = {cz()};
            for (int g = g0 + tid; g < g1; g += nt) {
                double2 h = rhs[g];
                for (int v = 0; v < P.nocc; ++v) h = csub(h, cmul(coef[v], P.psi[(size_t)v * npw + g]));
                const double2 b = make_double2(-h.x, -h.y);
                R[0][g] = b;
                RT[g] = b;
                U[0][g] = cz();
                acc[0].x += cabs2(b);
            }
            part_sum<1>(P, Rd, acc, s_dot);
        }
        for (int j = 0; j < ns; ++j)
            for (int g = g0 + tid; g < g1; g += nt) {
                X[(size_t)j * npw + g] = cz();
                UW[(size_t)j * npw + g] = cz();
            }
        if (tid == 0) {
            S.bnorm = sqrt(s_dot[0].x);
            S.rho0 = make_double2(1.0, 0.0);
            S.alpha = cz();
            S.omega = make_double2(1.0, 0.0);
            S.alpha_prev = make_double2(1.0, 0.0);
            S.first = 1;
            S.fail = isfinite(S.bnorm) ? 0 : SGW_PAIR_NONFINITE;
            S.nact = (S.bnorm > 0.0 && S.fail == 0) ? ns : 0;
        }
        for (int j = tid; j < ns; j += nt) {
            zp[j] = zc[j] = Psi[j] = make_double2(1.0, 0.0);
            las[j] = make_double2(1.0, 0.0);
            st[j] = -1;
            mv[j] = 0;
            est[j] = 1.0;
            act[j] = j;
        }
        __syncthreads();
        if (S.nact == 0) {
            // zero right-hand side: dpsi = 0 exactly; a non-finite one is reported as such
            for (int j = tid; j < ns; j += nt) {
                st[j] = S.fail ? S.fail : SGW_PAIR_CONVERGED;
                est[j] = S.fail ? NAN : 0.0;
            }
        }
        int mvc = 0;

        while (S.nact > 0 && S.fail == 0 && mvc + 2 * ell <= A.max_mv) {
            if (tid == 0) S.rho0 = make_double2(-(S.omega.x * S.rho0.x - S.omega.y * S.rho0.y),
                                                -(S.omega.x * S.rho0.y + S.omega.y * S.rho0.x));
            __syncthreads();
            // ---------------------------------------------------------------- BiCG part
            for (int j = 0; j < ell; ++j) {
                owner_dots(P, q, Rd, RT, 1, 0, R[j], s_dot);
                if (tid == 0) {
                    const double2 rho1 = s_dot[0];
                    S.beta = cdiv(cmul(S.alpha, rho1), S.rho0);
                    S.rho0 = rho1;
                    if (!cfinite(S.beta) || (rho1.x == 0.0 && rho1.y == 0.0)) S.fail = SGW_PAIR_BREAKDOWN;
                }
                __syncthreads();
                if (S.fail) break;
                {
                    const double2 be = S.beta;
                    for (int g = g0 + tid; g < g1; g += nt)
                        for (int i = 0; i <= j; ++i) U[i][g] = csub(R[i][g], cmul(be, U[i][g]));
                }
                __syncthreads();
                apply_op(P, smem, q, Rd, U[j], U[j + 1], zs, pre, T1, T2);
                owner_dots(P, q, Rd, RT, 1, 0, U[j + 1], s_dot);
                if (tid == 0) {
                    const double2 gam = s_dot[0];
                    if (gam.x == 0.0 && gam.y == 0.0) S.fail = SGW_PAIR_BREAKDOWN;
                    else S.alpha = cdiv(S.rho0, gam);
                    if (!cfinite(S.alpha)) S.fail = SGW_PAIR_NONFINITE;
                }
                __syncthreads();
                if (S.fail) break;
                // shift scalars of this BiCG step
                {
                    const double2 al = S.alpha;
                    const double2 bb = S.first ? cz() : make_double2(-S.beta.x, -S.beta.y);
                    const double2 cf = S.first ? cz() : cdiv(cmul(al, bb), S.alpha_prev);
                    for (int a = tid; a < S.nact; a += nt) {
                        const int k = act[a];
                        const double2 one_c = make_double2(1.0 + cf.x + al.x * sig[k], cf.y + al.y * sig[k]);
                        const double2 znk = csub(cmul(one_c, zc[k]), cmul(cf, zp[k]));
                        zn[k] = znk;
                        as[k] = cdiv(cmul(al, zc[k]), znk);
                        const double2 q = cdiv(zp[k], zc[k]);
                        bs[k] = S.first ? cz() : cmul(bb, cmul(q, q));
                        cr[k] = cdiv(make_double2(1.0, 0.0), cmul(Psi[k], zc[k]));
                        if (!cfinite(as[k]) || !cfinite(bs[k]) || !cfinite(cr[k])) st[k] = SGW_PAIR_NONFINITE;
                    }
                }
                __syncthreads();
                // shift pass: u_j <- cr r + bs u_j ;  x_j <- x_j + as u_j
                {
                    const int na = S.nact;
                    for (int g = g0 + tid; g < g1; g += nt) {
                        const double2 r0 = R[0][g];
                        for (int a = 0; a < na; ++a) {
                            const int k = act[a];
                            if (st[k] >= 0) continue;
                            double2* up = UW + (size_t)k * npw + g;
                            double2* xp = X + (size_t)k * npw + g;
                            const double2 u = cfma(cr[k], r0, cmul(bs[k], *up));
                            *up = u;
                            *xp = cfma(as[k], u, *xp);
                        }
                    }
                }
                __syncthreads();
                {
                    const double2 al = S.alpha;
                    for (int g = g0 + tid; g < g1; g += nt)
                        for (int i = 0; i <= j; ++i) R[i][g] = csub(R[i][g], cmul(al, U[i + 1][g]));
                }
                __syncthreads();
                apply_op(P, smem, q, Rd, R[j], R[j + 1], zs, pre, T1, T2);
                for (int a = tid; a < S.nact; a += nt) {
                    const int k = act[a];
                    zp[k] = zc[k];
                    zc[k] = zn[k];
                    las[k] = as[k];
                }
                if (tid == 0) {
                    S.alpha_prev = S.alpha;
                    S.first = 0;
                }
                mvc += 2;
                __syncthreads();
            }
            if (S.fail) break;

            // ------------------------------------------------------------------ MR part
            {
                // Gram entries <R_i, R_k>, 1 <= i <= k <= ell, and <R_i, R_0>
                double2 acc[14];
#pragma unroll
                for (int i = 0; i < 14; ++i) acc[i] = cz();
                for (int g = g0 + tid; g < g1; g += nt) {
                    double2 rv[kMaxEll + 1];
#pragma unroll
                    for (int t = 0; t <= kMaxEll; ++t) rv[t] = t <= ell ? R[t][g] : cz();
                    int q = 0;
#pragma unroll
                    for (int i = 1; i <= kMaxEll; ++i) {
#pragma unroll
                        for (int k = i; k <= kMaxEll; ++k) {
                            acc[q] = cadd(acc[q], cmulc(rv[i], rv[k]));
                            ++q;
                        }
                    }
#pragma unroll
                    for (int i = 1; i <= kMaxEll; ++i) acc[9 + i] = cadd(acc[9 + i], cmulc(rv[i], rv[0]));
                }
                // 10 Gram entries (indices 0..9) + 4 projections (10..13)
                part_sum<14>(P, Rd, acc, s_dot);
                if (tid == 0) {
                    double2 M[kMaxEll][kMaxEll], v[kMaxEll], g[kMaxEll];
                    int q = 0;
                    for (int i = 1; i <= kMaxEll; ++i)
                        for (int k = i; k <= kMaxEll; ++k) {
                            const double2 e = s_dot[q++];
                            if (i <= ell && k <= ell) {
                                M[i - 1][k - 1] = e;
                                M[k - 1][i - 1] = make_double2(e.x, -e.y);
                            }
                        }
                    for (int i = 1; i <= ell; ++i) v[i - 1] = s_dot[9 + i];
                    if (!small_solve(M, v, ell, g)) {
                        S.fail = SGW_PAIR_BREAKDOWN;
                    } else {
                        for (int i = 0; i < ell; ++i) S.gam[i] = g[i];
                        S.omega = g[ell - 1];
                        if (!cfinite(S.omega) || (S.omega.x == 0.0 && S.omega.y == 0.0)) S.fail = SGW_PAIR_BREAKDOWN;
                    }
                }
                __syncthreads();
                if (S.fail) break;
            }
            // per-shift coefficients of the MR update
            for (int a = tid; a < S.nact; a += nt) {
                const int k = act[a];
                const double2 sg = make_double2(sig[k], 0.0);
                const double2 msg = make_double2(-sig[k], 0.0);
                // c_m: coefficients of q(mu - sigma) = 1 - sum_i gamma_i (mu - sigma)^i
                double2 c[kMaxEll + 1];
                c[0] = make_double2(1.0, 0.0);
                for (int m = 1; m <= ell; ++m) c[m] = cz();
                for (int i = 1; i <= ell; ++i)
                    for (int m = 0; m <= i; ++m)
                        c[m] = csub(c[m], cscal(cmul(S.gam[i - 1], cpowr(msg, i - m)), (double)binom(i, m)));
                const double2 q0 = c[0];
                double2 gs[kMaxEll];
                for (int i = 1; i <= ell; ++i) gs[i - 1] = cdiv(make_double2(-c[i].x, -c[i].y), q0);
                const double2 rsc = cdiv(make_double2(1.0, 0.0), cmul(Psi[k], zc[k]));
                const double2 rpre = cdiv(make_double2(1.0, 0.0), cmul(Psi[k], zp[k]));
                const double2 aa = cdiv(csub(rpre, rsc), las[k]);
                const double2 bc = cdiv(cmul(rpre, S.alpha_prev), las[k]);
                for (int t = 0; t < ell; ++t) {
                    double2 d = cz();
                    for (int i = t + 1; i <= ell; ++i)
                        d = cadd(d, cscal(cmul(gs[i - 1], cpowr(sg, i - 1 - t)), (double)binom(i - 1, t)));
                    cx[k * kMaxEll + t] = cmul(rsc, d);
                    ca[k * kMaxEll + t] = cmul(d, aa);
                    cb[k * kMaxEll + t] = cmul(d, bc);
                }
                Psi[k] = cmul(Psi[k], q0);
                if (!cfinite(q0) || !cfinite(aa) || !cfinite(bc)) st[k] = SGW_PAIR_NONFINITE;
            }
            __syncthreads();
            // MR pass: shifts, then the seed's R_0 and U_0
            {
                const int na = S.nact;
                double2 acc[1] = {cz()};
                for (int g = g0 + tid; g < g1; g += nt) {
                    double2 rv[kMaxEll + 1], uv[kMaxEll + 1];
#pragma unroll
                    for (int t = 0; t <= kMaxEll; ++t) {
                        rv[t] = t <= ell ? R[t][g] : cz();
                        uv[t] = t <= ell ? U[t][g] : cz();
                    }
                    for (int a = 0; a < na; ++a) {
                        const int k = act[a];
                        if (st[k] >= 0) continue;
                        double2* up = UW + (size_t)k * npw + g;
                        double2* xp = X + (size_t)k * npw + g;
                        double2 xv = *xp, u = *up;
#pragma unroll
                        for (int t = 0; t < kMaxEll; ++t) {
                            if (t < ell) {
                                xv = cfma(cx[k * kMaxEll + t], rv[t], xv);
                                u = csub(u, cadd(cmul(ca[k * kMaxEll + t], rv[t]), cmul(cb[k * kMaxEll + t], uv[t + 1])));
                            }
                        }
                        *xp = xv;
                        *up = u;
                    }
                    double2 r0 = rv[0], u0 = uv[0];
#pragma unroll
                    for (int i = 1; i <= kMaxEll; ++i) {
                        if (i <= ell) {
                            r0 = csub(r0, cmul(S.gam[i - 1], rv[i]));
                            u0 = csub(u0, cmul(S.gam[i - 1], uv[i]));
                        }
                    }
                    R[0][g] = r0;
                    U[0][g] = u0;
                    acc[0].x += cabs2(r0);
                }
                part_sum<1>(P, Rd, acc, s_dot);
            }
            if (tid == 0) S.rnorm = sqrt(s_dot[0].x);
            __syncthreads();
            // convergence of each shift from the collinear residual; renormalise zeta
            for (int a = tid; a < S.nact; a += nt) {
                const int k = act[a];
                if (st[k] >= 0) { mv[k] = mvc; continue; }
                const double2 sc = cmul(Psi[k], zc[k]);
                const double e = S.rnorm / (sqrt(cabs2(sc)) * S.bnorm);
                est[k] = e;
                if (!isfinite(e)) {
                    st[k] = SGW_PAIR_NONFINITE;
                    mv[k] = mvc;
                } else if (e <= A.tol) {
                    st[k] = SGW_PAIR_CONVERGED;
                    mv[k] = mvc;
                }
                const double2 f = zc[k];
                zc[k] = make_double2(1.0, 0.0);
                zp[k] = cdiv(zp[k], f);
                Psi[k] = cmul(Psi[k], f);
            }
            __syncthreads();
            if (tid == 0) {
                int n = 0;
                for (int a = 0; a < S.nact; ++a)
                    if (st[act[a]] < 0) act[n++] = act[a];
                S.nact = n;
            }
            __syncthreads();
        }
        __syncthreads();
        if (pre) {   // the iterate solves A D y = b: x = D y
            for (int g = g0 + tid; g < g1; g += nt) X[g] = cscal(X[g], pre[g]);
        }
        if (q.rank == 0) {   // every rank holds the same per-shift results; rank 0 writes them
            for (int j = tid; j < ns; j += nt) {
                int s = st[j];
                if (s < 0) {
                    s = S.fail ? S.fail : SGW_PAIR_MAXITER;
                    mv[j] = mvc;
                }
                A.out_status[(size_t)r * ns + j] = s;
                A.out_mv[(size_t)r * ns + j] = mv[j];
                A.out_res[(size_t)r * ns + j] = est[j];
            }
        }
    }
}

// y_i = H x_i, or (P_c H P_c - z_i) x_i when `project` is set.  One CTA or cluster per vector
// (persistent over the batch); scratch holds the input and output in the policy's format
// per owner.
template <class Ar>
__global__ void __launch_bounds__(kThreads, 1) apply_kernel(Plan P, int nvec, const double2* __restrict__ x,
                                                            double2* __restrict__ y, const double2* __restrict__ z,
                                                            int project, double2* __restrict__ scratch) {
    using C = typename Ar::C;
    extern __shared__ __align__(16) unsigned char smem[];
    load_twiddles<Ar>(P, smem);
    const ApplySmem L = apply_smem_layout(P, (int)sizeof(C));
    Red R = make_red(P, smem, L);
    double2* coef = reinterpret_cast<double2*>(smem + L.coef);
    const Part q = make_part(P);
    const int npw = P.npw, tid = threadIdx.x, nt = blockDim.x;
    const int cl_id = blockIdx.x / P.csize, ncl = gridDim.x / P.csize;
    C* xa = reinterpret_cast<C*>(scratch + (size_t)cl_id * 2 * npw);         // input in the policy's format
    C* ya = reinterpret_cast<C*>(scratch + (size_t)cl_id * 2 * npw + npw);   // output in the policy's format
    for (int v = cl_id; v < nvec; v += ncl) {
        const double2* xv = x + (size_t)v * npw;
        double2* yv = y + (size_t)v * npw;
        if (project) {
            part_dots_f64(P, q, R, P.psi, P.nocc, npw, xv, coef);
            for (int g = q.g0 + tid; g < q.g1; g += nt) {
                double2 h = xv[g];
                for (int o = 0; o < P.nocc; ++o) h = csub(h, cmul(coef[o], P.psi[(size_t)o * npw + g]));
                xa[g] = Ar::from_d(h);
            }
        } else {
            for (int g = q.g0 + tid; g < q.g1; g += nt) xa[g] = Ar::from_d(xv[g]);
        }
        __syncthreads();
        apply_h_block<Ar>(P, smem, q, R, xa, ya, cz(), project ? APPLY_PROJ_OUT : 0);
        const double2 zz = project ? z[v] : cz();
        for (int g = q.g0 + tid; g < q.g1; g += nt) yv[g] = csub(Ar::to_d(ya[g]), cmul(zz, xv[g]));
        __syncthreads();
    }
}

// For every listed pair p = r * ns + j (all pairs when list is NULL):
//   res = -P_c rhs_r - (P_c H P_c - z_rj) x_rj,
//   rel[p] = |res| / |P_c rhs_r|,  cert[p] = |res| / (|Im z_rj| |x_rj|),
// and, when store is given, store[i] = -res (the right-hand side of the correction
// equation in the solver's convention b = -P_c rhs).  With `clean` set, x_rj is first
// replaced by P_c x_rj (the solution lies in range(P_c), and the correction solves act there
// only: an occupied component -- rounding of a single-precision pass, or a caller's initial
// guess -- is removed exactly instead of being left in the residual).  The projections, the
// assembly of res and the norms are FP64; H (P_c x) is applied in the policy Ar (FP64, or
// float-float with a relative error near 1e-14).  One CTA or cluster per pair; scratch: 2 n_pw
// values per owner.
template <class Ar>
__global__ void __launch_bounds__(kResThreads, 1) residual_kernel(Plan P, int nrhs, int ns, const int* __restrict__ list,
                                                               int nlist, const double2* __restrict__ rhs,
                                                               const double* __restrict__ e_ref,
                                                               const double* __restrict__ omega, double eta,
                                                               double2* __restrict__ x,
                                                               double2* __restrict__ scratch, double* __restrict__ rel,
                                                               double* __restrict__ cert, double2* __restrict__ store,
                                                               const double* __restrict__ eta_s,
                                                               const double2* __restrict__ bvec, int clean) {
    using C = typename Ar::C;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double2 s_dot[kRedSlots];
    load_twiddles<Ar>(P, smem);
    const ApplySmem L = apply_smem_layout(P, (int)sizeof(C));
    Red R = make_red(P, smem, L);
    double2* coef = reinterpret_cast<double2*>(smem + L.coef);
    const Part q = make_part(P);
    const int npw = P.npw, tid = threadIdx.x, nt = blockDim.x;
    const int cl_id = blockIdx.x / P.csize, ncl = gridDim.x / P.csize;
    double2* xs = scratch + (size_t)cl_id * 2 * npw;   // P_c x, stored in the policy's format
    double2* ys = xs + npw;                             // H P_c x in the policy's format
    C* xa = reinterpret_cast<C*>(xs);
    C* ya = reinterpret_cast<C*>(ys);
    const int count = list ? nlist : nrhs * ns;
    for (int i = cl_id; i < count; i += ncl) {
        const int pq = list ? list[i] : i;
        const int r = pq / ns, j = pq % ns;
        double2* xv = x + (size_t)pq * npw;
        const double2* rv = rhs + (size_t)r * npw;
        const double2 z = make_double2(e_ref[r] + omega[j], eta_s ? eta_s[j] : eta);
        part_dots_f64(P, q, R, P.psi, P.nocc, npw, xv, coef);
        for (int g = q.g0 + tid; g < q.g1; g += nt) {
            double2 h = xv[g];
            for (int o = 0; o < P.nocc; ++o) h = csub(h, cmul(coef[o], P.psi[(size_t)o * npw + g]));
            xa[g] = Ar::from_d(h);   // same thread, same slot: no FP64 value is read back
            if (clean) xv[g] = h;    // read again below by this thread only
        }
        __syncthreads();
        apply_h_block<Ar>(P, smem, q, R, xa, ya, cz(), APPLY_PROJ_OUT);
        const double2* bv = bvec ? bvec + (size_t)r * npw : nullptr;   // -P_c rhs, when precomputed
        if (!bv) part_dots_f64(P, q, R, P.psi, P.nocc, npw, rv, coef);
        double2 acc[3] = {cz(), cz(), cz()};
        for (int g = q.g0 + tid; g < q.g1; g += nt) {
            double2 b;
            if (bv) {
                b = bv[g];
            } else {
                double2 h = rv[g];
                for (int o = 0; o < P.nocc; ++o) h = csub(h, cmul(coef[o], P.psi[(size_t)o * npw + g]));
                b = make_double2(-h.x, -h.y);
            }
            const double2 ax = csub(Ar::to_d(ya[g]), cmul(z, xv[g]));
            const double2 res = csub(b, ax);
            if (store) store[(size_t)i * npw + g] = make_double2(-res.x, -res.y);
            acc[0].x += cabs2(res);
            acc[1].x += cabs2(b);
            acc[2].x += cabs2(xv[g]);
        }
        part_sum<3>(P, R, acc, s_dot);
        if (q.rank == 0 && tid == 0) {
            const double rn = sqrt(s_dot[0].x), bn = sqrt(s_dot[1].x), xn = sqrt(s_dot[2].x);
            if (!isfinite(rn) || !isfinite(bn) || !isfinite(xn)) {
                rel[pq] = NAN;   // a non-finite input or solution is never reported converged
                cert[pq] = NAN;
            } else {
                rel[pq] = bn > 0.0 ? rn / bn : (rn > 0.0 ? INFINITY : 0.0);
                cert[pq] = xn > 0.0 ? rn / (fabs(z.y) * xn) : (rn > 0.0 ? INFINITY : 0.0);
            }
        }
        __syncthreads();
    }
}

// b[r] = -P_c rhs[r] in FP64 (the right-hand sides of the shifted systems), one CTA per vector.
__global__ void __launch_bounds__(kThreads) project_rhs_kernel(Plan P, int nrhs, const double2* __restrict__ rhs,
                                                               double2* __restrict__ b) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2* red = reinterpret_cast<double2*>(smem);
    double2* coef = red + (kMaxThreads / 32) * kRedSlots;
    const int npw = P.npw;
    for (int r = blockIdx.x; r < nrhs; r += gridDim.x) {
        const double2* rv = rhs + (size_t)r * npw;
        block_dots(P.psi, P.nocc, npw, rv, npw, red, coef);
        for (int g = threadIdx.x; g < npw; g += blockDim.x) {
            double2 h = rv[g];
            for (int o = 0; o < P.nocc; ++o) h = csub(h, cmul(coef[o], P.psi[(size_t)o * npw + g]));
            b[(size_t)r * npw + g] = make_double2(-h.x, -h.y);
        }
        __syncthreads();
    }
}

// rhs[c] = e_{cols[c]}: the unit right-hand sides of the Green's-function equation (Eq. 2).
__global__ void unit_rhs_kernel(const int* __restrict__ cols, int ncol, int npw, double2* __restrict__ rhs) {
    const size_t n = (size_t)ncol * npw;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / npw), g = (int)(t % npw);
        rhs[t] = make_double2(g == cols[c] ? 1.0 : 0.0, 0.0);
    }
}

// ------------------------------------------------------------- density response (Eq. 5)
//
// One k-point's contribution to the density response,
//   dn[G][G'][j] += weight * sum_v sum_{+-} FT_G[ conj(u_v(r)) du_{v,G'}(r; +-w_j) ],
// computed coefficient by coefficient in reciprocal space: the box Fourier coefficient of
// the product at G is sum_{G1} conj(psi_v(G1)) du(G1 + G) = <dV_G psi_v | du> (the
// convolution theorem; the box holds the product without aliasing), and dV_G psi_v in the
// k+q basis is exactly the Eq. 8 right-hand side R[v][G].  So, with X the Sternheimer
// solutions [v * np + p][2 nw][npw] (shift j at +w_j, nw + j at -w_j),
//   dn[po][pi][j] += weight * sum_v sum_g conj(R[v np + po][g]) (X[v np + pi][j][g] + X[..][nw + j][g]).
// A CTA owns a tile of kDnP output G's x kDnJ frequencies for one G'; it walks v and the
// plane waves in chunks staged in shared memory (rows padded by one element so the 16-byte
// reads of one quarter-warp fall in distinct banks); each thread accumulates one output in
// FP64.  X is read once from HBM, R (a few MB) from L2.
constexpr int kDnP = 32, kDnJ = 8, kDnCh = 64;

__global__ void __launch_bounds__(kDnP * kDnJ) density_kernel(int n_v, int n_p, int nw, int npw,
                                                              const double2* __restrict__ R,
                                                              const double2* __restrict__ X, double weight,
                                                              double2* __restrict__ dn) {
    __shared__ double2 rs[kDnP][kDnCh + 1];
    __shared__ double2 ys[kDnJ][kDnCh + 1];
    const int tid = threadIdx.x;
    const int jl = tid % kDnJ, pl = tid / kDnJ;
    const int po0 = blockIdx.x * kDnP, pi = blockIdx.y, j0 = blockIdx.z * kDnJ;
    double2 acc = cz();
    for (int v = 0; v < n_v; ++v) {
        const double2* rv = R + (size_t)v * n_p * npw;
        const double2* xv = X + ((size_t)v * n_p + pi) * 2 * nw * npw;
        for (int g0 = 0; g0 < npw; g0 += kDnCh) {
            for (int i = tid; i < kDnP * kDnCh; i += blockDim.x) {
                const int p = i / kDnCh, g = i % kDnCh;
                rs[p][g] = (po0 + p < n_p && g0 + g < npw) ? rv[(size_t)(po0 + p) * npw + g0 + g] : cz();
            }
            for (int i = tid; i < kDnJ * kDnCh; i += blockDim.x) {
                const int j = i / kDnCh, g = i % kDnCh;
                double2 y = cz();
                if (j0 + j < nw && g0 + g < npw)
                    y = cadd(xv[(size_t)(j0 + j) * npw + g0 + g], xv[(size_t)(nw + j0 + j) * npw + g0 + g]);
                ys[j][g] = y;
            }
            __syncthreads();
#pragma unroll 8
            for (int g = 0; g < kDnCh; ++g) acc = cadd(acc, cmulc(rs[pl][g], ys[jl][g]));
            __syncthreads();
        }
    }
    const int po = po0 + pl, j = j0 + jl;
    if (po < n_p && j < nw) {
        double2* o = dn + ((size_t)po * n_p + pi) * nw + j;
        *o = make_double2(o->x + weight * acc.x, o->y + weight * acc.y);
    }
}

// ----------------------------------------------- screening: epsilon^-1 and W-bar (Eq. 4, 9)
//
// One CTA per frequency j.  v(q + G) is the Coulomb potential cut off at R_cut (Sec. 2.6:
// 4 pi / q^2 [1 - cos(q R_cut)], its series 4 pi R^2 (1/2 - x^2/24 + x^4/720), x = q R, for
// x < 1e-4; the bare 4 pi / q^2 when R_cut <= 0).  The dielectric matrix
//   eps[G][G'] = delta - dn[G][G'][j] v(q + G') / Omega
// (the response to the Coulomb potential of a unit plane-wave charge at q + G') is inverted
// in shared memory by Gauss-Jordan elimination with partial pivoting on [eps | 1] in FP64;
// rows and columns with q + G = 0 keep only their diagonal (Sec. 2.4), and
//   W-bar[G][G'] = v(q + G) (eps^-1[G][G'] - delta).
// A zero or non-finite pivot marks the frequency singular: its outputs are NaN and *bad is set.
__device__ __forceinline__ double coulomb_cut(double q, double r_cut) {
    if (r_cut <= 0.0) return 4.0 * M_PI / (q * q);
    const double x = q * r_cut;
    if (x < 1e-4) return 4.0 * M_PI * r_cut * r_cut * (0.5 - x * x / 24.0 + x * x * x * x / 720.0);
    return 4.0 * M_PI / (q * q) * (1.0 - cos(x));
}

__global__ void __launch_bounds__(kThreads) screening_kernel(int n, int nw, const double2* __restrict__ dn,
                                                             const double* __restrict__ qg, double inv_vol,
                                                             double r_cut, double2* __restrict__ einv,
                                                             double2* __restrict__ wbar, int* __restrict__ bad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w2 = 2 * n + 1;                       // row stride of [eps | 1] (odd: bank spread)
    double2* a = reinterpret_cast<double2*>(smem);  // [n][w2]
    double* v = reinterpret_cast<double*>(a + (size_t)n * w2);
    double2* f = reinterpret_cast<double2*>(v + n + (n & 1));   // column factors
    __shared__ int s_piv, s_bad;
    const int j = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    for (int g = tid; g < n; g += nt) {
        const double q = sqrt(qg[3 * g] * qg[3 * g] + qg[3 * g + 1] * qg[3 * g + 1] + qg[3 * g + 2] * qg[3 * g + 2]);
        v[g] = coulomb_cut(q, r_cut);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int i = tid; i < n * 2 * n; i += nt) {
        const int r = i / (2 * n), c = i - r * 2 * n;
        double2 e;
        if (c < n) {
            const double2 d = dn[((size_t)r * n + c) * nw + j];
            const double s = v[c] * inv_vol;
            e = make_double2((r == c ? 1.0 : 0.0) - d.x * s, -d.y * s);
        } else {
            e = make_double2(c - n == r ? 1.0 : 0.0, 0.0);
        }
        a[(size_t)r * w2 + c] = e;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            int p = k;
            double best = -1.0;
            for (int i = k; i < n; ++i) {
                const double m = cabs2(a[(size_t)i * w2 + k]);
                if (m > best) {
                    best = m;
                    p = i;
                }
            }
            if (!(best > 0.0) || !isfinite(best)) s_bad = 1;
            s_piv = p;
        }
        __syncthreads();
        if (s_bad) break;
        const int p = s_piv;
        if (p != k)
            for (int c = tid; c < 2 * n; c += nt) {
                const double2 t = a[(size_t)k * w2 + c];
                a[(size_t)k * w2 + c] = a[(size_t)p * w2 + c];
                a[(size_t)p * w2 + c] = t;
            }
        __syncthreads();
        const double2 inv = cdiv(make_double2(1.0, 0.0), a[(size_t)k * w2 + k]);
        __syncthreads();
        for (int c = tid; c < 2 * n; c += nt) a[(size_t)k * w2 + c] = cmul(a[(size_t)k * w2 + c], inv);
        for (int i = tid; i < n; i += nt) f[i] = a[(size_t)i * w2 + k];
        __syncthreads();
        for (int i = tid; i < n * 2 * n; i += nt) {
            const int r = i / (2 * n), c = i - r * 2 * n;
            if (r != k) a[(size_t)r * w2 + c] = csub(a[(size_t)r * w2 + c], cmul(f[r], a[(size_t)k * w2 + c]));
        }
        __syncthreads();
    }
    const bool sing = s_bad != 0;
    if (sing && tid == 0) atomicExch(bad, 1);
    for (int i = tid; i < n * n; i += nt) {
        const int r = i / n, c = i - r * n;
        double2 e = a[(size_t)r * w2 + n + c];
        const bool zr = qg[3 * r] == 0.0 && qg[3 * r + 1] == 0.0 && qg[3 * r + 2] == 0.0;
        const bool zc = qg[3 * c] == 0.0 && qg[3 * c + 1] == 0.0 && qg[3 * c + 2] == 0.0;
        if (r != c && (zr || zc)) e = cz();
        if (sing) e = make_double2(NAN, NAN);
        const size_t o = ((size_t)r * n + c) * nw + j;
        if (einv) einv[o] = e;
        wbar[o] = cscal(make_double2(e.x - (r == c ? 1.0 : 0.0), e.y), v[r]);
    }
}

int screening_smem_bytes(int n) { return (int)(sizeof(double2) * ((size_t)n * (2 * n + 1) + n + 1) + 8 * (n + 1)); }

// ------------------------------------------------ AAA rational approximation (Sec. 2.7)
//
// One CTA per function (FP64 throughout).  Greedy AAA (Nakatsukasa, Sete, Trefethen 2018):
// the first approximant is the mean of the samples; each step moves the sample where the
// approximant errs most (the first on ties) into the support set, builds the Loewner matrix
// A[i][j] = (F_i - f_j) / (Z_i - z_j) over the other samples (support rows left at zero,
// which changes no right singular vector), and takes the barycentric weights from the right
// singular vector of its smallest singular value.  The SVD is one-sided Jacobi (Hestenes):
// column pairs in a round-robin order, one warp per pair, complex rotations that make each
// pair orthogonal, accumulated in V, until a sweep rotates nothing (at most kAaaSweeps).
// The loop ends when the largest deviation on the remaining samples is <= tol max|F|, at
// mmax support points, or when no sample is left; the approximant is then evaluated at the
// targets (the support value where a target coincides with a support point).
constexpr int kAaaMaxM = 128, kAaaMaxK = 32, kAaaSweeps = 40, kAaaThreads = 256;

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void __launch_bounds__(kAaaThreads) aaa_kernel(int m, const double2* __restrict__ z, const double2* __restrict__ f,
                                                          double tol, int mmax, int ne,
                                                          const double2* __restrict__ ze, double2* __restrict__ re,
                                                          int* __restrict__ degree, int* __restrict__ bad) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2 (*A)[kAaaMaxM] = reinterpret_cast<double2 (*)[kAaaMaxM]>(smem);   // A[col][row], Loewner matrix
    double2 (*V)[kAaaMaxK] = reinterpret_cast<double2 (*)[kAaaMaxK]>(smem + sizeof(double2) * kAaaMaxK * kAaaMaxM);
    __shared__ double2 Z[kAaaMaxM], F[kAaaMaxM], R[kAaaMaxM];
    __shared__ double2 W[kAaaMaxK];
    __shared__ int sup[kAaaMaxK], rest[kAaaMaxM];
    __shared__ double s_red[kAaaThreads / 32];
    __shared__ int s_idx[kAaaThreads / 32];
    __shared__ int s_k, s_done, s_rot, s_bad;
    __shared__ double2 s_mean;
    __shared__ double s_fmax;
    const int fn = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kAaaThreads / 32;
    const double2* fv = f + (size_t)fn * m;
    for (int i = tid; i < m; i += kAaaThreads) {
        Z[i] = z[i];
        F[i] = fv[i];
        rest[i] = 1;
    }
    if (tid == 0) {
        s_k = 0;
        s_done = 0;
        s_bad = 0;
    }
    __syncthreads();
    if (tid == 0) {
        double2 acc = cz();
        double mx = 0.0;
        for (int i = 0; i < m; ++i) {
            acc = cadd(acc, F[i]);
            const double a = sqrt(cabs2(F[i]));
            if (!(a <= mx)) mx = a;   // NaN-propagating
            if (!cfinite(F[i])) s_bad = 1;
        }
        s_mean = cscal(acc, 1.0 / m);
        s_fmax = mx;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) atomicExch(bad, 1);
        for (int e = tid; e < ne; e += kAaaThreads) re[(size_t)fn * ne + e] = make_double2(NAN, NAN);
        if (tid == 0 && degree) degree[fn] = 0;
        return;
    }
    for (int i = tid; i < m; i += kAaaThreads) R[i] = s_mean;
    __syncthreads();
    const int kcap = min(min(mmax, m), kAaaMaxK);
    while (!s_done) {
        // the remaining sample with the largest deviation (first index on ties)
        double best = -1.0;
        int bi = m;
        for (int i = tid; i < m; i += kAaaThreads) {
            if (!rest[i]) continue;
            const double e = sqrt(cabs2(csub(F[i], R[i])));
            if (e > best) {
                best = e;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_red[warp] = best;
            s_idx[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double b = -1.0;
            int ix = m;
            for (int w = 0; w < nw; ++w)
                if (s_red[w] > b || (s_red[w] == b && s_idx[w] < ix)) {
                    b = s_red[w];
                    ix = s_idx[w];
                }
            if (ix >= m)   // no finite deviation left: the first remaining sample
                for (ix = 0; ix < m - 1 && !rest[ix]; ++ix) {
                }
            sup[s_k] = ix;
            rest[ix] = 0;
            s_k = s_k + 1;
        }
        __syncthreads();
        const int k = s_k;
        // Loewner matrix (support rows zero) and V = 1
        for (int t = tid; t < k * m; t += kAaaThreads) {
            const int c = t / m, i = t - c * m;
            const int j = sup[c];
            A[c][i] = rest[i] ? cdiv(csub(F[i], F[j]), csub(Z[i], Z[j])) : cz();
        }
        for (int t = tid; t < k * k; t += kAaaThreads) {
            const int c = t / k, r = t - c * k;
            V[c][r] = make_double2(c == r ? 1.0 : 0.0, 0.0);
        }
        __syncthreads();
        // one-sided Jacobi: round-robin pairs over K = k rounded up to even (index >= k: dummy)
        const int K = (k + 1) & ~1;
        for (int sweep = 0; sweep < kAaaSweeps && k > 1; ++sweep) {
            if (tid == 0) s_rot = 0;
            __syncthreads();
            for (int rnd = 0; rnd < K - 1; ++rnd) {
                for (int pi = warp; pi < K / 2; pi += nw) {
                    // positions 0..K-1: 0 fixed, the others rotated by rnd
                    const int a0 = pi, b0 = K - 1 - pi;
                    const int p = a0 == 0 ? 0 : 1 + (a0 - 1 + rnd) % (K - 1);
                    const int q = 1 + (b0 - 1 + rnd) % (K - 1);
                    if (p >= k || q >= k) continue;
                    double al = 0.0, be = 0.0;
                    double2 ga = cz();
                    for (int i = lane; i < m; i += 32) {
                        const double2 x = A[p][i], y = A[q][i];
                        al += cabs2(x);
                        be += cabs2(y);
                        ga = cadd(ga, cmulc(x, y));
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
                        ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
                    }
                    const double g = sqrt(cabs2(ga));
                    if (!(g > 1e-15 * sqrt(al * be)) || g == 0.0) continue;
                    const double2 ph = make_double2(ga.x / g, ga.y / g);     // e^{i phi}
                    const double zeta = (be - al) / (2.0 * g);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                    const double2 phc = cconj(ph);
                    for (int i = lane; i < m; i += 32) {
                        const double2 x = A[p][i], y = cmul(phc, A[q][i]);
                        A[p][i] = csub(cscal(x, c), cscal(y, sn));
                        A[q][i] = cadd(cscal(x, sn), cscal(y, c));
                    }
                    for (int i = lane; i < k; i += 32) {
                        const double2 x = V[p][i], y = cmul(phc, V[q][i]);
                        V[p][i] = csub(cscal(x, c), cscal(y, sn));
                        V[q][i] = cadd(cscal(x, sn), cscal(y, c));
                    }
                    if (lane == 0) s_rot = 1;
                }
                __syncthreads();
            }
            const int rot = s_rot;
            __syncthreads();
            if (!rot) break;
        }
        // weights: the V column whose A column has the smallest norm
        if (tid == 0) {
            int cmin = 0;
            double nmin = INFINITY;
            for (int c = 0; c < k; ++c) {
                double nrm = 0.0;
                for (int i = 0; i < m; ++i) nrm += cabs2(A[c][i]);
                if (nrm < nmin) {
                    nmin = nrm;
                    cmin = c;
                }
            }
            s_idx[0] = cmin;
        }
        __syncthreads();
        if (tid < k) W[tid] = V[s_idx[0]][tid];
        __syncthreads();
        // new approximant on the remaining samples and its largest deviation
        double dev = 0.0;
        for (int i = tid; i < m; i += kAaaThreads) {
            if (!rest[i]) {
                R[i] = F[i];
                continue;
            }
            double2 num = cz(), den = cz();
            for (int c = 0; c < k; ++c) {
                const double2 cw = cdiv(W[c], csub(Z[i], Z[sup[c]]));
                num = cadd(num, cmul(cw, F[sup[c]]));
                den = cadd(den, cw);
            }
            R[i] = cdiv(num, den);
            const double e = sqrt(cabs2(csub(F[i], R[i])));
            if (!(e <= dev)) dev = e;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double od = __shfl_down_sync(0xffffffffu, dev, o);
            if (!(od <= dev)) dev = od;
        }
        if (lane == 0) s_red[warp] = dev;
        __syncthreads();
        if (tid == 0) {
            double d = 0.0;
            for (int w = 0; w < nw; ++w)
                if (!(s_red[w] <= d)) d = s_red[w];
            if (d <= tol * s_fmax || k >= kcap || k >= m) s_done = 1;
        }
        __syncthreads();
    }
    const int k = s_k;
    for (int e = tid; e < ne; e += kAaaThreads) {
        const double2 x = ze[e];
        double2 num = cz(), den = cz(), hit = cz();
        bool on = false;
        for (int c = 0; c < k; ++c) {
            const double2 d = csub(x, Z[sup[c]]);
            if (d.x == 0.0 && d.y == 0.0) {
                on = true;
                hit = F[sup[c]];
                break;
            }
            const double2 cw = cdiv(W[c], d);
            num = cadd(num, cmul(cw, F[sup[c]]));
            den = cadd(den, cw);
        }
        re[(size_t)fn * ne + e] = on ? hit : cdiv(num, den);
    }
    if (tid == 0 && degree) degree[fn] = k;
}

// x[list[i]] += d[i] for the listed pairs (refinement update).
__global__ void pair_axpy_kernel(int nlist, const int* __restrict__ list, int npw, const double2* __restrict__ d,
                                 double2* __restrict__ x) {
    const size_t n = (size_t)nlist * npw;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / npw, g = t % npw;
        double2* xp = x + (size_t)list[i] * npw + g;
        *xp = cadd(*xp, d[t]);
    }
}

// ---------------------------------------------------------- diagonal preconditioners
//
// D_G for the per-shift systems (the paper does not say how its systems are
// preconditioned; these are additions):
//   plain    M_G = 1 / max(1, T_G / e_prec), e_prec = 1.35 <r|T|r> / <r|r> of the item's
//            right-hand side r;
//   Jacobi   J_G = 1 / max(|H_GG - z|, delta), H_GG = T_G + <V_loc> + sum_p D_p |beta_p(G)|^2;
//   learned  M_G exp(f(phi_G)), phi_G = (T_G / (E_cut/2), omega / 2.205 Ha, e_ref, <V_loc>), f a
//            4-64-64-1 erf-GELU perceptron evaluated with bf16 weights and FP32 accumulation.
__device__ __forceinline__ double h_diag(const Plan& P, int g, double v_mean) {
    double h = P.kin[g] + v_mean;
    for (int p = 0; p < P.nproj; ++p) h += P.dkb[p] * cabs2(P.beta[(size_t)p * P.npw + g]);
    return h;
}

__device__ __forceinline__ double plain_e_prec(const Plan& P, const double2* rv, double2* red, double2* out) {
    double2 acc[2] = {cz(), cz()};
    for (int g = threadIdx.x; g < P.npw; g += blockDim.x) {
        const double m2 = cabs2(rv[g]);
        acc[0].x += m2 * P.kin[g];
        acc[1].x += m2;
    }
    block_sum<2>(acc, red, out);
    return out[1].x > 0.0 ? 1.35 * out[0].x / out[1].x : 1.0;
}

__global__ void __launch_bounds__(kThreads) precond_kernel(Plan P, PrecondArgs a) {
    __shared__ double2 red[(kMaxThreads / 32) * kRedSlots];
    __shared__ double2 out[kRedSlots];
    __shared__ float w[kMlpParams];
    const int tid = threadIdx.x, nt = blockDim.x, npw = P.npw;
    if (a.mode == SGW_PRECOND_LEARNED) {
        for (int i = tid; i < kMlpParams; i += nt) w[i] = __bfloat162float(a.mlp[i]);
    }
    for (int it = blockIdx.x; it < a.n; it += gridDim.x) {
        const double e_prec = plain_e_prec(P, a.rhs + (size_t)it * npw, red, out);
        const double zr = a.e_ref[it] + a.omega[it];
        const double delta = a.delta ? a.delta[it] : 0.0;
        for (int g = tid; g < npw; g += nt) {
            double m = 1.0 / fmax(1.0, P.kin[g] / e_prec);
            if (a.mode == SGW_PRECOND_JACOBI) {
                const double hr = h_diag(P, g, a.v_mean) - zr;
                m = 1.0 / fmax(sqrt(hr * hr + a.eta * a.eta), delta);
            } else if (a.mode == SGW_PRECOND_LEARNED) {
                float x[4] = {(float)(P.kin[g] / a.half_ecut), (float)(a.omega[it] / kOmegaScale), (float)a.e_ref[it],
                              (float)a.v_mean};
                m *= exp((double)mlp_eval(w, x));
            }
            a.d[(size_t)it * npw + g] = m;
        }
        __syncthreads();
    }
}

// Training rows of the learned preconditioner: per plane wave of each pair, phi_G and
// target log(clip(J_G / M_G, e^-3, e^3)) with J the Jacobi diagonal at the pair's best floor
// delta_i (the floor that solved the pair in the fewest H applications), or 0 where the
// plain scaling won (delta_i <= 0).
__global__ void __launch_bounds__(kThreads) training_rows_kernel(Plan P, TrainRowsArgs a) {
    __shared__ double2 red[(kMaxThreads / 32) * kRedSlots];
    __shared__ double2 out[kRedSlots];
    const int tid = threadIdx.x, nt = blockDim.x, npw = P.npw;
    for (int it = blockIdx.x; it < a.n; it += gridDim.x) {
        const double e_prec = plain_e_prec(P, a.rhs + (size_t)it * npw, red, out);
        const double zr = a.e_ref[it] + a.omega[it];
        const double delta = a.delta[it];
        for (int g = tid; g < npw; g += nt) {
            const size_t row = (size_t)it * npw + g;
            const double m = 1.0 / fmax(1.0, P.kin[g] / e_prec);
            double t = 0.0;
            if (delta > 0.0) {
                const double hr = h_diag(P, g, a.v_mean) - zr;
                const double j = 1.0 / fmax(sqrt(hr * hr + a.eta * a.eta), delta);
                t = fmin(fmax(log(j / m), -3.0), 3.0);
            }
            a.feats[4 * row + 0] = (float)(P.kin[g] / a.half_ecut);
            a.feats[4 * row + 1] = (float)(a.omega[it] / kOmegaScale);
            a.feats[4 * row + 2] = (float)a.e_ref[it];
            a.feats[4 * row + 3] = (float)a.v_mean;
            a.targets[row] = (float)t;
        }
        __syncthreads();
    }
}

cudaError_t launch_training_rows(const Plan& P, const TrainRowsArgs& a, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    training_rows_kernel<<<a.n < 4096 ? a.n : 4096, kThreads, 0, st>>>(P, a);
    return cudaGetLastError();
}

cudaError_t launch_precond(const Plan& P, const PrecondArgs& a, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    precond_kernel<<<a.n < 4096 ? a.n : 4096, kThreads, 0, st>>>(P, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ host launchers

namespace {
int bicg_extra(int ns) { return shift_layout(0, ns).end; }
}  // namespace

int optin_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Raises a kernel's dynamic shared-memory limit to everything the device allows next to its
// static shared memory (and allows clusters of 16).  Always the same values for a kernel, so
// concurrent solves of systems of different sizes (several host threads) never lower them
// under one another's launch.
cudaError_t allow_max_smem(const void* kernel) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin_smem() - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// The plan with as many xy-planes per pass (4, 2 or 1) as fit next to `extra` bytes of
// kernel-specific shared memory, for es-byte complex values.
Plan tuned_plan(const Plan& P, int extra, int es) {
    Plan Q = P;
    const int cap = optin_smem() - 1024;   // static shared memory of the kernels
    for (int np : {4, 2, 1}) {
        Q.nplanes = np;
        if (apply_smem_layout(Q, es).end + extra <= cap) return Q;
    }
    Q.nplanes = 1;
    return Q;
}

int apply_smem_bytes(const Plan& P, int es) { return apply_smem_layout(tuned_plan(P, 0, es), es).end; }

int solve_smem_bytes(const Plan& P, int nshift) {
    return apply_smem_layout(tuned_plan(P, bicg_extra(nshift), 16), 16).end + bicg_extra(nshift);
}

cudaError_t resident_grid(const void* kernel, int smem, int* grid, int threads) {
    int dev = 0, nsm = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = allow_max_smem(kernel);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    *grid = nsm * per;
    return cudaSuccess;
}

namespace {
cudaLaunchConfig_t owned_config(const Plan& P, int owners, int threads, int smem, cudaStream_t st,
                                cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(owners * P.csize));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    if (P.csize > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)P.csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cfg;
}
}  // namespace

// Vector owners (CTAs, or clusters of P.csize CTAs) of `kernel` that are resident at once.
cudaError_t owner_capacity(const void* kernel, const Plan& P, int threads, int smem, int* owners) {
    if (P.csize == 1) return resident_grid(kernel, smem, owners, threads);
    cudaError_t e = allow_max_smem(kernel);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = owned_config(P, 1, threads, smem, nullptr, attr);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    *owners = n;
    return cudaSuccess;
}

// Launches `kernel` with `owners` vector owners: owners CTAs, or owners clusters of P.csize.
cudaError_t launch_owned(const void* kernel, const Plan& P, int owners, int threads, int smem, cudaStream_t st,
                         void** args) {
    cudaError_t e = allow_max_smem(kernel);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = owned_config(P, owners, threads, smem, st, attr);
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

// Vector owners of the BiCGstab kernel resident at once (CTAs, or clusters when the box is
// split), at most nrhs and at least one.
cudaError_t solve_grid(const Plan& P, int nshift, int nrhs, int* grid) {
    int g = 0;
    cudaError_t e = owner_capacity((const void*)ms_solve_kernel, P, kThreads, solve_smem_bytes(P, nshift), &g);
    if (e != cudaSuccess) return e;
    *grid = g < nrhs ? g : nrhs;
    if (*grid < 1) *grid = 1;
    return cudaSuccess;
}

// grid: vector owners (solve_grid); one CTA each, or one cluster of P0.csize CTAs each.
cudaError_t launch_solve(const Plan& P0, const SolveArgs& a, int grid, cudaStream_t st) {
    const Plan P = tuned_plan(P0, bicg_extra(a.nshift), 16);
    const int smem = solve_smem_bytes(P0, a.nshift);
    cudaError_t e = allow_max_smem((const void*)ms_solve_kernel);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (P.csize == 1) {
        ms_solve_kernel<<<grid, kThreads, smem, st>>>(P, a);
        return cudaGetLastError();
    }
    SolveArgs aa = a;
    void* args[] = {(void*)&P, (void*)&aa};
    return launch_owned((const void*)ms_solve_kernel, P, grid, kThreads, smem, st, args);
}

namespace {
const void* apply_ptr(int precision) {
    if (precision == SGW_PREC_DF32) return (const void*)apply_kernel<ArDF>;
    if (precision == SGW_PREC_FP32) return (const void*)apply_kernel<ArF32>;
    return (const void*)apply_kernel<ArF64>;
}
const void* residual_ptr(int precision) {
    return precision == SGW_PREC_FP64 ? (const void*)residual_kernel<ArF64> : (const void*)residual_kernel<ArDF>;
}
int residual_bytes(int precision) { return precision == SGW_PREC_FP64 ? 16 : 16; }
}  // namespace

cudaError_t apply_owners(const Plan& P, int precision, int* owners) {
    const int es = prec_bytes(precision);
    return owner_capacity(apply_ptr(precision), P, kThreads, apply_smem_bytes(P, es), owners);
}

cudaError_t launch_apply(const Plan& P0, int nvec, const double2* x, double2* y, const double2* z, int project,
                         double2* scratch, int owners, int precision, cudaStream_t st) {
    const int es = prec_bytes(precision);
    const Plan P = tuned_plan(P0, 0, es);
    const int smem = apply_smem_bytes(P0, es);
    void* args[] = {(void*)&P, (void*)&nvec, (void*)&x, (void*)&y, (void*)&z, (void*)&project, (void*)&scratch};
    return launch_owned(apply_ptr(precision), P, owners, kThreads, smem, st, args);
}

cudaError_t residual_owners(const Plan& P, int precision, int* owners) {
    return owner_capacity(residual_ptr(precision), P, kResThreads, apply_smem_bytes(P, residual_bytes(precision)),
                          owners);
}

cudaError_t launch_residual(const Plan& P0, int nrhs, int nshift, const int* list, int nlist, const double2* rhs,
                            const double* e_ref, const double* omega, double eta, const double2* x, double2* scratch,
                            double* rel, double* cert, double2* store, int owners, cudaStream_t st,
                            const double* eta_s, const double2* bvec, int precision, int clean) {
    const int es = residual_bytes(precision);
    const Plan P = tuned_plan(P0, 0, es);
    const int smem = apply_smem_bytes(P0, es);
    double2* xm = const_cast<double2*>(x);   // written only with clean set
    void* args[] = {(void*)&P,     (void*)&nrhs,    (void*)&nshift, (void*)&list,  (void*)&nlist,
                    (void*)&rhs,   (void*)&e_ref,   (void*)&omega,  (void*)&eta,   (void*)&xm,
                    (void*)&scratch, (void*)&rel,   (void*)&cert,   (void*)&store, (void*)&eta_s,
                    (void*)&bvec,  (void*)&clean};
    return launch_owned(residual_ptr(precision), P, owners, kResThreads, smem, st, args);
}

cudaError_t launch_density(int n_v, int n_p, int nw, int npw, const double2* R, const double2* X, double weight,
                           double2* dn, cudaStream_t st) {
    if (n_v == 0 || n_p == 0 || nw == 0) return cudaSuccess;
    const dim3 grid((n_p + kDnP - 1) / kDnP, n_p, (nw + kDnJ - 1) / kDnJ);
    density_kernel<<<grid, kDnP * kDnJ, 0, st>>>(n_v, n_p, nw, npw, R, X, weight, dn);
    return cudaGetLastError();
}
cudaError_t launch_screening(int n, int nw, const double2* dn, const double* qg, double inv_vol, double r_cut,
                             double2* einv, double2* wbar, int* bad, cudaStream_t st) {
    if (n == 0 || nw == 0) return cudaSuccess;
    const int smem = screening_smem_bytes(n);
    cudaError_t e = allow_max_smem((const void*)screening_kernel);
    if (e != cudaSuccess) return e;
    screening_kernel<<<nw, kThreads, smem, st>>>(n, nw, dn, qg, inv_vol, r_cut, einv, wbar, bad);
    return cudaGetLastError();
}
cudaError_t launch_aaa(int nfun, int m, const double2* z, const double2* f, double tol, int mmax, int ne,
                       const double2* ze, double2* re, int* degree, int* bad, cudaStream_t st) {
    if (nfun == 0) return cudaSuccess;
    const int smem = (int)(sizeof(double2) * (kAaaMaxK * kAaaMaxM + kAaaMaxK * kAaaMaxK));
    cudaError_t e = allow_max_smem((const void*)aaa_kernel);
    if (e != cudaSuccess) return e;
    aaa_kernel<<<nfun, kAaaThreads, smem, st>>>(m, z, f, tol, mmax, ne, ze, re, degree, bad);
    return cudaGetLastError();
}
cudaError_t launch_project_rhs(const Plan& P, int nrhs, const double2* rhs, double2* b, cudaStream_t st) {
    if (nrhs == 0) return cudaSuccess;
    const int smem = (int)(sizeof(double2) * ((kMaxThreads / 32) * kRedSlots + ((P.nocc + 7) / 8 * 8 + 8)));
    cudaError_t e = allow_max_smem((const void*)project_rhs_kernel);
    if (e != cudaSuccess) return e;
    project_rhs_kernel<<<nrhs < 1024 ? nrhs : 1024, kThreads, smem, st>>>(P, nrhs, rhs, b);
    return cudaGetLastError();
}
cudaError_t launch_unit_rhs(const int* cols, int ncol, int npw, double2* rhs, cudaStream_t st) {
    const size_t n = (size_t)ncol * npw;
    if (n == 0) return cudaSuccess;
    unit_rhs_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(cols, ncol, npw, rhs);
    return cudaGetLastError();
}
cudaError_t launch_pair_axpy(int nlist, const int* list, int npw, const double2* d, double2* x, cudaStream_t st) {
    if (nlist == 0) return cudaSuccess;
    pair_axpy_kernel<<<1024, 256, 0, st>>>(nlist, list, npw, d, x);
    return cudaGetLastError();
}

const void* solve_kernel_ptr() { return (const void*)ms_solve_kernel; }

int lanczos_smem_f64(const Plan& P, int nshift);
int lanczos_smem_df(const Plan& P, int nshift);
int lanczos_smem_f32(const Plan& P, int nshift);
cudaError_t lanczos_capacity_f64(const Plan& P, int nshift, int threads, int* owners);
cudaError_t lanczos_capacity_df(const Plan& P, int nshift, int threads, int* owners);
cudaError_t lanczos_capacity_f32(const Plan& P, int nshift, int threads, int* owners);
cudaError_t lanczos_launch_f64(const Plan& P, const LanczosArgs& a, int owners, int threads, cudaStream_t st);
cudaError_t lanczos_launch_df(const Plan& P, const LanczosArgs& a, int owners, int threads, cudaStream_t st);
cudaError_t lanczos_launch_f32(const Plan& P, const LanczosArgs& a, int owners, int threads, cudaStream_t st);

cudaError_t lanczos_batch_capacity_f64(const Plan& P, int threads, int smem, int* owners);
cudaError_t lanczos_batch_capacity_df(const Plan& P, int threads, int smem, int* owners);
cudaError_t lanczos_batch_capacity_f32(const Plan& P, int threads, int smem, int* owners);
cudaError_t lanczos_batch_launch_f64(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                     int owners, int threads, int smem, cudaStream_t st);
cudaError_t lanczos_batch_launch_df(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                    int owners, int threads, int smem, cudaStream_t st);
cudaError_t lanczos_batch_launch_f32(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                     int owners, int threads, int smem, cudaStream_t st);

cudaError_t lanczos_batch_capacity(const Plan& P, int threads, int precision, int smem, int* owners) {
    const int nt = lanczos_threads(threads, precision);
    if (precision == SGW_PREC_DF32) return lanczos_batch_capacity_df(P, nt, smem, owners);
    if (precision == SGW_PREC_FP32) return lanczos_batch_capacity_f32(P, nt, smem, owners);
    return lanczos_batch_capacity_f64(P, nt, smem, owners);
}

cudaError_t launch_lanczos_batch(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                 int owners, int precision, int threads, int smem, cudaStream_t st) {
    const int nt = lanczos_threads(threads, precision);
    if (precision == SGW_PREC_DF32)
        return lanczos_batch_launch_df(P, items, start, nitems, counter, owners, nt, smem, st);
    if (precision == SGW_PREC_FP32)
        return lanczos_batch_launch_f32(P, items, start, nitems, counter, owners, nt, smem, st);
    return lanczos_batch_launch_f64(P, items, start, nitems, counter, owners, nt, smem, st);
}

// CTA size: the requested 256 / 384 / 512, else the measured best for the precision (512 for
// float-float and FP32, 384 for FP64 on the config-2 workload)
int lanczos_threads(int requested, int precision) {
    if (requested == 256 || requested == 384 || requested == 512) return requested;
    return precision == SGW_PREC_FP64 ? 384 : 512;
}

int lanczos_smem_bytes(const Plan& P, int nshift, int precision) {
    if (precision == SGW_PREC_DF32) return lanczos_smem_df(P, nshift);
    if (precision == SGW_PREC_FP32) return lanczos_smem_f32(P, nshift);
    return lanczos_smem_f64(P, nshift);
}

cudaError_t lanczos_capacity(const Plan& P, int nshift, int threads, int precision, int* owners) {
    const int nt = lanczos_threads(threads, precision);
    if (precision == SGW_PREC_DF32) return lanczos_capacity_df(P, nshift, nt, owners);
    if (precision == SGW_PREC_FP32) return lanczos_capacity_f32(P, nshift, nt, owners);
    return lanczos_capacity_f64(P, nshift, nt, owners);
}

cudaError_t launch_lanczos(const Plan& P, const LanczosArgs& a, int owners, int precision, int threads,
                           cudaStream_t st) {
    const int nt = lanczos_threads(threads, precision);
    if (precision == SGW_PREC_DF32) return lanczos_launch_df(P, a, owners, nt, st);
    if (precision == SGW_PREC_FP32) return lanczos_launch_f32(P, a, owners, nt, st);
    return lanczos_launch_f64(P, a, owners, nt, st);
}

}  // namespace sgw
