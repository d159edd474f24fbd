// Shifted Lanczos (FOM) multishift kernel, templated over the arithmetic policy; each
// policy is instantiated in its own translation unit (lanczos_f64.cu, lanczos_df.cu,
// lanczos_f32.cu).
//
// Multishift solve by the Hermitian Lanczos process on A = P_c H P_c (Sec. 2.2: systems
// that differ only in the frequency share one Krylov space).  With b = beta_1 v_1,
//   A V_k = V_k T_k + beta_{k+1} v_{k+1} e_k^T,   T_k real symmetric tridiagonal (alpha, beta),
// the Galerkin solution of shift j is x_j = V_k y_j with (T_k - z_j) y_j = beta_1 e_1.  The
// LDL^T pivots of the complex-symmetric T_k - z_j,
//   eta_1 = alpha_1 - z_j,  l_i = beta_i / eta_{i-1},  eta_i = alpha_i - z_j - l_i beta_i,
// never vanish because Im z_j != 0 and T_k has a real spectrum; the forward sweep
// u_i = -l_i u_{i-1} (u_1 = beta_1) gives the residual norm |beta_{k+1} u_k / eta_k| of every
// shift from scalars alone, and the residuals of all shifts stay collinear with v_{k+1}.
//
// Stopping.  Shift j stops at the first step whose residual estimate is at most its target,
// initially tol.  With a certificate tolerance c > 0 the error bound |r| / (|Im z_j| |x_j|)
// must also hold: once every shift has stopped, y_j and |x_j| = |y_j| (orthonormal basis) are
// formed, and a shift whose estimated certificate est_j |b| / (|Im z_j| |y_j|) exceeds c gets
// the target c |Im z_j| |y_j| / (2 |b|) and resumes.  The pivots of every shift are kept
// current at every step, so a resumed shift continues without recomputation (at most three
// such rounds).
//
// The basis is kept (one slice of global memory per vector owner); when every shift has
// stopped (or the basis is full) each y_j is formed by the backward sweep
// y_i = u_i/eta_i - l_{i+1} y_{i+1} and x_j = V y_j over the basis.
//
// One CTA or one cluster owns a right-hand side at a time (a work queue hands them out); in a
// cluster every rank runs the same scalar recurrences on bit-identical reduced values and
// works on its own plane waves only.
#pragma once

#include <cuda_runtime.h>

#include "setup.h"
#include "sgw_internal.cuh"

namespace sgw {

// Right-hand side r of the system (P, A): the whole multishift solve by the CTA or cluster
// that owns it.  All threads of every rank call.
template <class Ar, int NT>
__device__ __noinline__ void lanczos_rhs(const Plan& P, const LanczosArgs& A, unsigned char* smem, int r) {
    using C = typename Ar::C;
    __shared__ double2 s_dot[kRedSlots];
    __shared__ int s_nact, s_kmax, s_fail, s_more;
    const ApplySmem L = apply_smem_layout(P, (int)sizeof(C));
    Red R = make_red(P, smem, L);
    double2* coef = reinterpret_cast<double2*>(smem + L.coef);
    const Part q = make_part(P);
    const int ns = A.nshift, npw = P.npw, tid = threadIdx.x, nt = blockDim.x, maxk = A.maxk;
    const int g0 = q.g0, g1 = q.g1;
    const int cl_id = blockIdx.x / P.csize;
    // per-shift state after the apply's shared memory
    int off = L.end;
    double2* zsh = reinterpret_cast<double2*>(smem + off); off = align16(off + ns * 16);
    double2* eta = reinterpret_cast<double2*>(smem + off); off = align16(off + ns * 16);
    double2* zeta = reinterpret_cast<double2*>(smem + off); off = align16(off + ns * 16);
    double* est = reinterpret_cast<double*>(smem + off); off = align16(off + ns * 8);    // current estimate
    double* estc = reinterpret_cast<double*>(smem + off); off = align16(off + ns * 8);   // at the stopping step
    double* tgt = reinterpret_cast<double*>(smem + off); off = align16(off + ns * 8);    // target
    int* kc = reinterpret_cast<int*>(smem + off); off = align16(off + ns * 4);
    int* st = reinterpret_cast<int*>(smem + off);

    // per-owner basis, per-CTA recurrence scalars and coefficients (strides fixed per launch, so
    // that systems of several sizes can share one workspace)
    C* V = reinterpret_cast<C*>(A.basis) + (size_t)cl_id * A.vstride;
    double* al = A.ab + (size_t)blockIdx.x * 2 * (maxk + 1);     // alpha[0..maxk), beta[0..maxk]
    double* be = al + (maxk + 1);
    double2* Ysc = A.ysc + (size_t)blockIdx.x * A.ystride;       // [maxk][ns] y, [maxk][ns] l
    double2* Lsc = Ysc + (size_t)maxk * ns;
    C* Yc = reinterpret_cast<C*>(Lsc);                          // y in the policy's format, after the sweeps

    {
        const double2* rhs = A.rhs + (size_t)r * npw;
        double2* X = A.x + (size_t)r * ns * npw;

        // b = -P_c rhs (FP64), beta_1 = |b|, V[0] = b / beta_1 in the policy's format
        part_dots_f64(P, q, R, P.psi, P.nocc, npw, rhs, coef);
        {
            double2 acc[1] = {cz()};
            for (int g = g0 + tid; g < g1; g += nt) {
                double2 h = rhs[g];
                for (int v = 0; v < P.nocc; ++v) h = csub(h, cmul(coef[v], P.psi[(size_t)v * npw + g]));
                acc[0].x += cabs2(h);
            }
            part_sum<1>(P, R, acc, s_dot);
        }
        const double b1 = sqrt(s_dot[0].x);
        const bool zero = !(b1 > 0.0), bad = !isfinite(b1);
        {
            const double inv = (zero || bad) ? 0.0 : -1.0 / b1;
            for (int g = g0 + tid; g < g1; g += nt) {
                double2 h = rhs[g];
                for (int v = 0; v < P.nocc; ++v) h = csub(h, cmul(coef[v], P.psi[(size_t)v * npw + g]));
                V[g] = Ar::from_d(cscal(h, inv));
            }
        }
        for (int j = tid; j < ns; j += nt) {
            zsh[j] = make_double2(A.e_ref[r] + A.omega[j], A.eta_r ? A.eta_r[r] : (A.eta_s ? A.eta_s[j] : A.eta));
            est[j] = zero ? 0.0 : 1.0;
            estc[j] = est[j];
            tgt[j] = A.tol;
            kc[j] = 0;
            st[j] = bad ? SGW_PAIR_NONFINITE : (zero ? SGW_PAIR_CONVERGED : -1);
        }
        if (tid == 0) {
            s_nact = (zero || bad) ? 0 : ns;
            s_fail = 0;
            be[0] = 0.0;
        }
        __syncthreads();
        int k = 0;
        for (int round = 0;; ++round) {
            while (s_nact > 0 && k < maxk) {
                C* vk = V + (size_t)k * npw;
                C* w = V + (size_t)(k + 1) * npw;
                apply_h_block<Ar>(P, smem, q, R, vk, w, cz(), APPLY_PROJ_OUT);
                const double bk = be[k];
                const C* vkm = k > 0 ? V + (size_t)(k - 1) * npw : nullptr;
                {
                    const typename Ar::R bkr = Ar::real(bk);
                    C acc = Ar::zero();
                    for (int g = g0 + tid; g < g1; g += nt) {
                        C h = w[g];
                        if (vkm) h = Ar::sub(h, Ar::scalr(vkm[g], bkr));
                        w[g] = h;
                        acc = Ar::add(acc, Ar::mul(Ar::conj(vk[g]), h));
                    }
                    C a2[1] = {acc};
                    part_sum<1>(P, R, a2, s_dot);
                }
                const double a = s_dot[0].x;
                {
                    const typename Ar::R ar = Ar::real(a);
                    C acc = Ar::zero();
                    for (int g = g0 + tid; g < g1; g += nt) {
                        const C h = Ar::sub(w[g], Ar::scalr(vk[g], ar));
                        w[g] = h;
                        acc = Ar::acc_norm(acc, h);
                    }
                    C a2[1] = {acc};
                    part_sum<1>(P, R, a2, s_dot);
                }
                const double bn = sqrt(s_dot[0].x);
                {
                    const typename Ar::R inv = Ar::real(bn > 0.0 ? 1.0 / bn : 0.0);
                    for (int g = g0 + tid; g < g1; g += nt) w[g] = Ar::scalr(w[g], inv);
                }
                if (tid == 0) {
                    al[k] = a;
                    be[k + 1] = bn;
                    if (!isfinite(a) || !isfinite(bn)) s_fail = SGW_PAIR_NONFINITE;
                }
                // per-shift pivots and residual estimates, kept current for stopped shifts too
                for (int j = tid; j < ns; j += nt) {
                    if (st[j] == SGW_PAIR_NONFINITE) continue;
                    const double2 d = make_double2(a - zsh[j].x, -zsh[j].y);
                    double2 e, u;
                    if (k == 0) {
                        e = d;
                        u = make_double2(b1, 0.0);
                    } else {
                        const double2 l = cdiv(make_double2(bk, 0.0), eta[j]);
                        e = csub(d, cscal(l, bk));
                        u = cmul(make_double2(-l.x, -l.y), zeta[j]);
                    }
                    const double2 qq = cdiv(u, e);
                    const double rr = bn * sqrt(cabs2(qq)) / b1;
                    if (!isfinite(rr)) {
                        if (st[j] < 0) st[j] = SGW_PAIR_NONFINITE;
                        continue;   // a stopped shift keeps its solution and is not resumed
                    }
                    eta[j] = e;
                    zeta[j] = u;
                    est[j] = rr;
                    if (st[j] < 0) {
                        kc[j] = k + 1;
                        estc[j] = rr;
                        if (rr <= tgt[j] || bn == 0.0) st[j] = SGW_PAIR_CONVERGED;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int n = 0;
                    for (int j = 0; j < ns; ++j) n += st[j] < 0 ? 1 : 0;
                    s_nact = s_fail ? 0 : n;
                }
                ++k;
                __syncthreads();
                if (bn == 0.0) break;
            }
            const bool can_resume = A.cert_tol > 0.0 && round < 3 && k < maxk && !s_fail && be[k] != 0.0;
            if (tid == 0) s_more = 0;
            __syncthreads();
            // y_j = (T_kj - z_j)^{-1} beta_1 e_1 by forward / backward sweeps (one thread per shift),
            // then the certificate check of the stopped shifts
            for (int j = tid; j < ns; j += nt) {
                const int kj = kc[j];
                if (kj == 0 || st[j] == SGW_PAIR_NONFINITE) continue;
                double2 e = make_double2(al[0] - zsh[j].x, -zsh[j].y);
                double2 u = make_double2(b1, 0.0);
                Ysc[j] = cdiv(u, e);
                for (int i = 1; i < kj; ++i) {
                    const double2 l = cdiv(make_double2(be[i], 0.0), e);
                    e = csub(make_double2(al[i] - zsh[j].x, -zsh[j].y), cscal(l, be[i]));
                    u = cmul(make_double2(-l.x, -l.y), u);
                    Lsc[(size_t)i * ns + j] = l;
                    Ysc[(size_t)i * ns + j] = cdiv(u, e);
                }
                double yn2 = cabs2(Ysc[(size_t)(kj - 1) * ns + j]);
                for (int i = kj - 2; i >= 0; --i) {
                    const double2 y = csub(Ysc[(size_t)i * ns + j],
                                           cmul(Lsc[(size_t)(i + 1) * ns + j], Ysc[(size_t)(i + 1) * ns + j]));
                    Ysc[(size_t)i * ns + j] = y;
                    yn2 += cabs2(y);
                }
                if (can_resume && st[j] == SGW_PAIR_CONVERGED) {
                    // certificate |r| / (|Im z| |x|) with |r| = est |b| and |x| = |y|
                    const double need = A.cert_tol * fabs(zsh[j].y) * sqrt(yn2) / b1;
                    if (estc[j] > need && est[j] != 0.0) {
                        tgt[j] = fmin(tgt[j], 0.5 * need);
                        if (est[j] <= tgt[j]) {
                            kc[j] = k;          // already there at the current step: move its stop
                            estc[j] = est[j];
                        } else {
                            st[j] = -1;         // resume
                        }
                        s_more = 1;
                    }
                }
            }
            __syncthreads();
            if (!s_more) break;
            if (tid == 0) {
                int n = 0;
                for (int j = 0; j < ns; ++j) n += st[j] < 0 ? 1 : 0;
                s_nact = n;
            }
            __syncthreads();
        }
        // budget exhausted / failure
        for (int j = tid; j < ns; j += nt)
            if (st[j] < 0) st[j] = s_fail ? s_fail : SGW_PAIR_MAXITER;
        if (tid == 0) {
            int m = 0;
            for (int j = 0; j < ns; ++j) m = max(m, kc[j]);
            s_kmax = m;
        }
        __syncthreads();
        const int K = s_kmax;
        // y in the policy's format, zero beyond each shift's own stopping step
        for (int j = tid; j < ns; j += nt) {
            const int kj = (st[j] == SGW_PAIR_NONFINITE) ? 0 : kc[j];
            for (int i = 0; i < K; ++i) Yc[(size_t)i * ns + j] = i < kj ? Ar::from_d(Ysc[(size_t)i * ns + j]) : Ar::zero();
        }
        __syncthreads();
        // x_j = V y_j over this rank's plane waves, shifts in tiles of TJ.  The tile's y
        // coefficients are staged in the (now idle) FFT buffers of shared memory, KC Lanczos
        // steps at a time; every thread reads them as broadcasts.
        constexpr int TJ = NT >= 384 ? 4 : 8;
        {
            C* ys = reinterpret_cast<C*>(smem + L.sticks);
            const int KC = (L.red - L.sticks) / (TJ * (int)sizeof(C));
            for (int j0 = 0; j0 < ns; j0 += TJ) {
                const int cnt = min(TJ, ns - j0);
                int Kt = 0;   // the tile's longest Lanczos run (y is zero beyond each shift's own)
                for (int t = 0; t < cnt; ++t) Kt = max(Kt, st[j0 + t] == SGW_PAIR_NONFINITE ? 0 : kc[j0 + t]);
                if (Kt == 0)
                    for (int t = 0; t < cnt; ++t)
                        for (int g = g0 + tid; g < g1; g += nt) X[(size_t)(j0 + t) * npw + g] = cz();
                for (int k0 = 0; k0 < Kt; k0 += KC) {
                    const int kn = min(KC, Kt - k0);
                    __syncthreads();
                    for (int i = tid; i < kn * TJ; i += nt) {
                        const int ii = i / TJ, t = i - ii * TJ;
                        ys[i] = t < cnt ? Yc[(size_t)(k0 + ii) * ns + j0 + t] : Ar::zero();
                    }
                    __syncthreads();
                    for (int g = g0 + tid; g < g1; g += nt) {
                        C acc[TJ];
#pragma unroll
                        for (int t = 0; t < TJ; ++t) acc[t] = Ar::zero();
                        const C* vg = V + (size_t)k0 * npw + g;
#pragma unroll 2
                        for (int i = 0; i < kn; ++i) {
                            const C v = vg[(size_t)i * npw];
                            const C* yr = ys + i * TJ;
#pragma unroll
                            for (int t = 0; t < TJ; ++t) acc[t] = Ar::add(acc[t], Ar::mul(yr[t], v));
                        }
#pragma unroll
                        for (int t = 0; t < TJ; ++t) {
                            if (t < cnt) {
                                double2* xo = X + (size_t)(j0 + t) * npw + g;
                                const double2 d = Ar::to_d(acc[t]);
                                *xo = k0 == 0 ? d : cadd(*xo, d);
                            }
                        }
                    }
                }
            }
        }
        if (q.rank == 0) {
            for (int j = tid; j < ns; j += nt) {
                A.out_status[(size_t)r * ns + j] = st[j];
                A.out_mv[(size_t)r * ns + j] = kc[j];
                A.out_res[(size_t)r * ns + j] = estc[j];
            }
        }
        __syncthreads();
    }
}

// One system: a work queue hands its right-hand sides to the owners.
template <class Ar, int NT>
__global__ void __launch_bounds__(NT, 1) lanczos_solve_kernel(Plan P, LanczosArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    load_twiddles<Ar>(P, smem);
    for (;;) {
        const int r = next_item(P, A.counter);
        if (r >= A.nrhs) break;
        lanczos_rhs<Ar, NT>(P, A, smem, r);
    }
}

// Several systems (uneven sizes, one cluster size) in one persistent launch: the queue hands
// out (system, right-hand side) items in the order of the items array (the host puts the
// costliest systems first); start[i] is the first queue index of system i.
template <class Ar, int NT>
__global__ void __launch_bounds__(NT, 1) lanczos_batch_kernel(const BatchItem* __restrict__ items, const int* __restrict__ start,
                                                             int nitems, int* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int total = start[nitems];
    int cur = -1;
    for (;;) {
        const int t = next_item(items[0].plan, counter);
        if (t >= total) break;
        int lo = 0, hi = nitems - 1;   // the system holding queue index t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const Plan& P = items[lo].plan;
        if (lo != cur) {
            __syncthreads();   // the previous system's twiddles are no longer read
            load_twiddles<Ar>(P, smem);
            cur = lo;
        }
        lanczos_rhs<Ar, NT>(P, items[lo].args, smem, t - start[lo]);
    }
}

template <class Ar>
const void* lanczos_ptr_t(int nt) {
    if (nt == 512) return (const void*)lanczos_solve_kernel<Ar, 512>;
    if (nt == 384) return (const void*)lanczos_solve_kernel<Ar, 384>;
    return (const void*)lanczos_solve_kernel<Ar, 256>;
}

template <class Ar>
int lanczos_smem_t(const Plan& P, int nshift) {
    const int es = (int)sizeof(typename Ar::C);
    return apply_smem_layout(tuned_plan(P, lanczos_extra(nshift), es), es).end + lanczos_extra(nshift);
}

template <class Ar>
cudaError_t lanczos_capacity_t(const Plan& P, int nshift, int threads, int* owners) {
    return owner_capacity(lanczos_ptr_t<Ar>(threads), P, threads, lanczos_smem_t<Ar>(P, nshift), owners);
}

template <class Ar>
cudaError_t lanczos_launch_t(const Plan& P0, const LanczosArgs& a0, int owners, int threads, cudaStream_t st) {
    const int es = (int)sizeof(typename Ar::C);
    const Plan P = tuned_plan(P0, lanczos_extra(a0.nshift), es);
    const int smem = lanczos_smem_t<Ar>(P0, a0.nshift);
    LanczosArgs a = a0;
    if (a.vstride == 0) a.vstride = (size_t)(a.maxk + 1) * P.npw;
    if (a.ystride == 0) a.ystride = 2 * (size_t)a.maxk * a.nshift;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&P, (void*)&a};
    return launch_owned(lanczos_ptr_t<Ar>(threads), P, owners, threads, smem, st, args);
}

template <class Ar>
const void* lanczos_batch_ptr_t(int nt) {
    if (nt == 512) return (const void*)lanczos_batch_kernel<Ar, 512>;
    if (nt == 384) return (const void*)lanczos_batch_kernel<Ar, 384>;
    return (const void*)lanczos_batch_kernel<Ar, 256>;
}

// items: device array (plans already tuned for smem bytes of dynamic shared memory).
template <class Ar>
cudaError_t lanczos_batch_launch_t(const Plan& P0, const BatchItem* items, const int* start, int nitems, int* counter,
                                   int owners, int threads, int smem, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&items, (void*)&start, (void*)&nitems, (void*)&counter};
    return launch_owned(lanczos_batch_ptr_t<Ar>(threads), P0, owners, threads, smem, st, args);
}

template <class Ar>
cudaError_t lanczos_batch_capacity_t(const Plan& P, int threads, int smem, int* owners) {
    return owner_capacity(lanczos_batch_ptr_t<Ar>(threads), P, threads, smem, owners);
}

}  // namespace sgw
