// Set-up kernels: the plane-wave sphere of Eq. 1, sphere -> box maps, Kleinman-Bylander
// projectors in reciprocal space (Sec. 2.1), FFT twiddles, the Eq. 8 right-hand-side
// gather and the overlap matrix of the occupied states.
#include <cuda_runtime.h>

#include <algorithm>

#include "sgw_internal.cuh"
#include "setup.h"

namespace sgw {

// ---------------------------------------------------------------------- G-sphere (Eq. 1)

// One CTA enumerates the Miller box [-M1,M1] x [-M2,M2] x [-M3,M3] in lexicographic order
// (m1 outermost) and keeps m with |k + m.B|^2 <= ecut, evaluated in FP64 with every
// product and sum rounded separately (no contraction), in the documented order:
//   k_x = (k1 b1x + k2 b2x) + k3 b3x ;  g_x = ((k_x + m1 b1x) + m2 b2x) + m3 b3x ;
//   |g|^2 = (g_x g_x + g_y g_y) + g_z g_z.
// The kept triples are compacted in order with a block-wide exclusive scan.
__global__ void __launch_bounds__(1024) sphere_kernel(SphereArgs a, int* __restrict__ miller,
                                                      double* __restrict__ kin, int* __restrict__ count) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int e1 = 2 * a.M[0] + 1, e2 = 2 * a.M[1] + 1, e3 = 2 * a.M[2] + 1;
    const long long total = (long long)e1 * e2 * e3;
    double kc[3];
#pragma unroll
    for (int x = 0; x < 3; ++x)
        kc[x] = __dadd_rn(__dadd_rn(__dmul_rn(a.k[0], a.b[0][x]), __dmul_rn(a.k[1], a.b[1][x])),
                          __dmul_rn(a.k[2], a.b[2][x]));
    if (tid == 0) base = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < total; c0 += blockDim.x) {
        const long long c = c0 + tid;
        int keep = 0;
        int m1 = 0, m2 = 0, m3 = 0;
        double n2 = 0.0;
        if (c < total) {
            m1 = (int)(c / ((long long)e2 * e3)) - a.M[0];
            m2 = (int)((c / e3) % e2) - a.M[1];
            m3 = (int)(c % e3) - a.M[2];
            double g[3];
#pragma unroll
            for (int x = 0; x < 3; ++x)
                g[x] = __dadd_rn(__dadd_rn(__dadd_rn(kc[x], __dmul_rn((double)m1, a.b[0][x])),
                                           __dmul_rn((double)m2, a.b[1][x])),
                                 __dmul_rn((double)m3, a.b[2][x]));
            n2 = __dadd_rn(__dadd_rn(__dmul_rn(g[0], g[0]), __dmul_rn(g[1], g[1])), __dmul_rn(g[2], g[2]));
            keep = n2 <= a.ecut ? 1 : 0;
        }
        // exclusive scan of keep over the block
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int inwarp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int t = warp_tot[w];
            if (w < warp) off += t;
            tot += t;
        }
        const int pos = base + off + inwarp;
        if (keep && pos < a.cap) {
            miller[3 * pos + 0] = m1;
            miller[3 * pos + 1] = m2;
            miller[3 * pos + 2] = m3;
            kin[pos] = 0.5 * n2;
        }
        __syncthreads();
        if (tid == 0) base += tot;
        __syncthreads();
    }
    if (tid == 0) *count = base;
}

// Sphere -> box index ((m1 mod N1) N2 + (m2 mod N2)) N3 + (m3 mod N3).
__global__ void boxmap_kernel(const int* __restrict__ miller, int npw, int n1, int n2, int n3,
                              int* __restrict__ map) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npw) return;
    const int x = ((miller[3 * g] % n1) + n1) % n1;
    const int y = ((miller[3 * g + 1] % n2) + n2) % n2;
    const int z = ((miller[3 * g + 2] % n3) + n3) % n3;
    map[g] = (x * n2 + y) * n3 + z;
}

// <k+G|beta_p> = Omega^(-1/2) (4 pi w^2)^(3/4) exp(-w^2 |k+G|^2 / 2) exp(-i (k+G).tau_p)
// for the normalised s-type Gaussian beta(r) = (pi w^2)^(-3/4) exp(-r^2 / 2w^2).
__global__ void beta_kernel(BetaArgs a, const int* __restrict__ miller, int npw, double2* __restrict__ beta) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (g >= npw) return;
    double kg[3];
#pragma unroll
    for (int x = 0; x < 3; ++x)
        kg[x] = (miller[3 * g] + a.k[0]) * a.b[0][x] + (miller[3 * g + 1] + a.k[1]) * a.b[1][x] +
                (miller[3 * g + 2] + a.k[2]) * a.b[2][x];
    const double kg2 = kg[0] * kg[0] + kg[1] * kg[1] + kg[2] * kg[2];
    const double w = a.width[p];
    const double amp = a.inv_sqrt_vol * pow(4.0 * 3.14159265358979323846 * w * w, 0.75) * exp(-0.5 * w * w * kg2);
    const double ph = -(kg[0] * a.tau[p][0] + kg[1] * a.tau[p][1] + kg[2] * a.tau[p][2]);
    double s, c;
    sincos(ph, &s, &c);
    beta[(size_t)p * npw + g] = make_double2(amp * c, amp * s);
}

// tw[m] = exp(-2 pi i m / n) for each axis, concatenated.
__global__ void twiddle_kernel(int n1, int n2, int n3, double2* __restrict__ tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1 + n2 + n3) return;
    int n, m;
    if (i < n1) { n = n1; m = i; }
    else if (i < n1 + n2) { n = n2; m = i - n1; }
    else { n = n3; m = i - n1 - n2; }
    double s, c;
    sincospi(-2.0 * m / n, &s, &c);
    tw[i] = make_double2(c, s);
}

// Eq. 8 driving field in the k+q basis: rhs[v*np + p][g'] = psi_k[v][idx(m' - G_p)], or 0.
__global__ void rhs_kernel(RhsArgs a, const int* __restrict__ miller_kq, int npw_kq,
                           const int* __restrict__ lut_k, const double2* __restrict__ psi_k, int npw_k,
                           const int* __restrict__ gp, int n_v, int n_pert, double2* __restrict__ rhs) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (g >= npw_kq) return;
    int src = -1;
    int m[3];
    bool inside = true;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        m[x] = miller_kq[3 * g + x] - gp[3 * p + x] - a.lo[x];
        inside = inside && m[x] >= 0 && m[x] < a.ext[x];
    }
    if (inside) src = lut_k[(m[0] * a.ext[1] + m[1]) * a.ext[2] + m[2]];
    for (int v = 0; v < n_v; ++v) {
        const double2 val = src >= 0 ? psi_k[(size_t)v * npw_k + src] : make_double2(0.0, 0.0);
        rhs[((size_t)v * n_pert + p) * npw_kq + g] = val;
    }
}

// S[v][w] = <psi_v|psi_w>, one CTA per entry.
__global__ void __launch_bounds__(kThreads) gram_kernel(const double2* __restrict__ psi, int nocc, int npw,
                                                        double2* __restrict__ S) {
    __shared__ double2 red[(kThreads / 32) * kRedSlots];
    __shared__ double2 out[1];
    const int v = blockIdx.x / nocc, w = blockIdx.x % nocc;
    double2 acc[1] = {make_double2(0.0, 0.0)};
    for (int g = threadIdx.x; g < npw; g += blockDim.x)
        acc[0] = cadd(acc[0], cmulc(psi[(size_t)v * npw + g], psi[(size_t)w * npw + g]));
    block_sum<1>(acc, red, out);
    if (threadIdx.x == 0) S[blockIdx.x] = out[0];
}

// ------------------------------------------------------------------------ host launchers

cudaError_t launch_sphere(const SphereArgs& a, int* miller, double* kin, int* count, cudaStream_t st) {
    sphere_kernel<<<1, 1024, 0, st>>>(a, miller, kin, count);
    return cudaGetLastError();
}
cudaError_t launch_boxmap(const int* miller, int npw, const int dims[3], int* map, cudaStream_t st) {
    boxmap_kernel<<<(npw + 255) / 256, 256, 0, st>>>(miller, npw, dims[0], dims[1], dims[2], map);
    return cudaGetLastError();
}
cudaError_t launch_beta(const BetaArgs& a, int nproj, const int* miller, int npw, double2* beta, cudaStream_t st) {
    if (nproj == 0) return cudaSuccess;
    beta_kernel<<<dim3((npw + 255) / 256, nproj), 256, 0, st>>>(a, miller, npw, beta);
    return cudaGetLastError();
}
cudaError_t launch_twiddles(const int dims[3], double2* tw, cudaStream_t st) {
    const int n = dims[0] + dims[1] + dims[2];
    twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(dims[0], dims[1], dims[2], tw);
    return cudaGetLastError();
}
cudaError_t launch_rhs(const RhsArgs& a, const int* miller_kq, int npw_kq, const int* lut_k, const double2* psi_k,
                       int npw_k, const int* gp, int n_v, int n_pert, double2* rhs, cudaStream_t st) {
    if (n_pert == 0 || npw_kq == 0) return cudaSuccess;
    rhs_kernel<<<dim3((npw_kq + 255) / 256, n_pert), 256, 0, st>>>(a, miller_kq, npw_kq, lut_k, psi_k, npw_k, gp,
                                                                    n_v, n_pert, rhs);
    return cudaGetLastError();
}
// Each FP64 value as the float pair (hi, lo) with hi = fl32(x) and lo = fl32(x - hi); a
// double2 array converts into the (re.hi, re.lo, im.hi, im.lo) layout of the float-float policy.
__global__ void to_dd_kernel(const double* __restrict__ src, size_t n, float2* __restrict__ dst) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = src[i];
        const float h = __double2float_rn(x);
        dst[i] = make_float2(h, __double2float_rn(x - (double)h));
    }
}

cudaError_t launch_to_dd(const double* src, size_t n, float2* dst, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    to_dd_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, n, dst);
    return cudaGetLastError();
}
// Each FP64 value rounded to FP32 (the single-precision policy's copies of T, beta, psi).
__global__ void to_f32_kernel(const double* __restrict__ src, size_t n, float* __restrict__ dst) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}

cudaError_t launch_to_f32(const double* src, size_t n, float* dst, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    to_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, n, dst);
    return cudaGetLastError();
}
cudaError_t launch_gram(const double2* psi, int nocc, int npw, double2* S, cudaStream_t st) {
    gram_kernel<<<nocc * nocc, kThreads, 0, st>>>(psi, nocc, npw, S);
    return cudaGetLastError();
}

}  // namespace sgw
