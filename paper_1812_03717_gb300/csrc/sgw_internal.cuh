// Internal declarations of the GB300 shifted-Sternheimer library.
//
// Data layout in device memory (all complex values are FP64 pairs, double2):
//   plane-wave vectors      [nvec][npw]              canonical G order (Miller lexicographic)
//   local potential         [N3][N1][N2p]            one contiguous (padded) xy-plane per z, each
//                                                    axis in the order that the in-place FFT
//                                                    leaves real space in
//   stick buffer (on chip)  [nstick][N3p]            z-columns of the box that hold a G (N3p odd)
//   plane buffer (on chip)  [nplanes][N1][N2p]       a few xy-planes of the box, rows padded to odd N2p
//   KB projectors           [nproj][npw]             <k+G|beta_p>
//   occupied states         [nocc][npw]              psi_v of the basis (Eq. 7-8)
//
// One CTA, or one thread-block cluster of P.csize CTAs, owns one whole vector during an H
// application (Sec. 2.1: kinetic and non-local parts in reciprocal space, V_loc in real space
// through the FFT).  The whole pruned box of that vector -- only the z-columns ("sticks")
// through the sphere, plus a few xy-planes at a time -- lives in shared memory, so an
// application reads x once and writes y once.  In a cluster, rank r holds the sticks
// [s0, s1) and owns the plane waves of those sticks, [g0, g1) (a contiguous range: the G of one
// stick are consecutive in canonical order); it transforms the xy-planes [z0, z1), gathering
// each plane's stick elements from the other ranks' shared memory (distributed shared memory)
// and scattering the result back.  Dot products over the vector are summed over the cluster
// in rank order, so every rank holds bit-identical scalars.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "sgw.h"

namespace sgw {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;          // threads per CTA of the library kernels
constexpr int kResThreads = 384;       // threads per CTA of the FP64 true-residual kernel
constexpr int kMaxThreads = 512;       // largest CTA any kernel launches (sizes the reduction scratch)
constexpr int kMaxStages = 12;         // radix stages per axis (N <= 5^12)
constexpr int kMaxShifts = 512;        // frequencies per solve
constexpr int kMaxEll = 4;             // BiCGstab(ell)
constexpr int kRedSlots = 16;          // complex values reduced per block reduction
constexpr int kMaxCluster = 16;        // CTAs sharing one vector's box (16 needs the non-portable size)

struct AxisPlan {
    int n;
    int nst;
    int rad[kMaxStages];    // radices R_0, R_1, ... (R_0 acts on the full length)
    int span[kMaxStages];   // m_s = n / (R_0 ... R_s)
    int npart;              // > 0: prime-factor algorithm over these coprime parts (2^a, 3^b, 5^c
    int part[3];            //      in {2, 3, 4, 5, 8, 9}); 0: the radix stages above
};

// Everything an H application needs; passed by value to kernels.
struct Plan {
    int n1, n2, n3, npw, nstick, nxcol;
    int n2p;                 // row stride of the on-chip xy-plane: n2 rounded up to odd (bank spread)
    int n3p;                 // stride of the on-chip sticks: n3 rounded up to odd
    int nplanes;             // xy-planes transformed together per barrier (chosen per launch)
    AxisPlan ax[3];
    const int* g2s;          // [npw]    stick * n3p + (m3 mod n3)
    const int* stick_xy;     // [nstick] (m1 mod n1) * n2p + (m2 mod n2): the stick's place in the plane
    const int* xbase;        // [nxcol]  x * n2p for every x that has a stick
    const double* vloc;      // [n3][n1][n2p] (pad entries 0)
    const float2* vloc_dd;   // [n3][n1][n2p] the same as float-float (hi, lo)
    const double* kin;       // [npw]
    const double2* twid;     // [n1 + n2 + n3]  exp(-2 pi i m / n_axis)
    int nproj;
    const double2* beta;     // [nproj][npw]
    const double* dkb;       // [nproj]
    int nocc;
    const double2* psi;      // [nocc][npw]
    double inv_nbox;         // 1 / (n1 n2 n3)
    // float-float mirrors (hi, lo) used by the float-float arithmetic policy
    const float4* psi_dd;    // [nocc][npw]
    const float4* beta_dd;   // [nproj][npw]
    const float2* kin_dd;    // [npw]
    // FP32 mirrors used by the single-precision policy
    const float* vloc_f;     // [n3][n1][n2p]
    const float2* psi_f;     // [nocc][npw]
    const float2* beta_f;    // [nproj][npw]
    const float* kin_f;      // [npw]
    // cluster split of the box (csize == 1: one CTA holds it all)
    int csize;               // CTAs per vector
    int nstick_loc;          // most sticks one rank holds (sizes the stick buffer)
    const int* part;         // [2][kMaxCluster + 1]: plane-wave bounds g_r, then stick bounds s_r
    const int* stick_loc;    // [nstick] (owner rank << 16) | index of the stick in its owner's buffer
};

// Shared-memory carve-up of an H application (byte offsets from the dynamic base).
struct ApplySmem {
    int tw, sticks, plane, red, coef, coefc, part, end;
};

inline __host__ __device__ int align16(int b) { return (b + 15) & ~15; }

// Complex values per parity buffer of the cluster partial sums (and of the coefficient slots).
inline __host__ __device__ int coef_slots(const Plan& p) {
    int nc = p.nocc > p.nproj ? p.nocc : p.nproj;
    if (nc < kRedSlots) nc = kRedSlots;
    return (nc + 7) / 8 * 8 + 8;
}

// es: bytes per complex value of the arithmetic policy (16 FP64 / float-float, 8 FP32).
inline __host__ __device__ ApplySmem apply_smem_layout(const Plan& p, int es) {
    ApplySmem s;
    int off = 0;
    const int ns = coef_slots(p);
    s.tw = off;     off = align16(off + (p.n1 + p.n2 + p.n3) * es);
    s.sticks = off; off = align16(off + p.nstick_loc * p.n3p * es);
    s.plane = off;  off = align16(off + p.nplanes * p.n1 * p.n2p * es);
    s.red = off;    off = align16(off + (kMaxThreads / 32) * kRedSlots * 16);
    s.coef = off;   off = align16(off + ns * 16);
    s.coefc = off;  off = align16(off + ns * es);
    s.part = off;   off = align16(off + (p.csize > 1 ? 2 * ns * 16 : 0));
    s.end = off;
    return s;
}

// Shared memory of the Lanczos kernel's per-shift state after the H application's carve-up.
inline __host__ __device__ int lanczos_extra(int ns) {
    return 3 * align16(ns * 16) + 3 * align16(ns * 8) + 2 * align16(ns * 4);
}

// The part of a vector one CTA works on: rank `rank` of the cluster owns the plane waves
// [g0, g1) and holds the sticks [s0, s1) (the whole vector when P.csize == 1).
struct Part {
    int rank, g0, g1, s0, s1;
};

__device__ __forceinline__ Part make_part(const Plan& P) {
    Part q;
    if (P.csize > 1) {
        q.rank = (int)cg::this_cluster().block_rank();
        q.g0 = P.part[q.rank];
        q.g1 = P.part[q.rank + 1];
        q.s0 = P.part[kMaxCluster + 1 + q.rank];
        q.s1 = P.part[kMaxCluster + 2 + q.rank];
    } else {
        q.rank = 0;
        q.g0 = 0;
        q.g1 = P.npw;
        q.s0 = 0;
        q.s1 = P.nstick;
    }
    return q;
}

// The next work item of the launch for this owner: rank 0 of a cluster takes it from the
// queue and every rank reads it (rank 0 overwrites it, or exits, only after all have read).
__device__ __forceinline__ int next_item(const Plan& P, int* counter) {
    __shared__ int s_r;
    if (P.csize == 1) {
        __syncthreads();
        if (threadIdx.x == 0) s_r = atomicAdd(counter, 1);
        __syncthreads();
        return s_r;
    }
    cg::cluster_group cl = cg::this_cluster();
    if (cl.block_rank() == 0 && threadIdx.x == 0) s_r = atomicAdd(counter, 1);
    cl.sync();
    const int r = *cl.map_shared_rank(&s_r, 0u);
    cl.sync();
    return r;
}

// Scratch of the block and cluster reductions.  Cluster partial sums alternate between two
// buffers (par), so one cluster barrier per reduction suffices: a rank writes buffer par of
// reduction n + 2 only after the barrier of reduction n + 1, which every rank reaches after
// reading the buffers of reduction n.
struct Red {
    double2* red;     // per-warp slots of block_sum
    double2* part;    // [2][stride] this CTA's partial sums (clusters only)
    int stride;
    int par;
};

__device__ __forceinline__ Red make_red(const Plan& P, unsigned char* smem, const ApplySmem& L) {
    Red R;
    R.red = reinterpret_cast<double2*>(smem + L.red);
    R.part = reinterpret_cast<double2*>(smem + L.part);
    R.stride = coef_slots(P);
    R.par = 0;
    return R;
}

// ----------------------------------------------------------------------- complex helpers

__device__ __forceinline__ double2 cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cscal(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a * b + c
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // scaled division (Smith's method) to avoid overflow in |b|^2
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// ------------------------------------------------------------------- block reductions

// Sums NV complex values over the CTA; the totals land in out[0..NV).  All threads call.
template <int NV>
__device__ __forceinline__ void block_sum(double2 (&v)[NV], double2* red, double2* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[i].x += __shfl_down_sync(0xffffffffu, v[i].x, o);
            v[i].y += __shfl_down_sync(0xffffffffu, v[i].y, o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[warp * kRedSlots + i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double2 s = cz();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, red[w * kRedSlots + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// out[v] = sum_g conj(V[v*ld + g]) x[g] for v < nv (out must hold nv rounded up to 8).
__device__ __forceinline__ void block_dots(const double2* V, int nv, int ld,
                                           const double2* x, int n, double2* red, double2* out) {
    for (int v0 = 0; v0 < nv; v0 += 8) {
        double2 acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = cz();
        const int cnt = min(8, nv - v0);
        for (int g = threadIdx.x; g < n; g += blockDim.x) {
            const double2 xv = x[g];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < cnt) acc[i] = cadd(acc[i], cmulc(V[(size_t)(v0 + i) * ld + g], xv));
        }
        block_sum<8>(acc, red, out + v0);
    }
}

// ------------------------------------------------------------------ arithmetic policies
//
// The FFT part of an H application is written once over a policy type Ar:
//   Ar::C      complex value held in shared memory / registers (16 bytes for both policies)
//   ArF64      native FP64 (the FP64 pipe: ~1/64 of the FP32 rate on this GPU)
//   ArDF       float-float ("double-FP32") numbers hi + lo on the FP32 pipes, ~48-bit
//              significand, from Dekker's and Knuth's error-free transformations:
//              two_sum(a, b) = (s, e) with s = fl(a + b), e = a + b - s exactly;
//              two_prod(a, b) = (p, e) with p = fl(a b), e = fma(a, b, -p) exactly.

struct ArF64 {
    using C = double2;
    static __device__ __forceinline__ C add(C a, C b) { return cadd(a, b); }
    static __device__ __forceinline__ C sub(C a, C b) { return csub(a, b); }
    static __device__ __forceinline__ C mul(C a, C b) { return cmul(a, b); }
    static __device__ __forceinline__ C conj(C a) { return make_double2(a.x, -a.y); }
    // a * (sign i)
    template <int SIGN>
    static __device__ __forceinline__ C muli(C a) { return make_double2(-SIGN * a.y, SIGN * a.x); }
    // a * c for a real constant c given as (hi, lo) float pair and its double value
    static __device__ __forceinline__ C scal(C a, double c, float, float) { return cscal(a, c); }
    static __device__ __forceinline__ C from_d(double2 a) { return a; }
    static __device__ __forceinline__ double2 to_d(C a) { return a; }
    static __device__ __forceinline__ C zero() { return cz(); }
    // the potential sample in this policy's format, and the product with it
    using VT = double;
    static __device__ __forceinline__ VT vload(const Plan& P, size_t i) { return P.vloc[i]; }
    static __device__ __forceinline__ C vmul(C a, VT v) { return cscal(a, v); }
    // real scalars and reciprocal-space data in this policy's format
    using R = double;
    static __device__ __forceinline__ R real(double x) { return x; }
    static __device__ __forceinline__ C scalr(C a, R s) { return cscal(a, s); }
    static __device__ __forceinline__ C psi(const Plan& P, size_t i) { return P.psi[i]; }
    static __device__ __forceinline__ C beta(const Plan& P, size_t i) { return P.beta[i]; }
    static __device__ __forceinline__ C kinx(const Plan& P, int g, C x) { return cscal(x, P.kin[g]); }
    // |a|^2 accumulated into the real part of acc
    static __device__ __forceinline__ C acc_norm(C acc, C a) { return make_double2(acc.x + cabs2(a), acc.y); }
    // long sums (dots and projections): the accumulator is a value of the policy's type
    using A = C;
    static __device__ __forceinline__ A acc_of(C a) { return a; }
    static __device__ __forceinline__ void acc_cmac(A& a, C r, C x) { a = add(a, mul(conj(r), x)); }   // a += conj(r) x
    static __device__ __forceinline__ void acc_mac(A& a, C c, C p) { a = add(a, mul(c, p)); }          // a += c p
    static __device__ __forceinline__ void acc_msub(A& a, C c, C p) { a = sub(a, mul(c, p)); }         // a -= c p
    static __device__ __forceinline__ C acc_val(A a) { return a; }
};

struct dd {
    float hi, lo;
};

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return dd{h, e - (h - s)};
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
// The leading product is rounded on its own (__fmul_rn): the compiler must not fuse it into
// the renormalising sum, whose error term assumes p = fl(a.hi b.hi).
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return dd{h, e - (h - p)};
}
__device__ __forceinline__ dd dd_from(double x) {
    const float h = __double2float_rn(x);
    return dd{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dd_to(dd a) { return (double)a.hi + (double)a.lo; }

struct ArDF {
    using C = float4;   // (re.hi, re.lo, im.hi, im.lo)
    static __device__ __forceinline__ dd re(C a) { return dd{a.x, a.y}; }
    static __device__ __forceinline__ dd im(C a) { return dd{a.z, a.w}; }
    static __device__ __forceinline__ C mk(dd r, dd i) { return make_float4(r.hi, r.lo, i.hi, i.lo); }
    static __device__ __forceinline__ C add(C a, C b) { return mk(dd_add(re(a), re(b)), dd_add(im(a), im(b))); }
    static __device__ __forceinline__ C sub(C a, C b) {
        return mk(dd_add(re(a), dd_neg(re(b))), dd_add(im(a), dd_neg(im(b))));
    }
    // a b with each part formed as one error-free sum: the two leading products and their
    // exact errors (FMA), their sum by TwoSum, the four cross terms hi * lo accumulated in
    // the low word, one renormalisation (38 FP32 operations instead of 50 for two dd_mul
    // pairs and two dd_add; the same terms are kept).
    static __device__ __forceinline__ dd dot2(float a, float al, float b, float bl, float c, float cl, float d,
                                             float dl) {
        // a b + c d, (a, al) etc. being the (hi, lo) words
        const float p = __fmul_rn(a, b), q = __fmul_rn(c, d);   // not fused into the sums below
        const float ep = fmaf(a, b, -p), eq = fmaf(c, d, -q);
        const float s = p + q;
        const float bb = s - p;
        float t = (p - (s - bb)) + (q - bb);
        t += ep + eq;
        t = fmaf(a, bl, t);
        t = fmaf(al, b, t);
        t = fmaf(c, dl, t);
        t = fmaf(cl, d, t);
        const float h = s + t;
        return dd{h, t - (h - s)};
    }
    static __device__ __forceinline__ C mul(C a, C b) {
        const dd r = dot2(a.x, a.y, b.x, b.y, -a.z, -a.w, b.z, b.w);
        const dd i = dot2(a.x, a.y, b.z, b.w, a.z, a.w, b.x, b.y);
        return mk(r, i);
    }
    static __device__ __forceinline__ C conj(C a) { return make_float4(a.x, a.y, -a.z, -a.w); }
    template <int SIGN>
    static __device__ __forceinline__ C muli(C a) {
        return SIGN > 0 ? make_float4(-a.z, -a.w, a.x, a.y) : make_float4(a.z, a.w, -a.x, -a.y);
    }
    static __device__ __forceinline__ C scal(C a, double, float ch, float cl) {
        const dd c{ch, cl};
        return mk(dd_mul(re(a), c), dd_mul(im(a), c));
    }
    static __device__ __forceinline__ C from_d(double2 a) { return mk(dd_from(a.x), dd_from(a.y)); }
    static __device__ __forceinline__ double2 to_d(C a) { return make_double2(dd_to(re(a)), dd_to(im(a))); }
    static __device__ __forceinline__ C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    using VT = float2;
    static __device__ __forceinline__ VT vload(const Plan& P, size_t i) { return P.vloc_dd[i]; }
    static __device__ __forceinline__ C vmul(C a, VT v) {
        const dd c{v.x, v.y};
        return mk(dd_mul(re(a), c), dd_mul(im(a), c));
    }
    using R = dd;
    static __device__ __forceinline__ R real(double x) { return dd_from(x); }
    static __device__ __forceinline__ C scalr(C a, R s) { return mk(dd_mul(re(a), s), dd_mul(im(a), s)); }
    static __device__ __forceinline__ C psi(const Plan& P, size_t i) { return P.psi_dd[i]; }
    static __device__ __forceinline__ C beta(const Plan& P, size_t i) { return P.beta_dd[i]; }
    static __device__ __forceinline__ C kinx(const Plan& P, int g, C x) {
        const float2 t = P.kin_dd[g];
        return scalr(x, dd{t.x, t.y});
    }
    static __device__ __forceinline__ C acc_norm(C acc, C a) {
        const dd m = dd_add(dd_mul(re(a), re(a)), dd_mul(im(a), im(a)));
        return mk(dd_add(re(acc), m), im(acc));
    }
    // Long sums (the projector and occupied-state dots and projections) accumulate lazily:
    // per part an unevaluated pair (s, e) -- the leading products enter s by TwoSum, and e
    // gathers their exact rounding errors (FMA), the TwoSum errors and the hi * lo cross
    // terms -- renormalised once at the end (48 FP32 operations per complex term instead of
    // 60 for a float-float multiply and add; the same terms are kept, and the error of the
    // sum stays at the float-float level: e's own rounding is 2^-24 of terms that are
    // themselves 2^-24 of the products).  That holds for short sums only: e grows with the
    // number of terms n and its own rounding with it (about n^2 2^-48 of the largest partial
    // sum at worst), so the lazy form serves the per-thread sums of a few hundred terms (the
    // dots' per-lane partials, the projections over the occupied states and projectors) and
    // not the sums over thousands of Lanczos steps in x = V y.
    using A = float4;   // (s_re, e_re, s_im, e_im); a float-float value (hi, lo) is such a pair
    // (s, e) += a b + c d for the (hi, lo) words (a, al), (b, bl), (c, cl), (d, dl)
    static __device__ __forceinline__ void lazy2(float& s, float& e, float a, float al, float b, float bl, float c,
                                                 float cl, float d, float dl) {
        const float p = __fmul_rn(a, b), q = __fmul_rn(c, d);   // not fused into the sums below
        const float ep = fmaf(a, b, -p), eq = fmaf(c, d, -q);
        const float s1 = s + p, b1 = s1 - s;
        const float t1 = (s - (s1 - b1)) + (p - b1);
        const float s2 = s1 + q, b2 = s2 - s1;
        const float t2 = (s1 - (s2 - b2)) + (q - b2);
        float f = e + ((ep + eq) + (t1 + t2));
        f = fmaf(a, bl, f);
        f = fmaf(al, b, f);
        f = fmaf(c, dl, f);
        f = fmaf(cl, d, f);
        s = s2;
        e = f;
    }
    static __device__ __forceinline__ A acc_of(C a) { return a; }
    static __device__ __forceinline__ void acc_cmac(A& a, C r, C x) {   // a += conj(r) x
        lazy2(a.x, a.y, r.x, r.y, x.x, x.y, r.z, r.w, x.z, x.w);       // rr xr + ri xi
        lazy2(a.z, a.w, r.x, r.y, x.z, x.w, -r.z, -r.w, x.x, x.y);     // rr xi - ri xr
    }
    static __device__ __forceinline__ void acc_mac(A& a, C c, C p) {    // a += c p
        lazy2(a.x, a.y, c.x, c.y, p.x, p.y, -c.z, -c.w, p.z, p.w);     // cr pr - ci pi
        lazy2(a.z, a.w, c.x, c.y, p.z, p.w, c.z, c.w, p.x, p.y);       // cr pi + ci pr
    }
    static __device__ __forceinline__ void acc_msub(A& a, C c, C p) {   // a -= c p
        acc_mac(a, make_float4(-c.x, -c.y, -c.z, -c.w), p);
    }
    static __device__ __forceinline__ C acc_val(A a) {   // TwoSum of each pair
        const float hr = a.x + a.y, br = hr - a.x, hi = a.z + a.w, bi = hi - a.z;
        return make_float4(hr, (a.x - (hr - br)) + (a.y - br), hi, (a.z - (hi - bi)) + (a.w - bi));
    }
};

// Single precision: complex64 values, FP32 arithmetic and accumulation.
struct ArF32 {
    using C = float2;
    static __device__ __forceinline__ C add(C a, C b) { return make_float2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ C sub(C a, C b) { return make_float2(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ C mul(C a, C b) {
        return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
    }
    static __device__ __forceinline__ C conj(C a) { return make_float2(a.x, -a.y); }
    template <int SIGN>
    static __device__ __forceinline__ C muli(C a) { return make_float2(-SIGN * a.y, SIGN * a.x); }
    static __device__ __forceinline__ C scal(C a, double, float ch, float) { return make_float2(a.x * ch, a.y * ch); }
    static __device__ __forceinline__ C from_d(double2 a) {
        return make_float2(__double2float_rn(a.x), __double2float_rn(a.y));
    }
    static __device__ __forceinline__ double2 to_d(C a) { return make_double2((double)a.x, (double)a.y); }
    static __device__ __forceinline__ C zero() { return make_float2(0.f, 0.f); }
    using VT = float;
    static __device__ __forceinline__ VT vload(const Plan& P, size_t i) { return P.vloc_f[i]; }
    static __device__ __forceinline__ C vmul(C a, VT v) { return make_float2(a.x * v, a.y * v); }
    using R = float;
    static __device__ __forceinline__ R real(double x) { return __double2float_rn(x); }
    static __device__ __forceinline__ C scalr(C a, R s) { return make_float2(a.x * s, a.y * s); }
    static __device__ __forceinline__ C psi(const Plan& P, size_t i) { return P.psi_f[i]; }
    static __device__ __forceinline__ C beta(const Plan& P, size_t i) { return P.beta_f[i]; }
    static __device__ __forceinline__ C kinx(const Plan& P, int g, C x) { return scalr(x, P.kin_f[g]); }
    static __device__ __forceinline__ C acc_norm(C acc, C a) {
        return make_float2(fmaf(a.x, a.x, fmaf(a.y, a.y, acc.x)), acc.y);
    }
    // long sums (dots and projections): the accumulator is a value of the policy's type
    using A = C;
    static __device__ __forceinline__ A acc_of(C a) { return a; }
    static __device__ __forceinline__ void acc_cmac(A& a, C r, C x) { a = add(a, mul(conj(r), x)); }   // a += conj(r) x
    static __device__ __forceinline__ void acc_mac(A& a, C c, C p) { a = add(a, mul(c, p)); }          // a += c p
    static __device__ __forceinline__ void acc_msub(A& a, C c, C p) { a = sub(a, mul(c, p)); }         // a -= c p
    static __device__ __forceinline__ C acc_val(A a) { return a; }
};

// Real constants of the small DFTs as (double, float hi, float lo).
#define SGW_CONST(name, val)                                      \
    constexpr double name##_d = val;                              \
    constexpr float name##_h = (float)(val);                      \
    constexpr float name##_l = (float)((val) - (double)(float)(val));
SGW_CONST(kS3, 0.86602540378443864676)    // sin(2 pi / 3)
SGW_CONST(kC51, 0.30901699437494742410)   // cos(2 pi / 5)
SGW_CONST(kC52, -0.80901699437494742410)  // cos(4 pi / 5)
SGW_CONST(kS51, 0.95105651629515357212)   // sin(2 pi / 5)
SGW_CONST(kS52, 0.58778525229247312917)   // sin(4 pi / 5)
SGW_CONST(kHalf, 0.5)
#undef SGW_CONST

// Block sums of NV complex values per thread in the policy's format: the FP64 pair goes
// through block_sum; float-float values are reduced within each warp in float-float on the
// FP32 pipes (shuffles of the four floats), and only the per-warp partials are converted
// and summed in FP64 by NV threads (GB300's FP64 pipe is ~1/64 of its FP32 rate, so a
// shuffle tree of FP64 additions costs more than the dot products it finishes).
template <int NV>
__device__ __forceinline__ void block_sum_c(double2 (&v)[NV], double2* red, double2* out) {
    block_sum<NV>(v, red, out);
}
template <int NV>
__device__ __forceinline__ void block_sum_c(float4 (&v)[NV], double2* red, double2* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float4 t;
            t.x = __shfl_down_sync(0xffffffffu, v[i].x, o);
            t.y = __shfl_down_sync(0xffffffffu, v[i].y, o);
            t.z = __shfl_down_sync(0xffffffffu, v[i].z, o);
            t.w = __shfl_down_sync(0xffffffffu, v[i].w, o);
            v[i] = ArDF::add(v[i], t);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[warp * kRedSlots + i] = ArDF::to_d(v[i]);
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double2 s = cz();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, red[w * kRedSlots + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// FP32 complex values: warp sums in FP32, per-warp partials summed in FP64.
template <int NV>
__device__ __forceinline__ void block_sum_c(float2 (&v)[NV], double2* red, double2* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[i].x += __shfl_down_sync(0xffffffffu, v[i].x, o);
            v[i].y += __shfl_down_sync(0xffffffffu, v[i].y, o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[warp * kRedSlots + i] = make_double2((double)v[i].x, (double)v[i].y);
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double2 s = cz();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, red[w * kRedSlots + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// out[0..n) = sum over the ranks of the cluster, in rank order, of each rank's loc[0..n)
// (loc: the same shared-memory offset on every rank).  Every rank gets bit-identical sums.
__device__ __forceinline__ void cluster_combine(const Plan& P, const double2* loc, int n, double2* out) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double2 s = cz();
        for (int r = 0; r < P.csize; ++r) s = cadd(s, cl.map_shared_rank(loc, (unsigned)r)[i]);
        out[i] = s;
    }
    __syncthreads();
}

// Sums NV complex values per thread over the vector's owners (the CTA, or the cluster) into
// out[0..NV) (shared memory of this CTA).  All threads of every rank call.
template <int NV, class T>
__device__ __forceinline__ void part_sum(const Plan& P, Red& R, T (&v)[NV], double2* out) {
    if (P.csize == 1) {
        block_sum_c<NV>(v, R.red, out);
        return;
    }
    double2* loc = R.part + R.par * R.stride;
    R.par ^= 1;
    block_sum_c<NV>(v, R.red, loc);
    cluster_combine(P, loc, NV, out);
}

// Warp sum of NV complex values of the policy's type; lane 0 ends with the totals.
template <int NV>
__device__ __forceinline__ void warp_sum_c(double2 (&v)[NV]) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[i].x += __shfl_down_sync(0xffffffffu, v[i].x, o);
            v[i].y += __shfl_down_sync(0xffffffffu, v[i].y, o);
        }
}
template <int NV>
__device__ __forceinline__ void warp_sum_c(float4 (&v)[NV]) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float4 t;
            t.x = __shfl_down_sync(0xffffffffu, v[i].x, o);
            t.y = __shfl_down_sync(0xffffffffu, v[i].y, o);
            t.z = __shfl_down_sync(0xffffffffu, v[i].z, o);
            t.w = __shfl_down_sync(0xffffffffu, v[i].w, o);
            v[i] = ArDF::add(v[i], t);
        }
}
template <int NV>
__device__ __forceinline__ void warp_sum_c(float2 (&v)[NV]) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[i].x += __shfl_down_sync(0xffffffffu, v[i].x, o);
            v[i].y += __shfl_down_sync(0xffffffffu, v[i].y, o);
        }
}

// Rows of a dot product: the occupied states (WHICH = 0) or projectors (WHICH = 1) in the
// policy's format, or FP64 rows V[v ld + g] (WHICH = 2).
template <class Ar, int WHICH>
struct DotRows {
    const Plan& P;
    const double2* V;
    int ld;
    __device__ __forceinline__ typename Ar::C operator()(int v, int g) const {
        if constexpr (WHICH == 0) return Ar::psi(P, (size_t)v * P.npw + g);
        else if constexpr (WHICH == 1) return Ar::beta(P, (size_t)v * P.npw + g);
        else return V[(size_t)v * ld + g];
    }
};

// out[v] = sum_g conj(row_v[g]) x[g] for v < nv over the plane waves of the vector's owners.
// The rows come in groups of kDotRows; the (group, slice) work items -- a slice being every
// slices-th 32-wide chunk of the plane waves -- are spread over the warps, so both many rows
// (the occupied states of a large cell) and few rows keep every warp busy.  Each item is
// summed within its warp in the policy's arithmetic; the per-slice partials (FP64) are
// summed by one thread per row; one block barrier, and the cluster sum in FP64 (rank order).
// out (and the cluster partial buffer) must hold nv rounded up to 8.
constexpr int kDotRows = 4;          // rows per warp work item
constexpr bool kDotPrefetch = true;   // loads of the next pass before the arithmetic
constexpr int kDotChunks = 1;        // 32-wide plane-wave chunks per pass

template <class Ar, int WHICH>
__device__ __forceinline__ void part_dots_rows(const Plan& P, const Part& q, Red& R, int nv, const DotRows<Ar, WHICH>& row,
                                               const typename Ar::C* x, double2* out) {
    using C = typename Ar::C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double2* dst = P.csize == 1 ? out : R.part + R.par * R.stride;
    constexpr int RW = kDotRows;
    const int ngroups = (nv + RW - 1) / RW;
    const int slices = max(1, nw / max(ngroups, 1));
    for (int t = warp; t < ngroups * slices; t += nw) {
        const int gi = t / slices, sl = t - gi * slices;
        const int v0 = gi * RW, cnt = min(RW, nv - v0);
        const int gs = 32 * slices;
        typename Ar::A a[RW];
#pragma unroll
        for (int i = 0; i < RW; ++i) a[i] = Ar::acc_of(Ar::zero());
        int g = q.g0 + sl * 32 + lane;
        // U chunks of 32 plane waves per pass: their loads first, then their arithmetic;
        // with kDotPrefetch the next pass's loads are issued before this pass's arithmetic.
        // Rows past the end of a chunk read as zeros, which add nothing.
        constexpr int U = kDotChunks;
        C xn[U], rn[U][RW];
        auto load = [&](int gb) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int gg = gb + u * gs;
                const bool ok = gg < q.g1;
                xn[u] = ok ? x[gg] : Ar::zero();
#pragma unroll
                for (int i = 0; i < RW; ++i) rn[u][i] = (ok && i < cnt) ? row(v0 + i, gg) : Ar::zero();
            }
        };
        if constexpr (kDotPrefetch) load(g);
        for (; g < q.g1; g += U * gs) {
            if constexpr (!kDotPrefetch) load(g);
            C xv[U], rv[U][RW];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                xv[u] = xn[u];
#pragma unroll
                for (int i = 0; i < RW; ++i) rv[u][i] = rn[u][i];
            }
            if constexpr (kDotPrefetch)
                if (g + U * gs < q.g1) load(g + U * gs);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < RW; ++i)
                    if (i < cnt) Ar::acc_cmac(a[i], rv[u][i], xv[u]);
        }
        C acc[RW];
#pragma unroll
        for (int i = 0; i < RW; ++i) acc[i] = Ar::acc_val(a[i]);
        warp_sum_c<RW>(acc);
        if (lane == 0) {
            for (int i = 0; i < cnt; ++i) {
                const double2 d = Ar::to_d(acc[i]);
                if (slices == 1) dst[v0 + i] = d;
                else R.red[(v0 + i) * slices + sl] = d;
            }
        }
    }
    __syncthreads();
    if (slices > 1) {
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            double2 s = cz();
            for (int sl = 0; sl < slices; ++sl) s = cadd(s, R.red[v * slices + sl]);
            dst[v] = s;
        }
        __syncthreads();
    }
    if (P.csize > 1) {
        R.par ^= 1;
        cluster_combine(P, dst, nv, out);
    }
}

// Dots with the occupied states (WHICH = 0) or the projectors (WHICH = 1), policy format.
template <class Ar, int WHICH>
__device__ __forceinline__ void part_dots(const Plan& P, const Part& q, Red& R, int nv, const typename Ar::C* x,
                                          double2* out) {
    const DotRows<Ar, WHICH> row{P, nullptr, 0};
    part_dots_rows<Ar, WHICH>(P, q, R, nv, row, x, out);
}

// FP64 dots out[v] = sum_g conj(V[v ld + g]) x[g] over the owners' plane waves (V: FP64 rows).
__device__ __forceinline__ void part_dots_f64(const Plan& P, const Part& q, Red& R, const double2* V, int nv, int ld,
                                              const double2* x, double2* out) {
    const DotRows<ArF64, 2> row{P, V, ld};
    part_dots_rows<ArF64, 2>(P, q, R, nv, row, x, out);
}

// -------------------------------------------------------------- shared-memory FFT lines

// Small DFTs of radix 2, 3, 4, 5 with exponent sign SIGN (-1 forward, +1 inverse).
template <class Ar, int SIGN>
__device__ __forceinline__ void dft_small(typename Ar::C (&v)[5], int R) {
    using C = typename Ar::C;
    if (R == 4) {
        const C t0 = Ar::add(v[0], v[2]), t1 = Ar::sub(v[0], v[2]);
        const C t2 = Ar::add(v[1], v[3]);
        const C t3 = Ar::template muli<SIGN>(Ar::sub(v[1], v[3]));
        v[0] = Ar::add(t0, t2);
        v[2] = Ar::sub(t0, t2);
        v[1] = Ar::add(t1, t3);
        v[3] = Ar::sub(t1, t3);
    } else if (R == 2) {
        const C a = v[0];
        v[0] = Ar::add(a, v[1]);
        v[1] = Ar::sub(a, v[1]);
    } else if (R == 3) {
        const C t1 = Ar::add(v[1], v[2]), t2 = Ar::sub(v[1], v[2]);
        const C m1 = Ar::sub(v[0], Ar::scal(t1, kHalf_d, kHalf_h, kHalf_l));
        const C m2 = Ar::template muli<SIGN>(Ar::scal(t2, kS3_d, kS3_h, kS3_l));
        v[0] = Ar::add(v[0], t1);
        v[1] = Ar::add(m1, m2);
        v[2] = Ar::sub(m1, m2);
    } else {  // R == 5
        const C t1 = Ar::add(v[1], v[4]), t2 = Ar::add(v[2], v[3]);
        const C t3 = Ar::sub(v[1], v[4]), t4 = Ar::sub(v[2], v[3]);
        const C a1 = Ar::add(v[0], Ar::add(Ar::scal(t1, kC51_d, kC51_h, kC51_l), Ar::scal(t2, kC52_d, kC52_h, kC52_l)));
        const C a2 = Ar::add(v[0], Ar::add(Ar::scal(t1, kC52_d, kC52_h, kC52_l), Ar::scal(t2, kC51_d, kC51_h, kC51_l)));
        const C b1 = Ar::add(Ar::scal(t3, kS51_d, kS51_h, kS51_l), Ar::scal(t4, kS52_d, kS52_h, kS52_l));
        const C b2 = Ar::sub(Ar::scal(t3, kS52_d, kS52_h, kS52_l), Ar::scal(t4, kS51_d, kS51_h, kS51_l));
        const C ib1 = Ar::template muli<SIGN>(b1);
        const C ib2 = Ar::template muli<SIGN>(b2);
        v[0] = Ar::add(v[0], Ar::add(t1, t2));
        v[1] = Ar::add(a1, ib1);
        v[4] = Ar::sub(a1, ib1);
        v[2] = Ar::add(a2, ib2);
        v[3] = Ar::sub(a2, ib2);
    }
}

// Butterfly `b` of a stage of fft_inplace: its first element's index in `data`.  The line
// index varies fastest with b, so the eight threads of a quarter-warp read the same offset
// of eight neighbouring lines: line starts N3p or N2p (odd) elements apart, or adjacent
// rows, which fall in distinct shared-memory banks for 16-byte elements.
// q = a / n, r = a - q n for 0 <= a < 2^22 and n >= 1, given inv = 1.0f / n: the float
// quotient is within one of the true one and is corrected exactly (an integer division by a
// run-time divisor costs several times more instructions than this).
__device__ __forceinline__ int divmod_f(int a, int n, float inv, int& r) {
    int q = __float2int_rz(__int2float_rn(a) * inv);
    r = a - q * n;
    if (r < 0) {
        --q;
        r += n;
    } else if (r >= n) {
        ++q;
        r -= n;
    }
    return q;
}

struct FftIdx {   // per-stage divisors of fft_bfly_base and their reciprocals
    int nlines, m, lpp;
    float inv_nlines, inv_m, inv_lpp;
};

__device__ __forceinline__ int fft_bfly_base(int b, const FftIdx& d, int L, int pstride,
                                             const int* __restrict__ line_base, int ls, int es, int& j) {
    int l, q;
    const int rem = divmod_f(b, d.nlines, d.inv_nlines, l);
    const int blk = divmod_f(rem, d.m, d.inv_m, j);
    const int pl = divmod_f(l, d.lpp, d.inv_lpp, q);
    return pl * pstride + (line_base ? line_base[q] : q * ls) + (blk * L + j) * es;
}

// One stage of fft_inplace with a compile-time radix R: every butterfly reads its R
// elements m * es apart, twiddles (before the DFT for DIT, after it for DIF), applies the
// R-point DFT and writes back to the same places.  Butterflies b and b + nt run together.
template <class Ar, int SIGN, bool DIF, int R>
__device__ __forceinline__ void fft_stage(typename Ar::C* data, int total, int nlines, int m, int lpp, int pstride,
                                          const int* __restrict__ line_base, int ls, int es,
                                          const typename Ar::C* tw, int twstep) {
    using C = typename Ar::C;
    const int L = m * R, mes = m * es, nt = blockDim.x;
    const FftIdx d{nlines, m, lpp, 1.0f / (float)nlines, 1.0f / (float)m, 1.0f / (float)lpp};
    for (int b0 = threadIdx.x; b0 < total; b0 += 2 * nt) {
        const bool two = b0 + nt < total;
        int j[2], base[2];
        C v[2][5];
        base[0] = fft_bfly_base(b0, d, L, pstride, line_base, ls, es, j[0]);
        base[1] = two ? fft_bfly_base(b0 + nt, d, L, pstride, line_base, ls, es, j[1]) : base[0];
        if (!two) j[1] = j[0];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int k = 0; k < R; ++k) v[u][k] = data[base[u] + k * mes];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!DIF && j[u] != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    C w = tw[j[u] * k * twstep];
                    if (SIGN > 0) w = Ar::conj(w);
                    v[u][k] = Ar::mul(v[u][k], w);
                }
            }
            dft_small<Ar, SIGN>(v[u], R);
            if (DIF && j[u] != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    C w = tw[j[u] * k * twstep];
                    if (SIGN > 0) w = Ar::conj(w);
                    v[u][k] = Ar::mul(v[u][k], w);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) data[base[0] + k * mes] = v[0][k];
        if (two) {
#pragma unroll
            for (int k = 0; k < R; ++k) data[base[1] + k * mes] = v[1][k];
        }
    }
}

// P-point DFT of v[0..P) in registers, sign SIGN, for P in {2, 3, 4, 5, 8, 9}.  A composite
// P = Q R is split as X[k1 + Q k2] = sum_n2 w_R^(n2 k2) w_P^(n2 k1) sum_n1 v[R n1 + n2] w_Q^(n1 k1)
// (Cooley-Tukey inside the thread); w_P^m = tw[tstep m] with tw[i] = exp(-2 pi i i / N),
// tstep = N / P (conjugated for SIGN > 0).
template <class Ar, int SIGN, int P>
__device__ __forceinline__ void dft_reg(typename Ar::C* v, const typename Ar::C* tw, int tstep) {
    using C = typename Ar::C;
    if constexpr (P <= 5) {
        C t[5];
#pragma unroll
        for (int k = 0; k < P; ++k) t[k] = v[k];
        dft_small<Ar, SIGN>(t, P);
#pragma unroll
        for (int k = 0; k < P; ++k) v[k] = t[k];
    } else {
        constexpr int Q = P == 8 ? 4 : 3;
        constexpr int R = P / Q;
        C y[P];
#pragma unroll
        for (int n2 = 0; n2 < R; ++n2) {
            C t[Q];
#pragma unroll
            for (int n1 = 0; n1 < Q; ++n1) t[n1] = v[R * n1 + n2];
            dft_reg<Ar, SIGN, Q>(t, tw, tstep);
#pragma unroll
            for (int k1 = 0; k1 < Q; ++k1) {
                if (n2 != 0 && k1 != 0) {
                    C w = tw[tstep * n2 * k1];
                    if (SIGN > 0) w = Ar::conj(w);
                    t[k1] = Ar::mul(t[k1], w);
                }
                y[n2 * Q + k1] = t[k1];
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) {
            C t[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) t[n2] = y[n2 * Q + k1];
            dft_reg<Ar, SIGN, R>(t, tw, tstep);
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) v[k1 + Q * k2] = t[k2];
        }
    }
}

// One stage of the prime-factor algorithm (Good-Thomas) for the coprime part P of N: for
// m < N / P, the P elements at (P m + (N / P) k) mod N, k < P, are replaced by their P-point
// DFT.  The stages of all parts commute and need no twiddles between them; starting from
// natural order they leave X_f at the position p with p mod P_t = (N / P_t) k_t mod P_t, f the
// CRT combination of the k_t (and take that order back to natural order with the opposite
// sign).  Line l = p * lpp + q as in fft_inplace; consecutive threads take neighbouring lines.
template <class Ar, int SIGN, int P>
__device__ __forceinline__ void fft_pfa_stage(typename Ar::C* data, int nlines, int lpp, int pstride,
                                              const int* __restrict__ line_base, int ls, int es, int N,
                                              const typename Ar::C* tw) {
    using C = typename Ar::C;
    const int st = N / P, total = nlines * st, nt = blockDim.x;
    const float inv_nlines = 1.0f / (float)nlines, inv_lpp = 1.0f / (float)lpp;
    for (int b = threadIdx.x; b < total; b += nt) {
        int l, q;
        const int m = divmod_f(b, nlines, inv_nlines, l);
        const int pl = divmod_f(l, lpp, inv_lpp, q);
        const int base = pl * pstride + (line_base ? line_base[q] : q * ls);
        int pos[P];
        C v[P];
        int p0 = P * m;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            pos[k] = base + p0 * es;
            v[k] = data[pos[k]];
            p0 += st;
            if (p0 >= N) p0 -= N;
        }
        dft_reg<Ar, SIGN, P>(v, tw, st);
#pragma unroll
        for (int k = 0; k < P; ++k) data[pos[k]] = v[k];
    }
}

// In-place batched mixed-radix FFT (sign SIGN: exp(SIGN 2 pi i n k / N), unnormalised) of
// `nlines` lines of length N = ax.n in shared memory, `lpp` lines per plane, planes
// `pstride` elements apart; line l = p * lpp + q starts at
// p * pstride + (line_base ? line_base[q] : q * ls), element i at base + i * es.
// Decimation in frequency (DIF) takes natural order to digit-reversed order: with
// k = r_0 + R_0 (r_1 + R_1 (r_2 + ...)), X_k lands at position sum_s r_s m_s.  Decimation in
// time (DIT, the stages in reverse) takes that order back to natural order.  A stage with
// radix R on blocks of L = m R elements reads x[blk L + j + k m] (k < R), applies the
// R-point DFT and the twiddles w_L^(j k), and writes back to the same places, so the
// butterflies of a stage are disjoint and need no barrier between them: one barrier per
// stage.  When the axis has prime-factor parts (ax.npart > 0) the stages are those of the
// prime-factor algorithm instead (fft_pfa_stage: no twiddles between stages, another
// permutation of real space; DIF = true runs the parts in order, DIT in reverse).
// tw[i] = exp(-2 pi i i / N).  All threads of the CTA must call.
template <class Ar, int SIGN, bool DIF>
__device__ void fft_inplace(typename Ar::C* data, int nlines, int lpp, int pstride, const int* __restrict__ line_base,
                            int ls, int es, const AxisPlan& ax, const typename Ar::C* tw) {
    const int N = ax.n;
    if (ax.npart > 0) {   // prime-factor algorithm: parts in order for DIF, reversed for DIT
        for (int ti = 0; ti < ax.npart; ++ti) {
            const int P = ax.part[DIF ? ti : ax.npart - 1 - ti];
            switch (P) {
                case 2: fft_pfa_stage<Ar, SIGN, 2>(data, nlines, lpp, pstride, line_base, ls, es, N, tw); break;
                case 3: fft_pfa_stage<Ar, SIGN, 3>(data, nlines, lpp, pstride, line_base, ls, es, N, tw); break;
                case 4: fft_pfa_stage<Ar, SIGN, 4>(data, nlines, lpp, pstride, line_base, ls, es, N, tw); break;
                case 5: fft_pfa_stage<Ar, SIGN, 5>(data, nlines, lpp, pstride, line_base, ls, es, N, tw); break;
                case 8: fft_pfa_stage<Ar, SIGN, 8>(data, nlines, lpp, pstride, line_base, ls, es, N, tw); break;
                default: fft_pfa_stage<Ar, SIGN, 9>(data, nlines, lpp, pstride, line_base, ls, es, N, tw); break;
            }
            __syncthreads();
        }
        return;
    }
    for (int si = 0; si < ax.nst; ++si) {
        const int s = DIF ? si : ax.nst - 1 - si;
        const int R = ax.rad[s], m = ax.span[s];
        const int nb = N / R, twstep = N / (m * R), total = nlines * nb;
        switch (R) {
            case 4: fft_stage<Ar, SIGN, DIF, 4>(data, total, nlines, m, lpp, pstride, line_base, ls, es, tw, twstep); break;
            case 3: fft_stage<Ar, SIGN, DIF, 3>(data, total, nlines, m, lpp, pstride, line_base, ls, es, tw, twstep); break;
            case 5: fft_stage<Ar, SIGN, DIF, 5>(data, total, nlines, m, lpp, pstride, line_base, ls, es, tw, twstep); break;
            default: fft_stage<Ar, SIGN, DIF, 2>(data, total, nlines, m, lpp, pstride, line_base, ls, es, tw, twstep); break;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------- H application

enum : int {
    APPLY_PROJ_OUT = 1,   // y <- P_c y
    APPLY_SUB_Z = 2       // y <- y - z x
};

// Loads the twiddle tables of the plan into shared memory (call once per kernel).
template <class Ar>
__device__ __forceinline__ void load_twiddles(const Plan& P, unsigned char* smem) {
    const ApplySmem L = apply_smem_layout(P, (int)sizeof(typename Ar::C));
    typename Ar::C* tw = reinterpret_cast<typename Ar::C*>(smem + L.tw);
    for (int i = threadIdx.x; i < P.n1 + P.n2 + P.n3; i += blockDim.x) tw[i] = Ar::from_d(P.twid[i]);
    __syncthreads();
}

// y = H x  (+ options) for one vector, by the CTA or the cluster that owns it (each rank
// reads and writes only its own plane waves [q.g0, q.g1) of x and y); x and y are vectors of
// the policy's type (global, must not alias).  Steps: KB coefficients c_p = <beta_p|x>;
// scatter x into the sticks; inverse FFT along z on the sticks; per group of z-planes (this
// rank's planes): gather the planes' stick elements (from every rank's shared memory in a
// cluster), inverse FFT along y (only the x-columns that hold sticks) and x, multiply by V(r),
// forward FFT along x and y, scatter back into the sticks; forward FFT along z; gather the
// sphere, scale by 1/N^3 and add T_G x_G + sum_p D_p c_p beta_p(G); optionally project with
// P_c and subtract z x.  (The inverse FFTs leave real space permuted along each axis --
// digit-reversed or in the prime-factor order -- where V is stored in the same order; the
// forward FFTs return to natural order, so the permutation costs nothing.)  All vector
// arithmetic in the policy's arithmetic; the reductions of the projections in FP64.
// x and y may have been written earlier in the same kernel, so they are read through the
// coherent path (no __restrict__ / read-only cache).
template <class Ar>
__device__ __noinline__ void apply_h_block(const Plan& P, unsigned char* smem, const Part& q, Red& R,
                                           const typename Ar::C* x, typename Ar::C* y, double2 zsh, int mode) {
    using C = typename Ar::C;
    const ApplySmem L = apply_smem_layout(P, (int)sizeof(C));
    const C* tw = reinterpret_cast<const C*>(smem + L.tw);
    C* sticks = reinterpret_cast<C*>(smem + L.sticks);
    C* plane = reinterpret_cast<C*>(smem + L.plane);
    double2* coef = reinterpret_cast<double2*>(smem + L.coef);
    C* coefc = reinterpret_cast<C*>(smem + L.coefc);   // the coefficients in the policy's format
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3, npw = P.npw, nst = P.nstick;
    const int g0 = q.g0, g1 = q.g1, nsl = q.s1 - q.s0;
    const C* tw1 = tw;
    const C* tw2 = tw + n1;
    const C* tw3 = tw + n1 + n2;

    // non-local: D_p <beta_p|x>, kept in the policy's format
    if (P.nproj > 0) {
        part_dots<Ar, 1>(P, q, R, P.nproj, x, coef);
        if (tid < P.nproj) coefc[tid] = Ar::from_d(cscal(coef[tid], P.dkb[tid]));
        __syncthreads();
    }

    // sphere -> this rank's sticks
    const int n3p = P.n3p;
    for (int i = tid; i < nsl * n3p; i += nt) sticks[i] = Ar::zero();
    __syncthreads();
    for (int g = g0 + tid; g < g1; g += nt) sticks[P.g2s[g]] = x[g];
    __syncthreads();
    fft_inplace<Ar, +1, true>(sticks, nsl, nsl, 0, nullptr, n3p, 1, P.ax[2], tw3);
    if (P.csize > 1) cg::this_cluster().sync();   // every rank's sticks transformed

    // this rank's xy-planes, nplanes per pass: one set of barriers serves all of them
    const int n2p = P.n2p, psz = n1 * n2p;
    const int z0 = q.rank * n3 / P.csize, z1 = (q.rank + 1) * n3 / P.csize;
    for (int iz0 = z0; iz0 < z1; iz0 += P.nplanes) {
        const int npl = min(P.nplanes, z1 - iz0);
        for (int i = tid; i < npl * psz; i += nt) plane[i] = Ar::zero();
        __syncthreads();
        if (P.csize == 1) {
            for (int i = tid; i < npl * nst; i += nt) {
                const int pl = i / nst, s = i - pl * nst;
                plane[pl * psz + P.stick_xy[s]] = sticks[s * n3p + iz0 + pl];
            }
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int i = tid; i < npl * nst; i += nt) {
                const int pl = i / nst, s = i - pl * nst;
                const int loc = P.stick_loc[s];
                const C* src = cl.map_shared_rank(sticks, (unsigned)(loc >> 16));
                plane[pl * psz + P.stick_xy[s]] = src[(loc & 0xffff) * n3p + iz0 + pl];
            }
        }
        __syncthreads();
        fft_inplace<Ar, +1, true>(plane, npl * P.nxcol, P.nxcol, psz, P.xbase, 0, 1, P.ax[1], tw2);  // y, occupied x
        fft_inplace<Ar, +1, true>(plane, npl * n2, n2, psz, nullptr, 1, n2p, P.ax[0], tw1);          // x, every y
        const size_t zo = (size_t)iz0 * psz;
        {   // four potential loads in flight per thread
            const int cnt = npl * psz;
            for (int i0 = tid; i0 < cnt; i0 += 4 * nt) {
                typename Ar::VT vv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u * nt < cnt) vv[u] = Ar::vload(P, zo + i0 + u * nt);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u * nt < cnt) plane[i0 + u * nt] = Ar::vmul(plane[i0 + u * nt], vv[u]);
            }
        }
        __syncthreads();
        fft_inplace<Ar, -1, false>(plane, npl * n2, n2, psz, nullptr, 1, n2p, P.ax[0], tw1);
        fft_inplace<Ar, -1, false>(plane, npl * P.nxcol, P.nxcol, psz, P.xbase, 0, 1, P.ax[1], tw2);
        if (P.csize == 1) {
            for (int i = tid; i < npl * nst; i += nt) {
                const int pl = i / nst, s = i - pl * nst;
                sticks[s * n3p + iz0 + pl] = plane[pl * psz + P.stick_xy[s]];
            }
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int i = tid; i < npl * nst; i += nt) {
                const int pl = i / nst, s = i - pl * nst;
                const int loc = P.stick_loc[s];
                C* dst = cl.map_shared_rank(sticks, (unsigned)(loc >> 16));
                dst[(loc & 0xffff) * n3p + iz0 + pl] = plane[pl * psz + P.stick_xy[s]];
            }
        }
        __syncthreads();
    }
    if (P.csize > 1) cg::this_cluster().sync();   // every plane scattered back
    fft_inplace<Ar, -1, false>(sticks, nsl, nsl, 0, nullptr, n3p, 1, P.ax[2], tw3);

    // gather + kinetic + non-local
    {
        const typename Ar::R invn = Ar::real(P.inv_nbox);
        for (int g = g0 + tid; g < g1; g += nt) {
            typename Ar::A h = Ar::acc_of(Ar::add(Ar::scalr(sticks[P.g2s[g]], invn), Ar::kinx(P, g, x[g])));
#pragma unroll 8
            for (int p = 0; p < P.nproj; ++p) Ar::acc_mac(h, coefc[p], Ar::beta(P, (size_t)p * npw + g));
            y[g] = Ar::acc_val(h);
        }
    }
    __syncthreads();

    if (mode & APPLY_PROJ_OUT) {
        part_dots<Ar, 0>(P, q, R, P.nocc, y, coef);
        for (int v = tid; v < P.nocc; v += nt) coefc[v] = Ar::from_d(coef[v]);
        __syncthreads();
        const C zc = Ar::from_d(zsh);
        for (int g = g0 + tid; g < g1; g += nt) {
            typename Ar::A a = Ar::acc_of(y[g]);
#pragma unroll 8
            for (int v = 0; v < P.nocc; ++v) Ar::acc_msub(a, coefc[v], Ar::psi(P, (size_t)v * npw + g));
            C h = Ar::acc_val(a);
            if (mode & APPLY_SUB_Z) h = Ar::sub(h, Ar::mul(zc, x[g]));
            y[g] = h;
        }
    } else if (mode & APPLY_SUB_Z) {
        const C zc = Ar::from_d(zsh);
        for (int g = g0 + tid; g < g1; g += nt) y[g] = Ar::sub(y[g], Ar::mul(zc, x[g]));
    }
    __syncthreads();
}

}  // namespace sgw
