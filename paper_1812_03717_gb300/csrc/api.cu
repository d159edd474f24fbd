// C ABI of the shifted-Sternheimer library (declared in include/sgw.h).
//
// Host responsibilities: argument validation, the reciprocal lattice, the alias check of
// the FFT box, the stick tables, staging of host buffers, workspace management and the
// per-pair report.  Every arithmetic step of the path runs in the kernels of setup.cu
// and kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "setup.h"
#include "sgw.h"
#include "sgw_internal.cuh"

// NVTX ranges name the stages of each call for a profiler's timeline (header-only NVTX 3; a
// no-op unless a profiler is attached).
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define SGW_HAVE_NVTX 1
#endif

namespace sgw {
const void* solve_kernel_ptr();
}  // namespace sgw

using namespace sgw;

struct sgw_system {
    int dev = 0;
    double a[3][3];
    double b[3][3];
    double vol = 0.0;
    double k[3];
    double ecut = 0.0;
    int dims[3];
    int npw = 0, nstick = 0, nxcol = 0, nproj = 0, nocc = 0;
    std::vector<int> miller;     // [npw][3]
    std::vector<double> kin;     // [npw]
    std::vector<int> map;        // [npw]
    std::vector<double> eps;
    int lo[3], ext[3];           // Miller bounding box of the sphere (for Eq. 8 lookups)
    double v_mean = 0.0;         // <V_loc> over the box (preconditioner feature)
    // device
    int* d_miller = nullptr;
    double* d_kin = nullptr;
    int* d_stick_xy = nullptr;
    int* d_xbase = nullptr;
    double* d_vloc = nullptr;
    float2* d_vloc_dd = nullptr;
    double2* d_twid = nullptr;
    double2* d_beta = nullptr;
    double* d_dkb = nullptr;
    double2* d_psi = nullptr;
    float2* d_kin_dd = nullptr;  // float-float mirrors of T_G, beta_p(G), psi_v(G)
    float4* d_beta_dd = nullptr;
    float4* d_psi_dd = nullptr;
    int* d_lut = nullptr;
    float* d_vloc_f = nullptr;   // FP32 mirrors of V_loc(r), T_G, beta_p(G), psi_v(G)
    float* d_kin_f = nullptr;
    float2* d_beta_f = nullptr;
    float2* d_psi_f = nullptr;
    // sticks in canonical order (first plane wave of each), their plane-wave counts and places
    std::vector<int> stick_g0, stick_cnt, stick_xy, stick_of;   // stick_of: [npw]
    // the two cluster splits of the box: [0] 16-byte complex policies, [1] FP32
    int* d_g2s_s[2] = {nullptr, nullptr};
    int* d_stick_loc[2] = {nullptr, nullptr};
    int* d_part[2] = {nullptr, nullptr};
    void* d_ws = nullptr;        // solver workspace, grown on demand
    size_t ws_bytes = 0;
    Plan plan;                   // 16-byte policies (FP64, float-float)
    Plan plan8;                  // FP32 policy
    int forced_csize = 0;        // sgw_set_split: cluster size chosen by the caller (0: automatic)
};

namespace {

thread_local std::string g_err;

sgw_status fail(sgw_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

sgw_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    g_err = m;
    return e == cudaErrorMemoryAllocation ? SGW_ENOMEM : SGW_ECUDA;
}

#define SGW_CUDA(call, what)                              \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

// One NVTX range per stage of a call: next() closes the current stage and opens the next one;
// the last closes when the object goes out of scope (an early error return included).
struct Trace {
    bool open = false;
    explicit Trace(const char* name) { next(name); }
    void next(const char* name) {
#ifdef SGW_HAVE_NVTX
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
#else
        (void)name;
#endif
    }
    ~Trace() {
#ifdef SGW_HAVE_NVTX
        if (open) nvtxRangePop();
#endif
    }
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;
};

// Makes a system's device current for the rest of an entry point and gives the caller's
// current device back when it returns (work already queued on a stream is unaffected).
// Declared before anything whose destructor frees device memory, so those frees run while
// the system's device is still current.
struct DeviceScope {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A vector argument that may live on the host or the device.  Host data is copied to a
// temporary device buffer (in) and/or back (out).
// Staging buffers come from the stream-ordered allocator: no device-wide synchronisation,
// so solves of several systems on several streams stay concurrent.
struct Staged {
    void* dev = nullptr;
    const void* host_src = nullptr;
    void* host_dst = nullptr;
    size_t bytes = 0;
    bool owned = false;
    cudaStream_t st = nullptr;
    ~Staged() {
        if (owned && dev) cudaFreeAsync(dev, st);
    }
};

sgw_status stage_in(const void* p, size_t bytes, Staged& s, cudaStream_t st, const char* name) {
    s.bytes = bytes;
    if (is_device_ptr(p)) {
        s.dev = const_cast<void*>(p);
        return SGW_OK;
    }
    if (bytes == 0) return SGW_OK;
    SGW_CUDA(cudaMallocAsync(&s.dev, bytes, st), name);
    s.owned = true;
    s.st = st;
    s.host_src = p;
    SGW_CUDA(cudaMemcpyAsync(s.dev, p, bytes, cudaMemcpyHostToDevice, st), name);
    return SGW_OK;
}

sgw_status stage_out(void* p, size_t bytes, Staged& s, const char* name, cudaStream_t st = nullptr) {
    s.bytes = bytes;
    if (is_device_ptr(p)) {
        s.dev = p;
        return SGW_OK;
    }
    if (bytes == 0) return SGW_OK;
    SGW_CUDA(cudaMallocAsync(&s.dev, bytes, st), name);
    s.owned = true;
    s.st = st;
    s.host_dst = p;
    return SGW_OK;
}

sgw_status finish_out(Staged& s, cudaStream_t st, const char* name) {
    if (s.owned && s.host_dst && s.bytes) {
        SGW_CUDA(cudaMemcpyAsync(s.host_dst, s.dev, s.bytes, cudaMemcpyDeviceToHost, st), name);
    }
    return SGW_OK;
}

template <typename T>
sgw_status upload(T** dst, const T* src, size_t n, const char* name) {
    if (n == 0) return SGW_OK;
    SGW_CUDA(cudaMalloc((void**)dst, n * sizeof(T)), name);
    SGW_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice), name);
    return SGW_OK;
}

bool factor_235(int n, AxisPlan& ax) {
    ax.n = n;
    ax.nst = 0;
    if (n < 1) return false;
    int m = n;
    const int rads[4] = {4, 2, 3, 5};
    for (int r : rads) {
        while (m % r == 0) {
            if (ax.nst >= kMaxStages) return false;
            m /= r;
            ax.span[ax.nst] = m;
            ax.rad[ax.nst++] = r;
        }
    }
    if (m != 1) return false;
    // prime-factor parts 2^a, 3^b, 5^c when every one has a register DFT (2, 3, 4, 5, 8, 9)
    ax.npart = 0;
    int rest = n;
    bool ok = true;
    for (int p : {2, 3, 5}) {
        int q = 1;
        while (rest % p == 0) {
            rest /= p;
            q *= p;
        }
        if (q > 1) {
            ok = ok && (q == 2 || q == 3 || q == 4 || q == 5 || q == 8 || q == 9);
            if (ax.npart < 3) ax.part[ax.npart] = q;
            ++ax.npart;
        }
    }
    if (!ok || ax.npart > 3) ax.npart = 0;
    return true;
}

int mod_inverse(int a, int m) {
    for (int x = 1; x < m; ++x)
        if ((long long)a * x % m == 1) return x;
    return m == 1 ? 0 : -1;
}

// Real-space index held at each position after the inverse in-place FFT of the axis.
// Radix stages (decimation in frequency): frequency k = r_0 + R_0 (r_1 + R_1 (...)) lands
// at sum_s r_s m_s.  Prime-factor parts P_t: position p holds i_t = (p mod P_t) u_t mod P_t
// per part, u_t = (N / P_t)^-1 mod P_t, i.e. frequency sum_t (N / P_t) u_t i_t mod N.
std::vector<int> real_order(const AxisPlan& ax) {
    std::vector<int> k_at(ax.n);
    if (ax.npart > 0) {
        for (int p = 0; p < ax.n; ++p) {
            long long f = 0;
            for (int t = 0; t < ax.npart; ++t) {
                const int P = ax.part[t], c = ax.n / P, u = mod_inverse(c % P, P);
                const int i = (p % P) * u % P;
                f += (long long)c * u * i;
            }
            k_at[p] = (int)(f % ax.n);
        }
        return k_at;
    }
    for (int k = 0; k < ax.n; ++k) {
        int rest = k, pos = 0;
        for (int s = 0; s < ax.nst; ++s) {
            pos += (rest % ax.rad[s]) * ax.span[s];
            rest /= ax.rad[s];
        }
        k_at[pos] = k;
    }
    return k_at;
}

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

void free_system(sgw_system* s) {
    if (!s) return;
    cudaFree(s->d_miller);
    cudaFree(s->d_kin);
    cudaFree(s->d_stick_xy);
    cudaFree(s->d_xbase);
    cudaFree(s->d_vloc);
    cudaFree(s->d_vloc_dd);
    cudaFree(s->d_twid);
    cudaFree(s->d_beta);
    cudaFree(s->d_dkb);
    cudaFree(s->d_psi);
    cudaFree(s->d_kin_dd);
    cudaFree(s->d_beta_dd);
    cudaFree(s->d_psi_dd);
    cudaFree(s->d_lut);
    cudaFree(s->d_vloc_f);
    cudaFree(s->d_kin_f);
    cudaFree(s->d_beta_f);
    cudaFree(s->d_psi_f);
    for (int i = 0; i < 2; ++i) {
        cudaFree(s->d_g2s_s[i]);
        cudaFree(s->d_stick_loc[i]);
        cudaFree(s->d_part[i]);
    }
    cudaFree(s->d_ws);
    delete s;
}

sgw_status ensure_ws(sgw_system* s, size_t bytes) {
    if (bytes <= s->ws_bytes) return SGW_OK;
    if (s->d_ws) cudaFree(s->d_ws);
    s->d_ws = nullptr;
    s->ws_bytes = 0;
    SGW_CUDA(cudaMalloc(&s->d_ws, bytes), "workspace allocation");
    s->ws_bytes = bytes;
    return SGW_OK;
}

int max_optin_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Shifts whose per-shift state every split reserves shared memory for; solves with more
// shifts run only where the box leaves room for them.
constexpr int kPlanShifts = 256;

// A split of the sticks over csize ranks: rank r holds sticks [bs[r], bs[r+1]) and owns
// plane waves [bg[r], bg[r+1]).
struct Split {
    int csize = 0;
    int nstick_loc = 0;
    std::vector<int> bs, bg;
};

// Contiguous stick ranges (canonical order) for C ranks that minimise the largest plane-wave
// count of a rank while no rank holds more than `cap` sticks: binary search on that count,
// greedy fill.  false when no such split exists.
bool split_sticks(const std::vector<int>& cnt, int C, int cap, Split& out) {
    const int N = (int)cnt.size();
    if (cap < 1 || (long long)cap * C < N) return false;
    long long tot = 0;
    for (int c : cnt) tot += c;
    std::vector<int> b;
    auto fill = [&](long long T) -> bool {
        b.assign(1, 0);
        int j = 0;
        for (int r = 0; r < C; ++r) {
            long long g = 0;
            int n = 0;
            while (j < N && g + cnt[j] <= T && n < cap) {
                g += cnt[j];
                ++n;
                ++j;
            }
            b.push_back(j);
        }
        return j == N;
    };
    if (!fill(tot)) return false;
    long long lo = (tot + C - 1) / C, hi = tot;
    while (lo < hi) {
        const long long m = (lo + hi) / 2;
        if (fill(m)) hi = m;
        else lo = m + 1;
    }
    fill(lo);
    out.csize = C;
    out.bs = b;
    out.nstick_loc = 0;
    for (int r = 0; r < C; ++r) out.nstick_loc = std::max(out.nstick_loc, b[r + 1] - b[r]);
    return true;
}

// The split of the box for es-byte complex values: the cluster size (1 .. kMaxCluster) whose
// Lanczos kernel keeps the most SMs busy (resident clusters x size, as the occupancy
// calculator reports for this GPU), the smaller size on ties; csize 0 when none fits.
Split choose_split(const sgw_system* s, const Plan& base, int es) {
    const int budget = max_optin_smem() - 1024;   // static shared memory of the kernels
    Split best;
    long long best_score = -1;
    for (int C = 1; C <= kMaxCluster; ++C) {
        if (s->forced_csize > 0 && C != s->forced_csize) continue;
        Plan Q = base;
        Q.csize = C;
        Q.nstick_loc = 0;
        Q.nplanes = 1;
        const int fixed = apply_smem_layout(Q, es).end + lanczos_extra(kPlanShifts);
        const int cap = (budget - fixed) / (Q.n3p * es);
        Split sp;
        if (!split_sticks(s->stick_cnt, C, cap, sp)) continue;
        if (C == 1 || s->forced_csize > 0) return sp;   // one CTA per vector: no cluster overhead at all
        Q.nstick_loc = sp.nstick_loc;
        int owners = 0;
        if (lanczos_capacity(Q, 128, 0, es == 8 ? SGW_PREC_FP32 : SGW_PREC_DF32, &owners) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const long long score = (long long)owners * C;
        if (score > best_score) {
            best_score = score;
            best = sp;
        }
    }
    return best;
}

// (Re)builds both splits of the box for the current occupied states and uploads their tables.
sgw_status build_plans(sgw_system* s) {
    const int npw = s->npw, n3 = s->dims[2], n3p = s->plan.n3p;
    Plan* plans[2] = {&s->plan, &s->plan8};
    for (int c = 0; c < 2; ++c) {
        const int es = c == 0 ? 16 : 8;
        const Split sp = choose_split(s, *plans[c], es);
        plans[c]->csize = sp.csize;
        cudaFree(s->d_g2s_s[c]);
        cudaFree(s->d_stick_loc[c]);
        cudaFree(s->d_part[c]);
        s->d_g2s_s[c] = s->d_stick_loc[c] = s->d_part[c] = nullptr;
        if (sp.csize == 0) {
            if (c == 0) {
                char buf[200];
                std::snprintf(buf, sizeof buf,
                              "the pruned FFT box (%d sticks x %d) does not fit the shared memory of a cluster of %d "
                              "CTAs",
                              s->nstick, n3, kMaxCluster);
                return fail(SGW_EUNSUPPORTED, buf);
            }
            continue;   // FP32 solves of this system report SGW_EUNSUPPORTED
        }
        std::vector<int> g2s(npw), loc(s->nstick), part(2 * (kMaxCluster + 1), 0);
        std::vector<int> owner(s->nstick);
        for (int r = 0; r < sp.csize; ++r)
            for (int st = sp.bs[r]; st < sp.bs[r + 1]; ++st) {
                owner[st] = r;
                loc[st] = (r << 16) | (st - sp.bs[r]);
            }
        for (int g = 0; g < npw; ++g) {
            const int st = s->stick_of[g];
            g2s[g] = (st - sp.bs[owner[st]]) * n3p + s->map[g] % n3;
        }
        for (int r = 0; r <= kMaxCluster; ++r) {
            const int b = sp.bs[std::min(r, sp.csize)];
            part[r] = b < s->nstick ? s->stick_g0[b] : npw;
            part[kMaxCluster + 1 + r] = b;
        }
        sgw_status rs;
        if ((rs = upload(&s->d_g2s_s[c], g2s.data(), g2s.size(), "upload g2s")) != SGW_OK ||
            (rs = upload(&s->d_stick_loc[c], loc.data(), loc.size(), "upload stick owners")) != SGW_OK ||
            (rs = upload(&s->d_part[c], part.data(), part.size(), "upload split")) != SGW_OK)
            return rs;
        plans[c]->g2s = s->d_g2s_s[c];
        plans[c]->stick_loc = s->d_stick_loc[c];
        plans[c]->part = s->d_part[c];
        plans[c]->nstick_loc = sp.nstick_loc;
    }
    return SGW_OK;
}

}  // namespace

namespace sgw {

sgw_status noalloc_fail(sgw_status s, const char* msg) { return fail(s, msg); }

sgw_status noalloc_plan(const sgw_system* sys, const Plan** plan, int* dev) {
    g_err.clear();
    if (!sys) return fail(SGW_EINVAL, "NULL system");
    *plan = &sys->plan;
    *dev = sys->dev;
    return SGW_OK;
}

}  // namespace sgw

extern "C" {

const char* sgw_last_error(void) { return g_err.c_str(); }

sgw_status sgw_create_system(const sgw_cell* cell, double ecut_ry, const double k_frac[3], const int fft_dims[3],
                             const double* vloc_r, const sgw_kb* kb, sgw_system** out) {
    g_err.clear();
    if (!out) return fail(SGW_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cell || !k_frac || !fft_dims || !vloc_r) return fail(SGW_EINVAL, "NULL argument");
    if (!(ecut_ry > 0.0) || !std::isfinite(ecut_ry)) return fail(SGW_EINVAL, "ecut_ry must be positive and finite");
    if (!finite_all(&cell->a[0][0], 9) || !finite_all(k_frac, 3)) return fail(SGW_EINVAL, "non-finite cell or k");
    if (cell->n_atoms < 0 || (cell->n_atoms > 0 && !cell->tau)) return fail(SGW_EINVAL, "bad atom list");
    if (cell->n_atoms > 0 && !finite_all(cell->tau, 3 * (size_t)cell->n_atoms)) return fail(SGW_EINVAL, "non-finite tau");
    const int nproj = kb ? kb->n_proj : 0;
    if (nproj < 0 || nproj > kMaxProj) return fail(SGW_EUNSUPPORTED, "n_proj must be in [0, 64]");
    if (nproj > 0 && (!kb->atom || !kb->width || !kb->D)) return fail(SGW_EINVAL, "NULL projector arrays");
    for (int p = 0; p < nproj; ++p) {
        if (kb->atom[p] < 0 || kb->atom[p] >= cell->n_atoms) return fail(SGW_EINVAL, "projector atom index out of range");
        if (!(kb->width[p] > 0.0) || !std::isfinite(kb->width[p]) || !std::isfinite(kb->D[p]))
            return fail(SGW_EINVAL, "projector width must be positive, D finite");
    }
    int dev = 0;
    {
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || ndev == 0) return cuda_fail(e == cudaSuccess ? cudaErrorNoDevice : e, "no CUDA device");
        SGW_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    }
    sgw_system* s = new sgw_system();
    s->dev = dev;
    std::memcpy(s->a, cell->a, sizeof(s->a));
    const double* a0 = cell->a[0];
    const double* a1 = cell->a[1];
    const double* a2 = cell->a[2];
    double cr[3][3] = {{a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]},
                       {a2[1] * a0[2] - a2[2] * a0[1], a2[2] * a0[0] - a2[0] * a0[2], a2[0] * a0[1] - a2[1] * a0[0]},
                       {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]}};
    const double det = a0[0] * cr[0][0] + a0[1] * cr[0][1] + a0[2] * cr[0][2];
    if (!(std::fabs(det) > 1e-12)) {
        free_system(s);
        return fail(SGW_EINVAL, "degenerate lattice");
    }
    s->vol = std::fabs(det);
    const double twopi = 6.283185307179586476925286766559;
    for (int i = 0; i < 3; ++i)
        for (int x = 0; x < 3; ++x) s->b[i][x] = cr[i][x] * (twopi / det);
    std::memcpy(s->k, k_frac, sizeof(s->k));
    s->ecut = ecut_ry;
    for (int i = 0; i < 3; ++i) s->dims[i] = fft_dims[i];
    for (int i = 0; i < 3; ++i) {
        if (!factor_235(fft_dims[i], s->plan.ax[i])) {
            free_system(s);
            return fail(SGW_EINVAL, "FFT dims must be positive products of 2, 3 and 5");
        }
    }
    const size_t nbox = (size_t)fft_dims[0] * fft_dims[1] * fft_dims[2];
    if (!finite_all(vloc_r, nbox)) {
        free_system(s);
        return fail(SGW_EINVAL, "non-finite V_loc");
    }
    {
        double acc = 0.0;
        for (size_t i = 0; i < nbox; ++i) acc += vloc_r[i];
        s->v_mean = acc / (double)nbox;
    }
    double len[3];
    for (int i = 0; i < 3; ++i)
        len[i] = std::sqrt(cell->a[i][0] * cell->a[i][0] + cell->a[i][1] * cell->a[i][1] + cell->a[i][2] * cell->a[i][2]);
    // alias check: the box must hold every |G|^2 <= 4 ecut (potential band) without folding.
    {
        int mr[3] = {0, 0, 0};
        int bnd[3];
        for (int i = 0; i < 3; ++i) bnd[i] = (int)std::ceil(2.0 * std::sqrt(ecut_ry) * len[i] / twopi) + 1;
        for (int m1 = -bnd[0]; m1 <= bnd[0]; ++m1)
            for (int m2 = -bnd[1]; m2 <= bnd[1]; ++m2)
                for (int m3 = -bnd[2]; m3 <= bnd[2]; ++m3) {
                    double g2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        const double gx = m1 * s->b[0][x] + m2 * s->b[1][x] + m3 * s->b[2][x];
                        g2 += gx * gx;
                    }
                    if (g2 <= 4.0 * ecut_ry) {
                        mr[0] = std::max(mr[0], std::abs(m1));
                        mr[1] = std::max(mr[1], std::abs(m2));
                        mr[2] = std::max(mr[2], std::abs(m3));
                    }
                }
        for (int i = 0; i < 3; ++i)
            if (fft_dims[i] < 2 * mr[i] + 1) {
                free_system(s);
                char buf[160];
                std::snprintf(buf, sizeof buf, "FFT box axis %d: %d < 2*%d+1 (potential band |G|^2 <= 4 E_cut would alias)",
                              i, fft_dims[i], mr[i]);
                return fail(SGW_EALIAS, buf);
            }
    }
    // ---- G-sphere on the device
    SphereArgs sa;
    std::memcpy(sa.b, s->b, sizeof(sa.b));
    std::memcpy(sa.k, k_frac, sizeof(sa.k));
    sa.ecut = ecut_ry;
    long long cand = 1;
    for (int i = 0; i < 3; ++i) {
        sa.M[i] = (int)std::ceil(std::sqrt(ecut_ry) * len[i] / twopi + std::fabs(k_frac[i])) + 1;
        cand *= 2 * sa.M[i] + 1;
    }
    if (cand > 50000000LL) {
        free_system(s);
        return fail(SGW_EUNSUPPORTED, "Miller box too large");
    }
    sa.cap = (int)cand;
    int *d_mil = nullptr, *d_cnt = nullptr;
    double* d_kin = nullptr;
    auto cleanup_tmp = [&]() {
        cudaFree(d_mil);
        cudaFree(d_cnt);
        cudaFree(d_kin);
    };
    cudaError_t e = cudaMalloc(&d_mil, sizeof(int) * 3 * cand);
    if (e == cudaSuccess) e = cudaMalloc(&d_kin, sizeof(double) * cand);
    if (e == cudaSuccess) e = cudaMalloc(&d_cnt, sizeof(int));
    if (e == cudaSuccess) e = launch_sphere(sa, d_mil, d_kin, d_cnt, 0);
    int npw = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&npw, d_cnt, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cleanup_tmp();
        free_system(s);
        return cuda_fail(e, "G-sphere kernel");
    }
    if (npw < 1) {
        cleanup_tmp();
        free_system(s);
        return fail(SGW_EINVAL, "empty plane-wave sphere");
    }
    s->npw = npw;
    s->miller.resize(3 * (size_t)npw);
    s->kin.resize(npw);
    e = cudaMemcpy(s->miller.data(), d_mil, sizeof(int) * 3 * npw, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(s->kin.data(), d_kin, sizeof(double) * npw, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_miller, sizeof(int) * 3 * npw);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_miller, d_mil, sizeof(int) * 3 * npw, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_kin, sizeof(double) * npw);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_kin, d_kin, sizeof(double) * npw, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_kin_dd, sizeof(float2) * npw);
    if (e == cudaSuccess) e = launch_to_dd(s->d_kin, npw, s->d_kin_dd, 0);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_kin_f, sizeof(float) * npw);
    if (e == cudaSuccess) e = launch_to_f32(s->d_kin, npw, s->d_kin_f, 0);
    cleanup_tmp();
    if (e != cudaSuccess) {
        free_system(s);
        return cuda_fail(e, "G-sphere copy");
    }
    // ---- box map (device) and stick tables (host, integer bookkeeping)
    {
        int* d_map = nullptr;
        e = cudaMalloc(&d_map, sizeof(int) * npw);
        if (e == cudaSuccess) e = launch_boxmap(s->d_miller, npw, fft_dims, d_map, 0);
        s->map.resize(npw);
        if (e == cudaSuccess) e = cudaMemcpy(s->map.data(), d_map, sizeof(int) * npw, cudaMemcpyDeviceToHost);
        cudaFree(d_map);
        if (e != cudaSuccess) {
            free_system(s);
            return cuda_fail(e, "box map kernel");
        }
    }
    const int n1 = fft_dims[0], n2 = fft_dims[1], n3 = fft_dims[2];
    // sticks (z-columns holding plane waves) in canonical order: the plane waves of one stick,
    // fixed (m1, m2), are consecutive in the Miller-lexicographic order, so each stick is a
    // range [stick_g0, stick_g0 + stick_cnt) of the coefficient arrays
    const int n2p = n2 | 1;   // odd row stride: strided (x-direction) FFT lines spread over all banks
    std::vector<int> xs_used(n1, 0);
    s->stick_of.resize(npw);
    for (int g = 0; g < npw; ++g) {
        const int xy = s->map[g] / n3;
        if (g == 0 || xy != s->map[g - 1] / n3) {
            s->stick_g0.push_back(g);
            s->stick_cnt.push_back(0);
            s->stick_xy.push_back((xy / n2) * n2p + xy % n2);
        }
        ++s->stick_cnt.back();
        s->stick_of[g] = (int)s->stick_g0.size() - 1;
        xs_used[xy / n2] = 1;
    }
    const int n3p = n3 | 1;   // odd stick stride
    std::vector<int> xbase;
    for (int x = 0; x < n1; ++x)
        if (xs_used[x]) xbase.push_back(x * n2p);
    s->nstick = (int)s->stick_xy.size();
    s->nxcol = (int)xbase.size();
    // potential, one contiguous (padded) plane per z: [z][x][y < n2p], every axis in the
    // order in which the inverse FFTs leave real space
    const size_t nboxp = (size_t)n1 * n2p * n3;
    std::vector<double> vz(nboxp, 0.0);
    const std::vector<int> ox = real_order(s->plan.ax[0]), oy = real_order(s->plan.ax[1]), oz = real_order(s->plan.ax[2]);
    for (int px = 0; px < n1; ++px)
        for (int py = 0; py < n2; ++py)
            for (int pz = 0; pz < n3; ++pz)
                vz[((size_t)pz * n1 + px) * n2p + py] = vloc_r[((size_t)ox[px] * n2 + oy[py]) * n3 + oz[pz]];
    std::vector<float2> vzdd(nboxp);
    std::vector<float> vzf(nboxp);
    for (size_t i = 0; i < nboxp; ++i) {
        const float h = (float)vz[i];
        vzdd[i] = make_float2(h, (float)(vz[i] - (double)h));
        vzf[i] = h;
    }
    sgw_status rs;
    if ((rs = upload(&s->d_vloc_dd, vzdd.data(), vzdd.size(), "upload V_loc")) != SGW_OK ||
        (rs = upload(&s->d_vloc_f, vzf.data(), vzf.size(), "upload V_loc")) != SGW_OK) {
        free_system(s);
        return rs;
    }
    if ((rs = upload(&s->d_stick_xy, s->stick_xy.data(), s->stick_xy.size(), "upload sticks")) != SGW_OK ||
        (rs = upload(&s->d_xbase, xbase.data(), xbase.size(), "upload xbase")) != SGW_OK ||
        (rs = upload(&s->d_vloc, vz.data(), vz.size(), "upload V_loc")) != SGW_OK) {
        free_system(s);
        return rs;
    }
    e = cudaMalloc(&s->d_twid, sizeof(double2) * (n1 + n2 + n3));
    if (e == cudaSuccess) e = launch_twiddles(fft_dims, s->d_twid, 0);
    if (e != cudaSuccess) {
        free_system(s);
        return cuda_fail(e, "twiddles");
    }
    // ---- KB projectors
    s->nproj = nproj;
    if (nproj > 0) {
        BetaArgs ba;
        std::memcpy(ba.b, s->b, sizeof(ba.b));
        std::memcpy(ba.k, k_frac, sizeof(ba.k));
        ba.inv_sqrt_vol = 1.0 / std::sqrt(s->vol);
        std::vector<double> d(nproj);
        for (int p = 0; p < nproj; ++p) {
            ba.width[p] = kb->width[p];
            for (int x = 0; x < 3; ++x) ba.tau[p][x] = cell->tau[3 * kb->atom[p] + x];
            d[p] = kb->D[p];
        }
        e = cudaMalloc(&s->d_beta, sizeof(double2) * (size_t)nproj * npw);
        if (e == cudaSuccess) e = launch_beta(ba, nproj, s->d_miller, npw, s->d_beta, 0);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_beta_dd, sizeof(float4) * (size_t)nproj * npw);
        if (e == cudaSuccess)
            e = launch_to_dd(reinterpret_cast<const double*>(s->d_beta), 2 * (size_t)nproj * npw,
                             reinterpret_cast<float2*>(s->d_beta_dd), 0);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_beta_f, sizeof(float2) * (size_t)nproj * npw);
        if (e == cudaSuccess)
            e = launch_to_f32(reinterpret_cast<const double*>(s->d_beta), 2 * (size_t)nproj * npw,
                              reinterpret_cast<float*>(s->d_beta_f), 0);
        if (e != cudaSuccess) {
            free_system(s);
            return cuda_fail(e, "projector kernel");
        }
        if ((rs = upload(&s->d_dkb, d.data(), d.size(), "upload D")) != SGW_OK) {
            free_system(s);
            return rs;
        }
    }
    // ---- Miller lookup table for Eq. 8 gathers into this basis's coefficients
    {
        int hi[3];
        for (int x = 0; x < 3; ++x) {
            s->lo[x] = 1 << 30;
            hi[x] = -(1 << 30);
        }
        for (int g = 0; g < npw; ++g)
            for (int x = 0; x < 3; ++x) {
                s->lo[x] = std::min(s->lo[x], s->miller[3 * g + x]);
                hi[x] = std::max(hi[x], s->miller[3 * g + x]);
            }
        for (int x = 0; x < 3; ++x) s->ext[x] = hi[x] - s->lo[x] + 1;
        std::vector<int> lut((size_t)s->ext[0] * s->ext[1] * s->ext[2], -1);
        for (int g = 0; g < npw; ++g) {
            const int i0 = s->miller[3 * g] - s->lo[0], i1 = s->miller[3 * g + 1] - s->lo[1],
                      i2 = s->miller[3 * g + 2] - s->lo[2];
            lut[((size_t)i0 * s->ext[1] + i1) * s->ext[2] + i2] = g;
        }
        if ((rs = upload(&s->d_lut, lut.data(), lut.size(), "upload lookup")) != SGW_OK) {
            free_system(s);
            return rs;
        }
    }
    // ---- plan
    Plan& P = s->plan;
    P.n1 = n1;
    P.n2 = n2;
    P.n3 = n3;
    P.n2p = n2p;
    P.n3p = n3p;
    P.nplanes = 1;
    P.npw = npw;
    P.nstick = s->nstick;
    P.nxcol = s->nxcol;
    P.g2s = nullptr;   // per split (build_plans)
    P.stick_xy = s->d_stick_xy;
    P.xbase = s->d_xbase;
    P.vloc = s->d_vloc;
    P.vloc_dd = s->d_vloc_dd;
    P.kin = s->d_kin;
    P.kin_dd = s->d_kin_dd;
    P.twid = s->d_twid;
    P.nproj = nproj;
    P.beta = s->d_beta;
    P.beta_dd = s->d_beta_dd;
    P.dkb = s->d_dkb;
    P.nocc = 0;
    P.psi = nullptr;
    P.psi_dd = nullptr;
    P.inv_nbox = 1.0 / (double)nbox;
    P.vloc_f = s->d_vloc_f;
    P.kin_f = s->d_kin_f;
    P.beta_f = s->d_beta_f;
    P.psi_f = nullptr;
    P.csize = 1;
    P.nstick_loc = s->nstick;
    P.part = nullptr;
    P.stick_loc = nullptr;
    s->plan8 = P;
    if ((rs = build_plans(s)) != SGW_OK) {
        free_system(s);
        return rs;
    }
    SGW_CUDA(cudaDeviceSynchronize(), "create_system");
    *out = s;
    return SGW_OK;
}

sgw_status sgw_get_gvectors(const sgw_system* s, int* n_pw, int* miller, double* kin) {
    if (!s) return fail(SGW_EINVAL, "NULL system");
    if (n_pw) *n_pw = s->npw;
    if (miller) std::memcpy(miller, s->miller.data(), sizeof(int) * 3 * s->npw);
    if (kin) std::memcpy(kin, s->kin.data(), sizeof(double) * s->npw);
    return SGW_OK;
}

sgw_status sgw_get_box_map(const sgw_system* s, int* map) {
    if (!s || !map) return fail(SGW_EINVAL, "NULL argument");
    std::memcpy(map, s->map.data(), sizeof(int) * s->npw);
    return SGW_OK;
}

sgw_status sgw_set_split(sgw_system* s, int csize) {
    g_err.clear();
    if (!s) return fail(SGW_EINVAL, "NULL system");
    if (csize < 0 || csize > kMaxCluster) return fail(SGW_EINVAL, "csize must be in [0, 16]");
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    SGW_CUDA(cudaDeviceSynchronize(), "set_split");   // the tables may be in use by queued work
    const int prev = s->forced_csize;
    s->forced_csize = csize;
    sgw_status r = build_plans(s);
    if (r != SGW_OK) {
        const std::string msg = g_err;
        s->forced_csize = prev;
        build_plans(s);
        return fail(r, msg);
    }
    if (csize > 0 && s->plan.csize != csize) {
        s->forced_csize = prev;
        build_plans(s);
        return fail(SGW_EUNSUPPORTED, "the box does not split over that many CTAs");
    }
    return SGW_OK;
}

sgw_status sgw_get_split(const sgw_system* s, int* csize, int* csize_fp32) {
    if (!s) return fail(SGW_EINVAL, "NULL system");
    if (csize) *csize = s->plan.csize;
    if (csize_fp32) *csize_fp32 = s->plan8.csize;
    return SGW_OK;
}

sgw_status sgw_solve_capacity(const sgw_system* s, int nomega, int precision, int threads, int* owners) {
    g_err.clear();
    if (!s || !owners) return fail(SGW_EINVAL, "NULL argument");
    if (nomega < 1 || nomega > kMaxShifts) return fail(SGW_EINVAL, "nomega must be in [1, 512]");
    if (precision != SGW_PREC_FP64 && precision != SGW_PREC_DF32 && precision != SGW_PREC_FP32)
        return fail(SGW_EINVAL, "unknown precision");
    const Plan& plan = precision == SGW_PREC_FP32 ? s->plan8 : s->plan;
    if (plan.csize == 0) return fail(SGW_EUNSUPPORTED, "the FFT box does not fit on chip in FP32");
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    int n = 0;
    SGW_CUDA(lanczos_capacity(plan, nomega, threads, precision, &n), "solver occupancy");
    *owners = n;
    return SGW_OK;
}

sgw_status sgw_set_occupied(sgw_system* s, int n_occ, const void* psi_v, const double* eps_v) {
    g_err.clear();
    if (!s) return fail(SGW_EINVAL, "NULL system");
    if (n_occ < 0 || n_occ > 4096) return fail(SGW_EINVAL, "n_occ out of range");
    if (n_occ > 0 && (!psi_v || !eps_v)) return fail(SGW_EINVAL, "NULL psi_v or eps_v");
    if (n_occ > 0 && !finite_all(eps_v, n_occ)) return fail(SGW_EINVAL, "non-finite eps_v");
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_set_occupied");
    const size_t bytes = sizeof(double2) * (size_t)n_occ * s->npw;
    double2* d_new = nullptr;
    if (n_occ > 0) {
        SGW_CUDA(cudaMalloc(&d_new, bytes), "psi_v allocation");
        cudaError_t e = cudaMemcpy(d_new, psi_v, bytes, cudaMemcpyDefault);
        if (e != cudaSuccess) {
            cudaFree(d_new);
            return cuda_fail(e, "psi_v copy");
        }
        // orthonormality: max |psi^H psi - I| <= 1e-10 (also catches NaN/Inf)
        double2* d_S = nullptr;
        std::vector<double2> S((size_t)n_occ * n_occ);
        e = cudaMalloc(&d_S, sizeof(double2) * S.size());
        if (e == cudaSuccess) e = launch_gram(d_new, n_occ, s->npw, d_S, 0);
        if (e == cudaSuccess) e = cudaMemcpy(S.data(), d_S, sizeof(double2) * S.size(), cudaMemcpyDeviceToHost);
        cudaFree(d_S);
        if (e != cudaSuccess) {
            cudaFree(d_new);
            return cuda_fail(e, "overlap kernel");
        }
        double worst = 0.0;
        for (int v = 0; v < n_occ; ++v)
            for (int w = 0; w < n_occ; ++w) {
                const double2 q = S[(size_t)v * n_occ + w];
                const double dr = q.x - (v == w ? 1.0 : 0.0);
                const double d = std::sqrt(dr * dr + q.y * q.y);
                if (!(d <= worst)) worst = d;   // NaN-propagating max
            }
        if (!(worst <= 1e-10)) {
            cudaFree(d_new);
            char buf[120];
            std::snprintf(buf, sizeof buf, "psi_v not orthonormal: max |psi^H psi - I| = %.3e > 1e-10", worst);
            return fail(SGW_EINVAL, buf);
        }
    }
    float4* d_new_dd = nullptr;
    float2* d_new_f = nullptr;
    if (n_occ > 0) {
        cudaError_t e = cudaMalloc(&d_new_dd, sizeof(float4) * (size_t)n_occ * s->npw);
        if (e == cudaSuccess)
            e = launch_to_dd(reinterpret_cast<const double*>(d_new), 2 * (size_t)n_occ * s->npw,
                             reinterpret_cast<float2*>(d_new_dd), 0);
        if (e == cudaSuccess) e = cudaMalloc(&d_new_f, sizeof(float2) * (size_t)n_occ * s->npw);
        if (e == cudaSuccess)
            e = launch_to_f32(reinterpret_cast<const double*>(d_new), 2 * (size_t)n_occ * s->npw,
                              reinterpret_cast<float*>(d_new_f), 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(d_new);
            cudaFree(d_new_dd);
            cudaFree(d_new_f);
            return cuda_fail(e, "psi_v float-float copy");
        }
    }
    cudaFree(s->d_psi);
    cudaFree(s->d_psi_dd);
    cudaFree(s->d_psi_f);
    s->d_psi = d_new;
    s->d_psi_dd = d_new_dd;
    s->d_psi_f = d_new_f;
    s->nocc = n_occ;
    s->eps.assign(eps_v, eps_v + n_occ);
    for (Plan* p : {&s->plan, &s->plan8}) {
        p->nocc = n_occ;
        p->psi = d_new;
        p->psi_dd = d_new_dd;
        p->psi_f = d_new_f;
    }
    // the coefficient slots grow with n_occ: the split of the box is chosen again
    return build_plans(s);
}

sgw_status sgw_make_rhs(const sgw_system* kq, const sgw_system* k, int n_v, const void* psi_k, int n_pert,
                        const int* gp_miller, void* rhs, void* stream) {
    g_err.clear();
    if (!kq || !k || !rhs || (n_v > 0 && !psi_k) || (n_pert > 0 && !gp_miller))
        return fail(SGW_EINVAL, "NULL argument");
    if (n_v < 0 || n_pert < 0) return fail(SGW_EINVAL, "negative size");
    if (n_v == 0 || n_pert == 0) return SGW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Staged in, out;
    sgw_status r;
    if ((r = stage_in(psi_k, sizeof(double2) * (size_t)n_v * k->npw, in, st, "psi_k")) != SGW_OK) return r;
    if ((r = stage_out(rhs, sizeof(double2) * (size_t)n_v * n_pert * kq->npw, out, "rhs", st)) != SGW_OK) return r;
    int* d_gp = nullptr;
    SGW_CUDA(cudaMalloc(&d_gp, sizeof(int) * 3 * n_pert), "gp allocation");
    cudaError_t e = cudaMemcpyAsync(d_gp, gp_miller, sizeof(int) * 3 * n_pert, cudaMemcpyHostToDevice, st);
    RhsArgs ra;
    for (int x = 0; x < 3; ++x) {
        ra.lo[x] = k->lo[x];
        ra.ext[x] = k->ext[x];
    }
    if (e == cudaSuccess)
        e = launch_rhs(ra, kq->d_miller, kq->npw, k->d_lut, (const double2*)in.dev, k->npw, d_gp, n_v, n_pert,
                       (double2*)out.dev, st);
    if (e == cudaSuccess && (r = finish_out(out, st, "rhs copy")) != SGW_OK) {
        cudaFree(d_gp);
        return r;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_gp);
    if (e != cudaSuccess) return cuda_fail(e, "rhs kernel");
    return SGW_OK;
}

static sgw_status apply_common(sgw_system* s, int nvec, const void* x, const double* z, void* y, void* stream,
                               int project, int precision) {
    g_err.clear();
    if (!s || !x || !y) return fail(SGW_EINVAL, "NULL argument");
    if (nvec < 0) return fail(SGW_EINVAL, "negative nvec");
    if (nvec == 0) return SGW_OK;
    if (project && s->nocc == 0) return fail(SGW_ESTATE, "sgw_set_occupied has not been called");
    if (project && (!z || !finite_all(z, 2 * (size_t)nvec))) return fail(SGW_EINVAL, "bad shifts");
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_apply_h");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vb = sizeof(double2) * (size_t)nvec * s->npw;
    Staged in, out;
    sgw_status r;
    if ((r = stage_in(x, vb, in, st, "x")) != SGW_OK) return r;
    if ((r = stage_out(y, vb, out, "y", st)) != SGW_OK) return r;
    if (precision != SGW_PREC_FP64 && precision != SGW_PREC_DF32 && precision != SGW_PREC_FP32)
        return fail(SGW_EINVAL, "unknown precision");
    const Plan& plan = precision == SGW_PREC_FP32 ? s->plan8 : s->plan;
    if (plan.csize == 0) return fail(SGW_EUNSUPPORTED, "the FFT box does not fit on chip in this precision");
    int owners = 0;
    SGW_CUDA(apply_owners(plan, precision, &owners), "apply occupancy");
    owners = std::min(owners, nvec);
    const size_t scratch = 2 * sizeof(double2) * (size_t)owners * s->npw;
    const size_t zb = project ? sizeof(double2) * nvec : 0;
    if ((r = ensure_ws(s, scratch + zb + 256)) != SGW_OK) return r;
    double2* d_scr = (double2*)s->d_ws;
    double2* d_z = (double2*)((char*)s->d_ws + ((scratch + 255) / 256) * 256);
    if (project) SGW_CUDA(cudaMemcpyAsync(d_z, z, zb, cudaMemcpyHostToDevice, st), "z copy");
    SGW_CUDA(launch_apply(plan, nvec, (const double2*)in.dev, (double2*)out.dev, d_z, project, d_scr, owners,
                          precision, st),
             "apply kernel");
    if ((r = finish_out(out, st, "y copy")) != SGW_OK) return r;
    SGW_CUDA(cudaStreamSynchronize(st), "apply");
    return SGW_OK;
}

sgw_status sgw_apply_h(sgw_system* s, int nvec, const void* x, void* y, int precision, void* stream) {
    return apply_common(s, nvec, x, nullptr, y, stream, 0, precision);
}

sgw_status sgw_apply_shifted(sgw_system* s, int nvec, const void* x, const double* z, void* y, int precision,
                             void* stream) {
    return apply_common(s, nvec, x, z, y, stream, 1, precision);
}

namespace {

// Bump allocator over the system's workspace.
struct Carve {
    size_t off = 0;
    size_t take(size_t b) {
        const size_t o = off;
        off += (b + 255) / 256 * 256;
        return o;
    }
};

}  // namespace

// The multishift solve of every (rhs, shift) pair with its FP64 true-residual check and
// per-shift corrections: z_rj = e_ref[r] + omega[j] + i Im z_j, Im z_j = eta_s[j] when
// eta_s (host) is given, else eta.  rhs_d and X are device buffers; `project` selects the
// operator (P_c H P_c with the system's occupied states, else H itself).  A pair is
// converged when rel_res <= tol and its certificate <= cert_tol.  Returns SGW_ENOCONV, with X
// and the report written, when a pair misses either.
// The multishift pass of a packed multi-system launch (sgw_solve_batched): device per-pair
// Krylov steps, recursive estimates and statistics, and the launch's kernel time.
struct PassDone {
    const int* mv;
    const double* est;
    const int* st;
    double kernel_ms;
    int launches;
};

static sgw_status multishift(sgw_system* s, bool project, int nrhs, const double2* rhs_d, const double* e_ref,
                             int nomega, const double* omega, const double* eta_s, double eta, double tol,
                             const sgw_solve_opts* opts, double2* X, sgw_report* report, cudaStream_t st,
                             const PassDone* done = nullptr) {
    const int method = opts ? opts->method : SGW_METHOD_LANCZOS;
    const int precision = opts ? opts->precision : SGW_PREC_FP64;
    const int threads = opts ? opts->threads : 0;
    const int precond = opts ? opts->precond : SGW_PRECOND_NONE;
    const sgw_mlp* mlp = opts ? opts->mlp : nullptr;
    const double cert_tol = !opts || opts->cert_tol == 0.0 ? 1e-8 : opts->cert_tol;   // < 0: not checked
    const bool use_cert = cert_tol > 0.0;
    if (precision != SGW_PREC_FP64 && precision != SGW_PREC_DF32 && precision != SGW_PREC_FP32)
        return fail(SGW_EINVAL, "unknown precision");
    if (method != SGW_METHOD_LANCZOS && method != SGW_METHOD_BICGSTAB) return fail(SGW_EINVAL, "unknown method");
    if (precision == SGW_PREC_FP32 && method != SGW_METHOD_LANCZOS)
        return fail(SGW_EUNSUPPORTED, "the FP32 inner solve is the Lanczos method");
    if (eta_s && method != SGW_METHOD_LANCZOS)
        return fail(SGW_EUNSUPPORTED, "shifts with different imaginary parts need the Lanczos method");
    if (precond != SGW_PRECOND_NONE && precond != SGW_PRECOND_PLAIN && precond != SGW_PRECOND_LEARNED)
        return fail(SGW_EINVAL, "precond must be SGW_PRECOND_NONE, _PLAIN or _LEARNED");
    if (precond == SGW_PRECOND_LEARNED && !mlp) return fail(SGW_EINVAL, "the learned preconditioner needs opts.mlp");
    if (precond != SGW_PRECOND_NONE && !project)
        return fail(SGW_EUNSUPPORTED, "preconditioned corrections solve the projected Sternheimer operator only");
    if (!std::isfinite(cert_tol)) return fail(SGW_EINVAL, "non-finite cert_tol");
    const int ell = opts && opts->ell ? opts->ell : 4;
    if (ell < 1 || ell > kMaxEll) return fail(SGW_EINVAL, "ell must be 1, 2, 3 or 4");
    int seed = opts ? opts->seed_index : -1;
    if (seed < 0) {
        seed = 0;
        for (int j = 1; j < nomega; ++j)
            if (omega[j] > omega[seed]) seed = j;
    }
    if (seed >= nomega) return fail(SGW_EINVAL, "seed_index out of range");
    const bool lanczos = method == SGW_METHOD_LANCZOS;
    const bool have_x0 = opts && opts->x0 && !done;
    // plans: the pass in its precision; the FP64 check and the corrections in the 16-byte split
    // (corrections of an FP32 pass run in float-float: FP64 iterative refinement)
    Plan plan = precision == SGW_PREC_FP32 ? s->plan8 : s->plan;
    Plan plan16 = s->plan;
    if (plan.csize == 0) return fail(SGW_EUNSUPPORTED, "the FFT box does not fit on chip in FP32");
    if (!project) {
        for (Plan* p : {&plan, &plan16}) {
            p->nocc = 0;
            p->psi = nullptr;
            p->psi_dd = nullptr;
            p->psi_f = nullptr;
        }
    }
    const int res_prec = precision == SGW_PREC_FP64 ? SGW_PREC_FP64 : SGW_PREC_DF32;
    const int corr_prec = precision == SGW_PREC_FP32 ? SGW_PREC_DF32 : precision;
    // Lanczos keeps its basis: the default budget of 16384 steps (further capped by free device
    // memory) bounds its memory; the 64-atom cell's highest frequencies need some 14 000 steps
    const int max_mv = opts && opts->max_matvec > 0 ? opts->max_matvec : (lanczos ? 16384 : 40000);
    const int max_refine = !opts || opts->max_refine == 0 ? 3 : std::max(0, opts->max_refine);
    const int plain_budget = opts && opts->plain_budget > 0 ? opts->plain_budget : 0;
    if (lanczos && !have_x0 && !done && lanczos_smem_bytes(plan, nomega, precision) > max_optin_smem())
        return fail(SGW_EUNSUPPORTED, "too many frequencies for the on-chip shift state");
    if (!lanczos && solve_smem_bytes(plan, nomega) > max_optin_smem())
        return fail(SGW_EUNSUPPORTED, "too many frequencies for the on-chip shift state");
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    const size_t np = (size_t)nrhs * nomega;
    if (np > (size_t)INT_MAX) return fail(SGW_EUNSUPPORTED, "nrhs * nomega above INT_MAX");
    sgw_status r;
    const int chunk = (int)std::min<size_t>(np, 4096);
    int own = 0, own1 = 0, own_r = 0, grid_b = 0;
    if (lanczos) {
        SGW_CUDA(lanczos_capacity(plan, nomega, threads, precision, &own), "solver occupancy");
        own = std::min(own, nrhs);
    } else {
        SGW_CUDA(solve_grid(plan, nomega, nrhs, &own), "solver occupancy");
    }
    SGW_CUDA(lanczos_capacity(plan16, 1, threads, corr_prec, &own1), "solver occupancy");
    own1 = std::min(own1, chunk);
    // corrections: single-shift Lanczos, or BiCGstab(ell) when the method is BiCGstab or a
    // preconditioner is asked for
    const bool bicg_corr = !lanczos || precond != SGW_PRECOND_NONE;
    if (bicg_corr) SGW_CUDA(solve_grid(plan16, 1, chunk, &grid_b), "solver occupancy");
    SGW_CUDA(residual_owners(plan16, res_prec, &own_r), "residual occupancy");
    own_r = (int)std::min<size_t>(own_r, np);
    // Krylov workspace of one launch (reused by the correction solves); the basis per owner
    int maxk = max_mv;
    const size_t eb = (size_t)prec_bytes(precision) * s->npw;   // basis vector of the pass
    // basis [owners][mk + 1][n_pw], then alpha / beta [ctas][2][mk + 1], then the y and l
    // coefficients [ctas][2][mk][ns]; each part starts on a 256-byte boundary
    auto al256 = [](size_t b) { return (b + 255) / 256 * 256; };
    auto lanczos_bytes = [&](int owners, int ctas, int ns, int mk, size_t vbytes) -> size_t {
        return al256((size_t)owners * (size_t)(mk + 1) * vbytes) + al256((size_t)ctas * 2 * (size_t)(mk + 1) * 8) +
               (size_t)ctas * 2 * (size_t)mk * ns * 16 + 4096;
    };
    // The Krylov workspaces are allocated for the duration of the call only (stream-ordered), so
    // systems solved one after another or side by side do not keep each other's bases.  The pass
    // basis is capped by half the free device memory; a correction solve (one shift, a fraction
    // of a digit or a few digits to gain) gets at most 4096 steps and one owner per pair.
    size_t free_b = 0, total_b = 0;
    SGW_CUDA(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    const size_t budget = std::min<size_t>(free_b / 2, (size_t)96 << 30);
    const bool pass = !have_x0 && !done;
    if (lanczos && pass) {
        const size_t per_k = (size_t)own * (eb + 16 * plan.csize) + (size_t)own * plan.csize * 32 * (size_t)nomega;
        const size_t cap = budget / std::max<size_t>(per_k, 1);
        if (cap < 8) return fail(SGW_ENOMEM, "not enough device memory for a Lanczos basis");
        maxk = (int)std::min<size_t>((size_t)max_mv, cap - 2);
    }
    int maxk_c = std::min(max_mv, 4096);
    {
        const size_t per_k = (size_t)own1 * (vb + 16 * plan16.csize + 32 * plan16.csize);
        const size_t cap = budget / std::max<size_t>(per_k, 1);
        if (cap < 8) return fail(SGW_ENOMEM, "not enough device memory for a correction basis");
        maxk_c = (int)std::min<size_t>((size_t)maxk_c, cap - 2);
    }
    size_t pass_bytes = 0;
    if (pass) {
        pass_bytes = lanczos ? lanczos_bytes(own, own * plan.csize, nomega, maxk, eb)
                             : (size_t)own * (vb * (2 * ell + 3) + vb * (size_t)nomega) + 4096;
    }
    auto corr_bytes = [&](int nc) -> size_t {
        if (!bicg_corr) {
            const int o = std::min(own1, nc);
            return lanczos_bytes(o, o * plan16.csize, 1, maxk_c, vb);
        }
        return (size_t)std::min(grid_b, nc) * vb * (2 * ell + 6) + 4096;   // BiCGstab seeds, directions, scratch
    };
    Staged passbuf;
    if (pass_bytes) {
        SGW_CUDA(cudaMallocAsync(&passbuf.dev, pass_bytes, st), "Krylov workspace");
        passbuf.owned = true;
        passbuf.st = st;
    }
    char* pw = (char*)passbuf.dev;
    Carve c;
    const size_t o_eref = c.take(sizeof(double) * nrhs);
    const size_t o_om = c.take(sizeof(double) * nomega);
    const size_t o_sig = c.take(sizeof(double) * nomega);
    const size_t o_cnt = c.take(sizeof(int));
    const size_t o_mv = c.take(sizeof(int) * np);
    const size_t o_est = c.take(sizeof(double) * np);
    const size_t o_st = c.take(sizeof(int) * np);
    const size_t o_rscr = c.take(2 * vb * own_r);
    const size_t o_rel = c.take(sizeof(double) * np);
    const size_t o_bvec = project ? c.take(vb * nrhs) : 0;
    const size_t o_cert = c.take(sizeof(double) * np);
    const size_t o_list = c.take(sizeof(int) * chunk);
    const size_t o_rvec = c.take(vb * chunk);
    const size_t o_dbuf = c.take(vb * chunk);
    const size_t o_eref1 = c.take(sizeof(double) * chunk);
    const size_t o_eta1 = c.take(sizeof(double) * chunk);
    const size_t o_etas = c.take(sizeof(double) * nomega);
    const size_t o_zero = c.take(sizeof(double));
    const size_t o_mv1 = c.take(sizeof(int) * chunk);
    const size_t o_est1 = c.take(sizeof(double) * chunk);
    const size_t o_st1 = c.take(sizeof(int) * chunk);
    const size_t o_pe = precond != SGW_PRECOND_NONE ? c.take(sizeof(double) * chunk) : 0;
    const size_t o_po = precond != SGW_PRECOND_NONE ? c.take(sizeof(double) * chunk) : 0;
    const size_t o_pre = precond != SGW_PRECOND_NONE ? c.take(sizeof(double) * s->npw * (size_t)chunk) : 0;
    if ((r = ensure_ws(s, c.off)) != SGW_OK) return r;
    char* w = (char*)s->d_ws;
    std::vector<double> sig(nomega);
    for (int j = 0; j < nomega; ++j) sig[j] = omega[seed] - omega[j];
    SGW_CUDA(cudaMemcpyAsync(w + o_eref, e_ref, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st), "e_ref copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_om, omega, sizeof(double) * nomega, cudaMemcpyHostToDevice, st), "omega copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_sig, sig.data(), sizeof(double) * nomega, cudaMemcpyHostToDevice, st), "sig copy");
    SGW_CUDA(cudaMemsetAsync(w + o_zero, 0, sizeof(double), st), "memset");
    const double* d_etas = nullptr;
    if (eta_s) {
        SGW_CUDA(cudaMemcpyAsync(w + o_etas, eta_s, sizeof(double) * nomega, cudaMemcpyHostToDevice, st), "eta copy");
        d_etas = (const double*)(w + o_etas);
    }

    // One Lanczos launch: z_rj = e_ref_d[r] + omega_d[j] + i Im z, with Im z = eta_r_d[r], else
    // eta_s_d[j], else eta.
    auto run_lanczos = [&](char* base, int mk, const Plan& pl, int prec, int nr, int ns, const double2* rhs_d,
                           const double* e_ref_d, const double* omega_d, double tl, double ctl, double2* x_d, int* mv_d,
                           double* est_d, int* st_d, int owners, const double* eta_s_d,
                           const double* eta_r_d) -> cudaError_t {
        LanczosArgs L;
        L.nrhs = nr;
        L.nshift = ns;
        L.maxk = mk;
        L.rhs = rhs_d;
        L.e_ref = e_ref_d;
        L.omega = omega_d;
        L.eta = eta;
        L.tol = tl;
        L.cert_tol = ctl;
        L.x = x_d;
        const size_t vbytes = (size_t)prec_bytes(prec) * s->npw;
        const size_t o_ab = al256((size_t)owners * (mk + 1) * vbytes);
        L.basis = (double2*)base;
        L.ab = (double*)(base + o_ab);
        L.ysc = (double2*)(base + o_ab + al256((size_t)owners * pl.csize * 2 * (size_t)(mk + 1) * 8));
        L.counter = (int*)(w + o_cnt);
        L.out_mv = mv_d;
        L.out_res = est_d;
        L.out_status = st_d;
        L.eta_s = eta_s_d;
        L.eta_r = eta_r_d;
        return launch_lanczos(pl, L, owners, prec, threads, st);
    };

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool timed = report && report->kernel_ms;
    int launches = 0;
    if (timed) {
        SGW_CUDA(cudaEventCreate(&ev0), "event");
        SGW_CUDA(cudaEventCreate(&ev1), "event");
        SGW_CUDA(cudaEventRecord(ev0, st), "event");
    }
    Trace stage("sgw: multishift pass");
    if (done) {
        // 1''. the pass ran in a packed multi-system launch: take over its per-pair results
        SGW_CUDA(cudaMemcpyAsync(w + o_mv, done->mv, sizeof(int) * np, cudaMemcpyDeviceToDevice, st), "pass copy");
        SGW_CUDA(cudaMemcpyAsync(w + o_est, done->est, sizeof(double) * np, cudaMemcpyDeviceToDevice, st), "pass copy");
        SGW_CUDA(cudaMemcpyAsync(w + o_st, done->st, sizeof(int) * np, cudaMemcpyDeviceToDevice, st), "pass copy");
        launches += done->launches;
    } else if (have_x0) {
        // 1'. resume from the caller's solutions: every pair goes straight to the check
        SGW_CUDA(cudaMemcpyAsync(X, opts->x0, vb * np, cudaMemcpyDefault, st), "x0 copy");
        SGW_CUDA(cudaMemsetAsync(w + o_mv, 0, sizeof(int) * np, st), "memset");
        SGW_CUDA(cudaMemsetAsync(w + o_st, 0, sizeof(int) * np, st), "memset");
        SGW_CUDA(cudaMemsetAsync(w + o_est, 0, sizeof(double) * np, st), "memset");
    } else if (lanczos) {
        // 1. multishift pass
        SGW_CUDA(run_lanczos(pw, maxk, plan, precision, nrhs, nomega, rhs_d, (const double*)(w + o_eref),
                             (const double*)(w + o_om), tol, use_cert ? cert_tol : 0.0, X, (int*)(w + o_mv),
                             (double*)(w + o_est), (int*)(w + o_st), own, d_etas, nullptr),
                 "solver kernel");
        ++launches;
    } else {
        SolveArgs A;
        A.nrhs = nrhs;
        A.nshift = nomega;
        A.ell = ell;
        A.max_mv = max_mv;
        A.rhs = rhs_d;
        A.e_ref = (const double*)(w + o_eref);
        A.sig = (const double*)(w + o_sig);
        A.omega_seed = omega[seed];
        A.eta = eta;
        A.tol = tol;
        A.x = X;
        A.seedw = (double2*)pw;
        A.uw = (double2*)(pw + (size_t)own * vb * (2 * ell + 3));
        A.counter = (int*)(w + o_cnt);
        A.out_mv = (int*)(w + o_mv);
        A.out_res = (double*)(w + o_est);
        A.out_status = (int*)(w + o_st);
        SGW_CUDA(launch_solve(plan, A, own, st), "solver kernel");
        ++launches;
    }
    if (timed) SGW_CUDA(cudaEventRecord(ev1, st), "event");

    // 2. true residual of every pair (H in FP64 for the FP64 mode, else in float-float; the
    //    assembly and the norms in FP64)
    stage.next("sgw: FP64 residual check");
    double* d_rel = (double*)(w + o_rel);
    double* d_cert = (double*)(w + o_cert);
    const double* d_eref = (const double*)(w + o_eref);
    const double* d_om = (const double*)(w + o_om);
    // b = -P_c rhs once per right-hand side, shared by every residual check of its shifts
    const double2* d_b = project ? (const double2*)(w + o_bvec) : nullptr;
    if (project) {
        SGW_CUDA(launch_project_rhs(plan16, nrhs, rhs_d, (double2*)(w + o_bvec), st), "projection kernel");
        ++launches;
    }
    SGW_CUDA(launch_residual(plan16, nrhs, nomega, nullptr, 0, rhs_d, d_eref, d_om, eta, X, (double2*)(w + o_rscr),
                             d_rel, d_cert, nullptr, own_r, st, d_etas, d_b, res_prec, 1),
             "residual kernel");
    ++launches;
    std::vector<int> stv(np), mvv(np);
    std::vector<double> estv(np), relv(np), certv(np);
    SGW_CUDA(cudaMemcpyAsync(stv.data(), w + o_st, sizeof(int) * np, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(mvv.data(), w + o_mv, sizeof(int) * np, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(estv.data(), w + o_est, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(relv.data(), d_rel, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(certv.data(), d_cert, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaStreamSynchronize(st), "solve");
    if (timed) {
        float ms = 0.f;
        SGW_CUDA(cudaEventElapsedTime(&ms, ev0, ev1), "event");
        *report->kernel_ms = done ? done->kernel_ms : ms;
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    // Correction solves repair pairs the pass left near convergence (single-precision rounding,
    // the recursive / true residual gap, a certificate short of its target).  A pair still above
    // 1e-3 after the pass (its Krylov budget ran out far from the answer) is reported, not
    // corrected: one single-shift solve per such pair would cost up to nomega times the pass.
    // With x0 every pair is repaired (the caller asked for it).
    auto needs = [&](size_t q) {
        return std::isfinite(relv[q]) && stv[q] != SGW_PAIR_NONFINITE &&
               (relv[q] > tol || (use_cert && certv[q] > cert_tol)) && (have_x0 || relv[q] <= 1e-3);
    };

    if (passbuf.dev) {   // the pass's basis is released before the corrections
        SGW_CUDA(cudaFreeAsync(passbuf.dev, st), "Krylov workspace");
        passbuf.dev = nullptr;
    }

    // 3. per-shift correction solves for pairs above tol or the certificate target:
    //    A_j d = r_j, x_j += d (Lanczos in the correction precision, or preconditioned BiCGstab)
    stage.next("sgw: correction solves");
    std::vector<int> list, mv1(chunk);
    std::vector<double> eref1(chunk), eta1(chunk), pe(chunk), po(chunk);
    int fallbacks = 0;
    const int rounds = have_x0 ? std::max(max_refine, 1) : max_refine;
    for (int round = 0; round < rounds; ++round) {
        list.clear();
        for (size_t q = 0; q < np; ++q)
            if (needs(q)) list.push_back((int)q);
        if (list.empty()) break;
        // the learned diagonal drives the first preconditioned round (budget 2x the plain one when
        // given); the pairs it leaves unconverged restart from their current x with the plain one
        const int pc = precond == SGW_PRECOND_LEARNED && round > 0 ? SGW_PRECOND_PLAIN : precond;
        if (precond == SGW_PRECOND_LEARNED && round == 1) fallbacks += (int)list.size();
        for (size_t c0 = 0; c0 < list.size(); c0 += chunk) {
            const int nc = (int)std::min<size_t>(chunk, list.size() - c0);
            double need = 1.0;   // the smallest factor by which a pair's residual must drop
            for (int i = 0; i < nc; ++i) {
                const int q = list[c0 + i];
                eref1[i] = e_ref[q / nomega] + omega[q % nomega];
                eta1[i] = eta_s ? eta_s[q % nomega] : eta;
                pe[i] = e_ref[q / nomega];
                po[i] = omega[q % nomega];
                double f = tol / relv[q];
                if (use_cert && certv[q] > 0.0) f = std::min(f, cert_tol / certv[q]);
                need = std::min(need, f);
            }
            SGW_CUDA(cudaMemcpyAsync(w + o_list, list.data() + c0, sizeof(int) * nc, cudaMemcpyHostToDevice, st),
                     "list copy");
            SGW_CUDA(cudaMemcpyAsync(w + o_eref1, eref1.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st),
                     "list copy");
            SGW_CUDA(cudaMemcpyAsync(w + o_eta1, eta1.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st),
                     "list copy");
            const int* d_list = (const int*)(w + o_list);
            Staged corrbuf;   // this chunk's Krylov workspace
            SGW_CUDA(cudaMallocAsync(&corrbuf.dev, corr_bytes(nc), st), "correction workspace");
            corrbuf.owned = true;
            corrbuf.st = st;
            char* cw = (char*)corrbuf.dev;
            SGW_CUDA(launch_residual(plan16, nrhs, nomega, d_list, nc, rhs_d, d_eref, d_om, eta, X,
                                     (double2*)(w + o_rscr), d_rel, d_cert, (double2*)(w + o_rvec),
                                     std::min(own_r, nc), st, d_etas, d_b, res_prec, 1),
                     "residual kernel");
            const double tl = std::min(0.5, std::max(1e-13, 0.3 * need));
            if (!bicg_corr) {
                SGW_CUDA(run_lanczos(cw, maxk_c, plan16, corr_prec, nc, 1, (const double2*)(w + o_rvec),
                                     (const double*)(w + o_eref1), (const double*)(w + o_zero), tl, 0.0,
                                     (double2*)(w + o_dbuf), (int*)(w + o_mv1), (double*)(w + o_est1),
                                     (int*)(w + o_st1), std::min(own1, nc), nullptr, (const double*)(w + o_eta1)),
                         "correction solve");
            } else {
                // the diagonal of each pair from its correction right-hand side (plain: kinetic
                // scaling by the residual's kinetic energy; learned: the perceptron on top)
                if (pc != SGW_PRECOND_NONE) {
                SGW_CUDA(cudaMemcpyAsync(w + o_pe, pe.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st), "copy");
                SGW_CUDA(cudaMemcpyAsync(w + o_po, po.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st), "copy");
                PrecondArgs pa;
                pa.n = nc;
                pa.mode = pc;
                pa.rhs = (const double2*)(w + o_rvec);
                pa.e_ref = (const double*)(w + o_pe);
                pa.omega = (const double*)(w + o_po);
                pa.delta = nullptr;
                pa.eta = eta;
                pa.half_ecut = 0.5 * s->ecut;
                pa.v_mean = s->v_mean;
                pa.mlp = pc == SGW_PRECOND_LEARNED ? mlp_weights(mlp) : nullptr;
                pa.d = (double*)(w + o_pre);
                SGW_CUDA(launch_precond(plan16, pa, st), "preconditioner kernel");
                }
                SolveArgs A;
                A.nrhs = nc;
                A.nshift = 1;
                A.ell = ell;
                A.max_mv = (pc == SGW_PRECOND_LEARNED && plain_budget > 0) ? 2 * plain_budget
                                                                              : std::max(max_mv, 40000);
                A.rhs = (const double2*)(w + o_rvec);
                A.e_ref = (const double*)(w + o_eref1);
                A.sig = (const double*)(w + o_zero);
                A.omega_seed = 0.0;
                A.eta = eta;
                A.tol = tl;
                A.x = (double2*)(w + o_dbuf);
                const int gb = std::min(grid_b, nc);
                A.seedw = (double2*)cw;
                A.uw = (double2*)(cw + (size_t)gb * vb * (2 * ell + 3));
                A.pscr = (double2*)(cw + (size_t)gb * vb * (2 * ell + 4));
                A.pre = pc != SGW_PRECOND_NONE ? (const double*)(w + o_pre) : nullptr;
                A.counter = (int*)(w + o_cnt);
                A.out_mv = (int*)(w + o_mv1);
                A.out_res = (double*)(w + o_est1);
                A.out_status = (int*)(w + o_st1);
                SGW_CUDA(launch_solve(plan16, A, gb, st), "preconditioned correction solve");
                ++launches;
            }
            SGW_CUDA(launch_pair_axpy(nc, d_list, s->npw, (const double2*)(w + o_dbuf), X, st), "refinement update");
            SGW_CUDA(launch_residual(plan16, nrhs, nomega, d_list, nc, rhs_d, d_eref, d_om, eta, X,
                                     (double2*)(w + o_rscr), d_rel, d_cert, nullptr, std::min(own_r, nc), st, d_etas,
                                     d_b, res_prec, 1),
                     "residual kernel");
            launches += 4;
            SGW_CUDA(cudaMemcpyAsync(mv1.data(), w + o_mv1, sizeof(int) * nc, cudaMemcpyDeviceToHost, st), "report");
            SGW_CUDA(cudaStreamSynchronize(st), "refinement");
            for (int i = 0; i < nc; ++i) mvv[list[c0 + i]] += mv1[i];
        }
        SGW_CUDA(cudaMemcpyAsync(relv.data(), d_rel, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "report");
        SGW_CUDA(cudaMemcpyAsync(certv.data(), d_cert, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "report");
        SGW_CUDA(cudaStreamSynchronize(st), "refinement");
    }
    bool all = true;
    for (size_t q = 0; q < np; ++q) {
        const bool ok = relv[q] <= tol && (!use_cert || certv[q] <= cert_tol);
        if (ok) stv[q] = SGW_PAIR_CONVERGED;
        else if (stv[q] == SGW_PAIR_CONVERGED) stv[q] = SGW_PAIR_MAXITER;
        all = all && stv[q] == SGW_PAIR_CONVERGED;
    }
    if (report) {
        if (report->status) std::memcpy(report->status, stv.data(), sizeof(int) * np);
        if (report->matvecs) std::memcpy(report->matvecs, mvv.data(), sizeof(int) * np);
        if (report->est_res) std::memcpy(report->est_res, estv.data(), sizeof(double) * np);
        if (report->rel_res) std::memcpy(report->rel_res, relv.data(), sizeof(double) * np);
        if (report->cert) std::memcpy(report->cert, certv.data(), sizeof(double) * np);
        if (report->launches) *report->launches = launches;
        if (report->fallbacks) *report->fallbacks = fallbacks;
    }
    if (!all) return fail(SGW_ENOCONV, "some (rhs, omega) pairs did not reach the tolerance or the certificate");
    return SGW_OK;
}


sgw_status sgw_solve_shifted(sgw_system* s, int nrhs, const void* rhs, const double* e_ref, int nomega,
                             const double* omega, double eta, double tol, const sgw_solve_opts* opts, void* dpsi,
                             sgw_report* report) {
    g_err.clear();
    if (!s || !rhs || !e_ref || !omega || !dpsi) return fail(SGW_EINVAL, "NULL argument");
    if (nrhs < 0 || nomega < 1) return fail(SGW_EINVAL, "need nrhs >= 0 and nomega >= 1");
    if (nomega > kMaxShifts) return fail(SGW_EUNSUPPORTED, "nomega above 512");
    if (!(eta > 0.0) || !std::isfinite(eta))
        return fail(SGW_EINVAL, "eta must be positive (the shifted systems are singular at eta = 0)");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(SGW_EINVAL, "tol must be positive");
    if (!finite_all(e_ref, nrhs) || !finite_all(omega, nomega)) return fail(SGW_EINVAL, "non-finite e_ref or omega");
    if (s->nocc == 0) return fail(SGW_ESTATE, "sgw_set_occupied has not been called");
    if (nrhs == 0) return SGW_OK;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_solve_shifted");
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    Staged in, out;
    sgw_status r;
    if ((r = stage_in(rhs, vb * nrhs, in, st, "rhs")) != SGW_OK) return r;
    if ((r = stage_out(dpsi, vb * (size_t)nrhs * nomega, out, "dpsi", st)) != SGW_OK) return r;
    const sgw_status rs = multishift(s, true, nrhs, (const double2*)in.dev, e_ref, nomega, omega, nullptr, eta, tol,
                                     opts, (double2*)out.dev, report, st);
    if (rs != SGW_OK && rs != SGW_ENOCONV) return rs;
    if ((r = finish_out(out, st, "dpsi copy")) != SGW_OK) return r;
    SGW_CUDA(cudaStreamSynchronize(st), "solve");
    return rs;
}

sgw_status sgw_solve_batched(int nitems, const sgw_batch_item* items, double eta, double tol,
                             const sgw_solve_opts* opts) {
    g_err.clear();
    if (nitems < 0 || (nitems > 0 && !items)) return fail(SGW_EINVAL, "bad item list");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(SGW_EINVAL, "eta must be positive");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(SGW_EINVAL, "tol must be positive");
    if (opts && opts->method != SGW_METHOD_LANCZOS) return fail(SGW_EUNSUPPORTED, "batched solves use the Lanczos method");
    if (opts && opts->x0) return fail(SGW_EUNSUPPORTED, "batched solves take no x0");
    const int precision = opts ? opts->precision : SGW_PREC_FP64;
    if (precision != SGW_PREC_FP64 && precision != SGW_PREC_DF32 && precision != SGW_PREC_FP32)
        return fail(SGW_EINVAL, "unknown precision");
    const int threads = opts ? opts->threads : 0;
    const double cert_tol = !opts || opts->cert_tol == 0.0 ? 1e-8 : opts->cert_tol;
    if (nitems == 0) return SGW_OK;
    const int dev = items[0].sys ? items[0].sys->dev : 0;
    for (int i = 0; i < nitems; ++i) {
        const sgw_batch_item& it = items[i];
        if (!it.sys || !it.rhs || !it.e_ref || !it.omega || !it.dpsi) return fail(SGW_EINVAL, "NULL field in an item");
        if (it.sys->dev != dev) return fail(SGW_EINVAL, "items on different devices");
        if (it.nrhs < 0 || it.nomega < 1 || it.nomega > kMaxShifts) return fail(SGW_EINVAL, "item sizes out of range");
        if (!finite_all(it.e_ref, it.nrhs) || !finite_all(it.omega, it.nomega))
            return fail(SGW_EINVAL, "non-finite e_ref or omega");
        if (it.sys->nocc == 0) return fail(SGW_ESTATE, "sgw_set_occupied has not been called");
        for (int j = 0; j < i; ++j)
            if (items[j].sys == it.sys) return fail(SGW_EINVAL, "a system appears in two items (merge their rhs)");
        const Plan& pl = precision == SGW_PREC_FP32 ? it.sys->plan8 : it.sys->plan;
        if (pl.csize == 0) return fail(SGW_EUNSUPPORTED, "an item's box does not fit on chip in FP32");
        if (lanczos_smem_bytes(pl, it.nomega, precision) > max_optin_smem())
            return fail(SGW_EUNSUPPORTED, "too many frequencies for the on-chip shift state");
    }
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
    DeviceScope dscope(dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_solve_batched");
    const int es = prec_bytes(precision);
    const int max_mv = opts && opts->max_matvec > 0 ? opts->max_matvec : 16384;
    // every item's buffers on the device
    std::vector<Staged> in(nitems), out(nitems);
    sgw_status r;
    for (int i = 0; i < nitems; ++i) {
        const size_t vb = sizeof(double2) * (size_t)items[i].sys->npw;
        if ((r = stage_in(items[i].rhs, vb * items[i].nrhs, in[i], st, "rhs")) != SGW_OK) return r;
        if ((r = stage_out(items[i].dpsi, vb * (size_t)items[i].nrhs * items[i].nomega, out[i], "dpsi", st)) !=
            SGW_OK)
            return r;
    }
    // per-item device arrays: e_ref, omega and the pass's per-pair outputs
    std::vector<size_t> o_er(nitems), o_om(nitems), o_mv(nitems), o_es(nitems), o_stt(nitems);
    Carve c;
    for (int i = 0; i < nitems; ++i) {
        const size_t np = (size_t)items[i].nrhs * items[i].nomega;
        o_er[i] = c.take(sizeof(double) * items[i].nrhs);
        o_om[i] = c.take(sizeof(double) * items[i].nomega);
        o_mv[i] = c.take(sizeof(int) * np);
        o_es[i] = c.take(sizeof(double) * np);
        o_stt[i] = c.take(sizeof(int) * np);
    }
    Staged small;
    SGW_CUDA(cudaMallocAsync(&small.dev, c.off, st), "batch allocation");
    small.owned = true;
    small.st = st;
    char* ws = (char*)small.dev;
    for (int i = 0; i < nitems; ++i) {
        SGW_CUDA(cudaMemcpyAsync(ws + o_er[i], items[i].e_ref, sizeof(double) * items[i].nrhs, cudaMemcpyHostToDevice,
                                 st),
                 "e_ref copy");
        SGW_CUDA(cudaMemcpyAsync(ws + o_om[i], items[i].omega, sizeof(double) * items[i].nomega,
                                 cudaMemcpyHostToDevice, st),
                 "omega copy");
    }
    // items with the same cluster size share one persistent launch; the largest systems first
    std::map<int, std::vector<int>> groups;
    for (int i = 0; i < nitems; ++i) {
        const Plan& pl = precision == SGW_PREC_FP32 ? items[i].sys->plan8 : items[i].sys->plan;
        if (items[i].nrhs > 0) groups[pl.csize].push_back(i);
    }
    std::vector<double> group_ms(nitems, 0.0);
    std::vector<int> group_launch(nitems, 0);
    auto al256 = [](size_t b) { return (b + 255) / 256 * 256; };
    for (auto& kv : groups) {
        std::vector<int> idx = kv.second;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return items[a].sys->npw > items[b].sys->npw; });
        int smem = 0, max_npw = 0, max_ns = 0, total = 0;
        for (int i : idx) {
            const Plan& pl = precision == SGW_PREC_FP32 ? items[i].sys->plan8 : items[i].sys->plan;
            smem = std::max(smem, lanczos_smem_bytes(pl, items[i].nomega, precision));
            max_npw = std::max(max_npw, items[i].sys->npw);
            max_ns = std::max(max_ns, items[i].nomega);
            total += items[i].nrhs;
        }
        const Plan& p0 = precision == SGW_PREC_FP32 ? items[idx[0]].sys->plan8 : items[idx[0]].sys->plan;
        int owners = 0;
        SGW_CUDA(lanczos_batch_capacity(p0, threads, precision, smem, &owners), "solver occupancy");
        owners = std::max(1, std::min(owners, total));
        // every owner's basis sized for the largest system, capped by free memory
        size_t free_b = 0, total_b = 0;
        SGW_CUDA(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
        const size_t budget = std::min<size_t>(free_b / 2, (size_t)96 << 30);
        const int ctas = owners * p0.csize;
        const size_t per_k = (size_t)owners * es * max_npw + (size_t)ctas * (16 + 32 * (size_t)max_ns);
        const size_t cap = budget / std::max<size_t>(per_k, 1);
        if (cap < 8) return fail(SGW_ENOMEM, "not enough device memory for the Lanczos bases");
        const int maxk = (int)std::min<size_t>((size_t)max_mv, cap - 2);
        const size_t vstride = (size_t)(maxk + 1) * max_npw;
        const size_t ystride = 2 * (size_t)maxk * max_ns;
        const size_t o_ab = al256((size_t)owners * vstride * es);
        const size_t o_ysc = o_ab + al256((size_t)ctas * 2 * (maxk + 1) * 8);
        const size_t o_items = o_ysc + al256((size_t)ctas * ystride * 16);
        const size_t o_start = o_items + al256(sizeof(BatchItem) * idx.size());
        const size_t o_cnt = o_start + al256(sizeof(int) * (idx.size() + 1));
        Staged gbuf;   // the group's Krylov workspace, for this launch only
        SGW_CUDA(cudaMallocAsync(&gbuf.dev, o_cnt + 256, st), "batch workspace");
        gbuf.owned = true;
        gbuf.st = st;
        char* w = (char*)gbuf.dev;
        std::vector<BatchItem> hb(idx.size());
        std::vector<int> start(idx.size() + 1, 0);
        for (size_t t = 0; t < idx.size(); ++t) {
            const int i = idx[t];
            const Plan& pl = precision == SGW_PREC_FP32 ? items[i].sys->plan8 : items[i].sys->plan;
            hb[t].plan = tuned_plan(pl, lanczos_extra(items[i].nomega), es);
            LanczosArgs& A = hb[t].args;
            A = LanczosArgs();
            A.nrhs = items[i].nrhs;
            A.nshift = items[i].nomega;
            A.maxk = maxk;
            A.rhs = (const double2*)in[i].dev;
            A.e_ref = (const double*)(ws + o_er[i]);
            A.omega = (const double*)(ws + o_om[i]);
            A.eta = eta;
            A.tol = tol;
            A.cert_tol = cert_tol > 0.0 ? cert_tol : 0.0;
            A.x = (double2*)out[i].dev;
            A.basis = (double2*)w;
            A.ab = (double*)(w + o_ab);
            A.ysc = (double2*)(w + o_ysc);
            A.counter = (int*)(w + o_cnt);
            A.out_mv = (int*)(ws + o_mv[i]);
            A.out_res = (double*)(ws + o_es[i]);
            A.out_status = (int*)(ws + o_stt[i]);
            A.vstride = vstride;
            A.ystride = ystride;
            start[t + 1] = start[t] + items[i].nrhs;
        }
        SGW_CUDA(cudaMemcpyAsync(w + o_items, hb.data(), sizeof(BatchItem) * hb.size(), cudaMemcpyHostToDevice, st),
                 "items copy");
        SGW_CUDA(cudaMemcpyAsync(w + o_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, st),
                 "start copy");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        SGW_CUDA(cudaEventCreate(&e0), "event");
        SGW_CUDA(cudaEventCreate(&e1), "event");
        SGW_CUDA(cudaEventRecord(e0, st), "event");
        SGW_CUDA(launch_lanczos_batch(hb[0].plan, (const BatchItem*)(w + o_items), (const int*)(w + o_start),
                                      (int)idx.size(), (int*)(w + o_cnt), owners, precision, threads, smem, st),
                 "batched solver kernel");
        SGW_CUDA(cudaEventRecord(e1, st), "event");
        SGW_CUDA(cudaEventSynchronize(e1), "batched solver kernel");   // the workspace is reused next
        float ms = 0.f;
        SGW_CUDA(cudaEventElapsedTime(&ms, e0, e1), "event");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (size_t t = 0; t < idx.size(); ++t) {
            group_ms[idx[t]] = ms;
            group_launch[idx[t]] = t == 0 ? 1 : 0;
        }
    }
    // the FP64 check and the corrections of every item, as in sgw_solve_shifted
    sgw_status worst = SGW_OK;
    for (int i = 0; i < nitems; ++i) {
        if (items[i].nrhs == 0) continue;
        const PassDone done{(const int*)(ws + o_mv[i]), (const double*)(ws + o_es[i]), (const int*)(ws + o_stt[i]),
                            group_ms[i], group_launch[i]};
        const sgw_status rs = multishift(items[i].sys, true, items[i].nrhs, (const double2*)in[i].dev, items[i].e_ref,
                                         items[i].nomega, items[i].omega, nullptr, eta, tol, opts,
                                         (double2*)out[i].dev, items[i].report, st, &done);
        if (rs != SGW_OK && rs != SGW_ENOCONV) return rs;
        if (rs == SGW_ENOCONV) worst = rs;
        if ((r = finish_out(out[i], st, "dpsi copy")) != SGW_OK) return r;
    }
    SGW_CUDA(cudaStreamSynchronize(st), "batched solve");
    if (worst != SGW_OK) return fail(worst, "some (rhs, omega) pairs did not reach the tolerance or the certificate");
    return SGW_OK;
}

sgw_status sgw_solve_green(sgw_system* s, int ncol, const int* cols, int nz, const double* z, double tol,
                           const sgw_solve_opts* opts, void* g, sgw_report* report) {
    g_err.clear();
    if (!s || !z || !g || (ncol > 0 && !cols)) return fail(SGW_EINVAL, "NULL argument");
    if (ncol < 0 || nz < 1) return fail(SGW_EINVAL, "need ncol >= 0 and nz >= 1");
    if (nz > kMaxShifts) return fail(SGW_EUNSUPPORTED, "nz above 512");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(SGW_EINVAL, "tol must be positive");
    std::vector<double> zre(nz), zim(nz);
    for (int j = 0; j < nz; ++j) {
        zre[j] = z[2 * j];
        zim[j] = z[2 * j + 1];
        if (!std::isfinite(zre[j]) || !std::isfinite(zim[j])) return fail(SGW_EINVAL, "non-finite z");
        if (zim[j] == 0.0) return fail(SGW_EINVAL, "Im z must be nonzero (z - H is singular on the real axis)");
    }
    if (ncol > 0 && is_device_ptr(cols)) return fail(SGW_EINVAL, "cols must be a host array");
    for (int c = 0; c < ncol; ++c)
        if (cols[c] < 0 || cols[c] >= s->npw) return fail(SGW_EINVAL, "column index outside [0, n_pw)");
    if (ncol == 0) return SGW_OK;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_solve_green");
    // the operator is H itself: no occupied states
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    Staged in_cols, rb, out;
    sgw_status r;
    if ((r = stage_in(cols, sizeof(int) * ncol, in_cols, st, "cols")) != SGW_OK) return r;
    SGW_CUDA(cudaMallocAsync(&rb.dev, vb * ncol, st), "rhs allocation");
    rb.owned = true;
    rb.st = st;
    SGW_CUDA(launch_unit_rhs((const int*)in_cols.dev, ncol, s->npw, (double2*)rb.dev, st), "unit rhs kernel");
    if ((r = stage_out(g, vb * (size_t)ncol * nz, out, "g", st)) != SGW_OK) return r;
    std::vector<double> e0(ncol, 0.0);
    const sgw_status rs = multishift(s, false, ncol, (const double2*)rb.dev, e0.data(), nz, zre.data(), zim.data(), 0.0,
                                     tol, opts, (double2*)out.dev, report, st);
    if (rs != SGW_OK && rs != SGW_ENOCONV) return rs;
    if (report && report->launches) *report->launches += 1;
    if ((r = finish_out(out, st, "g copy")) != SGW_OK) return r;
    SGW_CUDA(cudaStreamSynchronize(st), "solve");
    return rs;
}

// One k-point's contribution to Eq. 5 at complex frequencies w_j = wre[j] + i wim[j]
// (Im w_j != 0): shifts z = eps_v + w_j and eps_v - w_j in one Krylov space per right-hand side.
static sgw_status density_common(sgw_system* s, int n_v, int n_pert, const void* rhs, const double* eps_v,
                                 int nomega, const double* wre, const double* wim, double weight, double tol,
                                 const sgw_solve_opts* opts, void* dn, sgw_report* report) {
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(SGW_EINVAL, "tol must be positive");
    if (!std::isfinite(weight)) return fail(SGW_EINVAL, "non-finite weight");
    if (!finite_all(eps_v, n_v)) return fail(SGW_EINVAL, "non-finite eps_v");
    if (s->nocc == 0) return fail(SGW_ESTATE, "sgw_set_occupied has not been called");
    const int nrhs = n_v * n_pert;
    if (nrhs == 0) return SGW_OK;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_density_response");
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    const size_t dn_bytes = sizeof(double2) * (size_t)n_pert * n_pert * nomega;
    Staged in, xb, dnb;
    sgw_status r;
    if ((r = stage_in(rhs, vb * nrhs, in, st, "rhs")) != SGW_OK) return r;
    if ((r = stage_in(dn, dn_bytes, dnb, st, "dn")) != SGW_OK) return r;
    SGW_CUDA(cudaMallocAsync(&xb.dev, vb * (size_t)nrhs * 2 * nomega, st), "solution allocation");
    xb.owned = true;
    xb.st = st;
    // shifts z = eps_v + w_j (j < nomega) and eps_v - w_j (the -w branch)
    std::vector<double> e_rows(nrhs), om2(2 * nomega), eta2(2 * nomega);
    for (int i = 0; i < nrhs; ++i) e_rows[i] = eps_v[i / n_pert];
    for (int j = 0; j < nomega; ++j) {
        om2[j] = wre[j];
        eta2[j] = wim[j];
        om2[nomega + j] = -wre[j];
        eta2[nomega + j] = -wim[j];
    }
    const sgw_status rs = multishift(s, true, nrhs, (const double2*)in.dev, e_rows.data(), 2 * nomega, om2.data(),
                                     eta2.data(), 1.0, tol, opts, (double2*)xb.dev, report, st);
    if (rs != SGW_OK && rs != SGW_ENOCONV) return rs;
    SGW_CUDA(launch_density(n_v, n_pert, nomega, s->npw, (const double2*)in.dev, (const double2*)xb.dev, weight,
                            (double2*)dnb.dev, st),
             "density kernel");
    if (report && report->launches) *report->launches += 1;
    if (dnb.owned) SGW_CUDA(cudaMemcpyAsync(dn, dnb.dev, dn_bytes, cudaMemcpyDeviceToHost, st), "dn copy");
    SGW_CUDA(cudaStreamSynchronize(st), "density response");
    return rs;
}

sgw_status sgw_density_response(sgw_system* s, int n_v, int n_pert, const void* rhs, const double* eps_v, int nomega,
                                const double* omega, double eta, double weight, double tol,
                                const sgw_solve_opts* opts, void* dn, sgw_report* report) {
    g_err.clear();
    if (!s || !eps_v || !omega || !dn || (n_v > 0 && n_pert > 0 && !rhs)) return fail(SGW_EINVAL, "NULL argument");
    if (n_v < 0 || n_pert < 0 || nomega < 1) return fail(SGW_EINVAL, "need n_v, n_pert >= 0 and nomega >= 1");
    if (2 * nomega > kMaxShifts) return fail(SGW_EUNSUPPORTED, "nomega above 256 (2 nomega shifts per right-hand side)");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(SGW_EINVAL, "eta must be positive");
    if (!finite_all(omega, nomega)) return fail(SGW_EINVAL, "non-finite omega");
    std::vector<double> wim(nomega, eta);
    return density_common(s, n_v, n_pert, rhs, eps_v, nomega, omega, wim.data(), weight, tol, opts, dn, report);
}

sgw_status sgw_density_response_w(sgw_system* s, int n_v, int n_pert, const void* rhs, const double* eps_v, int nw,
                                  const double* w, double weight, double tol, const sgw_solve_opts* opts, void* dn,
                                  sgw_report* report) {
    g_err.clear();
    if (!s || !eps_v || !w || !dn || (n_v > 0 && n_pert > 0 && !rhs)) return fail(SGW_EINVAL, "NULL argument");
    if (n_v < 0 || n_pert < 0 || nw < 1) return fail(SGW_EINVAL, "need n_v, n_pert >= 0 and nw >= 1");
    if (2 * nw > kMaxShifts) return fail(SGW_EUNSUPPORTED, "nw above 256 (2 nw shifts per right-hand side)");
    std::vector<double> wre(nw), wim(nw);
    for (int j = 0; j < nw; ++j) {
        wre[j] = w[2 * j];
        wim[j] = w[2 * j + 1];
        if (!std::isfinite(wre[j]) || !std::isfinite(wim[j])) return fail(SGW_EINVAL, "non-finite w");
        if (wim[j] == 0.0) return fail(SGW_EINVAL, "Im w must be nonzero (the shifted systems are singular on the real axis)");
    }
    return density_common(s, n_v, n_pert, rhs, eps_v, nw, wre.data(), wim.data(), weight, tol, opts, dn, report);
}

sgw_status sgw_aaa(int nfun, int m, const void* z, const void* f, double tol, int mmax, int n_eval, const void* z_eval,
                   void* r_eval, int* degree, void* stream) {
    g_err.clear();
    if (nfun < 0 || m < 0 || n_eval < 0 || mmax < 1) return fail(SGW_EINVAL, "negative size or mmax < 1");
    if (nfun == 0) return SGW_OK;
    if (m < 1) return fail(SGW_EINVAL, "need at least one sample");
    if (!z || !f || (n_eval > 0 && (!z_eval || !r_eval))) return fail(SGW_EINVAL, "NULL argument");
    if (m > 128 || mmax > 32) return fail(SGW_EUNSUPPORTED, "m above 128 or mmax above 32");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(SGW_EINVAL, "tol must be >= 0");
    if (is_device_ptr(z) || (n_eval > 0 && is_device_ptr(z_eval)))
        return fail(SGW_EINVAL, "z and z_eval must be host arrays");
    const double* zd = (const double*)z;
    if (!finite_all(zd, 2 * (size_t)m) || (n_eval > 0 && !finite_all((const double*)z_eval, 2 * (size_t)n_eval)))
        return fail(SGW_EINVAL, "non-finite sample or evaluation point");
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j)
            if (zd[2 * i] == zd[2 * j] && zd[2 * i + 1] == zd[2 * j + 1]) return fail(SGW_EINVAL, "repeated sample point");
    cudaStream_t st = (cudaStream_t)stream;
    Staged zb, fb, eb, rb, db, flag;
    sgw_status r;
    if ((r = stage_in(z, sizeof(double2) * m, zb, st, "z")) != SGW_OK) return r;
    if ((r = stage_in(f, sizeof(double2) * (size_t)nfun * m, fb, st, "f")) != SGW_OK) return r;
    if (n_eval > 0) {
        if ((r = stage_in(z_eval, sizeof(double2) * n_eval, eb, st, "z_eval")) != SGW_OK) return r;
        if ((r = stage_out(r_eval, sizeof(double2) * (size_t)nfun * n_eval, rb, "r_eval", st)) != SGW_OK) return r;
    }
    if (degree && (r = stage_out(degree, sizeof(int) * nfun, db, "degree", st)) != SGW_OK) return r;
    SGW_CUDA(cudaMallocAsync(&flag.dev, sizeof(int), st), "flag allocation");
    flag.owned = true;
    flag.st = st;
    SGW_CUDA(cudaMemsetAsync(flag.dev, 0, sizeof(int), st), "memset");
    SGW_CUDA(launch_aaa(nfun, m, (const double2*)zb.dev, (const double2*)fb.dev, tol, mmax, n_eval,
                        (const double2*)eb.dev, (double2*)rb.dev, degree ? (int*)db.dev : nullptr, (int*)flag.dev, st),
             "AAA kernel");
    int bad = 0;
    SGW_CUDA(cudaMemcpyAsync(&bad, flag.dev, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
    if (n_eval > 0 && (r = finish_out(rb, st, "r_eval copy")) != SGW_OK) return r;
    if (degree && (r = finish_out(db, st, "degree copy")) != SGW_OK) return r;
    SGW_CUDA(cudaStreamSynchronize(st), "AAA");
    if (bad) return fail(SGW_EINVAL, "non-finite samples (their functions' outputs are NaN)");
    return SGW_OK;
}

sgw_status sgw_screened_coulomb(int n_g, int nomega, const void* dn, const double* qg, double volume, double r_cut,
                                void* eps_inv, void* wbar, void* stream) {
    g_err.clear();
    if (n_g < 0 || nomega < 0) return fail(SGW_EINVAL, "negative size");
    if (n_g == 0 || nomega == 0) return SGW_OK;
    if (!dn || !qg || !wbar) return fail(SGW_EINVAL, "NULL argument");
    if (n_g > 64) return fail(SGW_EUNSUPPORTED, "n_g above 64 (the matrix is inverted in shared memory)");
    if (!(volume > 0.0) || !std::isfinite(volume)) return fail(SGW_EINVAL, "volume must be positive");
    if (!std::isfinite(r_cut)) return fail(SGW_EINVAL, "non-finite r_cut");
    if (is_device_ptr(qg)) return fail(SGW_EINVAL, "qg must be a host array");
    if (!finite_all(qg, 3 * (size_t)n_g)) return fail(SGW_EINVAL, "non-finite q + G");
    if (r_cut <= 0.0)
        for (int g = 0; g < n_g; ++g)
            if (qg[3 * g] == 0.0 && qg[3 * g + 1] == 0.0 && qg[3 * g + 2] == 0.0)
                return fail(SGW_EINVAL, "q + G = 0 needs a truncated Coulomb potential (r_cut > 0)");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t mb = sizeof(double2) * (size_t)n_g * n_g * nomega;
    Staged in, q, oe, ow, flag;
    sgw_status r;
    if ((r = stage_in(dn, mb, in, st, "dn")) != SGW_OK) return r;
    if ((r = stage_in(qg, sizeof(double) * 3 * (size_t)n_g, q, st, "q + G")) != SGW_OK) return r;
    if (eps_inv && (r = stage_out(eps_inv, mb, oe, "eps_inv", st)) != SGW_OK) return r;
    if ((r = stage_out(wbar, mb, ow, "wbar", st)) != SGW_OK) return r;
    SGW_CUDA(cudaMallocAsync(&flag.dev, sizeof(int), st), "flag allocation");
    flag.owned = true;
    flag.st = st;
    SGW_CUDA(cudaMemsetAsync(flag.dev, 0, sizeof(int), st), "memset");
    SGW_CUDA(launch_screening(n_g, nomega, (const double2*)in.dev, (const double*)q.dev, 1.0 / volume, r_cut,
                              eps_inv ? (double2*)oe.dev : nullptr, (double2*)ow.dev, (int*)flag.dev, st),
             "screening kernel");
    int bad = 0;
    SGW_CUDA(cudaMemcpyAsync(&bad, flag.dev, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
    if (eps_inv && (r = finish_out(oe, st, "eps_inv copy")) != SGW_OK) return r;
    if ((r = finish_out(ow, st, "wbar copy")) != SGW_OK) return r;
    SGW_CUDA(cudaStreamSynchronize(st), "screening");
    if (bad) return fail(SGW_ENOCONV, "epsilon is singular at some frequency (its outputs are NaN)");
    return SGW_OK;
}

static sgw_status precond_common(sgw_system* s, int npairs, const double2* rhs_d, const double* eref_d,
                                 const double* om_d, const double* delta_d, double eta, int precond,
                                 const sgw_mlp* mlp, double* d_d, cudaStream_t st) {
    PrecondArgs a;
    a.n = npairs;
    a.mode = precond;
    a.rhs = rhs_d;
    a.e_ref = eref_d;
    a.omega = om_d;
    a.delta = delta_d;
    a.eta = eta;
    a.half_ecut = 0.5 * s->ecut;
    a.v_mean = s->v_mean;
    a.mlp = precond == SGW_PRECOND_LEARNED ? mlp_weights(mlp) : nullptr;
    a.d = d_d;
    SGW_CUDA(launch_precond(s->plan, a, st), "preconditioner kernel");
    return SGW_OK;
}

static sgw_status check_precond(int precond, const double* delta, int n, const sgw_mlp* mlp) {
    if (precond < SGW_PRECOND_NONE || precond > SGW_PRECOND_JACOBI) return fail(SGW_EINVAL, "bad precond");
    if (precond == SGW_PRECOND_LEARNED && !mlp) return fail(SGW_EINVAL, "learned preconditioner needs an sgw_mlp");
    if (precond == SGW_PRECOND_JACOBI) {
        if (!delta) return fail(SGW_EINVAL, "Jacobi preconditioner needs delta");
        for (int i = 0; i < n; ++i)
            if (!(delta[i] > 0.0) || !std::isfinite(delta[i])) return fail(SGW_EINVAL, "delta must be positive");
    }
    return SGW_OK;
}

sgw_status sgw_precond_diag(sgw_system* s, int npairs, const void* rhs, const double* e_ref, const double* omega,
                            double eta, int precond, const double* delta, const sgw_mlp* mlp, double* d, void* stream) {
    g_err.clear();
    if (!s || !rhs || !e_ref || !omega || !d) return fail(SGW_EINVAL, "NULL argument");
    sgw_status r;
    if ((r = check_precond(precond, delta, npairs, mlp)) != SGW_OK) return r;
    if (precond == SGW_PRECOND_NONE) return fail(SGW_EINVAL, "no diagonal for SGW_PRECOND_NONE");
    if (npairs <= 0) return SGW_OK;
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_precond_diag");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    Staged in, out;
    if ((r = stage_in(rhs, vb * npairs, in, st, "rhs")) != SGW_OK) return r;
    if ((r = stage_out(d, sizeof(double) * s->npw * (size_t)npairs, out, "d", st)) != SGW_OK) return r;
    Carve c;
    const size_t o_e = c.take(sizeof(double) * npairs), o_o = c.take(sizeof(double) * npairs),
                 o_d = c.take(sizeof(double) * npairs);
    if ((r = ensure_ws(s, c.off)) != SGW_OK) return r;
    char* w = (char*)s->d_ws;
    SGW_CUDA(cudaMemcpyAsync(w + o_e, e_ref, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_o, omega, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    if (delta) SGW_CUDA(cudaMemcpyAsync(w + o_d, delta, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    if ((r = precond_common(s, npairs, (const double2*)in.dev, (const double*)(w + o_e), (const double*)(w + o_o),
                            delta ? (const double*)(w + o_d) : nullptr, eta, precond, mlp, (double*)out.dev, st)) !=
        SGW_OK)
        return r;
    if ((r = finish_out(out, st, "d copy")) != SGW_OK) return r;
    SGW_CUDA(cudaStreamSynchronize(st), "precond");
    return SGW_OK;
}

sgw_status sgw_training_rows(sgw_system* s, int npairs, const void* rhs, const double* e_ref, const double* omega,
                             double eta, const double* delta, float* feats, float* targets, void* stream) {
    g_err.clear();
    if (!s || !rhs || !e_ref || !omega || !delta || !feats || !targets) return fail(SGW_EINVAL, "NULL argument");
    if (npairs <= 0) return SGW_OK;
    if (!is_device_ptr(rhs) || !is_device_ptr(feats) || !is_device_ptr(targets))
        return fail(SGW_EINVAL, "training rows take device buffers");
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_training_rows");
    cudaStream_t st = (cudaStream_t)stream;
    Carve c;
    const size_t o_e = c.take(sizeof(double) * npairs), o_o = c.take(sizeof(double) * npairs),
                 o_d = c.take(sizeof(double) * npairs);
    sgw_status r;
    if ((r = ensure_ws(s, c.off)) != SGW_OK) return r;
    char* w = (char*)s->d_ws;
    SGW_CUDA(cudaMemcpyAsync(w + o_e, e_ref, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_o, omega, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_d, delta, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    TrainRowsArgs a;
    a.n = npairs;
    a.rhs = (const double2*)rhs;
    a.e_ref = (const double*)(w + o_e);
    a.omega = (const double*)(w + o_o);
    a.delta = (const double*)(w + o_d);
    a.eta = eta;
    a.half_ecut = 0.5 * s->ecut;
    a.v_mean = s->v_mean;
    a.feats = feats;
    a.targets = targets;
    SGW_CUDA(launch_training_rows(s->plan, a, st), "training rows kernel");
    SGW_CUDA(cudaStreamSynchronize(st), "training rows");
    return SGW_OK;
}

sgw_status sgw_solve_pershift(sgw_system* s, int npairs, const void* rhs, const double* e_ref, const double* omega,
                              double eta, double tol, int precond, const double* delta, const sgw_mlp* mlp,
                              const sgw_solve_opts* opts, void* x, sgw_report* report) {
    g_err.clear();
    if (!s || !rhs || !e_ref || !omega || !x) return fail(SGW_EINVAL, "NULL argument");
    if (npairs < 0) return fail(SGW_EINVAL, "negative npairs");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(SGW_EINVAL, "eta must be positive");
    if (!(tol > 0.0)) return fail(SGW_EINVAL, "tol must be positive");
    {
        const sgw_status pr = check_precond(precond, delta, npairs, mlp);
        if (pr != SGW_OK) return pr;
    }
    if (!finite_all(e_ref, npairs) || !finite_all(omega, npairs)) return fail(SGW_EINVAL, "non-finite e_ref or omega");
    if (s->nocc == 0) return fail(SGW_ESTATE, "sgw_set_occupied has not been called");
    if (npairs == 0) return SGW_OK;
    const int ell = opts && opts->ell ? opts->ell : 4;
    if (ell < 1 || ell > kMaxEll) return fail(SGW_EINVAL, "ell must be 1..4");
    const int max_mv = opts && opts->max_matvec > 0 ? opts->max_matvec : 40000;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_solve_pershift");
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    Staged in, out;
    sgw_status r;
    if ((r = stage_in(rhs, vb * npairs, in, st, "rhs")) != SGW_OK) return r;
    if ((r = stage_out(x, vb * npairs, out, "x", st)) != SGW_OK) return r;
    int grid = 0, grid_r = 0;
    SGW_CUDA(solve_grid(s->plan, 1, npairs, &grid), "solver occupancy");
    SGW_CUDA(residual_owners(s->plan, SGW_PREC_FP64, &grid_r), "residual occupancy");
    grid_r = std::min(grid_r, npairs);
    Carve c;
    const size_t o_seed = c.take(vb * (2 * ell + 3) * grid);
    const size_t o_uw = c.take(vb * grid);
    const size_t o_pscr = c.take(2 * vb * grid);
    const size_t o_pre = c.take(sizeof(double) * s->npw * (size_t)npairs);
    const size_t o_z = c.take(sizeof(double) * npairs);
    const size_t o_e = c.take(sizeof(double) * npairs);
    const size_t o_o = c.take(sizeof(double) * npairs);
    const size_t o_dl = c.take(sizeof(double) * npairs);
    const size_t o_zero = c.take(sizeof(double));
    const size_t o_cnt = c.take(sizeof(int));
    const size_t o_mv = c.take(sizeof(int) * npairs);
    const size_t o_est = c.take(sizeof(double) * npairs);
    const size_t o_st = c.take(sizeof(int) * npairs);
    const size_t o_rscr = c.take(2 * vb * grid_r);
    const size_t o_rel = c.take(sizeof(double) * npairs);
    const size_t o_cert = c.take(sizeof(double) * npairs);
    if ((r = ensure_ws(s, c.off)) != SGW_OK) return r;
    char* w = (char*)s->d_ws;
    std::vector<double> zre(npairs);
    for (int i = 0; i < npairs; ++i) zre[i] = e_ref[i] + omega[i];
    SGW_CUDA(cudaMemcpyAsync(w + o_z, zre.data(), sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_e, e_ref, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    SGW_CUDA(cudaMemcpyAsync(w + o_o, omega, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    SGW_CUDA(cudaMemsetAsync(w + o_zero, 0, sizeof(double), st), "memset");
    if (delta) SGW_CUDA(cudaMemcpyAsync(w + o_dl, delta, sizeof(double) * npairs, cudaMemcpyHostToDevice, st), "copy");
    int launches = 0;
    if (precond != SGW_PRECOND_NONE) {
        if ((r = precond_common(s, npairs, (const double2*)in.dev, (const double*)(w + o_e), (const double*)(w + o_o),
                                delta ? (const double*)(w + o_dl) : nullptr, eta, precond, mlp, (double*)(w + o_pre),
                                st)) != SGW_OK)
            return r;
        ++launches;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool timed = report && report->kernel_ms;
    if (timed) {
        SGW_CUDA(cudaEventCreate(&ev0), "event");
        SGW_CUDA(cudaEventCreate(&ev1), "event");
        SGW_CUDA(cudaEventRecord(ev0, st), "event");
    }
    SolveArgs A;
    A.nrhs = npairs;
    A.nshift = 1;
    A.ell = ell;
    A.max_mv = max_mv;
    A.rhs = (const double2*)in.dev;
    A.e_ref = (const double*)(w + o_z);
    A.sig = (const double*)(w + o_zero);
    A.omega_seed = 0.0;
    A.eta = eta;
    A.tol = tol;
    A.x = (double2*)out.dev;
    A.uw = (double2*)(w + o_uw);
    A.seedw = (double2*)(w + o_seed);
    A.counter = (int*)(w + o_cnt);
    A.out_mv = (int*)(w + o_mv);
    A.out_res = (double*)(w + o_est);
    A.out_status = (int*)(w + o_st);
    A.pre = precond != SGW_PRECOND_NONE ? (const double*)(w + o_pre) : nullptr;
    A.pscr = (double2*)(w + o_pscr);
    SGW_CUDA(launch_solve(s->plan, A, grid, st), "per-shift solver");
    ++launches;
    if (timed) SGW_CUDA(cudaEventRecord(ev1, st), "event");
    SGW_CUDA(launch_residual(s->plan, npairs, 1, nullptr, 0, (const double2*)in.dev, (const double*)(w + o_z),
                             (const double*)(w + o_zero), eta, (const double2*)out.dev, (double2*)(w + o_rscr),
                             (double*)(w + o_rel), (double*)(w + o_cert), nullptr, grid_r, st),
             "residual kernel");
    ++launches;
    if ((r = finish_out(out, st, "x copy")) != SGW_OK) return r;
    std::vector<int> stv(npairs), mvv(npairs);
    std::vector<double> estv(npairs), relv(npairs), certv(npairs);
    SGW_CUDA(cudaMemcpyAsync(stv.data(), w + o_st, sizeof(int) * npairs, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(mvv.data(), w + o_mv, sizeof(int) * npairs, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(estv.data(), w + o_est, sizeof(double) * npairs, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(relv.data(), w + o_rel, sizeof(double) * npairs, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaMemcpyAsync(certv.data(), w + o_cert, sizeof(double) * npairs, cudaMemcpyDeviceToHost, st), "report");
    SGW_CUDA(cudaStreamSynchronize(st), "per-shift solve");
    bool all = true;
    for (int i = 0; i < npairs; ++i) {
        if (relv[i] <= tol) stv[i] = SGW_PAIR_CONVERGED;
        else if (stv[i] == SGW_PAIR_CONVERGED) stv[i] = SGW_PAIR_MAXITER;
        all = all && stv[i] == SGW_PAIR_CONVERGED;
    }
    if (report) {
        if (report->status) std::memcpy(report->status, stv.data(), sizeof(int) * npairs);
        if (report->matvecs) std::memcpy(report->matvecs, mvv.data(), sizeof(int) * npairs);
        if (report->est_res) std::memcpy(report->est_res, estv.data(), sizeof(double) * npairs);
        if (report->rel_res) std::memcpy(report->rel_res, relv.data(), sizeof(double) * npairs);
        if (report->cert) std::memcpy(report->cert, certv.data(), sizeof(double) * npairs);
        if (report->launches) *report->launches = launches;
        if (timed) {
            float ms = 0.f;
            SGW_CUDA(cudaEventElapsedTime(&ms, ev0, ev1), "event");
            *report->kernel_ms = ms;
        }
    }
    if (timed) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    if (!all) return fail(SGW_ENOCONV, "some pairs did not reach the tolerance");
    return SGW_OK;
}

sgw_status sgw_residual(sgw_system* s, int nrhs, const void* rhs, const double* e_ref, int nomega, const double* omega,
                        double eta, const void* dpsi, double* rel_res, double* cert, void* stream) {
    g_err.clear();
    if (!s || !rhs || !e_ref || !omega || !dpsi) return fail(SGW_EINVAL, "NULL argument");
    if (nrhs < 0 || nomega < 0) return fail(SGW_EINVAL, "negative size");
    if (!(eta > 0.0)) return fail(SGW_EINVAL, "eta must be positive");
    if (s->nocc == 0) return fail(SGW_ESTATE, "sgw_set_occupied has not been called");
    const size_t np = (size_t)nrhs * nomega;
    if (np == 0) return SGW_OK;
    DeviceScope dscope(s->dev);
    SGW_CUDA(dscope.err, "cudaSetDevice");
    Trace trace("sgw_residual");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vb = sizeof(double2) * (size_t)s->npw;
    Staged in_r, in_x;
    sgw_status r;
    if ((r = stage_in(rhs, vb * nrhs, in_r, st, "rhs")) != SGW_OK) return r;
    if ((r = stage_in(dpsi, vb * np, in_x, st, "dpsi")) != SGW_OK) return r;
    int grid = 0;
    SGW_CUDA(residual_owners(s->plan, SGW_PREC_FP64, &grid), "residual occupancy");
    grid = (int)std::min<size_t>(grid, np);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t off_er = al(2 * vb * grid);
    const size_t off_om = off_er + al(sizeof(double) * nrhs);
    const size_t off_rel = off_om + al(sizeof(double) * nomega);
    const size_t off_cert = off_rel + al(sizeof(double) * np);
    const size_t total = off_cert + al(sizeof(double) * np);
    if ((r = ensure_ws(s, total)) != SGW_OK) return r;
    char* w = (char*)s->d_ws;
    SGW_CUDA(cudaMemcpyAsync(w + off_er, e_ref, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st), "e_ref copy");
    SGW_CUDA(cudaMemcpyAsync(w + off_om, omega, sizeof(double) * nomega, cudaMemcpyHostToDevice, st), "omega copy");
    SGW_CUDA(launch_residual(s->plan, nrhs, nomega, nullptr, 0, (const double2*)in_r.dev, (const double*)(w + off_er),
                             (const double*)(w + off_om), eta, (const double2*)in_x.dev, (double2*)w,
                             (double*)(w + off_rel), (double*)(w + off_cert), nullptr, grid, st),
             "residual kernel");
    std::vector<double> relv(np), certv(np);
    SGW_CUDA(cudaMemcpyAsync(relv.data(), w + off_rel, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "copy");
    SGW_CUDA(cudaMemcpyAsync(certv.data(), w + off_cert, sizeof(double) * np, cudaMemcpyDeviceToHost, st), "copy");
    SGW_CUDA(cudaStreamSynchronize(st), "residual");
    if (rel_res) std::memcpy(rel_res, relv.data(), sizeof(double) * np);
    if (cert) std::memcpy(cert, certv.data(), sizeof(double) * np);
    return SGW_OK;
}

void sgw_destroy_system(sgw_system* s) {
    if (!s) return;
    DeviceScope dscope(s->dev);
    cudaDeviceSynchronize();
    free_system(s);
}

}  // extern "C"
