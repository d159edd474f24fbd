// Training and inference kernels of the learned diagonal preconditioner, and their C ABI.
//
// Training: mean squared error of f(phi) against per-plane-wave targets, full-batch or
// mini-batch gradients, Adam on FP32 master weights; the forward and backward passes use
// the bf16-rounded weights with FP32 accumulation (the precision inference uses).
//
// Gradient kernel: each CTA takes tiles of 128 rows.  Per row (one thread): the forward
// pass stores a1, h1 = gelu(a1), a2 in shared memory; the backward pass turns them into
// da2 = dy w3 gelu'(a2) and da1 = (W2^T da2) gelu'(a1).  Per parameter (threads stride the
// 4545 entries): dW2[o][i] = sum_rows da2[o] h1[i] and the other sums over the tile.  Each
// CTA accumulates over its tiles and writes one partial; a second kernel sums the partials
// and applies Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mlp.cuh"
#include "sgw.h"
#include "sgw_internal.cuh"

namespace sgw {
sgw_status noalloc_fail(sgw_status s, const char* msg);
}

using namespace sgw;

struct sgw_mlp {
    int dev = 0;
    float* d_master = nullptr;          // FP32 master weights
    __nv_bfloat16* d_w = nullptr;       // bf16 copy used by every forward pass
    float* d_m = nullptr;               // Adam moments
    float* d_v = nullptr;
    float* d_partial = nullptr;         // [grid][kMlpParams + 1] gradient (+ loss) partials
    float* d_grad = nullptr;            // [kMlpParams + 1] summed gradient (+ loss)
    int grid = 0;
    int step = 0;
};

namespace {

constexpr int kTile = 128;
constexpr int kGradThreads = 256;
constexpr int kLd = kMlpH + 1;   // odd row stride of the per-row activations (one row per thread)

__global__ void round_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ w, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = __float2bfloat16_rn(master[i]);
}

__global__ void __launch_bounds__(kGradThreads) mlp_grad_kernel(const __nv_bfloat16* __restrict__ wq, int n,
                                                                const float* __restrict__ feats,
                                                                const float* __restrict__ targets,
                                                                const float* __restrict__ weight, float inv_n,
                                                                float* __restrict__ partial) {
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                                   // kMlpParams (rounded weights as float)
    float* A1 = w + ((kMlpParams + 3) & ~3);         // [kTile][kLd] a1 -> da1
    float* H1 = A1 + kTile * kLd;                    // [kTile][kLd] h1
    float* A2 = H1 + kTile * kLd;                    // [kTile][kLd] a2 -> da2
    float* H2 = A2 + kTile * kLd;                    // [kTile][kLd] h2
    float* X = H2 + kTile * kLd;                     // [kTile][4]
    float* DY = X + kTile * kMlpIn;                  // [kTile]
    const int tid = threadIdx.x;
    for (int i = tid; i < kMlpParams; i += blockDim.x) w[i] = __bfloat162float(wq[i]);
    // per-thread gradient accumulators for the parameters it owns (strided)
    constexpr int kOwn = (kMlpParams + kGradThreads - 1) / kGradThreads;   // 18
    float g[kOwn];
#pragma unroll
    for (int k = 0; k < kOwn; ++k) g[k] = 0.f;
    float loss = 0.f;
    __syncthreads();
    for (int t0 = blockIdx.x * kTile; t0 < n; t0 += gridDim.x * kTile) {
        const int nr = min(kTile, n - t0);
        // forward + output error, one row per thread
        for (int r = tid; r < kTile; r += blockDim.x) {
            float* a1 = A1 + r * kLd;
            float* h1 = H1 + r * kLd;
            float* a2 = A2 + r * kLd;
            float* h2 = H2 + r * kLd;
            if (r >= nr) {
                for (int o = 0; o < kMlpH; ++o) a1[o] = h1[o] = a2[o] = h2[o] = 0.f;
                for (int i = 0; i < kMlpIn; ++i) X[r * kMlpIn + i] = 0.f;
                DY[r] = 0.f;
                continue;
            }
            float x[kMlpIn];
            for (int i = 0; i < kMlpIn; ++i) x[i] = X[r * kMlpIn + i] = feats[(size_t)(t0 + r) * kMlpIn + i];
            for (int o = 0; o < kMlpH; ++o) {
                float a = w[kOffB1 + o];
                for (int i = 0; i < kMlpIn; ++i) a = fmaf(w[kOffW1 + o * kMlpIn + i], x[i], a);
                a1[o] = a;
                h1[o] = gelu_f(a);
            }
            float y = w[kOffB3];
            for (int o = 0; o < kMlpH; ++o) {
                float a = w[kOffB2 + o];
                for (int i = 0; i < kMlpH; ++i) a = fmaf(w[kOffW2 + o * kMlpH + i], h1[i], a);
                a2[o] = a;
                h2[o] = gelu_f(a);
                y = fmaf(w[kOffW3 + o], h2[o], y);
            }
            const float wr = weight ? weight[t0 + r] : 1.f;
            const float res = y - targets[t0 + r];
            loss += wr * res * res;
            const float dy = 2.f * inv_n * wr * res;
            DY[r] = dy;
            // backward through layer 2 and layer 1 (in place)
            for (int o = 0; o < kMlpH; ++o) a2[o] = dy * w[kOffW3 + o] * gelu_grad_f(a2[o]);
            for (int i = 0; i < kMlpH; ++i) {
                float d = 0.f;
                for (int o = 0; o < kMlpH; ++o) d = fmaf(w[kOffW2 + o * kMlpH + i], a2[o], d);
                a1[i] = d * gelu_grad_f(a1[i]);
            }
        }
        __syncthreads();
        // parameter gradients summed over the tile
#pragma unroll
        for (int k = 0; k < kOwn; ++k) {
            const int p = tid + k * kGradThreads;
            if (p >= kMlpParams) break;
            float s = 0.f;
            if (p < kOffB1) {
                const int o = p / kMlpIn, i = p % kMlpIn;
                for (int r = 0; r < kTile; ++r) s = fmaf(A1[r * kLd + o], X[r * kMlpIn + i], s);
            } else if (p < kOffW2) {
                const int o = p - kOffB1;
                for (int r = 0; r < kTile; ++r) s += A1[r * kLd + o];
            } else if (p < kOffB2) {
                const int o = (p - kOffW2) / kMlpH, i = (p - kOffW2) % kMlpH;
                for (int r = 0; r < kTile; ++r) s = fmaf(A2[r * kLd + o], H1[r * kLd + i], s);
            } else if (p < kOffW3) {
                const int o = p - kOffB2;
                for (int r = 0; r < kTile; ++r) s += A2[r * kLd + o];
            } else if (p < kOffB3) {
                const int o = p - kOffW3;
                for (int r = 0; r < kTile; ++r) s = fmaf(DY[r], H2[r * kLd + o], s);
            } else {
                for (int r = 0; r < kTile; ++r) s += DY[r];
            }
            g[k] += s;
        }
        __syncthreads();
    }
    float* out = partial + (size_t)blockIdx.x * (kMlpParams + 1);
#pragma unroll
    for (int k = 0; k < kOwn; ++k) {
        const int p = tid + k * kGradThreads;
        if (p < kMlpParams) out[p] = g[k];
    }
    // loss partial: block reduction
    __shared__ float red[kGradThreads / 32];
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0) red[tid >> 5] = loss;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int i = 0; i < kGradThreads / 32; ++i) s += red[i];
        out[kMlpParams] = s * inv_n;
    }
}

// Sums the partial gradients; optionally applies Adam and refreshes the bf16 weights.
__global__ void mlp_reduce_adam_kernel(const float* __restrict__ partial, int grid, float* __restrict__ grad_out,
                                       float* master, float* m, float* v, __nv_bfloat16* wq, int adam, float lr,
                                       float b1t, float b2t) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    float s = 0.f;
    for (int c = 0; c < grid; ++c) s += partial[(size_t)c * (kMlpParams + 1) + p];
    if (grad_out) grad_out[p] = s;
    if (!adam || p == kMlpParams) return;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const float mm = beta1 * m[p] + (1.f - beta1) * s;
    const float vv = beta2 * v[p] + (1.f - beta2) * s * s;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.f - b1t), vh = vv / (1.f - b2t);
    const float th = master[p] - lr * mh / (sqrtf(vh) + eps);
    master[p] = th;
    wq[p] = __float2bfloat16_rn(th);
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const __nv_bfloat16* __restrict__ wq, int n,
                                                          const float* __restrict__ feats, float* __restrict__ out) {
    __shared__ float w[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = __bfloat162float(wq[i]);
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        float x[kMlpIn];
        for (int i = 0; i < kMlpIn; ++i) x[i] = feats[(size_t)r * kMlpIn + i];
        out[r] = mlp_eval(w, x);
    }
}

int grad_smem() { return (((kMlpParams + 3) & ~3) + 4 * kTile * kLd + kTile * kMlpIn + kTile) * 4; }

thread_local std::string g_mlp_err;

sgw_status mfail(sgw_status s, const std::string& msg) {
    noalloc_fail(s, msg.c_str());
    return s;
}

#define MLP_CUDA(call, what)                                                                           \
    do {                                                                                               \
        cudaError_t e__ = (call);                                                                      \
        if (e__ != cudaSuccess)                                                                        \
            return mfail(e__ == cudaErrorMemoryAllocation ? SGW_ENOMEM : SGW_ECUDA,                    \
                         std::string(what) + ": " + cudaGetErrorString(e__));                          \
    } while (0)

}  // namespace

namespace sgw {
const __nv_bfloat16* mlp_weights(const sgw_mlp* m) { return m ? m->d_w : nullptr; }
}  // namespace sgw

extern "C" {

sgw_status sgw_mlp_create(const float* params, sgw_mlp** out) {
    if (!params || !out) return mfail(SGW_EINVAL, "NULL argument");
    *out = nullptr;
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(params[i])) return mfail(SGW_EINVAL, "non-finite parameter");
    sgw_mlp* m = new sgw_mlp();
    MLP_CUDA(cudaGetDevice(&m->dev), "cudaGetDevice");
    int nsm = 0;
    MLP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->dev), "attribute");
    m->grid = nsm;
    const size_t pb = sizeof(float) * kMlpParams;
    cudaError_t e = cudaMalloc(&m->d_master, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_w, sizeof(__nv_bfloat16) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_partial, sizeof(float) * (size_t)m->grid * (kMlpParams + 1));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_grad, sizeof(float) * (kMlpParams + 1));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_master, params, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, pb);
    if (e == cudaSuccess) {
        round_kernel<<<(kMlpParams + 255) / 256, 256>>>(m->d_master, m->d_w, kMlpParams);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)mlp_grad_kernel,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, grad_smem());
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sgw_mlp_destroy(m);
        return mfail(SGW_ECUDA, std::string("mlp create: ") + cudaGetErrorString(e));
    }
    *out = m;
    return SGW_OK;
}

sgw_status sgw_mlp_get_params(const sgw_mlp* m, float* params) {
    if (!m || !params) return mfail(SGW_EINVAL, "NULL argument");
    MLP_CUDA(cudaMemcpy(params, m->d_master, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost), "copy");
    return SGW_OK;
}

sgw_status sgw_mlp_forward(const sgw_mlp* m, int n, const float* feats, float* out, void* stream) {
    if (!m || (n > 0 && (!feats || !out))) return mfail(SGW_EINVAL, "NULL argument");
    if (n <= 0) return SGW_OK;
    mlp_forward_kernel<<<std::min((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(m->d_w, n, feats, out);
    MLP_CUDA(cudaGetLastError(), "forward kernel");
    return SGW_OK;
}

static sgw_status grad_common(sgw_mlp* m, int n, const float* feats, const float* targets, const float* weight,
                              float* grad, float* loss, int adam, float lr, void* stream) {
    if (!m || n <= 0 || !feats || !targets) return mfail(SGW_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = std::min(m->grid, (n + kTile - 1) / kTile);
    mlp_grad_kernel<<<grid, kGradThreads, grad_smem(), st>>>(m->d_w, n, feats, targets, weight, 1.0f / n,
                                                             m->d_partial);
    MLP_CUDA(cudaGetLastError(), "gradient kernel");
    float* d_grad = m->d_grad;
    std::vector<float> h(kMlpParams + 1);
    int t = m->step + (adam ? 1 : 0);
    const float b1t = adam ? (float)std::pow(0.9, t) : 0.f, b2t = adam ? (float)std::pow(0.999, t) : 0.f;
    mlp_reduce_adam_kernel<<<(kMlpParams + 256) / 256, 256, 0, st>>>(m->d_partial, grid, d_grad, m->d_master, m->d_m,
                                                                      m->d_v, m->d_w, adam, lr, b1t, b2t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_grad, sizeof(float) * (kMlpParams + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return mfail(SGW_ECUDA, std::string("reduce/adam: ") + cudaGetErrorString(e));
    if (adam) m->step = t;
    if (grad) std::memcpy(grad, h.data(), sizeof(float) * kMlpParams);
    if (loss) *loss = h[kMlpParams];
    return SGW_OK;
}

sgw_status sgw_mlp_grad(sgw_mlp* m, int n, const float* feats, const float* targets, const float* weight,
                        float* grad, float* loss, void* stream) {
    return grad_common(m, n, feats, targets, weight, grad, loss, 0, 0.f, stream);
}

sgw_status sgw_mlp_train_step(sgw_mlp* m, int n, const float* feats, const float* targets, const float* weight,
                              float lr, float* loss, void* stream) {
    if (!(lr > 0.f)) return mfail(SGW_EINVAL, "lr must be positive");
    return grad_common(m, n, feats, targets, weight, nullptr, loss, 1, lr, stream);
}

void sgw_mlp_destroy(sgw_mlp* m) {
    if (!m) return;
    cudaFree(m->d_master);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_w);
    cudaFree(m->d_partial);
    cudaFree(m->d_grad);
    delete m;
}

}  // extern "C"
