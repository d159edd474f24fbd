// Learned diagonal preconditioner: a 4 -> 64 -> 64 -> 1 perceptron with erf-GELU
// activations.  Packed parameter layout (4545 floats):
//   w1 [64][4] @ 0, b1 [64] @ 256, w2 [64][64] @ 320, b2 [64] @ 4416, w3 [64] @ 4480, b3 @ 4544.
// Inference uses bf16-rounded weights with FP32 accumulation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sgw {

constexpr int kMlpIn = 4;
constexpr int kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;   // 4545
constexpr int kOffW1 = 0, kOffB1 = 256, kOffW2 = 320, kOffB2 = 4416, kOffW3 = 4480, kOffB3 = 4544;
constexpr double kOmegaScale = 2.205;   // Ha (60 eV): frequency feature scale

// x Phi(x) with Phi the standard normal distribution function, through CUDA's erff.
__device__ __forceinline__ float gelu_f(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
// d/dx [x Phi(x)] = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad_f(float a) {
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

// f(x) for one row; w = the packed parameters (FP32 copies of the bf16 weights).
__device__ __forceinline__ float mlp_eval(const float* w, const float (&x)[kMlpIn]) {
    float h1[kMlpH];
#pragma unroll
    for (int o = 0; o < kMlpH; ++o) {
        float a = w[kOffB1 + o];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) a = fmaf(w[kOffW1 + o * kMlpIn + i], x[i], a);
        h1[o] = gelu_f(a);
    }
    float y = w[kOffB3];
    for (int o = 0; o < kMlpH; ++o) {
        float a = w[kOffB2 + o];
#pragma unroll
        for (int i = 0; i < kMlpH; ++i) a = fmaf(w[kOffW2 + o * kMlpH + i], h1[i], a);
        y = fmaf(w[kOffW3 + o], gelu_f(a), y);
    }
    return y;
}

}  // namespace sgw
