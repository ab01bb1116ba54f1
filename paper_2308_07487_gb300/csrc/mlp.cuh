// Learned von Mises-Fisher proposal network (device forward pass).
//
// x (the 3z neighbour spin components) -> h1 = tanh(W1 x + b1) -> h2 = tanh(W2 h1 + b2)
// [-> h3 = tanh(Wm h2 + bm) with three hidden layers] -> o = W3 h_last + b3;  mean
// direction mu = o[0:3] / |o[0:3]|,  kappa = softplus(o[3]).
// Weights are BF16 (row-major [out][in]), biases and all arithmetic FP32.
#pragma once

#include <cuda_bf16.h>

#include "../../include/asd.h"

namespace asd {

constexpr int kMlpHidden = 64;
constexpr int kMlpMaxIn = 24;
constexpr int kMlpMaxDepth = 3;   // hidden layers: 2 or 3

struct MlpView {
    int n_in;
    int depth;                       // hidden layers (2 or 3)
    const __nv_bfloat16 *W1, *W2, *Wm, *W3;
    const float *b1, *b2, *bm, *b3;
};

inline int mlp_depth(const asd_mlp &m) { return m.depth == 0 ? 2 : m.depth; }

inline MlpView mlp_view(const asd_mlp &m)
{
    MlpView v;
    v.n_in = m.n_in;
    v.depth = mlp_depth(m);
    v.W1 = reinterpret_cast<const __nv_bfloat16 *>(m.W1);
    v.W2 = reinterpret_cast<const __nv_bfloat16 *>(m.W2);
    v.Wm = reinterpret_cast<const __nv_bfloat16 *>(m.Wm);
    v.W3 = reinterpret_cast<const __nv_bfloat16 *>(m.W3);
    v.b1 = m.b1;
    v.b2 = m.b2;
    v.bm = m.bm;
    v.b3 = m.b3;
    return v;
}

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// Forward pass; also returns the pre-normalisation output o[4] and hidden activations
// when the pointers are non-null (used by the training kernels).
__device__ __forceinline__ void mlp_forward(const MlpView &n, const float *x, float *h1, float *h2,
                                            float *o)
{
    for (int k = 0; k < kMlpHidden; ++k) {
        float a = __ldg(n.b1 + k);
        for (int c = 0; c < n.n_in; ++c) a = fmaf(__bfloat162float(n.W1[k * n.n_in + c]), x[c], a);
        h1[k] = tanhf(a);
    }
    for (int k = 0; k < kMlpHidden; ++k) {
        float a = __ldg(n.b2 + k);
#pragma unroll 8
        for (int c = 0; c < kMlpHidden; ++c)
            a = fmaf(__bfloat162float(n.W2[k * kMlpHidden + c]), h1[c], a);
        h2[k] = tanhf(a);
    }
    if (n.depth == 3) {
        // the third hidden layer reads h2 and writes into h1's storage, then moves back
        for (int k = 0; k < kMlpHidden; ++k) {
            float a = __ldg(n.bm + k);
#pragma unroll 8
            for (int c = 0; c < kMlpHidden; ++c)
                a = fmaf(__bfloat162float(n.Wm[k * kMlpHidden + c]), h2[c], a);
            h1[k] = tanhf(a);
        }
        for (int k = 0; k < kMlpHidden; ++k) h2[k] = h1[k];
    }
    for (int k = 0; k < 4; ++k) {
        float a = __ldg(n.b3 + k);
#pragma unroll 8
        for (int c = 0; c < kMlpHidden; ++c)
            a = fmaf(__bfloat162float(n.W3[k * kMlpHidden + c]), h2[c], a);
        o[k] = a;
    }
}

__device__ __forceinline__ void mlp_vmf(const MlpView &n, const float *x, float *mu, float *kappa)
{
    float h1[kMlpHidden], h2[kMlpHidden], o[4];
    mlp_forward(n, x, h1, h2, o);
    const float inv = rsqrtf(fmaxf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2], 1e-30f));
    mu[0] = o[0] * inv;
    mu[1] = o[1] * inv;
    mu[2] = o[2] * inv;
    *kappa = softplus_f(o[3]) + 1e-4f;
}

}  // namespace asd
