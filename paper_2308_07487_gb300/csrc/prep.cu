// Operand preparation for the fused contraction (HBM-bound, once per call).
//
// The paper rebuilds its N x 3M GEMM operand from the trajectory at every time step
// and centres it while doing so (Section 3.2, Eq. 5).  Here the trajectory row of
// site i, traj[i][s][f][a], is already K-contiguous, so the operand for
// displacement t is the K-offset window that starts at element s*3F + 3t of that row.
// A TMA copy must start on a 16-byte boundary, so the row is stored in 16/elem_bytes
// shifted copies (copy c holds row[x + c] at x); the window then starts at
// x = s*3F + 3t - c in the copy with c = (s*3F + 3t) mod (16/elem_bytes).
//
// B (the t0 frames) is stored once, zero-padded per sample to Kseg = roundup(3*T0, BK)
// so that the extra columns of every A window meet zeros.  With center = 1, B is
// centred by the per-site mean over (s, t0 < T0); centring A as well would subtract a
// constant per (i, t) that multiplies sum_{s,t0}(B - mean B) = 0, so Eq. 5 and Eq. 4
// are reached with B alone.
//
// Precision forms: BF16 hi = RN(x); split-BF16 lo = RN(x - hi); TF32 = RNA to 10-bit
// mantissa (the tensor core would otherwise truncate); FP32 keeps B in FP32.
#include <cuda_bf16.h>

#include "asd_internal.h"

namespace asd {
namespace {

__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// mean over (s, t0 < T0) of each component, one warp per site
__global__ void means_kernel(const float *__restrict__ traj, int64_t N, int S, int F, int T0,
                             float *__restrict__ mean)
{
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    double acc[3] = {0, 0, 0};
    for (int s = 0; s < S; ++s) {
        const float *row = traj + ((i * S + s) * (int64_t)F) * 3;
        for (int k = lane; k < 3 * T0; k += 32) acc[k % 3] += row[k];
    }
    // each lane holds partial sums per component; reduce each over the warp
    for (int a = 0; a < 3; ++a) {
        double v = acc[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[a] = v;
    }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) mean[3 * i + a] = (float)(acc[a] / ((double)S * T0));
}

// B operand: [N][S*Kseg], 8 consecutive k per thread
template <int FORM>
__global__ void prep_b_kernel(const float *__restrict__ traj, int64_t N, int S, int F, int T0,
                              int Kseg, const float *__restrict__ mean, int center, void *out0,
                              void *out1)
{
    const int64_t chunks_per_row = (int64_t)S * Kseg / 8;
    const int64_t total = N * chunks_per_row;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = g / chunks_per_row;
        const int64_t kk = (g % chunks_per_row) * 8;
        const int s = (int)(kk / Kseg);
        const int k0 = (int)(kk % Kseg);
        const float *row = traj + ((j * S + s) * (int64_t)F) * 3;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            float x = 0.f;
            if (k < 3 * T0) {
                x = row[k];
                if (center) x -= mean[3 * j + k % 3];
            }
            v[u] = x;
        }
        const int64_t off = j * (int64_t)S * Kseg + kk;
        if (FORM == ASD_FP32 || FORM == ASD_TF32) {
            float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(out0) + off);
            if (FORM == ASD_TF32)
                for (int u = 0; u < 8; ++u) v[u] = tf32_round(v[u]);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                hi[u] = __float2bfloat16_rn(v[u]);
                lo[u] = __float2bfloat16_rn(v[u] - __bfloat162float(hi[u]));
            }
            *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out0) + off) =
                *reinterpret_cast<uint4 *>(hi);
            if (FORM == ASD_SPLIT_BF16)
                *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out1) + off) =
                    *reinterpret_cast<uint4 *>(lo);
        }
    }
}

struct CopyPtrs {
    void *p[2][kMaxCopies];
};

// A operand copies: copy c, row i, elements x..x+V-1 (V = 16 / elem_bytes)
template <int FORM>
__global__ void prep_a_kernel(const float *__restrict__ traj, int64_t row_begin, int64_t row_end,
                              int64_t R, int64_t Rpad, CopyPtrs cp)
{
    constexpr int V = (FORM == ASD_TF32) ? 4 : 8;  // elements per 16-byte store = copies
    const int64_t chunks = Rpad / V;
    const int64_t total = (row_end - row_begin) * chunks;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = row_begin + g / chunks;
        const int64_t x0 = (g % chunks) * V;
        const float *row = traj + i * R;
        float w[2 * V];
#pragma unroll
        for (int u = 0; u < 2 * V - 1; ++u) {
            const int64_t x = x0 + u;
            w[u] = x < R ? __ldg(row + x) : 0.f;
        }
        const int64_t off = i * Rpad + x0;
#pragma unroll
        for (int c = 0; c < V; ++c) {
            if (FORM == ASD_TF32) {
                float4 o = make_float4(tf32_round(w[c]), tf32_round(w[c + 1]), tf32_round(w[c + 2]),
                                       tf32_round(w[c + 3]));
                *reinterpret_cast<float4 *>(static_cast<float *>(cp.p[0][c]) + off) = o;
            } else {
                __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    hi[u] = __float2bfloat16_rn(w[c + u]);
                    lo[u] = __float2bfloat16_rn(w[c + u] - __bfloat162float(hi[u]));
                }
                *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(cp.p[0][c]) + off) =
                    *reinterpret_cast<uint4 *>(hi);
                if (FORM == ASD_SPLIT_BF16)
                    *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(cp.p[1][c]) + off) =
                        *reinterpret_cast<uint4 *>(lo);
            }
        }
    }
}

unsigned grid_for(int64_t work, int sm_count)
{
    int64_t b = (work + 255) / 256;
    int64_t cap = (int64_t)sm_count * 16;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

int launch_prep(asd_corr_plan *p, const float *traj, int64_t row_begin, int64_t row_end,
                cudaStream_t s)
{
    const int T0 = p->T0, F = p->F, S = p->S;
    if (p->center) {
        means_kernel<<<(unsigned)((p->N + 7) / 8), 256, 0, s>>>(traj, p->N, S, F, T0, p->meanB);
        ASD_CUDA_TRY(cudaGetLastError());
    }
    const int64_t bwork = p->N * p->Kb / 8;
    const unsigned gb = grid_for(bwork, p->sm_count);
    switch (p->prec) {
    case ASD_FP32:
        prep_b_kernel<ASD_FP32><<<gb, 256, 0, s>>>(traj, p->N, S, F, T0, (int)p->Kseg, p->meanB,
                                                   p->center, p->Bf32, nullptr);
        break;
    case ASD_TF32:
        prep_b_kernel<ASD_TF32><<<gb, 256, 0, s>>>(traj, p->N, S, F, T0, (int)p->Kseg, p->meanB,
                                                   p->center, p->B[0], nullptr);
        break;
    case ASD_BF16:
        prep_b_kernel<ASD_BF16><<<gb, 256, 0, s>>>(traj, p->N, S, F, T0, (int)p->Kseg, p->meanB,
                                                   p->center, p->B[0], nullptr);
        break;
    default:
        prep_b_kernel<ASD_SPLIT_BF16><<<gb, 256, 0, s>>>(traj, p->N, S, F, T0, (int)p->Kseg,
                                                         p->meanB, p->center, p->B[0], p->B[1]);
        break;
    }
    ASD_CUDA_TRY(cudaGetLastError());
    if (!p->tc) return ASD_OK;
    CopyPtrs cp{};
    for (int pl = 0; pl < p->n_planes; ++pl)
        for (int c = 0; c < p->n_copies; ++c) cp.p[pl][c] = p->A[pl][c];
    const int V = p->prec == ASD_TF32 ? 4 : 8;
    const int64_t awork = (row_end - row_begin) * (p->Rpad / V);
    const unsigned ga = grid_for(awork, p->sm_count);
    if (p->prec == ASD_TF32)
        prep_a_kernel<ASD_TF32><<<ga, 256, 0, s>>>(traj, row_begin, row_end, p->R, p->Rpad, cp);
    else if (p->prec == ASD_BF16)
        prep_a_kernel<ASD_BF16><<<ga, 256, 0, s>>>(traj, row_begin, row_end, p->R, p->Rpad, cp);
    else
        prep_a_kernel<ASD_SPLIT_BF16><<<ga, 256, 0, s>>>(traj, row_begin, row_end, p->R, p->Rpad,
                                                         cp);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // namespace asd
