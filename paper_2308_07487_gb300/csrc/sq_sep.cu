// Separable evaluation of the phase-weighted sum (the cosine part of Eq. 3 with the
// weights of Eq. 6).  cos(q.(r_i - r_j)) = cos(q.r_i) cos(q.r_j) + sin(q.r_i) sin(q.r_j)
// splits the pair sum into per-site transforms of every frame,
//   Fc(q; s, f, a) = sum_i cos(q.r_i) S_i(s, f, a),   Fs likewise with sin,
// and then
//   Sq_sum[t][q] = sum_{s, a, t0 < T0} Fc(s, t0 + t, a) Fc_B(s, t0, a) + Fs(...) Fs_B(...),
// where the B factors are the transforms of the (optionally centred) B operand: centring
// B per site subtracts its mean over (s, t0 < T0), which in the transform subtracts the
// same mean of Fc_B.  Cost O(N S F n_q) instead of O(N^2 S T0 n_t).
#include <cuda_runtime.h>

#include "asd_internal.h"

namespace asd {
namespace {

constexpr int kTM = 64;     // transform rows (cos / sin of 32 q) per block
constexpr int kTN = 128;    // trajectory columns per block
constexpr int kTS = 16;     // sites per shared-memory step
constexpr int kSlice = 4096;  // sites per block; slices are combined with FP64 atomics

// Fb[m][k] += sum_{i in this block's slice} W[i][m] X[i][k]:  W = the (cos, sin) table seen
// as [N][ldw] floats (m = 2q: cos, 2q + 1: sin), X = the trajectory [N][K].  FP32 inside
// a slice, FP64 across slices.
__global__ void __launch_bounds__(256) nudft_kernel(const float *__restrict__ W, int ldw, int M,
                                                    const float *__restrict__ X, int64_t K,
                                                    int64_t N, double *__restrict__ Fb)
{
    __shared__ float sw[kTS][kTM];
    __shared__ float sx[kTS][kTN];
    const int tid = threadIdx.x;
    const int tm = tid >> 5, tn = tid & 31;  // 8 rows x 4 columns per thread
    const int m0 = blockIdx.y * kTM;
    const int64_t k0 = (int64_t)blockIdx.x * kTN;
    const int64_t i0 = (int64_t)blockIdx.z * kSlice;
    const int64_t i1 = i0 + kSlice < N ? i0 + kSlice : N;
    float acc[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int64_t i = i0; i < i1; i += kTS) {
        for (int e = tid; e < kTS * kTM; e += 256) {
            const int r = e / kTM, c = e % kTM;
            const int64_t ii = i + r;
            sw[r][c] = (ii < i1 && m0 + c < ldw) ? W[ii * ldw + m0 + c] : 0.f;
        }
        for (int e = tid; e < kTS * kTN; e += 256) {
            const int r = e / kTN, c = e % kTN;
            const int64_t ii = i + r;
            sx[r][c] = (ii < i1 && k0 + c < K) ? X[ii * K + k0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kTS; ++r) {
            float a[8], b[4];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = sw[r][tm * 8 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = sx[r][tn + 32 * v];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int m = m0 + tm * 8 + u;
        if (m >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t k = k0 + tn + 32 * v;
            if (k < K) atomicAdd(&Fb[(int64_t)m * K + k], (double)acc[u][v]);
        }
    }
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// Sq_sum[t][q] += sum_{s, a, t0 < T0} Fc(s, t0 + t, a) (Fc(s, t0, a) - mc_a)
//              + Fs(s, t0 + t, a) (Fs(s, t0, a) - ms_a),
// mc_a / ms_a = the mean over (s, t0 < T0) when centring, else 0.  Block (q, t-group).
constexpr int kTPB = 8;  // displacements per block

__global__ void __launch_bounds__(256) sq_corr_kernel(const double *__restrict__ Fb, int64_t K,
                                                      int S, int F, int T0, int n_t, int center,
                                                      int n_q, int parts,
                                                      double *__restrict__ Sq_sum)
{
    __shared__ double red[8];
    const int q = blockIdx.x;
    const double *fc = Fb + (int64_t)(2 * q) * K;
    const double *fs = Fb + (int64_t)(2 * q + 1) * K;
    const int n_terms = S * T0 * 3;
    double mc[3] = {0.0, 0.0, 0.0}, ms[3] = {0.0, 0.0, 0.0};
    if (center) {
        for (int a = 0; a < 3; ++a) {
            double vc = 0.0, vs = 0.0;
            for (int e = threadIdx.x; e < S * T0; e += blockDim.x) {
                const int s = e / T0, t0 = e % T0;
                const int64_t k = ((int64_t)s * F + t0) * 3 + a;
                vc += fc[k];
                vs += fs[k];
            }
            mc[a] = block_sum(vc, red) / (double)(S * T0);
            ms[a] = block_sum(vs, red) / (double)(S * T0);
        }
    }
    const int tb = blockIdx.y * kTPB;
    for (int t = tb; t < tb + kTPB && t < n_t; ++t) {
        double v = 0.0, vs = 0.0;
        for (int e = threadIdx.x; e < n_terms; e += blockDim.x) {
            const int a = e % 3, st = e / 3;
            const int s = st / T0, t0 = st % T0;
            const int64_t kb = ((int64_t)s * F + t0) * 3 + a;
            const int64_t ka = kb + 3 * (int64_t)t;
            v = fma(fc[ka], fc[kb] - mc[a], v);
            v = fma(fs[ka], fs[kb] - ms[a], v);
            // sine part: sin(a - b) = sin a cos b - cos a sin b
            vs = fma(fs[ka], fc[kb] - mc[a], vs);
            vs = fma(-fc[ka], fs[kb] - ms[a], vs);
        }
        v = block_sum(v, red);
        if (threadIdx.x == 0) Sq_sum[((int64_t)t * n_q + q) * parts] += v;
        if (parts == 2) {
            vs = block_sum(vs, red);
            if (threadIdx.x == 0) Sq_sum[((int64_t)t * n_q + q) * 2 + 1] += vs;
        }
    }
}

}  // namespace
}  // namespace asd

int asd_pair_corr_sq_separable(asd_corr_plan *p, const float *traj, double *Sq_sum, void *stream)
{
    using namespace asd;
    ASD_CHECK_ARG(p && traj && Sq_sum, "null argument");
    ASD_CHECK_ARG(p->n_q > 0 && p->sqF, "plan has no q-vectors");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t K = (int64_t)p->S * 3 * p->F;
    const int nqp = (p->n_q + kQChunk - 1) / kQChunk * kQChunk;
    const int M = 2 * p->n_q;
    ASD_CUDA_TRY(cudaMemsetAsync(p->sqF, 0, sizeof(double) * (size_t)M * K, s));
    const int64_t slices = (p->N + kSlice - 1) / kSlice;
    ASD_CHECK_ARG(slices <= 65535, "too many sites for the separable transform");
    dim3 g1((unsigned)((K + kTN - 1) / kTN), (unsigned)((M + kTM - 1) / kTM), (unsigned)slices);
    nudft_kernel<<<g1, 256, 0, s>>>(reinterpret_cast<const float *>(p->cs), 2 * nqp, M, traj, K,
                                   p->N, p->sqF);
    ASD_CUDA_TRY(cudaGetLastError());
    dim3 g2((unsigned)p->n_q, (unsigned)((p->n_t + kTPB - 1) / kTPB), 1);
    sq_corr_kernel<<<g2, 256, 0, s>>>(p->sqF, K, p->S, p->F, p->T0, p->n_t, p->center, p->n_q,
                                      p->q_parts, Sq_sum);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}
