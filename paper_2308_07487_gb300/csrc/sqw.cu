// Dynamical structure factor S(q, omega) from S(q, t) (Section 4): the windowed cosine
// transform of the even extension S(q, -t) = S(q, t) of the displacement series,
//   S(q, w_k) = dt * ( v_0 S(q, 0) + 2 sum_{t=1}^{n_t-1} v_t S(q, t) cos(w_k t dt) ),
// with v_t = 1 (no window), 0.5 (1 + cos(pi t / n_t)) (Hann) or exp(-(t / (width n_t))^2 / 2)
// (Gaussian).  The cosine advances by a rotation per step, re-seeded from sincos every 32
// steps, in FP64.
#include <cuda_runtime.h>

#include "asd_internal.h"

namespace asd {
namespace {

constexpr int kMaxNt = 6000;  // window weights in shared memory (48 KB)

__global__ void sq_omega_kernel(const double *__restrict__ S, int n_t, int n_q, double dt,
                                int window, double width, const double *__restrict__ omega,
                                double *__restrict__ Sqw)
{
    extern __shared__ double v[];
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
        double w = 1.0;
        if (window == 1) w = 0.5 * (1.0 + cospi((double)t / n_t));
        else if (window == 2) {
            const double x = (double)t / (width * n_t);
            w = exp(-0.5 * x * x);
        }
        v[t] = w;
    }
    __syncthreads();
    const int k = blockIdx.x;
    const double th = omega[k] * dt;
    double sr, cr;
    sincos(th, &sr, &cr);  // rotation by one step
    for (int q = threadIdx.x; q < n_q; q += blockDim.x) {
        double acc = 0.0, c = 1.0, s = 0.0;
        for (int t = 1; t < n_t; ++t) {
            if ((t & 31) == 0) {
                sincos(th * t, &s, &c);
            } else {
                const double c2 = c * cr - s * sr;
                s = s * cr + c * sr;
                c = c2;
            }
            acc = fma(v[t] * S[(int64_t)t * n_q + q], c, acc);
        }
        Sqw[(int64_t)k * n_q + q] = dt * (v[0] * S[q] + 2.0 * acc);
    }
}

}  // namespace
}  // namespace asd

int asd_sq_omega(const double *S, int n_t, int n_q, double dt, int window, double width,
                 const double *omega, int n_w, double *Sqw, void *stream)
{
    using namespace asd;
    ASD_CHECK_ARG(S && omega && Sqw, "null argument");
    ASD_CHECK_ARG(n_t >= 1 && n_t <= kMaxNt, "n_t: 1..6000");
    ASD_CHECK_ARG(n_q >= 1 && n_w >= 1 && n_w <= 65535, "n_q >= 1, n_w in 1..65535");
    ASD_CHECK_ARG(dt > 0.0, "dt > 0");
    ASD_CHECK_ARG(window >= 0 && window <= 2, "window: 0 none, 1 Hann, 2 Gaussian");
    ASD_CHECK_ARG(window != 2 || width > 0.0, "Gaussian window needs width > 0");
    sq_omega_kernel<<<n_w, 128, sizeof(double) * n_t, (cudaStream_t)stream>>>(
        S, n_t, n_q, dt, window, width, omega, Sqw);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}
