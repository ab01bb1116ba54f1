// Device-side distance rule shared by the pair-count, SIMT and tcgen05 kernels.
//
// bin(i,j) = max{k >= 0 : (k*w)^2 <= d2(i,j)} (distance bins of C(r - r', t), Eq. 4),
// evaluated exactly against a host-built table thr[k] = (k*w)^2 rounded UP to FP32:
// for an FP32 value d2,  d2 >= (k*w)^2  <=>  d2 >= thr[k].  The first guess comes from
// a fast reciprocal square root; one step each way fixes it.
#pragma once

#include <cuda_runtime.h>

namespace asd {

// Squared minimum-image distance of two lattice sites (exact integer).
__device__ __forceinline__ int lattice_d2i(int4 a, int4 b, int Lx, int Ly, int Lz, int periodic)
{
    int dx = abs(b.x - a.x), dy = abs(b.y - a.y), dz = abs(b.z - a.z);
    if (periodic) {
        dx = min(dx, Lx - dx);
        dy = min(dy, Ly - dy);
        dz = min(dz, Lz - dz);
    }
    return dx * dx + dy * dy + dz * dz;
}

// The same as a float (exact: lattice d2 stays far below 2^24).
__device__ __forceinline__ float lattice_d2(int4 a, int4 b, int Lx, int Ly, int Lz, int periodic)
{
    return (float)lattice_d2i(a, b, Lx, Ly, Lz, periodic);
}

// FP32 positions rule: dx = x_j - x_i, d2 = fma(dz,dz, fma(dy,dy, dx*dx)), no contraction.
__device__ __forceinline__ float position_d2(float4 a, float4 b)
{
    float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y), dz = __fsub_rn(b.z, a.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Exact bin from d2; returns a value in [0, n_bins+1]; >= n_bins means "dropped".
// thr must hold n_bins+2 entries (thr[0] = 0).
__device__ __forceinline__ int bin_of_d2(float d2, float inv_w, int n_bins, const float *thr)
{
    float r = d2 * rsqrtf(fmaxf(d2, 1e-30f));
    int k = min((int)(r * inv_w), n_bins);
    k += (d2 >= thr[k + 1]) ? 1 : 0;
    k -= (d2 < thr[k]) ? 1 : 0;
    return k;
}

}  // namespace asd
