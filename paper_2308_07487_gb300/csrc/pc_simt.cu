// FP32 form: the fused contraction + epilogue on the CUDA cores (FFMA).
//
// It is the accuracy and speed baseline of the tensor-core forms.  Each CTA owns a
// 128 x 128 tile of G_t = A_t B^T for one displacement t (the paper's thread-block
// tile, Section 3.3), accumulates it in registers (8 x 8 per thread), and reduces the
// tile in place: distance bins through FP32 shared-memory atomics into one copy of the
// bins per warp (summed across the warps in FP64 at the end of the tile; FP64 shared
// atomics where the copies do not fit), phase weights
// through cos(a-b) = cos a cos b + sin a sin b with warp shuffles (Section 3.3, the
// shuffle + shared-memory + atomic reduction), then one FP64 global atomic per bin
// (and per q) per tile.  In the deterministic mode the same sums are 64-bit fixed point
// (integer atomics, the same bits in any order).  A is read straight from the trajectory row at the K-offset
// s*3F + 3t; B is the prepared, zero-padded FP32 copy.
#include "asd_internal.h"
#include "geom.cuh"

namespace asd {
namespace {

constexpr int TM = 128, TN = 128, TK = 8;

struct SimtParams {
    const float *traj;
    const float *B;
    int64_t R;        // trajectory row length S*3F
    int F3;
    int K3;           // 3*T0
    int Kseg;         // B segment per sample
    int S;
    int N;
    int row_begin, row_end;
    int t_begin;      // displacement of grid slice blockIdx.z = 0
    int warp_bins;    // per-warp FP32 bin copies after the FP64 arrays
    EpiParams e;
    int *err;         // device error word (index checks of a checked build)
};

// (two CTAs per SM: at most 128 registers a thread)
__global__ void __launch_bounds__(256, 2) simt_kernel(SimtParams P)
{
    __shared__ __align__(16) float As[2][TK][TM];
    __shared__ __align__(16) float Bs[2][TK][TN];
    extern __shared__ double red[];  // [n_bins] then [n_q][q_parts], then [8][n_bins] FP32
    double *sbins = red;
    double *sq = red + P.e.n_bins;
    float *wbins = reinterpret_cast<float *>(sq + P.e.n_q * P.e.q_parts);
    // deterministic mode: the same arrays as fixed point
    long long *sbins_i = reinterpret_cast<long long *>(sbins);
    long long *sq_i = reinterpret_cast<long long *>(sq);
    const double fscale = P.e.fix_scale ? *P.e.fix_scale : 0.0;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int t = P.t_begin + blockIdx.z;
    const int m0 = P.row_begin + blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    for (int k = tid; k < P.e.n_bins + P.e.n_q * P.e.q_parts; k += 256) red[k] = 0.0;
    const bool wb_on = P.warp_bins && fscale == 0.0;
    if (wb_on)
        for (int k = tid; k < 8 * P.e.n_bins; k += 256) wbins[k] = 0.f;

    // loader mapping: one row (or column) and 4 consecutive k per thread
    const int lr = tid >> 1, lk = (tid & 1) * 4;
    const int li = m0 + lr, lj = n0 + lr;
    const bool a_ok = li < P.row_end;
    const bool b_ok = lj < P.N;
    const float *arow = P.traj + (int64_t)(a_ok ? li : 0) * P.R + 3 * t;
    const float *brow = P.B + (int64_t)(b_ok ? lj : 0) * P.S * P.Kseg;

    const int steps_per_seg = P.Kseg / TK;
    const int n_steps = P.S * steps_per_seg;
    float ra[4], rb[4];
    auto load = [&](int st) {
        const int s = st / steps_per_seg;
        const int kl = (st % steps_per_seg) * TK + lk;
        const float *ap = arow + (int64_t)s * P.F3 + kl;
#pragma unroll
        for (int u = 0; u < 4; ++u) ra[u] = (a_ok && kl + u < P.K3) ? __ldg(ap + u) : 0.f;
        float4 bv = b_ok ? __ldg(reinterpret_cast<const float4 *>(brow + (int64_t)s * P.Kseg + kl))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
        rb[0] = bv.x; rb[1] = bv.y; rb[2] = bv.z; rb[3] = bv.w;
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[buf][lk + u][lr] = ra[u];
            Bs[buf][lk + u][lr] = rb[u];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

    load(0);
    store(0);
    __syncthreads();
    for (int st = 0; st < n_steps; ++st) {
        const int buf = st & 1;
        if (st + 1 < n_steps) load(st + 1);
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[8], b[8];
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        if (st + 1 < n_steps) store(buf ^ 1);
        __syncthreads();
    }

    // ---------------- epilogue: reduce the tile ----------------
    int ri[8], cj[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        ri[u] = m0 + (u < 4 ? ty * 4 + u : 64 + ty * 4 + u - 4);
        cj[u] = n0 + (u < 4 ? tx * 4 + u : 64 + tx * 4 + u - 4);
    }
    const EpiParams &e = P.e;
    float *myb = wbins + (tid >> 5) * e.n_bins;
    if (e.n_bins > 0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const bool rok = ri[r] < P.row_end;
            const int ir = rok ? ri[r] : P.row_begin;
            const int4 ci = e.coords[ir];
            const float4 pi = e.pos[ir];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const bool ok = rok && cj[c] < P.N;
                const int jc = cj[c] < P.N ? cj[c] : 0;
                const float d2 = e.geom == ASD_GEOM_LATTICE
                                     ? lattice_d2(ci, e.coords[jc], e.Lx, e.Ly, e.Lz, e.periodic)
                                     : position_d2(pi, e.pos[jc]);
                const int b = bin_of_d2(d2, e.inv_w, e.n_bins, e.thr);
                if (ok && b < e.n_bins && ASD_INB(b >= 0, BND_SIMT_BIN, P.err)) {
                    if (fscale != 0.0) add_fixed(&sbins_i[b], to_fixed((double)acc[r][c], fscale));
                    else if (wb_on) atomicAdd(&myb[b], acc[r][c]);
                    else atomicAdd(&sbins[b], (double)acc[r][c]);
                }
            }
        }
    }
    if (e.n_q > 0) {
        const int lane = tid & 31;
        for (int q = 0; q < e.n_q; ++q) {
            float part = 0.f, part_s = 0.f;
            float2 wc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                wc[c] = cj[c] < P.N ? e.cs[(int64_t)cj[c] * e.nq_pad + q] : make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float2 wr = ri[r] < P.row_end ? e.cs[(int64_t)ri[r] * e.nq_pad + q]
                                                    : make_float2(0.f, 0.f);
                float u = 0.f, v = 0.f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    u = fmaf(wc[c].x, acc[r][c], u);
                    v = fmaf(wc[c].y, acc[r][c], v);
                }
                part = fmaf(wr.x, u, fmaf(wr.y, v, part));        // cos(a - b)
                part_s = fmaf(wr.y, u, fmaf(-wr.x, v, part_s));   // sin(a - b)
            }
            // the warp's 32 partial sums (64 pairs each) in FP32, one FP64 add per warp
            // (FP64 arithmetic runs on a narrow pipe on this part)
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            const bool qok = lane == 0 && ASD_INB(q < e.nq_pad, BND_SIMT_Q, P.err);
            if (qok) {
                if (fscale != 0.0) add_fixed(&sq_i[q * e.q_parts], to_fixed((double)part, fscale));
                else atomicAdd(&sq[q * e.q_parts], (double)part);
            }
            if (e.q_parts == 2) {
                for (int o = 16; o > 0; o >>= 1) part_s += __shfl_xor_sync(0xffffffffu, part_s, o);
                if (qok) {
                    if (fscale != 0.0) add_fixed(&sq_i[2 * q + 1], to_fixed((double)part_s, fscale));
                    else atomicAdd(&sq[2 * q + 1], (double)part_s);
                }
            }
        }
    }
    __syncthreads();
    if (fscale != 0.0) {
        for (int b = tid; b < e.n_bins; b += 256)
            if (sbins_i[b] != 0) add_fixed(&e.C_fix[(int64_t)t * e.n_bins + b], sbins_i[b]);
        for (int o = tid; o < e.n_q * e.q_parts; o += 256)
            if (sq_i[o] != 0) add_fixed(&e.Sq_fix[(int64_t)t * e.n_q * e.q_parts + o], sq_i[o]);
        return;
    }
    for (int b = tid; b < e.n_bins; b += 256) {
        double v = sbins[b];
        if (wb_on)
#pragma unroll
            for (int w = 0; w < 8; ++w) v += (double)wbins[w * e.n_bins + b];
        if (v != 0.0) atomicAdd(&e.C_sum[(int64_t)t * e.n_bins + b], v);
    }
    for (int o = tid; o < e.n_q * e.q_parts; o += 256)
        if (sq[o] != 0.0) atomicAdd(&e.Sq_sum[(int64_t)t * e.n_q * e.q_parts + o], sq[o]);
}

}  // namespace

int launch_simt(asd_corr_plan *p, const float *traj, int64_t row_begin, int64_t row_end,
                int t_begin, int t_end, double *C_sum, double *Sq_sum, cudaStream_t s)
{
    SimtParams P{};
    P.traj = traj;
    P.B = p->Bf32;
    P.R = p->R;
    P.F3 = 3 * p->F;
    P.K3 = 3 * p->T0;
    P.Kseg = (int)p->Kseg;
    P.S = p->S;
    P.N = (int)p->N;
    P.row_begin = (int)row_begin;
    P.row_end = (int)row_end;
    P.t_begin = t_begin;
    EpiParams &e = P.e;
    e.geom = p->d.geometry;
    e.Lx = p->d.L[0];
    e.Ly = p->d.L[1];
    e.Lz = p->d.L[2];
    e.periodic = p->d.periodic;
    e.inv_w = p->n_bins > 0 ? (float)(1.0 / p->d.bin_width) : 1.f;
    e.n_bins = p->n_bins;
    e.n_q = p->n_q;
    e.coords = p->coords;
    e.pos = p->pos;
    e.thr = p->thr;
    e.nq_pad = (p->n_q + kQChunk - 1) / kQChunk * kQChunk;
    e.q_parts = p->q_parts;
    e.cs = p->cs;
    e.C_sum = C_sum;
    e.Sq_sum = Sq_sum;
    e.C_fix = p->C_fix;
    e.Sq_fix = p->Sq_fix;
    e.fix_scale = p->d.deterministic ? p->fix_scale : nullptr;
    P.err = device_error_word();
    if (!P.err) return ASD_ECUDA;
    dim3 grid((unsigned)((row_end - row_begin + TM - 1) / TM), (unsigned)((p->N + TN - 1) / TN),
              (unsigned)(t_end - t_begin));
    if (grid.y > 65535u || grid.z > 65535u) {
        set_error_text("FP32 form: grid too large (N or n_t)");
        return ASD_EUNSUPPORTED;
    }
    size_t smem = sizeof(double) * (p->n_bins + p->n_q * p->q_parts);
    // per-warp FP32 bin copies where they fit the default 48 KB of dynamic shared memory
    P.warp_bins = !p->d.deterministic && smem + sizeof(float) * 8 * p->n_bins <= 48 * 1024;
    if (P.warp_bins) smem += sizeof(float) * 8 * p->n_bins;
    simt_kernel<<<grid, 256, smem, s>>>(P);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // namespace asd
