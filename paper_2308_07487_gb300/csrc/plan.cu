// Plan lifecycle, geometry tables, pair counts, dispatch and normalisation (C ABI).
//
// The method (arXiv 2308.07487, Sections 3.2-3.4): for each time displacement the
// pair sum is one GEMM-shaped contraction A_t B^T over K = 3*T0 (x S samples) whose
// N x N result is reduced in the kernel epilogue, either over distance bins or with
// the phase weights of Eq. 6.  This file owns everything around the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "asd_internal.h"
#include "geom.cuh"

namespace asd {

static thread_local std::string g_err_text;

void set_cuda_error(cudaError_t e, const char *where)
{
    g_err_text = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e) + " (" + where + ")";
}
void set_error_text(const std::string &s) { g_err_text = s; }

// One error word per device, at module scope.
__device__ int g_device_error;

int *device_error_word()
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    return static_cast<int *>(p);
}

// ---------------------------------------------------------------------------------
// pair counts: exact ordered-pair count of every bin over all N x N pairs
// ---------------------------------------------------------------------------------
__global__ void count_pairs_kernel(int64_t N, EpiParams e, unsigned long long *counts)
{
    extern __shared__ unsigned int hist[];
    for (int b = threadIdx.x; b < e.n_bins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x;
    if (i < N) {
        for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
            float d2 = e.geom == ASD_GEOM_LATTICE
                           ? lattice_d2(e.coords[i], e.coords[j], e.Lx, e.Ly, e.Lz, e.periodic)
                           : position_d2(e.pos[i], e.pos[j]);
            int b = bin_of_d2(d2, e.inv_w, e.n_bins, e.thr);
            if (b < e.n_bins) atomicAdd(&hist[b], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < e.n_bins; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

__global__ void normalize_kernel(const double *C_sum, double *C, int n_t, int n_bins,
                                 const double *inv_n, const double *Sq_sum, double *Sq, int n_q,
                                 double inv_nq)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (C_sum && k < (int64_t)n_t * n_bins) C[k] = C_sum[k] * inv_n[k % n_bins];
    if (Sq_sum && k < (int64_t)n_t * n_q) Sq[k] = Sq_sum[k] * inv_nq;
}

// Deterministic mode.  Largest |x| of the trajectory (FP32 bits of non-negative floats
// order like the floats, so an integer max is exact and order-free).
__global__ void amax_kernel(const float *__restrict__ x, int64_t n, unsigned int *out)
{
    unsigned int m = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(x[k])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Fixed-point scale 2^e of one launch: the largest power of two with
// bound * 2^e < 2^61, bound = 2 rows N K max|a| max|b| (>= the sum of |terms| of any
// partial or total sum the launch forms, with room for rounding).
__global__ void fix_scale_kernel(const unsigned int *amax_bits, double rows, double N, double K,
                                 double b_factor, double *scale)
{
    const double a = (double)__uint_as_float(*amax_bits);
    const double bound = 2.0 * rows * N * K * a * (a * b_factor);
    double sc = 1.0;
    if (bound > 0.0 && bound < 1e300) {
        int ex;
        frexp(bound, &ex);             // bound in [2^(ex-1), 2^ex)
        sc = ldexp(1.0, 61 - ex);      // bound * sc < 2^61
    }
    *scale = sc;
}

// out[k] += fix[k] / scale for k < n (then the next launch starts from zeroed sums)
__global__ void fix_add_kernel(const long long *__restrict__ fix, int64_t n,
                               const double *scale, double *__restrict__ out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] += (double)fix[k] / *scale;
}

static EpiParams epi_of(const asd_corr_plan *p)
{
    EpiParams e{};
    e.geom = p->d.geometry;
    e.Lx = p->d.L[0];
    e.Ly = p->d.L[1];
    e.Lz = p->d.L[2];
    e.periodic = p->d.periodic;
    e.inv_w = p->n_bins > 0 ? (float)(1.0 / p->d.bin_width) : 1.0f;
    e.w = (float)p->d.bin_width;
    e.thr_exact = p->thr_exact;
    e.n_bins = p->n_bins;
    e.NW = p->NW;
    e.use_window = p->use_window;
    e.n_q = p->n_q;
    e.coords = p->coords;
    e.pos = p->pos;
    e.thr = p->thr;
    e.lut = p->lut;
    e.n_lut = p->n_lut;
    // fast lattice binning: coordinates fit a byte (the minimum image |d| <= L/2 and, for
    // open lattices, |d| <= 127 so that min(d, 255 - d) = d), every bin is private, and
    // table entries scaled to private-bin offsets fit 16 bits
    e.fast = 0;
    e.Lpk = 0;
    if (p->tc && p->d.geometry == ASD_GEOM_LATTICE && p->n_bins > 0 && !p->use_window) {
        const int lim = p->d.periodic ? 255 : 128;
        bool ok = p->d.L[0] <= lim && p->d.L[1] <= lim && p->d.L[2] <= lim;
        if (p->n_lut > 0) ok = ok && (int64_t)(p->n_bins + 1) * bin_stride(p->EW) <= 65536;
        if (ok) {
            e.fast = 1;
            e.Lpk = p->d.periodic ? ((uint32_t)p->d.L[0] | ((uint32_t)p->d.L[1] << 8) |
                                     ((uint32_t)p->d.L[2] << 16))
                                  : 0x00ffffffu;
        }
    }
    e.nq_pad = (p->n_q + kQChunk - 1) / kQChunk * kQChunk;
    e.npass = p->tc && p->n_q > 0 ? (p->n_q + kPhaseQ - 1) / kPhaseQ : 0;
    e.q_parts = p->q_parts;
    e.cs = p->cs;
    e.C_fix = p->C_fix;
    e.Sq_fix = p->Sq_fix;
    e.fix_scale = p->d.deterministic ? p->fix_scale : nullptr;
    return e;
}

// Round to the nearest BF16 (ties to even); the inputs here are finite.
static uint16_t bf16_rn(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static double bf16_value(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static void carve(char *&cur, size_t bytes, void **out)
{
    *out = cur;
    cur += (bytes + 255) & ~(size_t)255;
}

// Encode one 2D tiled tensor map through the driver entry point (no libcuda link).
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode()
{
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &ptr, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(ptr);
    });
    return fn;
}

static int encode_2d(CUtensorMap *m, void *base, int elem_bytes, uint64_t inner, uint64_t rows,
                     uint32_t box_inner, uint32_t box_rows, int swizzle_bytes)
{
    PFN_encodeTiled enc = get_encode();
    if (!enc) {
        set_error_text("cuTensorMapEncodeTiled unavailable");
        return ASD_EUNSUPPORTED;
    }
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * (uint64_t)elem_bytes};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                                 : CU_TENSOR_MAP_SWIZZLE_64B;
    CUresult r = enc(m, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[128];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        set_error_text(buf);
        return ASD_ECUDA;
    }
    return ASD_OK;
}

static int fill_problem(asd_corr_plan *p, TcProblem *tp, int64_t row_begin, int64_t row_end)
{
    memset(tp, 0, sizeof(*tp));
    for (int pl = 0; pl < p->n_planes; ++pl) {
        for (int c = 0; c < p->n_copies; ++c) {
            int rc = encode_2d(&tp->mapA[pl][c], p->A[pl][c], p->elem_bytes, (uint64_t)p->Rpad,
                               (uint64_t)p->N, (uint32_t)p->BK, kBM, p->swizzle_bytes);
            if (rc) return rc;
        }
        // (a CTA pair loads half of the tile's B columns in each CTA)
        int rc = encode_2d(&tp->mapB[pl], p->B[pl], p->elem_bytes, (uint64_t)p->Kb, (uint64_t)p->N,
                           (uint32_t)p->BK, (uint32_t)(p->BN / p->CG), p->swizzle_bytes);
        if (rc) return rc;
    }
    // phase column weights: boxes of 64 sites x one pass (128 rows), BF16, 128-byte swizzle
    if (p->W) {
        const int npass = (p->n_q + kPhaseQ - 1) / kPhaseQ;
        const size_t plane = (size_t)npass * 2 * kPhaseQ * p->Wld * 2;
        for (int pl = 0; pl < 2; ++pl) {
            int rc = encode_2d(&tp->mapW[pl], static_cast<char *>(p->W) + pl * plane, 2,
                               (uint64_t)p->Wld, (uint64_t)npass * 2 * kPhaseQ, 64,
                               (uint32_t)(2 * kPhaseQ / p->CG), 128);
            if (rc) return rc;
        }
    }
    tp->N = (int)p->N;
    tp->row_begin = (int)row_begin;
    tp->row_end = (int)row_end;
    tp->tiles_m = (int)((row_end - row_begin + kBM * p->CG - 1) / (kBM * p->CG));
    tp->tiles_n = (int)((p->N + p->BN - 1) / p->BN);
    tp->n_t = p->n_t;
    tp->S = p->S;
    tp->F3 = 3 * p->F;
    tp->Kseg = (int)p->Kseg;
    tp->nkb = (int)(p->Kseg / p->BK);
    tp->n_copies = p->n_copies;
    tp->group_m = p->d.raster_m > 0 ? p->d.raster_m : 16;
    tp->k_chunks = p->k_chunks;
    tp->n_tiles = tc_work_items(p->n_t, tp->tiles_m, tp->tiles_n);
    tp->epi = epi_of(p);
    return ASD_OK;
}

// ---- deterministic mode (asd_corr_desc.deterministic) ----
// Largest |x| of the trajectory, the operand bound of the fixed-point scale.
static int fix_amax(asd_corr_plan *p, const float *traj, cudaStream_t s)
{
    if (!p->d.deterministic) return ASD_OK;
    ASD_CUDA_TRY(cudaMemsetAsync(p->amax_bits, 0, sizeof(unsigned int), s));
    const int64_t n = p->N * p->R;
    amax_kernel<<<(unsigned)(p->sm_count * 8), 256, 0, s>>>(traj, n, p->amax_bits);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

int fix_begin(asd_corr_plan *p, int64_t rows, int t_begin, int t_end, cudaStream_t s)
{
    if (!p->d.deterministic) return ASD_OK;
    const int64_t nt = t_end - t_begin;
    if (p->n_bins > 0)
        ASD_CUDA_TRY(cudaMemsetAsync(p->C_fix + (int64_t)t_begin * p->n_bins, 0,
                                     sizeof(long long) * nt * p->n_bins, s));
    if (p->n_q > 0)
        ASD_CUDA_TRY(cudaMemsetAsync(p->Sq_fix + (int64_t)t_begin * p->n_q * p->q_parts, 0,
                                     sizeof(long long) * nt * p->n_q * p->q_parts, s));
    // centring subtracts a mean from B: |b| <= 2 max|x|
    fix_scale_kernel<<<1, 1, 0, s>>>(p->amax_bits, (double)rows, (double)p->N,
                                     (double)p->S * 3.0 * p->T0, p->center ? 2.0 : 1.0,
                                     p->fix_scale);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

int fix_end(asd_corr_plan *p, int t_begin, int t_end, double *C_sum, double *Sq_sum,
            cudaStream_t s)
{
    if (!p->d.deterministic) return ASD_OK;
    const int64_t nt = t_end - t_begin;
    if (p->n_bins > 0 && C_sum) {
        const int64_t n = nt * p->n_bins, o = (int64_t)t_begin * p->n_bins;
        fix_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->C_fix + o, n, p->fix_scale,
                                                                  C_sum + o);
        ASD_CUDA_TRY(cudaGetLastError());
    }
    if (p->n_q > 0 && Sq_sum) {
        const int64_t n = nt * p->n_q * p->q_parts, o = (int64_t)t_begin * p->n_q * p->q_parts;
        fix_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->Sq_fix + o, n,
                                                                  p->fix_scale, Sq_sum + o);
        ASD_CUDA_TRY(cudaGetLastError());
    }
    return ASD_OK;
}

}  // namespace asd

using namespace asd;

extern "C" {

const char *asd_strerror(int status)
{
    static thread_local std::string s;
    const char *base = "unknown status";
    switch (status) {
    case ASD_OK: base = "ok"; break;
    case ASD_EINVAL: base = "invalid argument"; break;
    case ASD_ENOMEM: base = "out of memory"; break;
    case ASD_ECUDA: base = "CUDA error"; break;
    case ASD_ETIMEOUT: base = "bounded device wait timed out"; break;
    case ASD_EUNSUPPORTED: base = "unsupported"; break;
    case ASD_EBOUNDS: base = "index check failed (checked build)"; break;
    }
    s = base;
    if (status != ASD_OK && !g_err_text.empty()) s += ": " + g_err_text;
    return s.c_str();
}

int asd_sync_status(void *stream)
{
    ASD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int v = 0;
    ASD_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_device_error, sizeof(int)));
    if (v != 0) {
        int zero = 0;
        ASD_CUDA_TRY(cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int)));
        char buf[96];
        if (v >= DEV_BOUNDS) {
            snprintf(buf, sizeof buf, "device error word = %d (index check site %d)", v,
                     v - (int)DEV_BOUNDS);
            set_error_text(buf);
            return ASD_EBOUNDS;
        }
        snprintf(buf, sizeof buf, "device error word = %d", v);
        set_error_text(buf);
        return ASD_ETIMEOUT;
    }
    return ASD_OK;
}

void asd_pair_corr_plan_destroy(asd_corr_plan *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFree(p->ws);
    cudaFree(p->coords);
    cudaFree(p->pos);
    cudaFree(p->thr);
    cudaFree(p->lut);
    cudaFree(p->cs);
    cudaFree(p->W);
    cudaFree(p->sqF);
    cudaFree(p->counter);
    cudaFree(p->C_fix);
    cudaFree(p->inv_counts);
    cudaFree(p->d_prob);
    cudaFree(p->batch_desc);
    delete p->batch_last;
    delete p->h_prob;
    delete[] p->counts_h;
    delete p;
}

int64_t asd_pair_corr_workspace_bytes(const asd_corr_plan *p) { return p ? (int64_t)p->ws_bytes : 0; }

int asd_pair_corr_counts(const asd_corr_plan *p, int64_t *counts)
{
    ASD_CHECK_ARG(p && counts, "null argument");
    for (int b = 0; b < p->n_bins; ++b) counts[b] = p->counts_h[b];
    return ASD_OK;
}

int asd_pair_corr_plan_create(const asd_corr_desc *d, asd_corr_plan **out)
{
    ASD_CHECK_ARG(d && out, "null argument");
    *out = nullptr;
    ASD_CHECK_ARG(d->n_sites >= 1 && d->n_sites < (1LL << 31) - 512, "n_sites out of range");
    ASD_CHECK_ARG(d->n_samples >= 1 && d->T0 >= 1 && d->n_t >= 1, "S, T0, n_t must be >= 1");
    ASD_CHECK_ARG((int64_t)d->T0 + d->n_t - 1 <= d->n_frames, "need T0 + n_t - 1 <= F");
    ASD_CHECK_ARG(d->precision >= ASD_FP32 && d->precision <= ASD_SPLIT_BF16, "bad precision");
    ASD_CHECK_ARG(d->center == 0 || d->center == 1, "center must be 0 or 1");
    ASD_CHECK_ARG(d->geometry == ASD_GEOM_LATTICE || d->geometry == ASD_GEOM_POSITIONS,
                  "bad geometry");
    ASD_CHECK_ARG(d->n_bins >= 0 && d->n_bins <= 4096, "n_bins out of range [0,4096]");
    ASD_CHECK_ARG(d->n_q >= 0 && d->n_q <= 256, "n_q out of range [0,256]");
    ASD_CHECK_ARG(d->n_bins > 0 || d->n_q > 0, "nothing to compute (n_bins = n_q = 0)");
    ASD_CHECK_ARG(d->n_bins == 0 || d->bin_width > 0, "bin_width must be > 0");
    ASD_CHECK_ARG(d->n_q == 0 || d->q, "q required when n_q > 0");
    ASD_CHECK_ARG(d->tile_n == 0 || d->tile_n == 128 || d->tile_n == 192 || d->tile_n == 256,
                  "tile_n: 0, 128, 192, 256");
    ASD_CHECK_ARG(d->raster_m >= 0 && d->raster_m <= 64, "raster_m: 0..64");
    ASD_CHECK_ARG(d->stages == 0 || (d->stages >= 2 && d->stages <= 8), "stages: 0 or 2..8");
    ASD_CHECK_ARG(d->k_chunks >= 0 && d->k_chunks <= 256, "k_chunks: 0..256");
    ASD_CHECK_ARG(d->epi_warps == 0 || d->epi_warps == 4 || d->epi_warps == 8, "epi_warps: 0, 4 or 8");
    {
        // instantiated tensor-core kernels: 256- and 192-wide tiles with either warp
        // count; 128-wide tiles with 4 warps.  Phase weights run on the tensor core, whose
        // product needs 128 TMEM columns beside the two accumulators: tiles of at most 192
        // columns.
        ASD_CHECK_ARG(!(d->tile_n == 128 && d->epi_warps == 8),
                      "tile_n = 128 needs 4 epilogue warps");
        if (d->precision != ASD_FP32 && d->n_q > 0)
            ASD_CHECK_ARG(d->tile_n != 256, "phase weights need tile_n <= 192");
    }
    ASD_CHECK_ARG(d->static_schedule == 0 || d->static_schedule == 1, "static_schedule: 0 or 1");
    ASD_CHECK_ARG(d->phase_sine == 0 || d->phase_sine == 1, "phase_sine: 0 or 1");
    ASD_CHECK_ARG(d->deterministic == 0 || d->deterministic == 1, "deterministic: 0 or 1");
    ASD_CHECK_ARG(d->cta_pair == 0 || d->cta_pair == 1, "cta_pair: 0 or 1");
    ASD_CHECK_ARG(!d->cta_pair || d->precision != ASD_FP32, "cta_pair needs a tensor form");
    ASD_CHECK_ARG(!d->cta_pair || d->tile_n != 128, "cta_pair needs tile_n 192 or 256");
    if (d->geometry == ASD_GEOM_LATTICE) {
        ASD_CHECK_ARG(d->coords, "coords required for lattice geometry");
        for (int a = 0; a < 3; ++a) ASD_CHECK_ARG(d->L[a] >= 1 && d->L[a] <= 1 << 20, "bad L");
        for (int64_t i = 0; i < d->n_sites; ++i)
            for (int a = 0; a < 3; ++a)
                ASD_CHECK_ARG(d->coords[3 * i + a] >= 0 && d->coords[3 * i + a] < d->L[a],
                              "coords outside [0, L)");
    } else {
        ASD_CHECK_ARG(d->pos, "pos required for positions geometry");
    }
    const int64_t R = (int64_t)d->n_samples * 3 * d->n_frames;
    ASD_CHECK_ARG(d->n_sites * R < (1LL << 40), "trajectory too large");

    int dev = 0;
    ASD_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    ASD_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    const bool tc = d->precision != ASD_FP32;
    if (tc && !(prop.major == 10 || prop.major == 11)) {
        set_error_text("tensor-core forms need a tcgen05 (sm_10x) device");
        return ASD_EUNSUPPORTED;
    }

    asd_corr_plan *p = new (std::nothrow) asd_corr_plan();
    if (!p) return ASD_ENOMEM;
    memset(p, 0, sizeof(*p));
    p->d = *d;
    p->d.coords = nullptr;
    p->d.pos = nullptr;
    p->d.q = nullptr;
    p->device = dev;
    p->sm_count = prop.multiProcessorCount;
    p->N = d->n_sites;
    p->S = d->n_samples;
    p->F = d->n_frames;
    p->T0 = d->T0;
    p->n_t = d->n_t;
    p->n_bins = d->n_bins;
    p->n_q = d->n_q;
    p->q_parts = 1 + d->phase_sine;
    p->prec = d->precision;
    p->center = d->center;
    p->R = R;
    p->tc = tc;
    p->counts_h = new (std::nothrow) int64_t[d->n_bins > 0 ? d->n_bins : 1];
    if (!p->counts_h) {
        delete p;
        return ASD_ENOMEM;
    }
    int rc = ASD_OK;
    auto fail = [&](int code) {
        asd_pair_corr_plan_destroy(p);
        return code;
    };

    // ---- operand layout ----
    if (tc) {
        p->n_planes = d->precision == ASD_SPLIT_BF16 ? 2 : 1;
        p->elem_bytes = d->precision == ASD_TF32 ? 4 : 2;
        p->n_copies = 16 / p->elem_bytes;
        p->swizzle_bytes = d->precision == ASD_SPLIT_BF16 ? 64 : 128;
        p->BK = p->swizzle_bytes / p->elem_bytes;
        p->BN = d->tile_n ? d->tile_n : (p->N <= 4096 ? 128 : (d->n_q > 0 ? 192 : 256));
        // CTA pairs: 192- or 256-wide tiles only
        p->CG = d->cta_pair ? 2 : 1;
        if (p->CG == 2 && p->BN == 128) p->BN = d->n_q > 0 ? 192 : 256;
        p->Rpad = (R + 7) / 8 * 8;
        p->Kseg = ((int64_t)3 * d->T0 + p->BK - 1) / p->BK * p->BK;
        // epilogue warps: two per scheduler (8) hide the latency of the binning epilogue
        // where it is longest, the FP32 position rule (measured on the 32^3 jittered glass,
        // split-BF16 with two K chunks: 453 against 340 TFLOP/s); lattices keep 4 (their
        // packed-coordinate binning is short: 540 against 492 on the 26^3 lattice).
        // 128-wide tiles run with 4 warps.
        p->EW = d->epi_warps ? d->epi_warps
                             : (d->geometry == ASD_GEOM_POSITIONS && p->BN != 128 ? 8 : 4);
        if (p->EW != 4 && p->BN == 128) p->BN = d->n_q > 0 ? 192 : 256;
        // K chunks: split-BF16 is the FP32-accurate form; each chunk's accumulator starts
        // from zero, bounding the FP32 accumulation error of the tensor core (it adds each
        // MMA's products into the FP32 accumulator with truncation) to at most 1024 terms
        // per partial sum at any K (measured on the 64^3 glass, K = 1536, 12 random blocks
        // of 16 rows, thermalised LL trajectory: one chunk 4.6e-5 worst per bin, two chunks
        // of 768 7.5e-6; on the 40^3 lattice, K = 3000: one chunk 1.4e-5, two 7.9e-6, three
        // 6.2e-6).  The other forms are limited by their operand rounding.  Each chunk's
        // epilogue runs while the next chunk's MMAs do.
        const int64_t nk = (int64_t)p->S * (p->Kseg / p->BK);
        int kc = d->k_chunks;
        if (kc == 0)
            kc = d->precision == ASD_SPLIT_BF16 ? (int)((p->S * p->Kseg + 1023) / 1024) : 1;
        if (kc > 256) kc = 256;
        if (kc > nk) kc = (int)nk;
        p->k_chunks = kc < 1 ? 1 : kc;
    } else {
        p->Rpad = 0;
        p->Kseg = ((int64_t)3 * d->T0 + 15) / 16 * 16;
        p->BN = 128;
        p->CG = 1;
    }
    p->Kb = p->S * p->Kseg;

    // lattice d2 -> bin table size (largest minimum-image d2 + 1), built with the tables
    p->n_lut = 0;
    if (d->geometry == ASD_GEOM_LATTICE && p->n_bins > 0) {
        int64_t max_d2 = 0;
        for (int a = 0; a < 3; ++a) {
            const int64_t m = d->periodic ? d->L[a] / 2 : d->L[a] - 1;
            max_d2 += m * m;
        }
        if (max_d2 < kLutMax) p->n_lut = (int)(max_d2 + 1);
    }

    // ---- bins: private window per epilogue thread ----
    if (tc) {
        rc = tc_configure(p);
        if (rc) return fail(rc);
    }

    // ---- workspace ----
    size_t bytes = 0;
    const size_t a_bytes = tc ? (size_t)p->N * p->Rpad * p->elem_bytes : 0;
    const size_t b_bytes = (size_t)p->N * p->Kb * (tc ? p->elem_bytes : 4);
    const size_t r256 = 256;
    auto up = [&](size_t b) { return (b + r256 - 1) / r256 * r256; };
    if (tc) bytes += p->n_planes * p->n_copies * up(a_bytes) + p->n_planes * up(b_bytes);
    else bytes += up(b_bytes);
    bytes += up((size_t)p->N * 3 * sizeof(float));  // centring means
    if (cudaMalloc(&p->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error_text("workspace allocation failed");
        return fail(ASD_ENOMEM);
    }
    p->ws_bytes = bytes;
    {
        char *cur = static_cast<char *>(p->ws);
        if (tc) {
            for (int pl = 0; pl < p->n_planes; ++pl)
                for (int c = 0; c < p->n_copies; ++c) carve(cur, a_bytes, &p->A[pl][c]);
            for (int pl = 0; pl < p->n_planes; ++pl) carve(cur, b_bytes, &p->B[pl]);
        } else {
            void *b = nullptr;
            carve(cur, b_bytes, &b);
            p->Bf32 = static_cast<float *>(b);
        }
        void *m = nullptr;
        carve(cur, (size_t)p->N * 3 * sizeof(float), &m);
        p->meanB = static_cast<float *>(m);
    }

    // ---- geometry tables ----
    {
        std::vector<int4> hc((size_t)p->N);
        std::vector<float4> hp((size_t)p->N);
        for (int64_t i = 0; i < p->N; ++i) {
            if (d->geometry == ASD_GEOM_LATTICE) {
                hc[i] = make_int4(d->coords[3 * i], d->coords[3 * i + 1], d->coords[3 * i + 2], 0);
                hp[i] = make_float4((float)hc[i].x, (float)hc[i].y, (float)hc[i].z, 0.f);
            } else {
                hc[i] = make_int4(0, 0, 0, 0);
                hp[i] = make_float4(d->pos[3 * i], d->pos[3 * i + 1], d->pos[3 * i + 2], 0.f);
            }
        }
        if (cudaMalloc(&p->coords, sizeof(int4) * p->N) != cudaSuccess ||
            cudaMalloc(&p->pos, sizeof(float4) * p->N) != cudaSuccess) {
            cudaGetLastError();
            return fail(ASD_ENOMEM);
        }
        if (cudaMemcpy(p->coords, hc.data(), sizeof(int4) * p->N, cudaMemcpyHostToDevice) ||
            cudaMemcpy(p->pos, hp.data(), sizeof(float4) * p->N, cudaMemcpyHostToDevice))
            return fail(ASD_ECUDA);
        // thresholds (k*w)^2 in FP64, rounded up to FP32
        const int nb = p->n_bins;
        std::vector<float> thr(nb + 2);
        thr[0] = 0.f;
        for (int k = 1; k < nb + 2; ++k) {
            double v = ((double)k * d->bin_width) * ((double)k * d->bin_width);
            float f = (float)v;
            if ((double)f < v) f = nextafterf(f, INFINITY);
            thr[k] = f;
        }
        // the kernels may compute the thresholds when each equals the FP32 square of the
        // FP32 product k w (same operations, same rounding, on both sides)
        p->thr_exact = nb > 0 && (double)(float)d->bin_width == d->bin_width;
        for (int k = 0; k < nb + 2 && p->thr_exact; ++k) {
            volatile float kw = (float)k * (float)d->bin_width;
            volatile float sq = kw * kw;
            p->thr_exact = sq == thr[k];
        }
        if (cudaMalloc(&p->thr, sizeof(float) * (nb + 2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ASD_ENOMEM);
        }
        if (cudaMemcpy(p->thr, thr.data(), sizeof(float) * (nb + 2), cudaMemcpyHostToDevice))
            return fail(ASD_ECUDA);
        // lattices: d2 is an integer below max_d2 + 1, so the bin of every possible d2 can
        // be tabulated (same rule: largest k with (k w)^2 <= d2, n_bins when dropped)
        if (p->n_lut > 0) {
            const int64_t max_d2 = p->n_lut - 1;
            {
                std::vector<uint16_t> lut((size_t)max_d2 + 1);
                for (int64_t d2 = 0; d2 <= max_d2; ++d2) {
                    int k = 0;
                    while (k < nb && ((double)(k + 1) * d->bin_width) * ((double)(k + 1) * d->bin_width) <=
                                         (double)d2)
                        ++k;
                    lut[d2] = (uint16_t)k;  // k == nb only when (nb w)^2 <= d2: dropped
                }
                // (size fixed before the shared-memory configuration)
                if (cudaMalloc(&p->lut, sizeof(uint16_t) * lut.size()) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ASD_ENOMEM);
                }
                if (cudaMemcpy(p->lut, lut.data(), sizeof(uint16_t) * lut.size(),
                               cudaMemcpyHostToDevice))
                    return fail(ASD_ECUDA);
            }
        }
        if (p->n_q > 0) {
            // rows padded with zeros to whole q-chunks (aligned float4 loads, no tail)
            const int nqp = (p->n_q + kQChunk - 1) / kQChunk * kQChunk;
            std::vector<float2> cs((size_t)p->N * nqp, make_float2(0.f, 0.f));
            for (int64_t i = 0; i < p->N; ++i) {
                double r[3];
                for (int a = 0; a < 3; ++a)
                    r[a] = d->geometry == ASD_GEOM_LATTICE ? (double)d->coords[3 * i + a]
                                                           : (double)d->pos[3 * i + a];
                for (int q = 0; q < p->n_q; ++q) {
                    double ph = d->q[3 * q] * r[0] + d->q[3 * q + 1] * r[1] + d->q[3 * q + 2] * r[2];
                    cs[(size_t)i * nqp + q] = make_float2((float)cos(ph), (float)sin(ph));
                }
            }
            if (cudaMalloc(&p->cs, sizeof(float2) * cs.size()) != cudaSuccess) {
                cudaGetLastError();
                return fail(ASD_ENOMEM);
            }
            if (cudaMemcpy(p->cs, cs.data(), sizeof(float2) * cs.size(), cudaMemcpyHostToDevice))
                return fail(ASD_ECUDA);
            // column weights of the tensor-core phase product, pass by pass: row
            // pp * 128 + o holds cos(q.r_c) of q = 64 pp + o (o < 64) or sin(q.r_c) of
            // q = 64 pp + o - 64, zero for q >= n_q, as BF16 hi = RN(x) and
            // lo = RN(x - hi) in two planes
            if (tc) {
                const int npass = (p->n_q + kPhaseQ - 1) / kPhaseQ;
                p->Wld = (p->N + 7) / 8 * 8;
                const size_t rows = (size_t)npass * 2 * kPhaseQ, plane = rows * p->Wld;
                std::vector<uint16_t> W(2 * plane, 0);
                for (int64_t c = 0; c < p->N; ++c) {
                    double r[3];
                    for (int a = 0; a < 3; ++a)
                        r[a] = d->geometry == ASD_GEOM_LATTICE ? (double)d->coords[3 * c + a]
                                                               : (double)d->pos[3 * c + a];
                    for (int q = 0; q < p->n_q; ++q) {
                        const double ph = d->q[3 * q] * r[0] + d->q[3 * q + 1] * r[1] +
                                          d->q[3 * q + 2] * r[2];
                        const double x2[2] = {cos(ph), sin(ph)};
                        for (int part = 0; part < 2; ++part) {
                            const size_t row = (size_t)(q / kPhaseQ) * 2 * kPhaseQ +
                                               part * kPhaseQ + q % kPhaseQ;
                            const uint16_t hi = bf16_rn((float)x2[part]);
                            W[row * p->Wld + c] = hi;
                            W[plane + row * p->Wld + c] =
                                bf16_rn((float)(x2[part] - bf16_value(hi)));
                        }
                    }
                }
                if (cudaMalloc(&p->W, sizeof(uint16_t) * W.size()) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ASD_ENOMEM);
                }
                if (cudaMemcpy(p->W, W.data(), sizeof(uint16_t) * W.size(),
                               cudaMemcpyHostToDevice))
                    return fail(ASD_ECUDA);
            }
            // transforms of the separable phase form (asd_pair_corr_sq_separable)
            const size_t fb = sizeof(double) * 2 * (size_t)p->n_q * p->S * 3 * p->F;
            if (cudaMalloc(&p->sqF, fb) != cudaSuccess) {
                cudaGetLastError();
                return fail(ASD_ENOMEM);
            }
        }
    }

    // ---- exact pair counts ----
    if (p->n_bins > 0) {
        unsigned long long *dc = nullptr;
        if (cudaMalloc(&dc, sizeof(unsigned long long) * p->n_bins) != cudaSuccess) {
            cudaGetLastError();
            return fail(ASD_ENOMEM);
        }
        rc = launch_counts(p, 0, dc);
        if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = ASD_ECUDA;
        if (!rc) {
            std::vector<unsigned long long> hc(p->n_bins);
            if (cudaMemcpy(hc.data(), dc, sizeof(unsigned long long) * p->n_bins,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = ASD_ECUDA;
            for (int b = 0; b < p->n_bins; ++b) p->counts_h[b] = (int64_t)hc[b];
        }
        cudaFree(dc);
        if (rc) return fail(rc);
        std::vector<double> inv(p->n_bins);
        for (int b = 0; b < p->n_bins; ++b)
            inv[b] = p->counts_h[b] > 0
                         ? 1.0 / ((double)p->S * p->T0 * (double)p->counts_h[b]) : 0.0;
        if (cudaMalloc(&p->inv_counts, sizeof(double) * p->n_bins) != cudaSuccess) {
            cudaGetLastError();
            return fail(ASD_ENOMEM);
        }
        if (cudaMemcpy(p->inv_counts, inv.data(), sizeof(double) * p->n_bins,
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(ASD_ECUDA);
    }

    // ---- deterministic mode: fixed-point sums, operand bound, scale (one allocation) ----
    if (d->deterministic) {
        const size_t nc = (size_t)p->n_t * p->n_bins, nq = (size_t)p->n_t * p->n_q * p->q_parts;
        const size_t bytes = 8 * (nc + nq) + 16;
        if (cudaMalloc(&p->C_fix, bytes) != cudaSuccess) {
            cudaGetLastError();
            p->C_fix = nullptr;
            return fail(ASD_ENOMEM);
        }
        if (cudaMemset(p->C_fix, 0, bytes) != cudaSuccess) return fail(ASD_ECUDA);
        p->Sq_fix = p->C_fix + nc;
        p->fix_scale = reinterpret_cast<double *>(p->C_fix + nc + nq);
        p->amax_bits = reinterpret_cast<unsigned int *>(p->fix_scale + 1);
    }

    // ---- tensor maps for the whole row range ----
    if (tc) {
        p->h_prob = new (std::nothrow) TcProblem;
        if (!p->h_prob || cudaMalloc(&p->d_prob, sizeof(TcProblem)) != cudaSuccess ||
            cudaMalloc(&p->counter, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ASD_ENOMEM);
        }
        rc = fill_problem(p, p->h_prob, 0, p->N);
        if (rc) return fail(rc);
        if (cudaMemcpy(p->d_prob, p->h_prob, sizeof(TcProblem), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(ASD_ECUDA);
    }
    *out = p;
    return ASD_OK;
}

int asd_pair_corr(asd_corr_plan *p, const float *traj, int64_t row_begin, int64_t row_end,
                  double *C_sum, double *Sq_sum, void *stream)
{
    ASD_CHECK_ARG(p && traj, "null argument");
    ASD_CHECK_ARG(0 <= row_begin && row_begin <= row_end && row_end <= p->N, "bad row range");
    ASD_CHECK_ARG(p->n_bins == 0 || C_sum, "C_sum required when n_bins > 0");
    ASD_CHECK_ARG(p->n_q == 0 || Sq_sum, "Sq_sum required when n_q > 0");
    ASD_CHECK_ARG(((uintptr_t)traj & 15) == 0, "traj must be 16-byte aligned");
    if (row_begin == row_end) return ASD_OK;
    int rc = asd_pair_corr_prepare(p, traj, row_begin, row_end, stream);
    if (rc) return rc;
    return asd_pair_corr_contract(p, row_begin, row_end, C_sum, Sq_sum, stream);
}

int asd_pair_corr_prepare(asd_corr_plan *p, const float *traj, int64_t row_begin, int64_t row_end,
                          void *stream)
{
    ASD_CHECK_ARG(p && traj, "null argument");
    ASD_CHECK_ARG(0 <= row_begin && row_begin <= row_end && row_end <= p->N, "bad row range");
    ASD_CHECK_ARG(((uintptr_t)traj & 15) == 0, "traj must be 16-byte aligned");
    int rc = launch_prep(p, traj, row_begin, row_end, (cudaStream_t)stream);
    if (rc) return rc;
    rc = fix_amax(p, traj, (cudaStream_t)stream);
    if (rc) return rc;
    p->prepared_traj = traj;
    p->prepared_begin = row_begin;
    p->prepared_end = row_end;
    return ASD_OK;
}

int asd_pair_corr_contract(asd_corr_plan *p, int64_t row_begin, int64_t row_end, double *C_sum,
                           double *Sq_sum, void *stream)
{
    ASD_CHECK_ARG(p, "null plan");
    return asd_pair_corr_contract_range(p, row_begin, row_end, 0, p->n_t, C_sum, Sq_sum, stream);
}

int asd_pair_corr_contract_range(asd_corr_plan *p, int64_t row_begin, int64_t row_end,
                                 int32_t t_begin, int32_t t_end, double *C_sum, double *Sq_sum,
                                 void *stream)
{
    ASD_CHECK_ARG(p, "null plan");
    ASD_CHECK_ARG(0 <= t_begin && t_begin <= t_end && t_end <= p->n_t, "bad displacement range");
    ASD_CHECK_ARG(p->prepared_traj, "asd_pair_corr_prepare has not been called");
    ASD_CHECK_ARG(p->prepared_begin <= row_begin && row_begin <= row_end &&
                      row_end <= p->prepared_end,
                  "rows outside the prepared range");
    ASD_CHECK_ARG(p->n_bins == 0 || C_sum, "C_sum required when n_bins > 0");
    ASD_CHECK_ARG(p->n_q == 0 || Sq_sum, "Sq_sum required when n_q > 0");
    if (row_begin == row_end || t_begin == t_end) return ASD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = fix_begin(p, row_end - row_begin, t_begin, t_end, s);
    if (rc) return rc;
    if (!p->tc) {
        rc = launch_simt(p, p->prepared_traj, row_begin, row_end, t_begin, t_end, C_sum, Sq_sum, s);
        return rc ? rc : fix_end(p, t_begin, t_end, C_sum, Sq_sum, s);
    }
    TcOverride ov{};
    ov.active = 1;
    ov.row_begin = (int)row_begin;
    ov.row_end = (int)row_end;
    ov.t_begin = t_begin;
    ov.n_t = t_end - t_begin;
    ov.tiles_m = (int)((row_end - row_begin + kBM * p->CG - 1) / (kBM * p->CG));
    ov.n_tiles = tc_work_items(ov.n_t, ov.tiles_m, p->h_prob->tiles_n);
    ov.C_sum = C_sum;
    ov.Sq_sum = Sq_sum;
    rc = launch_tc(p->d_prob, 1, ov.n_tiles, ov, p->prec, p->BN, p->swizzle_bytes, p->stages,
                   p->smem_bytes, tc_var_bytes(p->NW, p->n_bins, p->n_lut, p->EW), p->n_bins,
                   p->n_q, p->EW, p->d.deterministic, p->CG, p->sm_count,
                   p->d.static_schedule || p->CG == 2 ? nullptr : p->counter, s);
    return rc ? rc : fix_end(p, t_begin, t_end, C_sum, Sq_sum, s);
}

int asd_pair_corr_batched(asd_corr_plan *const *plans, const float *const *trajs, int n,
                          double *const *C_sum, double *const *Sq_sum, void *stream)
{
    ASD_CHECK_ARG(plans && trajs && n >= 1 && n <= kMaxProblems, "bad batch");
    const asd_corr_plan *p0 = plans[0];
    ASD_CHECK_ARG(p0 && p0->tc, "batched launch needs tensor-core plans");
    int max_nb = 0, max_nq = 0, stages = 1 << 30;
    size_t smem = 0;
    for (int k = 0; k < n; ++k) {
        const asd_corr_plan *p = plans[k];
        ASD_CHECK_ARG(p && trajs[k], "null plan or trajectory");
        ASD_CHECK_ARG(p->tc && p->prec == p0->prec && p->BN == p0->BN && p->EW == p0->EW,
                      "batched plans must share precision and tile width");
        ASD_CHECK_ARG(p->d.deterministic == p0->d.deterministic,
                      "batched plans must share the deterministic mode");
        ASD_CHECK_ARG(p->CG == 1, "batched launches use one CTA per tile (cta_pair = 0)");
        ASD_CHECK_ARG(p->device == p0->device, "plans on different devices");
        ASD_CHECK_ARG(p->n_bins == 0 || (C_sum && C_sum[k]), "C_sum required");
        ASD_CHECK_ARG(p->n_q == 0 || (Sq_sum && Sq_sum[k]), "Sq_sum required");
        ASD_CHECK_ARG(((uintptr_t)trajs[k] & 15) == 0, "traj must be 16-byte aligned");
        max_nq = p->n_q > max_nq ? p->n_q : max_nq;
        max_nb = p->n_bins > max_nb ? p->n_bins : max_nb;
    }
    // one smem configuration for the whole batch: the fixed epilogue arrays for the
    // largest n_bins / n_q, and the per-problem region (bins + bin table) for the largest
    // problem.  While that region costs the third pipeline stage, the problem that needs
    // the most bins with a d2 table switches to the threshold rule (n_lut = 0 below).
    std::vector<int> nlut((size_t)n);
    uint32_t vb = 0;
    {
        size_t stage_bytes = (size_t)p0->n_planes * (kBM + p0->BN) * p0->swizzle_bytes;
        const size_t cap = 232448 - 2048;
        auto region = [&](int k) { return tc_var_bytes(plans[k]->NW, plans[k]->n_bins, nlut[k], p0->EW); };
        auto largest = [&]() {
            uint32_t m = 0;
            for (int k = 0; k < n; ++k) m = region(k) > m ? region(k) : m;
            return m;
        };
        for (int k = 0; k < n; ++k) nlut[k] = plans[k]->n_lut;
        vb = largest();
        while (tc_epilogue_smem_vb(vb, max_nb, max_nq, p0->BN, p0->EW, p0->d.deterministic) + 3 * stage_bytes > cap) {
            int kk = -1;
            for (int k = 0; k < n; ++k)
                if (nlut[k] > 0 && (kk < 0 || region(k) > region(kk))) kk = k;
            if (kk < 0) break;
            nlut[kk] = 0;
            vb = largest();
        }
        const size_t epi = tc_epilogue_smem_vb(vb, max_nb, max_nq, p0->BN, p0->EW, p0->d.deterministic);
        if (epi + 2 * stage_bytes > cap) {
            set_error_text("batched epilogue does not fit shared memory");
            return ASD_EUNSUPPORTED;
        }
        stages = (int)((cap - epi) / stage_bytes);
        if (stages > 6) stages = 6;
        smem = epi + stages * stage_bytes + 2048;
        if (smem < kMinSmem) smem = kMinSmem;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Work list: built on the host every call and kept in the first plan, uploaded only
    // when it differs from that plan's previous upload (the first call for a batch may
    // synchronise and allocate; repeated identical calls only enqueue kernels, so they
    // can be captured, and a captured graph stays valid until its first plan leads a
    // different batch or is destroyed).
    asd_corr_plan *owner = plans[0];
    if (!owner->batch_desc) {
        // descriptors for the largest batch, then the work-item counter
        if (cudaMalloc(&owner->batch_desc, sizeof(TcProblem) * kMaxProblems + 256) != cudaSuccess) {
            cudaGetLastError();
            owner->batch_desc = nullptr;
            return ASD_ENOMEM;
        }
        owner->batch_last = new (std::nothrow) std::vector<TcProblem>();
        if (!owner->batch_last) {
            cudaFree(owner->batch_desc);
            owner->batch_desc = nullptr;
            return ASD_ENOMEM;
        }
    }
    std::vector<TcProblem> &last = *owner->batch_last;
    TcProblem *dbuf = owner->batch_desc;
    // The work list takes the problems largest first (longest-processing-time order):
    // measured on a mixed ensemble, this order matches the throughput of one launch per
    // problem, while the caller's order may interleave sizes and lose 10-15 %.  Each
    // descriptor carries its own outputs, so the order is invisible to the caller.
    std::vector<int> order((size_t)n);
    for (int k = 0; k < n; ++k) order[k] = k;
    auto items = [&](int k) {
        const asd_corr_plan *p = plans[k];
        return p->k_chunks *
               tc_work_items(p->n_t, (int)((p->N + kBM - 1) / kBM), p->h_prob->tiles_n);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items(a) > items(b); });
    std::vector<TcProblem> h((size_t)n);
    int64_t total = 0;
    for (int pos = 0; pos < n; ++pos) {
        const int k = order[pos];
        const asd_corr_plan *p = plans[k];
        TcProblem &hk = h[pos];
        hk = *p->h_prob;
        hk.row_begin = 0;
        hk.row_end = (int)p->N;
        hk.tiles_m = (int)((p->N + kBM - 1) / kBM);
        hk.n_tiles = tc_work_items(p->n_t, hk.tiles_m, hk.tiles_n);
        hk.tile_begin = total;
        hk.epi.n_lut = nlut[k];  // 0: the threshold rule (see above)
        hk.epi.C_sum = C_sum ? C_sum[k] : nullptr;
        hk.epi.Sq_sum = Sq_sum ? Sq_sum[k] : nullptr;
        total += hk.n_tiles;
    }
    const bool same = last.size() == h.size() &&
                      memcmp(last.data(), h.data(), sizeof(TcProblem) * h.size()) == 0;
    if (!same) {
        ASD_CUDA_TRY(cudaStreamSynchronize(s));
        ASD_CUDA_TRY(cudaMemcpy(dbuf, h.data(), sizeof(TcProblem) * n, cudaMemcpyHostToDevice));
        last = h;
    }
    for (int k = 0; k < n; ++k) {
        int rc = launch_prep(plans[k], trajs[k], 0, plans[k]->N, s);
        if (!rc) rc = fix_amax(plans[k], trajs[k], s);
        if (!rc) rc = fix_begin(plans[k], plans[k]->N, 0, plans[k]->n_t, s);
        if (rc) return rc;
    }
    TcOverride ov{};
    // dynamic schedule unless any plan of the batch asks for the static order; the
    // counter lives behind the work list
    bool dyn = true;
    for (int k = 0; k < n; ++k) dyn = dyn && !plans[k]->d.static_schedule;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(dbuf + kMaxProblems);
    int rc = launch_tc(dbuf, n, total, ov, p0->prec, p0->BN, p0->swizzle_bytes, stages, smem, vb,
                       max_nb, max_nq, p0->EW, p0->d.deterministic, 1, p0->sm_count,
                       dyn ? ctr : nullptr, s);
    for (int k = 0; k < n && !rc; ++k)
        rc = fix_end(plans[k], 0, plans[k]->n_t, C_sum ? C_sum[k] : nullptr,
                     Sq_sum ? Sq_sum[k] : nullptr, s);
    return rc;
}

int asd_pair_corr_normalize(const asd_corr_plan *p, const double *C_sum, const double *Sq_sum,
                            double *C, double *Sq, void *stream)
{
    ASD_CHECK_ARG(p, "null plan");
    ASD_CHECK_ARG((C_sum == nullptr) == (C == nullptr), "C_sum and C go together");
    ASD_CHECK_ARG((Sq_sum == nullptr) == (Sq == nullptr), "Sq_sum and Sq go together");
    if (!C_sum && !Sq_sum) return ASD_OK;
    ASD_CHECK_ARG(!C_sum || p->n_bins > 0, "plan has no bins");
    ASD_CHECK_ARG(!Sq_sum || p->n_q > 0, "plan has no q-vectors");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n =
        std::max<int64_t>((int64_t)p->n_t * p->n_bins, (int64_t)p->n_t * p->n_q * p->q_parts);
    const double inv_nq = 1.0 / ((double)p->N * p->S * p->T0);
    normalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        C_sum, C, p->n_t, p->n_bins, p->inv_counts, Sq_sum, Sq, p->n_q * p->q_parts, inv_nq);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // extern "C"

namespace asd {
int launch_counts(asd_corr_plan *p, cudaStream_t s, unsigned long long *d_counts)
{
    ASD_CUDA_TRY(cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * p->n_bins, s));
    EpiParams e = epi_of(p);
    size_t sm = sizeof(unsigned int) * p->n_bins;
    count_pairs_kernel<<<(unsigned)p->N, 256, sm, s>>>(p->N, e, d_counts);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}
}  // namespace asd
