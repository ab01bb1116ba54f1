// Internal declarations of the GB300 pair-correlation library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/asd.h"

namespace asd {

// ----------------------------------------------------------------------------------
// status handling
// ----------------------------------------------------------------------------------
void set_cuda_error(cudaError_t e, const char *where);
void set_error_text(const std::string &s);

#define ASD_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            ::asd::set_cuda_error(_e, #expr);                \
            return ASD_ECUDA;                                \
        }                                                    \
    } while (0)

#define ASD_CHECK_ARG(cond, msg)                             \
    do {                                                     \
        if (!(cond)) {                                       \
            ::asd::set_error_text(msg);                      \
            return ASD_EINVAL;                               \
        }                                                    \
    } while (0)

// Device error word (one per device, module scope): bounded waits write a code here,
// and so do the index checks of a checked build (DEV_BOUNDS + site).
enum DeviceError : int {
    DEV_OK = 0,
    DEV_TIMEOUT_TMA = 1,
    DEV_TIMEOUT_MMA = 2,
    DEV_TIMEOUT_EPI = 3,
    DEV_TIMEOUT_SELFTEST = 4,
    DEV_BOUNDS = 256
};
int *device_error_word();          // device address of the word for the current device

// Sites of the index checks (ASD_CHECK_BOUNDS builds).
enum BoundSite : int {
    BND_SELFTEST = 0,   // asd_selftest_bounds
    BND_WORK = 1,       // decoded work item (displacement) outside its problem
    BND_PRIV = 2,       // private-bin offset outside the window rows (+ trash row)
    BND_FALLBACK = 3,   // fallback bin outside the launch's bin arrays
    BND_LUT = 4,        // lattice d2 outside the d2 -> bin table
    BND_THR = 5,        // threshold index outside [0, n_bins]
    BND_REGION = 6,     // a problem's bins and table larger than the launch's region
    BND_Q = 7,          // q index outside the phase arrays or the cos / sin rows
    BND_CACC = 8,       // per-CTA bin accumulator index
    BND_SIMT_BIN = 9,   // FP32 form: bin index
    BND_SIMT_Q = 10,    // FP32 form: q index
    BND_N_SITES
};

#ifndef ASD_CHECK_BOUNDS
#define ASD_CHECK_BOUNDS 0
#endif
#if ASD_CHECK_BOUNDS
// Checked build: a failed index check records the first failure and the caller skips
// the access (no trap: the kernel carries on and the host reads the word).
__device__ __forceinline__ bool in_bounds(bool ok, int site, int *err)
{
    if (!ok) atomicCAS(err, 0, (int)DEV_BOUNDS + site);
    return ok;
}
#define ASD_INB(cond, site, err) (::asd::in_bounds((cond), (site), (err)))
#else
#define ASD_INB(cond, site, err) (true)
#endif

// Deterministic sums (asd_corr_desc.deterministic): values become 64-bit fixed point,
// x -> round(x 2^e), so sums over threads and tiles are integer adds whose result does
// not depend on their order.  The scale 2^e comes from a bound on every partial sum.
__device__ __forceinline__ long long to_fixed(double x, double scale)
{
    return __double2ll_rn(x * scale);
}
__device__ __forceinline__ void add_fixed(long long *dst, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)v);
}

// ----------------------------------------------------------------------------------
// tensor-core operand layout
// ----------------------------------------------------------------------------------
constexpr int kBM = 128;            // rows (sites i) per tile = TMEM lanes
constexpr int kMaxCopies = 8;       // shifted operand copies (16-byte TMA start rule)
constexpr int kMaxProblems = 4096;  // batched work list
constexpr size_t kMinSmem = 120 * 1024;  // tensor-core kernel: one CTA per SM
constexpr int kLutMax = 16384;           // largest d2 -> bin table kept in shared memory
constexpr int kQChunk = 16;              // q-vectors per chunk of the phase epilogue (cs
                                         // rows are zero padded to whole chunks)
constexpr int kPhaseQ = 64;              // q-vectors per pass of the tensor-core phase
                                         // product (128 output columns: cos and sin)

// Private-bin stride (floats) of the tensor-core epilogue with `ew` epilogue warps: one
// column per accumulator row, so a warp's 32 lanes address 32 distinct banks.
__host__ __device__ constexpr int bin_stride(int ew) { return 128 * (ew / 4); }

// Epilogue geometry + output parameters of one problem (device-visible POD).
struct EpiParams {
    int geom;               // ASD_GEOM_*
    int Lx, Ly, Lz;
    int periodic;
    float inv_w;
    float w;                // bin width in FP32
    int thr_exact;          // every threshold thr[k] = RN(RN(k w)^2) (computable in-kernel)
    int n_bins;
    int NW;                 // private bins held per thread (window width)
    int use_window;         // 1: window start derived from per-tile boxes
    int n_q;
    const int4 *coords;     // [N] (x,y,z,0)
    const float4 *pos;      // [N] (x,y,z,0)
    const float *thr;       // [n_bins+2]: FP32 thresholds (k*w)^2 rounded up; thr[0]=0
    const uint16_t *lut;    // lattices: bin of every integer d2 < n_lut (n_bins = dropped)
    int n_lut;              // 0 when the table is not used
    int fast;               // lattice with byte-sized coordinates and every bin private:
                            // packed-coordinate d2, table entries are private-bin offsets
    uint32_t Lpk;           // fast: per-byte minimum-image modulus (x | y<<8 | z<<16)
    int nq_pad;             // row length of cs (n_q rounded up to the q-chunk, zero padded)
    int npass;              // passes of kPhaseQ q-vectors (0 without phase weights)
    int q_parts;            // 1: cosine part of the phase sum; 2: cosine and sine parts
    const float2 *cs;       // [N][nq_pad] (cos, sin)(q.r_i)
    double *C_sum;          // [n_t][n_bins]
    double *Sq_sum;         // [n_t][n_q]
    // deterministic mode: fixed-point sums [n_t][n_bins] and [n_t][n_q][q_parts] and the
    // scale 2^e (device, set after the operands are prepared); null otherwise
    long long *C_fix;
    long long *Sq_fix;
    const double *fix_scale;
};

// One problem of the (possibly batched) tensor-core launch.
struct TcProblem {
    CUtensorMap mapA[2][kMaxCopies];  // [plane][copy]
    CUtensorMap mapB[2];              // [plane]
    CUtensorMap mapW[2];              // phase column weights [plane]: rows (pass, output),
                                      // columns = sites (BF16 hi / lo)
    int64_t tile_begin;               // first flattened work item of this problem
    int64_t n_tiles;                  // work items: n_t * tiles_m * tiles_n
    int N;                            // columns (sites)
    int row_begin, row_end;
    int tiles_m, tiles_n;
    int n_t;
    int S;
    int F3;                           // 3*F: sample stride inside a trajectory row
    int Kseg;                         // B segment per sample (multiple of BK)
    int nkb;                          // K blocks per sample
    int n_copies;                     // shifted copies (8 for BF16, 4 for TF32)
    int group_m;                      // raster group height (row tiles)
    int k_chunks;                     // partial accumulators along K per tile
    EpiParams epi;
};

// Per-launch override of a single problem's row range and outputs (lets the device
// copy of the descriptor be uploaded once per plan).
struct TcOverride {
    int active;
    int row_begin, row_end, tiles_m;
    int t_begin, n_t;              // displacements [t_begin, t_begin + n_t)
    int64_t n_tiles;
    double *C_sum;
    double *Sq_sum;
};

// Kernel parameters of one tensor-core launch.
struct TcLaunchArgs {
    const TcProblem *probs;
    int n_probs;
    int64_t total_tiles;
    TcOverride ov;
    int stages;
    uint32_t VB;           // bytes of the per-problem epilogue region (largest problem)
    unsigned long long *counter;  // dynamic schedule: work-item counter (zero at launch), or null
    int NB, NQ;            // epilogue shared-memory layout maxima
    int det;               // 1: some problem sums in fixed point (fallback bins 8 bytes)
    int *err;
};

template <int FORM>
int tc_launch_form(const TcLaunchArgs &a, size_t smem, int BN, int ew, int cg, int sm_count,
                   cudaStream_t s);

}  // namespace asd

// Opaque plan (global namespace, forward-declared in asd.h).
struct asd_corr_plan {
    asd_corr_desc d;
    int device;
    int sm_count;
    int64_t N;
    int S, F, T0, n_t, n_bins, n_q, prec, center;
    int64_t R;                 // row length of the trajectory: S*3F
    // tensor-core operands
    int tc;                    // 1 for the tcgen05 forms
    int n_planes;              // 1, or 2 for split-BF16
    int n_copies;
    int elem_bytes;
    int BK;                    // K elements per pipeline stage
    int swizzle_bytes;         // 128 or 64
    int BN;                    // tile width (columns)
    int64_t Rpad;              // row length of an A copy (elements)
    int64_t Kseg;              // B elements per sample (3*T0 rounded up to BK)
    int64_t Kb;                // B row length S*Kseg
    void *ws;                  // one allocation for everything below
    size_t ws_bytes;
    void *A[2][asd::kMaxCopies];
    void *B[2];
    float *Bf32;               // FP32 form: B operand
    float *meanB;              // [N][3] centring means
    // geometry (device)
    int4 *coords;
    float4 *pos;
    float *thr;
    int thr_exact;             // thr[k] == RN(RN(k w)^2) for every k (see EpiParams)
    uint16_t *lut;             // lattice d2 -> bin table (nullptr when d2 can reach kLutMax)
    int n_lut;
    float2 *cs;
    void *W;                   // phase column weights [2 planes][npass * 128][Wld] BF16
    int64_t Wld;               // row length of W (N rounded up to 8)
    double *sqF;               // separable phase form: transforms [2 n_q][S*3F] (n_q > 0)
    unsigned long long *counter;  // work-item counter of the dynamic schedule
    int q_parts;               // 1 + desc.phase_sine: values per (t, q) in Sq_sum
    int tiles_m_all, tiles_n;
    int use_window;
    int NW;
    int64_t *counts_h;
    double *inv_counts;        // device [n_bins]: 1/(S*T0*n_b), 0 for empty bins
    // single-problem descriptor (tensor forms): host copy + device copy uploaded once
    asd::TcProblem *d_prob;
    asd::TcProblem *h_prob;
    // work list of a batched launch whose first plan this is: device descriptors for
    // kMaxProblems problems followed by the launch's work-item counter (allocated once, so
    // a captured graph's pointer never dangles), and the host copy of the last upload
    asd::TcProblem *batch_desc;
    std::vector<asd::TcProblem> *batch_last;
    int stages;
    size_t smem_bytes;
    int EW;                    // epilogue warps (4 or 8)
    int CG;                    // CTAs per tile: 1, or 2 for CTA pairs (256-row tiles)
    int k_chunks;
    // deterministic mode: fixed-point sums, the operand bound and the scale (device)
    long long *C_fix, *Sq_fix;
    unsigned int *amax_bits;   // max |x| over the prepared trajectory rows (FP32 bits)
    double *fix_scale;         // 2^e of the current launch
    // last asd_pair_corr_prepare
    const float *prepared_traj;
    int64_t prepared_begin, prepared_end;
};

namespace asd {
// prep.cu
int launch_prep(asd_corr_plan *p, const float *traj, int64_t row_begin, int64_t row_end,
                cudaStream_t s);
int launch_counts(asd_corr_plan *p, cudaStream_t s, unsigned long long *d_counts);
// pc_simt.cu
int launch_simt(asd_corr_plan *p, const float *traj, int64_t row_begin, int64_t row_end,
                int t_begin, int t_end, double *C_sum, double *Sq_sum, cudaStream_t s);
// pc_tc.cu
int tc_configure(asd_corr_plan *p);    // stages / smem for the plan's form
int launch_tc(const TcProblem *d_probs, int n_probs, int64_t total_tiles, TcOverride ov, int prec,
              int BN, int swizzle_bytes, int stages, size_t smem, uint32_t var_bytes,
              int max_nb, int max_nq, int ew, int det, int cg, int sm_count,
              unsigned long long *counter, cudaStream_t s);
// work items of one problem: one per (displacement, row tile, column tile); the K chunks
// of an item run as consecutive sub-items on one CTA
inline int64_t tc_work_items(int n_t, int tiles_m, int tiles_n)
{
    return (int64_t)n_t * tiles_m * tiles_n;
}
size_t tc_epilogue_smem(int NW, int n_bins, int n_q, int BN, int n_lut, int ew, int det);
// bytes of the per-problem epilogue region (private bins + bin table)
uint32_t tc_var_bytes(int NW, int n_bins, int n_lut, int ew);
// epilogue bytes with the per-problem region given separately
size_t tc_epilogue_smem_vb(uint32_t var_bytes, int n_bins, int n_q, int BN, int ew, int det);
// deterministic mode (plan.cu): before a launch over `rows` rows, zero the plan's
// fixed-point sums of displacements [t_begin, t_end) and set its scale; after it, add
// them to C_sum / Sq_sum
int fix_begin(asd_corr_plan *p, int64_t rows, int t_begin, int t_end, cudaStream_t s);
int fix_end(asd_corr_plan *p, int t_begin, int t_end, double *C_sum, double *Sq_sum,
            cudaStream_t s);
}  // namespace asd
