// Tensor-core forms (TF32, BF16, split-BF16): fused contraction + reduction epilogue.
//
// The method casts the pair sum of Eq. 4 / Eq. 5 for one time displacement as a GEMM
// G_t = A_t B^T (Section 3.2) and fuses the element-wise reduction that follows it --
// the bin sums or the phase-weighted inner product of Eq. 3 / Eq. 6 -- into the GEMM
// epilogue so that G_t never reaches memory (Sections 3.3-3.4).  On sm_103a this is:
//
//   warp 0      TMA producer: streams 128-row A tiles (K-offset windows of the
//               trajectory copies) and BN-row B tiles into a shared-memory ring;
//   warp 1      allocates TMEM and, from one thread, issues tcgen05.mma into one of two
//               128 x BN FP32 accumulators in tensor memory (double buffered), committing
//               each stage back to the ring and each finished tile to the epilogue;
//   warps 2-5   epilogue: tcgen05.ld one accumulator row per thread and reduce it --
//               per-thread private FP32 bins in shared memory (conflict-free [bin][row]
//               layout), phase weights from per-site cos/sin tables -- then FP64.
//
// The accumulator living in TMEM plays the role of the paper's OTF_SM shared-memory
// staging of the C tile (Section 3.4): the epilogue never holds the tile in registers.
// The per-pair phase factor uses cos(a - b) = cos a cos b + sin a sin b on tables made
// once per plan, so no transcendental is evaluated per pair (the register-spill
// problem of the paper's OTF_REG variant).
//
// Persistent: one CTA per SM walks a static round-robin list of
// (problem, t, row tile, column tile) work items, grouped 8 row tiles at a time so
// concurrently running CTAs share A and B panels in L2.  Several problems (a batched
// ensemble) share the list.  Every wait is bounded: after kTimeoutNs a role records
// an error in the device error word and stops; the CTA then drains its own in-flight
// copies and MMAs, frees TMEM and exits.
#include <cuda_bf16.h>

#include "asd_internal.h"
#include "geom.cuh"

namespace asd {
namespace {

constexpr int kThreads = 192;
constexpr int kEpiThreads = 128;
constexpr int kQC = 16;                       // q-vectors per epilogue pass
constexpr unsigned long long kTimeoutNs = 4000000000ull;
constexpr int kBinStride = 129;               // [bin][row] with odd stride: conflict-free

// ------------------------------------------------------------------------------------
// PTX wrappers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false after kTimeoutNs (the error
// word then holds `code`).
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, int code)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 1023u) == 0 && gtimer() - t0 > kTimeoutNs) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

template <bool TF32>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc)
{
    if (TF32)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 32 lanes x 32 consecutive 32-bit columns; the wait is tied to the registers so no
// use of them can be scheduled before it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ void epi_sync()
{
    __syncwarp();
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Epilogue barrier that also ANDs a flag over the 128 epilogue threads, so that every
// thread takes the same branch after a bounded wait.
__device__ __forceinline__ bool epi_sync_and(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Shared-memory matrix descriptor, K-major, swizzled (128B: mode 2, 64B: mode 4).
// SBO = 8 rows x swizzle span; LBO unused for swizzled K-major; version 1 (sm_100).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, int swb)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8u * swb) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(swb == 128 ? 2 : 4) << 61;
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B = BF16 (1) or TF32 (2), both K-major.
__host__ __device__ constexpr uint32_t idesc(bool tf32, int N)
{
    return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// ------------------------------------------------------------------------------------
// shared-memory layout of the epilogue region
// ------------------------------------------------------------------------------------
struct EpiLayout {
    uint32_t cacc, qacc, qred, bins, fb, colgeo, colcs, boxred, total;
};

__host__ __device__ inline uint32_t take(uint32_t &o, uint32_t bytes)
{
    o = (o + 15u) & ~15u;
    uint32_t r = o;
    o += bytes;
    return r;
}

__host__ __device__ inline EpiLayout epi_layout(int NW, int nb, int nq, int BN)
{
    EpiLayout L;
    uint32_t o = 0;
    L.cacc = take(o, 8u * (nb > 0 ? nb : 1));
    L.qacc = take(o, 8u * (nq > 0 ? nq : 1));
    L.qred = take(o, 8u * 4 * kQC);
    L.bins = take(o, 4u * (NW + 1) * kBinStride);
    L.fb = take(o, 4u * (nb > 0 ? nb : 1));
    L.colgeo = take(o, 16u * BN);
    L.colcs = nq > 0 ? take(o, 8u * BN * kQC) : 0u;
    L.boxred = take(o, 4u * 4 * 12);
    L.total = (o + 1023u) & ~1023u;
    return L;
}

struct TileInfo {
    int p, t, m0, n0, row_end;
};

__device__ __forceinline__ TileInfo decode(const TcProblem *__restrict__ probs, int n_probs,
                                           const TcOverride &ov, int64_t tau, int BN)
{
    int p = 0;
    if (n_probs > 1) {
        int lo = 0, hi = n_probs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (probs[mid].tile_begin <= tau) lo = mid;
            else hi = mid - 1;
        }
        p = lo;
    }
    const TcProblem &P = probs[p];
    const int tiles_m = ov.active ? ov.tiles_m : P.tiles_m;
    const int row_begin = ov.active ? ov.row_begin : P.row_begin;
    const int64_t l = tau - (ov.active ? 0 : P.tile_begin);
    const int64_t per_t = (int64_t)tiles_m * P.tiles_n;
    TileInfo ti;
    ti.p = p;
    ti.t = (int)(l / per_t);
    const int64_t rem = l % per_t;
    const int G = P.group_m;
    const int64_t gspan = (int64_t)G * P.tiles_n;
    const int first_m = (int)(rem / gspan) * G;
    const int gsz = min(G, tiles_m - first_m);
    const int64_t r2 = rem % gspan;
    ti.m0 = row_begin + (first_m + (int)(r2 % gsz)) * kBM;
    ti.n0 = (int)(r2 / gsz) * BN;
    ti.row_end = ov.active ? ov.row_end : P.row_end;
    return ti;
}

struct LaunchArgs {
    const TcProblem *probs;
    int n_probs;
    int64_t total_tiles;
    TcOverride ov;
    int stages;
    int NW, NB, NQ;  // epilogue layout maxima
    int *err;
};

// ------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------
template <int FORM, int BN, int SWB>
__global__ void __launch_bounds__(kThreads, 1) pc_tc_kernel(const __grid_constant__ LaunchArgs args)
{
    constexpr bool kTF32 = FORM == ASD_TF32;
    constexpr int kPlanes = FORM == ASD_SPLIT_BF16 ? 2 : 1;
    constexpr uint32_t kABytes = kBM * SWB;
    constexpr uint32_t kBBytes = BN * SWB;
    constexpr uint32_t kStageBytes = kPlanes * (kABytes + kBBytes);
    constexpr int kKSteps = SWB / 32;          // one MMA k-step covers 32 bytes of K
    constexpr int kBK = SWB / (kTF32 ? 4 : 2); // K elements per stage
    constexpr uint32_t kIdesc = idesc(kTF32, BN);
    constexpr uint32_t kTmemCols = 2 * BN;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~(uintptr_t)1023);
    const int stages = args.stages;
    uint8_t *tiles = smem;
    uint8_t *epi = tiles + (size_t)stages * kStageBytes;
    const EpiLayout EL = epi_layout(args.NW, args.NB, args.NQ, BN);
    uint64_t *bars = reinterpret_cast<uint64_t *>(epi + EL.total);
    // bars: full[stages], empty[stages], tfull[2], tempty[2], drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 5);
    const uint32_t full0 = saddr(bars), empty0 = saddr(bars + stages);
    const uint32_t tfull0 = saddr(bars + 2 * stages), tempty0 = saddr(bars + 2 * stages + 2);
    const uint32_t drain = saddr(bars + 2 * stages + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 4);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(saddr(tmem_slot), kTmemCols);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    const TcProblem *__restrict__ probs = args.probs;

    if (warp == 0) {
        // ======================= TMA producer =======================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t tau = blockIdx.x; tau < args.total_tiles && ok; tau += gridDim.x) {
                const TileInfo ti = decode(probs, args.n_probs, args.ov, tau, BN);
                const TcProblem &P = probs[ti.p];
                for (int s = 0; s < P.S && ok; ++s) {
                    const int xw = s * P.F3 + 3 * ti.t;
                    const int c = xw % P.n_copies;
                    for (int kb = 0; kb < P.nkb; ++kb) {
                        if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, args.err, DEV_TIMEOUT_TMA)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = full0 + 8 * stage;
                        mbar_expect_tx(fb, kStageBytes);
                        uint8_t *st = tiles + (size_t)stage * kStageBytes;
#pragma unroll
                        for (int pl = 0; pl < kPlanes; ++pl) {
                            tma_load_2d(saddr(st + pl * kABytes), &P.mapA[pl][c], fb,
                                        xw - c + kb * kBK, ti.m0);
                            tma_load_2d(saddr(st + kPlanes * kABytes + pl * kBBytes), &P.mapB[pl],
                                        fb, s * P.Kseg + kb * kBK, ti.n0);
                        }
                        if (++stage == stages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
            // drain: wait until the last fill of every stage has landed
            for (int k = 0; k < stages; ++k) {
                if (--stage < 0) {
                    stage = stages - 1;
                    phase ^= 1;
                }
                // the most recent fill of `stage` used parity `phase`; if that stage was never
                // filled, its barrier is still in phase 0 and parity 1 reads as complete
                mbar_wait(full0 + 8 * stage, phase, args.err, DEV_TIMEOUT_TMA);
            }
        }
    } else if (warp == 1) {
        // ======================= MMA issuer =======================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t v = 0;
            bool ok = true;
            for (int64_t tau = blockIdx.x; tau < args.total_tiles && ok; tau += gridDim.x, ++v) {
                const TileInfo ti = decode(probs, args.n_probs, args.ov, tau, BN);
                const TcProblem &P = probs[ti.p];
                const uint32_t acc = v & 1, use = v >> 1;
                if (!mbar_wait(tempty0 + 8 * acc, (use & 1) ^ 1, args.err, DEV_TIMEOUT_MMA)) {
                    ok = false;
                    break;
                }
                tc_after();
                const uint32_t d = tmem + acc * BN;
                const int nk = P.S * P.nkb;
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase, args.err, DEV_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc_after();
                    uint8_t *st = tiles + (size_t)stage * kStageBytes;
                    const uint64_t a0 = sdesc(saddr(st), SWB);
                    const uint64_t b0 = sdesc(saddr(st + kPlanes * kABytes), SWB);
#pragma unroll
                    for (int ks = 0; ks < kKSteps; ++ks) {
                        const uint64_t off = (uint64_t)(ks * 32) >> 4;
                        const uint32_t first = (kb | ks) != 0;
                        if (kPlanes == 1) {
                            tc_mma<kTF32>(d, a0 + off, b0 + off, kIdesc, first);
                        } else {
                            const uint64_t a1 = sdesc(saddr(st + kABytes), SWB);
                            const uint64_t b1 = sdesc(saddr(st + 2 * kABytes + kBBytes), SWB);
                            tc_mma<false>(d, a0 + off, b0 + off, kIdesc, first);  // hi*hi
                            tc_mma<false>(d, a0 + off, b1 + off, kIdesc, 1u);     // hi*lo
                            tc_mma<false>(d, a1 + off, b0 + off, kIdesc, 1u);     // lo*hi
                        }
                    }
                    tc_commit(empty0 + 8 * stage);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                tc_commit(tfull0 + 8 * acc);
            }
            // drain every MMA this thread issued before TMEM is released
            tc_commit(drain);
            mbar_wait(drain, 0, args.err, DEV_TIMEOUT_MMA);
        }
    } else {
        // ======================= epilogue =======================
        const int et = threadIdx.x - 64;          // 0..127
        const int q4 = warp & 3;                  // TMEM lane quarter of this warp
        const int r = q4 * 32 + lane;             // accumulator row = tile row
        float *bins = reinterpret_cast<float *>(epi + EL.bins);
        float *fb = reinterpret_cast<float *>(epi + EL.fb);
        double *cacc = reinterpret_cast<double *>(epi + EL.cacc);
        double *qacc = reinterpret_cast<double *>(epi + EL.qacc);
        double *qred = reinterpret_cast<double *>(epi + EL.qred);
        float4 *colgeo = reinterpret_cast<float4 *>(epi + EL.colgeo);
        float4 *colcs = reinterpret_cast<float4 *>(epi + EL.colcs);
        float *boxred = reinterpret_cast<float *>(epi + EL.boxred);
        for (int k = et; k < (args.NW + 1) * kBinStride; k += kEpiThreads) bins[k] = 0.f;
        for (int k = et; k < args.NB; k += kEpiThreads) {
            fb[k] = 0.f;
            cacc[k] = 0.0;
        }
        for (int k = et; k < args.NQ; k += kEpiThreads) qacc[k] = 0.0;

        int cur_p = -1, cur_t = -1;
        uint32_t v = 0;
        bool ok = true;
        // per-CTA FP64 sums of the current (problem, t), added to the outputs when it changes
        auto flush_acc = [&](int p, int t) {
            const EpiParams &E = probs[p].epi;
            double *Cs = args.ov.active ? args.ov.C_sum : E.C_sum;
            double *Qs = args.ov.active ? args.ov.Sq_sum : E.Sq_sum;
            for (int b = et; b < E.n_bins; b += kEpiThreads) {
                if (cacc[b] != 0.0) atomicAdd(&Cs[(int64_t)t * E.n_bins + b], cacc[b]);
                cacc[b] = 0.0;
            }
            for (int q = et; q < E.n_q; q += kEpiThreads) {
                if (qacc[q] != 0.0) atomicAdd(&Qs[(int64_t)t * E.n_q + q], qacc[q]);
                qacc[q] = 0.0;
            }
        };
        for (int64_t tau = blockIdx.x; tau < args.total_tiles; tau += gridDim.x, ++v) {
            const TileInfo ti = decode(probs, args.n_probs, args.ov, tau, BN);
            const TcProblem &P = probs[ti.p];
            const EpiParams &E = P.epi;
            const int i = ti.m0 + r;
            const bool row_ok = i < ti.row_end;
            const int ic = row_ok ? i : ti.m0;
            const bool lattice = E.geom == ASD_GEOM_LATTICE;
            // column geometry of this tile
            for (int c = et; c < BN; c += kEpiThreads) {
                const int j = min(ti.n0 + c, P.N - 1);
                if (lattice) {
                    const int4 g = E.coords[j];
                    colgeo[c] = make_float4(__int_as_float(g.x), __int_as_float(g.y),
                                            __int_as_float(g.z), 0.f);
                } else {
                    colgeo[c] = E.pos[j];
                }
            }
            const int4 ri = E.coords[ic];
            const float4 rp = E.pos[ic];
            // bounding boxes for the bin window (only when the bins do not all fit)
            if (E.use_window) {
                float v6[12];
                v6[0] = v6[3] = rp.x;
                v6[1] = v6[4] = rp.y;
                v6[2] = v6[5] = rp.z;
                float cl[3] = {3e38f, 3e38f, 3e38f}, ch[3] = {-3e38f, -3e38f, -3e38f};
                for (int c = et; c < BN; c += kEpiThreads) {
                    const int j = min(ti.n0 + c, P.N - 1);
                    const float4 pj = E.pos[j];
                    cl[0] = fminf(cl[0], pj.x); ch[0] = fmaxf(ch[0], pj.x);
                    cl[1] = fminf(cl[1], pj.y); ch[1] = fmaxf(ch[1], pj.y);
                    cl[2] = fminf(cl[2], pj.z); ch[2] = fmaxf(ch[2], pj.z);
                }
                for (int a = 0; a < 3; ++a) {
                    v6[6 + a] = cl[a];
                    v6[9 + a] = ch[a];
                }
                if (!row_ok) {
                    for (int a = 0; a < 3; ++a) {
                        v6[a] = 3e38f;
                        v6[3 + a] = -3e38f;
                    }
                }
                for (int o = 16; o > 0; o >>= 1)
                    for (int k = 0; k < 12; ++k) {
                        const float w = __shfl_xor_sync(0xffffffffu, v6[k], o);
                        v6[k] = ((k % 6) < 3) ? fminf(v6[k], w) : fmaxf(v6[k], w);
                    }
                if (lane == 0)
                    for (int k = 0; k < 12; ++k) boxred[q4 * 12 + k] = v6[k];
            }
            epi_sync();  // colgeo / boxred ready; previous tile fully flushed
            if (ti.p != cur_p || ti.t != cur_t) {
                if (cur_p >= 0) flush_acc(cur_p, cur_t);
                cur_p = ti.p;
                cur_t = ti.t;
            }
            int blo = 0;
            if (E.use_window) {
                float d2min = 0.f;
                for (int a = 0; a < 3; ++a) {
                    float rl = 3e38f, rh = -3e38f, cl = 3e38f, ch = -3e38f;
                    for (int w = 0; w < 4; ++w) {
                        rl = fminf(rl, boxred[w * 12 + a]);
                        rh = fmaxf(rh, boxred[w * 12 + 3 + a]);
                        cl = fminf(cl, boxred[w * 12 + 6 + a]);
                        ch = fmaxf(ch, boxred[w * 12 + 9 + a]);
                    }
                    float gap = fmaxf(0.f, fmaxf(cl - rh, rl - ch));
                    if (lattice && E.periodic) {
                        const float L = a == 0 ? E.Lx : a == 1 ? E.Ly : E.Lz;
                        gap = fminf(gap, fmaxf(0.f, fmaxf(cl + L - rh, rl - (ch + L))));
                        gap = fminf(gap, fmaxf(0.f, fmaxf(cl - L - rh, rl - (ch - L))));
                    }
                    d2min += gap * gap;
                }
                blo = max(0, bin_of_d2(d2min * 0.999f, E.inv_w, E.n_bins, E.thr) - 1);
            }

            const uint32_t acc = v & 1, use = v >> 1;
            const bool got = mbar_wait(tfull0 + 8 * acc, use & 1, args.err, DEV_TIMEOUT_EPI);
            ok = epi_sync_and(got);
            if (!ok) break;
            tc_after();
            const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + acc * BN;

            if (E.n_bins > 0) {
                float *mybins = bins + r;
                const int NWp = E.use_window ? args.NW : E.n_bins;
                for (int ch = 0; ch < BN / 32; ++ch) {
                    uint32_t g[32];
                    tmem_ld32(tbase + ch * 32, g);
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const float val = row_ok ? __uint_as_float(g[k]) : 0.f;
                        const float4 cg = colgeo[ch * 32 + k];
                        float d2;
                        if (lattice) {
                            int4 cj = make_int4(__float_as_int(cg.x), __float_as_int(cg.y),
                                                __float_as_int(cg.z), 0);
                            d2 = lattice_d2(ri, cj, E.Lx, E.Ly, E.Lz, E.periodic);
                        } else {
                            d2 = position_d2(rp, cg);
                        }
                        const int b = bin_of_d2(d2, E.inv_w, E.n_bins, E.thr);
                        const int lb = b - blo;
                        const bool inwin = (unsigned)lb < (unsigned)NWp;
                        mybins[(inwin ? lb : args.NW) * kBinStride] += val;
                        if (!inwin && b < E.n_bins) atomicAdd(&fb[b], val);
                    }
                }
            }
            if (E.n_q > 0) {
                for (int qc = 0; qc < E.n_q; qc += kQC) {
                    const int nqc = min(kQC, E.n_q - qc);
                    epi_sync();  // previous users of colcs / qred are done
                    for (int k = et; k < BN * kQC / 2; k += kEpiThreads) {
                        const int c = k / (kQC / 2), q2 = (k % (kQC / 2)) * 2;
                        const int j = min(ti.n0 + c, P.N - 1);
                        float2 w0 = make_float2(0.f, 0.f), w1 = w0;
                        if (q2 < nqc) w0 = E.cs[(int64_t)j * E.n_q + qc + q2];
                        if (q2 + 1 < nqc) w1 = E.cs[(int64_t)j * E.n_q + qc + q2 + 1];
                        colcs[k] = make_float4(w0.x, w0.y, w1.x, w1.y);
                    }
                    float cr[kQC], sr[kQC], u[kQC], vv[kQC];
#pragma unroll
                    for (int q = 0; q < kQC; ++q) {
                        const float2 w = q < nqc ? E.cs[(int64_t)ic * E.n_q + qc + q]
                                                 : make_float2(0.f, 0.f);
                        cr[q] = w.x;
                        sr[q] = w.y;
                        u[q] = 0.f;
                        vv[q] = 0.f;
                    }
                    epi_sync();
                    for (int ch = 0; ch < BN / 32; ++ch) {
                        uint32_t g[32];
                        tmem_ld32(tbase + ch * 32, g);
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const float val = row_ok ? __uint_as_float(g[k]) : 0.f;
                            const float4 *w = colcs + (ch * 32 + k) * (kQC / 2);
#pragma unroll
                            for (int q2 = 0; q2 < kQC / 2; ++q2) {
                                const float4 w4 = w[q2];
                                u[2 * q2] = fmaf(w4.x, val, u[2 * q2]);
                                vv[2 * q2] = fmaf(w4.y, val, vv[2 * q2]);
                                u[2 * q2 + 1] = fmaf(w4.z, val, u[2 * q2 + 1]);
                                vv[2 * q2 + 1] = fmaf(w4.w, val, vv[2 * q2 + 1]);
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kQC; ++q) {
                        double c = (double)fmaf(cr[q], u[q], sr[q] * vv[q]);
                        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                        if (lane == 0) qred[q4 * kQC + q] = c;
                    }
                    epi_sync();
                    if (et < nqc)
                        qacc[qc + et] += qred[et] + qred[kQC + et] + qred[2 * kQC + et] +
                                         qred[3 * kQC + et];
                }
            }
            // accumulator buffer free for the MMA warp
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
            epi_sync();  // all private bins written
            if (E.n_bins > 0) {
                const int NWp = E.use_window ? args.NW : E.n_bins;
                for (int b = et; b < NWp; b += kEpiThreads) {
                    float *row = bins + b * kBinStride;
                    double s = 0.0;
                    for (int x = 0; x < kBM; ++x) {
                        s += (double)row[x];
                        row[x] = 0.f;
                    }
                    if (blo + b < E.n_bins) cacc[blo + b] += s;
                }
                for (int b = et; b < E.n_bins; b += kEpiThreads) {
                    if (fb[b] != 0.f) {
                        cacc[b] += (double)fb[b];
                        fb[b] = 0.f;
                    }
                }
            }
        }
        epi_sync();
        if (ok && cur_p >= 0) flush_acc(cur_p, cur_t);
    }
    __syncwarp();
    __syncthreads();
    if (warp == 1) {
        tc_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

template <int FORM, int BN, int SWB>
int launch_one(const LaunchArgs &a, size_t smem, int grid, cudaStream_t s)
{
    auto k = pc_tc_kernel<FORM, BN, SWB>;
    ASD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kThreads, smem, s>>>(a);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // namespace

size_t tc_epilogue_smem(int NW, int n_bins, int n_q, int BN)
{
    return epi_layout(NW, n_bins, n_q, BN).total;
}

int tc_configure(asd_corr_plan *p)
{
    const size_t cap = 232448 - 1024 /*alignment slack*/ - 1024 /*barriers*/;
    const size_t stage_bytes = (size_t)p->n_planes * (kBM + p->BN) * p->swizzle_bytes;
    // private bins: as many as fit with at least 3 stages (2 when tight)
    int NW = p->n_bins;
    p->use_window = 0;
    auto epi = [&](int nw) { return tc_epilogue_smem(nw, p->n_bins, p->n_q, p->BN); };
    for (int min_st = 3; min_st >= 2; --min_st) {
        NW = p->n_bins;
        while (NW > 8 && epi(NW) + min_st * stage_bytes > cap) NW = (NW * 3) / 4;
        if (epi(NW) + min_st * stage_bytes <= cap) break;
    }
    if (epi(NW) + 2 * stage_bytes > cap) {
        set_error_text("epilogue does not fit shared memory");
        return ASD_EUNSUPPORTED;
    }
    if (NW < p->n_bins) p->use_window = 1;
    if (p->n_bins == 0) NW = 0;
    p->NW = NW;
    int st = (int)((cap - epi(NW)) / stage_bytes);
    if (st > 8) st = 8;
    if (p->d.stages > 0 && p->d.stages < st) st = p->d.stages;
    p->stages = st;
    p->smem_bytes = epi(NW) + (size_t)p->stages * stage_bytes + 2048;
    // more than half of the SM's shared memory: never two CTAs (and TMEM owners) per SM
    if (p->smem_bytes < kMinSmem) p->smem_bytes = kMinSmem;
    return ASD_OK;
}

int launch_tc(const TcProblem *d_probs, int n_probs, int64_t total_tiles, TcOverride ov, int prec,
              int BN, int swizzle_bytes, int stages, size_t smem, int max_nw, int max_nb,
              int max_nq, int sm_count, cudaStream_t s)
{
    if (total_tiles <= 0) return ASD_OK;
    LaunchArgs a{};
    a.probs = d_probs;
    a.n_probs = n_probs;
    a.total_tiles = total_tiles;
    a.ov = ov;
    a.stages = stages;
    a.NW = max_nw;
    a.NB = max_nb;
    a.NQ = max_nq;
    a.err = device_error_word();
    if (!a.err) return ASD_ECUDA;
    (void)swizzle_bytes;
    const int grid = (int)(total_tiles < sm_count ? total_tiles : sm_count);
    switch (prec) {
    case ASD_BF16:
        return BN == 256 ? launch_one<ASD_BF16, 256, 128>(a, smem, grid, s)
                         : launch_one<ASD_BF16, 128, 128>(a, smem, grid, s);
    case ASD_TF32:
        return BN == 256 ? launch_one<ASD_TF32, 256, 128>(a, smem, grid, s)
                         : launch_one<ASD_TF32, 128, 128>(a, smem, grid, s);
    case ASD_SPLIT_BF16:
        return BN == 256 ? launch_one<ASD_SPLIT_BF16, 256, 64>(a, smem, grid, s)
                         : launch_one<ASD_SPLIT_BF16, 128, 64>(a, smem, grid, s);
    default:
        return ASD_EINVAL;
    }
}

}  // namespace asd
