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
//               each stage back to the ring and each finished work item to the epilogue;
//   warps 2..   epilogue (EW = 4 or 8 warps): reads the accumulator from TMEM and
//               reduces it -- per-thread private FP32 bins in shared memory
//               (conflict-free [bin][row] layout), phase weights from per-site cos/sin
//               tables -- then FP64 per-CTA sums and FP64 atomics into the outputs.
//
// The accumulator living in TMEM plays the role of the paper's OTF_SM shared-memory
// staging of the C tile (Section 3.4): the epilogue never holds the tile in registers.
// The per-pair phase factor uses cos(a - b) = cos a cos b + sin a sin b (and
// sin(a - b) = sin a cos b - cos a sin b for the sine part) on tables made once per
// plan, so no transcendental is evaluated per pair (the register-spill problem of the
// paper's OTF_REG variant).
//
// Persistent: one CTA per SM takes (problem, t, K chunk, row tile, column tile) work
// items in grouped raster order (raster_m row tiles per group, 16 by default) so
// concurrently running CTAs share A and B panels in L2; the TMA thread claims each item
// from a global counter (or, static, takes every n-th) and passes its index to the other
// roles.  Several problems (a batched ensemble) share the list.  Every wait is bounded: after
// kTimeoutNs a role records an error in the device error word and stops; the CTA then
// drains its own in-flight copies and MMAs, frees TMEM and exits.
#pragma once

#include <cuda_bf16.h>

#include "asd_internal.h"
#include "fma2.cuh"
#include "geom.cuh"

namespace asd {
namespace {

// Epilogue warps EW (template parameter): 4 (one per TMEM lane quarter, all columns) or
// 8 (two per quarter, half the columns each).  Threads = TMA warp + MMA warp + EW warps.
constexpr int kMaxEpiWarps = 8;
constexpr int kQC = kQChunk;                  // (cos, sin) rows are padded to whole kQC
// q-vectors per pass of the phase loop: 8 with 4 epilogue warps; 4 with 8 warps, whose
// register budget (two warps per scheduler) has no room for 8 q of accumulators
__host__ __device__ constexpr int qp_of(int ew) { return ew == 8 ? 4 : 8; }
static_assert(kQC % qp_of(4) == 0 && kQC % qp_of(8) == 0, "q passes tile the padded q rows");
constexpr unsigned long long kTimeoutNs = 4000000000ull;
// Work items are handed from the TMA thread to the MMA thread and the epilogue warps
// through a ring of kWQ slots in shared memory.  With the dynamic schedule the TMA thread
// claims each item from a global counter, so the items in flight across the grid stay
// together whatever each item costs (L2 reuse of A / B panels, no drift, balanced tail);
// the static schedule takes items cid, cid + gridDim.x, ...
constexpr int kWQ = 4;
// Private bins are a [bin][128 * EW/4] array: epilogue thread (row r, column half h)
// only ever touches column r + 128 h, i.e. bank r mod 32, so the per-pair accumulation
// is free of bank conflicts whatever the bins of the 32 lanes are (with an odd stride,
// bins that fall as the row index rises put a whole warp on one bank).  The per-tile
// flush reads whole bin rows warp-cooperatively (bin_stride, asd_internal.h).

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
__device__ __noinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, int *err, int code,
                                          unsigned long long limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 1023u) == 0 && gtimer() - t0 > limit_ns) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, int code)
{
    return mbar_wait_for(bar, parity, err, code, kTimeoutNs);
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

// 16 lanes x 256 bits, 4 repetitions along the columns (32 columns): register 4m + e
// holds (lane l/4, column 8m + 2(l%4) + e) and register 4m + 2 + e holds (lane l/4 + 8,
// the same column), l = this thread's lane in the warp.  Valid after tmem_wait16x2.
__device__ __forceinline__ void tmem_ld16x256b_x4(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Wait for two 16x256b.x4 loads, tied to their registers.
__device__ __forceinline__ void tmem_wait16x2(uint32_t (&a)[16], uint32_t (&b)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                   "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]),
                   "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]),
                   "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                   "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]),
                   "+r"(b[14]), "+r"(b[15])
                 :
                 : "memory");
}

// Asynchronous 16-byte global -> shared copy (completion per thread by commit groups).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Issue half of tmem_ld32: the registers are valid only after tmem_wait32 on them.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32])
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
}

// Wait for the TMEM loads of this thread; tied to the registers so no use of them can be
// scheduled before it.
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32])
{
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

__device__ __forceinline__ void epi_sync(int nthreads)
{
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Epilogue barrier that also ANDs a flag over the 128 epilogue threads, so that every
// thread takes the same branch after a bounded wait.
__device__ __forceinline__ bool epi_sync_and(bool v, int nthreads)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(nthreads)
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
    uint32_t cacc, qacc, qred, fb, colgeo, colpk, colcs, rowcs, boxred, var, total;
};

__host__ __device__ inline uint32_t take(uint32_t &o, uint32_t bytes)
{
    o = (o + 15u) & ~15u;
    uint32_t r = o;
    o += bytes;
    return r;
}

// The per-problem part of the epilogue's shared memory: the private bins (NW + 1 rows,
// the last one the trash row of dropped pairs) followed by the bin threshold pairs (FP32)
// or, for lattices, the d2 -> bin table (uint16).  A batched launch sizes it for the
// largest problem and lays it out again whenever the problem changes.
__host__ __device__ inline uint32_t var_bins_bytes(int NW, int ew)
{
    return (4u * (NW + 1) * bin_stride(ew) + 15u) & ~15u;
}
__host__ __device__ inline uint32_t var_bytes(int NW, int nb, int nlut, int ew)
{
    const uint32_t tb = 8u * (nb + 1), lb = 2u * nlut;
    return var_bins_bytes(NW, ew) + (((tb > lb ? tb : lb) + 15u) & ~15u);
}

// Epilogue shared memory: the fixed arrays (sized for the largest n_bins / n_q of the
// launch) and the per-problem region of `vb` bytes.
__host__ __device__ inline EpiLayout epi_layout(uint32_t vb, int nb, int nq, int BN, int ew)
{
    EpiLayout L;
    uint32_t o = 0;
    L.cacc = take(o, 8u * (nb > 0 ? nb : 1));
    // phase sums per q: (cosine, sine) parts
    L.qacc = take(o, 8u * 2 * (nq > 0 ? nq : 1));
    // one slot per (pass, warp, q): the passes of a tile are reduced once at its end
    const int qp = qp_of(ew);
    L.qred = take(o, 8u * 2 * ew * (nq > 0 ? (nq + qp - 1) / qp * qp : qp));
    L.fb = take(o, 4u * (nb > 0 ? nb : 1));
    L.colgeo = take(o, 16u * BN);
    L.colpk = take(o, 4u * BN);
    // phase weights of one pass, double buffered: columns (BN) and rows (128) of the tile
    L.colcs = nq > 0 ? take(o, 2u * 8u * BN * qp) : 0u;
    L.rowcs = nq > 0 ? take(o, 2u * 8u * kBM * qp) : 0u;
    L.boxred = take(o, 4u * ew * 12);
    L.var = take(o, vb);
    L.total = (o + 1023u) & ~1023u;
    return L;
}

struct TileInfo {
    int p, t, m0, n0, row_end;
    int kg0, kg1;  // K blocks [kg0, kg1) of the S * nkb blocks of a full row
};

// Work item `tau` -> (problem, t, K chunk, row tile, column tile).  K chunks split the
// contraction so that each partial accumulator starts from zero.
// Per-role walk over the work list.  A role visits its work items in increasing order,
// so the problem of the next item is found by stepping forward from the current one, and
// the fields that decoding needs stay in registers until the problem changes (a batched
// launch would otherwise repeat a search over the descriptors in global memory per item).
struct WorkCursor {
    int p = -1;
    int64_t begin = 0, end = 0;  // flattened items [begin, end) belong to problem p
    int tiles_m, tiles_n, kch, G, nk, row_begin, row_end;
    int64_t per_kc;
};

__device__ __forceinline__ TileInfo decode(WorkCursor &cu, const TcProblem *__restrict__ probs,
                                           int n_probs, const TcOverride &ov, int64_t tau,
                                           int BN)
{
    if (cu.p < 0 || tau >= cu.end) {
        int p = cu.p < 0 ? 0 : cu.p;
        if (n_probs > 1) {
            if (cu.p < 0) {
                int lo = 0, hi = n_probs - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (probs[mid].tile_begin <= tau) lo = mid;
                    else hi = mid - 1;
                }
                p = lo;
            } else {
                while (p + 1 < n_probs && probs[p + 1].tile_begin <= tau) ++p;
            }
        }
        const TcProblem &P = probs[p];
        cu.p = p;
        const int tiles_m = ov.active ? ov.tiles_m : P.tiles_m;
        cu.begin = ov.active ? 0 : P.tile_begin;
        cu.end = cu.begin + (ov.active ? ov.n_tiles : P.n_tiles);
        cu.tiles_m = tiles_m;
        cu.tiles_n = P.tiles_n;
        cu.kch = P.k_chunks;
        cu.G = max(1, P.group_m);
        cu.nk = P.S * P.nkb;
        cu.row_begin = ov.active ? ov.row_begin : P.row_begin;
        cu.row_end = ov.active ? ov.row_end : P.row_end;
        cu.per_kc = (int64_t)cu.tiles_m * cu.tiles_n;
    }
    const int64_t l = tau - cu.begin;
    TileInfo ti;
    ti.p = cu.p;
    ti.t = (int)(l / (cu.per_kc * cu.kch));
    const int64_t rem0 = l % (cu.per_kc * cu.kch);
    const int kc = (int)(rem0 / cu.per_kc);
    const int64_t rem = rem0 % cu.per_kc;
    const int64_t gspan = (int64_t)cu.G * cu.tiles_n;
    const int first_m = (int)(rem / gspan) * cu.G;
    const int gsz = min(cu.G, cu.tiles_m - first_m);
    const int64_t r2 = rem % gspan;
    ti.m0 = cu.row_begin + (first_m + (int)(r2 % gsz)) * kBM;
    ti.n0 = (int)(r2 / gsz) * BN;
    ti.row_end = cu.row_end;
    ti.kg0 = (int)((int64_t)kc * cu.nk / cu.kch);
    ti.kg1 = (int)((int64_t)(kc + 1) * cu.nk / cu.kch);
    return ti;
}

// Exact bin of an FP32 d2 from a table of threshold pairs thr2[k] = (thr[k], thr[k+1]),
// thr[k] = (k w)^2 rounded up to FP32: a first guess from the square root, then one
// 8-byte load corrects it by one either way (the same result as two dependent fix-ups,
// since the guess is within one bin).  Returns 0 .. n_bins + 1 (>= n_bins: dropped).
__device__ __forceinline__ int bin_of_d2_pair(float d2, float inv_w, int nb,
                                              const float2 *__restrict__ thr2)
{
    const float r = d2 * rsqrtf(fmaxf(d2, 1e-30f));
    const int k = min((int)(r * inv_w), nb);
    const float2 t = thr2[k];
    return k + (d2 >= t.y ? 1 : 0) - (d2 < t.x ? 1 : 0);
}

// Per-tile constants of the binning epilogue, held in registers.
struct BinArgs {
    int Lx, Ly, Lz, periodic;
    float inv_w;
    int nb, blo, nwp, trash;
};

enum { BIN_LUT = 0, BIN_THR = 1, BIN_POS = 2 };

// Bin 32 consecutive columns of one accumulator row.  Phase 1 computes the exact bin
// slot of every pair (loads of geometry and tables only, so the 32 independent chains
// overlap); phase 2 adds the 32 values into this thread's private bins (its column of
// the [bin][STRIDE] array) or, for bins outside the window, into the shared fallback
// bins.  Without a window, blo = 0 and nwp = nb, so every kept bin is private.
// MODE: BIN_LUT (lattice, d2 -> bin table), BIN_THR (lattice, thresholds), BIN_POS
// (FP32 positions, thresholds).
template <int MODE, int STRIDE>
__device__ __forceinline__ void bin_chunk(const uint32_t (&g)[32], bool row_ok, int4 ri, float4 rp,
                                          const float4 *__restrict__ cgeo,
                                          const float *__restrict__ thr,
                                          float *__restrict__ myb, float *__restrict__ fb,
                                          const BinArgs ba)
{
    int slot[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float4 cg = cgeo[k];
        int b;
        if (MODE == BIN_POS) {
            b = bin_of_d2_pair(position_d2(rp, cg), ba.inv_w, ba.nb,
                               reinterpret_cast<const float2 *>(thr));
        } else {
            const int4 cj = make_int4(__float_as_int(cg.x), __float_as_int(cg.y),
                                      __float_as_int(cg.z), 0);
            const int d2 = lattice_d2i(ri, cj, ba.Lx, ba.Ly, ba.Lz, ba.periodic);
            if (MODE == BIN_LUT)
                b = reinterpret_cast<const uint16_t *>(thr)[d2];
            else
                b = bin_of_d2_pair((float)d2, ba.inv_w, ba.nb,
                                   reinterpret_cast<const float2 *>(thr));
        }
        const int lb = b - ba.blo;
        slot[k] = (unsigned)lb < (unsigned)ba.nwp ? lb : (b < ba.nb ? -1 - b : ba.trash);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        // rows past the range: their accumulator rows may come from A rows that were
        // never prepared, so the value is replaced (a product with 0 would keep a NaN)
        const float val = row_ok ? __uint_as_float(g[k]) : 0.f;
        if (slot[k] < 0) atomicAdd(&fb[-1 - slot[k]], val);
        else myb[slot[k] * STRIDE] += val;
    }
}

// Fast lattice form of bin_chunk's first phase (EpiParams::fast): coordinates packed one per byte
// (x | y<<8 | z<<16), the per-axis minimum image from byte-wise |a - b| and
// min(d, L - d), d2 from a byte dot product, then the private-bin word offset from the
// d2 table (LUT, entries pre-scaled by the bin stride) or from the thresholds (THR).
// Dropped pairs land in the trash row, so no pair takes a branch.
template <bool LUT, int STRIDE>
__device__ __forceinline__ void pk_offsets(uint32_t (&off)[32], uint32_t rpk, uint32_t Lpk,
                                           const uint4 *__restrict__ cpk,
                                           const void *__restrict__ tab, float inv_w, int nb,
                                           uint32_t trash_off)
{
#pragma unroll
    for (int k4 = 0; k4 < 8; ++k4) {
        const uint4 c4 = cpk[k4];
        const uint32_t cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint32_t d = __vabsdiffu4(cc[u], rpk);
            d = __vminu4(d, __vsub4(Lpk, d));
            const uint32_t d2 = __dp4a(d, d, 0u);
            if (LUT) {
                off[4 * k4 + u] = reinterpret_cast<const uint16_t *>(tab)[d2];
            } else {
                const int b =
                    bin_of_d2_pair((float)d2, inv_w, nb, reinterpret_cast<const float2 *>(tab));
                off[4 * k4 + u] = b < nb ? (uint32_t)(b * STRIDE) : trash_off;
            }
        }
    }
}

using LaunchArgs = TcLaunchArgs;

// ------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------
template <int FORM, int BN, int SWB, int EW>
__global__ void __launch_bounds__(64 + 32 * EW, 1) pc_tc_kernel(const __grid_constant__ LaunchArgs args)
{
    constexpr int kEpiWarps = EW;
    constexpr int kEpiThreads = 32 * EW;
    constexpr int kBinStride = bin_stride(EW);
    constexpr int kHalves = EW / 4;
    constexpr int kQP = qp_of(EW);
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
    const EpiLayout EL = epi_layout(args.VB, args.NB, args.NQ, BN, EW);
    uint64_t *bars = reinterpret_cast<uint64_t *>(epi + EL.total);
    // bars: full[stages], empty[stages], tfull[2], tempty[2], drain, wqfull[kWQ],
    // wqempty[kWQ]; then the work ring wq[kWQ] and the TMEM address slot
    const uint32_t wqfull0 = saddr(bars + 2 * stages + 5);
    const uint32_t wqempty0 = saddr(bars + 2 * stages + 5 + kWQ);
    volatile int64_t *wq = reinterpret_cast<volatile int64_t *>(bars + 2 * stages + 5 + 2 * kWQ);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 5 + 3 * kWQ);
    const uint32_t full0 = saddr(bars), empty0 = saddr(bars + stages);
    const uint32_t tfull0 = saddr(bars + 2 * stages), tempty0 = saddr(bars + 2 * stages + 2);
    const uint32_t drain = saddr(bars + 2 * stages + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            // a stage is free again once the MMAs that read it have completed
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, kEpiWarps);
        }
        mbar_init(drain, 1);
        for (int k = 0; k < kWQ; ++k) {
            mbar_init(wqfull0 + 8 * k, 1);
            // released by the MMA thread and one lane of every epilogue warp
            mbar_init(wqempty0 + 8 * k, 1 + kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(saddr(tmem_slot), kTmemCols);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    const TcProblem *__restrict__ probs = args.probs;
    const int64_t cid = blockIdx.x, n_ctas = gridDim.x;

    if (warp == 0) {
        // ======================= TMA producer =======================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            WorkCursor cu;
            for (int64_t v = 0; ok; ++v) {
                // publish the next work item (-1: none left) once its ring slot is free
                const int qs = (int)(v % kWQ);
                if (!mbar_wait(wqempty0 + 8 * qs, (uint32_t)((v / kWQ) & 1) ^ 1u, args.err,
                               DEV_TIMEOUT_TMA)) {
                    ok = false;
                    break;
                }
                int64_t tau = args.counter ? (int64_t)atomicAdd(args.counter, 1ull)
                                           : cid + v * n_ctas;
                if (tau >= args.total_tiles) tau = -1;
                wq[qs] = tau;
                mbar_arrive(wqfull0 + 8 * qs);  // release: the slot is visible to the waiters
                if (tau < 0) break;
                const TileInfo ti = decode(cu, probs, args.n_probs, args.ov, tau, BN);
                const TcProblem &P = probs[ti.p];
                for (int kg = ti.kg0; kg < ti.kg1; ++kg) {
                    const int s = kg / P.nkb, kb = kg % P.nkb;
                    const int xw = s * P.F3 + 3 * ti.t;
                    const int c = xw % P.n_copies;
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
                        tma_load_2d(saddr(st + kPlanes * kABytes + pl * kBBytes), &P.mapB[pl], fb,
                                    s * P.Kseg + kb * kBK, ti.n0);
                    }
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1;
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
            WorkCursor cu;
            for (;; ++v) {
                const int qs = (int)(v % kWQ);
                if (!mbar_wait(wqfull0 + 8 * qs, (v / kWQ) & 1, args.err, DEV_TIMEOUT_MMA)) {
                    ok = false;
                    break;
                }
                const int64_t tau = wq[qs];
                mbar_arrive(wqempty0 + 8 * qs);
                if (tau < 0) break;
                const TileInfo ti = decode(cu, probs, args.n_probs, args.ov, tau, BN);
                const uint32_t acc = v & 1, use = v >> 1;
                if (!mbar_wait(tempty0 + 8 * acc, (use & 1) ^ 1, args.err, DEV_TIMEOUT_MMA)) {
                    ok = false;
                    break;
                }
                tc_after();
                const uint32_t d = tmem + acc * BN;
                for (int kg = ti.kg0; kg < ti.kg1; ++kg) {
                    const int kb = kg - ti.kg0;  // 0 for the first block of this chunk
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
        const int ew = warp - 2;                  // epilogue warp 0..7
        const int half = ew >> 2;                 // which part of the columns (EW = 8)
        const int ch0 = half * (BN / 32 / kHalves), ch1 = ch0 + BN / 32 / kHalves;
        // private bins and bin table of the current problem (set when the problem changes)
        float *bins = reinterpret_cast<float *>(epi + EL.var);
        float *fb = reinterpret_cast<float *>(epi + EL.fb);
        double *cacc = reinterpret_cast<double *>(epi + EL.cacc);
        double *qacc = reinterpret_cast<double *>(epi + EL.qacc);
        double *qred = reinterpret_cast<double *>(epi + EL.qred);
        float4 *colgeo = reinterpret_cast<float4 *>(epi + EL.colgeo);
        uint32_t *colpk = reinterpret_cast<uint32_t *>(epi + EL.colpk);
        float4 *colcs = reinterpret_cast<float4 *>(epi + EL.colcs);
        float4 *rowcs = reinterpret_cast<float4 *>(epi + EL.rowcs);
        float *boxred = reinterpret_cast<float *>(epi + EL.boxred);
        float *thr_s = bins;
        for (int k = et; k < args.NB; k += kEpiThreads) {
            fb[k] = 0.f;
            cacc[k] = 0.0;
        }
        for (int k = et; k < 2 * args.NQ; k += kEpiThreads) qacc[k] = 0.0;

        int cur_p = -1, cur_t = -1, tab_p = -1;
        WorkCursor cu;
        // fast lattice binning also needs the private-bin offsets of this launch (the
        // largest window of a batch, plus its trash row) to fit the 16-bit table entries
        auto fast_ok = [&](const EpiParams &E) {
            return E.fast && (E.NW + 1) * kBinStride <= 65536;
        };
        // phase weights of pass `pass` (q = pass*kQP ...) of a tile into buffer pass & 1:
        // the tile's column and row (cos, sin) rows, as asynchronous copies (rows are zero
        // padded to whole chunks, two q per float4; indices past the problem are clamped,
        // their accumulator entries being zero or their rows weighed by 0)
        auto stage_phase = [&](const TileInfo &tq, const TcProblem &Pq, int pass) {
            const float4 *cs4 = reinterpret_cast<const float4 *>(Pq.epi.cs);
            const int64_t qo = (int64_t)pass * kQP / 2;
            const int64_t rl = Pq.epi.nq_pad / 2;
            float4 *cb = colcs + (pass & 1) * (BN * kQP / 2);
            float4 *rb = rowcs + (pass & 1) * (kBM * kQP / 2);
            // shared layouts: columns [c/8][q2][c%8] (the 4 column pairs a warp reads at
            // once are 32 bytes apart: distinct banks), rows [q2][row]
            for (int k = et; k < BN * kQP / 2; k += kEpiThreads) {
                const int c = k / (kQP / 2), q2 = k % (kQP / 2);
                const int j = min(tq.n0 + c, Pq.N - 1);
                cp_async16(cb + ((c >> 3) * (kQP / 2) + q2) * 8 + (c & 7),
                           cs4 + (int64_t)j * rl + qo + q2);
            }
            for (int k = et; k < kBM * kQP / 2; k += kEpiThreads) {
                const int r = k / (kQP / 2), q2 = k % (kQP / 2);
                const int i = min(tq.m0 + r, Pq.N - 1);
                cp_async16(rb + q2 * kBM + r, cs4 + (int64_t)i * rl + qo + q2);
            }
            cp_async_commit();
        };
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
            for (int q = et; q < E.n_q; q += kEpiThreads)
                for (int part = 0; part < E.q_parts; ++part) {
                    double &acc = qacc[2 * q + part];
                    if (acc != 0.0)
                        atomicAdd(&Qs[((int64_t)t * E.n_q + q) * E.q_parts + part], acc);
                    acc = 0.0;
                }
        };
        for (;; ++v) {
            const int qs = (int)(v % kWQ);
            {
                const bool gotq = mbar_wait(wqfull0 + 8 * qs, (v / kWQ) & 1, args.err,
                                            DEV_TIMEOUT_EPI);
                ok = epi_sync_and(gotq, kEpiThreads);
                if (!ok) break;
            }
            const int64_t tau = wq[qs];
            __syncwarp();
            if (lane == 0) mbar_arrive(wqempty0 + 8 * qs);
            if (tau < 0) break;
            const TileInfo ti = decode(cu, probs, args.n_probs, args.ov, tau, BN);
            const TcProblem &P = probs[ti.p];
            const EpiParams &E = P.epi;
            const int i = ti.m0 + r;
            const bool row_ok = i < ti.row_end;
            // rows past the range (ragged tiles) read the
            // geometry of a valid site and contribute zeros
            const int ic = row_ok ? i : P.N - 1;
            const bool lattice = E.geom == ASD_GEOM_LATTICE;
            // bin thresholds of this problem, then the column geometry of this tile
            if (E.n_bins > 0 && ti.p != tab_p) {
                // lay out the per-problem region for this problem: every thread is done
                // with the previous problem's bins (flushed and zeroed at each tile's end)
                // and table, then the new bins are zeroed and the new table loaded
                epi_sync(kEpiThreads);
                bins = reinterpret_cast<float *>(epi + EL.var);
                thr_s = reinterpret_cast<float *>(epi + EL.var + var_bins_bytes(E.NW, EW));
                for (int k = et; k < (E.NW + 1) * kBinStride; k += kEpiThreads) bins[k] = 0.f;
                // thresholds, or the lattice d2 -> bin table, of this problem
                if (E.n_lut > 0) {
                    // fast form: entries become private-bin word offsets (the host checked
                    // that (n_bins + 1) * stride fits 16 bits)
                    // (dropped pairs: the trash row E.NW, which no flush reads)
                    uint16_t *lut_s = reinterpret_cast<uint16_t *>(thr_s);
                    for (int k = et; k < E.n_lut; k += kEpiThreads) {
                        const int b = E.lut[k];
                        lut_s[k] = (uint16_t)(fast_ok(E) ? (b < E.n_bins ? b : E.NW) * kBinStride
                                                         : b);
                    }
                } else {
                    float2 *thr2 = reinterpret_cast<float2 *>(thr_s);
                    for (int k = et; k <= E.n_bins; k += kEpiThreads)
                        thr2[k] = make_float2(E.thr[k], E.thr[k + 1]);
                }
                tab_p = ti.p;
            }
            for (int c = et; c < BN; c += kEpiThreads) {
                const int j = min(ti.n0 + c, P.N - 1);
                if (lattice) {
                    const int4 g = E.coords[j];
                    colgeo[c] = make_float4(__int_as_float(g.x), __int_as_float(g.y),
                                            __int_as_float(g.z), 0.f);
                    colpk[c] = (uint32_t)g.x | ((uint32_t)g.y << 8) | ((uint32_t)g.z << 16);
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
                    for (int k = 0; k < 12; ++k) boxred[ew * 12 + k] = v6[k];
            }
            epi_sync(kEpiThreads);  // colgeo / boxred ready; previous tile fully flushed
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
                    for (int w = 0; w < kEpiWarps; ++w) {
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

            if (E.n_q > 0) stage_phase(ti, P, 0);  // lands while the MMAs finish
            const uint32_t acc = v & 1, use = v >> 1;
            const bool got = mbar_wait(tfull0 + 8 * acc, use & 1, args.err, DEV_TIMEOUT_EPI);
            ok = epi_sync_and(got, kEpiThreads);
            if (!ok) break;
            tc_after();
            const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + acc * BN;

            if (E.n_bins > 0) {
                BinArgs ba;
                ba.Lx = E.Lx;
                ba.Ly = E.Ly;
                ba.Lz = E.Lz;
                ba.periodic = E.periodic;
                ba.inv_w = E.inv_w;
                ba.nb = E.n_bins;
                ba.blo = E.use_window ? blo : 0;
                ba.nwp = E.use_window ? E.NW : E.n_bins;
                ba.trash = E.NW;
                const int mode = !lattice ? BIN_POS : (E.n_lut > 0 ? BIN_LUT : BIN_THR);
                if (fast_ok(E)) {
                    // rows past the range skip the pairs (the TMEM loads stay warp-wide)
                    const uint32_t rpk =
                        (uint32_t)ri.x | ((uint32_t)ri.y << 8) | ((uint32_t)ri.z << 16);
                    float *mb = bins + r + kBM * half;
                    const bool lut = E.n_lut > 0;
                    const uint32_t trash_off = (uint32_t)E.NW * kBinStride;
                    for (int ch = ch0; ch < ch1; ++ch) {
                        // the TMEM load runs while the bin offsets are computed
                        uint32_t g[32], off[32];
                        tmem_ld32_issue(tbase + ch * 32, g);
                        const uint4 *cp = reinterpret_cast<const uint4 *>(colpk + ch * 32);
                        if (lut)
                            pk_offsets<true, kBinStride>(off, rpk, E.Lpk, cp, thr_s, E.inv_w,
                                                         E.n_bins, trash_off);
                        else
                            pk_offsets<false, kBinStride>(off, rpk, E.Lpk, cp, thr_s, E.inv_w,
                                                          E.n_bins, trash_off);
                        tmem_wait32(g);
                        if (row_ok) {
#pragma unroll
                            for (int k = 0; k < 32; ++k) mb[off[k]] += __uint_as_float(g[k]);
                        }
                    }
                } else
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t g[32];
                    tmem_ld32(tbase + ch * 32, g);
                    const float4 *cg = colgeo + ch * 32;
                    float *mb = bins + r + kBM * half;
                    if (mode == BIN_LUT)
                        bin_chunk<BIN_LUT, kBinStride>(g, row_ok, ri, rp, cg, thr_s, mb, fb, ba);
                    else if (mode == BIN_THR)
                        bin_chunk<BIN_THR, kBinStride>(g, row_ok, ri, rp, cg, thr_s, mb, fb, ba);
                    else
                        bin_chunk<BIN_POS, kBinStride>(g, row_ok, ri, rp, cg, thr_s, mb, fb, ba);
                }
            }
            if (E.n_q > 0) {
                // Phase weights, kQP q per pass.  The accumulator is read in the 16x256b
                // shape: a thread holds rows {l/4, l/4+8} (+16 for the second half-quarter)
                // and columns {2(l%4), 2(l%4)+1} of every 8-column block, so each (cos, sin)
                // column weight loaded from shared memory serves 4 rows:
                //   u_r(q) = sum_j c_j(q) G_rj,  v_r(q) = sum_j s_j(q) G_rj  (partial over the
                // thread's columns), then sum_r c_r(q) u_r(q) + s_r(q) v_r(q) over the warp.
                // The weights of pass p+1 are copied while pass p computes.
                const int npass = (E.n_q + kQP - 1) / kQP;
                const int cq = 2 * (lane & 3);  // this thread's column pair in a block
                for (int pass = 0; pass < npass; ++pass) {
                    cp_async_wait_all();
                    // everyone's copies of this pass are visible; everyone is done with the
                    // buffer that the next pass's copies overwrite
                    epi_sync(kEpiThreads);
                    if (pass + 1 < npass) stage_phase(ti, P, pass + 1);
                    const float4 *cb = colcs + (pass & 1) * (BN * kQP / 2);
                    const float4 *rb = rowcs + (pass & 1) * (kBM * kQP / 2);
                    float u[4][kQP], vv[4][kQP];
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                        for (int q = 0; q < kQP; ++q) {
                            u[rr][q] = 0.f;
                            vv[rr][q] = 0.f;
                        }
                    // rows of this thread past the range (unprepared A rows): values replaced
                    bool okr[4];
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr)
                        okr[rr] = ti.m0 + q4 * 32 + 16 * (rr >> 1) + 8 * (rr & 1) + (lane >> 2) <
                                  ti.row_end;
                    auto chunk = [&](const uint32_t (&g)[2][16], int ch) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const float4 *w = cb + (ch * 4 + m) * (kQP / 2) * 8 + cq + e;
#pragma unroll
                                for (int q2 = 0; q2 < kQP / 2; ++q2) {
                                    const float4 w4 = w[q2 * 8];
#pragma unroll
                                    for (int rr = 0; rr < 4; ++rr) {
                                        const float gv =
                                            okr[rr] ? __uint_as_float(g[rr >> 1][4 * m + 2 * (rr & 1) + e])
                                                    : 0.f;
                                        fma2(u[rr][2 * q2], vv[rr][2 * q2], w4.x, w4.y, gv);
                                        fma2(u[rr][2 * q2 + 1], vv[rr][2 * q2 + 1], w4.z, w4.w, gv);
                                    }
                                }
                            }
                        }
                    };
                    for (int ch = ch0; ch < ch1; ++ch) {
                        uint32_t g[2][16];
                        tmem_ld16x256b_x4(tbase + ch * 32, g[0]);
                        tmem_ld16x256b_x4(tbase + (16u << 16) + ch * 32, g[1]);
                        tmem_wait16x2(g[0], g[1]);
                        chunk(g, ch);
                    }
                    // row weights of the thread's 4 rows (rows past the range weigh 0):
                    // cosine part c_r u + s_r v, sine part s_r u - c_r v (angle difference)
                    float x[kQP], y[kQP];
#pragma unroll
                    for (int q = 0; q < kQP; ++q) {
                        x[q] = 0.f;
                        y[q] = 0.f;
                    }
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr) {
                        const int rrow = q4 * 32 + 16 * (rr >> 1) + 8 * (rr & 1) + (lane >> 2);
                        const bool ok_r = ti.m0 + rrow < ti.row_end;
#pragma unroll
                        for (int q2 = 0; q2 < kQP / 2; ++q2) {
                            float4 w = rb[q2 * kBM + rrow];
                            if (!ok_r) w = make_float4(0.f, 0.f, 0.f, 0.f);
                            const float u0 = u[rr][2 * q2], v0 = vv[rr][2 * q2];
                            const float u1 = u[rr][2 * q2 + 1], v1 = vv[rr][2 * q2 + 1];
                            x[2 * q2] = fmaf(w.x, u0, fmaf(w.y, v0, x[2 * q2]));
                            x[2 * q2 + 1] = fmaf(w.z, u1, fmaf(w.w, v1, x[2 * q2 + 1]));
                            y[2 * q2] = fmaf(w.y, u0, fmaf(-w.x, v0, y[2 * q2]));
                            y[2 * q2 + 1] = fmaf(w.w, u1, fmaf(-w.z, v1, y[2 * q2 + 1]));
                        }
                    }
                    // sum over the warp's 32 lanes by recursive halving: each exchange sends
                    // the half of the q-values this lane does not keep; after log2(kQP)
                    // steps a lane holds one q (set by its top lane bits), the remaining
                    // exchanges add the lanes that hold the same q
                    constexpr int kLanesPerQ = 32 / kQP;
                    auto warp_sum = [&](float (&z)[kQP]) {
#pragma unroll
                        for (int hh = kQP / 2, o = 16; hh >= 1; hh >>= 1, o >>= 1) {
                            const bool up = (lane & o) != 0;
#pragma unroll
                            for (int k = 0; k < hh; ++k) {
                                const float send = up ? z[k] : z[k + hh];
                                const float keep = up ? z[k + hh] : z[k];
                                z[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                            }
                        }
#pragma unroll
                        for (int o = kLanesPerQ / 2; o >= 1; o >>= 1)
                            z[0] += __shfl_xor_sync(0xffffffffu, z[0], o);
                    };
                    const int qme = lane / kLanesPerQ;
                    double *slot = qred + ((pass * kEpiWarps + ew) * kQP + qme) * 2;
                    warp_sum(x);
                    if (lane % kLanesPerQ == 0) slot[0] = (double)x[0];
                    if (E.q_parts == 2) {
                        warp_sum(y);
                        if (lane % kLanesPerQ == 0) slot[1] = (double)y[0];
                    }
                }
                epi_sync(kEpiThreads);
                for (int q = et; q < E.n_q; q += kEpiThreads)
                    for (int part = 0; part < E.q_parts; ++part) {
                        double sq = 0.0;
                        for (int w = 0; w < kEpiWarps; ++w)
                            sq += qred[(((q / kQP) * kEpiWarps + w) * kQP + q % kQP) * 2 + part];
                        qacc[2 * q + part] += sq;
                    }
            }
            // accumulator buffer free for the MMA warp
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
            epi_sync(kEpiThreads);  // all private bins written
            if (E.n_bins > 0) {
                const int NWp = E.use_window ? E.NW : E.n_bins;
                // epilogue warp ew reduces bins b = ew (mod 8): 8 conflict-free loads per
                // lane, an FP32 tree over the 256 entries, one FP64 add per bin (the FP64
                // pipe is narrow on this part, so FP64 work is kept per bin, not per row)
                for (int b = ew; b < NWp; b += kEpiWarps) {
                    float *row = bins + b * kBinStride;
                    float v = 0.f;
#pragma unroll
                    for (int m = 0; m < kBinStride / 32; ++m) {
                        v += row[lane + 32 * m];
                        row[lane + 32 * m] = 0.f;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0 && blo + b < E.n_bins) cacc[blo + b] += (double)v;
                }
                if (E.use_window) {
                    epi_sync(kEpiThreads);  // the fallback bins update the same accumulators
                    for (int b = et; b < E.n_bins; b += kEpiThreads) {
                        if (fb[b] != 0.f) {
                            cacc[b] += (double)fb[b];
                            fb[b] = 0.f;
                        }
                    }
                }
            }
        }
        cp_async_wait_all();  // no copy into this CTA's shared memory outlives it
        epi_sync(kEpiThreads);
        if (ok && cur_p >= 0) flush_acc(cur_p, cur_t);
    }
    __syncwarp();
    __syncthreads();
    if (warp == 1) {
        tc_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

template <int FORM, int BN, int SWB, int EW>
int launch_one(const LaunchArgs &a, size_t smem, int sm_count, cudaStream_t s)
{
    auto k = pc_tc_kernel<FORM, BN, SWB, EW>;
    constexpr int kThreads = 64 + 32 * EW;
    ASD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent: one CTA per SM, no more CTAs than work items
    const int grid = (int)(a.total_tiles < sm_count ? a.total_tiles : sm_count);
    k<<<grid, kThreads, smem, s>>>(a);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // namespace

// Launch one precision form.  Instantiated combinations (the rest are rejected):
//   BN = 256 with 4 or 8 epilogue warps; BN = 128 with 4 warps.
template <int FORM>
int tc_launch_form(const TcLaunchArgs &a, size_t smem, int BN, int ew, int sm_count,
                   cudaStream_t s)
{
    constexpr int SWB = FORM == ASD_SPLIT_BF16 ? 64 : 128;
    if (BN == 256 && ew == 4) return launch_one<FORM, 256, SWB, 4>(a, smem, sm_count, s);
    if (BN == 256 && ew == 8) return launch_one<FORM, 256, SWB, 8>(a, smem, sm_count, s);
    if (BN == 128 && ew == 4) return launch_one<FORM, 128, SWB, 4>(a, smem, sm_count, s);
    set_error_text("tensor-core kernel: unsupported (tile width, epilogue warps)");
    return ASD_EUNSUPPORTED;
}

}  // namespace asd
