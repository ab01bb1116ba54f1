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
// Persistent: one CTA per SM (or one CTA pair per two SMs) takes (problem, t, row tile,
// column tile) work items in grouped raster order (raster_m row tiles per group, 16 by
// default) so concurrently running CTAs share A and B panels in L2; the TMA thread claims
// each item from a global counter (or, static, takes every n-th) and passes its K chunks,
// one sub-item each, to the other roles.  Several problems (a batched ensemble) share the
// list.  Every wait is bounded: after kTimeoutNs a role records an error in the device
// error word and stops; the CTA then drains its own in-flight copies and MMAs, frees TMEM
// and exits.
#pragma once

#include <cuda_bf16.h>

#include "asd_internal.h"
#include "geom.cuh"

namespace asd {
namespace {

// Epilogue warps EW (template parameter): 4 (one per TMEM lane quarter, all columns) or
// 8 (two per quarter, half the columns each).  Threads = TMA warp + MMA warp + EW warps.
constexpr int kMaxEpiWarps = 8;
constexpr unsigned long long kTimeoutNs = 4000000000ull;
// TMEM: 512 columns per CTA (one CTA per SM): two BN-column accumulators, then (phase
// workloads, BN <= 192) the 128-column phase product P of one pass of 64 q-vectors.
constexpr uint32_t kTmemAlloc = 512;
constexpr int kPCols = 2 * kPhaseQ;           // u (cosine weights) and v (sine weights)
constexpr uint32_t kWBytes = 128u * 128u;     // one plane of a W stage: 128 rows x 64 BF16
// Work items are handed from the TMA thread to the MMA thread and the epilogue warps
// through a ring of kWQ slots in shared memory.  With the dynamic schedule the TMA thread
// claims each item from a global counter, so the items in flight across the grid stay
// together whatever each item costs (L2 reuse of A / B panels, no drift, balanced tail);
// the static schedule takes, in round k of n CTAs, item k n + (cid + k) mod n.
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
// word then holds `code`).  (A CTA pair's waits on barriers the other CTA signals use the
// same test: the tcgen05 fences around the arrive and the wait order the tensor-memory
// accesses, and TMA and MMA completions are counted by the barrier itself; a cluster-scope
// acquire in every wait measured 30 % slower.)
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

// ---- CTA pairs (tcgen05 cta_group::2): two CTAs of a cluster share one 256-row MMA ----
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared-memory address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive on a barrier of any CTA of the cluster (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_cl(uint32_t cl_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr)
                 : "memory");
}

// TMA tile load into this CTA's shared memory whose completion is counted on a barrier
// of the pair's first CTA (cl_bar: a cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map,
                                                 uint32_t cl_bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile"
        ".mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(cl_bar), "r"(x), "r"(y)
        : "memory");
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

// TMEM allocation by one warp; with CG = 2 one warp of each CTA of the pair performs it
// together (the same columns in both CTAs).
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_slot, uint32_t ncols)
{
    if constexpr (CG == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dst_slot),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dst_slot),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

template <int CG>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    if constexpr (CG == 2)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(ncols)
                     : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(ncols)
                     : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Arrive on `bar` (a cluster address with CG = 2: this CTA's or the peer's) once the
// MMAs this thread issued so far have completed.
template <int CG = 1>
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    if constexpr (CG == 2)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
    else
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
}

// D (TMEM) = / += A B^T with A and B in shared memory.  CG = 2: a 256-row MMA over the
// pair, A rows 0-127 and B columns 0-N/2 from this CTA, the rest from the peer at the
// same addresses, D rows split between the two CTAs' TMEM.
template <bool TF32, int CG = 1>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc)
{
    if constexpr (CG == 2) {
        if (TF32)
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(a), "l"(b), "r"(idesc), "r"(acc));
        else
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
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
}

// MMA with the A operand in tensor memory (128 lanes = rows, K along the columns, two
// BF16 elements per 32-bit column, the even element in the low half) and B in shared
// memory: the phase product P = G W of the epilogue.
template <int CG = 1>
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                          uint32_t acc)
{
    if constexpr (CG == 2)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

// 32 lanes x 16 consecutive 32-bit columns (this thread's lane), and its wait, tied to the
// registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
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

// Store 16 consecutive 32-bit columns of this thread's lane; complete after tmem_wait_st.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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

// Instruction descriptor: FP32 accumulate, A/B = BF16 (1) or TF32 (2), both K-major,
// N columns, M rows (128, or 256 for a CTA pair).
__host__ __device__ constexpr uint32_t idesc(bool tf32, int N, int M = kBM)
{
    return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------------------------------
// shared-memory layout of the epilogue region
// ------------------------------------------------------------------------------------
struct EpiLayout {
    uint32_t cacc, qacc, fb, colgeo, colpk, boxred, var, total;
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
__host__ __device__ inline EpiLayout epi_layout(uint32_t vb, int nb, int nq, int BN, int ew,
                                                int det)
{
    EpiLayout L;
    uint32_t o = 0;
    // per-CTA bin sums (FP64, or 64-bit fixed point in the deterministic mode)
    L.cacc = take(o, 8u * (nb > 0 ? nb : 1));
    // phase sums per q: (cosine, sine) parts (FP64 or fixed point)
    L.qacc = take(o, 8u * 2 * (nq > 0 ? nq : 1));
    // fallback bins of pairs outside the private window (FP32, or fixed point)
    L.fb = take(o, (det ? 8u : 4u) * (nb > 0 ? nb : 1));
    L.colgeo = take(o, 16u * BN);
    L.colpk = take(o, 4u * BN);
    // per-warp row / column boxes, then the boxes of the tile's 32-column chunks (up to 8)
    L.boxred = take(o, 4u * (ew * 12 + 8 * 6));
    L.var = take(o, vb);
    L.total = (o + 1023u) & ~1023u;
    return L;
}

struct TileInfo {
    int p, t, m0, n0, row_end;
    int kg0, kg1;  // K blocks [kg0, kg1) of the S * nkb blocks of a full row
};

// Work item `tau` -> (problem, t, row tile, column tile), sub-item c -> its K chunk c.  K
// chunks split the contraction so that each partial accumulator starts from zero.
// Per-role walk over the work list.  A role visits its work items in increasing order,
// so the problem of the next item is found by stepping forward from the current one, and
// the fields that decoding needs stay in registers until the problem changes (a batched
// launch would otherwise repeat a search over the descriptors in global memory per item).
struct WorkCursor {
    int p = -1;
    int64_t begin = 0, end = 0;  // flattened work items [begin, end) belong to problem p
    int tiles_m, tiles_n, kch, G, nk, row_begin, row_end, t_begin;
    int64_t per_t;
};

// A work item is one (problem, displacement, row tile, column tile); its K chunks are
// consecutive sub-items on the same CTA (they share the tile's geometry and private
// bins).  decode(tau, c) gives chunk c of work item tau.  Row tiles are row_step rows
// (256 for a CTA pair, whose second CTA takes rows row_off = 128 on).
__device__ __forceinline__ TileInfo decode(WorkCursor &cu, const TcProblem *__restrict__ probs,
                                           int n_probs, const TcOverride &ov, int64_t tau,
                                           int c, int BN, int row_step = kBM, int row_off = 0)
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
        cu.t_begin = ov.active ? ov.t_begin : 0;
        cu.per_t = (int64_t)cu.tiles_m * cu.tiles_n;
    }
    const int64_t l = tau - cu.begin;
    TileInfo ti;
    ti.p = cu.p;
    ti.t = cu.t_begin + (int)(l / cu.per_t);
    const int kc = c;
    const int64_t rem = l % cu.per_t;
    const int64_t gspan = (int64_t)cu.G * cu.tiles_n;
    const int first_m = (int)(rem / gspan) * cu.G;
    const int gsz = min(cu.G, cu.tiles_m - first_m);
    const int64_t r2 = rem % gspan;
    ti.m0 = cu.row_begin + (first_m + (int)(r2 % gsz)) * row_step + row_off;
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
                                              const float2 *__restrict__ thr2, int *err)
{
    const float r = d2 * rsqrtf(fmaxf(d2, 1e-30f));
    const int k = min((int)(r * inv_w), nb);
    if (!ASD_INB(k >= 0, BND_THR, err)) return nb;  // dropped
    (void)err;
    const float2 t = thr2[k];
    return k + (d2 >= t.y ? 1 : 0) - (d2 < t.x ? 1 : 0);
}

// Per-tile constants of the binning epilogue, held in registers.
struct BinArgs {
    int Lx, Ly, Lz, periodic;
    float inv_w;
    int nb, blo, nwp, trash;
    int NB;                  // fallback bins of the launch
    int n_lut;
    double fscale;           // fixed-point scale (deterministic mode), else 0
    int *err;
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
                                          float *__restrict__ myb, void *__restrict__ fbv,
                                          const BinArgs ba)
{
    int slot[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float4 cg = cgeo[k];
        int b;
        if (MODE == BIN_POS) {
            b = bin_of_d2_pair(position_d2(rp, cg), ba.inv_w, ba.nb,
                               reinterpret_cast<const float2 *>(thr), ba.err);
        } else {
            const int4 cj = make_int4(__float_as_int(cg.x), __float_as_int(cg.y),
                                      __float_as_int(cg.z), 0);
            const int d2 = lattice_d2i(ri, cj, ba.Lx, ba.Ly, ba.Lz, ba.periodic);
            if (MODE == BIN_LUT)
                b = ASD_INB((unsigned)d2 < (unsigned)ba.n_lut, BND_LUT, ba.err)
                        ? reinterpret_cast<const uint16_t *>(thr)[d2]
                        : ba.nb;
            else
                b = bin_of_d2_pair((float)d2, ba.inv_w, ba.nb,
                                   reinterpret_cast<const float2 *>(thr), ba.err);
        }
        const int lb = b - ba.blo;
        slot[k] = (unsigned)lb < (unsigned)ba.nwp ? lb : (b < ba.nb ? -1 - b : ba.trash);
    }
    const bool det = ba.fscale != 0.0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        // rows past the range: their accumulator rows may come from A rows that were
        // never prepared, so the value is replaced (a product with 0 would keep a NaN)
        const float val = row_ok ? __uint_as_float(g[k]) : 0.f;
        if (slot[k] < 0) {
            const int b = -1 - slot[k];
            if (!ASD_INB(b < ba.NB, BND_FALLBACK, ba.err)) continue;
            // deterministic mode: fixed-point sums (integer adds in any order)
            if (det) add_fixed(static_cast<long long *>(fbv) + b, to_fixed(val, ba.fscale));
            else atomicAdd(static_cast<float *>(fbv) + b, val);
        } else if (ASD_INB(slot[k] <= ba.trash, BND_PRIV, ba.err)) {
            myb[slot[k] * STRIDE] += val;
        }
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
                                           uint32_t trash_off, int n_lut, int *err)
{
    (void)n_lut;
    (void)err;
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
                off[4 * k4 + u] = ASD_INB(d2 < (uint32_t)n_lut, BND_LUT, err)
                                      ? reinterpret_cast<const uint16_t *>(tab)[d2]
                                      : trash_off;
            } else {
                const int b = bin_of_d2_pair((float)d2, inv_w, nb,
                                             reinterpret_cast<const float2 *>(tab), err);
                off[4 * k4 + u] = b < nb ? (uint32_t)(b * STRIDE) : trash_off;
            }
        }
    }
}

// The same bin when every threshold is an exact FP32 square (k w)^2 = RN(RN(k w)^2), as
// for a power-of-two width (the host checks the whole table): the two thresholds around
// the first guess are computed instead of loaded.
__device__ __forceinline__ int bin_of_d2_exact(float d2, float inv_w, float w, int nb)
{
    const float r = d2 * rsqrtf(fmaxf(d2, 1e-30f));
    const int k = min((int)(r * inv_w), nb);
    const float kw = __fmul_rn((float)k, w), kw1 = __fmul_rn((float)(k + 1), w);
    const float lo = __fmul_rn(kw, kw), hi = __fmul_rn(kw1, kw1);
    return k + (d2 >= hi ? 1 : 0) - (d2 < lo ? 1 : 0);
}

// Fast form of bin_chunk's first phase for FP32 positions, when every pair of the tile
// falls inside the private window (see the epilogue): the exact bin of each pair from
// its FP32 d2 and the thresholds (loaded, or computed when EXACT), as a private-bin word
// offset; dropped pairs go to the trash row, so no pair takes a branch.
template <int STRIDE, bool EXACT>
__device__ __forceinline__ void pos_offsets(uint32_t (&off)[32], float4 rp,
                                            const float4 *__restrict__ cgeo,
                                            const float2 *__restrict__ thr2, float inv_w,
                                            float w, int nb, int blo, uint32_t trash_off,
                                            int *err)
{
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float d2 = position_d2(rp, cgeo[k]);
        const int b = EXACT ? bin_of_d2_exact(d2, inv_w, w, nb)
                            : bin_of_d2_pair(d2, inv_w, nb, thr2, err);
        off[k] = b < nb ? (uint32_t)((b - blo) * STRIDE) : trash_off;
    }
}

using LaunchArgs = TcLaunchArgs;

// Sum of 16 per-lane values over the warp's 32 lanes by recursive halving: each exchange
// sends the half of the values this lane does not keep; after four steps lanes 2m and
// 2m + 1 hold partial sums of value m, which the last exchange adds.
__device__ __forceinline__ float warp_sum16(float (&z)[16], int lane)
{
#pragma unroll
    for (int hh = 8, o = 16; hh >= 1; hh >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < hh; ++k) {
            const float send = up ? z[k] : z[k + hh];
            const float keep = up ? z[k + hh] : z[k];
            z[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return z[0] + __shfl_xor_sync(0xffffffffu, z[0], 1);
}

// K block of a work item before which sub-pass g (of G) of the previous item's phase
// product is loaded and issued.  A sub-pass is one W stage (64 columns of one pass, the
// pass's kWStages sub-passes in order).  The epilogue needs the first part of the item to
// bin and convert the previous tile (the first sub-pass waits for that), the rest of it
// to read the product out before the accumulator is needed again.  Sub-passes go in from
// kSlotLo / kSlotDen of the item, evenly spaced up to kSlotHi / kSlotDen.  Measured on the
// 32^3 glass (bins + 64 q, one pass of 3 sub-passes): all at 2/3 of the item 95.0 ms;
// spread over [1/2, 5/6] 102.0, [1/3, 2/3] 101.4, [1/2, 1] 107.6, [1/6, 5/6] 112.1: the
// binning of the previous tile sets the earliest slot, the read-out the latest.
constexpr int kSlotLo = 2, kSlotHi = 2, kSlotDen = 3;
__device__ __forceinline__ int phase_slot(int g, int nk, int G)
{
    return (nk * kSlotLo) / kSlotDen + (g * nk * (kSlotHi - kSlotLo)) / (kSlotDen * G);
}

// ------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------
// CG = 2: CTA pairs (clusters of two).  The pair computes a 256-row tile with one MMA
// thread (in the first CTA) issuing tcgen05 cta_group::2 MMAs: each CTA loads its own
// 128 A rows and half of the B columns, so per SM the operand traffic of a 256 x BN
// tile is that of a 128 x (128 + BN/2) one; each CTA's TMEM holds its 128 rows and its
// epilogue bins them.  Both CTAs walk the same fixed order of work items; the second
// CTA's epilogue warps release accumulators and phase products on the first CTA's
// barriers.
template <int FORM, int BN, int SWB, int EW, int CG>
__global__ void __launch_bounds__(64 + 32 * EW, 1) pc_tc_kernel(const __grid_constant__ LaunchArgs args)
{
    constexpr int kEpiWarps = EW;
    constexpr int kEpiThreads = 32 * EW;
    constexpr int kBinStride = bin_stride(EW);
    constexpr int kHalves = EW / 4;
    constexpr int kChunks = BN / 32;                                 // 32-column chunks
    constexpr int kColM = (BN + kEpiThreads - 1) / kEpiThreads;      // columns per thread
    static_assert(kChunks <= 8, "chunk boxes of a tile (and one lane per chunk)");
    constexpr bool kTF32 = FORM == ASD_TF32;
    constexpr int kPlanes = FORM == ASD_SPLIT_BF16 ? 2 : 1;
    constexpr uint32_t kABytes = kBM * SWB;
    constexpr uint32_t kBBytes = (BN / CG) * SWB;   // this CTA's B columns
    constexpr uint32_t kStageBytes = kPlanes * (kABytes + kBBytes);
    constexpr int kKSteps = SWB / 32;          // one MMA k-step covers 32 bytes of K
    constexpr int kBK = SWB / (kTF32 ? 4 : 2); // K elements per stage
    constexpr uint32_t kIdesc = idesc(kTF32, BN, kBM * CG);
    // Phase weights on the tensor core (problems with n_q > 0; the plan picks BN <= 192):
    // after the epilogue has binned a K chunk of a tile it stores the chunk's G, split
    // into BF16 hi + lo, back over the accumulator's own columns (chunk of 32 columns ->
    // 16 columns of hi, then 16 of lo), and one pass of kPhaseQ q-vectors is the
    // 128 x 128 x BN product P = G W with W[c][o] = cos / sin(q_o . r_c) of the tile's
    // columns, streamed through the operand ring (64 columns c per stage).  Split-BF16 and
    // TF32 issue hi*hi + hi*lo + lo*hi (the FP32-accurate sum); BF16 issues hi*hi.
    constexpr bool kPhaseOK = 2 * BN + kPCols <= (int)kTmemAlloc;
    constexpr int kWPlanes = FORM == ASD_BF16 ? 1 : 2;
    constexpr int kWStages = BN / 64;          // W stages per pass (64 columns c each)
    constexpr uint32_t kWB = kWBytes / CG;     // one W plane of this CTA (its output half)
    constexpr uint32_t kIdescP = idesc(false, kPCols, kBM * CG);
    static_assert(!kPhaseOK || (kStageBytes >= kWPlanes * kWB && BN % 64 == 0),
                  "a W stage fits a ring stage");
    static_assert(CG == 1 || CG == 2, "CTA groups of one or two");

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~(uintptr_t)1023);
    const int stages = args.stages;
    uint8_t *tiles = smem;
    uint8_t *epi = tiles + (size_t)stages * kStageBytes;
    const EpiLayout EL = epi_layout(args.VB, args.NB, args.NQ, BN, EW, args.det);
    uint64_t *bars = reinterpret_cast<uint64_t *>(epi + EL.total);
    // bars: full[stages], empty[stages], tfull[2], tempty[2], drain, wqfull[kWQ],
    // wqempty[kWQ], conv, pfull, pempty, tmm[2]; then the work ring wq[kWQ] and the TMEM
    // address slot
    const uint32_t wqfull0 = saddr(bars + 2 * stages + 5);
    const uint32_t wqempty0 = saddr(bars + 2 * stages + 5 + kWQ);
    // conv: the epilogue has stored a chunk's G as BF16 hi / lo (one arrival per warp);
    // pfull: the phase product to be read out is complete; pempty: the epilogue has read
    // it; tmm[a]: the phase product of the chunk in accumulator a is complete, so the
    // buffer is free (for phase work the MMA thread releases the accumulator, not the
    // epilogue)
    const uint32_t conv = saddr(bars + 2 * stages + 5 + 2 * kWQ);
    const uint32_t pfull = conv + 8, pempty = conv + 16, tmm0 = conv + 24;
    volatile int64_t *wq = reinterpret_cast<volatile int64_t *>(bars + 2 * stages + 10 + 2 * kWQ);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 10 + 3 * kWQ);
    const uint32_t full0 = saddr(bars), empty0 = saddr(bars + stages);
    const uint32_t tfull0 = saddr(bars + 2 * stages), tempty0 = saddr(bars + 2 * stages + 2);
    const uint32_t drain = saddr(bars + 2 * stages + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // CTA pair: rank in the pair; the first CTA (rank 0) issues the MMAs.  lead(a) is the
    // cluster address of barrier a in the first CTA, peer(a) in the other one.
    const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
    const bool leader = rank == 0;
    auto lead = [&](uint32_t a) { return CG == 2 ? mapa(a, 0) : a; };
    auto peer = [&](uint32_t a) { return CG == 2 ? mapa(a, 1) : a; };
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            // a stage is free again once the MMAs that read it have completed
            mbar_init(empty0 + 8 * s, 1);
        }
        // (a pair's epilogue barriers count the warps of both CTAs)
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, kEpiWarps * CG);
        }
        mbar_init(drain, 1);
        for (int k = 0; k < kWQ; ++k) {
            mbar_init(wqfull0 + 8 * k, 1);
            // released by the MMA thread (the first CTA of a pair only) and one lane of
            // every epilogue warp
            mbar_init(wqempty0 + 8 * k, (leader ? 1 : 0) + kEpiWarps);
        }
        mbar_init(conv, kEpiWarps * CG);
        mbar_init(pfull, 1);
        mbar_init(pempty, kEpiWarps * CG);
        mbar_init(tmm0, 1);
        mbar_init(tmm0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc<CG>(saddr(tmem_slot), kTmemAlloc);
    tc_before();
    __syncthreads();
    // a pair's barriers are initialised in both CTAs before either signals the other
    if constexpr (CG == 2) cluster_sync();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    const TcProblem *__restrict__ probs = args.probs;
    // work units: CTAs, or pairs
    const int64_t cid = blockIdx.x / CG, n_ctas = gridDim.x / CG;
    const int row_step = kBM * CG, row_off = kBM * (int)rank;

    if (warp == 0) {
        // ======================= TMA producer =======================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            WorkCursor cu;
            // the previous work item, while its phase sub-passes are still to be loaded:
            // they go in among this item's K blocks (sub-pass g before block
            // phase_slot(g)), so the phase product of item v - 1 runs while item v's MMAs
            // run
            int pend_p = -1, pend_n0 = 0, pend_G = 0;
            int64_t n_claimed = 0;  // work items claimed (static schedule)
            auto next_stage = [&]() {
                if (++stage == stages) {
                    stage = 0;
                    phase ^= 1;
                }
            };
            // W stage j of pass pp (sub-pass g = pp kWStages + j)
            // (a pair: each CTA loads its half of the outputs; the first CTA's full barrier
            // counts the bytes of both)
            auto load_sub = [&](int g) {
                const TcProblem &Q = probs[pend_p];
                const int pp = g / kWStages, j = g % kWStages;
                if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, args.err, DEV_TIMEOUT_TMA))
                    return false;
                const uint32_t fb = full0 + 8 * stage;
                if (leader) mbar_expect_tx(fb, CG * kWPlanes * kWB);
                uint8_t *st = tiles + (size_t)stage * kStageBytes;
#pragma unroll
                for (int pl = 0; pl < kWPlanes; ++pl) {
                    const int y = pp * kPCols + (int)rank * (kPCols / CG);
                    if constexpr (CG == 2)
                        tma_load_2d_pair(saddr(st + pl * kWB), &Q.mapW[pl], lead(fb),
                                         pend_n0 + 64 * j, y);
                    else
                        tma_load_2d(saddr(st + pl * kWB), &Q.mapW[pl], fb, pend_n0 + 64 * j, y);
                }
                next_stage();
                return true;
            };
            // Sub-items (a work item's K chunks) in this CTA's work ring.  A lone CTA claims
            // work items from the counter (dynamic schedule) or in a fixed order; both CTAs
            // of a pair walk the same fixed order (measured against handing each item from
            // the first CTA to the second: 542 against 506 TFLOP/s on the 26^3 lattice).
            // The fixed order: in round k of n CTAs (pairs), CTA c takes item
            // k n + (c + k) mod n.  Without the rotation a raster group of a multiple of n
            // items would put every CTA on the same columns in every group, so the costly
            // column tiles would always land on the same CTAs.
            int64_t tau = 0;
            int kci = 0, kch = 0;
            for (int64_t v = 0; ok; ++v) {
                const int qs = (int)(v % kWQ);
                // the next chunk of the current item, or the first of a new one
                if (++kci >= kch) {
                    tau = args.counter && CG == 1
                              ? (int64_t)atomicAdd(args.counter, 1ull)
                              : n_claimed * n_ctas + (cid + n_claimed) % n_ctas;
                    ++n_claimed;
                    if (tau >= args.total_tiles) tau = -1;
                    kci = 0;
                    kch = tau < 0 ? 1
                                  : probs[decode(cu, probs, args.n_probs, args.ov, tau, 0, BN,
                                                 row_step, row_off).p].k_chunks;
                }
                // publish the sub-item (tau 256 + chunk; -1: none left) once its ring slot
                // is free
                if (!mbar_wait(wqempty0 + 8 * qs, (uint32_t)((v / kWQ) & 1) ^ 1u, args.err,
                               DEV_TIMEOUT_TMA)) {
                    ok = false;
                    break;
                }
                wq[qs] = tau < 0 ? -1 : tau * 256 + kci;
                mbar_arrive(wqfull0 + 8 * qs);  // release: the slot is visible to the waiters
                if (tau < 0) break;
                const TileInfo ti =
                    decode(cu, probs, args.n_probs, args.ov, tau, kci, BN, row_step, row_off);
                const TcProblem &P = probs[ti.p];
                const int nk = ti.kg1 - ti.kg0;
                int g = 0;
                for (int kg = ti.kg0; kg < ti.kg1 && ok; ++kg) {
                    if constexpr (kPhaseOK) {
                        while (pend_p >= 0 && g < pend_G &&
                               kg - ti.kg0 == phase_slot(g, nk, pend_G)) {
                            if (!load_sub(g++)) {
                                ok = false;
                                break;
                            }
                        }
                        if (!ok) break;
                    }
                    const int s = kg / P.nkb, kb = kg % P.nkb;
                    const int xw = s * P.F3 + 3 * ti.t;
                    const int c = xw % P.n_copies;

                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, args.err, DEV_TIMEOUT_TMA)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * stage;
                    if (leader) mbar_expect_tx(fb, CG * kStageBytes);
                    uint8_t *st = tiles + (size_t)stage * kStageBytes;
                    // this CTA's B columns (a pair splits the tile's columns)
                    const int nb0 = ti.n0 + (int)rank * (BN / CG);
#pragma unroll
                    for (int pl = 0; pl < kPlanes; ++pl) {
                        if constexpr (CG == 2) {
                            tma_load_2d_pair(saddr(st + pl * kABytes), &P.mapA[pl][c],
                                             lead(fb), xw - c + kb * kBK, ti.m0);
                            tma_load_2d_pair(saddr(st + kPlanes * kABytes + pl * kBBytes),
                                             &P.mapB[pl], lead(fb), s * P.Kseg + kb * kBK,
                                             nb0);
                        } else {
                            tma_load_2d(saddr(st + pl * kABytes), &P.mapA[pl][c], fb,
                                        xw - c + kb * kBK, ti.m0);
                            tma_load_2d(saddr(st + kPlanes * kABytes + pl * kBBytes),
                                        &P.mapB[pl], fb, s * P.Kseg + kb * kBK, nb0);
                        }
                    }
                    next_stage();
                }
                pend_p = -1;
                if (kPhaseOK && P.epi.n_q > 0) {
                    pend_p = ti.p;
                    pend_n0 = ti.n0;
                    pend_G = P.epi.npass * kWStages;
                }
            }
            // the last item's phase sub-passes
            if (kPhaseOK && ok && pend_p >= 0)
                for (int g = 0; g < pend_G && ok; ++g) ok = load_sub(g);
            // drain: wait until the last fill of every stage has landed
            for (int k = 0; k < stages; ++k) {
                if (--stage < 0) {
                    stage = stages - 1;
                    phase ^= 1;
                }
                // the most recent fill of `stage` used parity `phase`; if that stage was never
                // filled, its barrier is still in phase 0 and parity 1 reads as complete (a
                // pair's fills all complete on the first CTA's barriers: it waits for both)
                if (leader) mbar_wait(full0 + 8 * stage, phase, args.err, DEV_TIMEOUT_TMA);
            }
        }
    } else if (warp == 1) {
        // ======================= MMA issuer =======================
        // (a pair's MMAs are issued by the first CTA; its commits release the stages and
        // hand the accumulators to the epilogues of both CTAs)
        auto commit_both = [&](uint32_t a) {
            if constexpr (CG == 2) {
                tc_commit<2>(a);
                tc_commit<2>(peer(a));
            } else {
                tc_commit(a);
            }
        };
        if (lane == 0 && leader) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t v = 0;
            bool ok = true;
            WorkCursor cu;
            // previous sub-item with phase sub-passes still to issue: its accumulator
            // buffer and sub-pass count; whether its product adds to P (a later K chunk of
            // a tile with one pass: P sums the chunks and is read out once) and whether it
            // completes P for the read-out
            int pend_acc = -1, pend_G = 0;
            bool pend_add = false, pend_done = false;
            // converted chunks waited for; passes that started P afresh (one read-out each)
            uint32_t n_conv = 0, n_own = 0;
            // how each accumulator was last released (0: not used yet, 1: by the epilogue
            // on tempty, 2: by this thread's commit on tmm after the chunk's phase product)
            // and the waits taken on each barrier
            int rel[2] = {0, 0};
            uint32_t n_te[2] = {0, 0}, n_tm[2] = {0, 0};
            const uint32_t ptm = tmem + 2 * BN;  // phase product P
            // sub-pass g of the previous item's phase product: pass pp = g / kWStages adds
            // G[:, c] W[c, :] for the 64 columns c of W stage j = g % kWStages to P, A = the
            // BF16 hi / lo copy of G in its accumulator columns
            auto issue_sub = [&](int g) {
                const int pp = g / kWStages, j = g % kWStages;
                const uint32_t g0 = tmem + (uint32_t)pend_acc * BN;
                if (!mbar_wait(full0 + 8 * stage, phase, args.err, DEV_TIMEOUT_MMA))
                    return false;
                if (j == 0) {
                    // G stored as BF16 by the epilogue (once per chunk); a pass that starts
                    // P afresh waits until the previous P has been read out
                    if (pp == 0 &&
                        !mbar_wait(conv, n_conv++ & 1, args.err, DEV_TIMEOUT_MMA))
                        return false;
                    if (!pend_add) {
                        if (!mbar_wait(pempty, (n_own & 1) ^ 1, args.err, DEV_TIMEOUT_MMA))
                            return false;
                        ++n_own;
                    }
                }
                tc_after();
                uint8_t *st = tiles + (size_t)stage * kStageBytes;
                const uint64_t w0 = sdesc(saddr(st), 128);
                const uint64_t w1 = sdesc(saddr(st + kWB), 128);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    // columns c = 64 j + 16 ks: chunk c / 32 holds hi in its first 16 TMEM
                    // columns and lo in the next 16
                    const int c = 64 * j + 16 * ks;
                    const uint32_t ahi = g0 + 32 * (c >> 5) + 8 * ((c >> 4) & 1);
                    const uint64_t off = (uint64_t)(ks * 32) >> 4;
                    const uint32_t accum = pend_add || (j | ks) != 0;
                    tc_mma_ts<CG>(ptm, ahi, w0 + off, kIdescP, accum);           // hi*hi
                    if (kWPlanes == 2) {
                        tc_mma_ts<CG>(ptm, ahi, w1 + off, kIdescP, 1u);          // hi*lo
                        tc_mma_ts<CG>(ptm, ahi + 16, w0 + off, kIdescP, 1u);     // lo*hi
                    }
                }
                commit_both(empty0 + 8 * stage);
                if (++stage == stages) {
                    stage = 0;
                    phase ^= 1;
                }
                if (j == kWStages - 1 && pend_done) commit_both(pfull);
                // the chunk's accumulator is free once its phase product has completed
                if (g == pend_G - 1) tc_commit<CG>(tmm0 + 8 * pend_acc);
                return true;
            };
            for (;; ++v) {
                const int qs = (int)(v % kWQ);
                if (!mbar_wait(wqfull0 + 8 * qs, (v / kWQ) & 1, args.err, DEV_TIMEOUT_MMA)) {
                    ok = false;
                    break;
                }
                const int64_t tau = wq[qs];
                mbar_arrive(wqempty0 + 8 * qs);
                if (tau < 0) break;
                const int kci = (int)(tau & 255);
                const TileInfo ti = decode(cu, probs, args.n_probs, args.ov, tau >> 8, kci, BN,
                                           row_step, row_off);
                const TcProblem &P = probs[ti.p];
                const bool phs = kPhaseOK && P.epi.n_q > 0;
                const uint32_t acc = v & 1;
                // wait until the accumulator's previous chunk has released it
                if (rel[acc] == 1 && !mbar_wait(tempty0 + 8 * acc, n_te[acc]++ & 1, args.err,
                                                DEV_TIMEOUT_MMA)) {
                    ok = false;
                    break;
                }
                if (rel[acc] == 2 && !mbar_wait(tmm0 + 8 * acc, n_tm[acc]++ & 1, args.err,
                                                DEV_TIMEOUT_MMA)) {
                    ok = false;
                    break;
                }
                rel[acc] = phs ? 2 : 1;
                tc_after();
                const uint32_t d = tmem + acc * BN;
                const int nk = ti.kg1 - ti.kg0;
                int g = 0;
                for (int kg = ti.kg0; kg < ti.kg1; ++kg) {
                    const int kb = kg - ti.kg0;  // 0 for the first block of this chunk
                    if constexpr (kPhaseOK) {
                        while (pend_acc >= 0 && g < pend_G && kb == phase_slot(g, nk, pend_G)) {
                            if (!issue_sub(g++)) {
                                ok = false;
                                break;
                            }
                        }
                        if (!ok) break;
                    }
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
                            tc_mma<kTF32, CG>(d, a0 + off, b0 + off, kIdesc, first);
                        } else {
                            const uint64_t a1 = sdesc(saddr(st + kABytes), SWB);
                            const uint64_t b1 = sdesc(saddr(st + 2 * kABytes + kBBytes), SWB);
                            tc_mma<false, CG>(d, a0 + off, b0 + off, kIdesc, first);  // hi*hi
                            tc_mma<false, CG>(d, a0 + off, b1 + off, kIdesc, 1u);     // hi*lo
                            tc_mma<false, CG>(d, a1 + off, b0 + off, kIdesc, 1u);     // lo*hi
                        }
                    }
                    commit_both(empty0 + 8 * stage);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                commit_both(tfull0 + 8 * acc);
                pend_acc = -1;
                if (phs) {
                    // one pass: P sums the tile's chunks and is read out after the last
                    const bool across = P.epi.npass == 1;
                    pend_acc = (int)acc;
                    pend_G = P.epi.npass * kWStages;
                    pend_add = across && kci > 0;
                    pend_done = !across || kci == P.k_chunks - 1;
                }
            }
            // the last item's phase sub-passes
            if (kPhaseOK && ok && pend_acc >= 0)
                for (int g = 0; g < pend_G && ok; ++g) ok = issue_sub(g);
            // drain every MMA this thread issued before TMEM is released
            tc_commit<CG>(drain);
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
        // the same arrays as 64-bit fixed point (problems in the deterministic mode)
        long long *fbi = reinterpret_cast<long long *>(epi + EL.fb);
        long long *cacci = reinterpret_cast<long long *>(epi + EL.cacc);
        long long *qacci = reinterpret_cast<long long *>(epi + EL.qacc);
        float4 *colgeo = reinterpret_cast<float4 *>(epi + EL.colgeo);
        uint32_t *colpk = reinterpret_cast<uint32_t *>(epi + EL.colpk);
        float *boxred = reinterpret_cast<float *>(epi + EL.boxred);
        float *chbox = boxred + kEpiWarps * 12;
        float *thr_s = bins;
        for (int k = et; k < args.NB; k += kEpiThreads) {
            if (args.det) fbi[k] = 0;
            else fb[k] = 0.f;
            cacc[k] = 0.0;  // (all-zero bits: also fixed-point zero)
        }
        for (int k = et; k < 2 * args.NQ; k += kEpiThreads) qacc[k] = 0.0;

        int cur_p = -1, cur_t = -1, tab_p = -1;
        WorkCursor cu;
        // fast lattice binning also needs the private-bin offsets of this launch (the
        // largest window of a batch, plus its trash row) to fit the 16-bit table entries
        auto fast_ok = [&](const EpiParams &E) {
            return E.fast && (E.NW + 1) * kBinStride <= 65536;
        };
        // phase passes read out so far (parity of pfull)
        uint32_t n_pass = 0;
        // Store a 32-column chunk of this thread's accumulator row back as BF16 hi / lo
        // (16 columns each, two values per column, the even column in the low half):
        // the A operand of the phase product.  Rows past the range store zeros.
        auto to_bf16 = [&](const uint32_t (&g)[32], uint32_t tcol, bool keep) {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float a = keep ? __uint_as_float(g[2 * k]) : 0.f;
                const float b = keep ? __uint_as_float(g[2 * k + 1]) : 0.f;
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                const float2 hf = __bfloat1622float2(h);
                const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
                hi[k] = *reinterpret_cast<const uint32_t *>(&h);
                lo[k] = *reinterpret_cast<const uint32_t *>(&l);
            }
            tmem_st16(tcol, hi);
            tmem_st16(tcol + 16, lo);
        };
        uint32_t v = 0;
        bool ok = true;
        // geometry of the current tile, set by its first K chunk: this thread's row site,
        // the bin window start and, for positions, whether the tile's bins fit the window
        int4 ri = make_int4(0, 0, 0, 0);
        float4 rp = make_float4(0.f, 0.f, 0.f, 0.f);
        int blo = 0, bhi_tile = 0;
        bool pos_fit = false;
        // positions: a tile whose columns span two far-apart groups of sites may take two
        // windows, private rows [0, n1) for bins blo + k (column chunks before `split`) and
        // rows [n1, nwp) for bins blo2 + k - n1 (the chunks from `split` on)
        int blo2 = 0, n1 = 0, split = 0, nwp = 0;
        // per-CTA FP64 sums of the current (problem, t), added to the outputs when it changes
        // (deterministic mode: fixed-point sums into the problem's fixed-point arrays)
        auto flush_acc = [&](int p, int t) {
            const EpiParams &E = probs[p].epi;
            double *Cs = args.ov.active ? args.ov.C_sum : E.C_sum;
            double *Qs = args.ov.active ? args.ov.Sq_sum : E.Sq_sum;
            const bool det = E.fix_scale != nullptr;
            const bool t_ok = ASD_INB((unsigned)t < (unsigned)probs[p].n_t, BND_WORK, args.err);
            for (int b = et; b < E.n_bins; b += kEpiThreads) {
                const int64_t o = (int64_t)t * E.n_bins + b;
                if (det) {
                    if (cacci[b] != 0 && t_ok) add_fixed(&E.C_fix[o], cacci[b]);
                } else if (cacc[b] != 0.0 && t_ok) {
                    atomicAdd(&Cs[o], cacc[b]);
                }
                cacc[b] = 0.0;
            }
            for (int q = et; q < E.n_q; q += kEpiThreads)
                for (int part = 0; part < E.q_parts; ++part) {
                    const int64_t o = ((int64_t)t * E.n_q + q) * E.q_parts + part;
                    if (det) {
                        if (qacci[2 * q + part] != 0 && t_ok)
                            add_fixed(&E.Sq_fix[o], qacci[2 * q + part]);
                    } else if (qacc[2 * q + part] != 0.0 && t_ok) {
                        atomicAdd(&Qs[o], qacc[2 * q + part]);
                    }
                    qacc[2 * q + part] = 0.0;
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
            const int kci = (int)(tau & 255);
            const TileInfo ti = decode(cu, probs, args.n_probs, args.ov, tau >> 8, kci, BN,
                                       row_step, row_off);
            const TcProblem &P = probs[ti.p];
            const EpiParams &E = P.epi;
            // the first K chunk of a tile sets up its geometry and bin window; the chunks
            // add into the same private bins, which the last one reduces
            const bool first = kci == 0, last = kci == P.k_chunks - 1;
            const int i = ti.m0 + r;
            const bool row_ok = i < ti.row_end;
            // rows past the range (ragged tiles) read the
            // geometry of a valid site and contribute zeros
            const int ic = row_ok ? i : P.N - 1;
            const bool lattice = E.geom == ASD_GEOM_LATTICE;
            // (a checked build also tests that the problem's bins and table fit the
            // launch's per-problem region; if not, the problem is not binned)
            const bool bins_on =
                E.n_bins > 0 &&
                ASD_INB(var_bytes(E.NW, E.n_bins, E.n_lut, EW) <= args.VB, BND_REGION, args.err);
            // fixed-point scale of a problem in the deterministic mode (0: FP sums)
            const double fscale = E.fix_scale ? *E.fix_scale : 0.0;
            if (first) {
                // bin thresholds of this problem, then the column geometry of this tile
                if (bins_on && ti.p != tab_p) {
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
                // column geometry of the tile (one load per column, which also feeds the
                // column bounding box when the bins do not all fit the window)
                float cl[3] = {3e38f, 3e38f, 3e38f}, ch[3] = {-3e38f, -3e38f, -3e38f};
                // (and the box of each 32-column chunk this warp loads: chunk ew + m EW)
                float cm[kColM][6];
#pragma unroll
                for (int m = 0; m < kColM; ++m)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        cm[m][a] = 3e38f;
                        cm[m][3 + a] = -3e38f;
                    }
#pragma unroll
                for (int m = 0; m < kColM; ++m) {
                    const int c = et + m * kEpiThreads;
                    if (c >= BN) break;
                    const int j = min(ti.n0 + c, P.N - 1);
                    float4 pj;
                    if (lattice) {
                        const int4 g = E.coords[j];
                        colgeo[c] = make_float4(__int_as_float(g.x), __int_as_float(g.y),
                                                __int_as_float(g.z), 0.f);
                        colpk[c] = (uint32_t)g.x | ((uint32_t)g.y << 8) | ((uint32_t)g.z << 16);
                        pj = make_float4((float)g.x, (float)g.y, (float)g.z, 0.f);
                    } else {
                        pj = E.pos[j];
                        colgeo[c] = pj;
                    }
                    cl[0] = fminf(cl[0], pj.x); ch[0] = fmaxf(ch[0], pj.x);
                    cl[1] = fminf(cl[1], pj.y); ch[1] = fmaxf(ch[1], pj.y);
                    cl[2] = fminf(cl[2], pj.z); ch[2] = fmaxf(ch[2], pj.z);
                    cm[m][0] = pj.x; cm[m][1] = pj.y; cm[m][2] = pj.z;
                    cm[m][3] = pj.x; cm[m][4] = pj.y; cm[m][5] = pj.z;
                }
                ri = E.coords[ic];
                rp = lattice ? make_float4((float)ri.x, (float)ri.y, (float)ri.z, 0.f) : E.pos[ic];
                // bounding boxes for the bin window (only when the bins do not all fit)
                if (E.use_window) {
                    float v6[12];
                    v6[0] = v6[3] = rp.x;
                    v6[1] = v6[4] = rp.y;
                    v6[2] = v6[5] = rp.z;
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
                    if (!lattice) {
#pragma unroll
                        for (int m = 0; m < kColM; ++m) {
                            const int chk = ew + m * kEpiWarps;  // warp-uniform
                            if (chk >= kChunks) break;
                            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                                for (int k = 0; k < 6; ++k) {
                                    const float w = __shfl_xor_sync(0xffffffffu, cm[m][k], o);
                                    cm[m][k] = k < 3 ? fminf(cm[m][k], w) : fmaxf(cm[m][k], w);
                                }
                            if (lane == 0)
#pragma unroll
                                for (int k = 0; k < 6; ++k) chbox[chk * 6 + k] = cm[m][k];
                        }
                    }
                }
                epi_sync(kEpiThreads);  // colgeo / boxred ready; previous tile fully flushed
                if (ti.p != cur_p || ti.t != cur_t) {
                    if (cur_p >= 0) flush_acc(cur_p, cur_t);
                    cur_p = ti.p;
                    cur_t = ti.t;
                }
                blo = 0;
                n1 = E.NW;
                split = kChunks;
                nwp = E.n_bins;
                // positions: whether every kept bin of the tile lies inside the private window
                // [blo, blo + NW), from the largest distance between the two bounding boxes
                pos_fit = !E.use_window;
                bhi_tile = E.n_bins - 1;
                if (E.use_window) {
                    float d2min = 0.f, d2max = 0.f;
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
                        const float far = fmaxf(ch - rl, rh - cl);
                        d2max += far * far;
                    }
                    // (the thresholds from shared memory unless it holds the lattice table)
                    const float2 *thr2 = reinterpret_cast<const float2 *>(thr_s);
                    const bool tab = E.n_lut > 0;
                    blo = max(0, (tab ? bin_of_d2(d2min * 0.999f, E.inv_w, E.n_bins, E.thr)
                                      : bin_of_d2_pair(d2min * 0.999f, E.inv_w, E.n_bins, thr2,
                                                       args.err)) - 1);
                    if (!lattice) {
                        bhi_tile = min(E.n_bins - 1,
                                       bin_of_d2_pair(d2max * 1.001f + 1e-30f, E.inv_w, E.n_bins,
                                                      thr2, args.err) + 1);
                        pos_fit = bhi_tile - blo < E.NW;
                        nwp = bhi_tile - blo + 1;
                        if (!pos_fit) {
                            // bins of each 32-column chunk (lane c computes chunk c), then the
                            // first split of the chunks into two windows that together fit
                            int lo_c = 1 << 30, hi_c = -1;
                            if (lane < kChunks) {
                                float dmin = 0.f, dmax = 0.f;
                                for (int a = 0; a < 3; ++a) {
                                    float rl = 3e38f, rh = -3e38f;
                                    for (int w = 0; w < kEpiWarps; ++w) {
                                        rl = fminf(rl, boxred[w * 12 + a]);
                                        rh = fmaxf(rh, boxred[w * 12 + 3 + a]);
                                    }
                                    const float cl = chbox[lane * 6 + a], ch = chbox[lane * 6 + 3 + a];
                                    const float gap = fmaxf(0.f, fmaxf(cl - rh, rl - ch));
                                    const float far = fmaxf(ch - rl, rh - cl);
                                    dmin += gap * gap;
                                    dmax += far * far;
                                }
                                lo_c = max(0, bin_of_d2_pair(dmin * 0.999f, E.inv_w, E.n_bins, thr2,
                                                             args.err) - 1);
                                hi_c = min(E.n_bins - 1,
                                           bin_of_d2_pair(dmax * 1.001f + 1e-30f, E.inv_w,
                                                          E.n_bins, thr2, args.err) + 1);
                            }
                            int lo[kChunks], hi[kChunks];
#pragma unroll
                            for (int c = 0; c < kChunks; ++c) {
                                lo[c] = __shfl_sync(0xffffffffu, lo_c, c);
                                hi[c] = __shfl_sync(0xffffffffu, hi_c, c);
                            }
                            // one window over the chunks' bins (narrower than the tile's
                            // box); only when that does not fit, two windows, which are then
                            // disjoint (two overlapping ones would span no more than their
                            // sum), so no bin has two private rows
                            int l0 = 1 << 30, h0 = -1;
#pragma unroll
                            for (int c = 0; c < kChunks; ++c) {
                                l0 = min(l0, lo[c]);
                                h0 = max(h0, hi[c]);
                            }
                            int best = E.NW + 1;
                            if (h0 - l0 + 1 <= E.NW) {
                                best = h0 - l0 + 1;
                                blo = l0;
                                n1 = E.NW;
                                split = kChunks;
                            }
#pragma unroll
                            for (int sp = 1; sp < kChunks && best > E.NW; ++sp) {
                                int l1 = 1 << 30, h1 = -1, l2 = 1 << 30, h2 = -1;
#pragma unroll
                                for (int c = 0; c < kChunks; ++c) {
                                    if (c < sp) { l1 = min(l1, lo[c]); h1 = max(h1, hi[c]); }
                                    else { l2 = min(l2, lo[c]); h2 = max(h2, hi[c]); }
                                }
                                const int need = (h1 - l1 + 1) + (h2 - l2 + 1);
                                if (need < best) {
                                    best = need;
                                    blo = l1;
                                    n1 = h1 - l1 + 1;
                                    blo2 = l2;
                                    split = sp;
                                }
                            }
                            if (best <= E.NW) {
                                pos_fit = true;
                                nwp = best;
                            } else {
                                blo = max(0, (tab ? bin_of_d2(d2min * 0.999f, E.inv_w, E.n_bins, E.thr)
                                                  : bin_of_d2_pair(d2min * 0.999f, E.inv_w, E.n_bins,
                                                                   thr2, args.err)) - 1);
                                n1 = E.NW;
                                split = kChunks;
                            }
                        } else {
                            n1 = E.NW;
                            split = kChunks;
                        }
                    }
                }
            }  // first chunk

            // phase weights of this item go through the tensor core (see kPhaseOK)
            const bool ph = kPhaseOK && E.n_q > 0;
            const uint32_t acc = v & 1, use = v >> 1;
            const bool got = mbar_wait(tfull0 + 8 * acc, use & 1, args.err, DEV_TIMEOUT_EPI);
            ok = epi_sync_and(got, kEpiThreads);
            if (!ok) break;
            tc_after();
            const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + acc * BN;

            if (bins_on) {
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
                ba.NB = args.NB;
                ba.n_lut = E.n_lut;
                ba.fscale = fscale;
                ba.err = args.err;
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
                                                         E.n_bins, trash_off, E.n_lut, args.err);
                        else
                            pk_offsets<false, kBinStride>(off, rpk, E.Lpk, cp, thr_s, E.inv_w,
                                                          E.n_bins, trash_off, E.n_lut, args.err);
                        tmem_wait32(g);
                        if (row_ok) {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (ASD_INB(off[k] <= trash_off, BND_PRIV, args.err))
                                    mb[off[k]] += __uint_as_float(g[k]);
                        }
                        if (ph) to_bf16(g, tbase + ch * 32, row_ok);
                    }
                } else if (mode == BIN_POS && pos_fit) {
                    // rows past the range skip the pairs (the TMEM loads stay warp-wide)
                    float *mb = bins + r + kBM * half;
                    const uint32_t trash_off = (uint32_t)E.NW * kBinStride;
                    const float2 *thr2 = reinterpret_cast<const float2 *>(thr_s);
                    for (int ch = ch0; ch < ch1; ++ch) {
                        // (private row of bin b: b - blo, or b - blo2 + n1 in a second window)
                        const int b0 = !E.use_window ? 0 : ch < split ? blo : blo2 - n1;
                        uint32_t g[32], off[32];
                        tmem_ld32_issue(tbase + ch * 32, g);
                        if (E.thr_exact)
                            pos_offsets<kBinStride, true>(off, rp, colgeo + ch * 32, thr2,
                                                          E.inv_w, E.w, E.n_bins, b0, trash_off,
                                                          args.err);
                        else
                            pos_offsets<kBinStride, false>(off, rp, colgeo + ch * 32, thr2,
                                                           E.inv_w, E.w, E.n_bins, b0,
                                                           trash_off, args.err);
                        tmem_wait32(g);
                        if (row_ok) {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (ASD_INB(off[k] <= trash_off, BND_PRIV, args.err))
                                    mb[off[k]] += __uint_as_float(g[k]);
                        }
                        if (ph) to_bf16(g, tbase + ch * 32, row_ok);
                    }
                } else
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t g[32];
                    tmem_ld32(tbase + ch * 32, g);
                    const float4 *cg = colgeo + ch * 32;
                    float *mb = bins + r + kBM * half;
                    void *fbv = fscale != 0.0 ? static_cast<void *>(fbi) : static_cast<void *>(fb);
                    if (mode == BIN_LUT)
                        bin_chunk<BIN_LUT, kBinStride>(g, row_ok, ri, rp, cg, thr_s, mb, fbv, ba);
                    else if (mode == BIN_THR)
                        bin_chunk<BIN_THR, kBinStride>(g, row_ok, ri, rp, cg, thr_s, mb, fbv, ba);
                    else
                        bin_chunk<BIN_POS, kBinStride>(g, row_ok, ri, rp, cg, thr_s, mb, fbv, ba);
                    if (ph) to_bf16(g, tbase + ch * 32, row_ok);
                }
            } else if (ph) {
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t g[32];
                    tmem_ld32(tbase + ch * 32, g);
                    to_bf16(g, tbase + ch * 32, row_ok);
                }
            }
            // without phase weights the accumulator buffer is free for the MMA warp now;
            // with them the BF16 copy of G is in place and the MMA thread may start the
            // phase product (the accumulator stays taken until that product is complete)
            if (ph) tmem_wait_st();
            tc_before();
            __syncwarp();
            // (a pair's epilogue warps arrive on the first CTA's barriers)
            if (lane == 0) {
                const uint32_t a = ph ? conv : tempty0 + 8 * acc;
                if constexpr (CG == 2) mbar_arrive_cl(lead(a));
                else mbar_arrive(a);
            }
            if (last) epi_sync(kEpiThreads);  // all private bins written
            if (bins_on && last) {
                // private rows this tile may have written: with the branch-free position
                // path only the tile's own bin range, else the whole window / bin set
                const int NWp = !E.use_window ? E.n_bins
                                : (!lattice && pos_fit ? min(E.NW, nwp) : E.NW);
                // epilogue warp ew reduces bins b = 4 ew + u (mod 4 EW), four at a time (the
                // four shuffle trees overlap): conflict-free loads, an FP32 tree over the
                // stride, one FP64 add per bin (the FP64 pipe is narrow on this part, so
                // FP64 work is kept per bin, not per row)
                for (int b0 = 4 * ew; b0 < NWp; b0 += 4 * kEpiWarps) {
                    float v4[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        v4[u] = 0.f;
                        if (b0 + u < NWp) {
                            float *row = bins + (b0 + u) * kBinStride;
#pragma unroll
                            for (int m = 0; m < kBinStride / 32; ++m) {
                                v4[u] += row[lane + 32 * m];
                                row[lane + 32 * m] = 0.f;
                            }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int u = 0; u < 4; ++u) v4[u] += __shfl_xor_sync(0xffffffffu, v4[u], o);
                    if (lane == 0)
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int k = b0 + u;
                            const int b = k < n1 ? blo + k : blo2 + (k - n1);
                            if (k < NWp && b < E.n_bins &&
                                ASD_INB(b < args.NB, BND_CACC, args.err)) {
                                if (fscale != 0.0) cacci[b] += to_fixed((double)v4[u], fscale);
                                else cacc[b] += (double)v4[u];
                            }
                        }
                }
                if (E.use_window) {
                    epi_sync(kEpiThreads);  // the fallback bins update the same accumulators
                    for (int b = et; b < E.n_bins; b += kEpiThreads) {
                        if (fscale != 0.0) {
                            cacci[b] += fbi[b];
                            fbi[b] = 0;
                        } else if (fb[b] != 0.f) {
                            cacc[b] += (double)fb[b];
                            fb[b] = 0.f;
                        }
                    }
                }
            }
            // the phase product is read out once per pass; with one pass per tile P sums
            // the tile's K chunks and is read out after the last
            if (ph && (E.npass > 1 || last)) {
                // Phase product of each pass: P[r][o] = sum_c G_rc W_co, u = P[.][0:64)
                // (cosine column weights), v = P[.][64:128) (sine).  Row r adds
                // cos(q.r_i) u + sin(q.r_i) v (cosine part) and sin(q.r_i) u - cos(q.r_i) v
                // (sine part), the angle-difference identities of Eq. 6's weight; the warp
                // then sums its 32 rows by recursive halving (each lane ends with one q
                // of the 16) and adds it to the CTA's FP64 sums.
                const float4 *cs4 = reinterpret_cast<const float4 *>(E.cs) +
                                    (int64_t)ic * (E.nq_pad / 2);
                const uint32_t pt = tmem + ((uint32_t)(q4 * 32) << 16) + 2 * BN;
                // (with 8 epilogue warps the two warps of a lane quarter take half of
                // the pass's q-vectors each)
                constexpr int kJ = kPhaseQ / 16 / kHalves;
                // row weights of 16 q-vectors (8 float4: cos, sin of two q each): the
                // loads of the next group are in flight while the current one is used,
                // those of a pass's first group while its product completes
                auto load_cs = [&](float4 (&c)[8], int q0) {
                    if (q0 < E.n_q && ASD_INB(q0 + 16 <= E.nq_pad, BND_Q, args.err))
#pragma unroll
                        for (int k = 0; k < 8; ++k) c[k] = cs4[q0 / 2 + k];
                };
                for (int pp = 0; pp < E.npass && ok; ++pp) {
                    float4 c4[8];
                    load_cs(c4, pp * kPhaseQ + 16 * half * kJ);
                    const bool gotp = mbar_wait(pfull, n_pass & 1, args.err, DEV_TIMEOUT_EPI);
                    ++n_pass;
                    ok = epi_sync_and(gotp, kEpiThreads);
                    if (!ok) break;
                    tc_after();
                    for (int j = half * kJ; j < (half + 1) * kJ; ++j) {
                        const int q0 = pp * kPhaseQ + 16 * j;
                        if (q0 >= E.n_q) break;
                        uint32_t u[16], w[16];
                        if (j > half * kJ) load_cs(c4, q0);
                        tmem_ld16(pt + 16 * j, u);
                        tmem_ld16(pt + kPhaseQ + 16 * j, w);
                        tmem_wait16x2(u, w);
                        float x[16], y[16];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float ca = c4[k].x, sa = c4[k].y, cb = c4[k].z, sb = c4[k].w;
                            const float u0 = __uint_as_float(u[2 * k]), v0 = __uint_as_float(w[2 * k]);
                            const float u1 = __uint_as_float(u[2 * k + 1]);
                            const float v1 = __uint_as_float(w[2 * k + 1]);
                            x[2 * k] = fmaf(ca, u0, sa * v0);
                            x[2 * k + 1] = fmaf(cb, u1, sb * v1);
                            y[2 * k] = fmaf(sa, u0, -ca * v0);
                            y[2 * k + 1] = fmaf(sb, u1, -cb * v1);
                        }
                        const int qme = q0 + (lane >> 1);
                        const bool qok = (lane & 1) == 0 && qme < E.n_q &&
                                         ASD_INB(qme < args.NQ, BND_Q, args.err);
                        // deterministic mode: fixed-point adds (any order, same bits)
                        const float xs = warp_sum16(x, lane);
                        if (qok) {
                            if (fscale != 0.0)
                                add_fixed(&qacci[2 * qme], to_fixed((double)xs, fscale));
                            else atomicAdd(&qacc[2 * qme], (double)xs);
                        }
                        if (E.q_parts == 2) {
                            const float ys = warp_sum16(y, lane);
                            if (qok) {
                                if (fscale != 0.0)
                                    add_fixed(&qacci[2 * qme + 1], to_fixed((double)ys, fscale));
                                else
                                    atomicAdd(&qacc[2 * qme + 1], (double)ys);
                            }
                        }
                    }
                    // P read: the next pass (or item) may overwrite it
                    tc_before();
                    __syncwarp();
                    if (lane == 0) {
                        if constexpr (CG == 2) mbar_arrive_cl(lead(pempty));
                        else mbar_arrive(pempty);
                    }
                }
                if (!ok) break;
            }
        }
        epi_sync(kEpiThreads);
        if (ok && cur_p >= 0) flush_acc(cur_p, cur_t);
    }
    __syncwarp();
    __syncthreads();
    // a pair: neither CTA leaves (or frees TMEM) while the other may still signal it or
    // the first CTA's MMAs may still write its accumulators
    if constexpr (CG == 2) cluster_sync();
    if (warp == 1) {
        tc_after();
        tmem_dealloc<CG>(tmem, kTmemAlloc);
    }
}

template <int FORM, int BN, int SWB, int EW, int CG>
int launch_one(const LaunchArgs &a, size_t smem, int sm_count, cudaStream_t s)
{
    auto k = pc_tc_kernel<FORM, BN, SWB, EW, CG>;
    constexpr int kThreads = 64 + 32 * EW;
    ASD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if constexpr (CG == 1) {
        // persistent: one CTA per SM, no more CTAs than work items
        const int grid = (int)(a.total_tiles < sm_count ? a.total_tiles : sm_count);
        k<<<grid, kThreads, smem, s>>>(a);
    } else {
        // persistent pairs: clusters of two CTAs, as many as can be resident at once (one
        // CTA per SM), no more than work items
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)sm_count, 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int clusters = 0;
        ASD_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, k, &cfg));
        if (clusters < 1) {
            set_error_text("no CTA pair fits on the device");
            return ASD_EUNSUPPORTED;
        }
        const int64_t pairs = a.total_tiles < clusters ? a.total_tiles : clusters;
        cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
        ASD_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, a));
    }
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // namespace

// Launch one precision form with CTA pairs (tile widths 256 and 192, 4 or 8 epilogue
// warps); instantiated in its own translation unit per form (pc_tc_*_pair.cu).
template <int FORM>
int tc_launch_pair(const TcLaunchArgs &a, size_t smem, int BN, int ew, int sm_count,
                   cudaStream_t s)
{
    constexpr int SWB = FORM == ASD_SPLIT_BF16 ? 64 : 128;
    if (BN == 256 && ew == 4) return launch_one<FORM, 256, SWB, 4, 2>(a, smem, sm_count, s);
    if (BN == 256 && ew == 8) return launch_one<FORM, 256, SWB, 8, 2>(a, smem, sm_count, s);
    if (BN == 192 && ew == 4) return launch_one<FORM, 192, SWB, 4, 2>(a, smem, sm_count, s);
    if (BN == 192 && ew == 8) return launch_one<FORM, 192, SWB, 8, 2>(a, smem, sm_count, s);
    set_error_text("tensor-core kernel: CTA pairs need 192- or 256-wide tiles");
    return ASD_EUNSUPPORTED;
}

// Launch one precision form.  Instantiated combinations (the rest are rejected):
//   BN = 256 and BN = 192 with 4 or 8 epilogue warps; BN = 128 with 4 warps (192 and 128
//   are the tile widths that leave TMEM room for the phase product); cg = 2 goes to the
//   CTA-pair kernels.
template <int FORM>
int tc_launch_form(const TcLaunchArgs &a, size_t smem, int BN, int ew, int cg, int sm_count,
                   cudaStream_t s)
{
    constexpr int SWB = FORM == ASD_SPLIT_BF16 ? 64 : 128;
    if (cg == 2) return tc_launch_pair<FORM>(a, smem, BN, ew, sm_count, s);
    if (BN == 256 && ew == 4) return launch_one<FORM, 256, SWB, 4, 1>(a, smem, sm_count, s);
    if (BN == 256 && ew == 8) return launch_one<FORM, 256, SWB, 8, 1>(a, smem, sm_count, s);
    if (BN == 192 && ew == 4) return launch_one<FORM, 192, SWB, 4, 1>(a, smem, sm_count, s);
    if (BN == 192 && ew == 8) return launch_one<FORM, 192, SWB, 8, 1>(a, smem, sm_count, s);
    if (BN == 128 && ew == 4) return launch_one<FORM, 128, SWB, 4, 1>(a, smem, sm_count, s);
    set_error_text("tensor-core kernel: unsupported (tile width, epilogue warps)");
    return ASD_EUNSUPPORTED;
}

}  // namespace asd
