// Tensor-core forms: shared-memory configuration of a plan and launch dispatch.  The
// kernel itself is in pc_tc_kernel.cuh, instantiated once per precision form in
// pc_tc_bf16.cu, pc_tc_tf32.cu and pc_tc_split.cu (compiled in parallel).
#include "pc_tc_kernel.cuh"

namespace asd {

// instantiated in the per-form translation units
extern template int tc_launch_form<ASD_BF16>(const TcLaunchArgs &, size_t, int, int, int, int,
                                             cudaStream_t);
extern template int tc_launch_form<ASD_TF32>(const TcLaunchArgs &, size_t, int, int, int, int,
                                             cudaStream_t);
extern template int tc_launch_form<ASD_SPLIT_BF16>(const TcLaunchArgs &, size_t, int, int, int, int,
                                                   cudaStream_t);

uint32_t tc_var_bytes(int NW, int n_bins, int n_lut, int ew) { return var_bytes(NW, n_bins, n_lut, ew); }

size_t tc_epilogue_smem_vb(uint32_t vb, int n_bins, int n_q, int BN, int ew, int det)
{
    return epi_layout(vb, n_bins, n_q, BN, ew, det).total;
}

size_t tc_epilogue_smem(int NW, int n_bins, int n_q, int BN, int n_lut, int ew, int det)
{
    return epi_layout(var_bytes(NW, n_bins, n_lut, ew), n_bins, n_q, BN, ew, det).total;
}

// Bins window and stage count for the plan's current table choice; returns the number of
// stages that fit (before any user cap), 0 when the epilogue does not fit at all.
static int configure_once(asd_corr_plan *p, size_t cap, size_t stage_bytes)
{
    // private bins: as many as fit with at least 3 stages (2 when tight)
    int NW = p->n_bins;
    p->use_window = 0;
    auto epi = [&](int nw) {
        return tc_epilogue_smem(nw, p->n_bins, p->n_q, p->BN, p->n_lut, p->EW, p->d.deterministic);
    };
    for (int min_st = 3; min_st >= 2; --min_st) {
        NW = p->n_bins;
        while (NW > 8 && epi(NW) + min_st * stage_bytes > cap) NW = (NW * 3) / 4;
        if (epi(NW) + min_st * stage_bytes <= cap) break;
    }
    if (epi(NW) + 2 * stage_bytes > cap) return 0;
    if (NW < p->n_bins) p->use_window = 1;
    if (p->n_bins == 0) NW = 0;
    p->NW = NW;
    return (int)((cap - epi(NW)) / stage_bytes);
}

int tc_configure(asd_corr_plan *p)
{
    const size_t cap = 232448 - 1024 /*alignment slack*/ - 1024 /*barriers*/;
    // (a CTA pair's stage holds this CTA's half of the B columns)
    const size_t stage_bytes = (size_t)p->n_planes * (kBM + p->BN / p->CG) * p->swizzle_bytes;
    int st = configure_once(p, cap, stage_bytes);
    // a d2 -> bin table that costs the third pipeline stage (or the whole bin set) is
    // dropped: the threshold rule bins the same pairs with a few more instructions, and
    // the third stage is worth more (measured)
    if (p->n_lut > 0 && (st < 3 || p->use_window)) {
        const int keep = p->n_lut;
        p->n_lut = 0;
        const int st2 = configure_once(p, cap, stage_bytes);
        if (st2 >= 3 && !p->use_window) {
            st = st2;
        } else {
            p->n_lut = keep;
            st = configure_once(p, cap, stage_bytes);
        }
    }
    if (st == 0) {
        set_error_text("epilogue does not fit shared memory");
        return ASD_EUNSUPPORTED;
    }
    if (st > 8) st = 8;
    if (p->d.stages > 0 && p->d.stages < st) st = p->d.stages;
    p->stages = st;
    p->smem_bytes = tc_epilogue_smem(p->NW, p->n_bins, p->n_q, p->BN, p->n_lut, p->EW,
                                     p->d.deterministic) +
                    (size_t)p->stages * stage_bytes + 2048;
    // more than half of the SM's shared memory: never two CTAs (and TMEM owners) per SM
    if (p->smem_bytes < kMinSmem) p->smem_bytes = kMinSmem;
    return ASD_OK;
}

int launch_tc(const TcProblem *d_probs, int n_probs, int64_t total_tiles, TcOverride ov, int prec,
              int BN, int swizzle_bytes, int stages, size_t smem, uint32_t var_bytes_,
              int max_nb, int max_nq, int ew, int det, int cg, int sm_count,
              unsigned long long *counter, cudaStream_t s)
{
    if (total_tiles <= 0) return ASD_OK;
    LaunchArgs a{};
    a.probs = d_probs;
    a.n_probs = n_probs;
    a.total_tiles = total_tiles;
    a.ov = ov;
    a.stages = stages;
    a.VB = var_bytes_;
    // dynamic schedule: the counter starts at zero for every launch (stream-ordered)
    a.counter = counter;
    if (a.counter) ASD_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s));
    a.NB = max_nb;
    a.NQ = max_nq;
    a.det = det;
    a.err = device_error_word();
    if (!a.err) return ASD_ECUDA;
    (void)swizzle_bytes;
    switch (prec) {
    case ASD_BF16: return tc_launch_form<ASD_BF16>(a, smem, BN, ew, cg, sm_count, s);
    case ASD_TF32: return tc_launch_form<ASD_TF32>(a, smem, BN, ew, cg, sm_count, s);
    case ASD_SPLIT_BF16: return tc_launch_form<ASD_SPLIT_BF16>(a, smem, BN, ew, cg, sm_count,
                                                                   s);
    default: return ASD_EINVAL;
    }
}

// One thread waits, through the bounded wait of the tensor-core kernel, on an mbarrier
// that nothing arrives on: after limit_ns the wait records DEV_TIMEOUT_SELFTEST in the
// device error word and the kernel returns.
__global__ void wait_selftest_kernel(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(saddr(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        (void)mbar_wait_for(saddr(&bar), 0, err, DEV_TIMEOUT_SELFTEST, limit_ns);
    }
}

}  // namespace asd

#if ASD_CHECK_BOUNDS
namespace asd {
// One thread stores into a 16-entry shared array at index 16: the check fails, the store
// is skipped and BND_SELFTEST is recorded.
__global__ void bounds_selftest_kernel(int *err, int idx)
{
    __shared__ int a[16];
    if (threadIdx.x == 0 && ASD_INB(idx >= 0 && idx < 16, BND_SELFTEST, err)) a[idx] = 1;
}
}  // namespace asd
#endif

int asd_build_flags(void) { return ASD_CHECK_BOUNDS ? ASD_BUILD_CHECK_BOUNDS : 0; }

int asd_selftest_bounds(void *stream)
{
#if ASD_CHECK_BOUNDS
    using namespace asd;
    int *err = device_error_word();
    if (!err) return ASD_ECUDA;
    bounds_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(err, 16);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
#else
    (void)stream;
    asd::set_error_text("not a checked build (ASD_CHECK_BOUNDS)");
    return ASD_EUNSUPPORTED;
#endif
}

int asd_selftest_timeout(int64_t limit_ns, void *stream)
{
    using namespace asd;
    ASD_CHECK_ARG(limit_ns > 0 && limit_ns <= 1000000000, "limit_ns: 1 .. 1e9");
    int *err = device_error_word();
    if (!err) return ASD_ECUDA;
    wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(err, (unsigned long long)limit_ns);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}
