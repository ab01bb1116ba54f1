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
extern template int tc_launch_form<ASD_SPLIT_BF16>(const TcLaunchArgs &, size_t, int, int, int,
                                                   int, cudaStream_t);

size_t tc_epilogue_smem(int NW, int n_bins, int n_q, int BN, int n_lut, int ew)
{
    return epi_layout(NW, n_bins, n_q, BN, n_lut, ew).total;
}

int tc_configure(asd_corr_plan *p)
{
    const size_t cap = 232448 - 1024 /*alignment slack*/ - 1024 /*barriers*/;
    const size_t stage_bytes = (size_t)p->n_planes * (kBM + p->BN) * p->swizzle_bytes;
    // private bins: as many as fit with at least 3 stages (2 when tight)
    int NW = p->n_bins;
    p->use_window = 0;
    auto epi = [&](int nw) { return tc_epilogue_smem(nw, p->n_bins, p->n_q, p->BN, p->n_lut, p->EW); };
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
              int max_nq, int max_nlut, int cl, int ew, int sm_count, cudaStream_t s)
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
    a.NLUT = max_nlut;
    a.err = device_error_word();
    if (!a.err) return ASD_ECUDA;
    (void)swizzle_bytes;
    switch (prec) {
    case ASD_BF16: return tc_launch_form<ASD_BF16>(a, smem, BN, cl, ew, sm_count, s);
    case ASD_TF32: return tc_launch_form<ASD_TF32>(a, smem, BN, cl, ew, sm_count, s);
    case ASD_SPLIT_BF16: return tc_launch_form<ASD_SPLIT_BF16>(a, smem, BN, cl, ew, sm_count, s);
    default: return ASD_EINVAL;
    }
}

}  // namespace asd
