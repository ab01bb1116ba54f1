/*
 * asd.h -- C ABI of the GB300 spin-dynamics pair-correlation library.
 *
 * Method: arXiv 2308.07487, "Kernel Fusion in Atomistic Spin Dynamics Simulations
 * on Nvidia GPUs using Tensor Core".  The library evaluates the space- and
 * time-displaced spin pair correlation (Eq. 4 / Eq. 5), reduced over distance bins
 * or weighted by the phase factors of Eq. 6 (the real part of Eq. 3), as one fused
 * tensor-core contraction per time displacement (Sections 3.2-3.4) whose N x N
 * result is never written to memory.
 *
 * Conventions for every entry point
 *  - Pointers marked "device" are CUDA device pointers owned by the caller; "host"
 *    pointers are read during the call only.  Nothing is retained except by plans.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work
 *    on it and return without synchronising unless stated otherwise.
 *  - Return value: ASD_OK (0) or a negative ASD_E* code.  Arguments are validated on
 *    the host before anything is launched; on ASD_EINVAL nothing was enqueued.
 *    ASD_ECUDA keeps the CUDA error text for asd_strerror().  A bounded device-side
 *    wait that gave up is reported as ASD_ETIMEOUT by asd_sync_status(), a failed
 *    index check of a checked build (ASD_CHECK_BOUNDS) as ASD_EBOUNDS.
 *  - Units: the device is the current CUDA device of the calling thread.
 */
#ifndef ASD_H
#define ASD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASD_ABI_VERSION 3

enum asd_status {
    ASD_OK = 0,
    ASD_EINVAL = -1,       /* bad shape or argument; nothing launched            */
    ASD_ENOMEM = -2,       /* device or host allocation failed                   */
    ASD_ECUDA = -3,        /* a CUDA runtime/driver call failed                  */
    ASD_ETIMEOUT = -4,     /* a bounded device wait gave up (device error word)  */
    ASD_EUNSUPPORTED = -5, /* valid request this build or device cannot serve    */
    ASD_EBOUNDS = -6       /* a kernel index check of a checked build failed (the
                              access was skipped; device error word)               */
};

/* Precision forms of the contraction (the epilogue and bins are FP32 per tile,
 * FP64 across tiles in every form). */
enum asd_precision {
    ASD_FP32 = 0,        /* FP32 FFMA on the CUDA cores (accuracy baseline)        */
    ASD_TF32 = 1,        /* tcgen05 kind::tf32, operands pre-rounded to TF32       */
    ASD_BF16 = 2,        /* tcgen05 kind::f16 with BF16 operands                   */
    ASD_SPLIT_BF16 = 3   /* x = hi + lo in BF16; hi*hi + hi*lo + lo*hi per product */
};

enum asd_geometry {
    ASD_GEOM_LATTICE = 0,   /* integer coordinates, optional minimum image        */
    ASD_GEOM_POSITIONS = 1  /* FP32 Cartesian positions, no periodicity           */
};

/*
 * Description of one correlation problem.
 *
 * Trajectory layout (device, FP32): traj[i][s][f][a] -- site i = 0..N-1, sample
 * s = 0..S-1, frame f = 0..F-1, component a = 0..2; element offset
 * ((i*S + s)*F + f)*3 + a.  Samples are concatenated along the contraction axis
 * (the paper stacks its M Monte Carlo realisations the same way, Section 3.2).
 *
 * For displacement t = 0..n_t-1 the library forms, for every ordered pair (i,j),
 *   G_ij(t) = sum_{s, t0 < T0, a} A_{i,s,a}(t0 + t) * B_{j,s,a}(t0)
 * with A = B = S (center = 0) or with both operands centred by their mean over
 * (s, t0) (center = 1, Eq. 5).  Requires T0 + n_t - 1 <= F.
 *
 * Distance bins (n_bins > 0): bin(i,j) = max{k >= 0 : (k*w)^2 <= d2(i,j)}, pairs with
 * bin >= n_bins dropped.  d2 is the exact integer squared displacement of the
 * integer coordinates (lattice; minimum image per axis when periodic) or the FP32
 * value fmaf(dz,dz,fmaf(dy,dy,dx*dx)) with dx = x_j - x_i in FP32 (positions).
 * Phase weights (n_q > 0): cos(q.(r_i - r_j)) with r = coords (lattice) or pos.
 */
typedef struct asd_corr_desc {
    int64_t n_sites;        /* N >= 1                                                  */
    int32_t n_frames;       /* F                                                       */
    int32_t n_samples;      /* S >= 1                                                  */
    int32_t T0;             /* time origins >= 1                                       */
    int32_t n_t;            /* displacements >= 1                                      */
    int32_t precision;      /* enum asd_precision                                      */
    int32_t center;         /* 0 or 1                                                  */
    int32_t geometry;       /* enum asd_geometry                                       */
    int32_t L[3];           /* lattice extents (lattice geometry; 1 for unused axes)   */
    int32_t periodic;       /* minimum image per axis (lattice geometry)               */
    const int32_t *coords;  /* host [N][3], lattice geometry (required)                */
    const float *pos;       /* host [N][3], positions geometry (required)              */
    double bin_width;       /* w > 0 when n_bins > 0                                   */
    int32_t n_bins;         /* 0 .. 4096                                               */
    int32_t n_q;            /* 0 .. 256                                                */
    const double *q;        /* host [n_q][3]                                           */
    int32_t tile_n;         /* 0 = automatic (128 for N <= 4096, else 192 with phase
                               weights and 256 without), else 128, 192 or 256 (tensor
                               forms; phase weights need <= 192)                        */
    int32_t raster_m;       /* 0 = automatic, else row tiles per raster group (1..64)  */
    int32_t stages;         /* 0 = automatic, else shared-memory pipeline stages (2..8) */
    int32_t k_chunks;       /* 0 = automatic (split-BF16: one per <= 1024 K elements;
                               other forms: 1), else partial accumulators per tile along K
                               (1..256): each starts from zero, which bounds the
                               tensor-core FP32 accumulation error; the chunks of a tile
                               run back to back on one CTA and the epilogue adds each into
                               the tile's private bins (FP32 within a tile, FP64 across
                               tiles)                                                     */
    int32_t epi_warps;      /* 0 = automatic (8 for positions with 192- or 256-wide
                               tiles, else 4), 4 or 8 epilogue warps per CTA (8 needs
                               tile_n 192 or 256)                                         */
    int32_t phase_sine;     /* 0: Sq_sum[t][q] holds the cosine part of Eq. 3's phase sum;
                               1: Sq_sum[t][q][2] holds (cosine, sine) parts, the sine
                               part sum_ij sin(q.(r_i - r_j)) G_ij(t) (Eq. 3's imaginary
                               part is its negative)                                     */
    int32_t static_schedule;/* 0: work items claimed from a global counter (dynamic,
                               the default); 1: static order (round k of n CTAs: CTA c
                               takes item k n + (c + k) mod n)                            */
    int32_t deterministic;  /* 0: sums across threads and tiles by FP32 / FP64 atomics
                               (the last bits depend on the schedule); 1: every such sum
                               in 64-bit fixed point (integer adds, any order gives the
                               same bits), so C_sum / Sq_sum are bitwise reproducible for
                               any schedule, raster, stage count and batch order at a
                               given precision, tile width and epilogue-warp count.  The
                               fixed-point unit is 2^-e, 2^e the largest power of two
                               with 2 x rows x N x S*3*T0 x max|x|^2 x 2^e < 2^61 (rows of
                               the launch, max|x| over the prepared trajectory, twice that
                               with centring): no sum can overflow, and each rounded term
                               (one per tile, K-chunk and bin or q; one per pair for bins
                               outside a tile's private window) adds at most half a unit.
                               Tensor-core and FP32 forms; not the separable route.      */
    int32_t cta_pair;       /* 0: one CTA per tile (128 rows); 1: tensor forms only, CTA
                               pairs (clusters of two CTAs on two SMs, tcgen05
                               cta_group::2): 256-row tiles, each CTA loading its 128 A
                               rows and half of the B columns, which halves the B-operand
                               traffic per SM; tile_n 192 or 256; static schedule; not
                               for batched launches                                       */
} asd_corr_desc;

typedef struct asd_corr_plan asd_corr_plan;

/*
 * Build a plan: validates `d`, uploads geometry tables (bin thresholds, coordinates
 * or positions, per-site cos/sin(q.r_i) tables), computes the exact ordered-pair
 * count of every bin on the device, allocates the operand workspace (BF16 hi/lo or
 * TF32 copies of the trajectory, zero-padded B operand) and encodes the TMA
 * descriptors.  Synchronises the device.  The plan owns all of it.
 * Errors: ASD_EINVAL (shape/argument), ASD_ENOMEM, ASD_ECUDA, ASD_EUNSUPPORTED
 * (tensor-core form requested on a device without tcgen05).
 */
int asd_pair_corr_plan_create(const asd_corr_desc *d, asd_corr_plan **plan);

/* Free a plan (synchronises the device).  NULL is a no-op. */
void asd_pair_corr_plan_destroy(asd_corr_plan *plan);

/* Bytes of device workspace the plan holds. */
int64_t asd_pair_corr_workspace_bytes(const asd_corr_plan *plan);

/* Exact ordered-pair count of every bin over all N x N pairs (host [n_bins]). */
int asd_pair_corr_counts(const asd_corr_plan *plan, int64_t *counts);

/*
 * The hot path (Sections 3.2-3.4): prepares the operands from `traj` and runs the
 * fused contraction + epilogue for rows i in [row_begin, row_end) against every
 * column j, for every displacement t.  Accumulates (+=) into
 *   C_sum  device FP64 [n_t][n_bins]: sum over pairs in bin b of G_ij(t)
 *   Sq_sum device FP64 [n_t][n_q]:    sum over pairs of cos(q.(r_i-r_j)) G_ij(t)
 * The caller zeroes them; row ranges therefore compose (the row split of the
 * paper's Section 3.5).  Either output may be NULL when its count is 0.
 * traj: device FP32 [N][S][F][3], 16-byte aligned.
 * A plan owns one operand workspace and one work-item counter (the dynamic schedule):
 * calls on one plan must not overlap on the GPU (issue them on one stream or order the
 * streams); different plans are independent.
 */
int asd_pair_corr(asd_corr_plan *plan, const float *traj, int64_t row_begin, int64_t row_end,
                  double *C_sum, double *Sq_sum, void *stream);

/*
 * The two halves of asd_pair_corr.  _prepare builds the operands (the paper's per-step
 * rearrangement and centring, Section 3.2 / Eq. 5) for rows [row_begin, row_end) into
 * the plan's workspace and remembers `traj` (which must stay valid until the last
 * _contract that uses it).  _contract runs the fused contraction + epilogue for any row
 * range inside the last prepared one (ASD_EINVAL otherwise), accumulating like
 * asd_pair_corr.
 */
int asd_pair_corr_prepare(asd_corr_plan *plan, const float *traj, int64_t row_begin,
                          int64_t row_end, void *stream);
int asd_pair_corr_contract(asd_corr_plan *plan, int64_t row_begin, int64_t row_end,
                           double *C_sum, double *Sq_sum, void *stream);

/*
 * asd_pair_corr_contract restricted to the displacements t in [t_begin, t_end)
 * (0 <= t_begin <= t_end <= n_t): every displacement is an independent contraction
 * (the time loop of Algorithm 2), so a long run can be cut into blocks of displacements
 * that accumulate into the same outputs.  C_sum / Sq_sum keep their full [n_t][...] shape
 * and only rows t_begin .. t_end-1 are added to.  ASD_EINVAL for a bad range; an empty
 * range is a no-op.
 */
int asd_pair_corr_contract_range(asd_corr_plan *plan, int64_t row_begin, int64_t row_end,
                                 int32_t t_begin, int32_t t_end, double *C_sum, double *Sq_sum,
                                 void *stream);

/*
 * Several independent problems (each its own plan, trajectory and outputs) in ONE
 * persistent launch over a flattened (problem, t, tile) work list.  All plans must
 * use the same tensor-core precision, tile width and epilogue warp count.  Operand preparation
 * for every problem is enqueued first on the same stream.  Capturable into a CUDA
 * graph (no host synchronisation, no allocation) once the same batch has run eagerly:
 * the work list and its counter live in the first plan (about 10 MB of device memory,
 * allocated by its first batched call, never moved), so a captured graph stays valid
 * until that plan leads a batch of other problems or is destroyed.  None of the plans
 * may be in use by another call that can overlap on the GPU.
 */
int asd_pair_corr_batched(asd_corr_plan *const *plans, const float *const *trajs, int n,
                          double *const *C_sum, double *const *Sq_sum, void *stream);

/*
 * Separable evaluation of the phase-weighted sum: the same quantity as the Sq_sum of
 * asd_pair_corr (the cosine part of Eq. 3 with the weights of Eq. 6, over all ordered
 * pairs, B centred when the plan centres), through cos(a - b) = cos a cos b + sin a sin b:
 * per-site transforms Fc(q; s,f,a) = sum_i cos(q.r_i) S_i(s,f,a) (and Fs with sin) of every
 * frame (FP32 within slices of 4096 sites, FP64 across slices), then
 *   Sq_sum[t][q] += sum_{s,a,t0<T0} Fc(s,t0+t,a) Fc_B(s,t0,a) + Fs(s,t0+t,a) Fs_B(s,t0,a)
 * in FP64.  O(N S F n_q) work instead of O(N^2 S T0 n_t); the paper evaluates the pair
 * form, which asd_pair_corr keeps.
 *   plan    a plan with n_q > 0 (any precision form; the transform is FP32 SIMT)
 *   traj    device [N][S][F][3] FP32, all sites (no row range)
 *   Sq_sum  device [n_t][n_q] FP64, accumulated into
 * Uses the plan's transform buffer (allocated at plan creation): calls on one plan must
 * not overlap.  Enqueue-only (no synchronisation, no allocation).
 */
int asd_pair_corr_sq_separable(asd_corr_plan *plan, const float *traj, double *Sq_sum,
                               void *stream);

/*
 * Dynamical structure factor (Section 4: S(q, omega) from the Fourier transform of S(q,t)
 * in time).  With S(q, -t) = S(q, t) (the cosine form is symmetric under i <-> j):
 *   Sqw[k][q] = dt * ( v_0 S[0][q] + 2 sum_{t=1}^{n_t-1} v_t S[t][q] cos(omega[k] t dt) )
 *   window 0: v_t = 1;  1 (Hann): v_t = (1 + cos(pi t / n_t)) / 2;
 *          2 (Gaussian): v_t = exp(-(t / (width n_t))^2 / 2).
 *   S      device [n_t][n_q] FP64 (any normalisation; typically asd_pair_corr_normalize's)
 *   omega  device [n_w] FP64 angular frequencies, in the inverse unit of dt
 *   Sqw    device [n_w][n_q] FP64, overwritten
 * n_t <= 6000, n_w <= 65535.  FP64 throughout.  Enqueue-only.
 */
int asd_sq_omega(const double *S, int n_t, int n_q, double dt, int window, double width,
                 const double *omega, int n_w, double *Sqw, void *stream);

/*
 * Eq. 3 / Eq. 4 normalisation (device buffers, may alias their inputs):
 *   C[t][b]  = C_sum[t][b] / (S*T0*n_b)   (0 where n_b = 0)
 *   Sq[t][q] = Sq_sum[t][q] / (N*S*T0)
 * Either pair of pointers may be NULL.
 */
int asd_pair_corr_normalize(const asd_corr_plan *plan, const double *C_sum, const double *Sq_sum,
                            double *C, double *Sq, void *stream);

/* Synchronise `stream` and report (then clear) the device error word:
 * ASD_OK, ASD_ETIMEOUT, ASD_EBOUNDS or ASD_ECUDA. */
int asd_sync_status(void *stream);

/* Build flags of the loaded library: bit 0 (ASD_BUILD_CHECK_BOUNDS) is set in a checked
 * build.  A checked build (compiled with ASD_CHECK_BOUNDS=1) tests, in its kernels, every
 * computed index into shared memory and tables -- private-bin offsets and rows, fallback
 * bins, the lattice d2 table, bin thresholds, decoded work items, column and q indices --
 * before the access; the first failure is recorded in the device error word (reported by
 * asd_sync_status as ASD_EBOUNDS, with its site in the error text) and the access is
 * skipped.  It stands in for a memory checker and is slower; results are otherwise the
 * same. */
#define ASD_BUILD_CHECK_BOUNDS 1
int asd_build_flags(void);

/*
 * Self-test of the index-check path of a checked build (the paper has no counterpart).
 * Enqueues one thread that tests an index equal to the length of a 16-entry shared array
 * it owns, the check fails, the store is skipped and the failure is recorded, so the next
 * asd_sync_status reports ASD_EBOUNDS.  In an unchecked build the call returns
 * ASD_EUNSUPPORTED and enqueues nothing.
 */
int asd_selftest_bounds(void *stream);

/*
 * Self-test of the failure path (the paper has no counterpart).  Enqueues on `stream` one
 * thread that waits, through the same bounded wait every mbarrier wait of the tensor-core
 * kernel uses, on a barrier that nothing ever arrives on.  After limit_ns nanoseconds
 * (1 .. 1e9) the wait gives up, records a timeout in the device error word and the kernel
 * returns, so the context stays usable and the next asd_sync_status reports ASD_ETIMEOUT
 * (and clears the word).  Returns ASD_EINVAL for a limit out of range; nothing is allocated.
 */
int asd_selftest_timeout(int64_t limit_ns, void *stream);

/* Static text for a status code (ASD_ECUDA includes the last CUDA error). */
const char *asd_strerror(int status);

/* -------------------------------------------------------------------------------
 * Producers of the trajectory: Monte Carlo sampling (Section 2.1) and
 * Landau-Lifshitz dynamics (Eq. 2, Algorithm 1, RK4 as in Section 3.1).
 * ------------------------------------------------------------------------------- */

/*
 * Spin system for the producers: H = sum_<ij> J_ij S_i.S_j - Hz sum_i S^z_i
 * (Eq. 1 without DM and anisotropy).  Each undirected bond appears in both
 * endpoints' neighbour lists with the same J.
 */
typedef struct asd_system {
    int64_t n_sites;              /* N                                               */
    int32_t z;                    /* neighbour slots per site (1..32)                 */
    const int32_t *nbr;           /* device [N][z], -1 = empty slot                   */
    const float *J;               /* device [N][z]                                    */
    float Hz;                     /* field along z                                    */
    int32_t n_colors;             /* independent-set colouring for parallel updates   */
    const int32_t *color_sites;   /* device: sites of colour 0, then colour 1, ...    */
    const int64_t *color_offsets; /* host [n_colors+1] offsets into color_sites       */
    const float *D;               /* device [N][z][3] DM vector of the directed bond
                                     (i, nbr[i][k]), D_ji = -D_ij; NULL = no DM term  */
    float A;                      /* single-ion anisotropy: -A sum_i (S^z_i)^2        */
} asd_system;
/* H = sum_<ij> J_ij S_i.S_j - sum_<ij> D_ij.(S_i x S_j) - A sum_i (S^z_i)^2
 *     - Hz sum_i S^z_i  (Eq. 1); the local field is
 * h_i = dH/dS_i = sum_j J_ij S_j + sum_j D_ij x S_j - 2 A S^z_i z^ - Hz z^. */

/*
 * Landau-Lifshitz dynamics dS_i/dt = (dH/dS_i) x S_i (Eq. 2), classic RK4 without
 * renormalisation (Section 3.1), for S samples at once.
 *   spins0 device [S][N][3]; traj device [N][S][n_frames][3]: frame 0 = spins0,
 *   frame f = state after f*stride steps of size dt.  spins_out (device [S][N][3],
 *   nullable) receives the final state.  Enqueues 4 kernels per step.
 */
int asd_ll_integrate(const asd_system *sys, int n_samples, const float *spins0, float dt,
                     int n_frames, int stride, float *traj, float *spins_out, void *stream);

/*
 * Same computation and arguments as asd_ll_integrate, for callers that cannot allocate
 * device memory: for example code that runs while another thread holds a global-mode
 * stream capture (cudaMalloc is refused then), processes whose device memory is owned
 * entirely by their own pool allocator, or latency-critical loops that cannot take the
 * implicit synchronisation of cudaMalloc / cudaFree.  The paper has no counterpart; this
 * is a deployment variant only.
 *
 * The RK4 work buffers live in one fixed array in device memory that the library
 * reserves when it is loaded (12 MiB on every GPU that loads it, held until the process
 * exits).  Limit: n_sites * n_samples <= 262144; larger requests return ASD_EINVAL and
 * launch nothing.  The first call on each device looks up that array's device address
 * (a runtime query, no allocation), so make that first call before any stream capture
 * begins.  The address is looked up again when the device's context has changed (after
 * a cudaDeviceReset, for instance).  All calls share the one array: calls whose work can
 * overlap on the GPU (on different streams without ordering) race on it and give wrong
 * results; calls on one stream are safe.  Nothing in the array needs to start at zero: every buffer is fully
 * written before it is read.  Allocates nothing (no cudaMalloc, cudaMallocAsync or
 * cudaFree).
 */
int asd_ll_integrate_noalloc(const asd_system *sys, int n_samples, const float *spins0, float dt,
                             int n_frames, int stride, float *traj, float *spins_out,
                             void *stream);

enum asd_proposal {
    ASD_METROPOLIS = 0,  /* uniform on the sphere, or a cone about the old spin       */
    ASD_HEATBATH = 1,    /* exact conditional: von Mises-Fisher about -h             */
    ASD_LEARNED = 2      /* MLP-proposed von Mises-Fisher + Metropolis-Hastings       */
};

/* Small MLP that maps a site's neighbour spins to a von Mises-Fisher proposal
 * (mean direction, concentration).  Weights are device BF16, row-major [out][in]. */
typedef struct asd_mlp {
    int32_t n_in, n_hidden;       /* n_in = 3 * z                                     */
    const uint16_t *W1, *W2, *W3; /* device bf16 [H][n_in], [H][H], [4][H]            */
    const float *b1, *b2, *b3;    /* device fp32 [H], [H], [4]                        */
    int32_t depth;                /* hidden layers: 2 (0 reads as 2) or 3              */
    const uint16_t *Wm;           /* depth 3: device bf16 [H][H], the third hidden layer
                                     h3 = tanh(Wm h2 + bm) that feeds W3               */
    const float *bm;              /* depth 3: device fp32 [H]                          */
} asd_mlp;

typedef struct asd_mc_stats {
    int64_t proposed;
    int64_t accepted;
    float cone;                   /* final cone half-angle (Metropolis)               */
} asd_mc_stats;

/*
 * Checkerboard Monte Carlo (Section 2.1) at temperature T for S samples
 * (spins device [S][N][3], updated in place), n_sweeps sweeps over all colours.
 * Random numbers: Philox4x32-10 keyed by `seed`, counter (counter + sweep, site,
 * colour); or, when `uniforms` (device [n_sweeps][S][N][4] FP32 in [0,1)) is given,
 * exactly those numbers.  `cone` (radians, <= 0 = whole sphere) is the initial
 * trial-cone half-angle; with adapt != 0 it is rescaled after every sweep to keep the
 * acceptance near 0.5 and never below 0.2.  `stats` (host, nullable) synchronises
 * the stream and returns the totals.
 */
int asd_thermalize(const asd_system *sys, int n_samples, float *spins, float T, int n_sweeps,
                   int proposal, const asd_mlp *net, float cone, int adapt, uint64_t seed,
                   uint64_t counter, const float *uniforms, asd_mc_stats *stats, void *stream);

/* -------------------------------------------------------------------------------
 * Training of the learned proposal network (no counterpart in the paper: an
 * extension of the Monte Carlo sampler of Section 2.1).  Maximum likelihood of a
 * site's spin given its neighbours' spins, on configurations from plain Monte Carlo.
 *
 * `depth` = hidden layers of H = 64 units: 2 or 3.  Parameter vector (device FP32,
 * P = asd_mlp_param_count(n_in, depth) entries):
 *   [W1 H*n_in][b1 H][W2 H*H][b2 H]([Wm H*H][bm H] when depth = 3)[W3 4*H][b3 4]
 * (row-major [out][in]).  BF16 weight buffer (device, asd_mlp_param_count_bf16
 * entries): [W1][W2]([Wm])[W3].  An asd_mlp view for inference points W1, W2, Wm, W3
 * into the BF16 buffer and the biases into the parameter vector.  n_in outside 3..24 or
 * depth outside {2, 3}: count 0, ASD_EINVAL from the other calls.
 * ------------------------------------------------------------------------------- */
int64_t asd_mlp_param_count(int n_in, int depth);
int64_t asd_mlp_param_count_bf16(int n_in, int depth);

/* Initial parameters (Glorot / Xavier uniform): every weight of a layer with fan_in inputs
 * and fan_out outputs is drawn from U(-a, a), a = sqrt(6 / (fan_in + fan_out)), biases are
 * zero.  One Philox4x32-10 draw per parameter (counter = its index in the parameter vector,
 * key = seed), so the result depends on the seed only.  params device FP32 [P], written;
 * w_bf16 device [asd_mlp_param_count_bf16] (nullable) receives the BF16 weight copy.
 * Random initial weights break the symmetry between hidden units that an all-zero start
 * keeps through training.  ASD_EINVAL for n_in outside 3..24. */
int asd_mlp_init(float *params, int n_in, int depth, uint64_t seed, uint16_t *w_bf16,
                 void *stream);

/* BF16 weight copy [W1][W2][W3] of a parameter vector (round to nearest even), for an
 * asd_mlp view of parameters set by the caller.  params device FP32 [P]; w_bf16 device. */
int asd_mlp_weights_bf16(const float *params, int n_in, int depth, uint16_t *w_bf16,
                         void *stream);

/* Training pairs: for sample s and site i (k = s*N + i), x[k] = the z neighbour spins
 * (3z floats, zeros for empty slots) and y[k] = S_i.  spins device [S][N][3];
 * x device [S*N][3z]; y device [S*N][3]. */
int asd_mlp_gather(const asd_system *sys, int n_samples, const float *spins, float *x, float *y,
                   void *stream);

/* Negative log-likelihood of y under vMF(mu(x), kappa(x)) summed over the n pairs,
 * added to *loss (device FP64 scalar), and its gradient with respect to the parameter
 * vector (evaluated at the BF16-rounded weights of `net`) added to grad (device FP32 [P]).
 * kappa = softplus(o_4) + 1e-4. */
int asd_mlp_loss_grad(const asd_mlp *net, int64_t n, const float *x, const float *y, float *grad,
                      double *loss, void *stream);

/* One Adam step (bias-corrected, step >= 1) on params with gradient grad * grad_scale,
 * moments m, v (device FP32 [P]); then writes the BF16 copy of the weights to w_bf16. */
int asd_mlp_adam_step(float *params, const float *grad, float grad_scale, float *m, float *v,
                      int n_in, int depth, float lr, float beta1, float beta2, float eps,
                      int step, uint16_t *w_bf16, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ASD_H */
