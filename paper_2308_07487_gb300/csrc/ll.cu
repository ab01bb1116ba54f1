// Landau-Lifshitz dynamics (Eq. 2): dS_i/dt = (dH/dS_i) x S_i, classic RK4.
//
// H of Eq. 1 (exchange, DM, single-ion anisotropy, field), so the local field is
// h_i = sum_j J_ij S_j + sum_j D_ij x S_j - 2 A S^z_i z^ - Hz z^ (D_ij the DM vector of the
// directed bond, D_ji = -D_ij: Algorithm 1's exchange, DMI, anisotropy and field
// contributions).  As in Algorithm 1, one thread handles
// one site and the S samples are processed by the same launch (the paper passes its
// M configurations to one kernel, Section 3.1); the RK4 stages keep their derivative
// in separate arrays so sites never race (Section 3.1).  No renormalisation: the paper
// notes its RK4 evolution is not norm preserving.
//
// Each RK4 stage is one launch over (sample, site) -- a stage needs every neighbour's
// previous stage.  The last stage writes the new state and, every `stride` steps, the
// trajectory frame in the site-major layout traj[i][s][f][a] consumed by asd_pair_corr.
#include "asd_internal.h"

namespace asd {
namespace {

struct LLArgs {
    int64_t N;
    int S;
    int z;
    const int *nbr;
    const float *J;
    float Hz;
    const float *D;  // [N][z][3] or null
    float A;
};

__device__ __forceinline__ float3 field(const LLArgs &a, const float *__restrict__ Y, int s,
                                        int64_t i)
{
    const float *Ys = Y + (int64_t)s * a.N * 3;
    float3 h = make_float3(0.f, 0.f, -a.Hz);
    for (int k = 0; k < a.z; ++k) {
        const int j = __ldg(a.nbr + i * a.z + k);
        if (j < 0) continue;
        const float Jij = __ldg(a.J + i * a.z + k);
        h.x = fmaf(Jij, Ys[3 * (int64_t)j + 0], h.x);
        h.y = fmaf(Jij, Ys[3 * (int64_t)j + 1], h.y);
        h.z = fmaf(Jij, Ys[3 * (int64_t)j + 2], h.z);
        if (a.D) {  // D_ij x S_j
            const float *d = a.D + (i * a.z + k) * 3;
            const float dx = __ldg(d), dy = __ldg(d + 1), dz = __ldg(d + 2);
            const float sx = Ys[3 * (int64_t)j], sy = Ys[3 * (int64_t)j + 1],
                        sz = Ys[3 * (int64_t)j + 2];
            h.x += dy * sz - dz * sy;
            h.y += dz * sx - dx * sz;
            h.z += dx * sy - dy * sx;
        }
    }
    h.z = fmaf(-2.f * a.A, Ys[3 * i + 2], h.z);
    return h;
}

__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// stage k (1..4): reads Yin (the stage input), writes the next stage input and the
// running combination acc = k1 + 2 k2 + 2 k3.
template <int STAGE>
__global__ void rk4_stage(LLArgs a, float *__restrict__ Y, const float *__restrict__ Yin,
                          float *__restrict__ Yout, float *__restrict__ acc, float dt, float *traj,
                          int F, int frame)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.N * a.S) return;
    const int s = (int)(g / a.N);
    const int64_t i = g % a.N;
    const int64_t o = (int64_t)s * a.N * 3 + 3 * i;
    const float3 h = field(a, Yin, s, i);
    const float3 x = make_float3(Yin[o], Yin[o + 1], Yin[o + 2]);
    const float3 k = cross(h, x);
    const float3 y = make_float3(Y[o], Y[o + 1], Y[o + 2]);
    if (STAGE == 1) {
        acc[o] = k.x; acc[o + 1] = k.y; acc[o + 2] = k.z;
    } else if (STAGE < 4) {
        acc[o] += 2.f * k.x; acc[o + 1] += 2.f * k.y; acc[o + 2] += 2.f * k.z;
    }
    if (STAGE < 4) {
        const float c = STAGE == 3 ? dt : 0.5f * dt;
        Yout[o] = fmaf(c, k.x, y.x);
        Yout[o + 1] = fmaf(c, k.y, y.y);
        Yout[o + 2] = fmaf(c, k.z, y.z);
    } else {
        const float c = dt / 6.f;
        const float3 n = make_float3(fmaf(c, acc[o] + k.x, y.x), fmaf(c, acc[o + 1] + k.y, y.y),
                                     fmaf(c, acc[o + 2] + k.z, y.z));
        Y[o] = n.x; Y[o + 1] = n.y; Y[o + 2] = n.z;
        if (frame >= 0) {
            float *dst = traj + ((i * a.S + s) * (int64_t)F + frame) * 3;
            dst[0] = n.x; dst[1] = n.y; dst[2] = n.z;
        }
    }
}

__global__ void write_frame0(const float *__restrict__ Y, int64_t N, int S, float *traj, int F)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N * S) return;
    const int s = (int)(g / N);
    const int64_t i = g % N;
    const float *src = Y + (int64_t)s * N * 3 + 3 * i;
    float *dst = traj + ((i * S + s) * (int64_t)F) * 3;
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2];
}

}  // namespace
}  // namespace asd

using namespace asd;

extern "C" int asd_ll_integrate(const asd_system *sys, int n_samples, const float *spins0,
                                float dt, int n_frames, int stride, float *traj, float *spins_out,
                                void *stream)
{
    ASD_CHECK_ARG(sys && spins0 && traj, "null argument");
    ASD_CHECK_ARG(sys->n_sites >= 1 && sys->z >= 0 && sys->z <= 32, "bad system");
    ASD_CHECK_ARG(sys->z == 0 || (sys->nbr && sys->J), "neighbour table required");
    ASD_CHECK_ARG(n_samples >= 1 && n_frames >= 1 && stride >= 1, "bad n_samples/n_frames/stride");
    cudaStream_t s = (cudaStream_t)stream;
    LLArgs a{sys->n_sites, n_samples, sys->z, sys->nbr, sys->J, sys->Hz, sys->D, sys->A};
    const int64_t n = sys->n_sites * n_samples;
    const size_t bytes = sizeof(float) * 3 * (size_t)n;
    float *ws = nullptr;
    ASD_CUDA_TRY(cudaMallocAsync(&ws, 4 * bytes, s));
    float *Y = ws, *T1 = ws + 3 * n, *T2 = ws + 6 * n, *acc = ws + 9 * n;
    int rc = ASD_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    do {
        if (cudaMemcpyAsync(Y, spins0, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = ASD_ECUDA;
            break;
        }
        write_frame0<<<blocks, 256, 0, s>>>(Y, sys->n_sites, n_samples, traj, n_frames);
        for (int f = 1; f < n_frames; ++f) {
            for (int k = 0; k < stride; ++k) {
                const int frame = k == stride - 1 ? f : -1;
                rk4_stage<1><<<blocks, 256, 0, s>>>(a, Y, Y, T1, acc, dt, traj, n_frames, -1);
                rk4_stage<2><<<blocks, 256, 0, s>>>(a, Y, T1, T2, acc, dt, traj, n_frames, -1);
                rk4_stage<3><<<blocks, 256, 0, s>>>(a, Y, T2, T1, acc, dt, traj, n_frames, -1);
                rk4_stage<4><<<blocks, 256, 0, s>>>(a, Y, T1, nullptr, acc, dt, traj, n_frames,
                                                    frame);
            }
        }
        if (cudaGetLastError() != cudaSuccess) {
            rc = ASD_ECUDA;
            break;
        }
        if (spins_out &&
            cudaMemcpyAsync(spins_out, Y, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = ASD_ECUDA;
    } while (0);
    cudaFreeAsync(ws, s);
    if (rc == ASD_ECUDA) set_error_text("asd_ll_integrate: launch failed");
    return rc;
}

// ---------------------------------------------------------------------------------------
// No-allocation variant: the same RK4 launches with their four work buffers (state,
// two stage inputs, derivative sum) carved from one fixed device array reserved with the
// library, for callers that cannot allocate device memory (see include/asd.h).
// ---------------------------------------------------------------------------------------
#include <mutex>

namespace asd {
namespace {

constexpr int64_t kLLStaticMaxSiteSamples = 1 << 18;  // n_sites * n_samples limit
constexpr int kLLStaticMaxDevices = 64;

// 4 buffers x 3 components x 262144 site-samples x 4 B = 12 MiB per device
static __device__ __align__(256) float g_ll_scratch[4 * 3 * kLLStaticMaxSiteSamples];

std::mutex g_ll_scratch_mu;
struct ScratchSlot {
    unsigned long long ctx_id;  // context the address belongs to (0: not looked up)
    float *addr;
};
ScratchSlot g_ll_scratch_slot[kLLStaticMaxDevices] = {};

// Unique ID of the calling thread's current context (cuCtxGetId through the runtime's
// driver entry point; no link against libcuda), or 0 when the query is unavailable.
typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long *);
unsigned long long current_context_id()
{
    static PFN_ctxGetCurrent get_cur = nullptr;
    static PFN_ctxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &a, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPoint("cuCtxGetId", &b, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<PFN_ctxGetCurrent>(a);
            get_id = reinterpret_cast<PFN_ctxGetId>(b);
        }
    });
    if (!get_cur || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_ll_scratch in the current context.  In host code the symbol itself
// is only a host-side stand-in; kernels must be given this address.  It is looked up
// once per device and again whenever the device's context has changed (after
// cudaDeviceReset the module, and with it the array, lives at a new address).
int ll_scratch_address(float **out)
{
    int dev = 0;
    ASD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kLLStaticMaxDevices) {
        set_error_text("asd_ll_integrate_noalloc: device index out of range");
        return ASD_EUNSUPPORTED;
    }
    // (cudaGetDevice above leaves the device's primary context current for this thread
    // once the runtime has initialised it; with no context to identify, id is 0 and the
    // address is looked up on every call)
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_ll_scratch_mu);
    ScratchSlot &sl = g_ll_scratch_slot[dev];
    if (!sl.addr || id == 0 || sl.ctx_id != id) {
        void *p = nullptr;
        ASD_CUDA_TRY(cudaGetSymbolAddress(&p, g_ll_scratch));
        sl.addr = static_cast<float *>(p);
        sl.ctx_id = id;
    }
    *out = sl.addr;
    return ASD_OK;
}

}  // namespace
}  // namespace asd

extern "C" int asd_ll_integrate_noalloc(const asd_system *sys, int n_samples, const float *spins0,
                                        float dt, int n_frames, int stride, float *traj,
                                        float *spins_out, void *stream)
{
    ASD_CHECK_ARG(sys && spins0 && traj, "null argument");
    ASD_CHECK_ARG(sys->n_sites >= 1 && sys->z >= 0 && sys->z <= 32, "bad system");
    ASD_CHECK_ARG(sys->z == 0 || (sys->nbr && sys->J), "neighbour table required");
    ASD_CHECK_ARG(n_samples >= 1 && n_frames >= 1 && stride >= 1, "bad n_samples/n_frames/stride");
    ASD_CHECK_ARG(sys->n_sites * (int64_t)n_samples <= kLLStaticMaxSiteSamples,
                  "asd_ll_integrate_noalloc: n_sites * n_samples exceeds the fixed work area "
                  "(262144 site-samples); use asd_ll_integrate");
    float *ws = nullptr;
    int rc = ll_scratch_address(&ws);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    LLArgs a{sys->n_sites, n_samples, sys->z, sys->nbr, sys->J, sys->Hz, sys->D, sys->A};
    const int64_t n = sys->n_sites * n_samples;
    const size_t bytes = sizeof(float) * 3 * (size_t)n;
    // every buffer is written before it is read: Y by the copy, acc by stage 1, T1 / T2
    // by the stage that produces them, so no clearing is needed
    float *Y = ws, *T1 = ws + 3 * n, *T2 = ws + 6 * n, *acc = ws + 9 * n;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    ASD_CUDA_TRY(cudaMemcpyAsync(Y, spins0, bytes, cudaMemcpyDeviceToDevice, s));
    write_frame0<<<blocks, 256, 0, s>>>(Y, sys->n_sites, n_samples, traj, n_frames);
    for (int f = 1; f < n_frames; ++f) {
        for (int k = 0; k < stride; ++k) {
            const int frame = k == stride - 1 ? f : -1;
            rk4_stage<1><<<blocks, 256, 0, s>>>(a, Y, Y, T1, acc, dt, traj, n_frames, -1);
            rk4_stage<2><<<blocks, 256, 0, s>>>(a, Y, T1, T2, acc, dt, traj, n_frames, -1);
            rk4_stage<3><<<blocks, 256, 0, s>>>(a, Y, T2, T1, acc, dt, traj, n_frames, -1);
            rk4_stage<4><<<blocks, 256, 0, s>>>(a, Y, T1, nullptr, acc, dt, traj, n_frames, frame);
        }
    }
    ASD_CUDA_TRY(cudaGetLastError());
    if (spins_out)
        ASD_CUDA_TRY(cudaMemcpyAsync(spins_out, Y, bytes, cudaMemcpyDeviceToDevice, s));
    return ASD_OK;
}
