// Classical Monte Carlo for Heisenberg spins (Section 2.1), checkerboard-parallel.
//
// Metropolis: a trial spin is drawn uniformly on the sphere, or inside a cone about the
// current spin whose half-angle adapts between sweeps (the paper keeps the acceptance
// rate at least 20 %); it is accepted with probability min(1, exp(-beta dE)).
// Heat-bath: the new spin is drawn from the exact conditional of the terms linear in S,
// p(S) ~ exp(-beta S.h), a von Mises-Fisher law with mean -h/|h| and concentration
// beta|h|; with single-ion anisotropy the draw is a Metropolis-Hastings proposal accepted
// with min(1, exp(beta A (Sz_new^2 - Sz_old^2))), which keeps the chain exact.
// Energy change of a move: dE = (S' - S).h - A (S'z^2 - Sz^2), h = sum_j J_ij S_j +
// sum_j D_ij x S_j - Hz z^ (Eq. 1).
// Learned: a small MLP maps the neighbour spins to a vMF proposal; the
// Metropolis-Hastings ratio exp(-beta dE) q(S_old)/q(S_new) keeps the chain exact.
//
// Sites of one colour have no neighbours of that colour, so a colour is updated in
// one launch without races.  Randomness: Philox4x32-10 (Salmon et al., SC'11) keyed
// by the seed, counter (sweep, colour, sample, site); or caller-supplied uniforms.
#include <cuda_bf16.h>

#include "asd_internal.h"
#include "mlp.cuh"
#include "philox.cuh"

namespace asd {
namespace {

struct MCArgs {
    int64_t N;
    int S;
    int z;
    const int *nbr;
    const float *J;
    float Hz;
    const float *D;     // [N][z][3] DM vectors or null
    float A;            // single-ion anisotropy
    float beta;
    int proposal;
    const int *sites;   // this colour's sites
    int64_t n_sites_c;
    uint64_t seed;
    uint64_t ctr;       // counter + sweep
    int color;
    const float *uni;   // optional [S][N][4] uniforms of this sweep
    const float *cone;  // device cone half-angle
    unsigned long long *stats;  // [2]: proposed, accepted
    MlpView net;
};

__device__ __forceinline__ float3 f3(const float *p) { return make_float3(p[0], p[1], p[2]); }

// unit vectors e1, e2 with (e1, e2, m) right-handed; the same rule as the oracle
__device__ __forceinline__ void frame_of(float3 m, float3 &e1, float3 &e2)
{
    float3 a = fabsf(m.z) < 0.9f ? make_float3(0.f, 0.f, 1.f) : make_float3(1.f, 0.f, 0.f);
    float3 c = make_float3(a.y * m.z - a.z * m.y, a.z * m.x - a.x * m.z, a.x * m.y - a.y * m.x);
    const float inv = rsqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
    e1 = make_float3(c.x * inv, c.y * inv, c.z * inv);
    e2 = make_float3(m.y * e1.z - m.z * e1.y, m.z * e1.x - m.x * e1.z, m.x * e1.y - m.y * e1.x);
}

__device__ __forceinline__ float3 around(float3 m, float c, float phi)
{
    float3 e1, e2;
    frame_of(m, e1, e2);
    const float s = sqrtf(fmaxf(0.f, 1.f - c * c));
    float sp, cp;
    sincosf(phi, &sp, &cp);
    return make_float3(c * m.x + s * (cp * e1.x + sp * e2.x), c * m.y + s * (cp * e1.y + sp * e2.y),
                       c * m.z + s * (cp * e1.z + sp * e2.z));
}

// cos of the angle to the mean for vMF(kappa) in 3D, from u in (0, 1]
__device__ __forceinline__ float vmf_w(float kappa, float u)
{
    if (kappa < 1e-6f) return 1.f - 2.f * u;
    return fmaxf(-1.f, 1.f + logf(u + (1.f - u) * expf(-2.f * kappa)) / kappa);
}

__global__ void mc_color_kernel(MCArgs a, float *__restrict__ spins)
{
    __shared__ unsigned int cnt[2];
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool prop = false, acc = false;
    if (g < a.n_sites_c * a.S) {
        const int s = (int)(g / a.n_sites_c);
        const int64_t i = a.sites[g % a.n_sites_c];
        float *Ys = spins + (int64_t)s * a.N * 3;
        float3 h = make_float3(0.f, 0.f, -a.Hz);
        float nb[32 * 3];
        for (int k = 0; k < a.z; ++k) {
            const int j = a.nbr[i * a.z + k];
            const float3 sj = j >= 0 ? f3(Ys + 3 * (int64_t)j) : make_float3(0.f, 0.f, 0.f);
            const float Jij = j >= 0 ? a.J[i * a.z + k] : 0.f;
            h.x = fmaf(Jij, sj.x, h.x);
            h.y = fmaf(Jij, sj.y, h.y);
            h.z = fmaf(Jij, sj.z, h.z);
            if (a.D && j >= 0) {  // D_ij x S_j
                const float *d = a.D + (i * a.z + k) * 3;
                h.x += d[1] * sj.z - d[2] * sj.y;
                h.y += d[2] * sj.x - d[0] * sj.z;
                h.z += d[0] * sj.y - d[1] * sj.x;
            }
            if (a.proposal == ASD_LEARNED && k < 32) {
                nb[3 * k] = sj.x;
                nb[3 * k + 1] = sj.y;
                nb[3 * k + 2] = sj.z;
            }
        }
        float u[4];
        if (a.uni) {
            const float *up = a.uni + ((int64_t)s * a.N + i) * 4;
            u[0] = up[0]; u[1] = up[1]; u[2] = up[2]; u[3] = up[3];
        } else {
            const U4 r = philox4x32_10(U4{(uint32_t)i, (uint32_t)(i >> 32) ^ ((uint32_t)s << 8) ^
                                                           ((uint32_t)a.color << 28),
                                          (uint32_t)a.ctr, (uint32_t)(a.ctr >> 32)},
                                       (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
            u[0] = u01(r.x); u[1] = u01(r.y); u[2] = u01(r.z); u[3] = u01(r.w);
        }
        const float3 old = f3(Ys + 3 * i);
        float3 nw;
        float logq_ratio = 0.f;  // log q(old) - log q(new) for the learned proposal
        const float TWO_PI = 6.283185307179586f;
        if (a.proposal == ASD_HEATBATH) {
            const float hn = sqrtf(h.x * h.x + h.y * h.y + h.z * h.z);
            const float kappa = a.beta * hn;
            float3 m = hn > 0.f ? make_float3(-h.x / hn, -h.y / hn, -h.z / hn)
                                : make_float3(0.f, 0.f, 1.f);
            nw = around(m, vmf_w(kappa, u[0]), TWO_PI * u[1]);
        } else if (a.proposal == ASD_LEARNED) {
            float mu[3], kappa;
            mlp_vmf(a.net, nb, mu, &kappa);
            const float3 m = make_float3(mu[0], mu[1], mu[2]);
            nw = around(m, vmf_w(kappa, u[0]), TWO_PI * u[1]);
            logq_ratio = kappa * ((old.x - nw.x) * m.x + (old.y - nw.y) * m.y + (old.z - nw.z) * m.z);
        } else {
            const float cone = *a.cone;
            const float cmin = cone <= 0.f || cone >= 3.14159265f ? -1.f : cosf(cone);
            nw = around(old, 1.f - u[0] * (1.f - cmin), TWO_PI * u[1]);
        }
        prop = true;
        const float daniso = a.A * (nw.z * nw.z - old.z * old.z);  // -(anisotropy change)
        if (a.proposal == ASD_HEATBATH) {
            const float la = a.beta * daniso;
            acc = la >= 0.f || u[2] < expf(la);
        } else {
            const float dE = (nw.x - old.x) * h.x + (nw.y - old.y) * h.y +
                             (nw.z - old.z) * h.z - daniso;
            const float la = -a.beta * dE + logq_ratio;
            acc = la >= 0.f || u[2] < expf(la);
        }
        if (acc) {
            Ys[3 * i] = nw.x;
            Ys[3 * i + 1] = nw.y;
            Ys[3 * i + 2] = nw.z;
        }
    }
    if (prop) atomicAdd(&cnt[0], 1u);
    if (acc) atomicAdd(&cnt[1], 1u);
    __syncthreads();
    if (threadIdx.x == 0 && cnt[0]) {
        atomicAdd(&a.stats[0], (unsigned long long)cnt[0]);
        atomicAdd(&a.stats[1], (unsigned long long)cnt[1]);
    }
}

// cone <- cone * clamp(acceptance / 0.5, 0.5, 2), at most pi; counters of the sweep reset
__global__ void adapt_cone(unsigned long long *sweep_stats, unsigned long long *total, float *cone)
{
    const unsigned long long p = sweep_stats[0], a = sweep_stats[1];
    total[0] += p;
    total[1] += a;
    sweep_stats[0] = sweep_stats[1] = 0;
    if (p == 0) return;
    float r = (float)a / (float)p / 0.5f;
    r = fminf(2.f, fmaxf(0.5f, r));
    float c = *cone <= 0.f ? 3.14159265f : *cone;
    *cone = fminf(3.14159265f, c * r);
}

__global__ void accumulate_stats(unsigned long long *sweep_stats, unsigned long long *total)
{
    total[0] += sweep_stats[0];
    total[1] += sweep_stats[1];
    sweep_stats[0] = sweep_stats[1] = 0;
}

}  // namespace
}  // namespace asd

using namespace asd;

extern "C" int asd_thermalize(const asd_system *sys, int n_samples, float *spins, float T,
                              int n_sweeps, int proposal, const asd_mlp *net, float cone,
                              int adapt, uint64_t seed, uint64_t counter, const float *uniforms,
                              asd_mc_stats *stats, void *stream)
{
    ASD_CHECK_ARG(sys && spins, "null argument");
    ASD_CHECK_ARG(sys->n_sites >= 1 && sys->z >= 0 && sys->z <= 32, "bad system");
    ASD_CHECK_ARG(sys->z == 0 || (sys->nbr && sys->J), "neighbour table required");
    ASD_CHECK_ARG(sys->n_colors >= 1 && sys->color_sites && sys->color_offsets, "colouring required");
    ASD_CHECK_ARG(sys->color_offsets[0] == 0 && sys->color_offsets[sys->n_colors] == sys->n_sites,
                  "colour offsets must cover every site once");
    ASD_CHECK_ARG(n_samples >= 1 && n_sweeps >= 0 && T > 0.f, "bad n_samples/n_sweeps/T");
    ASD_CHECK_ARG(proposal >= ASD_METROPOLIS && proposal <= ASD_LEARNED, "bad proposal");
    MlpView view{};
    if (proposal == ASD_LEARNED) {
        ASD_CHECK_ARG(net && net->W1 && net->W2 && net->W3 && net->b1 && net->b2 && net->b3,
                      "learned proposal needs a network");
        ASD_CHECK_ARG(net->n_in == 3 * sys->z && net->n_in <= kMlpMaxIn &&
                          net->n_hidden == kMlpHidden,
                      "network shape must be [3z -> 64 (x2 or x3) -> 4]");
        ASD_CHECK_ARG(mlp_depth(*net) == 2 || (mlp_depth(*net) == 3 && net->Wm && net->bm),
                      "network depth must be 2, or 3 with the third layer's weights");
        view = mlp_view(*net);
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *cnt = nullptr;
    ASD_CUDA_TRY(cudaMallocAsync(&cnt, 4 * sizeof(unsigned long long) + sizeof(float), s));
    float *d_cone = reinterpret_cast<float *>(cnt + 4);
    int rc = ASD_OK;
    do {
        if (cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess ||
            cudaMemcpyAsync(d_cone, &cone, sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = ASD_ECUDA;
            break;
        }
        MCArgs a{};
        a.N = sys->n_sites;
        a.S = n_samples;
        a.z = sys->z;
        a.nbr = sys->nbr;
        a.J = sys->J;
        a.Hz = sys->Hz;
        a.D = sys->D;
        a.A = sys->A;
        a.beta = 1.f / T;
        a.proposal = proposal;
        a.seed = seed;
        a.cone = d_cone;
        a.stats = cnt;
        a.net = view;
        for (int sw = 0; sw < n_sweeps; ++sw) {
            a.ctr = counter + (uint64_t)sw;
            a.uni = uniforms ? uniforms + (size_t)sw * n_samples * sys->n_sites * 4 : nullptr;
            for (int c = 0; c < sys->n_colors; ++c) {
                a.color = c;
                a.sites = sys->color_sites + sys->color_offsets[c];
                a.n_sites_c = sys->color_offsets[c + 1] - sys->color_offsets[c];
                const int64_t n = a.n_sites_c * n_samples;
                if (n == 0) continue;
                mc_color_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a, spins);
            }
            if (adapt && proposal == ASD_METROPOLIS) adapt_cone<<<1, 1, 0, s>>>(cnt, cnt + 2, d_cone);
            else accumulate_stats<<<1, 1, 0, s>>>(cnt, cnt + 2);
        }
        if (cudaGetLastError() != cudaSuccess) {
            rc = ASD_ECUDA;
            break;
        }
        if (stats) {
            unsigned long long h[2];
            float hc;
            if (cudaMemcpyAsync(h, cnt + 2, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(&hc, d_cone, sizeof hc, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = ASD_ECUDA;
                break;
            }
            stats->proposed = (int64_t)h[0];
            stats->accepted = (int64_t)h[1];
            stats->cone = hc;
        }
    } while (0);
    cudaFreeAsync(cnt, s);
    if (rc == ASD_ECUDA) set_error_text("asd_thermalize: CUDA call failed");
    return rc;
}
