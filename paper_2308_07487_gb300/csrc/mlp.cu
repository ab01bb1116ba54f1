// Training of the learned von Mises-Fisher proposal (extension of the Monte Carlo of
// Section 2.1; the paper has no learned component).
//
// Model: x (neighbour spins, 3z) -> tanh(W1 x + b1) -> tanh(W2 h1 + b2)
// [-> tanh(Wm h2 + bm) with three hidden layers] -> o = W3 h_last + b3,
// mu = o[0:3]/|o[0:3]|, kappa = softplus(o[3]) + 1e-4.  Loss: the negative log-likelihood
// of the site spin y under vMF(mu, kappa):
//   NLL = -log kappa + log(2 pi) + kappa + log(1 - e^{-2 kappa}) - kappa mu.y
// (log of the normaliser 4 pi sinh(kappa) / kappa written to stay finite).
// Gradients: dNLL/dkappa = coth(kappa) - 1/kappa - mu.y (the Langevin function, with a
// series below kappa = 1e-2), dNLL/dv = -kappa (y - mu (mu.y)) / |v| for v = o[0:3],
// then back through the tanh layers.
//
// loss_grad: persistent blocks of 64 threads, one sample per thread per chunk.  The
// activations and deltas of a chunk go to shared memory (rows padded to H + 1 floats, so
// a thread's own row and a warp's sweep along one row are both free of bank conflicts);
// each thread then owns a strided set of parameter entries and sums their gradient over
// the chunk, so the whole launch issues one global atomic per parameter per block.
#include <cuda_bf16.h>

#include "asd_internal.h"
#include "mlp.cuh"
#include "philox.cuh"

namespace asd {
namespace {

constexpr int H = kMlpHidden;
constexpr int kChunk = 64;
constexpr int kHP = H + 1;   // padded activation row

// Packed parameters [W1 H*nin][b1 H] then, per further hidden layer, [W H*H][b H], then
// [W3 4*H][b3 4]; BF16 weights [W1]([W2][Wm])[W3].
__host__ __device__ inline int64_t n_params(int nin, int depth)
{
    return (int64_t)H * nin + H + (int64_t)(depth - 1) * (H * H + H) + 4 * H + 4;
}
__host__ __device__ inline int64_t n_weights(int nin, int depth)
{
    return (int64_t)H * nin + (int64_t)(depth - 1) * H * H + 4 * H;
}
inline bool shape_ok(int nin, int depth)
{
    return nin >= 3 && nin <= kMlpMaxIn && (depth == 2 || depth == 3);
}

__global__ void gather_kernel(int64_t N, int S, int z, const int *__restrict__ nbr,
                              const float *__restrict__ spins, float *__restrict__ x,
                              float *__restrict__ y)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N * S) return;
    const int64_t s = k / N, i = k % N;
    const float *Ys = spins + s * N * 3;
    for (int a = 0; a < z; ++a) {
        const int j = nbr[i * z + a];
        for (int c = 0; c < 3; ++c) x[k * 3 * z + 3 * a + c] = j >= 0 ? Ys[3 * (int64_t)j + c] : 0.f;
    }
    for (int c = 0; c < 3; ++c) y[3 * k + c] = Ys[3 * i + c];
}

__device__ __forceinline__ float langevin(float k)
{
    if (k < 1e-2f) return k * (1.f / 3.f) - k * k * k * (1.f / 45.f);
    return 1.f / tanhf(k) - 1.f / k;
}

__global__ void __launch_bounds__(kChunk) loss_grad_kernel(MlpView net, int64_t n,
                                                            const float *__restrict__ x,
                                                            const float *__restrict__ y,
                                                            float *__restrict__ grad,
                                                            double *__restrict__ loss)
{
    const int nin = net.n_in, depth = net.depth;
    const int P = (int)n_params(nin, depth);
    extern __shared__ float sm[];
    float *W1 = sm;                                 // [H][nin]
    float *Wh = W1 + H * nin;                       // [depth - 1][H][H]: W2 (Wm)
    float *W3 = Wh + (depth - 1) * H * H;           // [4][H]
    float *Xs = W3 + 4 * H;                         // [chunk][nin + 1]
    float *Hs = Xs + kChunk * (nin + 1);            // [depth][chunk][kHP] activations
    float *Ds = Hs + depth * kChunk * kHP;          // [depth][chunk][kHP] deltas
    float *DO = Ds + depth * kChunk * kHP;          // [chunk][4]
    float *acc = DO + kChunk * 4;                   // [P] gradient accumulator of this block
    __shared__ double lsum[kChunk];

    const int t = threadIdx.x;
    for (int e = t; e < H * nin; e += kChunk) W1[e] = __bfloat162float(net.W1[e]);
    for (int e = t; e < H * H; e += kChunk) Wh[e] = __bfloat162float(net.W2[e]);
    if (depth == 3)
        for (int e = t; e < H * H; e += kChunk) Wh[H * H + e] = __bfloat162float(net.Wm[e]);
    for (int e = t; e < 4 * H; e += kChunk) W3[e] = __bfloat162float(net.W3[e]);
    for (int e = t; e < P; e += kChunk) acc[e] = 0.f;
    double my_loss = 0.0;
    __syncthreads();

    const int nin1 = nin + 1;
    for (int64_t base = (int64_t)blockIdx.x * kChunk; base < n; base += (int64_t)gridDim.x * kChunk) {
        const int64_t s = base + t;
        const bool ok = s < n;
        float xv[kMlpMaxIn];
        for (int c = 0; c < nin; ++c) {
            xv[c] = ok ? x[s * nin + c] : 0.f;
            Xs[t * nin1 + c] = xv[c];
        }
        // forward: hc = the current layer, hp = the one before it
        float hp[H], hc[H], o[4];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            float a = __ldg(net.b1 + k);
            for (int c = 0; c < nin; ++c) a = fmaf(W1[k * nin + c], xv[c], a);
            hc[k] = tanhf(a);
            Hs[t * kHP + k] = hc[k];
        }
        for (int l = 1; l < depth; ++l) {
            const float *Wl = Wh + (l - 1) * H * H;
            const float *bl = l == 1 ? net.b2 : net.bm;
#pragma unroll
            for (int k = 0; k < H; ++k) hp[k] = hc[k];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                float a = __ldg(bl + k);
#pragma unroll
                for (int c = 0; c < H; ++c) a = fmaf(Wl[k * H + c], hp[c], a);
                hc[k] = tanhf(a);
                Hs[(l * kChunk + t) * kHP + k] = hc[k];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float a = __ldg(net.b3 + k);
#pragma unroll
            for (int c = 0; c < H; ++c) a = fmaf(W3[k * H + c], hc[c], a);
            o[k] = a;
        }
        float yv[3] = {0.f, 0.f, 0.f};
        if (ok)
            for (int c = 0; c < 3; ++c) yv[c] = y[s * 3 + c];
        const float vn = sqrtf(fmaxf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2], 1e-30f));
        const float mu[3] = {o[0] / vn, o[1] / vn, o[2] / vn};
        const float kap = softplus_f(o[3]) + 1e-4f;
        const float muy = mu[0] * yv[0] + mu[1] * yv[1] + mu[2] * yv[2];
        float dO[4];
        if (ok) {
            my_loss += (double)(-logf(kap) + 1.8378770664093453f + kap + log1pf(-expf(-2.f * kap)) -
                                kap * muy);
            const float dk = langevin(kap) - muy;
            dO[3] = dk / (1.f + expf(-o[3]));  // d softplus / d o3 = sigmoid(o3)
            for (int c = 0; c < 3; ++c) dO[c] = -kap * (yv[c] - mu[c] * muy) / vn;
        } else {
            dO[0] = dO[1] = dO[2] = dO[3] = 0.f;
        }
        // backward: delta of the last hidden layer, then down through the layers
        float d[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            float g = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) g = fmaf(W3[q * H + k], dO[q], g);
            d[k] = g * (1.f - hc[k] * hc[k]);
            Ds[((depth - 1) * kChunk + t) * kHP + k] = d[k];
        }
        for (int l = depth - 1; l >= 1; --l) {
            const float *Wl = Wh + (l - 1) * H * H;
            const float *hl = Hs + ((l - 1) * kChunk + t) * kHP;
#pragma unroll
            for (int c = 0; c < H; ++c) {
                float g = 0.f;
#pragma unroll
                for (int k = 0; k < H; ++k) g = fmaf(Wl[k * H + c], d[k], g);
                hp[c] = g * (1.f - hl[c] * hl[c]);
            }
#pragma unroll
            for (int c = 0; c < H; ++c) {
                d[c] = hp[c];
                Ds[((l - 1) * kChunk + t) * kHP + c] = d[c];
            }
        }
        for (int q = 0; q < 4; ++q) DO[t * 4 + q] = dO[q];
        __syncthreads();
        // parameter gradients summed over the chunk: layer l's weights pair its deltas
        // with the previous layer's activations (the inputs for l = 0)
        for (int e = t; e < P; e += kChunk) {
            float g = 0.f;
            int r = e;
            if (r < H * nin) {
                const int k = r / nin, c = r % nin;
                for (int m = 0; m < kChunk; ++m) g = fmaf(Ds[m * kHP + k], Xs[m * nin1 + c], g);
            } else if ((r -= H * nin) < H) {
                for (int m = 0; m < kChunk; ++m) g += Ds[m * kHP + r];
            } else {
                r -= H;
                bool done = false;
                for (int l = 1; l < depth && !done; ++l) {
                    const float *Dl = Ds + l * kChunk * kHP, *Hp = Hs + (l - 1) * kChunk * kHP;
                    if (r < H * H) {
                        const int k = r / H, c = r % H;
                        for (int m = 0; m < kChunk; ++m) g = fmaf(Dl[m * kHP + k], Hp[m * kHP + c], g);
                        done = true;
                    } else if ((r -= H * H) < H) {
                        for (int m = 0; m < kChunk; ++m) g += Dl[m * kHP + r];
                        done = true;
                    } else {
                        r -= H;
                    }
                }
                if (!done) {
                    const float *Hl = Hs + (depth - 1) * kChunk * kHP;
                    if (r < 4 * H) {
                        const int q = r / H, c = r % H;
                        for (int m = 0; m < kChunk; ++m) g = fmaf(DO[m * 4 + q], Hl[m * kHP + c], g);
                    } else {
                        r -= 4 * H;
                        for (int m = 0; m < kChunk; ++m) g += DO[m * 4 + r];
                    }
                }
            }
            acc[e] += g;
        }
        __syncthreads();
    }
    for (int e = t; e < P; e += kChunk)
        if (acc[e] != 0.f) atomicAdd(&grad[e], acc[e]);
    lsum[t] = my_loss;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int k = 0; k < kChunk; ++k) s += lsum[k];
        atomicAdd(loss, s);
    }
}

// Position of parameter e of the packed vector in the packed BF16 weight buffer; -1 for
// biases.  *fan receives fan_in + fan_out of the weight's layer.
__device__ __forceinline__ int64_t weight_slot(int64_t e, int nin, int depth, int *fan)
{
    int64_t o = 0, w = 0;   // start of the layer in the parameters / in the BF16 buffer
    *fan = 0;
    if (e < o + (int64_t)H * nin) {
        *fan = nin + H;
        return w + (e - o);
    }
    o += (int64_t)H * nin + H;
    w += (int64_t)H * nin;
    if (e < o) return -1;   // b1
    for (int l = 1; l < depth; ++l) {
        if (e < o + H * H) {
            *fan = 2 * H;
            return w + (e - o);
        }
        o += H * H + H;
        w += H * H;
        if (e < o) return -1;
    }
    if (e < o + 4 * H) {
        *fan = H + 4;
        return w + (e - o);
    }
    return -1;              // b3
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float scale,
                            float *__restrict__ m, float *__restrict__ v, int64_t P, int nin,
                            int depth, float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *__restrict__ wb)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    const float gr = g[e] * scale;
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float np = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = np;
    int fan = 0;
    const int64_t w = weight_slot(e, nin, depth, &fan);
    if (w >= 0) wb[w] = __float2bfloat16_rn(np);
}

// Glorot-uniform weights (U(-a, a), a = sqrt(6 / (fan_in + fan_out))) from one Philox draw
// per parameter (counter = its index, key = the seed), zero biases; the BF16 copy beside.
__global__ void init_kernel(float *__restrict__ p, int64_t P, int nin, int depth, uint32_t k0,
                            uint32_t k1, __nv_bfloat16 *__restrict__ wb)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    int fan = 0;
    const int64_t w = weight_slot(e, nin, depth, &fan);
    float v = 0.f;
    if (w >= 0) {
        const U4 r = philox4x32_10(U4{(uint32_t)e, (uint32_t)(e >> 32), 0x6D6C7069u, 0u}, k0, k1);
        const float a = sqrtf(6.f / (float)fan);
        v = a * (2.f * u01(r.x) - 1.f);
    }
    p[e] = v;
    if (w >= 0 && wb) wb[w] = __float2bfloat16_rn(v);
}

__global__ void bf16_kernel(const float *__restrict__ p, int64_t P, int nin, int depth,
                            __nv_bfloat16 *__restrict__ wb)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    int fan = 0;
    const int64_t w = weight_slot(e, nin, depth, &fan);
    if (w >= 0) wb[w] = __float2bfloat16_rn(p[e]);
}

}  // namespace
}  // namespace asd

using namespace asd;

extern "C" {

int64_t asd_mlp_param_count(int n_in, int depth)
{
    return shape_ok(n_in, depth) ? n_params(n_in, depth) : 0;
}
int64_t asd_mlp_param_count_bf16(int n_in, int depth)
{
    return shape_ok(n_in, depth) ? n_weights(n_in, depth) : 0;
}

int asd_mlp_gather(const asd_system *sys, int n_samples, const float *spins, float *x, float *y,
                   void *stream)
{
    ASD_CHECK_ARG(sys && spins && x && y, "null argument");
    ASD_CHECK_ARG(sys->n_sites >= 1 && sys->z >= 1 && sys->z <= kMlpMaxIn / 3 && sys->nbr,
                  "bad system (z must be 1..8)");
    ASD_CHECK_ARG(n_samples >= 1, "bad n_samples");
    const int64_t n = sys->n_sites * n_samples;
    gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        sys->n_sites, n_samples, sys->z, sys->nbr, spins, x, y);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

int asd_mlp_loss_grad(const asd_mlp *net, int64_t n, const float *x, const float *y, float *grad,
                      double *loss, void *stream)
{
    ASD_CHECK_ARG(net && x && y && grad && loss, "null argument");
    const int depth = mlp_depth(*net);
    ASD_CHECK_ARG(net->n_hidden == kMlpHidden && shape_ok(net->n_in, depth),
                  "network shape must be [n_in <= 24 -> 64 (x2 or x3) -> 4]");
    ASD_CHECK_ARG(net->W1 && net->W2 && net->W3 && net->b1 && net->b2 && net->b3, "null weights");
    ASD_CHECK_ARG(depth == 2 || (net->Wm && net->bm), "null weights of the third layer");
    ASD_CHECK_ARG(n >= 0, "bad n");
    if (n == 0) return ASD_OK;
    const int nin = net->n_in;
    const size_t smem =
        sizeof(float) * ((size_t)H * nin + (size_t)(depth - 1) * H * H + 4 * H +
                         kChunk * (nin + 1) + 2 * (size_t)depth * kChunk * kHP + kChunk * 4 +
                         n_params(nin, depth));
    auto k = loss_grad_kernel;
    ASD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    ASD_CUDA_TRY(cudaGetDevice(&dev));
    ASD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // as many resident blocks per SM as shared memory allows (the kernel is latency-bound:
    // two blocks of a two-layer network fit, one of a three-layer network)
    int smem_sm = 0;
    ASD_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    int per_sm = smem_sm / (int)(smem + 1024);
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    int64_t chunks = (n + kChunk - 1) / kChunk;
    int64_t blocks = chunks < (int64_t)sms * per_sm ? chunks : (int64_t)sms * per_sm;
    k<<<(unsigned)blocks, kChunk, smem, (cudaStream_t)stream>>>(mlp_view(*net), n, x, y, grad, loss);
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

int asd_mlp_adam_step(float *params, const float *grad, float grad_scale, float *m, float *v,
                      int n_in, int depth, float lr, float beta1, float beta2, float eps,
                      int step, uint16_t *w_bf16, void *stream)
{
    ASD_CHECK_ARG(params && grad && m && v && w_bf16, "null argument");
    ASD_CHECK_ARG(shape_ok(n_in, depth) && step >= 1, "bad n_in, depth or step");
    const int64_t P = n_params(n_in, depth);
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        params, grad, grad_scale, m, v, P, n_in, depth, lr, beta1, beta2, eps, c1, c2,
        reinterpret_cast<__nv_bfloat16 *>(w_bf16));
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

int asd_mlp_init(float *params, int n_in, int depth, uint64_t seed, uint16_t *w_bf16,
                 void *stream)
{
    ASD_CHECK_ARG(params, "null argument");
    ASD_CHECK_ARG(shape_ok(n_in, depth), "bad n_in (3..24) or depth (2, 3)");
    const int64_t P = n_params(n_in, depth);
    init_kernel<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        params, P, n_in, depth, (uint32_t)seed, (uint32_t)(seed >> 32),
        reinterpret_cast<__nv_bfloat16 *>(w_bf16));
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

int asd_mlp_weights_bf16(const float *params, int n_in, int depth, uint16_t *w_bf16,
                         void *stream)
{
    ASD_CHECK_ARG(params && w_bf16, "null argument");
    ASD_CHECK_ARG(shape_ok(n_in, depth), "bad n_in (3..24) or depth (2, 3)");
    const int64_t P = n_params(n_in, depth);
    bf16_kernel<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        params, P, n_in, depth, reinterpret_cast<__nv_bfloat16 *>(w_bf16));
    ASD_CUDA_TRY(cudaGetLastError());
    return ASD_OK;
}

}  // extern "C"
