// kc_mlp.cu -- the learned node scorer: a 12 -> 64 -> 64 -> 2 ReLU perceptron
// with bfloat16 weight matrices and float32 biases, activations and
// accumulation.  Output r is the predicted cost (log2 of the work in the
// subtree / 40) of branching a node with rule r.  Inference (one warp per node), training (a fused forward +
// backward kernel over chunks of 32 samples staged in shared memory, gradient
// sums merged with atomics, then Adam) -- all hand-written.
//
// Loss per sample: m0 (y0 - t0)^2 / 2 + m1 (y1 - t1)^2 / 2, averaged over the
// batch.  Parameter vector: [W1 64x12, b1 64, W2 64x64, b2 64,
// W3 2x64, b3 2] (row major), 5122 floats.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "kc_internal.cuh"

namespace kc {
namespace {

constexpr int NIN = 12, NH = 64, NOUT = 2;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NOUT * NH, NPARAM = OB3 + NOUT;
constexpr int NW_BF = NH * NIN + NH * NH + NOUT * NH;   // bf16 matrix entries
constexpr int CHUNK = 32;                               // samples per CTA step in training

struct Weights {
    const __nv_bfloat16 *w1, *w2, *w3;   // bf16 matrices
    const float *b1, *b2, *b3;           // float biases (inside the parameter vector)
};

__device__ __forceinline__ float bf(const __nv_bfloat16 *p, int i) { return __bfloat162float(p[i]); }

// Forward pass of one sample by one warp: lane holds hidden units lane and
// lane + 32 of each layer.  Returns y (valid in every lane).
__device__ __forceinline__ void warp_forward(const Weights &W, const float *x, float &z1a, float &z1b, float &z2a,
                                             float &z2b, float &y0, float &y1)
{
    const int lane = threadIdx.x & 31;
    z1a = W.b1[lane];
    z1b = W.b1[lane + 32];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
        z1a = fmaf(bf(W.w1, lane * NIN + i), x[i], z1a);
        z1b = fmaf(bf(W.w1, (lane + 32) * NIN + i), x[i], z1b);
    }
    const float h1a = fmaxf(z1a, 0.f), h1b = fmaxf(z1b, 0.f);
    z2a = W.b2[lane];
    z2b = W.b2[lane + 32];
#pragma unroll 8
    for (int i = 0; i < NH; ++i) {
        const float hi = __shfl_sync(0xffffffffu, i < 32 ? h1a : h1b, i & 31);
        z2a = fmaf(bf(W.w2, lane * NH + i), hi, z2a);
        z2b = fmaf(bf(W.w2, (lane + 32) * NH + i), hi, z2b);
    }
    const float h2a = fmaxf(z2a, 0.f), h2b = fmaxf(z2b, 0.f);
    float p0 = fmaf(bf(W.w3, lane), h2a, bf(W.w3, lane + 32) * h2b);
    float p1 = fmaf(bf(W.w3, NH + lane), h2a, bf(W.w3, NH + lane + 32) * h2b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, o);
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    }
    y0 = p0 + W.b3[0];
    y1 = p1 + W.b3[1];
}

__global__ void mlp_forward_kernel(Weights W, const float *__restrict__ feats, int B, float *__restrict__ out)
{
    const int warps = blockDim.x / 32;
    for (int b = blockIdx.x * warps + (threadIdx.x >> 5); b < B; b += gridDim.x * warps) {
        float x[NIN];
#pragma unroll
        for (int i = 0; i < NIN; ++i) x[i] = feats[(size_t)b * NIN + i];
        float z1a, z1b, z2a, z2b, y0, y1;
        warp_forward(W, x, z1a, z1b, z2a, z2b, y0, y1);
        if ((threadIdx.x & 31) == 0) {
            out[(size_t)b * NOUT] = y0;
            out[(size_t)b * NOUT + 1] = y1;
        }
    }
}


// Gradient of the mean loss over the n samples idx[0..n) (idx NULL: 0..n-1),
// added into grad[NPARAM]; the loss added into *loss.
__global__ void __launch_bounds__(256)
mlp_grad_kernel(Weights W, const float *__restrict__ feats, const float *__restrict__ targets,
                const float *__restrict__ masks, const int *__restrict__ idx, int n, float inv_n,
                float *__restrict__ grad, float *__restrict__ loss)
{
    extern __shared__ __align__(16) float sm[];
    float *xs = sm;                         // [CHUNK][NIN]
    float *h1s = xs + CHUNK * NIN;          // [CHUNK][NH]
    float *h2s = h1s + CHUNK * NH;
    float *dz1s = h2s + CHUNK * NH;
    float *dz2s = dz1s + CHUNK * NH;
    float *dys = dz2s + CHUNK * NH;         // [CHUNK][2]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = blockIdx.x * CHUNK; c0 < n; c0 += gridDim.x * CHUNK) {
        const int nb = min(CHUNK, n - c0);
        __syncthreads();
        for (int j = warp; j < CHUNK; j += 8) {
            if (j >= nb) {
                // padding rows contribute nothing
                h1s[j * NH + lane] = h1s[j * NH + lane + 32] = 0.f;
                h2s[j * NH + lane] = h2s[j * NH + lane + 32] = 0.f;
                dz1s[j * NH + lane] = dz1s[j * NH + lane + 32] = 0.f;
                dz2s[j * NH + lane] = dz2s[j * NH + lane + 32] = 0.f;
                if (lane < NIN) xs[j * NIN + lane] = 0.f;
                if (lane < 2) dys[j * 2 + lane] = 0.f;
                continue;
            }
            const int s = idx ? idx[c0 + j] : c0 + j;
            float x[NIN];
#pragma unroll
            for (int i = 0; i < NIN; ++i) x[i] = feats[(size_t)s * NIN + i];
            if (lane < NIN) xs[j * NIN + lane] = x[lane];
            float z1a, z1b, z2a, z2b, y0, y1;
            warp_forward(W, x, z1a, z1b, z2a, z2b, y0, y1);
            const float t0 = targets[(size_t)s * 2], t1 = targets[(size_t)s * 2 + 1];
            const float m0 = masks[(size_t)s * 2], m1 = masks[(size_t)s * 2 + 1];
            const float dy0 = m0 * (y0 - t0) * inv_n, dy1 = m1 * (y1 - t1) * inv_n;
            if (lane == 0) {
                dys[j * 2] = dy0;
                dys[j * 2 + 1] = dy1;
                const float l = m0 * 0.5f * (y0 - t0) * (y0 - t0) + m1 * 0.5f * (y1 - t1) * (y1 - t1);
                atomicAdd(loss, l * inv_n);
            }
            h1s[j * NH + lane] = fmaxf(z1a, 0.f);
            h1s[j * NH + lane + 32] = fmaxf(z1b, 0.f);
            h2s[j * NH + lane] = fmaxf(z2a, 0.f);
            h2s[j * NH + lane + 32] = fmaxf(z2b, 0.f);
            // back through layer 3 and the second ReLU
            const float dz2a = z2a > 0.f ? dy0 * bf(W.w3, lane) + dy1 * bf(W.w3, NH + lane) : 0.f;
            const float dz2b = z2b > 0.f ? dy0 * bf(W.w3, lane + 32) + dy1 * bf(W.w3, NH + lane + 32) : 0.f;
            dz2s[j * NH + lane] = dz2a;
            dz2s[j * NH + lane + 32] = dz2b;
            // back through layer 2 and the first ReLU: dh1[u] = sum_i dz2[i] W2[i][u]
            float dh1a = 0.f, dh1b = 0.f;
#pragma unroll 8
            for (int i = 0; i < NH; ++i) {
                const float di = __shfl_sync(0xffffffffu, i < 32 ? dz2a : dz2b, i & 31);
                dh1a = fmaf(di, bf(W.w2, i * NH + lane), dh1a);
                dh1b = fmaf(di, bf(W.w2, i * NH + lane + 32), dh1b);
            }
            dz1s[j * NH + lane] = z1a > 0.f ? dh1a : 0.f;
            dz1s[j * NH + lane + 32] = z1b > 0.f ? dh1b : 0.f;
        }
        __syncthreads();
        // weight and bias gradients of this chunk
        for (int e = threadIdx.x; e < NPARAM; e += blockDim.x) {
            float acc = 0.f;
            if (e < OB1) {
                const int u = e / NIN, i = e % NIN;
                for (int j = 0; j < nb; ++j) acc = fmaf(dz1s[j * NH + u], xs[j * NIN + i], acc);
            } else if (e < OW2) {
                const int u = e - OB1;
                for (int j = 0; j < nb; ++j) acc += dz1s[j * NH + u];
            } else if (e < OB2) {
                const int u = (e - OW2) / NH, i = (e - OW2) % NH;
                for (int j = 0; j < nb; ++j) acc = fmaf(dz2s[j * NH + u], h1s[j * NH + i], acc);
            } else if (e < OW3) {
                const int u = e - OB2;
                for (int j = 0; j < nb; ++j) acc += dz2s[j * NH + u];
            } else if (e < OB3) {
                const int o = (e - OW3) / NH, i = (e - OW3) % NH;
                for (int j = 0; j < nb; ++j) acc = fmaf(dys[j * 2 + o], h2s[j * NH + i], acc);
            } else {
                const int o = e - OB3;
                for (int j = 0; j < nb; ++j) acc += dys[j * 2 + o];
            }
            atomicAdd(&grad[e], acc);
        }
    }
}

__global__ void mlp_to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NW_BF; i += gridDim.x * blockDim.x) {
        int src;
        if (i < NH * NIN) src = OW1 + i;
        else if (i < NH * NIN + NH * NH) src = OW2 + (i - NH * NIN);
        else src = OW3 + (i - NH * NIN - NH * NH);
        w[i] = __float2bfloat16_rn(p[src]);
    }
}

// Adam (Kingma & Ba): bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void mlp_adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                                const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1,
                                float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// splitmix64 (Steele, Lea, Flood 2014): the permutation stream of training.
uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace kc

struct kc_mlp {
    int dev = 0;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *loss = nullptr;
    __nv_bfloat16 *w = nullptr;
    kc::DevBuf data;   // staged training data
    int64_t t = 0;     // Adam steps taken
    std::string err;
};

namespace kc {
namespace {

kc_status mset(kc_mlp *m, kc_status st, const char *msg)
{
    m->err = msg;
    return st;
}

#define KC_MLP_CUDA(m, call)                                                               \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (m)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return KC_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

Weights weights_of(const kc_mlp *m)
{
    Weights W;
    W.w1 = m->w;
    W.w2 = m->w + NH * NIN;
    W.w3 = m->w + NH * NIN + NH * NH;
    W.b1 = m->p + OB1;
    W.b2 = m->p + OB2;
    W.b3 = m->p + OB3;
    return W;
}

kc_status refresh_bf16(kc_mlp *m)
{
    mlp_to_bf16_kernel<<<(NW_BF + 255) / 256, 256, 0, m->stream>>>(m->p, m->w);
    KC_MLP_CUDA(m, cudaGetLastError());
    return KC_OK;
}

size_t grad_smem() { return ((size_t)CHUNK * NIN + 4 * (size_t)CHUNK * NH + 2 * CHUNK) * sizeof(float); }

kc_status launch_grad(kc_mlp *m, const float *feats, const float *targets, const float *masks, const int *idx, int n)
{
    static bool attr = false;
    const size_t smem = grad_smem();
    if (!attr) {
        KC_MLP_CUDA(m, cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const int grid = std::max(1, std::min(1024, (n + CHUNK - 1) / CHUNK));
    mlp_grad_kernel<<<grid, 256, smem, m->stream>>>(weights_of(m), feats, targets, masks, idx, n, 1.f / (float)n,
                                                    m->g, m->loss);
    KC_MLP_CUDA(m, cudaGetLastError());
    return KC_OK;
}

}  // namespace

// Used by the solver: scores B nodes (device features [B][12] -> device [B][2]).
kc_status mlp_forward_device(kc_mlp *m, const float *feats, int B, float *out, cudaStream_t stream)
{
    if (B <= 0) return KC_OK;
    mlp_forward_kernel<<<std::max(1, std::min(1024, (B + 7) / 8)), 256, 0, stream>>>(weights_of(m), feats, B, out);
    KC_MLP_CUDA(m, cudaGetLastError());
    return KC_OK;
}

}  // namespace kc

using namespace kc;

extern "C" {

kc_status kc_mlp_create(const float *params, void *stream, kc_mlp **out)
{
    if (!out || !params) return KC_EINVAL;
    *out = nullptr;
    kc_mlp *m = new (std::nothrow) kc_mlp;
    if (!m) return KC_ENOMEM;
    m->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&m->dev);
    void *buf = nullptr;
    const size_t fbytes = (size_t)(4 * NPARAM + 16) * sizeof(float);
    if (cudaMalloc(&buf, fbytes + (size_t)NW_BF * sizeof(__nv_bfloat16) + 256) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return KC_ENOMEM;
    }
    m->p = static_cast<float *>(buf);
    m->m = m->p + NPARAM;
    m->v = m->m + NPARAM;
    m->g = m->v + NPARAM;
    m->loss = m->g + NPARAM;
    m->w = reinterpret_cast<__nv_bfloat16 *>(static_cast<char *>(buf) + ((fbytes + 255) & ~(size_t)255));
    const bool dev = is_device_ptr(params);
    if (cudaMemcpyAsync(m->p, params, NPARAM * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->m, 0, 2 * NPARAM * sizeof(float), m->stream) != cudaSuccess ||
        refresh_bf16(m) != KC_OK || cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        delete m;
        return KC_ECUDA;
    }
    *out = m;
    return KC_OK;
}

void kc_mlp_destroy(kc_mlp *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->p);
    if (m->data.p) cudaFree(m->data.p);
    delete m;
}

const char *kc_mlp_last_error(const kc_mlp *m) { return m ? m->err.c_str() : "null scorer"; }

kc_status kc_mlp_get_params(kc_mlp *m, float *params)
{
    if (!m || !params) return KC_EINVAL;
    KC_MLP_CUDA(m, cudaMemcpyAsync(params, m->p, NPARAM * sizeof(float), cudaMemcpyDefault, m->stream));
    KC_MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return KC_OK;
}

kc_status kc_mlp_forward(kc_mlp *m, const float *feats, int32_t B, float *out)
{
    if (!m || B < 0) return KC_EINVAL;
    if (B == 0) return KC_OK;
    if (!feats || !out) return mset(m, KC_EINVAL, "kc_mlp_forward: NULL argument");
    const bool fdev = is_device_ptr(feats), odev = is_device_ptr(out);
    const float *f = feats;
    float *o = out;
    if (!fdev || !odev) {
        const size_t need = (size_t)B * (NIN + NOUT) * sizeof(float) + 256;
        if (m->data.bytes < need) {
            if (m->data.p) cudaFree(m->data.p);
            m->data.p = nullptr;
            m->data.bytes = 0;
            KC_MLP_CUDA(m, cudaMalloc(&m->data.p, need));
            m->data.bytes = need;
        }
        float *d = static_cast<float *>(m->data.p);
        if (!fdev) {
            KC_MLP_CUDA(m, cudaMemcpyAsync(d, feats, (size_t)B * NIN * sizeof(float), cudaMemcpyHostToDevice, m->stream));
            f = d;
        }
        if (!odev) o = d + (size_t)B * NIN;
    }
    KC_TRY(mlp_forward_device(m, f, B, o, m->stream));
    if (!odev) {
        KC_MLP_CUDA(m, cudaMemcpyAsync(out, o, (size_t)B * NOUT * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        KC_MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    return KC_OK;
}

// Stages (feats, targets, masks) of n samples in device memory.
static kc_status stage_data(kc_mlp *m, const float *feats, const float *targets, const float *masks, int n,
                            const float **f, const float **t, const float **k, int **perm)
{
    const size_t nf = (size_t)n * NIN, n2 = (size_t)n * 2;
    const size_t need = (nf + 2 * n2) * sizeof(float) + (size_t)n * sizeof(int) + 1024;
    if (m->data.bytes < need) {
        if (m->data.p) cudaFree(m->data.p);
        m->data.p = nullptr;
        m->data.bytes = 0;
        KC_MLP_CUDA(m, cudaMalloc(&m->data.p, need));
        m->data.bytes = need;
    }
    float *d = static_cast<float *>(m->data.p);
    KC_MLP_CUDA(m, cudaMemcpyAsync(d, feats, nf * sizeof(float), cudaMemcpyDefault, m->stream));
    KC_MLP_CUDA(m, cudaMemcpyAsync(d + nf, targets, n2 * sizeof(float), cudaMemcpyDefault, m->stream));
    KC_MLP_CUDA(m, cudaMemcpyAsync(d + nf + n2, masks, n2 * sizeof(float), cudaMemcpyDefault, m->stream));
    *f = d;
    *t = d + nf;
    *k = d + nf + n2;
    *perm = reinterpret_cast<int *>(d + nf + 2 * n2);
    return KC_OK;
}

kc_status kc_mlp_grad(kc_mlp *m, const float *feats, const float *targets, const float *masks, int32_t n,
                      float *loss_out, float *grad_out)
{
    if (!m || n <= 0 || !feats || !targets || !masks) return KC_EINVAL;
    const float *f, *t, *k;
    int *perm;
    KC_TRY(stage_data(m, feats, targets, masks, n, &f, &t, &k, &perm));
    KC_MLP_CUDA(m, cudaMemsetAsync(m->g, 0, (NPARAM + 16) * sizeof(float), m->stream));
    KC_TRY(launch_grad(m, f, t, k, nullptr, n));
    if (grad_out)
        KC_MLP_CUDA(m, cudaMemcpyAsync(grad_out, m->g, NPARAM * sizeof(float), cudaMemcpyDefault, m->stream));
    if (loss_out) KC_MLP_CUDA(m, cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDefault, m->stream));
    KC_MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return KC_OK;
}

kc_status kc_mlp_train(kc_mlp *m, const float *feats, const float *targets, const float *masks, int32_t n,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float *loss_out)
{
    if (!m || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.f)) return KC_EINVAL;
    const float *f, *t, *k;
    int *perm_dev;
    KC_TRY(stage_data(m, feats, targets, masks, n, &f, &t, &k, &perm_dev));
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    uint64_t s = seed;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = n - 1; i > 0; --i) {   // Fisher-Yates with splitmix64
            const int j = (int)(splitmix64(s) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        KC_MLP_CUDA(m, cudaMemcpyAsync(perm_dev, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice,
                                       m->stream));
        KC_MLP_CUDA(m, cudaStreamSynchronize(m->stream));   // perm is reused next epoch
        for (int s0 = 0; s0 < n; s0 += batch) {
            const int nb = std::min(batch, n - s0);
            KC_MLP_CUDA(m, cudaMemsetAsync(m->g, 0, (NPARAM + 16) * sizeof(float), m->stream));
            KC_TRY(launch_grad(m, f, t, k, perm_dev + s0, nb));
            ++m->t;
            const float c1 = (float)(1.0 - std::pow(0.9, (double)m->t));
            const float c2 = (float)(1.0 - std::pow(0.999, (double)m->t));
            mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->p, m->m, m->v, m->g, lr, b1, b2, eps, c1, c2);
            KC_MLP_CUDA(m, cudaGetLastError());
            KC_TRY(refresh_bf16(m));
        }
    }
    if (loss_out) {
        KC_MLP_CUDA(m, cudaMemsetAsync(m->g, 0, (NPARAM + 16) * sizeof(float), m->stream));
        KC_TRY(launch_grad(m, f, t, k, nullptr, n));
        KC_MLP_CUDA(m, cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDefault, m->stream));
    }
    KC_MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return KC_OK;
}

}  // extern "C"
