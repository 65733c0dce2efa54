// kc_data.cu -- dataset ingest (attribute-major padded copy), the root region
// M0 of Section 2.1 (per-attribute min / max) with the non-finite check, and
// stream compaction of the surviving samples after sample reduction.
#include <cuda_runtime.h>

#include <algorithm>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

namespace {

// Row-major [N][D] -> attribute-major [D][ld], zero padding in [N, ld).
template <typename T>
__global__ void transpose_in(const T *__restrict__ src, int64_t N, int D, int64_t ld, T *__restrict__ dst)
{
    const int64_t total = (int64_t)D * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / ld);
        const int64_t s = i - (int64_t)a * ld;
        dst[i] = s < N ? src[s * D + a] : T(0);
    }
}

// Rows s0 .. s0 + n of a row-major dataset, staged at src as [n][D] ->
// attribute-major dst[a * ld + s0 + i] (one chunk of a host upload).
template <typename T>
__global__ void transpose_rows(const T *__restrict__ src, int64_t s0, int64_t n, int D, int64_t ld,
                               T *__restrict__ dst)
{
    const int64_t total = (int64_t)D * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / n);
        const int64_t s = i - (int64_t)a * n;
        dst[(size_t)a * ld + s0 + s] = src[s * D + a];
    }
}

// Per-attribute min / max with order-preserving integer atomics (exact), and
// a flag for NaN / Inf.
template <typename T>
__global__ void root_box_kernel(const T *__restrict__ X, int64_t ld, int64_t N, int D,
                                unsigned long long *__restrict__ omin, unsigned long long *__restrict__ omax,
                                int *__restrict__ nonfinite)
{
    __shared__ unsigned long long smin[kMaxD], smax[kMaxD];
    __shared__ int sbad;
    for (int a = threadIdx.x; a < D; a += blockDim.x) { smin[a] = ~0ull; smax[a] = 0ull; }
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    for (int a = 0; a < D; ++a) {
        unsigned long long mn = ~0ull, mx = 0ull;
        int bad = 0;
        for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N;
             s += (int64_t)gridDim.x * blockDim.x) {
            const T v = X[(size_t)a * ld + s];
            if (!isfinite((double)v)) bad = 1;
            unsigned long long o;
            if constexpr (sizeof(T) == 4) o = ord_f32((float)v);
            else o = ord_f64((double)v);
            mn = o < mn ? o : mn;
            mx = o > mx ? o : mx;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long a2 = __shfl_xor_sync(0xffffffffu, mn, off);
            const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, mx, off);
            mn = a2 < mn ? a2 : mn;
            mx = b2 > mx ? b2 : mx;
        }
        bad = __any_sync(0xffffffffu, bad);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&smin[a], mn);
            atomicMax(&smax[a], mx);
            if (bad) sbad = 1;
        }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < D; a += blockDim.x) {
        atomicMin(&omin[a], smin[a]);
        atomicMax(&omax[a], smax[a]);
    }
    if (threadIdx.x == 0 && sbad) atomicOr(nonfinite, 1);
}

__global__ void init_minmax(unsigned long long *omin, unsigned long long *omax, int D, int *flag)
{
    for (int a = threadIdx.x; a < D; a += blockDim.x) { omin[a] = ~0ull; omax[a] = 0ull; }
    if (threadIdx.x == 0 && flag) *flag = 0;
}

template <typename T>
__global__ void decode_minmax(const unsigned long long *omin, const unsigned long long *omax, int D, T *lo, T *hi)
{
    for (int a = threadIdx.x; a < D; a += blockDim.x) {
        if constexpr (sizeof(T) == 4) {
            lo[a] = unord_f32((uint32_t)omin[a]);
            hi[a] = unord_f32((uint32_t)omax[a]);
        } else {
            lo[a] = unord_f64(omin[a]);
            hi[a] = unord_f64(omax[a]);
        }
    }
}

}  // namespace

kc_status launch_ingest(kc_ctx *c, const void *src_dev, kc_layout layout, int64_t N, int D)
{
    // src_dev is device memory holding the caller's layout.
    if (layout == KC_COL_MAJOR) {
        KC_CUDA(c, cudaMemcpy2DAsync(c->X, c->ldx * c->esize, src_dev, N * c->esize, N * c->esize, D,
                                     cudaMemcpyDeviceToDevice, c->stream));
        if (c->ldx > N)
            KC_CUDA(c, cudaMemset2DAsync(static_cast<char *>(c->X) + N * c->esize, c->ldx * c->esize, 0,
                                         (c->ldx - N) * c->esize, D, c->stream));
        return KC_OK;
    }
    const int grid = c->num_sms * 8;
    if (c->dt == KC_F32)
        transpose_in<float><<<grid, 256, 0, c->stream>>>(static_cast<const float *>(src_dev), N, D, c->ldx,
                                                         static_cast<float *>(c->X));
    else
        transpose_in<double><<<grid, 256, 0, c->stream>>>(static_cast<const double *>(src_dev), N, D, c->ldx,
                                                          static_cast<double *>(c->X));
    return after_launch(c, "ingest transpose");
}

kc_status launch_ingest_rows(kc_ctx *c, const void *chunk_dev, int64_t s0, int64_t n)
{
    if (n <= 0) return KC_OK;
    const int grid = (int)std::min<int64_t>((int64_t)c->num_sms * 8, ((int64_t)c->D * n + 255) / 256);
    if (c->dt == KC_F32)
        transpose_rows<float><<<grid, 256, 0, c->stream>>>(static_cast<const float *>(chunk_dev), s0, n, c->D, c->ldx,
                                                           static_cast<float *>(c->X));
    else
        transpose_rows<double><<<grid, 256, 0, c->stream>>>(static_cast<const double *>(chunk_dev), s0, n, c->D,
                                                            c->ldx, static_cast<double *>(c->X));
    return after_launch(c, "ingest transpose (chunk)");
}

kc_status launch_root_box(kc_ctx *c, void *lo, void *hi, int *nonfinite_dev)
{
    const int D = c->D;
    KC_TRY(ensure(c, c->part, (size_t)2 * kMaxD * 8 + 16));
    unsigned long long *omin = static_cast<unsigned long long *>(c->part.p);
    unsigned long long *omax = omin + kMaxD;
    init_minmax<<<1, 64, 0, c->stream>>>(omin, omax, D, nonfinite_dev);
    KC_TRY(after_launch(c, "root box init"));
    const int grid = c->num_sms * 4;
    if (c->dt == KC_F32)
        root_box_kernel<float><<<grid, 256, 0, c->stream>>>(static_cast<const float *>(c->X), c->ldx, c->N, D,
                                                            omin, omax, nonfinite_dev);
    else
        root_box_kernel<double><<<grid, 256, 0, c->stream>>>(static_cast<const double *>(c->X), c->ldx, c->N,
                                                             D, omin, omax, nonfinite_dev);
    KC_TRY(after_launch(c, "root box"));
    if (c->dt == KC_F32)
        decode_minmax<float><<<1, 64, 0, c->stream>>>(omin, omax, D, static_cast<float *>(lo),
                                                      static_cast<float *>(hi));
    else
        decode_minmax<double><<<1, 64, 0, c->stream>>>(omin, omax, D, static_cast<double *>(lo),
                                                       static_cast<double *>(hi));
    return after_launch(c, "root box decode");
}

// ------------------------------------------------------------ compaction
// Stable stream compaction of the samples a mask keeps: per-block counts,
// one exclusive scan, then a scatter that preserves sample order (so
// positions stay ordered like sample indices).

namespace {

constexpr int kCompPer = 16;                       // samples per thread
constexpr int kCompBlock = 256 * kCompPer;         // samples per block

__global__ void comp_count(const uint8_t *__restrict__ mask, int64_t n, unsigned *__restrict__ counts)
{
    const int64_t b0 = (int64_t)blockIdx.x * kCompBlock;
    unsigned c = 0;
    for (int i = threadIdx.x; i < kCompBlock; i += 256) {
        const int64_t s = b0 + i;
        if (s < n && mask[s]) ++c;
    }
    __shared__ unsigned red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < 8; ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}

// Exclusive scan of nb counts by one block of 1024 threads; total -> *total.
__global__ void comp_scan(unsigned *__restrict__ counts, int64_t nb, unsigned long long *__restrict__ total)
{
    __shared__ unsigned long long part[1024];
    const int64_t per = (nb + 1023) / 1024;
    const int64_t s0 = threadIdx.x * per, s1 = (s0 + per < nb) ? s0 + per : nb;
    unsigned long long acc = 0;
    for (int64_t i = s0; i < s1; ++i) acc += counts[i];
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < 1024; ++i) {
            const unsigned long long v = part[i];
            part[i] = run;
            run += v;
        }
        *total = run;
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (int64_t i = s0; i < s1; ++i) {
        const unsigned v = counts[i];
        counts[i] = (unsigned)run;
        run += v;
    }
}

template <typename T>
__global__ void comp_scatter(const T *__restrict__ X, int64_t ld, int64_t n, int D, const uint32_t *__restrict__ ids,
                             const uint8_t *__restrict__ mask, const unsigned *__restrict__ offs, T *__restrict__ Xo,
                             int64_t ldo, uint32_t *__restrict__ ido)
{
    __shared__ unsigned wsum[8];
    const int64_t b0 = (int64_t)blockIdx.x * kCompBlock;
    unsigned base = offs[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = 0; r < kCompPer; ++r) {
        const int64_t s = b0 + (int64_t)r * 256 + threadIdx.x;
        const bool keep = s < n && mask[s];
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        unsigned before = 0, tot = 0;
        for (int q = 0; q < 8; ++q) {
            if (q < w) before += wsum[q];
            tot += wsum[q];
        }
        if (keep) {
            const unsigned p = base + before + __popc(bal & ((1u << lane) - 1u));
            for (int a = 0; a < D; ++a) Xo[(size_t)a * ldo + p] = X[(size_t)a * ld + s];
            ido[p] = ids ? ids[s] : (uint32_t)s;
        }
        base += tot;
        __syncthreads();
    }
}

}  // namespace

kc_status launch_compact(kc_ctx *c, const View &v, const uint8_t *mask, void *Xo, int64_t ldo, uint32_t *ido,
                         unsigned *scratch_counts, unsigned long long *total_dev)
{
    const int64_t nb = (v.n + kCompBlock - 1) / kCompBlock;
    if (nb == 0) {
        KC_CUDA(c, cudaMemsetAsync(total_dev, 0, 8, c->stream));
        return KC_OK;
    }
    comp_count<<<(unsigned)nb, 256, 0, c->stream>>>(mask, v.n, scratch_counts);
    KC_TRY(after_launch(c, "compaction count"));
    comp_scan<<<1, 1024, 0, c->stream>>>(scratch_counts, nb, total_dev);
    KC_TRY(after_launch(c, "compaction scan"));
    if (c->dt == KC_F32)
        comp_scatter<float><<<(unsigned)nb, 256, 0, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, c->D, v.ids,
                                                                 mask, scratch_counts, static_cast<float *>(Xo), ldo, ido);
    else
        comp_scatter<double><<<(unsigned)nb, 256, 0, c->stream>>>(static_cast<const double *>(v.X), v.ld, v.n, c->D,
                                                                  v.ids, mask, scratch_counts, static_cast<double *>(Xo),
                                                                  ldo, ido);
    return after_launch(c, "compaction scatter");
}

int64_t compact_blocks(int64_t n) { return (n + kCompBlock - 1) / kCompBlock; }

}  // namespace kc
