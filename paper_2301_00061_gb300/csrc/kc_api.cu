// kc_api.cu -- the C ABI of include/kc.h: context lifetime, argument
// validation, host/device pointer staging, and the entry points that are a
// single kernel family (root box, lower bounds, upper bounds, FFT).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <new>

#include "kc_internal.cuh"

namespace kc {

namespace {
thread_local std::string g_create_err;
}

kc_status set_err(kc_ctx *c, kc_status st, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_err = buf;
    return st;
}

kc_status after_launch(kc_ctx *c, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(c, KC_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    ++c->launches;
    return KC_OK;
}

kc_status ensure(kc_ctx *c, DevBuf &b, size_t bytes)
{
    if (bytes <= b.bytes) return KC_OK;
    size_t nb = std::max(bytes, b.bytes + b.bytes / 2);
    nb = (nb + 4095) & ~(size_t)4095;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);   // implicitly waits for work using it
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return set_err(c, KC_ECUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return set_err(c, KC_ENOMEM, "cudaMalloc(%zu bytes): %s", nb, cudaGetErrorString(e));
    }
    b.bytes = nb;
    return KC_OK;
}

kc_status ensure_pinned(kc_ctx *c, size_t bytes)
{
    if (bytes <= c->pinned_bytes) return KC_OK;
    if (c->pinned) {
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaFreeHost(c->pinned);
        c->pinned = nullptr;
        c->pinned_bytes = 0;
    }
    size_t nb = (std::max(bytes, (size_t)1 << 16) + 4095) & ~(size_t)4095;
    if (cudaMallocHost(&c->pinned, nb) != cudaSuccess) {
        c->pinned = nullptr;
        cudaGetLastError();
        return set_err(c, KC_ENOMEM, "cudaMallocHost(%zu bytes) failed", nb);
    }
    c->pinned_bytes = nb;
    return KC_OK;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace kc

using namespace kc;

extern "C" {

const char *kc_create_error(void) { return g_create_err.c_str(); }

const char *kc_last_error(const kc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t kc_launch_count(const kc_ctx *ctx) { return ctx ? ctx->launches : 0; }

kc_status kc_set_stream(kc_ctx *ctx, void *stream)
{
    if (!ctx) return KC_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return KC_OK;
}

void kc_destroy(kc_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (DevBuf *b : {&ctx->part, &ctx->stage_in, &ctx->stage_out, &ctx->work})
        if (b->p) cudaFree(b->p);
    if (ctx->X) cudaFree(ctx->X);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
}

kc_status kc_create(const void *X, int64_t N, int32_t D, int32_t K, kc_dtype dt, kc_layout layout, void *stream,
                    kc_ctx **out)
{
    g_create_err.clear();
    if (!out) return set_err(nullptr, KC_EINVAL, "kc_create: out is NULL");
    *out = nullptr;
    if (!X) return set_err(nullptr, KC_EINVAL, "kc_create: X is NULL");
    if (dt != KC_F32 && dt != KC_F64) return set_err(nullptr, KC_EINVAL, "kc_create: bad dtype %d", (int)dt);
    if (layout != KC_ROW_MAJOR && layout != KC_COL_MAJOR)
        return set_err(nullptr, KC_EINVAL, "kc_create: bad layout %d", (int)layout);
    if (K < 1 || K > kMaxK) return set_err(nullptr, KC_EINVAL, "kc_create: K=%d outside [1, %d]", K, kMaxK);
    if (D < 1 || D > kMaxD) return set_err(nullptr, KC_EINVAL, "kc_create: D=%d outside [1, %d]", D, kMaxD);
    if (N < K || N > 4294967294ll)
        return set_err(nullptr, KC_EINVAL, "kc_create: N=%lld outside [K, 4294967294]", (long long)N);

    kc_ctx *c = new (std::nothrow) kc_ctx;
    if (!c) return set_err(nullptr, KC_ENOMEM, "kc_create: out of host memory");
    auto fail = [&](kc_status st) {
        g_create_err = c->err;
        kc_destroy(c);
        return st;
    };
    c->stream = static_cast<cudaStream_t>(stream);
    c->N = N;
    c->D = D;
    c->K = K;
    c->dt = dt;
    c->esize = dt == KC_F32 ? 4 : 8;
    const int64_t align = 256 / (int64_t)c->esize;
    c->ldx = (N + align - 1) / align * align;
    if (cudaGetDevice(&c->dev) != cudaSuccess) {
        set_err(c, KC_ECUDA, "kc_create: no CUDA device");
        return fail(KC_ECUDA);
    }
    int sms = 0, smem_optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, KC_ECUDA, "kc_create: cannot query the device");
        return fail(KC_ECUDA);
    }
    c->num_sms = sms;
    if (const char *e = getenv("KC_LB_ST")) c->lb_st = atoi(e);
    c->smem_optin = (size_t)smem_optin;
    const size_t xbytes = (size_t)D * c->ldx * c->esize;
    if (cudaMalloc(&c->X, xbytes) != cudaSuccess) {
        cudaGetLastError();
        c->X = nullptr;
        set_err(c, KC_ENOMEM, "kc_create: cannot allocate %zu bytes for the data", xbytes);
        return fail(KC_ENOMEM);
    }
    const size_t src_bytes = (size_t)N * D * c->esize;
    kc_status st = KC_OK;
    if (is_device_ptr(X)) {
        st = launch_ingest(c, X, layout, N, D);
    } else if (layout == KC_COL_MAJOR) {
        cudaError_t e = cudaMemcpy2DAsync(c->X, c->ldx * c->esize, X, N * c->esize, N * c->esize, D,
                                          cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && c->ldx > N)
            e = cudaMemset2DAsync(static_cast<char *>(c->X) + N * c->esize, c->ldx * c->esize, 0,
                                  (c->ldx - N) * c->esize, D, c->stream);
        if (e != cudaSuccess) st = set_err(c, KC_ECUDA, "kc_create: upload failed: %s", cudaGetErrorString(e));
    } else {
        // host rows: upload in chunks of at most 32 MiB through one staging
        // buffer, each transposed into place (stream order keeps the next
        // upload behind the previous transpose)
        const int64_t row_bytes = (int64_t)D * c->esize;
        const int64_t rows = std::min<int64_t>(N, std::max<int64_t>(1, ((int64_t)32 << 20) / row_bytes));
        st = ensure(c, c->work, (size_t)(rows * row_bytes));
        for (int64_t s0 = 0; st == KC_OK && s0 < N; s0 += rows) {
            const int64_t n = std::min(rows, N - s0);
            cudaError_t e = cudaMemcpyAsync(c->work.p, static_cast<const char *>(X) + s0 * row_bytes,
                                            (size_t)(n * row_bytes), cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) st = set_err(c, KC_ECUDA, "kc_create: upload failed: %s", cudaGetErrorString(e));
            else st = launch_ingest_rows(c, c->work.p, s0, n);
        }
        if (st == KC_OK && c->ldx > N) {
            cudaError_t e = cudaMemset2DAsync(static_cast<char *>(c->X) + N * c->esize, c->ldx * c->esize, 0,
                                              (c->ldx - N) * c->esize, D, c->stream);
            if (e != cudaSuccess) st = set_err(c, KC_ECUDA, "kc_create: padding failed: %s", cudaGetErrorString(e));
        }
    }
    if (st != KC_OK) return fail(st);
    // non-finite scan (with the root box, which is cheap)
    st = ensure(c, c->stage_out, 2 * (size_t)kMaxD * 8 + 256);
    if (st != KC_OK) return fail(st);
    char *so = static_cast<char *>(c->stage_out.p);
    int *flag_dev = reinterpret_cast<int *>(so + 2 * (size_t)kMaxD * 8);
    st = launch_root_box(c, so, so + (size_t)kMaxD * 8, flag_dev);
    if (st != KC_OK) return fail(st);
    int flag = 0;
    if (cudaMemcpyAsync(&flag, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        set_err(c, KC_ECUDA, "kc_create: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(KC_ECUDA);
    }
    if (flag) {
        set_err(c, KC_EINVAL, "kc_create: the data contain NaN or infinite values");
        return fail(KC_EINVAL);
    }
    if (src_bytes > ((size_t)64 << 20) && c->work.p) {   // release the upload staging buffer of large datasets
        cudaFree(c->work.p);
        c->work.p = nullptr;
        c->work.bytes = 0;
    }
    *out = c;
    return KC_OK;
}

kc_status kc_root_box(kc_ctx *c, void *lo, void *hi)
{
    if (!c) return KC_EINVAL;
    if (!lo || !hi) return set_err(c, KC_EINVAL, "kc_root_box: NULL output");
    const size_t bytes = (size_t)c->D * c->esize;
    Stager sg(c);
    int ilo = sg.add(lo, bytes, false), ihi = sg.add(hi, bytes, false);
    KC_TRY(sg.begin());
    KC_TRY(ensure(c, c->stage_out, 2 * (size_t)kMaxD * 8 + 256));
    int *flag = reinterpret_cast<int *>(static_cast<char *>(c->stage_out.p) + 2 * (size_t)kMaxD * 8);
    KC_TRY(launch_root_box(c, sg.dev(ilo), sg.dev(ihi), flag));
    return sg.finish();
}

kc_status kc_lower_bounds(kc_ctx *c, const void *lo, const void *hi, int32_t B, double *lb_out,
                          double *lb_raw_out, int64_t *argmax_out)
{
    if (!c) return KC_EINVAL;
    if (B < 0) return set_err(c, KC_EINVAL, "kc_lower_bounds: B=%d < 0", B);
    if (B == 0) return KC_OK;
    if (!lo || !hi || !lb_out) return set_err(c, KC_EINVAL, "kc_lower_bounds: NULL argument");
    const size_t box = (size_t)B * c->K * c->D * c->esize;
    Stager sg(c);
    int ilo = sg.add(lo, box, true), ihi = sg.add(hi, box, true);
    int ilb = sg.add(lb_out, (size_t)B * 8, false);
    int iraw = sg.add(lb_raw_out, (size_t)B * 8, false);
    int iarg = sg.add(argmax_out, (size_t)B * 8, false);
    KC_TRY(sg.begin());
    KC_TRY(launch_lower_bounds(c, sg.dev(ilo), sg.dev(ihi), B, static_cast<double *>(sg.dev(ilb)),
                               static_cast<double *>(sg.dev(iraw)), static_cast<int64_t *>(sg.dev(iarg))));
    return sg.finish();
}

kc_status kc_autotune(kc_ctx *c, const void *lo, const void *hi, int32_t B, int32_t *st_out, int32_t *chunk_out,
                      float *ms_out)
{
    if (!c) return KC_EINVAL;
    if (B <= 0 || !lo || !hi) return set_err(c, KC_EINVAL, "kc_autotune: empty node batch");
    const size_t box = (size_t)B * c->K * c->D * c->esize;
    Stager sg(c);
    const int ilo = sg.add(lo, box, true), ihi = sg.add(hi, box, true);
    KC_TRY(sg.begin());
    KC_TRY(ensure(c, c->stage_out, (size_t)B * 8 + 2 * (size_t)kMaxD * 8 + 512));
    int st = 0, ch = 0;
    float ms = 0.f;
    KC_TRY(autotune_lower_bounds(c, sg.dev(ilo), sg.dev(ihi), B,
                                 reinterpret_cast<double *>(static_cast<char *>(c->stage_out.p) + 2 * (size_t)kMaxD * 8 + 256),
                                 &st, &ch, &ms));
    if (st_out) *st_out = st;
    if (chunk_out) *chunk_out = ch;
    if (ms_out) *ms_out = ms;
    return KC_OK;
}

static kc_status check_centers(kc_ctx *c, const int64_t *centers, size_t count)
{
    std::vector<int64_t> h(count);
    const int64_t *p = centers;
    if (is_device_ptr(centers)) {
        KC_CUDA(c, cudaMemcpyAsync(h.data(), centers, count * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        p = h.data();
    }
    for (size_t i = 0; i < count; ++i)
        if (p[i] < 0 || p[i] >= c->N)
            return set_err(c, KC_EINVAL, "center index %lld outside [0, %lld)", (long long)p[i], (long long)c->N);
    return KC_OK;
}

kc_status kc_upper_bound(kc_ctx *c, const int64_t *centers, int32_t S, double *ub_out, int64_t *worst_out)
{
    if (!c) return KC_EINVAL;
    if (S < 0) return set_err(c, KC_EINVAL, "kc_upper_bound: S=%d < 0", S);
    if (S == 0) return KC_OK;
    if (!centers || !ub_out) return set_err(c, KC_EINVAL, "kc_upper_bound: NULL argument");
    KC_TRY(check_centers(c, centers, (size_t)S * c->K));
    Stager sg(c);
    int ic = sg.add(centers, (size_t)S * c->K * 8, true);
    int iu = sg.add(ub_out, (size_t)S * 8, false);
    int iw = sg.add(worst_out, (size_t)S * 8, false);
    KC_TRY(sg.begin());
    KC_TRY(launch_objective(c, full_view(c), static_cast<const int64_t *>(sg.dev(ic)), S, c->K,
                            __builtin_huge_val(), static_cast<double *>(sg.dev(iu)),
                            static_cast<int64_t *>(sg.dev(iw))));
    return sg.finish();
}

kc_status kc_fft(kc_ctx *c, int64_t start, int64_t *centers_out, double *obj_out)
{
    if (!c) return KC_EINVAL;
    if (!centers_out) return set_err(c, KC_EINVAL, "kc_fft: NULL argument");
    if (start < 0 || start >= c->N) return set_err(c, KC_EINVAL, "kc_fft: start %lld outside [0, N)", (long long)start);
    Stager sg(c);
    int ic = sg.add(centers_out, (size_t)c->K * 8, false);
    int io = sg.add(obj_out, 8, false);
    KC_TRY(sg.begin());
    int64_t *T = static_cast<int64_t *>(sg.dev(ic));
    KC_CUDA(c, cudaMemcpyAsync(T, &start, 8, cudaMemcpyHostToDevice, c->stream));
    KC_CUDA(c, cudaStreamSynchronize(c->stream));   // `start` lives on this stack frame
    KC_TRY(ensure(c, c->stage_out, 2 * (size_t)kMaxD * 8 + 256 + 64));
    double *scratch = reinterpret_cast<double *>(static_cast<char *>(c->stage_out.p) + 2 * (size_t)kMaxD * 8 + 256);
    // Algorithm 2: the t-th point is the sample farthest from the first t.
    for (int t = 1; t < c->K; ++t)
        KC_TRY(launch_objective(c, full_view(c), T, 1, t, __builtin_huge_val(), scratch, T + t));
    if (obj_out)
        KC_TRY(launch_objective(c, full_view(c), T, 1, c->K, __builtin_huge_val(), static_cast<double *>(sg.dev(io)),
                                nullptr));
    return sg.finish();
}

}  // extern "C"

// ------------------------------------------------------------------------
// Farthest first traversal from S starts at once, and lower bounds over a
// caller-given subset of the samples.

namespace kc {
namespace {

// centers [S][K] with the first t filled -> packed [S][t]
__global__ void fft_pack_kernel(const int64_t *__restrict__ C, int S, int K, int t, int64_t *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S * t; i += gridDim.x * blockDim.x)
        out[i] = C[(size_t)(i / t) * K + (i % t)];
}

// centers[s][t] = arg[s]; t = 0 seeds the sets with the starts
__global__ void fft_put_kernel(int64_t *__restrict__ C, int S, int K, int t, const int64_t *__restrict__ arg)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x)
        C[(size_t)s * K + t] = arg[s];
}

// largest id of a list (ordered max into *out, which starts at 0)
__global__ void max_id_kernel(const uint32_t *__restrict__ ids, int64_t n, unsigned *__restrict__ out)
{
    unsigned m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = ids[i] > m ? ids[i] : m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned w = __shfl_xor_sync(0xffffffffu, m, o);
        m = w > m ? w : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

}  // namespace
}  // namespace kc

extern "C" {

kc_status kc_fft_multi(kc_ctx *c, const int64_t *starts, int32_t S, int64_t *centers_out, double *obj_out)
{
    if (!c) return KC_EINVAL;
    if (S < 0 || S > 65536) return set_err(c, KC_EINVAL, "kc_fft_multi: S=%d outside [0, 65536]", S);
    if (S == 0) return KC_OK;
    if (!starts || !centers_out) return set_err(c, KC_EINVAL, "kc_fft_multi: NULL argument");
    KC_TRY(check_centers(c, starts, (size_t)S));
    const int K = c->K;
    Stager sg(c);
    const int is = sg.add(starts, (size_t)S * 8, true);
    const int ic = sg.add(centers_out, (size_t)S * K * 8, false);
    const int io = sg.add(obj_out, (size_t)S * 8, false);
    KC_TRY(sg.begin());
    const size_t packed = (size_t)S * K * 8, argb = (size_t)S * 8;
    KC_TRY(ensure(c, c->work, packed + argb + (size_t)S * 8 + 512));
    char *w = static_cast<char *>(c->work.p);
    int64_t *T = reinterpret_cast<int64_t *>(w);
    int64_t *arg = reinterpret_cast<int64_t *>(w + ((packed + 255) & ~(size_t)255));
    double *val = reinterpret_cast<double *>(w + ((packed + 255) & ~(size_t)255) + ((argb + 255) & ~(size_t)255));
    int64_t *C = static_cast<int64_t *>(sg.dev(ic));
    const int grid = std::max(1, std::min(c->num_sms * 4, (S * K + 255) / 256));
    fft_put_kernel<<<grid, 256, 0, c->stream>>>(C, S, K, 0, static_cast<const int64_t *>(sg.dev(is)));
    KC_TRY(after_launch(c, "fft start"));
    // Algorithm 2 for every start at once: the t-th point of set s is the
    // sample farthest from its first t points (one pass over the samples
    // serves all S sets)
    for (int t = 1; t < K; ++t) {
        fft_pack_kernel<<<grid, 256, 0, c->stream>>>(C, S, K, t, T);
        KC_TRY(after_launch(c, "fft pack"));
        KC_TRY(launch_objective(c, full_view(c), T, S, t, __builtin_huge_val(), val, arg));
        fft_put_kernel<<<grid, 256, 0, c->stream>>>(C, S, K, t, arg);
        KC_TRY(after_launch(c, "fft put"));
    }
    if (obj_out)
        KC_TRY(launch_objective(c, full_view(c), C, S, K, __builtin_huge_val(), static_cast<double *>(sg.dev(io)),
                                nullptr));
    return sg.finish();
}

kc_status kc_upper_bound_points(kc_ctx *c, const void *pts, int32_t S, int32_t Kc, double *ub_out, int64_t *worst_out)
{
    if (!c) return KC_EINVAL;
    if (S < 0 || S > 65536) return set_err(c, KC_EINVAL, "kc_upper_bound_points: S=%d outside [0, 65536]", S);
    if (Kc < 1 || Kc > kMaxK) return set_err(c, KC_EINVAL, "kc_upper_bound_points: Kc=%d outside [1, %d]", Kc, kMaxK);
    if (S == 0) return KC_OK;
    if (!pts || !ub_out) return set_err(c, KC_EINVAL, "kc_upper_bound_points: NULL argument");
    const size_t bytes = (size_t)S * Kc * c->D * c->esize;
    Stager sg(c);
    const int ip = sg.add(pts, bytes, true);
    const int iu = sg.add(ub_out, (size_t)S * 8, false);
    const int iw = sg.add(worst_out, (size_t)S * 8, false);
    KC_TRY(sg.begin());
    {
        // the points must be finite (checked on the host)
        std::vector<char> h(bytes);
        KC_CUDA(c, cudaMemcpyAsync(h.data(), sg.dev(ip), bytes, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        const size_t m = (size_t)S * Kc * c->D;
        for (size_t i = 0; i < m; ++i) {
            const double v = c->dt == KC_F32 ? (double)reinterpret_cast<const float *>(h.data())[i]
                                             : reinterpret_cast<const double *>(h.data())[i];
            if (!std::isfinite(v)) return set_err(c, KC_EINVAL, "kc_upper_bound_points: non-finite coordinate");
        }
    }
    KC_TRY(launch_objective(c, full_view(c), nullptr, S, Kc, __builtin_huge_val(), static_cast<double *>(sg.dev(iu)),
                            static_cast<int64_t *>(sg.dev(iw)), sg.dev(ip)));
    return sg.finish();
}

kc_status kc_lower_bounds_subset(kc_ctx *c, const uint32_t *ids, int64_t n, const void *lo, const void *hi, int32_t B,
                                 double *lb_out, double *lb_raw_out, int64_t *argmax_out, float *kernel_ms_out)
{
    if (!c) return KC_EINVAL;
    if (B < 0 || B > 4096) return set_err(c, KC_EINVAL, "kc_lower_bounds_subset: B=%d outside [0, 4096]", B);
    if (n < 0 || n > c->N) return set_err(c, KC_EINVAL, "kc_lower_bounds_subset: n=%lld outside [0, N]", (long long)n);
    if (c->dt != KC_F32) return set_err(c, KC_EINVAL, "kc_lower_bounds_subset: float data only");
    if (c->D > 8) return set_err(c, KC_EINVAL, "kc_lower_bounds_subset: D <= 8 (got %d)", c->D);
    if (B == 0) return KC_OK;
    if (!lo || !hi || !lb_out || (n > 0 && !ids)) return set_err(c, KC_EINVAL, "kc_lower_bounds_subset: NULL argument");
    const size_t box = (size_t)B * c->K * c->D * c->esize;
    Stager sg(c);
    const int iid = sg.add(n > 0 ? ids : nullptr, (size_t)n * 4, true);
    const int ilo = sg.add(lo, box, true), ihi = sg.add(hi, box, true);
    const int ilb = sg.add(lb_out, (size_t)B * 8, false);
    const int iraw = sg.add(lb_raw_out, (size_t)B * 8, false);
    const int iarg = sg.add(argmax_out, (size_t)B * 8, false);
    KC_TRY(sg.begin());
    const uint32_t *dids = static_cast<const uint32_t *>(sg.dev(iid));
    // the batch descriptor: one group (every node shares the subset), then
    // scratch for the per-node keys and the id check
    const int LT = list_tile();
    const size_t desc = 512, keys_off = desc, chk_off = keys_off + (((size_t)B * 8 + 255) & ~(size_t)255);
    KC_TRY(ensure(c, c->work, chk_off + 256));
    char *w = static_cast<char *>(c->work.p);
    unsigned *dmax = reinterpret_cast<unsigned *>(w + chk_off);
    if (n > 0) {
        // every id must name a sample: one pass over the ids, checked on the host
        KC_CUDA(c, cudaMemsetAsync(dmax, 0, 4, c->stream));
        max_id_kernel<<<std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8)), 256, 0,
                        c->stream>>>(dids, n, dmax);
        KC_TRY(after_launch(c, "subset id check"));
        unsigned hmax = 0;
        KC_CUDA(c, cudaMemcpyAsync(&hmax, dmax, 4, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        if ((int64_t)hmax >= c->N)
            return set_err(c, KC_EINVAL, "kc_lower_bounds_subset: id %u outside [0, N)", hmax);
    }
    int64_t hd[7] = {0, n, 0, (n + LT - 1) / LT, 0, 0, 0};   // seg_off, seg_n, tile_prefix[2], node_start[2]
    int *ns = reinterpret_cast<int *>(&hd[4]);
    ns[0] = 0;
    ns[1] = B;
    KC_CUDA(c, cudaMemcpyAsync(w, hd, sizeof(hd), cudaMemcpyHostToDevice, c->stream));
    const int64_t *dd = reinterpret_cast<const int64_t *>(w);
    ListBatch L;
    L.pool = dids;
    L.seg_off = dd;
    L.seg_n = dd + 1;
    L.tile_prefix = dd + 2;
    L.node_start = reinterpret_cast<const int *>(dd + 4);
    L.B = 1;
    L.W = hd[3];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (kernel_ms_out) {
        KC_CUDA(c, cudaEventCreate(&e0));
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return set_err(c, KC_ECUDA, "kc_lower_bounds_subset: cudaEventCreate failed");
        }
        cudaEventRecord(e0, c->stream);
    }
    kc_status st = launch_seg_lb(c, L, sg.dev(ilo), sg.dev(ihi), B, reinterpret_cast<unsigned long long *>(w + keys_off),
                                 static_cast<double *>(sg.dev(ilb)), static_cast<double *>(sg.dev(iraw)),
                                 static_cast<int64_t *>(sg.dev(iarg)));
    if (kernel_ms_out) {
        cudaEventRecord(e1, c->stream);
        if (st == KC_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(kernel_ms_out, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    KC_TRY(st);
    return sg.finish();
}

}  // extern "C"
