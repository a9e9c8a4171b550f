// gf_forest.cu -- forest lifecycle (import, export, free), screening copies and the query entry
// points of the C ABI.
#include "gf_internal.cuh"

#include <atomic>
#include "gf_trace.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

// ---------------------------------------------------------------- errors

static thread_local std::string g_last_error;

int gf_fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int gf_cuda_fail(cudaError_t e, const char *what) {
    const int code = (e == cudaErrorMemoryAllocation) ? GF_ENOMEM : GF_ECUDA;
    return gf_fail(code, "%s: %s", what, cudaGetErrorString(e));
}

// gf_debug_fail_alloc: the number of library allocations that still succeed before one fails
// (-1: none fails)
static std::atomic<int> g_alloc_countdown{-1};

extern "C" int gf_debug_fail_alloc(int32_t after) {
    g_alloc_countdown.store(after < 0 ? -1 : after);
    return GF_OK;
}

int gf_dmalloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return GF_OK;
    for (int c = g_alloc_countdown.load(); c >= 0;) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 0) return gf_fail(GF_ENOMEM, "cudaMalloc(%zu bytes): refused (gf_debug_fail_alloc)", bytes);
            break;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();  // clear the sticky-free allocation error
        return gf_fail(GF_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return GF_OK;
}

extern "C" const char *gf_last_error(void) { return g_last_error.c_str(); }
extern "C" int32_t gf_version(void) { return 100; }

extern "C" void gf_rand_params_default(gf_rand_params *rp) {
    if (!rp) return;
    rp->t = 5;
    rp->shuffle = 1;
    rp->var_scope = GF_VAR_NODE;
    rp->householder = 0;
}

extern "C" void gf_query_opts_default(gf_query_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = GF_FP32;
}

// ---------------------------------------------------------------- forest storage

// Destroy everything the forest owns (tolerates partially built forests).
static void forest_release(gf_forest *F) {
    if (!F) return;
    if (F->owns_x) cudaFree(F->x);
    cudaFree(F->nodes);
    cudaFree(F->perm);
    cudaFree(F->xb);
    cudaFree(F->xbn);
    cudaFree(F->x8);
    cudaFree(F->scale8);
    cudaFree(F->x8n);
    cudaFree(F->U);
    delete F;
}

// Shape fields and the storage of x / nodes / perm.  borrow: keep X itself.  X may be a device or
// a host pointer when it is copied (the copies infer the direction from the address).
int gf_forest_alloc(gf_forest **out, const float *X, int64_t n, int32_t d, int32_t T,
                    int32_t leaf_size, bool borrow, cudaStream_t st) {
    *out = nullptr;
    if (!X) return gf_fail(GF_EINVAL, "X is null");
    if (n < 1 || n > 0x7fffffffLL) return gf_fail(GF_EINVAL, "n=%lld outside [1, 2^31)", (long long)n);
    if (d < 1 || d > 65535) return gf_fail(GF_EINVAL, "d=%d outside [1, 65535]", d);
    if (T < 1 || T > 4096) return gf_fail(GF_EINVAL, "T=%d outside [1, 4096]", T);
    if (leaf_size < 1) return gf_fail(GF_EINVAL, "leaf_size=%d < 1", leaf_size);
    gf_forest *F = new gf_forest();
    F->n = n; F->d = d; F->T = T; F->leaf_size = leaf_size;
    F->L = depth_of(n, leaf_size);
    if (F->L > 30) {
        const int32_t L = F->L;
        delete F;
        return gf_fail(GF_EINVAL, "tree depth %d too large", L);
    }
    F->max_leaf = (int32_t)((n + ((int64_t)1 << F->L) - 1) >> F->L);
    const int64_t cap = (int64_t)T * F->max_leaf;
    if (cap > (1 << 24)) { delete F; return gf_fail(GF_EINVAL, "T * leaf size = %lld too large", (long long)cap); }
    F->cand_cap = (int32_t)cap;
    F->ldx = round_up(d, 4);
    F->ldb = round_up(d, 8);
    F->ld8 = round_up(d, 16);
    cudaGetDevice(&F->device);
    cudaDeviceGetAttribute(&F->num_sms, cudaDevAttrMultiProcessorCount, F->device);
    const size_t nn = ((size_t)1 << F->L) - 1;
    int r;
    if (borrow) {
        if (d % 4 != 0 || ((uintptr_t)X & 15) != 0) {
            delete F;
            return gf_fail(GF_EINVAL, "borrowed X needs d %% 4 == 0 and 16-byte alignment");
        }
        F->x = const_cast<float *>(X);
        F->owns_x = false;
    } else {
        if ((r = gf_dmalloc((void **)&F->x, (size_t)n * F->ldx * 4))) { forest_release(F); return r; }
        F->owns_x = true;
        if (F->ldx != d) {
            cudaError_t e = cudaMemsetAsync(F->x, 0, (size_t)n * F->ldx * 4, st);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(F->x, (size_t)F->ldx * 4, X, (size_t)d * 4, (size_t)d * 4, (size_t)n,
                                      cudaMemcpyDefault, st);
            if (e != cudaSuccess) { forest_release(F); return gf_cuda_fail(e, "copy X"); }
        } else {
            cudaError_t e = cudaMemcpyAsync(F->x, X, (size_t)n * d * 4, cudaMemcpyDefault, st);
            if (e != cudaSuccess) { forest_release(F); return gf_cuda_fail(e, "copy X"); }
        }
    }
    if ((r = gf_dmalloc((void **)&F->nodes, (size_t)T * nn * sizeof(int2)))) { forest_release(F); return r; }
    if ((r = gf_dmalloc((void **)&F->perm, (size_t)T * n * 4))) { forest_release(F); return r; }
    F->device_bytes = (borrow ? 0 : (int64_t)n * F->ldx * 4) + (int64_t)(T * nn * sizeof(int2)) + (int64_t)T * n * 4;
    *out = F;
    return GF_OK;
}

void gf_forest_destroy(gf_forest *F) { forest_release(F); }

// Count non-finite entries of X (rows of d floats).
__global__ void k_count_nonfinite(const float *__restrict__ X, long long total, unsigned long long *bad) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        c += !isfinite(X[i]);
    c = __reduce_add_sync(0xffffffffu, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

int gf_check_finite(const float *X, int64_t count, cudaStream_t st) {
    unsigned long long *bad = nullptr;
    int r = gf_dmalloc((void **)&bad, sizeof *bad);
    if (r) return r;
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof *bad, st);
    if (e == cudaSuccess) {
        k_count_nonfinite<<<1216, 256, 0, st>>>(X, count, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(bad);
    if (e != cudaSuccess) return gf_cuda_fail(e, "finite check");
    if (h) return gf_fail(GF_EINVAL, "X holds %llu NaN/Inf values", h);
    return GF_OK;
}

// ---------------------------------------------------------------- import / export

// Validate a host tree structure and copy it into F (nodes, perm), then check X for NaN/Inf.
// On error F is left for the caller to release.
int gf_forest_fill_structure(gf_forest *F, const int32_t *split_dim_host, const float *split_val_host,
                             const int32_t *perm_host) {
    const int64_t n = F->n;
    const int32_t d = F->d, T = F->T;
    const size_t nn = ((size_t)1 << F->L) - 1;
    std::vector<int2> nodes((size_t)T * nn);
    for (size_t i = 0; i < nodes.size(); ++i) {
        if (split_dim_host[i] < 0 || split_dim_host[i] >= d)
            return gf_fail(GF_EINVAL, "split_dim[%zu] = %d outside [0, %d)", i, split_dim_host[i], d);
        int32_t bits;
        std::memcpy(&bits, &split_val_host[i], 4);
        nodes[i] = make_int2(split_dim_host[i], bits);
    }
    std::vector<unsigned char> seen((size_t)n);
    for (int32_t t = 0; t < T; ++t) {
        std::fill(seen.begin(), seen.end(), 0);
        for (int64_t i = 0; i < n; ++i) {
            const int32_t v = perm_host[(size_t)t * n + i];
            if (v < 0 || v >= n || seen[v])
                return gf_fail(GF_EINVAL, "perm row %d is not a permutation of 0..n-1", t);
            seen[v] = 1;
        }
    }
    cudaError_t e = cudaMemcpy(F->nodes, nodes.data(), nodes.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(F->perm, perm_host, (size_t)T * n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return gf_cuda_fail(e, "import copy");
    return gf_check_finite(F->x, (int64_t)n * F->ldx, 0);
}

extern "C" int gf_forest_import(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                                const int32_t *split_dim_host, const float *split_val_host,
                                const int32_t *perm_host, gf_forest **out) {
    GfRange range("gf_forest_import");
    if (!out) return gf_fail(GF_EINVAL, "out is null");
    *out = nullptr;
    if (!split_dim_host || !split_val_host || !perm_host) return gf_fail(GF_EINVAL, "null host array");
    gf_forest *F = nullptr;
    int r = gf_forest_alloc(&F, X, n, d, T, leaf_size, false, 0);
    if (r) return r;
    if ((r = gf_forest_fill_structure(F, split_dim_host, split_val_host, perm_host))) {
        forest_release(F);
        return r;
    }
    *out = F;
    return GF_OK;
}

extern "C" int gf_forest_export(const gf_forest *F, int32_t *split_dim_host, float *split_val_host,
                                int32_t *perm_host) {
    if (!F) return gf_fail(GF_EINVAL, "null forest");
    const size_t nn = ((size_t)1 << F->L) - 1;
    std::vector<int2> nodes((size_t)F->T * nn);
    if (!nodes.empty()) GF_CUDA_TRY(cudaMemcpy(nodes.data(), F->nodes, nodes.size() * sizeof(int2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < nodes.size(); ++i) {
        if (split_dim_host) split_dim_host[i] = nodes[i].x;
        if (split_val_host) std::memcpy(&split_val_host[i], &nodes[i].y, 4);
    }
    if (perm_host) GF_CUDA_TRY(cudaMemcpy(perm_host, F->perm, (size_t)F->T * F->n * 4, cudaMemcpyDeviceToHost));
    return GF_OK;
}

extern "C" int gf_forest_get_info(const gf_forest *F, gf_forest_info *info) {
    if (!F || !info) return gf_fail(GF_EINVAL, "null argument");
    info->n = F->n; info->d = F->d; info->T = F->T; info->leaf_size = F->leaf_size; info->L = F->L;
    info->max_leaf = F->max_leaf; info->cand_cap = F->cand_cap;
    info->screens = (F->xb ? (1 << GF_BF16_RERANK) : 0) | (F->x8 ? (1 << GF_FP8_RERANK) : 0);
    info->device_bytes = F->device_bytes;
    return GF_OK;
}

// Copy the per-tree Householder vectors (host [T][d]) into the forest.
int gf_forest_set_U(gf_forest *F, const float *U_host) {
    const size_t bytes = (size_t)F->T * F->d * 4;
    if (!F->U) {
        int r = gf_dmalloc((void **)&F->U, bytes);
        if (r) return r;
        F->device_bytes += (int64_t)bytes;
    }
    GF_CUDA_TRY(cudaMemcpy(F->U, U_host, bytes, cudaMemcpyHostToDevice));
    return GF_OK;
}

extern "C" int gf_forest_set_reflections(gf_forest *F, const float *U_host) {
    if (!F || !U_host) return gf_fail(GF_EINVAL, "null argument");
    for (size_t i = 0; i < (size_t)F->T * F->d; ++i)
        if (!std::isfinite(U_host[i])) return gf_fail(GF_EINVAL, "U holds NaN/Inf");
    return gf_forest_set_U(F, U_host);
}

extern "C" int gf_forest_free(gf_forest *F) {
    if (!F) return GF_OK;
    cudaDeviceSynchronize();
    forest_release(F);
    return GF_OK;
}

extern "C" int gf_forest_set_tuning(gf_forest *F, int32_t precision, int32_t warps_per_cta,
                                    int32_t ctas_per_sm, int32_t rerank_R, int32_t rows_in_flight) {
    if (!F || precision < 0 || precision > 2) return gf_fail(GF_EINVAL, "bad forest or precision");
    if (warps_per_cta < 1 || warps_per_cta > 32 || ctas_per_sm < 0 || ctas_per_sm > GF_MAX_CTAS_PER_SM ||
        rerank_R < 0 || rerank_R > GF_MAX_SHORTLIST ||
        (rows_in_flight != 0 && rows_in_flight != 2 && rows_in_flight != 4))
        return gf_fail(GF_EINVAL, "bad tuning values");
    F->tune_warps[precision] = warps_per_cta;
    F->tune_ctas[precision] = ctas_per_sm;
    if (rerank_R > 0) F->tune_R[precision] = rerank_R;
    if (rows_in_flight > 0) F->tune_G[precision] = rows_in_flight;
    return GF_OK;
}

// ---------------------------------------------------------------- screening copies

// xb[i][j] = bf16_rne(x[i][j]) for j < d, 0 in the padding.
__global__ void k_to_bf16(const float *__restrict__ x, int ldx, long long n, int d, int ldb,
                          __nv_bfloat16 *xb) {
    const long long total = n * ldb;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long i = g / ldb;
        const int j = (int)(g - i * ldb);
        xb[g] = __float2bfloat16_rn(j < d ? x[i * ldx + j] : 0.f);
    }
}

// One warp per row: a = max |x|, scale = a / 448, codes = e4m3_rne_satfinite(x * (448 / a)).
__global__ void k_to_fp8(const float *__restrict__ x, int ldx, long long n, int d, int ld8, uint8_t *x8,
                         float *scale) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < n; i += nw) {
        const float *r = x + i * ldx;
        float a = 0.f;
        for (int j = lane; j < d; j += 32) a = fmaxf(a, fabsf(r[j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        const float inv = a > 0.f ? 448.0f / a : 0.f;
        if (lane == 0) scale[i] = a > 0.f ? a / 448.0f : 1.0f;
        for (int j = lane; j < ld8; j += 32) {
            const float v = j < d ? r[j] * inv : 0.f;
            x8[i * ld8 + j] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// xbn[i] = sum_j xb[i][j]^2, accumulated in float64 and rounded once: a warp per row.
__global__ void k_bf16_sqnorm(const __nv_bfloat16 *__restrict__ xb, long long n, int ldb, float *xbn) {
    const int lane = threadIdx.x & 31;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((long long)gridDim.x * blockDim.x) >> 5) {
        double acc = 0.0;
        for (int j = lane; j < ldb; j += 32) {
            const double v = (double)__bfloat162float(xb[i * ldb + j]);
            acc += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) xbn[i] = (float)acc;
    }
}

// x8n[i] = sum_j (scale_i x8[i][j])^2, accumulated in float64 and rounded once: a warp per row.
__global__ void k_fp8_sqnorm(const uint8_t *__restrict__ x8, const float *__restrict__ scale, long long n, int ld8,
                             float *x8n) {
    const int lane = threadIdx.x & 31;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((long long)gridDim.x * blockDim.x) >> 5) {
        double acc = 0.0;
        for (int j = lane; j < ld8; j += 32) {
            const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)x8[i * ld8 + j], __NV_E4M3);
            const double v = (double)__half2float(*reinterpret_cast<const __half *>(&h));
            acc += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double sc = (double)scale[i];
        if (lane == 0) x8n[i] = (float)(acc * sc * sc);
    }
}

extern "C" int gf_forest_add_screen(gf_forest *F, int32_t precision, void *stream) {
    GfRange range("gf_forest_add_screen");
    if (!F) return gf_fail(GF_EINVAL, "null forest");
    cudaStream_t st = (cudaStream_t)stream;
    int r;
    if (precision == GF_BF16_RERANK) {
        if (F->xb) return GF_OK;
        if ((r = gf_dmalloc((void **)&F->xb, (size_t)F->n * F->ldb * 2))) return r;
        if ((r = gf_dmalloc((void **)&F->xbn, (size_t)F->n * 4))) { cudaFree(F->xb); F->xb = nullptr; return r; }
        k_to_bf16<<<F->num_sms * 8, 256, 0, st>>>(F->x, F->ldx, F->n, F->d, F->ldb, F->xb);
        k_bf16_sqnorm<<<F->num_sms * 8, 256, 0, st>>>(F->xb, F->n, F->ldb, F->xbn);
        F->device_bytes += (int64_t)F->n * F->ldb * 2 + F->n * 4;
    } else if (precision == GF_FP8_RERANK) {
        if (F->x8) return GF_OK;
        if ((r = gf_dmalloc((void **)&F->x8, (size_t)F->n * F->ld8))) return r;
        if ((r = gf_dmalloc((void **)&F->scale8, (size_t)F->n * 4))) { cudaFree(F->x8); F->x8 = nullptr; return r; }
        if ((r = gf_dmalloc((void **)&F->x8n, (size_t)F->n * 4))) {
            cudaFree(F->x8);
            cudaFree(F->scale8);
            F->x8 = nullptr;
            F->scale8 = nullptr;
            return r;
        }
        k_to_fp8<<<F->num_sms * 8, 256, 0, st>>>(F->x, F->ldx, F->n, F->d, F->ld8, F->x8, F->scale8);
        k_fp8_sqnorm<<<F->num_sms * 8, 256, 0, st>>>(F->x8, F->scale8, F->n, F->ld8, F->x8n);
        F->device_bytes += (int64_t)F->n * F->ld8 + F->n * 8;
    } else {
        return gf_fail(GF_EINVAL, "precision %d has no screening copy", precision);
    }
    GF_CUDA_TRY(cudaGetLastError());
    GF_CUDA_TRY(cudaStreamSynchronize(st));
    return GF_OK;
}

// ---------------------------------------------------------------- queries

extern "C" int gf_query_ex(const gf_forest *F, const float *Q, int64_t m, int32_t k,
                           const gf_query_opts *o, int64_t *ids, float *dists) {
    GfRange range("gf_query");
    if (!F) return gf_fail(GF_EINVAL, "null forest");
    if (m < 0) return gf_fail(GF_EINVAL, "m < 0");
    if (k < 1) return gf_fail(GF_EINVAL, "k=%d < 1", k);
    if (m == 0) return GF_OK;
    if (!Q || !ids || !dists) return gf_fail(GF_EINVAL, "null pointer");
    gf_query_opts def;
    gf_query_opts_default(&def);
    if (!o) o = &def;
    const int p = o->precision;
    if (p < 0 || p > 2) return gf_fail(GF_EINVAL, "unknown precision %d", p);
    if (p == GF_BF16_RERANK && !F->xb) return gf_fail(GF_EINVAL, "forest has no bf16 copy (gf_forest_add_screen)");
    if (p == GF_FP8_RERANK && !F->x8) return gf_fail(GF_EINVAL, "forest has no fp8 copy (gf_forest_add_screen)");
    const int R = o->rerank_R > 0 ? o->rerank_R : F->tune_R[p];
    if (p != GF_FP32 && k > R) return gf_fail(GF_EINVAL, "k=%d exceeds the shortlist R=%d", k, R);
    const int warps = o->warps_per_cta > 0 ? o->warps_per_cta : F->tune_warps[p];
    if (warps > 32) return gf_fail(GF_EINVAL, "warps_per_cta=%d > 32", warps);
    const int cps = o->ctas_per_sm > 0 ? o->ctas_per_sm : F->tune_ctas[p];
    if (o->algo < GF_ALGO_AUTO || o->algo > GF_ALGO_LEAF) return gf_fail(GF_EINVAL, "unknown algo %d", o->algo);
    QueryExtra x;
    x.algo = o->algo;
    x.workspace = o->workspace;
    x.workspace_bytes = o->workspace_bytes;
    x.ncand_out = o->ncand_out;
    x.rows_in_flight = o->rows_in_flight > 0 ? o->rows_in_flight : F->tune_G[p];
    if (o->order < GF_ORDER_AUTO || o->order > GF_ORDER_LOCALITY) return gf_fail(GF_EINVAL, "unknown order %d", o->order);
    x.order = o->order;
    if (o->checks < 0 || !(o->eps >= 0.0)) return gf_fail(GF_EINVAL, "checks < 0 or eps < 0");
    x.leaf_budget = leaf_budget_of(F, o->checks, o->eps);
    x.events = (cudaEvent_t *)o->events;
    if (x.leaf_budget > 0) {
        if (((unsigned long long)F->T << F->L) > 0xffffffffull)
            return gf_fail(GF_EUNSUPPORTED, "priority search needs T * 2^L <= 2^32");
        if (x.leaf_budget > 4096) return gf_fail(GF_EUNSUPPORTED, "leaf budget %d above 4096", x.leaf_budget);
    }
    return gf_launch_query(F, Q, m, k, p, R, warps, cps, (cudaStream_t)o->stream, ids, dists, x);
}

extern "C" int gf_query_workspace_size(const gf_forest *F, int64_t m, const gf_query_opts *o, int64_t *bytes) {
    if (!F || !bytes) return gf_fail(GF_EINVAL, "null argument");
    gf_query_opts def;
    gf_query_opts_default(&def);
    if (!o) o = &def;
    const int p = o->precision;
    if (p < 0 || p > 2) return gf_fail(GF_EINVAL, "unknown precision %d", p);
    // the streaming kernel runs at most 8 warps per CTA; fewer threads per CTA only raise the
    // occupancy-derived grid, so the clamp keeps the size an upper bound
    const int warps = std::min(8, o->warps_per_cta > 0 ? o->warps_per_cta : F->tune_warps[p]);
    const int cps = o->ctas_per_sm > 0 ? o->ctas_per_sm : F->tune_ctas[p];
    const int R = o->rerank_R > 0 ? o->rerank_R : F->tune_R[p];
    long long grid = 0;
    int r = gf_stream_grid(F, m, warps, cps, p, 1, R, &grid);
    if (r) return r;
    // A launch's own grid can be below this one (a larger k or R lowers the occupancy), and AUTO
    // reorders every batch longer than the launch's grid: count the order arrays for any m > 1.
    const bool ordered = o->order == GF_ORDER_LOCALITY || (o->order == GF_ORDER_AUTO && m > 1);
    if ((r = gf_stream_workspace_bytes(F, m, grid, ordered, leaf_budget_of(F, o->checks, o->eps), bytes))) return r;
    if (o->algo == GF_ALGO_LEAF || o->algo == GF_ALGO_AUTO) {
        // the leaf-major path's scratch; AUTO gets the larger of the two
        QueryExtra x;
        x.leaf_budget = leaf_budget_of(F, o->checks, o->eps);
        x.ncand_out = o->ncand_out;
        const bool leaf_ok = gf_leaf_unsupported(F, m, 1, p, R, x) == nullptr;
        const int64_t lb = gf_leaf_workspace_bytes(F, m, p, R, o->order, x.leaf_budget);
        if (o->algo == GF_ALGO_LEAF) *bytes = lb;
        else if (leaf_ok && gf_leaf_preferred(F, m, 1, p, R, x)) *bytes = std::max(*bytes, lb);
    }
    return GF_OK;
}

extern "C" int gf_query(const gf_forest *F, const float *Q, int64_t m, int32_t k, int64_t *ids,
                        float *dists) {
    return gf_query_ex(F, Q, m, k, nullptr, ids, dists);
}
