// gf_noalloc.cu -- a query entry point that allocates no memory.
//
// Some callers cannot allocate device memory at query time: code running under a memory pool they
// do not own (a framework's caching allocator that must see every byte), a real-time loop that
// may not call into the driver's allocator, or an embedding that forbids cudaMalloc after start-up.
// The streaming query kernel needs scratch (one "seen" bitmap of ceil(n / 32) words per CTA), which
// gf_query_ex either allocates stream-ordered or takes from the caller.  gf_query_noalloc takes it
// instead from a fixed array of device memory that is part of this library's image: it exists on
// every GPU that loads the library, from the first use until the process exits.
#include "gf_internal.cuh"

#include <algorithm>
#include <mutex>

// The scratch: GF_NOALLOC_SCRATCH_BYTES of device memory, shared by every call on a device.
static __device__ __align__(256) unsigned g_noalloc_scratch[GF_NOALLOC_SCRATCH_BYTES / 4];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// The device address of the scratch on the current device, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so the address must come from the runtime.
int scratch_on_current_device(void **out) {
    int dev = 0;
    GF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return gf_fail(GF_EUNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return gf_cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GF_OK;
}

}  // namespace

extern "C" int gf_query_noalloc(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t precision,
                                int32_t rerank_R, void *stream, int64_t *ids, float *dists) {
    if (!F) return gf_fail(GF_EINVAL, "gf_query_noalloc: null forest");
    if (m < 0 || k < 1) return gf_fail(GF_EINVAL, "gf_query_noalloc: bad sizes");
    if (m == 0) return GF_OK;
    if (!Q || !ids || !dists) return gf_fail(GF_EINVAL, "gf_query_noalloc: null pointer");
    if (precision < 0 || precision > 2) return gf_fail(GF_EINVAL, "gf_query_noalloc: unknown precision %d", precision);
    const int64_t words = (F->n + 31) / 32;
    const int64_t per_cta = words * 4;
    const int64_t max_ctas = (int64_t)GF_NOALLOC_SCRATCH_BYTES / per_cta;
    if (max_ctas < 1)
        return gf_fail(GF_EINVAL,
                       "gf_query_noalloc: a forest of %lld points needs %lld bytes of scratch per CTA, "
                       "more than the %lld-byte no-alloc scratch",
                       (long long)F->n, (long long)per_cta, (long long)GF_NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    int r = scratch_on_current_device(&scratch);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    gf_query_opts o;
    gf_query_opts_default(&o);
    o.precision = precision;
    o.rerank_R = rerank_R;
    o.stream = stream;
    o.algo = GF_ALGO_STREAM;
    o.workspace = scratch;
    o.workspace_bytes = GF_NOALLOC_SCRATCH_BYTES;
    // The queries go in launches of `chunk` rows: the longest whose whole scratch layout -- the
    // launch's bitmaps and, when its CTAs take the queries in locality order, 12 bytes a query --
    // fits in the array.  The layout grows with the rows of a launch, so a bisection finds it.
    auto need = [&](int64_t rows, int64_t *bytes) { return gf_query_workspace_size(F, rows, &o, bytes); };
    int64_t bytes = 0;
    int64_t chunk = m;
    if ((r = need(m, &bytes))) return r;
    if (bytes > GF_NOALLOC_SCRATCH_BYTES) {
        int64_t lo = 1, hi = m;  // need(lo) fits, need(hi) does not
        while (hi - lo > 1) {
            const int64_t mid = lo + (hi - lo) / 2;
            if ((r = need(mid, &bytes))) return r;
            (bytes <= GF_NOALLOC_SCRATCH_BYTES ? lo : hi) = mid;
        }
        chunk = lo;
    }
    // Only the bitmaps must start at zero (the locality keys are written before they are read).
    // They are the first grid * per_cta bytes, grid being at most the CTA count the size bound
    // above assumed for a launch of `chunk` rows.  The array keeps whatever the last call left in
    // it, e.g. another forest's keys, so they are cleared here.
    long long grid = 0;
    if ((r = gf_stream_grid(F, chunk, std::min(8, F->tune_warps[precision]), F->tune_ctas[precision], precision, 1,
                            rerank_R > 0 ? rerank_R : F->tune_R[precision], &grid)))
        return r;
    GF_CUDA_TRY(cudaMemsetAsync(scratch, 0, (size_t)(grid * per_cta), st));
    for (int64_t off = 0; off < m; off += chunk) {
        const int64_t mc = std::min<int64_t>(chunk, m - off);
        r = gf_query_ex(F, Q + off * F->d, mc, k, &o, ids + off * k, dists + off * k);
        if (r) return r;
    }
    return GF_OK;
}
