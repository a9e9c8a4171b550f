// gf_internal.cuh -- shared definitions of the GB300 kd-GeRaF library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

#include "gf.h"

// ---------------------------------------------------------------- the forest object
//
// Device layout (all row-major, all owned by the forest unless borrowed):
//   x       float [n][ldx]        points, rows padded with zeros to ldx = round_up(d, 4) floats
//   nodes   int2  [T][2^L - 1]    internal nodes in heap order: .x split dim, .y split value bits
//   perm    int32 [T][n]          leaf permutation of every tree (leaf b = [b n >> L, (b+1) n >> L))
//   xb      bf16  [n][ldb]        optional screening copy, ldb = round_up(d, 8)
//   xbn     float [n]             |xb_i|^2 (float64 sum rounded once), with xb
//   x8      e4m3  [n][ld8]        optional screening copy, ld8 = round_up(d, 16)
//   scale8  float [n]             per-row scale of x8
//   x8n     float [n]             |scale8_i x8_i|^2 (float64 sum rounded once), with x8
struct gf_forest {
    int64_t n = 0;
    int32_t d = 0, T = 0, leaf_size = 0, L = 0;
    int32_t max_leaf = 0, cand_cap = 0;
    int32_t ldx = 0, ldb = 0, ld8 = 0;
    float *x = nullptr;
    bool owns_x = true;
    int2 *nodes = nullptr;
    int32_t *perm = nullptr;
    __nv_bfloat16 *xb = nullptr;
    float *xbn = nullptr;
    uint8_t *x8 = nullptr;
    float *scale8 = nullptr;
    float *x8n = nullptr;
    float *U = nullptr;  // [T][d] Householder vectors (Sec. 2.2), or null: trees on X itself
    int device = 0;
    int num_sms = 0;
    // per-precision kernel shape and shortlist (written by the autotuner)
    int32_t tune_warps[3] = {8, 8, 8};
    int32_t tune_ctas[3] = {0, 0, 0};
    int32_t tune_R[3] = {0, 64, 128};
    int32_t tune_G[3] = {0, 0, 0};  // rows in flight per warp, 0 = kernel default
    int64_t device_bytes = 0;
};

// Limits of the tuning values (gf_forest_set_tuning, forest files): an SM runs at most 32 CTAs,
// and the streaming kernel keeps at most 2048 keys (k or R) per query.
constexpr int32_t GF_MAX_CTAS_PER_SM = 32;
constexpr int32_t GF_MAX_SHORTLIST = 2048;

// Read-only view handed to kernels by value.
struct ForestView {
    const float *x;
    const __nv_bfloat16 *xb;
    const float *xbn;
    const uint8_t *x8;
    const float *scale8;
    const float *x8n;
    const float *U;  // [T][d] or null
    const int2 *nodes;
    const int32_t *perm;
    long long n;
    int d, ldx, ldb, ld8, T, L, nnodes, max_leaf, cand_cap;
};

inline ForestView view_of(const gf_forest *F) {
    ForestView v;
    v.x = F->x; v.xb = F->xb; v.xbn = F->xbn; v.x8 = F->x8; v.scale8 = F->scale8; v.x8n = F->x8n; v.U = F->U;
    v.nodes = F->nodes; v.perm = F->perm;
    v.n = F->n; v.d = F->d; v.ldx = F->ldx; v.ldb = F->ldb; v.ld8 = F->ld8;
    v.T = F->T; v.L = F->L; v.nnodes = (1 << F->L) - 1;
    v.max_leaf = F->max_leaf; v.cand_cap = F->cand_cap;
    return v;
}

// ---------------------------------------------------------------- Householder reflection
// Sec. 2.2: each tree may be built on P x = x - 2 (u^T x) u, and queries are reflected the same way
// before descending it.  Evaluated in float32 in a fixed order with every multiply and add rounded
// on its own (no fused multiply-add), so the library and any reference that follows the same order
// produce identical coordinates: w2 = 2 * sum_j u_j x_j (j ascending), x'_j = x_j - w2 * u_j.
__device__ __forceinline__ float reflect_w2(const float *u, const float *x, int d) {
    float w = 0.f;
    for (int j = 0; j < d; ++j) w = __fadd_rn(w, __fmul_rn(__ldg(u + j), x[j]));
    return 2.f * w;
}

__device__ __forceinline__ float reflect_coord(float x, float w2, float u) { return __fsub_rn(x, __fmul_rn(w2, u)); }

// ---------------------------------------------------------------- shape helpers

inline int32_t depth_of(int64_t n, int32_t p) {
    int32_t L = 0;
    while (((n + ((int64_t)1 << L) - 1) >> L) > p) L++;
    return L;
}

inline int32_t round_up(int32_t a, int32_t b) { return (a + b - 1) / b * b; }

inline int32_t next_pow2(int32_t v) {
    int32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// ---------------------------------------------------------------- errors

int gf_fail(int code, const char *fmt, ...);  // records the thread's message, returns code
int gf_cuda_fail(cudaError_t e, const char *what);

#define GF_CUDA_TRY(expr)                                    \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return gf_cuda_fail(e_, #expr); \
    } while (0)

// Allocation with the library's error code (nothing is leaked on failure).
int gf_dmalloc(void **p, size_t bytes);

// ---------------------------------------------------------------- entry points between units

// Forest storage (gf_forest.cu).  gf_forest_alloc: shape fields and storage of x / nodes / perm;
// X is copied (from a device or host address) unless borrow.  gf_forest_fill_structure: validate
// a host tree structure, upload it and check X for NaN/Inf (on error the caller releases F).
int gf_forest_alloc(gf_forest **out, const float *X, int64_t n, int32_t d, int32_t T,
                    int32_t leaf_size, bool borrow, cudaStream_t st);
void gf_forest_destroy(gf_forest *F);
int gf_check_finite(const float *X, int64_t count, cudaStream_t st);
int gf_forest_fill_structure(gf_forest *F, const int32_t *split_dim_host, const float *split_val_host,
                             const int32_t *perm_host);
int gf_forest_set_U(gf_forest *F, const float *U_host);

struct QueryExtra {
    int32_t algo = GF_ALGO_AUTO;
    void *workspace = nullptr;
    int64_t workspace_bytes = 0;
    int32_t *ncand_out = nullptr;
    int32_t rows_in_flight = 0;
    int32_t order = GF_ORDER_AUTO;
    int32_t leaf_budget = 0;  // leaves per query for the priority search (0: one per tree)
    cudaEvent_t *events = nullptr;  // recorded around the scoring kernel's launches (timing)
};

// Record events[i] on st when the caller asked for timing events.
inline cudaError_t gf_record(const QueryExtra &x, int i, cudaStream_t st) {
    return x.events ? cudaEventRecord(x.events[i], st) : cudaSuccess;
}

int gf_launch_prio_leaves(const gf_forest *F, const float *Q, int64_t m, int budget, unsigned *leaves,
                          int *nleaves, cudaStream_t st);
size_t gf_prio_smem_bytes(int budget, int T);
int gf_stream_workspace_bytes(const gf_forest *F, int64_t m, long long grid, bool ordered, int leaf_budget,
                              int64_t *bytes);
// CTAs of a streaming launch of m queries with this shape (warps, ctas_per_sm 0 = occupancy limit)
int gf_stream_grid(const gf_forest *F, int64_t m, int warps, int ctas_per_sm, int precision, int k, int R,
                   long long *grid);

// Leaves the priority search checks per query: max(T, ceil(checks / (1 + eps))), 0 when that is T.
inline int32_t leaf_budget_of(const gf_forest *F, int32_t checks, double eps) {
    if (checks <= F->T) return 0;
    const double budget = (double)checks / (1.0 + eps);
    long long nl = F->T;
    while ((double)nl < budget) ++nl;  // the same comparison the search loop makes
    return nl > F->T ? (int32_t)nl : 0;
}

// Leaf-major batched path (GF_ALGO_LEAF): float32 or the bf16 screen.
// leaf_budget > 0: the priority search's leaves (QueryExtra::leaf_budget), else one leaf per tree.
// ctas_per_sm: the tensor-core kernel's shape, 1 = one CTA per SM (deeper ring), else two.
int gf_launch_leaf(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t precision, int32_t R,
                   int32_t order, int32_t leaf_budget, cudaStream_t st, int64_t *ids, float *dists,
                   void *workspace, int64_t workspace_bytes, cudaEvent_t *events = nullptr,
                   int32_t ctas_per_sm = 0);
int64_t gf_leaf_workspace_bytes(const gf_forest *F, int64_t m, int32_t precision, int32_t R, int32_t order,
                                int32_t leaf_budget);
// Whether GF_ALGO_AUTO takes the leaf-major path for this batch.
bool gf_leaf_preferred(const gf_forest *F, int64_t m, int32_t k, int32_t precision, int32_t R, const QueryExtra &x);
// Why the leaf-major path cannot run this query (nullptr: it can).
const char *gf_leaf_unsupported(const gf_forest *F, int64_t m, int32_t k, int32_t precision, int32_t R,
                                const QueryExtra &x);

int gf_launch_query(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t precision,
                    int32_t R, int32_t warps, int32_t ctas_per_sm, cudaStream_t s, int64_t *ids,
                    float *dists, const QueryExtra &x);
