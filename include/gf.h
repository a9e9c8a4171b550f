/*
 * gf.h -- C ABI of the GB300 kd-GeRaF library (batched approximate nearest-neighbour search over a
 * forest of randomized k-d trees; Avrithis, Emiris, Samaras, arXiv 1603.09596).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named X, Q, ids, dists, leaf, cand, ncand are DEVICE pointers (cudaMalloc'ed or from
 *    a framework allocator) on the current CUDA device, unless the name ends in _host.
 *  - Matrices are row-major and contiguous: X is [n][d] float32, Q is [m][d] float32.
 *  - Outputs are allocated by the caller; the library never keeps a pointer to a caller buffer
 *    after the call returns (except the dataset when gf_build_ex is asked to borrow it).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  Query and
 *    stage calls are asynchronous on that stream: they return once the work is enqueued.  Build,
 *    import, export and free are synchronous.
 *  - Every function returns GF_OK (0) or a negative GF_E* code; no C++ exception crosses the ABI.
 *    gf_last_error() returns a message for the calling thread's most recent failure.
 *  - A const forest may be queried from several host threads at once (a query writes only to its
 *    own outputs and its own scratch).
 *
 * Tree layout (readings of the paper stated once here and used throughout):
 *  - Trees are perfect (Sec. 3 "Tree structure"): depth L = min{l >= 0 : ceil(n / 2^l) <= p} for
 *    leaf_size p; internal node j (heap order, children 2j+1 and 2j+2) stores (split dimension,
 *    split value); leaf b (0 <= b < 2^L) holds the points perm[t][floor(b n / 2^L) ..
 *    floor((b+1) n / 2^L)) of tree t, listed in ascending id order.
 */
#ifndef GF_H
#define GF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define GF_OK 0
#define GF_EINVAL (-1)        /* bad argument: null pointer, size out of range, t > d, k < 1 ... */
#define GF_ENOMEM (-2)        /* a device or host allocation failed; nothing was leaked */
#define GF_ECUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define GF_ETIMEOUT (-4)      /* a bounded wait ran out (serving loop) */
#define GF_EUNSUPPORTED (-5)  /* valid request the library does not implement (e.g. householder) */
#define GF_EIO (-6)           /* file could not be read or written, or has a bad format */

/* ---------------------------------------------------------------- parameters */

/* Variance scope for the split-dimension choice. */
#define GF_VAR_NODE 0   /* variance of each node's own points (default) */
#define GF_VAR_GLOBAL 1 /* variance of the whole dataset, once (Alg. 1 as printed) */

/* Randomization of the trees (Sec. 2.1). */
typedef struct gf_rand_params {
    int32_t t;           /* split dimension drawn uniformly from the t highest-variance dims */
    int32_t shuffle;     /* 1: per-tree random order breaks ties of equal coordinates
                            (Sec. 2.1 "Shuffling"); 0: ties broken by point id */
    int32_t var_scope;   /* GF_VAR_NODE or GF_VAR_GLOBAL */
    int32_t householder; /* per-tree reflection (Sec. 2.2): only with gf_build_reflected */
} gf_rand_params;

/* Candidate scoring precision (how the leaf points are ranked, Sec. 3 "Distance computation"). */
#define GF_FP32 0         /* exact float32 squared L2 over all candidates */
#define GF_BF16_RERANK 1  /* bfloat16 screen -> shortlist of R -> float32 rerank */
#define GF_FP8_RERANK 2   /* FP8-E4M3 (per-row float32 scale) screen -> R -> float32 rerank */

/* Query kernel.  Both give the same results (same distances, same (distance, id) order). */
#define GF_ALGO_AUTO 0   /* SORT for small candidate bounds, STREAM otherwise */
#define GF_ALGO_SORT 1   /* candidates sorted and de-duplicated in shared memory; needs
                            8 * next_pow2(T * max_leaf) bytes of shared memory per CTA */
#define GF_ALGO_STREAM 2 /* candidates de-duplicated through a per-CTA bitmap over the point ids
                            in device memory ("seen" array, Sec. 2.3); any candidate count */
#define GF_ALGO_LEAF 3   /* leaf-major batch (one leaf per tree): the (query, tree) pairs are
                            grouped by the leaf they reach, and each leaf's rows are read once per
                            group of up to 16 queries and scored against all of them -- the bf16
                            screen on the tensor cores, float32 (direct form) on the CUDA cores;
                            per query the trees' lists are merged and de-duplicated by id, and the
                            screen's R best reranked in float32.  Runs the priority search too (the
                            pairs are (query, leaf checked)); AUTO takes it for one leaf per tree
                            only.  bf16: R <= 32; float32: k <= 32; (leaves per query) * R <= 8192,
                            T * 2^L <= 2^22; the workspace need not be zero and is left zero */

/* Order in which the streaming kernel's CTAs take the queries of a batch.  Results do not depend
 * on it; throughput does: queries that reach the same leaf of tree 0 share most candidates, and
 * CTAs working on them at the same time find the shared rows in L2. */
#define GF_ORDER_AUTO 0      /* LOCALITY when the batch has more queries than the launch has CTAs */
#define GF_ORDER_GIVEN 1     /* as given */
#define GF_ORDER_LOCALITY 2  /* sorted by the leaf of tree 0 (chunks of 16,384 queries) */

typedef struct gf_query_opts {
    int32_t precision;       /* GF_FP32, GF_BF16_RERANK or GF_FP8_RERANK */
    int32_t rerank_R;        /* shortlist length for the screened precisions; 0 = forest default */
    int32_t warps_per_cta;   /* kernel shape; 0 = forest default (set by gf_forest_set_tuning) */
    int32_t ctas_per_sm;     /* kernel shape; 0 = forest default, else occupancy limit (LEAF with a
                                screen: 1 = one CTA per SM with a deeper ring, else two) */
    void *stream;            /* cudaStream_t */
    int32_t algo;            /* GF_ALGO_* */
    int32_t rows_in_flight;  /* STREAM only: rows each warp scores at once, 2 or 4; 0 = default */
    void *workspace;         /* STREAM only: device scratch of at least gf_query_workspace_size()
                                bytes, zero-filled before its first use (every query leaves it zero
                                again); NULL = the library allocates it stream-ordered
                                (cudaMallocAsync / cudaFreeAsync) for this call */
    int64_t workspace_bytes; /* size of `workspace` */
    int32_t *ncand_out;      /* STREAM only, optional: device [m] int32, number of distinct
                                candidates of each query */
    int32_t order;           /* STREAM only, GF_ORDER_*: the order in which CTAs take queries */
    int32_t checks;          /* the paper's c, max. leaf checks (Alg. 2, Sec. 3 "Parameters");
                                <= T: one leaf per tree (the default search) */
    double eps;              /* the paper's epsilon >= 0: c / (1 + eps) leaves are checked */
    void *events;            /* optional, for timing: two cudaEvent_t (created by the caller); the
                                query records events[0] on `stream` just before the first launch of
                                its scoring kernel (k_leaf_score / k_leaf_f32 on the leaf-major path,
                                else the streaming or sort query kernel) and events[1] just after the
                                last, so that kernel can be timed alone; NULL: no events */
} gf_query_opts;

typedef struct gf_forest gf_forest; /* opaque; owned by the library */

typedef struct gf_forest_info {
    int64_t n;           /* points */
    int32_t d;           /* dimensions */
    int32_t T;           /* trees */
    int32_t leaf_size;   /* p */
    int32_t L;           /* tree depth */
    int32_t max_leaf;    /* ceil(n / 2^L) */
    int32_t cand_cap;    /* T * max_leaf: upper bound on candidates per query */
    int32_t screens;     /* bit (1 << GF_BF16_RERANK) / (1 << GF_FP8_RERANK): derived copies held */
    int64_t device_bytes;/* device memory owned by the forest */
} gf_forest_info;

void gf_rand_params_default(gf_rand_params *rp); /* t = 5, shuffle = 1, var_scope = NODE */
void gf_query_opts_default(gf_query_opts *o);    /* FP32, everything else 0 / NULL */

/* ---------------------------------------------------------------- forest */

/*
 * gf_build -- build a forest of T randomized k-d trees on the GPU (Alg. 1; Alg. 3 variance;
 * Sec. 3 "Median, variances").  At every internal node one dimension is drawn uniformly among the
 * rp->t dimensions of largest variance and the node's points are split at the median in that
 * dimension (ties in the coordinate broken by the tree's random order when rp->shuffle).
 *   X          device, [n][d] float32, finite; copied into the forest (the caller may free it)
 *   n, d       1 <= n < 2^31, 1 <= d <= 65535
 *   T          number of trees, >= 1
 *   leaf_size  p >= 1: leaves hold at most p points
 *   rp         NULL for defaults
 *   seed       forest seed: the same (X, parameters, seed) always gives the same forest
 *   out        receives the new forest
 * Errors: GF_EINVAL (bad sizes, NaN/Inf in X, t outside [1, d], householder without vectors),
 * GF_ENOMEM, GF_ECUDA.  Synchronous.
 */
int gf_build(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
             const gf_rand_params *rp, uint64_t seed, gf_forest **out);

/* As gf_build, on `stream`; borrow_x = 1 keeps a pointer to X instead of copying it (X must then
 * outlive the forest and have d % 4 == 0 and 16-byte alignment). */
int gf_build_ex(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                const gf_rand_params *rp, uint64_t seed, int32_t borrow_x, void *stream,
                gf_forest **out);

/*
 * gf_build_reflected -- gf_build_ex with a Householder reflection per tree (Sec. 2.2): tree t is
 * built on P_t x = x - 2 (u_t^T x) u_t, and every query is reflected the same way before it
 * descends tree t (Sec. 2.3); distances are always between the original query and points.
 *   U_host  host [T][d] float32, the vectors u_t (unit length expected; used as given), copied
 * The reflection is evaluated in float32 in a fixed order, every multiply and add rounded on its
 * own: w2 = 2 * sum_j u_j x_j over j ascending, then x'_j = x_j - w2 * u_j.  A global variance
 * scope is not defined for reflected points (GF_EINVAL).  Other arguments and errors as gf_build_ex.
 */
int gf_build_reflected(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                       const gf_rand_params *rp, uint64_t seed, const float *U_host,
                       int32_t borrow_x, void *stream, gf_forest **out);

/* Give a forest (e.g. an imported one) per-tree Householder vectors, host [T][d] float32: from
 * now on its queries are reflected before descending.  Errors: GF_EINVAL (NaN/Inf), GF_ENOMEM. */
int gf_forest_set_reflections(gf_forest *F, const float *U_host);

/*
 * gf_forest_import -- make a forest from a given tree structure (used to query a forest built
 * elsewhere, e.g. by a CPU reference, with the GPU search).  split_dim_host / split_val_host are
 * host [T][2^L - 1], perm_host is host [T][n] with L = depth(n, leaf_size); X as in gf_build.
 * Errors: GF_EINVAL (a split dimension outside [0, d), a perm row that is not a permutation of
 * 0..n-1), GF_ENOMEM, GF_ECUDA.  Synchronous.
 */
int gf_forest_import(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                     const int32_t *split_dim_host, const float *split_val_host,
                     const int32_t *perm_host, gf_forest **out);

/* Copy the tree structure out to host arrays shaped as in gf_forest_import.  Synchronous. */
int gf_forest_export(const gf_forest *F, int32_t *split_dim_host, float *split_val_host,
                     int32_t *perm_host);

int gf_forest_get_info(const gf_forest *F, gf_forest_info *info);

/*
 * gf_forest_save -- write the forest to a file: its points, the split of every node and the leaf
 * order of every tree (Alg. 1's output), its Householder vectors (Sec. 2.2) if any, which
 * screening copies it holds and its tuning.  The file is written next to `path` and renamed onto
 * it once complete, so an existing file is replaced whole or not at all.
 * Layout (little-endian): a 128-byte header -- "GFFOREST", u32 version 1, u32 0x01020304, i64 n,
 * i32 d, T, leaf_size, L, u32 flags (1 reflections, 2 bf16 screen, 4 fp8 screen), i32 tuning
 * warps[3] ctas[3] rerank_R[3] rows_in_flight[3], u32 0, u64 payload bytes, u64 s1, u64 s2,
 * u64 0 -- then nodes [T][2^L - 1] x (i32 dim, f32 value), perm [T][n] i32, U [T][d] f32 (flag 1
 * only), X [n][d] f32.  s1 = sum w_i and s2 = sum (i + 1) w_i (mod 2^64), the w_i the u32 words of
 * header bytes 0..95 followed by those of the payload.
 * Errors: GF_EINVAL (null forest or empty path), GF_EIO (the file cannot be created or written;
 * no partial file is left), GF_ENOMEM, GF_ECUDA.  Synchronous.
 */
int gf_forest_save(const gf_forest *F, const char *path);

/*
 * gf_forest_load -- read a file written by gf_forest_save (or by any writer of the same layout)
 * into a new forest that answers every query exactly as the saved one did; screening copies are
 * derived again from X.  The whole file is read and checked on the host before the device is
 * touched.  Errors: GF_EINVAL (null argument), GF_EIO (missing or unreadable file, bad magic,
 * version, header or sizes, truncated or trailing bytes, checksum mismatch, a split dimension or
 * leaf order that is not valid, NaN/Inf in X or U), GF_ENOMEM, GF_ECUDA.  Synchronous.
 */
int gf_forest_load(const char *path, gf_forest **out);

/*
 * gf_forest_add_screen -- derive the low-precision copy of the points used by a screened
 * precision (Sec. 3 "Distance computation": ranking cost is the distance evaluation).
 *   GF_BF16_RERANK: xb[i][j] = bf16_rne(X[i][j])
 *   GF_FP8_RERANK:  a_i = max_j |X[i][j]|; scale_i = a_i / 448 (1 if a_i == 0);
 *                   x8[i][j] = e4m3_rne_satfinite(X[i][j] * (448 / a_i))  (0 if a_i == 0)
 * Synchronous.  Errors: GF_EINVAL, GF_ENOMEM, GF_ECUDA.
 */
int gf_forest_add_screen(gf_forest *F, int32_t precision, void *stream);

/* Set the forest's default kernel shape and shortlist for one precision (what the autotuner
 * writes); gf_query_ex uses them where its options hold 0.  rerank_R / rows_in_flight 0 keep the
 * current value.  Limits: 1 <= warps_per_cta <= 32, 0 <= ctas_per_sm <= 32, 0 <= rerank_R <= 2048,
 * rows_in_flight 0, 2 or 4 (else GF_EINVAL); forest files are held to the same limits. */
int gf_forest_set_tuning(gf_forest *F, int32_t precision, int32_t warps_per_cta,
                         int32_t ctas_per_sm, int32_t rerank_R, int32_t rows_in_flight);

int gf_forest_free(gf_forest *F);

/* ---------------------------------------------------------------- query (hot path) */

/*
 * gf_query -- k approximate nearest neighbours of m queries (Alg. 2 with one leaf per tree:
 * every query descends every tree to one leaf, Eq. 1; the points of the T leaves reached are
 * de-duplicated (Sec. 2.3 "seen" array), scored by squared L2 distance and the k nearest kept).
 *   Q      device [m][d] float32
 *   ids    device [m][k] int64: point ids ordered by (distance, id); -1 where a query has fewer
 *          than k candidates
 *   dists  device [m][k] float32: squared L2 distances (float32 arithmetic); +inf with id -1
 * With opts.checks = c > T (gf_query_ex) the search is Alg. 2 with the shared priority queue: after
 * the first leaf of every tree, nodes are taken from one queue over all trees in order of
 * (|q_s - v|, tree, node) and descended, until max(T, ceil(c / (1 + eps))) leaves were checked;
 * the points of all checked leaves are the candidates (at most 4096 leaves; needs T * 2^L <= 2^32).
 * Precision GF_FP32 on the legacy default stream.  m = 0 is a no-op.  Queries containing NaN give
 * unspecified ids but never read or write out of bounds.  The streaming kernel allocates its
 * scratch stream-ordered unless gf_query_ex is given a workspace.
 * Errors: GF_EINVAL (k < 1, m < 0, null pointers), GF_ECUDA.
 */
int gf_query(const gf_forest *F, const float *Q, int64_t m, int32_t k, int64_t *ids, float *dists);

/* As gf_query with options (precision, shortlist, kernel shape, stream).  The screened precisions
 * need gf_forest_add_screen first (else GF_EINVAL); their output distances are the float32 rerank
 * distances.  k must not exceed the shortlist R for screened precisions. */
int gf_query_ex(const gf_forest *F, const float *Q, int64_t m, int32_t k, const gf_query_opts *o,
                int64_t *ids, float *dists);

/* Bytes of device scratch a GF_ALGO_STREAM query of m rows needs with these options: one bitmap of
 * ceil(n / 32) words per CTA of the launch, plus 12 bytes per query when the batch is reordered
 * (GF_ORDER_*).  An upper bound for every k.  o may be NULL for the defaults. */
int gf_query_workspace_size(const gf_forest *F, int64_t m, const gf_query_opts *o, int64_t *bytes);

/* The first error a library kernel recorded on the current device since the last call, 0 if none
 * (a bounded wait that ran out records GF_ETIMEOUT); clears it.  Synchronizes the device.  The
 * paper has no counterpart.  Errors: GF_EINVAL (null pointer), GF_ECUDA. */
int gf_kernel_status(int32_t *status);

/* ---------------------------------------------------------------- query without allocation
 * gf_query_noalloc -- the query of gf_query_ex with GF_ALGO_STREAM, for callers that may not
 * allocate device memory while they run queries (a framework whose caching allocator must own
 * every device byte, a latency-critical loop that must stay out of the driver's allocator, a host
 * that fixes its memory at start-up).  The paper has no counterpart: its search is a single-threaded
 * CPU routine with no device memory at all.
 *
 * The kernel's scratch (one seen-bitmap of ceil(n / 32) 32-bit words per CTA) comes from a static
 * device array of GF_NOALLOC_SCRATCH_BYTES that is part of the library image: every GPU that loads
 * the library holds it until the process exits.  The queries run in consecutive launches, each of
 * as many rows as its whole scratch layout fits in the array (the bitmaps of its CTAs, plus 12 bytes
 * a query when the launch reorders its queries for locality), so a forest of more than
 * 8 * GF_NOALLOC_SCRATCH_BYTES points (536,870,912) is rejected with GF_EINVAL.  Arguments,
 * outputs and errors are those of gf_query_ex; precision and rerank_R as in gf_query_opts.
 *  - The first call on a device looks the array's device address up (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture on the device.  Under
 *    CUDA's lazy module loading that lookup is also when the driver loads the library's module on
 *    the device and sets the array aside: device free memory drops by GF_NOALLOC_SCRATCH_BYTES at
 *    the first call, and never during later calls.
 *  - The array is shared by every call in the process and keeps what the last call left in it;
 *    each call clears the part it uses before its kernels run.  Calls whose work overlaps on the GPU
 *    (on different streams, or from several threads) race on the array and give wrong answers:
 *    order them on one stream or synchronize between them.
 */
#define GF_NOALLOC_SCRATCH_BYTES (64ll << 20)

int gf_query_noalloc(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t precision,
                     int32_t rerank_R, void *stream, int64_t *ids, float *dists);

/* ---------------------------------------------------------------- the path in stages
 * The same computation as gf_query, one step per call, with the intermediate results in caller
 * buffers (used to check every step on its own).  All asynchronous on `stream`.
 */

/* Step 1 (Alg. 2 "descend", Eq. 1): leaf[i][t] = leaf of tree t reached by query i.
 * leaf: device [m][T] int32. */
int gf_descend(const gf_forest *F, const float *Q, int64_t m, int32_t *leaf, void *stream);

/* Step 2 (Sec. 2.3, "seen" array): the sorted union of the leaves' points of each query.
 * cand: device [m][cand_cap] int32 (cand_cap from gf_forest_get_info), row i holds ncand[i]
 * ascending ids followed by unspecified values; ncand: device [m] int32. */
int gf_candidates(const gf_forest *F, const int32_t *leaf, int64_t m, int32_t *cand, int32_t *ncand,
                  void *stream);

/* Steps 3-4 (Alg. 2 leaf check, squared L2, min-heap of k): float32 distances of each query's
 * candidates and the k smallest by (distance, id).  cand / ncand as produced by gf_candidates,
 * with row stride cand_stride >= max(ncand).  ids / dists as in gf_query. */
int gf_score_topk(const gf_forest *F, const float *Q, int64_t m, const int32_t *cand,
                  const int32_t *ncand, int32_t cand_stride, int32_t k, int64_t *ids,
                  float *dists, void *stream);

/* Step 3 alone, any precision (Sec. 3 "Distance computation"): dist[i][j] = squared L2 distance
 * of query i to candidate cand[i][j] for j < ncand[i], computed as the chosen precision's screen
 * computes it (GF_FP32: float32 points; GF_BF16_RERANK: bfloat16 points; GF_FP8_RERANK: scale_i
 * times the E4M3 codes), float32 arithmetic.  dist: device [m][cand_stride] float32; entries past
 * ncand[i] are left untouched; an id outside [0, n) gives NaN.  The screened precisions need
 * gf_forest_add_screen first (else GF_EINVAL). */
int gf_score_screened(const gf_forest *F, const float *Q, int64_t m, const int32_t *cand,
                      const int32_t *ncand, int32_t cand_stride, int32_t precision, float *dist,
                      void *stream);

/* ---------------------------------------------------------------- serving loop
 * Continuous batching of single-query requests over several resident forests (no counterpart in
 * the paper, whose search is one query at a time, Sec. 3 "Parallelization"; batched queries are
 * its stated future work, Sec. 5).
 *
 * A server owns `slots` batch slots, each with its own CUDA stream and every buffer a batch needs
 * (pinned staging, device queries/results, the streaming kernel's workspace), all reserved at
 * creation.  The number of slots is min(opts.slots, hbm_budget_bytes / bytes_per_slot): that is the
 * HBM admission rule -- a batch is dispatched exactly when a slot and its memory are free.  A
 * dispatcher thread takes up to max_batch requests of the forest whose oldest request waited
 * longest; batches on different slots overlap on the device; requests arriving meanwhile join the
 * next batch.  A batch runs the streaming kernel, whose answers equal gf_query on each query
 * alone (same kernel, same arithmetic), or -- when the server allows it and the batch is large
 * enough to share leaves -- the leaf-major path, whose answers are those of the same search within
 * the screens' tolerance (a screened score is computed in another form there).  The forests must
 * outlive the server and must not be freed while it runs.
 */
typedef struct gf_server gf_server;

typedef struct gf_server_opts {
    int32_t max_batch;         /* requests per batch (default 1024) */
    int32_t slots;             /* batch slots, i.e. batches in flight at most (default 4) */
    int64_t hbm_budget_bytes;  /* device memory the slots may reserve (default 4 GiB) */
    int32_t k_max;             /* largest k a request may ask for (default 10) */
    int32_t precision;         /* GF_FP32 / GF_BF16_RERANK / GF_FP8_RERANK for every batch */
    int32_t rerank_R;          /* shortlist for the screened precisions (0 = forest default) */
    int32_t checks;            /* leaf checks c of every batch (gf_query_opts.checks) */
    double eps;                /* gf_query_opts.eps */
    int32_t algo;              /* GF_ALGO_AUTO (default): a batch that shares leaves enough (the rule
                                  of GF_ALGO_AUTO) runs the leaf-major path, any other the streaming
                                  kernel; GF_ALGO_STREAM: the streaming kernel always */
} gf_server_opts;

typedef struct gf_server_stats {
    int64_t completed;    /* requests finished since the last reset */
    int64_t batches;      /* batches launched */
    double mean_batch;    /* requests per batch */
    double p50_ms;        /* latency, submission to completion */
    double p99_ms;
    double max_ms;
    double span_s;        /* first submission to last completion */
    double qps;           /* completed / span_s */
    int32_t slots;
    int32_t leaf_batches; /* batches that ran the leaf-major path (capped at INT32_MAX) */
} gf_server_stats;

void gf_server_opts_default(gf_server_opts *o);

/* Errors: GF_EINVAL (no forests, a forest without the screening copy `precision` needs, bad
 * options), GF_ENOMEM (the budget holds no slot, or an allocation failed), GF_ECUDA. */
int gf_server_create(gf_forest *const *forests, int32_t nforests, const gf_server_opts *opts,
                     gf_server **out);
int gf_server_slots(const gf_server *S);

/* Queue one query (host [d] float32 of the forest's d, copied) for forest index `forest` with
 * 1 <= k <= k_max; *ticket identifies it.  Thread-safe, non-blocking. */
int gf_server_submit(gf_server *S, int32_t forest, const float *q_host, int32_t k, uint64_t *ticket);

/* Wait up to timeout_us for a request; on completion copy its k ids / distances to host buffers
 * (either may be NULL) and forget the ticket.  GF_ETIMEOUT if it has not finished by then (the
 * ticket stays valid); the request's own error code if its batch failed. */
int gf_server_poll(gf_server *S, uint64_t ticket, int64_t *ids_host, float *dists_host,
                   int32_t timeout_us);

int gf_server_get_stats(gf_server *S, gf_server_stats *st);
int gf_server_reset_stats(gf_server *S);

/* Open-loop load for measurement: Poisson arrivals at rate_qps for duration_s seconds, each for a
 * forest drawn uniformly, queries taken in turn from queries_host[f] (host [nq[f]][d_f]); waits up
 * to timeout_ms per request, then fills st. */
int gf_server_run_poisson(gf_server *S, const float *const *queries_host, const int64_t *nq,
                          double rate_qps, double duration_s, int32_t k, uint64_t seed,
                          int32_t timeout_ms, gf_server_stats *st);

/* Stop the threads after the batches in flight finish, free the slots.  Pending tickets die. */
int gf_server_destroy(gf_server *S);

/* The leaves Alg. 2's priority search checks for each query (the first step of gf_query_ex with
 * opts.checks = c), in the order it checks them: the first leaf of every tree, then leaves taken
 * from the shared queue by (|q_s - v|, tree, node).  leaves: device [m][stride] uint32, each
 * (tree << L) | leaf; nleaves: device [m] int32, the number checked (fewer than stride only when
 * the queue runs dry).  stride must equal the leaf budget max(T, ceil(c / (1 + eps))) (<= 4096).
 * Errors: GF_EINVAL, GF_EUNSUPPORTED (T * 2^L > 2^32, budget above 4096). */
int gf_prio_leaves(const gf_forest *F, const float *Q, int64_t m, int32_t checks, double eps,
                   uint32_t *leaves, int32_t *nleaves, int32_t stride, void *stream);

/* ---------------------------------------------------------------- failure injection (tests)
 * Hooks that make the library's failure paths run on purpose, for tests of its error handling
 * without a device fault.  The paper has no counterpart.  Both settings are process-wide and apply
 * to calls made after them.
 */

/* The (after + 1)-th device allocation the library makes from now on fails as if the device had no
 * memory left: the call that made it returns GF_ENOMEM after releasing what it had allocated (a
 * failed build leaves no forest, *out stays NULL).  One failure, then the hook disarms itself;
 * after < 0 disarms it at once.  Counts the allocations of forest storage and build scratch
 * (gf_build*, gf_forest_import, gf_forest_load, gf_forest_add_screen, gf_forest_set_reflections).
 * Errors: none (GF_OK). */
int gf_debug_fail_alloc(int32_t after);

/* Time limit, in nanoseconds, of the waits of the leaf-major tensor-core scoring kernel's pipeline
 * (0: the default, about two seconds).  A wait that runs out records GF_ETIMEOUT for
 * gf_kernel_status; every role of the kernel then leaves its loop, its copies and tensor-core
 * operations are drained (under the default limit, whatever this one) and its tensor memory freed.
 * The results of a query whose kernel gave up are unspecified, but its reads and writes stay in
 * bounds.  A limit of a few hundred nanoseconds makes the waits run out.  Errors: none (GF_OK). */
int gf_debug_set_wait_limit(uint64_t ns);

/* ---------------------------------------------------------------- misc */

const char *gf_last_error(void);
int32_t gf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GF_H */
