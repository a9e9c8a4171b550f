/*
 * gf_oracle.c -- plain, slow CPU oracle for the kd-GeRaF forest search
 * (Avrithis, Emiris, Samaras, "High-dimensional approximate nearest neighbor: k-d Generalized
 * Randomized Forests", arXiv 1603.09596).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and the benchmark's
 * CPU-baseline leg load this library.  The CUDA library never links, loads or calls it, and the two
 * share no source: this file includes only the C standard library.
 *
 * Arithmetic.  Inputs are float32; every variance and every distance is computed in double
 * precision on the exactly promoted inputs.  Compile with -ffp-contract=off so that no
 * multiply-add is fused and results are identical on every host.
 *
 * Readings of the paper that this oracle fixes (each one is repeated where it is used):
 *  R1  Perfect trees (Sec. 3 "Tree structure"): depth L = min{l >= 0 : ceil(n / 2^l) <= p}; the node
 *      at depth l with in-level index a owns sequence positions [floor(a n / 2^l), floor((a+1) n / 2^l)).
 *      Heap numbering: node j has children 2j+1 and 2j+2; the internal nodes of a tree are
 *      0 .. 2^L - 2 and leaf b (0 <= b < 2^L) owns [floor(b n / 2^L), floor((b+1) n / 2^L)).
 *  R2  Shuffling (Sec. 2.1 "Shuffling") only decides how equal coordinates are ordered.  Each tree
 *      gets a pseudo-random order of the point ids, rk_t(i) = fmix32(i XOR key_t), a bijection on
 *      32-bit integers; ties in the split coordinate are broken by rk_t.  The sequence a node is
 *      built from starts as the ids 0..n-1 in ascending order and every split is a stable
 *      partition, so every node (and leaf) lists its points in ascending id order.
 *  R3  Variance (Alg. 3) over the node's points in that order ("per-node" scope), or once over all
 *      of X (Alg. 1 literal, "global" scope).
 *  R4  Split dimension (Sec. 2.1 "Split dimension", Alg. 1): dimensions ranked by (variance
 *      descending, index ascending); s = D[u mod t] with u the node's SplitMix64 draw.
 *  R5  Median split (Alg. 1, Sec. 3 "Median, variances"): order the node's points by the key
 *      (x_s, rk_t(i)) with -0.0 read as +0.0; the left child takes the first h points, where h is
 *      fixed by R1; the split value v is x_s of the first right point (no rounding), or +inf
 *      when the right child is empty (possible only with leaf_size 1).
 *  R6  Descent (Alg. 2 "descend", Eq. 1): signed distance d = q_s - v; d < 0 goes left, otherwise
 *      right.  Evaluated as the comparison q_s < v, which has the same sign without rounding.
 *  R7  Search with one leaf per tree (c = T, no priority queue): candidates are the sorted union
 *      of the leaves reached in all trees, each point scored once ("seen" array, Sec. 2.3);
 *      k results ordered by (distance, id); missing results padded with id -1, distance +inf.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) and the MurmurHash3 32-bit
 * finalizer fmix32 (Appleby), both written here from their published definitions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ random numbers */

/* SplitMix64: state advances by the golden gamma; the output mixes the state. */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 stream whose state starts at s0. */
uint64_t gfo_splitmix64_at(uint64_t s0, uint64_t i) {
    return sm64_mix(s0 + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

/* MurmurHash3 fmix32: a bijection on 32-bit integers. */
uint32_t gfo_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6BU;
    h ^= h >> 13;
    h *= 0xC2B2AE35U;
    h ^= h >> 16;
    return h;
}

/* Key of tree t: output t of the stream seeded with the forest seed. */
uint64_t gfo_tree_key(uint64_t seed, int32_t t) { return gfo_splitmix64_at(seed, (uint64_t)t); }

/* Tie-break order of point i in tree t (R2).  Without shuffling it is the id itself. */
uint32_t gfo_rank(uint64_t seed, int32_t t, int32_t shuffle, uint32_t i) {
    if (!shuffle) return i;
    uint32_t key = (uint32_t)gfo_splitmix64_at(gfo_tree_key(seed, t), 0);
    return gfo_fmix32(i ^ key);
}

/* Random draw of internal node j (heap index) of tree t (R4): output j+1 of the tree's stream. */
uint64_t gfo_node_draw(uint64_t seed, int32_t t, int64_t j) {
    return gfo_splitmix64_at(gfo_tree_key(seed, t), (uint64_t)j + 1);
}

/* ------------------------------------------------------------------ tree shape (R1) */

int32_t gfo_depth(int64_t n, int32_t p) {
    int32_t L = 0;
    if (n < 1 || p < 1) return -1;
    /* ceil(n / 2^L) <= p */
    while (((n + ((int64_t)1 << L) - 1) >> L) > p) L++;
    return L;
}

/* First sequence position owned by node a (in-level index) at depth l. */
static int64_t pos_of(int64_t n, int32_t l, int64_t a) {
    return (int64_t)(((__int128)a * n) >> l);
}

/* ------------------------------------------------------------------ Householder reflection */

/*
 * Sec. 2.2: the reflection of x across the hyperplane normal to u is Px = x - 2 (u^T x) u.  Here
 * u is taken as given (a unit vector is expected).  Reading: the reflection only shapes the trees,
 * so it is evaluated in float32 with a fixed order -- w = u^T x summed over j ascending, then each
 * coordinate x_j - (2w) u_j -- every multiply and add rounded on its own (this file is compiled
 * without fused multiply-add).
 */
void gfo_reflect(const float *x, const float *u, int32_t d, float *out) {
    float w = 0.0f;
    for (int32_t j = 0; j < d; j++) w = w + u[j] * x[j];
    const float w2 = 2.0f * w;
    for (int32_t j = 0; j < d; j++) out[j] = x[j] - w2 * u[j];
}

/* ------------------------------------------------------------------ Alg. 3 variance */

/*
 * Modified Knuth online variance (Alg. 3, Sec. 3 "Median, variances"), run on the sequence of
 * rows X[idx[0]], ..., X[idx[cnt-1]] and on all d coordinates at once, in double precision:
 *   alpha = 1/i; delta = x_i - mu; mu += alpha * delta; v += delta o (x_i - mu);  return v / (cnt-1).
 * A sequence of fewer than two vectors has variance zero.
 */
void gfo_variance(const float *X, int32_t d, const int32_t *idx, int64_t cnt, double *var) {
    double *mu = (double *)calloc((size_t)d, sizeof(double));
    memset(var, 0, sizeof(double) * (size_t)d);
    if (cnt >= 2) {
        for (int64_t i = 1; i <= cnt; i++) {
            const float *x = X + (int64_t)idx[i - 1] * d;
            double alpha = 1.0 / (double)i;
            for (int32_t j = 0; j < d; j++) {
                double xi = (double)x[j];
                double delta = xi - mu[j];
                mu[j] = mu[j] + alpha * delta;
                var[j] = var[j] + delta * (xi - mu[j]);
            }
        }
        for (int32_t j = 0; j < d; j++) var[j] = var[j] / (double)(cnt - 1);
    }
    free(mu);
}

/* ------------------------------------------------------------------ split-dimension choice */

/* The t dimensions of largest variance, ranked by (variance descending, index ascending) (R4). */
void gfo_top_dims(const double *var, int32_t d, int32_t t, int32_t *D) {
    char *taken = (char *)calloc((size_t)d, 1);
    for (int32_t r = 0; r < t; r++) {
        int32_t best = -1;
        for (int32_t j = 0; j < d; j++) {
            if (taken[j]) continue;
            if (best < 0 || var[j] > var[best]) best = j;
        }
        taken[best] = 1;
        D[r] = best;
    }
    free(taken);
}

/* ------------------------------------------------------------------ median split (R5) */

static float canon(float x) { return x == 0.0f ? 0.0f : x; } /* -0.0 reads as +0.0 */

typedef struct {
    float x;       /* split coordinate of the point */
    uint32_t rk;   /* tie-break order */
    int32_t id;    /* point id */
} key_t_;

static int key_cmp(const void *pa, const void *pb) {
    const key_t_ *a = (const key_t_ *)pa, *b = (const key_t_ *)pb;
    if (a->x < b->x) return -1;
    if (a->x > b->x) return 1;
    if (a->rk < b->rk) return -1;
    if (a->rk > b->rk) return 1;
    return 0;
}

/*
 * Split the sequence seq[0..cnt) on coordinate s: the h points of smallest key (x_s, rk) form the
 * left child.  On return seq holds the left points followed by the right points, each group in its
 * previous relative order (stable partition), and the split value is returned.
 */
static float split_node(const float *X, int32_t d, int32_t *seq, int64_t cnt, int64_t h, int32_t s,
                        uint64_t seed, int32_t tree, int32_t shuffle) {
    key_t_ *k = (key_t_ *)malloc(sizeof(key_t_) * (size_t)cnt);
    for (int64_t i = 0; i < cnt; i++) {
        k[i].x = canon(X[(int64_t)seq[i] * d + s]);
        k[i].rk = gfo_rank(seed, tree, shuffle, (uint32_t)seq[i]);
        k[i].id = seq[i];
    }
    qsort(k, (size_t)cnt, sizeof(key_t_), key_cmp);
    /* With leaf_size 1 the perfect shape can leave the right child empty (h == cnt); the split
     * value is then +inf, so every point and every finite query goes left. */
    key_t_ first_right = {INFINITY, 0, -1};
    if (h < cnt) first_right = k[h];
    float v = first_right.x;
    /* a point goes left iff its key is below the key of the first right point */
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)cnt);
    int64_t nl = 0, nr = 0;
    for (int64_t i = 0; i < cnt; i++) {
        key_t_ ki = {canon(X[(int64_t)seq[i] * d + s]), gfo_rank(seed, tree, shuffle, (uint32_t)seq[i]), seq[i]};
        if (key_cmp(&ki, &first_right) < 0) tmp[nl++] = seq[i];
    }
    for (int64_t i = 0; i < cnt; i++) {
        key_t_ ki = {canon(X[(int64_t)seq[i] * d + s]), gfo_rank(seed, tree, shuffle, (uint32_t)seq[i]), seq[i]};
        if (key_cmp(&ki, &first_right) >= 0) tmp[nl + nr++] = seq[i];
    }
    memcpy(seq, tmp, sizeof(int32_t) * (size_t)cnt);
    free(tmp);
    free(k);
    return v;
}

/* ------------------------------------------------------------------ Alg. 1 build */

typedef struct {
    const float *X;
    int64_t n;
    int32_t d, L, t, shuffle, var_scope, tree;
    uint64_t seed;
    const int32_t *Dglob;  /* global top-t dims (var_scope == 1) */
    int32_t *split_dim;    /* [2^L - 1] of this tree */
    float *split_val;
    int32_t *seq;          /* [n]: the tree's point sequence, becomes the leaf permutation */
    double *var;           /* [d] scratch */
    int32_t *D;            /* [t] scratch */
} build_ctx;

/* Recursive build of node (depth l, in-level index a) -- Alg. 1 "build". */
static void build_node(build_ctx *c, int32_t l, int64_t a) {
    if (l == c->L) return; /* leaf: |X| <= p by the choice of L (R1) */
    int64_t lo = pos_of(c->n, l, a), hi = pos_of(c->n, l, a + 1);
    int64_t mid = pos_of(c->n, l + 1, 2 * a + 1);
    int64_t j = ((int64_t)1 << l) - 1 + a; /* heap index */
    const int32_t *D = c->Dglob;
    if (c->var_scope == 0) { /* variance of the node's own points (R3) */
        gfo_variance(c->X, c->d, c->seq + lo, hi - lo, c->var);
        gfo_top_dims(c->var, c->d, c->t, c->D);
        D = c->D;
    }
    int32_t s = D[gfo_node_draw(c->seed, c->tree, j) % (uint64_t)c->t];
    float v = split_node(c->X, c->d, c->seq + lo, hi - lo, mid - lo, s, c->seed, c->tree, c->shuffle);
    c->split_dim[j] = s;
    c->split_val[j] = v;
    build_node(c, l + 1, 2 * a);
    build_node(c, l + 1, 2 * a + 1);
}

/*
 * Build a forest of T trees (Alg. 1).  Outputs, caller-allocated:
 *   split_dim [T][2^L - 1], split_val [T][2^L - 1], perm [T][n]   (L = gfo_depth(n, p)).
 * Trees are independent and built one per thread (Sec. 3 "Parallelization").
 * Returns L, or -1 on invalid arguments.
 */
int32_t gfo_build_reflected(const float *X, int64_t n, int32_t d, int32_t T, int32_t p, int32_t t,
                            int32_t shuffle, int32_t var_scope, uint64_t seed, const float *U,
                            int32_t *split_dim, float *split_val, int32_t *perm);

int32_t gfo_build(const float *X, int64_t n, int32_t d, int32_t T, int32_t p, int32_t t,
                  int32_t shuffle, int32_t var_scope, uint64_t seed, int32_t *split_dim,
                  float *split_val, int32_t *perm) {
    return gfo_build_reflected(X, n, d, T, p, t, shuffle, var_scope, seed, NULL, split_dim, split_val, perm);
}

/* As gfo_build; with U (T x d) every tree is built on its own reflected points P_t X (Sec. 2.2:
 * "build on transformed X, store f"). */
int32_t gfo_build_reflected(const float *X, int64_t n, int32_t d, int32_t T, int32_t p, int32_t t,
                            int32_t shuffle, int32_t var_scope, uint64_t seed, const float *U,
                            int32_t *split_dim, float *split_val, int32_t *perm) {
    if (!X || n < 1 || d < 1 || T < 1 || p < 1 || t < 1 || t > d || n > 0x7FFFFFFFLL) return -1;
    int32_t L = gfo_depth(n, p);
    int64_t nn = ((int64_t)1 << L) - 1;
    int32_t *Dglob = (int32_t *)malloc(sizeof(int32_t) * (size_t)t);
    if (var_scope == 1 && U) return -1; /* a global ranking of reflected coordinates is per tree */
    if (var_scope == 1) { /* Alg. 1 literal: V and D computed once for the input set */
        int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        double *var = (double *)malloc(sizeof(double) * (size_t)d);
        for (int64_t i = 0; i < n; i++) ids[i] = (int32_t)i;
        gfo_variance(X, d, ids, n, var);
        gfo_top_dims(var, d, t, Dglob);
        free(var);
        free(ids);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t tr = 0; tr < T; tr++) {
        build_ctx c;
        float *Xt = NULL;
        if (U) { /* this tree's reflected points */
            Xt = (float *)malloc(sizeof(float) * (size_t)n * (size_t)d);
            for (int64_t i = 0; i < n; i++) gfo_reflect(X + i * d, U + (int64_t)tr * d, d, Xt + i * d);
        }
        c.X = U ? Xt : X; c.n = n; c.d = d; c.L = L; c.t = t; c.shuffle = shuffle; c.var_scope = var_scope;
        c.tree = tr; c.seed = seed; c.Dglob = Dglob;
        c.split_dim = split_dim + (int64_t)tr * nn;
        c.split_val = split_val + (int64_t)tr * nn;
        c.seq = perm + (int64_t)tr * n;
        for (int64_t i = 0; i < n; i++) c.seq[i] = (int32_t)i; /* R2: ascending ids */
        c.var = (double *)malloc(sizeof(double) * (size_t)d);
        c.D = (int32_t *)malloc(sizeof(int32_t) * (size_t)t);
        build_node(&c, 0, 0);
        free(c.var);
        free(c.D);
        free(Xt);
    }
    free(Dglob);
    return L;
}

/* ------------------------------------------------------------------ Alg. 2 descent */

/* Leaf reached by q in one tree (Alg. 2 "descend", Eq. 1, R6).  Returns the leaf index b. */
int64_t gfo_descend_one(const int32_t *split_dim, const float *split_val, int32_t L, const float *q) {
    int64_t j = 0;
    for (int32_t l = 0; l < L; l++) {
        int32_t s = split_dim[j];
        float v = split_val[j];
        if (q[s] < v) j = 2 * j + 1; /* d = q_s - v < 0: left */
        else j = 2 * j + 2;          /* otherwise right */
    }
    return j - (((int64_t)1 << L) - 1);
}

/* The query a tree's descent sees: q itself, or its reflection P_t q when the forest has U (the
 * query is reflected before descending, Sec. 2.3; distances still use q). */
static const float *tree_query(const float *q, const float *U, int32_t t, int32_t d, float *buf) {
    if (!U) return q;
    gfo_reflect(q, U + (int64_t)t * d, d, buf);
    return buf;
}

/* leaf[i][t] for every query i and tree t. */
void gfo_descend_reflected(const int32_t *split_dim, const float *split_val, int32_t L, int32_t T,
                           const float *Q, int64_t m, int32_t d, const float *U, int32_t *leaf) {
    int64_t nn = ((int64_t)1 << L) - 1;
#pragma omp parallel
    {
        float *buf = (float *)malloc(sizeof(float) * (size_t)d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; i++)
            for (int32_t t = 0; t < T; t++)
                leaf[i * T + t] = (int32_t)gfo_descend_one(split_dim + t * nn, split_val + t * nn, L,
                                                           tree_query(Q + i * d, U, t, d, buf));
        free(buf);
    }
}

void gfo_descend(const int32_t *split_dim, const float *split_val, int32_t L, int32_t T,
                 const float *Q, int64_t m, int32_t d, int32_t *leaf) {
    gfo_descend_reflected(split_dim, split_val, L, T, Q, m, d, NULL, leaf);
}

/* ------------------------------------------------------------------ candidates (R7) */

static int int_cmp(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Candidates of one query: the points of the T leaves it reached, each listed once, ascending.
 * Writes them to out (capacity >= sum of leaf sizes) and returns their number.
 */
int64_t gfo_candidates_one(const int32_t *perm, int64_t n, int32_t L, int32_t T, const int32_t *leaf,
                           int32_t *out) {
    int64_t c = 0;
    for (int32_t t = 0; t < T; t++) {
        int64_t lo = pos_of(n, L, leaf[t]), hi = pos_of(n, L, (int64_t)leaf[t] + 1);
        for (int64_t p = lo; p < hi; p++) out[c++] = perm[(int64_t)t * n + p];
    }
    qsort(out, (size_t)c, sizeof(int32_t), int_cmp);
    int64_t u = 0;
    for (int64_t i = 0; i < c; i++)
        if (u == 0 || out[i] != out[u - 1]) out[u++] = out[i];
    return u;
}

/* Candidate sets of m queries in CSR form: offs[m+1], ids[offs[i] .. offs[i+1]). */
int64_t gfo_candidates(const int32_t *perm, int64_t n, int32_t L, int32_t T, const int32_t *leaf,
                       int64_t m, int64_t *offs, int32_t *ids) {
    int64_t cap = (n + ((int64_t)1 << L) - 1) >> L; /* largest leaf */
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap * T));
    offs[0] = 0;
    for (int64_t i = 0; i < m; i++) {
        int64_t c = gfo_candidates_one(perm, n, L, T, leaf + i * T, tmp);
        memcpy(ids + offs[i], tmp, sizeof(int32_t) * (size_t)c);
        offs[i + 1] = offs[i] + c;
    }
    free(tmp);
    return offs[m];
}

/* ------------------------------------------------------------------ distances and top-k */

/* Squared Euclidean distance ||q - x||^2 in double precision (Alg. 2 leaf check). */
double gfo_dist2(const float *q, const float *x, int32_t d) {
    double s = 0.0;
    for (int32_t j = 0; j < d; j++) {
        double e = (double)q[j] - (double)x[j];
        s += e * e;
    }
    return s;
}

typedef struct {
    double dist;
    int64_t id;
} res_t;

static int res_cmp(const void *pa, const void *pb) {
    const res_t *a = (const res_t *)pa, *b = (const res_t *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* The k results of smallest (distance, id) among cnt scored points; pads with (-1, +inf). */
static void take_k(res_t *r, int64_t cnt, int32_t k, int64_t *out_ids, double *out_d) {
    qsort(r, (size_t)cnt, sizeof(res_t), res_cmp);
    for (int32_t i = 0; i < k; i++) {
        if (i < cnt) { out_ids[i] = r[i].id; out_d[i] = r[i].dist; }
        else { out_ids[i] = -1; out_d[i] = INFINITY; }
    }
}

/* Score every candidate of every query and keep the k nearest (R7). */
void gfo_topk(const float *X, int32_t d, const float *Q, int64_t m, const int64_t *offs,
              const int32_t *ids, int32_t k, int64_t *out_ids, double *out_d) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < m; i++) {
        int64_t c = offs[i + 1] - offs[i];
        res_t *r = (res_t *)malloc(sizeof(res_t) * (size_t)(c > 0 ? c : 1));
        for (int64_t j = 0; j < c; j++) {
            int64_t id = ids[offs[i] + j];
            r[j].id = id;
            r[j].dist = gfo_dist2(Q + i * d, X + id * d, d);
        }
        take_k(r, c, k, out_ids + i * k, out_d + i * k);
        free(r);
    }
}

/*
 * The whole search for m queries (Alg. 2 with c = T, R7): descend every tree, gather and
 * de-duplicate the leaf points, score them, keep the k nearest.  Queries run in parallel.
 * If ncand is not NULL it receives each query's candidate count.
 */
void gfo_search_reflected(const float *X, int64_t n, int32_t d, const int32_t *split_dim,
                          const float *split_val, const int32_t *perm, int32_t L, int32_t T,
                          const float *Q, int64_t m, int32_t k, const float *U, int64_t *out_ids,
                          double *out_d, int64_t *ncand);

void gfo_search(const float *X, int64_t n, int32_t d, const int32_t *split_dim,
                const float *split_val, const int32_t *perm, int32_t L, int32_t T, const float *Q,
                int64_t m, int32_t k, int64_t *out_ids, double *out_d, int64_t *ncand) {
    gfo_search_reflected(X, n, d, split_dim, split_val, perm, L, T, Q, m, k, NULL, out_ids, out_d, ncand);
}

void gfo_search_reflected(const float *X, int64_t n, int32_t d, const int32_t *split_dim,
                          const float *split_val, const int32_t *perm, int32_t L, int32_t T,
                          const float *Q, int64_t m, int32_t k, const float *U, int64_t *out_ids,
                          double *out_d, int64_t *ncand) {
    int64_t nn = ((int64_t)1 << L) - 1;
    int64_t cap = ((n + ((int64_t)1 << L) - 1) >> L) * T;
#pragma omp parallel
    {
        int32_t *leaf = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
        int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
        res_t *r = (res_t *)malloc(sizeof(res_t) * (size_t)cap);
        float *qbuf = (float *)malloc(sizeof(float) * (size_t)d);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < m; i++) {
            const float *q = Q + i * d;
            for (int32_t t = 0; t < T; t++)
                leaf[t] = (int32_t)gfo_descend_one(split_dim + t * nn, split_val + t * nn, L,
                                                   tree_query(q, U, t, d, qbuf));
            int64_t c = gfo_candidates_one(perm, n, L, T, leaf, cand);
            for (int64_t j = 0; j < c; j++) {
                r[j].id = cand[j];
                r[j].dist = gfo_dist2(q, X + (int64_t)cand[j] * d, d);
            }
            take_k(r, c, k, out_ids + i * k, out_d + i * k);
            if (ncand) ncand[i] = c;
        }
        free(leaf);
        free(cand);
        free(r);
        free(qbuf);
    }
}

/*
 * The same search (Alg. 2 with c = T) with every distance in float32 arithmetic, a plain sequential
 * loop: the CPU baseline of what a float32 search costs on the host, timed beside the float64
 * search.  Not used as a reference for any result.  Its distances differ from gfo_dist2's by at
 * most (d + 2) 2^-24 relative (a sum of d non-negative rounded terms, each rounded twice).
 */
static float dist2_f32(const float *q, const float *x, int32_t d) {
    float s = 0.0f;
    for (int32_t j = 0; j < d; j++) {
        float e = q[j] - x[j];
        s += e * e;
    }
    return s;
}

void gfo_search_f32(const float *X, int64_t n, int32_t d, const int32_t *split_dim,
                    const float *split_val, const int32_t *perm, int32_t L, int32_t T, const float *Q,
                    int64_t m, int32_t k, int64_t *out_ids, double *out_d) {
    int64_t nn = ((int64_t)1 << L) - 1;
    int64_t cap = ((n + ((int64_t)1 << L) - 1) >> L) * T;
#pragma omp parallel
    {
        int32_t *leaf = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
        int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
        res_t *r = (res_t *)malloc(sizeof(res_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < m; i++) {
            const float *q = Q + i * d;
            for (int32_t t = 0; t < T; t++)
                leaf[t] = (int32_t)gfo_descend_one(split_dim + t * nn, split_val + t * nn, L, q);
            int64_t c = gfo_candidates_one(perm, n, L, T, leaf, cand);
            for (int64_t j = 0; j < c; j++) {
                r[j].id = cand[j];
                r[j].dist = (double)dist2_f32(q, X + (int64_t)cand[j] * d, d);
            }
            take_k(r, c, k, out_ids + i * k, out_d + i * k);
        }
        free(leaf);
        free(cand);
        free(r);
    }
}

/* ------------------------------------------------------------------ Alg. 2 priority search */

/*
 * Alg. 2 with the shared min-priority queue Q over all trees (Sec. 2.3).  Each descent from a node
 * to a leaf pushes, at every internal node passed, the child not taken with key |q_s - v| (Eq. 1);
 * the leaf reached is checked: its points not seen before get their distance and enter the
 * k-best list H.  Reading R8: the first descent of every tree checks its leaf too and counts as a
 * checked leaf (with c = T the search is exactly R7); afterwards nodes are extracted from Q in
 * order of (key, tree, node) and descended while fewer than c / (1 + eps) leaves were checked.
 * If leaf_seq is not NULL, row i receives the first seq_cap leaves checked, as (tree << L) | leaf.
 */
typedef struct {
    double key;
    int32_t tree;
    int64_t node;
} qent_t;

static int qent_less(const qent_t *a, const qent_t *b) {
    if (a->key != b->key) return a->key < b->key;
    if (a->tree != b->tree) return a->tree < b->tree;
    return a->node < b->node;
}

static void heap_push(qent_t *h, int64_t *sz, qent_t e) {
    int64_t i = (*sz)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!qent_less(&h[i], &h[p])) break;
        qent_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static qent_t heap_pop(qent_t *h, int64_t *sz) {
    qent_t top = h[0];
    h[0] = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *sz && qent_less(&h[l], &h[b])) b = l;
        if (r < *sz && qent_less(&h[r], &h[b])) b = r;
        if (b == i) break;
        qent_t t = h[i]; h[i] = h[b]; h[b] = t;
        i = b;
    }
    return top;
}

typedef struct {
    res_t *best;   /* k best so far, sorted by (dist, id) */
    int32_t nb, k;
} kbest_t;

static void kbest_insert(kbest_t *H, res_t r) {
    if (H->nb == H->k && res_cmp(&r, &H->best[H->k - 1]) >= 0) return;
    int32_t pos = H->nb < H->k ? H->nb++ : H->k - 1;
    while (pos > 0 && res_cmp(&r, &H->best[pos - 1]) < 0) { H->best[pos] = H->best[pos - 1]; pos--; }
    H->best[pos] = r;
}

void gfo_search_priority(const float *X, int64_t n, int32_t d, const int32_t *split_dim,
                         const float *split_val, const int32_t *perm, int32_t L, int32_t T,
                         const float *Q, int64_t m, int32_t k, int64_t c, double eps,
                         int64_t *out_ids, double *out_d, int64_t *ncand, int64_t *nleaves,
                         int64_t *leaf_seq, int64_t seq_cap, const float *U) {
    int64_t nn = ((int64_t)1 << L) - 1;
    double budget = (double)c / (1.0 + eps);
#pragma omp parallel
    {
        unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
        int64_t hcap = (int64_t)T * (L + 1) + (int64_t)(budget + T + 1) * (L + 1) + 16;
        qent_t *heap = (qent_t *)malloc(sizeof(qent_t) * (size_t)hcap);
        res_t *best = (res_t *)malloc(sizeof(res_t) * (size_t)k);
        int32_t *touched = NULL;
        int64_t tcap = 0;
        float *qt = U ? (float *)malloc(sizeof(float) * (size_t)T * (size_t)d) : NULL;
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < m; i++) {
            const float *q = Q + i * d;
            if (U) /* every tree's reflection of the query, for its descents (Sec. 2.3) */
                for (int32_t t = 0; t < T; t++) gfo_reflect(q, U + (int64_t)t * d, d, qt + (int64_t)t * d);
            int64_t hs = 0, checked = 0, nc = 0, ntouch = 0;
            kbest_t H = {best, 0, k};
            /* one descent from node j of tree t to a leaf, pushing the siblings, checking the leaf */
#define GFO_DESCEND(t_, j_)                                                                        \
            do {                                                                                   \
                const int32_t tree_ = (t_);   /* arguments evaluated once, before any push */     \
                int64_t j = (j_);                                                                  \
                const int32_t *sd = split_dim + (int64_t)tree_ * nn;                               \
                const float *sv = split_val + (int64_t)tree_ * nn;                                 \
                const float *qd = U ? qt + (int64_t)tree_ * d : q;                                 \
                while (j < nn) {                                                                   \
                    double dd = (double)qd[sd[j]] - (double)sv[j];                                 \
                    qent_t pushed_;                                                                \
                    pushed_.key = fabs(dd);                                                        \
                    pushed_.tree = tree_;                                                          \
                    if (qd[sd[j]] < sv[j]) { pushed_.node = 2 * j + 2; j = 2 * j + 1; }            \
                    else { pushed_.node = 2 * j + 1; j = 2 * j + 2; }                              \
                    heap_push(heap, &hs, pushed_);                                                 \
                }                                                                                  \
                int64_t b = j - nn;                                                                \
                if (leaf_seq && checked < seq_cap)                                                 \
                    leaf_seq[i * seq_cap + checked] = ((int64_t)tree_ << L) | b;                   \
                int64_t lo = pos_of(n, L, b), hi = pos_of(n, L, b + 1);                            \
                for (int64_t p = lo; p < hi; p++) {                                                \
                    int32_t id = perm[(int64_t)tree_ * n + p];                                     \
                    if (seen[id]) continue;                                                        \
                    seen[id] = 1;                                                                  \
                    if (ntouch == tcap) {                                                          \
                        tcap = tcap ? 2 * tcap : 4096;                                             \
                        touched = (int32_t *)realloc(touched, sizeof(int32_t) * (size_t)tcap);     \
                    }                                                                              \
                    touched[ntouch++] = id;                                                        \
                    res_t r = {gfo_dist2(q, X + (int64_t)id * d, d), id};                          \
                    kbest_insert(&H, r);                                                           \
                    nc++;                                                                          \
                }                                                                                  \
                checked++;                                                                         \
            } while (0)
            for (int32_t t = 0; t < T; t++) GFO_DESCEND(t, 0);
            while (hs > 0 && (double)checked < budget) {
                if (hs + L + 1 > hcap) break;
                const qent_t top = heap_pop(heap, &hs);
                GFO_DESCEND(top.tree, top.node);
            }
#undef GFO_DESCEND
            for (int32_t j = 0; j < k; j++) {
                if (j < H.nb) { out_ids[i * k + j] = H.best[j].id; out_d[i * k + j] = H.best[j].dist; }
                else { out_ids[i * k + j] = -1; out_d[i * k + j] = INFINITY; }
            }
            for (int64_t u = 0; u < ntouch; u++) seen[touched[u]] = 0;
            if (ncand) ncand[i] = nc;
            if (nleaves) nleaves[i] = checked;
        }
        free(seen);
        free(heap);
        free(best);
        free(touched);
        free(qt);
    }
}

/* ------------------------------------------------------------------ exact reference */

/*
 * Exact k nearest neighbours by brute force over all n points (Def. 1 with epsilon = 0), ordered by
 * (distance, id).  A bounded insertion list keeps the k best seen so far.
 */
void gfo_bruteforce(const float *X, int64_t n, int32_t d, const float *Q, int64_t m, int32_t k,
                    int64_t *out_ids, double *out_d) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; i++) {
        res_t *best = (res_t *)malloc(sizeof(res_t) * (size_t)k);
        int32_t nb = 0;
        for (int64_t x = 0; x < n; x++) {
            res_t r = {gfo_dist2(Q + i * d, X + x * d, d), x};
            if (nb == k && res_cmp(&r, &best[k - 1]) >= 0) continue;
            int32_t pos = nb < k ? nb++ : k - 1;
            while (pos > 0 && res_cmp(&r, &best[pos - 1]) < 0) { best[pos] = best[pos - 1]; pos--; }
            best[pos] = r;
        }
        for (int32_t j = 0; j < k; j++) {
            if (j < nb) { out_ids[i * k + j] = best[j].id; out_d[i * k + j] = best[j].dist; }
            else { out_ids[i * k + j] = -1; out_d[i * k + j] = INFINITY; }
        }
        free(best);
    }
}

int32_t gfo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
