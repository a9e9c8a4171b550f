// gf_build.cu -- GPU forest construction (Alg. 1; Alg. 3 variance; Sec. 2.1 randomization;
// Sec. 3 "Median, variances", "Tree structure").
//
// All T trees are built together, one tree level per step.  At level l every tree has 2^l nodes;
// node a of tree t owns the positions [a n >> l, (a+1) n >> l) of the tree's point sequence, and
// every step is a stable partition of each node's positions into its two children, so each
// sequence ends as the tree's leaf permutation (leaves list their points in ascending id order
// because the sequences start as 0..n-1).
//
// Per node:
//   1. per-dimension variance of the node's points from the sums of (x - K) and (x - K)^2 with K
//      the node's first point (no cancellation), accumulated as compensated float32 pairs and
//      combined in float64, then var = (S2 - S1^2 / c) / (c - 1);
//   2. the t dimensions of largest variance, ranked by (variance desc, index asc), and the split
//      dimension s = D[u mod t] with u the node's SplitMix64 draw;
//   3. the split: points ordered by the unique 64-bit key (order-preserving bits of x_s, rk_t(id))
//      where rk_t is the tree's fmix32 permutation of the ids; the h = |left child| smallest keys
//      go left.  The h-th key is found by an 8-pass radix select; v = x_s of that key (+inf when
//      the right child is empty, which only leaf_size 1 can produce);
//   4. the stable partition.
// Levels whose nodes hold more than SMALL points use chunked kernels over all nodes of the level
// (the variance partial sums of the chunks are added in a fixed order, so the build is
// deterministic); deeper levels use one CTA per node that keeps the node's keys in shared memory.
#include "gf_internal.cuh"
#include "gf_device.cuh"
#include "gf_trace.cuh"

#include <algorithm>
#include <utility>
#include <vector>

namespace {

using namespace gfdev;

constexpr int NT = 256;        // threads per CTA in every build kernel
constexpr int DPT = 4;         // dimensions per thread per dimension block
constexpr int DB = NT * DPT;   // dimensions per block
constexpr int CHUNK = 2048;    // points per chunk on the chunked levels
constexpr int SMALL = 8192;    // nodes up to this size are built by one CTA
constexpr int TMAX = 64;       // largest supported t

// ---------------------------------------------------------------- random numbers
// SplitMix64 (Steele, Lea, Flood 2014) output number i of the stream starting at s0, and the
// MurmurHash3 32-bit finalizer (a bijection), from their published definitions.
__device__ __forceinline__ unsigned long long sm64_at(unsigned long long s0, unsigned long long i) {
    unsigned long long z = s0 + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned fmix32(unsigned h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

struct BuildParams {
    const float *x;
    long long n;
    int d, ldx, T, t, shuffle, global_scope;
    unsigned long long seed;
    int2 *nodes;  // [T][2^L - 1]
    int nnodes;
    int *D;       // [TMAX] global top dims (global scope)
    const float *U;   // [T][d] Householder vectors, or null (trees on X itself)
    const float *W2;  // [T][n] 2 * u_t^T x_i of every point, when U is set
};

// Coordinate `dim` of point `id` as tree `tree` sees it: x itself, or its reflection (Sec. 2.2).
__device__ __forceinline__ float tree_coord(const BuildParams &P, int tree, int id, int dim) {
    const float x = __ldg(P.x + (size_t)id * P.ldx + dim);
    if (!P.U) return x;
    return reflect_coord(x, __ldg(P.W2 + (size_t)tree * P.n + id), __ldg(P.U + (size_t)tree * P.d + dim));
}

__device__ __forceinline__ unsigned long long tree_key(const BuildParams &P, int tree) {
    return sm64_at(P.seed, (unsigned long long)tree);
}

// tie-break order of point id in a tree whose key is tk
__device__ __forceinline__ unsigned rank_of(const BuildParams &P, unsigned long long tk, unsigned id) {
    return P.shuffle ? fmix32(id ^ (unsigned)sm64_at(tk, 0)) : id;
}

__device__ __forceinline__ unsigned ordered_bits(float f) {
    const unsigned u = __float_as_uint(f == 0.f ? 0.f : f);  // -0.0 reads as +0.0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o ^ 0x80000000u) : ~o);
}

__device__ __forceinline__ unsigned long long point_key(const BuildParams &P, unsigned long long tk, int tree,
                                                        int id, int s) {
    return ((unsigned long long)ordered_bits(tree_coord(P, tree, id, s)) << 32) | rank_of(P, tk, (unsigned)id);
}

// node geometry at level l
struct NodeGeo {
    int tree, a, j;
    long long lo, hi, mid;
};

__device__ __forceinline__ NodeGeo geo(const BuildParams &P, int l, long long seg) {
    NodeGeo g;
    g.tree = (int)(seg >> l);
    g.a = (int)(seg & ((1ll << l) - 1));
    g.j = (1 << l) - 1 + g.a;
    g.lo = ((long long)g.a * P.n) >> l;
    g.hi = ((long long)(g.a + 1) * P.n) >> l;
    g.mid = ((long long)(2 * g.a + 1) * P.n) >> (l + 1);
    return g;
}

// ---------------------------------------------------------------- variance

// Error-free transformations on float32 (Knuth's TwoSum; Dekker's product with an FMA): the
// result pair (s, e) satisfies s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated sum hi + lo of float32 terms: hi is the running float32 sum, lo collects every
// rounding error of hi exactly (plus its own, second-order, rounding).
struct FF {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(FF &a, float x, float xlo) {
    float s, e;
    two_sum(a.hi, x, s, e);
    a.hi = s;
    a.lo += e + xlo;
}

// Shifted sums over rows[0..cnt) for the dims dbase + tid + NT*u, u < DPT: S1 = sum (x - K),
// S2 = sum (x - K)^2 with K the node's first point.  Each difference is split exactly into
// float32 hi + lo, its square into a float32 product plus its exact FMA error (the lo^2 term is
// below 2^-48 relative and dropped), and both sums are compensated, so the relative error is of
// order cnt * 2^-48 -- float64 accuracy at float32 instruction rates (GB300's float64 rate is a
// small fraction of its float32 rate).
__device__ __forceinline__ void var_accum(const BuildParams &P, int tree, const int *__restrict__ rows,
                                          long long cnt, int krow, int dbase, double S1[DPT], double S2[DPT]) {
    float K[DPT], uu[DPT];
    int dim[DPT];
    FF s1[DPT], s2[DPT];
    const float *W2 = P.U ? P.W2 + (size_t)tree * P.n : nullptr;
#pragma unroll
    for (int u = 0; u < DPT; ++u) {
        dim[u] = dbase + threadIdx.x + NT * u;
        K[u] = dim[u] < P.d ? tree_coord(P, tree, krow, dim[u]) : 0.f;
        uu[u] = (P.U && dim[u] < P.d) ? __ldg(P.U + (size_t)tree * P.d + dim[u]) : 0.f;
        s1[u] = FF{0.f, 0.f};
        s2[u] = FF{0.f, 0.f};
    }
    auto add = [&](int u, float x) {
        float dh, dl;
        two_sum(x, -K[u], dh, dl);          // x - K = dh + dl exactly
        const float p = dh * dh;
        float pe = fmaf(dh, dh, -p);         // dh^2 = p + pe exactly
        pe = fmaf(2.f * dh, dl, pe);         // + 2 dh dl
        ff_add(s1[u], dh, dl);
        ff_add(s2[u], p, pe);
    };
    long long r = 0;
    for (; r + 4 <= cnt; r += 4) {
        float v[4][DPT], w2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int id = __ldg(rows + r + q);
            const float *row = P.x + (size_t)id * P.ldx;
            w2[q] = W2 ? __ldg(W2 + id) : 0.f;
#pragma unroll
            for (int u = 0; u < DPT; ++u) v[q][u] = dim[u] < P.d ? __ldg(row + dim[u]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int u = 0; u < DPT; ++u) add(u, W2 ? reflect_coord(v[q][u], w2[q], uu[u]) : v[q][u]);
    }
    for (; r < cnt; ++r) {
        const int id = __ldg(rows + r);
        const float *row = P.x + (size_t)id * P.ldx;
        const float w2 = W2 ? __ldg(W2 + id) : 0.f;
#pragma unroll
        for (int u = 0; u < DPT; ++u) {
            const float x = dim[u] < P.d ? __ldg(row + dim[u]) : 0.f;
            add(u, W2 ? reflect_coord(x, w2, uu[u]) : x);
        }
    }
#pragma unroll
    for (int u = 0; u < DPT; ++u) {
        S1[u] = (double)s1[u].hi + (double)s1[u].lo;
        S2[u] = (double)s2[u].hi + (double)s2[u].lo;
    }
}

__device__ __forceinline__ double var_of(double S1, double S2, long long c) {
    if (c < 2) return 0.0;
    return (S2 - S1 * S1 / (double)c) / (double)(c - 1);
}

__device__ __forceinline__ bool better(double va, int da, double vb, int db) {
    return va > vb || (va == vb && da < db);
}

// Warp 0 merges the block's variances vblk[0..nb) (dims dbase..) into the running top list
// (topv/topi, *have entries) and keeps the t best.  Called by all threads (syncs inside).
__device__ void topt_merge(const double *vblk, int nb, int dbase, double *topv, int *topi, int *have, int t) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int h = *have, tot = h + nb;
        unsigned long long picked = 0ull;
        double nv[TMAX];
        int ni[TMAX];
        const int rounds = min(t, tot);
        for (int r = 0; r < rounds; ++r) {
            double bv = -1.0;
            int bd = 0x7fffffff, bslot = -1;
            for (int c = lane, k = 0; c < tot; c += 32, ++k) {
                if ((picked >> k) & 1ull) continue;
                const double v = c < h ? topv[c] : vblk[c - h];
                const int dd = c < h ? topi[c] : dbase + (c - h);
                if (bslot < 0 || better(v, dd, bv, bd)) { bv = v; bd = dd; bslot = k; }
            }
            // warp argmax over (bv, bd); lanes with no candidate carry bslot < 0
            int owner = lane;
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(FULL, bv, o);
                const int od = __shfl_xor_sync(FULL, bd, o);
                const int os = __shfl_xor_sync(FULL, bslot, o);
                const int ow = __shfl_xor_sync(FULL, owner, o);
                const bool take = os >= 0 && (bslot < 0 || better(ov, od, bv, bd) ||
                                              (ov == bv && od == bd && ow < owner));
                if (take) { bv = ov; bd = od; bslot = os; owner = ow; }
            }
            if (lane == owner) picked |= 1ull << bslot;
            nv[r] = bv;
            ni[r] = bd;
        }
        __syncwarp();
        if (lane == 0) {
            for (int r = 0; r < rounds; ++r) { topv[r] = nv[r]; topi[r] = ni[r]; }
            *have = rounds;
        }
    }
    __syncthreads();
}

// Split dimension of node j of a tree: top list -> D[u mod t]
__device__ __forceinline__ int pick_dim(const BuildParams &P, unsigned long long tk, int j, const int *D) {
    const unsigned long long u = sm64_at(tk, (unsigned long long)j + 1ull);
    return D[u % (unsigned long long)P.t];
}

// Stable partition of rows[0..cnt) by key < kh into out[0..h) and out[h..cnt).
__device__ void block_partition(const int *__restrict__ rows, const unsigned long long *keys, int cnt,
                                unsigned long long kh, int h, int *out, int *wcnt, int *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) { sh[0] = 0; sh[1] = 0; }
    __syncthreads();
    for (int base = 0; base < cnt; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const bool in = i < cnt;
        const bool left = in && keys[i] < kh;
        const unsigned bl = __ballot_sync(FULL, left), bi = __ballot_sync(FULL, in);
        if (lane == 0) { wcnt[w] = __popc(bl); wcnt[32 + w] = __popc(bi & ~bl); }
        __syncthreads();
        int lo_l = sh[0], lo_r = sh[1];
        for (int q = 0; q < w; ++q) { lo_l += wcnt[q]; lo_r += wcnt[32 + q]; }
        const unsigned below = (1u << lane) - 1u;
        if (in) {
            const int id = rows[i];
            if (left) out[lo_l + __popc(bl & below)] = id;
            else out[h + lo_r + __popc(bi & ~bl & below)] = id;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tl = 0, tr = 0;
            for (int q = 0; q < nw; ++q) { tl += wcnt[q]; tr += wcnt[32 + q]; }
            sh[0] += tl;
            sh[1] += tr;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- small levels: CTA per node

struct SmallSmem {
    double vblk[DB];
    double topv[TMAX];
    int topi[TMAX];
    unsigned hist[256];
    int wcnt[64];
    int sh[4];
    int have;
    int s;
    int hs;
    unsigned long long pref;
};

__global__ void __launch_bounds__(NT) k_level_small(BuildParams P, int l, const int *__restrict__ pin,
                                                    int *pout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem &S = *reinterpret_cast<SmallSmem *>(smem_raw);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem_raw + sizeof(SmallSmem));
    const NodeGeo g = geo(P, l, blockIdx.x);
    const int cnt = (int)(g.hi - g.lo), h = (int)(g.mid - g.lo);
    const int *rows = pin + (size_t)g.tree * P.n + g.lo;
    const unsigned long long tk = tree_key(P, g.tree);
    // 1-2: split dimension
    if (P.global_scope && l > 0) {
        if (threadIdx.x == 0) S.s = pick_dim(P, tk, g.j, P.D);
    } else {
        if (threadIdx.x == 0) S.have = 0;
        for (int dbase = 0; dbase < P.d; dbase += DB) {
            double S1[DPT], S2[DPT];
            var_accum(P, g.tree, rows, cnt, rows[0], dbase, S1, S2);
#pragma unroll
            for (int u = 0; u < DPT; ++u) S.vblk[threadIdx.x + NT * u] = var_of(S1[u], S2[u], cnt);
            topt_merge(S.vblk, min(DB, P.d - dbase), dbase, S.topv, S.topi, &S.have, P.t);
        }
        if (threadIdx.x == 0) {
            S.s = pick_dim(P, tk, g.j, S.topi);
            if (P.global_scope)  // level 0 of the global scope: the root's top dims serve every node
                for (int r = 0; r < P.t; ++r) P.D[r] = S.topi[r];
        }
    }
    __syncthreads();
    const int s = S.s;
    // 3: keys, split key, split value
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) keys[i] = point_key(P, tk, g.tree, rows[i], s);
    __syncthreads();
    unsigned long long kh = ~0ull;
    float v = __int_as_float(0x7f800000);
    if (h < cnt) {
        kh = block_select(keys, cnt, h, S.hist, &S.pref, &S.hs);
        v = from_ordered((unsigned)(kh >> 32));
    }
    // 4: stable partition
    block_partition(rows, keys, cnt, kh, h, pout + (size_t)g.tree * P.n + g.lo, S.wcnt, S.sh);
    if (threadIdx.x == 0) P.nodes[(size_t)g.tree * P.nnodes + g.j] = make_int2(s, __float_as_int(v));
}

// ---------------------------------------------------------------- chunked levels

struct ChunkGeo {
    NodeGeo g;
    long long seg;
    int ci;
    long long beg, end;  // positions of the chunk (absolute within the tree's sequence)
};

__device__ __forceinline__ ChunkGeo chunk_geo(const BuildParams &P, int l, int nch, long long c) {
    ChunkGeo q;
    q.seg = c / nch;
    q.ci = (int)(c - q.seg * nch);
    q.g = geo(P, l, q.seg);
    q.beg = min(q.g.lo + (long long)q.ci * CHUNK, q.g.hi);
    q.end = min(q.beg + CHUNK, q.g.hi);
    return q;
}

// variance partial sums of one chunk: part[c][0..d) = S1, part[c][d..2d) = S2
__global__ void __launch_bounds__(NT) k_var_partial(BuildParams P, int l, int nch, const int *__restrict__ pin,
                                                    double *part) {
    const ChunkGeo q = chunk_geo(P, l, nch, blockIdx.x);
    const int *seq = pin + (size_t)q.g.tree * P.n;
    const int dbase = blockIdx.y * DB;
    double S1[DPT], S2[DPT];
    var_accum(P, q.g.tree, seq + q.beg, q.end - q.beg, seq[q.g.lo], dbase, S1, S2);
    double *o = part + (size_t)blockIdx.x * 2 * P.d;
#pragma unroll
    for (int u = 0; u < DPT; ++u) {
        const int dim = dbase + threadIdx.x + NT * u;
        if (dim < P.d) { o[dim] = S1[u]; o[P.d + dim] = S2[u]; }
    }
}

// add a node's chunk partials in chunk order, rank the dims, pick the split dimension
__global__ void __launch_bounds__(NT) k_var_combine(BuildParams P, int l, int nch, const double *__restrict__ part,
                                                    int *seg_s) {
    __shared__ double vblk[DB];
    __shared__ double topv[TMAX];
    __shared__ int topi[TMAX];
    __shared__ int have;
    const NodeGeo g = geo(P, l, blockIdx.x);
    const long long cnt = g.hi - g.lo;
    if (threadIdx.x == 0) have = 0;
    for (int dbase = 0; dbase < P.d; dbase += DB) {
#pragma unroll
        for (int u = 0; u < DPT; ++u) {
            const int dim = dbase + threadIdx.x + NT * u;
            double S1 = 0.0, S2 = 0.0;
            if (dim < P.d)
                for (int ci = 0; ci < nch; ++ci) {
                    const double *p = part + ((size_t)blockIdx.x * nch + ci) * 2 * P.d;
                    S1 += p[dim];
                    S2 += p[P.d + dim];
                }
            vblk[threadIdx.x + NT * u] = var_of(S1, S2, cnt);
        }
        topt_merge(vblk, min(DB, P.d - dbase), dbase, topv, topi, &have, P.t);
    }
    if (threadIdx.x == 0) {
        const unsigned long long tk = tree_key(P, g.tree);
        seg_s[blockIdx.x] = pick_dim(P, tk, g.j, topi);
        if (P.global_scope)
            for (int r = 0; r < P.t; ++r) P.D[r] = topi[r];
    }
}

// global scope below the root: s = D[u mod t]
__global__ void k_pick_global(BuildParams P, int l, long long nseg, int *seg_s) {
    const long long sg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const NodeGeo g = geo(P, l, sg);
    seg_s[sg] = pick_dim(P, tree_key(P, g.tree), g.j, P.D);
}

// keys of every position of every tree at level l
__global__ void k_keys(BuildParams P, int l, const int *__restrict__ pin, const int *__restrict__ seg_s,
                       unsigned long long *keys) {
    const long long tot = P.n * P.T;
    for (long long gidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; gidx < tot;
         gidx += (long long)gridDim.x * blockDim.x) {
        const int tree = (int)(gidx / P.n);
        const long long p = gidx - (long long)tree * P.n;
        const long long a = ((((p + 1) << l)) - 1) / P.n;  // node owning position p
        const long long seg = ((long long)tree << l) + a;
        keys[gidx] = point_key(P, tree_key(P, tree), tree, pin[gidx], seg_s[seg]);
    }
}

// radix-select state of a node: prefix of the wanted key, its rank among the keys with that prefix
struct SelState {
    unsigned long long pref;
    int hrem;
    int active;  // 0 when the right child is empty (no split key)
};

__global__ void k_sel_init(BuildParams P, int l, long long nseg, SelState *st, unsigned *ghist) {
    const long long sg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const NodeGeo g = geo(P, l, sg);
    st[sg].pref = 0ull;
    st[sg].hrem = (int)(g.mid - g.lo);
    st[sg].active = g.mid < g.hi;
    for (int b = 0; b < 256; ++b) ghist[sg * 256 + b] = 0;
}

__global__ void __launch_bounds__(NT) k_sel_hist(BuildParams P, int l, int nch, int pass,
                                                 const unsigned long long *__restrict__ keys,
                                                 const SelState *__restrict__ st, unsigned *ghist) {
    __shared__ unsigned hist[256];
    const ChunkGeo q = chunk_geo(P, l, nch, blockIdx.x);
    const SelState s = st[q.seg];
    if (!s.active) return;  // uniform per CTA
    for (int b = threadIdx.x; b < 256; b += NT) hist[b] = 0;
    __syncthreads();
    const int shift = 56 - 8 * pass;
    const unsigned long long *kk = keys + (size_t)q.g.tree * P.n;
    for (long long base = q.beg; base < q.end; base += NT) {
        const long long i = base + threadIdx.x;
        bool act = false;
        unsigned bin = 0;
        if (i < q.end) {
            const unsigned long long k = kk[i];
            act = pass == 0 || ((k ^ s.pref) >> (shift + 8)) == 0ull;
            bin = (unsigned)(k >> shift) & 255u;
        }
        hist_add(hist, bin, act);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += NT)
        if (hist[b]) atomicAdd(ghist + q.seg * 256 + b, hist[b]);
}

// one warp per node: find the bucket holding the wanted rank, extend the prefix, clear the histogram
__global__ void k_sel_pick(long long nseg, int pass, SelState *st, unsigned *ghist) {
    const long long sg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sg >= nseg) return;
    if (!st[sg].active) return;
    const int shift = 56 - 8 * pass;
    unsigned *hh = ghist + sg * 256;
    unsigned c[8], s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { c[q] = hh[8 * lane + q]; s += c[q]; }
    unsigned incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned before = incl - s;
    const unsigned hr = (unsigned)st[sg].hrem;
    const unsigned long long pref = st[sg].pref;
    __syncwarp();
    if (hr >= before && hr < incl) {
        unsigned acc = before;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (hr >= acc && hr < acc + c[q]) {
                st[sg].pref = pref | ((unsigned long long)(8 * lane + q) << shift);
                st[sg].hrem = (int)(hr - acc);
            }
            acc += c[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) hh[8 * lane + q] = 0;
}

__device__ __forceinline__ unsigned long long split_key(const SelState &s) { return s.active ? s.pref : ~0ull; }

// number of left points (key < split key) per chunk
__global__ void __launch_bounds__(NT) k_part_count(BuildParams P, int l, int nch,
                                                   const unsigned long long *__restrict__ keys,
                                                   const SelState *__restrict__ st, int *lcount) {
    __shared__ int wsum[NT / 32];
    const ChunkGeo q = chunk_geo(P, l, nch, blockIdx.x);
    const unsigned long long kh = split_key(st[q.seg]);
    const unsigned long long *kk = keys + (size_t)q.g.tree * P.n;
    int c = 0;
    for (long long i = q.beg + threadIdx.x; i < q.end; i += NT) c += kk[i] < kh;
    c = __reduce_add_sync(FULL, c);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < NT / 32; ++w) s += wsum[w];
        lcount[blockIdx.x] = s;
    }
}

// per node: chunk offsets of the left and right points; node record
__global__ void k_part_scan(BuildParams P, int l, int nch, long long nseg, const SelState *__restrict__ st,
                            const int *__restrict__ seg_s, const int *__restrict__ lcount, int *loff, int *roff) {
    const long long sg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const NodeGeo g = geo(P, l, sg);
    int accl = 0, accr = 0;
    for (int ci = 0; ci < nch; ++ci) {
        const long long c = sg * nch + ci;
        const long long beg = min(g.lo + (long long)ci * CHUNK, g.hi);
        const long long end = min(beg + CHUNK, g.hi);
        loff[c] = accl;
        roff[c] = accr;
        accl += lcount[c];
        accr += (int)(end - beg) - lcount[c];
    }
    const SelState s = st[sg];
    const float v = s.active ? from_ordered((unsigned)(s.pref >> 32)) : __int_as_float(0x7f800000);
    P.nodes[(size_t)g.tree * P.nnodes + g.j] = make_int2(seg_s[sg], __float_as_int(v));
}

__global__ void __launch_bounds__(NT) k_part_write(BuildParams P, int l, int nch, const int *__restrict__ pin,
                                                   const unsigned long long *__restrict__ keys,
                                                   const SelState *__restrict__ st, const int *__restrict__ loff,
                                                   const int *__restrict__ roff, int *pout) {
    __shared__ int wcnt[64];
    __shared__ int sh[4];
    const ChunkGeo q = chunk_geo(P, l, nch, blockIdx.x);
    const unsigned long long kh = split_key(st[q.seg]);
    const size_t toff = (size_t)q.g.tree * P.n;
    const int h = (int)(q.g.mid - q.g.lo);
    const int cnt = (int)(q.end - q.beg);
    // partition the chunk into a local view of the node's output: left part starts at
    // lo + loff, right part at lo + h + roff
    int *outL = pout + toff + q.g.lo + loff[blockIdx.x];
    int *outR = pout + toff + q.g.lo + h + roff[blockIdx.x];
    const int *rows = pin + toff + q.beg;
    const unsigned long long *kk = keys + toff + q.beg;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) { sh[0] = 0; sh[1] = 0; }
    __syncthreads();
    for (int base = 0; base < cnt; base += NT) {
        const int i = base + threadIdx.x;
        const bool in = i < cnt;
        const bool left = in && kk[i] < kh;
        const unsigned bl = __ballot_sync(FULL, left), bi = __ballot_sync(FULL, in);
        if (lane == 0) { wcnt[w] = __popc(bl); wcnt[32 + w] = __popc(bi & ~bl); }
        __syncthreads();
        int lo_l = sh[0], lo_r = sh[1];
        for (int qq = 0; qq < w; ++qq) { lo_l += wcnt[qq]; lo_r += wcnt[32 + qq]; }
        const unsigned below = (1u << lane) - 1u;
        if (in) {
            if (left) outL[lo_l + __popc(bl & below)] = rows[i];
            else outR[lo_r + __popc(bi & ~bl & below)] = rows[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tl = 0, tr = 0;
            for (int qq = 0; qq < NT / 32; ++qq) { tl += wcnt[qq]; tr += wcnt[32 + qq]; }
            sh[0] += tl;
            sh[1] += tr;
        }
        __syncthreads();
    }
}

// W2[t][i] = 2 * u_t^T x_i, one warp per point and one lane per tree, summed over j ascending with
// every multiply and add rounded on its own (the order reflect_w2 uses for queries).
__global__ void k_reflect_w2(const float *__restrict__ x, int ldx, long long n, int d, int T,
                             const float *__restrict__ U, float *W2) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < n; i += nw) {
        const float *row = x + i * ldx;
        for (int t0 = 0; t0 < T; t0 += 32) {
            const int t = t0 + lane;
            if (t < T) W2[(size_t)t * n + i] = reflect_w2(U + (size_t)t * d, row, d);
        }
    }
}

__global__ void k_iota(int *perm, long long n, int T) {
    const long long tot = n * T;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
         g += (long long)gridDim.x * blockDim.x)
        perm[g] = (int)(g % n);
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

}  // namespace

static int build_levels(gf_forest *F, const gf_rand_params &rp, uint64_t seed, cudaStream_t st) {
    const long long n = F->n;
    const int T = F->T, L = F->L;
    DevBuf tmp, Dbuf;
    int r;
    if ((r = gf_dmalloc(&tmp.p, (size_t)T * n * 4))) return r;
    if ((r = gf_dmalloc(&Dbuf.p, TMAX * sizeof(int)))) return r;
    // sequences ping-pong so that the last level writes into F->perm
    int *bufA = (L % 2 == 0) ? F->perm : (int *)tmp.p;
    int *bufB = (L % 2 == 0) ? (int *)tmp.p : F->perm;
    k_iota<<<F->num_sms * 8, 256, 0, st>>>(bufA, n, T);
    GF_CUDA_TRY(cudaGetLastError());

    BuildParams P;
    P.x = F->x; P.n = n; P.d = F->d; P.ldx = F->ldx; P.T = T; P.t = rp.t; P.shuffle = rp.shuffle ? 1 : 0;
    P.global_scope = rp.var_scope == GF_VAR_GLOBAL; P.seed = seed; P.nodes = F->nodes;
    P.nnodes = (1 << L) - 1; P.D = (int *)Dbuf.p;
    P.U = F->U;
    P.W2 = nullptr;
    DevBuf w2buf;
    if (F->U) {  // every tree sees its reflected points (Sec. 2.2)
        if ((r = gf_dmalloc(&w2buf.p, (size_t)T * n * 4))) return r;
        k_reflect_w2<<<F->num_sms * 16, 256, 0, st>>>(F->x, F->ldx, n, F->d, T, F->U, (float *)w2buf.p);
        GF_CUDA_TRY(cudaGetLastError());
        P.W2 = (const float *)w2buf.p;
    }

    // chunked-level scratch, sized for the deepest chunked level
    int lc = -1;  // last chunked level
    for (int l = 0; l < L; ++l)
        if (((n + (1ll << l) - 1) >> l) > SMALL) lc = l;
    DevBuf part, keys, segs, sel, ghist, lcnt, loff, roff;
    long long maxch = 0, maxseg = 0;
    if (lc >= 0) {
        for (int l = 0; l <= lc; ++l) {
            const long long cm = (n + (1ll << l) - 1) >> l;
            const long long nch = (cm + CHUNK - 1) / CHUNK;
            maxch = std::max(maxch, ((long long)T << l) * nch);
            maxseg = std::max(maxseg, (long long)T << l);
        }
        if ((r = gf_dmalloc(&part.p, (size_t)maxch * 2 * F->d * sizeof(double)))) return r;
        if ((r = gf_dmalloc(&keys.p, (size_t)T * n * 8))) return r;
        if ((r = gf_dmalloc(&segs.p, (size_t)maxseg * 4))) return r;
        if ((r = gf_dmalloc(&sel.p, (size_t)maxseg * sizeof(SelState)))) return r;
        if ((r = gf_dmalloc(&ghist.p, (size_t)maxseg * 256 * 4))) return r;
        if ((r = gf_dmalloc(&lcnt.p, (size_t)maxch * 4))) return r;
        if ((r = gf_dmalloc(&loff.p, (size_t)maxch * 4))) return r;
        if ((r = gf_dmalloc(&roff.p, (size_t)maxch * 4))) return r;
    }
    int dev = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t small_max = sizeof(SmallSmem) + (size_t)SMALL * 8;
    if (small_max > (size_t)smem_optin) return gf_fail(GF_EUNSUPPORTED, "build needs %zu B shared memory", small_max);
    GF_CUDA_TRY(cudaFuncSetAttribute(k_level_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_max));

    const int ndb = (F->d + DB - 1) / DB;
    for (int l = 0; l < L; ++l) {
        GfRange level_range("gf_build: level");
        const long long cm = (n + (1ll << l) - 1) >> l;
        const long long nseg = (long long)T << l;
        if (cm <= SMALL) {
            const size_t smem = sizeof(SmallSmem) + (size_t)cm * 8;
            k_level_small<<<(unsigned)nseg, NT, smem, st>>>(P, l, bufA, bufB);
            GF_CUDA_TRY(cudaGetLastError());
        } else {
            const int nch = (int)((cm + CHUNK - 1) / CHUNK);
            const long long nchunks = nseg * nch;
            int *seg_s = (int *)segs.p;
            SelState *ss = (SelState *)sel.p;
            unsigned *gh = (unsigned *)ghist.p;
            const unsigned gseg = (unsigned)((nseg + 255) / 256);
            if (!P.global_scope || l == 0) {
                k_var_partial<<<dim3((unsigned)nchunks, ndb), NT, 0, st>>>(P, l, nch, bufA, (double *)part.p);
                k_var_combine<<<(unsigned)nseg, NT, 0, st>>>(P, l, nch, (const double *)part.p, seg_s);
            } else {
                k_pick_global<<<gseg, 256, 0, st>>>(P, l, nseg, seg_s);
            }
            k_keys<<<F->num_sms * 16, 256, 0, st>>>(P, l, bufA, seg_s, (unsigned long long *)keys.p);
            k_sel_init<<<gseg, 256, 0, st>>>(P, l, nseg, ss, gh);
            for (int pass = 0; pass < 8; ++pass) {
                k_sel_hist<<<(unsigned)nchunks, NT, 0, st>>>(P, l, nch, pass, (const unsigned long long *)keys.p, ss, gh);
                k_sel_pick<<<(unsigned)((nseg * 32 + 255) / 256), 256, 0, st>>>(nseg, pass, ss, gh);
            }
            k_part_count<<<(unsigned)nchunks, NT, 0, st>>>(P, l, nch, (const unsigned long long *)keys.p, ss,
                                                           (int *)lcnt.p);
            k_part_scan<<<gseg, 256, 0, st>>>(P, l, nch, nseg, ss, seg_s, (const int *)lcnt.p, (int *)loff.p,
                                              (int *)roff.p);
            k_part_write<<<(unsigned)nchunks, NT, 0, st>>>(P, l, nch, bufA, (const unsigned long long *)keys.p, ss,
                                                           (const int *)loff.p, (const int *)roff.p, bufB);
            GF_CUDA_TRY(cudaGetLastError());
        }
        std::swap(bufA, bufB);
    }
    GF_CUDA_TRY(cudaStreamSynchronize(st));
    return GF_OK;
}

static int build_any(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size, const gf_rand_params *rp_in,
                     uint64_t seed, const float *U_host, int32_t borrow_x, void *stream, gf_forest **out);

extern "C" int gf_build_ex(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                           const gf_rand_params *rp_in, uint64_t seed, int32_t borrow_x, void *stream,
                           gf_forest **out) {
    return build_any(X, n, d, T, leaf_size, rp_in, seed, nullptr, borrow_x, stream, out);
}

extern "C" int gf_build_reflected(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                                  const gf_rand_params *rp, uint64_t seed, const float *U_host,
                                  int32_t borrow_x, void *stream, gf_forest **out) {
    if (!U_host) return gf_fail(GF_EINVAL, "gf_build_reflected: U is null");
    return build_any(X, n, d, T, leaf_size, rp, seed, U_host, borrow_x, stream, out);
}

static int build_any(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size, const gf_rand_params *rp_in,
                     uint64_t seed, const float *U_host, int32_t borrow_x, void *stream, gf_forest **out) {
    GfRange range("gf_build");
    if (!out) return gf_fail(GF_EINVAL, "out is null");
    *out = nullptr;
    gf_rand_params rp;
    gf_rand_params_default(&rp);
    if (rp_in) rp = *rp_in;
    if (rp.householder && !U_host)
        return gf_fail(GF_EINVAL, "householder = 1 needs the per-tree vectors: use gf_build_reflected");
    if (U_host && rp.var_scope == GF_VAR_GLOBAL)
        return gf_fail(GF_EINVAL, "a global variance ranking is not defined for per-tree reflected points");
    if (rp.t < 1 || rp.t > d || rp.t > TMAX) return gf_fail(GF_EINVAL, "t=%d outside [1, min(d, %d)]", rp.t, TMAX);
    if (rp.var_scope != GF_VAR_NODE && rp.var_scope != GF_VAR_GLOBAL) return gf_fail(GF_EINVAL, "bad var_scope");
    if (n >= 1 && leaf_size >= 1) {
        const int L = depth_of(n, leaf_size);
        if (L > 0 && ((long long)T << (L - 1)) >= (1ll << 31))
            return gf_fail(GF_EUNSUPPORTED, "T * 2^(L-1) nodes per level exceeds 2^31");
    }
    cudaStream_t st = (cudaStream_t)stream;
    gf_forest *F = nullptr;
    int r = gf_forest_alloc(&F, X, n, d, T, leaf_size, borrow_x != 0, st);
    if (r) return r;
    if ((r = gf_check_finite(F->x, (int64_t)n * F->ldx, st))) { gf_forest_destroy(F); return r; }
    if (U_host && (r = gf_forest_set_U(F, U_host))) { gf_forest_destroy(F); return r; }
    if ((r = build_levels(F, rp, seed, st))) { gf_forest_destroy(F); return r; }
    *out = F;
    return GF_OK;
}

extern "C" int gf_build(const float *X, int64_t n, int32_t d, int32_t T, int32_t leaf_size,
                        const gf_rand_params *rp, uint64_t seed, gf_forest **out) {
    return gf_build_ex(X, n, d, T, leaf_size, rp, seed, 0, nullptr, out);
}
