// gf_query.cu -- the query hot path: descent, candidate gather + de-duplication, squared-L2
// scoring and top-k selection (Alg. 2 with one leaf per tree; Eq. 1; Sec. 2.3; Sec. 3 "Distance
// computation").
//
// One CTA owns one query at a time and keeps everything the query needs in shared memory:
//   - the query row (float32, zero-padded),
//   - the T leaf ranges reached by the descent,
//   - the gathered candidate ids, sorted and de-duplicated in place (the "seen" array of Sec. 2.3
//     becomes a sort-unique over at most T * max_leaf ids),
//   - one 64-bit key (distance bits << 32 | id) per candidate, sorted to give the k nearest by
//     (distance, id).
// The scoring loop is the only part that touches HBM in bulk: every candidate row is streamed
// once with 16-byte read-only loads that bypass L1, a warp per row, two rows in flight per warp.
#include "gf_internal.cuh"
#include "gf_device.cuh"
#include "gf_score.cuh"

#include <algorithm>
#include <climits>

namespace {

// ---------------------------------------------------------------- descent (Alg. 2, Eq. 1)

// Leaf of one tree reached by query q: at each node the signed distance q_s - v decides the
// side; negative goes left (2j+1), zero or positive goes right (2j+2).
__device__ __forceinline__ int descend_tree(const int2 *__restrict__ nodes, int L, const float *q) {
    int j = 0;
    for (int l = 0; l < L; ++l) {
        const int2 nd = __ldg(nodes + j);
        j = 2 * j + (q[nd.x] < __int_as_float(nd.y) ? 1 : 2);
    }
    return j - ((1 << L) - 1);
}

// Leaf of tree t: when the forest has Householder vectors the query is reflected with the tree's
// vector before it descends (Sec. 2.2); only the coordinates the path reads are formed.
__device__ __forceinline__ int descend_tree_t(const ForestView &F, int t, const float *q) {
    const int2 *nodes = F.nodes + (size_t)t * F.nnodes;
    if (!F.U) return descend_tree(nodes, F.L, q);
    const float *u = F.U + (size_t)t * F.d;
    const float w2 = reflect_w2(u, q, F.d);
    int j = 0;
    for (int l = 0; l < F.L; ++l) {
        const int2 nd = __ldg(nodes + j);
        j = 2 * j + (reflect_coord(q[nd.x], w2, __ldg(u + nd.x)) < __int_as_float(nd.y) ? 1 : 2);
    }
    return j - ((1 << F.L) - 1);
}


// Copy the distinct values of the sorted a[0..tot) to u[] (keeping order); returns their number.
__device__ int block_unique(const int *a, int tot, int *u, int *wtmp) {
    const int nt = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = nt >> 5;
    const int E = (tot + nt - 1) / nt;
    const int beg = threadIdx.x * E, end = min(beg + E, tot);
    int cnt = 0;
    for (int i = beg; i < end; ++i) cnt += (i == 0 || a[i] != a[i - 1]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? wtmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += t;
        }
        if (lane < nw) wtmp[lane] = v;
    }
    __syncthreads();
    int pos = (w ? wtmp[w - 1] : 0) + incl - cnt;
    const int total = wtmp[nw - 1];
    for (int i = beg; i < end; ++i)
        if (i == 0 || a[i] != a[i - 1]) u[pos++] = a[i];
    __syncthreads();
    return total;
}

// Gather the points of the T leaves (ranges lofs/lcnt of each tree's perm) into cand, sort them
// and keep each id once (Sec. 2.3).  Returns the number of distinct candidates, written to u.
__device__ int gather_unique(const ForestView &F, const int *lofs, const int *lcnt, int *lpos,
                             int *cand, int *u, int *wtmp, int *sh) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < F.T; ++t) {
            lpos[t] = acc;
            acc += lcnt[t];
        }
        sh[0] = acc;
    }
    __syncthreads();
    const int tot = sh[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = w; t < F.T; t += nw) {
        const int32_t *src = F.perm + (size_t)t * F.n + lofs[t];
        int *dst = cand + lpos[t];
        for (int j = lane; j < lcnt[t]; j += 32) dst[j] = __ldg(src + j);
    }
    int P = 1;
    while (P < tot) P <<= 1;
    for (int i = tot + threadIdx.x; i < P; i += blockDim.x) cand[i] = INT_MAX;
    block_sort<int>(cand, P);
    return block_unique(cand, tot, u, wtmp);
}


// The query values matching a lane's chunks (NC > 0: chunks lane, lane+32, ...), in registers.
template <int PREC, int NC>
__device__ __forceinline__ void load_qreg(const ForestView &F, const float *qs, float4 *qr) {
    constexpr int QF4 = Prec<PREC>::QF4;
    const int lane = threadIdx.x & 31;
    const int nch = (int)(row_pitch<PREC>(F) >> 4);
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
#pragma unroll
    for (int c = 0; c < (NC > 0 ? NC : 0); ++c) {
        const int cc = lane + 32 * c;
#pragma unroll
        for (int h = 0; h < QF4; ++h)
            qr[c * QF4 + h] = cc < nch ? q4[cc * QF4 + h] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Squared distances of the query to rows i0 and i1 (both valid ids), by the whole warp; every
// lane returns both sums.  NC > 0: a lane holds at most NC 16-byte chunks of a row and the query's
// matching values in qr; NC == 0: any row length, query read from shared memory.
template <int PREC, int NC>
__device__ __forceinline__ void warp_dist2(const ForestView &F, const float4 *qr, const float *qs, int i0,
                                           int i1, float &d0, float &d1) {
    constexpr int QF4 = Prec<PREC>::QF4;
    const int lane = threadIdx.x & 31;
    const size_t pitch = row_pitch<PREC>(F);
    const int nch = (int)(pitch >> 4);
    const unsigned char *r0 = row_base<PREC>(F) + (size_t)i0 * pitch;
    const unsigned char *r1 = row_base<PREC>(F) + (size_t)i1 * pitch;
    const float s0 = PREC == P_FP8 ? __ldg(F.scale8 + i0) : 0.f;
    const float s1 = PREC == P_FP8 ? __ldg(F.scale8 + i1) : 0.f;
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    constexpr int UB = NC > 0 ? NC : 4;  // chunks per lane loaded before use
    for (int c0 = lane; c0 < nch; c0 += 32 * UB) {
        uint4 x0[UB], x1[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int cc = c0 + 32 * u;
            if (cc < nch) {
                x0[u] = ld_u4(r0 + ((size_t)cc << 4));
                x1[u] = ld_u4(r1 + ((size_t)cc << 4));
            }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int cc = c0 + 32 * u;
            if (cc < nch) {
                float4 qa[QF4];
#pragma unroll
                for (int h = 0; h < QF4; ++h) qa[h] = NC > 0 ? qr[u * QF4 + h] : q4[cc * QF4 + h];
                if (PREC == P_F32) {
                    acc4(a0, qa[0], *reinterpret_cast<const float4 *>(&x0[u]));
                    acc4(a1, qa[0], *reinterpret_cast<const float4 *>(&x1[u]));
                } else if (PREC == P_BF16) {
                    acc_bf16(a0, qa[0], qa[1], x0[u]);
                    acc_bf16(a1, qa[0], qa[1], x1[u]);
                } else {
                    acc_fp8w(a0, qa[0], x0[u].x, s0); acc_fp8w(a0, qa[1], x0[u].y, s0);
                    acc_fp8w(a0, qa[2], x0[u].z, s0); acc_fp8w(a0, qa[3], x0[u].w, s0);
                    acc_fp8w(a1, qa[0], x1[u].x, s1); acc_fp8w(a1, qa[1], x1[u].y, s1);
                    acc_fp8w(a1, qa[2], x1[u].z, s1); acc_fp8w(a1, qa[3], x1[u].w, s1);
                }
            }
        }
        if (NC > 0) break;  // one pass covers the row
    }
    d0 = warp_sum(sum4(a0));
    d1 = warp_sum(sum4(a1));
}

// Score candidates ids[0..C) of the query in qs (float32, zero-padded to a multiple of 16) and
// write one key per candidate.  Warp w takes rows w, w + nw, ...; two rows are in flight per
// warp.  An id outside [0, n) gets the empty key.
template <int PREC, int NC>
__device__ void score_rows(const ForestView &F, const float *qs, const int *ids, int C,
                           unsigned long long *keys) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float4 qr[(NC > 0 ? NC : 1) * Prec<PREC>::QF4];
    load_qreg<PREC, NC>(F, qs, qr);
    for (int j = w; j < C; j += 2 * nw) {
        const int j1 = j + nw;
        const int i0 = ids[j];
        const int i1 = j1 < C ? ids[j1] : i0;
        const bool v0 = (unsigned)i0 < (unsigned long long)F.n;
        const bool v1 = (unsigned)i1 < (unsigned long long)F.n;
        float d0, d1;
        warp_dist2<PREC, NC>(F, qr, qs, v0 ? i0 : 0, v1 ? i1 : 0, d0, d1);
        if (lane == 0) {
            keys[j] = v0 ? make_key(d0, i0) : KEY_NONE;
            if (j1 < C) keys[j1] = v1 ? make_key(d1, i1) : KEY_NONE;
        }
    }
}


// ---------------------------------------------------------------- shared-memory plan

struct Smem {
    unsigned long long *keys;  // [P]   (cand aliases it as int[P] before scoring)
    float *qs;                 // [ldq]
    int *u;                    // [cand_cap] distinct candidates / shortlist
    int *lofs, *lcnt, *lpos;   // [T]
    int *wtmp;                 // [32]
    int *sh;                   // [4]
};


// keys region: a power of two >= cap and >= 2, so that the float4 query row after it is aligned
__host__ __device__ inline int keys_len(int cap) {
    int P = 2;
    while (P < cap) P <<= 1;
    return P;
}

__host__ __device__ inline size_t smem_bytes(int d, int T, int cap) {
    const int P = keys_len(cap);
    return (size_t)P * 8 + (size_t)ldq_of(d) * 4 + (size_t)cap * 4 + (size_t)T * 12 + 32 * 4 + 16;
}

__device__ inline Smem carve(unsigned char *p, int d, int T, int cap) {
    Smem s;
    const int P = keys_len(cap);
    s.keys = reinterpret_cast<unsigned long long *>(p);
    p += (size_t)P * 8;
    s.qs = reinterpret_cast<float *>(p);
    p += (size_t)ldq_of(d) * 4;
    s.u = reinterpret_cast<int *>(p);
    p += (size_t)cap * 4;
    s.lofs = reinterpret_cast<int *>(p);
    s.lcnt = s.lofs + T;
    s.lpos = s.lcnt + T;
    s.wtmp = s.lpos + T;
    s.sh = s.wtmp + 32;
    return s;
}

__device__ void leaf_range(const ForestView &F, int t, int b, int *lofs, int *lcnt) {
    const long long lo = ((long long)b * F.n) >> F.L;
    const long long hi = ((long long)(b + 1) * F.n) >> F.L;
    lofs[t] = (int)lo;
    lcnt[t] = (int)(hi - lo);
}

// ---------------------------------------------------------------- kernels

// Stage 1: one thread per (query, tree); the query row is read through L1.
__global__ void k_descend(ForestView F, const float *__restrict__ Q, long long m, int *leaf) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= m * F.T) return;
    const long long i = g / F.T;
    const int t = (int)(g - i * F.T);
    leaf[g] = descend_tree_t(F, t, Q + i * F.d);
}

// Stage 2: one CTA per query.
__global__ void k_candidates(ForestView F, const int *__restrict__ leaf, long long m, int *cand,
                             int *ncand) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem s = carve(smem_raw, F.d, F.T, F.cand_cap);
    for (long long i = blockIdx.x; i < m; i += gridDim.x) {
        for (int t = threadIdx.x; t < F.T; t += blockDim.x) {
            int b = leaf[i * F.T + t];
            b = min(max(b, 0), (1 << F.L) - 1);
            leaf_range(F, t, b, s.lofs, s.lcnt);
        }
        __syncthreads();
        const int C = gather_unique(F, s.lofs, s.lcnt, s.lpos, reinterpret_cast<int *>(s.keys), s.u,
                                    s.wtmp, s.sh);
        for (int j = threadIdx.x; j < C; j += blockDim.x) cand[(size_t)i * F.cand_cap + j] = s.u[j];
        if (threadIdx.x == 0) ncand[i] = C;
        __syncthreads();
    }
}

// Stages 3-4 (float32): one CTA per query.
template <int NC>
__global__ void k_score_topk(ForestView F, const float *__restrict__ Q, long long m,
                             const int *__restrict__ cand, const int *__restrict__ ncand, int stride,
                             int k, long long *ids, float *dists) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem s = carve(smem_raw, F.d, F.T, F.cand_cap);
    for (long long i = blockIdx.x; i < m; i += gridDim.x) {
        load_query(Q + i * F.d, F.d, s.qs);
        const int C = min(max(ncand[i], 0), min(stride, F.cand_cap));
        for (int j = threadIdx.x; j < C; j += blockDim.x) s.u[j] = cand[(size_t)i * stride + j];
        __syncthreads();
        score_rows<P_F32, NC>(F, s.qs, s.u, C, s.keys);
        sort_keys(s.keys, C);
        write_topk(s.keys, C, k, ids + i * k, dists + i * k);
        __syncthreads();
    }
}

// Screened distance of every candidate (no selection), for checking the screen arithmetic.  The
// candidates go through shared memory in blocks of SCORE_BLOCK, so any candidate count fits.
constexpr int SCORE_BLOCK = 2048;

__host__ __device__ inline size_t score_all_smem(int d) {
    return (size_t)SCORE_BLOCK * 8 + (size_t)ldq_of(d) * 4 + (size_t)SCORE_BLOCK * 4;
}

template <int PREC, int NC>
__global__ void k_score_all(ForestView F, const float *__restrict__ Q, long long m,
                            const int *__restrict__ cand, const int *__restrict__ ncand, int stride,
                            float *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem_raw);
    float *qs = reinterpret_cast<float *>(keys + SCORE_BLOCK);
    int *u = reinterpret_cast<int *>(qs + ldq_of(F.d));
    for (long long i = blockIdx.x; i < m; i += gridDim.x) {
        load_query(Q + i * F.d, F.d, qs);
        const int C = min(max(ncand[i], 0), stride);
        for (int b0 = 0; b0 < C; b0 += SCORE_BLOCK) {
            const int nb = min(SCORE_BLOCK, C - b0);
            for (int j = threadIdx.x; j < nb; j += blockDim.x) u[j] = cand[(size_t)i * stride + b0 + j];
            __syncthreads();
            score_rows<PREC, NC>(F, qs, u, nb, keys);
            __syncthreads();
            for (int j = threadIdx.x; j < nb; j += blockDim.x)
                out[(size_t)i * stride + b0 + j] = keys[j] == KEY_NONE ? __int_as_float(0x7fc00000)
                                                                        : __uint_as_float((unsigned)(keys[j] >> 32));
            __syncthreads();
        }
    }
}

// The whole path per query (persistent: CTAs stride over the queries).  Screened precisions rank
// the candidates by the low-precision distance, keep the R best and rerank them in float32.
template <int PREC, int NC, int NCF>
__global__ void k_query_fused(ForestView F, const float *__restrict__ Q, long long m, int k, int R,
                              long long *ids, float *dists) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem s = carve(smem_raw, F.d, F.T, F.cand_cap);
    for (long long i = blockIdx.x; i < m; i += gridDim.x) {
        load_query(Q + i * F.d, F.d, s.qs);
        __syncthreads();
        for (int t = threadIdx.x; t < F.T; t += blockDim.x)
            leaf_range(F, t, descend_tree_t(F, t, s.qs), s.lofs, s.lcnt);
        __syncthreads();
        int C = gather_unique(F, s.lofs, s.lcnt, s.lpos, reinterpret_cast<int *>(s.keys), s.u, s.wtmp,
                              s.sh);
        score_rows<PREC, NC>(F, s.qs, s.u, C, s.keys);
        sort_keys(s.keys, C);
        if (PREC != P_F32) {
            // shortlist: the R best by the screened distance, rescored in float32
            const int Rn = min(R, C);
            for (int j = threadIdx.x; j < Rn; j += blockDim.x)
                s.u[j] = (int)(unsigned)(s.keys[j] & 0xffffffffu);
            __syncthreads();
            score_rows<P_F32, NCF>(F, s.qs, s.u, Rn, s.keys);
            sort_keys(s.keys, Rn);
            C = Rn;
        }
        write_topk(s.keys, C, k, ids + i * k, dists + i * k);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- streaming path
//
// For candidate sets of any size.  The query's leaf positions (the concatenated leaf ranges of the
// T trees) are processed in phases of LIST positions:
//   A. every thread takes positions of the phase, reads their ids from the permutations and
//      test-and-sets them in a bitmap over the point ids -- one per CTA in device memory, the
//      "seen" array of Sec. 2.3 -- so each id is admitted once per query; admitted ids are packed
//      into a shared list;
//   B. the warps score the listed rows, G rows in flight per warp, and append the keys that beat
//      the running threshold to a shared buffer (no barrier inside the phase);
//   then, if the buffer holds more than `keep` keys, a radix select keeps the best `keep` and
//   raises the threshold.  After the last phase the kept keys are sorted (a screened precision
//   rescores its R best in float32) and the query's bits are cleared, so the bitmap is all zero
//   between queries.

constexpr int LIST = GF_MAX_SHORTLIST;  // positions per phase; also the longest k or R

struct StreamLayout {
    size_t buf, list, qs, pref, lbase, lcnt, lpos, hist, wtmp, sh, total;
};

// Every region starts on a 16-byte boundary (the query row is read as float4, the keys as u64).
// nl: leaves per query (T for one leaf per tree, the leaf budget for the priority search)
__host__ __device__ inline StreamLayout stream_layout(int d, int nl, int buf_len) {
    StreamLayout L;
    size_t o = 0;
    auto take = [&o](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.buf = take((size_t)buf_len * 8);
    L.list = take((size_t)LIST * 4);
    L.qs = take((size_t)ldq_of(d) * 4);
    L.pref = take(16);  // select prefix, threshold
    L.lbase = take((size_t)nl * 8);
    L.lcnt = take((size_t)nl * 4);
    L.lpos = take((size_t)(nl + 1) * 4);
    L.hist = take(256 * 4);
    L.wtmp = take(64 * 4);
    L.sh = take(8 * 4);
    L.total = o;
    return L;
}

// largest t with lpos[t] <= pos (lpos[0] = 0 <= pos < lpos[T])
__device__ __forceinline__ int tree_of_pos(const int *lpos, int T, int pos) {
    int lo = 0, hi = T;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (lpos[mid] <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// id at concatenated position pos: leaf j's ids start at perm offset lbase[j]
__device__ __forceinline__ int id_at(const ForestView &F, const int *lpos, const long long *lbase, int nl, int pos) {
    const int j = tree_of_pos(lpos, nl, pos);
    return __ldg(F.perm + lbase[j] + (pos - lpos[j]));
}

// In-place stable compaction of buf[0..cnt) to the keys <= kth.
__device__ void compact_le(unsigned long long *buf, int cnt, unsigned long long kth, int *wtmp, int *run) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) *run = 0;
    __syncthreads();
    for (int base = 0; base < cnt; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const unsigned long long key = i < cnt ? buf[i] : KEY_NONE;
        const bool keep = i < cnt && key <= kth;
        const unsigned bl = __ballot_sync(FULL, keep);
        if (lane == 0) wtmp[w] = __popc(bl);
        __syncthreads();
        int off = *run;
        for (int q = 0; q < w; ++q) off += wtmp[q];
        off += __popc(bl & ((1u << lane) - 1u));
        if (keep) buf[off] = key;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int q = 0; q < nw; ++q) t += wtmp[q];
            *run += t;
        }
        __syncthreads();
    }
}


template <int PREC, int NC, int NCF, int G>
__global__ void __launch_bounds__(256, 2) k_query_stream(ForestView F, const float *__restrict__ Q, long long m,
                                                      int k, int R, int buf_len, unsigned *bitmaps, int nwords,
                                                      const int *__restrict__ order,
                                                      const unsigned *__restrict__ leaf_list,
                                                      const int *__restrict__ nleaf_list, int nl_max,
                                                      long long *ids, float *dists, int *ncand_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const StreamLayout Ly = stream_layout(F.d, nl_max, buf_len);
    unsigned long long *buf = reinterpret_cast<unsigned long long *>(smem_raw + Ly.buf);
    int *list = reinterpret_cast<int *>(smem_raw + Ly.list);
    float *qs = reinterpret_cast<float *>(smem_raw + Ly.qs);
    unsigned long long *pref = reinterpret_cast<unsigned long long *>(smem_raw + Ly.pref);
    unsigned long long *thr = pref + 1;
    long long *lbase = reinterpret_cast<long long *>(smem_raw + Ly.lbase);
    int *lcnt = reinterpret_cast<int *>(smem_raw + Ly.lcnt);
    int *lpos = reinterpret_cast<int *>(smem_raw + Ly.lpos);
    unsigned *hist = reinterpret_cast<unsigned *>(smem_raw + Ly.hist);
    int *wtmp = reinterpret_cast<int *>(smem_raw + Ly.wtmp);
    // sh: [0] compaction scratch [1] buffer count [2] positions [3] admitted ids [4] select [5] list count
    //     [6] leaves of the current query
    int *sh = reinterpret_cast<int *>(smem_raw + Ly.sh);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int keep = PREC == P_F32 ? k : R;
    unsigned *bm = bitmaps + (size_t)blockIdx.x * nwords;
    const unsigned lt = (1u << lane) - 1u;

    for (long long qs_i = blockIdx.x; qs_i < m; qs_i += gridDim.x) {
        const long long qi = order ? (long long)order[qs_i] : qs_i;  // CTAs walk the batch in `order`
        load_query(Q + qi * F.d, F.d, qs);
        __syncthreads();
        // the leaves this query checks: one per tree (descent, Eq. 1) or a given list
        const int nl = leaf_list ? min(nleaf_list[qi], nl_max) : F.T;
        for (int j = threadIdx.x; j < nl; j += blockDim.x) {
            int t, b;
            if (leaf_list) {
                const unsigned code = leaf_list[qi * nl_max + j];
                t = (int)(code >> F.L);
                b = (int)(code & ((1u << F.L) - 1u));
            } else {
                t = j;
                b = descend_tree_t(F, t, qs);
            }
            const long long lo = ((long long)b * F.n) >> F.L;
            const long long hi = ((long long)(b + 1) * F.n) >> F.L;
            lbase[j] = (long long)t * F.n + lo;
            lcnt[j] = (int)(hi - lo);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int j = 0; j < nl; ++j) {
                lpos[j] = acc;
                acc += lcnt[j];
            }
            lpos[nl] = acc;
            sh[1] = 0;
            sh[2] = acc;
            sh[3] = 0;
            sh[6] = nl;
            *thr = KEY_NONE;
        }
        __syncthreads();
        const int tot = sh[2];
        for (int p0 = 0; p0 < tot; p0 += LIST) {
            // ---- A: admit the phase's ids through the bitmap, pack them into the list
            if (threadIdx.x == 0) sh[5] = 0;
            __syncthreads();
            const int pend = min(LIST, tot - p0);
            for (int b0 = 0; b0 < pend; b0 += 4 * blockDim.x) {
                int id[4];
                unsigned old[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int off = b0 + u * blockDim.x + threadIdx.x;
                    id[u] = off < pend ? id_at(F, lpos, lbase, nl, p0 + off) : -1;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    old[u] = id[u] >= 0 ? atomicOr(bm + (id[u] >> 5), 1u << (id[u] & 31)) : ~0u;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool fresh = id[u] >= 0 && !(old[u] & (1u << (id[u] & 31)));
                    const unsigned bl = __ballot_sync(FULL, fresh);
                    int base = 0;
                    if (lane == 0 && bl) base = atomicAdd(&sh[5], __popc(bl));
                    base = __shfl_sync(FULL, base, 0);
                    if (fresh) list[base + __popc(bl & lt)] = id[u];
                }
            }
            __syncthreads();
            const int nadm = sh[5];
            // ---- B: score the admitted rows, G per warp at a time
            for (int j0 = w * G; j0 < nadm; j0 += nw * G) {
                int rid[G];
                float dd[G];
#pragma unroll
                for (int g = 0; g < G; ++g) rid[g] = list[min(j0 + g, nadm - 1)];
                warp_dist_g<PREC, NC, G>(F, qs, rid, dd);
                if (lane == 0) {
                    const unsigned long long th = *reinterpret_cast<volatile unsigned long long *>(thr);
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (j0 + g >= nadm) break;
                        const unsigned long long key = make_key(dd[g], rid[g]);
                        if (key < th) buf[atomicAdd(&sh[1], 1)] = key;
                    }
                }
            }
            __syncthreads();
            const int cnt_now = sh[1];
            if (threadIdx.x == 0) sh[3] += nadm;
            __syncthreads();  // every thread has read the count before it changes
            if (cnt_now > keep) {
                const unsigned long long kth = gfdev::block_select(buf, cnt_now, keep - 1, hist, pref, &sh[4]);
                compact_le(buf, cnt_now, kth, wtmp, &sh[0]);
                if (threadIdx.x == 0) {
                    sh[1] = keep;
                    *thr = kth;
                }
                __syncthreads();
            }
        }
        const int cnt = min(sh[1], keep);
        sort_keys(buf, cnt);
        if (PREC != P_F32) {
            for (int j = threadIdx.x; j < cnt; j += blockDim.x) list[j] = (int)(unsigned)(buf[j] & 0xffffffffu);
            __syncthreads();
            rescore_f32<NCF>(F, qs, list, cnt, buf);
            sort_keys(buf, cnt);
        }
        write_topk(buf, cnt, k, ids + qi * k, dists + qi * k);
        for (int pos = threadIdx.x; pos < tot; pos += blockDim.x) bm[id_at(F, lpos, lbase, nl, pos) >> 5] = 0u;
        if (threadIdx.x == 0 && ncand_out) ncand_out[qi] = sh[3];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- query order (locality)
//
// Queries that reach the same leaf of tree 0 share most of their candidates, so a batch walked in
// order of that leaf lets CTAs running at the same time read the same rows (from L2).  The order
// changes no result: every query's answer is computed on its own.

constexpr int ORDER_CHUNK = 16384;  // queries sorted together by one CTA

__global__ void k_order_keys(ForestView F, const float *__restrict__ Q, long long m, unsigned long long *keys) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int leaf0 = descend_tree_t(F, 0, Q + i * F.d);
    keys[i] = ((unsigned long long)(unsigned)leaf0 << 32) | (unsigned long long)(i & 0xffffffffll);
}

__global__ void k_order_sort(long long m, const unsigned long long *__restrict__ keys, int *order) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *k = reinterpret_cast<unsigned long long *>(smem_raw);
    const long long base = (long long)blockIdx.x * ORDER_CHUNK;
    const int cnt = (int)min((long long)ORDER_CHUNK, m - base);
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int j = threadIdx.x; j < P; j += blockDim.x) k[j] = j < cnt ? keys[base + j] : KEY_NONE;
    block_sort<unsigned long long>(k, P);
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) order[base + j] = (int)(unsigned)(k[j] & 0xffffffffu);
}

// ---------------------------------------------------------------- host side

int nc_for(int chunks) {
    if (chunks <= 32) return 1;
    if (chunks <= 64) return 2;
    if (chunks <= 128) return 4;
    if (chunks <= 256) return 8;
    return 0;
}

template <typename KernelT>
int prep_kernel(KernelT kern, size_t smem) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return gf_cuda_fail(e, "cudaFuncSetAttribute(max dynamic smem)");
    }
    return GF_OK;
}

int check_smem(const gf_forest *F, size_t smem) {
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)lim)
        return gf_fail(GF_EUNSUPPORTED,
                       "per-query shared memory %zu B (d=%d, T=%d, candidates<=%d) exceeds %d B",
                       smem, F->d, F->T, F->cand_cap, lim);
    return GF_OK;
}

template <int PREC, int NC, int NCF>
int launch_fused(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t R, int warps,
                 int ctas_per_sm, cudaStream_t st, int64_t *ids, float *dists, const QueryExtra &x) {
    const size_t smem = smem_bytes(F->d, F->T, F->cand_cap);
    int r = check_smem(F, smem);
    if (r) return r;
    auto kern = k_query_fused<PREC, NC, NCF>;
    if ((r = prep_kernel(kern, smem))) return r;
    const int threads = warps * 32;
    cudaFuncAttributes fa;
    GF_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    if (threads > fa.maxThreadsPerBlock)
        return gf_fail(GF_EINVAL, "warps_per_cta=%d exceeds this kernel's limit of %d threads (%d registers)",
                       warps, fa.maxThreadsPerBlock, fa.numRegs);
    if (ctas_per_sm <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
        ctas_per_sm = occ > 0 ? occ : 1;
    }
    long long grid = (long long)F->num_sms * ctas_per_sm;
    if (grid > m) grid = m;
    GF_CUDA_TRY(gf_record(x, 0, st));
    kern<<<(unsigned)grid, threads, smem, st>>>(view_of(F), Q, m, k, R, (long long *)ids, dists);
    GF_CUDA_TRY(cudaGetLastError());
    GF_CUDA_TRY(gf_record(x, 1, st));
    return GF_OK;
}

// Device scratch of one streaming launch, in this order (each part 16-byte aligned):
//   bitmaps  grid * ceil(n/32) words, zero between queries
//   okeys    m * 8  and  order  m * 4          (locality order)
//   leaves   m * nl * 4  and  nleaves  m * 4   (priority search leaf lists)
struct StreamWorkspace {
    size_t okeys, order, leaves, nleaves, total;
};

StreamWorkspace stream_workspace(const gf_forest *F, long long m, long long grid, bool ordered, int nl) {
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    StreamWorkspace W;
    size_t o = al((size_t)grid * ((F->n + 31) / 32) * 4);
    W.okeys = o;
    W.order = ordered ? al(o + (size_t)m * 8) : o;
    o = ordered ? al(W.order + (size_t)m * 4) : o;
    W.leaves = o;
    W.nleaves = nl > 0 ? al(o + (size_t)m * nl * 4) : o;
    o = nl > 0 ? al(W.nleaves + (size_t)m * 4) : o;
    W.total = o;
    return W;
}

// buffer: the kept keys plus one phase of appends
int stream_buf_len(int keep) { return keep + LIST; }

// default rows in flight per warp: four when a lane holds at most two 16-byte chunks of a row,
// else two (more would spill registers)
int default_rows_in_flight(int nc) { return (nc == 0 || nc >= 4) ? 2 : 4; }

template <int PREC, int NC, int NCF, int G>
int launch_stream_g(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t R, int warps,
                    int ctas_per_sm, cudaStream_t st, int64_t *ids, float *dists, const QueryExtra &x,
                    long long *grid_only) {
    const int keep = PREC == P_F32 ? k : R;
    if (keep > LIST) return gf_fail(GF_EUNSUPPORTED, "k or R = %d above %d", keep, LIST);
    const int buf_len = stream_buf_len(keep);
    const bool prio = x.leaf_budget > F->T;  // Alg. 2 priority search: a leaf list per query
    const int nl_max = prio ? x.leaf_budget : F->T;
    const size_t smem = stream_layout(F->d, nl_max, buf_len).total;
    int r = check_smem(F, smem);
    if (r) return r;
    if (warps > 8) return gf_fail(GF_EINVAL, "warps_per_cta=%d above 8 for the streaming kernel", warps);
    auto kern = k_query_stream<PREC, NC, NCF, G>;
    if ((r = prep_kernel(kern, smem))) return r;
    const int threads = warps * 32;
    cudaFuncAttributes fa;
    GF_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    if (threads > fa.maxThreadsPerBlock)
        return gf_fail(GF_EINVAL, "warps_per_cta=%d exceeds this kernel's limit of %d threads (%d registers)",
                       warps, fa.maxThreadsPerBlock, fa.numRegs);
    if (ctas_per_sm <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
        ctas_per_sm = occ > 0 ? occ : 1;
    }
    long long grid = (long long)F->num_sms * ctas_per_sm;
    if (grid > m) grid = m;
    if (grid_only) {
        *grid_only = grid;
        return GF_OK;
    }
    const int nwords = (int)((F->n + 31) / 32);
    const bool ordered = x.order == GF_ORDER_LOCALITY || (x.order == GF_ORDER_AUTO && m > grid);
    const StreamWorkspace W = stream_workspace(F, m, grid, ordered, prio ? nl_max : 0);
    const size_t ws_bytes = W.total;
    unsigned *bitmaps = (unsigned *)x.workspace;
    bool own = false;
    if (bitmaps) {
        if ((size_t)x.workspace_bytes < ws_bytes)
            return gf_fail(GF_EINVAL, "workspace of %lld bytes, %zu needed", (long long)x.workspace_bytes, ws_bytes);
    } else {
        cudaError_t e = cudaMallocAsync((void **)&bitmaps, ws_bytes, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return gf_fail(GF_ENOMEM, "query workspace of %zu bytes: %s", ws_bytes, cudaGetErrorString(e));
        }
        own = true;
        e = cudaMemsetAsync(bitmaps, 0, ws_bytes, st);
        if (e != cudaSuccess) { cudaFreeAsync(bitmaps, st); return gf_cuda_fail(e, "workspace memset"); }
    }
    int *order = nullptr;
    unsigned *leaf_list = nullptr;
    int *nleaf_list = nullptr;
    if (prio) {
        leaf_list = (unsigned *)((char *)bitmaps + W.leaves);
        nleaf_list = (int *)((char *)bitmaps + W.nleaves);
        if ((r = gf_launch_prio_leaves(F, Q, m, nl_max, leaf_list, nleaf_list, st))) {
            if (own) cudaFreeAsync(bitmaps, st);
            return r;
        }
    }
    if (ordered) {
        unsigned long long *okeys = (unsigned long long *)((char *)bitmaps + W.okeys);
        order = (int *)((char *)bitmaps + W.order);
        k_order_keys<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(view_of(F), Q, m, okeys);
        const long long chunks = (m + ORDER_CHUNK - 1) / ORDER_CHUNK;
        const int P = next_pow2((int)std::min<long long>(m, ORDER_CHUNK));
        const size_t osmem = (size_t)P * 8;
        if ((r = prep_kernel(k_order_sort, osmem))) {
            if (own) cudaFreeAsync(bitmaps, st);
            return r;
        }
        k_order_sort<<<(unsigned)chunks, 1024, osmem, st>>>(m, okeys, order);
    }
    cudaError_t e = gf_record(x, 0, st);
    kern<<<(unsigned)grid, threads, smem, st>>>(view_of(F), Q, m, k, R, buf_len, bitmaps, nwords, order,
                                               leaf_list, nleaf_list, nl_max, (long long *)ids, dists,
                                               x.ncand_out);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = gf_record(x, 1, st);
    if (own) cudaFreeAsync(bitmaps, st);
    if (e != cudaSuccess) return gf_cuda_fail(e, "k_query_stream launch");
    return GF_OK;
}

template <int PREC, int NC, int NCF>
int launch_stream(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t R, int warps,
                  int ctas_per_sm, cudaStream_t st, int64_t *ids, float *dists, const QueryExtra &x,
                  long long *grid_only = nullptr) {
    const int g = x.rows_in_flight > 0 ? x.rows_in_flight : default_rows_in_flight(NC);
    if (g == 2) return launch_stream_g<PREC, NC, NCF, 2>(F, Q, m, k, R, warps, ctas_per_sm, st, ids, dists, x, grid_only);
    if (g == 4) return launch_stream_g<PREC, NC, NCF, 4>(F, Q, m, k, R, warps, ctas_per_sm, st, ids, dists, x, grid_only);
    return gf_fail(GF_EINVAL, "rows_in_flight=%d (2 or 4)", g);
}

template <int PREC>
int stream_grid_prec(const gf_forest *F, int64_t m, int k, int R, int warps, int cps, long long *grid) {
    const int chunks = PREC == P_F32 ? F->ldx / 4 : PREC == P_BF16 ? F->ldb / 8 : F->ld8 / 16;
    const int ncf = nc_for(F->ldx / 4);
    const int nc = nc_for(chunks);
    QueryExtra x;
#define GF_G(A, B) \
    if (nc == A && ncf == B) return launch_stream<PREC, A, B>(F, nullptr, m, k, R, warps, cps, 0, nullptr, nullptr, x, grid);
    if (PREC == P_F32) {
        GF_G(1, 1) GF_G(2, 2) GF_G(4, 4) GF_G(8, 8) GF_G(0, 0)
    } else {
        GF_G(1, 1) GF_G(1, 2) GF_G(1, 4) GF_G(2, 4) GF_G(2, 8) GF_G(4, 8)
        GF_G(1, 8) GF_G(4, 0) GF_G(8, 0) GF_G(0, 0) GF_G(2, 0) GF_G(1, 0)
    }
#undef GF_G
    return gf_fail(GF_EUNSUPPORTED, "no kernel for chunk classes %d/%d", nc, ncf);
}

template <int PREC>
int dispatch_prec(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t R, int warps,
                  int cps, cudaStream_t st, int64_t *ids, float *dists, const QueryExtra &x) {
    const int chunks = PREC == P_F32 ? F->ldx / 4 : PREC == P_BF16 ? F->ldb / 8 : F->ld8 / 16;
    const int ncf = nc_for(F->ldx / 4);
    const int nc = nc_for(chunks);
    int algo = x.algo;
    if (x.leaf_budget > F->T) {
        if (algo == GF_ALGO_SORT) return gf_fail(GF_EINVAL, "the priority search runs in the streaming kernel only");
        algo = GF_ALGO_STREAM;
    }
    if (algo == GF_ALGO_AUTO) {
        const size_t sort_smem = smem_bytes(F->d, F->T, F->cand_cap);
        algo = (F->cand_cap <= 4096 && sort_smem <= 100 * 1024 && !x.ncand_out) ? GF_ALGO_SORT : GF_ALGO_STREAM;
    }
    if (algo == GF_ALGO_SORT && x.ncand_out)
        return gf_fail(GF_EINVAL, "candidate counts are reported by the streaming kernel only");
#define GF_CASE(A, B)                                                                              \
    if (nc == A && ncf == B)                                                                       \
        return algo == GF_ALGO_SORT ? launch_fused<PREC, A, B>(F, Q, m, k, R, warps, cps, st, ids, dists, x) \
                                    : launch_stream<PREC, A, B>(F, Q, m, k, R, warps, cps, st, ids, dists, x);
    if (PREC == P_F32) {
        GF_CASE(1, 1) GF_CASE(2, 2) GF_CASE(4, 4) GF_CASE(8, 8) GF_CASE(0, 0)
    } else {
        // the screened row is shorter than the float32 row, so its class is never larger
        GF_CASE(1, 1) GF_CASE(1, 2) GF_CASE(1, 4) GF_CASE(2, 4) GF_CASE(2, 8) GF_CASE(4, 8)
        GF_CASE(1, 8) GF_CASE(4, 0) GF_CASE(8, 0) GF_CASE(0, 0) GF_CASE(2, 0) GF_CASE(1, 0)
    }
#undef GF_CASE
    return gf_fail(GF_EUNSUPPORTED, "no kernel for chunk classes %d/%d", nc, ncf);
}

}  // namespace

int gf_launch_query(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t precision,
                    int32_t R, int32_t warps, int32_t ctas_per_sm, cudaStream_t st, int64_t *ids,
                    float *dists, const QueryExtra &x) {
    if (x.algo == GF_ALGO_LEAF || (x.algo == GF_ALGO_AUTO && gf_leaf_preferred(F, m, k, precision, R, x))) {
        const char *why = gf_leaf_unsupported(F, m, k, precision, R, x);
        if (why) return gf_fail(GF_EUNSUPPORTED, "GF_ALGO_LEAF: %s", why);
        return gf_launch_leaf(F, Q, m, k, precision, R, x.order, x.leaf_budget, st, ids, dists, x.workspace,
                              x.workspace_bytes, x.events, ctas_per_sm);
    }
    switch (precision) {
        case GF_FP32: return dispatch_prec<P_F32>(F, Q, m, k, R, warps, ctas_per_sm, st, ids, dists, x);
        case GF_BF16_RERANK: return dispatch_prec<P_BF16>(F, Q, m, k, R, warps, ctas_per_sm, st, ids, dists, x);
        case GF_FP8_RERANK: return dispatch_prec<P_FP8>(F, Q, m, k, R, warps, ctas_per_sm, st, ids, dists, x);
    }
    return gf_fail(GF_EINVAL, "unknown precision %d", precision);
}

int gf_stream_workspace_bytes(const gf_forest *F, int64_t m, long long grid, bool ordered, int leaf_budget,
                              int64_t *bytes) {
    *bytes = (int64_t)stream_workspace(F, m, grid, ordered, leaf_budget > F->T ? leaf_budget : 0).total;
    return GF_OK;
}

int gf_stream_grid(const gf_forest *F, int64_t m, int warps, int ctas_per_sm, int precision, int k, int R,
                   long long *grid) {
    switch (precision) {
        case GF_FP32: return stream_grid_prec<P_F32>(F, m, k, R, warps, ctas_per_sm, grid);
        case GF_BF16_RERANK: return stream_grid_prec<P_BF16>(F, m, k, R, warps, ctas_per_sm, grid);
        case GF_FP8_RERANK: return stream_grid_prec<P_FP8>(F, m, k, R, warps, ctas_per_sm, grid);
    }
    return gf_fail(GF_EINVAL, "unknown precision %d", precision);
}

// ---------------------------------------------------------------- ABI: staged path

extern "C" int gf_descend(const gf_forest *F, const float *Q, int64_t m, int32_t *leaf, void *stream) {
    if (!F) return gf_fail(GF_EINVAL, "gf_descend: null forest");
    if (m < 0) return gf_fail(GF_EINVAL, "gf_descend: m < 0");
    if (m == 0) return GF_OK;
    if (!Q || !leaf) return gf_fail(GF_EINVAL, "gf_descend: null pointer");
    const long long tot = (long long)m * F->T;
    const int threads = 256;
    k_descend<<<(unsigned)((tot + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
        view_of(F), Q, m, leaf);
    GF_CUDA_TRY(cudaGetLastError());
    return GF_OK;
}

extern "C" int gf_candidates(const gf_forest *F, const int32_t *leaf, int64_t m, int32_t *cand,
                             int32_t *ncand, void *stream) {
    if (!F) return gf_fail(GF_EINVAL, "gf_candidates: null forest");
    if (m < 0) return gf_fail(GF_EINVAL, "gf_candidates: m < 0");
    if (m == 0) return GF_OK;
    if (!leaf || !cand || !ncand) return gf_fail(GF_EINVAL, "gf_candidates: null pointer");
    const size_t smem = smem_bytes(F->d, F->T, F->cand_cap);
    int r = check_smem(F, smem);
    if (r) return r;
    if ((r = prep_kernel(k_candidates, smem))) return r;
    const long long grid = m < (long long)F->num_sms * 8 ? m : (long long)F->num_sms * 8;
    k_candidates<<<(unsigned)grid, 256, smem, (cudaStream_t)stream>>>(view_of(F), leaf, m, cand, ncand);
    GF_CUDA_TRY(cudaGetLastError());
    return GF_OK;
}

extern "C" int gf_score_topk(const gf_forest *F, const float *Q, int64_t m, const int32_t *cand,
                             const int32_t *ncand, int32_t cand_stride, int32_t k, int64_t *ids,
                             float *dists, void *stream) {
    if (!F) return gf_fail(GF_EINVAL, "gf_score_topk: null forest");
    if (m < 0 || k < 1 || cand_stride < 0) return gf_fail(GF_EINVAL, "gf_score_topk: bad sizes");
    if (m == 0) return GF_OK;
    if (!Q || !cand || !ncand || !ids || !dists) return gf_fail(GF_EINVAL, "gf_score_topk: null pointer");
    const size_t smem = smem_bytes(F->d, F->T, F->cand_cap);
    int r = check_smem(F, smem);
    if (r) return r;
    const long long grid = m < (long long)F->num_sms * 4 ? m : (long long)F->num_sms * 4;
    const int nc = nc_for(F->ldx / 4);
    cudaStream_t st = (cudaStream_t)stream;
#define GF_SCORE(NCV)                                                                        \
    if (nc == NCV) {                                                                         \
        if ((r = prep_kernel(k_score_topk<NCV>, smem))) return r;                           \
        k_score_topk<NCV><<<(unsigned)grid, 256, smem, st>>>(view_of(F), Q, m, cand, ncand, \
                                                             cand_stride, k, (long long *)ids, dists); \
    }
    GF_SCORE(1) GF_SCORE(2) GF_SCORE(4) GF_SCORE(8) GF_SCORE(0)
#undef GF_SCORE
    GF_CUDA_TRY(cudaGetLastError());
    return GF_OK;
}

extern "C" int gf_score_screened(const gf_forest *F, const float *Q, int64_t m, const int32_t *cand,
                                 const int32_t *ncand, int32_t cand_stride, int32_t precision,
                                 float *dist, void *stream) {
    if (!F) return gf_fail(GF_EINVAL, "gf_score_screened: null forest");
    if (m < 0 || cand_stride < 0) return gf_fail(GF_EINVAL, "gf_score_screened: bad sizes");
    if (m == 0) return GF_OK;
    if (!Q || !cand || !ncand || !dist) return gf_fail(GF_EINVAL, "gf_score_screened: null pointer");
    if (precision == GF_BF16_RERANK && !F->xb) return gf_fail(GF_EINVAL, "no bf16 copy");
    if (precision == GF_FP8_RERANK && !F->x8) return gf_fail(GF_EINVAL, "no fp8 copy");
    if (precision < 0 || precision > 2) return gf_fail(GF_EINVAL, "unknown precision %d", precision);
    const size_t smem = score_all_smem(F->d);
    int r = check_smem(F, smem);
    if (r) return r;
    const long long grid = m < (long long)F->num_sms * 4 ? m : (long long)F->num_sms * 4;
    const int chunks = precision == GF_FP32 ? F->ldx / 4 : precision == GF_BF16_RERANK ? F->ldb / 8 : F->ld8 / 16;
    const int nc = nc_for(chunks);
    cudaStream_t st = (cudaStream_t)stream;
#define GF_ALL(PV, NCV)                                                                          \
    if (precision == PV && nc == NCV) {                                                          \
        auto kern = k_score_all<PV, NCV>;                                                        \
        if ((r = prep_kernel(kern, smem))) return r;                                            \
        kern<<<(unsigned)grid, 256, smem, st>>>(view_of(F), Q, m, cand, ncand, cand_stride, dist); \
    }
    GF_ALL(P_F32, 1) GF_ALL(P_F32, 2) GF_ALL(P_F32, 4) GF_ALL(P_F32, 8) GF_ALL(P_F32, 0)
    GF_ALL(P_BF16, 1) GF_ALL(P_BF16, 2) GF_ALL(P_BF16, 4) GF_ALL(P_BF16, 8) GF_ALL(P_BF16, 0)
    GF_ALL(P_FP8, 1) GF_ALL(P_FP8, 2) GF_ALL(P_FP8, 4) GF_ALL(P_FP8, 8) GF_ALL(P_FP8, 0)
#undef GF_ALL
    GF_CUDA_TRY(cudaGetLastError());
    return GF_OK;
}
