// gf_prio.cu -- the leaves a query checks under Alg. 2's shared priority queue (Sec. 2.3).
//
// For each query, in the order of Alg. 2:
//   * every tree is descended from its root (Eq. 1); each node passed pushes the child not taken
//     with key |q_s - v|; the leaf reached is checked (reading: these first T leaves count toward
//     the budget, so a budget of T leaves is exactly the one-leaf-per-tree search);
//   * then, while fewer than `budget` leaves were checked, the entry of smallest
//     (key, tree, node) is taken from the queue and descended the same way to one more leaf.
// The keys are computed in float64 (the difference of two floats is exact there), so the order,
// including ties, is exactly the CPU oracle's.  A key is non-negative, so its IEEE bits order as the
// value does: the queue compares the bits as 64-bit integers (GB300's float64 compare rate is a
// small fraction of its integer rate).
//
// One warp per query.  The queue is two sorted arrays in shared memory: a large one A and a small
// one B (at most 64 entries).  A pop takes the smaller of their heads.  The entries a descent pushes
// (at most L <= 30) are merged into B by the warp; once B holds more than 32 it is merged into A in
// place (from the top down), so the large array moves once every few pops instead of at every one.
// The first phase (one entry per tree and level) merges into A directly.  Entries ranked beyond the
// number of pops still to come can never be taken and are dropped, so A never holds more than
// `budget` entries past its head.  The order of the pops is that of a single sorted queue: every
// pop takes the smallest (key, tree, node) held.  The output is the list of leaves in the order
// checked, encoded (tree << L) | leaf.
#include "gf_internal.cuh"
#include "gf_trace.cuh"

#include <algorithm>

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PRIO_WARPS = 4;  // at most this many warps (queries) per CTA

struct PQE {
    unsigned long long key;  // bits of the float64 key |q_s - v| (>= 0)
    int tree;
    int node;
};

__device__ __forceinline__ bool pq_less(const PQE &a, const PQE &b) {
    if (a.key != b.key) return a.key < b.key;
    if (a.tree != b.tree) return a.tree < b.tree;
    return a.node < b.node;
}

__device__ __forceinline__ unsigned long long pq_key(float qs, float v) {
    return (unsigned long long)__double_as_longlong(fabs((double)qs - (double)v));
}

__device__ __forceinline__ PQE pq_inf() {
    PQE e;
    e.key = 0x7ff0000000000000ull;  // +inf
    e.tree = 0x7fffffff;
    e.node = 0x7fffffff;
    return e;
}

// Merge the nb (<= 32) entries of stage[] into the sorted array src[0..cnt); write the first
// min(cnt + nb, keep) entries of the merged order to dst[]; returns their number.  Warp-wide.
__device__ int pq_merge(const PQE *src, int cnt, PQE *stage, int nb, PQE *dst, int keep, PQE *sorted) {
    const int lane = threadIdx.x & 31;
    // rank of every staged entry among the staged entries (all distinct)
    PQE mine = lane < nb ? stage[lane] : pq_inf();
    int r = 0;
    for (int i = 0; i < nb; ++i) r += pq_less(stage[i], mine);
    __syncwarp();
    if (lane < nb) sorted[r] = mine;
    __syncwarp();
    // staged entry r goes to r + (number of src entries below it)
    if (lane < nb) {
        int lo = 0, hi = cnt;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (pq_less(src[mid], mine)) lo = mid + 1;
            else hi = mid;
        }
        const int pos = r + lo;
        if (pos < keep) dst[pos] = mine;
    }
    // src entry j goes to j + (number of staged entries below it)
    for (int j = lane; j < cnt; j += 32) {
        const PQE e = src[j];
        int lo = 0, hi = nb;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (pq_less(sorted[mid], e)) lo = mid + 1;
            else hi = mid;
        }
        const int pos = j + lo;
        if (pos < keep) dst[pos] = e;
    }
    __syncwarp();
    return min(cnt + nb, keep);
}

// Number of entries of the sorted array a[0..n) below e.  Warp lanes call it independently.
__device__ __forceinline__ int pq_lower(const PQE *a, int n, const PQE &e) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pq_less(a[mid], e)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// sorted[0..nb) = the nb (<= 32) staged entries in order.  Warp-wide.
__device__ void pq_sort_stage(const PQE *stage, int nb, PQE *sorted) {
    const int lane = threadIdx.x & 31;
    const PQE mine = lane < nb ? stage[lane] : pq_inf();
    int r = 0;
    for (int i = 0; i < nb; ++i) r += pq_less(stage[i], mine);
    __syncwarp();
    if (lane < nb) sorted[r] = mine;
    __syncwarp();
}

// Merge the sorted array s[0..ns) (ns <= 64, not overlapping a) into the sorted array a[0..na) in
// place, keeping the first min(na + ns, keep) entries of the merged order in a[]; returns their
// number.  a[] must have room for them.  An entry of a moves up by the number of s entries below
// it, so a is moved from the top down, 32 entries at a time, each group read before it is written.
// Warp-wide.
__device__ int pq_merge_into(PQE *a, int na, const PQE *s, int ns, int keep) {
    const int lane = threadIdx.x & 31;
    // the positions of s's entries in the merged order, against a as it is now
    int ps[2];
    PQE es[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        es[h] = i < ns ? s[i] : pq_inf();
        ps[h] = i < ns ? i + pq_lower(a, na, es[h]) : keep;
    }
    __syncwarp();
    for (int top = na; top > 0; top -= 32) {
        const int j = top - 32 + lane;
        PQE e;
        int pos = keep;
        if (j >= 0) {
            e = a[j];
            pos = j + pq_lower(s, ns, e);
        }
        __syncwarp();
        if (j >= 0 && pos < keep) a[pos] = e;
        __syncwarp();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (ps[h] < keep) a[ps[h]] = es[h];
    __syncwarp();
    return min(na + ns, keep);
}

__device__ __forceinline__ unsigned leaf_code(int tree, int leaf, int L) {
    return ((unsigned)tree << L) | (unsigned)leaf;
}

constexpr int PQ_BCAP = 64;  // entries of each small queue array

// per-warp shared memory: the large queue array (`budget` + 64 entries), the small one (two
// buffers), the staged batch and its sorted copy, then one reflection weight per tree
__host__ __device__ inline size_t prio_warp_bytes(int budget, int T) {
    return (size_t)(budget + 64 + 2 * PQ_BCAP + 64) * sizeof(PQE) + (size_t)(T + 3) / 4 * 16;
}

__global__ void __launch_bounds__(PRIO_WARPS * 32) k_prio_leaves(ForestView F, const float *__restrict__ Q,
                                                                long long m, int budget, int cap,
                                                                unsigned *leaves, int *nleaves) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *mine = smem_raw + (size_t)w * prio_warp_bytes(budget, F.T);
    PQE *base = reinterpret_cast<PQE *>(mine);
    PQE *qa = base;                                   // A [cap]
    PQE *qb = base + cap, *qb2 = qb + PQ_BCAP;        // B, double-buffered
    PQE *stage = qb2 + PQ_BCAP, *sorted = stage + 32;
    float *w2s = reinterpret_cast<float *>(sorted + 32);
    const int nn = (1 << F.L) - 1;
    const int nwq = blockDim.x >> 5;
    for (long long qi = (long long)blockIdx.x * nwq + w; qi < m; qi += (long long)gridDim.x * nwq) {
        const float *q = Q + qi * F.d;
        unsigned *out = leaves + qi * budget;
        int acnt = 0, ahead = 0, bcnt = 0, bhead = 0, checked = 0;  // A holds [ahead, acnt), B [bhead, bcnt)
        // ---- first descent of every tree, 32 trees at a time, one level per merge
        for (int t0 = 0; t0 < F.T; t0 += 32) {
            const int t = t0 + lane;
            const bool act = t < F.T;
            float w2 = 0.f;
            if (act && F.U) {  // the query's reflection for this tree (Sec. 2.3)
                w2 = reflect_w2(F.U + (size_t)t * F.d, q, F.d);
                w2s[t] = w2;
            }
            int j = 0;
            for (int l = 0; l < F.L; ++l) {
                PQE e = pq_inf();
                if (act) {
                    const int2 nd = __ldg(F.nodes + (size_t)t * F.nnodes + j);
                    const float qx = __ldg(q + nd.x);
                    const float qs = F.U ? reflect_coord(qx, w2, __ldg(F.U + (size_t)t * F.d + nd.x)) : qx;
                    const float v = __int_as_float(nd.y);
                    e.key = pq_key(qs, v);
                    e.tree = t;
                    e.node = qs < v ? 2 * j + 2 : 2 * j + 1;  // the child not taken
                    j = qs < v ? 2 * j + 1 : 2 * j + 2;
                }
                stage[lane] = e;
                __syncwarp();
                const int nb = min(32, F.T - t0);
                const int keep = min(cap, max(0, budget - F.T));
                pq_sort_stage(stage, nb, sorted);
                acnt = pq_merge_into(qa, acnt, sorted, nb, keep);
            }
            if (act && t < budget) out[t] = leaf_code(t, j - nn, F.L);
        }
        checked = min(F.T, budget);
        // ---- pops in queue order
        while (checked < budget && (ahead < acnt || bhead < bcnt)) {
            // the smaller head of A and B
            const PQE ta = ahead < acnt ? qa[ahead] : pq_inf(), tb = bhead < bcnt ? qb[bhead] : pq_inf();
            const bool fromb = pq_less(tb, ta);
            const PQE top = fromb ? tb : ta;
            if (fromb) ++bhead;
            else ++ahead;
            // descend from the popped node, staging the siblings passed.  The warp loads the
            // five-level subtree below the current node at once (lane i: node i in breadth-first
            // order, with its query coordinate), then walks it through shuffles: five levels cost
            // one round of loads instead of five dependent ones.  Same path, same pushes.
            const int tr = top.tree;
            const int2 *tnodes = F.nodes + (size_t)tr * F.nnodes;
            const float *u = F.U ? F.U + (size_t)tr * F.d : nullptr;
            const float w2 = u ? w2s[tr] : 0.f;
            const int lv = 31 - __clz(lane + 1);  // lane's level in the subtree (lanes 0..30)
            int j = top.node, nb = 0;
            while (j < nn) {
                const long long node = (((long long)j + 1) << lv) - 1 + (lane + 1 - (1 << lv));
                float qs_l = 0.f, v_l = 0.f;
                if (lane < 31 && node < nn) {
                    const int2 nd = __ldg(tnodes + node);
                    const float qx = __ldg(q + nd.x);
                    qs_l = u ? reflect_coord(qx, w2, __ldg(u + nd.x)) : qx;
                    v_l = __int_as_float(nd.y);
                }
                int bi = 0;  // breadth-first index of the current node in the loaded subtree
                for (int l = 0; l < 5 && j < nn; ++l) {
                    const float qs = __shfl_sync(FULL, qs_l, bi);
                    const float v = __shfl_sync(FULL, v_l, bi);
                    const bool left = qs < v;
                    if (lane == 0) {
                        PQE e;
                        e.key = pq_key(qs, v);
                        e.tree = tr;
                        e.node = left ? 2 * j + 2 : 2 * j + 1;
                        stage[nb] = e;
                    }
                    ++nb;
                    j = left ? 2 * j + 1 : 2 * j + 2;
                    bi = left ? 2 * bi + 1 : 2 * bi + 2;
                }
            }
            if (lane == 0) out[checked] = leaf_code(tr, j - nn, F.L);
            __syncwarp();
            ++checked;
            // the pushes go to B (its popped prefix dropped); keep only what later pops can take
            const int keep = max(0, budget - checked);
            bcnt = pq_merge(qb + bhead, bcnt - bhead, stage, nb, qb2, min(PQ_BCAP, keep), sorted);
            bhead = 0;
            PQE *tmp = qb; qb = qb2; qb2 = tmp;
            __syncwarp();
            if (bcnt > PQ_BCAP - 32) {  // the next pushes might not fit: B into A
                acnt = ahead + pq_merge_into(qa + ahead, acnt - ahead, qb, bcnt, keep);
                bcnt = 0;
            }
        }
        if (lane == 0) nleaves[qi] = checked;
        __syncwarp();
    }
}

}  // namespace

size_t gf_prio_smem_bytes(int budget, int T) { return prio_warp_bytes(budget, T); }

int gf_launch_prio_leaves(const gf_forest *F, const float *Q, int64_t m, int budget, unsigned *leaves,
                          int *nleaves, cudaStream_t st) {
    const int cap = budget + 64;
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t per_warp = prio_warp_bytes(budget, F->T);
    const int warps = (int)std::min<size_t>(PRIO_WARPS, (size_t)lim / per_warp);
    if (warps < 1) return gf_fail(GF_EUNSUPPORTED, "leaf budget %d needs %zu B of shared memory", budget, per_warp);
    const size_t smem = per_warp * warps;
    if (smem > 48 * 1024) GF_CUDA_TRY(cudaFuncSetAttribute(k_prio_leaves, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long blocks = std::min<long long>((m + warps - 1) / warps, (long long)F->num_sms * 16);
    k_prio_leaves<<<(unsigned)blocks, warps * 32, smem, st>>>(view_of(F), Q, m, budget, cap, leaves, nleaves);
    GF_CUDA_TRY(cudaGetLastError());
    return GF_OK;
}

extern "C" int gf_prio_leaves(const gf_forest *F, const float *Q, int64_t m, int32_t checks, double eps,
                              uint32_t *leaves, int32_t *nleaves, int32_t stride, void *stream) {
    GfRange range("gf_prio_leaves");
    if (!F) return gf_fail(GF_EINVAL, "gf_prio_leaves: null forest");
    if (m < 0 || checks < 0 || !(eps >= 0.0)) return gf_fail(GF_EINVAL, "gf_prio_leaves: bad arguments");
    if (m == 0) return GF_OK;
    if (!Q || !leaves || !nleaves) return gf_fail(GF_EINVAL, "gf_prio_leaves: null pointer");
    if (((unsigned long long)F->T << F->L) > 0xffffffffull)
        return gf_fail(GF_EUNSUPPORTED, "priority search needs T * 2^L <= 2^32");
    const int lb = leaf_budget_of(F, checks, eps);
    const int budget = lb > 0 ? lb : F->T;
    if (budget > 4096) return gf_fail(GF_EUNSUPPORTED, "leaf budget %d above 4096", budget);
    if (stride != budget) return gf_fail(GF_EINVAL, "stride %d, the leaf budget is %d", stride, budget);
    return gf_launch_prio_leaves(F, Q, m, budget, leaves, nleaves, (cudaStream_t)stream);
}
