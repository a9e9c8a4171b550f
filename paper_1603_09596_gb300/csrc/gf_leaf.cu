// gf_leaf.cu -- the leaf-major batched query path (GF_ALGO_LEAF): the one-leaf-per-tree search
// (Alg. 2 with c = T), bf16 screen + float32 rerank on the tensor cores or plain float32 on the CUDA
// cores (k_leaf_f32, further down), regrouped so that every leaf's points are read once per group
// of queries that reach it.
//
// A query's candidates are the points of the leaves it checks: one per tree (Eq. 1), or the leaves
// of Alg. 2's shared priority queue (the first descent of every tree, then pops: slot t < T of a
// query's list is tree t's first leaf); its answer is the k nearest of their union.  In a large
// batch many queries check the same leaf (10^4 queries over 2^10 leaves per tree: about ten each),
// and a per-query kernel reads that leaf's rows once per query.  Here:
//   1. the leaves: leaf[q][t] by descent, or the priority search's list of S leaves per query;
//   2. bucket the (query, slot) pairs by leaf (tree, leaf) (counting sort);
//   3. cut every bucket into chunks of at most NQ queries and order the chunks: those of tree 0
//      first, then the others by the smallest tree-0 leaf among their queries, so chunks of
//      different trees that cover the same region of the data run at about the same time and find
//      each other's rows in L2;
//   4. score (k_leaf_score): two persistent CTAs per SM walk the chunks.  A chunk's leaf rows are
//      staged in shared memory 128 at a time through a ring of 128-byte k-slices, each gathered by
//      its own producer warp, and multiplied against the chunk's queries on the tensor cores
//      (tcgen05.mma, M = 128 rows, N = the queries' hi and lo parts, bf16 inputs, float32
//      accumulators in tensor memory, issued by one thread of each CTA).  Leaves of at most 64
//      rows (the paper's leaf sizes, and the priority search's) pair up: two chunks share each row
//      tile, each with its own queries in the B operand.  The screened
//      score of point x for query q is |x~|^2 - 2 x~.q, which orders the points of one query as
//      |x~ - q|^2 does (the two differ by |q|^2).  x~ is the bf16 copy of the forest; the query
//      enters as two bf16 parts hi + lo (hi = bf16(q), lo = bf16(q - hi)), i.e. with about 16
//      significant bits, so the screen is the distance to the bf16 points, as in the other kernels.
//      Each (query, slot) keeps the R best (score, id) keys of its leaf that lie below the query's
//      bound tau_q, an upper bound on the R-th best key of the query's whole candidate union: the
//      R-th best key of any of its leaves is one.  The chunks of tree 0 run first (a launch of
//      their own) and set tau_q; every later chunk lowers it with its own R-th best (atomicMin).
//      Nothing in the union's R best is lost: such a key lies below tau_q and among the R best of
//      its leaf;
//   5. merge (k_leaf_merge): per query the keys of its S lists at or below its final bound are
//      de-duplicated by id, the R best screened ids are rescored in float32 (direct form, the same
//      code as the other kernels' rerank) and the k nearest are written in (distance, id) order.
// Results are those of the screened search of the other kernels: the screen ranks the query's
// candidate union, its R best are rescored exactly.  Screen scores near the shortlist boundary can
// order differently from another kernel's screen (different float32 rounding), as between any two
// screens.
//
// Waits on mbarriers are bounded (about two seconds).  A wait that runs out records
// GF_ETIMEOUT in a device status word (gf_kernel_status reads it), and every role of the CTA leaves
// its loop, lets its copies and tensor-core operations complete and frees its tensor memory.
#include "gf_internal.cuh"
#include "gf_device.cuh"
#include "gf_score.cuh"

#include <algorithm>
#include <atomic>
#include <climits>

__device__ int g_kernel_status = 0;  // first error a kernel of the library recorded

// gf_debug_set_wait_limit: the scoring kernel's wait limit in nanoseconds (0: WAIT_NS)
static std::atomic<unsigned long long> g_wait_limit_ns{0};

namespace {

constexpr int NQ = 16;           // queries per chunk (the MMA's N is QP NQ: the queries' parts)
constexpr int BM = 128;          // leaf rows per tile: the MMA's M, one tensor-memory lane each
constexpr int R_MAX = 32;        // longest shortlist per (query, tree): one key per lane
constexpr int EPI_THREADS = 128; // warps 0-3: tensor-memory lane quadrants 0-3
constexpr int MAX_KEYS = 8192;   // T * R limit of the merge

// Screen formats of the tensor-core scoring kernel.
//   bf16: the points' bf16 copy against the query's parts hi = bf16(q), lo = bf16(q - hi)
//         (kind::f16, K = 16 per MMA);
//   fp8:  the points' E4M3 codes (row scale s_x) against three E4M3 parts of the query with
//         scales c, c/16, c/256 (c a power of two, q ~ c (p0 + p1/16 + p2/256)): kind::f8f6f4,
//         K = 32 per MMA, so a row tile takes half the instructions and half the bytes.
constexpr int LF_BF16 = 0, LF_FP8 = 1;

// CPS: CTAs per SM, the kernel's shape (the autotuner's choice per forest and precision).
// CH: chunks per row tile.  Leaves of at most 64 rows (the paper's leaf sizes) would fill half a
// 128-row tile, so two chunks share every tile: rows 0-63 are one chunk's leaf, 64-127 the other's,
// and the B operand holds both chunks' queries (N doubles; an M = 128 MMA costs the same up to
// N = 64).  Each epilogue warp scores its rows against its own chunk's queries only.
template <int FMT, int CPS = 2, int CH = 1>
struct LeafCfg {
    static constexpr int QP = FMT == LF_FP8 ? 3 : 2;       // query parts
    static constexpr int ESZ = FMT == LF_FP8 ? 1 : 2;      // bytes per value
    static constexpr int NQT = NQ * CH;                    // query rows of a part in a tile
    static constexpr int ROWS_PER = BM / CH;               // tile rows of one chunk
    static constexpr int LW = 4 / CH;                      // epilogue warps (lists) per chunk
    // sub-tiles (128-byte k-slices) per stage -- one wait and one release each -- and stages, one
    // producer warp per sub-tile of the ring.  Two CTAs per SM (two MMA issuers and eight epilogue
    // warps per SM): rings of four (bf16) or three (E4M3) k-slices, 96 registers a thread.  One CTA
    // per SM: rings of nine (3 x 3, bf16) or eight (4 x 2, E4M3; a 960-value row fills it exactly),
    // 128 registers a thread.
    // With two chunks a tile (sub-tiles of 24 or 28 KB): rings of three (two CTAs) or of eight
    // (bf16) / seven (E4M3) k-slices (one CTA).
    static constexpr int SUB = CH == 2 || CPS == 2 ? 1 : FMT == LF_FP8 ? 2 : 3;
    static constexpr int STAGES = CH == 2 ? (CPS == 2 ? 3 : FMT == LF_FP8 ? 7 : 8)
                                          : CPS == 2 ? (FMT == LF_FP8 ? 3 : 4) : FMT == LF_FP8 ? 4 : 3;
    static constexpr int CTAS_PER_SM = CPS;
    // registers a thread: at most 65,536 / (CTAs x threads) and, per SM sub-partition (16,384
    // registers, every fourth warp of a CTA), 5 * 32 * 96 or 4 * 32 * 128
    static constexpr int REGS = CPS == 2 ? 96 : 128;
    static constexpr int PROD_WARPS = SUB * STAGES;  // producer warps; each loads whole sub-tiles
    static constexpr int A_BYTES = BM * 128;
    static constexpr int B_BYTES = NQT * 128;        // one query part of the tile's chunks
    static constexpr int SUBTILE_BYTES = A_BYTES + QP * B_BYTES;  // leaf rows, then the parts
    static constexpr int STAGE_BYTES = SUB * SUBTILE_BYTES;
    static constexpr int MMA_N = QP * NQT;           // the parts side by side
    static constexpr int ACC_COLS = MMA_N <= 64 ? 64 : 128;  // columns per accumulator
    static constexpr int TMEM_COLS = 2 * ACC_COLS;   // two accumulators
    static constexpr int MMA_WARP = 4 + PROD_WARPS;  // warps 4 .. 3 + PROD_WARPS load
    static constexpr int THREADS = (MMA_WARP + 1) * 32;
    // shared-memory plan (offsets from a 1024-aligned base)
    static constexpr int SM_WL = STAGES * STAGE_BYTES;            // the epilogue warps' lists [4][NQ][32]
    static constexpr int SM_SV = SM_WL + 4 * NQ * 32 * 8;         // a tile's x~.q~ [4][NQ][32] (float)
    static constexpr int SM_THR = SM_SV + 4 * NQ * 32 * 4;        // the lists' bounds [4][NQ]
    static constexpr int SM_BAR = SM_THR + 4 * NQ * 8;            // full[STAGES] empty[STAGES] dfull[2] dempty[2] fin
    static constexpr int SM_MISC = SM_BAR + (2 * STAGES + 5) * 8; // tensor-memory base, abort flag
    static constexpr int SMEM_BYTES = SM_MISC + 16 + 1024;        // slack for aligning the base
    // instruction descriptor: float32 D, A and B K-major, M = BM, N = MMA_N; bf16 inputs (kind::f16)
    // or E4M3 inputs (kind::f8f6f4, format code 0)
    static constexpr uint32_t IDESC = (1u << 4) | (FMT == LF_BF16 ? (1u << 7) | (1u << 10) : 0u) |
                                      ((uint32_t)(MMA_N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    static_assert(SUBTILE_BYTES % 1024 == 0, "sub-tiles must keep the 1024-byte swizzle alignment");
    static_assert(MMA_N % 16 == 0 && MMA_N <= ACC_COLS && MMA_N <= 256, "MMA shape");
    static_assert(CH == 1 || CH == 2, "one or two chunks a tile");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
    static_assert(CTAS_PER_SM * (SMEM_BYTES + 1024) <= 228 * 1024, "shared memory of the CTAs of one SM");
    static_assert(CPS == 1 || CPS == 2, "one or two CTAs per SM");
    static_assert(CTAS_PER_SM * THREADS * REGS <= 65536, "registers of the CTAs of one SM");
    static_assert((CTAS_PER_SM * THREADS / 32 + 3) / 4 * 32 * REGS <= 16384, "registers of one SM sub-partition");
};

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr uint64_t WAIT_NS = 2000000000ull;  // a wait gives up after about two seconds

// Wait for the phase of `parity` to complete.  Returns false (and raises the CTA's abort flag and
// the device status) if it did not within limit_ns, or if another role of the CTA aborted.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                            uint64_t limit_ns) {
    const uint64_t t0 = globaltimer();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_test(bar, parity)) return true;
        // the clock is read every 256 tries, or at every try under a limit shorter than the default
        // (a test limit of a few hundred nanoseconds must be able to run out)
        if ((spin & 255) == 0 || limit_ns < WAIT_NS) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > limit_ns) {
                *abort_flag = 1;
                atomicCAS(&g_kernel_status, 0, GF_ETIMEOUT);
                return false;
            }
            __nanosleep(64);
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns) {
    return mbar_test(bar, parity) || mbar_wait_slow(bar, parity, abort_flag, limit_ns);
}

// 16-byte global -> shared copy that reads `bytes` (0..16) bytes and zero-fills the rest
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// make this thread's completed generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzled layout: rows
// of 128 bytes (64 bf16), 16-byte chunk c of row r stored at chunk c ^ (r % 8), groups of 8 rows
// 1024 bytes apart; the tile starts on a 1024-byte boundary.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused by this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// The MMAs of one 128-byte k-slice (four steps of 32 bytes: K = 16 bf16 or 32 E4M3 values each):
// D (+)= A B^T, accumulating from the first unless `accumulate` is 0.  Descriptors advance 32 bytes
// (2 in units of 16) per step.  nk < 4 issues the first nk steps only (the row's end).
#define GF_MMA4(KIND)                                                                                          \
    asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %3, 0;\n setp.eq.b32 q, 0, 0;\n"                    \
                 " tcgen05.mma.cta_group::1.kind::" KIND " [%0], %1, %2, %4, p;\n"                           \
                 " tcgen05.mma.cta_group::1.kind::" KIND " [%0], %5, %6, %4, q;\n"                           \
                 " tcgen05.mma.cta_group::1.kind::" KIND " [%0], %7, %8, %4, q;\n"                           \
                 " tcgen05.mma.cta_group::1.kind::" KIND " [%0], %9, %10, %4, q;\n}" ::"r"(d_tmem),          \
                 "l"(a), "l"(b), "r"(accumulate), "r"(idesc), "l"(a + 2), "l"(b + 2), "l"(a + 4), "l"(b + 4), \
                 "l"(a + 6), "l"(b + 6)                                                                     \
                 : "memory")
#define GF_MMA1(KIND)                                                                                          \
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"                                             \
                 " tcgen05.mma.cta_group::1.kind::" KIND " [%0], %1, %2, %4, p;\n}" ::"r"(d_tmem),            \
                 "l"(a + 2 * i), "l"(b + 2 * i), "r"(i > 0 ? 1u : accumulate), "r"(idesc)                   \
                 : "memory")

template <int FMT, int CH>
__device__ __forceinline__ void mma_slice(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate, int nk) {
    constexpr uint32_t idesc = LeafCfg<FMT, 2, CH>::IDESC;
    if (nk >= 4) {
        if constexpr (FMT == LF_FP8) GF_MMA4("f8f6f4");
        else GF_MMA4("f16");
    } else {
        for (int i = 0; i < nk; ++i) {
            if constexpr (FMT == LF_FP8) GF_MMA1("f8f6f4");
            else GF_MMA1("f16");
        }
    }
}
#undef GF_MMA4
#undef GF_MMA1

// arrive on `bar` once every tensor-core operation this thread issued so far has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive float32 columns of this thread's tensor-memory lane (completed by tmem_wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory"); }

// barrier of the epilogue threads that also returns whether any of them passed `v` true, so that
// all of them take the same branch after it
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(EPI_THREADS)
        : "memory");
    return r != 0;
}

// float -> unsigned with the same order (negative values below positive ones)
__device__ __forceinline__ uint32_t ord_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------- per-warp key lists
//
// A list is the ascending sequence of the best keys seen so far, one key per lane: lane i holds
// entry i of the first RL lanes (RL = the shortlist rounded up to a power of two), KEY_NONE where
// the list is not full.

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a < b ? b : a; }

// ascending bitonic sort of one key per lane over the warp
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned long long y = __shfl_xor_sync(FULL, x, stride);
            const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
            x = keep_min ? umin64(x, y) : umax64(x, y);
        }
    }
    return x;
}

// The RL smallest keys of two ascending lists a and b, ascending.  min(a_i, b_{RL-1-i}) is the
// lower half of a bitonic merge: a bitonic sequence holding the RL smallest of a and b; the
// half-cleaners sort it.
__device__ __forceinline__ unsigned long long warp_merge_top(unsigned long long a, unsigned long long b, int RL) {
    const int lane = threadIdx.x & 31;
    const unsigned long long br = __shfl_sync(FULL, b, (RL - 1 - lane) & 31);
    unsigned long long c = lane < RL ? umin64(a, br) : KEY_NONE;
    for (int stride = RL >> 1; stride > 0; stride >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL, c, stride);
        c = (lane & stride) == 0 ? umin64(c, y) : umax64(c, y);
    }
    return c;
}

// Add the keys of the lanes in `bl` (all below the list's R-th key when the ballot was taken) to
// the list: one by one when they are few (eight or fewer), else sorted and merged.
__device__ __noinline__ unsigned long long list_add(unsigned long long lst, unsigned long long key, unsigned bl, int R,
                                                    int RL) {
    const int lane = threadIdx.x & 31;
    if (__popc(bl) > 8) return warp_merge_top(lst, warp_sort32((bl >> lane) & 1u ? key : KEY_NONE), RL);
    while (bl) {
        const int src = __ffs(bl) - 1;
        bl &= bl - 1;
        const unsigned long long kk = __shfl_sync(FULL, key, src);
        if (kk < __shfl_sync(FULL, lst, R - 1)) {
            const int pos = __popc(__ballot_sync(FULL, lane < RL && lst < kk));
            const unsigned long long up = __shfl_up_sync(FULL, lst, 1);
            if (lane < RL && lane > pos) lst = up;
            if (lane == pos) lst = kk;
        }
    }
    return lst;
}

// ---------------------------------------------------------------- the scoring kernel

struct LeafArgs {
    const int2 *items;     // (bucket, first query of the chunk)
    const int *item_lo;    // device: first item of this launch
    const int *item_hi;    // device: end of this launch's items
    const int *bcnt;       // queries per bucket
    const int *boff;       // first position of each bucket in qlist
    const int *qlist;      // (query, slot) pairs q S + s grouped by bucket
    const unsigned char *qpart;      // [QP][m][row] the query parts of the tensor-core screen:
                                     // bf16 hi, lo ([m][ldb]) or E4M3 p0, p1, p2 ([m][ld8])
    long long qpart_stride;          // bytes from one part to the next (m rows)
    const float *qc;                 // [m] E4M3 parts: the scale c of part 0 (a power of two)
    const float *qf;                 // [m][ldx] the queries, rows padded (float32 kernel)
    unsigned long long *part;        // [m][S][R] keys of every (query, slot)
    unsigned long long *tau;         // [m] upper bound on each query's R-th best key
    int R;
    int S;                           // slots (leaves) per query: T, or the priority search's budget
    unsigned long long wait_ns;      // time limit of the pipeline's mbarrier waits
};

__device__ __forceinline__ void chunk_of(const ForestView &F, const LeafArgs &A, int w, int &t, long long &lo,
                                         int &rows, int &q0pos, int &nq) {
    const int2 it = A.items[w];
    const int u = it.x;
    t = u >> F.L;
    const int b = u & ((1 << F.L) - 1);
    lo = ((long long)b * F.n) >> F.L;
    rows = (int)((((long long)(b + 1) * F.n) >> F.L) - lo);
    q0pos = A.boff[u] + it.y;
    nq = min(NQ, A.bcnt[u] - it.y);
}

template <int FMT, int CPS, int CH>
__global__ void __maxnreg__((LeafCfg<FMT, CPS, CH>::REGS)) k_leaf_score(ForestView F, LeafArgs A) {
    using Cfg = LeafCfg<FMT, CPS, CH>;
    constexpr int NQT = Cfg::NQT, ROWS_PER = Cfg::ROWS_PER, LW = Cfg::LW;
    constexpr int QP = Cfg::QP, SUB = Cfg::SUB, STAGES = Cfg::STAGES, PROD_WARPS = Cfg::PROD_WARPS;
    constexpr int A_BYTES = Cfg::A_BYTES, B_BYTES = Cfg::B_BYTES, SUBTILE_BYTES = Cfg::SUBTILE_BYTES;
    constexpr int STAGE_BYTES = Cfg::STAGE_BYTES, MMA_WARP = Cfg::MMA_WARP, ACC_COLS = Cfg::ACC_COLS;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned long long *wl = reinterpret_cast<unsigned long long *>(sm + Cfg::SM_WL);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + Cfg::SM_BAR);
    uint64_t *empty = full + STAGES;
    uint64_t *dfull = empty + STAGES;
    uint64_t *dempty = dfull + 2;
    uint64_t *fin = dempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + Cfg::SM_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + Cfg::SM_MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 32 * SUB);  // the lanes of the stage's SUB producer warps
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(dfull + b, 1);
            mbar_init(dempty + b, EPI_THREADS);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {  // the MMA warp owns the tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int item_lo = *A.item_lo, item_hi = *A.item_hi;
    // bytes of a row that hold values, and of a padded row
    const int row_bytes = F.d * Cfg::ESZ;
    const int pitch = FMT == LF_FP8 ? F.ld8 : F.ldb * 2;
    const unsigned char *xrows = FMT == LF_FP8 ? F.x8 : reinterpret_cast<const unsigned char *>(F.xb);
    const int KC = (row_bytes + SUB * 128 - 1) / (SUB * 128);  // stages per row tile
    const uint32_t stage0 = smem_u32(sm);

    if (warp >= 4 && warp < MMA_WARP) {
        // ------------------------------------------------ producers: leaf rows and query parts
        // Sub-tile h = SUB g + u of the CTA's stream (stage g, k-slice u) belongs to producer warp
        // h % PROD_WARPS.  The warp copies the whole sub-tile (lane: one 16-byte column chunk of
        // every fourth row), waits for its own copies, makes them visible to the tensor cores and
        // arrives on the stage's full barrier: no sub-tile waits for another one's copies.
        // A warp always fills the same ring slot (PROD_WARPS sub-tiles make one turn of the ring), so
        // the query parts it copied last are still there: when a row tile takes exactly one turn of
        // the ring (a row of as many k-slices as the ring holds), every later tile of the chunk finds
        // its k-slice's parts in place and the warp copies the leaf rows alone.
        const int pw = warp - 4;
        const int c = lane & 7, r0 = lane >> 3;  // column chunk; rows r0, r0 + 4, ...
        uint32_t it = 0;                          // stages of the CTA's earlier units
        bool ok = true;
        int held_w = -1, held_k = -1;             // unit and k-slice of the query parts in the slot
        // a unit: the CH consecutive chunks item_lo + wu CH + (0 .. CH-1) that share its row tiles
        for (int wu = blockIdx.x; item_lo + wu * CH < item_hi && ok; wu += gridDim.x) {
            int t[CH], rows[CH], q0pos[CH], nq[CH];
            long long lo[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                t[q] = rows[q] = q0pos[q] = nq[q] = 0;
                lo[q] = 0;
                if (item_lo + wu * CH + q < item_hi) chunk_of(F, A, item_lo + wu * CH + q, t[q], lo[q], rows[q], q0pos[q], nq[q]);
            }
            // B row j = r0 + 4 i: query j % NQ of chunk j / NQ (= i / 4, as r0 < 4)
            int qid[NQT / 4];
#pragma unroll
            for (int i = 0; i < NQT / 4; ++i) {
                const int q = i / 4, j = r0 + 4 * (i % 4);
                qid[i] = j < nq[q] ? A.qlist[q0pos[q] + j] / A.S : -1;
            }
            const int nst = (CH == 1 ? (rows[0] + BM - 1) / BM : 1) * KC * SUB;  // the unit's sub-tiles
            int ids[BM / 4];  // point ids of the lane's rows of tile `cur`
            int cur = -1;
            for (int sh = (int)((pw + PROD_WARPS - it % PROD_WARPS) % PROD_WARPS); sh < nst; sh += PROD_WARPS) {
                const uint32_t h = it + sh;
                const uint32_t g = h / SUB, s = g % STAGES;
                const int st = sh / SUB, u = sh - st * SUB;
                const int mt = st / KC, kc = st - mt * KC;
                if (mt != cur) {
                    cur = mt;
                    // tile row r0 + 4 i: row r0 + 4 (i % (ROWS_PER / 4)) of chunk i / (ROWS_PER / 4)
#pragma unroll
                    for (int i = 0; i < BM / 4; ++i) {
                        const int q = i / (ROWS_PER / 4);
                        const int gr = mt * BM + r0 + 4 * (i % (ROWS_PER / 4));
                        ids[i] = gr < rows[q] ? __ldg(F.perm + (size_t)t[q] * F.n + lo[q] + gr) : -1;
                    }
                }
                if (!mbar_wait(empty + s, ((g / STAGES) & 1) ^ 1, abort_flag, A.wait_ns)) { ok = false; break; }
                const int kbyte = (kc * SUB + u) * 128;
                if (kbyte >= row_bytes) {  // past the row: nothing to load, the MMA skips this sub-tile
                    mbar_arrive(full + s);
                    continue;
                }
                const int col = kbyte + c * 16;
                const int nb = max(0, min(16, row_bytes - col));
                const uint32_t sa = stage0 + s * STAGE_BYTES + u * SUBTILE_BYTES;
#pragma unroll
                for (int i = 0; i < BM / 4; ++i) {
                    const int r = r0 + 4 * i;
                    const bool live = ids[i] >= 0 && nb > 0;
                    const unsigned char *src = live ? xrows + (size_t)ids[i] * pitch + col : xrows;
                    cp_async16(sa + r * 128 + ((c ^ (r & 7)) << 4), src, live ? nb : 0);
                }
                if (held_w != wu || held_k != kbyte) {
                    held_w = wu;
                    held_k = kbyte;
#pragma unroll
                    for (int h = 0; h < QP; ++h) {
                        const unsigned char *qb = A.qpart + h * A.qpart_stride;
#pragma unroll
                        for (int i = 0; i < NQT / 4; ++i) {
                            const int j = r0 + 4 * i;
                            const bool live = qid[i] >= 0 && nb > 0;
                            const unsigned char *src = live ? qb + (size_t)qid[i] * pitch + col : qb;
                            cp_async16(sa + A_BYTES + h * B_BYTES + j * 128 + ((c ^ (j & 7)) << 4), src, live ? nb : 0);
                        }
                    }
                }
                cp_async_commit();
                cp_async_wait<0>();
                fence_proxy_async();
                mbar_arrive(full + s);
            }
            it += nst;
        }
        cp_async_wait<0>();
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------ MMA issue (one thread)
        if (lane == 0) {
            uint32_t tile = 0, s = 0, ph = 0;  // next stage slot and the parity of its fill
            bool ok = true;
            const uint64_t da0 = sdesc_sw128(stage0);            // stage 0's leaf rows
            const uint64_t db0 = sdesc_sw128(stage0 + A_BYTES);  // stage 0's query parts
            for (int wu = blockIdx.x; item_lo + wu * CH < item_hi && ok; wu += gridDim.x) {
                int MT = 1;  // two chunks a tile: leaves of at most 64 rows, one tile
                if (CH == 1) {
                    int t, rows, q0pos, nq;
                    long long lo;
                    chunk_of(F, A, item_lo + wu, t, lo, rows, q0pos, nq);
                    MT = (rows + BM - 1) / BM;
                }
                for (int mt = 0; mt < MT && ok; ++mt, ++tile) {
                    const uint32_t buf = tile & 1;
                    if (!mbar_wait(dempty + buf, ((tile >> 1) & 1) ^ 1, abort_flag, A.wait_ns)) { ok = false; break; }
                    tc_fence_after();  // the epilogue's reads of this accumulator are done
                    const uint32_t d_tmem = tmem_base + buf * ACC_COLS;
                    for (int kc = 0; kc < KC; ++kc) {
                        if (!mbar_wait(full + s, ph, abort_flag, A.wait_ns)) { ok = false; break; }
#pragma unroll
                        for (int u = 0; u < SUB; ++u) {
                            const int kbyte = (kc * SUB + u) * 128;
                            if (kbyte >= row_bytes) break;
                            const uint64_t off = (uint64_t)((s * STAGE_BYTES + u * SUBTILE_BYTES) >> 4);
                            mma_slice<FMT, CH>(d_tmem, da0 + off, db0 + off, (kc | u) != 0, (row_bytes - kbyte + 31) >> 5);
                        }
                        mma_commit(empty + s);
                        if (++s == STAGES) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(dfull + buf);
                }
            }
            // every issued operation has completed before the tensor memory is freed (the full
            // limit, whatever the pipeline waits were given)
            mma_commit(fin);
            volatile int no_abort = 0;
            mbar_wait_slow(fin, 0, &no_abort, WAIT_NS);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue: screened keys, R best per query
        // Each warp keeps, for every query of its chunk, the list of the R best keys of its own
        // 32 rows of every tile (in shared memory, with the list's bound: its R-th key or tau_q);
        // the chunk's LW lists are merged when the chunk is done.  A tile's scores go through
        // shared memory too, so that the query loop is a short rolled loop (four queries a turn)
        // and not one unrolled copy per query.
        const int et = tid;  // tile row and tensor-memory lane
        const int cw = warp / LW, wi = warp % LW;  // the chunk of the warp's rows; the warp's rank in it
        const int R = A.R;
        int RL = 1;
        while (RL < R) RL <<= 1;
        float *sv = reinterpret_cast<float *>(sm + Cfg::SM_SV) + warp * NQ * 32;  // [NQ][lane]
        unsigned long long *sl = wl + warp * NQ * 32;                             // [NQ][lane]
        unsigned long long *sthr = reinterpret_cast<unsigned long long *>(sm + Cfg::SM_THR) + warp * NQ;
        uint32_t tile = 0;
        bool ok = true;
        for (int wu = blockIdx.x; item_lo + wu * CH < item_hi; wu += gridDim.x) {
            int t = 0, rows = 0, q0pos = 0, nq = 0;  // an absent second chunk: no rows, no queries
            long long lo = 0;
            if (item_lo + wu * CH + cw < item_hi) chunk_of(F, A, item_lo + wu * CH + cw, t, lo, rows, q0pos, nq);
            // lane j: query j of the chunk, its bound and (E4M3 parts) the scale of its part 0
            const int my_qid = lane < nq ? A.qlist[q0pos + lane] / A.S : 0;
            const unsigned long long my_tau = lane < nq ? __ldcg(A.tau + my_qid) : KEY_NONE;
            const float my_c = FMT == LF_FP8 && lane < nq ? __ldg(A.qc + my_qid) : 1.f;
            for (int j = 0; j < nq; ++j) sl[j * 32 + lane] = KEY_NONE;
            if (lane < nq) sthr[lane] = my_tau;
            __syncwarp();
            const int MT = CH == 1 ? (rows + BM - 1) / BM : 1;  // the MMA's tiles of this unit
            for (int mt = 0; mt < MT && ok; ++mt, ++tile) {
                const int r = mt * BM + et - cw * ROWS_PER;  // the lane's row of its chunk's leaf
                const bool valid = r < rows;
                const int id = valid ? __ldg(F.perm + (size_t)t * F.n + lo + r) : 0;
                // |x~|^2 and the factor of x~.q in the score: -2 (bf16), -2 s_x (E4M3 codes)
                const float xn = valid ? __ldg(FMT == LF_FP8 ? F.x8n + id : F.xbn + id) : 0.f;
                const float kx = FMT == LF_FP8 ? (valid ? -2.f * __ldg(F.scale8 + id) : 0.f) : -2.f;
                const uint32_t buf = tile & 1;
                if (!mbar_wait(dfull + buf, (tile >> 1) & 1, abort_flag, A.wait_ns)) ok = false;
                ok = __all_sync(FULL, ok);
                if (!ok) break;
                tc_fence_after();
                const uint32_t ta = tmem_base + ((uint32_t)(warp * 32) << 16) + buf * ACC_COLS;
                {
                    uint32_t acc[QP][16];
#pragma unroll
                    for (int p = 0; p < QP; ++p) tmem_ld16(ta + p * NQT + cw * NQ, acc[p]);
                    tmem_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float v;  // x~ . q~ of the lane's row for query i (codes for E4M3)
                        if (FMT == LF_FP8)  // p0 + p1 / 16 + p2 / 256 (exact scalings)
                            v = __uint_as_float(acc[0][i]) +
                                fmaf(__uint_as_float(acc[2][i]), 1.f / 16.f, __uint_as_float(acc[1][i])) * (1.f / 16.f);
                        else
                            v = __uint_as_float(acc[0][i]) + __uint_as_float(acc[1][i]);
                        sv[i * 32 + lane] = v;
                    }
                }
                tc_fence_before();
                mbar_arrive(dempty + buf);
                // the queries four at a time: their keys and ballots first, then the (rare) list
                // insertions
                constexpr int QB = 4;
#pragma unroll 1
                for (int j0 = 0; j0 < nq; j0 += QB) {
                    unsigned long long key[QB];
                    unsigned bl[QB];
#pragma unroll
                    for (int b = 0; b < QB; ++b) {
                        const int j = min(j0 + b, NQ - 1);
                        // screened score |x~|^2 - 2 x~.q~; for E4M3 -2 s_x c is a power-of-two
                        // multiple of s_x, so the product is exact
                        const float kj = FMT == LF_FP8 ? kx * __shfl_sync(FULL, my_c, j) : kx;
                        const float s = fmaf(kj, sv[j * 32 + lane], xn);
                        key[b] = valid ? (((unsigned long long)ord_f32(s) << 32) | (unsigned)id) : KEY_NONE;
                        bl[b] = __ballot_sync(FULL, j0 + b < nq && key[b] < sthr[j]);
                    }
#pragma unroll
                    for (int b = 0; b < QB; ++b) {
                        if (bl[b]) {
                            const int j = j0 + b;
                            const unsigned long long nl = list_add(sl[j * 32 + lane], key[b], bl[b], R, RL);
                            sl[j * 32 + lane] = nl;
                            const unsigned long long kth = __shfl_sync(FULL, nl, R - 1);
                            if (lane == 0) sthr[j] = umin64(sthr[j], kth);
                            __syncwarp();
                        }
                    }
                }
            }
            // all four warps are done with the unit's lists; the warps of each chunk merge its LW
            if (epi_any(!ok)) break;
            for (int j = wi; j < nq; j += LW) {
                const unsigned long long *lw0 = wl + (size_t)(cw * LW) * NQ * 32;  // the chunk's first list
                unsigned long long a = lw0[(0 * NQ + j) * 32 + lane], b = lw0[(1 * NQ + j) * 32 + lane];
                unsigned long long c = LW == 4 ? lw0[(2 * NQ + j) * 32 + lane] : KEY_NONE;
                unsigned long long d = LW == 4 ? lw0[(3 * NQ + j) * 32 + lane] : KEY_NONE;
                if (lane >= RL) a = b = c = d = KEY_NONE;
                const unsigned long long best =
                    LW == 4 ? warp_merge_top(warp_merge_top(a, b, RL), warp_merge_top(c, d, RL), RL)
                            : warp_merge_top(a, b, RL);
                const int pr = A.qlist[q0pos + j];
                if (lane < R) A.part[(size_t)pr * R + lane] = best;
                const unsigned long long kth = __shfl_sync(FULL, best, R - 1);
                if (lane == 0 && kth != KEY_NONE) atomicMin(A.tau + pr / A.S, kth);
            }
            epi_sync();  // the merges have read the lists before the next unit resets them
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(Cfg::TMEM_COLS)
                     : "memory");
}

// ---------------------------------------------------------------- float32 scoring (CUDA cores)
//
// The plain float32 search through the same regrouping: each chunk's leaf rows against its
// queries in the direct form sum_j (q_j - x_j)^2, float32 arithmetic (packed f32x2 pairs, rounded
// per lane as the scalar instructions), on the CUDA cores.  Row tiles of 256 rows: lane l of warp w
// owns rows 64 w + l and 64 w + 32 + l of the tile and accumulates every query of the chunk for
// them.  The rows stream through a two-stage cp.async ring of 32-float slabs (128 bytes per row);
// the 16-byte chunk c of row r sits at chunk c ^ (r & 7), so a warp's 16-byte loads of 32
// consecutive rows fall on distinct banks.  The queries' slabs sit beside them (a padded float32
// copy of the batch) and are read by broadcast.  Keys are (distance bits, id); the per-warp lists,
// the bound tau_q and the per-chunk merge are those of the bf16 kernel, with the k best kept per
// (query, tree); the lists are merged in the ring's memory, idle between chunks.
namespace f32k {
constexpr int THREADS = 128;
constexpr int CTAS_PER_SM = 3;
constexpr int ROWS = 256;
constexpr int KS = 32;                          // floats per slab: one 128-byte row segment
constexpr int STAGES = 2;
constexpr int X_BYTES = ROWS * KS * 4;          // the tile's rows of one slab
constexpr int Q_BYTES = NQ * KS * 4;            // the chunk's queries of one slab
constexpr int STAGE_BYTES = X_BYTES + Q_BYTES;
constexpr int WL_BYTES = 4 * NQ * 32 * 8;       // the four warps' lists
constexpr int SMEM = STAGES * STAGE_BYTES;
static_assert(THREADS / 8 == NQ, "copy duty: eight threads per query row");
static_assert(WL_BYTES <= SMEM, "the lists reuse the ring");
__device__ __forceinline__ int swz(int r, int c) { return c ^ (r & 7); }
}  // namespace f32k

__global__ void __launch_bounds__(f32k::THREADS, f32k::CTAS_PER_SM) k_leaf_f32(ForestView F, LeafArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *wl = reinterpret_cast<unsigned long long *>(smem_raw);  // between chunks only
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item_lo = *A.item_lo, item_hi = *A.item_hi;
    const int NS = (F.d + f32k::KS - 1) / f32k::KS;  // slabs per row tile
    const int R = A.R;
    int RL = 1;
    while (RL < R) RL <<= 1;
    const int cc = tid & 7, cr = tid >> 3;  // copy duty: 16-byte chunk cc of rows cr + 16 i, query cr
    const uint32_t sbase = smem_u32(smem_raw);
    for (int w = item_lo + blockIdx.x; w < item_hi; w += gridDim.x) {
        int t, rows, q0pos, nq;
        long long lo;
        chunk_of(F, A, w, t, lo, rows, q0pos, nq);
        const int ng = (nq + 3) >> 2;  // groups of four queries
        const int qid_c = cr < nq ? A.qlist[q0pos + cr] / A.S : -1;
        const int my_qid = lane < nq ? A.qlist[q0pos + lane] / A.S : 0;
        const unsigned long long my_tau = lane < nq ? __ldcg(A.tau + my_qid) : KEY_NONE;
        unsigned long long lst[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) lst[j] = KEY_NONE;
        const int *perm_leaf = F.perm + (size_t)t * F.n + lo;
        const int MT = (rows + f32k::ROWS - 1) / f32k::ROWS;
        for (int mt = 0; mt < MT; ++mt) {
            int ids[f32k::ROWS / 16];
#pragma unroll
            for (int i = 0; i < f32k::ROWS / 16; ++i) {
                const int r = mt * f32k::ROWS + cr + 16 * i;
                ids[i] = r < rows ? __ldg(perm_leaf + r) : -1;
            }
            auto load_slab = [&](int sl, int stg) {
                const int col = sl * f32k::KS + cc * 4;
                const int nbytes = max(0, min(16, (F.d - col) * 4));
                const uint32_t xs = sbase + stg * f32k::STAGE_BYTES;
#pragma unroll
                for (int i = 0; i < f32k::ROWS / 16; ++i) {
                    const int r = cr + 16 * i;
                    const bool live = ids[i] >= 0 && nbytes > 0;
                    const float *src = live ? F.x + (size_t)ids[i] * F.ldx + col : F.x;
                    cp_async16(xs + r * (f32k::KS * 4) + (f32k::swz(r, cc) << 4), src, live ? nbytes : 0);
                }
                {
                    const bool live = qid_c >= 0 && nbytes > 0;
                    const float *src = live ? A.qf + (size_t)qid_c * F.ldx + col : A.qf;
                    cp_async16(xs + f32k::X_BYTES + cr * f32k::KS * 4 + cc * 16, src, live ? nbytes : 0);
                }
                cp_async_commit();
            };
            unsigned long long acc[2][NQ];  // packed (even, odd) partial sums per (row, query)
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int j = 0; j < NQ; ++j) acc[a][j] = 0ull;
            // double buffer: slab sl + 1 is requested while slab sl is scored
            load_slab(0, 0);
            for (int sl = 0; sl < NS; ++sl) {
                if (sl + 1 < NS) load_slab(sl + 1, (sl + 1) & 1);
                else cp_async_commit();
                cp_async_wait<1>();
                __syncthreads();
                const unsigned char *xs = smem_raw + (sl & 1) * f32k::STAGE_BYTES;
                const float *qs = reinterpret_cast<const float *>(xs + f32k::X_BYTES);
                const int r0 = 64 * warp + lane, r1 = r0 + 32;
#pragma unroll 2
                for (int c4 = 0; c4 < f32k::KS / 4; ++c4) {
                    // four floats as two packed pairs (low half first): no repacking
                    const ulonglong2 x0 = *reinterpret_cast<const ulonglong2 *>(xs + r0 * (f32k::KS * 4) + (f32k::swz(r0, c4) << 4));
                    const ulonglong2 x1 = *reinterpret_cast<const ulonglong2 *>(xs + r1 * (f32k::KS * 4) + (f32k::swz(r1, c4) << 4));
                    const unsigned long long a01 = x0.x, a23 = x0.y, b01 = x1.x, b23 = x1.y;
#pragma unroll
                    for (int g = 0; g < NQ / 4; ++g) {
                        if (g < ng) {
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int j = 4 * g + jj;
                                const ulonglong2 qv = *reinterpret_cast<const ulonglong2 *>(qs + j * f32k::KS + c4 * 4);
                                const unsigned long long q01 = qv.x, q23 = qv.y;
                                unsigned long long e = sub2(q01, a01);
                                acc[0][j] = fma2(e, e, acc[0][j]);
                                e = sub2(q23, a23);
                                acc[0][j] = fma2(e, e, acc[0][j]);
                                e = sub2(q01, b01);
                                acc[1][j] = fma2(e, e, acc[1][j]);
                                e = sub2(q23, b23);
                                acc[1][j] = fma2(e, e, acc[1][j]);
                            }
                        }
                    }
                }
                __syncthreads();  // the stage is refilled two slabs later
            }
            // the tile's distances: the warp's 64 rows against every query of the chunk
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r = mt * f32k::ROWS + 64 * warp + 32 * a + lane;
                const bool valid = r < rows;
                const int id = valid ? __ldg(perm_leaf + r) : 0;
#pragma unroll
                for (int j = 0; j < NQ; ++j) {
                    if (j < nq) {
                        const float2 s = upk(acc[a][j]);
                        const unsigned long long key = valid ? make_key(s.x + s.y, id) : KEY_NONE;
                        const unsigned long long thr =
                            umin64(__shfl_sync(FULL, lst[j], R - 1), __shfl_sync(FULL, my_tau, j));
                        const unsigned bl = __ballot_sync(FULL, key < thr);
                        if (bl) lst[j] = list_add(lst[j], key, bl, R, RL);
                    }
                }
            }
        }
        // the chunk is done: merge the four warps' lists; each query's R best of this leaf
#pragma unroll
        for (int j = 0; j < NQ; ++j)
            if (j < nq) wl[(warp * NQ + j) * 32 + lane] = lst[j];
        __syncthreads();
        for (int j = warp; j < nq; j += 4) {
            unsigned long long a = wl[(0 * NQ + j) * 32 + lane], b = wl[(1 * NQ + j) * 32 + lane];
            unsigned long long c = wl[(2 * NQ + j) * 32 + lane], d = wl[(3 * NQ + j) * 32 + lane];
            if (lane >= RL) a = b = c = d = KEY_NONE;
            const unsigned long long best = warp_merge_top(warp_merge_top(a, b, RL), warp_merge_top(c, d, RL), RL);
            const int pr = A.qlist[q0pos + j];  // q S + slot
            if (lane < R) A.part[(size_t)pr * R + lane] = best;
            const unsigned long long kth = __shfl_sync(FULL, best, R - 1);
            if (lane == 0 && kth != KEY_NONE) atomicMin(A.tau + pr / A.S, kth);
        }
        __syncthreads();  // the lists are rewritten by the next chunk
    }
}

// q -> a float32 copy with rows padded to ldx (16-byte aligned rows for the copies)
__global__ void k_qpad(const float *__restrict__ Q, long long m, int d, int ldx, float *qf) {
    const long long total = m * ldx;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long i = g / ldx;
        const int j = (int)(g - i * ldx);
        qf[g] = j < d ? Q[i * d + j] : 0.f;
    }
}

// ---------------------------------------------------------------- batch regrouping

// The bucket (leaf code tree << L | leaf) of pair g = q S + s, or -1 when the query checks fewer
// than s + 1 leaves.  One leaf per tree: S = T and leaf[q T + t]; priority search: the list plist.
__device__ __forceinline__ int pair_code(long long g, int S, int L, const int *leaf, const unsigned *plist,
                                         const int *pn) {
    const long long q = g / S;
    const int sl = (int)(g - q * S);
    if (plist) return sl < pn[q] ? (int)plist[g] : -1;
    return (sl << L) + leaf[g];
}

// The leaf of tree 0 that query q reaches (slot 0 of either list).
__device__ __forceinline__ int leaf0_of(long long q, int S, int L, const int *leaf, const unsigned *plist) {
    return plist ? (int)(plist[q * S] & ((1u << L) - 1u)) : leaf[q * S];
}

struct PairSource {
    const int *leaf;       // [m][T] (one leaf per tree) or null
    const unsigned *plist; // [m][S] leaf codes in the order checked (priority search) or null
    const int *pn;         // [m] leaves in each list
    int S, L;
};

__global__ void k_pair_count(long long pairs, PairSource P, int *bcnt) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pairs) return;
    const int c = pair_code(g, P.S, P.L, P.leaf, P.plist, P.pn);
    if (c >= 0) atomicAdd(bcnt + c, 1);
}

__global__ void k_pair_fill(long long pairs, PairSource P, const int *__restrict__ boff, int *bfill, int *qlist) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pairs) return;
    const int c = pair_code(g, P.S, P.L, P.leaf, P.plist, P.pn);
    if (c >= 0) qlist[boff[c] + atomicAdd(bfill + c, 1)] = (int)g;
}

// Order key of a bucket (tree t = u >> L): in locality order 2^L * (t > 0) + the smallest tree-0
// leaf among its queries, in tree-major order the bucket itself.  Either way the buckets of tree 0
// take the keys below 2^L.
__device__ __forceinline__ int bucket_key(int u, const int *bcnt, const int *boff, const int *qlist,
                                          const PairSource &P, bool locality) {
    if (!locality) return u;
    int key = INT_MAX;
    for (int i = 0; i < bcnt[u]; ++i) key = min(key, leaf0_of(qlist[boff[u] + i] / P.S, P.S, P.L, P.leaf, P.plist));
    return ((u >> P.L) > 0 ? (1 << P.L) : 0) + key;
}

__global__ void k_item_count(int nb, const int *__restrict__ bcnt, const int *__restrict__ boff,
                             const int *__restrict__ qlist, PairSource P, int locality, int *kcnt) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nb || bcnt[u] == 0) return;
    atomicAdd(kcnt + bucket_key(u, bcnt, boff, qlist, P, locality), (bcnt[u] + NQ - 1) / NQ);
}

__global__ void k_item_fill(int nb, const int *__restrict__ bcnt, const int *__restrict__ boff,
                            const int *__restrict__ qlist, PairSource P, int locality,
                            const int *__restrict__ koff, int *kfill, int2 *items) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nb || bcnt[u] == 0) return;
    const int key = bucket_key(u, bcnt, boff, qlist, P, locality);
    const int n_it = (bcnt[u] + NQ - 1) / NQ;
    const int base = koff[key] + atomicAdd(kfill + key, n_it);
    for (int i = 0; i < n_it; ++i) items[base + i] = make_int2(u, i * NQ);
}

constexpr int SCAN_TILE = 4096;  // elements one CTA of k_scan_tiles scans (four a thread)

// Exclusive prefix sums within the tiles of a[0..N): off[i] = the sum of a over [i's tile start,
// i), tsum[b] = tile b's total.  Thread t takes four consecutive elements (coalesced loads); the
// thread sums are scanned by warp shuffles, then the 32 warp totals by warp 0.
__global__ void __launch_bounds__(1024) k_scan_tiles(const int *__restrict__ a, int N, int *off, int *tsum) {
    __shared__ int wsum[32];
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v[4], s = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[e] = base + e < N ? a[base + e] : 0;
        s += v[e];
    }
    int inc = s;  // inclusive scan of the warp's thread sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        wsum[lane] = x;  // inclusive over the warps
    }
    __syncthreads();
    int run = inc - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (base + e < N) off[base + e] = run;
        run += v[e];
    }
    if (threadIdx.x == 1023) tsum[blockIdx.x] = wsum[31];
}

// Adds each tile's offset toff[b] (the exclusive scan of the tile totals) to its elements, and
// writes off[N] = the total.
__global__ void __launch_bounds__(1024) k_scan_add(int N, int *off, const int *__restrict__ toff) {
    const int i = blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    const int add = toff[blockIdx.x];
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (i + e < N) off[i + e] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) off[N] = toff[gridDim.x];
}

// Exclusive prefix sum of a[0..N) into off[0..N], off[N] = total; one CTA of 1024 threads (the
// tile totals of k_scan_tiles).
__global__ void __launch_bounds__(1024) k_scan(const int *__restrict__ a, int N, int *off) {
    __shared__ int part[1024];
    const int per = (N + 1023) / 1024;
    const int beg = min(N, threadIdx.x * per), end = min(N, beg + per);
    int s = 0;
    for (int i = beg; i < end; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan of the thread sums
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int i = beg; i < end; ++i) {
        off[i] = run;
        run += a[i];
    }
    if (threadIdx.x == 1023) off[N] = part[1023];
}

// q -> (hi, lo): hi = bf16(q), lo = bf16(q - hi), zero in the row padding
__global__ void k_qsplit(const float *__restrict__ Q, long long m, int d, int ldb, __nv_bfloat16 *qhi,
                         __nv_bfloat16 *qlo) {
    const long long total = m * ldb;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long i = g / ldb;
        const int j = (int)(g - i * ldb);
        const float v = j < d ? Q[i * d + j] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        qhi[g] = h;
        qlo[g] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// q -> three E4M3 parts for the kind::f8f6f4 screen, one warp per query.  c = the smallest power of
// two with max_j |q_j| / c <= 448 (1 for a zero query); then part p holds e4m3_rne(r_p / c_p) with
// c_p = c / 16^p, r_0 = q and r_{p+1} = r_p - c_p p_p (exact in float32: c_p p_p holds the leading
// bits of r_p).  Rounding to E4M3 leaves at most 2^-4 of a value, or half a subnormal step
// (2^-10 c_p), so |r_{p+1}| <= max(2^-4 |r_p|, 2^-10 c_p): every part's values stay within +-448,
// and q = c (p_0 + p_1 / 16 + p_2 / 256) + e with |e_j| <= 2^-12 |q_j| + 2^-18 c.  Zero in the row
// padding.
__global__ void k_qsplit8(const float *__restrict__ Q, long long m, int d, int ld8, unsigned char *parts,
                          long long part_stride, float *qc) {
    const int lane = threadIdx.x & 31;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m;
         i += ((long long)gridDim.x * blockDim.x) >> 5) {
        const float *q = Q + i * d;
        float a = 0.f;
        for (int j = lane; j < d; j += 32) a = fmaxf(a, fabsf(q[j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(FULL, a, o));
        // the smallest power of two c with a / c <= 448
        float c = 1.f;
        if (a > 0.f) {
            int e;
            frexpf(a / 448.f, &e);  // a / 448 = f 2^e, f in [0.5, 1)
            c = ldexpf(1.f, e);
            if (a / ldexpf(1.f, e - 1) <= 448.f) c = ldexpf(1.f, e - 1);
        }
        if (lane == 0) qc[i] = c;
        for (int j = lane; j < ld8; j += 32) {
            float r = j < d ? q[j] : 0.f;
            float cp = c;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const __nv_fp8_storage_t b = __nv_cvt_float_to_fp8(r / cp, __NV_SATFINITE, __NV_E4M3);
                parts[p * part_stride + i * ld8 + j] = (unsigned char)b;
                const __half_raw hv = __nv_cvt_fp8_to_halfraw(b, __NV_E4M3);
                r = r - cp * __half2float(*reinterpret_cast<const __half *>(&hv));
                cp *= (1.f / 16.f);
            }
        }
    }
}

// ---------------------------------------------------------------- merge + rerank

// Per query: the keys of its S lists of R at or below its final bound tau_q (every key of the
// union's R best is) -> distinct ids -> the R best -> (screened keys: float32 rerank) -> k nearest.
// One CTA per query at a time.
template <int NCF>
__global__ void __launch_bounds__(128) k_leaf_merge(ForestView F, const float *__restrict__ Q, long long m, int k,
                                                    int R, int S, int rerank,
                                                    const unsigned long long *__restrict__ part,
                                                    const unsigned long long *__restrict__ tau, long long *ids,
                                                    float *dists) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TR = S * R;
    int Pmax = 2;
    while (Pmax < TR) Pmax <<= 1;
    unsigned long long *a = reinterpret_cast<unsigned long long *>(smem_raw);
    float *qs = reinterpret_cast<float *>(a + Pmax);
    int *sid = reinterpret_cast<int *>(qs + ldq_of(F.d));
    unsigned char *dup = reinterpret_cast<unsigned char *>(sid + R);  // [Pmax]
    __shared__ int nshort, nkeep;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (long long qi = blockIdx.x; qi < m; qi += gridDim.x) {
        const unsigned long long tq = tau[qi];
        if (threadIdx.x == 0) {
            nshort = 0;
            nkeep = 0;
        }
        __syncthreads();
        // the keys that can still be among the R best, as (id, score): the copies of an id
        // come together, its best score first.  Eight loads in flight a thread; a warp appends its
        // keepers with one atomic.
        const unsigned long long *pq = part + qi * TR;
        for (int base = 0; base < TR; base += blockDim.x * 8) {
            unsigned long long kv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * blockDim.x + threadIdx.x;
                kv[u] = i < TR ? __ldcs(pq + i) : KEY_NONE;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const unsigned long long key = kv[u];
                // (an id outside [0, n) is a list no scoring CTA wrote: its launch gave up a wait)
                const bool keep = key != KEY_NONE && key <= tq && (key & 0xffffffffull) < (unsigned long long)F.n;
                const unsigned bal = __ballot_sync(FULL, keep);
                if (bal) {
                    int at = 0;
                    if (lane == 0) at = atomicAdd(&nkeep, __popc(bal));
                    at = __shfl_sync(FULL, at, 0);
                    if (keep) a[at + __popc(bal & lt)] = (key << 32) | (key >> 32);
                }
            }
        }
        __syncthreads();
        const int n = nkeep;
        int P = 2;
        while (P < n) P <<= 1;
        for (int i = n + threadIdx.x; i < P; i += blockDim.x) a[i] = KEY_NONE;
        block_sort<unsigned long long>(a, P);
        // every id once, with its best score; back to (score, id) for the second sort
        for (int i = threadIdx.x; i < P; i += blockDim.x) dup[i] = i > 0 && (a[i] >> 32) == (a[i - 1] >> 32);
        __syncthreads();
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const unsigned long long v = a[i];
            a[i] = dup[i] ? KEY_NONE : ((v << 32) | (v >> 32));
        }
        block_sort<unsigned long long>(a, P);
        for (int i = threadIdx.x; i < R && i < P; i += blockDim.x) {
            if (a[i] != KEY_NONE) {
                sid[i] = (int)(unsigned)(a[i] & 0xffffffffu);
                atomicAdd(&nshort, 1);
            }
        }
        if (rerank) load_query(Q + qi * F.d, F.d, qs);
        __syncthreads();
        const int C = nshort;  // the valid keys are a prefix of the sorted list
        if (rerank) {
            // the shortlist's ids are in sid: the keys' buffer is free for the float32 scores
            rescore_f32<NCF>(F, qs, sid, C, a);
            sort_keys(a, C);
            write_topk(a, C, k, ids + qi * k, dists + qi * k);
        } else {  // the keys are float32 distances already, in order
            write_topk(a, C, k, ids + qi * k, dists + qi * k);
        }
        __syncthreads();
    }
}

size_t merge_smem(const gf_forest *F, int S, int R) {
    int P = 2;
    while (P < S * R) P <<= 1;
    return (size_t)P * 8 + (size_t)ldq_of(F->d) * 4 + (size_t)R * 4 + (size_t)P;
}

// ---------------------------------------------------------------- workspace

struct LeafWorkspace {
    size_t bcnt, bfill, kcnt, kfill, zero_end;  // counters, zeroed by every call
    size_t boff, koff, tsum, toff, leaf, pn, qlist, items, qpart, qc, part, tau, total;
    size_t qpart_stride;  // bytes per query part ([m] rows)
};

// S: leaves per query (T, or the priority search's budget)
LeafWorkspace leaf_workspace(const gf_forest *F, int64_t m, int S, int R, int order) {
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t nb = (size_t)F->T << F->L;
    const size_t nk = order == GF_ORDER_GIVEN ? nb : ((size_t)2 << F->L);
    const size_t pairs = (size_t)m * S;
    LeafWorkspace W;
    size_t o = 0;
    W.bcnt = o; o = al(o + nb * 4);
    W.bfill = o; o = al(o + nb * 4);
    W.kcnt = o; o = al(o + nk * 4);
    W.kfill = o; o = al(o + nk * 4);
    W.zero_end = o;
    W.boff = o; o = al(o + (nb + 1) * 4);
    W.koff = o; o = al(o + (nk + 1) * 4);
    const size_t nt = (std::max(nb, nk) + SCAN_TILE - 1) / SCAN_TILE;  // scan tiles
    W.tsum = o; o = al(o + nt * 4);
    W.toff = o; o = al(o + (nt + 1) * 4);
    W.leaf = o; o = al(o + pairs * 4);  // leaf[m][T] or the priority lists [m][S]
    W.pn = o; o = al(o + (size_t)m * 4);
    W.qlist = o; o = al(o + pairs * 4);
    W.items = o; o = al(o + pairs * 8);
    // the query parts: bf16 hi and lo [m][ldb], or three E4M3 parts [m][ld8] (and their scales),
    // or the float32 kernel's padded copy [m][ldx]; room for the largest
    W.qpart_stride = std::max((size_t)m * F->ldb * 2, al((size_t)m * F->ld8));
    W.qpart = o; o = al(o + std::max(3 * W.qpart_stride, (size_t)m * F->ldx * 4));
    W.qc = o; o = al(o + (size_t)m * 4);
    W.part = o; o = al(o + pairs * R * 8);
    W.tau = o; o = al(o + (size_t)m * 8);
    W.total = o;
    return W;
}

int order_of(int order) { return order == GF_ORDER_GIVEN ? GF_ORDER_GIVEN : GF_ORDER_LOCALITY; }

template <int FMT, int CPS, int CH>
cudaError_t leaf_smem_attr() {
    return cudaFuncSetAttribute(k_leaf_score<FMT, CPS, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                LeafCfg<FMT, CPS, CH>::SMEM_BYTES);
}

template <int FMT, int CPS, int CH>
void launch_score(const gf_forest *F, const LeafArgs &A, cudaStream_t st) {
    using Cfg = LeafCfg<FMT, CPS, CH>;
    k_leaf_score<FMT, CPS, CH><<<F->num_sms * Cfg::CTAS_PER_SM, Cfg::THREADS, Cfg::SMEM_BYTES, st>>>(view_of(F), A);
}

// the tensor-core kernel for a format, shape (CTAs per SM) and chunks per tile
template <int FMT>
cudaError_t score_attr(int cps, int ch) {
    return cps == 1 ? (ch == 2 ? leaf_smem_attr<FMT, 1, 2>() : leaf_smem_attr<FMT, 1, 1>())
                    : (ch == 2 ? leaf_smem_attr<FMT, 2, 2>() : leaf_smem_attr<FMT, 2, 1>());
}

template <int FMT>
void score_launch(int cps, int ch, const gf_forest *F, const LeafArgs &A, cudaStream_t st) {
    if (cps == 1) ch == 2 ? launch_score<FMT, 1, 2>(F, A, st) : launch_score<FMT, 1, 1>(F, A, st);
    else ch == 2 ? launch_score<FMT, 2, 2>(F, A, st) : launch_score<FMT, 2, 1>(F, A, st);
}

}  // namespace

const char *gf_leaf_unsupported(const gf_forest *F, int64_t m, int32_t k, int32_t precision, int32_t R,
                                const QueryExtra &x) {
    if (precision < GF_FP32 || precision > GF_FP8_RERANK) return "unknown precision";
    if (precision == GF_BF16_RERANK && (!F->xb || !F->xbn)) return "the forest has no bf16 copy";
    if (precision == GF_FP8_RERANK && (!F->x8 || !F->x8n)) return "the forest has no fp8 copy";
    if (x.ncand_out) return "candidate counts are reported by the streaming kernel only";
    const int S = x.leaf_budget > 0 ? x.leaf_budget : F->T;  // leaves per query
    if (x.leaf_budget > 0 && ((unsigned long long)F->T << F->L) > 0xffffffffull)
        return "the priority search needs T * 2^L <= 2^32";
    if (precision == GF_FP32) {
        if (k > R_MAX) return "the leaf-major float32 path keeps at most 32 per (query, leaf): k <= 32";
        R = k;
    }
    if (R < 1 || R > R_MAX) return "the leaf-major path keeps a shortlist of 1..32";
    if (k > R) return "k exceeds the shortlist";
    if ((int64_t)S * R > MAX_KEYS) return "(leaves per query) * R above 8192";
    if (((int64_t)F->T << F->L) > ((int64_t)1 << 22)) return "T * 2^L above 2^22 buckets";
    if (m * S > INT_MAX / 2) return "m * (leaves per query) above 2^30";
    return nullptr;
}

// The regrouping pays once leaves are shared: on average at least LEAF_MIN_SHARE queries per leaf.
constexpr int LEAF_MIN_SHARE = 4;

// Sharing is m S / (T 2^L) queries per (tree, leaf): m / 2^L for one leaf per tree, and for the
// priority search with S leaves a query as many as its budget spreads over the forest's leaves.
// The priority search's small leaves (the paper's p of a few dozen points) pair up in the
// tensor-core kernel's row tiles (at 10^6 x 960, p = 64, c = 512: 37.3 ms against 45.7 ms for the
// streaming kernel per 10^4 queries, bf16); the float32 kernel's 256-row tiles would stay mostly
// empty there, so float32 priority searches remain with the streaming kernel.
bool gf_leaf_preferred(const gf_forest *F, int64_t m, int32_t k, int32_t precision, int32_t R, const QueryExtra &x) {
    if (x.leaf_budget > 0 && precision == GF_FP32) return false;
    const int64_t S = x.leaf_budget > 0 ? x.leaf_budget : F->T;
    return gf_leaf_unsupported(F, m, k, precision, R, x) == nullptr &&
           m * S / ((int64_t)F->T << F->L) >= LEAF_MIN_SHARE;
}

int64_t gf_leaf_workspace_bytes(const gf_forest *F, int64_t m, int32_t precision, int32_t R, int32_t order,
                                int32_t leaf_budget) {
    // float32 keeps k <= 32 per (query, leaf): size for the most
    const int len = precision == GF_FP32 ? R_MAX : std::max(1, std::min(R, R_MAX));
    const int S = leaf_budget > 0 ? leaf_budget : F->T;
    return (int64_t)leaf_workspace(F, m, S, len, order_of(order)).total;
}

int gf_launch_leaf(const gf_forest *F, const float *Q, int64_t m, int32_t k, int32_t precision, int32_t R,
                   int32_t order, int32_t leaf_budget, cudaStream_t st, int64_t *ids, float *dists,
                   void *workspace, int64_t workspace_bytes, cudaEvent_t *events, int32_t ctas_per_sm) {
    order = order_of(order);
    const bool f32 = precision == GF_FP32;
    if (f32) R = k;  // the exact distances: the k best of every (query, leaf) suffice
    const bool prio = leaf_budget > 0;  // Alg. 2's priority search: a list of S leaves per query
    const int S = prio ? leaf_budget : F->T;
    const LeafWorkspace W = leaf_workspace(F, m, S, R, order);
    char *ws = (char *)workspace;
    bool own = false;
    if (ws) {
        if ((size_t)workspace_bytes < W.total)
            return gf_fail(GF_EINVAL, "workspace of %lld bytes, %zu needed", (long long)workspace_bytes, W.total);
    } else {
        cudaError_t e = cudaMallocAsync((void **)&ws, W.total, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return gf_fail(GF_ENOMEM, "leaf-major workspace of %zu bytes: %s", W.total, cudaGetErrorString(e));
        }
        own = true;
    }
    auto fail = [&](cudaError_t e, const char *what) {
        if (own) cudaFreeAsync(ws, st);
        return gf_cuda_fail(e, what);
    };
    int *bcnt = (int *)(ws + W.bcnt), *bfill = (int *)(ws + W.bfill);
    int *kcnt = (int *)(ws + W.kcnt), *kfill = (int *)(ws + W.kfill);
    int *boff = (int *)(ws + W.boff), *koff = (int *)(ws + W.koff);
    int *leaf = (int *)(ws + W.leaf), *pn = (int *)(ws + W.pn), *qlist = (int *)(ws + W.qlist);
    int2 *items = (int2 *)(ws + W.items);
    unsigned char *qpart = (unsigned char *)(ws + W.qpart);
    float *qc = (float *)(ws + W.qc);
    unsigned long long *part = (unsigned long long *)(ws + W.part);
    unsigned long long *tau = (unsigned long long *)(ws + W.tau);
    const int nb = F->T << F->L;
    const int nk = order == GF_ORDER_GIVEN ? nb : (2 << F->L);
    const long long pairs = (long long)m * S;
    const bool locality = order != GF_ORDER_GIVEN;

    cudaError_t e = cudaMemsetAsync(ws, 0, W.zero_end, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tau, 0xff, (size_t)m * 8, st);  // KEY_NONE: no bound yet
    if (e != cudaSuccess) return fail(e, "workspace memset");
    // the leaves of every query: the descents, or the priority search's lists
    int r = prio ? gf_launch_prio_leaves(F, Q, m, S, (unsigned *)leaf, pn, st) : gf_descend(F, Q, m, leaf, st);
    if (r) {
        if (own) cudaFreeAsync(ws, st);
        return r;
    }
    PairSource P;
    P.leaf = prio ? nullptr : leaf;
    P.plist = prio ? (const unsigned *)leaf : nullptr;
    P.pn = pn;
    P.S = S;
    P.L = F->L;
    const unsigned pg = (unsigned)((pairs + 255) / 256), bg = (unsigned)((nb + 255) / 256);
    int *tsum = (int *)(ws + W.tsum), *toff = (int *)(ws + W.toff);
    auto scan = [&](const int *a, int N, int *off) {  // exclusive scan: tiles, their totals, the offsets
        const int nt = (N + SCAN_TILE - 1) / SCAN_TILE;
        k_scan_tiles<<<nt, 1024, 0, st>>>(a, N, off, tsum);
        k_scan<<<1, 1024, 0, st>>>(tsum, nt, toff);
        k_scan_add<<<nt, 1024, 0, st>>>(N, off, toff);
    };
    k_pair_count<<<pg, 256, 0, st>>>(pairs, P, bcnt);
    scan(bcnt, nb, boff);
    k_pair_fill<<<pg, 256, 0, st>>>(pairs, P, boff, bfill, qlist);
    k_item_count<<<bg, 256, 0, st>>>(nb, bcnt, boff, qlist, P, locality, kcnt);
    scan(kcnt, nk, koff);
    k_item_fill<<<bg, 256, 0, st>>>(nb, bcnt, boff, qlist, P, locality, koff, kfill, items);
    // the queries as the scoring kernel reads them: the float32 kernel's padded copy, the bf16 parts
    // hi and lo, or the three E4M3 parts and their scales
    float *qf = (float *)qpart;
    const bool f8 = precision == GF_FP8_RERANK;
    if (f32) k_qpad<<<F->num_sms * 8, 256, 0, st>>>(Q, m, F->d, F->ldx, qf);
    else if (f8) k_qsplit8<<<F->num_sms * 8, 256, 0, st>>>(Q, m, F->d, F->ld8, qpart, (long long)W.qpart_stride, qc);
    else k_qsplit<<<F->num_sms * 8, 256, 0, st>>>(Q, m, F->d, F->ldb, (__nv_bfloat16 *)qpart,
                                                  (__nv_bfloat16 *)(qpart + W.qpart_stride));
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "leaf-major regrouping");

    // the tensor-core kernel's shape: one CTA per SM when the caller or the forest's tuning asks for
    // exactly one, else two
    const int cps = ctas_per_sm == 1 ? 1 : 2;
    // two chunks share a row tile when no leaf has more than 64 rows (half a tile)
    const int ch = ((F->n + (1ll << F->L) - 1) >> F->L) <= BM / 2 ? 2 : 1;
    e = f32 ? cudaFuncSetAttribute(k_leaf_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, f32k::SMEM)
        : f8 ? score_attr<LF_FP8>(cps, ch) : score_attr<LF_BF16>(cps, ch);
    if (e != cudaSuccess) return fail(e, "cudaFuncSetAttribute(leaf-major scoring)");
    LeafArgs A;
    A.items = items;
    A.bcnt = bcnt;
    A.boff = boff;
    A.qlist = qlist;
    A.qpart = qpart;
    A.qpart_stride = (long long)W.qpart_stride;
    A.qc = qc;
    A.qf = qf;
    A.part = part;
    A.tau = tau;
    A.R = R;
    A.S = S;
    const unsigned long long wl = g_wait_limit_ns.load();
    A.wait_ns = wl ? wl : WAIT_NS;
    // the chunks of tree 0 (keys below 2^L) set every query's bound; then all the others
    if (events && (e = cudaEventRecord(events[0], st)) != cudaSuccess) return fail(e, "cudaEventRecord");
    for (int wave = 0; wave < 2; ++wave) {
        A.item_lo = wave == 0 ? koff : koff + (1 << F->L);
        A.item_hi = wave == 0 ? koff + (1 << F->L) : koff + nk;
        if (f32) k_leaf_f32<<<F->num_sms * f32k::CTAS_PER_SM, f32k::THREADS, f32k::SMEM, st>>>(view_of(F), A);
        else if (f8) score_launch<LF_FP8>(cps, ch, F, A, st);
        else score_launch<LF_BF16>(cps, ch, F, A, st);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "leaf-major scoring launch");
    if (events && (e = cudaEventRecord(events[1], st)) != cudaSuccess) return fail(e, "cudaEventRecord");

    const size_t msmem = merge_smem(F, S, R);
    const unsigned mg = (unsigned)std::min<long long>(m, (long long)F->num_sms * 16);
    const int ncf = F->ldx / 4 <= 32 ? 1 : F->ldx / 4 <= 64 ? 2 : F->ldx / 4 <= 128 ? 4 : F->ldx / 4 <= 256 ? 8 : 0;
#define GF_MERGE(NCV)                                                                                    \
    if (ncf == NCV) {                                                                                    \
        if (msmem > 48 * 1024 &&                                                                         \
            (e = cudaFuncSetAttribute(k_leaf_merge<NCV>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                      (int)msmem)) != cudaSuccess)                                       \
            return fail(e, "cudaFuncSetAttribute(k_leaf_merge)");                                        \
        k_leaf_merge<NCV><<<mg, 128, msmem, st>>>(view_of(F), Q, m, k, R, S, !f32, part, tau, (long long *)ids, dists); \
    }
    GF_MERGE(1) GF_MERGE(2) GF_MERGE(4) GF_MERGE(8) GF_MERGE(0)
#undef GF_MERGE
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "k_leaf_merge launch");
    // a caller's workspace is handed back all zero, as the streaming kernel expects it
    if (!own && (e = cudaMemsetAsync(ws, 0, W.total, st)) != cudaSuccess) return fail(e, "workspace clear");
    if (own) cudaFreeAsync(ws, st);
    return GF_OK;
}

extern "C" int gf_debug_set_wait_limit(uint64_t ns) {
    g_wait_limit_ns.store(ns);
    return GF_OK;
}

extern "C" int gf_kernel_status(int32_t *status) {
    if (!status) return gf_fail(GF_EINVAL, "gf_kernel_status: null pointer");
    GF_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    const int zero = 0;
    GF_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_kernel_status, sizeof v));
    GF_CUDA_TRY(cudaMemcpyToSymbol(g_kernel_status, &zero, sizeof zero));
    *status = v;
    return GF_OK;
}
