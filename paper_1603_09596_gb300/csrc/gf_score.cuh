// gf_score.cuh -- device helpers shared by the query kernels: 16-byte streaming loads, (distance,
// id) keys, block sorts, the packed float32 squared-L2 accumulation of every precision, warp-wide
// row distances and the float32 rerank, and the top-k writer.  Internal to the library.
#pragma once

#include "gf_internal.cuh"
#include "gf_device.cuh"

namespace {

using gfdev::FULL;
constexpr unsigned long long KEY_NONE = ~0ull;

__device__ __forceinline__ uint4 ld_u4(const void *p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long make_key(float dist, int id) {
    return ((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)id;
}

// ---------------------------------------------------------------- block helpers

// Ascending bitonic sort of a[0..P), P a power of two, by the whole block.
template <typename K>
__device__ void block_sort(K *a, int P) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const K x = a[lo], y = a[hi];
                const bool asc = (lo & size) == 0;
                if ((x > y) == asc) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- scoring

// Packed float32 pairs (Blackwell f32x2 instructions): each lane of a pair is rounded exactly as
// the scalar instruction would round it, so results are bit-identical to scalar arithmetic.
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float2 upk(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Squared-difference accumulation: a.c += (q.c - x.c)^2 for the four components, each a chain of
// its own (the order of the terms of every chain is fixed, whichever kernel runs it).
__device__ __forceinline__ void acc_pairs(float4 &a, unsigned long long q01, unsigned long long q23,
                                          unsigned long long x01, unsigned long long x23) {
    unsigned long long a01 = pk(a.x, a.y), a23 = pk(a.z, a.w);
    const unsigned long long e01 = sub2(q01, x01), e23 = sub2(q23, x23);
    a01 = fma2(e01, e01, a01);
    a23 = fma2(e23, e23, a23);
    const float2 r01 = upk(a01), r23 = upk(a23);
    a = make_float4(r01.x, r01.y, r23.x, r23.y);
}

__device__ __forceinline__ void acc4(float4 &a, const float4 q, const float4 x) {
    acc_pairs(a, pk(q.x, q.y), pk(q.z, q.w), pk(x.x, x.y), pk(x.z, x.w));
}

__device__ __forceinline__ float sum4(const float4 a) { return (a.x + a.y) + (a.z + a.w); }

// a bfloat16 pair (low half first) as two floats: the bf16 bits are the float's upper 16 bits
__device__ __forceinline__ unsigned long long bf16x2_f32x2(unsigned w) {
    return pk(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// bfloat16 chunk (8 values) against 8 query floats
__device__ __forceinline__ void acc_bf16(float4 &a, const float4 q0, const float4 q1, const uint4 c) {
    acc_pairs(a, pk(q0.x, q0.y), pk(q0.z, q0.w), bf16x2_f32x2(c.x), bf16x2_f32x2(c.y));
    acc_pairs(a, pk(q1.x, q1.y), pk(q1.z, q1.w), bf16x2_f32x2(c.z), bf16x2_f32x2(c.w));
}

__device__ __forceinline__ float2 e4m3x2_to_float2(unsigned short v) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)v, __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}

// FP8-E4M3 word (4 codes) times the row scale against 4 query floats: delta = q - s * c.
__device__ __forceinline__ void acc_fp8w(float4 &a, const float4 q, unsigned w, float s) {
    const float2 lo = e4m3x2_to_float2((unsigned short)(w & 0xffffu));
    const float2 hi = e4m3x2_to_float2((unsigned short)(w >> 16));
    const unsigned long long ns = pk(-s, -s);
    unsigned long long a01 = pk(a.x, a.y), a23 = pk(a.z, a.w);
    const unsigned long long e01 = fma2(ns, pk(lo.x, lo.y), pk(q.x, q.y));
    const unsigned long long e23 = fma2(ns, pk(hi.x, hi.y), pk(q.z, q.w));
    a01 = fma2(e01, e01, a01);
    a23 = fma2(e23, e23, a23);
    const float2 r01 = upk(a01), r23 = upk(a23);
    a = make_float4(r01.x, r01.y, r23.x, r23.y);
}

// Precision tags
constexpr int P_F32 = 0, P_BF16 = 1, P_FP8 = 2;

template <int PREC>
struct Prec {
    static constexpr int QF4 = PREC == P_F32 ? 1 : PREC == P_BF16 ? 2 : 4;  // query float4s per chunk
};

// Row pitch (bytes) and base pointer of the points in a precision; a chunk is 16 bytes.
template <int PREC>
__device__ __forceinline__ size_t row_pitch(const ForestView &F) {
    return PREC == P_F32 ? (size_t)F.ldx * 4 : PREC == P_BF16 ? (size_t)F.ldb * 2 : (size_t)F.ld8;
}

template <int PREC>
__device__ __forceinline__ const unsigned char *row_base(const ForestView &F) {
    return PREC == P_F32 ? (const unsigned char *)F.x
         : PREC == P_BF16 ? (const unsigned char *)F.xb : F.x8;
}

// Sort keys[0..C) (padding to a power of two) so the k nearest come first.
__device__ void sort_keys(unsigned long long *keys, int C) {
    int P = 1;
    while (P < C) P <<= 1;
    __syncthreads();
    for (int i = C + threadIdx.x; i < P; i += blockDim.x) keys[i] = KEY_NONE;
    block_sort<unsigned long long>(keys, P);
}

__device__ void write_topk(const unsigned long long *keys, int C, int k, long long *ids,
                           float *dists) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const unsigned long long key = i < C ? keys[i] : KEY_NONE;
        if (key == KEY_NONE) {
            ids[i] = -1;
            dists[i] = __int_as_float(0x7f800000);
        } else {
            ids[i] = (long long)(unsigned)(key & 0xffffffffu);
            dists[i] = __uint_as_float((unsigned)(key >> 32));
        }
    }
}

__host__ __device__ inline int ldq_of(int d) { return (d + 15) / 16 * 16; }

// the query row into shared memory as float32, zero-padded to ldq_of(d), by the whole block
__device__ void load_query(const float *q, int d, float *qs) {
    const int ldq = ldq_of(d);
    for (int j = threadIdx.x; j < ldq; j += blockDim.x) qs[j] = j < d ? q[j] : 0.f;
}

// Squared distances of the query (shared memory) to G rows at once, by the whole warp; every lane
// returns all G sums.  NC > 0: at most NC 16-byte chunks per lane; NC == 0: any row length.
template <int PREC, int NC, int G>
__device__ __forceinline__ void warp_dist_g(const ForestView &F, const float *qs, const int (&ids)[G],
                                            float (&d)[G]) {
    constexpr int QF4 = Prec<PREC>::QF4;
    const int lane = threadIdx.x & 31;
    const size_t pitch = row_pitch<PREC>(F);
    const int nch = (int)(pitch >> 4);
    const unsigned char *base = row_base<PREC>(F);
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
    float4 acc[G];
    float sc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        sc[g] = PREC == P_FP8 ? __ldg(F.scale8 + ids[g]) : 0.f;
    }
    constexpr int UB = NC > 0 ? NC : 2;
    for (int c0 = lane; c0 < nch; c0 += 32 * UB) {
        uint4 x[G][UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int cc = c0 + 32 * u;
            if (cc < nch) {
#pragma unroll
                for (int g = 0; g < G; ++g) x[g][u] = ld_u4(base + (size_t)ids[g] * pitch + ((size_t)cc << 4));
            }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int cc = c0 + 32 * u;
            if (cc < nch) {
                float4 qa[QF4];
#pragma unroll
                for (int h = 0; h < QF4; ++h) qa[h] = q4[cc * QF4 + h];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (PREC == P_F32) {
                        acc4(acc[g], qa[0], *reinterpret_cast<const float4 *>(&x[g][u]));
                    } else if (PREC == P_BF16) {
                        acc_bf16(acc[g], qa[0], qa[1], x[g][u]);
                    } else {
                        acc_fp8w(acc[g], qa[0], x[g][u].x, sc[g]);
                        acc_fp8w(acc[g], qa[1], x[g][u].y, sc[g]);
                        acc_fp8w(acc[g], qa[2], x[g][u].z, sc[g]);
                        acc_fp8w(acc[g], qa[3], x[g][u].w, sc[g]);
                    }
                }
            }
        }
        if (NC > 0) break;  // one pass covers the row
    }
#pragma unroll
    for (int g = 0; g < G; ++g) d[g] = warp_sum(sum4(acc[g]));
}

// float32 keys of rows ids[0..C) (all valid), G rows in flight per warp, query in shared memory
template <int NCF>
__device__ void rescore_f32(const ForestView &F, const float *qs, const int *ids, int C, unsigned long long *keys) {
    constexpr int G = (NCF >= 8) ? 2 : 4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j0 = w * G; j0 < C; j0 += nw * G) {
        int rid[G];
        float dd[G];
#pragma unroll
        for (int g = 0; g < G; ++g) rid[g] = ids[min(j0 + g, C - 1)];
        warp_dist_g<P_F32, NCF, G>(F, qs, rid, dd);
        if (lane == 0) {
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (j0 + g < C) keys[j0 + g] = make_key(dd[g], rid[g]);
        }
    }
}

}  // namespace
