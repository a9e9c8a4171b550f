// gf_device.cuh -- device helpers shared by the build and the query kernels.
#pragma once

#include <cuda_runtime.h>

namespace gfdev {

constexpr unsigned FULL = 0xffffffffu;

// Aggregated shared-memory histogram increment (lanes with equal bins add once).
__device__ __forceinline__ void hist_add(unsigned *hist, unsigned bin, bool active) {
    const unsigned mask = __ballot_sync(FULL, active);
    if (!active) return;
    const unsigned peers = __match_any_sync(mask, bin);
    if ((threadIdx.x & 31) == (__ffs(peers) - 1)) atomicAdd(hist + bin, __popc(peers));
}

// Rank-h key (0-based) among keys[0..cnt) held in shared memory; keys are distinct.
static __device__ unsigned long long block_select(const unsigned long long *keys, int cnt, int h, unsigned *hist,
                                           unsigned long long *sh_pref, int *sh_h) {
    if (threadIdx.x == 0) { *sh_pref = 0ull; *sh_h = h; }
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const unsigned long long pref = *sh_pref;
        const int iters = (cnt + blockDim.x - 1) / blockDim.x;
        for (int it = 0; it < iters; ++it) {
            const int i = it * blockDim.x + threadIdx.x;
            bool act = false;
            unsigned bin = 0;
            if (i < cnt) {
                const unsigned long long k = keys[i];
                act = pass == 0 || ((k ^ pref) >> (shift + 8)) == 0ull;
                bin = (unsigned)(k >> shift) & 255u;
            }
            hist_add(hist, bin, act);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            // lane owns bins 8*lane .. 8*lane+7
            unsigned c[8], s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { c[q] = hist[8 * lane + q]; s += c[q]; }
            unsigned incl = s;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned before = incl - s;
            const unsigned hr = (unsigned)*sh_h;
            if (hr >= before && hr < incl) {
                unsigned acc = before;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (hr >= acc && hr < acc + c[q]) {
                        *sh_pref = pref | ((unsigned long long)(8 * lane + q) << shift);
                        *sh_h = (int)(hr - acc);
                    }
                    acc += c[q];
                }
            }
        }
        __syncthreads();
    }
    return *sh_pref;
}


}  // namespace gfdev
