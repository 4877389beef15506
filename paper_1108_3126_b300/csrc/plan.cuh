// plan.cuh -- device pieces of the length planner, shared by the planner
// kernels (kernels.cu) and the one-launch planned streaming kernel
// (stream.cu).  The planner is a counting sort of the strings by (class,
// length bucket), longest first within a class, so that the 32 lanes of a
// round walk strings of (nearly) equal length and finish together.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace rx {
namespace plan {

constexpr int kPlanThreads = 512;
constexpr int kPlanItems = 4;
constexpr int kPlanTile = kPlanThreads * kPlanItems;

// span = the string's length plus its start's offset in its 32-byte block:
// below 2 KiB the bucket is the number of 32-byte blocks the string
// touches, so the lanes of a round start and end their strings in the same
// iteration of the kernels' block loops
__device__ __forceinline__ int len_bucket(int64_t len) {
    if (len < 2048) return (int)((len + 31) >> 5);
    int lg = 63 - __clzll(len);  // >= 11
    int b = 128 + 4 * (lg - 11) + (int)((len >> (lg - 2)) & 3);
    return b < kLenBuckets ? b : kLenBuckets - 1;
}

// long_bytes: cached pairs longer than this go to kClsMemoLong
// mis: the strings buffer's address mod 32.  Invalid offsets (negative
// length) take the bucket of the empty string; the kernels reject them.
__device__ __forceinline__ int plan_key(const int64_t* off, const uint8_t* cls, long long i, long long long_bytes,
                                        int mis) {
    const int64_t o = off[i], len = off[i + 1] - o;
    int lb = len_bucket(len > 0 ? len + ((o + mis) & 31) : 0);
    int c = cls ? (int)cls[i] : 0;
    if (cls && c == kClsMemo && len > long_bytes) c = kClsMemoLong;
    return c * kLenBuckets + (kLenBuckets - 1 - lb);
}

// keys of the tile at `base` (-1 past hi); the loads are in flight together
__device__ __forceinline__ void plan_tile_keys(const int64_t* off, const uint8_t* cls, long long base, long long hi,
                                               long long long_bytes, int mis, int (&key)[kPlanItems]) {
#pragma unroll
    for (int k = 0; k < kPlanItems; k++) {
        const long long i = base + k * kPlanThreads + threadIdx.x;
        key[k] = i < hi ? plan_key(off, cls, i, long_bytes, mis) : -1;
    }
}

__device__ inline void plan_count(const int64_t* off, const uint8_t* cls, long long lo, long long hi,
                                  long long long_bytes, int mis, unsigned* sh) {
    for (long long base = lo; base < hi; base += kPlanTile) {
        int key[kPlanItems];
        plan_tile_keys(off, cls, base, hi, long_bytes, mis, key);
#pragma unroll
        for (int k = 0; k < kPlanItems; k++)
            if (key[k] >= 0) atomicAdd(&sh[key[k]], 1u);
    }
}

// exclusive scan of in[0..nbk) into out (shared memory), by the whole block
// (blockDim.x a multiple of 32, at most 1024)
__device__ inline void block_scan(const unsigned* __restrict__ in, int nbk, unsigned* out) {
    __shared__ unsigned wsum[32];
    const int nt = blockDim.x, nw = nt >> 5;
    const int per_t = (nbk + nt - 1) / nt;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    unsigned sum = 0;
    for (int j = 0; j < per_t; j++) {
        const int b = t * per_t + j;
        if (b < nbk) {
            const unsigned v = __ldcg(in + b);
            out[b] = v;
            sum += v;
        }
    }
    unsigned incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned w = lane < nw ? wsum[lane] : 0u, wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += v;
        }
        if (lane < nw) wsum[lane] = wi - w;
    }
    __syncthreads();
    unsigned run = wsum[wid] + incl - sum;
    for (int j = 0; j < per_t; j++) {
        const int b = t * per_t + j;
        if (b < nbk) {
            const unsigned v = out[b];
            out[b] = run;
            run += v;
        }
    }
    __syncthreads();
}

constexpr unsigned kBarrierSpins = 1u << 22;  // x >= 64 ns: about a quarter of a second

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of a cooperative launch on a counter that only grows: every
// block adds one and waits until the counter reaches `target` (gridDim.x for
// the first barrier on a zeroed counter, 2 * gridDim.x for the second, ...).
// The wait is bounded: a block that gives up counts one in *faults and gets
// false.
__device__ inline bool grid_barrier(unsigned* bar, unsigned target, unsigned* faults) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int good = 1;
        unsigned spins = 0;
        while (ld_acquire(bar) < target) {
            if (++spins > kBarrierSpins) {
                good = 0;
                atomicAdd(faults, 1u);
                break;
            }
            __nanosleep(64);
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace plan
}  // namespace rx
