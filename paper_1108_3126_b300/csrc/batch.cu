// batch.cu -- many (expression, string) pairs in one persistent launch.
//
// Every pair runs the lockstep machine of its own expression (Rathnayake &
// Thielecke, SOS 2011, Def 5.2; acceptance Def 5.3).  The pairs are ordered
// by (variant class, length) -- longest first within a class -- by the
// planner, and cut into warp tasks: one pair per task for the warp variant,
// 32 pairs of the same class per task otherwise, so every task is uniform
// in code path.  Warps of a persistent grid take tasks from a global
// counter until the queue is drained.  Tables are read from global memory
// (L1/L2 resident) since the lanes of a task may use different expressions.
//
// Long pairs with a cache of macro steps (kClsMemoLong) would make one lane
// the critical path of the whole launch, so a warp takes such a pair alone:
// its 32 lanes cut the string into 32 chunks; each lane runs every cache
// state over a short prefix of its chunk, then only the distinct states
// reached over the rest (the chunk's transfer function, exactly: a macro step
// acts on states, Def 5.2), and lane 0 composes the 32 functions from the
// start state.
#include <algorithm>

#include "kernels.cuh"
#include "steppers.cuh"

namespace rx {

namespace {

using namespace rx::dev;

constexpr int kPairPrefix = 32;
static_assert(kMemoMaxStates <= 256, "chunk maps hold cache state ids in one byte");

// one lane, bytes [s, e) (absolute addresses), cache state st (row offset
// in words), table T in global memory; stops when the set is empty
__device__ uint32_t lane_memo_run(const uint32_t* __restrict__ T, uint32_t st, uint64_t s, uint64_t e) {
    uint64_t blk = s & ~uint64_t(15);
    while (blk < e && st != 0) {
        uint4 v = ld_stream(reinterpret_cast<const uint8_t*>(blk));
#pragma unroll
        for (int k = 0; k < 16; k++) {
            uint64_t p = blk + k;
            if (p >= s && p < e) st = __ldg(T + st + byte_of(v, k));
        }
        blk += 16;
    }
    return st;
}

// one warp, one long pair: returns whether the pair matches (all lanes);
// wsm holds 32 chunk maps of `stride` bytes (stride >= memo_K)
__device__ bool warp_long_memo(const DevTables& t, uint64_t s, uint64_t e, uint8_t* wsm, int stride) {
    const int lane = threadIdx.x & 31;
    const int K = t.memo_K;
    const uint32_t* T = t.memo_T;
    const uint64_t L = e - s;
    const uint64_t C = ((L + 31) / 32 + 15) & ~uint64_t(15);
    uint64_t cs = s + (uint64_t)lane * C;
    if (cs > e) cs = e;
    uint64_t ce = cs + C < e ? cs + C : e;
    uint64_t cp = cs + kPairPrefix < ce ? cs + kPairPrefix : ce;
    uint8_t* map = wsm + lane * stride;
    // every incoming state over the prefix
    for (int k = 0; k < K; k++) map[k] = (uint8_t)(lane_memo_run(T, (uint32_t)k * 256u, cs, cp) >> 8);
    // the distinct states over the rest; a small cache of (state, result)
    uint32_t cv[8], cr[8];
    int nc = 0;
    for (int k = 0; k < K; k++) {
        uint32_t v = map[k], r = 0xffffffffu;
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nc && cv[q] == v) r = cr[q];
        if (r == 0xffffffffu) {
            r = lane_memo_run(T, v * 256u, cp, ce) >> 8;
            if (nc < 8) {
#pragma unroll
                for (int q = 0; q < 8; q++)
                    if (q == nc) {
                        cv[q] = v;
                        cr[q] = r;
                    }
                nc++;
            }
        }
        map[k] = (uint8_t)r;
    }
    __syncwarp();
    uint32_t acc = 0;
    if (lane == 0) {
        uint32_t x = t.memo_start >> 8;
        for (int l = 0; l < 32; l++) x = wsm[l * stride + x];
        acc = t.memo_acc[x];
    }
    __syncwarp();
    return __shfl_sync(FULL, acc, 0) != 0;
}

__global__ void __launch_bounds__(256) k_batch(const BatchTab* __restrict__ tabs, const uint32_t* __restrict__ pair_tab,
                                               const uint32_t* __restrict__ perm, const unsigned* __restrict__ starts,
                                               long long n, const uint8_t* __restrict__ str,
                                               const int64_t* __restrict__ off, uint8_t* __restrict__ out,
                                               unsigned* __restrict__ queue, int stride) {
    extern __shared__ __align__(16) uint8_t bsm[];  // 32 x stride bytes per warp
    __shared__ long long seg[kBatchClasses + 1];
    __shared__ long long tfirst[kBatchClasses + 1];
    if (threadIdx.x == 0) {
        for (int c = 0; c < kBatchClasses; c++) seg[c] = starts[c * kLenBuckets];
        seg[kBatchClasses] = n;
        long long acc = 0;
        for (int c = 0; c < kBatchClasses; c++) {
            tfirst[c] = acc;
            long long cnt = seg[c + 1] - seg[c];
            acc += (c == kClsWarp || c == kClsMemoLong) ? cnt : (cnt + 31) / 32;
        }
        tfirst[kBatchClasses] = acc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long ntasks = tfirst[kBatchClasses];
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(queue, 1u);
        task = __shfl_sync(FULL, task, 0);
        if ((long long)task >= ntasks) break;
        int c = 0;
        while (c + 1 < kBatchClasses && (long long)task >= tfirst[c + 1]) c++;
        const long long g = (long long)task - tfirst[c];
        if (c == kClsMemoLong) {
            const uint32_t p = perm[seg[c] + g];
            const DevTables& t = tabs[pair_tab[p]].t;
            const uint64_t s = base + (uint64_t)off[p], e = base + (uint64_t)off[p + 1];
            bool acc = warp_long_memo(t, s, e, bsm + (threadIdx.x >> 5) * 32 * stride, stride);
            if (lane == 0) out[p] = acc;
            continue;
        }
        if (c == kClsWarp) {
            const uint32_t p = perm[seg[c] + g];
            const DevTables& t = tabs[pair_tab[p]].t;
            const uint64_t s = base + (uint64_t)off[p], e = base + (uint64_t)off[p + 1];
            bool acc;
            if (t.W <= 32) acc = warp_string<1>(t, t.B, t.follow, s, e);
            else if (t.W <= 64) acc = warp_string<2>(t, t.B, t.follow, s, e);
            else acc = warp_string<4>(t, t.B, t.follow, s, e);
            if (lane == 0) out[p] = acc;
            continue;
        }
        const long long idx = seg[c] + g * 32 + lane;
        const bool valid = idx < seg[c + 1];
        const uint32_t p = valid ? perm[idx] : perm[seg[c]];
        const DevTables& t = tabs[pair_tab[p]].t;
        uint64_t s = base, e = base;
        if (valid) {
            s += (uint64_t)off[p];
            e += (uint64_t)off[p + 1];
        }
        switch (c) {
        case kClsMemo: {
            MemoStep st;
            st.bind_global(t);
            run_lane(st, s, e, valid, out + p);
            break;
        }
        case kClsThread1: {
            Thread1Step st;
            st.bind_global(t);
            run_lane(st, s, e, valid, out + p);
            break;
        }
        case kClsThread2: {
            Thread2Step st;
            st.bind_global(t);
            run_lane(st, s, e, valid, out + p);
            break;
        }
        case kClsSparse4: {
            SparseStep<4> st;
            st.bind_global(t);
            run_lane(st, s, e, valid, out + p);
            break;
        }
        default: {
            SparseStep<8> st;
            st.bind_global(t);
            run_lane(st, s, e, valid, out + p);
            break;
        }
        }
    }
}

}  // namespace

size_t batch_workspace_bytes(size_t n, size_t ntabs) {
    auto a = [](size_t x) { return (x + 255) & ~size_t(255); };
    return 256 + a(ntabs * sizeof(BatchTab)) + a(n * 4) + a(n) + plan_workspace_bytes(n, kBatchClasses);
}

cudaError_t launch_batch(const BatchTab* h_tabs, size_t ntabs, const uint32_t* h_pair_tab, const uint8_t* h_cls,
                         size_t n, const uint8_t* str, const int64_t* off, uint8_t* out, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
    // chunk maps of long pairs: 32 lanes x (largest cache over the batch's
    // expressions, rounded to 16) bytes per warp; none without a cache
    int stride = 0;
    for (size_t i = 0; i < ntabs; i++)
        stride = std::max(stride, (int)((h_tabs[i].t.memo_K + 15) & ~15));
    if (n == 0) return cudaSuccess;
    if (ws_bytes < batch_workspace_bytes(n, ntabs)) return cudaErrorInvalidValue;
    auto a = [](size_t x) { return (x + 255) & ~size_t(255); };
    uint8_t* w = static_cast<uint8_t*>(ws);
    unsigned* queue = reinterpret_cast<unsigned*>(w);
    BatchTab* tabs = reinterpret_cast<BatchTab*>(w + 256);
    uint32_t* pair_tab = reinterpret_cast<uint32_t*>(w + 256 + a(ntabs * sizeof(BatchTab)));
    uint8_t* cls = w + 256 + a(ntabs * sizeof(BatchTab)) + a(n * 4);
    void* plan_ws = w + 256 + a(ntabs * sizeof(BatchTab)) + a(n * 4) + a(n);
    cudaError_t e = cudaMemsetAsync(queue, 0, 256, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tabs, h_tabs, ntabs * sizeof(BatchTab), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pair_tab, h_pair_tab, n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cls, h_cls, n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    uint32_t* perm = nullptr;
    unsigned* starts = nullptr;
    e = launch_plan(off, cls, kBatchClasses, n, plan_ws, &perm, &starts, st, nullptr);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    const size_t sm = (size_t)8 * 32 * stride;  // at most 48 KiB (192 states)
    e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(sm, 1));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, 256, sm);
    if (e != cudaSuccess) return e;
    long long grid = std::min<long long>((long long)std::max(per_sm, 1) * sm_count(), ((long long)n * 32 + 255) / 256);
    {
        ProfScope ps(st);
        k_batch<<<(unsigned)std::max<long long>(grid, 1), 256, sm, st>>>(tabs, pair_tab, perm, starts, (long long)n,
                                                                         str, off, out, queue, stride);
    }
    return cudaGetLastError();
}

}  // namespace rx
