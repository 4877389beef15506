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
#include <algorithm>

#include "kernels.cuh"
#include "steppers.cuh"

namespace rx {

namespace {

using namespace rx::dev;

__global__ void __launch_bounds__(256) k_batch(const BatchTab* __restrict__ tabs, const uint32_t* __restrict__ pair_tab,
                                               const uint32_t* __restrict__ perm, const unsigned* __restrict__ starts,
                                               long long n, const uint8_t* __restrict__ str,
                                               const int64_t* __restrict__ off, uint8_t* __restrict__ out,
                                               unsigned* __restrict__ queue) {
    __shared__ long long seg[kBatchClasses + 1];
    __shared__ long long tfirst[kBatchClasses + 1];
    if (threadIdx.x == 0) {
        for (int c = 0; c < kBatchClasses; c++) seg[c] = starts[c * kLenBuckets];
        seg[kBatchClasses] = n;
        long long acc = 0;
        for (int c = 0; c < kBatchClasses; c++) {
            tfirst[c] = acc;
            long long cnt = seg[c + 1] - seg[c];
            acc += (c == kClsWarp) ? cnt : (cnt + 31) / 32;
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, 256, 0);
    if (e != cudaSuccess) return e;
    long long grid = std::min<long long>((long long)std::max(per_sm, 1) * sm_count(), ((long long)n * 32 + 255) / 256);
    {
        ProfScope ps(st);
        k_batch<<<(unsigned)std::max<long long>(grid, 1), 256, 0, st>>>(tabs, pair_tab, perm, starts, (long long)n,
                                                                        str, off, out, queue);
    }
    return cudaGetLastError();
}

}  // namespace rx
