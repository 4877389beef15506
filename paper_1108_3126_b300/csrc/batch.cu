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
// the critical path of the whole launch, so a warp takes such a pair alone
// (as it does every pair of an expression with only the wide cache tier,
// kClsWide, whose sets are too wide for a lane):
// its 32 lanes cut the string into 32 chunks; each lane computes its chunk's
// transfer function on cache states (exact: a macro step acts on states,
// Def 5.2), merging incoming states that meet within a short prefix, and
// lane 0 composes the 32 functions from the start state.
#include <algorithm>

#include "kernels.cuh"
#include "steppers.cuh"

namespace rx {

namespace {

using namespace rx::dev;

// one warp, one long pair: whether the pair matches (all lanes)
__device__ bool warp_long_memo(const DevTables& t, uint64_t s, uint64_t e, uint8_t* wsm, int stride) {
    const uint32_t x = warp_chunked_memo(t, t.memo_start >> 8, s, e, wsm, stride);
    return t.memo_acc[x] != 0;
}

// the same on the wide tier (two-byte state ids); not inlined, so that its
// registers do not press on the other classes' paths
__device__ __noinline__ bool warp_long_wide(const DevTables& t, uint64_t s, uint64_t e, uint8_t* wsm, int stride) {
    const uint32_t x = warp_chunked_wide(t, t.wide_start, s, e, wsm, stride);
    return t.wide_acc[x] != 0;
}

// 64 registers per thread (two 512-thread blocks per SM); the chunk maps of
// long pairs live in a per-warp slot of global scratch (`maps`, 64 * stride
// bytes per resident warp), which keeps shared memory free for occupancy
__global__ void __launch_bounds__(512, 2) k_batch(const BatchTab* __restrict__ tabs, const uint32_t* __restrict__ pair_tab,
                                               const uint32_t* __restrict__ perm, const unsigned* __restrict__ starts,
                                               long long n, const uint8_t* __restrict__ str,
                                               const int64_t* __restrict__ off, uint8_t* __restrict__ out,
                                               unsigned* __restrict__ queue, int stride, uint8_t* __restrict__ maps,
                                               unsigned long long* __restrict__ bad) {
    __shared__ long long seg[kBatchClasses + 1];
    __shared__ long long tfirst[kBatchClasses + 1];
    if (threadIdx.x == 0) {
        for (int c = 0; c < kBatchClasses; c++) seg[c] = starts[c * kLenBuckets];
        seg[kBatchClasses] = n;
        long long acc = 0;
        for (int c = 0; c < kBatchClasses; c++) {
            tfirst[c] = acc;
            long long cnt = seg[c + 1] - seg[c];
            acc += warp_class(c) ? cnt : (cnt + 31) / 32;
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
        if (warp_class(c)) {
            // one pair per warp: an invalid pair is answered by lane 0
            const uint32_t p = perm[seg[c] + g];
            uint64_t s, e;
            if (!string_span(off, p, base, s, e)) {
                if (lane == 0) {
                    out[p] = kResultInvalid;
                    count_bad(bad);
                }
                continue;
            }
        }
        if (c == kClsMemoLong || c == kClsWide) {
            const uint32_t p = perm[seg[c] + g];
            const DevTables& t = tabs[pair_tab[p]].t;
            const uint64_t s = base + (uint64_t)off[p], e = base + (uint64_t)off[p + 1];
            const size_t slot = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
            uint8_t* wsm = maps + slot * 64 * (size_t)stride;
            const bool acc = c == kClsWide ? warp_long_wide(t, s, e, wsm, stride) : warp_long_memo(t, s, e, wsm, stride);
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
        bool valid = idx < seg[c + 1];
        const uint32_t p = valid ? perm[idx] : perm[seg[c]];
        const DevTables& t = tabs[pair_tab[p]].t;
        uint64_t s = base, e = base;
        bool ok = true;
        if (valid) {
            ok = string_span(off, p, base, s, e);
            if (!ok) {
                out[p] = kResultInvalid;
                count_bad(bad);
            }
        }
        valid = valid && ok;
        switch (c) {
        case kClsMemo: {
            MemoStep8 st;
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

namespace {
size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchWs {
    unsigned* queue;
    BatchTab* tabs;
    uint32_t* pair_tab;
    uint8_t* cls;
    void* plan_ws;
};

BatchWs batch_ws(void* ws, size_t n, size_t ntabs) {
    uint8_t* w = static_cast<uint8_t*>(ws);
    BatchWs b;
    b.queue = reinterpret_cast<unsigned*>(w);
    b.tabs = reinterpret_cast<BatchTab*>(w + 256);
    b.pair_tab = reinterpret_cast<uint32_t*>(w + 256 + a256(ntabs * sizeof(BatchTab)));
    b.cls = w + 256 + a256(ntabs * sizeof(BatchTab)) + a256(n * 4);
    b.plan_ws = w + 256 + a256(ntabs * sizeof(BatchTab)) + a256(n * 4) + a256(n);
    return b;
}
}  // namespace

size_t batch_workspace_bytes(size_t n, size_t ntabs) {
    return 256 + a256(ntabs * sizeof(BatchTab)) + a256(n * 4) + a256(n) + plan_workspace_bytes(n, kBatchClasses);
}

// chunk functions of long pairs: a row of 2 + K bytes per lane (K the
// largest cache over the batch's expressions; on the wide tier 2 + the
// largest column image two-byte ids), rounded to 16; none without a cache
int batch_stride(const BatchTab* h_tabs, size_t ntabs) {
    int stride = 0;
    for (size_t i = 0; i < ntabs; i++) {
        const DevTables& t = h_tabs[i].t;
        if (t.memo_K > 0) stride = std::max(stride, (int)((t.memo_K + 2 + 15) & ~15));
        else if (t.wide_K > 0) stride = std::max(stride, (int)((2 * (t.wide_maximg + 2) + 15) & ~15));
    }
    return stride;
}

cudaError_t batch_upload(const BatchTab* h_tabs, size_t ntabs, const uint32_t* h_pair_tab, const uint8_t* h_cls,
                         size_t n, void* ws, cudaStream_t st) {
    BatchWs b = batch_ws(ws, n, ntabs);
    cudaError_t e = cudaMemcpyAsync(b.tabs, h_tabs, ntabs * sizeof(BatchTab), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.pair_tab, h_pair_tab, n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.cls, h_cls, n, cudaMemcpyHostToDevice, st);
    return e;
}

// resident blocks per SM for this block size
cudaError_t batch_configure(BatchLaunch& L) {
    if (L.block != 128 && L.block != 256 && L.block != 512) return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, L.block, 0);
    if (e != cudaSuccess) return e;
    L.grid_cap = (long long)std::max(per_sm, 1) * sm_count();
    return cudaSuccess;
}

long long batch_grid(const BatchLaunch& L, size_t n) {
    return std::max<long long>(1, std::min<long long>(L.grid_cap, ((long long)n * 32 + L.block - 1) / L.block));
}

// global scratch for the chunk maps of the warps of one launch
size_t batch_maps_bytes(const BatchLaunch& L, size_t n) {
    return (size_t)batch_grid(L, n) * (L.block / 32) * 64 * (size_t)std::max(L.stride, 1);
}

size_t batch_plan_bytes(const BatchPlan& P, size_t maps_bytes) {
    return align16(batch_workspace_bytes(P.n, P.ntabs)) + align16(maps_bytes);
}

void batch_plan_place(BatchPlan& P, size_t maps_bytes, void* base) {
    uint8_t* w = static_cast<uint8_t*>(base);
    P.ws = w;
    P.maps = maps_bytes ? w + align16(batch_workspace_bytes(P.n, P.ntabs)) : nullptr;
}

cudaError_t batch_plan_upload(const BatchPlan& P, const BatchTab* h_tabs, const uint32_t* h_pair_tab,
                              const uint8_t* h_cls, cudaStream_t st) {
    return batch_upload(h_tabs, P.ntabs, h_pair_tab, h_cls, P.n, P.ws, st);
}

// Every launch of one batched run, all on `st` (capturable into a graph):
// counter reset, planner, persistent kernel.
cudaError_t batch_run(const BatchPlan& P, const uint8_t* str, const int64_t* off, uint8_t* out, const BatchLaunch& L,
                      cudaStream_t st, bool profile) {
    if (P.n == 0) return cudaSuccess;
    BatchWs b = batch_ws(P.ws, P.n, P.ntabs);
    cudaError_t e = cudaMemsetAsync(b.queue, 0, 256, st);
    if (e != cudaSuccess) return e;
    uint32_t* perm = nullptr;
    unsigned* starts = nullptr;
    e = launch_plan(off, b.cls, kBatchClasses, P.n, b.plan_ws, &perm, &starts, st, nullptr, L.long_bytes, str);
    if (e != cudaSuccess) return e;
    const long long grid = batch_grid(L, P.n);
    if (profile) {
        ProfScope ps(st);
        k_batch<<<(unsigned)grid, L.block, 0, st>>>(b.tabs, b.pair_tab, perm, starts, (long long)P.n, str, off, out,
                                                    b.queue, L.stride, P.maps, bad_offsets_counter());
    } else {
        k_batch<<<(unsigned)grid, L.block, 0, st>>>(b.tabs, b.pair_tab, perm, starts, (long long)P.n, str, off, out,
                                                    b.queue, L.stride, P.maps, bad_offsets_counter());
        prof_count(1);
    }
    return cudaGetLastError();
}

}  // namespace rx
