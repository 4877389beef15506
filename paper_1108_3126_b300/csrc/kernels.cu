// kernels.cu -- lockstep kernels for sm_103a.
//
// The hot loop of every kernel is one macro step of the generic lockstep
// machine (Rathnayake & Thielecke, SOS 2011, Def 5.2) per input byte c:
//     S' = evolve({ cont p : p in S, pi(p) = c })            (Defs 5.1, 5.2)
// With F the evolved set (character positions plus null) this is
//     F' = U { follow[p] : p in F, pi(p) = c },  follow[p] = evolve({cont p})
// where the evolutions were precomputed by the host compiler with the
// pointer-equality visited set.  A string is accepted when null is in F
// after its last byte (Def 5.3); a string whose F empties is stuck and
// rejected without reading further (Fig 6.1).
//
// Variants (the step function is the same; the representation differs):
//   memo   : F is a state id of a cache of macro steps (one table load/byte)
//   thread : F in registers (<= 64 bits), one subset-table load per byte
//   sparse : F in registers (<= 256 bits), union of follow rows per active bit
//   warp   : one warp per string, lane l owns bitset words l, l+32, ...
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "kernels.cuh"
#include "plan.cuh"
#include "steppers.cuh"

namespace rx {

namespace {

using namespace rx::dev;

// ------------------------------------------------ thread-per-string kernel
// Persistent warps take tasks of 32 consecutive entries of the (length-
// sorted) order from a global counter.  Each lane walks its string in
// aligned 16-byte blocks; blocks that are whole for every lane run an
// unrolled step loop, the (few) boundary blocks a predicated one.  A lane
// whose string ends or whose set empties writes its result, then holds the
// empty set, which every step leaves empty.
template <class S>
__global__ void __launch_bounds__(256) k_thread(const DevTables t, const uint8_t* __restrict__ str,
                                                const int64_t* __restrict__ off, const uint32_t* __restrict__ perm,
                                                long long n, uint8_t* __restrict__ out, unsigned* __restrict__ queue,
                                                unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) uint8_t smem[];
    S::load(t, smem);
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    const int lane = threadIdx.x & 31;
    const long long ntasks = (n + 31) >> 5;
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(queue, 1u);
        task = __shfl_sync(FULL, task, 0);
        if ((long long)task >= ntasks) break;
        long long i = (long long)task * 32 + lane;
        bool valid = i < n;
        long long id = valid ? (perm ? (long long)perm[i] : i) : 0;
        // absolute addresses: blocks are aligned in memory, whatever the
        // alignment of `str`; a block is read only if it holds string bytes
        const uint64_t base = reinterpret_cast<uint64_t>(str);
        uint64_t s = base, e = base;
        const bool ok = !valid || string_span(off, id, base, s, e);
        if (!ok) {
            out[id] = kResultInvalid;
            count_bad(bad);
        }
        S st = proto;
        run_lane(st, s, e, valid && ok, out + id);
    }
}

// -------------------------------------------------- warp-per-string kernel
// Lane l owns words l, l+32, ... (K = ceil(W/32) per lane).  A step ANDs
// with B[c], then ORs the follow row of every active bit; the active bits
// are found with ballot / shuffle so the loop is warp-uniform.  The warp
// stages 512 input bytes at a time with one 16-byte load per lane.
template <int K>
__global__ void __launch_bounds__(256) k_warp(const DevTables t, const uint8_t* __restrict__ str,
                                              const int64_t* __restrict__ off, const uint32_t* __restrict__ perm,
                                              long long n, uint8_t* __restrict__ out, unsigned* __restrict__ queue,
                                              unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int W = t.W;
    const size_t bw = (size_t)256 * W, fw = (size_t)t.nbits * W;
    const bool in_smem = (bw + fw) * 4 <= 160 * 1024;
    const uint32_t* B = t.B;
    const uint32_t* follow = t.follow;
    if (in_smem) {
        copy_to_smem_serial(smem, t.B, bw * 4);
        copy_to_smem_serial(smem + align16(bw * 4), t.follow, fw * 4);
        __syncthreads();
        B = reinterpret_cast<const uint32_t*>(smem);
        follow = reinterpret_cast<const uint32_t*>(smem + align16(bw * 4));
    }
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(queue, 1u);
        task = __shfl_sync(FULL, task, 0);
        if ((long long)task >= n) break;
        long long id = perm ? (long long)perm[task] : (long long)task;
        const uint64_t base = reinterpret_cast<uint64_t>(str);
        uint64_t s, e;
        if (!string_span(off, id, base, s, e)) {  // warp-uniform
            if (lane == 0) {
                out[id] = kResultInvalid;
                count_bad(bad);
            }
            continue;
        }
        bool acc = warp_string<K>(t, B, follow, s, e);
        if (lane == 0) out[id] = acc;
    }
}

// One warp per string on the wide cache tier (two-byte state ids, sets of
// more than 256 positions): 32 chunk functions composed from the start
// state (warp_chunked_wide), their rows in shared memory (32 rows of
// `stride` bytes per warp), so the call needs no scratch.
constexpr int kWideBlock = 256;
__global__ void __launch_bounds__(kWideBlock) k_warp_wide(const DevTables t, const uint8_t* __restrict__ str,
                                                          const int64_t* __restrict__ off,
                                                          const uint32_t* __restrict__ perm, long long n,
                                                          uint8_t* __restrict__ out, unsigned* __restrict__ queue,
                                                          unsigned long long* __restrict__ bad, int stride) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t* wsm = smem + (size_t)(threadIdx.x >> 5) * 32 * stride;
    const int lane = threadIdx.x & 31;
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(queue, 1u);
        task = __shfl_sync(FULL, task, 0);
        if ((long long)task >= n) break;
        const long long id = perm ? (long long)perm[task] : (long long)task;
        uint64_t s, e;
        if (!string_span(off, id, base, s, e)) {  // warp-uniform
            if (lane == 0) {
                out[id] = kResultInvalid;
                count_bad(bad);
            }
            continue;
        }
        const uint32_t x = warp_chunked_wide(t, t.wide_start, s, e, wsm, stride);
        if (lane == 0) out[id] = t.wide_acc[x];
    }
}

cudaError_t launch_warp_wide(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                             const uint32_t* perm, uint8_t* out, unsigned* queue, cudaStream_t st) {
    const int stride = (2 * (t.wide_maximg + 2) + 15) & ~15;
    const size_t sm = (size_t)(kWideBlock / 32) * 32 * stride;
    cudaError_t err = allow_smem(k_warp_wide, sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp_wide, kWideBlock, sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>((long long)per_sm * sm_count(), (n * 32 + kWideBlock - 1) / kWideBlock);
    if (grid < 1) grid = 1;
    {
        ProfScope ps(st);
        k_warp_wide<<<(unsigned)grid, kWideBlock, sm, st>>>(t, str, off, perm, n, out, queue, bad_offsets_counter(),
                                                             stride);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------- length-sort planner
// Counting sort of the strings by (class, length bucket), longest first
// within a class, in two launches:
//   hist    : every block counts its range in shared memory and adds its
//             counts to the global bucket totals (block 0 also clears the
//             work counter of the kernel that follows)
//   scatter : every block scans the totals itself (the bucket starts; block
//             0 publishes them), counts its range again, claims one
//             contiguous range per bucket with one atomic add on a zeroed
//             cursor, and places its strings there with shared-memory
//             cursors
// When every block can be resident at once (one tile of kPlanTile strings
// per block) and the stream is not being captured, both passes run as ONE
// cooperative launch (k_plan_one): the keys stay in registers across a grid
// barrier, so the offsets are read once.  The barrier's wait is bounded; a
// block that gives up counts a planner fault (rx_device_faults) and writes
// the identity for its own tile, so every entry stays a valid index.
// Each thread holds the keys of kPlanItems strings at a time, so the loads
// of a tile are in flight together.  Within a bucket the order depends on
// which block claims first; the kernels only need equal lengths within a
// round of 32.
using namespace rx::plan;

__global__ void __launch_bounds__(kPlanThreads) k_plan_hist(const int64_t* __restrict__ off,
                                                            const uint8_t* __restrict__ cls, long long n,
                                                            long long per, int nbk, unsigned* __restrict__ totals,
                                                            unsigned* __restrict__ queue, long long long_bytes,
                                                            int mis) {
    extern __shared__ unsigned sh[];
    if (blockIdx.x == 0 && threadIdx.x == 0 && queue) *queue = 0;
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads) sh[b] = 0;
    __syncthreads();
    const long long lo = (long long)blockIdx.x * per, hi = min(lo + per, n);
    plan_count(off, cls, lo, hi, long_bytes, mis, sh);
    __syncthreads();
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads)
        if (sh[b]) atomicAdd(&totals[b], sh[b]);
}

// every block scans the totals itself (bucket starts), claims a range per
// bucket with one atomic add on a zeroed cursor, and places its strings;
// block 0 also publishes the starts
__global__ void __launch_bounds__(kPlanThreads) k_plan_scatter(const int64_t* __restrict__ off,
                                                               const uint8_t* __restrict__ cls, long long n,
                                                               long long per, int nbk,
                                                               const unsigned* __restrict__ totals,
                                                               unsigned* __restrict__ cursor,
                                                               unsigned* __restrict__ starts,
                                                               uint32_t* __restrict__ perm, long long long_bytes,
                                                               int mis) {
    extern __shared__ unsigned sh[];  // [nbk] counts, then [nbk] bucket starts
    unsigned* sc = sh + nbk;
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads) sh[b] = 0;
    __syncthreads();
    const long long lo = (long long)blockIdx.x * per, hi = min(lo + per, n);
    plan_count(off, cls, lo, hi, long_bytes, mis, sh);
    block_scan(totals, nbk, sc);
    if (blockIdx.x == 0)
        for (int b = threadIdx.x; b < nbk; b += kPlanThreads) starts[b] = sc[b];
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads)
        if (sh[b]) sh[b] = sc[b] + atomicAdd(&cursor[b], sh[b]);
    __syncthreads();
    for (long long base = lo; base < hi; base += kPlanTile) {
        int key[kPlanItems];
        plan_tile_keys(off, cls, base, hi, long_bytes, mis, key);
#pragma unroll
        for (int k = 0; k < kPlanItems; k++)
            if (key[k] >= 0) perm[atomicAdd(&sh[key[k]], 1u)] = (uint32_t)(base + k * kPlanThreads + threadIdx.x);
    }
}

__device__ unsigned g_plan_faults;

__global__ void __launch_bounds__(kPlanThreads) k_plan_one(const int64_t* __restrict__ off,
                                                           const uint8_t* __restrict__ cls, long long n, int nbk,
                                                           unsigned* __restrict__ totals, unsigned* __restrict__ bar,
                                                           unsigned* __restrict__ starts,
                                                           uint32_t* __restrict__ perm, unsigned* __restrict__ queue,
                                                           long long long_bytes, int mis) {
    extern __shared__ unsigned sh[];  // [nbk] counts, then [nbk] bucket starts
    unsigned* sc = sh + nbk;
    if (blockIdx.x == 0 && threadIdx.x == 0 && queue) *queue = 0;
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads) sh[b] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kPlanTile;
    int key[kPlanItems];
    plan_tile_keys(off, cls, base, n, long_bytes, mis, key);
#pragma unroll
    for (int k = 0; k < kPlanItems; k++)
        if (key[k] >= 0) atomicAdd(&sh[key[k]], 1u);
    __syncthreads();
    // adding to the totals also claims this block's range inside each bucket
    // (the value returned), so only the scan is left after the barrier
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads)
        if (sh[b]) sh[b] = atomicAdd(&totals[b], sh[b]);
    if (!grid_barrier(bar, gridDim.x, &g_plan_faults)) {
#pragma unroll
        for (int k = 0; k < kPlanItems; k++)
            if (key[k] >= 0) perm[base + k * kPlanThreads + threadIdx.x] = (uint32_t)(base + k * kPlanThreads + threadIdx.x);
        return;
    }
    block_scan(totals, nbk, sc);
    if (blockIdx.x == 0)
        for (int b = threadIdx.x; b < nbk; b += kPlanThreads) starts[b] = sc[b];
    for (int b = threadIdx.x; b < nbk; b += kPlanThreads) sh[b] += sc[b];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPlanItems; k++)
        if (key[k] >= 0) perm[atomicAdd(&sh[key[k]], 1u)] = (uint32_t)(base + k * kPlanThreads + threadIdx.x);
}

// ------------------------------------------------------------- trace
// One thread; row k (W words) is the evolved set before byte k.
__global__ void k_trace(const DevTables t, const uint8_t* __restrict__ str, int64_t len, uint32_t* __restrict__ rows) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int W = t.W;
    for (int k = 0; k < W; k++) rows[k] = t.start[k];
    for (int64_t i = 0; i < len; i++) {
        const uint32_t* F = rows + (size_t)i * W;
        uint32_t* G = rows + (size_t)(i + 1) * W;
        uint32_t c = str[i];
        for (int k = 0; k < W; k++) G[k] = 0;
        for (int w = 0; w < W; w++) {
            uint32_t s = F[w] & t.B[(size_t)c * W + w];
            while (s) {
                int b = __ffs(s) - 1;
                s &= s - 1;
                const uint32_t* row = t.follow + (size_t)(w * 32 + b) * W;
                for (int k = 0; k < W; k++) G[k] |= row[k];
            }
        }
    }
}

template <class S>
cudaError_t launch_thread_kernel(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                                 const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st) {
    size_t sm = S::smem_bytes(t);
    auto kern = k_thread<S>;
    cudaError_t err = allow_smem(kern, sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long warps_needed = (n + 31) / 32;
    long long grid = (long long)per_sm * sm_count();
    long long cap = (warps_needed * 32 + block - 1) / block;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    {
        ProfScope ps(st);
        kern<<<(unsigned)grid, block, sm, st>>>(t, str, off, perm, n, out, queue, bad_offsets_counter());
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_warp_kernel(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                               const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st) {
    size_t bw = (size_t)256 * t.W, fw = (size_t)t.nbits * t.W;
    size_t sm = ((bw + fw) * 4 <= 160 * 1024) ? align16(bw * 4) + align16(fw * 4) : 0;
    auto kern = k_warp<K>;
    cudaError_t err = allow_smem(kern, sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * sm_count();
    long long cap = (n * 32 + block - 1) / block;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, sm, st>>>(t, str, off, perm, n, out, queue, bad_offsets_counter());
    return cudaGetLastError();
}

__global__ void k_fill_offsets(int64_t* off, int64_t len) {
    if (threadIdx.x == 0) {
        off[0] = 0;
        off[1] = len;
    }
}

}  // namespace

cudaError_t launch_fill_offsets(int64_t* off, int64_t len, cudaStream_t st) {
    k_fill_offsets<<<1, 32, 0, st>>>(off, len);
    prof_count(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------ profiling
namespace {
std::atomic<bool> g_prof_on{false};
std::atomic<int64_t> g_launches{0};
std::mutex g_prof_mu;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_ev;
}  // namespace

void prof_count(int k) { g_launches += k; }
void prof_enable(bool on) { g_prof_on = on; }

ProfScope::ProfScope(cudaStream_t s) : st(s) {
    prof_count(1);
    if (!g_prof_on) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    ev0 = e;
}

ProfScope::~ProfScope() {
    if (!ev0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) != cudaSuccess) return;
    cudaEventRecord(e1, st);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_ev.emplace_back(static_cast<cudaEvent_t>(ev0), e1);
}

cudaError_t prof_read(int64_t* launches, int64_t* timed, double* ms) {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        ev.swap(g_prof_ev);
    }
    double tot = 0;
    cudaError_t err = cudaSuccess;
    for (auto& p : ev) {
        float t = 0;
        cudaError_t e = cudaEventSynchronize(p.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.first, p.second);
        if (e != cudaSuccess) err = e;
        tot += t;
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    if (launches) *launches = g_launches.exchange(0);
    if (timed) *timed = (int64_t)ev.size();
    if (ms) *ms = tot;
    return err;
}

cudaError_t allow_smem_raw(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> high;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& h = high[std::make_pair(dev, func)];
    if (bytes <= h && h > 0) return cudaSuccess;
    const size_t want = std::max<size_t>(bytes, 1);
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want);
    if (e == cudaSuccess) h = want;
    return e;
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// one tile per block up to 64 blocks per SM, then several tiles per block
int plan_blocks(size_t n) {
    long long g = ((long long)n + kPlanTile - 1) / kPlanTile;
    return (int)std::max<long long>(1, std::min<long long>(g, (long long)sm_count() * 64));
}

// totals, claim cursors and the grid-barrier counter (zeroed together),
// bucket starts, permutation
size_t plan_workspace_bytes(size_t n, int nclasses) {
    size_t nbk = (size_t)kLenBuckets * nclasses;
    return align16((2 * nbk + 1) * 4) + align16(nbk * 4) + align16(n * 4);
}

// strings whose offsets the kernels found invalid (rx_sync_check), per device
__device__ unsigned long long g_bad_offsets;

unsigned long long* bad_offsets_counter() {
    static std::mutex mu;
    static unsigned long long* addr[128] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bad_offsets) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        addr[dev] = static_cast<unsigned long long*>(p);
    }
    return addr[dev];
}

unsigned long long read_bad_offsets(bool reset) {
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_bad_offsets, sizeof(v));
    if (reset && v) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_bad_offsets, &z, sizeof(z));
    }
    return v;
}

unsigned read_plan_faults(bool reset) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_plan_faults, sizeof(v));
    if (reset) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_plan_faults, &z, sizeof(z));
    }
    return v;
}

namespace {
// blocks of k_plan_one that fit on the device at once (per device, cached)
long long plan_one_capacity(size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, size_t>, long long> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, smem});
    if (it != cache.end()) return it->second;
    int coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_one, kPlanThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    const long long cap = coop ? (long long)per_sm * sm_count() : 0;
    cache[{dev, smem}] = cap;
    return cap;
}
}  // namespace

cudaError_t launch_plan(const int64_t* off, const uint8_t* cls, int nclasses, size_t n, void* ws, uint32_t** perm,
                        unsigned** starts, cudaStream_t st, unsigned* queue, long long long_bytes,
                        const void* strings) {
    const int mis = (int)(reinterpret_cast<uintptr_t>(strings) & 31);
    const int nbk = kLenBuckets * nclasses;  // at most 7 x 384 buckets: 21 KiB of shared memory in the scatter
    const int G = plan_blocks(n);
    long long per = ((long long)n + G - 1) / G;
    per = (per + kPlanTile - 1) / kPlanTile * kPlanTile;
    uint8_t* w = static_cast<uint8_t*>(ws);
    unsigned* totals = reinterpret_cast<unsigned*>(w);
    unsigned* cursor = totals + nbk;
    unsigned* bar = cursor + nbk;
    const size_t head = align16((2 * (size_t)nbk + 1) * 4);
    unsigned* st_out = reinterpret_cast<unsigned*>(w + head);
    *perm = reinterpret_cast<uint32_t*>(w + head + align16((size_t)nbk * 4));
    *starts = st_out;
    cudaError_t e = cudaMemsetAsync(totals, 0, (2 * (size_t)nbk + 1) * 4, st);
    if (e != cudaSuccess) return e;
    // one cooperative launch when every tile gets its own resident block
    const long long tiles = ((long long)n + kPlanTile - 1) / kPlanTile;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {  // unknown: take the two-launch form
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    const size_t sm1 = 2 * (size_t)nbk * 4;
    if (cs == cudaStreamCaptureStatusNone && tiles >= 1 && tiles <= plan_one_capacity(sm1)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)tiles);
        cfg.blockDim = dim3(kPlanThreads);
        cfg.dynamicSmemBytes = sm1;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_plan_one, off, cls, (long long)n, nbk, totals, bar, st_out, *perm, queue,
                               long_bytes, mis);
        prof_count(1);
        return e;
    }
    k_plan_hist<<<G, kPlanThreads, (size_t)nbk * 4, st>>>(off, cls, (long long)n, per, nbk, totals, queue, long_bytes,
                                                                 mis);
    k_plan_scatter<<<G, kPlanThreads, 2 * (size_t)nbk * 4, st>>>(off, cls, (long long)n, per, nbk, totals, cursor,
                                                                 st_out, *perm, long_bytes, mis);
    prof_count(2);
    return cudaGetLastError();
}

size_t match_workspace_bytes(size_t n, int sort) {
    size_t b = 256;  // queue counter
    if (sort >= 1) b += plan_workspace_bytes(n, 1);
    return b;
}

int resolve_sort(int variant, int sort, size_t n) {
    const bool streams = variant == RX_VARIANT_MEMO || variant == RX_VARIANT_THREAD;
    if (sort < 0) {
        if (variant == RX_VARIANT_MEMO) sort = n >= 4096 ? 4 : 3;
        else if (variant == RX_VARIANT_THREAD) sort = n >= 4096 ? 2 : 3;
        else sort = n >= 4096 ? 1 : 0;
    }
    if (sort == 4 && variant != RX_VARIANT_MEMO) sort = 2;
    if (sort >= 2 && !streams) return sort == 3 ? 0 : 1;
    return sort;
}

cudaError_t launch_match(const DevTables& t, int variant, size_t n, const uint8_t* str, const int64_t* off,
                         uint8_t* out, int sort, int block, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (ws_bytes < match_workspace_bytes(n, sort)) return cudaErrorInvalidValue;
    uint8_t* w = static_cast<uint8_t*>(ws);
    unsigned* queue = reinterpret_cast<unsigned*>(w);
    uint32_t* perm = nullptr;
    cudaError_t err = cudaSuccess;
    if (sort == 4) {  // block-local length order in the streaming kernel, else sort 2
        bool launched = false;
        if (block == 0 || block == 768) {
            err = launch_stream_local(t, (long long)n, str, off, out, st, &launched);
            if (err != cudaSuccess || launched) return err;
        }
        sort = 2;
    }
    if (sort != 1 && sort != 2) {  // with the planner, its first kernel clears the counter
        err = cudaMemsetAsync(w, 0, 256, st);
        if (err != cudaSuccess) return err;
    }
    if (sort == 3) return launch_stream(t, variant, (long long)n, str, off, nullptr, out, queue, block, st);
    // the remaining kernels take 32..256 threads per block
    const int req_block = block;
    if (sort >= 1) {
        unsigned* starts = nullptr;
        err = launch_plan(off, nullptr, 1, n, w + 256, &perm, &starts, st, queue, 4096, str);
        if (err != cudaSuccess) return err;
        if (sort == 2) return launch_stream(t, variant, (long long)n, str, off, perm, out, queue, req_block, st);
    }
    if (block <= 0) block = 256;
    block = (block + 31) / 32 * 32;
    if (block > 256) block = 256;
    long long nn = (long long)n;
    switch (variant) {
    case RX_VARIANT_MEMO:
        return launch_thread_kernel<MemoStep>(t, nn, str, off, perm, out, queue, block, st);
    case RX_VARIANT_THREAD:
        if (t.W == 1) return launch_thread_kernel<Thread1Step>(t, nn, str, off, perm, out, queue, block, st);
        return launch_thread_kernel<Thread2Step>(t, nn, str, off, perm, out, queue, block, st);
    case RX_VARIANT_SPARSE:
        if (t.W <= 4) return launch_thread_kernel<SparseStep<4>>(t, nn, str, off, perm, out, queue, block, st);
        return launch_thread_kernel<SparseStep<8>>(t, nn, str, off, perm, out, queue, block, st);
    case RX_VARIANT_WARP:
        if (t.wide_K > 0) return launch_warp_wide(t, nn, str, off, perm, out, queue, st);
        if (t.W <= 32) return launch_warp_kernel<1>(t, nn, str, off, perm, out, queue, block, st);
        if (t.W <= 64) return launch_warp_kernel<2>(t, nn, str, off, perm, out, queue, block, st);
        return launch_warp_kernel<4>(t, nn, str, off, perm, out, queue, block, st);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_trace(const DevTables& t, const uint8_t* str, int64_t len, uint32_t* rows, cudaStream_t st) {
    k_trace<<<1, 32, 0, st>>>(t, str, len, rows);
    prof_count(1);
    return cudaGetLastError();
}

}  // namespace rx
