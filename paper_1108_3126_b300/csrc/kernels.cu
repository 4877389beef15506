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
#include <atomic>
#include <cstdio>
#include <mutex>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace rx {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint4 ld_stream(const uint8_t* p) {
    return __ldcs(reinterpret_cast<const uint4*>(p));
}

__device__ __forceinline__ uint32_t byte_of(const uint4& v, int k) {
    uint32_t w = (k < 4) ? v.x : (k < 8) ? v.y : (k < 12) ? v.z : v.w;
    return (w >> (8 * (k & 3))) & 0xffu;
}

// cooperative copy global -> shared (16-byte granules; sizes rounded up)
__device__ void copy_to_smem(void* dst, const void* src, size_t bytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    size_t n = (bytes + 15) / 16;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ------------------------------------------------------------- steppers
// Each stepper: smem_bytes(t), load(t, smem) [block-cooperative],
// bind(t, smem), init(), step(c), dead(), accept(), kill().

struct MemoStep {
    const uint32_t* T;
    const uint8_t* acc;
    uint32_t st;
    static size_t smem_bytes(const DevTables& t) { return align16((size_t)t.memo_K * 1024) + align16(t.memo_K); }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        copy_to_smem(sm, t.memo_T, (size_t)t.memo_K * 1024);
        copy_to_smem(sm + align16((size_t)t.memo_K * 1024), t.memo_acc, t.memo_K);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        T = reinterpret_cast<const uint32_t*>(sm);
        acc = sm + align16((size_t)t.memo_K * 1024);
        st = t.memo_start;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = T[st + c]; }
    __device__ __forceinline__ bool dead() const { return st == 0; }
    __device__ __forceinline__ bool accept() const { return acc[st >> 8] != 0; }
    __device__ __forceinline__ void kill() { st = 0; }
};

struct Thread1Step {
    const uint2* desc;
    const uint32_t* tt;
    uint32_t F, nb;
    static size_t smem_bytes(const DevTables& t) { return 256 * sizeof(uint2) + align16((size_t)t.gl_words * 4); }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        copy_to_smem(sm, t.gl_desc, 256 * sizeof(uint2));
        copy_to_smem(sm + 256 * sizeof(uint2), t.gl_tt, (size_t)t.gl_words * 4);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        desc = reinterpret_cast<const uint2*>(sm);
        tt = reinterpret_cast<const uint32_t*>(sm + 256 * sizeof(uint2));
        F = t.start[0];
        nb = t.null_bit;
    }
    __device__ __forceinline__ void step(uint32_t c) {
        uint2 d = desc[c];
        uint32_t x = (F >> (d.x & 31u)) & (d.x >> 8);
        F = tt[d.y + x];
    }
    __device__ __forceinline__ bool dead() const { return F == 0; }
    __device__ __forceinline__ bool accept() const { return (F >> nb) & 1u; }
    __device__ __forceinline__ void kill() { F = 0; }
};

struct Thread2Step {
    const uint2* desc;
    const uint2* tt;
    uint32_t F0, F1, nb;
    static size_t smem_bytes(const DevTables& t) { return 256 * sizeof(uint2) + align16((size_t)t.gl_words * 4); }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        copy_to_smem(sm, t.gl_desc, 256 * sizeof(uint2));
        copy_to_smem(sm + 256 * sizeof(uint2), t.gl_tt, (size_t)t.gl_words * 4);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        desc = reinterpret_cast<const uint2*>(sm);
        tt = reinterpret_cast<const uint2*>(sm + 256 * sizeof(uint2));
        F0 = t.start[0];
        F1 = t.start[1];
        nb = t.null_bit;
    }
    __device__ __forceinline__ void step(uint32_t c) {
        uint2 d = desc[c];
        uint32_t w = (d.x & 32u) ? F1 : F0;
        uint32_t x = (w >> (d.x & 31u)) & (d.x >> 8);
        uint2 e = tt[(d.y >> 1) + x];
        F0 = e.x;
        F1 = e.y;
    }
    __device__ __forceinline__ bool dead() const { return (F0 | F1) == 0; }
    __device__ __forceinline__ bool accept() const { return (((nb < 32) ? F0 : F1) >> (nb & 31)) & 1u; }
    __device__ __forceinline__ void kill() { F0 = F1 = 0; }
};

template <int W>
struct SparseStep {
    static_assert(W % 4 == 0, "W must be a multiple of 4");
    const uint32_t* B;
    const uint32_t* follow;
    uint32_t F[W];
    uint32_t nb;
    static size_t smem_bytes(const DevTables& t) { return (size_t)256 * W * 4 + (size_t)t.nbits * W * 4; }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        // tables are stored with t.W words per row; widen to W words
        uint32_t* b = reinterpret_cast<uint32_t*>(sm);
        uint32_t* f = b + 256 * W;
        for (int i = threadIdx.x; i < 256 * W; i += blockDim.x) {
            int r = i / W, k = i % W;
            b[i] = (k < t.W) ? t.B[(size_t)r * t.W + k] : 0u;
        }
        for (int i = threadIdx.x; i < t.nbits * W; i += blockDim.x) {
            int r = i / W, k = i % W;
            f[i] = (k < t.W) ? t.follow[(size_t)r * t.W + k] : 0u;
        }
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        B = reinterpret_cast<const uint32_t*>(sm);
        follow = B + 256 * W;
#pragma unroll
        for (int k = 0; k < W; k++) F[k] = (k < t.W) ? t.start[k] : 0u;
        nb = t.null_bit;
    }
    __device__ __forceinline__ void step(uint32_t c) {
        uint32_t S[W];
        const uint4* b4 = reinterpret_cast<const uint4*>(B + c * W);
#pragma unroll
        for (int q = 0; q < W / 4; q++) {
            uint4 v = b4[q];
            S[4 * q] = F[4 * q] & v.x;
            S[4 * q + 1] = F[4 * q + 1] & v.y;
            S[4 * q + 2] = F[4 * q + 2] & v.z;
            S[4 * q + 3] = F[4 * q + 3] & v.w;
        }
#pragma unroll
        for (int k = 0; k < W; k++) F[k] = 0;
#pragma unroll
        for (int w = 0; w < W; w++) {
            uint32_t s = S[w];
            while (s) {
                int b = __ffs(s) - 1;
                s &= s - 1;
                const uint4* r4 = reinterpret_cast<const uint4*>(follow + (size_t)(w * 32 + b) * W);
#pragma unroll
                for (int q = 0; q < W / 4; q++) {
                    uint4 v = r4[q];
                    F[4 * q] |= v.x;
                    F[4 * q + 1] |= v.y;
                    F[4 * q + 2] |= v.z;
                    F[4 * q + 3] |= v.w;
                }
            }
        }
    }
    __device__ __forceinline__ bool dead() const {
        uint32_t o = 0;
#pragma unroll
        for (int k = 0; k < W; k++) o |= F[k];
        return o == 0;
    }
    __device__ __forceinline__ bool accept() const {
        uint32_t r = 0;
#pragma unroll
        for (int k = 0; k < W; k++)
            if (k == (int)(nb >> 5)) r = (F[k] >> (nb & 31)) & 1u;
        return r != 0;
    }
    __device__ __forceinline__ void kill() {
#pragma unroll
        for (int k = 0; k < W; k++) F[k] = 0;
    }
};

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
                                                long long n, uint8_t* __restrict__ out, unsigned* __restrict__ queue) {
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
        if (valid) {
            s += (uint64_t)off[id];
            e += (uint64_t)off[id + 1];
        }
        S st = proto;
        bool active = valid && s < e;
        if (valid && !active) out[id] = st.accept();
        if (!active) st.kill();
        uint64_t blk = s & ~uint64_t(15);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (active) v = ld_stream(reinterpret_cast<const uint8_t*>(blk));
        while (__any_sync(FULL, active)) {
            uint64_t nb = blk + 16;
            uint4 vn = make_uint4(0, 0, 0, 0);
            if (active && nb < e) vn = ld_stream(reinterpret_cast<const uint8_t*>(nb));
            bool full = !active || (blk >= s && nb <= e);
            if (__all_sync(FULL, full)) {
#pragma unroll
                for (int k = 0; k < 16; k++) st.step(byte_of(v, k));
            } else {
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    S nx = st;
                    nx.step(byte_of(v, k));
                    bool ok = active && blk + k >= s && blk + k < e;
                    if (ok) st = nx;
                }
            }
            blk = nb;
            v = vn;
            if (active && (blk >= e || st.dead())) {
                out[id] = st.accept();
                st.kill();
                active = false;
            }
        }
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
                                              long long n, uint8_t* __restrict__ out, unsigned* __restrict__ queue) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int W = t.W;
    const size_t bw = (size_t)256 * W, fw = (size_t)t.nbits * W;
    const bool in_smem = (bw + fw) * 4 <= 160 * 1024;
    const uint32_t* B = t.B;
    const uint32_t* follow = t.follow;
    if (in_smem) {
        copy_to_smem(smem, t.B, bw * 4);
        copy_to_smem(smem + align16(bw * 4), t.follow, fw * 4);
        __syncthreads();
        B = reinterpret_cast<const uint32_t*>(smem);
        follow = reinterpret_cast<const uint32_t*>(smem + align16(bw * 4));
    }
    const int lane = threadIdx.x & 31;
    const int nbw = t.null_bit >> 5, nbb = t.null_bit & 31;
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(queue, 1u);
        task = __shfl_sync(FULL, task, 0);
        if ((long long)task >= n) break;
        long long id = perm ? (long long)perm[task] : (long long)task;
        const uint64_t base = reinterpret_cast<uint64_t>(str);
        const uint64_t s = base + (uint64_t)off[id], e = base + (uint64_t)off[id + 1];
        uint32_t F[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            int w = k * 32 + lane;
            F[k] = (w < W) ? t.start[w] : 0u;
        }
        bool dead = false;
        for (uint64_t win = s & ~uint64_t(511); win < e && !dead; win += 512) {
            uint4 v = make_uint4(0, 0, 0, 0);
            uint64_t my = win + 16 * lane;
            if (my < e && my + 16 > s) v = ld_stream(reinterpret_cast<const uint8_t*>(my));
            for (int src = 0; src < 32 && !dead; src++) {
                uint64_t blk = win + 16 * src;
                if (blk >= e) break;
                if (blk + 16 <= s) continue;
                uint32_t words[4];
                words[0] = __shfl_sync(FULL, v.x, src);
                words[1] = __shfl_sync(FULL, v.y, src);
                words[2] = __shfl_sync(FULL, v.z, src);
                words[3] = __shfl_sync(FULL, v.w, src);
#pragma unroll 1
                for (int kb = 0; kb < 16; kb++) {
                    uint64_t p = blk + kb;
                    if (p < s || p >= e) continue;
                    uint32_t c = (words[kb >> 2] >> (8 * (kb & 3))) & 0xffu;
                    uint32_t Sx[K];
#pragma unroll
                    for (int k = 0; k < K; k++) {
                        int w = k * 32 + lane;
                        Sx[k] = (w < W) ? (F[k] & B[(size_t)c * W + w]) : 0u;
                        F[k] = 0;
                    }
#pragma unroll
                    for (int k = 0; k < K; k++) {
                        unsigned act = __ballot_sync(FULL, Sx[k] != 0);
                        while (act) {
                            int srcl = __ffs(act) - 1;
                            act &= act - 1;
                            uint32_t bits = __shfl_sync(FULL, Sx[k], srcl);
                            while (bits) {
                                int b = __ffs(bits) - 1;
                                bits &= bits - 1;
                                const uint32_t* row = follow + (size_t)((k * 32 + srcl) * 32 + b) * W;
#pragma unroll
                                for (int kk = 0; kk < K; kk++) {
                                    int w = kk * 32 + lane;
                                    if (w < W) F[kk] |= row[w];
                                }
                            }
                        }
                    }
                    uint32_t any = 0;
#pragma unroll
                    for (int k = 0; k < K; k++) any |= F[k];
                    if (!__any_sync(FULL, any != 0)) {
                        dead = true;
                        break;
                    }
                }
            }
        }
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < K; k++)
            if (k == (nbw >> 5)) mine = F[k];
        uint32_t nw = __shfl_sync(FULL, mine, nbw & 31);
        if (lane == 0) out[id] = dead ? 0 : ((nw >> nbb) & 1u);
    }
}

// ---------------------------------------------------- length-sort planner
__device__ __forceinline__ int len_bucket(int64_t len) {
    if (len < 2048) return (int)len;
    int lg = 63 - __clzll(len);  // >= 11
    int b = 2048 + 4 * (lg - 11) + (int)((len >> (lg - 2)) & 3);
    return b < kLenBuckets ? b : kLenBuckets - 1;
}

__global__ void k_len_hist(const int64_t* __restrict__ off, long long n, unsigned* __restrict__ hist) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int b = len_bucket(off[i + 1] - off[i]);
        unsigned peers = __match_any_sync(__activemask(), b);
        int leader = __ffs(peers) - 1;
        if ((threadIdx.x & 31) == leader) atomicAdd(&hist[b], __popc(peers));
    }
}

// exclusive scan with the LONGEST bucket first: cursor[b] = sum_{b' > b} hist[b']
__global__ void k_len_scan(const unsigned* __restrict__ hist, unsigned* __restrict__ cursor) {
    __shared__ unsigned part[1024];
    constexpr int PER = (kLenBuckets + 1023) / 1024;
    int t = threadIdx.x;
    unsigned loc[PER];
    unsigned sum = 0;
    for (int j = 0; j < PER; j++) {
        int r = t * PER + j;  // position in descending order
        int b = kLenBuckets - 1 - r;
        loc[j] = (b >= 0) ? hist[b] : 0u;
        sum += loc[j];
    }
    part[t] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        unsigned v = (t >= d) ? part[t - d] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - sum;
    for (int j = 0; j < PER; j++) {
        int r = t * PER + j;
        int b = kLenBuckets - 1 - r;
        if (b >= 0) cursor[b] = run;
        run += loc[j];
    }
}

__global__ void k_len_scatter(const int64_t* __restrict__ off, long long n, unsigned* __restrict__ cursor,
                              uint32_t* __restrict__ perm) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int b = len_bucket(off[i + 1] - off[i]);
        unsigned peers = __match_any_sync(__activemask(), b);
        int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if ((threadIdx.x & 31) == leader) base = atomicAdd(&cursor[b], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        unsigned rank = __popc(peers & ((1u << (threadIdx.x & 31)) - 1u));
        perm[base + rank] = (uint32_t)i;
    }
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
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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
        kern<<<(unsigned)grid, block, sm, st>>>(t, str, off, perm, n, out, queue);
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_warp_kernel(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                               const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st) {
    size_t bw = (size_t)256 * t.W, fw = (size_t)t.nbits * t.W;
    size_t sm = ((bw + fw) * 4 <= 160 * 1024) ? align16(bw * 4) + align16(fw * 4) : 0;
    auto kern = k_warp<K>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * sm_count();
    long long cap = (n * 32 + block - 1) / block;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, sm, st>>>(t, str, off, perm, n, out, queue);
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

size_t match_workspace_bytes(size_t n, bool sort) {
    size_t b = 256;  // queue counter
    if (sort) b += align16((size_t)kLenBuckets * 4) * 2 + align16(n * 4);
    return b;
}

cudaError_t launch_match(const DevTables& t, int variant, size_t n, const uint8_t* str, const int64_t* off,
                         uint8_t* out, bool sort, int block, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (ws_bytes < match_workspace_bytes(n, sort)) return cudaErrorInvalidValue;
    uint8_t* w = static_cast<uint8_t*>(ws);
    unsigned* queue = reinterpret_cast<unsigned*>(w);
    uint32_t* perm = nullptr;
    cudaError_t err;
    if (sort) {
        unsigned* hist = reinterpret_cast<unsigned*>(w + 256);
        unsigned* cursor = reinterpret_cast<unsigned*>(w + 256 + align16((size_t)kLenBuckets * 4));
        perm = reinterpret_cast<uint32_t*>(w + 256 + 2 * align16((size_t)kLenBuckets * 4));
        err = cudaMemsetAsync(w, 0, 256 + align16((size_t)kLenBuckets * 4), st);
        if (err != cudaSuccess) return err;
        int g = (int)std::min<long long>((long long)(n + 255) / 256, (long long)sm_count() * 8);
        k_len_hist<<<g, 256, 0, st>>>(off, (long long)n, hist);
        k_len_scan<<<1, 1024, 0, st>>>(hist, cursor);
        k_len_scatter<<<g, 256, 0, st>>>(off, (long long)n, cursor, perm);
        prof_count(3);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    } else {
        err = cudaMemsetAsync(w, 0, 256, st);
        if (err != cudaSuccess) return err;
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
