// stream.cu -- the single-expression streaming kernel (rx_match default).
//
// One lane walks one string, one macro step of the lockstep machine
// (Rathnayake & Thielecke, SOS 2011, Def 5.2) per byte, the active set in
// registers (or a state id of the cache of macro steps) and the tables in
// shared memory.  Work distribution: the planner orders the strings by
// length, longest first; persistent warps take rounds of 32 consecutive
// entries from a global counter, so the lanes of a round have (nearly) the
// same length and finish together, and the longest rounds start first.
// Input: every lane reads its string in aligned 32-byte blocks (one full
// sector, two 16-byte loads) with loads issued two blocks ahead.
#include <algorithm>

#include "kernels.cuh"
#include "steppers.cuh"

namespace rx {

namespace {

using namespace rx::dev;

constexpr int STREAM_BLOCK = 256;
constexpr int STREAM_MAX_BLOCK = 512;

struct Blk32 {
    uint4 a, b;
};

// one 256-bit load of an aligned 32-byte block (a whole sector): one L1
// wavefront per lane instead of two for a pair of 128-bit loads
__device__ __forceinline__ Blk32 ld_blk(uint64_t addr, bool on) {
    Blk32 r;
    r.a = make_uint4(0, 0, 0, 0);
    r.b = r.a;
    if (on)
        asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r.a.x), "=r"(r.a.y), "=r"(r.a.z), "=r"(r.a.w), "=r"(r.b.x), "=r"(r.b.y), "=r"(r.b.z),
                       "=r"(r.b.w)
                     : "l"(addr));
    return r;
}

__device__ __forceinline__ uint32_t word_of(const Blk32& v, int q) {
    return q == 0 ? v.a.x : q == 1 ? v.a.y : q == 2 ? v.a.z : q == 3 ? v.a.w
         : q == 4 ? v.b.x : q == 5 ? v.b.y : q == 6 ? v.b.z : v.b.w;
}

// bytes of the 32-byte block at blk that lie in [s, e), as a bit mask
__device__ __forceinline__ uint32_t valid_mask(uint64_t blk, uint64_t s, uint64_t e, bool active) {
    if (!active || blk >= e || blk + 32 <= s) return 0u;
    uint32_t lo = blk >= s ? 0u : (uint32_t)(s - blk);
    uint32_t hi = blk + 32 <= e ? 32u : (uint32_t)(e - blk);
    uint32_t m_hi = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    return m_hi & ~((1u << lo) - 1u);
}

// Process one 32-byte block of every lane of the warp: the unrolled path
// when the block is whole for every lane that still has bytes, the masked
// path otherwise.  Lanes without bytes hold the empty set (harmless).
template <class S, class = void>
struct has_pairs {
    static constexpr bool value = false;
};
template <class S>
struct has_pairs<S, decltype(void(S::kPairs))> {
    static constexpr bool value = S::kPairs;
};

template <class S>
__device__ __forceinline__ void block32(S& st, const Blk32& v, uint32_t mask) {
    if constexpr (has_pairs<S>::value) {
        // two bytes per lookup when the block is whole and inside the window
        // for every lane that still has bytes
        uint32_t out = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) out |= st.out_of_window(word_of(v, q));
        bool pair_ok = mask == 0u || (mask == 0xffffffffu && out == 0u);
        if (__all_sync(FULL, pair_ok)) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                uint32_t w = word_of(v, q);
                st.step2(w);
                st.step2(w >> 16);
            }
            return;
        }
    }
    if (__all_sync(FULL, mask == 0xffffffffu || mask == 0u)) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            uint32_t w = word_of(v, q);
#pragma unroll
            for (int k = 0; k < 4; k++) st.step(byte_k(w, k));
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            uint32_t w = word_of(v, q);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                S nx = st;
                nx.step(byte_k(w, k));
                if ((mask >> (4 * q + k)) & 1u) st = nx;
            }
        }
    }
}

template <class S>
__global__ void __launch_bounds__(STREAM_MAX_BLOCK) k_stream(const DevTables t, const uint8_t* __restrict__ str,
                                                         const int64_t* __restrict__ off,
                                                         const uint32_t* __restrict__ perm, long long n,
                                                         uint8_t* __restrict__ out, unsigned* __restrict__ queue) {
    extern __shared__ __align__(16) uint8_t smem[];
    S::load(t, smem);
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    const int lane = threadIdx.x & 31;
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    const long long nround = (n + 31) / 32;
    for (;;) {
        unsigned r = 0;
        if (lane == 0) r = atomicAdd(queue, 1u);
        r = __shfl_sync(FULL, r, 0);
        if ((long long)r >= nround) break;
        const long long k = (long long)r * 32 + lane;
        const bool valid = k < n;
        const long long id = valid ? (perm ? (long long)perm[k] : k) : 0;
        uint64_t s = base, e = base;
        if (valid) {
            s += (uint64_t)off[id];
            e += (uint64_t)off[id + 1];
        }
        S st = proto;
        bool active = valid && s < e;
        if (valid && !active) out[id] = st.accept();
        if (!active) st.kill();
        uint64_t blk = s & ~uint64_t(31);
        Blk32 va = ld_blk(blk, active);
        Blk32 vb = ld_blk(blk + 32, active && blk + 32 < e);
        while (__any_sync(FULL, active)) {
            // block A at blk, then block B at blk + 32; each buffer is
            // refilled two blocks ahead right after it is consumed
            block32(st, va, valid_mask(blk, s, e, active));
            if (active && (blk + 32 >= e || st.dead())) {
                out[id] = st.accept();
                st.kill();
                active = false;
            }
            va = ld_blk(blk + 64, active && blk + 64 < e);
            if (!__any_sync(FULL, active)) break;
            block32(st, vb, valid_mask(blk + 32, s, e, active));
            if (active && (blk + 64 >= e || st.dead())) {
                out[id] = st.accept();
                st.kill();
                active = false;
            }
            vb = ld_blk(blk + 96, active && blk + 96 < e);
            blk += 64;
        }
    }
}

// Tasks of the chunked long-string mode: task i starts the cache of macro
// steps in state task_state[i] at byte task_chunk[i] * C + P of the text and
// runs to the end of that chunk; res[i] receives the final state id.  Tasks
// come chunk by chunk, so the 32 lanes of a round cover equal-length spans.
template <class S>
__global__ void __launch_bounds__(STREAM_MAX_BLOCK) k_span_tasks(const DevTables t, const uint8_t* __restrict__ str,
                                                               int64_t len, int64_t C, int64_t P,
                                                               const uint32_t* __restrict__ task_chunk,
                                                               const uint16_t* __restrict__ task_state,
                                                               const unsigned* __restrict__ ntask_p,
                                                               uint16_t* __restrict__ res,
                                                               unsigned* __restrict__ queue) {
    extern __shared__ __align__(16) uint8_t smem[];
    S::load(t, smem);
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    const int lane = threadIdx.x & 31;
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    const long long n = *ntask_p;
    const long long nround = (n + 31) / 32;
    for (;;) {
        unsigned r = 0;
        if (lane == 0) r = atomicAdd(queue, 1u);
        r = __shfl_sync(FULL, r, 0);
        if ((long long)r >= nround) break;
        const long long k = (long long)r * 32 + lane;
        const bool valid = k < n;
        uint64_t s = base, e = base;
        S st = proto;
        st.kill();
        if (valid) {
            const int64_t j = task_chunk[k];
            const int64_t lo = j * C, hi = min(lo + C, len);
            s += (uint64_t)min(lo + P, hi);
            e += (uint64_t)hi;
            st.set_state(task_state[k]);
        }
        bool active = valid && s < e && !st.dead();
        // the state when the lane's span ends: the warp keeps stepping every
        // lane while any is active, so a finished lane's state is taken here
        uint32_t fin = valid ? st.state_id() : 0u;
        if (!active) st.kill();
        uint64_t blk = s & ~uint64_t(31);
        Blk32 va = ld_blk(blk, active);
        Blk32 vb = ld_blk(blk + 32, active && blk + 32 < e);
        while (__any_sync(FULL, active)) {
            block32(st, va, valid_mask(blk, s, e, active));
            if (active && (blk + 32 >= e || st.dead())) {
                fin = st.state_id();
                st.kill();
                active = false;
            }
            va = ld_blk(blk + 64, active && blk + 64 < e);
            if (!__any_sync(FULL, active)) break;
            block32(st, vb, valid_mask(blk + 32, s, e, active));
            if (active && (blk + 64 >= e || st.dead())) {
                fin = st.state_id();
                st.kill();
                active = false;
            }
            vb = ld_blk(blk + 96, active && blk + 96 < e);
            blk += 64;
        }
        if (valid) res[k] = (uint16_t)fin;
    }
}

template <class S>
cudaError_t launch_span_t(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, int64_t P,
                          const uint32_t* task_chunk, const uint16_t* task_state, const unsigned* ntask_p,
                          uint16_t* res, unsigned* queue, long long max_tasks, cudaStream_t st) {
    size_t sm = S::smem_bytes(t);
    auto kern = k_span_tasks<S>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    const int block = 256;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>((max_tasks + block - 1) / block, (long long)per_sm * sm_count());
    {
        ProfScope ps(st);
        kern<<<(unsigned)std::max<long long>(grid, 1), block, sm, st>>>(t, str, len, C, P, task_chunk, task_state,
                                                                        ntask_p, res, queue);
    }
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_stream_t(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                            const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st) {
    size_t sm = S::smem_bytes(t);
    auto kern = k_stream<S>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long rounds = (n + 31) / 32;
    long long grid = std::min<long long>((rounds * 32 + block - 1) / block, (long long)per_sm * sm_count());
    {
        ProfScope ps(st);
        kern<<<(unsigned)std::max<long long>(grid, 1), block, sm, st>>>(t, str, off, perm, n, out, queue);
    }
    return cudaGetLastError();
}

}  // namespace

bool stream_pairs(const DevTables& t) { return t.bg_T != nullptr; }

cudaError_t launch_span_tasks(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, int64_t P,
                              const uint32_t* task_chunk, const uint16_t* task_state, const unsigned* ntask_p,
                              uint16_t* res, unsigned* queue, long long max_tasks, cudaStream_t st) {
    if (t.bg_T)
        return launch_span_t<MemoPair>(t, str, len, C, P, task_chunk, task_state, ntask_p, res, queue, max_tasks, st);
    return launch_span_t<MemoS>(t, str, len, C, P, task_chunk, task_state, ntask_p, res, queue, max_tasks, st);
}

bool stream_supported(const DevTables& t, int variant) {
    return variant == RX_VARIANT_MEMO || (variant == RX_VARIANT_THREAD && t.W <= 2);
}

cudaError_t launch_stream(const DevTables& t, int variant, long long n, const uint8_t* str, const int64_t* off,
                          const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st) {
    // an odd block request (e.g. 257) asks for the single-byte memo kernel
    const int block_req = block;
    const int single = block & 1;
    block &= ~1;
    block = (block == 128 || block == 64 || block == 512) ? block : STREAM_BLOCK;
    block |= single;
    if (variant == RX_VARIANT_MEMO) {
        // 512 threads: the autotuner's measured choice for the two-byte
        // kernel on the streaming workload (about 5% over 256)
        if (t.bg_T && !(block & 1))
            return launch_stream_t<MemoPair>(t, n, str, off, perm, out, queue, block_req == 0 ? 512 : block, st);
        return launch_stream_t<MemoS>(t, n, str, off, perm, out, queue, block & ~1, st);
    }
    if (t.W == 1) return launch_stream_t<Thread1S>(t, n, str, off, perm, out, queue, block & ~1, st);
    return launch_stream_t<Thread2S>(t, n, str, off, perm, out, queue, block & ~1, st);
}

}  // namespace rx
