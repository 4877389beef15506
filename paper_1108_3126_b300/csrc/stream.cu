// stream.cu -- the single-expression streaming kernel (rx_match default).
//
// One lane walks one string, one macro step of the lockstep machine
// (Rathnayake & Thielecke, SOS 2011, Def 5.2) per byte, the active set in
// registers (or a state id of the cache of macro steps) and the tables in
// shared memory.  Work distribution: the strings are ordered by length,
// longest first -- by default each block orders its own range in shared
// memory (k_stream_local), otherwise the planner orders the whole batch
// (k_stream) -- and warps take rounds of 32 consecutive entries from a
// counter, so the lanes of a round have (nearly) the same length and finish
// together, and the longest rounds start first.  Input: every lane reads its
// string in aligned 32-byte blocks (one full sector, one 256-bit load) with
// loads issued two blocks ahead.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "kernels.cuh"
#include "plan.cuh"
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

// the same load at addr + OFF, issued only when `on`; when it is not, the
// registers keep their values
template <int OFF>
__device__ __forceinline__ void ld_blk_if(Blk32& r, uint64_t addr, bool on) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %9, 0;\n"
        " @p ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8+%10];\n}"
        : "+r"(r.a.x), "+r"(r.a.y), "+r"(r.a.z), "+r"(r.a.w), "+r"(r.b.x), "+r"(r.b.y), "+r"(r.b.z), "+r"(r.b.w)
        : "l"(addr), "r"((uint32_t)on), "n"(OFF));
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

// byte i (0..31, any lane-dependent value) of the block
__device__ __forceinline__ uint32_t byte_at(const Blk32& v, uint32_t i) {
    const uint32_t q = i >> 2;
    const uint32_t lo = q & 1u ? (q & 2u ? v.a.w : v.a.y) : (q & 2u ? v.a.z : v.a.x);
    const uint32_t hi = q & 1u ? (q & 2u ? v.b.w : v.b.y) : (q & 2u ? v.b.z : v.b.x);
    return byte_k(q & 4u ? hi : lo, (int)(i & 3u));
}

// bytes 4q..4q+3 of `mask` widened to 0x00 / 0xFF per byte
__device__ __forceinline__ uint32_t byte_lanes(uint32_t mask, int q) {
    return (((mask >> (4 * q)) & 0xFu) * 0x00204081u & 0x01010101u) * 0xFFu;
}

// A block whose valid bytes [lo, hi) do not fill it (the first or last
// block of a string), with the two-byte table: an odd first byte alone,
// then the pairs that lie inside the range, then an odd last byte alone.
// Every lane issues every lookup; a lookup outside its range is dropped.
template <class S>
__device__ __forceinline__ void block32_pairs_masked(S& st, const Blk32& v, uint32_t mask) {
    const uint32_t lo = mask ? (uint32_t)__ffs(mask) - 1u : 0u;
    const uint32_t hi = mask ? 32u - (uint32_t)__clz(mask) : 0u;
    {
        S nx = st;
        nx.step(byte_at(v, lo));
        if (lo & 1u) st = nx;
    }
    const uint32_t lo2 = (lo + 1u) >> 1, hi2 = hi >> 1;  // pairs [lo2, hi2)
    const uint32_t pm = ((1u << hi2) - 1u) & ~((1u << lo2) - 1u);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const uint32_t w = word_of(v, q);
        S nx = st;
        nx.step2(w);
        if ((pm >> (2 * q)) & 1u) st = nx;
        nx = st;
        nx.step2(w >> 16);
        if ((pm >> (2 * q + 1)) & 1u) st = nx;
    }
    S nx = st;
    nx.step(byte_at(v, hi - 1u));
    if (hi & 1u) st = nx;
}

template <class S>
__device__ __forceinline__ void block32(S& st, const Blk32& v, uint32_t mask) {
    if constexpr (has_pairs<S>::value) {
        // two bytes per lookup when every valid byte of every lane is inside
        // the window; one vote decides between whole and partial blocks
        const bool whole = mask == 0u || mask == 0xffffffffu;
        uint32_t out = 0;
        if (whole) {
            if (mask) {
#pragma unroll
                for (int q = 0; q < 8; q++) out |= st.out_of_window(word_of(v, q));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++) out |= st.out_of_window(word_of(v, q)) & byte_lanes(mask, q);
        }
        const unsigned f = __reduce_or_sync(FULL, (whole ? 0u : 1u) | (out ? 2u : 0u));
        if (f == 0u) {
#pragma unroll
            for (int q = 0; q < 8; q++) st.step4(word_of(v, q));
            return;
        }
        if (f == 1u) {
            block32_pairs_masked(st, v, mask);
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

// A block that lies wholly inside the string of every lane still walking
// one: no masks and no ends.  `live`: the lane's set is not empty (a lane
// whose set is empty, or that has no string, skips the lookups).  With the
// two-byte table every label lies inside its 32-value window, so a byte
// outside it matches no position and empties the set (Def 5.2): the lane
// steps the block's pairs with the window bits dropped, then empties its
// set if any byte was outside.
template <class S>
__device__ __forceinline__ void block32_whole(S& st, const Blk32& v, bool live) {
    if constexpr (has_pairs<S>::value) {
        uint32_t x = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) x |= word_of(v, q) ^ st.win;
        if (live) {
#pragma unroll
            for (int q = 0; q < 8; q++) st.step4(word_of(v, q));
        }
        if (x & 0xE0E0E0E0u) st.kill();
    } else {
        if (live) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t w = word_of(v, q);
#pragma unroll
                for (int k = 0; k < 4; k++) st.step(byte_k(w, k));
            }
        }
    }
}

// One round: lane l walks string `id` (valid: the lane has a string) from
// its first 32-byte block to its end, or until its set empties (stuck), and
// writes its result; the warp steps while any lane is active.  A string
// touching nb blocks has whole blocks 1 .. nb-2; the lanes of a round (one
// length bucket) mostly share nb, so the round runs as its first block with
// per-lane masks, then the blocks that are whole for every lane with no
// per-lane bookkeeping, then the rest with masks and ends again.  Each
// lane's loads run two blocks ahead of its lookups.
template <class S>
__device__ __forceinline__ void stream_round(const S& proto, uint64_t base, const int64_t* __restrict__ off,
                                             long long id, bool valid, uint8_t* __restrict__ out,
                                             unsigned long long* __restrict__ bad) {
    uint64_t s = base, e = base;
    const bool ok = !valid || string_span(off, id, base, s, e);
    S st = proto;
    bool active = valid && ok && s < e;
    if (valid && !active) out[id] = ok ? (uint8_t)st.accept() : kResultInvalid;
    if (!ok) count_bad(bad);
    if (!active) st.kill();
    if (!__any_sync(FULL, active)) return;
    const uint64_t blk = s & ~uint64_t(31);
    // blocks touched (saturated: a string of 128 GiB or more counts 2^32 - 1;
    // the middle loop stops by 2^31 blocks and the rest compares addresses)
    const uint64_t nb64 = (e - blk + 31) >> 5;
    const uint32_t nb = active ? (nb64 < 0xffffffffull ? (uint32_t)nb64 : 0xffffffffu) : 0u;
    const uint32_t nb_lo = min(__reduce_min_sync(FULL, active ? nb : 0xffffffffu), 0x80000000u);
    Blk32 va = ld_blk(blk, active);
    Blk32 vb = ld_blk(blk + 32, nb > 1);
    // block 0
    block32(st, va, valid_mask(blk, s, e, active));
    if (active && (nb == 1 || st.dead())) {
        out[id] = st.accept();
        st.kill();
        active = false;
    }
    ld_blk_if<64>(va, blk, active && nb > 2);
    // vb holds block k and va block k + 1 (p = address of block k); blocks
    // k and k + 1 are whole for every lane while k + 3 <= nb_lo, and block
    // k + 2 exists for every lane still walking (k + 2 < nb_lo <= nb)
    uint32_t k = 1;
    uint64_t p = blk + 32;
    while (k + 3 <= nb_lo) {
        bool live = !st.dead();
        block32_whole(st, vb, live);
        ld_blk_if<64>(vb, p, live);
        live = !st.dead();
        block32_whole(st, va, live);
        ld_blk_if<96>(va, p, live && k + 3 < nb);
        k += 2;
        p += 64;
        if (!__any_sync(FULL, live)) break;
    }
    // the rest: per-lane masks and ends (vb holds the block at p, va the
    // block at p + 32)
    while (__any_sync(FULL, active)) {
        block32(st, vb, valid_mask(p, s, e, active));
        if (active && (p + 32 >= e || st.dead())) {
            out[id] = st.accept();
            st.kill();
            active = false;
        }
        ld_blk_if<64>(vb, p, active && p + 64 < e);
        if (!__any_sync(FULL, active)) break;
        block32(st, va, valid_mask(p + 32, s, e, active));
        if (active && (p + 64 >= e || st.dead())) {
            out[id] = st.accept();
            st.kill();
            active = false;
        }
        ld_blk_if<96>(va, p, active && p + 96 < e);
        p += 64;
    }
}

// the two-byte stepper is held to 40 registers: three 512-thread blocks
// (48 warps) per SM, which its shared memory (up to 3 planes) also allows
template <class S>
__global__ void __launch_bounds__(STREAM_MAX_BLOCK, has_pairs<S>::value ? 3 : 1)
    k_stream(const DevTables t, const uint8_t* __restrict__ str, const int64_t* __restrict__ off,
             const uint32_t* __restrict__ perm, long long n, uint8_t* __restrict__ out,
             unsigned* __restrict__ queue, unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) uint8_t smem[];
    S::load(t, smem);
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    // a warp takes round r (entries 32r .. 32r+31 of the order) from the
    // work counter; lane l walks string perm[32r + l] (32r + l without one)
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
        stream_round(proto, base, off, id, valid, out, bad);
    }
}

__device__ unsigned g_wait_faults;

// ------------------------------------------------ block-local length order
// One launch, no global planner and no scratch.  Block b owns the
// contiguous range of strings [b * per_block, (b + 1) * per_block) and walks
// it in tiles of up to kLocalTile strings.  For a tile it counts the length
// keys of its strings (the planner's buckets) in shared memory, scans the
// counts, and places the tile's strings into a shared order, longest first
// (each thread keeps its strings' keys in registers across the scan); its warps
// then take rounds of 32 consecutive entries from a shared counter, so the
// lanes of a round walk strings of (nearly) the same length, as with the
// global order: a range of a few thousand random strings has the length mix
// of the whole batch.  Nothing waits on another block.  Two 768-thread
// blocks per SM (48 warps, 40 registers) leave room in shared memory for
// the order beside the tables without changing the plain kernel's
// shared-memory carveout.
constexpr int kLocalThreads = 768;
constexpr int kLocalTile = 4096;

// exclusive scan of a[0..nbk) in shared memory, in place, by the block
__device__ inline void block_scan_smem(unsigned* a, int nbk) {
    __shared__ unsigned wsum[32];
    const int nt = blockDim.x, nw = nt >> 5;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned v = t < nbk ? a[t] : 0u;  // nbk <= blockDim.x
    unsigned incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned u = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned w = lane < nw ? wsum[lane] : 0u, wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_up_sync(FULL, wi, d);
            if (lane >= d) wi += u;
        }
        if (lane < nw) wsum[lane] = wi - w;
    }
    __syncthreads();
    if (t < nbk) a[t] = wsum[wid] + incl - v;
    __syncthreads();
}

constexpr int kLocalKeys = (kLocalTile + kLocalThreads - 1) / kLocalThreads;

template <class S>
__global__ void __launch_bounds__(kLocalThreads, has_pairs<S>::value ? 2 : 1)
    k_stream_local(const DevTables t, const uint8_t* __restrict__ str, const int64_t* __restrict__ off, long long n,
                   uint8_t* __restrict__ out, long long per_block, int mis, unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) uint8_t smem[];
    unsigned* cnt = reinterpret_cast<unsigned*>(smem + align16(S::smem_bytes(t)));
    uint16_t* ord = reinterpret_cast<uint16_t*>(cnt + kLenBuckets);
    __shared__ unsigned next_round;
    S::load(t, smem);
    S proto;
    proto.bind(t, smem);
    const long long lo = min((long long)blockIdx.x * per_block, n), hi = min(lo + per_block, n);
    // the host checked that the table's 16-bit shared addresses fit; in a
    // layout where they do not (block-uniform), the block counts a fault and
    // marks its strings invalid instead of walking them
    if constexpr (std::is_same<S, MemoPairA>::value) {
        if (!S::abs_fits(t, smem_addr(smem))) {
            if (threadIdx.x == 0) atomicAdd(&g_wait_faults, 1u);
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) out[i] = kResultInvalid;
            return;
        }
    }
    const int lane = threadIdx.x & 31;
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    for (long long t0 = lo; t0 < hi; t0 += kLocalTile) {
        const int m = (int)min((long long)kLocalTile, hi - t0);
        for (int b = threadIdx.x; b < kLenBuckets; b += blockDim.x) cnt[b] = 0;
        if (threadIdx.x == 0) next_round = 0;
        __syncthreads();  // also orders the table copy before the rounds
        int key[kLocalKeys];  // loads of a thread's keys in flight together
#pragma unroll
        for (int q = 0; q < kLocalKeys; q++) {
            const int j = q * kLocalThreads + (int)threadIdx.x;
            key[q] = j < m ? plan::plan_key(off, nullptr, t0 + j, 0, mis) : -1;
        }
#pragma unroll
        for (int q = 0; q < kLocalKeys; q++)
            if (key[q] >= 0) atomicAdd(&cnt[key[q]], 1u);
        __syncthreads();
        block_scan_smem(cnt, kLenBuckets);
#pragma unroll
        for (int q = 0; q < kLocalKeys; q++)
            if (key[q] >= 0) ord[atomicAdd(&cnt[key[q]], 1u)] = (uint16_t)(q * kLocalThreads + (int)threadIdx.x);
        __syncthreads();
        const int nround = (m + 31) / 32;
        for (;;) {
            unsigned r = 0;
            if (lane == 0) r = atomicAdd(&next_round, 1u);
            r = __shfl_sync(FULL, r, 0);
            if ((int)r >= nround) break;
            const int k = (int)r * 32 + lane;
            const bool valid = k < m;
            const long long id = valid ? t0 + ord[k] : 0;
            stream_round(proto, base, off, id, valid, out, bad);
        }
        __syncthreads();  // the order and the counts are reused by the next tile
    }
}

// ------------------------------------------------------------------ TMA
// The same rounds with the input staged into shared memory by the bulk-copy
// (TMA) engine instead of per-lane global loads: for every 32*CH-byte step
// of a round each lane asks for its next CH bytes (whole aligned 32-byte
// blocks) with one cp.async.bulk into its slot of a stage; the warp's
// stage completes on an mbarrier (lane 0 arrives with the warp's byte
// total, the copies complete the transaction count); lanes then read their
// slot with 128-bit shared loads.  NST stages per warp keep NST-1 steps in
// flight.  A lane slot is CH + 16 bytes, so the 32 lanes' 128-bit reads
// cover all 32 banks in four wavefronts.  Every wait is bounded: a warp
// whose stage does not complete counts a fault (rx_device_faults), waits a
// bounded time for its copies in flight and leaves.

// each try_wait suspends for at most about kWaitHintNs; a wait gives up
// after kWaitSpins of them (about 0.2 s)
constexpr uint32_t kWaitSpins = 10000;
constexpr uint32_t kWaitHintNs = 20000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of `bar` with this parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitSpins; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, uint64_t src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ Blk32 lds_blk(uint32_t a) {
    Blk32 r;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.a.x), "=r"(r.a.y), "=r"(r.a.z), "=r"(r.a.w)
                 : "r"(a));
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.b.x), "=r"(r.b.y), "=r"(r.b.z), "=r"(r.b.w)
                 : "r"(a + 16));
    return r;
}

template <int CH, int NST>
struct TmaLayout {
    static constexpr int kSlot = CH + 16;
    static constexpr size_t per_warp() { return (size_t)NST * 32 * kSlot + (size_t)NST * 8; }
};

template <class S, int CH, int NST>
__global__ void __launch_bounds__(1024, 1) k_stream_tma(const DevTables t, const uint8_t* __restrict__ str,
                                                     const int64_t* __restrict__ off,
                                                     const uint32_t* __restrict__ perm, long long n,
                                                     uint8_t* __restrict__ out, unsigned* __restrict__ queue,
                                                     unsigned long long* __restrict__ bad) {
    static_assert(CH % 32 == 0, "steps of whole 32-byte blocks");
    using Lay = TmaLayout<CH, NST>;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t tab = align16(S::smem_bytes(t));
    uint8_t* stg = smem + tab + (size_t)wid * NST * 32 * Lay::kSlot;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tab + (size_t)nw * NST * 32 * Lay::kSlot) + wid * NST;
    S::load(t, smem);
    if (lane == 0)
        for (int q = 0; q < NST; q++) mbar_init(smem_u32(bars + q), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    const uint32_t slot0 = smem_u32(stg) + lane * Lay::kSlot;
    const uint32_t bar0 = smem_u32(bars);
    uint32_t parity = 0;  // bit q: the parity of the next phase of stage q
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    const long long nround = (n + 31) / 32;
    bool failed = false;
    for (;;) {
        unsigned r = 0;
        if (lane == 0) r = atomicAdd(queue, 1u);
        r = __shfl_sync(FULL, r, 0);
        if ((long long)r >= nround) break;
        const long long k = (long long)r * 32 + lane;
        const bool valid = k < n;
        const long long id = valid ? (perm ? (long long)perm[k] : k) : 0;
        uint64_t s = base, e = base;
        const bool ok = !valid || string_span(off, id, base, s, e);
        S st = proto;
        bool active = valid && ok && s < e;
        if (valid && !active) out[id] = ok ? (uint8_t)st.accept() : kResultInvalid;
        if (!ok) count_bad(bad);
        if (!active) st.kill();
        const uint64_t blk0 = s & ~uint64_t(31);
        // steps of CH bytes this lane needs, and the round's
        const uint32_t my_steps = active ? (uint32_t)((e - blk0 + CH - 1) / CH) : 0u;
        const uint32_t nsteps = __reduce_max_sync(FULL, my_steps);
        // ask for step q of every lane that still reads into stage q % NST
        auto issue = [&](uint32_t q) {
            const uint64_t src = blk0 + (uint64_t)q * CH;
            uint32_t bytes = 0;
            if (active && src < e) {
                const uint64_t end = (e + 31) & ~uint64_t(31);
                bytes = (uint32_t)min((uint64_t)CH, end - src);
            }
            const uint32_t total = __reduce_add_sync(FULL, bytes);
            const uint32_t bar = bar0 + (q % NST) * 8u;
            if (lane == 0) mbar_arrive_expect(bar, total);
            __syncwarp();
            if (bytes) bulk_g2s(slot0 + (q % NST) * 32u * Lay::kSlot, src, bytes, bar);
        };
        uint32_t issued = 0;
        for (; issued < nsteps && issued < (uint32_t)NST - 1u; issued++) issue(issued);
        for (uint32_t q = 0; q < nsteps; q++) {
            if (issued < nsteps) {
                issue(issued);  // into the stage consumed at step q - 1
                issued++;
            }
            const uint32_t sq = q % NST;
            const bool ok = mbar_wait(bar0 + sq * 8u, (parity >> sq) & 1u);
            parity ^= 1u << sq;
            if (!__all_sync(FULL, ok)) {
                failed = true;
                break;
            }
            const uint32_t slot = slot0 + sq * 32u * Lay::kSlot;
#pragma unroll
            for (int b = 0; b < CH / 32; b++) {
                const Blk32 v = lds_blk(slot + b * 32);
                const uint64_t blk = blk0 + (uint64_t)q * CH + b * 32;
                block32(st, v, valid_mask(blk, s, e, active));
                if (active && (blk + 32 >= e || st.dead())) {
                    out[id] = st.accept();
                    st.kill();
                    active = false;
                }
            }
            // the reads of this stage are done before the next copy into it
            __syncwarp();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!__any_sync(FULL, active)) {
                // drain the steps already asked for
                for (uint32_t d = q + 1; d < issued; d++) {
                    const uint32_t sd = d % NST;
                    if (!__all_sync(FULL, mbar_wait(bar0 + sd * 8u, (parity >> sd) & 1u))) failed = true;
                    parity ^= 1u << sd;
                }
                break;
            }
        }
        if (failed) break;
    }
    if (failed) {
        // bounded waits for any copy still in flight into this warp's stages
        for (int q = 0; q < NST; q++) mbar_wait(bar0 + q * 8u, (parity >> q) & 1u);
        if (lane == 0) atomicAdd(&g_wait_faults, 1u);
    }
}

// ---------------------------------------------------------------- search
// Unanchored search: the earliest end of a matching substring.  The same
// rounds as k_stream over the search cache (the start set added back after
// every byte, so a match may begin anywhere); a lane records the first byte
// after which its state holds null and stops reading (SearchS).
// steps over the bytes of a 32-byte block selected by mask; returns the
// index of the first byte after which the state accepts (-1: none), and
// stops stepping there
__device__ __forceinline__ int search32(SearchS& st, const Blk32& v, uint32_t mask) {
    int hit = -1;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const uint32_t w = word_of(v, q);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int i = 4 * q + k;
            if (((mask >> i) & 1u) && hit < 0) {
                st.step(byte_k(w, k));
                if (st.accepted()) hit = i;
            }
        }
    }
    return hit;
}

__global__ void __launch_bounds__(STREAM_MAX_BLOCK) k_search(const DevTables t, const uint8_t* __restrict__ str,
                                                           const int64_t* __restrict__ off,
                                                           const uint32_t* __restrict__ perm, long long n,
                                                           int64_t* __restrict__ out, unsigned* __restrict__ queue,
                                                           unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) uint8_t smem[];
    SearchS::load(t, smem);
    __syncthreads();
    SearchS proto;
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
        const bool ok = !valid || string_span(off, id, base, s, e);
        if (!ok) count_bad(bad);
        SearchS st = proto;
        int64_t found = ok ? -1 : kSearchInvalid;
        if (valid && ok && st.accepted()) found = 0;  // the empty substring at 0
        bool active = valid && found == -1 && s < e;
        uint64_t blk = s & ~uint64_t(31);
        Blk32 va = ld_blk(blk, active);
        Blk32 vb = ld_blk(blk + 32, active && blk + 32 < e);
        while (__any_sync(FULL, active)) {
            int hit = search32(st, va, valid_mask(blk, s, e, active));
            if (active && hit >= 0) {
                found = (int64_t)(blk + hit - s) + 1;
                active = false;
            }
            if (active && blk + 32 >= e) active = false;
            va = ld_blk(blk + 64, active && blk + 64 < e);
            if (!__any_sync(FULL, active)) break;
            hit = search32(st, vb, valid_mask(blk + 32, s, e, active));
            if (active && hit >= 0) {
                found = (int64_t)(blk + 32 + hit - s) + 1;
                active = false;
            }
            if (active && blk + 64 >= e) active = false;
            vb = ld_blk(blk + 96, active && blk + 96 < e);
            blk += 64;
        }
        if (valid) out[id] = found;
    }
}

// Tasks of the chunked search: task i starts the search cache in state
// task_state[i] at byte task_chunk[i] * C + P of the text and runs to the end
// of that chunk or to its first accepting byte; res_acc[i] = that byte's end
// offset from the chunk start (-1: none), res[i] = the final state (only used
// when there is no accept).  Tasks come chunk by chunk.
__global__ void __launch_bounds__(STREAM_MAX_BLOCK) k_search_tasks(const DevTables t, const uint8_t* __restrict__ str,
                                                                 int64_t len, int64_t C, int64_t P,
                                                                 const uint32_t* __restrict__ task_chunk,
                                                                 const uint16_t* __restrict__ task_state,
                                                                 const unsigned* __restrict__ ntask_p,
                                                                 uint16_t* __restrict__ res,
                                                                 int32_t* __restrict__ res_acc,
                                                                 unsigned* __restrict__ queue) {
    extern __shared__ __align__(16) uint8_t smem[];
    SearchS::load(t, smem);
    __syncthreads();
    SearchS proto;
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
        uint64_t s = base, e = base, c0 = base;
        SearchS st = proto;
        if (valid) {
            const int64_t j = task_chunk[k];
            const int64_t lo = j * C, hi = min(lo + C, len);
            c0 += (uint64_t)lo;
            s += (uint64_t)min(lo + P, hi);
            e += (uint64_t)hi;
            st.set_state(task_state[k]);
        }
        int32_t acc = -1;
        bool active = valid && s < e;
        uint64_t blk = s & ~uint64_t(31);
        Blk32 va = ld_blk(blk, active);
        Blk32 vb = ld_blk(blk + 32, active && blk + 32 < e);
        while (__any_sync(FULL, active)) {
            int hit = search32(st, va, valid_mask(blk, s, e, active));
            if (active && hit >= 0) {
                acc = (int32_t)(blk + hit - c0) + 1;
                active = false;
            }
            if (active && blk + 32 >= e) active = false;
            va = ld_blk(blk + 64, active && blk + 64 < e);
            if (!__any_sync(FULL, active)) break;
            hit = search32(st, vb, valid_mask(blk + 32, s, e, active));
            if (active && hit >= 0) {
                acc = (int32_t)(blk + 32 + hit - c0) + 1;
                active = false;
            }
            if (active && blk + 64 >= e) active = false;
            vb = ld_blk(blk + 96, active && blk + 96 < e);
            blk += 64;
        }
        if (valid) {
            res[k] = (uint16_t)st.state_id();
            res_acc[k] = acc;
        }
    }
}

constexpr int kSpanMaxBlock = 768;

// Tasks of the chunked long-string mode.  A task holds one or two live cache
// states of one chunk and runs from byte j * C + pstart[j] of the text (j =
// task_chunk[k]) to the end of that chunk.  Two states of one chunk share a
// lane: they read the same bytes, and since a macro step is a function of
// the state (Def 5.2), two states that meet -- compared after every 32-byte
// block -- stay together, so the second is dropped there and takes the
// first one's result.  The first state's final id goes to res[task_res[k]],
// the second's to res[task_res[k] + 1].  ntask[0] two-state tasks sit at
// [pair_base, pair_base + ntask[0]), ntask[1] one-state tasks at
// [0, ntask[1]); the two-state rounds are taken first.  Spans of one chunk
// size, so the 32 lanes of a round cover equal-length spans.

// one 32-byte block for both states of the lanes (b: dead where hasb is
// false); the pair loop when every valid byte of every lane is in the window
template <class S>
__device__ __forceinline__ void block32_two(S& a, S& b, bool hasb, const Blk32& v, uint32_t mask) {
    if constexpr (has_pairs<S>::value) {
        const bool whole = mask == 0u || mask == 0xffffffffu;
        uint32_t outw = 0;
        if (whole && mask) {
#pragma unroll
            for (int q = 0; q < 8; q++) outw |= a.out_of_window(word_of(v, q));
        }
        if (__all_sync(FULL, whole && outw == 0u)) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t w = word_of(v, q);
                a.step2(w);
                if (hasb) b.step2(w);
                a.step2(w >> 16);
                if (hasb) b.step2(w >> 16);
            }
            return;
        }
    }
    block32(a, v, mask);
    block32(b, v, hasb ? mask : 0u);
}

// one block of a task's span, then the checks that end, merge or drop its
// states.  The first state's result slot is ia, the second's ia + 1; tie:
// the second met the first and takes its result.  two: warp-uniform, some
// lane of a two-state round still holds two states.
// rem: bytes of the span from this block's start, skip: bytes of this block
// before the span (first block only)
template <class S>
__device__ __forceinline__ void span_block(S& a, S& b, bool& hasb, bool& tie, bool& active, uint32_t& ia, bool two,
                                           const Blk32& v, uint32_t rem, uint32_t skip,
                                           uint16_t* __restrict__ res) {
    const uint32_t mask = !active ? 0u : (rem >= 32u ? 0xffffffffu : (1u << rem) - 1u) & ~((1u << skip) - 1u);
    if (two) block32_two(a, b, hasb, v, mask);
    else block32(a, v, mask);
    if (!active) return;
    if (hasb && a.st == b.st) {  // met: the second state follows the first
        tie = true;
        hasb = false;
        b.kill();
    }
    if (hasb && b.dead()) {
        res[ia + 1] = 0;
        hasb = false;
    }
    if (a.dead()) {
        res[ia] = 0;
        if (tie) res[ia + 1] = 0;
        tie = false;
        if (hasb) {  // the second state carries on alone
            a = b;
            ia += 1;
            hasb = false;
            b.kill();
        } else {
            active = false;
            return;
        }
    }
    if (rem <= 32u) {
        const uint16_t f = (uint16_t)a.state_id();
        res[ia] = f;
        if (tie || hasb) res[ia + 1] = tie ? f : (uint16_t)b.state_id();
        a.kill();
        b.kill();
        hasb = false;
        active = false;
    }
}

// The pair stepper is held to 40 registers (two 768-thread blocks per SM);
// the block size is picked per table size from 256, 512 and 768 threads,
// whichever keeps the most warps resident beside the planes of the table.
template <class S>
__global__ void __launch_bounds__(kSpanMaxBlock, has_pairs<S>::value ? 2 : 1)
    k_span_tasks(const DevTables t, const uint8_t* __restrict__ str, int64_t len, int64_t C,
                 const uint32_t* __restrict__ task_chunk, const uint16_t* __restrict__ task_state,
                 const uint32_t* __restrict__ task_res, const unsigned* __restrict__ ntask, long long pair_base,
                 const uint16_t* __restrict__ pstart, uint16_t* __restrict__ res, unsigned* __restrict__ queue) {
    extern __shared__ __align__(16) uint8_t smem[];
    S::load(t, smem);
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    const int lane = threadIdx.x & 31;
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    const long long n2 = ntask[0], n1 = ntask[1];
    const long long r2 = (n2 + 31) / 32, nround = r2 + (n1 + 31) / 32;
    for (;;) {
        unsigned r = 0;
        if (lane == 0) r = atomicAdd(queue, 1u);
        r = __shfl_sync(FULL, r, 0);
        if ((long long)r >= nround) break;
        const bool two_round = (long long)r < r2;  // warp-uniform
        const long long k = (two_round ? (long long)r : (long long)r - r2) * 32 + lane;
        const bool valid = k < (two_round ? n2 : n1);
        const long long ti = two_round ? pair_base + k : k;
        uint64_t s = base, e = base;
        S a = proto, b = proto;
        a.kill();
        b.kill();
        uint32_t ia = 0;
        bool hasb = false, tie = false;
        if (valid) {
            const int64_t j = task_chunk[ti];
            const int64_t lo = j * C, hi = min(lo + C, len);
            s += (uint64_t)min(lo + (int64_t)pstart[j], hi);
            e += (uint64_t)hi;
            const uint32_t ts = task_state[ti];
            ia = task_res[ti];
            a.set_state(ts & 0xFFu);
            if (two_round) {
                b.set_state(ts >> 8);
                hasb = true;
            }
        }
        bool active = valid && s < e;
        if (valid && !active) {  // the prefix took the whole chunk
            res[ia] = (uint16_t)a.state_id();
            if (hasb) res[ia + 1] = (uint16_t)b.state_id();
        }
        if (!active) {
            a.kill();
            b.kill();
            hasb = false;
        }
        // the span [s, e) as its first aligned block, the bytes from there
        // to e (spans are below 4 GiB: chunks are) and the bytes skipped
        uint64_t blk = s & ~uint64_t(31);
        uint32_t rem = (uint32_t)(e - blk), skip = (uint32_t)(s - blk);
        Blk32 va = ld_blk(blk, active);
        Blk32 vb = ld_blk(blk + 32, active && rem > 32u);
        while (__any_sync(FULL, active)) {
            // block A at blk, then block B at blk + 32, each refilled two
            // blocks ahead right after it is consumed
            span_block(a, b, hasb, tie, active, ia, two_round && __any_sync(FULL, hasb), va, rem, skip, res);
            va = ld_blk(blk + 64, active && rem > 64u);
            if (!__any_sync(FULL, active)) break;
            span_block(a, b, hasb, tie, active, ia, two_round && __any_sync(FULL, hasb), vb, rem - 32u, 0u, res);
            vb = ld_blk(blk + 96, active && rem > 96u);
            blk += 64;
            rem -= 64u;
            skip = 0u;
        }
    }
}

int resident_blocks(const void* kern, int block, size_t smem);

// the block size (of 768, 512, 256) that keeps the most threads of the span
// kernel resident beside its table; per_sm = 0 when none fits
template <class S>
void span_shape(const DevTables& t, int* block, int* per_sm) {
    const size_t sm = S::smem_bytes(t);
    const void* kern = reinterpret_cast<const void*>(k_span_tasks<S>);
    *block = 256;
    *per_sm = 0;
    for (int b : {kSpanMaxBlock, 512, 256}) {
        const int r = resident_blocks(kern, b, sm);
        if (r * b > *per_sm * *block) {
            *per_sm = r;
            *block = b;
        }
    }
}

template <class S>
cudaError_t launch_span_t(const DevTables& t, const uint8_t* str, int64_t len, int64_t C,
                          const uint32_t* task_chunk, const uint16_t* task_state, const uint32_t* task_res,
                          const unsigned* ntask, long long pair_base, const uint16_t* pstart, uint16_t* res,
                          unsigned* queue, long long max_tasks, cudaStream_t st) {
    size_t sm = S::smem_bytes(t);
    auto kern = k_span_tasks<S>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0, block = 256;
    span_shape<S>(t, &block, &per_sm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>((max_tasks + block - 1) / block, (long long)per_sm * sm_count());
    {
        ProfScope ps(st);
        kern<<<(unsigned)std::max<long long>(grid, 1), block, sm, st>>>(t, str, len, C, task_chunk, task_state,
                                                                        task_res, ntask, pair_base, pstart, res,
                                                                        queue);
    }
    return cudaGetLastError();
}

// blocks of `kern` resident per SM with `smem` bytes of dynamic shared
// memory (cached per device)
int resident_blocks(const void* kern, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, kern, block, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (allow_smem_raw(kern, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    cache[key] = per_sm;
    return per_sm;
}

// The block-local order: launched (*launched = true) when two blocks of
// the kernel fit on an SM beside the tables (else nothing is launched).
template <class S>
cudaError_t launch_stream_local_t(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                                  uint8_t* out, cudaStream_t st, bool* launched) {
    static_assert(kLocalThreads >= kLenBuckets, "one bucket per thread in the scan");
    static_assert(kLocalTile <= 65536, "tile indices in 16 bits");
    *launched = false;
    if (n <= 0) return cudaSuccess;
    auto kern = k_stream_local<S>;
    const size_t sm = align16(S::smem_bytes(t)) + (size_t)kLenBuckets * 4 + (size_t)kLocalTile * 2;
    const int per_sm = resident_blocks(reinterpret_cast<const void*>(kern), kLocalThreads, sm);
    if (per_sm < 2) return cudaSuccess;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>((long long)per_sm * sm_count(), (n + 31) / 32);
    const long long per_block = (n + grid - 1) / grid;
    const int mis = (int)(reinterpret_cast<uintptr_t>(str) & 31);
    {
        ProfScope ps(st);
        kern<<<(unsigned)grid, kLocalThreads, sm, st>>>(t, str, off, n, out, per_block, mis, bad_offsets_counter());
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) *launched = true;
    return e;
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
        kern<<<(unsigned)std::max<long long>(grid, 1), block, sm, st>>>(t, str, off, perm, n, out, queue,
                                                                        bad_offsets_counter());
    }
    return cudaGetLastError();
}

cudaError_t launch_search_k(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                            const uint32_t* perm, int64_t* out, unsigned* queue, cudaStream_t st) {
    const size_t sm = SearchS::smem_bytes(t);
    const int block = 512;
    cudaError_t e = allow_smem(k_search, sm);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search, block, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long rounds = (n + 31) / 32;
    long long grid = std::min<long long>((rounds * 32 + block - 1) / block, (long long)per_sm * sm_count());
    {
        ProfScope ps(st);
        k_search<<<(unsigned)std::max<long long>(grid, 1), block, sm, st>>>(t, str, off, perm, n, out, queue,
                                                                             bad_offsets_counter());
    }
    return cudaGetLastError();
}

template <class S, int CH, int NST>
cudaError_t launch_stream_tma_t(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                                const uint32_t* perm, uint8_t* out, unsigned* queue, cudaStream_t st) {
    const size_t tab = align16(S::smem_bytes(t));
    const size_t per = TmaLayout<CH, NST>::per_warp();
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((size_t)optin <= tab + 4 * per) return cudaErrorInvalidConfiguration;
    const int nw = (int)std::min<size_t>(32, ((size_t)optin - tab) / per);
    const size_t sm = tab + (size_t)nw * per;
    auto kern = k_stream_tma<S, CH, NST>;
    e = allow_smem(kern, sm);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nw * 32, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long rounds = (n + 31) / 32;
    long long grid = std::min<long long>((rounds + nw - 1) / nw, (long long)per_sm * sm_count());
    {
        ProfScope ps(st);
        kern<<<(unsigned)std::max<long long>(grid, 1), nw * 32, sm, st>>>(t, str, off, perm, n, out, queue,
                                                                          bad_offsets_counter());
    }
    return cudaGetLastError();
}

}  // namespace

bool stream_pairs(const DevTables& t) { return t.bgp_T != nullptr; }

unsigned read_wait_faults(bool reset) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_wait_faults, sizeof(v));
    if (reset) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_wait_faults, &z, sizeof(z));
    }
    return v;
}

size_t search_workspace_bytes(size_t n) { return 256 + plan_workspace_bytes(n, 1); }

cudaError_t launch_search(const DevTables& t, size_t n, const uint8_t* str, const int64_t* off, int64_t* out,
                          void* ws, size_t ws_bytes, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (t.srch_K <= 0) return cudaErrorInvalidValue;
    if (ws_bytes < search_workspace_bytes(n)) return cudaErrorInvalidValue;
    uint8_t* w = static_cast<uint8_t*>(ws);
    unsigned* queue = reinterpret_cast<unsigned*>(w);
    uint32_t* perm = nullptr;
    unsigned* starts = nullptr;
    cudaError_t e = launch_plan(off, nullptr, 1, n, w + 256, &perm, &starts, st, queue, 4096, str);
    if (e != cudaSuccess) return e;
    return launch_search_k(t, (long long)n, str, off, perm, out, queue, st);
}

cudaError_t launch_search_tasks(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, int64_t P,
                                const uint32_t* task_chunk, const uint16_t* task_state, const unsigned* ntask_p,
                                uint16_t* res, int32_t* res_acc, unsigned* queue, long long max_tasks,
                                cudaStream_t st) {
    const size_t sm = SearchS::smem_bytes(t);
    const int block = 256;
    cudaError_t e = allow_smem(k_search_tasks, sm);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search_tasks, block, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>((max_tasks + block - 1) / block, (long long)per_sm * sm_count());
    {
        ProfScope ps(st);
        k_search_tasks<<<(unsigned)std::max<long long>(grid, 1), block, sm, st>>>(t, str, len, C, P, task_chunk,
                                                                                 task_state, ntask_p, res, res_acc,
                                                                                 queue);
    }
    return cudaGetLastError();
}

long long span_resident_warps(const DevTables& t) {
    int block = 0, per_sm = 0;
    if (t.bgp_T) span_shape<MemoPairP>(t, &block, &per_sm);
    else span_shape<MemoS>(t, &block, &per_sm);
    return (long long)per_sm * (block / 32) * sm_count();
}

cudaError_t launch_span_tasks(const DevTables& t, const uint8_t* str, int64_t len, int64_t C,
                              const uint32_t* task_chunk, const uint16_t* task_state, const uint32_t* task_res,
                              const unsigned* ntask, long long pair_base, const uint16_t* pstart, uint16_t* res,
                              unsigned* queue, long long max_tasks, cudaStream_t st) {
    if (t.bgp_T)
        return launch_span_t<MemoPairP>(t, str, len, C, task_chunk, task_state, task_res, ntask, pair_base, pstart,
                                        res, queue, max_tasks, st);
    return launch_span_t<MemoS>(t, str, len, C, task_chunk, task_state, task_res, ntask, pair_base, pstart, res,
                                queue, max_tasks, st);
}

// An upper bound on the shared address where the dynamic shared memory of
// the absolute-address kernel starts: the block's reserved shared memory,
// then its static shared memory, plus 1 KiB of slack (65536 when the
// attributes cannot be read: the absolute form is then never taken).
static size_t local_abs_smem_start() {
    static const size_t v = [] {
        cudaFuncAttributes a{};
        int dev = 0, reserved = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(k_stream_local<MemoPairA>)) != cudaSuccess ||
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
            cudaGetLastError();
            return (size_t)65536;
        }
        return (size_t)reserved + a.sharedSizeBytes + 1024;
    }();
    return v;
}

cudaError_t launch_stream_local(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                                uint8_t* out, cudaStream_t st, bool* launched) {
    *launched = false;
    if (!t.bgp_T) return cudaSuccess;
    if (MemoPairA::abs_fits(t, local_abs_smem_start()))
        return launch_stream_local_t<MemoPairA>(t, n, str, off, out, st, launched);
    return launch_stream_local_t<MemoPairP>(t, n, str, off, out, st, launched);
}

bool stream_supported(const DevTables& t, int variant) {
    return variant == RX_VARIANT_MEMO || (variant == RX_VARIANT_THREAD && t.W <= 2);
}

cudaError_t launch_stream(const DevTables& t, int variant, long long n, const uint8_t* str, const int64_t* off,
                          const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st) {
    // the low bits of a block request choose the memo kernel: bit 0 the
    // single-byte lookup (else two bytes per lookup), bits 2-4 input staged
    // by the bulk-copy engine (4: 32-byte steps x 3 stages, 12: 64 x 2,
    // 20: 64 x 3)
    const int block_req = block & ~31;
    const int single = block & 1, tma = block & 28;
    block &= ~31;
    block = (block == 128 || block == 64 || block == 512) ? block : STREAM_BLOCK;
    if (variant == RX_VARIANT_MEMO) {
        if (t.bgp_T && !single && tma) {
            cudaError_t e = cudaErrorInvalidConfiguration;
            if (tma == 4) e = launch_stream_tma_t<MemoPairP, 32, 3>(t, n, str, off, perm, out, queue, st);
            if (tma == 12) e = launch_stream_tma_t<MemoPairP, 64, 2>(t, n, str, off, perm, out, queue, st);
            if (tma == 20) e = launch_stream_tma_t<MemoPairP, 64, 3>(t, n, str, off, perm, out, queue, st);
            if (e != cudaErrorInvalidConfiguration) return e;
            cudaGetLastError();  // tables too large to stage beside: the plain kernel below
        }
        // 512 threads: the autotuner's measured choice for the two-byte
        // kernel on the streaming workload (about 5% over 256)
        const int pb = block_req == 0 ? 512 : block;
        if (t.bgp_T && !single) return launch_stream_t<MemoPairP>(t, n, str, off, perm, out, queue, pb, st);
        return launch_stream_t<MemoS>(t, n, str, off, perm, out, queue, block, st);
    }
    if (t.W == 1) return launch_stream_t<Thread1S>(t, n, str, off, perm, out, queue, block & ~1, st);
    return launch_stream_t<Thread2S>(t, n, str, off, perm, out, queue, block & ~1, st);
}

}  // namespace rx
