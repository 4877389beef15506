// steppers.cuh -- device-side building blocks shared by the kernels: input
// loads and the steppers, each of which holds one active set and advances
// it by one macro step of the lockstep machine (Rathnayake & Thielecke,
// SOS 2011, Def 5.2) per input byte.
#pragma once

#include <cstdint>

#include "rx_internal.h"

namespace rx {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint4 ld_stream(const uint8_t* p) {
    return __ldcs(reinterpret_cast<const uint4*>(p));
}

__device__ __forceinline__ uint32_t byte_of(const uint4& v, int k) {
    uint32_t w = (k < 4) ? v.x : (k < 8) ? v.y : (k < 12) ? v.z : v.w;
    return (w >> (8 * (k & 3))) & 0xffu;
}

// cooperative copy global -> shared (16-byte granules; sizes rounded up);
// each thread issues four loads before it stores, so a table arrives in
// about one memory latency per 64 bytes a thread copies
__device__ inline void copy_to_smem(void* dst, const void* src, size_t bytes) {
    const uint4* __restrict__ s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    const size_t n = (bytes + 15) / 16, stride = blockDim.x;
    size_t i = threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = __ldg(s + i + k * stride);
#pragma unroll
        for (int k = 0; k < 4; k++) d[i + k * stride] = v[k];
    }
    for (; i < n; i += stride) d[i] = __ldg(s + i);
}
// the same, one load at a time (for kernels whose register budget is
// better spent elsewhere)
__device__ inline void copy_to_smem_serial(void* dst, const void* src, size_t bytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    const size_t n = (bytes + 15) / 16;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ------------------------------------------------------------- offsets
// String id of a batch is w = bytes[off[id] .. off[id+1]) (the problem
// statement e |v w of Section 2, one string per pair of offsets).  The pair
// is valid iff 0 <= off[id] <= off[id+1]; the kernels do not know the size
// of the bytes buffer, so off[n] is the caller's to keep inside it.  On a
// valid pair [s, e) are the absolute addresses of its bytes; on an invalid
// one s = e = base, so the lane reads nothing, and the kernel writes the
// marker result and counts the string in *bad (one atomic per bad string).
__device__ __forceinline__ bool string_span(const int64_t* __restrict__ off, long long id, uint64_t base,
                                            uint64_t& s, uint64_t& e) {
    const int64_t a = off[id], b = off[id + 1];
    const bool ok = a >= 0 && b >= a;
    s = base + (ok ? (uint64_t)a : 0ull);
    e = base + (ok ? (uint64_t)b : 0ull);
    return ok;
}
// result byte of a string with invalid offsets (RX_RESULT_INVALID of rx.h)
constexpr uint8_t kResultInvalid = 2;
// search result of a string with invalid offsets (RX_SEARCH_INVALID of rx.h)
constexpr int64_t kSearchInvalid = -2;
__device__ __forceinline__ void count_bad(unsigned long long* bad) { atomicAdd(bad, 1ull); }

// ------------------------------------------------------------- steppers
// A stepper holds one active set and advances it by one byte.  Interface:
//   smem_bytes(t) / load(t, smem) / bind(t, smem)   tables in shared memory
//   bind_global(t)                                  tables read from global
//   step(c)  dead()  accept()  kill()
//   set_unit(b)       the set {bit b} (start of a chunk transfer row)
//   store(dst)        write the set (ROW_WORDS words; memo writes the state id)

struct MemoStep {
    static constexpr int ROW_WORDS = 1;
    const uint32_t* T;
    const uint8_t* acc;
    uint32_t st;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return align16((size_t)t.memo_K * 1024) + align16(t.memo_K);
    }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        copy_to_smem(sm, t.memo_T, (size_t)t.memo_K * 1024);
        copy_to_smem(sm + align16((size_t)t.memo_K * 1024), t.memo_acc, t.memo_K);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        T = reinterpret_cast<const uint32_t*>(sm);
        acc = sm + align16((size_t)t.memo_K * 1024);
        st = t.memo_start;
    }
    __device__ void bind_global(const DevTables& t) {
        T = t.memo_T;
        acc = t.memo_acc;
        st = t.memo_start;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = T[st + c]; }
    __device__ __forceinline__ bool dead() const { return st == 0; }
    __device__ __forceinline__ bool accept() const { return acc[st >> 8] != 0; }
    __device__ __forceinline__ void kill() { st = 0; }
    __device__ __forceinline__ void set_state(uint32_t s) { st = s * 256u; }
    __device__ __forceinline__ void save(uint32_t* p) const { p[0] = st; }
    __device__ __forceinline__ void restore(const uint32_t* p) { st = p[0]; }
};

// The same cache read from global memory with one byte per entry (state
// ids < 256): a quarter of the footprint, so the tables of many expressions
// stay in L2.  st = state id * 256.
struct MemoStep8 {
    const uint8_t* T;
    const uint8_t* acc;
    uint32_t st;
    __device__ void bind_global(const DevTables& t) {
        T = t.memo_T8;
        acc = t.memo_acc;
        st = t.memo_start;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = (uint32_t)__ldg(T + st + c) << 8; }
    __device__ __forceinline__ bool dead() const { return st == 0; }
    __device__ __forceinline__ bool accept() const { return acc[st >> 8] != 0; }
    __device__ __forceinline__ void kill() { st = 0; }
    __device__ __forceinline__ void set_state(uint32_t s) { st = s * 256u; }
    __device__ __forceinline__ void save(uint32_t* p) const { p[0] = st; }
    __device__ __forceinline__ void restore(const uint32_t* p) { st = p[0]; }
};

struct Thread1Step {
    static constexpr int ROW_WORDS = 1;
    const uint2* desc;
    const uint32_t* tt;
    uint32_t F, nb;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return 256 * sizeof(uint2) + align16((size_t)t.gl_words * 4);
    }
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
    __device__ void bind_global(const DevTables& t) {
        desc = t.gl_desc;
        tt = t.gl_tt;
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
    __device__ __forceinline__ void set_unit(int b) { F = (b < 32) ? (1u << b) : 0u; }
    __device__ __forceinline__ void store(uint32_t* d) const { d[0] = F; }
    __device__ __forceinline__ void save(uint32_t* p) const { p[0] = F; }
    __device__ __forceinline__ void restore(const uint32_t* p) { F = p[0]; }
};

struct Thread2Step {
    static constexpr int ROW_WORDS = 2;
    const uint2* desc;
    const uint2* tt;
    uint32_t F0, F1, nb;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return 256 * sizeof(uint2) + align16((size_t)t.gl_words * 4);
    }
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
    __device__ void bind_global(const DevTables& t) {
        desc = t.gl_desc;
        tt = reinterpret_cast<const uint2*>(t.gl_tt);
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
    __device__ __forceinline__ void set_unit(int b) {
        F0 = (b < 32) ? (1u << b) : 0u;
        F1 = (b >= 32 && b < 64) ? (1u << (b - 32)) : 0u;
    }
    __device__ __forceinline__ void store(uint32_t* d) const {
        d[0] = F0;
        d[1] = F1;
    }
    __device__ __forceinline__ void save(uint32_t* p) const { store(p); }
    __device__ __forceinline__ void restore(const uint32_t* p) {
        F0 = p[0];
        F1 = p[1];
    }
};

// rows padded to W (4 or 8) words: t.sp_B [256*W], t.sp_follow [nbits*W]
template <int W>
struct SparseStep {
    static_assert(W % 4 == 0, "W must be a multiple of 4");
    static constexpr int ROW_WORDS = W;
    const uint32_t* B;
    const uint32_t* follow;
    uint32_t F[W];
    uint32_t nb;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return (size_t)256 * W * 4 + align16((size_t)t.nbits * W * 4);
    }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        copy_to_smem(sm, t.sp_B, (size_t)256 * W * 4);
        copy_to_smem(sm + (size_t)256 * W * 4, t.sp_follow, (size_t)t.nbits * W * 4);
    }
    __device__ void init(const DevTables& t) {
#pragma unroll
        for (int k = 0; k < W; k++) F[k] = t.sp_start[k];
        nb = t.null_bit;
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        B = reinterpret_cast<const uint32_t*>(sm);
        follow = B + 256 * W;
        init(t);
    }
    __device__ void bind_global(const DevTables& t) {
        B = t.sp_B;
        follow = t.sp_follow;
        init(t);
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
    __device__ __forceinline__ void set_unit(int b) {
#pragma unroll
        for (int k = 0; k < W; k++) F[k] = (k == (b >> 5)) ? (1u << (b & 31)) : 0u;
    }
    __device__ __forceinline__ void store(uint32_t* d) const {
#pragma unroll
        for (int k = 0; k < W; k++) d[k] = F[k];
    }
    __device__ __forceinline__ void save(uint32_t* p) const { store(p); }
    __device__ __forceinline__ void restore(const uint32_t* p) {
#pragma unroll
        for (int k = 0; k < W; k++) F[k] = p[k];
    }
};

// Advance a stepper over the bytes [s, e) (absolute addresses) -- every
// lane of the warp calls this with the SAME range (chunk kernels).  Stops
// early when every lane's set is empty.
template <class S>
__device__ __forceinline__ void run_range_uniform(S& st, uint64_t s, uint64_t e) {
    uint64_t blk = s & ~uint64_t(15);
    while (blk < e) {
        uint4 v = ld_stream(reinterpret_cast<const uint8_t*>(blk));
        if (blk >= s && blk + 16 <= e) {
#pragma unroll
            for (int k = 0; k < 16; k++) st.step(byte_of(v, k));
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) {
                bool ok = blk + k >= s && blk + k < e;
                if (ok) st.step(byte_of(v, k));
            }
        }
        blk += 16;
        if (__all_sync(FULL, st.dead())) break;
    }
}


}  // namespace dev
}  // namespace rx

namespace rx {
namespace dev {

// ---------------------------------------------------------------------------
// Shared-memory steppers addressed with 32-bit shared-window addresses.
// The tables are copied into shared memory with every stored pointer
// already converted to a shared address, so one step is: extract the byte,
// form the address, one 32-bit shared load.

__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t a) {
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds8(uint32_t a) {
    uint16_t v;
    asm("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte k (0..3) of w, zero-extended
__device__ __forceinline__ uint32_t byte_k(uint32_t w, int k) { return __byte_perm(w, 0u, 0x4440u | (uint32_t)k); }

// cache of macro steps: st = shared address of the current state's row of
// 256 entries; each entry is the shared address of the successor's row.
struct MemoS {
    uint32_t st, base, acc;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return align16((size_t)t.memo_K * 1024) + align16(t.memo_K);
    }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        uint32_t b = smem_addr(sm);
        uint32_t* T = reinterpret_cast<uint32_t*>(sm);
        for (int i = threadIdx.x; i < t.memo_K * 256; i += blockDim.x) T[i] = b + t.memo_T[i] * 4u;
        copy_to_smem(sm + align16((size_t)t.memo_K * 1024), t.memo_acc, t.memo_K);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        base = smem_addr(sm);
        acc = base + (uint32_t)align16((size_t)t.memo_K * 1024);
        st = base + t.memo_start * 4u;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = lds32(st + c * 4u); }
    __device__ __forceinline__ bool dead() const { return st == base; }
    __device__ __forceinline__ bool accept() const { return lds8(acc + ((st - base) >> 10)) != 0; }
    __device__ __forceinline__ void kill() { st = base; }
    __device__ __forceinline__ void set_state(uint32_t s) { st = base + s * 1024u; }
    __device__ __forceinline__ uint32_t state_id() const { return (st - base) >> 10; }
};

__device__ __forceinline__ uint32_t lds16(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// The two-byte cache in planes (see DevTables::bgp_T): st = shared address
// of the state's slot in its plane; a pair lookup (first byte i, second j)
// adds 2 * i + 516 * j to it -- pair rows are 516 bytes apart, so lanes in
// one state reading pairs with different second bytes fall in different
// banks -- and the entry read back is the successor's offset / 64.
// kAbs: the copy in shared memory holds the successor's shared address
// itself (base + offset), so a lookup needs no multiply-add after it; only
// for tables whose addresses fit in 16 bits (kAbsPlanes planes, checked by
// abs_fits on the host).
template <bool kAbs>
struct MemoPairT {
    static constexpr bool kPairs = true;
    static constexpr uint32_t PLANE = 20608;  // bytes per 8 states: 32 x 516 + 8 x 512
    static constexpr int kAbsPlanes = 3;
    uint32_t st, base, acc, win;
    __host__ __device__ static size_t planes(const DevTables& t) { return (size_t)(t.memo_K + 7) / 8; }
    __host__ __device__ static size_t smem_bytes(const DevTables& t) { return planes(t) * PLANE + align16(t.memo_K); }
    // the largest entry, base + offset of the last slot, below 2^16 when the
    // dynamic shared memory starts at or below smem_start
    __host__ __device__ static bool abs_fits(const DevTables& t, size_t smem_start) {
        return planes(t) <= (size_t)kAbsPlanes && smem_start + (planes(t) - 1) * PLANE + 7 * 64 < 65536;
    }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        if constexpr (kAbs) {
            const uint32_t b = smem_addr(sm);
            const uint32_t* __restrict__ src = reinterpret_cast<const uint32_t*>(t.bgp_T);
            uint32_t* d = reinterpret_cast<uint32_t*>(sm);
            const uint32_t n = (uint32_t)(planes(t) * PLANE / 4);
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t v = __ldg(src + i);
                d[i] = ((b + (v & 0xFFFFu) * 64u) & 0xFFFFu) | ((b + (v >> 16) * 64u) << 16);
            }
        } else {
            copy_to_smem(sm, t.bgp_T, planes(t) * PLANE);
        }
        copy_to_smem(sm + planes(t) * PLANE, t.memo_acc, t.memo_K);
    }
    // the state after the entry at shared address a
    __device__ __forceinline__ uint32_t next(uint32_t a) const { return kAbs ? lds16(a) : base + lds16(a) * 64u; }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        base = smem_addr(sm);
        acc = base + (uint32_t)(planes(t) * PLANE);
        set_state(t.memo_start >> 8);
        win = (uint32_t)t.bg_lo * 0x01010101u;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = next(st + 16512u + (c >> 5) * 512u + (c & 31u) * 2u); }
    // x: first byte in bits 0-7, second in bits 8-15 (both inside the
    // window); higher bits are ignored.  y = i + 256 j, y >> 7 = 2 j.
    __device__ __forceinline__ void step2(uint32_t x) {
        const uint32_t y = x & 0x1F1Fu;
        st = next(st + 2u * (y + (y >> 7)));
    }
    // both pairs of a word w (all four bytes inside the window): (b0, b1)
    // then (b2, b3).  With z = w & 0x1F1F1F1F, z << 1 holds 2 b0 + 512 b1 in
    // its low half and 2 b2 + 512 b3 in its high half, and
    // (z >> 6) & 0x007C007C adds 4 b1 and 4 b3 (the rows' pads): the two
    // offsets 2 i + 516 j of step2, from one word.
    __device__ __forceinline__ void step4(uint32_t w) {
        const uint32_t z = w & 0x1F1F1F1Fu;
        const uint32_t u = (z << 1) + ((z >> 6) & 0x007C007Cu);
        st = next(st + (u & 0xFFFFu));
        st = next(st + (u >> 16));
    }
    __device__ __forceinline__ uint32_t out_of_window(uint32_t w) const { return (w ^ win) & 0xE0E0E0E0u; }
    __device__ __forceinline__ bool dead() const { return st == base; }
    __device__ __forceinline__ uint32_t state_id() const {
        const uint32_t o = st - base, p = o / PLANE;
        return p * 8u + ((o - p * PLANE) >> 6);
    }
    __device__ __forceinline__ bool accept() const { return lds8(acc + state_id()) != 0; }
    __device__ __forceinline__ void kill() { st = base; }
    __device__ __forceinline__ void set_state(uint32_t s) { st = base + (s >> 3) * PLANE + (s & 7u) * 64u; }
};
using MemoPairP = MemoPairT<false>;
using MemoPairA = MemoPairT<true>;

// The search cache (the start set added back after every byte): rows of
// 256 successors as shared addresses, like MemoS.  Accepting states have the
// highest ids, so the test is one compare of the state's address.
struct SearchS {
    uint32_t st, base, thr;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) { return (size_t)t.srch_K * 1024; }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        const uint32_t b = smem_addr(sm);
        uint32_t* T = reinterpret_cast<uint32_t*>(sm);
        for (int i = threadIdx.x; i < t.srch_K * 256; i += blockDim.x) T[i] = b + t.srch_T[i] * 4u;
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        base = smem_addr(sm);
        st = base + t.srch_start * 4u;
        thr = base + (uint32_t)t.srch_acc0 * 1024u;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = lds32(st + c * 4u); }
    __device__ __forceinline__ bool accepted() const { return st >= thr; }
    __device__ __forceinline__ uint32_t state_id() const { return (st - base) >> 10; }
    __device__ __forceinline__ void set_state(uint32_t s) { st = base + s * 1024u; }
};

// register bitset (one word): desc[c] = {shift | mask << 8, shared address
// of the byte's subset table}; entry x of that table is the new set.
struct Thread1S {
    uint32_t F, nb, desc;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return 256 * 8 + align16((size_t)t.gl_words * 4);
    }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        uint32_t tt = smem_addr(sm) + 256 * 8;
        uint2* d = reinterpret_cast<uint2*>(sm);
        for (int c = threadIdx.x; c < 256; c += blockDim.x) {
            uint2 x = t.gl_desc[c];
            d[c] = make_uint2((x.x & 31u) | (x.x & 0xff00u), tt + x.y * 4u);
        }
        copy_to_smem(sm + 256 * 8, t.gl_tt, (size_t)t.gl_words * 4);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        desc = smem_addr(sm);
        F = t.start[0];
        nb = t.null_bit;
    }
    __device__ __forceinline__ void step(uint32_t c) {
        uint2 d = lds64(desc + c * 8u);
        uint32_t x = (F >> (d.x & 31u)) & (d.x >> 8);
        F = lds32(d.y + x * 4u);
    }
    __device__ __forceinline__ bool dead() const { return F == 0; }
    __device__ __forceinline__ bool accept() const { return (F >> nb) & 1u; }
    __device__ __forceinline__ void kill() { F = 0; }
};

struct Thread2S {
    uint32_t F0, F1, nb, desc;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) {
        return 256 * 8 + align16((size_t)t.gl_words * 4);
    }
    __device__ static void load(const DevTables& t, uint8_t* sm) {
        uint32_t tt = smem_addr(sm) + 256 * 8;
        uint2* d = reinterpret_cast<uint2*>(sm);
        for (int c = threadIdx.x; c < 256; c += blockDim.x) {
            uint2 x = t.gl_desc[c];
            d[c] = make_uint2(x.x, tt + x.y * 4u);
        }
        copy_to_smem(sm + 256 * 8, t.gl_tt, (size_t)t.gl_words * 4);
    }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        desc = smem_addr(sm);
        F0 = t.start[0];
        F1 = t.start[1];
        nb = t.null_bit;
    }
    __device__ __forceinline__ void step(uint32_t c) {
        uint2 d = lds64(desc + c * 8u);
        uint32_t w = (d.x & 32u) ? F1 : F0;
        uint32_t x = (w >> (d.x & 31u)) & (d.x >> 8);
        uint2 e = lds64(d.y + x * 8u);
        F0 = e.x;
        F1 = e.y;
    }
    __device__ __forceinline__ bool dead() const { return (F0 | F1) == 0; }
    __device__ __forceinline__ bool accept() const { return (((nb < 32) ? F0 : F1) >> (nb & 31)) & 1u; }
    __device__ __forceinline__ void kill() { F0 = F1 = 0; }
};

}  // namespace dev
}  // namespace rx

namespace rx {
namespace dev {

// ---------------------------------------------------------------------------
// One string per lane, [s, e) absolute addresses; warp-synchronous (every
// lane of the warp must call it).  The lane walks aligned 16-byte blocks
// with one block of prefetch; blocks whole for every lane take an unrolled
// path, boundary blocks a predicated one.  A lane whose string ends or whose
// set empties writes *outp and then holds the empty set, which every step
// keeps empty.
template <class S>
__device__ __forceinline__ void run_lane(S& st, uint64_t s, uint64_t e, bool valid, uint8_t* outp) {
    bool active = valid && s < e;
    if (valid && !active) *outp = st.accept();
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
            *outp = st.accept();
            st.kill();
            active = false;
        }
    }
}

// ---------------------------------------------------------------------------
// Chunked transfer functions on cache states for one long string per warp
// (the batched form's long pairs, the serving tick's long requests).
static_assert(kMemoMaxStates <= 256, "chunk maps hold cache state ids in one byte");

// Readers of the cache with one-byte entries (K rows of 256 successor
// ids): in global memory (L1/L2) or copied into shared memory.  Both also
// carry the column images (DevTables::memo_img) from global memory.
struct GlobalT8 {
    const uint8_t* __restrict__ T;
    const uint16_t* __restrict__ img_off;
    const uint8_t* __restrict__ img;
    const uint8_t* __restrict__ imgpos;  // DevTables::memo_imgpos
    int K;
    __device__ __forceinline__ uint32_t next(uint32_t x, uint32_t c) const { return __ldg(T + x * 256u + c); }
};

// The wide tier (DevTables::wide_T): the same with two-byte state ids.
struct GlobalT16 {
    const uint16_t* __restrict__ T;
    const uint32_t* __restrict__ img_off;
    const uint16_t* __restrict__ img;
    const uint16_t* __restrict__ imgpos;  // DevTables::wide_imgpos
    int K;
    __device__ __forceinline__ uint32_t next(uint32_t x, uint32_t c) const { return __ldg(T + x * 256u + c); }
};

// one lane, bytes [s, e) (absolute addresses), from cache state id x;
// returns the state id reached; stops when the set is empty (state 0).
// The next 16-byte block is loaded while the current one is stepped.
template <class R>
__device__ inline uint32_t run_t8(const R& rd, uint32_t x, uint64_t s, uint64_t e) {
    uint64_t blk = s & ~uint64_t(15);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (blk < e && x != 0) v = ld_stream(reinterpret_cast<const uint8_t*>(blk));
    while (blk < e && x != 0) {
        const uint64_t nb = blk + 16;
        uint4 vn = make_uint4(0, 0, 0, 0);
        if (nb < e) vn = ld_stream(reinterpret_cast<const uint8_t*>(nb));
        if (blk >= s && nb <= e) {
#pragma unroll
            for (int k = 0; k < 16; k++) x = rd.next(x, byte_of(v, k));
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const uint64_t q = blk + k;
                if (q >= s && q < e) x = rd.next(x, byte_of(v, k));
            }
        }
        blk = nb;
        v = vn;
    }
    return x;
}

// M states x[0..M) (0 = unused or empty) over bytes [s, e) together: their
// lookup chains are independent, so their loads overlap.  After every
// 16-byte block a state equal to an earlier one is dropped (a macro step is
// a function of the state, Def 5.2: the two stay equal) and at the end
// takes that one's result.  Returns the states reached in x.
template <int M, class R>
__device__ inline void run_t8_multi(const R& rd, uint32_t (&x)[M], uint64_t s, uint64_t e) {
    static_assert(M >= 2 && M <= 4, "two to four states");
    uint32_t link = 0;  // per state m: bit 8 + m set if it met state (link >> 2m) & 3
    auto any_live = [&]() {
        uint32_t o = 0;
#pragma unroll
        for (int m = 0; m < M; m++) o |= x[m];
        return o != 0;
    };
    uint64_t blk = s & ~uint64_t(15);
    uint4 v = make_uint4(0, 0, 0, 0);
    bool any = any_live();
    if (blk < e && any) v = ld_stream(reinterpret_cast<const uint8_t*>(blk));
    while (blk < e && any) {
        const uint64_t nb = blk + 16;
        uint4 vn = make_uint4(0, 0, 0, 0);
        if (nb < e) vn = ld_stream(reinterpret_cast<const uint8_t*>(nb));
        const bool whole = blk >= s && nb <= e;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const uint64_t q = blk + k;
            if (whole || (q >= s && q < e)) {
                const uint32_t c = byte_of(v, k);
#pragma unroll
                for (int m = 0; m < M; m++)
                    if (x[m]) x[m] = rd.next(x[m], c);
            }
        }
#pragma unroll
        for (int m = 1; m < M; m++) {
#pragma unroll
            for (int p = 0; p < m; p++)
                if (x[m] && x[m] == x[p]) {
                    link |= ((uint32_t)p << (2 * m)) | (1u << (8 + m));
                    x[m] = 0;
                }
        }
        any = any_live();
        blk = nb;
        v = vn;
    }
#pragma unroll
    for (int m = 1; m < M; m++)
        if (link & (1u << (8 + m))) {
            const uint32_t p = (link >> (2 * m)) & 3u;
#pragma unroll
            for (int q = 0; q < m; q++)
                if (q == (int)p) x[m] = x[q];
        }
}

constexpr int kMulti = 4;  // distinct states of a chunk's rest stepped together

constexpr int kPairPrefix = 128;  // bytes of a chunk in which incoming states are merged

// One lane computes the transfer function of bytes [cs, ce) (absolute
// addresses) on cache states, as a row of Id (the cache's state id type):
//   row[0] = the chunk's first byte c, row[1] = n = the size of the image
//   of column c (the distinct states any incoming state reaches on c),
//   row[2 + i] = the state reached from image entry i over the rest.
// An incoming state k then ends in row[2 + i] with img[i] = T[k][c] (exact:
// a macro step is a function of the set, Def 5.2, so k's path after c is
// that of T[k][c]).  The image is usually a few states, so no incoming
// state is stepped on its own.  They advance in stages of 3, 6, 12, ...
// bytes (at most kPairPrefix bytes in all) while at least two distinct live
// states are among them -- the empty set (state 0, always entry 0) stays
// empty at no cost, and two states that meet stay together -- and each
// distinct one then runs over the rest.  row holds 2 + n entries; n = 0
// marks an empty chunk (the identity).  An incoming state k maps to
// row[2 + imgpos[c*K + k]].  The rest of the chunk steps the first kMulti
// distinct states together (run_t8_multi) in a loop picked by the warp's
// largest count, so all 32 lanes of the warp must call this together.
template <class R, class Id>
__device__ inline void chunk_fn(const R& rd, uint64_t cs, uint64_t ce, Id* row) {
    const bool empty = ce <= cs;
    if (empty) row[1] = 0;
    const uint32_t c = empty ? 0u : __ldg(reinterpret_cast<const uint8_t*>(cs));
    const int lo = empty ? 0 : (int)rd.img_off[c], n = empty ? 0 : (int)rd.img_off[c + 1] - lo;
    Id* dv = row + 2;
    if (!empty) {
        row[0] = (Id)c;
        row[1] = (Id)n;
    }
    for (int i = 0; i < n; i++) dv[i] = rd.img[lo + i];
    const uint64_t pe = cs + kPairPrefix < ce ? cs + kPairPrefix : ce;
    uint64_t pos = cs + 1;
    bool several = n > 2;  // entry 0 is the empty set
    uint64_t len = 3;
    while (several && pos < pe) {
        const uint64_t end = pos + len < pe ? pos + len : pe;
        uint32_t first = 0;
        several = false;
        for (int i = 0; i < n; i++) {
            const uint32_t v = run_t8(rd, (uint32_t)dv[i], pos, end);
            dv[i] = (Id)v;
            if (v != 0) {
                if (first == 0) first = v;
                else if (v != first) several = true;
            }
        }
        pos = end;
        len *= 2;
    }
    // the rest of the chunk: the first kMulti distinct live states together
    // (run_t8_multi), any further one on its own (a repeat beyond the first
    // kMulti is run again, same result)
    uint32_t cv[kMulti], cr[kMulti];
    int nc = 0;
    for (int i = 0; i < n && nc < kMulti; i++) {
        const uint32_t v = dv[i];
        bool seen = v == 0;
#pragma unroll
        for (int q = 0; q < kMulti; q++)
            if (q < nc && cv[q] == v) seen = true;
        if (!seen) {
#pragma unroll
            for (int q = 0; q < kMulti; q++)
                if (q == nc) cv[q] = v;
            nc++;
        }
    }
#pragma unroll
    for (int q = 0; q < kMulti; q++) cr[q] = q < nc ? cv[q] : 0u;
    const int most = __reduce_max_sync(FULL, (unsigned)nc);  // warp-uniform
    if (most <= 1) {
        cr[0] = cr[0] ? run_t8(rd, cr[0], pos, ce) : 0u;
    } else if (most == 2) {
        uint32_t x2[2] = {cr[0], cr[1]};
        run_t8_multi<2>(rd, x2, pos, ce);
        cr[0] = x2[0];
        cr[1] = x2[1];
    } else {
        run_t8_multi<4>(rd, cr, pos, ce);
    }
    for (int i = 0; i < n; i++) {
        const uint32_t v = dv[i];
        uint32_t r = 0xffffffffu;
#pragma unroll
        for (int q = 0; q < kMulti; q++)
            if (q < nc && cv[q] == v) r = cr[q];
        if (r == 0xffffffffu) r = v == 0 ? 0u : run_t8(rd, v, pos, ce);
        dv[i] = (Id)r;
    }
}

// The state a chunk's row (chunk_fn) leads state x to: the row's entry for
// x's position in the image of the chunk's first byte.
template <class R, class Id>
__device__ __forceinline__ uint32_t chunk_apply(const R& rd, const Id* row, uint32_t x) {
    if (row[1] == 0) return x;
    return row[2 + __ldg(rd.imgpos + (uint32_t)row[0] * rd.K + x)];
}

// One warp advances the cache state x0 over bytes [s, e) (absolute
// addresses) and returns the state reached (the same in every lane).  rd
// reads the cache rows.  Lane l computes the transfer function of chunk l
// (of 32) with chunk_fn into row l of wsm (`stride` bytes each, at least
// (2 + the largest column image) ids); lane 0 applies the 32 rows to x0 in
// order (the rows were just written by this warp, so the chain mostly hits
// L1).
template <class R, class Id>
__device__ inline uint32_t warp_chunked(const R& rd, uint32_t x0, uint64_t s, uint64_t e, uint8_t* wsm, int stride) {
    const int lane = threadIdx.x & 31;
    const uint64_t L = e - s;
    const uint64_t C = ((L + 31) / 32 + 15) & ~uint64_t(15);
    uint64_t cs = s + (uint64_t)lane * C;
    if (cs > e) cs = e;
    const uint64_t ce = cs + C < e ? cs + C : e;
    chunk_fn<R, Id>(rd, cs, ce, reinterpret_cast<Id*>(wsm + lane * stride));
    __syncwarp();
    uint32_t x = x0;
    if (lane == 0)
        for (int l = 0; l < 32; l++) x = chunk_apply<R, Id>(rd, reinterpret_cast<const Id*>(wsm + l * stride), x);
    __syncwarp();
    return __shfl_sync(FULL, x, 0);
}

// the same with the rows in global memory (the batched and serving forms)
__device__ inline uint32_t warp_chunked_memo(const DevTables& t, uint32_t x0, uint64_t s, uint64_t e, uint8_t* wsm,
                                             int stride) {
    return warp_chunked<GlobalT8, uint8_t>(GlobalT8{t.memo_T8, t.memo_img_off, t.memo_img, t.memo_imgpos, t.memo_K},
                                           x0, s, e, wsm, stride);
}

// the wide tier (two-byte ids; rows of 2 + wide_maximg ids)
__device__ inline uint32_t warp_chunked_wide(const DevTables& t, uint32_t x0, uint64_t s, uint64_t e, uint8_t* wsm,
                                             int stride) {
    return warp_chunked<GlobalT16, uint16_t>(
        GlobalT16{t.wide_T, t.wide_img_off, t.wide_img, t.wide_imgpos, t.wide_K}, x0, s, e, wsm, stride);
}

// ---------------------------------------------------------------------------
// One string per warp: lane l owns words l, l+32, ... (K per lane) of the
// active set.  A step ANDs with B[c], then ORs the follow row of every
// active bit, found with ballot / shuffle so the loop is warp-uniform.  The
// warp stages 512 input bytes at a time with one 16-byte load per lane.
// Returns whether the string is accepted (same value in every lane).
// warp_span: advance the set F (lane-owned words) over [s, e); returns true
// if the set emptied (the string is stuck), in which case F is all zero.
template <int K>
__device__ bool warp_span(const DevTables& t, const uint32_t* B, const uint32_t* follow, uint64_t s, uint64_t e,
                          uint32_t (&F)[K]) {
    const int W = t.W;
    const int lane = threadIdx.x & 31;
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
    return dead;
}

// null bit of the lane-owned set (same value in every lane)
template <int K>
__device__ __forceinline__ bool warp_accepts(const DevTables& t, const uint32_t (&F)[K]) {
    const int nbw = t.null_bit >> 5, nbb = t.null_bit & 31;
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < K; k++)
        if (k == (nbw >> 5)) mine = F[k];
    uint32_t nw = __shfl_sync(FULL, mine, nbw & 31);
    return (nw >> nbb) & 1u;
}

template <int K>
__device__ bool warp_string(const DevTables& t, const uint32_t* B, const uint32_t* follow, uint64_t s, uint64_t e) {
    const int lane = threadIdx.x & 31;
    uint32_t F[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        int w = k * 32 + lane;
        F[k] = (w < t.W) ? t.start[w] : 0u;
    }
    bool dead = warp_span<K>(t, B, follow, s, e, F);
    return !dead && warp_accepts<K>(t, F);
}

// Advance one lane's set over [s, e) (absolute addresses), warp-
// synchronously; lanes with active == false only keep step with the others.
// Stops reading once the set is empty.
template <class S>
__device__ __forceinline__ void run_lane_span(S& st, uint64_t s, uint64_t e, bool active) {
    active = active && s < e;
    uint64_t blk = s & ~uint64_t(15);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (active) v = ld_stream(reinterpret_cast<const uint8_t*>(blk));
    while (__any_sync(FULL, active)) {
        uint64_t nb = blk + 16;
        uint4 vn = make_uint4(0, 0, 0, 0);
        if (active && nb < e) vn = ld_stream(reinterpret_cast<const uint8_t*>(nb));
#pragma unroll
        for (int k = 0; k < 16; k++) {
            S nx = st;
            nx.step(byte_of(v, k));
            bool ok = active && blk + k >= s && blk + k < e;
            if (ok) st = nx;
        }
        blk = nb;
        v = vn;
        if (active && (blk >= e || st.dead())) active = false;
    }
}

}  // namespace dev
}  // namespace rx
