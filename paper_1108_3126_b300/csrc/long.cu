// long.cu -- exact chunked matching of one long string (rx_match_long).
//
// A macro step maps a set of pointers to the union of the images of its
// elements: Defs 5.1 and 5.2 (Rathnayake & Thielecke, SOS 2011) quantify
// "exists p in S".  So the effect of a whole chunk of input on any incoming
// set is fixed by its effect on single elements, and chunks can be
// processed in parallel and composed afterwards:
//
//   memo form    incoming state s of the cache (state 0 = empty set):
//                map_j[s] = state after chunk j starting from s
//   bitset form  incoming set {b} for each bit b (position or null):
//                row_j[b] = set after chunk j starting from {b};
//                tau_j(X) = U_{b in X} row_j[b]
//
// Composition runs left to right in blocks of G functions held in shared
// memory, level after level, until one function remains; it is applied to
// the evolution of {root} and the null bit (or the accepting flag of the
// final cache state) is the answer.
#include <algorithm>

#include "kernels.cuh"
#include "steppers.cuh"

namespace rx {

namespace {

using namespace rx::dev;

// Phase 1: one thread per chunk.  After the chunk's first byte c every
// incoming cache state is in the image of column c (the distinct
// successors on c, usually a few states; DevTables::memo_img), so those
// states are the chunk's representatives and no incoming state is stepped
// on its own.  The representatives advance in stages (3, 4, 8, 16, ...
// bytes, kMaxPrefix in all) until at most one distinct live state is among
// them (the empty set, state 0, stays empty at no cost) -- two states that
// meet stay together, since a macro step is a function of the set (Def
// 5.2).  Each distinct live state left needs the rest of the chunk (phase
// 2); its result slot is toff[j] + its rank among them.  Phase 2 tasks take
// them in pairs (ranks 2m, 2m + 1: one lane steps both, and drops the
// second once they meet) and an odd last one alone; pair tasks are stored
// from index pair_base, one-state tasks from 0.  The slots and tasks of a
// warp's 32 chunks are allotted with one scan and three atomic adds (ctr[0]
// slots, ctr[2] pair tasks, ctr[3] one-state tasks).  Per chunk j: cb0[j] =
// c; slot[j*K + i] = result slot (relative to toff[j]) of the state image
// entry i has reached, 0xFFFF if it is the empty set; toff[j] = first slot;
// pstart[j] = prefix bytes consumed.  An incoming state k is then mapped through entry
// memo_imgpos[c*K + k].  The prefix is kept short because a warp's 32 chunks
// go through it together.  Each thread keeps dv[K] (the representatives'
// states) and rk[K] (task number of a state id) as bytes in shared memory
// after the table, interleaved across the block's threads (entry k of
// thread x at k * blockDim + x) so that a warp's accesses fall in distinct
// banks.
// The kernel is held to 48 registers (five 256-thread blocks per SM), so
// the chunks of the automatic chunk size (about 0.8 x 32 per resident warp
// of phase 2) run in one wave of threads.
constexpr int kMaxPrefix = 128;

// a set of cache state ids (< 192) in six registers
struct IdSet {
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    __device__ __forceinline__ void add(uint32_t v) {
        const uint32_t b = 1u << (v & 31), q = v >> 5;
        w0 |= q == 0 ? b : 0u;
        w1 |= q == 1 ? b : 0u;
        w2 |= q == 2 ? b : 0u;
        w3 |= q == 3 ? b : 0u;
        w4 |= q == 4 ? b : 0u;
        w5 |= q == 5 ? b : 0u;
    }
    __device__ __forceinline__ uint32_t word(int q) const {
        return q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : q == 3 ? w3 : q == 4 ? w4 : w5;
    }
    __device__ __forceinline__ int count() const {
        return __popc(w0) + __popc(w1) + __popc(w2) + __popc(w3) + __popc(w4) + __popc(w5);
    }
};
static_assert(kMemoMaxStates <= 192, "IdSet holds 192 ids");

// The cache of macro steps with one-byte entries in shared memory (a
// quarter of MemoS's rows, so more blocks fit an SM): st = shared address
// of the state's row of 256 successor ids.
struct MemoS8 {
    uint32_t st, base;
    __host__ __device__ static size_t smem_bytes(const DevTables& t) { return align16((size_t)t.memo_K * 256); }
    __device__ static void load(const DevTables& t, uint8_t* sm) { copy_to_smem(sm, t.memo_T8, (size_t)t.memo_K * 256); }
    __device__ void bind(const DevTables& t, uint8_t* sm) {
        base = smem_addr(sm);
        st = base + (t.memo_start >> 8) * 256u;
    }
    __device__ __forceinline__ void step(uint32_t c) { st = base + (lds8(st + c) << 8); }
    __device__ __forceinline__ void set_state(uint32_t s) { st = base + s * 256u; }
    __device__ __forceinline__ uint32_t state_id() const { return (st - base) >> 8; }
};

// N macro steps over the bytes packed in b (byte q at bits 8*(q%4) of b[q/4])
template <int N, class S>
__device__ __forceinline__ void step_bytes(S& st, const uint32_t (&b)[4]) {
#pragma unroll
    for (int q = 0; q < N; q++) st.step((b[q >> 2] >> (8 * (q & 3))) & 0xffu);
}

// the state reached from `s` over the n (<= 16) bytes packed in b
template <class S>
__device__ __forceinline__ uint32_t step_n(const S& proto, uint32_t s, const uint32_t (&b)[4], int n) {
    S st = proto;
    st.set_state(s);
    if (n == 4) {
        step_bytes<4>(st, b);
    } else if (n == 8) {
        step_bytes<8>(st, b);
    } else if (n == 16) {
        step_bytes<16>(st, b);
    } else {
#pragma unroll
        for (int q = 0; q < 16; q++)
            if (q < n) st.step((b[q >> 2] >> (8 * (q & 3))) & 0xffu);
    }
    return st.state_id();
}

// the next n (<= 16) bytes at p, packed
__device__ __forceinline__ void load_bytes(const uint8_t* p, int n, uint32_t (&b)[4]) {
    b[0] = b[1] = b[2] = b[3] = 0u;
#pragma unroll
    for (int i = 0; i < 16; i++)
        if (i < n) b[i >> 2] |= (uint32_t)__ldg(p + i) << (8 * (i & 3));
}

__global__ void __launch_bounds__(256, 5) k_chunk_stage(const DevTables t, const uint8_t* __restrict__ str, int64_t len,
                                                     int64_t C, long long J, uint16_t* __restrict__ slot,
                                                     uint8_t* __restrict__ cb0, uint16_t* __restrict__ pstart,
                                                     unsigned* __restrict__ toff, uint32_t* __restrict__ task_chunk,
                                                     uint16_t* __restrict__ task_state,
                                                     uint32_t* __restrict__ task_res, long long pair_base,
                                                     unsigned* __restrict__ ctr) {
    extern __shared__ __align__(16) uint8_t smem[];
    MemoS8::load(t, smem);
    __syncthreads();
    MemoS8 proto;
    proto.bind(t, smem);
    const int K = t.memo_K;
    const int nt = blockDim.x, lane = threadIdx.x & 31;
    uint8_t* dv = smem + MemoS8::smem_bytes(t) + threadIdx.x;
    uint8_t* rk = dv + (size_t)K * nt;
    // warp-uniform loop over groups of 32 chunks
    const long long wstride = (long long)gridDim.x * blockDim.x;
    for (long long j0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < J; j0 += wstride) {
        const long long j = j0 + lane;
        const bool valid = j < J;
        int nr = 0, nl = 0;
        int64_t cs = 0, pos = 0;
        uint32_t c0 = 0;
        IdSet fin;  // the distinct live states at the end of the prefix
        if (valid) {
            cs = j * C;
            const int64_t pe = min(cs + kMaxPrefix, min(cs + C, len));
            // the image of the first byte's column: the representatives
            c0 = __ldg(str + cs);
            const int lo = t.memo_img_off[c0];
            nr = (int)t.memo_img_off[c0 + 1] - lo;
            for (int i = 0; i < nr; i++) {
                const uint32_t v = t.memo_img[lo + i];
                dv[i * nt] = (uint8_t)v;
                fin.add(v);
            }
            pos = cs + 1;
            int live = nr - 1;  // entry 0 is the empty set
            int L = 3, stage = 0;
            uint32_t b[4];
            // further stages: the representatives only
            while (live > 1 && pos < pe) {
                const int n = (int)min((int64_t)L, pe - pos);
                load_bytes(str + pos, n, b);
                IdSet s2;
                for (int i = 0; i < nr; i++) {
                    const uint32_t v = step_n(proto, dv[i * nt], b, n);
                    dv[i * nt] = (uint8_t)v;
                    s2.add(v);
                }
                fin = s2;
                live = s2.count() - (int)(s2.w0 & 1u);
                pos += n;
                stage++;
                L = stage < 2 ? 4 : (stage == 2 ? 8 : 16);
            }
            // tasks: the distinct live states, numbered in id order
#pragma unroll
            for (int w = 0; w < 6; w++) {
                uint32_t x = fin.word(w) & (w == 0 ? ~1u : ~0u);
                while (x) {
                    const int id = w * 32 + __ffs(x) - 1;
                    rk[id * nt] = (uint8_t)nl;
                    nl++;
                    x &= x - 1;
                }
            }
        }
        // slots and tasks of the warp's chunks: one scan of the three counts
        // packed (slots <= 32 * 192 in bits 0-12, pair tasks <= 32 * 96 in
        // bits 13-24, one-state tasks <= 32 in bits 25-30)
        const unsigned mine = (unsigned)nl | ((unsigned)(nl >> 1) << 13) | ((unsigned)(nl & 1) << 25);
        unsigned incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned x = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += x;
        }
        unsigned b_slot = 0, b_pair = 0, b_one = 0;
        if (lane == 31) {
            b_slot = atomicAdd(ctr, incl & 0x1FFFu);
            b_pair = atomicAdd(ctr + 2, (incl >> 13) & 0xFFFu);
            b_one = atomicAdd(ctr + 3, incl >> 25);
        }
        const unsigned excl = incl - mine;
        const unsigned base = __shfl_sync(FULL, b_slot, 31) + (excl & 0x1FFFu);
        const unsigned pbase = __shfl_sync(FULL, b_pair, 31) + ((excl >> 13) & 0xFFFu);
        const unsigned obase = __shfl_sync(FULL, b_one, 31) + (excl >> 25);
        if (valid) {
            for (int i = 0; i < nr; i++) {
                const uint32_t v = dv[i * nt];
                slot[j * K + i] = v == 0 ? (uint16_t)0xFFFF : (uint16_t)rk[v * nt];
            }
            cb0[j] = (uint8_t)c0;
            int i = 0;
            uint32_t first = 0;  // the first state of the pending pair
#pragma unroll
            for (int w = 0; w < 6; w++) {
                uint32_t x = fin.word(w) & (w == 0 ? ~1u : ~0u);
                while (x) {
                    const uint32_t id = (uint32_t)(w * 32 + __ffs(x) - 1);
                    if (i & 1) {
                        const long long tk = pair_base + pbase + (i >> 1);
                        task_chunk[tk] = (uint32_t)j;
                        task_state[tk] = (uint16_t)(first | (id << 8));
                        task_res[tk] = base + (unsigned)i - 1u;
                    } else {
                        first = id;
                    }
                    i++;
                    x &= x - 1;
                }
            }
            if (nl & 1) {
                task_chunk[obase] = (uint32_t)j;
                task_state[obase] = (uint16_t)first;
                task_res[obase] = base + (unsigned)nl - 1u;
            }
            toff[j] = base;
            pstart[j] = (uint16_t)(pos - cs);
        }
    }
}

// first level of the composition, reading the chunk maps straight from the
// tasks' results: map_j[k] = res[toff[j] + slot[j*K + i]] with i =
// memo_imgpos[cb0[j]*K + k] (0 for the empty set); block b composes chunks
// [b*G, min((b+1)*G, J)) into out[b]
// Maps m[0..nmap) of K entries in shared memory, m[0] applied first: leaves
// their composition in m[0].  Pairwise in log2(nmap) levels: at stride d,
// m[j] <- m[j + d] o m[j] for j a multiple of 2d (composition is
// associative, so this bracketing gives the left-to-right result).
__device__ void compose_tree(uint16_t* m, int nmap, int K) {
    for (int d = 1; d < nmap; d *= 2) {
        const int pairs = (nmap - d + 2 * d - 1) / (2 * d);  // j = 0, 2d, ... with j + d < nmap
        for (int i = threadIdx.x; i < pairs * K; i += blockDim.x) {
            const int j = (i / K) * 2 * d, k = i % K;
            m[j * K + k] = m[(j + d) * K + m[j * K + k]];
        }
        __syncthreads();
    }
}

__global__ void k_compose_first(const uint16_t* __restrict__ slot, const uint8_t* __restrict__ cb0,
                                const uint8_t* __restrict__ imgpos, const unsigned* __restrict__ toff,
                                const uint16_t* __restrict__ res, long long J, int K, int G,
                                uint16_t* __restrict__ out) {
    extern __shared__ __align__(16) uint16_t sm16[];
    const long long lo = (long long)blockIdx.x * G;
    const long long hi = std::min<long long>(lo + G, J);
    const int nmap = (int)(hi - lo);
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int c = threadIdx.x >> 5; c < nmap; c += warps) {
        const unsigned o = toff[lo + c];
        const uint32_t b0 = cb0[lo + c];
        for (int k = lane; k < K; k += 32) {
            const uint16_t r = slot[(lo + c) * K + __ldg(imgpos + b0 * K + k)];
            sm16[c * K + k] = r == 0xFFFF ? (uint16_t)0 : res[o + r];
        }
    }
    __syncthreads();
    // one thread per incoming state walks the maps in order (the gather
    // above dominates; a pairwise tree here was slower)
    for (int s = threadIdx.x; s < K; s += blockDim.x) {
        int x = s;
        for (int j = 0; j < nmap; j++) x = sm16[j * K + x];
        out[(long long)blockIdx.x * K + s] = (uint16_t)x;
    }
}

// level of the composition: block b composes maps [b*G, min((b+1)*G, cnt))
__global__ void k_compose_maps(const uint16_t* __restrict__ in, long long cnt, int K, int G,
                               uint16_t* __restrict__ out) {
    extern __shared__ __align__(16) uint16_t sm16[];
    long long lo = (long long)blockIdx.x * G;
    long long hi = std::min<long long>(lo + G, cnt);
    int nmap = (int)(hi - lo);
    for (int i = threadIdx.x; i < nmap * K; i += blockDim.x) sm16[i] = in[lo * K + i];
    __syncthreads();
    compose_tree(sm16, nmap, K);
    for (int s = threadIdx.x; s < K; s += blockDim.x) out[(long long)blockIdx.x * K + s] = sm16[s];
}

__global__ void k_finish_memo(const DevTables t, const uint16_t* __restrict__ map, int has_map, uint8_t* out) {
    // has_map == 0: the empty text, accepted iff the start state holds null
    if (threadIdx.x != 0) return;
    uint32_t s = t.memo_start >> 8;
    if (has_map) s = map[s];
    out[0] = t.memo_acc[s];
}

// one warp per (chunk, group of 32 incoming bits); lanes = incoming bits
template <class S>
__global__ void __launch_bounds__(256) k_chunk_rows(const DevTables t, const uint8_t* __restrict__ str, int64_t len,
                                                    int64_t C, long long J, int groups, uint32_t* __restrict__ rows) {
    extern __shared__ __align__(16) uint8_t smem[];
    S::load(t, smem);
    __syncthreads();
    S proto;
    proto.bind(t, smem);
    const int lane = threadIdx.x & 31;
    const int nbits = t.nbits;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    for (long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < J * groups;
         task += warps) {
        long long j = task / groups;
        int b = (int)(task % groups) * 32 + lane;
        S st = proto;
        if (b < nbits) st.set_unit(b);
        else st.kill();
        uint64_t s = base + (uint64_t)(j * C), e = base + (uint64_t)std::min<int64_t>((j + 1) * C, len);
        run_range_uniform(st, s, e);
        if (b < nbits) st.store(rows + ((size_t)j * nbits + b) * S::ROW_WORDS);
    }
}

// level of the composition of row matrices (RW words per row, nbits rows)
template <int RW>
__global__ void k_compose_rows(const uint32_t* __restrict__ in, long long cnt, int nbits, int G,
                               uint32_t* __restrict__ out) {
    extern __shared__ __align__(16) uint32_t sm32[];
    long long lo = (long long)blockIdx.x * G;
    long long hi = std::min<long long>(lo + G, cnt);
    int nmat = (int)(hi - lo);
    const size_t mat = (size_t)nbits * RW;
    for (size_t i = threadIdx.x; i < (size_t)nmat * mat; i += blockDim.x) sm32[i] = in[lo * mat + i];
    __syncthreads();
    for (int b = threadIdx.x; b < nbits; b += blockDim.x) {
        uint32_t x[RW];
#pragma unroll
        for (int k = 0; k < RW; k++) x[k] = (k == (b >> 5)) ? (1u << (b & 31)) : 0u;
        for (int j = 0; j < nmat; j++) {
            uint32_t y[RW];
#pragma unroll
            for (int k = 0; k < RW; k++) y[k] = 0;
            const uint32_t* M = sm32 + (size_t)j * mat;
#pragma unroll
            for (int w = 0; w < RW; w++) {
                uint32_t bits = x[w];
                while (bits) {
                    int q = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
#pragma unroll
                    for (int k = 0; k < RW; k++) y[k] |= M[(size_t)q * RW + k];
                }
            }
#pragma unroll
            for (int k = 0; k < RW; k++) x[k] = y[k];
        }
#pragma unroll
        for (int k = 0; k < RW; k++) out[(long long)blockIdx.x * mat + (size_t)b * RW + k] = x[k];
    }
}

template <int RW>
__global__ void k_finish_rows(const DevTables t, const uint32_t* __restrict__ M, int has_map, uint8_t* out) {
    if (threadIdx.x != 0) return;
    uint32_t F[RW];
#pragma unroll
    for (int k = 0; k < RW; k++) F[k] = (k < t.W) ? t.start[k] : 0u;
    if (has_map) {
        uint32_t y[RW];
#pragma unroll
        for (int k = 0; k < RW; k++) y[k] = 0;
        for (int w = 0; w < RW; w++) {
            uint32_t bits = F[w];
            while (bits) {
                int q = w * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                if (q >= t.nbits) continue;
                for (int k = 0; k < RW; k++) y[k] |= M[(size_t)q * RW + k];
            }
        }
#pragma unroll
        for (int k = 0; k < RW; k++) F[k] = y[k];
    }
    int nb = t.null_bit;
    uint32_t wv = 0;
#pragma unroll
    for (int k = 0; k < RW; k++)
        if (k == (nb >> 5)) wv = F[k];
    out[0] = (wv >> (nb & 31)) & 1u;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// pick the stepper used for bitset rows; 0 = none
int rows_kind(const DevTables& t) {
    if (t.gl_words > 0) return t.W == 1 ? 1 : 2;
    if (t.sp_W == 4) return 4;
    if (t.sp_W == 8) return 8;
    return 0;
}

template <class S>
cudaError_t launch_chunk_rows(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, long long J,
                              uint32_t* rows, cudaStream_t st) {
    int groups = (t.nbits + 31) / 32;
    size_t sm = S::smem_bytes(t);
    auto kern = k_chunk_rows<S>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
    if (e != cudaSuccess) return e;
    long long need = (J * groups + 7) / 8;
    long long grid = std::min<long long>(need, (long long)std::max(per_sm, 1) * sm_count());
    {
        ProfScope ps(st);
        kern<<<(unsigned)std::max<long long>(grid, 1), 256, sm, st>>>(t, str, len, C, J, groups, rows);
    }
    return cudaGetLastError();
}

template <int RW>
cudaError_t compose_rows(const DevTables& t, uint32_t* a, uint32_t* b, long long J, uint8_t* out, cudaStream_t st) {
    const size_t mat = (size_t)t.nbits * RW * 4;
    int G = (int)std::max<size_t>(2, std::min<size_t>(64, (96 * 1024) / std::max<size_t>(mat, 1)));
    cudaError_t e = allow_smem(k_compose_rows<RW>, G * mat);
    if (e != cudaSuccess) return e;
    long long cnt = J;
    uint32_t* cur = a;
    uint32_t* nxt = b;
    while (cnt > 1) {
        long long nb = (cnt + G - 1) / G;
        k_compose_rows<RW><<<(unsigned)nb, 128, G * mat, st>>>(cur, cnt, t.nbits, G, nxt);
        prof_count(1);
        std::swap(cur, nxt);
        cnt = nb;
    }
    k_finish_rows<RW><<<1, 32, 0, st>>>(t, cur, J > 0 ? 1 : 0, out);
    prof_count(1);
    return cudaGetLastError();
}

// ---- chunked mode on the wide cache tier (two-byte state ids)
// The text is cut into segments; a warp takes a segment, computes the
// transfer functions of its 32 chunks on the tier (chunk_fn, rows in shared
// memory) and composes them into one row of the segment in the same image
// form -- first byte c, image size n, and for each image entry i the state
// reached from img[c][i] at the segment's end -- its lanes taking the
// entries.  Rows compose pairwise, (c1, n1, r1) then (c2, n2, r2) =
// (c1, n1, i -> r2[imgpos[c2][r1[i]]]), level by level; the last row is
// applied to the start state.  Exact: chunk functions act on states (Def
// 5.2).  Rows are wide_maximg + 2 entries apart in global memory.
__device__ __forceinline__ uint32_t wide_apply(const DevTables& t, const uint16_t* row, uint32_t x) {
    if (row[1] == 0) return x;
    return row[2 + __ldg(t.wide_imgpos + (uint32_t)row[0] * t.wide_K + x)];
}

constexpr int kWideSegBlock = 256;

__global__ void __launch_bounds__(kWideSegBlock) k_wide_segments(const DevTables t, const uint8_t* __restrict__ str,
                                                                 int64_t len, int64_t seg, long long S,
                                                                 uint16_t* __restrict__ rows, int rs, int stride) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t* wsm = smem + (size_t)(threadIdx.x >> 5) * 32 * stride;
    const int lane = threadIdx.x & 31;
    const GlobalT16 rd{t.wide_T, t.wide_img_off, t.wide_img, t.wide_imgpos, t.wide_K};
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long k = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < S; k += wstride) {
        const int64_t a0 = k * seg < len ? k * seg : len, a1 = (k + 1) * seg < len ? (k + 1) * seg : len;
        const uint64_t s = base + (uint64_t)a0, e = base + (uint64_t)a1;
        const uint64_t L = e - s;
        const uint64_t C = ((L + 31) / 32 + 15) & ~uint64_t(15);
        uint64_t cs = s + (uint64_t)lane * C;
        if (cs > e) cs = e;
        const uint64_t ce = cs + C < e ? cs + C : e;
        chunk_fn<GlobalT16, uint16_t>(rd, cs, ce, reinterpret_cast<uint16_t*>(wsm + lane * stride));
        __syncwarp();
        const uint16_t* r0 = reinterpret_cast<const uint16_t*>(wsm);
        uint16_t* out = rows + (size_t)k * rs;
        const int n0 = r0[1];
        if (lane == 0) {
            out[0] = r0[0];
            out[1] = (uint16_t)n0;
        }
        for (int i = lane; i < n0; i += 32) {
            uint32_t x = r0[2 + i];
            for (int l = 1; l < 32; l++) x = wide_apply(t, reinterpret_cast<const uint16_t*>(wsm + l * stride), x);
            out[2 + i] = (uint16_t)x;
        }
        __syncwarp();
    }
}

// one level: row p of out = row 2p of in, then row 2p + 1 (if any); a warp
// per pair, its lanes over the first row's image entries
__global__ void k_wide_compose(const DevTables t, const uint16_t* __restrict__ in, long long cnt,
                               uint16_t* __restrict__ out, int rs) {
    const int lane = threadIdx.x & 31;
    const long long np = (cnt + 1) / 2;
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long p = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < np; p += wstride) {
        const uint16_t* a = in + (size_t)(2 * p) * rs;
        const uint16_t* b = 2 * p + 1 < cnt ? in + (size_t)(2 * p + 1) * rs : nullptr;
        uint16_t* o = out + (size_t)p * rs;
        const int na = a[1];
        const uint16_t* first = (na == 0 && b) ? b : a;  // an empty first row is the identity
        const uint16_t* second = (na == 0) ? nullptr : b;
        const int n = first[1];
        if (lane == 0) {
            o[0] = first[0];
            o[1] = (uint16_t)n;
        }
        for (int i = lane; i < n; i += 32) {
            const uint32_t x = first[2 + i];
            o[2 + i] = (uint16_t)(second ? wide_apply(t, second, x) : x);
        }
    }
}

__global__ void k_wide_finish(const DevTables t, const uint16_t* __restrict__ row, int has_row, uint8_t* out) {
    if (threadIdx.x == 0) {
        const uint32_t x = has_row ? wide_apply(t, row, t.wide_start) : t.wide_start;
        out[0] = t.wide_acc[x];
    }
}

}  // namespace

// wide tier: a row per segment (two buffers); 32 rows a warp in shared
// memory in the segment kernel
static size_t wide_row_entries(const DevTables& t) { return (size_t)t.wide_maximg + 2; }
static size_t wide_seg_smem(const DevTables& t) {
    const size_t stride = (2 * wide_row_entries(t) + 15) & ~size_t(15);
    return (size_t)(kWideSegBlock / 32) * 32 * stride;
}

int64_t long_chunk_auto(const DevTables& t, int64_t len) {
    if (t.memo_K > 0) {
        // Phase 2 in one wave: every resident warp of the span kernel takes
        // at most one round of 32 tasks, all of one chunk length, so the
        // tasks end together.  Tasks run about one per chunk (pairs of live
        // states share a lane); chunks are sized for up to 1.25 tasks per
        // chunk.  Fewer, longer chunks also cut phase 1 and the composition,
        // whose work grows with the number of chunks.
        const long long warps = std::max<long long>(span_resident_warps(t), 1);
        const long long target = std::max<long long>(warps * 32 * 4 / 5, 1);
        int64_t C = (len + target - 1) / target;
        C = std::max<int64_t>(C, 1024);
        return std::min<int64_t>((C + 31) & ~int64_t(31), (int64_t(1) << 32) - 32);
    }
    if (t.wide_K > 0) {
        // one segment per resident warp of the segment kernel, at least 4 KiB
        // (128 bytes a chunk)
        int per_sm = 0;
        if (allow_smem(k_wide_segments, wide_seg_smem(t)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wide_segments, kWideSegBlock,
                                                          wide_seg_smem(t)) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
        const long long warps = std::max<long long>(1, (long long)per_sm * (kWideSegBlock / 32) * sm_count());
        int64_t C = (len + warps - 1) / warps;
        C = std::max<int64_t>(C, 4096);
        return std::min<int64_t>((C + 31) & ~int64_t(31), (int64_t(1) << 32) - 32);
    }
    int groups = (t.nbits + 31) / 32;
    long long target = (long long)sm_count() * 64 * 8 / std::max(groups, 1);
    int64_t C = (len + target - 1) / std::max<long long>(target, 1);
    C = std::max<int64_t>(C, 4096);
    return (C + 15) & ~int64_t(15);
}

struct MemoLongWs {
    uint16_t *pstart, *slot, *task_state, *res, *maps_a, *maps_b;
    uint8_t* cb0;
    uint32_t *task_chunk, *task_res;
    // ctr[0]: result slots allotted, ctr[1]: work counter of phase 2,
    // ctr[2]: pair tasks, ctr[3]: one-state tasks
    unsigned *toff, *ctr;
};

// phase 2 tasks: at most one one-state task per chunk at [0, J), pair tasks
// (at most K / 2 per chunk) from J on
static long long memo_long_tasks(long long J, int K) { return J + J * (long long)(K / 2); }

static size_t memo_long_layout(long long J, int K, uint8_t* w, MemoLongWs* o) {
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t x = off;
        off += al256(b);
        return w ? w + x : nullptr;
    };
    const size_t JK = (size_t)J * K, NT = (size_t)memo_long_tasks(J, K);
    uint8_t* p_pre = take((size_t)J * 2);
    uint8_t* p_slot = take(JK * 2);
    uint8_t* p_ts = take(NT * 2);
    uint8_t* p_res = take(JK * 2);
    uint8_t* p_ma = take(JK * 2);
    uint8_t* p_mb = take(JK * 2);
    uint8_t* p_tc = take(NT * 4);
    uint8_t* p_tr = take(NT * 4);
    uint8_t* p_toff = take((size_t)J * 4);
    uint8_t* p_cb0 = take((size_t)J);
    uint8_t* p_q = take(256);
    if (o) {
        o->pstart = reinterpret_cast<uint16_t*>(p_pre);
        o->slot = reinterpret_cast<uint16_t*>(p_slot);
        o->task_state = reinterpret_cast<uint16_t*>(p_ts);
        o->res = reinterpret_cast<uint16_t*>(p_res);
        o->maps_a = reinterpret_cast<uint16_t*>(p_ma);
        o->maps_b = reinterpret_cast<uint16_t*>(p_mb);
        o->task_chunk = reinterpret_cast<uint32_t*>(p_tc);
        o->task_res = reinterpret_cast<uint32_t*>(p_tr);
        o->toff = reinterpret_cast<unsigned*>(p_toff);
        o->cb0 = p_cb0;
        o->ctr = reinterpret_cast<unsigned*>(p_q);
    }
    return off;
}

size_t long_workspace_bytes(const DevTables& t, int64_t len, int64_t C) {
    long long J = (len + C - 1) / C;
    if (t.memo_K > 0) return memo_long_layout(std::max(J, 1LL), t.memo_K, nullptr, nullptr) + 256;
    if (t.wide_K > 0) return 2 * al256((size_t)std::max(J, 1LL) * wide_row_entries(t) * 2) + 256;
    int k = rows_kind(t);
    if (!k) return 0;
    int RW = (k == 1) ? 1 : (k == 2 ? 2 : k);
    return 2 * al256((size_t)J * t.nbits * RW * 4) + 256;
}

bool long_supported(const DevTables& t) { return t.memo_K > 0 || t.wide_K > 0 || rows_kind(t) != 0; }


cudaError_t launch_long(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, uint8_t* out, void* ws,
                        size_t ws_bytes, cudaStream_t st) {
    long long J = len > 0 ? (len + C - 1) / C : 0;
    uint8_t* w = static_cast<uint8_t*>(ws);
    if (ws_bytes < long_workspace_bytes(t, len, C)) return cudaErrorInvalidValue;
    cudaError_t e;
    if (t.memo_K > 0) {
        const int K = t.memo_K;
        if (J == 0) {
            k_finish_memo<<<1, 32, 0, st>>>(t, nullptr, 0, out);
            prof_count(1);
            return cudaGetLastError();
        }
        MemoLongWs L;
        memo_long_layout(J, K, w, &L);
        // phase 1: staged prefixes, distinct states per chunk
        const size_t tab = MemoS8::smem_bytes(t);
        int dev = 0, optin = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        int threads = (int)std::min<size_t>(256, ((size_t)optin - tab) / (2 * (size_t)K)) & ~31;
        if (threads < 32) return cudaErrorInvalidConfiguration;
        const size_t sm = tab + (size_t)threads * 2 * K;
        e = allow_smem(k_chunk_stage, sm);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chunk_stage, threads, sm);
        if (e != cudaSuccess) return e;
        long long grid = std::min<long long>((J + threads - 1) / threads, (long long)std::max(per_sm, 1) * sm_count());
        e = cudaMemsetAsync(L.ctr, 0, 256, st);
        if (e != cudaSuccess) return e;
        {
            ProfScope ps(st);
            k_chunk_stage<<<(unsigned)std::max<long long>(grid, 1), threads, sm, st>>>(
                t, str, len, C, J, L.slot, L.cb0, L.pstart, L.toff, L.task_chunk, L.task_state, L.task_res, J, L.ctr);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // phase 2: the distinct live states over the rest of their chunks
        e = launch_span_tasks(t, str, len, C, L.task_chunk, L.task_state, L.task_res, L.ctr + 2, J, L.pstart, L.res,
                              L.ctr + 1, memo_long_tasks(J, K), st);
        if (e != cudaSuccess) return e;
        // composition, left to right; the first level gathers the chunk maps
        // blocks of at most 64 maps: the first level gathers through
        // dependent loads (image position, slot, result) and the later ones
        // fold in log2(G) barrier-separated steps, so many small blocks keep
        // more SMs and warps busy than a few large ones
        const int G = std::max(2, std::min(64, (48 * 1024) / (K * 2)));
        long long cnt = (J + G - 1) / G;
        k_compose_first<<<(unsigned)cnt, 256, (size_t)G * K * 2, st>>>(L.slot, L.cb0, t.memo_imgpos, L.toff, L.res,
                                                                       J, K, G, L.maps_a);
        prof_count(1);
        uint16_t* cur = L.maps_a;
        uint16_t* nxt = L.maps_b;
        while (cnt > 1) {
            long long nb = (cnt + G - 1) / G;
            k_compose_maps<<<(unsigned)nb, 512, (size_t)G * K * 2, st>>>(cur, cnt, K, G, nxt);
            prof_count(1);
            std::swap(cur, nxt);
            cnt = nb;
        }
        k_finish_memo<<<1, 32, 0, st>>>(t, cur, 1, out);
        prof_count(1);
        return cudaGetLastError();
    }
    if (t.wide_K > 0) {
        const int rs = (int)wide_row_entries(t);
        const int stride = (int)((2 * (size_t)rs + 15) & ~size_t(15));
        if (J == 0) {
            k_wide_finish<<<1, 32, 0, st>>>(t, nullptr, 0, out);
            prof_count(1);
            return cudaGetLastError();
        }
        uint16_t* ra = reinterpret_cast<uint16_t*>(w);
        uint16_t* rb = reinterpret_cast<uint16_t*>(w + al256((size_t)J * rs * 2));
        const size_t sm = wide_seg_smem(t);
        e = allow_smem(k_wide_segments, sm);
        int per_sm = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wide_segments, kWideSegBlock, sm);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const long long wpb = kWideSegBlock / 32;
        long long grid = std::min<long long>((J + wpb - 1) / wpb, (long long)per_sm * sm_count());
        {
            ProfScope ps(st);
            k_wide_segments<<<(unsigned)std::max<long long>(grid, 1), kWideSegBlock, sm, st>>>(t, str, len, C, J, ra,
                                                                                             rs, stride);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        long long cnt = J;
        while (cnt > 1) {
            const long long np = (cnt + 1) / 2;
            const long long g = std::min<long long>((np + 7) / 8, (long long)sm_count() * 16);
            k_wide_compose<<<(unsigned)std::max<long long>(g, 1), 256, 0, st>>>(t, ra, cnt, rb, rs);
            prof_count(1);
            std::swap(ra, rb);
            cnt = np;
        }
        k_wide_finish<<<1, 32, 0, st>>>(t, ra, 1, out);
        prof_count(1);
        return cudaGetLastError();
    }
    int k = rows_kind(t);
    int RW = (k == 1) ? 1 : (k == 2 ? 2 : k);
    uint32_t* a = reinterpret_cast<uint32_t*>(w);
    uint32_t* b = reinterpret_cast<uint32_t*>(w + al256((size_t)J * t.nbits * RW * 4));
    if (J > 0) {
        switch (k) {
        case 1: e = launch_chunk_rows<Thread1Step>(t, str, len, C, J, a, st); break;
        case 2: e = launch_chunk_rows<Thread2Step>(t, str, len, C, J, a, st); break;
        case 4: e = launch_chunk_rows<SparseStep<4>>(t, str, len, C, J, a, st); break;
        case 8: e = launch_chunk_rows<SparseStep<8>>(t, str, len, C, J, a, st); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    switch (RW) {
    case 1: return compose_rows<1>(t, a, b, J, out, st);
    case 2: return compose_rows<2>(t, a, b, J, out, st);
    case 4: return compose_rows<4>(t, a, b, J, out, st);
    case 8: return compose_rows<8>(t, a, b, J, out, st);
    }
    return cudaErrorInvalidValue;
}


// ------------------------------------------------------------ chunked search
// Unanchored search of one long text (not in the paper): the earliest end j
// of a substring the expression matches.  Over the search cache (the start
// set added back after every byte), the effect of chunk j on an incoming
// state k is a pair: the state at the chunk's end, and the end offset of the
// first accepting byte in the chunk (none: -1).  Pairs compose as
//   (f1, a1) then (f2, a2) = (f2 o f1, a1(k) if a1(k) >= 0 else
//                             len1 + a2(f1(k)) if that is >= 0 else -1),
// which is associative, so chunks are computed in parallel and composed
// left to right; once a(k) is set, f(k) is never consulted.
//   phase A: one thread per chunk runs every incoming state over the first
//            P bytes, recording its first accept; the distinct states that
//            have not accepted become tasks (one atomic add per 32 chunks)
//   phase B: each task runs over the rest of its chunk (k_search_tasks)
//   phase C: the first composition level gathers each chunk's pairs, later
//            levels fold the blocks; the last pair applied to the start state
//            is the answer
namespace {

constexpr int kSearchPrefix = 64;

__global__ void __launch_bounds__(256, 4) k_search_stage(const DevTables t, const uint8_t* __restrict__ str,
                                                      int64_t len, int64_t C, long long J,
                                                      uint16_t* __restrict__ slot, uint8_t* __restrict__ pacc,
                                                      unsigned* __restrict__ toff, uint32_t* __restrict__ task_chunk,
                                                      uint16_t* __restrict__ task_state,
                                                      unsigned* __restrict__ ntask) {
    extern __shared__ __align__(16) uint8_t smem[];
    SearchS::load(t, smem);
    __syncthreads();
    SearchS proto;
    proto.bind(t, smem);
    const int K = t.srch_K;
    const int nt = blockDim.x, lane = threadIdx.x & 31;
    uint8_t* stv = smem + align16(SearchS::smem_bytes(t)) + threadIdx.x;  // state reached (interleaved)
    const long long wstride = (long long)gridDim.x * blockDim.x;
    for (long long j0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < J; j0 += wstride) {
        const long long j = j0 + lane;
        const bool valid = j < J;
        int nl = 0;
        IdSet live;  // states reached by incoming states that have not accepted
        if (valid) {
            const int64_t cs = j * C, pe = min(cs + kSearchPrefix, min(cs + C, len));
            const int n = (int)(pe - cs);
            // the prefix, read once into registers (every state walks it)
            uint32_t wb[kSearchPrefix / 4];
#pragma unroll
            for (int i = 0; i < kSearchPrefix / 4; i++) wb[i] = 0;
#pragma unroll
            for (int q = 0; q < kSearchPrefix; q++)
                if (q < n) wb[q >> 2] |= (uint32_t)__ldg(str + cs + q) << (8 * (q & 3));
            for (int k = 0; k < K; k++) {
                SearchS st = proto;
                st.set_state((uint32_t)k);
                int a = -1;
#pragma unroll
                for (int q = 0; q < kSearchPrefix; q++) {
                    if (q < n && a < 0) {
                        st.step((wb[q >> 2] >> (8 * (q & 3))) & 0xFFu);
                        if (st.accepted()) a = q + 1;
                    }
                }
                pacc[j * K + k] = a < 0 ? (uint8_t)0xFF : (uint8_t)a;
                stv[k * nt] = (uint8_t)st.state_id();
                if (a < 0) live.add(st.state_id());
            }
            nl = live.count();
        }
        int incl = nl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += x;
        }
        unsigned base = 0;
        if (lane == 31) base = atomicAdd(ntask, (unsigned)incl);
        base = __shfl_sync(FULL, base, 31) + (unsigned)(incl - nl);
        if (valid) {
            // rank of each live state id = its task index
            for (int k = 0; k < K; k++) {
                const uint32_t v = stv[k * nt];
                uint32_t r = 0;
#pragma unroll
                for (int w = 0; w < 6; w++) {
                    const uint32_t x = live.word(w);
                    r += __popc(w < (int)(v >> 5) ? x : (w == (int)(v >> 5) ? x & ((1u << (v & 31)) - 1u) : 0u));
                }
                slot[j * K + k] = pacc[j * K + k] != 0xFF ? (uint16_t)0xFFFF : (uint16_t)r;
            }
            int i = 0;
#pragma unroll
            for (int w = 0; w < 6; w++) {
                uint32_t x = live.word(w);
                while (x) {
                    task_chunk[base + i] = (uint32_t)j;
                    task_state[base + i] = (uint16_t)(w * 32 + __ffs(x) - 1);
                    i++;
                    x &= x - 1;
                }
            }
            toff[j] = base;
        }
    }
}

// each chunk's pair for every incoming state: F = state at the chunk's end,
// A = end offset of its first accepting byte (-1: none)
__global__ void k_search_pairs(const uint16_t* __restrict__ slot, const uint8_t* __restrict__ pacc,
                               const unsigned* __restrict__ toff, const uint16_t* __restrict__ res,
                               const int32_t* __restrict__ res_acc, long long J, int K, uint16_t* __restrict__ F,
                               int64_t* __restrict__ A) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < J * K;
         i += (long long)gridDim.x * blockDim.x) {
        const uint16_t r = slot[i];
        if (r == 0xFFFF) {
            F[i] = 0;
            A[i] = pacc[i];
        } else {
            const unsigned q = toff[i / K] + r;
            F[i] = res[q];
            A[i] = res_acc[q];
        }
    }
}

// level of the composition: block b folds entries [b*G, min((b+1)*G, cnt))
// (staged in shared memory) for every incoming state; entry lengths are li,
// or, with li null, chunk lengths (C, the last one shorter)
__global__ void k_search_compose(const uint16_t* __restrict__ Fi, const int64_t* __restrict__ Ai,
                                 const int64_t* __restrict__ li, int64_t C, int64_t len, long long cnt, int K, int G,
                                 uint16_t* __restrict__ Fo, int64_t* __restrict__ Ao, int64_t* __restrict__ lo_out) {
    extern __shared__ __align__(16) uint8_t sm[];
    int64_t* sa = reinterpret_cast<int64_t*>(sm);             // [G*K]
    int64_t* sl = sa + (size_t)G * K;                         // [G]
    uint16_t* sf = reinterpret_cast<uint16_t*>(sl + G);       // [G*K]
    const long long lo = (long long)blockIdx.x * G;
    const long long hi = std::min<long long>(lo + G, cnt);
    const int nb = (int)(hi - lo);
    for (int i = threadIdx.x; i < nb * K; i += blockDim.x) {
        sf[i] = Fi[lo * K + i];
        sa[i] = Ai[lo * K + i];
    }
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        sl[b] = li ? li[lo + b] : std::min<int64_t>(C, len - (lo + b) * C);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        uint32_t x = (uint32_t)k;
        int64_t a = -1, off = 0;
        for (int b = 0; b < nb && a < 0; b++) {
            const int64_t ab = sa[b * K + x];
            if (ab >= 0) a = off + ab;
            else x = sf[b * K + x];
            off += sl[b];
        }
        Fo[(long long)blockIdx.x * K + k] = (uint16_t)x;
        Ao[(long long)blockIdx.x * K + k] = a;
    }
    if (threadIdx.x == 0) {
        int64_t L = 0;
        for (int b = 0; b < nb; b++) L += sl[b];
        lo_out[blockIdx.x] = L;
    }
}

__global__ void k_search_finish(const DevTables t, const int64_t* __restrict__ A, int64_t* out) {
    if (threadIdx.x != 0) return;
    const uint32_t s0 = t.srch_start >> 8;
    out[0] = s0 >= (uint32_t)t.srch_acc0 ? 0 : (A ? A[s0] : -1);
}

struct SearchLongWs {
    uint16_t *slot, *task_state, *res, *fa, *fb, *fj;
    int64_t* aj;
    uint8_t* pacc;
    int32_t* res_acc;
    uint32_t* task_chunk;
    unsigned *toff, *ctr;
    int64_t *aa, *ab, *la, *lb;
};

size_t search_long_layout(long long J, int K, uint8_t* w, SearchLongWs* o) {
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t x = off;
        off += al256(b);
        return w ? w + x : nullptr;
    };
    const size_t JK = (size_t)J * K;
    const long long B = (J + 1) / 2 + 1;  // entries of the first composition level at most
    uint8_t* p_slot = take(JK * 2);
    uint8_t* p_pacc = take(JK);
    uint8_t* p_ts = take(JK * 2);
    uint8_t* p_tc = take(JK * 4);
    uint8_t* p_res = take(JK * 2);
    uint8_t* p_racc = take(JK * 4);
    uint8_t* p_toff = take((size_t)J * 4);
    uint8_t* p_ctr = take(256);
    uint8_t* p_fa = take((size_t)B * K * 2);
    uint8_t* p_fb = take((size_t)B * K * 2);
    uint8_t* p_aa = take((size_t)B * K * 8);
    uint8_t* p_ab = take((size_t)B * K * 8);
    uint8_t* p_la = take((size_t)B * 8);
    uint8_t* p_lb = take((size_t)B * 8);
    uint8_t* p_fj = take(JK * 2);
    uint8_t* p_aj = take(JK * 8);
    if (o) {
        o->fj = reinterpret_cast<uint16_t*>(p_fj);
        o->aj = reinterpret_cast<int64_t*>(p_aj);
        o->slot = reinterpret_cast<uint16_t*>(p_slot);
        o->pacc = p_pacc;
        o->task_state = reinterpret_cast<uint16_t*>(p_ts);
        o->task_chunk = reinterpret_cast<uint32_t*>(p_tc);
        o->res = reinterpret_cast<uint16_t*>(p_res);
        o->res_acc = reinterpret_cast<int32_t*>(p_racc);
        o->toff = reinterpret_cast<unsigned*>(p_toff);
        o->ctr = reinterpret_cast<unsigned*>(p_ctr);
        o->fa = reinterpret_cast<uint16_t*>(p_fa);
        o->fb = reinterpret_cast<uint16_t*>(p_fb);
        o->aa = reinterpret_cast<int64_t*>(p_aa);
        o->ab = reinterpret_cast<int64_t*>(p_ab);
        o->la = reinterpret_cast<int64_t*>(p_la);
        o->lb = reinterpret_cast<int64_t*>(p_lb);
    }
    return off;
}

}  // namespace

int64_t search_long_chunk_auto(const DevTables& t, int64_t len) {
    long long target = (long long)sm_count() * 1536 * 2;
    int64_t C = (len + target - 1) / std::max<long long>(target, 1);
    C = std::max<int64_t>(C, 1024);
    return (C + 31) & ~int64_t(31);
}

size_t search_long_workspace_bytes(const DevTables& t, int64_t len, int64_t C) {
    long long J = (len + C - 1) / C;
    return search_long_layout(std::max(J, 1LL), std::max(t.srch_K, 1), nullptr, nullptr) + 256;
}

cudaError_t launch_search_long(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, int64_t* out,
                               void* ws, size_t ws_bytes, cudaStream_t st) {
    if (t.srch_K <= 0 || C < kSearchPrefix) return cudaErrorInvalidValue;
    if (ws_bytes < search_long_workspace_bytes(t, len, C)) return cudaErrorInvalidValue;
    const long long J = len > 0 ? (len + C - 1) / C : 0;
    if (J == 0) {
        k_search_finish<<<1, 32, 0, st>>>(t, nullptr, out);
        prof_count(1);
        return cudaGetLastError();
    }
    const int K = t.srch_K;
    SearchLongWs L;
    search_long_layout(J, K, static_cast<uint8_t*>(ws), &L);
    // phase A
    const size_t tab = align16(SearchS::smem_bytes(t));
    const int threads = 256;
    const size_t sm = tab + (size_t)threads * K;
    cudaError_t e = allow_smem(k_search_stage, sm);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search_stage, threads, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>((J + threads - 1) / threads, (long long)per_sm * sm_count());
    e = cudaMemsetAsync(L.ctr, 0, 256, st);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(st);
        k_search_stage<<<(unsigned)std::max<long long>(grid, 1), threads, sm, st>>>(
            t, str, len, C, J, L.slot, L.pacc, L.toff, L.task_chunk, L.task_state, L.ctr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // phase B
    e = launch_search_tasks(t, str, len, C, kSearchPrefix, L.task_chunk, L.task_state, L.ctr, L.res, L.res_acc,
                            L.ctr + 1, J * K, st);
    if (e != cudaSuccess) return e;
    // phase C
    long long g3 = std::min<long long>((J * K + 255) / 256, (long long)sm_count() * 16);
    k_search_pairs<<<(unsigned)std::max<long long>(g3, 1), 256, 0, st>>>(L.slot, L.pacc, L.toff, L.res, L.res_acc, J,
                                                                         K, L.fj, L.aj);
    prof_count(1);
    const int G = (int)std::max<size_t>(2, std::min<size_t>(64, (40 * 1024) / ((size_t)K * 10 + 8)));
    const size_t csm = (size_t)G * K * 10 + (size_t)G * 8 + 16;
    const uint16_t* fi = L.fj;
    const int64_t* ai = L.aj;
    const int64_t* li = nullptr;
    uint16_t *fc = L.fa, *fn = L.fb;
    int64_t *ac = L.aa, *an = L.ab, *lc = L.la, *ln = L.lb;
    long long cnt = J;
    do {
        const long long nb = (cnt + G - 1) / G;
        k_search_compose<<<(unsigned)nb, 64, csm, st>>>(fi, ai, li, C, len, cnt, K, G, fc, ac, lc);
        prof_count(1);
        fi = fc;
        ai = ac;
        li = lc;
        std::swap(fc, fn);
        std::swap(ac, an);
        std::swap(lc, ln);
        cnt = nb;
    } while (cnt > 1);
    ac = const_cast<int64_t*>(ai);
    k_search_finish<<<1, 32, 0, st>>>(t, ac, out);
    prof_count(1);
    return cudaGetLastError();
}

}  // namespace rx
