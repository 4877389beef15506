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

// Phase 1: one warp per (chunk, group of 32 incoming states); lanes =
// incoming states; every lane reads the same bytes, the first P of the chunk.
__global__ void __launch_bounds__(256) k_chunk_memo(const DevTables t, const uint8_t* __restrict__ str, int64_t len,
                                                    int64_t C, int64_t P, long long J, int groups,
                                                    uint16_t* __restrict__ maps) {
    extern __shared__ __align__(16) uint8_t smem[];
    MemoStep::load(t, smem);
    __syncthreads();
    MemoStep proto;
    proto.bind(t, smem);
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const uint64_t base = reinterpret_cast<uint64_t>(str);
    for (long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < J * groups;
         task += warps) {
        long long j = task / groups;
        int g = (int)(task % groups);
        int s0 = g * 32 + lane;
        MemoStep st = proto;
        st.set_state(s0 < t.memo_K ? (uint32_t)s0 : 0u);
        const int64_t lo = j * C;
        uint64_t s = base + (uint64_t)lo, e = base + (uint64_t)min(min(lo + P, lo + C), len);
        run_range_uniform(st, s, e);
        if (s0 < t.memo_K) maps[j * t.memo_K + s0] = (uint16_t)(st.st >> 8);
    }
}

// The distinct states the K incoming states reach after the prefix: per
// chunk, slot[s] = rank of pre[s] among them, dlist[r] = the r-th, cnt.
// One warp per chunk; a bitmap of states (K <= 192) per warp in shared memory.
__global__ void __launch_bounds__(256) k_distinct(const uint16_t* __restrict__ pre, long long J, int K,
                                                  uint16_t* __restrict__ slot, uint16_t* __restrict__ dlist,
                                                  unsigned* __restrict__ cnt) {
    __shared__ unsigned bm_all[8][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned* bm = bm_all[wid];
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long j = (long long)blockIdx.x * (blockDim.x >> 5) + wid; j < J; j += warps) {
        if (lane < 8) bm[lane] = 0;
        __syncwarp();
        for (int s = lane; s < K; s += 32) {
            unsigned v = pre[j * K + s];
            atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
        __syncwarp();
        unsigned word = lane < 8 ? bm[lane] : 0u;
        unsigned c = __popc(word), incl = c;
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            unsigned x = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += x;
        }
        unsigned excl = incl - c;
        unsigned total = __shfl_sync(0xffffffffu, incl, 7);
        for (int s = lane; s < K; s += 32) {
            unsigned v = pre[j * K + s];
            unsigned w = v >> 5;
            // rank = number of distinct states below v
            unsigned base_w = 0;
            for (unsigned q = 0; q < w; q++) base_w += __popc(bm[q]);
            slot[j * K + s] = (uint16_t)(base_w + __popc(bm[w] & ((1u << (v & 31)) - 1u)));
        }
        if (lane < 8) {
            unsigned r = excl;
            unsigned x = word;
            while (x) {
                int b = __ffs(x) - 1;
                x &= x - 1;
                dlist[j * K + r++] = (uint16_t)(lane * 32 + b);
            }
        }
        if (lane == 0) cnt[j] = total;
        __syncwarp();
    }
}

// exclusive scan of the per-chunk task counts (one block); also clears the
// work counter of the span kernel that follows
__global__ void k_scan_cnt(const unsigned* __restrict__ cnt, long long J, unsigned* __restrict__ toff,
                           unsigned* __restrict__ queue) {
    __shared__ unsigned part[1024];
    const int t = threadIdx.x;
    if (t == 0) *queue = 0;
    const long long per = (J + 1023) / 1024;
    unsigned sum = 0;
    for (long long i = t * per; i < min((long long)(t + 1) * per, J); i++) sum += cnt[i];
    part[t] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        unsigned v = (t >= d) ? part[t - d] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - sum;
    for (long long i = t * per; i < min((long long)(t + 1) * per, J); i++) {
        toff[i] = run;
        run += cnt[i];
    }
    if (t == 1023) toff[J] = part[1023];
}

__global__ void k_tasks(const unsigned* __restrict__ cnt, const unsigned* __restrict__ toff,
                        const uint16_t* __restrict__ dlist, long long J, int K, uint32_t* __restrict__ task_chunk,
                        uint16_t* __restrict__ task_state) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long j = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < J; j += warps) {
        const unsigned c = cnt[j], o = toff[j];
        for (unsigned r = lane; r < c; r += 32) {
            task_chunk[o + r] = (uint32_t)j;
            task_state[o + r] = dlist[j * K + r];
        }
    }
}

__global__ void k_final_maps(const uint16_t* __restrict__ slot, const unsigned* __restrict__ toff,
                             const uint16_t* __restrict__ res, long long J, int K, uint16_t* __restrict__ maps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < J * K;
         i += (long long)gridDim.x * blockDim.x) {
        long long j = i / K;
        maps[i] = res[toff[j] + slot[i]];
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
    for (int s = threadIdx.x; s < K; s += blockDim.x) {
        int x = s;
        for (int j = 0; j < nmap; j++) x = sm16[j * K + x];
        out[(long long)blockIdx.x * K + s] = (uint16_t)x;
    }
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

}  // namespace

int64_t long_chunk_auto(const DevTables& t, int64_t len) {
    if (t.memo_K > 0) {
        // enough chunks that the converged tasks (about one per chunk) fill
        // every lane of the GPU a few times over
        long long target = (long long)sm_count() * 1536 * 2;
        int64_t C = (len + target - 1) / std::max<long long>(target, 1);
        C = std::max<int64_t>(C, 1024);
        return (C + 31) & ~int64_t(31);
    }
    int groups = (t.nbits + 31) / 32;
    long long target = (long long)sm_count() * 64 * 8 / std::max(groups, 1);
    int64_t C = (len + target - 1) / std::max<long long>(target, 1);
    C = std::max<int64_t>(C, 4096);
    return (C + 15) & ~int64_t(15);
}

// prefix every incoming state runs before the distinct states are taken
constexpr int64_t kLongPrefix = 128;

struct MemoLongWs {
    uint16_t *pre, *slot, *dlist, *task_state, *res, *maps_a, *maps_b;
    uint32_t* task_chunk;
    unsigned *cnt, *toff, *queue;
};

static size_t memo_long_layout(long long J, int K, uint8_t* w, MemoLongWs* o) {
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t x = off;
        off += al256(b);
        return w ? w + x : nullptr;
    };
    const size_t JK = (size_t)J * K;
    uint8_t* p_pre = take(JK * 2);
    uint8_t* p_slot = take(JK * 2);
    uint8_t* p_dl = take(JK * 2);
    uint8_t* p_ts = take(JK * 2);
    uint8_t* p_res = take(JK * 2);
    uint8_t* p_ma = take(JK * 2);
    uint8_t* p_mb = take(JK * 2);
    uint8_t* p_tc = take(JK * 4);
    uint8_t* p_cnt = take((size_t)J * 4);
    uint8_t* p_toff = take((size_t)(J + 1) * 4);
    uint8_t* p_q = take(256);
    if (o) {
        o->pre = reinterpret_cast<uint16_t*>(p_pre);
        o->slot = reinterpret_cast<uint16_t*>(p_slot);
        o->dlist = reinterpret_cast<uint16_t*>(p_dl);
        o->task_state = reinterpret_cast<uint16_t*>(p_ts);
        o->res = reinterpret_cast<uint16_t*>(p_res);
        o->maps_a = reinterpret_cast<uint16_t*>(p_ma);
        o->maps_b = reinterpret_cast<uint16_t*>(p_mb);
        o->task_chunk = reinterpret_cast<uint32_t*>(p_tc);
        o->cnt = reinterpret_cast<unsigned*>(p_cnt);
        o->toff = reinterpret_cast<unsigned*>(p_toff);
        o->queue = reinterpret_cast<unsigned*>(p_q);
    }
    return off;
}

size_t long_workspace_bytes(const DevTables& t, int64_t len, int64_t C) {
    long long J = (len + C - 1) / C;
    if (t.memo_K > 0) return memo_long_layout(std::max(J, 1LL), t.memo_K, nullptr, nullptr) + 256;
    int k = rows_kind(t);
    if (!k) return 0;
    int RW = (k == 1) ? 1 : (k == 2 ? 2 : k);
    return 2 * al256((size_t)J * t.nbits * RW * 4) + 256;
}

bool long_supported(const DevTables& t) { return t.memo_K > 0 || rows_kind(t) != 0; }

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
        const int64_t P = std::min<int64_t>(kLongPrefix, C);
        // phase 1: every incoming state over the first P bytes of each chunk
        int groups = (K + 31) / 32;
        size_t sm = MemoStep::smem_bytes(t);
        e = allow_smem(k_chunk_memo, sm);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chunk_memo, 256, sm);
        if (e != cudaSuccess) return e;
        long long need = (J * groups + 7) / 8;
        long long grid = std::min<long long>(need, (long long)std::max(per_sm, 1) * sm_count() * 4);
        {
            ProfScope ps(st);
            k_chunk_memo<<<(unsigned)std::max<long long>(grid, 1), 256, sm, st>>>(t, str, len, C, P, J, groups, L.pre);
        }
        // the distinct states reached, one task per (chunk, distinct state)
        long long g2 = std::min<long long>((J + 7) / 8, (long long)sm_count() * 16);
        k_distinct<<<(unsigned)std::max<long long>(g2, 1), 256, 0, st>>>(L.pre, J, K, L.slot, L.dlist, L.cnt);
        k_scan_cnt<<<1, 1024, 0, st>>>(L.cnt, J, L.toff, L.queue);
        k_tasks<<<(unsigned)std::max<long long>(g2, 1), 256, 0, st>>>(L.cnt, L.toff, L.dlist, J, K, L.task_chunk,
                                                                     L.task_state);
        prof_count(3);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // phase 2: the distinct states over the rest of their chunks
        e = launch_span_tasks(t, str, len, C, P, L.task_chunk, L.task_state, L.toff + J, L.res, L.queue, J * K, st);
        if (e != cudaSuccess) return e;
        long long g3 = std::min<long long>((J * K + 255) / 256, (long long)sm_count() * 16);
        k_final_maps<<<(unsigned)std::max<long long>(g3, 1), 256, 0, st>>>(L.slot, L.toff, L.res, J, K, L.maps_a);
        prof_count(1);
        // composition, left to right
        int G = std::max(2, std::min(512, (48 * 1024) / (K * 2)));
        long long cnt = J;
        uint16_t* cur = L.maps_a;
        uint16_t* nxt = L.maps_b;
        while (cnt > 1) {
            long long nb = (cnt + G - 1) / G;
            k_compose_maps<<<(unsigned)nb, 128, (size_t)G * K * 2, st>>>(cur, cnt, K, G, nxt);
            prof_count(1);
            std::swap(cur, nxt);
            cnt = nb;
        }
        k_finish_memo<<<1, 32, 0, st>>>(t, cur, 1, out);
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

}  // namespace rx
