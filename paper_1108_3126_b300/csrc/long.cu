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

// one warp per (chunk, group of 32 incoming states); lanes = incoming states
__global__ void __launch_bounds__(256) k_chunk_memo(const DevTables t, const uint8_t* __restrict__ str, int64_t len,
                                                    int64_t C, long long J, int groups, uint16_t* __restrict__ maps) {
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
        uint64_t s = base + (uint64_t)(j * C), e = base + (uint64_t)std::min<int64_t>((j + 1) * C, len);
        run_range_uniform(st, s, e);
        if (s0 < t.memo_K) maps[j * t.memo_K + s0] = (uint16_t)(st.st >> 8);
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
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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
    cudaError_t e = cudaFuncSetAttribute(k_compose_rows<RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(G * mat));
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
    int groups = t.memo_K > 0 ? (t.memo_K + 31) / 32 : (t.nbits + 31) / 32;
    long long target = (long long)sm_count() * 64 * 8 / std::max(groups, 1);
    int64_t C = (len + target - 1) / std::max<long long>(target, 1);
    C = std::max<int64_t>(C, 4096);
    return (C + 15) & ~int64_t(15);
}

size_t long_workspace_bytes(const DevTables& t, int64_t len, int64_t C) {
    long long J = (len + C - 1) / C;
    if (t.memo_K > 0) return 2 * al256((size_t)J * t.memo_K * 2) + 256;
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
        uint16_t* a = reinterpret_cast<uint16_t*>(w);
        uint16_t* b = reinterpret_cast<uint16_t*>(w + al256((size_t)J * K * 2));
        if (J > 0) {
            int groups = (K + 31) / 32;
            size_t sm = MemoStep::smem_bytes(t);
            e = cudaFuncSetAttribute(k_chunk_memo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chunk_memo, 256, sm);
            if (e != cudaSuccess) return e;
            long long need = (J * groups + 7) / 8;
            long long grid = std::min<long long>(need, (long long)std::max(per_sm, 1) * sm_count());
            {
                ProfScope ps(st);
                k_chunk_memo<<<(unsigned)std::max<long long>(grid, 1), 256, sm, st>>>(t, str, len, C, J, groups, a);
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            int G = std::max(2, std::min(512, (48 * 1024) / (K * 2)));
            long long cnt = J;
            uint16_t* cur = a;
            uint16_t* nxt = b;
            while (cnt > 1) {
                long long nb = (cnt + G - 1) / G;
                k_compose_maps<<<(unsigned)nb, 128, (size_t)G * K * 2, st>>>(cur, cnt, K, G, nxt);
                prof_count(1);
                std::swap(cur, nxt);
                cnt = nb;
            }
            k_finish_memo<<<1, 32, 0, st>>>(t, cur, 1, out);
        } else {
            k_finish_memo<<<1, 32, 0, st>>>(t, a, 0, out);
        }
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
