// host_io.cpp -- rx_match_host: rx_match on host buffers, the copies to and
// from the device pipelined with the matching.
//
// The batch is cut at string boundaries into pieces of about kPieceBytes.
// Piece k is copied on a copy stream into staging buffer k % 2 while piece
// k-1 is matched on the caller's stream; its booleans are copied back on the
// caller's stream.  Events order the reuse of each staging buffer; calls
// on one device are serialised on the host (the copy stream and its events
// are shared).  The
// kernel reads a piece through a base pointer shifted by the piece's first
// offset, so the caller's offsets are used unchanged.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace rx {
rx_status get_workspace(cudaStream_t st, size_t bytes, void** out);
void set_error(const std::string& msg);
int resolve_variant(const rx_regex* h, int v);
bool tuned_choice(const rx_regex* h, int64_t len_hint, int* variant, int* block);
}  // namespace rx

namespace {

constexpr int64_t kPieceBytes = int64_t(64) << 20;
constexpr int64_t kPieceMaxStrings = 1 << 20;

struct CopyStream {
    cudaStream_t st = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    std::mutex call;  // one call at a time uses this stream and these events
};
std::mutex g_copy_mu;
CopyStream g_copy[128];

rx_status copy_stream(CopyStream** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        rx::set_error("rx_match_host: no current device");
        return RX_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_copy_mu);
    CopyStream& c = g_copy[dev];
    if (!c.st) {
        bool ok = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 2 && ok; i++)
            ok = cudaEventCreateWithFlags(&c.ready[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c.freed[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            rx::set_error("rx_match_host: stream/event creation failed");
            return RX_ERR_CUDA;
        }
    }
    *out = &c;
    return RX_OK;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

rx_status bad_offsets(size_t i) {
    rx::set_error("rx_match_host: offsets decrease (or are negative) at " + std::to_string(i));
    return RX_ERR_INVALID_ARG;
}

// first i in [i0, i1) with offsets[i + 1] < offsets[i] or < 0 (offsets[i0]
// >= 0 is known), else -1.  A branch-free pass per block of 4096 (it
// vectorises): with every offset >= 0 a difference has its sign bit set
// exactly when it is negative.
size_t first_decrease(const int64_t* offsets, size_t i0, size_t i1) {
    for (size_t b = i0; b < i1; b += 4096) {
        const size_t e = std::min(i1, b + 4096);
        uint64_t acc = 0;
        for (size_t i = b; i < e; i++) {
            const uint64_t hi = (uint64_t)offsets[i + 1], lo = (uint64_t)offsets[i];
            acc |= hi | (hi - lo);
        }
        if (acc >> 63)
            for (size_t i = b; i < e; i++)
                if (offsets[i + 1] < 0 || offsets[i + 1] < offsets[i]) return i;
    }
    return (size_t)-1;
}

}  // namespace

extern "C" rx_status rx_match_host(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets,
                                   uint8_t* out, void* stream) {
    try {
        if (!h || h->host_only) {
            rx::set_error("rx_match_host: null or host-only handle");
            return RX_ERR_INVALID_ARG;
        }
        if (n == 0) return RX_OK;
        if (!offsets || !out || (!strings && offsets[n] > offsets[0])) {
            rx::set_error("rx_match_host: null argument");
            return RX_ERR_INVALID_ARG;
        }
        // pieces at string boundaries, found by binary search on the offsets
        // (each piece's offsets are checked just before its copy is queued,
        // so the checks of later pieces overlap the copies of earlier ones;
        // the cut points themselves are checked here, as they size the
        // staging buffers)
        std::vector<size_t> cut{0};
        int64_t max_bytes = 0;
        size_t max_n = 0;
        if (offsets[0] < 0) return bad_offsets(0);
        for (size_t i = 0; i < n;) {
            const size_t hi = std::min(n, i + (size_t)kPieceMaxStrings);
            size_t j = (size_t)(std::upper_bound(offsets + i + 1, offsets + hi + 1, offsets[i] + kPieceBytes) -
                                offsets) - 1;
            if (j <= i) j = i + 1;  // a string longer than a piece is a piece
            if (offsets[j] < offsets[i]) return bad_offsets(i);
            max_bytes = std::max<int64_t>(max_bytes, offsets[j] - offsets[i]);
            max_n = std::max(max_n, j - i);
            cut.push_back(j);
            i = j;
        }
        int variant = rx::resolve_variant(h, RX_VARIANT_AUTO), block = 0;
        {
            int tv = 0, tb = 0;
            if (rx::tuned_choice(h, 0, &tv, &tb)) {
                variant = tv;
                block = tb;
            }
        }
        const int sort = rx::resolve_sort(variant, -1, max_n);
        const size_t mws = rx::match_workspace_bytes(max_n, sort);
        const size_t buf = a256((size_t)max_bytes + 64), offb = a256((max_n + 1) * 8), resb = a256(max_n);
        const size_t total = 2 * (buf + offb + resb) + mws;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        void* ws = nullptr;
        rx_status s = rx::get_workspace(st, total, &ws);
        if (s != RX_OK) return s;
        CopyStream* cs = nullptr;
        s = copy_stream(&cs);
        if (s != RX_OK) return s;
        std::lock_guard<std::mutex> call_lock(cs->call);
        uint8_t* w = static_cast<uint8_t*>(ws);
        uint8_t* d_buf[2] = {w, w + buf};
        int64_t* d_off[2] = {reinterpret_cast<int64_t*>(w + 2 * buf), reinterpret_cast<int64_t*>(w + 2 * buf + offb)};
        uint8_t* d_res[2] = {w + 2 * (buf + offb), w + 2 * (buf + offb) + resb};
        void* mw = w + 2 * (buf + offb + resb);
        // the copy stream starts after everything already on the caller's stream
        cudaError_t e = cudaEventRecord(cs->freed[0], st);
        if (e == cudaSuccess) e = cudaEventRecord(cs->freed[1], st);
        size_t bad = (size_t)-1;
        for (size_t k = 0; k + 1 < cut.size() && e == cudaSuccess; k++) {
            const int b = (int)(k & 1);
            const size_t i0 = cut[k], i1 = cut[k + 1];
            bad = first_decrease(offsets, i0, i1);
            if (bad != (size_t)-1) break;
            const int64_t o0 = offsets[i0], bytes = offsets[i1] - o0;
            e = cudaStreamWaitEvent(cs->st, cs->freed[b], 0);
            if (e == cudaSuccess && bytes > 0)
                e = cudaMemcpyAsync(d_buf[b], strings + o0, (size_t)bytes, cudaMemcpyHostToDevice, cs->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_off[b], offsets + i0, (i1 - i0 + 1) * 8, cudaMemcpyHostToDevice, cs->st);
            if (e == cudaSuccess) e = cudaEventRecord(cs->ready[b], cs->st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, cs->ready[b], 0);
            // the kernel adds the caller's offsets to this base: piece bytes
            // start at d_buf[b]
            const uint8_t* base = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(d_buf[b]) -
                                                                   (uintptr_t)o0);
            if (e == cudaSuccess)
                e = rx::launch_match(h->dev, variant, i1 - i0, base, d_off[b], d_res[b], sort, block, mw, mws, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(out + i0, d_res[b], i1 - i0, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(cs->freed[b], st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs->st);
        if (e != cudaSuccess) {
            rx::set_error(std::string("rx_match_host: ") + cudaGetErrorString(e));
            return RX_ERR_CUDA;
        }
        if (bad != (size_t)-1) return bad_offsets(bad);
        return RX_OK;
    } catch (...) {
        rx::set_error("rx_match_host: host allocation failed");
        return RX_ERR_OOM;
    }
}
