// tune.cpp -- the autotuner: measured choice of kernel variant and block
// size per (position-count bucket, mean-length bucket, cache present).
//
// rx_autotune times every variant that can run an expression, at several
// block sizes (and, for the cache of macro steps, the one- and two-byte
// lookups), on a sample batch supplied by the caller, with CUDA events on
// the caller's stream, and records the fastest.  rx_match with
// variant AUTO looks the handle's bucket up (tuned_choice).
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.cuh"

namespace rx {

rx_status get_workspace(cudaStream_t st, size_t bytes, void** out);
void set_error(const std::string& msg);

namespace {

std::mutex g_tune_mu;
// key: (pos_bucket, len_bucket (-1 = any), memo)
std::map<std::tuple<int, int, int>, rx_tune_entry> g_tune;

int log2_bucket(int64_t x) {
    int b = 0;
    uint64_t v = (uint64_t)(x + 1);
    while (v > 1) {
        v >>= 1;
        b++;
    }
    return b;
}

}  // namespace

int pos_bucket(int m) { return log2_bucket(m); }
int len_bucket(int64_t mean_len) { return log2_bucket(mean_len); }

// Tuned (variant, block) for a handle, if the table has one that can run it.
bool tuned_choice(const rx_regex* h, int64_t len_hint, int* variant, int* block) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int pb = pos_bucket(h->host.m), memo = h->host.memo_K > 0 ? 1 : 0;
    auto try_key = [&](int lb) {
        auto it = g_tune.find(std::make_tuple(pb, lb, memo));
        if (it == g_tune.end()) return false;
        if (!((h->host.variants >> it->second.variant) & 1u)) return false;
        *variant = it->second.variant;
        *block = it->second.block;
        return true;
    };
    if (len_hint > 0 && try_key(len_bucket(len_hint))) return true;
    return try_key(-1);
}

}  // namespace rx

using namespace rx;

extern "C" {

rx_status rx_autotune(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                      void* stream, rx_tune_entry* chosen) {
    try {
        if (!h || h->host_only || n == 0 || !offsets || !out) {
            set_error("rx_autotune: bad argument");
            return RX_ERR_INVALID_ARG;
        }
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        int64_t ends[2] = {0, 0};
        cudaError_t e = cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], offsets + n, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("rx_autotune: ") + cudaGetErrorString(e));
            return RX_ERR_CUDA;
        }
        const int64_t total = ends[1] - ends[0];
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        rx_tune_entry best{};
        best.gb_per_s = -1.f;
        const int variants[4] = {RX_VARIANT_MEMO, RX_VARIANT_THREAD, RX_VARIANT_SPARSE, RX_VARIANT_WARP};
        // even block sizes; for the cache of macro steps an odd size asks for
        // the one-byte-per-lookup kernel instead of the two-byte one
        const int blocks[5] = {128, 256, 512, 257, 513};
        for (int v : variants) {
            if (!((h->host.variants >> v) & 1u)) continue;
            for (int blk : blocks) {
                if ((blk & 1) && v != RX_VARIANT_MEMO) continue;
                if (blk > 256 && v != RX_VARIANT_MEMO && v != RX_VARIANT_THREAD) continue;
                int sort = resolve_sort(v, -1, n);
                size_t need = match_workspace_bytes(n, sort);
                void* ws = nullptr;
                rx_status s = get_workspace(st, need, &ws);
                if (s != RX_OK) {
                    cudaEventDestroy(a);
                    cudaEventDestroy(b);
                    return s;
                }
                e = launch_match(h->dev, v, n, strings, offsets, out, sort, blk, ws, need, st);  // warm-up
                const int reps = 3;
                cudaEventRecord(a, st);
                for (int r = 0; r < reps && e == cudaSuccess; r++)
                    e = launch_match(h->dev, v, n, strings, offsets, out, sort, blk, ws, need, st);
                cudaEventRecord(b, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e != cudaSuccess) {
                    cudaEventDestroy(a);
                    cudaEventDestroy(b);
                    set_error(std::string("rx_autotune: ") + cudaGetErrorString(e));
                    return RX_ERR_CUDA;
                }
                float gbps = (float)((double)total / (ms / reps * 1e-3) / 1e9);
                if (gbps > best.gb_per_s) {
                    best.variant = v;
                    best.block = blk;
                    best.gb_per_s = gbps;
                }
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        best.pos_bucket = pos_bucket(h->host.m);
        best.memo = h->host.memo_K > 0 ? 1 : 0;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            best.len_bucket = len_bucket(total / (int64_t)n);
            g_tune[std::make_tuple(best.pos_bucket, best.len_bucket, best.memo)] = best;
            rx_tune_entry any = best;
            any.len_bucket = -1;
            g_tune[std::make_tuple(best.pos_bucket, -1, best.memo)] = any;
        }
        if (chosen) *chosen = best;
        return RX_OK;
    } catch (...) {
        set_error("rx_autotune: host allocation failed");
        return RX_ERR_OOM;
    }
}

size_t rx_autotune_table(rx_tune_entry* out, size_t cap) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    size_t k = 0;
    for (auto& kv : g_tune) {
        if (out && k < cap) out[k] = kv.second;
        k++;
    }
    return k;
}

void rx_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // extern "C"
