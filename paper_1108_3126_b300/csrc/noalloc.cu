// noalloc.cu -- rx_match_static: rx_match without any device allocation.
//
// rx_match keeps a scratch buffer per stream and grows it with cudaMalloc
// (after a stream synchronisation and a cudaFree) the first time it meets a
// larger batch.  Some callers cannot accept that: a caller that must not
// block on the device, or one whose device-memory budget is fixed up front,
// cannot let the library allocate or free behind its back.  This entry point
// runs the same planner and streaming kernel with its scratch in a fixed
// array that is part of the library image on every GPU that loads it.
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace rx {
int resolve_variant(const rx_regex* h, int v);
bool on_handle_device(const rx_regex* h, const char* who);
void set_error(const std::string& msg);
}  // namespace rx

namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB per device
constexpr size_t kStaticMaxStrings = 262144;

// The scratch: queue counter, planner histograms and the length order.
// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[128] = {};  // device address of g_static_scratch, per device

// Device address of the array on the current device, looked up once per
// device with that device current.  (In host code the symbol itself is only
// a host-side stand-in, never a usable device address.)
rx_status static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        rx::set_error(std::string("rx_match_static: no current device: ") + cudaGetErrorString(e));
        return RX_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            rx::set_error(std::string("rx_match_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return RX_ERR_CUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return RX_OK;
}

}  // namespace

extern "C" rx_status rx_match_static(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets,
                                     uint8_t* out, void* stream) {
    RX_GUARD_BEGIN
    if (!h || h->host_only) {
        rx::set_error("rx_match_static: null or host-only handle");
        return RX_ERR_INVALID_ARG;
    }
    if (n == 0) return RX_OK;
    if (!offsets || !out) {
        rx::set_error("rx_match_static: null offsets or out");
        return RX_ERR_INVALID_ARG;
    }
    // the tables' addresses belong to the compile device, and the array's
    // address is looked up on the current one: they must be the same
    if (!rx::on_handle_device(h, "rx_match_static")) return RX_ERR_INVALID_ARG;
    if (n > kStaticMaxStrings) {
        rx::set_error("rx_match_static: " + std::to_string(n) + " strings exceed the limit of " +
                      std::to_string(kStaticMaxStrings) + " per call (use rx_match, which allocates)");
        return RX_ERR_TOO_LARGE;
    }
    const int variant = rx::resolve_variant(h, RX_VARIANT_AUTO);
    const int sort = rx::resolve_sort(variant, -1, n);
    const size_t need = rx::match_workspace_bytes(n, sort);
    if (need > kStaticScratchBytes) {
        rx::set_error("rx_match_static: scratch of " + std::to_string(need) + " bytes exceeds the fixed " +
                      std::to_string(kStaticScratchBytes));
        return RX_ERR_TOO_LARGE;
    }
    void* ws = nullptr;
    rx_status s = static_scratch(&ws);
    if (s != RX_OK) return s;
    // launch_match clears the work counter itself (the only part that must
    // start at zero); the planner overwrites the rest before reading it.
    cudaError_t e = rx::launch_match(h->dev, variant, n, strings, offsets, out, sort, 0, ws, kStaticScratchBytes,
                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        rx::set_error(std::string("rx_match_static launch: ") + cudaGetErrorString(e));
        return RX_ERR_CUDA;
    }
    return RX_OK;
    RX_GUARD_END
}
