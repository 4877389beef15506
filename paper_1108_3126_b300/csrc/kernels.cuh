// kernels.cuh -- launchers of the device kernels (kernels.cu), called by the
// C ABI layer (api.cpp).  All launchers are asynchronous on `stream`.
#pragma once

#include "rx_internal.h"

namespace rx {

// Length buckets used to order strings longest first.
constexpr int kLenBuckets = 2048 + 256;

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
};

// Bytes of scratch rx_match needs for n strings.
size_t match_workspace_bytes(size_t n, bool sort);

// Single expression, n strings.  variant is resolved (not AUTO).
cudaError_t launch_match(const DevTables& t, int variant, size_t n, const uint8_t* str, const int64_t* off,
                         uint8_t* out, bool sort, int block, void* ws, size_t ws_bytes, cudaStream_t stream);

// Frontier after every byte of one string.
cudaError_t launch_trace(const DevTables& t, const uint8_t* str, int64_t len, uint32_t* rows, cudaStream_t stream);

// off[0] = 0, off[1] = len (device).
cudaError_t launch_fill_offsets(int64_t* off, int64_t len, cudaStream_t stream);

// Profiling (rx_profile_*): count every launch; time main kernels when on.
void prof_count(int launches);
struct ProfScope {
    cudaStream_t st;
    void* ev0 = nullptr;
    explicit ProfScope(cudaStream_t s);
    ~ProfScope();
};
cudaError_t prof_read(int64_t* launches, int64_t* timed, double* ms);
void prof_enable(bool on);

// Device properties cached per device.
int sm_count();

}  // namespace rx
