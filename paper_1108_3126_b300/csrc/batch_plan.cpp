// batch_plan.cpp -- prepared batches (rx_batch_*): the pairs' expressions
// fixed once, the launches of a run captured into a CUDA graph and
// replayed, and a measured choice of the launch shape.
//
// rx_batch_prepare uploads the distinct tables, the table index and the
// class of every pair into device memory the plan owns (with the planner's
// and the kernel's scratch).  rx_batch_run captures, on a private stream,
// the launches of one batched run -- work-counter reset, the two planner
// launches, the persistent kernel -- for the given (strings, offsets, out)
// into a graph, and launches the graph on the caller's stream; later runs
// with the same buffers replay it.  rx_batch_autotune times the launch
// shapes (threads per block; the length above which a cached pair takes a
// whole warp) on the caller's batch and keeps the fastest.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace rx {
void set_error(const std::string& msg);
}  // namespace rx

struct rx_batch {
    int device = -1;
    size_t n = 0;
    void* ws = nullptr;  // one allocation: the workspace and the chunk-function scratch
    rx::BatchPlan P;     // its parts
    rx::BatchLaunch L;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_str = nullptr;
    const void* g_off = nullptr;
    const void* g_out = nullptr;
    bool tuned = false;
    std::mutex mu;
};

namespace {

rx_status cuda_fail(cudaError_t e, const char* what) {
    rx::set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RX_ERR_CUDA;
}

void drop_graph(rx_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->g_str = b->g_off = b->g_out = nullptr;
}

// capture the launches of one run for these buffers
cudaError_t capture(rx_batch* b, const uint8_t* str, const int64_t* off, uint8_t* out) {
    drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t er = rx::batch_run(b->P, str, off, out, b->L, b->cap, false);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (er != cudaSuccess) e = er;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return e;
    }
    b->g_str = str;
    b->g_off = off;
    b->g_out = out;
    return cudaSuccess;
}

}  // namespace

extern "C" {

rx_status rx_batch_prepare(const rx_handle* handles, size_t n, rx_batch** out) {
    try {
        if (!out || (n > 0 && !handles)) {
            rx::set_error("rx_batch_prepare: null argument");
            return RX_ERR_INVALID_ARG;
        }
        *out = nullptr;
        std::vector<rx::BatchTab> tabs;
        std::vector<uint32_t> pair_tab;
        std::vector<uint8_t> cls;
        rx_status s = rx::collect_pairs(handles, n, "rx_batch_prepare", tabs, pair_tab, cls);
        if (s != RX_OK) return s;
        rx_batch* b = new rx_batch();
        cudaGetDevice(&b->device);
        b->n = n;
        b->L.stride = rx::batch_stride(tabs.data(), tabs.size());
        b->P.n = n;
        b->P.ntabs = tabs.size();
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        // chunk-function scratch for the largest resident grid of any block
        // size the autotuner may pick
        size_t maps = 0;
        const int blocks[3] = {128, 256, 512};
        for (int i = 0; i < 3 && e == cudaSuccess; i++) {
            rx::BatchLaunch Lb = b->L;
            Lb.block = blocks[i];
            e = rx::batch_configure(Lb);
            if (e == cudaSuccess) maps = std::max(maps, rx::batch_maps_bytes(Lb, n));
        }
        if (e == cudaSuccess && n > 0) e = cudaMalloc(&b->ws, rx::batch_plan_bytes(b->P, maps));
        if (e == cudaSuccess && n > 0) rx::batch_plan_place(b->P, maps, b->ws);
        if (e == cudaSuccess && n > 0)
            e = rx::batch_plan_upload(b->P, tabs.data(), pair_tab.data(), cls.data(), b->cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
        if (e == cudaSuccess) e = rx::batch_configure(b->L);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rx_batch_free(b);
            return e == cudaErrorMemoryAllocation ? (rx::set_error("rx_batch_prepare: device allocation failed"),
                                                     RX_ERR_OOM)
                                                  : cuda_fail(e, "rx_batch_prepare");
        }
        *out = b;
        return RX_OK;
    } catch (...) {
        rx::set_error("rx_batch_prepare: host allocation failed");
        return RX_ERR_OOM;
    }
}

rx_status rx_batch_run(rx_batch* b, const uint8_t* strings, const int64_t* offsets, uint8_t* out, void* stream) {
    if (!b || (b->n > 0 && (!offsets || !out))) {
        rx::set_error("rx_batch_run: null argument");
        return RX_ERR_INVALID_ARG;
    }
    if (b->n == 0) return RX_OK;
    std::lock_guard<std::mutex> lk(b->mu);
    cudaError_t e = cudaSuccess;
    if (!b->exec || b->g_str != strings || b->g_off != offsets || b->g_out != out) e = capture(b, strings, offsets, out);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rx_batch_run");
    rx::prof_count(3);  // kernels in the graph: the planner's two launches (under capture) and k_batch
    return RX_OK;
}

rx_status rx_batch_autotune(rx_batch* b, const uint8_t* strings, const int64_t* offsets, uint8_t* out, void* stream,
                            rx_batch_tune* chosen) {
    if (!b || (b->n > 0 && (!offsets || !out))) {
        rx::set_error("rx_batch_autotune: null argument");
        return RX_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(b->mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rx_batch_tune best{b->L.long_bytes, b->L.block, -1.f};
    if (b->n > 0) {
        const long long longs[8] = {512, 1024, 2048, 3072, 4096, 6144, 8192, (long long)1 << 62};
        const int blocks[3] = {128, 256, 512};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        for (int bi = 0; bi < 3 && e == cudaSuccess; bi++)
            for (int li = 0; li < 8 && e == cudaSuccess; li++) {
                rx::BatchLaunch L = b->L;
                L.block = blocks[bi];
                L.long_bytes = longs[li];
                e = rx::batch_configure(L);
                if (e == cudaErrorInvalidValue || (e == cudaSuccess && L.grid_cap < 1)) {
                    cudaGetLastError();  // shape not launchable with this stride
                    e = cudaSuccess;
                    continue;
                }
                if (e == cudaSuccess) e = rx::batch_run(b->P, strings, offsets, out, L, st, false);
                const int reps = 3;
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int r = 0; r < reps && e == cudaSuccess; r++) e = rx::batch_run(b->P, strings, offsets, out, L, st, false);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess && ms > 0.f) {
                    const float rate = (float)reps / ms;  // runs per ms
                    if (rate > best.gb_per_s) {           // compared as runs per ms, converted below
                        best.gb_per_s = rate;
                        best.long_pair_bytes = L.long_bytes;
                        best.block = L.block;
                    }
                }
            }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(e, "rx_batch_autotune");
        if (best.gb_per_s > 0.f) {
            b->L.block = best.block;
            b->L.long_bytes = best.long_pair_bytes;
            e = rx::batch_configure(b->L);
            if (e != cudaSuccess) return cuda_fail(e, "rx_batch_autotune");
            drop_graph(b);
            b->tuned = true;
        }
        // bytes per run, for the report
        int64_t ends[2] = {0, 0};
        e = cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], offsets + b->n, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "rx_batch_autotune");
        best.gb_per_s = (float)((double)(ends[1] - ends[0]) * best.gb_per_s * 1e3 / 1e9);
    }
    if (chosen) *chosen = best;
    return RX_OK;
}

rx_status rx_batch_set_shape(rx_batch* b, const rx_batch_tune* shape) {
    if (!b || !shape || (shape->block != 128 && shape->block != 256 && shape->block != 512) ||
        shape->long_pair_bytes < 1) {
        rx::set_error("rx_batch_set_shape: null argument, block not 128/256/512, or long_pair_bytes < 1");
        return RX_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(b->mu);
    rx::BatchLaunch L = b->L;
    L.block = shape->block;
    L.long_bytes = shape->long_pair_bytes;
    cudaError_t e = rx::batch_configure(L);
    if (e == cudaSuccess && L.grid_cap < 1) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "rx_batch_set_shape");
    }
    b->L = L;
    drop_graph(b);
    return RX_OK;
}

void rx_batch_free(rx_batch* b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        drop_graph(b);
        if (b->cap) cudaStreamSynchronize(b->cap);
        if (b->ws) cudaFree(b->ws);
        if (b->cap) cudaStreamDestroy(b->cap);
    }
    delete b;
}

}  // extern "C"
