// kernels.cuh -- launchers of the device kernels (kernels.cu), called by the
// C ABI layer (api.cpp).  All launchers are asynchronous on `stream`.
#pragma once

#include <vector>

#include "rx_internal.h"

namespace rx {

// Length buckets used to order strings longest first: below 2 KiB one
// bucket per number of 32-byte blocks a string touches (the lanes of a round
// then start and end their strings in the same block iterations),
// quarter-octave buckets above.
constexpr int kLenBuckets = 384;

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
};

// Work order of rx_match: 0 = input order, 1 = global sort by length
// (planner kernels) + the per-variant kernel, 2 = global sort + the
// streaming kernel (memo and thread variants), 3 = the streaming kernel in
// input order, 4 = the two-byte streaming kernel with a block-local length
// order (memo variant; 2 where that kernel cannot run).
int resolve_sort(int variant, int sort, size_t n);

// Bytes of scratch rx_match needs for n strings.
size_t match_workspace_bytes(size_t n, int sort);

// Single expression, n strings.  variant and sort are resolved.
cudaError_t launch_match(const DevTables& t, int variant, size_t n, const uint8_t* str, const int64_t* off,
                         uint8_t* out, int sort, int block, void* ws, size_t ws_bytes, cudaStream_t stream);

// The two-byte streaming kernel with a block-local length order (memo
// variant with the two-byte cache): one launch, no planner, no scratch.
// *launched = false (nothing enqueued) when two of its blocks do not fit on
// an SM beside the tables.
cudaError_t launch_stream_local(const DevTables& t, long long n, const uint8_t* str, const int64_t* off,
                                uint8_t* out, cudaStream_t st, bool* launched);

// Streaming kernel (memo and thread variants); perm may be NULL.
cudaError_t launch_stream(const DevTables& t, int variant, long long n, const uint8_t* str, const int64_t* off,
                          const uint32_t* perm, uint8_t* out, unsigned* queue, int block, cudaStream_t st);

// Planner: order n strings by (class, length), longest first per class.
// cls (device, n bytes) may be NULL (one class).  Writes *perm (n u32) and
// *starts (first slot of every bucket) inside ws.
size_t plan_workspace_bytes(size_t n, int nclasses);
// long_bytes: with classes, cached pairs longer than this are planned as
// kClsMemoLong (see below).  strings: the buffer the offsets index (only its
// address mod 32 is used: below 2 KiB the length key counts 32-byte blocks)
cudaError_t launch_plan(const int64_t* off, const uint8_t* cls, int nclasses, size_t n, void* ws, uint32_t** perm,
                        unsigned** starts, cudaStream_t st, unsigned* queue, long long long_bytes,
                        const void* strings);

// Batched pairs (batch.cu).  Variant classes, in task order.
struct BatchTab {
    DevTables t;
};
// kClsMemoLong: memo pairs longer than BatchLaunch::long_bytes (assigned on
// the device by the planner from the pair's length), one warp per pair,
// chunked.  kClsWide: expressions with the wide cache tier only (sets of
// more than 256 positions), one warp per pair, chunked on two-byte ids.
constexpr int kBatchClasses = 8;
// Task order (longest serial work per lane first): the classes whose lanes
// walk a whole string, the cached pairs up to long_bytes, then the chunked
// classes, whose lanes walk 1/32 of one.
enum { kClsWarp = 0, kClsSparse8 = 1, kClsSparse4 = 2, kClsThread2 = 3, kClsThread1 = 4, kClsMemo = 5,
       kClsMemoLong = 6, kClsWide = 7 };
// one warp per pair (task) rather than 32 pairs a task
__host__ __device__ constexpr bool warp_class(int c) { return c == kClsWarp || c == kClsMemoLong || c == kClsWide; }
struct BatchLaunch {
    int stride = 0;               // chunk-function row bytes per lane (batch_stride)
    int block = 256;              // threads per block: 128, 256 or 512
    long long long_bytes = 1024;  // cached pairs longer than this take a warp
    long long grid_cap = 1;       // resident blocks (set by batch_configure)
};

// Everything one batched run needs beside the pairs themselves: sizes and
// the places of its device scratch.
struct BatchPlan {
    size_t n = 0, ntabs = 0;
    void* ws = nullptr;       // batch_workspace_bytes
    uint8_t* maps = nullptr;  // batch_maps_bytes (chunk functions of long cached pairs)
};
// device bytes of a plan whose chunk-function scratch takes maps_bytes,
// and the placement of its parts in one allocation
size_t batch_plan_bytes(const BatchPlan& P, size_t maps_bytes);
void batch_plan_place(BatchPlan& P, size_t maps_bytes, void* base);
size_t batch_workspace_bytes(size_t n, size_t ntabs);
// bytes of a chunk-function row (2 + the largest cache, rounded to 16)
int batch_stride(const BatchTab* h_tabs, size_t ntabs);
cudaError_t batch_configure(BatchLaunch& L);
long long batch_grid(const BatchLaunch& L, size_t n);
// scratch for the chunk functions of long pairs (64 rows per resident warp)
size_t batch_maps_bytes(const BatchLaunch& L, size_t n);
cudaError_t batch_run(const BatchPlan& P, const uint8_t* str, const int64_t* off, uint8_t* out, const BatchLaunch& L,
                      cudaStream_t st, bool profile);
// uploads of a batch: tables, per-pair table and class
cudaError_t batch_plan_upload(const BatchPlan& P, const BatchTab* h_tabs, const uint32_t* h_pair_tab,
                              const uint8_t* h_cls, cudaStream_t st);
// host arrays of a batch: distinct tables, table index and class per pair
// (api.cpp); `who` prefixes error messages
rx_status collect_pairs(const rx_handle* handles, size_t n, const char* who, std::vector<BatchTab>& tabs,
                        std::vector<uint32_t>& pair_tab, std::vector<uint8_t>& cls);

// Spans of the chunked mode run from given cache states (stream.cu).  A
// task of chunk j = task_chunk[k] runs from j * C + pstart[j] to the chunk's
// end with one state (task_state[k] & 0xFF) or, for the ntask[0] tasks at
// [pair_base, pair_base + ntask[0]), two (the second in bits 8-15); results
// go to res[task_res[k]] (and + 1).  ntask[1] one-state tasks sit at
// [0, ntask[1]).
// warps of the span kernel resident on the whole GPU for this table
long long span_resident_warps(const DevTables& t);
cudaError_t launch_span_tasks(const DevTables& t, const uint8_t* str, int64_t len, int64_t C,
                              const uint32_t* task_chunk, const uint16_t* task_state, const uint32_t* task_res,
                              const unsigned* ntask, long long pair_base, const uint16_t* pstart, uint16_t* res,
                              unsigned* queue, long long max_tasks, cudaStream_t st);

// Unanchored search over the search cache (stream.cu): out[i] = earliest
// end of a matching substring of string i, -1 if none.
size_t search_workspace_bytes(size_t n);
cudaError_t launch_search(const DevTables& t, size_t n, const uint8_t* str, const int64_t* off, int64_t* out,
                          void* ws, size_t ws_bytes, cudaStream_t st);

// Tasks of the chunked search (stream.cu): from byte task_chunk * C + P to
// the chunk's end or first accepting byte.
cudaError_t launch_search_tasks(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, int64_t P,
                                const uint32_t* task_chunk, const uint16_t* task_state, const unsigned* ntask_p,
                                uint16_t* res, int32_t* res_acc, unsigned* queue, long long max_tasks,
                                cudaStream_t st);
// Chunked search of one long text (long.cu): out[0] = earliest end of a
// matching substring, -1 if none.
int64_t search_long_chunk_auto(const DevTables& t, int64_t len);
size_t search_long_workspace_bytes(const DevTables& t, int64_t len, int64_t C);
cudaError_t launch_search_long(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, int64_t* out,
                               void* ws, size_t ws_bytes, cudaStream_t st);

// Chunked single-string mode (long.cu).
bool long_supported(const DevTables& t);
int64_t long_chunk_auto(const DevTables& t, int64_t len);
size_t long_workspace_bytes(const DevTables& t, int64_t len, int64_t C);
cudaError_t launch_long(const DevTables& t, const uint8_t* str, int64_t len, int64_t C, uint8_t* out, void* ws,
                        size_t ws_bytes, cudaStream_t st);

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

// Section 8's machine on one string (paper_machine.cu); host-driven.
cudaError_t paper_match_one(const DevTables& t, const uint8_t* str, int64_t len, int* scratch, int* hflags,
                            uint8_t* out_host, cudaStream_t st);

// Waits of the bulk-copy streaming kernel that gave up (a device-wide
// counter; optionally cleared).
unsigned read_wait_faults(bool reset);
// Grid barriers of the one-launch planner that gave up (likewise).
unsigned read_plan_faults(bool reset);
// Device address (current device) of the counter of strings with invalid
// offsets, which every kernel that reads offsets receives; and its value,
// optionally cleared (synchronous).
unsigned long long* bad_offsets_counter();
unsigned long long read_bad_offsets(bool reset);

// Device properties cached per device.
int sm_count();

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it, so a launch or a captured graph made for a larger size by
// another thread or plan stays valid).
cudaError_t allow_smem_raw(const void* func, size_t bytes);
template <class F>
cudaError_t allow_smem(F* func, size_t bytes) {
    return allow_smem_raw(reinterpret_cast<const void*>(func), bytes);
}

}  // namespace rx
