// serve.cu -- continuous-batching matcher (rx_serve_*).
//
// A host scheduler thread owns a CUDA stream and a table of device slots.
// Each iteration ("tick") it
//   1. admits pending requests while a slot is free and the device bytes
//      held by in-flight requests stay under the budget (the payload copy is
//      issued on a copy stream, the tick waits for it with an event);
//   2. launches one kernel that advances EVERY in-flight request by up to
//      tick_bytes -- one macro step (Rathnayake & Thielecke, SOS 2011,
//      Def 5.2) per byte, the active set saved in the slot between ticks;
//   3. reads back the slots' done flags and results, completes finished
//      requests (latency = completion - submission) and frees their memory.
// Requests arriving while a tick runs join at the next tick, so their work
// overlaps on the device with requests already in flight.  A request with a
// cache of macro steps and more than 2 ticks of bytes left takes a whole
// warp in that tick: 32 lanes advance 32 consecutive spans of tick bytes as
// chunk transfer functions composed from the saved state (exact, Def 5.2
// acts on states), so long requests move 32 times as far per tick.
// Requests longer than long_threshold run the exact chunked mode (long.cu)
// on their own stream and complete when its event fires.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "steppers.cuh"

namespace rx {

rx_status get_workspace(cudaStream_t st, size_t bytes, void** out);

namespace {

using namespace rx::dev;

constexpr int kStateWords = kWarpMaxWords;  // saved set per slot (words)
constexpr int kMapStride = (kMemoMaxStates + 2 + 15) & ~15;  // chunk-function row per lane of a long slot

struct ServeSlot {
    const DevTables* tab;
    const uint8_t* data;
    int64_t len;
    int64_t pos;
    int32_t cls;
    int32_t pad;
};

int serve_class(const rx_regex* h) {
    const Compiled& C = h->host;
    if (C.memo_K > 0) return kClsMemo;
    if (C.wide_K > 0) return kClsWide;
    if (C.gl_ok) return C.W == 1 ? kClsThread1 : kClsThread2;
    if (C.W <= 4) return kClsSparse4;
    if (C.W <= 8) return kClsSparse8;
    return kClsWarp;
}

template <class S>
__device__ __forceinline__ void tick_lane(const ServeSlot& sl, bool valid, int64_t tick, uint32_t* state,
                                          uint8_t* status) {
    // every lane binds a table -- a lane past the class's slots gets the
    // table of the class's first slot -- because the span loop steps every
    // lane (killed ones on the empty set) and a step reads the table
    S st;
    st.bind_global(*sl.tab);
    if (valid) {
        if (sl.pos > 0) st.restore(state);
    } else {
        st.kill();
    }
    const uint64_t base = reinterpret_cast<uint64_t>(sl.data);
    int64_t end = valid ? min(sl.len, sl.pos + tick) : 0;
    uint64_t s = base + (uint64_t)(valid ? sl.pos : 0), e = base + (uint64_t)end;
    run_lane_span(st, s, e, valid);
    if (!valid) return;
    if (end >= sl.len || st.dead()) {
        status[0] = 1;
        status[1] = (end >= sl.len) ? (uint8_t)st.accept() : 0;
    } else {
        st.save(state);
        status[0] = 0;
    }
}

template <int K>
__device__ void tick_warp(const ServeSlot& sl, int64_t tick, uint32_t* state, uint8_t* status) {
    const DevTables& t = *sl.tab;
    const int lane = threadIdx.x & 31;
    uint32_t F[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        int w = k * 32 + lane;
        F[k] = (w < t.W) ? (sl.pos > 0 ? state[w] : t.start[w]) : 0u;
    }
    const uint64_t base = reinterpret_cast<uint64_t>(sl.data);
    int64_t end = min(sl.len, sl.pos + tick);
    bool dead = warp_span<K>(t, t.B, t.follow, base + sl.pos, base + end, F);
    bool acc = warp_accepts<K>(t, F);
    if (end >= sl.len || dead) {
        if (lane == 0) {
            status[0] = 1;
            status[1] = (end >= sl.len && !dead) ? (uint8_t)acc : 0;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; k++) {
            int w = k * 32 + lane;
            if (w < t.W) state[w] = F[k];
        }
        if (lane == 0) status[0] = 0;
    }
}

// a cached request with many bytes left: the warp advances it by up to 32
// spans of `tick` bytes (32 chunks) from its saved state; wsm: the slot's
// chunk-map scratch (64 rows of kMapStride bytes)
__device__ void tick_memo_long(const ServeSlot& sl, int64_t tick, uint32_t* state, uint8_t* status, uint8_t* wsm) {
    const DevTables& t = *sl.tab;
    const int lane = threadIdx.x & 31;
    const uint32_t x0 = sl.pos > 0 ? state[0] >> 8 : t.memo_start >> 8;
    const uint64_t base = reinterpret_cast<uint64_t>(sl.data);
    const int64_t end = min(sl.len, sl.pos + 32 * tick);
    const uint32_t x = warp_chunked_memo(t, x0, base + sl.pos, base + end, wsm, kMapStride);
    if (lane != 0) return;
    if (end >= sl.len || x == 0) {
        status[0] = 1;
        status[1] = end >= sl.len ? t.memo_acc[x] : 0;
    } else {
        state[0] = x << 8;
        status[0] = 0;
    }
}

// the same on the wide tier (two-byte state ids): every request of such an
// expression takes a warp, whatever is left
__device__ void tick_wide(const ServeSlot& sl, int64_t tick, uint32_t* state, uint8_t* status, uint8_t* wsm) {
    const DevTables& t = *sl.tab;
    const int lane = threadIdx.x & 31;
    const uint32_t x0 = sl.pos > 0 ? state[0] : t.wide_start;
    const uint64_t base = reinterpret_cast<uint64_t>(sl.data);
    const int64_t end = min(sl.len, sl.pos + 32 * tick);
    const uint32_t x = warp_chunked_wide(t, x0, base + sl.pos, base + end, wsm, kMapStride);
    if (lane != 0) return;
    if (end >= sl.len || x == 0) {
        status[0] = 1;
        status[1] = end >= sl.len ? t.wide_acc[x] : 0;
    } else {
        state[0] = x;
        status[0] = 0;
    }
}
static_assert(2 * (kWideMaxImg + 2) <= kMapStride, "a wide chunk row fits a slot's row");

struct Segs {
    int32_t lo[kBatchClasses + 1];   // slot-order segment of each class
    int32_t task[kBatchClasses + 1]; // first task of each class
    int64_t span[kBatchClasses];     // bytes a request of the class advances (per lane / chunk)
};

// A tick's bytes per class: the classes without a cache of macro steps cost
// a lane more per byte (a bitset step; the warp class a ballot loop over
// the active bits), so they take a smaller share, which keeps one slow
// request from setting the length of the whole tick; a cached request
// advances `tick` bytes (32 spans of it when it has a warp).
int64_t class_span(int c, int64_t tick, int64_t base) {
    switch (c) {
    case kClsWarp: return std::max<int64_t>(256, base / 16);
    case kClsSparse8:
    case kClsSparse4: return std::max<int64_t>(256, base / 2);
    case kClsThread1:
    case kClsThread2: return base;
    default: return tick;
    }
}

// one warp per task: a warp-class slot, or up to 32 slots of one class
__global__ void __launch_bounds__(256) k_serve_tick(const ServeSlot* __restrict__ slots,
                                                    const int32_t* __restrict__ order, Segs sg,
                                                    uint32_t* __restrict__ state, uint8_t* __restrict__ status,
                                                    uint8_t* __restrict__ maps) {
    const int lane = threadIdx.x & 31;
    const int task = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (task >= sg.task[kBatchClasses]) return;
    int c = 0;
    while (c + 1 < kBatchClasses && task >= sg.task[c + 1]) c++;
    const int g = task - sg.task[c];
    const int64_t tick = sg.span[c];
    if (c == kClsMemoLong || c == kClsWide) {
        const int slot = order[sg.lo[c] + g];
        uint8_t* wsm = maps + (size_t)slot * 64 * kMapStride;
        if (c == kClsWide) tick_wide(slots[slot], tick, state + (size_t)slot * kStateWords, status + 2 * slot, wsm);
        else tick_memo_long(slots[slot], tick, state + (size_t)slot * kStateWords, status + 2 * slot, wsm);
        return;
    }
    if (c == kClsWarp) {
        const int slot = order[sg.lo[c] + g];
        const ServeSlot sl = slots[slot];
        uint32_t* stp = state + (size_t)slot * kStateWords;
        uint8_t* stt = status + 2 * slot;
        int W = sl.tab->W;
        if (W <= 32) tick_warp<1>(sl, tick, stp, stt);
        else if (W <= 64) tick_warp<2>(sl, tick, stp, stt);
        else tick_warp<4>(sl, tick, stp, stt);
        return;
    }
    const int idx = sg.lo[c] + g * 32 + lane;
    const bool valid = idx < sg.lo[c + 1];
    const int slot = valid ? order[idx] : order[sg.lo[c]];
    const ServeSlot sl = slots[slot];
    uint32_t* stp = state + (size_t)slot * kStateWords;
    uint8_t* stt = status + 2 * slot;
    switch (c) {
    case kClsMemo: tick_lane<MemoStep8>(sl, valid, tick, stp, stt); break;
    case kClsThread1: tick_lane<Thread1Step>(sl, valid, tick, stp, stt); break;
    case kClsThread2: tick_lane<Thread2Step>(sl, valid, tick, stp, stt); break;
    case kClsSparse4: tick_lane<SparseStep<4>>(sl, valid, tick, stp, stt); break;
    default: tick_lane<SparseStep<8>>(sl, valid, tick, stp, stt); break;
    }
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

}  // namespace rx

using namespace rx;

struct Request {
    uint64_t ticket;
    rx_regex* h;
    std::vector<uint8_t> host;  // host payload copy (payload mode 0)
    const uint8_t* hsrc = nullptr;  // caller's host payload (mode 2, borrowed)
    const uint8_t* dptr;        // device payload (caller's or ours)
    uint8_t* owned;             // device payload we allocated
    int64_t len;
    int64_t t_submit;
    int slot = -1;
    bool is_long = false;   // runs the chunked mode alone on a side stream
    void* long_ws = nullptr;
    size_t res_off = 0;     // offset of the result byte in long_ws
    cudaEvent_t ev = nullptr;
    int64_t charged = 0;
};

struct Done {
    uint64_t ticket;
    uint8_t result;
    rx_status st;
};

struct rx_server {
    rx_serve_cfg cfg{};
    int device = 0;
    int64_t budget = 0, long_threshold = 1 << 20;
    static constexpr int64_t kRowsLong = 1 << 20;  // chunked mode for uncached requests from here
    static constexpr int kLongStreams = 4;
    static constexpr int64_t kTickGrow = 8;
    static constexpr size_t kMaxLong = 32;
    cudaStream_t st = nullptr, copy_st = nullptr, long_st[kLongStreams] = {};
    int next_long = 0;
    ServeSlot* d_slots = nullptr;
    ServeSlot* h_slots = nullptr;  // pinned
    int32_t* d_order = nullptr;
    int32_t* h_order = nullptr;  // pinned
    uint32_t* d_state = nullptr;
    uint8_t* d_maps = nullptr;  // chunk maps of the long cached slots
    uint8_t* d_status = nullptr;
    uint8_t* h_status = nullptr;  // pinned
    std::vector<Request*> slots;
    std::vector<Request*> longs;
    std::deque<Request*> pending;
    std::deque<Done> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::atomic<uint64_t> next_ticket{1};
    // stats
    uint64_t submitted = 0, completed = 0;
    std::vector<double> lat;
    int64_t t_first = 0, t_last = 0, bytes_done = 0, ticks = 0, peak_inflight = 0, peak_bytes = 0;
    int64_t inflight_bytes = 0;
    std::string fail;

    void run();
    void complete(Request* r, uint8_t res, rx_status s);
};

void rx_server::complete(Request* r, uint8_t res, rx_status s) {
    int64_t t = now_ns();
    if (r->owned) cudaFreeAsync(r->owned, st);
    if (r->long_ws) cudaFreeAsync(r->long_ws, st);
    if (r->ev) cudaEventDestroy(r->ev);
    {
        std::lock_guard<std::mutex> lk(mu);
        done.push_back(Done{r->ticket, res, s});
        completed++;
        lat.push_back((double)(t - r->t_submit));
        t_last = t;
        bytes_done += r->len;
        inflight_bytes -= r->charged;
    }
    cv_done.notify_all();
    delete r;
}

void rx_server::run() {
    cudaSetDevice(device);
    const int nslot = cfg.max_inflight;
    std::vector<int> free_slots;
    for (int i = nslot - 1; i >= 0; i--) free_slots.push_back(i);
    std::vector<int64_t> tick_span(nslot, 0);  // bytes each slot advances this tick
    std::vector<Request*> admitted;
    while (true) {
        admitted.clear();
        {
            std::unique_lock<std::mutex> lk(mu);
            bool idle = std::all_of(slots.begin(), slots.end(), [](Request* r) { return r == nullptr; }) &&
                        longs.empty();
            if (idle && pending.empty() && !stop) cv_work.wait_for(lk, std::chrono::milliseconds(2));
            if (stop) break;
            // admission: by free slots / long capacity and the device-byte budget
            while (!pending.empty()) {
                Request* r = pending.front();
                // without a cache a request advances only a few KiB per tick
                // (bitset steppers), so from 1 MiB it runs the chunked mode
                const int64_t lt = (r->h->dev.memo_K > 0 || r->h->dev.wide_K > 0)
                                       ? long_threshold
                                       : std::min<int64_t>(long_threshold, kRowsLong);
                bool lng = r->len > lt && long_supported(r->h->dev);
                int64_t need = (cfg.device_payload == 1 ? 0 : r->len);
                if (lng) need += (int64_t)long_workspace_bytes(r->h->dev, r->len, long_chunk_auto(r->h->dev, r->len));
                bool room = lng ? longs.size() < kMaxLong : !free_slots.empty();
                if (!room || (inflight_bytes + need > budget && inflight_bytes > 0)) break;
                pending.pop_front();
                r->charged = need;
                r->is_long = lng;
                inflight_bytes += need;
                if (!lng) {
                    r->slot = free_slots.back();
                    free_slots.pop_back();
                }
                admitted.push_back(r);
            }
            peak_bytes = std::max(peak_bytes, inflight_bytes);
        }
        // payload copies (copy stream) and long launches
        for (Request* r : admitted) {
            if (cfg.device_payload != 1 && r->len > 0) {
                cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&r->owned), (size_t)r->len, copy_st);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    r->owned = nullptr;
                    if (r->slot >= 0) free_slots.push_back(r->slot);
                    complete(r, 0, RX_ERR_OOM);
                    continue;
                }
                // mode 0: our pageable copy (staged by the driver); mode 2:
                // the caller's buffer, a direct DMA when it is page-locked
                cudaMemcpyAsync(r->owned, cfg.device_payload == 2 ? r->hsrc : r->host.data(), (size_t)r->len,
                                cudaMemcpyHostToDevice, copy_st);
                r->dptr = r->owned;
            }
            if (r->is_long) {
                cudaStream_t ls = long_st[next_long];
                next_long = (next_long + 1) % kLongStreams;
                cudaEvent_t ce = nullptr;
                cudaEventCreateWithFlags(&ce, cudaEventDisableTiming);
                cudaEventRecord(ce, copy_st);
                cudaStreamWaitEvent(ls, ce, 0);
                cudaEventDestroy(ce);
                const int64_t C = long_chunk_auto(r->h->dev, r->len);
                const size_t wsb = long_workspace_bytes(r->h->dev, r->len, C);
                if (cudaMallocAsync(&r->long_ws, wsb + 256, ls) != cudaSuccess) {
                    cudaGetLastError();
                    r->long_ws = nullptr;
                    complete(r, 0, RX_ERR_OOM);
                    continue;
                }
                r->res_off = wsb;
                cudaError_t e = launch_long(r->h->dev, r->dptr, r->len, C, static_cast<uint8_t*>(r->long_ws) + wsb,
                                            r->long_ws, wsb, ls);
                r->host.clear();
                r->host.shrink_to_fit();
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    complete(r, 0, RX_ERR_UNSUPPORTED);
                    continue;
                }
                cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
                cudaEventRecord(r->ev, ls);
                longs.push_back(r);
                continue;
            }
            ServeSlot& sl = h_slots[r->slot];
            sl.tab = r->h->dev_self;
            sl.data = r->dptr;
            sl.len = r->len;
            sl.pos = 0;
            sl.cls = serve_class(r->h);
            slots[r->slot] = r;
        }
        if (!admitted.empty()) {
            cudaEvent_t e2 = nullptr;
            cudaEventCreateWithFlags(&e2, cudaEventDisableTiming);
            cudaEventRecord(e2, copy_st);
            cudaStreamWaitEvent(st, e2, 0);
            cudaEventDestroy(e2);
        }
        // one tick over every short in-flight request
        std::vector<int> cls_slots[kBatchClasses];
        int inflight = 0;
        for (int i = 0; i < nslot; i++)
            if (slots[i]) inflight++;
        // a tick advances every request by `tick` bytes; with few requests
        // in flight the GPU would idle between short ticks, so the tick
        // grows (up to kTickGrow times) as the in-flight count falls
        const int64_t grow = std::max<int64_t>(1, std::min<int64_t>(kTickGrow, kTickGrow / std::max(inflight, 1)));
        const int64_t tick = cfg.tick_bytes * grow;
        int64_t span[kBatchClasses];
        for (int c = 0; c < kBatchClasses; c++) span[c] = class_span(c, tick, cfg.tick_bytes);
        for (int i = 0; i < nslot; i++)
            if (slots[i]) {
                int c = h_slots[i].cls;
                // a cached request with more than a tick left takes a warp
                if (c == kClsMemo && h_slots[i].len - h_slots[i].pos > tick) c = kClsMemoLong;
                cls_slots[c].push_back(i);
                tick_span[i] = (c == kClsMemoLong || c == kClsWide) ? 32 * span[c] : span[c];
            }
        {
            std::lock_guard<std::mutex> lk(mu);
            peak_inflight = std::max<int64_t>(peak_inflight, inflight + (int64_t)longs.size());
        }
        if (inflight > 0) {
            Segs sg{};
            int k = 0, tasks = 0;
            for (int c = 0; c < kBatchClasses; c++) {
                sg.span[c] = span[c];
                sg.lo[c] = k;
                sg.task[c] = tasks;
                for (int i : cls_slots[c]) h_order[k++] = i;
                int cnt = (int)cls_slots[c].size();
                tasks += warp_class(c) ? cnt : (cnt + 31) / 32;
            }
            sg.lo[kBatchClasses] = k;
            sg.task[kBatchClasses] = tasks;
            cudaMemcpyAsync(d_slots, h_slots, sizeof(ServeSlot) * nslot, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(d_order, h_order, sizeof(int32_t) * k, cudaMemcpyHostToDevice, st);
            int blocks = (tasks * 32 + 255) / 256;
            {
                ProfScope ps(st);
                k_serve_tick<<<blocks, 256, 0, st>>>(d_slots, d_order, sg, d_state, d_status, d_maps);
            }
            cudaMemcpyAsync(h_status, d_status, 2 * (size_t)nslot, cudaMemcpyDeviceToHost, st);
            cudaError_t e = cudaStreamSynchronize(st);
            ticks++;
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(mu);
                fail = cudaGetErrorString(e);
            }
            for (int i = 0; i < nslot; i++) {
                Request* r = slots[i];
                if (!r) continue;
                if (h_status[2 * i] == 1 || e != cudaSuccess) {
                    slots[i] = nullptr;
                    free_slots.push_back(i);
                    complete(r, h_status[2 * i + 1], e == cudaSuccess ? RX_OK : RX_ERR_CUDA);
                } else {
                    h_slots[i].pos = std::min(h_slots[i].len, h_slots[i].pos + tick_span[i]);
                }
            }
        } else if (!longs.empty()) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        // long requests whose chunked run has finished
        for (size_t i = 0; i < longs.size();) {
            Request* r = longs[i];
            cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) {
                i++;
                continue;
            }
            uint8_t res = 0;
            if (q == cudaSuccess)
                q = cudaMemcpy(&res, static_cast<uint8_t*>(r->long_ws) + r->res_off, 1, cudaMemcpyDeviceToHost);
            longs.erase(longs.begin() + i);
            complete(r, res, q == cudaSuccess ? RX_OK : RX_ERR_CUDA);
        }
    }
}

extern "C" {

rx_status rx_serve_create(const rx_serve_cfg* cfg, rx_server** out) {
    try {
        if (!out) {
            set_error("rx_serve_create: null out");
            return RX_ERR_INVALID_ARG;
        }
        *out = nullptr;
        if (cfg && (cfg->device_payload < 0 || cfg->device_payload > 2)) {
            set_error("rx_serve_create: device_payload must be 0, 1 or 2");
            return RX_ERR_INVALID_ARG;
        }
        rx_server* s = new rx_server();
        if (cfg) s->cfg = *cfg;
        if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 1024;
        if (s->cfg.queue_capacity <= 0) s->cfg.queue_capacity = 1 << 16;
        if (s->cfg.tick_bytes <= 0) s->cfg.tick_bytes = 1 << 13;
        s->long_threshold = s->cfg.long_threshold > 0 ? s->cfg.long_threshold : (1 << 25);
        cudaGetDevice(&s->device);
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            delete s;
            set_error(std::string("rx_serve_create: ") + cudaGetErrorString(e));
            return RX_ERR_CUDA;
        }
        s->budget = s->cfg.device_budget_bytes > 0 ? s->cfg.device_budget_bytes : (int64_t)(fr / 4);
        const int n = s->cfg.max_inflight;
        bool ok = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < rx_server::kLongStreams && ok; i++)
            ok = cudaStreamCreateWithFlags(&s->long_st[i], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok &&
                  cudaMalloc(&s->d_slots, sizeof(ServeSlot) * n) == cudaSuccess &&
                  cudaMalloc(&s->d_order, sizeof(int32_t) * n) == cudaSuccess &&
                  cudaMalloc(&s->d_state, sizeof(uint32_t) * (size_t)kStateWords * n) == cudaSuccess &&
                  cudaMalloc(&s->d_maps, (size_t)64 * kMapStride * n) == cudaSuccess &&
                  cudaMalloc(&s->d_status, 2 * (size_t)n) == cudaSuccess &&
                  cudaMallocHost(&s->h_slots, sizeof(ServeSlot) * n) == cudaSuccess &&
                  cudaMallocHost(&s->h_order, sizeof(int32_t) * n) == cudaSuccess &&
                  cudaMallocHost(&s->h_status, 2 * (size_t)n) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rx_serve_destroy(s);
            set_error("rx_serve_create: device or pinned allocation failed");
            return RX_ERR_OOM;
        }
        std::memset(s->h_slots, 0, sizeof(ServeSlot) * n);
        s->slots.assign(n, nullptr);
        s->worker = std::thread([s] { s->run(); });
        *out = s;
        return RX_OK;
    } catch (...) {
        set_error("rx_serve_create: host allocation failed");
        return RX_ERR_OOM;
    }
}

rx_status rx_serve_submit(rx_server* s, rx_handle h, const uint8_t* bytes, int64_t len, uint64_t* ticket) {
    try {
        if (!s || !h || h->host_only || len < 0 || (len > 0 && !bytes)) {
            set_error("rx_serve_submit: bad argument");
            return RX_ERR_INVALID_ARG;
        }
        Request* r = new Request();
        r->h = h;
        r->len = len;
        r->owned = nullptr;
        r->dptr = s->cfg.device_payload == 1 ? bytes : nullptr;
        r->hsrc = s->cfg.device_payload == 2 ? bytes : nullptr;
        if (s->cfg.device_payload == 0 && len > 0) r->host.assign(bytes, bytes + len);
        r->t_submit = now_ns();
        uint64_t tk = 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if ((int64_t)s->pending.size() >= s->cfg.queue_capacity) {
                delete r;
                set_error("rx_serve_submit: queue full");
                return RX_ERR_BUSY;
            }
            tk = r->ticket = s->next_ticket++;
            if (s->submitted == 0) s->t_first = r->t_submit;
            s->submitted++;
            s->pending.push_back(r);
            // from here on the worker owns r (it may complete and free it at once)
        }
        s->cv_work.notify_one();
        if (ticket) *ticket = tk;
        return RX_OK;
    } catch (...) {
        set_error("rx_serve_submit: host allocation failed");
        return RX_ERR_OOM;
    }
}

rx_status rx_serve_replay(rx_server* s, const rx_handle* handles, const uint8_t* const* payloads,
                          const int64_t* lens, const int64_t* arrival_ns, size_t n, uint64_t* tickets,
                          int64_t* late_ns) {
    if (!s || (n && (!handles || !payloads || !lens || !arrival_ns))) {
        set_error("rx_serve_replay: bad argument");
        return RX_ERR_INVALID_ARG;
    }
    const int64_t t0 = now_ns();
    int64_t late = 0;
    for (size_t i = 0; i < n; i++) {
        const int64_t due = t0 + arrival_ns[i];
        while (now_ns() < due) {
        }
        late = std::max(late, now_ns() - due);
        uint64_t t = 0;
        rx_status st;
        while ((st = rx_serve_submit(s, handles[i], payloads[i], lens[i], &t)) == RX_ERR_BUSY)
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        if (st != RX_OK) return st;
        if (tickets) tickets[i] = t;
    }
    if (late_ns) *late_ns = late;
    return RX_OK;
}

size_t rx_serve_poll(rx_server* s, uint64_t* tickets, uint8_t* results, rx_status* st, size_t max) {
    if (!s) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    size_t k = 0;
    while (k < max && !s->done.empty()) {
        const Done& d = s->done.front();
        if (tickets) tickets[k] = d.ticket;
        if (results) results[k] = d.result;
        if (st) st[k] = d.st;
        s->done.pop_front();
        k++;
    }
    return k;
}

rx_status rx_serve_drain(rx_server* s, int64_t timeout_ms) {
    if (!s) {
        set_error("rx_serve_drain: null server");
        return RX_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                  [s] { return s->completed == s->submitted; });
    if (!ok) {
        set_error("rx_serve_drain: timed out");
        return RX_ERR_TIMEOUT;
    }
    return RX_OK;
}

rx_status rx_serve_stats(rx_server* s, rx_serve_stats_t* out) {
    if (!s || !out) {
        set_error("rx_serve_stats: null argument");
        return RX_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        auto pct = [&](double q) {
            size_t k = std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        out->p50_ns = pct(0.50);
        out->p99_ns = pct(0.99);
        out->p999_ns = pct(0.999);
        out->max_ns = *std::max_element(v.begin(), v.end());
        double span = (double)(s->t_last - s->t_first) * 1e-9;
        if (span > 0) {
            out->req_per_s = (double)s->completed / span;
            out->gb_per_s = (double)s->bytes_done / span / 1e9;
        }
    }
    out->ticks = s->ticks;
    out->peak_inflight = s->peak_inflight;
    out->peak_device_bytes = s->peak_bytes;
    return RX_OK;
}

rx_status rx_serve_destroy(rx_server* s) {
    if (!s) return RX_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->st) cudaStreamSynchronize(s->st);
    for (int i = 0; i < rx_server::kLongStreams; i++)
        if (s->long_st[i]) cudaStreamSynchronize(s->long_st[i]);
    if (s->copy_st) cudaStreamSynchronize(s->copy_st);
    for (Request* r : s->slots)
        if (r) {
            if (r->owned) cudaFree(r->owned);
            delete r;
        }
    for (Request* r : s->longs) {
        if (r->owned) cudaFree(r->owned);
        if (r->long_ws) cudaFree(r->long_ws);
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
    }
    for (Request* r : s->pending) delete r;
    cudaFree(s->d_slots);
    cudaFree(s->d_order);
    cudaFree(s->d_state);
    cudaFree(s->d_maps);
    cudaFree(s->d_status);
    cudaFreeHost(s->h_slots);
    cudaFreeHost(s->h_order);
    cudaFreeHost(s->h_status);
    if (s->st) cudaStreamDestroy(s->st);
    if (s->copy_st) cudaStreamDestroy(s->copy_st);
    for (int i = 0; i < rx_server::kLongStreams; i++)
        if (s->long_st[i]) cudaStreamDestroy(s->long_st[i]);
    delete s;
    return RX_OK;
}

}  // extern "C"
