// api.cpp -- the C ABI of include/rx.h: handles, device upload, per-stream
// scratch, argument checks and dispatch to the kernels.  No exception
// crosses the boundary: every entry point catches and returns a status.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>

#include "kernels.cuh"
#include "rx_internal.h"

namespace rx {

namespace {
thread_local std::string g_last_error = "no error";

size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

// per-(device, stream) scratch, grown on demand
struct WsKey {
    int dev;
    cudaStream_t st;
    bool operator<(const WsKey& o) const { return dev != o.dev ? dev < o.dev : st < o.st; }
};
std::mutex g_ws_mu;
std::map<WsKey, Workspace> g_ws;

rx_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RX_ERR_CUDA;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

// Scratch of at least `bytes` for this stream (the buffer stays owned by the
// library; callers on the same stream are ordered by the stream).
rx_status get_workspace(cudaStream_t st, size_t bytes, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace& w = g_ws[WsKey{dev, st}];
    if (w.bytes < bytes) {
        if (w.base) {
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(w.base);
            w.base = nullptr;
            w.bytes = 0;
        }
        size_t want = std::max<size_t>(bytes, 1 << 20);
        want = (want + (1 << 20) - 1) & ~size_t((1 << 20) - 1);
        e = cudaMalloc(&w.base, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("scratch allocation failed");
            return RX_ERR_OOM;
        }
        w.bytes = want;
        w.stream = st;
        w.device = dev;
    }
    *out = w.base;
    return RX_OK;
}

static rx_status upload(rx_regex* h) {
    Compiled& C = h->host;
    const int W = C.W;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += a16(b);
        return o;
    };
    size_t o_start = take(W * 4), o_B = take((size_t)256 * W * 4), o_fol = take((size_t)C.nbits * W * 4);
    size_t o_desc = take(256 * sizeof(uint2)), o_tt = take(std::max<size_t>(C.gl_tt.size(), 1) * 4);
    size_t o_T = take(std::max<size_t>(C.memo_T.size(), 1) * 4), o_acc = take(std::max<size_t>(C.memo_acc.size(), 1));
    size_t o_T8 = take(std::max<size_t>(C.memo_T.size(), 1));
    size_t o_imo = take(std::max<size_t>(C.memo_img_off.size(), 1) * 2), o_img = take(std::max<size_t>(C.memo_img.size(), 1));
    size_t o_imp = take(std::max<size_t>(C.memo_imgpos.size(), 1));
    size_t o_sT = take(std::max<size_t>(C.srch_T.size(), 1) * 4);
    size_t o_wT = take(std::max<size_t>(C.wide_T.size(), 1) * 2), o_wacc = take(std::max<size_t>(C.wide_acc.size(), 1));
    size_t o_wio = take(std::max<size_t>(C.wide_img_off.size(), 1) * 4), o_wim = take(std::max<size_t>(C.wide_img.size(), 1) * 2);
    size_t o_wip = take(std::max<size_t>(C.wide_imgpos.size(), 1) * 2);
    size_t o_nd = take(C.nodes.size() * sizeof(int4));
    const int spW = (W <= 4) ? 4 : (W <= 8 ? 8 : 0);
    size_t o_sps = take(spW * 4 + 16), o_spB = take((size_t)256 * spW * 4 + 16),
           o_spF = take((size_t)C.nbits * spW * 4 + 16);
    size_t o_bgp = take(std::max<size_t>(C.bgp_T.size(), 1) * 2);
    size_t o_self = take(sizeof(DevTables));
    size_t total = off;
    std::vector<uint8_t> blob(total, 0);
    auto put = [&](size_t o, const void* p, size_t b) {
        if (b) std::memcpy(blob.data() + o, p, b);
    };
    put(o_start, C.start.data(), W * 4);
    put(o_B, C.B.data(), C.B.size() * 4);
    put(o_fol, C.follow_bit.data(), C.follow_bit.size() * 4);
    put(o_desc, C.gl_desc.data(), 256 * sizeof(uint2));
    put(o_tt, C.gl_tt.data(), C.gl_tt.size() * 4);
    put(o_T, C.memo_T.data(), C.memo_T.size() * 4);
    put(o_sT, C.srch_T.data(), C.srch_T.size() * 4);
    for (size_t i = 0; i < C.memo_T.size(); i++) blob[o_T8 + i] = (uint8_t)(C.memo_T[i] / 256u);  // ids < 192
    put(o_acc, C.memo_acc.data(), C.memo_acc.size());
    put(o_imo, C.memo_img_off.data(), C.memo_img_off.size() * 2);
    put(o_img, C.memo_img.data(), C.memo_img.size());
    put(o_imp, C.memo_imgpos.data(), C.memo_imgpos.size());
    put(o_wT, C.wide_T.data(), C.wide_T.size() * 2);
    put(o_wacc, C.wide_acc.data(), C.wide_acc.size());
    put(o_wio, C.wide_img_off.data(), C.wide_img_off.size() * 4);
    put(o_wim, C.wide_img.data(), C.wide_img.size() * 2);
    put(o_wip, C.wide_imgpos.data(), C.wide_imgpos.size() * 2);
    std::vector<int4> pn(C.nodes.size());
    for (size_t i = 0; i < C.nodes.size(); i++)
        pn[i] = make_int4((int)C.nodes[i].kind | ((int)C.nodes[i].byte << 8), C.nodes[i].l, C.nodes[i].r, C.cont[i]);
    put(o_nd, pn.data(), pn.size() * sizeof(int4));
    put(o_bgp, C.bgp_T.data(), C.bgp_T.size() * 2);
    if (spW) {
        std::vector<uint32_t> ps(spW, 0u), pB((size_t)256 * spW, 0u), pF((size_t)C.nbits * spW, 0u);
        for (int k = 0; k < W; k++) ps[k] = C.start[k];
        for (int r = 0; r < 256; r++)
            for (int k = 0; k < W; k++) pB[(size_t)r * spW + k] = C.B[(size_t)r * W + k];
        for (int r = 0; r < C.nbits; r++)
            for (int k = 0; k < W; k++) pF[(size_t)r * spW + k] = C.follow_bit[(size_t)r * W + k];
        put(o_sps, ps.data(), ps.size() * 4);
        put(o_spB, pB.data(), pB.size() * 4);
        put(o_spF, pF.data(), pF.size() * 4);
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaMalloc(&h->dev_blob, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->dev_blob = nullptr;
        set_error("device allocation for tables failed");
        return RX_ERR_OOM;
    }
    e = cudaMemcpy(h->dev_blob, blob.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy tables");
    h->dev_bytes = (int64_t)total;
    uint8_t* b = static_cast<uint8_t*>(h->dev_blob);
    DevTables& t = h->dev;
    t.m = C.m;
    t.W = W;
    t.nbits = C.nbits;
    t.null_bit = C.null_bit;
    t.start = reinterpret_cast<const uint32_t*>(b + o_start);
    t.B = reinterpret_cast<const uint32_t*>(b + o_B);
    t.follow = reinterpret_cast<const uint32_t*>(b + o_fol);
    t.gl_desc = reinterpret_cast<const uint2*>(b + o_desc);
    t.gl_tt = reinterpret_cast<const uint32_t*>(b + o_tt);
    t.gl_words = C.gl_ok ? (int32_t)C.gl_tt.size() : 0;
    t.sp_W = spW;
    t.sp_start = reinterpret_cast<const uint32_t*>(b + o_sps);
    t.sp_B = reinterpret_cast<const uint32_t*>(b + o_spB);
    t.sp_follow = reinterpret_cast<const uint32_t*>(b + o_spF);
    t.memo_K = C.memo_K;
    t.memo_T = reinterpret_cast<const uint32_t*>(b + o_T);
    t.memo_T8 = b + o_T8;
    t.srch_K = C.srch_K;
    t.srch_T = reinterpret_cast<const uint32_t*>(b + o_sT);
    t.srch_start = C.srch_start;
    t.srch_acc0 = C.srch_acc0;
    t.memo_acc = b + o_acc;
    t.memo_img_off = reinterpret_cast<const uint16_t*>(b + o_imo);
    t.memo_img = b + o_img;
    t.memo_imgpos = b + o_imp;
    t.memo_start = C.memo_start;
    t.wide_K = C.wide_K;
    t.wide_maximg = C.wide_maximg;
    t.wide_T = reinterpret_cast<const uint16_t*>(b + o_wT);
    t.wide_acc = b + o_wacc;
    t.wide_img_off = reinterpret_cast<const uint32_t*>(b + o_wio);
    t.wide_img = reinterpret_cast<const uint16_t*>(b + o_wim);
    t.wide_imgpos = reinterpret_cast<const uint16_t*>(b + o_wip);
    t.wide_start = C.wide_start;
    t.bgp_T = C.bgp_T.empty() ? nullptr : reinterpret_cast<const uint16_t*>(b + o_bgp);
    t.bg_lo = C.bg_lo;
    t.variants = C.variants;
    t.nullable = C.nullable ? 1 : 0;
    t.nn = (int32_t)C.nodes.size();
    t.pnodes = reinterpret_cast<const int4*>(b + o_nd);
    t.proot = 0;
    h->dev_self = reinterpret_cast<const DevTables*>(b + o_self);
    e = cudaMemcpy(b + o_self, &t, sizeof(DevTables), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy table header");
    // the kernels' counter of invalid offsets is looked up once per device,
    // here, so that no later call (possibly under stream capture) does it
    if (!bad_offsets_counter()) {
        set_error("cudaGetSymbolAddress of the invalid-offsets counter failed");
        return RX_ERR_CUDA;
    }
    return RX_OK;
}

static rx_status finish_compile(rx_regex* h, uint32_t flags) {
    if (flags & RX_COMPILE_HOST_ONLY) {
        h->host_only = true;
        return RX_OK;
    }
    return upload(h);
}

bool tuned_choice(const rx_regex* h, int64_t len_hint, int* variant, int* block);

int resolve_variant(const rx_regex* h, int v) {
    if (v != RX_VARIANT_AUTO) return v;
    uint32_t ok = h->host.variants;
    if (ok & (1u << RX_VARIANT_MEMO)) return RX_VARIANT_MEMO;
    if (ok & (1u << RX_VARIANT_THREAD)) return RX_VARIANT_THREAD;
    if (ok & (1u << RX_VARIANT_SPARSE)) return RX_VARIANT_SPARSE;
    return RX_VARIANT_WARP;
}

// The handle's tables live on the device it was compiled on; a kernel on
// another device would be given that device's addresses.
bool on_handle_device(const rx_regex* h, const char* who) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    if (dev == h->device) return true;
    set_error(std::string(who) + ": handle was compiled on device " + std::to_string(h->device) +
              ", current device is " + std::to_string(dev));
    return false;
}

}  // namespace rx

using namespace rx;

// Section 8's machine, one string after another (prior-art comparison; every
// micro-iteration is a launch followed by a flag read-back).
static rx_status match_paper(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                             void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int64_t> off(n + 1);
    cudaError_t e = cudaMemcpyAsync(off.data(), offsets, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match (paper): offsets read-back");
    for (size_t i = 0; i < n; i++)
        if (off[i] < 0 || off[i + 1] < off[i]) {
            set_error("rx_match (paper): invalid offsets at string " + std::to_string(i));
            return RX_ERR_INVALID_ARG;
        }
    size_t need = (2 * (size_t)(h->dev.nn + 1) + 4) * sizeof(int);
    void* ws = nullptr;
    rx_status s = get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    int* hflags = nullptr;
    e = cudaMallocHost(&hflags, 4 * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "rx_match (paper): pinned flags");
    std::vector<uint8_t> res(n);
    for (size_t i = 0; i < n && e == cudaSuccess; i++)
        e = paper_match_one(h->dev, strings + off[i], off[i + 1] - off[i], static_cast<int*>(ws), hflags, &res[i], st);
    cudaFreeHost(hflags);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match (paper) launch");
    e = cudaMemcpyAsync(out, res.data(), n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match (paper): results");
    return RX_OK;
}

extern "C" {

const char* rx_last_error(void) { return g_last_error.c_str(); }

const char* rx_version(void) { return "rx-b300 0.1 (sm_103a)"; }

rx_status rx_compile(const char* pat, size_t len, uint32_t flags, rx_handle* out, size_t* err_pos) {
    RX_GUARD_BEGIN
    if (!out || (!pat && len)) {
        set_error("rx_compile: null argument");
        return RX_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::vector<rx_node> nodes;
    size_t ep = 0;
    std::string msg;
    rx_status s = parse_pattern(pat ? pat : "", len, nodes, ep, msg);
    if (s != RX_OK) {
        if (err_pos) *err_pos = ep;
        set_error(msg);
        return s;
    }
    rx_regex* h = new rx_regex();
    s = compile_tree(nodes.data(), nodes.size(), 0, flags, h->host, msg);
    if (s == RX_OK) s = finish_compile(h, flags);
    else set_error(msg);
    if (s != RX_OK) {
        rx_free(h);
        return s;
    }
    *out = h;
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_compile_ast(const rx_node* nodes, size_t n, int32_t root, uint32_t flags, rx_handle* out) {
    RX_GUARD_BEGIN
    if (!out || !nodes) {
        set_error("rx_compile_ast: null argument");
        return RX_ERR_INVALID_ARG;
    }
    *out = nullptr;
    rx_regex* h = new rx_regex();
    std::string msg;
    rx_status s = compile_tree(nodes, n, root, flags, h->host, msg);
    if (s == RX_OK) s = finish_compile(h, flags);
    else set_error(msg);
    if (s != RX_OK) {
        rx_free(h);
        return s;
    }
    *out = h;
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_info(rx_handle h, rx_info_t* out) {
    if (!h || !out) {
        set_error("rx_info: null argument");
        return RX_ERR_INVALID_ARG;
    }
    out->nodes = (int32_t)h->host.nodes.size();
    out->positions = h->host.m;
    out->words = h->host.W;
    out->nullable = h->host.nullable ? 1 : 0;
    out->memo_states = h->host.memo_K;
    out->variants = h->host.variants;
    out->device_bytes = h->dev_bytes;
    out->search_states = h->host.srch_K;
    out->wide_states = h->host.wide_K;
    return RX_OK;
}

void rx_free(rx_handle h) {
    if (!h) return;
    if (h->dev_blob) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (h->device >= 0 && h->device != cur) cudaSetDevice(h->device);
        cudaFree(h->dev_blob);
        if (h->device >= 0 && h->device != cur && cur >= 0) cudaSetDevice(cur);
    }
    delete h;
}

rx_status rx_tables(rx_handle h, int32_t* cont, int32_t* pos_node, int32_t* pos_bit, int32_t* null_bit,
                    uint32_t* start, uint32_t* follow) {
    if (!h) {
        set_error("rx_tables: null handle");
        return RX_ERR_INVALID_ARG;
    }
    const Compiled& C = h->host;
    if (cont) std::copy(C.cont.begin(), C.cont.end(), cont);
    if (pos_node) std::copy(C.pos_node.begin(), C.pos_node.end(), pos_node);
    if (pos_bit) std::copy(C.pos_bit.begin(), C.pos_bit.end(), pos_bit);
    if (null_bit) *null_bit = C.null_bit;
    if (start) std::copy(C.start.begin(), C.start.end(), start);
    if (follow) std::copy(C.follow_pos.begin(), C.follow_pos.end(), follow);
    return RX_OK;
}

rx_status rx_tree(rx_handle h, rx_node* out, size_t cap, size_t* n) {
    if (!h || !n || (!out && cap)) {
        set_error("rx_tree: null argument");
        return RX_ERR_INVALID_ARG;
    }
    *n = h->host.nodes.size();
    size_t k = std::min(cap, h->host.nodes.size());
    if (k) std::memcpy(out, h->host.nodes.data(), k * sizeof(rx_node));
    return RX_OK;
}

rx_status rx_match_ex(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                      void* stream, const rx_match_opts* opts) {
    RX_GUARD_BEGIN
    if (!h) {
        set_error("rx_match: null handle");
        return RX_ERR_INVALID_ARG;
    }
    if (h->host_only) {
        set_error("rx_match: handle was compiled with RX_COMPILE_HOST_ONLY");
        return RX_ERR_INVALID_ARG;
    }
    if (n == 0) return RX_OK;
    if (!on_handle_device(h, "rx_match")) return RX_ERR_INVALID_ARG;
    if (!offsets || !out) {
        set_error("rx_match: null offsets or out");
        return RX_ERR_INVALID_ARG;
    }
    if (n > 0xffffffffull / 2) {
        set_error("rx_match: more than 2^31 strings");
        return RX_ERR_TOO_LARGE;
    }
    int req = opts ? opts->variant : RX_VARIANT_AUTO;
    int block = opts ? opts->block : 0;
    int variant = RX_VARIANT_AUTO;
    if (req == RX_VARIANT_AUTO) {
        int tv = 0, tb = 0;
        if (tuned_choice(h, opts ? opts->len_hint : 0, &tv, &tb)) {
            variant = tv;
            if (block == 0) block = tb;
        }
    }
    if (variant == RX_VARIANT_AUTO) variant = resolve_variant(h, req);
    if (variant == RX_VARIANT_PAPER) return match_paper(h, n, strings, offsets, out, stream);
    if (variant <= 0 || variant > RX_VARIANT_WARP || !((h->host.variants >> variant) & 1u)) {
        set_error("rx_match: variant " + std::to_string(variant) + " cannot run this expression");
        return RX_ERR_UNSUPPORTED;
    }
    int sort = rx::resolve_sort(variant, opts ? opts->sort : -1, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* ws = nullptr;
    size_t need = match_workspace_bytes(n, sort);
    rx_status s = get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    cudaError_t e = launch_match(h->dev, variant, n, strings, offsets, out, sort, block, ws, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match launch");
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_search(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, int64_t* out_end,
                    void* stream) {
    RX_GUARD_BEGIN
    if (!h || h->host_only || (n > 0 && (!offsets || !out_end))) {
        set_error("rx_search: bad argument");
        return RX_ERR_INVALID_ARG;
    }
    if (n == 0) return RX_OK;
    if (h->dev.srch_K <= 0) {
        set_error("rx_search: no search cache (compile with RX_COMPILE_SEARCH; at most 192 states)");
        return RX_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* ws = nullptr;
    const size_t need = rx::search_workspace_bytes(n);
    rx_status s = get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    cudaError_t e = rx::launch_search(h->dev, n, strings, offsets, out_end, ws, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_search launch");
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_search_long(rx_handle h, const uint8_t* str, int64_t len, int64_t chunk_bytes, int64_t* out_end,
                         void* stream) {
    RX_GUARD_BEGIN
    if (!h || h->host_only || !out_end || len < 0 || (len > 0 && !str) || chunk_bytes < 0 ||
        (chunk_bytes > 0 && chunk_bytes < 64)) {
        set_error("rx_search_long: bad argument (chunk_bytes 0 or >= 64)");
        return RX_ERR_INVALID_ARG;
    }
    if (h->dev.srch_K <= 0) {
        set_error("rx_search_long: no search cache (compile with RX_COMPILE_SEARCH; at most 192 states)");
        return RX_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t C = chunk_bytes > 0 ? chunk_bytes : rx::search_long_chunk_auto(h->dev, len);
    const size_t need = rx::search_long_workspace_bytes(h->dev, len, C);
    if (need > (size_t(16) << 30)) {
        set_error("rx_search_long: chunk size too small for this length (tables exceed 16 GiB)");
        return RX_ERR_TOO_LARGE;
    }
    void* ws = nullptr;
    rx_status s = get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    cudaError_t e = rx::launch_search_long(h->dev, str, len, C, out_end, ws, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_search_long launch");
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_sync_check(void* stream, int64_t* bad_strings) {
    RX_GUARD_BEGIN
    if (bad_strings) *bad_strings = 0;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rx_sync_check: stream synchronisation");
    const unsigned long long bad = rx::read_bad_offsets(true);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rx_sync_check: counter read");
    if (bad_strings) *bad_strings = (int64_t)bad;
    if (bad) {
        set_error("rx_sync_check: " + std::to_string(bad) +
                  " string(s) with invalid offsets (offsets[i] < 0 or offsets[i+1] < offsets[i]); "
                  "their results hold RX_RESULT_INVALID / RX_SEARCH_INVALID");
        return RX_ERR_INVALID_ARG;
    }
    return RX_OK;
    RX_GUARD_END
}

int64_t rx_device_faults(int32_t reset) {
    cudaDeviceSynchronize();
    return (int64_t)rx::read_wait_faults(reset != 0) + (int64_t)rx::read_plan_faults(reset != 0);
}

rx_status rx_match(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                   void* stream) {
    return rx_match_ex(h, n, strings, offsets, out, stream, nullptr);
}

rx_status rx_trace(rx_handle h, const uint8_t* str, int64_t len, uint32_t* frontiers, void* stream) {
    RX_GUARD_BEGIN
    if (!h || h->host_only || !frontiers || len < 0 || (len > 0 && !str)) {
        set_error("rx_trace: bad argument");
        return RX_ERR_INVALID_ARG;
    }
    cudaError_t e = launch_trace(h->dev, str, len, frontiers, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rx_trace launch");
    return RX_OK;
    RX_GUARD_END
}

}  // extern "C"

namespace rx {
rx_status get_workspace(cudaStream_t st, size_t bytes, void** out);
}

extern "C" {

rx_status rx_match_pairs(const rx_handle* handles, size_t n, const uint8_t* strings, const int64_t* offsets,
                         uint8_t* out, void* stream) {
    RX_GUARD_BEGIN
    if (n == 0) return RX_OK;
    if (!handles || !offsets || !out) {
        rx::set_error("rx_match_pairs: null argument");
        return RX_ERR_INVALID_ARG;
    }
    rx_match_opts o{RX_VARIANT_AUTO, 0, 0, 0};
    for (size_t i = 0; i < n; i++) {
        rx_status s = rx_match_ex(handles[i], 1, strings, offsets + i, out + i, stream, &o);
        if (s != RX_OK) return s;
    }
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_match_seq(rx_handle h, const uint8_t* str, int64_t len, uint8_t* out, void* stream) {
    RX_GUARD_BEGIN
    if (!h || h->host_only || !out || len < 0 || (len > 0 && !str)) {
        rx::set_error("rx_match_seq: bad argument");
        return RX_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int variant = rx::resolve_variant(h, RX_VARIANT_AUTO);
    if (variant == RX_VARIANT_WARP) variant = RX_VARIANT_WARP;
    size_t need = rx::match_workspace_bytes(1, 0) + 256;
    void* ws = nullptr;
    rx_status s = rx::get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    int64_t* off = reinterpret_cast<int64_t*>(static_cast<uint8_t*>(ws) + rx::match_workspace_bytes(1, 0));
    cudaError_t e = rx::launch_fill_offsets(off, len, st);
    if (e == cudaSuccess)
        e = rx::launch_match(h->dev, variant, 1, str, off, out, 0, 32, ws, rx::match_workspace_bytes(1, 0), st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match_seq launch");
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_profile_enable(int on) {
    rx::prof_enable(on != 0);
    return RX_OK;
}

rx_status rx_profile_read(int64_t* launches, int64_t* timed, double* kernel_ms) {
    cudaError_t e = rx::prof_read(launches, timed, kernel_ms);
    if (e != cudaSuccess) return cuda_fail(e, "rx_profile_read");
    return RX_OK;
}

// class of a handle in the batched kernel (the variant it runs there)
static int batch_class(const rx_regex* h) {
    const Compiled& C = h->host;
    if (C.memo_K > 0) return rx::kClsMemo;
    if (C.wide_K > 0) return rx::kClsWide;
    if (C.gl_ok) return C.W == 1 ? rx::kClsThread1 : rx::kClsThread2;
    if (C.W <= 4) return rx::kClsSparse4;
    if (C.W <= 8) return rx::kClsSparse8;
    return rx::kClsWarp;
}

}  // extern "C"

namespace rx {
// Distinct tables of the pairs' expressions, the table index and the class
// of every pair (host arrays for the batched kernel).
rx_status collect_pairs(const rx_handle* handles, size_t n, const char* who, std::vector<BatchTab>& tabs,
                        std::vector<uint32_t>& pair_tab, std::vector<uint8_t>& cls) {
    if (n > 0x7fffffffull) {
        set_error(std::string(who) + ": more than 2^31 pairs");
        return RX_ERR_TOO_LARGE;
    }
    std::unordered_map<const rx_regex*, uint32_t> index;
    std::vector<uint8_t> tab_cls;
    pair_tab.resize(n);
    cls.resize(n);
    const rx_regex* last = nullptr;
    uint32_t last_i = 0;
    for (size_t i = 0; i < n; i++) {
        const rx_regex* h = handles[i];
        if (h != last) {
            if (!h || h->host_only) {
                set_error(std::string(who) + ": null or host-only handle at pair " + std::to_string(i));
                return RX_ERR_INVALID_ARG;
            }
            auto it = index.find(h);
            if (it == index.end()) {
                it = index.emplace(h, (uint32_t)tabs.size()).first;
                BatchTab bt;
                bt.t = h->dev;
                tabs.push_back(bt);
                tab_cls.push_back((uint8_t)batch_class(h));
            }
            last = h;
            last_i = it->second;
        }
        pair_tab[i] = last_i;
        cls[i] = tab_cls[last_i];
    }
    return RX_OK;
}
}  // namespace rx

extern "C" {

rx_status rx_match_batch(const rx_handle* handles, size_t n, const uint8_t* strings, const int64_t* offsets,
                         uint8_t* out, void* stream) {
    RX_GUARD_BEGIN
    if (n == 0) return RX_OK;
    if (!handles || !offsets || !out) {
        rx::set_error("rx_match_batch: null argument");
        return RX_ERR_INVALID_ARG;
    }
    std::vector<rx::BatchTab> tabs;
    std::vector<uint32_t> pair_tab;
    std::vector<uint8_t> cls;
    rx_status s = rx::collect_pairs(handles, n, "rx_match_batch", tabs, pair_tab, cls);
    if (s != RX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rx::BatchLaunch L;
    L.stride = rx::batch_stride(tabs.data(), tabs.size());
    cudaError_t e = rx::batch_configure(L);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match_batch configure");
    rx::BatchPlan P;
    P.n = n;
    P.ntabs = tabs.size();
    const size_t maps = rx::batch_maps_bytes(L, n);
    const size_t need = rx::batch_plan_bytes(P, maps);
    void* ws = nullptr;
    s = rx::get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    rx::batch_plan_place(P, maps, ws);
    e = rx::batch_plan_upload(P, tabs.data(), pair_tab.data(), cls.data(), st);
    if (e == cudaSuccess) e = rx::batch_run(P, strings, offsets, out, L, st, true);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match_batch launch");
    return RX_OK;
    RX_GUARD_END
}

rx_status rx_match_long(rx_handle h, const uint8_t* str, int64_t len, int64_t chunk_bytes, uint8_t* out,
                        void* stream) {
    RX_GUARD_BEGIN
    if (!h || h->host_only || !out || len < 0 || (len > 0 && !str) || chunk_bytes < 0 ||
        chunk_bytes >= (int64_t(1) << 32) - 32) {
        rx::set_error("rx_match_long: bad argument (chunk_bytes 0 or in [1, 2^32 - 32))");
        return RX_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!rx::long_supported(h->dev)) return rx_match_seq(h, str, len, out, stream);
    int64_t C = chunk_bytes > 0 ? chunk_bytes : rx::long_chunk_auto(h->dev, len);
    size_t need = rx::long_workspace_bytes(h->dev, len, C);
    if (need > (size_t(16) << 30)) {
        rx::set_error("rx_match_long: chunk size too small for this length (transfer tables exceed 16 GiB)");
        return RX_ERR_TOO_LARGE;
    }
    void* ws = nullptr;
    rx_status s = rx::get_workspace(st, need, &ws);
    if (s != RX_OK) return s;
    cudaError_t e = rx::launch_long(h->dev, str, len, C, out, ws, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "rx_match_long launch");
    return RX_OK;
    RX_GUARD_END
}

}  // extern "C"
