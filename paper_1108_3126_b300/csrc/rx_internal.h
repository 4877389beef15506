// rx_internal.h -- shared declarations of the host compiler, the kernels and
// the C ABI layer.  Not installed; include/rx.h is the public surface.
#pragma once

#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rx.h"

namespace rx {

// Largest macro-step cache kept: rows of 256 x u32 must fit in shared memory.
constexpr int kMemoMaxStates = 192;
// Wide tier: a larger cache with two-byte state ids, for expressions whose
// reachable sets outgrow the one above (global-memory tables, read by the
// warp-chunked form).  Kept only when every byte's column image holds at
// most kWideMaxImg states (a chunk function row is then 4 + 2 * n bytes,
// within the serving slots' 208-byte rows) and the build stays within
// kWideMaxWork word operations.
constexpr int kWideMaxStates = 4096;
constexpr int kWideMaxImg = 100;
constexpr long long kWideMaxWork = 200000000;
// Largest group of same-byte positions one thread-variant lookup covers.
constexpr int kGroupMaxBits = 8;
// Largest cache for which the two-byte rows are built (2.5 KB per state).
constexpr int kPairMaxStates = 64;
// Widest active set per thread for the sparse thread variant (32-bit words).
constexpr int kSparseMaxWords = 8;
// Widest active set per warp for the warp variant (lane-owned words).
constexpr int kWarpMaxWords = 128;

// Tables of one compiled expression as the kernels see them (device
// pointers into one allocation).  Passed by value to kernels.
struct DevTables {
    int32_t m;         // positions (CHAR leaves)
    int32_t W;         // 32-bit words per active set
    int32_t nbits;     // bits used (positions + padding + null)
    int32_t null_bit;  // bit index of null
    const uint32_t* start;   // [W]        evolution of {root}
    const uint32_t* B;       // [256*W]    positions labelled c
    const uint32_t* follow;  // [nbits*W]  evolution of {cont p} by bit of p
    // thread variant: one lookup per byte into a per-byte subset table
    const uint2* gl_desc;    // [256] x = shift | word<<5 | mask<<8, y = word offset of the byte's table
    const uint32_t* gl_tt;   // tables, W words per entry
    int32_t gl_words;        // words in gl_tt (0: variant unavailable)
    // sparse variant: the same tables with rows padded to sp_W (4 or 8) words
    int32_t sp_W;            // 0: W > 8
    const uint32_t* sp_start;
    const uint32_t* sp_B;
    const uint32_t* sp_follow;
    // macro-step cache
    int32_t memo_K;          // states (0: unavailable); state 0 is the empty set
    const uint32_t* memo_T;  // [K*256] next state * 256 (row start, in words)
    const uint8_t* memo_T8;  // [K*256] next state id (the same table, one byte per entry, for global reads)
    const uint8_t* memo_acc; // [K] 1 iff the state's set holds null
    // image of each byte's column of the cache: the distinct successor ids
    // of byte c, ascending, are memo_img[memo_img_off[c] .. memo_img_off[c+1])
    // (state 0, the empty set, is always among them: it stays empty)
    const uint16_t* memo_img_off;  // [257]
    const uint8_t* memo_img;
    const uint8_t* memo_imgpos;    // [256*K] entry c*K + k: index of T[k][c] in the image of c
    uint32_t memo_start;     // start state * 256
    // wide tier (memo_K == 0 only): ids in two bytes, same layout otherwise
    int32_t wide_K;          // states (0: unavailable); state 0 is the empty set
    int32_t wide_maximg;     // largest column image
    const uint16_t* wide_T;  // [K*256] next state id
    const uint8_t* wide_acc; // [K]
    const uint32_t* wide_img_off;  // [257]
    const uint16_t* wide_img;
    const uint16_t* wide_imgpos;   // [256*K]
    uint32_t wide_start;     // start state id
    // cache for unanchored search (start set added after every byte);
    // states >= srch_acc0 hold null (a match ends there)
    int32_t srch_K;          // 0: unavailable
    const uint32_t* srch_T;  // [K*256] next state * 256
    uint32_t srch_start;     // start state * 256
    int32_t srch_acc0;
    // two-byte cache, for labels inside one 32-value window [bg_lo, bg_lo+32),
    // in planes of 8 states: plane p = s / 8 holds 32 pair rows of 516
    // bytes (512 + a pad) then 8 rows of 512; pair row j holds, for slot
    // q = s % 8 at byte 64q, the 32 successors after bytes (lo+i, lo+j);
    // the single rows hold the 256 byte successors (c at single row c/32,
    // entry c % 32).  Entries are the successor's shared-memory offset / 64
    // (plane * 322 + slot), so a lookup is (state offset) + 2 * i + 516 * j
    const uint16_t* bgp_T;   // [ceil(K/8) * 10304], 0 = unavailable
    int32_t bg_lo;
    uint32_t variants;       // bit v: rx_variant v can run
    int32_t nullable;
    // the paper's own machine (Section 8): node array + cont
    int32_t nn;              // nodes in the flattened tree
    const int4* pnodes;      // [nn] x = kind | byte<<8, y = l, z = r, w = cont (-1 = null)
    int32_t proot;
};

// Host-side compiled expression.
struct Compiled {
    // tree (renumbered: preorder from the root, root = 0)
    std::vector<rx_node> nodes;
    std::vector<int32_t> orig_id;  // new id -> caller's id
    std::vector<int32_t> cont;     // Def 4.4, -1 = null (new ids)
    int m = 0;
    std::vector<int32_t> pos_node;  // canonical position (left-to-right) -> new node id
    std::vector<int32_t> pos_bit;   // canonical position -> bit index
    int nbits = 0, W = 0, null_bit = 0;
    bool nullable = false;
    std::vector<uint32_t> start;       // W
    std::vector<uint32_t> follow_pos;  // m*W, canonical position order
    std::vector<uint32_t> follow_bit;  // nbits*W, by bit
    std::vector<uint32_t> B;           // 256*W
    // thread variant
    bool gl_ok = false;
    std::vector<uint2> gl_desc;  // 256
    std::vector<uint32_t> gl_tt;
    // cache of macro steps
    int memo_K = 0;
    std::vector<uint32_t> memo_T;  // K*256
    int srch_K = 0, srch_acc0 = 0;  // search cache (see DevTables::srch_T)
    uint32_t srch_start = 0;
    std::vector<uint32_t> srch_T;
    std::vector<uint8_t> memo_acc;
    std::vector<uint16_t> memo_img_off;  // 257 (see DevTables::memo_img)
    std::vector<uint8_t> memo_img;
    std::vector<uint8_t> memo_imgpos;    // K*256
    uint32_t memo_start = 0;
    // wide tier (see DevTables::wide_T)
    int wide_K = 0, wide_maximg = 0;
    uint32_t wide_start = 0;
    std::vector<uint16_t> wide_T;
    std::vector<uint8_t> wide_acc;
    std::vector<uint32_t> wide_img_off;
    std::vector<uint16_t> wide_img;
    std::vector<uint16_t> wide_imgpos;
    // two-byte cache: per state a row of 1024 pair successors (entry
    // 32*j + i after bytes lo+i, lo+j) then 256 byte successors, u16 ids
    // (host only; the device gets the planes below)
    std::vector<uint16_t> bg_T;
    std::vector<uint16_t> bgp_T;  // planes layout (see DevTables::bgp_T)
    int bg_lo = -1;
    uint32_t variants = 0;
};

// Compile a tree (caller ids).  Returns RX_OK or an error with msg set.
rx_status compile_tree(const rx_node* nodes, size_t n, int32_t root, uint32_t flags, Compiled& out,
                       std::string& msg);
// Parse pattern text into a node array (root = 0).
rx_status parse_pattern(const char* pat, size_t len, std::vector<rx_node>& nodes, size_t& err_pos,
                        std::string& msg);

void set_error(const std::string& msg);

}  // namespace rx

// Body of every extern "C" entry point: no C++ exception leaves the ABI
// (an allocation failure is RX_ERR_OOM, anything else an internal error).
#define RX_GUARD_BEGIN try {
#define RX_GUARD_END                                      \
    }                                                     \
    catch (const std::bad_alloc&) {                       \
        rx::set_error("host allocation failed");          \
        return RX_ERR_OOM;                                \
    }                                                     \
    catch (const std::exception& ex) {                    \
        rx::set_error(std::string("internal: ") + ex.what()); \
        return RX_ERR_INVALID_ARG;                        \
    }                                                     \
    catch (...) {                                         \
        rx::set_error("internal error");                  \
        return RX_ERR_INVALID_ARG;                        \
    }

struct rx_regex {
    rx::Compiled host;
    rx::DevTables dev{};
    const rx::DevTables* dev_self = nullptr;  // device copy of `dev` (inside dev_blob)
    void* dev_blob = nullptr;
    int64_t dev_bytes = 0;
    int device = -1;
    bool host_only = false;
};
