/*
 * rx.h -- C ABI of the B300 lockstep regular-expression matcher.
 *
 * The library decides whole-string membership  e |v w  (Rathnayake &
 * Thielecke, "Regular Expression Matching and Operational Semantics",
 * SOS 2011, Section 2, Fig 2.1) for expressions over the byte alphabet
 *     e ::= eps | a | e* | e1 e2 | e1 | e2          (Section 2)
 * by the lockstep construction of Section 5: the expression is laid out as a
 * pointer tree with continuation pointers (Section 4, Defs 4.1-4.4), every
 * input byte advances the whole set of active tree positions at once
 * (Def 5.2), and the evolution of Def 5.1 is deduplicated by node identity
 * (pointer equality, Section 3).  A string is accepted when null is in the
 * evolved set after the last byte (Def 5.3).
 *
 * Conventions for every entry point:
 *   - No C++ exception crosses this boundary; every call that can fail
 *     returns an rx_status, and rx_last_error() returns a thread-local
 *     message describing the most recent failure on the calling thread.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary (pageable or pinned) memory.
 *   - Streams are cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls marked "async" only enqueue work on that stream; the
 *     caller synchronises before reading results.
 *   - Handles are owned by the library and released with rx_free(); all
 *     other buffers are owned by the caller.
 *   - Threads: handles may be shared by threads for matching.  Calls that
 *     use the library's per-stream scratch (rx_match*, rx_search*,
 *     rx_match_batch, rx_match_long) may run concurrently on different
 *     streams; calls on one stream from several host threads must be
 *     serialised by the caller (the scratch can be regrown between them).
 *     rx_match_host serialises itself per device.
 */
#ifndef RX_H
#define RX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- basic types */
typedef enum {
    RX_OK = 0,
    RX_ERR_PARSE = 1,        /* pattern text is not in the syntax below        */
    RX_ERR_INVALID_ARG = 2,  /* null pointer, bad size, malformed tree/offsets */
    RX_ERR_TOO_LARGE = 3,    /* more nodes/positions than the limits below     */
    RX_ERR_OOM = 4,          /* host or device allocation failed               */
    RX_ERR_CUDA = 5,         /* a CUDA runtime call failed                     */
    RX_ERR_TIMEOUT = 6,      /* a bounded device or host wait gave up          */
    RX_ERR_BUSY = 7,         /* serving queue full; retry after rx_serve_poll   */
    RX_ERR_UNSUPPORTED = 8   /* the requested variant cannot run this handle   */
} rx_status;

/* Node kinds of the abstract syntax of Section 2. */
enum { RX_CHAR = 0, RX_EPS = 1, RX_STAR = 2, RX_CAT = 3, RX_ALT = 4 };

/* One node of the heap pi of Section 4 (Def 4.3): kind, the byte of a CHAR
 * node, and child indices l, r (-1 when absent: CHAR/EPS have none, STAR has
 * only l).  12 bytes, little-endian, no padding beyond `pad`. */
typedef struct {
    uint8_t kind;
    uint8_t byte;
    uint16_t pad;
    int32_t l;
    int32_t r;
} rx_node;

typedef struct rx_regex* rx_handle;

/* Limits.  Positions are the CHAR leaves of the tree (the elements the
 * active set ranges over); the active set has positions+1 bits (null). */
#define RX_MAX_NODES 65536
#define RX_MAX_POSITIONS 4095

/* Kernel variants (see rx_match_ex).  AUTO lets the library choose. */
typedef enum {
    RX_VARIANT_AUTO = 0,
    RX_VARIANT_MEMO = 1,   /* cached macro steps: one table lookup per byte      */
    RX_VARIANT_THREAD = 2, /* one thread per string, register bitset (<= 63 pos) */
    RX_VARIANT_SPARSE = 3, /* one thread per string, bitset words + follow rows  */
    RX_VARIANT_WARP = 4,   /* one warp per string, lane-owned bitset words; for
                              an expression with the wide cache tier, 32 chunk
                              functions on it instead                           */
    RX_VARIANT_PAPER = 5   /* Section 8's machine: one thread per node, c/n
                              stamp vectors, one launch per micro-step          */
} rx_variant;

/* compile flags */
#define RX_COMPILE_HOST_ONLY 1u /* build host tables only; the handle cannot be
                                   matched (used to inspect the compiler)  */
#define RX_COMPILE_NO_MEMO 2u   /* do not build the macro-step cache       */
#define RX_COMPILE_SEARCH 4u    /* also build the search cache (rx_search)  */
#define RX_COMPILE_NO_WIDE 8u   /* do not build the wide cache tier        */

typedef struct {
    int32_t nodes;        /* nodes reachable from the root                  */
    int32_t positions;    /* m: CHAR leaves                                  */
    int32_t words;        /* 32-bit words of the active-set bitset           */
    int32_t nullable;     /* 1 iff the expression matches the empty string   */
    int32_t memo_states;  /* cached macro-step states, 0 if no cache         */
    uint32_t variants;    /* bit v set iff rx_variant v can run this handle  */
    int64_t device_bytes; /* device memory held by the handle                */
    int32_t search_states; /* search cache size (0: none; RX_COMPILE_SEARCH) */
    int32_t wide_states;  /* wide cache tier size: sets of more than 256
                             positions whose cache outgrows memo_states' 192
                             (up to 4096 states, two-byte ids); 0 if none */
} rx_info_t;

/* --------------------------------------------------------------- compiling */
/*
 * rx_compile -- parse pattern text into the pointer tree of Section 4, wire
 * cont (Def 4.4), precompute the evolutions of Def 5.1 (one depth-first walk
 * per continuation target, deduplicated by node id), build the per-byte
 * successor tables of Def 5.2, and upload them to the current device.
 *
 * Text syntax (the paper fixes none): '|' binds loosest, then juxtaposition,
 * then postfix '*'; both binary operators associate to the left.
 * Parentheses group; an empty alternative or "()" is eps, as is "\e".
 * "\xHH" is the byte 0xHH; "\" before any other byte is that byte literally
 * (so "\|", "\*", "\(", "\)", "\\").  Every other byte stands for itself.
 *
 *   pat      host, len bytes (need not be NUL-terminated)
 *   flags    RX_COMPILE_* bits
 *   out      receives the handle (library-owned; release with rx_free)
 *   err_pos  optional; on RX_ERR_PARSE receives the byte offset of the error
 * Errors: RX_ERR_PARSE, RX_ERR_TOO_LARGE (limits above), RX_ERR_OOM,
 * RX_ERR_CUDA.  On error *out is set to NULL.
 */
rx_status rx_compile(const char* pat, size_t len, uint32_t flags, rx_handle* out, size_t* err_pos);

/*
 * rx_compile_ast -- as rx_compile, from a node array (host).  The tree is
 * the part reachable from `root`; it must be a tree (no node reachable
 * twice, no cycles: the disjointness of Def 4.3) with valid child indices.
 * Nodes not reachable from the root are ignored.
 * Errors: RX_ERR_INVALID_ARG for malformed trees, otherwise as rx_compile.
 */
rx_status rx_compile_ast(const rx_node* nodes, size_t n, int32_t root, uint32_t flags, rx_handle* out);

/* rx_info -- sizes of a compiled handle.  Errors: RX_ERR_INVALID_ARG. */
rx_status rx_info(rx_handle h, rx_info_t* out);

/* rx_free -- release a handle and its device tables (NULL is ignored).
 * The caller must ensure no enqueued work still uses the handle. */
void rx_free(rx_handle h);

/*
 * rx_tables -- host copies of the compiled tables, for inspection.  Any
 * output pointer may be NULL.  Bit b of an active set is word b/32, bit b%32.
 *   cont      [nodes]        cont of each node (Def 4.4), -1 = null, indexed
 *                            by the preorder ids of rx_tree
 *   pos_node  [positions]    preorder id of each position, left-to-right order
 *   pos_bit   [positions]    bitset index of each position
 *   null_bit                 bitset index of null
 *   start     [words]        evolution of {root} (Def 5.1, with null)
 *   follow    [positions*words] evolution of {cont p} for position p
 *                            (left-to-right order), with null
 * Errors: RX_ERR_INVALID_ARG.
 */
rx_status rx_tables(rx_handle h, int32_t* cont, int32_t* pos_node, int32_t* pos_bit, int32_t* null_bit,
                    uint32_t* start, uint32_t* follow);

/*
 * rx_tree -- the tree a handle was compiled from, renumbered in preorder
 * (root = node 0; for rx_compile this is the parsed pattern).  Writes up
 * to cap nodes to out (host) and the node count to *n.
 * Errors: RX_ERR_INVALID_ARG.
 */
rx_status rx_tree(rx_handle h, rx_node* out, size_t cap, size_t* n);

/* ---------------------------------------------------------------- matching */
/*
 * Device offsets.  String i of a device batch is strings[offsets[i] ..
 * offsets[i+1]) (the w of the problem e |v w, Section 2).  The kernels check
 * every pair: it is valid iff 0 <= offsets[i] <= offsets[i+1].  A string
 * with an invalid pair is not read at all; its result is the marker
 * RX_RESULT_INVALID (RX_SEARCH_INVALID for rx_search) and it is counted on
 * the device, and rx_sync_check() returns RX_ERR_INVALID_ARG for it.  The
 * size of the strings buffer is not passed, so offsets[n] <= that size is
 * the caller's to guarantee.  (rx_match_host checks its host offsets before
 * any copy and returns RX_ERR_INVALID_ARG directly.)
 */
#define RX_RESULT_INVALID 2
#define RX_SEARCH_INVALID (-2)

/*
 * rx_sync_check -- synchronise `stream`, then read and clear the count of
 * strings with invalid offsets (see above) that the kernels of any call on
 * the current device have met since the last rx_sync_check.  The count is
 * kept per device, not per stream or call: work still running on other
 * streams may add to it.  *bad_strings (optional) receives the count.
 * The paper has no counterpart (it concerns only the encoding of a batch).
 * Errors: RX_ERR_INVALID_ARG when the count is > 0; RX_ERR_CUDA.
 */
rx_status rx_sync_check(void* stream, int64_t* bad_strings);

/*
 * rx_match -- one expression against n strings (async).  out[i] = 1 iff
 * e |v w_i (Def 5.3: null in the evolved set after the last byte), else 0,
 * where w_i = strings[offsets[i] .. offsets[i+1]); RX_RESULT_INVALID for a
 * string whose offsets are invalid (see "Device offsets").
 *   strings  device, offsets[n] bytes, packed
 *   offsets  device, n+1 int64, non-decreasing, offsets[0] >= 0
 *   out      device, n bytes
 *   h        compiled on the current device
 * The input bytes are read once; a string whose active set empties is not
 * read further (it is stuck, Fig 6.1).  Scratch space is library-owned per
 * stream and grows on demand (may synchronise the stream the first time a
 * larger batch is seen).
 * Errors: RX_ERR_INVALID_ARG (NULL pointers with n > 0, host-only handle,
 * handle compiled on another device), RX_ERR_OOM, RX_ERR_CUDA (launch
 * failure).  Invalid offsets are reported by rx_sync_check.
 */
rx_status rx_match(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                   void* stream);

typedef struct {
    int32_t variant;    /* rx_variant; AUTO = tuned or library choice        */
    int32_t block;      /* threads per block, 0 = tuned or default; for the
                           cache of macro steps an odd value selects the
                           one-byte-per-lookup kernel (block - 1 threads)    */
    int32_t sort;       /* -1 = auto, 0 = input order, 1 = length order +
                           per-variant kernel, 2 = length order + streaming
                           kernel, 3 = streaming kernel in input order, 4 =
                           streaming kernel with a length order per block
                           (one launch, no planner; memo variant with the
                           two-byte cache, else as 2).  Auto: 4 for the memo
                           variant and 2 for the thread variant from 4096
                           strings, 3 below; 1 / 0 for the others          */
    int32_t len_hint;   /* mean string length if known (selects the tuned
                           entry of that length bucket), 0 = unknown         */
} rx_match_opts;

/* rx_match_ex -- rx_match with an explicit variant / launch shape.
 * Errors: as rx_match, plus RX_ERR_UNSUPPORTED when the variant cannot run
 * this handle (see rx_info_t.variants). */
rx_status rx_match_ex(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                      void* stream, const rx_match_opts* opts);

/*
 * rx_match_static -- rx_match for callers that cannot let the library
 * allocate device memory.  (The paper has no counterpart: this concerns
 * only how scratch space is obtained.)  rx_match grows a per-stream scratch
 * buffer with cudaMalloc, after synchronising the stream and freeing the old
 * buffer, whenever it meets a larger batch; a caller that must not block on
 * the device, or whose device-memory budget is fixed in advance, cannot
 * accept that.  rx_match_static runs the same planner and kernels with its
 * scratch in one fixed 4 MiB array compiled into the library: every GPU that
 * loads the library holds that array until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   Arguments, layout and result: as rx_match (async on `stream`); the
 *   offsets are checked the same way (RX_RESULT_INVALID, rx_sync_check).
 *   The handle must have been compiled on the current device (else
 *   RX_ERR_INVALID_ARG).
 *   Limit: at most 262,144 strings per call; larger n returns
 *   RX_ERR_TOO_LARGE with nothing launched.
 *   The first call on a device looks up the array's device address with
 *   that device current; make that first call before any stream capture.
 *   Every call shares the one array (the work counter is cleared by each
 *   call; the rest keeps the last call's contents): calls that overlap on
 *   the GPU -- on different streams, or from different threads -- race and
 *   must be serialised by the caller.
 * Errors: RX_ERR_INVALID_ARG, RX_ERR_TOO_LARGE, RX_ERR_CUDA.
 */
rx_status rx_match_static(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                          void* stream);

/*
 * rx_match_host -- rx_match on HOST buffers (synchronous).  Decides, for
 * every string, whether the expression matches it (Def 5.3) exactly as
 * rx_match does; the paper has no counterpart for the transfer, which
 * concerns only where the input lives.
 *   strings  host bytes, offsets host int64[n+1] (non-decreasing, >= 0),
 *   out      host uint8[n]: 1 = match, 0 = no match.
 * The batch is cut at string boundaries into pieces of up to 64 MiB (or
 * 2^20 strings; a longer single string is one piece); piece k is copied to
 * the device on an internal stream while piece k-1 is matched on `stream`,
 * and each piece's booleans are copied back on `stream`.  Host buffers in
 * page-locked memory (cudaHostAlloc / pin_memory) let the copies run at
 * full link speed; pageable buffers work but are staged by the driver.
 * Device scratch: two staging buffers of the largest piece plus the
 * planner's workspace, from the per-stream scratch buffer rx_match uses.
 * Returns when `out` is written (the stream is synchronised).
 * Each piece's offsets are checked just before its copy is queued, so the
 * checks overlap the copies of earlier pieces.
 * Errors: RX_ERR_INVALID_ARG (null handle/pointer, decreasing or negative
 * offsets: the pieces before the first bad one may already have their
 * booleans in `out`, the rest of `out` is untouched), RX_ERR_OOM,
 * RX_ERR_CUDA.
 */
rx_status rx_match_host(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                        void* stream);

/*
 * rx_search -- unanchored search (async).  Not in the paper, which decides
 * whole-string membership only: out_end[i] = the smallest j such that some
 * substring w[i0..j) of string i (i0 <= j) is matched by the expression
 * (e |v w[i0..j), Fig 2.1), or -1 when no substring matches; a nullable
 * expression gives 0.  Computed by the lockstep machine with the start set
 * added back after every byte (Defs 5.1-5.3 on the Sigma* e machine), as a
 * cache of macro steps built when the handle is compiled with
 * RX_COMPILE_SEARCH (at most 192 states).
 *   strings/offsets as in rx_match; out_end DEVICE int64[n]
 *   (RX_SEARCH_INVALID for a string with invalid offsets).
 * Errors: RX_ERR_INVALID_ARG, RX_ERR_UNSUPPORTED (no search cache: flag
 * missing, or the cache would exceed 192 states), RX_ERR_OOM, RX_ERR_CUDA.
 */
rx_status rx_search(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, int64_t* out_end,
                    void* stream);

/*
 * rx_search_long -- rx_search on one long string, chunked (async).  Over the
 * search cache, each chunk's effect on an incoming state is a pair (state at
 * the chunk's end, end offset of its first accepting byte or none); pairs
 * compose associatively, so chunks are computed in parallel and composed
 * left to right, exactly as the one-string answer.
 *   str DEVICE bytes [len]; chunk_bytes 0 = automatic, else >= 64;
 *   out_end DEVICE int64[1] = earliest end of a matching substring, -1 if none.
 * Errors: RX_ERR_INVALID_ARG, RX_ERR_UNSUPPORTED (no search cache),
 * RX_ERR_TOO_LARGE (chunk size too small for this length), RX_ERR_OOM,
 * RX_ERR_CUDA.
 */
rx_status rx_search_long(rx_handle h, const uint8_t* str, int64_t len, int64_t chunk_bytes, int64_t* out_end,
                         void* stream);

/*
 * rx_device_faults -- bounded device-side waits that gave up, counted on
 * the current device since the last reset (the streaming kernel that stages
 * input with bulk copies counts one per warp that stopped waiting for a
 * stage; that warp's strings of the round are left unwritten; the
 * one-launch length planner counts one per block that stopped waiting at
 * its grid barrier, whose strings then keep their input order; the
 * block-local streaming kernel, in its form whose two-byte cache holds
 * 16-bit shared addresses, counts one per block whose shared memory starts
 * too high for them, a layout the host check rules out; that block's
 * strings get RX_RESULT_INVALID).  0 in normal operation.  reset != 0 clears the counter after reading.  Synchronises
 * the device.  The paper has no counterpart.
 */
int64_t rx_device_faults(int32_t reset);

/*
 * rx_match_batch -- n (expression, string) pairs in one persistent launch
 * (async).  out[i] = 1 iff pair i's own expression matches its string
 * (e |v w, Fig 2.1, decided by the lockstep machine: null in the evolved
 * set after the last byte, Def 5.3), else 0; RX_RESULT_INVALID for invalid
 * offsets.  handles is a HOST array of n handles (pair i uses handles[i]);
 * strings/offsets/out as in rx_match.  Pairs are bucketed by variant class
 * and length and ordered by serial work per lane (classes whose lanes walk
 * a whole string, longest first; then cached pairs up to the long-pair
 * threshold; then long cached pairs, a warp each, chunked; then pairs of
 * expressions with only the wide cache tier, a warp each, chunked on
 * two-byte state ids), and drained by
 * a device work queue; the tables of all distinct handles are uploaded
 * once per call.  The paper has no counterpart for the batching (its
 * closing section names persistent threads and task queues as future work).
 * Errors: as rx_match.
 */
rx_status rx_match_batch(const rx_handle* handles, size_t n, const uint8_t* strings, const int64_t* offsets,
                         uint8_t* out, void* stream);

/*
 * rx_match_pairs -- the plain form: one kernel launch per pair, in order
 * (async).  Same arguments and result as rx_match_batch (Def 5.3 for each
 * pair's own expression, Fig 2.1); kept as the comparison point for the
 * batched form.
 */
rx_status rx_match_pairs(const rx_handle* handles, size_t n, const uint8_t* strings, const int64_t* offsets,
                         uint8_t* out, void* stream);

/*
 * Prepared batches -- the pairs' expressions fixed once, every run replayed
 * from a captured CUDA graph.  Each pair is decided as in rx_match_batch
 * (Def 5.3 for its own expression); the paper has no counterpart for the
 * preparation, which concerns only how launches are issued.
 *
 * rx_batch_prepare: handles is a HOST array of n handles (pair i uses
 *   handles[i]; they must outlive the plan).  Uploads the distinct tables,
 *   the per-pair table index and class, and allocates the plan's device
 *   scratch (9 bytes per pair, a table header per expression and the
 *   planner's buckets) with cudaMalloc on the current device; synchronous.
 *   Errors: RX_ERR_INVALID_ARG (null or host-only handle), RX_ERR_TOO_LARGE
 *   (n >= 2^31), RX_ERR_OOM, RX_ERR_CUDA.  On error *out is NULL.
 * rx_batch_run: strings/offsets/out are DEVICE buffers laid out as in
 *   rx_match_batch, for the plan's n pairs (async on `stream`).  The first
 *   run with a given (strings, offsets, out) captures the run's launches
 *   (work-counter reset, planner, persistent kernel) into a graph on a
 *   private stream; later runs with the same three pointers replay it, a
 *   different triple captures anew.  Runs on one plan must not overlap on
 *   the GPU (they share the plan's scratch): serialise them on one stream.
 *   Errors: RX_ERR_INVALID_ARG, RX_ERR_CUDA.
 * rx_batch_autotune: runs the batch (results written to out) with every
 *   launch shape -- 128, 256 or 512 threads per block; cached pairs longer
 *   than 0.5, 1, 2, 3, 4, 6 or 8 KiB (1 KiB before tuning), or never,
 *   taking a whole warp (32 chunks whose transfer functions are composed) --
 *   timed with CUDA events on `stream`, and keeps the fastest for later
 *   runs; *chosen (optional) receives it and its rate.  Synchronous.
 *   Errors: as rx_batch_run.
 * rx_batch_set_shape: sets the launch shape of later runs without timing
 *   (e.g. one kept from an earlier rx_batch_autotune): shape->block is 128,
 *   256 or 512; shape->long_pair_bytes >= 1 (cached pairs longer than it take
 *   a warp); gb_per_s is ignored.  The next run captures anew.  Must not be
 *   called while a run of the plan is being issued from another thread.
 *   Errors: RX_ERR_INVALID_ARG (null, bad block or length), RX_ERR_CUDA.
 * rx_batch_free: releases the plan; no run of it may still be in flight.
 */
typedef struct rx_batch* rx_batch_handle;
typedef struct rx_batch_tune {
    int64_t long_pair_bytes;  /* cached pairs longer than this take a warp */
    int32_t block;            /* threads per block of the persistent kernel */
    float gb_per_s;           /* measured input bytes per second / 1e9     */
} rx_batch_tune;
rx_status rx_batch_prepare(const rx_handle* handles, size_t n, rx_batch_handle* out);
rx_status rx_batch_run(rx_batch_handle b, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                       void* stream);
rx_status rx_batch_autotune(rx_batch_handle b, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                            void* stream, rx_batch_tune* chosen);
rx_status rx_batch_set_shape(rx_batch_handle b, const rx_batch_tune* shape);
void rx_batch_free(rx_batch_handle b);

/*
 * rx_match_long -- one long string, exact chunked mode (async).  The input
 * is cut into chunks; for each chunk the transfer function of the macro
 * step (Def 5.2) over the chunk is computed in parallel from every possible
 * incoming state -- exact because a macro step maps a set to the union of
 * the images of its elements ("exists p in S", Defs 5.1, 5.2) -- and the
 * functions are composed starting from the evolution of {root}.  With the
 * cache of macro steps the functions act on its states; with only the wide
 * cache tier a warp takes each chunk (`chunk_bytes` is then the segment a
 * warp cuts into 32); otherwise on bitset rows of singleton images (sets up
 * to 256 bits), else the call runs rx_match_seq.
 *   str          device, len bytes
 *   chunk_bytes  chunk size, 0 = automatic; any value in [1, 2^32 - 32)
 *                is valid (RX_ERR_INVALID_ARG from 2^32 - 32 on: a span's
 *                byte count, with the bytes before it in its first 32-byte
 *                block, is kept in 32 bits)
 *   out          device, 1 byte: 1 iff e |v str
 * Errors: as rx_match.
 */
rx_status rx_match_long(rx_handle h, const uint8_t* str, int64_t len, int64_t chunk_bytes, uint8_t* out,
                        void* stream);

/*
 * rx_match_seq -- one string, one thread, sequential lockstep (async); the
 * reference point for rx_match_long.  Arguments as rx_match_long.
 */
rx_status rx_match_seq(rx_handle h, const uint8_t* str, int64_t len, uint8_t* out, void* stream);

/*
 * rx_trace -- the active set after every byte (async; debugging aid).
 * frontiers (device) receives (len+1) rows of `words` uint32: row k is the
 * evolved set (Def 5.1) before reading str[k], null included; row len is
 * the set after the last byte (null bit set iff the string is accepted).
 * The set is not cut short when it empties.  Errors: as rx_match.
 */
rx_status rx_trace(rx_handle h, const uint8_t* str, int64_t len, uint32_t* frontiers, void* stream);

/* ----------------------------------------------------------------- serving */
typedef struct {
    int64_t device_budget_bytes; /* admission cap on device bytes held by
                                    in-flight requests (0 = 1/4 of free)   */
    int32_t max_inflight;        /* concurrent requests on the device      */
    int32_t queue_capacity;      /* pending requests before RX_ERR_BUSY    */
    int64_t tick_bytes;          /* bytes each in-flight request advances
                                    per device tick (0 = 8 KiB); with k
                                    short requests in flight a tick covers
                                    tick_bytes * max(1, min(8, 8 / k))     */
    int32_t device_payload;      /* where submit()'s bytes live: 0 = host,
                                    copied before submit returns; 1 = device,
                                    valid until the result is polled; 2 =
                                    host, borrowed until the result is
                                    polled (no copy at submit; page-locked
                                    memory is copied at full link speed)  */
    int32_t long_threshold;      /* requests longer than this (bytes) run
                                    the chunked mode (rx_match_long) on
                                    their own streams; 0 = 32 MiB; requests
                                    without a cache of macro steps from
                                    min(this, 1 MiB).  Below it, a request
                                    with a cache and more than a tick left
                                    (with the wide cache tier: every
                                    request) takes a warp per tick and
                                    advances 32 ticks' bytes (chunk
                                    transfer functions)                    */
} rx_serve_cfg;

typedef struct {
    uint64_t submitted, completed;
    double p50_ns, p99_ns, p999_ns, max_ns; /* submit -> result latency */
    double req_per_s, gb_per_s;             /* over the completed requests */
    int64_t ticks;
    int64_t peak_inflight;
    int64_t peak_device_bytes;
} rx_serve_stats_t;

typedef struct rx_server rx_server;

/* Every request of a server is decided as rx_match decides a string: 1 iff
 * its expression matches its whole payload (e |v w, Fig 2.1; null in the
 * evolved set after the last byte, Def 5.3), else 0.  Continuous batching
 * itself has no counterpart in the paper; a request's saved active set
 * between ticks is the machine state of Def 5.2 after the bytes read so
 * far, so resuming it is exact. */

/* rx_serve_create -- start a continuous-batching server on the current
 * device (its own host thread and CUDA stream).  Errors: RX_ERR_INVALID_ARG
 * (device_payload not 0, 1 or 2), RX_ERR_OOM, RX_ERR_CUDA. */
rx_status rx_serve_create(const rx_serve_cfg* cfg, rx_server** out);

/* rx_serve_submit -- enqueue one match (thread-safe).  `bytes` is, by
 * cfg.device_payload: 0, host memory copied before the call returns; 1, a
 * device pointer; 2, host memory the server reads when it admits the
 * request.  In modes 1 and 2 the bytes must stay valid until the result is
 * polled.  The handle must outlive the request.  *ticket identifies the
 * result.  Errors: RX_ERR_BUSY (queue full), RX_ERR_INVALID_ARG, RX_ERR_OOM. */
rx_status rx_serve_submit(rx_server* s, rx_handle h, const uint8_t* bytes, int64_t len, uint64_t* ticket);

/* rx_serve_poll -- collect up to max finished requests (thread-safe);
 * returns how many were written.  results[i] is 0/1, st[i] the status of
 * that request. */
size_t rx_serve_poll(rx_server* s, uint64_t* tickets, uint8_t* results, rx_status* st, size_t max);

/* rx_serve_replay -- load generator for measurement: submit n requests,
 * request i at time t0 + arrival_ns[i] (t0 = entry to the call; the calling
 * thread waits between submissions), handles[i] / payloads[i] / lens[i] as
 * in rx_serve_submit.  tickets (optional, n) receives the tickets.  Returns
 * when all are submitted (not completed); a full queue is retried.
 * *late_ns (optional) receives the largest lateness of a submission behind
 * its arrival time.  Errors: as rx_serve_submit. */
rx_status rx_serve_replay(rx_server* s, const rx_handle* handles, const uint8_t* const* payloads,
                          const int64_t* lens, const int64_t* arrival_ns, size_t n, uint64_t* tickets,
                          int64_t* late_ns);

/* rx_serve_drain -- wait until every submitted request has completed, up
 * to timeout_ms.  Errors: RX_ERR_TIMEOUT. */
rx_status rx_serve_drain(rx_server* s, int64_t timeout_ms);

rx_status rx_serve_stats(rx_server* s, rx_serve_stats_t* out);

/* rx_serve_destroy -- stop the server thread, free its device memory.
 * Outstanding requests are cancelled. */
rx_status rx_serve_destroy(rx_server* s);

/* ---------------------------------------------------------------- autotune */
/*
 * The library's choice of kernel variant and block size per (position-count
 * bucket, mean-length bucket, cache present) is kept in a process-wide table
 * filled by measurement.  rx_match / rx_match_ex with variant AUTO use the
 * entry for the handle's position count and, when opts->len_hint is given,
 * its length bucket (else the bucket-independent entry); without an entry
 * they fall back to memo > thread > sparse > warp.
 */
typedef struct {
    int32_t pos_bucket;  /* floor(log2(positions + 1))                       */
    int32_t len_bucket;  /* floor(log2(mean length + 1)); -1 = any length    */
    int32_t memo;        /* 1: entry for handles with a macro-step cache     */
    int32_t variant;     /* chosen rx_variant                                */
    int32_t block;       /* chosen threads per block                         */
    float gb_per_s;      /* input GB/s of the choice on the tuning sample    */
} rx_tune_entry;

/*
 * rx_autotune -- time every variant that can run h, at 128/256/512 threads
 * per block (and, for the cache of macro steps, the one- and two-byte
 * lookups), on the caller's sample batch (device strings/offsets as in
 * rx_match; `out` device scratch of n bytes), and record the fastest in the
 * table (for the sample's length bucket and as the bucket-independent
 * entry).  Synchronises `stream`.  *chosen (optional) receives the entry.
 * Errors: as rx_match.
 */
rx_status rx_autotune(rx_handle h, size_t n, const uint8_t* strings, const int64_t* offsets, uint8_t* out,
                      void* stream, rx_tune_entry* chosen);

/* rx_autotune_table -- copy up to cap entries of the table; returns the
 * number of entries in the table. */
size_t rx_autotune_table(rx_tune_entry* out, size_t cap);

/* rx_autotune_reset -- empty the table. */
void rx_autotune_reset(void);

/* -------------------------------------------------------------- profiling */
/*
 * rx_profile_enable -- opt-in timing of the lockstep kernels (off by
 * default).  While on, every launch of a main lockstep kernel (the
 * per-string, per-pair and chunk kernels, not the planners) is bracketed by
 * two CUDA events recorded on the stream it is launched on.  Every kernel
 * launch of the library is counted whether or not timing is on.
 */
rx_status rx_profile_enable(int on);

/*
 * rx_profile_read -- launches counted since the last read (all library
 * kernels), and for the timed main kernels their count and summed device
 * time in milliseconds (waits for the recorded events).  Resets both.
 * Any pointer may be NULL.  Errors: RX_ERR_CUDA.
 */
rx_status rx_profile_read(int64_t* launches, int64_t* timed, double* kernel_ms);

/* ------------------------------------------------------------------- misc */
/* Thread-local description of the last error (never NULL). */
const char* rx_last_error(void);

/* Library version string. */
const char* rx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RX_H */
