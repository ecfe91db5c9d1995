/*
 * wt_gb300 -- bottom-up wavelet tree / wavelet matrix construction on GB300.
 *
 * Method: Fischer, Kurpicz, Loebel, "Simple, Fast and Lightweight Parallel
 * Wavelet Tree Construction" (arXiv:1702.07578), prefix counting (Alg. 1 and
 * Alg. 2, Sec. 3; wavelet matrix adaption, Sec. 5.1).
 *
 * Problem (Sec. 2): a text T[0, n) over the alphabet [0, sigma) is turned into
 * L = ceil(lg sigma) bit vectors BV_0 .. BV_{L-1} of n bits each.  Level l of
 * the wavelet tree (WT) holds bit l (counted from the most significant of the
 * L code bits) of the symbols stably sorted by their l-bit prefix (Obs. 1).
 * Level l of the wavelet matrix (WM) holds bit l of the symbols stably sorted
 * by their reversed l-bit prefix (Obs. 2), and Z[l] is its number of zeros.
 * Only the bit vectors are built; rank/select support is not (Sec. 4).
 *
 * Output layout (the paper does not fix the bit order inside a word): level l
 * occupies 64-bit words [l*W, (l+1)*W) of d_bv with W = wt_words_per_level(n);
 * bit j of a level is bit (j & 63) of word (j >> 6), least significant first;
 * bits >= n of the last word are written as zero.  d_zeros receives L values.
 *
 * Memory: every pointer named d_* is device memory owned by the caller.  The
 * library allocates nothing in the build calls; it uses the caller's
 * workspace (size from the *_workspace_size calls, any alignment >= 256 B).
 * Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 * void*, NULL = legacy default stream).  A workspace must not be shared by
 * two builds in flight.
 *
 * Errors: argument errors are returned at once and nothing is launched.
 * Errors found on the device (a symbol >= sigma) are recorded in the
 * workspace; wt_sync_status() synchronises the stream and returns them.
 * After a device-detected error the contents of d_bv / d_zeros are
 * unspecified (the kernels still write only inside the caller's buffers).
 * No call aborts the process.
 *
 * Limits: n < 2^32 per text; sigma <= 2^32 for the WM; sigma <= 2^24 for
 * the WT (larger alphabets return WT_ERR_INVALID_ARG).  The storage type
 * must hold sigma - 1 (sigma <= 2^8 for WT_U8, <= 2^16 for WT_U16).
 */
#ifndef WT_GB300_H
#define WT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WT_OK = 0,
    WT_ERR_INVALID_ARG = 1,    /* bad pointer, size, type or alphabet      */
    WT_ERR_SYMBOL_RANGE = 2,   /* device found a symbol >= sigma           */
    WT_ERR_OUT_OF_MEMORY = 3,  /* workspace too small / allocation failed  */
    WT_ERR_CUDA = 4,           /* a CUDA runtime call failed               */
    WT_ERR_TIMEOUT = 5,        /* a bounded wait ran out                   */
    WT_ERR_BUSY = 6,           /* server: request cannot be admitted now   */
    WT_ERR_NOT_FOUND = 7       /* server: unknown or released ticket       */
} wt_status;

typedef enum { WT_U8 = 1, WT_U16 = 2, WT_U32 = 4 } wt_symtype;   /* bytes per symbol */
typedef enum { WT_TREE = 0, WT_MATRIX = 1 } wt_kind;

/* L = ceil(lg sigma), the number of levels (Sec. 2); 0 when sigma <= 1. */
uint32_t wt_levels(uint64_t sigma);

/* W = ceil(n / 64), the 64-bit words of one level. */
uint64_t wt_words_per_level(uint64_t n);

/* Human-readable name of a status code (static storage). */
const char *wt_status_string(wt_status s);

/* Workspace bytes needed by wt_build (kind = WT_TREE) or wm_build
 * (kind = WT_MATRIX) for one text of n symbols over [0, sigma). */
wt_status wt_workspace_size(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma,
                            size_t *bytes);

/* Wavelet tree of one text (Alg. 1 / Alg. 2 with id = identity, Sec. 3).
 *   d_text  n symbols of the given storage type, each < sigma
 *   d_bv    L * W words, written completely (see layout above)
 *   d_ws    workspace of ws_bytes >= wt_workspace_size(WT_TREE, ...)
 * n = 0 or sigma = 1 is valid and writes nothing. */
wt_status wt_build(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                   uint64_t *d_bv, void *d_ws, size_t ws_bytes, void *stream);

/* Wavelet matrix of one text (Sec. 5.1: id replaced by the bit-reversal
 * permutation).  d_zeros receives Z[0..L) (Sec. 5, number of zeros of each
 * level); it may be NULL when L = 0. */
wt_status wm_build(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                   uint64_t *d_bv, uint64_t *d_zeros, void *d_ws, size_t ws_bytes,
                   void *stream);

/* Synchronise the stream and return the first error the device recorded in
 * this workspace during the last build on it (WT_OK if none), then clear it. */
wt_status wt_sync_status(void *d_ws, void *stream);

/* ---- texts of any length: domain decomposition (Sec. 3.3) ---------------------
 * For texts of 2^32 symbols or more (up to 2^40), which the builds above do not
 * take, and for sigma <= 256.  The text is cut into consecutive slices of `slice`
 * symbols (0: 2^31; at most 2^32 - 1, at most 2^16 slices); each slice is built
 * on its own (wt_build / wm_build) into partial levels in the workspace, and the
 * partial levels are merged: merged level l is, prefix by prefix in id order (WT)
 * or bit-reversal order (WM), the slices' intervals of that prefix in slice order,
 * placed by a zero-based prefix sum of their sizes; Z[l] is the sum of the slices'.
 * The output is bit-identical to wt_build / wm_build of the whole text, with the
 * same layout (W = ceil(n / 64) words per level, now 64-bit counts).  The
 * workspace (wt_large_workspace_size) holds one slice build's workspace, the
 * partial levels (about L * n / 8 bytes) and small tables.  wt_sync_status on
 * the workspace returns the first device-detected error of any slice. */
wt_status wt_large_workspace_size(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t slice,
                                  size_t *bytes);
wt_status wt_build_large(wt_kind kind, const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                         uint64_t slice, uint64_t *d_bv, uint64_t *d_zeros, void *d_ws, size_t ws_bytes,
                         void *stream);

/* ---- the stable order as a by-product ----------------------------------------
 * The splits that build the levels leave the symbols, after the last level, in
 * one stable order (Obs. 1 and Obs. 2 one level past the last): for the WT, T
 * stably sorted by symbol (the sorted text psWT builds level by level,
 * Sec. 3.2.1); for the WM, T stably sorted by the bit-reversed L-bit code.
 * wt_build_order / wm_build_order build the levels (bit-identical to wt_build /
 * wm_build) and also write
 *   d_perm[j]    text position of the j-th symbol in that order (n uint32,
 *                required when n > 0)
 *   d_sorted[j]  T[d_perm[j]] (n symbols of the text's type; may be NULL).
 * For sigma = 1 the order is the text order.  The workspace is
 * wt_order_workspace_size bytes (it adds n uint32 of positions carried through
 * each round that cuts).  Texts that want the order take the block path for
 * every job, also for jobs of at most 4096 symbols. */
wt_status wt_order_workspace_size(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes);
wt_status wt_build_order(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv,
                         uint32_t *d_perm, void *d_sorted, void *d_ws, size_t ws_bytes, void *stream);
wt_status wm_build_order(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv,
                         uint64_t *d_zeros, uint32_t *d_perm, void *d_sorted, void *d_ws, size_t ws_bytes,
                         void *stream);

/* ---- the wavelet tree and the wavelet matrix of one text, together ------------
 * Level l of the WT and level l of the WM hold the same bits interval by
 * interval: both are stable splits of the same symbols, and only the order of
 * the intervals in the level differs (id order for the WT, bit-reversal order
 * for the WM, Sec. 5.1 and Sec. 5.2).  wt_wm_build builds both from one
 * histogram pass and one split pass over the text when sigma <= 256 and
 * n > 4096: every tile's class runs are split once and written to both.
 * Otherwise it runs wt_build and then wm_build on the stream.  The output is
 * bit-identical to wt_build (d_bv_wt) plus wm_build (d_bv_wm, d_zeros); the
 * arguments, limits and errors are theirs (wt_sync_status reads device
 * errors).  The workspace is wt_wm_workspace_size bytes. */
wt_status wt_wm_workspace_size(wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes);
wt_status wt_wm_build(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv_wt,
                      uint64_t *d_bv_wm, uint64_t *d_zeros, void *d_ws, size_t ws_bytes, void *stream);

/* ---- host buffers in, host buffers out ----------------------------------------
 * The problem of Sec. 2 with the text and the levels in host memory.  On `stream`
 * the call copies the text into the device workspace, builds the WT
 * (h_bv_wt != NULL) and/or the WM (h_bv_wm != NULL), and copies the levels
 * (L * W words each, the layout above) and, for the WM, Z[0..L) (h_zeros) back.
 * The builds are wt_build and wm_build, or wt_wm_build (both from one pass)
 * when both are asked for and one_pass != 0; the results are bit-identical.
 *   h_text   n symbols of the given type (host memory; may be NULL when n = 0)
 *   h_bv_wt  L * W words or NULL;  h_bv_wm  L * W words or NULL (not both NULL)
 *   h_zeros  L words, required with h_bv_wm when L > 0
 *   d_ws     device memory of ws_bytes >= wt_host_workspace_size(...): the
 *            build workspace at offset 0 (so wt_sync_status(d_ws) reads the
 *            builds' device-detected errors), then the device copy of the text
 *            and the device levels of both kinds.
 * The copies are cudaMemcpyAsync on `stream`: with page-locked host buffers the
 * call returns before they finish (synchronise the stream, or call
 * wt_sync_status, before reading or reusing the host buffers); with pageable
 * buffers CUDA makes them synchronous for the host.  Argument errors are
 * returned before anything is queued; limits are those of the builds. */
wt_status wt_host_workspace_size(wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes);
wt_status wt_build_host(const void *h_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *h_bv_wt,
                        uint64_t *h_bv_wm, uint64_t *h_zeros, int one_pass, void *d_ws, size_t ws_bytes,
                        void *stream);

/* ---- wavelet tree without any device allocation --------------------------
 * The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory: code running under a host
 * framework that owns every device allocation, services that must keep a
 * memory footprint fixed at start-up, or code paths that may not call
 * cudaMalloc / cudaFree because those calls can synchronise the device.
 *
 * Same result as wt_build (bit-identical), but the workspace is a fixed
 * array of 1 MiB in device memory inside this library, which every GPU that
 * loads the library holds until the process exits.  The caller still passes the text and the output buffer.  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *
 * Limit: a text is accepted when wt_workspace_size(WT_TREE, type, n, sigma)
 * is at most 1,048,576 bytes (the exact test); larger ones are rejected with
 * WT_ERR_OUT_OF_MEMORY before anything is launched.  That is n <= 11,010,048
 * symbols for sigma <= 256, n <= 948,736 for sigma = 257 and n <= 882,688 for
 * sigma = 4096 (uint16 storage; alphabets above 256 also need a re-sorted copy
 * of the text), and no text at all for sigma = 65536 or more (the per-subtree
 * tables of the later rounds alone exceed the array).
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The call
 * reads no host memory on the stream: the text's descriptor reaches the array
 * as a kernel argument.  All calls
 * share the one array and every call re-initialises what it reads from it, so
 * calls are correct one after the other; two calls that overlap on the GPU
 * (different streams, or different host threads) race on the array and give
 * wrong results.  Errors the device would detect (a symbol >= sigma) are not
 * reported by this call: such symbols give unspecified bit vectors (the
 * kernels still write only inside d_bv). */
wt_status wt_build_static_ws(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                             uint64_t *d_bv, void *stream);

/* ---- batched construction ---------------------------------------------
 * Many independent texts built together (all WT or all WM, one storage
 * type).  Each descriptor names its device text, length, alphabet and
 * output buffers (d_zeros only for WT_MATRIX).  The descriptors are read
 * from host memory during the call and may be reused after it returns.
 * Output is bit-identical to one wt_build / wm_build per text. */
typedef struct {
    const void *d_text;
    uint64_t n;
    uint64_t sigma;
    uint64_t *d_bv;
    uint64_t *d_zeros;
} wt_text_desc;

wt_status wt_batched_workspace_size(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs,
                                    uint32_t count, size_t *bytes);

wt_status wt_build_batched(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs,
                           uint32_t count, void *d_ws, size_t ws_bytes, void *stream);

/* ---- batched construction replayed from a CUDA graph ------------------------
 * For a batch whose shapes repeat (same count, same n and sigma per text):
 * wt_batch_plan_create plans the build, uploads the descriptors into the
 * workspace and records every kernel of the build once into a CUDA graph by
 * stream capture on `stream` (which must not be the legacy default stream;
 * nothing executes during the capture).  wt_batch_plan_launch replays the
 * graph: one launch for the whole batch.  wt_batch_plan_update replaces the
 * device pointers of the texts and outputs (same n and sigma per text, else
 * WT_ERR_INVALID_ARG): it waits for the stream, then copies the new
 * descriptors into the workspace on the stream, in place, so the same graph
 * builds the new texts.  The workspace (size from wt_batched_workspace_size)
 * and every buffer named by the descriptors must stay valid while the plan is
 * used.  symbols_per_block: symbols one build block processes, a multiple of
 * 32768 up to 2^24; 0 takes the value the autotuner stored for batches of this
 * shape (WT_TUNE_CACHE), else the default.  The plan holds host memory and the
 * graph; wt_batch_plan_destroy frees them. */
typedef struct wt_batch_plan wt_batch_plan;

wt_status wt_batch_plan_create(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs, uint32_t count,
                               uint32_t symbols_per_block, void *d_ws, size_t ws_bytes, void *stream,
                               wt_batch_plan **out);
wt_status wt_batch_plan_update(wt_batch_plan *plan, const wt_text_desc *h_descs, void *stream);
wt_status wt_batch_plan_launch(wt_batch_plan *plan, void *stream);
uint32_t wt_batch_plan_symbols_per_block(const wt_batch_plan *plan);
void wt_batch_plan_destroy(wt_batch_plan *plan);

/* Autotuner: builds the batch (for real, into its output buffers) with each
 * candidate symbols-per-block value (32768, 65536, 131072, 262144), times three
 * builds of each with CUDA events on `stream`, and returns the fastest.  If the
 * environment variable WT_TUNE_CACHE names a file, the choice is stored there
 * (a JSON object) under a key made of the kind, the storage width and buckets
 * of the batch's count, total and largest length and rounds; plans created with
 * symbols_per_block = 0 look it up.  Synchronises the stream. */
wt_status wt_autotune_batched(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs, uint32_t count,
                              void *d_ws, size_t ws_bytes, void *stream, uint32_t *best_symbols_per_block);

/* ---- serving -------------------------------------------------------------
 * A server owns device memory (bounded by hbm_budget_bytes) and a set of
 * CUDA streams on one device.  Requests (host texts) are admitted while
 * their footprint (text + output + workspace) fits in the budget, batched
 * as they arrive, built concurrently on the streams, and kept resident on
 * the device until released.  All server calls are thread-safe. */
typedef struct wt_server wt_server;

typedef struct {
    size_t hbm_budget_bytes;   /* device memory the server may hold            */
    uint32_t max_batch;        /* requests per batch launch (>= 1)             */
    uint32_t streams;          /* concurrent CUDA streams (>= 1)               */
    int device;                /* CUDA device ordinal                          */
    uint32_t max_pending;      /* queued requests before submit returns BUSY   */
} wt_server_config;

typedef struct {
    wt_kind kind;
    wt_symtype type;
    const void *h_text;        /* host text; copied during submit              */
    uint64_t n;
    uint64_t sigma;
} wt_request;

typedef struct {
    const uint64_t *d_bv;      /* L * W words, device, valid until release     */
    const uint64_t *d_zeros;   /* L values for WT_MATRIX, else NULL            */
    uint32_t levels;
    uint64_t words_per_level;
    uint64_t n;
    wt_status status;          /* build status of this request                 */
    double latency_us;         /* submit -> completion                         */
} wt_result;

typedef struct {
    uint64_t submitted, completed, rejected, in_flight;
    double p50_us, p99_us;     /* latency over completed requests              */
    double symbols_per_s;      /* completed symbols / wall time since create   */
    size_t hbm_in_use;
} wt_server_stats;

wt_status wt_server_create(const wt_server_config *cfg, wt_server **out);
/* Copy the request's text and queue it; WT_ERR_BUSY if the queue is full or
 * the request alone exceeds the budget.  *ticket identifies it. */
wt_status wt_server_submit(wt_server *s, const wt_request *req, uint64_t *ticket);
/* As wt_server_submit, without the host copy: req->h_text must be page-locked
 * host memory (cudaHostAlloc or cudaHostRegister; anything else gives
 * WT_ERR_INVALID_ARG) and must stay allocated and unchanged until
 * wt_server_wait has returned the request as done.  The batch's device copy
 * reads it directly. */
wt_status wt_server_submit_pinned(wt_server *s, const wt_request *req, uint64_t *ticket);
/* Wait until the request is built (timeout_us < 0: no limit); WT_ERR_TIMEOUT
 * if the limit passes first. */
wt_status wt_server_wait(wt_server *s, uint64_t ticket, int64_t timeout_us, wt_result *res);
/* Copy a finished request's bit vectors (L * W words) and, for WT_MATRIX,
 * Z (L values) to host memory; blocks until the copy is done.  h_zeros may be
 * NULL.  WT_ERR_BUSY if the request has not finished. */
wt_status wt_server_read(wt_server *s, uint64_t ticket, uint64_t *h_bv, uint64_t *h_zeros);
/* Free the request's device memory; the ticket becomes invalid. */
wt_status wt_server_release(wt_server *s, uint64_t ticket);
wt_status wt_server_get_stats(wt_server *s, wt_server_stats *st);
/* Let the batches already launched finish, drop the requests not launched yet
 * (queued, or admitted and waiting for a stream), and free everything: every
 * ticket of the server is invalid afterwards.  No other call on the server may
 * run at the same time or later. */
void wt_server_destroy(wt_server *s);

/* ---- queries: access / rank / select on built bit vectors ---------------------
 * Queries on a built WT or WM (Sec. 2: "the bit vectors are augmented by binary
 * rank and select structures" answer access, rank and select in O(lg sigma)).
 *
 * Rank support (caller-owned device memory of wt_rank_support_size bytes):
 * for every level, the number of ones before each 256-bit block; for the WT,
 * also every node's start and the ones before it, per level (levels < L).
 * wt_rank_support_build fills it from d_bv (and, for the WM, d_zeros) on the
 * stream.  n < 2^32.  The bit vectors must stay unchanged while queries run.
 *
 *   wt_access   d_out[k] = T[d_pos[k]]                      (d_pos[k] < n)
 *   wt_rank     d_out[k] = number of d_sym[k] in T[0, d_pos[k])  (d_pos[k] <= n)
 *   wt_select   d_out[k] = position of the d_j[k]-th (1-based) d_sym[k] in T,
 *               or UINT64_MAX when there is no such occurrence
 * Positions or symbols out of range give UINT64_MAX (rank, select) or
 * 0xFFFFFFFF (access) in that slot.  All arrays are device memory; the calls
 * are asynchronous on the stream. */
wt_status wt_rank_support_size(wt_kind kind, uint64_t n, uint64_t sigma, size_t *bytes);
wt_status wt_rank_support_build(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, uint64_t n,
                                uint64_t sigma, void *d_rs, size_t rs_bytes, void *stream);
wt_status wt_access(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, const void *d_rs, uint64_t n,
                    uint64_t sigma, const uint64_t *d_pos, uint32_t count, uint32_t *d_out, void *stream);
wt_status wt_rank(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, const void *d_rs, uint64_t n,
                  uint64_t sigma, const uint32_t *d_sym, const uint64_t *d_pos, uint32_t count, uint64_t *d_out,
                  void *stream);
wt_status wt_select(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, const void *d_rs, uint64_t n,
                    uint64_t sigma, const uint32_t *d_sym, const uint64_t *d_j, uint32_t count, uint64_t *d_out,
                    void *stream);

/* ---- WT position -> WM position (Sec. 5.2, Lemma 3) --------------------------
 * For a text whose WT and WM are both built: position i of WT level l and
 * position j of WM level l hold the bit of the same text symbol, with
 *   j = i                                  for l <= 1,
 *   j = X[2^l - 2 + bp] + off              otherwise,
 * bp = prefix(l, rank0(U, select1(U, i+1))) and
 * off = i - rank1(U, select0(U, bp << (L - l))).
 * U is the unary histogram 1^h(0) 0 1^h(1) 0 ... of the 2^L characters (n + 2^L
 * bits, with its own rank directory); X holds the WM interval starts of levels
 * 1 .. L-1, level l at X[2^l - 2, 2^(l+1) - 2).  (The lemma's statement writes
 * X[2^(l-1) - 2 + bp]; that form lets levels overlap, and the proof's index is
 * the one used here.)
 *
 * wt_wt2wm_size    bytes of the map for (n, sigma); sigma <= 2^24 as for the WT
 *                  rank support.
 * wt_wt2wm_build   fills d_map (caller-owned device memory, map_bytes >= size)
 *                  from the WT bit vectors d_bv and their rank support d_rs
 *                  (wt_rank_support_build with kind WT_TREE, same n and sigma);
 *                  the histogram is read off the node tables of level L-1.
 *                  Asynchronous on the stream; d_bv and d_rs must stay unchanged
 *                  until it has run.  WT_ERR_OUT_OF_MEMORY if map_bytes is short.
 * wt_wt2wm         d_out[k] = j for (d_level[k], d_pos[k]); UINT64_MAX where
 *                  d_level[k] >= L or d_pos[k] >= n.  Device arrays, asynchronous.
 * Select on U is a binary search over its rank directory plus a scan of one
 * 256-bit block (O(lg n)), not the constant-time select the lemma assumes. */
wt_status wt_wt2wm_size(uint64_t n, uint64_t sigma, size_t *bytes);
wt_status wt_wt2wm_build(const uint64_t *d_bv, const void *d_rs, uint64_t n, uint64_t sigma, void *d_map,
                         size_t map_bytes, void *stream);
wt_status wt_wt2wm(const void *d_map, uint64_t n, uint64_t sigma, const uint32_t *d_level, const uint64_t *d_pos,
                   uint32_t count, uint64_t *d_out, void *stream);

/* ---- diagnostics ----------------------------------------------------------
 * Per-kernel device time.  While enabled, every build records CUDA events on
 * its own stream before and after each kernel it launches (the work itself is
 * unchanged).  wt_profile_read() waits for the recorded events and returns the
 * summed milliseconds and launch counts per kernel family since the last
 * reset:  [0] split/scatter (k_build_bs, k_build_small)   [1] histogram (k_hist)
 *         [2] segmented scan (3 kernels) [3] job lists (2-3 kernels).
 * Not thread-safe with concurrent builds; meant for benchmarks. */
typedef struct {
    double ms[4];
    uint64_t launches[4];
} wt_profile;

void wt_profile_enable(int on);
wt_status wt_profile_read(wt_profile *out, int reset);

/* ---- bounds checks (a debug build of the library) -------------------------
 * The paper has no counterpart: these calls check the construction kernels'
 * own indexing, in place of a memory checker.  When the library is compiled
 * with -DWT_DEBUG_BOUNDS, the construction kernels (histogram pass, split
 * kernels, small-job kernel) compare every index of a global or shared access
 * whose bound is not evident from the loop around it with the size of the
 * buffer it addresses: symbols read inside the text (or the round's buffer),
 * bit-vector words inside L * W, histogram and job rows inside the round's
 * tables, shared-memory indexes inside their arrays, re-sorted symbols written
 * below n.  A failed check skips that access (the output is then wrong) and
 * counts; the first failure's site, index and bound are kept.  The default
 * build compiles no checks and runs the same code as before.
 *
 * wt_debug_bounds_read: the report of the device that is current, after a
 * cudaDeviceSynchronize; reset != 0 clears it afterwards.  A library built
 * without the checks returns enabled = 0 and all zeros, touching no device.
 * wt_debug_bounds_selftest: on `stream`, evaluates one check that fails (site
 * WT_BOUNDS_SELFTEST, index 1, bound 1) and one that holds, with no memory
 * access behind either, so that a test can see that failures are recorded.
 * WT_ERR_INVALID_ARG in a build without the checks. */
typedef enum {
    WT_BOUNDS_SELFTEST = 0,   /* wt_debug_bounds_selftest                     */
    WT_BOUNDS_TEXT = 1,       /* a symbol read past the text / round buffer   */
    WT_BOUNDS_LEVEL = 2,      /* a bit-vector word outside L * W              */
    WT_BOUNDS_TABLE = 3,      /* a job, group or tile row outside the round's */
    WT_BOUNDS_SHARED = 4,     /* a shared-memory index outside its array      */
    WT_BOUNDS_NEXT = 5        /* a re-sorted symbol or position at >= n       */
} wt_bounds_site;

typedef struct {
    uint32_t enabled;         /* 1: this library was built with the checks    */
    uint32_t failures;        /* failed checks since the last reset           */
    uint32_t site;            /* first failure: a wt_bounds_site              */
    uint32_t pad;
    uint64_t index;           /* first failure: the index ...                 */
    uint64_t bound;           /* ... and the bound it had to stay below       */
} wt_bounds_report;

wt_status wt_debug_bounds_read(wt_bounds_report *out, int reset);
wt_status wt_debug_bounds_selftest(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* WT_GB300_H */
