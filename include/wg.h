/* wg.h -- C-ABI of libwg: semi-naive Datalog fixpoints (transitive closure,
 * same-generation) on one GB300 GPU.
 *
 * Problem statement (paper, Sec. Background): a relation is a SET of tuples;
 * recursive rules are applied until no new tuple is derived.  The library
 * evaluates, over uint32 vertex ids,
 *   TC:  T(x,y) <- E(x,y).   T(x,z) <- T(x,y), E(y,z).            (Sec. Background)
 *   SG:  sg(x,y) <- E(p,x), E(p,y), x != y.                         (base rule)
 *        sg(x,y) <- E(a,x), sg(a,b), E(b,y).                        (Sec. Generalization;
 *        the paper's parent(X,P) is read as the edge P -> X)
 * by semi-naive evaluation (Sec. Background, "Semi-Naive Evaluation", steps
 * 1-5): each iteration joins the newest delta with E, sorts the candidates,
 * removes duplicates and tuples already known, and merges the survivors into
 * the full relation (Secs. Sorted-Array Pipeline and Asynchronous Fixpoint
 * Engine).  The loop runs on the device; the host sees only the end result.
 *
 * Conventions for every entry point
 *  - Return value: WG_OK (0) or a negative WG_E_* code.  Nothing aborts, traps
 *    or exits.  wg_last_error() gives a message for the calling thread.
 *  - "host" pointers are ordinary CPU memory (pageable or pinned); "device"
 *    pointers are CUDA global memory of the context's device.
 *  - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *    The library owns relations and query results until the matching *_free.
 *  - Tuples are returned as packed keys (uint64_t(src) << 32) | dst in
 *    ascending order, i.e. the lexicographic (src, dst) order the paper keeps
 *    every relation in (Sec. Binary-Search Join).  Ids span all of uint32.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - Every call is stream-ordered on the context's stream.
 */
#ifndef WG_H
#define WG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WG_OK 0
#define WG_E_INVAL (-1)          /* bad argument, handle or state */
#define WG_E_NOMEM (-2)          /* a device allocation failed */
#define WG_E_BUDGET (-3)         /* the request does not fit the context's memory budget */
#define WG_E_CAPACITY (-4)       /* caller buffer too small; the needed size is returned */
#define WG_E_NOT_READY (-5)      /* the query has not finished (wg_wait timed out) */
#define WG_E_ITER_CAP (-6)       /* max_iters iterations ran without reaching the fixpoint */
#define WG_E_DEVICE_TIMEOUT (-7) /* a bounded device-side wait gave up; the result is void */
#define WG_E_CUDA (-8)           /* a CUDA runtime call failed */

typedef struct wg_ctx wg_ctx;
typedef uint64_t wg_rel;   /* relation handle, 0 = none */
typedef uint64_t wg_query; /* query handle, 0 = none */

/* Device memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes (256-byte aligned) usable in stream order on `stream`, or NULL.  free
 * releases it.  Both may be NULL in wg_init: the library then calls
 * cudaMallocAsync / cudaFreeAsync on the context stream. */
typedef void* (*wg_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*wg_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

enum wg_kind { WG_TC = 0, WG_SG = 1 };

enum wg_loop {
  WG_LOOP_DEVICE = 0, /* one CUDA graph per run: a conditional WHILE node holds the
                         iteration; no host synchronisation between iterations */
  WG_LOOP_HOST = 1,   /* the host launches each iteration and reads the delta size
                         back once per iteration (one sync per iteration), for
                         comparison */
  WG_LOOP_HOST_STAGED = 2 /* the host launches every stage and reads the control block
                         back after each one, waiting for it (about 10-14 syncs per
                         iteration: the per-stage readback of the host-driven
                         pipelines of Sec. Motivation, "Stage-Wise Synchronization"),
                         for comparison.  Single queries (wg_tc / wg_sg) only */
};

/* wg_opts.flags */
#define WG_FLAG_SEPARATE_STAGES 1u /* run deduplication + set difference and the merge as the
                                      paper's separate stages (Secs. Fused Deduplication and
                                      Set Difference, Disjoint Merge) instead of one fused
                                      merge-path pass that also writes the merged relation */
#define WG_FLAG_FULL_WIDTH 2u      /* ablation: radix-sort every key bit (32 or 64) instead of
                                      only the significant bits, and no per-source sort (the
                                      fixed-width baseline of Sec. Buffer Routing and Adaptive
                                      Radix Sort); same result */
#define WG_FLAG_COPY_BACK 4u       /* ablation (single queries, fused stages): copy the merged
                                      relation back into the Full buffer every iteration
                                      instead of swapping the two buffers (the copy-back
                                      baseline of the paper's ping-pong evaluation); same
                                      result */
#define WG_FLAG_HASH_JOIN 8u       /* ablation (TC queries): look up E(y, .) in a linear-probing
                                      hash table of E keyed by source (built once per relation,
                                      compare-and-swap inserts) and emit one delta tuple per
                                      thread, instead of the CSR range lookup and the
                                      load-balanced emit (Sec. Data Skew in Hash-Based Join);
                                      same result.  Ignored by SG queries and by wg_submit */
#define WG_FLAG_MERGE_EVERY_ITER 16u /* ablation (single queries, fused stages): merge the new
                                      tuples into the full relation at every iteration (the
                                      disjoint merge of Sec. Disjoint Merge after each pass).
                                      By default the full relation is kept as a main run and
                                      a small side run of the newest tuples: an iteration
                                      whose candidates are at most 1/8 of the main run finds
                                      its new tuples against both runs and merges them into
                                      the side run only, so the main run is not rewritten;
                                      the side run is folded back when it outgrows its pool
                                      (an eighth of the full relation's) or when the
                                      candidates grow again, and the final relation is the
                                      two runs merged.  Same result either way */
#define WG_FLAG_SIDE_RUN_ALWAYS 32u /* testing (single queries, fused stages): take the side run
                                      in every iteration it fits, however many candidates;
                                      same result */

typedef struct wg_opts {
  uint32_t max_iters;    /* iteration cap; 0 = 1<<20 */
  uint32_t loop;         /* enum wg_loop */
  uint32_t profile;      /* 1 = time every kernel with CUDA events (forces WG_LOOP_HOST) */
  uint32_t flags;        /* WG_FLAG_* */
  uint64_t reserve_full; /* initial capacity of the full relation, tuples; 0 = auto */
  uint64_t reserve_cand; /* initial capacity of the candidate buffers, tuples; 0 = auto */
} wg_opts;

enum wg_state { WG_PENDING = 0, WG_RUNNING = 1, WG_DONE = 2, WG_FAILED = 3 };

typedef struct wg_status {
  int32_t state;       /* enum wg_state */
  int32_t error;       /* WG_OK or the WG_E_* code of a failed query */
  uint64_t n_tuples;   /* size of the result relation once DONE */
  uint32_t iterations; /* index of the first empty delta (the chain a->b->c->d gives 3) */
  uint32_t regrows;    /* how often buffers were grown and the loop resumed */
  uint64_t candidates; /* sum over iterations of the join output size |C| */
  uint64_t gpu_launches; /* kernels this query launched */
  double device_ms;    /* device time from the first launch to completion (CUDA events) */
} wg_status;

typedef struct wg_request {
  int32_t kind;        /* enum wg_kind */
  uint32_t reserved0;
  wg_rel edges;
  wg_opts opts;        /* loop and profile are ignored in batches */
} wg_request;

/* Per-kernel timing of a profiled query (opts.profile = 1).  `bytes` is the
 * ALGORITHMIC traffic of all its launches: the bytes the method must move,
 * counted from the relation sizes, not from hardware counters. */
typedef struct wg_kernel_stat {
  char name[32];
  uint64_t launches;
  double total_ms;
  double bytes;
} wg_kernel_stat;

/* ---- context -------------------------------------------------------------
 * wg_init: binds `device`, creates or adopts `cuda_stream` (a cudaStream_t;
 * NULL = a new non-blocking stream owned by the context).  mem_budget_bytes
 * caps the device memory the context holds at any time (0 = 90% of the free
 * memory).  Errors: WG_E_INVAL (bad device), WG_E_CUDA. */
int wg_init(int device, size_t mem_budget_bytes, wg_alloc_fn alloc, wg_free_fn free_fn,
            void* user, void* cuda_stream, wg_ctx** out);
/* Waits for the stream, releases every relation, query and buffer. */
void wg_destroy(wg_ctx* ctx);
/* Message of the last failing call on this thread ("" if none). */
const char* wg_last_error(void);
/* Device bytes currently held by the context. */
size_t wg_mem_used(const wg_ctx* ctx);

/* ---- relations -----------------------------------------------------------
 * wg_relation_load: the edge set {(src[i], dst[i]) : i < n} from HOST arrays
 * (copied; duplicates removed, self-loops kept).  The relation is sorted once
 * here and never modified (Sec. Binary-Search Join: E is sorted at dataset
 * load); a CSR index on the source is built for the join.  Vertex ids are
 * relabelled internally to their rank among the distinct ids, which keeps
 * the lexicographic order and picks the narrowest key width (the adaptive
 * radix width of Sec. Buffer Routing and Adaptive Radix Sort).  n = 0 is a
 * valid empty relation.  Errors: WG_E_INVAL (NULL arrays with n > 0, n >= 2^32),
 * WG_E_NOMEM / WG_E_BUDGET. */
int wg_relation_load(wg_ctx* ctx, const uint32_t* src, const uint32_t* dst, size_t n,
                     wg_rel* out);
/* Same, from DEVICE arrays (read in stream order, not retained). */
int wg_relation_load_device(wg_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, size_t n,
                            wg_rel* out);
/* Distinct edges, distinct vertices, and bits per vertex field of a relation. */
int wg_relation_info(wg_ctx* ctx, wg_rel rel, uint64_t* n_edges, uint32_t* n_vertices,
                     uint32_t* field_bits);
void wg_relation_free(wg_ctx* ctx, wg_rel rel);

/* ---- single queries ------------------------------------------------------
 * wg_tc / wg_sg: enqueue one fixpoint on the context stream and return at once.
 * opts may be NULL (defaults).  The result is ready when wg_poll reports
 * WG_DONE or wg_wait returns WG_OK; buffers that turn out too small are grown
 * and the loop resumed inside wg_poll / wg_wait.  Errors: WG_E_INVAL (bad
 * handle), WG_E_NOMEM / WG_E_BUDGET (the first pools do not fit; idle
 * engines' pools are released first).  On an error no query is left behind
 * and *out is 0. */
int wg_tc(wg_ctx* ctx, wg_rel edges, const wg_opts* opts, wg_query* out);
int wg_sg(wg_ctx* ctx, wg_rel edges, const wg_opts* opts, wg_query* out);

/* ---- batches and serving -------------------------------------------------
 * wg_submit: admit n independent fixpoints (TC or SG, any mix) that run
 * TOGETHER: every stage of every iteration is one launch over the tiles of
 * all running queries, and the iteration loop is one CUDA graph.  Queries
 * submitted while earlier ones run join the running set at the next
 * iteration boundary that wg_poll / wg_wait / wg_serve_step reaches
 * (continuous batching).  ids[i] receives the handle of reqs[i].  Queries
 * are grouped into batch engines by key width and size class; a request
 * over 65,536 edges instead runs on a single-query engine (one at a time, on
 * the context stream) beside the batch engines -- one such fixpoint already
 * fills the GPU.  Admission is by device-memory budget: a request that
 * cannot be admitted now stays queued (state WG_PENDING).  When pools cannot
 * grow within the budget, idle engines' pools are released first, then the
 * most recently admitted query of the engine is requeued (it restarts
 * later); a query left alone in its engine that still cannot grow pauses
 * with its state until the other engines drain (nothing else is admitted
 * meanwhile) and resumes with the whole budget.  Only a query that does not
 * fit with the whole budget fails, with WG_E_BUDGET.  The results do not
 * depend on any of this (each query's result equals its result alone).
 * Errors: WG_E_INVAL; WG_E_BUDGET / WG_E_NOMEM when a new engine's first
 * pools do not fit. */
int wg_submit(wg_ctx* ctx, const wg_request* reqs, size_t n, wg_query* ids);
/* Advance the batch engine by at most `iters` iterations (admitting queued
 * requests and retiring finished ones) and return without waiting for the
 * device beyond that.  *n_running receives the number of queries in flight. */
int wg_serve_step(wg_ctx* ctx, uint32_t iters, size_t* n_running);

/* Ids of batch queries that reached DONE or FAILED since the previous call
 * (at most cap of them; *n_out = how many were written; the rest stay queued
 * for the next call).  Lets a serving loop find finished queries without
 * polling every handle.  Errors: WG_E_INVAL. */
int wg_take_completed(wg_ctx* ctx, wg_query* ids, size_t cap, size_t* n_out);

/* ---- completion and results ---------------------------------------------- */
/* Non-blocking: fills *st. */
int wg_poll(wg_ctx* ctx, wg_query q, wg_status* st);
/* Blocks until the query is DONE/FAILED or timeout_us elapses (0 = no limit).
 * Returns WG_OK, WG_E_NOT_READY on timeout, or the query's own error. */
int wg_wait(wg_ctx* ctx, wg_query q, uint64_t timeout_us);
/* Copy the result (sorted packed keys) into a HOST buffer of cap entries.
 * *n_out = result size; WG_E_CAPACITY (nothing copied) when cap < size. */
int wg_result_copy(wg_ctx* ctx, wg_query q, uint64_t* keys, size_t cap, size_t* n_out);
/* Same into a DEVICE buffer (stream-ordered; synchronises the stream). */
int wg_result_copy_device(wg_ctx* ctx, wg_query q, uint64_t* d_keys, size_t cap, size_t* n_out);
/* Digest of the result without copying it: sum over i of
 * mix64(keys[i] + i * 0x9E3779B97F4A7C15) mod 2^64, keys[i] the i-th sorted
 * packed tuple as wg_result_copy returns it and mix64 the output function of
 * SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).  Computed on the device; a
 * caller compares it with the same sum over a reference result (the
 * benchmarks check every batched and served result this way).  The paper has
 * no counterpart.  Synchronous.  Errors: WG_E_INVAL, WG_E_NOT_READY or the
 * query's own error, WG_E_NOMEM / WG_E_BUDGET, WG_E_CUDA. */
int wg_result_digest(wg_ctx* ctx, wg_query q, uint64_t* digest);
/* Per-iteration delta sizes |Delta^0|, ..., |Delta^iterations| (last entry 0
 * at the fixpoint) into a HOST buffer; WG_E_CAPACITY when cap is too small. */
int wg_result_iters(wg_ctx* ctx, wg_query q, uint64_t* delta_sizes, size_t cap, size_t* n_out);
/* Per-kernel statistics of a profiled query; WG_E_CAPACITY when cap is too small. */
int wg_result_profile(wg_ctx* ctx, wg_query q, wg_kernel_stat* stats, size_t cap,
                      size_t* n_out);
void wg_query_free(wg_ctx* ctx, wg_query q);

/* ---- tile shapes and the autotuner --------------------------------------
 * Three stages have a compiled choice of tile shape: the join count (delta
 * tuples per tile: 2,048 or 1,024), the join emit (merged items per tile --
 * one per group of 8 delta tuples plus the candidates: 4,096 or 2,048) and
 * the fused deduplication / set difference / merge pass (merged keys per
 * tile: 4,096 or 2,048 for 4-byte keys, 2,048 or 1,024 for 8-byte keys).
 * Sec. Fused Deduplication fixes its own workgroup tile (256 threads x 12
 * keys) for its hardware; here the shape is an engine setting, the same
 * results for every choice.  The radix-sort mode (wg_sort_mode below, which
 * includes the digit width) is tuned with them.
 *
 * wg_autotune: time each candidate on a profiled fixpoint of `edges` (kind
 * WG_TC or WG_SG; one warm-up run and one timed run per candidate, the join
 * count, the join emit, the radix sort and the fused stage timed with CUDA
 * events) and keep
 * the fastest choice of each stage in the context for the relation's key
 * width: every engine created afterwards (single, batched, served) uses it.  `out` may be
 * NULL.  Synchronous; runs on the context stream.  Errors: WG_E_INVAL (bad
 * handle or kind), WG_E_NOMEM / WG_E_BUDGET (a run's pools do not fit),
 * WG_E_CUDA.  On an error the context keeps its previous shapes.
 *
 * wg_set_tiles: set the shapes for key width key_bytes (4 or 8) directly,
 * e.g. from a saved wg_tune; 0 = the compiled default.  Errors: WG_E_INVAL
 * (a shape that is not one of the compiled candidates). */
typedef struct wg_tune {
  uint32_t key_bytes;           /* key width the shapes apply to */
  uint32_t count_tile;          /* chosen delta tuples per join-count tile */
  uint32_t fuse_tile;           /* chosen merged keys per fused-pass tile */
  uint32_t count_cand[2];       /* candidates (default first) */
  uint32_t fuse_cand[2];
  uint32_t sort_mode;           /* chosen enum wg_sort_mode (TC relations of at most
                                   2^18 vertices; otherwise the default, untimed) */
  uint32_t emit_tile;           /* chosen merged items (delta groups + candidates) per
                                   join-emit tile */
  uint32_t emit_cand[2];
  uint32_t reserved0;
  double count_ms[2];           /* join-count time per fixpoint, per candidate */
  double fuse_ms[2];            /* fused-stage time per fixpoint, per candidate */
  double sort_ms[4];            /* radix sort (histogram + passes) per fixpoint, per
                                   wg_sort_mode; 0 when not timed */
  double emit_ms[2];            /* join-emit time per fixpoint, per candidate */
} wg_tune;
int wg_autotune(wg_ctx* ctx, wg_rel edges, int kind, wg_tune* out);
int wg_set_tiles(wg_ctx* ctx, int key_bytes, uint32_t count_tile, uint32_t fuse_tile,
                 uint32_t emit_tile);

/* The radix sort of a single TC query's candidates (sorted per source on the
 * destination field, Sec. Buffer Routing and Adaptive Radix Sort): one CTA
 * takes a source's whole segment through every pass, with 16 or 8 keys per
 * thread and digits of at most 8 bits (used while no source has more than
 * 128 tiles of candidates in an iteration, else the decoupled-lookback
 * passes over all tiles), or only the lookback passes, or (SEGMENT_WIDE) one
 * CTA per segment, 8 keys per thread, with digits of up to 9 bits for every
 * segment -- two passes instead of three for the 17- and 18-bit fields of
 * relations of 2^16 to 2^18 vertices (the radix digit width of Sec. Buffer
 * Routing and Adaptive Radix Sort as a tuning choice).  The same result for
 * every mode.  wg_set_sort picks it for engines of key width key_bytes
 * created afterwards; wg_autotune times all four.  Errors: WG_E_INVAL. */
enum wg_sort_mode { WG_SORT_SEGMENT16 = 0, WG_SORT_SEGMENT8 = 1, WG_SORT_PASSES = 2,
                    WG_SORT_SEGMENT_WIDE = 3 };
int wg_set_sort(wg_ctx* ctx, int key_bytes, uint32_t mode);

/* ---- self-test of the bounded device wait --------------------------------
 * wg_selftest_wait_timeout: run the wait of the decoupled lookback (the one
 * every scan stage uses) against a predecessor that never publishes its
 * count.  The wait gives up after its poll limit (a second or a few),
 * records the timeout and the kernel returns, so the context stays usable.
 * The same wait then runs once in the control block of the allocation-free
 * sort (wg_sort_keys_noalloc), whose next check (a call with n = 0) reports
 * it; run it while no allocation-free sort is in flight.
 * Returns WG_E_DEVICE_TIMEOUT when the context's wait gave up (the expected
 * outcome), WG_OK if the wait completed, WG_E_NOMEM / WG_E_BUDGET / WG_E_CUDA. */
int wg_selftest_wait_timeout(wg_ctx* ctx);

/* ---- sorted-array primitives (the stages of one iteration) ---------------
 * Device buffers of packed keys, key_bytes = 4 (uint32) or 8 (uint64).  They
 * run on the context stream, use context scratch, and synchronise the stream
 * before returning sizes.
 *
 * wg_sort_keys: LSD radix sort of n keys on their low `bits` bits (1..64;
 * higher bits must be zero), in place (Sec. Buffer Routing and Adaptive Radix
 * Sort: histogram, prefix sum, scatter per digit).  Every pass after the
 * first is stable; keys equal on the sorted bits are identical, so the
 * result is the unique sorted sequence. */
int wg_sort_keys(wg_ctx* ctx, void* d_keys, size_t n, int key_bytes, uint32_t bits);
/* wg_unique_diff: out = { c in sorted `cand` : c differs from its predecessor
 * and c is not in sorted `full` } in input order (Sec. Fused Deduplication and
 * Set Difference).  n_full = 0 gives plain deduplication.  `out` holds n
 * entries; *n_out = survivors. */
int wg_unique_diff(wg_ctx* ctx, const void* d_cand, size_t n, const void* d_full, size_t n_full,
                   void* d_out, size_t* n_out, int key_bytes);
/* wg_merge_disjoint: out = merge of sorted a and sorted b, which share no key
 * (Sec. Disjoint Merge); out holds na + nb entries. */
int wg_merge_disjoint(wg_ctx* ctx, const void* d_a, size_t na, const void* d_b, size_t nb,
                      void* d_out, int key_bytes);

/* ---- triangle counting ----------------------------------------------------
 * wg_triangles: *count = the number of tuples (a, b, c) of
 *     triangle(a,b,c) <- edge(a,b), edge(b,c), edge(c,a)
 * over the relation's edge set (Sec. Generalization, "Triangle Counting"; a
 * single non-recursive pass).  Each edge (a,b) takes its deg(b) two-paths
 * from the join count, and each two-path (a,b,c) is tested for edge(c,a) by
 * binary search in c's sorted adjacency (the binary-search join).  A directed
 * 3-cycle gives 3 tuples, an undirected triangle (both directions of each
 * edge) 6, a self-loop (a,a,a) 1.  Synchronous on the context stream; scratch
 * is |E| * 8 bytes plus 8 bytes per 4,096 two-paths.  Errors: WG_E_INVAL (bad
 * argument or relation), WG_E_NOMEM / WG_E_BUDGET, WG_E_CAPACITY (more than
 * 2^44 two-paths), WG_E_DEVICE_TIMEOUT. */
int wg_triangles(wg_ctx* ctx, wg_rel edges, uint64_t* count);

/* ---- allocation-free radix sort ------------------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory -- code running inside another runtime's
 * memory arena, or a process that must not call cudaMalloc or any allocator
 * (PyTorch's included), e.g. to keep its device footprint fixed.  It performs
 * the same sort as wg_sort_keys (LSD radix sort of n keys on their low `bits`
 * bits, in place; key_bytes = 4 or 8; higher bits must be zero) but takes
 * no context and allocates nothing: its scratch (stage records, digit
 * histograms, lookback words and the ping-pong key buffer) is one fixed static
 * device array of WG_NOALLOC_SCRATCH_BYTES (8,934,912 bytes, 8.5 MiB) that every
 * GPU loading the library holds until the process exits.
 *  - n <= WG_NOALLOC_MAX_KEYS (1,048,576); a larger n returns WG_E_CAPACITY and
 *    touches nothing.
 *  - n = 0 (d_keys may be NULL) sorts nothing: it is the failure check.  It
 *    synchronises `cuda_stream` and returns WG_E_DEVICE_TIMEOUT if a call on this
 *    device gave up a bounded device wait since the last check (that call's keys
 *    are unspecified), else WG_OK, and clears the record.  Every sort call
 *    returns before its kernels run, so only this check can report such a
 *    failure.
 *  - Asynchronous on `cuda_stream` (a cudaStream_t; NULL = the legacy default
 *    stream) of the current device; the caller synchronises.
 *  - All calls share the scratch array, which keeps the previous call's
 *    contents (each call clears what must start at zero): calls whose work
 *    overlaps on the GPU race; keep them ordered, e.g. on one stream.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress): make that first call before any stream capture.
 * Errors: WG_E_INVAL (NULL keys with n > 0, bad key_bytes or bits),
 * WG_E_CAPACITY, WG_E_CUDA, WG_E_DEVICE_TIMEOUT (the check, n = 0). */
#define WG_NOALLOC_MAX_KEYS 1048576u
#define WG_NOALLOC_SCRATCH_BYTES 8934912u
int wg_sort_keys_noalloc(void* d_keys, size_t n, int key_bytes, uint32_t bits, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* WG_H */
