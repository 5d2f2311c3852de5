// wg_device.cuh -- device-resident descriptors and block primitives shared by
// the sm_103a kernels of the semi-naive fixpoint.
//
// Every kernel of the loop is "indirect": its grid is fixed (a persistent grid
// sized to the SM count) and it reads how much work there is, and where, from
// device memory written by the previous stage.  This is the CUDA counterpart of
// the paper's indirect dispatch (Sec. Batched Indirect-Dispatch Loop): stage
// sizes never travel to the host, so one iteration -- and the whole loop -- can
// be captured once in a CUDA graph.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wg {

constexpr int kThreads = 256;                 // every stage kernel
constexpr int kWarps = kThreads / 32;
constexpr int kItemsC = 16;                   // keys per thread, candidate stages
constexpr int kTileC = kThreads * kItemsC;    // 4096 keys per candidate tile
constexpr int kItemsD = 8;                    // delta tuples per thread, join count
constexpr int kTileD = kThreads * kItemsD;    // 2048 delta tuples per tile
constexpr int kTileM = 4096;                  // merge output tile
// Join-emit tiles count one item per kEmitGroup delta tuples besides the
// candidates, so a tile holds at most kEmitGroup * kTileC delta tuples
// however many of their slabs are empty.
constexpr uint32_t kEmitGroupShift = 3;
constexpr uint32_t kEmitGroup = 1u << kEmitGroupShift;
constexpr int kRadix = 256;                   // digit buckets (digits of <= 8 bits)
constexpr int kMaxPasses = 8;
constexpr int kFWin = 2048;                   // full-relation keys staged by dedup/diff
constexpr uint32_t kSpinLimit = 1u << 22;     // polls before a lookback gives up

// device error codes (mirrored to WG_E_* on the host)
enum : uint32_t { DEV_OK = 0, DEV_TIMEOUT = 1 };

// instance states
enum : uint32_t { INST_FREE = 0, INST_ACTIVE = 1, INST_DONE = 2, INST_ITERCAP = 3 };
enum : uint32_t { KIND_TC = 0, KIND_SG = 1 };

// Control block of one engine.
struct Ctl {
  uint32_t abort;      // nonzero: every later kernel of this run returns at once
  uint32_t error;      // DEV_* set by a wait that gave up
  uint32_t epoch;      // lookback epoch, bumped once per lookback launch
  uint32_t cont;       // loop continues (mirrors the graph conditional)
  uint32_t launch_iters;  // iterations run in the current graph launch
  uint32_t iter_budget;   // per-launch iteration budget
  uint32_t n_active;
  uint32_t pad;
  unsigned long long need_cand;  // tuples needed in the candidate pools after an overflow
  unsigned long long need_full;
  unsigned long long need_res;
};

// One segment (one instance's part) of a segmented stage.
struct Seg {
  unsigned long long in_off, n;        // input range in the input pool
  unsigned long long out_off;          // output offset in the output pool
  unsigned long long aux_off, aux_n;   // auxiliary sorted range (full relation / delta)
  unsigned long long res;              // produced count (written by the stage)
  unsigned long long out2_off;         // second output offset (fused diff-merge: Full')
  uint32_t tile0, ntiles;              // global tiles [tile0, tile0 + ntiles)
  uint32_t inst, flags;                // owning instance; flags & 1: output to out2
};

// One launch's work: indirect grid, pools, lookback scratch.
struct Stage {
  const void* in;
  void* out;
  const void* aux;
  void* out2;
  Seg* segs;
  struct Inst* inst;
  Ctl* ctl;
  unsigned long long* status;   // lookback words
  unsigned long long* hist;     // radix digit counts [nseg][passes][kRadix]
  unsigned long long* pos;      // join prefix sums (one per delta tuple)
  unsigned long long* splits;   // per-tile start found by a partition kernel (or NULL)
  unsigned long long* splits2;  // join emit over merged tiles: each tile's first candidate
                                // (or NULL: a tile is kTileC consecutive candidates)
  unsigned long long* xlen;     // join count: candidates per source x (or NULL)
  uint32_t* tile_seg;           // tile -> segment map (or NULL: binary search)
  unsigned long long hist_n;    // join count: histogram counters to clear
  uint32_t nseg, ntiles;
  uint32_t ctr;                 // dynamic tile counter (zeroed by the writer)
  uint32_t epoch;
  uint32_t shift, dbits, pass, passes;
  unsigned long long* probe;    // join emit, triangle mode: count of candidates (a,b,c)
                                // with E(c,a) (nothing is written)
  const unsigned long long* htab;  // hash-join ablation: linear-probing table of E (or NULL)
  unsigned long long hmask;        // table slots - 1 (a power of two minus one)
  // fused pass: tiles holding candidates ("mixed"), listed after the
  // partition; the others hold Full elements only and are copied separately
  const uint32_t* mixl;            // mixed tiles in order (or NULL: every tile)
  const uint32_t* mixc;            // mixed tiles before tile t; [ntiles] = their number
  // radix sort: the largest segment's tile count (or NULL).  At most
  // kSegSortMaxTiles: one CTA per segment sorts the launch (k_sort_seg) and
  // the lookback passes have nothing to do; otherwise the reverse.
  const uint32_t* maxt;
  // per-segment sort: the non-empty segments in claim order -- those of at
  // least kSegBig tiles from the front (order_n[0] of them), the others from
  // the back (order_n[1]) -- or NULL: every segment, claimed by scanning.
  const uint32_t* order;
  const uint32_t* order_n;
};

// Hash-join ablation (the hash-based join the paper's sorted-array join
// replaces, Sec. "Data Skew in Hash-Based Join"): E in an open-addressing
// table with linear probing, entry = (src rank << 32) | dst rank, keyed by
// the source, empty slots all ones.  Every edge of a source lies in the
// cluster that starts at its hash slot, before the first empty slot.
constexpr unsigned long long kHashEmpty = ~0ull;
__device__ __forceinline__ unsigned long long hash_slot(uint32_t key, unsigned long long mask) {
  return (((unsigned long long)key * 0x9E3779B97F4A7C15ull) >> 29) & mask;
}

// One fixpoint instance (a query in flight).
struct Inst {
  const uint32_t* off;    // CSR offsets over source ranks [nv + 1]
  const uint32_t* adj;    // destination ranks, sorted within each source [ne]
  uint32_t nv, w;         // distinct vertices, bits per field
  uint32_t kind, state;
  uint32_t iter;          // index of the pass about to run (0 = base rule)
  uint32_t max_iters;
  unsigned long long n_delta, n_full, n_cand, n_new;
  unsigned long long d_off, f_off, c_off;
  unsigned long long res_off;  // final relation: pool res_pool at res_off
  uint32_t res_pool, iters_done;
  unsigned long long cand_total;
  unsigned long long* log;     // |Delta^0|, |Delta^1|, ...
  uint32_t log_cap;
  uint32_t fresh;              // admitted, delta not yet initialised
  // Full kept as two sorted runs (single-query fused engines): the main run
  // (n_full - n_side keys in pool F at f_off) and a side run of the newest
  // tuples (n_side keys in pool G[gphase] at 0), disjoint.  An iteration with
  // few candidates (side_iter) takes its new tuples against both runs and
  // merges them into the side run only; the main run is rewritten only when
  // the side run is folded back (a pre-merge, or the final merge).
  unsigned long long n_side;
  unsigned long long n_new0;   // side iteration: candidates not in the main run (deduplicated)
  uint32_t gphase, side_iter;
};

// Stage slots of an engine (one Stage record per kernel of the iteration).
// S_FUSE2: the side run's fused pass; S_PREM: folding the side run into the main run.
// The radix sort alone uses the stages below S_SORT_END.
enum StageId : int { S_COUNT = 0, S_EMIT, S_HIST, S_UNIQ, S_MERGE, S_FUSE, S_PASS0,
                     S_SORT_END = S_PASS0 + kMaxPasses, S_FUSE2 = S_SORT_END, S_PREM, S_NUM };

// Full-relation window staged by dedup + diff (separate-stage mode).
template <typename K> struct FWin { static constexpr int n = sizeof(K) == 4 ? 2048 : 1024; };

// Tile of the fused dedup + set difference + merge: 16 KB of keys by default
// (half of it is the other compiled shape the autotuner may pick).
template <typename K> struct FuseTile {
  static constexpr int T = sizeof(K) == 4 ? 4096 : 2048;
  static constexpr int E = T / kThreads;
};

// Side-run iterations: taken when the candidates are at most 1/kSideRatio of
// the main run (the main run then is mostly copied, not merged) and the side
// run plus the candidates fit its pool.
constexpr unsigned long long kSideRatio = 8;

// Per-segment radix sort (k_sort_seg): used when no segment has more tiles.
constexpr uint32_t kSegSortMaxTiles = 128;
// segments of at least this many tiles are claimed first (the long ones must
// not start last)
constexpr uint32_t kSegBig = 16;

// x-grouped sort: relations of up to kXSegMaxVertices vertices, segment
// records built by chunks of kXChunk source vertices.
constexpr uint32_t kXSegMaxVertices = 1u << 18;
constexpr uint32_t kXChunk = 256;
constexpr uint32_t kXChunks = kXSegMaxVertices / kXChunk;

// Device-resident state of one engine: pools, the instance table, the stage
// records the plan kernels write, and the graph conditional handle.  Pools are
// reached through this block only, so growing a pool never re-captures the graph.
struct Dev {
  Ctl ctl;
  Stage st[S_NUM];
  Inst* inst;
  Seg* segD;  // join count: delta per instance
  Seg* segE;  // join emit
  Seg* segS;  // radix sort
  Seg* segU;  // dedup + diff
  Seg* segM;  // merge (separate mode) / retire copy (fused mode)
  Seg* segF;  // fused dedup + diff + merge
  Seg* segF2; // the side run's fused pass
  void* D[2];  // delta / new-delta pools (swap every iteration)
  void* C[2];  // candidate pools (radix ping-pong)
  void* F[2];  // full relation pools (swap every iteration)
  void* R;     // retired results (batch engines)
  unsigned long long capC, capF, capR;
  unsigned long long* pos;            // join prefix sums, capC entries
  unsigned long long* status_scalar;  // lookback words of scalar scans
  unsigned long long* status_sort;    // lookback words of radix passes
  unsigned long long* hist;           // [n_inst][passes][kRadix]
  unsigned long long* splits;         // tile partitions, as many entries as status_scalar
  unsigned long long* csplits;        // join emit: first candidate of each merged tile
  unsigned long long* xlen;           // candidates per source vertex (x-grouped sort)
  Seg* segX;                          // one sort segment per source vertex
  uint32_t* tile_seg;                 // tile -> x-segment map of the x-grouped sort
  uint32_t* xord;                     // x-segments in claim order (see Stage::order)
  unsigned long long* xsum;           // [kXChunks][2]: candidates and tiles per chunk of x
  const unsigned long long* htab;     // hash-join ablation: the relation's table (or NULL)
  unsigned long long hmask;
  uint32_t* mixl;                     // fused pass: mixed tile list [tiles]
  uint32_t* mixc;                     // mixed tiles before each tile [tiles + 1]
  uint32_t* mixs;                     // mixed tiles per chunk of kThreads tiles
  void* G[2];                         // side-run pools (swap at every side iteration)
  unsigned long long capG;            // keys each side-run pool holds
  unsigned long long mix_cap;         // tiles the per-tile arrays hold
  unsigned long long r_used;
  unsigned long long cond;            // cudaGraphConditionalHandle
  uint32_t n_inst, single, use_cond, fuse, fuse_tile;
  uint32_t xseg;                      // sort each source's candidates on the low field only
  uint32_t copyback;                  // single fused engine: copy Full' back into the Full
                                      // buffer each iteration instead of swapping buffers
  uint32_t count_tile;                // delta tuples per join-count tile
  uint32_t emit_tile;                 // merged items per join-emit tile
  uint32_t seg_sort;                  // x-grouped: the per-segment sort may take the launch
  uint32_t dphase, fphase;
  uint32_t bits, passes, dbits;
  uint32_t xseg_maxt;                 // x-grouped sort: tiles of the largest source segment
  uint32_t side;                      // side run: 0 never, 1 when the candidates are few,
                                      // 2 whenever it fits (tests)
  uint32_t xord_n[2];                 // big / small x-segments listed in xord
  uint32_t seg_wide;                  // x-grouped: the per-segment sort with 9-bit digits
                                      // takes every launch (no lookback passes)
  uint32_t zero_word;                 // always 0 (the largest segment "size" of seg_wide)
};

// Shared-memory index with one pad word per 32: threads that walk their own
// contiguous run (blocked order, stride 16 words) then hit distinct banks.
__device__ __forceinline__ uint32_t pad32(uint32_t i) { return i + (i >> 5); }
template <int N> struct Padded { static constexpr int n = N + N / 32 + 1; };

// Copy n <= kThreads*ITEMS consecutive elements to shared memory with every
// global load in flight at once: a fixed-trip, predicated, unrolled loop
// (a loop bounded by n would pay one load latency per iteration).
template <int ITEMS, typename T, typename Idx>
__device__ __forceinline__ void tile_to_smem(T* dst, const T* src, uint32_t n, Idx idx) {
  T v[ITEMS];
#pragma unroll
  for (int e = 0; e < ITEMS; ++e) {
    const uint32_t i = threadIdx.x + e * kThreads;
    v[e] = i < n ? src[i] : (T)0;
  }
#pragma unroll
  for (int e = 0; e < ITEMS; ++e) {
    const uint32_t i = threadIdx.x + e * kThreads;
    if (i < n) dst[idx(i)] = v[e];
  }
}
struct Ident { __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return i; } };
struct Pad32 { __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return i + (i >> 5); } };

// ---------------------------------------------------------------- status words
// [63:40] epoch (24 bits) | [39:38] flag | [37:0] value
constexpr unsigned long long kValMask = (1ull << 38) - 1;
constexpr uint32_t FLAG_AGG = 1, FLAG_INC = 2;

__device__ __forceinline__ unsigned long long st_pack(uint32_t epoch, uint32_t flag,
                                                      unsigned long long v) {
  return ((unsigned long long)(epoch & 0xFFFFFFu) << 40) | ((unsigned long long)flag << 38) |
         (v & kValMask);
}
__device__ __forceinline__ void st_put(unsigned long long* p, unsigned long long v) {
  *(volatile unsigned long long*)p = v;
}
__device__ __forceinline__ unsigned long long st_get(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}
__device__ __forceinline__ bool st_ready(unsigned long long s, uint32_t epoch) {
  return (uint32_t)(s >> 40) == (epoch & 0xFFFFFFu) && ((s >> 38) & 3u) != 0;
}

__device__ __forceinline__ void fail_timeout(Ctl* ctl) {
  atomicExch(&ctl->error, DEV_TIMEOUT);
  atomicExch(&ctl->abort, 1u);
}

// Warp-cooperative decoupled lookback (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016): exclusive prefix of
// tile t over tiles [t0, t).  Every lane of the calling warp participates.
// Each poll is bounded; on timeout the control block records DEV_TIMEOUT and
// the returned value is meaningless (the run is void).
__device__ __forceinline__ unsigned long long lookback_scalar(const unsigned long long* status,
                                                              uint32_t t, uint32_t t0,
                                                              uint32_t epoch, Ctl* ctl) {
  const uint32_t lane = threadIdx.x & 31;
  unsigned long long excl = 0;
  long long base = (long long)t - 1;
  while (base >= (long long)t0) {
    long long idx = base - lane;
    unsigned long long s;
    uint32_t flag, timed_out = 0;
    if (idx >= (long long)t0) {
      uint32_t spins = 0;
      s = st_get(status + idx);
      while (!st_ready(s, epoch)) {
        if (++spins > kSpinLimit || *(volatile uint32_t*)&ctl->abort) { timed_out = 1; break; }
        __nanosleep(64);
        s = st_get(status + idx);
      }
      flag = (uint32_t)(s >> 38) & 3u;
    } else {
      s = 0;
      flag = FLAG_INC;  // before the segment: an inclusive zero
    }
    if (__any_sync(0xffffffffu, timed_out)) {
      if (lane == 0 && !*(volatile uint32_t*)&ctl->abort) fail_timeout(ctl);
      return 0;
    }
    unsigned long long v = s & kValMask;
    uint32_t inc = __ballot_sync(0xffffffffu, flag == FLAG_INC);
    uint32_t upto = inc ? (uint32_t)(__ffs(inc) - 1) : 31u;
    unsigned long long mine = lane <= upto ? v : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    excl += mine;
    if (inc) break;
    base -= 32;
  }
  return excl;
}

// Block-wide exclusive scan of one 64-bit value per thread; *total = block sum.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* sh /*kWarps*/,
                                                              unsigned long long* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < (uint32_t)kWarps ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    if (lane < (uint32_t)kWarps) sh[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  unsigned long long wp = warp ? sh[warp - 1] : 0ull;
  *total = sh[kWarps - 1];
  __syncthreads();
  return wp + x - v;
}

// Global tile -> segment: the segment k with tile0 <= t < tile0 + ntiles.
__device__ __forceinline__ uint32_t find_seg(const Seg* segs, uint32_t nseg, uint32_t t,
                                             const uint32_t* tile_seg = nullptr) {
  if (tile_seg) return tile_seg[t];
  uint32_t lo = 0, hi = nseg;  // largest k with tile0 <= t
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (segs[mid].tile0 <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Dynamic tile claim: thread 0 takes the next tile; returns it to every thread.
__device__ __forceinline__ uint32_t claim_tile(Stage* stp, uint32_t* sh) {
  __syncthreads();
  if (threadIdx.x == 0) *sh = atomicAdd(&stp->ctr, 1u);
  __syncthreads();
  return *sh;
}

template <typename K>
__device__ __forceinline__ unsigned long long lower_bound_k(const K* a, unsigned long long n, K x) {
  unsigned long long lo = 0, hi = n;
  while (lo < hi) {
    unsigned long long mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
template <typename K>
__device__ __forceinline__ unsigned long long upper_bound_k(const K* a, unsigned long long n, K x) {
  unsigned long long lo = 0, hi = n;
  while (lo < hi) {
    unsigned long long mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace wg
