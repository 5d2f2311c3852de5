// wg_kern_join.cu -- the join of one semi-naive iteration and the engine's
// device-side control (sm_103a).
//
// Join (Sec. Binary-Search Join, "Two-phase algorithm"): a count phase gives
// every delta tuple the size of its output slab -- for TC the out-degree of its
// destination, for SG the product of the two out-degrees -- and a single-pass
// scan (decoupled lookback) turns the counts into slab offsets; the emit phase
// writes every candidate into its slab with no atomics.  The edge relation is
// sorted once at load and indexed by source (CSR offsets), so the range lookup
// is two loads instead of a binary search.  Emit is partitioned by OUTPUT
// position (load-balanced search over the slab offsets), so a hub with
// thousands of edges is spread over many threads instead of serialising one.
//
// Plan kernels (one CTA) are the CUDA form of the paper's lightweight
// dispatch-parameter kernel (Sec. Batched Indirect-Dispatch Loop): they read
// the sizes the previous stage left in device memory and write the next
// stage's work description.  plan_post (fused stages) / plan_merge (separate
// stages) also make the termination decision (Sec. Background, step 5) and
// set the graph's WHILE condition.  The x-segment kernels build the per-source
// sort segments of single TC queries.
//
// Also here: the emit kernel's probe mode for triangle counting (Sec.
// Generalization, "Triangle Counting") and the hash-join ablation (a
// linear-probing table of E, Sec. "Data Skew in Hash-Based Join").
#include "wg_device.cuh"
#include "wg_launch.h"

namespace wg {

constexpr int kPlanThreads = 1024;

__device__ __forceinline__ unsigned long long scan1024(unsigned long long v, unsigned long long* sh,
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
    unsigned long long w = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  const unsigned long long wp = warp ? sh[warp - 1] : 0ull;
  *total = sh[31];
  __syncthreads();
  return wp + x - v;
}

__device__ __forceinline__ uint32_t deg(const uint32_t* off, uint32_t v) { return off[v + 1] - off[v]; }

// Hash-join ablation: number of entries with source y, walking y's cluster
// one dependent load at a time (the serialized probe chain of a hub).
__device__ __forceinline__ uint32_t hash_count(const unsigned long long* T,
                                               unsigned long long mask, uint32_t y) {
  uint32_t n = 0;
  unsigned long long s = hash_slot(y, mask);
  for (unsigned long long step = 0; step <= mask; ++step) {
    const unsigned long long e = T[s];
    if (e == kHashEmpty) break;
    n += (uint32_t)(e >> 32) == y;
    s = (s + 1) & mask;
  }
  return n;
}

// Build the table: one thread per edge claims a slot by compare-and-swap,
// moving to the next slot after every failure (the retry chains of a hub).
template <typename K>
__global__ void k_hash_build(const K* E, unsigned long long ne, uint32_t w,
                             unsigned long long* T, unsigned long long mask) {
  const K fmask = (K)(((K)1 << w) - 1);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t src = (uint32_t)(E[i] >> w), dst = (uint32_t)(E[i] & fmask);
    const unsigned long long entry = ((unsigned long long)src << 32) | dst;
    unsigned long long s = hash_slot(src, mask);
    for (unsigned long long step = 0; step <= mask; ++step) {  // the table is at most half full
      if (atomicCAS(T + s, kHashEmpty, entry) == kHashEmpty) break;
      s = (s + 1) & mask;
    }
  }
}

// Hash-join emit (TC): one thread per delta tuple (x, y) walks y's cluster
// again and writes (x, z) for every entry (y, z) into its slab -- the usual
// GPU hash join, not load-balanced over outputs.
template <typename K>
__global__ void __launch_bounds__(kThreads) k_join_emit_hash(Stage* stp) {
  if (*(volatile uint32_t*)&stp->ctl->abort) return;
  const K* D = (const K*)stp->in;
  K* C = (K*)stp->out;
  for (uint32_t k = 0; k < stp->nseg; ++k) {
    const Seg sg = stp->segs[k];
    const Inst* I = stp->inst + sg.inst;
    const uint32_t w = I->w;
    const K mask = (K)(((K)1 << w) - 1);
    const unsigned long long* P = stp->pos + sg.in_off;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         i < sg.n; i += (unsigned long long)gridDim.x * blockDim.x) {
      const K key = D[sg.in_off + i];
      const uint32_t x = (uint32_t)(key >> w), y = (uint32_t)(key & mask);
      K* o = C + sg.out_off + P[i];
      unsigned long long s = hash_slot(y, stp->hmask);
      for (unsigned long long step = 0; step <= stp->hmask; ++step) {
        const unsigned long long e = stp->htab[s];
        if (e == kHashEmpty) break;
        if ((uint32_t)(e >> 32) == y) *o++ = ((K)x << w) | (K)(uint32_t)e;
        s = (s + 1) & stp->hmask;
      }
    }
  }
}

// ------------------------------------------------------------------ join count
// ITEMS delta tuples per thread: a tile of kThreads * ITEMS (the tile shape
// is an engine setting the autotuner picks; kItemsD by default).
// Shared layouts padded against bank conflicts: each thread reads its ITEMS
// consecutive tuples (one pad word per 32 keys) and writes their 64-bit slab
// offsets (one pad offset per 16).
__device__ __forceinline__ uint32_t pad16(uint32_t i) { return i + (i >> 4); }
template <typename K, int ITEMS>
__global__ void __launch_bounds__(kThreads, 6) k_join_count(Stage* stp) {
  constexpr int kTile = kThreads * ITEMS;
  __shared__ K sd[Padded<kTile>::n];
  __shared__ unsigned long long sp[kTile + kTile / 16];
  __shared__ unsigned long long s_scan[kWarps];
  __shared__ unsigned long long s_excl;
  __shared__ uint32_t s_xprev, s_xnext;  // sources of the delta tuples around the tile
  __shared__ uint32_t s_t, s_bad;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  // the radix histogram of this iteration starts from zero
  const unsigned long long nz = stp->hist_n;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kThreads + threadIdx.x; i < nz;
       i += (unsigned long long)gridDim.x * kThreads)
    stp->hist[i] = 0;
  const K* D = (const K*)stp->in;
  unsigned long long* pos = stp->pos;
  const uint32_t nseg = stp->nseg, ntiles = stp->ntiles, epoch = stp->epoch;
  unsigned long long* status = stp->status;
  for (;;) {
    const uint32_t t = claim_tile(stp, &s_t);
    if (t >= ntiles) return;
    const uint32_t k = find_seg(stp->segs, nseg, t);
    const Seg sg = stp->segs[k];
    const Inst* I = stp->inst + sg.inst;
    const uint32_t* off = I->off;
    const uint32_t w = I->w, kind = I->kind, iter = I->iter;
    const K mask = (K)(((K)1 << w) - 1);
    const unsigned long long start = (unsigned long long)(t - sg.tile0) * kTile;
    const uint32_t n = (uint32_t)min((unsigned long long)kTile, sg.n - start);
    const K* p = D + sg.in_off + start;
    tile_to_smem<ITEMS>(sd, p, n, Pad32());
    if (threadIdx.x == 0) {
      s_bad = 0;
      s_xprev = start > 0 ? (uint32_t)(p[-1] >> w) : 0xFFFFFFFFu;
      s_xnext = start + n < sg.n ? (uint32_t)(p[n] >> w) : 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t b = threadIdx.x * ITEMS;
    unsigned long long c[ITEMS], sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      c[i] = 0;
      if (b + i < n) {
        const K key = sd[pad32(b + i)];
        const uint32_t x = (uint32_t)(key >> w), y = (uint32_t)(key & mask);
        if (kind == KIND_TC) {
          c[i] = stp->htab ? hash_count(stp->htab, stp->hmask, y) : deg(off, y);  // T(x,y), E(y,z)
        } else if (iter == 0) {
          const unsigned long long d = deg(off, x);            // E(p,x), E(p,y), x != y
          c[i] = d ? d * (d - 1) : 0;
        } else {
          c[i] = (unsigned long long)deg(off, x) * deg(off, y);  // E(a,x), sg(a,b), E(b,y)
        }
        sum += c[i];
      }
    }
    unsigned long long tot;
    const unsigned long long texcl = block_excl_scan(sum, s_scan, &tot);
    const bool first = (t == sg.tile0);
    if (threadIdx.x == 0) st_put(status + t, st_pack(epoch, first ? FLAG_INC : FLAG_AGG, tot));
    if (!first && threadIdx.x < 32) {
      const unsigned long long ex = lookback_scalar(status, t, sg.tile0, epoch, ctl);
      if (threadIdx.x == 0) {
        s_excl = ex;
        if (*(volatile uint32_t*)&ctl->abort) s_bad = 1;
        st_put(status + t, st_pack(epoch, FLAG_INC, ex + tot));
      }
    } else if (first && threadIdx.x == 0) {
      s_excl = 0;
    }
    __syncthreads();
    if (s_bad) return;
    unsigned long long run = s_excl + texcl;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      if (b + i < n) { sp[pad16(b + i)] = run; run += c[i]; }
    if (stp->xlen) {
      // candidates per source x.  Delta is sorted by x, so x's tuples are one
      // run and its total is (prefix at the run's end) - (prefix at its
      // start): one atomic where the run starts, one where it ends.
      unsigned long long r = s_excl + texcl;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        if (b + i < n) {
          const uint32_t x = (uint32_t)(sd[pad32(b + i)] >> w);
          const uint32_t xp = b + i > 0 ? (uint32_t)(sd[pad32(b + i - 1)] >> w) : s_xprev;
          const uint32_t xn = b + i + 1 < n ? (uint32_t)(sd[pad32(b + i + 1)] >> w) : s_xnext;
          if (x != xp) atomicAdd(stp->xlen + x, 0ull - r);
          r += c[i];
          if (x != xn) atomicAdd(stp->xlen + x, r);
        }
      }
    }
    __syncthreads();
    unsigned long long* q = pos + sg.in_off + start;
    for (uint32_t i = threadIdx.x; i < n; i += kThreads) q[i] = sp[pad16(i)];
    if (threadIdx.x == 0 && t == sg.tile0 + sg.ntiles - 1) stp->segs[k].res = s_excl + tot;
  }
}

// ------------------------------------------------------------------ join emit
// Load-balanced over output positions: a tile holds at most kTileC
// consecutive candidates of one instance (plus at most kEmitGroup * kTileC
// delta tuples, however many of their slabs are empty).  The delta tuples
// whose slabs cover the tile -- from the slab owner of the tile's first
// candidate to that of the next tile's first -- are taken in chunks of
// EmitWin<K>::n:
//  1. a chunk becomes a slab table in shared memory: tile-relative slab
//     start and the CSR offsets the slab reads (every load of the round in
//     flight at once);
//  2. every non-empty slab marks its first position in an owner array of
//     the tile's positions, and one block-wide max-scan fills in the slab of
//     every position (slab indices grow with their starts);
//  3. each thread takes positions tile_start + e * kThreads + lane order, so a
//     warp reads consecutive adjacency entries of a slab and stores 32
//     consecutive candidates: coalesced, without a staging copy.
// Most tiles take one chunk; a long run of empty slabs (sinks) takes more.
template <typename K> struct EmitWin {
  static constexpr int n = sizeof(K) == 4 ? 1536 : 1024;
};

// Block-wide inclusive max-scan of the owner array over the tile's IE *
// kThreads positions: each thread scans its IE consecutive entries, then the
// threads' maxima.
template <int IE>
__device__ __forceinline__ void owner_max_scan(uint16_t* own, uint32_t* s_w) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t b = threadIdx.x * IE;
  uint32_t v[IE];
  uint32_t m = 0;
#pragma unroll
  for (int e = 0; e < IE; ++e) {
    m = max(m, (uint32_t)own[b + e]);
    v[e] = m;
  }
  uint32_t x = m;  // inclusive warp max-scan of the thread maxima
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x = max(x, y);
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint32_t before = 0;  // max over the earlier warps and the earlier lanes
  for (uint32_t w = 0; w < warp; ++w) before = max(before, s_w[w]);
  const uint32_t prev = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane) before = max(before, prev);
#pragma unroll
  for (int e = 0; e < IE; ++e) own[b + e] = (uint16_t)max(before, v[e]);
}

// kProbe (triangle counting, Sec. Generalization "Triangle Counting"): the
// delta is E itself and every candidate (a, b, c) of E(a,b), E(b,c) is tested
// for E(c,a) by binary search in c's sorted adjacency -- the binary-search
// join probe -- and only the number of hits is kept.
// TE: items per tile (an engine setting the autotuner picks; kTileC by default).
template <typename K, bool kProbe, int TE = kTileC>
__global__ void __launch_bounds__(kThreads, 5) k_join_emit(Stage* stp) {
  constexpr int W = EmitWin<K>::n;
  constexpr int IE = TE / kThreads;  // positions per thread
  __shared__ uint32_t s_start[W];  // slab's first candidate, relative to the tile
  __shared__ uint32_t s_x[W];      // TC: x            SG: off[x]
  __shared__ uint32_t s_a[W];      // TC: adj index of the slab's candidate 0 of the tile
                                   // SG: off[y] (recursive rule)
  __shared__ uint32_t s_d[W];      // SG: divisor that splits a slab index in two
  __shared__ uint16_t s_own[TE];      // slab (chunk index) of each position
  __shared__ unsigned long long s_scan[kWarps];
  __shared__ uint32_t s_w[kWarps];
  __shared__ unsigned long long s_i0, s_i1, s_o0, s_o1;
  __shared__ uint32_t s_r0, s_ce, s_t, s_k;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  const K* D = (const K*)stp->in;
  K* C = (K*)stp->out;
  const unsigned long long* pos_all = stp->pos;
  const uint32_t nseg = stp->nseg, ntiles = stp->ntiles;
  // Thread 0 claims a tile and reads where it lies (segment, candidate range,
  // delta range) into shared memory.  It does so for the next tile while the
  // CTA works on the current one, so that chain of dependent loads is off the
  // critical path (tiles are independent: no lookback orders them).
  auto fetch = [&]() {
    const uint32_t t = atomicAdd(&stp->ctr, 1u);
    s_t = t;
    if (t >= ntiles) return;
    const uint32_t k = find_seg(stp->segs, nseg, t);
    const Seg& sg = stp->segs[k];
    const bool last_tile = t == sg.tile0 + sg.ntiles - 1;
    unsigned long long o0, o1;
    if (stp->splits2) {         // merged tiles (at most TE candidates each)
      o0 = stp->splits2[t];
      o1 = last_tile ? sg.aux_n : stp->splits2[t + 1];
    } else {
      o0 = (unsigned long long)(t - sg.tile0) * TE;
      o1 = min(o0 + (unsigned long long)TE, sg.aux_n);
    }
    // delta tuples i0..i1: every slab before i0 ends at or before o0 and
    // every slab after i1 starts after o1
    const unsigned long long* P = pos_all + sg.in_off;
    unsigned long long i0, i1;
    if (stp->splits) {
      i0 = stp->splits[t];
      i1 = last_tile ? sg.n - 1 : stp->splits[t + 1];
    } else {
      i0 = upper_bound_k(P, sg.n, o0) - 1;
      i1 = upper_bound_k(P, sg.n, o1 - 1) - 1;
    }
    s_k = k; s_o0 = o0; s_o1 = o1; s_i0 = i0; s_i1 = i1;
  };
  if (threadIdx.x == 0) fetch();
  __syncthreads();
  for (;;) {
    const uint32_t t = s_t;
    if (t >= ntiles) return;
    const uint32_t k = s_k;
    const unsigned long long o0 = s_o0, o1 = s_o1, i0 = s_i0, m = s_i1 - i0 + 1;
    __syncthreads();  // every thread has the tile; thread 0 fetches the next one
    if (threadIdx.x == 0) fetch();
    const Seg sg = stp->segs[k];
    const Inst* I = stp->inst + sg.inst;
    const uint32_t* off = I->off;
    const uint32_t* adj = I->adj;
    const uint32_t w = I->w, kind = I->kind, iter = I->iter;
    const bool tc = kind == KIND_TC;
    const K mask = (K)(((K)1 << w) - 1);
    const unsigned long long* P = pos_all + sg.in_off + i0;  // from the tile's first delta tuple
    const K* Dq = D + sg.in_off + i0;
    const uint32_t nout = (uint32_t)(o1 - o0);
    K* Cq = C + sg.out_off + o0;
    unsigned long long hits = 0;  // triangle mode
    for (unsigned long long c0 = 0; c0 < m; c0 += W) {
      const uint32_t mc = (uint32_t)min((unsigned long long)W, m - c0);
      {  // round 1: the chunk's slab table
        constexpr int kPer = (W + kThreads - 1) / kThreads;
        unsigned long long p[kPer];
        K key[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          const uint32_t i = threadIdx.x + e * kThreads;
          p[e] = i < mc ? P[c0 + i] : 0ull;
          key[e] = i < mc ? Dq[c0 + i] : (K)0;
        }
        if (threadIdx.x == 0)  // the chunk covers candidates [its first slab's start, s_ce)
          s_ce = c0 + mc < m ? (uint32_t)(P[c0 + mc] - o0) : nout;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          const uint32_t i = threadIdx.x + e * kThreads;
          // slab i0 starts at or before o0; slabs after it start inside (o0, o1]
          if (i < mc) s_start[i] = c0 == 0 && i == 0 ? 0u : (uint32_t)(p[e] - o0);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          const uint32_t i = threadIdx.x + e * kThreads;
          // an empty slab (sink of the join) needs no CSR offsets
          if (i < mc && s_start[i] < (i + 1 < mc ? s_start[i + 1] : s_ce)) {
            const bool head = c0 == 0 && i == 0;  // the slab owning the tile's first candidate
            const uint32_t x = (uint32_t)(key[e] >> w), y = (uint32_t)(key[e] & mask);
            const uint32_t r0 = head ? (uint32_t)(o0 - p[e]) : 0u;  // its candidates before the tile
            if (tc) {
              s_x[i] = x;
              s_a[i] = off[y] + r0;                                 // T(x,y), E(y,z)
            } else {
              const uint32_t ox = off[x];
              s_x[i] = ox;
              if (iter == 0) {
                s_a[i] = 0;
                s_d[i] = off[x + 1] - ox - 1;                       // distinct children of x
              } else {
                const uint32_t oy = off[y];
                s_a[i] = oy;
                s_d[i] = off[y + 1] - oy;                           // E(a,x), sg(a,b), E(b,y)
              }
              if (head) s_r0 = r0;
            }
          }
        }
      }
      __syncthreads();
      const uint32_t cs = s_start[0], ce = s_ce;  // this chunk's candidates [cs, ce)
      if (cs < ce) {  // (a chunk of empty slabs only has none)
        // round 2: each non-empty slab marks its first position
#pragma unroll
        for (int e = 0; e < IE; ++e) s_own[threadIdx.x * IE + e] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < mc; i += kThreads) {
          const uint32_t st = s_start[i], nx = i + 1 < mc ? s_start[i + 1] : ce;
          if (st < nx) s_own[st] = (uint16_t)i;
        }
        __syncthreads();
        owner_max_scan<IE>(s_own, s_w);
        __syncthreads();
        // round 3: positions in lane order, every load of a thread in flight
        if constexpr (kProbe) {
#pragma unroll
          for (int h = 0; h < IE; h += 4) {
            uint32_t a[4], lo[4], hi[4], end[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const uint32_t q = (h + g) * kThreads + threadIdx.x;
              const bool ok = q >= cs && q < ce;
              uint32_t c = 0;
              a[g] = 0;
              if (ok) {
                const uint32_t i = s_own[q];
                c = adj[s_a[i] + q - s_start[i]];
                a[g] = s_x[i];
              }
              lo[g] = ok ? off[c] : 0u;
              end[g] = ok ? off[c + 1] : 0u;
              hi[g] = end[g];
            }
            for (;;) {  // at most log2(max degree) + 1 rounds
              bool any = false;
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                if (lo[g] < hi[g]) {
                  const uint32_t mid = (lo[g] + hi[g]) >> 1;
                  if (adj[mid] < a[g]) lo[g] = mid + 1; else hi[g] = mid;
                  any = true;
                }
              }
              if (!any) break;
            }
#pragma unroll
            for (int g = 0; g < 4; ++g) hits += lo[g] < end[g] && adj[lo[g]] == a[g];
          }
        } else if (tc) {
          constexpr int kB = IE / 2;  // positions whose loads are in flight together
#pragma unroll
          for (int h = 0; h < IE; h += kB) {
            uint32_t u[kB], z[kB];
#pragma unroll
            for (int e = 0; e < kB; ++e) {
              const uint32_t q = (h + e) * kThreads + threadIdx.x;
              u[e] = 0;
              z[e] = 0;
              if (q >= cs && q < ce) {
                const uint32_t i = s_own[q];
                u[e] = s_x[i];
                z[e] = adj[s_a[i] + q - s_start[i]];
              }
            }
#pragma unroll
            for (int e = 0; e < kB; ++e) {
              const uint32_t q = (h + e) * kThreads + threadIdx.x;
              if (q >= cs && q < ce) Cq[q] = ((K)u[e] << w) | (K)z[e];
            }
          }
        } else {
          constexpr int kB = IE / 2;
#pragma unroll
          for (int h = 0; h < IE; h += kB) {
            uint32_t u[kB], z[kB];
#pragma unroll
            for (int e = 0; e < kB; ++e) {
              const uint32_t q = (h + e) * kThreads + threadIdx.x;
              u[e] = 0;
              z[e] = 0;
              if (q >= cs && q < ce) {
                const uint32_t i = s_own[q];
                const uint32_t rr = q - s_start[i] + (c0 == 0 && i == 0 ? s_r0 : 0u), d = s_d[i];
                const uint32_t qa = rr / d;
                uint32_t qb = rr - qa * d;
                if (iter == 0) qb += qb >= qa;
                u[e] = adj[s_x[i] + qa];
                z[e] = adj[(iter == 0 ? s_x[i] : s_a[i]) + qb];
              }
            }
#pragma unroll
            for (int e = 0; e < kB; ++e) {
              const uint32_t q = (h + e) * kThreads + threadIdx.x;
              if (q >= cs && q < ce) Cq[q] = ((K)u[e] << w) | (K)z[e];
            }
          }
        }
      }
      __syncthreads();  // the table and owners are read; the next chunk may overwrite them
      // The range ends at the slab holding the next tile's first candidate,
      // so it takes in a run of empty slabs that starts exactly at the tile's
      // end; once the next chunk starts at or past the end, it and every
      // later one emit nothing here.
      if (ce >= nout) break;
    }
    if constexpr (kProbe) {
      unsigned long long tot;
      block_excl_scan(hits, s_scan, &tot);
      if (threadIdx.x == 0 && tot) atomicAdd(stp->probe, tot);
    }
    __syncthreads();  // thread 0's fetch of the next tile is visible
  }
}

// ------------------------------------------------------------------ plan kernels
__global__ void __launch_bounds__(kPlanThreads) k_plan_delta(Dev* dv) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long s_carry;
  Ctl& ctl = dv->ctl;
  if (ctl.abort) return;
  const uint32_t N = dv->n_inst;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < N; base += kPlanThreads) {
    const uint32_t q = base + threadIdx.x;
    const bool valid = q < N;
    const Inst* I = valid ? dv->inst + q : nullptr;
    const bool act = valid && I->state == INST_ACTIVE;
    const unsigned long long nd = act ? I->n_delta : 0ull;
    const unsigned long long nt = (nd + dv->count_tile - 1) / dv->count_tile;
    unsigned long long tot;
    const unsigned long long ex = scan1024(nt, sh, &tot);
    if (valid) {
      Seg s{};
      s.in_off = I->d_off; s.n = nd; s.out_off = I->d_off; s.aux_off = 0; s.aux_n = 0; s.res = 0;
      s.tile0 = (uint32_t)(s_carry + ex); s.ntiles = (uint32_t)nt; s.inst = q; s.flags = 0;
      dv->segD[q] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  const uint32_t nvx = dv->xseg ? dv->inst[0].nv : 0u;
  for (uint32_t x = threadIdx.x; x < nvx; x += kPlanThreads) dv->xlen[x] = 0;
  if (threadIdx.x == 0) { dv->xseg_maxt = 0; dv->xord_n[0] = 0; dv->xord_n[1] = 0; }
  if (threadIdx.x == 0) {
    Stage& s = dv->st[S_COUNT];
    s.in = dv->D[dv->dphase]; s.out = nullptr; s.aux = nullptr; s.out2 = nullptr;
    s.segs = dv->segD; s.inst = dv->inst; s.ctl = &dv->ctl;
    s.status = dv->status_scalar; s.hist = dv->hist; s.pos = dv->pos;
    s.nseg = N; s.ntiles = (uint32_t)s_carry; s.ctr = 0; s.epoch = ++ctl.epoch;
    s.passes = dv->passes; s.dbits = dv->dbits; s.shift = 0; s.pass = 0;
    s.xlen = dv->xseg ? dv->xlen : nullptr;
    s.htab = dv->htab; s.hmask = dv->hmask;
    // (x-grouped: the segment builder zeroes the rows of non-empty sources)
    s.hist_n = dv->xseg ? 0ull : (unsigned long long)N * dv->passes * kRadix;
  }
}

// x-grouped sort (single TC instance): the join emits candidates grouped by
// source x in ascending order (Delta is sorted and each slab is contiguous),
// so sorting each x-group on the destination field sorts the whole array.
// Every source vertex becomes one sort segment: offsets and tile ranges from
// the per-x candidate totals the count kernel accumulated.
// Pass 1: candidates and tiles of each chunk of kXChunk source vertices.
__global__ void __launch_bounds__(kXChunk) k_xseg_sum(Dev* dv) {
  __shared__ unsigned long long sh[kXChunk / 32];
  if (dv->ctl.abort) return;
  const Inst& I = dv->inst[0];
  const uint32_t nv = I.state == INST_ACTIVE ? I.nv : 0u;
  const uint32_t x = blockIdx.x * kXChunk + threadIdx.x;
  if (blockIdx.x * kXChunk >= nv) return;
  const unsigned long long len = x < nv ? dv->xlen[x] : 0ull;
  unsigned long long tl, tt;
  block_excl_scan(len, sh, &tl);
  block_excl_scan((len + kTileC - 1) / kTileC, sh, &tt);
  if (threadIdx.x == 0) {
    dv->xsum[2 * blockIdx.x] = tl;
    dv->xsum[2 * blockIdx.x + 1] = tt;
  }
}

// Pass 2: one sort segment per source vertex (offsets from the chunk sums
// before it plus a scan inside the chunk), the tile -> segment map, and zeroed
// radix-histogram rows for the sources that have candidates.  The chunk that
// holds the last vertex points the sort stages at the new segments.
__global__ void __launch_bounds__(kXChunk) k_xseg_fill(Dev* dv) {
  __shared__ unsigned long long sh[kXChunk / 32];
  __shared__ unsigned long long slen[kXChunk];
  Ctl& ctl = dv->ctl;
  if (ctl.abort) return;
  const Inst& I = dv->inst[0];
  const uint32_t nv = I.state == INST_ACTIVE ? I.nv : 0u;
  const uint32_t nchunks = nv ? (nv + kXChunk - 1) / kXChunk : 1u;
  const uint32_t b = blockIdx.x;
  if (b >= nchunks) return;
  unsigned long long pl = 0, pt = 0, tl, tt;
  for (uint32_t j = threadIdx.x; j < b; j += kXChunk) {
    pl += dv->xsum[2 * j];
    pt += dv->xsum[2 * j + 1];
  }
  block_excl_scan(pl, sh, &pl);
  block_excl_scan(pt, sh, &pt);
  const uint32_t x = b * kXChunk + threadIdx.x;
  const unsigned long long len = x < nv ? dv->xlen[x] : 0ull;
  const unsigned long long nt = (len + kTileC - 1) / kTileC;
  const unsigned long long el = block_excl_scan(len, sh, &tl);
  const unsigned long long et = block_excl_scan(nt, sh, &tt);
  slen[threadIdx.x] = len;
  {  // the largest segment's tile count picks the sort kernel (k_sort_seg or the passes)
    const uint32_t wm = __reduce_max_sync(0xffffffffu, (uint32_t)min(nt, 0xFFFFFFFFull));
    if ((threadIdx.x & 31) == 0 && wm) atomicMax(&dv->xseg_maxt, wm);
  }
  {  // claim order of the per-segment sort: segments of at least kSegBig
     // tiles from the front of xord, the other non-empty ones from the back
    const bool big = nt >= kSegBig, small = nt > 0 && nt < kSegBig;  // (x >= nv: nt = 0)
    const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    const uint32_t mb = __ballot_sync(0xffffffffu, big), ms = __ballot_sync(0xffffffffu, small);
    uint32_t bb = 0, bs = 0;
    if (lane == 0) {
      if (mb) bb = atomicAdd(&dv->xord_n[0], (uint32_t)__popc(mb));
      if (ms) bs = atomicAdd(&dv->xord_n[1], (uint32_t)__popc(ms));
    }
    bb = __shfl_sync(0xffffffffu, bb, 0);
    bs = __shfl_sync(0xffffffffu, bs, 0);
    if (big) dv->xord[bb + __popc(mb & lt)] = x;
    if (small) dv->xord[nv - 1 - (bs + __popc(ms & lt))] = x;
  }
  if (x < nv) {
    const unsigned long long off = I.c_off + pl + el;
    const uint32_t tile0 = (uint32_t)(pt + et);
    Seg g{};
    g.in_off = off; g.n = len; g.out_off = off;
    g.tile0 = tile0; g.ntiles = (uint32_t)nt; g.inst = 0;
    dv->segX[x] = g;
    for (uint32_t j = 0; j < (uint32_t)nt; ++j) dv->tile_seg[tile0 + j] = x;
  }
  __syncthreads();
  // histogram rows of this chunk's non-empty sources start from zero
  const uint32_t row = dv->passes * kRadix;
  const uint32_t nx = min(kXChunk, nv - min(nv, b * kXChunk));
  unsigned long long* hrow = dv->hist + (unsigned long long)b * kXChunk * row;
  for (uint32_t i = threadIdx.x; i < nx * row; i += kXChunk)
    if (slen[i / row]) hrow[i] = 0;
  if (b == nchunks - 1 && threadIdx.x == 0) {
    const uint32_t ntiles = (uint32_t)(pt + tt);
    dv->st[S_HIST].segs = dv->segX; dv->st[S_HIST].nseg = nv;
    dv->st[S_HIST].ntiles = ntiles; dv->st[S_HIST].tile_seg = dv->tile_seg;
    // the per-segment sort when the engine uses it, for segments of at most
    // kSegSortMaxTiles tiles (with 9-bit digits for every segment: the
    // lookback passes take 8-bit digits only); else the lookback passes
    const uint32_t* mt = dv->seg_sort ? (dv->seg_wide ? &dv->zero_word : &dv->xseg_maxt) : nullptr;
    dv->st[S_HIST].maxt = mt;
    for (uint32_t p = 0; p < dv->passes; ++p) {
      dv->st[S_PASS0 + p].segs = dv->segX; dv->st[S_PASS0 + p].nseg = nv;
      dv->st[S_PASS0 + p].ntiles = ntiles; dv->st[S_PASS0 + p].tile_seg = dv->tile_seg;
      dv->st[S_PASS0 + p].maxt = mt;
      dv->st[S_PASS0 + p].order = dv->xord; dv->st[S_PASS0 + p].order_n = dv->xord_n;
    }
  }
}

__global__ void __launch_bounds__(kPlanThreads) k_plan_cand(Dev* dv) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long s_cc, s_ct, s_fc, s_ft, s_et, s_pt;
  __shared__ uint32_t s_side;
  Ctl& ctl = dv->ctl;
  if (ctl.abort) return;
  const uint32_t N = dv->n_inst;
  if (threadIdx.x == 0) { s_cc = 0; s_ct = 0; s_fc = 0; s_ft = 0; s_et = 0; s_pt = 0; s_side = 0; }
  __syncthreads();
  for (uint32_t base = 0; base < N; base += kPlanThreads) {
    const uint32_t q = base + threadIdx.x;
    const bool valid = q < N;
    Inst* I = valid ? dv->inst + q : nullptr;
    const bool act = valid && I->state == INST_ACTIVE;
    const unsigned long long nc = act ? dv->segD[q].res : 0ull;
    const unsigned long long nd = act ? I->n_delta : 0ull;
    const unsigned long long nt = (nc + kTileC - 1) / kTileC;
    // join emit: tiles over merged items (one per group of kEmitGroup delta
    // tuples, then their slabs' candidates), so long runs of empty slabs are
    // spread over tiles too
    const unsigned long long ng = (nd + kEmitGroup - 1) >> kEmitGroupShift;
    const unsigned long long te = dv->emit_tile;
    const unsigned long long net = nc ? (nc + ng + te - 1) / te : 0ull;
    unsigned long long totc, tott, tote;
    const unsigned long long exc = scan1024(nc, sh, &totc);
    const unsigned long long ext = scan1024(nt, sh, &tott);
    const unsigned long long exe = scan1024(net, sh, &tote);
    if (valid) {
      const unsigned long long c_off = s_cc + exc;
      const uint32_t tile0 = (uint32_t)(s_ct + ext);
      I->n_cand = nc;
      I->c_off = c_off;
      Seg e{};
      e.in_off = I->d_off; e.n = nd; e.out_off = c_off;
      e.aux_off = 0; e.aux_n = nc; e.res = 0;
      e.tile0 = (uint32_t)(s_et + exe); e.ntiles = (uint32_t)net;
      e.inst = q; e.flags = 0;
      dv->segE[q] = e;
      Seg s = e;
      s.in_off = c_off; s.n = nc; s.aux_n = 0; s.tile0 = tile0; s.ntiles = (uint32_t)nt;
      dv->segS[q] = s;
      Seg u = s;
      u.aux_off = I->f_off; u.aux_n = act ? I->n_full : 0ull;
      dv->segU[q] = u;
    }
    if (dv->fuse) {
      // fused dedup + diff + merge: Full' of q at an upper bound |Full| + |C|
      const unsigned long long nf = act ? I->n_full : 0ull, tf = dv->fuse_tile;
      // Full as a main run and a side run (single-query engines, see Inst):
      // with few candidates the pass reads the main run only and writes no
      // Full' (k_plan_side then takes the side run); otherwise a side run
      // left from earlier iterations is first merged into the main run
      const unsigned long long ns = act ? I->n_side : 0ull, nf0 = nf - ns;
      const bool side = dv->side && act && ns + nc <= dv->capG &&
                        (ns + nc + tf - 1) / tf <= dv->mix_cap &&
                        (dv->side == 2 || nc * kSideRatio <= nf0);
      const bool prem = dv->side && act && !side && ns > 0;
      const unsigned long long nfa = side ? nf0 : nf;  // keys of the run the pass reads
      const unsigned long long ft = (nfa + nc + tf - 1) / tf;
      unsigned long long totf, totft;
      const unsigned long long exf = scan1024(nf + nc, sh, &totf);
      const unsigned long long exft = scan1024(ft, sh, &totft);
      if (valid) {
        Seg f{};
        f.in_off = I->f_off; f.n = nfa; f.aux_off = s_cc + exc; f.aux_n = nc;
        f.out_off = s_cc + exc; f.out2_off = s_fc + exf; f.res = 0;
        f.tile0 = (uint32_t)(s_ft + exft); f.ntiles = (uint32_t)ft; f.inst = q; f.flags = 0;
        dv->segF[q] = f;
        if (act) I->side_iter = side ? 1u : 0u;
      }
      if (prem) {  // both runs into the other Full pool at the same offset (one instance)
        Seg m{};
        m.in_off = I->f_off; m.n = nf0; m.aux_off = 0; m.aux_n = ns; m.out_off = I->f_off;
        m.res = 0; m.tile0 = 0; m.ntiles = (uint32_t)((nf + kTileM - 1) / kTileM); m.inst = q;
        m.flags = 0;
        dv->segM[q] = m;
        s_pt = m.ntiles;  // capacity: the merged run is the nf of the check below
      }
      if (side) s_side = 1;
      __syncthreads();
      if (threadIdx.x == 0) { s_fc += totf; s_ft += totft; }
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_cc += totc; s_ct += tott; s_et += tote; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (s_cc > dv->capC || (dv->fuse && s_fc > dv->capF)) {
      // candidates or Full' might not fit: stop before anything is written
      if (s_cc > dv->capC) ctl.need_cand = s_cc;
      if (dv->fuse && s_fc > dv->capF) ctl.need_full = s_fc;
      ctl.abort = 1;
      return;
    }
    const uint32_t nt = (uint32_t)s_ct;
    Stage base{};
    base.segs = dv->segS; base.inst = dv->inst; base.ctl = &dv->ctl; base.hist = dv->hist;
    base.pos = dv->pos; base.nseg = N; base.ntiles = nt; base.ctr = 0;
    base.passes = dv->passes; base.dbits = dv->dbits;
    Stage e = base;
    e.in = dv->D[dv->dphase]; e.out = dv->C[0]; e.segs = dv->segE; e.splits = dv->splits;
    e.splits2 = dv->csplits; e.ntiles = (uint32_t)s_et;
    e.htab = dv->htab; e.hmask = dv->hmask;
    dv->st[S_EMIT] = e;
    Stage h = base;
    h.in = dv->C[0];
    dv->st[S_HIST] = h;
    for (uint32_t p = 0; p < dv->passes; ++p) {
      Stage s = base;
      s.in = dv->C[p & 1]; s.out = dv->C[(p + 1) & 1];
      s.status = dv->status_sort; s.shift = p * dv->dbits; s.pass = p; s.epoch = ++ctl.epoch;
      dv->st[S_PASS0 + p] = s;
    }
    for (uint32_t p = dv->passes; p < kMaxPasses; ++p) {
      // digits above every active instance's keys: launched, but no tiles
      Stage s = base;
      s.ntiles = 0;
      dv->st[S_PASS0 + p] = s;
    }
    if (dv->fuse) {
      uint32_t fph = dv->fphase;
      Stage pm = base;
      pm.segs = dv->segM; pm.ntiles = 0;
      if (s_pt) {  // fold the side run into the main run before the pass (one instance)
        const Inst& I0 = dv->inst[0];
        pm.in = dv->F[fph]; pm.aux = dv->G[I0.gphase]; pm.out = dv->F[fph ^ 1];
        pm.ntiles = (uint32_t)s_pt; pm.splits = dv->splits;  // k_partition finds the tile splits
        dv->inst[0].n_side = 0;
        fph ^= 1u;
        dv->fphase = fph;
      }
      dv->st[S_PREM] = pm;
      Stage f = base;
      f.in = dv->F[fph]; f.aux = dv->C[dv->passes & 1];
      if (s_side) {  // new w.r.t. the main run into the spare candidate pool; no Full'
        f.out = dv->C[(dv->passes & 1) ^ 1]; f.out2 = nullptr;
      } else {
        f.out = dv->D[dv->dphase ^ 1]; f.out2 = dv->F[fph ^ 1];
      }
      f.segs = dv->segF; f.status = dv->status_scalar; f.epoch = ++ctl.epoch;
      f.ntiles = (uint32_t)s_ft; f.splits = dv->splits;
      f.mixl = dv->mixl; f.mixc = dv->mixc;
      dv->st[S_FUSE] = f;
    } else {
      Stage u = base;
      u.in = dv->C[dv->passes & 1]; u.aux = dv->F[dv->fphase]; u.out = dv->D[dv->dphase ^ 1];
      u.segs = dv->segU; u.status = dv->status_scalar; u.epoch = ++ctl.epoch;
      dv->st[S_UNIQ] = u;
    }
  }
}

__device__ __forceinline__ void set_continue(Dev* dv, uint32_t v) {
  dv->ctl.cont = v;
  if (dv->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)dv->cond, v);
}

__global__ void __launch_bounds__(kPlanThreads) k_plan_merge(Dev* dv) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long s_f, s_r, s_t, s_act;
  Ctl& ctl = dv->ctl;
  if (ctl.abort) {
    if (threadIdx.x == 0) set_continue(dv, 0);
    return;
  }
  const uint32_t N = dv->n_inst;
  const bool single = dv->single != 0;
  // pass 1: sizes only, so that a capacity overflow leaves the state untouched
  if (threadIdx.x == 0) { s_f = 0; s_r = 0; }
  __syncthreads();
  for (uint32_t base = 0; base < N; base += kPlanThreads) {
    const uint32_t q = base + threadIdx.x;
    unsigned long long fsz = 0, rsz = 0;
    if (q < N) {
      const Inst* I = dv->inst + q;
      if (I->state == INST_ACTIVE) {
        const unsigned long long nn = dv->segU[q].res, nf = I->n_full + nn;
        const bool done = I->iter >= 1 && nn == 0;
        const bool fin = done || I->iter >= I->max_iters;
        if (done && single) {
          // the full relation is final where it is
        } else if (fin && !single) {
          rsz = nf;
        } else {
          fsz = nf;
        }
      }
    }
    unsigned long long tf, tr;
    scan1024(fsz, sh, &tf);
    scan1024(rsz, sh, &tr);
    if (threadIdx.x == 0) { s_f += tf; s_r += tr; }
    __syncthreads();
  }
  if (s_f > dv->capF || dv->r_used + s_r > dv->capR) {
    if (threadIdx.x == 0) {
      ctl.need_full = s_f;
      ctl.need_res = dv->r_used + s_r;
      ctl.abort = 1;
      set_continue(dv, 0);
    }
    return;
  }
  // pass 2: commit the iteration
  const uint32_t fph = dv->fphase, dph = dv->dphase;
  if (threadIdx.x == 0) { s_f = 0; s_r = dv->r_used; s_t = 0; s_act = 0; }
  __syncthreads();
  for (uint32_t base = 0; base < N; base += kPlanThreads) {
    const uint32_t q = base + threadIdx.x;
    const bool valid = q < N;
    Inst* I = valid ? dv->inst + q : nullptr;
    const bool act = valid && I->state == INST_ACTIVE;
    unsigned long long nn = 0, nf = 0, fsz = 0, rsz = 0, mt = 0;
    bool fin = false, done = false, toR = false, keep = false;
    if (act) {
      nn = dv->segU[q].res;
      nf = I->n_full + nn;
      done = I->iter >= 1 && nn == 0;
      fin = done || I->iter >= I->max_iters;
      keep = done && single;  // nothing to merge and nothing runs after it
      toR = fin && !single;
      if (keep) {
      } else if (toR) {
        rsz = nf;
      } else {
        fsz = nf;
      }
      mt = keep ? 0ull : (nf + kTileM - 1) / kTileM;
    }
    unsigned long long tf, tr, tt, ta;
    const unsigned long long exf = scan1024(fsz, sh, &tf);
    const unsigned long long exr = scan1024(rsz, sh, &tr);
    const unsigned long long ext = scan1024(mt, sh, &tt);
    const unsigned long long exa = scan1024((act && !fin) ? 1ull : 0ull, sh, &ta);
    (void)exa;
    if (valid) {
      Seg m{};
      m.in_off = I->f_off; m.n = act ? I->n_full : 0ull; m.aux_off = I->c_off; m.aux_n = nn;
      m.res = 0; m.tile0 = (uint32_t)(s_t + ext); m.ntiles = (uint32_t)mt; m.inst = q;
      m.flags = toR ? 1u : 0u;
      const unsigned long long dst_off = keep ? I->f_off : (toR ? s_r + exr : s_f + exf);
      m.out_off = dst_off;
      dv->segM[q] = m;
      if (act) {
        const uint32_t it = I->iter;
        if (it < I->log_cap) I->log[it] = nn;
        I->n_new = nn;
        I->cand_total += I->n_cand;
        I->n_full = nf;
        I->f_off = dst_off;
        if (fin) {
          I->state = done ? INST_DONE : INST_ITERCAP;
          I->iters_done = it;
          I->res_pool = keep ? fph : (toR ? 2u : (fph ^ 1u));
          I->res_off = dst_off;
          I->n_delta = 0;
        } else {
          I->d_off = I->c_off;
          I->n_delta = nn;
          I->iter = it + 1;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_f += tf; s_r += tr; s_t += tt; s_act += ta; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Stage m{};
    m.in = dv->F[fph]; m.aux = dv->D[dph ^ 1]; m.out = dv->F[fph ^ 1]; m.out2 = dv->R;
    m.segs = dv->segM; m.inst = dv->inst; m.ctl = &dv->ctl; m.nseg = N; m.splits = dv->splits;
    m.ntiles = (uint32_t)s_t; m.ctr = 0;
    dv->st[S_MERGE] = m;
    dv->r_used = s_r;
    dv->fphase = fph ^ 1u;
    dv->dphase = dph ^ 1u;
    ctl.n_active = (uint32_t)s_act;
    ctl.launch_iters += 1;
    set_continue(dv, (s_act > 0 && ctl.launch_iters < ctl.iter_budget) ? 1u : 0u);
  }
}

// Side iteration (single-query engines, one instance), after the main run's
// pass: its output -- the candidates new with respect to the main run,
// deduplicated and sorted, in the spare candidate pool -- against the side
// run.  One more fused pass over (side run, that output) keeps what the side
// run lacks (the new delta) and writes the merged side run to the other side
// pool.  Every tile is classified (no mixed-tile list: the runs are small).
__global__ void k_plan_side(Dev* dv) {
  Ctl& ctl = dv->ctl;
  if (ctl.abort || threadIdx.x != 0) return;
  Inst* I = dv->inst;
  const bool act = I->state == INST_ACTIVE && I->side_iter;
  const unsigned long long n0 = act ? dv->segF[0].res : 0ull, ns = act ? I->n_side : 0ull;
  const unsigned long long tf = dv->fuse_tile;
  Seg f{};
  f.in_off = 0; f.n = ns; f.aux_off = I->c_off; f.aux_n = n0; f.out_off = I->c_off;
  f.out2_off = 0; f.res = 0; f.tile0 = 0; f.inst = 0; f.flags = 0;
  f.ntiles = act ? (uint32_t)((ns + n0 + tf - 1) / tf) : 0u;
  dv->segF2[0] = f;
  if (act) I->n_new0 = n0;
  Stage s{};
  s.segs = dv->segF2; s.inst = dv->inst; s.ctl = &dv->ctl; s.nseg = 1; s.ntiles = f.ntiles;
  s.ctr = 0; s.in = dv->G[I->gphase]; s.aux = dv->C[(dv->passes & 1) ^ 1];
  s.out = dv->D[dv->dphase ^ 1]; s.out2 = dv->G[I->gphase ^ 1];
  s.status = dv->status_scalar; s.epoch = ++ctl.epoch; s.splits = dv->splits;
  s.mixl = nullptr; s.mixc = nullptr;
  dv->st[S_FUSE2] = s;
}

// After the fused stage: commit the iteration (log, termination, new delta,
// Full' as the full relation) and schedule the copy of finished batch
// instances into the retire pool.  After a side iteration the main run stays
// where it is and the merged side run becomes the side run; when that
// iteration ends the fixpoint, the final relation is the merge of both runs
// (scheduled here as the S_MERGE stage) unless the side run is empty.
__global__ void __launch_bounds__(kPlanThreads) k_plan_post(Dev* dv) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long s_r, s_t, s_act;
  __shared__ uint32_t s_keep, s_fmerge;
  Ctl& ctl = dv->ctl;
  if (ctl.abort) {
    if (threadIdx.x == 0) set_continue(dv, 0);
    return;
  }
  const uint32_t N = dv->n_inst;
  const bool single = dv->single != 0;
  if (threadIdx.x == 0) s_r = 0;
  __syncthreads();
  for (uint32_t base = 0; base < N; base += kPlanThreads) {
    const uint32_t q = base + threadIdx.x;
    unsigned long long rsz = 0;
    if (q < N && !single) {
      const Inst* I = dv->inst + q;
      if (I->state == INST_ACTIVE) {
        const unsigned long long nn = dv->segF[q].res;
        const bool fin = (I->iter >= 1 && nn == 0) || I->iter >= I->max_iters;
        if (fin) rsz = I->n_full + nn;
      }
    }
    unsigned long long tr;
    scan1024(rsz, sh, &tr);
    if (threadIdx.x == 0) s_r += tr;
    __syncthreads();
  }
  if (dv->r_used + s_r > dv->capR && !single) {
    if (threadIdx.x == 0) {
      ctl.need_res = dv->r_used + s_r;
      ctl.abort = 1;
      set_continue(dv, 0);
    }
    return;
  }
  const uint32_t fph = dv->fphase, dph = dv->dphase;
  __syncthreads();
  if (threadIdx.x == 0) { s_r = dv->r_used; s_t = 0; s_act = 0; s_keep = 0; s_fmerge = 0; }
  __syncthreads();
  for (uint32_t base = 0; base < N; base += kPlanThreads) {
    const uint32_t q = base + threadIdx.x;
    const bool valid = q < N;
    Inst* I = valid ? dv->inst + q : nullptr;
    const bool act = valid && I->state == INST_ACTIVE;
    unsigned long long nn = 0, nf = 0, rsz = 0, mt = 0, ns1 = 0;
    bool fin = false, done = false, toR = false, side = false, fmerge = false;
    if (act) {
      side = I->side_iter != 0;
      nn = side ? dv->segF2[q].res : dv->segF[q].res;
      nf = I->n_full + nn;
      done = I->iter >= 1 && nn == 0;
      fin = done || I->iter >= I->max_iters;
      toR = fin && !single;
      if (toR || dv->copyback) { rsz = nf; mt = (nf + kTileM - 1) / kTileM; }
      if (side) {  // single-query engine: neither toR nor copyback
        ns1 = I->n_side + nn;
        fmerge = fin && ns1 > 0;
        if (fmerge) mt = (nf + kTileM - 1) / kTileM;
      }
    }
    unsigned long long tr, tt, ta;
    const unsigned long long exr = scan1024(rsz, sh, &tr);
    const unsigned long long ext = scan1024(mt, sh, &tt);
    scan1024((act && !fin) ? 1ull : 0ull, sh, &ta);
    if (valid) {
      const unsigned long long fo = side ? I->f_off : dv->segF[q].out2_off;
      Seg m{};
      if (fmerge) {  // the final relation: main run and side run, merged
        m.in_off = fo; m.n = nf - ns1; m.aux_off = 0; m.aux_n = ns1; m.out_off = fo;
        m.flags = 0;
      } else {
        // the retire copy (batch: to the result pool) or, copying back,
        // Full' onto the same offsets of the Full buffer
        m.in_off = fo; m.n = rsz; m.aux_off = 0; m.aux_n = 0;
        m.out_off = dv->copyback ? fo : s_r + exr;
        m.flags = 1u;
      }
      m.res = 0; m.out2_off = 0; m.tile0 = (uint32_t)(s_t + ext);
      m.ntiles = (uint32_t)mt; m.inst = q;
      dv->segM[q] = m;
      if (act) {
        const uint32_t it = I->iter;
        if (it < I->log_cap) I->log[it] = nn;
        I->n_new = nn;
        I->cand_total += I->n_cand;
        I->n_full = nf;
        I->f_off = fo;
        if (fin) {
          I->state = done ? INST_DONE : INST_ITERCAP;
          I->iters_done = it;
          if (side) {  // in place when nothing is in the side run
            I->res_pool = fmerge ? (fph ^ 1u) : fph;
            I->res_off = fo;
            I->n_side = 0;
          } else {
            I->res_pool = toR ? 2u : dv->copyback ? fph : (fph ^ 1u);
            I->res_off = toR ? s_r + exr : fo;
          }
          I->n_delta = 0;
        } else {
          if (side) {
            I->n_side = ns1;
            I->gphase ^= 1u;
          }
          I->d_off = I->c_off;
          I->n_delta = nn;
          I->iter = it + 1;
        }
      }
      if (side && !fmerge) s_keep = 1;  // the main run stays in pool fph
      if (fmerge) s_fmerge = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_r += tr; s_t += tt; s_act += ta; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Stage m{};
    m.in = dv->F[fph ^ 1]; m.aux = nullptr; m.out = dv->R;
    m.out2 = dv->copyback ? dv->F[fph] : dv->R;
    if (s_fmerge) {  // one instance: its side run is in G[gphase ^ 1] (not swapped when final)
      m.in = dv->F[fph]; m.aux = dv->G[dv->inst[0].gphase ^ 1u]; m.out = dv->F[fph ^ 1];
      m.out2 = nullptr; m.splits = dv->splits;  // k_partition finds the tile splits
    }
    m.segs = dv->segM; m.inst = dv->inst; m.ctl = &dv->ctl; m.nseg = N;
    m.ntiles = (uint32_t)s_t; m.ctr = 0;
    dv->st[S_MERGE] = m;
    dv->r_used = s_r;
    dv->fphase = (dv->copyback || s_keep) ? fph : fph ^ 1u;
    dv->dphase = dph ^ 1u;
    ctl.n_active = (uint32_t)s_act;
    ctl.launch_iters += 1;
    set_continue(dv, (s_act > 0 && ctl.launch_iters < ctl.iter_budget) ? 1u : 0u);
  }
}

// Delta^{-1} of a fresh instance: the diagonal {(v, v)}.  Joining it with E
// through the ordinary TC join yields E itself (the TC base rule); through the
// SG base-rule join it yields the sibling pairs.
// Only instances admitted since the last launch (fresh) are touched; the
// range [first, first + count) may also hold running or free slots.
template <typename K>
__global__ void k_init_diag(Inst* inst, uint32_t first, uint32_t count, K* dpool) {
  for (uint32_t q = first + blockIdx.x; q < first + count; q += gridDim.x) {
    const Inst I = inst[q];
    if (!I.fresh || I.state != INST_ACTIVE) continue;  // uniform across the block
    K* o = dpool + I.d_off;
    for (uint32_t v = threadIdx.x; v < I.nv; v += blockDim.x) o[v] = ((K)v << I.w) | (K)v;
    __syncthreads();
    if (threadIdx.x == 0) inst[q].fresh = 0;
  }
}

// ------------------------------------------------------------------ load / result
template <typename K>
__global__ void k_rank_edges(const uint32_t* src, const uint32_t* dst, unsigned long long n,
                             const uint32_t* V, uint32_t nv, uint32_t w, K* keys) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t rs = (uint32_t)lower_bound_k(V, nv, src[i]);
    const uint32_t rd = (uint32_t)lower_bound_k(V, nv, dst[i]);
    keys[i] = ((K)rs << w) | (K)rd;
  }
}

template <typename K>
__global__ void k_csr(const K* E, unsigned long long ne, uint32_t nv, uint32_t w, uint32_t* off,
                      uint32_t* adj) {
  const K mask = (K)(((K)1 << w) - 1);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long v = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; v <= nv;
       v += stride)
    off[v] = v == nv ? (uint32_t)ne : (uint32_t)lower_bound_k(E, ne, (K)((K)v << w));
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
       i += stride)
    adj[i] = (uint32_t)(E[i] & mask);
}

template <typename K>
__global__ void k_result_map(const K* F, unsigned long long n, uint32_t w, const uint32_t* V,
                             unsigned long long* out) {
  const K mask = (K)(((K)1 << w) - 1);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const K k = F[i];
    out[i] = ((unsigned long long)V[(uint32_t)(k >> w)] << 32) | V[(uint32_t)(k & mask)];
  }
}

// Digest of a result: sum over i of mix64(key_i + i * phi) mod 2^64, key_i =
// (id(x) << 32) | id(y) of the i-th sorted tuple, mix64 = the SplitMix64
// output function (Steele, Lea, Flood 2014).  `first` is the index of F[0] in
// the whole result (results are digested in chunks).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
template <typename K>
__global__ void __launch_bounds__(256) k_result_digest(const K* F, unsigned long long n,
                                                       unsigned long long first, uint32_t w,
                                                       const uint32_t* V, unsigned long long* out) {
  __shared__ unsigned long long sh[kWarps];
  const K mask = (K)(((K)1 << w) - 1);
  unsigned long long acc = 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const K k = F[i];
    const unsigned long long key = ((unsigned long long)V[(uint32_t)(k >> w)] << 32) | V[(uint32_t)(k & mask)];
    acc += mix64(key + (first + i) * 0x9E3779B97F4A7C15ull);
  }
  unsigned long long tot;
  block_excl_scan(acc, sh, &tot);
  if (threadIdx.x == 0 && tot) atomicAdd(out, tot);
}

// ------------------------------------------------------------------ launchers
// Self-test of the bounded device wait: one warp looks back, as every scan
// stage does, for a predecessor tile whose status word is never published
// (epoch 1 is never written).  The wait gives up after kSpinLimit polls,
// records DEV_TIMEOUT in the control block and the kernel returns.
__global__ void k_selftest_wait(const unsigned long long* status, Ctl* ctl, unsigned long long* out) {
  const unsigned long long e = lookback_scalar(status, 1u, 0u, 1u, ctl);
  if (threadIdx.x == 0) *out = e;
}
void launch_selftest_wait(const unsigned long long* status, Ctl* ctl, unsigned long long* out,
                          cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(status, ctl, out);
}

template <typename K>
void launch_join_count(Stage* st, int grid, cudaStream_t s, uint32_t tile) {
  if (tile == (uint32_t)kTileD / 2) k_join_count<K, kItemsD / 2><<<grid, kThreads, 0, s>>>(st);
  else k_join_count<K, kItemsD><<<grid, kThreads, 0, s>>>(st);
}
template <typename K>
void launch_join_emit(Stage* st, int grid, cudaStream_t s, uint32_t tile) {
  if (tile == kTileC / 2) k_join_emit<K, false, kTileC / 2><<<grid, kThreads, 0, s>>>(st);
  else k_join_emit<K, false><<<grid, kThreads, 0, s>>>(st);
}
template <typename K>
void launch_tri_probe(Stage* st, int grid, cudaStream_t s) { k_join_emit<K, true><<<grid, kThreads, 0, s>>>(st); }
template <typename K>
void launch_join_emit_hash(Stage* st, int grid, cudaStream_t s) { k_join_emit_hash<K><<<grid, kThreads, 0, s>>>(st); }
template <typename K>
void launch_hash_build(const K* E, unsigned long long ne, uint32_t w, unsigned long long* T,
                       unsigned long long mask, int grid, cudaStream_t s) {
  if (ne) k_hash_build<K><<<grid, 256, 0, s>>>(E, ne, w, T, mask);
}
template <typename K>
int occupancy_join(int which) {
  // largest shared-memory carveout first (see occupancy_of in wg_kern_sort.cu)
  auto one = [](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, 0);
    return b;
  };
  switch (which) {
    case 0: return one(k_join_count<K, kItemsD>);
    case 1: return one(k_join_emit<K, false>);
    case 2: return one(k_join_emit<K, true>);
    case 4: return one(k_join_emit<K, false, kTileC / 2>);
    default: return one(k_join_count<K, kItemsD / 2>);
  }
}
void launch_plan_delta(Dev* dv, cudaStream_t s) { k_plan_delta<<<1, kPlanThreads, 0, s>>>(dv); }
void launch_plan_cand(Dev* dv, cudaStream_t s) { k_plan_cand<<<1, kPlanThreads, 0, s>>>(dv); }
void launch_plan_merge(Dev* dv, cudaStream_t s) { k_plan_merge<<<1, kPlanThreads, 0, s>>>(dv); }
void launch_plan_post(Dev* dv, cudaStream_t s) { k_plan_post<<<1, kPlanThreads, 0, s>>>(dv); }
void launch_plan_side(Dev* dv, cudaStream_t s) { k_plan_side<<<1, 32, 0, s>>>(dv); }
void launch_xseg_build(Dev* dv, cudaStream_t s) {
  k_xseg_sum<<<kXChunks, kXChunk, 0, s>>>(dv);
  k_xseg_fill<<<kXChunks, kXChunk, 0, s>>>(dv);
}
template <typename K>
void launch_init_diag(Inst* inst, uint32_t first, uint32_t count, void* dpool, cudaStream_t s) {
  if (count) k_init_diag<K><<<count < 4096 ? count : 4096, 256, 0, s>>>(inst, first, count, (K*)dpool);
}
template <typename K>
void launch_rank_edges(const uint32_t* src, const uint32_t* dst, unsigned long long n,
                       const uint32_t* V, uint32_t nv, uint32_t w, K* keys, int grid,
                       cudaStream_t s) {
  k_rank_edges<K><<<grid, 256, 0, s>>>(src, dst, n, V, nv, w, keys);
}
template <typename K>
void launch_csr(const K* E, unsigned long long ne, uint32_t nv, uint32_t w, uint32_t* off,
                uint32_t* adj, int grid, cudaStream_t s) {
  k_csr<K><<<grid, 256, 0, s>>>(E, ne, nv, w, off, adj);
}
template <typename K>
void launch_result_map(const K* F, unsigned long long n, uint32_t w, const uint32_t* V,
                       unsigned long long* out, int grid, cudaStream_t s) {
  k_result_map<K><<<grid, 256, 0, s>>>(F, n, w, V, out);
}
template <typename K>
void launch_result_digest(const K* F, unsigned long long n, uint32_t w, const uint32_t* V,
                          unsigned long long* out, int grid, cudaStream_t s) {
  if (n) k_result_digest<K><<<grid, 256, 0, s>>>(F, n, 0ull, w, V, out);
}

#define WG_INST(K)                                                                          \
  template void launch_join_count<K>(Stage*, int, cudaStream_t, uint32_t);                  \
  template void launch_join_emit<K>(Stage*, int, cudaStream_t, uint32_t);                   \
  template void launch_tri_probe<K>(Stage*, int, cudaStream_t);                             \
  template void launch_join_emit_hash<K>(Stage*, int, cudaStream_t);                        \
  template void launch_hash_build<K>(const K*, unsigned long long, uint32_t,                 \
                                     unsigned long long*, unsigned long long, int, cudaStream_t); \
  template int occupancy_join<K>(int);                                                      \
  template void launch_init_diag<K>(Inst*, uint32_t, uint32_t, void*, cudaStream_t);        \
  template void launch_rank_edges<K>(const uint32_t*, const uint32_t*, unsigned long long,  \
                                     const uint32_t*, uint32_t, uint32_t, K*, int,          \
                                     cudaStream_t);                                         \
  template void launch_csr<K>(const K*, unsigned long long, uint32_t, uint32_t, uint32_t*,  \
                              uint32_t*, int, cudaStream_t);                                \
  template void launch_result_map<K>(const K*, unsigned long long, uint32_t, const uint32_t*, \
                                     unsigned long long*, int, cudaStream_t);                  \
  template void launch_result_digest<K>(const K*, unsigned long long, uint32_t, const uint32_t*, \
                                        unsigned long long*, int, cudaStream_t);
WG_INST(uint32_t)
WG_INST(unsigned long long)
#undef WG_INST

}  // namespace wg
