// wg_kern_sort.cu -- sorted-array stages of one semi-naive iteration (sm_103a):
//   * LSD radix sort of packed keys (Sec. Buffer Routing and Adaptive Radix Sort):
//     one upfront histogram of every digit, then one pass per digit that ranks a
//     tile in shared memory, finds its global offset by decoupled lookback (and
//     the digit's start in the segment by a block scan of the segment's
//     histogram row) and scatters through shared memory so that stores come
//     out in digit runs;
//   * fused deduplication + set difference against the full relation
//     (Sec. Fused Deduplication and Set Difference) that also writes the
//     merged relation (Sec. Disjoint Merge): one merge-path pass over
//     (Full, sorted candidates); the tiles holding candidates are classified
//     (block scan, decoupled lookback, ordered scatter), the Full-only tiles
//     are copied by a plain kernel;
//   * the paper's separate stages: dedup + diff against Full (k_unique_diff)
//     and the disjoint merge (k_merge: merge-path partitions, |out| = |Full| +
//     |Delta| exactly, no atomics).
// All kernels are segmented (one segment per fixpoint instance) and indirect:
// their work comes from a device-resident Stage record.
#include "wg_device.cuh"
#include "wg_launch.h"

namespace wg {

template <typename K>
__device__ __forceinline__ uint32_t digit(K k, uint32_t shift, uint32_t mask) {
  return (uint32_t)(k >> shift) & mask;
}

// Digit extraction of one pass.  Whole-byte digits (8-bit digits at a shift
// that is a multiple of 8: every pass of a 16- or 32-bit sort) take one byte
// permute of the 32-bit word that holds them.
struct Digit {
  uint32_t shift, mask, sel, hi;  // sel: byte selector of a whole-byte digit; hi: word
  __device__ __forceinline__ Digit(uint32_t sh, uint32_t bits)
      : shift(sh), mask((1u << bits) - 1u), sel(0x4440u | ((sh & 31u) >> 3)), hi(sh >= 32) {}
  template <bool kByte, typename K>
  __device__ __forceinline__ uint32_t operator()(K k) const {
    if constexpr (kByte) {
      const uint32_t w = sizeof(K) == 4 ? (uint32_t)k : (uint32_t)(hi ? (k >> 32) : k);
      return __byte_perm(w, 0u, sel);
    } else {
      return (uint32_t)(k >> shift) & mask;
    }
  }
};

// ------------------------------------------------------------------ histogram
// Digit counts per segment from one read of the keys.  For the lookback
// passes it counts the FIRST pass's digit only: each pass counts the next
// pass's digits while it ranks its tile.  For the per-source segments (the
// stage has `maxt`, so k_sort_seg may sort the launch) it counts the digits of
// every pass, and no pass counts any.
// NP > 0: that many digits per key (unrolled); NP == 0: np digits.
template <typename K, bool kByte, int NP>
__device__ __forceinline__ void hist_tile(const K* p, uint32_t n, uint32_t dbits, uint32_t np,
                                          uint32_t* sh) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wbase = warp * 32 * kItemsC + lane;
  K key[kItemsC];
#pragma unroll
  for (int i = 0; i < kItemsC; ++i) {
    const uint32_t idx = wbase + i * 32;
    key[i] = idx < n ? p[idx] : (K)0;
  }
  const uint32_t npass = NP ? (uint32_t)NP : np;
#pragma unroll
  for (uint32_t ps = 0; ps < (NP ? (uint32_t)NP : (uint32_t)kMaxPasses); ++ps) {
    if (ps >= npass) break;
    const Digit dg(ps * dbits, dbits);
    uint32_t* h = sh + ps * kRadix;
#pragma unroll
    for (int i = 0; i < kItemsC; ++i)
      if (wbase + i * 32 < n) atomicAdd(&h[dg.operator()<kByte>(key[i])], 1u);
  }
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 6) k_sort_hist(Stage* stp) {
  __shared__ uint32_t sh[kMaxPasses * kRadix];
  __shared__ const K* s_p;
  __shared__ unsigned long long* s_row;
  __shared__ uint32_t s_t, s_n;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  // the per-segment sort counts its segments' digits itself
  if (stp->maxt && *stp->maxt <= kSegSortMaxTiles) return;
  const K* in = (const K*)stp->in;
  const uint32_t passes = stp->passes, nseg = stp->nseg, ntiles = stp->ntiles;
  const uint32_t np = stp->maxt ? passes : 1u;  // digits counted per key
  const bool byte = stp->dbits == 8;
  for (;;) {
    __syncthreads();  // the previous tile's counts are flushed
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(&stp->ctr, 1u);
      s_t = t;
      if (t < ntiles) {
        const uint32_t k = find_seg(stp->segs, nseg, t, stp->tile_seg);
        const Seg& sg = stp->segs[k];
        const unsigned long long start = (unsigned long long)(t - sg.tile0) * kTileC;
        s_p = in + sg.in_off + start;
        s_n = (uint32_t)min((unsigned long long)kTileC, sg.n - start);
        s_row = stp->hist + (unsigned long long)k * passes * kRadix;
      }
    }
    for (uint32_t i = threadIdx.x; i < np * kRadix; i += kThreads) sh[i] = 0;
    __syncthreads();
    if (s_t >= ntiles) return;
    if (byte && np == 1) hist_tile<K, true, 1>(s_p, s_n, 8, 1, sh);
    else if (byte && np == 2) hist_tile<K, true, 2>(s_p, s_n, 8, 2, sh);
    else if (byte) hist_tile<K, true, 0>(s_p, s_n, 8, np, sh);
    else hist_tile<K, false, 0>(s_p, s_n, stp->dbits, np, sh);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < np * kRadix; i += kThreads) {
      const uint32_t c = sh[i];
      if (c) atomicAdd(&s_row[i], (unsigned long long)c);
    }
  }
}

// ------------------------------------------------------------------ one radix pass
constexpr int kLookW = 8;  // lookback words a digit thread loads at once

// Tile metadata, written by thread 0 when the tile is claimed.
struct PassMeta {
  unsigned long long in;    // the tile's first key in the input pool
  unsigned long long out;   // the segment's first key in the output pool
  unsigned long long* nrow; // the segment's histogram row of the next pass (or NULL)
  uint32_t t, k, n, tile0;  // tile, segment, keys in the tile, first tile of the segment
  uint32_t first, rel32;    // first tile of its segment; segment of < 2^32 keys
};

template <typename K>
struct PassSmem {
  static constexpr int kSlots = sizeof(K) == 4 ? 2 : 1;  // two tiles in flight fit for 32-bit keys
  K sk[kSlots][kTileC];                 // a ranked tile in digit order
  // rank phase: per-warp digit counters, then the tile-local start of
  // (warp, digit): the digit's start in the tile plus the earlier warps' keys
  uint32_t wbase[kWarps][kRadix];
  // write phase: global base of each digit minus its start in the tile:
  // absolute, or from the segment's start (segments < 2^32 keys).  Not shared
  // with wbase: the next tile's ranking starts right after the stores of the
  // tile written, with no barrier in between.
  union {
    unsigned long long gdst[kRadix];
    uint32_t gdst32[kRadix];
  };
  uint32_t nxt[kRadix];                    // next pass's digit counts of the tile being ranked
  uint32_t tstart[kSlots][kRadix + 1];     // digit starts inside the tile; [kRadix] = tile size
  unsigned long long hstart[kSlots][kRadix];  // digit starts inside the segment
  unsigned long long s_scan[kWarps];
  PassMeta meta[kSlots + 1];  // tiles in flight: written next, ranked, being loaded
  uint32_t s_t, s_bad;
};

// Claim the next tile and (thread 0) describe it in meta[mi].
template <typename K>
__device__ __forceinline__ uint32_t pass_claim(Stage* stp, PassSmem<K>& S, int mi) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&stp->ctr, 1u);
    S.s_t = t;
    if (t < stp->ntiles) {
      const uint32_t k = find_seg(stp->segs, stp->nseg, t, stp->tile_seg);
      const Seg& sg = stp->segs[k];
      const unsigned long long start = (unsigned long long)(t - sg.tile0) * kTileC;
      PassMeta m;
      m.in = sg.in_off + start;
      m.out = sg.out_off;
      // the next pass's digits are counted here unless the histogram
      // kernel counted every pass's (stages with maxt)
      m.nrow = stp->pass + 1 < stp->passes && !stp->maxt
                   ? stp->hist + ((unsigned long long)k * stp->passes + stp->pass + 1) * kRadix
                   : nullptr;
      m.t = t; m.k = k; m.tile0 = sg.tile0;
      m.n = (uint32_t)min((unsigned long long)kTileC, sg.n - start);
      m.first = t == sg.tile0;
      m.rel32 = sg.n <= 0xFFFFFFFFull;
      S.meta[mi] = m;
    }
  }
  __syncthreads();
  return S.s_t;
}

// Issue the loads of tile meta[mi] into registers (warp-striped: warp w owns
// keys [w*32*kItemsC, (w+1)*32*kItemsC)).  Nothing waits for them here: the
// caller writes out the previous tile while they are in flight.
template <typename K>
__device__ __forceinline__ void pass_load(const Stage* stp, const PassMeta& m, K (&key)[kItemsC]) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wb = warp * 32 * kItemsC + lane;
  const K* p = (const K*)stp->in + m.in;
  if (m.n == (uint32_t)kTileC) {
#pragma unroll
    for (int i = 0; i < kItemsC; ++i) key[i] = p[wb + i * 32];
  } else {
#pragma unroll
    for (int i = 0; i < kItemsC; ++i) {
      const uint32_t idx = wb + i * 32;
      key[i] = idx < m.n ? p[idx] : (K)0;
    }
  }
}

// Rank tile meta[mi] (its keys in registers) into slot sl: rank every key
// within its digit (per warp), publish the tile's digit counts, find the
// digit starts in the tile and in the segment (one scan), and place the keys
// in digit order in sk[sl].  Nothing here waits for another tile.  kFull: the
// tile holds kTileC keys (every bounds test folds away); kByte: whole-byte
// digits.
template <typename K, bool kFull, bool kByte>
__device__ __forceinline__ void pass_rank_tile(Stage* stp, PassSmem<K>& S, int sl, int mi,
                                               const K (&key)[kItemsC]) {
  const PassMeta& m = S.meta[mi];
  const uint32_t pass = stp->pass;
  const Digit dg(stp->shift, stp->dbits), dn(stp->shift + stp->dbits, stp->dbits);
  const bool ahead = m.nrow != nullptr;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t n = kFull ? (uint32_t)kTileC : m.n;
  const uint32_t wb = warp * 32 * kItemsC + lane;
  // this warp's counters and the block's next-digit counters start at zero
  uint32_t* wc = S.wbase[warp];
#pragma unroll
  for (int j = 0; j < kRadix / 32; ++j) wc[lane + 32 * j] = 0;
  S.nxt[threadIdx.x] = 0;
  __syncthreads();

  uint32_t rk[kItemsC / 2];  // ranks (< kTileC) packed two per word
#pragma unroll
  for (int i = 0; i < kItemsC / 2; ++i) rk[i] = 0;
  if (pass == 0) {
    // first pass: the input order carries nothing, so any order of equal
    // digits is correct -- one shared atomic per key gives its rank.  Keys
    // that tie on every sorted bit are identical (the bits above are zero),
    // so the sorted output equals that of a stable sort.
#pragma unroll
    for (int i = 0; i < kItemsC; ++i) {
      if (kFull || wb + i * 32 < n)
        rk[i >> 1] |= atomicAdd(&wc[dg.operator()<kByte>(key[i])], 1u) << (16 * (i & 1));
    }
  } else {
    // later passes: stable rank within the warp -- peers with the same
    // digit, in (i, lane) order
#pragma unroll
    for (int i = 0; i < kItemsC; ++i) {
      const bool ok = kFull || wb + i * 32 < n;
      const uint32_t d = ok ? dg.operator()<kByte>(key[i]) : 0xFFFFFFFFu;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = 0;
      if (ok) before = wc[d];
      rk[i >> 1] |= (before + __popc(peers & lt_mask)) << (16 * (i & 1));
      __syncwarp();
      if (ok && lane == (uint32_t)(__ffs(peers) - 1)) wc[d] = before + __popc(peers);
      __syncwarp();
    }
  }
  if (ahead) {  // the next pass's digits of the same keys
#pragma unroll
    for (int i = 0; i < kItemsC; ++i)
      if (kFull || wb + i * 32 < n) atomicAdd(&S.nxt[dn.operator()<kByte>(key[i])], 1u);
  }
  __syncthreads();

  // thread d owns digit d: per-warp counts, tile count, publish it; the
  // segment's count of the digit (loaded first, its latency overlaps)
  const uint32_t d = threadIdx.x;
  const unsigned long long hcount =
      stp->hist[((unsigned long long)m.k * stp->passes + pass) * kRadix + d];
  uint32_t cnt = 0;  // the warps' counts become exclusive prefixes over warps
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = S.wbase[w][d];
    S.wbase[w][d] = cnt;
    cnt += c;
  }
  st_put(stp->status + (unsigned long long)m.t * kRadix + d,
         st_pack(stp->epoch, m.first ? FLAG_INC : FLAG_AGG, cnt));
  if (ahead) {
    const uint32_t nx = S.nxt[d];
    if (nx) atomicAdd(m.nrow + d, (unsigned long long)nx);
  }
  // one scan gives both starts: the tile count (<= kTileC < 2^13) in the low
  // 13 bits, the segment count above them
  unsigned long long tot;
  const unsigned long long ex = block_excl_scan((hcount << 13) | cnt, S.s_scan, &tot);
  const uint32_t ts = (uint32_t)(ex & 0x1FFFu);
  S.tstart[sl][d] = ts;
  if (d == kRadix - 1) S.tstart[sl][kRadix] = ts + cnt;
  S.hstart[sl][d] = ex >> 13;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) S.wbase[w][d] += ts;
  __syncthreads();
  // the tile in digit order: a key's place inside the tile needs no global offset
#pragma unroll
  for (int i = 0; i < kItemsC; ++i)
    if (kFull || wb + i * 32 < n)
      S.sk[sl][wc[dg.operator()<kByte>(key[i])] + ((rk[i >> 1] >> (16 * (i & 1))) & 0xFFFFu)] = key[i];
}

template <typename K, bool kByte>
__device__ __forceinline__ void pass_rank(Stage* stp, PassSmem<K>& S, int sl, int mi,
                                          const K (&key)[kItemsC]) {
  if constexpr (sizeof(K) == 4) {
    if (S.meta[mi].n == (uint32_t)kTileC) {
      pass_rank_tile<K, true, kByte>(stp, S, sl, mi, key);
      return;
    }
  }
  pass_rank_tile<K, false, kByte>(stp, S, sl, mi, key);
}

// Global offsets of the tile in slot `sl` by per-digit lookback, then stream
// its digit runs out.  False when a lookback gave up (the run is void).
template <typename K, bool kByte>
__device__ __forceinline__ bool pass_write(Stage* stp, PassSmem<K>& S, int sl, int mi) {
  __syncthreads();  // the slot's keys, starts and meta are visible
  const PassMeta& m = S.meta[mi];
  const Digit dg(stp->shift, stp->dbits);
  const uint32_t epoch = stp->epoch;
  Ctl* ctl = stp->ctl;
  unsigned long long* status = stp->status;
  const uint32_t d = threadIdx.x;
  const uint32_t ts = S.tstart[sl][d], cnt = S.tstart[sl][d + 1] - ts;
  unsigned long long excl = 0;
  if (!m.first) {
    // per-digit lookback over earlier tiles of this segment: the words of a
    // window of kLookW predecessors are loaded at once, then consumed nearest
    // first until an inclusive one (a walk of dependent loads would cost one
    // L2 round trip per tile, and tiles behind this one wait for it)
    const long long tile0 = m.tile0;
    long long j = (long long)m.t - 1;
    bool done = false;
    while (!done) {
      const long long w = min((long long)kLookW, j - tile0 + 1);
      unsigned long long sw[kLookW];
#pragma unroll
      for (int q = 0; q < kLookW; ++q)
        sw[q] = q < w ? st_get(status + (unsigned long long)(j - q) * kRadix + d) : 0ull;
#pragma unroll
      for (int q = 0; q < kLookW; ++q) {
        if (done || q >= w) break;
        unsigned long long s = sw[q];
        uint32_t spins = 0;
        while (!st_ready(s, epoch)) {
          if (++spins > kSpinLimit || *(volatile uint32_t*)&ctl->abort) break;
          __nanosleep(64);
          s = st_get(status + (unsigned long long)(j - q) * kRadix + d);
        }
        if (!st_ready(s, epoch)) {
          if (!*(volatile uint32_t*)&ctl->abort) fail_timeout(ctl);
          S.s_bad = 1;
          done = true;
          break;
        }
        excl += s & kValMask;
        if (((s >> 38) & 3u) == FLAG_INC || j - q == tile0) done = true;
      }
      j -= w;
    }
    st_put(status + (unsigned long long)m.t * kRadix + d, st_pack(epoch, FLAG_INC, excl + cnt));
  }
  const unsigned long long g = S.hstart[sl][d] + excl;
  if (m.rel32) S.gdst32[d] = (uint32_t)g - ts;
  else S.gdst[d] = m.out + g - ts;
  __syncthreads();
  if (S.s_bad) return false;
  K* out = (K*)stp->out;
  if (m.rel32) {
    K* outs = out + m.out;
    if (m.n == (uint32_t)kTileC) {
#pragma unroll
      for (int e = 0; e < kItemsC; ++e) {
        const uint32_t i = threadIdx.x + e * kThreads;
        const K v = S.sk[sl][i];
        outs[S.gdst32[dg.operator()<kByte>(v)] + i] = v;
      }
    } else {
      for (uint32_t i = threadIdx.x; i < m.n; i += kThreads) {
        const K v = S.sk[sl][i];
        outs[S.gdst32[dg.operator()<kByte>(v)] + i] = v;
      }
    }
  } else {
    for (uint32_t i = threadIdx.x; i < m.n; i += kThreads) {
      const K v = S.sk[sl][i];
      out[S.gdst[dg.operator()<kByte>(v)] + i] = v;
    }
  }
  return true;
}

// One LSD pass (onesweep-style), software-pipelined over the tiles a CTA
// claims.  Each step ranks tile A (its keys already in registers) and
// publishes its counts, claims tile B and issues B's loads, and only then
// writes out a ranked tile -- so B's loads are in flight during that tile's
// lookback and stores.  With two slots (32-bit keys) the tile written is the
// one ranked a step earlier (its predecessors have had one step to publish);
// with one slot it is A.  Deadlock-free: ranking, publishing and loading
// never wait, and a tile that is claimed but not yet ranked sits in a CTA
// writing an older tile, so the oldest tile being written can always finish
// its lookback.
template <typename K, bool kByte>
__device__ __forceinline__ void pass_loop(Stage* stp, PassSmem<K>& S) {
  const uint32_t ntiles = stp->ntiles;
  if (threadIdx.x == 0) S.s_bad = 0;
  K key[kItemsC];
  int ma = 0, sa = 0;  // tile A: meta entry, slot
  if (pass_claim<K>(stp, S, ma) >= ntiles) return;
  pass_load<K>(stp, S.meta[ma], key);
  if constexpr (PassSmem<K>::kSlots == 2) {
    bool hasP = false;
    int mp = 0, sp = 0;  // tile P (ranked, not yet written)
    for (;;) {
      pass_rank<K, kByte>(stp, S, sa, ma, key);
      int mb = ma == 2 ? 0 : ma + 1;
      if (hasP && mb == mp) mb = mb == 2 ? 0 : mb + 1;
      const bool more = pass_claim<K>(stp, S, mb) < ntiles;
      if (more) pass_load<K>(stp, S.meta[mb], key);
      if (hasP && !pass_write<K, kByte>(stp, S, sp, mp)) return;
      if (!more) {
        pass_write<K, kByte>(stp, S, sa, ma);
        return;
      }
      hasP = true;
      mp = ma; sp = sa;
      ma = mb; sa = sp ^ 1;
    }
  } else {
    for (;;) {
      pass_rank<K, kByte>(stp, S, 0, ma, key);
      const int mb = ma ^ 1;
      const bool more = pass_claim<K>(stp, S, mb) < ntiles;
      if (more) pass_load<K>(stp, S.meta[mb], key);
      if (!pass_write<K, kByte>(stp, S, 0, ma) || !more) return;
      ma = mb;
    }
  }
}

// kByte: whole-byte digits (dbits == 8; the host knows the pass plan and
// picks the instantiation).
template <typename K, bool kByte>
__global__ void __launch_bounds__(kThreads, 4) k_sort_pass(Stage* stp) {
  __shared__ PassSmem<K> S;
  if (*(volatile uint32_t*)&stp->ctl->abort) return;
  if (stp->maxt && *stp->maxt <= kSegSortMaxTiles) return;  // k_sort_seg sorts this launch
  pass_loop<K, kByte>(stp, S);
}

// ------------------------------------------------------------------ per-segment sort
// Many segments of at most kSegSortMaxTiles tiles (the per-source segments of
// the x-grouped sort): one CTA takes a whole segment through every pass, its
// tiles in order, so each digit's next output offset in the segment is a
// running count in shared memory -- no lookback and no status words.  The CTA
// first counts every pass's digits of its segment in one read (which also
// brings the segment into L2 for the first pass); the histogram kernel then
// has nothing to do.  Every pass after the first ranks stably within a tile
// and takes the tiles in order, so it is stable.  A CTA claims the segments of
// at least kSegBig tiles first, then the others, so the longest ones do not
// start last.  NT threads of IT keys each make a tile.
// the per-source segments sort fields of at most 18 bits (kXSegMaxVertices):
// at most three passes
constexpr uint32_t kSegMaxPasses = 3;
// three compiled shapes (engine setting, wg_set_sort): 256 threads of 16 keys
// at 4 CTAs per SM (64 registers) or of 8 keys at 6 CTAs per SM (40), with
// digits of up to 8 bits (RB = 256 buckets); and 8 keys with digits of up to
// 9 bits (RB = 512), so that the 17- and 18-bit fields of relations of up to
// 2^18 vertices take two passes instead of three.
constexpr int kSegNT = 256;
constexpr int kWideRadix = 512;
template <int IT> struct SegShape { static constexpr int minb = IT == 16 ? 4 : 6; };

template <typename K, int NT, int IT, int RB>
struct SegSmem {
  static constexpr int NW = NT / 32, TILE = NT * IT;
  K sk[TILE];                     // a ranked tile in digit order
  uint32_t wbase[NW][RB];         // per-warp counters -> tile-local start of (warp, digit)
  uint32_t gdst[RB];              // output offset in the segment minus the digit's tile start
  uint32_t run[RB];               // next output offset of each digit in the segment
  uint32_t hc[kSegMaxPasses][RB]; // the segment's count of each digit, per pass
  uint32_t s_scan[NW];
  uint32_t s_k;
};

// Exclusive scan of one 32-bit value per thread over a CTA of NT threads.
template <int NT>
__device__ __forceinline__ uint32_t cta_excl_scan32(uint32_t v, uint32_t* sh) {
  constexpr int NW = NT / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (NW == 1) return x - v;
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (uint32_t)NW ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    if (lane < (uint32_t)NW) sh[lane] = w;
  }
  __syncthreads();
  const uint32_t r = (warp ? sh[warp - 1] : 0u) + x - v;
  __syncthreads();
  return r;
}

// Digits owned by a thread in the per-digit steps: DPT consecutive digits
// (CTAs of fewer than RB threads), else digit threadIdx.x (if < RB).
template <int NT, int RB> struct SegDig {
  static constexpr int DPT = NT >= RB ? 1 : RB / NT;
  __device__ static bool owns() { return NT <= RB || threadIdx.x < (uint32_t)RB; }
  __device__ static uint32_t first() { return threadIdx.x * DPT; }
};

// The next segment for a CTA (thread 0): from the claim order list when the
// stage has one (one atomic ticket, one load), else by scanning the segments
// (the big ones on a first sweep of the tickets, the others on a second).
// 0xFFFFFFFF when none is left.
__device__ __forceinline__ uint32_t seg_claim(Stage* st0) {
  const uint32_t nseg = st0->nseg;
  if (st0->order) {
    const uint32_t v = atomicAdd(&st0->ctr, 1u);
    const uint32_t nb = st0->order_n[0], ns = st0->order_n[1];
    if (v < nb) return st0->order[v];
    if (v < nb + ns) return st0->order[nseg - 1 - (v - nb)];
    return 0xFFFFFFFFu;
  }
  for (;;) {
    const uint32_t v = atomicAdd(&st0->ctr, 1u);
    if (v >= 2 * nseg) return 0xFFFFFFFFu;
    const uint32_t kk = v < nseg ? v : v - nseg;
    const uint32_t nt = st0->segs[kk].ntiles;
    if (nt != 0 && (v < nseg) == (nt >= kSegBig)) return kk;
  }
}

// Load n <= NT*IT keys from p into registers, warp-striped.
template <typename K, int NT, int IT>
__device__ __forceinline__ void seg_load(const K* p, uint32_t n, K (&key)[IT]) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wb = warp * 32 * IT + lane;
  if (n == (uint32_t)(NT * IT)) {
#pragma unroll
    for (int i = 0; i < IT; ++i) key[i] = p[wb + i * 32];
  } else {
#pragma unroll
    for (int i = 0; i < IT; ++i) key[i] = wb + i * 32 < n ? p[wb + i * 32] : (K)0;
  }
}

// One tile of one pass: rank (unstable for the first pass, stable after),
// count the next pass's digits, place the keys in digit order, compute their
// output offsets from the running counts.  The caller writes the tile out.
template <typename K, bool kByte, bool kFull, int NT, int IT, int RB>
__device__ __forceinline__ void seg_rank_tile(SegSmem<K, NT, IT, RB>& S, const K (&key)[IT],
                                              uint32_t n, const Digit& dg, bool first_pass) {
  using D = SegDig<NT, RB>;
  constexpr int NW = NT / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t wb = warp * 32 * IT + lane;
  uint32_t* wc = S.wbase[warp];
  // this warp's counters: the previous tile's per-digit step and scatter
  // are behind a barrier already, and only this warp touches its row until
  // the next barrier
#pragma unroll
  for (int j = 0; j < RB / 32; ++j) wc[lane + 32 * j] = 0;
  __syncwarp();
  uint32_t rk[(IT + 1) / 2];
#pragma unroll
  for (int i = 0; i < (IT + 1) / 2; ++i) rk[i] = 0;
  if (first_pass) {
#pragma unroll
    for (int i = 0; i < IT; ++i)
      if (kFull || wb + i * 32 < n)
        rk[i >> 1] |= atomicAdd(&wc[dg.operator()<kByte>(key[i])], 1u) << (16 * (i & 1));
  } else {
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const bool ok = kFull || wb + i * 32 < n;
      const uint32_t d = ok ? dg.operator()<kByte>(key[i]) : 0xFFFFFFFFu;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = 0;
      if (ok) before = wc[d];
      rk[i >> 1] |= (before + __popc(peers & lt_mask)) << (16 * (i & 1));
      __syncwarp();
      if (ok && lane == (uint32_t)(__ffs(peers) - 1)) wc[d] = before + __popc(peers);
      __syncwarp();
    }
  }
  __syncthreads();
  // per digit: per-warp prefixes and the tile's count; the digit's start in
  // the tile (a scan over the digits) and its output offset; the running
  // count moves on
  uint32_t cnt[D::DPT];
  uint32_t tsum = 0;
  if (D::owns()) {
#pragma unroll
    for (int j = 0; j < D::DPT; ++j) {
      const uint32_t d = D::first() + j;
      uint32_t c = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t x = S.wbase[w][d];
        S.wbase[w][d] = c;
        c += x;
      }
      cnt[j] = c;
      tsum += c;
    }
  }
  uint32_t ts = cta_excl_scan32<NT>(tsum, S.s_scan);
  if (D::owns()) {
#pragma unroll
    for (int j = 0; j < D::DPT; ++j) {
      const uint32_t d = D::first() + j;
#pragma unroll
      for (int w = 0; w < NW; ++w) S.wbase[w][d] += ts;
      const uint32_t r = S.run[d];
      S.gdst[d] = r - ts;
      S.run[d] = r + cnt[j];
      ts += cnt[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < IT; ++i)
    if (kFull || wb + i * 32 < n)
      S.sk[wc[dg.operator()<kByte>(key[i])] + ((rk[i >> 1] >> (16 * (i & 1))) & 0xFFFFu)] = key[i];
  __syncthreads();
}

// Every pass's digit counts of a segment of n keys at p, into S.hc (one read).
template <typename K, bool kByte, int NT, int IT, int RB>
__device__ __forceinline__ void seg_count(SegSmem<K, NT, IT, RB>& S, const K* p, uint32_t n,
                                          uint32_t passes, uint32_t dbits) {
  constexpr uint32_t TILE = NT * IT;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wb = warp * 32 * IT + lane;
  for (uint32_t i = threadIdx.x; i < kSegMaxPasses * RB; i += NT) (&S.hc[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
    const uint32_t tn = min(n - t0, TILE);
    K key[IT];
    seg_load<K, NT, IT>(p + t0, tn, key);
#pragma unroll
    for (uint32_t ps = 0; ps < kSegMaxPasses; ++ps) {
      if (ps >= passes) break;
      const Digit dg(ps * dbits, dbits);
      if (tn == TILE) {
#pragma unroll
        for (int i = 0; i < IT; ++i) atomicAdd(&S.hc[ps][dg.operator()<kByte>(key[i])], 1u);
      } else {
#pragma unroll
        for (int i = 0; i < IT; ++i)
          if (wb + i * 32 < tn) atomicAdd(&S.hc[ps][dg.operator()<kByte>(key[i])], 1u);
      }
    }
  }
  __syncthreads();
}

template <typename K, bool kByte, int NT, int IT, int RB>
__device__ __forceinline__ void seg_sort(Stage* st0, SegSmem<K, NT, IT, RB>& S, uint32_t k) {
  using D = SegDig<NT, RB>;
  constexpr uint32_t TILE = NT * IT;
  const Seg& sg = st0->segs[k];
  const unsigned long long in_off = sg.in_off, out_off = sg.out_off;
  const uint32_t n = (uint32_t)sg.n, passes = st0->passes, dbits = st0->dbits;
  const uint32_t nt = (n + TILE - 1) / TILE;
  seg_count<K, kByte, NT, IT, RB>(S, (const K*)st0->in + in_off, n, passes, dbits);
  for (uint32_t p = 0; p < passes; ++p) {
    const Stage* sp = st0 + p;
    const K* in = (const K*)sp->in + in_off;
    K* out = (K*)sp->out + out_off;
    const Digit dg(sp->shift, dbits);
    K key[IT];
    seg_load<K, NT, IT>(in, min(n, TILE), key);
    // the segment's count of each digit in this pass; their scan starts
    // the running counts
    uint32_t c[D::DPT], csum = 0;
    if (D::owns()) {
#pragma unroll
      for (int j = 0; j < D::DPT; ++j) {
        c[j] = S.hc[p][D::first() + j];
        csum += c[j];
      }
    }
    uint32_t hs = cta_excl_scan32<NT>(csum, S.s_scan);
    if (D::owns()) {
#pragma unroll
      for (int j = 0; j < D::DPT; ++j) {
        S.run[D::first() + j] = hs;
        hs += c[j];
      }
    }
    __syncthreads();
    for (uint32_t j = 0; j < nt; ++j) {
      const uint32_t tn = min(n - j * TILE, TILE);
      if (tn == TILE) seg_rank_tile<K, kByte, true, NT, IT, RB>(S, key, tn, dg, p == 0);
      else seg_rank_tile<K, kByte, false, NT, IT, RB>(S, key, tn, dg, p == 0);
      if (j + 1 < nt)  // the next tile's loads fly during this tile's stores
        seg_load<K, NT, IT>(in + (unsigned long long)(j + 1) * TILE, min(n - (j + 1) * TILE, TILE), key);
      if (tn == TILE) {
#pragma unroll
        for (int e = 0; e < IT; ++e) {
          const uint32_t i = threadIdx.x + e * NT;
          const K v = S.sk[i];
          out[S.gdst[dg.operator()<kByte>(v)] + i] = v;  // offsets are from the segment's start
        }
      } else {
        for (uint32_t i = threadIdx.x; i < tn; i += NT) {
          const K v = S.sk[i];
          out[S.gdst[dg.operator()<kByte>(v)] + i] = v;
        }
      }
    }
    __syncthreads();  // this pass's output (global) is complete before the next pass reads it
  }
}

template <typename K, bool kByte, int IT, int RB = kRadix>
__global__ void __launch_bounds__(kSegNT, SegShape<IT>::minb) k_sort_seg(Stage* st0) {
  __shared__ SegSmem<K, kSegNT, IT, RB> S;
  if (*(volatile uint32_t*)&st0->ctl->abort) return;
  // the lookback passes sort it (never for wide digits: their stages point
  // maxt at a zero word)
  if (!st0->maxt || *st0->maxt > kSegSortMaxTiles) return;
  // thread 0 claims the CTA's next segment while the CTA sorts the current one
  if (threadIdx.x == 0) S.s_k = seg_claim(st0);
  __syncthreads();
  for (;;) {
    const uint32_t k = S.s_k;
    if (k == 0xFFFFFFFFu) return;
    __syncthreads();  // every thread has k
    if (threadIdx.x == 0) S.s_k = seg_claim(st0);
    seg_sort<K, kByte, kSegNT, IT, RB>(st0, S, k);  // ends with a barrier
  }
}

// ------------------------------------------------------------------ dedup + diff
template <typename K>
__global__ void __launch_bounds__(kThreads, 4) k_unique_diff(Stage* stp) {
  __shared__ K sk[Padded<kTileC>::n];
  __shared__ K sf[FWin<K>::n];
  __shared__ unsigned long long s_scan[kWarps];
  __shared__ unsigned long long s_lo, s_hi, s_excl;
  __shared__ K s_prev;
  __shared__ uint32_t s_t, s_bad;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  const K* in = (const K*)stp->in;
  const K* full = (const K*)stp->aux;
  K* out = (K*)stp->out;
  const uint32_t nseg = stp->nseg, ntiles = stp->ntiles, epoch = stp->epoch;
  unsigned long long* status = stp->status;

  for (;;) {
    const uint32_t t = claim_tile(stp, &s_t);
    if (t >= ntiles) return;
    const uint32_t k = find_seg(stp->segs, nseg, t, stp->tile_seg);
    const Seg sg = stp->segs[k];
    const unsigned long long start = (unsigned long long)(t - sg.tile0) * kTileC;
    const uint32_t n = (uint32_t)min((unsigned long long)kTileC, sg.n - start);
    const K* p = in + sg.in_off + start;
    tile_to_smem<kItemsC>(sk, p, n, Pad32());
    if (threadIdx.x == 0 && start > 0) s_prev = p[-1];
    __syncthreads();
    const K* F = full + sg.aux_off;
    const unsigned long long nf = sg.aux_n;
    if (threadIdx.x == 0) s_lo = lower_bound_k(F, nf, sk[0]);
    if (threadIdx.x == 32) s_hi = upper_bound_k(F, nf, sk[pad32(n - 1)]);
    __syncthreads();
    const unsigned long long lo = s_lo, hi = s_hi;
    const bool staged = hi - lo <= (unsigned long long)FWin<K>::n;
    if (staged) tile_to_smem<FWin<K>::n / kThreads>(sf, F + lo, (uint32_t)(hi - lo), Ident());
    __syncthreads();

    // classify a blocked run of keys: first copy and not in Full
    const uint32_t b = threadIdx.x * kItemsC;
    K key[kItemsC];
    uint32_t keep = 0;
    unsigned long long cur = staged ? 0 : lo;
    const unsigned long long end = staged ? hi - lo : hi;
    const K* S = staged ? sf : F;
#pragma unroll
    for (int i = 0; i < kItemsC; ++i) {
      const uint32_t j = b + i;
      key[i] = 0;
      if (j < n) {
        const K c = sk[pad32(j)];
        key[i] = c;
        const bool firstc = j ? (c != sk[pad32(j - 1)]) : (start == 0 || c != s_prev);
        if (firstc) {
          unsigned long long a = cur, z = end;  // lower bound of c in S[cur, end)
          while (a < z) {
            const unsigned long long m = (a + z) >> 1;
            if (S[m] < c) a = m + 1; else z = m;
          }
          cur = a;
          if (!(a < end && S[a] == c)) keep |= 1u << i;
        }
      }
    }
    unsigned long long tot;
    const unsigned long long texcl = block_excl_scan((unsigned long long)__popc(keep), s_scan, &tot);
    const bool first = (t == sg.tile0);
    if (threadIdx.x == 0) {
      s_bad = 0;
      st_put(status + t, st_pack(epoch, first ? FLAG_INC : FLAG_AGG, tot));
    }
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
    __syncthreads();  // every read of sk is done: compact in place
    if (s_bad) return;
    uint32_t w = (uint32_t)texcl;
#pragma unroll
    for (int i = 0; i < kItemsC; ++i)
      if (keep >> i & 1u) sk[pad32(w++)] = key[i];
    __syncthreads();
    const unsigned long long ex = s_excl;
    K* o = out + sg.out_off + ex;
    for (uint32_t i = threadIdx.x; i < tot; i += kThreads) o[i] = sk[pad32(i)];
    if (threadIdx.x == 0 && t == sg.tile0 + sg.ntiles - 1) stp->segs[k].res = ex + tot;
  }
}

// ------------------------------------------------------------------ disjoint merge
// Merge path (Green, McColl, Bader 2012): number of A-elements among the first
// d outputs of merge(A, B) when A and B share no key.
template <typename K>
__device__ __forceinline__ unsigned long long merge_path(const K* A, unsigned long long na,
                                                         const K* B, unsigned long long nb,
                                                         unsigned long long d) {
  unsigned long long lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const unsigned long long m = (lo + hi) >> 1;
    if (A[m] < B[d - 1 - m]) lo = m + 1; else hi = m;
  }
  return lo;
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_merge(Stage* stp) {
  __shared__ K sm[kTileM];
  __shared__ unsigned long long s_a0, s_a1;
  __shared__ uint32_t s_t;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  const K* A_all = (const K*)stp->in;
  const K* B_all = (const K*)stp->aux;
  const uint32_t nseg = stp->nseg, ntiles = stp->ntiles;
  for (;;) {
    const uint32_t t = claim_tile(stp, &s_t);
    if (t >= ntiles) return;
    const uint32_t k = find_seg(stp->segs, nseg, t, stp->tile_seg);
    const Seg sg = stp->segs[k];
    const K* A = A_all + sg.in_off;
    const K* B = B_all + sg.aux_off;
    const unsigned long long na = sg.n, nb = sg.aux_n;
    K* out = (K*)((sg.flags & 1u) ? stp->out2 : stp->out) + sg.out_off;
    const unsigned long long d0 = (unsigned long long)(t - sg.tile0) * kTileM;
    const unsigned long long d1 = min(d0 + kTileM, na + nb);
    const bool last = t == sg.tile0 + sg.ntiles - 1;
    if (stp->splits) {
      if (threadIdx.x == 0) s_a0 = stp->splits[t];
      if (threadIdx.x == 32) s_a1 = last ? na : stp->splits[t + 1];
    } else {
      if (threadIdx.x == 0) s_a0 = merge_path(A, na, B, nb, d0);
      if (threadIdx.x == 32) s_a1 = merge_path(A, na, B, nb, d1);
    }
    __syncthreads();
    const unsigned long long a0 = s_a0, a1 = s_a1, b0 = d0 - a0, b1 = d1 - a1;
    const uint32_t la = (uint32_t)(a1 - a0), lb = (uint32_t)(b1 - b0);
    if (lb == 0 || la == 0) {  // one side only: a straight copy
      const K* src = lb == 0 ? A + a0 : B + b0;
      const uint32_t cnt = lb == 0 ? la : lb;
      K v[kTileM / kThreads];
#pragma unroll
      for (int e = 0; e < kTileM / kThreads; ++e) {
        const uint32_t i = threadIdx.x + e * kThreads;
        v[e] = i < cnt ? src[i] : (K)0;
      }
#pragma unroll
      for (int e = 0; e < kTileM / kThreads; ++e) {
        const uint32_t i = threadIdx.x + e * kThreads;
        if (i < cnt) out[d0 + i] = v[e];
      }
    } else {
      {
        K v[kTileM / kThreads];
#pragma unroll
        for (int e = 0; e < kTileM / kThreads; ++e) {
          const uint32_t i = threadIdx.x + e * kThreads;
          v[e] = i < la ? A[a0 + i] : (i < la + lb ? B[b0 + i - la] : (K)0);
        }
#pragma unroll
        for (int e = 0; e < kTileM / kThreads; ++e) {
          const uint32_t i = threadIdx.x + e * kThreads;
          if (i < la + lb) sm[i] = v[e];
        }
      }
      __syncthreads();
      const K* SA = sm;
      const K* SB = sm + la;
      for (uint32_t q = threadIdx.x; q < la + lb; q += kThreads) {
        uint32_t lo = q > lb ? q - lb : 0, hi = q < la ? q : la;
        while (lo < hi) {
          const uint32_t m = (lo + hi) >> 1;
          if (SA[m] < SB[q - 1 - m]) lo = m + 1; else hi = m;
        }
        const uint32_t ib = q - lo;
        const bool takeA = lo < la && (ib >= lb || SA[lo] < SB[ib]);
        out[d0 + q] = takeA ? SA[lo] : SB[ib];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ fused dedup + diff + merge
// One merge-path pass over (Full, sorted candidates C) per instance.  In the
// merged order ties put the Full element first, so a candidate is new exactly
// when it differs from the element just before it: that single predicate is
// both filters of Sec. Fused Deduplication and Set Difference.  Every kept
// element is also written, in merged order, as Full' = Full u N -- the
// disjoint merge of Sec. Disjoint Merge in the same pass, so Full is streamed
// once (no binary searches) and N is never read back.  Output positions: a
// tile's N-prefix comes from a decoupled lookback; the Full' position of a
// kept element is (Full elements before it) + (N elements before it).
template <typename K>
__device__ __forceinline__ unsigned long long mpath_tie(const K* A, unsigned long long na,
                                                        const K* B, unsigned long long nb,
                                                        unsigned long long d) {
  // number of A elements among the first d of the merge (A first on ties)
  unsigned long long lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const unsigned long long m = (lo + hi) >> 1;
    if (A[m] <= B[d - 1 - m]) lo = m + 1; else hi = m;
  }
  return lo;
}

// Per-tile state a CTA keeps between classifying a tile and writing it out.
struct FuseMeta {
  unsigned long long a0;  // Full elements before the tile
  uint32_t j, j0, k;      // mixed-tile index (lookback words), first one of the segment, segment
  uint32_t totK, totN;    // kept elements (Full' part) and new tuples of the tile
  uint32_t first, last;   // first / last mixed tile of its segment
};

// Classify tile t into slot `sb`: load its Full and candidate parts, merge,
// mark kept and new elements, publish the tile's new-tuple count, and leave
// the kept elements in Full' order in sbuf plus, per thread, where its kept
// run starts, how many new tuples precede it, and its two masks.
template <typename K, int T>
__device__ __forceinline__ void fuse_classify(Stage* stp, uint32_t j, K* sbuf, uint32_t* smask,
                                              uint32_t* spre, FuseMeta* meta,
                                              unsigned long long* s_scan,
                                              unsigned long long* s_a0, unsigned long long* s_a1,
                                              K* s_prev, uint32_t* s_hasprev) {
  constexpr int E = T / kThreads;
  const K* Aall = (const K*)stp->in;     // Full
  const K* Ball = (const K*)stp->aux;    // sorted candidates
  const uint32_t t = stp->mixl ? stp->mixl[j] : j;
  const uint32_t k = find_seg(stp->segs, stp->nseg, t, stp->tile_seg);
  const Seg sg = stp->segs[k];
  const uint32_t j0 = stp->mixc ? stp->mixc[sg.tile0] : sg.tile0;
  const uint32_t jl = (stp->mixc ? stp->mixc[sg.tile0 + sg.ntiles] : sg.tile0 + sg.ntiles) - 1;
  const K* A = Aall + sg.in_off;
  const K* B = Ball + sg.aux_off;
  const unsigned long long na = sg.n, nb = sg.aux_n;
  const unsigned long long d0 = (unsigned long long)(t - sg.tile0) * T;
  const unsigned long long d1 = min(d0 + (unsigned long long)T, na + nb);
  const bool last = t == sg.tile0 + sg.ntiles - 1;
  if (stp->splits) {
    if (threadIdx.x == 0) *s_a0 = stp->splits[t];
    if (threadIdx.x == 32) *s_a1 = last ? na : stp->splits[t + 1];
  } else {
    if (threadIdx.x == 0) *s_a0 = mpath_tie(A, na, B, nb, d0);
    if (threadIdx.x == 32) *s_a1 = mpath_tie(A, na, B, nb, d1);
  }
  __syncthreads();
  const unsigned long long a0 = *s_a0, a1 = *s_a1, b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t la = (uint32_t)(a1 - a0), lb = (uint32_t)(b1 - b0), L = la + lb;
  {  // Full part then candidate part, every load in flight at once
    const K* pa0 = A + a0;
    const K* pb0 = B + b0;
    K v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = threadIdx.x + e * kThreads;
      const K* src = i < la ? pa0 + i : pb0 + (i - la);
      v[e] = i < L ? *src : (K)0;
    }
    K pa = 0, pb = 0;
    if (threadIdx.x == 0) {
      // the element just before this tile in merged order (its largest predecessor)
      if (a0 > 0) pa = A[a0 - 1];
      if (b0 > 0) pb = B[b0 - 1];
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = threadIdx.x + e * kThreads;
      if (i < L) sbuf[pad32(i)] = v[e];
    }
    if (threadIdx.x == 0) {
      *s_hasprev = d0 > 0;
      *s_prev = pb > pa ? pb : pa;
    }
  }
  __syncthreads();
  // padded views of the Full part (SA) and the candidate part (SB)
  auto SA = [&](uint32_t i) { return sbuf[pad32(i)]; };
  auto SB = [&](uint32_t j) { return sbuf[pad32(la + j)]; };
  // blocked: thread owns merged positions [q0, q0 + E)
  const uint32_t q0 = threadIdx.x * E;
  K val[E];
  uint32_t isN = 0, kept = 0;   // bit i: output i is a new tuple / is kept
  if (q0 < L) {
    uint32_t i, j;
    {  // merge path inside the tile (Full first on ties)
      uint32_t lo = q0 > lb ? q0 - lb : 0, hi = q0 < la ? q0 : la;
      while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (SA(m) <= SB(q0 - 1 - m)) lo = m + 1; else hi = m;
      }
      i = lo;
      j = q0 - i;
    }
    // the merged predecessor of position q0; with none (the segment's first
    // element) the complement of that element, so it counts as different
    K prev;
    if (q0 > 0) {
      prev = i > 0 ? SA(i - 1) : (K)0;
      if (j > 0 && SB(j - 1) > prev) prev = SB(j - 1);
    } else if (*s_hasprev) {
      prev = *s_prev;
    } else {
      prev = ~((la > 0 && (lb == 0 || SA(0) <= SB(0))) ? SA(0) : SB(0));
    }
    // branch-free merge, heads in registers: each step reads the next element
    // of the side that advanced (index <= L <= T: inside sbuf).  An exhausted
    // B side reads as the largest key, so A wins every comparison until it is
    // exhausted too; an exhausted A side is never taken (i < la fails).
    K a = SA(i), b = j < lb ? SB(j) : ~(K)0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      val[e] = 0;
      if (q0 + e < L) {
        const bool takeA = i < la && a <= b;
        const K v = takeA ? a : b;
        const K w = sbuf[pad32(takeA ? i + 1 : la + j + 1)];
        i += takeA ? 1u : 0u;
        j += takeA ? 0u : 1u;
        a = takeA ? w : a;
        b = takeA ? b : (j < lb ? w : ~(K)0);
        const bool isnew = !takeA && v != prev;
        kept |= (takeA || isnew ? 1u : 0u) << e;
        isN |= (isnew ? 1u : 0u) << e;
        val[e] = v;
        prev = v;
      }
    }
  }
  // one scan for both counts: N in the high half, kept in the low half
  unsigned long long tot;
  const unsigned long long both = ((unsigned long long)__popc(isN) << 32) | __popc(kept);
  const unsigned long long ex = block_excl_scan(both, s_scan, &tot);  // ends with a barrier:
  const uint32_t totN = (uint32_t)(tot >> 32), totK = (uint32_t)tot;  // sbuf reads are done
  const bool first = (j == j0);
  if (threadIdx.x == 0) {
    st_put(stp->status + j, st_pack(stp->epoch, first ? FLAG_INC : FLAG_AGG, totN));
    meta->a0 = a0; meta->j = j; meta->j0 = j0; meta->k = k; meta->totK = totK; meta->totN = totN;
    meta->first = first; meta->last = j == jl;
  }
  // kept elements in Full' order, at tile-local positions
  uint32_t wk = (uint32_t)ex;
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (kept >> e & 1u) sbuf[pad32(wk++)] = val[e];
  smask[threadIdx.x] = (isN << 16) | kept;           // E <= 16
  spre[threadIdx.x] = ((uint32_t)(ex >> 32) << 16) | (uint32_t)ex;  // both < 2^16 (T <= 4096)
}

// Write out a classified tile once its new-tuple prefix exN is known.
template <typename K, int T>
__device__ __forceinline__ void fuse_write(Stage* stp, const K* sbuf, const uint32_t* smask,
                                           const uint32_t* spre, const FuseMeta& m,
                                           unsigned long long exN) {
  constexpr int E = T / kThreads;
  const Seg& sg = stp->segs[m.k];
  K* Nall = (K*)stp->out;                // new delta
  K* Fall = (K*)stp->out2;               // Full'
  // new tuples are few: each thread stores its own run of them directly,
  // visiting only the set bits (a new tuple's place among the kept elements
  // is the number of kept bits below it)
  const uint32_t mk = smask[threadIdx.x], pr = spre[threadIdx.x];
  const uint32_t kept = mk & 0xFFFFu, wk0 = pr & 0xFFFFu;
  K* no = Nall + sg.out_off + exN + (pr >> 16);
  for (uint32_t nb = mk >> 16; nb; nb &= nb - 1) {
    const uint32_t e = __ffs(nb) - 1;
    *no++ = sbuf[pad32(wk0 + __popc(kept & ((1u << e) - 1u)))];
  }
  if (Fall) {  // no Full' when the pass only finds what the main run lacks (side iteration)
    K* fo = Fall + sg.out2_off + m.a0 + exN;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = threadIdx.x + e * kThreads;
      if (i < m.totK) fo[i] = sbuf[pad32(i)];
    }
  }
  if (threadIdx.x == 0 && m.last) stp->segs[m.k].res = exN + m.totN;
}

// The fused pass over the mixed tiles (k_fuse_list's order; every tile when
// the stage has no list).  Lookback words are indexed by the mixed-tile index:
// Full-only tiles add no new tuples.  Software-pipelined over two tiles: a CTA
// classifies its next tile (and publishes that tile's count) before it looks
// back for the previous one, so the predecessors the lookback waits on have
// had one tile time to publish.  Deadlock-free: publishing a tile's count
// never waits, so the oldest unfinished tile can always complete its lookback.
template <typename K, int T>
__global__ void __launch_bounds__(kThreads, 5) k_diff_merge(Stage* stp) {
  static_assert(T / kThreads <= 16 && T <= 65535, "masks and prefixes are packed in 16 bits");
  __shared__ K sbuf[2][Padded<T>::n];  // tile input, then its kept elements in Full' order
  __shared__ uint32_t smask[2][kThreads], spre[2][kThreads];
  __shared__ FuseMeta smeta[2];
  __shared__ unsigned long long s_scan[kWarps];
  __shared__ unsigned long long s_a0, s_a1, s_excl;
  __shared__ K s_prev;
  __shared__ uint32_t s_hasprev, s_t, s_bad;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  // the tiles holding candidates (the others are copied by k_fuse_copy)
  const uint32_t ntiles = stp->mixc ? stp->mixc[stp->ntiles] : stp->ntiles;
  uint32_t cur = 0;
  uint32_t t = claim_tile(stp, &s_t);
  if (t >= ntiles) return;
  fuse_classify<K, T>(stp, t, sbuf[0], smask[0], spre[0], &smeta[0], s_scan, &s_a0, &s_a1, &s_prev,
                      &s_hasprev);
  for (;;) {
    // next tile first (claim_tile's barriers also publish smeta[cur])
    const uint32_t tn = claim_tile(stp, &s_t);
    const bool more = tn < ntiles;
    if (more)
      fuse_classify<K, T>(stp, tn, sbuf[cur ^ 1], smask[cur ^ 1], spre[cur ^ 1], &smeta[cur ^ 1],
                          s_scan, &s_a0, &s_a1, &s_prev, &s_hasprev);
    const FuseMeta m = smeta[cur];
    if (threadIdx.x == 0) s_bad = 0;
    if (!m.first && threadIdx.x < 32) {
      const unsigned long long e = lookback_scalar(stp->status, m.j, m.j0, stp->epoch, ctl);
      if (threadIdx.x == 0) {
        s_excl = e;
        if (*(volatile uint32_t*)&ctl->abort) s_bad = 1;
        st_put(stp->status + m.j, st_pack(stp->epoch, FLAG_INC, e + m.totN));
      }
    } else if (m.first && threadIdx.x == 0) {
      s_excl = 0;
    }
    __syncthreads();  // the kept elements, masks and s_excl of the previous tile are visible
    if (s_bad) return;
    fuse_write<K, T>(stp, sbuf[cur], smask[cur], spre[cur], m, s_excl);
    if (!more) return;
    cur ^= 1;
  }
}

// ------------------------------------------------------------------ fused pass: tile kinds
// After the merge-path partition, a tile of the fused pass either holds
// candidates ("mixed": classified by k_diff_merge) or Full elements only --
// all kept, in order, none new.  Most tiles are of the second kind once the
// deltas are small; k_fuse_copy moves them with plain coalesced copies, shifted
// by the new-tuple prefix of the last mixed tile before them, so k_diff_merge
// claims, classifies and looks back over the mixed tiles only.
__device__ __forceinline__ bool fuse_tile_mixed(const Stage& f, uint32_t t, uint32_t T) {
  const uint32_t k = find_seg(f.segs, f.nseg, t, f.tile_seg);
  const Seg& sg = f.segs[k];
  const unsigned long long na = sg.n, nb = sg.aux_n;
  const unsigned long long d0 = (unsigned long long)(t - sg.tile0) * T;
  const unsigned long long d1 = min(d0 + (unsigned long long)T, na + nb);
  const unsigned long long a0 = f.splits[t];
  const unsigned long long a1 = t == sg.tile0 + sg.ntiles - 1 ? na : f.splits[t + 1];
  return d1 - d0 > a1 - a0;  // fewer Full elements than positions: candidates inside
}

// Pass 1: mark mixed tiles (mixc[t] = 0/1) and count them per chunk of kThreads.
__global__ void __launch_bounds__(kThreads) k_fuse_mark(Dev* dv) {
  if (dv->ctl.abort) return;
  const Stage& f = dv->st[S_FUSE];
  const uint32_t ntiles = f.ntiles, T = dv->fuse_tile;
  const uint32_t nch = (ntiles + kThreads - 1) / kThreads;
  for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint32_t t = c * kThreads + threadIdx.x;
    const int mixed = t < ntiles && fuse_tile_mixed(f, t, T);
    if (t < ntiles) dv->mixc[t] = (uint32_t)mixed;
    const int cnt = __syncthreads_count(mixed);
    if (threadIdx.x == 0) dv->mixs[c] = (uint32_t)cnt;
  }
}

// Pass 2: mixc[t] = mixed tiles before t (mixc[ntiles] = all of them) and the
// list of mixed tiles in order.
__global__ void __launch_bounds__(kThreads) k_fuse_list(Dev* dv) {
  __shared__ unsigned long long sh[kWarps];
  if (dv->ctl.abort) return;
  const Stage& f = dv->st[S_FUSE];
  const uint32_t ntiles = f.ntiles;
  const uint32_t nch = (ntiles + kThreads - 1) / kThreads;
  if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) dv->mixc[0] = 0;
  for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
    unsigned long long pre = 0, tp;
    for (uint32_t q = threadIdx.x; q < c; q += kThreads) pre += dv->mixs[q];
    block_excl_scan(pre, sh, &tp);  // mixed tiles in the chunks before this one
    const uint32_t t = c * kThreads + threadIdx.x;
    const uint32_t mixed = t < ntiles ? dv->mixc[t] : 0u;
    unsigned long long tot;
    const uint32_t j = (uint32_t)(tp + block_excl_scan(mixed, sh, &tot));
    if (t < ntiles) {
      dv->mixc[t] = j;
      if (mixed) dv->mixl[j] = t;
    }
    if (t + 1 == ntiles) dv->mixc[ntiles] = j + mixed;
  }
}

// Pass 4 (after k_diff_merge): copy the Full-only tiles to Full'.
template <typename K, int T>
__global__ void __launch_bounds__(kThreads) k_fuse_copy(Stage* stp) {
  constexpr int E = T / kThreads;
  Ctl* ctl = stp->ctl;
  if (*(volatile uint32_t*)&ctl->abort) return;
  const uint32_t ntiles = stp->ntiles;
  const K* Aall = (const K*)stp->in;
  K* Fall = (K*)stp->out2;
  if (!Fall) return;  // side iteration: no Full' is written
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (stp->mixc[t + 1] != stp->mixc[t]) continue;  // mixed: k_diff_merge wrote it
    const uint32_t k = find_seg(stp->segs, stp->nseg, t, stp->tile_seg);
    const Seg& sg = stp->segs[k];
    const bool last = t == sg.tile0 + sg.ntiles - 1;
    const unsigned long long a0 = stp->splits[t], a1 = last ? sg.n : stp->splits[t + 1];
    const uint32_t la = (uint32_t)(a1 - a0);
    if ((unsigned long long)la > (unsigned long long)T) {  // not a Full-only tile: corrupt input
      if (threadIdx.x == 0) fail_timeout(ctl);
      return;
    }
    const uint32_t j0 = stp->mixc[sg.tile0], jp = stp->mixc[t];
    unsigned long long exN = 0;  // new tuples before the tile: last mixed tile's inclusive count
    if (jp > j0) {
      const unsigned long long w = st_get(stp->status + jp - 1);
      if (!st_ready(w, stp->epoch) || ((w >> 38) & 3u) != FLAG_INC) {
        if (threadIdx.x == 0) fail_timeout(ctl);
        return;
      }
      exN = w & kValMask;
    }
    const K* src = Aall + sg.in_off + a0;
    K* dst = Fall + sg.out2_off + a0 + exN;
    K v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = threadIdx.x + e * kThreads;
      v[e] = i < la ? src[i] : (K)0;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = threadIdx.x + e * kThreads;
      if (i < la) dst[i] = v[e];
    }
  }
}

// ------------------------------------------------------------------ tile partitions
// One thread per tile of the consumer stage: the merge-path split at the
// tile's first output (mode 0: merge of in/aux, Full first on ties), the
// delta tuple whose join slab holds the tile's first candidate (mode 1: tiles
// of `tile` candidates), or both the first candidate and its slab for join
// tiles over merged items (mode 2: each group of kEmitGroup delta tuples
// counts as one item ahead of its slabs' candidates, so a tile of `tile`
// items holds at most kEmitGroup * `tile` delta tuples however many slabs
// are empty).  All the binary searches are in flight at once instead of
// heading every tile.
template <typename K>
__global__ void k_partition(Stage* cons, int mode, uint32_t tile) {
  if (*(volatile uint32_t*)&cons->ctl->abort) return;
  const uint32_t ntiles = cons->ntiles, nseg = cons->nseg;
  unsigned long long* splits = cons->splits;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    const uint32_t k = find_seg(cons->segs, nseg, t);
    const Seg& sg = cons->segs[k];
    const unsigned long long d = (unsigned long long)(t - sg.tile0) * tile;
    if (mode == 0) {
      const K* A = (const K*)cons->in + sg.in_off;
      const K* B = (const K*)cons->aux + sg.aux_off;
      splits[t] = mpath_tie(A, sg.n, B, sg.aux_n, d);
    } else if (mode == 1) {
      splits[t] = upper_bound_k(cons->pos + sg.in_off, sg.n, d) - 1;
    } else {
      // merged item d: the item of group j sits at pos[j * kEmitGroup] + j
      // (increasing in j); h groups have theirs before d, so d - h
      // candidates precede it
      const unsigned long long* P = cons->pos + sg.in_off;
      unsigned long long lo = 0, hi = (sg.n + kEmitGroup - 1) >> kEmitGroupShift;
      while (lo < hi) {
        const unsigned long long m = (lo + hi) >> 1;
        if (P[m << kEmitGroupShift] + m < d) lo = m + 1; else hi = m;
      }
      const unsigned long long c0 = d - lo;
      cons->splits2[t] = c0;
      splits[t] = upper_bound_k(P, sg.n, c0) - 1;
    }
  }
}

// ------------------------------------------------------------------ launchers
template <typename K>
void launch_sort_hist(Stage* st, int grid, cudaStream_t s) { k_sort_hist<K><<<grid, kThreads, 0, s>>>(st); }
template <typename K>
void launch_sort_pass(Stage* st, int grid, cudaStream_t s, uint32_t dbits) {
  if (dbits == 8) k_sort_pass<K, true><<<grid, kThreads, 0, s>>>(st);
  else k_sort_pass<K, false><<<grid, kThreads, 0, s>>>(st);
}
template <typename K>
void launch_sort_seg(Stage* st0, int grid, cudaStream_t s, uint32_t dbits, int items, bool wide) {
  if (wide) {  // digits of up to 9 bits, 8 keys per thread
    if (dbits == 8) k_sort_seg<K, true, 8, kWideRadix><<<grid, kSegNT, 0, s>>>(st0);
    else k_sort_seg<K, false, 8, kWideRadix><<<grid, kSegNT, 0, s>>>(st0);
  } else if (items == 8) {
    if (dbits == 8) k_sort_seg<K, true, 8><<<grid, kSegNT, 0, s>>>(st0);
    else k_sort_seg<K, false, 8><<<grid, kSegNT, 0, s>>>(st0);
  } else {
    if (dbits == 8) k_sort_seg<K, true, 16><<<grid, kSegNT, 0, s>>>(st0);
    else k_sort_seg<K, false, 16><<<grid, kSegNT, 0, s>>>(st0);
  }
}
template <typename K>
void launch_unique_diff(Stage* st, int grid, cudaStream_t s) { k_unique_diff<K><<<grid, kThreads, 0, s>>>(st); }
template <typename K>
void launch_merge(Stage* st, int grid, cudaStream_t s) { k_merge<K><<<grid, kThreads, 0, s>>>(st); }
template <typename K>
void launch_diff_merge(Stage* st, int grid, cudaStream_t s, uint32_t tile) {
  constexpr int T = FuseTile<K>::T;
  if (tile == (uint32_t)T / 2) k_diff_merge<K, T / 2><<<grid, kThreads, 0, s>>>(st);
  else k_diff_merge<K, T><<<grid, kThreads, 0, s>>>(st);
}
void launch_fuse_mark(Dev* dv, int grid, cudaStream_t s) { k_fuse_mark<<<grid, kThreads, 0, s>>>(dv); }
void launch_fuse_list(Dev* dv, int grid, cudaStream_t s) { k_fuse_list<<<grid, kThreads, 0, s>>>(dv); }
template <typename K>
void launch_fuse_copy(Stage* st, int grid, cudaStream_t s, uint32_t tile) {
  constexpr int T = FuseTile<K>::T;
  if (tile == (uint32_t)T / 2) k_fuse_copy<K, T / 2><<<grid, kThreads, 0, s>>>(st);
  else k_fuse_copy<K, T><<<grid, kThreads, 0, s>>>(st);
}
template <typename K>
void launch_partition(Stage* consumer, int mode, uint32_t tile, int grid, cudaStream_t s) {
  k_partition<K><<<grid, 256, 0, s>>>(consumer, mode, tile);
}

// Resident CTAs per SM of a persistent kernel.  The kernel first asks for the
// largest shared-memory carveout: with the default split the SM would host
// fewer CTAs than its registers allow.
template <typename F>
int occupancy_of(F kern, int threads = kThreads) {
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, 0);
  return b;
}

template <typename K>
int occupancy_sort(int which) {
  switch (which) {
    case 0: return occupancy_of(k_sort_hist<K>);
    case 1: return occupancy_of(k_sort_pass<K, true>);
    case 2: return occupancy_of(k_unique_diff<K>);
    case 3: return occupancy_of(k_merge<K>);
    case 4: return occupancy_of(k_diff_merge<K, FuseTile<K>::T>);
    case 5: return occupancy_of(k_diff_merge<K, FuseTile<K>::T / 2>);
    case 6: return occupancy_of(k_sort_seg<K, true, 16>, kSegNT);
    case 7: return occupancy_of(k_sort_seg<K, true, 8>, kSegNT);
    case 8: return occupancy_of(k_sort_seg<K, false, 8, kWideRadix>, kSegNT);
    default: return 0;
  }
}

#define WG_INST(K)                                              \
  template void launch_sort_hist<K>(Stage*, int, cudaStream_t);  \
  template void launch_sort_pass<K>(Stage*, int, cudaStream_t, uint32_t); \
  template void launch_sort_seg<K>(Stage*, int, cudaStream_t, uint32_t, int, bool); \
  template void launch_unique_diff<K>(Stage*, int, cudaStream_t); \
  template void launch_merge<K>(Stage*, int, cudaStream_t);      \
  template void launch_diff_merge<K>(Stage*, int, cudaStream_t, uint32_t); \
  template void launch_fuse_copy<K>(Stage*, int, cudaStream_t, uint32_t);  \
  template void launch_partition<K>(Stage*, int, uint32_t, int, cudaStream_t); \
  template int occupancy_sort<K>(int);
WG_INST(uint32_t)
WG_INST(unsigned long long)
#undef WG_INST

}  // namespace wg
