// wg_launch.h -- host-side launchers of the sm_103a kernels (one translation
// unit per kernel family; the host engine only sees these declarations).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wg {

// Records `msg` as the calling thread's wg_last_error() and returns `code`.
int set_error(int code, const char* msg);

struct Stage;
struct Dev;
struct Inst;

// sorted-array stages (wg_kern_sort.cu); K = uint32_t or unsigned long long
template <typename K> void launch_sort_hist(Stage* st, int grid, cudaStream_t s);
// dbits: digit width of the pass plan (8 picks the whole-byte-digit kernel)
template <typename K> void launch_sort_pass(Stage* st, int grid, cudaStream_t s, uint32_t dbits);
// every pass of segments of at most kSegSortMaxTiles tiles, one CTA per segment
// (st0: the first pass's stage; the later passes' stages follow it)
template <typename K> void launch_sort_seg(Stage* st0, int grid, cudaStream_t s, uint32_t dbits,
                                           int items, bool wide);  // keys per thread: 16 or 8
template <typename K> void launch_unique_diff(Stage* st, int grid, cudaStream_t s);
template <typename K> void launch_merge(Stage* st, int grid, cudaStream_t s);
// tile: merged keys per fused-pass tile, FuseTile<K>::T or half of it
template <typename K> void launch_diff_merge(Stage* st, int grid, cudaStream_t s, uint32_t tile);
// mode 0: merge-path splits of a (Full, candidates) / (Full, delta) stage;
// mode 1: join-slab owner of each emit tile.  `tile` = outputs per tile.
template <typename K>
void launch_partition(Stage* consumer, int mode, uint32_t tile, int grid, cudaStream_t s);
template <typename K> int occupancy_sort(int which);  // 0 hist, 1 pass, 2 uniq, 3 merge, 4 fused,
                                                      // 5 fused with half tiles, 6 / 7 segment sort
                                                      // of 16 / 8 keys per thread

// join and engine control (wg_kern_join.cu)
// tile: delta tuples per count tile, kTileD or kTileD / 2
template <typename K> void launch_join_count(Stage* st, int grid, cudaStream_t s, uint32_t tile);
template <typename K> void launch_join_emit(Stage* st, int grid, cudaStream_t s, uint32_t tile);
template <typename K> void launch_tri_probe(Stage* st, int grid, cudaStream_t s);
void launch_fuse_mark(Dev* dv, int grid, cudaStream_t s);
void launch_fuse_list(Dev* dv, int grid, cudaStream_t s);
template <typename K> void launch_fuse_copy(Stage* st, int grid, cudaStream_t s, uint32_t tile);
template <typename K> void launch_join_emit_hash(Stage* st, int grid, cudaStream_t s);
template <typename K>
void launch_hash_build(const K* E, unsigned long long ne, uint32_t w, unsigned long long* T,
                       unsigned long long mask, int grid, cudaStream_t s);
template <typename K> int occupancy_join(int which);  // 0 count, 1 emit, 2 triangle probe,
                                                      // 3 count with half tiles
// one warp waiting on a status word that is never published (bounded wait self-test)
struct Ctl;
void launch_selftest_wait(const unsigned long long* status, Ctl* ctl, unsigned long long* out,
                          cudaStream_t s);
// the same wait in the allocation-free sort's control block (wg_noalloc.cu)
int noalloc_selftest_wait(cudaStream_t s);
void launch_plan_delta(Dev* dv, cudaStream_t s);
void launch_plan_cand(Dev* dv, cudaStream_t s);
void launch_plan_merge(Dev* dv, cudaStream_t s);
void launch_plan_post(Dev* dv, cudaStream_t s);
void launch_plan_side(Dev* dv, cudaStream_t s);
void launch_xseg_build(Dev* dv, cudaStream_t s);
template <typename K>
void launch_init_diag(Inst* inst, uint32_t first, uint32_t count, void* dpool, cudaStream_t s);

// relation load and result extraction
template <typename K>
void launch_rank_edges(const uint32_t* src, const uint32_t* dst, unsigned long long n,
                       const uint32_t* V, uint32_t nv, uint32_t w, K* keys, int grid,
                       cudaStream_t s);
template <typename K>
void launch_csr(const K* E, unsigned long long ne, uint32_t nv, uint32_t w, uint32_t* off,
                uint32_t* adj, int grid, cudaStream_t s);
template <typename K>
void launch_result_map(const K* F, unsigned long long n, uint32_t w, const uint32_t* V,
                       unsigned long long* out, int grid, cudaStream_t s);
// adds the digest of the n tuples F (ranks mapped to ids through V) to *out
template <typename K>
void launch_result_digest(const K* F, unsigned long long n, uint32_t w, const uint32_t* V,
                          unsigned long long* out, int grid, cudaStream_t s);

}  // namespace wg
