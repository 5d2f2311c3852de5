// wg_host.cu -- host runtime of libwg: context, device memory, relation load,
// the fixpoint engine (a CUDA graph whose conditional WHILE node holds the
// semi-naive loop), batching / continuous serving, and the C-ABI of wg.h.
//
// Engine rule (Sec. Asynchronous Fixpoint Engine): the GPU decides every
// stage, iteration and buffer transition; the host only learns that the
// fixpoint was reached.  Here the device also decides termination (the WHILE
// condition is set by the plan kernel that sees the empty delta), so a query
// costs one graph launch unless a buffer turns out too small: then the run
// stops before writing past it, the host grows the pools (live data copied),
// and the same graph is launched again from the unchanged (Full, Delta, i).
#include <algorithm>
#include <chrono>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/wg.h"
#include "wg_device.cuh"
#include "wg_launch.h"

using namespace wg;

namespace {
thread_local std::string g_err;

int set_err(int code, const std::string& m) {
  g_err = m;
  return code;
}
#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(WG_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)
#define TRY(call)               \
  do {                          \
    int r_ = (call);            \
    if (r_ != WG_OK) return r_; \
  } while (0)

}  // namespace

int wg::set_error(int code, const char* msg) { return set_err(code, msg); }

namespace {
uint32_t bits_for(uint64_t nv) {  // bits to hold ranks 0..nv-1 (at least 1)
  uint32_t w = 1;
  while (w < 32 && (1ull << w) < nv) ++w;
  return w;
}
size_t round_up(size_t b) { return (b + 255) & ~size_t(255); }
double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct Relation;
struct Query;
struct EngineBase;

// ------------------------------------------------------------------ context
struct wg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  wg_alloc_fn alloc = nullptr;
  wg_free_fn free_fn = nullptr;
  void* user = nullptr;
  size_t budget = 0, used = 0;
  int num_sms = 0;
  uint64_t next_id = 1;
  std::map<uint64_t, std::unique_ptr<Relation>> rels;
  std::map<uint64_t, std::unique_ptr<Query>> queries;
  std::vector<std::unique_ptr<EngineBase>> idle;  // single-query engines ready for reuse
  std::map<int, std::unique_ptr<EngineBase>> batch;  // batch engines by key class
  // one stream per batch key class, kept across engine rebuilds: an allocator
  // that caches freed blocks per stream (PyTorch's) can then hand a rebuilt
  // engine the blocks its predecessor freed instead of allocating anew
  std::map<int, cudaStream_t> class_st;
  std::vector<uint64_t> pending;                  // submitted, not yet admitted
  std::vector<uint64_t> completed;                // batch queries finished, not yet taken
  uint64_t excl = 0;  // batch query that runs with the whole budget (0: none), see batch_preempt
  uint64_t solo_run = 0;  // the served request running on a single-query engine (0: none)
  // tile shapes engines are built with, per key width (index 0: 4-byte keys,
  // 1: 8-byte); 0 = the compiled default.  Set by wg_autotune / wg_set_tiles.
  uint32_t tune_count[2] = {0, 0}, tune_fuse[2] = {0, 0}, tune_emit[2] = {0, 0};
  uint32_t tune_sort[2] = {WG_SORT_SEGMENT16, WG_SORT_SEGMENT16};  // enum wg_sort_mode
  cudaStream_t alloc_stream = nullptr;            // stream of allocations in progress (NULL: stream)
  // scratch of the standalone primitives
  void* s_tmp = nullptr; size_t s_tmp_bytes = 0;
  unsigned long long* s_status = nullptr; size_t s_status_n = 0;
  unsigned long long* s_hist = nullptr;
  Stage* s_stage = nullptr;
  Seg* s_seg = nullptr;
  Ctl* s_ctl = nullptr;
  uint32_t s_epoch = 0;
};

static void drop_idle_engines(wg_ctx* c, size_t bytes);
static int dev_alloc(wg_ctx* c, size_t bytes, void** out, cudaStream_t st) {
  *out = nullptr;
  if (bytes == 0) return WG_OK;
  bytes = round_up(bytes);
  if (c->used + bytes > c->budget) drop_idle_engines(c, bytes);  // unused pools go first
  if (c->used + bytes > c->budget)
    return set_err(WG_E_BUDGET, "allocation of " + std::to_string(bytes) +
                                    " bytes exceeds the memory budget");
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, (void*)st, c->user);
  } else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) return set_err(WG_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  c->used += bytes;
  *out = p;
  return WG_OK;
}
static int dev_alloc(wg_ctx* c, size_t bytes, void** out) {
  return dev_alloc(c, bytes, out, c->alloc_stream ? c->alloc_stream : c->stream);
}
static void dev_free(wg_ctx* c, void* p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  bytes = round_up(bytes);
  if (c->free_fn) c->free_fn(p, bytes, (void*)st, c->user);
  else cudaFreeAsync(p, st);
  c->used -= bytes;
}
static void dev_free(wg_ctx* c, void* p, size_t bytes) { dev_free(c, p, bytes, c->stream); }

// Allocations made inside this scope are stream-ordered on `st` (an engine's
// own stream), and their buffers are later freed on it.
struct AllocScope {
  wg_ctx* c;
  cudaStream_t prev;
  AllocScope(wg_ctx* c_, cudaStream_t st) : c(c_), prev(c_->alloc_stream) { c->alloc_stream = st; }
  ~AllocScope() { c->alloc_stream = prev; }
};

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;  // the stream the buffer was allocated on
  int get(wg_ctx* c, size_t b) {
    if (b <= bytes && p) return WG_OK;
    release(c);
    st = c->alloc_stream ? c->alloc_stream : c->stream;
    TRY(dev_alloc(c, b, &p, st));
    bytes = round_up(b);
    return WG_OK;
  }
  void release(wg_ctx* c) {
    dev_free(c, p, bytes, st ? st : c->stream);
    p = nullptr;
    bytes = 0;
  }
};

static int grid_of(wg_ctx* c, int occ) { return c->num_sms * std::max(1, occ); }

// ------------------------------------------------------------------ primitives
// Standalone segmented stages on one segment (relation load, wg_sort_keys,
// wg_unique_diff, wg_merge_disjoint).  Same kernels as the fixpoint loop.
static int prim_scratch(wg_ctx* c, size_t tmp_bytes, size_t ntiles) {
  if (!c->s_stage) {
    void* p;
    TRY(dev_alloc(c, sizeof(Stage) * S_NUM, &p)); c->s_stage = (Stage*)p;
    TRY(dev_alloc(c, sizeof(Seg), &p)); c->s_seg = (Seg*)p;
    TRY(dev_alloc(c, sizeof(Ctl), &p)); c->s_ctl = (Ctl*)p;
    TRY(dev_alloc(c, sizeof(unsigned long long) * kMaxPasses * kRadix, &p));
    c->s_hist = (unsigned long long*)p;
    CK(cudaMemsetAsync(c->s_ctl, 0, sizeof(Ctl), c->stream));
  }
  if (tmp_bytes > c->s_tmp_bytes) {
    dev_free(c, c->s_tmp, c->s_tmp_bytes);
    c->s_tmp = nullptr; c->s_tmp_bytes = 0;
    TRY(dev_alloc(c, tmp_bytes, &c->s_tmp));
    c->s_tmp_bytes = round_up(tmp_bytes);
  }
  const size_t need = (ntiles + 1) * kRadix;
  if (need > c->s_status_n) {
    dev_free(c, c->s_status, c->s_status_n * 8);
    c->s_status = nullptr; c->s_status_n = 0;
    void* p;
    TRY(dev_alloc(c, need * 8, &p));
    c->s_status = (unsigned long long*)p;
    c->s_status_n = need;
    CK(cudaMemsetAsync(c->s_status, 0, need * 8, c->stream));
    c->s_epoch = 0;
  }
  return WG_OK;
}
static uint32_t prim_epoch(wg_ctx* c) {
  if (++c->s_epoch >= (1u << 23)) {  // epochs wrap at 24 bits: clear the words first
    cudaMemsetAsync(c->s_status, 0, c->s_status_n * 8, c->stream);
    c->s_epoch = 1;
  }
  return c->s_epoch;
}
static Stage prim_stage(wg_ctx* c, uint32_t ntiles) {
  Stage s{};
  s.segs = c->s_seg; s.ctl = c->s_ctl; s.status = c->s_status; s.hist = c->s_hist;
  s.nseg = 1; s.ntiles = ntiles;
  return s;
}
static int prim_put(wg_ctx* c, int slot, const Stage& s) {
  CK(cudaMemcpyAsync(c->s_stage + slot, &s, sizeof(Stage), cudaMemcpyHostToDevice, c->stream));
  return WG_OK;
}
static int prim_seg(wg_ctx* c, const Seg& s) {
  CK(cudaMemcpyAsync(c->s_seg, &s, sizeof(Seg), cudaMemcpyHostToDevice, c->stream));
  return WG_OK;
}

static void pass_plan(uint32_t bits, uint32_t* passes, uint32_t* dbits) {
  bits = std::max(1u, bits);
  *passes = (bits + 7) / 8;
  *dbits = (bits + *passes - 1) / *passes;
}

template <typename K>
static int prim_sort(wg_ctx* c, K* keys, size_t n, uint32_t bits) {
  if (n <= 1) return WG_OK;
  const uint32_t ntiles = (uint32_t)((n + kTileC - 1) / kTileC);
  TRY(prim_scratch(c, n * sizeof(K), ntiles));
  uint32_t passes, dbits;
  pass_plan(bits, &passes, &dbits);
  Seg sg{};
  sg.n = n; sg.tile0 = 0; sg.ntiles = ntiles;
  TRY(prim_seg(c, sg));
  CK(cudaMemsetAsync(c->s_hist, 0, sizeof(unsigned long long) * passes * kRadix, c->stream));
  // a wait that gave up in an earlier primitive must not make these passes
  // skip their work: the control block starts clear (the caller reads it after)
  CK(cudaMemsetAsync(c->s_ctl, 0, sizeof(Ctl), c->stream));
  Stage h = prim_stage(c, ntiles);
  h.in = keys; h.passes = passes; h.dbits = dbits;
  TRY(prim_put(c, S_HIST, h));
  K* buf[2] = {keys, (K*)c->s_tmp};
  for (uint32_t p = 0; p < passes; ++p) {
    Stage s = h;
    s.in = buf[p & 1]; s.out = buf[(p + 1) & 1];
    s.shift = p * dbits; s.pass = p; s.epoch = prim_epoch(c);
    TRY(prim_put(c, S_PASS0 + p, s));
  }
  launch_sort_hist<K>(c->s_stage + S_HIST, grid_of(c, occupancy_sort<K>(0)), c->stream);
  for (uint32_t p = 0; p < passes; ++p)
    launch_sort_pass<K>(c->s_stage + S_PASS0 + p, grid_of(c, occupancy_sort<K>(1)), c->stream, dbits);
  CK(cudaGetLastError());
  if (passes & 1) CK(cudaMemcpyAsync(keys, c->s_tmp, n * sizeof(K), cudaMemcpyDeviceToDevice, c->stream));
  return WG_OK;
}

template <typename K>
static int prim_unique(wg_ctx* c, const K* in, size_t n, const K* full, size_t nf, K* out,
                       size_t* n_out) {
  *n_out = 0;
  if (n == 0) return WG_OK;
  const uint32_t ntiles = (uint32_t)((n + kTileC - 1) / kTileC);
  TRY(prim_scratch(c, 0, ntiles));
  Seg sg{};
  sg.n = n; sg.aux_n = nf; sg.ntiles = ntiles;
  TRY(prim_seg(c, sg));
  Stage u = prim_stage(c, ntiles);
  u.in = in; u.aux = full; u.out = out; u.epoch = prim_epoch(c);
  TRY(prim_put(c, S_UNIQ, u));
  launch_unique_diff<K>(c->s_stage + S_UNIQ, grid_of(c, occupancy_sort<K>(2)), c->stream);
  CK(cudaGetLastError());
  Seg back{};
  Ctl ctl{};
  CK(cudaMemcpyAsync(&back, c->s_seg, sizeof(Seg), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&ctl, c->s_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (ctl.error) {
    cudaMemsetAsync(c->s_ctl, 0, sizeof(Ctl), c->stream);
    return set_err(WG_E_DEVICE_TIMEOUT, "a device lookback wait gave up");
  }
  *n_out = back.res;
  return WG_OK;
}

template <typename K>
static int prim_merge(wg_ctx* c, const K* a, size_t na, const K* b, size_t nb, K* out) {
  if (na + nb == 0) return WG_OK;
  const uint32_t ntiles = (uint32_t)((na + nb + kTileM - 1) / kTileM);
  TRY(prim_scratch(c, 0, 0));
  Seg sg{};
  sg.n = na; sg.aux_n = nb; sg.ntiles = ntiles;
  TRY(prim_seg(c, sg));
  Stage m = prim_stage(c, ntiles);
  m.in = a; m.aux = b; m.out = out;
  TRY(prim_put(c, S_MERGE, m));
  launch_merge<K>(c->s_stage + S_MERGE, grid_of(c, occupancy_sort<K>(3)), c->stream);
  CK(cudaGetLastError());
  return WG_OK;
}

// ------------------------------------------------------------------ relations
struct Relation {
  uint64_t ne = 0;
  uint32_t nv = 0, w = 1;
  int kb = 4;
  DBuf keys, off, adj, V;
  DBuf htab;                      // hash-join ablation: E in a linear-probing table (lazy)
  unsigned long long hmask = 0;
  uint64_t peak_cand = 0, peak_full = 0;  // capacities seen by earlier queries
  void release(wg_ctx* c) {
    keys.release(c); off.release(c); adj.release(c); V.release(c); htab.release(c);
  }
};

template <typename K>
static int build_edges(wg_ctx* c, Relation* R, const uint32_t* d_src, const uint32_t* d_dst,
                       size_t n) {
  DBuf kt, ke;
  TRY(kt.get(c, n * sizeof(K)));
  launch_rank_edges<K>(d_src, d_dst, n, (const uint32_t*)R->V.p, R->nv, R->w, (K*)kt.p,
                       grid_of(c, 4), c->stream);
  CK(cudaGetLastError());
  TRY(prim_sort<K>(c, (K*)kt.p, n, 2 * R->w));
  TRY(ke.get(c, n * sizeof(K)));
  size_t ne = 0;
  TRY(prim_unique<K>(c, (const K*)kt.p, n, (const K*)nullptr, 0, (K*)ke.p, &ne));
  kt.release(c);
  R->ne = ne;
  R->keys = ke;
  TRY(R->off.get(c, (size_t(R->nv) + 1) * 4));
  TRY(R->adj.get(c, std::max<size_t>(ne, 1) * 4));
  launch_csr<K>((const K*)ke.p, ne, R->nv, R->w, (uint32_t*)R->off.p, (uint32_t*)R->adj.p,
                grid_of(c, 4), c->stream);
  CK(cudaGetLastError());
  return WG_OK;
}

static int load_relation(wg_ctx* c, const uint32_t* d_src, const uint32_t* d_dst, size_t n,
                         Relation* R) {
  if (n >= (1ull << 32)) return set_err(WG_E_INVAL, "at most 2^32 - 1 edges");
  if (n == 0) {
    R->nv = 0; R->w = 1; R->kb = 4; R->ne = 0;
    TRY(R->off.get(c, 4));
    TRY(R->adj.get(c, 4));
    TRY(R->V.get(c, 4));
    CK(cudaMemsetAsync(R->off.p, 0, 4, c->stream));
    return WG_OK;
  }
  // distinct vertex ids, sorted: ranks keep the order of ids
  DBuf ids, vt;
  TRY(ids.get(c, 2 * n * 4));
  CK(cudaMemcpyAsync(ids.p, d_src, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync((uint32_t*)ids.p + n, d_dst, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  TRY(prim_sort<uint32_t>(c, (uint32_t*)ids.p, 2 * n, 32));
  TRY(vt.get(c, 2 * n * 4));
  size_t nv = 0;
  TRY(prim_unique<uint32_t>(c, (const uint32_t*)ids.p, 2 * n, nullptr, 0, (uint32_t*)vt.p, &nv));
  ids.release(c);
  TRY(R->V.get(c, nv * 4));
  CK(cudaMemcpyAsync(R->V.p, vt.p, nv * 4, cudaMemcpyDeviceToDevice, c->stream));
  vt.release(c);
  R->nv = (uint32_t)nv;
  R->w = bits_for(nv);
  R->kb = 2 * R->w <= 32 ? 4 : 8;
  if (R->kb == 4) return build_edges<uint32_t>(c, R, d_src, d_dst, n);
  return build_edges<unsigned long long>(c, R, d_src, d_dst, n);
}

// ------------------------------------------------------------------ triangle counting
// triangle(a,b,c) <- edge(a,b), edge(b,c), edge(c,a) (Sec. Generalization,
// "Triangle Counting"): one pass of the sorted-array join with E as the
// delta.  The join count gives each edge (a,b) its slab of deg(b) two-paths;
// the emit kernel in probe mode tests each two-path (a,b,c) for E(c,a) by
// binary search and counts the hits.
template <typename K>
static int tri_count(wg_ctx* c, Relation* R, unsigned long long* count) {
  *count = 0;
  const size_t ne = R->ne;
  if (ne == 0) return WG_OK;
  const uint32_t ntd = (uint32_t)((ne + kTileD - 1) / kTileD);
  TRY(prim_scratch(c, 0, ntd));
  DBuf inst, pos, spl, hits;
  TRY(inst.get(c, sizeof(Inst)));
  TRY(pos.get(c, ne * 8));
  TRY(hits.get(c, 8));
  Inst I{};
  I.off = (const uint32_t*)R->off.p; I.adj = (const uint32_t*)R->adj.p;
  I.nv = R->nv; I.w = R->w; I.kind = KIND_TC; I.state = INST_ACTIVE; I.iter = 1; I.n_delta = ne;
  CK(cudaMemcpyAsync(inst.p, &I, sizeof(Inst), cudaMemcpyHostToDevice, c->stream));
  Seg sd{};
  sd.n = ne; sd.ntiles = ntd;
  TRY(prim_seg(c, sd));
  Stage k = prim_stage(c, ntd);
  k.in = R->keys.p; k.inst = (Inst*)inst.p; k.pos = (unsigned long long*)pos.p;
  k.epoch = prim_epoch(c);
  TRY(prim_put(c, S_COUNT, k));
  launch_join_count<K>(c->s_stage + S_COUNT, grid_of(c, occupancy_join<K>(0)), c->stream, kTileD);
  CK(cudaGetLastError());
  Seg back{};
  Ctl ctl{};
  CK(cudaMemcpyAsync(&back, c->s_seg, sizeof(Seg), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&ctl, c->s_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int rc = WG_OK;
  const unsigned long long paths = back.res;  // two-paths (a,b,c)
  if (!ctl.error && paths) {
    const unsigned long long ntiles = (paths + kTileC - 1) / kTileC;
    if (ntiles >= (1ull << 32)) return set_err(WG_E_CAPACITY, "too many two-paths");
    TRY(spl.get(c, (size_t)(ntiles + 1) * 8));  // (the probe has no lookback: no status words)
    Seg se{};
    se.n = ne; se.aux_n = paths; se.ntiles = (uint32_t)ntiles;
    TRY(prim_seg(c, se));
    CK(cudaMemsetAsync(hits.p, 0, 8, c->stream));
    Stage e = prim_stage(c, (uint32_t)ntiles);
    e.in = R->keys.p; e.inst = (Inst*)inst.p; e.pos = (unsigned long long*)pos.p;
    e.splits = (unsigned long long*)spl.p; e.probe = (unsigned long long*)hits.p;
    TRY(prim_put(c, S_EMIT, e));
    launch_partition<K>(c->s_stage + S_EMIT, 1, kTileC, c->num_sms * 4, c->stream);
    launch_tri_probe<K>(c->s_stage + S_EMIT, grid_of(c, occupancy_join<K>(2)), c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(count, hits.p, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&ctl, c->s_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (ctl.error) {
    cudaMemsetAsync(c->s_ctl, 0, sizeof(Ctl), c->stream);
    *count = 0;
    rc = set_err(WG_E_DEVICE_TIMEOUT, "a device lookback wait gave up");
  }
  inst.release(c); pos.release(c); spl.release(c); hits.release(c);
  return rc;
}

// ------------------------------------------------------------------ engine
struct KStat {
  const char* name;
  uint64_t launches = 0;
  double ms = 0, bytes = 0;
};

struct EngineBase {
  virtual ~EngineBase() {}
  virtual int kb() const = 0;
  virtual uint32_t bits() const = 0;
  virtual uint32_t slots() const = 0;
  virtual bool fused() const = 0;
  virtual bool xgrouped() const = 0;
  virtual bool copyback() const = 0;
  virtual bool hashjoin() const = 0;
  virtual uint32_t count_tile() const = 0;
  virtual uint32_t fuse_tile() const = 0;
  virtual uint32_t emit_tile() const = 0;
  virtual uint32_t sort_mode() const = 0;
  virtual uint32_t side_mode() const = 0;
  virtual size_t held() const = 0;       // device bytes of the engine's buffers
  virtual size_t grow_peak() const = 0;  // held() at the peak of the growth the last run asked for
  virtual void release() = 0;
};

// The tile shapes a new engine of key type K takes from the context.
template <typename K> static uint32_t count_tile_of(const wg_ctx* c) {
  const uint32_t v = c->tune_count[sizeof(K) == 8];
  return v ? v : (uint32_t)kTileD;
}
template <typename K> static uint32_t fuse_tile_of(const wg_ctx* c) {
  const uint32_t v = c->tune_fuse[sizeof(K) == 8];
  return v ? v : (uint32_t)FuseTile<K>::T;
}
template <typename K> static uint32_t emit_tile_of(const wg_ctx* c) {
  const uint32_t v = c->tune_emit[sizeof(K) == 8];
  return v ? v : (uint32_t)kTileC;
}

struct Query {
  uint64_t id = 0;
  int kind = WG_TC;
  Relation* rel = nullptr;
  uint64_t rel_id = 0;
  wg_opts opts{};
  int state = WG_PENDING, error = WG_OK;
  EngineBase* eng = nullptr;     // single engine owned while the query lives
  std::unique_ptr<EngineBase> own;
  bool batch = false;
  int bclass = -1;
  uint32_t slot = 0;
  // served through a single-query engine (a large request, see solo_round)
  bool solo = false;
  bool solo_wait = false;        // paused after a growth over the budget
  size_t wait_used = 0;          // the context's allocated bytes when it paused
  // results
  uint64_t n_tuples = 0;
  uint32_t iterations = 0, regrows = 0;
  uint64_t candidates = 0, launches = 0;
  double device_ms = 0;
  double t_submit_us = 0, t_done_us = 0;
  std::vector<unsigned long long> log;
  std::vector<KStat> prof;
  // where the result lives (rank-space keys of width kb)
  const void* res_ptr = nullptr;
  DBuf res_own;                  // batch results copied out of the retire pool
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

template <typename K>
struct Engine : EngineBase {
  wg_ctx* c;
  cudaStream_t st = nullptr;  // the engine's stream (the context stream for single queries)
  bool own_st = false;
  bool single, fuse, xseg;
  uint32_t nv_cap = 0;  // vertices the x-grouped sort buffers can hold
  uint32_t n_slots, bits_, passes, dbits;
  Dev* dv = nullptr;   // device block
  Dev h{};             // host mirror (read back after each run)
  std::vector<Inst> hi;
  DBuf b_dev, b_inst, b_seg, b_log;
  DBuf D[2], C[2], F[2], R, pos, st_s, st_k, hist, spl, xlen_b, segx_b, tseg_b, xsum_b, mix_b;
  DBuf G[2];  // side-run pools (single-query fused engines)
  DBuf xord_b;  // x-grouped: claim order of the per-source sort segments
  unsigned long long capC = 0, capF = 0, capR = 0, capG = 0;
  size_t mix_tiles = 0;  // tiles the per-tile arrays (st_s, spl, mix_b) hold
  uint32_t log_cap = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int g_count = 0, g_emit = 0, g_hist = 0, g_pass = 0, g_seg = 0, g_uniq = 0, g_merge = 0, g_fuse = 0;
  bool in_flight = false;
  bool grow_wait = false;  // batch: paused after an overflow until the memory comes back
  size_t wait_used = 0;    // the context's allocated bytes when the pause began
  cudaEvent_t ev_done = nullptr;
  uint64_t launches_issued = 0;
  uint32_t regrows = 0;
  int kernels_per_iter() const {
    return 10 + (fuse ? 3 : 0) + (int)passes + (xseg ? 2 : 0) +
           (xseg && sort_mode_ != WG_SORT_PASSES ? 1 : 0) - (hash_join ? 1 : 0) +
           (side_ ? 6 : 0);
  }

  bool copy_back = false;  // copy Full' back every iteration instead of swapping buffers
  bool hash_join = false;  // join through the relation's hash table (ablation)
  uint32_t count_tile_, fuse_tile_;  // delta tuples per join-count tile, keys per fused tile
  uint32_t emit_tile_;               // merged items per join-emit tile
  uint32_t sort_mode_;               // enum wg_sort_mode (x-grouped engines)
  uint32_t side_;                    // side run of Full: 0 never, 1 with few candidates, 2 always
  Engine(wg_ctx* ctx, bool single_, uint32_t n, uint32_t bits, uint32_t logcap, bool fuse_,
         bool xseg_, bool copy_back_ = false, bool hash_join_ = false, uint32_t side = 0)
      : c(ctx), single(single_), fuse(fuse_), xseg(xseg_), n_slots(n), bits_(bits),
        log_cap(logcap), copy_back(copy_back_), hash_join(hash_join_),
        count_tile_(count_tile_of<K>(ctx)), fuse_tile_(fuse_tile_of<K>(ctx)),
        emit_tile_(emit_tile_of<K>(ctx)), sort_mode_(ctx->tune_sort[sizeof(K) == 8]),
        side_(single_ && fuse_ && n == 1 && !copy_back_ ? side : 0u) {
    pass_plan(bits, &passes, &dbits);
    if (xseg && sort_mode_ == WG_SORT_SEGMENT_WIDE && bits > 8) {  // digits of up to 9 bits
      passes = (bits + 8) / 9;
      dbits = (bits + passes - 1) / passes;
    }
  }
  ~Engine() override { release(); }
  int kb() const override { return (int)sizeof(K); }
  bool fused() const override { return fuse; }
  bool xgrouped() const override { return xseg; }
  bool copyback() const override { return copy_back; }
  bool hashjoin() const override { return hash_join; }
  uint32_t count_tile() const override { return count_tile_; }
  uint32_t emit_tile() const override { return emit_tile_; }
  uint32_t fuse_tile() const override { return fuse_tile_; }
  uint32_t sort_mode() const override { return sort_mode_; }
  uint32_t side_mode() const override { return side_; }
  uint32_t bits() const override { return bits_; }
  uint32_t slots() const override { return n_slots; }

  void release() override {
    if (st) cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr; graph = nullptr;
    if (ev_done) cudaEventDestroy(ev_done);
    ev_done = nullptr;
    DBuf* all[] = {&b_dev, &b_inst, &b_seg, &b_log, &D[0], &D[1], &C[0], &C[1], &F[0], &F[1],
                   &R, &pos, &st_s, &st_k, &hist, &spl, &xlen_b, &segx_b, &tseg_b, &xsum_b,
                   &mix_b, &G[0], &G[1], &xord_b};
    for (DBuf* b : all) b->release(c);
    capC = capF = capR = capG = 0;
    mix_tiles = 0;
    nv_cap = 0;
    if (own_st && st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
      st = nullptr;
      own_st = false;
    }
  }

  int init(cudaStream_t stream = nullptr) {
    if (!st) {
      if (single) {
        st = c->stream;
      } else if (stream) {  // batch engines run on their class's stream, concurrently
        st = stream;
      } else {
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own_st = true;
      }
    }
    AllocScope scope(c, st);
    TRY(b_dev.get(c, sizeof(Dev)));
    TRY(b_inst.get(c, sizeof(Inst) * n_slots));
    TRY(b_seg.get(c, sizeof(Seg) * n_slots * 7));
    TRY(b_log.get(c, sizeof(unsigned long long) * (size_t)n_slots * log_cap));
    TRY(hist.get(c, sizeof(unsigned long long) * (size_t)n_slots * passes * kRadix));
    dv = (Dev*)b_dev.p;
    hi.assign(n_slots, Inst{});
    CK(cudaMemsetAsync(b_inst.p, 0, sizeof(Inst) * n_slots, st));
    std::memset(&h, 0, sizeof(h));
    h.inst = (Inst*)b_inst.p;
    Seg* s = (Seg*)b_seg.p;
    h.segD = s; h.segE = s + n_slots; h.segS = s + 2 * n_slots; h.segU = s + 3 * n_slots;
    h.segM = s + 4 * n_slots; h.segF = s + 5 * n_slots; h.segF2 = s + 6 * n_slots;
    h.side = side_;
    h.fuse = fuse ? 1 : 0; h.fuse_tile = fuse_tile_; h.xseg = xseg ? 1 : 0;
    h.copyback = copy_back && single && fuse ? 1 : 0;
    h.count_tile = count_tile_;
    h.emit_tile = emit_tile_;
    // (the per-segment sort counts up to three passes' digits: fields of <= 24 bits)
    h.seg_sort = xseg && sort_mode_ != WG_SORT_PASSES && passes <= 3 ? 1 : 0;
    h.seg_wide = h.seg_sort && sort_mode_ == WG_SORT_SEGMENT_WIDE ? 1 : 0;
    h.hist = (unsigned long long*)hist.p;
    h.n_inst = n_slots; h.single = single ? 1 : 0;
    h.bits = bits_; h.passes = passes; h.dbits = dbits;
    h.ctl.iter_budget = 0xFFFFFFFFu;
    // Every stage kernel first reads its record's control block: a run whose
    // first plan kernel stops on an overflow launches the later stages with
    // records no plan kernel has written yet -- no tiles, but a valid block.
    for (int i = 0; i < S_NUM; ++i) h.st[i].ctl = (Ctl*)((char*)dv + offsetof(Dev, ctl));
    CK(cudaMemcpyAsync(dv, &h, sizeof(Dev), cudaMemcpyHostToDevice, st));
    CK(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
    g_count = grid_of(c, occupancy_join<K>(count_tile_ == (uint32_t)kTileD ? 0 : 3));
    g_emit = grid_of(c, occupancy_join<K>(emit_tile_ == (uint32_t)kTileC ? 1 : 4));
    g_hist = grid_of(c, occupancy_sort<K>(0));
    g_pass = grid_of(c, occupancy_sort<K>(1));
    g_seg = grid_of(c, occupancy_sort<K>(sort_mode_ == WG_SORT_SEGMENT8 ? 7
                                         : sort_mode_ == WG_SORT_SEGMENT_WIDE ? 8 : 6));
    g_uniq = grid_of(c, occupancy_sort<K>(2));
    g_merge = grid_of(c, occupancy_sort<K>(3));
    g_fuse = grid_of(c, occupancy_sort<K>(fuse_tile_ == (uint32_t)FuseTile<K>::T ? 4 : 5));
    return WG_OK;
  }

  // write the pool fields (D .. hist) of the device block
  int put_pools() {
    h.D[0] = D[0].p; h.D[1] = D[1].p; h.C[0] = C[0].p; h.C[1] = C[1].p;
    h.F[0] = F[0].p; h.F[1] = F[1].p; h.R = R.p;
    h.capC = capC; h.capF = capF; h.capR = capR;
    h.pos = (unsigned long long*)pos.p;
    h.status_scalar = (unsigned long long*)st_s.p;
    h.status_sort = (unsigned long long*)st_k.p;
    h.splits = (unsigned long long*)spl.p;
    h.csplits = spl.p ? h.splits + mix_tiles + 1 : nullptr;
    h.hist = (unsigned long long*)hist.p;
    h.xlen = (unsigned long long*)xlen_b.p;
    h.segX = (Seg*)segx_b.p;
    h.tile_seg = (uint32_t*)tseg_b.p;
    h.xord = (uint32_t*)xord_b.p;
    h.xsum = (unsigned long long*)xsum_b.p;
    // [mix_tiles] list | [mix_tiles + 1] prefix | [mix_tiles / kThreads + 2] chunk counts
    h.mixl = (uint32_t*)mix_b.p;
    h.mixc = mix_b.p ? h.mixl + mix_tiles : nullptr;
    h.mixs = mix_b.p ? h.mixc + mix_tiles + 1 : nullptr;
    h.G[0] = G[0].p; h.G[1] = G[1].p; h.capG = capG;
    h.mix_cap = mix_tiles;
    const size_t a = offsetof(Dev, D), b = offsetof(Dev, r_used);
    CK(cudaMemcpyAsync((char*)dv + a, (char*)&h + a, b - a, cudaMemcpyHostToDevice, st));
    return WG_OK;
  }

  // (Re)size the pools; live data (the current delta and full relation and the
  // retired results) is copied into the new buffers.  A buffer is released only
  // once its successor is allocated, and the device block is rewritten on
  // every exit: a growth that fails (over the budget, out of memory) leaves
  // the engine whole, at the capacities it reached, never pointing at freed
  // memory.
  int ensure(unsigned long long wantC, unsigned long long wantF, unsigned long long wantR,
             bool keep) {
    AllocScope scope(c, st);
    wantC = std::max<unsigned long long>(wantC, 1ull << 16);
    wantF = std::max<unsigned long long>(wantF, 1ull << 16);
    wantR = single ? 0 : std::max<unsigned long long>(wantR, 1ull << 16);
    uint64_t liveD = 0, liveF = 0, liveG = 0;
    if (keep) {
      for (const Inst& I : hi)
        if (I.state == INST_ACTIVE) {
          liveD = std::max<uint64_t>(liveD, I.d_off + I.n_delta);
          liveF = std::max<uint64_t>(liveF, I.f_off + I.n_full - I.n_side);  // the main run
          liveG = std::max<uint64_t>(liveG, I.n_side);
        }
    }
    bool clear = false;  // lookback words must start over (a status array is new)
    auto finish = [&](int rc) -> int {
      if (clear) {
        if (st_s.p) CK(cudaMemsetAsync(st_s.p, 0, st_s.bytes, st));
        if (st_k.p) CK(cudaMemsetAsync(st_k.p, 0, st_k.bytes, st));
        h.ctl.epoch = 0;
      }
      const int pr = put_pools();
      return rc != WG_OK ? rc : pr;
    };
    {  // per-tile arrays first, for the capacities about to be reached: the
       // scalar lookback words (join-count and fused / dedup tiles), the tile
       // partitions and the fused pass's mixed-tile list, prefix and chunk
       // counts.  Sized by an exact tile count (mix_tiles), never by the
       // rounded-up byte size of one of them: they are carved differently
      const unsigned long long nC = std::max(capC, wantC), nF = std::max(capF, wantF);
      const size_t tiles = std::max<size_t>(nC / count_tile_, nF / fuse_tile_) + n_slots + 2;
      if (tiles > mix_tiles) {
        DBuf ns, np, nm;
        int rc = ns.get(c, tiles * 8);
        if (rc == WG_OK) rc = np.get(c, 2 * (tiles + 1) * 8);  // splits | emit tile starts
        if (rc == WG_OK) rc = nm.get(c, (2 * tiles + 1 + tiles / kThreads + 2) * 4);
        if (rc != WG_OK) {
          ns.release(c); np.release(c); nm.release(c);
          return finish(rc);
        }
        st_s.release(c); spl.release(c); mix_b.release(c);
        st_s = ns; spl = np; mix_b = nm;
        mix_tiles = tiles;
        clear = true;
      }
    }
    if (wantC > capC) {
      DBuf nd[2], nc[2], np, nk, nt;
      auto undo = [&](int rc) {
        for (int i = 0; i < 2; ++i) { nd[i].release(c); nc[i].release(c); }
        np.release(c); nk.release(c); nt.release(c);
        return finish(rc);
      };
      int rc = WG_OK;
      for (int i = 0; i < 2 && rc == WG_OK; ++i) {
        rc = nd[i].get(c, wantC * sizeof(K));
        if (rc == WG_OK) rc = nc[i].get(c, wantC * sizeof(K));
      }
      if (rc == WG_OK) rc = np.get(c, wantC * 8);
      if (rc == WG_OK) rc = nk.get(c, (wantC / kTileC + std::max(n_slots, nv_cap) + 2) * kRadix * 8);
      if (rc == WG_OK && xseg) rc = nt.get(c, (wantC / kTileC + nv_cap + 2) * 4);
      if (rc != WG_OK) return undo(rc);
      if (liveD)
        CK(cudaMemcpyAsync(nd[h.dphase].p, D[h.dphase].p, liveD * sizeof(K),
                           cudaMemcpyDeviceToDevice, st));
      for (int i = 0; i < 2; ++i) {
        D[i].release(c); C[i].release(c);
        D[i] = nd[i]; C[i] = nc[i];
      }
      pos.release(c); st_k.release(c);
      pos = np; st_k = nk;
      if (xseg) { tseg_b.release(c); tseg_b = nt; }
      capC = wantC;
      clear = true;
    }
    if (wantF > capF) {
      DBuf nf[2];
      int rc = nf[0].get(c, wantF * sizeof(K));
      if (rc == WG_OK) rc = nf[1].get(c, wantF * sizeof(K));
      if (rc != WG_OK) { nf[0].release(c); nf[1].release(c); return finish(rc); }
      if (liveF)
        CK(cudaMemcpyAsync(nf[h.fphase].p, F[h.fphase].p, liveF * sizeof(K),
                           cudaMemcpyDeviceToDevice, st));
      for (int i = 0; i < 2; ++i) { F[i].release(c); F[i] = nf[i]; }
      capF = wantF;
    }
    if (side_) {  // side-run pools: an eighth of the Full pools
      const unsigned long long wantG = std::max<unsigned long long>(capF / 8, 1ull << 16);
      if (wantG > capG) {
        // optional: without room the iterations keep merging into the main run
        DBuf ng[2];
        int rc = ng[0].get(c, wantG * sizeof(K));
        if (rc == WG_OK) rc = ng[1].get(c, wantG * sizeof(K));
        if (rc != WG_OK) {
          ng[0].release(c); ng[1].release(c);
          cudaGetLastError();
        } else {
          const uint32_t gp = hi.empty() ? 0u : hi[0].gphase & 1u;
          if (liveG)
            CK(cudaMemcpyAsync(ng[gp].p, G[gp].p, liveG * sizeof(K), cudaMemcpyDeviceToDevice, st));
          for (int i = 0; i < 2; ++i) { G[i].release(c); G[i] = ng[i]; }
          capG = wantG;
        }
      }
    }
    if (!single && wantR > capR) {
      DBuf nr;
      const int rc = nr.get(c, wantR * sizeof(K));
      if (rc != WG_OK) return finish(rc);
      if (keep && h.r_used)
        CK(cudaMemcpyAsync(nr.p, R.p, h.r_used * sizeof(K), cudaMemcpyDeviceToDevice, st));
      R.release(c);
      R = nr;
      capR = wantR;
    }
    return finish(WG_OK);
  }

  // The kernels of one semi-naive iteration (Secs. Per-Iteration Pipeline and
  // Fused Deduplication): join count -> plan -> join emit -> radix histogram ->
  // radix passes -> fused dedup + set difference -> plan (termination) -> merge.
  // staged: after every stage the host reads the control block back and
  // waits for it (the per-stage readback of the host-driven pipelines of Sec.
  // Motivation, "Stage-Wise Synchronization"); an overflow seen there stops
  // the iteration's remaining launches.  Returns the host syncs issued.
  uint32_t launch_iteration(cudaStream_t s, std::vector<KStat>* prof = nullptr,
                            std::vector<cudaEvent_t>* evs = nullptr, bool staged = false) {
    auto mark = [&]() {
      if (evs) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        evs->push_back(e);
      }
    };
    (void)prof;
    uint32_t syncs = 0;
    bool stop = false;
    auto stage = [&]() {  // one stage's readback; true = the iteration goes on
      if (!staged || stop) return !stop;
      Ctl back{};
      cudaMemcpyAsync(&back, &dv->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      ++syncs;
      stop = back.abort != 0;
      return !stop;
    };
    launch_plan_delta(dv, s);
    if (!stage()) return syncs;
    mark(); launch_join_count<K>(dv->st + S_COUNT, g_count, s, count_tile_); mark();
    if (!stage()) return syncs;
    launch_plan_cand(dv, s);
    if (!stage()) return syncs;
    if (xseg) {
      launch_xseg_build(dv, s);
      if (!stage()) return syncs;
    }
    if (hash_join) {
      mark(); launch_join_emit_hash<K>(dv->st + S_EMIT, g_emit, s); mark();
    } else {
      launch_partition<K>(dv->st + S_EMIT, 2, emit_tile_, c->num_sms * 4, s);
      if (!stage()) return syncs;
      mark(); launch_join_emit<K>(dv->st + S_EMIT, g_emit, s, emit_tile_); mark();
    }
    if (!stage()) return syncs;
    mark(); launch_sort_hist<K>(dv->st + S_HIST, g_hist, s); mark();
    if (!stage()) return syncs;
    if (xseg) {
      // per-source segments: one CTA per segment through every pass when no
      // segment is longer than kSegSortMaxTiles tiles, else the lookback
      // passes (each kernel finds out on the device and the other returns)
      mark();
      if (sort_mode_ != WG_SORT_PASSES)
        launch_sort_seg<K>(dv->st + S_PASS0, g_seg, s, dbits, sort_mode_ == WG_SORT_SEGMENT8 ? 8 : 16,
                           sort_mode_ == WG_SORT_SEGMENT_WIDE);
      for (uint32_t p = 0; p < passes; ++p) launch_sort_pass<K>(dv->st + S_PASS0 + p, g_pass, s, dbits);
      mark();
      if (!stage()) return syncs;
    } else {
      for (uint32_t p = 0; p < passes; ++p) {
        mark(); launch_sort_pass<K>(dv->st + S_PASS0 + p, g_pass, s, dbits); mark();
        if (!stage()) return syncs;
      }
    }
    if (fuse) {
      // timed together as the fused stage: folding the side run back into
      // the main run (when the plan asked for it), the merge-path partition,
      // mixed tiles through the fused kernel, Full-only tiles by a plain
      // copy, and in a side iteration the side run's pass
      mark();
      if (side_) {
        launch_partition<K>(dv->st + S_PREM, 0, kTileM, c->num_sms * 4, s);
        launch_merge<K>(dv->st + S_PREM, g_merge, s);
        if (!stage()) return syncs;
      }
      launch_partition<K>(dv->st + S_FUSE, 0, fuse_tile_, c->num_sms * 4, s);
      if (!stage()) return syncs;
      launch_fuse_mark(dv, c->num_sms * 2, s);
      launch_fuse_list(dv, c->num_sms * 2, s);
      launch_diff_merge<K>(dv->st + S_FUSE, g_fuse, s, fuse_tile_);
      launch_fuse_copy<K>(dv->st + S_FUSE, c->num_sms * 8, s, fuse_tile_);
      if (side_) {
        if (!stage()) return syncs;
        launch_plan_side(dv, s);
        if (!stage()) return syncs;
        launch_partition<K>(dv->st + S_FUSE2, 0, fuse_tile_, c->num_sms * 4, s);
        if (!stage()) return syncs;
        launch_diff_merge<K>(dv->st + S_FUSE2, g_fuse, s, fuse_tile_);
      }
      mark();
      if (!stage()) return syncs;
      launch_plan_post(dv, s);
      if (!stage()) return syncs;
      // retire copy, or with a side run the final merge of both runs
      mark();
      if (side_) launch_partition<K>(dv->st + S_MERGE, 0, kTileM, c->num_sms * 4, s);
      launch_merge<K>(dv->st + S_MERGE, g_merge, s);
      mark();
    } else {
      mark(); launch_unique_diff<K>(dv->st + S_UNIQ, g_uniq, s); mark();
      if (!stage()) return syncs;
      launch_plan_merge(dv, s);
      if (!stage()) return syncs;
      launch_partition<K>(dv->st + S_MERGE, 0, kTileM, c->num_sms * 4, s);
      if (!stage()) return syncs;
      mark(); launch_merge<K>(dv->st + S_MERGE, g_merge, s); mark();
    }
    return syncs;
  }

  int capture() {
    if (exec) return WG_OK;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_iteration(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &body);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return set_err(WG_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&exec, graph, 0));
    h.cond = (unsigned long long)cond;
    CK(cudaMemcpyAsync(&dv->cond, &h.cond, sizeof(h.cond), cudaMemcpyHostToDevice, st));
    return WG_OK;
  }

  int put_ctl(uint32_t budget, bool use_cond) {
    h.ctl.abort = 0; h.ctl.error = 0; h.ctl.cont = 1; h.ctl.launch_iters = 0;
    h.ctl.iter_budget = budget;
    h.ctl.need_cand = h.ctl.need_full = h.ctl.need_res = 0;
    if (h.ctl.epoch > (1u << 22)) {  // clear lookback words before the epoch wraps
      CK(cudaMemsetAsync(st_s.p, 0, st_s.bytes, st));
      CK(cudaMemsetAsync(st_k.p, 0, st_k.bytes, st));
      h.ctl.epoch = 0;
    }
    CK(cudaMemcpyAsync(&dv->ctl, &h.ctl, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    h.use_cond = use_cond ? 1 : 0;
    CK(cudaMemcpyAsync(&dv->use_cond, &h.use_cond, 4, cudaMemcpyHostToDevice, st));
    return WG_OK;
  }

  int read_back() {
    CK(cudaMemcpyAsync(&h.ctl, &dv->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h.r_used, &dv->r_used, sizeof(h.r_used), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h.dphase, &dv->dphase, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hi.data(), b_inst.p, sizeof(Inst) * n_slots, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return WG_OK;
  }

  // Radix passes of the next launch.  A batch engine's passes cover its key
  // class; its instances' keys use 2w bits (w of the widest active one), so
  // the passes above them are skipped (their kernels find no tiles).
  int put_passes() {
    uint32_t need = 0;
    if (!single) {
      for (const Inst& I : hi)
        if (I.state == INST_ACTIVE) need = std::max(need, 2 * I.w);
    }
    const uint32_t np = single || need == 0 ? passes
                                            : std::min(passes, std::max(1u, (need + dbits - 1) / dbits));
    if (np != h.passes) {
      h.passes = np;
      CK(cudaMemcpyAsync(&dv->passes, &h.passes, sizeof(h.passes), cudaMemcpyHostToDevice, st));
    }
    return WG_OK;
  }

  // Launch the loop: the graph (WG_LOOP_DEVICE), one host round trip per
  // iteration (WG_LOOP_HOST) or one per stage (WG_LOOP_HOST_STAGED).
  uint64_t host_syncs = 0;
  int launch(uint32_t budget, int mode) {
    TRY(put_passes());
    if (mode != WG_LOOP_DEVICE) {
      TRY(put_ctl(budget, false));
      for (;;) {
        host_syncs += launch_iteration(st, nullptr, nullptr, mode == WG_LOOP_HOST_STAGED);
        launches_issued += kernels_per_iter();
        uint32_t flags[2] = {0, 0};  // cont, abort
        CK(cudaMemcpyAsync(&flags[0], &dv->ctl.cont, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&flags[1], &dv->ctl.abort, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));  // the per-iteration host sync
        ++host_syncs;
        // an overflow stops the loop (a staged iteration stops before the
        // plan kernel that would clear the continue flag)
        if (!flags[0] || flags[1]) break;
      }
      CK(cudaGetLastError());
    } else {
      TRY(capture());
      TRY(put_ctl(budget, true));
      CK(cudaGraphLaunch(exec, st));
    }
    CK(cudaEventRecord(ev_done, st));
    in_flight = true;
    return WG_OK;
  }

  // After a launch completed: read the state back; grow and report when a
  // pool overflowed.  *again = the same loop must be launched once more.
  int settle(bool* again) {
    *again = false;
    in_flight = false;
    TRY(read_back());
    // kernels actually issued inside the graph: launch_iters iterations
    if (exec && h.use_cond)  // body executions: committed iterations, plus one if it aborted
      launches_issued += (uint64_t)(h.ctl.launch_iters + (h.ctl.abort ? 1u : 0u)) * kernels_per_iter();
    if (h.ctl.error) return set_err(WG_E_DEVICE_TIMEOUT, "a bounded device wait gave up");
    if (h.ctl.abort) {
      ++regrows;
      *again = true;
      return grow();
    }
    *again = h.ctl.n_active > 0;
    return WG_OK;
  }

  // Hash-join ablation: the table the join stages read.
  int put_htab(const void* tab, unsigned long long mask) {
    h.htab = (const unsigned long long*)tab;
    h.hmask = mask;
    CK(cudaMemcpyAsync((char*)dv + offsetof(Dev, htab), (char*)&h + offsetof(Dev, htab),
                       offsetof(Dev, hmask) + sizeof(h.hmask) - offsetof(Dev, htab),
                       cudaMemcpyHostToDevice, st));
    return WG_OK;
  }

  // Buffers of the x-grouped sort for relations of up to nv vertices (all
  // allocated before any is replaced, as in ensure()).
  int ensure_nv(uint32_t nv) {
    if (!xseg || nv <= nv_cap) return WG_OK;
    AllocScope scope(c, st);
    DBuf nx, ns, nh, nk, nt, nz, no;
    int rc = nx.get(c, (size_t)nv * 8);
    if (rc == WG_OK) rc = ns.get(c, (size_t)nv * sizeof(Seg));
    if (rc == WG_OK) rc = nh.get(c, (size_t)std::max(n_slots, nv) * passes * kRadix * 8);
    if (rc == WG_OK) rc = nk.get(c, (capC / kTileC + std::max(n_slots, nv) + 2) * kRadix * 8);
    if (rc == WG_OK) rc = nt.get(c, (capC / kTileC + nv + 2) * 4);
    if (rc == WG_OK && !xsum_b.p) rc = nz.get(c, (size_t)kXChunks * 2 * 8);
    if (rc == WG_OK) rc = no.get(c, (size_t)nv * 4);
    if (rc != WG_OK) {
      DBuf* tmp[] = {&nx, &ns, &nh, &nk, &nt, &nz, &no};
      for (DBuf* b : tmp) b->release(c);
      return rc;  // nothing was replaced: the device block is still current
    }
    xlen_b.release(c); segx_b.release(c); hist.release(c); st_k.release(c); tseg_b.release(c);
    xord_b.release(c);
    xlen_b = nx; segx_b = ns; hist = nh; st_k = nk; tseg_b = nt; xord_b = no;
    if (nz.p) xsum_b = nz;
    CK(cudaMemsetAsync(st_k.p, 0, st_k.bytes, st));
    h.ctl.epoch = 0;
    if (st_s.p) CK(cudaMemsetAsync(st_s.p, 0, st_s.bytes, st));
    nv_cap = nv;
    return put_pools();
  }

  // Grow the pools to what the aborted run asked for (plus headroom).
  void grow_target(unsigned long long* wc, unsigned long long* wf, unsigned long long* wr) const {
    const unsigned long long nc = h.ctl.need_cand ? h.ctl.need_cand + h.ctl.need_cand / 4 + 4096 : 0;
    const unsigned long long nf = h.ctl.need_full ? h.ctl.need_full + h.ctl.need_full / 4 + 4096 : 0;
    const unsigned long long nr = h.ctl.need_res ? h.ctl.need_res + h.ctl.need_res / 2 + 4096 : 0;
    *wc = std::max(capC, nc); *wf = std::max(capF, nf); *wr = std::max(capR, nr);
  }
  int grow() {
    unsigned long long wc, wf, wr;
    grow_target(&wc, &wf, &wr);
    return ensure(wc, wf, wr, true);
  }
  size_t held() const override {
    const DBuf* all[] = {&b_dev, &b_inst, &b_seg, &b_log, &D[0], &D[1], &C[0], &C[1], &F[0], &F[1],
                         &R, &pos, &st_s, &st_k, &hist, &spl, &xlen_b, &segx_b, &tseg_b,
                         &xsum_b, &mix_b, &G[0], &G[1], &xord_b};
    size_t b = 0;
    for (const DBuf* x : all) b += x->bytes;
    return b;
  }
  // The bytes grow() would make the engine hold at its peak: ensure()
  // allocates each group of buffers before it releases the group it replaces
  // (the optional side-run pools are left out).
  size_t grow_peak() const override {
    unsigned long long wantC, wantF, wantR;
    grow_target(&wantC, &wantF, &wantR);
    wantC = std::max<unsigned long long>(wantC, 1ull << 16);
    wantF = std::max<unsigned long long>(wantF, 1ull << 16);
    wantR = single ? 0 : std::max<unsigned long long>(wantR, 1ull << 16);
    size_t cur = held(), peak = cur;
    auto step = [&](size_t add, size_t drop) {
      peak = std::max(peak, cur + add);
      cur = cur + add - drop;
    };
    const unsigned long long nC = std::max(capC, wantC), nF = std::max(capF, wantF);
    const size_t tiles = std::max<size_t>(nC / count_tile_, nF / fuse_tile_) + n_slots + 2;
    if (tiles > mix_tiles)
      step(round_up(tiles * 8) + round_up(2 * (tiles + 1) * 8) +
               round_up((2 * tiles + 1 + tiles / kThreads + 2) * 4),
           st_s.bytes + spl.bytes + mix_b.bytes);
    if (wantC > capC)
      step(4 * round_up(wantC * sizeof(K)) + round_up(wantC * 8) +
               round_up((wantC / kTileC + std::max(n_slots, nv_cap) + 2) * kRadix * 8) +
               (xseg ? round_up((wantC / kTileC + nv_cap + 2) * 4) : 0),
           D[0].bytes + D[1].bytes + C[0].bytes + C[1].bytes + pos.bytes + st_k.bytes +
               (xseg ? tseg_b.bytes : 0));
    if (wantF > capF) step(2 * round_up(wantF * sizeof(K)), F[0].bytes + F[1].bytes);
    if (!single && wantR > capR) step(round_up(wantR * sizeof(K)), R.bytes);
    return peak;
  }
  // Take instance `slot` out of the running set (its state is dropped).
  int evict(uint32_t slot) {
    Inst I = hi[slot];
    I.state = INST_FREE;
    I.n_delta = 0; I.n_full = 0;
    hi[slot] = I;
    CK(cudaMemcpyAsync((Inst*)b_inst.p + slot, &I, sizeof(Inst), cudaMemcpyHostToDevice, st));
    return WG_OK;
  }

  // Fresh instance in `slot` over relation R.
  int admit(uint32_t slot, Relation* Rl, int kind, uint32_t max_iters, unsigned long long d_off) {
    Inst I{};
    I.off = (const uint32_t*)Rl->off.p;
    I.adj = (const uint32_t*)Rl->adj.p;
    I.nv = Rl->nv; I.w = Rl->w;
    I.kind = kind == WG_SG ? KIND_SG : KIND_TC;
    I.state = INST_ACTIVE;
    I.iter = 0;
    I.max_iters = max_iters;
    I.n_delta = Rl->nv;
    I.d_off = d_off;
    I.log = (unsigned long long*)b_log.p + (size_t)slot * log_cap;
    I.log_cap = log_cap;
    I.fresh = 1;
    hi[slot] = I;
    CK(cudaMemcpyAsync((Inst*)b_inst.p + slot, &I, sizeof(Inst), cudaMemcpyHostToDevice, st));
    return WG_OK;
  }
  int init_deltas(uint32_t first, uint32_t count) {
    launch_init_diag<K>((Inst*)b_inst.p, first, count, D[h.dphase].p, st);
    CK(cudaGetLastError());
    return WG_OK;
  }
  int reset_single() {
    h.dphase = 0; h.fphase = 0; h.r_used = 0;
    CK(cudaMemcpyAsync(&dv->r_used, &h.r_used, sizeof(h.r_used), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(&dv->dphase, &h.dphase, 8, cudaMemcpyHostToDevice, st));
    return WG_OK;
  }
  const void* pool_ptr(uint32_t pool) const {
    return pool == 2 ? R.p : F[pool & 1].p;
  }
};

// Free the pools of idle single-query engines, least recently used first,
// until `bytes` more fit in the budget (a cached engine only saves the next
// query of its kind a pool allocation and a graph capture).
static void drop_idle_engines(wg_ctx* c, size_t bytes) {
  while (!c->idle.empty() && c->used + bytes > c->budget) c->idle.erase(c->idle.begin());
}

static EngineBase* new_engine(wg_ctx* c, int kb, bool single, uint32_t slots, uint32_t bits,
                              uint32_t logcap, bool fuse, bool xseg, int* rc,
                              bool copyback = false, bool hashjoin = false, uint32_t side = 0,
                              cudaStream_t stream = nullptr) {
  EngineBase* e;
  if (kb == 4) {
    auto* x = new Engine<uint32_t>(c, single, slots, bits, logcap, fuse, xseg, copyback, hashjoin,
                                   side);
    *rc = x->init(stream);
    e = x;
  } else {
    auto* x = new Engine<unsigned long long>(c, single, slots, bits, logcap, fuse, xseg, copyback,
                                             hashjoin, side);
    *rc = x->init(stream);
    e = x;
  }
  if (*rc != WG_OK) { delete e; return nullptr; }
  return e;
}

// ------------------------------------------------------------------ single queries
// The loop a single query runs: a profiled run is host-driven (one event
// pair per kernel), otherwise the requested one.
static int loop_mode(const Query* q) {
  return q->opts.profile && q->opts.loop == WG_LOOP_DEVICE ? (int)WG_LOOP_HOST : (int)q->opts.loop;
}

template <typename K>
static int single_start(wg_ctx* c, Query* q) {
  auto* E = static_cast<Engine<K>*>(q->eng);
  Relation* Rl = q->rel;
  const unsigned long long wantC = std::max<unsigned long long>(
      {q->opts.reserve_cand, Rl->peak_cand, 8ull * Rl->ne + Rl->nv, 1ull << 16});
  const unsigned long long wantF = std::max<unsigned long long>(
      {q->opts.reserve_full, Rl->peak_full, 4ull * Rl->ne, 1ull << 16});
  TRY(E->reset_single());
  TRY(E->ensure_nv(Rl->nv));
  TRY(E->ensure(wantC, wantF, 0, false));
  TRY(E->admit(0, Rl, q->kind, q->opts.max_iters, 0));
  TRY(E->init_deltas(0, 1));
  CK(cudaEventRecord(q->ev0, c->stream));
  if (q->opts.profile) {
    // profiled run: host loop with CUDA events around every stage kernel
    for (;;) {
      TRY(E->put_ctl(0xFFFFFFFFu, false));
      for (;;) {
        Inst before{};
        CK(cudaMemcpyAsync(&before, E->b_inst.p, sizeof(Inst), cudaMemcpyDeviceToHost, c->stream));
        std::vector<cudaEvent_t> evs;
        E->launch_iteration(c->stream, nullptr, &evs);
        E->launches_issued += E->kernels_per_iter();
        Inst after{};
        uint32_t cont = 0, abort = 0;
        CK(cudaMemcpyAsync(&after, E->b_inst.p, sizeof(Inst), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&cont, &E->dv->ctl.cont, 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&abort, &E->dv->ctl.abort, 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (!abort) {
          const double kb = sizeof(K);
          const double nd = (double)before.n_delta, nc = (double)after.n_cand,
                       nn = (double)after.n_new, nf = (double)before.n_full;
          // algorithmic bytes of each kernel (see the kernel headers)
          // the per-segment sort reads its keys once more to count their
          // digits (the histogram kernel then returns at once)
          uint32_t maxt = 0;
          if (E->xgrouped() && E->h.seg_sort)
            CK(cudaMemcpy(&maxt, &E->dv->xseg_maxt, 4, cudaMemcpyDeviceToHost));
          const bool seg = E->xgrouped() && E->h.seg_sort && (E->h.seg_wide || maxt <= kSegSortMaxTiles);
          std::vector<std::pair<const char*, double>> names = {
              {"join_count", nd * (kb + 8 + 8)},
              {"join_emit", nd * (kb + 8) + nc * (kb + 4)},
              {"sort_hist", seg ? 0.0 : nc * kb}};
          if (E->xgrouped())  // every pass in one timed region (k_sort_seg or the passes)
            names.push_back({"sort_pass", (E->passes * 2 + (seg ? 1 : 0)) * nc * kb});
          else
            for (uint32_t p = 0; p < E->passes; ++p) names.push_back({"sort_pass", 2 * nc * kb});
          if (E->fuse) {
            const double ns = (double)before.n_side, n0 = (double)after.n_new0;
            const bool side = after.side_iter != 0;
            const bool prem = !side && before.n_side > 0;
            const bool fmerge = side && after.state != INST_ACTIVE && ns + nn > 0;
            // side iteration: C and the main run read, the new candidates
            // written, then the side run's pass (side run and those read, the
            // new delta and the merged side run written); a pre-merge reads
            // both runs and writes them merged
            const double fused = side ? nc + (nf - ns) + 2 * n0 + 2 * ns + 2 * nn
                                      : nc + 2 * nf + 2 * nn + (prem ? 2 * nf : 0.0);
            names.push_back({"dedup_diff_merge", fused * kb});
            names.push_back({"retire_copy", E->copyback() || fmerge ? 2 * (nf + nn) * kb : 0.0});
          } else {
            names.push_back({"dedup_diff", (nc + nn) * kb});
            names.push_back({"merge", 2 * (nf + nn) * kb});
          }
          for (size_t i = 0; i < names.size(); ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]);
            KStat* st = nullptr;
            for (auto& s : q->prof)
              if (!std::strcmp(s.name, names[i].first)) st = &s;
            if (!st) { q->prof.push_back(KStat{names[i].first}); st = &q->prof.back(); }
            st->launches += 1; st->ms += ms; st->bytes += names[i].second;
          }
        }
        for (auto e : evs) cudaEventDestroy(e);
        if (!cont) break;
      }
      bool again = false;
      E->in_flight = true;
      TRY(E->settle(&again));
      if (!again) break;
    }
    CK(cudaEventRecord(q->ev1, c->stream));
    CK(cudaEventRecord(E->ev_done, c->stream));
    E->in_flight = true;
    q->state = WG_RUNNING;
    return WG_OK;
  }
  TRY(E->launch(0xFFFFFFFFu, loop_mode(q)));
  q->state = WG_RUNNING;
  return WG_OK;
}

template <typename K>
static int single_progress(wg_ctx* c, Query* q, bool block, bool pause_on_budget = false) {
  auto* E = static_cast<Engine<K>*>(q->eng);
  for (;;) {
    if (E->in_flight) {
      if (block) {
        CK(cudaEventSynchronize(E->ev_done));
      } else {
        cudaError_t e = cudaEventQuery(E->ev_done);
        if (e == cudaErrorNotReady) return WG_OK;
        if (e != cudaSuccess) return set_err(WG_E_CUDA, cudaGetErrorString(e));
      }
    }
    bool again = false;
    int rc = E->settle(&again);
    if (rc != WG_OK && pause_on_budget && (rc == WG_E_BUDGET || rc == WG_E_NOMEM)) {
      cudaGetLastError();  // the pools stay whole at their old capacities
      q->solo_wait = true;
      q->wait_used = c->used;
      return WG_OK;
    }
    if (rc != WG_OK) {
      q->state = WG_FAILED;
      q->error = rc;
      return rc;
    }
    if (again) {
      TRY(E->launch(0xFFFFFFFFu, loop_mode(q)));
      continue;
    }
    const Inst& I = E->hi[0];
    if (!q->opts.profile) CK(cudaEventRecord(q->ev1, c->stream));
    CK(cudaEventSynchronize(q->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, q->ev0, q->ev1);
    q->device_ms = ms;
    q->n_tuples = I.n_full;
    q->iterations = I.iters_done;
    q->candidates = I.cand_total;
    q->regrows = E->regrows;
    q->launches = E->launches_issued;
    q->res_ptr = (const K*)E->pool_ptr(I.res_pool) + I.res_off;
    const uint32_t nlog = std::min<uint32_t>(I.iters_done + 1, E->log_cap);
    q->log.assign(nlog, 0);
    CK(cudaMemcpy(q->log.data(), I.log, nlog * 8, cudaMemcpyDeviceToHost));
    q->rel->peak_cand = std::max<uint64_t>(q->rel->peak_cand, E->capC);
    q->rel->peak_full = std::max<uint64_t>(q->rel->peak_full, E->capF);
    if (I.state == INST_ITERCAP) {
      q->state = WG_FAILED;
      q->error = WG_E_ITER_CAP;
    } else {
      q->state = WG_DONE;
    }
    q->t_done_us = now_us();
    return WG_OK;
  }
}

// ------------------------------------------------------------------ batches
// Key classes of batch engines: 32-bit keys (fields <= 16 bits), 64-bit keys
// with fields <= 24 bits, 64-bit keys with fields <= 32 bits.
// Queries are also split by size: small ones (<= kSmallVertices vertices) and
// large ones run in different engines on different streams, so the short
// iterations of small queries never wait for the long ones of large queries.
constexpr uint32_t kSmallVertices = 4096;
static int batch_class(const Relation* R) {
  const int key = R->kb == 4 ? 0 : (R->w <= 24 ? 1 : 2);
  return key * 2 + (R->nv > kSmallVertices ? 1 : 0);
}
static uint32_t class_bits(int cls) { return cls / 2 == 0 ? 32 : (cls / 2 == 1 ? 48 : 64); }
constexpr uint32_t kBatchSlots = 1024;    // queries running at once per key class
// Served requests over more edges than this run one at a time on a
// single-query engine (per-source sort, exact pass plan) beside the batch
// engines: one such fixpoint already fills the GPU.
constexpr uint64_t kSoloEdges = 1u << 16;
constexpr uint32_t kBatchLogCap = 1024;   // per-iteration delta sizes kept per query

struct BatchInfo {
  std::vector<uint64_t> slot_q;    // query id per slot (0 = free)
  std::vector<double> est;         // admission estimate of the slot's final size
  std::vector<uint64_t> seq;       // admission order of the slot's instance
  uint64_t next_seq = 1;
  bool hold = false;               // no admissions after a preemption until one retires
};
static std::map<wg_ctx*, std::map<int, BatchInfo>> g_binfo;

// Whether batch engine `cls` holds work: a launch in flight, an admitted
// instance or a result not yet retired (queued requests do not count: the
// engine is built again for them when it was dropped).
template <typename K>
static bool batch_holds_work(wg_ctx* c, int cls) {
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  if (E->in_flight) return true;
  for (const Inst& I : E->hi)
    if (I.state == INST_ACTIVE) return true;
  for (uint64_t q : g_binfo[c][cls].slot_q)
    if (q) return true;
  return false;
}
static bool batch_holds_work_any(wg_ctx* c, int cls) {
  if (!c->batch[cls]) return false;
  return c->batch[cls]->kb() == 4 ? batch_holds_work<uint32_t>(c, cls)
                                  : batch_holds_work<unsigned long long>(c, cls);
}

// Release the pools of the other batch engines that hold no work; true when
// any was released.
static bool drop_idle_batch(wg_ctx* c, int keep) {
  bool dropped = false;
  for (auto& kv : c->batch) {
    if (kv.first == keep || !kv.second || batch_holds_work_any(c, kv.first)) continue;
    kv.second.reset();
    g_binfo[c].erase(kv.first);
    dropped = true;
  }
  return dropped;
}

// The exclusive query (see batch_preempt), or NULL; a stale id is cleared.
static Query* excl_query(wg_ctx* c) {
  if (!c->excl) return nullptr;
  auto it = c->queries.find(c->excl);
  if (it == c->queries.end() || it->second->state == WG_DONE || it->second->state == WG_FAILED) {
    c->excl = 0;
    return nullptr;
  }
  return it->second.get();
}

// Whether memory that may come back is held outside batch engine `cls`:
// another batch engine's pools, or the served request running on a
// single-query engine.
static bool solo_running(wg_ctx* c) {
  if (!c->solo_run) return false;
  auto it = c->queries.find(c->solo_run);
  return it != c->queries.end() && it->second->state == WG_RUNNING;
}
static bool held_elsewhere(wg_ctx* c, int cls) {
  for (auto& kv : c->batch)
    if (kv.first != cls && kv.second) return true;
  return solo_running(c);
}

// Whether the growth engine e's last run asked for could fit the budget once
// the other engines' pools are released (the batch engines drained and
// dropped, the idle engines freed, the served request running on a single
// engine finished).  When it could not, waiting for them as the exclusive
// query would only stall every other request before failing.
static bool growth_could_fit(wg_ctx* c, const EngineBase* e) {
  size_t others = 0;
  for (auto& kv : c->batch)
    if (kv.second && kv.second.get() != e) others += kv.second->held();
  for (auto& x : c->idle)
    if (x.get() != e) others += x->held();
  if (c->solo_run) {
    auto it = c->queries.find(c->solo_run);
    if (it != c->queries.end() && it->second->eng && it->second->eng != e)
      others += it->second->eng->held();
  }
  const size_t mine = e->held();
  const size_t fixed = c->used > mine + others ? c->used - mine - others : 0;
  return fixed + e->grow_peak() <= c->budget;
}

// Query q of class cls does not fit in its engine although it runs there
// alone: while other engines hold pools it becomes the exclusive query (if
// there is none yet) and stays queued; with the whole budget it fails, and so
// it does at once when the growth its engine's last run asked for (grown:
// the failure came from that growth) could not fit even the whole budget.
// True when it failed.
static bool alone_too_large(wg_ctx* c, int cls, Query* q, int why, bool grown = false) {
  const bool others =
      held_elsewhere(c, cls) && !(grown && !growth_could_fit(c, c->batch[cls].get()));
  if (c->excl == q->id || !others) {
    if (c->excl == q->id) c->excl = 0;
    q->state = WG_FAILED;
    q->error = why;
    q->t_done_us = now_us();
    c->completed.push_back(q->id);
    return true;
  }
  if (!excl_query(c)) c->excl = q->id;
  return false;
}

// Admission estimate of a query's final relation: at most nv^2 tuples, capped
// so that a single large query is still admitted into an idle engine.
static double admit_estimate(const Relation* R, unsigned long long capF) {
  return std::min((double)R->nv * (double)R->nv, (double)capF / 4.0);
}

template <typename K>
static int batch_admit(wg_ctx* c, int cls) {
  auto& B = g_binfo[c][cls];
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  unsigned long long dend = 0;
  double load = 0;
  uint32_t active = 0;
  for (uint32_t s = 0; s < E->n_slots; ++s)
    if (E->hi[s].state == INST_ACTIVE) {
      dend = std::max<unsigned long long>(dend, E->hi[s].d_off + E->hi[s].n_delta);
      load += B.est[s];
      ++active;
    }
  Query* x = excl_query(c);
  if (x) {  // the exclusive query only, once nothing else runs anywhere
    if (x->solo || x->state != WG_PENDING || x->bclass != cls || active > 0) return WG_OK;
    if (solo_running(c)) return WG_OK;
    for (auto& kv : c->batch)
      if (kv.first != cls && batch_holds_work_any(c, kv.first)) return WG_OK;
    drop_idle_batch(c, cls);
  } else {
    if (B.hold && active > 0) return WG_OK;
  }
  B.hold = false;
  uint32_t first = 0xFFFFFFFFu, last = 0, next_free = 0;
  std::vector<uint64_t> still;
  for (uint64_t qid : c->pending) {
    auto it = c->queries.find(qid);
    if (it == c->queries.end()) continue;
    Query* q = it->second.get();
    if (q->solo || q->bclass != cls || (x && q != x)) { still.push_back(qid); continue; }
    while (next_free < E->n_slots &&
           (B.slot_q[next_free] != 0 || E->hi[next_free].state == INST_ACTIVE))
      ++next_free;
    if (active == 0 && q->rel->nv > E->capC) {
      // an idle engine too small for the base rule of q: grow it first
      const unsigned long long want = 2ull * q->rel->nv + 4096;
      int rc = E->ensure(want, E->capF, E->capR, true);
      if ((rc == WG_E_BUDGET || rc == WG_E_NOMEM) && drop_idle_batch(c, cls)) {
        cudaGetLastError();
        rc = E->ensure(want, E->capF, E->capR, true);
      }
      if (rc == WG_E_BUDGET || rc == WG_E_NOMEM) {
        cudaGetLastError();
        if (!alone_too_large(c, cls, q, rc)) still.push_back(qid);
        continue;
      }
      TRY(rc);
    }
    const double est = admit_estimate(q->rel, E->capF);
    const bool fits = dend + q->rel->nv <= E->capC && (active == 0 || load + est <= (double)E->capF);
    if (next_free >= E->n_slots || !fits) { still.push_back(qid); continue; }
    const uint32_t slot = next_free;
    TRY(E->admit(slot, q->rel, q->kind, q->opts.max_iters, dend));
    dend += q->rel->nv;
    load += est;
    ++active;
    B.slot_q[slot] = qid;
    B.est[slot] = est;
    B.seq[slot] = B.next_seq++;
    q->slot = slot;
    q->state = WG_RUNNING;
    first = std::min(first, slot);
    last = std::max(last, slot);
  }
  c->pending.swap(still);
  if (first != 0xFFFFFFFFu) TRY(E->init_deltas(first, last - first + 1));
  return WG_OK;
}

// The pools cannot grow within the budget: requeue the most recently
// admitted running instance (it restarts later from its base rule), and admit
// nothing new until some instance retires.  Evicting the youngest keeps the
// oldest instance progressing.  A query that runs alone in its engine and
// still does not fit while other engines hold pools becomes the exclusive
// query: requeued, it is admitted once every other engine has drained (no
// admissions anywhere meanwhile) and been dropped, so it runs with the whole
// budget; only then does a query that does not fit fail with WG_E_BUDGET.
template <typename K>
static int batch_preempt(wg_ctx* c, int cls, int why) {
  auto& B = g_binfo[c][cls];
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  uint32_t victim = 0xFFFFFFFFu, active = 0;
  uint64_t young = 0;
  for (uint32_t s = 0; s < E->n_slots; ++s) {
    const Inst& I = E->hi[s];
    if (I.state != INST_ACTIVE) continue;
    ++active;
    if (victim == 0xFFFFFFFFu || B.seq[s] > young) { young = B.seq[s]; victim = s; }
  }
  B.hold = true;
  if (victim == 0xFFFFFFFFu) return set_err(why, "batch pools cannot grow");
  const uint64_t qid = B.slot_q[victim];
  B.slot_q[victim] = 0;
  TRY(E->evict(victim));
  auto it = c->queries.find(qid);
  if (it == c->queries.end()) return WG_OK;
  Query* q = it->second.get();
  if (active == 1 && alone_too_large(c, cls, q, why, true)) return WG_OK;
  q->state = WG_PENDING;
  q->regrows += 1;
  c->pending.insert(c->pending.begin(), qid);
  return WG_OK;
}

template <typename K>
static int batch_retire(wg_ctx* c, int cls) {
  auto& B = g_binfo[c][cls];
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  for (uint32_t s = 0; s < E->n_slots; ++s) {
    if (!B.slot_q[s]) continue;
    const Inst& I = E->hi[s];
    if (I.state != INST_DONE && I.state != INST_ITERCAP) continue;
    auto it = c->queries.find(B.slot_q[s]);
    B.slot_q[s] = 0;
    B.hold = false;  // room was freed: admissions may resume
    Inst done = I;
    TRY(E->evict(s));
    if (it == c->queries.end()) continue;  // freed while running
    Query* q = it->second.get();
    q->n_tuples = done.n_full;
    q->iterations = done.iters_done;
    q->candidates = done.cand_total;
    const uint32_t nlog = std::min<uint32_t>(done.iters_done + 1, E->log_cap);
    q->log.assign(nlog, 0);
    CK(cudaMemcpyAsync(q->log.data(), done.log, nlog * 8, cudaMemcpyDeviceToHost, E->st));
    int rc;
    {
      AllocScope scope(c, E->st);
      rc = q->res_own.get(c, std::max<size_t>(done.n_full, 1) * sizeof(K));
    }
    if (rc != WG_OK) {
      q->state = WG_FAILED;
      q->error = rc;
      q->t_done_us = now_us();
      c->completed.push_back(q->id);
      continue;
    }
    if (done.n_full)
      CK(cudaMemcpyAsync(q->res_own.p, (const K*)E->pool_ptr(done.res_pool) + done.res_off,
                         done.n_full * sizeof(K), cudaMemcpyDeviceToDevice, E->st));
    q->res_ptr = q->res_own.p;
    q->state = done.state == INST_DONE ? WG_DONE : WG_FAILED;
    q->error = done.state == INST_DONE ? WG_OK : WG_E_ITER_CAP;
    q->t_done_us = now_us();
    c->completed.push_back(q->id);
  }
  // every retired result has been copied out: the retire pool starts over
  E->h.r_used = 0;
  CK(cudaMemcpyAsync(&E->dv->r_used, &E->h.r_used, 8, cudaMemcpyHostToDevice, E->st));
  CK(cudaStreamSynchronize(E->st));
  return WG_OK;
}

template <typename K>
static void batch_fail_all(wg_ctx* c, int cls, int rc) {
  auto& B = g_binfo[c][cls];
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  for (uint32_t s = 0; s < E->n_slots; ++s)
    if (B.slot_q[s]) {
      auto it = c->queries.find(B.slot_q[s]);
      if (it != c->queries.end()) {
        it->second->state = WG_FAILED;
        it->second->error = rc;
        c->completed.push_back(it->first);
      }
      B.slot_q[s] = 0;
      E->evict(s);
    }
}

// Grow the pools after an overflow (or retry a paused growth).  Over the
// budget, idle engines' pools are released and the growth tried once more.
// An engine that still cannot grow with one instance left, while other
// engines hold work, pauses with that instance's state as the exclusive
// query: nothing is admitted anywhere, the others drain and are dropped, and
// the loop resumes from the iteration that overflowed.  Otherwise preempt.
template <typename K>
static int batch_grow(wg_ctx* c, int cls) {
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  int rc = E->grow();
  if ((rc == WG_E_BUDGET || rc == WG_E_NOMEM) && drop_idle_batch(c, cls)) {
    cudaGetLastError();
    rc = E->grow();
  }
  if (rc == WG_OK) {
    E->grow_wait = false;
    return WG_OK;
  }
  E->grow_wait = false;
  if (rc != WG_E_BUDGET && rc != WG_E_NOMEM) {
    batch_fail_all<K>(c, cls, rc);
    return rc;
  }
  cudaGetLastError();
  uint32_t active = 0, slot = 0;
  for (uint32_t s = 0; s < E->n_slots; ++s)
    if (E->hi[s].state == INST_ACTIVE) { ++active; slot = s; }
  const bool others = held_elsewhere(c, cls);  // (idle engines were dropped above)
  const uint64_t qid = active == 1 ? g_binfo[c][cls].slot_q[slot] : 0;
  Query* x = excl_query(c);
  // (a growth that could not fit even the whole budget fails in batch_preempt)
  if (qid && others && growth_could_fit(c, E) && c->queries.count(qid) && (!x || x->id == qid)) {
    c->excl = qid;
    E->grow_wait = true;
    E->wait_used = c->used;
    return WG_OK;
  }
  return batch_preempt<K>(c, cls, rc);
}

// One scheduling round: finish the launch in flight (grow or preempt after an
// overflow, retire finished queries), admit queued queries, launch again.
template <typename K>
static int batch_round(wg_ctx* c, int cls, uint32_t iters, bool wait_launch, bool* progressed) {
  auto* E = static_cast<Engine<K>*>(c->batch[cls].get());
  if (E->in_flight) {
    if (!wait_launch) {
      cudaError_t e = cudaEventQuery(E->ev_done);
      if (e == cudaErrorNotReady) return WG_OK;
    }
    *progressed = true;
    CK(cudaEventSynchronize(E->ev_done));
    E->in_flight = false;
    TRY(E->read_back());
    if (E->exec && E->h.use_cond)
      E->launches_issued += (uint64_t)(E->h.ctl.launch_iters + (E->h.ctl.abort ? 1u : 0u)) *
                            E->kernels_per_iter();
    if (E->h.ctl.error) {
      batch_fail_all<K>(c, cls, WG_E_DEVICE_TIMEOUT);
      return set_err(WG_E_DEVICE_TIMEOUT, "a bounded device wait gave up");
    }
    if (E->h.ctl.abort) {
      ++E->regrows;
      TRY(batch_grow<K>(c, cls));
    }
    TRY(batch_retire<K>(c, cls));
  } else if (E->grow_wait) {  // paused: retry once memory has come back
    if (drop_idle_batch(c, cls) || c->used < E->wait_used) {
      TRY(batch_grow<K>(c, cls));
      if (!E->grow_wait) *progressed = true;
    }
  }
  if (E->grow_wait) return WG_OK;
  TRY(batch_admit<K>(c, cls));
  uint32_t active = 0;
  for (const Inst& I : E->hi) active += I.state == INST_ACTIVE;
  if (active) {
    // a lone query (nothing queued, nothing else running anywhere) runs to
    // its fixpoint in this one launch, as the plain loop would: capping its
    // iterations only adds host round trips while nobody waits to join
    bool lone = active == 1 && c->pending.empty() && !solo_running(c);
    for (auto& kv : c->batch)
      if (lone && kv.first != cls && batch_holds_work_any(c, kv.first)) lone = false;
    TRY(E->launch(lone ? 0xFFFFFFFFu : iters, WG_LOOP_DEVICE));
    *progressed = true;
  }
  return WG_OK;
}

static int ensure_batch_engine(wg_ctx* c, int cls, Relation* R);

// A dropped engine is built again for the requests of its class still queued
// (not while another class's exclusive query waits for the memory).  If its
// first pools do not fit although no other batch engine holds any, those
// requests fail with the allocation's error.
static int rebuild_batch(wg_ctx* c, int cls) {
  Query* x = excl_query(c);
  if (x && (x->solo || x->bclass != cls)) return WG_OK;
  Query* p = nullptr;
  for (uint64_t qid : c->pending) {
    auto it = c->queries.find(qid);
    if (it != c->queries.end() && !it->second->solo && it->second->bclass == cls) {
      p = it->second.get();
      break;
    }
  }
  if (!p) return WG_OK;
  const int rc = ensure_batch_engine(c, cls, p->rel);
  if (rc != WG_E_BUDGET && rc != WG_E_NOMEM) return rc;
  cudaGetLastError();
  for (auto& kv : c->batch)
    if (kv.second) return WG_OK;  // memory may come back: retry next round
  if (held_elsewhere(c, cls)) return WG_OK;
  std::vector<uint64_t> still;
  for (uint64_t qid : c->pending) {
    auto it = c->queries.find(qid);
    if (it == c->queries.end()) continue;
    Query* q = it->second.get();
    if (q->solo || q->bclass != cls) { still.push_back(qid); continue; }
    q->state = WG_FAILED;
    q->error = rc;
    q->t_done_us = now_us();
    c->completed.push_back(qid);
  }
  c->pending.swap(still);
  return WG_OK;
}

static int batch_round_any(wg_ctx* c, int cls, uint32_t iters, bool wait_launch,
                           bool* progressed) {
  if (!c->batch[cls]) TRY(rebuild_batch(c, cls));
  if (!c->batch[cls]) return WG_OK;
  return c->batch[cls]->kb() == 4
             ? batch_round<uint32_t>(c, cls, iters, wait_launch, progressed)
             : batch_round<unsigned long long>(c, cls, iters, wait_launch, progressed);
}

static bool batch_busy(wg_ctx* c) {
  for (auto& kv : c->batch) {
    if (!kv.second) continue;
    const bool fl = kv.second->kb() == 4 ? static_cast<Engine<uint32_t>*>(kv.second.get())->in_flight
                                         : static_cast<Engine<unsigned long long>*>(kv.second.get())->in_flight;
    if (fl) return true;
  }
  return false;
}

// One serving round over every batch engine, without waiting on one engine
// while another could run: engines whose launch finished are retired,
// admitted and relaunched; if none had finished, wait briefly and retry.
static int solo_round(wg_ctx* c, bool* progressed, bool* busy);

static int serve_round(wg_ctx* c, uint32_t iters) {
  for (long spin = 0;; ++spin) {
    bool progressed = false, solo_busy = false;
    TRY(solo_round(c, &progressed, &solo_busy));
    for (auto& kv : c->batch) TRY(batch_round_any(c, kv.first, iters, false, &progressed));
    if (progressed || !(batch_busy(c) || solo_busy)) return WG_OK;
    if (spin > 12000000) {  // ~10 min without any launch finishing
      return set_err(WG_E_DEVICE_TIMEOUT, "no launch finished");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

static int ensure_batch_engine(wg_ctx* c, int cls, Relation* R) {
  if (c->batch[cls]) return WG_OK;
  int rc = WG_OK;
  cudaStream_t& cs = c->class_st[cls];
  if (!cs) CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  EngineBase* e = new_engine(c, R->kb, false, kBatchSlots, class_bits(cls), kBatchLogCap, true,
                             false, &rc, false, false, 0, cs);
  if (!e) return rc;
  c->batch[cls].reset(e);
  g_binfo[c][cls].slot_q.assign(kBatchSlots, 0);
  g_binfo[c][cls].est.assign(kBatchSlots, 0.0);
  g_binfo[c][cls].seq.assign(kBatchSlots, 0);
  // start with pools worth about a third of the free budget; they grow later
  // only as far as the budget allows (then the largest instance is preempted)
  const double per_key = 4.0 * R->kb + 8.5 + 2.0 * R->kb + R->kb / 4.0;
  const bool small = (cls & 1) == 0;  // small-query engines need far smaller pools
  const double avail = (double)(c->budget - c->used) / (small ? 8.0 : 3.0);
  const unsigned long long capC = std::max<unsigned long long>(1ull << 16, (unsigned long long)(avail / per_key));
  const int prc = R->kb == 4
                      ? static_cast<Engine<uint32_t>*>(e)->ensure(capC, capC, capC / 4, false)
                      : static_cast<Engine<unsigned long long>*>(e)->ensure(capC, capC, capC / 4, false);
  if (prc != WG_OK) {  // no pools: drop the engine, a later request builds it again
    c->batch[cls].reset();
    g_binfo[c].erase(cls);
  }
  return prc;
}

template <typename K>
static int copy_result(wg_ctx* c, Query* q, unsigned long long* dst, bool host) {
  const size_t n = q->n_tuples;
  if (!n) return WG_OK;
  // a page-locked destination takes large DMA chunks; pageable memory is
  // staged by the driver anyway, so keep the device buffer small there
  bool locked = false;
  if (host) {
    cudaPointerAttributes pa{};
    locked = cudaPointerGetAttributes(&pa, dst) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();  // pageable pointers are not an error
  }
  const size_t chunk = host ? (size_t)1 << (locked ? 26 : 24) : n;
  DBuf tmp;
  if (host) TRY(tmp.get(c, std::min(n, chunk) * 8));
  for (size_t at = 0; at < n; at += chunk) {
    const size_t m = std::min(chunk, n - at);
    unsigned long long* o = host ? (unsigned long long*)tmp.p : dst + at;
    launch_result_map<K>((const K*)q->res_ptr + at, m, q->rel->w, (const uint32_t*)q->rel->V.p, o,
                         grid_of(c, 4), c->stream);
    CK(cudaGetLastError());
    if (host) CK(cudaMemcpyAsync(dst + at, tmp.p, m * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  tmp.release(c);
  return WG_OK;
}

// ------------------------------------------------------------------ C-ABI
extern "C" {

const char* wg_last_error(void) { return g_err.c_str(); }

int wg_init(int device, size_t budget, wg_alloc_fn alloc, wg_free_fn free_fn, void* user,
            void* stream, wg_ctx** out) {
  if (!out) return set_err(WG_E_INVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return set_err(WG_E_INVAL, "no such device");
  CK(cudaSetDevice(device));
  auto c = std::make_unique<wg_ctx>();
  c->device = device;
  c->alloc = alloc; c->free_fn = free_fn; c->user = user;
  CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  c->budget = budget ? budget : (size_t)(0.9 * (double)fr);
  *out = c.release();
  return WG_OK;
}

void wg_destroy(wg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->queries) kv.second->res_own.release(c);
  for (auto& kv : c->queries) {
    Query* q = kv.second.get();
    if (q->ev0) cudaEventDestroy(q->ev0);
    if (q->ev1) cudaEventDestroy(q->ev1);
    if (q->eng) q->eng->release();
  }
  c->queries.clear();
  for (auto& e : c->idle) e->release();
  c->idle.clear();
  for (auto& kv : c->batch) if (kv.second) kv.second->release();
  c->batch.clear();
  for (auto& kv : c->class_st) {
    cudaStreamSynchronize(kv.second);
    cudaStreamDestroy(kv.second);
  }
  c->class_st.clear();
  g_binfo.erase(c);
  for (auto& kv : c->rels) kv.second->release(c);
  c->rels.clear();
  dev_free(c, c->s_tmp, c->s_tmp_bytes);
  dev_free(c, c->s_status, c->s_status_n * 8);
  dev_free(c, c->s_hist, sizeof(unsigned long long) * kMaxPasses * kRadix);
  dev_free(c, c->s_stage, sizeof(Stage) * S_NUM);
  dev_free(c, c->s_seg, sizeof(Seg));
  dev_free(c, c->s_ctl, sizeof(Ctl));
  cudaStreamSynchronize(c->stream);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

size_t wg_mem_used(const wg_ctx* c) { return c ? c->used : 0; }

static int load_common(wg_ctx* c, const uint32_t* d_src, const uint32_t* d_dst, size_t n,
                       wg_rel* out) {
  auto R = std::make_unique<Relation>();
  int rc = load_relation(c, d_src, d_dst, n, R.get());
  if (rc != WG_OK) { R->release(c); return rc; }
  CK(cudaStreamSynchronize(c->stream));
  const uint64_t id = c->next_id++;
  c->rels[id] = std::move(R);
  *out = id;
  return WG_OK;
}

int wg_relation_load(wg_ctx* c, const uint32_t* src, const uint32_t* dst, size_t n, wg_rel* out) {
  if (!c || !out || (n && (!src || !dst))) return set_err(WG_E_INVAL, "bad argument");
  *out = 0;
  DBuf s, d;
  if (n) {
    TRY(s.get(c, n * 4));
    TRY(d.get(c, n * 4));
    CK(cudaMemcpyAsync(s.p, src, n * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d.p, dst, n * 4, cudaMemcpyHostToDevice, c->stream));
  }
  int rc = load_common(c, (const uint32_t*)s.p, (const uint32_t*)d.p, n, out);
  s.release(c);
  d.release(c);
  return rc;
}

int wg_relation_load_device(wg_ctx* c, const uint32_t* d_src, const uint32_t* d_dst, size_t n,
                            wg_rel* out) {
  if (!c || !out || (n && (!d_src || !d_dst))) return set_err(WG_E_INVAL, "bad argument");
  *out = 0;
  return load_common(c, d_src, d_dst, n, out);
}

int wg_relation_info(wg_ctx* c, wg_rel r, uint64_t* ne, uint32_t* nv, uint32_t* bits) {
  if (!c) return set_err(WG_E_INVAL, "ctx is NULL");
  auto it = c->rels.find(r);
  if (it == c->rels.end()) return set_err(WG_E_INVAL, "no such relation");
  if (ne) *ne = it->second->ne;
  if (nv) *nv = it->second->nv;
  if (bits) *bits = it->second->w;
  return WG_OK;
}

void wg_relation_free(wg_ctx* c, wg_rel r) {
  if (!c) return;
  auto it = c->rels.find(r);
  if (it == c->rels.end()) return;
  for (auto& kv : c->queries)
    if (kv.second->rel == it->second.get() && kv.second->state == WG_RUNNING) return;  // in use
  cudaStreamSynchronize(c->stream);
  it->second->release(c);
  c->rels.erase(it);
}

static int make_query(wg_ctx* c, int kind, wg_rel edges, const wg_opts* opts, Query** out) {
  if (opts && opts->loop > WG_LOOP_HOST_STAGED) return set_err(WG_E_INVAL, "unknown loop mode");
  auto it = c->rels.find(edges);
  if (it == c->rels.end()) return set_err(WG_E_INVAL, "no such relation");
  auto q = std::make_unique<Query>();
  q->id = c->next_id++;
  q->kind = kind;
  q->rel = it->second.get();
  q->rel_id = edges;
  if (opts) q->opts = *opts;
  if (q->opts.max_iters == 0) q->opts.max_iters = 1u << 20;
  CK(cudaEventCreate(&q->ev0));
  CK(cudaEventCreate(&q->ev1));
  q->t_submit_us = now_us();
  *out = q.get();
  c->queries[q->id] = std::move(q);
  return WG_OK;
}

// Give query q a single-query engine (an idle one of the same key width, pass
// plan and stage layout, else a new one) and start its fixpoint.
static int single_begin(wg_ctx* c, Query* q) {
  Relation* R = q->rel;
  const int kind = q->kind;
  const bool fuse = !(q->opts.flags & WG_FLAG_SEPARATE_STAGES);
  const bool full_width = (q->opts.flags & WG_FLAG_FULL_WIDTH) != 0;
  const bool copyback = fuse && (q->opts.flags & WG_FLAG_COPY_BACK) != 0;
  const bool hashjoin = kind == WG_TC && (q->opts.flags & WG_FLAG_HASH_JOIN) != 0;
  // Full as a main run plus a side run of the newest tuples (fused stages,
  // no copy-back): unless the query asks for the merge every iteration
  const uint32_t side = !fuse || copyback || (q->opts.flags & WG_FLAG_MERGE_EVERY_ITER) ? 0u
                        : (q->opts.flags & WG_FLAG_SIDE_RUN_ALWAYS) ? 2u : 1u;
  if (hashjoin && !R->htab.p) {
    // the table of E, built once per relation like its CSR: at most half full
    unsigned long long cap = 1024;
    while (cap < 2 * (unsigned long long)R->ne) cap <<= 1;
    int brc = R->htab.get(c, cap * 8);
    if (brc == WG_OK && cudaMemsetAsync(R->htab.p, 0xFF, cap * 8, c->stream) != cudaSuccess)
      brc = set_err(WG_E_CUDA, "hash table clear");
    if (brc == WG_OK) {
      R->hmask = cap - 1;
      if (R->kb == 4)
        launch_hash_build<uint32_t>((const uint32_t*)R->keys.p, R->ne, R->w,
                                    (unsigned long long*)R->htab.p, R->hmask, grid_of(c, 8),
                                    c->stream);
      else
        launch_hash_build<unsigned long long>((const unsigned long long*)R->keys.p, R->ne, R->w,
                                              (unsigned long long*)R->htab.p, R->hmask,
                                              grid_of(c, 8), c->stream);
      if (cudaGetLastError() != cudaSuccess) brc = set_err(WG_E_CUDA, "hash table build");
    }
    if (brc != WG_OK) { R->htab.release(c); return brc; }
  }
  // TC candidates leave the join grouped by source: sort each group on the
  // destination field only (per-vertex histograms bound the vertex count)
  const bool xseg = !full_width && kind == WG_TC && R->nv <= kXSegMaxVertices;
  const uint32_t bits = full_width ? 8u * R->kb : xseg ? R->w : 2 * R->w;
  const uint32_t ct = R->kb == 4 ? count_tile_of<uint32_t>(c) : count_tile_of<unsigned long long>(c);
  const uint32_t ft = R->kb == 4 ? fuse_tile_of<uint32_t>(c) : fuse_tile_of<unsigned long long>(c);
  const uint32_t et = R->kb == 4 ? emit_tile_of<uint32_t>(c) : emit_tile_of<unsigned long long>(c);
  for (size_t i = 0; i < c->idle.size() && !q->own; ++i)
    if (c->idle[i]->kb() == R->kb && c->idle[i]->bits() == bits && c->idle[i]->fused() == fuse &&
        c->idle[i]->xgrouped() == xseg && c->idle[i]->copyback() == copyback &&
        c->idle[i]->hashjoin() == hashjoin && c->idle[i]->count_tile() == ct &&
        c->idle[i]->fuse_tile() == ft && c->idle[i]->sort_mode() == c->tune_sort[R->kb == 8] &&
        c->idle[i]->emit_tile() == et &&
        c->idle[i]->side_mode() == side) {
      q->own = std::move(c->idle[i]);
      c->idle.erase(c->idle.begin() + i);
    }
  int rc = WG_OK;
  if (!q->own) {
    EngineBase* e = new_engine(c, R->kb, true, 1, bits, 1u << 16, fuse, xseg, &rc, copyback,
                               hashjoin, side);
    if (!e) return rc;
    q->own.reset(e);
  }
  q->eng = q->own.get();
  if (hashjoin) {  // this relation's table, in the host mirror too (pool regrowth rewrites it)
    TRY(R->kb == 4
            ? static_cast<Engine<uint32_t>*>(q->eng)->put_htab(R->htab.p, R->hmask)
            : static_cast<Engine<unsigned long long>*>(q->eng)->put_htab(R->htab.p, R->hmask));
  }
  if (R->kb == 4) {
    auto* E = static_cast<Engine<uint32_t>*>(q->eng);
    E->regrows = 0; E->launches_issued = 0;
    return single_start<uint32_t>(c, q);
  }
  auto* E = static_cast<Engine<unsigned long long>*>(q->eng);
  E->regrows = 0; E->launches_issued = 0;
  return single_start<unsigned long long>(c, q);
}

static int single_query(wg_ctx* c, int kind, wg_rel edges, const wg_opts* opts, wg_query* out) {
  if (!c || !out) return set_err(WG_E_INVAL, "bad argument");
  *out = 0;
  Query* q;
  TRY(make_query(c, kind, edges, opts, &q));
  const int rc = single_begin(c, q);
  if (rc != WG_OK) {  // nothing left running: drop the query, its engine goes back idle
    q->state = WG_FAILED;
    q->error = rc;
    wg_query_free(c, q->id);
    return rc;
  }
  *out = q->id;
  return WG_OK;
}

}  // extern "C" (templates below)

// ------------------------------------------------------------------ served large requests
// A served request over more than kSoloEdges edges runs on a single-query
// engine, one at a time on the context stream, while the batch engines take
// the small requests.  A growth over the budget pauses it with its state as
// the exclusive query: the batch engines admit nothing, drain and are
// dropped, then it grows and resumes from the iteration that overflowed; if
// it does not fit with the whole budget it fails.  If another query is
// already exclusive it is requeued instead (restarting later).
template <typename K>
static int solo_resume(wg_ctx* c, Query* q) {
  auto* E = static_cast<Engine<K>*>(q->eng);
  const int rc = E->grow();
  if (rc == WG_E_BUDGET || rc == WG_E_NOMEM) {
    cudaGetLastError();
    q->wait_used = c->used;
    return WG_OK;
  }
  TRY(rc);
  q->solo_wait = false;
  return E->launch(0xFFFFFFFFu, loop_mode(q));
}

static void solo_requeue(wg_ctx* c, Query* q) {
  if (q->own) c->idle.push_back(std::move(q->own));  // its pools may be dropped meanwhile
  q->eng = nullptr;
  q->solo_wait = false;
  q->state = WG_PENDING;
  q->regrows += 1;
  c->pending.insert(c->pending.begin(), q->id);
  if (c->solo_run == q->id) c->solo_run = 0;
}

static void solo_finish(wg_ctx* c, Query* q, int rc) {
  if (rc != WG_OK && q->state != WG_FAILED) {
    q->state = WG_FAILED;
    q->error = rc;
  }
  if (c->excl == q->id) c->excl = 0;
  q->t_done_us = now_us();
  c->completed.push_back(q->id);
  if (c->solo_run == q->id) c->solo_run = 0;
}

static int solo_round(wg_ctx* c, bool* progressed, bool* busy) {
  *busy = false;
  if (c->solo_run && !solo_running(c)) c->solo_run = 0;  // freed while running
  if (c->solo_run) {
    Query* q = c->queries.find(c->solo_run)->second.get();
    const bool k4 = q->eng->kb() == 4;
    if (q->solo_wait) {
      Query* x = excl_query(c);
      if (x && x != q) {  // another query waits for the whole budget first
        solo_requeue(c, q);
        *progressed = true;
        return WG_OK;
      }
      c->excl = q->id;
      if (drop_idle_batch(c, -1) || c->used < q->wait_used) {
        TRY(k4 ? solo_resume<uint32_t>(c, q) : solo_resume<unsigned long long>(c, q));
        if (!q->solo_wait) *progressed = true;
      }
      if (q->solo_wait) {
        bool held = false;  // memory that may still come back
        for (auto& kv : c->batch) held |= kv.second != nullptr;
        if (!held) {
          solo_finish(c, q, WG_E_BUDGET);
          *progressed = true;
        }
        return WG_OK;
      }
    }
    const int rc = k4 ? single_progress<uint32_t>(c, q, false, true)
                      : single_progress<unsigned long long>(c, q, false, true);
    if (q->solo_wait && !growth_could_fit(c, q->eng)) {  // hopeless: fail now
      solo_finish(c, q, set_err(WG_E_BUDGET, "the request does not fit the memory budget"));
      *progressed = true;
      return WG_OK;
    }
    if (q->solo_wait) {  // paused: exclusive from now on, unless another query is
      Query* x = excl_query(c);
      if (x && x != q) solo_requeue(c, q);
      else c->excl = q->id;
      *progressed = true;
      return WG_OK;
    }
    if (q->state == WG_RUNNING && rc == WG_OK) {
      *busy = true;
      return WG_OK;
    }
    solo_finish(c, q, rc);
    *progressed = true;
    if (rc == WG_E_CUDA || rc == WG_E_DEVICE_TIMEOUT) return rc;
  }
  // start the next queued large request
  Query* x = excl_query(c);
  for (size_t i = 0; i < c->pending.size(); ++i) {
    auto it = c->queries.find(c->pending[i]);
    if (it == c->queries.end() || !it->second->solo) continue;
    Query* q = it->second.get();
    if (x && x != q) return WG_OK;  // only the exclusive query may start
    if (x == q) {  // once the batch engines hold no work, they go
      for (auto& kv : c->batch)
        if (batch_holds_work_any(c, kv.first)) return WG_OK;
      drop_idle_batch(c, -1);
    }
    c->pending.erase(c->pending.begin() + i);
    q->state = WG_RUNNING;
    c->solo_run = q->id;
    *progressed = true;
    const int rc = single_begin(c, q);
    if (rc == WG_OK) {
      *busy = true;
      return WG_OK;
    }
    if (rc != WG_E_BUDGET && rc != WG_E_NOMEM) {
      solo_finish(c, q, rc);
      return WG_OK;  // the request failed; the server carries on
    }
    cudaGetLastError();
    bool held = false;
    for (auto& kv : c->batch) held |= kv.second != nullptr;
    if (held && (!x || x == q)) {  // wait for the whole budget
      solo_requeue(c, q);
      q->regrows -= 1;
      c->excl = q->id;
    } else {
      solo_finish(c, q, rc);
    }
    return WG_OK;
  }
  return WG_OK;
}

extern "C" {

int wg_tc(wg_ctx* c, wg_rel edges, const wg_opts* opts, wg_query* out) {
  return single_query(c, WG_TC, edges, opts, out);
}
int wg_sg(wg_ctx* c, wg_rel edges, const wg_opts* opts, wg_query* out) {
  return single_query(c, WG_SG, edges, opts, out);
}

int wg_submit(wg_ctx* c, const wg_request* reqs, size_t n, wg_query* ids) {
  if (!c || (n && (!reqs || !ids))) return set_err(WG_E_INVAL, "bad argument");
  for (size_t i = 0; i < n; ++i) {
    ids[i] = 0;
    if (reqs[i].kind != WG_TC && reqs[i].kind != WG_SG) return set_err(WG_E_INVAL, "bad kind");
    Query* q;
    TRY(make_query(c, reqs[i].kind, reqs[i].edges, &reqs[i].opts, &q));
    q->batch = true;
    q->bclass = batch_class(q->rel);
    q->solo = q->rel->ne > kSoloEdges;
    if (q->solo) {
      // runs on a single-query engine (solo_round)
    } else if (!excl_query(c)) {
      TRY(ensure_batch_engine(c, q->bclass, q->rel));
    } else {
      c->batch[q->bclass];  // the class is listed; its engine is built on demand
    }
    c->pending.push_back(q->id);
    ids[i] = q->id;
  }
  return WG_OK;
}

int wg_serve_step(wg_ctx* c, uint32_t iters, size_t* n_running) {
  if (!c) return set_err(WG_E_INVAL, "ctx is NULL");
  if (iters == 0) iters = 0xFFFFFFFFu;
  TRY(serve_round(c, iters));
  if (n_running) {
    size_t r = 0;
    for (auto& kv : c->queries) r += kv.second->batch && kv.second->state == WG_RUNNING;
    *n_running = r + c->pending.size();
  }
  return WG_OK;
}

int wg_take_completed(wg_ctx* c, wg_query* ids, size_t cap, size_t* n_out) {
  if (!c || !n_out || (cap && !ids)) return set_err(WG_E_INVAL, "bad argument");
  const size_t n = std::min(cap, c->completed.size());
  for (size_t i = 0; i < n; ++i) ids[i] = c->completed[i];
  c->completed.erase(c->completed.begin(), c->completed.begin() + n);
  *n_out = n;
  return WG_OK;
}

static Query* find_q(wg_ctx* c, wg_query id) {
  auto it = c->queries.find(id);
  return it == c->queries.end() ? nullptr : it->second.get();
}

static int progress(wg_ctx* c, Query* q, bool block) {
  if (q->state == WG_DONE || q->state == WG_FAILED) return WG_OK;
  if (q->batch) {
    // drive the batch engines until this query is retired
    if (!block) {
      bool progressed = false, busy = false;
      TRY(solo_round(c, &progressed, &busy));
      for (auto& kv : c->batch) TRY(batch_round_any(c, kv.first, 0xFFFFFFFFu, false, &progressed));
      return WG_OK;
    }
    while (q->state != WG_DONE && q->state != WG_FAILED) TRY(serve_round(c, 0xFFFFFFFFu));
    return WG_OK;
  }
  return q->eng->kb() == 4 ? single_progress<uint32_t>(c, q, block)
                           : single_progress<unsigned long long>(c, q, block);
}

int wg_poll(wg_ctx* c, wg_query id, wg_status* st) {
  if (!c || !st) return set_err(WG_E_INVAL, "bad argument");
  Query* q = find_q(c, id);
  if (!q) return set_err(WG_E_INVAL, "no such query");
  int rc = progress(c, q, false);
  st->state = q->state;
  st->error = q->error;
  st->n_tuples = q->n_tuples;
  st->iterations = q->iterations;
  st->regrows = q->regrows;
  st->candidates = q->candidates;
  st->gpu_launches = q->launches;
  st->device_ms = q->device_ms;
  return rc == WG_E_DEVICE_TIMEOUT || rc == WG_E_CUDA ? rc : WG_OK;
}

int wg_wait(wg_ctx* c, wg_query id, uint64_t timeout_us) {
  if (!c) return set_err(WG_E_INVAL, "ctx is NULL");
  Query* q = find_q(c, id);
  if (!q) return set_err(WG_E_INVAL, "no such query");
  const double t0 = now_us();
  for (;;) {
    const bool block = timeout_us == 0;
    TRY(progress(c, q, block));
    if (q->state == WG_DONE) return WG_OK;
    if (q->state == WG_FAILED) return set_err(q->error, "query failed");
    if (timeout_us && now_us() - t0 > (double)timeout_us) return WG_E_NOT_READY;
  }
}

static int result_common(wg_ctx* c, wg_query id, uint64_t* keys, size_t cap, size_t* n_out,
                         bool host) {
  if (!c || !n_out) return set_err(WG_E_INVAL, "bad argument");
  Query* q = find_q(c, id);
  if (!q) return set_err(WG_E_INVAL, "no such query");
  if (q->state != WG_DONE) return set_err(q->state == WG_FAILED ? q->error : WG_E_NOT_READY, "result not ready");
  *n_out = q->n_tuples;
  if (cap < q->n_tuples) return set_err(WG_E_CAPACITY, "buffer too small");
  if (q->n_tuples && !keys) return set_err(WG_E_INVAL, "keys is NULL");
  return q->rel->kb == 4 ? copy_result<uint32_t>(c, q, (unsigned long long*)keys, host)
                         : copy_result<unsigned long long>(c, q, (unsigned long long*)keys, host);
}

int wg_result_digest(wg_ctx* c, wg_query id, uint64_t* digest) {
  if (!c || !digest) return set_err(WG_E_INVAL, "bad argument");
  Query* q = find_q(c, id);
  if (!q) return set_err(WG_E_INVAL, "no such query");
  if (q->state != WG_DONE) return set_err(q->state == WG_FAILED ? q->error : WG_E_NOT_READY, "result not ready");
  *digest = 0;
  if (!q->n_tuples) return WG_OK;
  DBuf acc;
  TRY(acc.get(c, 8));
  int rc = WG_OK;
  unsigned long long h = 0;
  if (cudaMemsetAsync(acc.p, 0, 8, c->stream) != cudaSuccess) {
    rc = set_err(WG_E_CUDA, "digest clear");
  } else {
    const uint32_t* V = (const uint32_t*)q->rel->V.p;
    if (q->rel->kb == 4)
      launch_result_digest<uint32_t>((const uint32_t*)q->res_ptr, q->n_tuples, q->rel->w, V,
                                     (unsigned long long*)acc.p, grid_of(c, 8), c->stream);
    else
      launch_result_digest<unsigned long long>((const unsigned long long*)q->res_ptr, q->n_tuples,
                                               q->rel->w, V, (unsigned long long*)acc.p,
                                               grid_of(c, 8), c->stream);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, acc.p, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      rc = set_err(WG_E_CUDA, "digest");
  }
  acc.release(c);
  *digest = h;
  return rc;
}

int wg_result_copy(wg_ctx* c, wg_query q, uint64_t* keys, size_t cap, size_t* n_out) {
  return result_common(c, q, keys, cap, n_out, true);
}
int wg_result_copy_device(wg_ctx* c, wg_query q, uint64_t* d_keys, size_t cap, size_t* n_out) {
  return result_common(c, q, d_keys, cap, n_out, false);
}

int wg_result_iters(wg_ctx* c, wg_query id, uint64_t* sizes, size_t cap, size_t* n_out) {
  if (!c || !n_out) return set_err(WG_E_INVAL, "bad argument");
  Query* q = find_q(c, id);
  if (!q) return set_err(WG_E_INVAL, "no such query");
  if (q->state != WG_DONE && q->state != WG_FAILED) return set_err(WG_E_NOT_READY, "not finished");
  *n_out = q->log.size();
  if (cap < q->log.size()) return set_err(WG_E_CAPACITY, "buffer too small");
  if (!q->log.empty()) std::memcpy(sizes, q->log.data(), q->log.size() * 8);
  return WG_OK;
}

int wg_result_profile(wg_ctx* c, wg_query id, wg_kernel_stat* stats, size_t cap, size_t* n_out) {
  if (!c || !n_out) return set_err(WG_E_INVAL, "bad argument");
  Query* q = find_q(c, id);
  if (!q) return set_err(WG_E_INVAL, "no such query");
  *n_out = q->prof.size();
  if (cap < q->prof.size()) return set_err(WG_E_CAPACITY, "buffer too small");
  for (size_t i = 0; i < q->prof.size(); ++i) {
    std::memset(&stats[i], 0, sizeof(wg_kernel_stat));
    std::snprintf(stats[i].name, sizeof(stats[i].name), "%s", q->prof[i].name);
    stats[i].launches = q->prof[i].launches;
    stats[i].total_ms = q->prof[i].ms;
    stats[i].bytes = q->prof[i].bytes;
  }
  return WG_OK;
}

int wg_selftest_wait_timeout(wg_ctx* c) {
  if (!c) return set_err(WG_E_INVAL, "ctx is NULL");
  DBuf b;  // Ctl | status words | result
  const size_t ctl_bytes = (sizeof(Ctl) + 63) / 64 * 64;
  TRY(b.get(c, ctl_bytes + 64));
  char* base = (char*)b.p;
  Ctl* ctl = (Ctl*)base;
  unsigned long long* status = (unsigned long long*)(base + ctl_bytes);
  int rc = WG_OK;
  if (cudaMemsetAsync(base, 0, ctl_bytes + 64, c->stream) != cudaSuccess) {
    rc = set_err(WG_E_CUDA, "self-test clear");
  } else {
    launch_selftest_wait(status, ctl, status + 4, c->stream);
    Ctl h{};
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      rc = set_err(WG_E_CUDA, "self-test launch");
    else if (h.error == DEV_TIMEOUT)
      rc = set_err(WG_E_DEVICE_TIMEOUT, "the bounded device wait gave up (self-test)");
  }
  b.release(c);
  if (rc == WG_E_DEVICE_TIMEOUT) {
    // the allocation-free sort's control block records the same timeout
    const int r2 = noalloc_selftest_wait(c->stream);
    if (r2 != WG_OK) return r2;
    set_err(WG_E_DEVICE_TIMEOUT, "the bounded device wait gave up (self-test)");
  }
  return rc;
}

int wg_set_tiles(wg_ctx* c, int key_bytes, uint32_t count_tile, uint32_t fuse_tile,
                 uint32_t emit_tile) {
  if (!c || (key_bytes != 4 && key_bytes != 8)) return set_err(WG_E_INVAL, "bad argument");
  const uint32_t T = key_bytes == 4 ? FuseTile<uint32_t>::T : FuseTile<unsigned long long>::T;
  if (count_tile && count_tile != (uint32_t)kTileD && count_tile != (uint32_t)kTileD / 2)
    return set_err(WG_E_INVAL, "count tile is not a compiled shape");
  if (fuse_tile && fuse_tile != T && fuse_tile != T / 2)
    return set_err(WG_E_INVAL, "fused tile is not a compiled shape");
  if (emit_tile && emit_tile != (uint32_t)kTileC && emit_tile != (uint32_t)kTileC / 2)
    return set_err(WG_E_INVAL, "emit tile is not a compiled shape");
  c->tune_count[key_bytes == 8] = count_tile;
  c->tune_fuse[key_bytes == 8] = fuse_tile;
  c->tune_emit[key_bytes == 8] = emit_tile;
  return WG_OK;
}

int wg_set_sort(wg_ctx* c, int key_bytes, uint32_t mode) {
  if (!c || (key_bytes != 4 && key_bytes != 8) || mode > WG_SORT_SEGMENT_WIDE)
    return set_err(WG_E_INVAL, "bad argument");
  c->tune_sort[key_bytes == 8] = mode;
  return WG_OK;
}

// One profiled fixpoint: the join-count, radix-sort and fused-stage times (ms).
static int tune_run(wg_ctx* c, wg_rel edges, int kind, double* count_ms, double* fuse_ms,
                    double* sort_ms = nullptr, double* emit_ms = nullptr) {
  wg_opts o{};
  o.profile = 1;
  wg_query id = 0;
  TRY(single_query(c, kind, edges, &o, &id));
  const int rc = wg_wait(c, id, 0);
  *count_ms = *fuse_ms = 0;
  if (sort_ms) *sort_ms = 0;
  if (emit_ms) *emit_ms = 0;
  if (rc == WG_OK) {
    Query* q = find_q(c, id);
    for (const KStat& k : q->prof) {
      if (!std::strcmp(k.name, "join_count")) *count_ms = k.ms;
      if (emit_ms && !std::strcmp(k.name, "join_emit")) *emit_ms = k.ms;
      if (!std::strcmp(k.name, "dedup_diff_merge") || !std::strcmp(k.name, "dedup_diff")) *fuse_ms += k.ms;
      if (sort_ms && (!std::strcmp(k.name, "sort_hist") || !std::strcmp(k.name, "sort_pass")))
        *sort_ms += k.ms;
    }
  }
  wg_query_free(c, id);
  return rc;
}

int wg_autotune(wg_ctx* c, wg_rel edges, int kind, wg_tune* out) {
  if (!c || (kind != WG_TC && kind != WG_SG)) return set_err(WG_E_INVAL, "bad argument");
  auto it = c->rels.find(edges);
  if (it == c->rels.end()) return set_err(WG_E_INVAL, "no such relation");
  const int kb = it->second->kb, i = kb == 8;
  const uint32_t T = kb == 4 ? FuseTile<uint32_t>::T : FuseTile<unsigned long long>::T;
  wg_tune t{};
  t.key_bytes = (uint32_t)kb;
  t.count_cand[0] = kTileD; t.count_cand[1] = kTileD / 2;
  t.fuse_cand[0] = T; t.fuse_cand[1] = T / 2;
  t.emit_cand[0] = kTileC; t.emit_cand[1] = kTileC / 2;
  const uint32_t keep_count = c->tune_count[i], keep_fuse = c->tune_fuse[i],
                 keep_emit = c->tune_emit[i];
  for (int v = 0; v < 2; ++v) {
    // the three stages are separate kernels: one run per candidate triple times all
    c->tune_count[i] = t.count_cand[v];
    c->tune_fuse[i] = t.fuse_cand[v];
    c->tune_emit[i] = t.emit_cand[v];
    for (int rep = 0; rep < 2; ++rep) {  // the first run grows the engine's pools
      const int rc = tune_run(c, edges, kind, &t.count_ms[v], &t.fuse_ms[v], nullptr,
                              &t.emit_ms[v]);
      if (rc != WG_OK) {
        c->tune_count[i] = keep_count;
        c->tune_fuse[i] = keep_fuse;
        c->tune_emit[i] = keep_emit;
        return rc;
      }
    }
  }
  t.count_tile = t.count_ms[1] < t.count_ms[0] ? t.count_cand[1] : t.count_cand[0];
  t.fuse_tile = t.fuse_ms[1] < t.fuse_ms[0] ? t.fuse_cand[1] : t.fuse_cand[0];
  t.emit_tile = t.emit_ms[1] < t.emit_ms[0] ? t.emit_cand[1] : t.emit_cand[0];
  c->tune_count[i] = t.count_tile;
  c->tune_fuse[i] = t.fuse_tile;
  c->tune_emit[i] = t.emit_tile;
  // the radix sort of the per-source segments (single TC queries that sort
  // per source): each mode with the chosen tiles
  const uint32_t keep_sort = c->tune_sort[i];
  t.sort_mode = keep_sort;
  if (kind == WG_TC && it->second->nv <= kXSegMaxVertices) {
    for (uint32_t m = 0; m <= WG_SORT_SEGMENT_WIDE; ++m) {
      c->tune_sort[i] = m;
      double cm = 0, fm = 0;
      for (int rep = 0; rep < 2; ++rep) {
        const int rc = tune_run(c, edges, kind, &cm, &fm, &t.sort_ms[m]);
        if (rc != WG_OK) {
          c->tune_sort[i] = keep_sort;
          return rc;
        }
      }
    }
    t.sort_mode = 0;
    for (uint32_t m = 1; m <= WG_SORT_SEGMENT_WIDE; ++m)
      if (t.sort_ms[m] < t.sort_ms[t.sort_mode]) t.sort_mode = m;
  }
  c->tune_sort[i] = t.sort_mode;
  if (out) *out = t;
  return WG_OK;
}

void wg_query_free(wg_ctx* c, wg_query id) {
  if (!c) return;
  auto it = c->queries.find(id);
  if (it == c->queries.end()) return;
  Query* q = it->second.get();
  if (q->state == WG_RUNNING && !q->batch) progress(c, q, true);
  if (q->batch && q->state == WG_PENDING) {
    c->pending.erase(std::remove(c->pending.begin(), c->pending.end(), id), c->pending.end());
  }
  cudaStreamSynchronize(c->stream);
  q->res_own.release(c);
  if (q->ev0) cudaEventDestroy(q->ev0);
  if (q->ev1) cudaEventDestroy(q->ev1);
  if (q->own) c->idle.push_back(std::move(q->own));  // keep pools and graph for the next query
  c->queries.erase(it);
}

int wg_sort_keys(wg_ctx* c, void* d_keys, size_t n, int kb, uint32_t bits) {
  if (!c || (n && !d_keys) || (kb != 4 && kb != 8) || bits == 0 || bits > 8u * kb)
    return set_err(WG_E_INVAL, "bad argument");
  int rc = kb == 4 ? prim_sort<uint32_t>(c, (uint32_t*)d_keys, n, bits)
                   : prim_sort<unsigned long long>(c, (unsigned long long*)d_keys, n, bits);
  if (rc != WG_OK) return rc;
  if (n <= 1) return WG_OK;  // nothing was launched
  Ctl ctl{};
  CK(cudaMemcpyAsync(&ctl, c->s_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (ctl.error) {  // a pass gave up: the keys are unspecified
    CK(cudaMemsetAsync(c->s_ctl, 0, sizeof(Ctl), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return set_err(WG_E_DEVICE_TIMEOUT, "a radix pass's lookback wait gave up");
  }
  return WG_OK;
}

int wg_unique_diff(wg_ctx* c, const void* cand, size_t n, const void* full, size_t nf, void* out,
                   size_t* n_out, int kb) {
  if (!c || !n_out || (n && (!cand || !out)) || (nf && !full) || (kb != 4 && kb != 8))
    return set_err(WG_E_INVAL, "bad argument");
  return kb == 4 ? prim_unique<uint32_t>(c, (const uint32_t*)cand, n, (const uint32_t*)full, nf,
                                         (uint32_t*)out, n_out)
                 : prim_unique<unsigned long long>(c, (const unsigned long long*)cand, n,
                                                   (const unsigned long long*)full, nf,
                                                   (unsigned long long*)out, n_out);
}

int wg_triangles(wg_ctx* c, wg_rel r, uint64_t* count) {
  if (!c || !count) return set_err(WG_E_INVAL, "bad argument");
  auto it = c->rels.find(r);
  if (it == c->rels.end()) return set_err(WG_E_INVAL, "no such relation");
  Relation* R = it->second.get();
  unsigned long long n = 0;
  const int rc = R->kb == 4 ? tri_count<uint32_t>(c, R, &n) : tri_count<unsigned long long>(c, R, &n);
  *count = n;
  return rc;
}

int wg_merge_disjoint(wg_ctx* c, const void* a, size_t na, const void* b, size_t nb, void* out,
                      int kb) {
  if (!c || (na && !a) || (nb && !b) || (na + nb && !out) || (kb != 4 && kb != 8))
    return set_err(WG_E_INVAL, "bad argument");
  int rc = kb == 4 ? prim_merge<uint32_t>(c, (const uint32_t*)a, na, (const uint32_t*)b, nb, (uint32_t*)out)
                   : prim_merge<unsigned long long>(c, (const unsigned long long*)a, na,
                                                    (const unsigned long long*)b, nb,
                                                    (unsigned long long*)out);
  if (rc != WG_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return WG_OK;
}

}  // extern "C"
