// wg_oracle.cpp -- CPU oracle for the semi-naive TC / SG fixpoints.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
// CPU-baseline leg load this library.  It shares no code, header, table or
// helper with the CUDA path; the only thing both sides see is the edge list
// produced by the seeded generators.
//
// What it computes (paper, Sec. Background):
//   * Relations are sets (Sec. Background, "derived relations are sets").
//   * TC:  T(x,y) <- E(x,y).   T(x,z) <- T(x,y), E(y,z).
//   * SG:  sg(x,y) <- edge(p,x), edge(p,y), x != y.            (base rule)
//          sg(x,y) <- edge(a,x), sg(a,b), edge(b,y).           (Sec. Generalization,
//          the paper's parent(X,P) read as edge(P,X), i.e. edges point parent -> child)
//   * Semi-naive evaluation, steps 1-5 of Sec. Background "Semi-Naive Evaluation":
//       1. Delta^0 <- base rule;  Full <- Delta^0.
//       2. iteration i joins Delta^{i-1} with E giving candidates C;
//       3. duplicates are removed from C and Full is subtracted;
//       4. the survivors are Delta^i and are merged into Full;
//       5. stop when Delta^i is empty.
//     The iteration count reported is the index i of the first empty Delta^i
//     (the worked chain a->b->c->d example stops at iteration 3 with |T| = 6).
//     The log holds |Delta^0|, |Delta^1|, ..., |Delta^i| (last entry 0).
//   * Keys are packed (uint64(src) << 32) | dst, so numeric order is the
//     lexicographic (src, dst) order the paper keeps every relation in
//     (Sec. Binary-Search Join, "lexicographically sorted at every stage").
//
// The join looks up the range of edges with a given source in the sorted edge
// array with std::equal_range, the binary-search range lookup of Sec.
// Binary-Search Join.  Full is a std::set<uint64_t>.  Nothing is blocked,
// fused or reordered beyond the five steps above.
//
// oracle_triangles counts the tuples of the non-recursive triangle rule
// (Sec. Generalization, "Triangle Counting") with the same range lookup.
//
// oracle_tc_reach is TC by its plain definition instead of the loop: (x, z) is
// in T exactly when a walk of length >= 1 leads from x to z (the least
// relation closed under the two rules of Sec. Background), found by a
// breadth-first search from every source.  The semi-naive loop adds the pairs
// at shortest walk length k+1 in its iteration k, so the per-length counts are
// the Delta sizes and the longest shortest walk is the iteration count.  It
// reports the closure size, those counts and a digest of the sorted closure
// without storing it (the batched and served benchmarks check every result
// this way): digest = sum over i of mix64(key_i + i * 0x9E3779B97F4A7C15)
// mod 2^64, where key_i is the i-th packed tuple in sorted order and mix64 is
// the output function of SplitMix64 (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014).
//
// oracle_tc_rows runs the same five steps on the rows T(x, .) of chosen
// sources x, one row at a time: the TC recursive rule never changes the first
// component, so row x of T, and row x of every Delta^i, depend only on row x of
// Delta^0 = E(x, .).  Summing the per-row Delta sizes gives the global log.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <set>
#include <thread>
#include <vector>

namespace {

using Key = uint64_t;

inline Key pack(uint32_t s, uint32_t d) { return (Key(s) << 32) | Key(d); }
inline uint32_t src_of(Key k) { return uint32_t(k >> 32); }
inline uint32_t dst_of(Key k) { return uint32_t(k & 0xFFFFFFFFu); }

// E as a sorted array of unique packed keys (set semantics of the input).
std::vector<Key> edge_set(const uint32_t* src, const uint32_t* dst, size_t n) {
  std::set<Key> s;
  for (size_t i = 0; i < n; ++i) s.insert(pack(src[i], dst[i]));
  return std::vector<Key>(s.begin(), s.end());
}

// Range of edges (b, *) in the sorted edge array: binary search on the source.
std::pair<size_t, size_t> edges_from(const std::vector<Key>& E, uint32_t b) {
  auto lo = std::lower_bound(E.begin(), E.end(), pack(b, 0));
  auto hi = std::upper_bound(E.begin(), E.end(), pack(b, 0xFFFFFFFFu));
  return {size_t(lo - E.begin()), size_t(hi - E.begin())};
}

struct Result {
  std::vector<Key> full;        // sorted
  std::vector<uint64_t> log;    // |Delta^0| .. |Delta^iters|
  uint32_t iters = 0;
  int status = 0;               // 0 ok, 1 iteration cap reached
};

// Steps 3-4 of the loop: N = dedup(C) minus Full, then Full <- Full u N.
std::vector<Key> filter_and_merge(std::vector<Key>& C, std::set<Key>& full) {
  std::sort(C.begin(), C.end());
  C.erase(std::unique(C.begin(), C.end()), C.end());
  std::vector<Key> N;
  for (Key c : C)
    if (full.count(c) == 0) N.push_back(c);
  for (Key c : N) full.insert(c);
  return N;
}

// The semi-naive loop (steps 2-5) given Delta^0 = Full^0 = base.
template <class Join>
Result seminaive(std::vector<Key> base, uint32_t max_iters, Join join) {
  Result r;
  std::set<Key> full(base.begin(), base.end());
  std::vector<Key> delta(full.begin(), full.end());
  r.log.push_back(delta.size());
  uint32_t i = 0;
  for (;;) {
    if (i >= max_iters) { r.status = 1; break; }
    ++i;
    std::vector<Key> C;
    for (Key t : delta) join(t, C);
    std::vector<Key> N = filter_and_merge(C, full);
    r.log.push_back(N.size());
    if (N.empty()) break;
    delta.swap(N);
  }
  r.iters = i;
  r.full.assign(full.begin(), full.end());
  return r;
}

Result tc(const std::vector<Key>& E, std::vector<Key> base, uint32_t max_iters) {
  return seminaive(std::move(base), max_iters, [&](Key t, std::vector<Key>& C) {
    // T(x,y), E(y,z) -> T(x,z)
    auto [lo, hi] = edges_from(E, dst_of(t));
    for (size_t j = lo; j < hi; ++j) C.push_back(pack(src_of(t), dst_of(E[j])));
  });
}

std::vector<Key> sg_base(const std::vector<Key>& E) {
  // sg(x,y) <- edge(p,x), edge(p,y), x != y
  std::set<Key> b;
  size_t i = 0;
  while (i < E.size()) {
    size_t j = i;
    while (j < E.size() && src_of(E[j]) == src_of(E[i])) ++j;
    for (size_t a = i; a < j; ++a)
      for (size_t c = i; c < j; ++c)
        if (dst_of(E[a]) != dst_of(E[c])) b.insert(pack(dst_of(E[a]), dst_of(E[c])));
    i = j;
  }
  return std::vector<Key>(b.begin(), b.end());
}

Result sg(const std::vector<Key>& E, uint32_t max_iters) {
  return seminaive(sg_base(E), max_iters, [&](Key t, std::vector<Key>& C) {
    // edge(a,x), sg(a,b), edge(b,y) -> sg(x,y)
    auto [alo, ahi] = edges_from(E, src_of(t));
    auto [blo, bhi] = edges_from(E, dst_of(t));
    for (size_t p = alo; p < ahi; ++p)
      for (size_t q = blo; q < bhi; ++q) C.push_back(pack(dst_of(E[p]), dst_of(E[q])));
  });
}

// Triangle counting (Sec. Generalization, "Triangle Counting"): the number of
// tuples of  triangle(a,b,c) <- edge(a,b), edge(b,c), edge(c,a),  a single
// non-recursive pass.  Each (a,b) in E takes the edges (b,c) from the
// binary-search range lookup and tests edge(c,a) by binary search in E.  The
// edges are split over threads; each thread counts its own share.
uint64_t triangles(const std::vector<Key>& E, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  std::vector<uint64_t> part(n_threads, 0);
  auto work = [&](int t) {
    uint64_t n = 0;
    for (size_t i = t; i < E.size(); i += n_threads) {
      const uint32_t a = src_of(E[i]), b = dst_of(E[i]);
      auto [lo, hi] = edges_from(E, b);
      for (size_t j = lo; j < hi; ++j)
        if (std::binary_search(E.begin(), E.end(), pack(dst_of(E[j]), a))) ++n;
    }
    part[t] = n;
  };
  std::vector<std::thread> ths;
  for (int t = 1; t < n_threads; ++t) ths.emplace_back(work, t);
  work(0);
  for (auto& th : ths) th.join();
  uint64_t n = 0;
  for (uint64_t v : part) n += v;
  return n;
}

inline uint64_t mix64(uint64_t z) {  // SplitMix64 output function
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// TC by reachability.  Vertices are the distinct ids in increasing order; a
// breadth-first search from each source x lists the z reachable by a walk of
// length >= 1 with their shortest walk length.  Pass 1 counts each source's
// row; pass 2 repeats the searches and digests each row at its offset in the
// sorted closure.  Sources are spread over n_threads std::threads.
struct Reach {
  uint64_t n = 0, digest = 0;
  std::vector<uint64_t> by_len;  // by_len[d - 1] = pairs at shortest walk length d
};

Reach tc_reach(const std::vector<Key>& E, int n_threads) {
  std::vector<uint32_t> ids;
  for (Key k : E) { ids.push_back(src_of(k)); ids.push_back(dst_of(k)); }
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  const size_t nv = ids.size();
  auto rank = [&](uint32_t v) { return uint32_t(std::lower_bound(ids.begin(), ids.end(), v) - ids.begin()); };
  std::vector<uint32_t> off(nv + 1, 0), adj(E.size());
  for (Key k : E) off[rank(src_of(k)) + 1]++;
  for (size_t v = 0; v < nv; ++v) off[v + 1] += off[v];
  for (size_t i = 0; i < E.size(); ++i) adj[i] = rank(dst_of(E[i]));  // E sorted: rows in order
  if (n_threads < 1) n_threads = 1;
  std::vector<uint64_t> row(nv, 0), rowoff(nv + 1, 0);
  std::vector<std::vector<uint64_t>> lens(n_threads);
  std::vector<uint64_t> part(n_threads, 0);
  auto search = [&](uint32_t x, std::vector<int32_t>& dist, std::vector<uint32_t>& q) {
    size_t h = 0;
    q.clear();
    for (uint32_t j = off[x]; j < off[x + 1]; ++j)
      if (dist[adj[j]] < 0) { dist[adj[j]] = 1; q.push_back(adj[j]); }
    while (h < q.size()) {
      const uint32_t y = q[h++];
      for (uint32_t j = off[y]; j < off[y + 1]; ++j)
        if (dist[adj[j]] < 0) { dist[adj[j]] = dist[y] + 1; q.push_back(adj[j]); }
    }
  };
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1)
      for (size_t v = 0; v < nv; ++v) rowoff[v + 1] = rowoff[v] + row[v];
    std::vector<std::thread> pool;
    for (int t = 0; t < n_threads; ++t) {
      pool.emplace_back([&, t] {
        std::vector<int32_t> dist(nv, -1);
        std::vector<uint32_t> q;
        for (size_t x = size_t(t); x < nv; x += size_t(n_threads)) {
          search(uint32_t(x), dist, q);
          if (pass == 0) {
            row[x] = q.size();
            for (uint32_t z : q) {
              const size_t d = size_t(dist[z]);
              if (lens[t].size() < d) lens[t].resize(d, 0);
              lens[t][d - 1]++;
            }
          } else {
            std::sort(q.begin(), q.end());  // ranks follow ids: the row's order
            uint64_t i = rowoff[x], h = 0;
            for (uint32_t z : q) h += mix64(pack(ids[x], ids[z]) + (i++) * 0x9E3779B97F4A7C15ull);
            part[t] += h;
          }
          for (uint32_t z : q) dist[z] = -1;
        }
      });
    }
    for (auto& th : pool) th.join();
  }
  Reach r;
  r.n = rowoff[nv];
  for (uint64_t h : part) r.digest += h;
  for (auto& l : lens) {
    if (r.by_len.size() < l.size()) r.by_len.resize(l.size(), 0);
    for (size_t d = 0; d < l.size(); ++d) r.by_len[d] += l[d];
  }
  return r;
}

int export_result(const Result& r, uint64_t** keys, size_t* n_keys, uint64_t** log,
                  size_t* n_log, uint32_t* iters) {
  *n_keys = r.full.size();
  *keys = static_cast<uint64_t*>(std::malloc(sizeof(uint64_t) * (r.full.size() + 1)));
  *n_log = r.log.size();
  *log = static_cast<uint64_t*>(std::malloc(sizeof(uint64_t) * (r.log.size() + 1)));
  if (!*keys || !*log) return -2;
  if (!r.full.empty()) std::memcpy(*keys, r.full.data(), sizeof(uint64_t) * r.full.size());
  std::memcpy(*log, r.log.data(), sizeof(uint64_t) * r.log.size());
  *iters = r.iters;
  return r.status;
}

}  // namespace

extern "C" {

// Transitive closure of the edge set {(src[i], dst[i])}.  Returns 0, or 1 when
// max_iters iterations ran without reaching the fixpoint.  *keys (sorted packed
// tuples) and *log are malloc'd; release them with oracle_free.
int oracle_tc(const uint32_t* src, const uint32_t* dst, size_t n, uint32_t max_iters,
              uint64_t** keys, size_t* n_keys, uint64_t** log, size_t* n_log, uint32_t* iters) {
  std::vector<Key> E = edge_set(src, dst, n);
  return export_result(tc(E, E, max_iters), keys, n_keys, log, n_log, iters);
}

// Same-generation over the edge set (edges point parent -> child).
int oracle_sg(const uint32_t* src, const uint32_t* dst, size_t n, uint32_t max_iters,
              uint64_t** keys, size_t* n_keys, uint64_t** log, size_t* n_log, uint32_t* iters) {
  std::vector<Key> E = edge_set(src, dst, n);
  return export_result(sg(E, max_iters), keys, n_keys, log, n_log, iters);
}

// Rows T(x, .) for the given sources (each row from its own semi-naive loop
// seeded with Delta^0 = E(x, .)), concatenated in the order of `sources`.
// row_len[k] = |T(sources[k], .)|.  log_sum[i] accumulates sum over the given
// rows of |Delta^i restricted to the row| for i < log_cap; *max_iters_out is
// the largest per-row iteration count (0 for a source without out-edges).
// Rows are spread over n_threads std::threads.
int oracle_tc_rows(const uint32_t* src, const uint32_t* dst, size_t n, const uint32_t* sources,
                   size_t n_sources, int n_threads, uint64_t** keys, size_t* n_keys,
                   uint64_t* row_len, uint64_t* log_sum, size_t log_cap, uint32_t* max_iters_out) {
  std::vector<Key> E = edge_set(src, dst, n);
  std::vector<Result> rows(n_sources);
  if (n_threads < 1) n_threads = 1;
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t) {
    pool.emplace_back([&, t] {
      for (size_t k = size_t(t); k < n_sources; k += size_t(n_threads)) {
        auto [lo, hi] = edges_from(E, sources[k]);
        std::vector<Key> base(E.begin() + lo, E.begin() + hi);
        if (base.empty()) continue;  // the row never enters the loop
        rows[k] = tc(E, std::move(base), 0xFFFFFFFFu);
      }
    });
  }
  for (auto& th : pool) th.join();
  size_t total = 0;
  for (auto& r : rows) total += r.full.size();
  *n_keys = total;
  *keys = static_cast<uint64_t*>(std::malloc(sizeof(uint64_t) * (total + 1)));
  if (!*keys) return -2;
  uint32_t mx = 0;
  size_t at = 0;
  for (size_t k = 0; k < n_sources; ++k) {
    const Result& r = rows[k];
    row_len[k] = r.full.size();
    if (!r.full.empty()) std::memcpy(*keys + at, r.full.data(), sizeof(uint64_t) * r.full.size());
    at += r.full.size();
    for (size_t i = 0; i < r.log.size() && i < log_cap; ++i) log_sum[i] += r.log[i];
    mx = std::max(mx, r.iters);
  }
  *max_iters_out = mx;
  return 0;
}

// TC by reachability (see tc_reach): *n_tuples, *iters (the index of the
// first empty Delta, as oracle_tc reports it), log[0..*n_log) = |Delta^0| ..
// |Delta^iters| (at most log_cap entries are written) and the digest of the
// sorted closure.
int oracle_tc_reach(const uint32_t* src, const uint32_t* dst, size_t n, int n_threads,
                    uint64_t* n_tuples, uint32_t* iters, uint64_t* log, size_t log_cap,
                    size_t* n_log, uint64_t* digest) {
  const Reach r = tc_reach(edge_set(src, dst, n), n_threads);
  *n_tuples = r.n;
  *digest = r.digest;
  // Delta^k = pairs at shortest walk length k + 1; the loop stops at the
  // first empty one (at least iteration 1)
  const size_t it = std::max<size_t>(1, r.by_len.size());
  *iters = uint32_t(it);
  *n_log = it + 1;
  for (size_t k = 0; k <= it && k < log_cap; ++k) log[k] = k < r.by_len.size() ? r.by_len[k] : 0;
  return 0;
}

void oracle_free(void* p) { std::free(p); }

// Number of tuples of triangle(a,b,c) over the edge set {(src[i], dst[i])}.
uint64_t oracle_triangles(const uint32_t* src, const uint32_t* dst, size_t n, int n_threads) {
  return triangles(edge_set(src, dst, n), n_threads);
}

}  // extern "C"
