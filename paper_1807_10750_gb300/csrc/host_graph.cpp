// Host-side layout builder (see host_graph.h).
//
// The problem statement is the max-cut instance of Sec. III (Eq. 4) on a
// general graph (Sec. II-A: arbitrary connections). Repeated edges are merged by
// summing their weights and a merged weight of 0 is dropped (the paper is
// silent; a zero weight couples nothing). Self-loops are rejected: they only
// add a constant to the energy and can never be cut.
//
// Deterministic sweeps need a colouring (the checkerboard of Sec. IV-B, made
// general): greedy first fit over the vertices in order of decreasing degree,
// ties broken by smaller id (Welsh-Powell), in two tiers. Vertices with at
// least ISING_HUB_DEGREE distinct neighbours (hubs) lead that order and are
// coloured among themselves; every later vertex takes the smallest colour at
// or above the hubs' colour count, so hub classes hold hubs only and come
// first in the sweep. On a regular graph such as an even torus there are no
// hubs and the order is natural order, which gives the checkerboard.
#include "host_graph.h"
#include "host_parallel.h"

#include <algorithm>
#include <cstdlib>
#include <limits>
#include <memory>
#include <new>

#include "../../include/ising.h"

namespace isingx {

namespace {

// A reusable barrier for a fixed set of threads (spinning, then yielding:
// the waits between colouring levels are short).
class SpinBarrier {
 public:
  explicit SpinBarrier(int n) : n_(n) {}
  void wait() {
    const int gen = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) == n_ - 1) {
      count_.store(0, std::memory_order_relaxed);
      gen_.store(gen + 1, std::memory_order_release);
      return;
    }
    for (int spin = 0; gen_.load(std::memory_order_acquire) == gen; ++spin)
      if (spin > 4096) std::this_thread::yield();
  }

 private:
  const int n_;
  std::atomic<int> count_{0};
  std::atomic<int> gen_{0};
};

// First-fit colours of the two tiers, relative to each tier (the hubs from 0,
// the other vertices from 0: the caller adds the hubs' colour count), equal to
// the sequential first fit in `order`. A vertex's colour depends only on the
// colours of its same-tier neighbours earlier in the order.
//
// The hubs, the order's first vertices, are close to a clique on a power-law
// graph: their dependencies form a chain hundreds of levels deep with one or
// two hubs per level. So every hub's earlier hub neighbours are listed first
// (all threads, by rank), and one thread then colours the hubs in order from
// those lists.
//
// The other vertices are coloured level by level: a vertex joins the next
// level when its last earlier same-tier neighbour has been coloured (a
// per-vertex countdown), and the threads split each level. Each such row is
// first partitioned in place (neighbours with their weights): earlier
// same-tier neighbours, then later same-tier ones, then the hubs, so a level
// reads only the entries it needs. The rows' order is otherwise free: the
// colour-ordered CSR sorts them again. Returns false (nothing written) when
// no helper thread could be started; the caller then colours sequentially.
bool colour_levels(size_t N, const int64_t* moff, int32_t* mnb, int32_t* mwt, const int32_t* deg,
                   const std::vector<int32_t>& order, int32_t maxdeg, int32_t* rel) {
  const int T = host_threads();
  if (T <= 1) return false;
  std::vector<int32_t> rank(N);
  parallel_ranges((int64_t)N, 1 << 16, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) rank[(size_t)order[(size_t)i]] = (int32_t)i;
  });
  auto hub = [&](size_t v) { return deg[v] >= kHubDegree; };
  // the hub tier: the hubs hold ranks [0, X)
  size_t X = 0;
  while (X < N && hub((size_t)order[X])) ++X;
  if (X > 0) {
    std::vector<int64_t> hoff(X + 1, 0);  // the hubs' row lengths in rank order, for the split
    for (size_t i = 0; i < X; ++i) {
      const size_t v = (size_t)order[i];
      hoff[i + 1] = hoff[i] + (moff[v + 1] - moff[v]);
    }
    std::vector<std::vector<int32_t>> earlier(X);
    parallel_rows((int64_t)X, hoff.data(), [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        const size_t v = (size_t)order[(size_t)i];
        std::vector<int32_t>& e = earlier[(size_t)i];
        for (int64_t k = moff[v]; k < moff[v + 1]; ++k) {
          const int32_t r = rank[(size_t)mnb[(size_t)k]];
          if (r < i) e.push_back(r);  // a rank below i < X is a hub's
        }
      }
    });
    std::vector<int32_t> hc(X), mark((size_t)maxdeg + 2, -1);
    for (size_t i = 0; i < X; ++i) {
      const int32_t d = deg[(size_t)order[i]];
      for (const int32_t r : earlier[i])
        if (hc[(size_t)r] <= d) mark[(size_t)hc[(size_t)r]] = (int32_t)i;
      int32_t c = 0;
      while (mark[(size_t)c] == (int32_t)i) ++c;
      hc[i] = c;
      rel[(size_t)order[i]] = c;
    }
  }
  // the other tier: rows partitioned (earlier | later same-tier | hubs) and
  // countdowns of earlier same-tier neighbours
  std::unique_ptr<std::atomic<int32_t>[]> pending(new std::atomic<int32_t>[N]);
  std::vector<int32_t> n_earlier(N, 0), n_later(N, 0);  // per row: the first two parts' lengths
  parallel_ranges((int64_t)N, 1 << 14, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v) {
      int32_t c = -1;  // a hub: coloured above
      if (!hub((size_t)v)) {
        const int32_t rv = rank[(size_t)v];
        int64_t i = moff[v], lt = moff[v], gt = moff[v + 1];
        while (i < gt) {
          const int32_t u = mnb[(size_t)i];
          if (hub((size_t)u)) {
            --gt;
            std::swap(mnb[(size_t)i], mnb[(size_t)gt]);
            std::swap(mwt[(size_t)i], mwt[(size_t)gt]);
          } else if (rank[(size_t)u] < rv) {
            std::swap(mnb[(size_t)i], mnb[(size_t)lt]);
            std::swap(mwt[(size_t)i], mwt[(size_t)lt]);
            ++lt;
            ++i;
          } else {
            ++i;
          }
        }
        c = (int32_t)(lt - moff[v]);
        n_earlier[(size_t)v] = c;
        n_later[(size_t)v] = (int32_t)(gt - lt);
      }
      pending[(size_t)v].store(c, std::memory_order_relaxed);
    }
  });
  std::vector<int32_t> frontier;
  for (size_t v = 0; v < N; ++v)
    if (pending[v].load(std::memory_order_relaxed) == 0) frontier.push_back((int32_t)v);
  std::vector<std::vector<int32_t>> next((size_t)T);
  std::vector<int64_t> cum;               // the frontier's degrees, running sum
  auto rebuild_cum = [&] {
    cum.resize(frontier.size() + 1);
    cum[0] = 0;
    for (size_t i = 0; i < frontier.size(); ++i) cum[i + 1] = cum[i] + deg[frontier[i]] + 1;
  };
  rebuild_cum();
  int P = 1;                              // threads taking part (set before any starts work)
  std::unique_ptr<SpinBarrier> barrier_p;
  bool done = frontier.empty();
  auto work = [&](int t) {
    SpinBarrier& barrier = *barrier_p;
    std::vector<int32_t> mark((size_t)maxdeg + 2, -1);
    while (!done) {
      // this level's vertices, split by their entry counts: each is coloured
      // from its earlier same-tier neighbours (all final) and releases its
      // later same-tier neighbours (coloured from the next level on)
      const int64_t total = cum.back();
      const size_t lo = (size_t)(std::lower_bound(cum.begin(), cum.end(), total * t / P) - cum.begin());
      const size_t hi = (size_t)(std::lower_bound(cum.begin(), cum.end(), total * (t + 1) / P) - cum.begin());
      std::vector<int32_t>& out = next[(size_t)t];
      out.clear();
      for (size_t i = lo; i < hi && i < frontier.size(); ++i) {
        const int32_t v = frontier[i];
        const int32_t d = deg[v];
        const int64_t k0 = moff[v];
        const int64_t ke = k0 + n_earlier[(size_t)v];
        for (int64_t k = k0; k < ke; ++k) {
          const int32_t u = mnb[(size_t)k];
          if (rel[u] <= d) mark[(size_t)rel[u]] = v;
        }
        const int64_t kl = ke + n_later[(size_t)v];
        for (int64_t k = ke; k < kl; ++k) {
          const int32_t u = mnb[(size_t)k];
          if (pending[(size_t)u].fetch_sub(1, std::memory_order_relaxed) == 1) out.push_back(u);
        }
        int32_t c = 0;
        while (mark[(size_t)c] == v) ++c;
        rel[v] = c;
      }
      barrier.wait();  // this level's colours are final and its releases counted
      if (t == 0) {
        size_t F = 0;
        for (int j = 0; j < P; ++j) F += next[(size_t)j].size();
        frontier.resize(F);
        F = 0;
        for (int j = 0; j < P; ++j) {
          std::copy(next[(size_t)j].begin(), next[(size_t)j].end(), frontier.begin() + (std::ptrdiff_t)F);
          F += next[(size_t)j].size();
        }
        rebuild_cum();
        done = frontier.empty();
      }
      barrier.wait();  // the next level is in place
    }
  };
  // helpers wait for the gate; the barrier counts the threads that started
  std::atomic<int> gate{0};
  auto helper = [&](int t) {
    while (gate.load(std::memory_order_acquire) == 0) std::this_thread::yield();
    work(t);
  };
  std::vector<std::thread> pool;
  try {
    pool.reserve((size_t)T - 1);
    for (int t = 1; t < T; ++t) pool.emplace_back(helper, t);
  } catch (const std::system_error&) {
  } catch (const std::bad_alloc&) {
  }
  P = 1 + (int)pool.size();
  barrier_p.reset(new SpinBarrier(P));
  gate.store(1, std::memory_order_release);
  work(0);
  for (std::thread& th : pool) th.join();
  return true;
}

}  // namespace

int build_host_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     const int32_t* w, HostGraph* out) {
  if (out == nullptr || n <= 0 || m < 0) return ISING_EINVAL;
  if (m >= (int64_t(1) << 30)) return ISING_ERANGE;
  if (m > 0 && (src == nullptr || dst == nullptr || w == nullptr)) return ISING_EINVAL;
  constexpr int64_t kGrain = 1 << 18;  // indices per block: smaller graphs stay on one thread
  std::atomic<bool> bad(false);
  parallel_ranges(m, kGrain, [&](int64_t lo, int64_t hi) {
    for (int64_t e = lo; e < hi; ++e) {
      const int32_t u = src[e], v = dst[e];
      if (u < 0 || u >= n || v < 0 || v >= n || u == v) {
        bad.store(true, std::memory_order_relaxed);
        return;
      }
    }
  });
  if (bad.load()) return ISING_EINVAL;
  HostGraph& g = *out;
  g = HostGraph();
  g.n = n;
  const size_t N = (size_t)n;

  // Directed rows: every edge (u, v, w) becomes the entries v of row u and u
  // of row v, each held as the key (neighbour << 32) | (uint32) w; sorting
  // each row's keys then orders it by neighbour (then weight), so repeated
  // neighbours are adjacent. A row's entries arrive in edge order.
  //
  // On several threads, when a counter per part and vertex fits in 2^26
  // words: part t takes the edges [m t / P, m (t + 1) / P), counts its
  // entries per row, the counts become each part's first slot in every row,
  // and every part fills its own slots (each edge read twice in all).
  // Otherwise each thread owns a contiguous range of rows, scans every edge
  // and fills only its own rows.
  const int64_t parts = m >= 2 * kGrain ? host_threads() : 1;
  std::vector<int64_t> off(N + 1, 0);
  std::unique_ptr<uint64_t[]> key;  // scratch, left uninitialised (every slot is written before it is read)
  if (parts > 1 && (uint64_t)parts * N <= (uint64_t(1) << 26)) {
    auto edge_lo = [&](int64_t t) { return m * t / parts; };
    std::unique_ptr<int32_t[]> cur(new int32_t[(size_t)parts * N]);
    parallel_ranges(parts, 1, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        int32_t* c = cur.get() + (size_t)t * N;
        std::fill(c, c + N, 0);
        for (int64_t e = edge_lo(t); e < edge_lo(t + 1); ++e) {
          ++c[(size_t)src[e]];
          ++c[(size_t)dst[e]];
        }
      }
    });
    parallel_ranges((int64_t)N, 1 << 14, [&](int64_t lo, int64_t hi) {
      for (int64_t v = lo; v < hi; ++v) {
        int64_t len = 0;
        for (int64_t t = 0; t < parts; ++t) len += cur[(size_t)t * N + (size_t)v];
        off[(size_t)v + 1] = len;
      }
    });
    for (size_t i = 0; i < N; ++i) off[i + 1] += off[i];
    // each part's first slot in every row (below 2m < 2^31)
    parallel_ranges((int64_t)N, 1 << 14, [&](int64_t lo, int64_t hi) {
      for (int64_t v = lo; v < hi; ++v) {
        int64_t run = off[(size_t)v];
        for (int64_t t = 0; t < parts; ++t) {
          const int32_t c = cur[(size_t)t * N + (size_t)v];
          cur[(size_t)t * N + (size_t)v] = (int32_t)run;
          run += c;
        }
      }
    });
    key.reset(new uint64_t[std::max<size_t>((size_t)off[N], 1)]);
    parallel_ranges(parts, 1, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        int32_t* c = cur.get() + (size_t)t * N;
        for (int64_t e = edge_lo(t); e < edge_lo(t + 1); ++e) {
          const uint32_t u = (uint32_t)src[e], v = (uint32_t)dst[e], wt = (uint32_t)w[e];
          key[(size_t)c[u]++] = ((uint64_t)v << 32) | wt;
          key[(size_t)c[v]++] = ((uint64_t)u << 32) | wt;
        }
      }
    });
  } else {
    auto part_lo = [&](int64_t t) { return (int64_t)N * t / parts; };
    parallel_ranges(parts, 1, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        const uint32_t lo = (uint32_t)part_lo(t), span = (uint32_t)(part_lo(t + 1) - part_lo(t));
        for (int64_t e = 0; e < m; ++e) {
          const uint32_t u = (uint32_t)src[e], v = (uint32_t)dst[e];
          if (u - lo < span) ++off[(size_t)u + 1];
          if (v - lo < span) ++off[(size_t)v + 1];
        }
      }
    });
    for (size_t i = 0; i < N; ++i) off[i + 1] += off[i];
    key.reset(new uint64_t[std::max<size_t>((size_t)off[N], 1)]);
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    parallel_ranges(parts, 1, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        const uint32_t lo = (uint32_t)part_lo(t), span = (uint32_t)(part_lo(t + 1) - part_lo(t));
        for (int64_t e = 0; e < m; ++e) {
          const uint32_t u = (uint32_t)src[e], v = (uint32_t)dst[e], wt = (uint32_t)w[e];
          if (u - lo < span) key[(size_t)fill[u]++] = ((uint64_t)v << 32) | wt;
          if (v - lo < span) key[(size_t)fill[v]++] = ((uint64_t)u << 32) | wt;
        }
      }
    });
  }

  // Merge repeated neighbours, drop zero sums, bound every field. Each row's
  // merged entries are written over the front of its own key range.
  std::vector<int32_t> mdeg(N, 0);
  std::atomic<bool> too_wide(false), not8(false);
  std::atomic<int64_t> total_directed(0);
  parallel_rows((int64_t)N, off.data(), [&](int64_t lo, int64_t hi) {
    int64_t total = 0;
    bool over = false, wide8 = false;
    for (int64_t u = lo; u < hi && !over; ++u) {
      uint64_t* row = key.get() + off[(size_t)u];
      const int64_t len = off[(size_t)u + 1] - off[(size_t)u];
      std::sort(row, row + len);
      int64_t k = 0, out_k = 0, abs_sum = 0;
      while (k < len) {
        const uint32_t v = (uint32_t)(row[k] >> 32);
        int64_t s = 0;
        while (k < len && (uint32_t)(row[k] >> 32) == v) {
          s += (int32_t)(uint32_t)row[k];
          ++k;
        }
        if (s == 0) continue;
        abs_sum += s < 0 ? -s : s;
        if (abs_sum > (int64_t)std::numeric_limits<int32_t>::max()) {
          over = true;
          break;
        }
        if (s > 127 || s < -127) wide8 = true;
        row[out_k++] = ((uint64_t)v << 32) | (uint32_t)(int32_t)s;
        total += s;
      }
      mdeg[(size_t)u] = (int32_t)out_k;
    }
    if (over) too_wide.store(true, std::memory_order_relaxed);
    if (wide8) not8.store(true, std::memory_order_relaxed);
    total_directed.fetch_add(total, std::memory_order_relaxed);
  });
  if (too_wide.load()) return ISING_ERANGE;
  std::vector<int64_t> moff(N + 1, 0);
  int32_t maxdeg = 0;
  for (size_t u = 0; u < N; ++u) {
    moff[u + 1] = moff[u] + mdeg[u];
    maxdeg = std::max(maxdeg, mdeg[u]);
  }
  std::unique_ptr<int32_t[]> mnb(new int32_t[std::max<int64_t>(moff[N], 1)]);
  std::unique_ptr<int32_t[]> mwt(new int32_t[std::max<int64_t>(moff[N], 1)]);
  parallel_rows((int64_t)N, moff.data(), [&](int64_t lo, int64_t hi) {
    for (int64_t u = lo; u < hi; ++u) {
      const uint64_t* row = key.get() + off[(size_t)u];
      for (int64_t k = 0; k < mdeg[(size_t)u]; ++k) {
        mnb[(size_t)(moff[(size_t)u] + k)] = (int32_t)(row[k] >> 32);
        mwt[(size_t)(moff[(size_t)u] + k)] = (int32_t)(uint32_t)row[k];
      }
    }
  });
  g.nnz = moff[N];
  g.num_edges = g.nnz / 2;
  g.total_weight = total_directed.load() / 2;
  g.fits_int8 = !not8.load();
  g.max_degree = maxdeg;

  // Welsh-Powell order: degree descending, id ascending (bucketed by degree).
  auto degree = [&](size_t v) { return mdeg[v]; };
  std::vector<int32_t> order(N);
  {
    std::vector<int64_t> bucket((size_t)maxdeg + 2, 0);
    for (size_t v = 0; v < N; ++v) bucket[(size_t)(maxdeg - degree(v)) + 1]++;
    for (size_t d = 0; d + 1 < bucket.size(); ++d) bucket[d + 1] += bucket[d];
    for (size_t v = 0; v < N; ++v) order[(size_t)bucket[(size_t)(maxdeg - degree(v))]++] = (int32_t)v;
  }
  // First-fit colouring in two tiers. The hubs come first in the order; once
  // the order reaches a non-hub, colours are counted from `base`, the hubs'
  // colour count, and the (smaller) colours of hub neighbours are ignored.
  g.colour.assign(N, -1);
  // large graphs (8M entries and more; smaller ones colour in a few ms):
  // level by level on several threads, the same colours
  if (moff[N] >= (int64_t(1) << 23) &&
      colour_levels(N, moff.data(), mnb.get(), mwt.get(), mdeg.data(), order, maxdeg, g.colour.data())) {
    int32_t hubs = 0, hub_c = 0, other_c = -1;
    for (size_t v = 0; v < N; ++v) {
      if (degree(v) >= kHubDegree) {
        ++hubs;
        hub_c = std::max(hub_c, g.colour[v] + 1);
      } else {
        other_c = std::max(other_c, g.colour[v]);
      }
    }
    for (size_t v = 0; v < N; ++v)
      if (degree(v) < kHubDegree) g.colour[v] += hub_c;
    g.num_hubs = hubs;
    g.hub_colours = hub_c;
    g.num_colours = hub_c + other_c + 1;
  } else {
    std::vector<int32_t> mark((size_t)maxdeg + 2, -1);
    int32_t C = 0, base = 0;
    bool hubs = true;
    for (size_t i = 0; i < N; ++i) {
      const int32_t v = order[i];
      const int32_t d = degree((size_t)v);
      if (hubs && d < kHubDegree) {
        hubs = false;
        base = C;
        g.hub_colours = C;
        g.num_hubs = (int32_t)i;
      }
      for (int64_t k = moff[(size_t)v]; k < moff[(size_t)v + 1]; ++k) {
        const int32_t c = g.colour[(size_t)mnb[(size_t)k]] - base;
        if (c >= 0 && c <= d) mark[(size_t)c] = v;
      }
      int32_t c = 0;
      while (mark[(size_t)c] == v) ++c;
      g.colour[(size_t)v] = base + c;
      C = std::max(C, base + c + 1);
    }
    if (hubs) {  // every vertex is a hub
      g.hub_colours = C;
      g.num_hubs = (int32_t)N;
    }
    g.num_colours = C;
  }
  // Positions: by colour, then the Welsh-Powell order (degree desc, id asc).
  const size_t C = (size_t)g.num_colours;
  g.class_begin.assign(C + 1, 0);
  for (size_t v = 0; v < N; ++v) g.class_begin[(size_t)g.colour[v] + 1]++;
  for (size_t c = 0; c < C; ++c) g.class_begin[c + 1] += g.class_begin[c];
  g.perm.assign(N, 0);
  g.pos.assign(N, 0);
  {
    std::vector<int32_t> fill(g.class_begin.begin(), g.class_begin.end() - 1);
    for (int32_t v : order) {
      int32_t p = fill[(size_t)g.colour[(size_t)v]]++;
      g.perm[(size_t)p] = v;
      g.pos[(size_t)v] = p;
    }
  }
  // Colour-ordered CSR with each row sorted by neighbour position: row p
  // lists vertex perm[p]'s neighbours as (position << 32) | weight keys,
  // sorted (positions in a row are distinct), in the key buffer's front.
  g.row_ptr.assign(N + 1, 0);
  for (size_t p = 0; p < N; ++p) g.row_ptr[p + 1] = g.row_ptr[p] + degree((size_t)g.perm[p]);
  g.col.resize((size_t)g.nnz);  // every entry is written below
  g.w.resize((size_t)g.nnz);
  parallel_rows((int64_t)N, g.row_ptr.data(), [&](int64_t lo, int64_t hi) {
    for (int64_t p = lo; p < hi; ++p) {
      const size_t x = (size_t)g.perm[(size_t)p];
      uint64_t* row = key.get() + g.row_ptr[(size_t)p];
      const int64_t len = moff[x + 1] - moff[x];
      for (int64_t k = 0; k < len; ++k)
        row[k] = ((uint64_t)(uint32_t)g.pos[(size_t)mnb[(size_t)(moff[x] + k)]] << 32) |
                 (uint32_t)mwt[(size_t)(moff[x] + k)];
      std::sort(row, row + len);
      for (int64_t k = 0; k < len; ++k) {
        g.col[(size_t)(g.row_ptr[(size_t)p] + k)] = (int32_t)(row[k] >> 32);
        g.w[(size_t)(g.row_ptr[(size_t)p] + k)] = (int32_t)(uint32_t)row[k];
      }
    }
  });
  return ISING_OK;
}

void build_work_plan(const HostGraph& g, int32_t target_warps, int32_t min_edges,
                     int32_t max_rows, int32_t light_slots, WorkPlan* plan) {
  plan->items.clear();
  plan->split_parts.clear();
  plan->ell_col.clear();
  plan->ell_w.clear();
  plan->class_item_begin.assign((size_t)g.num_colours + 1, 0);
  plan->max_class_items = 0;
  if (target_warps < 1) target_warps = 1;
  if (min_edges < light_slots) min_edges = light_slots;
  if (max_rows < 1) max_rows = 1;
  auto degree = [&](int32_t v) { return (int64_t)g.row_ptr[(size_t)v + 1] - g.row_ptr[(size_t)v]; };
  std::vector<int32_t> light;  // the light items, filled after the split
  int64_t ell_words = 0;
  for (int32_t c = 0; c < g.num_colours; ++c) {
    const int32_t vb = g.class_begin[(size_t)c], ve = g.class_begin[(size_t)c + 1];
    const int64_t E = (int64_t)g.row_ptr[(size_t)ve] - g.row_ptr[(size_t)vb];
    const int64_t L = std::max<int64_t>(min_edges, (E + target_warps - 1) / target_warps);
    int32_t v = vb;
    while (v < ve) {
      const int64_t d = degree(v);
      if (d > L) {
        // at most 65535 slices per row (the packed combine counts them in 16 bits)
        const int64_t parts = std::min<int64_t>((d + L - 1) / L, 65535);
        const int64_t chunk = (d + parts - 1) / parts;
        const int32_t slot = (int32_t)plan->split_parts.size();
        plan->split_parts.push_back((int32_t)parts);
        const int64_t e0 = g.row_ptr[(size_t)v];
        for (int64_t k = 0; k < parts; ++k) {
          const int64_t a0 = e0 + k * chunk;
          const int64_t b0 = std::min<int64_t>(e0 + d, a0 + chunk);
          plan->items.push_back({v, -(slot + 1), (int32_t)a0, (int32_t)b0});
        }
        ++v;
        continue;
      }
      if (d > light_slots) {
        // group item: CSR rows until the edge budget, the row cap, or the
        // first light row
        int32_t end = v;
        int64_t edges = 0;
        while (end < ve && end - v < max_rows && degree(end) > light_slots &&
               (end == v || edges + degree(end) <= L)) {
          edges += degree(end);
          ++end;
        }
        plan->items.push_back({v, end, g.row_ptr[(size_t)v], g.row_ptr[(size_t)end]});
        v = end;
        continue;
      }
      // light item: the widest row is the first (degree order)
      const int32_t D = (int32_t)d;
      const int32_t R = D <= light_slots / 4 ? 4 : (D <= light_slots / 2 ? 2 : 1);
      int32_t end = v;
      int64_t edges = 0;
      while (end < ve && end - v < 32 * R && (end == v || edges + degree(end) <= L)) {
        edges += degree(end);
        ++end;
      }
      const int32_t nv = end - v;
      light.push_back((int32_t)plan->items.size());
      plan->items.push_back({v, end, (int32_t)ell_words, -(D + 1)});
      ell_words += (int64_t)D * nv;
      v = end;
    }
    plan->class_item_begin[(size_t)c + 1] = (int32_t)plan->items.size();
    plan->max_class_items = std::max<int32_t>(
        plan->max_class_items,
        plan->class_item_begin[(size_t)c + 1] - plan->class_item_begin[(size_t)c]);
  }
  // Sliced ELL of the light items: slot k of row r of an item with nv rows
  // at word off is word off + k * nv + r; slots past a row's degree keep
  // (-1, 0). Items own disjoint word ranges.
  plan->ell_col.assign((size_t)ell_words, -1);
  plan->ell_w.assign((size_t)ell_words, 0);
  parallel_ranges((int64_t)light.size(), 1024, [&](int64_t lo, int64_t hi) {
    for (int64_t q = lo; q < hi; ++q) {
      const WorkItem& it = plan->items[(size_t)light[(size_t)q]];
      const int32_t nv = it.v_end - it.v_begin;
      const int64_t off = it.e_begin;
      for (int32_t r = 0; r < nv; ++r) {
        const int64_t rb = g.row_ptr[(size_t)(it.v_begin + r)];
        const int64_t deg = degree(it.v_begin + r);
        for (int64_t k = 0; k < deg; ++k) {
          plan->ell_col[(size_t)(off + k * nv + r)] = g.col[(size_t)(rb + k)];
          plan->ell_w[(size_t)(off + k * nv + r)] = g.w[(size_t)(rb + k)];
        }
      }
    }
  });
}

bool build_item_deps(const HostGraph& g, const WorkPlan& plan, std::vector<int32_t>* dep_ptr,
                     std::vector<int32_t>* deps) {
  dep_ptr->clear();
  deps->clear();
  const int32_t ni = (int32_t)plan.items.size();
  std::vector<int32_t> item_of((size_t)g.n, -1), class_of((size_t)ni, 0);
  for (int32_t c = 0; c < g.num_colours; ++c)
    for (int32_t i = plan.class_item_begin[(size_t)c]; i < plan.class_item_begin[(size_t)c + 1]; ++i)
      class_of[(size_t)i] = c;
  for (int32_t i = 0; i < ni; ++i) {
    const WorkItem& it = plan.items[(size_t)i];
    if (it.v_end < 0) return false;  // a slice of a heavy row
    for (int32_t v = it.v_begin; v < it.v_end; ++v) item_of[(size_t)v] = i;
  }
  // Items in contiguous blocks, one per thread, each with its own marker
  // array: seen[j] == i + 1 marks j as already listed for item i. The blocks'
  // lists are joined in item order, so the result does not depend on the
  // number of threads.
  const int32_t threads = g.nnz < (int64_t(1) << 19) ? 1 : host_threads();
  const int64_t grain = std::max<int64_t>(1, ((int64_t)ni + threads - 1) / threads);
  std::vector<std::vector<int32_t>> block_deps, block_cnt;
  const int64_t nblocks = ni == 0 ? 0 : ((int64_t)ni + grain - 1) / grain;
  block_deps.resize((size_t)nblocks);
  block_cnt.resize((size_t)nblocks);
  std::atomic<bool> no_memory(false);  // an allocation failed in a worker
  parallel_ranges(nblocks, 1, [&](int64_t b0, int64_t b1) {
    try {
      std::vector<int32_t> seen((size_t)ni, 0);
      for (int64_t b = b0; b < b1; ++b) {
        std::vector<int32_t>& out = block_deps[(size_t)b];
        std::vector<int32_t>& cnt = block_cnt[(size_t)b];
        for (int64_t i = b * grain; i < std::min<int64_t>(ni, (b + 1) * grain); ++i) {
          const WorkItem& it = plan.items[(size_t)i];
          const size_t before = out.size();
          for (int32_t v = it.v_begin; v < it.v_end; ++v)
            for (int32_t k = g.row_ptr[(size_t)v]; k < g.row_ptr[(size_t)v + 1]; ++k) {
              const int32_t j = item_of[(size_t)g.col[(size_t)k]];
              if (j == i || seen[(size_t)j] == i + 1) continue;
              seen[(size_t)j] = (int32_t)i + 1;
              out.push_back((j << 1) | (class_of[(size_t)j] > class_of[(size_t)i] ? 1 : 0));
            }
          cnt.push_back((int32_t)(out.size() - before));
        }
      }
    } catch (const std::bad_alloc&) {
      no_memory.store(true);
    }
  });
  if (no_memory.load()) throw std::bad_alloc();
  dep_ptr->reserve((size_t)ni + 1);
  dep_ptr->push_back(0);
  for (int64_t b = 0; b < nblocks; ++b) {
    for (int32_t c : block_cnt[(size_t)b]) dep_ptr->push_back(dep_ptr->back() + c);
    deps->insert(deps->end(), block_deps[(size_t)b].begin(), block_deps[(size_t)b].end());
  }
  return true;
}

void build_block_plan(const HostGraph& g, BlockPlan* bp) {
  *bp = BlockPlan();
  const int32_t C = g.num_colours;
  if (!g.fits_int8 || g.n > kBlockMaxVertices || C > kBlockMaxClasses) return;
  bp->class_chunk.push_back(0);
  for (int32_t c = 0; c < C; ++c) {
    const int64_t start = (int64_t)bp->words.size();
    for (int32_t v = g.class_begin[(size_t)c]; v < g.class_begin[(size_t)c + 1]; ++v)
      for (int32_t k = g.row_ptr[(size_t)v]; k < g.row_ptr[(size_t)v + 1]; ++k)
        bp->words.push_back((int32_t)(((uint32_t)v << 20) | ((uint32_t)g.col[(size_t)k] << 8) |
                                      ((uint32_t)g.w[(size_t)k] & 0xffu)));
    while (bp->words.size() % 4 != 0) bp->words.push_back((int32_t)((uint32_t)g.n << 20));
    const int64_t end = (int64_t)bp->words.size();
    for (int64_t a = start; a < end; a += kBlockChunkWords) {
      bp->chunk_off.push_back((int32_t)a);
      bp->chunk_len.push_back((int32_t)std::min<int64_t>(kBlockChunkWords, end - a));
    }
    bp->class_chunk.push_back((int32_t)bp->chunk_off.size());
    if ((int32_t)bp->chunk_off.size() > kBlockMaxChunks) {
      *bp = BlockPlan();
      return;
    }
  }
  bp->ok = true;
}

}  // namespace isingx
