// Host-side plan of the halo engine (see host_graph.h): parts by recursive
// breadth-first bisection, each part's D-hop region, and its sliced-ELL rows
// over local indices.
//
// The sweep order is the one every engine follows (Algorithm 2 over greedy
// colour classes, classes in increasing order): a vertex of class c in sweep t
// sees its earlier-class neighbours after their sweep-t update and its
// later-class neighbours after their sweep t - 1 update. A block that holds
// every vertex within D hops of its part can run D phases alone: phase j
// updates the class-(j - 1) mod K vertices at most D - j hops out, and each of
// their neighbours (at most D - j + 1 hops out) was current after phase j - 1.
// After D phases the part itself is current.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <memory>
#include <thread>
#include <vector>

#include "host_graph.h"

namespace isingx {

namespace {

// Runs fn(i) for i in [0, count) on up to `threads` threads.
template <typename Fn>
void parallel_for(int32_t count, int32_t threads, Fn fn) {
  threads = std::max<int32_t>(1, std::min(threads, count));
  if (threads == 1) {
    for (int32_t i = 0; i < count; ++i) fn(i, 0);
    return;
  }
  std::atomic<int32_t> next(0);
  std::vector<std::thread> pool;
  for (int32_t w = 0; w < threads; ++w)
    pool.emplace_back([&, w] {
      for (int32_t i = next.fetch_add(1); i < count; i = next.fetch_add(1)) fn(i, w);
    });
  for (std::thread& t : pool) t.join();
}

int32_t plan_threads() {
  const unsigned hw = std::thread::hardware_concurrency();
  return static_cast<int32_t>(std::max(1u, std::min(hw == 0 ? 1u : hw, 16u)));
}

}  // namespace

static bool cancelled(const std::atomic<bool>* cancel) {
  return cancel != nullptr && cancel->load(std::memory_order_relaxed);
}

void bisect_parts(const HostGraph& g, int32_t parts, std::vector<int32_t>* part,
                  const std::atomic<bool>* cancel) {
  const int32_t n = g.n;
  part->assign(static_cast<size_t>(n), 0);
  if (parts <= 1 || n == 0) return;
  // mark[v] = id while v is an unvisited member of subset id, -id once the
  // subset's breadth-first pass reached it. Subsets of one level are disjoint
  // and handled by different threads; a pass only compares a neighbour's mark
  // with its own id, which no other thread writes.
  std::unique_ptr<std::atomic<int32_t>[]> mark(new std::atomic<int32_t>[static_cast<size_t>(n)]);
  for (int32_t v = 0; v < n; ++v) mark[static_cast<size_t>(v)].store(1, std::memory_order_relaxed);
  auto bfs = [&](int32_t s, int32_t id, std::vector<int32_t>& out) {
    if (mark[static_cast<size_t>(s)].load(std::memory_order_relaxed) != id) return;
    mark[static_cast<size_t>(s)].store(-id, std::memory_order_relaxed);
    size_t head = out.size();
    out.push_back(s);
    while (head < out.size()) {
      const int32_t u = out[head++];
      for (int32_t k = g.row_ptr[static_cast<size_t>(u)]; k < g.row_ptr[static_cast<size_t>(u) + 1]; ++k) {
        const int32_t v = g.col[static_cast<size_t>(k)];
        if (mark[static_cast<size_t>(v)].load(std::memory_order_relaxed) == id) {
          mark[static_cast<size_t>(v)].store(-id, std::memory_order_relaxed);
          out.push_back(v);
        }
      }
    }
  };
  struct Task {
    std::vector<int32_t> verts;  // in the order they were listed
    int32_t parts, base, id, start;
  };
  std::vector<Task> level(1);
  // the top subset starts from the last vertex a pass from vertex 0 reaches
  {
    std::vector<int32_t> order;
    order.reserve(static_cast<size_t>(n));
    bfs(0, 1, order);
    for (int32_t v = 0; v < n; ++v) bfs(v, 1, order);
    level[0].start = order[static_cast<size_t>(n) - 1];
    level[0].verts = std::move(order);
    level[0].parts = parts;
    level[0].base = 0;
    level[0].id = 1;
  }
  const int32_t threads = plan_threads();
  int32_t next_id = 2;
  while (!level.empty() && !cancelled(cancel)) {
    std::vector<Task> next(2 * level.size());
    for (size_t i = 0; i < level.size(); ++i) {
      next[2 * i].id = next_id++;
      next[2 * i + 1].id = next_id++;
    }
    parallel_for(static_cast<int32_t>(level.size()), threads, [&](int32_t i, int32_t) {
      Task& t = level[static_cast<size_t>(i)];
      if (t.parts == 1 || t.verts.size() <= 1) {
        for (int32_t v : t.verts) (*part)[static_cast<size_t>(v)] = t.base;
        next[2 * static_cast<size_t>(i)].parts = next[2 * static_cast<size_t>(i) + 1].parts = 0;
        return;
      }
      // breadth-first order from a far vertex (the last one a pass from the
      // start vertex reaches); further components follow
      for (int32_t v : t.verts) mark[static_cast<size_t>(v)].store(t.id, std::memory_order_relaxed);
      std::vector<int32_t> order;
      order.reserve(t.verts.size());
      bfs(t.start, t.id, order);
      const int32_t far = order.back();
      for (int32_t v : order) mark[static_cast<size_t>(v)].store(t.id, std::memory_order_relaxed);
      order.clear();
      bfs(far, t.id, order);
      if (order.size() < t.verts.size())
        for (int32_t v : t.verts) bfs(v, t.id, order);
      const int32_t pl = t.parts / 2;
      const size_t k = static_cast<size_t>(static_cast<int64_t>(t.verts.size()) * pl / t.parts);
      Task& lo = next[2 * static_cast<size_t>(i)];
      Task& hi = next[2 * static_cast<size_t>(i) + 1];
      lo.verts.assign(order.begin(), order.begin() + static_cast<std::ptrdiff_t>(k));
      hi.verts.assign(order.begin() + static_cast<std::ptrdiff_t>(k), order.end());
      lo.parts = pl;
      lo.base = t.base;
      hi.parts = t.parts - pl;
      hi.base = t.base + pl;
      // each side's next pass starts from a vertex on its far rim
      lo.start = lo.verts.empty() ? 0 : lo.verts.back();
      hi.start = hi.verts.empty() ? 0 : hi.verts.back();
      t.verts = std::vector<int32_t>();
    });
    level.clear();
    for (Task& t : next)
      if (t.parts > 0 && !t.verts.empty()) level.push_back(std::move(t));
  }
}

namespace {

// One part's tables, with offsets relative to the part (build_halo_plan
// concatenates them).
struct PartTables {
  bool ok = false;
  int32_t hdr[kHaloHdr] = {};
  std::vector<int32_t> words, slices, gpos, imports, nbrs, quads;
  int64_t smem = 0;
  double ratio = 0.0;
};

// tag[v] = ((p + 1) << 32) | value marks v as in part p's region; the value
// is v's hop count while the region grows, then its local index.
void build_part(const HostGraph& g, const std::vector<int32_t>& part, const std::vector<int32_t>& cls,
                const int32_t* own, int32_t owned, int32_t p, int32_t K, int32_t D, int32_t S,
                std::vector<int64_t>& tag, PartTables* pt) {
  const int64_t key = static_cast<int64_t>(p + 1) << 32;
  auto in_region = [&](int32_t v) { return (tag[static_cast<size_t>(v)] >> 32) == p + 1; };
  auto value = [&](int32_t v) { return static_cast<int32_t>(tag[static_cast<size_t>(v)] & 0xffffffff); };
  std::vector<int32_t> region(own, own + owned);
  for (int32_t v : region) tag[static_cast<size_t>(v)] = key;
  size_t layer_b = 0;
  for (int32_t h = 1; h <= D; ++h) {
    const size_t layer_e = region.size();
    for (size_t q = layer_b; q < layer_e; ++q) {
      const int32_t u = region[q];
      for (int32_t k = g.row_ptr[static_cast<size_t>(u)]; k < g.row_ptr[static_cast<size_t>(u) + 1]; ++k) {
        const int32_t v = g.col[static_cast<size_t>(k)];
        if (!in_region(v)) {
          tag[static_cast<size_t>(v)] = key | h;
          region.push_back(v);
        }
      }
    }
    layer_b = layer_e;
  }
  const int32_t R = static_cast<int32_t>(region.size());
  // local order: (class, hops, position)
  std::vector<uint64_t> keys(region.size());
  for (size_t q = 0; q < region.size(); ++q) {
    const int32_t v = region[q];
    keys[q] = (static_cast<uint64_t>(cls[static_cast<size_t>(v)]) << 56) |
              (static_cast<uint64_t>(value(v)) << 32) | static_cast<uint32_t>(v);
  }
  std::sort(keys.begin(), keys.end());
  int32_t* H = pt->hdr;
  H[kHaloR] = R;
  H[kHaloOwned] = owned;
  pt->gpos.resize(static_cast<size_t>(R));
  for (int32_t l = 0; l < R; ++l) {
    const int32_t v = static_cast<int32_t>(keys[static_cast<size_t>(l)] & 0xffffffffu);
    if (((keys[static_cast<size_t>(l)] >> 32) & 0xffffff) > 0) {
      pt->imports.push_back(l);
      pt->imports.push_back(v);
    }
    tag[static_cast<size_t>(v)] = key | l;
    pt->gpos[static_cast<size_t>(l)] = v;
  }
  for (int32_t c = 0; c < K; ++c) {
    int32_t* T = H + kHaloHdrClass + c * (D + 3);
    const uint64_t lo = static_cast<uint64_t>(c) << 56;
    const int32_t seg = static_cast<int32_t>(std::lower_bound(keys.begin(), keys.end(), lo) - keys.begin());
    T[0] = seg;
    for (int32_t h = 0; h <= D; ++h) {
      const uint64_t hi = lo | (static_cast<uint64_t>(h + 1) << 32);
      T[2 + h] = static_cast<int32_t>(std::lower_bound(keys.begin(), keys.end(), hi) - keys.begin()) - seg;
    }
  }
  // sliced ELL of each class's updated rows (at most D - 1 hops out)
  const int32_t pad = static_cast<int32_t>(static_cast<uint32_t>(R) << 8);
  for (int32_t c = 0; c < K; ++c) {
    int32_t* T = H + kHaloHdrClass + c * (D + 3);
    T[1] = static_cast<int32_t>(pt->slices.size());
    const int32_t U = T[2 + D - 1];
    for (int32_t r0 = 0; r0 < U; r0 += 32) {
      int32_t width = 0;
      for (int32_t r = r0; r < std::min(U, r0 + 32); ++r) {
        const int32_t v = pt->gpos[static_cast<size_t>(T[0] + r)];
        width = std::max(width, g.row_ptr[static_cast<size_t>(v) + 1] - g.row_ptr[static_cast<size_t>(v)]);
      }
      const size_t off = pt->words.size();
      if (off >= (size_t(1) << 25)) return;
      pt->slices.push_back(static_cast<int32_t>((off << 6) | static_cast<size_t>(width)));
      pt->words.resize(off + static_cast<size_t>(width) * 32, pad);
      for (int32_t lane = 0; lane < 32 && r0 + lane < U; ++lane) {
        const int32_t v = pt->gpos[static_cast<size_t>(T[0] + r0 + lane)];
        int32_t kk = 0;
        for (int32_t k = g.row_ptr[static_cast<size_t>(v)]; k < g.row_ptr[static_cast<size_t>(v) + 1]; ++k, ++kk)
          pt->words[off + static_cast<size_t>(kk) * 32 + static_cast<size_t>(lane)] =
              static_cast<int32_t>((static_cast<uint32_t>(value(g.col[static_cast<size_t>(k)])) << 8) |
                                   (static_cast<uint32_t>(g.w[static_cast<size_t>(k)]) & 0xffu));
      }
    }
  }
  while (pt->words.size() % 4 != 0) pt->words.push_back(pad);
  H[kHaloWordsLen] = static_cast<int32_t>(pt->words.size());
  H[kHaloSlicesLen] = static_cast<int32_t>(pt->slices.size());
  H[kHaloImportLen] = static_cast<int32_t>(pt->imports.size() / 2);
  for (int32_t v : region)
    if (region.size() > static_cast<size_t>(owned) && part[static_cast<size_t>(v)] != p)
      pt->nbrs.push_back(part[static_cast<size_t>(v)]);
  std::sort(pt->nbrs.begin(), pt->nbrs.end());
  pt->nbrs.erase(std::unique(pt->nbrs.begin(), pt->nbrs.end()), pt->nbrs.end());
  H[kHaloNbrLen] = static_cast<int32_t>(pt->nbrs.size());
  // rows of a full epoch: phase j updates class (j - 1) mod K at most D - j
  // hops out
  int64_t rows = 0;
  for (int32_t j = 1; j <= D; ++j) rows += H[kHaloHdrClass + ((j - 1) % K) * (D + 3) + 2 + (D - j)];
  pt->ratio = static_cast<double>(rows) / (static_cast<double>(S) * owned);
  const int32_t flipw = S * H[kHaloSlicesLen];
  H[kHaloFlipWords] = flipw;
  // quads of the updated rows (at most D - 1 hops out), by quad id, with
  // every member's slot
  if (int64_t(H[kHaloSlicesLen]) * 32 >= 0xffff) return;
  std::vector<uint64_t> qk;  // (q << 34) | (k << 32) | slot
  for (int32_t c = 0; c < K; ++c) {
    const int32_t* T = H + kHaloHdrClass + c * (D + 3);
    for (int32_t r = 0; r < T[2 + D - 1]; ++r) {
      const int32_t l = T[0] + r;
      const uint32_t o = static_cast<uint32_t>(g.perm[static_cast<size_t>(pt->gpos[static_cast<size_t>(l)])]);
      const uint32_t slot = static_cast<uint32_t>((T[1] + (r >> 5)) * 32 + (r & 31));
      qk.push_back((static_cast<uint64_t>(o >> 2) << 34) | (static_cast<uint64_t>(o & 3u) << 32) | slot);
    }
  }
  std::sort(qk.begin(), qk.end());
  for (size_t a = 0; a < qk.size();) {
    const uint64_t q = qk[a] >> 34;
    uint32_t lk[4] = {0xffffu, 0xffffu, 0xffffu, 0xffffu};
    for (; a < qk.size() && (qk[a] >> 34) == q; ++a) lk[(qk[a] >> 32) & 3u] = static_cast<uint32_t>(qk[a] & 0xffffffffu);
    pt->quads.push_back(static_cast<int32_t>(q));
    pt->quads.push_back(static_cast<int32_t>(lk[0] | (lk[1] << 16)));
    pt->quads.push_back(static_cast<int32_t>(lk[2] | (lk[3] << 16)));
  }
  H[kHaloQuadLen] = static_cast<int32_t>(pt->quads.size() / 3);
  pt->smem = halo_smem_bytes(R, H[kHaloWordsLen], H[kHaloSlicesLen], flipw, H[kHaloQuadLen]);
  pt->ok = pt->smem <= kHaloSmemLimit;
}

}  // namespace

void build_halo_plan(const HostGraph& g, int32_t parts, int32_t sweeps_per_epoch, HaloPlan* hp,
                     const std::atomic<bool>* cancel) {
  *hp = HaloPlan();
  const int32_t K = g.num_colours;
  const int32_t n = g.n;
  if (parts < 1 || sweeps_per_epoch < 1 || K < 1 || K > kHaloMaxClasses) return;
  const int32_t D = sweeps_per_epoch * K;
  if (D > kHaloMaxDepth || !g.fits_int8 || g.max_degree > kHaloMaxWidth) return;
  if (n < parts || n >= (1 << 24) - 1) return;
  if (kHaloHdrClass + K * (D + 3) > kHaloHdr) return;

  std::vector<int32_t> part;
  bisect_parts(g, parts, &part, cancel);
  if (cancelled(cancel)) return;
  std::vector<int32_t> cls(static_cast<size_t>(n));
  for (int32_t c = 0; c < K; ++c)
    for (int32_t v = g.class_begin[static_cast<size_t>(c)]; v < g.class_begin[static_cast<size_t>(c) + 1]; ++v)
      cls[static_cast<size_t>(v)] = c;
  // vertices of every part, in position order
  std::vector<int32_t> part_ptr(static_cast<size_t>(parts) + 1, 0), part_verts(static_cast<size_t>(n));
  for (int32_t v = 0; v < n; ++v) part_ptr[static_cast<size_t>(part[static_cast<size_t>(v)]) + 1]++;
  for (int32_t p = 0; p < parts; ++p) {
    if (part_ptr[static_cast<size_t>(p) + 1] == 0) return;  // an empty part
    part_ptr[static_cast<size_t>(p) + 1] += part_ptr[static_cast<size_t>(p)];
  }
  {
    std::vector<int32_t> fill(part_ptr.begin(), part_ptr.end() - 1);
    for (int32_t v = 0; v < n; ++v)
      part_verts[static_cast<size_t>(fill[static_cast<size_t>(part[static_cast<size_t>(v)])]++)] = v;
  }
  std::vector<PartTables> tables(static_cast<size_t>(parts));
  const int32_t threads = std::min(plan_threads(), parts);
  std::vector<std::vector<int64_t>> tags(static_cast<size_t>(threads));
  parallel_for(parts, threads, [&](int32_t p, int32_t w) {
    if (cancelled(cancel)) return;  // the part stays !ok
    std::vector<int64_t>& tag = tags[static_cast<size_t>(w)];
    if (tag.empty()) tag.assign(static_cast<size_t>(n), 0);
    const int32_t b = part_ptr[static_cast<size_t>(p)];
    build_part(g, part, cls, part_verts.data() + b, part_ptr[static_cast<size_t>(p) + 1] - b, p, K, D,
               sweeps_per_epoch, tag, &tables[static_cast<size_t>(p)]);
  });
  // mailboxes: import i of a part reads slot (the part's first import) + i;
  // its vertex's owner writes that slot between epochs, from its own copy
  std::vector<int32_t> owner_local(static_cast<size_t>(n), 0);
  std::vector<int64_t> import_base(static_cast<size_t>(parts) + 1, 0);
  for (int32_t p = 0; p < parts; ++p) {
    const PartTables& pt = tables[static_cast<size_t>(p)];
    if (!pt.ok) {
      *hp = HaloPlan();
      return;
    }
    import_base[static_cast<size_t>(p) + 1] = import_base[static_cast<size_t>(p)] + static_cast<int64_t>(pt.imports.size() / 2);
    for (int32_t c = 0; c < K; ++c) {
      const int32_t* T = pt.hdr + kHaloHdrClass + c * (D + 3);
      for (int32_t l = T[0]; l < T[0] + T[2]; ++l) owner_local[static_cast<size_t>(pt.gpos[static_cast<size_t>(l)])] = l;
    }
  }
  if (import_base[static_cast<size_t>(parts)] >= (int64_t(1) << 31)) {
    *hp = HaloPlan();
    return;
  }
  std::vector<std::vector<int32_t>> out(static_cast<size_t>(parts));  // per owner: (local, slot)
  for (int32_t q = 0; q < parts; ++q) {
    const PartTables& pt = tables[static_cast<size_t>(q)];
    for (size_t i = 0; 2 * i < pt.imports.size(); ++i) {
      const int32_t v = pt.imports[2 * i + 1];
      std::vector<int32_t>& o = out[static_cast<size_t>(part[static_cast<size_t>(v)])];
      o.push_back(owner_local[static_cast<size_t>(v)]);
      o.push_back(static_cast<int32_t>(import_base[static_cast<size_t>(q)] + static_cast<int64_t>(i)));
    }
  }
  hp->mailbox_slots = import_base[static_cast<size_t>(parts)];
  hp->hdr.assign(static_cast<size_t>(parts) * kHaloHdr, 0);
  int64_t smem_max = 0;
  for (int32_t p = 0; p < parts; ++p) {
    PartTables& pt = tables[static_cast<size_t>(p)];
    if (!pt.ok) {
      *hp = HaloPlan();
      return;
    }
    int32_t* H = hp->hdr.data() + static_cast<size_t>(p) * kHaloHdr;
    std::copy(pt.hdr, pt.hdr + kHaloHdr, H);
    H[kHaloWordsOff] = static_cast<int32_t>(hp->words.size());
    H[kHaloSlicesOff] = static_cast<int32_t>(hp->slices.size());
    H[kHaloGposOff] = static_cast<int32_t>(hp->gpos.size());
    H[kHaloImportOff] = static_cast<int32_t>(hp->imports.size());
    H[kHaloNbrOff] = static_cast<int32_t>(hp->nbrs.size());
    H[kHaloQuadOff] = static_cast<int32_t>(hp->quads.size());
    hp->quads.insert(hp->quads.end(), pt.quads.begin(), pt.quads.end());
    H[kHaloExportOff] = static_cast<int32_t>(hp->exports.size());
    hp->exports.insert(hp->exports.end(), out[static_cast<size_t>(p)].begin(), out[static_cast<size_t>(p)].end());
    H[kHaloExportLen] = static_cast<int32_t>(out[static_cast<size_t>(p)].size() / 2);
    out[static_cast<size_t>(p)] = std::vector<int32_t>();
    hp->words.insert(hp->words.end(), pt.words.begin(), pt.words.end());
    hp->slices.insert(hp->slices.end(), pt.slices.begin(), pt.slices.end());
    hp->gpos.insert(hp->gpos.end(), pt.gpos.begin(), pt.gpos.end());
    hp->imports.insert(hp->imports.end(), pt.imports.begin(), pt.imports.end());
    hp->nbrs.insert(hp->nbrs.end(), pt.nbrs.begin(), pt.nbrs.end());
    smem_max = std::max(smem_max, pt.smem);
    hp->max_work_ratio = std::max(hp->max_work_ratio, pt.ratio);
    pt = PartTables();
  }
  hp->ok = true;
  hp->parts = parts;
  hp->sweeps_per_epoch = sweeps_per_epoch;
  hp->depth = D;
  hp->classes = K;
  hp->smem_bytes = static_cast<int32_t>(smem_max);
}

}  // namespace isingx
