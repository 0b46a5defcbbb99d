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
// ties broken by smaller id (Welsh-Powell). On a regular graph such as an even
// torus this is natural order, which gives the checkerboard.
#include "host_graph.h"

#include <algorithm>
#include <cstdlib>
#include <limits>

#include "../../include/ising.h"

namespace isingx {

int build_host_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     const int32_t* w, HostGraph* out) {
  if (out == nullptr || n <= 0 || m < 0) return ISING_EINVAL;
  if (m >= (int64_t(1) << 30)) return ISING_ERANGE;
  if (m > 0 && (src == nullptr || dst == nullptr || w == nullptr)) return ISING_EINVAL;
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v) return ISING_EINVAL;
  }
  HostGraph& g = *out;
  g = HostGraph();
  g.n = n;
  const size_t N = (size_t)n;

  // Pass 1: unsorted directed rows.
  std::vector<int64_t> off(N + 1, 0);
  for (int64_t e = 0; e < m; ++e) {
    off[(size_t)src[e] + 1]++;
    off[(size_t)dst[e] + 1]++;
  }
  for (size_t i = 0; i < N; ++i) off[i + 1] += off[i];
  const size_t D = (size_t)off[N];
  std::vector<int32_t> nb1(D), wt1(D);
  {
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int64_t e = 0; e < m; ++e) {
      int32_t u = src[e], v = dst[e];
      size_t a = (size_t)fill[(size_t)u]++;
      nb1[a] = v;
      wt1[a] = w[e];
      size_t b = (size_t)fill[(size_t)v]++;
      nb1[b] = u;
      wt1[b] = w[e];
    }
  }
  // Pass 2: rows sorted by neighbour id. Row x lists the y with an entry
  // (y -> x); visiting x in increasing order appends x to row y in order.
  std::vector<int32_t> nb2(D), wt2(D);
  {
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (size_t x = 0; x < N; ++x) {
      for (int64_t k = off[x]; k < off[x + 1]; ++k) {
        size_t y = (size_t)nb1[(size_t)k];
        size_t a = (size_t)fill[y]++;
        nb2[a] = (int32_t)x;
        wt2[a] = wt1[(size_t)k];
      }
    }
  }
  nb1.clear();
  nb1.shrink_to_fit();
  wt1.clear();
  wt1.shrink_to_fit();

  // Merge repeated neighbours, drop zero sums, bound every field.
  std::vector<int64_t> moff(N + 1, 0);
  std::vector<int32_t> mnb;
  std::vector<int32_t> mwt;
  mnb.reserve(D);
  mwt.reserve(D);
  int64_t total_directed = 0;
  bool fits8 = true;
  int32_t maxdeg = 0;
  for (size_t u = 0; u < N; ++u) {
    int64_t k = off[u];
    int64_t abs_sum = 0;
    while (k < off[u + 1]) {
      int32_t v = nb2[(size_t)k];
      int64_t s = 0;
      while (k < off[u + 1] && nb2[(size_t)k] == v) {
        s += wt2[(size_t)k];
        ++k;
      }
      if (s == 0) continue;
      abs_sum += s < 0 ? -s : s;
      if (abs_sum > (int64_t)std::numeric_limits<int32_t>::max()) return ISING_ERANGE;
      if (s > 127 || s < -127) fits8 = false;
      mnb.push_back(v);
      mwt.push_back((int32_t)s);
      total_directed += s;
    }
    moff[u + 1] = (int64_t)mnb.size();
    maxdeg = std::max<int32_t>(maxdeg, (int32_t)(moff[u + 1] - moff[u]));
  }
  nb2.clear();
  nb2.shrink_to_fit();
  wt2.clear();
  wt2.shrink_to_fit();
  g.nnz = (int64_t)mnb.size();
  g.num_edges = g.nnz / 2;
  g.total_weight = total_directed / 2;
  g.fits_int8 = fits8;
  g.max_degree = maxdeg;

  // Welsh-Powell order: degree descending, id ascending (bucketed by degree).
  auto degree = [&](size_t v) { return (int32_t)(moff[v + 1] - moff[v]); };
  std::vector<int32_t> order(N);
  {
    std::vector<int64_t> bucket((size_t)maxdeg + 2, 0);
    for (size_t v = 0; v < N; ++v) bucket[(size_t)(maxdeg - degree(v)) + 1]++;
    for (size_t d = 0; d + 1 < bucket.size(); ++d) bucket[d + 1] += bucket[d];
    for (size_t v = 0; v < N; ++v) order[(size_t)bucket[(size_t)(maxdeg - degree(v))]++] = (int32_t)v;
  }
  // First-fit colouring.
  g.colour.assign(N, -1);
  {
    std::vector<int32_t> mark((size_t)maxdeg + 2, -1);
    int32_t C = 0;
    for (int32_t v : order) {
      const int32_t d = degree((size_t)v);
      for (int64_t k = moff[(size_t)v]; k < moff[(size_t)v + 1]; ++k) {
        int32_t c = g.colour[(size_t)mnb[(size_t)k]];
        if (c >= 0 && c <= d) mark[(size_t)c] = v;
      }
      int32_t c = 0;
      while (mark[(size_t)c] == v) ++c;
      g.colour[(size_t)v] = c;
      C = std::max(C, c + 1);
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
  // Colour-ordered CSR with each row sorted by neighbour position (visit
  // target positions in increasing order and append to the rows that list it).
  g.row_ptr.assign(N + 1, 0);
  for (size_t p = 0; p < N; ++p) g.row_ptr[p + 1] = g.row_ptr[p] + degree((size_t)g.perm[p]);
  g.col.assign((size_t)g.nnz, 0);
  g.w.assign((size_t)g.nnz, 0);
  {
    std::vector<int32_t> fill(g.row_ptr.begin(), g.row_ptr.end() - 1);
    for (size_t p = 0; p < N; ++p) {
      const size_t x = (size_t)g.perm[p];
      for (int64_t k = moff[x]; k < moff[x + 1]; ++k) {
        const size_t row = (size_t)g.pos[(size_t)mnb[(size_t)k]];
        const size_t a = (size_t)fill[row]++;
        g.col[a] = (int32_t)p;
        g.w[a] = mwt[(size_t)k];
      }
    }
  }
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
      const int64_t off = (int64_t)plan->ell_col.size();
      plan->ell_col.resize((size_t)(off + (int64_t)D * nv), -1);
      plan->ell_w.resize((size_t)(off + (int64_t)D * nv), 0);
      for (int32_t r = 0; r < nv; ++r) {
        const int64_t rb = g.row_ptr[(size_t)(v + r)];
        const int64_t deg = degree(v + r);
        for (int64_t k = 0; k < deg; ++k) {
          plan->ell_col[(size_t)(off + k * nv + r)] = g.col[(size_t)(rb + k)];
          plan->ell_w[(size_t)(off + k * nv + r)] = g.w[(size_t)(rb + k)];
        }
      }
      plan->items.push_back({v, end, (int32_t)off, -(D + 1)});
      v = end;
    }
    plan->class_item_begin[(size_t)c + 1] = (int32_t)plan->items.size();
    plan->max_class_items = std::max<int32_t>(
        plan->max_class_items,
        plan->class_item_begin[(size_t)c + 1] - plan->class_item_begin[(size_t)c]);
  }
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
  dep_ptr->reserve((size_t)ni + 1);
  dep_ptr->push_back(0);
  // seen[j] == i + 1 marks j as already listed for item i (no sorting)
  std::vector<int32_t> seen((size_t)ni, 0);
  for (int32_t i = 0; i < ni; ++i) {
    const WorkItem& it = plan.items[(size_t)i];
    for (int32_t v = it.v_begin; v < it.v_end; ++v)
      for (int32_t k = g.row_ptr[(size_t)v]; k < g.row_ptr[(size_t)v + 1]; ++k) {
        const int32_t j = item_of[(size_t)g.col[(size_t)k]];
        if (j == i || seen[(size_t)j] == i + 1) continue;
        seen[(size_t)j] = i + 1;
        deps->push_back((j << 1) | (class_of[(size_t)j] > class_of[(size_t)i] ? 1 : 0));
      }
    dep_ptr->push_back((int32_t)deps->size());
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
