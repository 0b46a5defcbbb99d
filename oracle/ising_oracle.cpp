// CPU oracle for the deterministic Ising max-cut annealer.
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
// CPU-baseline leg load this library. It shares no code with the CUDA path:
// its own Philox, its own adjacency build, colouring, schedule and reductions.
// Everything is written for clarity, not speed: int64 arithmetic throughout,
// the adjacency rebuilt from the edge list on every call.
//
// What it computes (paper: Cook, Zhao, Sato, Hiromoto, Tan, "GPU Ising
// Computing for Combinatorial Optimization Problems in VLSI Physical Design"):
//   * max-cut objective, Eq. 4, and its Ising form, Eq. 5 (with the sign
//     reading below);
//   * the local spin update, Eq. 2: the spin takes the value that minimises
//     its local energy given its neighbours;
//   * Algorithm 2: every sweep updates every spin and, right after its own
//     update, flips it with probability F_p; F_p is reduced after each sweep;
//   * the checkerboard idea of Sec. IV-B generalised to greedy colour classes:
//     the classes are swept one after another in increasing colour order.
//
// Readings where the paper is silent or inconsistent (each is repeated in the
// design notes):
//   R1 energy sign: H(s) = sum_{(i,j) in E} w_ij s_i s_j (Eq. 3/5 with J = -w),
//      so that minimising H maximises the cut of Eq. 4:
//      cut(s) = (W - H(s)) / 2, W = sum of the merged edge weights.
//      The update is then s_i <- -sign(f_i) with f_i = sum_j w_ij s_j.
//   R2 tie f_i = 0 (Eq. 2 allows either value): keep the current spin.
//   R3 initial spins: s_i = +1 or -1 from bit 31 of replica r's draw on
//      stream 1 (R5).
//   R4 schedule: F_p decays linearly from p0 at sweep 0 to 0 at sweep T-1,
//      as a 32-bit integer threshold thr[t] = floor(T0 (T-1-t) / (T-1)),
//      T0 = round(p0 2^32) clamped to [0, 2^32-1]; a spin flips iff the 32-bit
//      random word x0 < thr[t].
//   R5 randomness: Philox4x32-10 (Salmon et al., SC'11), key = (lo32(seed),
//      hi32(seed) ^ instance * 0x9E3779B9); a flip (stream 0) or initial spin
//      (stream 1) of vertex v (original id) in replica r uses word v mod 4 of
//      counter (floor(v / 4), sweep t (0 for the initial spins), r, stream),
//      so the four vertices 4q .. 4q + 3 share one evaluation.
//   R6 colouring: greedy first fit over the vertices in order of decreasing
//      degree (ties: smaller id first), i.e. Welsh-Powell, in two tiers. A
//      vertex with at least 256 distinct neighbours is a hub. The hubs take
//      colours 0 .. m-1 by first fit among themselves; every other vertex
//      takes the smallest colour >= m that no already coloured neighbour has,
//      so hub and non-hub vertices never share a class. A graph without hubs
//      gets plain Welsh-Powell. Classes are swept in increasing colour order
//      (the hub classes first), and inside a class the order is irrelevant
//      because no two vertices of a class are adjacent.
//   R11 flip bias (project addition, oracle_anneal_biased): a per-vertex
//      factor q_v / 128 on the flip threshold, in integers.
//   R7 edges: undirected; repeated pairs are merged by summing their weights;
//      a merged weight of 0 is no edge; self-loops and ids outside [0, n) are
//      rejected.
//
// Parity of the exact trajectory (which spin flips when) is pinned only by
// the properties the tests check (brute-force energy/cut, the zero-temperature
// local-minimum invariant, known optima, Philox known answers, flip rates);
// the full trajectory is otherwise "parity unpinned" by the paper, which
// prints no worked example.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10, from the definition in Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two
// 32x32->64 multiplications with the round keys bumped by the Weyl constants.
// ---------------------------------------------------------------------------
struct Words4 {
  uint32_t x[4];
};

const uint32_t kPhiloxMulA = 0xD2511F53u;
const uint32_t kPhiloxMulB = 0xCD9E8D57u;
const uint32_t kWeylA = 0x9E3779B9u;
const uint32_t kWeylB = 0xBB67AE85u;

Words4 philox_round(const Words4& c, uint32_t k0, uint32_t k1) {
  uint64_t pa = (uint64_t)kPhiloxMulA * (uint64_t)c.x[0];
  uint64_t pb = (uint64_t)kPhiloxMulB * (uint64_t)c.x[2];
  uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
  uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
  Words4 r;
  r.x[0] = hi_b ^ c.x[1] ^ k0;
  r.x[1] = lo_b;
  r.x[2] = hi_a ^ c.x[3] ^ k1;
  r.x[3] = lo_a;
  return r;
}

Words4 philox4x32_10(Words4 ctr, uint32_t k0, uint32_t k1) {
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kWeylA;
      k1 += kWeylB;
    }
    ctr = philox_round(ctr, k0, k1);
  }
  return ctr;
}

// R5: the key for (seed, instance) and the x0 word for a counter.
uint32_t random_word(uint64_t seed, uint32_t instance, uint32_t c0, uint32_t c1, uint32_t c2,
                     uint32_t c3) {
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
  uint32_t k1 = (uint32_t)(seed >> 32) ^ (uint32_t)(instance * kWeylA);
  Words4 c = {{c0, c1, c2, c3}};
  return philox4x32_10(c, k0, k1).x[0];
}

// R5: the draw of vertex v in sweep t of replica r on stream s (0 flips,
// 1 initial spins): word v mod 4 of the counter (floor(v / 4), t, r, s), so
// the four vertices 4q .. 4q + 3 share one Philox evaluation.
uint32_t vertex_word(uint64_t seed, uint32_t instance, uint32_t v, uint32_t t,
                     uint32_t replica, uint32_t stream) {
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
  uint32_t k1 = (uint32_t)(seed >> 32) ^ (uint32_t)(instance * kWeylA);
  Words4 c = {{v >> 2, t, replica, stream}};
  return philox4x32_10(c, k0, k1).x[v & 3u];
}

// ---------------------------------------------------------------------------
// R7: undirected weighted adjacency with merged duplicates.
// ---------------------------------------------------------------------------
struct Adjacency {
  int32_t n = 0;
  std::vector<int64_t> start;      // n + 1 offsets
  std::vector<int32_t> neighbour;  // sorted by id within each vertex
  std::vector<int64_t> weight;
  // each undirected edge once (u < v), with its merged weight
  std::vector<int32_t> eu, ev;
  std::vector<int64_t> ew;
};

struct DirectedEdge {
  int32_t from, to;
  int64_t w;
};

bool edge_less(const DirectedEdge& a, const DirectedEdge& b) {
  if (a.from != b.from) return a.from < b.from;
  return a.to < b.to;
}

int build_adjacency(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                    const int32_t* w, Adjacency* adj) {
  if (n <= 0 || m < 0) return -1;
  if (m > 0 && (src == nullptr || dst == nullptr || w == nullptr)) return -1;
  std::vector<DirectedEdge> list;
  list.reserve((size_t)(2 * m));
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) return -1;
    if (u == v) return -1;
    list.push_back({u, v, (int64_t)w[e]});
    list.push_back({v, u, (int64_t)w[e]});
  }
  std::sort(list.begin(), list.end(), edge_less);
  adj->n = n;
  adj->start.assign((size_t)n + 1, 0);
  adj->neighbour.clear();
  adj->weight.clear();
  adj->eu.clear();
  adj->ev.clear();
  adj->ew.clear();
  size_t i = 0;
  std::vector<int64_t> count((size_t)n, 0);
  while (i < list.size()) {
    size_t j = i;
    int64_t sum = 0;
    while (j < list.size() && list[j].from == list[i].from && list[j].to == list[i].to) {
      sum += list[j].w;
      ++j;
    }
    if (sum != 0) {
      adj->neighbour.push_back(list[i].to);
      adj->weight.push_back(sum);
      count[(size_t)list[i].from] += 1;
      if (list[i].from < list[i].to) {
        adj->eu.push_back(list[i].from);
        adj->ev.push_back(list[i].to);
        adj->ew.push_back(sum);
      }
    }
    i = j;
  }
  for (int32_t v = 0; v < n; ++v) adj->start[(size_t)v + 1] = adj->start[(size_t)v] + count[(size_t)v];
  return 0;
}

// R6: two-tier Welsh-Powell greedy colouring. Returns the number of colours.
const int64_t kHubDegree = 256;  // a vertex with this many neighbours or more is a hub

int32_t colour_graph(const Adjacency& adj, std::vector<int32_t>* colour) {
  const int32_t n = adj.n;
  std::vector<int32_t> order((size_t)n);
  for (int32_t v = 0; v < n; ++v) order[(size_t)v] = v;
  auto degree = [&](int32_t v) { return adj.start[(size_t)v + 1] - adj.start[(size_t)v]; };
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (degree(a) != degree(b)) return degree(a) > degree(b);
    return a < b;
  });
  colour->assign((size_t)n, -1);
  // smallest colour >= lowest that no coloured neighbour of v has
  auto first_free = [&](int32_t v, int32_t lowest) {
    std::vector<int32_t> taken;
    for (int64_t k = adj.start[(size_t)v]; k < adj.start[(size_t)v + 1]; ++k) {
      int32_t c = (*colour)[(size_t)adj.neighbour[(size_t)k]];
      if (c >= lowest) taken.push_back(c);
    }
    std::sort(taken.begin(), taken.end());
    int32_t c = lowest;
    for (int32_t t : taken)
      if (t == c) ++c;
    return c;
  };
  // tier 1: the hubs, first fit among the hubs coloured before them
  int32_t hub_colours = 0;
  for (int32_t v : order) {
    if (degree(v) < kHubDegree) continue;
    int32_t c = first_free(v, 0);
    (*colour)[(size_t)v] = c;
    hub_colours = std::max(hub_colours, c + 1);
  }
  // tier 2: every other vertex, in the same order, above the hub colours
  int32_t num_colours = hub_colours;
  for (int32_t v : order) {
    if (degree(v) >= kHubDegree) continue;
    int32_t c = first_free(v, hub_colours);
    (*colour)[(size_t)v] = c;
    num_colours = std::max(num_colours, c + 1);
  }
  return num_colours;
}

// R4: the flip threshold of sweep t of a T-sweep linear schedule.
uint32_t flip_threshold(double p0, uint64_t T, uint64_t t) {
  double scaled = std::floor(p0 * 4294967296.0 + 0.5);
  uint64_t T0;
  if (!(scaled > 0.0))
    T0 = 0;
  else if (scaled >= 4294967295.0)
    T0 = 4294967295u;
  else
    T0 = (uint64_t)scaled;
  if (T <= 1 || t >= T) return 0;
  return (uint32_t)(T0 * (T - 1 - t) / (T - 1));
}

// f_i = sum_j w_ij s_j over the merged adjacency.
int64_t local_field(const Adjacency& adj, const int8_t* s, int32_t v) {
  int64_t f = 0;
  for (int64_t k = adj.start[(size_t)v]; k < adj.start[(size_t)v + 1]; ++k)
    f += adj.weight[(size_t)k] * (int64_t)s[(size_t)adj.neighbour[(size_t)k]];
  return f;
}

}  // namespace

extern "C" {

int oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  Words4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
  Words4 r = philox4x32_10(c, key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.x[i];
  return 0;
}

uint32_t oracle_random_word(uint64_t seed, uint32_t instance, uint32_t c0, uint32_t c1,
                            uint32_t c2, uint32_t c3) {
  return random_word(seed, instance, c0, c1, c2, c3);
}

uint32_t oracle_threshold(double p0, uint64_t T, uint64_t t) { return flip_threshold(p0, T, t); }

// Number of merged undirected edges, or -1 on invalid input.
int64_t oracle_num_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int32_t* w) {
  Adjacency adj;
  if (build_adjacency(n, m, src, dst, w, &adj) != 0) return -1;
  return (int64_t)adj.eu.size();
}

// Writes colour[v] for every vertex; returns the number of colours or -1.
int32_t oracle_colouring(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int32_t* w, int32_t* colour_out) {
  Adjacency adj;
  if (build_adjacency(n, m, src, dst, w, &adj) != 0) return -1;
  std::vector<int32_t> colour;
  int32_t C = colour_graph(adj, &colour);
  for (int32_t v = 0; v < n; ++v) colour_out[v] = colour[(size_t)v];
  return C;
}

// R3: initial spins.
int oracle_init_spins(int32_t n, uint64_t seed, uint32_t instance, uint32_t replica,
                      int8_t* s) {
  if (n <= 0) return -1;
  for (int32_t i = 0; i < n; ++i) {
    uint32_t x = vertex_word(seed, instance, (uint32_t)i, 0u, replica, 1u);
    s[i] = (x >> 31) ? (int8_t)-1 : (int8_t)1;
  }
  return 0;
}

// Energy H (R1), total weight W and cut value of Eq. 4 for spins s.
int oracle_energy_cut(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      const int32_t* w, const int8_t* s, int64_t* energy, int64_t* total_weight,
                      int64_t* cut) {
  Adjacency adj;
  if (build_adjacency(n, m, src, dst, w, &adj) != 0) return -1;
  int64_t H = 0, W = 0;
  for (size_t e = 0; e < adj.eu.size(); ++e) {
    H += adj.ew[e] * (int64_t)s[(size_t)adj.eu[e]] * (int64_t)s[(size_t)adj.ev[e]];
    W += adj.ew[e];
  }
  if (energy) *energy = H;
  if (total_weight) *total_weight = W;
  if (cut) *cut = (W - H) / 2;
  return 0;
}

// Deterministic annealing (Algorithm 2 over colour classes): sweeps
// t_begin .. t_begin + sweeps - 1 of a T-sweep schedule, updating s in place.
// Returns 0, or -1 on invalid input.
//
// bias (may be null): a per-vertex flip bias q_v in 0..255, a project addition
// with no counterpart in the paper (R11): vertex v flips iff
// x < min((thr[t] * q_v) >> 7, 2^32 - 1), computed in 64-bit integers, so
// q_v = 128 is Algorithm 2 unchanged and q_v = 0 never flips.
int oracle_anneal_biased(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int32_t* w, int8_t* s, uint64_t seed, uint32_t instance,
                         uint32_t replica, double p0, uint64_t T, uint64_t t_begin,
                         uint64_t sweeps, const uint8_t* bias) {
  if (!(p0 >= 0.0 && p0 <= 1.0)) return -1;
  if (T >= 4294967296ull || t_begin + sweeps > T) return -1;
  Adjacency adj;
  if (build_adjacency(n, m, src, dst, w, &adj) != 0) return -1;
  for (int32_t i = 0; i < n; ++i)
    if (s[i] != 1 && s[i] != -1) return -1;
  std::vector<int32_t> colour;
  int32_t C = colour_graph(adj, &colour);
  std::vector<std::vector<int32_t>> members((size_t)C);
  for (int32_t v = 0; v < n; ++v) members[(size_t)colour[(size_t)v]].push_back(v);

  for (uint64_t t = t_begin; t < t_begin + sweeps; ++t) {
    uint32_t thr = flip_threshold(p0, T, t);
    for (int32_t c = 0; c < C; ++c) {
      for (int32_t v : members[(size_t)c]) {
        // Eq. 2 under R1/R2.
        int64_t f = local_field(adj, s, v);
        if (f > 0)
          s[v] = -1;
        else if (f < 0)
          s[v] = 1;
        // Algorithm 2: flip right after the update with probability F_p.
        uint64_t thr_v = thr;
        if (bias != nullptr) {
          thr_v = ((uint64_t)thr * (uint64_t)bias[v]) >> 7;
          if (thr_v > 4294967295ull) thr_v = 4294967295ull;
        }
        uint32_t x = vertex_word(seed, instance, (uint32_t)v, (uint32_t)t, replica, 0u);
        if ((uint64_t)x < thr_v) s[v] = (int8_t)(-s[v]);
      }
    }
  }
  return 0;
}

int oracle_anneal(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                  const int32_t* w, int8_t* s, uint64_t seed, uint32_t instance,
                  uint32_t replica, double p0, uint64_t T, uint64_t t_begin, uint64_t sweeps) {
  return oracle_anneal_biased(n, m, src, dst, w, s, seed, instance, replica, p0, T, t_begin,
                              sweeps, nullptr);
}

// Algorithm 1's schedule: a sweep updates every spin (colour classes as in
// oracle_anneal, no per-spin random flip), then flips N_t distinct randomly
// chosen spins, and N decreases: N_t = floor(N0 (T-1-t) / (T-1)) (R4's linear
// decay applied to the count), N0 <= n. Reading R10 (the paper only says
// "randomly choose and flip N spin glasses"): the candidates are
// c_j = floor(x_j * n / 2^32), x_j = Philox word 0 with counter (j, t, replica,
// 2), j = 0, 1, 2, ...; the first N_t distinct candidates are flipped.
int oracle_anneal_nflip(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                        const int32_t* w, int8_t* s, uint64_t seed, uint32_t instance,
                        uint32_t replica, uint32_t n0, uint64_t T, uint64_t t_begin,
                        uint64_t sweeps) {
  if (T >= 4294967296ull || t_begin + sweeps > T) return -1;
  if ((int64_t)n0 > (int64_t)n) return -1;
  Adjacency adj;
  if (build_adjacency(n, m, src, dst, w, &adj) != 0) return -1;
  for (int32_t i = 0; i < n; ++i)
    if (s[i] != 1 && s[i] != -1) return -1;
  std::vector<int32_t> colour;
  int32_t C = colour_graph(adj, &colour);
  std::vector<std::vector<int32_t>> members((size_t)C);
  for (int32_t v = 0; v < n; ++v) members[(size_t)colour[(size_t)v]].push_back(v);
  std::vector<char> chosen((size_t)n, 0);
  std::vector<int32_t> picked;
  for (uint64_t t = t_begin; t < t_begin + sweeps; ++t) {
    for (int32_t c = 0; c < C; ++c)
      for (int32_t v : members[(size_t)c]) {
        int64_t f = local_field(adj, s, v);
        if (f > 0)
          s[v] = -1;
        else if (f < 0)
          s[v] = 1;
      }
    const uint64_t Nt = T <= 1 ? 0 : (uint64_t)n0 * (T - 1 - t) / (T - 1);
    picked.clear();
    for (uint32_t j = 0; picked.size() < Nt; ++j) {
      uint32_t x = random_word(seed, instance, j, (uint32_t)t, replica, 2u);
      int32_t v = (int32_t)(((uint64_t)x * (uint64_t)n) >> 32);
      if (!chosen[(size_t)v]) {
        chosen[(size_t)v] = 1;
        picked.push_back(v);
      }
    }
    for (int32_t v : picked) {
      s[v] = (int8_t)(-s[v]);
      chosen[(size_t)v] = 0;
    }
  }
  return 0;
}

}  // extern "C"
