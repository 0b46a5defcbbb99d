// Batched annealing: many independent max-cut instances, each annealed in up
// to eight replicas, in one persistent kernel (the deterministic colour-class
// schedule of ising.h applied to every instance and replica).
//
// Each instance is built by the same host pipeline as a single graph (merged
// duplicates, greedy colouring, colour-ordered CSR of packed (col << 8 | w)
// words) and the instances are concatenated. A block takes instances from a
// work queue (largest first), keeps the instance's spins in shared memory as
// one byte per vertex (bit r = replica r, set for spin -1), runs every sweep
// with __syncthreads between colour classes, and writes the spins back. No
// block ever waits on another block.
//
// Randomness (Algorithm 2's flips and the initial spins) follows ising.h with
// the instance folded into the key: key = (lo32(seed), hi32(seed) ^
// instance * 0x9E3779B9). Vertex v (id within the instance) of replica r
// draws word v mod 4 of counter (floor(v / 4), sweep t, r, 0) for its flip
// and of (floor(v / 4), 0, r, 1) for its initial spin, so the four vertices
// 4q .. 4q + 3 share one Philox evaluation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/ising.h"
#include "batch_view.h"
#include "host_graph.h"
#include "philox.cuh"

namespace {

using isingx::HostGraph;
using isingx::PhiloxKey;

struct BatchGraph {
  int32_t n;           // vertices
  int32_t num_classes;
  int32_t vtx_base;    // first vertex in the concatenated vertex arrays
  int32_t row_base;    // first entry of this instance's row_ptr (n + 1 entries)
  int32_t class_base;  // first entry of this instance's class bounds (num_classes + 1)
  int32_t byte_lanes;  // 2: every weight is +1 or -1; 1: every |w| is at most 31 (byte-lane
                       // sums); 0: per-replica sums
  int32_t flush;       // heavy rows, byte-lane modes: entries a lane adds before its byte
                       // lanes could reach 255 (then they are moved to int sums)
};

struct BatchDev {
  const BatchGraph* graphs;
  const int32_t* order;      // instances by decreasing size
  const int32_t* row_ptr;    // per instance, absolute offsets into adj
  const int32_t* adj;        // packed (col << 8) | (w & 0xff), col local to the instance
  const int32_t* orig;       // position -> vertex id within the instance
  const int32_t* class_pos;  // per instance: first position of each class, then n
  const int32_t* class_heavy;  // per instance and class: the end of the class's heavy rows
                               // (positions class_pos[c] .. class_heavy[c] - 1; a class lists
                               // its rows by decreasing degree)
  uint8_t* spins;            // replica bits per position
  uint8_t* flips;            // the sweep's flip bits per vertex id (bit r = replica r)
};

// Philox4x32-10, all four words; vertex o of replica r draws word o mod 4
// of counter (o / 4, t, r, stream), so one evaluation serves four vertices.
__device__ __forceinline__ uint4 batch_philox(uint32_t x0, uint32_t x1, uint32_t x2,
                                              uint32_t x3, uint32_t ka, uint32_t kb) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa = static_cast<uint64_t>(0xD2511F53u) * x0;
    const uint64_t pb = static_cast<uint64_t>(0xCD9E8D57u) * x2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ x1 ^ ka;
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ x3 ^ kb;
    x1 = static_cast<uint32_t>(pb);
    x3 = static_cast<uint32_t>(pa);
    x0 = n0;
    x2 = n2;
    ka += 0x9E3779B9u;
    kb += 0xBB67AE85u;
  }
  return make_uint4(x0, x1, x2, x3);
}

// A row's field terms for every replica: accumulator words for the
// byte-lane paths or per-replica sums, and the sum of the weights.
struct RowSums {
  uint32_t a0, a1, a2, a3;  // byte lanes: lo / hi counts (+-1), or plo / phi / nlo / nhi
  int acc[8];               // per-replica path
  int wsum;
};

// The field terms of one row's entries [e0, e1) taken with stride S (the
// row is shared by S consecutive threads, this one starting at e0 + sub).
template <int S>
__device__ __forceinline__ void row_sums(const BatchDev& d, const uint8_t* sp, int mode, int e0, int e1,
                                         int sub, RowSums& r) {
  r.a0 = r.a1 = r.a2 = r.a3 = 0u;
  r.wsum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.acc[k] = 0;
  if (mode == 2) {
    // +-1 weights: w_j s_j = -1 exactly when the neighbour's spin bit
    // differs from the weight's sign bit, so with x = b ^ (0xff if w < 0)
    // the byte lanes count the negative products and f_r = degree - 2 *
    // count_r (each nibble of x spread into byte lanes as below)
    for (int e = e0 + sub; e < e1; e += S) {
      const uint32_t word = static_cast<uint32_t>(__ldg(d.adj + e));
      // 0, or 0xffffffff for a negative weight byte
      const uint32_t neg = static_cast<uint32_t>(static_cast<int32_t>(word << 24) >> 31);
      const uint32_t b = sp[word >> 8];
      r.a0 += (((b ^ neg) & 0xfu) * 0x00204081u) & 0x01010101u;
      r.a1 += ((((b >> 4) ^ neg) & 0xfu) * 0x00204081u) & 0x01010101u;
      r.wsum += 1;
    }
  } else if (mode == 1) {
    // the 8 replica bits of a neighbour spread into 8 byte lanes (4 per
    // word: x * 0x00204081 puts bit k of a nibble at bit 8k), weighted by
    // |w| into a positive and a negative accumulator; no lane can exceed 255
    // because the row's sum of |w| does not
    for (int e = e0 + sub; e < e1; e += S) {
      const int word = __ldg(d.adj + e);
      const int wgt = (word << 24) >> 24;
      const uint32_t b = sp[static_cast<unsigned>(word) >> 8];
      r.wsum += wgt;
      const uint32_t lo = ((b & 0xfu) * 0x00204081u) & 0x01010101u;
      const uint32_t hi = ((b >> 4) * 0x00204081u) & 0x01010101u;
      const uint32_t mag = static_cast<uint32_t>(wgt < 0 ? -wgt : wgt);
      if (wgt > 0) {
        r.a0 += lo * mag;
        r.a1 += hi * mag;
      } else {
        r.a2 += lo * mag;
        r.a3 += hi * mag;
      }
    }
  } else {
    for (int e = e0 + sub; e < e1; e += S) {
      const int word = __ldg(d.adj + e);
      const int wgt = (word << 24) >> 24;
      const int b = sp[static_cast<unsigned>(word) >> 8];
      r.wsum += wgt;
#pragma unroll
      for (int k = 0; k < 8; ++k) r.acc[k] += (b >> k) & 1 ? wgt : 0;
    }
  }
}

// Combine the S partial sums of a row's threads (consecutive lanes of one
// warp, group mask m): byte-lane words add without carries because no lane
// of a row's total exceeds 255.
template <int S>
__device__ __forceinline__ void row_combine(RowSums& r, unsigned m) {
#pragma unroll
  for (int o = 1; o < S; o <<= 1) {
    r.a0 += __shfl_xor_sync(m, r.a0, o);
    r.a1 += __shfl_xor_sync(m, r.a1, o);
    r.a2 += __shfl_xor_sync(m, r.a2, o);
    r.a3 += __shfl_xor_sync(m, r.a3, o);
    r.wsum += __shfl_xor_sync(m, r.wsum, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) r.acc[k] += __shfl_xor_sync(m, r.acc[k], o);
  }
}

// The decision of one vertex for every replica (Eq. 2 under the max-cut sign,
// then Algorithm 2's flip bits): the new replica byte.
__device__ __forceinline__ int decide_replicas(const RowSums& r, int mode, int own, int fl, int replicas) {
  int acc[8];
  if (mode == 2) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[k] = static_cast<int>((r.a0 >> (8 * k)) & 0xffu);
      acc[k + 4] = static_cast<int>((r.a1 >> (8 * k)) & 0xffu);
    }
  } else if (mode == 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[k] = static_cast<int>((r.a0 >> (8 * k)) & 0xffu) - static_cast<int>((r.a2 >> (8 * k)) & 0xffu);
      acc[k + 4] = static_cast<int>((r.a1 >> (8 * k)) & 0xffu) - static_cast<int>((r.a3 >> (8 * k)) & 0xffu);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = r.acc[k];
  }
  // f_r = sum_j w_j s_j = wsum - 2 * sum over neighbours with spin -1
  int nb = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k >= replicas) break;
    const int f = r.wsum - 2 * acc[k];
    int bit = (own >> k) & 1;  // 1 = spin -1
    if (f > 0)
      bit = 1;
    else if (f < 0)
      bit = 0;
    bit ^= (fl >> k) & 1;
    nb |= bit << k;
  }
  return nb;
}

// A heavy row (more entries than byte lanes can sum: degree * max|w| > 255)
// decided by a whole warp: lanes stride the entries; in the byte-lane modes a
// lane moves its byte lanes into int sums every `flush` entries, so no lane
// overflows; the lanes' sums meet by warp shuffles and lane 0 decides.
__device__ __forceinline__ void heavy_row(const BatchDev& d, uint8_t* sp, const BatchGraph& G, int mode,
                                          const int32_t* rp, int v, int lane, uint32_t thr, int replicas) {
  int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int wsum = 0;
  const int e1 = __ldg(rp + v + 1);
  int e = __ldg(rp + v) + lane;
  if (mode == 0) {
    for (; e < e1; e += 32) {
      const int word = __ldg(d.adj + e);
      const int wgt = (word << 24) >> 24;
      const int b = sp[static_cast<unsigned>(word) >> 8];
      wsum += wgt;
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += (b >> k) & 1 ? wgt : 0;
    }
  } else {
    while (e < e1) {
      uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u;
      for (int i = 0; i < G.flush && e < e1; ++i, e += 32) {
        const uint32_t word = static_cast<uint32_t>(__ldg(d.adj + e));
        const uint32_t b = sp[word >> 8];
        if (mode == 2) {
          const uint32_t neg = static_cast<uint32_t>(static_cast<int32_t>(word << 24) >> 31);
          a0 += (((b ^ neg) & 0xfu) * 0x00204081u) & 0x01010101u;
          a1 += ((((b >> 4) ^ neg) & 0xfu) * 0x00204081u) & 0x01010101u;
          wsum += 1;
        } else {
          const int wgt = static_cast<int>(word << 24) >> 24;
          const uint32_t lo = ((b & 0xfu) * 0x00204081u) & 0x01010101u;
          const uint32_t hi = ((b >> 4) * 0x00204081u) & 0x01010101u;
          const uint32_t mag = static_cast<uint32_t>(wgt < 0 ? -wgt : wgt);
          wsum += wgt;
          if (wgt > 0) {
            a0 += lo * mag;
            a1 += hi * mag;
          } else {
            a2 += lo * mag;
            a3 += hi * mag;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        acc[k] += static_cast<int>((a0 >> (8 * k)) & 0xffu) - static_cast<int>((a2 >> (8 * k)) & 0xffu);
        acc[k + 4] += static_cast<int>((a1 >> (8 * k)) & 0xffu) - static_cast<int>((a3 >> (8 * k)) & 0xffu);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  }
  if (lane == 0) {
    RowSums r;
    r.a0 = r.a1 = r.a2 = r.a3 = 0u;
    r.wsum = wsum;
#pragma unroll
    for (int k = 0; k < 8; ++k) r.acc[k] = acc[k];
    const int fl = thr != 0u ? __ldcg(d.flips + G.vtx_base + __ldg(d.orig + G.vtx_base + v)) : 0;
    sp[v] = static_cast<uint8_t>(decide_replicas(r, 0, sp[v], fl, replicas));
  }
}

// One instance per block iteration; all sweeps t_begin .. t_begin + sweeps - 1.
// Tuning (ising_batch_autotune): BLOCK threads; S threads share each row
// (the row's entries strided over them); classes of at most `tail` vertices
// are decided by warp 0 alone with warp barriers (the other warps wait at
// the next larger class's block barrier).
template <int BLOCK, int S>
__global__ void __launch_bounds__(BLOCK)
    batch_anneal_kernel(BatchDev d, int num_graphs, unsigned* work, uint64_t t_begin,
                        uint32_t sweeps, uint64_t T, uint64_t T0, uint32_t seed_lo,
                        uint32_t seed_hi, int replicas, int tail) {
  extern __shared__ uint8_t sp[];
  __shared__ int slot_shared;
  const int lane = threadIdx.x & 31;
  const int sub = lane % S;
  const unsigned gmask = (S == 32 ? 0xffffffffu : ((1u << S) - 1u)) << (lane - sub);
  for (;;) {
    if (threadIdx.x == 0) slot_shared = static_cast<int>(atomicAdd(work, 1u));
    __syncthreads();
    const int slot = slot_shared;
    if (slot >= num_graphs) return;
    const int gi = __ldg(d.order + slot);
    const BatchGraph G = d.graphs[gi];
    for (int v = threadIdx.x; v < G.n; v += BLOCK) sp[v] = d.spins[G.vtx_base + v];
    __syncthreads();
    const uint32_t ka = seed_lo;
    const uint32_t kb = seed_hi ^ (static_cast<uint32_t>(gi) * 0x9E3779B9u);
    const int32_t* rp = d.row_ptr + G.row_base;
    const int32_t* cls = d.class_pos + G.class_base;
    const int32_t* hcls = d.class_heavy + G.class_base;
    const int mode = G.byte_lanes;
    for (uint32_t k = 0; k < sweeps; ++k) {
      const uint64_t t = t_begin + k;
      const uint32_t thr = (T <= 1) ? 0u : static_cast<uint32_t>((T0 * (T - 1 - t)) / (T - 1));
      // the sweep's flips, four vertices per Philox evaluation and replica
      // (R5), into the instance's flip bytes (read back through L2 below)
      if (thr != 0u) {
        for (int q = threadIdx.x; q < (G.n + 3) / 4; q += BLOCK) {
          uint32_t fb = 0;  // byte k: vertex 4q + k, bit r: replica r
          for (int r = 0; r < replicas; ++r) {
            const uint4 x = batch_philox(static_cast<uint32_t>(q), static_cast<uint32_t>(t),
                                         static_cast<uint32_t>(r), 0u, ka, kb);
            fb |= (static_cast<uint32_t>(x.x < thr) << r) | (static_cast<uint32_t>(x.y < thr) << (8 + r)) |
                  (static_cast<uint32_t>(x.z < thr) << (16 + r)) | (static_cast<uint32_t>(x.w < thr) << (24 + r));
          }
          uint8_t* fq = d.flips + G.vtx_base + 4 * q;
          for (int k = 0; k < 4 && 4 * q + k < G.n; ++k) fq[k] = static_cast<uint8_t>(fb >> (8 * k));
        }
        __syncthreads();
      }
      bool tail_run = false;  // warp 0 has decided tail classes since the last block barrier
      for (int c = 0; c < G.num_classes; ++c) {
        const int cb = __ldg(cls + c), ce = __ldg(cls + c + 1), hb = __ldg(hcls + c);
        const bool small = ce - cb <= tail;
        if (small) {
          // warp 0 alone: the heavy rows one at a time, then one light vertex per lane
          if (threadIdx.x < 32) {
            for (int v = cb; v < hb; ++v) heavy_row(d, sp, G, mode, rp, v, lane, thr, replicas);
            const int v = hb + lane;
            if (v < ce) {
              RowSums r;
              row_sums<1>(d, sp, mode, __ldg(rp + v), __ldg(rp + v + 1), 0, r);
              const int fl = thr != 0u ? __ldcg(d.flips + G.vtx_base + __ldg(d.orig + G.vtx_base + v)) : 0;
              sp[v] = static_cast<uint8_t>(decide_replicas(r, mode, sp[v], fl, replicas));
            }
            __syncwarp();
          }
          tail_run = true;
          continue;
        }
        if (tail_run) {  // warp 0's tail classes are complete and visible
          __syncthreads();
          tail_run = false;
        }
        for (int v = cb + static_cast<int>(threadIdx.x) / 32; v < hb; v += BLOCK / 32)
          heavy_row(d, sp, G, mode, rp, v, lane, thr, replicas);
        for (int v = hb + static_cast<int>(threadIdx.x) / S; v < ce; v += BLOCK / S) {
          RowSums r;
          row_sums<S>(d, sp, mode, __ldg(rp + v), __ldg(rp + v + 1), sub, r);
          if (S > 1) row_combine<S>(r, gmask);
          if (sub == 0) {
            const int fl = thr != 0u ? __ldcg(d.flips + G.vtx_base + __ldg(d.orig + G.vtx_base + v)) : 0;
            sp[v] = static_cast<uint8_t>(decide_replicas(r, mode, sp[v], fl, replicas));
          }
        }
        __syncthreads();
      }
      if (tail_run) __syncthreads();
    }
    for (int v = threadIdx.x; v < G.n; v += BLOCK) d.spins[G.vtx_base + v] = sp[v];
    __syncthreads();
  }
}

// Initial spins of every instance and replica (one block per instance).
__global__ void batch_init_kernel(BatchDev d, uint32_t seed_lo, uint32_t seed_hi, int replicas) {
  const BatchGraph G = d.graphs[blockIdx.x];
  const uint32_t kb = seed_hi ^ (static_cast<uint32_t>(blockIdx.x) * 0x9E3779B9u);
  for (int v = threadIdx.x; v < G.n; v += blockDim.x) {
    const uint32_t o = static_cast<uint32_t>(d.orig[G.vtx_base + v]);
    int byte = 0;
    for (int r = 0; r < replicas; ++r) {
      const uint4 x = batch_philox(o >> 2, 0u, static_cast<uint32_t>(r), 1u, seed_lo, kb);
      const uint32_t k = o & 3u;
      const uint32_t word = k == 0u ? x.x : (k == 1u ? x.y : (k == 2u ? x.z : x.w));
      byte |= static_cast<int>(word >> 31) << r;
    }
    d.spins[G.vtx_base + v] = static_cast<uint8_t>(byte);
  }
}

// twice the energy of every replica of every instance: sum_v s_v f_v (one block per instance)
__global__ void batch_energy_kernel(BatchDev d, int replicas, long long* out2) {
  const BatchGraph G = d.graphs[blockIdx.x];
  const int32_t* rp = d.row_ptr + G.row_base;
  long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int v = threadIdx.x; v < G.n; v += blockDim.x) {
    const int own = d.spins[G.vtx_base + v];
    int f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      const int word = d.adj[e];
      const int wgt = (word << 24) >> 24;
      const int b = d.spins[G.vtx_base + (static_cast<unsigned>(word) >> 8)];
      for (int r = 0; r < 8; ++r) f[r] += wgt * (1 - 2 * ((b >> r) & 1));
    }
    for (int r = 0; r < 8; ++r) acc[r] += static_cast<long long>(1 - 2 * ((own >> r) & 1)) * f[r];
  }
  __shared__ long long part[8][32];
  for (int r = 0; r < 8; ++r) {
    long long x = acc[r];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) part[r][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < replicas) {
    long long s = 0;
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) s += part[threadIdx.x][k];
    out2[static_cast<size_t>(blockIdx.x) * replicas + threadIdx.x] = s;
  }
}

uint64_t batch_t0(double p0) {
  const double scaled = std::floor(p0 * 4294967296.0 + 0.5);
  if (scaled >= 4294967295.0) return 4294967295ull;
  if (scaled > 0.0) return static_cast<uint64_t>(scaled);
  return 0;
}

constexpr int kBlockChoices[3] = {128, 256, 512};
constexpr int kSplitChoices[3] = {1, 2, 4};
constexpr int kTailChoices[2] = {0, 32};
constexpr int kTuneConfigs = 18;  // block x split x tail

}  // namespace

struct ising_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  int status = ISING_OK;
  int num_sms = 1;
  int32_t num_graphs = 0;
  int replicas = 1;
  int32_t max_n = 0;
  int block = 256;  // chosen by ising_batch_autotune (with split and tail below)
  uint64_t launches = 0;
  std::vector<int32_t> n;                  // per instance
  std::vector<int64_t> total_weight;       // per instance
  std::vector<std::vector<int32_t>> pos;   // per instance: vertex id -> position
  std::vector<int32_t> vtx_base;           // per instance
  BatchGraph* d_graphs = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_row_ptr = nullptr;
  int32_t* d_adj = nullptr;
  int32_t* d_orig = nullptr;
  int32_t* d_class_pos = nullptr;
  int32_t* d_class_heavy = nullptr;
  uint8_t* d_spins = nullptr;
  uint8_t* d_flips = nullptr;
  unsigned* d_work = nullptr;
  long long* d_energy2 = nullptr;
  // captured launch, reused while the block size stays the same
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraphNode_t kernel_node = nullptr;
  const void* graph_kernel = nullptr;  // the kernel the captured graph launches
  int split = 1;  // threads per row (ising_batch_autotune)
  int tail = 0;   // classes up to this size decided by one warp
  float probe_ms[kTuneConfigs] = {};  // the autotuner's probe times
  int64_t total_nnz = 0;
  // the instances as one graph, for the warm-start network (batch_union)
  int32_t* d_union_row_ptr = nullptr;
  int32_t* d_union_vbase = nullptr;
  int32_t* d_gnn_rowid = nullptr;
  int32_t* d_gnn_hchunk = nullptr;
  int32_t* d_gnn_chunk_row = nullptr;
  int32_t gnn_num_chunks = -1;

  BatchDev dev() const {
    BatchDev d;
    d.graphs = d_graphs;
    d.order = d_order;
    d.row_ptr = d_row_ptr;
    d.adj = d_adj;
    d.orig = d_orig;
    d.class_pos = d_class_pos;
    d.class_heavy = d_class_heavy;
    d.spins = d_spins;
    d.flips = d_flips;
    return d;
  }
};

namespace {

void batch_free(ising_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* ptrs[] = {b->d_graphs,       b->d_order,       b->d_row_ptr,    b->d_adj,
                  b->d_orig,         b->d_class_pos,   b->d_spins,      b->d_flips,
                  b->d_work,         b->d_energy2,     b->d_union_row_ptr, b->d_union_vbase,
                  b->d_gnn_rowid,    b->d_gnn_hchunk,  b->d_gnn_chunk_row, b->d_class_heavy};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

int batch_enter(ising_batch* b) {
  if (b == nullptr) return ISING_EINVAL;
  if (b->status != ISING_OK) return b->status;
  if (cudaSetDevice(b->device) != cudaSuccess) {
    cudaGetLastError();
    b->status = ISING_ECUDA;
    return ISING_ECUDA;
  }
  return ISING_OK;
}

#define BATCH_CUDA(b, call)          \
  do {                               \
    cudaError_t e_ = (call);         \
    if (e_ != cudaSuccess) {         \
      cudaGetLastError();            \
      (b)->status = ISING_ECUDA;     \
      return ISING_ECUDA;            \
    }                                \
  } while (0)

// Row table of the disjoint union: every instance's rows by position, with
// the instance's first position beside each row.
__global__ void union_rows_kernel(const BatchGraph* graphs, const int32_t* row_ptr, int num_graphs,
                                  int32_t* urow, int32_t* vbase) {
  for (int gi = blockIdx.x; gi < num_graphs; gi += gridDim.x) {
    const BatchGraph G = graphs[gi];
    for (int v = threadIdx.x; v < G.n; v += blockDim.x) {
      urow[G.vtx_base + v] = row_ptr[G.row_base + v];
      vbase[G.vtx_base + v] = G.vtx_base;
    }
  }
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
  const size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
  if (e != cudaSuccess) return e;
  if (!src.empty()) return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  return cudaMemsetAsync(*dst, 0, bytes, s);
}

template <int BLOCK>
const void* batch_kernel_split(int split) {
  if (split == 2) return reinterpret_cast<const void*>(batch_anneal_kernel<BLOCK, 2>);
  if (split == 4) return reinterpret_cast<const void*>(batch_anneal_kernel<BLOCK, 4>);
  return reinterpret_cast<const void*>(batch_anneal_kernel<BLOCK, 1>);
}

const void* batch_kernel_for(int block, int split) {
  if (block == 128) return batch_kernel_split<128>(split);
  if (block == 512) return batch_kernel_split<512>(split);
  return batch_kernel_split<256>(split);
}

// Blocks of the persistent batch kernel: every co-resident block (shared
// memory holds the largest instance's spins).
int batch_grid(ising_batch* b, int block, int split, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(block, split), block, smem);
  cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  return std::min(per_sm * b->num_sms, std::max(1, b->num_graphs));
}

// Enqueue one anneal of every instance: reset the work queue, launch the
// persistent kernel. The pair is captured into a CUDA graph once per block
// size and replayed with this call's parameters.
int batch_launch(ising_batch* b, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                 uint64_t seed) {
  const size_t smem = static_cast<size_t>(std::max(b->max_n, 1));
  const void* kernel = batch_kernel_for(b->block, b->split);
  BATCH_CUDA(b, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
  const int grid = batch_grid(b, b->block, b->split, smem);
  BatchDev d = b->dev();
  int num_graphs = b->num_graphs;
  unsigned* work = b->d_work;
  uint32_t seed_lo = static_cast<uint32_t>(seed), seed_hi = static_cast<uint32_t>(seed >> 32);
  int replicas = b->replicas;
  int tail = b->tail;
  void* args[] = {&d, &num_graphs, &work, &t_begin, &sweeps, &T, &T0, &seed_lo, &seed_hi, &replicas, &tail};
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(kernel);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(b->block);
  kp.sharedMemBytes = static_cast<unsigned>(smem);
  kp.kernelParams = args;
  if (b->graph_exec == nullptr || b->graph_kernel != kernel) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    BATCH_CUDA(b, cudaGraphCreate(&b->graph, 0));
    cudaGraphNode_t memset_node;
    cudaMemsetParams mp = {};
    mp.dst = b->d_work;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = 1;
    mp.height = 1;
    BATCH_CUDA(b, cudaGraphAddMemsetNode(&memset_node, b->graph, nullptr, 0, &mp));
    BATCH_CUDA(b, cudaGraphAddKernelNode(&b->kernel_node, b->graph, &memset_node, 1, &kp));
    BATCH_CUDA(b, cudaGraphInstantiate(&b->graph_exec, b->graph, 0));
    b->graph_kernel = kernel;
  } else {
    BATCH_CUDA(b, cudaGraphExecKernelNodeSetParams(b->graph_exec, b->kernel_node, &kp));
  }
  b->launches++;
  BATCH_CUDA(b, cudaGraphLaunch(b->graph_exec, b->stream));
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_batch_create(int32_t num_graphs, const int32_t* n, const int64_t* m, const int32_t* src,
                       const int32_t* dst, const int32_t* w, uint32_t replicas, void* cuda_stream,
                       ising_batch** out) {
  if (out == nullptr) return ISING_EINVAL;
  *out = nullptr;
  if (num_graphs <= 0 || n == nullptr || m == nullptr) return ISING_EINVAL;
  if (replicas < 1 || replicas > 8) return ISING_EINVAL;
  ising_batch* b = new (std::nothrow) ising_batch();
  if (b == nullptr) return ISING_ENOMEM;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->num_graphs = num_graphs;
  b->replicas = static_cast<int>(replicas);
  std::vector<BatchGraph> graphs((size_t)num_graphs);
  std::vector<int32_t> row_ptr, adj, orig, class_pos, class_heavy;
  std::vector<int64_t> size_key((size_t)num_graphs);
  int64_t edge_off = 0, vtx = 0;
  int rc = ISING_OK;
  try {
    b->n.assign(n, n + num_graphs);
    b->total_weight.resize((size_t)num_graphs);
    b->pos.resize((size_t)num_graphs);
    b->vtx_base.resize((size_t)num_graphs);
    int64_t in_off = 0;
    for (int32_t gi = 0; gi < num_graphs && rc == ISING_OK; ++gi) {
      if (m[gi] < 0) {
        rc = ISING_EINVAL;
        break;
      }
      HostGraph hg;
      rc = isingx::build_host_graph(n[gi], m[gi], src ? src + in_off : nullptr,
                                    dst ? dst + in_off : nullptr, w ? w + in_off : nullptr, &hg);
      in_off += m[gi];
      if (rc != ISING_OK) break;
      if (!hg.fits_int8 || hg.n >= (1 << 24) - 1) {
        rc = ISING_ERANGE;
        break;
      }
      if (vtx + hg.n >= (int64_t(1) << 31) || edge_off + hg.nnz >= (int64_t(1) << 31)) {
        rc = ISING_ERANGE;
        break;
      }
      BatchGraph& G = graphs[(size_t)gi];
      G.n = hg.n;
      G.num_classes = hg.num_colours;
      G.vtx_base = static_cast<int32_t>(vtx);
      G.row_base = static_cast<int32_t>(row_ptr.size());
      G.class_base = static_cast<int32_t>(class_pos.size());
      int64_t wmax = 0;  // largest |w|
      for (size_t k = 0; k < (size_t)hg.nnz; ++k)
        wmax = std::max<int64_t>(wmax, std::abs(static_cast<int64_t>(hg.w[k])));
      const bool unit = wmax <= 1;  // every weight +1 or -1 (merged weights are never 0)
      // byte lanes hold sums up to 255: a light row has degree * max|w| <= 255
      G.byte_lanes = unit ? 2 : (wmax <= 31 ? 1 : 0);
      const int64_t heavy_deg = unit ? 255 : (wmax <= 31 ? 255 / std::max<int64_t>(wmax, 1) : 64);
      G.flush = static_cast<int32_t>(G.byte_lanes ? heavy_deg : 0);
      for (int32_t c = 0; c < hg.num_colours; ++c) {
        const int32_t cb = hg.class_begin[(size_t)c], ce = hg.class_begin[(size_t)c + 1];
        int32_t hb = cb;  // one past the class's last heavy row
        for (int32_t p = cb; p < ce; ++p)
          if (hg.row_ptr[(size_t)p + 1] - hg.row_ptr[(size_t)p] > heavy_deg) hb = p + 1;
        class_heavy.push_back(hb);
      }
      class_heavy.push_back(hg.n);  // same layout as the class bounds
      for (size_t v = 0; v <= (size_t)hg.n; ++v)
        row_ptr.push_back(static_cast<int32_t>(edge_off + hg.row_ptr[v]));
      for (size_t k = 0; k < (size_t)hg.nnz; ++k)
        adj.push_back(static_cast<int32_t>((static_cast<uint32_t>(hg.col[k]) << 8) |
                                           (static_cast<uint32_t>(hg.w[k]) & 0xffu)));
      orig.insert(orig.end(), hg.perm.begin(), hg.perm.end());
      class_pos.insert(class_pos.end(), hg.class_begin.begin(), hg.class_begin.end());
      b->total_weight[(size_t)gi] = hg.total_weight;
      b->pos[(size_t)gi] = hg.pos;
      b->vtx_base[(size_t)gi] = G.vtx_base;
      b->max_n = std::max(b->max_n, hg.n);
      size_key[(size_t)gi] = hg.nnz + hg.n;
      edge_off += hg.nnz;
      vtx += hg.n;
    }
    b->total_nnz = edge_off;
  } catch (const std::bad_alloc&) {
    rc = ISING_ENOMEM;
  }
  if (rc == ISING_OK && b->max_n > 200 * 1024) rc = ISING_ERANGE;  // spins must fit in shared memory
  if (rc != ISING_OK) {
    delete b;
    return rc;
  }
  std::vector<int32_t> order((size_t)num_graphs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t c) { return size_key[(size_t)a] > size_key[(size_t)c]; });
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ISING_ECUDA;
  }
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (b->num_sms < 1) b->num_sms = 1;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = upload(&b->d_graphs, graphs, b->stream)) != cudaSuccess) break;
    if ((e = upload(&b->d_order, order, b->stream)) != cudaSuccess) break;
    if ((e = upload(&b->d_row_ptr, row_ptr, b->stream)) != cudaSuccess) break;
    if ((e = upload(&b->d_adj, adj, b->stream)) != cudaSuccess) break;
    if ((e = upload(&b->d_orig, orig, b->stream)) != cudaSuccess) break;
    if ((e = upload(&b->d_class_pos, class_pos, b->stream)) != cudaSuccess) break;
    if ((e = upload(&b->d_class_heavy, class_heavy, b->stream)) != cudaSuccess) break;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_spins), std::max<int64_t>(vtx, 16))) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(b->d_spins, 0, std::max<int64_t>(vtx, 16), b->stream)) != cudaSuccess) break;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_flips), std::max<int64_t>(vtx, 16))) != cudaSuccess) break;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_work), 16)) != cudaSuccess) break;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_energy2),
                        sizeof(long long) * (size_t)num_graphs * replicas)) != cudaSuccess) break;
    e = cudaStreamSynchronize(b->stream);
  } while (false);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? ISING_ENOMEM : ISING_ECUDA;
  }
  *out = b;
  return ISING_OK;
}

}  // extern "C"

namespace isingx {

int batch_union(ising_batch* b, BatchUnion* out) {
  const int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  const int32_t n = b->vtx_base.back() + b->n.back();
  if (b->d_union_row_ptr == nullptr) {
    BATCH_CUDA(b, cudaMalloc(reinterpret_cast<void**>(&b->d_union_row_ptr), sizeof(int32_t) * (size_t(n) + 1)));
    BATCH_CUDA(b, cudaMalloc(reinterpret_cast<void**>(&b->d_union_vbase), sizeof(int32_t) * std::max<size_t>(n, 1)));
    union_rows_kernel<<<std::min(b->num_graphs, b->num_sms * 8), 256, 0, b->stream>>>(
        b->d_graphs, b->d_row_ptr, b->num_graphs, b->d_union_row_ptr, b->d_union_vbase);
    b->launches++;
    BATCH_CUDA(b, cudaGetLastError());
    const int32_t end = static_cast<int32_t>(b->total_nnz);
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_union_row_ptr + n, &end, sizeof(int32_t), cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  }
  out->device = b->device;
  out->stream = b->stream;
  out->num_sms = b->num_sms;
  out->n = n;
  out->nnz = b->total_nnz;
  out->replicas = b->replicas;
  out->row_ptr = b->d_union_row_ptr;
  out->adj = b->d_adj;
  out->vbase = b->d_union_vbase;
  out->orig = b->d_orig;
  out->spins = b->d_spins;
  out->rowid = &b->d_gnn_rowid;
  out->hchunk = &b->d_gnn_hchunk;
  out->chunk_row = &b->d_gnn_chunk_row;
  out->num_chunks = &b->gnn_num_chunks;
  return ISING_OK;
}

}  // namespace isingx

extern "C" {

void ising_batch_destroy(ising_batch* b) {
  if (b == nullptr) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  cudaGetLastError();
  batch_free(b);
  delete b;
}

int ising_batch_init_random(ising_batch* b, uint64_t seed) {
  int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  batch_init_kernel<<<b->num_graphs, 256, 0, b->stream>>>(
      b->dev(), static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), b->replicas);
  b->launches++;
  BATCH_CUDA(b, cudaGetLastError());
  return ISING_OK;
}

int ising_batch_anneal(ising_batch* b, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                       void* cuda_stream) {
  int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  if (sched == nullptr || sched->kind != ISING_SCHED_LINEAR) return ISING_EINVAL;
  if (!(sched->p0 >= 0.0 && sched->p0 <= 1.0)) return ISING_EINVAL;
  if (sched->t_total >= (1ull << 32)) return ISING_EINVAL;
  if (sched->t_begin > sched->t_total || sweeps > sched->t_total - sched->t_begin) return ISING_EINVAL;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (sweeps == 0) return ISING_OK;
  return batch_launch(b, sched->t_begin, sweeps, sched->t_total, batch_t0(sched->p0), seed);
}

int ising_batch_cuts(ising_batch* b, int64_t* out_cuts) {
  int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  if (out_cuts == nullptr) return ISING_EINVAL;
  batch_energy_kernel<<<b->num_graphs, 256, 0, b->stream>>>(b->dev(), b->replicas, b->d_energy2);
  b->launches++;
  BATCH_CUDA(b, cudaGetLastError());
  std::vector<long long> e2((size_t)b->num_graphs * b->replicas);
  BATCH_CUDA(b, cudaMemcpyAsync(e2.data(), b->d_energy2, e2.size() * sizeof(long long),
                                cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  for (int32_t gi = 0; gi < b->num_graphs; ++gi)
    for (int r = 0; r < b->replicas; ++r) {
      const size_t k = (size_t)gi * b->replicas + r;
      out_cuts[k] = (b->total_weight[(size_t)gi] - e2[k] / 2) / 2;
    }
  return ISING_OK;
}

int ising_batch_get_spins(ising_batch* b, int32_t graph, uint32_t replica, int8_t* out) {
  int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  if (out == nullptr || graph < 0 || graph >= b->num_graphs || replica >= (uint32_t)b->replicas)
    return ISING_EINVAL;
  const int32_t nn = b->n[(size_t)graph];
  std::vector<uint8_t> bytes((size_t)nn);
  BATCH_CUDA(b, cudaMemcpyAsync(bytes.data(), b->d_spins + b->vtx_base[(size_t)graph], (size_t)nn,
                                cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  const std::vector<int32_t>& pos = b->pos[(size_t)graph];
  for (int32_t v = 0; v < nn; ++v) out[v] = ((bytes[(size_t)pos[(size_t)v]] >> replica) & 1) ? -1 : 1;
  return ISING_OK;
}

int ising_batch_set_spins(ising_batch* b, int32_t graph, uint32_t replica, const int8_t* in) {
  int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  if (in == nullptr || graph < 0 || graph >= b->num_graphs || replica >= (uint32_t)b->replicas)
    return ISING_EINVAL;
  const int32_t nn = b->n[(size_t)graph];
  for (int32_t v = 0; v < nn; ++v)
    if (in[v] != 1 && in[v] != -1) return ISING_EINVAL;
  std::vector<uint8_t> bytes((size_t)nn);
  uint8_t* dptr = b->d_spins + b->vtx_base[(size_t)graph];
  BATCH_CUDA(b, cudaMemcpyAsync(bytes.data(), dptr, (size_t)nn, cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  const std::vector<int32_t>& pos = b->pos[(size_t)graph];
  for (int32_t v = 0; v < nn; ++v) {
    uint8_t& x = bytes[(size_t)pos[(size_t)v]];
    x = static_cast<uint8_t>((x & ~(1u << replica)) | ((in[v] < 0 ? 1u : 0u) << replica));
  }
  BATCH_CUDA(b, cudaMemcpyAsync(dptr, bytes.data(), (size_t)nn, cudaMemcpyHostToDevice, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  return ISING_OK;
}

int ising_batch_autotune(ising_batch* b, uint32_t probe_sweeps, int32_t* out_block) {
  int rc = batch_enter(b);
  if (rc != ISING_OK) return rc;
  if (probe_sweeps == 0) probe_sweeps = 1;
  // time every configuration (block size x threads per row x tail mode) on
  // the batch itself, then restore the spins
  const int64_t total = b->vtx_base.empty() ? 0 : b->vtx_base.back() + b->n.back();
  uint8_t* saved = nullptr;
  BATCH_CUDA(b, cudaMalloc(reinterpret_cast<void**>(&saved), std::max<int64_t>(total, 16)));
  cudaError_t e = cudaMemcpyAsync(saved, b->d_spins, (size_t)total, cudaMemcpyDeviceToDevice, b->stream);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  float best_ms = 1e30f;
  int best = 0;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  for (int cfg = 0; cfg < kTuneConfigs && e == cudaSuccess; ++cfg) {
    b->block = kBlockChoices[cfg / 6];
    b->split = kSplitChoices[(cfg / 2) % 3];
    b->tail = kTailChoices[cfg % 2];
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms the captured graph
      e = cudaEventRecord(t0, b->stream);
      if (e == cudaSuccess && batch_launch(b, 0, probe_sweeps, probe_sweeps + 1, batch_t0(0.1), 1) != ISING_OK)
        e = cudaErrorUnknown;
      if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    b->probe_ms[cfg] = ms;
    if (e == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = cfg;
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_spins, saved, (size_t)total, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(saved);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->status = ISING_ECUDA;
    return ISING_ECUDA;
  }
  b->block = kBlockChoices[best / 6];
  b->split = kSplitChoices[(best / 2) % 3];
  b->tail = kTailChoices[best % 2];
  if (out_block) *out_block = b->block;
  return ISING_OK;
}

int ising_batch_set_block(ising_batch* b, int32_t block) {
  if (b == nullptr) return ISING_EINVAL;
  if (block != 128 && block != 256 && block != 512) return ISING_EINVAL;
  b->block = block;
  return ISING_OK;
}

int ising_batch_set_tuning(ising_batch* b, int32_t block, int32_t row_split, int32_t tail) {
  if (b == nullptr) return ISING_EINVAL;
  if (block != 128 && block != 256 && block != 512) return ISING_EINVAL;
  if (row_split != 1 && row_split != 2 && row_split != 4) return ISING_EINVAL;
  if (tail < 0 || tail > 32) return ISING_EINVAL;
  b->block = block;
  b->split = row_split;
  b->tail = tail;
  return ISING_OK;
}

int ising_batch_tuning(ising_batch* b, int32_t* out_block, int32_t* out_row_split, int32_t* out_tail,
                       float* out_probe_ms) {
  if (b == nullptr) return ISING_EINVAL;
  if (out_block) *out_block = b->block;
  if (out_row_split) *out_row_split = b->split;
  if (out_tail) *out_tail = b->tail;
  if (out_probe_ms)
    for (int k = 0; k < kTuneConfigs; ++k) out_probe_ms[k] = b->probe_ms[k];
  return ISING_OK;
}

int ising_batch_info(ising_batch* b, int32_t* out_num_graphs, int64_t* out_vertices,
                     int32_t* out_block, uint64_t* out_launches) {
  if (b == nullptr) return ISING_EINVAL;
  if (out_num_graphs) *out_num_graphs = b->num_graphs;
  if (out_vertices) *out_vertices = b->vtx_base.empty() ? 0 : b->vtx_base.back() + b->n.back();
  if (out_block) *out_block = b->block;
  if (out_launches) *out_launches = b->launches;
  return ISING_OK;
}

}  // extern "C"
