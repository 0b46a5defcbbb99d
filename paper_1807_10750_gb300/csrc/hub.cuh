// Hub engine: one cooperative launch per anneal call for graphs with hubs
// (vertices of at least ISING_HUB_DEGREE neighbours, ising.h).
//
// The two-tier colouring puts the hubs in colour classes of their own, swept
// first: classes 0 .. m-1 hold hubs only, classes m .. C-1 the other vertices.
// On a power-law graph the hubs form a near-clique, so m is large (83 on the
// 2^20-vertex workload) while each hub class is small (2 to 400 vertices);
// the other classes are few (11) and large. A grid barrier per class would
// cost ~1.4 us 94 times per sweep. Here block 0 (the chain block) runs all m
// hub classes alone, with block barriers between them, and the other blocks
// (the workers) run the other classes with a grid barrier after each.
//
// The chain block keeps, in shared memory, every hub's state byte and its
// field split in two parts (Eq. 2): f_v = A_v + B_v, with A_v the sum of
// w_vu s_u over the non-hub neighbours u and B_v the sum over the hub
// neighbours. Within a sweep the non-hub spins do not change while the hubs
// are updated (their classes come later), so A_v is summed once per sweep by
// the workers. B_v is kept current incrementally: when hub u changes from -s
// to s, every hub neighbour v gets B_v += 2 w_uv s, one shared-memory atomic
// per entry of u's hub row, before the next class is decided. Only the rows
// of hubs that change are read, a few hundred per sweep.
//
// One sweep t:
//   1. workers: A_v for every hub from the current non-hub spins (and, in the
//      launch's first sweep, B_v from the hub spins), added into a global
//      array with atomics; the chain's flip bits of sweep t (Algorithm 2's
//      draws, optional flip bias); then they arrive at the grid barrier;
//   2. chain block: waits for every worker's arrival, loads A (and B), runs
//      the m hub classes (decide from A_v + B_v, flip, write the state byte,
//      push the changed hubs' rows into B), arrives at the barrier;
//   3. workers: the non-hub classes m .. C-1 with the sweep kernels' work
//      items (sweep.cuh), reading the hubs' new spins; a grid barrier after
//      each class (the chain block only arrives and waits).
// Every wait is bounded (sweep.cuh, barrier_wait).
#pragma once

#include <cstdint>

#include "host_graph.h"
#include "philox.cuh"
#include "sweep.cuh"

namespace isingx {

constexpr int kHubBlock = 512;
constexpr int kHubWarps = kHubBlock / 32;
constexpr int kHubMaxHubs = 10240;  // shared memory of the chain block (hub_smem_bytes)
constexpr int kHubSumChunk = 512;   // CSR entries per field-sum item
constexpr int kHubPiece = 256;      // entries of a changed hub's row pushed by one warp task

struct HubArgs {
  int32_t hubs;         // X: hubs hold positions [0, X)
  int32_t hub_classes;  // m
  int32_t classes;      // C
  const int32_t* class_begin;  // C + 1 first positions
  const int32_t* class_items;  // C + 1 first work items
  const int32_t* hub_end;      // per hub: first CSR entry of its row past the hubs
  const int4* sums;            // field-sum items (hub, first entry, end entry, 0 = A / 1 = B)
  int32_t num_b_items;         // items [0, num_b_items) sum B, the rest A
  int32_t num_items;
  int32_t* acc;                // [0, X): A sums, [X, 2X): B sums; zero between uses
  uint32_t* flips;             // ceil(X / 32) words: flip bits of the coming chain
};

// Shared memory of the chain block: A[X], B[X] (int32), the state bytes S[X]
// (padded to 4), the flip bits F[W], the class table cls[m + 1], the list of
// one step's changed hubs (kHubBlock int4) and two step counters.
__host__ __device__ inline int hub_smem_bytes(int X, int m) {
  const int W = (X + 31) / 32;
  return 8 * X + ((X + 3) / 4) * 4 + 4 * W + 4 * (m + 1) + 16 * kHubBlock + 8 + 16;
}

struct HubSmem {
  int32_t* A;
  int32_t* B;
  uint8_t* S;
  uint32_t* F;
  int32_t* cls;
  int4* list;
  int* cnt;
};

__device__ __forceinline__ HubSmem hub_smem(unsigned char* base, int X, int m) {
  HubSmem s;
  const int W = (X + 31) / 32;
  int4* list = reinterpret_cast<int4*>(base);  // 16-byte aligned first
  s.list = list;
  s.A = reinterpret_cast<int32_t*>(list + kHubBlock);
  s.B = s.A + X;
  s.F = reinterpret_cast<uint32_t*>(s.B + X);
  s.cls = reinterpret_cast<int32_t*>(s.F + W);
  s.cnt = s.cls + (m + 1);
  s.S = reinterpret_cast<uint8_t*>(s.cnt + 2);
  return s;
}

// Field-sum item i: sum of w * s over CSR entries [e0, e1) of hub u, added
// into acc[kind * X + u]. Eight loads in flight per lane.
template <bool PACKED>
__device__ __forceinline__ void hub_sum_item(const DevGraph& d, const HubArgs& h, int i, int lane) {
  const int4 it = __ldg(h.sums + i);
  int f = 0;
  for (int e = it.y + lane; e < it.z; e += 32 * 8) {
    Edge<PACKED> x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u].load(d, e + 32 * u, e + 32 * u < it.z);
    int b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) b[u] = d.spins[x[u].col()];
#pragma unroll
    for (int u = 0; u < 8; ++u) f += x[u].weight() * spin_of(b[u]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
  if (lane == 0 && f != 0) atomicAdd(h.acc + it.w * h.hubs + it.x, f);
}

// Flip bits of hubs 32 j .. 32 j + 31 in sweep a.t (Algorithm 2; the flip
// bias scales the threshold as in flip_drawn).
__device__ __forceinline__ void hub_flip_word(const DevGraph& d, const HubArgs& h, int j,
                                              const SweepArgs& a, const PhiloxRounds& rk,
                                              int lane) {
  const int v = 32 * j + lane;
  bool flip = false;
  if (v < h.hubs) flip = flip_drawn(d, v, static_cast<uint32_t>(__ldg(d.orig + v)), a, rk);
  const unsigned bits = __ballot_sync(kFullMask, flip);
  if (lane == 0) h.flips[j] = bits;
}

// Push hub u's change (new spin ns) into B of its hub neighbours: entries
// [e0, e1) of its row. Piece p of list entry k (kHubPiece entries) belongs to
// warp (k + p) mod kHubWarps, so a few changed hubs with long rows still
// spread over every warp.
template <bool PACKED>
__device__ __forceinline__ void hub_push(const DevGraph& d, const HubSmem& s, int K, int warp,
                                         int lane) {
  for (int k = 0; k < K; ++k) {
    const int4 e = s.list[k];  // (u, new spin, first entry, end entry)
    const int pieces = (e.w - e.z + kHubPiece - 1) / kHubPiece;
    int p = (warp - k) % kHubWarps;
    if (p < 0) p += kHubWarps;
    for (; p < pieces; p += kHubWarps) {
      const int e0 = e.z + p * kHubPiece;
      const int e1 = min(e.w, e0 + kHubPiece);
      Edge<PACKED> x[kHubPiece / 32];
#pragma unroll
      for (int i = 0; i < kHubPiece / 32; ++i) x[i].load(d, e0 + lane + 32 * i, e0 + lane + 32 * i < e1);
#pragma unroll
      for (int i = 0; i < kHubPiece / 32; ++i)
        if (e0 + lane + 32 * i < e1) atomicAdd(s.B + x[i].col(), 2 * e.y * x[i].weight());
    }
  }
}

// The m hub classes of one sweep, run by the chain block. `first`: the
// launch's first sweep (B and the state bytes are loaded from global memory).
// `step` counts decision steps across the launch (it selects the counter of
// the step's changed list).
template <bool PACKED>
__device__ __forceinline__ void hub_chain(const DevGraph& d, const HubArgs& h, const HubSmem& s,
                                          bool first, int& step) {
  const int X = h.hubs, m = h.hub_classes;
  const int W = (X + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = threadIdx.x; v < X; v += kHubBlock) {
    s.A[v] = h.acc[v];
    h.acc[v] = 0;
    if (first) {
      s.B[v] = h.acc[X + v];
      h.acc[X + v] = 0;
      s.S[v] = static_cast<uint8_t>(d.spins[v]);
    }
  }
  for (int j = threadIdx.x; j < W; j += kHubBlock) s.F[j] = h.flips[j];
  if (first)
    for (int c = threadIdx.x; c <= m; c += kHubBlock) s.cls[c] = __ldg(h.class_begin + c);
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    const int cb = s.cls[c], ce = s.cls[c + 1];
    for (int base = cb; base < ce; base += kHubBlock) {
      const int v = base + static_cast<int>(threadIdx.x);
      bool changed = false;
      int ns = 0, e0 = 0, e1 = 0;
      if (v < ce) {
        e0 = __ldg(d.row_ptr + v);
        e1 = __ldg(h.hub_end + v);
        const int b = s.S[v];
        const int sv = spin_of(b);
        const int f = s.A[v] + s.B[v];
        ns = sv;
        if (f > 0)
          ns = -1;
        else if (f < 0)
          ns = 1;
        if ((s.F[v >> 5] >> (v & 31)) & 1u) ns = -ns;
        const int nb = state_byte(ns, ((b >> 1) & 1) ^ 1);
        s.S[v] = static_cast<uint8_t>(nb);
        d.spins[v] = static_cast<int8_t>(nb);
        changed = ns != sv && e1 > e0;
      }
      const unsigned ball = __ballot_sync(kFullMask, changed);
      int at = 0;
      if (lane == 0 && ball != 0u) at = atomicAdd(s.cnt + (step & 1), __popc(ball));
      at = __shfl_sync(kFullMask, at, 0);
      if (changed) s.list[at + __popc(ball & ((1u << lane) - 1u))] = make_int4(v, ns, e0, e1);
      if (threadIdx.x == 0) s.cnt[(step + 1) & 1] = 0;
      __syncthreads();
      const int K = s.cnt[step & 1];
      ++step;
      if (K == 0) continue;
      hub_push<PACKED>(d, s, K, warp, lane);
      __syncthreads();
    }
  }
}

template <bool PACKED>
__global__ void __launch_bounds__(kHubBlock, 2)
    hub_kernel(DevGraph d, HubArgs h, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
               uint32_t replica, PhiloxRounds rk, BarrierState* bs) {
  extern __shared__ __align__(16) unsigned char hub_shared[];
  const int lane = threadIdx.x & 31;
  const bool chain = blockIdx.x == 0;
  const int warp = (static_cast<int>(blockIdx.x) - 1) * kHubWarps + static_cast<int>(threadIdx.x >> 5);
  const int nwarps = (static_cast<int>(gridDim.x) - 1) * kHubWarps;
  const int W = (h.hubs + 31) / 32;
  HubSmem s = hub_smem(hub_shared, h.hubs, h.hub_classes);
  if (chain && threadIdx.x < 2) s.cnt[threadIdx.x] = 0;
  bool skip = bs->skip_block == static_cast<int>(blockIdx.x) + 1;
  unsigned target = 0;
  int step = 0;
  long long unused = 0;
  for (uint32_t k = 0; k < sweeps; ++k) {
    const SweepArgs a = sweep_args(t_begin + k, T, T0, replica);
    target += gridDim.x;
    if (!chain) {
      // 1. the hubs' field sums and flip bits of sweep t
      for (int i = (k == 0 ? 0 : h.num_b_items) + warp; i < h.num_items; i += nwarps)
        hub_sum_item<PACKED>(d, h, i, lane);
      for (int j = warp; j < W; j += nwarps) hub_flip_word(d, h, j, a, rk, lane);
      barrier_arrive(bs, skip);
      skip = false;
    } else {
      // 2. the hub classes, once every worker has arrived
      if (!barrier_wait(bs, target - 1)) return;
      hub_chain<PACKED>(d, h, s, k == 0, step);
      barrier_arrive(bs, skip);
      skip = false;
    }
    if (!barrier_wait(bs, target)) return;
    // 3. the other classes
    for (int c = h.hub_classes; c < h.classes; ++c) {
      if (!chain) {
        const int ie = __ldg(h.class_items + c + 1);
        for (int i = __ldg(h.class_items + c) + warp; i < ie; i += nwarps) {
          Staged<PACKED> st;
          stage_item<PACKED>(d, d.items[i], a, rk, lane, st);
          finish_item<PACKED, kPassDet>(d, st, a, rk, lane, unused);
        }
      }
      if (c + 1 == h.classes && k + 1 == sweeps) break;
      barrier_arrive(bs, skip);
      skip = false;
      target += gridDim.x;
      if (!barrier_wait(bs, target)) return;
    }
  }
}

}  // namespace isingx
