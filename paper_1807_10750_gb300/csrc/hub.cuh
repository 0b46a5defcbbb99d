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
// per entry of u's hub row. Only the entries into later hub classes are
// pushed before the next class is decided; those into earlier classes are
// needed only in the next sweep and are pushed while the workers run the
// other classes.
//
// Spins during a launch live in a bit map (bit p set for spin -1), with one
// copy in global memory and, when it fits, one in every worker block's shared
// memory. The vertices of a class hold a contiguous range of positions, so
// after each grid barrier a worker block refreshes only the words of the
// class just updated, and every neighbour read of a sweep is a shared-memory
// read instead of a random L2 access. New spins go to the global map: the
// warp that decides 32 consecutive positions xors their changed bits in with
// at most two atomics. The state bytes are rebuilt from the map once, at the
// end of the launch (every vertex's update parity has flipped once per sweep).
//
// One sweep t:
//   1. workers: A_v for every hub from the non-hub spins (and, in the
//      launch's first sweep, B_v from the hub spins), added into a global
//      array with atomics; the chain's flip bits of sweep t (Algorithm 2's
//      draws, optional flip bias); then they arrive at the grid barrier;
//   2. chain block: waits for every worker's arrival, loads A (and B), runs
//      the m hub classes, arrives at the barrier, then pushes the deferred
//      entries;
//   3. workers: refresh the hub words of their map copy, then the non-hub
//      classes m .. C-1 from the sweep's work items, a workers-only grid
//      barrier and a refresh of the class's words after each.
// Every wait is bounded (sweep.cuh, barrier_wait).
#pragma once

#include <cstdint>

#include "host_graph.h"
#include "philox.cuh"
#include "sweep.cuh"

namespace isingx {

constexpr int kHubBlock = 1024;
constexpr int kHubWarps = kHubBlock / 32;
constexpr int kHubMaxHubs = 10240;  // shared memory of the chain block (hub_smem_bytes)
constexpr int kHubSumChunk = 512;   // CSR entries per field-sum item
constexpr int kHubSlot = 128;       // row entries per push task (4 per lane)
constexpr int kHubListCap = 3072;   // push tasks one block-wide decision step can list
constexpr int kHubDeferCap = 2048;  // changed hubs whose earlier-class pushes wait
constexpr int kHubSmallClass = 32;  // classes up to this size are decided by warp 0 alone
constexpr int kHubSmallWarps = 4;   // warps that push a small class's changes
constexpr int kHubGroupLoads = 8;   // CSR words in flight per lane in a group-row batch
constexpr int kHubGroupScratch = 65;  // per warp: 33 row offsets and 32 fields

struct HubArgs {
  int32_t hubs;         // X: hubs hold positions [0, X)
  int32_t hub_classes;  // m
  int32_t classes;      // C
  const int32_t* class_begin;  // C + 1 first positions
  const int32_t* class_items;  // C + 1 first work items
  const int32_t* hub_split;    // per hub: first CSR entry of its row in a later hub class
  const int32_t* hub_end;      // per hub: first CSR entry of its row past the hubs
  const int4* sums;            // field-sum items (hub, first entry, end entry, 0 = A / 1 = B)
  int32_t num_b_items;         // items [0, num_b_items) sum B, the rest A
  int32_t num_items;
  int32_t* acc;                // [0, X) and [X, 2X): A by sweep parity, [2X, 3X): B; zero
                               // between uses
  uint32_t* flips;             // ceil(X / 32) words: flip bits of the coming chain
  uint32_t* bits;              // the spin map: bit p of word p / 32 set for spin -1 (the pad
                               // position n reads 0); bit_words words, zero at launch
  int32_t bit_words;
  int32_t stage_bits;          // 1: worker blocks keep a copy of the map in shared memory
  int32_t par_end;             // update parity of every state byte after the launch
  uint32_t* pflips;            // the sweep's flips by position (bit_words words)
  const int32_t* pos;          // original id -> position
  const int32_t* blk;          // per non-hub class: G first items of the worker blocks + end
};

// Shared memory. The chain block: the push tasks of one block-wide step
// (kHubListCap int4: hub | sign << 31, first entry, end entry, unused), the
// changed hubs of a small class (kHubSmallClass int4: first entry, end entry,
// new spin, unused), the deferred hubs (kHubDeferCap int: hub | sign << 31), the fields F[X] = A + B
// (int32), the flip bits fl[W], the class table cls[m + 1], four counters and
// the state bytes S[X]. A worker block: the group-row scratch (kHubWarps x
// kHubGroupScratch int) and, with stage_bits, the copy of the spin map.
__host__ __device__ inline int hub_chain_smem(int X, int m) {
  const int W = (X + 31) / 32;
  return 16 * kHubListCap + 16 * kHubSmallClass + 4 * kHubDeferCap + 4 * X + 4 * W + 4 * (m + 1) + 16 +
         ((X + 3) / 4) * 4 + 16;
}
__host__ __device__ inline int hub_worker_smem(int bit_words, bool stage) {
  return 4 * kHubWarps * kHubGroupScratch + 16 + (stage ? 4 * bit_words : 0) + 16;
}
__host__ __device__ inline int hub_smem_bytes(int X, int m, int bit_words, bool stage) {
  const int c = hub_chain_smem(X, m), w = hub_worker_smem(bit_words, stage);
  return c > w ? c : w;
}

struct HubSmem {
  int4* list;
  int4* small;
  int32_t* defer;
  int32_t* F;
  uint32_t* fl;
  int32_t* cls;
  int* cnt;  // [0], [1]: push tasks of a block-wide step, by step parity; [2]: deferred hubs;
             // [3]: changed hubs of a small class
  uint8_t* S;
};

__device__ __forceinline__ HubSmem hub_smem(unsigned char* base, int X, int m) {
  HubSmem s;
  const int W = (X + 31) / 32;
  s.list = reinterpret_cast<int4*>(base);  // 16-byte aligned first
  s.small = s.list + kHubListCap;
  s.defer = reinterpret_cast<int32_t*>(s.small + kHubSmallClass);
  s.F = s.defer + kHubDeferCap;
  s.fl = reinterpret_cast<uint32_t*>(s.F + X);
  s.cls = reinterpret_cast<int32_t*>(s.fl + W);
  s.cnt = s.cls + (m + 1);
  s.S = reinterpret_cast<uint8_t*>(s.cnt + 4);
  return s;
}

// Spin-map reads: the bit of position p (1 for spin -1) and the spin.
__device__ __forceinline__ int map_bit(const uint32_t* sb, int p) { return (sb[p >> 5] >> (p & 31)) & 1; }
__device__ __forceinline__ int map_spin(const uint32_t* sb, int p) { return 1 - 2 * map_bit(sb, p); }

// Lane l of the warp owns position p0 + l: xor the bits of the lanes whose
// spin changed into the global map (at most two words, one atomic each).
__device__ __forceinline__ void map_publish(uint32_t* g, int p0, bool changed, int lane) {
  const unsigned m = __ballot_sync(kFullMask, changed);
  if (lane == 0 && m != 0u) {
    const int w = p0 >> 5, sh = p0 & 31;
    atomicXor(g + w, m << sh);
    if (sh != 0 && (m >> (32 - sh)) != 0u) atomicXor(g + w + 1, m >> (32 - sh));
  }
}

// Eq. 2 under the max-cut sign (f > 0 gives -1, f < 0 gives +1, f = 0 keeps
// the spin), then Algorithm 2's flip, on map bits (1 = spin -1).
__device__ __forceinline__ int decide_bit(int f, int old, bool flip) {
  int b = old;
  if (f > 0)
    b = 1;
  else if (f < 0)
    b = 0;
  return flip ? b ^ 1 : b;
}

// Field-sum item i: sum of w * s over CSR entries [e0, e1) of hub u, added
// into the A array of sweep parity `par` (kind 0) or into B (kind 1). Eight
// loads in flight per lane.
template <bool PACKED>
__device__ __forceinline__ void hub_sum_item(const DevGraph& d, const HubArgs& h,
                                             const uint32_t* sb, int i, int par, int lane) {
  const int4 it = __ldg(h.sums + i);
  int f = 0;
  for (int e = it.y + lane; e < it.z; e += 32 * 8) {
    Edge<PACKED> x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u].load(d, e + 32 * u, e + 32 * u < it.z);
#pragma unroll
    for (int u = 0; u < 8; ++u) f += x[u].weight() * map_spin(sb, x[u].col());
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
  if (lane == 0 && f != 0) atomicAdd(h.acc + (it.w == 1 ? 2 : par) * h.hubs + it.x, f);
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

// Push entries [e0, e1) of a changed hub's row (at most kHubSlot of them,
// kHubSlot / 32 per lane, all loaded before any is applied): each entry (v, w) adds
// 2 w ns to F_v, ns the hub's new spin.
template <bool PACKED>
__device__ __forceinline__ void hub_push_range(const DevGraph& d, const HubSmem& s, int e0, int e1,
                                               int ns, int lane) {
  constexpr int U = kHubSlot / 32;
  Edge<PACKED> x[U];
#pragma unroll
  for (int i = 0; i < U; ++i) x[i].load(d, e0 + lane + 32 * i, e0 + lane + 32 * i < e1);
#pragma unroll
  for (int i = 0; i < U; ++i)
    if (e0 + lane + 32 * i < e1) atomicAdd(s.F + x[i].col(), 2 * ns * x[i].weight());
}

// A whole row range pushed by one warp, kHubSlot entries per round.
template <bool PACKED>
__device__ __forceinline__ void hub_push_rows(const DevGraph& d, const HubSmem& s, int e0, int e1,
                                              int ns, int lane) {
  for (int e = e0; e < e1; e += kHubSlot) hub_push_range<PACKED>(d, s, e, min(e1, e + kHubSlot), ns, lane);
}

// Bring hub row entries [e0, e1) into L2 (one prefetch per 128-byte line),
// so that the chain's pushes from them do not wait on HBM.
template <bool PACKED>
__device__ __forceinline__ void hub_prefetch(const DevGraph& d, int e0, int e1, int lane) {
  const int per_line = 32;  // int32 entries per 128-byte line
  for (int e = (e0 & ~(per_line - 1)) + lane * per_line; e < e1; e += 32 * per_line) {
    if (PACKED) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(d.adj + e));
    } else {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(d.col + e));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(d.w + e));
    }
  }
}

// The decision of hub v (Eq. 2 under the max-cut sign, then Algorithm 2's
// flip): returns the new spin and keeps the new state byte in shared memory
// (its update parity flips); the caller publishes the spin to the map.
__device__ __forceinline__ int hub_decide(const HubSmem& s, int v, int* old_spin) {
  const int b = s.S[v];
  const int sv = spin_of(b);
  const int f = s.F[v];
  int ns = sv;
  if (f > 0)
    ns = -1;
  else if (f < 0)
    ns = 1;
  if ((s.fl[v >> 5] >> (v & 31)) & 1u) ns = -ns;
  const int nb = state_byte(ns, ((b >> 1) & 1) ^ 1);
  s.S[v] = static_cast<uint8_t>(nb);
  *old_spin = sv;
  return ns;
}

// A changed hub whose row reaches earlier hub classes: queue it (its pushes
// there are needed only in the next sweep); push at once if the queue is full.
template <bool PACKED>
__device__ __forceinline__ void hub_defer(const DevGraph& d, const HubSmem& s, bool want, int v,
                                          int ns, int r0, int sp, int lane) {
  const unsigned ball = __ballot_sync(kFullMask, want);
  if (ball == 0u) return;
  int at = 0;
  if (lane == 0) at = atomicAdd(s.cnt + 2, __popc(ball));
  at = __shfl_sync(kFullMask, at, 0) + __popc(ball & ((1u << lane) - 1u));
  const bool full = want && at >= kHubDeferCap;
  if (want && !full) s.defer[at] = v | (ns < 0 ? static_cast<int>(0x80000000u) : 0);
  unsigned over = __ballot_sync(kFullMask, full);
  while (over != 0u) {
    const int src = __ffs(over) - 1;
    over &= over - 1;
    hub_push_rows<PACKED>(d, s, __shfl_sync(kFullMask, r0, src), __shfl_sync(kFullMask, sp, src),
                          __shfl_sync(kFullMask, ns, src), lane);
  }
}

// The pushes of the queued hubs into earlier hub classes, by the whole chain
// block while the other blocks run the non-hub classes: warp w takes queued
// hubs w, w + kHubWarps, ...
template <bool PACKED>
__device__ __forceinline__ void hub_deferred(const DevGraph& d, const HubArgs& h, const HubSmem& s,
                                             int warp, int lane) {
  const int nq = min(s.cnt[2], kHubDeferCap);
  for (int q = warp; q < nq; q += kHubWarps) {
    const int x = s.defer[q];
    const int u = x & 0x7fffffff;
    hub_push_rows<PACKED>(d, s, __ldg(d.row_ptr + u), __ldg(h.hub_split + u), x < 0 ? -1 : 1, lane);
  }
}

// The barrier of the warps that run the small hub classes (named barrier 1).
__device__ __forceinline__ void small_barrier() {
  asm volatile("bar.sync 1, %0;" ::"r"(32 * kHubSmallWarps) : "memory");
}

// The m hub classes of one sweep, run by the chain block. `first`: the
// launch's first sweep (B and the state bytes come from global memory).
// `step` counts block-wide decision steps (it selects the step's counter).
//
// Classes of at most kHubSmallClass hubs are decided by warp 0 alone and
// their changes pushed by kHubSmallWarps warps, with a named barrier of those
// warps only; larger classes use the whole block: decide, list the push tasks, block barrier, push, block
// barrier. Only the pushes into later hub classes are made here; the rest
// wait in the deferred queue (hub_deferred).
template <bool PACKED>
__device__ __forceinline__ void hub_chain(const DevGraph& d, const HubArgs& h, const HubSmem& s,
                                          uint32_t k, int& step) {
  const int X = h.hubs, m = h.hub_classes;
  const int W = (X + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int par = static_cast<int>(k & 1u);
  // F = A + B: the new A replaces the previous sweep's (both are in global
  // memory); the previous one is cleared for the next sweep's sums
  int32_t* a_new = h.acc + par * X;
  int32_t* a_old = h.acc + (par ^ 1) * X;
  for (int v = threadIdx.x; v < X; v += kHubBlock) {
    if (k == 0) {
      s.F[v] = a_new[v] + h.acc[2 * X + v];
      h.acc[2 * X + v] = 0;
      s.S[v] = static_cast<uint8_t>(d.spins[v]);
    } else {
      s.F[v] += a_new[v] - a_old[v];
      a_old[v] = 0;
    }
  }
  for (int j = threadIdx.x; j < W; j += kHubBlock) s.fl[j] = h.flips[j];
  if (k == 0)
    for (int c = threadIdx.x; c <= m; c += kHubBlock) s.cls[c] = __ldg(h.class_begin + c);
  if (threadIdx.x == 0) s.cnt[2] = 0;
  __syncthreads();
  // Steps: class c, hubs [base, base + kHubBlock). Each thread loads its hub's
  // row bounds one step ahead, so no global load waits before a decision.
  int c = 0, base = s.cls[0];
  int r0n = 0, spn = 0, hen = 0;
  if (m > 0 && base + static_cast<int>(threadIdx.x) < s.cls[1]) {
    r0n = __ldg(d.row_ptr + base + threadIdx.x);
    spn = __ldg(h.hub_split + base + threadIdx.x);
    hen = __ldg(h.hub_end + base + threadIdx.x);
  }
  bool small_run = false;  // warp 0 has decided small classes since the last block barrier
  while (c < m) {
    const int cb = s.cls[c];
    const int ce = s.cls[c + 1];
    const int v = base + static_cast<int>(threadIdx.x);
    const int r0 = r0n, sp = spn, he = hen;
    const bool small = ce - cb <= kHubSmallClass;
    int nc = c, nbase = base + kHubBlock;
    if (nbase >= ce) {
      nc = c + 1;
      nbase = ce;  // class c + 1 starts where class c ends
    }
    if (nc < m && nbase + static_cast<int>(threadIdx.x) < s.cls[nc + 1]) {
      r0n = __ldg(d.row_ptr + nbase + threadIdx.x);
      spn = __ldg(h.hub_split + nbase + threadIdx.x);
      hen = __ldg(h.hub_end + nbase + threadIdx.x);
    }
    c = nc;
    base = nbase;
    if (small) {
      // warp 0 decides (one hub per lane); warps 0 .. kHubSmallWarps - 1 push
      // the changed hubs' entries into later classes, one hub per warp at a
      // time; a named barrier of those warps on either side of the pushes
      if (warp < kHubSmallWarps) {
        if (warp == 0) {
          int ns = 0, sv = 0;
          if (v < ce) ns = hub_decide(s, v, &sv);
          const bool changed = v < ce && ns != sv;
          map_publish(h.bits, cb, changed, lane);
          const bool later = changed && he > sp;
          const unsigned ch = __ballot_sync(kFullMask, later);
          if (later) s.small[__popc(ch & ((1u << lane) - 1u))] = make_int4(sp, he, ns, 0);
          if (lane == 0) s.cnt[3] = __popc(ch);
          hub_defer<PACKED>(d, s, changed && sp > r0, v, ns, r0, sp, lane);
        }
        small_barrier();
        const int nch = s.cnt[3];
        for (int k = warp; k < nch; k += kHubSmallWarps) {
          const int4 t = s.small[k];
          hub_push_rows<PACKED>(d, s, t.x, t.y, t.z, lane);
        }
        small_barrier();
      }
      small_run = true;
      continue;
    }
    if (small_run) {  // warp 0's small classes are complete and visible
      __syncthreads();
      small_run = false;
    }
    int ns = 0, at = 0, ntask = 0;
    bool spill = false;
    if (v - lane < ce) {  // warps past the class's end skip the decision step
      int sv = 0;
      if (v < ce) ns = hub_decide(s, v, &sv);
      const bool changed = v < ce && ns != sv;
      map_publish(h.bits, v - lane, changed, lane);  // the warp's 32 consecutive positions
      hub_defer<PACKED>(d, s, changed && sp > r0, v, ns, r0, sp, lane);
      // list the push tasks into later classes: one per kHubSlot entries; the
      // warp reserves its tasks with one atomic (exclusive scan of the counts)
      ntask = changed ? (he - sp + kHubSlot - 1) / kHubSlot : 0;
      int incl = ntask;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
      }
      const int warp_tasks = __shfl_sync(kFullMask, incl, 31);
      if (lane == 0 && warp_tasks != 0) at = atomicAdd(s.cnt + (step & 1), warp_tasks);
      at = __shfl_sync(kFullMask, at, 0) + incl - ntask;
      // tasks past the list's capacity stay with the deciding lane
      for (int j = 0; j < ntask; ++j) {
        if (at + j < kHubListCap)
          s.list[at + j] = make_int4(v | (ns < 0 ? static_cast<int>(0x80000000u) : 0),
                                     sp + j * kHubSlot, min(he, sp + (j + 1) * kHubSlot), 0);
        else
          spill = true;
      }
    }
    if (threadIdx.x == 0) s.cnt[(step + 1) & 1] = 0;
    __syncthreads();
    const int Q = s.cnt[step & 1];
    ++step;
    if (Q == 0) continue;
    for (int q = warp; q < min(Q, kHubListCap); q += kHubWarps) {
      const int4 e = s.list[q];
      hub_push_range<PACKED>(d, s, e.y, e.z, e.x < 0 ? -1 : 1, lane);
    }
    // rare: tasks that did not fit, pushed by the warp that decided them
    unsigned spw = __ballot_sync(kFullMask, spill);
    while (spw != 0u) {
      const int src = __ffs(spw) - 1;
      spw &= spw - 1;
      const int sat = __shfl_sync(kFullMask, at, src), sn = __shfl_sync(kFullMask, ntask, src);
      const int s0 = __shfl_sync(kFullMask, sp, src), s1 = __shfl_sync(kFullMask, he, src);
      const int sns = __shfl_sync(kFullMask, ns, src);
      for (int j = 0; j < sn; ++j)
        if (sat + j >= kHubListCap)
          hub_push_range<PACKED>(d, s, s0 + j * kHubSlot, min(s1, s0 + (j + 1) * kHubSlot), sns, lane);
    }
    __syncthreads();
  }
  if (small_run) __syncthreads();
}

// ---------------------------------------------------------------------------
// Worker items (the non-hub classes), on the spin map `sb` (the block's copy
// or the global map). New spins go to the global map; the flip of position p
// is bit p of the sweep's flip map.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool pos_flip(const HubArgs& h, const SweepArgs& a, int p) {
  return a.thr != 0u && ((h.pflips[p >> 5] >> (p & 31)) & 1u);
}

// Light rows (sliced ELL): every word of the item loaded before any is used.
template <bool PACKED, int R>
__device__ __forceinline__ void hub_light(const DevGraph& d, const HubArgs& h, const uint32_t* sb,
                                          const WorkItem& it, const SweepArgs& a, int lane) {
  constexpr int DM = light_slots(PACKED) / R;
  const int nv = it.v_end - it.v_begin;
  const int D = -it.e_end - 1;
  Edge<PACKED> x[R * DM];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = lane + 32 * r;
#pragma unroll
    for (int k = 0; k < DM; ++k) x[r * DM + k].load_ell(d, it.e_begin + k * nv + row, row < nv && k < D);
  }
  bool flip[R];
#pragma unroll
  for (int r = 0; r < R; ++r) flip[r] = lane + 32 * r < nv && pos_flip(h, a, it.v_begin + lane + 32 * r);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int f = 0;
#pragma unroll
    for (int k = 0; k < DM; ++k) f += x[r * DM + k].weight() * map_spin(sb, x[r * DM + k].col());
    const int row = lane + 32 * r;
    const int p = it.v_begin + row;
    bool changed = false;
    if (row < nv) {
      const int old = map_bit(sb, p);
      changed = decide_bit(f, old, flip[r]) != old;
    }
    map_publish(h.bits, it.v_begin + 32 * r, changed, lane);
  }
}

// Rows between the light and the sliced sizes, 32 at a time: eight lanes per
// row, four rows at a time. Lane q of a row's eight sums the row's entries
// q, q + 8, q + 16, ... (kHubGroupLoads loads in flight), shuffles combine the
// eight partial sums, and the row's field goes to the warp's shared scratch;
// lane l then decides row l.
template <bool PACKED>
__device__ __forceinline__ void hub_group(const DevGraph& d, const HubArgs& h, const uint32_t* sb,
                                          int* scratch, const WorkItem& it, const SweepArgs& a,
                                          int lane) {
  int* rp = scratch;
  int* acc = scratch + 33;
  const int sub = lane >> 3, q = lane & 7;
  for (int base = it.v_begin; base < it.v_end; base += 32) {
    const int rows = min(32, it.v_end - base);
    const bool own = lane < rows;
    if (own) rp[lane] = __ldg(d.row_ptr + base + lane);
    if (lane == 0) rp[rows] = __ldg(d.row_ptr + base + rows);
    const bool flip = own && pos_flip(h, a, base + lane);
    __syncwarp();
    for (int r0 = 0; r0 < rows; r0 += 4) {
      const int r = r0 + sub;
      int f = 0;
      if (r < rows) {
        const int e1 = rp[r + 1];
        for (int eb = rp[r] + q; eb < e1; eb += 8 * kHubGroupLoads) {
          Edge<PACKED> x[kHubGroupLoads];
#pragma unroll
          for (int u = 0; u < kHubGroupLoads; ++u) x[u].load(d, eb + 8 * u, eb + 8 * u < e1);
#pragma unroll
          for (int u = 0; u < kHubGroupLoads; ++u) f += x[u].weight() * map_spin(sb, x[u].col());
        }
      }
      f += __shfl_xor_sync(kFullMask, f, 1);
      f += __shfl_xor_sync(kFullMask, f, 2);
      f += __shfl_xor_sync(kFullMask, f, 4);
      if (q == 0 && r < rows) acc[r] = f;
    }
    __syncwarp();
    bool changed = false;
    if (own) {
      const int old = map_bit(sb, base + lane);
      changed = decide_bit(acc[lane], old, flip) != old;
    }
    map_publish(h.bits, base, changed, lane);
    __syncwarp();
  }
}

// A slice of a heavy row: its partial field joins the row's 64-bit
// accumulator (count and biased sum, as in sweep.cuh); the slice that
// completes the row decides it.
template <bool PACKED>
__device__ __forceinline__ void hub_slice(const DevGraph& d, const HubArgs& h, const uint32_t* sb,
                                          const WorkItem& it, const SweepArgs& a, int lane) {
  int f = 0;
  for (int e = it.e_begin + lane; e < it.e_end; e += 32 * kHubGroupLoads) {
    Edge<PACKED> x[kHubGroupLoads];
#pragma unroll
    for (int u = 0; u < kHubGroupLoads; ++u) x[u].load(d, e + 32 * u, e + 32 * u < it.e_end);
#pragma unroll
    for (int u = 0; u < kHubGroupLoads; ++u) f += x[u].weight() * map_spin(sb, x[u].col());
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
  if (lane == 0) {
    const int v = it.v_begin;
    const int slot = 2 * (-it.v_end - 1);
    const int parts = __ldg(d.slice_parts + (-it.v_end - 1));
    const unsigned long long mine =
        kSliceUnit + static_cast<unsigned long long>(static_cast<long long>(f) + kSliceBias);
    const unsigned long long old = atomicAdd(d.slice_acc + slot, mine);
    if (static_cast<int>(old >> 48) == parts - 1) {
      const long long low = static_cast<long long>((old & kSliceLowMask) + (mine & kSliceLowMask));
      const int total = static_cast<int>(low - static_cast<long long>(parts) * kSliceBias);
      d.slice_acc[slot] = 0ull;
      const int ob = map_bit(sb, v);
      if (decide_bit(total, ob, pos_flip(h, a, v)) != ob) atomicXor(h.bits + (v >> 5), 1u << (v & 31));
    }
  }
}

static_assert(sizeof(WorkItem) == sizeof(int4), "a work item is one 16-byte load");
__device__ __forceinline__ WorkItem load_item(const DevGraph& d, int i) {
  const int4 x = __ldg(reinterpret_cast<const int4*>(d.items) + i);
  return WorkItem{x.x, x.y, x.z, x.w};
}

template <bool PACKED>
__device__ __forceinline__ void hub_item(const DevGraph& d, const HubArgs& h, const uint32_t* sb,
                                         int* scratch, const WorkItem& it, const SweepArgs& a, int lane) {
  const int kind = item_kind(it);
  if (kind == kStageGroup) {
    hub_group<PACKED>(d, h, sb, scratch, it, a, lane);
  } else if (kind == kStageSlice) {
    hub_slice<PACKED>(d, h, sb, it, a, lane);
  } else {
    const int R = light_rows_per_lane(-it.e_end - 1, PACKED);
    if (R == 4)
      hub_light<PACKED, 4>(d, h, sb, it, a, lane);
    else if (R == 2)
      hub_light<PACKED, 2>(d, h, sb, it, a, lane);
    else
      hub_light<PACKED, 1>(d, h, sb, it, a, lane);
  }
}

// The sweep's flips by position: Philox evaluation q gives the draws of
// original ids 4q .. 4q + 3 (R5); each id below its threshold (with the flip
// bias of its position, as in flip_drawn) sets its position's bit. Called by
// the workers while the chain block runs, on a map cleared before.
__device__ __forceinline__ void hub_flip_map(const DevGraph& d, const HubArgs& h, const SweepArgs& a,
                                             const PhiloxRounds& rk, int gthread, int nthreads) {
  if (a.thr == 0u) return;
  const int n = d.pad_col;
  for (int q = gthread; 4 * q < n; q += nthreads) {
    const uint4 x = philox4x32_10(static_cast<uint32_t>(q), a.t, a.replica, 0u, rk);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int o = 4 * q + k;
      if (o >= n) break;
      uint64_t thr = a.thr;
      const int p = __ldg(h.pos + o);
      if (d.bias != nullptr) {
        thr = (static_cast<uint64_t>(a.thr) * __ldg(d.bias + p)) >> 7;
        if (thr > 0xffffffffull) thr = 0xffffffffull;
      }
      if (w[k] < thr) atomicOr(h.pflips + (p >> 5), 1u << (p & 31));
    }
  }
}

// Copy map words [w0, w1) from global memory into the block's copy: every
// thread issues up to 16 loads before it stores any, so a class of up to
// 16 x 32 x 1024 vertices costs one L2 round trip.
__device__ __forceinline__ void map_refresh(uint32_t* sb, const uint32_t* g, int w0, int w1) {
  constexpr int U = 16;
  for (int wb = w0 + static_cast<int>(threadIdx.x); wb < w1; wb += U * kHubBlock) {
    uint32_t x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = wb + u * kHubBlock < w1 ? __ldcg(g + wb + u * kHubBlock) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (wb + u * kHubBlock < w1) sb[wb + u * kHubBlock] = x[u];
  }
  __syncthreads();
}

// One launch: sweeps t_begin .. t_begin + sweeps - 1.
//
// Grid barrier bookkeeping (the counter only grows): the prologue barrier
// counts the G - 1 workers; per sweep the chain barrier counts G (G - 1
// workers, then the chain block) and each of the P non-hub classes G - 1
// (workers only: the chain block meanwhile pushes its deferred hubs); the
// epilogue barrier counts the workers again.
template <bool PACKED, bool STAGE>
__global__ void __launch_bounds__(kHubBlock, 1)
    hub_kernel(DevGraph d, HubArgs h, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
               uint32_t replica, PhiloxRounds rk, BarrierState* bs) {
  extern __shared__ __align__(16) unsigned char hub_shared[];
  const int lane = threadIdx.x & 31;
  const bool chain = blockIdx.x == 0;
  const int wb = static_cast<int>(blockIdx.x) - 1;  // worker block index
  const int warp = wb * kHubWarps + static_cast<int>(threadIdx.x >> 5);
  const int nwarps = (static_cast<int>(gridDim.x) - 1) * kHubWarps;
  const int W = (h.hubs + 31) / 32;
  const unsigned G = gridDim.x;
  const int P = h.classes - h.hub_classes;
  HubSmem s = hub_smem(hub_shared, h.hubs, h.hub_classes);
  int* scratch = reinterpret_cast<int*>(hub_shared) + (threadIdx.x >> 5) * kHubGroupScratch;
  int* queue = reinterpret_cast<int*>(hub_shared) + kHubWarps * kHubGroupScratch;
  uint32_t* sb_copy = reinterpret_cast<uint32_t*>(queue + 4);
  const uint32_t* sb = STAGE ? sb_copy : h.bits;
  if (chain && threadIdx.x < 4) s.cnt[threadIdx.x] = 0;
  bool skip = bs->skip_block == static_cast<int>(blockIdx.x) + 1;
  unsigned target = 0;
  int step = 0;
  // prologue: the workers build the global map from the state bytes, then
  // (after a workers-only barrier) their copies
  target += G - 1;
  if (!chain) {
    for (int j = warp; j < h.bit_words; j += nwarps) {
      const int p = 32 * j + lane;
      const bool neg = p < d.pad_col && (d.spins[p] & 1);
      const unsigned m = __ballot_sync(kFullMask, neg);
      if (lane == 0) h.bits[j] = m;
    }
    barrier_arrive(bs, skip);
    skip = false;
    if (!barrier_wait(bs, target)) return;
    if (STAGE) map_refresh(sb_copy, h.bits, 0, h.bit_words);
  }
  for (uint32_t k = 0; k < sweeps; ++k) {
    const SweepArgs a = sweep_args(t_begin + k, T, T0, replica);
    target += G;
    if (!chain) {
      // 1. the hubs' field sums and flip bits of sweep t; the hub rows the
      // chain pushes from into L2; the flip map cleared
      for (int i = (k == 0 ? 0 : h.num_b_items) + warp; i < h.num_items; i += nwarps)
        hub_sum_item<PACKED>(d, h, sb, i, static_cast<int>(k & 1u), lane);
      for (int j = warp; j < W; j += nwarps) hub_flip_word(d, h, j, a, rk, lane);
      if (k > 0)
        for (int i = warp; i < h.num_b_items; i += nwarps) {
          const int4 it = __ldg(h.sums + i);
          hub_prefetch<PACKED>(d, it.y, it.z, lane);
        }
      if (a.thr != 0u)
        for (int j = warp * 32 + lane; j < h.bit_words; j += nwarps * 32) h.pflips[j] = 0u;
      barrier_arrive(bs, skip);
      skip = false;
      // while the chain block runs the hub classes: once every worker has
      // cleared its part, the flip map of the sweep; then wait, polling sparsely
      if (!barrier_wait(bs, target - 1)) return;
      hub_flip_map(d, h, a, rk, warp * 32 + lane, nwarps * 32);
      if (!barrier_wait_sleep(bs, target, 256)) return;
      if (STAGE) map_refresh(sb_copy, h.bits, 0, W);
      // 3. the other classes, a workers-only grid barrier after each; the
      // block's items of a class are a contiguous range of equal estimated
      // work, taken by its warps from a shared counter
      for (int c = h.hub_classes; c < h.classes; ++c) {
        const int* blk = h.blk + (c - h.hub_classes) * static_cast<int>(G);
        const int i0 = __ldg(blk + wb), i1 = __ldg(blk + wb + 1);
        if (threadIdx.x == 0) queue[0] = 0;
        __syncthreads();
        int i = 0;
        if (lane == 0) i = atomicAdd(queue, 1);
        i = __shfl_sync(kFullMask, i, 0) + i0;
        // the next item's descriptor is loaded before the current item runs
        WorkItem cur = i < i1 ? load_item(d, i) : WorkItem{};
        while (i < i1) {
          int nxt = 0;
          if (lane == 0) nxt = atomicAdd(queue, 1);
          nxt = __shfl_sync(kFullMask, nxt, 0) + i0;
          const WorkItem nx = nxt < i1 ? load_item(d, nxt) : WorkItem{};
          hub_item<PACKED>(d, h, sb, scratch, cur, a, lane);
          i = nxt;
          cur = nx;
        }
        barrier_arrive(bs, false);
        target += G - 1;
        if (!barrier_wait(bs, target)) return;
        if (STAGE)
          map_refresh(sb_copy, h.bits, __ldg(h.class_begin + c) >> 5, (__ldg(h.class_begin + c + 1) + 31) >> 5);
      }
    } else {
      // 2. the hub classes, once every worker has arrived; then the deferred
      // pushes while the workers run the other classes
      if (!barrier_wait(bs, target - 1)) return;
      hub_chain<PACKED>(d, h, s, k, step);
      barrier_arrive(bs, skip);
      skip = false;
      hub_deferred<PACKED>(d, h, s, threadIdx.x >> 5, lane);
      __syncthreads();
      target += static_cast<unsigned>(P) * (G - 1);
    }
  }
  // epilogue: the state bytes from the map, every vertex's update parity
  // flipped once per sweep (the last class's barrier above orders the map)
  if (!chain)
    for (int p = wb * kHubBlock + static_cast<int>(threadIdx.x); p < d.pad_col;
         p += (static_cast<int>(G) - 1) * kHubBlock)
      d.spins[p] = static_cast<int8_t>(state_byte(1 - 2 * map_bit(h.bits, p), h.par_end));
}

}  // namespace isingx
