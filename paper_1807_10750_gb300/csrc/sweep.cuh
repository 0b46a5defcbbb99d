// Device side of a sweep: work-item staging, the field gather, the spin
// update with its random flip, and the bounded grid barrier of the persistent
// engine.
//
// A warp processes one work item (see host_graph.h) in two steps:
//  * stage_item: everything that does not depend on the spins -- for light
//    rows the sliced-ELL words of the item and the random-flip decisions of
//    Algorithm 2 (Philox words against the sweep's threshold), for a slice of
//    a heavy row its first round of CSR words;
//  * finish_item: the neighbour-spin gathers, the local fields
//    f_i = sum_j w_ij s_j (Eq. 2), the update s_i <- -sign(f_i) (f_i = 0 keeps
//    s_i), the flip and the spin store.
// The persistent engine stages the next colour class's item while it waits at
// the grid barrier, so only the gathers and the update follow the barrier.
#pragma once

#include <cstdint>

#include "host_graph.h"
#include "philox.cuh"

namespace isingx {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kRowsPerLane = 4;  // light items hold at most 32 * kRowsPerLane rows

// Words a lane stages for a light item: 16 packed words or 8 split
// (column, weight) pairs, shaped as rows-per-lane x slots-per-row =
// 4 x 4, 2 x 8 or 1 x 16 (packed) and 4 x 2, 2 x 4 or 1 x 8 (split).
__host__ __device__ constexpr int light_slots(bool packed) { return packed ? 16 : 8; }

// Rows per lane of a light item whose widest row has D slots.
__host__ __device__ constexpr int light_rows_per_lane(int D, bool packed) {
  return D <= light_slots(packed) / 4 ? 4 : (D <= light_slots(packed) / 2 ? 2 : 1);
}

// kPassDet: deterministic colour-class sweep behind grid barriers or launch
// boundaries; kPassRacy: the asynchronous mode; kPassEnergy: energy reduction;
// kPassFlow: the deterministic sweep without barriers, each gather waiting
// until its neighbour's state byte shows the update the colour order requires.
enum ItemPass { kPassDet = 0, kPassRacy = 1, kPassEnergy = 2, kPassFlow = 3 };

// Spin storage: one state byte per vertex. Bit 0 is 1 for spin -1; bit 1 is
// the parity of the number of updates the vertex has had since the spins were
// last set. Every update flips bit 1.
__host__ __device__ constexpr int spin_of(int b) { return 1 - 2 * (b & 1); }
__host__ __device__ constexpr int state_byte(int s, int parity) {
  return (s < 0 ? 1 : 0) | ((parity & 1) << 1);
}

// Edge formats. Packed: one int32 per entry, (col << 8) | (w & 0xff), used
// when every weight fits in int8 and n < 2^24 - 1 (so no valid word is -1).
// Split: an int32 column array and an int32 weight array (column -1 = none).
// CSR arrays hold every row; the sliced-ELL arrays hold the light items' rows
// (item-major, then slot-major, then row: slot k of row r of an item with nv
// rows starting at word b is word b + k * nv + r; padding slots hold the pad
// entry).
// Missing entries (ELL padding, slots past a row's degree, loads past a range)
// read as the pad entry: column n, weight 0. spins[n] exists and is 0, so every
// slot contributes w * s without a validity test.
struct DevGraph {
  int32_t pad_col;  // n
  int* error;       // bounded waits record a timeout here
  const int32_t* row_ptr;
  const int32_t* adj;      // CSR packed
  const int32_t* col;      // CSR split
  const int32_t* w;        // CSR split
  const int32_t* ell;      // sliced ELL packed
  const int32_t* ell_col;  // sliced ELL split
  const int32_t* ell_w;    // sliced ELL split
  int8_t* spins;
  const int32_t* orig;
  const WorkItem* items;
  unsigned long long* slice_acc;  // packed partial fields of sliced rows
  const int32_t* slice_parts;
  const uint8_t* bias;  // per-position flip bias q (threshold * q / 128), or null
};

struct SweepArgs {
  uint32_t thr;      // flip iff the vertex's Philox word (vertex_word) < thr
  uint32_t t;        // sweep index (counter word 1)
  uint32_t replica;  // counter word 2
  int class_lo;      // kPassFlow: first position of the current colour class
  int par_cur;       // kPassFlow: update parity every vertex had at the sweep's start
};

// Arguments of sweep t of a linear schedule of T sweeps starting at threshold
// T0 (ISING_SCHED_LINEAR in ising.h).
__device__ __forceinline__ SweepArgs sweep_args(uint64_t t, uint64_t T, uint64_t T0,
                                                uint32_t replica) {
  SweepArgs sa;
  sa.class_lo = 0;
  sa.par_cur = 0;
  sa.t = static_cast<uint32_t>(t);
  sa.replica = replica;
  sa.thr = (T <= 1) ? 0u : static_cast<uint32_t>((T0 * (T - 1 - t)) / (T - 1));
  return sa;
}

// Sliced rows: each slice adds (1 << 48) + (partial + 2^31) to one 64-bit
// word. The high 16 bits count the slices, the low 48 bits hold the biased sum
// (at most 65535 slices of 32-bit partials, so no carry reaches the count).
// The slice whose add returns count == parts - 1 is the last; it recovers the
// field from the returned value and resets the word for the next sweep.
constexpr unsigned long long kSliceUnit = 1ull << 48;
constexpr unsigned long long kSliceLowMask = kSliceUnit - 1;
constexpr long long kSliceBias = 1ll << 31;

// Racy and dataflow passes: spin bytes change while they are read, so reads
// and writes are relaxed atomics at GPU scope (defined behaviour under the
// memory model). They order nothing else, so the compiler may schedule other
// memory operations around them freely (no "memory" clobber); volatile keeps
// each re-read of a dataflow wait.
__device__ __forceinline__ int ld_relaxed_s8(const int8_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s8 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_s8(int8_t* p, int v) {
  asm volatile("st.relaxed.gpu.global.s8 [%0], %1;" ::"l"(p), "r"(v));
}

__device__ __forceinline__ long long flow_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// State byte of vertex j (relaxed for the racy and dataflow passes, whose
// neighbours change during the pass).
template <int PASS>
__device__ __forceinline__ int load_state(const DevGraph& d, int j) {
  return (PASS == kPassRacy || PASS == kPassFlow) ? (ld_relaxed_s8(d.spins + j) & 3)
                                                  : static_cast<int>(d.spins[j]);
}

constexpr long long kFlowBudgetNs = 2000000000LL;  // 2 s per wait

// kPassFlow: neighbour j of a vertex in the current class must have had the
// update of this sweep if its class comes earlier (parity par_cur ^ 1), and not
// yet if it comes later (parity par_cur); the pad entry never changes. Re-reads
// until that holds; gives up (recording a timeout) after kFlowBudgetNs or once
// any wait has failed.
static __device__ __noinline__ int flow_wait(const DevGraph& d, int j, int need) {
  const long long t0 = flow_ns();
  for (;;) {
    const int b = ld_relaxed_s8(d.spins + j) & 3;
    if (((b >> 1) & 1) == need) return b;
    if (*reinterpret_cast<volatile int*>(d.error) != 0) return b;
    if (flow_ns() - t0 > kFlowBudgetNs) {
      atomicExch(d.error, 1);
      return b;
    }
  }
}

template <int PASS>
__device__ __forceinline__ int ready_spin(const DevGraph& d, int j, int b, const SweepArgs& a) {
  if (PASS == kPassFlow && j != d.pad_col) {
    const int need = (j < a.class_lo) ? (a.par_cur ^ 1) : a.par_cur;
    if (((b >> 1) & 1) != need) b = flow_wait(d, j, need);
  }
  return spin_of(b);
}

// One loaded entry (or none) in either format.
template <bool PACKED>
struct Edge;

template <>
struct Edge<true> {
  int word;
  __device__ __forceinline__ void load(const DevGraph& d, int e, bool ok) {
    word = ok ? __ldg(d.adj + e) : (d.pad_col << 8);
  }
  __device__ __forceinline__ void load_ell(const DevGraph& d, int e, bool ok) {
    word = ok ? __ldg(d.ell + e) : (d.pad_col << 8);
  }
  __device__ __forceinline__ int col() const { return static_cast<int>(static_cast<unsigned>(word) >> 8); }
  __device__ __forceinline__ int weight() const { return (word << 24) >> 24; }
};

template <>
struct Edge<false> {
  int c, w;
  __device__ __forceinline__ void load(const DevGraph& d, int e, bool ok) {
    c = ok ? __ldg(d.col + e) : d.pad_col;
    w = ok ? __ldg(d.w + e) : 0;
  }
  __device__ __forceinline__ void load_ell(const DevGraph& d, int e, bool ok) {
    c = ok ? __ldg(d.ell_col + e) : d.pad_col;
    w = ok ? __ldg(d.ell_w + e) : 0;
  }
  __device__ __forceinline__ int col() const { return c; }
  __device__ __forceinline__ int weight() const { return w; }
};

// sum of w_e * s_col[e] over CSR entries e = e0, e0 + step, ... < e1, four per
// round so that each lane keeps several loads in flight.
template <bool PACKED, int PASS>
__device__ __forceinline__ int strided_field(const DevGraph& d, int e0, int e1, int step,
                                             const SweepArgs& a) {
  int f = 0;
  for (int e = e0; e < e1; e += 4 * step) {
    Edge<PACKED> x[4];
    int b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u].load(d, e + u * step, e + u * step < e1);
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = load_state<PASS>(d, x[u].col());
#pragma unroll
    for (int u = 0; u < 4; ++u) f += x[u].weight() * ready_spin<PASS>(d, x[u].col(), b[u], a);
  }
  return f;
}

// Algorithm 2's random flip of the vertex at position v whose caller id is
// o, in sweep a.t. With a flip bias the threshold is min((thr * q_v) >> 7,
// 2^32 - 1) in 64-bit integers (q_v = 128 leaves it unchanged).
__device__ __forceinline__ bool flip_drawn(const DevGraph& d, int v, uint32_t o,
                                           const SweepArgs& a, const PhiloxRounds& rk) {
  if (a.thr == 0u) return false;
  uint32_t thr = a.thr;
  if (d.bias != nullptr) {
    const unsigned long long t =
        (static_cast<unsigned long long>(a.thr) * __ldg(d.bias + v)) >> 7;
    thr = t > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(t);
  }
  return vertex_word(o, a.t, a.replica, 0u, rk) < thr;
}

// Eq. 2 under the max-cut sign (s <- -sign f, f = 0 keeps s), then the flip;
// the state byte's update parity flips.
template <int PASS>
__device__ __forceinline__ void apply_update(const DevGraph& d, int v, int f, bool flip,
                                             const SweepArgs& a) {
  int b = load_state<PASS>(d, v);
  // dataflow: a sliced row's previous update may come from another warp; wait
  // until its state shows that update
  if (PASS == kPassFlow && ((b >> 1) & 1) != a.par_cur) b = flow_wait(d, v, a.par_cur);
  int s = spin_of(b);
  if (f > 0)
    s = -1;
  else if (f < 0)
    s = 1;
  if (flip) s = -s;
  const int nb = state_byte(s, ((b >> 1) & 1) ^ 1);
  if (PASS == kPassRacy || PASS == kPassFlow)
    st_relaxed_s8(d.spins + v, nb);
  else
    d.spins[v] = static_cast<int8_t>(nb);
}

enum StageKind { kStageLight = 0, kStageSlice = 1, kStageGroup = 2 };

template <bool PACKED>
struct Staged {
  WorkItem it;
  int kind;
  unsigned flips;                       // light: bit r = row lane + 32 r flips
  Edge<PACKED> x[light_slots(PACKED)];  // light: rows x slots; slice: first round
};

__device__ __forceinline__ int item_kind(const WorkItem& it) {
  if (it.v_end < 0) return kStageSlice;
  return it.e_end < 0 ? kStageLight : kStageGroup;
}

template <bool PACKED, int R>
__device__ __forceinline__ void stage_light_shape(const DevGraph& d, Staged<PACKED>& s,
                                                  const SweepArgs& a, const PhiloxRounds& rk,
                                                  int lane) {
  constexpr int DM = light_slots(PACKED) / R;
  const int nv = s.it.v_end - s.it.v_begin;
  const int D = -s.it.e_end - 1;
  const int base = s.it.e_begin;
  int orig[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = lane + 32 * r;
    const bool valid = row < nv;
    orig[r] = valid ? __ldg(d.orig + s.it.v_begin + row) : -1;
#pragma unroll
    for (int k = 0; k < DM; ++k) s.x[r * DM + k].load_ell(d, base + k * nv + row, valid && k < D);
  }
  s.flips = 0;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (orig[r] >= 0 &&
        flip_drawn(d, s.it.v_begin + lane + 32 * r, static_cast<uint32_t>(orig[r]), a, rk))
      s.flips |= 1u << r;
}

template <bool PACKED>
__device__ __forceinline__ void stage_item(const DevGraph& d, const WorkItem& it,
                                           const SweepArgs& a, const PhiloxRounds& rk, int lane,
                                           Staged<PACKED>& s) {
  s.it = it;
  s.kind = item_kind(it);
  if (s.kind == kStageSlice) {
    const int e0 = it.e_begin + lane;
#pragma unroll
    for (int u = 0; u < 4; ++u) s.x[u].load(d, e0 + 32 * u, e0 + 32 * u < it.e_end);
    return;
  }
  if (s.kind == kStageGroup) return;
  const int R = light_rows_per_lane(-it.e_end - 1, PACKED);
  if (R == 4)
    stage_light_shape<PACKED, 4>(d, s, a, rk, lane);
  else if (R == 2)
    stage_light_shape<PACKED, 2>(d, s, a, rk, lane);
  else
    stage_light_shape<PACKED, 1>(d, s, a, rk, lane);
}

template <bool PACKED, int PASS, int R>
__device__ __forceinline__ void finish_light_shape(const DevGraph& d, const Staged<PACKED>& s,
                                                   const SweepArgs& a, int lane,
                                                   long long& energy) {
  constexpr int DM = light_slots(PACKED) / R;
  const int nv = s.it.v_end - s.it.v_begin;
  int b[R * DM];
#pragma unroll
  for (int j = 0; j < R * DM; ++j) b[j] = load_state<PASS>(d, s.x[j].col());
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int f = 0;
#pragma unroll
    for (int k = 0; k < DM; ++k)
      f += s.x[r * DM + k].weight() * ready_spin<PASS>(d, s.x[r * DM + k].col(), b[r * DM + k], a);
    if (lane + 32 * r < nv) {
      const int v = s.it.v_begin + lane + 32 * r;
      if (PASS == kPassEnergy)
        energy += static_cast<long long>(spin_of(d.spins[v])) * f;
      else
        apply_update<PASS>(d, v, f, (s.flips >> r) & 1u, a);
    }
  }
}

// Rows too heavy for a light item but not sliced, 32 at a time: their CSR
// entries are contiguous, so the warp streams them lane-strided (lane l takes
// entries e0 + l + 32 k, kGroupLoads in flight), finds each entry's row among
// the block's 33 row offsets (one binary search per batch, then forward
// steps), and adds each run of a row's terms into the row's shared
// accumulator; lane l then updates row l. Every kernel that finishes items
// runs at most kGroupWarps warps per block.
constexpr int kGroupWarps = 16;
constexpr int kGroupLoads = 4;

template <bool PACKED, int PASS>
__device__ __forceinline__ void finish_group_rows(const DevGraph& d, const WorkItem& it,
                                                  const SweepArgs& a, const PhiloxRounds& rk,
                                                  int lane, long long& energy) {
  __shared__ int group_scratch[kGroupWarps][65];  // per warp: 33 row offsets, 32 fields
  int* rp = group_scratch[threadIdx.x >> 5];
  int* acc = rp + 33;
  for (int base = it.v_begin; base < it.v_end; base += 32) {
    const int rows = min(32, it.v_end - base);
    if (lane < rows) rp[lane] = __ldg(d.row_ptr + base + lane);
    if (lane == 0) rp[rows] = __ldg(d.row_ptr + base + rows);
    acc[lane] = 0;
    __syncwarp();
    const int e0 = rp[0], e1 = rp[rows];
    for (int eb = e0; eb < e1; eb += 32 * kGroupLoads) {
      Edge<PACKED> x[kGroupLoads];
      int b[kGroupLoads];
#pragma unroll
      for (int u = 0; u < kGroupLoads; ++u) x[u].load(d, eb + lane + 32 * u, eb + lane + 32 * u < e1);
#pragma unroll
      for (int u = 0; u < kGroupLoads; ++u) b[u] = load_state<PASS>(d, x[u].col());
      int e = eb + lane;
      if (e < e1) {
        // the row holding entry e: the largest r with rp[r] <= e
        int lo = 0, hi = rows - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (rp[mid] <= e)
            lo = mid;
          else
            hi = mid - 1;
        }
        int r = lo;
        int run = 0;
#pragma unroll
        for (int u = 0; u < kGroupLoads; ++u) {
          e = eb + lane + 32 * u;
          if (e < e1) {
            while (rp[r + 1] <= e) {
              if (run != 0) atomicAdd(acc + r, run);
              run = 0;
              ++r;
            }
            run += x[u].weight() * ready_spin<PASS>(d, x[u].col(), b[u], a);
          }
        }
        if (run != 0) atomicAdd(acc + r, run);
      }
    }
    __syncwarp();
    const int v = base + lane;
    if (lane < rows) {
      const int f = acc[lane];
      if (PASS == kPassEnergy)
        energy += static_cast<long long>(spin_of(d.spins[v])) * f;
      else
        apply_update<PASS>(d, v, f, flip_drawn(d, v, static_cast<uint32_t>(__ldg(d.orig + v)), a, rk), a);
    }
    __syncwarp();
  }
}

template <bool PACKED, int PASS>
__device__ __forceinline__ void finish_item(const DevGraph& d, const Staged<PACKED>& s,
                                            const SweepArgs& a, const PhiloxRounds& rk, int lane,
                                            long long& energy) {
  if (s.kind == kStageLight) {
    const int R = light_rows_per_lane(-s.it.e_end - 1, PACKED);
    if (R == 4)
      finish_light_shape<PACKED, PASS, 4>(d, s, a, lane, energy);
    else if (R == 2)
      finish_light_shape<PACKED, PASS, 2>(d, s, a, lane, energy);
    else
      finish_light_shape<PACKED, PASS, 1>(d, s, a, lane, energy);
    return;
  }
  if (s.kind == kStageGroup) {
    finish_group_rows<PACKED, PASS>(d, s.it, a, rk, lane, energy);
    return;
  }
  // a slice of one heavy row
  int f = 0;
  {
    int b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = load_state<PASS>(d, s.x[u].col());
#pragma unroll
    for (int u = 0; u < 4; ++u) f += s.x[u].weight() * ready_spin<PASS>(d, s.x[u].col(), b[u], a);
  }
  f += strided_field<PACKED, PASS>(d, s.it.e_begin + lane + 128, s.it.e_end, 32, a);
  const int v = s.it.v_begin;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
  if (PASS == kPassEnergy) {
    if (lane == 0) energy += static_cast<long long>(spin_of(d.spins[v])) * f;
    return;
  }
  if (lane == 0) {
    // two accumulators per sliced row: the dataflow pass alternates them by
    // sweep parity, so a later sweep's slices never meet this sweep's sum
    const int slot = 2 * (-s.it.v_end - 1) + (PASS == kPassFlow ? a.par_cur : 0);
    const int parts = __ldg(d.slice_parts + (-s.it.v_end - 1));
    const unsigned long long mine =
        kSliceUnit + static_cast<unsigned long long>(static_cast<long long>(f) + kSliceBias);
    const unsigned long long old = atomicAdd(d.slice_acc + slot, mine);
    if (static_cast<int>(old >> 48) == parts - 1) {
      const long long low = static_cast<long long>((old & kSliceLowMask) + (mine & kSliceLowMask));
      const int total = static_cast<int>(low - static_cast<long long>(parts) * kSliceBias);
      d.slice_acc[slot] = 0ull;
      // only the slice that completes the row draws its flip
      apply_update<PASS>(d, v, total, flip_drawn(d, v, static_cast<uint32_t>(__ldg(d.orig + v)), a, rk), a);
    }
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1's end-of-sweep flips (ISING_SCHED_NFLIP), run by one warp after
// every update of sweep t is visible: the first N distinct candidates
// c_j = floor(x_j * n / 2^32), x_j = Philox word 0 with counter
// (j, t, replica, 2), j = 0, 1, 2, ..., are flipped (spin bit only; the update
// parity is unchanged). Candidates are drawn 32 at a time; inside a batch a
// repeated candidate keeps its first occurrence, and a bitmap of the chosen
// vertices (zero on entry, cleared again on exit) rejects candidates chosen in
// earlier batches, so the chosen set is exactly the sequential definition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_relaxed_u32g(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void nflip_step(const DevGraph& d, const int32_t* pos, unsigned* bitmap,
                                           int32_t* picked, uint32_t N, uint32_t t,
                                           uint32_t replica, const PhiloxRounds& rk, int lane) {
  const uint64_t n = static_cast<uint64_t>(d.pad_col);
  uint32_t count = 0;
  for (uint32_t j0 = 0; count < N; j0 += 32) {
    const uint32_t x = philox4x32_10_word0(j0 + lane, t, replica, 2u, rk);
    const uint32_t c = static_cast<uint32_t>((static_cast<uint64_t>(x) * n) >> 32);
    const unsigned same = __match_any_sync(kFullMask, c);
    const bool first = (__ffs(same) - 1) == lane;
    const bool seen = (ld_relaxed_u32g(bitmap + (c >> 5)) >> (c & 31)) & 1u;
    const bool fresh = first && !seen;
    const unsigned fmask = __ballot_sync(kFullMask, fresh);
    const uint32_t take = min(static_cast<uint32_t>(__popc(fmask)), N - count);
    const uint32_t rank = static_cast<uint32_t>(__popc(fmask & ((1u << lane) - 1u)));
    if (fresh && rank < take) {
      atomicOr(bitmap + (c >> 5), 1u << (c & 31));
      picked[count + rank] = static_cast<int32_t>(c);
    }
    count += take;
    __syncwarp();
  }
  for (uint32_t k = lane; k < N; k += 32) {
    const uint32_t c = static_cast<uint32_t>(picked[k]);
    const int p = __ldg(pos + c);
    d.spins[p] = static_cast<int8_t>(d.spins[p] ^ 1);
    atomicAnd(bitmap + (c >> 5), ~(1u << (c & 31)));
  }
  __syncwarp();
}

// Flips of sweep t of an N-flip schedule: floor(N0 (T-1-t) / (T-1)).
__host__ __device__ inline uint32_t nflip_count(uint32_t n0, uint64_t T, uint64_t t) {
  if (T <= 1 || t >= T) return 0u;
  return static_cast<uint32_t>(static_cast<uint64_t>(n0) * (T - 1 - t) / (T - 1));
}

// ---------------------------------------------------------------------------
// Grid barrier of the persistent engine: a counter that only grows. A block
// arrives with one release-add by thread 0 (after __syncthreads, so the whole
// block's spin stores are ordered before it) and waits until the counter
// reaches its target with acquire loads. Every wait is bounded: after
// kBarrierBudgetNs the block records a timeout and returns false; blocks also
// give up as soon as another block has recorded one.
// ---------------------------------------------------------------------------
constexpr long long kBarrierBudgetNs = 2000000000LL;  // 2 s

struct BarrierState {
  unsigned int count;
  int error;            // 0 ok, 1 a wait timed out
  int skip_block;       // failure-detection tests: block skip_block - 1 skips its first arrival
  int pad;
  long long budget_ns;  // bound of every wait (0: kBarrierBudgetNs)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void barrier_arrive(BarrierState* bs, bool skip = false) {
  __syncthreads();
  if (threadIdx.x == 0 && !skip)
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bs->count) : "memory");
}

__device__ __forceinline__ bool barrier_wait(BarrierState* bs, unsigned target) {
  __shared__ int ok_shared;
  if (threadIdx.x == 0) {
    int ok = 1;
    long long t0 = 0;
    const long long budget = bs->budget_ns > 0 ? bs->budget_ns : kBarrierBudgetNs;
    for (unsigned it = 0; static_cast<int>(ld_acquire_u32(&bs->count) - target) < 0; ++it) {
      if ((it & 63u) == 0u) {
        if (it == 0u) t0 = global_ns();
        if (ld_relaxed_s32(&bs->error) != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > budget) {
          atomicExch(&bs->error, 1);
          ok = 0;
          break;
        }
      }
    }
    ok_shared = ok;
  }
  __syncthreads();
  return ok_shared != 0;
}

// barrier_wait for a wait known to be long (the hub engine's workers while
// one block runs the hub classes): thread 0 sleeps sleep_ns between polls, so
// hundreds of waiting blocks do not keep the counter's L2 line busy. Bounded
// like barrier_wait.
__device__ __forceinline__ bool barrier_wait_sleep(BarrierState* bs, unsigned target,
                                                   unsigned sleep_ns) {
  __shared__ int ok_sleep;
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long budget = bs->budget_ns > 0 ? bs->budget_ns : kBarrierBudgetNs;
    const long long t0 = global_ns();
    while (static_cast<int>(ld_acquire_u32(&bs->count) - target) < 0) {
      if (ld_relaxed_s32(&bs->error) != 0) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > budget) {
        atomicExch(&bs->error, 1);
        ok = 0;
        break;
      }
      __nanosleep(sleep_ns);
    }
    ok_sleep = ok;
  }
  __syncthreads();
  return ok_sleep != 0;
}

}  // namespace isingx
