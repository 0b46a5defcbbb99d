// Device side of a sweep: work-item staging, the field gather, the spin
// update with its random flip, and the bounded grid barrier of the persistent
// engine.
//
// A warp processes one work item (see host_graph.h) in two steps:
//  * stage_item: everything that does not depend on the spins -- the item,
//    its row offsets, the first round of (column, weight) pairs and the
//    random-flip decisions (Philox words compared with the sweep's threshold);
//  * finish_item: the neighbour-spin gathers, the local fields
//    f_i = sum_j w_ij s_j (Eq. 2), the update s_i <- -sign(f_i) (tie keeps) and
//    the flip of Algorithm 2, then the spin stores.
// The persistent engine stages the next colour class's item while it waits at
// the grid barrier, so only the gathers and the update follow the barrier.
#pragma once

#include <cstdint>

#include "host_graph.h"
#include "philox.cuh"

namespace isingx {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kRowsPerLane = 4;      // work items hold at most 32 * kRowsPerLane rows
// Edges per row (light rows) or per lane (slices) loaded per round: 4 packed
// words, or 2 split (column, weight) pairs, to stay within 64 registers.
template <bool PACKED>
__host__ __device__ constexpr int edge_slots() {
  return PACKED ? 4 : 2;
}
constexpr int kLightMeanDegree = 16;  // items up to this mean degree use one lane per row

enum ItemPass { kPassDet = 0, kPassRacy = 1, kPassEnergy = 2 };

// Edge formats. Packed: one int32 per CSR entry, (col << 8) | (w & 0xff),
// used when every weight fits in int8 and n < 2^24 - 1 (so no valid word is
// -1). Split: an int32 column array and an int32 weight array.
struct DevGraph {
  const int32_t* row_ptr;
  const int32_t* adj;  // packed entries (packed format)
  const int32_t* col;  // split format
  const int32_t* w;    // split format
  int8_t* spins;
  const int32_t* orig;
  const WorkItem* items;
  unsigned long long* slice_acc;  // packed partial fields of sliced rows
  const int32_t* slice_parts;
};

struct SweepArgs {
  uint32_t thr;      // flip iff Philox word 0 < thr
  uint32_t t;        // sweep index (counter word 1)
  uint32_t replica;  // counter word 2
  PhiloxKey key;
};

// Sliced rows: each slice adds (1 << 48) + (partial + 2^31) to one 64-bit
// word. The high 16 bits count the slices, the low 48 bits hold the biased sum
// (at most 65535 slices of 32-bit partials, so no carry reaches the count).
// The slice whose add returns count == parts - 1 is the last; it recovers the
// field from the returned value and resets the word for the next sweep.
constexpr unsigned long long kSliceUnit = 1ull << 48;
constexpr unsigned long long kSliceLowMask = kSliceUnit - 1;
constexpr long long kSliceBias = 1ll << 31;

// Racy mode: neighbour reads and own writes race by design (Sec. IV-B); they
// are relaxed atomics at GPU scope so the races are defined behaviour.
__device__ __forceinline__ int ld_relaxed_s8(const int8_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s8 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_s8(int8_t* p, int v) {
  asm volatile("st.relaxed.gpu.global.s8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int PASS>
__device__ __forceinline__ int spin_at(const DevGraph& d, int j) {
  return (PASS == kPassRacy) ? ld_relaxed_s8(d.spins + j) : static_cast<int>(d.spins[j]);
}

// One loaded CSR entry (or none) in either format.
template <bool PACKED>
struct Edge;

template <>
struct Edge<true> {
  int word;
  __device__ __forceinline__ void load(const DevGraph& d, int e, bool ok) {
    word = ok ? __ldg(d.adj + e) : -1;
  }
  __device__ __forceinline__ bool valid() const { return word != -1; }
  __device__ __forceinline__ int col() const { return static_cast<int>(static_cast<unsigned>(word) >> 8); }
  __device__ __forceinline__ int weight() const { return (word << 24) >> 24; }
};

template <>
struct Edge<false> {
  int c, w;
  __device__ __forceinline__ void load(const DevGraph& d, int e, bool ok) {
    c = ok ? __ldg(d.col + e) : -1;
    w = ok ? __ldg(d.w + e) : 0;
  }
  __device__ __forceinline__ bool valid() const { return c >= 0; }
  __device__ __forceinline__ int col() const { return c; }
  __device__ __forceinline__ int weight() const { return w; }
};

template <bool PACKED, int PASS>
__device__ __forceinline__ int edge_term(const DevGraph& d, const Edge<PACKED>& x) {
  return x.valid() ? x.weight() * spin_at<PASS>(d, x.col()) : 0;
}

// sum of w_e * s_col[e] over e = e0, e0 + step, ... < e1, several edges per
// round so that each lane keeps several loads in flight.
template <bool PACKED, int PASS>
__device__ __forceinline__ int strided_field(const DevGraph& d, int e0, int e1, int step) {
  constexpr int S = edge_slots<PACKED>();
  int f = 0;
  for (int e = e0; e < e1; e += S * step) {
    Edge<PACKED> x[S];
#pragma unroll
    for (int u = 0; u < S; ++u) x[u].load(d, e + u * step, e + u * step < e1);
#pragma unroll
    for (int u = 0; u < S; ++u) f += edge_term<PACKED, PASS>(d, x[u]);
  }
  return f;
}

// Algorithm 2's random flip for position v (caller's id orig[v]) in sweep a.t.
__device__ __forceinline__ bool flip_drawn(const DevGraph& d, int v, const SweepArgs& a) {
  if (a.thr == 0u) return false;
  const uint32_t o = static_cast<uint32_t>(__ldg(d.orig + v));
  return philox4x32_10_word0(o, a.t, a.replica, 0u, a.key) < a.thr;
}

// Eq. 2 under the max-cut sign (s <- -sign f, f = 0 keeps s), then the flip.
template <int PASS>
__device__ __forceinline__ void apply_update(const DevGraph& d, int v, int f, bool flip) {
  int s = spin_at<PASS>(d, v);
  if (f > 0)
    s = -1;
  else if (f < 0)
    s = 1;
  if (flip) s = -s;
  if (PASS == kPassRacy)
    st_relaxed_s8(d.spins + v, s);
  else
    d.spins[v] = static_cast<int8_t>(s);
}

enum StageKind { kStageLight = 0, kStageSlice = 1, kStageGroup = 2 };

template <bool PACKED>
struct Staged {
  WorkItem it;
  int kind;
  int rp[kRowsPerLane];  // light: row begin
  int re[kRowsPerLane];  // light: row end
  Edge<PACKED> x[kRowsPerLane][edge_slots<PACKED>()];
  unsigned flips;  // light: bit r for row lane + 32 r; slice: bit 0 (lane 0)
};

template <bool PACKED>
__device__ __forceinline__ void stage_item(const DevGraph& d, int index, const SweepArgs& a,
                                           int lane, Staged<PACKED>& s) {
  constexpr int S = edge_slots<PACKED>();
  s.it = d.items[index];
  s.flips = 0;
  if (s.it.v_end < 0) {
    s.kind = kStageSlice;
    const int e0 = s.it.e_begin + lane;
#pragma unroll
    for (int u = 0; u < S; ++u) s.x[0][u].load(d, e0 + 32 * u, e0 + 32 * u < s.it.e_end);
    if (lane == 0 && flip_drawn(d, s.it.v_begin, a)) s.flips = 1;
    return;
  }
  const int nv = s.it.v_end - s.it.v_begin;
  if (s.it.e_end - s.it.e_begin > kLightMeanDegree * nv) {
    s.kind = kStageGroup;
    return;
  }
  s.kind = kStageLight;
#pragma unroll
  for (int r = 0; r < kRowsPerLane; ++r) {
    const int v = s.it.v_begin + lane + 32 * r;
    s.rp[r] = 0;
    s.re[r] = 0;
    if (v < s.it.v_end) {
      s.rp[r] = __ldg(d.row_ptr + v);
      s.re[r] = __ldg(d.row_ptr + v + 1);
    }
  }
#pragma unroll
  for (int r = 0; r < kRowsPerLane; ++r)
#pragma unroll
    for (int u = 0; u < S; ++u) s.x[r][u].load(d, s.rp[r] + u, s.rp[r] + u < s.re[r]);
#pragma unroll
  for (int r = 0; r < kRowsPerLane; ++r) {
    const int v = s.it.v_begin + lane + 32 * r;
    if (v < s.it.v_end && flip_drawn(d, v, a)) s.flips |= 1u << r;
  }
}

// Rows of mean degree above kLightMeanDegree: lane groups of g lanes (power of
// two >= a quarter of the mean degree) gather one row per pass, 32 / g rows per
// pass; the 32 fields of a chunk are then moved to one lane each.
template <bool PACKED, int PASS>
__device__ __forceinline__ void finish_group_rows(const DevGraph& d, const WorkItem& it,
                                                  const SweepArgs& a, int lane,
                                                  long long& energy) {
  const int nv = it.v_end - it.v_begin;
  const int mean = (it.e_end - it.e_begin + nv - 1) / nv;
  int lg = 0;
  while ((4 << lg) < mean && lg < 5) ++lg;
  const int g = 1 << lg;
  const int rows_per_pass = 32 >> lg;
  const int sub = lane & (g - 1);
  const int grp = lane >> lg;
  for (int base = it.v_begin; base < it.v_end; base += 32) {
    const int rows = min(32, it.v_end - base);
    const int passes = (rows + rows_per_pass - 1) / rows_per_pass;
    int my_f = 0;
    for (int p = 0; p < passes; ++p) {
      const int v = base + p * rows_per_pass + grp;
      int f = 0;
      if (v < it.v_end)
        f = strided_field<PACKED, PASS>(d, __ldg(d.row_ptr + v) + sub, __ldg(d.row_ptr + v + 1), g);
      for (int o = g >> 1; o > 0; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
      const int got = __shfl_sync(kFullMask, f, (lane % rows_per_pass) << lg);
      if (lane / rows_per_pass == p) my_f = got;
    }
    const int v = base + lane;
    if (v < it.v_end) {
      if (PASS == kPassEnergy)
        energy += static_cast<long long>(d.spins[v]) * my_f;
      else
        apply_update<PASS>(d, v, my_f, flip_drawn(d, v, a));
    }
  }
}

template <bool PACKED, int PASS>
__device__ __forceinline__ void finish_item(const DevGraph& d, Staged<PACKED>& s,
                                            const SweepArgs& a, int lane, long long& energy) {
  constexpr int S = edge_slots<PACKED>();
  if (s.kind == kStageGroup) {
    finish_group_rows<PACKED, PASS>(d, s.it, a, lane, energy);
    return;
  }
  if (s.kind == kStageSlice) {
    int f = 0;
#pragma unroll
    for (int u = 0; u < S; ++u) f += edge_term<PACKED, PASS>(d, s.x[0][u]);
    f += strided_field<PACKED, PASS>(d, s.it.e_begin + lane + 32 * S, s.it.e_end, 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
    const int v = s.it.v_begin;
    if (PASS == kPassEnergy) {
      if (lane == 0) energy += static_cast<long long>(d.spins[v]) * f;
      return;
    }
    if (lane == 0) {
      const int slot = -s.it.v_end - 1;
      const int parts = __ldg(d.slice_parts + slot);
      const unsigned long long mine =
          kSliceUnit + static_cast<unsigned long long>(static_cast<long long>(f) + kSliceBias);
      const unsigned long long old = atomicAdd(d.slice_acc + slot, mine);
      if (static_cast<int>(old >> 48) == parts - 1) {
        const long long low = static_cast<long long>((old & kSliceLowMask) + (mine & kSliceLowMask));
        const int total = static_cast<int>(low - static_cast<long long>(parts) * kSliceBias);
        d.slice_acc[slot] = 0ull;
        apply_update<PASS>(d, v, total, s.flips & 1u);
      }
    }
    return;
  }
  // light rows: the staged round, then further rounds (reusing the staged
  // registers) for rows longer than S
  int f[kRowsPerLane];
  int kmax = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerLane; ++r) {
    f[r] = 0;
#pragma unroll
    for (int u = 0; u < S; ++u) f[r] += edge_term<PACKED, PASS>(d, s.x[r][u]);
    kmax = max(kmax, s.re[r] - s.rp[r]);
  }
  for (int k = S; k < kmax; k += S) {
#pragma unroll
    for (int r = 0; r < kRowsPerLane; ++r)
#pragma unroll
      for (int u = 0; u < S; ++u) s.x[r][u].load(d, s.rp[r] + k + u, s.rp[r] + k + u < s.re[r]);
#pragma unroll
    for (int r = 0; r < kRowsPerLane; ++r)
#pragma unroll
      for (int u = 0; u < S; ++u) f[r] += edge_term<PACKED, PASS>(d, s.x[r][u]);
  }
#pragma unroll
  for (int r = 0; r < kRowsPerLane; ++r) {
    const int v = s.it.v_begin + lane + 32 * r;
    if (v < s.it.v_end) {
      if (PASS == kPassEnergy)
        energy += static_cast<long long>(d.spins[v]) * f[r];
      else
        apply_update<PASS>(d, v, f[r], (s.flips >> r) & 1u);
    }
  }
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
  int error;  // 0 ok, 1 a wait timed out
  int pad[2];
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

__device__ __forceinline__ void barrier_arrive(BarrierState* bs) {
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bs->count) : "memory");
}

__device__ __forceinline__ bool barrier_wait(BarrierState* bs, unsigned target) {
  __shared__ int ok_shared;
  if (threadIdx.x == 0) {
    int ok = 1;
    long long t0 = 0;
    for (unsigned it = 0; static_cast<int>(ld_acquire_u32(&bs->count) - target) < 0; ++it) {
      if ((it & 63u) == 0u) {
        if (it == 0u) t0 = global_ns();
        if (ld_relaxed_s32(&bs->error) != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > kBarrierBudgetNs) {
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

}  // namespace isingx
