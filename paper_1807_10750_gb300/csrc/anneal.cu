// Sweep kernels and the C ABI of include/ising.h.
//
// Layout in device memory (all owned by the handle):
//   row_ptr  int32[n+1]   CSR offsets, vertices ordered by colour class
//   adj      int32[nnz]   packed (col << 8) | (w & 0xff) entries, rows sorted by
//                         neighbour position; or col / w int32[nnz] each (split)
//   ell*     sliced-ELL copies of the light rows (host_graph.h)
//   spins    int8[n+1]    state byte per position: bit 0 the spin (1 = -1), bit 1
//                         the update parity; byte n is the pad entry's spin 0
//   orig     int32[n]     position -> caller's vertex id (Philox counter word 0)
//   pos      int32[n]     caller's vertex id -> position
//   items    WorkItem[]   per-class warp work (host_graph.h)
//   slice_*  partial-field combine for rows sliced across warps
//   deps     item dependencies of the item-dataflow engine; block_* the
//            packed words of the one-block engine (block.cuh)
//
// One warp processes one work item (sweep.cuh): the local fields
// f_i = sum_j w_ij s_j of its rows (Eq. 2), then the update rule and the
// random flip of Algorithm 2. The engines differ in how a colour class waits
// for the previous one: a launch per class, a grid barrier, per-neighbour or
// per-item dataflow waits, or block barriers for small graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <system_error>
#include <vector>

#include "../../include/ising.h"
#include "host_graph.h"
#include "host_parallel.h"
#include "philox.cuh"
#include "sweep.cuh"
#include "block.cuh"
#include "graph_handle.h"
#include "halo.cuh"
#include "hub.cuh"

using isingx::HostGraph;
using isingx::PhiloxKey;
using isingx::WorkItem;
using isingx::WorkPlan;

namespace {

using isingx::BarrierState;
using isingx::DevGraph;
using isingx::SweepArgs;
using isingx::sweep_args;
using isingx::kPassDet;
using isingx::kPassEnergy;
using isingx::kPassFlow;
using isingx::kPassRacy;

constexpr int kBlock = 256;
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kPersistBlock = 512;
// AUTO takes the halo engine while no block updates more than this many
// times the rows it owns per sweep
constexpr double kHaloAutoRatio = 1.6;

// Item kernel of the per-launch engine. Deterministic sweeps launch it once
// per colour class (phase_begin + 1 == phase_end); the racy mode launches it
// once per sweep over every class, each warp walking the classes in order with
// no wait between them; the energy pass covers all items.
template <bool PACKED, int PASS>
__global__ void __launch_bounds__(kBlock, 4)
    items_kernel(DevGraph d, const int32_t* __restrict__ phase_items, int phase_begin,
                 int phase_end, SweepArgs a, isingx::PhiloxRounds rk,
                 unsigned long long* energy_out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = gridDim.x * kWarpsPerBlock;
  long long energy = 0;
  for (int c = phase_begin; c < phase_end; ++c) {
    const int ie = __ldg(phase_items + c + 1);
    for (int i = __ldg(phase_items + c) + warp; i < ie; i += nwarps) {
      isingx::Staged<PACKED> st;
      isingx::stage_item<PACKED>(d, d.items[i], a, rk, lane, st);
      isingx::finish_item<PACKED, PASS>(d, st, a, rk, lane, energy);
    }
  }
  if (PASS == kPassEnergy) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) energy += __shfl_xor_sync(isingx::kFullMask, energy, o);
    __shared__ long long part[kWarpsPerBlock];
    if (lane == 0) part[threadIdx.x >> 5] = energy;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long sum = 0;
      for (int k = 0; k < kWarpsPerBlock; ++k) sum += part[k];
      atomicAdd(energy_out, static_cast<unsigned long long>(sum));
    }
  }
}

// First item of colour class cls for this warp. Deterministic passes: item
// warp of every class (a barrier follows each class). The racy pass walks
// all classes without a barrier; when the sweep has at least as many items as
// warps they are dealt round-robin over the whole sweep -- item i, counted
// across classes, belongs to warp i mod nwarps -- so a warp gets as many items
// as any other instead of one in every class. With fewer items than warps
// that dealing would run every class at once (a synchronous update, which can
// oscillate), so there a warp keeps item warp of every class, in class order.
template <int PASS>
__device__ __forceinline__ int class_start(const int32_t* phase_items, int cls, int warp,
                                           int nwarps, bool rotate) {
  const int ib = __ldg(phase_items + cls);
  if (PASS != kPassRacy || !rotate) return ib + warp;
  int r = (warp - ib) % nwarps;
  if (r < 0) r += nwarps;
  return ib + r;
}

// The warp's first item of colour class cls, or an empty item if it has none.
template <int PASS>
__device__ __forceinline__ WorkItem first_item(const DevGraph& d, const int32_t* phase_items,
                                               int cls, int warp, int nwarps, bool rotate) {
  const int i = class_start<PASS>(phase_items, cls, warp, nwarps, rotate);
  WorkItem it = {0, 0, 0, 0};
  if (i < __ldg(phase_items + cls + 1)) it = d.items[i];
  return it;
}

// Persistent engine: one cooperative launch runs every sweep of an anneal
// call. Warp w takes items w, w + nwarps, ... of each colour class. Between
// arriving at the grid barrier and waiting on it, the warp stages its first
// item of the next class (loads and random flips need no spins), so after the
// barrier only the neighbour gathers and the update remain. Deterministic:
// a barrier after every class. Racy: only after every sweep (Sec. IV-B).
template <bool PACKED, int PASS>
__global__ void __launch_bounds__(kPersistBlock, 2)
    persistent_kernel(DevGraph d, const int32_t* __restrict__ phase_items, int num_phases,
                      uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0, uint32_t replica,
                      isingx::PhiloxRounds rk, BarrierState* bs, uint32_t nflip0,
                      const int32_t* __restrict__ pos, unsigned* bitmap, int32_t* picked) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kPersistBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kPersistBlock) >> 5;
  long long unused = 0;
  unsigned target = 0;
  uint32_t k = 0;
  int c = 0;
  SweepArgs a = sweep_args(t_begin + 0, T, T0, replica);
  const bool rotate = __ldg(phase_items + num_phases) >= nwarps;
  if (PASS == kPassRacy && rotate) {
    // racy pass over at least as many items as warps: item i of the sweep
    // (classes in order) belongs to warp i mod nwarps, so a warp meets its
    // items in class order without walking the classes; a grid barrier ends
    // every sweep
    const int ni = __ldg(phase_items + num_phases);
    bool skip = bs->skip_block == static_cast<int>(blockIdx.x) + 1;
    isingx::Staged<PACKED> sr;
    for (uint32_t kk = 0; kk < sweeps; ++kk) {
      const SweepArgs ak = sweep_args(t_begin + kk, T, T0, replica);
      for (int i = warp; i < ni; i += nwarps) {
        isingx::stage_item<PACKED>(d, d.items[i], ak, rk, lane, sr);
        isingx::finish_item<PACKED, PASS>(d, sr, ak, rk, lane, unused);
      }
      if (nflip0 != 0u) {
        // Algorithm 1: once every update of the sweep is visible, one warp
        // flips the sweep's N random spins; the barrier below publishes them
        isingx::barrier_arrive(bs, skip);
        skip = false;
        target += gridDim.x;
        if (!isingx::barrier_wait(bs, target)) return;
        const uint32_t N = isingx::nflip_count(nflip0, T, t_begin + kk);
        if (blockIdx.x == 0 && threadIdx.x < 32 && N > 0u)
          isingx::nflip_step(d, pos, bitmap, picked, N, static_cast<uint32_t>(t_begin + kk), replica,
                             rk, lane);
      }
      if (kk + 1 == sweeps) break;
      isingx::barrier_arrive(bs, skip);
      skip = false;
      target += gridDim.x;
      if (!isingx::barrier_wait(bs, target)) return;
    }
    return;
  }
  int ib = class_start<PASS>(phase_items, 0, warp, nwarps, rotate), ie = __ldg(phase_items + 1);
  isingx::Staged<PACKED> st;
  bool have = ib < ie;
  if (have) isingx::stage_item<PACKED>(d, d.items[ib], a, rk, lane, st);
  // the warp's first item of the following class, loaded one class ahead
  WorkItem next = first_item<PASS>(d, phase_items, num_phases > 1 ? 1 : 0, warp, nwarps, rotate);
  // failure-detection tests: this block may skip its first barrier arrival
  bool skip_arrival = bs->skip_block == static_cast<int>(blockIdx.x) + 1;
  for (;;) {
    if (have) {
      isingx::finish_item<PACKED, PASS>(d, st, a, rk, lane, unused);
      for (int i = ib + nwarps; i < ie; i += nwarps) {
        isingx::stage_item<PACKED>(d, d.items[i], a, rk, lane, st);
        isingx::finish_item<PACKED, PASS>(d, st, a, rk, lane, unused);
      }
    }
    const bool sweep_end = (c + 1 == num_phases);
    if (nflip0 != 0u && sweep_end) {
      // Algorithm 1: once every update of the sweep is visible, one warp flips
      // the sweep's N random spins; the barrier below publishes them.
      isingx::barrier_arrive(bs, skip_arrival);
      skip_arrival = false;
      target += gridDim.x;
      if (!isingx::barrier_wait(bs, target)) return;
      const uint32_t N = isingx::nflip_count(nflip0, T, t_begin + k);
      if (blockIdx.x == 0 && threadIdx.x < 32 && N > 0u)
        isingx::nflip_step(d, pos, bitmap, picked, N, static_cast<uint32_t>(t_begin + k), replica,
                           rk, lane);
    }
    if (sweep_end && k + 1 == sweeps) break;
    const bool sync = (PASS != kPassRacy) || sweep_end;
    if (sync) {
      isingx::barrier_arrive(bs, skip_arrival);
      skip_arrival = false;
    }
    if (sweep_end) {
      c = 0;
      ++k;
      a = sweep_args(t_begin + k, T, T0, replica);
    } else {
      ++c;
    }
    ib = class_start<PASS>(phase_items, c, warp, nwarps, rotate);
    ie = __ldg(phase_items + c + 1);
    have = ib < ie;
    if (have) isingx::stage_item<PACKED>(d, next, a, rk, lane, st);
    next = first_item<PASS>(d, phase_items, c + 1 < num_phases ? c + 1 : 0, warp, nwarps, rotate);
    if (sync) {
      target += gridDim.x;
      if (!isingx::barrier_wait(bs, target)) return;
    }
  }
}

// Small graphs whose whole packed CSR fits in one block's shared memory (the
// 800-vertex workload: 38k entries, 160 KB): one block of 1024 threads holds
// the row offsets, the entries, every state byte and the sweep's flips, for
// the whole anneal call. A class is one pass in which 16 lanes share a row
// (its entries strided over them, four in flight per lane, four shuffles to
// combine) and the row's
// first lane decides it at once, then one block barrier. The state bytes go
// back to global memory at the end of the call. Deterministic linear
// schedule (flip bias allowed); the spins equal one grid phase per class.
constexpr int kCsrBlockThreads = 1024;
constexpr int kCsrRowLanes = 16;

struct CsrBlockLayout {
  int rp, adj, cls, state, flip, total;
};

__host__ __device__ inline CsrBlockLayout csr_block_layout(int n, long long nnz, int ncls) {
  CsrBlockLayout L{};
  long long o = 0;
  L.rp = 0;
  o += 4LL * (n + 1);
  L.adj = static_cast<int>((o + 15) & ~15LL);
  o = L.adj + 4LL * nnz;
  L.cls = static_cast<int>(o);
  o += 4LL * (ncls + 1);
  L.state = static_cast<int>(o);
  o += n + 1;  // one spare state byte (spin +1) for a padding column
  L.flip = static_cast<int>(o);
  o += n;
  o = (o + 15) & ~15LL;
  L.total = o > 0x7fffffffLL ? 0x7fffffff : static_cast<int>(o);
  return L;
}

__global__ void __launch_bounds__(kCsrBlockThreads, 1)
    csr_block_kernel(DevGraph d, int n, int nnz, int ncls, const int32_t* __restrict__ class_pos,
                     uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0, uint32_t replica,
                     isingx::PhiloxRounds rk) {
  extern __shared__ __align__(16) unsigned char csr_mem[];
  const CsrBlockLayout L = csr_block_layout(n, nnz, ncls);
  int32_t* rp = reinterpret_cast<int32_t*>(csr_mem + L.rp);
  int32_t* adj = reinterpret_cast<int32_t*>(csr_mem + L.adj);
  int32_t* cls = reinterpret_cast<int32_t*>(csr_mem + L.cls);
  uint8_t* state = csr_mem + L.state;
  uint8_t* flip = csr_mem + L.flip;
  const int tid = threadIdx.x;
  for (int i = tid; i <= n; i += kCsrBlockThreads) rp[i] = __ldg(d.row_ptr + i);
  for (int i = tid; i < nnz; i += kCsrBlockThreads) adj[i] = __ldg(d.adj + i);
  for (int i = tid; i <= ncls; i += kCsrBlockThreads) cls[i] = __ldg(class_pos + i);
  for (int i = tid; i < n; i += kCsrBlockThreads) state[i] = static_cast<uint8_t>(d.spins[i]);
  if (tid == 0) state[n] = 0;
  const int q = tid % kCsrRowLanes;                  // lane within the row's group
  const int grp = tid / kCsrRowLanes;                // row group
  const int ngrp = kCsrBlockThreads / kCsrRowLanes;
  __syncthreads();
  for (uint32_t k = 0; k < sweeps; ++k) {
    const SweepArgs a = sweep_args(t_begin + k, T, T0, replica);
    for (int i = tid; i < n; i += kCsrBlockThreads)
      flip[i] = flip_drawn(d, i, static_cast<uint32_t>(__ldg(d.orig + i)), a, rk) ? 1 : 0;
    __syncthreads();
    for (int c = 0; c < ncls; ++c) {
      const int ce = cls[c + 1];
      for (int r0 = cls[c]; r0 < ce; r0 += ngrp) {
        const int r = r0 + grp;
        int f = 0;
        if (r < ce) {
          const int e1 = rp[r + 1];
          int e = rp[r] + q;
          for (; e + 3 * kCsrRowLanes < e1; e += 4 * kCsrRowLanes) {
            uint32_t x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = static_cast<uint32_t>(adj[e + u * kCsrRowLanes]);
            int sp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) sp[u] = state[x[u] >> 8];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              f += static_cast<int>(static_cast<int8_t>(static_cast<uint8_t>(x[u] & 0xffu))) * isingx::spin_of(sp[u]);
          }
          for (; e < e1; e += kCsrRowLanes) {
            const uint32_t x = static_cast<uint32_t>(adj[e]);
            const int w = static_cast<int>(static_cast<int8_t>(static_cast<uint8_t>(x & 0xffu)));
            f += w * isingx::spin_of(state[x >> 8]);
          }
        }
        // every lane of the warp reaches the shuffles (r0 is uniform)
#pragma unroll
        for (int o = 1; o < kCsrRowLanes; o <<= 1) f += __shfl_xor_sync(isingx::kFullMask, f, o, kCsrRowLanes);
        if (r < ce && q == 0) {
          const int bt = state[r];
          int sv = isingx::spin_of(bt);
          if (f > 0)
            sv = -1;
          else if (f < 0)
            sv = 1;
          if (flip[r]) sv = -sv;
          state[r] = static_cast<uint8_t>(isingx::state_byte(sv, ((bt >> 1) & 1) ^ 1));
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += kCsrBlockThreads) d.spins[i] = static_cast<int8_t>(state[i]);
}

// Block engine (block.cuh): a graph of at most 4095 vertices, every sweep of
// an anneal call in one block; deterministic pass, with Algorithm 1's flips
// after each sweep when nflip0 > 0.
__global__ void __launch_bounds__(isingx::kBlockThreads)
    block_kernel(DevGraph d, isingx::BlockArgs ba, uint64_t t_begin, uint32_t sweeps, uint64_t T,
                 uint64_t T0, uint32_t replica, isingx::PhiloxRounds rk, uint32_t nflip0,
                 const int32_t* __restrict__ pos, unsigned* bitmap, int32_t* picked) {
  extern __shared__ __align__(128) unsigned char block_mem[];
  const isingx::BlockShared sh = isingx::block_shared(block_mem, ba);
  isingx::block_setup(ba, sh);
  __syncthreads();
  unsigned seq = 0;
  for (uint32_t k = 0; k < sweeps; ++k) {
    const SweepArgs a = sweep_args(t_begin + k, T, T0, replica);
    if (ba.resident_words > 0)
      isingx::block_sweep_resident(d, ba, a, rk, sh);
    else if (!isingx::block_sweep(d, ba, a, rk, sh, seq))
      return;
    if (nflip0 != 0u) {
      // the sweep's updates are in global memory; warp 0 flips N_t spins
      const uint32_t N = isingx::nflip_count(nflip0, T, t_begin + k);
      if (threadIdx.x < 32 && N > 0u)
        isingx::nflip_step(d, pos, bitmap, picked, N, static_cast<uint32_t>(t_begin + k), replica,
                           rk, threadIdx.x & 31);
      __syncthreads();
    }
  }
}

// Item-dataflow engine: one cooperative launch runs every sweep with no grid
// barrier and no per-vertex waits. Warp w takes items w, w + nwarps, ... of
// each colour class in (sweep, class) order; before updating item i in the
// launch's k-th sweep it waits (bounded) until done[j] >= k + 1 for every
// dependency j of an earlier class and done[j] >= k for every j of a later
// class (host_graph.h, build_item_deps), then gathers with ordinary loads and
// publishes done[i] = k + 1 with a release store. The items' own loads and
// Philox draws are staged before the wait. All warps are resident and each
// follows the (sweep, class) order, so the earliest unfinished item can
// always proceed.
// Completion counters sit one per 128-byte line, so pollers of different
// items do not share lines.
constexpr int kDoneStride = 32;

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every lane takes some of item i's dependencies; true once all are met,
// false (and the error flag set) after `budget` ns or when another warp has
// already failed. Warp-uniform.
__device__ __forceinline__ bool wait_item_deps(const int32_t* __restrict__ dep_ptr,
                                               const int32_t* __restrict__ deps, const int* done,
                                               int i, int k, int* error, long long budget, int lane) {
  bool ok = true;
  const int e = __ldg(dep_ptr + i + 1);
  for (int q = __ldg(dep_ptr + i) + lane; q < e && ok; q += 32) {
    const int dj = __ldg(deps + q);
    const int need = (dj & 1) ? k : k + 1;
    long long t0 = 0;
    for (unsigned it = 0; ld_acquire_s32(done + (dj >> 1) * kDoneStride) < need; ++it) {
      if ((it & 63u) == 0u) {
        const long long now = isingx::global_ns();
        if (it == 0u) {
          t0 = now;
        } else if (now - t0 > budget || isingx::ld_relaxed_s32(error) != 0) {
          atomicExch(error, 1);
          ok = false;
          break;
        }
      }
    }
  }
  return __all_sync(isingx::kFullMask, ok);
}

template <bool PACKED>
__global__ void __launch_bounds__(kPersistBlock, 2)
    itemflow_kernel(DevGraph d, const int32_t* __restrict__ phase_items, int num_phases,
                    uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0, uint32_t replica,
                    isingx::PhiloxRounds rk, const int32_t* __restrict__ dep_ptr,
                    const int32_t* __restrict__ deps, int* done, int* error, long long budget) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kPersistBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kPersistBlock) >> 5;
  long long unused = 0;
  isingx::Staged<PACKED> st;
  for (uint32_t k = 0; k < sweeps; ++k) {
    const SweepArgs a = sweep_args(t_begin + k, T, T0, replica);
    for (int c = 0; c < num_phases; ++c) {
      const int ie = __ldg(phase_items + c + 1);
      for (int i = __ldg(phase_items + c) + warp; i < ie; i += nwarps) {
        isingx::stage_item<PACKED>(d, d.items[i], a, rk, lane, st);
        if (!wait_item_deps(dep_ptr, deps, done, i, static_cast<int>(k), error, budget, lane)) return;
        isingx::finish_item<PACKED, kPassDet>(d, st, a, rk, lane, unused);
        __syncwarp();
        if (lane == 0) st_release_s32(done + i * kDoneStride, static_cast<int>(k) + 1);
      }
    }
  }
}

// Dataflow engine: one cooperative launch runs every sweep with no grid
// barrier. Warp w takes items w, w + nwarps, ... of each colour class in
// (sweep, class) order; every neighbour gather waits until the neighbour's
// state byte shows the update the colour order requires (sweep.cuh,
// kPassFlow). All warps are resident and each follows that order, so the
// earliest unfinished item can always proceed. A wait that gives up stops
// the kernel; the host reports ISING_ETIMEOUT.
template <bool PACKED>
__global__ void __launch_bounds__(kPersistBlock, 2)
    flow_kernel(DevGraph d, const int32_t* __restrict__ phase_items,
                const int32_t* __restrict__ class_begin, int num_phases, uint64_t t_begin,
                uint32_t sweeps, uint64_t T, uint64_t T0, uint32_t replica, int par0,
                isingx::PhiloxRounds rk) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kPersistBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kPersistBlock) >> 5;
  long long unused = 0;
  isingx::Staged<PACKED> st;
  for (uint32_t k = 0; k < sweeps; ++k) {
    SweepArgs a = sweep_args(t_begin + k, T, T0, replica);
    a.par_cur = par0 ^ static_cast<int>(k & 1u);
    for (int c = 0; c < num_phases; ++c) {
      a.class_lo = __ldg(class_begin + c);
      const int ie = __ldg(phase_items + c + 1);
      for (int i = __ldg(phase_items + c) + warp; i < ie; i += nwarps) {
        isingx::stage_item<PACKED>(d, d.items[i], a, rk, lane, st);
        isingx::finish_item<PACKED, kPassFlow>(d, st, a, rk, lane, unused);
      }
    }
  }
}

// Algorithm 1's end-of-sweep flips for the per-launch engine (one warp).
__global__ void nflip_kernel(DevGraph d, const int32_t* pos, unsigned* bitmap, int32_t* picked,
                             uint32_t N, uint32_t t, uint32_t replica, isingx::PhiloxRounds rk) {
  isingx::nflip_step(d, pos, bitmap, picked, N, t, replica, rk, threadIdx.x & 31);
}

__global__ void init_random_kernel(int8_t* spins, const int32_t* orig, int n,
                                   isingx::PhiloxRounds rk, uint32_t replica) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t x = isingx::vertex_word(static_cast<uint32_t>(orig[p]), 0u, replica, 1u, rk);
    spins[p] = static_cast<int8_t>(isingx::state_byte((x >> 31) ? -1 : 1, 0));
  }
}

__global__ void gather_spins_kernel(int8_t* out, const int8_t* spins, const int32_t* pos, int n) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x)
    out[o] = static_cast<int8_t>(isingx::spin_of(spins[pos[o]]));
}

__global__ void check_spins_kernel(const int8_t* in, int n, int32_t* bad) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x)
    if (in[o] != 1 && in[o] != -1) atomicExch(bad, 1);
}

__global__ void scatter_spins_kernel(int8_t* spins, const int8_t* in, const int32_t* pos, int n) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x)
    spins[pos[o]] = static_cast<int8_t>(isingx::state_byte(in[o], 0));
}

__global__ void fill_spins_kernel(int8_t* spins, int n, int8_t value) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    spins[p] = value;
}

// T0 = round(p0 * 2^32) clamped to [0, 2^32 - 1] (ISING_SCHED_LINEAR, ising.h).
uint64_t linear_t0(double p0) {
  const double scaled = std::floor(p0 * 4294967296.0 + 0.5);
  if (scaled >= 4294967295.0) return 4294967295ull;
  if (scaled > 0.0) return static_cast<uint64_t>(scaled);
  return 0;
}

// Flip threshold of sweep t.
uint32_t linear_threshold(double p0, uint64_t T, uint64_t t) {
  const uint64_t t0 = linear_t0(p0);
  if (T <= 1 || t >= T) return 0u;
  return static_cast<uint32_t>(t0 * (T - 1 - t) / (T - 1));
}

int grid_for(int64_t work, int per_block, int cap) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return static_cast<int>(b);
}

}  // namespace


namespace {

void free_device(ising_graph* g) {
  void* ptrs[] = {g->d_row_ptr, g->d_adj, g->d_col,  g->d_w,  g->d_ell, g->d_ell_col, g->d_ell_w, g->d_spins,
                  g->d_orig,    g->d_pos,         g->d_items,       g->d_slice_acc,
                  g->d_slice_parts, g->d_energy,  g->d_flag,
                  g->d_tmp,     g->d_class_items, g->d_all_items, g->d_barrier,
                  g->d_class_begin, g->d_trace, g->d_nflip_bits, g->d_nflip_list,
                  g->d_bias,    g->d_rowid, g->d_block_words, g->d_block_chunk_off,
                  g->d_block_chunk_len, g->d_block_class_chunk, g->d_dep_ptr, g->d_deps,
                  g->d_done, g->d_halo_hdr, g->d_halo_words, g->d_halo_slices, g->d_halo_gpos,
                  g->d_halo_imports, g->d_halo_nbrs, g->d_halo_exports, g->d_halo_quads, g->d_halo_flags,
                  g->d_spins2, g->d_hub_split, g->d_hub_end, g->d_hub_sums, g->d_hub_acc,
                  g->d_hub_flips, g->d_hub_bits, g->d_hub_pflips, g->d_hub_blk,
                  g->d_gnn_hchunk, g->d_gnn_chunk_row};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// Drop the halo plan (its device arrays); the next anneal that asks for the
// engine plans again.
void free_halo(ising_graph* g) {
  void* ptrs[] = {g->d_halo_hdr, g->d_halo_words, g->d_halo_slices, g->d_halo_gpos,
                  g->d_halo_imports, g->d_halo_nbrs, g->d_halo_exports, g->d_halo_quads, g->d_halo_flags,
                  g->d_spins2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  g->d_halo_hdr = g->d_halo_words = g->d_halo_slices = g->d_halo_gpos = nullptr;
  g->d_halo_imports = g->d_halo_nbrs = g->d_halo_exports = g->d_halo_quads = nullptr;
  g->d_halo_flags = nullptr;
  g->d_spins2 = nullptr;
  g->halo_state = 0;
}

// Latch a CUDA failure in the handle.
int cuda_fail(ising_graph* g, cudaError_t e) {
  (void)e;
  cudaGetLastError();
  if (g) g->status = ISING_ECUDA;
  return ISING_ECUDA;
}

#define ISING_CUDA(g, call)                      \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail((g), e_); \
  } while (0)

int enter(ising_graph* g) {
  if (g == nullptr) return ISING_EINVAL;
  if (g->status != ISING_OK) return g->status;
  if (cudaSetDevice(g->device) != cudaSuccess) return cuda_fail(g, cudaErrorInvalidDevice);
  return ISING_OK;
}

template <typename T>
cudaError_t alloc_copy(T** dst, const T* src, size_t count, cudaStream_t s) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
  if (e != cudaSuccess) return e;
  if (src && count) return cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
  return cudaMemsetAsync(*dst, 0, bytes, s);
}

// Launch the item kernel over phases [pb, pe) of `phase_items` (device) whose
// host copy is `host_items`.
template <int PASS>
cudaError_t launch_items(ising_graph* g, const int32_t* phase_items, const int32_t* host_items,
                         int pb, int pe, const SweepArgs& a, const isingx::PhiloxRounds& rk,
                         unsigned long long* energy_out) {
  int widest = 0;
  for (int c = pb; c < pe; ++c) widest = std::max(widest, host_items[c + 1] - host_items[c]);
  if (widest == 0) return cudaSuccess;
  const int grid = grid_for(widest, kWarpsPerBlock, g->num_sms * 64);
  const DevGraph d = g->dev();
  g->launches++;
  if (g->packed)
    items_kernel<true, PASS><<<grid, kBlock, 0, g->stream>>>(d, phase_items, pb, pe, a, rk, energy_out);
  else
    items_kernel<false, PASS><<<grid, kBlock, 0, g->stream>>>(d, phase_items, pb, pe, a, rk, energy_out);
  return cudaGetLastError();
}

// The barrier state at the start of a launch: zero counts and errors, the
// wait bound and the injected fault of ising_debug_fault.
cudaError_t barrier_init(ising_graph* g) {
  BarrierState init{};
  init.skip_block = g->fault_kind == ISING_FAULT_SKIP_ARRIVAL ? 1 : 0;
  init.budget_ns = static_cast<long long>(g->wait_budget_ns);
  return cudaMemcpyAsync(g->d_barrier, &init, sizeof(init), cudaMemcpyHostToDevice, g->stream);
}

// A persistent launch that timed out leaves error != 0 in the barrier state;
// synchronising calls report it (and latch it).
int check_device_error(ising_graph* g) {
  int err = 0;
  ISING_CUDA(g, cudaMemcpyAsync(&err, &g->d_barrier->error, sizeof(err), cudaMemcpyDeviceToHost, g->stream));
  ISING_CUDA(g, cudaStreamSynchronize(g->stream));
  if (err != 0) {
    g->status = ISING_ETIMEOUT;
    return ISING_ETIMEOUT;
  }
  return ISING_OK;
}

template <bool PACKED, int PASS>
cudaError_t launch_persistent_t(ising_graph* g, const int32_t* phase_items, int num_phases,
                                uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                                uint32_t replica, isingx::PhiloxRounds rk, uint32_t nflip0) {
  auto kernel = persistent_kernel<PACKED, PASS>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPersistBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  per_sm = std::min(per_sm, 2);
  const int grid = per_sm * g->num_sms;
  g->persist_grid = grid;
  e = barrier_init(g);
  if (e != cudaSuccess) return e;
  DevGraph d = g->dev();
  BarrierState* bs = g->d_barrier;
  const int32_t* pos = g->d_pos;
  unsigned* bitmap = g->d_nflip_bits;
  int32_t* picked = g->d_nflip_list;
  void* args[] = {&d,       &phase_items, &num_phases, &t_begin, &sweeps, &T,     &T0,
                  &replica, &rk,          &bs,         &nflip0,  &pos,    &bitmap, &picked};
  g->launches++;
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid),
                                     dim3(kPersistBlock), args, 0, g->stream);
}

template <bool PACKED>
cudaError_t launch_itemflow_t(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T,
                              uint64_t T0, uint32_t replica, const isingx::PhiloxRounds& rk_in) {
  auto kernel = itemflow_kernel<PACKED>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPersistBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  per_sm = std::min(per_sm, 2);
  const int grid = per_sm * g->num_sms;
  if ((e = barrier_init(g)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(g->d_done, 0, kDoneStride * sizeof(int32_t) * static_cast<size_t>(g->num_items),
                           g->stream)) != cudaSuccess)
    return e;
  DevGraph d = g->dev();
  const int32_t* phase_items = g->d_class_items;
  int num_phases = g->num_colours;
  isingx::PhiloxRounds rk = rk_in;
  const int32_t* dep_ptr = g->d_dep_ptr;
  const int32_t* deps = g->d_deps;
  int* done = g->d_done;
  int* error = &g->d_barrier->error;
  long long budget = g->wait_budget_ns > 0 ? static_cast<long long>(g->wait_budget_ns)
                                           : isingx::kBarrierBudgetNs;
  void* args[] = {&d, &phase_items, &num_phases, &t_begin, &sweeps, &T, &T0, &replica, &rk,
                  &dep_ptr, &deps, &done, &error, &budget};
  g->launches++;
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid),
                                     dim3(kPersistBlock), args, 0, g->stream);
}

cudaError_t launch_itemflow(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T,
                            uint64_t T0, uint32_t replica, const isingx::PhiloxRounds& rk) {
  if (g->packed) return launch_itemflow_t<true>(g, t_begin, sweeps, T, T0, replica, rk);
  return launch_itemflow_t<false>(g, t_begin, sweeps, T, T0, replica, rk);
}

cudaError_t launch_block(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                         uint32_t replica, const isingx::PhiloxRounds& rk, uint32_t nflip0) {
  isingx::BlockArgs ba{};
  ba.n = g->n;
  ba.num_chunks = g->block_num_chunks;
  ba.num_classes = g->num_colours;
  ba.words = reinterpret_cast<const uint32_t*>(g->d_block_words);
  ba.chunk_off = g->d_block_chunk_off;
  ba.chunk_len = g->d_block_chunk_len;
  ba.class_chunk = g->d_block_class_chunk;
  ba.class_pos = g->d_class_begin;
  ba.wait_ns = static_cast<long long>(g->wait_budget_ns);
  ba.short_copy = g->fault_kind == ISING_FAULT_SHORT_COPY ? 1 : 0;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
  // the whole packed CSR in shared memory (linear schedule; not under the
  // short-copy test, which needs the copies)
  if (g->packed && nflip0 == 0u && !ba.short_copy && g->nnz < (1LL << 30)) {
    const int csr_smem = csr_block_layout(g->n, g->nnz, g->num_colours).total;
    if (csr_smem <= optin) {
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(csr_block_kernel),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem);
      if (e != cudaSuccess) return e;
      g->launches++;
      csr_block_kernel<<<1, kCsrBlockThreads, csr_smem, g->stream>>>(
          g->dev(), g->n, static_cast<int>(g->nnz), g->num_colours, g->d_class_begin, t_begin, sweeps, T, T0,
          replica, rk);
      return cudaGetLastError();
    }
  }
  // every word resident in shared memory when it fits (not under the
  // short-copy test, which needs the copies)
  const int words = g->block_num_words;
  ba.resident_words = 0;
  if (!ba.short_copy && words > 0 &&
      isingx::block_layout(ba.n, ba.num_chunks, ba.num_classes, words).total <= optin)
    ba.resident_words = words;
  const int smem = isingx::block_layout(ba.n, ba.num_chunks, ba.num_classes, ba.resident_words).total;
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(block_kernel),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = barrier_init(g);
  if (e != cudaSuccess) return e;
  g->launches++;
  block_kernel<<<1, isingx::kBlockThreads, smem, g->stream>>>(
      g->dev(), ba, t_begin, sweeps, T, T0, replica, rk, nflip0, g->d_pos, g->d_nflip_bits,
      g->d_nflip_list);
  return cudaGetLastError();
}

template <int PASS>
cudaError_t launch_persistent(ising_graph* g, const int32_t* phase_items, int num_phases,
                              uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                              uint32_t replica, const isingx::PhiloxRounds& rk, uint32_t nflip0) {
  if (g->packed)
    return launch_persistent_t<true, PASS>(g, phase_items, num_phases, t_begin, sweeps, T, T0,
                                           replica, rk, nflip0);
  return launch_persistent_t<false, PASS>(g, phase_items, num_phases, t_begin, sweeps, T, T0,
                                          replica, rk, nflip0);
}

template <bool PACKED>
cudaError_t launch_flow_t(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T,
                          uint64_t T0, uint32_t replica, int par0,
                          const isingx::PhiloxRounds& rk_in) {
  auto kernel = flow_kernel<PACKED>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPersistBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  per_sm = std::min(per_sm, 2);
  const int grid = per_sm * g->num_sms;
  e = barrier_init(g);
  if (e != cudaSuccess) return e;
  DevGraph d = g->dev();
  const int32_t* phase_items = g->d_class_items;
  const int32_t* class_begin = g->d_class_begin;
  int num_phases = g->num_colours;
  isingx::PhiloxRounds rk = rk_in;
  void* args[] = {&d, &phase_items, &class_begin, &num_phases, &t_begin, &sweeps, &T, &T0,
                  &replica, &par0, &rk};
  g->launches++;
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid),
                                     dim3(kPersistBlock), args, 0, g->stream);
}

cudaError_t launch_flow(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                        uint32_t replica, int par0, const isingx::PhiloxRounds& rk) {
  if (g->packed) return launch_flow_t<true>(g, t_begin, sweeps, T, T0, replica, par0, rk);
  return launch_flow_t<false>(g, t_begin, sweeps, T, T0, replica, par0, rk);
}

// The halo plan for sweeps-per-exchange request S (host_graph.h,
// build_halo_plan): one part per SM; S as requested, or S = 2 unless that
// plan does not fit or repeats more than kHaloAutoRatio times the work and
// S = 1 fits. Host only.
void choose_halo_plan(const HostGraph& hg, int32_t parts, int32_t S, isingx::HaloPlan* hp,
                      const std::atomic<bool>* cancel) {
  try {
    if (S > 0) {
      isingx::build_halo_plan(hg, parts, S, hp, cancel);
    } else {
      isingx::build_halo_plan(hg, parts, 2, hp, cancel);
      if (!hp->ok || hp->max_work_ratio > kHaloAutoRatio) {
        isingx::HaloPlan one;
        isingx::build_halo_plan(hg, parts, 1, &one, cancel);
        if (one.ok) *hp = std::move(one);
      }
    }
  } catch (const std::bad_alloc&) {
    *hp = isingx::HaloPlan();
  }
}

// Start the planner thread for the handle's current request (no-op without
// a host graph or while one runs); without threads, plan right here.
void start_planner(ising_graph* g) {
  if (!g->host || g->planner.joinable() || g->pending) return;
  g->pending.reset(new (std::nothrow) isingx::HaloPlan());
  if (!g->pending) return;
  g->planned.store(false, std::memory_order_relaxed);
  const HostGraph* hg = g->host.get();
  isingx::HaloPlan* out = g->pending.get();
  std::atomic<bool>* done = &g->planned;
  const std::atomic<bool>* cancel = &g->plan_cancel;
  const int32_t parts = g->num_sms, S = g->halo_sweeps;
  try {
    g->planner = std::thread([hg, out, done, cancel, parts, S] {
      choose_halo_plan(*hg, parts, S, out, cancel);
      done->store(true, std::memory_order_release);
    });
  } catch (const std::system_error&) {
    choose_halo_plan(*hg, parts, S, out, cancel);
    g->planned.store(true, std::memory_order_release);
  }
}

void join_planner(ising_graph* g) {
  if (g->planner.joinable()) g->planner.join();
}

// Upload the halo plan once it exists. wait = false: if the planner is still
// running, return with halo_state 0 (not planned yet; a planner is started
// if none ran). halo_state 1 on success, -1 if no plan is possible; returns a
// CUDA error only.
cudaError_t plan_halo(ising_graph* g, bool wait) {
  if (g->halo_state != 0) return cudaSuccess;
  if (!g->host) {
    g->halo_state = -1;
    return cudaSuccess;
  }
  start_planner(g);
  if (!wait && !g->planned.load(std::memory_order_acquire)) return cudaSuccess;
  join_planner(g);
  g->halo_state = -1;
  if (!g->pending) return cudaSuccess;
  isingx::HaloPlan hp = std::move(*g->pending);
  g->pending.reset();
  if (!hp.ok) return cudaSuccess;
  auto kernel = isingx::halo_kernel;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hp.smem_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;  // the device cannot give this much shared memory: no plan
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, isingx::kHaloBlock, hp.smem_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaSuccess;
  do {
    if ((e = alloc_copy(&g->d_halo_hdr, hp.hdr.data(), hp.hdr.size(), g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_words, hp.words.data(), hp.words.size(), g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_slices, hp.slices.data(), hp.slices.size(), g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_gpos, hp.gpos.data(), hp.gpos.size(), g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_imports, hp.imports.data(), std::max<size_t>(1, hp.imports.size()),
                        g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_nbrs, hp.nbrs.data(), std::max<size_t>(1, hp.nbrs.size()),
                        g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_exports, hp.exports.data(), std::max<size_t>(2, hp.exports.size()),
                        g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_halo_quads, hp.quads.data(), std::max<size_t>(3, hp.quads.size()),
                        g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy<unsigned>(&g->d_halo_flags, nullptr,
                                  static_cast<size_t>(hp.parts) * isingx::kHaloFlagStride, g->stream)) != cudaSuccess)
      break;
    if ((e = alloc_copy<int8_t>(&g->d_spins2, nullptr, 2 * static_cast<size_t>(hp.mailbox_slots) + 2,
                                g->stream)) != cudaSuccess)
      break;
    g->halo_mail = static_cast<size_t>(hp.mailbox_slots) + 1;
    // the host vectors are freed on return: wait for the copies
    e = cudaStreamSynchronize(g->stream);
  } while (false);
  if (e != cudaSuccess) {
    free_halo(g);
    g->halo_state = -1;
    if (e != cudaErrorMemoryAllocation) return e;
    cudaGetLastError();  // out of memory: no plan, and no error left for later checks
    return cudaSuccess;
  }
  g->halo_state = 1;
  g->halo_parts = hp.parts;
  g->halo_S = hp.sweeps_per_epoch;
  g->halo_smem = hp.smem_bytes;
  g->halo_ratio = hp.max_work_ratio;
  return cudaSuccess;
}

cudaError_t launch_halo(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                        uint32_t replica, const isingx::PhiloxRounds& rk_in, int par0) {
  cudaError_t e;
  if ((e = barrier_init(g)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(g->d_halo_flags, 0,
                           sizeof(unsigned) * isingx::kHaloFlagStride * static_cast<size_t>(g->halo_parts),
                           g->stream)) != cudaSuccess)
    return e;
  DevGraph d = g->dev();
  isingx::HaloArgs h{};
  h.hdr = g->d_halo_hdr;
  h.words = g->d_halo_words;
  h.slices = g->d_halo_slices;
  h.gpos = g->d_halo_gpos;
  h.imports = g->d_halo_imports;
  h.exports = g->d_halo_exports;
  h.quads = g->d_halo_quads;
  h.nbrs = g->d_halo_nbrs;
  h.mail0 = g->d_spins2;
  h.mail1 = g->d_spins2 + g->halo_mail;
  h.flags = g->d_halo_flags;
  h.error = &g->d_barrier->error;
  h.budget = g->wait_budget_ns > 0 ? static_cast<long long>(g->wait_budget_ns) : isingx::kBarrierBudgetNs;
  h.skip_block = g->fault_kind == ISING_FAULT_SKIP_ARRIVAL ? 1 : 0;
  h.classes = g->num_colours;
  h.sweeps_per_epoch = g->halo_S;
  isingx::PhiloxRounds rk = rk_in;
  void* args[] = {&d, &h, &t_begin, &sweeps, &T, &T0, &replica, &rk, &par0};
  g->launches++;
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(isingx::halo_kernel), dim3(g->halo_parts),
                                     dim3(isingx::kHaloBlock), args, static_cast<size_t>(g->halo_smem), g->stream);
}

// The hub engine (hub.cuh): one cooperative launch, block 0 runs the hub
// classes. Returns cudaErrorCooperativeLaunchTooLarge when fewer than two
// blocks fit on the device.
template <bool PACKED, bool STAGE>
cudaError_t launch_hub_t(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                         uint32_t replica, const isingx::PhiloxRounds& rk_in) {
  auto kernel = isingx::hub_kernel<PACKED, STAGE>;
  const int bit_words = g->n / 32 + 2;
  // the worker blocks keep a copy of the spin map when it fits beside the
  // chain block's tables in one block's shared memory
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
  if (e != cudaSuccess) return e;
  const bool stage = STAGE;
  const int smem = isingx::hub_smem_bytes(g->num_hubs, g->hub_colours, bit_words, stage);
  if (smem > optin) return cudaErrorCooperativeLaunchTooLarge;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, isingx::kHubBlock, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::min(per_sm, 1);
  const int grid = per_sm * g->num_sms;
  // the work split of the non-hub classes was made for one block per SM
  if (grid < 2 || grid != g->hub_grid) return cudaErrorCooperativeLaunchTooLarge;
  if ((e = barrier_init(g)) != cudaSuccess) return e;
  // the sums start at zero (a launch that gave up may have left partial sums)
  if ((e = cudaMemsetAsync(g->d_hub_acc, 0, 3 * sizeof(int32_t) * static_cast<size_t>(g->num_hubs),
                           g->stream)) != cudaSuccess)
    return e;
  DevGraph d = g->dev();
  isingx::HubArgs h{};
  h.hubs = g->num_hubs;
  h.hub_classes = g->hub_colours;
  h.classes = g->num_colours;
  h.class_begin = g->d_class_begin;
  h.class_items = g->d_class_items;
  h.hub_split = g->d_hub_split;
  h.hub_end = g->d_hub_end;
  h.sums = g->d_hub_sums;
  h.num_b_items = g->hub_num_b;
  h.num_items = g->hub_num_items;
  h.acc = g->d_hub_acc;
  h.flips = g->d_hub_flips;
  h.bits = g->d_hub_bits;
  h.bit_words = bit_words;
  h.stage_bits = stage ? 1 : 0;
  h.par_end = g->parity;  // anneal_impl has already advanced it by this call's sweeps
  h.pflips = g->d_hub_pflips;
  h.pos = g->d_pos;
  h.blk = g->d_hub_blk;
  isingx::PhiloxRounds rk = rk_in;
  BarrierState* bs = g->d_barrier;
  void* args[] = {&d, &h, &t_begin, &sweeps, &T, &T0, &replica, &rk, &bs};
  g->launches++;
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid),
                                     dim3(isingx::kHubBlock), args, static_cast<size_t>(smem), g->stream);
}

cudaError_t launch_hub(ising_graph* g, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                       uint32_t replica, const isingx::PhiloxRounds& rk) {
  // the worker blocks keep a copy of the spin map when it fits beside the
  // chain block's tables in one block's shared memory
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
  if (e != cudaSuccess) return e;
  const bool stage = isingx::hub_smem_bytes(g->num_hubs, g->hub_colours, g->n / 32 + 2, true) <= optin;
  if (g->packed)
    return stage ? launch_hub_t<true, true>(g, t_begin, sweeps, T, T0, replica, rk)
                 : launch_hub_t<true, false>(g, t_begin, sweeps, T, T0, replica, rk);
  return stage ? launch_hub_t<false, true>(g, t_begin, sweeps, T, T0, replica, rk)
               : launch_hub_t<false, false>(g, t_begin, sweeps, T, T0, replica, rk);
}

// The non-hub classes' work split for G blocks (block 0 runs the hub
// classes): per class, G item offsets; worker block b takes items
// [blk[b], blk[b + 1]) of the class, a contiguous range of about equal
// estimated work (entries streamed, plus a per-item and per-row cost).
void build_hub_blocks(const WorkPlan& plan, int32_t hub_colours, int32_t num_colours, int32_t G,
                      std::vector<int32_t>* blk) {
  const int32_t workers = G - 1;
  blk->clear();
  std::vector<int64_t> cost;
  for (int32_t c = hub_colours; c < num_colours; ++c) {
    const int32_t ib = plan.class_item_begin[static_cast<size_t>(c)];
    const int32_t ie = plan.class_item_begin[static_cast<size_t>(c) + 1];
    cost.assign(static_cast<size_t>(ie - ib) + 1, 0);
    for (int32_t i = ib; i < ie; ++i) {
      const WorkItem& it = plan.items[static_cast<size_t>(i)];
      int64_t w;
      if (it.v_end < 0)  // slice
        w = 64 + (it.e_end - it.e_begin);
      else if (it.e_end < 0)  // light rows: nv x D words
        w = 32 + static_cast<int64_t>(it.v_end - it.v_begin) * (-it.e_end - 1);
      else  // group rows
        w = 64 + (it.e_end - it.e_begin) + 8 * static_cast<int64_t>(it.v_end - it.v_begin);
      cost[static_cast<size_t>(i - ib) + 1] = cost[static_cast<size_t>(i - ib)] + w;
    }
    const int64_t total = cost.back();
    for (int32_t b = 0; b < workers; ++b) {
      const int64_t goal = total * b / workers;
      blk->push_back(ib + static_cast<int32_t>(std::lower_bound(cost.begin(), cost.end(), goal) - cost.begin()));
    }
    blk->push_back(ie);
    // lower_bound can land on an item boundary past the goal: make the
    // offsets non-decreasing and within the class
    for (size_t k = blk->size() - static_cast<size_t>(G); k < blk->size(); ++k) {
      (*blk)[k] = std::min<int32_t>(std::max<int32_t>((*blk)[k], ib), ie);
      if (k > blk->size() - static_cast<size_t>(G)) (*blk)[k] = std::max((*blk)[k], (*blk)[k - 1]);
    }
  }
}

// Host plan of the hub engine. Rows are sorted by neighbour position and the
// hubs hold the first positions, class by class, so a hub's row lists its
// neighbours in earlier hub classes, then those in later hub classes, then
// the non-hubs: per hub the start of the later-class entries (hub_split) and
// of the non-hub entries (hub_end). Then the field-sum items over the hubs'
// rows, kHubSumChunk entries each: first the hub entries (B, summed once per
// launch), then the other entries (A, summed every sweep).
void build_hub_plan(const HostGraph& hg, std::vector<int32_t>* hub_split, std::vector<int32_t>* hub_end,
                    std::vector<int4>* items, int32_t* num_b) {
  const int32_t X = hg.num_hubs;
  hub_split->assign(static_cast<size_t>(X), 0);
  hub_end->assign(static_cast<size_t>(X), 0);
  int32_t c = 0;
  for (int32_t u = 0; u < X; ++u) {
    while (hg.class_begin[static_cast<size_t>(c) + 1] <= u) ++c;
    const int32_t* b = hg.col.data() + hg.row_ptr[static_cast<size_t>(u)];
    const int32_t* e = hg.col.data() + hg.row_ptr[static_cast<size_t>(u) + 1];
    const int32_t* he = std::lower_bound(b, e, X);
    (*hub_end)[static_cast<size_t>(u)] = static_cast<int32_t>(he - hg.col.data());
    (*hub_split)[static_cast<size_t>(u)] = static_cast<int32_t>(
        std::lower_bound(b, he, hg.class_begin[static_cast<size_t>(c) + 1]) - hg.col.data());
  }
  items->clear();
  for (int kind = 1; kind >= 0; --kind) {
    for (int32_t u = 0; u < X; ++u) {
      const int32_t lo = kind == 1 ? hg.row_ptr[static_cast<size_t>(u)] : (*hub_end)[static_cast<size_t>(u)];
      const int32_t hi = kind == 1 ? (*hub_end)[static_cast<size_t>(u)] : hg.row_ptr[static_cast<size_t>(u) + 1];
      for (int32_t e = lo; e < hi; e += isingx::kHubSumChunk)
        items->push_back(make_int4(u, e, std::min(hi, e + isingx::kHubSumChunk), kind));
    }
    if (kind == 1) *num_b = static_cast<int32_t>(items->size());
  }
}

// Enqueue twice the energy into *slot (device), no host synchronisation.
int enqueue_energy(ising_graph* g, unsigned long long* slot) {
  ISING_CUDA(g, cudaMemsetAsync(slot, 0, sizeof(unsigned long long), g->stream));
  SweepArgs a{};
  const isingx::PhiloxRounds rk{};
  const int32_t all_items[2] = {0, g->num_items};
  ISING_CUDA(g, launch_items<kPassEnergy>(g, g->d_all_items, all_items, 0, 1, a, rk, slot));
  return ISING_OK;
}

int compute_energy(ising_graph* g, int64_t* out) {
  ISING_CUDA(g, cudaMemsetAsync(g->d_energy, 0, sizeof(unsigned long long), g->stream));
  SweepArgs a{};
  const isingx::PhiloxRounds rk{};
  const int32_t all_items[2] = {0, g->num_items};
  ISING_CUDA(g, launch_items<kPassEnergy>(g, g->d_all_items, all_items, 0, 1, a, rk, g->d_energy));
  unsigned long long twice = 0;
  ISING_CUDA(g, cudaMemcpyAsync(&twice, g->d_energy, sizeof(twice), cudaMemcpyDeviceToHost, g->stream));
  ISING_CUDA(g, cudaStreamSynchronize(g->stream));
  const int rc = check_device_error(g);
  if (rc != ISING_OK) return rc;
  *out = static_cast<long long>(twice) / 2;
  return ISING_OK;
}

}  // namespace

extern "C" {

const char* ising_strerror(int status) {
  switch (status) {
    case ISING_OK: return "ok";
    case ISING_EINVAL: return "invalid argument";
    case ISING_ENOMEM: return "out of memory";
    case ISING_ECUDA: return "CUDA error (latched in the handle)";
    case ISING_ETIMEOUT: return "a bounded device-side wait timed out";
    case ISING_ESTATE: return "call not valid in the current state";
    case ISING_ERANGE: return "size or weight out of the supported range";
    default: return "unknown status";
  }
}

int ising_create(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                 uint32_t flags, void* cuda_stream, ising_graph** out) {
  if (out == nullptr) return ISING_EINVAL;
  *out = nullptr;
  if ((flags & ~uint32_t(ISING_CREATE_WEIGHTS_I32)) != 0) return ISING_EINVAL;
  HostGraph hg;
  int rc;
  try {
    rc = isingx::build_host_graph(n, m, src, dst, w, &hg);
  } catch (const std::bad_alloc&) {
    return ISING_ENOMEM;
  }
  if (rc != ISING_OK) return rc;

  ising_graph* g = new (std::nothrow) ising_graph();
  if (g == nullptr) return ISING_ENOMEM;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return ISING_ECUDA;
  }
  cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
  if (g->num_sms < 1) g->num_sms = 1;
  g->n = hg.n;
  g->num_edges = hg.num_edges;
  g->nnz = hg.nnz;
  g->total_weight = hg.total_weight;
  g->num_colours = hg.num_colours;
  // Packed entries need int8 weights and column indices below 2^24 - 1.
  g->packed = hg.fits_int8 && hg.n < (1 << 24) - 1 && !(flags & ISING_CREATE_WEIGHTS_I32);

  WorkPlan plan;
  try {
    // ~32 resident warps per SM share a class; rows longer than a share are sliced.
    isingx::build_work_plan(hg, g->num_sms * 32, 64, 32 * isingx::kRowsPerLane,
                            isingx::light_slots(g->packed), &plan);
    g->colour = hg.colour;
    g->class_item_begin = plan.class_item_begin;
  } catch (const std::bad_alloc&) {
    delete g;
    return ISING_ENOMEM;
  }
  g->num_items = static_cast<int32_t>(plan.items.size());
  g->num_slots = static_cast<int32_t>(plan.split_parts.size());
  // the hub engine's plan (before the columns are packed)
  std::vector<int32_t> hub_split, hub_end, hub_blk;
  std::vector<int4> hub_items;
  g->num_hubs = hg.num_hubs;
  g->hub_colours = hg.hub_colours;
  if (hg.num_hubs >= 1 && hg.num_hubs <= isingx::kHubMaxHubs) {
    try {
      build_hub_plan(hg, &hub_split, &hub_end, &hub_items, &g->hub_num_b);
    } catch (const std::bad_alloc&) {
      delete g;
      return ISING_ENOMEM;
    }
    g->hub_num_items = static_cast<int32_t>(hub_items.size());
    try {
      build_hub_blocks(plan, hg.hub_colours, hg.num_colours, g->num_sms, &hub_blk);
    } catch (const std::bad_alloc&) {
      delete g;
      return ISING_ENOMEM;
    }
  }
  isingx::BlockPlan block;
  std::vector<int32_t> dep_ptr, deps;  // item dependencies (before the columns are packed)
  bool have_deps = false;
  std::vector<int32_t> packed_words;  // graphs kept for the halo plan pack into a copy
  try {
    if (g->packed) isingx::build_block_plan(hg, &block);
    have_deps = isingx::build_item_deps(hg, plan, &dep_ptr, &deps);
  } catch (const std::bad_alloc&) {
    delete g;
    return ISING_ENOMEM;
  }
  // graphs the halo engine may take keep their host graph for its plan
  const bool keep_host = g->packed && !block.ok && hg.num_colours <= isingx::kHaloMaxClasses &&
                         hg.max_degree <= isingx::kHaloMaxWidth && hg.n >= 64 * g->num_sms;

  cudaError_t e = cudaSuccess;
  const size_t N = static_cast<size_t>(hg.n);
  const size_t NNZ = static_cast<size_t>(hg.nnz);
  do {
    if ((e = alloc_copy(&g->d_row_ptr, hg.row_ptr.data(), N + 1, g->stream)) != cudaSuccess) break;
    if (g->packed) {
      // the packed words go into the host column array, or into a copy when
      // the host graph is kept
      int32_t* words = hg.col.data();
      if (keep_host) {
        try {
          packed_words.resize(NNZ);
        } catch (const std::bad_alloc&) {
          e = cudaErrorMemoryAllocation;
          break;
        }
        words = packed_words.data();
      }
      isingx::parallel_ranges(static_cast<int64_t>(NNZ), int64_t(1) << 18, [&](int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; ++k)
          words[k] = static_cast<int32_t>((static_cast<uint32_t>(hg.col[k]) << 8) |
                                          (static_cast<uint32_t>(hg.w[k]) & 0xffu));
      });
      if ((e = alloc_copy(&g->d_adj, words, NNZ, g->stream)) != cudaSuccess) break;
    } else {
      if ((e = alloc_copy(&g->d_col, hg.col.data(), NNZ, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_w, hg.w.data(), NNZ, g->stream)) != cudaSuccess) break;
    }
    const size_t NELL = plan.ell_col.size();
    if (g->packed) {
      isingx::parallel_ranges(static_cast<int64_t>(NELL), int64_t(1) << 18, [&](int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; ++k)
          plan.ell_col[k] = plan.ell_col[k] < 0
                                ? static_cast<int32_t>(static_cast<uint32_t>(hg.n) << 8)
                                : static_cast<int32_t>((static_cast<uint32_t>(plan.ell_col[k]) << 8) |
                                                       (static_cast<uint32_t>(plan.ell_w[k]) & 0xffu));
      });
      if ((e = alloc_copy(&g->d_ell, plan.ell_col.data(), NELL, g->stream)) != cudaSuccess) break;
    } else {
      isingx::parallel_ranges(static_cast<int64_t>(NELL), int64_t(1) << 18, [&](int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; ++k)
          if (plan.ell_col[k] < 0) plan.ell_col[k] = hg.n;  // pad entry, weight 0
      });
      if ((e = alloc_copy(&g->d_ell_col, plan.ell_col.data(), NELL, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_ell_w, plan.ell_w.data(), NELL, g->stream)) != cudaSuccess) break;
    }
    // spins[n] is the pad entry's spin and stays 0
    if ((e = alloc_copy<int8_t>(&g->d_spins, nullptr, N + 1, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_orig, hg.perm.data(), N, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_pos, hg.pos.data(), N, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_items, plan.items.data(), plan.items.size(), g->stream)) != cudaSuccess) break;
    const size_t slots = plan.split_parts.size();
    if ((e = alloc_copy<unsigned long long>(&g->d_slice_acc, nullptr, 2 * slots, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_slice_parts, plan.split_parts.data(), slots, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy<unsigned long long>(&g->d_energy, nullptr, 1, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy<int32_t>(&g->d_flag, nullptr, 1, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy<int8_t>(&g->d_tmp, nullptr, N, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_class_items, plan.class_item_begin.data(),
                        plan.class_item_begin.size(), g->stream)) != cudaSuccess) break;
    const int32_t all_items[2] = {0, g->num_items};
    if ((e = alloc_copy(&g->d_all_items, all_items, 2, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy(&g->d_class_begin, hg.class_begin.data(), hg.class_begin.size(),
                        g->stream)) != cudaSuccess) break;
    if (have_deps) {
      if ((e = alloc_copy(&g->d_dep_ptr, dep_ptr.data(), dep_ptr.size(), g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_deps, deps.data(), deps.size(), g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy<int32_t>(&g->d_done, nullptr, kDoneStride * plan.items.size(), g->stream)) != cudaSuccess) break;
      g->itemflow_ok = true;
    }
    if (block.ok) {
      if ((e = alloc_copy(&g->d_block_words, block.words.data(), block.words.size(), g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_block_chunk_off, block.chunk_off.data(), block.chunk_off.size(),
                          g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_block_chunk_len, block.chunk_len.data(), block.chunk_len.size(),
                          g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_block_class_chunk, block.class_chunk.data(), block.class_chunk.size(),
                          g->stream)) != cudaSuccess) break;
      g->block_ok = true;
      g->block_num_chunks = static_cast<int32_t>(block.chunk_off.size());
      g->block_num_words = static_cast<int32_t>(block.words.size());
    }
    if (!hub_end.empty()) {
      const size_t X = hub_end.size();
      if ((e = alloc_copy(&g->d_hub_split, hub_split.data(), X, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_hub_end, hub_end.data(), X, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_hub_sums, hub_items.data(), hub_items.size(), g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy<int32_t>(&g->d_hub_acc, nullptr, 3 * X, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy<uint32_t>(&g->d_hub_flips, nullptr, (X + 31) / 32, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy<uint32_t>(&g->d_hub_bits, nullptr, N / 32 + 2, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy<uint32_t>(&g->d_hub_pflips, nullptr, N / 32 + 2, g->stream)) != cudaSuccess) break;
      if ((e = alloc_copy(&g->d_hub_blk, hub_blk.data(), hub_blk.size(), g->stream)) != cudaSuccess) break;
      g->hub_grid = g->num_sms;
      g->hub_ok = true;
    }
    if ((e = alloc_copy<unsigned>(&g->d_nflip_bits, nullptr, (N + 31) / 32, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy<int32_t>(&g->d_nflip_list, nullptr, N, g->stream)) != cudaSuccess) break;
    if ((e = alloc_copy<BarrierState>(&g->d_barrier, nullptr, 1, g->stream)) != cudaSuccess) break;
    fill_spins_kernel<<<grid_for(hg.n, 256, g->num_sms * 8), 256, 0, g->stream>>>(
        g->d_spins, hg.n, static_cast<int8_t>(isingx::state_byte(1, 0)));
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    e = cudaStreamSynchronize(g->stream);
  } while (false);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_device(g);
    delete g;
    return e == cudaErrorMemoryAllocation ? ISING_ENOMEM : ISING_ECUDA;
  }
  if (keep_host) g->host.reset(new (std::nothrow) HostGraph(std::move(hg)));
  *out = g;
  return ISING_OK;
}

void ising_destroy(ising_graph* g) {
  if (g == nullptr) return;
  g->plan_cancel.store(true, std::memory_order_relaxed);
  join_planner(g);
  cudaSetDevice(g->device);
  cudaStreamSynchronize(g->stream);
  cudaGetLastError();
  free_device(g);
  delete g;
}

static int check_anneal_args(const ising_graph* g, const ising_schedule* sched, uint32_t sweeps,
                             int mode) {
  if (sched == nullptr) return ISING_EINVAL;
  if (sched->kind == ISING_SCHED_LINEAR) {
    if (!(sched->p0 >= 0.0 && sched->p0 <= 1.0)) return ISING_EINVAL;
  } else if (sched->kind == ISING_SCHED_NFLIP) {
    if (static_cast<int64_t>(sched->n0) > static_cast<int64_t>(g->n)) return ISING_EINVAL;
  } else {
    return ISING_EINVAL;
  }
  if (mode != ISING_MODE_DET && mode != ISING_MODE_RACY) return ISING_EINVAL;
  if (sched->t_total >= (1ull << 32)) return ISING_EINVAL;
  if (sched->t_begin > sched->t_total || sweeps > sched->t_total - sched->t_begin) return ISING_EINVAL;
  return ISING_OK;
}

static int anneal_impl(ising_graph* g, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                       int mode);

int ising_anneal(ising_graph* g, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                 int mode, void* cuda_stream) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  rc = check_anneal_args(g, sched, sweeps, mode);
  if (rc != ISING_OK) return rc;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  return anneal_impl(g, sched, sweeps, seed, mode);
}

static int anneal_trace_impl(ising_graph* g, const ising_schedule* sched, uint32_t sweeps,
                             uint64_t seed, int mode, uint32_t every, int64_t* out_energy);

int ising_anneal_trace(ising_graph* g, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                       int mode, uint32_t every, int64_t* out_energy, void* cuda_stream) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  rc = check_anneal_args(g, sched, sweeps, mode);
  if (rc != ISING_OK) return rc;
  if (every == 0 || out_energy == nullptr) return ISING_EINVAL;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  return anneal_trace_impl(g, sched, sweeps, seed, mode, every, out_energy);
}

static int init_random_impl(ising_graph* g, uint64_t seed, uint32_t replica);

int ising_convergence_region(ising_graph* g, const ising_schedule* sched, uint32_t sweeps,
                             const uint64_t* seeds, uint32_t num_seeds, int mode, uint32_t every,
                             int64_t* out_cut, int64_t* out_min, int64_t* out_max,
                             void* cuda_stream) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  rc = check_anneal_args(g, sched, sweeps, mode);
  if (rc != ISING_OK) return rc;
  if (every == 0 || seeds == nullptr || num_seeds == 0 || out_cut == nullptr || out_min == nullptr ||
      out_max == nullptr)
    return ISING_EINVAL;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t points = (static_cast<size_t>(sweeps) + every - 1) / every;
  std::vector<int64_t> energy;
  try {
    energy.resize(points);
  } catch (const std::bad_alloc&) {
    return ISING_ENOMEM;
  }
  for (uint32_t k = 0; k < num_seeds; ++k) {
    rc = init_random_impl(g, seeds[k], sched->replica);
    if (rc != ISING_OK) return rc;
    rc = anneal_trace_impl(g, sched, sweeps, seeds[k], mode, every, energy.data());
    if (rc != ISING_OK) return rc;
    for (size_t i = 0; i < points; ++i) {
      // Eq. 4 under reading R1: cut = (W - H) / 2
      const int64_t cut = (g->total_weight - energy[i]) / 2;
      out_cut[static_cast<size_t>(k) * points + i] = cut;
      out_min[i] = k == 0 ? cut : std::min(out_min[i], cut);
      out_max[i] = k == 0 ? cut : std::max(out_max[i], cut);
    }
  }
  return ISING_OK;
}

static int anneal_trace_impl(ising_graph* g, const ising_schedule* sched, uint32_t sweeps,
                             uint64_t seed, int mode, uint32_t every, int64_t* out_energy) {
  int rc;
  const size_t points = (static_cast<size_t>(sweeps) + every - 1) / every;
  if (points == 0) return ISING_OK;
  if (points > g->trace_cap) {
    if (g->d_trace) cudaFree(g->d_trace);
    g->d_trace = nullptr;
    g->trace_cap = 0;
    ISING_CUDA(g, cudaMalloc(reinterpret_cast<void**>(&g->d_trace), points * sizeof(unsigned long long)));
    g->trace_cap = points;
  }
  ising_schedule chunk = *sched;
  for (size_t i = 0; i < points; ++i) {
    const uint32_t k = static_cast<uint32_t>(std::min<uint64_t>(every, sweeps - i * every));
    chunk.t_begin = sched->t_begin + i * every;
    rc = anneal_impl(g, &chunk, k, seed, mode);
    if (rc != ISING_OK) return rc;
    rc = enqueue_energy(g, g->d_trace + i);
    if (rc != ISING_OK) return rc;
  }
  std::vector<unsigned long long> twice(points);
  ISING_CUDA(g, cudaMemcpyAsync(twice.data(), g->d_trace, points * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, g->stream));
  ISING_CUDA(g, cudaStreamSynchronize(g->stream));
  rc = check_device_error(g);
  if (rc != ISING_OK) return rc;
  for (size_t i = 0; i < points; ++i) out_energy[i] = static_cast<long long>(twice[i]) / 2;
  return ISING_OK;
}

static int anneal_impl(ising_graph* g, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                       int mode) {
  if (sweeps == 0) return ISING_OK;
  const isingx::PhiloxRounds rk = isingx::philox_rounds(isingx::philox_key(seed, 0u));
  // AUTO: the persistent engine when the device supports cooperative launches.
  int engine = g->engine;
  if (engine == ISING_ENGINE_AUTO) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
    // small graphs: the block engine (inside PERSISTENT); graphs without
    // sliced rows: the item-dataflow engine for deterministic linear
    // schedules; else the grid barrier
    if (!coop) {
      engine = ISING_ENGINE_PHASE;
    } else if (!g->block_ok && mode == ISING_MODE_DET && sched->kind == ISING_SCHED_LINEAR &&
               g->hub_ok) {
      engine = ISING_ENGINE_HUB;
    } else if (!g->block_ok && mode == ISING_MODE_DET && sched->kind == ISING_SCHED_LINEAR) {
      // a handle that anneals more than once gets the halo plan: the second
      // call starts the planner, and no call waits for it
      if (g->auto_calls++ > 0) ISING_CUDA(g, plan_halo(g, false));
      if (g->halo_state == 1 && g->halo_ratio <= kHaloAutoRatio)
        engine = ISING_ENGINE_HALO;
      else
        engine = g->itemflow_ok ? ISING_ENGINE_ITEMFLOW : ISING_ENGINE_PERSISTENT;
    } else {
      engine = ISING_ENGINE_PERSISTENT;
    }
  }
  // every sweep updates every vertex once, flipping its update parity
  const int par0 = g->parity;
  g->parity ^= static_cast<int>(sweeps & 1u);
  // Algorithm 1 (N-flip): no per-spin flips during the sweep, N_t random
  // flips after it. Algorithm 2 (linear): per-spin flips with threshold thr[t].
  const bool nflip = sched->kind == ISING_SCHED_NFLIP;
  const uint32_t n0 = nflip ? sched->n0 : 0u;
  const uint64_t T0 = nflip ? 0 : linear_t0(sched->p0);
  if (engine == ISING_ENGINE_DATAFLOW && mode == ISING_MODE_DET && !nflip) {
    g->engine_used = ISING_ENGINE_DATAFLOW;
    ISING_CUDA(g, launch_flow(g, sched->t_begin, sweeps, sched->t_total, T0, sched->replica, par0, rk));
    return ISING_OK;
  }
  if (engine == ISING_ENGINE_HUB) {
    if (mode == ISING_MODE_DET && !nflip && g->hub_ok) {
      const cudaError_t e = launch_hub(g, sched->t_begin, sweeps, sched->t_total, T0, sched->replica, rk);
      if (e == cudaSuccess) {
        g->engine_used = ISING_ENGINE_HUB;
        return ISING_OK;
      }
      if (e != cudaErrorCooperativeLaunchTooLarge) return cuda_fail(g, e);
      cudaGetLastError();
    }
    engine = ISING_ENGINE_PERSISTENT_GRID;  // racy, N-flip, no hub plan or too few blocks
  }
  if (engine == ISING_ENGINE_HALO) {
    if (mode == ISING_MODE_DET && !nflip) {
      ISING_CUDA(g, plan_halo(g, true));
      if (g->halo_state == 1) {
        g->engine_used = ISING_ENGINE_HALO;
        ISING_CUDA(g, launch_halo(g, sched->t_begin, sweeps, sched->t_total, T0, sched->replica, rk, par0));
        return ISING_OK;
      }
    }
    engine = ISING_ENGINE_ITEMFLOW;  // racy, N-flip or no plan
  }
  if (engine == ISING_ENGINE_ITEMFLOW) {
    if (mode == ISING_MODE_DET && !nflip && g->itemflow_ok) {
      g->engine_used = ISING_ENGINE_ITEMFLOW;
      ISING_CUDA(g, launch_itemflow(g, sched->t_begin, sweeps, sched->t_total, T0, sched->replica, rk));
      return ISING_OK;
    }
    engine = ISING_ENGINE_PERSISTENT_GRID;  // racy, N-flip or sliced rows
  }
  if (engine == ISING_ENGINE_PERSISTENT && mode == ISING_MODE_DET && g->block_ok) {
    g->engine_used = ISING_ENGINE_USED_BLOCK;
    ISING_CUDA(g, launch_block(g, sched->t_begin, sweeps, sched->t_total, T0, sched->replica, rk, n0));
    return ISING_OK;
  }
  if (engine == ISING_ENGINE_PERSISTENT || engine == ISING_ENGINE_DATAFLOW ||
      engine == ISING_ENGINE_PERSISTENT_GRID) {
    g->engine_used = ISING_ENGINE_PERSISTENT_GRID;
    if (mode == ISING_MODE_RACY)
      ISING_CUDA(g, launch_persistent<kPassRacy>(g, g->d_class_items, g->num_colours,
                                                 sched->t_begin, sweeps, sched->t_total, T0,
                                                 sched->replica, rk, n0));
    else
      ISING_CUDA(g, launch_persistent<kPassDet>(g, g->d_class_items, g->num_colours,
                                                sched->t_begin, sweeps, sched->t_total, T0,
                                                sched->replica, rk, n0));
    return ISING_OK;
  }
  g->engine_used = ISING_ENGINE_PHASE;
  SweepArgs a{};
  a.replica = sched->replica;
  for (uint32_t k = 0; k < sweeps; ++k) {
    const uint64_t t = sched->t_begin + k;
    a.t = static_cast<uint32_t>(t);
    a.thr = nflip ? 0u : linear_threshold(sched->p0, sched->t_total, t);
    const int32_t* hi = g->class_item_begin.data();
    if (mode == ISING_MODE_RACY) {
      ISING_CUDA(g, launch_items<kPassRacy>(g, g->d_class_items, hi, 0, g->num_colours, a, rk, nullptr));
    } else {
      for (int32_t c = 0; c < g->num_colours; ++c)
        ISING_CUDA(g, launch_items<kPassDet>(g, g->d_class_items, hi, c, c + 1, a, rk, nullptr));
    }
    const uint32_t N = nflip ? isingx::nflip_count(n0, sched->t_total, t) : 0u;
    if (N > 0u) {
      g->launches++;
      nflip_kernel<<<1, 32, 0, g->stream>>>(g->dev(), g->d_pos, g->d_nflip_bits, g->d_nflip_list, N,
                                            static_cast<uint32_t>(t), sched->replica, rk);
      ISING_CUDA(g, cudaGetLastError());
    }
  }
  return ISING_OK;
}

int ising_energy(ising_graph* g, int64_t* out_energy) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  if (out_energy == nullptr) return ISING_EINVAL;
  return compute_energy(g, out_energy);
}

int ising_cut(ising_graph* g, int64_t* out_cut) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  if (out_cut == nullptr) return ISING_EINVAL;
  int64_t H = 0;
  rc = compute_energy(g, &H);
  if (rc != ISING_OK) return rc;
  *out_cut = (g->total_weight - H) / 2;
  return ISING_OK;
}

int ising_total_weight(ising_graph* g, int64_t* out_w) {
  if (g == nullptr || out_w == nullptr) return ISING_EINVAL;
  *out_w = g->total_weight;
  return ISING_OK;
}

int ising_get_spins(ising_graph* g, int8_t* out, int on_device) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  if (out == nullptr) return ISING_EINVAL;
  const int grid = grid_for(g->n, 256, g->num_sms * 8);
  int8_t* target = on_device ? out : g->d_tmp;
  g->launches++;
  gather_spins_kernel<<<grid, 256, 0, g->stream>>>(target, g->d_spins, g->d_pos, g->n);
  ISING_CUDA(g, cudaGetLastError());
  if (!on_device) {
    ISING_CUDA(g, cudaMemcpyAsync(out, g->d_tmp, static_cast<size_t>(g->n), cudaMemcpyDeviceToHost, g->stream));
    ISING_CUDA(g, cudaStreamSynchronize(g->stream));
    return check_device_error(g);
  }
  return ISING_OK;
}

int ising_set_spins(ising_graph* g, const int8_t* in, int on_device) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  if (in == nullptr) return ISING_EINVAL;
  const int grid = grid_for(g->n, 256, g->num_sms * 8);
  const int8_t* source = in;
  if (on_device) {
    ISING_CUDA(g, cudaMemsetAsync(g->d_flag, 0, sizeof(int32_t), g->stream));
    g->launches++;
  check_spins_kernel<<<grid, 256, 0, g->stream>>>(in, g->n, g->d_flag);
    ISING_CUDA(g, cudaGetLastError());
    int32_t bad = 0;
    ISING_CUDA(g, cudaMemcpyAsync(&bad, g->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, g->stream));
    ISING_CUDA(g, cudaStreamSynchronize(g->stream));
    if (bad) return ISING_EINVAL;
  } else {
    for (int32_t o = 0; o < g->n; ++o)
      if (in[o] != 1 && in[o] != -1) return ISING_EINVAL;
    ISING_CUDA(g, cudaMemcpyAsync(g->d_tmp, in, static_cast<size_t>(g->n), cudaMemcpyHostToDevice, g->stream));
    source = g->d_tmp;
  }
  g->launches++;
  scatter_spins_kernel<<<grid, 256, 0, g->stream>>>(g->d_spins, source, g->d_pos, g->n);
  g->parity = 0;
  ISING_CUDA(g, cudaGetLastError());
  if (!on_device) ISING_CUDA(g, cudaStreamSynchronize(g->stream));
  return ISING_OK;
}

int ising_init_random(ising_graph* g, uint64_t seed, uint32_t replica) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  return init_random_impl(g, seed, replica);
}

static int init_random_impl(ising_graph* g, uint64_t seed, uint32_t replica) {
  const int grid = grid_for(g->n, 256, g->num_sms * 8);
  g->launches++;
  g->parity = 0;
  init_random_kernel<<<grid, 256, 0, g->stream>>>(g->d_spins, g->d_orig, g->n,
                                                  isingx::philox_rounds(isingx::philox_key(seed, 0u)),
                                                  replica);
  ISING_CUDA(g, cudaGetLastError());
  return ISING_OK;
}

int ising_num_colours(ising_graph* g, int32_t* out) {
  if (g == nullptr || out == nullptr) return ISING_EINVAL;
  *out = g->num_colours;
  return ISING_OK;
}

int ising_colouring(ising_graph* g, int32_t* out_colour) {
  if (g == nullptr || out_colour == nullptr) return ISING_EINVAL;
  std::memcpy(out_colour, g->colour.data(), g->colour.size() * sizeof(int32_t));
  return ISING_OK;
}

int ising_num_edges(ising_graph* g, int64_t* out_m) {
  if (g == nullptr || out_m == nullptr) return ISING_EINVAL;
  *out_m = g->num_edges;
  return ISING_OK;
}

int ising_plan_colouring(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int32_t* w, int32_t* out_colour, int32_t* out_num_colours) {
  if (out_colour == nullptr || out_num_colours == nullptr) return ISING_EINVAL;
  HostGraph hg;
  try {
    const int rc = isingx::build_host_graph(n, m, src, dst, w, &hg);
    if (rc != ISING_OK) return rc;
  } catch (const std::bad_alloc&) {
    return ISING_ENOMEM;
  }
  std::memcpy(out_colour, hg.colour.data(), hg.colour.size() * sizeof(int32_t));
  *out_num_colours = hg.num_colours;
  return ISING_OK;
}

int ising_plan_halo(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                    int32_t parts, uint32_t sweeps_per_exchange, int32_t* out_part,
                    int32_t* out_smem_bytes, double* out_work_ratio) {
  if (parts < 1 || sweeps_per_exchange < 1 || sweeps_per_exchange > static_cast<uint32_t>(isingx::kHaloMaxDepth))
    return ISING_EINVAL;
  HostGraph hg;
  isingx::HaloPlan hp;
  std::vector<int32_t> part;
  try {
    const int rc = isingx::build_host_graph(n, m, src, dst, w, &hg);
    if (rc != ISING_OK) return rc;
    if (out_part != nullptr) {
      isingx::bisect_parts(hg, parts, &part);
      for (int32_t o = 0; o < hg.n; ++o) out_part[o] = part[static_cast<size_t>(hg.pos[static_cast<size_t>(o)])];
    }
    isingx::build_halo_plan(hg, parts, static_cast<int32_t>(sweeps_per_exchange), &hp);
  } catch (const std::bad_alloc&) {
    return ISING_ENOMEM;
  }
  if (!hp.ok) return ISING_ESTATE;
  if (out_smem_bytes) *out_smem_bytes = hp.smem_bytes;
  if (out_work_ratio) *out_work_ratio = hp.max_work_ratio;
  return ISING_OK;
}

int ising_launch_count(ising_graph* g, uint64_t* out) {
  if (g == nullptr || out == nullptr) return ISING_EINVAL;
  *out = g->launches;
  return ISING_OK;
}

int ising_engine_used(ising_graph* g, int32_t* out) {
  if (g == nullptr || out == nullptr) return ISING_EINVAL;
  *out = g->engine_used;
  return ISING_OK;
}

int ising_debug_fault(ising_graph* g, int kind, uint64_t wait_budget_ns) {
  if (g == nullptr) return ISING_EINVAL;
  if (kind != ISING_FAULT_NONE && kind != ISING_FAULT_SKIP_ARRIVAL && kind != ISING_FAULT_SHORT_COPY)
    return ISING_EINVAL;
  if (wait_budget_ns > 60000000000ull) return ISING_EINVAL;
  g->fault_kind = kind;
  g->wait_budget_ns = wait_budget_ns;
  return ISING_OK;
}

int ising_set_engine(ising_graph* g, int engine) {
  if (g == nullptr) return ISING_EINVAL;
  if (engine != ISING_ENGINE_AUTO && engine != ISING_ENGINE_PHASE &&
      engine != ISING_ENGINE_PERSISTENT && engine != ISING_ENGINE_DATAFLOW &&
      engine != ISING_ENGINE_PERSISTENT_GRID && engine != ISING_ENGINE_ITEMFLOW &&
      engine != ISING_ENGINE_HALO && engine != ISING_ENGINE_HUB)
    return ISING_EINVAL;
  g->engine = engine;
  return ISING_OK;
}

int ising_set_halo_sweeps(ising_graph* g, uint32_t sweeps_per_exchange) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  if (sweeps_per_exchange > static_cast<uint32_t>(isingx::kHaloMaxDepth)) return ISING_EINVAL;
  if (static_cast<int>(sweeps_per_exchange) == g->halo_sweeps) return ISING_OK;
  ISING_CUDA(g, cudaStreamSynchronize(g->stream));  // no launch still reads the old plan
  join_planner(g);
  g->pending.reset();
  free_halo(g);
  g->halo_sweeps = static_cast<int>(sweeps_per_exchange);
  return ISING_OK;
}

int ising_halo_info(ising_graph* g, int32_t* out_parts, int32_t* out_sweeps, int32_t* out_smem_bytes,
                    double* out_work_ratio) {
  int rc = enter(g);
  if (rc != ISING_OK) return rc;
  ISING_CUDA(g, plan_halo(g, true));
  if (g->halo_state != 1) return ISING_ESTATE;
  if (out_parts) *out_parts = g->halo_parts;
  if (out_sweeps) *out_sweeps = g->halo_S;
  if (out_smem_bytes) *out_smem_bytes = g->halo_smem;
  if (out_work_ratio) *out_work_ratio = g->halo_ratio;
  return ISING_OK;
}

}  // extern "C"

namespace isingx {
int graph_enter(ising_graph* g) { return enter(g); }
int graph_cuda_fail(ising_graph* g, cudaError_t e) { return cuda_fail(g, e); }
}  // namespace isingx
