// Halo engine: one block per part of the graph (host_graph.h, HaloPlan), one
// cooperative launch per anneal call, every sweep of it.
//
// A block keeps its region's spins (int8 +1 / -1), sliced-ELL rows and the
// epoch's flip bits in shared memory. An epoch of S sweeps runs D = S * K
// colour phases there with only block barriers between them (phase j: class
// (j - 1) mod K, rows at most D - j hops out). At the end of the epoch the
// block writes the state bytes of its vertices that other parts import into
// their mailbox slots (one slot per import, laid out in each importer's
// order; two mailbox buffers alternate by epoch), publishes the epoch number
// with a release store, and before the next epoch waits (bounded) until every
// part whose vertices lie in its halo has published the same epoch, then
// reloads its halo from its own contiguous slots. The Philox flip decisions of
// Algorithm 2 do not depend on the spins, so a block draws the next epoch's
// flips before it waits. After the last epoch every block writes its
// vertices into the handle's spin buffer, which the other blocks read only
// for their first epoch.
//
// Mailbox reuse is safe: a block writes buffer (e + 1) & 1 at the end of epoch
// e, after it has seen every neighbour part publish epoch e, i.e. after those
// parts finished reading that buffer in epoch e - 1 (the neighbour relation is
// symmetric: within D hops either way).
#pragma once

#include <cstdint>

#include "host_graph.h"
#include "philox.cuh"
#include "sweep.cuh"

namespace isingx {

constexpr int kHaloBlock = 1024;
constexpr int kHaloFlagStride = 32;  // one completion flag per 128-byte line

struct HaloArgs {
  const int32_t* hdr;
  const int32_t* words;
  const int32_t* slices;
  const int32_t* gpos;
  const int32_t* imports;
  const int32_t* exports;
  const int32_t* quads;
  const int32_t* nbrs;
  int8_t* mail0;      // mailbox buffers (one slot per import of every part), by epoch parity
  int8_t* mail1;
  unsigned* flags;    // per part: epochs published in this launch
  int* error;         // a wait that gave up sets it
  long long budget;   // ns per wait
  int skip_block;     // failure-detection tests: block skip_block - 1 never publishes
  int classes;        // K
  int sweeps_per_epoch;  // S
};

__device__ __forceinline__ unsigned halo_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void halo_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp 0 waits until every neighbour part has published `epoch`; false for
// the whole block once a wait ran out or another block already failed.
__device__ __forceinline__ bool halo_wait(const HaloArgs& h, const int* nbr, int nbr_len, unsigned epoch,
                                          int* abort_flag) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    bool ok = true;
    for (int q = lane; q < nbr_len && ok; q += 32) {
      const unsigned* f = h.flags + static_cast<size_t>(__ldg(nbr + q)) * kHaloFlagStride;
      long long t0 = 0;
      for (unsigned it = 0; halo_ld_acquire(f) < epoch; ++it) {
        if ((it & 63u) == 0u) {
          const long long now = global_ns();
          if (it == 0u) {
            t0 = now;
          } else if (now - t0 > h.budget || ld_relaxed_s32(h.error) != 0) {
            atomicExch(h.error, 1);
            ok = false;
            break;
          }
        }
      }
    }
    ok = __all_sync(kFullMask, ok);
    if (lane == 0 && !ok) *abort_flag = 1;
  }
  __syncthreads();
  return *abort_flag == 0;
}

// Rows [0, rows) of one class's phase (local indices base + r, slices from
// sbeg; spins as int8 +1 / -1): the local field f_i = sum_j w_ij s_j over the
// row's sliced-ELL words, the update of Eq. 2 under the max-cut sign (s_i <-
// -sign f_i, f_i = 0 keeps s_i) and the drawn flip (bit `lane` of the slice's
// word in `bits`). Rows of one class never neighbour one another, so a warp
// gathers up to kChunk of its slices before it writes any update.
__device__ __forceinline__ void halo_rows(const int32_t* sw, const int32_t* ssl, int8_t* sp,
                                          const unsigned* bits, int base, int sbeg, int rows,
                                          int warp, int lane) {
  constexpr int kWarps = kHaloBlock / 32;
  constexpr int kChunk = 4;
  const int ns = (rows + 31) >> 5;
  for (int s0 = warp; s0 < ns; s0 += kChunk * kWarps) {
    int f[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int s = s0 + u * kWarps;
      f[u] = 0;
      if (s < ns) {
        const int sl = ssl[sbeg + s];
        const int32_t* wp = sw + (sl >> 6) + lane;
        const int width = sl & 63;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k < width) {
            const int word = wp[32 * k];
            f[u] += ((word << 24) >> 24) * sp[static_cast<unsigned>(word) >> 8];
          }
        }
        for (int k = 4; k < width; ++k) {
          const int word = wp[32 * k];
          f[u] += ((word << 24) >> 24) * sp[static_cast<unsigned>(word) >> 8];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int s = s0 + u * kWarps;
      const int r = 32 * s + lane;
      if (s < ns && r < rows) {
        int sv = sp[base + r];
        if (f[u] > 0)
          sv = -1;
        else if (f[u] < 0)
          sv = 1;
        if ((bits[sbeg + s] >> lane) & 1u) sv = -sv;
        sp[base + r] = static_cast<int8_t>(sv);
      }
    }
  }
}

// State byte of spin sv with update parity par (bit 0: spin -1; bit 1: parity).
__device__ __forceinline__ int8_t halo_state(int sv, int par) {
  return static_cast<int8_t>((sv < 0 ? 1 : 0) | (par << 1));
}

// par0: the update parity every state byte carries at the launch (every
// sweep updates every vertex once, so it stays uniform).
__global__ void __launch_bounds__(kHaloBlock, 1)
    halo_kernel(DevGraph d, HaloArgs h, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                uint32_t replica, PhiloxRounds rk, int par0) {
  extern __shared__ __align__(16) unsigned char halo_smem[];
  __shared__ int abort_flag;
  __shared__ uint32_t sthr[kHaloMaxDepth];  // the epoch's sweep thresholds
  int* hd = reinterpret_cast<int*>(halo_smem);
  const int p = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x < kHaloHdr) hd[threadIdx.x] = __ldg(h.hdr + static_cast<size_t>(p) * kHaloHdr + threadIdx.x);
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  const int R = hd[kHaloR];
  const int words_len = hd[kHaloWordsLen];
  const int nslices = hd[kHaloSlicesLen];
  const int nquads = hd[kHaloQuadLen];
  const int K = h.classes;
  const int S = h.sweeps_per_epoch;
  const int D = S * K;
  const int ct = kHaloHdrClass;  // class c's table: hd[ct + c * (D + 3) + ...]
  int32_t* sw = hd + kHaloHdr;                                                    // words
  int32_t* ssl = sw + words_len;                                                  // slices
  unsigned* sflip = reinterpret_cast<unsigned*>(ssl + (nslices + 3) / 4 * 4);     // flip bitmap
  uint32_t* squad = sflip + hd[kHaloFlipWords];                                   // quads
  int8_t* sp = reinterpret_cast<int8_t*>(squad + 3 * nquads);                     // spins, R + 1
  uint8_t* sq = reinterpret_cast<uint8_t*>(sp) + (R + 1 + 15) / 16 * 16;          // biases by slot
  const int32_t* gp = h.gpos + hd[kHaloGposOff];
  const int2* imp = reinterpret_cast<const int2*>(h.imports) + hd[kHaloImportOff] / 2;
  const int2* exq = reinterpret_cast<const int2*>(h.exports) + hd[kHaloExportOff] / 2;
  const int32_t* nbr = h.nbrs + hd[kHaloNbrOff];
  const int nbr_len = hd[kHaloNbrLen];

  {
    const int4* gw = reinterpret_cast<const int4*>(h.words + hd[kHaloWordsOff]);
    int4* s4 = reinterpret_cast<int4*>(sw);
    for (int i = threadIdx.x; i < words_len / 4; i += kHaloBlock) s4[i] = __ldg(gw + i);
    for (int i = threadIdx.x; i < nslices; i += kHaloBlock) ssl[i] = __ldg(h.slices + hd[kHaloSlicesOff] + i);
    for (int i = threadIdx.x; i < 3 * nquads; i += kHaloBlock)
      squad[i] = static_cast<uint32_t>(__ldg(h.quads + hd[kHaloQuadOff] + i));
    for (int l = threadIdx.x; l < R; l += kHaloBlock)
      sp[l] = static_cast<int8_t>(1 - 2 * (__ldcg(d.spins + __ldg(gp + l)) & 1));
    if (threadIdx.x == 0) sp[R] = 0;  // the padding entries' spin (weight 0)
    if (d.bias != nullptr) {
      // slot 32 * slice + lane of class c: row (slice - first slice) * 32 + lane
      for (int c = 0; c < K; ++c) {
        const int* tc = hd + ct + c * (D + 3);
        const int U = tc[2 + D - 1];
        for (int r = threadIdx.x; r < U; r += kHaloBlock)
          sq[(tc[1] + (r >> 5)) * 32 + (r & 31)] = __ldg(d.bias + __ldg(gp + tc[0] + r));
      }
    }
  }
  __syncthreads();

  const uint32_t E = (sweeps + static_cast<uint32_t>(S) - 1u) / static_cast<uint32_t>(S);
  for (uint32_t e = 0; e < E; ++e) {
    const int se = static_cast<int>(min(static_cast<uint32_t>(S), sweeps - e * static_cast<uint32_t>(S)));
    const int De = se * K;
    const uint64_t t0 = t_begin + static_cast<uint64_t>(e) * static_cast<uint64_t>(S);
    if (threadIdx.x < se) sthr[threadIdx.x] = sweep_args(t0 + threadIdx.x, T, T0, replica).thr;
    for (int i = threadIdx.x; i < se * nslices; i += kHaloBlock) sflip[i] = 0u;
    __syncthreads();
    // the epoch's flip decisions (Algorithm 2 with R5's draws): one Philox
    // evaluation per quad and sweep sets the bit of every member row that
    // flips in sweep i's bitmap
    for (int i = 0; i < se; ++i) {
      const uint32_t thr0 = sthr[i];
      if (thr0 == 0u) continue;
      const uint32_t t = static_cast<uint32_t>(t0) + static_cast<uint32_t>(i);
      unsigned* bits = sflip + i * nslices;
      for (int q = threadIdx.x; q < nquads; q += kHaloBlock) {
        const uint4 x = philox4x32_10(squad[3 * q], t, replica, 0u, rk);
        const uint32_t s01 = squad[3 * q + 1], s23 = squad[3 * q + 2];
        const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
        const uint32_t slot[4] = {s01 & 0xffffu, s01 >> 16, s23 & 0xffffu, s23 >> 16};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (slot[k] == 0xffffu) continue;
          uint32_t thr = thr0;
          if (d.bias != nullptr) {
            const unsigned long long tq = (static_cast<unsigned long long>(thr0) * sq[slot[k]]) >> 7;
            thr = tq > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(tq);
          }
          if (xs[k] < thr) atomicOr(bits + (slot[k] >> 5), 1u << (slot[k] & 31u));
        }
      }
    }
    if (e > 0) {
      if (!halo_wait(h, nbr, nbr_len, e, &abort_flag)) return;
      const int8_t* mail = ((e & 1u) ? h.mail1 : h.mail0) + hd[kHaloImportOff] / 2;
      const int nimp = hd[kHaloImportLen];
      for (int q = threadIdx.x; q < nimp; q += kHaloBlock)
        sp[__ldg(imp + q).x] = static_cast<int8_t>(1 - 2 * (__ldcg(mail + q) & 1));
    }
    __syncthreads();
    // D_e phases: phase j updates class (j - 1) mod K at most D_e - j hops out
    for (int j = 1; j <= De; ++j) {
      const int* tc = hd + ct + ((j - 1) % K) * (D + 3);
      halo_rows(sw, ssl, sp, sflip + ((j - 1) / K) * nslices, tc[0], tc[1], tc[2 + De - j], warp, lane);
      __syncthreads();
    }
    // publish: the mailbox slots other parts import for epoch e + 1; after
    // the last epoch (from the second on, every neighbour has finished the
    // first epoch's load of the handle's buffer) every own vertex into the
    // handle's buffer
    const int par = par0 ^ static_cast<int>(min((e + 1u) * static_cast<uint32_t>(S), sweeps) & 1u);
    if (e + 1u < E) {
      int8_t* mail = ((e + 1u) & 1u) ? h.mail1 : h.mail0;
      const int nexp = hd[kHaloExportLen];
      for (int q = threadIdx.x; q < nexp; q += kHaloBlock) {
        const int2 ls = __ldg(exq + q);
        mail[ls.y] = halo_state(sp[ls.x], par);
      }
    } else if (E > 1u) {
      for (int c = 0; c < K; ++c) {
        const int* tc = hd + ct + c * (D + 3);
        for (int r = threadIdx.x; r < tc[2]; r += kHaloBlock)
          d.spins[__ldg(gp + tc[0] + r)] = halo_state(sp[tc[0] + r], par);
      }
    }
    // the block barrier orders every thread's export before thread 0's
    // release, and a release covers all writes ordered before it
    __syncthreads();
    if (threadIdx.x == 0 && h.skip_block != p + 1)
      halo_st_release(h.flags + static_cast<size_t>(p) * kHaloFlagStride, e + 1u);
  }
  // a single epoch: write the part's vertices once every neighbour has
  // finished it (and with it its load of the handle's buffer)
  if (E == 1u) {
    if (!halo_wait(h, nbr, nbr_len, 1u, &abort_flag)) return;
    const int par = par0 ^ static_cast<int>(sweeps & 1u);
    for (int c = 0; c < K; ++c) {
      const int* tc = hd + ct + c * (D + 3);
      for (int r = threadIdx.x; r < tc[2]; r += kHaloBlock)
        d.spins[__ldg(gp + tc[0] + r)] = halo_state(sp[tc[0] + r], par);
    }
  }
}

}  // namespace isingx
