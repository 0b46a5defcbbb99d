// Halo engine: one block per part of the graph (host_graph.h, HaloPlan), one
// cooperative launch per anneal call, every sweep of it.
//
// A block keeps its region's state bytes, sliced-ELL rows and the epoch's flip
// bits in shared memory. An epoch of S sweeps runs D = S * K colour phases
// there with only block barriers between them (phase j: class (j - 1) mod K,
// rows at most D - j hops out). At the end of the epoch the block writes its
// own vertices' state bytes to the epoch's spin buffer (two buffers
// alternate), publishes the epoch number with a release store, and before the
// next epoch waits (bounded) until every part whose vertices lie in its halo
// has published the same epoch, then reloads the halo from that buffer. The
// Philox flip decisions of Algorithm 2 do not depend on the spins, so a block
// draws the next epoch's flips before it waits.
//
// Buffer reuse is safe: a block writes buffer (e + 1) & 1 at the end of epoch
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
  int8_t* buf1;       // second spin buffer (the first is DevGraph::spins)
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

__global__ void __launch_bounds__(kHaloBlock, 1)
    halo_kernel(DevGraph d, HaloArgs h, uint64_t t_begin, uint32_t sweeps, uint64_t T, uint64_t T0,
                uint32_t replica, PhiloxRounds rk) {
  extern __shared__ __align__(16) unsigned char halo_smem[];
  __shared__ int abort_flag;
  __shared__ uint32_t sthr[kHaloMaxDepth];  // the epoch's sweep thresholds
  int* hd = reinterpret_cast<int*>(halo_smem);
  const int p = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int kWarps = kHaloBlock / 32;
  if (threadIdx.x < kHaloHdr) hd[threadIdx.x] = __ldg(h.hdr + static_cast<size_t>(p) * kHaloHdr + threadIdx.x);
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  const int R = hd[kHaloR];
  const int words_len = hd[kHaloWordsLen];
  const int nslices = hd[kHaloSlicesLen];
  const int K = h.classes;
  const int S = h.sweeps_per_epoch;
  const int D = S * K;
  const int ct = kHaloHdrClass;  // class c's table: hd[ct + c * (D + 3) + ...]
  int32_t* sw = hd + kHaloHdr;                                      // words
  int32_t* ssl = sw + words_len;                                    // slices
  unsigned* sflip = reinterpret_cast<unsigned*>(ssl + (nslices + 3) / 4 * 4);  // flip bitmap
  const int nquads = hd[kHaloQuadLen];
  uint32_t* squad = sflip + hd[kHaloFlipWords];                     // quads, 3 words each
  uint8_t* sp = reinterpret_cast<uint8_t*>(squad + 3 * nquads);     // state bytes, R + 1
  uint8_t* sq = sp + (R + 1 + 15) / 16 * 16;                        // flip biases, R
  const int fw = (R + 31) >> 5;                                     // bitmap words per sweep
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
    for (int l = threadIdx.x; l < R; l += kHaloBlock) {
      const int v = __ldg(gp + l);
      sp[l] = static_cast<uint8_t>(__ldcg(d.spins + v));
      sq[l] = d.bias != nullptr ? __ldg(d.bias + v) : static_cast<uint8_t>(128);
    }
    if (threadIdx.x == 0) sp[R] = 0;  // the padding entries' spin (weight 0)
  }
  __syncthreads();

  const uint32_t E = (sweeps + static_cast<uint32_t>(S) - 1u) / static_cast<uint32_t>(S);
  for (uint32_t e = 0; e < E; ++e) {
    const int se = static_cast<int>(min(static_cast<uint32_t>(S), sweeps - e * static_cast<uint32_t>(S)));
    const int De = se * K;
    const uint64_t t0 = t_begin + static_cast<uint64_t>(e) * static_cast<uint64_t>(S);
    if (threadIdx.x < se) sthr[threadIdx.x] = sweep_args(t0 + threadIdx.x, T, T0, replica).thr;
    for (int i = threadIdx.x; i < se * fw; i += kHaloBlock) sflip[i] = 0u;
    __syncthreads();
    // the epoch's flip decisions (Algorithm 2 with R5's draws): one Philox
    // evaluation per quad and sweep sets bit l of sweep i's bitmap words for
    // every member row l that flips
    for (int i = 0; i < se; ++i) {
      const uint32_t thr0 = sthr[i];
      if (thr0 == 0u) continue;
      const uint32_t t = static_cast<uint32_t>(t0) + static_cast<uint32_t>(i);
      unsigned* bits = sflip + i * fw;
      for (int q = threadIdx.x; q < nquads; q += kHaloBlock) {
        const uint4 x = philox4x32_10(squad[3 * q], t, replica, 0u, rk);
        const uint32_t l01 = squad[3 * q + 1], l23 = squad[3 * q + 2];
        const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
        const uint32_t ls[4] = {l01 & 0xffffu, l01 >> 16, l23 & 0xffffu, l23 >> 16};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (ls[k] == 0xffffu) continue;
          uint32_t thr = thr0;
          if (d.bias != nullptr) {
            const unsigned long long tq = (static_cast<unsigned long long>(thr0) * sq[ls[k]]) >> 7;
            thr = tq > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(tq);
          }
          if (xs[k] < thr) atomicOr(bits + (ls[k] >> 5), 1u << (ls[k] & 31u));
        }
      }
    }
    if (e > 0) {
      if (!halo_wait(h, nbr, nbr_len, e, &abort_flag)) return;
      const int8_t* src = (e & 1u) ? h.buf1 : d.spins;
      const int nimp = hd[kHaloImportLen];
      for (int q = threadIdx.x; q < nimp; q += kHaloBlock) {
        const int2 lv = __ldg(imp + q);
        sp[lv.x] = static_cast<uint8_t>(__ldcg(src + lv.y));
      }
    }
    __syncthreads();
    // D_e phases (Eq. 2 under the max-cut sign, then the drawn flip)
    for (int j = 1; j <= De; ++j) {
      const unsigned* bits = sflip + ((j - 1) / K) * fw;
      const int c = (j - 1) % K;
      const int* tc = hd + ct + c * (D + 3);
      const int rows = tc[2 + De - j];
      const int ns = (rows + 31) >> 5;
      const int base = tc[0];
      const int sbeg = tc[1];
      // a phase's rows read only other classes' state bytes, so a warp
      // gathers up to kChunk of its slices before it writes any update
      constexpr int kChunk = 4;
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
#pragma unroll 4
            for (int k = 0; k < width; ++k) {
              const int word = wp[32 * k];
              const int wgt = (word << 24) >> 24;
              f[u] += (sp[static_cast<unsigned>(word) >> 8] & 1) ? -wgt : wgt;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int s = s0 + u * kWarps;
          const int r = 32 * s + lane;
          if (s < ns && r < rows) {
            const int b = sp[base + r];
            int bit = b & 1;  // 1 = spin -1
            if (f[u] > 0)
              bit = 1;
            else if (f[u] < 0)
              bit = 0;
            bit ^= static_cast<int>((bits[(base + r) >> 5] >> ((base + r) & 31)) & 1u);
            sp[base + r] = static_cast<uint8_t>(bit | ((b ^ 2) & 2));
          }
        }
      }
      __syncthreads();
    }
    // publish the part's own state bytes for epoch e + 1: those other parts
    // import; after the last epoch every own vertex, into the handle's buffer
    // (directly after an even number of epochs, below after an odd one)
    int8_t* dst = ((e + 1u) & 1u) ? h.buf1 : d.spins;
    if (e + 1u < E) {
      const int nexp = hd[kHaloExportLen];
      for (int q = threadIdx.x; q < nexp; q += kHaloBlock) {
        const int2 lv = __ldg(exq + q);
        dst[lv.y] = static_cast<int8_t>(sp[lv.x]);
      }
    } else if ((E & 1u) == 0u) {
      for (int c = 0; c < K; ++c) {
        const int* tc = hd + ct + c * (D + 3);
        for (int r = threadIdx.x; r < tc[2]; r += kHaloBlock)
          dst[__ldg(gp + tc[0] + r)] = static_cast<int8_t>(sp[tc[0] + r]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && h.skip_block != p + 1) {
      __threadfence();
      halo_st_release(h.flags + static_cast<size_t>(p) * kHaloFlagStride, e + 1u);
    }
  }
  // after an odd number of epochs the handle's buffer was read in epoch
  // E - 1: write the part's vertices once every neighbour has published E
  if (E & 1u) {
    if (!halo_wait(h, nbr, nbr_len, E, &abort_flag)) return;
    for (int c = 0; c < K; ++c) {
      const int* tc = hd + ct + c * (D + 3);
      for (int r = threadIdx.x; r < tc[2]; r += kHaloBlock)
        d.spins[__ldg(gp + tc[0] + r)] = static_cast<int8_t>(sp[tc[0] + r]);
    }
  }
}

}  // namespace isingx
