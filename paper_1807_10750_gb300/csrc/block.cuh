// The block engine: a graph of at most 4095 vertices (host_graph.h,
// build_block_plan) annealed by one block of 512 threads, with block barriers
// between colour classes instead of grid barriers.
//
// The block keeps every state byte in shared memory. Each colour class's
// packed words (row, column, weight) stream into a ring of shared buffers by
// one-dimensional bulk copies (cp.async.bulk, completion on an mbarrier,
// every wait bounded; up to kBlockRing - 1 copies in flight, crossing class
// boundaries); each thread adds the terms w * s_col of eight consecutive
// words into per-row shared accumulators (a running sum flushed where the row
// changes, then a segmented scan across the warp), and each vertex of the
// class applies Eq. 2 and Algorithm 2's flip exactly as the grid engines do.
// The spins are identical to a sweep of one grid phase per class.
//
// When every packed word fits in shared memory with the tables (the
// 800-vertex workload's 38k words take 154 KB), the block loads them once per
// launch instead (resident form): no copies, no waits, and a class costs two
// block barriers.
#pragma once

#include <cstdint>

#include "host_graph.h"
#include "philox.cuh"
#include "sweep.cuh"

namespace isingx {

struct BlockArgs {
  int n;                        // vertices (positions 0 .. n-1)
  int num_chunks;               // word chunks per sweep
  int num_classes;
  const uint32_t* words;        // packed words, by class
  const int32_t* chunk_off;     // per chunk: first word
  const int32_t* chunk_len;     // per chunk: words
  const int32_t* class_chunk;   // per class + 1
  const int32_t* class_pos;     // per class + 1: first position
  long long wait_ns;            // bound of every wait (0: kBlockWaitNs)
  int short_copy;               // failure-detection tests: the first chunk expects 16 more bytes
  int resident_words;           // > 0: every word is kept in shared memory (that many words)
};

constexpr int kBlockThreads = 512;
constexpr int kBlockRing = 4;  // chunk buffers
constexpr int kBlockChunkBytes = kBlockChunkWords * 4;
constexpr int kBlockWordsPerThread = kBlockChunkWords / kBlockThreads;
static_assert(kBlockWordsPerThread % 4 == 0, "whole 16-byte loads per thread");

// Dynamic shared memory: kBlockRing mbarriers and chunk buffers (or, in the
// resident form, every word), an int accumulator per vertex (plus a spare slot
// for the padding words), the chunk table, the class tables, then per vertex
// its state byte, its spin (+1/-1) and its flip decision. Offsets in bytes.
struct BlockLayout {
  int acc, chunk, cls_chunk, cls_pos, state, spin, flip, total;
};

__host__ __device__ inline BlockLayout block_layout(int n, int nch, int ncls, int resident_words) {
  BlockLayout L{};
  int o = 128 + (resident_words > 0 ? ((4 * resident_words + 15) & ~15) : kBlockRing * kBlockChunkBytes);
  L.acc = o;
  o += 4 * (n + 1);
  o = (o + 7) & ~7;
  L.chunk = o;
  o += 8 * nch;
  L.cls_chunk = o;
  o += 4 * (ncls + 1);
  L.cls_pos = o;
  o += 4 * (ncls + 1);
  L.state = o;
  o += n;
  L.spin = o;
  o += n;
  L.flip = o;
  o += n;
  L.total = (o + 15) & ~15;
  return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the barrier initialisation visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: expect `bytes` on bar, then copy [src, src + bytes) to dst.
// dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar, unsigned extra = 0) {
  // extra: bytes expected beyond the copy (failure-detection tests only)
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes + extra)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr long long kBlockWaitNs = 2000000000LL;  // 2 s

// Waits until phase `parity` of bar completes; false after `budget` ns
// (kBlockWaitNs if budget <= 0).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long budget) {
  if (budget <= 0) budget = kBlockWaitNs;
  long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 63u) == 0u) {
      long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (it == 0u)
        t0 = now;
      else if (now - t0 > budget)
        return false;
    }
  }
}

struct BlockShared {
  unsigned long long* bar;  // [kBlockRing]
  uint32_t* buf;            // [kBlockRing][kBlockChunkWords]
  int* acc;                 // [n + 1]
  int2* chunk;              // [nch]: first word, words
  int* cls_chunk;           // [ncls + 1]
  int* cls_pos;             // [ncls + 1]
  uint8_t* state;           // [n]
  int8_t* spin;             // [n]
  uint8_t* flip;            // [n]
};

__device__ __forceinline__ BlockShared block_shared(unsigned char* base, const BlockArgs& ba) {
  const BlockLayout L = block_layout(ba.n, ba.num_chunks, ba.num_classes, ba.resident_words);
  BlockShared s;
  s.bar = reinterpret_cast<unsigned long long*>(base);
  s.buf = reinterpret_cast<uint32_t*>(base + 128);
  s.acc = reinterpret_cast<int*>(base + L.acc);
  s.chunk = reinterpret_cast<int2*>(base + L.chunk);
  s.cls_chunk = reinterpret_cast<int*>(base + L.cls_chunk);
  s.cls_pos = reinterpret_cast<int*>(base + L.cls_pos);
  s.state = base + L.state;
  s.spin = reinterpret_cast<int8_t*>(base + L.spin);
  s.flip = base + L.flip;
  return s;
}

// Once per launch: the mbarriers and the tables.
__device__ __forceinline__ void block_setup(const BlockArgs& ba, const BlockShared& sh) {
  if (threadIdx.x == 0) {
    for (int b = 0; b < kBlockRing; ++b) mbar_init(sh.bar + b, 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < ba.num_chunks; i += blockDim.x)
    sh.chunk[i] = make_int2(ba.chunk_off[i], ba.chunk_len[i]);
  for (int i = threadIdx.x; i <= ba.num_classes; i += blockDim.x) {
    sh.cls_chunk[i] = ba.class_chunk[i];
    sh.cls_pos[i] = ba.class_pos[i];
  }
  // resident form: every word, once (the word count is a multiple of 4)
  for (int i = threadIdx.x; i < ba.resident_words / 4; i += blockDim.x)
    reinterpret_cast<uint4*>(sh.buf)[i] = __ldg(reinterpret_cast<const uint4*>(ba.words) + i);
}

// Issue chunk q of this sweep, whose launch-wide sequence number is sq.
__device__ __forceinline__ void block_issue(const BlockArgs& ba, const BlockShared& sh, int q,
                                            unsigned sq) {
  const unsigned b = sq % kBlockRing;
  // order earlier generic accesses of the buffer before the async write
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int2 c = sh.chunk[q];
  bulk_load(sh.buf + b * kBlockChunkWords, ba.words + c.x, 4u * static_cast<unsigned>(c.y),
            sh.bar + b, (ba.short_copy && sq == 0u) ? 16u : 0u);
}

// The terms of one chunk's words (len of them at buf) added into the rows'
// shared accumulators: each thread takes kBlockWordsPerThread consecutive
// words (a chunk is one pass of the block).
__device__ __forceinline__ void block_chunk(const BlockShared& sh, const uint32_t* buf, int len, int n,
                                            int tid, int lane) {
  // each thread takes kBlockWordsPerThread consecutive words (a chunk is
  // one pass of the block): all terms first (independent shared loads),
  // then a running sum per row, flushed where the row changes
  const int w0 = tid * kBlockWordsPerThread;
  if (__any_sync(kFullMask, w0 < len)) {
    int row[kBlockWordsPerThread], val[kBlockWordsPerThread];
    const uint32_t pad = static_cast<uint32_t>(n) << 20;
#pragma unroll
    for (int h = 0; h < kBlockWordsPerThread / 4; ++h) {
      // chunk lengths are multiples of 4 words: past the end, pad words
      // (spare row n, weight 0)
      const uint4 x = w0 + 4 * h < len ? *reinterpret_cast<const uint4*>(buf + w0 + 4 * h)
                                       : make_uint4(pad, pad, pad, pad);
      const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t w = wv[u];
        const int col = static_cast<int>((w >> 8) & 0xfffu);
        row[4 * h + u] = static_cast<int>(w >> 20);
        val[4 * h + u] = static_cast<int>(static_cast<int8_t>(static_cast<uint8_t>(w & 0xffu))) *
                         sh.spin[col < n ? col : 0];
      }
    }
    int cur = row[0], sum = 0;
#pragma unroll
    for (int h = 0; h < kBlockWordsPerThread; ++h) {
      if (row[h] != cur) {
        atomicAdd(sh.acc + (cur <= n ? cur : n), sum);
        cur = row[h];
        sum = 0;
      }
      sum += val[h];
    }
    // the last run of each thread: lanes ending on the same row add up
    // (segmented scan across the warp), the run's last lane adds to shared
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(kFullMask, sum, o);
      const int r = __shfl_up_sync(kFullMask, cur, o);
      if (lane >= o && r == cur) sum += u;
    }
    const int next = __shfl_down_sync(kFullMask, cur, 1);
    if (lane == 31 || next != cur) atomicAdd(sh.acc + (cur <= n ? cur : n), sum);
  }
}

// Eq. 2 and Algorithm 2 for the vertices of class k, from their accumulated
// fields; the new state bytes go to shared and global memory.
__device__ __forceinline__ void block_decide(const DevGraph& d, const BlockShared& sh, int k, int tid) {
  for (int i = sh.cls_pos[k] + tid; i < sh.cls_pos[k + 1]; i += blockDim.x) {
    const int f = sh.acc[i];
    const int bt = sh.state[i];
    int s = spin_of(bt);
    if (f > 0)
      s = -1;
    else if (f < 0)
      s = 1;
    if (sh.flip[i]) s = -s;
    const int nb = state_byte(s, ((bt >> 1) & 1) ^ 1);
    sh.state[i] = static_cast<uint8_t>(nb);
    sh.spin[i] = static_cast<int8_t>(s);
    d.spins[i] = static_cast<int8_t>(nb);
  }
}

// The sweep's start: state, spin and flip of every vertex into shared memory,
// accumulators cleared.
__device__ __forceinline__ void block_sweep_start(const DevGraph& d, const SweepArgs& a, const PhiloxRounds& rk,
                                                  const BlockShared& sh, int n, int tid) {
  for (int i = tid; i < n; i += blockDim.x) {
    const int b = d.spins[i];
    sh.state[i] = static_cast<uint8_t>(b);
    sh.spin[i] = static_cast<int8_t>(spin_of(b));
    sh.acc[i] = 0;
    sh.flip[i] = flip_drawn(d, i, static_cast<uint32_t>(__ldg(d.orig + i)), a, rk) ? 1 : 0;
  }
  if (tid == 0) sh.acc[n] = 0;
}

// One sweep in the resident form: every class's words are in shared memory
// already, so a class is its chunks, a block barrier, its decisions and a
// block barrier.
__device__ __forceinline__ void block_sweep_resident(const DevGraph& d, const BlockArgs& ba, const SweepArgs& a,
                                                     const PhiloxRounds& rk, const BlockShared& sh) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  block_sweep_start(d, a, rk, sh, ba.n, tid);
  __syncthreads();
  for (int k = 0; k < ba.num_classes; ++k) {
    for (int q = sh.cls_chunk[k]; q < sh.cls_chunk[k + 1]; ++q)
      block_chunk(sh, sh.buf + sh.chunk[q].x, sh.chunk[q].y, ba.n, tid, lane);
    __syncthreads();
    block_decide(d, sh, k, tid);
    __syncthreads();
  }
}

// One sweep a.t of every class. seq numbers chunks over the whole launch:
// chunk sq uses buffer and barrier sq % kBlockRing and completes phase
// (sq / kBlockRing) & 1 of that barrier. While chunk q is processed, chunks
// up to q + kBlockRing - 1 are in flight; the buffer a new copy lands in was
// last read by chunk q - 1, finished before the block barrier that ended its
// iteration. Returns false if a copy did not arrive in time: the error flag
// is set and every copy still in flight is waited for (bounded) first.
__device__ __forceinline__ bool block_sweep(const DevGraph& d, const BlockArgs& ba,
                                            const SweepArgs& a, const PhiloxRounds& rk,
                                            const BlockShared& sh, unsigned& seq) {
  const int tid = threadIdx.x;
  const int n = ba.n;
  const int lane = tid & 31;
  const int nch = ba.num_chunks;
  const unsigned seq0 = seq;  // sequence number of this sweep's chunk 0
  __shared__ int block_ok;
  if (tid == 0) {
    block_ok = 1;
    for (int q = 0; q < nch && q < kBlockRing - 1; ++q) block_issue(ba, sh, q, seq0 + q);
  }
  block_sweep_start(d, a, rk, sh, n, tid);
  __syncthreads();
  int q = 0;  // chunk index within this sweep
  for (int k = 0; k < ba.num_classes; ++k) {
    const int c_end = sh.cls_chunk[k + 1];
    for (; q < c_end; ++q) {
      const unsigned sq = seq0 + q;
      if (tid == 0) {
        if (q + kBlockRing - 1 < nch) block_issue(ba, sh, q + kBlockRing - 1, sq + kBlockRing - 1);
        if (!mbar_wait(sh.bar + sq % kBlockRing, (sq / kBlockRing) & 1u, ba.wait_ns)) {
          block_ok = 0;
          if (d.error) atomicExch(d.error, 1);
        }
      }
      __syncthreads();
      if (!block_ok) break;
      block_chunk(sh, sh.buf + (sq % kBlockRing) * kBlockChunkWords, sh.chunk[q].y, n, tid, lane);
      __syncthreads();
    }
    if (!block_ok) break;
    block_decide(d, sh, k, tid);
    __syncthreads();
  }
  seq = seq0 + static_cast<unsigned>(nch);
  if (block_ok) return true;
  // chunks q .. min(q + kBlockRing, nch) - 1 were issued and not consumed
  if (tid == 0) {
    const int last = q + kBlockRing < nch ? q + kBlockRing : nch;
    for (int j = q; j < last; ++j) {
      const unsigned sj = seq0 + j;
      mbar_wait(sh.bar + sj % kBlockRing, (sj / kBlockRing) & 1u, ba.wait_ns);
    }
  }
  __syncthreads();
  return false;
}

}  // namespace isingx
