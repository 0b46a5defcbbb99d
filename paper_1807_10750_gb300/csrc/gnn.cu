// Warm-start graph network (a project addition; the paper has no learned
// part). Three message-passing layers of width 64 read the annealer's spins
// and local fields (Eq. 2) and predict, per vertex, the spin a longer anneal
// ends in; the prediction seeds the spins (warm start) and scales the
// Algorithm 2 flip threshold per vertex (flip bias). The network is defined
// in include/ising.h (G1-G6); this file holds its inference and training
// kernels and their part of the C ABI.
//
// A graph handle, or a batch's instances taken together as one graph (their
// disjoint union), is seen through a GView; everything runs by graph
// position (colour order) on the graph's stream:
//   rowsum:   per-row sums of |w|, 1, w and w * s_j over the CSR entries,
//             lanes over entries, segmented warp sums, int atomics at row
//             ends (exact).
//   features: x (n x 8 bf16) and c = (d + 1)^-1/2 (G1, G2).
//   chunks:   rows with more than kHeavy entries (hubs) are summed in chunks
//             of kChunk entries, one warp per chunk, into per-chunk partial
//             sums of c_j w_rj h_j; the layer kernels add a heavy row's
//             partials in order. Every aggregate is thus summed in a fixed
//             order (no float atomics) and no tile waits on a hub.
//   layer:    one kernel per layer fuses the aggregation into the dense
//             layer: a 64-row tile gathers a = A_hat h for its rows (a
//             sub-warp per row, lanes over features), rounds [h, a] to bf16
//             into shared memory, and multiplies by W on tensor cores
//             (mma.sync m16n8k16, ldmatrix, fp32 accumulation); bias and
//             relu in the epilogue. a never goes to memory except, when
//             training, as the bf16 operand the backward pass reuses.
//   head:     z = h3 w_o + b_o per row (fp32), with the loss G4 and its
//             gradient when labels are given.
//   backward: one kernel per layer forms dL/dh' = (direct part) + A_hat da
//             of the layer above (the same fused gather), dU = dL/dh' *
//             (h' > 0), dX = dU W^T (tensor cores; direct part fp32, da
//             bf16) and dW += X^T dU (tensor cores, partial sums in
//             registers, fp32 atomics per block), db in fp32.
//   adam:     fp32 master weights, moments, and the bf16 copies the mma
//             kernels read.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ising.h"
#include "batch_view.h"
#include "graph_handle.h"
#include "sweep.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kF = 8;   // input features (G2)
constexpr int kH = 64;  // hidden width (G3)
// flat parameter layout (ising.h)
constexpr int kOffW0 = 0;
constexpr int kOffB0 = kOffW0 + 2 * kF * kH;
constexpr int kOffW1 = kOffB0 + kH;
constexpr int kOffB1 = kOffW1 + 2 * kH * kH;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + 2 * kH * kH;
constexpr int kOffWo = kOffB2 + kH;
constexpr int kOffBo = kOffWo + kH;
constexpr int kNumParams = kOffBo + 1;
static_assert(kNumParams == ISING_GNN_NUM_PARAMS, "parameter layout");

constexpr int kTile = 64;           // rows per tile of the layer kernels
constexpr int kLayerThreads = 256;  // eight warps
constexpr int kChunk = 64;          // CSR entries per chunk of a heavy row
constexpr int kHeavy = 64;          // rows with more entries are summed by chunks

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

struct EdgeView {
  const int32_t* adj;  // packed (col << 8) | (w & 0xff)
  const int32_t* col;  // split format
  const int32_t* w;
  int packed;
};

__device__ __forceinline__ void edge_at(const EdgeView& e, int k, int& col, int& w) {
  if (e.packed) {
    const uint32_t x = static_cast<uint32_t>(__ldg(e.adj + k));
    col = static_cast<int>(x >> 8);
    w = static_cast<int>(static_cast<int8_t>(static_cast<uint8_t>(x & 0xffu)));
  } else {
    col = __ldg(e.col + k);
    w = __ldg(e.w + k);
  }
}

// The graph as the network sees it: a graph handle, or a batch's instances
// as one graph (columns local to an instance, shifted by vbase).
struct GView {
  int n;
  long long nnz;
  const int32_t* row_ptr;
  EdgeView ev;
  const int32_t* vbase;  // per row: added to its entries' columns (null: none)
  const int32_t* rowid;  // row of every entry
  const uint8_t* spins;  // spin of position p is -1 when bit `shift` of spins[p] is set
  int shift;
  const int32_t* hchunk;     // per row: first chunk of a heavy row, else -1 (null: no heavy row)
  const int32_t* chunk_row;  // row of every chunk
  int num_chunks;
};

__device__ __forceinline__ int spin_of(const GView& v, int p) { return 1 - 2 * ((v.spins[p] >> v.shift) & 1); }

__device__ __forceinline__ int col_base(const GView& v, int row) { return v.vbase ? __ldg(v.vbase + row) : 0; }

__device__ __forceinline__ int spin_at(const int8_t* spins, int v) { return 1 - 2 * (spins[v] & 1); }

// Inclusive segmented sum across the warp. Lanes hold consecutive CSR
// entries, so equal rows are contiguous; lanes past the end carry row -1.
template <typename T>
__device__ __forceinline__ T seg_sum(T v, int row, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(kFull, v, o);
    const int r = __shfl_up_sync(kFull, row, o);
    if (lane >= o && r == row) v += u;
  }
  return v;
}

__device__ __forceinline__ bool seg_tail(int row, int lane) {
  const int next = __shfl_down_sync(kFull, row, 1);
  return row >= 0 && (lane == 31 || next != row);
}

__global__ void rowid_kernel(const int32_t* row_ptr, int n, int32_t* rowid) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int e1 = row_ptr[v + 1];
    for (int e = row_ptr[v]; e < e1; ++e) rowid[e] = v;
  }
}

// sums[v] = (sum |w|, degree, sum w, f = sum w s_j) of row v (zeroed first).
__global__ void rowsum_kernel(GView v, int4* sums) {
  const int lane = threadIdx.x & 31;
  const long long nw = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  for (long long base = ((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32;
       base < v.nnz; base += nw * 32) {
    const long long e = base + lane;
    int row = -1, a = 0, c = 0, ws = 0, f = 0;
    if (e < v.nnz) {
      int col, w;
      edge_at(v.ev, static_cast<int>(e), col, w);
      row = __ldg(v.rowid + e);
      a = w < 0 ? -w : w;
      c = 1;
      ws = w;
      f = w * spin_of(v, col + col_base(v, row));
    }
    a = seg_sum(a, row, lane);
    c = seg_sum(c, row, lane);
    ws = seg_sum(ws, row, lane);
    f = seg_sum(f, row, lane);
    if (seg_tail(row, lane)) {
      atomicAdd(&sums[row].x, a);
      atomicAdd(&sums[row].y, c);
      atomicAdd(&sums[row].z, ws);
      atomicAdd(&sums[row].w, f);
    }
  }
}

// G1/G2: x_v = [s, f c^2, s f c^2, log(1 + deg) / 8, (sum w) c^2, 1, 0, 0].
__global__ void features_kernel(GView v, const int4* sums, uint4* x, float* cvec) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < v.n; p += gridDim.x * blockDim.x) {
    const int4 q = sums[p];
    const float s = static_cast<float>(spin_of(v, p));
    const float d1 = static_cast<float>(q.x) + 1.0f;
    const float c2 = 1.0f / d1;
    const float f = static_cast<float>(q.w);
    cvec[p] = 1.0f / sqrtf(d1);
    bf162 p0 = __floats2bfloat162_rn(s, f * c2);
    bf162 p1 = __floats2bfloat162_rn(s * f * c2, log1pf(static_cast<float>(q.y)) * 0.125f);
    bf162 p2 = __floats2bfloat162_rn(static_cast<float>(q.z) * c2, 1.0f);
    bf162 p3 = __floats2bfloat162_rn(0.0f, 0.0f);
    uint4 out;
    memcpy(&out.x, &p0, 4);
    memcpy(&out.y, &p1, 4);
    memcpy(&out.z, &p2, 4);
    memcpy(&out.w, &p3, 4);
    x[p] = out;
  }
}

// ---------------------------------------------------------------------------
// Gathers. A row of width D is read by a sub-warp of G lanes, F features per
// lane: width 64 as 16 lanes x 4 (8-byte loads), width 8 as 4 lanes x 2.

template <int D>
struct RowIO;

template <>
struct RowIO<64> {
  static constexpr int G = 16, F = 4;
  using T = uint2;
  static __device__ __forceinline__ T load(const bf16* p, long long row, int q) {
    return __ldg(reinterpret_cast<const uint2*>(p) + row * 16 + q);
  }
  static __device__ __forceinline__ void store(bf16* p, long long row, int q, T val) {
    reinterpret_cast<uint2*>(p)[row * 16 + q] = val;
  }
  static __device__ __forceinline__ void put(bf16* s, T val) { *reinterpret_cast<uint2*>(s) = val; }
  static __device__ __forceinline__ void add(float (&acc)[F], float coef, T val) {
    bf162 a, b;
    memcpy(&a, &val.x, 4);
    memcpy(&b, &val.y, 4);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    acc[0] += coef * fa.x;
    acc[1] += coef * fa.y;
    acc[2] += coef * fb.x;
    acc[3] += coef * fb.y;
  }
  static __device__ __forceinline__ T pack(const float (&acc)[F]) {
    T out;
    bf162 a = __floats2bfloat162_rn(acc[0], acc[1]), b = __floats2bfloat162_rn(acc[2], acc[3]);
    memcpy(&out.x, &a, 4);
    memcpy(&out.y, &b, 4);
    return out;
  }
};

template <>
struct RowIO<8> {
  static constexpr int G = 4, F = 2;
  using T = uint32_t;
  static __device__ __forceinline__ T load(const bf16* p, long long row, int q) {
    return __ldg(reinterpret_cast<const uint32_t*>(p) + row * 4 + q);
  }
  static __device__ __forceinline__ void store(bf16* p, long long row, int q, T val) {
    reinterpret_cast<uint32_t*>(p)[row * 4 + q] = val;
  }
  static __device__ __forceinline__ void put(bf16* s, T val) { *reinterpret_cast<uint32_t*>(s) = val; }
  static __device__ __forceinline__ void add(float (&acc)[F], float coef, T val) {
    bf162 a;
    memcpy(&a, &val, 4);
    const float2 fa = __bfloat1622float2(a);
    acc[0] += coef * fa.x;
    acc[1] += coef * fa.y;
  }
  static __device__ __forceinline__ T pack(const float (&acc)[F]) {
    bf162 a = __floats2bfloat162_rn(acc[0], acc[1]);
    T out;
    memcpy(&out, &a, 4);
    return out;
  }
};

// acc += sum over entries [e0, e1) of w c_col src[col] (this lane's
// features). Width 64: the 16 lanes of a sub-warp decode up to 64 entries
// at once (column words and c_col, four per lane), then every lane reads its
// 8 bytes of each of those rows, eight rows in flight -- two dependent memory
// rounds per 64 entries. Width 8:
// each of the 4 lanes takes every fourth entry and whole 16-byte rows, four
// entries in flight, and the lanes' sums are combined at the end. Both fix
// the order of every sum.
template <int D>
__device__ __forceinline__ void gather_entries(const GView& v, const float* __restrict__ c,
                                               const bf16* __restrict__ src, int e0, int e1, int base,
                                               int q, float (&acc)[RowIO<D>::F]) {
  using IO = RowIO<D>;
  constexpr int G = IO::G;
  const unsigned lane = threadIdx.x & 31;
  const unsigned mask = ((1u << G) - 1u) << (lane & ~(G - 1u));
  if constexpr (D == 64) {
    // up to 64 entries per round: lane q decodes entries q, q + 16, q + 32,
    // q + 48 of the round (slots 0..3)
    for (int b = e0; b < e1; b += 4 * G) {
      const int cnt = min(4 * G, e1 - b);
      int col[4];
      float cf[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        col[u] = 0;
        cf[u] = 0.0f;
        if (u * G + q < cnt) {
          int w;
          edge_at(v.ev, b + u * G + q, col[u], w);
          col[u] += base;
          cf[u] = static_cast<float>(w);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u * G + q < cnt) cf[u] *= __ldg(c + col[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u * G >= cnt) break;
#pragma unroll
        for (int j0 = 0; j0 < G; j0 += 8) {
          if (u * G + j0 >= cnt) break;
          typename IO::T hv[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int cj = __shfl_sync(mask, col[u], j0 + k, G);
            hv[k] = u * G + j0 + k < cnt ? IO::load(src, cj, q) : typename IO::T{};
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) IO::add(acc, __shfl_sync(mask, cf[u], j0 + k, G), hv[k]);
        }
      }
    }
  } else {
    float a8[8] = {};
    for (int b = e0 + q; b < e1; b += 4 * G) {
      int col[4];
      float cf[4];
      uint4 hv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        col[u] = 0;
        cf[u] = 0.0f;
        if (b + u * G < e1) {
          int w;
          edge_at(v.ev, b + u * G, col[u], w);
          col[u] += base;
          cf[u] = static_cast<float>(w);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = b + u * G < e1;
        cf[u] *= ok ? __ldg(c + col[u]) : 0.0f;
        hv[u] = ok ? __ldg(reinterpret_cast<const uint4*>(src) + col[u]) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t words[4] = {hv[u].x, hv[u].y, hv[u].z, hv[u].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          bf162 p;
          memcpy(&p, &words[k], 4);
          const float2 f2 = __bfloat1622float2(p);
          a8[2 * k] += cf[u] * f2.x;
          a8[2 * k + 1] += cf[u] * f2.y;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a8[k] += __shfl_xor_sync(mask, a8[k], 1, G);
      a8[k] += __shfl_xor_sync(mask, a8[k], 2, G);
    }
#pragma unroll
    for (int f = 0; f < IO::F; ++f) acc[f] += a8[IO::F * q + f];
  }
}

// a_r = c_r * sum_j w_rj c_j src_j for one row (this lane's features): a
// light row by its entries, a heavy row by its chunks' partial sums.
template <int D>
__device__ __forceinline__ void aggregate_row(const GView& v, const float* __restrict__ c,
                                              const bf16* __restrict__ src, const float* __restrict__ partial,
                                              int r, int q, float (&acc)[RowIO<D>::F]) {
  constexpr int F = RowIO<D>::F;
  const int e0 = __ldg(v.row_ptr + r), e1 = __ldg(v.row_ptr + r + 1);
  const int hc = v.hchunk ? __ldg(v.hchunk + r) : -1;
  if (hc >= 0) {
    const int nc = (e1 - e0 + kChunk - 1) / kChunk;
    for (int k = 0; k < nc; ++k) {
      const float* pp = partial + static_cast<size_t>(hc + k) * D + q * F;
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] += pp[f];
    }
  } else {
    gather_entries<D>(v, c, src, e0, e1, col_base(v, r), q, acc);
  }
  const float cr = __ldg(c + r);
#pragma unroll
  for (int f = 0; f < F; ++f) acc[f] *= cr;
}

// partial[k] = sum over chunk k's entries of w c_col src[col] (width D), one
// sub-warp per chunk.
template <int D>
__global__ void __launch_bounds__(256)
    chunk_partial_kernel(GView v, const float* __restrict__ c, const bf16* __restrict__ src,
                         float* __restrict__ partial) {
  using IO = RowIO<D>;
  const int lane = threadIdx.x & 31, q = lane % IO::G;
  const int subs = (gridDim.x * blockDim.x) / IO::G;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / IO::G; k < v.num_chunks; k += subs) {
    const int row = __ldg(v.chunk_row + k);
    const int e0 = __ldg(v.row_ptr + row) + (k - __ldg(v.hchunk + row)) * kChunk;
    const int e1 = min(e0 + kChunk, __ldg(v.row_ptr + row + 1));
    float acc[IO::F] = {};
    gather_entries<D>(v, c, src, e0, e1, col_base(v, row), q, acc);
    float* out = partial + static_cast<size_t>(k) * D + q * IO::F;
#pragma unroll
    for (int f = 0; f < IO::F; ++f) out[f] = acc[f];
  }
}

// ---------------------------------------------------------------------------
// Tensor-core helpers: m16n8k16 bf16 x bf16 -> f32 and ldmatrix loads.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf162(float x, float y) {
  bf162 p = __floats2bfloat162_rn(x, y);
  uint32_t u;
  memcpy(&u, &p, 4);
  return u;
}

// Forward layer: hout = relu([h, a] W + b) with a = A_hat h gathered by the
// tile itself; W [2D][64] bf16 row-major. With a_store, a (bf16) is kept for
// the backward pass. Eight warps: the gather takes two rows (D = 64) or
// eight rows (D = 8) per warp at a time; the product gives each warp 16
// rows x 32 columns.
template <int D>
__global__ void __launch_bounds__(kLayerThreads)
    layer_fwd_kernel(GView v, const float* __restrict__ c, const bf16* __restrict__ h,
                     const float* __restrict__ partial, const bf16* __restrict__ W,
                     const float* __restrict__ bias, bf16* __restrict__ a_store, bf16* __restrict__ hout) {
  using IO = RowIO<D>;
  constexpr int K = 2 * D, KP = K + 8, NP = kH + 8;
  constexpr int RPW = 32 / IO::G;  // rows a warp gathers at a time
  __shared__ __align__(16) bf16 sW[K * NP];
  __shared__ __align__(16) bf16 sX[kTile * KP];
  __shared__ float sB[kH];
  for (int idx = threadIdx.x; idx < K * (kH / 8); idx += blockDim.x) {
    const int k = idx / (kH / 8), cc = idx % (kH / 8);
    *reinterpret_cast<uint4*>(sW + k * NP + cc * 8) = *reinterpret_cast<const uint4*>(W + k * kH + cc * 8);
  }
  if (threadIdx.x < kH) sB[threadIdx.x] = bias[threadIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int sub = lane / IO::G, q = lane % IO::G;
  const int g = lane >> 2, t = lane & 3;
  const int wm = wid & 3, wn = wid >> 2;
  const int n = v.n;
  for (int tile = blockIdx.x; tile * kTile < n; tile += gridDim.x) {
    const int r0 = tile * kTile;
    __syncthreads();
    for (int rl = wid * RPW + sub; rl < kTile; rl += 8 * RPW) {
      const int r = r0 + rl;
      typename IO::T own{}, ab{};
      if (r < n) {
        own = IO::load(h, r, q);
        float acc[IO::F] = {};
        aggregate_row<D>(v, c, h, partial, r, q, acc);
        ab = IO::pack(acc);
        if (a_store != nullptr) IO::store(a_store, r, q, ab);
      }
      IO::put(sX + rl * KP + q * IO::F, own);
      IO::put(sX + rl * KP + D + q * IO::F, ab);
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      uint32_t af[4];
      ldsm_x4(af, sX + (16 * wm + (lane & 7) + ((lane >> 3) & 1) * 8) * KP + ks * 16 + (lane >> 4) * 8);
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        uint32_t bfr[4];
        ldsm_x4_t(bfr, sW + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * NP + 32 * wn + np * 16 +
                           (lane >> 4) * 8);
        mma_bf16(acc[2 * np], af, bfr[0], bfr[1]);
        mma_bf16(acc[2 * np + 1], af, bfr[2], bfr[3]);
      }
    }
    const int rr = r0 + 16 * wm + g;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = 32 * wn + nt * 8 + 2 * t;
      const float b0 = sB[col], b1 = sB[col + 1];
      if (rr < n)
        *reinterpret_cast<uint32_t*>(hout + static_cast<size_t>(rr) * kH + col) =
            pack_bf162(fmaxf(acc[nt][0] + b0, 0.0f), fmaxf(acc[nt][1] + b1, 0.0f));
      if (rr + 8 < n)
        *reinterpret_cast<uint32_t*>(hout + static_cast<size_t>(rr + 8) * kH + col) =
            pack_bf162(fmaxf(acc[nt][2] + b0, 0.0f), fmaxf(acc[nt][3] + b1, 0.0f));
    }
  }
}

// ---------------------------------------------------------------------------
// Fifth-generation tensor cores (tcgen05): the forward layer's product on
// 128-row tiles with the accumulator in tensor memory, in a warp-specialised
// pipeline. Operands sit in shared memory in the canonical no-swizzle K-major
// layout: 8 x 8 bf16 core matrices of 128 contiguous bytes, K-adjacent ones
// kTcLbo bytes apart and 8-row groups K / 8 * 128 bytes apart.
//
//   gather warps (kTcProducers)  rows of a tile -> stage s of a ring of
//                                kTcStages tiles; each warp arrives on full[s]
//   one issuing thread           waits full[s] and a free accumulator, issues
//                                the K / 16 products 128 x 64 x 16, commits
//                                them to empty[s] and acc_full[a]
//   four epilogue warps          wait acc_full[a], read the 128 x 64 fp32
//                                accumulator (tcgen05.ld, one lane quarter
//                                each), arrive on acc_empty[a], add the bias,
//                                apply ReLU and store bf16
//
// No block-wide barrier inside the loop: a gather warp held up by a long row
// delays only its own tile, while the others fill the next stages.

constexpr int kTcRows = 128;       // rows per tile (the product's M)
constexpr int kTcProducers = 27;   // gather warps (with the five others, 1024 threads)
constexpr int kTcStages = 4;       // tiles in the shared-memory ring
constexpr int kTcAcc = 2;          // accumulators of 64 columns in tensor memory
constexpr int kTcIssueWarp = kTcProducers;
constexpr int kTcThreads = (kTcProducers + 1 + 4) * 32;
constexpr int kTcMinBlocks = kTcProducers <= 16 ? 2 : 1;  // blocks per SM the registers are sized for
constexpr int kTcLbo = 128;        // bytes between K-adjacent core matrices

// Byte offset of element (r, k) of a K-major tile with K columns.
__host__ __device__ constexpr int tc_canon(int r, int k, int K) {
  return (r / 8) * (K / 8) * 128 + (k / 8) * kTcLbo + (r % 8) * 16 + (k % 8) * 2;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row) byte offsets, the fixed version bits 46-48 = 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, int K) {
  const uint32_t sbo = static_cast<uint32_t>(K / 8) * 128u;
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((kTcLbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(kH >> 3) << 17) |
                              (static_cast<uint32_t>(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// The tile's products D = A B^T (A: kTcRows x K at sa, B: 64 x K at sb),
// issued by one thread.
template <int K>
__device__ __forceinline__ void tc_issue(uint32_t taddr, uint32_t sa, uint32_t sb) {
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = tc_desc(sa + ks * 2 * kTcLbo, K), db = tc_desc(sb + ks * 2 * kTcLbo, K);
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                 "l"(da), "l"(db), "r"(kTcIdesc), "r"(ks > 0 ? 1u : 0u)
                 : "memory");
  }
}

// bar's next phase completes once the products issued so far have.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mb_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

// Waits for phase `parity` of bar, at most 1 s and only while no role of the
// block has given up (*stop). A wait that runs out sets *stop and *err.
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity, volatile int* stop, int* err) {
  long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (done) return true;
    if (*stop) return false;
    long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (it == 0) {
      t0 = now;
    } else if (now - t0 > 1000000000LL) {
      *stop = 1;
      atomicExch(err, 1);
      return false;
    }
  }
}

// mb_wait by lane 0, its answer taken by the warp.
__device__ __forceinline__ bool mb_wait_warp(uint32_t bar, uint32_t parity, volatile int* stop, int* err) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mb_wait(bar, parity, stop, err) ? 1 : 0;
  return __shfl_sync(kFull, ok, 0) != 0;
}

// 16 consecutive fp32 columns of this warp's 32 accumulator lanes.
__device__ __forceinline__ void tc_ld16(uint32_t addr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared memory of layer_fwd_tc_kernel<D>: the ring of A tiles (kTcRows x
// 2D each), W transposed (64 x 2D), the bias, the mbarriers, the
// tensor-memory address and the stop flag.
__host__ __device__ constexpr int tc_layer_smem(int D) {
  return kTcStages * kTcRows * 2 * D * 2 + kH * 2 * D * 2 + kH * 4 + (2 * kTcStages + 2 * kTcAcc) * 8 + 16;
}

// The forward layer of layer_fwd_kernel with the product on tcgen05, one
// persistent block per SM walking tiles blockIdx.x, + gridDim.x, ... through
// the pipeline above. Any wait that runs out (1 s) sets *err, stops every
// role of the block and leaves the remaining outputs unwritten.
template <int D>
__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks)
    layer_fwd_tc_kernel(GView v, const float* __restrict__ c, const bf16* __restrict__ h,
                        const float* __restrict__ partial, const bf16* __restrict__ W,
                        const float* __restrict__ bias, bf16* __restrict__ a_store, bf16* __restrict__ hout,
                        int* err) {
  using IO = RowIO<D>;
  constexpr int K = 2 * D;
  constexpr int RPW = 32 / IO::G;
  constexpr int kStage = kTcRows * K * 2;
  extern __shared__ __align__(1024) unsigned char tc_mem[];
  unsigned char* sX = tc_mem;                              // kTcStages tiles of kTcRows x K
  unsigned char* sWt = tc_mem + kTcStages * kStage;        // 64 x K (W transposed)
  float* sB = reinterpret_cast<float*>(sWt + kH * K * 2);  // 64
  unsigned long long* full = reinterpret_cast<unsigned long long*>(sB + kH);
  unsigned long long* empty = full + kTcStages;
  unsigned long long* acc_full = empty + kTcStages;
  unsigned long long* acc_empty = acc_full + kTcAcc;
  uint32_t* slot = reinterpret_cast<uint32_t*>(acc_empty + kTcAcc);
  volatile int* stop = reinterpret_cast<volatile int*>(slot + 1);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int idx = tid; idx < K * kH; idx += blockDim.x) {
    const int k = idx / kH, o = idx % kH;
    *reinterpret_cast<bf16*>(sWt + tc_canon(o, k, K)) = W[idx];
  }
  if (tid < kH) sB[tid] = bias[tid];
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(full + s)), "r"(kTcProducers)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(empty + s)) : "memory");
    }
    for (int a = 0; a < kTcAcc; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(acc_full + a)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_addr(acc_empty + a)) : "memory");
    }
    *stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(kTcAcc * kH)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *slot;
  const int n = v.n;
  const int tiles = static_cast<int>((static_cast<long long>(n) + kTcRows - 1) / kTcRows);
  const int mine = tiles > static_cast<int>(blockIdx.x) ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (wid < kTcProducers) {
    const int sub = lane / IO::G, q = lane % IO::G;
    for (int i = 0; i < mine; ++i) {
      const int s = i % kTcStages;
      // stage s is free once the products of tile i - kTcStages completed
      if (i >= kTcStages && !mb_wait_warp(smem_addr(empty + s), ((i / kTcStages) - 1) & 1, stop, err)) break;
      unsigned char* X = sX + s * kStage;
      const int r0 = (blockIdx.x + i * gridDim.x) * kTcRows;
      for (int rl = wid * RPW + sub; rl < kTcRows; rl += kTcProducers * RPW) {
        const int r = r0 + rl;
        typename IO::T own{}, ab{};
        if (r < n) {
          own = IO::load(h, r, q);
          float acc[IO::F] = {};
          aggregate_row<D>(v, c, h, partial, r, q, acc);
          ab = IO::pack(acc);
          if (a_store != nullptr) IO::store(a_store, r, q, ab);
        }
        IO::put(reinterpret_cast<bf16*>(X + tc_canon(rl, q * IO::F, K)), own);
        IO::put(reinterpret_cast<bf16*>(X + tc_canon(rl, D + q * IO::F, K)), ab);
      }
      // this warp's rows, visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mb_arrive(smem_addr(full + s));
    }
  } else if (wid == kTcIssueWarp) {
    if (lane == 0) {
      for (int i = 0; i < mine; ++i) {
        const int s = i % kTcStages, a = i % kTcAcc;
        if (!mb_wait(smem_addr(full + s), (i / kTcStages) & 1, stop, err)) break;
        // accumulator a is free once the epilogue read tile i - kTcAcc
        if (i >= kTcAcc && !mb_wait(smem_addr(acc_empty + a), ((i / kTcAcc) - 1) & 1, stop, err)) break;
        tc_fence_after();
        tc_issue<K>(taddr + static_cast<uint32_t>(kH * a), smem_addr(sX + s * kStage), smem_addr(sWt));
        tc_commit(smem_addr(empty + s));
        tc_commit(smem_addr(acc_full + a));
      }
    }
    __syncwarp();
  } else {
    const int quarter = wid & 3;  // the tensor-memory lanes this warp may read
    for (int i = 0; i < mine; ++i) {
      const int a = i % kTcAcc;
      if (!mb_wait_warp(smem_addr(acc_full + a), (i / kTcAcc) & 1, stop, err)) break;
      tc_fence_after();
      const int row = (blockIdx.x + i * gridDim.x) * kTcRows + 32 * quarter + lane;
      uint4* dst = reinterpret_cast<uint4*>(hout + static_cast<size_t>(row) * kH);
#pragma unroll 1
      for (int c0 = 0; c0 < kH; c0 += 16) {
        uint32_t x[16];
        tc_ld16(taddr + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(kH * a + c0), x);
        if (row < n) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            uint4 o;
            o.x = pack_bf162(fmaxf(__uint_as_float(x[8 * j + 0]) + sB[c0 + 8 * j + 0], 0.0f),
                             fmaxf(__uint_as_float(x[8 * j + 1]) + sB[c0 + 8 * j + 1], 0.0f));
            o.y = pack_bf162(fmaxf(__uint_as_float(x[8 * j + 2]) + sB[c0 + 8 * j + 2], 0.0f),
                             fmaxf(__uint_as_float(x[8 * j + 3]) + sB[c0 + 8 * j + 3], 0.0f));
            o.z = pack_bf162(fmaxf(__uint_as_float(x[8 * j + 4]) + sB[c0 + 8 * j + 4], 0.0f),
                             fmaxf(__uint_as_float(x[8 * j + 5]) + sB[c0 + 8 * j + 5], 0.0f));
            o.w = pack_bf162(fmaxf(__uint_as_float(x[8 * j + 6]) + sB[c0 + 8 * j + 6], 0.0f),
                             fmaxf(__uint_as_float(x[8 * j + 7]) + sB[c0 + 8 * j + 7], 0.0f));
            dst[c0 / 8 + j] = o;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mb_arrive(smem_addr(acc_empty + a));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcAcc * kH) : "memory");
  }
}

// Head: z = h3 w_o + b_o. With labels y (+-1 by position): the loss G4 (sum
// over rows, divided by n on the host), dz = -y sigmoid(-y z) / n, dh3 = dz w_o
// and the head's gradients.
__global__ void head_kernel(const bf162* h3, const float* params, const int8_t* y, int n,
                            float inv_n, float* z, float* dh3, float* grad, double* loss) {
  const int lane = threadIdx.x & 31;
  const float w0 = params[kOffWo + 2 * lane], w1 = params[kOffWo + 2 * lane + 1];
  const float bo = params[kOffBo];
  float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
  double lsum = 0.0;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
    const float2 hv = __bfloat1622float2(h3[static_cast<size_t>(v) * 32 + lane]);
    float s = hv.x * w0 + hv.y * w1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    const float zv = s + bo;
    if (lane == 0) z[v] = zv;
    if (y != nullptr) {
      const float yv = y[v] > 0 ? 1.0f : -1.0f;
      const float m = -yv * zv;
      const float sig = 1.0f / (1.0f + expf(-m));  // sigmoid(-y z)
      const float dz = -yv * sig * inv_n;
      if (lane == 0) {
        lsum += static_cast<double>(fmaxf(m, 0.0f) + log1pf(expf(-fabsf(m))));
        gb += dz;
      }
      float2 d2 = make_float2(dz * w0, dz * w1);
      reinterpret_cast<float2*>(dh3)[static_cast<size_t>(v) * 32 + lane] = d2;
      g0 += dz * hv.x;
      g1 += dz * hv.y;
    }
  }
  if (y == nullptr) return;
  __shared__ float sg[kH + 1];
  __shared__ double sl;
  if (threadIdx.x <= kH) sg[threadIdx.x] = 0.0f;
  if (threadIdx.x == 0) sl = 0.0;
  __syncthreads();
  atomicAdd(&sg[2 * lane], g0);
  atomicAdd(&sg[2 * lane + 1], g1);
  if (lane == 0) {
    atomicAdd(&sg[kH], gb);
    atomicAdd(&sl, lsum);
  }
  __syncthreads();
  if (threadIdx.x < kH) atomicAdd(grad + kOffWo + threadIdx.x, sg[threadIdx.x]);
  if (threadIdx.x == kH) atomicAdd(grad + kOffBo, sg[kH]);
  if (threadIdx.x == 0) atomicAdd(loss, sl);
}

// Backward of one layer (h' = relu([h, a] W + b)). dL/dh' is `direct` plus,
// with AGG, A_hat da_src (da_src = dL/da of the layer above, gathered by the
// tile as in the forward pass). Then dU = dL/dh' * (h' > 0); gW += X^T dU;
// gb += colsum dU; with DX also dX = dU W^T, split into dh_out (fp32, the
// direct part for the layer below) and da_out (bf16, to be propagated).
template <int D, bool DX, bool AGG>
__global__ void __launch_bounds__(kLayerThreads, 2)
    layer_bwd_kernel(GView v, const float* __restrict__ c, const float* __restrict__ direct,
                     const bf16* __restrict__ da_src, const float* __restrict__ partial,
                     const bf16* __restrict__ hn, const bf16* __restrict__ h, const bf16* __restrict__ a,
                     const bf16* __restrict__ W, float* __restrict__ gW, float* __restrict__ gb,
                     float* __restrict__ dh_out, bf16* __restrict__ da_out) {
  constexpr int K2 = 2 * D, KP = K2 + 8, NP = kH + 8;
  constexpr int MT = K2 / 16;  // 16-row tiles of gW; 8 x MT tiles of 16 x 8, MT per warp
  constexpr int WR = DX ? K2 : 1;
  constexpr int XN = K2 / 16;  // dX: 8-column tiles per warp (half of K2 each)
  __shared__ __align__(16) bf16 sW[WR * NP];
  __shared__ __align__(16) bf16 sX[kTile * KP];
  __shared__ __align__(16) bf16 sU[kTile * NP];
  __shared__ float sdb[kH];
  if (DX) {
    for (int idx = threadIdx.x; idx < K2 * (kH / 8); idx += blockDim.x) {
      const int k = idx / (kH / 8), cc = idx % (kH / 8);
      *reinterpret_cast<uint4*>(sW + k * NP + cc * 8) = *reinterpret_cast<const uint4*>(W + k * kH + cc * 8);
    }
  }
  if (threadIdx.x < kH) sdb[threadIdx.x] = 0.0f;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int half = lane >> 4, hl = lane & 15;  // two rows per warp, four columns per lane
  const int wm = wid & 3, wn = wid >> 2;
  const int n = v.n;
  float accW[MT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i) accW[i][0] = accW[i][1] = accW[i][2] = accW[i][3] = 0.0f;
  float dbp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int tile = blockIdx.x; tile * kTile < n; tile += gridDim.x) {
    const int r0 = tile * kTile;
    __syncthreads();
    for (int rl = wid * 2 + half; rl < kTile; rl += 16) {
      const int r = r0 + rl;
      float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (r < n) {
        const float4 d4 = *reinterpret_cast<const float4*>(direct + static_cast<size_t>(r) * kH + 4 * hl);
        float dv[4] = {d4.x, d4.y, d4.z, d4.w};
        if (AGG) {
          float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          aggregate_row<kH>(v, c, da_src, partial, r, hl, acc);
#pragma unroll
          for (int i = 0; i < 4; ++i) dv[i] += acc[i];
        }
        const uint2 hraw = RowIO<kH>::load(hn, r, hl);
        bf162 p0, p1;
        memcpy(&p0, &hraw.x, 4);
        memcpy(&p1, &hraw.y, 4);
        const float2 h0 = __bfloat1622float2(p0), h1 = __bfloat1622float2(p1);
        u[0] = h0.x > 0.0f ? dv[0] : 0.0f;
        u[1] = h0.y > 0.0f ? dv[1] : 0.0f;
        u[2] = h1.x > 0.0f ? dv[2] : 0.0f;
        u[3] = h1.y > 0.0f ? dv[3] : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) dbp[i] += u[i];
      uint2 packed;
      packed.x = pack_bf162(u[0], u[1]);
      packed.y = pack_bf162(u[2], u[3]);
      *reinterpret_cast<uint2*>(sU + rl * NP + 4 * hl) = packed;
    }
    // X = [h, a], both bf16, 16-byte chunks
    constexpr int HC = D / 8, CH = 2 * HC;
    for (int idx = threadIdx.x; idx < kTile * CH; idx += blockDim.x) {
      const int rl = idx / CH, ch = idx % CH;
      const int row = r0 + rl;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (row < n) {
        const bf16* srcp = ch < HC ? h + static_cast<size_t>(row) * D + ch * 8
                                   : a + static_cast<size_t>(row) * D + (ch - HC) * 8;
        val = __ldg(reinterpret_cast<const uint4*>(srcp));
      }
      *reinterpret_cast<uint4*>(sX + rl * KP + ch * 8) = val;
    }
    __syncthreads();
    if (DX) {
      float acc[XN][4];
#pragma unroll
      for (int i = 0; i < XN; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < kH / 16; ++ks) {
        uint32_t af[4];
        ldsm_x4(af, sU + (16 * wm + (lane & 7) + ((lane >> 3) & 1) * 8) * NP + ks * 16 + (lane >> 4) * 8);
#pragma unroll
        for (int np = 0; np < XN / 2; ++np) {
          uint32_t bfr[4];
          // B[k][m] = W[m][k]: W rows are B's columns, so no transpose
          ldsm_x4(bfr, sW + (D * wn + np * 16 + (lane & 7) + (lane >> 4) * 8) * NP + ks * 16 +
                           ((lane >> 3) & 1) * 8);
          mma_bf16(acc[2 * np], af, bfr[0], bfr[1]);
          mma_bf16(acc[2 * np + 1], af, bfr[2], bfr[3]);
        }
      }
      const int rr = r0 + 16 * wm + g;
#pragma unroll
      for (int nt = 0; nt < XN; ++nt) {
        const int col = nt * 8 + 2 * t;  // within this warp's half: wn 0 -> dh, wn 1 -> da
        if (wn == 0) {
          if (rr < n)
            *reinterpret_cast<float2*>(dh_out + static_cast<size_t>(rr) * D + col) = make_float2(acc[nt][0], acc[nt][1]);
          if (rr + 8 < n)
            *reinterpret_cast<float2*>(dh_out + static_cast<size_t>(rr + 8) * D + col) = make_float2(acc[nt][2], acc[nt][3]);
        } else {
          if (rr < n)
            *reinterpret_cast<uint32_t*>(da_out + static_cast<size_t>(rr) * D + col) = pack_bf162(acc[nt][0], acc[nt][1]);
          if (rr + 8 < n)
            *reinterpret_cast<uint32_t*>(da_out + static_cast<size_t>(rr + 8) * D + col) = pack_bf162(acc[nt][2], acc[nt][3]);
        }
      }
    }
    // gW[m][j] += sum_rows X[row][m] dU[row][j]: A = X^T, B = dU (both via
    // transposing loads of the row-major tiles)
#pragma unroll
    for (int ks = 0; ks < kTile / 16; ++ks) {
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        const int tile_id = wid * MT + i;
        const int mt = tile_id / 8, nt = tile_id % 8;
        uint32_t af[4], bfr[4];
        ldsm_x4_t(af, sX + (ks * 16 + (lane & 7) + (lane >> 4) * 8) * KP + mt * 16 + ((lane >> 3) & 1) * 8);
        ldsm_x4_t(bfr, sU + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * NP + nt * 8);
        mma_bf16(accW[i], af, bfr[0], bfr[1]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const int tile_id = wid * MT + i;
    const int mt = tile_id / 8, nt = tile_id % 8;
    const int m = mt * 16 + g, j = nt * 8 + 2 * t;
    atomicAdd(gW + m * kH + j, accW[i][0]);
    atomicAdd(gW + m * kH + j + 1, accW[i][1]);
    atomicAdd(gW + (m + 8) * kH + j, accW[i][2]);
    atomicAdd(gW + (m + 8) * kH + j + 1, accW[i][3]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) atomicAdd(&sdb[4 * hl + i], dbp[i]);
  __syncthreads();
  if (threadIdx.x < kH) atomicAdd(gb + threadIdx.x, sdb[threadIdx.x]);
}

__global__ void cast_weights_kernel(const float* p, bf16* w0, bf16* w1, bf16* w2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * kH * kH; i += gridDim.x * blockDim.x) {
    if (i < 2 * kF * kH) w0[i] = __float2bfloat16_rn(p[kOffW0 + i]);
    w1[i] = __float2bfloat16_rn(p[kOffW1 + i]);
    w2[i] = __float2bfloat16_rn(p[kOffW2 + i]);
  }
}

// Adam (Kingma and Ba) on the fp32 master weights; bc1 = 1 - beta1^t and
// bc2 = 1 - beta2^t come from the host.
__global__ void adam_kernel(float* p, float* m, float* v, const float* g, float lr, float b1,
                            float b2, float bc1, float bc2, float eps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNumParams; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// pos_out[p] = caller[vbase[p] + orig[p]] (vbase null: 0).
__global__ void gather_labels_kernel(const int8_t* caller, const int32_t* orig, const int32_t* vbase, int n,
                                     int8_t* pos_out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    pos_out[v] = caller[(vbase ? vbase[v] : 0) + orig[v]];
}

// caller[vbase[p] + orig[p]] = z[p] (vbase null: 0).
__global__ void scatter_logits_kernel(const float* z, const int32_t* orig, const int32_t* vbase, int n,
                                      float* caller) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    caller[(vbase ? vbase[v] : 0) + orig[v]] = z[v];
}

__global__ void scatter_bias_kernel(const uint8_t* caller, const int32_t* pos, int n, uint8_t* bias) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x)
    bias[pos[o]] = caller[o];
}

__global__ void gather_bias_kernel(const uint8_t* bias, const int32_t* orig, int n, uint8_t* caller) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    caller[orig[v]] = bias[v];
}

// G5 warm start (every state byte rewritten with update parity 0) and,
// with a bias array, G6.
__global__ void warm_start_kernel(const float* z, int n, int8_t* spins, uint8_t* bias) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const float zv = z[v];
    int s = spin_at(spins, v);
    if (zv > 0.0f)
      s = 1;
    else if (zv < 0.0f)
      s = -1;
    spins[v] = static_cast<int8_t>(isingx::state_byte(s, 0));
    if (bias != nullptr) {
      const float q = rintf(512.0f / (1.0f + expf(fabsf(zv))));
      bias[v] = static_cast<uint8_t>(q > 255.0f ? 255.0f : q);
    }
  }
}

// G5 on one replica of a batch: bit `shift` of every position's spin byte.
__global__ void batch_warm_start_kernel(const float* z, int n, uint8_t* spins, int shift) {
  const uint8_t bit = static_cast<uint8_t>(1u << shift);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const float zv = z[v];
    if (zv > 0.0f)
      spins[v] = static_cast<uint8_t>(spins[v] & ~bit);
    else if (zv < 0.0f)
      spins[v] = static_cast<uint8_t>(spins[v] | bit);
  }
}

int grid_of(long long work, int per_block, int cap) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return static_cast<int>(b);
}

}  // namespace

struct ising_gnn {
  int device = 0;
  int status = ISING_OK;
  uint64_t step = 0;
  uint64_t launches = 0;
  float* d_params = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_grad = nullptr;
  bf16* d_w0 = nullptr;
  bf16* d_w1 = nullptr;
  bf16* d_w2 = nullptr;
  double* d_loss = nullptr;
  // workspace, grown to the largest graph seen
  int64_t n_cap = 0;
  int4* d_sums = nullptr;
  float* d_c = nullptr;
  bf16* d_x = nullptr;
  bf16* d_a0 = nullptr;                          // a^0 (bf16), kept for the backward pass
  bf16* d_h[3] = {nullptr, nullptr, nullptr};    // h1, h2, h3
  bf16* d_a[2] = {nullptr, nullptr};             // a^1, a^2 (bf16), kept for the backward pass
  float* d_z = nullptr;
  int8_t* d_y = nullptr;
  float* d_dh[2] = {nullptr, nullptr};           // direct parts of dL/dh
  bf16* d_da[2] = {nullptr, nullptr};            // dL/da of two consecutive layers
  float* d_out = nullptr;  // logits in caller order (host copies)
  int64_t chunk_cap = 0;
  float* d_partial = nullptr;  // per heavy-row chunk: its partial sum (width 64)
  int dense_path = ISING_GNN_DENSE_MMA_SYNC;  // forward layers' product
  int* d_err = nullptr;                      // a tensor-core product that timed out
  int tc_blocks[2] = {0, 0};                 // resident tcgen05 layer blocks per SM (D = 8, 64)
};

namespace {

void free_work(ising_gnn* net) {
  void* ptrs[] = {net->d_sums,  net->d_c,     net->d_x,     net->d_a0,    net->d_h[0],
                  net->d_h[1],  net->d_h[2],  net->d_a[0],  net->d_a[1],  net->d_z,
                  net->d_y,     net->d_dh[0], net->d_dh[1], net->d_da[0], net->d_da[1],
                  net->d_out};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  net->d_sums = nullptr;
  net->d_c = net->d_z = net->d_out = nullptr;
  net->d_x = net->d_a0 = nullptr;
  net->d_h[0] = net->d_h[1] = net->d_h[2] = nullptr;
  net->d_a[0] = net->d_a[1] = net->d_da[0] = net->d_da[1] = nullptr;
  net->d_dh[0] = net->d_dh[1] = nullptr;
  net->d_y = nullptr;
  net->n_cap = 0;
}

void free_net(ising_gnn* net) {
  free_work(net);
  void* ptrs[] = {net->d_params, net->d_m,  net->d_v,    net->d_grad,    net->d_w0,
                  net->d_w1,     net->d_w2, net->d_loss, net->d_partial, net->d_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), (count > 0 ? count : 1) * sizeof(T));
}

cudaError_t ensure_work(ising_gnn* net, int64_t n) {
  if (n <= net->n_cap) return cudaSuccess;
  free_work(net);
  const size_t N = static_cast<size_t>(n);
  cudaError_t e;
  if ((e = dalloc(&net->d_sums, N)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_c, N)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_x, N * kF)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_a0, N * kF)) != cudaSuccess) return e;
  for (int l = 0; l < 3; ++l)
    if ((e = dalloc(&net->d_h[l], N * kH)) != cudaSuccess) return e;
  for (int l = 0; l < 2; ++l) {
    if ((e = dalloc(&net->d_a[l], N * kH)) != cudaSuccess) return e;
    if ((e = dalloc(&net->d_dh[l], N * kH)) != cudaSuccess) return e;
    if ((e = dalloc(&net->d_da[l], N * kH)) != cudaSuccess) return e;
  }
  if ((e = dalloc(&net->d_z, N)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_y, N)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_out, N)) != cudaSuccess) return e;
  net->n_cap = n;
  return cudaSuccess;
}

cudaError_t ensure_partial(ising_gnn* net, int64_t chunks) {
  if (chunks <= net->chunk_cap) return cudaSuccess;
  if (net->d_partial) cudaFree(net->d_partial);
  net->d_partial = nullptr;
  net->chunk_cap = 0;
  const cudaError_t e = dalloc(&net->d_partial, static_cast<size_t>(chunks) * kH);
  if (e == cudaSuccess) net->chunk_cap = chunks;
  return e;
}

int net_fail(ising_gnn* net) {
  cudaGetLastError();
  net->status = ISING_ECUDA;
  return ISING_ECUDA;
}

#define GNN_CUDA(net, call)                          \
  do {                                               \
    if ((call) != cudaSuccess) return net_fail(net); \
  } while (0)

int net_enter(ising_gnn* net, ising_graph* g) {
  if (net == nullptr) return ISING_EINVAL;
  if (net->status != ISING_OK) return net->status;
  const int rc = isingx::graph_enter(g);
  if (rc != ISING_OK) return rc;
  if (g->device != net->device) return ISING_EINVAL;
  return ISING_OK;
}

// A graph and where the network runs it.
struct Ctx {
  GView v;
  cudaStream_t st;
  int sms;
  const int32_t* orig;   // position -> vertex id (within the instance)
  const int32_t* vbase;  // per position: the instance's first position (null: none)
};

// Row ids and heavy-row chunks of a row table, built once per graph and kept
// by its owner: rowid[e] = row of entry e; hchunk[r] = index of row r's first
// chunk if r has more than kHeavy entries, else -1; chunk_row[k] = row of
// chunk k. A graph without heavy rows keeps no chunk arrays.
cudaError_t build_row_tables(const int32_t* d_row_ptr, int n, long long nnz, cudaStream_t st, int sms,
                             int32_t** rowid, int32_t** hchunk, int32_t** chunk_row, int32_t* num_chunks,
                             uint64_t* launches) {
  cudaError_t e = cudaSuccess;
  if (*rowid == nullptr) {
    if ((e = dalloc(rowid, static_cast<size_t>(nnz))) != cudaSuccess) {
      *rowid = nullptr;
      return e;
    }
    rowid_kernel<<<grid_of(n, 256, sms * 8), 256, 0, st>>>(d_row_ptr, n, *rowid);
    (*launches)++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (*num_chunks >= 0) return cudaSuccess;
  std::vector<int32_t> rp(static_cast<size_t>(n) + 1);
  if ((e = cudaMemcpyAsync(rp.data(), d_row_ptr, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return e;
  std::vector<int32_t> hc(static_cast<size_t>(n), -1), rows;
  for (int r = 0; r < n; ++r) {
    const int deg = rp[static_cast<size_t>(r) + 1] - rp[static_cast<size_t>(r)];
    if (deg <= kHeavy) continue;
    hc[static_cast<size_t>(r)] = static_cast<int32_t>(rows.size());
    for (int k = 0; k < (deg + kChunk - 1) / kChunk; ++k) rows.push_back(r);
  }
  if (!rows.empty()) {
    if ((e = dalloc(hchunk, hc.size())) != cudaSuccess) {
      *hchunk = nullptr;
      return e;
    }
    if ((e = dalloc(chunk_row, rows.size())) != cudaSuccess) {
      *chunk_row = nullptr;
      return e;
    }
    if ((e = cudaMemcpyAsync(*hchunk, hc.data(), hc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(*chunk_row, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return e;
  }
  *num_chunks = static_cast<int32_t>(rows.size());
  return cudaSuccess;
}

int graph_ctx(ising_gnn* net, ising_graph* g, Ctx* ctx) {
  GNN_CUDA(net, build_row_tables(g->d_row_ptr, g->n, g->nnz, g->stream, g->num_sms, &g->d_rowid,
                                 &g->d_gnn_hchunk, &g->d_gnn_chunk_row, &g->gnn_num_chunks, &net->launches));
  GView& v = ctx->v;
  v.n = g->n;
  v.nnz = g->nnz;
  v.row_ptr = g->d_row_ptr;
  v.ev.adj = g->d_adj;
  v.ev.col = g->d_col;
  v.ev.w = g->d_w;
  v.ev.packed = g->packed ? 1 : 0;
  v.vbase = nullptr;
  v.rowid = g->d_rowid;
  v.spins = reinterpret_cast<const uint8_t*>(g->d_spins);
  v.shift = 0;
  v.num_chunks = g->gnn_num_chunks;
  v.hchunk = v.num_chunks > 0 ? g->d_gnn_hchunk : nullptr;
  v.chunk_row = g->d_gnn_chunk_row;
  ctx->st = g->stream;
  ctx->sms = g->num_sms;
  ctx->orig = g->d_orig;
  ctx->vbase = nullptr;
  return ISING_OK;
}

int batch_ctx(ising_gnn* net, ising_batch* b, uint32_t replica, Ctx* ctx, isingx::BatchUnion* u) {
  if (net == nullptr) return ISING_EINVAL;
  if (net->status != ISING_OK) return net->status;
  int rc = isingx::batch_union(b, u);
  if (rc != ISING_OK) return rc;
  if (u->device != net->device || replica >= static_cast<uint32_t>(u->replicas)) return ISING_EINVAL;
  GNN_CUDA(net, build_row_tables(u->row_ptr, u->n, u->nnz, u->stream, u->num_sms, u->rowid, u->hchunk,
                                 u->chunk_row, u->num_chunks, &net->launches));
  GView& v = ctx->v;
  v.n = u->n;
  v.nnz = u->nnz;
  v.row_ptr = u->row_ptr;
  v.ev.adj = u->adj;
  v.ev.col = nullptr;
  v.ev.w = nullptr;
  v.ev.packed = 1;
  v.vbase = u->vbase;
  v.rowid = *u->rowid;
  v.spins = u->spins;
  v.shift = static_cast<int>(replica);
  v.num_chunks = *u->num_chunks;
  v.hchunk = v.num_chunks > 0 ? *u->hchunk : nullptr;
  v.chunk_row = *u->chunk_row;
  ctx->st = u->stream;
  ctx->sms = u->num_sms;
  ctx->orig = u->orig;
  ctx->vbase = u->vbase;
  return ISING_OK;
}

// Chunk partial sums of src (width D) when the graph has heavy rows.
template <int D>
int run_chunks(ising_gnn* net, const Ctx& x, const bf16* src) {
  if (x.v.num_chunks <= 0) return ISING_OK;
  chunk_partial_kernel<D><<<grid_of(static_cast<long long>(x.v.num_chunks) * RowIO<D>::G, 256, x.sms * 16), 256, 0,
                            x.st>>>(x.v, net->d_c, src, net->d_partial);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  return ISING_OK;
}

// One forward layer (aggregation fused with the product) on the chosen
// dense path: tcgen05 with 128-row tiles, or mma.sync with 64-row tiles.
template <int D>
int run_layer(ising_gnn* net, const Ctx& x, const bf16* h, const bf16* W, const float* bias, bf16* a_store,
              bf16* hout) {
  const int n = x.v.n;
  if (net->dense_path == ISING_GNN_DENSE_TCGEN05) {
    const int smem = tc_layer_smem(D);
    int& per_sm = net->tc_blocks[D == kH ? 1 : 0];
    if (per_sm == 0) {
      const void* fn = reinterpret_cast<const void*>(layer_fwd_tc_kernel<D>);
      GNN_CUDA(net, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      GNN_CUDA(net, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, smem));
      // each block holds 128 of the SM's 512 tensor-memory columns
      per_sm = std::max(1, std::min(per_sm, 4));
    }
    const long long tiles = (static_cast<long long>(n) + kTcRows - 1) / kTcRows;
    const int grid = static_cast<int>(std::min<long long>(tiles, static_cast<long long>(x.sms) * per_sm));
    if (grid > 0)
      layer_fwd_tc_kernel<D><<<grid, kTcThreads, smem, x.st>>>(x.v, net->d_c, h, net->d_partial, W, bias, a_store,
                                                               hout, net->d_err);
  } else {
    layer_fwd_kernel<D><<<(n + kTile - 1) / kTile, kLayerThreads, 0, x.st>>>(x.v, net->d_c, h, net->d_partial, W,
                                                                            bias, a_store, hout);
  }
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  return ISING_OK;
}

// A tensor-core product that timed out (read after the stream has synchronised).
int check_err(ising_gnn* net) {
  int e = 0;
  GNN_CUDA(net, cudaMemcpy(&e, net->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    net->status = ISING_ETIMEOUT;
    return ISING_ETIMEOUT;
  }
  return ISING_OK;
}

// Forward pass over the graph from its current spins; with labels (by
// position in net->d_y) also the loss and dL/dh3 into net->d_dh[0], and the
// aggregates a^l kept for the backward pass.
int run_forward(ising_gnn* net, const Ctx& x, bool with_labels) {
  const int n = x.v.n;
  const long long nnz = x.v.nnz;
  cudaStream_t st = x.st;
  const int sms = x.sms;
  GNN_CUDA(net, ensure_work(net, n));
  GNN_CUDA(net, ensure_partial(net, x.v.num_chunks));
  const int ent_grid = grid_of((nnz + 31) / 32 * 32, 256, sms * 16);
  GNN_CUDA(net, cudaMemsetAsync(net->d_sums, 0, sizeof(int4) * static_cast<size_t>(n), st));
  if (nnz > 0) {
    rowsum_kernel<<<ent_grid, 256, 0, st>>>(x.v, net->d_sums);
    net->launches++;
  }
  features_kernel<<<grid_of(n, 256, sms * 8), 256, 0, st>>>(x.v, net->d_sums, reinterpret_cast<uint4*>(net->d_x),
                                                             net->d_c);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  int rc = run_chunks<kF>(net, x, net->d_x);
  if (rc != ISING_OK) return rc;
  rc = run_layer<kF>(net, x, net->d_x, net->d_w0, net->d_params + kOffB0, with_labels ? net->d_a0 : nullptr,
                     net->d_h[0]);
  if (rc != ISING_OK) return rc;
  for (int l = 1; l <= 2; ++l) {
    rc = run_chunks<kH>(net, x, net->d_h[l - 1]);
    if (rc != ISING_OK) return rc;
    rc = run_layer<kH>(net, x, net->d_h[l - 1], l == 1 ? net->d_w1 : net->d_w2,
                       net->d_params + (l == 1 ? kOffB1 : kOffB2), with_labels ? net->d_a[l - 1] : nullptr,
                       net->d_h[l]);
    if (rc != ISING_OK) return rc;
  }
  if (with_labels) GNN_CUDA(net, cudaMemsetAsync(net->d_loss, 0, sizeof(double), st));
  head_kernel<<<grid_of(static_cast<long long>(n) * 32, 256, sms * 8), 256, 0, st>>>(
      reinterpret_cast<const bf162*>(net->d_h[2]), net->d_params, with_labels ? net->d_y : nullptr, n,
      1.0f / static_cast<float>(n), net->d_z, net->d_dh[0], net->d_grad, net->d_loss);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  return ISING_OK;
}

// Backward pass after run_forward(with_labels): gradients into net->d_grad
// (zeroed by the caller before the head kernel ran).
int run_backward(ising_gnn* net, const Ctx& x) {
  const int n = x.v.n;
  cudaStream_t st = x.st;
  // two blocks per SM (registers); each keeps its dW partial sums to the end
  const int grid = grid_of((n + kTile - 1) / kTile, 1, x.sms * 2);
  // layer 2: dL/dh3 (d_dh[0]) -> direct part of dL/dh2 (d_dh[1]), dL/da2 (d_da[0])
  layer_bwd_kernel<kH, true, false><<<grid, kLayerThreads, 0, st>>>(
      x.v, net->d_c, net->d_dh[0], nullptr, nullptr, net->d_h[2], net->d_h[1], net->d_a[1], net->d_w2,
      net->d_grad + kOffW2, net->d_grad + kOffB2, net->d_dh[1], net->d_da[0]);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  // layer 1: dL/dh2 = d_dh[1] + A_hat d_da[0] -> d_dh[0], d_da[1]
  int rc = run_chunks<kH>(net, x, net->d_da[0]);
  if (rc != ISING_OK) return rc;
  layer_bwd_kernel<kH, true, true><<<grid, kLayerThreads, 0, st>>>(
      x.v, net->d_c, net->d_dh[1], net->d_da[0], net->d_partial, net->d_h[1], net->d_h[0], net->d_a[0],
      net->d_w1, net->d_grad + kOffW1, net->d_grad + kOffB1, net->d_dh[0], net->d_da[1]);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  // layer 0: dL/dh1 = d_dh[0] + A_hat d_da[1]
  rc = run_chunks<kH>(net, x, net->d_da[1]);
  if (rc != ISING_OK) return rc;
  layer_bwd_kernel<kF, false, true><<<grid, kLayerThreads, 0, st>>>(
      x.v, net->d_c, net->d_dh[0], net->d_da[1], net->d_partial, net->d_h[0], net->d_x, net->d_a0, net->d_w0,
      net->d_grad + kOffW0, net->d_grad + kOffB0, nullptr, nullptr);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  return ISING_OK;
}

int load_labels(ising_gnn* net, const Ctx& x, const int8_t* labels, int on_device) {
  const int n = x.v.n;
  const int8_t* src = labels;
  if (!on_device) {
    for (int i = 0; i < n; ++i)
      if (labels[i] != 1 && labels[i] != -1) return ISING_EINVAL;
    GNN_CUDA(net, cudaMemcpyAsync(net->d_out, labels, static_cast<size_t>(n), cudaMemcpyHostToDevice, x.st));
    src = reinterpret_cast<const int8_t*>(net->d_out);
  }
  gather_labels_kernel<<<grid_of(n, 256, x.sms * 8), 256, 0, x.st>>>(src, x.orig, x.vbase, n, net->d_y);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  if (!on_device) GNN_CUDA(net, cudaStreamSynchronize(x.st));
  return ISING_OK;
}

int gradients_impl(ising_gnn* net, const Ctx& x, const int8_t* labels, int on_device) {
  if (labels == nullptr) return ISING_EINVAL;
  GNN_CUDA(net, ensure_work(net, x.v.n));
  int rc = load_labels(net, x, labels, on_device);
  if (rc != ISING_OK) return rc;
  GNN_CUDA(net, cudaMemsetAsync(net->d_grad, 0, sizeof(float) * kNumParams, x.st));
  rc = run_forward(net, x, true);
  if (rc != ISING_OK) return rc;
  return run_backward(net, x);
}

// Logits of the context's graph into out (caller order), host or device.
int forward_out(ising_gnn* net, const Ctx& x, float* out_logits, int on_device) {
  int rc = run_forward(net, x, false);
  if (rc != ISING_OK) return rc;
  float* dst = on_device ? out_logits : net->d_out;
  scatter_logits_kernel<<<grid_of(x.v.n, 256, x.sms * 8), 256, 0, x.st>>>(net->d_z, x.orig, x.vbase, x.v.n, dst);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  if (!on_device) {
    GNN_CUDA(net, cudaMemcpyAsync(out_logits, net->d_out, sizeof(float) * static_cast<size_t>(x.v.n),
                                  cudaMemcpyDeviceToHost, x.st));
    GNN_CUDA(net, cudaStreamSynchronize(x.st));
    return check_err(net);
  }
  return ISING_OK;
}

int read_loss(ising_gnn* net, const Ctx& x, float* out_loss) {
  double l = 0.0;
  GNN_CUDA(net, cudaMemcpyAsync(&l, net->d_loss, sizeof(double), cudaMemcpyDeviceToHost, x.st));
  GNN_CUDA(net, cudaStreamSynchronize(x.st));
  *out_loss = static_cast<float>(l / static_cast<double>(x.v.n));
  return check_err(net);
}

// The gradient's public tail: copy it and the loss out when asked.
int gradients_out(ising_gnn* net, const Ctx& x, float* out_loss, float* out_grad) {
  if (out_grad != nullptr) {
    GNN_CUDA(net, cudaMemcpyAsync(out_grad, net->d_grad, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, x.st));
    GNN_CUDA(net, cudaStreamSynchronize(x.st));
    const int rc = check_err(net);
    if (rc != ISING_OK) return rc;
  }
  if (out_loss != nullptr) return read_loss(net, x, out_loss);
  return ISING_OK;
}

// One Adam step from net->d_grad, then fresh bf16 weight copies.
int adam_step(ising_gnn* net, const Ctx& x, float lr) {
  net->step++;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = static_cast<float>(1.0 - std::pow(b1, static_cast<double>(net->step)));
  const float bc2 = static_cast<float>(1.0 - std::pow(b2, static_cast<double>(net->step)));
  adam_kernel<<<grid_of(kNumParams, 256, 128), 256, 0, x.st>>>(net->d_params, net->d_m, net->d_v, net->d_grad, lr,
                                                               static_cast<float>(b1), static_cast<float>(b2), bc1,
                                                               bc2, 1e-8f);
  cast_weights_kernel<<<32, 256, 0, x.st>>>(net->d_params, net->d_w0, net->d_w1, net->d_w2);
  net->launches += 2;
  GNN_CUDA(net, cudaGetLastError());
  return ISING_OK;
}

int upload_params(ising_gnn* net, const float* params, cudaStream_t st) {
  for (int i = 0; i < kNumParams; ++i)
    if (!std::isfinite(params[i])) return ISING_EINVAL;
  GNN_CUDA(net, cudaMemcpyAsync(net->d_params, params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, st));
  cast_weights_kernel<<<32, 256, 0, st>>>(net->d_params, net->d_w0, net->d_w1, net->d_w2);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  GNN_CUDA(net, cudaStreamSynchronize(st));
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_gnn_create(const float* params, ising_gnn** out) {
  if (out == nullptr || params == nullptr) return ISING_EINVAL;
  *out = nullptr;
  ising_gnn* net = new (std::nothrow) ising_gnn();
  if (net == nullptr) return ISING_ENOMEM;
  if (cudaGetDevice(&net->device) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return ISING_ECUDA;
  }
  cudaError_t e = cudaSuccess;
  do {
    if ((e = dalloc(&net->d_params, kNumParams)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_m, kNumParams)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_v, kNumParams)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_grad, kNumParams)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_w0, 2 * kF * kH)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_w1, 2 * kH * kH)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_w2, 2 * kH * kH)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_loss, 1)) != cudaSuccess) break;
    if ((e = dalloc(&net->d_err, 1)) != cudaSuccess) break;
    if ((e = cudaMemset(net->d_err, 0, sizeof(int))) != cudaSuccess) break;
    if ((e = cudaMemset(net->d_m, 0, sizeof(float) * kNumParams)) != cudaSuccess) break;
    if ((e = cudaMemset(net->d_v, 0, sizeof(float) * kNumParams)) != cudaSuccess) break;
  } while (0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_net(net);
    delete net;
    return e == cudaErrorMemoryAllocation ? ISING_ENOMEM : ISING_ECUDA;
  }
  const int rc = upload_params(net, params, nullptr);
  if (rc != ISING_OK) {
    free_net(net);
    delete net;
    return rc;
  }
  *out = net;
  return ISING_OK;
}

int ising_gnn_set_params(ising_gnn* net, const float* params) {
  if (net == nullptr || params == nullptr) return ISING_EINVAL;
  if (net->status != ISING_OK) return net->status;
  if (cudaSetDevice(net->device) != cudaSuccess) return net_fail(net);
  GNN_CUDA(net, cudaMemset(net->d_m, 0, sizeof(float) * kNumParams));
  GNN_CUDA(net, cudaMemset(net->d_v, 0, sizeof(float) * kNumParams));
  net->step = 0;
  return upload_params(net, params, nullptr);
}

int ising_gnn_get_params(ising_gnn* net, float* out) {
  if (net == nullptr || out == nullptr) return ISING_EINVAL;
  if (net->status != ISING_OK) return net->status;
  if (cudaSetDevice(net->device) != cudaSuccess) return net_fail(net);
  GNN_CUDA(net, cudaDeviceSynchronize());
  GNN_CUDA(net, cudaMemcpy(out, net->d_params, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
  return ISING_OK;
}

int ising_gnn_forward(ising_gnn* net, ising_graph* g, float* out_logits, int on_device) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  if (out_logits == nullptr) return ISING_EINVAL;
  Ctx x;
  rc = graph_ctx(net, g, &x);
  if (rc != ISING_OK) return rc;
  return forward_out(net, x, out_logits, on_device);
}

int ising_gnn_batch_forward(ising_gnn* net, ising_batch* b, uint32_t replica, float* out_logits,
                            int on_device) {
  if (out_logits == nullptr) return ISING_EINVAL;
  Ctx x;
  isingx::BatchUnion u;
  const int rc = batch_ctx(net, b, replica, &x, &u);
  if (rc != ISING_OK) return rc;
  return forward_out(net, x, out_logits, on_device);
}

int ising_gnn_batch_warm_start(ising_gnn* net, ising_batch* b, uint32_t replica) {
  isingx::BatchUnion u;
  Ctx x;
  int rc = batch_ctx(net, b, 0, &x, &u);
  if (rc != ISING_OK) return rc;
  uint32_t r0 = replica, r1 = replica + 1;
  if (replica == ISING_ALL_REPLICAS) {
    r0 = 0;
    r1 = static_cast<uint32_t>(u.replicas);
  } else if (replica >= static_cast<uint32_t>(u.replicas)) {
    return ISING_EINVAL;
  }
  for (uint32_t r = r0; r < r1; ++r) {
    x.v.shift = static_cast<int>(r);
    rc = run_forward(net, x, false);
    if (rc != ISING_OK) return rc;
    batch_warm_start_kernel<<<grid_of(x.v.n, 256, x.sms * 8), 256, 0, x.st>>>(net->d_z, x.v.n, u.spins,
                                                                               static_cast<int>(r));
    net->launches++;
    GNN_CUDA(net, cudaGetLastError());
  }
  return ISING_OK;
}

int ising_gnn_gradients(ising_gnn* net, ising_graph* g, const int8_t* labels, int labels_on_device,
                        float* out_loss, float* out_grad) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  Ctx x;
  rc = graph_ctx(net, g, &x);
  if (rc != ISING_OK) return rc;
  rc = gradients_impl(net, x, labels, labels_on_device);
  if (rc != ISING_OK) return rc;
  return gradients_out(net, x, out_loss, out_grad);
}

int ising_gnn_train_step(ising_gnn* net, ising_graph* g, const int8_t* labels, int labels_on_device,
                         float lr, float* out_loss) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  if (!(lr >= 0.0f) || !std::isfinite(lr)) return ISING_EINVAL;
  Ctx x;
  rc = graph_ctx(net, g, &x);
  if (rc != ISING_OK) return rc;
  rc = gradients_impl(net, x, labels, labels_on_device);
  if (rc != ISING_OK) return rc;
  rc = adam_step(net, x, lr);
  if (rc != ISING_OK) return rc;
  return gradients_out(net, x, out_loss, nullptr);
}

int ising_gnn_batch_gradients(ising_gnn* net, ising_batch* b, uint32_t replica, const int8_t* labels,
                              int labels_on_device, float* out_loss, float* out_grad) {
  Ctx x;
  isingx::BatchUnion u;
  int rc = batch_ctx(net, b, replica, &x, &u);
  if (rc != ISING_OK) return rc;
  rc = gradients_impl(net, x, labels, labels_on_device);
  if (rc != ISING_OK) return rc;
  return gradients_out(net, x, out_loss, out_grad);
}

int ising_gnn_batch_train_step(ising_gnn* net, ising_batch* b, uint32_t replica, const int8_t* labels,
                               int labels_on_device, float lr, float* out_loss) {
  if (!(lr >= 0.0f) || !std::isfinite(lr)) return ISING_EINVAL;
  Ctx x;
  isingx::BatchUnion u;
  int rc = batch_ctx(net, b, replica, &x, &u);
  if (rc != ISING_OK) return rc;
  rc = gradients_impl(net, x, labels, labels_on_device);
  if (rc != ISING_OK) return rc;
  rc = adam_step(net, x, lr);
  if (rc != ISING_OK) return rc;
  return gradients_out(net, x, out_loss, nullptr);
}

int ising_gnn_warm_start(ising_gnn* net, ising_graph* g, int set_bias) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  Ctx x;
  rc = graph_ctx(net, g, &x);
  if (rc != ISING_OK) return rc;
  rc = run_forward(net, x, false);
  if (rc != ISING_OK) return rc;
  if (set_bias && g->d_bias == nullptr) {
    if (cudaMalloc(&g->d_bias, static_cast<size_t>(g->n)) != cudaSuccess) {
      g->d_bias = nullptr;
      return net_fail(net);
    }
  }
  warm_start_kernel<<<grid_of(g->n, 256, g->num_sms * 8), 256, 0, g->stream>>>(
      net->d_z, g->n, g->d_spins, set_bias ? g->d_bias : nullptr);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  g->parity = 0;
  return ISING_OK;
}

int ising_gnn_set_dense_path(ising_gnn* net, int path) {
  if (net == nullptr) return ISING_EINVAL;
  if (path != ISING_GNN_DENSE_TCGEN05 && path != ISING_GNN_DENSE_MMA_SYNC) return ISING_EINVAL;
  net->dense_path = path;
  return ISING_OK;
}

int ising_gnn_launch_count(ising_gnn* net, uint64_t* out) {
  if (net == nullptr || out == nullptr) return ISING_EINVAL;
  *out = net->launches;
  return ISING_OK;
}

void ising_gnn_destroy(ising_gnn* net) {
  if (net == nullptr) return;
  cudaSetDevice(net->device);
  cudaDeviceSynchronize();
  free_net(net);
  delete net;
}

int ising_set_flip_bias(ising_graph* g, const uint8_t* q, int on_device) {
  int rc = isingx::graph_enter(g);
  if (rc != ISING_OK) return rc;
  if (q == nullptr) {
    if (g->d_bias != nullptr) {
      if (cudaStreamSynchronize(g->stream) != cudaSuccess) return isingx::graph_cuda_fail(g, cudaErrorUnknown);
      cudaFree(g->d_bias);
      g->d_bias = nullptr;
    }
    return ISING_OK;
  }
  const size_t n = static_cast<size_t>(g->n);
  if (g->d_bias == nullptr && cudaMalloc(&g->d_bias, n) != cudaSuccess) {
    g->d_bias = nullptr;
    return isingx::graph_cuda_fail(g, cudaErrorMemoryAllocation);
  }
  const uint8_t* src = q;
  if (!on_device) {
    if (cudaMemcpyAsync(g->d_tmp, q, n, cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
      return isingx::graph_cuda_fail(g, cudaErrorUnknown);
    src = reinterpret_cast<const uint8_t*>(g->d_tmp);
  }
  scatter_bias_kernel<<<grid_of(g->n, 256, g->num_sms * 8), 256, 0, g->stream>>>(src, g->d_pos, g->n, g->d_bias);
  g->launches++;
  if (cudaGetLastError() != cudaSuccess) return isingx::graph_cuda_fail(g, cudaErrorUnknown);
  if (!on_device && cudaStreamSynchronize(g->stream) != cudaSuccess)
    return isingx::graph_cuda_fail(g, cudaErrorUnknown);
  return ISING_OK;
}

int ising_get_flip_bias(ising_graph* g, uint8_t* out) {
  int rc = isingx::graph_enter(g);
  if (rc != ISING_OK) return rc;
  if (out == nullptr) return ISING_EINVAL;
  if (g->d_bias == nullptr) return ISING_ESTATE;
  gather_bias_kernel<<<grid_of(g->n, 256, g->num_sms * 8), 256, 0, g->stream>>>(
      g->d_bias, g->d_orig, g->n, reinterpret_cast<uint8_t*>(g->d_tmp));
  g->launches++;
  if (cudaGetLastError() != cudaSuccess) return isingx::graph_cuda_fail(g, cudaErrorUnknown);
  if (cudaMemcpyAsync(out, g->d_tmp, static_cast<size_t>(g->n), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
      cudaStreamSynchronize(g->stream) != cudaSuccess)
    return isingx::graph_cuda_fail(g, cudaErrorUnknown);
  return ISING_OK;
}

}  // extern "C"
