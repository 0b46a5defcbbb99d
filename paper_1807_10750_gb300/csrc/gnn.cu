// Warm-start graph network (a project addition; the paper has no learned
// part). Three message-passing layers of width 64 read the annealer's spins
// and local fields (Eq. 2) and predict, per vertex, the spin a longer anneal
// ends in; the prediction seeds the spins (warm start) and scales the
// Algorithm 2 flip threshold per vertex (flip bias). The network is defined
// in include/ising.h (G1-G6); this file holds its inference and training
// kernels and their part of the C ABI.
//
// Data path, all by graph position (colour order) on the graph's stream:
//   rowsum:    per-row sums of |w|, 1, w and w * s_j over the CSR entries,
//              lanes over entries, segmented warp sums, int atomics at row
//              ends (exact).
//   features:  x (n x 8 bf16) and c = (d + 1)^-1/2 (G1, G2).
//   aggregate: a = A_hat h, split by CSR entries (not rows), so a hub row of
//              10k entries spreads over many warps: width 8 keeps one entry
//              per lane with a segmented warp sum, width 64 one entry per
//              warp step with two features per lane; fp32 atomics at row
//              ends into a zeroed (forward) or pre-filled (backward) buffer.
//   mlp:       u = [h, a] W + b, relu, on tensor cores (mma.sync m16n8k16,
//              bf16 operands from padded shared-memory tiles via ldmatrix,
//              fp32 accumulation); 64-row tiles, four warps per block.
//   head:      z = h3 w_o + b_o per row (fp32), with the loss G4 and its
//              gradient when labels are given.
//   backward:  per layer one kernel forms dU = dh * (h' > 0), dX = dU W^T
//              (tensor cores) and dW += X^T dU (tensor cores, partial sums
//              in registers, fp32 atomics per block), db in fp32.
//   adam:      fp32 master weights, moments, and the bf16 copies the mma
//              kernels read.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ising.h"
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

constexpr int kTileRows = 64;     // rows per mma tile
constexpr int kMlpThreads = 128;  // four warps, 16 rows each
constexpr int kAggChunk = 256;    // CSR entries per warp in the width-64 aggregation

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
__global__ void rowsum_kernel(EdgeView ev, const int32_t* rowid, const int8_t* spins, int nnz,
                              int4* sums) {
  const int lane = threadIdx.x & 31;
  const long long nw = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  for (long long base = ((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32;
       base < nnz; base += nw * 32) {
    const long long e = base + lane;
    int row = -1, a = 0, c = 0, ws = 0, f = 0;
    if (e < nnz) {
      int col, w;
      edge_at(ev, static_cast<int>(e), col, w);
      row = __ldg(rowid + e);
      a = w < 0 ? -w : w;
      c = 1;
      ws = w;
      f = w * spin_at(spins, col);
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
__global__ void features_kernel(const int4* sums, const int8_t* spins, int n, uint4* x, float* cvec) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int4 q = sums[v];
    const float s = static_cast<float>(spin_at(spins, v));
    const float d1 = static_cast<float>(q.x) + 1.0f;
    const float c2 = 1.0f / d1;
    const float f = static_cast<float>(q.w);
    cvec[v] = 1.0f / sqrtf(d1);
    bf162 p0 = __floats2bfloat162_rn(s, f * c2);
    bf162 p1 = __floats2bfloat162_rn(s * f * c2, log1pf(static_cast<float>(q.y)) * 0.125f);
    bf162 p2 = __floats2bfloat162_rn(static_cast<float>(q.z) * c2, 1.0f);
    bf162 p3 = __floats2bfloat162_rn(0.0f, 0.0f);
    uint4 out;
    memcpy(&out.x, &p0, 4);
    memcpy(&out.y, &p1, 4);
    memcpy(&out.z, &p2, 4);
    memcpy(&out.w, &p3, 4);
    x[v] = out;
  }
}

// out[row] += c_row * sum_j w_rj c_j h_j for width-8 rows (one entry per lane).
__global__ void aggregate8_kernel(EdgeView ev, const int32_t* rowid, const float* cvec,
                                  const uint4* h, int nnz, float* out) {
  const int lane = threadIdx.x & 31;
  const long long nw = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  for (long long base = ((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32;
       base < nnz; base += nw * 32) {
    const long long e = base + lane;
    int row = -1;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.0f;
    if (e < nnz) {
      int col, w;
      edge_at(ev, static_cast<int>(e), col, w);
      row = __ldg(rowid + e);
      const float coef = static_cast<float>(w) * __ldg(cvec + col);
      const uint4 raw = __ldg(h + col);
      const uint32_t words[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bf162 p;
        memcpy(&p, &words[k], 4);
        const float2 f2 = __bfloat1622float2(p);
        v[2 * k] = coef * f2.x;
        v[2 * k + 1] = coef * f2.y;
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = seg_sum(v[k], row, lane);
    if (seg_tail(row, lane)) {
      const float cr = __ldg(cvec + row);
#pragma unroll
      for (int k = 0; k < 8; ++k) atomicAdd(out + static_cast<size_t>(row) * 8 + k, cr * v[k]);
    }
  }
}

// out[row] += c_row * sum_j w_rj c_j h_j for width-64 rows. A warp walks
// kAggChunk consecutive CSR entries, 32 at a time: each lane decodes one
// entry (row, column, w c_col) into a per-warp shared buffer, then the two
// half-warps take alternate entries -- lane l of a half owns features
// 4(l mod 16) .. +3 and loads them with one 8-byte read -- four entries in
// flight per half. Rows are sorted, so each half flushes its running sum with
// one vector atomic where its row changes.
__device__ __forceinline__ void agg_flush(float* out, const float* cvec, int row, int hl,
                                          float4 acc) {
  if (row < 0) return;
  const float cr = __ldg(cvec + row);
  atomicAdd(reinterpret_cast<float4*>(out + static_cast<size_t>(row) * 64 + 4 * hl),
            make_float4(cr * acc.x, cr * acc.y, cr * acc.z, cr * acc.w));
}

__global__ void __launch_bounds__(256)
    aggregate64_kernel(EdgeView ev, const int32_t* rowid, const float* cvec, const bf162* h,
                       int nnz, float* out) {
  __shared__ int4 meta[8][32];  // per warp of the 256-thread block
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int half = lane >> 4, hl = lane & 15;
  const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const long long e_begin = warp * kAggChunk;
  if (e_begin >= nnz) return;
  const long long e_end = e_begin + kAggChunk < nnz ? e_begin + kAggChunk : nnz;
  const uint2* hq = reinterpret_cast<const uint2*>(h);  // 4 bf16 per uint2, 16 per row
  int cur = -1;
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (long long b = e_begin; b < e_end; b += 32) {
    const long long e = b + lane;
    int4 m = make_int4(-1, 0, 0, 0);
    if (e < e_end) {
      int col, w;
      edge_at(ev, static_cast<int>(e), col, w);
      m.x = __ldg(rowid + e);
      m.y = col;
      m.z = __float_as_int(static_cast<float>(w) * __ldg(cvec + col));
    }
    meta[wib][lane] = m;
    __syncwarp();
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 8) {
      int4 mm[4];
      uint2 hv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        mm[u] = meta[wib][j0 + 2 * u + half];
        hv[u] = mm[u].x >= 0 ? hq[static_cast<size_t>(mm[u].y) * 16 + hl] : make_uint2(0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (mm[u].x < 0) continue;  // past the chunk's end
        if (mm[u].x != cur) {
          agg_flush(out, cvec, cur, hl, acc);
          acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          cur = mm[u].x;
        }
        const float coef = __int_as_float(mm[u].z);
        bf162 p0, p1;
        memcpy(&p0, &hv[u].x, 4);
        memcpy(&p1, &hv[u].y, 4);
        const float2 f0 = __bfloat1622float2(p0), f1 = __bfloat1622float2(p1);
        acc.x += coef * f0.x;
        acc.y += coef * f0.y;
        acc.z += coef * f1.x;
        acc.w += coef * f1.y;
      }
    }
    __syncwarp();
  }
  agg_flush(out, cvec, cur, hl, acc);
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

// Stage rows [r0, r0 + 64) of X = [h, a] (bf16 h, fp32 a rounded to bf16)
// into sX (row stride KP elements); rows past n read as zero.
template <int D, int KP>
__device__ __forceinline__ void stage_x(bf16* sX, const bf16* h, const float* a, int r0, int n) {
  constexpr int HC = D / 8;      // 16-byte chunks of an h row
  constexpr int CH = 2 * HC;     // chunks of an X row
  for (int idx = threadIdx.x; idx < kTileRows * CH; idx += blockDim.x) {
    const int r = idx / CH, ch = idx % CH;
    const int row = r0 + r;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (row < n) {
      if (ch < HC) {
        val = *reinterpret_cast<const uint4*>(h + static_cast<size_t>(row) * D + ch * 8);
      } else {
        const float4* src = reinterpret_cast<const float4*>(a + static_cast<size_t>(row) * D + (ch - HC) * 8);
        const float4 f0 = src[0], f1 = src[1];
        val.x = pack_bf162(f0.x, f0.y);
        val.y = pack_bf162(f0.z, f0.w);
        val.z = pack_bf162(f1.x, f1.y);
        val.w = pack_bf162(f1.z, f1.w);
      }
    }
    *reinterpret_cast<uint4*>(sX + r * KP + ch * 8) = val;
  }
}

// Forward layer: hout = relu([h, a] W + b), W [2D][64] bf16 row-major.
template <int D>
__global__ void __launch_bounds__(kMlpThreads)
    mlp_fwd_kernel(const bf16* __restrict__ h, const float* __restrict__ a,
                   const bf16* __restrict__ W, const float* __restrict__ bias, int n,
                   bf16* __restrict__ hout) {
  constexpr int K = 2 * D, KP = K + 8, NP = kH + 8;
  __shared__ __align__(16) bf16 sW[K * NP];
  __shared__ __align__(16) bf16 sX[kTileRows * KP];
  __shared__ float sB[kH];
  for (int idx = threadIdx.x; idx < K * (kH / 8); idx += blockDim.x) {
    const int k = idx / (kH / 8), c = idx % (kH / 8);
    *reinterpret_cast<uint4*>(sW + k * NP + c * 8) = *reinterpret_cast<const uint4*>(W + k * kH + c * 8);
  }
  if (threadIdx.x < kH) sB[threadIdx.x] = bias[threadIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int tile = blockIdx.x; tile * kTileRows < n; tile += gridDim.x) {
    __syncthreads();
    stage_x<D, KP>(sX, h, a, tile * kTileRows, n);
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      uint32_t af[4];
      ldsm_x4(af, sX + (16 * wid + (lane & 7) + ((lane >> 3) & 1) * 8) * KP + ks * 16 + (lane >> 4) * 8);
#pragma unroll
      for (int np = 0; np < 4; ++np) {
        uint32_t bfr[4];
        ldsm_x4_t(bfr, sW + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * NP + np * 16 + (lane >> 4) * 8);
        mma_bf16(acc[2 * np], af, bfr[0], bfr[1]);
        mma_bf16(acc[2 * np + 1], af, bfr[2], bfr[3]);
      }
    }
    const int r0 = tile * kTileRows + 16 * wid + g;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + 2 * t;
      const float b0 = sB[col], b1 = sB[col + 1];
      if (r0 < n)
        *reinterpret_cast<uint32_t*>(hout + static_cast<size_t>(r0) * kH + col) =
            pack_bf162(fmaxf(acc[nt][0] + b0, 0.0f), fmaxf(acc[nt][1] + b1, 0.0f));
      if (r0 + 8 < n)
        *reinterpret_cast<uint32_t*>(hout + static_cast<size_t>(r0 + 8) * kH + col) =
            pack_bf162(fmaxf(acc[nt][2] + b0, 0.0f), fmaxf(acc[nt][3] + b1, 0.0f));
    }
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

// Backward of one layer (h' = relu([h, a] W + b)) given dh' = dL/dh':
// dU = dh' * (h' > 0); gW += X^T dU; gb += colsum dU; with DX also
// dX = dU W^T, split into dh (fp32, the direct part) and da (bf16, to be
// propagated through A_hat by the caller).
template <int D, bool DX>
__global__ void __launch_bounds__(kMlpThreads)
    mlp_bwd_kernel(const float* __restrict__ dhn, const bf16* __restrict__ hn,
                   const bf16* __restrict__ h, const float* __restrict__ a,
                   const bf16* __restrict__ W, int n, float* __restrict__ gW,
                   float* __restrict__ gb, float* __restrict__ dh, bf16* __restrict__ da) {
  constexpr int K2 = 2 * D, KP = K2 + 8, NP = kH + 8;
  constexpr int MT = K2 / 16;              // 16-row tiles of gW
  constexpr int TPW = MT * 8 / 4;          // gW 16x8 tiles per warp
  constexpr int WR = DX ? K2 : 1;
  __shared__ __align__(16) bf16 sW[WR * NP];
  __shared__ __align__(16) bf16 sX[kTileRows * KP];
  __shared__ __align__(16) bf16 sU[kTileRows * NP];
  __shared__ float sdb[kH];
  if (DX) {
    for (int idx = threadIdx.x; idx < K2 * (kH / 8); idx += blockDim.x) {
      const int k = idx / (kH / 8), c = idx % (kH / 8);
      *reinterpret_cast<uint4*>(sW + k * NP + c * 8) = *reinterpret_cast<const uint4*>(W + k * kH + c * 8);
    }
  }
  if (threadIdx.x < kH) sdb[threadIdx.x] = 0.0f;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float accW[TPW][4];
#pragma unroll
  for (int i = 0; i < TPW; ++i) accW[i][0] = accW[i][1] = accW[i][2] = accW[i][3] = 0.0f;
  float dbp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const int c4 = (threadIdx.x & 15) * 4;  // this thread's four columns of dU
  for (int tile = blockIdx.x; tile * kTileRows < n; tile += gridDim.x) {
    const int r0 = tile * kTileRows;
    __syncthreads();
    for (int r = threadIdx.x >> 4; r < kTileRows; r += kMlpThreads / 16) {
      const int row = r0 + r;
      float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (row < n) {
        const float4 d4 = *reinterpret_cast<const float4*>(dhn + static_cast<size_t>(row) * kH + c4);
        const uint2 hraw = *reinterpret_cast<const uint2*>(hn + static_cast<size_t>(row) * kH + c4);
        bf162 p0, p1;
        memcpy(&p0, &hraw.x, 4);
        memcpy(&p1, &hraw.y, 4);
        const float2 h0 = __bfloat1622float2(p0), h1 = __bfloat1622float2(p1);
        u[0] = h0.x > 0.0f ? d4.x : 0.0f;
        u[1] = h0.y > 0.0f ? d4.y : 0.0f;
        u[2] = h1.x > 0.0f ? d4.z : 0.0f;
        u[3] = h1.y > 0.0f ? d4.w : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) dbp[i] += u[i];
      uint2 packed;
      packed.x = pack_bf162(u[0], u[1]);
      packed.y = pack_bf162(u[2], u[3]);
      *reinterpret_cast<uint2*>(sU + r * NP + c4) = packed;
    }
    stage_x<D, KP>(sX, h, a, r0, n);
    __syncthreads();
    if (DX) {
      float acc[K2 / 8][4];
#pragma unroll
      for (int i = 0; i < K2 / 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < kH / 16; ++ks) {
        uint32_t af[4];
        ldsm_x4(af, sU + (16 * wid + (lane & 7) + ((lane >> 3) & 1) * 8) * NP + ks * 16 + (lane >> 4) * 8);
#pragma unroll
        for (int np = 0; np < K2 / 16; ++np) {
          uint32_t bfr[4];
          // B[k][m] = W[m][k]: W rows are B's columns, so no transpose
          ldsm_x4(bfr, sW + (np * 16 + (lane & 7) + (lane >> 4) * 8) * NP + ks * 16 + ((lane >> 3) & 1) * 8);
          mma_bf16(acc[2 * np], af, bfr[0], bfr[1]);
          mma_bf16(acc[2 * np + 1], af, bfr[2], bfr[3]);
        }
      }
      const int rr = r0 + 16 * wid + g;
#pragma unroll
      for (int nt = 0; nt < K2 / 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        if (col < D) {
          if (rr < n)
            *reinterpret_cast<float2*>(dh + static_cast<size_t>(rr) * D + col) = make_float2(acc[nt][0], acc[nt][1]);
          if (rr + 8 < n)
            *reinterpret_cast<float2*>(dh + static_cast<size_t>(rr + 8) * D + col) = make_float2(acc[nt][2], acc[nt][3]);
        } else {
          if (rr < n)
            *reinterpret_cast<uint32_t*>(da + static_cast<size_t>(rr) * D + col - D) = pack_bf162(acc[nt][0], acc[nt][1]);
          if (rr + 8 < n)
            *reinterpret_cast<uint32_t*>(da + static_cast<size_t>(rr + 8) * D + col - D) = pack_bf162(acc[nt][2], acc[nt][3]);
        }
      }
    }
    // gW[m][j] += sum_rows X[row][m] dU[row][j]: A = X^T, B = dU (both via
    // transposing loads of the row-major tiles)
#pragma unroll
    for (int ks = 0; ks < kTileRows / 16; ++ks) {
#pragma unroll
      for (int i = 0; i < TPW; ++i) {
        const int tile_id = wid * TPW + i;
        const int mt = tile_id / 8, nt = tile_id % 8;
        uint32_t af[4], bfr[4];
        ldsm_x4_t(af, sX + (ks * 16 + (lane & 7) + (lane >> 4) * 8) * KP + mt * 16 + ((lane >> 3) & 1) * 8);
        ldsm_x4_t(bfr, sU + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * NP + nt * 8);
        mma_bf16(accW[i], af, bfr[0], bfr[1]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < TPW; ++i) {
    const int tile_id = wid * TPW + i;
    const int mt = tile_id / 8, nt = tile_id % 8;
    const int m = mt * 16 + g, j = nt * 8 + 2 * t;
    atomicAdd(gW + m * kH + j, accW[i][0]);
    atomicAdd(gW + m * kH + j + 1, accW[i][1]);
    atomicAdd(gW + (m + 8) * kH + j, accW[i][2]);
    atomicAdd(gW + (m + 8) * kH + j + 1, accW[i][3]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) atomicAdd(&sdb[c4 + i], dbp[i]);
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

__global__ void gather_labels_kernel(const int8_t* caller, const int32_t* orig, int n, int8_t* pos_out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    pos_out[v] = caller[orig[v]];
}

__global__ void scatter_logits_kernel(const float* z, const int32_t* orig, int n, float* caller) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    caller[orig[v]] = z[v];
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
  float* d_a0 = nullptr;
  bf16* d_h[3] = {nullptr, nullptr, nullptr};  // h1, h2, h3
  float* d_a[2] = {nullptr, nullptr};          // a1, a2
  float* d_z = nullptr;
  int8_t* d_y = nullptr;
  float* d_dh[2] = {nullptr, nullptr};
  bf16* d_da = nullptr;
  float* d_out = nullptr;  // logits in caller order (host copies)
};

namespace {

void free_work(ising_gnn* net) {
  void* ptrs[] = {net->d_sums, net->d_c,     net->d_x,     net->d_a0,    net->d_h[0],
                  net->d_h[1], net->d_h[2],  net->d_a[0],  net->d_a[1],  net->d_z,
                  net->d_y,    net->d_dh[0], net->d_dh[1], net->d_da,    net->d_out};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  net->d_sums = nullptr;
  net->d_c = net->d_a0 = net->d_z = net->d_out = nullptr;
  net->d_x = net->d_da = nullptr;
  net->d_h[0] = net->d_h[1] = net->d_h[2] = nullptr;
  net->d_a[0] = net->d_a[1] = net->d_dh[0] = net->d_dh[1] = nullptr;
  net->d_y = nullptr;
  net->n_cap = 0;
}

void free_net(ising_gnn* net) {
  free_work(net);
  void* ptrs[] = {net->d_params, net->d_m, net->d_v, net->d_grad,
                  net->d_w0,     net->d_w1, net->d_w2, net->d_loss};
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
  }
  if ((e = dalloc(&net->d_z, N)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_y, N)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_da, N * kH)) != cudaSuccess) return e;
  if ((e = dalloc(&net->d_out, N)) != cudaSuccess) return e;
  net->n_cap = n;
  return cudaSuccess;
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

EdgeView edges_of(const ising_graph* g) {
  EdgeView ev;
  ev.adj = g->d_adj;
  ev.col = g->d_col;
  ev.w = g->d_w;
  ev.packed = g->packed ? 1 : 0;
  return ev;
}

// Forward pass over graph g from its current spins; with labels (by
// position in net->d_y) also the loss and dL/dh3 into net->d_dh[0].
int run_forward(ising_gnn* net, ising_graph* g, bool with_labels) {
  const int n = g->n;
  const long long nnz = g->nnz;
  cudaStream_t st = g->stream;
  const int sms = g->num_sms;
  GNN_CUDA(net, ensure_work(net, n));
  if (g->d_rowid == nullptr) {
    if (cudaMalloc(&g->d_rowid, static_cast<size_t>(nnz > 0 ? nnz : 1) * sizeof(int32_t)) != cudaSuccess) {
      g->d_rowid = nullptr;
      return net_fail(net);
    }
    rowid_kernel<<<grid_of(n, 256, sms * 8), 256, 0, st>>>(g->d_row_ptr, n, g->d_rowid);
    net->launches++;
    GNN_CUDA(net, cudaGetLastError());
  }
  const EdgeView ev = edges_of(g);
  const int ent_grid = grid_of((nnz + 31) / 32 * 32, 256, sms * 16);
  GNN_CUDA(net, cudaMemsetAsync(net->d_sums, 0, sizeof(int4) * static_cast<size_t>(n), st));
  if (nnz > 0) {
    rowsum_kernel<<<ent_grid, 256, 0, st>>>(ev, g->d_rowid, g->d_spins, static_cast<int>(nnz), net->d_sums);
    net->launches++;
  }
  features_kernel<<<grid_of(n, 256, sms * 8), 256, 0, st>>>(net->d_sums, g->d_spins, n,
                                                             reinterpret_cast<uint4*>(net->d_x), net->d_c);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  // about 36 KB of shared memory per block: six blocks fit on an SM
  const int mlp_grid = grid_of((n + kTileRows - 1) / kTileRows, 1, sms * 6);
  // layer 0
  GNN_CUDA(net, cudaMemsetAsync(net->d_a0, 0, sizeof(float) * static_cast<size_t>(n) * kF, st));
  if (nnz > 0) {
    aggregate8_kernel<<<ent_grid, 256, 0, st>>>(ev, g->d_rowid, net->d_c,
                                                reinterpret_cast<const uint4*>(net->d_x),
                                                static_cast<int>(nnz), net->d_a0);
    net->launches++;
  }
  mlp_fwd_kernel<kF><<<mlp_grid, kMlpThreads, 0, st>>>(net->d_x, net->d_a0, net->d_w0,
                                                       net->d_params + kOffB0, n, net->d_h[0]);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  // layers 1 and 2
  const long long agg_warps = (nnz + kAggChunk - 1) / kAggChunk;
  const int agg_grid = static_cast<int>((agg_warps + 7) / 8);
  for (int l = 1; l <= 2; ++l) {
    GNN_CUDA(net, cudaMemsetAsync(net->d_a[l - 1], 0, sizeof(float) * static_cast<size_t>(n) * kH, st));
    if (nnz > 0) {
      aggregate64_kernel<<<agg_grid, 256, 0, st>>>(ev, g->d_rowid, net->d_c,
                                                   reinterpret_cast<const bf162*>(net->d_h[l - 1]),
                                                   static_cast<int>(nnz), net->d_a[l - 1]);
      net->launches++;
    }
    mlp_fwd_kernel<kH><<<mlp_grid, kMlpThreads, 0, st>>>(
        net->d_h[l - 1], net->d_a[l - 1], l == 1 ? net->d_w1 : net->d_w2,
        net->d_params + (l == 1 ? kOffB1 : kOffB2), n, net->d_h[l]);
    net->launches++;
    GNN_CUDA(net, cudaGetLastError());
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
int run_backward(ising_gnn* net, ising_graph* g) {
  const int n = g->n;
  const long long nnz = g->nnz;
  cudaStream_t st = g->stream;
  const int sms = g->num_sms;
  const EdgeView ev = edges_of(g);
  const int mlp_grid = grid_of((n + kTileRows - 1) / kTileRows, 1, sms * 2);
  const long long agg_warps = (nnz + kAggChunk - 1) / kAggChunk;
  const int agg_grid = static_cast<int>((agg_warps + 7) / 8);
  // d_dh[0] holds dL/dh3; layers 2 and 1 produce dL/dh2, dL/dh1 alternately
  int cur = 0;
  for (int l = 2; l >= 1; --l) {
    const int nxt = cur ^ 1;
    const bf16* W = l == 2 ? net->d_w2 : net->d_w1;
    float* gW = net->d_grad + (l == 2 ? kOffW2 : kOffW1);
    float* gb = net->d_grad + (l == 2 ? kOffB2 : kOffB1);
    mlp_bwd_kernel<kH, true><<<mlp_grid, kMlpThreads, 0, st>>>(
        net->d_dh[cur], net->d_h[l], net->d_h[l - 1], net->d_a[l - 1], W, n, gW, gb, net->d_dh[nxt],
        net->d_da);
    net->launches++;
    GNN_CUDA(net, cudaGetLastError());
    if (nnz > 0) {
      aggregate64_kernel<<<agg_grid, 256, 0, st>>>(ev, g->d_rowid, net->d_c,
                                                   reinterpret_cast<const bf162*>(net->d_da),
                                                   static_cast<int>(nnz), net->d_dh[nxt]);
      net->launches++;
      GNN_CUDA(net, cudaGetLastError());
    }
    cur = nxt;
  }
  mlp_bwd_kernel<kF, false><<<mlp_grid, kMlpThreads, 0, st>>>(
      net->d_dh[cur], net->d_h[0], net->d_x, net->d_a0, net->d_w0, n, net->d_grad + kOffW0,
      net->d_grad + kOffB0, nullptr, nullptr);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  return ISING_OK;
}

int load_labels(ising_gnn* net, ising_graph* g, const int8_t* labels, int on_device) {
  const int n = g->n;
  const int8_t* src = labels;
  if (!on_device) {
    for (int i = 0; i < n; ++i)
      if (labels[i] != 1 && labels[i] != -1) return ISING_EINVAL;
    GNN_CUDA(net, cudaMemcpyAsync(net->d_out, labels, static_cast<size_t>(n), cudaMemcpyHostToDevice, g->stream));
    src = reinterpret_cast<const int8_t*>(net->d_out);
  }
  gather_labels_kernel<<<grid_of(n, 256, g->num_sms * 8), 256, 0, g->stream>>>(src, g->d_orig, n, net->d_y);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  if (!on_device) GNN_CUDA(net, cudaStreamSynchronize(g->stream));
  return ISING_OK;
}

int gradients_impl(ising_gnn* net, ising_graph* g, const int8_t* labels, int on_device) {
  if (labels == nullptr) return ISING_EINVAL;
  GNN_CUDA(net, ensure_work(net, g->n));
  int rc = load_labels(net, g, labels, on_device);
  if (rc != ISING_OK) return rc;
  GNN_CUDA(net, cudaMemsetAsync(net->d_grad, 0, sizeof(float) * kNumParams, g->stream));
  rc = run_forward(net, g, true);
  if (rc != ISING_OK) return rc;
  return run_backward(net, g);
}

int read_loss(ising_gnn* net, ising_graph* g, float* out_loss) {
  double l = 0.0;
  GNN_CUDA(net, cudaMemcpyAsync(&l, net->d_loss, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  GNN_CUDA(net, cudaStreamSynchronize(g->stream));
  *out_loss = static_cast<float>(l / static_cast<double>(g->n));
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
  rc = run_forward(net, g, false);
  if (rc != ISING_OK) return rc;
  float* dst = on_device ? out_logits : net->d_out;
  scatter_logits_kernel<<<grid_of(g->n, 256, g->num_sms * 8), 256, 0, g->stream>>>(net->d_z, g->d_orig, g->n, dst);
  net->launches++;
  GNN_CUDA(net, cudaGetLastError());
  if (!on_device) {
    GNN_CUDA(net, cudaMemcpyAsync(out_logits, net->d_out, sizeof(float) * static_cast<size_t>(g->n),
                                  cudaMemcpyDeviceToHost, g->stream));
    GNN_CUDA(net, cudaStreamSynchronize(g->stream));
  }
  return ISING_OK;
}

int ising_gnn_gradients(ising_gnn* net, ising_graph* g, const int8_t* labels, int labels_on_device,
                        float* out_loss, float* out_grad) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  rc = gradients_impl(net, g, labels, labels_on_device);
  if (rc != ISING_OK) return rc;
  if (out_grad != nullptr) {
    GNN_CUDA(net, cudaMemcpyAsync(out_grad, net->d_grad, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, g->stream));
    GNN_CUDA(net, cudaStreamSynchronize(g->stream));
  }
  if (out_loss != nullptr) return read_loss(net, g, out_loss);
  return ISING_OK;
}

int ising_gnn_train_step(ising_gnn* net, ising_graph* g, const int8_t* labels, int labels_on_device,
                         float lr, float* out_loss) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  if (!(lr >= 0.0f) || !std::isfinite(lr)) return ISING_EINVAL;
  rc = gradients_impl(net, g, labels, labels_on_device);
  if (rc != ISING_OK) return rc;
  net->step++;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = static_cast<float>(1.0 - std::pow(b1, static_cast<double>(net->step)));
  const float bc2 = static_cast<float>(1.0 - std::pow(b2, static_cast<double>(net->step)));
  adam_kernel<<<grid_of(kNumParams, 256, 128), 256, 0, g->stream>>>(
      net->d_params, net->d_m, net->d_v, net->d_grad, lr, static_cast<float>(b1), static_cast<float>(b2), bc1, bc2,
      1e-8f);
  cast_weights_kernel<<<32, 256, 0, g->stream>>>(net->d_params, net->d_w0, net->d_w1, net->d_w2);
  net->launches += 2;
  GNN_CUDA(net, cudaGetLastError());
  if (out_loss != nullptr) return read_loss(net, g, out_loss);
  return ISING_OK;
}

int ising_gnn_warm_start(ising_gnn* net, ising_graph* g, int set_bias) {
  int rc = net_enter(net, g);
  if (rc != ISING_OK) return rc;
  rc = run_forward(net, g, false);
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
