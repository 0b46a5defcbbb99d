// ising_energy_csr_static: energy and cut of a spin vector on a caller-owned
// CSR graph, without allocating any memory.
//
// Who needs this: callers that cannot call cudaMalloc. Examples are code that
// runs under a memory pool which owns all device memory, code with a fixed
// memory budget, and latency-sensitive loops where cudaMalloc/cudaFree would
// block the host and synchronise the device. The caller passes only its own
// input and output buffers; the reduction's scratch lives in a fixed-size
// device array defined in this file.
//
// The scratch array g_chunk_partials is file-scope device memory. Every GPU
// that loads the library holds it until the process exits. All calls on a
// device share it and it keeps the last call's contents. Each call rewrites
// every partial it reads before reading it, so nothing has to start at zero.
// Calls whose kernels overlap on the GPU (different streams, no ordering
// between them) race on the array and give wrong results; order such calls.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/ising.h"

namespace {

constexpr int kStaticBlock = 256;
constexpr int kRowsPerChunk = 1024;  // one block reduces one chunk of rows
constexpr int kMaxChunks = ISING_STATIC_MAX_VERTICES / kRowsPerChunk;
constexpr int kMaxDevices = 64;

// Per chunk: {sum_i s_i f_i, sum of all directed weights}; both are twice the
// undirected sums.
__device__ __align__(256) long long g_chunk_partials[kMaxChunks][2];

std::mutex g_setup_mutex;
long long (*g_partials_ptr[kMaxDevices])[2] = {};

__global__ void __launch_bounds__(kStaticBlock)
    static_energy_chunks(int32_t n, const int32_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ w,
                         const int8_t* __restrict__ spins, long long (*partials)[2]) {
  const int row0 = blockIdx.x * kRowsPerChunk;
  long long e2 = 0, w2 = 0;
  for (int r = row0 + threadIdx.x; r < min(n, row0 + kRowsPerChunk); r += kStaticBlock) {
    long long f = 0, ws = 0;
    for (int k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
      f += static_cast<long long>(w[k]) * spins[col[k]];
      ws += w[k];
    }
    e2 += spins[r] * f;
    w2 += ws;
  }
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    w2 += __shfl_xor_sync(0xffffffffu, w2, o);
  }
  __shared__ long long se[kStaticBlock / 32], sw[kStaticBlock / 32];
  if ((threadIdx.x & 31) == 0) {
    se[threadIdx.x >> 5] = e2;
    sw[threadIdx.x >> 5] = w2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a = 0, b = 0;
    for (int k = 0; k < kStaticBlock / 32; ++k) {
      a += se[k];
      b += sw[k];
    }
    partials[blockIdx.x][0] = a;
    partials[blockIdx.x][1] = b;
  }
}

__global__ void __launch_bounds__(kStaticBlock)
    static_energy_finish(int chunks, const long long (*partials)[2], int64_t* out) {
  long long e2 = 0, w2 = 0;
  for (int c = threadIdx.x; c < chunks; c += kStaticBlock) {
    e2 += partials[c][0];
    w2 += partials[c][1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    w2 += __shfl_xor_sync(0xffffffffu, w2, o);
  }
  __shared__ long long se[kStaticBlock / 32], sw[kStaticBlock / 32];
  if ((threadIdx.x & 31) == 0) {
    se[threadIdx.x >> 5] = e2;
    sw[threadIdx.x >> 5] = w2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a = 0, b = 0;
    for (int k = 0; k < kStaticBlock / 32; ++k) {
      a += se[k];
      b += sw[k];
    }
    const long long H = a / 2, W = b / 2;
    out[0] = H;
    out[1] = (W - H) / 2;
  }
}

// Device address of the scratch array for the current device, looked up once
// per device (the first call on a device does it) and kept for the life of the
// process. cudaDeviceReset unloads the module and may move the array, so the
// cached address is not valid across a reset of the device.
int partials_for_current_device(long long (**out)[2]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ISING_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return ISING_ERANGE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_partials_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_chunk_partials) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return ISING_ECUDA;
    }
    g_partials_ptr[dev] = static_cast<long long (*)[2]>(p);
  }
  *out = g_partials_ptr[dev];
  return ISING_OK;
}

}  // namespace

extern "C" int ising_energy_csr_static(int32_t n, const int32_t* row_ptr, const int32_t* col,
                                       const int32_t* w, const int8_t* spins, int64_t* out,
                                       void* cuda_stream) {
  if (n <= 0 || row_ptr == nullptr || spins == nullptr || out == nullptr) return ISING_EINVAL;
  // the kernels read col and w only for rows with entries, but a null pointer
  // there is never what the caller meant: an edgeless graph may pass any
  // valid pointer
  if (col == nullptr || w == nullptr) return ISING_EINVAL;
  if (n > ISING_STATIC_MAX_VERTICES) return ISING_ERANGE;
  // an error left pending by earlier, unrelated work is reported and left in
  // place for its owner: nothing is launched behind it
  if (cudaPeekAtLastError() != cudaSuccess) return ISING_ECUDA;
  long long (*partials)[2] = nullptr;
  const int rc = partials_for_current_device(&partials);
  if (rc != ISING_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int chunks = (n + kRowsPerChunk - 1) / kRowsPerChunk;
  static_energy_chunks<<<chunks, kStaticBlock, 0, s>>>(n, row_ptr, col, w, spins, partials);
  if (cudaGetLastError() != cudaSuccess) return ISING_ECUDA;
  static_energy_finish<<<1, kStaticBlock, 0, s>>>(chunks, partials, out);
  if (cudaGetLastError() != cudaSuccess) return ISING_ECUDA;
  return ISING_OK;
}
