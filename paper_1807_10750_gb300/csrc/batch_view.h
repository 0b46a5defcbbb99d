// A batch's instances seen as one graph (their disjoint union), by position,
// for the warm-start network (gnn.cu). Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ising.h"

namespace isingx {

struct BatchUnion {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  int32_t n = 0;       // vertices of all instances
  int64_t nnz = 0;     // CSR entries of all instances
  int32_t replicas = 1;
  const int32_t* row_ptr = nullptr;  // n + 1 absolute offsets into adj
  const int32_t* adj = nullptr;      // packed (col << 8) | (w & 0xff), col local to the instance
  const int32_t* vbase = nullptr;    // per position: first position of its instance
  const int32_t* orig = nullptr;     // per position: vertex id within its instance
  uint8_t* spins = nullptr;          // per position: bit r set when replica r's spin is -1
  // storage the network fills on first use; freed with the batch
  int32_t** rowid = nullptr;
  int32_t** hchunk = nullptr;
  int32_t** chunk_row = nullptr;
  int32_t* num_chunks = nullptr;     // -1 until built
};

// Enter the batch (argument and state check, device made current) and
// describe it; the union's row table is built on the first call.
int batch_union(ising_batch* b, BatchUnion* out);

}  // namespace isingx
