// The graph handle of include/ising.h, shared by the sweep engine
// (anneal.cu) and the warm-start network (gnn.cu). Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <thread>
#include <vector>

#include "../../include/ising.h"
#include "host_graph.h"
#include "sweep.cuh"

struct ising_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  int status = ISING_OK;
  int engine = ISING_ENGINE_AUTO;
  int engine_used = -1;  // the engine the last anneal call ran (ising_engine_used)
  int fault_kind = ISING_FAULT_NONE;  // ising_debug_fault
  uint64_t wait_budget_ns = 0;        // 0: the kernels' default bound
  int num_sms = 1;
  uint64_t launches = 0;

  int32_t n = 0;
  int parity = 0;  // update parity of every state byte (bit 1) between calls
  int64_t num_edges = 0;
  int64_t nnz = 0;
  int64_t total_weight = 0;
  int32_t num_colours = 0;
  bool packed = true;  // packed (col << 8 | w) edges, else split int32 col / w
  std::vector<int32_t> colour;  // by caller id
  std::vector<int32_t> class_item_begin;
  int32_t num_items = 0;
  int32_t num_slots = 0;

  int32_t* d_row_ptr = nullptr;
  int32_t* d_adj = nullptr;  // packed format
  int32_t* d_col = nullptr;  // split format
  int32_t* d_w = nullptr;    // split format
  int32_t* d_ell = nullptr;      // sliced ELL, packed format
  int32_t* d_ell_col = nullptr;  // sliced ELL, split format
  int32_t* d_ell_w = nullptr;    // sliced ELL, split format
  int8_t* d_spins = nullptr;
  int32_t* d_orig = nullptr;
  int32_t* d_pos = nullptr;
  isingx::WorkItem* d_items = nullptr;
  unsigned long long* d_slice_acc = nullptr;
  int32_t* d_slice_parts = nullptr;
  unsigned long long* d_energy = nullptr;
  int32_t* d_flag = nullptr;
  int8_t* d_tmp = nullptr;
  int32_t* d_class_items = nullptr;  // num_colours + 1 item offsets
  int32_t* d_class_begin = nullptr;  // num_colours + 1 first positions
  unsigned long long* d_trace = nullptr;  // energy trace (twice H per checkpoint)
  unsigned* d_nflip_bits = nullptr;        // N-flip: chosen-vertex bitmap (kept zero)
  int32_t* d_nflip_list = nullptr;         // N-flip: chosen vertices, n entries
  size_t trace_cap = 0;
  int32_t* d_all_items = nullptr;    // {0, num_items}: one phase over every item (energy)
  // item-dataflow engine (graphs without sliced rows)
  bool itemflow_ok = false;
  int32_t* d_dep_ptr = nullptr;
  int32_t* d_deps = nullptr;
  int32_t* d_done = nullptr;
  // block engine of small graphs (host_graph.h, block.cuh)
  bool block_ok = false;
  int32_t block_num_chunks = 0;
  int32_t block_num_words = 0;
  int32_t* d_block_words = nullptr;
  int32_t* d_block_chunk_off = nullptr;
  int32_t* d_block_chunk_len = nullptr;
  int32_t* d_block_class_chunk = nullptr;
  // halo engine (halo.cuh): the host graph is kept for its plan when the graph
  // can qualify; a host thread builds the plan while the caller goes on
  // (started by AUTO's second anneal call, or by a call that asks for the
  // engine and waits), and the first call that needs it uploads it
  std::unique_ptr<isingx::HostGraph> host;
  std::unique_ptr<isingx::HaloPlan> pending;  // written by the planner thread
  std::thread planner;
  std::atomic<bool> planned{false};           // the planner has finished `pending`
  std::atomic<bool> plan_cancel{false};       // ising_destroy: stop the planner early
  int halo_state = 0;   // 0 not planned, 1 planned, -1 no plan possible
  int halo_sweeps = 0;  // requested sweeps per exchange (0: automatic)
  uint64_t auto_calls = 0;  // AUTO's deterministic linear anneal calls
  int32_t halo_parts = 0, halo_S = 0, halo_smem = 0;
  double halo_ratio = 0.0;
  int32_t* d_halo_hdr = nullptr;
  int32_t* d_halo_words = nullptr;
  int32_t* d_halo_slices = nullptr;
  int32_t* d_halo_gpos = nullptr;
  int32_t* d_halo_imports = nullptr;
  int32_t* d_halo_nbrs = nullptr;
  int32_t* d_halo_exports = nullptr;
  int32_t* d_halo_quads = nullptr;
  unsigned* d_halo_flags = nullptr;
  int8_t* d_spins2 = nullptr;        // the two mailbox buffers of the halo engine
  size_t halo_mail = 0;              // bytes of one mailbox buffer
  // hub engine (hub.cuh): graphs with 1 .. kHubMaxHubs hubs
  bool hub_ok = false;
  int32_t num_hubs = 0, hub_colours = 0;
  int32_t hub_num_b = 0, hub_num_items = 0;
  int32_t* d_hub_split = nullptr;    // per hub: first CSR entry in a later hub class
  int32_t* d_hub_end = nullptr;      // per hub: first CSR entry past its hub neighbours
  int4* d_hub_sums = nullptr;        // field-sum items
  int32_t* d_hub_acc = nullptr;      // 3 * num_hubs sums (A by sweep parity, B)
  uint32_t* d_hub_flips = nullptr;   // flip bits of the chain's hubs
  uint32_t* d_hub_bits = nullptr;    // the spin map of a launch (n / 32 + 2 words)
  uint32_t* d_hub_pflips = nullptr;  // a sweep's flips by position (n / 32 + 2 words)
  int32_t* d_hub_blk = nullptr;      // non-hub classes' work split over the worker blocks
  int32_t hub_grid = 0;              // blocks the split was made for
  uint8_t* d_bias = nullptr;         // per-position flip bias (null: none)
  int32_t* d_rowid = nullptr;        // row of every CSR entry (built on first use)
  int32_t* d_gnn_hchunk = nullptr;   // warm-start network: per row, its first entry chunk or -1
  int32_t* d_gnn_chunk_row = nullptr;  // warm-start network: the row of every entry chunk
  int32_t gnn_num_chunks = -1;       // -1 until built
  isingx::BarrierState* d_barrier = nullptr;
  int persist_grid = 0;              // co-resident blocks of the persistent kernel

  isingx::DevGraph dev() const {
    isingx::DevGraph d;
    d.pad_col = n;
    d.row_ptr = d_row_ptr;
    d.adj = d_adj;
    d.col = d_col;
    d.w = d_w;
    d.ell = d_ell;
    d.ell_col = d_ell_col;
    d.ell_w = d_ell_w;
    d.spins = d_spins;
    d.orig = d_orig;
    d.items = d_items;
    d.slice_acc = d_slice_acc;
    d.error = d_barrier ? &d_barrier->error : nullptr;
    d.slice_parts = d_slice_parts;
    d.bias = d_bias;
    return d;
  }
};

namespace isingx {

// Argument and state check at the top of every entry point: the handle is
// valid, has no latched error, and its device is current.
int graph_enter(ising_graph* g);

// Latch a CUDA failure in the handle and return ISING_ECUDA.
int graph_cuda_fail(ising_graph* g, cudaError_t e);

}  // namespace isingx
