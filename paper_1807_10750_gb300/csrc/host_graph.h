// Host-side construction of the device layout: validation, duplicate merging,
// greedy colouring, colour-ordered CSR and the per-class work items the sweep
// kernels consume.
#pragma once

#include <cstdint>
#include <vector>

namespace isingx {

// A unit of sweep work for one warp. Three kinds:
//  * light rows (every row of degree <= the light slot count): vertices
//    [v_begin, v_end) of one colour class stored in sliced-ELL form starting
//    at ELL word e_begin, with e_end = -(D + 1) for D slots per row;
//  * group rows: vertices [v_begin, v_end) with all of their CSR entries
//    [e_begin, e_end) (e_end >= 0);
//  * a slice of one heavy row: vertex v_begin, CSR entries [e_begin, e_end),
//    and v_end = -(slot + 1) names the partial-sum slot that combines slices.
struct WorkItem {
  int32_t v_begin, v_end, e_begin, e_end;
};

struct HostGraph {
  int32_t n = 0;
  int64_t num_edges = 0;      // merged undirected edges
  int64_t nnz = 0;            // directed CSR entries (2 * num_edges)
  int64_t total_weight = 0;   // W
  int32_t num_colours = 0;
  int32_t max_degree = 0;
  bool fits_int8 = true;      // every merged |w| <= 127

  std::vector<int32_t> colour;       // per original id
  std::vector<int32_t> perm;         // position -> original id
  std::vector<int32_t> pos;          // original id -> position
  std::vector<int32_t> class_begin;  // num_colours + 1 positions
  std::vector<int32_t> row_ptr;      // n + 1, by position
  std::vector<int32_t> col;          // nnz, neighbour positions
  std::vector<int32_t> w;            // nnz
};

struct WorkPlan {
  std::vector<WorkItem> items;
  std::vector<int32_t> class_item_begin;  // num_colours + 1
  std::vector<int32_t> split_parts;       // per slot: number of slices
  std::vector<int32_t> ell_col;           // sliced-ELL columns of light items (-1: none)
  std::vector<int32_t> ell_w;             // sliced-ELL weights (0 where the column is -1)
  int32_t max_class_items = 0;
};

// Small graphs are annealed by one block (block.cuh) with block barriers
// between colour classes instead of grid barriers. Every CSR entry becomes a
// word (row << 20) | (col << 8) | (w & 0xff) over 12-bit positions; the words
// are grouped by the row's colour class, each class is padded to a multiple
// of four words with (n << 20) (a zero term on a spare row), and the classes
// are cut into chunks of at most kBlockChunkWords words that never cross a
// class.
constexpr int32_t kBlockMaxVertices = 4095;  // 12-bit positions
constexpr int32_t kBlockChunkWords = 4096;
constexpr int32_t kBlockMaxChunks = 1024;   // chunk table kept in shared memory
constexpr int32_t kBlockMaxClasses = 1024;  // class tables kept in shared memory

struct BlockPlan {
  bool ok = false;
  std::vector<int32_t> words;
  std::vector<int32_t> chunk_off;    // per chunk: first word (multiple of 4)
  std::vector<int32_t> chunk_len;    // per chunk: words (multiple of 4)
  std::vector<int32_t> class_chunk;  // per class + 1: first chunk
};

// Fills bp (ok = true) for a graph with int8 weights, at most
// kBlockMaxVertices vertices, kBlockMaxClasses classes and kBlockMaxChunks
// chunks; otherwise leaves bp->ok = false.
void build_block_plan(const HostGraph& g, BlockPlan* bp);

// Item dependencies for the item-dataflow engine. For graphs whose work
// items are all light or group items (no row sliced across warps), item i
// depends on every other item j holding a neighbour of one of i's rows;
// deps[dep_ptr[i] .. dep_ptr[i + 1]) lists (j << 1) | later, later = 1 if j's
// colour class comes after i's. In sweep t, i may update once every earlier
// j has finished sweep t and every later j has finished sweep t - 1.
// Returns false (and leaves the vectors empty) if some item is a slice.
bool build_item_deps(const HostGraph& g, const WorkPlan& plan, std::vector<int32_t>* dep_ptr,
                     std::vector<int32_t>* deps);

// Returns 0, or a negative ISING_* status.
int build_host_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     const int32_t* w, HostGraph* out);

// Splits each colour class into work items of at most L = max(min_edges,
// ceil(class edges / target_warps)) edges. Within a class rows are ordered by
// degree, so a class is: rows longer than L (sliced), then rows longer than
// light_slots (group items of up to max_rows rows), then light rows (items of
// up to 32 * rows_per_lane(D) rows, D = the item's widest row).
void build_work_plan(const HostGraph& g, int32_t target_warps, int32_t min_edges,
                     int32_t max_rows, int32_t light_slots, WorkPlan* plan);

}  // namespace isingx
