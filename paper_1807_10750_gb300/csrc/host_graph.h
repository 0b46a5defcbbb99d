// Host-side construction of the device layout: validation, duplicate merging,
// greedy colouring, colour-ordered CSR and the per-class work items the sweep
// kernels consume.
#pragma once

#include <atomic>
#include <cstdint>
#include <memory>
#include <new>
#include <utility>
#include <vector>

#include "../../include/ising.h"

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

// An allocator whose resize leaves new elements uninitialised, for the large
// arrays the build writes in full right after sizing them.
template <typename T>
struct NoInitAllocator : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAllocator<U>;
  };
  NoInitAllocator() = default;
  template <typename U>
  NoInitAllocator(const NoInitAllocator<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};

// Vertices with at least this many distinct neighbours are hubs (ising.h).
constexpr int32_t kHubDegree = ISING_HUB_DEGREE;

struct HostGraph {
  int32_t n = 0;
  int32_t num_hubs = 0;      // hubs hold positions [0, num_hubs)
  int32_t hub_colours = 0;   // hub classes are colours [0, hub_colours)
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
  std::vector<int32_t, NoInitAllocator<int32_t>> col;  // nnz, neighbour positions
  std::vector<int32_t, NoInitAllocator<int32_t>> w;    // nnz
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

// Halo engine (halo.cuh). The vertices are cut into P parts of n / P vertices
// by recursive bisection along breadth-first orders; block p owns part p. An
// epoch of S sweeps is D = S * K colour phases (K classes); its region is
// every vertex within D hops of the part, so the block can run all D phases on
// its own copy of the region -- phase j updates the class-(j-1) mod K vertices
// at most D - j hops out, whose neighbours are all current -- and exchanges
// only the halo (the region outside the part) between epochs.
//
// Per part the region's vertices get local indices ordered by (class, hops,
// position); the rows that some phase updates (at most D - 1 hops) are stored
// as 32-row slices in slot-major sliced ELL over local indices, word
// (local col << 8) | (w & 0xff), padding (R << 8) with R the region size. A
// header of kHaloHdr ints per part gives the offsets into the flat arrays and,
// per class c, the first local index seg, the first slice, and cnt[l] = the
// class's vertices at most l hops out (l = 0 .. D).
constexpr int32_t kHaloHdr = 128;
constexpr int32_t kHaloHdrClass = 16;  // per-class tables start here
constexpr int32_t kHaloMaxClasses = 4;
constexpr int32_t kHaloMaxDepth = 16;
constexpr int32_t kHaloMaxWidth = 63;  // row degree limit (6-bit slice width)
constexpr int32_t kHaloSmemLimit = 225 * 1024;
enum HaloHdr {
  kHaloR = 0,          // region vertices
  kHaloWordsOff = 1,   // first word in `words` (multiple of 4)
  kHaloWordsLen = 2,   // words (multiple of 4)
  kHaloSlicesOff = 3,  // first entry in `slices`
  kHaloSlicesLen = 4,
  kHaloGposOff = 5,    // first entry in `gpos` (R entries)
  kHaloImportOff = 6,  // first entry in `imports` (pairs)
  kHaloImportLen = 7,  // halo vertices
  kHaloNbrOff = 8,     // first entry in `nbrs`
  kHaloNbrLen = 9,
  kHaloOwned = 10,
  kHaloFlipWords = 11,  // flip bitmap words of a full epoch: S * slices
  kHaloExportOff = 12,  // first entry in `exports` (pairs)
  kHaloExportLen = 13,  // mailbox slots the part writes between epochs
  kHaloQuadOff = 14,    // first entry in `quads` (triples)
  kHaloQuadLen = 15     // vertex quads with an updated row in the region
};
// The per-class table of class c starts at kHaloHdrClass + c * (D + 3):
// seg, first slice, cnt[0 .. D].
//
// An updated row's slot is 32 * (its slice) + (its lane in the slice), slices
// counted from the part's first. Flips: the vertices 4q .. 4q + 3 (original
// ids) share one Philox evaluation per sweep, so a part lists every quad q
// with an updated row as (q, s0 | s1 << 16, s2 | s3 << 16), s_k the slot of
// vertex 4q + k or 0xffff if it is not an updated row here; a sweep's flip
// bitmap has one word per slice, bit `lane` for the row in that lane.
//
// A block's shared memory, in this order: the header, the words, the slices
// (padded to 4), the epoch's flip bitmap (S words per slice), the quads (3
// words each), the region's spins (int8 +1 / -1, R + 1, padded to 16) and the
// updated rows' flip biases by slot (32 per slice).
inline int64_t halo_smem_bytes(int32_t R, int32_t words, int32_t slices, int32_t flip_words,
                               int32_t quads) {
  return int64_t(kHaloHdr) * 4 + int64_t(words) * 4 + int64_t((slices + 3) / 4 * 4) * 4 +
         int64_t(flip_words) * 4 + int64_t(quads) * 12 + int64_t((R + 1 + 15) / 16 * 16) +
         int64_t(slices) * 32;
}

struct HaloPlan {
  bool ok = false;
  int32_t parts = 0, sweeps_per_epoch = 0, depth = 0, classes = 0;
  int32_t smem_bytes = 0;         // dynamic shared memory of the largest part
  double max_work_ratio = 0.0;    // max over parts: rows updated per sweep / owned rows
  std::vector<int32_t> hdr;       // kHaloHdr per part
  std::vector<int32_t> words;     // sliced ELL
  std::vector<int32_t> slices;    // (word offset within the part << 6) | width
  std::vector<int32_t> gpos;      // local index -> position
  std::vector<int32_t> imports;   // (local index, position) of halo vertices (> 0 hops); import i
                                  // of a part reads mailbox slot (the part's first import / 2) + i
  std::vector<int32_t> exports;   // (local index, mailbox slot): an own vertex some part imports
  int64_t mailbox_slots = 0;      // all parts' imports
  std::vector<int32_t> quads;     // (q, l0 | l1 << 16, l2 | l3 << 16) per quad
  std::vector<int32_t> nbrs;      // parts owning some vertex of the halo
};

// Parts of n / P vertices by recursive bisection: a subset is ordered
// breadth-first from a far vertex (the last one a pass from a vertex on the
// subset's rim reaches; further components follow in order) and split in
// proportion to the parts each side gets. part[v] for every position v.
// `cancel` (may be null) stops the work early once it reads true; the result
// is then incomplete.
void bisect_parts(const HostGraph& g, int32_t parts, std::vector<int32_t>* part,
                  const std::atomic<bool>* cancel = nullptr);

// Fills hp (ok = true) when K <= kHaloMaxClasses, D = S * K <= kHaloMaxDepth,
// every row has at most kHaloMaxWidth entries and int8 weights, every part is
// non-empty and each part's tables fit in kHaloSmemLimit bytes of shared
// memory; otherwise hp->ok = false. Once `cancel` (may be null) reads true it
// stops early with hp->ok = false.
void build_halo_plan(const HostGraph& g, int32_t parts, int32_t sweeps_per_epoch, HaloPlan* hp,
                     const std::atomic<bool>* cancel = nullptr);

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
