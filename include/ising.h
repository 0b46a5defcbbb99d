/*
 * ising.h -- C ABI of the GB300 Ising max-cut annealer.
 *
 * The library anneals the Ising form of a max-cut problem on a general sparse
 * weighted graph, following Cook, Zhao, Sato, Hiromoto and Tan, "GPU Ising
 * Computing for Combinatorial Optimization Problems in VLSI Physical Design":
 *
 *   max-cut objective (Eq. 4):  cut(s) = 1/2 sum_{i<j} w_ij (1 - s_i s_j)
 *   Ising energy (Eq. 3 and 5, with J = -w so that low energy = large cut):
 *                               H(s) = sum_{(i,j) in E} w_ij s_i s_j,
 *                               cut(s) = (W - H(s)) / 2,  W = sum_{(i,j)} w_ij
 *   local field and update (Eq. 2):  f_i = sum_j w_ij s_j;
 *                               s_i <- -1 if f_i > 0, +1 if f_i < 0,
 *                               unchanged if f_i = 0
 *   annealing (Algorithm 2):    every sweep updates every spin, and right after
 *                               its own update each spin flips with probability
 *                               F_p; F_p decreases from sweep to sweep.
 *
 * Spins, weights, fields, energies and cuts are exact integers. Nothing here
 * uses floating point inside a sweep.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every function returns an int status (ISING_OK or a negative ISING_E*
 *    code); ising_strerror() names it. No C++ exception crosses this ABI.
 *  - A handle owns all device memory it uses. Input arrays passed to a call are
 *    only read during that call (the caller keeps ownership).
 *  - Device work runs on the handle's CUDA stream: the stream given to
 *    ising_create(), replaced by the stream given to each ising_anneal() call.
 *    NULL means the legacy default stream. Calls that return a value to the
 *    host (ising_cut, ising_energy, ising_get_spins to host memory) synchronise
 *    that stream.
 *  - A handle is not thread-safe: calls on one handle must be serialised.
 *    Different handles are independent.
 *  - After a CUDA error the handle latches ISING_ECUDA and every later call on
 *    it returns ISING_ECUDA; destroy it.
 *  - Vertex ids in every array that crosses this ABI are the caller's original
 *    ids 0..n-1; the internal reordering is invisible.
 */
#ifndef ISING_H
#define ISING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ising_graph ising_graph; /* opaque */

/* Status codes. */
enum {
  ISING_OK = 0,
  ISING_EINVAL = -1,   /* invalid argument (null pointer, bad id, self-loop, bad spin value ...) */
  ISING_ENOMEM = -2,   /* host or device allocation failed */
  ISING_ECUDA = -3,    /* a CUDA call failed; latched in the handle */
  ISING_ETIMEOUT = -4, /* a bounded device-side wait gave up; the result is invalid */
  ISING_ESTATE = -5,   /* call not valid in the handle's current state */
  ISING_ERANGE = -6    /* sizes or weights beyond the supported range */
};

/* Degree (distinct neighbours after merging) from which a vertex is a hub:
 * hubs are coloured among themselves and their classes are swept first. */
#define ISING_HUB_DEGREE 256

/* Annealing modes. */
enum {
  /* Colour classes are swept one after another in increasing colour order (the
   * checkerboard scheme of Sec. IV-B generalised to a greedy colouring); no two
   * vertices of a class are adjacent, so the result is a deterministic function
   * of (graph, initial spins, schedule, seed) and matches the CPU oracle bit
   * for bit. */
  ISING_MODE_DET = 0,
  /* The paper's asynchronous update (Sec. IV-B): one pass over all spins per
   * sweep with no ordering inside the sweep; each update reads whatever
   * neighbour values are in memory at that moment. Results depend on hardware
   * scheduling and are judged by cut value only. */
  ISING_MODE_RACY = 1
};

/* Schedules. */
enum {
  /* Flip probability F_p decays linearly from p0 at sweep 0 to 0 at sweep
   * t_total - 1 (Sec. V-A: linear decay; Algorithm 2: "reduce F_p"). It is
   * applied as a 32-bit integer threshold:
   *   T0     = floor(p0 * 2^32 + 0.5) clamped to [0, 2^32 - 1]
   *   thr[t] = t_total <= 1 ? 0 : floor(T0 * (t_total - 1 - t) / (t_total - 1))
   * and spin i flips in sweep t iff x < thr[t], where, with o the original
   * id of i, x is word o mod 4 of Philox4x32-10 (Salmon et al., SC'11) with
   *   key     = (lo32(seed), hi32(seed))
   *   counter = (floor(o / 4), t, replica, 0)
   * (the four vertices 4q .. 4q + 3 share one evaluation).                */
  ISING_SCHED_LINEAR = 0,
  /* Algorithm 1: a sweep updates every spin (no per-spin flips), then flips
   * N_t distinct randomly chosen spins, N_t = floor(n0 (t_total-1-t) /
   * (t_total-1)) (n0 <= n). The spins are the first N_t distinct candidates
   * c_j = floor(x_j * n / 2^32), x_j = word 0 of Philox4x32-10 with the key
   * above and counter (j, t, replica, 2), j = 0, 1, 2, ... p0 is ignored. The
   * dataflow engine runs this schedule as ISING_ENGINE_PERSISTENT. */
  ISING_SCHED_NFLIP = 1
};

/* Which kernel engine runs a deterministic anneal (all give identical spins). */
enum {
  ISING_ENGINE_AUTO = 0,       /* with cooperative launches, for deterministic linear anneals:
                                  PERSISTENT's one-block form for small graphs, else HUB for graphs
                                  with hubs it can hold, else HALO when its
                                  plan is ready and repeats at most 1.6x the work (a host thread
                                  builds the plan from the handle's second such call on; no call
                                  waits for it), else ITEMFLOW for
                                  graphs without sliced rows, else PERSISTENT; racy and N-flip
                                  anneals: PERSISTENT; without cooperative launches: PHASE */
  ISING_ENGINE_PHASE = 1,      /* one kernel launch per colour class */
  ISING_ENGINE_PERSISTENT = 2, /* one cooperative launch per anneal call, bounded grid barrier;
                                  deterministic anneals of a graph with int8 weights and at most
                                  4095 vertices (at most 1024 colours and 4M CSR entries) run in
                                  one block instead: block barriers between classes, the packed
                                  adjacency streamed by bulk copies */
  ISING_ENGINE_DATAFLOW = 3,   /* one cooperative launch per anneal call without barriers: each
                                  neighbour read waits (bounded) until the neighbour carries the
                                  update the colour order requires; racy mode runs as PERSISTENT */
  ISING_ENGINE_PERSISTENT_GRID = 4, /* PERSISTENT without the one-block form for small graphs */
  ISING_ENGINE_ITEMFLOW = 5,   /* one cooperative launch per anneal call without barriers: each
                                  warp's work item waits (bounded) for the items holding its
                                  rows' neighbours to finish the sweep the colour order requires
                                  (per-item counters, release/acquire); for graphs whose rows
                                  are not sliced across warps, deterministic linear schedule;
                                  otherwise runs as PERSISTENT_GRID */
  ISING_ENGINE_HALO = 7,       /* one cooperative launch per anneal call, one block per SM: the
                                  graph is cut into one part per block (recursive breadth-first
                                  bisection); a block keeps every vertex within D = S * K hops of
                                  its part (K colour classes, S sweeps per exchange) in shared
                                  memory, runs S sweeps there with block barriers only, then
                                  exchanges its part's spins with the parts in its halo (bounded
                                  release/acquire waits). For graphs with at most 4 colours, rows
                                  of at most 63 entries, int8 weights and regions that fit in
                                  shared memory; deterministic linear schedule; otherwise runs as
                                  ITEMFLOW */
  ISING_ENGINE_HUB = 8         /* one cooperative launch per anneal call for graphs with 1 to 10240
                                  hubs (ISING_HUB_DEGREE): one block runs every hub class with
                                  block barriers, keeping the hubs' fields in shared memory and
                                  updating them from the rows of the hubs that change; the other
                                  blocks sum the hubs' fields from the other vertices and run the
                                  other classes with a bounded grid barrier after each.
                                  Deterministic linear schedule (flip bias allowed); otherwise runs
                                  as PERSISTENT_GRID */
};

/* ising_create flags. */
enum {
  /* Keep 32-bit weights on the device even when every merged weight fits in
   * 8 bits (by default such graphs store int8 weights). */
  ISING_CREATE_WEIGHTS_I32 = 1u << 0
};

typedef struct ising_schedule {
  uint32_t kind;     /* ISING_SCHED_LINEAR or ISING_SCHED_NFLIP */
  uint32_t replica;  /* counter word 2 of every Philox draw (independent replicas) */
  double p0;         /* LINEAR: initial flip probability, 0 <= p0 <= 1 */
  uint64_t t_begin;  /* index of the first sweep this call runs, within the schedule */
  uint64_t t_total;  /* length T of the whole schedule; t_begin + sweeps <= T < 2^32 */
  uint32_t n0;       /* NFLIP: flips at sweep 0, n0 <= n */
  uint32_t reserved; /* 0 */
} ising_schedule;

/*
 * ising_create -- build the device-resident problem from an undirected edge list
 * (the max-cut instance of Sec. III, Eq. 4).
 *
 *   n        number of vertices, 1 <= n < 2^31.
 *   m        number of listed edges, 0 <= m < 2^30.
 *   src,dst  host int32[m]: edge endpoints, ids in [0, n), src[e] != dst[e].
 *            Each undirected edge may be listed in either orientation; edges
 *            listed more than once are merged by summing their weights, and a
 *            merged weight of 0 removes the edge.
 *   w        host int32[m]: edge weights (J_ij = w_ij). For every vertex the sum
 *            of |merged weight| over its edges must be < 2^31 (so every local
 *            field fits in int32).
 *   flags    ISING_CREATE_* bits.
 *   cuda_stream  cudaStream_t used for the upload and later calls (NULL: default).
 *   out      receives the handle.
 *
 * The host colours the graph greedily (largest degree first, ties by smaller
 * id; first fit) in two tiers: vertices with at least ISING_HUB_DEGREE
 * distinct neighbours (hubs) take colours 0 .. m-1 among themselves, and every
 * other vertex takes the smallest colour >= m that none of its already
 * coloured neighbours has. A graph without hubs gets plain first fit (an even
 * torus: the checkerboard). The host then orders vertices by colour and
 * uploads a CSR adjacency
 * (int32 column indices, int8 or int32 weights). Spins start at +1; call
 * ising_init_random() or ising_set_spins() to choose them.
 * Errors: ISING_EINVAL (null pointer, id out of range, self-loop, n <= 0, m < 0),
 * ISING_ERANGE (n, m or a field bound too large), ISING_ENOMEM, ISING_ECUDA.
 * On error *out is set to NULL and nothing is leaked.
 */
int ising_create(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                 uint32_t flags, void* cuda_stream, ising_graph** out);

/*
 * ising_anneal -- run `sweeps` sweeps t = t_begin .. t_begin+sweeps-1 of the
 * schedule (Algorithm 2), updating the handle's spins in place.
 *
 *   sched        schedule (see ising_schedule); copied.
 *   sweeps       number of sweeps this call runs (0 is a no-op).
 *   seed         64-bit Philox key.
 *   mode         ISING_MODE_DET or ISING_MODE_RACY.
 *   cuda_stream  becomes the handle's stream.
 *
 * Because the random numbers are counter-based, running t = 0..k-1 and then
 * t = k..T-1 gives exactly the spins of one call over 0..T-1 (resume).
 * Asynchronous: returns once the work is enqueued (no host synchronisation).
 * Errors: ISING_EINVAL (null handle/schedule, p0 outside [0,1], unknown kind or
 * mode, t_begin + sweeps > t_total, t_total >= 2^32), ISING_ECUDA,
 * ISING_ETIMEOUT (persistent engine only; reported by a later synchronising call).
 */
int ising_anneal(ising_graph* g, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                 int mode, void* cuda_stream);

/*
 * ising_anneal_trace -- as ising_anneal, recording the energy along the way:
 * the sweeps run in chunks of `every` (the last chunk may be shorter) and
 * out_energy[i] (host int64[ceil(sweeps / every)]) receives H after chunk i.
 * Counter-based randomness makes the chunked run identical to one call. This
 * is the energy-versus-sweep view of the paper's convergence study (Fig. 4).
 * Synchronises the stream. Errors as ising_anneal, plus ISING_EINVAL for
 * every == 0 or a null out_energy.
 */
int ising_anneal_trace(ising_graph* g, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                       int mode, uint32_t every, int64_t* out_energy, void* cuda_stream);

/*
 * ising_convergence_region -- the paper's convergence study (Sec. V-C, Fig. 4:
 * the range of cut values that runs from different random starts reach after
 * each number of sweeps, and one run inside it). For seed k = 0 .. num_seeds-1
 * the call sets random spins from seeds[k] (as ising_init_random with
 * sched->replica), anneals with seed seeds[k] in chunks of `every` sweeps as
 * ising_anneal_trace does, and after chunk i stores the exact cut
 * (W - H) / 2 (Eq. 4) in out_cut[k * P + i], P = ceil(sweeps / every).
 * out_min[i] / out_max[i] receive the smallest / largest cut over the seeds
 * after chunk i; row 0 of out_cut is the one-run curve. All outputs are host
 * int64 arrays. The handle's spins end as seed num_seeds - 1 left them.
 * Synchronises the stream. Errors as ising_anneal_trace, plus ISING_EINVAL for
 * a null seeds / out_cut / out_min / out_max or num_seeds == 0.
 */
int ising_convergence_region(ising_graph* g, const ising_schedule* sched, uint32_t sweeps,
                             const uint64_t* seeds, uint32_t num_seeds, int mode, uint32_t every,
                             int64_t* out_cut, int64_t* out_min, int64_t* out_max,
                             void* cuda_stream);

/*
 * ising_energy -- H(s) = sum over merged undirected edges of w_ij s_i s_j
 * (Eq. 3/5 with J = -w), computed from scratch in int64. Synchronises the stream.
 */
int ising_energy(ising_graph* g, int64_t* out_energy);

/*
 * ising_cut -- cut(s) = (W - H(s)) / 2, the Eq. 4 objective of the current
 * spins, exact int64. Synchronises the stream.
 */
int ising_cut(ising_graph* g, int64_t* out_cut);

/* ising_total_weight -- W, the sum of the merged edge weights (host value). */
int ising_total_weight(ising_graph* g, int64_t* out_w);

/*
 * ising_get_spins / ising_set_spins -- copy the spins out / in, int8[n] in the
 * caller's vertex order, values +1 / -1. `on_device` = 1 if the pointer is a
 * device pointer (e.g. a torch tensor's data_ptr()), 0 for host memory.
 * ising_get_spins to host synchronises the stream. ising_set_spins rejects any
 * value other than +1/-1 with ISING_EINVAL (device input: reported by the call
 * itself, which then synchronises the stream), leaving the spins unchanged.
 */
int ising_get_spins(ising_graph* g, int8_t* out, int on_device);
int ising_set_spins(ising_graph* g, const int8_t* in, int on_device);

/*
 * ising_init_random -- initial spins (Algorithm 2, "initialize all sigma_i"):
 * s_i = -1 if bit 31 of word o mod 4 of Philox4x32-10 with counter
 * (floor(o / 4), 0, replica, 1) and key (lo32(seed), hi32(seed)) is set, else
 * +1, o the original id of i.
 */
int ising_init_random(ising_graph* g, uint64_t seed, uint32_t replica);

/* ising_num_colours / ising_colouring -- the greedy colouring the deterministic
 * mode sweeps in (int32[n] colour per original vertex id; host memory). */
int ising_num_colours(ising_graph* g, int32_t* out);
int ising_colouring(ising_graph* g, int32_t* out_colour);

/*
 * ising_plan_colouring -- host-only (no GPU, no handle): the colouring that
 * ising_create would build for this edge list, with the same validation and
 * merging rules. out_colour: host int32[n]; out_num_colours: host int32.
 * Errors as ising_create (except ISING_ECUDA / ISING_ENOMEM on the device).
 */
int ising_plan_colouring(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int32_t* w, int32_t* out_colour, int32_t* out_num_colours);

/* ising_num_edges -- number of merged undirected edges (after removing zero
 * weights). */
int ising_num_edges(ising_graph* g, int64_t* out_m);

/* ising_set_engine -- choose the deterministic-mode kernel engine
 * (ISING_ENGINE_*). Default ISING_ENGINE_AUTO. */
int ising_set_engine(ising_graph* g, int engine);

/* ising_set_halo_sweeps -- sweeps S per exchange of ISING_ENGINE_HALO
 * (1 .. 16 / K), or 0 for the automatic choice (S = 2, or S = 1 when the S = 2
 * plan does not fit or repeats more than 1.6x the work). The plan is rebuilt at the next anneal that uses the engine.
 * ISING_EINVAL for S > 16. */
int ising_set_halo_sweeps(ising_graph* g, uint32_t sweeps_per_exchange);

/* ising_halo_info -- plans the halo engine if needed and reports its parts
 * (blocks), sweeps per exchange, dynamic shared memory per block and the
 * largest ratio of rows a block updates to the rows it owns. ISING_ESTATE if
 * the graph does not qualify (see ISING_ENGINE_HALO); any pointer may be null. */
int ising_halo_info(ising_graph* g, int32_t* out_parts, int32_t* out_sweeps,
                    int32_t* out_smem_bytes, double* out_work_ratio);

/* ising_plan_halo -- host only (no device): the halo engine's partition and
 * plan for a graph given as in ising_create, with `parts` parts and S =
 * sweeps_per_exchange (1 .. 16). out_part (n entries, by vertex id; may be
 * null) receives every vertex's part whether or not a plan exists. Returns
 * ISING_OK with the plan's shared memory per block and largest work ratio
 * (pointers may be null), ISING_ESTATE if the graph does not qualify, or the
 * ising_create errors. */
int ising_plan_halo(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                    int32_t parts, uint32_t sweeps_per_exchange, int32_t* out_part,
                    int32_t* out_smem_bytes, double* out_work_ratio);

/* ------------------------------------------------------------------------
 * Batched annealing of many independent instances.
 *
 * Every instance (a max-cut graph as in ising_create) is annealed in
 * `replicas` independent replicas by the deterministic colour-class schedule
 * of ISING_MODE_DET, all in one persistent kernel launch (captured in a CUDA
 * graph and replayed). The randomness of instance g, replica r is Philox4x32-10
 * with key (lo32(seed), hi32(seed) ^ g * 0x9E3779B9): vertex v (id within g)
 * draws word v mod 4 of counter (floor(v / 4), sweep t, r, 0) for flips and
 * of (floor(v / 4), 0, r, 1) for
 * ising_batch_init_random -- so each instance/replica reproduces a single-graph
 * anneal keyed by that instance and replica exactly.
 * ------------------------------------------------------------------------ */
typedef struct ising_batch ising_batch; /* opaque */

/*
 * ising_batch_create -- num_graphs instances. Instance g has n[g] vertices and
 * m[g] listed edges; its edges are the m[g] consecutive entries of src/dst/w
 * starting after those of instances 0..g-1 (host int32 arrays; ids local to the
 * instance, same rules as ising_create). replicas: 1..8. Every merged weight
 * must fit in int8, and every instance must have at most 204800 vertices
 * (ISING_ERANGE otherwise). Spins start at +1.
 */
int ising_batch_create(int32_t num_graphs, const int32_t* n, const int64_t* m, const int32_t* src,
                       const int32_t* dst, const int32_t* w, uint32_t replicas, void* cuda_stream,
                       ising_batch** out);
/* ising_batch_init_random -- initial spins of every instance and replica. */
int ising_batch_init_random(ising_batch* b, uint64_t seed);
/* ising_batch_anneal -- sweeps t_begin .. t_begin + sweeps - 1 of `sched`
 * (ISING_SCHED_LINEAR only; sched->replica is ignored, every replica runs) for
 * every instance and replica. Asynchronous on cuda_stream. */
int ising_batch_anneal(ising_batch* b, const ising_schedule* sched, uint32_t sweeps, uint64_t seed,
                       void* cuda_stream);
/* ising_batch_cuts -- host int64[num_graphs * replicas]: cut of instance g,
 * replica r at index g * replicas + r. Synchronises the stream. */
int ising_batch_cuts(ising_batch* b, int64_t* out_cuts);
/* ising_batch_get_spins / ising_batch_set_spins -- host int8[n[graph]] of one
 * instance and replica in the caller's vertex order (set: values +1 / -1,
 * ISING_EINVAL otherwise). Synchronise the stream. */
int ising_batch_get_spins(ising_batch* b, int32_t graph, uint32_t replica, int8_t* out);
int ising_batch_set_spins(ising_batch* b, int32_t graph, uint32_t replica, const int8_t* in);
/* ising_batch_autotune -- times `probe_sweeps` sweeps of the batch (from its
 * current spins, which are restored afterwards) for each of 18 launch
 * configurations and keeps the fastest: the block size (128, 256 or 512
 * threads, one instance per block at a time), the threads that share a row's
 * entries (1, 2 or 4; their partial sums are combined by warp shuffles) and
 * the tail mode (0: every colour class with a block barrier after it; 32:
 * classes of at most 32 vertices decided by one warp with warp barriers).
 * Results do not depend on the configuration. out_block (may be NULL)
 * receives the chosen block size; ising_batch_tuning reports the rest.
 * Synchronises the batch's stream. */
int ising_batch_autotune(ising_batch* b, uint32_t probe_sweeps, int32_t* out_block);
/* ising_batch_set_block -- choose the block size directly (128, 256 or 512). */
int ising_batch_set_block(ising_batch* b, int32_t block);
/* ising_batch_set_tuning -- choose the whole configuration directly: block
 * 128/256/512, row_split 1/2/4, tail 0..32 (ISING_EINVAL otherwise). */
int ising_batch_set_tuning(ising_batch* b, int32_t block, int32_t row_split, int32_t tail);
/* ising_batch_tuning -- the current configuration and, in out_probe_ms (18
 * floats, may be NULL), the last autotune's probe time of configuration
 * k = 6 * block_index + 2 * split_index + tail_index (block 128/256/512,
 * split 1/2/4, tail 0/32; 0 before any autotune). Any pointer may be NULL. */
int ising_batch_tuning(ising_batch* b, int32_t* out_block, int32_t* out_row_split, int32_t* out_tail,
                       float* out_probe_ms);
/* ising_batch_info -- instances, total vertices, block size, kernel launches. */
int ising_batch_info(ising_batch* b, int32_t* out_num_graphs, int64_t* out_vertices,
                     int32_t* out_block, uint64_t* out_launches);
/* ising_batch_destroy -- free the batch (NULL is ignored). */
void ising_batch_destroy(ising_batch* b);

/* Largest vertex count ising_energy_csr_static accepts. */
#define ISING_STATIC_MAX_VERTICES (1 << 24)

/*
 * ising_energy_csr_static -- energy H and cut of a spin vector on a CSR graph
 * that the caller owns, computed without allocating any memory. The paper has
 * no counterpart to this call. It exists for callers that cannot call
 * cudaMalloc: code whose device memory all belongs to a pool it does not
 * control, code held to a fixed memory budget, and loops where cudaMalloc's
 * host blocking and implicit device synchronisation are not acceptable.
 *
 *   n        number of vertices, 1 <= n <= ISING_STATIC_MAX_VERTICES; a larger
 *            n returns ISING_ERANGE before any device work.
 *   row_ptr  device int32[n+1]; col, w: device int32[row_ptr[n]]. A symmetric
 *            CSR adjacency: every undirected edge in both rows, no self-loops,
 *            col entries in [0, n). Repeated entries simply add. Not validated.
 *   spins    device int8[n], values +1 / -1.
 *   out      device int64[2]; receives {H, cut}: H = sum over undirected edges
 *            of w_ij s_i s_j and cut = (W - H) / 2, W = sum of the weights.
 *   cuda_stream  stream for the two kernels (asynchronous; NULL = default).
 *
 * Scratch: one file-scope device array of ISING_STATIC_MAX_VERTICES / 1024
 * pairs of int64 (256 KiB). Every GPU that loads the library holds it until
 * the process exits. The first call on a device looks up the array's address
 * and keeps it; make that first call before any stream capture. The kept
 * address does not survive cudaDeviceReset: do not call this entry point on
 * a device after resetting it. All calls on a device share the array (each
 * call rewrites what it reads, so nothing needs clearing); calls whose
 * kernels overlap on the GPU race and return wrong results, so order them.
 * The call never allocates or frees device or host memory.
 * Errors: ISING_EINVAL (n <= 0, or a null row_ptr, col, w, spins or out; a
 * graph without entries may pass any valid col/w pointer), ISING_ERANGE,
 * ISING_ECUDA (a launch failed, or a CUDA error was already pending when the
 * call started: then nothing is launched and the pending error is left for
 * its owner to read).
 */
int ising_energy_csr_static(int32_t n, const int32_t* row_ptr, const int32_t* col,
                            const int32_t* w, const int8_t* spins, int64_t* out,
                            void* cuda_stream);

/* ------------------------------------------------------------------------
 * Per-vertex flip bias and the learned warm start. Neither is in the paper:
 * they are project additions built on its Algorithm 2 and Eq. 2.
 *
 * Flip bias (reading R11): with a bias q_v in 0..255 set on a graph, vertex v
 * flips in sweep t of a linear schedule iff its Philox word is below
 * min((thr[t] * q_v) >> 7, 2^32 - 1), computed in 64-bit integers -- q_v = 128
 * is Algorithm 2 unchanged, q_v = 0 never flips. It applies to ISING_MODE_DET
 * and ISING_MODE_RACY sweeps of every engine; the N-flip schedule and the
 * batched engine ignore it.
 *
 * Warm-start network (readings G1-G6), evaluated on a graph's current spins:
 *   G1  merged weights w (as in ising_create); d_i = sum_j |w_ij|,
 *       c_i = (d_i + 1)^-1/2, A_hat = C W C.
 *   G2  x_i = [s_i, f_i c_i^2, s_i f_i c_i^2, log(1 + deg_i) / 8,
 *       (sum_j w_ij) c_i^2, 1, 0, 0], f_i = sum_j w_ij s_j (Eq. 2's field),
 *       deg_i the number of merged neighbours.
 *   G3  for l = 0, 1, 2: a = A_hat h, h <- relu([h, a] W_l + b_l), h = x at
 *       first (widths 8 -> 64 -> 64 -> 64); logit z = h w_o + b_o.
 *   G4  training loss against annealer spins y: mean_i softplus(-y_i z_i).
 *   G5  warm start: s_i = +1 if z_i > 0, -1 if z_i < 0, else unchanged.
 *   G6  flip bias: q_i = min(255, round_half_even(512 / (1 + exp(|z_i|)))).
 * Parameters: ISING_GNN_NUM_PARAMS floats, row-major in this order:
 * W_0 [16][64], b_0 [64], W_1 [128][64], b_1 [64], W_2 [128][64], b_2 [64],
 * w_o [64], b_o [1]; row k of W_l multiplies feature k of [h, a].
 * Arithmetic: W_0..W_2 are used rounded to bf16 and every activation h, a is
 * stored in bf16 between kernels; sums and the head are fp32 (tensor-core
 * mma with fp32 accumulation for the dense layers). Logits therefore agree
 * with exact arithmetic to about 1e-2 relative, not bit for bit.
 * A network handle may serve several graphs on the same device, one call at a
 * time; its work runs on the graph's stream.
 * ------------------------------------------------------------------------ */
#define ISING_GNN_NUM_PARAMS 17665
typedef struct ising_gnn ising_gnn; /* opaque */

/* ising_set_flip_bias -- q: uint8[n] in the caller's vertex order (host, or
 * device with on_device = 1), or NULL to remove the bias. */
int ising_set_flip_bias(ising_graph* g, const uint8_t* q, int on_device);
/* ising_get_flip_bias -- host uint8[n] in the caller's order; ISING_ESTATE if
 * no bias is set. Synchronises the stream. */
int ising_get_flip_bias(ising_graph* g, uint8_t* out);
/* ising_gnn_create -- a network on the current device with the given host
 * parameters (ISING_EINVAL if any is not finite); Adam moments start at 0. */
int ising_gnn_create(const float* params, ising_gnn** out);
/* ising_gnn_set_params / ising_gnn_get_params -- host float[ISING_GNN_NUM_PARAMS];
 * set also resets the Adam state. */
int ising_gnn_set_params(ising_gnn* net, const float* params);
int ising_gnn_get_params(ising_gnn* net, float* out);
/* ising_gnn_forward -- logits z (G3) of every vertex of g from g's current
 * spins: float[n] in the caller's order, host (synchronises) or device. */
int ising_gnn_forward(ising_gnn* net, ising_graph* g, float* out_logits, int on_device);
/* ising_gnn_gradients -- loss G4 and its gradient for labels y (int8[n], +1 /
 * -1, caller order; host values are checked, device values are read as
 * y > 0 -> +1, else -1). out_loss and out_grad (host
 * float[ISING_GNN_NUM_PARAMS]) may be NULL; a non-NULL one synchronises. */
int ising_gnn_gradients(ising_gnn* net, ising_graph* g, const int8_t* labels, int labels_on_device,
                        float* out_loss, float* out_grad);
/* ising_gnn_train_step -- the same gradient, then one Adam step (beta1 0.9,
 * beta2 0.999, eps 1e-8) with learning rate lr on the fp32 master weights. */
int ising_gnn_train_step(ising_gnn* net, ising_graph* g, const int8_t* labels, int labels_on_device,
                         float lr, float* out_loss);
/* ising_gnn_warm_start -- forward pass, then G5 on g's spins (resets the
 * update parity, like ising_set_spins) and, if set_bias, G6 as g's flip bias.
 * Asynchronous on g's stream. */
int ising_gnn_warm_start(ising_gnn* net, ising_graph* g, int set_bias);
/* ising_gnn_batch_forward -- logits z (G3) of every vertex of every instance
 * of batch b from replica `replica`'s spins, the instances taken together as
 * one graph (no edge joins two instances, so each instance's logits are
 * those of the instance alone): float[total vertices], instance by instance
 * in batch order, each by vertex id; host (synchronises) or device.
 * ISING_EINVAL for a replica the batch does not have. */
int ising_gnn_batch_forward(ising_gnn* net, ising_batch* b, uint32_t replica, float* out_logits,
                            int on_device);
/* ising_gnn_batch_warm_start -- for replica `replica` (or every replica with
 * ISING_ALL_REPLICAS): a forward pass from its spins, then G5 on its spins.
 * Asynchronous on the batch's stream (the stream of its last anneal call). */
#define ISING_ALL_REPLICAS 0xFFFFFFFFu
int ising_gnn_batch_warm_start(ising_gnn* net, ising_batch* b, uint32_t replica);
/* ising_gnn_batch_gradients / ising_gnn_batch_train_step -- as
 * ising_gnn_gradients / ising_gnn_train_step on the batch's instances taken
 * together as one graph, from replica `replica`'s spins: the loss G4 is the
 * mean over every vertex of every instance (one minibatch of graphs).
 * labels: int8[total vertices] (+1 / -1), laid out as the logits of
 * ising_gnn_batch_forward; host values are checked. */
int ising_gnn_batch_gradients(ising_gnn* net, ising_batch* b, uint32_t replica, const int8_t* labels,
                              int labels_on_device, float* out_loss, float* out_grad);
int ising_gnn_batch_train_step(ising_gnn* net, ising_batch* b, uint32_t replica, const int8_t* labels,
                               int labels_on_device, float lr, float* out_loss);
/* ising_gnn_set_dense_path -- the tensor-core path of the forward layers'
 * products: ISING_GNN_DENSE_MMA_SYNC (the default; 64-row tiles, warp-level
 * mma.sync, several blocks per SM) or ISING_GNN_DENSE_TCGEN05 (128-row
 * tiles in a warp-specialised pipeline: gather warps fill a ring of shared
 * memory tiles, one thread issues tcgen05.mma into fp32 accumulators in
 * tensor memory, four warps read them back). The layer is bound by its
 * neighbour gather, not by the product, and the default keeps more warps
 * gathering per SM; it is the faster of the two on every graph measured.
 * Both round the same bf16 operands and accumulate in fp32; results differ
 * only in the order of the fp32 sums. A tcgen05 pipeline wait that does not
 * end within 1 s latches ISING_ETIMEOUT in the network (reported by the next
 * call that synchronises). ISING_EINVAL for any other value. */
#define ISING_GNN_DENSE_TCGEN05 0
#define ISING_GNN_DENSE_MMA_SYNC 1
int ising_gnn_set_dense_path(ising_gnn* net, int path);
/* ising_gnn_launch_count -- kernels launched by this network handle. */
int ising_gnn_launch_count(ising_gnn* net, uint64_t* out);
/* ising_gnn_destroy -- free the network (NULL is ignored). */
void ising_gnn_destroy(ising_gnn* net);

/* ising_engine_used -- the engine the last anneal call ran: ISING_ENGINE_PHASE,
 * ISING_ENGINE_PERSISTENT_GRID (the persistent grid-barrier kernel),
 * ISING_ENGINE_DATAFLOW, ISING_ENGINE_ITEMFLOW, ISING_ENGINE_HALO, ISING_ENGINE_HUB or
 * ISING_ENGINE_USED_BLOCK
 * (PERSISTENT's one-block form); -1 before the first anneal. */
#define ISING_ENGINE_USED_BLOCK 6
int ising_engine_used(ising_graph* g, int32_t* out);

/* Failure-detection test hook. Every device-side wait of the anneal kernels
 * is bounded (2 s by default); a wait that runs out records an error, the
 * kernel returns, and the next synchronising call reports ISING_ETIMEOUT and
 * latches it in the handle (create a new handle to continue; the CUDA
 * context stays usable). Kinds:
 *   ISING_FAULT_SKIP_ARRIVAL  persistent grid engine: block 0 skips its first
 *                             grid-barrier arrival, so every block's wait runs out;
 *   ISING_FAULT_SHORT_COPY    block engine: the first chunk's barrier expects 16
 *                             bytes that never arrive, so its wait runs out.
 * wait_budget_ns bounds every wait of later anneal calls (0: the default; at
 * most 60 s). No fault is a GPU fault: nothing traps or hangs. */
enum { ISING_FAULT_NONE = 0, ISING_FAULT_SKIP_ARRIVAL = 1, ISING_FAULT_SHORT_COPY = 2 };
int ising_debug_fault(ising_graph* g, int kind, uint64_t wait_budget_ns);

/* ising_launch_count -- number of CUDA kernels this handle has launched since
 * ising_create (a diagnostic for benchmarks). */
int ising_launch_count(ising_graph* g, uint64_t* out);

/* ising_destroy -- free the handle and its device memory (NULL is ignored).
 * Waits for the handle's outstanding work first. */
void ising_destroy(ising_graph* g);

/* ising_strerror -- static description of a status code. */
const char* ising_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */
