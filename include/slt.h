/* slt.h - sparse-tiled DG elastic-wave time stepping on one GB300 (sm_103a).
 *
 * C ABI of libslt.so.  Plain pointers and sizes only; every entry point returns an slt_status
 * (0 on success) and never throws or aborts.  slt_last_error() returns a thread-local message
 * describing the last failure of the calling thread.
 *
 * Conventions
 *  - "host" pointers are read (or written) during the call only and never retained;
 *    "device" pointers are CUDA global-memory pointers borrowed for the duration of the call.
 *  - Objects (chain, mesh, schedule) are owned by the library and freed by their destroy call.
 *  - Calls taking a `stream` (a cudaStream_t, NULL = legacy default stream) enqueue their GPU
 *    work on it; slt_inspect, slt_mesh_create and the slt_schedule_* queries synchronise the
 *    stream before returning.  Arguments are validated on the host before any launch:
 *    invalid input returns SLT_ERR_ARG with nothing launched.
 *  - Integers that index sets are int32; sizes are int64 (each set holds < 2^31 elements).
 *
 * Section and algorithm numbers refer to Luporini et al., "Automated Tiling of Unstructured
 * Mesh Computations with Application to Seismological Modelling" (arXiv:1708.03183).
 */
#ifndef SLT_H
#define SLT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SLT_OK = 0,
  SLT_ERR_ARG = -1,          /* invalid argument (checked before any GPU work) */
  SLT_ERR_OOM = -2,          /* device or host allocation failed */
  SLT_ERR_CUDA = -3,         /* a CUDA runtime call or kernel launch failed */
  SLT_ERR_TIMEOUT = -4,      /* a bounded device wait gave up */
  SLT_ERR_CONFLICT_CAP = -5, /* conflict buffer of the inspector overflowed */
  SLT_ERR_UNSUPPORTED = -6,  /* valid request outside what this library implements */
  SLT_ERR_STATE = -7         /* object used in the wrong state (e.g. schedule of another mesh) */
} slt_status;

typedef struct slt_chain_s* slt_chain;       /* loop chain description (host) */
typedef struct slt_schedule_s* slt_schedule; /* inspector output (device resident) */
typedef struct slt_mesh_s* slt_mesh;         /* DG elastic mesh (device resident) */
typedef struct slt_receivers_s* slt_receivers; /* point receivers on a mesh */
typedef struct slt_group_s* slt_group;       /* meshes advanced together (device resident) */

const char* slt_last_error(void);
/* Library version and the compute capability it was built for (e.g. 103). */
int slt_version(int32_t* major, int32_t* minor, int32_t* arch);

/* ------------------------------------------------------------------ loop chain (Section 2)
 * A loop chain is an ordered list of loops; each loop iterates over a set (iteration space)
 * and carries descriptors <map or direct, mode in {r, w, i}> (Section 2, Figure 2 right).
 * The order of slt_loop calls is the order of the chain.  Maps are flat arrays
 * values[i * arity + k], copied at the call. */
int slt_chain_create(slt_chain* out);
int slt_chain_destroy(slt_chain chain);
/* Declare a set of `size` >= 0 elements; returns its id (0, 1, ...). */
int slt_set(slt_chain chain, int64_t size, int32_t* set_id);
/* Declare a map from_set -> to_set^arity from host values (each in [0, size(to_set))).
   SLT_ERR_ARG for arity < 1, unknown sets or out-of-range values. */
int slt_map(slt_chain chain, int32_t from_set, int32_t to_set, int32_t arity,
            const int32_t* host_values, int32_t* map_id);
/* Append a loop over set_id with ndesc >= 1 descriptors: map_ids[d] (-1 = direct access)
   and modes[d] in {'r', 'w', 'i'}.  An indirect descriptor's map must start at set_id. */
int slt_loop(slt_chain chain, int32_t set_id, int32_t ndesc, const int32_t* map_ids,
             const char* modes, int32_t* loop_id);
/* Attach a 2-D point (host, [size][2] doubles) to every element of a set; the Hilbert
   renumbering of the seed partition uses the points of the seed set. */
int slt_set_points(slt_chain chain, int32_t set_id, const double* host_xy);
/* Counts of the chain's sets, maps and loops (host; a NULL output is skipped); SLT_ERR_ARG for a
   null chain. */
int slt_chain_info(slt_chain chain, int32_t* nsets, int32_t* nmaps, int32_t* nloops);

/* ------------------------------------------------------------------ inspector (Section 5.1)
 * slt_inspect runs Algorithm 1 (with Algorithms 2 and 3) as GPU kernels on every sub-chain
 * [split_k, split_{k+1}) of the chain (a fusion scheme: sub-chains are tiled independently and
 * executed one after the other).
 *
 *  seed loop  : the sub-chain's first loop, or seed_loop[k] loops after it (backward tiling).
 *  partition  : seed iterations ranked by identity (renumber = 0) or by a stable sort of the
 *               order-16 Hilbert index of their points quantised on a 65536^2 grid over the
 *               bounding box (renumber = 1); iteration of rank r goes to tile r / tile_size.
 *  adjacency  : through the first map of the sub-chain touching the seed set, plus fake edges.
 *  colouring  : colouring = 0: Jones-Plassmann with priorities splitmix64(tile ^ prio_seed),
 *               each tile taking the smallest colour unused by higher-priority neighbours;
 *               colouring = 1: tile t gets colour t.
 *  projection : MAX colour, previous projection kept on ties, all descriptors projected.
 *  conflicts  : two distinct same-colour tiles touching one element; they become fake edges and
 *               the sub-chain is re-coloured, up to max_rounds times or until the fake edges
 *               exceed 16 per tile, then colouring falls back to sequential.
 * The output is bit-identical to a sequential execution of the same rules. */
typedef struct {
  int32_t tile_size;     /* seed tile size ts >= 1 */
  int32_t colouring;     /* 0 = Jones-Plassmann greedy, 1 = sequential */
  int32_t renumber;      /* 0 = identity, 1 = Hilbert (needs points on the seed set) */
  int32_t max_rounds;    /* restarts before the sequential fallback (>= 0) */
  uint64_t prio_seed;    /* colouring priority seed */
  int32_t nsplit;        /* number of split points (0 = one sub-chain) */
  int32_t split[15];     /* strictly increasing loop indices in (0, nloops) */
  int32_t executor;      /* elastic chains: 0 = dataflow (default), 1 = colour phases,
                            2 = dataflow with one thread-block cluster of 256-thread CTAs per tile
                            (for large tiles; single-field runs), 3 = staged dataflow (each
                            tile's sub-chain out of shared memory; single-field runs),
                            4 = dataflow with each segment of a tile run as compacted passes
                            over the items that have each part (lists of executor 3, values
                            in global memory; single-field runs) */
  int32_t wait_spins;    /* dataflow: polls of a dependency before giving up (0 = 2^24, ~1 s+) */
  int32_t block_threads; /* threads per tile CTA: 128, 256 or 384, and 512 or 768 for executors
                            0 and 3 (0 = 256) */
  int32_t sub_tile_size[16]; /* seed tile size of sub-chain k (0 = tile_size): a fusion scheme
                                with its own tile size per sub-chain (Section 7.2) */
  int32_t cluster_size;      /* executor 2: CTAs per tile cluster, 1..8 (0 = 8) */
  int32_t shots_per_cta;     /* multi-shot runs with the dataflow executor: a tile CTA runs its
                                items for this many shots (0 = all); the shots go through the
                                queue in slices of this size, one persistent launch each */
  int32_t seed_loop[16];     /* seed loop of sub-chain k, counted from its first loop (0 = the
                                first loop, forward tiling only); > 0 selects backward tiling
                                for the loops before it (Section 5.1.1): MIN projections from
                                the seed towards the first loop, then MAX projections over the
                                loops up to the seed and forward tiling after it */
  int32_t release_order;     /* dataflow executors (0, 2, 3, 4), what a CTA does with the tiles its
                                finished tile released: 1 = run the first one itself (its cells
                                are still in L2) and queue the others, 2 = queue them all in
                                release order, 0 = the executor's default: 1 for the staged
                                executor (3), whose DRAM traffic it cuts by about a tenth, 2 for
                                the others, which it slows (1 % at ts 256, 16 % for 4-CTA tile
                                clusters at ts 2048: a kept tile runs ahead of older ready ones) */
} slt_options;

/* Default options: ts 1024, greedy colouring, Hilbert renumbering, 16 rounds, seed 0x5EED,
   no split, dataflow executor, no per-sub-chain tile sizes. */
int slt_options_default(slt_options* opt);
/* Inspect `chain` with the options `opt` (start from slt_options_default) on `stream` (a
   cudaStream_t; NULL = the default stream) and return a new schedule in *out, owned by the caller
   (slt_schedule_destroy).  The schedule copies what it needs from the chain.  Synchronises
   `stream`.  For chains made by slt_mesh_chain it also builds the executor plans (per-tile
   segment items) and the dataflow graph.  Errors: SLT_ERR_ARG for a null argument, a chain without
   loops, or invalid options (tile_size < 1, split points not strictly increasing inside
   (0, nloops), seed_loop outside its sub-chain, renumber = 1 without points on a seed set,
   executor, cluster_size, block_threads, wait_spins or release_order out of range, executors 3 and
   4 on a chain not made by slt_mesh_chain); SLT_ERR_UNSUPPORTED for 2^26 cells or more on a mesh
   chain, a cell touched by more than 16 tiles of one sub-chain (executor plans), or a tile whose
   footprint exceeds the staged executor's shared memory (executor 3) or the 1022 slots the
   staged and pass lists can name (executors 3 and 4); SLT_ERR_OOM / SLT_ERR_CUDA from the device.  *out is NULL on
   error. */
int slt_inspect(slt_chain chain, const slt_options* opt, void* stream, slt_schedule* out);
int slt_schedule_destroy(slt_schedule sched);
/* Per sub-chain statistics: info[0..7] = ntiles, ncolours, restarts, fell_back_to_sequential,
   conflict pairs in the last conflicting round, iterations with no projected element (sent to
   tile 0), first loop, number of loops. */
int slt_schedule_info(slt_schedule sched, int32_t subchain, int64_t info[8]);
/* The dependency graph of the dataflow executor (schedules inspected on slt_mesh_chain; a node
   is one (time step, tile) pair; its edges are the part of Algorithm 4's order that matters, tiles
   of lower colour before higher colour within a sub-chain and sub-chains in chain order, kept only
   between tiles that touch a common cell): info[0] = nodes per time step (tiles of all sub-chains),
   [1] dependency edges per step, [2] the longest dependency chain per step in the steady state,
   in nodes, [3] the same with every node weighted by its work items and divided by the mean items
   per node, [4] work items per step, [5] tiles in flight in the last dataflow run of the schedule
   (CTAs, or clusters for executor 2; 0 before the first run).  Time per step cannot fall below
   [3] node times however many tiles are in flight; it reaches the work bound only when
   [0] / [5] is well above [3].  SLT_ERR_ARG for a schedule without an executor plan. */
int slt_schedule_dataflow_info(slt_schedule sched, double info[6]);
/* FP64 lane accounting of one time step of the schedule's plans (schedules inspected on
   slt_mesh_chain), in warp-lane FP64 instructions, counted from the part functions' instruction
   counts at the mesh's degree: info[0] what the step needs (every item's parts), info[1] what the
   dataflow executors issue (warps of 32 consecutive plan items of a tile; a warp issues a part when
   any of its lanes has it, so idle lanes count), info[2] what the staged executor's compacted
   passes issue (each pass padded to whole warps), info[3] what the untiled chain issues (every
   cell, warps of 32 consecutive cells).  info[0] / info[1] is the lane efficiency of the tiled
   executors; the FP64 pipe spends a full issue slot on a warp instruction whatever its active
   lanes.  Synchronises. */
int slt_schedule_lane_info(slt_schedule sched, double info[4]);
/* Wall seconds slt_inspect spent per stage, each ended by a stream synchronisation: [0] seed
   partition (Hilbert ranks), [1] colouring, projections, tiling functions and conflict repair
   (Algorithms 1-3, every restart included), [2] iteration lists, [3] the executor
   plans, [4] the staged and pass executors' plans, [5] the dataflow dependency graph, [6..7] zero.  Summed
   over the sub-chains. */
int slt_schedule_inspection_times(slt_schedule sched, double seconds[8]);
/* Copy one integer array of the schedule to host memory.  Call with host_out = NULL to get
   the length in *n.  kind:
     0 rank of every seed element            (loop, desc ignored)
     1 colour of every tile                  (loop, desc ignored)
     2 tiling function sigma_j               (loop = j, chain-global index)
     3 iteration-list offsets [ntiles + 1]   (loop)
     4 iteration lists, ascending per tile   (loop)
     5 local-map footprint offsets [ntiles+1](loop, desc = indirect descriptor index; kinds 5-7 and
       14 build the loop's local maps on the device at their first request, then keep them)
     6 local-map footprints (sorted targets per tile)
     7 local maps: position of map[i*arity+k] in the footprint of tile sigma_j[i]
     8 dataflow graph: successor offsets [G + 1] over the G tiles of all sub-chains (tile t of
       sub-chain k is node cum_k + t, cum_k the tiles of the earlier sub-chains; loop, desc ignored)
     9 dataflow graph: successors, (node << 1) | 1 when the successor is the next step's node,
       ascending within each node's list (one entry per distinct dependency)
    10 dataflow graph: dependencies of each node's first-step instance [G] (same-step edges)
    11 dataflow graph: dependencies of each node's later instances [G] (all edges)
    12 staged executor: footprint offsets [ntiles + 1] of sub-chain `loop`
    13 staged executor: footprints, per tile the cells (caller numbering) its segments touch, in
       slot order (the tile's local map of the cell set over the whole sub-chain)
    14 export flags of loop `loop`, one per iteration: 1 when an element the iteration writes or
       increments is also touched, in some loop of its sub-chain, by a tile other than its own
       (a value the tile must write back for another tile rather than keep local; Algorithm 1,
       compute_local_maps).  Computed on the device from the tiling functions and the local
       maps at the call; synchronises
   The sub-chain is the one containing `loop` (kinds 0, 1: the sub-chain index in `loop`). */
int slt_schedule_export(slt_schedule sched, int32_t kind, int32_t loop, int32_t desc,
                        int32_t* host_out, int64_t* n);

/* ------------------------------------------------------------------ DG elastic mesh
 * Velocity-stress elastic waves in 2-D (Section 7.1): DG P_degree on affine triangles with
 * centered fluxes, free surface on every exterior facet, explicit fourth-order staggered
 * Taylor leapfrog.  Fields are nodal values on the equispaced points (i/p, j/p) of the
 * reference triangle (0,0),(1,0),(0,1), j outer, i inner; the local vertex order of each cell
 * defines its reference map.  Field layouts (host or device): v [ncell][2][Np] (vx, vy),
 * sigma [ncell][3][Np] (sxx, syy, sxy), Np = (p+1)(p+2)/2, cells in the caller's numbering.
 *
 * cell2vert [ncell][3] vertex ids (topology: two cells sharing two vertex ids share a facet),
 * cellxy [ncell][3][2] vertex coordinates per cell (periodic meshes: unwrapped per cell),
 * rho, lam, mu [ncell] material; src_xy [2] explosive point source position (NULL: none).
 * All host arrays, copied.  degree in 1..4.  The work layout on the device follows the
 * Hilbert order of the cell centroids. */
int slt_mesh_create(const int32_t* cell2vert, const double* cellxy, int64_t ncell, int32_t degree,
                    const double* rho, const double* lam, const double* mu, const double* src_xy,
                    void* stream, slt_mesh* out);
int slt_mesh_destroy(slt_mesh mesh);
/* info[0..7] = ncell, degree, Np, interior facets, exterior facets, source cell (-1: none),
   number of chain loops (17), velocity/stress split loop (9). */
int slt_mesh_info(slt_mesh mesh, int64_t info[8]);
/* Work of one time step on this mesh, as the executor performs it: cost[0] = FP64 flops
   (an FMA counts 2; structural zeros of the reference differentiation matrices are skipped;
   interior facets counted from both sides, as the per-cell pulls compute them), cost[1] =
   algorithmic DRAM bytes of the tiled chain when every tile's data stays on chip (v and sigma
   read and written once, geometry and material read once: (80 Np + 140) B per cell), cost[2]
   = algorithmic DRAM bytes of the untiled chain, every loop streaming its operands and results
   ((808 Np + 808) B per cell), cost[3] = nonzeros of Dr plus Ds. */
int slt_mesh_cost(slt_mesh mesh, double cost[4]);
/* The seventeen-loop chain of one time step over the sets cells (0), interior facets (1),
   exterior facets (2), with maps facet->cell (arity 2, map 0) and exterior facet->cell
   (arity 1, map 1); points: cell centroids ((x0 + x1) + x2) / 3 on set 0, facet midpoints
   (xa + xb) * 0.5 on sets 1 and 2 (endpoints taken from the facet's first cell).  Facets are numbered by
   (min vertex id, max vertex id); an interior facet lists its smaller cell id first.
   Loops: volB intB extB volD intD hookeB intB extB updV | volD intD hookeB intB extB volD intD updS. */
int slt_mesh_chain(slt_mesh mesh, slt_chain* out);

/* ------------------------------------------------------------------ executor (Section 5.2)
 * nsteps time steps on device fields v, sigma (layout above, updated in place).
 * ricker: device array [nsteps] of the source time function at t_{n+1/2} (NULL: no source).
 * sched = NULL runs the plain untiled chain: six launches per step, one per run of consecutive
 * loops in which no cell reads a value another cell writes during the run; four or more steps
 * replay a CUDA graph of one step.  Otherwise the schedule must come from slt_inspect on
 * slt_mesh_chain(mesh) and each tile executes its slice of every loop of its sub-chain in chain
 * order:
 *  - executor 1 (colour phases, Algorithm 4 in shared-memory mode): one launch per colour and
 *    sub-chain, all tiles of a colour in parallel, one CTA per tile;
 *  - executor 0 (dataflow, default): one persistent launch for all nsteps, one CTA per tile;
 *    each (step, tile) node runs once the tiles it overlaps have finished (lower colours of its
 *    sub-chain, the previous sub-chain's tiles on its cells): a linear extension of the same
 *    order.  Waits are bounded: SLT_ERR_TIMEOUT if one gives up;
 *  - executor 2: as executor 0 with one thread-block cluster of cluster_size CTAs per tile;
 *  - executor 3 (staged): as executor 0, with each node run out of shared memory: the tile's
 *    footprint (export kinds 12, 13) gets one slot per cell, the operands the tile has not
 *    produced itself are gathered once per segment, every segment runs as compacted passes
 *    (volume part, interior faces 0, 1, 2, free-surface faces, later cell loop) separated by
 *    barriers, and temporaries go to global memory only where another tile or sub-chain reads
 *    them.  slt_inspect fails with SLT_ERR_UNSUPPORTED when a tile's footprint exceeds the
 *    shared memory of one CTA (about 470 cells at p = 2, 180 at p = 4: use a smaller tile size).
 * The dataflow executors synchronise the stream before returning (they read their error flag);
 * the untiled and colour-phase executors return after queueing their launches on `stream`.
 * Results are bit-identical across the four executors for one schedule (the same per-cell
 * arithmetic in the same order), and to the untiled chain where a tile holds the whole mesh.
 * Work buffers are owned by the mesh. */
int slt_execute(slt_mesh mesh, slt_schedule sched, double* v, double* sigma, const double* ricker,
                double dt, int64_t nsteps, void* stream);
/* slt_execute that also times every kernel launch with CUDA events recorded on `stream` and
   synchronises before returning.  profile[0] = total ms of the chain kernels (with a dataflow
   executor: its persistent kernel alone), [1] their number of kernel launches, [2] ms of the
   layout kernels (caller <-> work layout), [3] their launches, [4] longest and [5] shortest
   timed chain interval in ms, [6] ms of the dataflow executor's queue set-up kernels (counter
   reset and seeding) and [7] their launches (0 without a dataflow executor).  Not thread-safe:
   one profiled call at a time per process. */
int slt_execute_profiled(slt_mesh mesh, slt_schedule sched, double* v, double* sigma, const double* ricker,
                         double dt, int64_t nsteps, void* stream, double profile[8]);
/* The same with HOST fields and source series (page-locked memory lets the copies run
   asynchronously): copies in, runs, copies out, synchronises.  The fields cross the host link in
   four chunks of cells on a private copy stream, and each chunk is converted into (out of) the
   work layout while the next one is on the link. */
int slt_execute_host(slt_mesh mesh, slt_schedule sched, double* host_v, double* host_sigma,
                     const double* host_ricker, double dt, int64_t nsteps, void* stream);
/* Many shots of the same mesh and material at once (the batched form): nshots runs with their
   own point sources src_xy [nshots][2] (host; NULL = no source), sharing the Ricker series.
   Fields are device arrays with the shots innermost: v [ncell][2][Np][nshots],
   sigma [ncell][3][Np][nshots], updated in place.  Each (cell, shot) computes exactly what a
   single-field run of that shot computes.  sched = NULL: untiled chain (6 launches per step,
   one thread per cell and shot); otherwise the dataflow executor, each tile's items expanded
   over the shots, in slices of the schedule's shots_per_cta (one persistent launch per slice).
   profile (NULL = none) as in slt_execute_profiled.  Synchronises.  Work memory: 15 Np ncell
   nshots doubles, kept by the mesh.  SLT_ERR_ARG for nshots outside 1..4096, a non-finite dt or
   a source outside the mesh; SLT_ERR_UNSUPPORTED when the schedule's executor is not 0;
   SLT_ERR_STATE for a schedule of another mesh. */
int slt_execute_batched(slt_mesh mesh, slt_schedule sched, int32_t nshots, const double* src_xy, double* v,
                        double* sigma, const double* ricker, double dt, int64_t nsteps, void* stream,
                        double* profile);
/* Several independent meshes (uneven sizes, any degrees) advanced together: the batched form
   over uneven meshes.  slt_group_create binds meshes[i] to scheds[i] (NULL = untiled; a schedule
   must come from its mesh's chain; a mesh may appear once; n in 1..256) and builds, for each
   degree, one combined dataflow plan over the tiled meshes of that degree: the disjoint union
   of their dependency graphs, tiles renumbered by a base per mesh.  slt_group_execute advances
   every mesh i by nsteps steps on its own device fields v[i], sigma[i] (caller layout), with
   source series ricker[i] (device, may be NULL) and time step dt[i] (host arrays of length n):
   one persistent kernel per degree runs the tiles of all its meshes from one ready queue
   (per-mesh dependency counters, no barrier across meshes), the degrees one after the other;
   untiled meshes run side by side on private streams forked from `stream`.  Synchronises;
   SLT_ERR_TIMEOUT if a wait gave up.  The meshes and schedules must outlive the group.
   Errors: SLT_ERR_ARG for n outside 1..256, a null or repeated mesh, a null field or a
   non-finite dt; SLT_ERR_STATE for a schedule of another mesh; SLT_ERR_UNSUPPORTED when tiled
   meshes of one degree use different CTA sizes.  slt_execute_many = create, execute once,
   destroy. */
int slt_group_create(int32_t n, const slt_mesh* meshes, const slt_schedule* scheds, slt_group* out);
/* The batched form in one persistent launch: as slt_group_create, with member i carrying
   nshots[i] shots (1 = one field; several: fields [cell][comp][node][shot] in
   slt_group_execute, sources at host src_xy[i] [nshots[i]][2], src_xy or src_xy[i] NULL = no
   sources; such a member needs a dataflow-executor schedule).  Every tiled member, whatever its
   degree (1-3) and layout, runs from one ready queue in one persistent kernel; the conversion of
   the fields into the work layout and back, the queue reset and seeding and the kernel are
   captured as one CUDA graph on the first slt_group_execute and replayed while nsteps and the
   field pointers stay the same (the source series and time steps may change between calls).
   Untiled members run after it.  SLT_ERR_UNSUPPORTED for a tiled member of degree 4 or with
   other than 256-thread tiles, or a member with several shots and no such schedule.
   slt_group_graph_replays: how often the group's cached graph has been launched since it was
   (re)captured. */
int slt_group_create_batched(int32_t n, const slt_mesh* meshes, const slt_schedule* scheds, const int32_t* nshots,
                             const double* const* src_xy, slt_group* out);
int slt_group_graph_replays(slt_group group, int64_t* replays);
int slt_group_destroy(slt_group group);
int slt_group_execute(slt_group group, double* const* v, double* const* sigma, const double* const* ricker,
                      const double* dt, int64_t nsteps, void* stream);
int slt_execute_many(int32_t n, const slt_mesh* meshes, const slt_schedule* scheds, double* const* v,
                     double* const* sigma, const double* const* ricker, const double* dt, int64_t nsteps,
                     void* stream);
/* Autotuner over tile size, tile shape, CTA size and shots per CTA (Section 7.3 searches tile
   size and shape empirically).  Times the untiled chain, then every candidate (tile_sizes[i],
   renumber, block_threads[b], shots_per_cta[k]): renumber 1 (Hilbert tiles) only, or also 0
   (chunks of the mesh numbering) when shapes != 0; the shots-per-CTA candidates apply to
   nshots > 1 (ngroup = 0 or nshots = 1: one candidate, all shots).  Each candidate is inspected
   with `base` for every other option (split points, executor ...), run 2 untimed steps and
   `steps` timed steps (CUDA events around the executor kernels) with zero fields and no source,
   nshots = 1: the single-field executor, nshots > 1: the multi-shot executor.  A candidate
   whose colouring fell back to sequential (its tiles would run one after another) is not
   timed: its row holds ms = -1.  *best = base with the fastest candidate's tile_size,
   renumber, block_threads and shots_per_cta; best->tile_size = 0 when the untiled chain was
   fastest.  table (host, may be NULL): rows (tile_size, renumber, block_threads, shots_per_cta,
   ms per step), the untiled chain first (0, 0, 0, 0, ms); 1 + ntile * (shapes ? 2 : 1) *
   nblock * max(ngroup, 1) rows (ngroup counted as 1 when nshots = 1).  Allocates the candidate
   fields (5 Np ncell nshots doubles) for the call; synchronises.  SLT_ERR_ARG for nshots outside
   1..4096, 0..64 tile sizes, 1..4 CTA sizes (each 128, 256 or 384), 0..16 shot counts, steps
   outside 1..1000, or nshots > 1 with an executor other than 0. */
int slt_autotune(slt_mesh mesh, const slt_options* base, int32_t nshots, const int32_t* tile_sizes,
                 int32_t ntile, int32_t shapes, const int32_t* block_threads, int32_t nblock,
                 const int32_t* shots_per_cta, int32_t ngroup, int32_t steps, void* stream, slt_options* best,
                 double* table);
/* Apply one operator once (for tests): op 0 = A (stress -> velocity rate, device
   in [ncell][3][Np], out [ncell][2][Np]); op 1 = B (velocity -> stress rate, in [ncell][2][Np],
   out [ncell][3][Np]).  Runs the untiled phase kernels of that operator (A: loops 0-2 of the chain;
   B: loops 3-5, whose Hooke step gives C E(v)).  Queued on `stream`; SLT_ERR_ARG for an op other
   than 0 or 1 or a null pointer. */
int slt_apply_operator(slt_mesh mesh, int32_t op, const double* in, double* out, void* stream);

/* ------------------------------------------------------------------ misfit and gradient
 * An extension of the paper's forward chain: the gradient of a seismogram misfit
 * with respect to per-cell rho, lambda, mu by the discrete adjoint of the time step.
 *
 * Replace the material (host arrays, caller numbering; mu > 0, lambda + mu > 0, rho > 0) or
 * the point source (NULL: none) of a mesh without rebuilding it; both synchronise `stream`. */
int slt_mesh_set_material(slt_mesh mesh, const double* rho, const double* lam, const double* mu, void* stream);
int slt_mesh_set_source(slt_mesh mesh, const double* src_xy, void* stream);
/* nrec point receivers at host positions xy [nrec][2] (each in some cell: the smallest cell id
   containing it); the velocity there is the DG field evaluated at the point. */
int slt_receivers_create(slt_mesh mesh, int32_t nrec, const double* host_xy, slt_receivers* out);
int slt_receivers_destroy(slt_receivers rec);
/* Run nsteps from rest (v = sigma = 0) and record traces [nsteps][nrec][2] (device) =
   velocity at every receiver at t_{n+1/2}.  sched as in slt_execute (NULL = untiled); the
   steps are executed one call at a time, so with the dataflow executor each step is one
   persistent launch (no overlap between steps) and the untiled chain is usually faster. */
int slt_record(slt_mesh mesh, slt_schedule sched, slt_receivers rec, const double* ricker, double dt,
               int64_t nsteps, double* traces, void* stream);
/* Misfit J = 1/2 dt sum_n sum_r |trace - data|^2 (data: device [nsteps][nrec][2]) of a run
   from rest, written to *misfit (host), and its gradient grad (device [3][ncell], caller
   numbering: d/drho, d/dlambda, d/dmu) by the discrete adjoint: the forward run (with sched's
   executor) keeps (v, sigma) every checkpoint_every = k steps (nsteps / k states); each segment
   is recomputed forward by the untiled loops, which leave the operator intermediates of every
   step (A sigma, E(A sigma), ABA sigma, E(v), AB v, E(AB v): 15 Np ncell doubles per step, k
   steps) for the backward sweep to read; with checkpoint_every = -k, or when that memory cannot
   be allocated, the segment keeps only its k states (5 Np ncell doubles each) and the backward
   sweep recomputes the intermediates (about 1.3x the time).  Synchronises.
   Uses the mesh's current material and source. */
int slt_adjoint(slt_mesh mesh, slt_schedule sched, slt_receivers rec, const double* ricker, double dt,
                int64_t nsteps, const double* data, int32_t checkpoint_every, double* grad, double* misfit,
                void* stream);
/* Many shots at once (Section 7.1's explosive source, one per shot; the shots of the batched
   form, fields with the shots innermost), untiled (sched = NULL) or on the tiles of an executor-0
   schedule with the {velocity, stress} fusion (split at loop 9; SLT_ERR_UNSUPPORTED otherwise).
   src_xy: host [nshots][2] source points (NULL: no sources); traces and data are device arrays
   [nsteps][nshots][nrec][2].  slt_record_batched records the traces of runs from rest.
   slt_adjoint_batched returns J = sum over the shots of the single-shot misfit and its gradient
   grad [3][ncell] (device, caller numbering, summed over the shots), by the discrete adjoint:
   the forward run keeps (v, sigma) every checkpoint_every = k >= 1 steps; each segment is
   recomputed one sub-chain at a time with every step's operator intermediates written to a keep
   slot (15 Np ncell nshots doubles per step, k steps); the reverse sweep runs, per step, the
   velocity sub-chain on the adjoint variables with -dt, the stress-update gradient terms, the
   receiver residuals, the stress sub-chain with -dt and the velocity-update gradient terms - the
   adjoint step is the same loop chain (the skew identity), so the forward schedule's tiles serve
   it as they are.  Synchronises.  slt_adjoint with such a schedule and checkpoint_every > 0 runs
   its single shot the same way. */
int slt_record_batched(slt_mesh mesh, slt_schedule sched, slt_receivers rec, int32_t nshots, const double* src_xy,
                       const double* ricker, double dt, int64_t nsteps, double* traces, void* stream);
int slt_adjoint_batched(slt_mesh mesh, slt_schedule sched, slt_receivers rec, int32_t nshots, const double* src_xy,
                        const double* ricker, double dt, int64_t nsteps, const double* data, int32_t checkpoint_every,
                        double* grad, double* misfit, void* stream);

/* ------------------------------------------------------------------ FP64 peak probe
 * The paper has no counterpart: it measures the arithmetic roof of this library's kernels on the
 * current GPU (the chain is FP64 arithmetic, and the driver's measured peaks cover only an HBM
 * copy and a bf16 GEMM).  Runs three probe kernels on `stream` (8 blocks of 256 threads per SM,
 * one warm-up launch each, CUDA-event timing) and synchronises:
 * out[0] = FP64 fused multiply-add throughput (TFLOP/s, an FMA counts 2: 8 independent chains
 * per thread), out[1] = FP64 warp-level tensor throughput (mma.sync.m8n8k4.f64, 512 flop per
 * instruction; 4 independent accumulators per warp), out[2] = both issued at once (half the warps
 * each, equal flops), out[3] = total ms of the three timed launches.  Allocates nothing. */
int slt_fp64_peak(void* stream, double out[4]);
/* How the FP64 pipe treats partial and few warps (the paper has no counterpart; the executors'
   design rests on these two facts): DFMA warp instructions per clock per SM (maximum clock) with
   out[0] 32 active lanes per warp, out[1] 16 active lanes, out[2] one warp per SM, out[3] four
   warps per SM.  Allocates nothing; synchronises. */
int slt_fp64_lane_probe(void* stream, double out[4]);
/* The volume contraction of the multi-shot form on the FP64 tensor instruction (the paper has no
   counterpart: it measures whether the [dof][shot] layout's small dense products pay on the
   warp-level FP64 tensor path, mma.sync.m8n8k4, which shares the pipe of DFMA).  For ncell cells
   of degree `degree` and nshots shots (a multiple of 8), U[cell][Np][shot] = W X[cell] with
   W = [Dr Ds] (Np x 2Np) and X[cell] a 2Np x nshots block of seeded values, computed twice on
   `stream`: (a) one thread per (cell, shot) with DFMA, the structural zeros of Dr and Ds skipped
   (as the executors do), (b) one warp per cell with m8n8k4 tiles (W zero-padded to multiples of
   8 rows and 4 columns).  out[0], out[1] = ms of (a) and (b) (CUDA events, second of two runs),
   out[2] = max |Ua - Ub| / max |Ua|, out[3] = useful flops (2 nnz ncell nshots), out[4] = flops
   the tensor form issues, out[5] = nnz of [Dr Ds].  Allocates (4 Np doubles per cell and shot,
   at most 32 GB; SLT_ERR_ARG beyond) and synchronises. */
int slt_fp64_contraction_probe(int32_t degree, int64_t ncell, int32_t nshots, void* stream, double out[6]);

/* ------------------------------------------------------------------ allocation-free ranking
 * The paper has no counterpart to this entry point: it serves callers who cannot allocate
 * device memory where they need the seed ordering (a framework that owns every allocation
 * through its own pool, or code where cudaMalloc would synchronise the device or is not
 * permitted).  It computes exactly the rank array of slt_inspect's Hilbert partition
 * (renumber = 1) for n points d_xy [n][2] (device, doubles) into d_rank [n] (device, int32),
 * asynchronously on `stream`, and allocates nothing: its scratch is one fixed device array of
 * 17.8 MB (17,826,560 bytes), held by every GPU that loads the library until the process exits.
 *  - n may not exceed 1,048,576 (SLT_ERR_ARG otherwise, nothing launched).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.  Every later call
 *    made outside stream capture looks it up again, so the address stays right after a
 *    cudaDeviceReset (which reloads the module).
 *  - All calls share the array: calls whose GPU work overlaps (different streams or host
 *    threads without ordering) race and give wrong ranks; order them on one stream. */
int slt_seed_rank_noalloc(const double* d_xy, int64_t n, int32_t* d_rank, void* stream);

#ifdef __cplusplus
}
#endif
#endif
