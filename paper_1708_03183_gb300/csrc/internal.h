// Internal declarations shared by the translation units of libslt.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "slt.h"

namespace slt {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
struct Error {
  int code;
  std::string msg;
};
// throw inside the library; every entry point catches and converts to a status
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define SLT_CUDA(x) ::slt::check_cuda((x), #x)

// ---------------------------------------------------------------- device buffer
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count == 0) return;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; n = 0; (void)cudaGetLastError(); fail(SLT_ERR_OOM, "cudaMalloc failed"); }
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void upload(const T* host, size_t count, cudaStream_t s) {
    if (count) SLT_CUDA(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s, size_t count = (size_t)-1) const {
    if (count == (size_t)-1) count = n;
    std::vector<T> h(count);
    if (count) SLT_CUDA(cudaMemcpyAsync(h.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    SLT_CUDA(cudaStreamSynchronize(s));
    return h;
  }
};

// ---------------------------------------------------------------- loop chain (host)
struct MapH {
  int32_t from, to, arity;
  std::vector<int32_t> values;
};
struct DescH {
  int32_t map;
  char mode;
};
struct LoopH {
  int32_t set;
  std::vector<DescH> descs;
  int32_t kernel;  // executor kernel id (elastic chains), -1 otherwise
};

struct Mesh;

}  // namespace slt

struct slt_chain_s {
  std::vector<int64_t> set_size;
  std::vector<slt::MapH> maps;
  std::vector<slt::LoopH> loops;
  std::vector<std::vector<double>> points;  // per set, empty when none
  slt_mesh mesh = nullptr;                  // set when built by slt_mesh_chain
};

namespace slt {

// executor kernel ids of the elastic chain loops
enum LoopKind : int32_t {
  K_VOLB = 0, K_INTB = 1, K_EXTB = 2, K_VOLD = 3, K_INTD = 4, K_HOOKEB = 5, K_UPDV = 6, K_UPDS = 7
};
// which field buffers each loop of the seventeen uses is fixed by its position (exec.cu)

#ifdef __CUDACC__
#define SLT_HD __host__ __device__
#else
#define SLT_HD
#endif

// The chain in six phases: runs of consecutive loops in which no thread reads a value another
// thread writes during the run.  phase_first(h) is the first loop of phase h (phase_first(6) = 17):
//   0: loops 0-2    A(S) -> U1 (volume, interior faces, free surface)
//   1: loops 3-5    E(U1) -> E, then S1 = C E and the volume part of A(S1) -> U2
//   2: loops 6-8    faces of A(S1) onto U2, then V += dt (U1 + dt^2/24 U2)
//   3: loops 9-11   E(V) -> E, then S1 = C E and the volume part of A(S1) -> U1
//   4: loops 12-13  faces of A(S1) onto U1
//   5: loops 14-16  E(U1) -> E, then S += dt (S1 + dt^2/24 C E) + source
// The neighbour values read inside a phase (S in 0, U1 in 1 and 5, S1 in 2 and 4, V in 3) are all
// written by an earlier phase.
SLT_HD constexpr int phase_first(int h) {
  return h == 0 ? 0 : h == 1 ? 3 : h == 2 ? 6 : h == 3 ? 9 : h == 4 ? 12 : h == 5 ? 14 : 17;
}
constexpr int kPhases = 6;
SLT_HD constexpr int phase_of(int J) {
  return J < 3 ? 0 : J < 6 ? 1 : J < 9 ? 2 : J < 12 ? 3 : J < 14 ? 4 : 5;
}
// loops over cells (the others run over interior or free-surface facets)
SLT_HD constexpr bool is_cell_loop(int J) {
  return J == 0 || J == 3 || J == 5 || J == 8 || J == 9 || J == 11 || J == 14 || J == 16;
}
// A segment is the part of a phase inside one sub-chain [first, last): the tiled executors run a
// tile's segments in order with one barrier after each.  The segment starting at loop J ends here.
SLT_HD constexpr int seg_end(int J, int last) {
  return phase_first(phase_of(J) + 1) < last ? phase_first(phase_of(J) + 1) : last;
}

// ---------------------------------------------------------------- primitives (sort.cu)
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key; tmp buffers of
// size n.  keys/vals are replaced by the sorted sequence.
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, uint32_t* tkeys,
                      uint32_t* tvals, cudaStream_t s);
// out[i] = sum_{k<i} in[k] for i < n, out[n] = total (out has n + 1 entries)
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
// offs[k] = first position p with sorted[p] >= k, for k = 0..nkeys (offs has nkeys + 1 entries)
void lower_bound_offsets(const uint32_t* sorted, int64_t n, int64_t nkeys, int32_t* offs, cudaStream_t s);
int bits_for(int64_t maxval);  // number of bits to represent values in [0, maxval]

// The same steps over caller-provided scratch (no allocation, no synchronisation).
void launch_bbox_init(unsigned long long* box, cudaStream_t s);
void launch_bbox(const double* xy, int64_t n, unsigned long long* box, cudaStream_t s);
void launch_hilbert_keys(const double* xy, int64_t n, const unsigned long long* box, uint32_t* keys,
                         uint32_t* vals, cudaStream_t s);
void launch_rank_from_order(const uint32_t* order, int64_t n, int32_t* rank, cudaStream_t s);
int radix_blocks(int64_t n);  // blocks of one radix pass; hist/offs need 256 * blocks (+1) ints
void radix_sort_pairs_with(uint32_t* keys, uint32_t* vals, int64_t n, int bits, uint32_t* tkeys,
                           uint32_t* tvals, int32_t* hist, int32_t* offs, cudaStream_t s);

// Seed ranks (identity or Hilbert order of points) on the device.
void seed_rank(const double* d_xy, int64_t n, int renumber, int32_t* d_rank, cudaStream_t s);

// ---------------------------------------------------------------- schedule
struct LocalMap {
  DevBuf<int32_t> fp_ptr, fp, lmap;
};
struct SubSched {
  int32_t first = 0, last = 0;
  int32_t seed = 0;  // seed loop relative to first (> 0: backward tiling before it)
  int32_t m = 0, ncolours = 0;
  int64_t restarts = 0, fell_back = 0, conflicts = 0, unprojected = 0;
  DevBuf<int32_t> rank, colour;
  std::vector<DevBuf<int32_t>> sigma, list_ptr, list;  // per loop of the sub-chain
  std::vector<std::vector<LocalMap>> lmaps;            // per loop, per descriptor
  // executor plan (elastic chains only)
  std::vector<int32_t> colour_ptr;                     // host, ncolours + 1
  DevBuf<int32_t> tiles_by_colour;
  std::vector<DevBuf<int32_t>> plan_ptr, plan_items;   // per segment, at its first loop (others empty)
  // staged executor (executor 3): each tile's footprint (the cells its segments touch, ascending
  // work id, slot = position), per segment seven lists of slot entries (see stage_build)
  DevBuf<int32_t> fp_ptr, fp_cell, fp_nsl;             // [m + 1]; work id | shared << 31; neighbour slots
  std::vector<DevBuf<int32_t>> st_off, st_ent;         // per segment: [7 m + 1] list offsets, entries
  int32_t max_fp = 0;                                  // largest footprint
};
// the seven lists of a segment of a tile, in the order the staged executor runs them
enum StageList : int32_t { SL_GATHER = 0, SL_INIT, SL_INT0, SL_INT1, SL_INT2, SL_EXT, SL_PB, SL_N };
// footprint slots: 0 .. kNoSlot - 2 a cell of the tile's footprint, kNoSlot - 1 a neighbour outside
// it, kNoSlot a free surface; three of them (a cell's face neighbours) share one 32-bit word
constexpr int32_t kSlotBits = 10, kNoSlot = (1 << kSlotBits) - 1;
// item flags of the staged lists: faces (3 bits), first cell loop (8), later cell loop (16), and
// 32 = the accumulated value starts from global memory (contributions made by another tile)
constexpr int32_t kLoadBit = 32;

}  // namespace slt

namespace slt {
// dependencies of the persistent dataflow executor (elastic chains)
struct DataflowPlan {
  std::vector<int32_t> cum;          // global tile id base per sub-chain, size nsub + 1
  DevBuf<int32_t> succ_ptr, succ;    // CSR over global tiles: (global tile << 1) | next step
  DevBuf<int32_t> indeg0, indeg;     // dependencies of a tile's first-step node / later nodes
  DevBuf<int32_t> indeg_sub;         // same-step dependencies inside the tile's own sub-chain
  DevBuf<int32_t> pending, queue;    // per run: [nsteps * tiles]
  DevBuf<unsigned long long> head;   // head, tail
  DevBuf<int32_t> err;
  int64_t ndeps = 0;
  // longest dependency chain per time step in the steady state, in nodes (each node counted once)
  // and in plan items (each node weighted by its items); items of all nodes of one step
  double cp_nodes = 0, cp_items = 0, items_per_step = 0;
  int64_t last_grid = 0;             // tiles in flight (CTAs or clusters) of the last launch
};
}  // namespace slt

struct slt_schedule_s {
  int32_t executor = 0;              // 0 dataflow, 1 colour phases, 2 dataflow with tile clusters, 3 staged,
                                     // 4 dataflow with compacted passes
  int32_t keep = 1;                  // dataflow: a CTA runs the first successor its tile released
  int32_t stage_cross = 0;           // staged: temporaries cross sub-chains, so every one is written out
  int32_t block = 256;               // threads per tile CTA (128, 256 or 384)
  int32_t shots_per_cta = 0;         // multi-shot dataflow runs: shots per queue pass (0 = all)
  int32_t cluster = 8;               // executor 2: CTAs per tile cluster
  slt::DevBuf<long long> df_slot;    // executor 2: node handed from each cluster's leader
  std::vector<slt::DevBuf<int32_t>> dmaps;  // device copies of the chain's maps (local maps on request)
  int64_t wait_spins = 1ll << 24;    // bounded dependency wait of the dataflow executor
  slt::DataflowPlan df;
  std::vector<slt::LoopH> loops;     // copy of the chain's loops
  std::vector<slt::MapH> maps_meta;  // from, to, arity (values not kept)
  std::vector<int64_t> set_size;
  slt_mesh mesh = nullptr;
  std::vector<slt::SubSched> subs;
  // seconds of slt_inspect per stage: seed partition, colouring with projections, tiling and
  // conflict repair (Algorithms 1-3), iteration lists and local maps, executor plans, staged
  // plans, dependency graph, (unused)
  double insp_s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace slt {

// ---------------------------------------------------------------- elastic mesh
struct RefElem {
  int p = 0, Np = 0, Nfp = 0;
  std::vector<double> nodes;  // [Np][2]
  std::vector<double> Dr, Ds; // [Np][Np], Dr[i*Np+j] = d phi_j / dr at node i
  std::vector<double> Minv;   // [Np][Np]
  std::vector<double> Lift;   // [3][Np][Nfp]
  std::vector<int> fnode;     // [3][Nfp]
  std::vector<double> Vinv;   // monomial coefficients of the basis
  std::vector<int> mono;      // [nmono][2]
  std::vector<double> eval(double r, double s) const;
};
RefElem make_refelem(int p);

}  // namespace slt

struct slt_mesh_s {
  int64_t nc = 0, ncp = 0;  // cells, padded stride
  int p = 0, Np = 0, Nfp = 0;
  int64_t nfi = 0, nfe = 0;
  slt::RefElem ref;
  // host topology in the caller's numbering (for the chain)
  std::vector<int32_t> f2c, e2c;      // [nfi][2], [nfe]
  std::vector<int8_t> f2f, e2f;       // local face of each side, [nfi][2], [nfe]
  std::vector<double> centroid;       // [nc][2]
  std::vector<double> fmid, emid;     // facet midpoints [nfi][2], [nfe][2]
  std::vector<int32_t> perm, iperm;   // work id -> cell, cell -> work id
  std::vector<double> affine;         // [nc][7]: x0, y0, rx, ry, sx, sy, |det J| (caller numbering)
  int64_t src_cell = -1;              // caller numbering
  int64_t cells_int = 0, cells_ext = 0;  // cells with an interior / exterior face
  // device, work layout (SoA, stride ncp)
  slt::DevBuf<double> geo, fgeo, mat, src;
  slt::DevBuf<double> pre;          // products of geometry and material hoisted out of the loops
  slt::DevBuf<int32_t> nbr, d_perm, d_iperm;
  int32_t src_w = -1;
  // work fields: V[2 Np], S[3 Np], U1[2 Np], U2[2 Np], E[3 Np], S1[3 Np] rows of ncp
  slt::DevBuf<double> work;
  slt::DevBuf<double> ricker_buf;   // for host-buffer execution
  slt::DevBuf<double> io_v, io_s;
  slt::DevBuf<double> adet;         // |det J| per cell, work order
  slt::DevBuf<double> work_b, bsrc;  // multi-shot work fields; per-shot source coefficients
  slt::DevBuf<int32_t> bsrc_w;       // per-shot source cell (work id, -1 = none)
  slt::DevBuf<long long> step_dev;   // step counter read by graph-captured untiled steps
  cudaStream_t capture = nullptr;    // private stream the untiled step is captured on
  cudaStream_t copy = nullptr;       // private stream of the host-field copies (slt_execute_host)
  ~slt_mesh_s() {
    if (capture) cudaStreamDestroy(capture);
    if (copy) cudaStreamDestroy(copy);
  }
};

// A group of meshes advanced together.  The tiled meshes of each degree share one combined
// dataflow plan (the disjoint union of their dependency graphs, tiles renumbered by a base per
// mesh), run by one persistent kernel; untiled meshes run side by side on private streams.
struct slt_group_s {
  struct Part {
    int p = 0, block = 256;
    int64_t wait_spins = 0;
    int32_t keep = 1;
    std::vector<int32_t> members;            // indices into meshes
    int32_t G = 0, K = 0;
    slt::DevBuf<int32_t> cum, first, last, mesh_of;   // (mesh, sub-chain) table
    slt::DevBuf<int32_t> succ_ptr, succ, indeg0, indeg, pending, queue, err;
    slt::DevBuf<unsigned long long> head;
    slt::DevBuf<unsigned char> params;       // per member: the executor's parameter block
  };
  std::vector<slt_mesh> meshes;
  std::vector<slt_schedule> scheds;
  std::vector<Part> parts;
  std::vector<int32_t> untiled;
  // one launch over all degrees (slt_group_create_batched): members with several shots (fields
  // with the shots innermost) and their sources; the tiled part captured as a CUDA graph,
  // replayed while the step count and the field pointers stay the same
  bool mixed = false;
  std::vector<int32_t> nshots;                 // per member (1 = one field)
  std::vector<slt::DevBuf<int32_t>> src_w;     // per member: source cell of every shot (work id)
  std::vector<slt::DevBuf<double>> src;        // per member: source coefficients [S][Np]
  cudaGraphExec_t graph = nullptr;
  std::vector<const void*> graph_key;
  cudaStream_t capture = nullptr;
  int64_t graph_launches = 0;                  // replays of the cached graph (for tests)
  ~slt_group_s() {
    if (graph) cudaGraphExecDestroy(graph);
    if (capture) cudaStreamDestroy(capture);
  }
};

struct slt_receivers_s {
  slt_mesh mesh = nullptr;
  int32_t n = 0;
  slt::DevBuf<int32_t> w;           // work id of the receiver's cell
  slt::DevBuf<double> phi, q;       // basis values at the receiver; M_hat^-1 phi / |det J|
};

namespace slt {
// exec.cu
void upload_constants(const RefElem& r);
// the mesh's hoisted per-cell products (pre) from its geometry and material, on s
void build_pre(slt_mesh m, cudaStream_t s);
void exec_run(slt_mesh m, slt_schedule sched, double* v, double* sigma, const double* ricker, double dt,
              int64_t nsteps, cudaStream_t s, double* profile = nullptr);
// the same with host fields and source series: copies overlapped with the layout conversion
void exec_run_host(slt_mesh m, slt_schedule sched, double* hv, double* hs, const double* hr, double dt,
                   int64_t nsteps, cudaStream_t s);
void group_build(slt_group g);
void group_run(slt_group g, double* const* v, double* const* sigma, const double* const* ricker, const double* dt,
               int64_t nsteps, cudaStream_t s);
void exec_apply(slt_mesh m, int op, const double* in, double* out, cudaStream_t s);
// time steps on the mesh's work buffers V, S (work layout), source series entry step0 + n
void exec_steps_work(slt_mesh m, slt_schedule sched, const double* ricker, double dt, int64_t step0,
                     int64_t nsteps, cudaStream_t s);
// A: stress-like [3Np][ncp] -> velocity rate [2Np][ncp]; E: velocity-like -> strain [3Np][ncp]
void exec_step_keep(slt_mesh m, const double* ricker, double dt, int64_t step, double* keep, cudaStream_t s);
void op_A(slt_mesh m, const double* in3, double* out2, cudaStream_t s);
void op_E(slt_mesh m, const double* in2, double* out3, cudaStream_t s);
// exec_batched.cu
void upload_constants_batched(const RefElem& r);
// One part of one time step on a multi-shot work layout (S shots; every buffer rows of ncp * S
// doubles, column cell * S + shot): part 0 the velocity sub-chain (loops 0-8), 1 the stress
// sub-chain (9-16), 2 the whole step.  Untiled when sched is null, else the dataflow executor (a
// part alone needs a {velocity, stress} schedule).  Synchronises when tiled.
struct ChainRun {
  int32_t S = 1;
  double* buf[6] = {};          // V, S, U1, U2, E, S1
  double* e5 = nullptr;         // where phase 5 leaves its strain (null: buf[4])
  const double* ricker = nullptr;  // source series at this step, or null (no source)
  double dt = 0;
  const int32_t* src_w = nullptr;  // [S] source cell of each shot (work id, -1 none), device
  const double* src = nullptr;     // [S][Np] source coefficients, device
};
void chain_part_b(slt_mesh m, slt_schedule sched, const ChainRun& r, int part, cudaStream_t s);
void exec_run_batched(slt_mesh m, slt_schedule sched, int32_t S, const int32_t* d_src_w, const double* d_src,
                      double* v, double* sigma, const double* ricker, double dt, int64_t nsteps, cudaStream_t s,
                      double* profile);
// tune.cpp
void autotune(slt_mesh m, const slt_options& base, int32_t nshots, const int32_t* tile_sizes, int32_t ntile,
              int32_t shapes, const int32_t* blocks, int32_t nblock, const int32_t* groups, int32_t ngroup,
              int32_t steps, cudaStream_t s, slt_options* best, double* table);
// adjoint.cu
void upload_adjoint_constants(const RefElem& r);
void record_run(slt_mesh m, slt_schedule sched, slt_receivers rec, const double* ricker, double dt, int64_t nsteps,
                double* traces, cudaStream_t s);
void adjoint_run(slt_mesh m, slt_schedule sched, slt_receivers rec, const double* ricker, double dt, int64_t N,
                 const double* data, int32_t k, double* grad_out, double* J_host, cudaStream_t s);
// S shots (sources d_src_w [S], d_src [S][Np], device), untiled or tiled: traces / data are
// [nsteps][S][nrec][2]; the gradient is summed over the shots
void record_run_b(slt_mesh m, slt_schedule sched, slt_receivers rec, int32_t S, const int32_t* d_src_w,
                  const double* d_src, const double* ricker, double dt, int64_t nsteps, double* traces,
                  cudaStream_t s);
void adjoint_run_b(slt_mesh m, slt_schedule sched, slt_receivers rec, int32_t S, const int32_t* d_src_w,
                   const double* d_src, const double* ricker, double dt, int64_t N, const double* data, int32_t k,
                   double* grad_out, double* J_host, cudaStream_t s);
void build_plan(slt_schedule sched, slt_mesh m, SubSched& sub, cudaStream_t s);
void build_dataflow(slt_schedule sched, slt_mesh m, cudaStream_t s);
void stage_build(slt_schedule sched, slt_mesh m, SubSched& sub, cudaStream_t s);
int32_t stage_capacity(int p);  // slots of shared memory the staged executor has per tile CTA
// compute_local_maps of loop jj of sub-chain S, for the descriptors not built yet; synchronises s
void ensure_local_maps(slt_schedule sched, SubSched& S, int jj, cudaStream_t s);
// export flags of loop J (1 per iteration: an element it writes is touched by another tile of
// its sub-chain), into out (device); synchronises s
void export_flags(slt_schedule sched, int32_t J, DevBuf<int32_t>& out, cudaStream_t s);
// FP64 lane accounting of a schedule's plans (see slt_schedule_lane_info)
void lane_info(slt_schedule sched, slt_mesh m, double out[4]);
// inspect.cu
void inspect_chain(slt_chain c, const slt_options& opt, cudaStream_t s, slt_schedule out);
}  // namespace slt
