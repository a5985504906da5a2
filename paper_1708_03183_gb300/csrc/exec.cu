// Executor of the DG elastic loop chain (Section 5.2, Algorithm 4, shared-memory mode).
//
// One thread per cell for every phase.  Facet loops are executed as pulls: the thread of cell c
// applies the contributions of the facets of c that belong to the loop's iteration set (a
// 3-bit face mask per cell), so two threads never increment the same cell and no atomics
// are needed.  The reference matrices live in constant memory and every lane of a warp reads
// the same entry at the same time (warp-uniform operands); the face loop is unrolled so that
// the lifting matrix of face f is addressed with compile-time offsets.
//
// The chain of one time step (seventeen loops, buffers named as in the work layout):
//   velocity: 0 volB S->U1, 1 intB S,U1+, 2 extB S,U1+, 3 volD U1->E, 4 intD U1,E+,
//             5 hookeB E->S1 and volB S1->U2, 6 intB S1,U2+, 7 extB S1,U2+, 8 updV V+=dt(U1+c U2)
//   stress:   9 volD V->E, 10 intD V,E+, 11 hookeB E->S1 and volB S1->U1, 12 intB S1,U1+,
//             13 extB S1,U1+, 14 volD U1->E, 15 intD U1,E+, 16 updS S+=dt(S1+c C E)+source
// with c = dt^2/24: the fourth-order staggered Taylor leapfrog.  The executors run it as the six
// phases of internal.h (loops 0-2, 3-5, 6-8, 9-11, 12-13, 14-16), one thread per cell and phase.
//
// Operators in nodal strong form (the mass matrix cancels in the volume terms):
//   A sigma = (1/rho) div(sigma) - sum_f (F_f / 2 rho) Lift_f ((sigma - sigma_nb) n_f)
//             - sum_{exterior f} (F_f / rho) Lift_f (sigma n_f)
//   E(v)    = (dvx/dx, dvy/dy, dvx/dy + dvy/dx) - sum_f (F_f / 2) Lift_f sym((v - v_nb) (x) n_f)
//   B v     = C E(v),  C the isotropic Hooke law on (xx, yy, 2xy)
// with F_f = |face f| / |det J| and n_f the outward unit normal of face f.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "internal.h"
#include "refmask.h"  // generated: dr_nz(p, i), ds_nz(p, i) nonzero bits of row i

namespace slt {

namespace {

#include "exec_body.cuh"

// Untiled chain: the PARTS of phase H (consecutive loops, see phase_first) over every cell, one
// thread per cell.  (A grid-stride form would let the compiler hoist the reference-matrix entries
// out of its loop into registers, more than doubling the register count.)
template <int P, int H, int PARTS>
__global__ void __launch_bounds__(128) k_phase(Params a) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= a.nc) return;
  run_phase<P, H, PARTS, false>(a, w, 0, (H == 5 && a.step_dev) ? (int64_t)*a.step_dev : a.step);
}

// advances the device step counter at the end of a graph-captured step
__global__ void k_step_inc(long long* step) { *step += 1; }

#include "dataflow.cuh"
#include "staged.cuh"
#include "passes.cuh"
#include "layout.cuh"

// Tiled chain: one CTA per tile of one colour; the tile runs its slice of every segment of the
// sub-chain [first, last) in order, segments separated by a CTA barrier.
template <int P, int BS>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_tiled(Params a, int first, int last,
                                                                       const int32_t* __restrict__ tiles) {
  const int t = tiles[blockIdx.x];
  for (int J = first; J < last; J = seg_end(J, last)) {
    const int32_t b = a.plan_ptr[J][t], e = a.plan_ptr[J][t + 1];
    const int32_t* items = a.plan_items[J];
    const int H = phase_of(J);
    for (int32_t i = b + threadIdx.x; i < e; i += BS) run_seg<P, false, false>(a, H, items[i], a.step);
    __syncthreads();
  }
}

template <int P, int H, int PARTS>
void launch_phase(const Params& a, cudaStream_t s);

// parts (kPartA, kPartF, kPartB) of phase h among the loops [lo, hi)
inline int phase_parts(int h, int lo, int hi) {
  int parts = 0;
  for (int J = std::max(lo, phase_first(h)); J < std::min(hi, phase_first(h + 1)); ++J)
    parts |= !is_cell_loop(J) ? kPartF : J == phase_first(h) ? kPartA : kPartB;
  return parts;
}

// The untiled loops [first, last) of the chain as phases: whole phases, and the operator E alone
// (loops 3-4 of phase 1); other partial phases are not built.
template <int P>
void launch_untiled_range(const Params& a, int first, int last, cudaStream_t s) {
  for (int h = 0; h < kPhases; ++h) {
    const int parts = phase_parts(h, first, last);
    if (!parts) continue;
    if (parts == phase_parts(h, 0, 17)) {
      switch (h) {
        case 0: launch_phase<P, 0, kAllParts>(a, s); break;
        case 1: launch_phase<P, 1, kAllParts>(a, s); break;
        case 2: launch_phase<P, 2, kAllParts>(a, s); break;
        case 3: launch_phase<P, 3, kAllParts>(a, s); break;
        case 4: launch_phase<P, 4, kAllParts>(a, s); break;
        case 5: launch_phase<P, 5, kAllParts>(a, s); break;
      }
    } else if (h == 1 && parts == (kPartA | kPartF)) {
      launch_phase<P, 1, kPartA | kPartF>(a, s);
    } else {
      fail(SLT_ERR_UNSUPPORTED, "loop range does not align with the untiled phases");
    }
  }
  SLT_CUDA(cudaGetLastError());
}

template <int P>
void launch_tiled_colour(const Params& a, int first, int last, const int32_t* tiles, int ntiles, int bs,
                         cudaStream_t s);

// caller layout [cell][comp][Np] <-> work layout [comp*Np + node][ncp] in work order
__global__ void k_to_work(const double* __restrict__ in, int rows, const int32_t* __restrict__ perm, int64_t nc,
                          int64_t ncp, double* __restrict__ out) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nc; w += (int64_t)gridDim.x * blockDim.x) {
    const double* src = in + (int64_t)perm[w] * rows;
    for (int q = 0; q < rows; ++q) out[(int64_t)q * ncp + w] = src[q];
  }
}
__global__ void k_from_work(const double* __restrict__ in, int rows, const int32_t* __restrict__ perm, int64_t nc,
                            int64_t ncp, double* __restrict__ out) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nc; w += (int64_t)gridDim.x * blockDim.x) {
    double* dst = out + (int64_t)perm[w] * rows;
    for (int q = 0; q < rows; ++q) dst[q] = in[(int64_t)q * ncp + w];
  }
}

// Optional per-launch timing: events recorded on the launch stream around every kernel.
struct Recorder {
  std::vector<cudaEvent_t> ev;  // pairs (start, stop)
  std::vector<int> cls;         // 0 = chain kernel, 1 = layout kernel, 2 = dataflow queue set-up
  std::vector<int> nl;          // kernel launches inside each timed pair
  bool on = false;
  void begin(int c, cudaStream_t s, int launches = 1) {
    if (!on) return;
    nl.push_back(launches);
    cudaEvent_t a, b;
    SLT_CUDA(cudaEventCreate(&a));
    SLT_CUDA(cudaEventCreate(&b));
    ev.push_back(a);
    ev.push_back(b);
    cls.push_back(c);
    SLT_CUDA(cudaEventRecord(a, s));
  }
  void end(cudaStream_t s) {
    if (on) SLT_CUDA(cudaEventRecord(ev.back(), s));
  }
  void finish(cudaStream_t s, double* out) {
    if (!on) return;
    SLT_CUDA(cudaStreamSynchronize(s));
    double tot[3] = {0, 0, 0}, cnt[3] = {0, 0, 0}, mx = 0, mn = 1e300;
    for (size_t i = 0; i < cls.size(); ++i) {
      float ms = 0;
      SLT_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
      tot[cls[i]] += ms;
      cnt[cls[i]] += nl[i];
      if (cls[i] == 0) { mx = std::max(mx, (double)ms); mn = std::min(mn, (double)ms); }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    out[0] = tot[0]; out[1] = cnt[0]; out[2] = tot[1]; out[3] = cnt[1];
    out[4] = cnt[0] ? mx : 0; out[5] = cnt[0] ? mn : 0; out[6] = tot[2]; out[7] = cnt[2];
  }
};
Recorder g_rec;

Params make_params(slt_mesh m) {
  Params a{};
  a.ncp = m->ncp;
  a.nc = m->nc;
  a.geo = m->geo.p;
  a.fgeo = m->fgeo.p;
  a.mat = m->mat.p;
  a.nbr = m->nbr.p;
  a.pre = m->pre.p;
  const int64_t Np = m->Np, n = m->ncp;
  double* base = m->work.p;
  a.buf[B_V] = base;
  a.buf[B_S] = base + 2 * Np * n;
  a.buf[B_U1] = base + 5 * Np * n;
  a.buf[B_U2] = base + 7 * Np * n;
  a.buf[B_E] = base + 9 * Np * n;
  a.buf[B_S1] = base + 12 * Np * n;
  a.src = m->src.p;
  a.src_w = m->src_w;
  a.S = 1;
  a.fs = m->ncp;
  return a;
}

template <int P, int H, int PARTS>
void launch_phase(const Params& a, cudaStream_t s) {
  constexpr int threads = 128;
  const int64_t blocks = (a.nc + threads - 1) / threads;
  g_rec.begin(0, s);
  k_phase<P, H, PARTS><<<(unsigned)blocks, threads, 0, s>>>(a);
  g_rec.end(s);
}

template <int P>
void launch_tiled_colour(const Params& a, int first, int last, const int32_t* tiles, int ntiles, int bs,
                         cudaStream_t s) {
  if (ntiles <= 0) return;
  g_rec.begin(0, s);
  if (bs == 128) k_tiled<P, 128><<<ntiles, 128, 0, s>>>(a, first, last, tiles);
  else if (bs == 384) k_tiled<P, 384><<<ntiles, 384, 0, s>>>(a, first, last, tiles);
  else k_tiled<P, 256><<<ntiles, 256, 0, s>>>(a, first, last, tiles);
  g_rec.end(s);
  SLT_CUDA(cudaGetLastError());
}

void io_grid(int64_t n, int& g) {
  int64_t b = (n + 255) / 256;
  g = (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}

template <int P>
void run_dataflow(slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s) {
  launch_dataflow<P, false>(sched, a, nsteps, s, [&](int c, int n) { g_rec.begin(c, s, n); },
                            [&] { g_rec.end(s); });
}

// executor 2: one cluster of `sched->cluster` 256-thread CTAs per tile, as many clusters as fit
template <int P>
void run_dataflow_cluster(slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s) {
  DF df;
  if (!prepare_dataflow(sched, a, nsteps, s, df, [&](int c, int n) { g_rec.begin(c, s, n); },
                        [&] { g_rec.end(s); }))
    return;
  const int C = sched->cluster;
  auto kernel = k_dataflow_cluster<P, 256>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(256, 1, 1);
  cfg.gridDim = dim3(C, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  SLT_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, (void*)kernel, &cfg));
  if (nclusters < 1) fail(SLT_ERR_UNSUPPORTED, "no cluster of this size fits on the GPU");
  nclusters = (int)std::min<long long>(nclusters, df.q.total);
  sched->df.last_grid = nclusters;
  if (sched->df_slot.n < (size_t)nclusters) sched->df_slot.alloc(nclusters);
  cfg.gridDim = dim3((unsigned)(nclusters * C), 1, 1);
  g_rec.begin(0, s, 1);
  SLT_CUDA(cudaLaunchKernelEx(&cfg, kernel, a, df, sched->df_slot.p));
  g_rec.end(s);
  SLT_CUDA(cudaGetLastError());
  dataflow_check(sched, s);
}

// executor 3: the staged dataflow executor, one CTA per SM (as many as the shared memory of the
// largest tile footprint allows)
template <int P, int BS>
void launch_staged(slt_schedule sched, const Params& a, const DF& df, const StageArgs& g, cudaStream_t s) {
  auto kernel = k_staged<P, BS>;
  const int64_t bytes = stage_smem_bytes(P, g.cap);
  SLT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int dev = 0, nsm = 0, per = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, BS, (size_t)bytes));
  if (per < 1) fail(SLT_ERR_UNSUPPORTED, "the staged executor's tile CTA does not fit on an SM");
  const long long grid = std::min<long long>((long long)nsm * per, df.q.total);
  sched->df.last_grid = grid;
  g_rec.begin(0, s, 1);
  kernel<<<(unsigned)grid, BS, (size_t)bytes, s>>>(a, df, g);
  g_rec.end(s);
  SLT_CUDA(cudaGetLastError());
}

template <int P>
void run_staged(slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s) {
  DF df;
  if (!prepare_dataflow(sched, a, nsteps, s, df, [&](int c, int n) { g_rec.begin(c, s, n); },
                        [&] { g_rec.end(s); }))
    return;
  StageArgs g{};
  int32_t cap = 4;
  for (size_t k = 0; k < sched->subs.size(); ++k) {
    const SubSched& sub = sched->subs[k];
    cap = std::max(cap, sub.max_fp);
    g.fp_ptr[k] = sub.fp_ptr.p;
    g.fp_cell[k] = sub.fp_cell.p;
    g.fp_nsl[k] = sub.fp_nsl.p;
    for (int j = sub.first; j < sub.last; ++j) {
      g.off[j] = sub.st_off[j - sub.first].p;
      g.ent[j] = sub.st_ent[j - sub.first].p;
    }
  }
  g.cap = (cap + 3) / 4 * 4;
  g.cross = sched->stage_cross;
  switch (sched->block) {
    case 128: launch_staged<P, 128>(sched, a, df, g, s); break;
    case 384: launch_staged<P, 384>(sched, a, df, g, s); break;
    case 512: launch_staged<P, 512>(sched, a, df, g, s); break;
    case 768: launch_staged<P, 768>(sched, a, df, g, s); break;
    default: launch_staged<P, 256>(sched, a, df, g, s); break;
  }
  dataflow_check(sched, s);
}

// executor 4: the dataflow executor running each segment as compacted passes (k_passes)
template <int P>
void run_passes(slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s) {
  DF df;
  if (!prepare_dataflow(sched, a, nsteps, s, df, [&](int c, int n) { g_rec.begin(c, s, n); },
                        [&] { g_rec.end(s); }))
    return;
  StageArgs g{};
  for (size_t k = 0; k < sched->subs.size(); ++k) {
    const SubSched& sub = sched->subs[k];
    g.fp_ptr[k] = sub.fp_ptr.p;
    g.fp_cell[k] = sub.fp_cell.p;
    g.fp_nsl[k] = sub.fp_nsl.p;
    for (int j = sub.first; j < sub.last; ++j) {
      g.off[j] = sub.st_off[j - sub.first].p;
      g.ent[j] = sub.st_ent[j - sub.first].p;
    }
  }
  int dev = 0, nsm = 0, per = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto launch = [&](auto kernel, int threads) {
    SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0));
    const long long grid = std::min<long long>((long long)nsm * std::max(per, 1), df.q.total);
    sched->df.last_grid = grid;
    g_rec.begin(0, s, 1);
    kernel<<<(unsigned)grid, threads, 0, s>>>(a, df, g);
    g_rec.end(s);
  };
  if (sched->block == 128) launch(k_passes<P, 128>, 128);
  else if (sched->block == 384) launch(k_passes<P, 384>, 384);
  else launch(k_passes<P, 256>, 256);
  SLT_CUDA(cudaGetLastError());
  dataflow_check(sched, s);
}

// The untiled step as one CUDA graph (the 6 phase kernels and the step-counter increment), captured
// on the mesh's private stream and launched nsteps times on s: the host issues one launch per
// step instead of six.  The step index comes from a device counter the graph advances.
template <int P>
void run_untiled_graph(slt_mesh m, Params a, int64_t nsteps, cudaStream_t s) {
  if (!m->step_dev.p) m->step_dev.alloc(1);
  if (!m->capture) SLT_CUDA(cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking));
  a.step_dev = m->step_dev.p;
  SLT_CUDA(cudaMemsetAsync(m->step_dev.p, 0, sizeof(long long), s));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const bool rec = g_rec.on;
  g_rec.on = false;  // no events inside the capture
  SLT_CUDA(cudaStreamBeginCapture(m->capture, cudaStreamCaptureModeThreadLocal));
  try {
    launch_untiled_range<P>(a, 0, 17, m->capture);
    k_step_inc<<<1, 1, 0, m->capture>>>(m->step_dev.p);
    SLT_CUDA(cudaGetLastError());
  } catch (...) {
    cudaStreamEndCapture(m->capture, &graph);
    if (graph) cudaGraphDestroy(graph);
    g_rec.on = rec;
    throw;
  }
  SLT_CUDA(cudaStreamEndCapture(m->capture, &graph));
  g_rec.on = rec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  SLT_CUDA(e);
  cudaError_t err = cudaSuccess;
  for (int64_t step = 0; step < nsteps && err == cudaSuccess; ++step) {
    g_rec.begin(0, s, kPhases + 1);
    err = cudaGraphLaunch(exec, s);
    g_rec.end(s);
  }
  cudaGraphExecDestroy(exec);
  SLT_CUDA(err);
}

// untiled steps of at least this count run as a captured graph
constexpr int64_t kGraphMinSteps = 4;

template <int P>
void run_steps(slt_mesh m, slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s) {
  if (sched && sched->executor == 0) {
    run_dataflow<P>(sched, a, nsteps, s);
    return;
  }
  if (sched && sched->executor == 2) {
    run_dataflow_cluster<P>(sched, a, nsteps, s);
    return;
  }
  if (sched && sched->executor == 3) {
    run_staged<P>(sched, a, nsteps, s);
    return;
  }
  if (sched && sched->executor == 4) {
    run_passes<P>(sched, a, nsteps, s);
    return;
  }
  if (!sched && nsteps >= kGraphMinSteps) {
    run_untiled_graph<P>(m, a, nsteps, s);
    return;
  }
  for (int64_t step = 0; step < nsteps; ++step) {
    a.step = step;
    if (!sched) {
      launch_untiled_range<P>(a, 0, 17, s);
      continue;
    }
    for (auto& sub : sched->subs) {
      for (int j = sub.first; j < sub.last; ++j) {
        a.plan_ptr[j] = sub.plan_ptr[j - sub.first].p;
        a.plan_items[j] = sub.plan_items[j - sub.first].p;
      }
      for (int c = 0; c < sub.ncolours; ++c)
        launch_tiled_colour<P>(a, sub.first, sub.last, sub.tiles_by_colour.p + sub.colour_ptr[c],
                               sub.colour_ptr[c + 1] - sub.colour_ptr[c], sched->block, s);
    }
  }
}

}  // namespace

void upload_constants(const RefElem& r) { upload_ref(r); }

namespace {
// the expressions the parts evaluated per application, once per cell
__global__ void k_build_pre(const double* __restrict__ geo, const double* __restrict__ fgeo,
                            const double* __restrict__ mat, int64_t nc, int64_t n, double* __restrict__ pre) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const double ir = mat[c];
    for (int k = 0; k < 4; ++k) pre[(PRE_RXR + k) * n + c] = geo[k * n + c] * ir;
    for (int f = 0; f < 3; ++f) {
      const double F = fgeo[(3 * f + 2) * n + c], fx = fgeo[(3 * f) * n + c], fy = fgeo[(3 * f + 1) * n + c];
      const double sc = -0.5 * F * ir;
      pre[(PRE_NB + 2 * f) * n + c] = sc * fx;
      pre[(PRE_NB + 2 * f + 1) * n + c] = sc * fy;
      const double h = -0.5 * F;
      pre[(PRE_ND + 2 * f) * n + c] = h * fx;
      pre[(PRE_ND + 2 * f + 1) * n + c] = h * fy;
    }
    pre[PRE_L2M * n + c] = fma(2.0, mat[2 * n + c], mat[n + c]);
  }
}
}  // namespace

void build_pre(slt_mesh m, cudaStream_t s) {
  if (m->pre.n < (size_t)kPreRows * m->ncp) m->pre.alloc((size_t)kPreRows * m->ncp);
  SLT_CUDA(cudaMemsetAsync(m->pre.p, 0, (size_t)kPreRows * m->ncp * sizeof(double), s));
  int g;
  io_grid(m->nc, g);
  k_build_pre<<<g, 256, 0, s>>>(m->geo.p, m->fgeo.p, m->mat.p, m->nc, m->ncp, m->pre.p);
  SLT_CUDA(cudaGetLastError());
}

void exec_steps_work(slt_mesh m, slt_schedule sched, const double* ricker, double dt, int64_t step0,
                     int64_t nsteps, cudaStream_t s) {
  Params a = make_params(m);
  a.dt = dt;
  a.c24 = dt * dt / 24.0;
  a.ricker = ricker ? ricker + step0 : nullptr;
  switch (m->p) {
    case 1: run_steps<1>(m, sched, a, nsteps, s); break;
    case 2: run_steps<2>(m, sched, a, nsteps, s); break;
    case 3: run_steps<3>(m, sched, a, nsteps, s); break;
    case 4: run_steps<4>(m, sched, a, nsteps, s); break;
  }
}

// One untiled step on the mesh's work fields that leaves its operator intermediates in `keep`
// (rows of ncp, work order): A sigma [2Np], E(A sigma) [3Np], ABA sigma [2Np], E(v) [3Np],
// AB v [2Np], E(AB v) [3Np] - the phases write them there instead of the scratch buffers (same
// phase bodies, so the same numbers).  The adjoint's reverse sweep reads them back.
void exec_step_keep(slt_mesh m, const double* ricker, double dt, int64_t step, double* keep, cudaStream_t s) {
  Params a = make_params(m);
  a.dt = dt;
  a.c24 = dt * dt / 24.0;
  a.ricker = ricker ? ricker + step : nullptr;
  a.step = 0;
  const int64_t r = m->Np * m->ncp;
  double* kA = keep;             // A sigma
  double* kEA = kA + 2 * r;      // E(A sigma)
  double* kABA = kEA + 3 * r;    // ABA sigma
  double* kEv = kABA + 2 * r;    // E(v)
  double* kABv = kEv + 3 * r;    // AB v
  double* kEABv = kABv + 2 * r;  // E(AB v)
  Params a1 = a, a2 = a, a3 = a, a4 = a;
  a1.buf[B_U1] = kA;     // loops 0-8: U1 = A sigma, E = E(A sigma), U2 = ABA sigma
  a1.buf[B_E] = kEA;
  a1.buf[B_U2] = kABA;
  a2.buf[B_E] = kEv;     // loops 9-11: E = E(v), U1 = volume part of AB v
  a2.buf[B_U1] = kABv;
  a3.buf[B_U1] = kABv;   // loops 12-13: U1 = AB v
  a4.buf[B_U1] = kABv;   // loops 14-16: E = E(AB v)
  a4.buf[B_E] = kEABv;
  auto run = [&](const Params& q, int first, int last) {
    switch (m->p) {
      case 1: launch_untiled_range<1>(q, first, last, s); break;
      case 2: launch_untiled_range<2>(q, first, last, s); break;
      case 3: launch_untiled_range<3>(q, first, last, s); break;
      case 4: launch_untiled_range<4>(q, first, last, s); break;
    }
  };
  run(a1, 0, 9);
  run(a2, 9, 12);
  run(a3, 12, 14);
  run(a4, 14, 17);
}

// Operators on work-layout buffers (untiled loops with redirected operands), for the adjoint.
void op_A(slt_mesh m, const double* in3, double* out2, cudaStream_t s) {
  Params a = make_params(m);
  a.buf[B_S] = const_cast<double*>(in3);
  a.buf[B_U1] = out2;
  switch (m->p) {
    case 1: launch_untiled_range<1>(a, 0, 3, s); break;
    case 2: launch_untiled_range<2>(a, 0, 3, s); break;
    case 3: launch_untiled_range<3>(a, 0, 3, s); break;
    case 4: launch_untiled_range<4>(a, 0, 3, s); break;
  }
}
void op_E(slt_mesh m, const double* in2, double* out3, cudaStream_t s) {
  Params a = make_params(m);
  a.buf[B_U1] = const_cast<double*>(in2);
  a.buf[B_E] = out3;
  switch (m->p) {
    case 1: launch_untiled_range<1>(a, 3, 5, s); break;
    case 2: launch_untiled_range<2>(a, 3, 5, s); break;
    case 3: launch_untiled_range<3>(a, 3, 5, s); break;
    case 4: launch_untiled_range<4>(a, 3, 5, s); break;
  }
}

namespace {
// caller cells [c0, c1) <-> work layout, one caller row block per cell (the pipelined host path
// converts each chunk as soon as it has arrived)
__global__ void k_to_work_cells(const double* __restrict__ in, int rows, const int32_t* __restrict__ iperm, int64_t c0,
                                int64_t c1, int64_t ncp, double* __restrict__ out) {
  const int64_t n = (c1 - c0) * rows;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = c0 + i / rows, q = i % rows;
    out[q * ncp + iperm[c]] = in[c * rows + q];
  }
}
__global__ void k_from_work_cells(const double* __restrict__ in, int rows, const int32_t* __restrict__ iperm,
                                  int64_t c0, int64_t c1, int64_t ncp, double* __restrict__ out) {
  const int64_t n = (c1 - c0) * rows;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = c0 + i / rows, q = i % rows;
    out[c * rows + q] = in[q * ncp + iperm[c]];
  }
}
}  // namespace

// Host fields: the copies overlap the layout conversion.  The fields go over in kHostChunks
// chunks of cells on a copy stream; each chunk is converted into the work layout on the
// compute stream as soon as its copy has finished, while the next chunk is on the link; the
// result comes back the same way (convert a chunk, copy it while the next converts).
void exec_run_host(slt_mesh m, slt_schedule sched, double* hv, double* hs, const double* hr, double dt,
                   int64_t nsteps, cudaStream_t s) {
  constexpr int kHostChunks = 4;
  g_rec = Recorder();
  const int Np = m->Np;
  const int64_t nc = m->nc, nv = nc * 2 * Np, ns = nc * 3 * Np;
  if (m->io_v.n < (size_t)nv) m->io_v.alloc(nv);
  if (m->io_s.n < (size_t)ns) m->io_s.alloc(ns);
  if (hr && m->ricker_buf.n < (size_t)std::max<int64_t>(nsteps, 1)) m->ricker_buf.alloc(std::max<int64_t>(nsteps, 1));
  if (!m->copy) SLT_CUDA(cudaStreamCreateWithFlags(&m->copy, cudaStreamNonBlocking));
  cudaStream_t cs = m->copy;
  cudaEvent_t ev[2 * kHostChunks + 1];
  for (auto& e : ev) SLT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  Params a = make_params(m);
  a.dt = dt;
  a.c24 = dt * dt / 24.0;
  a.ricker = hr ? m->ricker_buf.p : nullptr;
  auto chunk = [&](int k, int64_t& c0, int64_t& c1) {
    c0 = nc * k / kHostChunks;
    c1 = nc * (k + 1) / kHostChunks;
  };
  SLT_CUDA(cudaEventRecord(ev[2 * kHostChunks], s));  // the copies start after earlier work on s
  SLT_CUDA(cudaStreamWaitEvent(cs, ev[2 * kHostChunks], 0));
  if (hr) SLT_CUDA(cudaMemcpyAsync(m->ricker_buf.p, hr, nsteps * sizeof(double), cudaMemcpyHostToDevice, cs));
  for (int k = 0; k < kHostChunks; ++k) {
    int64_t c0, c1;
    chunk(k, c0, c1);
    SLT_CUDA(cudaMemcpyAsync(m->io_v.p + c0 * 2 * Np, hv + c0 * 2 * Np, (c1 - c0) * 2 * Np * sizeof(double),
                             cudaMemcpyHostToDevice, cs));
    SLT_CUDA(cudaMemcpyAsync(m->io_s.p + c0 * 3 * Np, hs + c0 * 3 * Np, (c1 - c0) * 3 * Np * sizeof(double),
                             cudaMemcpyHostToDevice, cs));
    SLT_CUDA(cudaEventRecord(ev[k], cs));
    SLT_CUDA(cudaStreamWaitEvent(s, ev[k], 0));
    int g;
    io_grid((c1 - c0) * 3 * Np, g);
    k_to_work_cells<<<g, 256, 0, s>>>(m->io_v.p, 2 * Np, m->d_iperm.p, c0, c1, m->ncp, a.buf[B_V]);
    k_to_work_cells<<<g, 256, 0, s>>>(m->io_s.p, 3 * Np, m->d_iperm.p, c0, c1, m->ncp, a.buf[B_S]);
  }
  SLT_CUDA(cudaGetLastError());
  switch (m->p) {
    case 1: run_steps<1>(m, sched, a, nsteps, s); break;
    case 2: run_steps<2>(m, sched, a, nsteps, s); break;
    case 3: run_steps<3>(m, sched, a, nsteps, s); break;
    case 4: run_steps<4>(m, sched, a, nsteps, s); break;
  }
  for (int k = 0; k < kHostChunks; ++k) {
    int64_t c0, c1;
    chunk(k, c0, c1);
    int g;
    io_grid((c1 - c0) * 3 * Np, g);
    k_from_work_cells<<<g, 256, 0, s>>>(a.buf[B_V], 2 * Np, m->d_iperm.p, c0, c1, m->ncp, m->io_v.p);
    k_from_work_cells<<<g, 256, 0, s>>>(a.buf[B_S], 3 * Np, m->d_iperm.p, c0, c1, m->ncp, m->io_s.p);
    SLT_CUDA(cudaEventRecord(ev[kHostChunks + k], s));
    SLT_CUDA(cudaStreamWaitEvent(cs, ev[kHostChunks + k], 0));
    SLT_CUDA(cudaMemcpyAsync(hv + c0 * 2 * Np, m->io_v.p + c0 * 2 * Np, (c1 - c0) * 2 * Np * sizeof(double),
                             cudaMemcpyDeviceToHost, cs));
    SLT_CUDA(cudaMemcpyAsync(hs + c0 * 3 * Np, m->io_s.p + c0 * 3 * Np, (c1 - c0) * 3 * Np * sizeof(double),
                             cudaMemcpyDeviceToHost, cs));
  }
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaStreamSynchronize(cs));
  SLT_CUDA(cudaStreamSynchronize(s));
  for (auto& e : ev) cudaEventDestroy(e);
}

void exec_run(slt_mesh m, slt_schedule sched, double* v, double* sigma, const double* ricker, double dt,
              int64_t nsteps, cudaStream_t s, double* profile) {
  g_rec = Recorder();
  g_rec.on = profile != nullptr;
  Params a = make_params(m);
  a.dt = dt;
  a.c24 = dt * dt / 24.0;
  a.ricker = ricker;
  const int Np = m->Np;
  int g;
  io_grid(m->nc, g);
  g_rec.begin(1, s, 2);
  k_to_work<<<g, 256, 0, s>>>(v, 2 * Np, m->d_perm.p, m->nc, m->ncp, a.buf[B_V]);
  k_to_work<<<g, 256, 0, s>>>(sigma, 3 * Np, m->d_perm.p, m->nc, m->ncp, a.buf[B_S]);
  g_rec.end(s);
  SLT_CUDA(cudaGetLastError());
  switch (m->p) {
    case 1: run_steps<1>(m, sched, a, nsteps, s); break;
    case 2: run_steps<2>(m, sched, a, nsteps, s); break;
    case 3: run_steps<3>(m, sched, a, nsteps, s); break;
    case 4: run_steps<4>(m, sched, a, nsteps, s); break;
  }
  g_rec.begin(1, s, 2);
  k_from_work<<<g, 256, 0, s>>>(a.buf[B_V], 2 * Np, m->d_perm.p, m->nc, m->ncp, v);
  k_from_work<<<g, 256, 0, s>>>(a.buf[B_S], 3 * Np, m->d_perm.p, m->nc, m->ncp, sigma);
  g_rec.end(s);
  SLT_CUDA(cudaGetLastError());
  g_rec.finish(s, profile);
  g_rec = Recorder();
}

// ------------------------------------------------------------------ groups of meshes
// The combined plan of each degree: tiles of member i renumbered by base_i (the sum of the
// earlier members' tiles), successor lists shifted accordingly; dependency counts copied.
void group_build(slt_group grp) {
  std::map<int, std::vector<int32_t>> by_degree;
  for (size_t i = 0; i < grp->meshes.size(); ++i) {
    slt_schedule sc = grp->scheds[i];
    if (sc && sc->executor == 0) by_degree[grp->mixed ? 0 : grp->meshes[i]->p].push_back((int32_t)i);
    else grp->untiled.push_back((int32_t)i);  // untiled, or the colour-phase or cluster executor
  }
  for (auto& kv : by_degree) {
    grp->parts.emplace_back();
    slt_group_s::Part& part = grp->parts.back();
    part.p = kv.first;
    part.members = kv.second;
    std::vector<int32_t> cum, first, last, mesh_of, succ_ptr, succ, indeg0, indeg;
    int32_t base = 0;
    part.block = grp->scheds[part.members[0]]->block;
    for (size_t mi = 0; mi < part.members.size(); ++mi) {
      slt_schedule sc = grp->scheds[part.members[mi]];
      if (sc->block != part.block) fail(SLT_ERR_UNSUPPORTED, "tiled meshes of one degree need one block size");
      if (grp->mixed && (sc->block != 256 || grp->meshes[part.members[mi]]->p > 3))
        fail(SLT_ERR_UNSUPPORTED, "one launch over all degrees takes degrees 1-3 and 256-thread tiles");
      if (sc->block > 384) fail(SLT_ERR_UNSUPPORTED, "group members take 128-384-thread tiles");
      part.wait_spins = std::max<int64_t>(part.wait_spins, sc->wait_spins);
      part.keep = std::min(part.keep, sc->keep);
      const DataflowPlan& D = sc->df;
      const int32_t G = D.cum.back();
      for (size_t k = 0; k < sc->subs.size(); ++k) {
        cum.push_back(base + D.cum[k]);
        first.push_back(sc->subs[k].first);
        last.push_back(sc->subs[k].last);
        mesh_of.push_back((int32_t)mi);
      }
      std::vector<int32_t> sp = D.succ_ptr.download(nullptr, G + 1);
      std::vector<int32_t> sv = D.succ.download(nullptr, std::max<int32_t>(sp[G], 1));
      std::vector<int32_t> i0 = D.indeg0.download(nullptr, G), i1 = D.indeg.download(nullptr, G);
      const int32_t off = succ_ptr.empty() ? 0 : (int32_t)succ.size();
      for (int32_t g = 0; g < G; ++g) succ_ptr.push_back(off + sp[g]);
      for (int32_t q = 0; q < sp[G]; ++q) succ.push_back((((sv[q] >> 1) + base) << 1) | (sv[q] & 1));
      indeg0.insert(indeg0.end(), i0.begin(), i0.end());
      indeg.insert(indeg.end(), i1.begin(), i1.end());
      base += G;
    }
    cum.push_back(base);
    succ_ptr.push_back((int32_t)succ.size());
    part.G = base;
    part.K = (int32_t)first.size();
    auto up = [](DevBuf<int32_t>& d, const std::vector<int32_t>& h) {
      d.alloc(std::max<size_t>(h.size(), 1));
      d.upload(h.data(), h.size(), nullptr);
    };
    up(part.cum, cum);
    up(part.first, first);
    up(part.last, last);
    up(part.mesh_of, mesh_of);
    up(part.succ_ptr, succ_ptr);
    up(part.succ, succ);
    up(part.indeg0, indeg0);
    up(part.indeg, indeg);
    part.err.alloc(1);
    part.head.alloc(2);
    part.params.alloc(part.members.size() * sizeof(Params));
  }
  SLT_CUDA(cudaDeviceSynchronize());
}

namespace {

template <int P>
void launch_group_part(slt_group_s::Part& part, int64_t nsteps, cudaStream_t s) {
  DFM df{};
  DFQ& q = df.q;
  q.G = part.G;
  q.nsteps = nsteps;
  q.total = (long long)nsteps * part.G;
  if (q.total == 0) return;
  if (q.total >= (1ll << 31)) fail(SLT_ERR_UNSUPPORTED, "steps x tiles must stay below 2^31");
  if (part.pending.n < (size_t)q.total) {  // (allocated ahead of a captured run: group_run_mixed)
    part.pending.alloc(q.total);
    part.queue.alloc(q.total);
  }
  q.succ_ptr = part.succ_ptr.p;
  q.succ = part.succ.p;
  q.pending = part.pending.p;
  q.queue = part.queue.p;
  q.head = part.head.p;
  q.tail = part.head.p + 1;
  q.err = part.err.p;
  q.max_spins = part.wait_spins;
  q.keep = part.keep;
  q.g_lo = 0;
  q.g_hi = q.G;
  df.K = part.K;
  df.cum = part.cum.p;
  df.first = part.first.p;
  df.last = part.last.p;
  df.mesh_of = part.mesh_of.p;
  df.params = reinterpret_cast<const Params*>(part.params.p);
  SLT_CUDA(cudaMemsetAsync(part.head.p, 0, 2 * sizeof(unsigned long long), s));
  SLT_CUDA(cudaMemsetAsync(part.err.p, 0, sizeof(int32_t), s));
  k_df_init<<<(unsigned)std::min<long long>((q.total + 255) / 256, 152 * 16), 256, 0, s>>>(q, part.indeg0.p,
                                                                                         part.indeg.p);
  k_df_seed<<<(q.G + 255) / 256, 256, 0, s>>>(q, part.indeg0.p);
  SLT_CUDA(cudaGetLastError());
  int dev = 0, nsm = 0, per = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto launch = [&](auto kernel, int threads) {
    SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0));
    const long long grid = std::min<long long>((long long)nsm * std::max(per, 1), q.total);
    kernel<<<(unsigned)grid, threads, 0, s>>>(df);
  };
  if constexpr (P == 0) launch(k_dataflow_mixed<256>, 256);
  else if (part.block == 128) launch(k_dataflow_group<P, 128>, 128);
  else if (part.block == 384) launch(k_dataflow_group<P, 384>, 384);
  else launch(k_dataflow_group<P, 256>, 256);
  SLT_CUDA(cudaGetLastError());
}

}  // namespace

// One call: every member's fields into its work layout; each degree's tiled members as one
// persistent kernel over their combined queue (one degree after the other, each with the whole
// GPU); the untiled members side by side on private streams; fields back.
void group_run_mixed(slt_group grp, double* const* v, double* const* sigma, const double* const* ricker,
                     const double* dt, int64_t nsteps, cudaStream_t s);

void group_run(slt_group grp, double* const* v, double* const* sigma, const double* const* ricker, const double* dt,
               int64_t nsteps, cudaStream_t s) {
  if (grp->mixed) {
    group_run_mixed(grp, v, sigma, ricker, dt, nsteps, s);
    return;
  }
  g_rec = Recorder();
  const int32_t n = (int32_t)grp->meshes.size();
  std::vector<Params> prm(n);
  for (int32_t i = 0; i < n; ++i) {
    slt_mesh m = grp->meshes[i];
    Params& a = prm[i];
    a = make_params(m);
    a.dt = dt[i];
    a.c24 = dt[i] * dt[i] / 24.0;
    a.ricker = ricker[i];
    if (slt_schedule sc = grp->scheds[i])
      for (auto& sub : sc->subs)
        for (int j = sub.first; j < sub.last; ++j) {
          a.plan_ptr[j] = sub.plan_ptr[j - sub.first].p;
          a.plan_items[j] = sub.plan_items[j - sub.first].p;
        }
    int g;
    io_grid(m->nc, g);
    k_to_work<<<g, 256, 0, s>>>(v[i], 2 * m->Np, m->d_perm.p, m->nc, m->ncp, a.buf[B_V]);
    k_to_work<<<g, 256, 0, s>>>(sigma[i], 3 * m->Np, m->d_perm.p, m->nc, m->ncp, a.buf[B_S]);
  }
  SLT_CUDA(cudaGetLastError());
  for (auto& part : grp->parts) {
    std::vector<Params> pp;
    for (int32_t i : part.members) pp.push_back(prm[i]);
    SLT_CUDA(cudaMemcpyAsync(part.params.p, pp.data(), pp.size() * sizeof(Params), cudaMemcpyHostToDevice, s));
    switch (part.p) {
      case 1: launch_group_part<1>(part, nsteps, s); break;
      case 2: launch_group_part<2>(part, nsteps, s); break;
      case 3: launch_group_part<3>(part, nsteps, s); break;
      case 4: launch_group_part<4>(part, nsteps, s); break;
    }
  }
  if (!grp->untiled.empty()) {  // fork, run side by side, join
    const size_t u = grp->untiled.size();
    std::vector<cudaStream_t> st(u, nullptr);
    std::vector<cudaEvent_t> ev(u + 1, nullptr);
    auto cleanup = [&] {
      for (cudaStream_t x : st)
        if (x) {
          cudaStreamSynchronize(x);
          cudaStreamDestroy(x);
        }
      for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    };
    try {
      SLT_CUDA(cudaEventCreateWithFlags(&ev[u], cudaEventDisableTiming));
      SLT_CUDA(cudaEventRecord(ev[u], s));
      for (size_t k = 0; k < u; ++k) {
        const int32_t i = grp->untiled[k];
        slt_mesh m = grp->meshes[i];
        SLT_CUDA(cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking));
        SLT_CUDA(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
        SLT_CUDA(cudaStreamWaitEvent(st[k], ev[u], 0));
        switch (m->p) {
          case 1: run_steps<1>(m, grp->scheds[i], prm[i], nsteps, st[k]); break;
          case 2: run_steps<2>(m, grp->scheds[i], prm[i], nsteps, st[k]); break;
          case 3: run_steps<3>(m, grp->scheds[i], prm[i], nsteps, st[k]); break;
          case 4: run_steps<4>(m, grp->scheds[i], prm[i], nsteps, st[k]); break;
        }
        SLT_CUDA(cudaEventRecord(ev[k], st[k]));
      }
      for (size_t k = 0; k < u; ++k) SLT_CUDA(cudaStreamWaitEvent(s, ev[k], 0));
    } catch (...) {
      cleanup();
      throw;
    }
    cleanup();
  }
  for (int32_t i = 0; i < n; ++i) {
    slt_mesh m = grp->meshes[i];
    int g;
    io_grid(m->nc, g);
    k_from_work<<<g, 256, 0, s>>>(prm[i].buf[B_V], 2 * m->Np, m->d_perm.p, m->nc, m->ncp, v[i]);
    k_from_work<<<g, 256, 0, s>>>(prm[i].buf[B_S], 3 * m->Np, m->d_perm.p, m->nc, m->ncp, sigma[i]);
  }
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaStreamSynchronize(s));
  for (auto& part : grp->parts) {
    int32_t herr = 0;
    SLT_CUDA(cudaMemcpy(&herr, part.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (herr && nsteps > 0) fail(SLT_ERR_TIMEOUT, "a wait of the dataflow executor gave up");
  }
}

// The batched form in one launch: every tiled member (any degree 1-3, one field or many shots)
// runs from one ready queue in one persistent kernel.  The fields' conversion into the work
// layout, the queue reset and seeding, the persistent kernel and the conversion back are
// captured once as a CUDA graph and replayed while nsteps and the field pointers stay the same
// (the parameter blocks, with the source series and time steps, are uploaded before each replay).
// Untiled members run afterwards as in group_run.
void group_run_mixed(slt_group grp, double* const* v, double* const* sigma, const double* const* ricker,
                     const double* dt, int64_t nsteps, cudaStream_t s) {
  g_rec = Recorder();
  const int32_t n = (int32_t)grp->meshes.size();
  std::vector<Params> prm(n);
  for (int32_t i = 0; i < n; ++i) {
    slt_mesh m = grp->meshes[i];
    const int32_t S = grp->nshots[i];
    Params& a = prm[i];
    if (S > 1) {
      const int64_t fs = m->ncp * S, need = 15 * m->Np * fs;
      if (m->work_b.n < (size_t)need) {
        m->work_b.alloc(need);
        SLT_CUDA(cudaMemsetAsync(m->work_b.p, 0, need * sizeof(double), s));
      }
      a = make_params(m);
      double* base = m->work_b.p;
      const int64_t Np = m->Np;
      a.buf[B_V] = base;
      a.buf[B_S] = base + 2 * Np * fs;
      a.buf[B_U1] = base + 5 * Np * fs;
      a.buf[B_U2] = base + 7 * Np * fs;
      a.buf[B_E] = base + 9 * Np * fs;
      a.buf[B_S1] = base + 12 * Np * fs;
      a.src = nullptr;
      a.src_w = -1;
      a.S = S;
      a.s0 = 0;
      a.sg = S;
      a.fs = fs;
      a.src_wb = grp->src_w[i].p;
      a.src_b = grp->src[i].p;
    } else {
      a = make_params(m);
    }
    a.p = m->p;
    a.dt = dt[i];
    a.c24 = dt[i] * dt[i] / 24.0;
    a.ricker = ricker[i];
    if (slt_schedule sc = grp->scheds[i])
      for (auto& sub : sc->subs)
        for (int j = sub.first; j < sub.last; ++j) {
          a.plan_ptr[j] = sub.plan_ptr[j - sub.first].p;
          a.plan_items[j] = sub.plan_items[j - sub.first].p;
        }
  }
  std::vector<int32_t> tiled;
  for (auto& part : grp->parts) {
    std::vector<Params> pp;
    for (int32_t i : part.members) {
      pp.push_back(prm[i]);
      tiled.push_back(i);
    }
    SLT_CUDA(cudaMemcpyAsync(part.params.p, pp.data(), pp.size() * sizeof(Params), cudaMemcpyHostToDevice, s));
    const long long total = (long long)nsteps * part.G;
    if (total >= (1ll << 31)) fail(SLT_ERR_UNSUPPORTED, "steps x tiles must stay below 2^31");
    if (part.pending.n < (size_t)total) {
      part.pending.alloc(total);
      part.queue.alloc(total);
    }
  }
  auto convert = [&](cudaStream_t st, bool in) {
    for (int32_t i : tiled) {
      slt_mesh m = grp->meshes[i];
      const int32_t S = grp->nshots[i];
      const int Np = m->Np;
      int g;
      io_grid(m->nc * (S > 1 ? 5 * Np * S : 1), g);
      if (S > 1) {
        if (in) {
          k_to_work_b<<<g, 256, 0, st>>>(v[i], 2 * Np, S, m->d_perm.p, m->nc, m->ncp, prm[i].buf[B_V]);
          k_to_work_b<<<g, 256, 0, st>>>(sigma[i], 3 * Np, S, m->d_perm.p, m->nc, m->ncp, prm[i].buf[B_S]);
        } else {
          k_from_work_b<<<g, 256, 0, st>>>(prm[i].buf[B_V], 2 * Np, S, m->d_perm.p, m->nc, m->ncp, v[i]);
          k_from_work_b<<<g, 256, 0, st>>>(prm[i].buf[B_S], 3 * Np, S, m->d_perm.p, m->nc, m->ncp, sigma[i]);
        }
      } else if (in) {
        k_to_work<<<g, 256, 0, st>>>(v[i], 2 * Np, m->d_perm.p, m->nc, m->ncp, prm[i].buf[B_V]);
        k_to_work<<<g, 256, 0, st>>>(sigma[i], 3 * Np, m->d_perm.p, m->nc, m->ncp, prm[i].buf[B_S]);
      } else {
        k_from_work<<<g, 256, 0, st>>>(prm[i].buf[B_V], 2 * Np, m->d_perm.p, m->nc, m->ncp, v[i]);
        k_from_work<<<g, 256, 0, st>>>(prm[i].buf[B_S], 3 * Np, m->d_perm.p, m->nc, m->ncp, sigma[i]);
      }
    }
  };
  if (!tiled.empty()) {
    std::vector<const void*> key = {reinterpret_cast<const void*>(nsteps)};
    for (int32_t i : tiled) {
      key.push_back(v[i]);
      key.push_back(sigma[i]);
    }
    if (!grp->graph || key != grp->graph_key) {
      if (grp->graph) {
        cudaGraphExecDestroy(grp->graph);
        grp->graph = nullptr;
      }
      if (!grp->capture) SLT_CUDA(cudaStreamCreateWithFlags(&grp->capture, cudaStreamNonBlocking));
      SLT_CUDA(cudaStreamSynchronize(s));  // the parameter uploads are on s
      cudaGraph_t graph = nullptr;
      SLT_CUDA(cudaStreamBeginCapture(grp->capture, cudaStreamCaptureModeThreadLocal));
      try {
        convert(grp->capture, true);
        for (auto& part : grp->parts) {
          switch (part.p) {
            case 0: launch_group_part<0>(part, nsteps, grp->capture); break;
            case 1: launch_group_part<1>(part, nsteps, grp->capture); break;
            case 2: launch_group_part<2>(part, nsteps, grp->capture); break;
            case 3: launch_group_part<3>(part, nsteps, grp->capture); break;
            default: launch_group_part<4>(part, nsteps, grp->capture); break;
          }
        }
        convert(grp->capture, false);
        SLT_CUDA(cudaGetLastError());
      } catch (...) {
        cudaStreamEndCapture(grp->capture, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      SLT_CUDA(cudaStreamEndCapture(grp->capture, &graph));
      cudaError_t e = cudaGraphInstantiate(&grp->graph, graph, 0);
      cudaGraphDestroy(graph);
      SLT_CUDA(e);
      grp->graph_key = key;
      grp->graph_launches = 0;
    }
    SLT_CUDA(cudaGraphLaunch(grp->graph, s));
    ++grp->graph_launches;
  }
  if (!grp->untiled.empty()) {
    for (int32_t i : grp->untiled) {
      slt_mesh m = grp->meshes[i];
      int g;
      io_grid(m->nc, g);
      k_to_work<<<g, 256, 0, s>>>(v[i], 2 * m->Np, m->d_perm.p, m->nc, m->ncp, prm[i].buf[B_V]);
      k_to_work<<<g, 256, 0, s>>>(sigma[i], 3 * m->Np, m->d_perm.p, m->nc, m->ncp, prm[i].buf[B_S]);
      switch (m->p) {
        case 1: run_steps<1>(m, grp->scheds[i], prm[i], nsteps, s); break;
        case 2: run_steps<2>(m, grp->scheds[i], prm[i], nsteps, s); break;
        case 3: run_steps<3>(m, grp->scheds[i], prm[i], nsteps, s); break;
        case 4: run_steps<4>(m, grp->scheds[i], prm[i], nsteps, s); break;
      }
      k_from_work<<<g, 256, 0, s>>>(prm[i].buf[B_V], 2 * m->Np, m->d_perm.p, m->nc, m->ncp, v[i]);
      k_from_work<<<g, 256, 0, s>>>(prm[i].buf[B_S], 3 * m->Np, m->d_perm.p, m->nc, m->ncp, sigma[i]);
    }
    SLT_CUDA(cudaGetLastError());
  }
  SLT_CUDA(cudaStreamSynchronize(s));
  for (auto& part : grp->parts) {
    int32_t herr = 0;
    SLT_CUDA(cudaMemcpy(&herr, part.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (herr && nsteps > 0) fail(SLT_ERR_TIMEOUT, "a wait of the dataflow executor gave up");
  }
}

void exec_apply(slt_mesh m, int op, const double* in, double* out, cudaStream_t s) {
  g_rec = Recorder();
  Params a = make_params(m);
  const int Np = m->Np;
  int g;
  io_grid(m->nc, g);
  if (op == 0) {
    k_to_work<<<g, 256, 0, s>>>(in, 3 * Np, m->d_perm.p, m->nc, m->ncp, a.buf[B_S]);
    switch (m->p) {
      case 1: launch_untiled_range<1>(a, 0, 3, s); break;
      case 2: launch_untiled_range<2>(a, 0, 3, s); break;
      case 3: launch_untiled_range<3>(a, 0, 3, s); break;
      case 4: launch_untiled_range<4>(a, 0, 3, s); break;
    }
    k_from_work<<<g, 256, 0, s>>>(a.buf[B_U1], 2 * Np, m->d_perm.p, m->nc, m->ncp, out);
  } else {
    // B v: volD and intD into E, then hookeB (S1 = C E; its U2 output is not used)
    k_to_work<<<g, 256, 0, s>>>(in, 2 * Np, m->d_perm.p, m->nc, m->ncp, a.buf[B_U1]);
    switch (m->p) {
      case 1: launch_untiled_range<1>(a, 3, 6, s); break;
      case 2: launch_untiled_range<2>(a, 3, 6, s); break;
      case 3: launch_untiled_range<3>(a, 3, 6, s); break;
      case 4: launch_untiled_range<4>(a, 3, 6, s); break;
    }
    k_from_work<<<g, 256, 0, s>>>(a.buf[B_S1], 3 * Np, m->d_perm.p, m->nc, m->ncp, out);
  }
  SLT_CUDA(cudaGetLastError());
}

}  // namespace slt
