// Multi-shot executor: S shots of the same mesh and material advance together, fields stored
// with the shots innermost ([cell][comp][node][shot] for the caller, rows of ncp * S doubles in
// the work layout).  Consecutive threads take consecutive shots of one cell, so field loads
// coalesce over shots and per-cell geometry, neighbours and face masks are warp-uniform; every
// shot has its own point source.  The phase bodies are those of exec_body.cuh; the arithmetic of
// each (cell, shot) is exactly that of a single-field run with that shot's source.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "refmask.h"

namespace slt {

namespace {

#include "exec_body.cuh"
#include "dataflow.cuh"
#include "layout.cuh"

// Untiled chain, phase H (see phase_first) over every (cell, shot).
template <int P, int H>
__global__ void __launch_bounds__(128) k_phase_b(Params a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // over nc * S
  if (t >= a.nc * a.S) return;
  run_phase<P, H, kAllParts, true>(a, t / a.S, (int)(t % a.S), a.step);
}

template <int P>
void launch_untiled_b(const Params& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.nc * a.S + 127) / 128);
  k_phase_b<P, 0><<<blocks, 128, 0, s>>>(a);
  k_phase_b<P, 1><<<blocks, 128, 0, s>>>(a);
  k_phase_b<P, 2><<<blocks, 128, 0, s>>>(a);
  k_phase_b<P, 3><<<blocks, 128, 0, s>>>(a);
  k_phase_b<P, 4><<<blocks, 128, 0, s>>>(a);
  k_phase_b<P, 5><<<blocks, 128, 0, s>>>(a);
  SLT_CUDA(cudaGetLastError());
}

struct Timer {
  std::vector<cudaEvent_t> ev;
  std::vector<int> nl, cls;  // launches and class (0 chain, 1 layout, 2 queue set-up) of each pair
  bool on = false;
  void begin(cudaStream_t s, int n, int c = 0) {
    if (!on) return;
    cudaEvent_t e0, e1;
    SLT_CUDA(cudaEventCreate(&e0));
    SLT_CUDA(cudaEventCreate(&e1));
    ev.push_back(e0);
    ev.push_back(e1);
    nl.push_back(n);
    cls.push_back(c);
    SLT_CUDA(cudaEventRecord(e0, s));
  }
  void end(cudaStream_t s) {
    if (on) SLT_CUDA(cudaEventRecord(ev.back(), s));
  }
};

template <int P>
void run_batched(slt_mesh m, slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s, Timer& tm) {
  if (sched) {  // the shots in slices of shots_per_cta, one queue pass each
    const int32_t g = sched->shots_per_cta > 0 ? std::min(sched->shots_per_cta, a.S) : a.S;
    for (int32_t s0 = 0; s0 < a.S; s0 += g) {
      a.s0 = s0;
      a.sg = std::min(g, a.S - s0);
      launch_dataflow<P, true>(sched, a, nsteps, s, [&](int c, int n) { tm.begin(s, n, c); },
                               [&] { tm.end(s); });
    }
    return;
  }
  for (int64_t step = 0; step < nsteps; ++step) {
    a.step = step;
    tm.begin(s, kPhases);
    launch_untiled_b<P>(a, s);
    tm.end(s);
  }
}

template <int P>
void part_b(slt_schedule sched, Params a, int part, cudaStream_t s) {
  if (!sched) {
    const unsigned blocks = (unsigned)((a.nc * a.S + 127) / 128);
    if (part != 1) {
      k_phase_b<P, 0><<<blocks, 128, 0, s>>>(a);
      k_phase_b<P, 1><<<blocks, 128, 0, s>>>(a);
      k_phase_b<P, 2><<<blocks, 128, 0, s>>>(a);
    }
    if (part != 0) {
      k_phase_b<P, 3><<<blocks, 128, 0, s>>>(a);
      k_phase_b<P, 4><<<blocks, 128, 0, s>>>(a);
      k_phase_b<P, 5><<<blocks, 128, 0, s>>>(a);
    }
    SLT_CUDA(cudaGetLastError());
    return;
  }
  const int32_t g = sched->shots_per_cta > 0 ? std::min(sched->shots_per_cta, a.S) : a.S;
  for (int32_t s0 = 0; s0 < a.S; s0 += g) {
    a.s0 = s0;
    a.sg = std::min(g, a.S - s0);
    launch_dataflow<P, true>(sched, a, 1, s, [](int, int) {}, [] {}, part == 2 ? -1 : part);
  }
}

}  // namespace

void chain_part_b(slt_mesh m, slt_schedule sched, const ChainRun& r, int part, cudaStream_t s) {
  if (sched && part != 2) {
    if (sched->executor != 0 || sched->subs.size() != 2 || sched->subs[0].last != 9)
      fail(SLT_ERR_UNSUPPORTED, "a sub-chain at a time needs the {velocity, stress} fusion and the dataflow executor");
  }
  Params a{};
  a.ncp = m->ncp;
  a.nc = m->nc;
  a.geo = m->geo.p;
  a.fgeo = m->fgeo.p;
  a.mat = m->mat.p;
  a.nbr = m->nbr.p;
  a.pre = m->pre.p;
  for (int b = 0; b < 6; ++b) a.buf[b] = r.buf[b];
  a.e5 = r.e5;
  a.ricker = r.ricker;
  a.src = nullptr;
  a.src_w = -1;
  a.dt = r.dt;
  a.c24 = r.dt * r.dt / 24.0;
  a.S = r.S;
  a.s0 = 0;
  a.sg = r.S;
  a.fs = m->ncp * r.S;
  a.src_wb = r.src_w;
  a.src_b = r.src;
  switch (m->p) {
    case 1: part_b<1>(sched, a, part, s); break;
    case 2: part_b<2>(sched, a, part, s); break;
    case 3: part_b<3>(sched, a, part, s); break;
    case 4: part_b<4>(sched, a, part, s); break;
  }
  if (sched) dataflow_check(sched, s);
}

void upload_constants_batched(const RefElem& r) { upload_ref(r); }

void exec_run_batched(slt_mesh m, slt_schedule sched, int32_t S, const int32_t* d_src_w, const double* d_src,
                      double* v, double* sigma, const double* ricker, double dt, int64_t nsteps, cudaStream_t s,
                      double* profile) {
  if (sched && sched->executor != 0)
    fail(SLT_ERR_UNSUPPORTED, "the multi-shot executor runs untiled or with the dataflow executor");
  const int64_t Np = m->Np, ncp = m->ncp, fs = ncp * S;
  const size_t need = 15 * Np * fs;
  if (m->work_b.n < need) {
    m->work_b.alloc(need);
    SLT_CUDA(cudaMemsetAsync(m->work_b.p, 0, need * sizeof(double), s));
  }
  double* base = m->work_b.p;
  Params a{};
  a.ncp = ncp;
  a.nc = m->nc;
  a.geo = m->geo.p;
  a.fgeo = m->fgeo.p;
  a.mat = m->mat.p;
  a.nbr = m->nbr.p;
  a.pre = m->pre.p;
  a.buf[B_V] = base;
  a.buf[B_S] = base + 2 * Np * fs;
  a.buf[B_U1] = base + 5 * Np * fs;
  a.buf[B_U2] = base + 7 * Np * fs;
  a.buf[B_E] = base + 9 * Np * fs;
  a.buf[B_S1] = base + 12 * Np * fs;
  a.ricker = ricker;
  a.src = nullptr;
  a.src_w = -1;
  a.dt = dt;
  a.c24 = dt * dt / 24.0;
  a.S = S;
  a.s0 = 0;
  a.sg = S;
  a.fs = fs;
  a.src_wb = d_src_w;
  a.src_b = d_src;
  Timer tm;
  tm.on = profile != nullptr;
  const int g = (int)std::min<int64_t>((m->nc * 5 * Np * S + 255) / 256, 152 * 32);
  tm.begin(s, 2, 1);
  k_to_work_b<<<g, 256, 0, s>>>(v, 2 * Np, S, m->d_perm.p, m->nc, ncp, a.buf[B_V]);
  k_to_work_b<<<g, 256, 0, s>>>(sigma, 3 * Np, S, m->d_perm.p, m->nc, ncp, a.buf[B_S]);
  tm.end(s);
  SLT_CUDA(cudaGetLastError());
  switch (m->p) {
    case 1: run_batched<1>(m, sched, a, nsteps, s, tm); break;
    case 2: run_batched<2>(m, sched, a, nsteps, s, tm); break;
    case 3: run_batched<3>(m, sched, a, nsteps, s, tm); break;
    case 4: run_batched<4>(m, sched, a, nsteps, s, tm); break;
  }
  tm.begin(s, 2, 1);
  k_from_work_b<<<g, 256, 0, s>>>(a.buf[B_V], 2 * Np, S, m->d_perm.p, m->nc, ncp, v);
  k_from_work_b<<<g, 256, 0, s>>>(a.buf[B_S], 3 * Np, S, m->d_perm.p, m->nc, ncp, sigma);
  tm.end(s);
  SLT_CUDA(cudaGetLastError());
  if (tm.on) {
    SLT_CUDA(cudaStreamSynchronize(s));
    double tot[3] = {0, 0, 0}, cnt[3] = {0, 0, 0}, mx = 0, mn = 1e300;
    const size_t npairs = tm.nl.size();
    for (size_t i = 0; i < npairs; ++i) {
      float ms = 0;
      SLT_CUDA(cudaEventElapsedTime(&ms, tm.ev[2 * i], tm.ev[2 * i + 1]));
      const int cls = tm.cls[i];
      tot[cls] += ms;
      cnt[cls] += tm.nl[i];
      if (!cls) { mx = std::max(mx, (double)ms); mn = std::min(mn, (double)ms); }
    }
    for (cudaEvent_t e : tm.ev) cudaEventDestroy(e);
    profile[0] = tot[0]; profile[1] = cnt[0]; profile[2] = tot[1]; profile[3] = cnt[1];
    profile[4] = cnt[0] ? mx : 0; profile[5] = cnt[0] ? mn : 0; profile[6] = tot[2]; profile[7] = cnt[2];
  }
}

}  // namespace slt
