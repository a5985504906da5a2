// Autotuner: tile size, tile shape and CTA size chosen by timing the candidates on the mesh
// itself (the paper finds the best tile size and shape depend on the mesh and the degree, and
// searches for them empirically, Section 7.3).  Candidates run with zero fields and no source:
// the executors' arithmetic and memory traffic do not depend on the field values.
#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "internal.h"

namespace slt {

namespace {

struct Fields {
  DevBuf<double> v, s;
};

// kernel time per step of `steps` steps after `warm` untimed steps
double time_candidate(slt_mesh m, slt_schedule sched, int32_t nshots, Fields& f, const int32_t* d_src_w,
                      const double* d_src, int steps, int warm, cudaStream_t s) {
  double prof[8] = {0};
  if (nshots == 1) {
    exec_run(m, sched, f.v.p, f.s.p, nullptr, 1e-3, warm, s);
    exec_run(m, sched, f.v.p, f.s.p, nullptr, 1e-3, steps, s, prof);
  } else {
    exec_run_batched(m, sched, nshots, d_src_w, d_src, f.v.p, f.s.p, nullptr, 1e-3, warm, s, nullptr);
    exec_run_batched(m, sched, nshots, d_src_w, d_src, f.v.p, f.s.p, nullptr, 1e-3, steps, s, prof);
  }
  SLT_CUDA(cudaStreamSynchronize(s));
  return prof[0] / steps;
}

}  // namespace

void autotune(slt_mesh m, const slt_options& base, int32_t nshots, const int32_t* tile_sizes, int32_t ntile,
              int32_t shapes, const int32_t* blocks, int32_t nblock, const int32_t* groups, int32_t ngroup,
              int32_t steps, cudaStream_t s, slt_options* best, double* table) {
  const int64_t per = (int64_t)m->nc * m->Np * nshots;
  Fields f;
  f.v.alloc(2 * per);
  f.s.alloc(3 * per);
  SLT_CUDA(cudaMemsetAsync(f.v.p, 0, 2 * per * sizeof(double), s));
  SLT_CUDA(cudaMemsetAsync(f.s.p, 0, 3 * per * sizeof(double), s));
  DevBuf<int32_t> src_w(nshots);
  DevBuf<double> src((size_t)nshots * m->Np);
  {
    std::vector<int32_t> hw(nshots, -1);
    src_w.upload(hw.data(), nshots, s);
    SLT_CUDA(cudaMemsetAsync(src.p, 0, (size_t)nshots * m->Np * sizeof(double), s));
  }
  const int warm = 2;
  slt_chain chain = nullptr;
  if (slt_mesh_chain(m, &chain) != SLT_OK) fail(SLT_ERR_STATE, "could not build the mesh's chain");
  std::unique_ptr<slt_chain_s, int (*)(slt_chain)> chain_guard(chain, slt_chain_destroy);

  *best = base;
  best->tile_size = 0;
  double best_ms = time_candidate(m, nullptr, nshots, f, src_w.p, src.p, steps, warm, s);
  int row = 0;
  auto put = [&](int32_t ts, int32_t rn, int32_t bt, int32_t g, double ms) {
    if (table) {
      table[5 * row + 0] = ts;
      table[5 * row + 1] = rn;
      table[5 * row + 2] = bt;
      table[5 * row + 3] = g;
      table[5 * row + 4] = ms;
    }
    ++row;
  };
  put(0, 0, 0, 0, best_ms);
  // shots per CTA only matter for several shots
  const int32_t one_group = 0;
  if (nshots == 1 || ngroup == 0) {
    groups = &one_group;
    ngroup = 1;
  }
  const int nshape = shapes ? 2 : 1;
  for (int i = 0; i < ntile; ++i)
    for (int r = 0; r < nshape; ++r)
      for (int b = 0; b < nblock; ++b) {
        slt_options o = base;
        o.tile_size = tile_sizes[i];
        o.renumber = r == 0 ? 1 : 0;
        o.block_threads = blocks[b];
        slt_schedule sched = nullptr;
        int rc = slt_inspect(chain, &o, s, &sched);
        if (rc != SLT_OK) fail(rc, "autotune: inspection of a candidate failed");
        std::unique_ptr<slt_schedule_s, int (*)(slt_schedule)> guard(sched, slt_schedule_destroy);
        bool serial = false;
        for (const SubSched& sub : sched->subs) serial |= sub.fell_back != 0 && sub.m > 1;
        for (int k = 0; k < ngroup; ++k) {
          o.shots_per_cta = groups[k];
          if (serial && o.colouring == 0) {
            put(o.tile_size, o.renumber, o.block_threads, o.shots_per_cta, -1.0);
            continue;
          }
          sched->shots_per_cta = o.shots_per_cta;  // an executor setting: no new inspection
          double ms = time_candidate(m, sched, nshots, f, src_w.p, src.p, steps, warm, s);
          put(o.tile_size, o.renumber, o.block_threads, o.shots_per_cta, ms);
          if (ms < best_ms) {
            best_ms = ms;
            *best = o;
          }
        }
      }
}

}  // namespace slt
