// C ABI of libslt.so: argument validation, object lifetimes, mesh set-up and the elastic chain.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <set>
#include <vector>

#include "internal.h"

namespace slt {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    fail(SLT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

}  // namespace slt

using namespace slt;

#define API_BEGIN try {
#define API_END                                             \
  }                                                         \
  catch (const slt::Error& e) {                             \
    slt::set_error(e.msg);                                  \
    return e.code;                                          \
  }                                                         \
  catch (const std::bad_alloc&) {                           \
    slt::set_error("host allocation failed");               \
    return SLT_ERR_OOM;                                     \
  }                                                         \
  catch (...) {                                             \
    slt::set_error("unexpected exception");                 \
    return SLT_ERR_CUDA;                                    \
  }                                                         \
  return SLT_OK;

#define REQUIRE(cond, msg) \
  do {                     \
    if (!(cond)) fail(SLT_ERR_ARG, msg); \
  } while (0)

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// Smallest cell id whose barycentric coordinates of xy are all >= -1e-12; (r, s) reference
// coordinates.  Returns -1 when no cell contains the point.
static int64_t locate(slt_mesh m, const double* xy, double* r, double* t) {
  for (int64_t c = 0; c < m->nc; ++c) {
    const double* a = &m->affine[7 * c];
    double dx = xy[0] - a[0], dy = xy[1] - a[1];
    double rr = a[2] * dx + a[3] * dy, tt = a[4] * dx + a[5] * dy;
    if (rr >= -1e-12 && tt >= -1e-12 && 1.0 - rr - tt >= -1e-12) {
      *r = rr;
      *t = tt;
      return c;
    }
  }
  return -1;
}

// Point source M_K^-1 phi(x_s) in the cell containing x_s (NULL: no source).
// Point source at xy: its cell (caller numbering) and the coefficients M^{-1} phi(xy) / |det J|
// of the nodal load in that cell (the DG form of a Dirac load, Section 7.1 source term).
static int64_t source_coeffs(slt_mesh m, const double* xy, double* coef) {
  REQUIRE(std::isfinite(xy[0]) && std::isfinite(xy[1]), "source position must be finite");
  double r = 0, t = 0;
  int64_t c = locate(m, xy, &r, &t);
  REQUIRE(c >= 0, "a source lies outside the mesh");
  std::vector<double> phi = m->ref.eval(r, t);
  for (int i = 0; i < m->Np; ++i) {
    double acc = 0.0;
    for (int j = 0; j < m->Np; ++j) acc += m->ref.Minv[i * m->Np + j] * phi[j];
    coef[i] = acc / m->affine[7 * c + 6];
  }
  return c;
}

static void set_source(slt_mesh m, const double* src_xy, cudaStream_t s) {
  std::vector<double> hsrc(m->Np, 0.0);
  m->src_cell = -1;
  m->src_w = -1;
  if (src_xy) {
    int64_t c = source_coeffs(m, src_xy, hsrc.data());
    m->src_cell = c;
    m->src_w = m->iperm[c];
  }
  m->src.upload(hsrc.data(), m->Np, s);
  SLT_CUDA(cudaStreamSynchronize(s));
}

extern "C" {

const char* slt_last_error(void) { return g_err.c_str(); }

int slt_version(int32_t* major, int32_t* minor, int32_t* arch) {
  API_BEGIN
  if (major) *major = 1;
  if (minor) *minor = 0;
  if (arch) *arch = 103;
  API_END
}

// ------------------------------------------------------------------ loop chain
int slt_chain_create(slt_chain* out) {
  API_BEGIN
  REQUIRE(out, "out is null");
  *out = new slt_chain_s();
  API_END
}

int slt_chain_destroy(slt_chain chain) {
  API_BEGIN
  delete chain;
  API_END
}

int slt_set(slt_chain c, int64_t size, int32_t* set_id) {
  API_BEGIN
  REQUIRE(c && set_id, "null argument");
  REQUIRE(size >= 0 && size < (int64_t(1) << 31), "set size must be in [0, 2^31)");
  c->set_size.push_back(size);
  c->points.emplace_back();
  *set_id = (int32_t)c->set_size.size() - 1;
  API_END
}

int slt_map(slt_chain c, int32_t from_set, int32_t to_set, int32_t arity, const int32_t* host_values, int32_t* map_id) {
  API_BEGIN
  REQUIRE(c && map_id, "null argument");
  const int32_t ns = (int32_t)c->set_size.size();
  REQUIRE(from_set >= 0 && from_set < ns && to_set >= 0 && to_set < ns, "unknown set");
  REQUIRE(arity >= 1 && arity <= 64, "arity must be in 1..64");
  const int64_t n = c->set_size[from_set] * (int64_t)arity;
  REQUIRE(n < (int64_t(1) << 31), "map too large");
  REQUIRE(host_values || n == 0, "values are null");
  MapH M{from_set, to_set, arity, std::vector<int32_t>(host_values, host_values + n)};
  for (int32_t v : M.values) REQUIRE(v >= 0 && v < c->set_size[to_set], "map value outside the target set");
  c->maps.push_back(std::move(M));
  *map_id = (int32_t)c->maps.size() - 1;
  API_END
}

int slt_loop(slt_chain c, int32_t set_id, int32_t ndesc, const int32_t* map_ids, const char* modes, int32_t* loop_id) {
  API_BEGIN
  REQUIRE(c && loop_id && map_ids && modes, "null argument");
  REQUIRE(set_id >= 0 && set_id < (int32_t)c->set_size.size(), "unknown set");
  REQUIRE(ndesc >= 1 && ndesc <= 8, "ndesc must be in 1..8");
  LoopH L{set_id, {}, -1};
  for (int d = 0; d < ndesc; ++d) {
    REQUIRE(modes[d] == 'r' || modes[d] == 'w' || modes[d] == 'i', "mode must be r, w or i");
    REQUIRE(map_ids[d] >= -1 && map_ids[d] < (int32_t)c->maps.size(), "unknown map");
    if (map_ids[d] >= 0) REQUIRE(c->maps[map_ids[d]].from == set_id, "map does not start at the loop's set");
    L.descs.push_back({map_ids[d], modes[d]});
  }
  c->loops.push_back(std::move(L));
  *loop_id = (int32_t)c->loops.size() - 1;
  API_END
}

int slt_set_points(slt_chain c, int32_t set_id, const double* xy) {
  API_BEGIN
  REQUIRE(c && xy, "null argument");
  REQUIRE(set_id >= 0 && set_id < (int32_t)c->set_size.size(), "unknown set");
  const int64_t n = c->set_size[set_id];
  for (int64_t i = 0; i < 2 * n; ++i) REQUIRE(std::isfinite(xy[i]), "points must be finite");
  c->points[set_id].assign(xy, xy + 2 * n);
  API_END
}

int slt_chain_info(slt_chain c, int32_t* nsets, int32_t* nmaps, int32_t* nloops) {
  API_BEGIN
  REQUIRE(c, "null chain");
  if (nsets) *nsets = (int32_t)c->set_size.size();
  if (nmaps) *nmaps = (int32_t)c->maps.size();
  if (nloops) *nloops = (int32_t)c->loops.size();
  API_END
}

// ------------------------------------------------------------------ inspector
int slt_options_default(slt_options* o) {
  API_BEGIN
  REQUIRE(o, "null options");
  std::memset(o, 0, sizeof(*o));
  o->tile_size = 1024;
  o->colouring = 0;
  o->renumber = 1;
  o->max_rounds = 16;
  o->prio_seed = 0x5EED;
  o->nsplit = 0;
  o->executor = 0;
  API_END
}

int slt_inspect(slt_chain c, const slt_options* opt, void* stream, slt_schedule* out) {
  API_BEGIN
  REQUIRE(c && opt && out, "null argument");
  *out = nullptr;
  REQUIRE(!c->loops.empty(), "the chain has no loop");
  REQUIRE(opt->tile_size >= 1, "tile_size must be >= 1");
  for (int k = 0; k < 16; ++k) REQUIRE(opt->sub_tile_size[k] >= 0, "sub_tile_size entries must be >= 0");
  REQUIRE(opt->colouring == 0 || opt->colouring == 1, "colouring must be 0 or 1");
  REQUIRE(opt->renumber == 0 || opt->renumber == 1, "renumber must be 0 or 1");
  REQUIRE(opt->max_rounds >= 0, "max_rounds must be >= 0");
  REQUIRE(opt->nsplit >= 0 && opt->nsplit <= 15, "nsplit must be in 0..15");
  REQUIRE(opt->executor >= 0 && opt->executor <= 4, "executor must be 0 to 4");
  REQUIRE(opt->cluster_size >= 0 && opt->cluster_size <= 8, "cluster_size must be in 0..8");
  REQUIRE(opt->wait_spins >= 0, "wait_spins must be >= 0");
  REQUIRE(opt->shots_per_cta >= 0, "shots_per_cta must be >= 0");
  REQUIRE(opt->release_order >= 0 && opt->release_order <= 2, "release_order must be 0, 1 or 2");
  REQUIRE(opt->block_threads == 0 || opt->block_threads == 128 || opt->block_threads == 256 ||
              opt->block_threads == 384 || opt->block_threads == 512 || opt->block_threads == 768,
          "block_threads must be 0, 128, 256, 384, 512 or 768");
  REQUIRE(opt->block_threads <= 384 || opt->executor == 0 || opt->executor == 3,
          "512- and 768-thread tiles are for the dataflow executors (executors 0 and 3)");
  REQUIRE((opt->executor != 3 && opt->executor != 4) || c->mesh,
          "the staged and pass executors run the elastic chain of a mesh");
  const int nl = (int)c->loops.size();
  int prev = 0;
  for (int k = 0; k < opt->nsplit; ++k) {
    REQUIRE(opt->split[k] > prev && opt->split[k] < nl, "split points must increase strictly inside (0, nloops)");
    prev = opt->split[k];
  }
  std::vector<int> starts = {0};
  for (int k = 0; k < opt->nsplit; ++k) starts.push_back(opt->split[k]);
  for (size_t k = 0; k < starts.size(); ++k) {
    const int end = k + 1 < starts.size() ? starts[k + 1] : nl;
    REQUIRE(opt->seed_loop[k] >= 0 && opt->seed_loop[k] < end - starts[k],
            "seed_loop[k] must lie inside sub-chain k");
    const int st = starts[k] + opt->seed_loop[k];
    int seed_set = c->loops[st].set;
    if (opt->renumber)
      REQUIRE((int64_t)c->points[seed_set].size() == 2 * c->set_size[seed_set],
              "renumber = 1 needs points on the seed set");
  }
  std::unique_ptr<slt_schedule_s> s(new slt_schedule_s());
  s->loops = c->loops;
  for (const MapH& M : c->maps) s->maps_meta.push_back({M.from, M.to, M.arity, {}});
  s->set_size = c->set_size;
  s->mesh = c->mesh;
  s->executor = opt->executor;
  // staged executor: temporaries stay in shared memory unless another tile reads them; with a
  // fusion other than {all loops} or {velocity, stress} some are read by a later sub-chain, so
  // every temporary is then written out as well
  s->stage_cross = !(opt->nsplit == 0 || (opt->nsplit == 1 && opt->split[0] == 9));
  if (opt->wait_spins > 0) s->wait_spins = opt->wait_spins;
  s->keep = opt->release_order == 1 || (opt->release_order == 0 && opt->executor == 3);
  if (opt->block_threads) s->block = opt->block_threads;
  s->shots_per_cta = opt->shots_per_cta;
  if (opt->cluster_size) s->cluster = opt->cluster_size;
  inspect_chain(c, *opt, as_stream(stream), s.get());
  *out = s.release();
  API_END
}

int slt_schedule_destroy(slt_schedule s) {
  API_BEGIN
  delete s;
  API_END
}

int slt_schedule_info(slt_schedule s, int32_t sub, int64_t info[8]) {
  API_BEGIN
  REQUIRE(s && info, "null argument");
  REQUIRE(sub >= 0 && sub < (int32_t)s->subs.size(), "unknown sub-chain");
  const SubSched& S = s->subs[sub];
  info[0] = S.m;
  info[1] = S.ncolours;
  info[2] = S.restarts;
  info[3] = S.fell_back;
  info[4] = S.conflicts;
  info[5] = S.unprojected;
  info[6] = S.first;
  info[7] = S.last - S.first;
  API_END
}

int slt_schedule_dataflow_info(slt_schedule s, double info[6]) {
  API_BEGIN
  REQUIRE(s && info, "null argument");
  const DataflowPlan& D = s->df;
  REQUIRE(!D.cum.empty(), "the schedule has no executor plan (not inspected on a mesh chain)");
  info[0] = D.cum.back();
  info[1] = (double)D.ndeps;
  info[2] = D.cp_nodes;
  info[3] = D.cp_items;
  info[4] = D.items_per_step;
  info[5] = (double)D.last_grid;
  API_END
}

int slt_schedule_inspection_times(slt_schedule s, double seconds[8]) {
  API_BEGIN
  REQUIRE(s && seconds, "null argument");
  for (int k = 0; k < 8; ++k) seconds[k] = s->insp_s[k];
  API_END
}

int slt_schedule_lane_info(slt_schedule s, double info[4]) {
  API_BEGIN
  REQUIRE(s && info, "null argument");
  REQUIRE(s->mesh && !s->df.cum.empty(), "the schedule has no executor plan (not inspected on a mesh chain)");
  lane_info(s, s->mesh, info);
  API_END
}

int slt_schedule_export(slt_schedule s, int32_t kind, int32_t loop, int32_t desc, int32_t* host_out, int64_t* n) {
  API_BEGIN
  REQUIRE(s && n, "null argument");
  REQUIRE(kind >= 0 && kind <= 14, "unknown kind");
  if (kind == 14) {  // export flags of loop `loop`
    REQUIRE(loop >= 0 && loop < (int32_t)s->loops.size(), "unknown loop");
    const int64_t len = s->set_size[s->loops[loop].set];
    *n = len;
    if (host_out && len) {
      DevBuf<int32_t> f;
      export_flags(s, loop, f, nullptr);
      SLT_CUDA(cudaMemcpy(host_out, f.p, len * 4, cudaMemcpyDeviceToHost));
    }
    return SLT_OK;
  }
  if (kind == 12 || kind == 13) {  // the staged executor's tile footprints of sub-chain `loop`
    REQUIRE(loop >= 0 && loop < (int32_t)s->subs.size(), "unknown sub-chain");
    const SubSched& S = s->subs[loop];
    REQUIRE(S.fp_ptr.p, "the schedule has no staged plan (inspect with executor 3)");
    if (kind == 12) {
      *n = S.m + 1;
      if (host_out) SLT_CUDA(cudaMemcpy(host_out, S.fp_ptr.p, (S.m + 1) * 4, cudaMemcpyDeviceToHost));
    } else {
      int32_t tot = 0;
      SLT_CUDA(cudaMemcpy(&tot, S.fp_ptr.p + S.m, 4, cudaMemcpyDeviceToHost));
      *n = tot;
      if (host_out && tot) {
        std::vector<int32_t> w = S.fp_cell.download(nullptr, tot);
        for (int32_t i = 0; i < tot; ++i) host_out[i] = s->mesh->perm[w[i] & 0x7fffffff];
      }
    }
    return SLT_OK;
  }
  if (kind >= 8) {  // the dataflow executor's dependency graph
    const DataflowPlan& D = s->df;
    REQUIRE(!D.cum.empty(), "the schedule has no executor plan (not inspected on a mesh chain)");
    const int32_t G = D.cum.back();
    const int32_t* src = kind == 8 ? D.succ_ptr.p : kind == 9 ? D.succ.p : kind == 10 ? D.indeg0.p : D.indeg.p;
    const int64_t len = kind == 8 ? G + 1 : kind == 9 ? D.ndeps : G;
    *n = len;
    if (host_out && len) SLT_CUDA(cudaMemcpy(host_out, src, len * 4, cudaMemcpyDeviceToHost));
    return SLT_OK;
  }
  SubSched* S = nullptr;
  int jj = 0;
  if (kind <= 1) {
    REQUIRE(loop >= 0 && loop < (int32_t)s->subs.size(), "unknown sub-chain");
    S = &s->subs[loop];
  } else {
    REQUIRE(loop >= 0 && loop < (int32_t)s->loops.size(), "unknown loop");
    for (SubSched& x : s->subs)
      if (loop >= x.first && loop < x.last) { S = &x; jj = loop - x.first; }
    REQUIRE(S, "loop not inspected");
  }
  const int32_t* src = nullptr;
  int64_t len = 0;
  const LoopH* L = kind >= 2 ? &s->loops[loop] : nullptr;
  switch (kind) {
    case 0: src = S->rank.p; len = s->set_size[s->loops[S->first + S->seed].set]; break;
    case 1: src = S->colour.p; len = S->m; break;
    case 2: src = S->sigma[jj].p; len = s->set_size[L->set]; break;
    case 3: src = S->list_ptr[jj].p; len = S->m + 1; break;
    case 4: src = S->list[jj].p; len = s->set_size[L->set]; break;
    default: {
      REQUIRE(desc >= 0 && desc < (int32_t)L->descs.size() && L->descs[desc].map >= 0,
              "desc must name an indirect descriptor");
      ensure_local_maps(s, *S, jj, nullptr);
      const LocalMap& lm = S->lmaps[jj][desc];
      if (kind == 5) { src = lm.fp_ptr.p; len = S->m + 1; }
      else if (kind == 6) {
        int32_t tot = 0;
        SLT_CUDA(cudaMemcpy(&tot, lm.fp_ptr.p + S->m, 4, cudaMemcpyDeviceToHost));
        src = lm.fp.p;
        len = tot;
      } else { src = lm.lmap.p; len = s->set_size[L->set] * (int64_t)s->maps_meta[L->descs[desc].map].arity; }
    }
  }
  *n = len;
  if (host_out && len) SLT_CUDA(cudaMemcpy(host_out, src, len * 4, cudaMemcpyDeviceToHost));
  API_END
}

// ------------------------------------------------------------------ mesh
int slt_mesh_create(const int32_t* cell2vert, const double* cellxy, int64_t nc, int32_t degree, const double* rho,
                    const double* lam, const double* mu, const double* src_xy, void* stream, slt_mesh* out) {
  API_BEGIN
  REQUIRE(out, "out is null");
  *out = nullptr;
  REQUIRE(cell2vert && cellxy && rho && lam && mu, "null argument");
  REQUIRE(nc >= 1 && nc < (int64_t(1) << 28), "ncell must be in [1, 2^28)");
  REQUIRE(degree >= 1 && degree <= 4, "degree must be in 1..4");
  cudaStream_t s = as_stream(stream);
  std::unique_ptr<slt_mesh_s> m(new slt_mesh_s());
  m->nc = nc;
  m->ncp = (nc + 63) / 64 * 64;
  m->p = degree;
  m->ref = make_refelem(degree);
  m->Np = m->ref.Np;
  m->Nfp = m->ref.Nfp;
  for (int64_t i = 0; i < 3 * nc; ++i) REQUIRE(cell2vert[i] >= 0, "negative vertex id");
  for (int64_t i = 0; i < 6 * nc; ++i) REQUIRE(std::isfinite(cellxy[i]), "coordinates must be finite");
  for (int64_t c = 0; c < nc; ++c) {
    REQUIRE(std::isfinite(rho[c]) && rho[c] > 0, "rho must be finite and positive");
    REQUIRE(std::isfinite(lam[c]) && std::isfinite(mu[c]), "lambda and mu must be finite");
  }
  // facets: (min vertex, max vertex, cell, local face, start vertex), sorted by key then cell
  struct Ent { int32_t lo, hi, cell, face, start; };
  std::vector<Ent> ent(3 * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int f = 0; f < 3; ++f) {
      int32_t a = cell2vert[3 * c + f], b = cell2vert[3 * c + (f + 1) % 3];
      REQUIRE(a != b, "a cell repeats a vertex");
      ent[3 * c + f] = {std::min(a, b), std::max(a, b), (int32_t)c, f, a};
    }
  std::sort(ent.begin(), ent.end(), [](const Ent& x, const Ent& y) {
    if (x.lo != y.lo) return x.lo < y.lo;
    if (x.hi != y.hi) return x.hi < y.hi;
    return x.cell < y.cell;
  });
  std::vector<std::array<int32_t, 3>> nbr_c(nc, {-1, -1, -1});   // neighbour cell, caller numbering
  std::vector<std::array<int8_t, 3>> nbr_f(nc), nbr_flip(nc);
  for (size_t i = 0; i < ent.size();) {
    size_t j = i + 1;
    while (j < ent.size() && ent[j].lo == ent[i].lo && ent[j].hi == ent[i].hi) ++j;
    REQUIRE(j - i <= 2, "an edge is shared by more than two cells");
    if (j - i == 2) {
      const Ent &A = ent[i], &B = ent[i + 1];
      REQUIRE(A.cell != B.cell, "a cell touches the same edge twice");
      int8_t flip = A.start != B.start;
      m->f2c.push_back(A.cell);
      m->f2c.push_back(B.cell);
      m->f2f.push_back((int8_t)A.face);
      m->f2f.push_back((int8_t)B.face);
      nbr_c[A.cell][A.face] = B.cell; nbr_f[A.cell][A.face] = (int8_t)B.face; nbr_flip[A.cell][A.face] = flip;
      nbr_c[B.cell][B.face] = A.cell; nbr_f[B.cell][B.face] = (int8_t)A.face; nbr_flip[B.cell][B.face] = flip;
    } else {
      m->e2c.push_back(ent[i].cell);
      m->e2f.push_back((int8_t)ent[i].face);
    }
    i = j;
  }
  // facet midpoints (x_a + x_b) * 0.5 from the first listed cell, points of the facet sets
  auto midpoint = [&](int32_t c, int f, std::vector<double>& out) {
    const double* X = cellxy + 6 * (int64_t)c;
    out.push_back((X[2 * f] + X[2 * ((f + 1) % 3)]) * 0.5);
    out.push_back((X[2 * f + 1] + X[2 * ((f + 1) % 3) + 1]) * 0.5);
  };
  for (size_t k = 0; k < m->f2c.size() / 2; ++k) midpoint(m->f2c[2 * k], m->f2f[2 * k], m->fmid);
  for (size_t k = 0; k < m->e2c.size(); ++k) midpoint(m->e2c[k], m->e2f[k], m->emid);
  m->nfi = (int64_t)m->f2c.size() / 2;
  m->nfe = (int64_t)m->e2c.size();
  for (int64_t c = 0; c < nc; ++c) {
    bool in = false, ex = false;
    for (int f = 0; f < 3; ++f) (nbr_c[c][f] >= 0 ? in : ex) = true;
    m->cells_int += in;
    m->cells_ext += ex;
  }
  // geometry (caller numbering)
  std::vector<double> rx(nc), ry(nc), sx(nc), sy(nc), adet(nc), fg(9 * nc);
  m->centroid.resize(2 * nc);
  m->affine.resize(7 * nc);
  for (int64_t c = 0; c < nc; ++c) {
    const double* X = cellxy + 6 * c;
    double j11 = X[2] - X[0], j21 = X[3] - X[1], j12 = X[4] - X[0], j22 = X[5] - X[1];
    double det = j11 * j22 - j12 * j21;
    REQUIRE(det != 0.0 && std::isfinite(det), "degenerate cell");
    rx[c] = j22 / det; ry[c] = -j12 / det; sx[c] = -j21 / det; sy[c] = j11 / det;
    adet[c] = std::fabs(det);
    const double aff[7] = {X[0], X[1], rx[c], ry[c], sx[c], sy[c], adet[c]};
    std::copy(aff, aff + 7, m->affine.begin() + 7 * c);
    for (int f = 0; f < 3; ++f) {
      const double *P = X + 2 * f, *Q = X + 2 * ((f + 1) % 3), *O = X + 2 * ((f + 2) % 3);
      double tx = Q[0] - P[0], ty = Q[1] - P[1];
      double len = std::hypot(tx, ty);
      double nx = ty / len, ny = -tx / len;
      if (nx * (O[0] - P[0]) + ny * (O[1] - P[1]) > 0) { nx = -nx; ny = -ny; }
      fg[9 * c + 3 * f] = nx;
      fg[9 * c + 3 * f + 1] = ny;
      fg[9 * c + 3 * f + 2] = len / adet[c];
    }
    m->centroid[2 * c] = ((X[0] + X[2]) + X[4]) / 3.0;
    m->centroid[2 * c + 1] = ((X[1] + X[3]) + X[5]) / 3.0;
  }
  // work order: Hilbert order of the centroids
  {
    DevBuf<double> xy(2 * nc);
    xy.upload(m->centroid.data(), 2 * nc, s);
    DevBuf<int32_t> rank(nc);
    seed_rank(xy.p, nc, 1, rank.p, s);
    m->iperm = rank.download(s);
    m->perm.assign(nc, 0);
    for (int64_t c = 0; c < nc; ++c) m->perm[m->iperm[c]] = (int32_t)c;
  }
  const int64_t ncp = m->ncp;
  std::vector<double> hgeo(4 * ncp, 0.0), hfgeo(9 * ncp, 0.0), hmat(3 * ncp, 0.0);
  std::vector<int32_t> hnbr(3 * ncp, -1);
  for (int64_t w = 0; w < nc; ++w) {
    int64_t c = m->perm[w];
    hgeo[w] = rx[c]; hgeo[ncp + w] = ry[c]; hgeo[2 * ncp + w] = sx[c]; hgeo[3 * ncp + w] = sy[c];
    for (int q = 0; q < 9; ++q) hfgeo[q * ncp + w] = fg[9 * c + q];
    hmat[w] = 1.0 / rho[c]; hmat[ncp + w] = lam[c]; hmat[2 * ncp + w] = mu[c];
    for (int f = 0; f < 3; ++f)
      if (nbr_c[c][f] >= 0)
        hnbr[f * ncp + w] = (m->iperm[nbr_c[c][f]] << 3) | (nbr_f[c][f] << 1) | nbr_flip[c][f];
  }
  m->geo.alloc(4 * ncp); m->geo.upload(hgeo.data(), 4 * ncp, s);
  m->fgeo.alloc(9 * ncp); m->fgeo.upload(hfgeo.data(), 9 * ncp, s);
  m->mat.alloc(3 * ncp); m->mat.upload(hmat.data(), 3 * ncp, s);
  build_pre(m.get(), s);
  m->nbr.alloc(3 * ncp); m->nbr.upload(hnbr.data(), 3 * ncp, s);
  m->d_perm.alloc(nc); m->d_perm.upload(m->perm.data(), nc, s);
  {
    std::vector<double> hdet(ncp, 0.0);
    for (int64_t w = 0; w < nc; ++w) hdet[w] = adet[m->perm[w]];
    m->adet.alloc(ncp);
    m->adet.upload(hdet.data(), ncp, s);
  }
  m->d_iperm.alloc(nc); m->d_iperm.upload(m->iperm.data(), nc, s);
  m->src.alloc(m->Np);
  set_source(m.get(), src_xy, s);
  upload_constants(m->ref);
  upload_constants_batched(m->ref);
  upload_adjoint_constants(m->ref);
  m->work.alloc(15 * (int64_t)m->Np * ncp);
  SLT_CUDA(cudaMemsetAsync(m->work.p, 0, 15 * (int64_t)m->Np * ncp * sizeof(double), s));
  SLT_CUDA(cudaStreamSynchronize(s));
  *out = m.release();
  API_END
}

int slt_mesh_destroy(slt_mesh m) {
  API_BEGIN
  delete m;
  API_END
}

int slt_mesh_info(slt_mesh m, int64_t info[8]) {
  API_BEGIN
  REQUIRE(m && info, "null argument");
  info[0] = m->nc;
  info[1] = m->p;
  info[2] = m->Np;
  info[3] = m->nfi;
  info[4] = m->nfe;
  info[5] = m->src_cell;
  info[6] = 17;
  info[7] = 9;
  API_END
}

int slt_mesh_cost(slt_mesh m, double cost[4]) {
  API_BEGIN
  REQUIRE(m && cost, "null argument");
  const double Np = m->Np, Nfp = m->Nfp;
  double mx = 0.0;
  for (double x : m->ref.Dr) mx = std::fmax(mx, std::fabs(x));
  for (double x : m->ref.Ds) mx = std::fmax(mx, std::fabs(x));
  double nnz = 0.0;
  for (double x : m->ref.Dr) nnz += std::fabs(x) > 1e-12 * mx;
  for (double x : m->ref.Ds) nnz += std::fabs(x) > 1e-12 * mx;
  // FP64 flops of the kernels in exec.cu (an FMA counts 2), structural zeros skipped; the
  // per-cell products of geometry and material (metric terms over rho, scaled face normals,
  // lambda + 2 mu) are computed once per mesh, not per step
  const double volB = 12 * Np + 4 * nnz, volD = 13 * Np + 4 * nnz, hookeB = 7 * Np + volB;
  const double cell = volB + 2 * hookeB + 3 * volD + 8 * Np + 19 * Np;
  const double side = (9 * Nfp + 4 * Np * Nfp) + (2 * Nfp + Np * (4 * Nfp + 6));
  const double ext = 2 + 6 * Nfp + 4 * Np * Nfp;
  // (the facet loops accumulate onto the loaded field values: no separate increment adds)
  cost[0] = m->nc * cell + 2.0 * m->nfi * 3 * side + m->nfe * 3 * ext;
  cost[1] = m->nc * (80 * Np + 140);
  cost[2] = m->nc * (808 * Np + 808);
  cost[3] = nnz;
  API_END
}

int slt_mesh_chain(slt_mesh m, slt_chain* out) {
  API_BEGIN
  REQUIRE(m && out, "null argument");
  std::unique_ptr<slt_chain_s> c(new slt_chain_s());
  c->set_size = {m->nc, m->nfi, m->nfe};
  c->points.resize(3);
  c->points[0] = m->centroid;
  c->points[1] = m->fmid;
  c->points[2] = m->emid;
  c->maps.push_back({1, 0, 2, m->f2c});
  c->maps.push_back({2, 0, 1, m->e2c});
  // (set, kernel) of the seventeen loops; cell loops: direct read + direct write (updates:
  // increment); facet loops: read and increment cells through their facet->cell map
  static const int32_t sets[17] = {0, 1, 2, 0, 1, 0, 1, 2, 0, 0, 1, 0, 1, 2, 0, 1, 0};
  static const int32_t kern[17] = {K_VOLB, K_INTB, K_EXTB, K_VOLD, K_INTD, K_HOOKEB, K_INTB, K_EXTB, K_UPDV,
                                   K_VOLD, K_INTD, K_HOOKEB, K_INTB, K_EXTB, K_VOLD, K_INTD, K_UPDS};
  for (int j = 0; j < 17; ++j) {
    LoopH L{sets[j], {}, kern[j]};
    if (sets[j] == 0) {
      L.descs.push_back({-1, 'r'});
      L.descs.push_back({-1, (kern[j] == K_UPDV || kern[j] == K_UPDS) ? 'i' : 'w'});
    } else {
      int mid = sets[j] == 1 ? 0 : 1;
      L.descs.push_back({mid, 'r'});
      L.descs.push_back({mid, 'i'});
    }
    c->loops.push_back(L);
  }
  c->mesh = m;
  *out = c.release();
  API_END
}

// ------------------------------------------------------------------ executor
int slt_execute(slt_mesh m, slt_schedule sched, double* v, double* sigma, const double* ricker, double dt,
                int64_t nsteps, void* stream) {
  API_BEGIN
  REQUIRE(m && v && sigma, "null argument");
  REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  REQUIRE(std::isfinite(dt), "dt must be finite");
  if (sched) {
    if (sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  }
  exec_run(m, sched, v, sigma, ricker, dt, nsteps, as_stream(stream));
  API_END
}

int slt_execute_profiled(slt_mesh m, slt_schedule sched, double* v, double* sigma, const double* ricker, double dt,
                         int64_t nsteps, void* stream, double profile[8]) {
  API_BEGIN
  REQUIRE(m && v && sigma && profile, "null argument");
  REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  REQUIRE(std::isfinite(dt), "dt must be finite");
  if (sched && sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  exec_run(m, sched, v, sigma, ricker, dt, nsteps, as_stream(stream), profile);
  API_END
}

int slt_execute_host(slt_mesh m, slt_schedule sched, double* hv, double* hs, const double* hr, double dt,
                     int64_t nsteps, void* stream) {
  API_BEGIN
  REQUIRE(m && hv && hs, "null argument");
  REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  REQUIRE(std::isfinite(dt), "dt must be finite");
  if (sched) {
    if (sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  }
  exec_run_host(m, sched, hv, hs, hr, dt, nsteps, as_stream(stream));
  API_END
}

int slt_mesh_set_source(slt_mesh m, const double* src_xy, void* stream) {
  API_BEGIN
  REQUIRE(m, "null mesh");
  set_source(m, src_xy, as_stream(stream));
  API_END
}

int slt_mesh_set_material(slt_mesh m, const double* rho, const double* lam, const double* mu, void* stream) {
  API_BEGIN
  REQUIRE(m && rho && lam && mu, "null argument");
  for (int64_t c = 0; c < m->nc; ++c) {
    REQUIRE(std::isfinite(rho[c]) && rho[c] > 0, "rho must be finite and positive");
    REQUIRE(std::isfinite(lam[c]) && std::isfinite(mu[c]) && mu[c] > 0 && lam[c] + mu[c] > 0,
            "lambda, mu must be finite with mu > 0 and lambda + mu > 0");
  }
  const int64_t ncp = m->ncp;
  std::vector<double> hmat(3 * ncp, 0.0);
  for (int64_t w = 0; w < m->nc; ++w) {
    int64_t c = m->perm[w];
    hmat[w] = 1.0 / rho[c];
    hmat[ncp + w] = lam[c];
    hmat[2 * ncp + w] = mu[c];
  }
  m->mat.upload(hmat.data(), 3 * ncp, as_stream(stream));
  build_pre(m, as_stream(stream));
  SLT_CUDA(cudaStreamSynchronize(as_stream(stream)));
  API_END
}

int slt_receivers_create(slt_mesh m, int32_t nrec, const double* xy, slt_receivers* out) {
  API_BEGIN
  REQUIRE(m && out && (xy || nrec == 0), "null argument");
  REQUIRE(nrec >= 0 && nrec <= 65536, "nrec must be in 0..65536");
  std::unique_ptr<slt_receivers_s> r(new slt_receivers_s());
  r->mesh = m;
  r->n = nrec;
  const int Np = m->Np;
  std::vector<int32_t> hw(std::max(nrec, 1));
  std::vector<double> hphi(std::max(nrec, 1) * Np), hq(std::max(nrec, 1) * Np);
  for (int32_t k = 0; k < nrec; ++k) {
    double rr = 0, tt = 0;
    REQUIRE(std::isfinite(xy[2 * k]) && std::isfinite(xy[2 * k + 1]), "receiver positions must be finite");
    int64_t c = locate(m, xy + 2 * k, &rr, &tt);
    REQUIRE(c >= 0, "a receiver lies outside the mesh");
    hw[k] = m->iperm[c];
    std::vector<double> phi = m->ref.eval(rr, tt);
    for (int i = 0; i < Np; ++i) {
      hphi[k * Np + i] = phi[i];
      double acc = 0.0;
      for (int j = 0; j < Np; ++j) acc += m->ref.Minv[i * Np + j] * phi[j];
      hq[k * Np + i] = acc / m->affine[7 * c + 6];
    }
  }
  r->w.alloc(hw.size());
  r->w.upload(hw.data(), hw.size(), nullptr);
  r->phi.alloc(hphi.size());
  r->phi.upload(hphi.data(), hphi.size(), nullptr);
  r->q.alloc(hq.size());
  r->q.upload(hq.data(), hq.size(), nullptr);
  SLT_CUDA(cudaStreamSynchronize(nullptr));
  *out = r.release();
  API_END
}

int slt_receivers_destroy(slt_receivers r) {
  API_BEGIN
  delete r;
  API_END
}

static void shot_sources(slt_mesh m, int32_t nshots, const double* src_xy, DevBuf<int32_t>& w, DevBuf<double>& c,
                         cudaStream_t s);

// the tiled adjoint runs one sub-chain at a time on the dataflow executor
static bool tiled_adjoint_ok(slt_schedule sched) {
  return sched->executor == 0 && sched->subs.size() == 2 && sched->subs[0].last == 9;
}

int slt_record(slt_mesh m, slt_schedule sched, slt_receivers rec, const double* ricker, double dt, int64_t nsteps,
               double* traces, void* stream) {
  API_BEGIN
  REQUIRE(m && rec && traces, "null argument");
  REQUIRE(rec->mesh == m, "the receivers belong to another mesh");
  REQUIRE(nsteps >= 0 && std::isfinite(dt), "nsteps >= 0 and finite dt required");
  if (sched && sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  record_run(m, sched, rec, ricker, dt, nsteps, traces, as_stream(stream));
  API_END
}

int slt_adjoint(slt_mesh m, slt_schedule sched, slt_receivers rec, const double* ricker, double dt, int64_t nsteps,
                const double* data, int32_t checkpoint_every, double* grad, double* misfit, void* stream) {
  API_BEGIN
  REQUIRE(m && rec && data && grad && misfit, "null argument");
  REQUIRE(rec->mesh == m, "the receivers belong to another mesh");
  REQUIRE(nsteps >= 1 && std::isfinite(dt), "nsteps >= 1 and finite dt required");
  REQUIRE(checkpoint_every != 0 && checkpoint_every != INT32_MIN, "checkpoint_every must be nonzero");
  if (sched && sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  if (sched && tiled_adjoint_ok(sched) && checkpoint_every > 0) {
    // the whole adjoint on the schedule's tiles: one shot of the chain-executor path
    cudaStream_t s = as_stream(stream);
    DevBuf<int32_t> w(1);
    const int32_t hw = m->src_w;
    w.upload(&hw, 1, s);
    DevBuf<double> coef(m->Np);
    if (m->src.p) SLT_CUDA(cudaMemcpyAsync(coef.p, m->src.p, m->Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else SLT_CUDA(cudaMemsetAsync(coef.p, 0, m->Np * sizeof(double), s));
    adjoint_run_b(m, sched, rec, 1, w.p, coef.p, ricker, dt, nsteps, data, checkpoint_every, grad, misfit, s);
  } else {
    adjoint_run(m, sched, rec, ricker, dt, nsteps, data, checkpoint_every, grad, misfit, as_stream(stream));
  }
  API_END
}

// per-shot source cells (work ids) and coefficients on the device
static void shot_sources(slt_mesh m, int32_t nshots, const double* src_xy, DevBuf<int32_t>& w, DevBuf<double>& c,
                         cudaStream_t s) {
  const int Np = m->Np;
  std::vector<int32_t> hw(nshots, -1);
  std::vector<double> hs((size_t)nshots * Np, 0.0);
  if (src_xy)
    for (int32_t k = 0; k < nshots; ++k) hw[k] = m->iperm[source_coeffs(m, src_xy + 2 * k, hs.data() + (size_t)k * Np)];
  w.alloc(nshots);
  c.alloc((size_t)nshots * Np);
  w.upload(hw.data(), nshots, s);
  c.upload(hs.data(), (size_t)nshots * Np, s);
}

int slt_record_batched(slt_mesh m, slt_schedule sched, slt_receivers rec, int32_t nshots, const double* src_xy,
                       const double* ricker, double dt, int64_t nsteps, double* traces, void* stream) {
  API_BEGIN
  REQUIRE(m && rec && traces, "null argument");
  REQUIRE(rec->mesh == m, "the receivers belong to another mesh");
  REQUIRE(nshots >= 1 && nshots <= 4096, "nshots must be in 1..4096");
  REQUIRE(nsteps >= 0 && std::isfinite(dt), "nsteps >= 0 and finite dt required");
  if (sched && sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  if (sched && sched->executor != 0) fail(SLT_ERR_UNSUPPORTED, "many shots run untiled or with executor 0");
  cudaStream_t s = as_stream(stream);
  DevBuf<int32_t> w;
  DevBuf<double> c;
  shot_sources(m, nshots, src_xy, w, c, s);
  record_run_b(m, sched, rec, nshots, w.p, c.p, ricker, dt, nsteps, traces, s);
  API_END
}

int slt_adjoint_batched(slt_mesh m, slt_schedule sched, slt_receivers rec, int32_t nshots, const double* src_xy,
                        const double* ricker, double dt, int64_t nsteps, const double* data, int32_t checkpoint_every,
                        double* grad, double* misfit, void* stream) {
  API_BEGIN
  REQUIRE(m && rec && data && grad && misfit, "null argument");
  REQUIRE(rec->mesh == m, "the receivers belong to another mesh");
  REQUIRE(nshots >= 1 && nshots <= 4096, "nshots must be in 1..4096");
  REQUIRE(nsteps >= 1 && std::isfinite(dt), "nsteps >= 1 and finite dt required");
  REQUIRE(checkpoint_every >= 1, "checkpoint_every must be >= 1");
  if (sched && sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  if (sched && !tiled_adjoint_ok(sched))
    fail(SLT_ERR_UNSUPPORTED, "the tiled adjoint needs executor 0 and the {velocity, stress} fusion (split at 9)");
  cudaStream_t s = as_stream(stream);
  DevBuf<int32_t> w;
  DevBuf<double> c;
  shot_sources(m, nshots, src_xy, w, c, s);
  adjoint_run_b(m, sched, rec, nshots, w.p, c.p, ricker, dt, nsteps, data, checkpoint_every, grad, misfit, s);
  API_END
}

int slt_execute_batched(slt_mesh m, slt_schedule sched, int32_t nshots, const double* src_xy, double* v,
                        double* sigma, const double* ricker, double dt, int64_t nsteps, void* stream,
                        double* profile) {
  API_BEGIN
  REQUIRE(m && v && sigma, "null argument");
  REQUIRE(nshots >= 1 && nshots <= 4096, "nshots must be in 1..4096");
  REQUIRE(nsteps >= 0 && std::isfinite(dt), "nsteps >= 0 and finite dt required");
  if (sched && sched->mesh != m) fail(SLT_ERR_STATE, "the schedule was not inspected on this mesh's chain");
  cudaStream_t s = as_stream(stream);
  const int Np = m->Np;
  std::vector<int32_t> hw(nshots, -1);
  std::vector<double> hs((size_t)nshots * Np, 0.0);
  if (src_xy)
    for (int32_t k = 0; k < nshots; ++k) hw[k] = m->iperm[source_coeffs(m, src_xy + 2 * k, hs.data() + (size_t)k * Np)];
  if (m->bsrc_w.n < (size_t)nshots) m->bsrc_w.alloc(nshots);
  if (m->bsrc.n < (size_t)nshots * Np) m->bsrc.alloc((size_t)nshots * Np);
  m->bsrc_w.upload(hw.data(), nshots, s);
  m->bsrc.upload(hs.data(), (size_t)nshots * Np, s);
  exec_run_batched(m, sched, nshots, m->bsrc_w.p, m->bsrc.p, v, sigma, ricker, dt, nsteps, s, profile);
  SLT_CUDA(cudaStreamSynchronize(s));
  API_END
}

int slt_group_create(int32_t n, const slt_mesh* meshes, const slt_schedule* scheds, slt_group* out) {
  API_BEGIN
  REQUIRE(out, "null argument");
  *out = nullptr;
  REQUIRE(n >= 1 && n <= 256, "n must be in 1..256");
  REQUIRE(meshes && scheds, "null argument");
  std::set<slt_mesh> seen;
  std::unique_ptr<slt_group_s> g(new slt_group_s());
  for (int32_t i = 0; i < n; ++i) {
    REQUIRE(meshes[i], "null mesh");
    REQUIRE(seen.insert(meshes[i]).second, "a mesh appears twice");
    if (scheds[i] && scheds[i]->mesh != meshes[i])
      fail(SLT_ERR_STATE, "a schedule was not inspected on its mesh's chain");
    g->meshes.push_back(meshes[i]);
    g->scheds.push_back(scheds[i]);
  }
  group_build(g.get());
  *out = g.release();
  API_END
}

int slt_group_create_batched(int32_t n, const slt_mesh* meshes, const slt_schedule* scheds, const int32_t* nshots,
                             const double* const* src_xy, slt_group* out) {
  API_BEGIN
  REQUIRE(out, "null argument");
  *out = nullptr;
  REQUIRE(n >= 1 && n <= 256, "n must be in 1..256");
  REQUIRE(meshes && scheds && nshots, "null argument");
  std::set<slt_mesh> seen;
  std::unique_ptr<slt_group_s> g(new slt_group_s());
  g->mixed = true;
  for (int32_t i = 0; i < n; ++i) {
    REQUIRE(meshes[i], "null mesh");
    REQUIRE(seen.insert(meshes[i]).second, "a mesh appears twice");
    REQUIRE(nshots[i] >= 1 && nshots[i] <= 4096, "nshots must be in 1..4096");
    if (scheds[i] && scheds[i]->mesh != meshes[i])
      fail(SLT_ERR_STATE, "a schedule was not inspected on its mesh's chain");
    if (nshots[i] > 1 && !(scheds[i] && scheds[i]->executor == 0))
      fail(SLT_ERR_UNSUPPORTED, "a member with several shots needs a schedule with the dataflow executor");
    g->meshes.push_back(meshes[i]);
    g->scheds.push_back(scheds[i]);
    g->nshots.push_back(nshots[i]);
  }
  g->src_w.resize(n);
  g->src.resize(n);
  for (int32_t i = 0; i < n; ++i)
    if (nshots[i] > 1) shot_sources(meshes[i], nshots[i], src_xy ? src_xy[i] : nullptr, g->src_w[i], g->src[i], nullptr);
  SLT_CUDA(cudaDeviceSynchronize());
  group_build(g.get());
  *out = g.release();
  API_END
}

int slt_group_graph_replays(slt_group g, int64_t* replays) {
  API_BEGIN
  REQUIRE(g && replays, "null argument");
  *replays = g->graph_launches;
  API_END
}

int slt_group_destroy(slt_group g) {
  API_BEGIN
  delete g;
  API_END
}

int slt_group_execute(slt_group g, double* const* v, double* const* sigma, const double* const* ricker,
                      const double* dt, int64_t nsteps, void* stream) {
  API_BEGIN
  REQUIRE(g && v && sigma && ricker && dt, "null argument");
  REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  for (size_t i = 0; i < g->meshes.size(); ++i) {
    REQUIRE(v[i] && sigma[i], "null field");
    REQUIRE(std::isfinite(dt[i]), "dt must be finite");
  }
  group_run(g, v, sigma, ricker, dt, nsteps, as_stream(stream));
  API_END
}

int slt_execute_many(int32_t n, const slt_mesh* meshes, const slt_schedule* scheds, double* const* v,
                     double* const* sigma, const double* const* ricker, const double* dt, int64_t nsteps,
                     void* stream) {
  slt_group g = nullptr;
  int rc = slt_group_create(n, meshes, scheds, &g);
  if (rc != SLT_OK) return rc;
  rc = slt_group_execute(g, v, sigma, ricker, dt, nsteps, stream);
  slt_group_destroy(g);
  return rc;
}

int slt_autotune(slt_mesh m, const slt_options* base, int32_t nshots, const int32_t* tile_sizes, int32_t ntile,
                 int32_t shapes, const int32_t* block_threads, int32_t nblock, const int32_t* shots_per_cta,
                 int32_t ngroup, int32_t steps, void* stream, slt_options* best, double* table) {
  API_BEGIN
  REQUIRE(m && base && best && tile_sizes && block_threads, "null argument");
  REQUIRE(nshots >= 1 && nshots <= 4096, "nshots must be in 1..4096");
  REQUIRE(ntile >= 0 && ntile <= 64 && nblock >= 1 && nblock <= 4, "0..64 tile sizes and 1..4 block sizes");
  REQUIRE(steps >= 1 && steps <= 1000, "steps must be in 1..1000");
  for (int i = 0; i < ntile; ++i) REQUIRE(tile_sizes[i] >= 1, "tile sizes must be >= 1");
  for (int b = 0; b < nblock; ++b)
    REQUIRE(block_threads[b] == 128 || block_threads[b] == 256 || block_threads[b] == 384,
            "block_threads must be 128, 256 or 384");
  if (nshots > 1) REQUIRE(base->executor == 0, "the multi-shot executor runs with executor 0");
  REQUIRE(ngroup >= 0 && ngroup <= 16 && (ngroup == 0 || shots_per_cta), "0..16 shots-per-CTA candidates");
  for (int k = 0; k < ngroup; ++k) REQUIRE(shots_per_cta[k] >= 0, "shots per CTA must be >= 0");
  autotune(m, *base, nshots, tile_sizes, ntile, shapes, block_threads, nblock, shots_per_cta, ngroup, steps,
           as_stream(stream), best, table);
  API_END
}

int slt_apply_operator(slt_mesh m, int32_t op, const double* in, double* out, void* stream) {
  API_BEGIN
  REQUIRE(m && in && out, "null argument");
  REQUIRE(op == 0 || op == 1, "op must be 0 (A) or 1 (B)");
  exec_apply(m, op, in, out, as_stream(stream));
  API_END
}

}  // extern "C"
