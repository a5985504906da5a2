// Phase bodies of the DG elastic chain (the parts of each loop, chained per cell into the six
// phases listed in internal.h), shared by the single-field executors (exec.cu, dataflow.cuh) and
// the multi-shot executor (exec_batched.cu).  Included inside an anonymous namespace of each
// translation unit, which therefore holds its own copy of the reference matrices.
//
// One thread computes one (cell, shot) work item.  Per-cell data (geometry, material,
// neighbours) is indexed by the cell's work id; fields are rows of `fs` doubles indexed by the
// item's column: the cell itself for one field (fs = ncp), cell * S + shot for S shots stored
// innermost (fs = ncp * S).  With BATCH = false, S = 1 and the column is the cell.
//
// Operators in nodal strong form (the mass matrix cancels in the volume terms):
//   A sigma = (1/rho) div(sigma) - sum_f (F_f / 2 rho) Lift_f ((sigma - sigma_nb) n_f)
//             - sum_{exterior f} (F_f / rho) Lift_f (sigma n_f)
//   E(v)    = (dvx/dx, dvy/dy, dvx/dy + dvy/dx) - sum_f (F_f / 2) Lift_f sym((v - v_nb) (x) n_f)
//   B v     = C E(v),  C the isotropic Hooke law on (xx, yy, 2xy)
// with F_f = |face f| / |det J| and n_f the outward unit normal of face f.  The reference
// matrices live in constant memory (warp-uniform operands); structural zeros of Dr, Ds are
// skipped through the generated dr_nz / ds_nz tables.
#pragma once

constexpr int MAXNP = 15, MAXNFP = 5;
struct RefC {
  double Dr[MAXNP * MAXNP];
  double Ds[MAXNP * MAXNP];
  double Lift[3 * MAXNP * MAXNFP];
};
__constant__ RefC c_ref[5];  // indexed by degree 1..4

__host__ __device__ constexpr int np_of(int P) { return (P + 1) * (P + 2) / 2; }
__host__ __device__ constexpr int nidx(int P, int i, int j) { return j * (P + 1) - j * (j - 1) / 2 + i; }
// node index of face node k of face f (face f runs from local vertex f to f+1)
template <int P>
__device__ __forceinline__ int fnode(int f, int k) {
  return f == 0 ? nidx(P, k, 0) : (f == 1 ? nidx(P, P - k, k) : nidx(P, 0, P - k));
}

// Field loads: plain (L1-cached) in the untiled and colour-phase kernels; L2-only (ld.global.cg)
// in the persistent dataflow kernel, where other SMs write the fields during the launch.
template <bool CG>
__device__ __forceinline__ double ld(const double* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// buffers of the work layout, each `rows` rows of fs doubles
enum Buf { B_V = 0, B_S = 1, B_U1 = 2, B_U2 = 3, B_E = 4, B_S1 = 5 };

// Per-cell products of geometry and material that every application of the operators would
// otherwise recompute (rows of ncp, work order): the metric terms over rho (volume part of A),
// the face normals scaled by -F / (2 rho) (interior facets of A; twice that on free-surface
// facets) and by -F / 2 (interior facets of E), and lambda + 2 mu (Hooke's law).  Each is the
// same expression the parts evaluated before, so the results do not change.
constexpr int PRE_RXR = 0, PRE_NB = 4, PRE_ND = 10, PRE_L2M = 16, kPreRows = 17;

struct Params {
  int64_t ncp, nc;
  const double* __restrict__ geo;   // [4][ncp]: rx ry sx sy
  const double* __restrict__ fgeo;  // [9][ncp]: nx ny F for faces 0, 1, 2
  const double* __restrict__ mat;   // [3][ncp]: 1/rho, lambda, mu
  const int32_t* __restrict__ nbr;  // [3][ncp]: (w_nb << 3) | (face_nb << 1) | flip, or -1
  const double* __restrict__ pre;   // [kPreRows][ncp]: per-cell products hoisted out of the parts
  double* buf[6];
  const double* ricker;             // [nsteps] or null
  const double* src;                // [Np] source coefficients (one field)
  int32_t src_w;                    // source cell (one field)
  int64_t step;
  const long long* step_dev;        // if set, the step index is read here (graph-captured steps)
  double dt, c24;
  const int32_t* plan_ptr[17];      // tiled: per segment (indexed by its first loop), tile offsets
  const int32_t* plan_items[17];    // and items (see run_seg)
  // multi-shot layout
  int32_t S;                        // shots per cell (1 for one field)
  int32_t s0, sg;                   // tiled multi-shot runs: shots s0 .. s0 + sg - 1 of the S
  int64_t fs;                       // field row stride: ncp * S
  const int32_t* src_wb;            // [S] source cell of every shot
  const double* src_b;              // [S][Np] source coefficients of every shot
  double* e5;                       // if set, phase 5 accumulates its strain here instead of buf[B_E]
  int32_t p;                        // degree (read by the kernels that serve meshes of several degrees)
};

// one (cell, shot) work item: c = cell work id, f = field column, s = shot
struct Pos {
  int64_t c, f;
  int s;
};

template <bool BATCH>
__device__ __forceinline__ int64_t fstride(const Params& a) {
  if constexpr (BATCH) return a.fs;
  else return a.ncp;
}
template <bool BATCH>
__device__ __forceinline__ int64_t ncol(const Params& a, int64_t wn, int s) {  // column of a neighbour
  if constexpr (BATCH) return wn * a.S + s;
  else return wn;
}

// The bodies are built from parts that accumulate in registers: a phase chains the parts of
// consecutive loops of one cell (volume, then interior faces, then free-surface faces) before a
// single store, in the order the loops would apply them one by one.

// The parts work on field views: a field as rows of `fs` doubles, the cell's values in column w
// (a neighbour's in column wn).  The views are global work buffers for the untiled, dataflow and
// multi-shot executors and shared-memory slots for the staged executor, which therefore runs the
// same arithmetic in the same order.  Per-cell data (geometry, material) comes from Params at
// work id c.

// volume part of A: u[comp * Np + i] = (div S)_i, the metric terms (rx .. sy) already over rho;
// x row from (sxx, sxy), y row from (sxy, syy)
template <int P, bool CG>
__device__ __forceinline__ void vol_div_v(const double* S, int64_t fs, int64_t w, double* u, double rx, double ry,
                                          double sx, double sy) {
  constexpr int Np = np_of(P);
  const RefC& R = c_ref[P];
#pragma unroll
  for (int comp = 0; comp < 2; ++comp) {
    double A[Np], B[Np];
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      double s1 = ld<CG>(&S[(int64_t)((comp == 0 ? 0 : 2) * Np + j) * fs + w]);
      double s2 = ld<CG>(&S[(int64_t)((comp == 0 ? 2 : 1) * Np + j) * fs + w]);
      A[j] = fma(ry, s2, rx * s1);
      B[j] = fma(sy, s2, sx * s1);
    }
#pragma unroll
    for (int i = 0; i < Np; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < Np; ++j) {
        if ((dr_nz(P, i) >> j) & 1u) acc = fma(R.Dr[i * MAXNP + j], A[j], acc);
        if ((ds_nz(P, i) >> j) & 1u) acc = fma(R.Ds[i * MAXNP + j], B[j], acc);
      }
      u[comp * Np + i] = acc;
    }
  }
}

template <int P, bool CG>
__device__ __forceinline__ void volB_v(const Params& a, int64_t c, const double* S, int64_t fs, int64_t w,
                                       double* u) {
  const int64_t n = a.ncp;
  vol_div_v<P, CG>(S, fs, w, u, a.pre[PRE_RXR * n + c], a.pre[(PRE_RXR + 1) * n + c], a.pre[(PRE_RXR + 2) * n + c],
                   a.pre[(PRE_RXR + 3) * n + c]);
}

// interior face f of A: u += -(F/2 rho) Lift_f ((S - S_nb) n); the neighbour's face fn, flip
template <int P, bool CG>
__device__ __forceinline__ void intB_face(const Params& a, int64_t c, int f, const double* S, int64_t fs, int64_t w,
                                          int64_t wn, int fn, int flip, double* u) {
  constexpr int Np = np_of(P), Nfp = P + 1;
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  const double nx = a.pre[(PRE_NB + 2 * f) * n + c], ny = a.pre[(PRE_NB + 2 * f + 1) * n + c];
  double gx[Nfp], gy[Nfp];
#pragma unroll
  for (int k = 0; k < Nfp; ++k) {
    const int i0 = fnode<P>(f, k);
    const int i1 = fnode<P>(fn, flip ? P - k : k);
    double dxx = ld<CG>(&S[(int64_t)i0 * fs + w]) - ld<CG>(&S[(int64_t)i1 * fs + wn]);
    double dyy = ld<CG>(&S[(int64_t)(Np + i0) * fs + w]) - ld<CG>(&S[(int64_t)(Np + i1) * fs + wn]);
    double dxy = ld<CG>(&S[(int64_t)(2 * Np + i0) * fs + w]) - ld<CG>(&S[(int64_t)(2 * Np + i1) * fs + wn]);
    gx[k] = fma(dxy, ny, dxx * nx);
    gy[k] = fma(dyy, ny, dxy * nx);
  }
#pragma unroll
  for (int i = 0; i < Np; ++i)
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      u[i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gx[k], u[i]);
      u[Np + i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gy[k], u[Np + i]);
    }
}

// free-surface face f of A: u += -(F/rho) Lift_f (S n)
template <int P, bool CG>
__device__ __forceinline__ void extB_face(const Params& a, int64_t c, int f, const double* S, int64_t fs, int64_t w,
                                          double* u) {
  constexpr int Np = np_of(P), Nfp = P + 1;
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  // (-F / rho) n = 2 (-F / 2 rho) n exactly: scaling by 2 commutes with rounding
  const double nx = 2.0 * a.pre[(PRE_NB + 2 * f) * n + c], ny = 2.0 * a.pre[(PRE_NB + 2 * f + 1) * n + c];
  double gx[Nfp], gy[Nfp];
#pragma unroll
  for (int k = 0; k < Nfp; ++k) {
    const int i0 = fnode<P>(f, k);
    double sxx = ld<CG>(&S[(int64_t)i0 * fs + w]), syy = ld<CG>(&S[(int64_t)(Np + i0) * fs + w]),
           sxy = ld<CG>(&S[(int64_t)(2 * Np + i0) * fs + w]);
    gx[k] = fma(sxy, ny, sxx * nx);
    gy[k] = fma(syy, ny, sxy * nx);
  }
#pragma unroll
  for (int i = 0; i < Np; ++i)
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      u[i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gx[k], u[i]);
      u[Np + i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gy[k], u[Np + i]);
    }
}

// volume part of E: e = (dvx/dx, dvy/dy, dvx/dy + dvy/dx) at the nodes, e[comp * Np + i]
template <int P, bool CG>
__device__ __forceinline__ void volD_v(const Params& a, int64_t c, const double* V, int64_t fs, int64_t w,
                                       double* e) {
  constexpr int Np = np_of(P);
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  double rx = a.geo[c], ry = a.geo[n + c], sx = a.geo[2 * n + c], sy = a.geo[3 * n + c];
  double vx[Np], vy[Np];
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    vx[j] = ld<CG>(&V[(int64_t)j * fs + w]);
    vy[j] = ld<CG>(&V[(int64_t)(Np + j) * fs + w]);
  }
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    double drx = 0.0, dsx = 0.0, dry = 0.0, dsy = 0.0;
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      if ((dr_nz(P, i) >> j) & 1u) {
        drx = fma(R.Dr[i * MAXNP + j], vx[j], drx);
        dry = fma(R.Dr[i * MAXNP + j], vy[j], dry);
      }
      if ((ds_nz(P, i) >> j) & 1u) {
        dsx = fma(R.Ds[i * MAXNP + j], vx[j], dsx);
        dsy = fma(R.Ds[i * MAXNP + j], vy[j], dsy);
      }
    }
    e[i] = fma(sx, dsx, rx * drx);
    e[Np + i] = fma(sy, dsy, ry * dry);
    e[2 * Np + i] = fma(sx, dsy, fma(rx, dry, fma(sy, dsx, ry * drx)));
  }
}

// interior face f of E: e += -(F/2) Lift_f sym((V - V_nb) (x) n)
template <int P, bool CG>
__device__ __forceinline__ void intD_face(const Params& a, int64_t c, int f, const double* V, int64_t fs, int64_t w,
                                          int64_t wn, int fn, int flip, double* e) {
  constexpr int Np = np_of(P), Nfp = P + 1;
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  const double cx = a.pre[(PRE_ND + 2 * f) * n + c], cy = a.pre[(PRE_ND + 2 * f + 1) * n + c];
  double dx[Nfp], dy[Nfp];
#pragma unroll
  for (int k = 0; k < Nfp; ++k) {
    const int i0 = fnode<P>(f, k);
    const int i1 = fnode<P>(fn, flip ? P - k : k);
    dx[k] = ld<CG>(&V[(int64_t)i0 * fs + w]) - ld<CG>(&V[(int64_t)i1 * fs + wn]);
    dy[k] = ld<CG>(&V[(int64_t)(Np + i0) * fs + w]) - ld<CG>(&V[(int64_t)(Np + i1) * fs + wn]);
  }
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    double lx = R.Lift[(f * MAXNP + i) * MAXNFP] * dx[0], ly = R.Lift[(f * MAXNP + i) * MAXNFP] * dy[0];
#pragma unroll
    for (int k = 1; k < Nfp; ++k) {
      lx = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], dx[k], lx);
      ly = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], dy[k], ly);
    }
    e[i] = fma(cx, lx, e[i]);
    e[Np + i] = fma(cy, ly, e[Np + i]);
    e[2 * Np + i] = fma(cy, lx, fma(cx, ly, e[2 * Np + i]));
  }
}

// The same parts on the global work layout at work item q: every face of the mask in turn
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void volB_part(const Params& a, const Pos& q, const double* S, double* u) {
  volB_v<P, CG>(a, q.c, S, fstride<BATCH>(a), q.f, u);
}
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void intB_part(const Params& a, const Pos& q, int mask, const double* S, double* u) {
  const int64_t n = a.ncp, c = q.c;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!((mask >> f) & 1)) continue;
    const int32_t nb = a.nbr[f * n + c];
    intB_face<P, CG>(a, c, f, S, fstride<BATCH>(a), q.f, ncol<BATCH>(a, nb >> 3, q.s), (nb >> 1) & 3, nb & 1, u);
  }
}
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void extB_part(const Params& a, const Pos& q, int mask, const double* S, double* u) {
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!((mask >> f) & 1)) continue;
    extB_face<P, CG>(a, q.c, f, S, fstride<BATCH>(a), q.f, u);
  }
}
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void volD_part(const Params& a, const Pos& q, const double* V, double* e) {
  volD_v<P, CG>(a, q.c, V, fstride<BATCH>(a), q.f, e);
}
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void intD_part(const Params& a, const Pos& q, int mask, const double* V, double* e) {
  const int64_t n = a.ncp, c = q.c;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!((mask >> f) & 1)) continue;
    const int32_t nb = a.nbr[f * n + c];
    intD_face<P, CG>(a, c, f, V, fstride<BATCH>(a), q.f, ncol<BATCH>(a, nb >> 3, q.s), (nb >> 1) & 3, nb & 1, e);
  }
}

template <int R, bool CG, bool BATCH>
__device__ __forceinline__ void load_rows(const Params& a, const Pos& q, const double* X, double* x) {
  const int64_t fs = fstride<BATCH>(a), w = q.f;
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = ld<CG>(&X[(int64_t)r * fs + w]);
}
template <int R, bool BATCH>
__device__ __forceinline__ void store_rows(const Params& a, const Pos& q, double* X, const double* x) {
  const int64_t fs = fstride<BATCH>(a), w = q.f;
#pragma unroll
  for (int r = 0; r < R; ++r) X[(int64_t)r * fs + w] = x[r];
}

// ---- bodies of the phases.  A phase is a run of consecutive loops of the chain that write only
// the cell's own outputs and read nothing another thread writes during the run (no neighbour
// value produced inside the run), so one thread can take a cell through all of them.  A work
// item covers a cell's share of each loop of the run: pa = the run's first loop, a cell loop
// (volume part); imask / emask = the interior / free-surface faces of its facet loops; pb = a
// later cell loop of the run (Hooke's law or an update).  Missing parts were done in another
// tile: the item starts from the stored output.

// A(S) -> U: volume part when pa, else U as stored; then the faces of imask, emask
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void segA(const Params& a, const Pos& q, bool pa, int imask, int emask,
                                     const double* S, double* U) {
  double u[2 * np_of(P)];
  if (pa) volB_part<P, CG, BATCH>(a, q, S, u);
  else load_rows<2 * np_of(P), CG, BATCH>(a, q, U, u);
  intB_part<P, CG, BATCH>(a, q, imask, S, u);
  extB_part<P, CG, BATCH>(a, q, emask, S, u);
  store_rows<2 * np_of(P), BATCH>(a, q, U, u);
}

// E(V) -> E (volume part when pa, else E as stored; the faces of imask), then, when pb, Hooke's
// law S1 = C E and the volume part of A(S1) -> U
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void segEB(const Params& a, const Pos& q, bool pa, bool pb, int imask, const double* V,
                                      double* E, double* S1, double* U) {
  constexpr int Np = np_of(P);
  double e[3 * Np];
  if (pa) volD_part<P, CG, BATCH>(a, q, V, e);
  else load_rows<3 * Np, CG, BATCH>(a, q, E, e);
  intD_part<P, CG, BATCH>(a, q, imask, V, e);
  if (pa || imask) store_rows<3 * Np, BATCH>(a, q, E, e);
  if (!pb) return;
  const int64_t n = a.ncp, c = q.c, fs = fstride<BATCH>(a), w = q.f;
  const double lam = a.mat[n + c], mu = a.mat[2 * n + c];
  const double l2m = a.pre[PRE_L2M * n + c];
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    S1[(int64_t)j * fs + w] = fma(lam, e[Np + j], l2m * e[j]);
    S1[(int64_t)(Np + j) * fs + w] = fma(lam, e[j], l2m * e[Np + j]);
    S1[(int64_t)(2 * Np + j) * fs + w] = mu * e[2 * Np + j];
  }
  double u[2 * Np];
  volB_part<P, CG, BATCH>(a, q, S1, u);
  store_rows<2 * Np, BATCH>(a, q, U, u);
}

// faces of A(S1) onto U2 (imask, emask), then, when pb, the velocity update
// V += dt (U1 + dt^2/24 U2)
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void segAV(const Params& a, const Pos& q, bool pb, int imask, int emask) {
  constexpr int Np = np_of(P);
  double* const* b = a.buf;
  double u[2 * Np];
  load_rows<2 * Np, CG, BATCH>(a, q, b[B_U2], u);
  if (imask | emask) {
    intB_part<P, CG, BATCH>(a, q, imask, b[B_S1], u);
    extB_part<P, CG, BATCH>(a, q, emask, b[B_S1], u);
    store_rows<2 * Np, BATCH>(a, q, b[B_U2], u);
  }
  if (!pb) return;
  const int64_t fs = fstride<BATCH>(a), w = q.f;
  double* V = b[B_V];
  const double* U1 = b[B_U1];
#pragma unroll
  for (int r = 0; r < 2 * Np; ++r) {
    int64_t o = (int64_t)r * fs + w;
    V[o] = fma(a.dt, fma(a.c24, u[r], ld<CG>(&U1[o])), ld<CG>(&V[o]));
  }
}

// E(U1) -> E as segEB, then, when pb, the stress update S += dt (S1 + dt^2/24 C E) + source
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void segES(const Params& a, const Pos& q, bool pa, bool pb, int imask, int64_t step) {
  constexpr int Np = np_of(P);
  double* const* b = a.buf;
  double* const E = a.e5 ? a.e5 : b[B_E];
  double e[3 * Np];
  if (pa) volD_part<P, CG, BATCH>(a, q, b[B_U1], e);
  else load_rows<3 * Np, CG, BATCH>(a, q, E, e);
  intD_part<P, CG, BATCH>(a, q, imask, b[B_U1], e);
  if (pa || imask) store_rows<3 * Np, BATCH>(a, q, E, e);
  if (!pb) return;
  const int64_t n = a.ncp, c = q.c, fs = fstride<BATCH>(a), w = q.f;
  double* S = b[B_S];
  const double* S1 = b[B_S1];
  const double lam = a.mat[n + c], mu = a.mat[2 * n + c];
  const double l2m = a.pre[PRE_L2M * n + c];
  int32_t sw;
  const double* sv;
  if constexpr (BATCH) {
    sw = a.src_wb ? a.src_wb[q.s] : -1;
    sv = a.src_b + (int64_t)q.s * Np;
  } else {
    sw = a.src_w;
    sv = a.src;
  }
  const bool src = (c == sw) && a.ricker != nullptr;
  const double gs = src ? a.dt * a.ricker[step] : 0.0;
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    const double exx = e[j], eyy = e[Np + j], g = e[2 * Np + j];
    double cxx = fma(lam, eyy, l2m * exx), cyy = fma(lam, exx, l2m * eyy), cxy = mu * g;
    int64_t oxx = (int64_t)j * fs + w, oyy = (int64_t)(Np + j) * fs + w, oxy = (int64_t)(2 * Np + j) * fs + w;
    double nxx = fma(a.dt, fma(a.c24, cxx, ld<CG>(&S1[oxx])), ld<CG>(&S[oxx]));
    double nyy = fma(a.dt, fma(a.c24, cyy, ld<CG>(&S1[oyy])), ld<CG>(&S[oyy]));
    S[oxy] = fma(a.dt, fma(a.c24, cxy, ld<CG>(&S1[oxy])), ld<CG>(&S[oxy]));
    if (src) {
      nxx += gs * sv[j];
      nyy += gs * sv[j];
    }
    S[oxx] = nxx;
    S[oyy] = nyy;
  }
}

// phase H at one (cell, shot); the phases and their loops are listed with phase_first
template <int P, int H, bool CG, bool BATCH>
__device__ __forceinline__ void phase_body(const Params& a, const Pos& q, bool pa, bool pb, int imask, int emask,
                                           int64_t step) {
  double* const* b = a.buf;
  if constexpr (H == 0) segA<P, CG, BATCH>(a, q, pa, imask, emask, b[B_S], b[B_U1]);
  else if constexpr (H == 1) segEB<P, CG, BATCH>(a, q, pa, pb, imask, b[B_U1], b[B_E], b[B_S1], b[B_U2]);
  else if constexpr (H == 2) segAV<P, CG, BATCH>(a, q, pb, imask, emask);
  else if constexpr (H == 3) segEB<P, CG, BATCH>(a, q, pa, pb, imask, b[B_V], b[B_E], b[B_S1], b[B_U1]);
  else if constexpr (H == 4) segA<P, CG, BATCH>(a, q, false, imask, emask, b[B_S1], b[B_U1]);
  else segES<P, CG, BATCH>(a, q, pa, pb, imask, step);
}

// the faces of `mask` that have a neighbour (interior) and those that do not (free surface)
__device__ __forceinline__ void split_mask(const Params& a, int64_t c, int mask, int& imask, int& emask) {
  imask = 0;
#pragma unroll
  for (int f = 0; f < 3; ++f)
    if (((mask >> f) & 1) && a.nbr[f * a.ncp + c] >= 0) imask |= 1 << f;
  emask = mask & ~imask;
}

// parts of a phase (untiled launches): the first cell loop, the facet loops, the later cell loop
constexpr int kPartA = 1, kPartF = 2, kPartB = 4, kAllParts = 7;

// Untiled: the PARTS of phase H at cell w, shot s (every face of the cell)
template <int P, int H, int PARTS, bool BATCH>
__device__ __forceinline__ void run_phase(const Params& a, int64_t w, int s, int64_t step) {
  Pos q;
  q.c = w;
  q.s = s;
  q.f = BATCH ? w * a.S + s : w;
  int imask = 0, emask = 0;
  if (PARTS & kPartF) split_mask(a, w, 7, imask, emask);
  phase_body<P, H, false, BATCH>(a, q, (PARTS & kPartA) != 0, (PARTS & kPartB) != 0, imask, emask, step);
}

// Tiled: one item of a segment of phase H,
// item = (work id << 5) | (later cell loop << 4) | (first cell loop << 3) | face mask
template <int P, bool CG, bool BATCH>
__device__ __forceinline__ void run_seg(const Params& a, int H, int32_t item, int64_t step, int s = 0) {
  Pos q;
  q.c = (int64_t)(item >> 5);
  q.s = s;
  q.f = BATCH ? q.c * a.S + s : q.c;
  const bool pa = (item >> 3) & 1, pb = (item >> 4) & 1;
  int imask, emask;
  split_mask(a, q.c, item & 7, imask, emask);
  switch (H) {
    case 0: phase_body<P, 0, CG, BATCH>(a, q, pa, pb, imask, emask, step); break;
    case 1: phase_body<P, 1, CG, BATCH>(a, q, pa, pb, imask, emask, step); break;
    case 2: phase_body<P, 2, CG, BATCH>(a, q, pa, pb, imask, emask, step); break;
    case 3: phase_body<P, 3, CG, BATCH>(a, q, pa, pb, imask, emask, step); break;
    case 4: phase_body<P, 4, CG, BATCH>(a, q, pa, pb, imask, emask, step); break;
    default: phase_body<P, 5, CG, BATCH>(a, q, pa, pb, imask, emask, step); break;
  }
}

// reference matrices of one degree into this translation unit's constant memory
inline void upload_ref(const slt::RefElem& r) {
  RefC h{};
  for (int i = 0; i < r.Np; ++i)
    for (int j = 0; j < r.Np; ++j) {
      h.Dr[i * MAXNP + j] = r.Dr[i * r.Np + j];
      h.Ds[i * MAXNP + j] = r.Ds[i * r.Np + j];
    }
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < r.Np; ++i)
      for (int k = 0; k < r.Nfp; ++k) h.Lift[(f * MAXNP + i) * MAXNFP + k] = r.Lift[(f * r.Np + i) * r.Nfp + k];
  SLT_CUDA(cudaMemcpyToSymbol(c_ref, &h, sizeof(RefC), r.p * sizeof(RefC)));
}
