// Executor of the DG elastic loop chain (Section 5.2, Algorithm 4, shared-memory mode).
//
// One thread per cell for every loop.  Facet loops are executed as pulls: the thread of cell c
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
// with c = dt^2/24: the fourth-order staggered Taylor leapfrog.
//
// Operators in nodal strong form (the mass matrix cancels in the volume terms):
//   A sigma = (1/rho) div(sigma) - sum_f (F_f / 2 rho) Lift_f ((sigma - sigma_nb) n_f)
//             - sum_{exterior f} (F_f / rho) Lift_f (sigma n_f)
//   E(v)    = (dvx/dx, dvy/dy, dvx/dy + dvy/dx) - sum_f (F_f / 2) Lift_f sym((v - v_nb) (x) n_f)
//   B v     = C E(v),  C the isotropic Hooke law on (xx, yy, 2xy)
// with F_f = |face f| / |det J| and n_f the outward unit normal of face f.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "refmask.h"  // generated: dr_nz(p, i), ds_nz(p, i) nonzero bits of row i

namespace slt {

namespace {

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

// Field loads: plain (L1-cached) in the per-loop and colour-phase kernels; L2-only (ld.global.cg)
// in the persistent dataflow kernel, where other SMs write the fields during the launch and L1
// is not coherent across SMs.
template <bool CG>
__device__ __forceinline__ double ld(const double* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// buffers of the work layout, each [rows][ncp]
enum Buf { B_V = 0, B_S = 1, B_U1 = 2, B_U2 = 3, B_E = 4, B_S1 = 5 };

struct Params {
  int64_t ncp, nc;
  const double* __restrict__ geo;   // [4][ncp]: rx ry sx sy
  const double* __restrict__ fgeo;  // [9][ncp]: nx ny F for faces 0, 1, 2
  const double* __restrict__ mat;   // [3][ncp]: 1/rho, lambda, mu
  const int32_t* __restrict__ nbr;  // [3][ncp]: (w_nb << 3) | (face_nb << 1) | flip, or -1
  double* buf[6];
  const double* ricker;             // [nsteps] or null
  const double* src;                // [Np] source coefficients
  int32_t src_w;
  int64_t step;
  double dt, c24;
  const int32_t* plan_ptr[17];
  const int32_t* plan_items[17];
};

template <int P, bool CG>
__device__ __forceinline__ void vol_div(const Params& a, int64_t w, const double* S, double* U, double rx, double ry,
                                        double sx, double sy) {
  // U = div(S) scaled (rx.. already divided by rho): x row uses (sxx, sxy), y row (sxy, syy)
  constexpr int Np = np_of(P);
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
#pragma unroll
  for (int comp = 0; comp < 2; ++comp) {
    double A[Np], B[Np];
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      double s1 = ld<CG>(&S[(int64_t)((comp == 0 ? 0 : 2) * Np + j) * n + w]);
      double s2 = ld<CG>(&S[(int64_t)((comp == 0 ? 2 : 1) * Np + j) * n + w]);
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
      U[(int64_t)(comp * Np + i) * n + w] = acc;
    }
  }
}

template <int P, bool CG>
__device__ __forceinline__ void volB(const Params& a, int64_t w, const double* S, double* U) {
  const int64_t n = a.ncp;
  double ir = a.mat[w];
  vol_div<P, CG>(a, w, S, U, a.geo[w] * ir, a.geo[n + w] * ir, a.geo[2 * n + w] * ir, a.geo[3 * n + w] * ir);
}

template <int P, bool CG>
__device__ __forceinline__ void volD(const Params& a, int64_t w, const double* V, double* E) {
  constexpr int Np = np_of(P);
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  double rx = a.geo[w], ry = a.geo[n + w], sx = a.geo[2 * n + w], sy = a.geo[3 * n + w];
  double vx[Np], vy[Np];
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    vx[j] = ld<CG>(&V[(int64_t)j * n + w]);
    vy[j] = ld<CG>(&V[(int64_t)(Np + j) * n + w]);
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
    E[(int64_t)i * n + w] = fma(sx, dsx, rx * drx);
    E[(int64_t)(Np + i) * n + w] = fma(sy, dsy, ry * dry);
    E[(int64_t)(2 * Np + i) * n + w] = fma(sx, dsy, fma(rx, dry, fma(sy, dsx, ry * drx)));
  }
}

// S1 = C E at the nodes, then U = div(S1)/rho
template <int P, bool CG>
__device__ __forceinline__ void hookeB(const Params& a, int64_t w, const double* E, double* S1, double* U) {
  constexpr int Np = np_of(P);
  const int64_t n = a.ncp;
  double lam = a.mat[n + w], mu = a.mat[2 * n + w];
  double l2m = fma(2.0, mu, lam);
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    double exx = ld<CG>(&E[(int64_t)j * n + w]), eyy = ld<CG>(&E[(int64_t)(Np + j) * n + w]),
           g = ld<CG>(&E[(int64_t)(2 * Np + j) * n + w]);
    S1[(int64_t)j * n + w] = fma(lam, eyy, l2m * exx);
    S1[(int64_t)(Np + j) * n + w] = fma(lam, exx, l2m * eyy);
    S1[(int64_t)(2 * Np + j) * n + w] = mu * g;
  }
  volB<P, CG>(a, w, S1, U);
}

template <int P, bool CG>
__device__ __forceinline__ void intB(const Params& a, int64_t w, int mask, const double* S, double* U) {
  constexpr int Np = np_of(P), Nfp = P + 1;
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  const double ir = a.mat[w];
  double ax[Np], ay[Np];
#pragma unroll
  for (int i = 0; i < Np; ++i) ax[i] = ay[i] = 0.0;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!((mask >> f) & 1)) continue;
    const int32_t nb = a.nbr[f * n + w];
    const int64_t wn = nb >> 3;
    const int fn = (nb >> 1) & 3, flip = nb & 1;
    const double sc = -0.5 * a.fgeo[(3 * f + 2) * n + w] * ir;
    const double nx = sc * a.fgeo[(3 * f) * n + w], ny = sc * a.fgeo[(3 * f + 1) * n + w];
    double gx[Nfp], gy[Nfp];
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      const int i0 = fnode<P>(f, k);
      const int i1 = fnode<P>(fn, flip ? P - k : k);
      double dxx = ld<CG>(&S[(int64_t)i0 * n + w]) - ld<CG>(&S[(int64_t)i1 * n + wn]);
      double dyy = ld<CG>(&S[(int64_t)(Np + i0) * n + w]) - ld<CG>(&S[(int64_t)(Np + i1) * n + wn]);
      double dxy = ld<CG>(&S[(int64_t)(2 * Np + i0) * n + w]) - ld<CG>(&S[(int64_t)(2 * Np + i1) * n + wn]);
      gx[k] = fma(dxy, ny, dxx * nx);
      gy[k] = fma(dyy, ny, dxy * nx);
    }
#pragma unroll
    for (int i = 0; i < Np; ++i)
#pragma unroll
      for (int k = 0; k < Nfp; ++k) {
        ax[i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gx[k], ax[i]);
        ay[i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gy[k], ay[i]);
      }
  }
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    U[(int64_t)i * n + w] = ld<CG>(&U[(int64_t)i * n + w]) + ax[i];
    U[(int64_t)(Np + i) * n + w] = ld<CG>(&U[(int64_t)(Np + i) * n + w]) + ay[i];
  }
}

template <int P, bool CG>
__device__ __forceinline__ void extB(const Params& a, int64_t w, int mask, const double* S, double* U) {
  constexpr int Np = np_of(P), Nfp = P + 1;
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  const double ir = a.mat[w];
  double ax[Np], ay[Np];
#pragma unroll
  for (int i = 0; i < Np; ++i) ax[i] = ay[i] = 0.0;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!((mask >> f) & 1)) continue;
    const double sc = -a.fgeo[(3 * f + 2) * n + w] * ir;
    const double nx = sc * a.fgeo[(3 * f) * n + w], ny = sc * a.fgeo[(3 * f + 1) * n + w];
    double gx[Nfp], gy[Nfp];
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      const int i0 = fnode<P>(f, k);
      double sxx = ld<CG>(&S[(int64_t)i0 * n + w]), syy = ld<CG>(&S[(int64_t)(Np + i0) * n + w]),
             sxy = ld<CG>(&S[(int64_t)(2 * Np + i0) * n + w]);
      gx[k] = fma(sxy, ny, sxx * nx);
      gy[k] = fma(syy, ny, sxy * nx);
    }
#pragma unroll
    for (int i = 0; i < Np; ++i)
#pragma unroll
      for (int k = 0; k < Nfp; ++k) {
        ax[i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gx[k], ax[i]);
        ay[i] = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], gy[k], ay[i]);
      }
  }
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    U[(int64_t)i * n + w] = ld<CG>(&U[(int64_t)i * n + w]) + ax[i];
    U[(int64_t)(Np + i) * n + w] = ld<CG>(&U[(int64_t)(Np + i) * n + w]) + ay[i];
  }
}

template <int P, bool CG>
__device__ __forceinline__ void intD(const Params& a, int64_t w, int mask, const double* V, double* E) {
  constexpr int Np = np_of(P), Nfp = P + 1;
  const RefC& R = c_ref[P];
  const int64_t n = a.ncp;
  double exx[Np], eyy[Np], eg[Np];
#pragma unroll
  for (int i = 0; i < Np; ++i) exx[i] = eyy[i] = eg[i] = 0.0;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!((mask >> f) & 1)) continue;
    const int32_t nb = a.nbr[f * n + w];
    const int64_t wn = nb >> 3;
    const int fn = (nb >> 1) & 3, flip = nb & 1;
    const double h = -0.5 * a.fgeo[(3 * f + 2) * n + w];
    const double cx = h * a.fgeo[(3 * f) * n + w], cy = h * a.fgeo[(3 * f + 1) * n + w];
    double dx[Nfp], dy[Nfp];
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      const int i0 = fnode<P>(f, k);
      const int i1 = fnode<P>(fn, flip ? P - k : k);
      dx[k] = ld<CG>(&V[(int64_t)i0 * n + w]) - ld<CG>(&V[(int64_t)i1 * n + wn]);
      dy[k] = ld<CG>(&V[(int64_t)(Np + i0) * n + w]) - ld<CG>(&V[(int64_t)(Np + i1) * n + wn]);
    }
#pragma unroll
    for (int i = 0; i < Np; ++i) {
      double lx = R.Lift[(f * MAXNP + i) * MAXNFP] * dx[0], ly = R.Lift[(f * MAXNP + i) * MAXNFP] * dy[0];
#pragma unroll
      for (int k = 1; k < Nfp; ++k) {
        lx = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], dx[k], lx);
        ly = fma(R.Lift[(f * MAXNP + i) * MAXNFP + k], dy[k], ly);
      }
      exx[i] = fma(cx, lx, exx[i]);
      eyy[i] = fma(cy, ly, eyy[i]);
      eg[i] = fma(cy, lx, fma(cx, ly, eg[i]));
    }
  }
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    E[(int64_t)i * n + w] = ld<CG>(&E[(int64_t)i * n + w]) + exx[i];
    E[(int64_t)(Np + i) * n + w] = ld<CG>(&E[(int64_t)(Np + i) * n + w]) + eyy[i];
    E[(int64_t)(2 * Np + i) * n + w] = ld<CG>(&E[(int64_t)(2 * Np + i) * n + w]) + eg[i];
  }
}

template <int P, bool CG>
__device__ __forceinline__ void updV(const Params& a, int64_t w) {
  constexpr int Np = np_of(P);
  const int64_t n = a.ncp;
  double* V = a.buf[B_V];
  const double* U1 = a.buf[B_U1];
  const double* U2 = a.buf[B_U2];
#pragma unroll
  for (int q = 0; q < 2 * Np; ++q) {
    int64_t o = (int64_t)q * n + w;
    V[o] = fma(a.dt, fma(a.c24, ld<CG>(&U2[o]), ld<CG>(&U1[o])), ld<CG>(&V[o]));
  }
}

template <int P, bool CG>
__device__ __forceinline__ void updS(const Params& a, int64_t w, int64_t step) {
  constexpr int Np = np_of(P);
  const int64_t n = a.ncp;
  double* S = a.buf[B_S];
  const double* S1 = a.buf[B_S1];
  const double* E = a.buf[B_E];
  double lam = a.mat[n + w], mu = a.mat[2 * n + w];
  double l2m = fma(2.0, mu, lam);
  const bool src = (w == a.src_w) && a.ricker != nullptr;
  const double gs = src ? a.dt * a.ricker[step] : 0.0;
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    double exx = ld<CG>(&E[(int64_t)j * n + w]), eyy = ld<CG>(&E[(int64_t)(Np + j) * n + w]),
           g = ld<CG>(&E[(int64_t)(2 * Np + j) * n + w]);
    double cxx = fma(lam, eyy, l2m * exx), cyy = fma(lam, exx, l2m * eyy), cxy = mu * g;
    int64_t oxx = (int64_t)j * n + w, oyy = (int64_t)(Np + j) * n + w, oxy = (int64_t)(2 * Np + j) * n + w;
    double nxx = fma(a.dt, fma(a.c24, cxx, ld<CG>(&S1[oxx])), ld<CG>(&S[oxx]));
    double nyy = fma(a.dt, fma(a.c24, cyy, ld<CG>(&S1[oyy])), ld<CG>(&S[oyy]));
    S[oxy] = fma(a.dt, fma(a.c24, cxy, ld<CG>(&S1[oxy])), ld<CG>(&S[oxy]));
    if (src) {
      nxx += gs * a.src[j];
      nyy += gs * a.src[j];
    }
    S[oxx] = nxx;
    S[oyy] = nyy;
  }
}

// one iteration of loop J; item = work id (cell loops) or (work id << 3) | face mask (facet loops)
template <int P, bool CG>
__device__ __forceinline__ void run_loop(const Params& a, int J, int32_t item, int64_t step) {
  double* const* b = a.buf;
  const int64_t w = (J == 1 || J == 2 || J == 4 || J == 6 || J == 7 || J == 10 || J == 12 || J == 13 || J == 15)
                        ? (int64_t)(item >> 3) : (int64_t)item;
  const int mask = item & 7;
  switch (J) {
    case 0: volB<P, CG>(a, w, b[B_S], b[B_U1]); break;
    case 1: intB<P, CG>(a, w, mask, b[B_S], b[B_U1]); break;
    case 2: extB<P, CG>(a, w, mask, b[B_S], b[B_U1]); break;
    case 3: volD<P, CG>(a, w, b[B_U1], b[B_E]); break;
    case 4: intD<P, CG>(a, w, mask, b[B_U1], b[B_E]); break;
    case 5: hookeB<P, CG>(a, w, b[B_E], b[B_S1], b[B_U2]); break;
    case 6: intB<P, CG>(a, w, mask, b[B_S1], b[B_U2]); break;
    case 7: extB<P, CG>(a, w, mask, b[B_S1], b[B_U2]); break;
    case 8: updV<P, CG>(a, w); break;
    case 9: volD<P, CG>(a, w, b[B_V], b[B_E]); break;
    case 10: intD<P, CG>(a, w, mask, b[B_V], b[B_E]); break;
    case 11: hookeB<P, CG>(a, w, b[B_E], b[B_S1], b[B_U1]); break;
    case 12: intB<P, CG>(a, w, mask, b[B_S1], b[B_U1]); break;
    case 13: extB<P, CG>(a, w, mask, b[B_S1], b[B_U1]); break;
    case 14: volD<P, CG>(a, w, b[B_U1], b[B_E]); break;
    case 15: intD<P, CG>(a, w, mask, b[B_U1], b[B_E]); break;
    case 16: updS<P, CG>(a, w, step); break;
    default: break;
  }
}

__host__ __device__ constexpr bool is_int_loop(int J) { return J == 1 || J == 4 || J == 6 || J == 10 || J == 12 || J == 15; }
__host__ __device__ constexpr bool is_ext_loop(int J) { return J == 2 || J == 7 || J == 13; }

// Untiled chain: loop J over every cell of the mesh (facet loops pull all interior or all
// exterior faces of the cell).
template <int P, int J>
__global__ void __launch_bounds__(128) k_loop(Params a) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= a.nc) return;
  int32_t item = (int32_t)w;
  if (is_int_loop(J) || is_ext_loop(J)) {
    int mask = 0;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      bool interior = a.nbr[f * a.ncp + w] >= 0;
      if (is_int_loop(J) ? interior : !interior) mask |= 1 << f;
    }
    if (!mask) return;
    item = (int32_t)((w << 3) | mask);
  }
  run_loop<P, false>(a, J, item, a.step);
}

// No register cap: forcing 24 warps per SM (80 registers at p = 2) made the tiled kernels slower
// (their loads are latency bound and more resident tiles overflow L2); one CTA is the minimum.
template <int P, int BS>
constexpr int tile_min_blocks() {
  return P <= 2 ? 768 / BS : 1;
}

// Tiled chain: one CTA per tile of one colour; the tile runs its slice of every loop of the
// sub-chain [first, last) in order, loops separated by a CTA barrier.
template <int P, int BS>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_tiled(Params a, int first, int last,
                                                                       const int32_t* __restrict__ tiles) {
  const int t = tiles[blockIdx.x];
  for (int J = first; J < last; ++J) {
    const int32_t b = a.plan_ptr[J][t], e = a.plan_ptr[J][t + 1];
    const int32_t* items = a.plan_items[J];
    for (int32_t i = b + threadIdx.x; i < e; i += BS) run_loop<P, false>(a, J, items[i], a.step);
    __syncthreads();
  }
}

// Field loads of the dataflow kernel go to L2 only (ld.global.cg).  Cacheable loads after the
// acquire fence and CTA barrier below are also correct by the PTX memory model; they measured
// no faster, so the conservative form is kept.
constexpr bool DF_L2_ONLY = true;

// Persistent dataflow executor with a ready queue.  A node is (step, tile); it depends on the
// tiles it overlaps (lower colours of its sub-chain, the previous sub-chain's tiles on its
// cells, wrapping to the previous step), a linear extension of the inspector's colour order.
// Each node keeps a count of unfinished dependencies; finishing a tile decrements the counts of
// its successors and publishes those that reach zero to the next queue slot.  CTAs take slots
// in order and run whatever node was published there, so no CTA waits on one particular
// dependency while other work is ready.  Every claimed slot is eventually filled (the graph is
// acyclic and every published node is run), so the bounded waits only end early on an error.
struct DF {
  long long total;                // nodes = nsteps * G
  long long nsteps;
  int32_t G;                      // tiles over all sub-chains
  int32_t cum[17];                // global tile id base of each sub-chain (cum[k] + local id)
  int32_t first[16], last[16];    // loop range of each sub-chain
  const int32_t* succ_ptr;        // [G + 1]
  const int32_t* succ;            // (global tile << 1) | 1 when the successor is the next step's node
  int32_t* pending;               // [nsteps * G] unfinished dependencies of each node
  int32_t* queue;                 // [nsteps * G] node ids in publication order, -1 = not yet
  unsigned long long* head;       // next slot to take
  unsigned long long* tail;       // next slot to publish
  int32_t* err;                   // set when a wait gave up
  long long max_spins;
};

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int atom_add_acq_rel(int32_t* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__global__ void k_df_init(DF df, const int32_t* __restrict__ indeg0, const int32_t* __restrict__ indeg) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < df.total;
       i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % df.G);
    df.pending[i] = i < df.G ? indeg0[g] : indeg[g];
    df.queue[i] = -1;
  }
}
__global__ void k_df_seed(DF df, const int32_t* __restrict__ indeg0) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < df.G; g += gridDim.x * blockDim.x)
    if (indeg0[g] == 0) {
      unsigned long long j = atomicAdd(df.tail, 1ull);
      df.queue[j] = g;
    }
}

template <int P, int BS>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_dataflow(Params a, DF df) {
  __shared__ long long s_node;
  __shared__ int s_stop;
  for (;;) {
    if (threadIdx.x == 0) {
      int stop = 0;
      long long node = -1;
      const unsigned long long slot = atomicAdd(df.head, 1ull);
      if ((long long)slot >= df.total || ld_acquire(df.err)) {
        stop = 1;
      } else {
        long long spins = 0;
        while ((node = ld_acquire(&df.queue[slot])) < 0) {
          if (++spins > df.max_spins || ld_acquire(df.err)) {
            atomicExch(df.err, 1);
            stop = 1;
            break;
          }
          __nanosleep(64);
        }
        __threadfence();
      }
      s_node = node;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) return;
    const long long node = s_node;
    const long long st = node / df.G;
    const int g = (int)(node % df.G);
    int k = 0;
    while (g >= df.cum[k + 1]) ++k;
    const int t = g - df.cum[k];
    for (int J = df.first[k]; J < df.last[k]; ++J) {
      const int32_t b = a.plan_ptr[J][t], e = a.plan_ptr[J][t + 1];
      const int32_t* items = a.plan_items[J];
      for (int32_t i = b + threadIdx.x; i < e; i += BS) run_loop<P, DF_L2_ONLY>(a, J, items[i], st);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      __threadfence();
      for (int q = df.succ_ptr[g]; q < df.succ_ptr[g + 1]; ++q) {
        const int e = df.succ[q];
        const long long s2 = st + (e & 1);
        if (s2 >= df.nsteps) continue;
        const long long n2 = s2 * df.G + (e >> 1);
        if (atom_add_acq_rel(&df.pending[n2], -1) == 1) {
          const unsigned long long j = atomicAdd(df.tail, 1ull);
          st_release(&df.queue[j], (int32_t)n2);
        }
      }
    }
  }
}

template <int P, int J>
void launch_loop(const Params& a, cudaStream_t s);

template <int P>
void launch_untiled_range(const Params& a, int first, int last, cudaStream_t s) {
  for (int J = first; J < last; ++J) {
    switch (J) {
      case 0: launch_loop<P, 0>(a, s); break;
      case 1: launch_loop<P, 1>(a, s); break;
      case 2: launch_loop<P, 2>(a, s); break;
      case 3: launch_loop<P, 3>(a, s); break;
      case 4: launch_loop<P, 4>(a, s); break;
      case 5: launch_loop<P, 5>(a, s); break;
      case 6: launch_loop<P, 6>(a, s); break;
      case 7: launch_loop<P, 7>(a, s); break;
      case 8: launch_loop<P, 8>(a, s); break;
      case 9: launch_loop<P, 9>(a, s); break;
      case 10: launch_loop<P, 10>(a, s); break;
      case 11: launch_loop<P, 11>(a, s); break;
      case 12: launch_loop<P, 12>(a, s); break;
      case 13: launch_loop<P, 13>(a, s); break;
      case 14: launch_loop<P, 14>(a, s); break;
      case 15: launch_loop<P, 15>(a, s); break;
      case 16: launch_loop<P, 16>(a, s); break;
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
  std::vector<int> cls;         // 0 = chain kernel, 1 = layout kernel
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
    double tot[2] = {0, 0}, cnt[2] = {0, 0}, mx = 0, mn = 1e300;
    for (size_t i = 0; i < cls.size(); ++i) {
      float ms = 0;
      SLT_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
      tot[cls[i]] += ms;
      cnt[cls[i]] += nl[i];
      if (cls[i] == 0) { mx = std::max(mx, (double)ms); mn = std::min(mn, (double)ms); }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    out[0] = tot[0]; out[1] = cnt[0]; out[2] = tot[1]; out[3] = cnt[1];
    out[4] = cnt[0] ? mx : 0; out[5] = cnt[0] ? mn : 0; out[6] = 0; out[7] = 0;
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
  return a;
}

template <int P, int J>
void launch_loop(const Params& a, cudaStream_t s) {
  int threads = 128;
  int64_t blocks = (a.nc + threads - 1) / threads;
  g_rec.begin(0, s);
  k_loop<P, J><<<(unsigned)blocks, threads, 0, s>>>(a);
  g_rec.end(s);
}

template <int P>
void launch_tiled_colour(const Params& a, int first, int last, const int32_t* tiles, int ntiles, int bs,
                         cudaStream_t s) {
  if (ntiles <= 0) return;
  g_rec.begin(0, s);
  if (bs == 128) k_tiled<P, 128><<<ntiles, 128, 0, s>>>(a, first, last, tiles);
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
  DataflowPlan& D = sched->df;
  DF df{};
  df.G = D.cum.back();
  df.nsteps = nsteps;
  df.total = (long long)nsteps * df.G;
  if (df.total == 0) return;
  if (df.total >= (1ll << 31)) fail(SLT_ERR_UNSUPPORTED, "steps x tiles must stay below 2^31");
  for (size_t k = 0; k < D.cum.size(); ++k) df.cum[k] = D.cum[k];
  for (size_t k = 0; k < sched->subs.size(); ++k) {
    const SubSched& sub = sched->subs[k];
    df.first[k] = sub.first;
    df.last[k] = sub.last;
    for (int j = sub.first; j < sub.last; ++j) {
      a.plan_ptr[j] = sub.plan_ptr[j - sub.first].p;
      a.plan_items[j] = sub.plan_items[j - sub.first].p;
    }
  }
  if (D.pending.n < (size_t)df.total) {
    D.pending.alloc(df.total);
    D.queue.alloc(df.total);
  }
  df.succ_ptr = D.succ_ptr.p;
  df.succ = D.succ.p;
  df.pending = D.pending.p;
  df.queue = D.queue.p;
  df.head = D.head.p;
  df.tail = D.head.p + 1;
  df.err = D.err.p;
  df.max_spins = sched->wait_spins;
  SLT_CUDA(cudaMemsetAsync(D.head.p, 0, 2 * sizeof(unsigned long long), s));
  SLT_CUDA(cudaMemsetAsync(D.err.p, 0, sizeof(int32_t), s));
  g_rec.begin(0, s, 3);
  k_df_init<<<(unsigned)std::min<long long>((df.total + 255) / 256, 152 * 16), 256, 0, s>>>(df, D.indeg0.p, D.indeg.p);
  k_df_seed<<<(df.G + 255) / 256, 256, 0, s>>>(df, D.indeg0.p);
  SLT_CUDA(cudaGetLastError());
  int dev = 0, nsm = 0, per = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int bs = sched->block;
  if (bs == 128) SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dataflow<P, 128>, 128, 0));
  else SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dataflow<P, 256>, 256, 0));
  long long grid = (long long)nsm * std::max(per, 1);
  if (grid > df.total) grid = df.total;
  if (bs == 128) k_dataflow<P, 128><<<(unsigned)grid, 128, 0, s>>>(a, df);
  else k_dataflow<P, 256><<<(unsigned)grid, 256, 0, s>>>(a, df);
  g_rec.end(s);
  SLT_CUDA(cudaGetLastError());
  int32_t herr = 0;
  SLT_CUDA(cudaMemcpyAsync(&herr, D.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  if (herr) fail(SLT_ERR_TIMEOUT, "a wait of the dataflow executor gave up");
}

template <int P>
void run_steps(slt_mesh m, slt_schedule sched, Params a, int64_t nsteps, cudaStream_t s) {
  if (sched && sched->executor == 0) {
    run_dataflow<P>(sched, a, nsteps, s);
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

void upload_constants(const RefElem& r) {
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
