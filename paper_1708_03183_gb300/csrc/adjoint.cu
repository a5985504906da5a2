// Seismogram misfit and its gradient with respect to per-cell rho, lambda, mu: the discrete
// adjoint of the fourth-order staggered Taylor leapfrog of the DG elastic chain.
//
// Misfit J = 1/2 dt sum_n sum_r |P_r v^{n+1/2} - d_r^n|^2 for a run from rest.  With
// A~ = A + c ABA, B~ = B + c BAB (c = dt^2/24) and the skew identity M_rho A = -B^T M_S of the
// centered-flux operators, the adjoint in mass-weighted variables (vt = M_rho^-1 adj v,
// st = M_S^-1 adj sigma) is the same leapfrog run backwards with -dt:
//     vt += -dt A~ st;   vt += dt M_rho^-1 P^T r^n;   st += -dt B~ vt,
// and the parameter derivatives are cell-local M-weighted bilinear forms (|det J| M_hat):
//   stress update (st, forward v = v^{n+1/2}):
//     g_lam += dt (<C^-1 st, C_lam E(v)> + c <C^-1 st, C_lam E(ABv)> + c <E(A st), C_lam E(v)>)
//     g_rho += c dt <A st, ABv>
//   velocity update (vt, forward sigma = sigma^n):
//     g_rho += -dt (<vt, A~ sigma> + c <AB vt, A sigma>);  g_lam += -c dt <E(vt), C_lam E(A sigma)>
// (mu likewise with C_mu).  Forward states are recomputed segment by segment from checkpoints
// of (v, sigma) taken every k steps.  The single-field path below runs the forward steps on the
// mesh's executor (tiled when a schedule is given) and the adjoint steps through the untiled
// operator loops; the many-shot path further down runs forward, recompute and adjoint steps
// alike as the chain's two sub-chains, untiled or on the schedule's tiles.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace slt {

namespace {

constexpr int MAXNP = 15;
__constant__ double c_mass[5][MAXNP * MAXNP];  // reference mass matrix per degree

inline int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}

// traces[s][r][c] = sum_j phi_rj V[c Np + j][w_r S + s] (rows of fs = ncp S doubles)
__global__ void k_record(const double* __restrict__ V, int64_t fs, int S, int Np, int nrec,
                         const int32_t* __restrict__ rw, const double* __restrict__ phi, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nrec * S) return;
  const int sh = t / (2 * nrec), r = (t >> 1) % nrec, c = t & 1;
  double acc = 0.0;
  for (int j = 0; j < Np; ++j)
    acc = fma(phi[r * Np + j], V[(int64_t)(c * Np + j) * fs + (int64_t)rw[r] * S + sh], acc);
  out[t] = acc;
}

// vt[c Np + i][w_r S + s] += dt (trace - data)[s][r][c] q_r[i] / rho, receivers in order (one block)
__global__ void k_inject(double* __restrict__ VT, int64_t fs, int S, int Np, int nrec, const int32_t* __restrict__ rw,
                         const double* __restrict__ q, const double* __restrict__ tr, const double* __restrict__ dat,
                         const double* __restrict__ irho, double dt) {
  for (int t = threadIdx.x; t < 2 * Np * S; t += blockDim.x) {
    const int sh = t / (2 * Np), c = (t / Np) % 2, i = t % Np;
    for (int r = 0; r < nrec; ++r) {
      int64_t w = rw[r];
      double res = tr[(sh * nrec + r) * 2 + c] - dat[(sh * nrec + r) * 2 + c];
      VT[(int64_t)(c * Np + i) * fs + w * S + sh] += dt * res * q[r * Np + i] * irho[w];
    }
  }
}

// J = 1/2 dt sum (tr - dat)^2 over n values (one block)
__global__ void k_misfit(const double* __restrict__ tr, const double* __restrict__ dat, int64_t n, double dt,
                         double* __restrict__ out) {
  __shared__ double part[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double d = tr[i] - dat[i];
    acc = fma(d, d, acc);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = 0.5 * dt * part[0];
}

// out = C in (stored strain -> stored stress), per cell and node
__global__ void k_hooke(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ mat,
                        int64_t nc, int64_t ncp, int Np) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nc; w += (int64_t)gridDim.x * blockDim.x) {
    double lam = mat[ncp + w], mu = mat[2 * ncp + w], l2m = fma(2.0, mu, lam);
    for (int j = 0; j < Np; ++j) {
      double exx = in[(int64_t)j * ncp + w], eyy = in[(int64_t)(Np + j) * ncp + w], g = in[(int64_t)(2 * Np + j) * ncp + w];
      out[(int64_t)j * ncp + w] = fma(lam, eyy, l2m * exx);
      out[(int64_t)(Np + j) * ncp + w] = fma(lam, exx, l2m * eyy);
      out[(int64_t)(2 * Np + j) * ncp + w] = mu * g;
    }
  }
}

// y += a x + b z over `rows` rows of nc entries
__global__ void k_axpy2(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ z, double a,
                        double b, int rows, int64_t nc, int64_t ncp) {
  const int64_t n = (int64_t)rows * nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / nc, w = i % nc, o = r * ncp + w;
    y[o] = fma(b, z[o], fma(a, x[o], y[o]));
  }
}

template <int Np>
__device__ __forceinline__ void mvec(const double* M, const double* x, double* y) {
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < Np; ++j) acc = fma(M[i * MAXNP + j], x[j], acc);
    y[i] = acc;
  }
}

template <int Np>
__device__ __forceinline__ void load_rows(const double* f, int row0, int64_t ncp, int64_t w, double* x) {
#pragma unroll
  for (int j = 0; j < Np; ++j) x[j] = f[(int64_t)(row0 + j) * ncp + w];
}

// sum_ij M_ij a_i b_j for one component of two fields
template <int Np>
__device__ __forceinline__ double mform(const double* M, const double* a, const double* b) {
  double Mb[Np];
  mvec<Np>(M, b, Mb);
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < Np; ++i) acc = fma(a[i], Mb[i], acc);
  return acc;
}

// <e1, C_lam e2>_M and <e1, C_mu e2>_M for strain-like fields (rows xx, yy, xy)
template <int Np>
__device__ __forceinline__ void cforms(const double* M, const double* e1f, const double* e2f, int64_t ncp, int64_t w,
                                       bool e1_is_stress_inv, double lam, double mu, double& fl, double& fm) {
  double a[3][Np], b[3][Np];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    load_rows<Np>(e1f, k * Np, ncp, w, a[k]);
    load_rows<Np>(e2f, k * Np, ncp, w, b[k]);
  }
  if (e1_is_stress_inv) {  // a <- C^-1 a: inverse of [[l2m, lam], [lam, l2m]] (+) mu
    double l2m = fma(2.0, mu, lam), det = l2m * l2m - lam * lam;
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      double sxx = a[0][j], syy = a[1][j];
      a[0][j] = (l2m * sxx - lam * syy) / det;
      a[1][j] = (l2m * syy - lam * sxx) / det;
      a[2][j] = a[2][j] / mu;
    }
  }
  double ta[Np], tb[Np];
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    ta[j] = a[0][j] + a[1][j];
    tb[j] = b[0][j] + b[1][j];
  }
  fl = mform<Np>(M, ta, tb);
  fm = 2.0 * mform<Np>(M, a[0], b[0]) + 2.0 * mform<Np>(M, a[1], b[1]) + mform<Np>(M, a[2], b[2]);
}

template <int Np>
__device__ __forceinline__ double vform(const double* M, const double* af, const double* bf, int64_t ncp, int64_t w) {
  double a[Np], b[Np], acc = 0.0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    load_rows<Np>(af, k * Np, ncp, w, a);
    load_rows<Np>(bf, k * Np, ncp, w, b);
    acc += mform<Np>(M, a, b);
  }
  return acc;
}

// stress-update terms: st (adjoint of sigma^{n+1}), Ev, E_ABv, E_Ast (strains), Ast, ABv
template <int P>
__global__ void k_grad_s(const double* __restrict__ st, const double* __restrict__ Ev, const double* __restrict__ EABv,
                         const double* __restrict__ EAst, const double* __restrict__ Ast, const double* __restrict__ ABv,
                         const double* __restrict__ mat, const double* __restrict__ adet, int64_t nc, int64_t ncp,
                         int S, double dt, double c, double* __restrict__ g) {
  constexpr int Np = (P + 1) * (P + 2) / 2;
  const double* M = c_mass[P];
  const int64_t fs = ncp * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc * S; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = t / S;
    const double lam = mat[ncp + w], mu = mat[2 * ncp + w], d = adet[w];
    double l1, m1, l2, m2, l3, m3;
    cforms<Np>(M, st, Ev, fs, t, true, lam, mu, l1, m1);
    cforms<Np>(M, st, EABv, fs, t, true, lam, mu, l2, m2);
    cforms<Np>(M, EAst, Ev, fs, t, false, lam, mu, l3, m3);
    g[t] += c * dt * d * vform<Np>(M, Ast, ABv, fs, t);
    g[fs + t] += dt * d * (l1 + c * l2 + c * l3);
    g[2 * fs + t] += dt * d * (m1 + c * m2 + c * m3);
  }
}

// velocity-update terms: vt (adjoint of v^{n+1/2}), Asig, ABAsig, ABvt, Evt, E_Asig
template <int P>
__global__ void k_grad_v(const double* __restrict__ vt, const double* __restrict__ Asig,
                         const double* __restrict__ ABAsig, const double* __restrict__ ABvt,
                         const double* __restrict__ Evt, const double* __restrict__ EAsig,
                         const double* __restrict__ mat, const double* __restrict__ adet, int64_t nc, int64_t ncp,
                         int S, double dt, double c, double* __restrict__ g) {
  constexpr int Np = (P + 1) * (P + 2) / 2;
  const double* M = c_mass[P];
  const int64_t fs = ncp * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc * S; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = t / S;
    const double lam = mat[ncp + w], mu = mat[2 * ncp + w], d = adet[w];
    const double f1 = vform<Np>(M, vt, Asig, fs, t) + c * vform<Np>(M, vt, ABAsig, fs, t);
    const double f2 = vform<Np>(M, ABvt, Asig, fs, t);
    double l, m;
    cforms<Np>(M, Evt, EAsig, fs, t, false, lam, mu, l, m);
    g[t] += -dt * d * (f1 + c * f2);
    g[fs + t] += -c * dt * d * l;
    g[2 * fs + t] += -c * dt * d * m;
  }
}

// the gradient in caller numbering, summed over the shots in order
__global__ void k_grad_out(const double* __restrict__ g, const int32_t* __restrict__ perm, int64_t nc, int64_t ncp,
                           int S, double* __restrict__ out) {
  const int64_t fs = ncp * S;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nc; w += (int64_t)gridDim.x * blockDim.x) {
    int64_t cell = perm[w];
    for (int k = 0; k < 3; ++k) {
      double acc = g[k * fs + w * S];
      for (int sh = 1; sh < S; ++sh) acc += g[k * fs + w * S + sh];
      out[k * nc + cell] = acc;
    }
  }
}

}  // namespace

void upload_adjoint_constants(const RefElem& r) {
  double h[MAXNP * MAXNP] = {};
  // reference mass matrix: inverse of the stored inverse (Minv) by Gauss-Jordan
  const int n = r.Np;
  std::vector<double> A(r.Minv), I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int row = col + 1; row < n; ++row)
      if (std::fabs(A[row * n + col]) > std::fabs(A[piv * n + col])) piv = row;
    for (int k = 0; k < n; ++k) { std::swap(A[col * n + k], A[piv * n + k]); std::swap(I[col * n + k], I[piv * n + k]); }
    double dd = A[col * n + col];
    for (int k = 0; k < n; ++k) { A[col * n + k] /= dd; I[col * n + k] /= dd; }
    for (int row = 0; row < n; ++row) {
      if (row == col) continue;
      double f = A[row * n + col];
      for (int k = 0; k < n; ++k) { A[row * n + k] -= f * A[col * n + k]; I[row * n + k] -= f * I[col * n + k]; }
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) h[i * MAXNP + j] = I[i * n + j];
  SLT_CUDA(cudaMemcpyToSymbol(c_mass, h, sizeof(h), r.p * sizeof(h)));
}

void record_run(slt_mesh m, slt_schedule sched, slt_receivers rec, const double* ricker, double dt, int64_t nsteps,
                double* traces, cudaStream_t s) {
  const int64_t ncp = m->ncp;
  double* V = m->work.p;
  SLT_CUDA(cudaMemsetAsync(m->work.p, 0, 5 * (int64_t)m->Np * ncp * sizeof(double), s));
  for (int64_t n = 0; n < nsteps; ++n) {
    exec_steps_work(m, sched, ricker, dt, n, 1, s);
    k_record<<<(2 * rec->n + 127) / 128, 128, 0, s>>>(V, ncp, 1, m->Np, rec->n, rec->w.p, rec->phi.p,
                                                      traces + n * 2 * rec->n);
  }
  SLT_CUDA(cudaGetLastError());
}

void adjoint_run(slt_mesh m, slt_schedule sched, slt_receivers rec, const double* ricker, double dt, int64_t N,
                 const double* data, int32_t k_arg, double* grad_out, double* J_host, cudaStream_t s) {
  const int32_t k = k_arg < 0 ? -k_arg : k_arg;  // k_arg < 0: segments keep states only
  const int Np = m->Np, P = m->p;
  const int64_t nc = m->nc, ncp = m->ncp, row = ncp;
  const int64_t nseg = (N + k - 1) / k;
  const int64_t state = 5 * (int64_t)Np * ncp;  // V [2Np] then S [3Np], as in the work buffer
  double* V = m->work.p;
  double* S = m->work.p + 2 * (int64_t)Np * ncp;
  DevBuf<double> ckpt(std::max<int64_t>(nseg, 1) * state), seg;
  // the forward intermediates of every step of a segment (15 Np rows each), when memory allows;
  // otherwise the segment keeps only its states and the reverse sweep recomputes them
  const int64_t keep_rows = 15 * (int64_t)Np * ncp;
  DevBuf<double> keep;
  if (k_arg > 0) {
    try {
      keep.alloc((int64_t)k * keep_rows);
    } catch (const Error&) {
      keep.release();
    }
  }
  if (!keep.p) seg.alloc((int64_t)k * state);
  DevBuf<double> traces(std::max<int64_t>(N * 2 * rec->n, 1)), Jd(1);
  DevBuf<double> adj(20 * (int64_t)Np * row), g(3 * row);
  double* vt = adj.p;
  double* st = vt + 2 * Np * row;
  double* T2a = st + 3 * Np * row;
  double* T2b = T2a + 2 * Np * row;
  double* T2c = T2b + 2 * Np * row;
  double* T3a = T2c + 2 * Np * row;
  double* T3b = T3a + 3 * Np * row;
  double* T3c = T3b + 3 * Np * row;
  const int gr = grid_for(nc);
  const double c = dt * dt / 24.0;
  // forward pass: checkpoints and traces
  SLT_CUDA(cudaMemsetAsync(m->work.p, 0, state * sizeof(double), s));
  for (int64_t n = 0; n < N; ++n) {
    if (n % k == 0)
      SLT_CUDA(cudaMemcpyAsync(ckpt.p + (n / k) * state, V, state * sizeof(double), cudaMemcpyDeviceToDevice, s));
    exec_steps_work(m, sched, ricker, dt, n, 1, s);
    k_record<<<(2 * rec->n + 127) / 128, 128, 0, s>>>(V, ncp, 1, Np, rec->n, rec->w.p, rec->phi.p,
                                                      traces.p + n * 2 * rec->n);
  }
  k_misfit<<<1, 1024, 0, s>>>(traces.p, data, N * 2 * rec->n, dt, Jd.p);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaMemsetAsync(adj.p, 0, adj.n * sizeof(double), s));
  SLT_CUDA(cudaMemsetAsync(g.p, 0, g.n * sizeof(double), s));
  auto hooke = [&](const double* in, double* out) {
    k_hooke<<<gr, 256, 0, s>>>(in, out, m->mat.p, nc, ncp, Np);
  };
  auto axpy = [&](double* y, const double* x, const double* z, double a, double b, int rows) {
    k_axpy2<<<grid_for((int64_t)rows * nc), 256, 0, s>>>(y, x, z, a, b, rows, nc, ncp);
  };
  for (int64_t j = nseg - 1; j >= 0; --j) {
    const int64_t n0 = j * k, n1 = std::min<int64_t>(N, n0 + k);
    SLT_CUDA(cudaMemcpyAsync(V, ckpt.p + j * state, state * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int64_t n = n0; n < n1; ++n) {  // recompute the segment
      if (keep.p) {  // the step's intermediates stay in its slot
        exec_step_keep(m, ricker, dt, n, keep.p + (n - n0) * keep_rows, s);
        continue;
      }
      double* slot = seg.p + (n - n0) * state;  // sigma^n before the step, v^{n+1/2} after it
      SLT_CUDA(cudaMemcpyAsync(slot + 2 * (int64_t)Np * ncp, S, 3 * (int64_t)Np * ncp * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
      exec_steps_work(m, sched, ricker, dt, n, 1, s);
      SLT_CUDA(cudaMemcpyAsync(slot, V, 2 * (int64_t)Np * ncp * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    for (int64_t n = n1 - 1; n >= n0; --n) {
      const int64_t r = (int64_t)Np * ncp;
      const double* kept = keep.p ? keep.p + (n - n0) * keep_rows : nullptr;
      // forward intermediates of step n: kept, or recomputed from the segment's states
      const double *Asig, *EAsig, *ABAsig, *Ev, *ABv, *EABv;
      if (kept) {
        Asig = kept;
        EAsig = kept + 2 * r;
        ABAsig = kept + 5 * r;
        Ev = kept + 7 * r;
        ABv = kept + 10 * r;
        EABv = kept + 12 * r;
      } else {
        const double* v = seg.p + (n - n0) * state;
        const double* sig = v + 2 * r;
        op_E(m, v, T3a, s);        // Ev
        hooke(T3a, T3b);           // Bv
        op_A(m, T3b, T2a, s);      // ABv
        op_E(m, T2a, T3b, s);      // E(ABv)
        op_A(m, sig, T2c, s);      // A sigma (kept in T2c until the velocity update)
        Ev = T3a;
        ABv = T2a;
        EABv = T3b;
        Asig = T2c;
        EAsig = ABAsig = nullptr;  // computed below, after T2a/T3a are free
      }
      // stress update (adjoint st of sigma^{n+1})
      op_A(m, st, T2b, s);       // A st
      op_E(m, T2b, T3c, s);      // E(A st)
      switch (P) {
        case 1: k_grad_s<1><<<gr, 128, 0, s>>>(st, Ev, EABv, T3c, T2b, ABv, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
        case 2: k_grad_s<2><<<gr, 128, 0, s>>>(st, Ev, EABv, T3c, T2b, ABv, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
        case 3: k_grad_s<3><<<gr, 128, 0, s>>>(st, Ev, EABv, T3c, T2b, ABv, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
        case 4: k_grad_s<4><<<gr, 128, 0, s>>>(st, Ev, EABv, T3c, T2b, ABv, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
      }
      hooke(T3c, T3a);           // BA st
      op_A(m, T3a, T2a, s);      // ABA st
      axpy(vt, T2b, T2a, -dt, -dt * c, 2 * Np);
      // receivers
      k_inject<<<1, 128, 0, s>>>(vt, ncp, 1, Np, rec->n, rec->w.p, rec->q.p, traces.p + n * 2 * rec->n,
                                 data + n * 2 * rec->n, m->mat.p, dt);
      // velocity update (adjoint vt of v^{n+1/2})
      if (!kept) {
        SLT_CUDA(cudaMemcpyAsync(T2a, Asig, 2 * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
        Asig = T2a;
        op_E(m, Asig, T3a, s);   // E(A sigma)
        hooke(T3a, T3b);         // BA sigma
        op_A(m, T3b, T2b, s);    // ABA sigma
        EAsig = T3a;
        ABAsig = T2b;
      }
      op_E(m, vt, T3b, s);       // E vt
      hooke(T3b, T3c);           // B vt
      op_A(m, T3c, T2c, s);      // AB vt
      switch (P) {
        case 1: k_grad_v<1><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, T2c, T3b, EAsig, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
        case 2: k_grad_v<2><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, T2c, T3b, EAsig, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
        case 3: k_grad_v<3><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, T2c, T3b, EAsig, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
        case 4: k_grad_v<4><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, T2c, T3b, EAsig, m->mat.p, m->adet.p, nc, ncp, 1, dt, c, g.p); break;
      }
      op_E(m, T2c, T3a, s);      // E(AB vt)
      hooke(T3a, T3b);           // BAB vt
      axpy(st, T3c, T3b, -dt, -dt * c, 3 * Np);
      SLT_CUDA(cudaGetLastError());
    }
  }
  k_grad_out<<<gr, 256, 0, s>>>(g.p, m->d_perm.p, nc, ncp, 1, grad_out);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaMemcpyAsync(J_host, Jd.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
}


// ------------------------------------------------------------------ many shots, tiled or untiled
// The same misfit and gradient for S shots at once (their sum over the shots), on the multi-shot
// work layout (rows of ncp S doubles, column cell S + shot), with every operator application
// run by the chain executors: the untiled phase kernels when sched is null, else the dataflow
// executor on the schedule's tiles ({velocity, stress} fusion).
//  - forward: one step at a time (the receivers record after each), checkpoints of (v, sigma)
//    every k steps;
//  - segment recompute: each step as its two sub-chains, their temporaries written into the
//    step's keep slot (A sigma, E(A sigma), ABA sigma from the velocity sub-chain; E(v), AB v,
//    E(AB v) from the stress sub-chain, whose last strain goes to its own slot);
//  - reverse sweep: the adjoint step is the leapfrog run with -dt on (vt, st), so each step is
//    the velocity sub-chain on (vt, st) (leaving A st and E(A st)), the stress-update gradient
//    terms, the receiver residuals, the stress sub-chain on (vt, st) (leaving E(vt) and AB vt),
//    and the velocity-update gradient terms.  The forward schedule serves unchanged: under the
//    skew identity the adjoint step is the same loop chain, so its tiles and colours are legal
//    for it as they are.
void record_run_b(slt_mesh m, slt_schedule sched, slt_receivers rec, int32_t S, const int32_t* d_src_w,
                  const double* d_src, const double* ricker, double dt, int64_t nsteps, double* traces,
                  cudaStream_t s) {
  const int64_t Np = m->Np, fs = m->ncp * S;
  DevBuf<double> fwd(15 * Np * fs);
  SLT_CUDA(cudaMemsetAsync(fwd.p, 0, 5 * Np * fs * sizeof(double), s));
  ChainRun r;
  r.S = S;
  for (int b = 0; b < 6; ++b) r.buf[b] = fwd.p + (b == 0 ? 0 : b == 1 ? 2 : b == 2 ? 5 : b == 3 ? 7 : b == 4 ? 9 : 12) * Np * fs;
  r.dt = dt;
  r.src_w = d_src_w;
  r.src = d_src;
  const int nrec = rec->n;
  for (int64_t n = 0; n < nsteps; ++n) {
    r.ricker = ricker ? ricker + n : nullptr;
    chain_part_b(m, sched, r, 2, s);
    k_record<<<(2 * nrec * S + 127) / 128, 128, 0, s>>>(r.buf[0], fs, S, (int)Np, nrec, rec->w.p, rec->phi.p,
                                                        traces + n * 2 * nrec * S);
  }
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaStreamSynchronize(s));
}

void adjoint_run_b(slt_mesh m, slt_schedule sched, slt_receivers rec, int32_t S, const int32_t* d_src_w,
                   const double* d_src, const double* ricker, double dt, int64_t N, const double* data, int32_t k,
                   double* grad_out, double* J_host, cudaStream_t s) {
  if (k < 1) fail(SLT_ERR_ARG, "checkpoint_every must be >= 1 for the multi-shot or tiled adjoint");
  const int Np = m->Np, P = m->p;
  const int64_t nc = m->nc, ncp = m->ncp, fs = ncp * S, R = Np * fs;  // R: Np rows
  const int64_t nseg = (N + k - 1) / k;
  const int nrec = rec->n;
  DevBuf<double> fwd(15 * R), ckpt(std::max<int64_t>(nseg, 1) * 5 * R), keep((int64_t)k * 15 * R);
  DevBuf<double> adj(18 * R), g(3 * fs), traces(std::max<int64_t>(N * 2 * nrec * S, 1)), Jd(1);
  double* V = fwd.p;
  double* Sg = fwd.p + 2 * R;
  double* fU1 = fwd.p + 5 * R;
  double* fU2 = fwd.p + 7 * R;
  double* fE = fwd.p + 9 * R;
  double* fS1 = fwd.p + 12 * R;
  double* vt = adj.p;             // 2 Np
  double* st = vt + 2 * R;        // 3 Np
  double* TA = st + 3 * R;        // 2 Np: A st, then AB vt
  double* TEA = TA + 2 * R;       // 3 Np: E(A st), then E(AB vt) (not used)
  double* TU2 = TEA + 3 * R;      // 2 Np
  double* TS1 = TU2 + 2 * R;      // 3 Np
  double* TE3 = TS1 + 3 * R;      // 3 Np: E(vt)
  const double c = dt * dt / 24.0;
  auto run = [&](double* v, double* sg, double* u1, double* u2, double* e, double* s1, double* e5,
                 const double* rk, double h, const int32_t* sw, const double* sv, int part) {
    ChainRun r;
    r.S = S;
    r.buf[0] = v; r.buf[1] = sg; r.buf[2] = u1; r.buf[3] = u2; r.buf[4] = e; r.buf[5] = s1;
    r.e5 = e5;
    r.ricker = rk;
    r.dt = h;
    r.src_w = sw;
    r.src = sv;
    chain_part_b(m, sched, r, part, s);
  };
  // forward: checkpoints and traces
  SLT_CUDA(cudaMemsetAsync(fwd.p, 0, 5 * R * sizeof(double), s));
  for (int64_t n = 0; n < N; ++n) {
    if (n % k == 0)
      SLT_CUDA(cudaMemcpyAsync(ckpt.p + (n / k) * 5 * R, V, 5 * R * sizeof(double), cudaMemcpyDeviceToDevice, s));
    run(V, Sg, fU1, fU2, fE, fS1, nullptr, ricker ? ricker + n : nullptr, dt, d_src_w, d_src, 2);
    k_record<<<(2 * nrec * S + 127) / 128, 128, 0, s>>>(V, fs, S, Np, nrec, rec->w.p, rec->phi.p,
                                                        traces.p + n * 2 * nrec * S);
  }
  k_misfit<<<1, 1024, 0, s>>>(traces.p, data, N * 2 * nrec * S, dt, Jd.p);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaMemsetAsync(adj.p, 0, adj.n * sizeof(double), s));
  SLT_CUDA(cudaMemsetAsync(g.p, 0, g.n * sizeof(double), s));
  const int gr = grid_for(nc * S);
  for (int64_t j = nseg - 1; j >= 0; --j) {
    const int64_t n0 = j * k, n1 = std::min<int64_t>(N, n0 + k);
    SLT_CUDA(cudaMemcpyAsync(V, ckpt.p + j * 5 * R, 5 * R * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int64_t n = n0; n < n1; ++n) {  // recompute, keeping each step's operator intermediates
      double* K = keep.p + (n - n0) * 15 * R;
      const double* rk = ricker ? ricker + n : nullptr;
      run(V, Sg, K, K + 5 * R, K + 2 * R, fS1, nullptr, rk, dt, d_src_w, d_src, 0);
      run(V, Sg, K + 10 * R, fU2, K + 7 * R, fS1, K + 12 * R, rk, dt, d_src_w, d_src, 1);
    }
    for (int64_t n = n1 - 1; n >= n0; --n) {
      const double* K = keep.p + (n - n0) * 15 * R;
      const double *Asig = K, *EAsig = K + 2 * R, *ABAsig = K + 5 * R, *Ev = K + 7 * R, *ABv = K + 10 * R,
                   *EABv = K + 12 * R;
      // velocity sub-chain of the adjoint step: vt -= dt (A st + c ABA st); leaves A st, E(A st)
      run(vt, st, TA, TU2, TEA, TS1, nullptr, nullptr, -dt, nullptr, nullptr, 0);
      switch (P) {
        case 1: k_grad_s<1><<<gr, 128, 0, s>>>(st, Ev, EABv, TEA, TA, ABv, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
        case 2: k_grad_s<2><<<gr, 128, 0, s>>>(st, Ev, EABv, TEA, TA, ABv, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
        case 3: k_grad_s<3><<<gr, 128, 0, s>>>(st, Ev, EABv, TEA, TA, ABv, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
        case 4: k_grad_s<4><<<gr, 128, 0, s>>>(st, Ev, EABv, TEA, TA, ABv, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
      }
      k_inject<<<1, 256, 0, s>>>(vt, fs, S, Np, nrec, rec->w.p, rec->q.p, traces.p + n * 2 * nrec * S,
                                 data + n * 2 * nrec * S, m->mat.p, dt);
      // stress sub-chain: st -= dt (B vt + c BAB vt); leaves E(vt) and AB vt
      run(vt, st, TA, TU2, TE3, TS1, TEA, nullptr, -dt, nullptr, nullptr, 1);
      switch (P) {
        case 1: k_grad_v<1><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, TA, TE3, EAsig, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
        case 2: k_grad_v<2><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, TA, TE3, EAsig, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
        case 3: k_grad_v<3><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, TA, TE3, EAsig, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
        case 4: k_grad_v<4><<<gr, 128, 0, s>>>(vt, Asig, ABAsig, TA, TE3, EAsig, m->mat.p, m->adet.p, nc, ncp, S, dt, c, g.p); break;
      }
      SLT_CUDA(cudaGetLastError());
    }
  }
  k_grad_out<<<grid_for(nc), 256, 0, s>>>(g.p, m->d_perm.p, nc, ncp, S, grad_out);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaMemcpyAsync(J_host, Jd.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace slt
