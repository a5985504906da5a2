// The volume contraction of the multi-shot form on the FP64 tensor instruction, against the DFMA
// form the executors use.
//
// With the shots innermost, the volume part of the operator A for one cell and one velocity
// component is a small dense product: u[i][s] = sum_k W[i][k] X[k][s], W = [Dr Ds] (Np x 2Np,
// the reference differentiation matrices side by side) and X the 2Np x S metric-combined stresses
// of the cell (rows rx sxx + ry sxy, then sx sxx + sy sxy at every node).  The executors evaluate
// it with one thread per (cell, shot) and DFMA, skipping the structural zeros of Dr and Ds.  Here
// the same product also runs as mma.sync.m8n8k4 FP64 tiles: one warp per cell, W in 8 x 4 tiles
// (zero-padded to 8-row and 4-column multiples), X in 4 x 8 tiles of 8 shots.  Both forms read
// the same X and write U[cell][Np][S]; the probe times each and returns their largest difference.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "refmask.h"

namespace {

constexpr int kMaxNp = 15;
__constant__ double c_w[kMaxNp * 2 * kMaxNp];  // W row-major, Np x 2Np

// a deterministic value in [-1, 1) of index i (splitmix64 finaliser)
__device__ __forceinline__ double unit_value(uint64_t i) {
  uint64_t z = i + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 4503599627370496.0) - 1.0;
}

__global__ void k_fill(double* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = unit_value((uint64_t)i);
}

// DFMA form: one thread per (cell, shot), structural zeros skipped at compile time
template <int P>
__global__ void __launch_bounds__(256) k_contract_dfma(const double* __restrict__ X, int64_t nc, int S,
                                                       double* __restrict__ U) {
  constexpr int Np = (P + 1) * (P + 2) / 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nc * S) return;
  const int64_t c = t / S;
  const int s = (int)(t % S);
  const double* x = X + c * 2 * Np * S + s;
  double a[Np], b[Np];
#pragma unroll
  for (int j = 0; j < Np; ++j) {
    a[j] = x[(int64_t)j * S];
    b[j] = x[(int64_t)(Np + j) * S];
  }
  double* u = U + c * Np * S + s;
#pragma unroll
  for (int i = 0; i < Np; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      if ((slt::dr_nz(P, i) >> j) & 1u) acc = fma(c_w[i * 2 * Np + j], a[j], acc);
      if ((slt::ds_nz(P, i) >> j) & 1u) acc = fma(c_w[i * 2 * Np + Np + j], b[j], acc);
    }
    u[(int64_t)i * S] = acc;
  }
}

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// DMMA form: one warp per cell; for each 8-shot column block and 8-row block of U, the K = 2Np
// columns of W in steps of 4.  Fragments of m8n8k4 (row.col): lane l holds A[l / 4][l % 4],
// B[l % 4][l / 4] and D[l / 4][2 (l % 4) + {0, 1}].  S is a multiple of 8.
template <int P>
__global__ void __launch_bounds__(256) k_contract_dmma(const double* __restrict__ X, int64_t nc, int S,
                                                       double* __restrict__ U) {
  constexpr int Np = (P + 1) * (P + 2) / 2, K = 2 * Np;
  constexpr int MT = (Np + 7) / 8, KT = (K + 3) / 4;
  const int lane = threadIdx.x & 31;
  const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (c >= nc) return;  // whole warps leave together
  double wa[MT][KT];  // this lane's element of every W tile
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      const int i = mt * 8 + lane / 4, k = kt * 4 + lane % 4;
      wa[mt][kt] = (i < Np && k < K) ? c_w[i * K + k] : 0.0;
    }
  const double* x = X + c * K * S;
  double* u = U + c * Np * S;
  for (int n0 = 0; n0 < S; n0 += 8) {
    double xb[KT];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      const int k = kt * 4 + lane % 4;
      xb[kt] = k < K ? x[(int64_t)k * S + n0 + lane / 4] : 0.0;
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      double d0 = 0.0, d1 = 0.0;
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) dmma(d0, d1, wa[mt][kt], xb[kt]);
      const int i = mt * 8 + lane / 4;
      if (i < Np) {
        u[(int64_t)i * S + n0 + 2 * (lane % 4)] = d0;
        u[(int64_t)i * S + n0 + 2 * (lane % 4) + 1] = d1;
      }
    }
  }
}

__global__ void k_maxdiff(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                          unsigned long long* __restrict__ out) {
  double m = 0.0, r = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    m = fmax(m, fabs(a[i] - b[i]));
    r = fmax(r, fabs(a[i]));
  }
  // non-negative doubles order like their bit patterns
  atomicMax(&out[0], (unsigned long long)__double_as_longlong(m));
  atomicMax(&out[1], (unsigned long long)__double_as_longlong(r));
}

template <int P>
void run_probe(int64_t nc, int S, cudaStream_t s, double out[6]) {
  constexpr int Np = (P + 1) * (P + 2) / 2;
  const slt::RefElem R = slt::make_refelem(P);
  std::vector<double> w((size_t)Np * 2 * Np);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      // the entries the build-time sparsity table marks as structural zeros are zero here too
      w[i * 2 * Np + j] = ((slt::dr_nz(P, i) >> j) & 1u) ? R.Dr[i * Np + j] : 0.0;
      w[i * 2 * Np + Np + j] = ((slt::ds_nz(P, i) >> j) & 1u) ? R.Ds[i * Np + j] : 0.0;
    }
  SLT_CUDA(cudaMemcpyToSymbolAsync(c_w, w.data(), w.size() * sizeof(double), 0, cudaMemcpyHostToDevice, s));
  int nnz = 0;
  for (double x : w) nnz += x != 0.0;
  const int64_t nx = nc * 2 * Np * S, nu = nc * Np * S;
  slt::DevBuf<double> X(nx), U0(nu), U1(nu);
  slt::DevBuf<unsigned long long> md(2);
  k_fill<<<152 * 16, 256, 0, s>>>(X.p, nx);
  const unsigned g0 = (unsigned)((nc * S + 255) / 256), g1 = (unsigned)((nc * 32 + 255) / 256);
  cudaEvent_t e[4];
  for (auto& x : e) SLT_CUDA(cudaEventCreate(&x));
  for (int rep = 0; rep < 2; ++rep) {  // the second repetition is timed
    SLT_CUDA(cudaEventRecord(e[0], s));
    k_contract_dfma<P><<<g0, 256, 0, s>>>(X.p, nc, S, U0.p);
    SLT_CUDA(cudaEventRecord(e[1], s));
    k_contract_dmma<P><<<g1, 256, 0, s>>>(X.p, nc, S, U1.p);
    SLT_CUDA(cudaEventRecord(e[2], s));
  }
  SLT_CUDA(cudaMemsetAsync(md.p, 0, 2 * sizeof(unsigned long long), s));
  k_maxdiff<<<152 * 8, 256, 0, s>>>(U0.p, U1.p, nu, md.p);
  SLT_CUDA(cudaGetLastError());
  unsigned long long h[2];
  SLT_CUDA(cudaMemcpyAsync(h, md.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  float t0 = 0, t1 = 0;
  SLT_CUDA(cudaEventElapsedTime(&t0, e[0], e[1]));
  SLT_CUDA(cudaEventElapsedTime(&t1, e[1], e[2]));
  for (auto& x : e) cudaEventDestroy(x);
  double dm, rm;
  std::memcpy(&dm, &h[0], 8);
  std::memcpy(&rm, &h[1], 8);
  out[0] = t0;
  out[1] = t1;
  out[2] = rm > 0 ? dm / rm : dm;
  out[3] = 2.0 * nnz * (double)nc * S;                                   // useful flops
  out[4] = 512.0 * ((Np + 7) / 8) * ((2 * Np + 3) / 4) * (double)nc * (S / 8);  // flops the DMMA form issues
  out[5] = nnz;
}

}  // namespace

extern "C" int slt_fp64_contraction_probe(int32_t degree, int64_t ncell, int32_t nshots, void* stream,
                                          double out[6]) {
  try {
    if (!out) slt::fail(SLT_ERR_ARG, "null argument");
    if (degree < 1 || degree > 4) slt::fail(SLT_ERR_ARG, "degree must be in 1..4");
    if (ncell < 1 || ncell > (int64_t(1) << 24)) slt::fail(SLT_ERR_ARG, "ncell must be in 1..2^24");
    if (nshots < 8 || nshots > 256 || nshots % 8) slt::fail(SLT_ERR_ARG, "nshots must be a multiple of 8 in 8..256");
    const int64_t np = (degree + 1) * (degree + 2) / 2;
    if (ncell * nshots * 4 * np > (int64_t(1) << 32))
      slt::fail(SLT_ERR_ARG, "ncell x nshots too large (the probe holds 4 Np doubles per cell and shot, at most 32 GB)");
    cudaStream_t s = (cudaStream_t)stream;
    switch (degree) {
      case 1: run_probe<1>(ncell, nshots, s, out); break;
      case 2: run_probe<2>(ncell, nshots, s, out); break;
      case 3: run_probe<3>(ncell, nshots, s, out); break;
      case 4: run_probe<4>(ncell, nshots, s, out); break;
    }
  } catch (const slt::Error& e) {
    slt::set_error(e.msg);
    return e.code;
  } catch (...) {
    slt::set_error("unexpected exception");
    return SLT_ERR_CUDA;
  }
  return SLT_OK;
}
