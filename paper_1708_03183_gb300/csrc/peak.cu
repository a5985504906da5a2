// FP64 throughput probe: the arithmetic peak the executors are measured against.
//
// The elastic chain is FP64 arithmetic; its roofline denominator comes from the FP64 units, which
// the measured peaks (an HBM copy and a bf16 GEMM) do not cover.  Three kernels, each
// timed with CUDA events on the caller's stream after one warm-up launch:
//   - DFMA: every thread runs 8 independent fused multiply-add chains;
//   - DMMA: every warp runs 4 independent mma.sync.m8n8k4 FP64 accumulations (the warp-level
//     FP64 tensor instruction; tcgen05 has no FP64 kind);
//   - both at once: the even warps of a block run the DFMA loop, the odd warps the DMMA loop.
// Grid: 8 blocks of 256 threads per SM.  Results are written to a sink only when a runtime flag
// that is never set asks for it, so the loops cannot be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ void dfma_loop(int iters, double x, double* out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = x + k;
  const double b = 1.0 - 1e-9, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  *out = s;
}

// D = A (8x4) B (4x8) + C, FP64, one warp; per lane one element of A and B and two of C/D
__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void dmma_loop(int iters, double x, double* out) {
  constexpr int kAcc = 4;
  double d[kAcc][2];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) d[k][0] = d[k][1] = x + k;
  const double a = 1e-9 * (threadIdx.x & 31), b = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kAcc; ++k) dmma(d[k][0], d[k][1], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kAcc; ++k) s += d[k][0] + d[k][1];
  *out = s;
}

// DFMA with only `lanes` active lanes per warp (the others return at once)
__global__ void __launch_bounds__(256) k_fp64_lanes(int iters, int lanes, int flag, double* sink) {
  if ((int)(threadIdx.x & 31) >= lanes) return;
  double r;
  dfma_loop(iters, threadIdx.x, &r);
  if (flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// mode 0: DFMA, 1: DMMA, 2: even warps DFMA, odd warps DMMA (iters_mma for those)
__global__ void __launch_bounds__(256) k_fp64_probe(int mode, int iters, int iters_mma, int flag, double* sink) {
  const int warp = threadIdx.x >> 5;
  double r;
  const bool mma = mode == 1 || (mode == 2 && (warp & 1));
  if (mma) dmma_loop(mode == 1 ? iters : iters_mma, threadIdx.x, &r);
  else dfma_loop(iters, threadIdx.x, &r);
  if (flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace

extern "C" int slt_fp64_peak(void* stream, double out[4]) {
  try {
    if (!out) slt::fail(SLT_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    SLT_CUDA(cudaGetDevice(&dev));
    SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * 8, threads = 256;
    // DFMA: 8 chains x 2 flop per iteration and thread; DMMA: 4 x 512 flop per iteration and warp
    const int it_fma = 4096, it_mma = 2048;
    cudaEvent_t e0, e1;
    SLT_CUDA(cudaEventCreate(&e0));
    SLT_CUDA(cudaEventCreate(&e1));
    // in the mixed run the DMMA warps take half the iterations, so both halves do equal flops
    auto timed = [&](int mode) {
      k_fp64_probe<<<blocks, threads, 0, s>>>(mode, mode == 1 ? it_mma : it_fma, it_mma / 2, 0, nullptr);
      SLT_CUDA(cudaEventRecord(e0, s));
      k_fp64_probe<<<blocks, threads, 0, s>>>(mode, mode == 1 ? it_mma : it_fma, it_mma / 2, 0, nullptr);
      SLT_CUDA(cudaEventRecord(e1, s));
      SLT_CUDA(cudaEventSynchronize(e1));
      SLT_CUDA(cudaGetLastError());
      float ms = 0;
      SLT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return (double)ms;
    };
    const double thr = (double)blocks * threads, warps = thr / 32;
    const double f_fma = thr * it_fma * kChains * 2.0;
    const double f_mma = warps * it_mma * 4 * 512.0;
    const double t0 = timed(0), t1 = timed(1), t2 = timed(2);
    out[0] = f_fma / (t0 * 1e-3) / 1e12;
    out[1] = f_mma / (t1 * 1e-3) / 1e12;
    out[2] = (0.5 * f_fma + 0.25 * f_mma) / (t2 * 1e-3) / 1e12;
    out[3] = t0 + t1 + t2;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } catch (const slt::Error& e) {
    slt::set_error(e.msg);
    return e.code;
  } catch (...) {
    slt::set_error("unexpected exception");
    return SLT_ERR_CUDA;
  }
  return SLT_OK;
}

// How the FP64 pipe treats partial warps and few warps (the two facts the executors' design rests
// on): out[0] = DFMA warp instructions per clock per SM with 32 active lanes, out[1] = the same
// with 16 active lanes, out[2] = with one 32-lane warp per SM, out[3] = with four warps per SM
// (clock from cudaDevAttrClockRate, the maximum).  Each timed after a warm-up launch.
extern "C" int slt_fp64_lane_probe(void* stream, double out[4]) {
  try {
    if (!out) slt::fail(SLT_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0, khz = 0;
    SLT_CUDA(cudaGetDevice(&dev));
    SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SLT_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    cudaEvent_t e0, e1;
    SLT_CUDA(cudaEventCreate(&e0));
    SLT_CUDA(cudaEventCreate(&e1));
    auto timed = [&](int blocks, int threads, int lanes, int iters) {
      k_fp64_lanes<<<blocks, threads, 0, s>>>(iters, lanes, 0, nullptr);
      SLT_CUDA(cudaEventRecord(e0, s));
      k_fp64_lanes<<<blocks, threads, 0, s>>>(iters, lanes, 0, nullptr);
      SLT_CUDA(cudaEventRecord(e1, s));
      SLT_CUDA(cudaEventSynchronize(e1));
      SLT_CUDA(cudaGetLastError());
      float ms = 0;
      SLT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double warp_instr = (double)blocks * threads / 32 * iters * kChains;
      return warp_instr / (ms * 1e-3) / ((double)khz * 1e3) / nsm;
    };
    out[0] = timed(nsm * 8, 256, 32, 2048);
    out[1] = timed(nsm * 8, 256, 16, 2048);
    out[2] = timed(nsm, 32, 32, 8192);
    out[3] = timed(nsm, 128, 32, 8192);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } catch (const slt::Error& e) {
    slt::set_error(e.msg);
    return e.code;
  } catch (...) {
    slt::set_error("unexpected exception");
    return SLT_ERR_CUDA;
  }
  return SLT_OK;
}
