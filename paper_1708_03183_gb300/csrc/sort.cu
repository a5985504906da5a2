// Device primitives of the inspector: stable LSD radix sort of (key, value) pairs, exclusive
// scan, CSR offsets from sorted keys, and the seed ranking (identity or Hilbert order).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace slt {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // items per block
constexpr int RS_BINS = 256;

__global__ void k_digit_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist,
                             int nblocks) {
  __shared__ int32_t cnt[RS_BINS];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: items are taken in (round, thread) order; within a round, equal digits are
// ranked by lane (warp match) and by warp (shared prefix), after all earlier rounds.
__global__ void k_digit_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                                int shift, const int32_t* __restrict__ offs, int nblocks, uint32_t* __restrict__ okeys,
                                uint32_t* __restrict__ ovals) {
  constexpr int NW = RS_THREADS / 32;
  __shared__ int32_t run[RS_BINS];
  __shared__ int32_t wcnt[NW][RS_BINS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    for (int w = 0; w < NW; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = base + r * RS_THREADS + threadIdx.x;
    bool valid = i < n;
    uint32_t k = valid ? keys[i] : 0u;
    uint32_t v = valid ? vals[i] : 0u;
    uint32_t d = valid ? ((k >> shift) & 0xFFu) : 0x100u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {  // per digit: prefix over warps, advance the running offset
      int d2 = threadIdx.x;
      int acc = run[d2];
      for (int w = 0; w < NW; ++w) {
        int c = wcnt[w][d2];
        wcnt[w][d2] = acc;
        acc += c;
      }
      run[d2] = acc;
    }
    __syncthreads();
    if (valid) {
      int pos = wcnt[warp][d] + rank;
      okeys[pos] = k;
      ovals[pos] = v;
    }
    __syncthreads();
  }
}

// Single-block exclusive scan of n int32 values (n + 1 outputs).
__global__ void k_scan_single(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  constexpr int T = 1024;
  __shared__ int64_t part[T];
  int64_t per = (n + T - 1) / T;
  int64_t lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    int64_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t acc = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t i = lo; i < hi; ++i) {
    out[i] = (int32_t)acc;
    acc += in[i];
  }
  if (threadIdx.x == T - 1) out[n] = (int32_t)part[T - 1];
}

// Multi-block exclusive scan: each block takes a tile of SC_THREADS x SC_ITEMS consecutive
// values (SC_ITEMS per thread); pass 1 writes the tile totals, a single block scans them, pass 2
// scans each tile from its offset.  Integer sums, so the result does not depend on the order.
constexpr int SC_THREADS = 512, SC_ITEMS = 8, SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ int32_t block_exclusive(int32_t x, int32_t* total) {
  __shared__ int32_t warp_sum[SC_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t w = lane < SC_THREADS / 32 ? warp_sum[lane] : 0, wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < SC_THREADS / 32) warp_sum[lane] = wi - w;  // exclusive prefix of the warps
    if (lane == SC_THREADS / 32 - 1) *total = wi;
  }
  __syncthreads();
  return warp_sum[wid] + incl - x;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_tiles(const int32_t* __restrict__ in, int64_t n,
                                                           int32_t* __restrict__ tsum) {
  __shared__ int32_t total;
  const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  int32_t s = 0;
#pragma unroll
  for (int v = 0; v < SC_ITEMS; ++v)
    if (base + v < n) s += in[base + v];
  block_exclusive(s, &total);
  if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                                                           const int32_t* __restrict__ toff,
                                                           int32_t* __restrict__ out) {
  __shared__ int32_t total;
  const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  int32_t v[SC_ITEMS], s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int32_t acc = toff[blockIdx.x] + block_exclusive(s, &total);
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k)
    if (base + k < n) {
      out[base + k] = acc;
      acc += v[k];
    }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = toff[gridDim.x];
}

__global__ void k_lower_bound(const uint32_t* __restrict__ sorted, int64_t n, int64_t nkeys, int32_t* __restrict__ offs) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t prev = p == 0 ? -1 : (int64_t)sorted[p - 1];
    int64_t cur = p == n ? nkeys : (int64_t)sorted[p];
    if (cur > nkeys) cur = nkeys;
    for (int64_t k = prev + 1; k <= cur; ++k) offs[k] = (int32_t)p;
  }
}

// ---------------------------------------------------------------- Hilbert ranking
__device__ __forceinline__ unsigned long long ord_of(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double of_ord(unsigned long long o) {
  unsigned long long b = (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o;
  return __longlong_as_double((long long)b);
}

__global__ void k_bbox(const double* __restrict__ xy, int64_t n, unsigned long long* __restrict__ box) {
  unsigned long long mnx = ~0ull, mny = ~0ull, mxx = 0, mxy = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long ox = ord_of(xy[2 * e]), oy = ord_of(xy[2 * e + 1]);
    mnx = ox < mnx ? ox : mnx; mxx = ox > mxx ? ox : mxx;
    mny = oy < mny ? oy : mny; mxy = oy > mxy ? oy : mxy;
  }
  atomicMin(&box[0], mnx);
  atomicMax(&box[1], mxx);
  atomicMin(&box[2], mny);
  atomicMax(&box[3], mxy);
}

// Hilbert index of (x, y) on a 2^16 grid; quadrant digits (lo,lo)=0, (lo,hi)=1, (hi,hi)=2,
// (hi,lo)=3 in (x, y), lower bits transposed in the lower quadrants and reflected in (hi,lo).
__device__ __forceinline__ uint32_t hilbert16(uint32_t x, uint32_t y) {
  uint32_t d = 0;
#pragma unroll 1
  for (int level = 15; level >= 0; --level) {
    uint32_t half = 1u << level;
    uint32_t hx = (x >> level) & 1u, hy = (y >> level) & 1u;
    d = (d << 2) | (hx ? (hy ? 2u : 3u) : (hy ? 1u : 0u));
    x &= half - 1u;
    y &= half - 1u;
    if (!hy) {
      if (hx) { x = half - 1u - x; y = half - 1u - y; }
      uint32_t t = x; x = y; y = t;
    }
  }
  return d;
}

__global__ void k_hilbert_keys(const double* __restrict__ xy, int64_t n, const unsigned long long* __restrict__ box,
                               uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  double xmin = of_ord(box[0]), xmax = of_ord(box[1]), ymin = of_ord(box[2]), ymax = of_ord(box[3]);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double tx = xmax > xmin ? __ddiv_rn(__dsub_rn(xy[2 * e], xmin), __dsub_rn(xmax, xmin)) : 0.0;
    double ty = ymax > ymin ? __ddiv_rn(__dsub_rn(xy[2 * e + 1], ymin), __dsub_rn(ymax, ymin)) : 0.0;
    long long qx = (long long)__dmul_rn(tx, 65535.0), qy = (long long)__dmul_rn(ty, 65535.0);
    qx = qx < 0 ? 0 : (qx > 65535 ? 65535 : qx);
    qy = qy < 0 ? 0 : (qy > 65535 ? 65535 : qy);
    keys[e] = hilbert16((uint32_t)qx, (uint32_t)qy);
    vals[e] = (uint32_t)e;
  }
}

__global__ void k_box_init(unsigned long long* __restrict__ box) {
  box[0] = ~0ull;
  box[1] = 0ull;
  box[2] = ~0ull;
  box[3] = 0ull;
}

__global__ void k_rank_from_order(const uint32_t* __restrict__ order, int64_t n, int32_t* __restrict__ rank) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    rank[order[p]] = (int32_t)p;
}
__global__ void k_iota(int32_t* __restrict__ a, int64_t n) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    a[p] = (int32_t)p;
}

inline int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

// ---- launch wrappers over caller-provided scratch (used by the allocation-free entry point)
void launch_bbox_init(unsigned long long* box, cudaStream_t s) {
  k_box_init<<<1, 1, 0, s>>>(box);
}
void launch_bbox(const double* xy, int64_t n, unsigned long long* box, cudaStream_t s) {
  k_bbox<<<grid_for(n), 256, 0, s>>>(xy, n, box);
}
void launch_hilbert_keys(const double* xy, int64_t n, const unsigned long long* box, uint32_t* keys, uint32_t* vals,
                         cudaStream_t s) {
  k_hilbert_keys<<<grid_for(n), 256, 0, s>>>(xy, n, box, keys, vals);
}
void launch_rank_from_order(const uint32_t* order, int64_t n, int32_t* rank, cudaStream_t s) {
  k_rank_from_order<<<grid_for(n), 256, 0, s>>>(order, n, rank);
}
int radix_blocks(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }
void radix_sort_pairs_with(uint32_t* keys, uint32_t* vals, int64_t n, int bits, uint32_t* tkeys, uint32_t* tvals,
                           int32_t* hist, int32_t* offs, cudaStream_t s) {
  if (n <= 1) return;
  int nblocks = radix_blocks(n);
  uint32_t *ik = keys, *iv = vals, *ok = tkeys, *ov = tvals;
  int passes = (bits + 7) / 8;
  for (int ps = 0; ps < passes; ++ps) {
    k_digit_hist<<<nblocks, RS_THREADS, 0, s>>>(ik, n, 8 * ps, hist, nblocks);
    k_scan_single<<<1, 1024, 0, s>>>(hist, offs, (int64_t)RS_BINS * nblocks);
    k_digit_scatter<<<nblocks, RS_THREADS, 0, s>>>(ik, iv, n, 8 * ps, offs, nblocks, ok, ov);
    uint32_t* t;
    t = ik; ik = ok; ok = t;
    t = iv; iv = ov; ov = t;
  }
  if (ik != keys) {
    SLT_CUDA(cudaMemcpyAsync(keys, ik, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    SLT_CUDA(cudaMemcpyAsync(vals, iv, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
}

int bits_for(int64_t maxval) {
  int b = 1;
  while (b < 32 && (int64_t(1) << b) <= maxval) ++b;
  return b;
}

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 4 * SC_TILE) {  // small: one block
    k_scan_single<<<1, 1024, 0, s>>>(in, out, n);
    SLT_CUDA(cudaGetLastError());
    return;
  }
  const int64_t nt = (n + SC_TILE - 1) / SC_TILE;
  DevBuf<int32_t> tsum(nt), toff(nt + 1);
  k_scan_tiles<<<(unsigned)nt, SC_THREADS, 0, s>>>(in, n, tsum.p);
  k_scan_single<<<1, 1024, 0, s>>>(tsum.p, toff.p, nt);
  k_scan_apply<<<(unsigned)nt, SC_THREADS, 0, s>>>(in, n, toff.p, out);
  SLT_CUDA(cudaGetLastError());
  // the temporaries are freed on return; the stream must have consumed them first
  SLT_CUDA(cudaStreamSynchronize(s));
}

void lower_bound_offsets(const uint32_t* sorted, int64_t n, int64_t nkeys, int32_t* offs, cudaStream_t s) {
  k_lower_bound<<<grid_for(n + 1), 256, 0, s>>>(sorted, n, nkeys, offs);
  SLT_CUDA(cudaGetLastError());
}

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, uint32_t* tkeys, uint32_t* tvals,
                      cudaStream_t s) {
  if (n <= 1) return;
  int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
  DevBuf<int32_t> hist((size_t)RS_BINS * nblocks), offs((size_t)RS_BINS * nblocks + 1);
  uint32_t *ik = keys, *iv = vals, *ok = tkeys, *ov = tvals;
  int passes = (bits + 7) / 8;
  for (int ps = 0; ps < passes; ++ps) {
    k_digit_hist<<<nblocks, RS_THREADS, 0, s>>>(ik, n, 8 * ps, hist.p, nblocks);
    SLT_CUDA(cudaGetLastError());
    exclusive_scan_i32(hist.p, offs.p, (int64_t)RS_BINS * nblocks, s);
    k_digit_scatter<<<nblocks, RS_THREADS, 0, s>>>(ik, iv, n, 8 * ps, offs.p, nblocks, ok, ov);
    SLT_CUDA(cudaGetLastError());
    uint32_t* t;
    t = ik; ik = ok; ok = t;
    t = iv; iv = ov; ov = t;
  }
  if (ik != keys) {
    SLT_CUDA(cudaMemcpyAsync(keys, ik, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    SLT_CUDA(cudaMemcpyAsync(vals, iv, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  SLT_CUDA(cudaStreamSynchronize(s));  // hist/offs are released on return
}

void seed_rank(const double* d_xy, int64_t n, int renumber, int32_t* d_rank, cudaStream_t s) {
  if (n == 0) return;
  if (!renumber) {
    k_iota<<<grid_for(n), 256, 0, s>>>(d_rank, n);
    SLT_CUDA(cudaGetLastError());
    return;
  }
  DevBuf<unsigned long long> box(4);
  unsigned long long init[4] = {~0ull, 0ull, ~0ull, 0ull};
  box.upload(init, 4, s);
  k_bbox<<<grid_for(n), 256, 0, s>>>(d_xy, n, box.p);
  SLT_CUDA(cudaGetLastError());
  DevBuf<uint32_t> k(n), v(n), tk(n), tv(n);
  k_hilbert_keys<<<grid_for(n), 256, 0, s>>>(d_xy, n, box.p, k.p, v.p);
  SLT_CUDA(cudaGetLastError());
  radix_sort_pairs(k.p, v.p, n, 32, tk.p, tv.p, s);
  k_rank_from_order<<<grid_for(n), 256, 0, s>>>(v.p, n, d_rank);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace slt
