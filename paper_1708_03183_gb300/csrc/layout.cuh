// Caller layout <-> work layout of the multi-shot fields: caller [cell][row][S] (shots fastest),
// work [(row * ncp + w) * S + s] (rows of ncp * S doubles, Hilbert work order).  Included inside
// an anonymous namespace of each translation unit that converts multi-shot fields.
#pragma once

// caller [cell][row][S] <-> work [(row * ncp + w) * S + s], shots fastest on both sides
__global__ void k_to_work_b(const double* __restrict__ in, int rows, int S, const int32_t* __restrict__ perm,
                            int64_t nc, int64_t ncp, double* __restrict__ out) {
  const int64_t n = nc * rows * S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i % S, r = (i / S) % rows, w = i / ((int64_t)S * rows);
    out[((int64_t)r * ncp + w) * S + s] = in[((int64_t)perm[w] * rows + r) * S + s];
  }
}
__global__ void k_from_work_b(const double* __restrict__ in, int rows, int S, const int32_t* __restrict__ perm,
                              int64_t nc, int64_t ncp, double* __restrict__ out) {
  const int64_t n = nc * rows * S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i % S, r = (i / S) % rows, w = i / ((int64_t)S * rows);
    out[((int64_t)perm[w] * rows + r) * S + s] = in[((int64_t)r * ncp + w) * S + s];
  }
}

