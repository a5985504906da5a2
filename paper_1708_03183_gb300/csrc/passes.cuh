// Executor 4: the persistent dataflow executor with each segment of a tile run as compacted passes
// (the lists of the staged plan: the first cell loop, interior faces 0, 1, 2, free-surface faces,
// the later cell loop), every value in global memory as in k_dataflow.  Included in exec.cu after
// staged.cuh.
//
// k_dataflow gives each plan item one thread for all its parts, so a warp issues every part any
// of its 32 items has: the items at tile boundaries (a cell whose facets belong to several tiles)
// leave lanes idle, and the FP64 pipe spends a full issue slot on a warp instruction whatever its
// active lanes.  Here each part runs as a pass over exactly the items that have it, so warps are
// full except for the last of each pass.  The price is a CTA barrier after each pass and the
// accumulated value passing between passes through L2 instead of registers.  The per-cell
// operations and their order are those of k_dataflow, so the results are bit-identical.
#pragma once

// global view of the phase's accumulated value, operand and work id of a list entry
__device__ __forceinline__ int64_t ps_w(const StageArgs& g, int k, int32_t f0, int32_t e) {
  return g.fp_cell[k][f0 + (e & slt::kNoSlot)] & 0x7fffffff;
}
__device__ __forceinline__ double* ps_acc(const Params& a, int H) {
  if (H == 5 && a.e5) return a.e5;
  return a.buf[H == 0 || H == 4 ? B_U1 : H == 2 ? B_U2 : B_E];
}
__device__ __forceinline__ const double* ps_in(const Params& a, int H) {
  return a.buf[H == 0 ? B_S : H == 1 || H == 5 ? B_U1 : H == 3 ? B_V : B_S1];
}

template <int P>
__device__ __forceinline__ void ps_init(const Params& a, int H, int64_t c, int fl) {
  constexpr int Np = np_of(P);
  if (!(fl & 8)) return;  // the value is already stored (partial sums of other tiles or segments)
  double acc[3 * Np];
  if (H == 0) {
    volB_v<P, true>(a, c, ps_in(a, H), a.ncp, c, acc);
    st_put<2 * Np>(ps_acc(a, H), a.ncp, c, acc);
  } else {
    volD_v<P, true>(a, c, ps_in(a, H), a.ncp, c, acc);
    st_put<3 * Np>(ps_acc(a, H), a.ncp, c, acc);
  }
}

template <int P, int F>
__device__ __forceinline__ void ps_face(const Params& a, int H, int64_t c) {
  constexpr int Np = np_of(P);
  const int64_t n = a.ncp;
  const int32_t nb = a.nbr[F * n + c];
  double* A = ps_acc(a, H);
  double acc[3 * Np];
  if (H == 0 || H == 2 || H == 4) {
    st_load<2 * Np>(A, n, c, acc);
    intB_face<P, true>(a, c, F, ps_in(a, H), n, c, nb >> 3, (nb >> 1) & 3, nb & 1, acc);
    st_put<2 * Np>(A, n, c, acc);
  } else {
    st_load<3 * Np>(A, n, c, acc);
    intD_face<P, true>(a, c, F, ps_in(a, H), n, c, nb >> 3, (nb >> 1) & 3, nb & 1, acc);
    st_put<3 * Np>(A, n, c, acc);
  }
}

template <int P>
__device__ __forceinline__ void ps_ext(const Params& a, int H, int64_t c, int fl) {
  constexpr int Np = np_of(P);
  const int64_t n = a.ncp;
  double* A = ps_acc(a, H);
  double acc[2 * Np];
  st_load<2 * Np>(A, n, c, acc);
#pragma unroll
  for (int f = 0; f < 3; ++f)
    if (((fl >> f) & 1) && a.nbr[f * n + c] < 0) extB_face<P, true>(a, c, f, ps_in(a, H), n, c, acc);
  st_put<2 * Np>(A, n, c, acc);
}

// the later cell loop, as segEB / segAV / segES do it after the item's facet parts
template <int P>
__device__ __forceinline__ void ps_pb(const Params& a, int H, int64_t c, int64_t step) {
  constexpr int Np = np_of(P);
  const int64_t n = a.ncp;
  double* const* b = a.buf;
  if (H == 1 || H == 3) {
    double e[3 * Np];
    st_load<3 * Np>(b[B_E], n, c, e);
    const double lam = a.mat[n + c], mu = a.mat[2 * n + c];
    const double l2m = a.pre[PRE_L2M * n + c];
    double* S1 = b[B_S1];
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      S1[(int64_t)j * n + c] = fma(lam, e[Np + j], l2m * e[j]);
      S1[(int64_t)(Np + j) * n + c] = fma(lam, e[j], l2m * e[Np + j]);
      S1[(int64_t)(2 * Np + j) * n + c] = mu * e[2 * Np + j];
    }
    double u[2 * Np];
    volB_v<P, true>(a, c, S1, n, c, u);
    st_put<2 * Np>(b[H == 1 ? B_U2 : B_U1], n, c, u);
  } else if (H == 2) {
    double* V = b[B_V];
    const double* U1 = b[B_U1];
    const double* U2 = b[B_U2];
#pragma unroll
    for (int r = 0; r < 2 * Np; ++r) {
      const int64_t o = (int64_t)r * n + c;
      V[o] = fma(a.dt, fma(a.c24, __ldcg(&U2[o]), __ldcg(&U1[o])), __ldcg(&V[o]));
    }
  } else {  // H == 5
    double* S = b[B_S];
    const double* E = a.e5 ? a.e5 : b[B_E];
    const double* S1 = b[B_S1];
    const double lam = a.mat[n + c], mu = a.mat[2 * n + c];
    const double l2m = a.pre[PRE_L2M * n + c];
    const bool src = (c == a.src_w) && a.ricker != nullptr;
    const double gs = src ? a.dt * a.ricker[step] : 0.0;
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      const int64_t oxx = (int64_t)j * n + c, oyy = (int64_t)(Np + j) * n + c, oxy = (int64_t)(2 * Np + j) * n + c;
      const double exx = __ldcg(&E[oxx]), eyy = __ldcg(&E[oyy]), gxy = __ldcg(&E[oxy]);
      double cxx = fma(lam, eyy, l2m * exx), cyy = fma(lam, exx, l2m * eyy), cxy = mu * gxy;
      double nxx = fma(a.dt, fma(a.c24, cxx, __ldcg(&S1[oxx])), __ldcg(&S[oxx]));
      double nyy = fma(a.dt, fma(a.c24, cyy, __ldcg(&S1[oyy])), __ldcg(&S[oyy]));
      S[oxy] = fma(a.dt, fma(a.c24, cxy, __ldcg(&S1[oxy])), __ldcg(&S[oxy]));
      if (src) {
        nxx += gs * a.src[j];
        nyy += gs * a.src[j];
      }
      S[oxx] = nxx;
      S[oyy] = nyy;
    }
  }
}

template <int P, int BS>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_passes(Params a, DF df, StageArgs g) {
  __shared__ long long s_node;
  long long kept = -1;  // (thread 0's copy is the one used)
  for (;;) {
    if (threadIdx.x == 0) s_node = kept >= 0 ? kept : df_take(df.q);
    __syncthreads();
    const long long node = s_node;
    if (node < 0) return;
    const long long st = node / df.q.G;
    const int gi = (int)(node % df.q.G);
    int k = 0;
    while (gi >= df.cum[k + 1]) ++k;
    const int t = gi - df.cum[k];
    const int32_t f0 = g.fp_ptr[k][t];
    for (int J = df.first[k]; J < df.last[k]; J = seg_end(J, df.last[k])) {
      const int H = phase_of(J);
      const int32_t* off = g.off[J] + t * slt::SL_N;
      const int32_t* ent = g.ent[J];
      int32_t o[slt::SL_N + 1];
#pragma unroll
      for (int L = 0; L <= slt::SL_N; ++L) o[L] = off[L];
      // (the gather list is not used: every value stays in global memory)
      if (o[2] > o[1]) {
        for (int32_t i = o[1] + threadIdx.x; i < o[2]; i += BS) {
          const int32_t e = ent[i];
          ps_init<P>(a, H, ps_w(g, k, f0, e), e >> slt::kSlotBits);
        }
        __syncthreads();
      }
      if (o[3] > o[2]) {
        for (int32_t i = o[2] + threadIdx.x; i < o[3]; i += BS) ps_face<P, 0>(a, H, ps_w(g, k, f0, ent[i]));
        __syncthreads();
      }
      if (o[4] > o[3]) {
        for (int32_t i = o[3] + threadIdx.x; i < o[4]; i += BS) ps_face<P, 1>(a, H, ps_w(g, k, f0, ent[i]));
        __syncthreads();
      }
      if (o[5] > o[4]) {
        for (int32_t i = o[4] + threadIdx.x; i < o[5]; i += BS) ps_face<P, 2>(a, H, ps_w(g, k, f0, ent[i]));
        __syncthreads();
      }
      if (o[6] > o[5]) {
        for (int32_t i = o[5] + threadIdx.x; i < o[6]; i += BS) {
          const int32_t e = ent[i];
          ps_ext<P>(a, H, ps_w(g, k, f0, e), e >> slt::kSlotBits);
        }
        __syncthreads();
      }
      if (o[7] > o[6]) {
        for (int32_t i = o[6] + threadIdx.x; i < o[7]; i += BS) ps_pb<P>(a, H, ps_w(g, k, f0, ent[i]), st);
        __syncthreads();
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) kept = df_publish(df.q, gi, st);
  }
}
