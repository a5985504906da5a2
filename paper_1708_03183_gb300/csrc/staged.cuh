// Staged executor (executor 3): the persistent dataflow executor with each tile's sub-chain run
// out of shared memory (Section 5.2, Algorithm 4: a tile's slice of every loop, fused; Section
// 3.2: the data of a tile reused across its loops).  Included in exec.cu after dataflow.cuh.
//
// A CTA takes ready (step, tile) nodes from the same queue as k_dataflow.  For a node it loads
// the tile's footprint (the cells its segments touch, slot = position; the inspector's local map
// of the cell set), then runs each segment as passes over compacted lists, with a CTA barrier
// after each pass:
//   gather + init   operands the tile has not produced itself are read once from global memory
//                   into shared memory (every read after this comes from shared memory); the
//                   accumulated value of each item starts (volume part, or the stored partial
//                   value another tile left)
//   faces 0, 1, 2   interior facet parts, one face index per pass (uniform, full warps)
//   free surface    exterior facet parts
//   later loop      Hooke's law and the volume part of A, or the updates of v and sigma
// Each cell's operations run in the order of the loop-by-loop chain with the same arithmetic as
// the other executors (the shared part functions of exec_body.cuh), so the results are
// bit-identical to theirs.  Temporaries stay in shared memory and are written to global memory
// only when another tile (or a later sub-chain) reads them: shared cells, partial sums.
//
// Shared memory per slot: three regions R0 [3 Np], R1 [3 Np], R2 [2 Np] (rows of `cap` doubles),
// reused as values die, plus the slot's work id and neighbour slots:
//   velocity sub-chain  R0 sigma (gathered) then E then S1 = C E, R2 U1 = A sigma, R1 U2
//   stress sub-chain    R1 v (gathered) then E(U1), R0 E then S1, R2 U1 = A S1
#pragma once

struct StageArgs {
  int32_t cap;                    // slots per region (row stride)
  int32_t cross;                  // every written temporary also goes to global memory
  const int32_t* fp_ptr[16];      // per sub-chain: footprint offsets per tile
  const int32_t* fp_cell[16];     // work id | shared << 31
  const int32_t* fp_nsl[16];      // neighbour slots, kSlotBits per face
  const int32_t* off[17];         // per segment (at its first loop): 7 list offsets per tile
  const int32_t* ent[17];         // list entries
};

// smem field views of the current node
struct StageMem {
  double* R[3];
  const int32_t* cell;            // work id | shared << 31 per slot
  const int32_t* nsl;             // neighbour slots per slot
  int64_t cap;
};

__device__ __forceinline__ int64_t st_w(const StageMem& M, int32_t sl) { return M.cell[sl] & 0x7fffffff; }
__device__ __forceinline__ bool st_shared(const StageMem& M, int32_t sl) { return M.cell[sl] < 0; }
__device__ __forceinline__ int32_t st_nb(const StageMem& M, int32_t sl, int f) {
  return (M.nsl[sl] >> (slt::kSlotBits * f)) & slt::kNoSlot;
}

template <int R>
__device__ __forceinline__ void st_load(const double* X, int64_t fs, int64_t w, double* x) {
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = __ldcg(&X[(int64_t)r * fs + w]);
}
template <int R>
__device__ __forceinline__ void st_put(double* X, int64_t fs, int64_t w, const double* x) {
#pragma unroll
  for (int r = 0; r < R; ++r) X[(int64_t)r * fs + w] = x[r];
}
template <int R>
__device__ __forceinline__ void st_get(const double* X, int64_t fs, int64_t w, double* x) {
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = X[(int64_t)r * fs + w];
}
// global rows of `src` at work id w into region rows at slot sl
template <int R>
__device__ __forceinline__ void st_gather(const double* src, int64_t ncp, int64_t w, double* dst, int64_t cap,
                                          int32_t sl) {
#pragma unroll
  for (int r = 0; r < R; ++r) dst[(int64_t)r * cap + sl] = __ldcg(&src[(int64_t)r * ncp + w]);
}

// Gather entry of phase H: kind 0 the segment's operand, kind 1 the later cell loop's own extra
// operand (U1 for the velocity update, S1 for the stress update).
template <int P>
__device__ __forceinline__ void st_gather_entry(const Params& a, const StageMem& M, int H, int32_t e) {
  constexpr int Np = np_of(P);
  const int32_t sl = e & slt::kNoSlot;
  const int kind = e >> slt::kSlotBits;
  const int64_t w = st_w(M, sl), n = a.ncp;
  double* const* b = a.buf;
  switch (H) {
    case 0: st_gather<3 * Np>(b[B_S], n, w, M.R[0], M.cap, sl); break;
    case 1: st_gather<2 * Np>(b[B_U1], n, w, M.R[2], M.cap, sl); break;
    case 2:
      if (kind == 0) st_gather<3 * Np>(b[B_S1], n, w, M.R[0], M.cap, sl);
      else st_gather<2 * Np>(b[B_U1], n, w, M.R[2], M.cap, sl);
      break;
    case 3: st_gather<2 * Np>(b[B_V], n, w, M.R[1], M.cap, sl); break;
    case 4: st_gather<3 * Np>(b[B_S1], n, w, M.R[0], M.cap, sl); break;
    default:
      if (kind == 0) st_gather<2 * Np>(b[B_U1], n, w, M.R[2], M.cap, sl);
      else st_gather<3 * Np>(b[B_S1], n, w, M.R[0], M.cap, sl);
      break;
  }
}

// The accumulated value of phase H: its region, rows, and global buffer.
template <int P>
__device__ __forceinline__ int st_acc_rows(int H) {
  return (H == 1 || H == 3 || H == 5) ? 3 * np_of(P) : 2 * np_of(P);
}
__device__ __forceinline__ int st_acc_region(int H) {
  return H == 0 || H == 4 ? 2 : H == 1 || H == 3 ? 0 : 1;
}
__device__ __forceinline__ int st_acc_buf(int H) {
  return H == 0 || H == 4 ? B_U1 : H == 2 ? B_U2 : B_E;
}
// the operand region of phase H's volume and facet parts
__device__ __forceinline__ int st_in_region(int H) {
  return H == 1 || H == 5 ? 2 : H == 3 ? 1 : 0;
}

// An item's accumulated value is final for this tile after its last facet part (or its first
// cell loop when it has none): write it out when another tile (or sub-chain) needs it.  The
// strain E and U2 are needed elsewhere exactly when this tile does not run the later cell loop;
// U1 when the cell is shared.
template <int P>
__device__ __forceinline__ void st_commit(const Params& a, const StageMem& M, const StageArgs& g, int H, int32_t sl,
                                          int fl, const double* acc) {
  constexpr int Np = np_of(P);
  const bool pb = fl & 16;
  const int64_t w = st_w(M, sl);
  if (H == 0 || H == 4) {
    if (st_shared(M, sl) || g.cross) st_put<2 * Np>(a.buf[B_U1], a.ncp, w, acc);
  } else if (H == 2) {
    if (!pb) st_put<2 * Np>(a.buf[B_U2], a.ncp, w, acc);
  } else {
    if (!pb) st_put<3 * Np>(a.buf[B_E], a.ncp, w, acc);
  }
}

// number of facet parts of an item that come after interior face f (to find its last one)
__device__ __forceinline__ bool st_last_face(const StageMem& M, int32_t sl, int fl, int f) {
  for (int g = f + 1; g < 3; ++g)
    if ((fl >> g) & 1) return false;  // a later interior face, or a free-surface face (after all)
  for (int g = 0; g <= f; ++g)
    if (((fl >> g) & 1) && st_nb(M, sl, g) == slt::kNoSlot) return false;  // a free-surface face
  return true;
}

// Init entry of phase H: the first cell loop's volume part, or the stored partial value, or
// nothing (the value is already in shared memory).  Commits items without facet parts.
template <int P>
__device__ __forceinline__ void st_init_entry(const Params& a, const StageMem& M, const StageArgs& g, int H,
                                              int32_t e) {
  constexpr int Np = np_of(P);
  const int32_t sl = e & slt::kNoSlot;
  const int fl = e >> slt::kSlotBits;
  const int64_t c = st_w(M, sl), cap = M.cap;
  double acc[3 * Np];
  const int rows = st_acc_rows<P>(H);
  double* A = M.R[st_acc_region(H)];
  if (fl & 8) {
    const double* X = M.R[st_in_region(H)];
    if (H == 0) volB_v<P, false>(a, c, X, cap, sl, acc);
    else volD_v<P, false>(a, c, X, cap, sl, acc);
  } else if (fl & slt::kLoadBit) {
    if (rows == 3 * Np) st_load<3 * Np>(a.buf[st_acc_buf(H)], a.ncp, c, acc);
    else st_load<2 * Np>(a.buf[st_acc_buf(H)], a.ncp, c, acc);
  } else {
    if (!(fl & 7)) {  // resident and nothing to add here: still commit below
      if (rows == 3 * Np) st_get<3 * Np>(A, cap, sl, acc);
      else st_get<2 * Np>(A, cap, sl, acc);
    } else {
      return;
    }
  }
  if (rows == 3 * Np) st_put<3 * Np>(A, cap, sl, acc);
  else st_put<2 * Np>(A, cap, sl, acc);
  if (!(fl & 7)) st_commit<P>(a, M, g, H, sl, fl, acc);
}

// Interior face F of an item: the facet part of phase H onto the accumulated value.
template <int P, int F>
__device__ __forceinline__ void st_face_entry(const Params& a, const StageMem& M, const StageArgs& g, int H,
                                              int32_t e) {
  constexpr int Np = np_of(P);
  const int32_t sl = e & slt::kNoSlot;
  const int fl = e >> slt::kSlotBits;
  const int64_t c = st_w(M, sl), cap = M.cap;
  const int32_t nb = a.nbr[F * a.ncp + c];
  const int32_t ns = st_nb(M, sl, F);
  const double* X = M.R[st_in_region(H)];
  double* A = M.R[st_acc_region(H)];
  double acc[3 * Np];
  if (H == 0 || H == 2 || H == 4) {
    st_get<2 * Np>(A, cap, sl, acc);
    intB_face<P, false>(a, c, F, X, cap, sl, ns, (nb >> 1) & 3, nb & 1, acc);
    st_put<2 * Np>(A, cap, sl, acc);
  } else {
    st_get<3 * Np>(A, cap, sl, acc);
    intD_face<P, false>(a, c, F, X, cap, sl, ns, (nb >> 1) & 3, nb & 1, acc);
    st_put<3 * Np>(A, cap, sl, acc);
  }
  if (st_last_face(M, sl, fl, F)) st_commit<P>(a, M, g, H, sl, fl, acc);
}

// Free-surface faces of an item (after all its interior faces), phases 0, 2, 4.
template <int P>
__device__ __forceinline__ void st_ext_entry(const Params& a, const StageMem& M, const StageArgs& g, int H,
                                             int32_t e) {
  constexpr int Np = np_of(P);
  const int32_t sl = e & slt::kNoSlot;
  const int fl = e >> slt::kSlotBits;
  const int64_t c = st_w(M, sl), cap = M.cap;
  const double* X = M.R[st_in_region(H)];
  double* A = M.R[st_acc_region(H)];
  double acc[2 * Np];
  st_get<2 * Np>(A, cap, sl, acc);
#pragma unroll
  for (int f = 0; f < 3; ++f)
    if (((fl >> f) & 1) && st_nb(M, sl, f) == slt::kNoSlot) extB_face<P, false>(a, c, f, X, cap, sl, acc);
  st_put<2 * Np>(A, cap, sl, acc);
  st_commit<P>(a, M, g, H, sl, fl, acc);
}

// The later cell loop of an item: Hooke's law and the volume part of A (phases 1, 3), the
// velocity update (2), the stress update and source (5); the same arithmetic as segEB, segAV and
// segES.
template <int P>
__device__ __forceinline__ void st_pb_entry(const Params& a, const StageMem& M, const StageArgs& g, int H, int32_t e,
                                            int64_t step) {
  constexpr int Np = np_of(P);
  const int32_t sl = e & slt::kNoSlot;
  const int64_t c = st_w(M, sl), cap = M.cap, n = a.ncp;
  double* const* b = a.buf;
  if (H == 1 || H == 3) {
    double* S1 = M.R[0];
    const double lam = a.mat[n + c], mu = a.mat[2 * n + c];
    const double l2m = a.pre[PRE_L2M * n + c];
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      const double exx = S1[(int64_t)j * cap + sl], eyy = S1[(int64_t)(Np + j) * cap + sl],
                   gxy = S1[(int64_t)(2 * Np + j) * cap + sl];
      S1[(int64_t)j * cap + sl] = fma(lam, eyy, l2m * exx);
      S1[(int64_t)(Np + j) * cap + sl] = fma(lam, exx, l2m * eyy);
      S1[(int64_t)(2 * Np + j) * cap + sl] = mu * gxy;
    }
    const bool out = st_shared(M, sl) || g.cross;
    if (out) {
      double s1[3 * Np];
      st_get<3 * Np>(S1, cap, sl, s1);
      st_put<3 * Np>(b[B_S1], n, c, s1);
    }
    double u[2 * Np];
    volB_v<P, false>(a, c, S1, cap, sl, u);
    st_put<2 * Np>(M.R[H == 1 ? 1 : 2], cap, sl, u);
    if (out) st_put<2 * Np>(b[H == 1 ? B_U2 : B_U1], n, c, u);
  } else if (H == 2) {
    double* V = b[B_V];
    const double* U1 = M.R[2];
    const double* U2 = M.R[1];
#pragma unroll
    for (int r = 0; r < 2 * Np; ++r) {
      const int64_t o = (int64_t)r * n + c;
      V[o] = fma(a.dt, fma(a.c24, U2[(int64_t)r * cap + sl], U1[(int64_t)r * cap + sl]), __ldcg(&V[o]));
    }
  } else {  // H == 5
    double* S = b[B_S];
    const double* E = M.R[1];
    const double* S1 = M.R[0];
    const double lam = a.mat[n + c], mu = a.mat[2 * n + c];
    const double l2m = a.pre[PRE_L2M * n + c];
    const bool src = (c == a.src_w) && a.ricker != nullptr;
    const double gs = src ? a.dt * a.ricker[step] : 0.0;
#pragma unroll
    for (int j = 0; j < Np; ++j) {
      const double exx = E[(int64_t)j * cap + sl], eyy = E[(int64_t)(Np + j) * cap + sl],
                   gxy = E[(int64_t)(2 * Np + j) * cap + sl];
      double cxx = fma(lam, eyy, l2m * exx), cyy = fma(lam, exx, l2m * eyy), cxy = mu * gxy;
      const int64_t oxx = (int64_t)j * n + c, oyy = (int64_t)(Np + j) * n + c, oxy = (int64_t)(2 * Np + j) * n + c;
      double nxx = fma(a.dt, fma(a.c24, cxx, S1[(int64_t)j * cap + sl]), __ldcg(&S[oxx]));
      double nyy = fma(a.dt, fma(a.c24, cyy, S1[(int64_t)(Np + j) * cap + sl]), __ldcg(&S[oyy]));
      S[oxy] = fma(a.dt, fma(a.c24, cxy, S1[(int64_t)(2 * Np + j) * cap + sl]), __ldcg(&S[oxy]));
      if (src) {
        nxx += gs * a.src[j];
        nyy += gs * a.src[j];
      }
      S[oxx] = nxx;
      S[oyy] = nyy;
    }
  }
}

// bytes of dynamic shared memory for `cap` slots at degree P
__host__ __device__ constexpr int64_t stage_smem_bytes(int P, int64_t cap) {
  return cap * (64 * (int64_t)np_of(P) + 8);
}

template <int P, int BS>
__global__ void __launch_bounds__(BS, 1) k_staged(Params a, DF df, StageArgs g) {
  extern __shared__ __align__(16) double st_sm[];
  __shared__ long long s_node;
  constexpr int Np = np_of(P);
  const int64_t cap = g.cap;
  StageMem M;
  M.R[0] = st_sm;
  M.R[1] = M.R[0] + 3 * Np * cap;
  M.R[2] = M.R[1] + 3 * Np * cap;
  int32_t* s_cell = reinterpret_cast<int32_t*>(M.R[2] + 2 * Np * cap);
  int32_t* s_nsl = s_cell + cap;
  M.cell = s_cell;
  M.nsl = s_nsl;
  M.cap = cap;
  long long kept = -1;
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
    const int32_t f0 = g.fp_ptr[k][t], nF = g.fp_ptr[k][t + 1] - f0;
    for (int32_t i = threadIdx.x; i < nF; i += BS) {
      s_cell[i] = g.fp_cell[k][f0 + i];
      s_nsl[i] = g.fp_nsl[k][f0 + i];
    }
    __syncthreads();
    for (int J = df.first[k]; J < df.last[k]; J = seg_end(J, df.last[k])) {
      const int H = phase_of(J);
      const int32_t* off = g.off[J] + t * slt::SL_N;
      const int32_t* ent = g.ent[J];
      int32_t o[slt::SL_N + 1];
#pragma unroll
      for (int L = 0; L <= slt::SL_N; ++L) o[L] = off[L];
      if (o[1] > o[0]) {
        for (int32_t i = o[0] + threadIdx.x; i < o[1]; i += BS) st_gather_entry<P>(a, M, H, ent[i]);
        __syncthreads();
      }
      if (o[2] > o[1]) {
        for (int32_t i = o[1] + threadIdx.x; i < o[2]; i += BS) st_init_entry<P>(a, M, g, H, ent[i]);
        __syncthreads();
      }
      if (o[3] > o[2]) {
        for (int32_t i = o[2] + threadIdx.x; i < o[3]; i += BS) st_face_entry<P, 0>(a, M, g, H, ent[i]);
        __syncthreads();
      }
      if (o[4] > o[3]) {
        for (int32_t i = o[3] + threadIdx.x; i < o[4]; i += BS) st_face_entry<P, 1>(a, M, g, H, ent[i]);
        __syncthreads();
      }
      if (o[5] > o[4]) {
        for (int32_t i = o[4] + threadIdx.x; i < o[5]; i += BS) st_face_entry<P, 2>(a, M, g, H, ent[i]);
        __syncthreads();
      }
      if (o[6] > o[5]) {
        for (int32_t i = o[5] + threadIdx.x; i < o[6]; i += BS) st_ext_entry<P>(a, M, g, H, ent[i]);
        __syncthreads();
      }
      if (o[7] > o[6]) {
        for (int32_t i = o[6] + threadIdx.x; i < o[7]; i += BS) st_pb_entry<P>(a, M, g, H, ent[i], st);
        __syncthreads();
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) kept = df_publish(df.q, gi, st);
  }
}
