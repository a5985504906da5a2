// Persistent dataflow executor of the tiled chain, shared by the single-field (exec.cu) and
// multi-shot (exec_batched.cu) translation units; included after exec_body.cuh inside an
// anonymous namespace.
#pragma once

// No register cap: forcing 24 warps per SM (80 registers at p = 2) made the tiled kernels slower
// (their loads are latency bound and more resident tiles overflow L2); one CTA is the minimum.
template <int P, int BS>
constexpr int tile_min_blocks() {
  return P <= 2 ? 768 / BS : 1;
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

template <int P, int BS, bool BATCH>
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
      if constexpr (BATCH) {  // every item for every shot, consecutive threads on consecutive shots
        const int64_t nwork = (int64_t)(e - b) * a.S;
        for (int64_t i = threadIdx.x; i < nwork; i += BS)
          run_loop<P, DF_L2_ONLY, true>(a, J, items[b + i / a.S], st, (int)(i % a.S));
      } else {
        for (int32_t i = b + threadIdx.x; i < e; i += BS) run_loop<P, DF_L2_ONLY, false>(a, J, items[i], st);
      }
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


// Launch the dataflow executor for nsteps on the schedule's plan; `rec_begin` / `rec_end` bracket
// the three kernels for the caller's timing.  Synchronises; SLT_ERR_TIMEOUT when a wait gave up.
template <int P, bool BATCH, class RB, class RE>
void launch_dataflow(::slt_schedule_s* sched, Params a, int64_t nsteps, cudaStream_t s, RB rec_begin, RE rec_end) {
  slt::DataflowPlan& D = sched->df;
  DF df{};
  df.G = D.cum.back();
  df.nsteps = nsteps;
  df.total = (long long)nsteps * df.G;
  if (df.total == 0) return;
  if (df.total >= (1ll << 31)) slt::fail(SLT_ERR_UNSUPPORTED, "steps x tiles must stay below 2^31");
  for (size_t k = 0; k < D.cum.size(); ++k) df.cum[k] = D.cum[k];
  for (size_t k = 0; k < sched->subs.size(); ++k) {
    const slt::SubSched& sub = sched->subs[k];
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
  rec_begin();
  k_df_init<<<(unsigned)std::min<long long>((df.total + 255) / 256, 152 * 16), 256, 0, s>>>(df, D.indeg0.p,
                                                                                          D.indeg.p);
  k_df_seed<<<(df.G + 255) / 256, 256, 0, s>>>(df, D.indeg0.p);
  SLT_CUDA(cudaGetLastError());
  int dev = 0, nsm = 0, per = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int bs = sched->block;
  if (bs == 128) SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dataflow<P, 128, BATCH>, 128, 0));
  else SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dataflow<P, 256, BATCH>, 256, 0));
  long long grid = (long long)nsm * std::max(per, 1);
  if (grid > df.total) grid = df.total;
  if (bs == 128) k_dataflow<P, 128, BATCH><<<(unsigned)grid, 128, 0, s>>>(a, df);
  else k_dataflow<P, 256, BATCH><<<(unsigned)grid, 256, 0, s>>>(a, df);
  rec_end();
  SLT_CUDA(cudaGetLastError());
  int32_t herr = 0;
  SLT_CUDA(cudaMemcpyAsync(&herr, D.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  if (herr) slt::fail(SLT_ERR_TIMEOUT, "a wait of the dataflow executor gave up");
}
