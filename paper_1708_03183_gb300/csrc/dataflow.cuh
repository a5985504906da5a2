// Persistent dataflow executor of the tiled chain, shared by the single-field (exec.cu) and
// multi-shot (exec_batched.cu) translation units; included after exec_body.cuh inside an
// anonymous namespace.
#pragma once

// Resident tiles per SM: at p <= 2, 768 threads (three 256-thread tiles, 80 registers; the
// heaviest phase bodies spill a little, which measured faster than two tiles at 128 registers);
// at p = 3 two 256-thread tiles (128 registers, about 90 bytes of spills; the tiles in flight
// double); at p = 4 the phase bodies need their registers and one tile is the minimum.
template <int P, int BS>
constexpr int tile_min_blocks() {
  return P <= 2 ? 768 / BS : (P == 3 && BS == 256) ? 2 : 1;
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
struct DFQ {
  long long total;                // nodes = nsteps * G
  long long nsteps;
  int32_t G;                      // tiles over all sub-chains (of all meshes of a group)
  const int32_t* succ_ptr;        // [G + 1]
  const int32_t* succ;            // (global tile << 1) | 1 when the successor is the next step's node
  int32_t* pending;               // [nsteps * G] unfinished dependencies of each node
  int32_t* queue;                 // [nsteps * G] node ids in publication order, -1 = not yet
  unsigned long long* head;       // next slot to take
  unsigned long long* tail;       // next slot to publish
  int32_t* err;                   // set when a wait gave up
  long long max_spins;
  int32_t g_lo, g_hi;             // nodes of this run: tiles g_lo .. g_hi - 1 (one sub-chain, or all)
  int32_t keep;                   // 1: a CTA runs one of the nodes its tile released next itself
};

// Queue slot value of a node that its releasing CTA kept: the slot is filled so that every slot
// is filled exactly once, and a CTA that takes it takes the next slot.
constexpr int32_t kSkipSlot = -2;
// one mesh: sub-chain table by value
struct DF {
  DFQ q;
  int32_t cum[17];                // global tile id base of each sub-chain (cum[k] + local id)
  int32_t first[16], last[16];    // loop range of each sub-chain
};
// a group of meshes of one degree: (mesh, sub-chain) table and per-mesh parameters in memory
struct DFM {
  DFQ q;
  int32_t K;                      // (mesh, sub-chain) entries
  const int32_t* cum;             // [K + 1] global tile id base of each entry
  const int32_t* first;           // [K] loop range of each entry
  const int32_t* last;
  const int32_t* mesh_of;         // [K] index into params
  const Params* params;           // per mesh of the group
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

__global__ void k_df_init(DFQ q, const int32_t* __restrict__ indeg0, const int32_t* __restrict__ indeg) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < q.total;
       i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % q.G);
    q.pending[i] = i < q.G ? indeg0[g] : indeg[g];
    q.queue[i] = -1;
  }
}
__global__ void k_df_seed(DFQ q, const int32_t* __restrict__ indeg0) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < q.G; g += gridDim.x * blockDim.x)
    if (indeg0[g] == 0) {
      unsigned long long j = atomicAdd(q.tail, 1ull);
      q.queue[j] = g;
    }
}

// Thread 0: claim the next slot and wait (bounded) until a node is published there; a slot of a
// kept node sends it to the next slot.  Returns the node, or -1 when the run is over or a wait
// gave up (the error flag is then set).
__device__ __forceinline__ long long df_take(const DFQ& q) {
  for (;;) {
    const unsigned long long slot = atomicAdd(q.head, 1ull);
    if ((long long)slot >= q.total || ld_acquire(q.err)) return -1;
    long long node;
    long long spins = 0;
    while ((node = ld_acquire(&q.queue[slot])) == -1) {
      if (++spins > q.max_spins || ld_acquire(q.err)) {
        atomicExch(q.err, 1);
        return -1;
      }
      __nanosleep(64);
    }
    if (node == kSkipSlot) continue;
    __threadfence();
    return node;
  }
}

// The first warp, after the CTA (or cluster) finished node (st, g) and passed a barrier: release
// its successors, one lane per successor (about ten per node), so that the decrements travel to L2
// side by side instead of one after another.  Each lane's fence and acq_rel decrement order the
// whole tile's writes, which the barrier made visible to it, before the successor can be taken.
// With q.keep, the first released successor is not queued: its slot gets kSkipSlot and the CTA
// runs it next (returned on every lane; -1 when none).  A released successor overlaps the tile
// just run, so its cells' data is still in L2 when it starts, where a node queued behind the
// rest of the ready nodes may find it evicted.  The releasing lane's acquire reaches the CTA's
// other threads through the barrier before the node's first load, as with df_take.
__device__ __forceinline__ long long df_publish(const DFQ& q, int g, long long st) {
  __threadfence();
  const int lane = (int)(threadIdx.x & 31);
  const int i0 = q.succ_ptr[g], i1 = q.succ_ptr[g + 1];
  long long kept = -1;
  for (int base = i0; base < i1; base += 32) {  // the same trip count on every lane
    const int i = base + lane;
    long long n2 = -1;
    if (i < i1) {
      const int e = q.succ[i];
      const long long s2 = st + (e & 1);
      if (s2 < q.nsteps && (e >> 1) >= q.g_lo && (e >> 1) < q.g_hi) {
        const long long c = s2 * q.G + (e >> 1);
        if (atom_add_acq_rel(&q.pending[c], -1) == 1) n2 = c;
      }
    }
    const unsigned rel = __ballot_sync(0xffffffffu, n2 >= 0);
    const int keeper = (q.keep && kept < 0 && rel) ? __ffs(rel) - 1 : -1;
    if (n2 >= 0) {
      const unsigned long long j = atomicAdd(q.tail, 1ull);
      st_release(&q.queue[j], lane == keeper ? kSkipSlot : (int32_t)n2);
    }
    if (keeper >= 0) kept = __shfl_sync(0xffffffffu, n2, keeper);
  }
  if (kept >= 0) __threadfence();
  return kept;
}

// One tile's slice of the segments of [first, last) at step st, segments separated by CTA
// barriers.  A segment with no item in this tile writes nothing, so it needs no barrier of its own
// (the condition is the same for every thread of the CTA); the last segment always ends with one.
template <int P, int BS, bool BATCH>
__device__ __forceinline__ void run_tile(const Params& a, int first, int last, int t, long long st) {
  for (int J = first; J < last; J = seg_end(J, last)) {
    const int32_t b = a.plan_ptr[J][t], e = a.plan_ptr[J][t + 1];
    if (b == e && seg_end(J, last) < last) continue;
    const int32_t* items = a.plan_items[J];
    const int H = phase_of(J);
    if constexpr (BATCH) {  // every item for each shot of the slice, consecutive threads on consecutive shots
      const int64_t nwork = (int64_t)(e - b) * a.sg;
      for (int64_t i = threadIdx.x; i < nwork; i += BS)
        run_seg<P, DF_L2_ONLY, true>(a, H, items[b + i / a.sg], st, a.s0 + (int)(i % a.sg));
    } else {
      for (int32_t i = b + threadIdx.x; i < e; i += BS) run_seg<P, DF_L2_ONLY, false>(a, H, items[i], st);
    }
    __syncthreads();
  }
}

template <int P, int BS, bool BATCH>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_dataflow(Params a, DF df) {
  __shared__ long long s_node;
  long long kept = -1;  // (thread 0's copy is the one used)
  for (;;) {
    if (threadIdx.x == 0) s_node = kept >= 0 ? kept : df_take(df.q);
    __syncthreads();
    const long long node = s_node;
    if (node < 0) return;
    const long long st = node / df.q.G;
    const int g = (int)(node % df.q.G);
    int k = 0;
    while (g >= df.cum[k + 1]) ++k;
    run_tile<P, BS, BATCH>(a, df.first[k], df.last[k], g - df.cum[k], st);
    if (threadIdx.x < 32) kept = df_publish(df.q, g, st);
  }
}

// The same executor over the tiles of several meshes of one degree: one queue, per-mesh
// dependency counters (the graphs are disjoint), each tile run with its mesh's parameters
// (copied to shared memory when the CTA takes the tile).
template <int P, int BS>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_dataflow_group(DFM df) {
  __shared__ long long s_node;
  __shared__ Params sp;
  static_assert(sizeof(Params) % 4 == 0, "Params is copied as 32-bit words");
  long long kept = -1;
  for (;;) {
    if (threadIdx.x == 0) s_node = kept >= 0 ? kept : df_take(df.q);
    __syncthreads();
    const long long node = s_node;
    if (node < 0) return;
    const long long st = node / df.q.G;
    const int g = (int)(node % df.q.G);
    int lo = 0, hi = df.K;  // entry k with cum[k] <= g < cum[k + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (df.cum[mid] <= g) lo = mid;
      else hi = mid;
    }
    const int k = lo;
    const int32_t* src = reinterpret_cast<const int32_t*>(&df.params[df.mesh_of[k]]);
    int32_t* dst = reinterpret_cast<int32_t*>(&sp);
    for (int i = threadIdx.x; i < (int)(sizeof(Params) / 4); i += BS) dst[i] = src[i];
    __syncthreads();
    run_tile<P, BS, false>(sp, df.first[k], df.last[k], g - df.cum[k], st);
    if (threadIdx.x < 32) kept = df_publish(df.q, g, st);
  }
}

// One queue over the tiles of meshes of several degrees, single-field or many-shot: the batched
// form as one persistent launch.  Each tile runs the phase bodies of its mesh's degree (Params.p)
// and layout (Params.S shots innermost when above 1, every shot of the tile's items in the tile);
// the kernel holds the bodies of degrees 1 to 3 and takes the registers of the largest.
template <int BS>
__global__ void __launch_bounds__(BS, 2) k_dataflow_mixed(DFM df) {
  __shared__ long long s_node;
  __shared__ Params sp;
  static_assert(sizeof(Params) % 4 == 0, "Params is copied as 32-bit words");
  long long kept = -1;
  for (;;) {
    if (threadIdx.x == 0) s_node = kept >= 0 ? kept : df_take(df.q);
    __syncthreads();
    const long long node = s_node;
    if (node < 0) return;
    const long long st = node / df.q.G;
    const int g = (int)(node % df.q.G);
    int lo = 0, hi = df.K;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (df.cum[mid] <= g) lo = mid;
      else hi = mid;
    }
    const int k = lo;
    const int32_t* src = reinterpret_cast<const int32_t*>(&df.params[df.mesh_of[k]]);
    int32_t* dst = reinterpret_cast<int32_t*>(&sp);
    for (int i = threadIdx.x; i < (int)(sizeof(Params) / 4); i += BS) dst[i] = src[i];
    __syncthreads();
    const int t = g - df.cum[k], f = df.first[k], l = df.last[k];
    switch (sp.p * 2 + (sp.S > 1 ? 1 : 0)) {
      case 2: run_tile<1, BS, false>(sp, f, l, t, st); break;
      case 3: run_tile<1, BS, true>(sp, f, l, t, st); break;
      case 4: run_tile<2, BS, false>(sp, f, l, t, st); break;
      case 5: run_tile<2, BS, true>(sp, f, l, t, st); break;
      case 6: run_tile<3, BS, false>(sp, f, l, t, st); break;
      default: run_tile<3, BS, true>(sp, f, l, t, st); break;
    }
    if (threadIdx.x < 32) kept = df_publish(df.q, g, st);
  }
}

// The same executor with one thread-block cluster per tile (large tiles, few boundary cells):
// the cluster's CTAs share each segment's items of the tile, separated by a cluster barrier.  The
// leader CTA's first thread takes nodes from the queue and publishes their successors; the node
// reaches the other CTAs through `slot[cluster]`, ordered by the barrier.  Every CTA of a cluster
// passes the same barriers and leaves together, so the barriers always complete.
template <int P, int BS>
__global__ void __launch_bounds__(BS, tile_min_blocks<P, BS>()) k_dataflow_cluster(Params a, DF df,
                                                                                  long long* __restrict__ slot) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const unsigned rank = cl.block_rank(), C = cl.num_blocks();
  const unsigned cid = blockIdx.x / C;
  long long kept = -1;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) slot[cid] = kept >= 0 ? kept : df_take(df.q);
    cl.sync();
    const long long node = *(volatile long long*)&slot[cid];
    if (node < 0) return;
    const long long st = node / df.q.G;
    const int g = (int)(node % df.q.G);
    int k = 0;
    while (g >= df.cum[k + 1]) ++k;
    const int t = g - df.cum[k];
    for (int J = df.first[k]; J < df.last[k]; J = seg_end(J, df.last[k])) {
      const int32_t b = a.plan_ptr[J][t], e = a.plan_ptr[J][t + 1];
      if (b == e && seg_end(J, df.last[k]) < df.last[k]) continue;  // empty slice: no writes to order
      const int32_t* items = a.plan_items[J];
      const int H = phase_of(J);
      for (int32_t i = b + (int32_t)(rank * BS + threadIdx.x); i < e; i += (int32_t)(C * BS))
        run_seg<P, DF_L2_ONLY, false>(a, H, items[i], st);
      cl.sync();
    }
    if (rank == 0 && threadIdx.x < 32) kept = df_publish(df.q, g, st);
  }
}

// Error flag of the schedule's last dataflow run (synchronises s): SLT_ERR_TIMEOUT if a wait
// gave up.
inline void dataflow_check(::slt_schedule_s* sched, cudaStream_t s) {
  int32_t herr = 0;
  SLT_CUDA(cudaMemcpyAsync(&herr, sched->df.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  if (herr) slt::fail(SLT_ERR_TIMEOUT, "a wait of the dataflow executor gave up");
}

// The queue state and sub-chain table of one run of the schedule's plan (plan pointers into `a`),
// the queue reset and seeded on s.  Returns false when there is nothing to run.  rec_begin(cls,
// launches) / rec_end() bracket the two set-up kernels (class 2) for the caller's timing.
template <class RB, class RE>
bool prepare_dataflow(::slt_schedule_s* sched, Params& a, int64_t nsteps, cudaStream_t s, DF& df, RB rec_begin,
                      RE rec_end) {
  slt::DataflowPlan& D = sched->df;
  df = DF{};
  DFQ& q = df.q;
  q.G = D.cum.back();
  q.nsteps = nsteps;
  q.total = (long long)nsteps * q.G;
  if (q.total == 0) return false;
  if (q.total >= (1ll << 31)) slt::fail(SLT_ERR_UNSUPPORTED, "steps x tiles must stay below 2^31");
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
  if (D.pending.n < (size_t)q.total) {
    D.pending.alloc(q.total);
    D.queue.alloc(q.total);
  }
  q.succ_ptr = D.succ_ptr.p;
  q.succ = D.succ.p;
  q.pending = D.pending.p;
  q.queue = D.queue.p;
  q.head = D.head.p;
  q.tail = D.head.p + 1;
  q.err = D.err.p;
  q.max_spins = sched->wait_spins;
  q.keep = sched->keep;
  q.g_lo = 0;
  q.g_hi = q.G;
  SLT_CUDA(cudaMemsetAsync(D.head.p, 0, 2 * sizeof(unsigned long long), s));
  SLT_CUDA(cudaMemsetAsync(D.err.p, 0, sizeof(int32_t), s));
  rec_begin(2, 2);
  k_df_init<<<(unsigned)std::min<long long>((q.total + 255) / 256, 152 * 16), 256, 0, s>>>(q, D.indeg0.p,
                                                                                          D.indeg.p);
  k_df_seed<<<(q.G + 255) / 256, 256, 0, s>>>(q, D.indeg0.p);
  rec_end();
  SLT_CUDA(cudaGetLastError());
  return true;
}

// One time step of sub-chain k alone (its tiles in colour order, nothing of the other sub-chains):
// the queue holds the sub-chain's tiles, each waiting only for the same-step dependencies inside
// the sub-chain.  Node ids are global tile ids at step 0.
__global__ void k_df_init_sub(DFQ q, const int32_t* __restrict__ indeg_sub) {
  const int32_t n = q.g_hi - q.g_lo;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    q.pending[q.g_lo + i] = indeg_sub[q.g_lo + i];
    q.queue[i] = -1;
  }
}
__global__ void k_df_seed_sub(DFQ q, const int32_t* __restrict__ indeg_sub) {
  for (int g = q.g_lo + blockIdx.x * blockDim.x + threadIdx.x; g < q.g_hi; g += gridDim.x * blockDim.x)
    if (indeg_sub[g] == 0) {
      unsigned long long j = atomicAdd(q.tail, 1ull);
      q.queue[j] = g;
    }
}
template <class RB, class RE>
bool prepare_dataflow_sub(::slt_schedule_s* sched, Params& a, int k, cudaStream_t s, DF& df, RB rec_begin,
                          RE rec_end) {
  slt::DataflowPlan& D = sched->df;
  df = DF{};
  DFQ& q = df.q;
  q.G = D.cum.back();
  q.nsteps = 1;
  q.g_lo = D.cum[k];
  q.g_hi = D.cum[k + 1];
  q.total = q.g_hi - q.g_lo;
  if (q.total == 0) return false;
  for (size_t j = 0; j < D.cum.size(); ++j) df.cum[j] = D.cum[j];
  for (size_t j = 0; j < sched->subs.size(); ++j) {
    const slt::SubSched& sub = sched->subs[j];
    df.first[j] = sub.first;
    df.last[j] = sub.last;
    for (int jj = sub.first; jj < sub.last; ++jj) {
      a.plan_ptr[jj] = sub.plan_ptr[jj - sub.first].p;
      a.plan_items[jj] = sub.plan_items[jj - sub.first].p;
    }
  }
  if (D.pending.n < (size_t)q.G) {
    D.pending.alloc(q.G);
    D.queue.alloc(q.G);
  }
  q.succ_ptr = D.succ_ptr.p;
  q.succ = D.succ.p;
  q.pending = D.pending.p;
  q.queue = D.queue.p;
  q.head = D.head.p;
  q.tail = D.head.p + 1;
  q.err = D.err.p;
  q.max_spins = sched->wait_spins;
  q.keep = sched->keep;
  SLT_CUDA(cudaMemsetAsync(D.head.p, 0, 2 * sizeof(unsigned long long), s));
  SLT_CUDA(cudaMemsetAsync(D.err.p, 0, sizeof(int32_t), s));
  rec_begin(2, 2);
  k_df_init_sub<<<(unsigned)std::min<long long>((q.total + 255) / 256, 152 * 16), 256, 0, s>>>(q, D.indeg_sub.p);
  k_df_seed_sub<<<(unsigned)((q.total + 255) / 256), 256, 0, s>>>(q, D.indeg_sub.p);
  rec_end();
  SLT_CUDA(cudaGetLastError());
  return true;
}

// Launch the dataflow executor for nsteps on the schedule's plan; `rec_begin(cls, launches)` /
// `rec_end()` bracket the set-up kernels (class 2) and the persistent kernel (class 0) for the
// caller's timing.  Synchronises; SLT_ERR_TIMEOUT when a wait gave up.
template <int P, bool BATCH, class RB, class RE>
void launch_dataflow(::slt_schedule_s* sched, Params a, int64_t nsteps, cudaStream_t s, RB rec_begin, RE rec_end,
                     int sub = -1) {
  DF df;
  if (sub >= 0 ? !prepare_dataflow_sub(sched, a, sub, s, df, rec_begin, rec_end)
               : !prepare_dataflow(sched, a, nsteps, s, df, rec_begin, rec_end))
    return;
  int dev = 0, nsm = 0, per = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int bs = sched->block;
  auto launch = [&](auto kernel, int threads) {
    SLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0));
    const long long grid = std::min<long long>((long long)nsm * std::max(per, 1), df.q.total);
    sched->df.last_grid = grid;
    rec_begin(0, 1);
    kernel<<<(unsigned)grid, threads, 0, s>>>(a, df);
  };
  if (bs == 128) launch(k_dataflow<P, 128, BATCH>, 128);
  else if (bs == 384) launch(k_dataflow<P, 384, BATCH>, 384);
  else if (bs == 512 || bs == 768) {
    if constexpr (BATCH) slt::fail(SLT_ERR_UNSUPPORTED, "the multi-shot dataflow executor takes 128-384 threads");
    else if (bs == 512) launch(k_dataflow<P, 512, false>, 512);
    else launch(k_dataflow<P, 768, false>, 768);
  }
  else launch(k_dataflow<P, 256, BATCH>, 256);
  rec_end();
  SLT_CUDA(cudaGetLastError());
  dataflow_check(sched, s);
}
