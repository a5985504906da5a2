// Sparse-tiling inspector on the GPU (Section 5.1: Algorithm 1 with Algorithms 2 and 3).
//
// Every step is a data-parallel kernel whose result does not depend on thread scheduling, so
// the integer output equals a sequential execution of the same rules:
//   partition   rank / ts, ranks from a stable radix sort of Hilbert keys (sort.cu)
//   adjacency   tile pairs through the seed map plus fake edges, sorted and de-duplicated
//   colouring   Jones-Plassmann rounds: a tile is coloured once all higher-priority neighbours
//               are; it takes the smallest colour none of them has (= greedy in priority order)
//   projection  one thread per element of the projected set walks its inverse-map row in
//               ascending (iteration, slot) order; strictly larger colour replaces; equal
//               colours of distinct tiles among the candidates are recorded as conflicts
//   tiling      one thread per iteration, descriptors and slots in order, strict maximum
//   lists       stable radix sort of iterations by tile
//   local maps  stable sorts of slots by (tile, target), de-duplicated per tile
// Conflict pairs (few) are de-duplicated on the host and become fake edges for the next round.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <set>
#include <utility>
#include <vector>

#include "internal.h"

namespace slt {

namespace {

inline int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}
#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_div(const int32_t* __restrict__ rank, int64_t n, int32_t ts, int32_t* __restrict__ sig) {
  GRID_STRIDE(e, n) sig[e] = rank[e] / ts;
}
__global__ void k_fill(int32_t* __restrict__ a, int64_t n, int32_t v) {
  GRID_STRIDE(e, n) a[e] = v;
}
__global__ void k_iota_u(uint32_t* __restrict__ a, int64_t n) {
  GRID_STRIDE(e, n) a[e] = (uint32_t)e;
}
__global__ void k_copy_i2u(const int32_t* __restrict__ a, int64_t n, uint32_t* __restrict__ b) {
  GRID_STRIDE(e, n) b[e] = (uint32_t)a[e];
}
// b[e] = src[idx[e] / div]
__global__ void k_gather_div(const int32_t* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n, int div,
                             uint32_t* __restrict__ b) {
  GRID_STRIDE(e, n) b[e] = (uint32_t)src[idx[e] / div];
}

// pairs of distinct slot tiles of every element of a map that targets the seed set
__global__ void k_pairs_target(const int32_t* __restrict__ map, int64_t nsrc, int a, const int32_t* __restrict__ sig0,
                               uint32_t m, uint32_t* __restrict__ pa, uint32_t* __restrict__ pb) {
  GRID_STRIDE(e, nsrc) {
    for (int x = 0; x < a; ++x)
      for (int y = 0; y < a; ++y) {
        uint32_t ta = (uint32_t)sig0[map[e * a + x]], tb = (uint32_t)sig0[map[e * a + y]];
        int64_t o = (e * a + x) * a + y;
        pa[o] = ta != tb ? ta : m;
        pb[o] = ta != tb ? tb : m;
      }
  }
}
// count deg^2 of every target element of a map leaving the seed set
__global__ void k_pairs_count(const int32_t* __restrict__ ioff, int64_t ntgt, int32_t* __restrict__ cnt) {
  GRID_STRIDE(e, ntgt) {
    int32_t d = ioff[e + 1] - ioff[e];
    cnt[e] = d * d;
  }
}
__global__ void k_pairs_source(const int32_t* __restrict__ ioff, const uint32_t* __restrict__ islot, int64_t ntgt,
                               int a, const int32_t* __restrict__ cntoff, const int32_t* __restrict__ sig0, uint32_t m,
                               uint32_t* __restrict__ pa, uint32_t* __restrict__ pb) {
  GRID_STRIDE(e, ntgt) {
    int32_t b = ioff[e], d = ioff[e + 1] - b;
    int64_t o = cntoff[e];
    for (int x = 0; x < d; ++x)
      for (int y = 0; y < d; ++y) {
        uint32_t ta = (uint32_t)sig0[islot[b + x] / a], tb = (uint32_t)sig0[islot[b + y] / a];
        pa[o] = ta != tb ? ta : m;
        pb[o] = ta != tb ? tb : m;
        ++o;
      }
  }
}
// first occurrence of each distinct (a, b) with a < m in a sequence sorted by (a, b)
__global__ void k_unique_flags(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, int64_t n, uint32_t m,
                               int32_t* __restrict__ flag) {
  GRID_STRIDE(p, n) flag[p] = (a[p] < m) && (p == 0 || a[p] != a[p - 1] || b[p] != b[p - 1]);
}
__global__ void k_compact2(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, const int32_t* __restrict__ flag,
                           const int32_t* __restrict__ pos, int64_t n, uint32_t* __restrict__ oa, int32_t* __restrict__ ob) {
  GRID_STRIDE(p, n) if (flag[p]) {
    oa[pos[p]] = a[p];
    ob[pos[p]] = (int32_t)b[p];
  }
}

__global__ void k_priorities(int32_t m, uint64_t seed, uint64_t* __restrict__ prio) {
  GRID_STRIDE(t, m) prio[t] = splitmix64((uint64_t)t ^ seed);
}
__global__ void k_jp_round(int32_t m, const int32_t* __restrict__ aoff, const int32_t* __restrict__ adj,
                           const uint64_t* __restrict__ prio, int32_t* col, int32_t* __restrict__ remaining) {
  GRID_STRIDE(t, m) {
    if (((volatile int32_t*)col)[t] >= 0) continue;
    const uint64_t pt = prio[t];
    bool ready = true;
    for (int32_t k = aoff[t]; k < aoff[t + 1] && ready; ++k) {
      int32_t u = adj[k];
      if (prio[u] > pt || (prio[u] == pt && u < t)) ready = ((volatile int32_t*)col)[u] >= 0;
    }
    if (!ready) {
      atomicAdd(remaining, 1);
      continue;
    }
    int32_t c = 0;
    for (;;) {
      bool used = false;
      for (int32_t k = aoff[t]; k < aoff[t + 1]; ++k) {
        int32_t u = adj[k];
        if ((prio[u] > pt || (prio[u] == pt && u < t)) && ((volatile int32_t*)col)[u] == c) { used = true; break; }
      }
      if (!used) break;
      ++c;
    }
    ((volatile int32_t*)col)[t] = c;
  }
}

__device__ __forceinline__ void push_conflict(int32_t x, int32_t y, int2* buf, int32_t* cnt, int32_t cap) {
  int32_t i = atomicAdd(cnt, 1);
  if (i < cap) buf[i] = make_int2(x < y ? x : y, x < y ? y : x);
}

// MAX projection (dir > 0, forward tiling) or MIN (dir < 0, backward tiling): does tile t
// strictly win over the current tile cur?
__device__ __forceinline__ bool wins(int dir, const int32_t* __restrict__ col, int32_t t, int32_t cur) {
  return dir > 0 ? col[t] > col[cur] : col[t] < col[cur];
}

__global__ void k_project_direct(int64_t n, const int32_t* __restrict__ sig, const int32_t* __restrict__ col,
                                 int32_t* __restrict__ phi, int2* cbuf, int32_t* ccnt, int32_t cap, int dir) {
  GRID_STRIDE(e, n) {
    int32_t old = phi[e], t = sig[e];
    if (old < 0 || wins(dir, col, t, old)) phi[e] = t;
    else if (t != old && col[t] == col[old]) push_conflict(old, t, cbuf, ccnt, cap);
  }
}
__global__ void k_project_indirect(int64_t n, const int32_t* __restrict__ ioff, const uint32_t* __restrict__ islot,
                                   int a, const int32_t* __restrict__ sig, const int32_t* __restrict__ col,
                                   int32_t* __restrict__ phi, int2* cbuf, int32_t* ccnt, int32_t cap, int dir) {
  GRID_STRIDE(e, n) {
    const int32_t b = ioff[e], d = ioff[e + 1] - b;
    const int32_t old = phi[e];
    int32_t cur = old;
    for (int k = 0; k < d; ++k) {
      int32_t t = sig[islot[b + k] / a];
      if (cur < 0 || wins(dir, col, t, cur)) cur = t;
    }
    phi[e] = cur;
    // conflicts: distinct same-colour tiles among {old} + touching iterations' tiles
    const int ncand = d + (old >= 0 ? 1 : 0);
    for (int x = 0; x < ncand; ++x) {
      int32_t tx = (old >= 0) ? (x == 0 ? old : sig[islot[b + x - 1] / a]) : sig[islot[b + x] / a];
      for (int y = x + 1; y < ncand; ++y) {
        int32_t ty = (old >= 0) ? (y == 0 ? old : sig[islot[b + y - 1] / a]) : sig[islot[b + y] / a];
        if (tx != ty && col[tx] == col[ty]) push_conflict(tx, ty, cbuf, ccnt, cap);
      }
    }
  }
}

constexpr int MAXD = 8;
struct TileDescs {
  int nd;
  const int32_t* map[MAXD];  // null for direct
  int arity[MAXD];
  const int32_t* phi[MAXD];  // projection of the target set (null: none yet)
};
__global__ void k_tile(int64_t n, TileDescs D, const int32_t* __restrict__ col, int32_t* __restrict__ sig,
                       int32_t* __restrict__ nbottom, int dir) {
  GRID_STRIDE(e, n) {
    int32_t cur = -1;
    for (int d = 0; d < D.nd; ++d) {
      const int32_t* p = D.phi[d];
      if (!p) continue;
      if (!D.map[d]) {
        int32_t t = p[e];
        if (t >= 0 && (cur < 0 || wins(dir, col, t, cur))) cur = t;
      } else {
        const int a = D.arity[d];
        for (int k = 0; k < a; ++k) {
          int32_t t = p[D.map[d][e * a + k]];
          if (t >= 0 && (cur < 0 || wins(dir, col, t, cur))) cur = t;
        }
      }
    }
    if (cur < 0) {
      cur = 0;
      atomicAdd(nbottom, 1);
    }
    sig[e] = cur;
  }
}

// local maps: p-th entry of the sequence sorted by (tile, target)
__global__ void k_lm_flags(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ slot,
                           const int32_t* __restrict__ map, int64_t n, int32_t* __restrict__ flag) {
  GRID_STRIDE(p, n) flag[p] = (p == 0 || tile[p] != tile[p - 1] || map[slot[p]] != map[slot[p - 1]]);
}
__global__ void k_lm_emit(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ slot,
                          const int32_t* __restrict__ map, const int32_t* __restrict__ flag,
                          const int32_t* __restrict__ pos, int64_t n, int32_t* __restrict__ fp,
                          uint32_t* __restrict__ utile) {
  GRID_STRIDE(p, n) if (flag[p]) {
    fp[pos[p]] = map[slot[p]];
    utile[pos[p]] = tile[p];
  }
}
__global__ void k_lm_local(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ slot,
                           const int32_t* __restrict__ pos, const int32_t* __restrict__ fp_ptr, int64_t n,
                           int32_t* __restrict__ lmap) {
  GRID_STRIDE(p, n) lmap[slot[p]] = pos[p + 1] - 1 - fp_ptr[tile[p]];
}

// executor plan of a facet loop: entries (tile, work id, face bit), sorted, OR-reduced per cell
// segment plan entries: one per (iteration, cell it writes) of a cell loop (its part bit) ...
__global__ void k_seg_cells(const int32_t* __restrict__ sig, const int32_t* __restrict__ iperm, int64_t n,
                            uint32_t bit, uint32_t* __restrict__ tile, uint32_t* __restrict__ wid,
                            uint32_t* __restrict__ bits) {
  GRID_STRIDE(p, n) {
    tile[p] = (uint32_t)sig[p];
    wid[p] = (uint32_t)iperm[p];
    bits[p] = bit;
  }
}
// ... and of a facet loop: slot p = facet * a + side, the face bit of that side's cell
__global__ void k_seg_facets(const int32_t* __restrict__ map, const int8_t* __restrict__ face, int64_t ns, int a,
                             const int32_t* __restrict__ sig, const int32_t* __restrict__ iperm,
                             uint32_t* __restrict__ tile, uint32_t* __restrict__ wid, uint32_t* __restrict__ bits) {
  GRID_STRIDE(p, ns) {
    tile[p] = (uint32_t)sig[p / a];
    wid[p] = (uint32_t)iperm[map[p]];
    bits[p] = 1u << face[p];
  }
}
// first entry of each run of equal (tile, work id) in sorted order
__global__ void k_run_heads(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ wid, int64_t n,
                                   int32_t* __restrict__ flag) {
  GRID_STRIDE(p, n) flag[p] = (p == 0 || tile[p] != tile[p - 1] || wid[p] != wid[p - 1]);
}
// one item per run: the work id and the union of the run's bits
__global__ void k_seg_emit(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ wid,
                           const uint32_t* __restrict__ bits, const int32_t* __restrict__ flag,
                           const int32_t* __restrict__ pos, int64_t n, int32_t* __restrict__ items,
                           uint32_t* __restrict__ utile) {
  GRID_STRIDE(p, n) if (flag[p]) {
    uint32_t b = 0;
    for (int64_t q = p; q < n && tile[q] == tile[p] && wid[q] == wid[p]; ++q) b |= bits[q];
    items[pos[p]] = (int32_t)((wid[p] << 5) | b);
    utile[pos[p]] = tile[p];
  }
}
// sort key of an item inside its tile: full flags (both cell loops and three faces) first
__global__ void k_flag_key(const int32_t* __restrict__ items, int64_t n, uint32_t* __restrict__ key) {
  GRID_STRIDE(p, n) key[p] = 31u - (uint32_t)(items[p] & 31);
}

struct InverseMap {
  DevBuf<int32_t> off;   // [ntgt + 1]
  DevBuf<uint32_t> slot; // [nsrc * arity], slots sorted by target (stable)
};

void build_inverse(const int32_t* d_map, int64_t nslot, int64_t ntgt, InverseMap& inv, cudaStream_t s) {
  DevBuf<uint32_t> k(nslot), tk(nslot), tv(nslot);
  inv.slot.alloc(nslot);
  inv.off.alloc(ntgt + 1);
  if (nslot) {
    k_copy_i2u<<<grid_for(nslot), 256, 0, s>>>(d_map, nslot, k.p);
    k_iota_u<<<grid_for(nslot), 256, 0, s>>>(inv.slot.p, nslot);
    radix_sort_pairs(k.p, inv.slot.p, nslot, bits_for(std::max<int64_t>(ntgt - 1, 1)), tk.p, tv.p, s);
  }
  lower_bound_offsets(k.p, nslot, ntgt, inv.off.p, s);
  SLT_CUDA(cudaStreamSynchronize(s));
}

// stable sort of n values by two keys: primary k1 (bits1), secondary k2 (bits2); returns the
// permutation (positions into the original sequence) and the sorted primary keys.
void sort_by_two(DevBuf<uint32_t>& k1, int bits1, DevBuf<uint32_t>& k2, int bits2, int64_t n, DevBuf<uint32_t>& order,
                 cudaStream_t s) {
  DevBuf<uint32_t> tk(n), tv(n), key(n);
  order.alloc(n);
  k_iota_u<<<grid_for(n), 256, 0, s>>>(order.p, n);
  SLT_CUDA(cudaMemcpyAsync(key.p, k2.p, n * 4, cudaMemcpyDeviceToDevice, s));
  radix_sort_pairs(key.p, order.p, n, bits2, tk.p, tv.p, s);
  // gather primary keys in the secondary order, then stable sort by them
  k_gather_div<<<grid_for(n), 256, 0, s>>>((const int32_t*)k1.p, order.p, n, 1, key.p);
  radix_sort_pairs(key.p, order.p, n, bits1, tk.p, tv.p, s);
  SLT_CUDA(cudaMemcpyAsync(k1.p, key.p, n * 4, cudaMemcpyDeviceToDevice, s));
  SLT_CUDA(cudaStreamSynchronize(s));
}

struct Ctx {
  slt_chain c;
  const slt_options* opt;
  cudaStream_t s;
  std::vector<DevBuf<int32_t>> dmaps;  // device copies of maps
  std::map<int, InverseMap> inverses;
};

const InverseMap& inverse_of(Ctx& X, int mid) {
  auto it = X.inverses.find(mid);
  if (it != X.inverses.end()) return it->second;
  const MapH& M = X.c->maps[mid];
  InverseMap& inv = X.inverses[mid];
  build_inverse(X.dmaps[mid].p, (int64_t)M.values.size(), X.c->set_size[M.to], inv, X.s);
  return inv;
}

// adjacency CSR (aoff [m+1], adj) from the seed map and fake edges
void build_adjacency(Ctx& X, int first, int last, int seed_set, const int32_t* sig0, int32_t m,
                     const std::vector<std::pair<int32_t, int32_t>>& fake, DevBuf<int32_t>& aoff, DevBuf<int32_t>& adj) {
  cudaStream_t s = X.s;
  slt_chain c = X.c;
  int mid = -1;
  bool target_kind = false;
  for (int j = first; j < last && mid < 0; ++j)
    for (const DescH& d : c->loops[j].descs) {
      if (d.map < 0) continue;
      const MapH& M = c->maps[d.map];
      if (M.to == seed_set) { mid = d.map; target_kind = true; break; }
      if (M.from == seed_set) { mid = d.map; target_kind = false; break; }
    }
  int64_t nmap = 0;
  DevBuf<int32_t> cntoff;
  if (mid >= 0) {
    const MapH& M = c->maps[mid];
    if (target_kind) {
      nmap = c->set_size[M.from] * (int64_t)M.arity * M.arity;
    } else {
      const InverseMap& inv = inverse_of(X, mid);
      int64_t nt = c->set_size[M.to];
      DevBuf<int32_t> cnt(nt);
      cntoff.alloc(nt + 1);
      k_pairs_count<<<grid_for(nt), 256, 0, s>>>(inv.off.p, nt, cnt.p);
      exclusive_scan_i32(cnt.p, cntoff.p, nt, s);
      int32_t total = 0;
      SLT_CUDA(cudaMemcpyAsync(&total, cntoff.p + nt, 4, cudaMemcpyDeviceToHost, s));
      SLT_CUDA(cudaStreamSynchronize(s));
      nmap = total;
    }
  }
  int64_t n = nmap + 2 * (int64_t)fake.size();
  DevBuf<uint32_t> pa(std::max<int64_t>(n, 1)), pb(std::max<int64_t>(n, 1));
  if (mid >= 0 && nmap > 0) {
    const MapH& M = c->maps[mid];
    if (target_kind)
      k_pairs_target<<<grid_for(c->set_size[M.from]), 256, 0, s>>>(X.dmaps[mid].p, c->set_size[M.from], M.arity, sig0,
                                                                   (uint32_t)m, pa.p, pb.p);
    else {
      const InverseMap& inv = inverse_of(X, mid);
      k_pairs_source<<<grid_for(c->set_size[M.to]), 256, 0, s>>>(inv.off.p, inv.slot.p, c->set_size[M.to], M.arity,
                                                                 cntoff.p, sig0, (uint32_t)m, pa.p, pb.p);
    }
    SLT_CUDA(cudaGetLastError());
  }
  if (!fake.empty()) {
    std::vector<uint32_t> ha, hb;
    for (auto& e : fake) {
      ha.push_back(e.first); hb.push_back(e.second);
      ha.push_back(e.second); hb.push_back(e.first);
    }
    SLT_CUDA(cudaMemcpyAsync(pa.p + nmap, ha.data(), ha.size() * 4, cudaMemcpyHostToDevice, s));
    SLT_CUDA(cudaMemcpyAsync(pb.p + nmap, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice, s));
  }
  aoff.alloc(m + 1);
  if (n == 0) {
    k_fill<<<grid_for(m + 1), 256, 0, s>>>(aoff.p, m + 1, 0);
    adj.alloc(1);
    SLT_CUDA(cudaStreamSynchronize(s));
    return;
  }
  // sort by (a, b): stable by b, then stable by a
  int bits = bits_for(m);
  DevBuf<uint32_t> order;
  sort_by_two(pa, bits, pb, bits, n, order, s);
  DevBuf<uint32_t> sb(n);
  k_gather_div<<<grid_for(n), 256, 0, s>>>((const int32_t*)pb.p, order.p, n, 1, sb.p);
  DevBuf<int32_t> flag(n), pos(n + 1);
  k_unique_flags<<<grid_for(n), 256, 0, s>>>(pa.p, sb.p, n, (uint32_t)m, flag.p);
  exclusive_scan_i32(flag.p, pos.p, n, s);
  int32_t nu = 0;
  SLT_CUDA(cudaMemcpyAsync(&nu, pos.p + n, 4, cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  DevBuf<uint32_t> ua(std::max(nu, 1));
  adj.alloc(std::max(nu, 1));
  k_compact2<<<grid_for(n), 256, 0, s>>>(pa.p, sb.p, flag.p, pos.p, n, ua.p, adj.p);
  lower_bound_offsets(ua.p, nu, m, aoff.p, s);
  SLT_CUDA(cudaStreamSynchronize(s));
}

void colour_tiles(Ctx& X, int32_t m, bool sequential, const DevBuf<int32_t>& aoff, const DevBuf<int32_t>& adj,
                  DevBuf<int32_t>& col) {
  cudaStream_t s = X.s;
  if (sequential) {
    DevBuf<uint32_t> tmp(m);
    k_iota_u<<<grid_for(m), 256, 0, s>>>(tmp.p, m);
    SLT_CUDA(cudaMemcpyAsync(col.p, tmp.p, m * 4, cudaMemcpyDeviceToDevice, s));
    SLT_CUDA(cudaStreamSynchronize(s));
    return;
  }
  DevBuf<uint64_t> prio(m);
  DevBuf<int32_t> remaining(1);
  k_priorities<<<grid_for(m), 256, 0, s>>>(m, X.opt->prio_seed, prio.p);
  k_fill<<<grid_for(m), 256, 0, s>>>(col.p, m, -1);
  for (int64_t round = 0;; ++round) {
    if (round > m + 1) fail(SLT_ERR_CUDA, "colouring did not converge");
    SLT_CUDA(cudaMemsetAsync(remaining.p, 0, 4, s));
    k_jp_round<<<grid_for(m), 256, 0, s>>>(m, aoff.p, adj.p, prio.p, col.p, remaining.p);
    SLT_CUDA(cudaGetLastError());
    int32_t left = 0;
    SLT_CUDA(cudaMemcpyAsync(&left, remaining.p, 4, cudaMemcpyDeviceToHost, s));
    SLT_CUDA(cudaStreamSynchronize(s));
    if (left == 0) break;
  }
}

void export_lists(Ctx& X, const int32_t* sig, int64_t n, int32_t m, DevBuf<int32_t>& ptr, DevBuf<int32_t>& list) {
  cudaStream_t s = X.s;
  ptr.alloc(m + 1);
  list.alloc(std::max<int64_t>(n, 1));
  DevBuf<uint32_t> k(std::max<int64_t>(n, 1)), v(std::max<int64_t>(n, 1)), tk(std::max<int64_t>(n, 1)),
      tv(std::max<int64_t>(n, 1));
  if (n) {
    k_copy_i2u<<<grid_for(n), 256, 0, s>>>(sig, n, k.p);
    k_iota_u<<<grid_for(n), 256, 0, s>>>(v.p, n);
    radix_sort_pairs(k.p, v.p, n, bits_for(std::max(m - 1, 1)), tk.p, tv.p, s);
    SLT_CUDA(cudaMemcpyAsync(list.p, v.p, n * 4, cudaMemcpyDeviceToDevice, s));
  }
  lower_bound_offsets(k.p, n, m, ptr.p, s);
  SLT_CUDA(cudaStreamSynchronize(s));
}

void build_local_map(const int32_t* dmap, int a, int64_t ntgt, const int32_t* sig, int64_t n, int32_t m,
                     LocalMap& L, cudaStream_t s) {
  const int64_t ns = n * a;
  L.fp_ptr.alloc(m + 1);
  L.lmap.alloc(std::max<int64_t>(ns, 1));
  if (ns == 0) {
    k_fill<<<grid_for(m + 1), 256, 0, s>>>(L.fp_ptr.p, m + 1, 0);
    L.fp.alloc(1);
    SLT_CUDA(cudaStreamSynchronize(s));
    return;
  }
  DevBuf<uint32_t> tile(ns), tgt(ns), order, slots(ns);
  k_iota_u<<<grid_for(ns), 256, 0, s>>>(slots.p, ns);
  k_gather_div<<<grid_for(ns), 256, 0, s>>>(sig, slots.p, ns, a, tile.p);
  k_copy_i2u<<<grid_for(ns), 256, 0, s>>>(dmap, ns, tgt.p);
  sort_by_two(tile, bits_for(std::max(m - 1, 1)), tgt, bits_for(std::max<int64_t>(ntgt - 1, 1)), ns, order, s);
  DevBuf<int32_t> flag(ns), pos(ns + 1);
  k_lm_flags<<<grid_for(ns), 256, 0, s>>>(tile.p, order.p, dmap, ns, flag.p);
  exclusive_scan_i32(flag.p, pos.p, ns, s);
  int32_t nu = 0;
  SLT_CUDA(cudaMemcpyAsync(&nu, pos.p + ns, 4, cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  L.fp.alloc(std::max(nu, 1));
  DevBuf<uint32_t> utile(std::max(nu, 1));
  k_lm_emit<<<grid_for(ns), 256, 0, s>>>(tile.p, order.p, dmap, flag.p, pos.p, ns, L.fp.p, utile.p);
  lower_bound_offsets(utile.p, nu, m, L.fp_ptr.p, s);
  // lmap[slot] = (inclusive count of uniques up to p) - 1 - fp_ptr[tile]
  DevBuf<int32_t> incl(ns + 1);
  SLT_CUDA(cudaMemcpyAsync(incl.p, pos.p + 1, ns * 4, cudaMemcpyDeviceToDevice, s));
  // pos[p+1] is the inclusive count at p; k_lm_local reads pos[p + 1]
  k_lm_local<<<grid_for(ns), 256, 0, s>>>(tile.p, order.p, pos.p, L.fp_ptr.p, ns, L.lmap.p);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void build_plan(slt_schedule sched, slt_mesh mesh, SubSched& sub, cudaStream_t s) {
  const int32_t m = sub.m;
  // tiles grouped by colour (stable: ascending tile id within a colour)
  {
    DevBuf<uint32_t> k(m), v(m), tk(m), tv(m);
    k_copy_i2u<<<grid_for(m), 256, 0, s>>>(sub.colour.p, m, k.p);
    k_iota_u<<<grid_for(m), 256, 0, s>>>(v.p, m);
    radix_sort_pairs(k.p, v.p, m, bits_for(std::max(sub.ncolours - 1, 1)), tk.p, tv.p, s);
    sub.tiles_by_colour.alloc(m);
    SLT_CUDA(cudaMemcpyAsync(sub.tiles_by_colour.p, v.p, m * 4, cudaMemcpyDeviceToDevice, s));
    DevBuf<int32_t> cp(sub.ncolours + 1);
    lower_bound_offsets(k.p, m, sub.ncolours, cp.p, s);
    sub.colour_ptr = cp.download(s);
  }
  DevBuf<int32_t> d_iperm(mesh->nc);
  d_iperm.upload(mesh->iperm.data(), mesh->nc, s);
  DevBuf<int32_t> d_f2c(std::max<int64_t>(mesh->nfi * 2, 1)), d_e2c(std::max<int64_t>(mesh->nfe, 1));
  DevBuf<int8_t> d_f2f(std::max<int64_t>(mesh->nfi * 2, 1)), d_e2f(std::max<int64_t>(mesh->nfe, 1));
  d_f2c.upload(mesh->f2c.data(), mesh->nfi * 2, s);
  d_e2c.upload(mesh->e2c.data(), mesh->nfe, s);
  d_f2f.upload(mesh->f2f.data(), mesh->nfi * 2, s);
  d_e2f.upload(mesh->e2f.data(), mesh->nfe, s);
  const int nl = sub.last - sub.first;
  sub.plan_ptr.clear();
  sub.plan_items.clear();
  sub.plan_ptr.resize(nl);
  sub.plan_items.resize(nl);
  if (mesh->nc >= (int64_t(1) << 26)) fail(SLT_ERR_UNSUPPORTED, "the tiled executors take below 2^26 cells");
  const int tbits = bits_for(std::max(m - 1, 1)), wbits = bits_for(std::max<int64_t>(mesh->nc - 1, 1));
  // one plan per segment (the part of a phase inside the sub-chain), stored at its first loop:
  // per tile, one item per cell the segment's loops touch,
  // (work id << 5) | (later cell loop << 4) | (first cell loop << 3) | faces
  for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last)) {
    const int J1 = seg_end(J0, sub.last);
    int64_t n = 0;
    for (int J = J0; J < J1; ++J) {
      const int set = sched->loops[J].set;
      n += set == 0 ? mesh->nc : set == 1 ? 2 * mesh->nfi : mesh->nfe;
    }
    const int jj = J0 - sub.first;
    sub.plan_ptr[jj].alloc(m + 1);
    if (n == 0) {
      k_fill<<<grid_for(m + 1), 256, 0, s>>>(sub.plan_ptr[jj].p, m + 1, 0);
      sub.plan_items[jj].alloc(1);
      continue;
    }
    // entries (tile, work id, bits) of every iteration of the segment's loops and cell it writes
    DevBuf<uint32_t> tile(n), wid(n), bits(n), order;
    int64_t o = 0;
    for (int J = J0; J < J1; ++J) {
      const int set = sched->loops[J].set;
      const int32_t* sig = sub.sigma[J - sub.first].p;
      if (set == 0) {
        const uint32_t bit = J == phase_first(phase_of(J)) ? 8u : 16u;
        k_seg_cells<<<grid_for(mesh->nc), 256, 0, s>>>(sig, d_iperm.p, mesh->nc, bit, tile.p + o, wid.p + o,
                                                         bits.p + o);
        o += mesh->nc;
      } else {
        const bool interior = set == 1;
        const int a = interior ? 2 : 1;
        const int64_t ns = (interior ? mesh->nfi : mesh->nfe) * a;
        if (ns == 0) continue;
        k_seg_facets<<<grid_for(ns), 256, 0, s>>>(interior ? d_f2c.p : d_e2c.p, interior ? d_f2f.p : d_e2f.p, ns, a,
                                                  sig, d_iperm.p, tile.p + o, wid.p + o, bits.p + o);
        o += ns;
      }
    }
    SLT_CUDA(cudaGetLastError());
    sort_by_two(tile, tbits, wid, wbits, n, order, s);  // tile sorted in place, order the permutation
    DevBuf<uint32_t> swid(n), sbits(n);
    k_gather_div<<<grid_for(n), 256, 0, s>>>((const int32_t*)wid.p, order.p, n, 1, swid.p);
    k_gather_div<<<grid_for(n), 256, 0, s>>>((const int32_t*)bits.p, order.p, n, 1, sbits.p);
    DevBuf<int32_t> flag(n), pos(n + 1);
    k_run_heads<<<grid_for(n), 256, 0, s>>>(tile.p, swid.p, n, flag.p);
    exclusive_scan_i32(flag.p, pos.p, n, s);
    int32_t nu = 0;
    SLT_CUDA(cudaMemcpyAsync(&nu, pos.p + n, 4, cudaMemcpyDeviceToHost, s));
    SLT_CUDA(cudaStreamSynchronize(s));
    DevBuf<int32_t> items(std::max(nu, 1));
    DevBuf<uint32_t> utile(std::max(nu, 1));
    k_seg_emit<<<grid_for(n), 256, 0, s>>>(tile.p, swid.p, sbits.p, flag.p, pos.p, n, items.p, utile.p);
    // inside each tile, items with the same flags side by side (stable, so work-id order within
    // equal flags), full ones first: a warp then runs only the parts its lanes have
    {
      DevBuf<uint32_t> mk(std::max(nu, 1)), ut(std::max(nu, 1)), ord;
      k_flag_key<<<grid_for(nu), 256, 0, s>>>(items.p, nu, mk.p);
      SLT_CUDA(cudaMemcpyAsync(ut.p, utile.p, (size_t)nu * 4, cudaMemcpyDeviceToDevice, s));
      sort_by_two(ut, tbits, mk, 5, nu, ord, s);
      sub.plan_items[jj].alloc(std::max(nu, 1));
      k_gather_div<<<grid_for(nu), 256, 0, s>>>(items.p, ord.p, nu, 1, (uint32_t*)sub.plan_items[jj].p);
    }
    lower_bound_offsets(utile.p, nu, m, sub.plan_ptr[jj].p, s);
    SLT_CUDA(cudaGetLastError());
    SLT_CUDA(cudaStreamSynchronize(s));
  }
}

void inspect_chain(slt_chain c, const slt_options& opt, cudaStream_t s, slt_schedule out) {
  // wall time of each stage (the stages end with a stream synchronisation)
  auto now = [] { return std::chrono::steady_clock::now(); };
  auto lap = [&](std::chrono::steady_clock::time_point& t0, int k) {
    SLT_CUDA(cudaStreamSynchronize(s));
    const auto t1 = now();
    out->insp_s[k] += std::chrono::duration<double>(t1 - t0).count();
    t0 = t1;
  };
  auto t0 = now();
  Ctx X{c, &opt, s, {}, {}};
  X.dmaps.resize(c->maps.size());
  for (size_t k = 0; k < c->maps.size(); ++k) {
    X.dmaps[k].alloc(std::max<size_t>(c->maps[k].values.size(), 1));
    X.dmaps[k].upload(c->maps[k].values.data(), c->maps[k].values.size(), s);
  }
  std::vector<int> bounds = {0};
  for (int k = 0; k < opt.nsplit; ++k) bounds.push_back(opt.split[k]);
  bounds.push_back((int)c->loops.size());
  const int nsets = (int)c->set_size.size();
  const int32_t cap = 1 << 22;
  DevBuf<int2> cbuf(cap);
  DevBuf<int32_t> ccnt(1), nbottom(1);

  for (size_t sc = 0; sc + 1 < bounds.size(); ++sc) {
    out->subs.emplace_back();
    SubSched& sub = out->subs.back();
    sub.first = bounds[sc];
    sub.last = bounds[sc + 1];
    const int nl = sub.last - sub.first;
    const int sl = opt.seed_loop[sc];  // seed loop, relative to the sub-chain's first loop
    sub.seed = sl;
    const int seed_set = c->loops[sub.first + sl].set;
    const int64_t nseed = c->set_size[seed_set];
    const int32_t ts = opt.sub_tile_size[sc] > 0 ? opt.sub_tile_size[sc] : opt.tile_size;
    const int32_t m = (int32_t)std::max<int64_t>((nseed + ts - 1) / ts, 1);
    sub.m = m;
    sub.rank.alloc(std::max<int64_t>(nseed, 1));
    {
      DevBuf<double> xy;
      if (opt.renumber) {
        xy.alloc(std::max<int64_t>(2 * nseed, 1));
        xy.upload(c->points[seed_set].data(), 2 * nseed, s);
      }
      seed_rank(xy.p, nseed, opt.renumber, sub.rank.p, s);
    }
    lap(t0, 0);
    sub.sigma.resize(nl);
    for (int jj = 0; jj < nl; ++jj) sub.sigma[jj].alloc(std::max<int64_t>(c->set_size[c->loops[sub.first + jj].set], 1));
    k_div<<<grid_for(nseed), 256, 0, s>>>(sub.rank.p, nseed, ts, sub.sigma[sl].p);
    SLT_CUDA(cudaGetLastError());
    sub.colour.alloc(m);
    std::vector<DevBuf<int32_t>> phi(nsets);
    std::vector<bool> has_phi(nsets);
    std::vector<std::pair<int32_t, int32_t>> fake;
    bool fell_back = false;
    for (;;) {
      DevBuf<int32_t> aoff, adj;
      build_adjacency(X, sub.first, sub.last, seed_set, sub.sigma[sl].p, m, fake, aoff, adj);
      colour_tiles(X, m, opt.colouring == 1 || fell_back, aoff, adj, sub.colour);
      for (int k = 0; k < nsets; ++k) has_phi[k] = false;
      SLT_CUDA(cudaMemsetAsync(ccnt.p, 0, 4, s));
      SLT_CUDA(cudaMemsetAsync(nbottom.p, 0, 4, s));
      auto project = [&](int jj, int dir) {
        const LoopH& L = c->loops[sub.first + jj];
        for (const DescH& d : L.descs) {
          int S = d.map < 0 ? L.set : c->maps[d.map].to;
          int64_t n = c->set_size[S];
          if (!has_phi[S]) {
            if (phi[S].n < (size_t)std::max<int64_t>(n, 1)) phi[S].alloc(std::max<int64_t>(n, 1));
            k_fill<<<grid_for(n), 256, 0, s>>>(phi[S].p, n, -1);
            has_phi[S] = true;
          }
          if (n == 0) continue;
          if (d.map < 0) {
            k_project_direct<<<grid_for(n), 256, 0, s>>>(n, sub.sigma[jj].p, sub.colour.p, phi[S].p, cbuf.p, ccnt.p, cap,
                                                        dir);
          } else {
            const InverseMap& inv = inverse_of(X, d.map);
            k_project_indirect<<<grid_for(n), 256, 0, s>>>(n, inv.off.p, inv.slot.p, c->maps[d.map].arity,
                                                          sub.sigma[jj].p, sub.colour.p, phi[S].p, cbuf.p, ccnt.p, cap,
                                                          dir);
          }
          SLT_CUDA(cudaGetLastError());
        }
      };
      auto tile = [&](int jj, int dir) {
        const LoopH& L = c->loops[sub.first + jj];
        TileDescs D{};
        D.nd = (int)L.descs.size();
        if (D.nd > MAXD) fail(SLT_ERR_UNSUPPORTED, "more than 8 descriptors in a loop");
        for (int d = 0; d < D.nd; ++d) {
          const DescH& ds = L.descs[d];
          int S = ds.map < 0 ? L.set : c->maps[ds.map].to;
          D.map[d] = ds.map < 0 ? nullptr : X.dmaps[ds.map].p;
          D.arity[d] = ds.map < 0 ? 1 : c->maps[ds.map].arity;
          D.phi[d] = has_phi[S] ? phi[S].p : nullptr;
        }
        int64_t n = c->set_size[L.set];
        if (n) k_tile<<<grid_for(n), 256, 0, s>>>(n, D, sub.colour.p, sub.sigma[jj].p, nbottom.p, dir);
        SLT_CUDA(cudaGetLastError());
      };
      if (sl > 0) {  // backward tiling: MIN from the seed loop towards the first loop
        project(sl, -1);
        for (int jj = sl - 1; jj >= 0; --jj) {
          tile(jj, -1);
          project(jj, -1);
        }
        for (int k = 0; k < nsets; ++k) has_phi[k] = false;
      }
      // forward tiling: MAX over the loops up to the seed, then the loops after it
      for (int jj = 0; jj <= sl; ++jj) project(jj, 1);
      for (int jj = sl + 1; jj < nl; ++jj) {
        tile(jj, 1);
        project(jj, 1);
      }
      int32_t nconf = 0, nbot = 0;
      SLT_CUDA(cudaMemcpyAsync(&nconf, ccnt.p, 4, cudaMemcpyDeviceToHost, s));
      SLT_CUDA(cudaMemcpyAsync(&nbot, nbottom.p, 4, cudaMemcpyDeviceToHost, s));
      SLT_CUDA(cudaStreamSynchronize(s));
      sub.unprojected = nbot;
      if (nconf > cap) fail(SLT_ERR_CONFLICT_CAP, "conflict buffer overflow");
      if (nconf == 0) break;
      std::vector<int2> h(nconf);
      SLT_CUDA(cudaMemcpyAsync(h.data(), cbuf.p, nconf * sizeof(int2), cudaMemcpyDeviceToHost, s));
      SLT_CUDA(cudaStreamSynchronize(s));
      std::set<std::pair<int32_t, int32_t>> pairs;
      for (const int2& p : h) pairs.insert({p.x, p.y});
      sub.conflicts = (int64_t)pairs.size();
      std::set<std::pair<int32_t, int32_t>> all(fake.begin(), fake.end());
      all.insert(pairs.begin(), pairs.end());
      fake.assign(all.begin(), all.end());
      ++sub.restarts;
      // sequential colouring after max_rounds restarts, or once the fake edges exceed 16 per
      // tile (scattered tiles would make every further round denser and slower)
      if ((opt.max_rounds >= 0 && sub.restarts > opt.max_rounds) || (int64_t)fake.size() > 16 * (int64_t)m)
        fell_back = true;
    }
    sub.fell_back = fell_back;
    lap(t0, 1);
    {
      std::vector<int32_t> hc = sub.colour.download(s, m);
      int32_t nc = 0;
      for (int32_t v : hc) nc = std::max(nc, v + 1);
      sub.ncolours = nc;
    }
    // assign: iteration lists (compute_local_maps runs when a local map is first asked for:
    // no executor reads them, and they cost a sort per indirect descriptor)
    sub.list_ptr.resize(nl);
    sub.list.resize(nl);
    sub.lmaps.resize(nl);
    for (int jj = 0; jj < nl; ++jj) {
      const LoopH& L = c->loops[sub.first + jj];
      int64_t n = c->set_size[L.set];
      export_lists(X, sub.sigma[jj].p, n, m, sub.list_ptr[jj], sub.list[jj]);
      sub.lmaps[jj].resize(L.descs.size());
    }
    lap(t0, 2);
    if (c->mesh) build_plan(out, c->mesh, sub, s);
    lap(t0, 3);
    if (c->mesh && out->executor == 4) stage_build(out, c->mesh, sub, s);  // its pass lists
    if (c->mesh && out->executor == 3) {
      stage_build(out, c->mesh, sub, s);
      const int32_t cap = stage_capacity(c->mesh->p);
      if (sub.max_fp > cap)
        fail(SLT_ERR_UNSUPPORTED, "staged executor: a tile touches " + std::to_string(sub.max_fp) +
                                      " cells, more than the " + std::to_string(cap) +
                                      " its shared memory holds at this degree; use a smaller tile size");
    }
    lap(t0, 4);
  }
  if (c->mesh) build_dataflow(out, c->mesh, s);
  lap(t0, 5);
  out->dmaps = std::move(X.dmaps);  // the local maps are built from them on request
}

// compute_local_maps for loop jj of sub-chain S (each indirect descriptor not built yet)
void ensure_local_maps(slt_schedule sched, SubSched& S, int jj, cudaStream_t s) {
  const LoopH& L = sched->loops[S.first + jj];
  const int64_t n = sched->set_size[L.set];
  for (size_t d = 0; d < L.descs.size(); ++d) {
    const int mid = L.descs[d].map;
    if (mid < 0 || S.lmaps[jj][d].fp_ptr.p) continue;
    const MapH& M = sched->maps_meta[mid];
    build_local_map(sched->dmaps[mid].p, M.arity, sched->set_size[M.to], S.sigma[jj].p, n, S.m, S.lmaps[jj][d], s);
  }
}

// Longest dependency chain per time step of the (step, tile) graph in the steady state: the
// chain lengths L over 12 steps, every node after its dependencies (within a step in order of
// sub-chain, then colour; wrapped dependencies from the step before), L(node) = weight +
// max L(dependency); the growth of max L over the last 5 steps divided by 5.  With unit weights
// it counts nodes; with plan-item weights it is divided by the mean items per node.
void critical_path(DataflowPlan& D, const std::vector<std::vector<int32_t>>& deps,
                   const std::vector<int32_t>& colour, const std::vector<double>& items_of) {
  const int32_t G = D.cum.back();
  D.items_per_step = 0;
  for (double x : items_of) D.items_per_step += x;
  if (G == 0) return;
  std::vector<int32_t> order(G);
  std::vector<int> sub_of(G);
  for (size_t k = 0; k + 1 < D.cum.size(); ++k)
    for (int32_t g = D.cum[k]; g < D.cum[k + 1]; ++g) sub_of[g] = (int)k;
  for (int32_t g = 0; g < G; ++g) order[g] = g;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return sub_of[x] != sub_of[y] ? sub_of[x] < sub_of[y] : colour[x] < colour[y];
  });
  constexpr int kSteps = 12, kTail = 5;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<double> prev(G, 0.0), cur(G, 0.0), top(kSteps, 0.0);
    for (int st = 0; st < kSteps; ++st) {
      for (int32_t g : order) {
        double m = 0;
        for (int32_t e : deps[g]) m = std::max(m, (e & 1) ? prev[e >> 1] : cur[e >> 1]);
        cur[g] = (pass ? items_of[g] : 1.0) + m;
        top[st] = std::max(top[st], cur[g]);
      }
      std::swap(prev, cur);
    }
    const double per_step = (top[kSteps - 1] - top[kSteps - 1 - kTail]) / kTail;
    if (pass == 0) D.cp_nodes = per_step;
    else D.cp_items = D.items_per_step > 0 ? per_step / (D.items_per_step / G) : 0;
  }
}

// Dependencies between tiles for the dataflow executor, from the cells each tile touches in
// each sub-chain (its plan items; both cells of an interior facet are items of the facet's tile):
// inside a sub-chain, a tile waits for the lower-colour tiles that touch one of its cells; across
// sub-chains, for the tiles of the previous sub-chain (in chain order, wrapping to the previous
// step) that touched the same cell.  Every access to a cell is thereby ordered as in the untiled
// chain.  Built on the device: per sub-chain the sorted, de-duplicated (cell, tile) pairs of the
// plan items give each cell's touching tiles; one pass counts each cell's edges, a scan places
// them, a second pass emits (dependency, node << 1 | previous step) pairs, and a sort removes the
// duplicates and leaves the successor lists in CSR order.
namespace {

constexpr int kMaxSub = 16;
struct TouchTables {
  const int32_t* ptr[kMaxSub];     // [nc + 1] per sub-chain
  const int32_t* tile[kMaxSub];    // tiles touching each cell, ascending
  const int32_t* colour[kMaxSub];  // colour of each tile
  int32_t cum[kMaxSub + 1];        // global tile id base
  int32_t K;
};

// (cell, tile) of every plan item of one segment: one thread per tile
__global__ void k_plan_pairs(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items, int32_t m,
                             uint32_t* __restrict__ cell, uint32_t* __restrict__ tile) {
  GRID_STRIDE(t, m) {
    for (int32_t i = ptr[t]; i < ptr[t + 1]; ++i) {
      cell[i] = (uint32_t)(items[i] >> 5);
      tile[i] = (uint32_t)t;
    }
  }
}

// the dependency edges of cell w: count (out == nullptr) or emit at pos
template <bool EMIT>
__device__ __forceinline__ int32_t cell_edges(const TouchTables& T, int64_t w, uint32_t* src, uint32_t* dst,
                                              int64_t pos) {
  int32_t n = 0;
  int first = -1, last = -1;
  for (int k = 0; k < T.K; ++k)
    if (T.ptr[k][w + 1] > T.ptr[k][w]) {
      if (first < 0) first = k;
      last = k;
    }
  int prev = last;  // the previous touching sub-chain, wrapping to the last one of the previous step
  for (int k = first; k >= 0 && k < T.K; ++k) {
    const int32_t b0 = T.ptr[k][w], b1 = T.ptr[k][w + 1];
    if (b1 == b0) continue;
    const uint32_t wrap = k == first ? 1u : 0u;
    const int32_t p0 = T.ptr[prev][w], p1 = T.ptr[prev][w + 1];
    for (int32_t x = b0; x < b1; ++x) {
      const int32_t tb = T.tile[k][x], gb = T.cum[k] + tb;
      const int32_t cb = T.colour[k][tb];
      for (int32_t y = b0; y < b1; ++y) {
        const int32_t ta = T.tile[k][y];
        if (T.colour[k][ta] < cb) {
          if (EMIT) {
            src[pos + n] = (uint32_t)(T.cum[k] + ta);
            dst[pos + n] = ((uint32_t)gb << 1);
          }
          ++n;
        }
      }
      for (int32_t y = p0; y < p1; ++y) {
        if (EMIT) {
          src[pos + n] = (uint32_t)(T.cum[prev] + T.tile[prev][y]);
          dst[pos + n] = ((uint32_t)gb << 1) | wrap;
        }
        ++n;
      }
    }
    prev = k;
  }
  return n;
}
__global__ void k_edge_count(TouchTables T, int64_t nc, int32_t* __restrict__ cnt) {
  GRID_STRIDE(w, nc) cnt[w] = cell_edges<false>(T, w, nullptr, nullptr, 0);
}
__global__ void k_edge_emit(TouchTables T, int64_t nc, const int32_t* __restrict__ pos, uint32_t* __restrict__ src,
                            uint32_t* __restrict__ dst) {
  GRID_STRIDE(w, nc) cell_edges<true>(T, w, src, dst, pos[w]);
}
// in-degrees: every distinct edge once; the ones from the same step also count for the first step
__global__ void k_indeg(const uint32_t* __restrict__ dst, int64_t n, int32_t* __restrict__ indeg0,
                        int32_t* __restrict__ indeg) {
  GRID_STRIDE(e, n) {
    const uint32_t d = dst[e];
    atomicAdd(&indeg[d >> 1], 1);
    if (!(d & 1)) atomicAdd(&indeg0[d >> 1], 1);
  }
}

// sort (a, b) pairs by a then b, drop repeats; returns the count (pairs compacted in place)
int64_t sort_unique_pairs(DevBuf<uint32_t>& a, int abits, DevBuf<uint32_t>& b, int bbits, int64_t n, cudaStream_t s) {
  if (n == 0) return 0;
  DevBuf<uint32_t> order;
  sort_by_two(a, abits, b, bbits, n, order, s);  // a sorted in place
  DevBuf<uint32_t> sb(n);
  k_gather_div<<<grid_for(n), 256, 0, s>>>((const int32_t*)b.p, order.p, n, 1, sb.p);
  DevBuf<int32_t> flag(n), pos(n + 1);
  k_run_heads<<<grid_for(n), 256, 0, s>>>(a.p, sb.p, n, flag.p);
  exclusive_scan_i32(flag.p, pos.p, n, s);
  int32_t nu = 0;
  SLT_CUDA(cudaMemcpyAsync(&nu, pos.p + n, 4, cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  DevBuf<uint32_t> ua(std::max(nu, 1)), ub(std::max(nu, 1));
  k_compact2<<<grid_for(n), 256, 0, s>>>(a.p, sb.p, flag.p, pos.p, n, ua.p, (int32_t*)ub.p);
  SLT_CUDA(cudaGetLastError());
  a = std::move(ua);
  b = std::move(ub);
  return nu;
}

}  // namespace

void build_dataflow(slt_schedule sched, slt_mesh mesh, cudaStream_t s) {
  DataflowPlan& D = sched->df;
  const int K = (int)sched->subs.size();
  if (K > kMaxSub) fail(SLT_ERR_UNSUPPORTED, "more than 16 sub-chains");
  const int64_t nc = mesh->nc;
  D.cum.assign(K + 1, 0);
  for (int k = 0; k < K; ++k) D.cum[k + 1] = D.cum[k] + sched->subs[k].m;
  const int32_t G = D.cum[K];
  TouchTables T{};
  T.K = K;
  std::vector<DevBuf<int32_t>> tptr(K), ttile(K);
  std::vector<double> items_of(G, 0.0);  // plan items of each node
  for (int k = 0; k < K; ++k) {
    SubSched& sub = sched->subs[k];
    T.cum[k] = D.cum[k];
    T.colour[k] = sub.colour.p;
    // (cell, tile) pairs of every segment's items
    std::vector<int32_t> seg_n;
    int64_t n = 0;
    for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last)) {
      std::vector<int32_t> ptr = sub.plan_ptr[J0 - sub.first].download(s, sub.m + 1);
      for (int32_t t = 0; t < sub.m; ++t) items_of[D.cum[k] + t] += ptr[t + 1] - ptr[t];
      seg_n.push_back(ptr[sub.m]);
      n += ptr[sub.m];
    }
    DevBuf<uint32_t> cell(std::max<int64_t>(n, 1)), tile(std::max<int64_t>(n, 1));
    int64_t o = 0, si = 0;
    for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last), ++si) {
      const int jj = J0 - sub.first;
      if (seg_n[si]) k_plan_pairs<<<grid_for(sub.m), 256, 0, s>>>(sub.plan_ptr[jj].p, sub.plan_items[jj].p, sub.m,
                                                                  cell.p + o, tile.p + o);
      o += seg_n[si];
    }
    SLT_CUDA(cudaGetLastError());
    const int64_t nu = sort_unique_pairs(cell, bits_for(std::max<int64_t>(nc - 1, 1)), tile,
                                         bits_for(std::max(sub.m - 1, 1)), n, s);
    tptr[k].alloc(nc + 1);
    lower_bound_offsets(cell.p, nu, nc, tptr[k].p, s);
    ttile[k].alloc(std::max<int64_t>(nu, 1));
    if (nu) SLT_CUDA(cudaMemcpyAsync(ttile[k].p, tile.p, nu * 4, cudaMemcpyDeviceToDevice, s));
    T.ptr[k] = tptr[k].p;
    T.tile[k] = ttile[k].p;
  }
  T.cum[K] = D.cum[K];
  // edges: count per cell, place, emit; then distinct (dependency, node code) pairs in order
  DevBuf<int32_t> cnt(nc), pos(nc + 1);
  k_edge_count<<<grid_for(nc), 256, 0, s>>>(T, nc, cnt.p);
  exclusive_scan_i32(cnt.p, pos.p, nc, s);
  int32_t ne = 0;
  SLT_CUDA(cudaMemcpyAsync(&ne, pos.p + nc, 4, cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  DevBuf<uint32_t> esrc(std::max(ne, 1)), edst(std::max(ne, 1));
  if (ne) k_edge_emit<<<grid_for(nc), 256, 0, s>>>(T, nc, pos.p, esrc.p, edst.p);
  SLT_CUDA(cudaGetLastError());
  const int64_t nd = sort_unique_pairs(esrc, bits_for(std::max(G - 1, 1)), edst,
                                       bits_for(std::max<int64_t>(2 * (int64_t)G - 1, 1)), ne, s);
  D.ndeps = nd;
  D.succ_ptr.alloc(G + 1);
  lower_bound_offsets(esrc.p, nd, G, D.succ_ptr.p, s);
  D.succ.alloc(std::max<int64_t>(nd, 1));
  if (nd) SLT_CUDA(cudaMemcpyAsync(D.succ.p, edst.p, nd * 4, cudaMemcpyDeviceToDevice, s));
  D.indeg0.alloc(G);
  D.indeg.alloc(G);
  SLT_CUDA(cudaMemsetAsync(D.indeg0.p, 0, G * 4, s));
  SLT_CUDA(cudaMemsetAsync(D.indeg.p, 0, G * 4, s));
  if (nd) k_indeg<<<grid_for(nd), 256, 0, s>>>(edst.p, nd, D.indeg0.p, D.indeg.p);
  SLT_CUDA(cudaGetLastError());
  D.err.alloc(1);
  D.head.alloc(2);
  // the longest chain per step, on the host over the (small) graph
  std::vector<int32_t> sp = D.succ_ptr.download(s, G + 1);
  std::vector<int32_t> sv = D.succ.download(s, std::max<int64_t>(nd, 1));
  std::vector<std::vector<int32_t>> deps(G);
  std::vector<int32_t> sub_of(G), indeg_sub(G, 0);
  for (int k = 0; k < K; ++k)
    for (int32_t g = D.cum[k]; g < D.cum[k + 1]; ++g) sub_of[g] = k;
  for (int32_t g = 0; g < G; ++g)
    for (int32_t i = sp[g]; i < sp[g + 1]; ++i) {
      deps[sv[i] >> 1].push_back((g << 1) | (sv[i] & 1));
      if (!(sv[i] & 1) && sub_of[sv[i] >> 1] == sub_of[g]) ++indeg_sub[sv[i] >> 1];
    }
  D.indeg_sub.alloc(std::max(G, 1));
  D.indeg_sub.upload(indeg_sub.data(), G, s);
  std::vector<int32_t> colour(G);
  for (int k = 0; k < K; ++k) {
    std::vector<int32_t> col = sched->subs[k].colour.download(s, sched->subs[k].m);
    for (int32_t i = 0; i < sched->subs[k].m; ++i) colour[D.cum[k] + i] = col[i];
  }
  critical_path(D, deps, colour, items_of);
  SLT_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ staged executor plan
// The staged executor (executor 3) runs one tile's sub-chain out of shared memory.  Its plan:
//   footprint   the cells the tile's segments touch (items of any segment), ascending work id; a
//               cell's slot is its position.  This is the tile's local map of the cell set
//               (Algorithm 1, compute_local_maps) for every loop of the sub-chain at once.  Each
//               entry carries a "shared" bit (another tile of the sub-chain touches the cell, so
//               values the tile writes for it go out to global memory) and the slots of the
//               cell's three face neighbours (kNoSlot: free surface, kNoSlot - 1: not in the
//               footprint).
//   lists       per segment and tile, seven lists of slot entries run as passes separated by a
//               barrier: gather (inputs read by the segment that no earlier segment of the tile
//               left in shared memory: slot | kind << 11, kind 0 the segment's operand, kind 1 the
//               later cell loop's own extra operand), init (the first cell loop, or the stored
//               partial value), interior faces 0, 1, 2, free-surface faces, later cell loop
//               (slot | flags << 11).  A cell's operations keep the order of the loop-by-loop chain.
// Residency of the temporaries, tracked per slot across the tile's segments (bits):
constexpr uint8_t RB_U1A = 1, RB_S1A = 2, RB_U2 = 4, RB_S1B = 8, RB_U1B = 16;
namespace {

__device__ __forceinline__ int32_t fp_find(const int32_t* __restrict__ fp, int32_t lo, int32_t hi, int32_t w) {
  int32_t a = lo, b = hi;  // first position with (fp & mask) >= w
  while (a < b) {
    const int32_t mid = (a + b) >> 1;
    if ((fp[mid] & 0x7fffffff) < w) a = mid + 1;
    else b = mid;
  }
  return (a < hi && (fp[a] & 0x7fffffff) == w) ? a - lo : -1;
}
__global__ void k_cell_count(const uint32_t* __restrict__ cell, int64_t n, int32_t* __restrict__ cnt) {
  GRID_STRIDE(e, n) atomicAdd(&cnt[cell[e]], 1);
}
// footprint entries: work id | shared << 31, neighbour slots (kSlotBits per face)
__global__ void k_fp_info(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ cell, int64_t n,
                          const int32_t* __restrict__ cnt, const int32_t* __restrict__ fp_ptr,
                          const int32_t* __restrict__ nbr, int64_t ncp, int32_t* __restrict__ fp_cell,
                          int32_t* __restrict__ fp_nsl) {
  GRID_STRIDE(e, n) fp_cell[e] = (int32_t)cell[e] | (cnt[cell[e]] > 1 ? (int32_t)0x80000000 : 0);
}
__global__ void k_fp_nsl(const uint32_t* __restrict__ tile, const uint32_t* __restrict__ cell, int64_t n,
                         const int32_t* __restrict__ fp_ptr, const int32_t* __restrict__ fp_cell,
                         const int32_t* __restrict__ nbr, int64_t ncp, int32_t* __restrict__ fp_nsl) {
  GRID_STRIDE(e, n) {
    const int32_t t = (int32_t)tile[e], w = (int32_t)cell[e];
    int32_t packed = 0;
    for (int f = 0; f < 3; ++f) {
      const int32_t nb = nbr[f * ncp + w];
      int32_t sl = kNoSlot;
      if (nb >= 0) {
        sl = fp_find(fp_cell, fp_ptr[t], fp_ptr[t + 1], nb >> 3);
        if (sl < 0) sl = kNoSlot - 1;
      }
      packed |= sl << (kSlotBits * f);
    }
    fp_nsl[e] = packed;
  }
}
// the segment's items as flags per footprint slot (| 64: the slot is an item)
__global__ void k_item_flags(const int32_t* __restrict__ ptr, const int32_t* __restrict__ items, int32_t m,
                             const int32_t* __restrict__ fp_ptr, const int32_t* __restrict__ fp_cell,
                             uint8_t* __restrict__ iflag) {
  GRID_STRIDE(t, m) {
    for (int32_t i = ptr[t]; i < ptr[t + 1]; ++i) {
      const int32_t sl = fp_find(fp_cell, fp_ptr[t], fp_ptr[t + 1], items[i] >> 5);
      if (sl >= 0) iflag[fp_ptr[t] + sl] = (uint8_t)((items[i] & 31) | 64);
    }
  }
}

// One tile per thread, slots ascending.  COUNT: need bits and list lengths; otherwise emit the
// lists at off and update the residency bits.
struct StageSeg {
  int H;            // phase
  uint8_t in_rb;    // residency bit of the segment's operand (0: never resident)
  uint8_t x_rb;     // residency bit of the later cell loop's extra operand (0: none)
  bool has_x;       // the later cell loop reads its own extra operand (phases 2, 5)
  uint8_t set_all;  // residency bits every item leaves
  uint8_t set_pb;   // residency bits the later cell loop leaves
  uint8_t acc_rb;   // residency bit of the accumulated value (phases 2, 4; else the first cell loop)
};
template <bool COUNT>
__global__ void k_stage_lists(StageSeg sg, int32_t m, const int32_t* __restrict__ fp_ptr,
                              const int32_t* __restrict__ fp_nsl, const uint8_t* __restrict__ iflag,
                              uint8_t* __restrict__ need, uint8_t* __restrict__ res, int32_t* __restrict__ cnt,
                              const int32_t* __restrict__ off, int32_t* __restrict__ ent, int32_t* __restrict__ bad) {
  GRID_STRIDE(t, m) {
    const int32_t b = fp_ptr[t], nF = fp_ptr[t + 1] - b;
    int32_t c[SL_N] = {0, 0, 0, 0, 0, 0, 0};
    int32_t o[SL_N];
    if (!COUNT)
      for (int L = 0; L < SL_N; ++L) o[L] = off[t * SL_N + L];
    if (COUNT) {
      for (int32_t sl = 0; sl < nF; ++sl) need[b + sl] = 0;
      for (int32_t sl = 0; sl < nF; ++sl) {
        const int fl = iflag[b + sl];
        if (!(fl & 64)) continue;
        const int32_t ns = fp_nsl[b + sl];
        if ((fl & 8) || (fl & 7)) need[b + sl] |= 1;
        for (int f = 0; f < 3; ++f) {
          const int32_t nsf = (ns >> (kSlotBits * f)) & kNoSlot;
          if (((fl >> f) & 1) && nsf < kNoSlot - 1) need[b + nsf] |= 1;
          if (((fl >> f) & 1) && nsf == kNoSlot - 1) atomicAdd(bad, 1);  // a facet with one cell outside
        }
        if (sg.has_x && (fl & 16)) need[b + sl] |= 2;
      }
    }
    auto put = [&](int L, int32_t v) {
      if (COUNT) ++c[L];
      else ent[o[L]++] = v;
    };
    // gather: operands read here that no earlier segment of the tile left in shared memory
    for (int32_t sl = 0; sl < nF; ++sl) {
      const uint8_t nd = need[b + sl], r = res[b + sl];
      if ((nd & 1) && !(sg.in_rb && (r & sg.in_rb))) put(SL_GATHER, sl);
      if ((nd & 2) && !(sg.x_rb && (r & sg.x_rb))) put(SL_GATHER, sl | (1 << kSlotBits));
    }
    // init: first cell loop items first, then the others (partial values, or already resident)
    for (int pass = 0; pass < 2; ++pass)
      for (int32_t sl = 0; sl < nF; ++sl) {
        int fl = iflag[b + sl];
        if (!(fl & 64) || (((fl & 8) != 0) != (pass == 0))) continue;
        fl &= 31;
        const bool load = (sg.acc_rb ? !(res[b + sl] & sg.acc_rb) : !(fl & 8));
        put(SL_INIT, sl | ((fl | (load ? kLoadBit : 0)) << kSlotBits));
      }
    for (int f = 0; f < 3; ++f)
      for (int32_t sl = 0; sl < nF; ++sl) {
        const int fl = iflag[b + sl];
        const int32_t nsf = (fp_nsl[b + sl] >> (kSlotBits * f)) & kNoSlot;
        if ((fl & 64) && ((fl >> f) & 1) && nsf != kNoSlot) put(SL_INT0 + f, sl | ((fl & 31) << kSlotBits));
      }
    for (int32_t sl = 0; sl < nF; ++sl) {
      const int fl = iflag[b + sl];
      if (!(fl & 64)) continue;
      bool ext = false;
      for (int f = 0; f < 3; ++f)
        ext |= ((fl >> f) & 1) && (((fp_nsl[b + sl] >> (kSlotBits * f)) & kNoSlot) == kNoSlot);
      if (ext) put(SL_EXT, sl | ((fl & 31) << kSlotBits));
    }
    for (int32_t sl = 0; sl < nF; ++sl) {
      const int fl = iflag[b + sl];
      if ((fl & 64) && (fl & 16)) put(SL_PB, sl | ((fl & 31) << kSlotBits));
    }
    if (COUNT) {
      for (int L = 0; L < SL_N; ++L) cnt[t * SL_N + L] = c[L];
    } else {
      for (int32_t sl = 0; sl < nF; ++sl) {
        const int fl = iflag[b + sl];
        if (!(fl & 64)) continue;
        res[b + sl] |= sg.set_all | ((fl & 16) ? sg.set_pb : 0);
      }
    }
  }
}

}  // namespace

int32_t stage_capacity(int p) {
  int dev = 0, smem = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  SLT_CUDA(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int Np = (p + 1) * (p + 2) / 2;
  // regions of 8 Np doubles per slot plus two int32 per slot; 1 KB for the kernel's own variables
  const int64_t per = 64 * (int64_t)Np + 8;
  return (int32_t)(std::min<int64_t>(kNoSlot - 1, (smem - 1024) / per) / 4 * 4);  // the kernel pads to 4
}

void stage_build(slt_schedule sched, slt_mesh mesh, SubSched& sub, cudaStream_t s) {
  const int32_t m = sub.m;
  const int64_t nc = mesh->nc;
  std::vector<int32_t> seg_n;
  int64_t n = 0;
  for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last)) {
    int32_t tot = 0;
    SLT_CUDA(cudaMemcpyAsync(&tot, sub.plan_ptr[J0 - sub.first].p + m, 4, cudaMemcpyDeviceToHost, s));
    SLT_CUDA(cudaStreamSynchronize(s));
    seg_n.push_back(tot);
    n += tot;
  }
  DevBuf<uint32_t> cell(std::max<int64_t>(n, 1)), tile(std::max<int64_t>(n, 1));
  {
    int64_t o = 0, si = 0;
    for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last), ++si) {
      const int jj = J0 - sub.first;
      if (seg_n[si]) k_plan_pairs<<<grid_for(m), 256, 0, s>>>(sub.plan_ptr[jj].p, sub.plan_items[jj].p, m,
                                                              cell.p + o, tile.p + o);
      o += seg_n[si];
    }
  }
  const int64_t nu = sort_unique_pairs(tile, bits_for(std::max(m - 1, 1)), cell,
                                       bits_for(std::max<int64_t>(nc - 1, 1)), n, s);
  sub.fp_ptr.alloc(m + 1);
  lower_bound_offsets(tile.p, nu, m, sub.fp_ptr.p, s);
  sub.fp_cell.alloc(std::max<int64_t>(nu, 1));
  sub.fp_nsl.alloc(std::max<int64_t>(nu, 1));
  {
    DevBuf<int32_t> cnt(nc);
    SLT_CUDA(cudaMemsetAsync(cnt.p, 0, nc * 4, s));
    if (nu) {
      k_cell_count<<<grid_for(nu), 256, 0, s>>>(cell.p, nu, cnt.p);
      k_fp_info<<<grid_for(nu), 256, 0, s>>>(tile.p, cell.p, nu, cnt.p, sub.fp_ptr.p, mesh->nbr.p, mesh->ncp,
                                             sub.fp_cell.p, sub.fp_nsl.p);
      k_fp_nsl<<<grid_for(nu), 256, 0, s>>>(tile.p, cell.p, nu, sub.fp_ptr.p, sub.fp_cell.p, mesh->nbr.p, mesh->ncp,
                                            sub.fp_nsl.p);
    }
    SLT_CUDA(cudaGetLastError());
    SLT_CUDA(cudaStreamSynchronize(s));
  }
  {
    std::vector<int32_t> fp = sub.fp_ptr.download(s, m + 1);
    sub.max_fp = 0;
    for (int32_t t = 0; t < m; ++t) sub.max_fp = std::max(sub.max_fp, fp[t + 1] - fp[t]);
  }
  if (sub.max_fp > kNoSlot - 1)  // the lists name cells by slot, kSlotBits bits each
    fail(SLT_ERR_UNSUPPORTED, "staged plan: a tile touches " + std::to_string(sub.max_fp) + " cells, more than the " +
                                  std::to_string(kNoSlot - 1) + " footprint slots its lists can name; use a smaller tile size");
  const int nl = sub.last - sub.first;
  sub.st_off.clear();
  sub.st_ent.clear();
  sub.st_off.resize(nl);
  sub.st_ent.resize(nl);
  DevBuf<uint8_t> res(std::max<int64_t>(nu, 1)), need(std::max<int64_t>(nu, 1)), iflag(std::max<int64_t>(nu, 1));
  SLT_CUDA(cudaMemsetAsync(res.p, 0, std::max<int64_t>(nu, 1), s));
  DevBuf<int32_t> cnt((size_t)m * SL_N), bad(1);
  SLT_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
  for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last)) {
    const int jj = J0 - sub.first;
    const int H = phase_of(J0);
    StageSeg sg{};
    sg.H = H;
    switch (H) {
      case 0: sg.in_rb = 0; sg.set_all = RB_U1A; break;
      case 1: sg.in_rb = RB_U1A; sg.set_pb = RB_S1A | RB_U2; break;
      case 2: sg.in_rb = RB_S1A; sg.has_x = true; sg.x_rb = RB_U1A; sg.acc_rb = RB_U2; break;
      case 3: sg.in_rb = 0; sg.set_pb = RB_S1B | RB_U1B; break;
      case 4: sg.in_rb = RB_S1B; sg.acc_rb = RB_U1B; sg.set_all = RB_U1B; break;
      default: sg.in_rb = RB_U1B; sg.has_x = true; sg.x_rb = RB_S1B; break;
    }
    SLT_CUDA(cudaMemsetAsync(iflag.p, 0, std::max<int64_t>(nu, 1), s));
    k_item_flags<<<grid_for(m), 256, 0, s>>>(sub.plan_ptr[jj].p, sub.plan_items[jj].p, m, sub.fp_ptr.p,
                                             sub.fp_cell.p, iflag.p);
    k_stage_lists<true><<<grid_for(m, 64), 64, 0, s>>>(sg, m, sub.fp_ptr.p, sub.fp_nsl.p, iflag.p, need.p, res.p,
                                                        cnt.p, nullptr, nullptr, bad.p);
    sub.st_off[jj].alloc((size_t)m * SL_N + 1);
    exclusive_scan_i32(cnt.p, sub.st_off[jj].p, (int64_t)m * SL_N, s);
    int32_t tot = 0;
    SLT_CUDA(cudaMemcpyAsync(&tot, sub.st_off[jj].p + (int64_t)m * SL_N, 4, cudaMemcpyDeviceToHost, s));
    SLT_CUDA(cudaStreamSynchronize(s));
    sub.st_ent[jj].alloc(std::max(tot, 1));
    k_stage_lists<false><<<grid_for(m, 64), 64, 0, s>>>(sg, m, sub.fp_ptr.p, sub.fp_nsl.p, iflag.p, need.p, res.p,
                                                         nullptr, sub.st_off[jj].p, sub.st_ent[jj].p, bad.p);
    SLT_CUDA(cudaGetLastError());
  }
  int32_t hbad = 0;
  SLT_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, s));
  SLT_CUDA(cudaStreamSynchronize(s));
  if (hbad) fail(SLT_ERR_UNSUPPORTED, "staged plan: a facet iteration's cell is outside its tile's footprint");
}

// ------------------------------------------------------------------ export flags (local maps)
// Per iteration of one loop: 1 when an element the iteration writes or increments is also
// touched, in some loop of its sub-chain, by a tile other than the iteration's own - the values
// a tile must export (write back for another tile) rather than keep local.  The (tile, element)
// pairs of every access of the sub-chain come from the tiling functions (direct accesses) and the
// local-map footprints (indirect ones); a sort drops repeats, and an element touched by more than
// one tile is shared.

namespace {

// (tile, element) of every entry of a footprint CSR: the tile by binary search in fp_ptr
__global__ void k_csr_pairs(const int32_t* __restrict__ fp_ptr, int32_t m, const int32_t* __restrict__ fp,
                            int64_t n, uint32_t* __restrict__ tile, uint32_t* __restrict__ elem) {
  GRID_STRIDE(e, n) {
    int32_t lo = 0, hi = m;  // the last t with fp_ptr[t] <= e
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (fp_ptr[mid] <= e) lo = mid;
      else hi = mid;
    }
    tile[e] = (uint32_t)lo;
    elem[e] = (uint32_t)fp[e];
  }
}
__global__ void k_direct_pairs(const int32_t* __restrict__ sig, int64_t n, uint32_t* __restrict__ tile,
                               uint32_t* __restrict__ elem) {
  GRID_STRIDE(e, n) {
    tile[e] = (uint32_t)sig[e];
    elem[e] = (uint32_t)e;
  }
}

constexpr int kMaxExpDesc = 8;
struct ExpDescs {
  int32_t n;
  int32_t arity[kMaxExpDesc];              // 0: direct access (the iteration's own element)
  const int32_t* fp_ptr[kMaxExpDesc];
  const int32_t* fp[kMaxExpDesc];
  const int32_t* lmap[kMaxExpDesc];
  const int32_t* cnt[kMaxExpDesc];         // distinct tiles per element of the target set
};
__global__ void k_export_flags(ExpDescs d, const int32_t* __restrict__ sig, int64_t n, int32_t* __restrict__ out) {
  GRID_STRIDE(i, n) {
    int32_t f = 0;
    for (int k = 0; k < d.n; ++k) {
      if (d.arity[k] == 0) {
        f |= d.cnt[k][i] > 1;
        continue;
      }
      const int32_t base = d.fp_ptr[k][sig[i]];
      for (int a = 0; a < d.arity[k]; ++a) f |= d.cnt[k][d.fp[k][base + d.lmap[k][i * d.arity[k] + a]]] > 1;
    }
    out[i] = f;
  }
}

}  // namespace

void export_flags(slt_schedule sched, int32_t J, DevBuf<int32_t>& out, cudaStream_t s) {
  SubSched* S = nullptr;
  for (SubSched& x : sched->subs)
    if (J >= x.first && J < x.last) S = &x;
  if (!S) fail(SLT_ERR_ARG, "loop not inspected");
  for (int jj = 0; jj < S->last - S->first; ++jj) ensure_local_maps(sched, *S, jj, s);
  const LoopH& L = sched->loops[J];
  const int64_t n = sched->set_size[L.set];
  // distinct tiles per element of a set, over every access of the sub-chain
  std::vector<std::pair<int32_t, DevBuf<int32_t>>> counts;
  auto count_for = [&](int32_t T) -> const int32_t* {
    for (auto& c : counts)
      if (c.first == T) return c.second.p;
    int64_t tot = 0;
    std::vector<std::pair<int, int>> parts;  // (loop, desc) accessing T
    std::vector<int64_t> len;
    for (int j = S->first; j < S->last; ++j)
      for (int d = 0; d < (int)sched->loops[j].descs.size(); ++d) {
        const DescH& D = sched->loops[j].descs[d];
        int64_t k = 0;
        if (D.map < 0 && sched->loops[j].set == T) k = sched->set_size[T];
        if (D.map >= 0 && sched->maps_meta[D.map].to == T) {
          int32_t e = 0;
          SLT_CUDA(cudaMemcpy(&e, S->lmaps[j - S->first][d].fp_ptr.p + S->m, 4, cudaMemcpyDeviceToHost));
          k = e;
        }
        if (k) {
          parts.push_back({j, d});
          len.push_back(k);
          tot += k;
        }
      }
    DevBuf<uint32_t> tile(std::max<int64_t>(tot, 1)), elem(std::max<int64_t>(tot, 1));
    int64_t o = 0;
    for (size_t q = 0; q < parts.size(); ++q) {
      const int j = parts[q].first, d = parts[q].second;
      if (sched->loops[j].descs[d].map < 0) {
        k_direct_pairs<<<grid_for(len[q]), 256, 0, s>>>(S->sigma[j - S->first].p, len[q], tile.p + o, elem.p + o);
      } else {
        const LocalMap& lm = S->lmaps[j - S->first][d];
        k_csr_pairs<<<grid_for(len[q]), 256, 0, s>>>(lm.fp_ptr.p, S->m, lm.fp.p, len[q], tile.p + o, elem.p + o);
      }
      o += len[q];
    }
    SLT_CUDA(cudaGetLastError());
    const int64_t nu = sort_unique_pairs(tile, bits_for(std::max(S->m - 1, 1)), elem,
                                         bits_for(std::max<int64_t>(sched->set_size[T] - 1, 1)), tot, s);
    DevBuf<int32_t> cnt(std::max<int64_t>(sched->set_size[T], 1));
    SLT_CUDA(cudaMemsetAsync(cnt.p, 0, std::max<int64_t>(sched->set_size[T], 1) * 4, s));
    if (nu) k_cell_count<<<grid_for(nu), 256, 0, s>>>(elem.p, nu, cnt.p);
    SLT_CUDA(cudaGetLastError());
    counts.push_back({T, std::move(cnt)});
    return counts.back().second.p;
  };
  ExpDescs ed{};
  for (int d = 0; d < (int)L.descs.size(); ++d) {
    const DescH& D = L.descs[d];
    if (D.mode == 'r') continue;
    if (ed.n == kMaxExpDesc) fail(SLT_ERR_UNSUPPORTED, "more than 8 written descriptors in one loop");
    if (D.map < 0) {
      ed.arity[ed.n] = 0;
      ed.cnt[ed.n] = count_for(L.set);
    } else {
      const LocalMap& lm = S->lmaps[J - S->first][d];
      ed.arity[ed.n] = sched->maps_meta[D.map].arity;
      ed.fp_ptr[ed.n] = lm.fp_ptr.p;
      ed.fp[ed.n] = lm.fp.p;
      ed.lmap[ed.n] = lm.lmap.p;
      ed.cnt[ed.n] = count_for(sched->maps_meta[D.map].to);
    }
    ++ed.n;
  }
  out.alloc(std::max<int64_t>(n, 1));
  if (n) k_export_flags<<<grid_for(n), 256, 0, s>>>(ed, S->sigma[J - S->first].p, n, out.p);
  SLT_CUDA(cudaGetLastError());
  SLT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace slt

namespace slt {

// FP64 instructions per work item of each part of a phase (an instruction counts once whatever
// its flops: the pipe takes one issue slot for each), as the part functions of the executors
// issue them at degree p with nnz nonzeros of Dr plus Ds: [0] the first cell loop (volume part),
// [1] an interior face, [2] a free-surface face, [3] the later cell loop.
static void part_costs(int H, int Np, int Nfp, double nnz, double c[4]) {
  const double volB = 8.0 * Np + 2 * nnz, volD = 2 * nnz + 8.0 * Np;
  const double intB = 7.0 * Nfp + 2.0 * Np * Nfp, extB = 2 + 4.0 * Nfp + 2.0 * Np * Nfp;
  const double intD = 2.0 * Nfp + 2.0 * Np * Nfp + 4.0 * Np;
  const bool A = H == 0 || H == 2 || H == 4;
  c[0] = H == 0 ? volB : (H == 1 || H == 3 || H == 5) ? volD : 0;
  c[1] = A ? intB : intD;
  c[2] = A ? extB : 0;
  c[3] = (H == 1 || H == 3) ? 5.0 * Np + volB : H == 2 ? 4.0 * Np : H == 5 ? 11.0 * Np : 0;
}

void lane_info(slt_schedule sched, slt_mesh mesh, double out[4]) {
  const int Np = mesh->Np, Nfp = mesh->Nfp;
  double mx = 0, nnz = 0;
  for (double x : mesh->ref.Dr) mx = std::max(mx, std::fabs(x));
  for (double x : mesh->ref.Ds) mx = std::max(mx, std::fabs(x));
  for (double x : mesh->ref.Dr) nnz += std::fabs(x) > 1e-12 * mx;
  for (double x : mesh->ref.Ds) nnz += std::fabs(x) > 1e-12 * mx;
  std::vector<int32_t> nbr = mesh->nbr.download(nullptr, 3 * mesh->ncp);
  auto ext = [&](int64_t w, int f) { return nbr[f * mesh->ncp + w] < 0; };
  double useful = 0, exec_df = 0, exec_st = 0, exec_un = 0;
  // one item's parts, and the union over a warp of items (interior and free-surface faces apart)
  auto item_cost = [&](int H, int64_t w, int fl, const double* c) {
    double u = ((fl & 8) ? c[0] : 0) + ((fl & 16) ? c[3] : 0);
    for (int f = 0; f < 3; ++f)
      if ((fl >> f) & 1) u += ext(w, f) ? c[2] : c[1];
    return u;
  };
  auto warp_cost = [&](int H, const std::vector<std::pair<int64_t, int>>& it, size_t a, size_t b, const double* c) {
    int pa = 0, pb = 0, fi = 0, fe = 0;
    for (size_t i = a; i < b; ++i) {
      const int fl = it[i].second;
      pa |= (fl >> 3) & 1;
      pb |= (fl >> 4) & 1;
      for (int f = 0; f < 3; ++f)
        if ((fl >> f) & 1) {
          if (ext(it[i].first, f)) fe |= 1 << f;
          else fi |= 1 << f;
        }
    }
    return 32.0 * (pa * c[0] + pb * c[3] + __builtin_popcount(fi) * c[1] + __builtin_popcount(fe) * c[2]);
  };
  for (const SubSched& sub : sched->subs) {
    for (int J0 = sub.first; J0 < sub.last; J0 = seg_end(J0, sub.last)) {
      const int H = phase_of(J0);
      double c[4];
      part_costs(H, Np, Nfp, nnz, c);
      std::vector<int32_t> ptr = sub.plan_ptr[J0 - sub.first].download(nullptr, sub.m + 1);
      std::vector<int32_t> items = sub.plan_items[J0 - sub.first].download(nullptr, std::max(ptr[sub.m], 1));
      for (int32_t t = 0; t < sub.m; ++t) {
        std::vector<std::pair<int64_t, int>> it;
        for (int32_t i = ptr[t]; i < ptr[t + 1]; ++i) it.push_back({items[i] >> 5, items[i] & 31});
        for (auto& x : it) useful += 32.0 * item_cost(H, x.first, x.second, c) / 32.0;
        for (size_t a = 0; a < it.size(); a += 32) exec_df += warp_cost(H, it, a, std::min(it.size(), a + 32), c);
        // staged passes: the first cell loop, each interior face index, the free surface, the
        // later cell loop, each over its compacted list
        int64_t npa = 0, npb = 0, nint[3] = {0, 0, 0}, next = 0;
        double ext_work = 0;
        for (auto& x : it) {
          npa += (x.second >> 3) & 1;
          npb += (x.second >> 4) & 1;
          bool e = false;
          for (int f = 0; f < 3; ++f)
            if ((x.second >> f) & 1) {
              if (ext(x.first, f)) e = true;
              else ++nint[f];
            }
          next += e;
        }
        auto padded = [](int64_t n) { return (double)((n + 31) / 32 * 32); };
        exec_st += padded(npa) * c[0] + padded(npb) * c[3] + padded(nint[0]) * c[1] + padded(nint[1]) * c[1] +
                   padded(nint[2]) * c[1] + padded(next) * c[2] * 1.0;
        (void)ext_work;
      }
    }
  }
  // the untiled chain: every phase over all cells, warps of 32 consecutive work ids, all parts
  for (int H = 0; H < kPhases; ++H) {
    double c[4];
    part_costs(H, Np, Nfp, nnz, c);
    for (int64_t w0 = 0; w0 < mesh->nc; w0 += 32) {
      int fe = 0;
      for (int64_t w = w0; w < std::min<int64_t>(mesh->nc, w0 + 32); ++w)
        for (int f = 0; f < 3; ++f)
          if (ext(w, f)) fe |= 1 << f;
      const int fi = 7;  // every warp has cells with each interior face
      exec_un += 32.0 * (c[0] + c[3] + __builtin_popcount(fi) * c[1] + __builtin_popcount(fe) * (H == 0 || H == 2 || H == 4 ? c[2] : 0));
    }
  }
  out[0] = useful;
  out[1] = exec_df;
  out[2] = exec_st;
  out[3] = exec_un;
}

}  // namespace slt
