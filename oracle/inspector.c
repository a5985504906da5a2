/* ORACLE (test infrastructure only; never linked into the product library).
 *
 * Sequential sparse-tiling inspector for a loop chain, following the paper's Algorithm 1
 * (inspection), Algorithm 2 (projection of a tiled loop) and Algorithm 3 (tiling function),
 * Section 5.1, in shared-memory mode (every set is a single core region).
 *
 * Readings of points the paper leaves open:
 *  - partition (Section 5.1.2): seed iterations are ranked (identity, or a stable sort by the
 *    order-16 Hilbert index of a per-element point quantised on a 65536x65536 grid over its
 *    bounding box); tile of rank r is r / ts.
 *  - find_map: the first map, in chain order (loops, then descriptors), whose source or target
 *    set is the seed set.  Two tiles are adjacent when one element of that map's source set
 *    touches both (target = seed), or when one target element is touched by seed elements of
 *    both (source = seed).  Fake edges from conflicts are added to this adjacency.
 *  - color: greedy in decreasing priority h(t) = splitmix64(t XOR seed); each tile takes the
 *    smallest colour not used by an already coloured neighbour (this equals Jones-Plassmann
 *    with the same priorities).  Sequential mode: tile t gets colour t.
 *  - projection (Algorithm 2): phi starts from the previous projection of the set (colour -1
 *    when there is none) instead of bottom, and takes the tiles of the iterations touching each
 *    element in ascending (iteration, slot) order; only a strictly larger colour replaces the
 *    current tile.  Direct descriptors are the identity map.  Every descriptor is projected,
 *    reads included.
 *  - tiling function (Algorithm 3): sigma is reset once per loop, then the maximum is taken
 *    over all descriptors in order and slots in order, strictly larger colour replaces.
 *    An iteration with no projected element goes to tile 0.
 *  - conflicts: any element whose candidate list (previous projection plus the touching
 *    iterations' tiles) holds two distinct tiles of equal colour records that pair.  The last
 *    loop of the chain is projected once more only to detect conflicts.  On conflicts the pairs
 *    become fake edges and inspection restarts from colouring (partition kept).  After
 *    max_rounds restarts, or as soon as the fake edges number more than 16 per tile (tiles
 *    scattered over the whole set, e.g. chunks of a random numbering, would otherwise make
 *    each round denser and slower), the colouring falls back to sequential mode, which cannot
 *    conflict.
 *  - backward tiling (Section 5.1.1: a seed loop in the middle of the chain, tiles grown
 *    towards the first loop with MIN in place of MAX): with seed loop s > 0, the seed loop is
 *    projected with MIN, then loops s-1, ..., 0 are tiled and projected in that order with MIN
 *    (smallest colour wins, earlier candidate kept on ties; no projection: tile 0).  Each
 *    earlier-loop iteration thereby runs in a tile of colour no larger than every later loop
 *    (up to s) touching its data.  Then a fresh MAX projection is built from loops 0, ..., s in
 *    order and loops s+1, ... are tiled forward as above, so they follow every earlier access.
 *    Conflicts are recorded in both phases with the same rule.  s = 0 is plain forward tiling.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static void invert(int64_t nsrc, int arity, const int32_t* m, int64_t ntgt, int64_t** off, int32_t** val);

static uint64_t splitmix64(uint64_t x) {
  /* SplitMix64 output function (Steele, Lea, Flood 2014): add the golden-ratio increment,
     then two xor-shift-multiply rounds and a final xor-shift. */
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Hilbert index of (x, y) in a 2^order grid: at each level from the top, the quadrant digit is
   0 for (lo,lo), 1 for (lo,hi), 2 for (hi,hi), 3 for (hi,lo) in (x,y); within the quadrant the
   lower bits are transposed (lower quadrants) and also reflected (lower-right quadrant). */
static uint32_t hilbert_index(uint32_t x, uint32_t y, int order) {
  uint32_t d = 0;
  for (int level = order - 1; level >= 0; --level) {
    uint32_t half = 1u << level;
    uint32_t hx = (x >> level) & 1u, hy = (y >> level) & 1u;
    uint32_t digit = hx ? (hy ? 2u : 3u) : (hy ? 1u : 0u);
    d = (d << 2) | digit;
    x &= half - 1u;
    y &= half - 1u;
    if (!hy) {
      if (hx) { x = half - 1u - x; y = half - 1u - y; }
      uint32_t t = x; x = y; y = t;
    }
  }
  return d;
}

void oracle_map_invert(int64_t nsrc, int arity, const int32_t* m, int64_t ntgt, int64_t* off, int32_t* val) {
  int64_t* o; int32_t* v;
  invert(nsrc, arity, m, ntgt, &o, &v);
  memcpy(off, o, (ntgt + 1) * sizeof(int64_t));
  memcpy(val, v, nsrc * arity * sizeof(int32_t));
  free(o); free(v);
}

uint32_t oracle_hilbert_index(uint32_t x, uint32_t y, int order) { return hilbert_index(x, y, order); }
uint64_t oracle_splitmix64(uint64_t x) { return splitmix64(x); }

typedef struct { uint64_t key; int64_t id; } kv_t;
static int cmp_kv_asc(const void* a, const void* b) {
  const kv_t *p = a, *q = b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->id < q->id ? -1 : (p->id > q->id);
}
typedef struct { int32_t a, b; } pair_t;
static int cmp_pair(const void* x, const void* y) {
  const pair_t *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  return p->b < q->b ? -1 : (p->b > q->b);
}

typedef struct { pair_t* v; int64_t n, cap; } pairvec;
static void pv_push(pairvec* pv, int32_t a, int32_t b) {
  if (pv->n == pv->cap) { pv->cap = pv->cap ? 2 * pv->cap : 1024; pv->v = realloc(pv->v, pv->cap * sizeof(pair_t)); }
  pv->v[pv->n].a = a; pv->v[pv->n].b = b; pv->n++;
}
static void pv_sort_unique(pairvec* pv) {
  if (!pv->n) return;
  qsort(pv->v, pv->n, sizeof(pair_t), cmp_pair);
  int64_t w = 1;
  for (int64_t i = 1; i < pv->n; ++i)
    if (pv->v[i].a != pv->v[w - 1].a || pv->v[i].b != pv->v[w - 1].b) pv->v[w++] = pv->v[i];
  pv->n = w;
}

/* Seed ranks: rank[e] = position of e in the seed ordering. */
void oracle_seed_rank(int64_t n, int renumber, const double* xy, int32_t* rank) {
  if (!renumber) { for (int64_t e = 0; e < n; ++e) rank[e] = (int32_t)e; return; }
  double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
  for (int64_t e = 1; e < n; ++e) {
    double x = xy[2 * e], y = xy[2 * e + 1];
    if (x < xmin) xmin = x;
    if (x > xmax) xmax = x;
    if (y < ymin) ymin = y;
    if (y > ymax) ymax = y;
  }
  kv_t* kv = malloc(n * sizeof(kv_t));
  for (int64_t e = 0; e < n; ++e) {
    double tx = xmax > xmin ? (xy[2 * e] - xmin) / (xmax - xmin) : 0.0;
    double ty = ymax > ymin ? (xy[2 * e + 1] - ymin) / (ymax - ymin) : 0.0;
    int64_t qx = (int64_t)(tx * 65535.0), qy = (int64_t)(ty * 65535.0);
    if (qx < 0) qx = 0;
    if (qx > 65535) qx = 65535;
    if (qy < 0) qy = 0;
    if (qy > 65535) qy = 65535;
    kv[e].key = hilbert_index((uint32_t)qx, (uint32_t)qy, 16);
    kv[e].id = e;
  }
  qsort(kv, n, sizeof(kv_t), cmp_kv_asc);
  for (int64_t r = 0; r < n; ++r) rank[kv[r].id] = (int32_t)r;
  free(kv);
}

/* CSR inverse of a map: for target e, the flat slots i*arity+k with map[i*arity+k] == e, in
   ascending order; values hold the source iteration i. */
static void invert(int64_t nsrc, int arity, const int32_t* m, int64_t ntgt, int64_t** off, int32_t** val) {
  int64_t* o = calloc(ntgt + 1, sizeof(int64_t));
  for (int64_t s = 0; s < nsrc * arity; ++s) o[m[s] + 1]++;
  for (int64_t e = 0; e < ntgt; ++e) o[e + 1] += o[e];
  int64_t* fill = malloc((ntgt + 1) * sizeof(int64_t));
  memcpy(fill, o, (ntgt + 1) * sizeof(int64_t));
  int32_t* v = malloc((nsrc * arity + 1) * sizeof(int32_t));
  for (int64_t s = 0; s < nsrc * arity; ++s) v[fill[m[s]]++] = (int32_t)(s / arity);
  free(fill);
  *off = o; *val = v;
}

typedef struct {
  int nsets; const int64_t* set_size;
  int nmaps; const int* map_from; const int* map_to; const int* map_arity; const int32_t* const* map_val;
  int nloops; const int* loop_set; const int* desc_ptr; const int* desc_map; const char* desc_mode;
} chain_t;

/* does tile t win over the current tile cur?  MAX (dir > 0) or MIN (dir < 0) colour, strictly */
static int wins(int dir, const int32_t* col, int32_t t, int32_t cur) {
  return dir > 0 ? col[t] > col[cur] : col[t] < col[cur];
}

/* Projection of loop j (Algorithm 2) into phi[] (per set), recording conflicts. */
static void project(const chain_t* L, int j, const int32_t* sig, int32_t** phi, const int32_t* col, pairvec* C,
                    int dir) {
  int Sj = L->loop_set[j];
  for (int d = L->desc_ptr[j]; d < L->desc_ptr[j + 1]; ++d) {
    int mid = L->desc_map[d];
    if (mid < 0) {
      int64_t n = L->set_size[Sj];
      if (!phi[Sj]) { phi[Sj] = malloc(n * sizeof(int32_t)); for (int64_t e = 0; e < n; ++e) phi[Sj][e] = -1; }
      for (int64_t e = 0; e < n; ++e) {
        int32_t old = phi[Sj][e], t = sig[e];
        if (old < 0 || wins(dir, col, t, old)) phi[Sj][e] = t;
        else if (t != old && col[t] == col[old]) pv_push(C, old < t ? old : t, old < t ? t : old);
      }
      continue;
    }
    int S = L->map_to[mid], a = L->map_arity[mid];
    int64_t n = L->set_size[S];
    int64_t* off; int32_t* val;
    invert(L->set_size[Sj], a, L->map_val[mid], n, &off, &val);
    if (!phi[S]) { phi[S] = malloc(n * sizeof(int32_t)); for (int64_t e = 0; e < n; ++e) phi[S][e] = -1; }
    int64_t maxdeg = 0;
    for (int64_t e = 0; e < n; ++e) if (off[e + 1] - off[e] > maxdeg) maxdeg = off[e + 1] - off[e];
    int32_t* cand = malloc((maxdeg + 1) * sizeof(int32_t));
    for (int64_t e = 0; e < n; ++e) {
      int nc = 0;
      int32_t cur = phi[S][e];
      if (cur >= 0) cand[nc++] = cur;
      for (int64_t k = off[e]; k < off[e + 1]; ++k) {
        int32_t t = sig[val[k]];
        cand[nc++] = t;
        if (cur < 0 || wins(dir, col, t, cur)) cur = t;
      }
      phi[S][e] = cur;
      for (int x = 0; x < nc; ++x)
        for (int y = x + 1; y < nc; ++y)
          if (cand[x] != cand[y] && col[cand[x]] == col[cand[y]])
            pv_push(C, cand[x] < cand[y] ? cand[x] : cand[y], cand[x] < cand[y] ? cand[y] : cand[x]);
    }
    free(cand); free(off); free(val);
  }
}

/* Tiling function of loop j (Algorithm 3). */
static void tile_loop(const chain_t* L, int j, int32_t* const* phi, const int32_t* col, int32_t* sig, int64_t* nbottom,
                      int dir) {
  int Sj = L->loop_set[j];
  int64_t n = L->set_size[Sj];
  for (int64_t e = 0; e < n; ++e) sig[e] = -1;
  for (int d = L->desc_ptr[j]; d < L->desc_ptr[j + 1]; ++d) {
    int mid = L->desc_map[d];
    if (mid < 0) {
      const int32_t* p = phi[Sj];
      if (!p) continue;
      for (int64_t e = 0; e < n; ++e) {
        int32_t t = p[e];
        if (t >= 0 && (sig[e] < 0 || wins(dir, col, t, sig[e]))) sig[e] = t;
      }
    } else {
      int S = L->map_to[mid], a = L->map_arity[mid];
      const int32_t* p = phi[S];
      if (!p) continue;
      const int32_t* m = L->map_val[mid];
      for (int64_t e = 0; e < n; ++e)
        for (int k = 0; k < a; ++k) {
          int32_t t = p[m[e * a + k]];
          if (t >= 0 && (sig[e] < 0 || wins(dir, col, t, sig[e]))) sig[e] = t;
        }
    }
  }
  for (int64_t e = 0; e < n; ++e) if (sig[e] < 0) { sig[e] = 0; (*nbottom)++; }
}

static void colour_tiles(int32_t m, const int64_t* aoff, const int32_t* adj, int sequential, uint64_t seed, int32_t* col) {
  if (sequential) { for (int32_t t = 0; t < m; ++t) col[t] = t; return; }
  kv_t* kv = malloc(m * sizeof(kv_t));
  for (int32_t t = 0; t < m; ++t) { kv[t].key = ~splitmix64((uint64_t)t ^ seed); kv[t].id = t; } /* descending priority */
  qsort(kv, m, sizeof(kv_t), cmp_kv_asc);
  for (int32_t t = 0; t < m; ++t) col[t] = -1;
  int32_t maxdeg = 0;
  for (int32_t t = 0; t < m; ++t) if (aoff[t + 1] - aoff[t] > maxdeg) maxdeg = (int32_t)(aoff[t + 1] - aoff[t]);
  char* used = calloc(maxdeg + 2, 1);
  for (int32_t i = 0; i < m; ++i) {
    int32_t t = (int32_t)kv[i].id;
    memset(used, 0, maxdeg + 2);
    for (int64_t k = aoff[t]; k < aoff[t + 1]; ++k) { int32_t c = col[adj[k]]; if (c >= 0 && c <= maxdeg) used[c] = 1; }
    int32_t c = 0; while (used[c]) ++c;
    col[t] = c;
  }
  free(used); free(kv);
}

/* Tile adjacency from the seed map plus fake edges, as CSR over m tiles. */
static void adjacency(const chain_t* L, int seed_set, const int32_t* sig0, int32_t m, const pairvec* fake,
                      int64_t** aoff, int32_t** adj) {
  pairvec P = {0};
  int found = 0;
  for (int j = 0; j < L->nloops && !found; ++j)
    for (int d = L->desc_ptr[j]; d < L->desc_ptr[j + 1] && !found; ++d) {
      int mid = L->desc_map[d];
      if (mid < 0) continue;
      int a = L->map_arity[mid];
      const int32_t* mv = L->map_val[mid];
      if (L->map_to[mid] == seed_set) {
        found = 1;
        for (int64_t i = 0; i < L->set_size[L->map_from[mid]]; ++i)
          for (int x = 0; x < a; ++x)
            for (int y = 0; y < a; ++y) {
              int32_t ta = sig0[mv[i * a + x]], tb = sig0[mv[i * a + y]];
              if (ta != tb) pv_push(&P, ta, tb);
            }
      } else if (L->map_from[mid] == seed_set) {
        found = 1;
        int64_t* off; int32_t* val;
        int64_t nt = L->set_size[L->map_to[mid]];
        invert(L->set_size[seed_set], a, mv, nt, &off, &val);
        for (int64_t e = 0; e < nt; ++e)
          for (int64_t x = off[e]; x < off[e + 1]; ++x)
            for (int64_t y = off[e]; y < off[e + 1]; ++y) {
              int32_t ta = sig0[val[x]], tb = sig0[val[y]];
              if (ta != tb) pv_push(&P, ta, tb);
            }
        free(off); free(val);
      }
    }
  for (int64_t k = 0; k < fake->n; ++k) { pv_push(&P, fake->v[k].a, fake->v[k].b); pv_push(&P, fake->v[k].b, fake->v[k].a); }
  pv_sort_unique(&P);
  int64_t* o = calloc(m + 1, sizeof(int64_t));
  for (int64_t k = 0; k < P.n; ++k) o[P.v[k].a + 1]++;
  for (int32_t t = 0; t < m; ++t) o[t + 1] += o[t];
  int32_t* v = malloc((P.n + 1) * sizeof(int32_t));
  for (int64_t k = 0; k < P.n; ++k) v[k] = P.v[k].b;
  free(P.v);
  *aoff = o; *adj = v;
}

/* Full inspection of one loop chain.  Outputs:
 *   rank[|S_seed|], colour[m], sigma (concatenated tiling functions of all loops, loop 0 first),
 *   stats[0..5] = m, ncolours, restarts, fell_back_to_sequential, conflict pairs in the last
 *   round with conflicts, iterations assigned to tile 0 for lack of any projection. */
int oracle_inspect(int nsets, const int64_t* set_size,
                   int nmaps, const int* map_from, const int* map_to, const int* map_arity,
                   const int32_t* const* map_val,
                   int nloops, const int* loop_set, const int* desc_ptr, const int* desc_map, const char* desc_mode,
                   int ts, int sequential, uint64_t prio_seed, int renumber, const double* seed_xy, int max_rounds,
                   int seed, int32_t* rank, int32_t* colour, int32_t* sigma, int64_t* stats) {
  if (ts <= 0 || nloops <= 0 || seed < 0 || seed >= nloops) return -1;
  chain_t L = {nsets, set_size, nmaps, map_from, map_to, map_arity, map_val, nloops, loop_set, desc_ptr, desc_map, desc_mode};
  int seed_set = loop_set[seed];
  int64_t nseed = set_size[seed_set];
  int32_t m = (int32_t)((nseed + ts - 1) / ts);
  oracle_seed_rank(nseed, renumber, seed_xy, rank);
  int64_t* sig_off = malloc((nloops + 1) * sizeof(int64_t));
  sig_off[0] = 0;
  for (int j = 0; j < nloops; ++j) sig_off[j + 1] = sig_off[j] + set_size[loop_set[j]];
  int32_t* sig_seed = sigma + sig_off[seed];
  for (int64_t e = 0; e < nseed; ++e) sig_seed[e] = rank[e] / ts;
  pairvec fake = {0};
  int restarts = 0, fell_back = 0;
  int64_t last_conflicts = 0, nbottom = 0;
  for (;;) {
    int64_t* aoff; int32_t* adj;
    adjacency(&L, seed_set, sig_seed, m, &fake, &aoff, &adj);
    colour_tiles(m, aoff, adj, sequential || fell_back, prio_seed, colour);
    free(aoff); free(adj);
    int32_t** phi = calloc(nsets, sizeof(int32_t*));
    pairvec C = {0};
    nbottom = 0;
    if (seed > 0) { /* backward: MIN from the seed loop towards loop 0 */
      project(&L, seed, sig_seed, phi, colour, &C, -1);
      for (int j = seed - 1; j >= 0; --j) {
        tile_loop(&L, j, phi, colour, sigma + sig_off[j], &nbottom, -1);
        project(&L, j, sigma + sig_off[j], phi, colour, &C, -1);
      }
      for (int s = 0; s < nsets; ++s) { free(phi[s]); phi[s] = NULL; }
    }
    /* forward: MAX over loops 0..seed, then tile and project the loops after the seed */
    for (int j = 0; j <= seed; ++j) project(&L, j, sigma + sig_off[j], phi, colour, &C, 1);
    for (int j = seed + 1; j < nloops; ++j) {
      tile_loop(&L, j, phi, colour, sigma + sig_off[j], &nbottom, 1);
      project(&L, j, sigma + sig_off[j], phi, colour, &C, 1);
    }
    for (int s = 0; s < nsets; ++s) free(phi[s]);
    free(phi);
    pv_sort_unique(&C);
    if (C.n == 0) { free(C.v); break; }
    last_conflicts = C.n;
    if (max_rounds < 0) { free(C.v); break; }  /* diagnostic mode: keep the first round */
    for (int64_t k = 0; k < C.n; ++k) pv_push(&fake, C.v[k].a, C.v[k].b);
    pv_sort_unique(&fake);
    free(C.v);
    ++restarts;
    if (restarts > max_rounds || fake.n > 16 * (int64_t)m) fell_back = 1;
  }
  int32_t nc = 0;
  for (int32_t t = 0; t < m; ++t) if (colour[t] + 1 > nc) nc = colour[t] + 1;
  stats[0] = m; stats[1] = nc; stats[2] = restarts; stats[3] = fell_back; stats[4] = last_conflicts; stats[5] = nbottom;
  free(fake.v); free(sig_off);
  return 0;
}
