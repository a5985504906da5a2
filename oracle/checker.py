"""ORACLE (test infrastructure only).  Brute-force legality checker for a sparse-tiling schedule.

The executor (Algorithm 4) runs colours in ascending order, the tiles of one colour in any
order or concurrently, and inside a tile the loops in chain order.  Using the dependence
classes of Section 4 at the granularity of sets (flow, anti and output dependences between
loops, reductions inside a loop), a schedule is legal when, for every element of every set and
every pair of accesses to it by iterations of loops x <= y in different tiles, with at least one
of the two a write or an increment:
  - x < y  requires colour(tile of the x access) < colour(tile of the y access);
  - x == y (both writes or increments) requires the two colours to differ.
It also checks coverage: every iteration of every loop belongs to exactly one existing tile.
Pure Python loops: meant for tiny meshes and chains.
"""
from collections import defaultdict

import numpy as np


def check(chain, sigma, colour):
    """Return a list of violations (empty when the schedule is legal)."""
    bad = []
    m = len(colour)
    for j, (s, _, _) in enumerate(chain.loops):
        sj = np.asarray(sigma[j])
        if sj.shape != (chain.set_size[s],) or (sj.size and (sj.min() < 0 or sj.max() >= m)):
            bad.append(("coverage", j))
    if bad:
        return bad
    acc = defaultdict(list)   # (set, element) -> [(loop, tile, writes)]
    for j, (s, descs, _) in enumerate(chain.loops):
        sj = sigma[j]
        for (mid, mode) in descs:
            w = mode in ("w", "i")
            if mid < 0:
                for e in range(chain.set_size[s]):
                    acc[(s, e)].append((j, int(sj[e]), w))
            else:
                frm, to, a, vals = chain.maps[mid]
                for e in range(chain.set_size[s]):
                    for k in range(a):
                        acc[(to, int(vals[e * a + k]))].append((j, int(sj[e]), w))
    for key, lst in acc.items():
        n = len(lst)
        for p in range(n):
            x, tx, wx = lst[p]
            for q in range(n):
                y, ty, wy = lst[q]
                if tx == ty or not (wx or wy):
                    continue
                if x < y and not colour[tx] < colour[ty]:
                    bad.append(("order", key, x, tx, y, ty))
                elif x == y and wx and wy and colour[tx] == colour[ty]:
                    bad.append(("race", key, x, tx, ty))
    return bad
