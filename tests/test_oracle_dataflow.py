"""The dataflow executor's ordering rule, checked on the CPU with the oracle inspector and exact
integer replay.  A node is a (time step, sub-chain, tile) triple; it waits for the lower-colour tiles
of its sub-chain that touch one of its elements, and for the previous sub-chain's tiles (the last
sub-chain of the previous step, for the first) that touched them.  Any order that respects these
waits, steps overlapping included, must give exactly the integers of the loop-by-loop chain run step
after step (Algorithm 4 runs one such order: colours in turn, sub-chains in turn, steps in turn)."""
import numpy as np
import pytest

import synth
from oracle import inspector as I

M61 = 2 ** 61 - 1
# the elastic chain's fields per loop: (fields read, fields written, increment?); facet loops read at
# both cells of the facet and increment both, cell loops read and assign at their cell (the updates
# read the field they assign)
FIELDS = [
    ("S", "U1", False), ("S", "U1", True), ("S", "U1", True), ("U1", "E", False), ("U1", "E", True),
    ("E", "S1 U2", False), ("S1", "U2", True), ("S1", "U2", True), ("U1 U2 V", "V", False),
    ("V", "E", False), ("V", "E", True), ("E", "S1 U1", False), ("S1", "U1", True), ("S1", "U1", True),
    ("U1", "E", False), ("U1", "E", True), ("E S1 S", "S", False),
]


def _replay_fields(mesh_facets, nc, order):
    """Integer model of the chain: one int64 per cell and field.  A facet iteration hashes the
    fields it reads at both cells and adds to the written field of both (increments commute); a
    cell iteration hashes its own cell's fields and assigns.  Any reordering of dependent
    iterations changes the integers."""
    inter, exter = mesh_facets
    data = {f: (np.arange(nc, dtype=np.int64) * 1000003 + 17 * (i + 1)) % M61
            for i, f in enumerate(("S", "U1", "E", "S1", "U2", "V"))}
    for (j, e) in order:
        reads, writes, inc = FIELDS[j]
        reads, writes = reads.split(), writes.split()
        kind = I.ELASTIC_LOOPS[j][0]
        cells = [int(inter[e, 0]), int(inter[e, 2])] if kind == "ifacets" else (
            [int(exter[e, 0])] if kind == "efacets" else [e])
        h = (j + 1) * 0x9E3779B1 + e
        for f in reads:
            for c in cells:
                h = (h * 31 + int(data[f][c])) % M61
        for k, c in enumerate(cells):
            for w, f in enumerate(writes):
                v = (h * (k + 1) * (w + 3)) % M61
                data[f][c] = (int(data[f][c]) + v) % M61 if inc else v
    return [data[f] for f in sorted(data)]


def _touched(ch, j, e):
    s, descs, _ = ch.loops[j]
    out = set()
    for mid, _mode in descs:
        if mid < 0:
            out.add((s, e))
        else:
            _frm, to, a, vals = ch.maps[mid]
            out.update((to, int(vals[e * a + k])) for k in range(a))
    return out


def _schedule(ch, bounds, ts):
    subs = []
    for lo, hi in bounds:
        s = I.inspect(ch.sub(lo, hi), ts, renumber=True, xy=ch.points[ch.loops[lo][0]])
        touch = {}  # element -> tiles of this sub-chain touching it
        for jj, (ptr, its) in enumerate(s["lists"]):
            for t in range(s["ntiles"]):
                for e in its[ptr[t]:ptr[t + 1]]:
                    for el in _touched(ch, lo + jj, int(e)):
                        touch.setdefault(el, set()).add(t)
        subs.append(dict(lo=lo, s=s, touch=touch))
    return subs


def _dependencies(subs, colour_order=True, across=True):
    """deps[(k, t)] = set of ((k', t'), wrap): wrap = 1 when the dependency is the previous step's."""
    K = len(subs)
    deps = {(k, t): set() for k in range(K) for t in range(subs[k]["s"]["ntiles"])}
    elements = set().union(*(sb["touch"].keys() for sb in subs))
    for el in elements:
        seq = [k for k in range(K) if el in subs[k]["touch"]]
        for i, k in enumerate(seq):
            col = subs[k]["s"]["colour"]
            tiles = subs[k]["touch"][el]
            prev, wrap = (seq[i - 1], 0) if i else (seq[-1], 1)
            for b in tiles:
                if colour_order:
                    deps[(k, b)].update(((k, a), 0) for a in tiles if col[a] < col[b])
                if across:
                    deps[(k, b)].update(((prev, a), wrap) for a in subs[prev]["touch"][el])
    return deps


def _random_order(subs, deps, nsteps, rng):
    """A random linear extension of the time-expanded graph (Kahn's algorithm, random ready node)."""
    nodes = [(st, k, t) for st in range(nsteps) for (k, t) in deps]
    preds = {}
    for (st, k, t) in nodes:
        ps = set()
        for (k2, t2), wrap in deps[(k, t)]:
            s2 = st - wrap
            if s2 >= 0:
                ps.add((s2, k2, t2))
        preds[(st, k, t)] = ps
    succ = {n: [] for n in nodes}
    for n, ps in preds.items():
        for p in ps:
            succ[p].append(n)
    count = {n: len(ps) for n, ps in preds.items()}
    ready = [n for n in nodes if count[n] == 0]
    order = []
    while ready:
        n = ready.pop(int(rng.integers(len(ready))))
        order.append(n)
        for m in succ[n]:
            count[m] -= 1
            if count[m] == 0:
                ready.append(m)
    assert len(order) == len(nodes), "the graph has a cycle"
    return order


def _iterations(subs, order):
    out = []
    for (_st, k, t) in order:
        sb = subs[k]
        for jj, (ptr, its) in enumerate(sb["s"]["lists"]):
            out += [(sb["lo"] + jj, int(e)) for e in its[ptr[t]:ptr[t + 1]]]
    return out


def _untiled(ch, nsteps):
    return [(j, e) for _ in range(nsteps) for j in range(len(ch.loops))
            for e in range(ch.set_size[ch.loops[j][0]])]


@pytest.mark.parametrize("split,ts", [((9,), 8), ((9,), 16), ((9,), 4), ((3, 9, 12), 8), ((), 12),
                                      ((1, 5, 9, 13), 6)])
@pytest.mark.parametrize("nx,ny,seed", [(6, 6, 9), (9, 7, 3)])
def test_any_order_the_dataflow_executor_allows_equals_the_chain(split, ts, nx, ny, seed):
    m = synth.make_mesh(nx, ny, seed=seed)
    ch, _, inter, exter = I.elastic_chain(m)
    nc = m["cell2vert"].shape[0]
    bounds = list(zip((0,) + split, split + (17,)))
    subs = _schedule(ch, bounds, ts)
    deps = _dependencies(subs)
    nsteps = 3
    ref = _replay_fields((inter, exter), nc, _untiled(ch, nsteps))
    rng = np.random.default_rng(ts + 100 * len(split) + seed)
    for _ in range(12):
        out = _replay_fields((inter, exter), nc, _iterations(subs, _random_order(subs, deps, nsteps, rng)))
        for a, b in zip(ref, out):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("drop", ["colour_order", "across"])
def test_dropping_either_kind_of_wait_breaks_the_result(drop):
    # the check is sharp: without the colour waits or without the waits across sub-chains and
    # steps, some allowed order differs from the chain
    m = synth.make_mesh(6, 6, seed=9)
    ch, _, inter, exter = I.elastic_chain(m)
    nc = m["cell2vert"].shape[0]
    bounds = [(0, 9), (9, 17)]
    subs = _schedule(ch, bounds, 8)
    deps = _dependencies(subs, **{drop: False})
    ref = _replay_fields((inter, exter), nc, _untiled(ch, 3))
    rng = np.random.default_rng(5)
    differs = False
    for _ in range(8):
        out = _replay_fields((inter, exter), nc, _iterations(subs, _random_order(subs, deps, 3, rng)))
        differs |= any(not np.array_equal(a, b) for a, b in zip(ref, out))
    assert differs


def _segment_items(ch, inter, exter, sub, t, a, b):
    """The items of tile t's segment [a, b): per cell, its share of each loop of the segment in loop
    order, as (loop, iteration, side) with side = the cell's place in the facet (0 for cell loops)."""
    items = {}
    ptrs = sub["s"]["lists"]
    for j in range(a, b):
        ptr, its = ptrs[j - sub["lo"]]
        kind = I.ELASTIC_LOOPS[j][0]
        for e in its[ptr[t]:ptr[t + 1]]:
            e = int(e)
            if kind == "cells":
                items.setdefault(e, []).append((j, e, 0))
            elif kind == "ifacets":
                items.setdefault(int(inter[e, 0]), []).append((j, e, 0))
                items.setdefault(int(inter[e, 2]), []).append((j, e, 1))
            else:
                items.setdefault(int(exter[e, 0]), []).append((j, e, 0))
    return items


def _replay_pull(mesh_facets, nc, ops):
    """The integer model with each facet iteration split into its two per-cell halves (the pull
    form): each half hashes the same reads and updates only its own cell."""
    inter, exter = mesh_facets
    data = {f: (np.arange(nc, dtype=np.int64) * 1000003 + 17 * (i + 1)) % M61
            for i, f in enumerate(("S", "U1", "E", "S1", "U2", "V"))}
    for (j, e, side) in ops:
        reads, writes, inc = FIELDS[j]
        reads, writes = reads.split(), writes.split()
        kind = I.ELASTIC_LOOPS[j][0]
        cells = [int(inter[e, 0]), int(inter[e, 2])] if kind == "ifacets" else (
            [int(exter[e, 0])] if kind == "efacets" else [e])
        h = (j + 1) * 0x9E3779B1 + e
        for f in reads:
            for c in cells:
                h = (h * 31 + int(data[f][c])) % M61
        c = cells[side]
        for w, f in enumerate(writes):
            v = (h * (side + 1) * (w + 3)) % M61
            data[f][c] = (int(data[f][c]) + v) % M61 if inc else v
    return [data[f] for f in sorted(data)]


@pytest.mark.parametrize("split,ts", [((9,), 8), ((3, 9, 12), 6), ((1, 5, 9, 13), 8)])
def test_segments_run_cell_by_cell_replay_the_chain(split, ts):
    # the tiled executors run each tile as segments (the part of each phase in the sub-chain): one
    # thread per touched cell takes it through the segment's loops, the cells of a segment in any
    # order.  With the phase table of the executors, any such run of any allowed tile order replays
    # the chain exactly.
    from tests.test_phases import phase_starts
    m = synth.make_mesh(7, 6, seed=11)
    ch, _, inter, exter = I.elastic_chain(m)
    nc = m["cell2vert"].shape[0]
    bounds = list(zip((0,) + split, split + (17,)))
    subs = _schedule(ch, bounds, ts)
    deps = _dependencies(subs)
    starts = phase_starts()
    nsteps = 2
    ref = _replay_fields((inter, exter), nc, _untiled(ch, nsteps))
    rng = np.random.default_rng(ts + 7 * len(split))
    for _ in range(6):
        ops = []
        for (_st, k, t) in _random_order(subs, deps, nsteps, rng):
            sub = subs[k]
            lo, hi = bounds[k]
            cuts = sorted({lo, hi} | {x for x in starts if lo < x < hi})
            for a, b in zip(cuts, cuts[1:]):
                items = list(_segment_items(ch, inter, exter, sub, t, a, b).values())
                rng.shuffle(items)
                for it in items:
                    ops += it
        out = _replay_pull((inter, exter), nc, ops)
        for x, y in zip(ref, out):
            assert np.array_equal(x, y)


def test_a_phase_that_reads_a_neighbour_value_it_writes_breaks_the_replay():
    # sharpness: cutting the chain into segments that run loop 5 (which writes S1) together with
    # loop 6 (which reads S1 across faces) makes some cell order differ from the chain
    m = synth.make_mesh(7, 6, seed=11)
    ch, _, inter, exter = I.elastic_chain(m)
    nc = m["cell2vert"].shape[0]
    bounds = [(0, 9), (9, 17)]
    subs = _schedule(ch, bounds, 8)
    ref = _replay_fields((inter, exter), nc, _untiled(ch, 1))
    rng = np.random.default_rng(3)
    bad = [0, 3, 9, 12, 14, 17]        # phase 1 widened to loops 3-8
    differs = False
    for _ in range(6):
        ops = []
        for k, sub in enumerate(subs):
            lo, hi = bounds[k]
            col = sub["s"]["colour"]
            cuts = sorted({lo, hi} | {x for x in bad if lo < x < hi})
            for c in range(sub["s"]["ncolours"]):
                for t in [t for t in range(sub["s"]["ntiles"]) if col[t] == c]:
                    for a, b in zip(cuts, cuts[1:]):
                        items = list(_segment_items(ch, inter, exter, sub, t, a, b).values())
                        rng.shuffle(items)
                        for it in items:
                            ops += it
        out = _replay_pull((inter, exter), nc, ops)
        differs |= any(not np.array_equal(x, y) for x, y in zip(ref, out))
    assert differs
