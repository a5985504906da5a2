"""Pins of the oracle inspector (Algorithms 1-3) against the paper's worked examples, the
definition of legality (Section 4) and exact integer replay of tiled schedules."""
import os

import numpy as np
import pytest

import synth
from oracle import inspector as I
from oracle import checker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    for x, y in rows:
        assert I.splitmix64(int(x, 16)) == int(y, 16)


def test_hilbert_curve_is_a_continuous_bijection():
    # order-1 digit layout and, for orders 2..5, every cell visited once with unit steps
    assert [I.hilbert_index(x, y, 1) for (x, y) in [(0, 0), (0, 1), (1, 1), (1, 0)]] == [0, 1, 2, 3]
    for order in range(2, 6):
        n = 1 << order
        pos = {}
        for x in range(n):
            for y in range(n):
                pos[I.hilbert_index(x, y, order)] = (x, y)
        assert sorted(pos) == list(range(n * n))
        for d in range(n * n - 1):
            (x0, y0), (x1, y1) = pos[d], pos[d + 1]
            assert abs(x0 - x1) + abs(y0 - y1) == 1
        assert pos[0] == (0, 0) and pos[n * n - 1] == (n - 1, 0)


def test_inverse_map_example():
    # Figure of Section 5.1.4: cell 1 touches vertices 3, 7 and 9; the inverse lists cell 1 in
    # the rows of vertices 3, 7 and 9, rows delimited by offset[v], offset[v+1].
    c2v = np.array([[0, 1, 2], [3, 7, 9], [2, 3, 4], [9, 8, 7]], dtype=np.int32)
    off, val = I.map_invert(c2v.ravel(), 3, 10)
    rows = {v: list(val[off[v]:off[v + 1]]) for v in range(10)}
    for v in (3, 7, 9):
        assert 1 in rows[v]
    assert rows[7] == [1, 3] and rows[9] == [1, 3] and rows[3] == [1, 2] and rows[5] == []
    assert off[-1] == 12


def _wheel_chain():
    """The running example's chain (Figure 2): L0 edges increment vertices, L1 cells increment
    vertices, L2 edges read vertices; on a wheel of 7 triangles around vertex v0."""
    spokes = [(0, k) for k in range(1, 8)]
    ring = [(k, k % 7 + 1) for k in range(1, 8)]          # ring[k-1] joins v_k and v_{k+1}
    # edge numbering: tile 0 = edges 0..6, tile 1 = edges 7..13 (ts = 7)
    edges = [spokes[0], spokes[1], ring[0], ring[1], ring[6], ring[2], ring[5],
             spokes[2], spokes[3], spokes[4], spokes[5], spokes[6], ring[3], ring[4]]
    cells = [(0, k, k % 7 + 1) for k in range(1, 8)]       # cell c_{k-1} = (v0, v_k, v_{k+1})
    ch = I.Chain()
    E, C, V = ch.set("edges", 14), ch.set("cells", 7), ch.set("verts", 8)
    e2v = ch.map(E, V, 2, np.array(edges))
    c2v = ch.map(C, V, 3, np.array(cells))
    ch.loop(E, [(-1, "r"), (e2v, "i")])
    ch.loop(C, [(-1, "r"), (c2v, "i")])
    ch.loop(E, [(-1, "w"), (e2v, "r")])
    return ch, edges, cells


def test_worked_example_projection_and_tiling():
    # Section 3.2: with green = colour 0 before blue = colour 1, vertex v0 with 2 incident edges
    # in the green tile and 5 in the blue tile projects to the blue tile, and the cell with
    # vertex tiles (blue, green, green) is tiled into the blue tile.
    ch, edges, cells = _wheel_chain()
    s = I.inspect(ch, 7, sequential=True)
    assert list(s["colour"]) == [0, 1]
    inc = [e for e, (a, b) in enumerate(edges) if 0 in (a, b)]
    assert sorted(int(s["sigma"][0][e]) for e in inc) == [0, 0, 1, 1, 1, 1, 1]
    c1 = cells.index((0, 1, 2))
    assert s["sigma"][1][c1] == 1                 # MAX(B, G, G) = B
    assert s["restarts"] == 0
    assert checker.check(ch, s["sigma"], s["colour"]) == []


def _strip_chain(nedges=8, nloops=3):
    """Edges of a 1-D path, every loop increments both end vertices of its edges."""
    ch = I.Chain()
    E, V = ch.set("edges", nedges), ch.set("verts", nedges + 1)
    e2v = ch.map(E, V, 2, np.array([(i, i + 1) for i in range(nedges)]))
    for _ in range(nloops):
        ch.loop(E, [(-1, "r"), (e2v, "i")])
    return ch


def test_conflicting_colours_are_detected_and_repaired():
    # Section 3.2, "Conflicting Colors": with two colours alternating along a strip of
    # two-edge tiles, same-colour tiles grow towards each other until they touch a common
    # vertex.  Some priority seeds 2-colour the strip; for those the first round conflicts,
    # the unrepaired schedule is illegal, and backtracking with fake edges repairs it.
    ch = _strip_chain()
    seen = 0
    for seed in range(64):
        first = I.inspect(ch, 2, prio_seed=seed, max_rounds=-1)
        fixed = I.inspect(ch, 2, prio_seed=seed)
        assert checker.check(ch, fixed["sigma"], fixed["colour"]) == []
        if first["conflicts"]:
            seen += 1
            assert checker.check(ch, first["sigma"], first["colour"]) != []
            assert fixed["restarts"] >= 1
        else:
            assert checker.check(ch, first["sigma"], first["colour"]) == []
    assert seen > 0


def test_sequential_colouring_never_conflicts_and_one_tile_is_untiled():
    m = synth.make_mesh(8, 6, seed=2)
    ch, xy, _, _ = I.elastic_chain(m)
    s = I.inspect(ch, 5, sequential=True, renumber=True, xy=xy)
    assert s["restarts"] == 0 and list(s["colour"]) == list(range(s["ntiles"]))
    assert checker.check(ch, s["sigma"], s["colour"]) == []
    one = I.inspect(ch, 10 ** 6)
    assert one["ntiles"] == 1 and all(np.all(x == 0) for x in one["sigma"])


@pytest.mark.parametrize("ts", [1, 2, 3, 7, 16, 40, 1000])
@pytest.mark.parametrize("renumber", [False, True])
def test_elastic_schedules_are_legal(ts, renumber):
    m = synth.make_mesh(6, 5, seed=ts)
    ch, xy, _, _ = I.elastic_chain(m)
    for lo, hi in ((0, 9), (9, 17), (0, 17)):
        sub = ch.sub(lo, hi)
        s = I.inspect(sub, ts, renumber=renumber, xy=xy, prio_seed=ts * 7 + lo)
        assert checker.check(sub, s["sigma"], s["colour"]) == []
        for j, (ptr, its) in enumerate(s["lists"]):
            assert np.array_equal(np.sort(its), np.arange(len(s["sigma"][j])))
            for t in range(s["ntiles"]):
                seg = its[ptr[t]:ptr[t + 1]]
                assert np.all(np.diff(seg) > 0) and np.all(s["sigma"][j][seg] == t)


def _random_chain(rng, nloops):
    ch = I.Chain()
    sizes = rng.integers(5, 30, size=3)
    S = [ch.set("s%d" % k, int(sizes[k])) for k in range(3)]
    maps = []
    for _ in range(4):
        a, b = (int(x) for x in rng.permutation(3)[:2])   # maps join distinct sets
        ar = int(rng.integers(1, 4))
        maps.append(ch.map(int(a), int(b), ar, rng.integers(0, sizes[b], size=sizes[a] * ar)))
    for _ in range(nloops):
        s = int(rng.integers(0, 3))
        own = [m for m in maps if ch.maps[m][0] == s]
        descs = [(-1, "r")]
        wset = None
        if own and rng.random() < 0.7:
            m = own[int(rng.integers(len(own)))]
            descs.append((m, "i"))
            wset = ch.maps[m][1]
        else:
            descs.append((-1, "w" if rng.random() < 0.5 else "i"))
            wset = s
        for m in own:   # indirect reads of sets other than the one written indirectly
            if ch.maps[m][1] != wset and rng.random() < 0.5:
                descs.append((m, "r"))
        ch.loop(s, descs)
    return ch


def _replay(ch, order):
    """Run the chain with integer kernels: data[set] int64 per element; each iteration hashes
    what it reads, then writes (w) or adds (i) to what it writes.  `order` is a list of
    (loop, iteration) pairs.  Increments commute; everything else is order-sensitive."""
    data = [np.arange(n, dtype=np.int64) * 1000003 + 17 * (k + 1) for k, n in enumerate(ch.set_size)]
    M = 2 ** 61 - 1
    for (j, e) in order:
        s, descs, _ = ch.loops[j]
        h = (j + 1) * 0x9E3779B1 + e
        for (mid, mode) in descs:
            if mode != "r":
                continue
            if mid < 0:
                h = (h * 31 + int(data[s][e])) % M
            else:
                frm, to, a, vals = ch.maps[mid]
                for k in range(a):
                    h = (h * 37 + int(data[to][vals[e * a + k]]) * (k + 1)) % M
        for (mid, mode) in descs:
            if mode == "r":
                continue
            if mid < 0:
                data[s][e] = h if mode == "w" else (int(data[s][e]) + h) % M
            else:
                frm, to, a, vals = ch.maps[mid]
                for k in range(a):
                    t = vals[e * a + k]
                    data[to][t] = (int(data[to][t]) + h * (k + 1)) % M
    return data


@pytest.mark.parametrize("seed", range(40))
def test_tiled_replay_equals_untiled_chain(seed):
    # Sparse tiling changes only the order of iterations (Section 1): replaying the schedule
    # (colours ascending, same-colour tiles in a random order, each tile loop by loop) gives
    # exactly the same integers as the loop-by-loop chain.
    rng = np.random.default_rng(seed)
    ch = _random_chain(rng, int(rng.integers(2, 6)))
    ts = int(rng.integers(1, 8))
    s = I.inspect(ch, ts, prio_seed=seed)
    assert checker.check(ch, s["sigma"], s["colour"]) == []
    ref = _replay(ch, [(j, e) for j in range(len(ch.loops)) for e in range(ch.set_size[ch.loops[j][0]])])
    order = []
    for c in range(s["ncolours"]):
        tiles = [t for t in range(s["ntiles"]) if s["colour"][t] == c]
        rng.shuffle(tiles)
        for t in tiles:
            for j, (ptr, its) in enumerate(s["lists"]):
                order += [(j, int(e)) for e in its[ptr[t]:ptr[t + 1]]]
    out = _replay(ch, order)
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)


def test_local_maps_address_each_tile_footprint():
    m = synth.make_mesh(6, 6, seed=9)
    ch, xy, _, _ = I.elastic_chain(m)
    s = I.inspect(ch.sub(0, 9), 8, renumber=True, xy=xy)
    sub = ch.sub(0, 9)
    for j, per in enumerate(s["local_maps"]):
        for d, lm in enumerate(per):
            if lm is None:
                continue
            fp_ptr, fp, lmap = lm
            mid = sub.loops[j][1][d][0]
            a, vals = sub.maps[mid][2], sub.maps[mid][3]
            for e in range(len(s["sigma"][j])):
                t = s["sigma"][j][e]
                seg = fp[fp_ptr[t]:fp_ptr[t + 1]]
                assert np.all(np.diff(seg) > 0)
                for k in range(a):
                    assert seg[lmap[e * a + k]] == vals[e * a + k]


# ---------------------------------------------------------------- backward tiling (Section 5.1.1)

def test_backward_tiling_worked_line_example():
    # A path of 8 vertices and 7 edges.  Loop 0 increments both end vertices of every edge,
    # loop 1 (the seed) writes every vertex, loop 2 reads the end vertices of every edge and
    # writes the edge.  Seed tiles of 4 vertices, sequential colours: tile 0 = {0..3},
    # tile 1 = {4..7}.  Backward (MIN): edge (3, 4) touches vertices of tiles 0 and 1 and must
    # run in the earlier tile 0.  Forward (MAX, over loops 0 and 1): edge (3, 4) reads vertex
    # 4, last written by tile 1, so loop 2's edge 3 runs in tile 1.
    ch = I.Chain()
    E, V = ch.set("edges", 7), ch.set("verts", 8)
    e2v = ch.map(E, V, 2, np.array([(i, i + 1) for i in range(7)]))
    ch.loop(E, [(-1, "r"), (e2v, "i")])
    ch.loop(V, [(-1, "w")])
    ch.loop(E, [(-1, "w"), (e2v, "r")])
    s = I.inspect(ch, 4, sequential=True, seed=1)
    assert list(s["colour"]) == [0, 1]
    assert list(s["sigma"][1]) == [0, 0, 0, 0, 1, 1, 1, 1]
    assert list(s["sigma"][0]) == [0, 0, 0, 0, 1, 1, 1]
    assert list(s["sigma"][2]) == [0, 0, 0, 1, 1, 1, 1]
    assert s["restarts"] == 0 and s["unprojected"] == 0
    assert checker.check(ch, s["sigma"], s["colour"]) == []
    # seeded at loop 0 instead, the edges are partitioned ({0..3}, {4..6}) and vertex 4, which
    # edge 4 of tile 1 increments, is written by tile 1 in loop 1 (MAX)
    f = I.inspect(ch, 4, sequential=True)
    assert list(f["sigma"][0]) == [0, 0, 0, 0, 1, 1, 1]
    assert list(f["sigma"][1]) == [0, 0, 0, 0, 1, 1, 1, 1]


def test_backward_conflicts_are_detected_and_repaired():
    # the strip of Section 3.2 seeded at its last loop: same-colour tiles grow backwards towards
    # each other; the MIN rule must see those meetings as conflicts
    ch = _strip_chain(nedges=10, nloops=4)
    seen = 0
    for ps in range(64):
        first = I.inspect(ch, 2, prio_seed=ps, max_rounds=-1, seed=3)
        fixed = I.inspect(ch, 2, prio_seed=ps, seed=3)
        assert checker.check(ch, fixed["sigma"], fixed["colour"]) == []
        if first["conflicts"]:
            seen += 1
            assert checker.check(ch, first["sigma"], first["colour"]) != []
        else:
            assert checker.check(ch, first["sigma"], first["colour"]) == []
    assert seen > 0


@pytest.mark.parametrize("ts", [1, 3, 8, 40])
@pytest.mark.parametrize("seed_loop", [1, 4, 8])
def test_backward_elastic_schedules_are_legal(ts, seed_loop):
    m = synth.make_mesh(6, 5, seed=ts + seed_loop)
    ch, xy, _, _ = I.elastic_chain(m)
    sub = ch.sub(0, 9)
    pts = ch.points[sub.loops[seed_loop][0]]
    s = I.inspect(sub, ts, renumber=True, xy=pts, prio_seed=ts * 11 + seed_loop, seed=seed_loop)
    assert checker.check(sub, s["sigma"], s["colour"]) == []
    assert s["rank"].shape == (sub.set_size[sub.loops[seed_loop][0]],)


@pytest.mark.parametrize("seed", range(40))
def test_backward_tiled_replay_equals_untiled_chain(seed):
    rng = np.random.default_rng(1000 + seed)
    ch = _random_chain(rng, int(rng.integers(2, 7)))
    ts = int(rng.integers(1, 8))
    sl = int(rng.integers(0, len(ch.loops)))
    s = I.inspect(ch, ts, prio_seed=seed, seed=sl)
    assert checker.check(ch, s["sigma"], s["colour"]) == []
    ref = _replay(ch, [(j, e) for j in range(len(ch.loops)) for e in range(ch.set_size[ch.loops[j][0]])])
    order = []
    for c in range(s["ncolours"]):
        tiles = [t for t in range(s["ntiles"]) if s["colour"][t] == c]
        rng.shuffle(tiles)
        for t in tiles:
            for j, (ptr, its) in enumerate(s["lists"]):
                order += [(j, int(e)) for e in its[ptr[t]:ptr[t + 1]]]
    out = _replay(ch, order)
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)


def _export_brute(ch, sig):
    # the definition, access by access: iteration i of loop j is flagged when some element it
    # writes or increments is read or written by an iteration of another tile in any loop
    acc = []   # (set, element, tile) of every access
    for j, (s, descs, _) in enumerate(ch.loops):
        for i in range(ch.set_size[s]):
            for (mid, mode) in descs:
                if mid < 0:
                    acc.append((s, i, int(sig[j][i])))
                else:
                    frm, to, a, vals = ch.maps[mid]
                    for k in range(a):
                        acc.append((to, int(vals[i * a + k]), int(sig[j][i])))
    out = []
    for j, (s, descs, _) in enumerate(ch.loops):
        f = np.zeros(ch.set_size[s], dtype=np.int32)
        for i in range(ch.set_size[s]):
            t = int(sig[j][i])
            written = []
            for (mid, mode) in descs:
                if mode == "r":
                    continue
                if mid < 0:
                    written.append((s, i))
                else:
                    frm, to, a, vals = ch.maps[mid]
                    written += [(to, int(vals[i * a + k])) for k in range(a)]
            f[i] = any((x[0], x[1]) == w and x[2] != t for w in written for x in acc)
        out.append(f)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_export_flags_match_the_access_by_access_definition(seed):
    rng = np.random.default_rng(100 + seed)
    ch = _random_chain(rng, int(rng.integers(2, 5)))
    ts = int(rng.integers(1, 8))
    s = I.inspect(ch, ts, prio_seed=seed)
    for a, b in zip(I.export_flags(ch, s["sigma"]), _export_brute(ch, s["sigma"])):
        assert np.array_equal(a, b)


def test_export_flags_worked_cases():
    # one tile: nothing is exported
    ch = _strip_chain()
    s = I.inspect(ch, 100)
    assert all(not f.any() for f in I.export_flags(ch, s["sigma"]))
    # a strip of 8 edges in tiles of 4 edges (edges 0-3 and 4-7, every loop incrementing both end
    # vertices): only the edges at vertex 4, where the tiles meet, write a vertex the other tile
    # touches - edge 3 (vertices 3, 4) and edge 4 (vertices 4, 5)
    ch = _strip_chain(8, 1)
    sig = [np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.int32)]
    assert list(I.export_flags(ch, sig)[0]) == [0, 0, 0, 1, 1, 0, 0, 0]
    # a read-only loop exports nothing; a write through a direct access of a set touched by one
    # tile per element exports nothing either
    ch = I.Chain()
    E, V = ch.set("edges", 4), ch.set("verts", 5)
    e2v = ch.map(E, V, 2, np.array([(i, i + 1) for i in range(4)]))
    ch.loop(E, [(-1, "w"), (e2v, "r")])
    ch.loop(E, [(e2v, "r")])
    sig = [np.array([0, 0, 1, 1], dtype=np.int32)] * 2
    f = I.export_flags(ch, sig)
    assert not f[0].any() and not f[1].any()
