"""ORACLE (test infrastructure only).  Loop-chain description, the sequential inspector of
Algorithms 1-3 (inspector.c, loaded through ctypes) and the derived per-tile structures.

A loop chain (Section 2) is a list of sets (iteration spaces), maps between sets (flat arrays
map[i*arity + k]) and loops, each loop being a set plus descriptors (map or None for a direct
access, mode 'r', 'w' or 'i').  `elastic_chain` builds the seventeen-loop chain of one time
step of the DG elastic-wave solver from a mesh, on its own (facet extraction included).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_inspector.so")


def build():
    """Compile inspector.c with gcc into oracle/_build/ (idempotent)."""
    src = os.path.join(_HERE, "inspector.c")
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.oracle_inspect.restype = ctypes.c_int
        _lib.oracle_inspect.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, P, ctypes.c_int, P, P, P, P,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P, ctypes.c_int,
                                        ctypes.c_int, P, P, P, P]
        _lib.oracle_hilbert_index.restype = ctypes.c_uint32
        _lib.oracle_hilbert_index.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int]
        _lib.oracle_splitmix64.restype = ctypes.c_uint64
        _lib.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        _lib.oracle_map_invert.argtypes = [ctypes.c_int64, ctypes.c_int, P, ctypes.c_int64, P, P]
        _lib.oracle_seed_rank.argtypes = [ctypes.c_int64, ctypes.c_int, P, P]
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Chain:
    """Sets, maps and loops of a loop chain, in the order they are declared."""

    def __init__(self):
        self.set_size, self.set_name = [], []
        self.maps = []    # (from, to, arity, int32 values)
        self.loops = []   # (set, [(map id or -1, mode)], name)

    def set(self, name, size):
        self.set_name.append(name)
        self.set_size.append(int(size))
        return len(self.set_size) - 1

    def map(self, frm, to, arity, values):
        v = np.ascontiguousarray(values, dtype=np.int32).ravel()
        if v.size != self.set_size[frm] * arity:
            raise ValueError("map size")
        if v.size and (v.min() < 0 or v.max() >= self.set_size[to]):
            raise ValueError("map value out of range")
        self.maps.append((frm, to, arity, v))
        return len(self.maps) - 1

    def loop(self, set_id, descs, name=""):
        self.loops.append((set_id, list(descs), name))
        return len(self.loops) - 1

    def sub(self, start, stop):
        c = Chain()
        c.set_size, c.set_name, c.maps = self.set_size, self.set_name, self.maps
        c.points = getattr(self, "points", {})
        c.loops = self.loops[start:stop]
        return c


# the seventeen loops of one time step, as (set, kernel name, descriptor pattern)
# v-chain: volB intB extB volD intD hookeB intB extB updV ; s-chain: volD intD hookeB intB extB volD intD updS
ELASTIC_LOOPS = [
    ("cells", "volB"), ("ifacets", "intB"), ("efacets", "extB"), ("cells", "volD"), ("ifacets", "intD"),
    ("cells", "hookeB"), ("ifacets", "intB"), ("efacets", "extB"), ("cells", "updV"),
    ("cells", "volD"), ("ifacets", "intD"), ("cells", "hookeB"), ("ifacets", "intB"), ("efacets", "extB"),
    ("cells", "volD"), ("ifacets", "intD"), ("cells", "updS"),
]
ELASTIC_SPLIT = 9   # the velocity sub-chain is loops 0..8, the stress sub-chain 9..16


def elastic_chain(mesh):
    """The DG elastic time step as a loop chain over cells, interior and exterior facets.

    Interior facet loops read and increment cell data through facet->cell (arity 2),
    exterior facet loops through facet->cell (arity 1), cell loops access cells directly;
    update loops increment the prognostic fields.  Also returns the seed points (cell
    centroids ((x0 + x1) + x2) / 3) used by the Hilbert renumbering."""
    from .dg import _facets
    c2v = np.asarray(mesh["cell2vert"])
    inter, exter = _facets(c2v)
    ch = Chain()
    C = ch.set("cells", c2v.shape[0])
    F = ch.set("ifacets", inter.shape[0])
    E = ch.set("efacets", exter.shape[0])
    f2c = ch.map(F, C, 2, np.stack([inter[:, 0], inter[:, 2]], 1))
    e2c = ch.map(E, C, 1, exter[:, 0])
    sets = {"cells": C, "ifacets": F, "efacets": E}
    for sname, kname in ELASTIC_LOOPS:
        if sname == "cells":
            mode = "i" if kname.startswith("upd") else "w"
            ch.loop(C, [(-1, "r"), (-1, mode)], kname)
        else:
            m = f2c if sname == "ifacets" else e2c
            ch.loop(sets[sname], [(m, "r"), (m, "i")], kname)
    X = np.asarray(mesh["cellxy"], dtype=np.float64)
    xy = np.stack([((X[:, 0, 0] + X[:, 1, 0]) + X[:, 2, 0]) / 3.0, ((X[:, 0, 1] + X[:, 1, 1]) + X[:, 2, 1]) / 3.0], 1)
    ch.points = {C: np.ascontiguousarray(xy),
                 F: _midpoints(X, inter[:, 0], inter[:, 1]), E: _midpoints(X, exter[:, 0], exter[:, 1])}
    return ch, np.ascontiguousarray(xy), inter, exter


def _midpoints(X, cells, faces):
    """(x_a + x_b) * 0.5 of local face f (vertices f, f+1) of each given cell."""
    a = X[cells, faces]
    b = X[cells, (faces + 1) % 3]
    return np.ascontiguousarray((a + b) * 0.5)


def inspect(chain, ts, sequential=False, prio_seed=0x5EED, renumber=False, xy=None, max_rounds=16, seed=0,
            with_local_maps=True):
    """Run Algorithm 1 on `chain` with seed loop `seed` (0: forward tiling from the first loop;
    > 0: backward tiling, MIN projections, for the loops before it).  Returns a dict with
    rank, colour, sigma (list, one tiling function per loop), stats, lists and (unless
    with_local_maps is false) local maps.  xy: points of the seed loop's set (renumber)."""
    lib = _load()
    nsets = len(chain.set_size)
    set_size = np.array(chain.set_size, dtype=np.int64)
    mf = np.array([m[0] for m in chain.maps], dtype=np.int32)
    mt = np.array([m[1] for m in chain.maps], dtype=np.int32)
    ma = np.array([m[2] for m in chain.maps], dtype=np.int32)
    mv = (ctypes.c_void_p * max(len(chain.maps), 1))(*[m[3].ctypes.data for m in chain.maps])
    ls = np.array([l[0] for l in chain.loops], dtype=np.int32)
    dptr = np.cumsum([0] + [len(l[1]) for l in chain.loops]).astype(np.int32)
    dmap = np.array([d[0] for l in chain.loops for d in l[1]], dtype=np.int32)
    dmode = np.frombuffer("".join(d[1] for l in chain.loops for d in l[1]).encode(), dtype=np.uint8).copy()
    seed_set = chain.loops[seed][0]
    nseed = set_size[seed_set]
    if renumber:
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        if xy.shape != (nseed, 2):
            raise ValueError("seed points")
    sizes = [int(set_size[l[0]]) for l in chain.loops]
    rank = np.zeros(nseed, dtype=np.int32)
    m = (nseed + ts - 1) // ts if ts > 0 else 0
    colour = np.zeros(max(m, 1), dtype=np.int32)
    sigma = np.zeros(sum(sizes), dtype=np.int32)
    stats = np.zeros(6, dtype=np.int64)
    rc = lib.oracle_inspect(nsets, _ptr(set_size), len(chain.maps), _ptr(mf), _ptr(mt), _ptr(ma),
                            ctypes.cast(mv, ctypes.c_void_p), len(chain.loops), _ptr(ls), _ptr(dptr), _ptr(dmap),
                            _ptr(dmode), int(ts), int(bool(sequential)), ctypes.c_uint64(prio_seed),
                            int(bool(renumber)), _ptr(xy) if renumber else None, int(max_rounds), int(seed),
                            _ptr(rank), _ptr(colour), _ptr(sigma), _ptr(stats))
    if rc != 0:
        raise ValueError("oracle_inspect failed (%d)" % rc)
    offs = np.cumsum([0] + sizes)
    sig = [sigma[offs[j]:offs[j + 1]] for j in range(len(sizes))]
    out = dict(rank=rank, colour=colour[:m], sigma=sig, ntiles=int(stats[0]), ncolours=int(stats[1]),
               restarts=int(stats[2]), fell_back=bool(stats[3]), conflicts=int(stats[4]), unprojected=int(stats[5]))
    out["lists"] = [iteration_lists(s, m) for s in sig]
    if with_local_maps:
        out["local_maps"] = local_maps(chain, sig, m)
    return out


def iteration_lists(sig, m):
    """assign: the iterations of each tile in ascending order, as CSR (tile_ptr[m+1], iters)."""
    order = np.argsort(sig, kind="stable").astype(np.int32)
    ptr = np.zeros(m + 1, dtype=np.int32)
    ptr[1:] = np.cumsum(np.bincount(sig, minlength=m))
    return ptr, order


def local_maps(chain, sig, m):
    """compute_local_maps: for every loop and indirect descriptor, each tile's footprint (the
    sorted distinct target elements its iterations touch, CSR fp_ptr[m+1], fp) and the local
    map lmap[i*arity + k] = position of map[i*arity + k] in the footprint of tile sigma[i]."""
    out = []
    for j, (s, descs, _) in enumerate(chain.loops):
        per = []
        for (mid, mode) in descs:
            if mid < 0:
                per.append(None)
                continue
            frm, to, a, vals = chain.maps[mid]
            tile_of_slot = np.repeat(sig[j], a).astype(np.int64)
            key = tile_of_slot * (chain.set_size[to] + 1) + vals
            uniq = np.unique(key)
            fp_tile = (uniq // (chain.set_size[to] + 1)).astype(np.int64)
            fp = (uniq % (chain.set_size[to] + 1)).astype(np.int32)
            fp_ptr = np.zeros(m + 1, dtype=np.int32)
            fp_ptr[1:] = np.cumsum(np.bincount(fp_tile, minlength=m))
            lmap = (np.searchsorted(uniq, key) - fp_ptr[tile_of_slot]).astype(np.int32)
            per.append((fp_ptr, fp, lmap))
        out.append(per)
    return out


def export_flags(chain, sig):
    """The export flag of every iteration of every loop (the per-tile data of Algorithm 1's
    compute_local_maps): 1 when an element that the iteration writes or increments (mode 'w' or
    'i') is also accessed, in some loop of the chain, by a tile other than the iteration's own,
    i.e. a value its tile must hand to another tile rather than keep local.  sig: one tiling
    function per loop.  Returns one int32 array per loop."""
    # every access of the chain as (set, tile, element)
    acc = {}
    for j, (s, descs, _) in enumerate(chain.loops):
        n = chain.set_size[s]
        for (mid, mode) in descs:
            if mid < 0:
                tgt, tiles, elems = s, sig[j].astype(np.int64), np.arange(n, dtype=np.int64)
            else:
                frm, tgt, a, vals = chain.maps[mid]
                tiles, elems = np.repeat(sig[j], a).astype(np.int64), vals.astype(np.int64)
            acc.setdefault(tgt, []).append((tiles, elems))
    # distinct tiles per element
    ntiles = {}
    for tgt, parts in acc.items():
        tiles = np.concatenate([p[0] for p in parts])
        elems = np.concatenate([p[1] for p in parts])
        span = int(tiles.max()) + 1 if tiles.size else 1
        pairs = np.unique(elems * span + tiles)          # each (element, tile) once
        ntiles[tgt] = np.bincount(pairs // span, minlength=chain.set_size[tgt])
    out = []
    for j, (s, descs, _) in enumerate(chain.loops):
        n = chain.set_size[s]
        f = np.zeros(n, dtype=bool)
        for (mid, mode) in descs:
            if mode == "r":
                continue
            if mid < 0:
                f |= ntiles[s] > 1
            else:
                frm, tgt, a, vals = chain.maps[mid]
                f |= (ntiles[tgt][vals] > 1).reshape(n, a).any(axis=1)
        out.append(f.astype(np.int32))
    return out


def map_invert(values, arity, ntgt):
    lib = _load()
    v = np.ascontiguousarray(values, dtype=np.int32)
    nsrc = v.size // arity
    off = np.zeros(ntgt + 1, dtype=np.int64)
    val = np.zeros(max(v.size, 1), dtype=np.int32)
    lib.oracle_map_invert(nsrc, arity, _ptr(v), ntgt, _ptr(off), _ptr(val))
    return off, val[:v.size]


def hilbert_index(x, y, order=16):
    return int(_load().oracle_hilbert_index(int(x), int(y), int(order)))


def splitmix64(x):
    return int(_load().oracle_splitmix64(ctypes.c_uint64(x)))


def seed_rank(xy):
    lib = _load()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    rank = np.zeros(xy.shape[0], dtype=np.int32)
    lib.oracle_seed_rank(xy.shape[0], 1, _ptr(xy), _ptr(rank))
    return rank
