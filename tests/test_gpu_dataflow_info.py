"""The dependency-graph figures of the dataflow executor (GPU inspector), recounted here from the
schedule's exported colours and tiling functions with the executor's ordering rule: inside a
sub-chain a tile follows the lower-colour tiles that touch one of its cells; across sub-chains it
follows the tiles of the previous sub-chain (the last one of the previous step for the first) that
touched the same cell."""
import numpy as np
import pytest

from oracle import inspector as OI
from tests.helpers import workload, gpu_mesh, gpu_run

pytestmark = pytest.mark.gpu


def _recount(lib, sched, cfg, bounds):
    _, _, inter, exter = OI.elastic_chain(cfg["mesh"])
    nc = cfg["mesh"]["cell2vert"].shape[0]
    K = len(bounds)
    cols, touch = [], []
    for k, (lo, hi) in enumerate(bounds):
        cols.append(lib.slt_schedule_export(sched, "colour", k))
        pairs = set()
        for J in range(lo, hi):
            sig = lib.slt_schedule_export(sched, "sigma", J)
            kind = OI.ELASTIC_LOOPS[J][0]
            if kind == "cells":
                pairs |= set(zip(range(nc), sig.tolist()))
            elif kind == "ifacets":
                pairs |= set(zip(inter[:, 0].tolist(), sig.tolist())) | set(zip(inter[:, 2].tolist(), sig.tolist()))
            else:
                pairs |= set(zip(exter[:, 0].tolist(), sig.tolist()))
        per_cell = [[] for _ in range(nc)]
        for c, t in pairs:
            per_cell[c].append(t)
        touch.append(per_cell)
    base = np.cumsum([0] + [len(c) for c in cols])
    deps = set()  # (node, dependency, from the previous step)
    for c in range(nc):
        for k in range(K):
            prev, wrap = (k - 1, 0) if k else (K - 1, 1)
            for b in touch[k][c]:
                for a in touch[k][c]:
                    if cols[k][a] < cols[k][b]:
                        deps.add((base[k] + b, base[k] + a, 0))
                for a in touch[prev][c]:
                    deps.add((base[k] + b, base[prev] + a, wrap))
    G = int(base[-1])
    by_node = [[] for _ in range(G)]
    for g, e, w in deps:
        by_node[g].append((e, w))
    order = sorted(range(G), key=lambda g: (np.searchsorted(base, g, side="right"), cols_of(cols, base, g)))
    prev_l, top = [0.0] * G, []
    for _ in range(12):
        cur = [0.0] * G
        for g in order:
            cur[g] = 1.0 + max([prev_l[e] if w else cur[e] for e, w in by_node[g]], default=0.0)
        top.append(max(cur))
        prev_l = cur
    return G, deps, (top[11] - top[6]) / 5


def cols_of(cols, base, g):
    k = int(np.searchsorted(base, g, side="right")) - 1
    return int(cols[k][g - base[k]])


@pytest.mark.parametrize("name,ts,split", [("small_p2", 32, (9,)), ("tiny", 24, (3, 9, 12)), ("small_p3", 40, ())])
def test_dataflow_graph_figures_match_a_recount(lib, name, ts, split):
    cfg = workload(name)
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=split)
    bounds = list(zip((0,) + tuple(split), tuple(split) + (17,)))
    G, deps, cp = _recount(lib, sched, cfg, bounds)
    info = lib.slt_schedule_dataflow_info(sched)
    assert info["nodes_per_step"] == G
    assert info["deps_per_step"] == len(deps)
    # the graph itself, edge by edge: successor lists in ascending order, in-degrees
    sp, sv = lib.slt_schedule_export(sched, "succ_ptr", 0), lib.slt_schedule_export(sched, "succ", 0)
    assert sp[0] == 0 and sp[-1] == len(sv) and len(sp) == G + 1 and np.all(np.diff(sp) >= 0)
    got = set()
    for a in range(G):
        lst = sv[sp[a]:sp[a + 1]]
        assert np.all(np.diff(lst) > 0)
        got |= {(int(e) >> 1, a, int(e) & 1) for e in lst}
    assert got == deps
    indeg = np.bincount([g for g, _, _ in deps], minlength=G)
    indeg0 = np.bincount([g for g, _, w in deps if not w], minlength=G)
    assert np.array_equal(lib.slt_schedule_export(sched, "indeg", 0), indeg)
    assert np.array_equal(lib.slt_schedule_export(sched, "indeg0", 0), indeg0)
    assert info["critical_path_nodes"] == pytest.approx(cp, rel=0, abs=1e-12)
    assert len(bounds) <= info["critical_path_nodes"] <= G
    assert info["tiles_in_flight"] == 0
    gpu_run(lib, cfg, nsteps=2, sched=sched, mesh=mesh)
    assert 0 < lib.slt_schedule_dataflow_info(sched)["tiles_in_flight"] <= 2 * G


def test_one_tile_per_subchain_is_a_chain_of_sub_chains(lib):
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=10 ** 6, split=(9,))
    info = lib.slt_schedule_dataflow_info(sched)
    assert info["nodes_per_step"] == 2 and info["critical_path_nodes"] == 2
    assert info["critical_path_items"] == pytest.approx(2.0)


def test_lane_accounting_is_invariant_under_tiling(lib):
    # sparse tiling reorders the iterations and splits cells' facet parts among tiles, but the
    # work of a step stays the same: the FP64 lane instructions needed are equal for every tile
    # size; the executors issue at least that much (idle lanes), small tiles waste more lanes than
    # one tile holding the whole mesh, and the staged executor's compacted passes waste fewer
    # than the item-per-thread warps on small tiles
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    infos = [lib.slt_schedule_lane_info(lib.slt_inspect(ch, tile_size=ts, split=(9,))) for ts in (24, 64, 200, 10 ** 6)]
    need = infos[0]["needed"]
    for inf in infos:
        assert inf["needed"] == pytest.approx(need, rel=1e-12)
        assert inf["dataflow"] >= need and inf["staged"] >= need and inf["untiled"] >= need
    for inf in infos[:2]:
        assert inf["staged"] < inf["dataflow"]
    assert infos[0]["dataflow_efficiency"] < infos[-1]["dataflow_efficiency"]
    assert infos[-1]["untiled"] == pytest.approx(infos[0]["untiled"], rel=1e-12)
