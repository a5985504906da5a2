"""The executors that run each segment as compacted passes over the staged plan's lists:
executor 3 (staged: each tile's sub-chain out of shared memory through the tile's footprint, its
local map of the cell set, temporaries written to global memory only where another tile reads
them) and executor 4 (the same passes with every value in global memory).  Both must give the
oracle's fields, and the same bits as the dataflow executor on the same schedule (the per-cell
arithmetic and its order are shared); the footprints must be the cells the tile's iterations
touch, recounted from the exported tiling functions."""
import numpy as np
import pytest

from oracle import inspector as OI
from tests.helpers import TOL, gpu_mesh, gpu_run, oracle_run, rel_l2, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("executor,block", [(3, 256), (3, 512), (4, 256), (4, 384)])
@pytest.mark.parametrize("name,ts", [("tiny", 64), ("tiny", 7), ("tiny", 10 ** 6), ("small_p2", 64),
                                     ("small_p2", 200), ("small_p3", 48), ("small_p4", 40)])
def test_staged_matches_oracle_and_dataflow_bitwise(lib, name, ts, executor, block):
    cfg = workload(name)
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    staged = lib.slt_inspect(ch, tile_size=ts, split=(9,), executor=executor, block_threads=block)
    v, s = gpu_run(lib, cfg, sched=staged, mesh=mesh)
    vo, so = oracle_run(name)
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL, (rel_l2(v, vo), rel_l2(s, so))
    v0, s0 = gpu_run(lib, cfg, sched=lib.slt_inspect(ch, tile_size=ts, split=(9,)), mesh=mesh)
    assert np.array_equal(v, v0) and np.array_equal(s, s0)


@pytest.mark.parametrize("executor", [3, 4])
@pytest.mark.parametrize("split", [(), (9,), (3, 9, 12), (4,), (2, 7, 13), tuple(range(1, 16))])
def test_staged_fusion_schemes(lib, split, executor):
    # other fusion schemes send temporaries across sub-chains (then every one is written out);
    # a split inside a phase leaves partial values for the next sub-chain
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    v, s = gpu_run(lib, cfg, sched=lib.slt_inspect(ch, tile_size=32, split=split, executor=executor), mesh=mesh)
    vo, so = oracle_run("tiny")
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL
    v0, s0 = gpu_run(lib, cfg, sched=lib.slt_inspect(ch, tile_size=32, split=split), mesh=mesh)
    assert np.array_equal(v, v0) and np.array_equal(s, s0)


@pytest.mark.parametrize("executor", [3, 4])
def test_staged_backward_tiling(lib, executor):
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    sched = lib.slt_inspect(ch, tile_size=48, split=(9,), seed_loop=(4, 5), executor=executor)
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run("small_p2")
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL


@pytest.mark.parametrize("name,ts,split", [("small_p2", 64, (9,)), ("tiny", 24, (3, 9, 12)), ("small_p3", 40, ())])
def test_staged_footprints_are_the_cells_each_tile_touches(lib, name, ts, split):
    # recount from the exported tiling functions: a tile touches the cells of its cell-loop
    # iterations and both cells of its facet iterations, over every loop of the sub-chain
    cfg = workload(name)
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=split, executor=3)
    _, _, inter, exter = OI.elastic_chain(cfg["mesh"])
    nc = cfg["mesh"]["cell2vert"].shape[0]
    bounds = list(zip((0,) + tuple(split), tuple(split) + (17,)))
    for k, (lo, hi) in enumerate(bounds):
        m = lib.slt_schedule_info(sched, k)["ntiles"]
        touched = [set() for _ in range(m)]
        for J in range(lo, hi):
            sig = lib.slt_schedule_export(sched, "sigma", J)
            kind = OI.ELASTIC_LOOPS[J][0]
            if kind == "cells":
                pairs = zip(range(nc), sig)
            elif kind == "ifacets":
                pairs = list(zip(inter[:, 0], sig)) + list(zip(inter[:, 2], sig))
            else:
                pairs = zip(exter[:, 0], sig)
            for c, t in pairs:
                touched[int(t)].add(int(c))
        ptr = lib.slt_schedule_export(sched, "fp_stage_ptr", k)
        fp = lib.slt_schedule_export(sched, "fp_stage", k)
        assert len(ptr) == m + 1 and ptr[-1] == len(fp)
        for t in range(m):
            got = fp[ptr[t]:ptr[t + 1]]
            assert len(set(got.tolist())) == len(got)
            assert set(got.tolist()) == touched[t], (k, t)


def test_staged_refuses_tiles_beyond_its_shared_memory(lib):
    cfg = workload("small_p4")
    mesh = gpu_mesh(lib, cfg)
    with pytest.raises(lib.SltError) as e:
        lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=10 ** 6, split=(9,), executor=3)
    assert e.value.code == -6


def test_staged_many_steps_one_launch(lib):
    # a persistent launch of many steps (nodes of several steps in flight at once)
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=32, split=(9,), executor=3)
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    v0, s0 = gpu_run(lib, cfg, sched=None, mesh=mesh)
    assert rel_l2(v, v0) < 1e-13 and rel_l2(s, s0) < 1e-13


def test_passes_refuses_tiles_beyond_its_slot_range(lib):
    # the pass lists name a cell by its slot in the tile's footprint (10 bits)
    import synth
    c0 = synth.CONFIGS["small_p2"]
    cfg = synth.build_config("small_p2", nx=2 * c0["nx"], ny=c0["ny"])
    assert cfg["mesh"]["cell2vert"].shape[0] > 2046
    mesh = gpu_mesh(lib, cfg)
    with pytest.raises(lib.SltError) as e:
        lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=10 ** 6, split=(9,), executor=4)
    assert e.value.code == -6


@pytest.mark.parametrize("executor", [0, 3, 4])
def test_kept_successors_give_the_queued_order_bits(lib, executor):
    # a CTA running a successor its tile released (release_order 1) instead of queueing it (2)
    # changes only the order in which independent tiles run: the same bits, several steps in
    # flight in one launch
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    runs = [gpu_run(lib, cfg, sched=lib.slt_inspect(ch, tile_size=40, split=(9,), executor=executor,
                                                    release_order=r), mesh=mesh) for r in (1, 2)]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    vo, so = oracle_run("small_p2")
    assert rel_l2(runs[0][0], vo) < TOL and rel_l2(runs[0][1], so) < TOL


@pytest.mark.parametrize("executor", [3, 4])
def test_footprints_of_many_slots(lib, executor):
    # P1 tiles whose footprints use slots 512 and above (three neighbour slots share one word per
    # cell, so the upper slot bits of the third face must survive): the dataflow executor's bits
    # and the oracle's fields
    cfg = workload("small_p2", p=1)
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    sched = lib.slt_inspect(ch, tile_size=650, split=(9,), executor=executor, block_threads=384)
    fp_ptr = lib.slt_schedule_export(sched, "fp_stage_ptr", 0)
    assert np.diff(fp_ptr).max() > 600
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    v0, s0 = gpu_run(lib, cfg, sched=lib.slt_inspect(ch, tile_size=650, split=(9,)), mesh=mesh)
    assert np.array_equal(v, v0) and np.array_equal(s, s0)
    vo, so = oracle_run("small_p2", p=1)
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL
