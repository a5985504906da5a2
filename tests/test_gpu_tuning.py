"""Fusion-scheme variants with their own tile size per sub-chain, and the autotuner (GPU).
Schedules bit-exact against the oracle inspector run per sub-chain at its tile size; the
tuned configuration still matches the oracle's untiled chain."""
import numpy as np
import pytest

from oracle import inspector as OI
from tests.helpers import TOL, rel_l2, workload, oracle_run, gpu_mesh, gpu_run, compare_schedules

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("split,sub_ts", [((9,), (64, 200)), ((9,), (7, 0)), ((3, 9, 12), (16, 48, 5, 100)),
                                          ((1, 5, 9, 13), (30, 0, 12, 64, 0))])
def test_per_subchain_tile_sizes_bit_exact_and_parity(lib, split, sub_ts):
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    ts0 = 40
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts0, split=split, sub_tile_size=sub_ts)
    ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
    bounds = list(zip((0,) + split, split + (17,)))
    for k, (lo, hi) in enumerate(bounds):
        sub = ch.sub(lo, hi)
        ts = sub_ts[k] if sub_ts[k] > 0 else ts0
        compare_schedules(lib, sched, sub, [(0, hi - lo)], ts, renumber=True, xy=ch.points[sub.loops[0][0]],
                          _offset=(k, lo))
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run("tiny")
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL


@pytest.mark.parametrize("nshots", [1, 3])
def test_autotune_table_and_tuned_run(lib, nshots):
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    groups = (1, 2) if nshots > 1 else ()
    best, table = lib.slt_autotune(mesh, [32, 96], nshots=nshots, shapes=True, block_threads=(128, 256),
                                   shots_per_cta=groups, steps=2, split=(9,))
    ng = max(len(groups), 1)
    assert table.shape == (1 + 2 * 2 * 2 * ng, 5)
    assert tuple(table[0, :4]) == (0, 0, 0, 0)
    assert {(int(r[0]), int(r[1]), int(r[2]), int(r[3])) for r in table[1:]} == {
        (t, r, b, g) for t in (32, 96) for r in (0, 1) for b in (128, 256) for g in (groups or (0,))}
    assert np.all((table[:, 4] > 0) | (table[:, 4] == -1))
    ms = np.where(table[:, 4] > 0, table[:, 4], np.inf)
    k = int(np.argmin(ms))
    assert best.tile_size == int(table[k, 0])
    if best.tile_size:
        assert (best.renumber, best.block_threads, best.shots_per_cta) == tuple(int(x) for x in table[k, 1:4])
        assert best.nsplit == 1 and best.split[0] == 9
    # the winner is an ordinary configuration: parity with the oracle
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), best) if best.tile_size else None
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run("small_p2")
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL


def test_autotune_rejects_bad_candidates(lib):
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    for kw in (dict(tile_sizes=[0]), dict(tile_sizes=[8], block_threads=(96,)), dict(tile_sizes=[8], steps=0)):
        with pytest.raises(lib.SltError) as e:
            lib.slt_autotune(mesh, **kw)
        assert e.value.code == -1
    with pytest.raises(lib.SltError):
        lib.slt_autotune(mesh, [8], nshots=2, executor=1)


@pytest.mark.parametrize("seeds,ts", [((4, 0), 16), ((8, 3), 40), ((1, 7), 7), ((5, 5), 200)])
def test_backward_tiling_bit_exact_and_parity(lib, seeds, ts):
    # seed loops in the middle of both sub-chains: the loops before them are tiled backwards
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,), seed_loop=seeds)
    ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
    for k, (lo, hi) in enumerate(((0, 9), (9, 17))):
        sub = ch.sub(lo, hi)
        compare_schedules(lib, sched, sub, [(0, hi - lo)], ts, renumber=True,
                          xy=ch.points[sub.loops[seeds[k]][0]], seed=seeds[k], _offset=(k, lo))
    for ex in (0, 1):
        sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,), seed_loop=seeds, executor=ex)
        v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
        vo, so = oracle_run("tiny")
        assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL


def test_backward_tiling_on_the_p2_workload(lib):
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=64, split=(9,), seed_loop=(4, 4))
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run("small_p2")
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL

