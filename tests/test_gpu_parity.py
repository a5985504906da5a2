"""CUDA path vs the oracle on the same seeded inputs (GPU).  FP64 results within 1e-11
relative L2 per field; integer schedules bit-exact."""
import numpy as np
import pytest

import synth
from oracle import inspector as OI
from oracle.dg import ElasticDG
from tests.helpers import TOL, rel_l2, workload, oracle_run, gpu_mesh, gpu_run, compare_schedules

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_operators_match_oracle(lib, p):
    import torch
    m = synth.make_mesh(9, 7, seed=p)
    rng = np.random.default_rng(p)
    nc = m["cell2vert"].shape[0]
    rho, lam, mu = rng.uniform(1, 3, nc), rng.uniform(1, 3, nc), rng.uniform(1, 3, nc)
    dg = ElasticDG(m, p, rho, lam, mu)
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], p, rho, lam, mu)
    s = rng.standard_normal((nc, 3, dg.Np))
    v = rng.standard_normal((nc, 2, dg.Np))
    out_a = torch.zeros((nc, 2, dg.Np), dtype=torch.float64, device="cuda")
    out_b = torch.zeros((nc, 3, dg.Np), dtype=torch.float64, device="cuda")
    lib.slt_apply_operator(mesh, 0, torch.tensor(s, device="cuda"), out_a)
    lib.slt_apply_operator(mesh, 1, torch.tensor(v, device="cuda"), out_b)
    torch.cuda.synchronize()
    assert rel_l2(out_a.cpu().numpy(), dg.apply_A(s)) < 1e-13
    assert rel_l2(out_b.cpu().numpy(), dg.apply_B(v)) < 1e-13


@pytest.mark.parametrize("name", ["tiny", "small_p2", "small_p3", "small_p4"])
def test_untiled_chain_matches_oracle(lib, name):
    cfg = workload(name)
    v, s = gpu_run(lib, cfg)
    vo, so = oracle_run(name)
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL, (rel_l2(v, vo), rel_l2(s, so))


@pytest.mark.parametrize("executor", [0, 1, 2])
@pytest.mark.parametrize("name,ts", [("tiny", 64), ("tiny", 7), ("tiny", 1), ("tiny", 10 ** 6),
                                     ("small_p2", 64), ("small_p2", 200), ("small_p3", 48), ("small_p4", 40)])
def test_tiled_chain_matches_oracle(lib, name, ts, executor):
    cfg = workload(name)
    mesh = gpu_mesh(lib, cfg)
    ch = lib.slt_mesh_chain(mesh)
    sched = lib.slt_inspect(ch, tile_size=ts, split=(9,), executor=executor)
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run(name)
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL, (rel_l2(v, vo), rel_l2(s, so))


@pytest.mark.parametrize("executor", [0, 1, 2])
@pytest.mark.parametrize("split", [(), (9,), (3, 9, 12), (2, 7, 13), tuple(range(1, 16))])
def test_fusion_schemes_match_oracle(lib, split, executor):
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=32, split=split, executor=executor)
    v, s = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run("tiny")
    assert rel_l2(v, vo) < TOL and rel_l2(s, so) < TOL


@pytest.mark.parametrize("name,ts", [("small_p2", 64), ("small_p3", 16)])
def test_dataflow_equals_colour_phases_bitwise(lib, name, ts):
    # each cell's arithmetic is the same whatever order the tiles run in: identical bits
    cfg = workload(name)
    mesh = gpu_mesh(lib, cfg)
    out = []
    for ex, cl in ((0, 0), (1, 0), (2, 2), (2, 8)):
        sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,), executor=ex, cluster_size=cl)
        out.append(gpu_run(lib, cfg, sched=sched, mesh=mesh))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])


@pytest.mark.parametrize("name", ["tiny", "small_p2", "small_p3", "small_p4"])
def test_untiled_phases_equal_tiled_loops_bitwise(lib, name):
    # the untiled chain fuses runs of loops into one pass per cell (ten launches); a schedule of
    # one tile runs the loops one by one over every cell: the sums are taken in the same order, so
    # the bits agree (smaller tiles may add one cell's faces in another order: rounding differs)
    cfg = workload(name)
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=10 ** 6, split=(9,))
    for n in (2, 8):  # one launch per phase; a replayed graph of one step
        vt, st = gpu_run(lib, cfg, nsteps=n, sched=sched, mesh=mesh)
        vu, su = gpu_run(lib, cfg, nsteps=n, sched=None, mesh=mesh)
        assert np.array_equal(vt, vu) and np.array_equal(st, su), (name, n)


@pytest.mark.parametrize("executor", [0, 2])
def test_dataflow_wait_limit_reports_timeout_and_context_survives(lib, executor):
    # with a one-poll wait limit the tiles that must wait for a neighbour give up: the kernel
    # sets its error flag and returns, the call reports SLT_ERR_TIMEOUT, and the next call works
    import torch
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    impatient = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,), wait_spins=1,
                                executor=executor, cluster_size=4)
    v = torch.tensor(cfg["v0"], device="cuda")
    s = torch.tensor(cfg["s0"], device="cuda")
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute(mesh, impatient, v, s, None, cfg["dt"], 20)
    assert e.value.code == -4
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,))
    vg, sg = gpu_run(lib, cfg, sched=sched, mesh=mesh)
    vo, so = oracle_run("tiny")
    assert rel_l2(vg, vo) < TOL and rel_l2(sg, so) < TOL


def test_host_buffers_and_no_source(lib):
    import torch
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=64, split=(9,))
    v = cfg["v0"].copy()
    s = cfg["s0"].copy()
    lib.slt_execute_host(mesh, sched, v, s, np.ascontiguousarray(cfg["ricker"]), cfg["dt"], 5)
    vd, sd = gpu_run(lib, cfg, nsteps=5, sched=sched, mesh=mesh)
    assert np.array_equal(v, vd) and np.array_equal(s, sd)
    # page-locked buffers (the end-to-end bench's case) give the same bits
    vp, sp = torch.tensor(cfg["v0"]).pin_memory(), torch.tensor(cfg["s0"]).pin_memory()
    lib.slt_execute_host(mesh, sched, vp, sp, np.ascontiguousarray(cfg["ricker"]), cfg["dt"], 5)
    assert np.array_equal(vp.numpy(), vd) and np.array_equal(sp.numpy(), sd)
    # no source: compare with the oracle without the source term
    dg = ElasticDG(cfg["mesh"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"])
    vo, so = dg.run(cfg["v0"].copy(), cfg["s0"].copy(), cfg["dt"], 4)
    vt = torch.tensor(cfg["v0"], device="cuda")
    st = torch.tensor(cfg["s0"], device="cuda")
    lib.slt_execute(mesh, sched, vt, st, None, cfg["dt"], 4)
    assert rel_l2(vt.cpu().numpy(), vo) < TOL and rel_l2(st.cpu().numpy(), so) < TOL
    # zero steps leave the fields untouched
    lib.slt_execute(mesh, None, vt, st, None, cfg["dt"], 0)
    assert rel_l2(vt.cpu().numpy(), vo) < TOL


def test_schedule_of_another_mesh_is_rejected(lib):
    import torch
    cfg = workload("tiny")
    m1, m2 = gpu_mesh(lib, cfg), gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(m1), tile_size=64)
    v = torch.tensor(cfg["v0"], device="cuda")
    s = torch.tensor(cfg["s0"], device="cuda")
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute(m2, sched, v, s, None, cfg["dt"], 1)
    assert e.value.code == -7


@pytest.mark.parametrize("ts", [1, 5, 64, 10 ** 6])
@pytest.mark.parametrize("renumber,colouring", [(1, 0), (0, 0), (1, 1)])
def test_elastic_inspector_bit_exact(lib, ts, renumber, colouring):
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, renumber=renumber, colouring=colouring,
                            split=(9,), prio_seed=0x5EED)
    ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
    compare_schedules(lib, sched, ch, [(0, 9), (9, 17)], ts, renumber=bool(renumber), xy=xy,
                      sequential=bool(colouring), prio_seed=0x5EED)


@pytest.mark.parametrize("split", [(3, 9, 12), (1, 5, 9, 13)])
def test_facet_seeded_subchains_bit_exact(lib, split):
    # sub-chains seeded at a facet loop rank facets by the Hilbert index of their midpoints
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=24, split=split)
    ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
    bounds = list(zip((0,) + split, split + (17,)))
    for k, (lo, hi) in enumerate(bounds):
        sub = ch.sub(lo, hi)
        compare_schedules(lib, sched, sub, [(0, hi - lo)], 24, renumber=True, xy=ch.points[sub.loops[0][0]],
                          _offset=(k, lo))


def _gpu_chain(lib, ch):
    g = lib.slt_chain_create()
    for n in ch.set_size:
        lib.slt_set(g, n)
    for (frm, to, a, vals) in ch.maps:
        lib.slt_map(g, frm, to, a, vals)
    for (s, descs, _) in ch.loops:
        lib.slt_loop(g, s, descs)
    return g


@pytest.mark.parametrize("seed", range(10))
def test_generic_chain_inspector_bit_exact(lib, seed):
    from tests.test_oracle_inspector import _random_chain, _strip_chain, _wheel_chain
    rng = np.random.default_rng(seed)
    ch = _random_chain(rng, int(rng.integers(2, 6)))
    for c, ts in ((ch, int(rng.integers(1, 8))), (_strip_chain(), 2), (_wheel_chain()[0], 7)):
        g = _gpu_chain(lib, c)
        sched = lib.slt_inspect(g, tile_size=ts, renumber=0, prio_seed=seed)
        compare_schedules(lib, sched, c, [(0, len(c.loops))], ts, prio_seed=seed)
