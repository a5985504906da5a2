"""Several meshes at once (uneven sizes, degrees 1-4, tiled and untiled; one combined queue per
degree) and the graph-captured untiled step (GPU).  Every mesh must give exactly what its own
single-mesh call gives, and the oracle's chain."""
import numpy as np
import pytest

from tests.helpers import TOL, rel_l2, workload, oracle_run, gpu_mesh, gpu_run

pytestmark = pytest.mark.gpu


def _fields(cfg):
    import torch
    return (torch.tensor(cfg["v0"], device="cuda"), torch.tensor(cfg["s0"], device="cuda"),
            torch.tensor(cfg["ricker"], device="cuda"))


@pytest.mark.parametrize("tiled", [(0, 1, 0, 1), (1, 1, 1, 1), (0, 0, 0, 0)])
def test_many_meshes_equal_single_runs_and_oracle(lib, tiled):
    names, ts = ["tiny", "small_p2", "small_p3", "small_p4"], [32, 64, 48, 40]
    cfgs = [workload(n) for n in names]
    meshes = [gpu_mesh(lib, c) for c in cfgs]
    scheds = [lib.slt_inspect(lib.slt_mesh_chain(m), tile_size=t, split=(9,)) if on else None
              for m, t, on in zip(meshes, ts, tiled)]
    n = 6
    vs, ss, rs = zip(*[_fields(c) for c in cfgs])
    lib.slt_execute_many(meshes, scheds, list(vs), list(ss), list(rs), [c["dt"] for c in cfgs], n)
    for k, (c, m, sc) in enumerate(zip(cfgs, meshes, scheds)):
        v1, s1 = gpu_run(lib, c, nsteps=n, sched=sc, mesh=m)
        assert np.array_equal(vs[k].cpu().numpy(), v1) and np.array_equal(ss[k].cpu().numpy(), s1), names[k]
    vo, so = oracle_run("small_p2", nsteps=n)
    assert rel_l2(vs[1].cpu().numpy(), vo) < TOL and rel_l2(ss[1].cpu().numpy(), so) < TOL


def test_group_of_same_degree_meshes_shares_one_queue(lib):
    # three P2 meshes of different sizes in one combined plan, executed twice through the group
    cfgs = [workload("small_p2"), workload("small_p2", seed_fields=5, nx=30, ny=10),
            workload("small_p2", seed_fields=6, nx=12, ny=30)]
    meshes = [gpu_mesh(lib, c) for c in cfgs]
    scheds = [lib.slt_inspect(lib.slt_mesh_chain(m), tile_size=ts, split=(9,)) for m, ts in zip(meshes, (64, 16, 200))]
    grp = lib.slt_group_create(meshes, scheds)
    vs, ss, rs = zip(*[_fields(c) for c in cfgs])
    lib.slt_group_execute(grp, list(vs), list(ss), list(rs), [c["dt"] for c in cfgs], 3)
    lib.slt_group_execute(grp, list(vs), list(ss), [r[3:] for r in rs], [c["dt"] for c in cfgs], 4)
    for k, (c, m, sc) in enumerate(zip(cfgs, meshes, scheds)):
        v1, s1 = gpu_run(lib, c, nsteps=7, sched=sc, mesh=m)
        assert np.array_equal(vs[k].cpu().numpy(), v1) and np.array_equal(ss[k].cpu().numpy(), s1), k


def test_graph_captured_steps_equal_single_steps(lib):
    # 8 untiled steps in one call run as a replayed CUDA graph; one step per call does not
    import torch
    cfg = workload("small_p3")
    mesh = gpu_mesh(lib, cfg)
    v, s, r = _fields(cfg)
    lib.slt_execute(mesh, None, v, s, r, cfg["dt"], 8)
    v1, s1, _ = _fields(cfg)
    for k in range(8):
        lib.slt_execute(mesh, None, v1, s1, r[k:], cfg["dt"], 1)
    torch.cuda.synchronize()
    assert torch.equal(v, v1) and torch.equal(s, s1)
    prof = lib.slt_execute_profiled(mesh, None, v, s, r, cfg["dt"], 5)
    assert prof["chain_launches"] == 5 * 7


def test_many_rejects_duplicates_and_foreign_schedules(lib):
    a, b = workload("tiny"), workload("small_p2")
    ma, mb = gpu_mesh(lib, a), gpu_mesh(lib, b)
    va, sa, ra = _fields(a)
    vb, sb, rb = _fields(b)
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute_many([ma, ma], [None, None], [va, va], [sa, sa], [ra, ra], [a["dt"]] * 2, 1)
    assert e.value.code == -1
    sched_b = lib.slt_inspect(lib.slt_mesh_chain(mb), tile_size=64, split=(9,))
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute_many([ma, mb], [sched_b, None], [va, vb], [sa, sb], [ra, rb], [a["dt"], b["dt"]], 1)
    assert e.value.code == -7


def test_batched_form_in_one_graph_captured_launch(lib):
    # meshes of degrees 1-3 and a P2 mesh with 3 shots, all in one persistent launch captured as
    # a CUDA graph: each member gives exactly its own run, the second call replays the graph
    import torch
    names, ts = ["tiny", "small_p2", "small_p3"], [32, 64, 48]
    cfgs = [workload(n) for n in names]
    meshes = [gpu_mesh(lib, c) for c in cfgs]
    scheds = [lib.slt_inspect(lib.slt_mesh_chain(m), tile_size=t, split=(9,)) for m, t in zip(meshes, ts)]
    shot_cfg = workload("small_p2", seed_fields=9, nx=24, ny=14)
    shot_mesh = gpu_mesh(lib, shot_cfg)
    shot_sched = lib.slt_inspect(lib.slt_mesh_chain(shot_mesh), tile_size=24, split=(9,))
    pts = np.array([[10.0, 12.0], [20.0, 5.0], [7.5, 3.3]])
    S = len(pts)
    nc, Np = shot_cfg["mesh"]["cell2vert"].shape[0], 6
    rng = np.random.default_rng(4)
    bv0, bs0 = 1e-3 * rng.standard_normal((nc, 2, Np, S)), 1e-3 * rng.standard_normal((nc, 3, Np, S))
    grp = lib.slt_group_create_batched(meshes + [shot_mesh], scheds + [shot_sched], [1, 1, 1, S],
                                       [None, None, None, pts])
    vs, ss, rs = [list(x) for x in zip(*[_fields(c) for c in cfgs])]
    bv, bs = torch.tensor(bv0, device="cuda"), torch.tensor(bs0, device="cuda")
    br = torch.tensor(shot_cfg["ricker"], device="cuda")
    dts = [c["dt"] for c in cfgs] + [shot_cfg["dt"]]
    lib.slt_group_execute(grp, vs + [bv], ss + [bs], rs + [br], dts, 3)
    lib.slt_group_execute(grp, vs + [bv], ss + [bs], [r[3:] for r in rs] + [br[3:]], dts, 3)
    assert lib.slt_group_graph_replays(grp) == 2
    for k, (c, m, sc) in enumerate(zip(cfgs, meshes, scheds)):
        v1, s1 = gpu_run(lib, c, nsteps=6, sched=sc, mesh=m)
        assert np.array_equal(vs[k].cpu().numpy(), v1) and np.array_equal(ss[k].cpu().numpy(), s1), names[k]
    v2, s2 = torch.tensor(bv0, device="cuda"), torch.tensor(bs0, device="cuda")
    lib.slt_execute_batched(shot_mesh, shot_sched, pts, v2, s2, br, shot_cfg["dt"], 6)
    assert torch.equal(bv, v2) and torch.equal(bs, s2)
    vo, so = oracle_run("small_p3", nsteps=6)
    assert rel_l2(vs[2].cpu().numpy(), vo) < TOL and rel_l2(ss[2].cpu().numpy(), so) < TOL


def test_batched_group_refuses_degree_four_members(lib):
    cfg = workload("small_p4")
    m = gpu_mesh(lib, cfg)
    sc = lib.slt_inspect(lib.slt_mesh_chain(m), tile_size=40, split=(9,))
    with pytest.raises(lib.SltError) as e:
        lib.slt_group_create_batched([m], [sc], [1], [None])
    assert e.value.code == -6
