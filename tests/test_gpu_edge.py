"""Degenerate and boundary cases of the GPU path: meshes of one and two cells (no or one interior
facet: empty facet loops, a single tile), and the queue-size limit of the dataflow executor."""
import numpy as np
import pytest

from oracle.dg import ElasticDG
from tests.helpers import TOL, rel_l2

pytestmark = pytest.mark.gpu


def _tiny_mesh(ncell):
    # one triangle, or two sharing the diagonal of the unit square (counter-clockwise)
    V = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    c2v = np.array([[0, 1, 2], [0, 2, 3]][:ncell], dtype=np.int32)
    return {"cell2vert": c2v, "cellxy": V[c2v], "coords": V, "nvert": 4}


@pytest.mark.parametrize("ncell", [1, 2])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_one_and_two_cell_meshes_match_oracle(lib, ncell, p):
    import torch
    m = _tiny_mesh(ncell)
    rng = np.random.default_rng(10 * ncell + p)
    mat = (rng.uniform(1, 2, ncell), rng.uniform(1, 2, ncell), rng.uniform(1, 2, ncell))
    Np = (p + 1) * (p + 2) // 2
    v0, s0 = rng.standard_normal((ncell, 2, Np)), rng.standard_normal((ncell, 3, Np))
    dt = 0.01
    vo, so = ElasticDG(m, p, *mat).run(v0.copy(), s0.copy(), dt, 5)
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], p, *mat)
    info = lib.slt_mesh_info(mesh)
    assert (info["nfi"], info["nfe"]) == (ncell - 1, 3 * ncell - 2 * (ncell - 1))
    for ex in (0, 1):
        for sched in (None, lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=1, split=(9,), executor=ex)):
            v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
            lib.slt_execute(mesh, sched, v, s, None, dt, 5)
            assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL


def test_dataflow_queue_limit_is_refused(lib):
    # steps x tiles must stay below 2^31 (the queue holds int32 node ids): refused, nothing hangs
    import torch
    m = _tiny_mesh(2)
    mat = (np.ones(2), np.ones(2), np.ones(2))
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], 1, *mat)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=1, split=(9,))
    G = sum(lib.slt_schedule_info(sched, k)["ntiles"] for k in range(2))
    v = torch.zeros((2, 2, 3), dtype=torch.float64, device="cuda")
    s = torch.zeros((2, 3, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute(mesh, sched, v, s, None, 0.01, (1 << 31) // G + 1)
    assert e.value.code == -6
    lib.slt_execute(mesh, sched, v, s, None, 0.01, 2)   # the context is still usable


@pytest.mark.parametrize("p,ts", [(1, 8), (2, 5), (3, 16)])
def test_mirror_symmetric_source_on_the_gpu(lib, p, ts):
    # the oracle's mirror pin, on the CUDA path: symmetric to round-off, tiled and untiled
    import torch
    import synth
    from tests.test_oracle_dg import _mirror_mesh, _mirror_pairs, mirror_defect
    m = _mirror_mesh()
    nc = m["cell2vert"].shape[0]
    mat = synth.homogeneous(m, 1.0, 2.0, 1.0)
    dt = synth.cfl_dt(m, 2.0, p)
    ricker = synth.ricker_series(5.0, dt, 30)
    xs = np.array([0.5, 0.70])
    vo, so = ElasticDG(m, p, *mat).run(np.zeros((nc, 2, (p + 1) * (p + 2) // 2)),
                                       np.zeros((nc, 3, (p + 1) * (p + 2) // 2)), dt, 30, ricker, xs)
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], p, *mat, xs)
    pairs = _mirror_pairs(m, p)
    Np = (p + 1) * (p + 2) // 2
    for sched in (None, lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,))):
        v = torch.zeros((nc, 2, Np), dtype=torch.float64, device="cuda")
        s = torch.zeros((nc, 3, Np), dtype=torch.float64, device="cuda")
        lib.slt_execute(mesh, sched, v, s, torch.tensor(ricker, device="cuda"), dt, 30)
        vg, sg = v.cpu().numpy(), s.cpu().numpy()
        assert mirror_defect(vg, sg, pairs) < 1e-12
        assert rel_l2(vg, vo) < TOL and rel_l2(sg, so) < TOL


@pytest.mark.parametrize("where", ["edge", "vertex"])
def test_source_on_a_shared_edge_or_vertex_goes_to_the_smallest_cell(lib, where):
    # a point source on an edge or vertex shared by several cells: the library projects it into
    # the smallest containing cell id, as the oracle does, so the fields agree from zero
    import torch
    import synth
    m = synth.make_mesh(8, 6, seed=5)
    c2v, coords = np.asarray(m["cell2vert"]), np.asarray(m["coords"])
    p, nc = 2, c2v.shape[0]
    Np = (p + 1) * (p + 2) // 2
    mat = synth.homogeneous(m, 1.0, 2.0, 1.0)
    dt = synth.cfl_dt(m, 2.0, p)
    ricker = synth.ricker_series(5.0, dt, 12)
    dg = ElasticDG(m, p, *mat)
    if where == "edge":
        c0, f0, c1 = (int(x) for x in dg.ifacets[len(dg.ifacets) // 2, :3])
        a, b = c2v[c0, f0], c2v[c0, (f0 + 1) % 3]
        xs, owners = 0.5 * (coords[a] + coords[b]), [c0, c1]
    else:
        v = next(v for v in range(coords.shape[0]) if (c2v == v).any(1).sum() == 6)
        xs, owners = coords[v], list(np.nonzero((c2v == v).any(1))[0])
    assert len(owners) >= 2 and dg.locate(xs)[0] == min(owners)
    vo, so = dg.run(np.zeros((nc, 2, Np)), np.zeros((nc, 3, Np)), dt, 12, ricker, xs)
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], p, *mat, xs)
    for sched in (None, lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,))):
        v = torch.zeros((nc, 2, Np), dtype=torch.float64, device="cuda")
        s = torch.zeros((nc, 3, Np), dtype=torch.float64, device="cuda")
        lib.slt_execute(mesh, sched, v, s, torch.tensor(ricker, device="cuda"), dt, 12)
        assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL
