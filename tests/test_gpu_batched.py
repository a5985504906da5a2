"""Multi-shot executor (GPU): S shots of one mesh, shots innermost.  Every shot must give what a
single-field run with that shot's source gives (CUDA single-shot path and the oracle), untiled
and under the dataflow executor."""
import numpy as np
import pytest

from oracle.dg import ElasticDG
from tests.helpers import TOL, rel_l2, workload, gpu_mesh

pytestmark = pytest.mark.gpu


def _shots(cfg, S, seed=3):
    xy = cfg["mesh"]["coords"]
    lo, hi = xy.min(0), xy.max(0)
    rng = np.random.default_rng(seed)
    pts = lo + (hi - lo) * rng.uniform(0.05, 0.95, (S, 2))
    pts[0] = cfg["src"]                       # the workload's own source
    if S > 2:
        pts[2] = pts[1]                       # two shots at the same point
    return pts


def _fields(cfg, S, seed=5):
    rng = np.random.default_rng(seed)
    nc = cfg["v0"].shape[0]
    Np = cfg["v0"].shape[2]
    v0 = 1e-3 * rng.standard_normal((nc, 2, Np, S))
    s0 = 1e-3 * rng.standard_normal((nc, 3, Np, S))
    return v0, s0


def _run_batched(lib, cfg, mesh, sched, pts, v0, s0, n):
    import torch
    v = torch.tensor(v0, device="cuda")
    s = torch.tensor(s0, device="cuda")
    r = torch.tensor(cfg["ricker"], device="cuda")
    lib.slt_execute_batched(mesh, sched, pts, v, s, r, cfg["dt"], n)
    return v.cpu().numpy(), s.cpu().numpy()


def _run_single(lib, cfg, mesh, sched, xy, v0, s0, n):
    import torch
    lib.slt_mesh_set_source(mesh, xy)
    v = torch.tensor(np.ascontiguousarray(v0), device="cuda")
    s = torch.tensor(np.ascontiguousarray(s0), device="cuda")
    r = torch.tensor(cfg["ricker"], device="cuda")
    lib.slt_execute(mesh, sched, v, s, r, cfg["dt"], n)
    return v.cpu().numpy(), s.cpu().numpy()


@pytest.mark.parametrize("tiled", [False, True])
@pytest.mark.parametrize("name,S,ts", [("tiny", 5, 32), ("small_p2", 7, 64), ("small_p3", 3, 40), ("small_p4", 2, 30)])
def test_batched_equals_single_shot_runs(lib, name, S, ts, tiled):
    cfg = workload(name)
    n = min(cfg["nsteps"], 6)
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,)) if tiled else None
    pts = _shots(cfg, S)
    v0, s0 = _fields(cfg, S)
    vb, sb = _run_batched(lib, cfg, mesh, sched, pts, v0, s0, n)
    for k in range(S):
        v1, s1 = _run_single(lib, cfg, mesh, sched, pts[k], v0[..., k], s0[..., k], n)
        # same loop bodies, same per-(cell, shot) operation order: equal to rounding at most
        assert rel_l2(vb[..., k], v1) < 1e-14 and rel_l2(sb[..., k], s1) < 1e-14, (k, rel_l2(vb[..., k], v1))


@pytest.mark.parametrize("tiled", [False, True])
def test_batched_matches_oracle(lib, tiled):
    cfg = workload("small_p2")
    n = 5
    S = 3
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=48, split=(9,)) if tiled else None
    pts = _shots(cfg, S, seed=8)
    v0, s0 = _fields(cfg, S, seed=9)
    vb, sb = _run_batched(lib, cfg, mesh, sched, pts, v0, s0, n)
    dg = ElasticDG(cfg["mesh"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"])
    for k in range(S):
        vo, so = dg.run(v0[..., k].copy(), s0[..., k].copy(), cfg["dt"], n, cfg["ricker"], pts[k])
        assert rel_l2(vb[..., k], vo) < TOL and rel_l2(sb[..., k], so) < TOL, (k, rel_l2(vb[..., k], vo))


def test_batched_untiled_equals_tiled_bitwise(lib):
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    pts = _shots(cfg, 4)
    v0, s0 = _fields(cfg, 4)
    out = [_run_batched(lib, cfg, mesh, None, pts, v0, s0, 4)]
    for ts in (16, 64, 10 ** 6):
        sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,))
        out.append(_run_batched(lib, cfg, mesh, sched, pts, v0, s0, 4))
    for o in out[1:]:
        assert rel_l2(o[0], out[0][0]) < 1e-14 and rel_l2(o[1], out[0][1]) < 1e-14


def test_batched_without_sources_and_errors(lib):
    import torch
    cfg = workload("tiny")
    mesh = gpu_mesh(lib, cfg)
    nc, _, Np = cfg["v0"].shape
    v0, s0 = _fields(cfg, 2)
    v = torch.tensor(v0, device="cuda")
    s = torch.tensor(s0, device="cuda")
    lib.slt_execute_batched(mesh, None, None, v, s, None, cfg["dt"], 3)
    for k in range(2):
        lib.slt_mesh_set_source(mesh, None)
        v1 = torch.tensor(np.ascontiguousarray(v0[..., k]), device="cuda")
        s1 = torch.tensor(np.ascontiguousarray(s0[..., k]), device="cuda")
        lib.slt_execute(mesh, None, v1, s1, None, cfg["dt"], 3)
        assert rel_l2(v[..., k].cpu().numpy(), v1.cpu().numpy()) < 1e-14
    # the colour-phase executor does not take shots; a source off the mesh is refused
    sched1 = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=32, split=(9,), executor=1)
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute_batched(mesh, sched1, None, v, s, None, cfg["dt"], 1)
    assert e.value.code == -6
    with pytest.raises(lib.SltError) as e:
        lib.slt_execute_batched(mesh, None, np.array([[1e9, 1e9], [0.5, 0.5]]), v, s, None, cfg["dt"], 1)
    assert e.value.code == -1
    # zero steps: only the layout round trip, fields unchanged
    v2 = v.clone()
    lib.slt_execute_batched(mesh, None, None, v, s, None, cfg["dt"], 0)
    assert torch.equal(v, v2)


@pytest.mark.parametrize("groups", [1, 2, 3, 7])
def test_shots_per_cta_slices_give_the_same_bits(lib, groups):
    # the dataflow executor runs the shots in slices of `groups`: same arithmetic per (cell, shot)
    cfg = workload("small_p2")
    mesh = gpu_mesh(lib, cfg)
    pts = _shots(cfg, 5)
    v0, s0 = _fields(cfg, 5)
    whole = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=48, split=(9,))
    sliced = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=48, split=(9,), shots_per_cta=groups)
    a = _run_batched(lib, cfg, mesh, whole, pts, v0, s0, 4)
    b = _run_batched(lib, cfg, mesh, sliced, pts, v0, s0, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("degree,S", [(1, 8), (2, 64), (3, 16), (4, 64)])
def test_tensor_core_volume_contraction_matches_dfma(lib, degree, S):
    # the multi-shot form's volume contraction on mma.sync.m8n8k4 FP64 tiles gives the DFMA
    # form's values (up to the order of the sums)
    r = lib.slt_fp64_contraction_probe(degree, 3001, S)
    np_ = (degree + 1) * (degree + 2) // 2
    assert r["rel_diff"] < 1e-13, r
    assert r["dfma_ms"] > 0 and r["dmma_ms"] > 0
    assert r["useful_flops"] == 2 * r["nnz"] * 3001 * S
    assert r["dmma_issued_flops"] == 512 * ((np_ + 7) // 8) * ((2 * np_ + 3) // 4) * 3001 * (S // 8)
