"""Parity at the full sizes of the benchmarked workloads, in the launch configurations bench.py
times: the large P2 mesh (1.0M cells; the whole schedule bit for bit against the oracle inspector,
two tiled steps against the oracle's chain, four steps in each launch form against it, and the
discrete energy over a 100-step launch), the P4 mesh, sampled shots of the 64-shot batched run,
sampled members of the 16-mesh group and of the whole batched configuration in one launch, and the
adjoint workload's gradient against central differences of its misfit (one shot untiled; eight
shots in one call on the tiles).  Minutes of oracle time: marked slow."""
import numpy as np
import pytest

import synth
from oracle import inspector as OI
from oracle.dg import ElasticDG
from tests.helpers import TOL, rel_l2, gpu_mesh

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TS = 256


@pytest.fixture(scope="module")
def large(lib):
    cfg = synth.build_config("large")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=TS, split=(9,))
    return cfg, mesh, sched


def test_fullsize_schedule_bit_exact(lib, large):
    cfg, mesh, sched = large
    ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
    for k, (lo, hi) in enumerate(((0, 9), (9, 17))):
        o = OI.inspect(ch.sub(lo, hi), TS, renumber=True, xy=xy)
        info = lib.slt_schedule_info(sched, k)
        assert (info["ntiles"], info["ncolours"], info["restarts"]) == (o["ntiles"], o["ncolours"], o["restarts"])
        assert np.array_equal(lib.slt_schedule_export(sched, "rank", k), o["rank"])
        assert np.array_equal(lib.slt_schedule_export(sched, "colour", k), o["colour"])
        for jj in range(hi - lo):
            assert np.array_equal(lib.slt_schedule_export(sched, "sigma", lo + jj), o["sigma"][jj])
            ptr, its = o["lists"][jj]
            assert np.array_equal(lib.slt_schedule_export(sched, "list_ptr", lo + jj), ptr)
            assert np.array_equal(lib.slt_schedule_export(sched, "list", lo + jj), its)
        # the local maps of the sub-chain's first facet loop (its increment descriptor), and the
        # export flags of every loop
        fp_ptr, fp, lmap = o["local_maps"][1][1]
        assert np.array_equal(lib.slt_schedule_export(sched, "fp_ptr", lo + 1, 1), fp_ptr)
        assert np.array_equal(lib.slt_schedule_export(sched, "fp", lo + 1, 1), fp)
        assert np.array_equal(lib.slt_schedule_export(sched, "lmap", lo + 1, 1), lmap)
        for jj, f in enumerate(OI.export_flags(ch.sub(lo, hi), o["sigma"])):
            assert np.array_equal(lib.slt_schedule_export(sched, "export", lo + jj), f), lo + jj


def test_fullsize_tiled_steps_match_oracle(lib, large):
    import torch
    cfg, mesh, sched = large
    nc = cfg["mesh"]["cell2vert"].shape[0]
    rng = np.random.default_rng(17)
    v0 = 1e-3 * rng.standard_normal((nc, 2, 6))
    s0 = 1e-3 * rng.standard_normal((nc, 3, 6))
    v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
    lib.slt_execute(mesh, sched, v, s, torch.tensor(cfg["ricker"], device="cuda"), cfg["dt"], 2)
    dg = ElasticDG(cfg["mesh"], 2, cfg["rho"], cfg["lam"], cfg["mu"])
    vo, so = dg.run(v0, s0, cfg["dt"], 2, cfg["ricker"], cfg["src"])
    assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL


@pytest.fixture(scope="module")
def large_oracle4(large):
    # four oracle steps at full size from seeded random fields, with the source
    cfg = large[0]
    nc = cfg["mesh"]["cell2vert"].shape[0]
    rng = np.random.default_rng(29)
    v0 = 1e-3 * rng.standard_normal((nc, 2, 6))
    s0 = 1e-3 * rng.standard_normal((nc, 3, 6))
    dg = ElasticDG(cfg["mesh"], 2, cfg["rho"], cfg["lam"], cfg["mu"])
    vo, so = dg.run(v0.copy(), s0.copy(), cfg["dt"], 4, cfg["ricker"], cfg["src"])
    return v0, s0, vo, so


@pytest.mark.parametrize("form", ["untiled_graph", "tiled_ts256", "cluster_ts2048_c4", "staged_ts256_bt384"])
def test_fullsize_four_steps_in_each_timed_launch_form(lib, large, large_oracle4, form):
    # the other launch forms bench.py times at full size: the untiled chain replayed as a CUDA graph
    # (four or more steps), the default dataflow executor, and the cluster executor of its
    # `cluster` key (ts 2048, 4-CTA clusters), each four steps in one call against the oracle
    import torch
    cfg, mesh, sched = large
    v0, s0, vo, so = large_oracle4
    if form == "untiled_graph":
        sc = None
    elif form == "tiled_ts256":
        sc = sched
    elif form == "cluster_ts2048_c4":
        sc = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=2048, split=(9,), executor=2, cluster_size=4)
    else:
        sc = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=256, split=(9,), executor=3, block_threads=384)
    v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
    lib.slt_execute(mesh, sc, v, s, torch.tensor(cfg["ricker"], device="cuda"), cfg["dt"], 4)
    assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL


def test_fullsize_energy_invariant_over_a_long_tiled_launch(lib, large):
    # source off, seeded random start: the leapfrog's discrete energy
    # E^n = 1/2 <v^{n+1/2}, M_rho v^{n-1/2}> + 1/2 <sigma^n, M_S sigma^n> is invariant (the operator
    # pair is skew-adjoint), so after one persistent 100-step launch, the bench's launch form, it
    # equals its starting value up to rounding; the inner products are the oracle's
    import torch
    cfg, mesh, sched = large
    nc = cfg["mesh"]["cell2vert"].shape[0]
    rng = np.random.default_rng(23)
    v0 = 1e-3 * rng.standard_normal((nc, 2, 6))
    s0 = 1e-3 * rng.standard_normal((nc, 3, 6))
    dg = ElasticDG(cfg["mesh"], 2, cfg["rho"], cfg["lam"], cfg["mu"])

    def energy(v, s):  # v = v^{n-1/2}, s = sigma^n; one more step gives v^{n+1/2}
        vt, st = torch.tensor(v, device="cuda"), torch.tensor(s, device="cuda")
        lib.slt_execute(mesh, sched, vt, st, None, cfg["dt"], 1)
        return 0.5 * dg.inner_v(vt.cpu().numpy(), v) + 0.5 * dg.inner_s(s, s)

    e0 = energy(v0, s0)
    v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
    lib.slt_execute(mesh, sched, v, s, None, cfg["dt"], 100)
    v1, s1 = v.cpu().numpy(), s.cpu().numpy()
    e100 = energy(v1, s1)
    assert np.isfinite(e100) and abs(e100 - e0) <= 1e-10 * abs(e0), (e0, e100)
    assert rel_l2(v1, v0) > 1e-2  # the fields did move


def test_fullsize_p4_tiled_steps_match_oracle(lib):
    # the P4 configuration in the bench's launch configuration: ts 256, 384-thread tiles
    import torch
    cfg = synth.build_config("p4")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=256, split=(9,), block_threads=384)
    nc = cfg["mesh"]["cell2vert"].shape[0]
    rng = np.random.default_rng(19)
    v0 = 1e-3 * rng.standard_normal((nc, 2, 15))
    s0 = 1e-3 * rng.standard_normal((nc, 3, 15))
    v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
    lib.slt_execute(mesh, sched, v, s, torch.tensor(cfg["ricker"], device="cuda"), cfg["dt"], 2)
    dg = ElasticDG(cfg["mesh"], 4, cfg["rho"], cfg["lam"], cfg["mu"])
    vo, so = dg.run(v0, s0, cfg["dt"], 2, cfg["ricker"], cfg["src"])
    assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL


@pytest.mark.parametrize("ts", [0, 16])
def test_fullsize_batched_sampled_shots_match_oracle(lib, ts):
    # the bench's batched configuration: 708x354 squares (501k cells), P2, 64 shots on the 8x8
    # grid, untiled and dataflow at ts 16; two sampled shots start from seeded random fields
    import torch
    cfg = synth.build_config("large", nx=708, ny=354)
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,)) if ts else None
    nc = cfg["mesh"]["cell2vert"].shape[0]
    S = 64
    grid = np.array([((i + 0.5) * 300.0 / 8, (j + 0.5) * 150.0 / 8) for j in range(8) for i in range(8)])
    v = torch.zeros((nc, 2, 6, S), dtype=torch.float64, device="cuda")
    s = torch.zeros((nc, 3, 6, S), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(23)
    init = {}
    for k in (5, 58):
        init[k] = (1e-3 * rng.standard_normal((nc, 2, 6)), 1e-3 * rng.standard_normal((nc, 3, 6)))
        v[..., k] = torch.tensor(init[k][0], device="cuda")
        s[..., k] = torch.tensor(init[k][1], device="cuda")
    lib.slt_execute_batched(mesh, sched, grid, v, s, torch.tensor(cfg["ricker"], device="cuda"), cfg["dt"], 2)
    dg = ElasticDG(cfg["mesh"], 2, cfg["rho"], cfg["lam"], cfg["mu"])
    for k, (v0, s0) in init.items():
        vo, so = dg.run(v0.copy(), s0.copy(), cfg["dt"], 2, cfg["ricker"], grid[k])
        assert rel_l2(v[..., k].cpu().numpy(), vo) < TOL and rel_l2(s[..., k].cpu().numpy(), so) < TOL, k
    # every other shot started from rest: only its own source has acted
    assert torch.isfinite(s).all() and float(s[..., 0].abs().max()) > 0


def test_fullsize_group_of_uneven_meshes(lib):
    # the bench's 16 uneven meshes (2.75M cells, P1-P3, ts 256) as one group for 2 steps: sampled
    # members equal their single-mesh runs bit for bit; the smallest equals the oracle
    import torch
    cfgs = synth.multi_configs(16, nsteps=2)
    meshes = [gpu_mesh(lib, c) for c in cfgs]
    scheds = [lib.slt_inspect(lib.slt_mesh_chain(m), tile_size=256, split=(9,)) for m in meshes]
    rng = np.random.default_rng(29)
    init = []
    for c in cfgs:
        nc, Np = c["mesh"]["cell2vert"].shape[0], (c["p"] + 1) * (c["p"] + 2) // 2
        init.append((1e-3 * rng.standard_normal((nc, 2, Np)), 1e-3 * rng.standard_normal((nc, 3, Np))))
    vs = [torch.tensor(a, device="cuda") for a, _ in init]
    ss = [torch.tensor(b, device="cuda") for _, b in init]
    rs = [torch.tensor(c["ricker"], device="cuda") for c in cfgs]
    grp = lib.slt_group_create(meshes, scheds)
    lib.slt_group_execute(grp, vs, ss, rs, [c["dt"] for c in cfgs], 2)
    small = int(np.argmin([c["mesh"]["cell2vert"].shape[0] for c in cfgs]))
    for k in sorted({0, 7, small}):
        v1, s1 = torch.tensor(init[k][0], device="cuda"), torch.tensor(init[k][1], device="cuda")
        lib.slt_execute(meshes[k], scheds[k], v1, s1, rs[k], cfgs[k]["dt"], 2)
        assert torch.equal(vs[k], v1) and torch.equal(ss[k], s1), k
    c = cfgs[small]
    dg = ElasticDG(c["mesh"], c["p"], c["rho"], c["lam"], c["mu"])
    vo, so = dg.run(init[small][0].copy(), init[small][1].copy(), c["dt"], 2, c["ricker"], c["src"])
    assert rel_l2(vs[small].cpu().numpy(), vo) < TOL and rel_l2(ss[small].cpu().numpy(), so) < TOL


def test_fullsize_adjoint_gradient_matches_central_differences(lib):
    # the bench's adjoint configuration: 448x224 squares (200k cells), P2, +-5 % perturbed layers,
    # one top-row shot, 50 receivers, 1000 steps, checkpoints every 50; two seeded directions
    import torch
    n = 1000
    cfg = synth.build_config("adjoint", nsteps=n)
    m = cfg["mesh"]
    shot = np.array([(0 + 0.5) * 300.0 / 8, (7 + 0.5) * 150.0 / 8])
    rec = np.stack([(np.arange(50) + 0.5) * 6.0, np.full(50, 149.0)], 1)
    base = synth.layered(m)
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], 2, *base, shot)
    r = lib.slt_receivers_create(mesh, rec)
    rk = torch.tensor(cfg["ricker"], device="cuda")
    data = torch.zeros((n, 50, 2), dtype=torch.float64, device="cuda")
    lib.slt_record(mesh, None, r, rk, cfg["dt"], n, data)
    model = (cfg["rho"], cfg["lam"], cfg["mu"])
    lib.slt_mesh_set_material(mesh, *model)
    g = torch.zeros((3, m["cell2vert"].shape[0]), dtype=torch.float64, device="cuda")
    J = lib.slt_adjoint(mesh, None, r, rk, cfg["dt"], n, data, 50, g)
    g = g.cpu().numpy()
    tr = torch.zeros_like(data)

    def misfit(mod):
        lib.slt_mesh_set_material(mesh, *mod)
        lib.slt_record(mesh, None, r, rk, cfg["dt"], n, tr)
        return 0.5 * cfg["dt"] * float(((tr - data) ** 2).sum())

    assert abs(misfit(model) - J) <= 1e-12 * J
    rng = np.random.default_rng(31)
    for _ in range(2):
        d = [a * rng.uniform(-1, 1, a.shape) for a in model]
        eps = 1e-5   # truncation ~ (eps / 0.05)^2 = 4e-8 of the derivative, round-off ~1e-9
        fd = (misfit([a + eps * b for a, b in zip(model, d)]) - misfit([a - eps * b for a, b in zip(model, d)])) / (2 * eps)
        ad = sum(g[k] @ d[k] for k in range(3))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_fullsize_eight_shot_tiled_adjoint(lib):
    # the bench's adjoint block: 8 top-row shots in one call, 1000 steps, checkpoints every 50, on
    # the tiles of a ts 64 schedule: the same misfit and gradient as the untiled run, and the
    # gradient along a seeded direction equal to central differences of the misfit
    import torch
    n = 1000
    cfg = synth.build_config("adjoint", nsteps=n)
    m = cfg["mesh"]
    nc = m["cell2vert"].shape[0]
    shots = np.array([((i + 0.5) * 300.0 / 8, (7 + 0.5) * 150.0 / 8) for i in range(8)])
    rec = np.stack([(np.arange(50) + 0.5) * 6.0, np.full(50, 149.0)], 1)
    mesh = lib.slt_mesh_create(m["cell2vert"], m["cellxy"], 2, *synth.layered(m))
    r = lib.slt_receivers_create(mesh, rec)
    rk = torch.tensor(cfg["ricker"], device="cuda")
    data = torch.zeros((n, 8, 50, 2), dtype=torch.float64, device="cuda")
    lib.slt_record_batched(mesh, None, r, shots, rk, cfg["dt"], n, data)
    model = (cfg["rho"], cfg["lam"], cfg["mu"])
    lib.slt_mesh_set_material(mesh, *model)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=64, split=(9,))
    out = []
    for sc in (sched, None):
        g = torch.zeros((3, nc), dtype=torch.float64, device="cuda")
        J = lib.slt_adjoint_batched(mesh, sc, r, shots, rk, cfg["dt"], n, data, 50, g)
        out.append((J, g.cpu().numpy()))
    (J, g), (J0, g0) = out
    assert abs(J - J0) <= 1e-12 * J0 and rel_l2(g, g0) < 1e-10
    tr = torch.zeros_like(data)

    def misfit(mod):
        lib.slt_mesh_set_material(mesh, *mod)
        lib.slt_record_batched(mesh, sched, r, shots, rk, cfg["dt"], n, tr)
        return 0.5 * cfg["dt"] * float(((tr - data) ** 2).sum())

    assert abs(misfit(model) - J) <= 1e-12 * J
    rng = np.random.default_rng(37)
    d = [a * rng.uniform(-1, 1, a.shape) for a in model]
    eps = 1e-5
    fd = (misfit([a + eps * b for a, b in zip(model, d)]) - misfit([a - eps * b for a, b in zip(model, d)])) / (2 * eps)
    ad = sum(g[k] @ d[k] for k in range(3))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_fullsize_batched_configuration_in_one_launch(lib):
    # the bench's one-launch block: the 64-shot 708x354 P2 mesh (ts 16) and the 16 uneven meshes
    # (ts 256) from one queue, 2 steps: sampled members equal their own runs bit for bit
    import torch
    bcfg = synth.build_config("large", nx=708, ny=354, nsteps=2)
    big = gpu_mesh(lib, bcfg)
    bsched = lib.slt_inspect(lib.slt_mesh_chain(big), tile_size=16, split=(9,))
    grid = np.array([((i + 0.5) * 300.0 / 8, (j + 0.5) * 150.0 / 8) for j in range(8) for i in range(8)])
    cfgs = synth.multi_configs(16, nsteps=2)
    meshes = [gpu_mesh(lib, c) for c in cfgs]
    scheds = [lib.slt_inspect(lib.slt_mesh_chain(m), tile_size=256, split=(9,)) for m in meshes]
    nc = bcfg["mesh"]["cell2vert"].shape[0]
    rng = np.random.default_rng(41)
    bv0 = 1e-3 * rng.standard_normal((nc, 2, 6, 64))
    bs0 = 1e-3 * rng.standard_normal((nc, 3, 6, 64))
    init = []
    for c in cfgs:
        n_, Np = c["mesh"]["cell2vert"].shape[0], (c["p"] + 1) * (c["p"] + 2) // 2
        init.append((1e-3 * rng.standard_normal((n_, 2, Np)), 1e-3 * rng.standard_normal((n_, 3, Np))))
    grp = lib.slt_group_create_batched([big] + meshes, [bsched] + scheds, [64] + [1] * 16, [grid] + [None] * 16)
    vs = [torch.tensor(bv0, device="cuda")] + [torch.tensor(a, device="cuda") for a, _ in init]
    ss = [torch.tensor(bs0, device="cuda")] + [torch.tensor(b, device="cuda") for _, b in init]
    rs = [torch.tensor(bcfg["ricker"], device="cuda")] + [torch.tensor(c["ricker"], device="cuda") for c in cfgs]
    dts = [bcfg["dt"]] + [c["dt"] for c in cfgs]
    lib.slt_group_execute(grp, vs, ss, rs, dts, 2)
    v2, s2 = torch.tensor(bv0, device="cuda"), torch.tensor(bs0, device="cuda")
    lib.slt_execute_batched(big, bsched, grid, v2, s2, rs[0], bcfg["dt"], 2)
    assert torch.equal(vs[0], v2) and torch.equal(ss[0], s2)
    for k in (0, 5, 11):
        v1, s1 = torch.tensor(init[k][0], device="cuda"), torch.tensor(init[k][1], device="cuda")
        lib.slt_execute(meshes[k], scheds[k], v1, s1, rs[k + 1], cfgs[k]["dt"], 2)
        assert torch.equal(vs[k + 1], v1) and torch.equal(ss[k + 1], s1), k

