"""Misfit and gradient on the GPU (slt_record, slt_adjoint, torch.autograd) against the oracle's
discrete adjoint and against central finite differences of the GPU misfit."""
import numpy as np
import pytest

import synth
from oracle import adjoint as OA
from oracle.dg import ElasticDG
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _problem(p=2, nx=8, ny=6, nsteps=30, seed=3):
    m = synth.make_mesh(nx, ny, seed=seed)
    rho, lam, mu = synth.homogeneous(m)
    rng = np.random.default_rng(seed)
    pert = lambda a: a * (1 + 0.05 * rng.uniform(-1, 1, a.shape))
    model0 = (rho, lam, mu)
    model = (pert(rho), pert(lam), pert(mu))
    vp = float(np.max(np.sqrt((model[1] + 2 * model[2]) / model[0])))
    dt = synth.cfl_dt(m, vp, p)
    ricker = synth.ricker_series(5.0, dt, nsteps)
    xs = np.array([0.5, 0.5])
    rec = np.array([[0.2, 0.9], [0.55, 0.85], [0.8, 0.3], [0.31, 0.12]])
    dg0 = ElasticDG(m, p, *model0)
    data, _, _ = OA.record(dg0, dt, nsteps, ricker, xs, OA.receivers(dg0, rec))
    return m, p, model, dt, nsteps, ricker, xs, rec, data


def _gpu(lib, m, p, model, xs):
    return lib.slt_mesh_create(m["cell2vert"], m["cellxy"], p, *model, xs)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_record_matches_oracle(lib, p):
    import torch
    m, p, model, dt, nsteps, ricker, xs, rec, data = _problem(p=p)
    mesh = _gpu(lib, m, p, model, xs)
    r = lib.slt_receivers_create(mesh, rec)
    tr = torch.zeros((nsteps, len(rec), 2), dtype=torch.float64, device="cuda")
    lib.slt_record(mesh, None, r, torch.tensor(ricker, device="cuda"), dt, nsteps, tr)
    dg = ElasticDG(m, p, *model)
    want, _, _ = OA.record(dg, dt, nsteps, ricker, xs, OA.receivers(dg, rec))
    assert rel_l2(tr.cpu().numpy(), want) < 1e-11


@pytest.mark.parametrize("p,tiled,k", [(1, False, 7), (2, False, 30), (2, True, 7), (3, True, 11),
                                       (1, False, -7), (2, True, -7), (3, False, -30)])
def test_adjoint_matches_oracle(lib, p, tiled, k):
    import torch
    m, p, model, dt, nsteps, ricker, xs, rec, data = _problem(p=p)
    mesh = _gpu(lib, m, p, model, xs)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,)) if tiled else None
    r = lib.slt_receivers_create(mesh, rec)
    g = torch.zeros((3, m["cell2vert"].shape[0]), dtype=torch.float64, device="cuda")
    J = lib.slt_adjoint(mesh, sched, r, torch.tensor(ricker, device="cuda"), dt, nsteps,
                        torch.tensor(data, device="cuda"), k, g)
    dg = ElasticDG(m, p, *model)
    Jo, *go = OA.gradient(dg, dt, nsteps, ricker, xs, rec, data)
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    g = g.cpu().numpy()
    for kk in range(3):
        assert rel_l2(g[kk], go[kk]) < 1e-10, (kk, rel_l2(g[kk], go[kk]))


def test_gpu_gradient_matches_central_differences(lib):
    import torch
    m, p, model, dt, nsteps, ricker, xs, rec, data = _problem(p=2, nsteps=40)
    mesh = _gpu(lib, m, p, model, xs)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,))
    r = lib.slt_receivers_create(mesh, rec)
    rk, dd = torch.tensor(ricker, device="cuda"), torch.tensor(data, device="cuda")
    g = torch.zeros((3, m["cell2vert"].shape[0]), dtype=torch.float64, device="cuda")
    lib.slt_adjoint(mesh, sched, r, rk, dt, nsteps, dd, 10, g)
    g = g.cpu().numpy()
    scratch = torch.zeros_like(torch.tensor(g, device="cuda"))
    rng = np.random.default_rng(21)
    for _ in range(10):   # ten seeded random directions
        d = [a * rng.uniform(-1, 1, a.shape) for a in model]
        eps = 1e-5
        Js = []
        for sgn in (1, -1):
            lib.slt_mesh_set_material(mesh, *[a + sgn * eps * b for a, b in zip(model, d)])
            Js.append(lib.slt_adjoint(mesh, sched, r, rk, dt, nsteps, dd, 10, scratch))
        lib.slt_mesh_set_material(mesh, *model)
        fd = (Js[0] - Js[1]) / (2 * eps)
        ad = sum(g[k] @ d[k] for k in range(3))
        assert abs(fd - ad) <= 1e-7 * abs(ad), (fd, ad)


def test_autograd_function_sums_shots(lib):
    import torch
    from paper_1708_03183_gb300.autograd import MisfitProblem
    m, p, model, dt, nsteps, ricker, xs, rec, data0 = _problem(p=1, nsteps=25)
    shots = np.array([[0.5, 0.5], [0.3, 0.7]])
    dg0 = ElasticDG(m, p, *synth.homogeneous(m))
    data = np.stack([OA.record(dg0, dt, nsteps, ricker, s, OA.receivers(dg0, rec))[0] for s in shots])
    mesh = _gpu(lib, m, p, model, shots[0])
    prob = MisfitProblem(mesh, None, rec, shots, torch.tensor(data, device="cuda"),
                         torch.tensor(ricker, device="cuda"), dt, nsteps, checkpoint_every=6)
    params = [torch.tensor(a, requires_grad=True) for a in model]
    J = prob(*params)
    J.backward()
    dg = ElasticDG(m, p, *model)
    want_J, want_g = 0.0, np.zeros((3, dg.nc))
    for s, xy in enumerate(shots):
        Jo, *go = OA.gradient(dg, dt, nsteps, ricker, xy, rec, data[s])
        want_J += Jo
        want_g += np.array(go)
    assert abs(J.item() - want_J) <= 1e-10 * want_J
    for k in range(3):
        assert rel_l2(params[k].grad.numpy(), want_g[k]) < 1e-10


def _shots_problem(p, nsteps=25, nshots=3):
    m, p, model, dt, nsteps, ricker, xs, rec, _ = _problem(p=p, nsteps=nsteps)
    shots = np.array([[0.5, 0.5], [0.3, 0.7], [0.77, 0.21], [0.4, 0.33]])[:nshots]
    dg0 = ElasticDG(m, p, *synth.homogeneous(m))
    data = np.stack([OA.record(dg0, dt, nsteps, ricker, s, OA.receivers(dg0, rec))[0] for s in shots])
    return m, p, model, dt, nsteps, ricker, rec, shots, data


@pytest.mark.parametrize("p,tiled,k", [(1, False, 6), (2, True, 5), (2, False, 25), (3, True, 9)])
def test_many_shots_adjoint_matches_oracle(lib, p, tiled, k):
    # several shots in one call, untiled or on the schedule's tiles (reverse sweep included): the
    # sum over the shots of the oracle's discrete-adjoint misfit and gradient
    import torch
    m, p, model, dt, nsteps, ricker, rec, shots, data = _shots_problem(p)
    mesh = _gpu(lib, m, p, model, shots[0])
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,)) if tiled else None
    r = lib.slt_receivers_create(mesh, rec)
    dd = torch.tensor(np.ascontiguousarray(data.transpose(1, 0, 2, 3)), device="cuda")
    g = torch.zeros((3, m["cell2vert"].shape[0]), dtype=torch.float64, device="cuda")
    J = lib.slt_adjoint_batched(mesh, sched, r, shots, torch.tensor(ricker, device="cuda"), dt, nsteps, dd, k, g)
    dg = ElasticDG(m, p, *model)
    want_J, want_g = 0.0, np.zeros((3, dg.nc))
    for s, xy in enumerate(shots):
        Jo, *go = OA.gradient(dg, dt, nsteps, ricker, xy, rec, data[s])
        want_J += Jo
        want_g += np.array(go)
    assert abs(J - want_J) <= 1e-10 * want_J
    g = g.cpu().numpy()
    for kk in range(3):
        assert rel_l2(g[kk], want_g[kk]) < 1e-10, (kk, rel_l2(g[kk], want_g[kk]))


def test_many_shots_record_matches_single_shots(lib):
    import torch
    m, p, model, dt, nsteps, ricker, rec, shots, _ = _shots_problem(2)
    mesh = _gpu(lib, m, p, model, shots[0])
    r = lib.slt_receivers_create(mesh, rec)
    rk = torch.tensor(ricker, device="cuda")
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(9,))
    for sc in (None, sched):
        tr = torch.zeros((nsteps, len(shots), len(rec), 2), dtype=torch.float64, device="cuda")
        lib.slt_record_batched(mesh, sc, r, shots, rk, dt, nsteps, tr)
        dg = ElasticDG(m, p, *model)
        for s, xy in enumerate(shots):
            want, _, _ = OA.record(dg, dt, nsteps, ricker, xy, OA.receivers(dg, rec))
            assert rel_l2(tr[:, s].cpu().numpy(), want) < 1e-11


def test_tiled_and_untiled_many_shot_gradients_agree(lib):
    import torch
    m, p, model, dt, nsteps, ricker, rec, shots, data = _shots_problem(2, nsteps=30, nshots=4)
    mesh = _gpu(lib, m, p, model, shots[0])
    r = lib.slt_receivers_create(mesh, rec)
    rk = torch.tensor(ricker, device="cuda")
    dd = torch.tensor(np.ascontiguousarray(data.transpose(1, 0, 2, 3)), device="cuda")
    out = []
    for sc in (None, lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=12, split=(9,), shots_per_cta=2)):
        g = torch.zeros((3, m["cell2vert"].shape[0]), dtype=torch.float64, device="cuda")
        J = lib.slt_adjoint_batched(mesh, sc, r, shots, rk, dt, nsteps, dd, 7, g)
        out.append((J, g.cpu().numpy()))
    assert abs(out[0][0] - out[1][0]) <= 1e-12 * out[0][0]
    assert rel_l2(out[1][1], out[0][1]) < 1e-12


def test_tiled_adjoint_needs_the_velocity_stress_fusion(lib):
    import torch
    m, p, model, dt, nsteps, ricker, rec, shots, data = _shots_problem(1, nsteps=5, nshots=2)
    mesh = _gpu(lib, m, p, model, shots[0])
    r = lib.slt_receivers_create(mesh, rec)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=16, split=(3, 9))
    g = torch.zeros((3, m["cell2vert"].shape[0]), dtype=torch.float64, device="cuda")
    dd = torch.zeros((nsteps, 2, len(rec), 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.SltError) as e:
        lib.slt_adjoint_batched(mesh, sched, r, shots, torch.tensor(ricker, device="cuda"), dt, nsteps, dd, 5, g)
    assert e.value.code == -6
