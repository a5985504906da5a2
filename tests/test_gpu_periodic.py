"""Periodic meshes on the GPU path (no exterior facets, so the exterior-facet loops are empty):
parity with the oracle, and convergence of the tiled GPU chain to an analytic elastic plane
wave at the DG order (a property of the method that holds at any size)."""
import numpy as np
import pytest

import synth
from oracle.dg import ElasticDG
from tests.helpers import TOL, rel_l2

pytestmark = pytest.mark.gpu


def _mesh(lib, m, p, mat):
    return lib.slt_mesh_create(m["cell2vert"], m["cellxy"], p, *mat)


@pytest.mark.parametrize("p,ts", [(1, 8), (2, 16), (3, 5)])
def test_periodic_mesh_matches_oracle(lib, p, ts):
    import torch
    m = synth.make_mesh(10, 8, seed=6, periodic=True)
    nc = m["cell2vert"].shape[0]
    rng = np.random.default_rng(p)
    mat = (rng.uniform(1, 2, nc), rng.uniform(1, 2, nc), rng.uniform(1, 2, nc))
    Np = (p + 1) * (p + 2) // 2
    v0 = rng.standard_normal((nc, 2, Np))
    s0 = rng.standard_normal((nc, 3, Np))
    dg = ElasticDG(m, p, *mat)
    dt = 0.5 * synth.cfl_dt(m, float(np.max(np.sqrt((mat[1] + 2 * mat[2]) / mat[0]))), p)
    vo, so = dg.run(v0.copy(), s0.copy(), dt, 6)
    mesh = _mesh(lib, m, p, mat)
    assert lib.slt_mesh_info(mesh)["nfe"] == 0
    for sched in (None, lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=ts, split=(9,))):
        v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
        lib.slt_execute(mesh, sched, v, s, None, dt, 6)
        assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL


@pytest.mark.parametrize("p", [1, 2, 3])
def test_plane_wave_convergence_on_the_gpu(lib, p):
    # P-wave v = d sin(theta), sigma = -(lambda I + 2 mu d d^T) sin(theta) / c_p,
    # theta = 2 pi k.x - omega t, k = (1, 1), on periodic jittered meshes; nodal errors weighted
    # by cell area; centered-flux DG converges at order >= p (dt ~ h keeps the time error small)
    import torch
    rho, lam, mu = 1.0, 2.0, 1.0
    cp = np.sqrt((lam + 2 * mu) / rho)
    k = np.array([1.0, 1.0])
    d = k / np.linalg.norm(k)
    om = 2 * np.pi * np.linalg.norm(k) * cp
    Sm = (lam * np.eye(2) + 2 * mu * np.outer(d, d)) / cp
    T = 0.1
    nodes = np.array([(i / p, j / p) for j in range(p + 1) for i in range(p + 1 - j)])
    errs = []
    for N in (8, 16, 32):
        m = synth.make_mesh(N, N, seed=4, periodic=True)
        nc = m["cell2vert"].shape[0]
        X = m["cellxy"]
        xy = X[:, None, 0, :] + nodes[None, :, 0:1] * (X[:, None, 1, :] - X[:, None, 0, :]) \
            + nodes[None, :, 1:2] * (X[:, None, 2, :] - X[:, None, 0, :])
        area = 0.5 * np.abs((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1])
                            - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1]))
        th = lambda t: 2 * np.pi * (xy[..., 0] * k[0] + xy[..., 1] * k[1]) - om * t
        vex = lambda t: np.stack([d[0] * np.sin(th(t)), d[1] * np.sin(th(t))], 1)
        sex = lambda t: -np.stack([Sm[0, 0] * np.sin(th(t)), Sm[1, 1] * np.sin(th(t)), Sm[0, 1] * np.sin(th(t))], 1)
        nsteps = int(np.ceil(T / (0.5 * synth.cfl_dt(m, cp, p))))
        dt = T / nsteps
        mesh = _mesh(lib, m, p, (np.full(nc, rho), np.full(nc, lam), np.full(nc, mu)))
        sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=32, split=(9,))
        v = torch.tensor(np.ascontiguousarray(vex(-dt / 2)), device="cuda")
        s = torch.tensor(np.ascontiguousarray(sex(0.0)), device="cuda")
        lib.slt_execute(mesh, sched, v, s, None, dt, nsteps)
        e = v.cpu().numpy() - vex(T - dt / 2)
        errs.append(np.sqrt(np.sum(area[:, None, None] * e ** 2) / e.shape[2]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= p - 0.1, (errs, rates)
