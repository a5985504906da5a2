"""Pin of the oracle's discrete adjoint: its gradient of the seismogram misfit with respect to
per-cell rho, lambda, mu matches central finite differences of the misfit itself."""
import numpy as np
import pytest

import synth
from oracle import adjoint as OA
from oracle.dg import ElasticDG


def _setup(p=2, nx=6, ny=5, nsteps=30, seed=3):
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
    rec = np.array([[0.2, 0.9], [0.55, 0.85], [0.8, 0.3]])
    dg0 = ElasticDG(m, p, *model0)
    data, _, _ = OA.record(dg0, dt, nsteps, ricker, xs, OA.receivers(dg0, rec))
    return m, p, model, dt, nsteps, ricker, xs, rec, data


def _J(m, p, model, dt, nsteps, ricker, xs, rec, data):
    dg = ElasticDG(m, p, *model)
    tr, _, _ = OA.record(dg, dt, nsteps, ricker, xs, OA.receivers(dg, rec))
    return OA.misfit(tr, data, dt)


@pytest.mark.parametrize("p", [1, 2])
def test_adjoint_gradient_matches_central_differences(p):
    m, p, model, dt, nsteps, ricker, xs, rec, data = _setup(p=p)
    dg = ElasticDG(m, p, *model)
    J, g_rho, g_lam, g_mu = OA.gradient(dg, dt, nsteps, ricker, xs, rec, data)
    assert J > 0
    assert np.isclose(J, _J(m, p, model, dt, nsteps, ricker, xs, rec, data), rtol=1e-14)
    rng = np.random.default_rng(7)
    for _ in range(10):   # ten seeded random directions
        d = [a * rng.uniform(-1, 1, a.shape) for a in model]
        # central differences: truncation error O(eps^2) (1e-9 here), far below a wrong term
        eps = 1e-5
        Jp = _J(m, p, [a + eps * b for a, b in zip(model, d)], dt, nsteps, ricker, xs, rec, data)
        Jm = _J(m, p, [a - eps * b for a, b in zip(model, d)], dt, nsteps, ricker, xs, rec, data)
        fd = (Jp - Jm) / (2 * eps)
        ad = g_rho @ d[0] + g_lam @ d[1] + g_mu @ d[2]
        assert abs(fd - ad) <= 1e-7 * abs(ad), (fd, ad)


def test_each_parameter_gradient_separately():
    m, p, model, dt, nsteps, ricker, xs, rec, data = _setup(p=1, nsteps=20)
    dg = ElasticDG(m, p, *model)
    J, *g = OA.gradient(dg, dt, nsteps, ricker, xs, rec, data)
    rng = np.random.default_rng(11)
    for k in range(3):
        d = [np.zeros_like(a) for a in model]
        d[k] = model[k] * rng.uniform(-1, 1, model[k].shape)
        eps = 1e-5
        Jp = _J(m, p, [a + eps * b for a, b in zip(model, d)], dt, nsteps, ricker, xs, rec, data)
        Jm = _J(m, p, [a - eps * b for a, b in zip(model, d)], dt, nsteps, ricker, xs, rec, data)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g[k] @ d[k]) <= 1e-7 * abs(fd), (k, fd, g[k] @ d[k])
