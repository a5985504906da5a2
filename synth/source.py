"""Explosive-source time series and the explicit time-step size (inputs to both sides)."""
import numpy as np


def ricker_series(f0, dt, nsteps, t0=None):
    """Ricker wavelet g(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t0 = 1/f0,
    sampled at the stress-update mid-points t_{n+1/2} = (n + 1/2) dt, n = 0..nsteps-1."""
    if t0 is None:
        t0 = 1.0 / f0
    t = (np.arange(nsteps) + 0.5) * dt
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def cfl_dt(mesh, vp_max, p, cfl=0.5):
    """dt = cfl * min_K(2 r_K) / (vp_max (2p+1)), r_K the inradius of cell K."""
    x = mesh["cellxy"]
    a = np.linalg.norm(x[:, 1] - x[:, 0], axis=1)
    b = np.linalg.norm(x[:, 2] - x[:, 1], axis=1)
    c = np.linalg.norm(x[:, 0] - x[:, 2], axis=1)
    e1, e2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    area = 0.5 * np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    r = 2.0 * area / (a + b + c)
    return cfl * float(np.min(2.0 * r)) / (vp_max * (2 * p + 1))
