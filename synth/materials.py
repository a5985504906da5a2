"""Per-cell isotropic material parameters (rho, lambda, mu) for the synthetic workloads."""
import numpy as np
from .mesh import cell_centroids_for_materials


def homogeneous(mesh, rho=1.0, lam=2.0, mu=1.0):
    nc = mesh["cell2vert"].shape[0]
    return (np.full(nc, rho), np.full(nc, lam), np.full(nc, mu))


def layered(mesh):
    """Three equal horizontal bands; top vp=1.5, rho=1.0; middle vp=3.0, rho=2.0;
    bottom vp=4.5, rho=2.5; vs = vp/sqrt(3), so mu = rho*vs^2 and lambda = rho*vp^2 - 2*mu."""
    y = cell_centroids_for_materials(mesh)[:, 1]
    Ly = mesh["Ly"]
    band = np.where(y > 2.0 * Ly / 3.0, 0, np.where(y > Ly / 3.0, 1, 2))
    vp = np.array([1.5, 3.0, 4.5])[band]
    rho = np.array([1.0, 2.0, 2.5])[band]
    mu = rho * vp * vp / 3.0
    lam = rho * vp * vp - 2.0 * mu
    return rho, lam, mu


def perturb(params, seed, amp=0.05):
    """Multiply each per-cell parameter by (1 + amp*U[-1,1]), seeded."""
    rng = np.random.default_rng(seed)
    return tuple(p * (1.0 + amp * rng.uniform(-1.0, 1.0, size=p.shape)) for p in params)
