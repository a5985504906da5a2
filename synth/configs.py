"""The synthetic workloads: sizes, materials and source placement.

Meshes use seed 0 (renumbering seed 1); material perturbation seed 2.  Every workload is an
explosive point source with a Ricker time function, a free surface on the whole boundary,
and a CFL-0.5 explicit time step.
"""
import numpy as np
from .mesh import make_mesh
from .materials import homogeneous, layered, perturb
from .source import ricker_series, cfl_dt

CONFIGS = {
    # 16x16 squares on the unit square, 512 triangles, P1, homogeneous, 100 steps, ts=64
    "tiny": dict(nx=16, ny=16, Lx=1.0, Ly=1.0, p=1, material="homogeneous", f0=5.0,
                 src=(0.5, 0.5), nsteps=100, ts=64),
    # 1000x500 squares on 300x150, 1.0M triangles, P2, three layers, 200 steps, ts 256..4096
    "large": dict(nx=1000, ny=500, Lx=300.0, Ly=150.0, p=2, material="layered", f0=8.0,
                  src=(150.0, 142.5), nsteps=200, ts=1024),
    # 500x250 squares on 300x150, 250k triangles, P4, three layers, 200 steps
    "p4": dict(nx=500, ny=250, Lx=300.0, Ly=150.0, p=4, material="layered", f0=8.0,
               src=(150.0, 142.5), nsteps=200, ts=512),
    # 448x224 squares on 300x150, 200k triangles, P2, layered +-5% per cell (gradient workload)
    "adjoint": dict(nx=448, ny=224, Lx=300.0, Ly=150.0, p=2, material="layered_perturbed",
                    f0=8.0, src=(150.0, 142.5), nsteps=1000, ts=512),
    # the same generator at small sizes, for parity tests spanning several tiles
    "small_p2": dict(nx=40, ny=24, Lx=30.0, Ly=15.0, p=2, material="layered", f0=8.0,
                     src=(15.0, 14.25), nsteps=20, ts=64),
    "small_p3": dict(nx=24, ny=16, Lx=30.0, Ly=15.0, p=3, material="layered", f0=8.0,
                     src=(15.0, 14.25), nsteps=10, ts=48),
    "small_p4": dict(nx=20, ny=12, Lx=30.0, Ly=15.0, p=4, material="layered", f0=8.0,
                     src=(15.0, 14.25), nsteps=8, ts=40),
}


def build_config(name, **override):
    """Materialise a workload: mesh, p, per-cell (rho, lam, mu), dt, Ricker series, source."""
    c = dict(CONFIGS[name])
    c.update(override)
    mesh = make_mesh(c["nx"], c["ny"], c["Lx"], c["Ly"], seed=c.get("seed", 0))
    if c["material"] == "homogeneous":
        rho, lam, mu = homogeneous(mesh)
    elif c["material"] == "layered":
        rho, lam, mu = layered(mesh)
    elif c["material"] == "layered_perturbed":
        rho, lam, mu = perturb(layered(mesh), seed=2)
    else:
        raise ValueError(c["material"])
    vp_max = float(np.max(np.sqrt((lam + 2.0 * mu) / rho)))
    dt = cfl_dt(mesh, vp_max, c["p"])
    ricker = ricker_series(c["f0"], dt, c["nsteps"])
    return dict(name=name, mesh=mesh, p=c["p"], rho=rho, lam=lam, mu=mu, dt=dt,
                ricker=ricker, src=np.array(c["src"], dtype=np.float64), nsteps=c["nsteps"],
                ts=c["ts"])


def multi_configs(n=16, seed=4, lo=20000, hi=400000, nsteps=20):
    """Uneven meshes for the many-mesh form: cell counts log-uniform in [lo, hi] (seeded), degree
    1 + (i mod 3), each an nx x nx/2 grid of squares on 300x150 with its own mesh seed, layered
    material and the large workload's source."""
    rng = np.random.default_rng(seed)
    ncells = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    out = []
    for i, nc in enumerate(ncells):
        nx = max(int(round(np.sqrt(nc))), 4)
        out.append(build_config("large", nx=nx, ny=max(nx // 2, 2), p=1 + i % 3, nsteps=nsteps, seed=100 + i))
    return out
