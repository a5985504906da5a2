"""The synthetic workloads have the sizes and structure of the configurations they stand in for:
cell and facet counts of the structured triangulations (closed forms), the mesh's geometric
validity, the layered material, the uneven-mesh table and the source series."""
import numpy as np
import pytest

import synth
from oracle.dg import _facets


def _counts(nx, ny):
    # nx x ny squares cut into two triangles: cells, interior and boundary edges
    edges = nx * (ny + 1) + (nx + 1) * ny + nx * ny
    boundary = 2 * (nx + ny)
    return 2 * nx * ny, edges - boundary, boundary


@pytest.mark.parametrize("name,nx,ny", [("tiny", 16, 16), ("small_p2", 40, 24), ("adjoint", 448, 224),
                                        ("large", 708, 354), ("p4", 500, 250)])
def test_cell_and_facet_counts(name, nx, ny):
    cfg = synth.build_config(name, nx=nx, ny=ny, nsteps=1)
    c2v = cfg["mesh"]["cell2vert"]
    inter, exter = _facets(c2v)
    assert (c2v.shape[0], inter.shape[0], exter.shape[0]) == _counts(nx, ny)


def test_the_large_mesh():
    cfg = synth.build_config("large", nsteps=1)
    m = cfg["mesh"]
    x = m["cellxy"]
    assert m["cell2vert"].shape[0] == 1_000_000 and cfg["p"] == 2
    # counter-clockwise cells of positive area tiling the 300 x 150 domain
    e1, e2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    assert area.min() > 0 and np.isclose(area.sum(), 300.0 * 150.0, rtol=1e-12)
    assert np.isclose(x[..., 0].min(), 0) and np.isclose(x[..., 0].max(), 300.0)
    assert np.isclose(x[..., 1].min(), 0) and np.isclose(x[..., 1].max(), 150.0)


def test_layered_material_bands():
    cfg = synth.build_config("small_p2", nsteps=1)
    x = cfg["mesh"]["cellxy"].mean(axis=1)
    vp = np.sqrt((cfg["lam"] + 2 * cfg["mu"]) / cfg["rho"])
    vs = np.sqrt(cfg["mu"] / cfg["rho"])
    Ly = 15.0
    for lo, hi, v, r in ((2 * Ly / 3, Ly, 1.5, 1.0), (Ly / 3, 2 * Ly / 3, 3.0, 2.0), (0, Ly / 3, 4.5, 2.5)):
        sel = (x[:, 1] > lo + 0.5) & (x[:, 1] < hi - 0.5)   # away from the band edges
        assert sel.any()
        assert np.allclose(vp[sel], v) and np.allclose(cfg["rho"][sel], r)
        assert np.allclose(vs[sel], v / np.sqrt(3.0)) and np.allclose(cfg["lam"][sel], cfg["mu"][sel])


def test_perturbed_material_stays_within_five_percent():
    base = synth.build_config("small_p2", nsteps=1)
    cfg = synth.build_config("small_p2", nsteps=1, material="layered_perturbed")
    for k in ("rho", "lam", "mu"):
        ratio = cfg[k] / base[k]
        assert ratio.min() >= 0.95 and ratio.max() <= 1.05 and ratio.std() > 0.01


def test_uneven_mesh_table():
    cfgs = synth.multi_configs(16, nsteps=1)
    nc = np.array([c["mesh"]["cell2vert"].shape[0] for c in cfgs])
    assert len(cfgs) == 16 and nc.min() >= 0.8 * 20000 and nc.max() <= 1.2 * 400000
    assert [c["p"] for c in cfgs] == [1 + i % 3 for i in range(16)]
    assert nc.sum() == 2749128


def test_ricker_series_peak_and_shape():
    f0, dt = 8.0, 1e-3
    g = synth.ricker_series(f0, dt, 400)
    t = (np.arange(400) + 0.5) * dt
    k = int(np.argmax(g))
    assert abs(t[k] - 1.0 / f0) <= dt and g[k] <= 1.0 and g[k] > 0.99
    # zero crossings of (1 - 2 pi^2 f0^2 (t - t0)^2) at t0 +- 1/(sqrt(2) pi f0)
    z = 1.0 / f0 + np.array([-1, 1]) / (np.sqrt(2.0) * np.pi * f0)
    for zt in z:
        i = int(zt / dt - 0.5)
        assert g[i] * g[i + 1] <= 0
