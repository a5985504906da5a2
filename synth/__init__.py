"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package holds no arithmetic of the discontinuous-Galerkin method or of the sparse
tiling inspector: it only generates meshes (topology and vertex coordinates), per-cell
material parameters, the explosive-source time series and the configuration table.
Both the CUDA library and the oracle derive everything else (facets, geometry, reference
element matrices, schedules) independently from these arrays.
"""
from .mesh import make_mesh, cell_centroids_for_materials
from .materials import homogeneous, layered, perturb
from .source import ricker_series, cfl_dt
from .configs import CONFIGS, build_config, multi_configs

__all__ = ["make_mesh", "cell_centroids_for_materials", "homogeneous", "layered", "perturb",
           "ricker_series", "cfl_dt", "CONFIGS", "build_config", "multi_configs"]
