"""Seeded unstructured triangle meshes of a rectangle.

The workloads of the paper (Section 7.4) are 2-D rectangles tessellated with unstructured
triangles.  These meshes stand in for them: an nx-by-ny grid of squares, each cut along a
seeded-random diagonal, interior vertices jittered by up to +-0.2 of the spacing, and cells,
vertices and the local vertex order of every cell randomly renumbered, so that nothing in the
CUDA path or the oracle can rely on a structured numbering.

Every cell is counter-clockwise in its local vertex order.  For a periodic mesh the vertices on
opposite sides are identified (the topology wraps around) and ``cellxy`` holds each cell's
unwrapped vertex coordinates.
"""
import numpy as np


def make_mesh(nx, ny, Lx=1.0, Ly=1.0, seed=0, periodic=False, jitter=0.2, renumber=True):
    """Return a dict with the mesh arrays.

    cell2vert : int32 [Nc, 3]   vertex ids of each cell, counter-clockwise
    cellxy    : float64 [Nc, 3, 2]  coordinates of those vertices (unwrapped when periodic)
    coords    : float64 [Nv, 2] vertex coordinates (None when periodic)
    nvert     : number of vertices
    """
    if periodic and (nx < 3 or ny < 3):
        raise ValueError("periodic meshes need nx, ny >= 3")
    rng = np.random.default_rng(seed)
    hx, hy = Lx / nx, Ly / ny
    if periodic:
        vx, vy = nx, ny
    else:
        vx, vy = nx + 1, ny + 1
    ii, jj = np.meshgrid(np.arange(vx), np.arange(vy), indexing="xy")
    base = np.stack([ii.ravel() * hx, jj.ravel() * hy], axis=1)
    jit = np.zeros_like(base)
    d = rng.uniform(-jitter, jitter, size=base.shape) * np.array([hx, hy])
    if periodic:
        jit = d
    else:
        interior = ((ii.ravel() > 0) & (ii.ravel() < nx) & (jj.ravel() > 0) & (jj.ravel() < ny))
        jit[interior] = d[interior]
    diag = rng.integers(0, 2, size=(ny, nx))

    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    I, J = I.ravel(), J.ravel()
    corners = {"a": (I, J), "b": (I + 1, J), "c": (I + 1, J + 1), "d": (I, J + 1)}

    def vid(i, j):
        if periodic:
            return (j % ny) * nx + (i % nx)
        return j * (nx + 1) + i

    def vpos(i, j):
        return np.stack([i * hx, j * hy], axis=1) + jit[vid(i, j)]

    dg = diag.ravel()
    # diagonal a-c: (a,b,c), (a,c,d); diagonal b-d: (a,b,d), (b,c,d); all counter-clockwise
    t0 = [np.where(dg == 0, corners[k0][q], corners[k1][q]) for k0, k1 in (("a", "a"), ("b", "b"), ("c", "d")) for q in (0, 1)]
    t1 = [np.where(dg == 0, corners[k0][q], corners[k1][q]) for k0, k1 in (("a", "b"), ("c", "c"), ("d", "d")) for q in (0, 1)]
    tri_i = np.empty((2 * nx * ny, 3), dtype=np.int64)
    tri_j = np.empty((2 * nx * ny, 3), dtype=np.int64)
    for k in range(3):
        tri_i[0::2, k], tri_j[0::2, k] = t0[2 * k], t0[2 * k + 1]
        tri_i[1::2, k], tri_j[1::2, k] = t1[2 * k], t1[2 * k + 1]
    cell2vert = vid(tri_i, tri_j)
    cellxy = np.stack([vpos(tri_i[:, k], tri_j[:, k]) for k in range(3)], axis=1)
    cells = cell2vert
    nvert = vx * vy
    coords = None if periodic else (base + jit)

    if renumber:
        rng2 = np.random.default_rng(seed + 1)
        cperm = rng2.permutation(len(cells))          # new cell k is old cell cperm[k]
        vperm = rng2.permutation(nvert)               # old vertex v becomes vperm[v]
        rot = rng2.integers(0, 3, size=len(cells))    # cyclic rotation of local vertex order
        cell2vert = vperm[cell2vert[cperm]]
        cellxy = cellxy[cperm]
        idx = (np.arange(3)[None, :] + rot[:, None]) % 3
        cell2vert = np.take_along_axis(cell2vert, idx, axis=1)
        cellxy = np.take_along_axis(cellxy, idx[:, :, None], axis=1)
        if coords is not None:
            newc = np.empty_like(coords)
            newc[vperm] = coords
            coords = newc

    e1 = cellxy[:, 1] - cellxy[:, 0]
    e2 = cellxy[:, 2] - cellxy[:, 0]
    cross = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    if not np.all(cross > 0):
        raise RuntimeError("generated a degenerate or clockwise cell")
    return {
        "cell2vert": np.ascontiguousarray(cell2vert, dtype=np.int32),
        "cellxy": np.ascontiguousarray(cellxy),
        "coords": None if coords is None else np.ascontiguousarray(coords),
        "nvert": int(nvert), "nx": nx, "ny": ny, "Lx": Lx, "Ly": Ly, "periodic": periodic,
    }


def cell_centroids_for_materials(mesh):
    """Cell centroids, used only to place material layers (an input, not the method)."""
    return mesh["cellxy"].mean(axis=1)
