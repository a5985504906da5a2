"""Pins of the oracle's DG chain against facts fixed by mathematics, not by the oracle itself.

Each check is chosen so that a plausible slip (a dropped facet term, a sign, a transposed
cross-face matrix, a wrong Taylor coefficient, a wrong geometric factor) fails one of them.
"""
import numpy as np
import pytest

import synth
from oracle import refelem
from oracle.dg import ElasticDG, taylor_leapfrog_step


# ----------------------------------------------------------------------- reference element
def test_p1_mass_is_textbook():
    # P1 Lagrange mass matrix on a triangle of area 1/2: (area/12) [[2,1,1],[1,2,1],[1,1,2]]
    M = refelem.matrices(1)["M"]
    assert np.allclose(M, np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 24.0, rtol=0, atol=1e-16)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_reference_identities(p):
    R = refelem.matrices(p)
    X = R["nodes"]
    # nodal: phi_j(node_i) = delta_ij
    assert np.allclose(refelem.eval_basis(p, X[:, 0], X[:, 1]), np.eye(R["Np"]), atol=1e-12)
    # partition of unity: total mass = area, derivative of a constant vanishes, edge length 1
    assert abs(R["M"].sum() - 0.5) < 1e-14
    assert np.allclose(R["Sr"].sum(axis=1), 0, atol=1e-13)
    assert np.allclose(R["Ss"].sum(axis=1), 0, atol=1e-13)
    for f in range(3):
        assert abs(R["Fsame"][f].sum() - 1.0) < 1e-14
    # integration by parts on the reference triangle:
    #   int_T d(phi_i phi_j)/dr = int_face1 phi_i phi_j dt - int_face2 phi_i phi_j dt
    #   int_T d(phi_i phi_j)/ds = int_face1 phi_i phi_j dt - int_face0 phi_i phi_j dt
    F = R["Fsame"]
    assert np.allclose(R["Sr"] + R["Sr"].T, F[1] - F[2], atol=1e-14)
    assert np.allclose(R["Ss"] + R["Ss"].T, F[1] - F[0], atol=1e-14)
    # exchanging the two sides of a facet transposes the cross matrix
    for fa in range(3):
        for fb in range(3):
            for flip in (False, True):
                assert np.allclose(R["Fcross"][(fa, fb, flip)].T, R["Fcross"][(fb, fa, flip)], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_face_mass_matches_1d_quadrature(p):
    # the trace of the nodal basis on face 0 (s=0) is the 1-D Lagrange basis on the p+1
    # equispaced points: compare with Gauss-Legendre quadrature of those 1-D polynomials.
    R = refelem.matrices(p)
    face_nodes = [i for i, (r, s) in enumerate(R["nodes"]) if s == 0]
    t, w = np.polynomial.legendre.leggauss(p + 2)
    t, w = 0.5 * (t + 1), 0.5 * w
    pts = np.linspace(0, 1, p + 1)
    L = np.array([[np.prod([(tt - pts[m]) / (pts[k] - pts[m]) for m in range(p + 1) if m != k])
                   for k in range(p + 1)] for tt in t])
    M1 = (L * w[:, None]).T @ L
    assert np.allclose(R["Fsame"][0][np.ix_(face_nodes, face_nodes)], M1, atol=1e-14)


# ----------------------------------------------------------------------- mesh bookkeeping
@pytest.mark.parametrize("nx,ny", [(4, 3), (16, 16), (7, 11)])
def test_facet_counts(nx, ny):
    m = synth.make_mesh(nx, ny, seed=5)
    dg = ElasticDG(m, 1, *synth.homogeneous(m))
    total_edges = nx * (ny + 1) + (nx + 1) * ny + nx * ny
    assert len(dg.efacets) == 2 * (nx + ny)
    assert len(dg.ifacets) == total_edges - 2 * (nx + ny)
    counts = np.bincount(np.concatenate([dg.ifacets[:, 0], dg.ifacets[:, 2], dg.efacets[:, 0]]), minlength=dg.nc)
    assert np.all(counts == 3)
    assert np.all(dg.ifacets[:, 0] < dg.ifacets[:, 2])
    assert np.all(dg.ifacets[:, 4] == 1)  # counter-clockwise neighbours traverse an edge oppositely
    # the outward normals of the two sides are opposite
    n0 = dg.fn[dg.ifacets[:, 0], dg.ifacets[:, 1]]
    n1 = dg.fn[dg.ifacets[:, 2], dg.ifacets[:, 3]]
    assert np.allclose(n0, -n1, atol=1e-12)


# ----------------------------------------------------------------------- operator pins
def _dg(nx=6, ny=5, p=2, seed=1, material="random", periodic=False):
    m = synth.make_mesh(nx, ny, seed=seed, periodic=periodic)
    if material == "random":
        rng = np.random.default_rng(seed + 10)
        nc = m["cell2vert"].shape[0]
        rho, lam, mu = rng.uniform(1, 3, nc), rng.uniform(1, 3, nc), rng.uniform(1, 3, nc)
    else:
        rho, lam, mu = synth.homogeneous(m)
    return m, ElasticDG(m, p, rho, lam, mu)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_weak_and_strong_realisations_agree(p):
    _, dg = _dg(p=p)
    rng = np.random.default_rng(p)
    s = rng.standard_normal((dg.nc, 3, dg.Np))
    v = rng.standard_normal((dg.nc, 2, dg.Np))
    a, b = dg.apply_A(s, "strong"), dg.apply_A(s, "weak")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    a, b = dg.apply_B(v, "weak_tau"), dg.apply_B(v, "strong_tau")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_skew_adjoint_pair(p):
    # <u, A sigma>_{M_rho} = b(sigma, u) = -d(u, sigma) = -<sigma, B u>_{M_S}
    _, dg = _dg(p=p)
    rng = np.random.default_rng(10 + p)
    s = rng.standard_normal((dg.nc, 3, dg.Np))
    u = rng.standard_normal((dg.nc, 2, dg.Np))
    lhs = dg.inner_v(u, dg.apply_A(s))
    rhs = -dg.inner_s(s, dg.apply_B(u))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_p0_is_cell_centred_finite_volumes():
    # With p = 0 the DG chain is the cell-centred finite-volume scheme with the arithmetic mean
    # of the two cell stresses on each face (free surface: no boundary flux).  Written here
    # with explicit loops over cells and their edge neighbours found by shared vertex pairs.
    m, dg = _dg(nx=5, ny=4, p=0)
    X, c2v = m["cellxy"], m["cell2vert"]
    nc = len(c2v)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((nc, 3))
    v = rng.standard_normal((nc, 2))
    edge_owner = {}
    for c in range(nc):
        for f in range(3):
            edge_owner.setdefault(frozenset((int(c2v[c, f]), int(c2v[c, (f + 1) % 3]))), []).append((c, f))
    u_fv = np.zeros((nc, 2))
    e_fv = np.zeros((nc, 3))
    for c in range(nc):
        e1, e2 = X[c, 1] - X[c, 0], X[c, 2] - X[c, 0]
        area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        cen = X[c].mean(0)
        for f in range(3):
            nb = [o for o in edge_owner[frozenset((int(c2v[c, f]), int(c2v[c, (f + 1) % 3])))] if o[0] != c]
            if not nb:
                continue
            o = nb[0][0]
            a, b = X[c, f], X[c, (f + 1) % 3]
            L = np.linalg.norm(b - a)
            n = np.array([b[1] - a[1], a[0] - b[0]]) / L
            if n @ (a - cen) < 0:
                n = -n
            S = lambda k: np.array([[s[k, 0], s[k, 2]], [s[k, 2], s[k, 1]]])
            u_fv[c] += L * 0.5 * (S(c) + S(o)) @ n / (dg.rho[c] * area)
            dv = v[c] - v[o]
            e_fv[c] += -0.5 * L * np.array([dv[0] * n[0], dv[1] * n[1], dv[0] * n[1] + dv[1] * n[0]]) / area
    lam, mu = dg.lam[:, None], dg.mu[:, None]
    s_fv = np.stack([lam[:, 0] * (e_fv[:, 0] + e_fv[:, 1]) + 2 * mu[:, 0] * e_fv[:, 0],
                     lam[:, 0] * (e_fv[:, 0] + e_fv[:, 1]) + 2 * mu[:, 0] * e_fv[:, 1], mu[:, 0] * e_fv[:, 2]], 1)
    assert np.allclose(dg.apply_A(s[:, :, None])[:, :, 0], u_fv, rtol=1e-12, atol=1e-12)
    assert np.allclose(dg.apply_B(v[:, :, None])[:, :, 0], s_fv, rtol=1e-12, atol=1e-12)


def _nodes_xy(dg):
    Xn = dg.R["nodes"]
    return dg.X0[:, None, :] + np.einsum("cab,nb->cna", dg.jac, Xn)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_polynomial_fields_are_differentiated_exactly(p):
    # For a continuous global polynomial field of degree p the facet jumps vanish, so on cells
    # without an exterior facet A sigma = div(sigma)/rho and B v = C eps(v) at the nodes.
    m, dg = _dg(p=p)
    xy = _nodes_xy(dg)
    x, y = xy[..., 0], xy[..., 1]
    rng = np.random.default_rng(p)
    cf = rng.standard_normal((5, 3))
    P = lambda k: cf[k, 0] * x ** p + cf[k, 1] * x * y ** (p - 1) + cf[k, 2] * y
    Px = lambda k: cf[k, 0] * p * x ** (p - 1) + cf[k, 1] * y ** (p - 1)
    Py = lambda k: cf[k, 1] * (p - 1) * x * y ** max(p - 2, 0) * (p > 1) + cf[k, 2]
    sig = np.stack([P(0), P(1), P(2)], 1)
    u = dg.apply_A(sig)
    inner = np.setdiff1d(np.arange(dg.nc), dg.efacets[:, 0])
    div = np.stack([Px(0) + Py(2), Px(2) + Py(1)], 1) / dg.rho[:, None, None]
    assert np.allclose(u[inner], div[inner], rtol=1e-11, atol=1e-11)
    v = np.stack([P(3), P(4)], 1)
    E = np.stack([Px(3), Py(4), Py(3) + Px(4)], 1)
    assert np.allclose(dg.apply_B(v), dg.hooke(E), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2])
def test_discrete_energy_is_conserved(p):
    # E^n = 1/2 <v^{n+1/2}, M_rho v^{n-1/2}> + 1/2 <sigma^n, M_S sigma^n> is exactly invariant
    # because the step is a staggered leapfrog with a skew-adjoint operator pair.
    m, dg = _dg(nx=6, ny=6, p=p)
    rng = np.random.default_rng(7)
    v = rng.standard_normal((dg.nc, 2, dg.Np))
    s = rng.standard_normal((dg.nc, 3, dg.Np))
    dt = 0.2 * synth.cfl_dt(m, float(np.max(np.sqrt((dg.lam + 2 * dg.mu) / dg.rho))), p)
    E = []
    for _ in range(30):
        vn, sn = dg.step(v, s, dt)
        E.append(0.5 * dg.inner_v(vn, v) + 0.5 * dg.inner_s(s, s))
        v, s = vn, sn
    E = np.array(E)
    assert np.abs(E - E[0]).max() <= 1e-12 * abs(E[0])


def test_momentum_is_conserved_with_source():
    m, dg = _dg(nx=6, ny=5, p=2)
    rng = np.random.default_rng(8)
    v = rng.standard_normal((dg.nc, 2, dg.Np))
    s = rng.standard_normal((dg.nc, 3, dg.Np))
    mom = lambda v: np.einsum("c,cki,ij,j->k", dg.rho * dg.det, v, dg.R["M"], np.ones(dg.Np))
    p0 = mom(v)
    src = dg.source_vector(np.array([0.5, 0.5]))
    for n in range(10):
        v, s = dg.step(v, s, 1e-3, g=1.0 + n, src=src)
    assert np.allclose(mom(v), p0, rtol=1e-12, atol=1e-12)


def test_taylor_leapfrog_is_fourth_order_scalar():
    # v' = -w s, s' = w v, exact s = sin(wt), v = cos(wt); the truncated Taylor leapfrog with
    # the dt^2/24 correction is fourth-order accurate (a coefficient other than 1/24 gives 2).
    w, T = 3.0, 2.0
    errs = []
    for N in (50, 100, 200):
        dt = T / N
        v, s = np.array([np.cos(-w * dt / 2)]), np.array([0.0])
        for _ in range(N):
            v, s = taylor_leapfrog_step(lambda q: -w * q, lambda q: w * q, v, s, dt)
        errs.append(abs(s[0] - np.sin(w * T)) + abs(v[0] - np.cos(w * (T - dt / 2))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.9), rates


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_plane_wave_convergence_periodic(p):
    # P-wave v = d sin(theta), sigma = -(lambda I + 2 mu d d^T) sin(theta)/c_p on a periodic
    # jittered mesh; theta = 2 pi k.x - omega t, k = (1, 1).  Centered-flux DG converges at
    # order >= p (dt ~ h, so the fourth-order time error is sub-dominant).
    rho, lam, mu = 1.0, 2.0, 1.0
    cp = np.sqrt((lam + 2 * mu) / rho)
    k = np.array([1.0, 1.0])
    d = k / np.linalg.norm(k)
    om = 2 * np.pi * np.linalg.norm(k) * cp
    T = 0.1
    errs = []
    for N in (8, 16, 32):
        m = synth.make_mesh(N, N, seed=4, periodic=True)
        dg = ElasticDG(m, p, *synth.homogeneous(m, rho, lam, mu))
        nsteps = int(np.ceil(T / (0.5 * synth.cfl_dt(m, cp, p))))
        dt = T / nsteps
        xy = _nodes_xy(dg)
        th = lambda t: 2 * np.pi * (xy[..., 0] * k[0] + xy[..., 1] * k[1]) - om * t
        vex = lambda t: np.stack([d[0] * np.sin(th(t)), d[1] * np.sin(th(t))], 1)
        Sm = (lam * np.eye(2) + 2 * mu * np.outer(d, d)) / cp
        sex = lambda t: -np.stack([Sm[0, 0] * np.sin(th(t)), Sm[1, 1] * np.sin(th(t)), Sm[0, 1] * np.sin(th(t))], 1)
        v, s = vex(-dt / 2), sex(0.0)
        for _ in range(nsteps):
            v, s = dg.step(v, s, dt)
        e = v - vex(T - dt / 2)
        errs.append(np.sqrt(dg.inner_v(e, e)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= p - 0.1, (errs, rates)


def _mirror_mesh(nx=5, ny=4):
    """Unit square of nx x ny squares, each cut into 4 triangles through its centre (all CCW):
    symmetric under x -> 1 - x; with nx odd, the top and bottom triangles of the middle column
    are themselves symmetric about x = 1/2."""
    V = [(i / nx, j / ny) for j in range(ny + 1) for i in range(nx + 1)]
    cells = []
    for j in range(ny):
        for i in range(nx):
            a, b = j * (nx + 1) + i, j * (nx + 1) + i + 1
            c, d = b + nx + 1, a + nx + 1
            o = len(V)
            V.append(((i + 0.5) / nx, (j + 0.5) / ny))
            cells += [(a, b, o), (b, c, o), (c, d, o), (d, a, o)]
    V = np.array(V)
    c2v = np.array(cells, dtype=np.int32)
    return {"cell2vert": c2v, "cellxy": V[c2v], "coords": V, "nvert": len(V)}


def _mirror_pairs(m, p):
    """(cell, node) -> (cell', node') with the node at (1 - x, y)."""
    X = m["cellxy"]
    nodes = np.array([(i / p, j / p) for j in range(p + 1) for i in range(p + 1 - j)])
    xy = X[:, None, 0, :] + nodes[None, :, 0:1] * (X[:, None, 1, :] - X[:, None, 0, :]) \
        + nodes[None, :, 1:2] * (X[:, None, 2, :] - X[:, None, 0, :])
    key = {}
    for c in range(xy.shape[0]):
        cen = tuple(np.round(X[c].mean(0), 9))
        for n in range(xy.shape[1]):
            key[(cen, tuple(np.round(xy[c, n], 9)))] = (c, n)
    pairs = []
    for c in range(xy.shape[0]):
        cen = X[c].mean(0)
        mc = (round(1 - cen[0], 9), round(cen[1], 9))
        for n in range(xy.shape[1]):
            q = (round(1 - xy[c, n, 0], 9), round(xy[c, n, 1], 9))
            pairs.append((c, n) + key[(mc, q)])
    return np.array(pairs)


def mirror_defect(v, s, pairs):
    """Largest violation of the mirror symmetry (vx, sxy odd; vy, sxx, syy even), relative."""
    c, n, c2, n2 = pairs.T
    sign_v = np.array([-1.0, 1.0])[None, :]
    sign_s = np.array([1.0, 1.0, -1.0])[None, :]
    dv = v[c, :, n] - sign_v * v[c2, :, n2]
    ds = s[c, :, n] - sign_s * s[c2, :, n2]
    return max(np.abs(dv).max() / np.abs(v).max(), np.abs(ds).max() / np.abs(s).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_source_on_the_mirror_axis_gives_a_symmetric_field(p):
    # a reflection-symmetric mesh, homogeneous material and a point source on the axis inside a
    # cell that is itself symmetric: the discrete field must be mirror-symmetric (to round-off);
    # a wrong sign or orientation in any facet term, or a misplaced source, breaks it
    m = _mirror_mesh()
    dg = ElasticDG(m, p, *synth.homogeneous(m, 1.0, 2.0, 1.0))
    dt = synth.cfl_dt(m, 2.0, p)
    ricker = synth.ricker_series(5.0, dt, 30)
    v = np.zeros((dg.nc, 2, dg.Np))
    s = np.zeros((dg.nc, 3, dg.Np))
    v, s = dg.run(v, s, dt, 30, ricker, np.array([0.5, 0.70]))
    assert np.abs(v).max() > 0
    assert mirror_defect(v, s, _mirror_pairs(m, p)) < 1e-12
    # and the check itself is sharp: a source off the axis breaks the symmetry
    v2, s2 = dg.run(np.zeros_like(v), np.zeros_like(s), dt, 30, ricker, np.array([0.47, 0.70]))
    assert mirror_defect(v2, s2, _mirror_pairs(m, p)) > 1e-3


# ----------------------------------------------------------------------- point source
def _cell_integrals(X, p, q):
    """int_K phi_i q dx for the nodal basis phi_i of the triangle with vertices X [3, 2] and a
    function q(x, y) (vectorised), by a collapsed Gauss-Legendre rule (exact for the degree-2p
    integrands here): (r, s) = (u (1 - v), v) on the unit square, Jacobian (1 - v)."""
    t, w = np.polynomial.legendre.leggauss(p + 3)
    t, w = 0.5 * (t + 1), 0.5 * w
    u, v = np.meshgrid(t, t, indexing="ij")
    wt = (w[:, None] * w[None, :] * (1 - v)).ravel()
    r, s = (u * (1 - v)).ravel(), v.ravel()
    x = X[0] + np.outer(r, X[1] - X[0]) + np.outer(s, X[2] - X[0])
    J = np.array([X[1] - X[0], X[2] - X[0]]).T
    phi = refelem.eval_basis(p, r, s)
    return abs(np.linalg.det(J)) * (phi * (wt * q(x[:, 0], x[:, 1]))[:, None]).sum(0)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_point_source_reproduces_point_evaluation(p):
    # The projected point source c = M_K^-1 phi(xs) / |det J_K| is the discrete delta: for every
    # q in P_p on the source cell, sum_i c_i int_K phi_i q = q(xs).  A dropped 1/|det J|, phi(xs)
    # in place of M^-1 phi(xs), or wrong reference coordinates of xs each break it.
    m, dg = _dg(nx=5, ny=4, p=p, seed=3)
    rng = np.random.default_rng(20 + p)
    X = np.asarray(m["cellxy"], dtype=np.float64)
    for _ in range(4):
        c0 = int(rng.integers(dg.nc))
        lam = rng.dirichlet(np.ones(3))
        xs = lam @ X[c0]
        cell, coef = dg.source_vector(xs)
        assert cell == c0
        for a in range(p + 1):
            for b in range(p + 1 - a):
                q = lambda x, y, a=a, b=b: x ** a * y ** b
                lhs = coef @ _cell_integrals(X[cell], p, q)
                assert abs(lhs - xs[0] ** a * xs[1] ** b) < 1e-12, (p, a, b, lhs)
        # a random polynomial of full degree p
        cf = rng.standard_normal((p + 1, p + 1))
        q = lambda x, y: sum(cf[a, b] * x ** a * y ** b for a in range(p + 1) for b in range(p + 1 - a))
        assert abs(coef @ _cell_integrals(X[cell], p, q) - q(xs[0], xs[1])) < 1e-11


def test_point_source_location_takes_the_smallest_containing_cell():
    # xs on an edge shared by two cells, and on a vertex shared by several: the cell is the
    # smallest original id among the cells containing xs
    m, dg = _dg(nx=6, ny=5, p=1, seed=4)
    c2v = np.asarray(m["cell2vert"])
    coords = np.asarray(m["coords"], dtype=np.float64)
    rng = np.random.default_rng(7)
    F = dg.ifacets
    for k in rng.choice(len(F), 6, replace=False):
        c0, f0, c1 = int(F[k, 0]), int(F[k, 1]), int(F[k, 2])
        a, b = c2v[c0, f0], c2v[c0, (f0 + 1) % 3]
        assert {a, b} <= set(c2v[c1].tolist())
        xs = 0.5 * (coords[a] + coords[b])
        assert dg.locate(xs)[0] == min(c0, c1)
    interior = [v for v in range(coords.shape[0]) if (c2v == v).any(1).sum() == 6]
    for v in rng.choice(interior, 4, replace=False):
        owners = np.nonzero((c2v == v).any(1))[0]
        assert dg.locate(coords[v])[0] == owners.min()
