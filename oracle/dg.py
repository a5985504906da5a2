"""ORACLE (test infrastructure only; only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import it).  Plain, slow, FP64 CPU implementation of the untiled discontinuous-
Galerkin elastic-wave time step that the sparse-tiled loop chain computes.

What it follows.  The paper fixes the method only in prose (Section 7.1: velocity-stress
formulation, DG in space, fourth-order explicit leapfrog built from a truncated Taylor series,
non-dissipative; Section 7.2: eight cell-local solves with block-diagonal mass matrices and
twenty-five loops over cells, interior facets and exterior facets per time step).  The
reading implemented here is:

  rho dv/dt = div(sigma),   dsigma/dt = lambda tr(eps(v)) I + 2 mu eps(v) + g(t) delta(x - xs) I

  b(sigma, w) = sum_K int_K div(sigma).w - sum_f int_f [[sigma n]].{w} - sum_e int_e (sigma n).w
              (strong form; free surface sigma n = 0 on every exterior facet)
  d(v, tau)   = sum_K int_K tau : grad v - sum_f int_f {tau} n . [[v]]      ( = -b(tau, v) )

  A sigma = M_rho^{-1} b(sigma, .),   B v = C (M^{-1} d(v, .))       (C = Hooke's law)

  v^{n+1/2} = v^{n-1/2} + dt (A sigma^n + dt^2/24 A B A sigma^n)
  sigma^{n+1} = sigma^n + dt (B v^{n+1/2} + dt^2/24 B A B v^{n+1/2}) + dt g(t_{n+1/2}) M^{-1} phi(xs) (1,1,0)

Interior facet f = (c0, c1) with c0 < c1; n is the unit normal pointing out of c0;
{a} = (a|c0 + a|c1)/2, [[a]] = a|c0 - a|c1.  Stress is stored as (xx, yy, xy); the xy test
function is phi (e_xy + e_yx), so tau : grad v counts the xy entry twice.

Every integral is exact (rational reference matrices from refelem.py).  Cell loops run over
all cells at once (numpy rows in ascending cell order).  A facet loop visits its facets class by
class, a class being the facets with the same (local face of c0, local face of c1, flip) and
hence the same reference face matrices; within a class the facets are in ascending order, and
each facet increments both of its cells (np.add.at).  Facet increments therefore reach a cell in
class order rather than in plain facet order, which changes only the rounding of the sums; the
loop-by-loop semantics are those of the chain (the paper lets iterations of a loop run in any
order, Section 2).  No blocking, fusion or reordering of loops: this is the untiled
loop-by-loop chain, with the assembly of b and the solve with the block-diagonal mass matrix
kept as separate steps.

Facets are numbered by (min vertex id, max vertex id) of the original vertex numbering.
"""
import numpy as np

from . import refelem


def _facets(cell2vert):
    """Interior and exterior facets, sorted by (min vertex, max vertex).

    Returns (interior, exterior): interior rows (c0, f0, c1, f1, flip), exterior rows (c, f).
    flip = 1 when c1 traverses the shared edge in the opposite direction to c0.
    """
    nc = cell2vert.shape[0]
    rows = []
    for f in range(3):
        a = cell2vert[:, f].astype(np.int64)
        b = cell2vert[:, (f + 1) % 3].astype(np.int64)
        rows.append(np.stack([np.minimum(a, b), np.maximum(a, b), np.arange(nc), np.full(nc, f), a], axis=1))
    R = np.concatenate(rows)
    R = R[np.lexsort((R[:, 2], R[:, 1], R[:, 0]))]  # by key, then cell id
    key_same_next = np.zeros(len(R), dtype=bool)
    key_same_next[:-1] = (R[:-1, 0] == R[1:, 0]) & (R[:-1, 1] == R[1:, 1])
    first = np.ones(len(R), dtype=bool)
    first[1:] = ~key_same_next[:-1]
    interior_start = first & key_same_next
    exterior = first & ~key_same_next
    i0 = np.nonzero(interior_start)[0]
    if np.any(key_same_next[i0 + 1]):
        raise ValueError("an edge is shared by more than two cells")
    A, B = R[i0], R[i0 + 1]        # A has the smaller cell id (sorted by cell within a key)
    flip = (A[:, 4] != B[:, 4]).astype(np.int64)
    interior = np.stack([A[:, 2], A[:, 3], B[:, 2], B[:, 3], flip], axis=1)
    E = R[exterior]
    return interior, np.stack([E[:, 2], E[:, 3]], axis=1)


class ElasticDG:
    """The semi-discrete operators A (stress -> velocity rate) and B (velocity -> stress rate)
    on one mesh, plus the fourth-order staggered Taylor leapfrog step."""

    def __init__(self, mesh, p, rho, lam, mu):
        self.p = p
        self.R = refelem.matrices(p)
        self.Np = self.R["Np"]
        self.cell2vert = np.asarray(mesh["cell2vert"])
        X = np.asarray(mesh["cellxy"], dtype=np.float64)
        self.nc = X.shape[0]
        self.rho, self.lam, self.mu = (np.asarray(a, dtype=np.float64) for a in (rho, lam, mu))
        # affine map x = X0 + (X1 - X0) r + (X2 - X0) s
        j11, j21 = X[:, 1, 0] - X[:, 0, 0], X[:, 1, 1] - X[:, 0, 1]
        j12, j22 = X[:, 2, 0] - X[:, 0, 0], X[:, 2, 1] - X[:, 0, 1]
        det = j11 * j22 - j12 * j21
        self.X0 = X[:, 0]
        self.jac = np.stack([np.stack([j11, j12], 1), np.stack([j21, j22], 1)], 1)
        self.det = np.abs(det)
        self.rx, self.ry = j22 / det, -j12 / det
        self.sx, self.sy = -j21 / det, j11 / det
        # face geometry: length and outward unit normal of local face f of every cell
        self.flen = np.zeros((self.nc, 3))
        self.fn = np.zeros((self.nc, 3, 2))
        for f in range(3):
            t = X[:, (f + 1) % 3] - X[:, f]
            L = np.hypot(t[:, 0], t[:, 1])
            n = np.stack([t[:, 1], -t[:, 0]], 1) / L[:, None]
            opp = X[:, (f + 2) % 3] - X[:, f]
            sgn = np.where((n * opp).sum(1) > 0, -1.0, 1.0)
            self.flen[:, f] = L
            self.fn[:, f] = n * sgn[:, None]
        self.ifacets, self.efacets = _facets(self.cell2vert)

    # ---------------------------------------------------------------- helpers
    def _mv(self, A, u):
        """Apply a reference matrix to the nodal vectors of every cell: [nc, Np] -> [nc, Np]."""
        return u @ A.T

    def _facet_groups(self):
        F = self.ifacets
        key = F[:, 1] * 6 + F[:, 3] * 2 + F[:, 4]
        for k in np.unique(key):
            idx = np.nonzero(key == k)[0]
            yield idx, int(F[idx[0], 1]), int(F[idx[0], 3]), bool(F[idx[0], 4])

    # ---------------------------------------------------------------- operator A
    def assemble_b(self, sig, form="strong"):
        """Right-hand side b(sigma, phi_i e_k) for every cell, node, velocity component."""
        R, nc = self.R, self.nc
        sxx, syy, sxy = sig[:, 0], sig[:, 1], sig[:, 2]
        rhs = np.zeros((nc, 2, self.Np))
        d = self.det[:, None]
        # cell loop: volume integrals
        if form == "strong":   # int_K div(sigma) . w
            Sr, Ss = R["Sr"], R["Ss"]
        else:                  # -int_K sigma : grad w
            Sr, Ss = -R["Sr"].T, -R["Ss"].T
        # (for the weak form Sr, Ss hold -Sr^T, -Ss^T: -int sxx dphi_i/dx + sxy dphi_i/dy)
        rx, ry, sx, sy = (a[:, None] for a in (self.rx, self.ry, self.sx, self.sy))
        rhs[:, 0] = d * (rx * self._mv(Sr, sxx) + sx * self._mv(Ss, sxx) + ry * self._mv(Sr, sxy) + sy * self._mv(Ss, sxy))
        rhs[:, 1] = d * (rx * self._mv(Sr, sxy) + sx * self._mv(Ss, sxy) + ry * self._mv(Sr, syy) + sy * self._mv(Ss, syy))
        # interior facet loop
        for idx, f0, f1, flip in self._facet_groups():
            c0, c1 = self.ifacets[idx, 0], self.ifacets[idx, 2]
            n = self.fn[c0, f0]
            L = self.flen[c0, f0][:, None]
            sn0 = np.stack([sxx[c0] * n[:, :1] + sxy[c0] * n[:, 1:], sxy[c0] * n[:, :1] + syy[c0] * n[:, 1:]], 1)
            sn1 = np.stack([sxx[c1] * n[:, :1] + sxy[c1] * n[:, 1:], sxy[c1] * n[:, :1] + syy[c1] * n[:, 1:]], 1)
            F00, F11 = R["Fsame"][f0], R["Fsame"][f1]
            F01, F10 = R["Fcross"][(f0, f1, flip)], R["Fcross"][(f1, f0, flip)]
            for k in range(2):
                if form == "strong":   # -int [[sigma n]] . {w}
                    to0 = -0.5 * L * (self._mv(F00, sn0[:, k]) - self._mv(F01, sn1[:, k]))
                    to1 = -0.5 * L * (self._mv(F10, sn0[:, k]) - self._mv(F11, sn1[:, k]))
                else:                  # +int {sigma} n . [[w]]
                    to0 = 0.5 * L * (self._mv(F00, sn0[:, k]) + self._mv(F01, sn1[:, k]))
                    to1 = -0.5 * L * (self._mv(F10, sn0[:, k]) + self._mv(F11, sn1[:, k]))
                np.add.at(rhs[:, k], c0, to0)
                np.add.at(rhs[:, k], c1, to1)
        # exterior facet loop (free surface; only the strong form has a term)
        if form == "strong":
            for f in range(3):
                sel = self.efacets[self.efacets[:, 1] == f, 0]
                n = self.fn[sel, f]
                L = self.flen[sel, f][:, None]
                sn = [sxx[sel] * n[:, :1] + sxy[sel] * n[:, 1:], sxy[sel] * n[:, :1] + syy[sel] * n[:, 1:]]
                for k in range(2):
                    np.add.at(rhs[:, k], sel, -L * self._mv(R["Fsame"][f], sn[k]))
        return rhs

    def solve_rho(self, rhs):
        """Cell-local solve with the block-diagonal mass matrix rho_K |det J_K| M_hat."""
        s = 1.0 / (self.rho * self.det)
        return s[:, None, None] * np.einsum("ij,ckj->cki", self.R["Minv"], rhs)

    def apply_A(self, sig, form="strong"):
        return self.solve_rho(self.assemble_b(sig, form))

    # ---------------------------------------------------------------- operator B
    def assemble_d(self, v, form="weak_tau"):
        """Right-hand side d(v, tau_i) for every cell, node, stored stress component."""
        R, nc = self.R, self.nc
        vx, vy = v[:, 0], v[:, 1]
        rhs = np.zeros((nc, 3, self.Np))
        d = self.det[:, None]
        rx, ry, sx, sy = (a[:, None] for a in (self.rx, self.ry, self.sx, self.sy))
        if form == "weak_tau":   # sum_K int tau : grad v
            Sr, Ss, sg = R["Sr"], R["Ss"], 1.0
        else:                    # -sum_K int div(tau) . v
            Sr, Ss, sg = R["Sr"].T, R["Ss"].T, -1.0
        dx_vx = rx * self._mv(Sr, vx) + sx * self._mv(Ss, vx)
        dy_vx = ry * self._mv(Sr, vx) + sy * self._mv(Ss, vx)
        dx_vy = rx * self._mv(Sr, vy) + sx * self._mv(Ss, vy)
        dy_vy = ry * self._mv(Sr, vy) + sy * self._mv(Ss, vy)
        rhs[:, 0] = sg * d * dx_vx
        rhs[:, 1] = sg * d * dy_vy
        rhs[:, 2] = sg * d * (dy_vx + dx_vy)
        for idx, f0, f1, flip in self._facet_groups():
            c0, c1 = self.ifacets[idx, 0], self.ifacets[idx, 2]
            n = self.fn[c0, f0]
            nx, ny = n[:, :1], n[:, 1:]
            L = self.flen[c0, f0][:, None]
            F = {(0, 0): R["Fsame"][f0], (0, 1): R["Fcross"][(f0, f1, flip)],
                 (1, 0): R["Fcross"][(f1, f0, flip)], (1, 1): R["Fsame"][f1]}
            for a, ca in ((0, c0), (1, c1)):
                if form == "weak_tau":   # -int {tau} n . [[v]]: jump of v tested on side a
                    jx = self._mv(F[(a, 0)], vx[c0]) - self._mv(F[(a, 1)], vx[c1])
                    jy = self._mv(F[(a, 0)], vy[c0]) - self._mv(F[(a, 1)], vy[c1])
                    w = -0.5 * L
                else:                    # +int [[tau n]] . {v}: average of v tested on side a
                    jx = self._mv(F[(a, 0)], vx[c0]) + self._mv(F[(a, 1)], vx[c1])
                    jy = self._mv(F[(a, 0)], vy[c0]) + self._mv(F[(a, 1)], vy[c1])
                    w = 0.5 * L * (1.0 if a == 0 else -1.0)
                np.add.at(rhs[:, 0], ca, w * nx * jx)
                np.add.at(rhs[:, 1], ca, w * ny * jy)
                np.add.at(rhs[:, 2], ca, w * (ny * jx + nx * jy))
        if form != "weak_tau":           # +int_e (tau n) . v
            for f in range(3):
                sel = self.efacets[self.efacets[:, 1] == f, 0]
                n = self.fn[sel, f]
                nx, ny = n[:, :1], n[:, 1:]
                L = self.flen[sel, f][:, None]
                mx, my = self._mv(R["Fsame"][f], vx[sel]), self._mv(R["Fsame"][f], vy[sel])
                np.add.at(rhs[:, 0], sel, L * nx * mx)
                np.add.at(rhs[:, 1], sel, L * ny * my)
                np.add.at(rhs[:, 2], sel, L * (ny * mx + nx * my))
        return rhs

    def solve_mass(self, rhs):
        """Cell-local solve with |det J_K| M_hat (the unweighted block-diagonal mass)."""
        return (1.0 / self.det)[:, None, None] * np.einsum("ij,ckj->cki", self.R["Minv"], rhs)

    def hooke(self, E):
        """Stored strain (exx, eyy, gamma = 2 exy) -> stored stress (sxx, syy, sxy)."""
        lam, mu = self.lam[:, None], self.mu[:, None]
        tr = E[:, 0] + E[:, 1]
        return np.stack([lam * tr + 2 * mu * E[:, 0], lam * tr + 2 * mu * E[:, 1], mu * E[:, 2]], 1)

    def apply_B(self, v, form="weak_tau"):
        return self.hooke(self.solve_mass(self.assemble_d(v, form)))

    # ---------------------------------------------------------------- source, energy
    def locate(self, xs):
        """Smallest cell id whose barycentric coordinates of xs are all >= -1e-12."""
        rel = xs[None, :] - self.X0
        r = self.rx * rel[:, 0] + self.ry * rel[:, 1]
        s = self.sx * rel[:, 0] + self.sy * rel[:, 1]
        ok = (r >= -1e-12) & (s >= -1e-12) & (1.0 - r - s >= -1e-12)
        c = int(np.nonzero(ok)[0][0])
        return c, float(r[c]), float(s[c])

    def source_vector(self, xs):
        """(cell, coefficients M_K^{-1} phi(xs)) of the projected point source."""
        c, r, s = self.locate(np.asarray(xs, dtype=np.float64))
        phi = refelem.eval_basis(self.p, r, s)[0]
        return c, (self.R["Minv"] @ phi) / self.det[c]

    def compliance(self):
        """Per-cell inverse of Hooke's law in the stored components, [nc, 3, 3]."""
        Cm = np.zeros((self.nc, 3, 3))
        Cm[:, 0, 0] = Cm[:, 1, 1] = self.lam + 2 * self.mu
        Cm[:, 0, 1] = Cm[:, 1, 0] = self.lam
        Cm[:, 2, 2] = self.mu
        return np.linalg.inv(Cm)

    def inner_v(self, a, b):
        """<a, M_rho b> for velocity fields."""
        return float(np.einsum("c,cki,ij,ckj->", self.rho * self.det, a, self.R["M"], b))

    def inner_s(self, a, b):
        """<a, M_S b> with M_S = |det J| M_hat (x) C^{-1} (compliance-weighted mass)."""
        Ci = self.compliance()
        return float(np.einsum("c,cki,ij,ckl,clj->", self.det, a, self.R["M"], Ci, b))

    # ---------------------------------------------------------------- time stepping
    def step(self, v, sig, dt, g=0.0, src=None):
        """One time step (velocity sub-chain, then stress sub-chain). Returns (v, sigma)."""
        return taylor_leapfrog_step(self.apply_A, self.apply_B, v, sig, dt, g, src)

    def run(self, v, sig, dt, nsteps, ricker=None, xs=None):
        src = None
        if xs is not None:
            c, coef = self.source_vector(xs)
            src = (c, coef)
        for n in range(nsteps):
            g = 0.0 if ricker is None else float(ricker[n])
            v, sig = self.step(v, sig, dt, g, src)
        return v, sig


def taylor_leapfrog_step(A, B, v, sig, dt, g=0.0, src=None):
    """Fourth-order staggered leapfrog from a truncated Taylor series (Section 7.1):
    v += dt (A s + dt^2/24 A B A s);  s += dt (B v + dt^2/24 B A B v) + dt g P(delta) (1,1,0).
    A and B are callables; with 1x1 arrays this is the scalar recurrence used as a pin."""
    c = dt * dt / 24.0
    u1 = A(sig)
    u2 = A(B(u1))
    v = v + dt * (u1 + c * u2)
    s1 = B(v)
    s2 = B(A(s1))
    sig = sig + dt * (s1 + c * s2)
    if src is not None and g != 0.0:
        cell, coef = src
        sig = sig.copy()
        sig[cell, 0] += dt * g * coef
        sig[cell, 1] += dt * g * coef
    return v, sig
