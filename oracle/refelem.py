"""ORACLE (test infrastructure only; never imported by the product path).

Exact reference-element matrices for the nodal P_p basis on the reference triangle
T = {(r, s): r >= 0, s >= 0, r + s <= 1}, computed in rational arithmetic.

The paper discretises velocity and stress with discontinuous Galerkin in space (Section 7.1)
and inverts block-diagonal mass matrices cell by cell (Section 7.2); it leaves the element
and basis to the Seigen paper.  The basis here is the nodal Lagrange basis on the equispaced
points (i/p, j/p), j = 0..p outer, i = 0..p-j inner (p = 0: the centroid).  The field layout
on both sides of the library boundary is the vector of nodal values in that order.

Every integral is exact: a Lagrange function is a combination of monomials r^a s^b, whose
integral over T is a! b! / (a + b + 2)!, and whose restriction to an edge is a polynomial in
the edge parameter t in [0, 1], integrated term by term.  Nothing here uses quadrature.

Faces: face f joins local vertices f and (f+1) mod 3 of the triangle (v0=(0,0), v1=(1,0),
v2=(0,1)); its parameter t runs from vertex f (t=0) to vertex f+1 (t=1).
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial, comb

import numpy as np


def nodes(p):
    if p == 0:
        return [(Fraction(1, 3), Fraction(1, 3))]
    return [(Fraction(i, p), Fraction(j, p)) for j in range(p + 1) for i in range(p + 1 - j)]


def monomials(p):
    return [(a, d - a) for d in range(p + 1) for a in range(d, -1, -1)]


def _inverse(A):
    """Gauss-Jordan inverse of a square matrix of Fractions."""
    n = len(A)
    M = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [x * inv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [row[n:] for row in M]


def _matmul(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(len(B))) for j in range(len(B[0]))]
            for i in range(len(A))]


def _transpose(A):
    return [list(r) for r in zip(*A)]


def _tri_int(a, b):
    """Integral of r^a s^b over the reference triangle."""
    return Fraction(factorial(a) * factorial(b), factorial(a + b + 2))


_FACE_LINE = {0: ((0, 0), (1, 0)), 1: ((1, 0), (-1, 1)), 2: ((0, 1), (0, -1))}
# face f: (r, s) = origin + t * direction


def _edge_poly(a, b, f, flip=False):
    """Coefficients (in t, ascending) of r^a s^b restricted to face f, t in [0,1].
    flip=True substitutes t -> 1 - t."""
    (r0, s0), (dr, ds) = _FACE_LINE[f]
    if flip:
        r0, s0, dr, ds = r0 + dr, s0 + ds, -dr, -ds

    def lin_pow(c0, c1, e):
        # (c0 + c1 t)^e
        return [Fraction(comb(e, k)) * Fraction(c0) ** (e - k) * Fraction(c1) ** k for k in range(e + 1)]

    pa, pb = lin_pow(r0, dr, a), lin_pow(s0, ds, b)
    out = [Fraction(0)] * (a + b + 1)
    for i, x in enumerate(pa):
        for j, y in enumerate(pb):
            out[i + j] += x * y
    return out


def _poly_int01(c1, c2):
    return sum(x * y / (i + j + 1) for i, x in enumerate(c1) for j, y in enumerate(c2))


@lru_cache(maxsize=None)
def exact(p):
    """Rational matrices for degree p.  Returns a dict of lists-of-lists of Fractions:

    C        monomial coefficients of the Lagrange functions (phi_j = sum_m C[m][j] mono_m)
    M        M[i][j]  = int_T phi_i phi_j
    Minv     inverse of M
    Sr, Ss   Sr[i][j] = int_T phi_i d(phi_j)/dr   (Ss likewise with d/ds)
    Fsame[f]          int_0^1 phi_i(face f, t) phi_j(face f, t) dt
    Fcross[(fa,fb,flip)]  int_0^1 phi_i(face fa, t) phi_j(face fb, t') dt, t' = 1-t if flip else t
    """
    X = nodes(p)
    mono = monomials(p)
    n = len(mono)
    V = [[r ** a * s ** b for (a, b) in mono] for (r, s) in X]
    C = _inverse(V)  # V C = I  =>  phi_j(node_i) = delta_ij
    G = [[_tri_int(am + an, bm + bn) for (an, bn) in mono] for (am, bm) in mono]
    Gr = [[(an * _tri_int(am + an - 1, bm + bn) if an > 0 else Fraction(0)) for (an, bn) in mono]
          for (am, bm) in mono]
    Gs = [[(bn * _tri_int(am + an, bm + bn - 1) if bn > 0 else Fraction(0)) for (an, bn) in mono]
          for (am, bm) in mono]
    Ct = _transpose(C)
    M = _matmul(_matmul(Ct, G), C)
    Sr = _matmul(_matmul(Ct, Gr), C)
    Ss = _matmul(_matmul(Ct, Gs), C)
    Minv = _inverse(M)
    Fsame, Fcross = {}, {}
    for fa in range(3):
        for fb in range(3):
            for flip in (False, True):
                H = [[_poly_int01(_edge_poly(am, bm, fa), _edge_poly(an, bn, fb, flip))
                      for (an, bn) in mono] for (am, bm) in mono]
                Fcross[(fa, fb, flip)] = _matmul(_matmul(Ct, H), C)
        Fsame[fa] = Fcross[(fa, fa, False)]
    return dict(C=C, M=M, Minv=Minv, Sr=Sr, Ss=Ss, Fsame=Fsame, Fcross=Fcross, n=n)


def _f64(A):
    return np.array([[float(x) for x in row] for row in A], dtype=np.float64)


@lru_cache(maxsize=None)
def matrices(p):
    """Float64 versions of the exact matrices (each entry correctly rounded)."""
    E = exact(p)
    return dict(
        p=p, Np=E["n"], nodes=np.array([[float(r), float(s)] for r, s in nodes(p)]),
        C=_f64(E["C"]), mono=monomials(p), M=_f64(E["M"]), Minv=_f64(E["Minv"]),
        Sr=_f64(E["Sr"]), Ss=_f64(E["Ss"]),
        Fsame={f: _f64(v) for f, v in E["Fsame"].items()},
        Fcross={k: _f64(v) for k, v in E["Fcross"].items()},
    )


def eval_basis(p, r, s):
    """Values of the nodal basis functions at reference points (r, s) (arrays): [npts, Np]."""
    m = matrices(p)
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    P = np.stack([r ** a * s ** b for (a, b) in m["mono"]], axis=1)
    return P @ m["C"]
