"""ORACLE (test infrastructure only).  Seismogram misfit and its exact discrete gradient with
respect to per-cell rho, lambda, mu for the DG elastic chain of oracle/dg.py.

Misfit: J = 1/2 dt sum_n sum_r |P_r v^{n+1/2} - d_r^n|^2, P_r the point evaluation of the DG
velocity at receiver r, the run starting from rest (v^{-1/2} = 0, sigma^0 = 0).

Discrete adjoint (derived from the time step, Section 7.1 scheme): with
  A~ = A + c ABA, B~ = B + c BAB, c = dt^2/24,  v' = v + dt A~ s,  s' = s + dt B~ v' + dt g src,
and the skew identity M_rho A = -B^T M_S (pinned in test_oracle_dg.py), the adjoint variables in
mass-weighted form (vt = M_rho^{-1} adj(v), st = M_S^{-1} adj(sigma)) obey the same leapfrog run
backwards with -dt:
  st_next = st,  vt += -dt A~ st,  vt += dt M_rho^{-1} P^T r^n,  st += -dt B~ vt.
A = R^{-1} A0 (R = rho per cell) and B = C B0 (C Hooke's law per cell), so every parameter
derivative is a cell-local bilinear form, M-weighted (|det J| M_hat on the cell):
  from the stress update (adjoint st of sigma^{n+1}, forward v = v^{n+1/2}):
    g_lam += dt <C^-1 st, C_lam E(v)> + c dt <C^-1 st, C_lam E(ABv)> + c dt <E(A st), C_lam E(v)>
    g_rho += c dt <A st, ABv>
  from the velocity update (adjoint vt of v^{n+1/2}, forward sigma = sigma^n):
    g_rho += -dt (<vt, A~ sigma> + c <AB vt, A sigma>)
    g_lam += -c dt <E(vt), C_lam E(A sigma)>
with the same for mu (C_mu); E(x) = M^{-1} d(x, .) is the strain (xx, yy, 2xy), C_lam = dC/dlambda,
C_mu = dC/dmu.  Every forward state is stored: for small cases only.
"""
import numpy as np

from . import refelem

C_LAM = np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 0.0], [0.0, 0.0, 0.0]])
C_MU = np.array([[2.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 1.0]])


def receivers(dg, rec_xy):
    """(cell, basis values) of every receiver: smallest cell id containing the point."""
    out = []
    for xy in np.asarray(rec_xy, dtype=np.float64):
        c, r, s = dg.locate(xy)
        out.append((c, refelem.eval_basis(dg.p, r, s)[0]))
    return out


def evaluate(rec, v):
    """P v: velocity (2 components) at every receiver, [nrec, 2]."""
    return np.array([[phi @ v[c, k] for k in range(2)] for (c, phi) in rec])


def record(dg, dt, nsteps, ricker, xs, rec):
    """Forward run from rest; traces[n] = P v^{n+1/2}.  Also returns every state."""
    src = dg.source_vector(xs)
    v = np.zeros((dg.nc, 2, dg.Np))
    s = np.zeros((dg.nc, 3, dg.Np))
    traces, sig_before, v_after = [], [], []
    for n in range(nsteps):
        sig_before.append(s)
        v, s = dg.step(v, s, dt, float(ricker[n]), src)
        v_after.append(v)
        traces.append(evaluate(rec, v))
    return np.array(traces), sig_before, v_after


def misfit(traces, data, dt):
    return 0.5 * dt * float(np.sum((traces - data) ** 2))


def _strain(dg, x):
    return dg.solve_mass(dg.assemble_d(x))


def _mdot(dg, a, b):
    """Per-cell M-weighted inner product |det J| sum_comp a^T M_hat b, [nc]."""
    return dg.det * np.einsum("cki,ij,ckj->c", a, dg.R["M"], b)


def _mdot_c(dg, e1, Cm, e2):
    """Per-cell |det J| sum_ij M_ij e1_i^T Cm e2_j for strain-like fields, [nc]."""
    return dg.det * np.einsum("cki,ij,kl,clj->c", e1, dg.R["M"], Cm, e2)


def gradient(dg, dt, nsteps, ricker, xs, rec_xy, data):
    """(J, g_rho, g_lam, g_mu) of the misfit against `data` [nsteps, nrec, 2]."""
    rec = receivers(dg, rec_xy)
    traces, sig_before, v_after = record(dg, dt, nsteps, ricker, xs, rec)
    J = misfit(traces, data, dt)
    A, B = dg.apply_A, dg.apply_B
    E = lambda x: _strain(dg, x)
    c = dt * dt / 24.0
    Ci = dg.compliance()
    g = np.zeros((3, dg.nc))
    vt = np.zeros((dg.nc, 2, dg.Np))
    st = np.zeros((dg.nc, 3, dg.Np))
    Minv = dg.R["Minv"]
    for n in range(nsteps - 1, -1, -1):
        v = v_after[n]
        sig = sig_before[n]
        # stress update: adjoint st of sigma^{n+1}, forward v^{n+1/2}
        Ev = E(v)
        ABv = A(B(v))
        E_ABv = E(ABv)
        sh = np.einsum("ckl,clj->ckj", Ci, st)
        Ast = A(st)
        E_Ast = E(Ast)
        for k, Cm in ((1, C_LAM), (2, C_MU)):
            g[k] += dt * (_mdot_c(dg, sh, Cm, Ev) + c * _mdot_c(dg, sh, Cm, E_ABv) + c * _mdot_c(dg, E_Ast, Cm, Ev))
        g[0] += c * dt * _mdot(dg, Ast, ABv)
        vt = vt - dt * (Ast + c * A(B(Ast)))
        # receivers: vt += dt M_rho^{-1} P^T r^n
        r = traces[n] - data[n]
        for (cell, phi), rr in zip(rec, r):
            q = (Minv @ phi) / (dg.rho[cell] * dg.det[cell])
            vt[cell, 0] += dt * rr[0] * q
            vt[cell, 1] += dt * rr[1] * q
        # velocity update: adjoint vt of v^{n+1/2}, forward sigma^n
        Asig = A(sig)
        ABAsig = A(B(Asig))
        E_Asig = E(Asig)
        ABvt = A(B(vt))
        Evt = E(vt)
        g[0] += -dt * (_mdot(dg, vt, Asig + c * ABAsig) + c * _mdot(dg, ABvt, Asig))
        for k, Cm in ((1, C_LAM), (2, C_MU)):
            g[k] += -c * dt * _mdot_c(dg, Evt, Cm, E_Asig)
        Bvt = B(vt)
        st = st - dt * (Bvt + c * B(A(Bvt)))
    return J, g[0], g[1], g[2]
