"""FP64 CPU oracle for the mass-lumped pressure system and for the projection
stage with a general equation of state solved by Newton's method (Section 3:
for a general EOS the energy equation carries the internal energy W_E(P, rho)
in place of the ideal gas's P/(gamma-1); with mass lumping the resulting
pressure system is mildly nonlinear and Newton-type methods solve it).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by
``tests/`` and ``bench.py``'s CPU legs, never by the product package, and
sharing no code with the CUDA library.  NumPy / SciPy in FP64; the stiffness
matrix comes from the C oracle (``PressureMatrix`` with part=2), element
volumes from ``projection.element_geometry``; a sparse direct solve is the
only linear-algebra machinery.

Lumped operator: A_L = diag(alpha_i m_i) + dt^2 K_beta on the free nodes,
m_i = int phi_i = sum over the elements e around i of w_e, w_e = |T_e|/(d+1)
(the alpha-weighted mass integral by vertex quadrature on every element).

General EOS (a reading: the paper names none): rho e(P, rho) = a P + b P^2/rho,
the caloric equation of a thermally perfect gas with c_v linear in the
temperature; b = 0 is the ideal gas with a = 1/(gamma-1).  Per Picard
iteration (H and rho K frozen) the unknown is dP on the free nodes and

    F_i(dP) = Q_i(dP_i) + dt^2 (K_H dP)_i - c_i = 0,
    Q_i(dP_i) = sum_e w_e rho e(P^n_i + dP_i, rho_e)   (vertex quadrature),
    c_i = int (W~_E - rho K) phi_i + dt int H W~~_u . grad phi_i,

the ideal-gas weak problem of Section 3.4 with the mass term lumped and the
internal energy left nonlinear.  Newton: dP <- dP - J^{-1} F(dP) with
J = diag(Q'(dP)) + dt^2 K_H, stopped when ||F|| <= tol ||c|| over the free
nodes (checked before every step and after the last) or after max_newton
steps.  Enthalpy per element H_e = (rho e(Pbar_e, rho_e) + Pbar_e) / rho_e.

Parity status: pinned by ``tests/test_oracle_lumped.py`` (row sums of the C
oracle's consistent mass for constant alpha, closed-form int phi_i on regular
meshes, a hand-derived two-triangle operator in ``tests/golden/``, O(h^2)
convergence of a manufactured solution, b = 0 reducing to one linear solve, a
manufactured root recovered, quadratic convergence, the enthalpy of the ideal
gas).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import PressureMatrix
from . import projection as PJ


def lumped_weights(dim, coords, conn, rho=None):
    """m_i = sum_e |T_e|/(d+1) and, if rho is given, s_i = sum_e |T_e|/((d+1) rho_e)."""
    conn = np.asarray(conn, dtype=np.int64)
    vol, _ = PJ.element_geometry(dim, coords, conn)
    n = np.asarray(coords).shape[0]
    w = vol / (dim + 1)
    m = np.zeros(n)
    np.add.at(m, conn, np.repeat(w[:, None], dim + 1, axis=1))
    if rho is None:
        return m
    s = np.zeros(n)
    np.add.at(s, conn, np.repeat((w / np.asarray(rho, dtype=np.float64))[:, None], dim + 1, axis=1))
    return m, s


class LumpedMatrix:
    """A_L = diag(alpha_i m_i) + dt2 K_beta, Dirichlet rows/columns removed."""

    def __init__(self, dim, coords, conn, dirichlet, alpha, beta, dt2):
        K = PressureMatrix(dim, coords, conn, dirichlet, alpha, beta, dt2, part=2)
        self.free_nodes = K.node_of_free
        self.n_nodes = K.n_nodes
        self.m = lumped_weights(dim, coords, conn)
        self.K = K.scipy()
        self.dt2 = float(dt2)
        d = (np.asarray(alpha, dtype=np.float64) * self.m)[self.free_nodes]
        self.A = (sp.diags(d) + self.dt2 * self.K).tocsr()

    def restrict(self, v):
        return np.asarray(v, dtype=np.float64)[self.free_nodes]

    def extend(self, v_red):
        out = np.zeros(self.n_nodes)
        out[self.free_nodes] = v_red
        return out

    def apply(self, x):
        return self.extend(self.A @ self.restrict(x))

    def solve(self, b):
        return self.extend(spla.spsolve(self.A.tocsc(), self.restrict(b)))

    def residual(self, b, x):
        br = self.restrict(b)
        r = br - self.A @ self.restrict(x)
        nb = np.linalg.norm(br)
        return float(np.linalg.norm(r) / (nb if nb > 0 else 1.0))


def energy(p, rho, a, b):
    """Internal energy density rho e(P, rho) = a P + b P^2 / rho."""
    return a * p + b * p * p / rho


def enthalpy(conn, p, rho, a, b):
    """H_e = (rho e(Pbar, rho_e) + Pbar) / rho_e, Pbar the vertex mean of P."""
    conn = np.asarray(conn, dtype=np.int64)
    rho = np.asarray(rho, dtype=np.float64)
    pbar = np.asarray(p, dtype=np.float64)[conn].mean(axis=1)
    return (energy(pbar, rho, a, b) + pbar) / rho


def mass_sum(dim, coords, conn, rho, p, a, b):
    """Q_i = sum_e w_e rho e(P_i, rho_e) and its derivative in P_i, by
    summing over the elements (no factorisation of the quadratic)."""
    conn = np.asarray(conn, dtype=np.int64)
    vol, _ = PJ.element_geometry(dim, coords, conn)
    w = vol / (dim + 1)
    rho = np.asarray(rho, dtype=np.float64)
    pv = np.asarray(p, dtype=np.float64)[conn]                 # [E, d+1]
    q_loc = w[:, None] * energy(pv, rho[:, None], a, b)
    dq_loc = w[:, None] * (a + 2.0 * b * pv / rho[:, None])
    n = np.asarray(coords).shape[0]
    q = np.zeros(n)
    dq = np.zeros(n)
    np.add.at(q, conn, q_loc)
    np.add.at(dq, conn, dq_loc)
    return q, dq


def newton(dim, coords, conn, dirichlet, rho, H, c, p_n, dp0, a, b, dt, max_newton, tol):
    """Newton's method for F(dP) = Q(dP) + dt^2 K_H dP - c = 0 on the free
    nodes (Dirichlet nodes: dP = 0).  Returns (dP, history of ||F||/||c||
    at every check, number of steps)."""
    K = PressureMatrix(dim, coords, conn, dirichlet, np.zeros(len(p_n)), H, 1.0, part=2)
    fr = K.node_of_free
    Kr = (dt * dt) * K.scipy()
    cr = np.asarray(c, dtype=np.float64)[fr]
    nc = np.linalg.norm(cr)
    nc = nc if nc > 0 else 1.0
    dp = np.zeros(len(p_n)) if dp0 is None else np.asarray(dp0, dtype=np.float64).copy()
    dp[np.asarray(dirichlet).astype(bool)] = 0.0
    hist = []
    steps = 0
    for j in range(max_newton + 1):
        q, dq = mass_sum(dim, coords, conn, rho, np.asarray(p_n) + dp, a, b)
        F = q[fr] + Kr @ dp[fr] - cr
        res = np.linalg.norm(F) / nc
        hist.append(res)
        if (tol > 0 and res <= tol) or j == max_newton:
            break
        J = (sp.diags(dq[fr]) + Kr).tocsc()
        dp[fr] = dp[fr] - spla.spsolve(J, F)
        steps += 1
    return dp, hist, steps


def projection_step_eos(dim, coords, conn, dirichlet, rho, wu_tt, we, p_n, a, b, dt, n_picard, max_newton,
                        tol=1e-8, dp0=None):
    """Projection stage with the general EOS: first guesses (H from P^n,
    rho K from W~~_u), then n_picard iterations of [right-hand side c without
    the mass term, Newton solve for dP (warm start: dp0, then the previous
    iterate), post-projection with the EOS enthalpy].  Returns a dict with
    dP, P, W_u, H, rho K and the per-iteration Newton histories."""
    conn = np.asarray(conn, dtype=np.int64)
    n = np.asarray(coords).shape[0]
    H = enthalpy(conn, p_n, rho, a, b)
    rhok = PJ.kinetic(wu_tt, rho, dim)
    dp = np.zeros(n) if dp0 is None else np.asarray(dp0, dtype=np.float64).copy()
    hists, steps = [], []
    p = np.asarray(p_n, dtype=np.float64).copy()
    wu = np.asarray(wu_tt, dtype=np.float64).reshape(-1, dim).copy()
    for _ in range(n_picard):
        c = PJ.rhs(dim, coords, conn, dirichlet, np.zeros(n), H, rhok, wu_tt, we, p_n, dt)
        dp, hist, st = newton(dim, coords, conn, dirichlet, rho, H, c, p_n, dp, a, b, dt, max_newton, tol)
        hists.append(hist)
        steps.append(st)
        p, wu, _, rhok = PJ.post(dim, coords, conn, p_n, dp, wu_tt, rho, 1.4, dt)
        H = enthalpy(conn, p, rho, a, b)
    return {"dp": dp, "p": p, "wu": wu, "H": H, "rhok": rhok, "hist": hists, "steps": steps}
