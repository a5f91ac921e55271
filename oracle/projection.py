"""FP64 CPU oracle for the projection stage around the pressure solve
(Sections 3.3-3.5): the right-hand side of the weak problem, the
post-projection updates, and the Picard loop that alternates them with the
solve.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by
``tests/`` and ``bench.py``'s CPU legs, never by the product package, and
sharing no code with the CUDA library.  Plain NumPy, FP64, written from the
definitions: element integrals of P1 hat functions (lambda_k barycentric),
no blocking or reordering beyond what the definitions state.

Inputs are per primal element (the values the pre-projection stage of
Section 3.3 produces: density rho, intermediate momentum W~~_u, intermediate
total energy W~_E) and per node (pressure P^n, mass coefficient alpha, the
paper's 1/(gamma - 1)); element order and node numbering are the caller's.

Readings of the paper taken here: the boundary term
-dt int_Gamma H W_u^{n+1}.eta z of the weak problem vanishes (closed walls,
W_u.eta = 0 on the Neumann boundary; on Dirichlet faces z = 0); element
values of the enthalpy use the vertex mean of the nodal pressure,
H_e = gamma/(gamma-1) mean_k(P_k) / rho_e; the first Picard guesses are
H^{n+1,1} from P^n and (rho K)^{n+1,1} = |W~~_u|^2 / (2 rho).

Parity status: pinned by ``tests/test_oracle_projection.py`` (partition of
unity, closed-form nodal integrals on regular meshes, the discrete divergence
theorem for P0 projections of linear fields, exact gradients of linear
fields, a single Picard iteration against a direct solve, and the element
values of the kinetic energy density and the enthalpy against hand-derived
values in ``tests/golden/projection_element_values.txt``).
"""
from __future__ import annotations

import math

import numpy as np

from . import PressureMatrix


def element_geometry(dim, coords, conn):
    """|T_e| and the gradients of the barycentric coordinates, grad[e, k, :]
    = grad lambda_k on element e (constant per element).  With J the matrix
    whose columns are x_k - x_0 (k = 1..d), lambda_k = (J^{-1}(x - x_0))_k,
    so grad lambda_k is row k-1 of J^{-1}; grad lambda_0 = -sum of the rest."""
    coords = np.asarray(coords, dtype=np.float64)
    conn = np.asarray(conn, dtype=np.int64)
    x = coords[conn]                                  # [E, d+1, d]
    J = np.transpose(x[:, 1:, :] - x[:, :1, :], (0, 2, 1))   # [E, d, d], columns x_k - x_0
    det = np.linalg.det(J)
    vol = np.abs(det) / math.factorial(dim)
    Jinv = np.linalg.inv(J)                           # [E, d, d]
    grad = np.empty((conn.shape[0], dim + 1, dim))
    grad[:, 1:, :] = Jinv
    grad[:, 0, :] = -Jinv.sum(axis=1)
    return vol, grad


def _triple_integral_weights(dim):
    """w[i, j, k] = int_T lambda_i lambda_j lambda_k / |T|
    = d! a! b! c! / (d + 3)! with the multiplicities of i, j, k."""
    nv = dim + 1
    w = np.empty((nv, nv, nv))
    for i in range(nv):
        for j in range(nv):
            for k in range(nv):
                mult = {}
                for t in (i, j, k):
                    mult[t] = mult.get(t, 0) + 1
                num = math.factorial(dim)
                for c in mult.values():
                    num *= math.factorial(c)
                w[i, j, k] = num / math.factorial(dim + 3)
    return w


def mass_alpha_full(dim, coords, conn, alpha, v):
    """(M_alpha v)_i = sum_e sum_{j,k} alpha_k v_j int_T lambda_i lambda_j lambda_k
    for every node i, with every column kept (no Dirichlet elimination)."""
    conn = np.asarray(conn, dtype=np.int64)
    vol, _ = element_geometry(dim, coords, conn)
    w = _triple_integral_weights(dim)
    av = np.asarray(alpha, dtype=np.float64)[conn]    # [E, d+1]
    vv = np.asarray(v, dtype=np.float64)[conn]
    # contribution to local vertex i: |T| sum_jk w_ijk v_j alpha_k
    loc = vol[:, None] * np.einsum("ijk,ej,ek->ei", w, vv, av)
    y = np.zeros(np.asarray(coords).shape[0])
    np.add.at(y, conn, loc)
    return y


def rhs(dim, coords, conn, dirichlet, alpha, H, rhok, wu, we, p_n, dt):
    """Right-hand side of the weak problem (Section 3.4) for the test function
    of every node i:
        b_i = int (W~_E - (rho K)) phi_i  -  int alpha_h P^n_h phi_i
              + dt int H W~~_u . grad phi_i
    with W~_E, rho K, H and W~~_u constant per element, alpha and P^n nodal
    (P1); b_i = 0 on Dirichlet nodes.  int_T lambda_i = |T| / (d + 1)."""
    conn = np.asarray(conn, dtype=np.int64)
    vol, grad = element_geometry(dim, coords, conn)
    nv = dim + 1
    src = (np.asarray(we, dtype=np.float64) - np.asarray(rhok, dtype=np.float64)) * vol / nv   # [E]
    wu = np.asarray(wu, dtype=np.float64).reshape(conn.shape[0], dim)
    div = dt * np.asarray(H, dtype=np.float64)[:, None] * vol[:, None] * np.einsum("ekd,ed->ek", grad, wu)
    loc = src[:, None] + div
    b = np.zeros(np.asarray(coords).shape[0])
    np.add.at(b, conn, loc)
    b -= mass_alpha_full(dim, coords, conn, alpha, p_n)
    b[np.asarray(dirichlet).astype(bool)] = 0.0
    return b


def enthalpy(conn, p, rho, gamma):
    """H_e = gamma / (gamma - 1) * mean over the vertices of P / rho_e."""
    conn = np.asarray(conn, dtype=np.int64)
    return gamma / (gamma - 1.0) * np.asarray(p, dtype=np.float64)[conn].mean(axis=1) / np.asarray(rho)


def kinetic(wu, rho, dim):
    """(rho K)_e = |W_u,e|^2 / (2 rho_e)."""
    wu = np.asarray(wu, dtype=np.float64).reshape(-1, dim)
    return (wu * wu).sum(axis=1) / (2.0 * np.asarray(rho, dtype=np.float64))


def post(dim, coords, conn, p_n, dp, wu_tt, rho, gamma, dt):
    """Post-projection updates (Section 3.4, after the weak problem):
    P = P^n + dP; W_u = W~~_u - dt grad dP_h (per element); H and rho K from
    them.  Returns (P, W_u [E, d], H [E], rho K [E])."""
    conn = np.asarray(conn, dtype=np.int64)
    _, grad = element_geometry(dim, coords, conn)
    g = np.einsum("ekd,ek->ed", grad, np.asarray(dp, dtype=np.float64)[conn])
    p = np.asarray(p_n, dtype=np.float64) + np.asarray(dp, dtype=np.float64)
    wu = np.asarray(wu_tt, dtype=np.float64).reshape(-1, dim) - dt * g
    return p, wu, enthalpy(conn, p, rho, gamma), kinetic(wu, rho, dim)


def projection_step(dim, coords, conn, dirichlet, alpha, rho, wu_tt, we, p_n, gamma, dt, n_picard,
                    dp0=None, tol=1e-13):
    """One time step's projection stage: first guesses (Section 3.3), then
    n_picard Picard iterations (Section 3.4) of [operator with beta = H,
    right-hand side, solve for dP (warm start: dp0, then the previous
    iterate), post-projection updates].  Returns a dict with dP, P, W_u, H,
    rho K (after the last update) and the per-iteration solve records."""
    conn = np.asarray(conn, dtype=np.int64)
    H = enthalpy(conn, p_n, rho, gamma)
    rhok = kinetic(wu_tt, rho, dim)
    dp = np.zeros(np.asarray(coords).shape[0]) if dp0 is None else np.asarray(dp0, dtype=np.float64).copy()
    solves = []
    p = np.asarray(p_n, dtype=np.float64).copy()
    wu = np.asarray(wu_tt, dtype=np.float64).reshape(-1, dim).copy()
    for _ in range(n_picard):
        A = PressureMatrix(dim, coords, conn.astype(np.int32), dirichlet, alpha, H, dt * dt)
        b = rhs(dim, coords, conn, dirichlet, alpha, H, rhok, wu_tt, we, p_n, dt)
        dp, st, it, rr = A.cg(b, x0_full=dp, precond=1, tol=tol)
        solves.append({"status": st, "iters": it, "rel_res": rr, "b": b, "H": H})
        p, wu, H, rhok = post(dim, coords, conn, p_n, dp, wu_tt, rho, gamma, dt)
    return {"dp": dp, "p": p, "wu": wu, "H": H, "rhok": rhok, "solves": solves}
