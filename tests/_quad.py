"""Brute-force quadrature on simplices for the oracle's pins (test helper).

Points come from the forward affine map of collapsed (Duffy) coordinates with
tensor Gauss-Legendre rules, so nothing here inverts a Jacobian or uses the
closed-form monomial integrals that the oracle uses.
"""
import numpy as np


def ref_rule(dim, order):
    """Points (barycentric lambda_1..lambda_d) and weights on the reference
    simplex {lambda >= 0, sum <= 1}, exact for polynomials up to degree
    2*order - 1 - (dim - 1)."""
    g, w = np.polynomial.legendre.leggauss(order)
    t = 0.5 * (g + 1.0)
    wt = 0.5 * w
    if dim == 2:
        T1, T2 = np.meshgrid(t, t, indexing="ij")
        W = np.outer(wt, wt)
        l1 = T1
        l2 = T2 * (1.0 - T1)
        jac = (1.0 - T1)
        return np.stack([l1.ravel(), l2.ravel()], 1), (W * jac).ravel()
    T1, T2, T3 = np.meshgrid(t, t, t, indexing="ij")
    W = wt[:, None, None] * wt[None, :, None] * wt[None, None, :]
    l1 = T1
    l2 = T2 * (1.0 - T1)
    l3 = T3 * (1.0 - T1) * (1.0 - T2)
    jac = (1.0 - T1) ** 2 * (1.0 - T2)
    return np.stack([l1.ravel(), l2.ravel(), l3.ravel()], 1), (W * jac).ravel()


def element_points(coords, conn, dim, order):
    """Physical quadrature points [E, Q, d], weights [E, Q] and barycentric
    values [Q, d+1] for every element."""
    lam, w = ref_rule(dim, order)
    bary = np.concatenate([1.0 - lam.sum(1, keepdims=True), lam], axis=1)  # [Q, d+1]
    V = coords[conn]                                   # [E, d+1, d]
    pts = np.einsum("qa,ead->eqd", bary, V)
    edges = V[:, 1:, :] - V[:, :1, :]                  # [E, d, d]
    detJ = np.abs(np.linalg.det(edges))
    return pts, detJ[:, None] * w[None, :], bary
