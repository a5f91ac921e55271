"""FP64 CPU oracle for periodic boundaries by vertex merging (Section 3.6:
the vertices of matching periodic boundary faces are merged, which reduces
the unknowns of the pressure system).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  The merged system
is built from its definition: with P the n_nodes x n_dofs matrix that maps
every vertex to its merged unknown (P[i, dof(i)] = 1), the periodic matrix is
P^T A P for the matrix A assembled on the unmerged mesh (every vertex free),
and the load of a merged unknown is P^T b; Dirichlet unknowns are removed
afterwards.  A library sparse product and a direct solve are the only
machinery.  Vectors come back in the caller's numbering with each vertex
carrying its unknown's value.

Parity status: pinned by ``tests/test_oracle_periodic.py`` (symmetry, zero
row sums of the stiffness part, the 5-point stencil across the periodic seam,
manufactured-solution O(h^2) convergence of a y-periodic field).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import PressureMatrix


class PeriodicMatrix:
    """Reduced periodic system (free merged unknowns only)."""

    def __init__(self, dim, coords, conn, dirichlet, master, alpha, beta, dt2, part: int = 0):
        n = np.asarray(coords).shape[0]
        master = np.asarray(master, dtype=np.int64)
        full = PressureMatrix(dim, coords, conn, np.zeros(n, np.uint8), alpha, beta, dt2, part)
        A = full.scipy()
        self.dofs = np.unique(master)                     # one unknown per master vertex
        self.dof_of_node = np.searchsorted(self.dofs, master)
        self.n_nodes, self.n_dofs = n, self.dofs.size
        self.P = sp.csr_matrix((np.ones(n), (np.arange(n), self.dof_of_node)), shape=(n, self.n_dofs))
        Ad = (self.P.T @ A @ self.P).tocsr()
        self.free = ~np.asarray(dirichlet, dtype=bool)[self.dofs]
        self.A = Ad[self.free][:, self.free].tocsr()
        self.A_dofs = Ad

    def to_dofs(self, x_user):
        """Unknowns from caller-numbered values: each master's value."""
        return np.asarray(x_user, dtype=np.float64)[self.dofs]

    def load(self, b_user):
        """Loads of the merged unknowns: P^T b (slaves add onto their master)."""
        return self.P.T @ np.asarray(b_user, dtype=np.float64)

    def to_user(self, x_dofs_free):
        xd = np.zeros(self.n_dofs)
        xd[self.free] = x_dofs_free
        return xd[self.dof_of_node]

    def apply(self, x_user):
        """y = A_periodic x in the caller's numbering (0 on Dirichlet unknowns)."""
        return self.to_user(self.A @ self.to_dofs(x_user)[self.free])

    def residual(self, b_user, x_user):
        b = self.load(b_user)[self.free]
        r = b - self.A @ self.to_dofs(x_user)[self.free]
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(r) / (nb if nb > 0 else 1.0))

    def solve(self, b_user):
        return self.to_user(spla.spsolve(self.A.tocsc(), self.load(b_user)[self.free]))
