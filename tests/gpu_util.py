"""Helpers shared by the GPU tests: upload through the C ABI, and oracle-side
reference values (oracle calls only; nothing here runs the CUDA path)."""
import numpy as np

import oracle


def upload(P, ctx, case, chunk=0, beta=None):
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk)
    P.ps_coeff_set(m, case.alpha, case.beta if beta is None else beta, case.dt2)
    return m


def row_scale(A, x_full):
    """s_i = sum_j |A_ij| |x_j| per free row (0 on Dirichlet rows): the size of
    the terms summed into (A x)_i, which bounds its rounding error."""
    xr = np.abs(A.restrict(x_full))
    s = np.zeros(A.n_free)
    for r in range(A.n_free):
        k0, k1 = A.rowptr[r], A.rowptr[r + 1]
        s[r] = np.abs(A.val[k0:k1]) @ xr[A.col[k0:k1]]
    return A.extend(s)


def row_scale_fast(A, x_full):
    import scipy.sparse as sp
    M = sp.csr_matrix((np.abs(A.val), A.col, A.rowptr), shape=(A.n_free, A.n_free))
    return A.extend(M @ np.abs(A.restrict(x_full)))


def sampled_rows(case, x_full, nodes):
    """(A x)_i for the given nodes, one row at a time from the oracle's element
    matrices (Dirichlet rows 0, Dirichlet columns dropped); also returns the
    row scales sum_j |A_ij x_j|."""
    dim, nv = case.dim, case.dim + 1
    conn = case.conn
    order = np.argsort(conn.ravel(), kind="stable")
    starts = np.searchsorted(conn.ravel()[order], nodes, side="left")
    ends = np.searchsorted(conn.ravel()[order], nodes, side="right")
    dirm = case.dirichlet.astype(bool)
    y = np.zeros(len(nodes))
    sc = np.zeros(len(nodes))
    for t, i in enumerate(nodes):
        if dirm[i]:
            continue
        acc, accs = 0.0, 0.0
        for k in order[starts[t]:ends[t]]:
            e, a = divmod(int(k), nv)
            v = conn[e]
            Ae, _, _, _, _ = oracle.element_matrices(dim, case.coords[v], case.alpha[v], case.beta[e], case.dt2)
            for j in range(nv):
                if not dirm[v[j]]:
                    acc += Ae[a, j] * x_full[v[j]]
                    accs += abs(Ae[a, j] * x_full[v[j]])
        y[t], sc[t] = acc, accs
    return y, sc
