/*
 * FP64 CPU oracle for the P1 finite-element pressure system.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes (Section 3.4, weak problem for the pressure correction):
 *   find dP in the P1 space on the primal simplex mesh with
 *     int alpha dP z  +  dt^2 int H grad dP . grad z  =  <b, z>   for all z,
 *   with alpha = 1/(gamma-1) taken as the P1 interpolant of a nodal field and
 *   H = beta piecewise constant per element.  The stiffness sign is the one
 *   Green's formula gives from the strong form (eq. pressure_dt), the only
 *   sign for which the system is SPD as Section 3.4 states.  The mass matrix
 *   is consistent (no lumping, Section 3.4).
 *
 * How: the plain definition, written out.
 *   1. element matrices from the affine map of each simplex (Gauss-Jordan
 *      inverse of the Jacobian; exact integrals of products of barycentric
 *      coordinates, int_T l0^a0 .. ld^ad = d! |T| prod(a_i!) / (d + sum a_i)!);
 *   2. assembly into CSR over the free (non-Dirichlet) nodes: Dirichlet rows
 *      and columns are eliminated (homogeneous Dirichlet, Section 3.6);
 *   3. textbook conjugate gradient (Hestenes-Stiefel), optionally with the
 *      Jacobi preconditioner, started from the caller's guess (Section 3.4
 *      uses the previous time level as first guess), stopped on the TRUE
 *      relative residual ||b - A x||_2 / ||b||_2;
 *   4. for small systems a dense Cholesky factorisation and solve.
 *
 * Built with -ffp-contract=off so that rounding does not depend on the
 * compiler's choice of fused multiply-adds.  The sparse product may run on
 * several OpenMP threads; each row is still summed in the same order, so
 * results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n_nodes;        /* all mesh nodes */
    int64_t n_free;         /* rows/cols of the reduced matrix */
    int64_t nnz;
    int64_t *rowptr;        /* [n_free+1] */
    int64_t *col;           /* [nnz], free indices, ascending per row */
    double *val;            /* [nnz] */
    int64_t *free_of_node;  /* [n_nodes] free index or -1 on Dirichlet nodes */
    int64_t *node_of_free;  /* [n_free] */
} orc_csr;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Invert the d x d matrix a (row-major) by Gauss-Jordan elimination with
 * partial pivoting.  Returns the determinant (0 if singular). */
static double gauss_jordan_inverse(int d, const double *a, double *inv) {
    double m[3][6];
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < 2 * d; ++c)
            m[r][c] = (c < d) ? a[r * d + c] : (c - d == r ? 1.0 : 0.0);
    double det = 1.0;
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (m[piv][c] == 0.0) return 0.0;
        if (piv != c) {
            for (int k = 0; k < 2 * d; ++k) {
                double t = m[c][k]; m[c][k] = m[piv][k]; m[piv][k] = t;
            }
            det = -det;
        }
        double p = m[c][c];
        det *= p;
        for (int k = 0; k < 2 * d; ++k) m[c][k] /= p;
        for (int r = 0; r < d; ++r) {
            if (r == c) continue;
            double f = m[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * d; ++k) m[r][k] -= f * m[c][k];
        }
    }
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) inv[r * d + c] = m[r][c + d];
    return det;
}

/*
 * Element matrices of one simplex.
 *   xv      [(d+1) * d] vertex coordinates, vertex-major
 *   alpha_v [d+1] nodal alpha at the vertices
 * Outputs (any may be NULL), row-major (d+1) x (d+1):
 *   Me[i][j] = int_T alpha_h phi_i phi_j, alpha_h = sum_k alpha_k phi_k
 *   Ke[i][j] = beta |T| grad phi_i . grad phi_j
 *   Ae       = Me + dt2 * Ke
 *   vol      = |T|, det = det of the affine map (signed)
 * Returns 0, or -1 for a degenerate element.
 */
int orc_element_matrix(int dim, const double *xv, const double *alpha_v, double beta,
                       double dt2, double *Ae, double *Me, double *Ke, double *vol,
                       double *det_out) {
    const int d = dim, nv = dim + 1;
    double J[9], Jinv[9], grad[4][3];
    /* column c of J is v_{c+1} - v_0 */
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) J[r * d + c] = xv[(c + 1) * d + r] - xv[r];
    double det = gauss_jordan_inverse(d, J, Jinv);
    if (det == 0.0) return -1;
    /* barycentric lambda = J^{-1} (x - v0) for vertices 1..d, lambda_0 = 1 - sum */
    for (int k = 1; k <= d; ++k)
        for (int c = 0; c < d; ++c) grad[k][c] = Jinv[(k - 1) * d + c];
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int k = 1; k <= d; ++k) s += grad[k][c];
        grad[0][c] = -s;
    }
    const double T = fabs(det) / factorial(d);
    const double dfac = factorial(d), d3fac = factorial(d + 3);
    for (int i = 0; i < nv; ++i) {
        for (int j = 0; j < nv; ++j) {
            double g = 0.0;
            for (int c = 0; c < d; ++c) g += grad[i][c] * grad[j][c];
            double kij = beta * T * g;
            double mij = 0.0;
            for (int k = 0; k < nv; ++k) {
                int a[4] = {0, 0, 0, 0};
                a[i] += 1; a[j] += 1; a[k] += 1;
                double pf = 1.0;
                for (int m = 0; m < nv; ++m) pf *= factorial(a[m]);
                mij += alpha_v[k] * dfac * T * pf / d3fac;
            }
            if (Me) Me[i * nv + j] = mij;
            if (Ke) Ke[i * nv + j] = kij;
            if (Ae) Ae[i * nv + j] = mij + dt2 * kij;
        }
    }
    if (vol) *vol = T;
    if (det_out) *det_out = det;
    return 0;
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

void orc_csr_free(orc_csr *A) {
    if (!A) return;
    free(A->rowptr); free(A->col); free(A->val);
    free(A->free_of_node); free(A->node_of_free);
    free(A);
}

/*
 * Assemble the reduced matrix A = M_alpha + dt2 K_beta over the free nodes.
 * part: 0 = A, 1 = M_alpha only, 2 = K_beta only (dt2 ignored).
 * Returns 0, -1 bad input (index out of range / degenerate element), -2 OOM.
 */
int orc_assemble(int dim, int64_t n_nodes, const double *coords, int64_t n_elems,
                 const int32_t *conn, const uint8_t *dirichlet, const double *alpha,
                 const double *beta, double dt2, int part, orc_csr **out) {
    const int nv = dim + 1;
    *out = NULL;
    if (dim != 2 && dim != 3) return -1;
    for (int64_t e = 0; e < n_elems * nv; ++e)
        if (conn[e] < 0 || conn[e] >= n_nodes) return -1;

    orc_csr *A = (orc_csr *)calloc(1, sizeof(orc_csr));
    if (!A) return -2;
    A->n_nodes = n_nodes;
    A->free_of_node = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_nodes > 0 ? n_nodes : 1));
    int64_t nf = 0;
    for (int64_t i = 0; i < n_nodes; ++i) A->free_of_node[i] = dirichlet[i] ? -1 : nf++;
    A->n_free = nf;
    A->node_of_free = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nf > 0 ? nf : 1));
    for (int64_t i = 0; i < n_nodes; ++i)
        if (A->free_of_node[i] >= 0) A->node_of_free[A->free_of_node[i]] = i;

    /* node -> element lists */
    int64_t *ne_ptr = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
    int64_t *ne = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_elems * nv + 1));
    for (int64_t e = 0; e < n_elems; ++e)
        for (int a = 0; a < nv; ++a) ne_ptr[conn[e * nv + a] + 1]++;
    for (int64_t i = 0; i < n_nodes; ++i) ne_ptr[i + 1] += ne_ptr[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_nodes + 1));
    memcpy(fill, ne_ptr, sizeof(int64_t) * (size_t)(n_nodes + 1));
    for (int64_t e = 0; e < n_elems; ++e)
        for (int a = 0; a < nv; ++a) ne[fill[conn[e * nv + a]]++] = e;
    free(fill);

    /* sparsity pattern: row i holds every free node that shares an element */
    A->rowptr = (int64_t *)calloc((size_t)nf + 1, sizeof(int64_t));
    int64_t *scratch = (int64_t *)malloc(sizeof(int64_t) * 4096);
    size_t scratch_cap = 4096;
    int64_t total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            A->nnz = total;
            A->col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
            A->val = (double *)calloc((size_t)(total > 0 ? total : 1), sizeof(double));
            if (!A->col || !A->val) { free(ne_ptr); free(ne); free(scratch); orc_csr_free(A); return -2; }
        }
        total = 0;
        for (int64_t r = 0; r < nf; ++r) {
            int64_t i = A->node_of_free[r];
            size_t cnt = 0;
            size_t need = (size_t)(ne_ptr[i + 1] - ne_ptr[i]) * (size_t)nv;
            if (need > scratch_cap) {
                scratch_cap = need;
                scratch = (int64_t *)realloc(scratch, sizeof(int64_t) * scratch_cap);
            }
            for (int64_t k = ne_ptr[i]; k < ne_ptr[i + 1]; ++k) {
                int64_t e = ne[k];
                for (int a = 0; a < nv; ++a) {
                    int64_t f = A->free_of_node[conn[e * nv + a]];
                    if (f >= 0) scratch[cnt++] = f;
                }
            }
            qsort(scratch, cnt, sizeof(int64_t), cmp_i64);
            size_t u = 0;
            for (size_t k = 0; k < cnt; ++k)
                if (u == 0 || scratch[k] != scratch[u - 1]) scratch[u++] = scratch[k];
            if (pass == 1) memcpy(A->col + total, scratch, sizeof(int64_t) * u);
            total += (int64_t)u;
            if (pass == 0) A->rowptr[r + 1] = total;
        }
    }
    free(scratch); free(ne_ptr); free(ne);

    /* values: element loop, scatter each entry into its (row, col) slot */
    double xv[12], av[4], Ae[16], Me[16], Ke[16], vol, det;
    for (int64_t e = 0; e < n_elems; ++e) {
        for (int a = 0; a < nv; ++a) {
            int64_t v = conn[e * nv + a];
            for (int c = 0; c < dim; ++c) xv[a * dim + c] = coords[v * dim + c];
            av[a] = alpha[v];
        }
        if (orc_element_matrix(dim, xv, av, beta[e], dt2, Ae, Me, Ke, &vol, &det) != 0) {
            orc_csr_free(A);
            return -1;
        }
        const double *src = part == 1 ? Me : (part == 2 ? Ke : Ae);
        for (int a = 0; a < nv; ++a) {
            int64_t r = A->free_of_node[conn[e * nv + a]];
            if (r < 0) continue;
            for (int b = 0; b < nv; ++b) {
                int64_t c = A->free_of_node[conn[e * nv + b]];
                if (c < 0) continue;
                int64_t lo = A->rowptr[r], hi = A->rowptr[r + 1] - 1;
                while (lo < hi) {
                    int64_t mid = (lo + hi) / 2;
                    if (A->col[mid] < c) lo = mid + 1; else hi = mid;
                }
                A->val[lo] += src[a * nv + b];
            }
        }
    }
    *out = A;
    return 0;
}

/* y = A x on the free nodes (reduced vectors of length n_free). */
void orc_spmv(const orc_csr *A, const double *x, double *y) {
    const int64_t n = A->n_free;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int64_t k = A->rowptr[r]; k < A->rowptr[r + 1]; ++k) s += A->val[k] * x[A->col[k]];
        y[r] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * Textbook (preconditioned) conjugate gradient on the reduced system.
 *   precond: 0 none, 1 Jacobi (diagonal of A)
 *   x: in = first guess, out = iterate.
 * Stops when the TRUE relative residual ||b - A x|| / ||b|| <= tol.  The
 * recursively updated residual is used to decide when to check; on a failed
 * check the recursion is restarted from the true residual.  After
 * `max_restarts` failed checks, or max_it iterations, it stops and returns 1.
 * stats[0] = iterations, stats[1] = final true relative residual,
 * stats[2] = restarts.
 * Returns 0 on convergence, 1 not converged, -1 breakdown (p.Ap <= 0), -2 OOM.
 */
int orc_cg(const orc_csr *A, const double *b, double *x, int precond, double tol,
           int64_t max_it, int max_restarts, double *stats) {
    const int64_t n = A->n_free;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *dinv = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!r || !z || !p || !q || !dinv) { free(r); free(z); free(p); free(q); free(dinv); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        double dii = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k)
            if (A->col[k] == i) dii = A->val[k];
        dinv[i] = (precond == 1 && dii > 0.0) ? 1.0 / dii : 1.0;
    }
    const double bnorm = sqrt(dot(n, b, b));
    const double target = tol * (bnorm > 0.0 ? bnorm : 1.0);
    int64_t it = 0;
    int restarts = 0, status = 1;
    double true_rel = 0.0;
    for (;;) {
        /* (re)start from the true residual */
        orc_spmv(A, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        double rn = sqrt(dot(n, r, r));
        true_rel = bnorm > 0.0 ? rn / bnorm : rn;
        if (rn <= target) { status = 0; break; }
        if (restarts > max_restarts || it >= max_it) { status = 1; break; }
        for (int64_t i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
        double rz = dot(n, r, z);
        while (it < max_it) {
            orc_spmv(A, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0)) { status = -1; goto done; }
            double a = rz / pq;
            for (int64_t i = 0; i < n; ++i) { x[i] += a * p[i]; r[i] -= a * q[i]; }
            ++it;
            if (sqrt(dot(n, r, r)) <= target) break;
            for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
            double rz_new = dot(n, r, z);
            double beta_cg = rz_new / rz;
            rz = rz_new;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta_cg * p[i];
        }
        ++restarts;
    }
done:
    if (status == -1) {
        orc_spmv(A, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        true_rel = bnorm > 0.0 ? sqrt(dot(n, r, r)) / bnorm : 0.0;
    }
    if (stats) { stats[0] = (double)it; stats[1] = true_rel; stats[2] = (double)restarts; }
    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}

/* Dense Cholesky solve of the reduced system (small n only).
 * Returns 0, -1 if a pivot is not positive (matrix not SPD), -2 OOM. */
int orc_cholesky_solve(const orc_csr *A, const double *b, double *x) {
    const int64_t n = A->n_free;
    double *L = (double *)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
    if (!L) return -2;
    for (int64_t r = 0; r < n; ++r)
        for (int64_t k = A->rowptr[r]; k < A->rowptr[r + 1]; ++k) L[r * n + A->col[k]] = A->val[k];
    for (int64_t j = 0; j < n; ++j) {
        double s = L[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) { free(L); return -1; }
        double ljj = sqrt(s);
        L[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = L[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i) {      /* L y = b */
        double t = b[i];
        for (int64_t k = 0; k < i; ++k) t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) { /* L^T x = y */
        double t = x[i];
        for (int64_t k = i + 1; k < n; ++k) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
    free(L);
    return 0;
}
