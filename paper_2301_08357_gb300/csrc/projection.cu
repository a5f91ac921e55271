// Projection stage of one time step around the pressure solve (Sections
// 3.3-3.5): first guesses of the enthalpy and kinetic energy, and a Picard
// loop of [operator update, right-hand side of the weak problem, solve,
// post-projection updates].  See ps_projection_step in pressure.h.
//
// These passes run once per Picard iteration (the solve inside runs hundreds
// of CG iterations), so they favour simplicity and determinism: FP64 element
// arithmetic in the caller's element order, the right-hand side gathered per
// node over a node-to-element list in ascending element order (no atomics,
// bitwise reproducible), element geometry recomputed from coordinates.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/pressure.h"
#include "internal.h"

namespace ps {
namespace {

constexpr int kT = 256;
constexpr int kRedBlocks = 256;   // fixed grid of the norm pass (deterministic order)

// Device data of the element passes (caller's numbering), built on first use.
struct ProjData {
    std::vector<DevAlloc> allocs;
    double *x = nullptr;          // [n_nodes * dim] coordinates
    int32_t *conn = nullptr;      // [n_elems * (dim + 1)] vertices of each element
    int64_t *n2e_ptr = nullptr;   // [n_nodes + 1]
    int32_t *n2e = nullptr;       // [n_elems * (dim + 1)]: element * 4 + local vertex
    double *alpha = nullptr;      // [n_nodes]
    uint8_t *dir = nullptr;       // [n_nodes] Dirichlet flags
    double *b = nullptr;          // [n_nodes] right-hand side
    double *loc = nullptr;        // [n_elems * (dim + 1)] per-element contributions before the gather
    double *geo = nullptr;        // [n_elems * (1 + (dim + 1) dim)] |T| and grad lambda_k per element
    int *flag = nullptr;          // enthalpy check
    int64_t alpha_version = -1;
    // general-EOS Newton iteration (allocated on its first call)
    std::vector<DevAlloc> eos_allocs;
    double *mi = nullptr;         // [n_nodes] m_i = sum_e |T_e| / (d+1)
    double *si = nullptr;         // [n_nodes] s_i = sum_e |T_e| / ((d+1) rho_e)
    double *c = nullptr;          // [n_nodes] right-hand side without the mass term
    double *r = nullptr;          // [n_nodes] Newton right-hand side J dP - F(dP)
    double *au = nullptr;         // [n_nodes] alpha_i = Q'_i / m_i
    double *y = nullptr;          // [n_nodes] J dP
    double *red = nullptr;        // [2 * kRedBlocks] partial sums of ||F||^2, ||c||^2
};

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return PS_OK;
    ps_set_last_error(cudaGetErrorString(e));
    return cuda_status(e);
}

// Cofactor vectors c_k of a simplex (grad lambda_k = c_k / det), k = 0..d,
// and det = det[x_1 - x_0, ..., x_d - x_0].
template <int D>
__device__ __forceinline__ double cofactors(const double (&v)[D + 1][D], double (&c)[D + 1][D]) {
    if constexpr (D == 3) {
        const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
        const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
        const double e3[3] = {v[3][0] - v[0][0], v[3][1] - v[0][1], v[3][2] - v[0][2]};
        c[1][0] = e2[1] * e3[2] - e2[2] * e3[1];
        c[1][1] = e2[2] * e3[0] - e2[0] * e3[2];
        c[1][2] = e2[0] * e3[1] - e2[1] * e3[0];
        c[2][0] = e3[1] * e1[2] - e3[2] * e1[1];
        c[2][1] = e3[2] * e1[0] - e3[0] * e1[2];
        c[2][2] = e3[0] * e1[1] - e3[1] * e1[0];
        c[3][0] = e1[1] * e2[2] - e1[2] * e2[1];
        c[3][1] = e1[2] * e2[0] - e1[0] * e2[2];
        c[3][2] = e1[0] * e2[1] - e1[1] * e2[0];
        for (int a = 0; a < 3; ++a) c[0][a] = -(c[1][a] + c[2][a] + c[3][a]);
        return e1[0] * c[1][0] + e1[1] * c[1][1] + e1[2] * c[1][2];
    } else {
        const double e1[2] = {v[1][0] - v[0][0], v[1][1] - v[0][1]};
        const double e2[2] = {v[2][0] - v[0][0], v[2][1] - v[0][1]};
        c[1][0] = e2[1];
        c[1][1] = -e2[0];
        c[2][0] = -e1[1];
        c[2][1] = e1[0];
        for (int a = 0; a < 2; ++a) c[0][a] = -(c[1][a] + c[2][a]);
        return e1[0] * e2[1] - e1[1] * e2[0];
    }
}

// Element enthalpy from the vertex mean Pbar of the pressure:
// H_e = (h1 Pbar + hb Pbar^2 / rho_e) / rho_e, i.e. (rho e(Pbar) + Pbar) / rho_e
// for rho e = a P + b P^2 / rho (h1 = a + 1, hb = b; the ideal gas passes
// h1 = gamma / (gamma - 1), hb = 0).
__device__ __forceinline__ double enthalpy(double pbar, double rho, double h1, double hb) {
    return (h1 * pbar + hb * pbar * pbar / rho) / rho;
}

// First guesses: H_e from P^n, (rho K)_e = |W~~_u,e|^2 / (2 rho_e).
template <int D>
__global__ void __launch_bounds__(kT) k_pj_first(int64_t n_el, const int32_t *__restrict__ conn,
                                                 const double *__restrict__ p, const double *__restrict__ rho,
                                                 const double *__restrict__ wu, double h1, double hb,
                                                 double *__restrict__ H, double *__restrict__ rhok) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        double pb = 0.0, u2 = 0.0;
        for (int k = 0; k <= D; ++k) pb += p[conn[e * (D + 1) + k]];
        for (int a = 0; a < D; ++a) u2 += wu[e * D + a] * wu[e * D + a];
        H[e] = enthalpy(pb / (D + 1), rho[e], h1, hb);
        rhok[e] = 0.5 * u2 / rho[e];
    }
}

__global__ void __launch_bounds__(kT) k_pj_check(int64_t n, const double *__restrict__ v, int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(v[i] > 0.0) || !isfinite(v[i])) atomicOr(flag, 1);
}

// Element geometry, once per mesh (FP64): geo[e G] = |T_e|, then
// grad lambda_k = c_k / det for k = 0..d (G = 1 + (d+1) d).  The element
// passes below read it instead of recomputing cofactors from coordinates:
// FP64 arithmetic is scarce on this part.
template <int D>
__global__ void __launch_bounds__(kT) k_pj_geometry(int64_t n_el, const int32_t *__restrict__ conn,
                                                    const double *__restrict__ x, double *__restrict__ geo) {
    constexpr int G = 1 + (D + 1) * D;
    constexpr double fact = D == 3 ? 6.0 : 2.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        double v[D + 1][D], c[D + 1][D];
        for (int q = 0; q <= D; ++q) {
            const int64_t g = conn[e * (D + 1) + q];
            for (int a = 0; a < D; ++a) v[q][a] = x[g * D + a];
        }
        const double det = cofactors<D>(v, c);
        const double inv = 1.0 / det;
        geo[e * G] = fabs(det) / fact;
        for (int k = 0; k <= D; ++k)
            for (int a = 0; a < D; ++a) geo[e * G + 1 + k * D + a] = c[k][a] * inv;
    }
}

// Right-hand side of the weak problem, in two passes.  Element pass (one
// thread per element): the contribution to each local vertex k,
//   (W~_E - rho K)_e |T| / (d+1)                       source term
// + dt H_e |T| W~~_u,e . grad lambda_k                 divergence term
// - (M^e_alpha P^n)_k = cm (S X + Q + S P_k + alpha_k (X + 2 P_k))
// with S = sum alpha, X = sum P, Q = sum alpha P over the element's vertices
// and cm = |T| d! / (d+3)!; alpha == nullptr drops the mass term (the
// general-EOS residual carries it itself).  Node pass (k_pj_gather): b_i is
// the sum of its vertices' contributions in ascending element order over a
// node-to-element list (deterministic, no atomics), 0 on Dirichlet nodes.
template <int D>
__global__ void __launch_bounds__(kT) k_pj_elem_rhs(int64_t n_el, const int32_t *__restrict__ conn,
                                                    const double *__restrict__ geo, const double *__restrict__ alpha,
                                                    const double *__restrict__ H, const double *__restrict__ rhok,
                                                    const double *__restrict__ wu, const double *__restrict__ we,
                                                    const double *__restrict__ p, double dt, double *__restrict__ loc) {
    constexpr int G = 1 + (D + 1) * D;
    constexpr double cmf = D == 3 ? 1.0 / 120.0 : 1.0 / 60.0;   // d! / (d+3)!
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const double *ge = geo + e * G;
        const double vol = ge[0];
        double al[D + 1], pv[D + 1], u[D];
        for (int q = 0; q <= D; ++q) {
            const int64_t g = conn[e * (D + 1) + q];
            al[q] = alpha ? alpha[g] : 0.0;
            pv[q] = alpha ? p[g] : 0.0;
        }
        for (int a = 0; a < D; ++a) u[a] = wu[e * D + a];
        double S = 0.0, X = 0.0, Q = 0.0;
        for (int q = 0; q <= D; ++q) {
            S += al[q];
            X += pv[q];
            Q += al[q] * pv[q];
        }
        const double cm = vol * cmf;
        const double src = (we[e] - rhok[e]) * vol / (D + 1);
        const double dhv = dt * H[e] * vol;
        for (int k = 0; k <= D; ++k) {
            double gw = 0.0;
            for (int a = 0; a < D; ++a) gw += ge[1 + k * D + a] * u[a];
            const double mass = alpha ? cm * (S * X + Q + S * pv[k] + al[k] * (X + 2.0 * pv[k])) : 0.0;
            loc[e * (D + 1) + k] = src + dhv * gw - mass;
        }
    }
}

// b_i = sum over the node's (element, vertex) incidences, ascending element
// order, of loc[e (d+1) + k]; 0 on Dirichlet nodes (dir may be nullptr: no
// masking).  Also the lumped weights: loc = w_e per element (nv = 1).
__global__ void __launch_bounds__(kT) k_pj_gather(int64_t n_nodes, const int64_t *__restrict__ n2e_ptr,
                                                  const int32_t *__restrict__ n2e, const uint8_t *__restrict__ dir,
                                                  const double *__restrict__ loc, int nv, double *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        if (dir && dir[i]) {
            b[i] = 0.0;
            continue;
        }
        double acc = 0.0;
        for (int64_t t = n2e_ptr[i]; t < n2e_ptr[i + 1]; ++t) {
            const int code = n2e[t];
            const int64_t e = code >> 2;
            acc += nv == 1 ? loc[e] : loc[e * nv + (code & 3)];
        }
        b[i] = acc;
    }
}

// Post-projection: W_u = W~~_u - dt grad dP_h, P = P^n + dP (vertex mean for
// H), H from it (enthalpy above), rho K = |W_u|^2 / (2 rho).
template <int D>
__global__ void __launch_bounds__(kT) k_pj_post(int64_t n_el, const int32_t *__restrict__ conn,
                                                const double *__restrict__ geo, const double *__restrict__ pn,
                                                const double *__restrict__ dp, const double *__restrict__ wu_tt,
                                                const double *__restrict__ rho, double h1, double hb, double dt,
                                                double *__restrict__ wu_new, double *__restrict__ H,
                                                double *__restrict__ rhok) {
    constexpr int G = 1 + (D + 1) * D;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const double *ge = geo + e * G;
        double d[D + 1];
        double pb = 0.0;
        for (int q = 0; q <= D; ++q) {
            const int64_t g = conn[e * (D + 1) + q];
            d[q] = dp[g];
            pb += pn[g] + dp[g];
        }
        double u2 = 0.0;
        for (int a = 0; a < D; ++a) {
            double gr = 0.0;
            for (int q = 0; q <= D; ++q) gr += ge[1 + q * D + a] * d[q];
            const double u = wu_tt[e * D + a] - dt * gr;
            wu_new[e * D + a] = u;
            u2 += u * u;
        }
        H[e] = enthalpy(pb / (D + 1), rho[e], h1, hb);
        rhok[e] = 0.5 * u2 / rho[e];
    }
}

__global__ void __launch_bounds__(kT) k_pj_add(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                                               double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a[i] + b[i];
}

// Lumped weights of the general-EOS mass sum, per element: w_e = |T_e|/(d+1)
// into w[e] and w_e / rho_e into wr[e]; k_pj_gather then forms
// m_i = sum_e w_e and s_i = sum_e w_e / rho_e over each node's elements in
// ascending order (vertex quadrature).
template <int D>
__global__ void __launch_bounds__(kT) k_nt_elem_weights(int64_t n_el, const double *__restrict__ geo,
                                                        const double *__restrict__ rho, double *__restrict__ w,
                                                        double *__restrict__ wr) {
    constexpr int G = 1 + (D + 1) * D;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const double we = geo[e * G] / (D + 1);
        w[e] = we;
        wr[e] = we / rho[e];
    }
}

// One Newton linearisation at dP (rho e = a P + b P^2 / rho, P = P^n + dP):
//   Q_i = sum_e w_ei rho e(P_i, rho_e) = P_i (a m_i + b s_i P_i)
//   Q'_i = a m_i + 2 b s_i P_i,   alpha_i = Q'_i / m_i
//   r_i = c_i - Q_i + Q'_i dP_i   (J dP - F(dP); 0 on Dirichlet nodes)
// flag: a free node whose Q'_i is not positive and finite.
__global__ void __launch_bounds__(kT) k_nt_linearise(int64_t n, const uint8_t *__restrict__ dir,
                                                     const double *__restrict__ pn, const double *__restrict__ dp,
                                                     const double *__restrict__ mi, const double *__restrict__ si,
                                                     const double *__restrict__ c, double a, double b,
                                                     double *__restrict__ alpha, double *__restrict__ r, int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double P = pn[i] + dp[i];
        const double m = mi[i], sw = si[i];
        const double q = P * (a * m + b * sw * P);
        const double qp = a * m + 2.0 * b * sw * P;
        const bool ok = qp > 0.0 && isfinite(qp);
        // a rejected entry still leaves a positive alpha in the node records
        // (their sign bit marks Dirichlet nodes); the call then fails
        alpha[i] = (m > 0.0 && ok) ? qp / m : a;
        if (dir[i]) {
            r[i] = 0.0;
            continue;
        }
        if (!ok) atomicOr(flag, 1);
        r[i] = c[i] - q + qp * dp[i];
    }
}

// Partial sums over free nodes of |J dP - r|^2 = |F(dP)|^2 and |c|^2, one per
// block of a fixed grid (kRedBlocks); the host adds them in block order.
__global__ void __launch_bounds__(kT) k_nt_norms(int64_t n, const uint8_t *__restrict__ dir,
                                                 const double *__restrict__ y, const double *__restrict__ r,
                                                 const double *__restrict__ c, double *__restrict__ red) {
    __shared__ double sf[kT], sc[kT];
    double f = 0.0, cc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (dir[i]) continue;
        const double d = y[i] - r[i];
        f += d * d;
        cc += c[i] * c[i];
    }
    sf[threadIdx.x] = f;
    sc[threadIdx.x] = cc;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sf[threadIdx.x] += sf[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        red[blockIdx.x] = sf[0];
        red[kRedBlocks + blockIdx.x] = sc[0];
    }
}

int grid(int64_t n, int sms) {
    int64_t g = (n + kT - 1) / kT;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    return (int)(g < 1 ? 1 : g);
}

// Build (or refresh) the device data of the element passes.  The caller
// holds the context mutex.
int ensure_proj(ps_mesh *m) {
    ProjData *P = static_cast<ProjData *>(m->proj);
    const PrepMesh &pm = m->prep;
    const int dim = pm.dim, nv = dim + 1;
    const int64_t N = pm.n_nodes, E = pm.n_elems;
    if (!P) {
        P = new ProjData();
        ps_ctx *c = m->ctx;
        auto A = [&](void **dst, size_t bytes) { return dalloc(c, dst, bytes, P->allocs); };
        void *p;
        int rc = A(&p, (size_t)N * dim * 8);
        P->x = (double *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)E * nv * 4), P->conn = (int32_t *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)(N + 1) * 8), P->n2e_ptr = (int64_t *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)E * nv * 4), P->n2e = (int32_t *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)N * 8), P->alpha = (double *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)N), P->dir = (uint8_t *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)N * 8), P->b = (double *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)E * nv * 8), P->loc = (double *)p;
        if (rc == PS_OK) rc = A(&p, (size_t)E * (1 + nv * dim) * 8), P->geo = (double *)p;
        if (rc == PS_OK) rc = A(&p, 256), P->flag = (int *)p;
        if (rc != PS_OK) {
            dfree_all(c, P->allocs);
            delete P;
            return rc;
        }
        // connectivity in the caller's element order, rebuilt from the patch
        // records (vertex order within an element is irrelevant to the passes)
        std::vector<int32_t> conn((size_t)E * nv, -1);
        for (int ch = 0; ch < pm.n_chunks; ++ch) {
            const ChunkDesc &cd = pm.chunks[ch];
            for (int q = 0; q < cd.n_patch; ++q) {
                const uint16_t *rec = &pm.pids[(int64_t)(cd.patch_off + q) * kPatchIds];
                const int mm = rec[0];
                for (int j = 0; j < mm; ++j) {
                    const int32_t src = pm.elem_src[(int64_t)(cd.patch_off + q) * kPatchMax + j];
                    int loc[4];
                    int nl = 0;
                    loc[nl++] = rec[1];
                    if (dim == 3) loc[nl++] = rec[2];
                    loc[nl++] = rec[3 + j];
                    loc[nl++] = rec[3 + j + 1];
                    for (int a = 0; a < nv; ++a)
                        conn[(size_t)src * nv + a] = pm.loc_orig[cd.node_off + loc[a]];
                }
            }
        }
        std::vector<int64_t> ptr(N + 1, 0);
        for (int64_t e = 0; e < E; ++e)
            for (int a = 0; a < nv; ++a) ptr[conn[(size_t)e * nv + a] + 1]++;
        for (int64_t i = 0; i < N; ++i) ptr[i + 1] += ptr[i];
        std::vector<int32_t> n2e((size_t)E * nv);
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t e = 0; e < E; ++e)
            for (int a = 0; a < nv; ++a) n2e[fill[conn[(size_t)e * nv + a]]++] = (int32_t)(e * 4 + a);
        std::vector<uint8_t> dir(N);
        for (int64_t i = 0; i < N; ++i) dir[i] = pm.dirichlet_new[pm.new_of_old[i]];
        cudaError_t er = cudaMemcpy(P->x, m->coords_host.data(), (size_t)N * dim * 8, cudaMemcpyHostToDevice);
        if (er == cudaSuccess) er = cudaMemcpy(P->conn, conn.data(), conn.size() * 4, cudaMemcpyHostToDevice);
        if (er == cudaSuccess) er = cudaMemcpy(P->n2e_ptr, ptr.data(), ptr.size() * 8, cudaMemcpyHostToDevice);
        if (er == cudaSuccess) er = cudaMemcpy(P->n2e, n2e.data(), n2e.size() * 4, cudaMemcpyHostToDevice);
        if (er == cudaSuccess) er = cudaMemcpy(P->dir, dir.data(), dir.size(), cudaMemcpyHostToDevice);
        if (er != cudaSuccess) {
            dfree_all(c, P->allocs);
            delete P;
            return cuda_rc(er);
        }
        // element geometry once per mesh: |T| and the barycentric gradients
        if (dim == 3) k_pj_geometry<3><<<grid(E, m->ctx->sms), kT>>>(E, P->conn, P->x, P->geo);
        else k_pj_geometry<2><<<grid(E, m->ctx->sms), kT>>>(E, P->conn, P->x, P->geo);
        er = cudaGetLastError();
        if (er == cudaSuccess) er = cudaDeviceSynchronize();
        if (er != cudaSuccess) {
            dfree_all(c, P->allocs);
            delete P;
            return cuda_rc(er);
        }
        m->proj = P;
    }
    if (P->alpha_version != m->alpha_version && (int64_t)m->alpha_host.size() == N) {
        cudaError_t er = cudaMemcpy(P->alpha, m->alpha_host.data(), (size_t)N * 8, cudaMemcpyHostToDevice);
        if (er != cudaSuccess) return cuda_rc(er);
        P->alpha_version = m->alpha_version;
    }
    return PS_OK;
}

// Device arrays of the general-EOS Newton iteration.  The caller holds the
// context mutex.
int ensure_eos(ps_mesh *m) {
    ProjData *P = static_cast<ProjData *>(m->proj);
    if (P->mi) return PS_OK;
    const int64_t N = m->prep.n_nodes;
    double **dst[] = {&P->mi, &P->si, &P->c, &P->r, &P->au, &P->y};
    for (double **d : dst) {
        void *q = nullptr;
        int rc = dalloc(m->ctx, &q, (size_t)N * 8, P->eos_allocs);
        if (rc == PS_OK) *d = (double *)q;
        else {
            dfree_all(m->ctx, P->eos_allocs);
            for (double **e : dst) *e = nullptr;
            return rc;
        }
    }
    void *q = nullptr;
    int rc = dalloc(m->ctx, &q, 2 * kRedBlocks * 8, P->eos_allocs);
    if (rc != PS_OK) {
        dfree_all(m->ctx, P->eos_allocs);
        for (double **e : dst) *e = nullptr;
        return rc;
    }
    P->red = (double *)q;
    return PS_OK;
}

// Check that every enthalpy is positive and finite (the operator needs it).
int check_positive(ps_mesh *m, const double *H, cudaStream_t s) {
    ProjData *P = static_cast<ProjData *>(m->proj);
    int rc = cuda_rc(cudaMemsetAsync(P->flag, 0, sizeof(int), s));
    if (rc != PS_OK) return rc;
    k_pj_check<<<grid(m->prep.n_elems, m->ctx->sms), kT, 0, s>>>(m->prep.n_elems, H, P->flag);
    int h = 0;
    rc = cuda_rc(cudaMemcpyAsync(&h, P->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (rc == PS_OK) rc = cuda_rc(cudaStreamSynchronize(s));
    if (rc != PS_OK) return rc;
    if (h) {
        ps_set_last_error("projection step: an element enthalpy is not positive and finite");
        return PS_EINVAL;
    }
    return PS_OK;
}

}  // namespace

void projection_release(ps_mesh *m) {
    if (!m->proj) return;
    ProjData *P = static_cast<ProjData *>(m->proj);
    dfree_all(m->ctx, P->eos_allocs);
    dfree_all(m->ctx, P->allocs);
    delete P;
    m->proj = nullptr;
}

}  // namespace ps

using namespace ps;

extern "C" void ps_projection_opts_default(ps_projection_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->gamma = 1.4;
    o->dt = 0.0;
    o->n_picard = 2;
    ps_solve_opts_default(&o->solve);
}

extern "C" int ps_projection_step(ps_mesh *m, const ps_projection_opts *o, const double *rho, const double *wu,
                                  const double *we, const double *pn, double *dp, double *p_out, double *wu_out,
                                  double *h_out, double *rhok_out, ps_solve_info *info, void *stream) {
    if (!m || !o || !rho || !wu || !we || !pn || !dp || !p_out || !wu_out || !h_out || !rhok_out) return PS_EINVAL;
    if (!(o->gamma > 1.0) || !std::isfinite(o->gamma) || !(o->dt > 0.0) || !std::isfinite(o->dt)) return PS_EINVAL;
    if (o->n_picard < 1 || o->n_picard > 64) return PS_EINVAL;
    if (!m->coeff_ok || !m->alpha_set || m->alpha_newton) return PS_ESTATE;
    if (m->prep.n_elems >= ((int64_t)1 << 29)) return PS_EINVAL;   // element * 4 + vertex fits in int32
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int dim = m->prep.dim;
    const int64_t N = m->prep.n_nodes, E = m->prep.n_elems;
    const double g1 = o->gamma / (o->gamma - 1.0);
    const double dt = o->dt;
    ps_solve_info acc;
    std::memset(&acc, 0, sizeof(acc));
    int rc;
    {
        std::lock_guard<std::mutex> lk(m->ctx->mu);
        rc = cuda_rc(cudaSetDevice(m->ctx->device));
        if (rc == PS_OK) rc = ensure_proj(m);
        if (rc != PS_OK) return rc;
        ProjData *P = static_cast<ProjData *>(m->proj);
        const int g = grid(E, m->ctx->sms);
        if (dim == 3) k_pj_first<3><<<g, kT, 0, s>>>(E, P->conn, pn, rho, wu, g1, 0.0, h_out, rhok_out);
        else k_pj_first<2><<<g, kT, 0, s>>>(E, P->conn, pn, rho, wu, g1, 0.0, h_out, rhok_out);
        rc = cuda_rc(cudaGetLastError());
        if (rc != PS_OK) return rc;
    }
    for (int k = 0; k < o->n_picard; ++k) {
        {
            std::lock_guard<std::mutex> lk(m->ctx->mu);
            ProjData *P = static_cast<ProjData *>(m->proj);
            rc = check_positive(m, h_out, s);
            if (rc == PS_OK) rc = beta_update_device(m, h_out, dt * dt, s);
            if (rc != PS_OK) return rc;
            const int ge = grid(E, m->ctx->sms);
            if (dim == 3)
                k_pj_elem_rhs<3><<<ge, kT, 0, s>>>(E, P->conn, P->geo, P->alpha, h_out, rhok_out, wu, we, pn, dt, P->loc);
            else
                k_pj_elem_rhs<2><<<ge, kT, 0, s>>>(E, P->conn, P->geo, P->alpha, h_out, rhok_out, wu, we, pn, dt, P->loc);
            k_pj_gather<<<grid(N, m->ctx->sms), kT, 0, s>>>(N, P->n2e_ptr, P->n2e, P->dir, P->loc, dim + 1, P->b);
            rc = cuda_rc(cudaGetLastError());
            if (rc != PS_OK) return rc;
        }
        ps_solve_info inf;
        rc = ps_pressure_solve(m, static_cast<ProjData *>(m->proj)->b, dp, &o->solve, &inf, stream);
        const int64_t it_in = acc.iters_inner + inf.iters_inner, it_out = acc.iters_outer + inf.iters_outer;
        const int64_t launches = acc.kernel_launches + inf.kernel_launches;
        acc = inf;
        acc.iters_inner = it_in;
        acc.iters_outer = it_out;
        acc.kernel_launches = launches;
        if (rc != PS_OK) break;
        {
            std::lock_guard<std::mutex> lk(m->ctx->mu);
            ProjData *P = static_cast<ProjData *>(m->proj);
            const int g = grid(E, m->ctx->sms);
            if (dim == 3)
                k_pj_post<3><<<g, kT, 0, s>>>(E, P->conn, P->geo, pn, dp, wu, rho, g1, 0.0, dt, wu_out, h_out, rhok_out);
            else
                k_pj_post<2><<<g, kT, 0, s>>>(E, P->conn, P->geo, pn, dp, wu, rho, g1, 0.0, dt, wu_out, h_out, rhok_out);
            k_pj_add<<<grid(N, m->ctx->sms), kT, 0, s>>>(N, pn, dp, p_out);
            rc = cuda_rc(cudaGetLastError());
            if (rc != PS_OK) return rc;
        }
    }
    if (rc == PS_OK) rc = cuda_rc(cudaStreamSynchronize(s));
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = acc;
    return rc;
}

// ---------------------------------------------------------------- general EOS
extern "C" void ps_eos_opts_default(ps_eos_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eos_a = 2.5;
    o->eos_b = 0.0;
    o->dt = 0.0;
    o->n_picard = 2;
    o->max_newton = 8;
    o->newton_tol = 1e-8;
    ps_solve_opts_default(&o->solve);
}

namespace {

void add_solve(ps_solve_info &acc, const ps_solve_info &inf) {
    const int64_t it_in = acc.iters_inner + inf.iters_inner, it_out = acc.iters_outer + inf.iters_outer;
    const int64_t launches = acc.kernel_launches + inf.kernel_launches;
    acc = inf;
    acc.iters_inner = it_in;
    acc.iters_outer = it_out;
    acc.kernel_launches = launches;
}

// ||F(dP)|| / ||c|| over the free nodes, F = J dP - r with J the lumped
// operator now on the mesh (FP64 apply); deterministic (fixed-order sums).
// Also returns the linearisation's rejection flag (one synchronisation for
// both).
int newton_residual(ps_mesh *m, const double *dp, cudaStream_t s, double *res, int *flag) {
    ProjData *P = static_cast<ProjData *>(m->proj);
    int rc = ps_pressure_apply(m, dp, P->y, PS_F64, s);
    if (rc != PS_OK) return rc;
    std::vector<double> red(2 * kRedBlocks);
    {
        std::lock_guard<std::mutex> lk(m->ctx->mu);
        k_nt_norms<<<kRedBlocks, kT, 0, s>>>(m->prep.n_nodes, P->dir, P->y, P->r, P->c, P->red);
        rc = cuda_rc(cudaGetLastError());
        if (rc == PS_OK)
            rc = cuda_rc(cudaMemcpyAsync(red.data(), P->red, red.size() * 8, cudaMemcpyDeviceToHost, s));
        if (rc == PS_OK) rc = cuda_rc(cudaMemcpyAsync(flag, P->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (rc == PS_OK) rc = cuda_rc(cudaStreamSynchronize(s));
        if (rc != PS_OK) return rc;
    }
    double ff = 0.0, cc = 0.0;
    for (int b = 0; b < kRedBlocks; ++b) {
        ff += red[b];
        cc += red[kRedBlocks + b];
    }
    *res = std::sqrt(ff) / (cc > 0.0 ? std::sqrt(cc) : 1.0);
    return PS_OK;
}

}  // namespace

extern "C" int ps_projection_step_eos(ps_mesh *m, const ps_eos_opts *o, const double *rho, const double *wu,
                                      const double *we, const double *pn, double *dp, double *p_out,
                                      double *wu_out, double *h_out, double *rhok_out, double *res_host,
                                      ps_solve_info *info, void *stream) {
    if (!m || !o || !rho || !wu || !we || !pn || !dp || !p_out || !wu_out || !h_out || !rhok_out) return PS_EINVAL;
    if (!(o->eos_a > 0.0) || !std::isfinite(o->eos_a) || !(o->eos_b >= 0.0) || !std::isfinite(o->eos_b))
        return PS_EINVAL;
    if (!(o->dt > 0.0) || !std::isfinite(o->dt) || std::isnan(o->newton_tol)) return PS_EINVAL;
    if (o->n_picard < 1 || o->n_picard > 64 || o->max_newton < 1 || o->max_newton > 64) return PS_EINVAL;
    if (m->d_slave_ptr) {
        ps_set_last_error("general-EOS projection: periodic meshes are not supported");
        return PS_EINVAL;
    }
    if (!m->dev.lumped) {
        ps_set_last_error("general-EOS projection: the mesh needs lumped mass (ps_mesh_set_mass)");
        return PS_ESTATE;
    }
    if (m->prep.n_elems >= ((int64_t)1 << 29)) return PS_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int dim = m->prep.dim;
    const int64_t N = m->prep.n_nodes, E = m->prep.n_elems;
    const double a = o->eos_a, b = o->eos_b, dt = o->dt;
    const double h1 = a + 1.0, hb = b;
    const double tol = o->newton_tol;
    const bool check = tol > 0.0 || res_host;
    const int stride = o->max_newton + 1;
    if (res_host)
        for (int k = 0; k < o->n_picard * stride; ++k) res_host[k] = -1.0;
    ps_solve_info acc;
    std::memset(&acc, 0, sizeof(acc));
    int rc;
    {
        std::lock_guard<std::mutex> lk(m->ctx->mu);
        rc = cuda_rc(cudaSetDevice(m->ctx->device));
        if (rc == PS_OK) rc = ensure_proj(m);
        if (rc == PS_OK) rc = ensure_eos(m);
        if (rc != PS_OK) return rc;
        ProjData *P = static_cast<ProjData *>(m->proj);
        const int ge = grid(E, m->ctx->sms), gn = grid(N, m->ctx->sms);
        // the per-element weights use the two halves of the contribution buffer
        double *w = P->loc, *wr = P->loc + E;
        if (dim == 3) {
            k_pj_first<3><<<ge, kT, 0, s>>>(E, P->conn, pn, rho, wu, h1, hb, h_out, rhok_out);
            k_nt_elem_weights<3><<<ge, kT, 0, s>>>(E, P->geo, rho, w, wr);
        } else {
            k_pj_first<2><<<ge, kT, 0, s>>>(E, P->conn, pn, rho, wu, h1, hb, h_out, rhok_out);
            k_nt_elem_weights<2><<<ge, kT, 0, s>>>(E, P->geo, rho, w, wr);
        }
        k_pj_gather<<<gn, kT, 0, s>>>(N, P->n2e_ptr, P->n2e, nullptr, w, 1, P->mi);
        k_pj_gather<<<gn, kT, 0, s>>>(N, P->n2e_ptr, P->n2e, nullptr, wr, 1, P->si);
        rc = cuda_rc(cudaGetLastError());
        if (rc != PS_OK) return rc;
    }
    bool converged = true;
    for (int k = 0; k < o->n_picard && rc == PS_OK; ++k) {
        {
            std::lock_guard<std::mutex> lk(m->ctx->mu);
            ProjData *P = static_cast<ProjData *>(m->proj);
            rc = check_positive(m, h_out, s);
            if (rc == PS_OK) rc = beta_update_device(m, h_out, dt * dt, s, false);
            if (rc != PS_OK) return rc;
            const int ge = grid(E, m->ctx->sms);
            if (dim == 3)
                k_pj_elem_rhs<3><<<ge, kT, 0, s>>>(E, P->conn, P->geo, nullptr, h_out, rhok_out, wu, we, pn, dt, P->loc);
            else
                k_pj_elem_rhs<2><<<ge, kT, 0, s>>>(E, P->conn, P->geo, nullptr, h_out, rhok_out, wu, we, pn, dt, P->loc);
            k_pj_gather<<<grid(N, m->ctx->sms), kT, 0, s>>>(N, P->n2e_ptr, P->n2e, P->dir, P->loc, dim + 1, P->c);
            rc = cuda_rc(cudaGetLastError());
            if (rc != PS_OK) return rc;
        }
        converged = !(tol > 0.0);
        for (int j = 0;; ++j) {
            {
                std::lock_guard<std::mutex> lk(m->ctx->mu);
                ProjData *P = static_cast<ProjData *>(m->proj);
                rc = cuda_rc(cudaMemsetAsync(P->flag, 0, sizeof(int), s));
                if (rc != PS_OK) return rc;
                k_nt_linearise<<<grid(N, m->ctx->sms), kT, 0, s>>>(N, P->dir, pn, dp, P->mi, P->si, P->c, a, b,
                                                                    P->au, P->r, P->flag);
                // the Jacobi preconditioner of this Picard iteration's Newton
                // solves is the diagonal of its first Jacobian (beta is fixed
                // within the iteration; alpha moves little between steps)
                rc = alpha_update_device(m, P->au, s, j == 0);
                if (rc != PS_OK) return rc;
                m->coeff_ok = true;
                m->alpha_set = true;
                m->alpha_newton = true;
            }
            int bad = 0;
            double res = 0.0;
            if (check) {
                rc = newton_residual(m, dp, s, &res, &bad);
            } else {
                std::lock_guard<std::mutex> lk(m->ctx->mu);
                rc = cuda_rc(cudaMemcpyAsync(&bad, static_cast<ProjData *>(m->proj)->flag, sizeof(int),
                                             cudaMemcpyDeviceToHost, s));
                if (rc == PS_OK) rc = cuda_rc(cudaStreamSynchronize(s));
            }
            if (rc != PS_OK) return rc;
            if (bad) {
                ps_set_last_error("general-EOS projection: a Jacobian entry Q'_i is not positive and finite");
                return PS_EINVAL;
            }
            if (check) {
                if (res_host) res_host[k * stride + j] = res;
                if (tol > 0.0 && res <= tol) {
                    converged = true;
                    break;
                }
            }
            if (j == o->max_newton) break;
            ps_solve_info inf;
            rc = ps_pressure_solve(m, static_cast<ProjData *>(m->proj)->r, dp, &o->solve, &inf, stream);
            add_solve(acc, inf);
            if (rc != PS_OK) break;
        }
        if (rc != PS_OK) break;
        {
            std::lock_guard<std::mutex> lk(m->ctx->mu);
            ProjData *P = static_cast<ProjData *>(m->proj);
            const int g = grid(E, m->ctx->sms);
            if (dim == 3)
                k_pj_post<3><<<g, kT, 0, s>>>(E, P->conn, P->geo, pn, dp, wu, rho, h1, hb, dt, wu_out, h_out, rhok_out);
            else
                k_pj_post<2><<<g, kT, 0, s>>>(E, P->conn, P->geo, pn, dp, wu, rho, h1, hb, dt, wu_out, h_out, rhok_out);
            k_pj_add<<<grid(N, m->ctx->sms), kT, 0, s>>>(N, pn, dp, p_out);
            rc = cuda_rc(cudaGetLastError());
            if (rc != PS_OK) return rc;
        }
    }
    if (rc == PS_OK) {
        // leave the mesh's Jacobi diagonal consistent with its final alpha
        std::lock_guard<std::mutex> lk(m->ctx->mu);
        rc = alpha_update_device(m, static_cast<ProjData *>(m->proj)->au, s, true);
    }
    if (rc == PS_OK) rc = cuda_rc(cudaStreamSynchronize(s));
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = acc;
    if (rc == PS_OK && !converged) return PS_ENOTCONV;
    return rc;
}
