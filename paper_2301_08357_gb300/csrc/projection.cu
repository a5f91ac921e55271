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
    int *flag = nullptr;          // enthalpy check
    int64_t alpha_version = -1;
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

// First guesses: H_e = g1 mean_k(P_k) / rho_e, (rho K)_e = |W~~_u,e|^2 / (2 rho_e).
template <int D>
__global__ void __launch_bounds__(kT) k_pj_first(int64_t n_el, const int32_t *__restrict__ conn,
                                                 const double *__restrict__ p, const double *__restrict__ rho,
                                                 const double *__restrict__ wu, double g1, double *__restrict__ H,
                                                 double *__restrict__ rhok) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        double pb = 0.0, u2 = 0.0;
        for (int k = 0; k <= D; ++k) pb += p[conn[e * (D + 1) + k]];
        for (int a = 0; a < D; ++a) u2 += wu[e * D + a] * wu[e * D + a];
        H[e] = g1 * (pb / (D + 1)) / rho[e];
        rhok[e] = 0.5 * u2 / rho[e];
    }
}

__global__ void __launch_bounds__(kT) k_pj_check(int64_t n, const double *__restrict__ v, int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(v[i] > 0.0) || !isfinite(v[i])) atomicOr(flag, 1);
}

// Right-hand side of the weak problem at node i, gathered over its elements
// in ascending order:
//   (W~_E - rho K)_e |T| / (d+1)                       source term
// + dt H_e |T| W~~_u,e . grad lambda_k                 divergence term
// - (M^e_alpha P^n)_k = cm (S X + Q + S P_k + alpha_k (X + 2 P_k))
// with k the local index of i in e, S = sum alpha, X = sum P, Q = sum alpha P
// over the element's vertices and cm = |T| d! / (d+3)!.
template <int D>
__global__ void __launch_bounds__(kT) k_pj_rhs(int64_t n_nodes, const int64_t *__restrict__ n2e_ptr,
                                               const int32_t *__restrict__ n2e, const int32_t *__restrict__ conn,
                                               const double *__restrict__ x, const double *__restrict__ alpha,
                                               const uint8_t *__restrict__ dir, const double *__restrict__ H,
                                               const double *__restrict__ rhok, const double *__restrict__ wu,
                                               const double *__restrict__ we, const double *__restrict__ p,
                                               double dt, double *__restrict__ b) {
    constexpr double fact = D == 3 ? 6.0 : 2.0;           // d!
    constexpr double cmden = D == 3 ? 720.0 : 120.0;      // cm = |T| d! / (d+3)! = |det| / (d+3)!
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        if (dir[i]) {
            b[i] = 0.0;
            continue;
        }
        double acc = 0.0;
        for (int64_t t = n2e_ptr[i]; t < n2e_ptr[i + 1]; ++t) {
            const int code = n2e[t];
            const int64_t e = code >> 2;
            const int k = code & 3;
            double v[D + 1][D], c[D + 1][D];
            double al[D + 1], pv[D + 1];
            for (int q = 0; q <= D; ++q) {
                const int64_t g = conn[e * (D + 1) + q];
                for (int a = 0; a < D; ++a) v[q][a] = x[g * D + a];
                al[q] = alpha[g];
                pv[q] = p[g];
            }
            const double det = cofactors<D>(v, c);
            const double adet = fabs(det);
            const double sgn = det > 0.0 ? 1.0 : -1.0;
            const double vol = adet / fact;
            double cw = 0.0;
            for (int a = 0; a < D; ++a) cw += c[k][a] * wu[e * D + a];
            double S = 0.0, X = 0.0, Q = 0.0;
            for (int q = 0; q <= D; ++q) {
                S += al[q];
                X += pv[q];
                Q += al[q] * pv[q];
            }
            const double cm = adet / cmden;
            const double mass = cm * (S * X + Q + S * pv[k] + al[k] * (X + 2.0 * pv[k]));
            acc += (we[e] - rhok[e]) * vol / (D + 1) + dt * H[e] * sgn * cw / fact - mass;
        }
        b[i] = acc;
    }
}

// Post-projection: W_u = W~~_u - dt grad dP_h, P = P^n + dP (vertex mean for
// H), H = g1 mean(P) / rho, rho K = |W_u|^2 / (2 rho).
template <int D>
__global__ void __launch_bounds__(kT) k_pj_post(int64_t n_el, const int32_t *__restrict__ conn,
                                                const double *__restrict__ x, const double *__restrict__ pn,
                                                const double *__restrict__ dp, const double *__restrict__ wu_tt,
                                                const double *__restrict__ rho, double g1, double dt,
                                                double *__restrict__ wu_new, double *__restrict__ H,
                                                double *__restrict__ rhok) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        double v[D + 1][D], c[D + 1][D], d[D + 1];
        double pb = 0.0;
        for (int q = 0; q <= D; ++q) {
            const int64_t g = conn[e * (D + 1) + q];
            for (int a = 0; a < D; ++a) v[q][a] = x[g * D + a];
            d[q] = dp[g];
            pb += pn[g] + dp[g];
        }
        const double det = cofactors<D>(v, c);
        double u2 = 0.0;
        for (int a = 0; a < D; ++a) {
            double gr = 0.0;
            for (int q = 0; q <= D; ++q) gr += c[q][a] * d[q];
            const double u = wu_tt[e * D + a] - dt * (gr / det);
            wu_new[e * D + a] = u;
            u2 += u * u;
        }
        H[e] = g1 * (pb / (D + 1)) / rho[e];
        rhok[e] = 0.5 * u2 / rho[e];
    }
}

__global__ void __launch_bounds__(kT) k_pj_add(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                                               double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a[i] + b[i];
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
        m->proj = P;
    }
    if (P->alpha_version != m->alpha_version) {
        cudaError_t er = cudaMemcpy(P->alpha, m->alpha_host.data(), (size_t)N * 8, cudaMemcpyHostToDevice);
        if (er != cudaSuccess) return cuda_rc(er);
        P->alpha_version = m->alpha_version;
    }
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
    if (!m->coeff_ok || !m->alpha_set) return PS_ESTATE;
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
        if (dim == 3) k_pj_first<3><<<g, kT, 0, s>>>(E, P->conn, pn, rho, wu, g1, h_out, rhok_out);
        else k_pj_first<2><<<g, kT, 0, s>>>(E, P->conn, pn, rho, wu, g1, h_out, rhok_out);
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
            const int g = grid(N, m->ctx->sms);
            if (dim == 3)
                k_pj_rhs<3><<<g, kT, 0, s>>>(N, P->n2e_ptr, P->n2e, P->conn, P->x, P->alpha, P->dir, h_out, rhok_out,
                                             wu, we, pn, dt, P->b);
            else
                k_pj_rhs<2><<<g, kT, 0, s>>>(N, P->n2e_ptr, P->n2e, P->conn, P->x, P->alpha, P->dir, h_out, rhok_out,
                                             wu, we, pn, dt, P->b);
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
                k_pj_post<3><<<g, kT, 0, s>>>(E, P->conn, P->x, pn, dp, wu, rho, g1, dt, wu_out, h_out, rhok_out);
            else
                k_pj_post<2><<<g, kT, 0, s>>>(E, P->conn, P->x, pn, dp, wu, rho, g1, dt, wu_out, h_out, rhok_out);
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
