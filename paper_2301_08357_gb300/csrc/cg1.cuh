// Preconditioned CG in one fused pass per iteration (FP32 inner solves of the
// mixed-precision solver; both the single-mesh graph engine and the batched
// persistent engine run it).
//
// The recurrences are the one-reduction form of Chronopoulos and Gear: with
// D the Jacobi preconditioner, s = A p carried by recurrence and w = A u
// computed,
//   s' = w + beta s,  r' = r - alpha s',  u' = D r',  p' = D r + beta p,
//   x' = x + alpha p',  w' = A u',
//   gamma' = r'.u',  delta' = u'.w',  rho' = r'.r',
//   beta'' = gamma' / gamma,  alpha'' = gamma' / (delta' - beta'' gamma' / alpha),
// which match Hestenes-Stiefel PCG in exact arithmetic.  One pass over the
// chunks does all of it:
//   * every chunk updates all its local nodes from the previous iteration's
//     values (vectors are double-buffered by iteration parity, so no chunk
//     reads a value another chunk has already overwritten); the values of a
//     shared node are written by its owner chunk only; a shared node's w is
//     never stored -- every chunk sums its partial sums from the previous pass;
//   * w' = A u' from the chunk's elements: interior rows stored, shared rows as
//     partial sums;
//   * delta' = sum_e u'_e^T A_e u'_e over the chunk's elements (every element
//     lies in one chunk), gamma' and rho' over the nodes the chunk owns;
//   * the last block to finish sums the per-chunk triples in chunk order and
//     forms the next alpha, beta (or stops).
// The first pass of a run uses alpha = beta = 0 with p = s = w = 0, which
// yields u_0, p_0 = u_0 and w_0 = A u_0.
#pragma once
#include "ops.cuh"

namespace ps {

struct NodeUpd {
    float s, r, u, p, x;
};
// Explicit roundings: the same inputs give bitwise the same outputs wherever
// this is evaluated (every chunk holding a shared node evaluates it).
__device__ __forceinline__ NodeUpd node_update(float r, float w, float s, float di, float p, float x, float alpha,
                                               float beta) {
    NodeUpd o;
    o.s = __fmaf_rn(beta, s, w);
    o.r = __fmaf_rn(-alpha, o.s, r);
    o.u = __fmul_rn(di, o.r);
    o.p = __fmaf_rn(beta, p, __fmul_rn(di, r));
    o.x = __fmaf_rn(alpha, o.p, x);
    return o;
}

// Double-buffered FP32 vectors of one mesh (internal numbering, n_pad).
struct CG1Vec {
    float *x[2], *r[2], *s[2], *p[2], *w[2];
    float *part[2];        // shared-node-major partial sums of w
    const float *dinv;
    float2 *dots;          // [n_chunks * 3]: gamma, delta, rho shares (float pairs)
};

// The buffers one pass reads (parity par) and writes (par ^ 1), selected
// without indexing the parameter arrays (which would place them in local
// memory).
struct CG1Pass {
    const float *r, *w, *s, *p, *x, *part;
    float *r_o, *w_o, *s_o, *p_o, *x_o, *part_o;
};
__device__ __forceinline__ CG1Pass cg1_pass(const CG1Vec &V, int par) {
    const bool o = par != 0;
    CG1Pass b;
    b.r = o ? V.r[1] : V.r[0];
    b.w = o ? V.w[1] : V.w[0];
    b.s = o ? V.s[1] : V.s[0];
    b.p = o ? V.p[1] : V.p[0];
    b.x = o ? V.x[1] : V.x[0];
    b.part = o ? V.part[1] : V.part[0];
    b.r_o = o ? V.r[0] : V.r[1];
    b.w_o = o ? V.w[0] : V.w[1];
    b.s_o = o ? V.s[0] : V.s[1];
    b.p_o = o ? V.p[0] : V.p[1];
    b.x_o = o ? V.x[0] : V.x[1];
    b.part_o = o ? V.part[0] : V.part[1];
    return b;
}

__device__ __forceinline__ float2 df_pack(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

// The fused pass over chunk c (block-uniform).  B: the buffers of this pass.
// acc: this thread's shares of gamma, delta, rho.
template <int D>
__device__ __forceinline__ void chunk_cg1f(const MeshDev &m, const CG1Pass &B, const float *__restrict__ dinv, int c,
                                           float alpha, float beta, const ChunkSmem<float> &S, uint32_t &phase,
                                           DotF acc[3], bool &failed) {
    const ChunkDesc cd = m.chunks[c];
    const int n_loc = cd.n_loc, n_int = cd.n_int;
    stage_issue<float>(m, cd, S);
    // The node updates need none of the staged data, so they run while the
    // bulk copies are in flight (S.val and S.aux are not staged regions).
    // No Dirichlet mask is needed: D^-1 = 0 there and r starts at 0, so u,
    // r, s, p and x stay 0 on those nodes.
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        NodeUpd o;
        if (l < n_int) {
            const int g = cd.int_begin + l;
            o = node_update(B.r[g], B.w[g], B.s[g], dinv[g], B.p[g], B.x[g], alpha, beta);
            B.s_o[g] = o.s;
            B.r_o[g] = o.r;
            B.p_o[g] = o.p;
            B.x_o[g] = o.x;
        } else {
            // shared node: w is the sum of the previous pass's partials in
            // a fixed order, so every chunk holding the node gets the same
            // values; only the owner stores them
            const int4 si = m.sh_info[cd.sh_off + (l - n_int)];
            const int g = si.x;
            float w = 0.f;
            for (int k = si.y; k < si.z; ++k) w += B.part[k];
            o = node_update(B.r[g], w, B.s[g], dinv[g], B.p[g], B.x[g], alpha, beta);
            if (si.w) {
                B.s_o[g] = o.s;
                B.r_o[g] = o.r;
                B.p_o[g] = o.p;
                B.x_o[g] = o.x;
            }
        }
        S.val[l] = o.u;
        S.aux[l] = o.r;
    }
    if (!stage_wait<float>(m, S, phase)) {    // also the barrier for S.val / S.aux
        failed = true;
        return;
    }
    patches_eval<D, float, false>(m, cd, S);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        float wv = node_sum(S, l);
        const float u = S.val[l], r = S.aux[l];
        if (is_dirichlet(S.node[l].w)) wv = 0.f;
        acc[1].add_prod(u, wv);                   // element-wise u^T A_e u
        if (l < n_int) {
            B.w_o[cd.int_begin + l] = wv;
            acc[0].add_prod(r, u);
            acc[2].add_prod(r, r);
        } else {
            const int j = cd.sh_off + (l - n_int);
            B.part_o[m.sh_dest[j]] = wv;
            if (m.sh_info[j].w) {
                acc[0].add_prod(r, u);
                acc[2].add_prod(r, r);
            }
        }
    }
}

// Parity of the next pass (the buffer it reads); after the run has stopped,
// the buffer holding the final x.  Pass 0 is the start pass; pass k >= 1
// leaves iteration k's vectors in buffer (k + 1) mod 2.
__device__ __forceinline__ int cg1_parity(int first, long long iters) { return first ? 0 : (int)((iters + 1) & 1); }

// Scalar update after a fused pass (one thread).  State fields: rz = gamma,
// pq = delta, rr = rho, rr0 = rho of the start pass, stop_rr = tol2 * rr0.
// Returns 1 if the run stops.
__device__ __forceinline__ int cg1_scalars(CgState *st, double g, double d, double rho) {
    int done = 0, status = kCgRunning;
    if (st->first) {
        st->first = 0;
        st->rr0 = rho;
        st->stop_rr = st->tol2 * rho;
        if (!(rho > 0.0)) {
            done = 1;
            status = kCgConverged;
        } else if (!(d > 0.0) || !isfinite(g) || !isfinite(d)) {
            done = 1;
            status = kCgBreakdown;
        } else {
            st->alpha = g / d;
            st->beta = 0.0;
        }
    } else {
        st->iters += 1;
        const double beta = g / st->rz;
        const double den = d - beta * g / st->alpha;
        if (!isfinite(rho) || !isfinite(g) || !isfinite(d) || !(den > 0.0)) {
            done = 1;
            status = kCgBreakdown;
        } else if (rho <= st->stop_rr) {
            done = 1;
            status = kCgConverged;
        } else if (st->iters >= st->max_iters) {
            done = 1;
            status = kCgMaxIter;
        } else {
            st->beta = beta;
            st->alpha = g / den;
        }
    }
    st->rz = g;
    st->pq = d;
    st->rr = rho;
    if (st->free_run) done = 0;
    if (done) {
        st->status = status;
        st->done = 1;
    }
    return done;
}

// Reduce a mesh's per-chunk triples (fixed chunk order); all threads call,
// results in out[3].
__device__ __forceinline__ void cg1_reduce(const float2 *dots, int n_chunks, double *red, double out[3]) {
    DotF ag, ad, ar;
    for (int k = threadIdx.x; k < n_chunks; k += blockDim.x) {
        const float2 g2 = __ldcg(dots + 3 * k), d2 = __ldcg(dots + 3 * k + 1), r2 = __ldcg(dots + 3 * k + 2);
        ag.merge(g2.x, g2.y);
        ad.merge(d2.x, d2.y);
        ar.merge(r2.x, r2.y);
    }
    const DotF v[3] = {ag, ad, ar};
    block_sum_n<3>(v, red, out);
}

// Graph engine: one block per chunk; the last block advances the scalars.
// The pass parity comes from the state, so any number of launches can be
// captured and replayed.
template <int D>
__global__ void __launch_bounds__(256) k_cg1_chunks(MeshDev m, CG1Vec V, CgState *st) {
    extern __shared__ __align__(128) unsigned char smem[];
    const ChunkSmem<float> S = chunk_smem<float>(smem, m.sm32);
    __shared__ float s_ab[2];
    __shared__ int s_done, s_par;
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        s_done = st->done;
        s_par = cg1_parity(st->first, st->iters);
        s_ab[0] = (float)st->alpha;
        s_ab[1] = (float)st->beta;
        mbar_init(S.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_done) return;
    uint32_t phase = 0;
    bool failed = false;
    DotF acc[3];
    chunk_cg1f<D>(m, cg1_pass(V, s_par), V.dinv, blockIdx.x, s_ab[0], s_ab[1], S, phase, acc, failed);
    if (failed) return;
    double out[3];
    block_sum_n<3>(acc, S.red, out);
    if (threadIdx.x == 0) {
        V.dots[3 * blockIdx.x] = df_pack(out[0]);
        V.dots[3 * blockIdx.x + 1] = df_pack(out[1]);
        V.dots[3 * blockIdx.x + 2] = df_pack(out[2]);
        const unsigned int t = atomic_add_acq_rel(&st->cnt_a, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    double tot[3];
    cg1_reduce(V.dots, m.n_chunks, S.red, tot);
    if (threadIdx.x == 0) {
        st->cnt_a = 0;
        cg1_scalars(st, tot[0], tot[1], tot[2]);
    }
}

// Start of an inner run: buffer 0 holds r = r64 * scale, everything else 0
// (x, p, s, w and the shared-node partials of buffer 0).
static __global__ void __launch_bounds__(256) k_cg1_start(int64_t n_pad, int64_t n_part, CG1Vec V, const double *__restrict__ r64,
                                                   double scale) {
    float *r = V.r[0], *x = V.x[0], *p = V.p[0], *s = V.s[0], *w = V.w[0], *part = V.part[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
        r[i] = (float)(r64[i] * scale);
        x[i] = 0.f;
        p[i] = 0.f;
        s[i] = 0.f;
        w[i] = 0.f;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_part; i += (int64_t)gridDim.x * blockDim.x)
        part[i] = 0.f;
}

static __global__ void k_cg1_init_state(CgState *st, double tol2, long long max_iters) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->rz = st->pq = st->alpha = st->beta = 0.0;
        st->rr = st->rr0 = st->stop_rr = st->bb = 0.0;
        st->tol2 = tol2;
        st->iters = 0;
        st->max_iters = max_iters;
        st->done = 0;
        st->status = kCgRunning;
        st->first = 1;
        st->free_run = 0;
        st->cnt_a = st->cnt_b = 0;
    }
}

// x64 += x32 / scale, x32 the buffer holding the final iterate.
static __global__ void __launch_bounds__(256) k_cg1_correct(int64_t n_pad, double *__restrict__ x64, CG1Vec V,
                                                     const CgState *st, double inv_scale) {
    const float *x32 = cg1_parity(st->first, st->iters) ? V.x[1] : V.x[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x)
        x64[i] += (double)x32[i] * inv_scale;
}

}  // namespace ps
