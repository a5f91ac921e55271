// Preconditioned CG in two kernels per iteration (the graph engine of
// ps_pressure_solve).
//
// Iteration k (standard Hestenes-Stiefel PCG, D = Jacobi):
//   K1 (one block per chunk): p = D^-1 r + beta_k p on the chunk's nodes
//      (stored for interior nodes), q = A p (interior rows stored, shared
//      rows as partial sums), and the chunk's share of
//      p.Ap = sum_e p_e^T A_e p_e over ALL its local nodes -- every element
//      lies in exactly one chunk, so these shares add up to p.Ap without a
//      pass over shared nodes.  The last block to finish sums the shares in
//      chunk order and forms alpha_k = rz_k / p.Ap.
//   K2 (fixed grid over nodes): shared nodes form q from their partial sums
//      and p with the same expression as K1; x += alpha p, r -= alpha q; the
//      last block sums the blocks' shares of rz_{k+1} = r.D^-1 r and
//      rr_{k+1} = r.r in block order, tests convergence and forms beta.
// Measured on this part, a grid-wide reduction costs about the same whether
// it is a last-block tail, a separate one-block kernel or a redundant
// reduction in the next kernel's blocks, so each kernel ends in one tail.
// Partial sums are stored as float pairs and reduced with FP32 error-free
// additions; the order is fixed, so results are bitwise reproducible.
#pragma once
#include "ops.cuh"

namespace ps {

template <typename T> struct PartOf;
template <> struct PartOf<float> { using type = float2; };   // double-float partials
template <> struct PartOf<double> { using type = double; };

__device__ __forceinline__ float2 part_pack(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ void part_pack(double v, double &out) { out = v; }
__device__ __forceinline__ void part_pack(double v, float2 &out) { out = part_pack(v); }

// Block-wide fixed-order sum of n partials.
__device__ __forceinline__ double part_sum(const float2 *a, int n, double *red) {
    DotF acc;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 v = __ldcg(a + i);
        acc.merge(v.x, v.y);
    }
    return block_sum(acc, red);
}
__device__ __forceinline__ double part_sum(const double *a, int n, double *red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(a + i);
    return block_sum(s, red);
}
__device__ __forceinline__ void block_sum2(const DotD &a, const DotD &b, double *red, double &ra, double &rb) {
    ra = block_sum(a, red);
    rb = block_sum(b, red);
}
__device__ __forceinline__ void part_sum2(const double *a, const double *b, int n, double *red, double &ra,
                                          double &rb) {
    ra = part_sum(a, n, red);
    rb = part_sum(b, n, red);
}
// Two fixed-order partial sums with one set of barriers (FP32 iteration).
__device__ __forceinline__ void part_sum2(const float2 *a, const float2 *b, int n, double *red, double &ra,
                                          double &rb) {
    DotF acc_a, acc_b;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 va = __ldcg(a + i), vb = __ldcg(b + i);
        acc_a.merge(va.x, va.y);
        acc_b.merge(vb.x, vb.y);
    }
    block_sum2(acc_a, acc_b, red, ra, rb);
}

template <typename T>
struct Cg2Args {
    using PT = typename PartOf<T>::type;
    T *x, *r, *p, *q;
    const T *dinv;
    T *partial;        // [sh_total] shared-node partial sums of q
    PT *pq;            // [n_chunks] chunk shares of p.Ap
    PT *z2;            // [2][g3]: block shares of rz and rr
    int g3;            // grid of K2 (and of the start kernel)
    CgState *st;
    // paired-patch operator kernel only (else null): per chunk-major shared
    // slot, (D^-1 r, p) of the slot's node, gathered after K2 for the next K1
    float2 *halo;
};

// K1: one block per chunk.  PRE: fetch the element phase's beta*dt^2 and the
// first shared nodes' partial-sum destinations into registers before the
// staging wait (FP32; costs registers, so it is used where shared memory, not
// registers, limits the blocks per SM).
template <int D, typename T, bool PRE = false>
__global__ void __launch_bounds__(256) k_cg2_chunks(MeshDev m, Cg2Args<T> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout &L = (sizeof(T) == 4) ? m.sm32 : m.sm64;
    const ChunkSmem<T> S = chunk_smem<T>(smem, L);
    __shared__ double s_beta;
    __shared__ int s_done;
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        s_done = a.st->done;
        s_beta = a.st->beta;
        mbar_init(S.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_done) return;
    const ChunkDesc cd = m.chunks[blockIdx.x];
    stage_issue<T>(m, cd, S);
    const T beta = (T)s_beta;
    const int n_loc = cd.n_loc, n_int = cd.n_int;
    // Every gather runs while the bulk copies are in flight: shared-node ids
    // come from sh_info in global memory (not from the staged copy) and S.val
    // is not a staged region.  No Dirichlet mask is needed: D^-1 = 0 and
    // r = 0 on Dirichlet nodes and p starts at 0, so p stays 0 there.  Loads
    // of four nodes are issued before any store (the stores to p could alias
    // them).
    // The element phase's beta*dt^2 values and the partial-sum destinations
    // of the thread's first shared nodes are fetched here as well.
    BdPrefetch<T> bdp;
    if constexpr (PRE) prefetch_bd<T>(m, cd, bdp);
    int dst[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int l = threadIdx.x + k * blockDim.x;
        dst[k] = (PRE && l >= n_int && l < n_loc) ? m.sh_dest[cd.sh_off + (l - n_int)] : -1;
    }
    for (int l0 = threadIdx.x; l0 < n_loc; l0 += 4 * blockDim.x) {
        int gg[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = l0 + k * blockDim.x;
            gg[k] = l < n_int ? cd.int_begin + l : (l < n_loc ? m.sh_info[cd.sh_off + (l - n_int)].x : -1);
        }
        T dv[4], rv[4], pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dv[k] = rv[k] = pv[k] = T(0);
            if (gg[k] >= 0) {
                dv[k] = a.dinv[gg[k]];
                rv[k] = a.r[gg[k]];
                pv[k] = a.p[gg[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = l0 + k * blockDim.x;
            if (gg[k] >= 0) {
                const T v = cg_dir(dv[k], rv[k], beta, pv[k]);
                S.val[l] = v;
                if (l < n_int) a.p[gg[k]] = v;
            }
        }
    }
    uint32_t ph = 0;
    if (!stage_wait<T>(m, S, ph)) return;   // also the barrier for S.val
    if constexpr (PRE)
        patches_eval_pre<D, T>(m, cd, S, bdp);
    else
        patches_eval<D, T, false>(m, cd, S);
    typename DotOf<T>::type acc;
    auto emit = [&](int l, int d) {
        T s = node_sum(S, l);
        acc.add_prod(S.val[l], s);                 // element-wise p^T A_e p over the chunk
        if (is_dirichlet(S.node[l].w)) s = T(0);
        if (l < n_int)
            a.q[cd.int_begin + l] = s;
        else
            a.partial[d] = s;
    };
    if constexpr (PRE) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = threadIdx.x + k * blockDim.x;
            if (l < n_loc) emit(l, dst[k]);
        }
        for (int l = threadIdx.x + 4 * blockDim.x; l < n_loc; l += blockDim.x)
            emit(l, l < n_int ? -1 : m.sh_dest[cd.sh_off + (l - n_int)]);
    } else {
        for (int l = threadIdx.x; l < n_loc; l += blockDim.x)
            emit(l, l < n_int ? -1 : m.sh_dest[cd.sh_off + (l - n_int)]);
    }
    const double v = block_sum(acc, S.red);
    if (threadIdx.x == 0) {
        part_pack(v, a.pq[blockIdx.x]);
        const unsigned int t = atomic_add_acq_rel(&a.st->cnt_a, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    const double pq = part_sum(a.pq, gridDim.x, S.red);
    if (threadIdx.x == 0) {
        CgState *st = a.st;
        st->cnt_a = 0;
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->status = kCgBreakdown;
            st->done = 1;
        } else {
            st->alpha = st->rz / pq;
        }
    }
}

// Warp-level double-float sum (xor butterfly); every lane gets the result.
__device__ __forceinline__ DotF warp_merge(DotF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, a.hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a.merge(h2, l2);
    }
    return a;
}

// K1, pipelined: a persistent CTA walks chunks blockIdx.x, +gridDim.x, ...
// with two shared-memory stages for the static chunk data: while chunk i is
// computed from one stage, the bulk copies of chunk i+1 fill the other.  The
// per-chunk p.Ap shares are reduced per warp and combined by thread 0 after
// the next block barrier (no extra barriers); they are indexed by chunk, so
// the result does not depend on the grid.  FP32 only.
template <int D>
__global__ void __launch_bounds__(256) k_cg2_chunks_pipe(MeshDev m, Cg2Args<float> a, SmemLayout L0, SmemLayout L1) {
    extern __shared__ __align__(128) unsigned char smem[];
    const ChunkSmem<float> S0 = chunk_smem<float>(smem, L0);
    const ChunkSmem<float> S1 = chunk_smem<float>(smem, L1);
    __shared__ float2 s_wred[8];
    __shared__ float s_beta;
    __shared__ int s_done;
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        s_done = a.st->done;
        s_beta = (float)a.st->beta;
        mbar_init(S0.bar, 1);
        mbar_init(S1.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_done) return;
    const float beta = s_beta;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t ph0 = 0, ph1 = 0;
    int c = blockIdx.x;
    if (c < m.n_chunks) stage_issue<float>(m, m.chunks[c], S0);
    int prev_c = -1;
    for (int it = 0; c < m.n_chunks; ++it, c += gridDim.x) {
        const ChunkSmem<float> &S = (it & 1) ? S1 : S0;
        const ChunkDesc cd = m.chunks[c];
        const int cn = c + gridDim.x;
        if (cn < m.n_chunks) stage_issue<float>(m, m.chunks[cn], (it & 1) ? S0 : S1);
        const int n_loc = cd.n_loc, n_int = cd.n_int;
        float vin[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = threadIdx.x + k * blockDim.x;
            vin[k] = 0.f;
            if (l < n_int) {
                const int g = cd.int_begin + l;
                vin[k] = cg_dir(a.dinv[g], a.r[g], beta, a.p[g]);
            }
        }
        // finish the previous chunk's share (its warp sums are in s_wred)
        if (threadIdx.x == 0 && prev_c >= 0) {
            DotF t;
            for (int w = 0; w < nw; ++w) t.merge(s_wred[w].x, s_wred[w].y);
            a.pq[prev_c] = part_pack((double)t.hi + (double)t.lo);
        }
        const bool ok = stage_wait<float>(m, S, (it & 1) ? ph1 : ph0);
        if (!ok) {
            // let the prefetch into the other stage land before leaving
            if (cn < m.n_chunks) stage_wait<float>(m, (it & 1) ? S0 : S1, (it & 1) ? ph0 : ph1);
            return;
        }
        auto finish = [&](int l, float v) {
            if (is_dirichlet(S.node[l].w)) v = 0.f;
            if (l < n_int) a.p[cd.int_begin + l] = v;
            S.val[l] = v;
        };
        auto fetch = [&](int l) -> float {
            const int g = l < n_int ? cd.int_begin + l : S.shid[l - n_int];
            return cg_dir(a.dinv[g], a.r[g], beta, a.p[g]);
        };
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = threadIdx.x + k * blockDim.x;
            if (l < n_loc) finish(l, l < n_int ? vin[k] : fetch(l));
        }
        for (int l = threadIdx.x + 4 * blockDim.x; l < n_loc; l += blockDim.x) finish(l, fetch(l));
        __syncthreads();
        patches_eval<D, float, false>(m, cd, S);
        DotF acc;
        for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
            float sv = node_sum(S, l);
            acc.add_prod(S.val[l], sv);
            if (is_dirichlet(S.node[l].w)) sv = 0.f;
            if (l < n_int)
                a.q[cd.int_begin + l] = sv;
            else
                a.partial[m.sh_dest[cd.sh_off + (l - n_int)]] = sv;
        }
        acc = warp_merge(acc);
        if (lane == 0) s_wred[wid] = make_float2(acc.hi, acc.lo);
        prev_c = c;
        __syncthreads();   // stage, val, contrib and s_wred released / published
    }
    if (threadIdx.x == 0 && prev_c >= 0) {
        DotF t;
        for (int w = 0; w < nw; ++w) t.merge(s_wred[w].x, s_wred[w].y);
        a.pq[prev_c] = part_pack((double)t.hi + (double)t.lo);
        const unsigned int t2 = atomic_add_acq_rel(&a.st->cnt_a, 1u);
        s_last = (t2 == gridDim.x - 1);
    } else if (threadIdx.x == 0) {
        const unsigned int t2 = atomic_add_acq_rel(&a.st->cnt_a, 1u);
        s_last = (t2 == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    const double pq = part_sum(a.pq, m.n_chunks, S0.red);
    if (threadIdx.x == 0) {
        CgState *st = a.st;
        st->cnt_a = 0;
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->status = kCgBreakdown;
            st->done = 1;
        } else {
            st->alpha = st->rz / pq;
        }
    }
}

// K2: fixed grid over the padded node range [0, n_pad).  Interior nodes in
// groups of 4 (16-byte vectors in FP32), then the rest (interior tail,
// shared nodes) one node per thread, so the dependent partial-sum gathers of
// shared nodes are spread over all threads.  Each thread loads its first
// group and its first remaining node (partial sums included) before the CG
// scalars arrive: none of those loads depends on them, so their latency
// overlaps the scalar read.
template <typename T>
struct K2Node {
    T d, r, p, q;
    bool dir;
};
template <typename T>
__device__ __forceinline__ K2Node<T> k2_load(const MeshDev &m, const Cg2Args<T> &a, int64_t i) {
    K2Node<T> v;
    v.d = a.dinv[i];
    v.r = a.r[i];
    v.p = a.p[i];
    v.dir = false;
    if (i < m.n_int) {
        v.q = a.q[i];
    } else {
        const int64_t s = i - m.n_int;
        T sum = T(0);
        for (int k = m.shr_ptr[s]; k < m.shr_ptr[s + 1]; ++k) sum += a.partial[k];
        v.q = sum;
        v.dir = m.dirichlet[i] != 0;
    }
    return v;
}

// FP32 path of K2: interior nodes in groups of four (16-byte vectors), two
// groups per thread in flight; then the shared nodes (and the interior tail),
// four per thread in flight: their partial-sum ranges are read first, then
// the partials of all four nodes slot by slot, so the dependent loads of
// different nodes overlap.  Each shared node sums its partials in slot order
// (the same sums as the one-node-at-a-time form).
template <typename Acc>
__device__ __forceinline__ void k2_f32(const MeshDev &m, const Cg2Args<float> &a, float alpha, float beta,
                                       int64_t tid, int64_t nthr, Acc &arz, Acc &arr) {
    const int64_t n4 = m.n_int / 4;
    const float4 *X4 = reinterpret_cast<const float4 *>(a.x);
    const float4 *R4 = reinterpret_cast<const float4 *>(a.r);
    const float4 *P4 = reinterpret_cast<const float4 *>(a.p);
    const float4 *Q4 = reinterpret_cast<const float4 *>(a.q);
    const float4 *D4 = reinterpret_cast<const float4 *>(a.dinv);
    constexpr int kG = 2;
    for (int64_t j0 = tid; j0 < n4; j0 += kG * nthr) {
        float4 x4[kG], r4[kG], p4[kG], q4[kG], d4[kG];
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            const int64_t j = j0 + k * nthr;
            if (j < n4) {
                x4[k] = X4[j];
                r4[k] = R4[j];
                p4[k] = P4[j];
                q4[k] = Q4[j];
                d4[k] = __ldg(D4 + j);
            }
        }
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            const int64_t j = j0 + k * nthr;
            if (j >= n4) continue;
            float4 xo, ro;
            xo.x = x4[k].x + alpha * p4[k].x; ro.x = r4[k].x - alpha * q4[k].x;
            xo.y = x4[k].y + alpha * p4[k].y; ro.y = r4[k].y - alpha * q4[k].y;
            xo.z = x4[k].z + alpha * p4[k].z; ro.z = r4[k].z - alpha * q4[k].z;
            xo.w = x4[k].w + alpha * p4[k].w; ro.w = r4[k].w - alpha * q4[k].w;
            reinterpret_cast<float4 *>(a.x)[j] = xo;
            reinterpret_cast<float4 *>(a.r)[j] = ro;
            arz.add_prod(ro.x, d4[k].x * ro.x); arr.add_prod(ro.x, ro.x);
            arz.add_prod(ro.y, d4[k].y * ro.y); arr.add_prod(ro.y, ro.y);
            arz.add_prod(ro.z, d4[k].z * ro.z); arr.add_prod(ro.z, ro.z);
            arz.add_prod(ro.w, d4[k].w * ro.w); arr.add_prod(ro.w, ro.w);
        }
    }
    constexpr int kS = 4;
    for (int64_t i0 = 4 * n4 + tid; i0 < m.n_nodes; i0 += kS * nthr) {
        int64_t ii[kS];
        int kb[kS], ke[kS];
        float dv[kS], rv[kS], pv[kS], qv[kS];
        bool dir[kS];
        int deg = 0;
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            ii[k] = i0 + k * nthr;
            kb[k] = ke[k] = 0;
            qv[k] = 0.f;
            dir[k] = false;
            if (ii[k] < m.n_nodes) {
                dv[k] = __ldg(a.dinv + ii[k]);
                rv[k] = a.r[ii[k]];
                pv[k] = a.p[ii[k]];
                if (ii[k] < m.n_int) {
                    qv[k] = a.q[ii[k]];
                } else {
                    const int64_t sh = ii[k] - m.n_int;
                    kb[k] = __ldg(m.shr_ptr + sh);
                    ke[k] = __ldg(m.shr_ptr + sh + 1);
                    dir[k] = __ldg(m.dirichlet + ii[k]) != 0;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kS; ++k) deg = max(deg, ke[k] - kb[k]);
        for (int t = 0; t < deg; ++t) {
            float pt[kS];
#pragma unroll
            for (int k = 0; k < kS; ++k) pt[k] = kb[k] + t < ke[k] ? __ldcg(a.partial + kb[k] + t) : 0.f;
#pragma unroll
            for (int k = 0; k < kS; ++k)
                if (kb[k] + t < ke[k]) qv[k] += pt[k];
        }
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            const int64_t i = ii[k];
            if (i >= m.n_nodes) continue;
            float pi = pv[k], qi = qv[k];
            if (i >= m.n_int) {
                pi = cg_dir(dv[k], rv[k], beta, pv[k]);
                if (dir[k]) {
                    pi = 0.f;
                    qi = 0.f;
                }
                a.p[i] = pi;   // (a shared row's q is not stored: nothing reads it after this kernel)
            }
            a.x[i] += alpha * pi;
            const float ri = rv[k] - alpha * qi;
            a.r[i] = ri;
            arz.add_prod(ri, dv[k] * ri);
            arr.add_prod(ri, ri);
        }
    }
}

// End of a CG iteration (one thread): rz, rr of the updated residual, the
// iteration count, the stop tests and beta.
__device__ __forceinline__ void cg2_update_tail(CgState *st, double rz, double rr) {
    st->cnt_b = 0;
    st->iters += 1;
    st->rr = rr;
    int done = 0;
    if (!isfinite(rz) || !isfinite(rr)) {
        st->status = kCgBreakdown;
        done = 1;
    } else if (rr <= st->stop_rr) {
        st->status = kCgConverged;
        done = 1;
    } else if (st->iters >= st->max_iters) {
        st->status = kCgMaxIter;
        done = 1;
    } else {
        st->beta = rz / st->rz;
        st->rz = rz;
    }
    if (done) st->done = 1;
}

// K2.  With the paired-patch operator kernel (a.halo set) the blocks only
// store their shares of rz and rr: the halo gather that follows in the same
// iteration sums them in its first block (k_halo_gather), concurrently with
// its gather, so no block of K2 waits for the others.
template <typename T>
__global__ void __launch_bounds__(256) k_cg2_update(MeshDev m, Cg2Args<T> a) {
    __shared__ double red[34];
    __shared__ double s_sc[2];
    __shared__ int s_done;
    __shared__ bool s_last;
    if constexpr (sizeof(T) == 4) {
        if (threadIdx.x == 0) {
            s_done = a.st->done;
            s_sc[0] = a.st->alpha;
            s_sc[1] = a.st->beta;
        }
        __syncthreads();
        if (s_done) return;
        DotF arz, arr;
        k2_f32(m, a, (float)s_sc[0], (float)s_sc[1], (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x, arz, arr);
        double vrz, vrr;
        block_sum2(arz, arr, red, vrz, vrr);
        const bool deferred = a.halo != nullptr;
        if (threadIdx.x == 0) {
            part_pack(vrz, a.z2[blockIdx.x]);
            part_pack(vrr, a.z2[a.g3 + blockIdx.x]);
            if (!deferred) {
                const unsigned int t = atomic_add_acq_rel(&a.st->cnt_b, 1u);
                s_last = (t == gridDim.x - 1);
            }
        }
        if (deferred) return;
        __syncthreads();
        if (!s_last) return;
        double rz, rr;
        part_sum2(a.z2, a.z2 + a.g3, gridDim.x, red, rz, rr);
        if (threadIdx.x == 0) cg2_update_tail(a.st, rz, rr);
        return;
    }
    const int64_t n4 = m.n_int / 4;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float4 x4f, r4f, p4f, q4f, d4f;
    const bool grp0 = sizeof(T) == 4 && tid < n4;
    if (grp0) {
        x4f = reinterpret_cast<const float4 *>(a.x)[tid];
        r4f = reinterpret_cast<const float4 *>(a.r)[tid];
        p4f = reinterpret_cast<const float4 *>(a.p)[tid];
        q4f = reinterpret_cast<const float4 *>(a.q)[tid];
        d4f = reinterpret_cast<const float4 *>(a.dinv)[tid];
    }
    const int64_t i1 = 4 * n4 + tid;
    K2Node<T> nd1;
    if (i1 < m.n_nodes) nd1 = k2_load(m, a, i1);
    if (threadIdx.x == 0) {
        s_done = a.st->done;
        s_sc[0] = a.st->alpha;
        s_sc[1] = a.st->beta;
    }
    __syncthreads();
    if (s_done) return;
    const T alpha = (T)s_sc[0];
    const T beta = (T)s_sc[1];
    typename DotOf<T>::type arz, arr;
    auto finish = [&](int64_t i, const K2Node<T> &v) {
        T pi = v.p, qi = v.q;
        if (i >= m.n_int) {
            pi = cg_dir(v.d, v.r, beta, v.p);
            if (v.dir) {
                pi = T(0);
                qi = T(0);
            }
            a.p[i] = pi;
            a.q[i] = qi;
        }
        a.x[i] += alpha * pi;
        const T ri = v.r - alpha * qi;
        a.r[i] = ri;
        arz.add_prod(ri, v.d * ri);
        arr.add_prod(ri, ri);
    };
    auto group = [&](int64_t j, const float4 &x4, const float4 &r4, const float4 &p4, const float4 &q4,
                     const float4 &d4) {
        const float al = (float)alpha;
        float4 xo, ro;
        xo.x = x4.x + al * p4.x; ro.x = r4.x - al * q4.x;
        xo.y = x4.y + al * p4.y; ro.y = r4.y - al * q4.y;
        xo.z = x4.z + al * p4.z; ro.z = r4.z - al * q4.z;
        xo.w = x4.w + al * p4.w; ro.w = r4.w - al * q4.w;
        reinterpret_cast<float4 *>(a.x)[j] = xo;
        reinterpret_cast<float4 *>(a.r)[j] = ro;
        arz.add_prod(ro.x, d4.x * ro.x); arr.add_prod(ro.x, ro.x);
        arz.add_prod(ro.y, d4.y * ro.y); arr.add_prod(ro.y, ro.y);
        arz.add_prod(ro.z, d4.z * ro.z); arr.add_prod(ro.z, ro.z);
        arz.add_prod(ro.w, d4.w * ro.w); arr.add_prod(ro.w, ro.w);
    };
    if (sizeof(T) == 4) {
        if (grp0) group(tid, x4f, r4f, p4f, q4f, d4f);
        for (int64_t j = tid + nthr; j < n4; j += nthr) {
            const float4 x4 = reinterpret_cast<const float4 *>(a.x)[j];
            const float4 r4 = reinterpret_cast<const float4 *>(a.r)[j];
            const float4 p4 = reinterpret_cast<const float4 *>(a.p)[j];
            const float4 q4 = reinterpret_cast<const float4 *>(a.q)[j];
            const float4 d4 = reinterpret_cast<const float4 *>(a.dinv)[j];
            group(j, x4, r4, p4, q4, d4);
        }
    } else {
        for (int64_t j = tid; j < n4; j += nthr)
            for (int t = 0; t < 4; ++t) finish(4 * j + t, k2_load(m, a, 4 * j + t));
    }
    if (i1 < m.n_nodes) finish(i1, nd1);
    for (int64_t i = i1 + nthr; i < m.n_nodes; i += nthr) finish(i, k2_load(m, a, i));
    double vrz, vrr;
    block_sum2(arz, arr, red, vrz, vrr);
    if (threadIdx.x == 0) {
        part_pack(vrz, a.z2[blockIdx.x]);
        part_pack(vrr, a.z2[a.g3 + blockIdx.x]);
        const unsigned int t = atomic_add_acq_rel(&a.st->cnt_b, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    double rz, rr;
    part_sum2(a.z2, a.z2 + a.g3, gridDim.x, red, rz, rr);
    if (threadIdx.x == 0) cg2_update_tail(a.st, rz, rr);
}

// Start of a CG run from the residual in r (FP64 mode) or from r64 * scale
// (mixed mode): the inner correction d = 0 when given, p = 0, beta = 0; the
// last block forms rz0, rr0 and the stop test: tol2 (absolute) or tol2 * rr0
// (relative).
template <typename T>
__global__ void __launch_bounds__(256) k_cg2_start(MeshDev m, Cg2Args<T> a, const double *__restrict__ rsrc,
                                                   double scale, T *d, double tol2, int relative,
                                                   long long max_iters) {
    __shared__ double red[34];
    __shared__ bool s_last;
    typename DotOf<T>::type arz, arr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m.n_pad; i += (int64_t)gridDim.x * blockDim.x) {
        T ri = rsrc ? (T)(rsrc[i] * scale) : a.r[i];
        if (rsrc) a.r[i] = ri;
        if (d) d[i] = T(0);
        a.p[i] = T(0);
        arz.add_prod(ri, a.dinv[i] * ri);
        arr.add_prod(ri, ri);
    }
    double vrz, vrr;
    block_sum2(arz, arr, red, vrz, vrr);
    if (threadIdx.x == 0) {
        part_pack(vrz, a.z2[blockIdx.x]);
        part_pack(vrr, a.z2[a.g3 + blockIdx.x]);
        const unsigned int t = atomic_add_acq_rel(&a.st->cnt_b, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    double rz0, rr0;
    part_sum2(a.z2, a.z2 + a.g3, gridDim.x, red, rz0, rr0);
    if (threadIdx.x == 0) {
        CgState *st = a.st;
        st->cnt_a = 0;
        st->cnt_b = 0;
        st->rz = rz0;
        st->rr0 = rr0;
        st->rr = rr0;
        st->beta = 0.0;
        st->alpha = 0.0;
        st->iters = 0;
        st->max_iters = max_iters;
        st->stop_rr = relative ? tol2 * rr0 : tol2;
        st->status = kCgRunning;
        st->done = 0;
        if (!isfinite(rz0) || !isfinite(rr0)) {
            st->status = kCgBreakdown;
            st->done = 1;
        } else if (rr0 <= st->stop_rr || rr0 == 0.0) {
            st->status = kCgConverged;
            st->done = 1;
        }
    }
}

}  // namespace ps
