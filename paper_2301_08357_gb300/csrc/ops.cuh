// Chunked matrix-free P1 operator and the fused CG kernels.
//
// One thread block processes one chunk (layout.h):
//   1. one elected thread moves the chunk's static data (node records,
//      local connectivity, beta*dt^2, incidence lists, shared-node ids) into
//      shared memory with bulk copies signalled on an mbarrier;
//   2. the block gathers the input vector for its local nodes (contiguous for
//      interior nodes, through the shared-node ids otherwise), masking
//      Dirichlet nodes; in CG mode it forms the new search direction
//      p = D^-1 r + beta p on the fly and stores it for its interior nodes;
//   3. one thread per element computes the element's (d+1) contributions into
//      shared memory;
//   4. one thread per local node sums its contributions in incidence-list
//      order and writes its row (interior node) or a partial sum (shared node).
// A second kernel adds the partial sums of shared nodes in a fixed order.
// Dot products are accumulated in FP64 per block and reduced by the last
// block to finish, in a fixed order, so every result is bitwise reproducible.
#pragma once
#include "device.cuh"

namespace ps {

enum Mode : int { kApply = 0, kCG = 1, kResid = 2, kDiag = 3 };

struct SmemLayout {
    uint32_t node, val, aux, pids, incp, inc, shid, contrib, red, bar, total;
};

// Shared memory of the paired-patch CG operator kernel (cg2u.cuh): node
// records | values | fixed-point node sums | partial-sum destinations of the
// shared nodes | per-thread dot partials | mbarrier.
struct UnitSmem {
    uint32_t node, val, acc, shd, urec, ubd, bar, total;
};

struct MeshDev {
    int dim, n_chunks;
    int64_t n_nodes, n_int, n_shared, n_pad;
    const ChunkDesc *chunks;
    const uint16_t *pids;    // [patch_total * kPatchIds]
    const uint16_t *incp, *inc;
    const int32_t *sh_ids, *shr_ptr, *sh_dest;
    const int4 *sh_info;     // [sh_total] node id, partial range [begin, end), owner flag
    const NodeF *node32;
    const NodeD *node64;
    const float *bdt2_32;
    const double *bdt2_64;
    const double *geo64;     // [patch_total * kPatchMax * kGeoWords<dim>] FP64 element geometry
    const float *dinv32;
    const double *dinv64;
    const uint8_t *dirichlet;
    int *err;
    int lumped;              // 1: mass term by vertex quadrature (mass-lumped variant)
    SmemLayout sm32, sm64;
    // paired-patch layout (3D; null in 2D)
    const ChunkUnits *chunks_u;
    const uint32_t *urec;    // [unit_total * kURecWords]
    const float *ubd;        // [unit_total * kPatchMax * 2] beta*dt^2/6 per (unit, element, half)
    const float *dmax;       // [n_chunks] largest diagonal entry over each chunk's free nodes
    UnitSmem smu;
};

// Scalars of one CG run, kept on the device.
struct CgState {
    double rz, pq, alpha, beta, rr, rr0, stop_rr, bb;
    long long iters, max_iters;
    int done, status;
    unsigned int cnt_a, cnt_b;
    int first, free_run;     // fused engine: first = the start pass is next;
                             // free_run = never stop (kernel timing only)
    double tol2;             // fused engine: relative stopping tolerance squared
};

enum CgStatus : int { kCgRunning = 0, kCgConverged = 1, kCgMaxIter = 2, kCgBreakdown = 3 };

template <typename T>
struct VecArgs {
    const T *x;      // apply / resid: input vector
    T *y;            // apply: output; cg: q; resid: r
    const T *b;      // resid: right-hand side (0 on Dirichlet nodes)
    T *p;            // cg: search direction (read old, write new)
    const T *r;      // cg: residual
    const T *dinv;   // cg: Jacobi inverse diagonal (0 on Dirichlet nodes)
    T *partial;      // [sh_total] partial sums of shared local nodes
    double *dotbuf;  // per-block dot partials
    CgState *st;
    int *host_done;  // optional host-mapped copy of st->done
};

__device__ __forceinline__ float cg_dir(float dinv, float r, float beta, float p) {
    return __fmaf_rn(beta, p, __fmul_rn(dinv, r));
}
__device__ __forceinline__ double cg_dir(double dinv, double r, double beta, double p) {
    return __fma_rn(beta, p, __dmul_rn(dinv, r));
}

__device__ __forceinline__ int ld_flag(const int *p) { return *(volatile const int *)p; }

// Shared-memory view of one staged chunk.
template <typename T>
struct ChunkSmem {
    typename NodeOf<T>::type *node;
    T *val, *aux, *contrib;
    uint16_t *pids, *incp, *inc;
    int32_t *shid;
    uint64_t *bar;
    double *red;
};

template <typename T>
__device__ __forceinline__ ChunkSmem<T> chunk_smem(unsigned char *smem, const SmemLayout &L) {
    ChunkSmem<T> S;
    S.node = reinterpret_cast<typename NodeOf<T>::type *>(smem + L.node);
    S.val = reinterpret_cast<T *>(smem + L.val);
    S.aux = reinterpret_cast<T *>(smem + L.aux);
    S.contrib = reinterpret_cast<T *>(smem + L.contrib);
    S.pids = reinterpret_cast<uint16_t *>(smem + L.pids);
    S.incp = reinterpret_cast<uint16_t *>(smem + L.incp);
    S.inc = reinterpret_cast<uint16_t *>(smem + L.inc);
    S.shid = reinterpret_cast<int32_t *>(smem + L.shid);
    S.bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    S.red = reinterpret_cast<double *>(smem + L.red);
    return S;
}

// Thread 0 issues the bulk copies of chunk cd's static data (node records,
// patch records, incidence pointers and lists, shared-node ids).  When the
// shared memory was used by an earlier chunk, the caller has synchronised the
// block; the proxy fence orders those generic-proxy reads before the
// async-proxy writes.
template <typename T>
__device__ __forceinline__ void stage_issue(const MeshDev &m, const ChunkDesc &cd, const ChunkSmem<T> &S) {
    using N4 = typename NodeOf<T>::type;
    if (threadIdx.x != 0) return;
    const int p_pad = (cd.n_patch + kPatchPad - 1) / kPatchPad * kPatchPad;
    const int incp_n = (cd.n_loc + 1 + kIncpPad - 1) / kIncpPad * kIncpPad;
    const int inc_n = (cd.n_inc + kIncPad - 1) / kIncPad * kIncPad;
    const int sh_n = (cd.n_sh + kShPad - 1) / kShPad * kShPad;
    const N4 *gnode = (sizeof(T) == 4) ? reinterpret_cast<const N4 *>(m.node32) : reinterpret_cast<const N4 *>(m.node64);
    const uint32_t b_node = (uint32_t)cd.n_loc * sizeof(N4);
    const uint32_t b_pids = (uint32_t)p_pad * (kPatchIds * 2u);
    const uint32_t b_incp = (uint32_t)incp_n * 2u;
    const uint32_t b_inc = (uint32_t)inc_n * 2u;
    const uint32_t b_sh = (uint32_t)sh_n * 4u;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(S.bar, b_node + b_pids + b_incp + b_inc + b_sh);
    bulk_g2s(S.node, gnode + cd.node_off, b_node, S.bar);
    bulk_g2s(S.pids, m.pids + (size_t)cd.patch_off * kPatchIds, b_pids, S.bar);
    bulk_g2s(S.incp, m.incp + cd.incp_off, b_incp, S.bar);
    bulk_g2s(S.inc, m.inc + cd.inc_off, b_inc, S.bar);
    if (b_sh) bulk_g2s(S.shid, m.sh_ids + cd.sh_off, b_sh, S.bar);
}

// Wait for the staged data (bounded); block-uniform result.  On timeout the
// error flag is set and the copies in flight are waited for once more.
template <typename T>
__device__ __forceinline__ bool stage_wait(const MeshDev &m, const ChunkSmem<T> &S, uint32_t &phase) {
    bool ok = mbar_wait_bounded(S.bar, phase);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(m.err, kErrMbarTimeout);
        mbar_wait_bounded(S.bar, phase);
    }
    phase ^= 1u;
    return ok;
}

// Element contributions of every star patch of the chunk into S.contrib
// (the mesh's mass form chosen once per chunk, so each variant of the loop
// is compiled on its own).
template <int D, typename T, bool DIAG>
__device__ __forceinline__ void patches_eval(const MeshDev &m, const ChunkDesc &cd, const ChunkSmem<T> &S) {
    using N4 = typename NodeOf<T>::type;
    const T *gbdt2 = (sizeof(T) == 4) ? reinterpret_cast<const T *>(m.bdt2_32) : reinterpret_cast<const T *>(m.bdt2_64);
    const T *g_bdt2 = gbdt2 + (size_t)cd.patch_off * kPatchMax;
    if constexpr (sizeof(T) == 8) {
        // FP64: element geometry precomputed per slot (patch_eval_geo)
        constexpr int GW = kGeoWords<D>;
        const double *g_geo = m.geo64 + (size_t)cd.patch_off * kPatchMax * GW;
        if (m.lumped) {
            for (int q = threadIdx.x; q < cd.n_patch; q += blockDim.x) {
                double bd[kPatchMax];
                load_bd(g_bdt2 + q * kPatchMax, bd);
                patch_eval_geo<D, DIAG, true>(S.node, S.val, S.pids + q * kPatchIds, bd, g_geo + q * kPatchMax * GW,
                                              S.contrib + q * kPatchSlots);
            }
        } else {
            for (int q = threadIdx.x; q < cd.n_patch; q += blockDim.x) {
                double bd[kPatchMax];
                load_bd(g_bdt2 + q * kPatchMax, bd);
                patch_eval_geo<D, DIAG, false>(S.node, S.val, S.pids + q * kPatchIds, bd, g_geo + q * kPatchMax * GW,
                                               S.contrib + q * kPatchSlots);
            }
        }
    } else if (m.lumped) {
        for (int q = threadIdx.x; q < cd.n_patch; q += blockDim.x) {
            T bd[kPatchMax];
            load_bd(g_bdt2 + q * kPatchMax, bd);
            patch_eval<D, T, N4, DIAG, true>(S.node, S.val, S.pids + q * kPatchIds, bd, S.contrib + q * kPatchSlots);
        }
    } else {
        for (int q = threadIdx.x; q < cd.n_patch; q += blockDim.x) {
            T bd[kPatchMax];
            load_bd(g_bdt2 + q * kPatchMax, bd);
            patch_eval<D, T, N4, DIAG>(S.node, S.val, S.pids + q * kPatchIds, bd, S.contrib + q * kPatchSlots);
        }
    }
    __syncthreads();
}

// The same with beta*dt^2 of the thread's first R patches loaded earlier
// (prefetch_bd, before the staging wait): the element phase then starts
// without a global-memory round trip.
constexpr int kBdRounds = 3;
template <typename T>
struct BdPrefetch {
    T v[kBdRounds][kPatchMax];
};
template <typename T>
__device__ __forceinline__ void prefetch_bd(const MeshDev &m, const ChunkDesc &cd, BdPrefetch<T> &P) {
    const T *gbdt2 = (sizeof(T) == 4) ? reinterpret_cast<const T *>(m.bdt2_32) : reinterpret_cast<const T *>(m.bdt2_64);
    const T *g_bdt2 = gbdt2 + (size_t)cd.patch_off * kPatchMax;
#pragma unroll
    for (int k = 0; k < kBdRounds; ++k) {
        const int q = threadIdx.x + k * blockDim.x;
        if (q < cd.n_patch) load_bd(g_bdt2 + q * kPatchMax, P.v[k]);
    }
}
template <int D, typename T, bool LUMP>
__device__ __forceinline__ void patches_eval_pre_v(const MeshDev &m, const ChunkDesc &cd, const ChunkSmem<T> &S,
                                                   const BdPrefetch<T> &P) {
    using N4 = typename NodeOf<T>::type;
#pragma unroll
    for (int k = 0; k < kBdRounds; ++k) {
        const int q = threadIdx.x + k * blockDim.x;
        if (q < cd.n_patch)
            patch_eval<D, T, N4, false, LUMP>(S.node, S.val, S.pids + q * kPatchIds, P.v[k],
                                              S.contrib + q * kPatchSlots);
    }
    const T *gbdt2 = (sizeof(T) == 4) ? reinterpret_cast<const T *>(m.bdt2_32) : reinterpret_cast<const T *>(m.bdt2_64);
    const T *g_bdt2 = gbdt2 + (size_t)cd.patch_off * kPatchMax;
    for (int q = threadIdx.x + kBdRounds * blockDim.x; q < cd.n_patch; q += blockDim.x) {
        T bd[kPatchMax];
        load_bd(g_bdt2 + q * kPatchMax, bd);
        patch_eval<D, T, N4, false, LUMP>(S.node, S.val, S.pids + q * kPatchIds, bd, S.contrib + q * kPatchSlots);
    }
}
template <int D, typename T>
__device__ __forceinline__ void patches_eval_pre(const MeshDev &m, const ChunkDesc &cd, const ChunkSmem<T> &S,
                                                 const BdPrefetch<T> &P) {
    if (m.lumped)
        patches_eval_pre_v<D, T, true>(m, cd, S, P);
    else
        patches_eval_pre_v<D, T, false>(m, cd, S, P);
    __syncthreads();
}

// Sum of the contributions of local node l in incidence order.
template <typename T>
__device__ __forceinline__ T node_sum(const ChunkSmem<T> &S, int l) {
    const int b = S.incp[l], e = S.incp[l + 1];
    // four independent partial sums (fixed pattern: deterministic)
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    int k = b;
    for (; k + 3 < e; k += 4) {
        s0 += S.contrib[S.inc[k]];
        s1 += S.contrib[S.inc[k + 1]];
        s2 += S.contrib[S.inc[k + 2]];
        s3 += S.contrib[S.inc[k + 3]];
    }
    for (; k < e; ++k) s0 += S.contrib[S.inc[k]];
    return (s0 + s1) + (s2 + s3);
}

// Process chunk c.  Returns this thread's share of the mode's dot product
// (CG: p.q, resid: r.r over interior nodes).  `phase` is the mbarrier parity
// to wait for; it flips on return.  Block-uniform; contains __syncthreads.
template <int D, typename T, int MODE>
__device__ typename DotOf<T>::type process_chunk(const MeshDev &m, const VecArgs<T> &a, int c, unsigned char *smem,
                                                 const SmemLayout &L, uint32_t &phase, T beta_cg, bool &failed) {
    using Acc = typename DotOf<T>::type;
    const ChunkDesc cd = m.chunks[c];
    const ChunkSmem<T> S = chunk_smem<T>(smem, L);
    const int n_loc = cd.n_loc, n_int = cd.n_int;
    stage_issue<T>(m, cd, S);
    // interior input values do not depend on the staged data: fetch them
    // while the bulk copies are in flight (masked below, once records landed)
    T vin[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int l = threadIdx.x + k * blockDim.x;
        vin[k] = T(0);
        if (MODE != kDiag && l < n_int) {
            const int g = cd.int_begin + l;
            vin[k] = (MODE == kCG) ? cg_dir(a.dinv[g], a.r[g], beta_cg, a.p[g]) : a.x[g];
        }
    }
    if (!stage_wait<T>(m, S, phase)) {
        failed = true;
        return Acc();
    }

    // ---- gather the input vector (masked on Dirichlet nodes).  Apply and
    // residual skip the element phase of a chunk whose input is zero on all
    // its nodes (a zero first guess, a zero correction): every contribution
    // is then exactly 0.
    bool nonzero = false;
    if (MODE != kDiag) {
        auto finish = [&](int l, T v) {
            if (is_dirichlet(S.node[l].w)) v = T(0);
            if (MODE == kCG && l < n_int) a.p[cd.int_begin + l] = v;
            S.val[l] = v;
            nonzero |= v != T(0);
        };
        auto fetch = [&](int l) -> T {
            const int g = l < n_int ? cd.int_begin + l : S.shid[l - n_int];
            return (MODE == kCG) ? cg_dir(a.dinv[g], a.r[g], beta_cg, a.p[g]) : a.x[g];
        };
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = threadIdx.x + k * blockDim.x;
            if (l < n_loc) finish(l, l < n_int ? vin[k] : fetch(l));
        }
        for (int l = threadIdx.x + 4 * blockDim.x; l < n_loc; l += blockDim.x) finish(l, fetch(l));
    }
    const bool work = (MODE == kApply || MODE == kResid) ? __syncthreads_or(nonzero) != 0 : true;
    if (MODE != kDiag && !(MODE == kApply || MODE == kResid)) __syncthreads();

    if (work) patches_eval<D, T, MODE == kDiag>(m, cd, S);

    // ---- per-node sums in incidence order
    Acc dot;
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        T s = work ? node_sum(S, l) : T(0);
        const bool dir = is_dirichlet(S.node[l].w);
        if (dir) s = T(0);
        if (l < n_int) {
            const int g = cd.int_begin + l;
            if (MODE == kApply) {
                a.y[g] = s;
            } else if (MODE == kCG) {
                a.y[g] = s;
                dot.add_prod(S.val[l], s);
            } else if (MODE == kResid) {
                const T rv = dir ? T(0) : a.b[g] - s;
                a.y[g] = rv;
                dot.add_prod(rv, rv);
            } else {  // diag: T == double here
                const double dv = dir ? 0.0 : 1.0 / (double)s;
                const_cast<double *>(m.dinv64)[g] = dv;
                const_cast<float *>(m.dinv32)[g] = (float)dv;
            }
        } else {
            a.partial[m.sh_dest[cd.sh_off + (l - n_int)]] = s;
        }
    }
    return dot;
}

// Kernel 1: one block per chunk.
template <int D, typename T, int MODE>
__global__ void __launch_bounds__(256) k_chunks(MeshDev m, VecArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout &L = (sizeof(T) == 4) ? m.sm32 : m.sm64;
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    double *s_red = reinterpret_cast<double *>(smem + L.red);
    // CG scalars are read once per block (not per thread: a same-address
    // hot spot) and broadcast through shared memory.
    if (threadIdx.x == 0) {
        if (MODE == kCG) {
            s_red[0] = a.st->beta;
            s_red[1] = (double)a.st->done;
        }
        mbar_init(s_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (MODE == kCG && s_red[1] != 0.0) return;
    const T beta_cg = (MODE == kCG) ? (T)s_red[0] : T(0);
    __syncthreads();
    uint32_t phase = 0;
    bool failed = false;
    const typename DotOf<T>::type acc = process_chunk<D, T, MODE>(m, a, blockIdx.x, smem, L, phase, beta_cg, failed);
    if (MODE == kCG || MODE == kResid) {
        const double dot = block_sum(acc, s_red);
        if (threadIdx.x == 0) a.dotbuf[blockIdx.x] = dot;
    }
}

// Kernel 2: shared nodes sum their partials in slot order.  The last block to
// finish also reduces all dot partials (kernel 1's n_first blocks, then this
// kernel's blocks) and updates the CG scalars.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_shared(MeshDev m, VecArgs<T> a, int n_first) {
    __shared__ double s_red[34];
    __shared__ bool s_last;
    if (MODE == kCG) {
        if (threadIdx.x == 0) {
            s_red[0] = a.st->beta;
            s_red[1] = (double)a.st->done;
        }
        __syncthreads();
        if (s_red[1] != 0.0) return;
    }
    const T beta_cg = (MODE == kCG) ? (T)s_red[0] : T(0);
    typename DotOf<T>::type acc;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m.n_shared;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = m.n_int + s;
        T sum = T(0);
        const int kb = m.shr_ptr[s], ke = m.shr_ptr[s + 1];
        for (int k = kb; k < ke; ++k) sum += a.partial[k];
        const bool dir = m.dirichlet[g] != 0;
        if (MODE == kApply) {
            a.y[g] = dir ? T(0) : sum;   // (partials of Dirichlet rows may be unmasked: paired-patch kernels)
        } else if (MODE == kCG) {
            T v = cg_dir(a.dinv[g], a.r[g], beta_cg, a.p[g]);
            if (dir) v = T(0);
            a.p[g] = v;
            a.y[g] = sum;
            acc.add_prod(v, sum);
        } else if (MODE == kResid) {
            const T rv = dir ? T(0) : a.b[g] - sum;
            a.y[g] = rv;
            acc.add_prod(rv, rv);
        } else {
            const double dv = dir ? 0.0 : 1.0 / (double)sum;
            const_cast<double *>(m.dinv64)[g] = dv;
            const_cast<float *>(m.dinv32)[g] = (float)dv;
        }
    }
    if (MODE != kCG && MODE != kResid) return;
    const double dot = block_sum(acc, s_red);
    if (threadIdx.x == 0) {
        a.dotbuf[n_first + blockIdx.x] = dot;
        const unsigned int t = atomic_add_acq_rel(&a.st->cnt_a, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    const double tot = block_sum_array(a.dotbuf, n_first + gridDim.x, s_red);
    if (threadIdx.x == 0) {
        CgState *st = a.st;
        st->cnt_a = 0;
        if (MODE == kCG) {
            st->pq = tot;
            if (!(tot > 0.0) || !isfinite(tot)) {
                st->status = kCgBreakdown;
                st->done = 1;
                if (a.host_done) *(volatile int *)a.host_done = 1;
            } else {
                st->alpha = st->rz / tot;
            }
        } else {
            st->rr = tot;
        }
    }
}

// Start of an inner FP32 solve of A d = r64 * scale (mixed mode), or of an
// FP64 PCG run from a residual already in r (mode FP64: rsrc == nullptr).
// Sets d = 0, p = 0, rz = r.D^-1 r, rr0 = r.r, stop_rr = tol2 * (rr0 or bb).
template <typename T>
__global__ void __launch_bounds__(256) k_cg_start(int64_t n_pad, const double *__restrict__ rsrc, double scale,
                                                  T *__restrict__ r, T *__restrict__ d, T *__restrict__ p,
                                                  const T *__restrict__ dinv, CgState *st, double *dotbuf,
                                                  double tol2, int relative, long long max_iters) {
    __shared__ double s_red[34];
    __shared__ bool s_last;
    typename DotOf<T>::type arz, arr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
        T ri = rsrc ? (T)(rsrc[i] * scale) : r[i];
        if (rsrc) r[i] = ri;
        if (d) d[i] = T(0);
        p[i] = T(0);
        arz.add_prod(ri, dinv[i] * ri);
        arr.add_prod(ri, ri);
    }
    const double rz = block_sum(arz, s_red);
    const double rr = block_sum(arr, s_red);
    if (threadIdx.x == 0) {
        dotbuf[blockIdx.x] = rz;
        dotbuf[gridDim.x + blockIdx.x] = rr;
        const unsigned int t = atomic_add_acq_rel(&st->cnt_b, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    const double rz0 = block_sum_array(dotbuf, gridDim.x, s_red);
    const double rr0 = block_sum_array(dotbuf + gridDim.x, gridDim.x, s_red);
    if (threadIdx.x == 0) {
        st->cnt_b = 0;
        st->cnt_a = 0;
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

// x64 += d32 / scale (mixed-mode correction), vectors padded to 4.
static __global__ void k_correct(int64_t n_pad, double *__restrict__ x, const float *__restrict__ d, double inv_scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i] * inv_scale;
}

// out_new[i] = in_old[old_of_new[i]] (0 on Dirichlet nodes); element types converted.
template <typename TI, typename TO>
__global__ void k_perm_in(int64_t n, const TI *__restrict__ in, TO *__restrict__ out, const int32_t *__restrict__ old_of_new,
                          const uint8_t *__restrict__ dirichlet) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dirichlet[i] ? TO(0) : (TO)in[old_of_new[i]];
}
// Merged periodic vertices: out[g] += sum of in[v] over the vertices merged
// into unknown g (ascending vertex id; 0 stays on Dirichlet unknowns).
static __global__ void k_add_slaves(int64_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ slave,
                                    const double *__restrict__ in, double *__restrict__ out,
                                    const uint8_t *__restrict__ dirichlet) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        if (dirichlet[g] || ptr[g] == ptr[g + 1]) continue;
        double v = out[g];
        for (int k = ptr[g]; k < ptr[g + 1]; ++k) v += in[slave[k]];
        out[g] = v;
    }
}
// out_old[j] = in_new[new_of_old[j]]
template <typename TI, typename TO>
__global__ void k_perm_out(int64_t n, const TI *__restrict__ in, TO *__restrict__ out, const int32_t *__restrict__ new_of_old) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = (TO)in[new_of_old[j]];
}

// Fill the alpha slot of every node record: w = +alpha, or -alpha (sign bit
// set, also for alpha = 0) on Dirichlet nodes.
static __global__ void k_set_alpha(int64_t n_loc, const int32_t *__restrict__ loc_node, const double *__restrict__ alpha_new,
                            const uint8_t *__restrict__ dirichlet, NodeF *node32, NodeD *node64) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_loc; k += (int64_t)gridDim.x * blockDim.x) {
        const int g = loc_node[k];
        const double a = alpha_new[g];
        double w64 = a;
        float w32 = (float)a;
        if (dirichlet[g]) {
            w64 = __longlong_as_double(__double_as_longlong(w64) | (long long)0x8000000000000000ULL);
            w32 = __int_as_float(__float_as_int(w32) | (int)0x80000000u);
        }
        node64[k].w = w64;
        node32[k].w = w32;
    }
}

// The same from caller-numbered alpha: unknown g takes alpha of its master
// vertex old_of_new[g].
static __global__ void k_set_alpha_user(int64_t n_loc, const int32_t *__restrict__ loc_node,
                                        const int32_t *__restrict__ old_of_new, const double *__restrict__ alpha_user,
                                        const uint8_t *__restrict__ dirichlet, NodeF *node32, NodeD *node64) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_loc; k += (int64_t)gridDim.x * blockDim.x) {
        const int g = loc_node[k];
        const double a = alpha_user[old_of_new[g]];
        double w64 = a;
        float w32 = (float)a;
        if (dirichlet[g]) {
            w64 = __longlong_as_double(__double_as_longlong(w64) | (long long)0x8000000000000000ULL);
            w32 = __int_as_float(__float_as_int(w32) | (int)0x80000000u);
        }
        node64[k].w = w64;
        node32[k].w = w32;
    }
}

// bdt2[k] = beta[elem_src[k]] * dt2 (0 on padding slots).
static __global__ void k_set_beta(int64_t n, const int32_t *__restrict__ elem_src, const double *__restrict__ beta,
                           double dt2, float *b32, double *b64) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int e = elem_src[k];
        const double v = e >= 0 ? beta[e] * dt2 : 0.0;
        b64[k] = v;
        b32[k] = (float)v;
    }
}

}  // namespace ps
