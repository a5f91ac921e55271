// Batched / persistent solver engine: see batched.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "../../include/pressure.h"
#include "batched.h"
#include "cg1.cuh"

namespace ps {

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_i32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// bar[0] = arrival count, bar[32] = generation, bar[64] = the stop word the
// last arriver publishes (separate 128-byte lines).  The last block to arrive
// has seen every block's work of the pass, so it reads the active-mesh count
// then and publishes "stop" before releasing the generation: every block
// takes the same decision.  The wait is bounded: on timeout the error flag is
// set and false returned; the caller then leaves the kernel (other blocks
// time out in turn).
__device__ bool grid_barrier_stop(unsigned int *bar, int *err, const int *active_cnt, int *s_stop,
                                  uint32_t spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int *count = bar, *gen = bar + 32, *stop = bar + 64;
        const unsigned int g = ld_acquire_u32(gen);
        const unsigned int arrived = atomic_add_acq_rel(count, 1u);
        int ok = 0;
        if (arrived == gridDim.x - 1) {
            *(volatile unsigned int *)count = 0u;
            *(volatile unsigned int *)stop = ld_acquire_i32(active_cnt) <= 0 ? 1u : 0u;
            st_release_u32(gen, g + 1u);
            ok = 1;
        } else {
            for (uint32_t i = 0; i < spin_limit; ++i) {
                if (ld_acquire_u32(gen) != g) {
                    ok = 1;
                    break;
                }
                __nanosleep(32);
            }
            if (!ok) atomicOr(err, kErrGridTimeout);
        }
        s_ok = ok;
        *s_stop = ok ? (int)*(volatile unsigned int *)stop : 1;
    }
    __syncthreads();
    return s_ok != 0;
}

enum VecOp : int { kPrepare = 0, kInnerInit = 1, kCorrect = 2, kFinish = 3 };

struct PcgArgs {
    const BMesh *meshes;
    const int2 *t1;                // (mesh, chunk) tasks, mesh-major
    int n_t1, n_meshes;
    unsigned int *bar;
    int *active_cnt;
    int *err;
    int max_it;
    uint32_t spin_limit;           // polls of the grid barrier before it gives up
    int order;                     // task order: 0 = (mesh, chunk) list, 1 = running meshes' chunks, compacted
    SmemLayout L;                  // chunk layout; the scalar cache follows at L.total
};

// The last chunk of mesh M to finish a pass: reduce the per-chunk triples and
// advance the mesh's inner scalars; a finished inner solve moves the mesh to
// the correction phase.
__device__ void batch_mesh_scalars(const BMesh &M, double *red, int *active_cnt) {
    double tot[3];
    cg1_reduce(M.v.dots, M.d.n_chunks, red, tot);
    if (threadIdx.x != 0) return;
    BState *st = M.st;
    st->in.cnt_a = 0;
    const int was_first = st->in.first;
    const int done = cg1_scalars(&st->in, tot[0], tot[1], tot[2]);
    if (!was_first) st->iters_total += 1;
    if (done) {
        st->phase = kPhCorrect;
        atomicSub(active_cnt, 1);
    }
}

// The persistent inner solver: up to max_it fused passes of every mesh in the
// inner phase, one grid barrier per pass.  At the start of a pass every block
// reads each mesh's (run, parity, alpha, beta) into its shared-memory cache,
// so a task costs no scalar round trip.
__global__ void __launch_bounds__(256) k_batch_pcg(PcgArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const ChunkSmem<float> S = chunk_smem<float>(smem, A.L);
    float2 *c_ab = reinterpret_cast<float2 *>(smem + A.L.total);          // [n_meshes]
    int *c_par = reinterpret_cast<int *>(c_ab + A.n_meshes);               // [n_meshes], -1 = idle
    // compacted order: chunks of each mesh (cached) and the first compacted
    // task of each mesh this pass (running meshes only), + scan scratch
    int *c_nch = c_par + A.n_meshes;                                       // [n_meshes]
    int *c_off = c_nch + A.n_meshes;                                       // [n_meshes + 1]
    int *c_scan = c_off + A.n_meshes + 1;                                  // [blockDim]
    __shared__ int s_stop;
    __shared__ bool s_last;
    // the current task's mesh descriptor and buffers, copied into shared
    // memory: read through a global reference, every pointer would be
    // reloaded after each global store the pass makes (possible aliasing)
    __shared__ __align__(16) MeshDev s_md;
    __shared__ __align__(16) CG1Vec s_v;
    __shared__ int s_mesh;
    if (threadIdx.x == 0) {
        s_mesh = -1;
        mbar_init(S.bar, 1);
        fence_mbar_init();
        // no mesh leaves the inner phase before this launch's first pass, so
        // every block reads the same count here; later decisions come from
        // the grid barrier
        s_stop = ld_acquire_i32(A.active_cnt) <= 0;
    }
    if (A.order == 1)
        for (int i = threadIdx.x; i < A.n_meshes; i += blockDim.x) c_nch[i] = A.meshes[i].d.n_chunks;
    __syncthreads();
    uint32_t phase = 0;
    bool failed = false;
    for (int it = 0; it < A.max_it && !s_stop; ++it) {
        for (int i = threadIdx.x; i < A.n_meshes; i += blockDim.x) {
            const BState *st = A.meshes[i].st;
            const bool run = __ldcg(&st->phase) == kPhInner && !__ldcg(&st->in.done);
            c_par[i] = run ? cg1_parity(__ldcg(&st->in.first), __ldcg(&st->in.iters)) : -1;
            c_ab[i] = make_float2((float)__ldcg(&st->in.alpha), (float)__ldcg(&st->in.beta));
        }
        __syncthreads();
        int n_tasks = A.n_t1;
        if (A.order == 1) {
            // exclusive scan of the running meshes' chunk counts: thread t
            // sums a contiguous range of meshes, the block scans the sums
            const int per = (A.n_meshes + blockDim.x - 1) / blockDim.x;
            const int i0 = threadIdx.x * per, i1 = min(A.n_meshes, i0 + per);
            int sum = 0;
            for (int i = i0; i < i1; ++i) sum += c_par[i] >= 0 ? c_nch[i] : 0;
            c_scan[threadIdx.x] = sum;
            __syncthreads();
            for (int d = 1; d < (int)blockDim.x; d <<= 1) {
                const int v = threadIdx.x >= (unsigned)d ? c_scan[threadIdx.x - d] : 0;
                __syncthreads();
                c_scan[threadIdx.x] += v;
                __syncthreads();
            }
            int off = c_scan[threadIdx.x] - sum;
            for (int i = i0; i < i1; ++i) {
                c_off[i] = off;
                off += c_par[i] >= 0 ? c_nch[i] : 0;
            }
            if (threadIdx.x == blockDim.x - 1) c_off[A.n_meshes] = c_scan[threadIdx.x];
            __syncthreads();
            n_tasks = c_off[A.n_meshes];
        }
        for (int t = blockIdx.x; t < n_tasks; t += gridDim.x) {
            int2 tk;
            if (A.order == 1) {
                // the running mesh whose compacted range holds task t
                int lo = 0, hi = A.n_meshes;       // c_off[lo] <= t < c_off[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (c_off[mid] <= t) lo = mid; else hi = mid;
                }
                tk = make_int2(lo, t - c_off[lo]);
            } else {
                tk = A.t1[t];
            }
            const int par = c_par[tk.x];
            if (par < 0) continue;                 // block-uniform
            const BMesh &M = A.meshes[tk.x];
            const float2 ab = c_ab[tk.x];
            if (s_mesh != tk.x) {                  // block-uniform
                __syncthreads();                   // the previous task's readers are done
                constexpr int nd = sizeof(MeshDev) / 4, nv = sizeof(CG1Vec) / 4;
                static_assert(sizeof(MeshDev) % 4 == 0 && sizeof(CG1Vec) % 4 == 0, "word copy");
                const uint32_t *src_d = reinterpret_cast<const uint32_t *>(&M.d);
                const uint32_t *src_v = reinterpret_cast<const uint32_t *>(&M.v);
                for (int k = threadIdx.x; k < nd + nv; k += blockDim.x) {
                    if (k < nd) reinterpret_cast<uint32_t *>(&s_md)[k] = src_d[k];
                    else reinterpret_cast<uint32_t *>(&s_v)[k - nd] = src_v[k - nd];
                }
                __syncthreads();
                if (threadIdx.x == 0) s_mesh = tk.x;
            }
            DotF acc[3];
            if (s_md.dim == 3)
                chunk_cg1f<3>(s_md, cg1_pass(s_v, par), s_v.dinv, tk.y, ab.x, ab.y, S, phase, acc, failed);
            else
                chunk_cg1f<2>(s_md, cg1_pass(s_v, par), s_v.dinv, tk.y, ab.x, ab.y, S, phase, acc, failed);
            if (failed) return;
            double out[3];
            block_sum_n<3>(acc, S.red, out);
            if (threadIdx.x == 0) {
                M.v.dots[3 * tk.y] = df_pack(out[0]);
                M.v.dots[3 * tk.y + 1] = df_pack(out[1]);
                M.v.dots[3 * tk.y + 2] = df_pack(out[2]);
                const unsigned int k = atomic_add_acq_rel(&M.st->in.cnt_a, 1u);
                s_last = (k == (unsigned)M.d.n_chunks - 1u);
            }
            __syncthreads();
            if (s_last) batch_mesh_scalars(M, S.red, A.active_cnt);
            __syncthreads();
        }
        if (!grid_barrier_stop(A.bar, A.err, A.active_cnt, &s_stop, A.spin_limit)) return;
    }
}

// ---- FP64 true residual over the batch: chunk tasks, then shared segments.
__global__ void __launch_bounds__(256) k_b_resid1(const BMesh *meshes, const int2 *t1, SmemLayout L) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int2 tk = t1[blockIdx.x];
    const BMesh &M = meshes[tk.x];
    __shared__ int s_run;
    const ChunkSmem<double> S = chunk_smem<double>(smem, L);
    if (threadIdx.x == 0) {
        s_run = M.st->phase == kPhResid;
        mbar_init(S.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (!s_run) return;
    VecArgs<double> a;
    a.x = M.x64;
    a.y = M.r64;
    a.b = M.b64;
    a.p = nullptr;
    a.r = nullptr;
    a.dinv = nullptr;
    a.partial = M.part64;
    a.dotbuf = nullptr;
    a.st = nullptr;
    a.host_done = nullptr;
    uint32_t phase = 0;
    bool failed = false;
    DotD acc = (M.d.dim == 3) ? process_chunk<3, double, kResid>(M.d, a, tk.y, smem, L, phase, 0.0, failed)
                              : process_chunk<2, double, kResid>(M.d, a, tk.y, smem, L, phase, 0.0, failed);
    const double v = block_sum(acc, S.red);
    if (threadIdx.x == 0) M.dots64[tk.y] = v;
}

__global__ void __launch_bounds__(256) k_b_resid2(const BMesh *meshes, const int2 *t2) {
    __shared__ double red[34];
    __shared__ bool s_last;
    __shared__ int s_run;
    const int2 tk = t2[blockIdx.x];
    const BMesh &M = meshes[tk.x];
    const MeshDev &m = M.d;
    if (threadIdx.x == 0) s_run = M.st->phase == kPhResid;
    __syncthreads();
    if (!s_run) return;
    const int64_t s0 = (int64_t)tk.y * kSegLen;
    const int64_t s1 = s0 + kSegLen < m.n_shared ? s0 + kSegLen : m.n_shared;
    DotD acc;
    for (int64_t sidx = s0 + threadIdx.x; sidx < s1; sidx += blockDim.x) {
        const int64_t g = m.n_int + sidx;
        double sum = 0.0;
        for (int k = m.shr_ptr[sidx]; k < m.shr_ptr[sidx + 1]; ++k) sum += M.part64[k];
        const double rv = m.dirichlet[g] ? 0.0 : M.b64[g] - sum;
        M.r64[g] = rv;
        acc.add_prod(rv, rv);
    }
    const double v = block_sum(acc, red);
    if (threadIdx.x == 0) {
        M.dots64[m.n_chunks + tk.y] = v;
        const unsigned int t = atomic_add_acq_rel(&M.st->cnt_r, 1u);
        s_last = (t == (unsigned)M.n_segs - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    const int n = m.n_chunks + M.n_segs;
    double rr = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) rr += __ldcg(M.dots64 + k);
    rr = block_sum(rr, red);
    if (threadIdx.x == 0) {
        BState *st = M.st;
        st->cnt_r = 0;
        st->rr64 = rr;
        const double bb = st->bb > 0.0 ? st->bb : 1.0;
        if (rr <= st->tol2 * bb) {
            st->converged = 1;
            st->phase = kPhOutput;
        } else if (st->outer >= st->max_outer || st->iters_total >= st->max_iters || st->in.status == kCgBreakdown) {
            st->phase = kPhOutput;
        } else {
            st->outer += 1;
            st->scale = 1.0 / sqrt(rr);
            CgState &in = st->in;
            in.rz = in.pq = in.alpha = in.beta = in.rr = in.rr0 = in.stop_rr = 0.0;
            // the inner reduction of the single-solve engines (inner_reduction)
            const double itol = sqrt(st->inner_tol2);
            const double need = 0.1 * sqrt(st->tol2) * sqrt(bb) / sqrt(rr);
            const double it_k = need > itol ? fmin(need, 0.5) : itol;
            in.tol2 = it_k * it_k;
            in.iters = 0;
            in.max_iters = st->max_iters - st->iters_total;
            in.done = 0;
            in.status = kCgRunning;
            in.first = 1;
            in.free_run = 0;
            in.cnt_a = in.cnt_b = 0;
            st->phase = kPhInnerInit;
        }
    }
}

// ---- node-range steps over the batch; each acts on meshes in one phase and
// the last block of a mesh advances it.
template <int OP>
__global__ void __launch_bounds__(256) k_b_vec(const BMesh *meshes, const int2 *t3, int *active_cnt) {
    constexpr int want = OP == kPrepare ? kPhPrepare : OP == kInnerInit ? kPhInnerInit
                       : OP == kCorrect ? kPhCorrect : kPhOutput;
    __shared__ double red[34];
    __shared__ bool s_last;
    __shared__ double s_sc[2];
    const int2 tk = t3[blockIdx.x];
    const BMesh &M = meshes[tk.x];
    const MeshDev &m = M.d;
    if (threadIdx.x == 0) {
        s_sc[0] = M.st->phase == want ? 1.0 : 0.0;
        s_sc[1] = M.st->scale;
    }
    __syncthreads();
    if (s_sc[0] == 0.0) return;
    const double scale = s_sc[1];
    const int64_t i0 = (int64_t)tk.y * kVecLen;
    const int64_t i1 = i0 + kVecLen < m.n_pad ? i0 + kVecLen : m.n_pad;
    DotD acc;
    // the tasks cover max(n_pad, partial slots); vector steps stop at n_pad
    if (OP == kPrepare) {
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            double bv = 0.0, xv = 0.0;
            if (i < m.n_nodes && !m.dirichlet[i]) {
                const int o = M.old_of_new[i];
                bv = M.b_user[o];
                xv = M.x_user[o];
                if (M.slave_ptr)    // loads of merged periodic vertices add onto the unknown
                    for (int k = M.slave_ptr[i]; k < M.slave_ptr[i + 1]; ++k) bv += M.b_user[M.slave[k]];
            }
            M.b64[i] = bv;
            M.x64[i] = xv;
            acc.add_prod(bv, bv);
        }
    } else if (OP == kInnerInit) {
        // pass 0 reads buffer 0: r = r64 / ||r64||, x = p = s = w = 0 and
        // the shared-node partial sums of w = 0
        float *r = M.v.r[0], *x = M.v.x[0], *p = M.v.p[0], *sv = M.v.s[0], *w = M.v.w[0], *part = M.v.part[0];
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            r[i] = (float)(M.r64[i] * scale);
            x[i] = 0.f;
            p[i] = 0.f;
            sv[i] = 0.f;
            w[i] = 0.f;
        }
        const int64_t j1 = i0 + kVecLen < M.n_part ? i0 + kVecLen : M.n_part;
        for (int64_t j = i0 + threadIdx.x; j < j1; j += blockDim.x) part[j] = 0.f;
    } else if (OP == kCorrect) {
        const double inv = 1.0 / scale;
        __shared__ int s_par;
        if (threadIdx.x == 0) s_par = cg1_parity(M.st->in.first, M.st->in.iters);
        __syncthreads();
        const float *x = s_par ? M.v.x[1] : M.v.x[0];
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) M.x64[i] += (double)x[i] * inv;
    } else {  // kFinish
        const int64_t j1 = i0 + kVecLen < M.n_user ? i0 + kVecLen : M.n_user;
        for (int64_t j = i0 + threadIdx.x; j < j1; j += blockDim.x) M.x_user[j] = M.x64[M.new_of_old[j]];
    }
    double v = 0.0;
    if (OP == kPrepare) v = block_sum(acc, red);
    if (threadIdx.x == 0) {
        if (OP == kPrepare) M.vdots[tk.y] = v;
        const unsigned int t = atomic_add_acq_rel(&M.st->cnt_v, 1u);
        s_last = (t == (unsigned)M.n_vt - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    double bb = 0.0;
    if (OP == kPrepare) {
        for (int k = threadIdx.x; k < M.n_vt; k += blockDim.x) bb += __ldcg(M.vdots + k);
        bb = block_sum(bb, red);
    }
    if (threadIdx.x == 0) {
        BState *st = M.st;
        st->cnt_v = 0;
        if (OP == kPrepare) {
            st->bb = bb;
            st->phase = kPhResid;
        } else if (OP == kInnerInit) {
            st->phase = kPhInner;
            atomicAdd(active_cnt, 1);
        } else if (OP == kCorrect) {
            st->phase = kPhResid;
        } else {
            st->phase = kPhDone;
        }
    }
}

// ---------------------------------------------------------------- host side
static int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return PS_OK;
    ps_set_last_error(cudaGetErrorString(e));
    return cuda_status(e);
}

// Opt a kernel in to the largest dynamic shared memory the device allows
// next to the kernel's own static shared memory.
template <typename F>
static cudaError_t allow_max_dyn_smem(F *func) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void *)func);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    return e;
}

int batched_set_attrs() {
    cudaError_t e = allow_max_dyn_smem(k_batch_pcg);
    if (e == cudaSuccess) e = allow_max_dyn_smem(k_b_resid1);
    return cuda_rc(e);
}

static int ensure_batch_ws(ps_mesh *m) {
    if (m->batch_ws) return PS_OK;
    int rc = ensure_workspace(m);
    if (rc != PS_OK) return rc;
    BatchMeshWs *w = new BatchMeshWs();
    const int64_t np = m->dev.n_pad;
    const int64_t span = std::max<int64_t>(std::max<int64_t>(np, m->prep.sh_total), m->prep.n_nodes);
    w->n_segs = (int)std::max<int64_t>(1, (m->prep.n_shared + kSegLen - 1) / kSegLen);
    w->n_vt = (int)((span + kVecLen - 1) / kVecLen);
    void *p;
    auto A = [&](void **dst, size_t bytes) -> int {
        int r = dalloc(m->ctx, dst, bytes, w->allocs);
        if (r == PS_OK) cudaMemset(*dst, 0, bytes);
        return r;
    };
    rc = A(&p, (size_t)(m->dev.n_chunks + w->n_segs) * 8);
    w->dots64 = (double *)p;
    if (rc == PS_OK) rc = A(&p, (size_t)w->n_vt * 8), w->vdots = (double *)p;
    if (rc != PS_OK) {
        dfree_all(m->ctx, w->allocs);
        delete w;
        return rc;
    }
    m->batch_ws = w;
    return PS_OK;
}

int64_t batch_ws_bytes(const ps_mesh *m) {
    // vectors of ps_mesh::ws and BatchMeshWs (an estimate for admission):
    // FP64 x b r p q, FP32 x r p q (two buffers each), s (two), D^-1 copies
    // of the unpreconditioned mode, partial sums, per-chunk dots
    const int64_t np = m->dev.n_pad, sh = m->prep.sh_total;
    return np * (5 * 8 + 12 * 4) + sh * 16 + (int64_t)m->dev.n_chunks * 48;
}

void batched_release_mesh(ps_mesh *m) {
    if (!m->batch_ws) return;
    BatchMeshWs *w = static_cast<BatchMeshWs *>(m->batch_ws);
    dfree_all(m->ctx, w->allocs);
    delete w;
    m->batch_ws = nullptr;
}

// A plan buffer of at least `bytes` (grown by half again when it is too
// small; the contents are not kept).
static int plan_buf(ps_ctx *ctx, DevAlloc &a, size_t bytes) {
    if (a.p && a.bytes >= bytes) return PS_OK;
    if (a.p) {
        cudaFree(a.p);
        ctx->bytes -= (int64_t)a.bytes;
        a = DevAlloc{nullptr, 0};
    }
    std::vector<DevAlloc> one;
    const int rc = dalloc(ctx, &a.p, std::max<size_t>(bytes + bytes / 2, 4096), one);
    if (rc == PS_OK) a.bytes = one[0].bytes;
    return rc;
}

void batch_plan_free(BatchPlan &plan) {
    if (plan.graph) cudaGraphExecDestroy(plan.graph);
    if (plan.cap) cudaStreamDestroy(plan.cap);
    if (plan.ctx) {
        for (DevAlloc *a : {&plan.buf_st, &plan.buf_meshes, &plan.buf_t[0], &plan.buf_t[1], &plan.buf_t[2]})
            if (a->p) {
                cudaFree(a->p);
                plan.ctx->bytes -= (int64_t)a->bytes;
            }
    }
    if (plan.h_st) cudaFreeHost(plan.h_st);
    plan = BatchPlan();
}

// Combined shared-memory layout: every mesh's segments fit.
static SmemLayout max_layout(const std::vector<ps_mesh *> &meshes, bool fp64) {
    int max_loc = 0, max_patch = 0, max_inc = 0, max_sh = 0;
    for (ps_mesh *m : meshes) {
        max_loc = std::max(max_loc, m->prep.max_loc);
        max_patch = std::max(max_patch, m->prep.max_patch);
        max_inc = std::max(max_inc, m->prep.max_inc);
        max_sh = std::max(max_sh, m->prep.max_sh);
    }
    return fp64 ? make_layout(8, sizeof(NodeD), max_loc, max_patch, max_inc, max_sh)
                : make_layout(4, sizeof(NodeF), max_loc, max_patch, max_inc, max_sh);
}

int batch_plan_build(ps_ctx *ctx, ps_mesh *const *meshes, int n, int epoch_iters, const ps_solve_opts &o,
                     cudaStream_t s, BatchPlan &plan) {
    if (plan.ctx && plan.ctx != ctx) batch_plan_free(plan);
    // a rebuild keeps the buffers, the pinned mirror and the capture stream;
    // the captured epoch belongs to the old task lists
    if (plan.graph) {
        cudaGraphExecDestroy(plan.graph);
        plan.graph = nullptr;
    }
    plan.graph_ok = true;
    plan.epochs = 0;
    if ((o.batch_threads != 0 && o.batch_threads != 128 && o.batch_threads != 256) || o.batch_order < 0 ||
        o.batch_order > 1) {
        ps_set_last_error("batch: batch_threads must be 0, 128 or 256 and batch_order 0 or 1");
        return PS_EINVAL;
    }
    plan.threads = o.batch_threads ? o.batch_threads : 256;
    plan.order = o.batch_order;
    plan.spin_limit = o.grid_spin_limit > 0 ? (uint32_t)o.grid_spin_limit : kGridSpinLimit;
    if (n < 1 || n > kMaxBatch) {
        ps_set_last_error("batch: between 1 and 4096 meshes per batch");
        return PS_EINVAL;
    }
    plan.ctx = ctx;
    plan.meshes.assign(meshes, meshes + n);
    plan.epoch_iters = epoch_iters > 0 ? epoch_iters : 256;
    std::vector<int2> t1, t2, t3;
    plan.h_meshes.resize(n);
    int rc = plan_buf(ctx, plan.buf_st, (size_t)n * sizeof(BState) + 4096);
    if (rc != PS_OK) return rc;
    plan.d_st = (BState *)plan.buf_st.p;
    // grid-barrier words and the active-mesh counter live after the states
    rc = cuda_rc(cudaMemsetAsync(plan.d_st, 0, (size_t)n * sizeof(BState) + 4096, s));
    if (rc != PS_OK) return rc;
    for (int i = 0; i < n; ++i) {
        ps_mesh *m = meshes[i];
        rc = ensure_batch_ws(m);
        if (rc != PS_OK) return rc;
        BatchMeshWs *w = static_cast<BatchMeshWs *>(m->batch_ws);
        BMesh &B = plan.h_meshes[i];
        std::memset(&B, 0, sizeof(B));
        B.d = m->dev;
        const Workspace &ws = m->ws;
        B.v.x[0] = ws.x32;
        B.v.x[1] = ws.x32b;
        B.v.r[0] = ws.r32;
        B.v.r[1] = ws.r32b;
        B.v.s[0] = ws.s32a;
        B.v.s[1] = ws.s32b;
        B.v.p[0] = ws.p32;
        B.v.p[1] = ws.p32b;
        B.v.w[0] = ws.q32;
        B.v.w[1] = ws.q32b;
        B.v.part[0] = ws.part32;
        B.v.part[1] = ws.part32b;
        B.v.dinv = m->dev.dinv32;
        B.v.dots = reinterpret_cast<float2 *>(ws.dots1);
        B.n_part = m->prep.sh_total;
        B.x64 = m->ws.x64;
        B.b64 = m->ws.b64;
        B.r64 = m->ws.r64;
        B.part64 = m->ws.part64;
        B.dots64 = w->dots64;
        B.vdots = w->vdots;
        B.old_of_new = m->d_old_of_new;
        B.new_of_old = m->d_new_of_old;
        B.slave_ptr = m->d_slave_ptr;
        B.slave = m->d_slave;
        B.n_user = m->prep.n_nodes;
        B.n_segs = w->n_segs;
        B.n_vt = w->n_vt;
        B.st = plan.d_st + i;
        for (int c = 0; c < m->dev.n_chunks; ++c) t1.push_back(make_int2(i, c));
        for (int sg = 0; sg < w->n_segs; ++sg) t2.push_back(make_int2(i, sg));
        for (int v = 0; v < w->n_vt; ++v) t3.push_back(make_int2(i, v));
    }
    plan.n_t1 = (int)t1.size();
    plan.n_t2 = (int)t2.size();
    plan.n_t3 = (int)t3.size();
    rc = plan_buf(ctx, plan.buf_meshes, (size_t)n * sizeof(BMesh));
    plan.d_meshes = (BMesh *)plan.buf_meshes.p;
    if (rc == PS_OK) rc = plan_buf(ctx, plan.buf_t[0], t1.size() * sizeof(int2)), plan.d_t1 = (int2 *)plan.buf_t[0].p;
    if (rc == PS_OK) rc = plan_buf(ctx, plan.buf_t[1], t2.size() * sizeof(int2)), plan.d_t2 = (int2 *)plan.buf_t[1].p;
    if (rc == PS_OK) rc = plan_buf(ctx, plan.buf_t[2], t3.size() * sizeof(int2)), plan.d_t3 = (int2 *)plan.buf_t[2].p;
    if (rc != PS_OK) return rc;
    // pageable sources: staged by the runtime before the calls return
    cudaError_t e = cudaMemcpyAsync(plan.d_t1, t1.data(), t1.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan.d_t2, t2.data(), t2.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan.d_t3, t3.data(), t3.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && plan.h_st_cap < (size_t)n) {
        // the pinned mirror grows; no copy of it is in flight (the previous
        // epoch's read-back completed before its stream synchronisation)
        if (plan.h_st) cudaFreeHost(plan.h_st);
        plan.h_st = nullptr;
        plan.h_st_cap = 0;
        const size_t cap = std::max<size_t>((size_t)n + n / 2, 16);
        e = cudaHostAlloc((void **)&plan.h_st, cap * sizeof(BState), cudaHostAllocDefault);
        if (e == cudaSuccess) plan.h_st_cap = cap;
    }
    if (e != cudaSuccess) return cuda_rc(e);
    std::memset(plan.h_st, 0, (size_t)n * sizeof(BState));
    plan.L32 = max_layout(plan.meshes, false);
    plan.L64 = max_layout(plan.meshes, true);
    // scalar cache (alpha, beta; parity) per mesh, then the compacted order's
    // chunk counts, offsets and scan scratch
    plan.pcg_smem = plan.L32.total + (uint32_t)n * (sizeof(float2) + sizeof(int)) +
                    (uint32_t)(2 * n + 1 + plan.threads) * sizeof(int);
    int per_sm = 0;
    rc = cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pcg, plan.threads, plan.pcg_smem));
    if (rc != PS_OK) return rc;
    if (per_sm < 1) {
        ps_set_last_error("batch: shared-memory layout too large for the persistent kernel");
        return PS_EINVAL;
    }
    const int cap = plan.threads == 128 ? 8 : 4;   // resident blocks per SM used
    plan.grid_pcg = std::max(1, std::min(ctx->sms * std::min(per_sm, cap), std::max(plan.n_t1, 1)));
    return PS_OK;
}

void batch_arm(BatchPlan &plan, int i, const double *b_user, double *x_user, const ps_solve_opts &o) {
    plan.h_meshes[i].b_user = b_user;
    plan.h_meshes[i].x_user = x_user;
    BState &st = plan.h_st[i];
    std::memset(&st, 0, sizeof(st));
    const double tol = o.tol > 0 ? o.tol : 1e-10;
    const double itol = o.inner_tol > 0 ? o.inner_tol : 1e-4;
    st.tol2 = tol * tol;
    st.inner_tol2 = itol * itol;
    st.max_iters = o.max_iters > 0 ? o.max_iters : 100000;
    st.max_outer = o.max_outer > 0 ? o.max_outer : 40;
    st.phase = kPhPrepare;
}

static unsigned int *plan_bar(const BatchPlan &plan) {
    return (unsigned int *)((char *)plan.d_st + plan.meshes.size() * sizeof(BState) + 1024);
}

int batch_upload_states(BatchPlan &plan, cudaStream_t s) {
    const int n = (int)plan.meshes.size();
    // meshes carried over mid inner solve are counted as active
    int act = 0;
    for (int i = 0; i < n; ++i) act += plan.h_st[i].phase == kPhInner && !plan.h_st[i].in.done;
    plan.h_active = act;
    int *active = (int *)(plan_bar(plan) + 128);
    cudaError_t e = cudaMemcpyAsync(plan.d_meshes, plan.h_meshes.data(), n * sizeof(BMesh), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(plan.d_st, plan.h_st, n * sizeof(BState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(active, &plan.h_active, sizeof(int), cudaMemcpyHostToDevice, s);
    // (no synchronisation: the host leaves h_st alone until the next epoch's
    // read-back has completed; the other two sources are pageable, staged)
    return cuda_rc(e);
}

// Enqueue one epoch on stream s (also used under stream capture).
static int epoch_enqueue(BatchPlan &plan, cudaStream_t s) {
    const int n = (int)plan.meshes.size();
    unsigned int *bar = plan_bar(plan);
    int *active = (int *)(bar + 128);
    k_b_vec<kPrepare><<<plan.n_t3, 256, 0, s>>>(plan.d_meshes, plan.d_t3, active);
    k_b_resid1<<<plan.n_t1, 256, plan.L64.total, s>>>(plan.d_meshes, plan.d_t1, plan.L64);
    k_b_resid2<<<plan.n_t2, 256, 0, s>>>(plan.d_meshes, plan.d_t2);
    k_b_vec<kInnerInit><<<plan.n_t3, 256, 0, s>>>(plan.d_meshes, plan.d_t3, active);
    int rc = cuda_rc(cudaGetLastError());
    if (rc != PS_OK) return rc;
    PcgArgs A;
    A.meshes = plan.d_meshes;
    A.t1 = plan.d_t1;
    A.n_t1 = plan.n_t1;
    A.n_meshes = n;
    A.bar = bar;
    A.active_cnt = active;
    A.err = plan.ctx->d_err;
    A.max_it = plan.epoch_iters;
    A.spin_limit = plan.spin_limit;
    A.order = plan.order;
    A.L = plan.L32;
    void *args[] = {&A};
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(plan.grid_pcg);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.pcg_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    rc = cuda_rc(cudaLaunchKernelExC(&cfg, (const void *)k_batch_pcg, args));
    if (rc != PS_OK) return rc;
    k_b_vec<kCorrect><<<plan.n_t3, 256, 0, s>>>(plan.d_meshes, plan.d_t3, active);
    k_b_vec<kFinish><<<plan.n_t3, 256, 0, s>>>(plan.d_meshes, plan.d_t3, active);
    rc = cuda_rc(cudaGetLastError());
    if (rc != PS_OK) return rc;
    return cuda_rc(cudaMemcpyAsync(plan.h_st, plan.d_st, n * sizeof(BState), cudaMemcpyDeviceToHost, s));
}

int batch_epoch(BatchPlan &plan, cudaStream_t s) {
    // the first epoch of a (re)built plan runs its launches directly: a plan
    // that is rebuilt after one epoch (the serving loop's membership
    // changes) never pays for a capture
    if (plan.graph_ok && !plan.graph && plan.epochs >= 1) {
        // capture the epoch once per plan; fall back to direct launches if
        // the runtime refuses to capture any of it
        if (!plan.cap && cudaStreamCreateWithFlags(&plan.cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            plan.graph_ok = false;
        }
        if (plan.graph_ok) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(plan.cap, cudaStreamCaptureModeThreadLocal);
            int rc = e == cudaSuccess ? epoch_enqueue(plan, plan.cap) : PS_ECUDA;
            cudaError_t e2 = cudaStreamEndCapture(plan.cap, &g);
            if (e == cudaSuccess && rc == PS_OK && e2 == cudaSuccess && g) {
                if (cudaGraphInstantiate(&plan.graph, g, 0) != cudaSuccess) plan.graph = nullptr;
            }
            if (g) cudaGraphDestroy(g);
            if (!plan.graph) {
                cudaGetLastError();
                plan.graph_ok = false;
            }
        }
    }
    int rc;
    if (plan.graph)
        rc = cuda_rc(cudaGraphLaunch(plan.graph, s));
    else
        rc = epoch_enqueue(plan, s);
    if (rc != PS_OK) return rc;
    plan.epochs++;
    rc = cuda_rc(cudaStreamSynchronize(s));
    if (rc != PS_OK) return rc;
    int herr = 0;
    cudaMemcpy(&herr, plan.ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr) {
        cudaMemset(plan.ctx->d_err, 0, sizeof(int));
        cudaMemset(plan_bar(plan), 0, 1024);
        ps_set_last_error("batch epoch: a bounded device wait timed out");
        return PS_ETIMEOUT;
    }
    return PS_OK;
}

void batch_info(const BatchPlan &plan, int i, ps_solve_info *inf) {
    const BState &st = plan.h_st[i];
    std::memset(inf, 0, sizeof(*inf));
    const double bb = st.bb > 0 ? st.bb : 1.0;
    inf->converged = st.converged;
    inf->status = st.converged ? PS_OK : (st.in.status == kCgBreakdown ? PS_EBREAKDOWN : PS_ENOTCONV);
    inf->iters_outer = st.outer + 1;
    inf->iters_inner = st.iters_total;
    inf->rel_res = std::sqrt(st.rr64 / bb);
    inf->bnorm = std::sqrt(st.bb);
    inf->n_free = plan.meshes[i]->prep.n_free;
}

int batch_solve_locked(ps_mesh *const *meshes, int n, const double *const *b_dev, double *const *x_dev,
                       const ps_solve_opts &o, ps_solve_info *infos, cudaStream_t s) {
    ps_ctx *ctx = meshes[0]->ctx;
    auto t0 = std::chrono::steady_clock::now();
    BatchPlan plan;
    const int epoch = o.graph_iters > 0 ? o.graph_iters * 8 : 256;
    int rc = batch_plan_build(ctx, meshes, n, epoch, o, s, plan);
    if (rc == PS_OK) {
        for (int i = 0; i < n; ++i) batch_arm(plan, i, b_dev[i], x_dev[i], o);
        rc = batch_upload_states(plan, s);
    }
    if (rc == PS_OK && o.graph_iters < 0) plan.graph_ok = false;
    // every epoch advances each unfinished mesh by at least one phase step;
    // bound the number of epochs by the iteration and outer-step caps
    long long max_epochs = 8;
    for (int i = 0; i < n && rc == PS_OK; ++i) {
        const BState &st = plan.h_st[i];
        max_epochs = std::max(max_epochs, (long long)st.max_outer * 3 + st.max_iters / plan.epoch_iters + 8);
    }
    long long ep = 0;
    while (rc == PS_OK) {
        bool all = true;
        for (int i = 0; i < n; ++i) all = all && plan.h_st[i].phase == kPhDone;
        if (all) break;
        if (++ep > max_epochs) {
            ps_set_last_error("batch solve: epoch budget exhausted");
            rc = PS_ETIMEOUT;
            break;
        }
        rc = batch_epoch(plan, s);
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int first_err = PS_OK;
    if (rc == PS_OK) {
        for (int i = 0; i < n; ++i) {
            ps_solve_info tmp;
            batch_info(plan, i, &tmp);
            tmp.seconds = secs;
            tmp.kernel_launches = ep * (plan.graph ? 7 : 7);
            if (infos) infos[i] = tmp;
            if (tmp.status != PS_OK && first_err == PS_OK) first_err = tmp.status;
        }
    }
    batch_plan_free(plan);
    return rc != PS_OK ? rc : first_err;
}

}  // namespace ps

using namespace ps;

extern "C" int ps_batch_solve(ps_mesh *const *meshes, int n, const double *const *b_dev, double *const *x_dev,
                              const ps_solve_opts *opts, ps_solve_info *infos, void *stream) {
    if (!meshes || n < 1 || !b_dev || !x_dev) return PS_EINVAL;
    ps_ctx *ctx = meshes[0] ? meshes[0]->ctx : nullptr;
    if (!ctx) return PS_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!meshes[i] || meshes[i]->ctx != ctx || !b_dev[i] || !x_dev[i]) return PS_EINVAL;
        if (!meshes[i]->coeff_ok) return PS_ESTATE;
        for (int j = 0; j < i; ++j)
            if (meshes[j] == meshes[i]) return PS_EINVAL;
    }
    ps_solve_opts o;
    if (opts) o = *opts; else ps_solve_opts_default(&o);
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_rc(e);
    return batch_solve_locked(meshes, n, b_dev, x_dev, o, infos, (cudaStream_t)stream);
}
