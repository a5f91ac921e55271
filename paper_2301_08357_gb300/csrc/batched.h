// Batched / persistent solver engine (internal).  Several meshes (each with
// its own right-hand side, iterate and scalars) advance together:
//   * FP64 true residuals and node-range vector steps run as one launch over
//     a task list covering every mesh of the batch;
//   * the FP32 inner solves run in one cooperative persistent kernel whose
//     blocks walk the (mesh, chunk) task list once per CG iteration, with one
//     grid barrier per iteration.
// The inner solver is the fused one-reduction PCG pass of cg1.cuh
// (Chronopoulos and Gear): each chunk updates its nodes from the previous
// pass's double-buffered vectors, applies A, and contributes its share of
// gamma, delta and rho; the last chunk of a mesh to finish advances that
// mesh's scalars.  Each mesh's arithmetic and reduction order depend only on
// that mesh, so a mesh gives bitwise the same result alone and in any batch.
#pragma once
#include <vector>

#include "internal.h"
#include "cg1.cuh"

namespace ps {

constexpr int kSegLen = 256;    // shared nodes per residual segment task (one per thread)
constexpr int kVecLen = 8192;   // nodes (and partial slots) per node-range task
constexpr int kMaxBatch = 4096; // meshes per plan (per-block scalar cache in shared memory)

// Per-mesh phase of a batched solve; every kernel of an epoch acts only on the
// meshes in its phase, and the last block to finish a mesh's part advances it.
enum BPhase : int {
    kPhIdle = 0,       // not part of the current work
    kPhPrepare = 1,    // copy b, x0 from the caller's numbering; ||b||^2
    kPhResid = 2,      // FP64 true residual, convergence / caps decision
    kPhInnerInit = 3,  // r32 = r64 / ||r64||, inner vectors zeroed
    kPhInner = 4,      // FP32 one-reduction PCG in the persistent kernel
    kPhCorrect = 5,    // x64 += d32 * ||r64||
    kPhOutput = 6,     // x back to the caller's numbering
    kPhDone = 7
};

struct BState {
    CgState in;                    // inner FP32 solve (fused pass, cg1.cuh)
    // outer FP64 defect correction
    double rr64, bb, scale, tol2, inner_tol2;
    long long iters_total, max_iters;
    int phase, outer, max_outer, converged;
    unsigned int cnt_r, cnt_v, pad0, pad1;
};

struct BMesh {
    MeshDev d;
    CG1Vec v;                      // double-buffered FP32 inner vectors, per-chunk dots
    double *x64, *b64, *r64;
    double *part64;                // shared-node partial sums (FP64)
    double *dots64;                // [n_chunks + n_segs]
    double *vdots;                 // [n_vt]
    const double *b_user;
    double *x_user;
    const int32_t *old_of_new, *new_of_old;
    const int32_t *slave_ptr, *slave;   // merged periodic vertices (null: none)
    int64_t n_user;                // caller's vertices (>= unknowns with merging)
    int n_segs, n_vt;
    int64_t n_part;                // partial-sum slots (sh_total)
    BState *st;
};

// Host-side batch plan: device arrays of meshes and task lists, the per-mesh
// states (device + pinned host mirror) and the captured epoch graph.
struct BatchPlan {
    ps_ctx *ctx = nullptr;
    std::vector<ps_mesh *> meshes;
    // device buffers, kept (and grown) across rebuilds of the plan: states,
    // mesh records, the three task lists
    DevAlloc buf_st{nullptr, 0}, buf_meshes{nullptr, 0}, buf_t[3] = {{nullptr, 0}, {nullptr, 0}, {nullptr, 0}};
    size_t h_st_cap = 0;           // BState entries the pinned mirror holds
    int epochs = 0;                // epochs run since the plan was (re)built
    BMesh *d_meshes = nullptr;
    int2 *d_t1 = nullptr, *d_t2 = nullptr, *d_t3 = nullptr;   // chunk, shared-segment, node-range tasks
    int n_t1 = 0, n_t2 = 0, n_t3 = 0;
    BState *d_st = nullptr;        // [n] contiguous device states
    BState *h_st = nullptr;        // [n] pinned host mirror (written by the epoch)
    std::vector<BMesh> h_meshes;
    SmemLayout L32, L64;
    uint32_t pcg_smem = 0;         // L32 plus the per-block scalar cache
    int grid_pcg = 0;
    int epoch_iters = 256;
    int h_active = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = true;
    uint32_t spin_limit = kGridSpinLimit;   // grid-barrier polls before giving up
    int threads = 256;                      // threads per block of the persistent kernel
    int order = 0;                          // task order (PcgArgs::order)
};

// Per-mesh batch workspace beyond ps_mesh::ws (FP64 reduction partials).
struct BatchMeshWs {
    std::vector<DevAlloc> allocs;
    double *dots64 = nullptr, *vdots = nullptr;
    int n_segs = 0, n_vt = 0;
};

// Build (or rebuild) the plan for `n` distinct meshes of one context
// (workspaces allocated on first use); states start in kPhIdle.  A rebuild
// keeps the plan's buffers when they are large enough; its copies are
// ordered on stream s (nothing synchronises the device).
int batch_plan_build(ps_ctx *ctx, ps_mesh *const *meshes, int n, int epoch_iters, const ps_solve_opts &o,
                     cudaStream_t s, BatchPlan &plan);
void batch_plan_free(BatchPlan &plan);
// Start a solve of mesh i: caller-numbering device vectors b (read) and x
// (first guess in, solution out), options; state -> kPhPrepare.  Takes effect
// at the next batch_upload_states.
void batch_arm(BatchPlan &plan, int i, const double *b_user, double *x_user, const ps_solve_opts &o);
int batch_upload_states(BatchPlan &plan, cudaStream_t s);
// One epoch: prepare / residual / inner-init / persistent PCG (<= epoch_iters
// iterations) / correct / output for every mesh in the matching phase, then
// the states are copied to plan.h_st.  Synchronises the stream.
int batch_epoch(BatchPlan &plan, cudaStream_t s);
// Fill a solve info from a finished mesh's state.
void batch_info(const BatchPlan &plan, int i, ps_solve_info *info);

}  // namespace ps
