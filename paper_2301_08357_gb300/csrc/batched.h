// Batched / persistent solver engine (internal).  Several meshes (each with
// its own right-hand side, iterate and scalars) advance together:
//   * FP64 true residuals and node-range vector steps run as one launch over
//     a task list covering every mesh of the batch;
//   * the FP32 inner solves run in one cooperative persistent kernel whose
//     blocks walk (mesh, chunk) and (mesh, shared-node segment) task lists
//     with grid barriers between the two phases of each iteration.
// The inner solver is preconditioned CG in the one-reduction form of
// Chronopoulos and Gear (s = A p carried by recurrence, w = A u computed,
// gamma = r.u, delta = w.u and rho = r.r reduced together once per
// iteration).  Each mesh's arithmetic and reduction order depend only on that
// mesh, so a mesh gives bitwise the same result alone and in any batch.
#pragma once
#include <vector>

#include "internal.h"

namespace ps {

constexpr int kSegLen = 2048;   // shared nodes per phase-2 task
constexpr int kVecLen = 8192;   // nodes per node-range task

struct BState {
    // inner FP32 solve (one-reduction PCG)
    double gamma, delta, rho, rho0, stop2, alpha, beta, inner_tol2;
    // outer FP64 defect correction
    double rr64, bb, scale, tol2;
    long long iters, max_iters, iters_total;
    int first, done, status, active;   // active: this mesh runs an inner solve in this outer step
    int finished;                      // set by the host: the mesh's solve is over
    unsigned int cnt2, cnt_r, cnt_v;
};

struct BMesh {
    MeshDev d;
    float *x, *r, *p, *s, *w;      // FP32 inner vectors
    float *part;                   // shared-node partial sums (FP32)
    double *dots;                  // [(n_chunks + n_segs) * 3]
    double *x64, *b64, *r64;
    double *part64;                // shared-node partial sums (FP64)
    double *dots64;                // [n_chunks + n_segs]
    double *vdots;                 // [n_vt]
    const double *b_user;
    double *x_user;
    const int32_t *old_of_new, *new_of_old;
    int n_segs, n_vt;
    BState *st;
};

// Host-side batch plan (device arrays of meshes and task lists).
struct BatchPlan {
    ps_ctx *ctx = nullptr;
    std::vector<ps_mesh *> meshes;
    std::vector<DevAlloc> allocs;
    BMesh *d_meshes = nullptr;
    int2 *d_t1 = nullptr, *d_t2 = nullptr, *d_t3 = nullptr;
    int n_t1 = 0, n_t2 = 0, n_t3 = 0;
    BState *d_st = nullptr;
    std::vector<BState> h_st;
    std::vector<BMesh> h_meshes;
    uint32_t smem32 = 0, smem64 = 0;
    int grid_pcg = 0;
    int *h_active = nullptr;       // pinned: active-mesh count read back per launch
};

// Per-mesh batch workspace (extra FP32 vectors beyond ps_mesh::ws).
struct BatchMeshWs {
    std::vector<DevAlloc> allocs;
    float *s32 = nullptr, *w32 = nullptr;
    double *dots = nullptr, *dots64 = nullptr, *vdots = nullptr;
    BState *st = nullptr;
    int n_segs = 0, n_vt = 0;
};

int batch_plan_build(ps_ctx *ctx, ps_mesh *const *meshes, int n, BatchPlan &plan);
void batch_plan_free(BatchPlan &plan);
// Set the per-call user vectors and options; resets every mesh's state.
int batch_begin(BatchPlan &plan, const double *const *b_user, double *const *x_user, double tol, double inner_tol,
                long long max_iters, cudaStream_t s);
// One outer step for all meshes not yet finished: FP64 residual; returns the
// number of meshes that still need an inner solve (after applying max_outer).
int batch_residual(BatchPlan &plan, cudaStream_t s, int *n_active);
// Inner FP32 solves of the active meshes, at most `epoch` iterations per
// persistent launch, until all of them finish.
int batch_inner(BatchPlan &plan, int epoch, cudaStream_t s);
int batch_correct(BatchPlan &plan, cudaStream_t s);
int batch_finish(BatchPlan &plan, cudaStream_t s);
int batch_read_states(BatchPlan &plan, cudaStream_t s);

}  // namespace ps
