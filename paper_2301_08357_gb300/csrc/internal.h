// Internal host-side types of libpressure (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <set>
#include <vector>

#include "../../include/pressure.h"
#include "mesh_prep.h"
#include "ops.cuh"

struct ps_mesh;

namespace ps {

struct DevAlloc {
    void *p;
    size_t bytes;
};

struct GraphRec {
    int kind;    // precision (0 FP32, 1 FP64) + 2 * (no preconditioner) + 4 * (fused engine)
    int iters;
    cudaGraphExec_t exec;
};

// Per-mesh solver workspace (allocated on first apply/solve).
struct Workspace {
    bool ready = false;
    std::vector<DevAlloc> allocs;
    double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float *part32 = nullptr;
    double *part64 = nullptr;
    double *dot1 = nullptr, *dot2 = nullptr;
    double *pq2 = nullptr, *z3 = nullptr;   // two-kernel CG partials
    // paired-patch operator kernel: chunk shares of p.Ap, all bits set
    // (0xffffffff, a NaN no arithmetic produces) while not yet written
    float2 *pqu = nullptr;
    // fused CG (FP32): second buffers of x, r, p, w (first: x32, r32, p32,
    // q32), both buffers of s, second partial buffer, per-chunk dot triples
    float *x32b = nullptr, *r32b = nullptr, *p32b = nullptr, *q32b = nullptr;
    float *s32a = nullptr, *s32b = nullptr, *part32b = nullptr;
    double *dots1 = nullptr;
    float2 *halo32 = nullptr;   // paired-patch CG: (D^-1 r, p) per chunk-major shared slot
    CgState *st = nullptr;
    CgState *h_st = nullptr;
    float *one32 = nullptr;
    double *one64 = nullptr;
    bool ones_ready = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphRec> graphs;
    int64_t last_iters[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // iterations of the last CG run per graph kind
};

int dalloc(ps_ctx *ctx, void **p, size_t bytes, std::vector<DevAlloc> &owner);
void dfree_all(ps_ctx *ctx, std::vector<DevAlloc> &owner);
int grid_for(int64_t n, int dev_sms);
int cuda_status(cudaError_t e);
SmemLayout make_layout(int esz, int nsz, int max_loc, int max_patch, int max_inc, int max_sh);
int ensure_workspace(ps_mesh *m);
template <typename T, int MODE>
int launch_pass(ps_mesh *m, const VecArgs<T> &a, cudaStream_t s);

int beta_update_device(ps_mesh *m, const double *beta_dev, double dt2, cudaStream_t s, bool diag = true);
// ps_pressure_solve with the context mutex held by the caller.
int pressure_solve_locked(ps_mesh *m, const double *b, double *x, const ps_solve_opts *opts, ps_solve_info *info,
                          cudaStream_t s);
int alpha_update_device(ps_mesh *m, const double *alpha_dev, cudaStream_t s, bool diag = true);
double inner_reduction(double itol, double tol, double bb, double rr);

// projection.cu
void projection_release(ps_mesh *m);

// apply_noalloc.cu
int noalloc_setup(int device);

// batched.cu
int batched_set_attrs();
void batched_release_mesh(ps_mesh *m);
int64_t batch_ws_bytes(const ps_mesh *m);
int batch_solve_locked(ps_mesh *const *meshes, int n, const double *const *b_dev, double *const *x_dev,
                       const ps_solve_opts &o, ps_solve_info *infos, cudaStream_t s);

}  // namespace ps

struct ps_ctx {
    int device = 0;
    size_t budget = 0;
    int sms = 1;
    std::atomic<int64_t> bytes{0};
    std::recursive_mutex mu_r;
    std::mutex mu;
    std::set<ps_mesh *> meshes;
    int *d_err = nullptr;
    unsigned int *d_bar = nullptr;   // grid-barrier words + active counter of the persistent solver
};

struct ps_mesh {
    ps_ctx *ctx = nullptr;
    ps::PrepMesh prep;
    ps::MeshDev dev;
    std::vector<ps::DevAlloc> allocs;
    int32_t *d_loc_node = nullptr, *d_elem_src = nullptr;
    int32_t *d_old_of_new = nullptr, *d_new_of_old = nullptr;
    int32_t *d_slave_ptr = nullptr, *d_slave = nullptr;   // merged periodic vertices (null: none)
    int grid2 = 1, grid3 = 1, g3c = 1;
    ps::SmemLayout pipe_L0, pipe_L1;   // two-stage layout of the pipelined CG kernel
    int pipe_grid = 0;                 // its persistent grid (0 = not used)
    int pipeline = 0;                  // ps_mesh_opts::pipeline
    int update_bps = 0;                // ps_mesh_opts::update_blocks_per_sm
    int k1_variant = 0;                // ps_mesh_opts::operator_kernel
    bool k1_pre = false;               // FP32 operator kernel variant (beta prefetch)
    bool use_units = false;            // FP32 CG operator kernel on paired patches (3D)
    int unit_threads = 128;            // its threads per block (ps_mesh_opts::operator_threads)
    int32_t *d_uelem = nullptr;        // element of each (unit, element, half) slot, -1 none
    bool coeff_ok = false, alpha_set = false;
    bool alpha_newton = false;         // alpha last set by the general-EOS Newton iteration
    double dt2 = 0.0;
    ps::Workspace ws;
    void *batch_ws = nullptr;   // owned by batched.cu
    void *proj = nullptr;       // owned by projection.cu
    std::vector<double> coords_host;   // [n_nodes * dim], caller's numbering
    std::vector<double> alpha_host;    // [n_nodes], caller's numbering (last ps_coeff_set)
    int64_t alpha_version = 0;
    int64_t launches = 0;       // kernel launches of the current call
};

extern "C" void ps_set_last_error(const char *msg);
