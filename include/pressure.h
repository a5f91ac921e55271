/*
 * pressure.h -- C ABI of libpressure: the P1 finite-element pressure system of
 * the semi-implicit hybrid FV/FE all-Mach scheme, solved matrix-free by
 * (preconditioned) conjugate gradient on one GB300 (sm_103a).
 *
 * The operator.  On the nodes of a primal triangle (dim 2) or tetrahedron
 * (dim 3) mesh, the projection stage (Section 3.4, weak problem) asks for the
 * pressure correction dP with
 *
 *     A dP = b,   A = M_alpha + dt^2 K_beta,
 *     (M_alpha)_ij = int alpha_h phi_i phi_j      (consistent mass, no lumping)
 *     (K_beta)_ij  = int beta grad phi_i . grad phi_j
 *
 * phi_i the P1 hat functions, alpha_h the P1 interpolant of a nodal field alpha
 * (the paper's constant 1/(gamma-1), eq. pressure_dt, generalised to a nodal
 * field), beta piecewise constant per element (the enthalpy H^{n+1,k} moved to
 * the primal elements, Section 3.3) and dt the time step.  The stiffness sign
 * is the one Green's formula gives from the strong form (eq. pressure_dt); it
 * is the sign that makes A symmetric positive definite, which Section 3.4
 * states and which the conjugate gradient method of the abstract needs.
 *
 * Dirichlet nodes (Section 3.6: the pressure is imposed on boundary vertices)
 * are homogeneous: their rows and columns are removed from A.  Every vector
 * crossing this ABI is a full nodal vector in the CALLER'S node numbering; on
 * Dirichlet nodes inputs are ignored and outputs are 0.  The library renumbers
 * nodes and reorders elements internally; that numbering never leaks out.
 *
 * Conventions.
 *  - Every function returns an int status (PS_OK = 0, negative = error); no
 *    C++ exception crosses this boundary.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Device pointers (suffix _dev) are caller-owned CUDA
 *    device allocations on the context's device; the library never frees them.
 *  - stream arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).  Work is ordered on that stream; functions that
 *    report scalars (solve info) synchronise it before returning.
 *  - A ps_ctx and the meshes created from it may be used from one host thread
 *    at a time; different contexts are independent.
 */
#ifndef PRESSURE_H
#define PRESSURE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PS_OK            0
#define PS_PENDING       1   /* ps_solve_poll: request not finished yet            */
#define PS_EINVAL       -1   /* bad argument: index out of range, degenerate or
                                non-finite element, alpha < 0, beta <= 0, ...     */
#define PS_ENOMEM       -2   /* device allocation failed or HBM budget exceeded   */
#define PS_ENOTCONV     -3   /* iteration limit reached; info is still filled      */
#define PS_EBREAKDOWN   -4   /* CG breakdown: p.Ap <= 0 or a non-finite scalar     */
#define PS_ETIMEOUT     -5   /* a bounded device-side wait gave up                 */
#define PS_ECUDA        -6   /* a CUDA runtime call failed                          */
#define PS_ESTATE       -7   /* call out of order (e.g. solve before coeff_set)     */
#define PS_ENOTFOUND    -8   /* unknown ticket / case id                            */

/* ---- precision of pressure_apply ------------------------------------- */
#define PS_F32 1             /* x, y are float  arrays; FP32 element arithmetic    */
#define PS_F64 2             /* x, y are double arrays; FP64 element arithmetic    */

/* ---- solver modes ---------------------------------------------------- */
#define PS_MODE_FP64   0     /* plain PCG, all vectors and arithmetic in FP64      */
#define PS_MODE_MIXED  1     /* FP32 PCG inner solves inside FP64 defect correction */

#define PS_PRECOND_NONE   0
#define PS_PRECOND_JACOBI 1

/* ---- mass form of the operator (ps_mesh_set_mass) -------------------- */
#define PS_MASS_CONSISTENT 0  /* int alpha_h phi_i phi_j (Section 3.4; default)   */
#define PS_MASS_LUMPED     1  /* vertex quadrature: diagonal (Section 3, general EOS) */

typedef struct ps_ctx ps_ctx;
typedef struct ps_mesh ps_mesh;
typedef struct ps_server ps_server;
typedef int64_t ps_ticket;

/* Mesh preprocessing options (all zero = defaults). */
typedef struct {
    int32_t chunk_elems;     /* target elements per chunk (0 = auto by size)       */
    int32_t chunk_nodes_max; /* cap on distinct nodes per chunk (0 = auto)          */
    int32_t pipeline;        /* FP32 CG operator kernel: 0 = one block per chunk,  */
                             /* 1 = persistent blocks with double-buffered staging */
    int32_t update_blocks_per_sm; /* grid of the CG update kernel in blocks per SM */
                             /* (0 = auto)                                          */
    int32_t operator_kernel; /* FP32 CG operator kernel of 3D meshes: 0 = auto     */
                             /* (paired patches), 1 = one patch per thread,        */
                             /* 2 = paired patches (packed FP32x2 arithmetic,      */
                             /* fixed-point node sums)                              */
    int32_t operator_threads; /* threads per block of the paired-patch kernel:     */
                             /* 0 = auto (128), 128 or 256                          */
    int32_t split_lead;      /* chunks at the head of the (Morton) chunk order split */
                             /* in halves when the mesh has at least four times as */
                             /* many, so the first wave of blocks ends out of step:*/
                             /* 0 = auto (3D meshes with the paired-patch kernel:  */
                             /* one per SM; ps_debug_prepare: none), -1 = none,    */
                             /* n > 0 = n                                           */
    int32_t reserved[1];
} ps_mesh_opts;

typedef struct {
    double tol;              /* stop when ||b - A x||_2 / ||b||_2 <= tol (FP64 true
                                residual over free nodes); default 1e-10            */
    int64_t max_iters;       /* cap on total CG iterations (0 = 100000)            */
    int32_t mode;            /* PS_MODE_FP64 or PS_MODE_MIXED                       */
    int32_t precond;         /* PS_PRECOND_JACOBI (default) or PS_PRECOND_NONE     */
    double inner_tol;        /* mixed: inner FP32 relative reduction (0 = 1e-4);   */
                             /* an outer step that needs less to reach tol asks    */
                             /* for 10x what it needs instead (at most 0.5)        */
    int32_t max_outer;       /* mixed: cap on defect-correction steps (0 = 40)     */
    int32_t graph_iters;     /* most iterations per captured CUDA graph launch     */
                             /* (0 = 32; shorter batches follow the previous run's */
                             /* iteration count;                                   */
                             /* negative = launch kernels directly, no graph)      */
    int32_t engine;          /* single solves, captured in CUDA graphs:             */
                             /* PS_ENGINE_GRAPH: two kernels per CG iteration;      */
                             /* PS_ENGINE_FUSED (mixed mode): one fused kernel per  */
                             /* inner iteration (one-reduction PCG): fewer launches */
                             /* and reductions, more vector traffic per pass; FP64  */
                             /* mode falls back to two kernels;                     */
                             /* PS_ENGINE_AUTO: FUSED for meshes of at most 200,000 */
                             /* nodes (where it measured faster), else GRAPH;       */
                             /* PS_ENGINE_PERSISTENT (mixed mode) runs the batched  */
                             /* persistent engine on a batch of one, which gives    */
                             /* bitwise the result the mesh gets in any batch       */
    int32_t grid_spin_limit; /* diagnostic: polls of the persistent kernel's grid   */
                             /* barrier before it gives up and the call returns     */
                             /* PS_ETIMEOUT (batched, persistent and served solves; */
                             /* 0 = 2^26 polls, each at least 32 ns apart)          */
    int32_t batch_threads;   /* batched / persistent / served solves: threads per   */
                             /* block of the persistent kernel (0 = 256, 128, 256)  */
    int32_t batch_order;     /* their task order per pass: 0 = the (mesh, chunk)    */
                             /* list in mesh order, static round robin over blocks; */
                             /* 1 = only the chunks of meshes still running,        */
                             /* compacted each pass, static round robin             */
    int32_t reserved[2];
} ps_solve_opts;

#define PS_ENGINE_AUTO        0
#define PS_ENGINE_GRAPH       1
#define PS_ENGINE_PERSISTENT  2
#define PS_ENGINE_FUSED       3

typedef struct {
    int32_t status;          /* PS_OK, PS_ENOTCONV, PS_EBREAKDOWN, ...             */
    int32_t converged;       /* 1 if rel_res <= tol                                */
    int64_t iters_outer;     /* FP64 true-residual evaluations (mixed: outer steps) */
    int64_t iters_inner;     /* CG iterations (mixed: FP32 inner iterations)       */
    double rel_res;          /* final TRUE relative residual ||b-Ax||/||b||, FP64  */
    double bnorm;            /* ||b||_2 over free nodes                            */
    int64_t n_free;          /* number of free (non-Dirichlet) nodes               */
    double seconds;          /* wall time of the call; for a served request the
                                latency from submission to completion             */
    int64_t kernel_launches; /* CUDA kernels this call launched (graph nodes included) */
    double queue_seconds;    /* served request: time queued before admission       */
    double reserved[2];
} ps_solve_info;

typedef struct {
    int64_t n_nodes, n_elems, n_free;
    int32_t dim, n_chunks;
    int64_t n_shared;        /* nodes touched by more than one chunk               */
    int64_t chunk_node_refs; /* sum over chunks of distinct nodes                  */
    int64_t device_bytes;    /* device memory held by this mesh                     */
    int32_t max_chunk_elems, max_chunk_nodes;
    int64_t solve_bytes;     /* device bytes of this mesh's solver state while a solve
                                is in flight (the serving loop's admission unit)    */
    int64_t operator_kernel; /* FP32 CG operator kernel in use: 1 one patch per
                                thread, 2 paired patches (ps_mesh_opts)             */
    int64_t reserved[2];
} ps_mesh_stats;

/* ---- library --------------------------------------------------------- */

/* Library version string (static storage). */
const char *ps_version(void);

/* Human-readable name of a status code (static storage). */
const char *ps_status_str(int status);

/* Message of the last error raised on the calling thread ("" if none;
 * thread-local static storage, valid until the next failing call). */
const char *ps_last_error(void);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory held by meshes, coefficients and solver workspaces of this context
 * (0 = no cap beyond the device).  *out receives the handle.  The first
 * context on a device also commits the 16 MiB scratch array of
 * ps_pressure_apply_noalloc on it (outside every budget; held until exit):
 * PS_ENOMEM if the device cannot provide it. */
int ps_ctx_create(ps_ctx **out, int device, size_t hbm_budget_bytes);

/* Destroy a context and every mesh still attached to it. */
void ps_ctx_destroy(ps_ctx *ctx);

/* Device bytes currently held by the context's meshes and workspaces. */
int64_t ps_ctx_bytes_in_use(const ps_ctx *ctx);

/* ---- mesh (Section 3.1: primal simplex mesh, P1 unknowns on vertices) ----
 *
 * ps_mesh_upload: copy a mesh to the device.
 *   dim         2 (triangles) or 3 (tetrahedra)
 *   coords      host [n_nodes][dim] double, vertex coordinates
 *   conn        host [n_elems][dim+1] int32, 0-based vertex ids (any orientation)
 *   dirichlet   host [n_nodes] uint8; nonzero = homogeneous Dirichlet node
 *               (may be NULL: no Dirichlet nodes)
 *   opts        preprocessing options or NULL
 * Host work: element partition into chunks along a Morton curve, node
 * renumbering (chunk-interior nodes contiguous per chunk, nodes shared between
 * chunks after them), per-chunk local connectivity and incidence lists, and
 * the FP64 stiffness weights of every element for the FP64 passes (about
 * 75 B per tetrahedron, 40 B per triangle of device memory, padding
 * included; ps_mesh_stats.device_bytes gives the total).
 * Errors: PS_EINVAL for dim not 2/3, n_elems < 1, a vertex id out of range, a
 * non-finite coordinate or an element of zero volume; PS_ENOMEM. */
int ps_mesh_upload(ps_ctx *ctx, int dim, int64_t n_nodes, const double *coords,
                   int64_t n_elems, const int32_t *conn, const uint8_t *dirichlet,
                   const ps_mesh_opts *opts, ps_mesh **out);

/* Release a mesh and its device memory. */
void ps_mesh_free(ps_mesh *mesh);

int ps_mesh_get_stats(const ps_mesh *mesh, ps_mesh_stats *out);

/* ---- periodic boundaries (Section 3.6: the vertices of matching periodic
 * boundary faces are merged, which reduces the unknowns of the pressure
 * system).  As ps_mesh_upload, plus
 *   periodic  host [n_nodes] int32: periodic[i] = the vertex whose unknown
 *             vertex i shares (its master), periodic[i] = i for ordinary
 *             vertices; a master is its own master; a vertex and its master
 *             carry the same Dirichlet flag; no element may hold two vertices
 *             of one unknown.
 * Each element keeps its own vertex coordinates, so the merged vertices may
 * lie on opposite sides of the domain.  Vectors still cross the ABI in the
 * caller's numbering over all n_nodes vertices: on input, x and the apply's
 * operand take each unknown's value from its master; a right-hand side is a
 * load vector, so the loads of merged vertices are added onto their unknown;
 * on output every vertex carries its unknown's value.  alpha is taken from
 * the master.  Errors: PS_EINVAL for an inconsistent map (ps_last_error
 * names the rule). */
int ps_mesh_upload_periodic(ps_ctx *ctx, int dim, int64_t n_nodes, const double *coords, int64_t n_elems,
                            const int32_t *conn, const uint8_t *dirichlet, const int32_t *periodic,
                            const ps_mesh_opts *opts, ps_mesh **out);

/* ---- coefficients (Section 3.4: 1/(gamma-1), H^{n+1,k}, dt) -----------
 *   alpha_nodal  host [n_nodes] double, >= 0, finite
 *   beta_elem    host [n_elems] double, > 0, finite (element order of upload)
 *   dt2          dt^2 > 0
 * Also builds the Jacobi diagonal D_ii = sum_e (M^e_ii + dt2 K^e_ii) on the
 * device.  May be called again to change coefficients (e.g. between Picard
 * iterations or time steps).  Errors: PS_EINVAL. */
int ps_coeff_set(ps_mesh *mesh, const double *alpha_nodal, const double *beta_elem, double dt2);

/* Only beta changes (alpha and dt2 kept): same checks and effect. */
int ps_coeff_set_beta(ps_mesh *mesh, const double *beta_elem);

/* ---- mass form (Section 3, the general equation of state: with mass
 * lumping the pressure system becomes mildly nonlinear and Newton-type
 * methods solve it) -------------------------------------------------------
 *   mass  PS_MASS_CONSISTENT (the form of Section 3.4) or PS_MASS_LUMPED:
 *         the alpha-weighted mass integral by vertex quadrature on every
 *         element, (M_alpha)_ij = delta_ij alpha_i m_i with
 *         m_i = int phi_i = sum over the elements e around i of |T_e|/(d+1).
 * Every apply and solve of the mesh (single, batched, served) uses the form
 * set last; the Jacobi diagonal is rebuilt if coefficients are set.  A server
 * reads the form when it admits a request: change it only while no request
 * of the mesh is in flight.  Errors: PS_EINVAL (unknown form). */
int ps_mesh_set_mass(ps_mesh *mesh, int mass);

/* ---- operator apply: y = A x (Dirichlet rows/cols removed) ---------------
 *   x_dev, y_dev  device [n_nodes] float (PS_F32) or double (PS_F64), caller
 *                 numbering; must not alias.
 * Matrix-free, element by element; no atomics; deterministic (the same
 * inputs give bitwise the same outputs).  Errors: PS_EINVAL, PS_ESTATE. */
int ps_pressure_apply(ps_mesh *mesh, const void *x_dev, void *y_dev, int precision, void *stream);

/* ---- operator apply without device allocation ---------------------------
 * Same arguments, result and errors as ps_pressure_apply, for callers that
 * cannot allocate device memory at the point of the call (their framework's
 * allocator already holds the memory they may use, or an allocation would
 * synchronise the device inside a time-critical loop).  The paper has no
 * counterpart: this is a deployment variant of the same operator.
 * Scratch (permuted copies of x and y, shared-node partial sums) lives in one
 * file-scope device array of 16 MiB that every GPU loading the library holds
 * until exit; meshes needing more (about 2 x n_nodes x 4 or 8 bytes plus the
 * partial sums) are rejected with PS_EINVAL and a ps_last_error message.  The
 * array's device address is looked up once per device when the first
 * context is created on it (ps_ctx_create), which loads the module and
 * commits the array's memory there, not inside this call; the cached address
 * assumes the device's primary context lives until the process exits (no
 * cudaDeviceReset in between).  The array lies outside the context's HBM
 * budget.  Calls share the array: calls whose work overlaps on the GPU race.
 * Calls no cudaMalloc or cudaFree.  If a bounded device wait gives up, y is
 * undefined and the context's error flag reports PS_ETIMEOUT at its next
 * synchronising call (a solve or coefficient update).  The mesh itself must
 * have been uploaded and its coefficients set. */
int ps_pressure_apply_noalloc(ps_mesh *mesh, const void *x_dev, void *y_dev, int precision, void *stream);

/* ---- solve A x = b (Section 3.4: SPD system, matrix-free CG, warm start) --
 *   b_dev  device [n_nodes] double, caller numbering (Dirichlet entries ignored)
 *   x_dev  device [n_nodes] double; in: first guess (e.g. the pressure of the
 *          previous time level), out: solution (0 on Dirichlet nodes)
 *   opts   NULL = defaults (mixed precision, Jacobi, tol 1e-10)
 *   info   may be NULL
 * Returns PS_OK when the FP64 true relative residual reaches opts->tol,
 * PS_ENOTCONV when an iteration cap stops it first (x holds the last iterate),
 * PS_EBREAKDOWN on p.Ap <= 0 or a non-finite scalar. */
int ps_pressure_solve(ps_mesh *mesh, const double *b_dev, double *x_dev,
                      const ps_solve_opts *opts, ps_solve_info *info, void *stream);

/* Fill opts with the defaults. */
void ps_solve_opts_default(ps_solve_opts *opts);

/* ---- projection stage of one time step (Sections 3.3-3.5) ----------------
 * The pressure solve inside its Picard loop, for the ideal gas of Section 2:
 * first guesses H^{n+1,1}_e = gamma/(gamma-1) mean_k(P^n_k) / rho_e and
 * (rho K)^{n+1,1}_e = |W~~_u,e|^2 / (2 rho_e) (Section 3.3); then n_picard
 * iterations (Section 3.4) of
 *   beta = H^{n+1,k} (operator and Jacobi diagonal updated on the device),
 *   b_i = int (W~_E - (rho K)^{n+1,k}) phi_i - int alpha_h P^n_h phi_i
 *         + dt int H^{n+1,k} W~~_u . grad phi_i          (weak problem)
 *   solve A dP = b (ps_pressure_solve with opts->solve; warm start: dp_dev,
 *         then the previous Picard iterate),
 *   P = P^n + dP,  W_u = W~~_u - dt grad dP_h,  H and rho K from them.
 * alpha is the mesh's nodal coefficient from ps_coeff_set (1/(gamma-1) for
 * the ideal gas); the mesh's dt2 becomes dt*dt and its beta the H of the last
 * solve.  Readings: the boundary term of the weak problem is taken as zero
 * (closed walls: W_u . eta = 0 on the Neumann boundary); element values of
 * the enthalpy use the vertex mean of the nodal pressure.
 * All arrays are device memory in the caller's numbering / element order:
 *   rho_dev  [n_elems]        density rho^{n+1} per element (> 0)
 *   wu_dev   [n_elems * dim]  intermediate momentum W~~_u per element
 *   we_dev   [n_elems]        intermediate total energy density W~_E per element
 *   pn_dev   [n_nodes]        pressure P^n
 *   dp_dev   [n_nodes]        in: first guess of dP, out: dP^{n+1} (0 on Dirichlet nodes)
 *   p_dev    [n_nodes]        out: P^{n+1} = P^n + dP
 *   wun_dev  [n_elems * dim]  out: W_u^{n+1}
 *   h_dev    [n_elems]        out: H from P^{n+1} (the next Picard guess)
 *   rhok_dev [n_elems]        out: (rho K) from W_u^{n+1}
 * info: the last solve's record, with iters_inner / iters_outer / seconds
 * summed over the Picard iterations (may be NULL).  Errors: PS_EINVAL (bad
 * argument, or an enthalpy that is not positive and finite), PS_ESTATE
 * (coefficients not set), and the statuses of ps_pressure_solve (a solve
 * that does not return PS_OK ends the step at once: dp_dev holds its last
 * iterate, h_dev and rhok_dev the guesses that solve used, p_dev and wun_dev
 * the previous Picard iteration's values, unset if it was the first).  Device
 * data for the element passes (coordinates, connectivity, node-to-element
 * lists) is allocated on the first call and counted in the context budget. */
typedef struct {
    double gamma;            /* ratio of specific heats, > 1                     */
    double dt;               /* time step, > 0                                   */
    int32_t n_picard;        /* Picard iterations, 1..64 (the paper uses 2)       */
    int32_t reserved[7];
    ps_solve_opts solve;     /* options of every pressure solve                  */
} ps_projection_opts;

void ps_projection_opts_default(ps_projection_opts *opts);
int ps_projection_step(ps_mesh *mesh, const ps_projection_opts *opts, const double *rho_dev,
                       const double *wu_dev, const double *we_dev, const double *pn_dev, double *dp_dev,
                       double *p_dev, double *wun_dev, double *h_dev, double *rhok_dev,
                       ps_solve_info *info, void *stream);

/* ---- projection stage with a general equation of state (Section 3: the
 * energy equation with W_E(P, rho) in place of the ideal gas; with lumped
 * mass the pressure system is mildly nonlinear, solved by Newton's method)
 * The internal energy density is
 *     rho e(P, rho) = eos_a P + eos_b P^2 / rho,
 * the caloric equation of a thermally perfect gas whose c_v is linear in the
 * temperature (eos_b = 0: the ideal gas, eos_a = 1/(gamma-1)).  Enthalpy per
 * element H_e = (rho e(Pbar, rho_e) + Pbar) / rho_e, Pbar the vertex mean.
 * Per Picard iteration k (H^{n+1,k}, (rho K)^{n+1,k} frozen, as in
 * ps_projection_step), with w_ei = |T_e|/(d+1) and dP on the free nodes:
 *   F_i(dP) = sum_e w_ei rho e(P^n_i + dP_i, rho_e) + dt^2 (K_H dP)_i - c_i,
 *   c_i = int (W~_E - rho K) phi_i + dt int H W~~_u . grad phi_i;
 * Newton from the current dP: J = diag(Q'_i) + dt^2 K_H, Q'_i the derivative
 * of the mass sum, set as the mesh's alpha_i = Q'_i / m_i (lumped operator),
 * then J dP_new = J dP - F(dP) solved by ps_pressure_solve (opts->solve,
 * warm start dP; its Jacobi preconditioner is the diagonal of the Picard
 * iteration's first Jacobian).  The step stops when ||F||_2 <= newton_tol ||c||_2 over
 * the free nodes (checked before each solve and after the last) or after
 * max_newton solves.  Then the post-projection of ps_projection_step with
 * the EOS enthalpy.
 *   requires ps_mesh_set_mass(mesh, PS_MASS_LUMPED); not for periodic meshes.
 *   Arrays and outputs: as ps_projection_step.  newton_res_host: NULL or host
 *   [n_picard * (max_newton + 1)] doubles, ||F||/||c|| at each check (-1
 *   where no check ran).  After the call the mesh's alpha is the last
 *   Jacobian's, beta the last H, dt2 = dt^2 (ps_projection_step then needs a
 *   new ps_coeff_set).  Errors: PS_EINVAL (bad argument, periodic mesh, an
 *   enthalpy or Jacobian entry Q'_i that is not positive and finite),
 *   PS_ESTATE (consistent mass), PS_ENOTCONV (newton_tol > 0 not reached in
 *   the last Picard iteration; outputs written), and the statuses of
 *   ps_pressure_solve: a linear solve that does not return PS_OK ends the
 *   step at once (dp_dev holds its last iterate, h_dev and rhok_dev the
 *   guesses of that Picard iteration, p_dev and wun_dev the previous one's,
 *   unset if it was the first). */
typedef struct {
    double eos_a;            /* > 0                                               */
    double eos_b;            /* >= 0                                              */
    double dt;               /* time step, > 0                                    */
    int32_t n_picard;        /* Picard iterations, 1..64                          */
    int32_t max_newton;      /* Newton solves per Picard iteration, 1..64          */
    double newton_tol;       /* relative nonlinear residual; <= 0: always          */
                             /* max_newton solves, no check (default 1e-8)         */
    double reserved[4];
    ps_solve_opts solve;     /* options of every linear solve                      */
} ps_eos_opts;

void ps_eos_opts_default(ps_eos_opts *opts);
int ps_projection_step_eos(ps_mesh *mesh, const ps_eos_opts *opts, const double *rho_dev,
                           const double *wu_dev, const double *we_dev, const double *pn_dev, double *dp_dev,
                           double *p_dev, double *wun_dev, double *h_dev, double *rhok_dev,
                           double *newton_res_host, ps_solve_info *info, void *stream);

/* ---- batched solve: many independent meshes in one persistent kernel ----
 *   meshes  [n] mesh handles of one context (distinct, coefficients set)
 *   b_dev   [n] device pointers, each [n_nodes_i] double, caller numbering
 *   x_dev   [n] device pointers, each [n_nodes_i] double (in: guess, out: sol)
 *   infos   [n] per-mesh results, may be NULL
 * Mixed precision only: every FP32 inner PCG iteration of all unconverged
 * meshes runs inside one cooperative persistent kernel (grid barriers with a
 * bounded spin), FP64 residuals and updates between epochs; the launch
 * sequence is captured in a CUDA graph when opts->graph_iters >= 0.
 * Each mesh's arithmetic and reduction order do not depend on which other
 * meshes share the batch.  Returns PS_OK if all converged, else the first
 * per-mesh error (every info filled). */
int ps_batch_solve(ps_mesh *const *meshes, int n, const double *const *b_dev,
                   double *const *x_dev, const ps_solve_opts *opts, ps_solve_info *infos,
                   void *stream);

/* ---- serving: continuous batching of solve requests ---------------------
 * A server owns a worker thread and a stream.  Cases (simulations) register a
 * mesh once; each request (one time step's solve) names a case, carries a host
 * right-hand side, and warm-starts from the case's previous solution kept on
 * the device (Section 3.4: the solution at t^n is the first guess).  Requests
 * are admitted while their workspace fits the HBM budget and a slot is free;
 * admitted requests share persistent-kernel epochs with requests already in
 * flight, and a request that converges frees its slot at the next epoch
 * boundary; with single_nodes set, requests of cases at least that large run
 * alone in the single-solve engine between epochs instead. */
typedef struct {
    int32_t max_slots;        /* requests in flight at once (0 = 64)                */
    int32_t epoch_iters;      /* inner iterations per epoch (0 = 64)                */
    size_t hbm_budget_bytes;  /* cap on workspaces of in-flight requests (0 = ctx)  */
    ps_solve_opts opts;       /* solver options for every request                   */
    int32_t single_nodes;     /* requests of cases whose mesh has at least this many
                                 nodes run alone, to convergence, in the single-solve
                                 engine (ps_pressure_solve with opts) on the worker's
                                 stream between epochs; 0 = every request batched    */
    int32_t reserved[7];
} ps_server_opts;

int ps_server_create(ps_ctx *ctx, const ps_server_opts *opts, ps_server **out);

/* Stop the worker (pending requests fail with PS_ESTATE) and free the server. */
void ps_server_destroy(ps_server *srv);

/* Register a case: mesh (coefficients set) and the initial warm start
 * (host [n_nodes] double or NULL = zeros).  *case_id receives its id. */
int ps_server_add_case(ps_server *srv, ps_mesh *mesh, const double *x0_host, int32_t *case_id);

/* Queue one solve of `case_id`.  b_host [n_nodes] double is copied before the
 * call returns.  If beta_host is not NULL ([n_elems] double) the case's beta is
 * replaced (the enthalpy drifts between time steps) before this request runs.
 * Requests of one case run in submission order. */
int ps_solve_submit(ps_server *srv, int32_t case_id, const double *b_host,
                    const double *beta_host, ps_ticket *out);

/* Poll a ticket: PS_PENDING while queued or running; otherwise the request's
 * final status, with info filled and, if x_out is not NULL, the solution copied
 * to x_out (host [n_nodes] double).  A finished ticket may be polled again
 * until ps_server_release is called for it. */
int ps_solve_poll(ps_server *srv, ps_ticket ticket, ps_solve_info *info, double *x_out);

/* Block until the ticket finishes (bounded by timeout_s seconds, <= 0 = 600). */
int ps_solve_wait(ps_server *srv, ps_ticket ticket, double timeout_s, ps_solve_info *info,
                  double *x_out);

/* Drop a finished ticket's record. */
int ps_server_release(ps_server *srv, ps_ticket ticket);

typedef struct {
    int64_t submitted, completed, failed, in_flight, queued;
    int64_t epochs;           /* persistent-kernel epochs launched                  */
    int64_t peak_in_flight;
    int64_t bytes_in_use;
    double busy_seconds;
    int64_t single_solves;    /* requests served alone by the single-solve engine   */
    int64_t reserved[3];
} ps_server_stats;

int ps_server_get_stats(ps_server *srv, ps_server_stats *out);

/* ---- host-only diagnostics ---------------------------------------------
 * Run the mesh preprocessing of ps_mesh_upload on the host (no device work)
 * and check the invariants the kernels rely on: every element vertex appears
 * exactly once in its chunk's incidence lists, chunk-interior nodes belong to
 * one chunk, partial-sum slots of shared nodes form a bijection.  Same
 * arguments as ps_mesh_upload; stats filled (device_bytes = shared memory per
 * block of the FP64 operator pass).  periodic as in ps_mesh_upload_periodic
 * (may be NULL).  PS_EINVAL for bad input, PS_ESTATE if an invariant fails
 * (ps_last_error names it). */
int ps_debug_prepare(int dim, int64_t n_nodes, const double *coords, int64_t n_elems,
                     const int32_t *conn, const uint8_t *dirichlet, const int32_t *periodic,
                     const ps_mesh_opts *opts, ps_mesh_stats *stats);

/* ---- Jacobi preconditioner of a mesh (diagnostics) ----------------------
 * Copy the inverse diagonal D^-1 that the Jacobi preconditioner applies, with
 * D_ii = sum over the elements e around node i of (M^e_ii + dt2 K^e_ii) (the
 * diagonal of the weak problem's matrix, Section 3.4; the mass term in the
 * mesh's current form), to host memory in the caller's numbering.
 *   precision  PS_F64: dinv_host is [n_nodes] double (the FP64 passes' copy);
 *              PS_F32: [n_nodes] float (the FP32 inner iterations' copy, the
 *              FP64 value rounded to nearest)
 *   stream     the diagonal is read after the work queued on this stream
 *              (coefficient updates of a projection step are stream-ordered)
 * Dirichlet nodes hold 0 (the preconditioned residual is zero there); merged
 * periodic vertices hold their unknown's value.  Synchronises the stream.
 * Errors: PS_EINVAL, PS_ESTATE (coefficients not set), PS_ECUDA. */
int ps_mesh_get_jacobi(const ps_mesh *mesh, int precision, void *dinv_host, void *stream);

/* ---- the FP32 CG operator kernel in isolation (diagnostics) --------------
 * One pass of the FP32 operator kernel of the two-kernel CG iteration (the
 * solver's dominant kernel, in the mesh's operator_kernel variant) with the
 * direction p = x: y = A x (Section 3.4's matrix, Dirichlet rows and columns
 * removed) and *pap = x^T A x as the kernel accumulates it (per element
 * p_e^T A_e p_e, double-float sums).
 *   x_dev, y_dev  device [n_nodes] float, caller numbering, must not alias
 *   pap           host double or NULL
 * Uses the mesh's solver workspace (its CG vectors are overwritten: run it
 * between solves, not during one).  Synchronises the stream.  Errors:
 * PS_EINVAL, PS_ESTATE (coefficients not set), PS_ETIMEOUT (a device wait
 * gave up), PS_ECUDA. */
int ps_debug_cg_apply(ps_mesh *mesh, const void *x_dev, void *y_dev, double *pap, void *stream);

/* ---- kernel timing (diagnostics for roofline reports) -------------------
 * Launch one internal kernel of the solver `reps` times back to back on
 * `stream` between two CUDA events recorded on that stream, and report the
 * average device time per launch in *avg_ms.  The workspace vectors are used
 * as inputs as they stand (run a solve first for meaningful data); results
 * are discarded.  which:
 *   PS_KERNEL_CG_F32     FP32 CG operator kernel: chunk staging, p = D^-1 r + beta p,
 *                        q = A p, chunk shares of p.Ap (the solver's dominant kernel)
 *   PS_KERNEL_UPDATE_F32 FP32 CG update kernel: shared-node rows, x and r update, rz, rr
 *                        (with the paired-patch kernel its blocks only store their
 *                        rz, rr shares: the halo gather sums them)
 *   PS_KERNEL_APPLY_F32  FP32 operator apply alone (chunk kernel + shared-node sums)
 *   PS_KERNEL_RESID_F64  FP64 true-residual chunk kernel
 *   PS_KERNEL_CG_F64     FP64 CG operator kernel
 *   PS_KERNEL_CG1_F32    FP32 fused one-reduction CG pass (node updates of x, r, s, p,
 *                        u = D^-1 r, w = A u, gamma, delta, rho): the whole inner
 *                        iteration of the default mixed-precision solve
 *   PS_KERNEL_HALO_F32   the paired-patch kernel's halo gather ((D^-1 r, p) of every
 *                        shared node into its chunks' slots) with, in its first block,
 *                        the sum of the update kernel's rz, rr shares and the end of
 *                        the iteration: the third kernel of that iteration (nothing
 *                        runs for the other kernel variants)
 * Errors: PS_EINVAL, PS_ESTATE (coefficients not set). */
#define PS_KERNEL_CG_F32     0
#define PS_KERNEL_UPDATE_F32 1
#define PS_KERNEL_APPLY_F32  2
#define PS_KERNEL_RESID_F64  3
#define PS_KERNEL_CG_F64     4
#define PS_KERNEL_CG1_F32    5
#define PS_KERNEL_HALO_F32   6
int ps_profile_kernel(ps_mesh *mesh, int which, int reps, void *stream, double *avg_ms);

#ifdef __cplusplus
}
#endif
#endif /* PRESSURE_H */
