/*
 * jfnk_gb300.h -- C ABI of the GB300 (sm_103a) Jacobian-free Newton-Krylov solver for
 * cell-centred finite-volume solid mechanics (Cardiff, Armfield, Tukovic, Batistic, 2025).
 *
 * The library evaluates, on one GPU, the matrix-free momentum residual R(u) of Sec. 2.3
 * (least-squares cell gradients, face tractions from the mechanical law, Rhie-Chow
 * stabilisation, face-to-cell summation), the finite-difference Jacobian action of Eq. JF,
 * the compact-stencil preconditioner of Sec. 3.1-3.2 (block-Jacobi or an aggregation
 * multigrid V-cycle on J~), restarted right-preconditioned GMRES(m) and the Newton loop
 * with line search and load stepping of Sec. 3.2-3.3.
 *
 * Conventions shared by every call
 *  - Status: every function returns JFNK_OK (0) or a negative JFNK_E* / JFNK_* code.  No
 *    call aborts, traps or exits; jfnk_last_error() gives a message owned by the context.
 *  - Vectors (u, R, v, Jv, z) are blocked per cell as in Sec. 2.2: double [n_cells][3] in
 *    the caller's cell numbering.  In 2-D (plane strain, one-cell-thick mesh) the z entry
 *    is ignored on input and returned as zero.
 *  - mem = JFNK_MEM_HOST: host pointers, copied in and out; the call returns when the result
 *    is in the caller's buffer.  mem = JFNK_MEM_DEVICE: device pointers of the context's
 *    device, borrowed for the duration of the work enqueued on `stream` (a cudaStream_t,
 *    cudaStreamLegacy or cudaStreamPerThread included; NULL means the context's own stream);
 *    the call returns once the work is enqueued and the caller synchronises the stream (or
 *    calls jfnk_synchronize) before reading the result.  A call on another stream than the
 *    previous call's is ordered after that call's work on the device, so the previous call's
 *    stream must still exist when the next call is made.
 *  - One context is not thread-safe: calls on a context must not overlap in time (they
 *    share device scratch buffers).  Distinct contexts are independent.
 *  - Host arrays passed to set-up calls are caller-owned and copied; they may be freed on
 *    return.  The context owns every device allocation it makes.
 *  - Environment variables (defaults in brackets): JFNK_VERBOSE [unset] prints the set-up's
 *    phase times to stderr.  Read when a context is created, changing no bit of any result:
 *    JFNK_SKIP_DONE [1] (0: a batch's passes evaluate every problem's rows, also those of
 *    problems whose Krylov cycle is done) and JFNK_PDL [0] (1: programmatic dependent launch
 *    of the hot-path kernels).  Read at set-up: JFNK_MG_SELL_MIN_ROWS [65536] (coarse
 *    multigrid levels of at least this many rows, and rows of at most 64 entries, are stored
 *    in sliced-ELL form and applied one thread per row, smaller levels as CSR by lane groups;
 *    the two sum a row's entries in different orders, so the FP32 V-cycle's rounding differs).
 */
#ifndef JFNK_GB300_H
#define JFNK_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define JFNK_OK 0
#define JFNK_EINVAL (-1)      /* invalid argument or mesh                                  */
#define JFNK_ENOMEM (-2)      /* device or host allocation failed                          */
#define JFNK_ECUDA (-3)       /* a CUDA runtime call failed                                */
#define JFNK_ESTATE (-4)      /* call out of order (e.g. no mesh or material yet)          */
#define JFNK_DIVERGED (-5)    /* NaN/Inf residual                                          */
#define JFNK_MAXIT (-6)       /* Newton did not reach the tolerance in max iterations       */
#define JFNK_LS_FAILED (-7)   /* the line search found no decrease                         */
#define JFNK_GMRES_STAGNATED (-8) /* GMRES ran out of restarts (solution still returned)   */

/* ---- enumerations ---------------------------------------------------------------------- */
enum { JFNK_BC_DISP = 0, JFNK_BC_TRAC = 1, JFNK_BC_SYMM = 2, JFNK_BC_EMPTY = 3 };
enum { JFNK_LAW_LINEAR = 0, JFNK_LAW_NEOHOOKEAN = 1, JFNK_LAW_STVK = 2 };
/* App. A: the two nonlinear-geometry forms of the momentum balance */
enum { JFNK_FORM_TOTAL_LAGRANGIAN = 0, JFNK_FORM_UPDATED_LAGRANGIAN = 1 };
enum { JFNK_PC_NONE = 0, JFNK_PC_BJACOBI = 1, JFNK_PC_MG = 2 };
enum { JFNK_MEM_HOST = 0, JFNK_MEM_DEVICE = 1 };
/* FP64: everything in double.  MIXED: preconditioner (matrix, smoother, V-cycle) and the
 * Krylov basis in float; residual, the eps-difference of Jv, Arnoldi arithmetic, the
 * Hessenberg/Givens data and the Newton update stay in double. */
enum { JFNK_PREC_FP64 = 0, JFNK_PREC_MIXED = 1 };

typedef struct jfnk_options {
    int device;             /* CUDA device ordinal                                    (0)   */
    int gmres_restart;      /* m of GMRES(m), 1..64 (Sec. 4.2 uses 30)                (30)  */
    double gmres_eta;       /* inner tolerance: |r| <= eta |R(u)| (Sec. 3.2: 1e-3)    (1e-3)*/
    int gmres_max_restarts; /* restarts per Newton iteration                           (100) */
    double newton_rtol;     /* |R| <= rtol |R(u0)| per load step (Sec. 3.3)           (1e-8)*/
    double newton_atol;     /* |R| <= atol (Sec. 3.3: 1e-50)                          (1e-50)*/
    int newton_max_its;     /* Newton iterations per load step                         (50)  */
    int line_search_max;    /* halvings of s in the backtracking line search           (10)  */
    double alpha_residual;  /* Rhie-Chow alpha in R(u) (Eq. RhieChow)                  (1)   */
    double alpha_pc;        /* alpha in the approximate Jacobian J~ (Sec. 3.1)         (1)   */
    double jv_eps_scale;    /* eps = jv_eps_scale (1 + |u|) / |v| (Eq. JF)             (1e-7)*/
    int pc;                 /* JFNK_PC_*                                         (BJACOBI)   */
    int precision;          /* JFNK_PREC_*                                          (FP64)   */
    int reorth;             /* classical Gram-Schmidt: 2 once; 0 twice when the first pass
                               lowers the norm below 1/sqrt(2) of it (selective);
                               1 always twice                                          (2)   */
    int renumber;           /* 1: reverse Cuthill-McKee cell renumbering               (1)   */
    int mg_max_levels;      /* multigrid levels (Sec. 4.2: up to 25)                   (25)  */
    int mg_coarse_max;      /* rows of the coarsest (dense Cholesky) level             (2000)*/
    double mg_theta;        /* strength threshold of the aggregation                   (0.4) */
    int mg_smooth_sweeps;   /* Jacobi sweeps before and after the coarse correction    (2)   */
    int mg_smoothed;        /* 1: smoothed-aggregation prolongation, 0: piecewise constant (1) */
    int autotune;           /* 1: time the candidate launch shapes at set-up and keep the
                               fastest (jfnk_get_tuning); 0: fixed defaults            (1)   */
    int gmres_aug;          /* loose GMRES (Sec. 4.2): corrections of earlier cycles kept
                               across restarts, 0..min(8, gmres_restart - 1); each cycle
                               has gmres_restart columns in all; 0 = GMRES(m)          (2)   */
    double seg_inner_tol;   /* jfnk_solve_segregated: each component's CG stops when its
                               residual has fallen by this factor (Sec. 3.2: 0.9)     (0.9) */
    int seg_max_outer;      /* jfnk_solve_segregated: outer iterations per load step (100000) */
    int seg_max_inner;      /* jfnk_solve_segregated: CG iterations per outer one    (1000)  */
    double density;         /* kg/m^3; > 0 adds the inertia term (Sec. 2.3, BDF2) for
                               jfnk_solve_dynamic; 0 = static                          (0)   */
    double dt;              /* time step of jfnk_solve_dynamic, s (> 0 when density > 0) (0) */
    int pc_side;            /* 0: right preconditioning, GMRES on J P^-1 (P^-1 x) = b, true
                               residual norms; 1: left, GMRES on P^-1 J x = P^-1 b with
                               preconditioned norms (the paper's choice, Sec. 3.2): each
                               Arnoldi column is P^-1 (R(u + eps v) - R(u)) / eps with
                               eps = jv_eps_scale (1 + |u|) for the unit vector v   (0)   */
} jfnk_options;

typedef struct jfnk_stats {
    int newton_its;          /* Newton iterations over all load steps                       */
    int gmres_its;           /* Arnoldi iterations over the whole solve                     */
    int residual_evals;      /* R evaluations (Jv and line-search included)                 */
    int load_steps_done;     /* load steps completed                                        */
    int status;              /* JFNK_OK or the failure code                                 */
    double final_rel_res;    /* |R| / |R(u0)| at the end of the last load step              */
    double final_abs_res;    /* |R| at the end                                              */
    double solve_ms;         /* wall time of the solve on the host clock                    */
    double hist[64];         /* |R| after each Newton iteration (first 64)                  */
    int n_hist;
    int reorth_its;          /* Arnoldi iterations that needed a second Gram-Schmidt pass   */
    int jv_products;         /* Jacobian-vector products of the Krylov solves: Arnoldi
                                iterations on new directions plus one per restart residual;
                                the columns of kept corrections need none                  */
    double arnoldi_cols;     /* sum over Arnoldi iterations of the basis vectors projected out
                                (j + 1 at index j): the work of the Gram-Schmidt passes     */
    double reorth_cols;      /* the same over the iterations that repeated the projection  */
} jfnk_stats;

typedef struct jfnk_ctx jfnk_ctx;

/* ---- life cycle ------------------------------------------------------------------------ */
/* Fills *opt with the defaults listed above. */
void jfnk_default_options(jfnk_options* opt);
/* Creates a context on opt->device (opt NULL = defaults).  *out is NULL on failure. */
int jfnk_create(jfnk_ctx** out, const jfnk_options* opt);
/* Frees every device and host resource of the context; NULL is accepted. */
int jfnk_destroy(jfnk_ctx* ctx);
/* Message of the last failure on this context (never NULL; owned by the context). */
const char* jfnk_last_error(const jfnk_ctx* ctx);
/* Replaces the options (takes effect at the next set-up or solve). */
int jfnk_set_options(jfnk_ctx* ctx, const jfnk_options* opt);

/* ---- problem definition (Sec. 2.3: face-addressed polyhedral mesh, three BC types) ----- */
/* dim: 2 (plane strain, one-cell-thick mesh whose front/back faces form EMPTY patches) or 3.
 * points [n_points][3]; faces as CSR face_ptr [n_faces+1] / face_pts; the right-hand normal
 * of each face's point loop points out of its owner.  Internal faces (0..n_internal-1) have a
 * neighbour; faces n_internal..n_faces-1 are boundary faces.  Every boundary face defaults to
 * traction-free until jfnk_set_patch() says otherwise.  Errors: JFNK_EINVAL for out-of-range
 * indices, an owner equal to its neighbour, non-positive cell volumes or a singular
 * least-squares tensor (a cell without neighbours spanning dim directions). */
int jfnk_set_mesh(jfnk_ctx* ctx, int dim, int32_t n_points, const double* points, int32_t n_faces,
                  const int32_t* face_ptr, const int32_t* face_pts, const int32_t* owner,
                  int32_t n_internal, const int32_t* neighbour, int32_t n_cells);
/* Convenience builder: the structured nx x ny x nz hexahedral block whose lattice points are
 * points [(nx+1)(ny+1)(nz+1)][3], point (i, j, k) at i + (nx+1)(j + (ny+1) k), cell (i, j, k)
 * numbered i + nx (j + ny k), as a face-addressed mesh (same semantics as jfnk_set_mesh):
 * internal faces ordered by (owner, neighbour), then six boundary patches x-min, x-max,
 * y-min, y-max, z-min, z-max (jfnk_hex_patch gives their face ranges).  dim = 2 needs nz = 1
 * and makes the z patches EMPTY.  Errors: JFNK_EINVAL for sizes below 1, a null array, or
 * more faces than int32 indexing holds; then those of jfnk_set_mesh. */
int jfnk_set_mesh_hex(jfnk_ctx* ctx, int nx, int ny, int nz, const double* points, int dim);
/* First face and face count of side 0..5 (x-min, x-max, y-min, y-max, z-min, z-max) of the
 * block built by jfnk_set_mesh_hex; pure arithmetic, no context.  JFNK_EINVAL otherwise. */
int jfnk_hex_patch(int nx, int ny, int nz, int side, int32_t* first_face, int32_t* n_faces);
/* Boundary faces [first_face, first_face + n_faces) get bc_type.  values [n_faces][3]:
 * prescribed displacement (DISP) or traction per unit (reference) area (TRAC); NULL = zero.
 * SYMM faces are symmetry planes (Eq. symm: shear-free, the face acting as a mirror; values
 * ignored).  EMPTY faces are the front/back planes of 2-D meshes.  With symmetry faces the
 * block-Jacobi preconditioner uses the 3x3 diagonal blocks of J~; the multigrid hierarchy is
 * built on the scalar part of J~ (without the n n terms of those faces). */
int jfnk_set_patch(jfnk_ctx* ctx, int32_t first_face, int32_t n_faces, int bc_type, const double* values);
/* App. B.  LINEAR (small strain, Eq. momentum_lingeom): p1 = E, p2 = nu.
 * NEOHOOKEAN (total Lagrangian, Eq. momentum_TL): p1 = mu, p2 = kappa.
 * STVK (St. Venant-Kirchhoff, total Lagrangian): p1 = E, p2 = nu.  Kbar = 4/3 mu + kappa. */
int jfnk_set_material(jfnk_ctx* ctx, int law, double p1, double p2);
/* App. A, Eq. momentum_TL (default) or Eq. momentum_UL.  In the updated-Lagrangian form each
 * load step of jfnk_solve is evaluated on the configuration of the last converged one: the mesh
 * points move with the displacement after every converged step (each point by the mean, over
 * the cells sharing it, of the cell's increment extrapolated with the cell gradient), the
 * geometry, least-squares vectors and face coefficients are rebuilt from the moved points, and
 * the face force is n_u . (j f^-1 sigma) with f = I + [grad (du)]^T the relative deformation
 * gradient of the increment du on the updated mesh, j = det f, sigma the Cauchy stress of
 * F = f F_n.  The unknown stays the total displacement (u of jfnk_solve), on which the
 * Rhie-Chow term acts as in the total-Lagrangian form; tractions and body forces are per unit
 * area and volume of the updated configuration.  A multigrid preconditioner keeps the
 * hierarchy of the reference configuration; block-Jacobi uses the current one.  Every
 * jfnk_solve starts from the reference configuration (u is the first step's initial guess) and
 * leaves the context in the final one (jfnk_get_geometry then gives the deformed mesh).
 * Updated Lagrangian needs one neo-Hookean 3-D problem without symmetry faces and without
 * inertia (else JFNK_EINVAL at set-up) and the Newton-Krylov solver (jfnk_solve_segregated
 * gives JFNK_ESTATE).  Takes effect at the next set-up. */
int jfnk_set_formulation(jfnk_ctx* ctx, int formulation);
/* Body force per unit volume [n_cells][3] (host, copied), NULL = none (Eq. volume_integral). */
int jfnk_set_body_force(jfnk_ctx* ctx, const double* fb);
/* Load factor lambda multiplying prescribed displacements, tractions and body forces. */
int jfnk_set_load_factor(jfnk_ctx* ctx, double lambda);
/* Builds everything the hot path needs (renumbering, geometry, coefficients, preconditioner).
 * Called implicitly by the calls below when the problem changed. */
int jfnk_setup(jfnk_ctx* ctx);

/* ---- hot path -------------------------------------------------------------------------- */
/* R(u), Eq. residual (static), with the paper's sign (surface forces + body force). */
int jfnk_residual(jfnk_ctx* ctx, const double* u, double* R, int mem, void* stream);
/* R(u) as jfnk_residual with device pointers, but without allocating anything.  The paper
 * has no counterpart: this is a service for callers that cannot allocate device memory when
 * they need a residual (inside a stream capture, under a framework whose pool owns the
 * device, or in loops that must not take the synchronisation of cudaMalloc/cudaFree).  Its
 * scratch is one fixed device array of 2^21 doubles (16 MiB) that every GPU loading the
 * library keeps until the process exits; the mesh must fit in it: 32 + 15 n_cells +
 * 3 (internal + displacement + symmetry faces) + 3 internal faces doubles, plus 9 n_cells for
 * any law other than LINEAR (and for a batch mixing laws), else JFNK_EINVAL.  u, R: device
 * (or managed) arrays [n_cells][3] of the context's device, in the caller's numbering; other
 * pointers give JFNK_EINVAL.  The work is enqueued on `stream` (NULL = the context's stream)
 * and the call never waits on the host; the current load factor is passed to the GPU by
 * value, so work recorded from the call (a captured graph) keeps that factor.  The context
 * must be set up already (jfnk_setup or an earlier call), else JFNK_ESTATE: this call never
 * sets up.  All calls share the array and it keeps the last call's contents (each call
 * writes everything it reads); calls that overlap on the GPU race, so serialise them.  The
 * first call on a device looks up the array's address with that device current; make it
 * before any stream capture. */
int jfnk_residual_noalloc(jfnk_ctx* ctx, const double* u, double* R, void* stream);
/* Jv ~ (R(u + eps v) - R(u)) / eps, eps = jv_eps_scale (1 + |u|_2) / |v|_2; Jv = 0 for v = 0
 * (Eq. JF).  Evaluates R(u) too. */
int jfnk_jv(jfnk_ctx* ctx, const double* u, const double* v, double* Jv, int mem, void* stream);
/* z ~ P^-1 v with P = J~ (Sec. 3.2), i.e. J~ z ~ v: JFNK_PC_BJACOBI (diagonal blocks of J~),
 * JFNK_PC_MG (one V-cycle; a mesh of at most opt.mg_coarse_max cells has a one-level
 * hierarchy, and the V-cycle is then the exact solve with J~), JFNK_PC_NONE (copy).
 * Precision follows opt.precision.  JFNK_ESTATE for JFNK_PC_MG when the context was set up
 * with another opt.pc (the hierarchy is built at set-up only for opt.pc = JFNK_PC_MG). */
int jfnk_precondition(jfnk_ctx* ctx, const double* v, double* z, int pc, int mem, void* stream);
/* Newton solve (Sec. 3.2-3.3): u holds the initial guess on entry and the solution on exit;
 * n_load_steps >= 1 ramps the load factor k / n_load_steps.  Returns JFNK_OK when every load
 * step met |R| <= max(atol, rtol |R(u0)|), else the failure code (u holds the last iterate).
 * For a batch every problem runs its own Newton loop; stats aggregates them (maximum Newton
 * count, summed Krylov counts, worst status and relative residual) and jfnk_batch_stats
 * gives each one.  The call synchronises the stream before returning. */
int jfnk_solve(jfnk_ctx* ctx, double* u, int mem, int n_load_steps, jfnk_stats* stats, void* stream);
/* The segregated quasi-Newton solve of Sec. 3.1, the method the paper compares with: per outer
 * iteration J~ du = -R(u) is solved component by component by preconditioned conjugate
 * gradients on -J~ (preconditioner opt.pc, the same block-Jacobi / multigrid) until each
 * component's residual has fallen by opt.seg_inner_tol, then u += du; convergence, load
 * steps, arguments, errors and batching as jfnk_solve.  stats.newton_its counts outer
 * iterations, stats.gmres_its the conjugate-gradient iterations (all components). */
int jfnk_solve_segregated(jfnk_ctx* ctx, double* u, int mem, int n_load_steps, jfnk_stats* stats, void* stream);
/* Time integration (options.density > 0, options.dt): n_steps steps of dt from the context's
 * state (at rest after jfnk_setup or jfnk_dynamic_reset; the state persists between calls, so
 * calls continue the motion).  Each step predicts u = u_t + dt v_t + dt^2/2 a_t (Eq. predictor)
 * and solves the momentum equation with the BDF2 inertia term of Eq. inertia2 at full load by
 * the Newton-Krylov method (method 0, options as jfnk_solve) or the segregated method of
 * Sec. 3.1 (method 1, as jfnk_solve_segregated), then updates velocity and acceleration by
 * BDF2.  u (host or device per mem, [n_cells][3], caller order) receives the displacement
 * after the last completed step; probe (host, [n_steps][3], or NULL) the displacement of cell
 * probe_cell (caller numbering) after each completed step.  stats sums the steps (newton_its,
 * gmres_its, ...), load_steps_done counts completed steps.  JFNK_ESTATE for a static context,
 * JFNK_EINVAL for bad arguments; a failed step stops the run with its status. */
int jfnk_solve_dynamic(jfnk_ctx* ctx, double* u, int mem, int n_steps, int32_t probe_cell, double* probe,
                       int method, jfnk_stats* stats, void* stream);
/* Puts the time-integration state back at rest (u = v = a = 0 at both previous levels). */
int jfnk_dynamic_reset(jfnk_ctx* ctx);
/* Checkpoint and restart of the time integration: the state that jfnk_solve_dynamic carries
 * between calls, five fields u_t, u_{t-1}, v_t, v_{t-1}, a_t, each [n_cells][3] in the caller's
 * cell order, as one host array state[5][n_cells][3].  get copies the context's state out, set
 * replaces it (same mesh and options: a context restarted from a checkpoint continues the
 * motion exactly as the one that wrote it).  Both wait for the copies.  JFNK_ESTATE before
 * set-up or for a static context (options.density = 0), JFNK_EINVAL for a null array. */
int jfnk_dynamic_get_state(jfnk_ctx* ctx, double* state);
int jfnk_dynamic_set_state(jfnk_ctx* ctx, const double* state);

/* ---- batches of independent problems in one index space -------------------------------- */
/* A context becomes a batch when problems are added to it instead of calling jfnk_set_mesh.
 * Each problem is defined in its own context (jfnk_set_mesh, jfnk_set_patch,
 * jfnk_set_material, jfnk_set_body_force; no set-up needed) and copied in; that context may be
 * destroyed afterwards.  The batch's cells are the problems' cells concatenated in the order
 * added, so every vector passed to jfnk_residual / jfnk_jv / jfnk_precondition / jfnk_solve on
 * the batch is [sum of n_cells][3].  All problems share the options, dimension, load factor
 * and load-step schedule; each keeps its own material, body force, Jv step eps, GMRES
 * iteration, line search and convergence test, so a problem's iterates do not depend on the
 * other problems except through the multigrid hierarchy, whose coarsest levels are built for
 * the whole batch.  *index receives the problem's position.  Errors: JFNK_ESTATE if the
 * context already holds a single mesh or the problem has no mesh/material; JFNK_EINVAL if the
 * dimensions differ. */
int jfnk_batch_add(jfnk_ctx* batch, const jfnk_ctx* problem, int32_t* index);
/* Number of problems (1 for a single-mesh context). */
int jfnk_batch_size(const jfnk_ctx* ctx);
/* First cell (in the concatenated numbering) and cell count of problem `index`. */
int jfnk_batch_problem_cells(const jfnk_ctx* ctx, int32_t index, int32_t* first_cell, int32_t* n_cells);
/* Per-problem statistics of the last jfnk_solve: per_problem [jfnk_batch_size(ctx)]. */
int jfnk_batch_stats(const jfnk_ctx* ctx, jfnk_stats* per_problem);

/* ---- inspection ------------------------------------------------------------------------ */
/* Geometry in the caller's numbering (host arrays, any may be NULL): face area vectors
 * Sf [n_faces][3] and centroids Cf [n_faces][3] (orientation of the input mesh), cell
 * volumes V [n_cells] and centroids C [n_cells][3]. */
int jfnk_get_geometry(jfnk_ctx* ctx, double* Sf, double* Cf, double* V, double* C);
/* Cell gradient (grad u)_P [n_cells][3][3], entry (i, j) = d u_j / d x_i, of the last R
 * evaluated (host array). */
int jfnk_get_gradient(jfnk_ctx* ctx, double* grad);
/* Internal cell order: new_to_old[n_cells] (host array). */
int jfnk_get_permutation(jfnk_ctx* ctx, int32_t* new_to_old);
/* Kernel timing: enable = 1 brackets every launch of the residual passes ("grad", "flux",
 * "finish"), the Gram-Schmidt kernels ("mdot", "update") and each preconditioner application
 * ("pc_mg", "pc_bjacobi") with CUDA events (the solver then launches kernels directly instead
 * of replaying its iteration graph); 2 also brackets the steps inside each V-cycle
 * ("mg_smooth", "mg_resid", "mg_restrict", "mg_prolong", "mg_coarse"), whose own events add to
 * "pc_mg"; 0 turns timing off. */
int jfnk_profile_enable(jfnk_ctx* ctx, int enable);
/* Accumulated time (ms) and launch count of kernel `name` since the last reset; returns
 * JFNK_EINVAL for unknown names.  Synchronises the context's last stream. */
int jfnk_profile_get(jfnk_ctx* ctx, const char* name, double* total_ms, int64_t* launches);
int jfnk_profile_reset(jfnk_ctx* ctx);
/* Waits until the work of the context's last call has finished (that call's stream; the
 * context's own stream after calls made with stream = NULL).  JFNK_ECUDA if that work failed. */
int jfnk_synchronize(jfnk_ctx* ctx);
/* Number of kernel launches made by the context since creation (every stream). */
int64_t jfnk_launch_count(const jfnk_ctx* ctx);
/* Device bytes held by the context. */
int64_t jfnk_device_bytes(const jfnk_ctx* ctx);
/* Launch shapes of the hot-path kernels (no counterpart in the paper: a property of this
 * implementation).  out[0..6): cells per block of the gradient pass {64,128,256}, faces per
 * block of the face pass {128,256}, 1 if that pass stages its owner cells' gradients in
 * shared memory, cells per block of the cell-sum pass {128,256,512}, rows per block of the
 * fine-level multigrid kernels {128,256,512}, 1 if chosen by the autotuner at jfnk_setup
 * (else the defaults 128, 256, 0, 256, 256).  n >= 6, else JFNK_EINVAL.  Results never depend
 * on the shapes, only the timing. */
int jfnk_get_tuning(jfnk_ctx* ctx, int32_t* out, int n);
/* Sets the five shapes of jfnk_get_tuning (in[0..5), n >= 5), replacing the autotuner's
 * choice until the next set-up; JFNK_EINVAL (nothing changed) for a value outside the
 * candidate sets.  Both calls run a pending set-up first (its errors are returned). */
int jfnk_set_tuning(jfnk_ctx* ctx, const int32_t* in, int n);
/* The multigrid hierarchy built at set-up (Sec. 3.2 and 4.2: one V-cycle per Krylov iteration
 * applies it): for level l < min(levels, max_levels), rows[l] = unknowns per displacement
 * component, nnz_a[l] = entries of that level's operator (off-diagonal entries plus one diagonal
 * per row; the finest level's are the J~ face couplings, 2 per internal face), nnz_p[l] =
 * entries of the prolongation from level l + 1 to level l (0 on the coarsest level, which is
 * solved by a dense inverse).  Host arrays of max_levels entries, any of them NULL.  Returns the
 * number of levels (0 when the context was set up without opt.pc = JFNK_PC_MG), or a negative
 * status (JFNK_EINVAL for max_levels < 0; set-up errors of a pending set-up). */
int jfnk_mg_hierarchy(jfnk_ctx* ctx, int max_levels, int64_t* rows, int64_t* nnz_a, int64_t* nnz_p);
/* Measured FP64 FMA throughput of `device` (TFLOP/s, an FMA counted as 2 flops): a full grid
 * of independent FMA chains timed with CUDA events (allocates and frees a small buffer).  The
 * residual and Arnoldi kernels are bound by this rate on GB300. */
int jfnk_measure_fp64_rate(int device, double* tflops);
/* The float -> double conversion the FP32 Krylov basis is read through (integer operations,
 * so it does not occupy the narrow FP64 pipe): out[i] = in[i] exactly for normal floats and
 * zeros; float subnormals give zero; Inf/NaN give NaN.  in/out are device arrays of n
 * elements; the work is enqueued on `stream` (a cudaStream_t, NULL = legacy default). */
int jfnk_convert_f32_to_f64(const float* in, double* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif
