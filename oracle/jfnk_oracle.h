/*
 * jfnk_oracle.h -- plain, slow FP64 CPU oracle of the cell-centred finite-volume
 * Jacobian-free Newton-Krylov method (Cardiff, Armfield, Tukovic, Batistic, 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code with the CUDA path.
 *
 * Vectors are blocked per cell, [n_cells][3] (Sec. 2.2: the residual and solution as
 * vectors of vectors).  In 2-D (plane strain, one-cell-thick meshes) the z entry of
 * every vector is ignored on input and zero on output.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form geometry, the uniform-stress patch
 * test, the 1-D Rhie-Chow stencil of App. C, the jump form of App. D, conservation,
 * second-order convergence on the manufactured solution, a brute-force finite-difference
 * Jacobian, quadratic Newton convergence, the small-strain limit and objectivity of the
 * neo-Hookean law.  GMRES and the multigrid internals are "parity unpinned" beyond the
 * properties the tests check (Krylov optimality on small dense systems, preconditioner
 * independence of the converged solution).
 */
#ifndef JFNK_ORACLE_H
#define JFNK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_DISP = 0, ORC_BC_TRAC = 1, ORC_BC_SYMM = 2, ORC_BC_EMPTY = 3 };
enum { ORC_LAW_LINEAR = 0, ORC_LAW_NEOHOOKEAN = 1, ORC_LAW_STVK = 2 };
enum { ORC_PC_NONE = 0, ORC_PC_BJACOBI = 1, ORC_PC_MG = 2 };

typedef struct orc_problem orc_problem;

typedef struct {
    int newton_its;        /* total Newton iterations over all load steps     */
    int gmres_its;         /* total GMRES (Arnoldi) iterations                */
    int residual_evals;    /* R(u) evaluations, including those inside Jv     */
    int status;            /* 0 converged, <0 failure                        */
    double final_rel_res;  /* |R| / |R0| of the last load step               */
    double hist[64];       /* |R| after each Newton iteration (first 64)     */
    int n_hist;
} orc_stats;

orc_problem* orc_create(int dim, int n_points, const double* points, int n_faces,
                        const int* face_ptr, const int* face_pts, const int* owner,
                        int n_internal, const int* neighbour, int n_cells);
void orc_destroy(orc_problem* p);
const char* orc_error(const orc_problem* p);

/* boundary faces [first_face, first_face+n) get type bc; values [n][3] (NULL = zero) */
int orc_set_patch(orc_problem* p, int first_face, int n, int bc, const double* values);
/* LINEAR: p1 = E, p2 = nu.  NEOHOOKEAN: p1 = mu, p2 = kappa (App. B). */
int orc_set_material(orc_problem* p, int law, double p1, double p2);
int orc_set_body_force(orc_problem* p, const double* fb /* [n_cells][3] per unit volume, NULL = 0 */);
void orc_set_alpha(orc_problem* p, double alpha_residual, double alpha_pc);
void orc_set_load_factor(orc_problem* p, double lambda);
int orc_prepare(orc_problem* p);   /* geometry, least-squares vectors, J~ coefficients */

/* geometry: Sf [nf][3], Cf [nf][3], V [nc], C [nc][3] (any may be NULL) */
void orc_get_geometry(const orc_problem* p, double* Sf, double* Cf, double* V, double* C);
void orc_gradient(const orc_problem* p, const double* u, double* grad /* [nc][3][3], (i,j) = d u_j / d x_i */);
void orc_traction_operator(const orc_problem* p, const double* grad, double* T /* [nc][3][3] */);
void orc_cauchy_stress(const orc_problem* p, const double* grad_cell /* [3][3] */, double* sigma /* [3][3] */);
void orc_residual(const orc_problem* p, const double* u, double* R);
/* Jv ~ (R(u + eps v) - R(u)) / eps, eps = 1e-7 (1 + |u|) / |v|; R_u may be NULL */
void orc_jv(const orc_problem* p, const double* u, const double* v, const double* R_u, double* Jv);
void orc_jtilde_apply(const orc_problem* p, const double* v, double* out);
void orc_jtilde_diag(const orc_problem* p, double* diag /* [nc] */);
void orc_bjacobi(const orc_problem* p, const double* v, double* z);

/* multigrid on -J~ (scalar, shared by the components) */
int orc_mg_setup(orc_problem* p, double theta, int max_levels, int coarse_max);  /* plain aggregation */
/* smoothed != 0: smoothed-aggregation prolongation */
int orc_mg_setup_ex(orc_problem* p, double theta, int max_levels, int coarse_max, int smoothed);
/* Jacobi sweeps before / after the coarse correction (default 1 and 1) */
void orc_mg_set_sweeps(orc_problem* p, int pre, int post);
int orc_mg_levels(const orc_problem* p, int* sizes /* [levels] or NULL */);
int orc_mg_aggregates(const orc_problem* p, int level, int* agg /* [size of level] */);
void orc_mg_vcycle(const orc_problem* p, const double* v, double* z);

/* right-preconditioned restarted GMRES(m) on J(u) x = b; x0 = 0 */
int orc_gmres(const orc_problem* p, const double* u, const double* R_u, const double* b, double* x,
              int m, double eta, int max_restarts, int pc, int* its_out, double* relres_out);
/* loose GMRES (LGMRES): restart m counts the Krylov columns plus up to kaug corrections of
 * earlier cycles kept across restarts (Sec. 4.2: 30 and 2); kaug = 0 is GMRES(m) */
int orc_lgmres(const orc_problem* p, const double* u, const double* R_u, const double* b, double* x,
               int m, int kaug, double eta, int max_restarts, int pc, int* its_out, double* relres_out);
/* Newton with backtracking line search over n_load_steps (lambda = k / n) */
int orc_newton(orc_problem* p, double* u, int n_load_steps, double rtol, double atol, int max_newton,
               int m, double eta, int pc, orc_stats* stats);
int orc_newton_ex(orc_problem* p, double* u, int n_load_steps, double rtol, double atol, int max_newton,
                  int m, int kaug, double eta, int pc, orc_stats* stats);
/* dynamics: density > 0 enables the inertia term (BDF2, from rest); set before the multigrid */
/* App. A updated-Lagrangian form (neo-Hookean, 3-D, static, no symmetry faces): on = 1 switches
 * it on (and resets to the reference configuration), 0 back to total Lagrangian.  orc_newton
 * then evaluates each load step on the configuration of the last converged one (the mesh moved
 * with the displacement); u stays the total displacement.  Every call starts from the
 * reference configuration and leaves the mesh in the final one.  Returns -1 (orc_error) for
 * unsupported problems. */
int orc_set_updated_lagrangian(orc_problem* p, int on);
void orc_ul_state(const orc_problem* p, double* F /* [nc][3][3] total deformation gradient */);
int orc_set_dynamics(orc_problem* p, double rho, double dt);
/* n_steps time steps of dt from the stored state; u returns the last displacement; probe
 * (if not NULL) receives the displacement of probe_cell after each step [n_steps][3] */
int orc_dynamic(orc_problem* p, double* u, int n_steps, double rtol, double atol, int max_newton, int m, int kaug,
                double eta, int pc, orc_stats* stats, int probe_cell, double* probe);
/* the segregated quasi-Newton method of Sec. 3.1: J~ du = -R per component by preconditioned
 * CG on -J~ to a residual reduction inner_tol (Sec. 3.2: 0.9); newton_its = outer iterations,
 * gmres_its = CG iterations */
int orc_segregated(orc_problem* p, double* u, int n_load_steps, double rtol, double atol, int max_outer,
                   double inner_tol, int max_inner, int pc, orc_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
