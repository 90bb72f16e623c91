/*
 * jfnk_oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * A literal, cell-by-cell transcription of the discretisation of Sec. 2.3 (Eqs.
 * volume_integral, divStressDiscret, stressInterp, leastSquaresGrad, RhieChow), the
 * mechanical laws of App. B (Hooke, neo-Hookean) in the total-Lagrangian form of App. A,
 * the compact-stencil approximate Jacobian of Sec. 3.1, and the Jacobian-free
 * Newton-Krylov algorithm of Sec. 3.2-3.3 (Eq. JF, right preconditioning, line search,
 * convergence tests).  Every loop visits cells and faces in the order of the input mesh;
 * nothing is fused or reordered for speed.  Where the paper is silent the reading taken
 * is stated at the function that uses it.
 *
 * Parity unpinned beyond the properties the oracle's tests check: the details of the
 * multigrid hierarchy (orc_mg_*: the aggregation is this project's reading of an algebraic
 * multigrid, not the paper's BoomerAMG; pinned only by a hand-worked aggregation, a symmetric
 * contracting V-cycle and the exact one-level solve) and the Krylov internals (orc_gmres,
 * orc_lgmres: only their end results are pinned, against dense solves).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark use this file.
 */
#include "jfnk_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

struct orc_problem {
    int dim, np, nf, ni, nc;
    double* pts;
    int *fptr, *fpts, *own, *nei;
    int* btype;     /* [nf - ni] boundary condition of each boundary face */
    double* bval;   /* [nf - ni][3] prescribed displacement or traction    */
    int *cfptr, *cf; /* faces of each cell (CSR, faces in increasing index) */
    double *Sf, *Cf, *V, *C; /* geometry */
    double* Ginv;   /* [nc][3][3] inverse of the least-squares tensor G_P */
    int law;
    double mu, lam, kappa, Kbar;
    double alpha_rc, alpha_pc;
    double* fb;     /* [nc][3] body force per unit volume */
    double load;
    int prepared;
    /* multigrid hierarchy on A = -J~ */
    int mg_levels;
    int* mg_n;          /* rows per level */
    int** mg_rowptr;    /* CSR per level (level 0 included) */
    int** mg_col;
    double** mg_val;
    int** mg_agg;       /* aggregate of each row of level l (l < levels-1) */
    int** mg_prp;       /* prolongation P_l (n_l x n_l+1) in CSR */
    int** mg_pcol;
    double** mg_pval;
    double* mg_chol;    /* dense Cholesky factor of the coarsest level */
    int mg_pre, mg_post; /* Jacobi sweeps before / after the coarse correction */
    /* dynamics (Sec. 2.3 inertia term, BDF2 of Eq. inertia2): density, time step, the
       state of the two previous time levels and the known part of the acceleration */
    int dynamic;
    double rho, dt;
    double *dyn_ut, *dyn_utm1, *dyn_vt, *dyn_vtm1, *dyn_at, *dyn_c; /* [nc][3] */
    /* updated-Lagrangian form (App. A, Eq. momentum_UL): the points of the reference mesh,
       the total deformation gradient of the last converged load step per cell and that
       step's load factor; the mesh (pts, geometry) is the last converged configuration */
    int ul;
    double* ul_pts0;  /* [np][3] */
    double* ul_F;     /* [nc][3][3], F_ij */
    double* ul_u;     /* [nc][3] displacement of the last converged step, u_n */
    double* ul_G;     /* [nc][3][3] its least-squares gradient on the updated mesh */
    char err[256];
};

/* ------------------------------------------------------------------ small helpers */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double det33(const double* A)
{
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
}
/* inverse by the adjugate; returns the determinant */
static double inv33(const double* A, double* B)
{
    double d = det33(A);
    B[0] = (A[4] * A[8] - A[5] * A[7]) / d;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / d;
    B[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / d;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    B[6] = (A[3] * A[7] - A[4] * A[6]) / d;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / d;
    return d;
}
static double vnorm(const double* a, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * a[i];
    return sqrt(s);
}
static double vdot(const double* a, const double* b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}
static void* xcalloc(size_t n, size_t s)
{
    void* p = calloc(n ? n : 1, s);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

/* ------------------------------------------------------------------ construction */
orc_problem* orc_create(int dim, int n_points, const double* points, int n_faces, const int* face_ptr,
                        const int* face_pts, const int* owner, int n_internal, const int* neighbour, int n_cells)
{
    orc_problem* p = (orc_problem*)xcalloc(1, sizeof(orc_problem));
    p->dim = dim; p->np = n_points; p->nf = n_faces; p->ni = n_internal; p->nc = n_cells;
    p->pts = (double*)xcalloc((size_t)n_points * 3, sizeof(double));
    memcpy(p->pts, points, sizeof(double) * 3 * (size_t)n_points);
    p->fptr = (int*)xcalloc((size_t)n_faces + 1, sizeof(int));
    memcpy(p->fptr, face_ptr, sizeof(int) * ((size_t)n_faces + 1));
    p->fpts = (int*)xcalloc((size_t)face_ptr[n_faces], sizeof(int));
    memcpy(p->fpts, face_pts, sizeof(int) * (size_t)face_ptr[n_faces]);
    p->own = (int*)xcalloc((size_t)n_faces, sizeof(int));
    memcpy(p->own, owner, sizeof(int) * (size_t)n_faces);
    p->nei = (int*)xcalloc((size_t)n_internal, sizeof(int));
    memcpy(p->nei, neighbour, sizeof(int) * (size_t)n_internal);
    p->btype = (int*)xcalloc((size_t)(n_faces - n_internal), sizeof(int));
    for (int b = 0; b < n_faces - n_internal; b++) p->btype[b] = ORC_BC_TRAC; /* traction-free default */
    p->bval = (double*)xcalloc((size_t)(n_faces - n_internal) * 3, sizeof(double));
    p->fb = (double*)xcalloc((size_t)n_cells * 3, sizeof(double));
    p->alpha_rc = 1.0;
    p->alpha_pc = 1.0;
    p->load = 1.0;
    p->law = ORC_LAW_LINEAR;
    return p;
}

static void mg_free(orc_problem* p)
{
    for (int l = 0; l < p->mg_levels; l++) {
        free(p->mg_rowptr[l]); free(p->mg_col[l]); free(p->mg_val[l]);
        if (p->mg_agg && p->mg_agg[l]) free(p->mg_agg[l]);
        if (p->mg_prp && p->mg_prp[l]) { free(p->mg_prp[l]); free(p->mg_pcol[l]); free(p->mg_pval[l]); }
    }
    free(p->mg_rowptr); free(p->mg_col); free(p->mg_val); free(p->mg_agg); free(p->mg_n); free(p->mg_chol);
    free(p->mg_prp); free(p->mg_pcol); free(p->mg_pval);
    p->mg_rowptr = NULL; p->mg_col = NULL; p->mg_val = NULL; p->mg_agg = NULL; p->mg_n = NULL; p->mg_chol = NULL;
    p->mg_prp = NULL; p->mg_pcol = NULL; p->mg_pval = NULL;
    p->mg_levels = 0;
}

void orc_destroy(orc_problem* p)
{
    if (!p) return;
    mg_free(p);
    free(p->pts); free(p->fptr); free(p->fpts); free(p->own); free(p->nei); free(p->btype); free(p->bval);
    free(p->cfptr); free(p->cf); free(p->Sf); free(p->Cf); free(p->V); free(p->C); free(p->Ginv); free(p->fb);
    free(p->dyn_ut); free(p->dyn_utm1); free(p->dyn_vt); free(p->dyn_vtm1); free(p->dyn_at); free(p->dyn_c);
    free(p->ul_pts0); free(p->ul_F); free(p->ul_u); free(p->ul_G);
    free(p);
}

const char* orc_error(const orc_problem* p) { return p->err; }

int orc_set_patch(orc_problem* p, int first_face, int n, int bc, const double* values)
{
    if (first_face < p->ni || first_face + n > p->nf || bc < 0 || bc > 3) {
        snprintf(p->err, sizeof p->err, "bad patch [%d, %d) type %d", first_face, first_face + n, bc);
        return -1;
    }
    for (int k = 0; k < n; k++) {
        int b = first_face - p->ni + k;
        p->btype[b] = bc;
        for (int c = 0; c < 3; c++) p->bval[3 * b + c] = values ? values[3 * k + c] : 0.0;
    }
    return 0;
}

/* App. B: mu = E / 2(1 + nu), lambda = E nu / (1 + nu)(1 - 2 nu); neo-Hookean takes mu and
 * kappa directly.  Sec. 2.3.3: Kbar = 4/3 mu + kappa = 2 mu + lambda. */
int orc_set_material(orc_problem* p, int law, double p1, double p2)
{
    p->law = law;
    if (law == ORC_LAW_LINEAR) {
        p->mu = p1 / (2.0 * (1.0 + p2));
        p->lam = p1 * p2 / ((1.0 + p2) * (1.0 - 2.0 * p2));
        p->kappa = p->lam + 2.0 * p->mu / 3.0;
    } else if (law == ORC_LAW_NEOHOOKEAN) {
        p->mu = p1;
        p->kappa = p2;
        p->lam = p->kappa - 2.0 * p->mu / 3.0;
    } else if (law == ORC_LAW_STVK) {  /* App. B: Lame parameters from E, nu as for Hooke */
        p->mu = p1 / (2.0 * (1.0 + p2));
        p->lam = p1 * p2 / ((1.0 + p2) * (1.0 - 2.0 * p2));
        p->kappa = p->lam + 2.0 * p->mu / 3.0;
    } else {
        snprintf(p->err, sizeof p->err, "unknown law %d", law);
        return -1;
    }
    p->Kbar = 4.0 * p->mu / 3.0 + p->kappa;
    return 0;
}

int orc_set_body_force(orc_problem* p, const double* fb)
{
    for (long i = 0; i < 3L * p->nc; i++) p->fb[i] = fb ? fb[i] : 0.0;
    return 0;
}

void orc_set_alpha(orc_problem* p, double alpha_residual, double alpha_pc)
{
    p->alpha_rc = alpha_residual;
    p->alpha_pc = alpha_pc;
}

void orc_set_load_factor(orc_problem* p, double lambda) { p->load = lambda; }

/* ------------------------------------------------------------------ geometry (Sec. 2.3)
 * Reading (the paper does not define the geometry of non-planar faces): each face is the
 * fan of triangles (a, p_i, p_i+1) about its point average a.  Its area vector is the sum
 * of the triangle area vectors and its centroid the area-weighted mean of the triangle
 * centroids.  Each cell is the polyhedron bounded by those triangles; its volume and
 * centroid are exact for that polyhedron, computed from tetrahedra joining each triangle
 * to the mean of the cell's face centroids. */
static void face_geometry(const orc_problem* p, int f, double* S, double* Cf)
{
    int n = p->fptr[f + 1] - p->fptr[f];
    const int* q = p->fpts + p->fptr[f];
    double a[3] = {0, 0, 0};
    for (int i = 0; i < n; i++)
        for (int c = 0; c < 3; c++) a[c] += p->pts[3 * q[i] + c] / n;
    double area = 0.0, acc[3] = {0, 0, 0};
    S[0] = S[1] = S[2] = 0.0;
    for (int i = 0; i < n; i++) {
        const double* p0 = p->pts + 3 * q[i];
        const double* p1 = p->pts + 3 * q[(i + 1) % n];
        double e0[3], e1[3], s[3];
        for (int c = 0; c < 3; c++) { e0[c] = p0[c] - a[c]; e1[c] = p1[c] - a[c]; }
        cross3(e0, e1, s);
        for (int c = 0; c < 3; c++) s[c] *= 0.5;
        double ms = norm3(s);
        for (int c = 0; c < 3; c++) {
            S[c] += s[c];
            acc[c] += ms * (a[c] + p0[c] + p1[c]) / 3.0;
        }
        area += ms;
    }
    for (int c = 0; c < 3; c++) Cf[c] = acc[c] / area;
}

static void cell_geometry(const orc_problem* p, int P, double* V, double* C)
{
    /* apex: mean of the cell's face centroids */
    double apex[3] = {0, 0, 0};
    int nfc = p->cfptr[P + 1] - p->cfptr[P];
    for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++)
        for (int c = 0; c < 3; c++) apex[c] += p->Cf[3 * p->cf[k] + c] / nfc;
    double vol = 0.0, mom[3] = {0, 0, 0};
    for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
        int f = p->cf[k];
        double sgn = (p->own[f] == P) ? 1.0 : -1.0; /* outward from P */
        int n = p->fptr[f + 1] - p->fptr[f];
        const int* q = p->fpts + p->fptr[f];
        double a[3] = {0, 0, 0};
        for (int i = 0; i < n; i++)
            for (int c = 0; c < 3; c++) a[c] += p->pts[3 * q[i] + c] / n;
        for (int i = 0; i < n; i++) {
            const double* p0 = p->pts + 3 * q[i];
            const double* p1 = p->pts + 3 * q[(i + 1) % n];
            double e0[3], e1[3], s[3], h[3];
            for (int c = 0; c < 3; c++) { e0[c] = p0[c] - a[c]; e1[c] = p1[c] - a[c]; h[c] = a[c] - apex[c]; }
            cross3(e0, e1, s);
            double tv = sgn * dot3(s, h) / 6.0; /* tetrahedron (apex, a, p0, p1) */
            vol += tv;
            for (int c = 0; c < 3; c++) mom[c] += tv * (apex[c] + a[c] + p0[c] + p1[c]) / 4.0;
        }
    }
    *V = vol;
    for (int c = 0; c < 3; c++) C[c] = mom[c] / vol;
}

static int face_is_active(const orc_problem* p, int f)
{
    return f < p->ni || p->btype[f - p->ni] != ORC_BC_EMPTY;
}

static int is_symm(const orc_problem* p, int f) { return f >= p->ni && p->btype[f - p->ni] == ORC_BC_SYMM; }

/* Symmetry face f of its owner P (Eq. symm, Eq. leastSquaresGrad, Eq. RhieChow).  Reading
 * (the paper names d_s without defining it): the mirror neighbour of P is its reflection in
 * the face plane, with value R u_P, R = I - 2 n n; so d_s = 2 delta n with delta = n . (x_f - x_P),
 * Delta_s = n, |d_s| = 2 delta.  Outward unit normal n, |Gamma| and delta. */
static void symm_geometry(const orc_problem* p, int f, double* n, double* mG, double* delta)
{
    *mG = norm3(p->Sf + 3 * f);
    for (int c = 0; c < 3; c++) n[c] = p->Sf[3 * f + c] / *mG;
    int P = p->own[f];
    double xd[3];
    for (int c = 0; c < 3; c++) xd[c] = p->Cf[3 * f + c] - p->C[3 * P + c];
    *delta = dot3(n, xd);
}

int orc_prepare(orc_problem* p)
{
    int nc = p->nc, nf = p->nf;
    for (int f = 0; f < nf; f++) {
        if (p->own[f] < 0 || p->own[f] >= nc || (f < p->ni && (p->nei[f] < 0 || p->nei[f] >= nc || p->nei[f] == p->own[f]))) {
            snprintf(p->err, sizeof p->err, "face %d has an out-of-range owner/neighbour", f);
            return -1;
        }
    }
    /* faces of each cell */
    free(p->cfptr); free(p->cf);
    p->cfptr = (int*)xcalloc((size_t)nc + 1, sizeof(int));
    for (int f = 0; f < nf; f++) {
        p->cfptr[p->own[f] + 1]++;
        if (f < p->ni) p->cfptr[p->nei[f] + 1]++;
    }
    for (int P = 0; P < nc; P++) p->cfptr[P + 1] += p->cfptr[P];
    p->cf = (int*)xcalloc((size_t)p->cfptr[nc], sizeof(int));
    int* fill = (int*)xcalloc((size_t)nc, sizeof(int));
    for (int f = 0; f < nf; f++) {
        p->cf[p->cfptr[p->own[f]] + fill[p->own[f]]++] = f;
        if (f < p->ni) p->cf[p->cfptr[p->nei[f]] + fill[p->nei[f]]++] = f;
    }
    free(fill);
    /* geometry */
    free(p->Sf); free(p->Cf); free(p->V); free(p->C); free(p->Ginv);
    p->Sf = (double*)xcalloc((size_t)nf * 3, sizeof(double));
    p->Cf = (double*)xcalloc((size_t)nf * 3, sizeof(double));
    p->V = (double*)xcalloc((size_t)nc, sizeof(double));
    p->C = (double*)xcalloc((size_t)nc * 3, sizeof(double));
    p->Ginv = (double*)xcalloc((size_t)nc * 9, sizeof(double));
    for (int f = 0; f < nf; f++) face_geometry(p, f, p->Sf + 3 * f, p->Cf + 3 * f);
    for (int P = 0; P < nc; P++) {
        cell_geometry(p, P, p->V + P, p->C + 3 * P);
        if (!(p->V[P] > 0.0)) {
            snprintf(p->err, sizeof p->err, "cell %d has non-positive volume", P);
            return -1;
        }
    }
    /* least-squares tensor G_P (Eq. leastSquaresGrad and the G_P definition after it).
     * Reading: the printed weights w (gradient) and (1 - w) (G) make the gradient exact
     * for linear fields only when w = 1/2; the paper allows w = 1/2 (after Eq.
     * stressInterp), so both sums use the weight |Gamma_f| (the common 1/2 cancels). */
    for (int P = 0; P < nc; P++) {
        double G[9] = {0};
        double scale = 0.0;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            double d[3];
            if (f >= p->ni) {
                /* traction and displacement faces are excluded; a symmetry face counts with
                   its mirror neighbour */
                if (!is_symm(p, f)) continue;
                double n[3], mGs, delta;
                symm_geometry(p, f, n, &mGs, &delta);
                for (int c = 0; c < 3; c++) d[c] = 2.0 * delta * n[c];
            } else {
                int N = (p->own[f] == P) ? p->nei[f] : p->own[f];
                for (int c = 0; c < 3; c++) d[c] = p->C[3 * N + c] - p->C[3 * P + c];
            }
            double w = norm3(p->Sf + 3 * f) / dot3(d, d);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) G[3 * i + j] += w * d[i] * d[j];
            scale += norm3(p->Sf + 3 * f);
        }
        double* Gi = p->Ginv + 9 * P;
        memset(Gi, 0, 9 * sizeof(double));
        if (p->dim == 2) {
            double det = G[0] * G[4] - G[1] * G[3];
            if (!(fabs(det) > 1e-12 * scale * scale)) {
                snprintf(p->err, sizeof p->err, "cell %d: singular least-squares tensor", P);
                return -1;
            }
            Gi[0] = G[4] / det; Gi[1] = -G[1] / det; Gi[3] = -G[3] / det; Gi[4] = G[0] / det;
        } else {
            double det = det33(G);
            if (!(fabs(det) > 1e-12 * scale * scale * scale)) {
                snprintf(p->err, sizeof p->err, "cell %d: singular least-squares tensor", P);
                return -1;
            }
            inv33(G, Gi);
        }
    }
    p->prepared = 1;
    return 0;
}

void orc_get_geometry(const orc_problem* p, double* Sf, double* Cf, double* V, double* C)
{
    if (Sf) memcpy(Sf, p->Sf, sizeof(double) * 3 * (size_t)p->nf);
    if (Cf) memcpy(Cf, p->Cf, sizeof(double) * 3 * (size_t)p->nf);
    if (V) memcpy(V, p->V, sizeof(double) * (size_t)p->nc);
    if (C) memcpy(C, p->C, sizeof(double) * 3 * (size_t)p->nc);
}

/* displacement of cell P with the plane-strain restriction applied */
static void cell_u(const orc_problem* p, const double* u, int P, double* out)
{
    out[0] = u[3 * P]; out[1] = u[3 * P + 1]; out[2] = (p->dim == 2) ? 0.0 : u[3 * P + 2];
}

/* ------------------------------------------------------------------ Eq. leastSquaresGrad
 * (grad u)_P = sum_{f internal} |Gamma_f| G_P^-1 d_f / (d_f . d_f)  (x)  (u_N - u_P),
 * entry (i, j) = d u_j / d x_i. */
void orc_gradient(const orc_problem* p, const double* u, double* grad)
{
    for (int P = 0; P < p->nc; P++) {
        double* g = grad + 9 * P;
        memset(g, 0, 9 * sizeof(double));
        double uP[3];
        cell_u(p, u, P, uP);
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            double d[3], uN[3], Gd[3], l[3];
            if (f >= p->ni) {
                if (!is_symm(p, f)) continue;
                /* mirror neighbour: value R u_P at x_P + d_s */
                double n[3], mGs, delta;
                symm_geometry(p, f, n, &mGs, &delta);
                double un = dot3(n, uP);
                for (int c = 0; c < 3; c++) {
                    d[c] = 2.0 * delta * n[c];
                    uN[c] = uP[c] - 2.0 * un * n[c];
                }
                if (p->dim == 2) uN[2] = 0.0;
            } else {
                int N = (p->own[f] == P) ? p->nei[f] : p->own[f];
                cell_u(p, u, N, uN);
                for (int c = 0; c < 3; c++) d[c] = p->C[3 * N + c] - p->C[3 * P + c];
            }
            const double* Gi = p->Ginv + 9 * P;
            for (int i = 0; i < 3; i++) Gd[i] = Gi[3 * i] * d[0] + Gi[3 * i + 1] * d[1] + Gi[3 * i + 2] * d[2];
            double coef = norm3(p->Sf + 3 * f) / dot3(d, d);
            for (int i = 0; i < 3; i++) l[i] = coef * Gd[i];
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) g[3 * i + j] += l[i] * (uN[j] - uP[j]);
        }
    }
}

/* ------------------------------------------------------------------ App. B
 * Linear elasticity (Eq. linearElastic): sigma = mu grad u + mu grad u^T + lambda tr(grad u) I.
 * Neo-Hookean (Eq. neoHook): F = I + (grad u)^T, J = det F, b = F F^T, bbar = J^-2/3 b,
 * sigma = mu/J dev(bbar) + kappa/2 (J^2 - 1)/J I. */
/* App. B neo-Hookean Cauchy stress of the deformation gradient F (J = det F):
 * sigma = mu / J dev(J^-2/3 F F^T) + kappa / 2 (J^2 - 1) / J I */
static void nh_cauchy(const orc_problem* p, const double* F, double J, double* s)
{
    double b[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += F[3 * i + k] * F[3 * j + k];
            b[3 * i + j] = acc;
        }
    double Jm23 = pow(J, -2.0 / 3.0);
    double trb = Jm23 * (b[0] + b[4] + b[8]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double bbar = Jm23 * b[3 * i + j];
            double dev = bbar - (i == j ? trb / 3.0 : 0.0);
            s[3 * i + j] = p->mu / J * dev + (i == j ? 0.5 * p->kappa * (J * J - 1.0) / J : 0.0);
        }
}

void orc_cauchy_stress(const orc_problem* p, const double* g, double* s)
{
    if (p->law == ORC_LAW_LINEAR) {
        double tr = g[0] + g[4] + g[8];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) s[3 * i + j] = p->mu * (g[3 * i + j] + g[3 * j + i]) + (i == j ? p->lam * tr : 0.0);
        return;
    }
    double F[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) F[3 * i + j] = (i == j ? 1.0 : 0.0) + g[3 * j + i];
    double J = det33(F);
    if (p->law == ORC_LAW_STVK) {
        /* App. B St. Venant-Kirchhoff: E = (grad u + grad u^T + grad u . grad u^T) / 2,
           S = 2 mu E + lambda tr(E) I, sigma = F S F^T / J (Eq. S2sigma) */
        double E[9], S[9], FS[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double gg = 0.0;
                for (int k = 0; k < 3; k++) gg += g[3 * i + k] * g[3 * j + k];
                E[3 * i + j] = 0.5 * (g[3 * i + j] + g[3 * j + i] + gg);
            }
        double trE = E[0] + E[4] + E[8];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) S[3 * i + j] = 2.0 * p->mu * E[3 * i + j] + (i == j ? p->lam * trE : 0.0);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += F[3 * i + k] * S[3 * k + j];
                FS[3 * i + j] = acc;
            }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += FS[3 * i + k] * F[3 * j + k];
                s[3 * i + j] = acc / J;
            }
        return;
    }
    nh_cauchy(p, F, J, s);
}

/* The tensor T_P whose contraction with an area vector gives the face force of cell P:
 * linear geometry (Eq. momentum_lingeom): T = sigma_s;  total Lagrangian (Eq. momentum_TL):
 * (J F^-T . n_o) . sigma = n_o . (J F^-1 . sigma), so T = J F^-1 . sigma. */
void orc_traction_operator(const orc_problem* p, const double* grad, double* T)
{
    if (p->ul) {
        /* updated Lagrangian (Eq. momentum_UL): grad is the gradient of the displacement on
           the updated mesh, so grad - G_n is that of the increment since the last converged
           step, f = I + (grad - G_n)^T, F = f F_n, and (j f^-T . n_u) . sigma =
           n_u . (j f^-1 . sigma), so T = j f^-1 . sigma(F) */
        for (int P = 0; P < p->nc; P++) {
            const double* g = grad + 9 * P;
            const double* Gn = p->ul_G + 9 * P;
            const double* Fn = p->ul_F + 9 * P;
            double f[9], fi[9], F[9], sg[9];
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) f[3 * i + j] = (i == j ? 1.0 : 0.0) + (g[3 * j + i] - Gn[3 * j + i]);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += f[3 * i + k] * Fn[3 * k + j];
                    F[3 * i + j] = acc;
                }
            nh_cauchy(p, F, det33(F), sg);
            double jf = inv33(f, fi);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += fi[3 * i + k] * sg[3 * k + j];
                    T[9 * P + 3 * i + j] = jf * acc;
                }
        }
        return;
    }
    for (int P = 0; P < p->nc; P++) {
        const double* g = grad + 9 * P;
        double s[9];
        orc_cauchy_stress(p, g, s);
        if (p->law == ORC_LAW_LINEAR) {
            memcpy(T + 9 * P, s, sizeof s);
            continue;
        }
        double F[9], Fi[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) F[3 * i + j] = (i == j ? 1.0 : 0.0) + g[3 * j + i];
        double J = inv33(F, Fi);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += Fi[3 * i + k] * s[3 * k + j];
                T[9 * P + 3 * i + j] = J * acc;
            }
    }
}

/* ------------------------------------------------------------------ the residual
 * Eq. residual (static): R_P = sum over the faces of P of the surface force
 * (Eq. divStressDiscret with face stresses from Eq. stressInterp), plus the Rhie-Chow
 * term (Eq. RhieChow), plus the body force f_b Omega_P (Eq. volume_integral).
 * Internal face of P: Gamma . T_f with T_f = w T_P + (1 - w) T_N,
 *   w = n . (x_N - x_f) / n . (x_N - x_P), plus
 *   alpha Kbar [ |Delta| (u_N - u_P) / |d| - Delta . (grad u)_f ] |Gamma|,
 *   Delta = d / (d . n), (grad u)_f interpolated like the stress.
 * Displacement face: Gamma . T_P + alpha Kbar [ |Delta| (ubar - u_P)/|d| - Delta . (grad u)_P ] |Gamma|,
 *   d from x_P to the face centroid.
 * Traction face: |Gamma| Tbar.  The load factor scales ubar, Tbar and f_b.
 * Reading: the residual keeps the paper's sign, R = surface forces + body force. */
void orc_residual(const orc_problem* p, const double* u, double* R)
{
    int nc = p->nc;
    double* grad = (double*)xcalloc((size_t)nc * 9, sizeof(double));
    double* T = (double*)xcalloc((size_t)nc * 9, sizeof(double));
    orc_gradient(p, u, grad);
    orc_traction_operator(p, grad, T);
    double aK = p->alpha_rc * p->Kbar;
    for (int P = 0; P < nc; P++) {
        double r[3] = {0, 0, 0}, uP[3];
        cell_u(p, u, P, uP);
        const double* gP = grad + 9 * P;
        const double* TP = T + 9 * P;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            if (!face_is_active(p, f)) continue;
            double sgn = (p->own[f] == P) ? 1.0 : -1.0;
            double G[3], n[3];
            for (int c = 0; c < 3; c++) G[c] = sgn * p->Sf[3 * f + c];
            double mG = norm3(G);
            for (int c = 0; c < 3; c++) n[c] = G[c] / mG;
            if (f < p->ni) {
                int N = (sgn > 0) ? p->nei[f] : p->own[f];
                double uN[3], d[3], xNf[3];
                cell_u(p, u, N, uN);
                for (int c = 0; c < 3; c++) {
                    d[c] = p->C[3 * N + c] - p->C[3 * P + c];
                    xNf[c] = p->C[3 * N + c] - p->Cf[3 * f + c];
                }
                double w = dot3(n, xNf) / dot3(n, d);
                const double* gN = grad + 9 * N;
                const double* TN = T + 9 * N;
                double Tf[9], gf[9];
                for (int i = 0; i < 9; i++) {
                    Tf[i] = w * TP[i] + (1.0 - w) * TN[i];
                    gf[i] = w * gP[i] + (1.0 - w) * gN[i];
                }
                double dn = dot3(d, n);
                double Dl[3];
                for (int c = 0; c < 3; c++) Dl[c] = d[c] / dn;
                double mD = norm3(Dl), md = norm3(d);
                for (int j = 0; j < 3; j++) {
                    double trac = 0.0, Dg = 0.0;
                    for (int i = 0; i < 3; i++) {
                        trac += G[i] * Tf[3 * i + j];
                        Dg += Dl[i] * gf[3 * i + j];
                    }
                    r[j] += trac + aK * (mD * (uN[j] - uP[j]) / md - Dg) * mG;
                }
            } else {
                int b = f - p->ni;
                if (p->btype[b] == ORC_BC_DISP) {
                    double ub[3], d[3];
                    for (int c = 0; c < 3; c++) {
                        ub[c] = p->load * p->bval[3 * b + c];
                        d[c] = p->Cf[3 * f + c] - p->C[3 * P + c];
                    }
                    if (p->dim == 2) ub[2] = 0.0;
                    double dn = dot3(d, n);
                    double Dl[3];
                    for (int c = 0; c < 3; c++) Dl[c] = d[c] / dn;
                    double mD = norm3(Dl), md = norm3(d);
                    for (int j = 0; j < 3; j++) {
                        double trac = 0.0, Dg = 0.0;
                        for (int i = 0; i < 3; i++) {
                            trac += G[i] * TP[3 * i + j];
                            Dg += Dl[i] * gP[3 * i + j];
                        }
                        r[j] += trac + aK * (mD * (ub[j] - uP[j]) / md - Dg) * mG;
                    }
                } else if (p->btype[b] == ORC_BC_TRAC) {
                    for (int j = 0; j < 3; j++) r[j] += mG * p->load * p->bval[3 * b + j];
                } else if (p->btype[b] == ORC_BC_SYMM) {
                    /* Reading of Eq. symm: the face stress is the mean of the cell's and its
                       mirror image's, T_s = (T_P + R T_P R) / 2 (the printed one-sided form
                       (I - n n) . sigma_P has no traction at all, while the text keeps the
                       normal stress); so Gamma . T_s = |Gamma| (n . T_P . n) n, and likewise
                       Delta . (grad u)_s = (n . (grad u)_P . n) n with Delta = n.  With the
                       mirror value, (R u_P - u_P) / |d| = -(n . u_P) n / delta. */
                    double ns[3], mGs, delta;
                    symm_geometry(p, f, ns, &mGs, &delta);
                    double Tnn = 0.0, Gnn = 0.0;
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++) {
                            Tnn += ns[i] * TP[3 * i + j] * ns[j];
                            Gnn += ns[i] * gP[3 * i + j] * ns[j];
                        }
                    double un = dot3(ns, uP);
                    for (int j = 0; j < 3; j++) r[j] += mGs * (Tnn - aK * (un / delta + Gnn)) * ns[j];
                }
            }
        }
        for (int j = 0; j < 3; j++) r[j] += p->load * p->fb[3 * P + j] * p->V[P];
        if (p->dynamic) {
            /* inertia (Eq. inertia): -rho Omega_P a_P with the BDF2 acceleration of
               Eq. inertia2, a_P = 9/(4 dt^2) u_P + c_P (c_P from the previous levels) */
            double k2 = 9.0 / (4.0 * p->dt * p->dt);
            for (int j = 0; j < 3; j++) r[j] -= p->rho * p->V[P] * (k2 * uP[j] + p->dyn_c[3 * P + j]);
        }
        if (p->dim == 2) r[2] = 0.0;
        for (int j = 0; j < 3; j++) R[3 * P + j] = r[j];
    }
    free(grad);
    free(T);
}

/* ------------------------------------------------------------------ Eq. JF
 * Jv ~ (R(u + eps v) - R(u)) / eps.  Reading (the paper leaves eps to PETSc):
 * eps = 1e-7 (1 + |u|_2) / |v|_2 over all unknowns; Jv = 0 when v = 0. */
void orc_jv(const orc_problem* p, const double* u, const double* v, const double* R_u, double* Jv)
{
    long n = 3L * p->nc;
    double nv = vnorm(v, n);
    if (nv == 0.0) {
        memset(Jv, 0, sizeof(double) * (size_t)n);
        return;
    }
    double eps = 1e-7 * (1.0 + vnorm(u, n)) / nv;
    double* w = (double*)xcalloc((size_t)n, sizeof(double));
    double* Rw = (double*)xcalloc((size_t)n, sizeof(double));
    double* Ru = NULL;
    for (long i = 0; i < n; i++) w[i] = u[i] + eps * v[i];
    orc_residual(p, w, Rw);
    if (!R_u) {
        Ru = (double*)xcalloc((size_t)n, sizeof(double));
        orc_residual(p, u, Ru);
        R_u = Ru;
    }
    for (long i = 0; i < n; i++) Jv[i] = (Rw[i] - R_u[i]) / eps;
    free(w); free(Rw); free(Ru);
}

/* ------------------------------------------------------------------ Sec. 3.1, approximate Jacobian
 * Static, no symmetry faces: each block is a multiple of I, one scalar matrix for all
 * components.  Off-diagonal (P, Q): alpha Kbar |Delta| |Gamma| / |d|; diagonal: minus the
 * same terms summed over the internal and displacement faces of P. */
static double face_coef(const orc_problem* p, int f, int P)
{
    double sgn = (p->own[f] == P) ? 1.0 : -1.0;
    double G[3], n[3], d[3];
    for (int c = 0; c < 3; c++) G[c] = sgn * p->Sf[3 * f + c];
    double mG = norm3(G);
    for (int c = 0; c < 3; c++) n[c] = G[c] / mG;
    if (f < p->ni) {
        int N = (sgn > 0) ? p->nei[f] : p->own[f];
        for (int c = 0; c < 3; c++) d[c] = p->C[3 * N + c] - p->C[3 * P + c];
    } else {
        for (int c = 0; c < 3; c++) d[c] = p->Cf[3 * f + c] - p->C[3 * P + c];
    }
    double dn = dot3(d, n);
    double Dl[3];
    for (int c = 0; c < 3; c++) Dl[c] = d[c] / dn;
    return p->alpha_pc * p->Kbar * norm3(Dl) * mG / norm3(d);
}

void orc_jtilde_diag(const orc_problem* p, double* diag)
{
    for (int P = 0; P < p->nc; P++) {
        double a = 0.0;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            if (f < p->ni || p->btype[f - p->ni] == ORC_BC_DISP) a -= face_coef(p, f, P);
        }
        if (p->dynamic) a -= 2.25 * p->rho * p->V[P] / (p->dt * p->dt);  /* Sec. 3.1: -(9/4) rho Omega / dt^2 */
        diag[P] = a;
    }
}

void orc_jtilde_apply(const orc_problem* p, const double* v, double* out)
{
    for (int P = 0; P < p->nc; P++) {
        double r[3] = {0, 0, 0}, vP[3];
        cell_u(p, v, P, vP);
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            if (f < p->ni) {
                int N = (p->own[f] == P) ? p->nei[f] : p->own[f];
                double c = face_coef(p, f, P), vN[3];
                cell_u(p, v, N, vN);
                for (int j = 0; j < 3; j++) r[j] += c * (vN[j] - vP[j]);
            } else if (p->btype[f - p->ni] == ORC_BC_DISP) {
                double c = face_coef(p, f, P);
                for (int j = 0; j < 3; j++) r[j] -= c * vP[j];
            } else if (p->btype[f - p->ni] == ORC_BC_SYMM) {
                /* Sec. 3.1 symmetry term: the compact part alpha Kbar |Delta| |Gamma| / |d|
                   (R v_P - v_P) = -2 c (n . v_P) n with the mirror distance (reading above) */
                double n[3], mGs, delta;
                symm_geometry(p, f, n, &mGs, &delta);
                double c = p->alpha_pc * p->Kbar * mGs / (2.0 * delta);
                double vn = dot3(n, vP);
                for (int j = 0; j < 3; j++) r[j] -= 2.0 * c * vn * n[j];
            }
        }
        if (p->dynamic)
            for (int j = 0; j < 3; j++) r[j] -= 2.25 * p->rho * p->V[P] / (p->dt * p->dt) * vP[j];
        if (p->dim == 2) r[2] = 0.0;
        for (int j = 0; j < 3; j++) out[3 * P + j] = r[j];
    }
}

/* Point-block Jacobi with the diagonal blocks of J~ (Sec. 3.1): z_P = [J~]_PP^-1 v_P.  The
 * block is the scalar diagonal times I, plus -2 c n n for each symmetry face of P. */
void orc_bjacobi(const orc_problem* p, const double* v, double* z)
{
    double* diag = (double*)xcalloc((size_t)p->nc, sizeof(double));
    orc_jtilde_diag(p, diag);
    for (int P = 0; P < p->nc; P++) {
        double B[9] = {diag[P], 0, 0, 0, diag[P], 0, 0, 0, diag[P]}, Bi[9];
        int has_symm = 0;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            if (!is_symm(p, f)) continue;
            double n[3], mGs, delta;
            symm_geometry(p, f, n, &mGs, &delta);
            double c = p->alpha_pc * p->Kbar * mGs / (2.0 * delta);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) B[3 * i + j] -= 2.0 * c * n[i] * n[j];
            has_symm = 1;
        }
        if (p->dim == 2) { B[2] = B[5] = B[6] = B[7] = 0.0; B[8] = 1.0; }
        if (!has_symm) {
            for (int j = 0; j < 3; j++) z[3 * P + j] = (p->dim == 2 && j == 2) ? 0.0 : v[3 * P + j] / diag[P];
            continue;
        }
        inv33(B, Bi);
        for (int i = 0; i < 3; i++) {
            double acc = 0.0;
            for (int j = 0; j < 3; j++) acc += Bi[3 * i + j] * v[3 * P + j];
            z[3 * P + i] = (p->dim == 2 && i == 2) ? 0.0 : acc;
        }
    }
    free(diag);
}

/* ------------------------------------------------------------------ multigrid on A = -J~
 * The paper uses HYPRE BoomerAMG (Sec. 4.2: one V-cycle per Krylov iteration, one pre- and
 * one post-smoothing sweep, interpolation with truncation).  Reading: an aggregation AMG
 * stands in for it.
 *   strength: j is strong for i if -a_ij >= theta * max_k(-a_ik) (values within a relative
 *             1e-10 count as equal, so ties do not depend on rounding);
 *   pass 1:   rows in index order; a row whose strong neighbours are all free starts an
 *             aggregate with them;
 *   pass 2:   each remaining row joins the aggregate of its strongest aggregated neighbour
 *             (lowest index among equals), else becomes a singleton;
 *   P:        piecewise constant (plain), or smoothed: P = (I - omega D^-1 A) P_tent with
 *             omega = 4 / (3 rho), rho the Gershgorin bound max_i sum_j |a_ij| / a_ii;
 *   A_c = P^T A P; coarsening stops at coarse_max rows, max_levels levels, or when a level
 *             shrinks by less than 10%;
 *   smoother: Jacobi with weight 2/3, `pre` sweeps before and `post` after the coarse
 *             correction (1 and 1 as in Sec. 4.2 unless set);
 *   coarsest: dense Cholesky.  */
#define MG_TIE 1e-10

static int mg_coarsen(int n, const int* rp, const int* col, const double* val, double theta, int* agg)
{
    for (int i = 0; i < n; i++) agg[i] = -1;
    int na = 0;
    char* strong = NULL;
    int nnz = rp[n];
    strong = (char*)xcalloc((size_t)nnz, 1);
    for (int i = 0; i < n; i++) {
        double mx = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; k++)
            if (col[k] != i && -val[k] > mx) mx = -val[k];
        for (int k = rp[i]; k < rp[i + 1]; k++)
            strong[k] = (col[k] != i && mx > 0.0 && -val[k] >= theta * mx * (1.0 - MG_TIE));
    }
    for (int i = 0; i < n; i++) {
        if (agg[i] >= 0) continue;
        int ok = 1, ns = 0;
        for (int k = rp[i]; k < rp[i + 1]; k++)
            if (strong[k]) { ns++; if (agg[col[k]] >= 0) ok = 0; }
        if (!ok || ns == 0) continue;
        agg[i] = na;
        for (int k = rp[i]; k < rp[i + 1]; k++)
            if (strong[k]) agg[col[k]] = na;
        na++;
    }
    for (int i = 0; i < n; i++) {
        if (agg[i] >= 0) continue;
        double mx = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; k++)
            if (col[k] != i && agg[col[k]] >= 0 && -val[k] > mx) mx = -val[k];
        int best = -1;
        if (mx > 0.0)
            for (int k = rp[i]; k < rp[i + 1]; k++)
                if (col[k] != i && agg[col[k]] >= 0 && -val[k] >= mx * (1.0 - MG_TIE)) { best = col[k]; break; }
        agg[i] = (best >= 0) ? agg[best] : na++;
    }
    free(strong);
    return na;
}

/* y = P^T A P for CSR A (n x n) and CSR P (n x nco), rows of the result with ascending columns */
static void galerkin(int n, const int* rp, const int* col, const double* val, int nco, const int* prp, const int* pcol,
                     const double* pval, int** crp_out, int** ccol_out, double** cval_out)
{
    /* transpose of P */
    int* tp = (int*)xcalloc((size_t)nco + 1, sizeof(int));
    for (int i = 0; i < n; i++)
        for (int k = prp[i]; k < prp[i + 1]; k++) tp[pcol[k] + 1]++;
    for (int J = 0; J < nco; J++) tp[J + 1] += tp[J];
    int* tr = (int*)xcalloc((size_t)prp[n], sizeof(int));
    double* tv = (double*)xcalloc((size_t)prp[n], sizeof(double));
    int* fill = (int*)xcalloc((size_t)nco, sizeof(int));
    for (int i = 0; i < n; i++)
        for (int k = prp[i]; k < prp[i + 1]; k++) {
            int J = pcol[k];
            tr[tp[J] + fill[J]] = i;
            tv[tp[J] + fill[J]] = pval[k];
            fill[J]++;
        }
    free(fill);
    double* acc = (double*)xcalloc((size_t)nco, sizeof(double));
    int* mark = (int*)xcalloc((size_t)nco, sizeof(int));
    int* list = (int*)xcalloc((size_t)nco, sizeof(int));
    for (int J = 0; J < nco; J++) mark[J] = -1;
    int cap_nnz = 16 * nco + 16, nnz = 0;
    int* crp = (int*)xcalloc((size_t)nco + 1, sizeof(int));
    int* ccol = (int*)xcalloc((size_t)cap_nnz, sizeof(int));
    double* cval = (double*)xcalloc((size_t)cap_nnz, sizeof(double));
    for (int I = 0; I < nco; I++) {
        int nl = 0;
        for (int t = tp[I]; t < tp[I + 1]; t++) {
            int i = tr[t];
            double pI = tv[t];
            for (int k = rp[i]; k < rp[i + 1]; k++) {
                int j = col[k];
                for (int q = prp[j]; q < prp[j + 1]; q++) {
                    int J = pcol[q];
                    if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; list[nl++] = J; }
                    acc[J] += pI * val[k] * pval[q];
                }
            }
        }
        for (int x = 1; x < nl; x++)
            for (int y = x; y > 0 && list[y - 1] > list[y]; y--) { int t = list[y]; list[y] = list[y - 1]; list[y - 1] = t; }
        if (nnz + nl > cap_nnz) {
            while (nnz + nl > cap_nnz) cap_nnz *= 2;
            ccol = (int*)realloc(ccol, sizeof(int) * (size_t)cap_nnz);
            cval = (double*)realloc(cval, sizeof(double) * (size_t)cap_nnz);
        }
        for (int x = 0; x < nl; x++) { ccol[nnz] = list[x]; cval[nnz] = acc[list[x]]; nnz++; }
        crp[I + 1] = nnz;
    }
    free(acc); free(mark); free(list); free(tp); free(tr); free(tv);
    *crp_out = crp; *ccol_out = ccol; *cval_out = cval;
}

int orc_mg_setup(orc_problem* p, double theta, int max_levels, int coarse_max)
{
    return orc_mg_setup_ex(p, theta, max_levels, coarse_max, 0);
}

void orc_mg_set_sweeps(orc_problem* p, int pre, int post)
{
    p->mg_pre = pre > 0 ? pre : 1;
    p->mg_post = post > 0 ? post : 1;
}

int orc_mg_setup_ex(orc_problem* p, double theta, int max_levels, int coarse_max, int smoothed)
{
    mg_free(p);
    if (p->mg_pre < 1) p->mg_pre = 1;
    if (p->mg_post < 1) p->mg_post = 1;
    int cap = max_levels > 0 ? max_levels : 25;
    p->mg_n = (int*)xcalloc((size_t)cap, sizeof(int));
    p->mg_rowptr = (int**)xcalloc((size_t)cap, sizeof(int*));
    p->mg_col = (int**)xcalloc((size_t)cap, sizeof(int*));
    p->mg_val = (double**)xcalloc((size_t)cap, sizeof(double*));
    p->mg_agg = (int**)xcalloc((size_t)cap, sizeof(int*));
    p->mg_prp = (int**)xcalloc((size_t)cap, sizeof(int*));
    p->mg_pcol = (int**)xcalloc((size_t)cap, sizeof(int*));
    p->mg_pval = (double**)xcalloc((size_t)cap, sizeof(double*));
    /* level 0: rows in cell order, columns ascending */
    int n = p->nc;
    int* rp = (int*)xcalloc((size_t)n + 1, sizeof(int));
    for (int P = 0; P < n; P++) {
        int cnt = 1;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) if (p->cf[k] < p->ni) cnt++;
        rp[P + 1] = rp[P] + cnt;
    }
    int* col = (int*)xcalloc((size_t)rp[n], sizeof(int));
    double* val = (double*)xcalloc((size_t)rp[n], sizeof(double));
    double* diag = (double*)xcalloc((size_t)n, sizeof(double));
    orc_jtilde_diag(p, diag);
    for (int P = 0; P < n; P++) {
        int pos = rp[P];
        col[pos] = P; val[pos] = -diag[P]; pos++;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            if (f >= p->ni) continue;
            col[pos] = (p->own[f] == P) ? p->nei[f] : p->own[f];
            val[pos] = -face_coef(p, f, P);
            pos++;
        }
        for (int a = rp[P] + 1; a < rp[P + 1]; a++)
            for (int b = a; b > rp[P] && col[b - 1] > col[b]; b--) {
                int tc = col[b]; col[b] = col[b - 1]; col[b - 1] = tc;
                double tv = val[b]; val[b] = val[b - 1]; val[b - 1] = tv;
            }
    }
    free(diag);
    int L = 0;
    p->mg_n[0] = n; p->mg_rowptr[0] = rp; p->mg_col[0] = col; p->mg_val[0] = val;
    L = 1;
    while (L < cap && p->mg_n[L - 1] > coarse_max) {
        int nf = p->mg_n[L - 1];
        const int* frp = p->mg_rowptr[L - 1];
        const int* fcol = p->mg_col[L - 1];
        const double* fval = p->mg_val[L - 1];
        int* agg = (int*)xcalloc((size_t)nf, sizeof(int));
        int nco = mg_coarsen(nf, frp, fcol, fval, theta, agg);
        if (nco > 0.9 * nf) { free(agg); break; }
        p->mg_agg[L - 1] = agg;
        /* prolongation */
        int* prp = (int*)xcalloc((size_t)nf + 1, sizeof(int));
        int* pcol;
        double* pval;
        if (!smoothed) {
            pcol = (int*)xcalloc((size_t)nf, sizeof(int));
            pval = (double*)xcalloc((size_t)nf, sizeof(double));
            for (int i = 0; i < nf; i++) { prp[i + 1] = i + 1; pcol[i] = agg[i]; pval[i] = 1.0; }
        } else {
            double rho = 0.0;
            for (int i = 0; i < nf; i++) {
                double s = 0.0, d = 0.0;
                for (int k = frp[i]; k < frp[i + 1]; k++) {
                    s += fabs(fval[k]);
                    if (fcol[k] == i) d = fval[k];
                }
                if (s / d > rho) rho = s / d;
            }
            double omega = 4.0 / (3.0 * rho);
            int cap_p = 8 * nf + 8, np = 0;
            pcol = (int*)xcalloc((size_t)cap_p, sizeof(int));
            pval = (double*)xcalloc((size_t)cap_p, sizeof(double));
            double* acc = (double*)xcalloc((size_t)nco, sizeof(double));
            int* mark = (int*)xcalloc((size_t)nco, sizeof(int));
            int* list = (int*)xcalloc((size_t)nco, sizeof(int));
            for (int J = 0; J < nco; J++) mark[J] = -1;
            for (int i = 0; i < nf; i++) {
                double d = 0.0;
                for (int k = frp[i]; k < frp[i + 1]; k++) if (fcol[k] == i) d = fval[k];
                int nl = 0;
                mark[agg[i]] = i; acc[agg[i]] = 1.0; list[nl++] = agg[i];
                for (int k = frp[i]; k < frp[i + 1]; k++) {
                    int J = agg[fcol[k]];
                    if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; list[nl++] = J; }
                    acc[J] -= omega * fval[k] / d;
                }
                for (int x = 1; x < nl; x++)
                    for (int y = x; y > 0 && list[y - 1] > list[y]; y--) { int t = list[y]; list[y] = list[y - 1]; list[y - 1] = t; }
                if (np + nl > cap_p) {
                    while (np + nl > cap_p) cap_p *= 2;
                    pcol = (int*)realloc(pcol, sizeof(int) * (size_t)cap_p);
                    pval = (double*)realloc(pval, sizeof(double) * (size_t)cap_p);
                }
                for (int x = 0; x < nl; x++) { pcol[np] = list[x]; pval[np] = acc[list[x]]; np++; }
                prp[i + 1] = np;
            }
            free(acc); free(mark); free(list);
        }
        p->mg_prp[L - 1] = prp; p->mg_pcol[L - 1] = pcol; p->mg_pval[L - 1] = pval;
        int *crp, *ccol;
        double* cval;
        galerkin(nf, frp, fcol, fval, nco, prp, pcol, pval, &crp, &ccol, &cval);
        p->mg_n[L] = nco; p->mg_rowptr[L] = crp; p->mg_col[L] = ccol; p->mg_val[L] = cval;
        L++;
    }
    p->mg_levels = L;
    /* dense Cholesky of the coarsest level */
    int nc = p->mg_n[L - 1];
    double* Ad = (double*)xcalloc((size_t)nc * nc, sizeof(double));
    for (int i = 0; i < nc; i++)
        for (int k = p->mg_rowptr[L - 1][i]; k < p->mg_rowptr[L - 1][i + 1]; k++) Ad[(size_t)i * nc + p->mg_col[L - 1][k]] = p->mg_val[L - 1][k];
    for (int j = 0; j < nc; j++) {
        double s = Ad[(size_t)j * nc + j];
        for (int k = 0; k < j; k++) s -= Ad[(size_t)j * nc + k] * Ad[(size_t)j * nc + k];
        if (!(s > 0.0)) {
            snprintf(p->err, sizeof p->err, "coarse matrix is not positive definite (row %d)", j);
            free(Ad);
            return -1;
        }
        Ad[(size_t)j * nc + j] = sqrt(s);
        for (int i = j + 1; i < nc; i++) {
            double t = Ad[(size_t)i * nc + j];
            for (int k = 0; k < j; k++) t -= Ad[(size_t)i * nc + k] * Ad[(size_t)j * nc + k];
            Ad[(size_t)i * nc + j] = t / Ad[(size_t)j * nc + j];
        }
    }
    p->mg_chol = Ad;
    return L;
}

int orc_mg_levels(const orc_problem* p, int* sizes)
{
    if (sizes)
        for (int l = 0; l < p->mg_levels; l++) sizes[l] = p->mg_n[l];
    return p->mg_levels;
}

int orc_mg_aggregates(const orc_problem* p, int level, int* agg)
{
    if (level < 0 || level >= p->mg_levels - 1) return -1;
    memcpy(agg, p->mg_agg[level], sizeof(int) * (size_t)p->mg_n[level]);
    return 0;
}

static void spmv(int n, const int* rp, const int* col, const double* val, const double* x, double* y)
{
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; k++) s += val[k] * x[col[k]];
        y[i] = s;
    }
}

static double row_diag(const int* rp, const int* col, const double* val, int i)
{
    for (int k = rp[i]; k < rp[i + 1]; k++)
        if (col[k] == i) return val[k];
    return 1.0;
}

/* one V-cycle for A x = b from x = 0 on level l */
static void vcycle(const orc_problem* p, int l, const double* b, double* x)
{
    int n = p->mg_n[l];
    const int* rp = p->mg_rowptr[l];
    const int* col = p->mg_col[l];
    const double* val = p->mg_val[l];
    if (l == p->mg_levels - 1) {
        const double* Lc = p->mg_chol;
        for (int i = 0; i < n; i++) {
            double s = b[i];
            for (int k = 0; k < i; k++) s -= Lc[(size_t)i * n + k] * x[k];
            x[i] = s / Lc[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = x[i];
            for (int k = i + 1; k < n; k++) s -= Lc[(size_t)k * n + i] * x[k];
            x[i] = s / Lc[(size_t)i * n + i];
        }
        return;
    }
    const double omega = 2.0 / 3.0;
    double* r = (double*)xcalloc((size_t)n, sizeof(double));
    /* pre-smoothing from zero */
    for (int i = 0; i < n; i++) x[i] = omega * b[i] / row_diag(rp, col, val, i);
    for (int s = 1; s < p->mg_pre; s++) {
        spmv(n, rp, col, val, x, r);
        for (int i = 0; i < n; i++) r[i] = x[i] + omega * (b[i] - r[i]) / row_diag(rp, col, val, i);
        memcpy(x, r, sizeof(double) * (size_t)n);
    }
    spmv(n, rp, col, val, x, r);
    for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
    int nco = p->mg_n[l + 1];
    double* bc = (double*)xcalloc((size_t)nco, sizeof(double));
    double* xc = (double*)xcalloc((size_t)nco, sizeof(double));
    const int* prp = p->mg_prp[l];
    const int* pcol = p->mg_pcol[l];
    const double* pval = p->mg_pval[l];
    for (int i = 0; i < n; i++)  /* b_c = P^T r */
        for (int k = prp[i]; k < prp[i + 1]; k++) bc[pcol[k]] += pval[k] * r[i];
    vcycle(p, l + 1, bc, xc);
    for (int i = 0; i < n; i++)  /* x += P x_c */
        for (int k = prp[i]; k < prp[i + 1]; k++) x[i] += pval[k] * xc[pcol[k]];
    for (int s = 0; s < p->mg_post; s++) {
        spmv(n, rp, col, val, x, r);
        for (int i = 0; i < n; i++) r[i] = x[i] + omega * (b[i] - r[i]) / row_diag(rp, col, val, i);
        memcpy(x, r, sizeof(double) * (size_t)n);
    }
    free(r); free(bc); free(xc);
}

/* z ~ J~^-1 v, componentwise: J~ = -A, so z = -Vcycle_A(v) */
void orc_mg_vcycle(const orc_problem* p, const double* v, double* z)
{
    int n = p->nc;
    double* b = (double*)xcalloc((size_t)n, sizeof(double));
    double* x = (double*)xcalloc((size_t)n, sizeof(double));
    for (int j = 0; j < 3; j++) {
        if (p->dim == 2 && j == 2) {
            for (int P = 0; P < n; P++) z[3 * P + 2] = 0.0;
            continue;
        }
        for (int P = 0; P < n; P++) b[P] = v[3 * P + j];
        vcycle(p, 0, b, x);
        for (int P = 0; P < n; P++) z[3 * P + j] = -x[P];
    }
    free(b); free(x);
}

static void apply_pc(const orc_problem* p, int pc, const double* v, double* z)
{
    long n = 3L * p->nc;
    if (pc == ORC_PC_BJACOBI) orc_bjacobi(p, v, z);
    else if (pc == ORC_PC_MG) orc_mg_vcycle(p, v, z);
    else memcpy(z, v, sizeof(double) * (size_t)n);
}

/* ------------------------------------------------------------------ Sec. 3.2, GMRES(m)
 * Right preconditioning: J P^-1 y = b, x = P^-1 y, with J P^-1 v applied as in Eq. JF with
 * the direction P^-1 v.  x0 = 0; classical Gram-Schmidt applied twice; Givens rotations;
 * stop when the rotated residual estimate is <= eta |b|; x += P^-1 (V y) at each restart. */
int orc_gmres(const orc_problem* p, const double* u, const double* R_u, const double* b, double* x,
              int m, double eta, int max_restarts, int pc, int* its_out, double* relres_out)
{
    long n = 3L * p->nc;
    double* V = (double*)xcalloc((size_t)(m + 1) * n, sizeof(double));
    double* H = (double*)xcalloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)xcalloc((size_t)m, sizeof(double));
    double* sn = (double*)xcalloc((size_t)m, sizeof(double));
    double* g = (double*)xcalloc((size_t)m + 1, sizeof(double));
    double* y = (double*)xcalloc((size_t)m, sizeof(double));
    double* h = (double*)xcalloc((size_t)m + 1, sizeof(double));
    double* w = (double*)xcalloc((size_t)n, sizeof(double));
    double* z = (double*)xcalloc((size_t)n, sizeof(double));
    memset(x, 0, sizeof(double) * (size_t)n);
    double beta0 = vnorm(b, n);
    int its = 0, status = -1;
    double rel = 0.0;
    if (beta0 == 0.0) { status = 0; goto done; }
    double target = eta * beta0;
    for (int rs = 0; rs < max_restarts; rs++) {
        /* r = b - J x */
        if (rs == 0) memcpy(w, b, sizeof(double) * (size_t)n);
        else {
            orc_jv(p, u, x, R_u, w);
            for (long i = 0; i < n; i++) w[i] = b[i] - w[i];
        }
        double beta = vnorm(w, n);
        rel = beta / beta0;
        if (beta <= target) { status = 0; break; }
        for (long i = 0; i < n; i++) V[i] = w[i] / beta;
        memset(g, 0, sizeof(double) * ((size_t)m + 1));
        memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
        g[0] = beta;
        int k = 0, conv = 0;
        for (int j = 0; j < m; j++) {
            apply_pc(p, pc, V + (size_t)j * n, z);
            orc_jv(p, u, z, R_u, w);
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i <= j; i++) h[i] = vdot(V + (size_t)i * n, w, n);
                for (int i = 0; i <= j; i++) {
                    for (long q = 0; q < n; q++) w[q] -= h[i] * V[(size_t)i * n + q];
                    H[i * m + j] += h[i];
                }
            }
            double hn = vnorm(w, n);
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (long q = 0; q < n; q++) V[(size_t)(j + 1) * n + q] = w[q] / hn;
            for (int i = 0; i < j; i++) {
                double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double r = hypot(a, bb);
            cs[j] = a / r; sn[j] = bb / r;
            H[j * m + j] = r; H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            its++;
            k = j + 1;
            rel = fabs(g[j + 1]) / beta0;
            if (fabs(g[j + 1]) <= target || hn == 0.0) { conv = 1; break; }
        }
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int q = i + 1; q < k; q++) s -= H[i * m + q] * y[q];
            y[i] = s / H[i * m + i];
        }
        memset(w, 0, sizeof(double) * (size_t)n);
        for (int i = 0; i < k; i++)
            for (long q = 0; q < n; q++) w[q] += y[i] * V[(size_t)i * n + q];
        apply_pc(p, pc, w, z);
        for (long q = 0; q < n; q++) x[q] += z[q];
        if (conv) { status = 0; break; }
    }
done:
    if (its_out) *its_out = its;
    if (relres_out) *relres_out = rel;
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(h); free(w); free(z);
    return status;
}

/* ------------------------------------------------------------------ Sec. 4.2, loose GMRES
 * The paper runs restarted GMRES in its "loose" form: a restart keeps a few extra vectors,
 * the corrections of earlier cycles (2 of them, restart 30), after Baker, Jessup and
 * Manteuffel's LGMRES.  Written from that published method:
 *   cycle i: the approximation space is K_{m-a}(J P^-1, r_i) (through P^-1 as in orc_gmres)
 *            plus the a <= kaug stored corrections z_l, whose products J z_l are stored too;
 *            the Arnoldi process runs over [P^-1 v_1 .. P^-1 v_{m-a}, z_1 .. z_a] (the images
 *            of the last a columns are the stored J z_l, no new product), the least-squares
 *            problem is the same as in GMRES, and the correction is
 *            d = P^-1 (V_{m-a} y_{1..m-a}) + sum_l y_{m-a+l} z_l;
 *   restart: r_{i+1} = b - J x_{i+1} (true residual); the newest correction is stored as
 *            z = d / |d| with J z = (r_i - r_{i+1}) / |d|; the oldest is dropped beyond kaug.
 * The total space per cycle stays m.  kaug = 0 is GMRES(m).  Newest correction first. */
int orc_lgmres(const orc_problem* p, const double* u, const double* R_u, const double* b, double* x,
               int m, int kaug, double eta, int max_restarts, int pc, int* its_out, double* relres_out)
{
    long n = 3L * p->nc;
    if (kaug < 0) kaug = 0;
    if (kaug > m - 1) kaug = m - 1;
    double* V = (double*)xcalloc((size_t)(m + 1) * n, sizeof(double));
    double* H = (double*)xcalloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)xcalloc((size_t)m, sizeof(double));
    double* sn = (double*)xcalloc((size_t)m, sizeof(double));
    double* g = (double*)xcalloc((size_t)m + 1, sizeof(double));
    double* y = (double*)xcalloc((size_t)m, sizeof(double));
    double* h = (double*)xcalloc((size_t)m + 1, sizeof(double));
    double* w = (double*)xcalloc((size_t)n, sizeof(double));
    double* z = (double*)xcalloc((size_t)n, sizeof(double));
    double* d = (double*)xcalloc((size_t)n, sizeof(double));
    double* rprev = (double*)xcalloc((size_t)n, sizeof(double));
    double* Z = (double*)xcalloc((size_t)(kaug > 0 ? kaug : 1) * n, sizeof(double));
    double* AZ = (double*)xcalloc((size_t)(kaug > 0 ? kaug : 1) * n, sizeof(double));
    int na = 0;  /* stored corrections */
    memset(x, 0, sizeof(double) * (size_t)n);
    double beta0 = vnorm(b, n);
    int its = 0, status = -1, have_d = 0;
    double rel = 0.0;
    if (beta0 == 0.0) { status = 0; goto done; }
    double target = eta * beta0;
    for (int rs = 0; rs < max_restarts; rs++) {
        /* r = b - J x */
        if (rs == 0) memcpy(w, b, sizeof(double) * (size_t)n);
        else {
            orc_jv(p, u, x, R_u, w);
            for (long i = 0; i < n; i++) w[i] = b[i] - w[i];
        }
        if (kaug > 0 && have_d) {
            double dn = vnorm(d, n);
            if (dn > 0.0) {
                for (int l = (na < kaug ? na : kaug - 1); l > 0; l--) {  /* shift older ones */
                    memcpy(Z + (size_t)l * n, Z + (size_t)(l - 1) * n, sizeof(double) * (size_t)n);
                    memcpy(AZ + (size_t)l * n, AZ + (size_t)(l - 1) * n, sizeof(double) * (size_t)n);
                }
                for (long i = 0; i < n; i++) {
                    Z[i] = d[i] / dn;
                    AZ[i] = (rprev[i] - w[i]) / dn;
                }
                if (na < kaug) na++;
            }
        }
        double beta = vnorm(w, n);
        rel = beta / beta0;
        if (beta <= target) { status = 0; break; }
        memcpy(rprev, w, sizeof(double) * (size_t)n);
        int mk = m - na;  /* Krylov columns of this cycle */
        for (long i = 0; i < n; i++) V[i] = w[i] / beta;
        memset(g, 0, sizeof(double) * ((size_t)m + 1));
        memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
        g[0] = beta;
        int k = 0, conv = 0;
        for (int j = 0; j < m; j++) {
            if (j < mk) {
                apply_pc(p, pc, V + (size_t)j * n, z);
                orc_jv(p, u, z, R_u, w);
            } else {
                memcpy(w, AZ + (size_t)(j - mk) * n, sizeof(double) * (size_t)n);
            }
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i <= j; i++) h[i] = vdot(V + (size_t)i * n, w, n);
                for (int i = 0; i <= j; i++) {
                    for (long q = 0; q < n; q++) w[q] -= h[i] * V[(size_t)i * n + q];
                    H[i * m + j] += h[i];
                }
            }
            double hn = vnorm(w, n);
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (long q = 0; q < n; q++) V[(size_t)(j + 1) * n + q] = w[q] / hn;
            for (int i = 0; i < j; i++) {
                double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double r = hypot(a, bb);
            cs[j] = a / r; sn[j] = bb / r;
            H[j * m + j] = r; H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            its++;
            k = j + 1;
            rel = fabs(g[j + 1]) / beta0;
            if (fabs(g[j + 1]) <= target || hn == 0.0) { conv = 1; break; }
        }
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int q = i + 1; q < k; q++) s -= H[i * m + q] * y[q];
            y[i] = s / H[i * m + i];
        }
        /* d = P^-1 (sum over the Krylov columns) + sum over the stored corrections */
        memset(w, 0, sizeof(double) * (size_t)n);
        for (int i = 0; i < k && i < mk; i++)
            for (long q = 0; q < n; q++) w[q] += y[i] * V[(size_t)i * n + q];
        apply_pc(p, pc, w, d);
        for (int l = 0; mk + l < k; l++)
            for (long q = 0; q < n; q++) d[q] += y[mk + l] * Z[(size_t)l * n + q];
        have_d = 1;
        for (long q = 0; q < n; q++) x[q] += d[q];
        if (conv) { status = 0; break; }
    }
done:
    if (its_out) *its_out = its;
    if (relres_out) *relres_out = rel;
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(h); free(w); free(z); free(d); free(rprev);
    free(Z); free(AZ);
    return status;
}

/* ------------------------------------------------------------------ dynamics (Sec. 2.3, 3.2)
 * Time integration of rho d2u/dt2 = div sigma + f with the BDF2 acceleration of Eq. inertia2
 * (velocity and acceleration both by the second-order backward difference), constant dt,
 * from rest (u = v = 0 at the two levels before the first step).  Each step solves the
 * momentum equation at t + dt by the Newton-Krylov method at full load, starting from the
 * transient-continuation predictor of Eq. predictor, u = u_t + dt v_t + dt^2/2 a_t; then
 * v_{t+1} = (3 u_{t+1} - 4 u_t + u_{t-1}) / (2 dt), a_{t+1} = (3 v_{t+1} - 4 v_t + v_{t-1}) / (2 dt).
 * The inertia term adds -(9/4) rho Omega / dt^2 to the diagonal of J~ (Sec. 3.1), so a
 * multigrid hierarchy is set up after orc_set_dynamics. */
int orc_set_dynamics(orc_problem* p, double rho, double dt)
{
    if (!(rho >= 0.0) || (rho > 0.0 && !(dt > 0.0))) {
        snprintf(p->err, sizeof p->err, "density must be >= 0 and dt > 0");
        return -1;
    }
    size_t n = 3 * (size_t)p->nc;
    double** bufs[6] = {&p->dyn_ut, &p->dyn_utm1, &p->dyn_vt, &p->dyn_vtm1, &p->dyn_at, &p->dyn_c};
    for (int k = 0; k < 6; k++) {
        free(*bufs[k]);
        *bufs[k] = (double*)xcalloc(n, sizeof(double));
    }
    p->rho = rho;
    p->dt = dt;
    p->dynamic = rho > 0.0;
    return 0;
}

int orc_dynamic(orc_problem* p, double* u, int n_steps, double rtol, double atol, int max_newton, int m, int kaug,
                double eta, int pc, orc_stats* st, int probe_cell, double* probe)
{
    if (!p->dynamic) {
        snprintf(p->err, sizeof p->err, "orc_dynamic needs orc_set_dynamics with a density > 0");
        return -1;
    }
    long n = 3L * p->nc;
    double dt = p->dt;
    double* vn = (double*)xcalloc((size_t)n, sizeof(double));
    orc_stats local, one;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    int status = 0;
    for (int step = 0; step < n_steps && status == 0; step++) {
        for (long i = 0; i < n; i++) {
            p->dyn_c[i] = (3.0 * (-4.0 * p->dyn_ut[i] + p->dyn_utm1[i]) / (2.0 * dt) - 4.0 * p->dyn_vt[i] + p->dyn_vtm1[i]) /
                          (2.0 * dt);
            u[i] = p->dyn_ut[i] + dt * p->dyn_vt[i] + 0.5 * dt * dt * p->dyn_at[i];
        }
        status = orc_newton_ex(p, u, 1, rtol, atol, max_newton, m, kaug, eta, pc, &one);
        st->newton_its += one.newton_its;
        st->gmres_its += one.gmres_its;
        st->residual_evals += one.residual_evals;
        st->final_rel_res = one.final_rel_res;
        if (st->n_hist < 64) st->hist[st->n_hist++] = one.final_rel_res;
        for (long i = 0; i < n; i++) {
            vn[i] = (3.0 * u[i] - 4.0 * p->dyn_ut[i] + p->dyn_utm1[i]) / (2.0 * dt);
            p->dyn_at[i] = (3.0 * vn[i] - 4.0 * p->dyn_vt[i] + p->dyn_vtm1[i]) / (2.0 * dt);
            p->dyn_utm1[i] = p->dyn_ut[i];
            p->dyn_ut[i] = u[i];
            p->dyn_vtm1[i] = p->dyn_vt[i];
            p->dyn_vt[i] = vn[i];
        }
        if (probe && probe_cell >= 0 && probe_cell < p->nc)
            for (int j = 0; j < 3; j++) probe[3 * step + j] = u[3 * probe_cell + j];
    }
    st->status = status;
    free(vn);
    return status;
}

/* ------------------------------------------------------------------ Sec. 3.1, segregated
 * The segregated solution algorithm as the paper states it: a quasi-Newton method whose
 * Jacobian is the compact-stencil J~, decoupled into one scalar system per displacement
 * component with the same matrix (no symmetry faces here): each outer iteration solves
 * J~ du = -R(u_k) component by component and sets u_{k+1} = u_k + du (the total-displacement
 * form of the paper adds J~ u_k to both sides: the same iterate).  The inner systems are
 * solved by preconditioned conjugate gradients on A = -J~ (symmetric positive definite once
 * displacement faces exist), from du = 0, until the component's residual has fallen by the
 * factor inner_tol (Sec. 3.2: 0.9 for the segregated approach).  Preconditioner: the
 * block-Jacobi diagonal of J~ or the multigrid V-cycle on A (both in their A-form, the
 * negatives of orc_bjacobi / orc_mg_vcycle).  Convergence as for Newton (Sec. 3.3).
 * stats: newton_its counts outer iterations, gmres_its the inner CG iterations. */
int orc_segregated(orc_problem* p, double* u, int n_load_steps, double rtol, double atol, int max_outer,
                   double inner_tol, int max_inner, int pc, orc_stats* st)
{
    long n = 3L * p->nc;
    int nc = p->nc;
    double* R = (double*)xcalloc((size_t)n, sizeof(double));
    double* v = (double*)xcalloc((size_t)n, sizeof(double));
    double* z = (double*)xcalloc((size_t)n, sizeof(double));
    double* r = (double*)xcalloc((size_t)nc, sizeof(double));
    double* zc = (double*)xcalloc((size_t)nc, sizeof(double));
    double* d = (double*)xcalloc((size_t)nc, sizeof(double));
    double* q = (double*)xcalloc((size_t)nc, sizeof(double));
    double* du = (double*)xcalloc((size_t)nc, sizeof(double));
    orc_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    int status = 0;
    int ncomp = (p->dim == 2) ? 2 : 3;
    if (p->dim == 2)
        for (int P = 0; P < nc; P++) u[3 * P + 2] = 0.0;
    for (int step = 1; step <= n_load_steps && status == 0; step++) {
        orc_set_load_factor(p, (double)step / n_load_steps);
        orc_residual(p, u, R);
        double r0 = vnorm(R, n), rn = r0;
        int conv = 0;
        for (int it = 0; it <= max_outer; it++) {
            if (!(rn == rn)) { status = -4; break; }
            if (rn <= fmax(atol, rtol * r0)) { conv = 1; break; }
            if (it == max_outer) break;
            for (int j = 0; j < ncomp; j++) {
                /* A du = R_j with A = -J~; r = R_j - A 0 */
                for (int P = 0; P < nc; P++) { r[P] = R[3 * P + j]; du[P] = 0.0; }
                double rr0 = sqrt(vdot(r, r, nc));
                if (rr0 == 0.0) continue;
                double rz = 0.0;
                for (int k = 0; k < max_inner; k++) {
                    /* zc = M^-1 r (A-form of the preconditioner, through the 3-component
                       routines with this component only) */
                    memset(v, 0, sizeof(double) * (size_t)n);
                    for (int P = 0; P < nc; P++) v[3 * P + j] = r[P];
                    if (pc == ORC_PC_BJACOBI) orc_bjacobi(p, v, z);
                    else if (pc == ORC_PC_MG) orc_mg_vcycle(p, v, z);
                    else memcpy(z, v, sizeof(double) * (size_t)n);
                    for (int P = 0; P < nc; P++) zc[P] = (pc == ORC_PC_NONE) ? z[3 * P + j] : -z[3 * P + j];
                    double rz_new = vdot(r, zc, nc);
                    if (k == 0) for (int P = 0; P < nc; P++) d[P] = zc[P];
                    else {
                        double beta = rz_new / rz;
                        for (int P = 0; P < nc; P++) d[P] = zc[P] + beta * d[P];
                    }
                    rz = rz_new;
                    /* q = A d = -J~ d */
                    memset(v, 0, sizeof(double) * (size_t)n);
                    for (int P = 0; P < nc; P++) v[3 * P + j] = d[P];
                    orc_jtilde_apply(p, v, z);
                    for (int P = 0; P < nc; P++) q[P] = -z[3 * P + j];
                    double alpha = rz / vdot(d, q, nc);
                    for (int P = 0; P < nc; P++) {
                        du[P] += alpha * d[P];
                        r[P] -= alpha * q[P];
                    }
                    st->gmres_its++;
                    if (sqrt(vdot(r, r, nc)) <= inner_tol * rr0) break;
                }
                for (int P = 0; P < nc; P++) u[3 * P + j] += du[P];
            }
            orc_residual(p, u, R);
            rn = vnorm(R, n);
            st->newton_its++;
            st->residual_evals++;
            if (st->n_hist < 64) st->hist[st->n_hist++] = rn;
        }
        st->final_rel_res = (r0 > 0.0) ? rn / r0 : 0.0;
        if (!conv && status == 0) status = -2;
    }
    st->status = status;
    free(R); free(v); free(z); free(r); free(zc); free(d); free(q); free(du);
    return status;
}

/* ------------------------------------------------------------------ Eq. NewtonRaphson, Sec. 3.3
 * J du = -R; u += s du with a backtracking line search.  Reading (the line search is not
 * specified): s = 1, 1/2, 1/4, ... (at most 10 halvings), accepted when
 * |R(u + s du)| <= (1 - 1e-4 s) |R(u)|.  Converged when |R| <= max(atol, rtol |R(u0)|),
 * |R(u0)| taken at the start of each load step; stol = 0. */
/* ------------------------------------------------------------------ App. A, updated Lagrangian
 * Eq. momentum_UL writes the balance on the configuration reached at the last converged load
 * step: the mesh there is the updated one (points moved with the displacement), f = I +
 * [grad (du)]^T is the relative deformation gradient of the increment du since that step
 * (gradient on the updated mesh), j = det f, and the surface force of a face is
 * (j f^-T . n_u) . sigma = n_u . (j f^-1 . sigma), sigma the Cauchy stress of the total
 * deformation F = f F_n, F_n the total deformation gradient of the last converged step.
 * Readings (the appendix gives the balance only):
 *  - the unknown stays the total displacement u = u_n + du (cell values): the gradient of du
 *    on the updated mesh is grad u - G_n, G_n the gradient of u_n on that mesh; the Rhie-Chow
 *    term of Eq. RhieChow acts on u, as in the total-Lagrangian form, with differences and
 *    gradients taken on the updated mesh (stabilising only the increment would leave the
 *    stabilisation of the earlier steps out of the balance: the two forms would then differ
 *    at first order, not by discretisation error);
 *  - j f^-1 sigma is interpolated to the faces like the total-Lagrangian operator;
 *    displacement faces prescribe the total displacement; tractions are per unit area and
 *    body forces per unit volume of the updated configuration;
 *  - after a step converges, every mesh point moves by the mean, over the cells sharing it,
 *    of the increment extrapolated from the cell centre with the cell gradient,
 *    du_P + (x_v - x_P) . (grad du)_P (exact for increments linear in space), the geometry
 *    and least-squares tensors are recomputed on the moved points, F_n <- f F_n, u_n <- u
 *    and G_n is the gradient of u_n on the moved mesh.
 * The preconditioner keeps the approximate Jacobian of the reference mesh when it is a
 * multigrid hierarchy (built once); block-Jacobi reads the current geometry.  Neo-Hookean
 * 3-D problems without symmetry faces and without inertia only. */
int orc_set_updated_lagrangian(orc_problem* p, int on)
{
    if (on) {
        if (p->law != ORC_LAW_NEOHOOKEAN || p->dim != 3 || p->dynamic) {
            snprintf(p->err, sizeof p->err, "updated Lagrangian: neo-Hookean 3-D static problems only");
            return -1;
        }
        for (int b = 0; b < p->nf - p->ni; b++)
            if (p->btype[b] == ORC_BC_SYMM) {
                snprintf(p->err, sizeof p->err, "updated Lagrangian: symmetry faces are not supported");
                return -1;
            }
        if (!p->ul_pts0) {
            p->ul_pts0 = (double*)xcalloc((size_t)p->np * 3, sizeof(double));
            memcpy(p->ul_pts0, p->pts, sizeof(double) * 3 * (size_t)p->np);
        }
        if (!p->ul_F) p->ul_F = (double*)xcalloc((size_t)p->nc * 9, sizeof(double));
        if (!p->ul_u) p->ul_u = (double*)xcalloc((size_t)p->nc * 3, sizeof(double));
        if (!p->ul_G) p->ul_G = (double*)xcalloc((size_t)p->nc * 9, sizeof(double));
    }
    /* back to the reference configuration */
    p->ul = 0;
    if (p->ul_pts0) memcpy(p->pts, p->ul_pts0, sizeof(double) * 3 * (size_t)p->np);
    if (p->ul_F)
        for (int P = 0; P < p->nc; P++)
            for (int q = 0; q < 9; q++) p->ul_F[9 * P + q] = (q % 4 == 0) ? 1.0 : 0.0;
    if (p->ul_u) memset(p->ul_u, 0, sizeof(double) * 3 * (size_t)p->nc);
    if (p->ul_G) memset(p->ul_G, 0, sizeof(double) * 9 * (size_t)p->nc);
    p->ul = on ? 1 : 0;
    return orc_prepare(p);
}

/* total deformation gradient of the last converged step, [nc][3][3] (identity before any) */
void orc_ul_state(const orc_problem* p, double* F)
{
    for (int P = 0; P < p->nc; P++)
        for (int q = 0; q < 9; q++) F[9 * P + q] = p->ul ? p->ul_F[9 * P + q] : ((q % 4 == 0) ? 1.0 : 0.0);
}

/* the end of a converged load step at displacement u: F_n <- f F_n, the points moved by the
   increment, the geometry rebuilt, u_n <- u and G_n its gradient on the moved mesh */
static int ul_advance(orc_problem* p, const double* u)
{
    int nc = p->nc, np = p->np;
    double* grad = (double*)xcalloc((size_t)nc * 9, sizeof(double));
    double* du = (double*)xcalloc((size_t)nc * 3, sizeof(double));
    orc_gradient(p, u, grad);
    for (int P = 0; P < nc; P++) {
        for (int q = 0; q < 9; q++) grad[9 * P + q] -= p->ul_G[9 * P + q];  /* gradient of the increment */
        for (int c = 0; c < 3; c++) du[3 * P + c] = u[3 * P + c] - p->ul_u[3 * P + c];
        const double* g = grad + 9 * P;
        double* Fn = p->ul_F + 9 * P;
        double f[9], F[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) f[3 * i + j] = (i == j ? 1.0 : 0.0) + g[3 * j + i];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += f[3 * i + k] * Fn[3 * k + j];
                F[3 * i + j] = acc;
            }
        memcpy(Fn, F, sizeof F);
    }
    /* point increments: mean over the cells sharing the point of du_P + (x_v - x_P) . grad du_P */
    double* dp = (double*)xcalloc((size_t)np * 3, sizeof(double));
    int* cnt = (int*)xcalloc((size_t)np, sizeof(int));
    int* mark = (int*)xcalloc((size_t)np, sizeof(int));
    for (int v = 0; v < np; v++) mark[v] = -1;
    for (int P = 0; P < nc; P++) {
        const double* g = grad + 9 * P;
        for (int k = p->cfptr[P]; k < p->cfptr[P + 1]; k++) {
            int f = p->cf[k];
            for (int q = p->fptr[f]; q < p->fptr[f + 1]; q++) {
                int v = p->fpts[q];
                if (mark[v] == P) continue;
                mark[v] = P;
                double r[3];
                for (int c = 0; c < 3; c++) r[c] = p->pts[3 * v + c] - p->C[3 * P + c];
                for (int j = 0; j < 3; j++) {
                    double e = du[3 * P + j];
                    for (int i = 0; i < 3; i++) e += r[i] * g[3 * i + j];
                    dp[3 * v + j] += e;
                }
                cnt[v]++;
            }
        }
    }
    for (int v = 0; v < np; v++)
        if (cnt[v] > 0)
            for (int c = 0; c < 3; c++) p->pts[3 * v + c] += dp[3 * v + c] / cnt[v];
    free(grad); free(du); free(dp); free(cnt); free(mark);
    if (orc_prepare(p)) return -1;
    memcpy(p->ul_u, u, sizeof(double) * 3 * (size_t)nc);
    orc_gradient(p, p->ul_u, p->ul_G);
    return 0;
}

int orc_newton(orc_problem* p, double* u, int n_load_steps, double rtol, double atol, int max_newton,
               int m, double eta, int pc, orc_stats* st)
{
    return orc_newton_ex(p, u, n_load_steps, rtol, atol, max_newton, m, 0, eta, pc, st);
}

/* as orc_newton with loose GMRES keeping kaug corrections (kaug = 0: GMRES) */
int orc_newton_ex(orc_problem* p, double* u, int n_load_steps, double rtol, double atol, int max_newton,
                  int m, int kaug, double eta, int pc, orc_stats* st)
{
    long n = 3L * p->nc;
    double* R = (double*)xcalloc((size_t)n, sizeof(double));
    double* b = (double*)xcalloc((size_t)n, sizeof(double));
    double* du = (double*)xcalloc((size_t)n, sizeof(double));
    double* ut = (double*)xcalloc((size_t)n, sizeof(double));
    double* Rt = (double*)xcalloc((size_t)n, sizeof(double));
    orc_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    int status = 0;
    if (p->dim == 2)
        for (int P = 0; P < p->nc; P++) u[3 * P + 2] = 0.0;
    /* updated Lagrangian: every solve starts from the reference configuration, with u as the
       initial guess of the first step; each converged step moves the mesh */
    if (p->ul && orc_set_updated_lagrangian(p, 1)) { free(R); free(b); free(du); free(ut); free(Rt); return -4; }
    for (int step = 1; step <= n_load_steps && status == 0; step++) {
        orc_set_load_factor(p, (double)step / n_load_steps);
        orc_residual(p, u, R);
        double r0 = vnorm(R, n), rn = r0;
        int conv = 0;
        for (int it = 0; it <= max_newton; it++) {
            if (rn <= fmax(atol, rtol * r0)) { conv = 1; break; }
            if (it == max_newton) break;
            for (long i = 0; i < n; i++) b[i] = -R[i];
            int gits = 0;
            double grel = 0;
            if (kaug > 0) orc_lgmres(p, u, R, b, du, m, kaug, eta, 100, pc, &gits, &grel);
            else orc_gmres(p, u, R, b, du, m, eta, 100, pc, &gits, &grel);
            st->gmres_its += gits;
            double s = 1.0;
            int accepted = 0;
            double rt = 0.0;
            for (int ls = 0; ls <= 10; ls++) {
                for (long i = 0; i < n; i++) ut[i] = u[i] + s * du[i];
                orc_residual(p, ut, Rt);
                rt = vnorm(Rt, n);
                if (rt <= (1.0 - 1e-4 * s) * rn) { accepted = 1; break; }
                s *= 0.5;
            }
            if (!accepted) { status = -3; break; }
            memcpy(u, ut, sizeof(double) * (size_t)n);
            memcpy(R, Rt, sizeof(double) * (size_t)n);
            rn = rt;
            st->newton_its++;
            if (st->n_hist < 64) st->hist[st->n_hist++] = rn;
        }
        st->final_rel_res = (r0 > 0.0) ? rn / r0 : 0.0;
        if (!conv && status == 0) status = -2;
        if (p->ul && status == 0 && ul_advance(p, u)) status = -4;
    }
    st->status = status;
    free(R); free(b); free(du); free(ut); free(Rt);
    return status;
}
