// Host orchestration of the device-resident Jacobian-free Newton-Krylov loop (Sec. 3.2-3.3).
//   gmres():  restarted right-preconditioned GMRES(m) on J(u) x = b, x0 = 0.  Each Arnoldi
//             iteration j enqueues: z = P^-1 V_j with eps = s (1 + |u|) / |z|; w = u + eps z;
//             the three residual passes ending in Jv = (R(w) - R(u)) / eps; Gram-Schmidt
//             (twice when needed); V_{j+1} = w / |w|; a Givens step.  Every scalar lives on
//             the device; the host only polls the `done` flag every few iterations.  At the
//             end of a cycle x += P^-1 (V y).
//   newton(): J du = -R per Newton iteration with inner tolerance eta (Sec. 3.2: three
//             orders), backtracking line search on |R| (s = 1, 1/2, ...; accepted when
//             |R(u + s du)| <= (1 - 1e-4 s) |R(u)|), convergence |R| <= max(atol, rtol |R(u0)|)
//             per load step with the load factor ramped k / n (Sec. 3.3).
#include <chrono>
#include <cmath>
#include <cstring>

#include "jfnk_internal.h"

namespace jfnk {

static int read_header(jfnk_ctx* c)
{
    // first fields of GmresDev (j, k, done, reorth, tickets, pad, eps, unorm, beta, target, inv, wn2, res)
    JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gd, offsetof(GmresDev, scratch), cudaMemcpyDeviceToHost, c->cur));
    JF_CUDA(c, cudaStreamSynchronize(c->cur));
    return JFNK_OK;
}

static int read_scalar(jfnk_ctx* c, const double* dev, double* out)
{
    JF_CUDA(c, cudaMemcpyAsync(c->scal_h, dev, sizeof(double), cudaMemcpyDeviceToHost, c->cur));
    JF_CUDA(c, cudaStreamSynchronize(c->cur));
    *out = c->scal_h[0];
    return JFNK_OK;
}

// Jx = (R(u + eps x) - R(u)) / eps into out (direction x, eps from |x|)
static int jv_direction(jfnk_ctx* c, const double* x, double* out)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    int rc = norm_mode(c, x, n, 1, nullptr);
    if (!rc) rc = perturb(c, c->u, x, c->w, nullptr);
    if (!rc) rc = residual(c, c->w, out, OUT_JV, &c->gd->eps);
    return rc;
}

int gmres(jfnk_ctx* c, const double* b, double* x, int* its_out, double* relres_out, int* status)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    const int m = c->opt.gmres_restart;
    const int pc = c->opt.pc;
    int its = 0;
    *status = JFNK_GMRES_STAGNATED;
    JF_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->cur));
    int rc = norm2(c, b, n, c->scal);
    if (rc) return rc;
    double beta0 = 0;
    if ((rc = read_scalar(c, c->scal, &beta0))) return rc;
    double rel = 0.0;
    if (!(beta0 > 0.0)) {
        *status = (beta0 == 0.0) ? JFNK_OK : JFNK_DIVERGED;
        if (its_out) *its_out = 0;
        if (relres_out) *relres_out = 0;
        return JFNK_OK;
    }
    const double target = c->opt.gmres_eta * beta0;
    c->scal_h[1] = target;
    JF_CUDA(c, cudaMemcpyAsync(&c->gd->target, c->scal_h + 1, sizeof(double), cudaMemcpyHostToDevice, c->cur));
    const int check = 4;
    const int* gate = &c->gd->done;
    for (int rs = 0; rs < c->opt.gmres_max_restarts; rs++) {
        // r = b - J x
        if (rs == 0) {
            JF_CUDA(c, cudaMemcpyAsync(c->wk, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->cur));
        } else {
            if ((rc = jv_direction(c, x, c->tmp))) return rc;
            if ((rc = axpby(c, n, 1.0, b, -1.0, c->tmp, c->wk))) return rc;
        }
        if ((rc = cycle_init(c, c->wk))) return rc;
        if ((rc = read_header(c))) return rc;
        rel = c->gh->beta / beta0;
        if (!(c->gh->beta == c->gh->beta)) { *status = JFNK_DIVERGED; break; }
        if (c->gh->beta <= target) { *status = JFNK_OK; break; }
        for (int j = 0; j < m; j++) {
            const void* vj = c->V_is_float ? (const void*)((const float*)c->V + (size_t)j * c->V_ld)
                                           : (const void*)(c->V + (size_t)j * c->V_ld);
            if ((rc = pc_apply_any(c, pc, vj, c->V_is_float, c->z, gate))) return rc;
            if ((rc = norm_mode(c, c->z, n, 1, gate))) return rc;
            if ((rc = perturb(c, c->u, c->z, c->w, gate))) return rc;
            if ((rc = residual_gated(c, c->w, c->wk, OUT_JV, &c->gd->eps, gate))) return rc;
            if ((rc = arnoldi_orthogonalise(c, c->wk))) return rc;
            if ((rc = arnoldi_finish_column(c, c->wk, j))) return rc;
            if ((j + 1) % check == 0 && j + 1 < m) {
                if ((rc = read_header(c))) return rc;
                if (c->gh->done) break;
            }
        }
        if ((rc = read_header(c))) return rc;
        const int k = c->gh->k;
        its += k;
        rel = c->gh->res / beta0;
        if (k > 0) {
            if ((rc = cycle_solution(c, c->tmp))) return rc;
            if ((rc = pc_apply_any(c, pc, c->tmp, 0, c->z, nullptr))) return rc;
            if ((rc = axpby(c, n, 1.0, x, 1.0, c->z, x))) return rc;
        }
        if (!(c->gh->res == c->gh->res)) { *status = JFNK_DIVERGED; break; }
        if (c->gh->res <= target) { *status = JFNK_OK; break; }
    }
    if (its_out) *its_out = its;
    if (relres_out) *relres_out = rel;
    return JFNK_OK;
}

int newton(jfnk_ctx* c, int n_load_steps, jfnk_stats* st)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    auto t0 = std::chrono::steady_clock::now();
    int status = JFNK_OK, rc;
    double rn = 0, r0 = 0;
    for (int step = 1; step <= n_load_steps && status == JFNK_OK; step++) {
        c->load = (double)step / n_load_steps;
        if ((rc = residual(c, c->u, c->Ru, OUT_R, nullptr))) return rc;
        st->residual_evals++;
        if ((rc = norm2(c, c->Ru, n, c->scal))) return rc;
        if ((rc = read_scalar(c, c->scal, &rn))) return rc;
        r0 = rn;
        bool conv = false;
        for (int it = 0;; it++) {
            if (!std::isfinite(rn)) { status = JFNK_DIVERGED; break; }
            if (rn <= std::max(c->opt.newton_atol, c->opt.newton_rtol * r0)) { conv = true; break; }
            if (it >= c->opt.newton_max_its) { status = JFNK_MAXIT; break; }
            if ((rc = axpby(c, n, -1.0, c->Ru, 0.0, c->Ru, c->bvec))) return rc;
            if ((rc = norm_mode(c, c->u, n, 2, nullptr))) return rc;
            int gits = 0, gst = 0;
            double grel = 0;
            if ((rc = gmres(c, c->bvec, c->x, &gits, &grel, &gst))) return rc;
            st->gmres_its += gits;
            st->residual_evals += gits;
            if (gst == JFNK_DIVERGED) { status = JFNK_DIVERGED; break; }
            double s = 1.0, rt = 0.0;
            bool acc = false;
            for (int ls = 0; ls <= c->opt.line_search_max; ls++) {
                if ((rc = axpby(c, n, s, c->x, 1.0, c->u, c->w))) return rc;
                if ((rc = residual(c, c->w, c->R, OUT_R, nullptr))) return rc;
                st->residual_evals++;
                if ((rc = norm2(c, c->R, n, c->scal))) return rc;
                if ((rc = read_scalar(c, c->scal, &rt))) return rc;
                if (rt <= (1.0 - 1e-4 * s) * rn) { acc = true; break; }
                s *= 0.5;
            }
            if (!acc) { status = JFNK_LS_FAILED; break; }
            std::swap(c->u, c->w);
            std::swap(c->Ru, c->R);
            rn = rt;
            st->newton_its++;
            if (st->n_hist < 64) st->hist[st->n_hist++] = rn;
        }
        st->final_rel_res = r0 > 0 ? rn / r0 : 0.0;
        st->final_abs_res = rn;
        if (conv) st->load_steps_done++;
    }
    st->status = status;
    st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

}  // namespace jfnk
