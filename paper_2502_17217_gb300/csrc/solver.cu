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
    // first fields of GmresDev (j, k, done, reorth, tickets, pad, eps, unorm, beta, target, inv, wn2, res, n_reorth)
    JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gd, offsetof(GmresDev, load), cudaMemcpyDeviceToHost, c->cur));
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

// One Arnoldi iteration, every kernel reading j from the device and returning at once when
// the cycle is done: z = P^-1 V_j, eps, w = u + eps z, Jv into wk, Gram-Schmidt (+ Givens),
// V_{j+1}; then the header (j, k, done, ...) is copied to pinned host memory.
static int enqueue_iteration(jfnk_ctx* c)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    const int* gate = &c->gd->done;
    int rc;
    if ((rc = pc_apply_dev(c, c->opt.pc, c->V, c->V_ld, &c->gd->j, c->V_is_float, c->z, gate))) return rc;
    if ((rc = norm_mode(c, c->z, n, 1, gate))) return rc;
    if ((rc = perturb(c, c->u, c->z, c->w, gate))) return rc;
    if ((rc = residual_gated(c, c->w, c->wk, OUT_JV, &c->gd->eps, gate))) return rc;
    if ((rc = arnoldi_orthogonalise(c, c->wk))) return rc;
    JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gd, offsetof(GmresDev, n_reorth), cudaMemcpyDeviceToHost, c->cur));
    return JFNK_OK;
}

static int capture_iteration(jfnk_ctx* c)
{
    if (c->it_graph) return JFNK_OK;
    cudaGraph_t g = nullptr;
    const int64_t before = c->launches;
    JF_CUDA(c, cudaStreamBeginCapture(c->cur, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(c);
    cudaError_t e = cudaStreamEndCapture(c->cur, &g);
    c->graph_kernels = c->launches - before;  // counted again at every replay
    c->launches = before;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return jfnk_cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->it_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->it_graph = nullptr;
        return jfnk_cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return JFNK_OK;
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
    const bool graphs = c->use_graphs && !c->prof.enabled;
    if (graphs && (rc = capture_iteration(c))) return rc;
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
        // Arnoldi iterations; at most two in flight ahead of the host's view of `done`
        for (int j = 0; j < m; j++) {
            if (j >= 2) {
                JF_CUDA(c, cudaEventSynchronize(c->it_ev[(j - 2) & 3]));
                if (((volatile GmresDev*)c->gh)->done) break;
            }
            if (graphs) {
                JF_CUDA(c, cudaGraphLaunch(c->it_graph, c->cur));
                c->launches += c->graph_kernels;
            } else if ((rc = enqueue_iteration(c))) {
                return rc;
            }
            JF_CUDA(c, cudaEventRecord(c->it_ev[j & 3], c->cur));
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
    JF_CUDA(c, cudaMemsetAsync(&c->gd->n_reorth, 0, sizeof(int), c->cur));
    for (int step = 1; step <= n_load_steps && status == JFNK_OK; step++) {
        c->load = (double)step / n_load_steps;
        if ((rc = sync_load(c))) return rc;
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
            // copies, not pointer swaps: the captured iteration graph holds these addresses
            JF_CUDA(c, cudaMemcpyAsync(c->u, c->w, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->cur));
            JF_CUDA(c, cudaMemcpyAsync(c->Ru, c->R, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->cur));
            rn = rt;
            st->newton_its++;
            if (st->n_hist < 64) st->hist[st->n_hist++] = rn;
        }
        st->final_rel_res = r0 > 0 ? rn / r0 : 0.0;
        st->final_abs_res = rn;
        if (conv) st->load_steps_done++;
    }
    if (read_header(c) == JFNK_OK) st->reorth_its = c->gh->n_reorth;
    st->status = status;
    st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

}  // namespace jfnk
