// Host orchestration of the device-resident Jacobian-free Newton-Krylov loop (Sec. 3.2-3.3)
// for P >= 1 independent problems advancing together.
//   gmres():  restarted preconditioned GMRES(m) on J_p(u_p) x_p = b_p for every active
//             problem, x0 = 0.  Right preconditioning (Eq. JF with P^-1): one Arnoldi
//             iteration enqueues z = P^-1 V_j; eps_p = s (1 + |u_p|) / |z_p|; w = u + eps z;
//             the three residual passes ending in Jv = (R(w) - R(u)) / eps_p; Gram-Schmidt
//             with each problem's Givens step; V_{j+1} = w / |w|; at the end of a cycle
//             x += P^-1 (V y).  Left preconditioning (the form of Sec. 3.2 the paper used):
//             w = u + eps V_j with eps_p = s (1 + |u_p|) (V_j has unit norm), the residual
//             passes, z = P^-1 Jv, Gram-Schmidt on z; the cycle starts from P^-1 (b - J x),
//             norms and the tolerance are the preconditioned ones, and x += V y.  The
//             iteration is captured once as a CUDA graph and replayed; every scalar lives on
//             the device and the host keeps two iterations in flight ahead of its view of the
//             `all done` flag.
//   newton(): per problem, J du = -R with inner tolerance eta (Sec. 3.2: three orders), a
//             backtracking line search on |R_p| (s = 1, 1/2, ...; accepted when
//             |R(u + s du)| <= (1 - 1e-4 s) |R(u)|), convergence |R_p| <= max(atol, rtol |R_p(u0)|)
//             per load step with the load factor ramped k / n (Sec. 3.3).  Problems that
//             converge (or fail) leave the active set; the others continue.
#include <chrono>
#include <cmath>
#include <cstring>

#include "jfnk_internal.h"

namespace jfnk {

// per-problem header fields (everything before the h array) to the pinned mirror
static int read_problems(jfnk_ctx* c)
{
    JF_CUDA(c, cudaMemcpy2DAsync(c->ph, sizeof(ProbDev), c->pd, sizeof(ProbDev), offsetof(ProbDev, h), c->nprob,
                                 cudaMemcpyDeviceToHost, c->cur));
    JF_CUDA(c, cudaStreamSynchronize(c->cur));
    return JFNK_OK;
}

// copies field `off` (a double) of every problem's host mirror to the device
static int write_problem_doubles(jfnk_ctx* c, size_t off)
{
    JF_CUDA(c, cudaMemcpy2DAsync((char*)c->pd + off, sizeof(ProbDev), (const char*)c->ph + off, sizeof(ProbDev),
                                 sizeof(double), c->nprob, cudaMemcpyHostToDevice, c->cur));
    return JFNK_OK;
}

static int write_problem_ints(jfnk_ctx* c, size_t off)
{
    JF_CUDA(c, cudaMemcpy2DAsync((char*)c->pd + off, sizeof(ProbDev), (const char*)c->ph + off, sizeof(ProbDev),
                                 sizeof(int), c->nprob, cudaMemcpyHostToDevice, c->cur));
    return JFNK_OK;
}

// Jx = (R(u + eps x) - R(u)) / eps_p into out (direction x, eps_p from |x_p|)
static int jv_direction(jfnk_ctx* c, const double* x, double* out)
{
    int rc = pnorm(c, x, 1, false);
    if (!rc) rc = perturb(c, c->u, x, c->w, false);
    if (!rc) rc = residual(c, c->w, out, OUT_JV, SKIP_INACTIVE);  // restarts: the problems still iterating
    return rc;
}

// One lockstep Arnoldi iteration; kernels read the iteration index and the per-problem flags
// from the device and return at once when every cycle is done.
static bool left_pc(const jfnk_ctx* c) { return c->opt.pc_side == 1 && c->opt.pc != JFNK_PC_NONE; }

static int enqueue_iteration(jfnk_ctx* c)
{
    const int* gate = &c->gdev->all_done;
    int rc;
    // a batch's rows of the problems whose cycle still runs, for this iteration's compacted
    // residual passes and V-cycle (the flags change only in the Gram-Schmidt step at its end)
    if ((rc = rowmap_build(c, SKIP_CYCLE))) return rc;
    if (left_pc(c)) {
        if ((rc = perturb_basis(c, c->u, c->w))) return rc;
        if ((rc = residual_gated(c, c->w, c->wk, OUT_JV, gate, SKIP_CYCLE))) return rc;
        if ((rc = pc_apply_any(c, c->opt.pc, c->wk, 0, c->z, gate, SKIP_CYCLE))) return rc;
        if ((rc = arnoldi_orthogonalise(c, c->z))) return rc;
        JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gdev, sizeof(GlobalDev), cudaMemcpyDeviceToHost, c->cur));
        return JFNK_OK;
    }
    bool eps_formed = false;
    // a batch's problems whose cycle is done (or that left the Newton iteration) sit out the
    // preconditioner and the residual passes as they sit out the vector kernels
    if ((rc = pc_apply_dev(c, c->opt.pc, c->V, c->V_ld, &c->gdev->jg, c->V_is_float, c->z, gate, &eps_formed, SKIP_CYCLE)))
        return rc;
    if (!eps_formed && (rc = pnorm(c, c->z, 1, true))) return rc;
    if ((rc = perturb(c, c->u, c->z, c->w, true))) return rc;
    if ((rc = residual_gated(c, c->w, c->wk, OUT_JV, gate, SKIP_CYCLE))) return rc;
    if ((rc = arnoldi_orthogonalise(c, c->wk))) return rc;
    JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gdev, sizeof(GlobalDev), cudaMemcpyDeviceToHost, c->cur));
    return JFNK_OK;
}

static int capture_iteration(jfnk_ctx* c)
{
    if (c->it_graph) return JFNK_OK;
    cudaGraph_t g = nullptr;
    const int64_t before = c->launches;
    // captured on the context's own stream (the caller's may be the legacy stream, which
    // cannot be captured); the graph is launched on the caller's
    cudaStream_t caller = c->cur;
    c->cur = c->stream;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->cur = caller;
        return jfnk_cuda_fail(c, e, "cudaStreamBeginCapture");
    }
    int rc = enqueue_iteration(c);
    e = cudaStreamEndCapture(c->stream, &g);
    c->cur = caller;
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

// One Arnoldi iteration on a kept correction (loose GMRES): its image J z_l is stored, so the
// column needs no preconditioner and no product, only the orthogonalisation.
static int enqueue_aug_iteration(jfnk_ctx* c, int slot)
{
    int rc;
    if ((rc = aug_load(c, slot, c->wk))) return rc;
    if ((rc = arnoldi_orthogonalise(c, c->wk))) return rc;
    return JFNK_OK;
}

// Loose / restarted GMRES for every problem whose ph[p].active is set on entry (uploaded
// here).  its[p] gains the Arnoldi iterations of problem p, jvs[p] its Jacobian products;
// conv[p] tells whether its tolerance was met.
//   cycle: m columns, of which the last na (0 <= na <= options.gmres_aug) are the kept
//   corrections of earlier cycles (newest first), the first m - na Krylov directions;
//   correction d = P^-1 (V y over the Krylov columns) + sum_l y_l z_l;  x += d;
//   restart: r = b - J x, then d is kept as a correction with J d = r_prev - r.
int gmres_batch(jfnk_ctx* c, const double* b, double* x, std::vector<int>& its, std::vector<int>& jvs,
                std::vector<int>& conv)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    const int m = c->opt.gmres_restart, P = c->nprob;
    const int kaug = c->opt.gmres_aug;
    const bool left = left_pc(c);
    int rc;
    JF_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->cur));
    // the norm the tolerance refers to: |b_p|, or |P^-1 b_p| (kept in wk for the first cycle)
    if (left && (rc = pc_apply_any(c, c->opt.pc, b, 0, c->wk, nullptr))) return rc;
    if ((rc = pnorm(c, left ? c->wk : b, 0, false))) return rc;
    std::vector<int> act(P);
    for (int p = 0; p < P; p++) act[p] = c->ph[p].active;
    if ((rc = read_problems(c))) return rc;
    for (int p = 0; p < P; p++) {
        conv[p] = 0;
        const double b0 = c->ph[p].nrm;
        if (act[p] && !(b0 > 0.0)) {  // zero right-hand side: x = 0 solves it; NaN: not converged
            conv[p] = (b0 == 0.0);
            act[p] = 0;
        }
        c->ph[p].target = c->opt.gmres_eta * b0;
        c->ph[p].active = act[p];
    }
    if ((rc = write_problem_doubles(c, offsetof(ProbDev, target)))) return rc;
    if ((rc = write_problem_ints(c, offsetof(ProbDev, active)))) return rc;
    const bool graphs = c->use_graphs && !c->prof.enabled;
    if (graphs && (rc = capture_iteration(c))) return rc;
    int na = 0, head = 0;  // kept corrections; ring slot of the next one
    bool have_d = false;
    for (int rs = 0; rs < c->opt.gmres_max_restarts; rs++) {
        int n_act = 0;
        for (int p = 0; p < P; p++) n_act += act[p];
        if (!n_act) break;
        // r = b - J x (left: r = P^-1 (b - J x); P^-1 b is in wk already for the first cycle)
        if (rs == 0) {
            if (!left) JF_CUDA(c, cudaMemcpyAsync(c->wk, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->cur));
        } else {
            if ((rc = jv_direction(c, x, c->tmp))) return rc;
            if ((rc = axpby(c, n, 1.0, b, -1.0, c->tmp, left ? c->z : c->wk))) return rc;
            if (left && (rc = pc_apply_any(c, c->opt.pc, c->z, 0, c->wk, nullptr, SKIP_INACTIVE))) return rc;
            for (int p = 0; p < P; p++) jvs[p] += act[p];
        }
        // left: the Arnoldi vectors have unit norm, so eps_p = s (1 + |u_p|) for the whole cycle
        // (the restart's product above set eps for x)
        if (left && (rc = pnorm(c, c->u, 4, false))) return rc;
        if (kaug > 0) {
            if (have_d) {
                if ((rc = aug_store(c, head, c->wk))) return rc;
                head = (head + 1) % kaug;
                na = std::min(na + 1, kaug);
            }
            JF_CUDA(c, cudaMemcpyAsync(c->rprev, c->wk, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->cur));
        }
        int slots[8];
        for (int l = 0; l < na; l++) slots[l] = ((head - 1 - l) % kaug + kaug) % kaug;  // newest first
        const int mk = m - na;
        if ((rc = cycle_init(c, c->wk))) return rc;
        JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gdev, sizeof(GlobalDev), cudaMemcpyDeviceToHost, c->cur));
        JF_CUDA(c, cudaStreamSynchronize(c->cur));
        if (!c->gh->all_done) {
            // Arnoldi iterations; at most two in flight ahead of the host's view of `all done`
            for (int j = 0; j < m; j++) {
                if (j >= 2) {
                    JF_CUDA(c, cudaEventSynchronize(c->it_ev[(j - 2) & 3]));
                    if (((volatile GlobalDev*)c->gh)->all_done) break;
                }
                if (j >= mk) {
                    if ((rc = enqueue_aug_iteration(c, slots[j - mk]))) return rc;
                } else if (graphs) {
                    JF_CUDA(c, cudaGraphLaunch(c->it_graph, c->cur));
                    c->launches += c->graph_kernels;
                } else if ((rc = enqueue_iteration(c))) {
                    return rc;
                }
                JF_CUDA(c, cudaEventRecord(c->it_ev[j & 3], c->cur));
            }
            if ((rc = cycle_solution(c, c->tmp, mk))) return rc;
            // the Krylov part of the correction: P^-1 (V y) (right) or V y (left)
            const double* dk = c->tmp;
            if (!left) {
                if ((rc = pc_apply_any(c, c->opt.pc, c->tmp, 0, c->z, nullptr, SKIP_INACTIVE))) return rc;
                dk = c->z;
            }
            // the correction reaches the problems of this cycle only: the others sat the
            // preconditioner out, so their part of dk is stale
            if (kaug > 0) {
                if ((rc = aug_add(c, slots, na, mk, dk, c->dcorr))) return rc;
                if ((rc = add_active(c, c->dcorr, x))) return rc;
                have_d = true;
            } else if ((rc = add_active(c, dk, x))) {
                return rc;
            }
        }
        if ((rc = read_problems(c))) return rc;
        bool any_change = false;
        for (int p = 0; p < P; p++) {
            if (!act[p]) continue;
            const ProbDev& Q = c->ph[p];
            its[p] += Q.k;
            jvs[p] += std::min(Q.k, mk);
            const bool nan = !(Q.beta == Q.beta) || !(Q.res == Q.res);
            if (Q.beta <= Q.target || (Q.k > 0 && Q.res <= Q.target) || nan) {
                conv[p] = !nan;
                act[p] = 0;
                c->ph[p].active = 0;
                any_change = true;
            }
        }
        if (any_change && (rc = write_problem_ints(c, offsetof(ProbDev, active)))) return rc;
    }
    return JFNK_OK;
}

int newton(jfnk_ctx* c, int n_load_steps, jfnk_stats* st)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    const int P = c->nprob;
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    std::vector<jfnk_stats>& S = c->pstats;
    S.assign(P, jfnk_stats());
    for (auto& s : S) std::memset(&s, 0, sizeof s);
    std::vector<int> status(P, JFNK_OK), act(P), its(P), jvs(P), conv(P), newton_its(P);
    std::vector<double> rn(P), r0(P);
    if ((rc = read_problems(c))) return rc;
    for (int p = 0; p < P; p++) {
        c->ph[p].n_reorth = 0;
        c->ph[p].active = 0;
        c->ph[p].n_cols = c->ph[p].n_rcols = 0.0;
    }
    if ((rc = write_problem_ints(c, offsetof(ProbDev, n_reorth)))) return rc;
    if ((rc = write_problem_doubles(c, offsetof(ProbDev, n_cols)))) return rc;
    if ((rc = write_problem_doubles(c, offsetof(ProbDev, n_rcols)))) return rc;
    if ((rc = write_problem_ints(c, offsetof(ProbDev, active)))) return rc;
    const bool ul = c->law_mode == 3;  // updated Lagrangian: from the reference configuration
    if (ul && (rc = ul_reset(c))) return rc;
    for (int step = 1; step <= n_load_steps; step++) {
        if (ul && step > 1) {
            if (status[0] != JFNK_OK) break;
            if ((rc = ul_advance(c))) return rc;  // the last step converged: move the mesh
        }
        c->load = (double)step / n_load_steps;
        if ((rc = sync_load(c))) return rc;
        if ((rc = residual(c, c->u, c->Ru, OUT_R))) return rc;
        if ((rc = pnorm(c, c->Ru, 0, false))) return rc;
        if ((rc = read_problems(c))) return rc;
        for (int p = 0; p < P; p++) {
            rn[p] = r0[p] = c->ph[p].nrm;
            S[p].residual_evals++;
            act[p] = status[p] == JFNK_OK;
            newton_its[p] = 0;
        }
        for (;;) {
            int n_act = 0;
            for (int p = 0; p < P; p++) {
                if (!act[p]) continue;
                if (!std::isfinite(rn[p])) { status[p] = JFNK_DIVERGED; act[p] = 0; }
                else if (rn[p] <= std::max(c->opt.newton_atol, c->opt.newton_rtol * r0[p])) { act[p] = 0; S[p].load_steps_done++; }
                else if (newton_its[p] >= c->opt.newton_max_its) { status[p] = JFNK_MAXIT; act[p] = 0; }
                n_act += act[p];
            }
            if (!n_act) break;
            if ((rc = axpby(c, n, -1.0, c->Ru, 0.0, c->Ru, c->bvec))) return rc;
            if ((rc = pnorm(c, c->u, 2, false))) return rc;
            for (int p = 0; p < P; p++) { c->ph[p].active = act[p]; its[p] = 0; jvs[p] = 0; }
            if ((rc = gmres_batch(c, c->bvec, c->x, its, jvs, conv))) return rc;
            for (int p = 0; p < P; p++) {
                if (!act[p]) continue;
                S[p].gmres_its += its[p];
                S[p].jv_products += jvs[p];
                S[p].residual_evals += jvs[p];
            }
            // backtracking line search, per problem
            std::vector<int> acc(P, 0), trial(act);
            std::vector<double> s(P, 1.0), rt(P, 0.0);
            for (int ls = 0; ls <= c->opt.line_search_max; ls++) {
                int n_trial = 0;
                for (int p = 0; p < P; p++) {
                    c->ph[p].active = trial[p];
                    c->ph[p].step = s[p];
                    n_trial += trial[p];
                }
                if (!n_trial) break;
                if ((rc = write_problem_ints(c, offsetof(ProbDev, active)))) return rc;
                if ((rc = write_problem_doubles(c, offsetof(ProbDev, step)))) return rc;
                if ((rc = line_trial(c, c->u, c->x, c->w))) return rc;
                if ((rc = residual(c, c->w, c->R, OUT_R, SKIP_INACTIVE))) return rc;  // the trial problems
                if ((rc = pnorm(c, c->R, 0, false))) return rc;
                if ((rc = read_problems(c))) return rc;
                bool any = false;
                for (int p = 0; p < P; p++) {
                    c->pmask_h[p] = 0;
                    if (!trial[p]) continue;
                    S[p].residual_evals++;
                    rt[p] = c->ph[p].nrm;
                    if (rt[p] <= (1.0 - 1e-4 * s[p]) * rn[p]) {
                        acc[p] = 1;
                        trial[p] = 0;
                        c->pmask_h[p] = 1;
                        any = true;
                    } else {
                        s[p] *= 0.5;
                    }
                }
                if (any) {
                    JF_CUDA(c, cudaMemcpyAsync(c->pmask, c->pmask_h, sizeof(int32_t) * P, cudaMemcpyHostToDevice, c->cur));
                    if ((rc = accept_masked(c, c->pmask, c->u, c->w, c->Ru, c->R))) return rc;
                }
            }
            JF_CUDA(c, cudaStreamSynchronize(c->cur));
            for (int p = 0; p < P; p++) {
                if (!act[p]) continue;
                if (!acc[p]) { status[p] = JFNK_LS_FAILED; act[p] = 0; continue; }
                rn[p] = rt[p];
                newton_its[p]++;
                S[p].newton_its++;
                if (S[p].n_hist < 64) S[p].hist[S[p].n_hist++] = rn[p];
            }
        }
        for (int p = 0; p < P; p++) {
            S[p].final_rel_res = r0[p] > 0 ? rn[p] / r0[p] : 0.0;
            S[p].final_abs_res = rn[p];
        }
    }
    if (ul && status[0] == JFNK_OK && (rc = ul_advance(c))) return rc;  // the final configuration
    if ((rc = read_problems(c))) return rc;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    // aggregate: maximum Newton count, sums of Krylov counts, worst status and residual
    std::memset(st, 0, sizeof *st);
    st->status = JFNK_OK;
    st->load_steps_done = n_load_steps;
    for (int p = 0; p < P; p++) {
        S[p].status = status[p];
        S[p].reorth_its = c->ph[p].n_reorth;
        S[p].arnoldi_cols = c->ph[p].n_cols;
        S[p].reorth_cols = c->ph[p].n_rcols;
        S[p].solve_ms = ms;
        st->newton_its = std::max(st->newton_its, S[p].newton_its);
        st->gmres_its += S[p].gmres_its;
        st->residual_evals += S[p].residual_evals;
        st->reorth_its += S[p].reorth_its;
        st->jv_products += S[p].jv_products;
        st->arnoldi_cols += S[p].arnoldi_cols;
        st->reorth_cols += S[p].reorth_cols;
        st->load_steps_done = std::min(st->load_steps_done, S[p].load_steps_done);
        st->final_rel_res = std::max(st->final_rel_res, S[p].final_rel_res);
        st->final_abs_res = std::max(st->final_abs_res, S[p].final_abs_res);
        if (status[p] != JFNK_OK && st->status == JFNK_OK) st->status = status[p];
    }
    if (P == 1) {
        st->n_hist = S[0].n_hist;
        std::memcpy(st->hist, S[0].hist, sizeof st->hist);
    }
    st->solve_ms = ms;
    return st->status;
}

}  // namespace jfnk
