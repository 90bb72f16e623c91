// The segregated quasi-Newton method of Sec. 3.1 on the device, for the same P >= 1 problems
// as the Newton-Krylov path (the comparison the paper draws, on the same hardware and with
// the same residual, J~ and preconditioners).
//
// Outer iteration k, per problem:  J~ du = -R(u_k) solved component by component (J~ has no
// coupling between components; one scalar matrix), u_{k+1} = u_k + du; converged when
// |R| <= max(atol, rtol |R(u0)|) per load step (Sec. 3.3).  Each component's system is
// A du = R with A = -J~ (symmetric positive definite once displacement faces exist), solved
// by preconditioned conjugate gradients from du = 0 until its residual has fallen by
// options.seg_inner_tol (Sec. 3.2: 0.9), the preconditioner being the A-form (negative) of
// the block-Jacobi or multigrid P^-1 of the Newton-Krylov path.
//
// All 3P component systems ("slots", slot = 3 p + k) advance in lockstep: each CG iteration
// (preconditioner, r.z, direction, A d, d.q, update + |r|) is one captured CUDA graph whose
// kernels read per-slot scalars and flags from device memory; a slot whose residual has
// fallen enough stops changing, and the graph's kernels return at once when every slot is
// done.  Reductions are per slot over its chunks (fixed order, ticketed last block), so the
// result is bitwise reproducible and the same for a problem alone or in a batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

namespace {

struct SlotChunks {
    const int64_t* beg;
    const int32_t* len;
    const int32_t* slot;   // slot of each chunk
    const int32_t* sbeg;   // first chunk of each slot
    const int32_t* scnt;   // chunks of each slot
};

__device__ void slot_finish(SegSlot& S, GlobalDev* gdev)
{
    S.done = 1;
    if (atomicSub(&gdev->n_active, 1) == 1) gdev->all_done = 1;
}

// mode 0: rr0 = |x|, r = x, du = 0, slot state reset (inactive problems' slots start done)
// mode 1: rz = zsign (x . y) with y = P^-1 r: the preconditioner of A = -J~ is -P^-1 for the
//         J~-approximations (block-Jacobi, multigrid; zsign = -1), the identity otherwise
// mode 2: alpha = rz / (x . y) with x = d, y = q = A d
template <int MODE>
__global__ void __launch_bounds__(kChunkThreads) k_seg_dot(SlotChunks ch, const double* __restrict__ x,
                                                          const double* __restrict__ y, double* __restrict__ r,
                                                          double* __restrict__ du, const ProbDev* __restrict__ pd,
                                                          SegSlot* sl, double* __restrict__ partials,
                                                          GlobalDev* gdev, double zsign)
{
    JF_PDL_ENTRY();
    if (MODE != 0 && gdev->all_done) return;
    const int c = blockIdx.x, s = ch.slot[c];
    SegSlot& S = sl[s];
    if (MODE != 0 && S.done) return;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    __shared__ double sh[32];
    double a = 0.0;
    for (int q = threadIdx.x; q < len; q += kChunkThreads) {
        const double xv = x[b0 + q];
        if (MODE == 0) {
            r[b0 + q] = xv;
            du[b0 + q] = 0.0;
            a = fma(xv, xv, a);
        } else {
            a = fma(xv, y[b0 + q], a);
        }
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[c] = a;
    if (!ticket_last(&S.ticket, (unsigned)ch.scnt[s])) return;
    if (threadIdx.x < 32) {
        const double tot = warp_sum_strided(partials + ch.sbeg[s], ch.scnt[s]);
        if (threadIdx.x == 0) {
            if (MODE == 0) {
                S.rr0 = sqrt(tot);
                S.rr = S.rr0;
                S.its = 0;
                S.rz = 0.0;
                S.beta = 0.0;
                S.alpha = 0.0;
                S.done = (!pd[s / 3].active || !(S.rr0 > 0.0)) ? 1 : 0;
            } else if (MODE == 1) {
                const double rz = zsign * tot;
                S.beta = (S.its == 0) ? 0.0 : rz / S.rz;
                S.rz = rz;
            } else {
                S.alpha = S.rz / tot;
            }
            S.ticket = 0u;
        }
    }
}

// d = zsign z + beta d (zsign z is the preconditioned residual of A, see k_seg_dot)
__global__ void __launch_bounds__(kChunkThreads) k_seg_dir(SlotChunks ch, const double* __restrict__ z,
                                                          const SegSlot* __restrict__ sl, const GlobalDev* gdev,
                                                          double zsign, double* __restrict__ d)
{
    JF_PDL_ENTRY();
    if (gdev->all_done) return;
    const int c = blockIdx.x;
    const SegSlot& S = sl[ch.slot[c]];
    if (S.done) return;
    const double beta = S.beta;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) d[b0 + q] = fma(beta, d[b0 + q], zsign * z[b0 + q]);
}

// du += alpha d, r -= alpha q, then |r|: the slot is done when |r| <= tol |r0| (or max_inner)
__global__ void __launch_bounds__(kChunkThreads) k_seg_update(SlotChunks ch, const double* __restrict__ d,
                                                             const double* __restrict__ q, double* __restrict__ du,
                                                             double* __restrict__ r, SegSlot* sl, double tol,
                                                             int max_inner, double* __restrict__ partials,
                                                             GlobalDev* gdev)
{
    JF_PDL_ENTRY();
    if (gdev->all_done) return;
    const int c = blockIdx.x, s = ch.slot[c];
    SegSlot& S = sl[s];
    if (S.done) return;
    const double alpha = S.alpha;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    __shared__ double sh[32];
    double a = 0.0;
    for (int e = threadIdx.x; e < len; e += kChunkThreads) {
        du[b0 + e] = fma(alpha, d[b0 + e], du[b0 + e]);
        const double rn = fma(-alpha, q[b0 + e], r[b0 + e]);
        r[b0 + e] = rn;
        a = fma(rn, rn, a);
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[c] = a;
    if (!ticket_last(&S.ticket, (unsigned)ch.scnt[s])) return;
    if (threadIdx.x < 32) {
        const double tot = warp_sum_strided(partials + ch.sbeg[s], ch.scnt[s]);
        if (threadIdx.x == 0) {
            S.rr = sqrt(tot);
            S.its++;
            if (!(S.rr > tol * S.rr0) || S.its >= max_inner) slot_finish(S, gdev);
            S.ticket = 0u;
        }
    }
}

// number of slots still iterating; clears the iteration flags
__global__ void k_seg_count(const SegSlot* sl, int nslots, GlobalDev* gdev)
{
    JF_PDL_ENTRY();
    int n = 0;
    for (int s = 0; s < nslots; s++) n += sl[s].done ? 0 : 1;
    gdev->n_active = n;
    gdev->all_done = n == 0 ? 1 : 0;
}

// q = A d = -J~ d over all cells (matrix-free from the J~ face coefficients; the slots' own
// rows only matter, the others are ignored)
__global__ void k_seg_apply(int nc, const int32_t* __restrict__ fo_ptr, const int32_t* __restrict__ fn_ptr,
                            const int32_t* __restrict__ fn_face, const int32_t* __restrict__ own,
                            const int32_t* __restrict__ nei, const double* __restrict__ jc,
                            const double* __restrict__ jdiag, const double* __restrict__ symd,
                            const double* __restrict__ d, const GlobalDev* gdev, double* __restrict__ q)
{
    JF_PDL_ENTRY();
    if (gdev->all_done) return;
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const double a = -jdiag[P];
    double o0 = a * d[P], o1 = a * d[nc + P], o2 = a * d[2 * (size_t)nc + P];
    if (symd) {  // symmetry faces: the component's own part of the n n block (Sec. 3.1)
        o0 = fma(symd[P], d[P], o0);
        o1 = fma(symd[nc + P], d[nc + P], o1);
        o2 = fma(symd[2 * (size_t)nc + P], d[2 * (size_t)nc + P], o2);
    }
    for (int f = fo_ptr[P]; f < fo_ptr[P + 1]; f++) {
        const int N = nei[f];
        const double cf = jc[f];
        o0 -= cf * d[N]; o1 -= cf * d[nc + N]; o2 -= cf * d[2 * (size_t)nc + N];
    }
    for (int k = fn_ptr[P]; k < fn_ptr[P + 1]; k++) {
        const int f = fn_face[k];
        const int N = own[f];
        const double cf = jc[f];
        o0 -= cf * d[N]; o1 -= cf * d[nc + N]; o2 -= cf * d[2 * (size_t)nc + N];
    }
    q[P] = o0; q[nc + P] = o1; q[2 * (size_t)nc + P] = o2;
}

inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// the per-slot chunk table (built once per set-up, from the per-problem one: a problem's
// chunks are ordered by component)
int seg_setup(jfnk_ctx* c)
{
    if (c->seg_slot) return JFNK_OK;
    const int P = c->nprob, nch = c->n_chunks;
    std::vector<int32_t> pbeg(P), pcnt(P), len(nch);
    std::vector<int64_t> beg(nch);
    int rc;
    if ((rc = jfnk_download(c, pbeg.data(), c->pch_beg, sizeof(int32_t) * P)) ||
        (rc = jfnk_download(c, pcnt.data(), c->pch_cnt, sizeof(int32_t) * P)) ||
        (rc = jfnk_download(c, beg.data(), c->ch_beg, sizeof(int64_t) * nch)) ||
        (rc = jfnk_download(c, len.data(), c->ch_len, sizeof(int32_t) * nch)))
        return rc;
    const int64_t nc = c->dm.nc;
    std::vector<int32_t> slot(nch), sbeg(3 * P, 0), scnt(3 * P, 0);
    for (int p = 0; p < P; p++)
        for (int q = pbeg[p]; q < pbeg[p] + pcnt[p]; q++) {
            const int k = (int)(beg[q] / nc);
            const int s = 3 * p + k;
            if (scnt[s] == 0) sbeg[s] = q;
            scnt[s]++;
            slot[q] = s;
        }
    auto up = [&](const std::vector<int32_t>& h) -> int32_t* {
        int32_t* d = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * std::max<size_t>(1, h.size()));
        if (d && jfnk_upload(c, d, h.data(), sizeof(int32_t) * h.size())) return (int32_t*)nullptr;
        return d;
    };
    c->seg_slot = up(slot);
    c->seg_sbeg = up(sbeg);
    c->seg_scnt = up(scnt);
    c->seg_state = (SegSlot*)jfnk_dalloc(c, sizeof(SegSlot) * 3 * (size_t)P);
    if (!c->seg_slot || !c->seg_sbeg || !c->seg_scnt || !c->seg_state)
        return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the segregated solver's tables failed");
    c->seg_state_h.assign(3 * (size_t)P, SegSlot());
    return JFNK_OK;
}

static SlotChunks slot_chunks(const jfnk_ctx* c)
{
    return SlotChunks{c->ch_beg, c->ch_len, c->seg_slot, c->seg_sbeg, c->seg_scnt};
}

// One CG iteration of every running slot (graph-safe: reads all scalars from the device).
// Vectors: r = c->wk, z = c->z, d = c->x, q = c->tmp, du = c->bvec.
static int seg_enqueue_iteration(jfnk_ctx* c)
{
    const int* gate = &c->gdev->all_done;
    const SlotChunks ch = slot_chunks(c);
    const double zsign = (c->opt.pc == JFNK_PC_NONE) ? 1.0 : -1.0;
    int rc;
    if ((rc = pc_apply_any(c, c->opt.pc, c->wk, 0, c->z, gate))) return rc;
    jfnk_launch(c, k_seg_dot<1>, dim3(c->n_chunks), dim3(kChunkThreads), ch, (const double*)c->wk, (const double*)c->z,
                (double*)nullptr, (double*)nullptr, (const ProbDev*)c->pd, c->seg_state, c->partials, c->gdev, zsign);
    JF_LAUNCHED(c);
    jfnk_launch(c, k_seg_dir, dim3(c->n_chunks), dim3(kChunkThreads), ch, (const double*)c->z,
                (const SegSlot*)c->seg_state, (const GlobalDev*)c->gdev, zsign, c->x);
    JF_LAUNCHED(c);
    const DevMesh& m = c->dm;
    jfnk_launch(c, k_seg_apply, dim3(nblk(m.nc, 256)), dim3(256), m.nc, m.fo_ptr, m.fn_ptr, m.fn_face, m.own, m.nei,
                (const double*)m.jt_c, (const double*)m.jt_diag, (const double*)m.seg_symd, (const double*)c->x,
                (const GlobalDev*)c->gdev, c->tmp);
    JF_LAUNCHED(c);
    jfnk_launch(c, k_seg_dot<2>, dim3(c->n_chunks), dim3(kChunkThreads), ch, (const double*)c->x, (const double*)c->tmp,
                (double*)nullptr, (double*)nullptr, (const ProbDev*)c->pd, c->seg_state, c->partials, c->gdev, zsign);
    JF_LAUNCHED(c);
    jfnk_launch(c, k_seg_update, dim3(c->n_chunks), dim3(kChunkThreads), ch, (const double*)c->x, (const double*)c->tmp,
                c->bvec, c->wk, c->seg_state, c->opt.seg_inner_tol, c->opt.seg_max_inner, c->partials, c->gdev);
    JF_LAUNCHED(c);
    JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gdev, sizeof(GlobalDev), cudaMemcpyDeviceToHost, c->cur));
    return JFNK_OK;
}

static int seg_capture(jfnk_ctx* c)
{
    if (c->seg_graph) return JFNK_OK;
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
    int rc = seg_enqueue_iteration(c);
    e = cudaStreamEndCapture(c->stream, &g);
    c->cur = caller;
    c->seg_graph_kernels = c->launches - before;
    c->launches = before;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return jfnk_cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->seg_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->seg_graph = nullptr;
        return jfnk_cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return JFNK_OK;
}

int segregated(jfnk_ctx* c, int n_load_steps, jfnk_stats* st)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    const int P = c->nprob;
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    if ((rc = seg_setup(c))) return rc;
    std::vector<jfnk_stats>& S = c->pstats;
    S.assign(P, jfnk_stats());
    for (auto& s : S) std::memset(&s, 0, sizeof s);
    std::vector<int> status(P, JFNK_OK), act(P), outer(P);
    std::vector<double> rn(P), r0(P);
    const bool graphs = c->use_graphs && !c->prof.enabled;
    const SlotChunks ch = slot_chunks(c);
    auto read_slots = [&]() -> int {
        JF_CUDA(c, cudaMemcpyAsync(c->seg_state_h.data(), c->seg_state, sizeof(SegSlot) * 3 * (size_t)P,
                                   cudaMemcpyDeviceToHost, c->cur));
        JF_CUDA(c, cudaStreamSynchronize(c->cur));
        return JFNK_OK;
    };
    for (int step = 1; step <= n_load_steps; step++) {
        c->load = (double)step / n_load_steps;
        if ((rc = sync_load(c))) return rc;
        if ((rc = residual(c, c->u, c->Ru, OUT_R))) return rc;
        if ((rc = pnorm(c, c->Ru, 0, false))) return rc;
        JF_CUDA(c, cudaMemcpy2DAsync(c->ph, sizeof(ProbDev), c->pd, sizeof(ProbDev), offsetof(ProbDev, h), P,
                                     cudaMemcpyDeviceToHost, c->cur));
        JF_CUDA(c, cudaStreamSynchronize(c->cur));
        for (int p = 0; p < P; p++) {
            rn[p] = r0[p] = c->ph[p].nrm;
            S[p].residual_evals++;
            act[p] = status[p] == JFNK_OK;
            outer[p] = 0;
        }
        for (;;) {
            int n_act = 0;
            for (int p = 0; p < P; p++) {
                if (!act[p]) continue;
                if (!std::isfinite(rn[p])) { status[p] = JFNK_DIVERGED; act[p] = 0; }
                else if (rn[p] <= std::max(c->opt.newton_atol, c->opt.newton_rtol * r0[p])) { act[p] = 0; S[p].load_steps_done++; }
                else if (outer[p] >= c->opt.seg_max_outer) { status[p] = JFNK_MAXIT; act[p] = 0; }
                n_act += act[p];
            }
            if (!n_act) break;
            for (int p = 0; p < P; p++) c->ph[p].active = act[p];
            JF_CUDA(c, cudaMemcpy2DAsync((char*)c->pd + offsetof(ProbDev, active), sizeof(ProbDev),
                                         (const char*)c->ph + offsetof(ProbDev, active), sizeof(ProbDev), sizeof(int), P,
                                         cudaMemcpyHostToDevice, c->cur));
            // r = R, du = 0, |r0| per slot; slots of converged problems start done
            jfnk_launch(c, k_seg_dot<0>, dim3(c->n_chunks), dim3(kChunkThreads), ch, (const double*)c->Ru,
                        (const double*)nullptr, c->wk, c->bvec, (const ProbDev*)c->pd, c->seg_state, c->partials, c->gdev,
                        1.0);
            JF_LAUNCHED(c);
            jfnk_launch(c, k_seg_count, dim3(1), dim3(1), (const SegSlot*)c->seg_state, 3 * P, c->gdev);
            JF_LAUNCHED(c);
            JF_CUDA(c, cudaMemcpyAsync(c->gh, c->gdev, sizeof(GlobalDev), cudaMemcpyDeviceToHost, c->cur));
            JF_CUDA(c, cudaStreamSynchronize(c->cur));
            if (graphs && (rc = seg_capture(c))) return rc;
            // CG iterations; at most two in flight ahead of the host's view of `all done`
            for (int k = 0; k < c->opt.seg_max_inner && !c->gh->all_done; k++) {
                if (k >= 2) {
                    JF_CUDA(c, cudaEventSynchronize(c->it_ev[(k - 2) & 3]));
                    if (((volatile GlobalDev*)c->gh)->all_done) break;
                }
                if (graphs) {
                    JF_CUDA(c, cudaGraphLaunch(c->seg_graph, c->cur));
                    c->launches += c->seg_graph_kernels;
                } else if ((rc = seg_enqueue_iteration(c))) {
                    return rc;
                }
                JF_CUDA(c, cudaEventRecord(c->it_ev[k & 3], c->cur));
            }
            // u += du for the problems that iterated (converged ones have du = 0)
            if ((rc = axpby(c, n, 1.0, c->u, 1.0, c->bvec, c->u))) return rc;
            if ((rc = residual(c, c->u, c->Ru, OUT_R))) return rc;
            if ((rc = pnorm(c, c->Ru, 0, false))) return rc;
            if ((rc = read_slots())) return rc;
            JF_CUDA(c, cudaMemcpy2DAsync(c->ph, sizeof(ProbDev), c->pd, sizeof(ProbDev), offsetof(ProbDev, h), P,
                                         cudaMemcpyDeviceToHost, c->cur));
            JF_CUDA(c, cudaStreamSynchronize(c->cur));
            for (int p = 0; p < P; p++) {
                if (!act[p]) continue;
                for (int k = 0; k < 3; k++) S[p].gmres_its += c->seg_state_h[3 * p + k].its;
                S[p].residual_evals++;
                S[p].newton_its++;
                outer[p]++;
                rn[p] = c->ph[p].nrm;
                if (S[p].n_hist < 64) S[p].hist[S[p].n_hist++] = rn[p];
            }
        }
        for (int p = 0; p < P; p++) {
            S[p].final_rel_res = r0[p] > 0 ? rn[p] / r0[p] : 0.0;
            S[p].final_abs_res = rn[p];
        }
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::memset(st, 0, sizeof *st);
    st->status = JFNK_OK;
    st->load_steps_done = n_load_steps;
    for (int p = 0; p < P; p++) {
        S[p].status = status[p];
        S[p].solve_ms = ms;
        st->newton_its = std::max(st->newton_its, S[p].newton_its);
        st->gmres_its += S[p].gmres_its;
        st->residual_evals += S[p].residual_evals;
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

extern "C" int jfnk_solve_segregated(jfnk_ctx* c, double* u, int mem, int n_load_steps, jfnk_stats* stats, void* stream)
{
    return jfnk_solve_method(c, u, mem, n_load_steps, stats, stream, 1);
}
