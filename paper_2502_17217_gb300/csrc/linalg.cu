// Vector kernels of the JFNK loop for P >= 1 independent problems held in one concatenated
// index space: caller-order <-> internal-order permutation, per-problem FP64 norms and the Jv
// step eps (Eq. JF), and the Arnoldi process of right-preconditioned GMRES(m) (Sec. 3.2) with
// one Hessenberg matrix, Givens sequence and convergence flag per problem.
//
// Segmented reductions run over a chunk table (every chunk lies inside one problem's range of
// one displacement component); each chunk's block writes a partial sum and the last block of
// a problem to arrive (a per-problem ticket) adds that problem's partials in chunk order, so
// results are bitwise reproducible and identical for a problem alone or in a batch.  All
// active problems advance in lockstep (one Arnoldi index); kernels skip problems whose cycle
// is done and return at once when every cycle is done.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

__global__ void k_perm_in(int nc, int dim, const int32_t* __restrict__ n2o, const double* __restrict__ ext,
                          double* __restrict__ out)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const size_t o = (size_t)n2o[P] * 3;
    out[P] = ext[o];
    out[nc + P] = ext[o + 1];
    out[2 * (size_t)nc + P] = dim == 2 ? 0.0 : ext[o + 2];
}

__global__ void k_perm_out(int nc, const int32_t* __restrict__ n2o, const double* __restrict__ in, double* __restrict__ ext)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const size_t o = (size_t)n2o[P] * 3;
    ext[o] = in[P];
    ext[o + 1] = in[nc + P];
    ext[o + 2] = in[2 * (size_t)nc + P];
}

__global__ void k_axpby(size_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = fma(a, x[e], b * y[e]);
}

struct Chunks {
    const int64_t* beg;
    const int32_t* len;
    const int32_t* prob;
    const int32_t* pbeg;  // first chunk of each problem
    const int32_t* pcnt;  // chunks of each problem
};

__device__ __forceinline__ bool skip_problem(const ProbDev& P) { return !P.active || P.done; }

// The last block of problem p to arrive returns true (after every block of p stored its
// partials); it must reset the ticket.
__device__ __forceinline__ bool last_of_problem(unsigned* ticket, unsigned expected)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == expected - 1);
    __syncthreads();
    return is_last;
}

// Sum of one problem's chunk partials (fixed order), by warp 0; valid in lane 0.
__device__ __forceinline__ double sum_problem_partials(const double* partials, int first, int count)
{
    double s = 0.0;
    for (int b = threadIdx.x & 31; b < count; b += 32) s += __ldcg(partials + first + b);
    return warp_sum(s);
}

// ------------------------------------------------------------------ per-problem norms
// mode 0: nrm = |x_p|;  1: eps = s (1 + unorm) / |x_p| (0 for x_p = 0);  2: unorm = |x_p|;
// 3: beta = |x_p|, inv = 1/beta (0 for beta = 0)
__global__ void __launch_bounds__(kChunkThreads) k_pnorm(Chunks ch, const double* __restrict__ x,
                                                        double* __restrict__ partials, ProbDev* pd, int mode,
                                                        double s, int gated, const GlobalDev* gdev)
{
    const int c = blockIdx.x, p = ch.prob[c];
    ProbDev& P = pd[p];
    if (gated && (gdev->all_done || skip_problem(P))) return;
    __shared__ double sh[32];
    double a = 0.0;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) {
        const double v = x[b0 + q];
        a = fma(v, v, a);
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[c] = a;
    if (!last_of_problem(&P.ticket[2], (unsigned)ch.pcnt[p])) return;
    if (threadIdx.x < 32) {
        const double tot = sum_problem_partials(partials, ch.pbeg[p], ch.pcnt[p]);
        if (threadIdx.x == 0) {
            const double nrm = sqrt(tot);
            if (mode == 0) P.nrm = nrm;
            else if (mode == 1) P.eps = (nrm > 0.0) ? s * (1.0 + P.unorm) / nrm : 0.0;
            else if (mode == 2) P.unorm = nrm;
            else { P.beta = nrm; P.inv = nrm > 0.0 ? 1.0 / nrm : 0.0; }
            P.ticket[2] = 0u;
        }
    }
}

// w = u + eps_p z (Eq. JF), active problems whose cycle runs
__global__ void __launch_bounds__(kChunkThreads) k_perturb(Chunks ch, const double* __restrict__ u,
                                                          const double* __restrict__ z, const ProbDev* __restrict__ pd,
                                                          const GlobalDev* __restrict__ gdev, int gated,
                                                          double* __restrict__ w)
{
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    if (gated && (gdev->all_done || skip_problem(P))) return;
    const double eps = P.eps;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) w[b0 + q] = fma(eps, z[b0 + q], u[b0 + q]);
}

// line-search trial w = u + s_p x for active problems, w = u for the others
__global__ void __launch_bounds__(kChunkThreads) k_line_trial(Chunks ch, const double* __restrict__ u,
                                                             const double* __restrict__ x, const ProbDev* __restrict__ pd,
                                                             double* __restrict__ w)
{
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    const double s = P.active ? P.step : 0.0;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) w[b0 + q] = fma(s, x[b0 + q], u[b0 + q]);
}

// u <- w, Ru <- R for problems whose mask is set
__global__ void __launch_bounds__(kChunkThreads) k_accept(Chunks ch, const int32_t* __restrict__ mask,
                                                         double* __restrict__ u, const double* __restrict__ w,
                                                         double* __restrict__ Ru, const double* __restrict__ R)
{
    const int c = blockIdx.x;
    if (!mask[ch.prob[c]]) return;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) {
        u[b0 + q] = w[b0 + q];
        Ru[b0 + q] = R[b0 + q];
    }
}

// ------------------------------------------------------------------ Arnoldi
// One block per problem: start a cycle (beta and inv already computed).
__global__ void k_cycle_init(ProbDev* pd, int m)
{
    ProbDev& P = pd[blockIdx.x];
    const int m1 = m + 1;
    for (int i = threadIdx.x; i < m1 * m; i += blockDim.x) P.H[i] = 0.0;
    for (int i = threadIdx.x; i < m1; i += blockDim.x) P.g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        P.g[0] = P.beta;
        P.j = 0;
        P.k = 0;
        P.reorth = 0;
        P.res = P.beta;
        P.done = (!P.active || !(P.beta > P.target)) ? 1 : 0;
    }
}

// Single thread: count the problems whose cycle runs.
__global__ void k_cycle_count(ProbDev* pd, int nprob, GlobalDev* gdev)
{
    int n = 0;
    for (int p = 0; p < nprob; p++) n += pd[p].done ? 0 : 1;
    gdev->n_active = n;
    gdev->all_done = n == 0;
    gdev->jg = 0;
}

// V_0 = r_p / beta_p
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_scale_first(Chunks ch, const double* __restrict__ r,
                                                              const ProbDev* __restrict__ pd, TV* __restrict__ V0)
{
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    const double s = P.done ? 0.0 : P.inv;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) V0[b0 + q] = (TV)(r[b0 + q] * s);
}

// Givens step on column j of problem P's H (one thread), sets done and advances j.
__device__ void givens_step(ProbDev& P, int m, GlobalDev* gdev)
{
    const int m1 = m + 1, j = P.j;
    double* H = P.H + (size_t)m1 * j;
    const double hn = H[j + 1];
    for (int i = 0; i < j; i++) {
        const double t = P.cs[i] * H[i] + P.sn[i] * H[i + 1];
        H[i + 1] = -P.sn[i] * H[i] + P.cs[i] * H[i + 1];
        H[i] = t;
    }
    const double a = H[j], b = H[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    P.cs[j] = c;
    P.sn[j] = s;
    H[j] = r;
    H[j + 1] = 0.0;
    const double gj = P.g[j];
    P.g[j + 1] = -s * gj;
    P.g[j] = c * gj;
    P.k = j + 1;
    P.res = fabs(P.g[j + 1]);
    P.j = j + 1;
    if (P.res <= P.target || hn == 0.0 || j + 1 >= m || !(P.res == P.res)) {
        P.done = 1;
        if (atomicSub(&gdev->n_active, 1) == 1) gdev->all_done = 1;
    }
}

// Multi-dot h_i = V_i . w (i <= j) and, in pass 0, |w|^2, per problem.  Grid: x = chunks,
// y = one basis vector per block.  Each thread multiplies 16 elements before the FP64 warp
// reduction.  Pass 1 runs only for problems whose pass-0 test asked for it.
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_mdot(Chunks ch, const TV* __restrict__ V, size_t ld,
                                                       const double* __restrict__ w, ProbDev* pd, int pass,
                                                       int reorth_mode, double* __restrict__ partials, int m,
                                                       const GlobalDev* __restrict__ gdev, int nchunks)
{
    if (gdev->all_done) return;
    const int c = blockIdx.x, p = ch.prob[c];
    ProbDev& P = pd[p];
    if (skip_problem(P) || (pass == 1 && !P.reorth)) return;
    const int j = P.j, nv = j + 1, m1 = m + 1;
    const int nvals = nv + (pass == 0 ? 1 : 0);
    const int i = blockIdx.y;
    __shared__ double sh[kChunkThreads / 32];
    __shared__ double sums[kMaxRestart + 2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (i < nvals) {
        const int64_t b0 = ch.beg[c];
        const int len = ch.len[c];
        double acc = 0.0;
        if (i < nv) {
            const TV* vi = V + (size_t)i * ld + b0;
#pragma unroll 8
            for (int q = threadIdx.x; q < len; q += kChunkThreads) acc = fma(to_f64(vi[q]), w[b0 + q], acc);
        } else {
#pragma unroll 8
            for (int q = threadIdx.x; q < len; q += kChunkThreads) {
                const double x = w[b0 + q];
                acc = fma(x, x, acc);
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) sh[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int x = 0; x < kChunkThreads / 32; x++) s += sh[x];
            partials[(size_t)i * nchunks + c] = s;
        }
    }
    if (!last_of_problem(&P.ticket[0], (unsigned)ch.pcnt[p] * gridDim.y)) return;
    const int first = ch.pbeg[p], cnt = ch.pcnt[p];
    for (int v = wid; v < nvals; v += kChunkThreads / 32) {
        double sacc = 0.0;
        for (int b = lane; b < cnt; b += 32) sacc += __ldcg(partials + (size_t)v * nchunks + first + b);
        sacc = warp_sum(sacc);
        if (lane == 0) sums[v] = sacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double hh = 0.0;
        for (int v = 0; v < nv; v++) {
            P.h[v] = sums[v];
            if (pass == 0) P.H[v + (size_t)m1 * j] = sums[v];
            else P.H[v + (size_t)m1 * j] += sums[v];
            hh += sums[v] * sums[v];
        }
        if (pass == 0) {
            const double wn2 = sums[nv];
            P.wn2 = wn2;
            // classical Gram-Schmidt is repeated when the projection removed more than half
            // of |w|^2, i.e. |w'| < |w| / sqrt(2) (the 'twice is enough' test)
            P.reorth = (reorth_mode == 1 || (reorth_mode == 0 && (wn2 - hh) < 0.5 * wn2)) ? 1 : 0;
        } else {
            P.n_reorth++;
        }
        P.ticket[0] = 0u;
    }
}

// w -= sum_i h_i V_i and |w|^2.  Grid: x = chunks, y = kUpdSub sub-blocks of a chunk (each
// thread updates kUpdE elements as independent FMA chains).  The final pass of a problem
// stores H(j+1, j) = |w|, 1/|w| and runs its Givens step.
constexpr int kUpdSub = 4, kUpdE = kChunk / (kUpdSub * kChunkThreads);

template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_update(Chunks ch, const TV* __restrict__ V, size_t ld,
                                                         double* __restrict__ w, ProbDev* pd, int pass,
                                                         double* __restrict__ partials, int m, GlobalDev* gdev)
{
    if (gdev->all_done) return;
    const int c = blockIdx.x, p = ch.prob[c];
    ProbDev& P = pd[p];
    if (skip_problem(P) || (pass == 1 && !P.reorth)) return;
    const int j = P.j, nv = j + 1, m1 = m + 1;
    __shared__ double hs[kMaxRestart + 1];
    __shared__ double sh[32];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = P.h[i];
    __syncthreads();
    const int sub0 = blockIdx.y * (kUpdE * kChunkThreads);
    const int64_t b0 = ch.beg[c] + sub0;
    const int len = ch.len[c] - sub0;  // may be <= 0 for the last chunk of a range
    double s[kUpdE];
#pragma unroll
    for (int q = 0; q < kUpdE; q++) {
        const int e = threadIdx.x + q * kChunkThreads;
        s[q] = e < len ? w[b0 + e] : 0.0;
    }
#pragma unroll 4
    for (int i = 0; i < nv; i++) {
        const TV* vi = V + (size_t)i * ld + b0;
        const double h = hs[i];
#pragma unroll
        for (int q = 0; q < kUpdE; q++) {
            const int e = threadIdx.x + q * kChunkThreads;
            if (e < len) s[q] = fma(-h, to_f64(vi[e]), s[q]);
        }
    }
    double a = 0.0;
#pragma unroll
    for (int q = 0; q < kUpdE; q++) {
        const int e = threadIdx.x + q * kChunkThreads;
        if (e < len) {
            w[b0 + e] = s[q];
            a = fma(s[q], s[q], a);
        }
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[(size_t)c * kUpdSub + blockIdx.y] = a;
    if (!last_of_problem(&P.ticket[1], (unsigned)ch.pcnt[p] * kUpdSub)) return;
    if (threadIdx.x < 32) {
        const double tot = sum_problem_partials(partials, ch.pbeg[p] * kUpdSub, ch.pcnt[p] * kUpdSub);
        if (threadIdx.x == 0) {
            if (pass == 1 || !P.reorth) {
                const double nrm = sqrt(tot);
                P.H[(j + 1) + (size_t)m1 * j] = nrm;
                P.inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
                givens_step(P, m, gdev);
            }
            P.ticket[1] = 0u;
        }
    }
}

// V_{j_p} = w * inv_p for the (already advanced) j_p of every problem whose cycle runs
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_scale_next(Chunks ch, const double* __restrict__ w,
                                                             const ProbDev* __restrict__ pd, const GlobalDev* __restrict__ gdev,
                                                             TV* __restrict__ V, size_t ld)
{
    if (gdev->all_done) return;
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    if (skip_problem(P)) return;
    const double s = P.inv;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    TV* out = V + (size_t)P.j * ld + b0;
    for (int q = threadIdx.x; q < len; q += kChunkThreads) out[q] = (TV)(w[b0 + q] * s);
}

// end of a lockstep iteration: the shared Arnoldi index advances
__global__ void k_iter_advance(GlobalDev* gdev)
{
    if (!gdev->all_done) gdev->jg++;
}

// one thread per problem: y = H^-1 g (upper triangular, k_p columns)
__global__ void k_solve_y(ProbDev* pd, int m, int nprob)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    ProbDev& P = pd[p];
    const int m1 = m + 1, k = P.k;
    for (int i = k - 1; i >= 0; i--) {
        double s = P.g[i];
        for (int q = i + 1; q < k; q++) s -= P.H[i + (size_t)m1 * q] * P.y[q];
        const double d = P.H[i + (size_t)m1 * i];
        P.y[i] = d != 0.0 ? s / d : 0.0;
    }
}

// out_p = sum_{i < k_p} y_i V_i (zero for problems without iterations)
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_combine(Chunks ch, const TV* __restrict__ V, size_t ld,
                                                          const ProbDev* __restrict__ pd, double* __restrict__ out)
{
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    __shared__ double ys[kMaxRestart];
    const int k = P.active ? P.k : 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = P.y[i];
    __syncthreads();
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) {
        double s = 0.0;
        for (int i = 0; i < k; i++) s = fma(ys[i], to_f64(V[(size_t)i * ld + b0 + q]), s);
        out[b0 + q] = s;
    }
}

__global__ void k_f2d(size_t n, const float* __restrict__ in, double* __restrict__ out)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = f2d(in[e]);
}

// ------------------------------------------------------------------ host wrappers
static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }
static inline int gsz(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)kRedBlocks * 4); }

static Chunks chunks(const jfnk_ctx* c) { return Chunks{c->ch_beg, c->ch_len, c->ch_prob, c->pch_beg, c->pch_cnt}; }

int build_chunks(jfnk_ctx* c)
{
    const int nc = c->dm.nc, P = c->nprob;
    std::vector<int64_t> beg;
    std::vector<int32_t> len, prob, pbeg(P), pcnt(P);
    for (int p = 0; p < P; p++) {
        pbeg[p] = (int32_t)beg.size();
        for (int k = 0; k < 3; k++) {
            const int64_t lo = (int64_t)k * nc + c->prob_c0[p], hi = (int64_t)k * nc + c->prob_c1[p];
            for (int64_t a = lo; a < hi; a += kChunk) {
                beg.push_back(a);
                len.push_back((int32_t)std::min<int64_t>(kChunk, hi - a));
                prob.push_back(p);
            }
        }
        pcnt[p] = (int32_t)beg.size() - pbeg[p];
    }
    c->n_chunks = (int)beg.size();
    auto up = [&](const void* h, size_t bytes) -> void* {
        void* d = jfnk_dalloc(c, std::max<size_t>(bytes, 8));
        if (d && bytes) cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
        return d;
    };
    c->ch_beg = (int64_t*)up(beg.data(), beg.size() * sizeof(int64_t));
    c->ch_len = (int32_t*)up(len.data(), len.size() * sizeof(int32_t));
    c->ch_prob = (int32_t*)up(prob.data(), prob.size() * sizeof(int32_t));
    c->pch_beg = (int32_t*)up(pbeg.data(), pbeg.size() * sizeof(int32_t));
    c->pch_cnt = (int32_t*)up(pcnt.data(), pcnt.size() * sizeof(int32_t));
    if (!c->ch_beg || !c->ch_len || !c->ch_prob || !c->pch_beg || !c->pch_cnt)
        return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the chunk table failed");
    return JFNK_OK;
}

int perm_in(jfnk_ctx* c, const double* ext, double* out)
{
    k_perm_in<<<nblk(c->dm.nc, 256), 256, 0, c->cur>>>(c->dm.nc, c->dm.dim, c->dm.n2o, ext, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int perm_out(jfnk_ctx* c, const double* in, double* ext)
{
    k_perm_out<<<nblk(c->dm.nc, 256), 256, 0, c->cur>>>(c->dm.nc, c->dm.n2o, in, ext);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int pnorm(jfnk_ctx* c, const double* x, int mode, bool gated)
{
    k_pnorm<<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), x, c->partials, c->pd, mode, c->opt.jv_eps_scale,
                                                        gated ? 1 : 0, c->gdev);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int axpby(jfnk_ctx* c, size_t n, double a, const double* x, double b, const double* y, double* out)
{
    k_axpby<<<gsz(n), 256, 0, c->cur>>>(n, a, x, b, y, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int perturb(jfnk_ctx* c, const double* u, const double* z, double* w, bool gated)
{
    k_perturb<<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), u, z, c->pd, c->gdev, gated ? 1 : 0, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int line_trial(jfnk_ctx* c, const double* u, const double* x, double* w)
{
    k_line_trial<<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), u, x, c->pd, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int accept_masked(jfnk_ctx* c, const int32_t* mask, double* u, const double* w, double* Ru, const double* R)
{
    k_accept<<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), mask, u, w, Ru, R);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int cycle_init(jfnk_ctx* c, const double* r)
{
    // beta_p = |r_p|, inv_p, per-problem cycle state, then V_0 = r / beta
    int rc = pnorm(c, r, 3, false);
    if (rc) return rc;
    k_cycle_init<<<c->nprob, 256, 0, c->cur>>>(c->pd, c->opt.gmres_restart);
    JF_LAUNCHED(c);
    k_cycle_count<<<1, 1, 0, c->cur>>>(c->pd, c->nprob, c->gdev);
    JF_LAUNCHED(c);
    if (c->V_is_float) k_scale_first<float><<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), r, c->pd, (float*)c->V);
    else k_scale_first<double><<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), r, c->pd, c->V);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int arnoldi_orthogonalise(jfnk_ctx* c, double* w)
{
    // classical Gram-Schmidt against V_0..V_j, repeated when needed; the final pass runs the
    // Givens step; then V_{j+1} = w / |w|; the lockstep index advances
    const int m = c->opt.gmres_restart;
    const int mode = c->opt.reorth;  // 0 selective, 1 always, 2 never
    const int sl_d = c->prof.enabled ? c->prof.slot("mdot") : -1;
    const int sl_u = c->prof.enabled ? c->prof.slot("update") : -1;
    const dim3 g_mdot((unsigned)c->n_chunks, (unsigned)(m + 1));
    for (int pass = 0; pass < 2; pass++) {
        jfnk_prof_begin(c, sl_d);
        if (c->V_is_float)
            k_mdot<float><<<g_mdot, kChunkThreads, 0, c->cur>>>(chunks(c), (const float*)c->V, c->V_ld, w, c->pd, pass, mode,
                                                                c->partials, m, c->gdev, c->n_chunks);
        else
            k_mdot<double><<<g_mdot, kChunkThreads, 0, c->cur>>>(chunks(c), c->V, c->V_ld, w, c->pd, pass, mode,
                                                                 c->partials, m, c->gdev, c->n_chunks);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, sl_d);
        jfnk_prof_begin(c, sl_u);
        if (c->V_is_float)
            k_update<float><<<dim3(c->n_chunks, kUpdSub), kChunkThreads, 0, c->cur>>>(chunks(c), (const float*)c->V, c->V_ld,
                                                                                      w, c->pd, pass, c->partials, m, c->gdev);
        else
            k_update<double><<<dim3(c->n_chunks, kUpdSub), kChunkThreads, 0, c->cur>>>(chunks(c), c->V, c->V_ld, w, c->pd,
                                                                                       pass, c->partials, m, c->gdev);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, sl_u);
    }
    if (c->V_is_float)
        k_scale_next<float><<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), w, c->pd, c->gdev, (float*)c->V, c->V_ld);
    else
        k_scale_next<double><<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), w, c->pd, c->gdev, c->V, c->V_ld);
    JF_LAUNCHED(c);
    k_iter_advance<<<1, 1, 0, c->cur>>>(c->gdev);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int cycle_solution(jfnk_ctx* c, double* out)
{
    k_solve_y<<<nblk(c->nprob, 64), 64, 0, c->cur>>>(c->pd, c->opt.gmres_restart, c->nprob);
    JF_LAUNCHED(c);
    if (c->V_is_float) k_combine<float><<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), (const float*)c->V, c->V_ld, c->pd, out);
    else k_combine<double><<<c->n_chunks, kChunkThreads, 0, c->cur>>>(chunks(c), c->V, c->V_ld, c->pd, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

}  // namespace jfnk

extern "C" int jfnk_convert_f32_to_f64(const float* in, double* out, int64_t n, void* stream)
{
    if ((!in || !out) && n > 0) return JFNK_EINVAL;
    if (n <= 0) return JFNK_OK;
    jfnk::k_f2d<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>((size_t)n, in, out);
    return cudaGetLastError() == cudaSuccess ? JFNK_OK : JFNK_ECUDA;
}
