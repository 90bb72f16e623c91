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
    JF_PDL_ENTRY();
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const size_t o = (size_t)n2o[P] * 3;
    out[P] = ext[o];
    out[nc + P] = ext[o + 1];
    out[2 * (size_t)nc + P] = dim == 2 ? 0.0 : ext[o + 2];
}

__global__ void k_perm_out(int nc, const int32_t* __restrict__ n2o, const double* __restrict__ in, double* __restrict__ ext)
{
    JF_PDL_ENTRY();
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
    JF_PDL_ENTRY();
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
    return ticket_last(ticket, expected);
}

// Sum of one problem's chunk partials (fixed order), by one warp; valid in lane 0.
__device__ __forceinline__ double sum_problem_partials(const double* partials, int first, int count)
{
    return warp_sum_strided(partials + first, count);
}

// ------------------------------------------------------------------ per-problem norms
// mode 0: nrm = |x_p|;  1: eps = s (1 + unorm) / |x_p| (0 for x_p = 0);  2: unorm = |x_p|;
// 3: beta = |x_p|, inv = 1/beta (0 for beta = 0);  4: unorm = |x_p| and eps = s (1 + unorm),
// the step for a unit direction (the Arnoldi vectors of left-preconditioned GMRES)
__global__ void __launch_bounds__(kChunkThreads) k_pnorm(Chunks ch, const double* __restrict__ x,
                                                        double* __restrict__ partials, ProbDev* pd, int mode,
                                                        double s, int gated, const GlobalDev* gdev)
{
    JF_PDL_ENTRY();
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
            else if (mode == 1) {
                P.eps = (nrm > 0.0) ? s * (1.0 + P.unorm) / nrm : 0.0;
                P.ieps = P.eps != 0.0 ? 1.0 / P.eps : 0.0;
            }
            else if (mode == 2) P.unorm = nrm;
            else if (mode == 4) {
                P.unorm = nrm;
                P.eps = s * (1.0 + nrm);
                P.ieps = 1.0 / P.eps;
            }
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
    JF_PDL_ENTRY();
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
    JF_PDL_ENTRY();
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
    JF_PDL_ENTRY();
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
// w = u + eps_p V_j with j = *jidx (the current Arnoldi vector, unit norm), active problems
// whose cycle runs: the perturbed state of a left-preconditioned Arnoldi column
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_perturb_basis(Chunks ch, const double* __restrict__ u,
                                                                const TV* __restrict__ V, size_t ld,
                                                                const int* __restrict__ jidx,
                                                                const ProbDev* __restrict__ pd,
                                                                const GlobalDev* __restrict__ gdev, double* __restrict__ w)
{
    JF_PDL_ENTRY();
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    if (gdev->all_done || skip_problem(P)) return;
    const double eps = P.eps;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    const TV* v = V + (size_t)(*jidx) * ld + b0;
    for (int q = threadIdx.x; q < len; q += kChunkThreads) w[b0 + q] = fma(eps, to_f64(v[q]), u[b0 + q]);
}

// One block per problem: start a cycle (beta and inv already computed).
__global__ void k_cycle_init(ProbDev* pd, int m)
{
    JF_PDL_ENTRY();
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
    JF_PDL_ENTRY();
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
    JF_PDL_ENTRY();
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

// ------------------------------------------------------------------ Arnoldi kernels
// One block of kArnThreads per chunk.  The FP64 pipe bounds this step on GB300, so the
// reductions are laid out to spend it on the products: a dot product of one basis vector
// with the chunk is taken by one warp (64 products per lane, lane-strided so the basis loads
// coalesce, the chunk of w read from shared memory) and closed by one warp reduction, rather
// than every thread forming partial sums of every dot.
constexpr int kArnThreads = 512;
constexpr int kArnE = kChunk / kArnThreads;  // elements per thread in the update
constexpr int kArnW = kArnThreads / 32;

// sum_e v[e] ws[e] over e < len by one warp (fixed order, four accumulators); lane 0
template <typename TV>
__device__ __forceinline__ double warp_dot_chunk(const TV* __restrict__ v, const double* ws, int len)
{
    const int lane = threadIdx.x & 31;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int e = lane;
#pragma unroll 4
    for (; e + 96 < len; e += 128) {
        a0 = fma(to_f64(v[e]), ws[e], a0);
        a1 = fma(to_f64(v[e + 32]), ws[e + 32], a1);
        a2 = fma(to_f64(v[e + 64]), ws[e + 64], a2);
        a3 = fma(to_f64(v[e + 96]), ws[e + 96], a3);
    }
    for (; e < len; e += 32) a0 = fma(to_f64(v[e]), ws[e], a0);
    return warp_sum((a0 + a1) + (a2 + a3));
}

// Pass-0 multi-dot of classical Gram-Schmidt: h_i = V_i . w (i <= j) and |w|^2 (value nv),
// per problem.  The last block of a problem stores h and the Hessenberg column and decides
// whether the projection is repeated.
template <typename TV>
__global__ void __launch_bounds__(kArnThreads) k_mdot(Chunks ch, const TV* __restrict__ V, size_t ld,
                                                     const double* __restrict__ w, ProbDev* pd, int reorth_mode,
                                                     double* __restrict__ partials, int m,
                                                     const GlobalDev* __restrict__ gdev, int nchunks)
{
    JF_PDL_ENTRY();
    if (gdev->all_done) return;
    const int c = blockIdx.x, p = ch.prob[c];
    ProbDev& P = pd[p];
    if (skip_problem(P)) return;
    const int j = P.j, nv = j + 1, nvals = nv + 1, m1 = m + 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ double ws[kChunk];
    __shared__ double sums[kMaxRestart + 2];
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int e = threadIdx.x; e < len; e += kArnThreads) ws[e] = w[b0 + e];
    __syncthreads();
    for (int i = wid; i < nvals; i += kArnW) {
        const double d = (i < nv) ? warp_dot_chunk(V + (size_t)i * ld + b0, ws, len) : warp_dot_chunk((const double*)ws, ws, len);
        if (lane == 0) partials[(size_t)i * nchunks + c] = d;
    }
    if (!last_of_problem(&P.ticket[0], (unsigned)ch.pcnt[p])) return;
    const int first = ch.pbeg[p], nch = ch.pcnt[p];
    for (int v = wid; v < nvals; v += kArnW) {
        const double t = warp_sum_strided(partials + (size_t)v * nchunks + first, nch);
        if (lane == 0) sums[v] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double hh = 0.0;
        for (int v = 0; v < nv; v++) {
            P.h[v] = sums[v];
            P.H[v + (size_t)m1 * j] = sums[v];
            hh += sums[v] * sums[v];
        }
        const double wn2 = sums[nv];
        P.wn2 = wn2;
        P.n_cols += nv;
        // the projection is repeated when it removed more than half of |w|^2, i.e.
        // |w'| < |w| / sqrt(2) (the 'twice is enough' test), or always / never by option
        P.reorth = (reorth_mode == 1 || (reorth_mode == 0 && (wn2 - hh) < 0.5 * wn2)) ? 1 : 0;
        P.ticket[0] = 0u;
    }
}

// w -= sum_i h_i V_i, each thread updating kArnE elements as independent FMA chains.  Pass 0
// of a problem that repeats the projection also forms that repetition's dots h'_i = V_i . w'
// from the updated chunk, staged in shared memory (the second multi-dot needs no pass over w
// of its own); the last block stores h' and adds it to the Hessenberg column.  Otherwise
// (pass 0 without repetition, or pass 1) the block sums |w|^2 and the last block stores
// H(j+1, j) = |w|, 1/|w| and runs the Givens step.
template <typename TV>
__global__ void __launch_bounds__(kArnThreads) k_update(Chunks ch, const TV* __restrict__ V, size_t ld,
                                                       double* __restrict__ w, ProbDev* pd, int pass,
                                                       double* __restrict__ partials, int m, GlobalDev* gdev)
{
    JF_PDL_ENTRY();
    if (gdev->all_done) return;
    const int c = blockIdx.x, p = ch.prob[c];
    ProbDev& P = pd[p];
    if (skip_problem(P) || (pass == 1 && !P.reorth)) return;
    const int j = P.j, nv = j + 1, m1 = m + 1;
    const bool dots = (pass == 0 && P.reorth);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t nchunks = gridDim.x;
    __shared__ double hs[kMaxRestart + 1];
    __shared__ double sh[kArnW];
    __shared__ double ws[kChunk];
    __shared__ double sums[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = P.h[i];
    __syncthreads();
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    double s[kArnE];
#pragma unroll
    for (int q = 0; q < kArnE; q++) {
        const int e = threadIdx.x + q * kArnThreads;
        s[q] = e < len ? w[b0 + e] : 0.0;
    }
#pragma unroll 4
    for (int i = 0; i < nv; i++) {
        const TV* vi = V + (size_t)i * ld + b0;
        const double h = hs[i];
#pragma unroll
        for (int q = 0; q < kArnE; q++) {
            const int e = threadIdx.x + q * kArnThreads;
            if (e < len) s[q] = fma(-h, to_f64(vi[e]), s[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kArnE; q++) {
        const int e = threadIdx.x + q * kArnThreads;
        if (e < len) w[b0 + e] = s[q];
    }
    if (dots) {
#pragma unroll
        for (int q = 0; q < kArnE; q++) {
            const int e = threadIdx.x + q * kArnThreads;
            if (e < len) ws[e] = s[q];
        }
        __syncthreads();
        for (int i = wid; i < nv; i += kArnW) {
            const double d = warp_dot_chunk(V + (size_t)i * ld + b0, ws, len);
            if (lane == 0) partials[(size_t)i * nchunks + c] = d;
        }
    } else {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < kArnE; q++) a = fma(s[q], s[q], a);  // s[q] = 0 past the end
        a = block_sum(a, sh);
        if (threadIdx.x == 0) partials[c] = a;
    }
    if (!last_of_problem(&P.ticket[1], (unsigned)ch.pcnt[p])) return;
    const int first = ch.pbeg[p], cnt = ch.pcnt[p];
    if (dots) {
        for (int v = wid; v < nv; v += kArnW) {
            const double t = warp_sum_strided(partials + (size_t)v * nchunks + first, cnt);
            if (lane == 0) sums[v] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int v = 0; v < nv; v++) {
                P.h[v] = sums[v];
                P.H[v + (size_t)m1 * j] += sums[v];
            }
            P.n_reorth++;
            P.n_rcols += nv;
            P.ticket[1] = 0u;
        }
    } else if (threadIdx.x < 32) {
        const double tot = sum_problem_partials(partials, first, cnt);
        if (threadIdx.x == 0) {
            const double nrm = sqrt(tot);
            P.H[(j + 1) + (size_t)m1 * j] = nrm;
            P.inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
            givens_step(P, m, gdev);
            P.ticket[1] = 0u;
        }
    }
}

// End of a lockstep iteration: V_{j_p} = w * inv_p for the (already advanced) j_p of every
// problem whose cycle runs; block 0 advances the shared Arnoldi index and stores the
// `all done` flag into the host's mapped mirror, which the host polls two iterations behind.
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_scale_next(Chunks ch, const double* __restrict__ w,
                                                             const ProbDev* __restrict__ pd, GlobalDev* gdev,
                                                             TV* __restrict__ V, size_t ld, GlobalDev* gh_dev)
{
    JF_PDL_ENTRY();
    const int all_done = *(volatile int*)&gdev->all_done;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!all_done) gdev->jg++;
        if (gh_dev) {
            *(volatile int*)&gh_dev->all_done = all_done;
            __threadfence_system();
        }
    }
    if (all_done) return;
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    if (skip_problem(P)) return;
    const double s = P.inv;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    TV* out = V + (size_t)P.j * ld + b0;
    for (int q = threadIdx.x; q < len; q += kChunkThreads) out[q] = (TV)(w[b0 + q] * s);
}

// one thread per problem: y = H^-1 g (upper triangular, k_p columns)
__global__ void k_solve_y(ProbDev* pd, int m, int nprob)
{
    JF_PDL_ENTRY();
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

// out_p = sum_{i < k_p} y_i V_i (zero for problems without iterations); grid as k_update
template <typename TV>
__global__ void __launch_bounds__(kChunkThreads) k_combine(Chunks ch, const TV* __restrict__ V, size_t ld,
                                                          const ProbDev* __restrict__ pd, int ncols, double* __restrict__ out)
{
    JF_PDL_ENTRY();
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    __shared__ double ys[kMaxRestart];
    const int k = P.active ? min(P.k, ncols) : 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = P.y[i];
    __syncthreads();
    const int sub0 = blockIdx.y * (kUpdE * kChunkThreads);
    const int64_t b0 = ch.beg[c] + sub0;
    const int len = ch.len[c] - sub0;
    double s[kUpdE];
#pragma unroll
    for (int q = 0; q < kUpdE; q++) s[q] = 0.0;
#pragma unroll 4
    for (int i = 0; i < k; i++) {
        const TV* vi = V + (size_t)i * ld + b0;
        const double y = ys[i];
#pragma unroll
        for (int q = 0; q < kUpdE; q++) {
            const int e = threadIdx.x + q * kChunkThreads;
            if (e < len) s[q] = fma(y, to_f64(vi[e]), s[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kUpdE; q++) {
        const int e = threadIdx.x + q * kChunkThreads;
        if (e < len) out[b0 + e] = s[q];
    }
}

// ------------------------------------------------------------------ loose GMRES (Sec. 4.2)
// The correction d of the last cycle is kept as z = d / |d_p| with J z = (r_prev - r) / |d_p|
// (r_prev, r: residuals at the start of the last and of this cycle), |d_p| from k_pnorm mode 0.
__global__ void __launch_bounds__(kChunkThreads) k_aug_store(Chunks ch, const double* __restrict__ d,
                                                            const double* __restrict__ rprev,
                                                            const double* __restrict__ r,
                                                            const ProbDev* __restrict__ pd, double* __restrict__ Z,
                                                            double* __restrict__ AZ)
{
    JF_PDL_ENTRY();
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    const double s = P.nrm > 0.0 ? 1.0 / P.nrm : 0.0;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) {
        Z[b0 + q] = d[b0 + q] * s;
        AZ[b0 + q] = (rprev[b0 + q] - r[b0 + q]) * s;
    }
}

// w = J z_l: the Arnoldi column of a kept correction needs no new product
__global__ void k_aug_load(size_t n, const double* __restrict__ AZ, const GlobalDev* __restrict__ gdev,
                           double* __restrict__ w)
{
    JF_PDL_ENTRY();
    if (gdev->all_done) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) w[e] = AZ[e];
}

constexpr int kMaxAug = 8;
struct AugSlots {
    const double* z[kMaxAug];
};

// out_p = zin_p + sum_l y_{ncols + l} z_l over the kept corrections whose columns ran
__global__ void __launch_bounds__(kChunkThreads) k_aug_add(Chunks ch, const ProbDev* __restrict__ pd, AugSlots Z, int na,
                                                          int ncols, const double* __restrict__ zin,
                                                          double* __restrict__ out)
{
    JF_PDL_ENTRY();
    const int c = blockIdx.x;
    const ProbDev& P = pd[ch.prob[c]];
    const int k = P.active ? P.k : 0;
    __shared__ double ya[kMaxAug];
    if (threadIdx.x < kMaxAug)
        ya[threadIdx.x] = ((int)threadIdx.x < na && ncols + (int)threadIdx.x < k) ? P.y[ncols + threadIdx.x] : 0.0;
    __syncthreads();
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    // a problem out of the iteration gets no correction (its zin may be a pass it sat out)
    for (int q = threadIdx.x; q < len; q += kChunkThreads) {
        double a = P.active ? zin[b0 + q] : 0.0;
        for (int l = 0; l < na; l++) a = fma(ya[l], Z.z[l][b0 + q], a);
        out[b0 + q] = a;
    }
}

// x += d for the problems that are active (the others' d may be a pass they sat out)
__global__ void __launch_bounds__(kChunkThreads) k_add_active(Chunks ch, const ProbDev* __restrict__ pd,
                                                             const double* __restrict__ d, double* __restrict__ x)
{
    JF_PDL_ENTRY();
    const int c = blockIdx.x;
    if (!pd[ch.prob[c]].active) return;
    const int64_t b0 = ch.beg[c];
    const int len = ch.len[c];
    for (int q = threadIdx.x; q < len; q += kChunkThreads) x[b0 + q] += d[b0 + q];
}

__global__ void k_f2d(size_t n, const float* __restrict__ in, double* __restrict__ out)
{
    JF_PDL_ENTRY();
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
        if (d && jfnk_upload(c, d, h, bytes)) return (void*)nullptr;
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
    jfnk_launch(c, k_perm_in, dim3(nblk(c->dm.nc, 256)), dim3(256), c->dm.nc, c->dm.dim, c->dm.n2o, ext, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int perm_out(jfnk_ctx* c, const double* in, double* ext)
{
    jfnk_launch(c, k_perm_out, dim3(nblk(c->dm.nc, 256)), dim3(256), c->dm.nc, c->dm.n2o, in, ext);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int pnorm(jfnk_ctx* c, const double* x, int mode, bool gated)
{
    jfnk_launch(c, k_pnorm, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), x, c->partials, c->pd, mode, c->opt.jv_eps_scale,
                                                        gated ? 1 : 0, c->gdev);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int axpby(jfnk_ctx* c, size_t n, double a, const double* x, double b, const double* y, double* out)
{
    jfnk_launch(c, k_axpby, dim3(gsz(n)), dim3(256), n, a, x, b, y, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int perturb(jfnk_ctx* c, const double* u, const double* z, double* w, bool gated)
{
    jfnk_launch(c, k_perturb, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), u, z, c->pd, c->gdev, gated ? 1 : 0, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int perturb_basis(jfnk_ctx* c, const double* u, double* w)
{
    if (c->V_is_float)
        jfnk_launch(c, k_perturb_basis<float>, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), u, (const float*)c->V,
                    c->V_ld, (const int*)&c->gdev->jg, (const ProbDev*)c->pd, (const GlobalDev*)c->gdev, w);
    else
        jfnk_launch(c, k_perturb_basis<double>, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), u, (const double*)c->V,
                    c->V_ld, (const int*)&c->gdev->jg, (const ProbDev*)c->pd, (const GlobalDev*)c->gdev, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int line_trial(jfnk_ctx* c, const double* u, const double* x, double* w)
{
    jfnk_launch(c, k_line_trial, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), u, x, c->pd, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int accept_masked(jfnk_ctx* c, const int32_t* mask, double* u, const double* w, double* Ru, const double* R)
{
    jfnk_launch(c, k_accept, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), mask, u, w, Ru, R);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int cycle_init(jfnk_ctx* c, const double* r)
{
    // beta_p = |r_p|, inv_p, per-problem cycle state, then V_0 = r / beta
    int rc = pnorm(c, r, 3, false);
    if (rc) return rc;
    jfnk_launch(c, k_cycle_init, dim3(c->nprob), dim3(256), c->pd, c->opt.gmres_restart);
    JF_LAUNCHED(c);
    jfnk_launch(c, k_cycle_count, dim3(1), dim3(1), c->pd, c->nprob, c->gdev);
    JF_LAUNCHED(c);
    if (c->V_is_float) jfnk_launch(c, k_scale_first<float>, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), r, c->pd, (float*)c->V);
    else jfnk_launch(c, k_scale_first<double>, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), r, c->pd, c->V);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int arnoldi_orthogonalise(jfnk_ctx* c, double* w)
{
    // classical Gram-Schmidt against V_0..V_j: multi-dot, update (which also forms the dots of
    // the repeated projection where the test asks for it), the repeated update; the final
    // update runs the Givens step; then V_{j+1} = w / |w| and the lockstep index advances
    const int m = c->opt.gmres_restart;
    const int mode = c->opt.reorth;  // 0 selective, 1 always, 2 never
    const int sl_d = c->prof.enabled ? c->prof.slot("mdot") : -1;
    const int sl_u = c->prof.enabled ? c->prof.slot("update") : -1;
    jfnk_prof_begin(c, sl_d);
    if (c->V_is_float)
        jfnk_launch(c, k_mdot<float>, dim3(c->n_chunks), dim3(kArnThreads), chunks(c), (const float*)c->V, c->V_ld, w, c->pd, mode,
                    c->partials, m, c->gdev, c->n_chunks);
    else
        jfnk_launch(c, k_mdot<double>, dim3(c->n_chunks), dim3(kArnThreads), chunks(c), (const double*)c->V, c->V_ld, w, c->pd, mode,
                    c->partials, m, c->gdev, c->n_chunks);
    JF_LAUNCHED(c);
    jfnk_prof_end(c, sl_d);
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1 && mode == 2) break;  // never repeated
        jfnk_prof_begin(c, sl_u);
        if (c->V_is_float)
            jfnk_launch(c, k_update<float>, dim3(c->n_chunks), dim3(kArnThreads), chunks(c), (const float*)c->V, c->V_ld, w, c->pd, pass,
                        c->partials, m, c->gdev);
        else
            jfnk_launch(c, k_update<double>, dim3(c->n_chunks), dim3(kArnThreads), chunks(c), (const double*)c->V, c->V_ld, w, c->pd, pass,
                        c->partials, m, c->gdev);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, sl_u);
    }
    if (c->V_is_float)
        jfnk_launch(c, k_scale_next<float>, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), (const double*)w, (const ProbDev*)c->pd,
                    c->gdev, (float*)c->V, c->V_ld, c->gh_dev);
    else
        jfnk_launch(c, k_scale_next<double>, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), (const double*)w, (const ProbDev*)c->pd,
                    c->gdev, c->V, c->V_ld, c->gh_dev);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int cycle_solution(jfnk_ctx* c, double* out, int ncols)
{
    jfnk_launch(c, k_solve_y, dim3(nblk(c->nprob, 64)), dim3(64), c->pd, c->opt.gmres_restart, c->nprob);
    JF_LAUNCHED(c);
    const dim3 g_upd((unsigned)c->n_chunks, (unsigned)kUpdSub);
    if (c->V_is_float) jfnk_launch(c, k_combine<float>, g_upd, dim3(kChunkThreads), chunks(c), (const float*)c->V, c->V_ld, (const ProbDev*)c->pd, ncols, out);
    else jfnk_launch(c, k_combine<double>, g_upd, dim3(kChunkThreads), chunks(c), (const double*)c->V, c->V_ld, (const ProbDev*)c->pd, ncols, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int aug_store(jfnk_ctx* c, int slot, const double* r)
{
    const size_t v3 = 3 * (size_t)c->dm.nc;
    int rc = pnorm(c, c->dcorr, 0, false);
    if (rc) return rc;
    jfnk_launch(c, k_aug_store, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), (const double*)c->dcorr,
                (const double*)c->rprev, r, (const ProbDev*)c->pd, c->Zaug + (size_t)slot * v3, c->AZaug + (size_t)slot * v3);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int aug_load(jfnk_ctx* c, int slot, double* w)
{
    const size_t v3 = 3 * (size_t)c->dm.nc;
    jfnk_launch(c, k_aug_load, dim3(gsz(v3)), dim3(256), v3, (const double*)(c->AZaug + (size_t)slot * v3),
                (const GlobalDev*)c->gdev, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int add_active(jfnk_ctx* c, const double* d, double* x)
{
    jfnk_launch(c, k_add_active, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), (const ProbDev*)c->pd, d, x);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int aug_add(jfnk_ctx* c, const int* slots, int na, int ncols, const double* z, double* out)
{
    const size_t v3 = 3 * (size_t)c->dm.nc;
    AugSlots Z{};
    for (int l = 0; l < na && l < kMaxAug; l++) Z.z[l] = c->Zaug + (size_t)slots[l] * v3;
    jfnk_launch(c, k_aug_add, dim3(c->n_chunks), dim3(kChunkThreads), chunks(c), (const ProbDev*)c->pd, Z, na, ncols, z, out);
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
