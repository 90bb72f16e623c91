// Vector kernels of the JFNK loop: caller-order <-> internal-order permutation, FP64 norms
// and the Jv step eps (Eq. JF), and the Arnoldi process of right-preconditioned GMRES(m)
// (Sec. 3.2): fused multi-dot products, the Gram-Schmidt update fused with the norm of the
// new vector, Givens rotations and the small triangular solve, all resident on the device.
// Every reduction runs on a fixed grid with warp-shuffle trees and a last-block finalisation
// in fixed order, so results are bitwise reproducible.  Kernels of a GMRES cycle return at
// once when the device flag `done` is set (converged, breakdown or cycle full).
#include <algorithm>
#include <cmath>

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

// mode 0: *out = |x|;  mode 1: gd->eps = s (1 + gd->unorm) / |x| (0 when x = 0);
// mode 2: gd->unorm = |x|;  mode 3: gd->beta = |x|, gd->inv = 1/|x| (0 when x = 0)
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_norm(size_t n, const T* __restrict__ x, double* __restrict__ partials,
                                                     unsigned* ticket, int mode, double s, double* out, GmresDev* gd,
                                                     const int* gate)
{
    if (gate && *gate) return;
    __shared__ double sh[32];
    double a = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)x[e];
        a = fma(v, v, a);
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
    if (!last_block(ticket)) return;
    const double tot = reduce_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        const double nrm = sqrt(tot);
        if (mode == 0) *out = nrm;
        else if (mode == 1) gd->eps = (nrm > 0.0) ? s * (1.0 + gd->unorm) / nrm : 0.0;
        else if (mode == 2) gd->unorm = nrm;
        else { gd->beta = nrm; gd->inv = nrm > 0.0 ? 1.0 / nrm : 0.0; }
        *ticket = 0u;
    }
}

__global__ void k_axpby(size_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = fma(a, x[e], b * y[e]);
}

// w = u + eps z with eps read from the device (Eq. JF)
__global__ void k_perturb(const int* gate, size_t n, const double* __restrict__ u, const double* __restrict__ z,
                          const GmresDev* __restrict__ gd, double* __restrict__ w)
{
    if (gate && *gate) return;
    const double eps = gd->eps;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        w[e] = fma(eps, z[e], u[e]);
}

// ------------------------------------------------------------------ Arnoldi
__global__ void k_cycle_init(GmresDev* gd, int m)
{
    const int m1 = m + 1;
    for (int i = threadIdx.x; i < m1 * m; i += blockDim.x) gd->H[i] = 0.0;
    for (int i = threadIdx.x; i < m1; i += blockDim.x) gd->g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        gd->g[0] = gd->beta;
        gd->j = 0;
        gd->k = 0;
        gd->done = (gd->beta > 0.0) ? 0 : 1;
        gd->reorth = 0;
        gd->res = gd->beta;
    }
}

template <typename TV>
__global__ void k_scale_to(const int* gate, size_t n, const double* __restrict__ w, const GmresDev* __restrict__ gd,
                           TV* __restrict__ out)
{
    if (gate && *gate) return;
    const double s = gd->inv;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = (TV)(w[e] * s);
}

// Sum of NV per-block partial arrays by one block: warp q handles values q, q + nwarps, ...
__device__ __forceinline__ void finalize_values(const double* partials, int nblocks, int nvals, double* sums)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < nvals; i += nw) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += __ldcg(partials + (size_t)i * nblocks + b);
        s = warp_sum(s);
        if (lane == 0) sums[i] = s;
    }
    __syncthreads();
}

// Givens step on column j of H (in place), by one thread: rotations of the previous columns,
// the new rotation, g update, residual estimate; sets done when converged, on breakdown or
// when the cycle is full, and advances j.
__device__ void givens_step(GmresDev* gd, int m)
{
    const int m1 = m + 1, j = gd->j;
    double* H = gd->H + (size_t)m1 * j;
    const double hn = H[j + 1];
    for (int i = 0; i < j; i++) {
        const double t = gd->cs[i] * H[i] + gd->sn[i] * H[i + 1];
        H[i + 1] = -gd->sn[i] * H[i] + gd->cs[i] * H[i + 1];
        H[i] = t;
    }
    const double a = H[j], b = H[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    gd->cs[j] = c;
    gd->sn[j] = s;
    H[j] = r;
    H[j + 1] = 0.0;
    const double gj = gd->g[j];
    gd->g[j + 1] = -s * gj;
    gd->g[j] = c * gj;
    gd->k = j + 1;
    gd->res = fabs(gd->g[j + 1]);
    if (gd->res <= gd->target || hn == 0.0 || j + 1 >= m || !(gd->res == gd->res)) gd->done = 1;
    gd->j = j + 1;
}

// Multi-dot h_i = V_i . w (i <= j) and, in pass 0, |w|^2.  Grid: x = element chunks of
// kMdotThreads * kMdotE elements, y = one basis vector per block (so the GPU has many
// independent blocks in flight); each thread keeps kMdotE elements of w in registers and
// accumulates kMdotE products before the FP64 warp reduction.  Pass 1 runs only when the
// pass-0 test asked for re-orthogonalisation.
constexpr int kMdotThreads = 128, kMdotE = 32;

template <typename TV>
__global__ void __launch_bounds__(kMdotThreads) k_mdot(size_t n, const TV* __restrict__ V, size_t ld,
                                                      const double* __restrict__ w, GmresDev* gd, int pass,
                                                      int always_reorth, double* __restrict__ partials, int m1)
{
    if (gd->done) return;
    if (pass == 1 && !gd->reorth) return;
    const int j = gd->j, nv = j + 1;
    const int nvals = nv + (pass == 0 ? 1 : 0);
    const unsigned nblk = gridDim.x * gridDim.y;
    __shared__ double sh[kMdotThreads / 32];
    __shared__ double sums[kMaxRestart + 2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.y;
    if (i < nvals) {
        const size_t base = (size_t)blockIdx.x * (kMdotThreads * kMdotE) + threadIdx.x;
        double acc = 0.0;
        if (i < nv) {
            const TV* vi = V + (size_t)i * ld;
            TV vv[kMdotE];
#pragma unroll
            for (int q = 0; q < kMdotE; q++) {
                const size_t e = base + (size_t)q * kMdotThreads;
                vv[q] = e < n ? vi[e] : (TV)0;
            }
#pragma unroll
            for (int q = 0; q < kMdotE; q++) {
                const size_t e = base + (size_t)q * kMdotThreads;
                if (e < n) acc = fma(to_f64(vv[q]), w[e], acc);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kMdotE; q++) {
                const size_t e = base + (size_t)q * kMdotThreads;
                if (e < n) { const double x = w[e]; acc = fma(x, x, acc); }
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) sh[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int x = 0; x < kMdotThreads / 32; x++) s += sh[x];
            partials[(size_t)i * gridDim.x + blockIdx.x] = s;
        }
    }
    // last block: sum the per-chunk partials of every value (warp per value)
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&gd->ticket[0], 1u) == nblk - 1);
    __syncthreads();
    if (!is_last) return;
    for (int v = wid; v < nvals; v += kMdotThreads / 32) {
        double sacc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) sacc += __ldcg(partials + (size_t)v * gridDim.x + b);
        sacc = warp_sum(sacc);
        if (lane == 0) sums[v] = sacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double hh = 0.0;
        for (int v = 0; v < nv; v++) {
            gd->h[v] = sums[v];
            if (pass == 0) gd->H[v + (size_t)m1 * j] = sums[v];
            else gd->H[v + (size_t)m1 * j] += sums[v];
            hh += sums[v] * sums[v];
        }
        if (pass == 0) {
            const double wn2 = sums[nv];
            gd->wn2 = wn2;
            // classical Gram-Schmidt is repeated when the projection removed more than half
            // of |w|^2, i.e. |w'| < |w| / sqrt(2) (the 'twice is enough' test)
            gd->reorth = (always_reorth == 1 || (always_reorth == 0 && (wn2 - hh) < 0.5 * wn2)) ? 1 : 0;
        } else {
            gd->n_reorth++;
        }
        gd->ticket[0] = 0u;
    }
}

// w -= sum_i h_i V_i, then |w|.  The final pass stores H(j+1, j) = |w|, 1/|w| and runs the
// Givens step (which advances j).  Each thread updates kUpdE elements (independent chains).
constexpr int kUpdThreads = 256, kUpdE = 2;

template <typename TV>
__global__ void __launch_bounds__(kUpdThreads) k_update(size_t n, const TV* __restrict__ V, size_t ld,
                                                       double* __restrict__ w, GmresDev* gd, int pass,
                                                       double* __restrict__ partials, int m)
{
    if (gd->done) return;
    if (pass == 1 && !gd->reorth) return;
    const int j = gd->j, nv = j + 1, m1 = m + 1;
    __shared__ double hs[kMaxRestart + 1];
    __shared__ double sh[32];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = gd->h[i];
    __syncthreads();
    double a = 0.0;
    for (size_t base = (size_t)blockIdx.x * (kUpdThreads * kUpdE) + threadIdx.x; base < n;
         base += (size_t)gridDim.x * (kUpdThreads * kUpdE)) {
        double s[kUpdE];
#pragma unroll
        for (int q = 0; q < kUpdE; q++) {
            const size_t e = base + (size_t)q * kUpdThreads;
            s[q] = e < n ? w[e] : 0.0;
        }
#pragma unroll 4
        for (int i = 0; i < nv; i++) {
            const TV* vi = V + (size_t)i * ld;
            const double h = hs[i];
#pragma unroll
            for (int q = 0; q < kUpdE; q++) {
                const size_t e = base + (size_t)q * kUpdThreads;
                if (e < n) s[q] = fma(-h, to_f64(vi[e]), s[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kUpdE; q++) {
            const size_t e = base + (size_t)q * kUpdThreads;
            if (e < n) {
                w[e] = s[q];
                a = fma(s[q], s[q], a);
            }
        }
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
    if (!last_block(&gd->ticket[1])) return;
    const double tot = reduce_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        if (pass == 1 || !gd->reorth) {
            const double nrm = sqrt(tot);
            gd->H[(j + 1) + (size_t)m1 * j] = nrm;
            gd->inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
            givens_step(gd, m);
        }
        gd->ticket[1] = 0u;
    }
}

// V_{j} = w * inv for the (already advanced) j: the next basis vector
template <typename TV>
__global__ void k_scale_next(size_t n, const double* __restrict__ w, const GmresDev* __restrict__ gd, TV* __restrict__ V,
                             size_t ld)
{
    if (gd->done) return;
    const double s = gd->inv;
    TV* out = V + (size_t)gd->j * ld;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = (TV)(w[e] * s);
}

__global__ void k_solve_y(GmresDev* gd, int m)
{
    const int m1 = m + 1, k = gd->k;
    for (int i = k - 1; i >= 0; i--) {
        double s = gd->g[i];
        for (int q = i + 1; q < k; q++) s -= gd->H[i + (size_t)m1 * q] * gd->y[q];
        const double d = gd->H[i + (size_t)m1 * i];
        gd->y[i] = d != 0.0 ? s / d : 0.0;
    }
}

template <typename TV>
__global__ void k_combine(size_t n, const TV* __restrict__ V, size_t ld, const GmresDev* __restrict__ gd,
                          double* __restrict__ out)
{
    __shared__ double ys[kMaxRestart];
    const int k = gd->k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = gd->y[i];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; i++) s = fma(ys[i], to_f64(V[(size_t)i * ld + e]), s);
        out[e] = s;
    }
}

__global__ void k_f2d(size_t n, const float* __restrict__ in, double* __restrict__ out)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = f2d(in[e]);
}

// ------------------------------------------------------------------ host wrappers
static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }
static inline int gsz(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)kRedBlocks * 2); }

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

int norm2(jfnk_ctx* c, const double* x, size_t n, double* out_dev)
{
    k_norm<double><<<kRedBlocks, kRedThreads, 0, c->cur>>>(n, x, c->partials, c->tickets, 0, 0.0, out_dev, c->gd, nullptr);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int norm_mode(jfnk_ctx* c, const double* x, size_t n, int mode, const int* gate)
{
    k_norm<double><<<kRedBlocks, kRedThreads, 0, c->cur>>>(n, x, c->partials, c->tickets + 1, mode,
                                                           c->opt.jv_eps_scale, nullptr, c->gd, gate);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int axpby(jfnk_ctx* c, size_t n, double a, const double* x, double b, const double* y, double* out)
{
    k_axpby<<<gsz(n), 256, 0, c->cur>>>(n, a, x, b, y, out);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int perturb(jfnk_ctx* c, const double* u, const double* z, double* w, const int* gate)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    k_perturb<<<gsz(n), 256, 0, c->cur>>>(gate, n, u, z, c->gd, w);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int cycle_init(jfnk_ctx* c, const double* r)
{
    // beta = |r|, inv = 1/beta, then V_0 = r / beta
    const size_t n = 3 * (size_t)c->dm.nc;
    int rc = norm_mode(c, r, n, 3, nullptr);
    if (rc) return rc;
    k_cycle_init<<<1, 256, 0, c->cur>>>(c->gd, c->opt.gmres_restart);
    JF_LAUNCHED(c);
    if (c->V_is_float) k_scale_to<float><<<gsz(n), 256, 0, c->cur>>>(nullptr, n, r, c->gd, (float*)c->V);
    else k_scale_to<double><<<gsz(n), 256, 0, c->cur>>>(nullptr, n, r, c->gd, c->V);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int arnoldi_orthogonalise(jfnk_ctx* c, double* w)
{
    // classical Gram-Schmidt against V_0..V_j, repeated when needed; the final pass runs the
    // Givens step; then V_{j+1} = w / |w|
    const size_t n = 3 * (size_t)c->dm.nc;
    const int m = c->opt.gmres_restart, m1 = m + 1;
    const int always = c->opt.reorth;  // 0 selective, 1 always, 2 never
    int sl_d = c->prof.enabled ? c->prof.slot("mdot") : -1;
    int sl_u = c->prof.enabled ? c->prof.slot("update") : -1;
    const dim3 gd_mdot((unsigned)((n + kMdotThreads * kMdotE - 1) / (kMdotThreads * kMdotE)), (unsigned)(m + 1));
    const int gu = (int)std::min<size_t>((n + kUpdThreads * kUpdE - 1) / (kUpdThreads * kUpdE), (size_t)kRedBlocks * 4);
    for (int pass = 0; pass < 2; pass++) {
        jfnk_prof_begin(c, sl_d);
        if (c->V_is_float)
            k_mdot<float><<<gd_mdot, kMdotThreads, 0, c->cur>>>(n, (const float*)c->V, c->V_ld, w, c->gd, pass, always, c->partials, m1);
        else
            k_mdot<double><<<gd_mdot, kMdotThreads, 0, c->cur>>>(n, c->V, c->V_ld, w, c->gd, pass, always, c->partials, m1);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, sl_d);
        jfnk_prof_begin(c, sl_u);
        if (c->V_is_float)
            k_update<float><<<gu, kUpdThreads, 0, c->cur>>>(n, (const float*)c->V, c->V_ld, w, c->gd, pass, c->partials, m);
        else
            k_update<double><<<gu, kUpdThreads, 0, c->cur>>>(n, c->V, c->V_ld, w, c->gd, pass, c->partials, m);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, sl_u);
    }
    if (c->V_is_float) k_scale_next<float><<<gsz(n), 256, 0, c->cur>>>(n, w, c->gd, (float*)c->V, c->V_ld);
    else k_scale_next<double><<<gsz(n), 256, 0, c->cur>>>(n, w, c->gd, c->V, c->V_ld);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int cycle_solution(jfnk_ctx* c, double* out)
{
    const size_t n = 3 * (size_t)c->dm.nc;
    k_solve_y<<<1, 1, 0, c->cur>>>(c->gd, c->opt.gmres_restart);
    JF_LAUNCHED(c);
    if (c->V_is_float) k_combine<float><<<gsz(n), 256, 0, c->cur>>>(n, (const float*)c->V, c->V_ld, c->gd, out);
    else k_combine<double><<<gsz(n), 256, 0, c->cur>>>(n, c->V, c->V_ld, c->gd, out);
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
