// Preconditioners of Sec. 3.2 built from the compact-stencil approximate Jacobian J~ of
// Sec. 3.1 (one scalar matrix shared by the displacement components):
//   block-Jacobi  z_P = [J~]_PP^-1 v_P  (a scalar per cell without symmetry faces);
//   multigrid     one V-cycle of an aggregation AMG on A = -J~ (the paper uses BoomerAMG,
//                 one V-cycle per Krylov iteration with one pre- and one post-sweep;
//                 Sec. 4.2).  The fine level is applied matrix-free over the cells'
//                 sliced-ELL neighbour slots with a per-slot copy of the J~ face
//                 coefficient; coarse levels are CSR rows taken by lane groups; the
//                 coarsest is a dense inverse.  All three components go through each level
//                 in one pass.
// Arithmetic: FP64 (precision FP64) or FP32 (precision MIXED: matrix, smoother, V-cycle).
// FP32 runs on the wide FP32 pipe of GB300, FP64 on a pipe ~64x narrower.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {


// ------------------------------------------------------------------ block-Jacobi
template <typename TV, typename TP>
__global__ void k_bjacobi(const int* gate, int nc, const TV* __restrict__ base, size_t ld, const int* __restrict__ jidx,
                          const TP* __restrict__ dinv, double* __restrict__ z)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const TV* v = jidx ? base + (size_t)(*jidx) * ld : base;
    const TP d = dinv[P];
#pragma unroll
    for (int k = 0; k < 3; k++) z[(size_t)k * nc + P] = to_f64((TP)v[(size_t)k * nc + P] * d);
}

// block-Jacobi with the 3x3 diagonal blocks of cells on symmetry faces (symmetric inverse
// [6][nc]: xx xy xz yy yz zz; the other cells' blocks are diag I)
template <typename TV, typename TP>
__global__ void k_bjacobi_block(const int* gate, int nc, const TV* __restrict__ base, size_t ld, const int* __restrict__ jidx,
                                const TP* __restrict__ binv, double* __restrict__ z)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const TV* v = jidx ? base + (size_t)(*jidx) * ld : base;
    const TP v0 = (TP)v[P], v1 = (TP)v[nc + P], v2 = (TP)v[2 * (size_t)nc + P];
    const TP b0 = binv[P], b1 = binv[nc + P], b2 = binv[2 * (size_t)nc + P];
    const TP b3 = binv[3 * (size_t)nc + P], b4 = binv[4 * (size_t)nc + P], b5 = binv[5 * (size_t)nc + P];
    z[P] = to_f64(b0 * v0 + b1 * v1 + b2 * v2);
    z[nc + P] = to_f64(b1 * v0 + b3 * v1 + b4 * v2);
    z[2 * (size_t)nc + P] = to_f64(b2 * v0 + b4 * v1 + b5 * v2);
}

template <typename TV>
__global__ void k_copy_vec(const int* gate, int nc, const TV* __restrict__ base, size_t ld, const int* __restrict__ jidx,
                           double* __restrict__ z)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const TV* v = jidx ? base + (size_t)(*jidx) * ld : base;
#pragma unroll
    for (int k = 0; k < 3; k++) z[(size_t)k * nc + P] = to_f64(v[(size_t)k * nc + P]);
}

template <typename TV>
__global__ void k_copy_to_double(const int* gate, size_t n, const TV* __restrict__ v, double* __restrict__ z)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        z[e] = to_f64(v[e]);
}

// ------------------------------------------------------------------ multigrid kernels
// Fine level (A = -J~, matrix-free):
//   (A x)_P = -diag_P x_P - sum_{internal faces f of P} c_f x_other(f)
// over the cell's sliced-ELL neighbour slots (32 cells per slice, slot-major, so a warp's
// loads coalesce), with the face coefficient copied per slot: one round of index and
// coefficient loads and one of neighbour values, instead of walking the owner and neighbour
// face lists (three to four dependent loads a face).  Padding (-1) and mirror neighbours of
// symmetry faces (>= nc, not part of the scalar multigrid operator) are skipped.
constexpr int kSellUnroll = 8;  // slots taken in one unrolled round (hexahedra have 6)

template <typename T, typename F>
__device__ __forceinline__ void for_sell_slots(int P, int nc, const int32_t* __restrict__ sell_off,
                                               const int32_t* __restrict__ sell_w, const int32_t* __restrict__ sell_nbr,
                                               const T* __restrict__ sc, F&& f)
{
    const int sl = P >> 5, lane = P & 31, base = sell_off[sl], w = sell_w[sl];
    // all index and coefficient loads of the first kSellUnroll slots first, so that they are
    // in flight together, then the neighbour terms in slot order
    int Ns[kSellUnroll];
    T cs[kSellUnroll];
#pragma unroll
    for (int k = 0; k < kSellUnroll; k++) {
        const int slot = base + 32 * k + lane;
        Ns[k] = k < w ? sell_nbr[slot] : -1;
        cs[k] = k < w ? sc[slot] : (T)0;
    }
#pragma unroll
    for (int k = 0; k < kSellUnroll; k++)
        if ((unsigned)Ns[k] < (unsigned)nc) f(Ns[k], cs[k]);
    for (int k = kSellUnroll; k < w; k++) {
        const int slot = base + 32 * k + lane;
        const int N = sell_nbr[slot];
        const T cf = sc[slot];
        if ((unsigned)N < (unsigned)nc) f(N, cf);
    }
}

template <typename T>
__device__ __forceinline__ void a0_row(int P, int nc, const int32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_w,
                                       const int32_t* __restrict__ sell_nbr, const T* __restrict__ sc,
                                       const T* __restrict__ adiag, const T* __restrict__ x, T out[3])
{
    const T d = adiag[P];
    out[0] = d * x[P]; out[1] = d * x[nc + P]; out[2] = d * x[2 * (size_t)nc + P];
    for_sell_slots<T>(P, nc, sell_off, sell_w, sell_nbr, sc, [&](int N, T cf) {
        out[0] -= cf * x[N]; out[1] -= cf * x[nc + N]; out[2] -= cf * x[2 * (size_t)nc + N];
    });
}

// one CSR row, the first kCsrUnroll entries' column indices and values loaded together
constexpr int kCsrUnroll = 8;

template <typename T>
__device__ __forceinline__ void csr_row(int i, int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                        const T* __restrict__ val, const T* __restrict__ x, int nx, T out[3])
{
    out[0] = out[1] = out[2] = (T)0;
    const int a = rp[i], b = rp[i + 1];
    int js[kCsrUnroll];
    T as[kCsrUnroll];
#pragma unroll
    for (int q = 0; q < kCsrUnroll; q++) {
        js[q] = a + q < b ? col[a + q] : 0;
        as[q] = a + q < b ? val[a + q] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < kCsrUnroll; q++)
        if (a + q < b) {
            const int j = js[q];
            out[0] += as[q] * x[j]; out[1] += as[q] * x[nx + j]; out[2] += as[q] * x[2 * (size_t)nx + j];
        }
    for (int q = a + kCsrUnroll; q < b; q++) {
        const int j = col[q];
        const T v = val[q];
        out[0] += v * x[j]; out[1] += v * x[nx + j]; out[2] += v * x[2 * (size_t)nx + j];
    }
    (void)n;
}

// Operator of one level: the fine level from per-slot face coefficients, coarse levels from CSR.
template <typename T>
struct LevelOp {
    int n;
    bool fine;
    const int32_t *p0, *p1, *p2;  // fine: sell_off, sell_w, sell_nbr; coarse: rp, col
    const T *vals, *adiag, *dinv;  // vals: fine per-slot coefficients, coarse CSR values
    __device__ __forceinline__ void row(int i, const T* x, T out[3]) const
    {
        if (fine) a0_row<T>(i, n, p0, p1, p2, vals, adiag, x, out);
        else csr_row<T>(i, n, p0, p1, vals, x, n, out);
    }
};

// Vectors of the coarse levels, and the finest level's residual, are interleaved: row i holds
// (x, y, z, 0) in p[4i .. 4i+3], so that a gathered row is one 16-byte load (FP32; two in FP64)
// instead of three loads from three arrays, each touching its own 32-byte sector.  The finest
// level's b and x stay component-major [3][n] like the Krylov vectors they come from and go to.
__device__ __forceinline__ void ld3(const float* __restrict__ p, int i, float& a, float& b, float& c)
{
    const float4 v = reinterpret_cast<const float4*>(p)[i];
    a = v.x; b = v.y; c = v.z;
}
__device__ __forceinline__ void ld3(const double* __restrict__ p, int i, double& a, double& b, double& c)
{
    const double2 v = reinterpret_cast<const double2*>(p)[2 * i];
    a = v.x; b = v.y; c = p[4 * (size_t)i + 2];
}
__device__ __forceinline__ void st3(float* __restrict__ p, int i, float a, float b, float c)
{
    reinterpret_cast<float4*>(p)[i] = make_float4(a, b, c, 0.0f);
}
__device__ __forceinline__ void st3(double* __restrict__ p, int i, double a, double b, double c)
{
    reinterpret_cast<double2*>(p)[2 * i] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[2 * i + 1] = make_double2(c, 0.0);
}
// component-major [3][n] access with the same signature
template <typename T>
__device__ __forceinline__ void ld3_soa(const T* __restrict__ p, size_t n, int i, T& a, T& b, T& c)
{
    a = p[i]; b = p[n + i]; c = p[2 * n + i];
}
template <typename T>
__device__ __forceinline__ void st3_soa(T* __restrict__ p, size_t n, int i, T a, T b, T c)
{
    p[i] = a; p[n + i] = b; p[2 * n + i] = c;
}

// level 0 entry: b = -v (so the cycle returns z = -A^-1 v = J~^-1 v), x = omega D^-1 b.
// v = base + (*jidx) * ld when jidx is given (the Krylov vector of the current iteration).
// Every thread-per-row kernel below walks the rows of its row map with a grid stride (one
// round on the identity map's full grid; a persistent grid over the compacted rows of a
// batch's problems taking part), warp by warp so that each warp finds its rows together.
#define JF_ROWS(rm, i)                                                                              \
    for (int w_ = blockIdx.x * blockDim.x + (int)(threadIdx.x & ~31u), tot_ = (rm).total(); w_ < tot_; \
         w_ += gridDim.x * blockDim.x)                                                              \
        if (const int v_ = w_ + (int)(threadIdx.x & 31u), i = warp_row((rm), v_, w_, tot_); v_ < tot_)

template <typename TV, typename T>
__global__ void k_mg_pre0(const int* gate, RowMap rm, int nc, const TV* __restrict__ base, size_t ld,
                          const int* __restrict__ jidx, const T* __restrict__ dinv, T omega, T* __restrict__ b,
                          T* __restrict__ x)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const TV* v = jidx ? base + (size_t)(*jidx) * ld : base;
    JF_ROWS(rm, P) {
        const T d = omega * dinv[P];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const T bb = -(T)v[(size_t)k * nc + P];
            b[(size_t)k * nc + P] = bb;
            x[(size_t)k * nc + P] = d * bb;
        }
    }
}

// a product rounded on its own (never fused into a following add), as when it is stored
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// level 0 entry fused with the first Jacobi sweep: b = -v, x0 = omega D^-1 b (formed where it
// is needed, also at the neighbours), x1 = x0 + omega D^-1 (b - A x0).  Same arithmetic, in the
// same order, as k_mg_pre0 followed by k_mg_jacobi.
template <typename TV, typename T>
__global__ void k_mg_pre0_jacobi(const int* gate, RowMap rm, LevelOp<T> op, const TV* __restrict__ base, size_t ld,
                                 const int* __restrict__ jidx, T omega, T* __restrict__ b, T* __restrict__ xo)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int nc = op.n;
    const TV* v = jidx ? base + (size_t)(*jidx) * ld : base;
    JF_ROWS(rm, P) {
        const T dP = omega * op.dinv[P];
        T bb[3], x0[3], ax[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            bb[k] = -(T)v[(size_t)k * nc + P];
            x0[k] = mul_rn(dP, bb[k]);
        }
        const T a = op.adiag[P];
#pragma unroll
        for (int k = 0; k < 3; k++) ax[k] = a * x0[k];
        for_sell_slots<T>(P, nc, op.p0, op.p1, op.p2, op.vals, [&](int N, T cf) {
            const T dN = omega * op.dinv[N];
#pragma unroll
            for (int k = 0; k < 3; k++) ax[k] -= cf * mul_rn(dN, -(T)v[(size_t)k * nc + N]);
        });
#pragma unroll
        for (int k = 0; k < 3; k++) {
            b[(size_t)k * nc + P] = bb[k];
            xo[(size_t)k * nc + P] = x0[k] + dP * (bb[k] - ax[k]);
        }
    }
}

template <typename T>
__global__ void k_mg_pre(const int* gate, RowMap rm, int n, const T* __restrict__ dinv, T omega,
                         const T* __restrict__ b, T* __restrict__ x)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    JF_ROWS(rm, i) {
        const T d = omega * dinv[i];
        T b0, b1, b2;
        ld3(b, i, b0, b1, b2);
        st3(x, i, d * b0, d * b1, d * b2);
    }
    (void)n;
}

// Jacobi sweep x_out = x + omega D^-1 (b - A x); zd != null writes the result as double
template <typename T>
__global__ void k_mg_jacobi(const int* gate, RowMap rm, LevelOp<T> op, T omega, const T* __restrict__ b,
                            const T* __restrict__ x, T* __restrict__ xo, double* __restrict__ zd)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int n = op.n;
    JF_ROWS(rm, i) {
        T ax[3];
        op.row(i, x, ax);
        const T d = omega * op.dinv[i];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const T xn = x[(size_t)k * n + i] + d * (b[(size_t)k * n + i] - ax[k]);
            if (zd) zd[(size_t)k * n + i] = to_f64(xn);
            else xo[(size_t)k * n + i] = xn;
        }
    }
}

// The last sweep of a V-cycle that feeds a Jacobian product (one problem): as k_mg_jacobi with
// z written as double, and |z|^2 summed per block; the last block forms the product's step
// eps = s (1 + |u|) / |z| (Eq. JF) and 1 / eps, as the norm pass would have (no launch of it)
struct EpsOut {
    ProbDev* pd;
    double* partials;  // one per block
    double s;          // jv_eps_scale
};

template <typename T>
__global__ void k_mg_jacobi_eps(const int* gate, LevelOp<T> op, T omega, const T* __restrict__ b, const T* __restrict__ x,
                                double* __restrict__ zd, EpsOut E)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    ProbDev& P = E.pd[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = op.n;
    double a = 0.0;
    if (i < n) {  // threads past the end still take part in the block sum
        T ax[3];
        op.row(i, x, ax);
        const T d = omega * op.dinv[i];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const T xn = x[(size_t)k * n + i] + d * (b[(size_t)k * n + i] - ax[k]);
            const double zv = to_f64(xn);
            zd[(size_t)k * n + i] = zv;
            a = fma(zv, zv, a);
        }
    }
    // partial sums per group of 128 cells (four warps), whatever the block size (a multiple of
    // 128 chosen by the autotuner), so that eps does not depend on the launch shape
    __shared__ double sh[32];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    const int gpb = blockDim.x / 128;  // groups per block
    if ((int)threadIdx.x < gpb) {
        const double* w = sh + 4 * threadIdx.x;
        E.partials[blockIdx.x * gpb + threadIdx.x] = (w[0] + w[1]) + (w[2] + w[3]);
    }
    if (!ticket_last(&P.ticket[2], gridDim.x)) return;
    if (threadIdx.x < 32) {
        const double tot = warp_sum_strided(E.partials, (n + 127) / 128);
        if (threadIdx.x == 0) {
            const double nrm = sqrt(tot);
            if (P.active && !P.done) {
                P.eps = (nrm > 0.0) ? E.s * (1.0 + P.unorm) / nrm : 0.0;
                P.ieps = P.eps != 0.0 ? 1.0 / P.eps : 0.0;
            }
            P.ticket[2] = 0u;
        }
    }
}

// r = b - A x
template <typename T>
__global__ void k_mg_resid(const int* gate, RowMap rm, LevelOp<T> op, const T* __restrict__ b,
                           const T* __restrict__ x, T* __restrict__ r)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int n = op.n;
    JF_ROWS(rm, i) {
        T ax[3];
        op.row(i, x, ax);
        st3(r, i, b[i] - ax[0], b[n + i] - ax[1], b[2 * (size_t)n + i] - ax[2]);
    }
}

// y += P x (prolongation) for a CSR matrix with nrow rows; x interleaved (a coarse level), y
// interleaved (AOSY) or component-major (the finest level)
template <typename T, bool AOSY>
__global__ void k_mg_prolong(const int* gate, RowMap rm, int nrow, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ col, const T* __restrict__ val, const T* __restrict__ x,
                             T* __restrict__ y)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    JF_ROWS(rm, i) {
        T s0 = 0, s1 = 0, s2 = 0;
        const int a = rp[i], b = rp[i + 1];
        int js[kCsrUnroll];
        T as[kCsrUnroll];
#pragma unroll
        for (int q = 0; q < kCsrUnroll; q++) {
            js[q] = a + q < b ? col[a + q] : 0;
            as[q] = a + q < b ? val[a + q] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < kCsrUnroll; q++)
            if (a + q < b) {
                T x0, x1, x2;
                ld3(x, js[q], x0, x1, x2);
                s0 += as[q] * x0; s1 += as[q] * x1; s2 += as[q] * x2;
            }
        for (int q = a + kCsrUnroll; q < b; q++) {
            T x0, x1, x2;
            ld3(x, col[q], x0, x1, x2);
            const T v = val[q];
            s0 += v * x0; s1 += v * x1; s2 += v * x2;
        }
        T y0, y1, y2;
        if (AOSY) {
            ld3(y, i, y0, y1, y2);
            st3(y, i, y0 + s0, y1 + s1, y2 + s2);
        } else {
            ld3_soa(y, (size_t)nrow, i, y0, y1, y2);
            st3_soa(y, (size_t)nrow, i, y0 + s0, y1 + s1, y2 + s2);
        }
    }
}

constexpr int kCoarseWarps = 4;  // warps per row of the block-per-row kernels

// Long CSR rows (P^T, coarse A) are taken by a group of G lanes (G a power of two <= 32,
// about half the row's mean length, so a warp holds 32/G rows and each lane two entries of a
// row per step, both loaded before they are used), then summed by a shuffle tree of the group.
template <int G, typename T>
__device__ __forceinline__ void group_sum(T& s0, T& s1, T& s2)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o, G);
        s1 += __shfl_down_sync(0xffffffffu, s1, o, G);
        s2 += __shfl_down_sync(0xffffffffu, s2, o, G);
    }
}

// sum_q a_q xin(j_q) over the group's share of row entries [qa, qb); xin(j, x0, x1, x2)
// gives the three components of row j
template <int G, typename T, typename X>
__device__ __forceinline__ void group_row(int qa, int qb, int sub, const int32_t* __restrict__ col,
                                          const T* __restrict__ val, X&& xin, T& s0, T& s1, T& s2)
{
    for (int q = qa + sub; q < qb; q += 2 * G) {
        const int q1 = q + G;
        const bool h1 = q1 < qb;
        const int j0 = col[q], j1 = h1 ? col[q1] : j0;
        const T a0 = val[q], a1 = h1 ? val[q1] : (T)0;
        T x00, x01, x02;
        xin(j0, x00, x01, x02);
        T x10 = 0, x11 = 0, x12 = 0;
        if (h1) xin(j1, x10, x11, x12);
        s0 += a0 * x00; s1 += a0 * x01; s2 += a0 * x02;
        if (h1) { s0 += a1 * x10; s1 += a1 * x11; s2 += a1 * x12; }
    }
}

// Kernels with G lanes per row walk the row map in rounds of blockDim / G rows (a grid stride
// whose bound is uniform over the block, so every lane takes part in every shuffle).
#define JF_GROUP_ROUNDS(rm, G, v, vw, sub, live, tot)                                             \
    const int tot = (rm).total();                                                                \
    for (int base_ = blockIdx.x * blockDim.x; base_ < tot * (G); base_ += gridDim.x * blockDim.x) \
        if (const int v = (base_ + (int)threadIdx.x) / (G), vw = (base_ + (int)(threadIdx.x & ~31u)) / (G), \
            sub = threadIdx.x & ((G)-1); true)                                                    \
            if (const bool live = v < tot; true)

// y = R x (restriction, R = P^T) with x and y interleaved
template <typename T, int G>
__global__ void k_mg_spmv_grp(const int* gate, RowMap rm, int nrow, int nx, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ col, const T* __restrict__ val, const T* __restrict__ x,
                              T* __restrict__ y)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    JF_GROUP_ROUNDS(rm, G, v, vw, sub, live, tot) {
        T s0 = 0, s1 = 0, s2 = 0;
        // lanes past the last row still take part in the shuffles
        const int i = warp_row(rm, v, vw, tot);
        if (live)
            group_row<G, T>(rp[i], rp[i + 1], sub, col, val, [&](int j, T& a, T& b, T& c) { ld3(x, j, a, b, c); }, s0, s1,
                            s2);
        group_sum<G>(s0, s1, s2);
        if (live && sub == 0) st3(y, i, s0, s1, s2);
    }
    (void)nrow; (void)nx;
}

// Jacobi sweep or residual on a coarse (CSR) level, vectors interleaved:
// mode 0: xo = x + omega D^-1 (b - A x);  mode 1: xo = b - A x;
// mode 2: the first sweep from x = omega D^-1 b, which is formed where it is needed (x unused)
template <typename T, int G>
__global__ void k_mg_csr_grp(const int* gate, RowMap rm, int n, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ col, const T* __restrict__ val, const T* __restrict__ dinv,
                             T omega, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ xo, int mode)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    JF_GROUP_ROUNDS(rm, G, v, vw, sub, live, tot) {
    T s0 = 0, s1 = 0, s2 = 0;
    // the row's own values, loaded ahead of the sums; lanes past the last row still take part
    // in the shuffles
    T bi0 = 0, bi1 = 0, bi2 = 0, xi0 = 0, xi1 = 0, xi2 = 0, di = 0;
    const int i = warp_row(rm, v, vw, tot);
    if (live) {
        if (sub == 0) {
            ld3(b, i, bi0, bi1, bi2);
            di = dinv[i];
            if (mode == 0) ld3(x, i, xi0, xi1, xi2);
        }
        const int qa = rp[i], qb = rp[i + 1];
        if (mode == 2)
            group_row<G, T>(qa, qb, sub, col, val,
                            [&](int j, T& a0, T& a1, T& a2) {
                                const T d = omega * dinv[j];
                                ld3(b, j, a0, a1, a2);
                                a0 = mul_rn(d, a0); a1 = mul_rn(d, a1); a2 = mul_rn(d, a2);
                            },
                            s0, s1, s2);
        else
            group_row<G, T>(qa, qb, sub, col, val, [&](int j, T& a0, T& a1, T& a2) { ld3(x, j, a0, a1, a2); }, s0, s1, s2);
    }
    group_sum<G>(s0, s1, s2);
    if (live && sub == 0) {
        const T r0 = bi0 - s0, r1 = bi1 - s1, r2 = bi2 - s2;
        if (mode == 1) st3(xo, i, r0, r1, r2);
        else if (mode == 2) {
            const T d = omega * di;
            st3(xo, i, mul_rn(d, bi0) + d * r0, mul_rn(d, bi1) + d * r1, mul_rn(d, bi2) + d * r2);
        } else {
            const T d = omega * di;
            st3(xo, i, xi0 + d * r0, xi1 + d * r1, xi2 + d * r2);
        }
    }
    }
    (void)n;
}

// y = R x (restriction) for rows longer than a warp's two-entry step: one block of
// kCoarseWarps warps per row, the warps' sums combined in shared memory
template <typename T>
__global__ void __launch_bounds__(32 * kCoarseWarps) k_mg_spmv_blk(const int* gate, RowMap rm, int nrow, int nx,
                                                                   const int32_t* __restrict__ rp,
                                                                   const int32_t* __restrict__ col,
                                                                   const T* __restrict__ val, const T* __restrict__ x,
                                                                   T* __restrict__ y)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ T part[3][kCoarseWarps];
    const int tot = rm.total();
    for (int v = blockIdx.x; v < tot; v += gridDim.x) {  // the whole block takes one row
    const int i = rm.row(v);
    T s0 = 0, s1 = 0, s2 = 0;
    group_row<32 * kCoarseWarps, T>(rp[i], rp[i + 1], threadIdx.x, col, val,
                                    [&](int j, T& a, T& b, T& c) { ld3(x, j, a, b, c); }, s0, s1, s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) { part[0][wid] = s0; part[1][wid] = s1; part[2][wid] = s2; }
    __syncthreads();
    if (threadIdx.x < 4) {  // (x, y, z, 0) of the interleaved row
        T t = 0;
        if (threadIdx.x < 3)
#pragma unroll
            for (int w = 0; w < kCoarseWarps; w++) t += part[threadIdx.x][w];
        y[4 * (size_t)i + threadIdx.x] = t;
    }
    __syncthreads();  // part[] is refilled in the next round
    }
    (void)nrow; (void)nx;
}

// sum_k a_k xin(j_k) over the sliced-ELL row i, eight entries' indices and values loaded
// together, then their rows gathered together, then summed in entry order
constexpr int kSellUnrollC = 8;
template <typename T, typename X>
__device__ __forceinline__ void sell_row(int i, const int32_t* __restrict__ soff, const int32_t* __restrict__ sw,
                                         const int32_t* __restrict__ scol, const T* __restrict__ sval, X&& xin, T& s0,
                                         T& s1, T& s2)
{
    const int sl = i >> 5, lane = i & 31, base = soff[sl], w = sw[sl];
    for (int k0 = 0; k0 < w; k0 += kSellUnrollC) {
        int js[kSellUnrollC];
        T as[kSellUnrollC], xs[kSellUnrollC][3];
#pragma unroll
        for (int q = 0; q < kSellUnrollC; q++) {
            const int slot = base + 32 * (k0 + q) + lane;
            js[q] = k0 + q < w ? scol[slot] : 0;
            as[q] = k0 + q < w ? sval[slot] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < kSellUnrollC; q++)
            if (k0 + q < w) xin(js[q], xs[q][0], xs[q][1], xs[q][2]);
#pragma unroll
        for (int q = 0; q < kSellUnrollC; q++)
            if (k0 + q < w) { s0 += as[q] * xs[q][0]; s1 += as[q] * xs[q][1]; s2 += as[q] * xs[q][2]; }
    }
}

// Jacobi sweep or residual on a coarse level in sliced-ELL form, one thread per row, vectors
// interleaved; modes as k_mg_csr_grp
template <typename T, int mode>
__global__ void k_mg_sell(const int* gate, RowMap rm, const int32_t* __restrict__ soff, const int32_t* __restrict__ sw,
                          const int32_t* __restrict__ scol, const T* __restrict__ sval, const T* __restrict__ dinv, T omega,
                          const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ xo)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    JF_ROWS(rm, i) {
        T bi0, bi1, bi2, xi0 = 0, xi1 = 0, xi2 = 0;
        ld3(b, i, bi0, bi1, bi2);
        const T di = dinv[i];
        if (mode == 0) ld3(x, i, xi0, xi1, xi2);
        T s0 = 0, s1 = 0, s2 = 0;
        if (mode == 2)
            sell_row<T>(i, soff, sw, scol, sval,
                        [&](int j, T& a0, T& a1, T& a2) {
                            const T d = omega * dinv[j];
                            ld3(b, j, a0, a1, a2);
                            a0 = mul_rn(d, a0); a1 = mul_rn(d, a1); a2 = mul_rn(d, a2);
                        },
                        s0, s1, s2);
        else
            sell_row<T>(i, soff, sw, scol, sval, [&](int j, T& a0, T& a1, T& a2) { ld3(x, j, a0, a1, a2); }, s0, s1, s2);
        const T r0 = bi0 - s0, r1 = bi1 - s1, r2 = bi2 - s2;
        const T d = omega * di;
        if (mode == 1) st3(xo, i, r0, r1, r2);
        else if (mode == 2) st3(xo, i, mul_rn(d, bi0) + d * r0, mul_rn(d, bi1) + d * r1, mul_rn(d, bi2) + d * r2);
        else st3(xo, i, xi0 + d * r0, xi1 + d * r1, xi2 + d * r2);
    }
}

// y = R x (restriction) in sliced-ELL form, one thread per coarse row, x and y interleaved
template <typename T>
__global__ void k_mg_restrict_sell(const int* gate, RowMap rm, const int32_t* __restrict__ soff,
                                   const int32_t* __restrict__ sw, const int32_t* __restrict__ scol,
                                   const T* __restrict__ sval, const T* __restrict__ x, T* __restrict__ y)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    JF_ROWS(rm, i) {
        T s0 = 0, s1 = 0, s2 = 0;
        sell_row<T>(i, soff, sw, scol, sval, [&](int j, T& a0, T& a1, T& a2) { ld3(x, j, a0, a1, a2); }, s0, s1, s2);
        st3(y, i, s0, s1, s2);
    }
}

// lanes per row for CSR rows of mean length `mean`: the power of two near half of it, 4..32,
// and 32 * kCoarseWarps (a block per row, restrictions only) for rows of more than two warp
// steps of two entries per lane
inline int group_lanes(double mean)
{
    if (mean > 4.0 * 32) return 32 * kCoarseWarps;
    int g = 4;
    while (g < 32 && 2.0 * g < mean) g *= 2;
    return g;
}

template <typename T, typename... A>
static void launch_csr_grp(jfnk_ctx* c, int g, long rows, const int* gate, const RowMap& rm, A... args)
{
    g = std::min(g, 32);
    auto go = [&](auto k) {
        const dim3 grid(rowmap_blocks(c, (const void*)k, 256, rows * g, 256, rm)), block(256);
        jfnk_launch(c, k, grid, block, gate, rm, args...);
    };
    switch (g) {
        case 4: go(k_mg_csr_grp<T, 4>); break;
        case 8: go(k_mg_csr_grp<T, 8>); break;
        case 16: go(k_mg_csr_grp<T, 16>); break;
        default: go(k_mg_csr_grp<T, 32>); break;
    }
}

template <typename T, typename... A>
static void launch_spmv_grp(jfnk_ctx* c, int g, long rows, const int* gate, const RowMap& rm, A... args)
{
    if (g > 32) {
        const dim3 grid(rowmap_blocks(c, (const void*)k_mg_spmv_blk<T>, 32 * kCoarseWarps, rows, 1, rm));
        jfnk_launch(c, k_mg_spmv_blk<T>, grid, dim3(32 * kCoarseWarps), gate, rm, args...);
        return;
    }
    auto go = [&](auto k) {
        const dim3 grid(rowmap_blocks(c, (const void*)k, 256, rows * g, 256, rm)), block(256);
        jfnk_launch(c, k, grid, block, gate, rm, args...);
    };
    switch (g) {
        case 4: go(k_mg_spmv_grp<T, 4>); break;
        case 8: go(k_mg_spmv_grp<T, 8>); break;
        case 16: go(k_mg_spmv_grp<T, 16>); break;
        default: go(k_mg_spmv_grp<T, 32>); break;
    }
}

// coarsest level: x = A_c^-1 b with the dense (symmetric) inverse, one block of kCoarseWarps
// warps per row, each warp a strided quarter of the row with two entries per lane and step
// loaded before use, the warps' sums combined in shared memory; b and x interleaved (AOS), or
// component-major when the coarsest level is the finest (one-level hierarchy)
template <typename T, bool AOS>
__global__ void __launch_bounds__(32 * kCoarseWarps) k_mg_coarse(const int* gate, RowMap rm, ProbSkip sk, int n,
                                                                 const T* __restrict__ Ainv, const T* __restrict__ b,
                                                                 T* __restrict__ x)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ T part[3][kCoarseWarps];
    const int tot = rm.total();
    for (int v = blockIdx.x; v < tot; v += gridDim.x) {  // the whole block takes one row
    const int r = rm.row(v);
    T s0 = 0, s1 = 0, s2 = 0;
    const T* row = Ainv + (size_t)r * n;
    constexpr int step = 32 * kCoarseWarps;
    for (int k = threadIdx.x; k < n; k += 2 * step) {
        const int k1 = k + step;
        const bool h1 = k1 < n;
        const T a0 = row[k], a1 = h1 ? row[k1] : (T)0;
        // rows of skipped problems hold values of an earlier cycle (or none yet): they enter
        // as zeros, so that nothing of another problem reaches this row's sum
        T b00 = 0, b01 = 0, b02 = 0;
        if (!sk(k)) {
            if (AOS) ld3(b, k, b00, b01, b02);
            else ld3_soa(b, (size_t)n, k, b00, b01, b02);
        }
        T b10 = 0, b11 = 0, b12 = 0;
        if (h1 && !sk(k1)) {
            if (AOS) ld3(b, k1, b10, b11, b12);
            else ld3_soa(b, (size_t)n, k1, b10, b11, b12);
        }
        s0 += a0 * b00; s1 += a0 * b01; s2 += a0 * b02;
        if (h1) { s0 += a1 * b10; s1 += a1 * b11; s2 += a1 * b12; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) { part[0][wid] = s0; part[1][wid] = s1; part[2][wid] = s2; }
    __syncthreads();
    if (threadIdx.x < (AOS ? 4 : 3)) {
        T t = 0;
        if (threadIdx.x < 3)
#pragma unroll
            for (int w = 0; w < kCoarseWarps; w++) t += part[threadIdx.x][w];
        if (AOS) x[4 * (size_t)r + threadIdx.x] = t;
        else x[(size_t)threadIdx.x * n + r] = t;
    }
    __syncthreads();  // part[] is refilled in the next round
    }
}

// ------------------------------------------------------------------ device hierarchy
template <typename T>
struct MgDev {
    struct Level {
        int n = 0, nco = 0;
        int32_t *rp = nullptr, *col = nullptr;    // A (coarse levels)
        T *val = nullptr, *adiag = nullptr, *dinv = nullptr;
        int32_t *prp = nullptr, *pcol = nullptr;  // P: n x nco
        T* pval = nullptr;
        int32_t *rrp = nullptr, *rcol = nullptr;  // R = P^T: nco x n
        T* rval = nullptr;
        int ga = 32, gr = 32;                      // lanes per row of A (coarse levels) and of R
        // A (coarse levels) and R in sliced-ELL form (32 rows per slice, entries slot-major,
        // one thread per row) where their rows are short enough; the CSR arrays are then unused
        bool a_sell = false, r_sell = false;
        int32_t *a_soff = nullptr, *a_sw = nullptr, *a_scol = nullptr;
        T* a_sval = nullptr;
        int32_t *r_soff = nullptr, *r_sw = nullptr, *r_scol = nullptr;
        T* r_sval = nullptr;
        int64_t nnz_a = 0, nnz_p = 0;              // operator entries (with the diagonal), P entries
        T *b = nullptr, *x = nullptr, *x2 = nullptr, *r = nullptr;
    };
    std::vector<Level> L;
    T* Ainv = nullptr;
    T* jc = nullptr;   // fine-level face coefficients in T
    T* sc = nullptr;   // the same per sliced-ELL neighbour slot (0 on padding and mirror slots)
};

struct MgState {
    MgDev<float> f;
    MgDev<double> d;
    bool ready = false;
    // batches: the problem of each row of every level (level 0: the context's cell map), for
    // skipping the problems that sit out an Arnoldi iteration; empty for single problems
    std::vector<const int32_t*> rprob;
    std::vector<std::vector<int32_t>> rprob_host;  // levels >= 1 on the host (compacted launches)
};

template <typename T>
static T* upload_as(jfnk_ctx* c, const std::vector<double>& h)
{
    std::vector<T> t(h.size());
    host_parallel((int)h.size(), 1 << 18, [&](int lo, int hi) {
        for (int i = lo; i < hi; i++) t[i] = (T)h[i];
    });
    T* d = (T*)jfnk_dalloc(c, sizeof(T) * std::max<size_t>(1, t.size()));
    if (d && jfnk_upload(c, d, t.data(), sizeof(T) * t.size())) return nullptr;
    return d;
}
static int32_t* upload_i(jfnk_ctx* c, const std::vector<int32_t>& h)
{
    int32_t* d = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * std::max<size_t>(1, h.size()));
    if (d && jfnk_upload(c, d, h.data(), sizeof(int32_t) * h.size())) return nullptr;
    return d;
}

// P of the fine level re-indexed to the internal cell order, and R = P^T for every level
struct HostTransfer {
    std::vector<int32_t> prp, pcol, rrp, rcol;
    std::vector<double> pval, rval;
};

static void make_transfer(const std::vector<int32_t>& prp, const std::vector<int32_t>& pcol, const std::vector<double>& pval,
                          int n, int nco, const std::vector<int32_t>* n2o, HostTransfer& t)
{
    // rows of P in the device numbering of this level
    t.prp.assign(n + 1, 0);
    for (int i = 0; i < n; i++) {
        const int src = n2o ? (*n2o)[i] : i;
        t.prp[i + 1] = t.prp[i] + (prp[src + 1] - prp[src]);
    }
    t.pcol.resize(t.prp[n]);
    t.pval.resize(t.prp[n]);
    host_parallel(n, 1 << 15, [&](int lo, int hi) {
        for (int i = lo; i < hi; i++) {
            const int src = n2o ? (*n2o)[i] : i;
            std::copy(pcol.begin() + prp[src], pcol.begin() + prp[src + 1], t.pcol.begin() + t.prp[i]);
            std::copy(pval.begin() + prp[src], pval.begin() + prp[src + 1], t.pval.begin() + t.prp[i]);
        }
    });
    t.rrp.assign(nco + 1, 0);
    for (int q = 0; q < (int)t.pcol.size(); q++) t.rrp[t.pcol[q] + 1]++;
    for (int J = 0; J < nco; J++) t.rrp[J + 1] += t.rrp[J];
    t.rcol.assign(t.pcol.size(), 0);
    t.rval.assign(t.pcol.size(), 0.0);
    std::vector<int32_t> fill(t.rrp.begin(), t.rrp.end() - 1);
    for (int i = 0; i < n; i++)
        for (int q = t.prp[i]; q < t.prp[i + 1]; q++) {
            const int J = t.pcol[q];
            t.rcol[fill[J]] = i;
            t.rval[fill[J]] = t.pval[q];
            fill[J]++;
        }
}

// Sliced ELL of a CSR matrix with n rows: 32 rows per slice, the slice as wide as its longest
// row, entry k of row i at slot off[i / 32] + 32 k + i % 32 (so a warp's loads of one entry
// index coalesce); padding slots repeat the row's first column with a zero value.
struct SellHost {
    std::vector<int32_t> off, w, col;
    std::vector<double> val;
};
static void csr_to_sell(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& col, const std::vector<double>& val,
                        SellHost& S)
{
    const int ns = (n + 31) / 32;
    S.off.assign(ns + 1, 0);
    S.w.assign(ns, 0);
    for (int sl = 0; sl < ns; sl++) {
        int w = 0;
        for (int i = 32 * sl; i < std::min(n, 32 * sl + 32); i++) w = std::max(w, rp[i + 1] - rp[i]);
        S.w[sl] = w;
        S.off[sl + 1] = S.off[sl] + 32 * w;
    }
    S.col.assign(std::max(1, S.off[ns]), 0);
    S.val.assign(std::max(1, S.off[ns]), 0.0);
    host_parallel(n, 1 << 15, [&](int lo, int hi) {
        for (int i = lo; i < hi; i++) {
            const int sl = i >> 5, lane = i & 31, a = rp[i], len = rp[i + 1] - a;
            for (int k = 0; k < S.w[sl]; k++) {
                const int slot = S.off[sl] + 32 * k + lane;
                S.col[slot] = len > 0 ? col[a + std::min(k, len - 1)] : 0;
                S.val[slot] = k < len ? val[a + k] : 0.0;
            }
        }
    });
}
// Levels of at least kSellMinRows rows whose mean row length is at most kSellMaxMean run one
// thread per row in sliced-ELL form; smaller levels (too few threads to fill 152 SMs: the
// 80k-cell cantilever's 10k-row level 1 ran 1.7x slower that way) and longer rows keep the
// lane-group CSR kernels
constexpr double kSellMaxMean = 64.0;
constexpr int kSellMinRows = 1 << 16;
constexpr int kSellWaves = 4;  // persistent-grid waves of the sliced-ELL kernels over compacted rows (4 measured 1 % faster than 1 on the 512-box batch)
// the row threshold, JFNK_MG_SELL_MIN_ROWS overriding it (read at set-up; tests run the
// sliced-ELL kernels on small meshes with 0)
static int sell_min_rows()
{
    const char* v = getenv("JFNK_MG_SELL_MIN_ROWS");
    return v ? std::max(0, atoi(v)) : kSellMinRows;
}

template <typename T>
static int mg_upload(jfnk_ctx* c, MgDev<T>& M, const std::vector<MgLevelHost>& lv, const std::vector<double>& inv,
                     const std::vector<double>& jc_h, const std::vector<double>& sc_h, const std::vector<double>& adiag0,
                     const std::vector<HostTransfer>& tr)
{
    const int nl = (int)lv.size();
    const int sell_rows = sell_min_rows();
    M.L.assign(nl, typename MgDev<T>::Level());
    M.jc = upload_as<T>(c, jc_h);
    M.sc = upload_as<T>(c, sc_h);
    for (int l = 0; l < nl; l++) {
        auto& D = M.L[l];
        const MgLevelHost& H = lv[l];
        D.n = H.n;
        D.nnz_a = (int64_t)H.col.size();
        std::vector<double> ad(H.n), di(H.n);
        if (l == 0) {
            ad = adiag0;
        } else {
            for (int i = 0; i < H.n; i++)
                for (int q = H.rp[i]; q < H.rp[i + 1]; q++)
                    if (H.col[q] == i) ad[i] = H.val[q];
            const double mean = (double)H.col.size() / std::max(1, H.n);
            D.a_sell = mean <= kSellMaxMean && H.n >= sell_rows;
            if (D.a_sell) {
                SellHost S;
                csr_to_sell(H.n, H.rp, H.col, H.val, S);
                D.a_soff = upload_i(c, S.off);
                D.a_sw = upload_i(c, S.w);
                D.a_scol = upload_i(c, S.col);
                D.a_sval = upload_as<T>(c, S.val);
                if (!D.a_soff || !D.a_sw || !D.a_scol || !D.a_sval) return jfnk_fail(c, JFNK_ENOMEM, "multigrid allocation failed");
            } else {
                D.rp = upload_i(c, H.rp);
                D.col = upload_i(c, H.col);
                D.val = upload_as<T>(c, H.val);
                D.ga = group_lanes(mean);
            }
        }
        for (int i = 0; i < H.n; i++) di[i] = 1.0 / ad[i];
        D.adiag = upload_as<T>(c, ad);
        D.dinv = upload_as<T>(c, di);
        // the finest level's b, x, x2 component-major [3][n]; its residual and every coarse
        // level's vectors interleaved [n][4]
        const size_t nv = (l == 0 ? 3 : 4) * (size_t)H.n, nr = 4 * (size_t)H.n;
        D.b = (T*)jfnk_dalloc(c, sizeof(T) * nv);
        D.x = (T*)jfnk_dalloc(c, sizeof(T) * nv);
        D.x2 = (T*)jfnk_dalloc(c, sizeof(T) * nv);
        D.r = (T*)jfnk_dalloc(c, sizeof(T) * nr);
        T* const vecs[4] = {D.b, D.x, D.x2, D.r};
        for (T* v : vecs)  // rows a cycle skips are read as finite values
            if (v) JF_CUDA(c, cudaMemsetAsync(v, 0, sizeof(T) * (v == D.r ? nr : nv), c->cur ? c->cur : c->stream));
        if (l < nl - 1) {
            D.nco = lv[l + 1].n;
            D.nnz_p = (int64_t)tr[l].pcol.size();
            D.prp = upload_i(c, tr[l].prp);
            D.pcol = upload_i(c, tr[l].pcol);
            D.pval = upload_as<T>(c, tr[l].pval);
            const double mean = (double)tr[l].rcol.size() / std::max(1, D.nco);
            D.r_sell = mean <= kSellMaxMean && D.nco >= sell_rows;
            if (D.r_sell) {
                SellHost S;
                csr_to_sell(D.nco, tr[l].rrp, tr[l].rcol, tr[l].rval, S);
                D.r_soff = upload_i(c, S.off);
                D.r_sw = upload_i(c, S.w);
                D.r_scol = upload_i(c, S.col);
                D.r_sval = upload_as<T>(c, S.val);
                if (!D.r_soff || !D.r_sw || !D.r_scol || !D.r_sval) return jfnk_fail(c, JFNK_ENOMEM, "multigrid allocation failed");
            } else {
                D.rrp = upload_i(c, tr[l].rrp);
                D.rcol = upload_i(c, tr[l].rcol);
                D.rval = upload_as<T>(c, tr[l].rval);
                D.gr = group_lanes(mean);
            }
        }
        if (!D.adiag || !D.dinv || !D.b || !D.x || !D.x2 || !D.r) return jfnk_fail(c, JFNK_ENOMEM, "multigrid allocation failed");
    }
    M.Ainv = upload_as<T>(c, inv);
    if (!M.Ainv || !M.jc || !M.sc) return jfnk_fail(c, JFNK_ENOMEM, "multigrid allocation failed");
    return JFNK_OK;
}

// ------------------------------------------------------------------ set-up
static MgState& mg_state(jfnk_ctx* c)
{
    if (!c->mgs) c->mgs = new MgState();
    return *(MgState*)c->mgs;
}

void mg_release(jfnk_ctx* c)
{
    delete (MgState*)c->mgs;
    c->mgs = nullptr;
}

int pc_setup(jfnk_ctx* c)
{
    MgState& S = mg_state(c);
    S.ready = false;
    if (c->opt.pc != JFNK_PC_MG) return JFNK_OK;
    // phase times, printed to stderr when JFNK_VERBOSE is set
    const bool verbose = getenv("JFNK_VERBOSE") != nullptr;
    auto tp = std::chrono::steady_clock::now();
    auto lap = [&](const char* what) {
        if (!verbose) return;
        const auto n = std::chrono::steady_clock::now();
        fprintf(stderr, "[jfnk]   preconditioner: %-26s %8.1f ms\n", what, std::chrono::duration<double, std::milli>(n - tp).count());
        tp = n;
    };
    const DevMesh& m = c->dm;
    const Topology& t = c->topo;
    const int nc = m.nc;
    std::vector<double> jc(std::max(1, m.nflux)), diag(nc);
    int rc;
    if ((rc = jfnk_download(c, jc.data(), m.jt_c, sizeof(double) * m.nflux)) ||
        (rc = jfnk_download(c, diag.data(), m.jt_diag, sizeof(double) * nc)))
        return rc;
    // level 0 in the caller's cell order (so the aggregation does not depend on the internal
    // renumbering): rows by input index, columns ascending
    MgLevelHost L0;
    L0.n = nc;
    // CSR, one host thread per block of rows: the diagonal, then one entry per internal face of
    // the cell in increasing face index (its owned faces merged with the faces it neighbours),
    // then each (short) row sorted by column
    L0.rp.assign(nc + 1, 0);
    for (int i = 0; i < nc; i++) {
        const int P = t.o2n[i];
        L0.rp[i + 1] = L0.rp[i] + 1 + (t.fo_ptr[P + 1] - t.fo_ptr[P]) + (t.fn_ptr[P + 1] - t.fn_ptr[P]);
    }
    L0.col.assign(L0.rp[nc], 0);
    L0.val.assign(L0.rp[nc], 0.0);
    host_parallel(nc, 1 << 15, [&](int lo, int hi) {
        for (int i = lo; i < hi; i++) {
            const int P = t.o2n[i];
            int q = L0.rp[i];
            L0.col[q] = i;
            L0.val[q++] = -diag[P];
            int a = t.fo_ptr[P], b = t.fn_ptr[P];
            const int ae = t.fo_ptr[P + 1], be = t.fn_ptr[P + 1];
            while (a < ae || b < be) {
                int f, other;
                if (b >= be || (a < ae && a < t.fn_face[b])) { f = a++; other = t.nei[f]; }
                else { f = t.fn_face[b++]; other = t.own[f]; }
                L0.col[q] = t.n2o[other];
                L0.val[q++] = -jc[f];
            }
        }
    });
    host_parallel(nc, 1 << 15, [&](int lo, int hi) {
        for (int i = lo; i < hi; i++)  // insertion sort: a handful of entries per row
            for (int q = L0.rp[i] + 1; q < L0.rp[i + 1]; q++) {
                const int32_t cq = L0.col[q];
                const double vq = L0.val[q];
                int r = q - 1;
                for (; r >= L0.rp[i] && L0.col[r] > cq; r--) { L0.col[r + 1] = L0.col[r]; L0.val[r + 1] = L0.val[r]; }
                L0.col[r + 1] = cq;
                L0.val[r + 1] = vq;
            }
    });
    lap("fine-level matrix (host)");
    std::vector<MgLevelHost> lv;
    std::vector<double> inv;
    const auto t0 = std::chrono::steady_clock::now();
    std::string e = mg_build_hierarchy(std::move(L0), c->opt.mg_theta, c->opt.mg_max_levels, c->opt.mg_coarse_max,
                                       c->opt.mg_smoothed != 0, lv, inv);
    if (getenv("JFNK_VERBOSE"))
        fprintf(stderr, "[jfnk] multigrid hierarchy (host) %8.1f ms\n",
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    if (!e.empty()) return jfnk_fail(c, JFNK_EINVAL, e);
    if (lv.size() == 1) {
        // the only level is the finest, whose vectors are in the internal numbering: its dense
        // inverse (built in the caller's order) is permuted to match
        std::vector<double> p(inv.size());
        for (int P = 0; P < nc; P++) {
            const size_t i = (size_t)t.n2o[P] * nc;
            for (int Q = 0; Q < nc; Q++) p[(size_t)P * nc + Q] = inv[i + t.n2o[Q]];
        }
        inv.swap(p);
    }
    tp = std::chrono::steady_clock::now();
    std::vector<HostTransfer> tr(lv.size());
    for (size_t l = 0; l + 1 < lv.size(); l++)
        make_transfer(lv[l].prp, lv[l].pcol, lv[l].pval, lv[l].n, lv[l + 1].n, l == 0 ? &t.n2o : nullptr, tr[l]);
    std::vector<double> adiag0(nc);
    for (int P = 0; P < nc; P++) adiag0[P] = -diag[P];
    // fine-level coefficient of every sliced-ELL neighbour slot
    std::vector<double> sc(std::max<size_t>(1, t.sell_nbr.size()), 0.0);
    host_parallel((int)t.sell_nbr.size(), 1 << 18, [&](int lo, int hi) {
        for (int q = lo; q < hi; q++)
            if (t.sell_nbr[q] >= 0 && t.sell_nbr[q] < nc) sc[q] = jc[t.sell_face[q]];
    });
    // the hierarchy in the precision the V-cycle runs in (a change of precision sets up again)
    lap("transfers, slot coefficients");
    if (c->opt.precision == JFNK_PREC_MIXED) rc = mg_upload<float>(c, S.f, lv, inv, jc, sc, adiag0, tr);
    else rc = mg_upload<double>(c, S.d, lv, inv, jc, sc, adiag0, tr);
    if (rc) return rc;
    // batches: the problem of every row of every level.  Aggregates never join cells of two
    // problems (the problems share no face, so no coupling), so each coarse row inherits the
    // problem of the rows aggregated into it.
    lap("upload (sliced ELL, CSR)");
    S.rprob.clear();
    S.rprob_host.clear();
    if (c->nprob > 1) {
        std::vector<int32_t> cur(nc, -1);  // level 0 in the caller's order
        for (int p = 0; p < c->nprob; p++)
            for (int P = c->prob_c0[p]; P < c->prob_c1[p]; P++) cur[t.n2o[P]] = p;
        std::vector<const int32_t*> rp{(const int32_t*)c->cell_prob};
        bool ok = true;
        for (size_t l = 0; ok && l + 1 < lv.size(); l++) {
            std::vector<int32_t> nxt(lv[l + 1].n, -1);
            ok = (int)lv[l].agg.size() == lv[l].n;
            for (int i = 0; ok && i < lv[l].n; i++) {
                const int a = lv[l].agg[i];
                ok = a >= 0 && a < lv[l + 1].n && cur[i] >= 0 && (nxt[a] < 0 || nxt[a] == cur[i]);
                if (ok) nxt[a] = cur[i];
            }
            for (int r = 0; ok && r < lv[l + 1].n; r++) ok = nxt[r] >= 0;
            if (ok) {
                const int32_t* d = upload_i(c, nxt);
                if (!d) return jfnk_fail(c, JFNK_ENOMEM, "multigrid allocation failed");
                rp.push_back(d);
                S.rprob_host.push_back(nxt);
                cur.swap(nxt);
            }
        }
        if (ok) S.rprob = rp;  // else every row of every level is always evaluated
        else S.rprob_host.clear();
        if (getenv("JFNK_VERBOSE"))
            fprintf(stderr, "[jfnk] multigrid row -> problem maps: %s (%zu levels)\n", ok ? "built" : "not built", rp.size());
    }
    lap("row -> problem maps");
    c->mg_coarse_n = lv.back().n;
    if (getenv("JFNK_VERBOSE")) {
        for (size_t l = 0; l < lv.size(); l++)
            fprintf(stderr, "[jfnk] multigrid level %zu: %d rows, %zu nonzeros, P nonzeros %zu\n", l, lv[l].n,
                    lv[l].col.size(), lv[l].pcol.size());
    }
    S.ready = true;
    c->mg_ready = true;
    return JFNK_OK;
}

const std::vector<std::vector<int32_t>>* mg_level_problems(jfnk_ctx* c)
{
    MgState& S = mg_state(c);
    return (S.ready && !S.rprob.empty()) ? &S.rprob_host : nullptr;
}

int mg_hierarchy_info(jfnk_ctx* c, std::vector<int64_t>& rows, std::vector<int64_t>& nnz_a, std::vector<int64_t>& nnz_p)
{
    MgState& S = mg_state(c);
    rows.clear();
    nnz_a.clear();
    nnz_p.clear();
    if (!S.ready) return 0;
    auto collect = [&](const auto& L) {
        for (size_t l = 0; l < L.size(); l++) {
            const auto& D = L[l];
            rows.push_back(D.n);
            // the finest level runs on the face coefficients: 2 couplings per internal face + diagonal
            nnz_a.push_back(l == 0 ? 2 * (int64_t)c->dm.ni + D.n : D.nnz_a);
            nnz_p.push_back(D.nnz_p);
        }
    };
    if (!S.f.L.empty()) collect(S.f.L);
    else collect(S.d.L);
    return (int)rows.size();
}

static inline int nb(long n, int t) { return (int)std::max<long>(1, (n + t - 1) / t); }

template <typename T>
static LevelOp<T> level_op(const jfnk_ctx* c, const MgDev<T>& M, int l)
{
    const auto& D = M.L[l];
    LevelOp<T> op;
    op.n = D.n;
    op.fine = (l == 0);
    if (l == 0) {
        op.p0 = c->dm.sell_off; op.p1 = c->dm.sell_w; op.p2 = c->dm.sell_nbr;
        op.vals = M.sc;
    } else {
        op.p0 = D.rp; op.p1 = D.col; op.p2 = nullptr;
        op.vals = D.val;
    }
    op.adiag = D.adiag;
    op.dinv = D.dinv;
    return op;
}

template <typename T, typename TV>
static int vcycle(jfnk_ctx* c, MgDev<T>& M, const TV* vbase, size_t ld, const int* jidx, double* z, const int* gate,
                  bool* eps_formed, int skip_mode)
{
    const MgState& S = mg_state(c);
    const bool skip = skip_mode != SKIP_NONE && c->nprob > 1 && c->skip_done && !S.rprob.empty();
    const int cyc = skip_mode == SKIP_CYCLE ? 1 : 0;
    // rows of each level the cycle visits: those of the problems taking part (compacted) when
    // problems sit the pass out, else all; the coarse solve also zeroes the columns of the
    // problems that sit out
    auto rm = [&](int l) {
        RowMap m;
        m.n = M.L[l].n;
        if (skip) m = rowmap(c, space_of_level(l), skip_mode, M.L[l].n);
        return m;
    };
    auto sk = [&](int l) { return ProbSkip{skip ? S.rprob[l] : nullptr, c->pd, cyc}; };
    if (skip && skip_mode == SKIP_INACTIVE) {
        const int rc = rowmap_build(c, SKIP_INACTIVE);
        if (rc) return rc;
    }
    const bool pf = c->prof.enabled && c->prof.detail;
    const int s_sm = pf ? c->prof.slot("mg_smooth") : -1, s_re = pf ? c->prof.slot("mg_resid") : -1;
    const int s_rs = pf ? c->prof.slot("mg_restrict") : -1, s_pr = pf ? c->prof.slot("mg_prolong") : -1;
    const int s_co = pf ? c->prof.slot("mg_coarse") : -1;
    const T omega = (T)(2.0 / 3.0);
    const int nl = (int)M.L.size();
    const int sweeps = std::max(1, c->opt.mg_smooth_sweeps);
    const int bs = c->tune.mg_bs;  // rows per block of the thread-per-row kernels
    // grid of a thread-per-row kernel over level l
    auto rows_grid = [&](const void* k, int l, const RowMap& m, int waves = 1) {
        return dim3(rowmap_blocks(c, k, bs, M.L[l].n, bs, m, waves));
    };
    auto coarse_grid = [&](int l, const RowMap& m) {
        return dim3(rowmap_blocks(c, (const void*)k_mg_coarse<T, true>, 32 * kCoarseWarps, M.L[l].n, 1, m));
    };
    // sweep (mode 0), residual (1) or first sweep (2) of a coarse level
    auto coarse_op = [&](int l, const RowMap& ml, const T* b, const T* x, T* xo, int mode) {
        auto& D = M.L[l];
        if (D.a_sell) {
            auto k = mode == 0 ? k_mg_sell<T, 0> : (mode == 1 ? k_mg_sell<T, 1> : k_mg_sell<T, 2>);
            jfnk_launch(c, k, rows_grid((const void*)k, l, ml, kSellWaves), dim3(bs), gate, ml, (const int32_t*)D.a_soff,
                        (const int32_t*)D.a_sw, (const int32_t*)D.a_scol, (const T*)D.a_sval, (const T*)D.dinv, omega, b, x, xo);
        } else
            launch_csr_grp<T>(c, D.ga, D.n, gate, ml, D.n, (const int32_t*)D.rp, (const int32_t*)D.col, (const T*)D.val,
                              (const T*)D.dinv, omega, b, x, xo, mode);
    };
    if (nl == 1) {
        auto& D = M.L[0];
        const RowMap m0 = rm(0);
        jfnk_launch(c, k_mg_pre0<TV, T>, rows_grid((const void*)k_mg_pre0<TV, T>, 0, m0), dim3(bs), gate, m0, D.n, vbase, ld,
                    jidx, D.dinv, (T)0, D.b, D.x2);
        JF_LAUNCHED(c);
        jfnk_launch(c, k_mg_coarse<T, false>, coarse_grid(0, m0), dim3(32 * kCoarseWarps), gate, m0, sk(0), D.n, M.Ainv, D.b, D.x);
        JF_LAUNCHED(c);
        jfnk_launch(c, k_copy_to_double<T>, dim3(nb(3L * D.n, 256)), dim3(256), gate, 3 * (size_t)D.n, D.x, z);
        JF_LAUNCHED(c);
        return JFNK_OK;
    }
    // downward
    for (int l = 0; l < nl - 1; l++) {
        auto& D = M.L[l];
        const LevelOp<T> op = level_op<T>(c, M, l);
        const RowMap ml = rm(l), mc = rm(l + 1);
        jfnk_prof_begin(c, s_sm);
        // the entry and the first sweep are one kernel when there are two or more sweeps
        if (sweeps >= 2) {
            if (l == 0)
                jfnk_launch(c, k_mg_pre0_jacobi<TV, T>, rows_grid((const void*)k_mg_pre0_jacobi<TV, T>, 0, ml), dim3(bs), gate,
                            ml, op, vbase, ld, jidx, omega, D.b, D.x);
            else coarse_op(l, ml, D.b, nullptr, D.x, 2);
        } else {
            if (l == 0)
                jfnk_launch(c, k_mg_pre0<TV, T>, rows_grid((const void*)k_mg_pre0<TV, T>, 0, ml), dim3(bs), gate, ml, D.n, vbase,
                            ld, jidx, D.dinv, omega, D.b, D.x);
            else jfnk_launch(c, k_mg_pre<T>, rows_grid((const void*)k_mg_pre<T>, l, ml), dim3(bs), gate, ml, D.n, D.dinv, omega, D.b, D.x);
        }
        JF_LAUNCHED(c);
        for (int sw = (sweeps >= 2 ? 2 : 1); sw < sweeps; sw++) {
            if (l == 0)
                jfnk_launch(c, k_mg_jacobi<T>, rows_grid((const void*)k_mg_jacobi<T>, 0, ml), dim3(bs), gate, ml, op, omega, D.b,
                            D.x, D.x2, nullptr);
            else coarse_op(l, ml, D.b, D.x, D.x2, 0);
            JF_LAUNCHED(c);
            std::swap(D.x, D.x2);
        }
        jfnk_prof_end(c, s_sm);
        jfnk_prof_begin(c, s_re);
        if (l == 0)
            jfnk_launch(c, k_mg_resid<T>, rows_grid((const void*)k_mg_resid<T>, 0, ml), dim3(bs), gate, ml, op, D.b, D.x, D.r);
        else coarse_op(l, ml, D.b, D.x, D.r, 1);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, s_re);
        auto& Cn = M.L[l + 1];
        jfnk_prof_begin(c, s_rs);
        if (D.r_sell)
            jfnk_launch(c, k_mg_restrict_sell<T>, rows_grid((const void*)k_mg_restrict_sell<T>, l + 1, mc, kSellWaves), dim3(bs), gate, mc,
                        (const int32_t*)D.r_soff, (const int32_t*)D.r_sw, (const int32_t*)D.r_scol, (const T*)D.r_sval,
                        (const T*)D.r, Cn.b);
        else
            launch_spmv_grp<T>(c, D.gr, D.nco, gate, mc, D.nco, D.n, (const int32_t*)D.rrp, (const int32_t*)D.rcol,
                               (const T*)D.rval, (const T*)D.r, Cn.b);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, s_rs);
    }
    {
        auto& Dc = M.L[nl - 1];
        const RowMap mcn = rm(nl - 1);
        jfnk_prof_begin(c, s_co);
        jfnk_launch(c, k_mg_coarse<T, true>, coarse_grid(nl - 1, mcn), dim3(32 * kCoarseWarps), gate, mcn, sk(nl - 1), Dc.n, M.Ainv,
                    Dc.b, Dc.x);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, s_co);
    }
    // upward
    for (int l = nl - 2; l >= 0; l--) {
        auto& D = M.L[l];
        auto& Cn = M.L[l + 1];
        const LevelOp<T> op = level_op<T>(c, M, l);
        const RowMap ml = rm(l);
        jfnk_prof_begin(c, s_pr);
        if (l == 0)
            jfnk_launch(c, k_mg_prolong<T, false>, rows_grid((const void*)k_mg_prolong<T, false>, l, ml), dim3(bs), gate, ml,
                        D.n, (const int32_t*)D.prp, (const int32_t*)D.pcol, (const T*)D.pval, (const T*)Cn.x, D.x);
        else
            jfnk_launch(c, k_mg_prolong<T, true>, rows_grid((const void*)k_mg_prolong<T, true>, l, ml), dim3(bs), gate, ml,
                        D.n, (const int32_t*)D.prp, (const int32_t*)D.pcol, (const T*)D.pval, (const T*)Cn.x, D.x);
        JF_LAUNCHED(c);
        jfnk_prof_end(c, s_pr);
        jfnk_prof_begin(c, s_sm);
        for (int sw = 0; sw < sweeps; sw++) {
            const bool last = (l == 0 && sw == sweeps - 1);
            if (last && eps_formed) {
                const EpsOut E{c->pd, c->partials, c->opt.jv_eps_scale};
                jfnk_launch(c, k_mg_jacobi_eps<T>, dim3(nb(D.n, bs)), dim3(bs), gate, op, omega, (const T*)D.b, (const T*)D.x, z, E);
                *eps_formed = true;
            } else if (l == 0)
                jfnk_launch(c, k_mg_jacobi<T>, rows_grid((const void*)k_mg_jacobi<T>, 0, ml), dim3(bs), gate, ml, op, omega, D.b,
                            D.x, D.x2, last ? z : nullptr);
            else coarse_op(l, ml, D.b, D.x, D.x2, 0);
            JF_LAUNCHED(c);
            if (!last) std::swap(D.x, D.x2);
        }
        jfnk_prof_end(c, s_sm);
    }
    return JFNK_OK;
}

// z = P^-1 v with v = vbase + (*jidx) * ld (jidx given) or vbase; v double or float; gate may be null
int pc_apply_dev(jfnk_ctx* c, int pc, const void* vbase, size_t ld, const int* jidx, int v_is_float, double* z, const int* gate,
                 bool* eps_formed, int skip)
{
    if (eps_formed) *eps_formed = false;
    // the multigrid's last sweep forms the Jv step of a single problem (batches keep the norm pass)
    bool* want_eps = (eps_formed && c->nprob == 1) ? eps_formed : nullptr;
    const int nc = c->dm.nc;
    const bool fp32 = c->opt.precision == JFNK_PREC_MIXED;
    int sl = c->prof.enabled ? c->prof.slot(pc == JFNK_PC_MG ? "pc_mg" : "pc_bjacobi") : -1;
    jfnk_prof_begin(c, sl);
    if (pc == JFNK_PC_BJACOBI && c->dm.jt_binv) {
        const double* bd = c->dm.jt_binv;
        const float* bf = c->dm.jt_binv_f;
        if (v_is_float) {
            if (fp32) jfnk_launch(c, k_bjacobi_block<float, float>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const float*)vbase, ld, jidx, bf, z);
            else jfnk_launch(c, k_bjacobi_block<float, double>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const float*)vbase, ld, jidx, bd, z);
        } else {
            if (fp32) jfnk_launch(c, k_bjacobi_block<double, float>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const double*)vbase, ld, jidx, bf, z);
            else jfnk_launch(c, k_bjacobi_block<double, double>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const double*)vbase, ld, jidx, bd, z);
        }
        JF_LAUNCHED(c);
    } else if (pc == JFNK_PC_BJACOBI) {
        if (v_is_float) {
            if (fp32) jfnk_launch(c, k_bjacobi<float, float>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const float*)vbase, ld, jidx, c->dm.jt_dinv_f, z);
            else jfnk_launch(c, k_bjacobi<float, double>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const float*)vbase, ld, jidx, c->dm.jt_dinv, z);
        } else {
            if (fp32) jfnk_launch(c, k_bjacobi<double, float>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const double*)vbase, ld, jidx, c->dm.jt_dinv_f, z);
            else jfnk_launch(c, k_bjacobi<double, double>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const double*)vbase, ld, jidx, c->dm.jt_dinv, z);
        }
        JF_LAUNCHED(c);
    } else if (pc == JFNK_PC_MG) {
        MgState& S = mg_state(c);
        if (!S.ready) return jfnk_fail(c, JFNK_ESTATE, "multigrid preconditioner not set up (options.pc must be JFNK_PC_MG at set-up)");
        int rc;
        if (fp32) rc = v_is_float ? vcycle<float, float>(c, S.f, (const float*)vbase, ld, jidx, z, gate, want_eps, skip)
                                  : vcycle<float, double>(c, S.f, (const double*)vbase, ld, jidx, z, gate, want_eps, skip);
        else rc = v_is_float ? vcycle<double, float>(c, S.d, (const float*)vbase, ld, jidx, z, gate, want_eps, skip)
                             : vcycle<double, double>(c, S.d, (const double*)vbase, ld, jidx, z, gate, want_eps, skip);
        if (rc) return rc;
    } else {
        if (v_is_float) jfnk_launch(c, k_copy_vec<float>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const float*)vbase, ld, jidx, z);
        else jfnk_launch(c, k_copy_vec<double>, dim3(nb(nc, 256)), dim3(256), gate, nc, (const double*)vbase, ld, jidx, z);
        JF_LAUNCHED(c);
    }
    jfnk_prof_end(c, sl);
    return JFNK_OK;
}

int pc_apply_any(jfnk_ctx* c, int pc, const void* v, int v_is_float, double* z, const int* gate, int skip)
{
    return pc_apply_dev(c, pc, v, 0, nullptr, v_is_float, z, gate, nullptr, skip);
}

int pc_apply(jfnk_ctx* c, int pc, const double* v, double* z) { return pc_apply_any(c, pc, v, 0, z, nullptr); }

}  // namespace jfnk
