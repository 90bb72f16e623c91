// The matrix-free momentum residual R(u) of Sec. 2.3 on the device, in three passes:
//   k_grad    per cell: least-squares gradient (Eq. leastSquaresGrad) from the sliced-ELL
//             neighbour table; neo-Hookean cells also form the total-Lagrangian traction
//             operator T = J F^-1 sigma (App. A, App. B Eq. neoHook);
//   k_flux    per internal and displacement face: the surface force of Eq. divStressDiscret
//             with the interpolated stress of Eq. stressInterp plus the Rhie-Chow term of
//             Eq. RhieChow, in owner-sorted face order;
//   k_finish  per cell: owner faces added, neighbour faces (neighbour-sorted list)
//             subtracted, plus the constant body/traction part; optionally the Jacobian
//             action (R(u + eps v) - R(u)) / eps of Eq. JF.  No atomics, fixed summation
//             order: the result is bitwise reproducible.
// FP64 throughout (the difference in Eq. JF cancels catastrophically otherwise).  The FP64
// pipe, not HBM, bounds these kernels on GB300, so the face coefficients are precomputed to
// keep the FP64 instruction count per face low.
#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

constexpr int kGradUnroll = 6;  // hexahedra have up to 6 internal neighbours
constexpr int kLawUpdated = 3;  // neo-Hookean in the updated-Lagrangian form

// gradient (and traction operator) of cell P
template <int LAW>
__device__ __forceinline__ void grad_cell(int P, int nc, int dim, const int32_t* __restrict__ sell_off,
                                          const int32_t* __restrict__ sell_w, const int32_t* __restrict__ sell_nbr,
                                          const double* __restrict__ sell_l, int n_slots,
                                          const double* __restrict__ u, double* __restrict__ G,
                                          double* __restrict__ T, const MatDev& mat, const int32_t* __restrict__ cell_prob,
                                          const double* __restrict__ sym_n, int nsy,
                                          const double* __restrict__ ul_Gn, const double* __restrict__ ul_F)
{
    const int s = P >> 5, lane = P & 31, base = sell_off[s], w = sell_w[s];
    const double u0 = u[P], u1 = u[nc + P], u2 = u[2 * nc + P];
    double g[9];
#pragma unroll
    for (int q = 0; q < 9; q++) g[q] = 0.0;
    // internal neighbours first; a cell's symmetry faces (mirror neighbours, coded N >= nc)
    // follow them in its slot list and are taken in a second loop, so meshes without
    // symmetry faces run the first loop alone
    // the first kGradUnroll slots' indices and weights are loaded together (one round of
    // loads in flight instead of one per neighbour), then summed in slot order
    auto add = [&](int N, double l0, double l1, double l2) {
        const double d0 = u[N] - u0, d1 = u[nc + N] - u1, d2 = u[2 * nc + N] - u2;
        g[0] = fma(l0, d0, g[0]); g[1] = fma(l0, d1, g[1]); g[2] = fma(l0, d2, g[2]);
        g[3] = fma(l1, d0, g[3]); g[4] = fma(l1, d1, g[4]); g[5] = fma(l1, d2, g[5]);
        g[6] = fma(l2, d0, g[6]); g[7] = fma(l2, d1, g[7]); g[8] = fma(l2, d2, g[8]);
    };
    int Ns[kGradUnroll];
    double ls[kGradUnroll][3];
#pragma unroll
    for (int q = 0; q < kGradUnroll; q++) {
        const int slot = base + 32 * q + lane;
        Ns[q] = q < w ? sell_nbr[slot] : -1;
        ls[q][0] = q < w ? sell_l[slot] : 0.0;
        ls[q][1] = q < w ? sell_l[n_slots + slot] : 0.0;
        ls[q][2] = q < w ? sell_l[2 * n_slots + slot] : 0.0;
    }
    int k = 0;
    bool internal = true;  // internal neighbours come first in a cell's slot list
#pragma unroll
    for (int q = 0; q < kGradUnroll; q++) {
        internal = internal && (unsigned)Ns[q] < (unsigned)nc;  // padding (-1) or a mirror neighbour ends them
        if (internal) {
            add(Ns[q], ls[q][0], ls[q][1], ls[q][2]);
            k = q + 1;
        }
    }
    if (internal)
        for (; k < w; k++) {
            const int slot = base + 32 * k + lane;
            const int N = sell_nbr[slot];
            if ((unsigned)N >= (unsigned)nc) break;
            add(N, sell_l[slot], sell_l[n_slots + slot], sell_l[2 * n_slots + slot]);
        }
    if (nsy > 0) {
        for (; k < w; k++) {
            const int slot = base + 32 * k + lane;
            const int N = sell_nbr[slot];
            if (N < 0) break;
            // symmetry face: the mirror value R u_P - u_P = -2 (n . u_P) n
            const double l0 = sell_l[slot], l1 = sell_l[n_slots + slot], l2 = sell_l[2 * n_slots + slot];
            const int q = N - nc;
            const double n0 = sym_n[q], n1 = sym_n[nsy + q], n2 = sym_n[2 * nsy + q];
            const double m2 = -2.0 * (n0 * u0 + n1 * u1 + n2 * u2);
            const double d0 = m2 * n0, d1 = m2 * n1, d2 = m2 * n2;
            g[0] = fma(l0, d0, g[0]); g[1] = fma(l0, d1, g[1]); g[2] = fma(l0, d2, g[2]);
            g[3] = fma(l1, d0, g[3]); g[4] = fma(l1, d1, g[4]); g[5] = fma(l1, d2, g[5]);
            g[6] = fma(l2, d0, g[6]); g[7] = fma(l2, d1, g[7]); g[8] = fma(l2, d2, g[8]);
        }
    }
#pragma unroll
    for (int q = 0; q < 9; q++) G[(size_t)q * nc + P] = g[q];
    const int pr = (LAW == JFNK_LAW_LINEAR || LAW == kLawUpdated) ? 0 : cell_prob[P];
    if (LAW == kLawUpdated) {
        // updated Lagrangian (App. A, Eq. momentum_UL), neo-Hookean: g is the gradient of the
        // displacement on the updated mesh and Gn that of the last converged step's, so the
        // increment's relative deformation gradient is f = I + (g - Gn)^T; the total one is
        // F = f Fn; the operator is T = j f^-1 sigma(F) = adj(f) sigma(F) with the Cauchy stress
        // sigma = mu J^-5/3 (b - tr(b)/3 I) + kappa/2 (J - 1/J) I, b = F F^T, J = det F
        const double mu = mat.mu[0], kappa = mat.kappa[0];
        double f[9], Fn[9], F[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) f[3 * i + j] = (i == j ? 1.0 : 0.0) + (g[3 * j + i] - ul_Gn[(size_t)(3 * j + i) * nc + P]);
#pragma unroll
        for (int q = 0; q < 9; q++) Fn[q] = ul_F[(size_t)q * nc + P];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double a = f[3 * i] * Fn[j];
                a = fma(f[3 * i + 1], Fn[3 + j], a);
                a = fma(f[3 * i + 2], Fn[6 + j], a);
                F[3 * i + j] = a;
            }
        const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                         F[2] * (F[3] * F[7] - F[4] * F[6]);
        double bb[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double a = F[3 * i] * F[3 * j];
                a = fma(F[3 * i + 1], F[3 * j + 1], a);
                a = fma(F[3 * i + 2], F[3 * j + 2], a);
                bb[3 * i + j] = a;
            }
        // one reciprocal cube root r3 = J^-1/3 gives J^-5/3 = r3^5 and 1/J = r3^3 (an inverted
        // cell, J <= 0, has no stress: NaN, which the line search rejects)
        const double r3 = (J > 0.0) ? rcbrt(J) : __longlong_as_double(0x7ff8000000000000LL);
        const double r32 = r3 * r3;
        const double rJ = r32 * r3;
        const double cdev = mu * r32 * rJ;                                  // mu J^-5/3
        const double cvol = 0.5 * kappa * (J - rJ) - cdev * (bb[0] + bb[4] + bb[8]) * (1.0 / 3.0);
        double sg[9];
#pragma unroll
        for (int q = 0; q < 9; q++) sg[q] = cdev * bb[q] + ((q % 4 == 0) ? cvol : 0.0);
        // adj(f) = j f^-1 (cofactors)
        const double A00 = f[4] * f[8] - f[5] * f[7], A01 = f[2] * f[7] - f[1] * f[8], A02 = f[1] * f[5] - f[2] * f[4];
        const double A10 = f[5] * f[6] - f[3] * f[8], A11 = f[0] * f[8] - f[2] * f[6], A12 = f[2] * f[3] - f[0] * f[5];
        const double A20 = f[3] * f[7] - f[4] * f[6], A21 = f[1] * f[6] - f[0] * f[7], A22 = f[0] * f[4] - f[1] * f[3];
        const double A[9] = {A00, A01, A02, A10, A11, A12, A20, A21, A22};
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double t = A[3 * i] * sg[j];
                t = fma(A[3 * i + 1], sg[3 + j], t);
                t = fma(A[3 * i + 2], sg[6 + j], t);
                T[(size_t)(3 * i + j) * nc + P] = t;
            }
    } else if (LAW == 2 && mat.law[pr] == JFNK_LAW_STVK) {
        // St. Venant-Kirchhoff (App. B): E = (G + G^T + G G^T) / 2, S = 2 mu E + lambda tr(E) I;
        // the total-Lagrangian operator J F^-1 sigma with sigma = F S F^T / J is S F^T
        // (F = I + G^T, so (S F^T)_ij = S_ij + sum_k S_ik G_kj)
        const double mu = mat.mu[pr], lam = mat.lam[pr];
        double E[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double gg = g[3 * i] * g[3 * j];
                gg = fma(g[3 * i + 1], g[3 * j + 1], gg);
                gg = fma(g[3 * i + 2], g[3 * j + 2], gg);
                E[3 * i + j] = 0.5 * (g[3 * i + j] + g[3 * j + i] + gg);
            }
        const double ltr = lam * (E[0] + E[4] + E[8]);
        double S[9];
#pragma unroll
        for (int q = 0; q < 9; q++) S[q] = 2.0 * mu * E[q] + ((q % 4 == 0) ? ltr : 0.0);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double t = S[3 * i + j];
                t = fma(S[3 * i], g[j], t);
                t = fma(S[3 * i + 1], g[3 + j], t);
                t = fma(S[3 * i + 2], g[6 + j], t);
                T[(size_t)(3 * i + j) * nc + P] = t;
            }
    } else if (LAW == JFNK_LAW_NEOHOOKEAN || (LAW == 2 && mat.law[pr] == JFNK_LAW_NEOHOOKEAN)) {
        const double mu = mat.mu[pr], kappa = mat.kappa[pr];
        // F = I + (grad u)^T: F_ij = delta_ij + g_ji
        const double F00 = 1.0 + g[0], F01 = g[3], F02 = g[6];
        const double F10 = g[1], F11 = 1.0 + g[4], F12 = g[7];
        const double F20 = g[2], F21 = g[5], F22 = 1.0 + g[8];
        // cofactor matrix: adj(F) = J F^-1
        const double A00 = F11 * F22 - F12 * F21, A01 = F02 * F21 - F01 * F22, A02 = F01 * F12 - F02 * F11;
        const double A10 = F12 * F20 - F10 * F22, A11 = F00 * F22 - F02 * F20, A12 = F02 * F10 - F00 * F12;
        const double A20 = F10 * F21 - F11 * F20, A21 = F01 * F20 - F00 * F21, A22 = F00 * F11 - F01 * F10;
        const double J = F00 * A00 + F01 * A10 + F02 * A20;
        // sigma = mu J^-5/3 (b - tr(b)/3 I) + kappa/2 (J - 1/J) I with b = F F^T, and
        // T = adj(F) sigma.  Since adj(F) b = J F^T:
        //   T = mu J^-2/3 F^T + (kappa/2 (J - 1/J) - mu J^-5/3 tr(b)/3) adj(F),
        // which needs tr(b) only, not b or the product adj(F) sigma.
        const double trb = F00 * F00 + F01 * F01 + F02 * F02 + F10 * F10 + F11 * F11 + F12 * F12 + F20 * F20 +
                           F21 * F21 + F22 * F22;
        // an inverted cell (J <= 0) has no stress: NaN makes the residual non-finite so the
        // line search rejects the state.  One reciprocal cube root r3 gives J^-2/3 = r3^2 and
        // 1/J = r3^3 (no divisions, no cube root: the FP64 pipe is the bound).
        const double r3 = (J > 0.0) ? rcbrt(J) : __longlong_as_double(0x7ff8000000000000LL);
        const double Jm23 = r3 * r3;
        const double rJ = Jm23 * r3;
        const double cF = mu * Jm23;                                             // mu J^-2/3
        const double cA = 0.5 * kappa * (J - rJ) - cF * rJ * trb * (1.0 / 3.0);  // coefficient of adj(F)
        double t[9];
        t[0] = cF * F00 + cA * A00; t[1] = cF * F10 + cA * A01; t[2] = cF * F20 + cA * A02;
        t[3] = cF * F01 + cA * A10; t[4] = cF * F11 + cA * A11; t[5] = cF * F21 + cA * A12;
        t[6] = cF * F02 + cA * A20; t[7] = cF * F12 + cA * A21; t[8] = cF * F22 + cA * A22;
#pragma unroll
        for (int q = 0; q < 9; q++) T[(size_t)q * nc + P] = t[q];
    }
    (void)dim;
}

// the cells of the row map, one per thread (a grid stride over compacted rows)
template <int LAW, int BS>
__global__ void __launch_bounds__(BS) k_grad(const int* __restrict__ gate, int nc, int dim, const int32_t* __restrict__ sell_off,
                                              const int32_t* __restrict__ sell_w, const int32_t* __restrict__ sell_nbr,
                                              const double* __restrict__ sell_l, int n_slots,
                                              const double* __restrict__ u, double* __restrict__ G,
                                              double* __restrict__ T, MatDev mat, const int32_t* __restrict__ cell_prob,
                                              const double* __restrict__ sym_n, int nsy, RowMap rm,
                                              const double* __restrict__ ul_Gn, const double* __restrict__ ul_F)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const int tot = rm.total();
    for (int vw = blockIdx.x * BS + (int)(threadIdx.x & ~31u); vw < tot; vw += gridDim.x * BS) {  // warp-uniform
        const int v = vw + (int)(threadIdx.x & 31u), P = warp_row(rm, v, vw, tot);
        if (v < tot)
            grad_cell<LAW>(P, nc, dim, sell_off, sell_w, sell_nbr, sell_l, n_slots, u, G, T, mat, cell_prob, sym_n, nsy, ul_Gn,
                           ul_F);
    }
}

// STAGE = 1: the block first copies the gradients (and, neo-Hookean, the traction operators)
// of the cell window [own[f0], own[f0] + BS) into shared memory, with coalesced loads, f0
// being the first face of the block's round; faces are owner-sorted, so the owners of the
// block's faces lie in that window unless a block spans the internal/boundary split, cells
// without faces or (compacted launches) two problems, and those read global memory.  Same
// arithmetic either way.
template <int LAW, int BS, int STAGE>
__device__ __forceinline__ void flux_face(int f, int Pw, const double* __restrict__ sg, const double* __restrict__ st,
                                          int ni, int nd, int nflux, int nc, const int32_t* __restrict__ own,
                                          const int32_t* __restrict__ nei, const double* __restrict__ coef,
                                          const double* __restrict__ u, const double* __restrict__ G,
                                          const double* __restrict__ T, const double* __restrict__ bval,
                                          const double* __restrict__ load_dev, const int32_t* __restrict__ fn_pos,
                                          const MatDev& mat, const int32_t* __restrict__ cell_prob,
                                          double* __restrict__ F, double* __restrict__ Fn)
{
    constexpr bool kT = (LAW != JFNK_LAW_LINEAR);
    if (f >= ni + nd) {
        // symmetry face (Eq. symm read as the mirror mean (T_P + R T_P R) / 2; Rhie-Chow with the
        // mirror neighbour at 2 delta n): t = Gamma [n.T_P.n - alpha Kbar ((n.u_P) / delta + n.G_P.n)]
        const int P = own[f];
        const double aK = coef[f], idelta = coef[nflux + f];
        const double n0 = coef[5 * (size_t)nflux + f], n1 = coef[6 * (size_t)nflux + f], n2 = coef[7 * (size_t)nflux + f];
        const double nv[3] = {n0, n1, n2};
        double Gnn = 0.0, Tnn = 0.0;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double gi = 0.0;
#pragma unroll
            for (int j = 0; j < 3; j++) gi = fma(G[(size_t)(3 * i + j) * nc + P], nv[j], gi);
            Gnn = fma(nv[i], gi, Gnn);
        }
        const int pr = cell_prob[P];
        const bool hooke_s = (LAW == JFNK_LAW_LINEAR) || (LAW == 2 && mat.law[pr] == JFNK_LAW_LINEAR);
        if (hooke_s) {
            const double tr = G[P] + G[4 * (size_t)nc + P] + G[8 * (size_t)nc + P];
            Tnn = 2.0 * mat.mu[pr] * Gnn + mat.lam[pr] * tr;
        } else {
#pragma unroll
            for (int i = 0; i < 3; i++) {
                double ti = 0.0;
#pragma unroll
                for (int j = 0; j < 3; j++) ti = fma(T[(size_t)(3 * i + j) * nc + P], nv[j], ti);
                Tnn = fma(nv[i], ti, Tnn);
            }
        }
        const double un = n0 * u[P] + n1 * u[nc + P] + n2 * u[2 * (size_t)nc + P];
        const double sc = Tnn - aK * fma(un, idelta, Gnn);
#pragma unroll
        for (int c = 0; c < 3; c++) F[(size_t)c * nflux + f] = coef[(size_t)(2 + c) * nflux + f] * sc;
        return;
    }
    const double load = *load_dev;
    const int P = own[f];
    const bool internal = f < ni;
    const int N = internal ? nei[f] : P;
    const double w = coef[f], kc = coef[nflux + f];
    const int kp = P - Pw;
    const bool staged = STAGE && kp >= 0 && kp < BS;
    double gf[9];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const double gp = staged ? sg[q * BS + kp] : G[(size_t)q * nc + P];
        if (internal) {
            const double gn = G[(size_t)q * nc + N];
            gf[q] = fma(w, gp - gn, gn);
        } else {
            gf[q] = gp;
        }
    }
    double du[3];
    if (internal) {
#pragma unroll
        for (int c = 0; c < 3; c++) du[c] = u[(size_t)c * nc + N] - u[(size_t)c * nc + P];
    } else {
        const int k = f - ni;
#pragma unroll
        for (int c = 0; c < 3; c++) du[c] = load * bval[(size_t)k * 3 + c] - u[(size_t)c * nc + P];
    }
    const double c0 = coef[2 * nflux + f], c1 = coef[3 * nflux + f], c2 = coef[4 * nflux + f];
    const double c3 = coef[5 * nflux + f], c4 = coef[6 * nflux + f], c5 = coef[7 * nflux + f];
    double t[3];
    const bool hooke = (LAW == JFNK_LAW_LINEAR) || (LAW == 2 && mat.law[cell_prob[P]] == JFNK_LAW_LINEAR);
    if (hooke) {
        // t_j = p . G_:j + q . G_j: + r_j tr(G) + kc du_j
        const double r0 = coef[8 * nflux + f], r1 = coef[9 * nflux + f], r2 = coef[10 * nflux + f];
        const double tr = gf[0] + gf[4] + gf[8];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double a = c0 * gf[j];
            a = fma(c1, gf[3 + j], a);
            a = fma(c2, gf[6 + j], a);
            a = fma(c3, gf[3 * j], a);
            a = fma(c4, gf[3 * j + 1], a);
            a = fma(c5, gf[3 * j + 2], a);
            a = fma((j == 0 ? r0 : (j == 1 ? r1 : r2)), tr, a);
            t[j] = fma(kc, du[j], a);
        }
    } else {
        // t_j = Gamma . T_f:j - a . G_f:j + kc du_j
        double tf[9];
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const double tp = (kT && staged) ? st[q * BS + kp] : T[(size_t)q * nc + P];
            if (internal) {
                const double tn = T[(size_t)q * nc + N];
                tf[q] = fma(w, tp - tn, tn);
            } else {
                tf[q] = tp;
            }
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double a = c0 * tf[j];
            a = fma(c1, tf[3 + j], a);
            a = fma(c2, tf[6 + j], a);
            a = fma(-c3, gf[j], a);
            a = fma(-c4, gf[3 + j], a);
            a = fma(-c5, gf[6 + j], a);
            t[j] = fma(kc, du[j], a);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) F[(size_t)c * nflux + f] = t[c];
    if (internal) {
        // the same flux in the neighbour-sorted order, so the cell pass reads contiguous ranges
        const int q = fn_pos[f];
#pragma unroll
        for (int c = 0; c < 3; c++) Fn[(size_t)c * ni + q] = t[c];
    }
}

template <int LAW, int BS, int STAGE>
__global__ void __launch_bounds__(BS) k_flux(const int* __restrict__ gate, int ni, int nd, int nflux, int nc, const int32_t* __restrict__ own,
                                             const int32_t* __restrict__ nei, const double* __restrict__ coef,
                                             const double* __restrict__ u, const double* __restrict__ G,
                                             const double* __restrict__ T, const double* __restrict__ bval,
                                             const double* __restrict__ load_dev, const int32_t* __restrict__ fn_pos,
                                             MatDev mat, const int32_t* __restrict__ cell_prob,
                                             double* __restrict__ F, double* __restrict__ Fn, RowMap rm)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    constexpr bool kT = (LAW != JFNK_LAW_LINEAR);
    __shared__ double sg[STAGE ? 9 * BS : 1];
    __shared__ double st[(STAGE && kT) ? 9 * BS : 1];
    const int tot = rm.total();
    // rounds of BS faces of the row map (a grid stride; the bound is uniform over the block)
    for (int v0 = blockIdx.x * BS; v0 < tot; v0 += gridDim.x * BS) {
        const int v = v0 + threadIdx.x;
        int Pw = 0;
        if (STAGE) {
            Pw = own[rm.row(v0)];
            const int cnt = min(BS, nc - Pw);
#pragma unroll
            for (int q = 0; q < 9; q++)
                for (int k = threadIdx.x; k < cnt; k += BS) {
                    sg[q * BS + k] = G[(size_t)q * nc + Pw + k];
                    if (kT) st[q * BS + k] = T[(size_t)q * nc + Pw + k];
                }
            __syncthreads();
        }
        const int f = warp_row(rm, v, v0 + (int)(threadIdx.x & ~31u), tot);
        if (v < tot)
            flux_face<LAW, BS, STAGE>(f, Pw, sg, st, ni, nd, nflux, nc, own, nei, coef, u, G, T, bval, load_dev, fn_pos, mat,
                                      cell_prob, F, Fn);
        if (STAGE) __syncthreads();  // the window is refilled in the next round
    }
}

// mode 0: out = R;  mode 1: out = (R - Ru) / eps_p with eps_p the Jv step of the cell's
// problem (0 -> out = 0).  Dynamics (rc != null): the inertia term -rho Omega_P a_P of the
// evaluated state u with the BDF2 acceleration a_P = 9/(4 dt^2) u_P + c_P (Eq. inertia2):
// R_P -= Omega_P (mk u_P + rc_P), mk = 9 rho / (4 dt^2), rc = rho c from the previous levels.
// One thread per (component, cell), component-major so that a warp's loads and stores of one
// component coalesce: three times the threads of a per-cell pass with a third of the dependent
// loads each (the pass is latency-bound).  Each component's sum is taken in the same order
// as before: owner faces, neighbour faces, displacement faces, symmetry faces.
// sums of one cell for K components: the face lists are read once for all of them, each
// component keeps its own summation order (body force, owner faces, neighbour faces,
// displacement faces, symmetry faces, inertia)
template <int K>
__device__ __forceinline__ void finish_cell(int P, int nc, int nflux, int ni, const int32_t* __restrict__ fo_ptr,
                                            const int32_t* __restrict__ fn_ptr, const double* __restrict__ Fn,
                                            const int32_t* __restrict__ fd_ptr, const int32_t* __restrict__ fs_ptr,
                                            const double* __restrict__ F, const double* __restrict__ b0, double load,
                                            const double* __restrict__ u, const double* __restrict__ vol,
                                            const double* __restrict__ rc, double mk, double* r)
{
#pragma unroll
    for (int k = 0; k < K; k++) r[k] = load * b0[(size_t)k * nc + P];
    const int o0 = fo_ptr[P], o1 = fo_ptr[P + 1], n0 = fn_ptr[P], n1 = fn_ptr[P + 1];
    const int d0 = fd_ptr[P], d1 = fd_ptr[P + 1], s0 = fs_ptr[P], s1 = fs_ptr[P + 1];
    for (int f = o0; f < o1; f++)
#pragma unroll
        for (int k = 0; k < K; k++) r[k] += F[(size_t)k * nflux + f];
    for (int q = n0; q < n1; q++)
#pragma unroll
        for (int k = 0; k < K; k++) r[k] -= Fn[(size_t)k * ni + q];
    for (int f = d0; f < d1; f++)
#pragma unroll
        for (int k = 0; k < K; k++) r[k] += F[(size_t)k * nflux + f];
    for (int f = s0; f < s1; f++)
#pragma unroll
        for (int k = 0; k < K; k++) r[k] += F[(size_t)k * nflux + f];
    if (rc) {
        const double V = vol[P];
#pragma unroll
        for (int k = 0; k < K; k++) r[k] -= V * fma(mk, u[(size_t)k * nc + P], rc[(size_t)k * nc + P]);
    }
}

__global__ void __launch_bounds__(512) k_finish(int nc, int nflux, int ni, int dim, const int32_t* __restrict__ fo_ptr,
                                                const int32_t* __restrict__ fn_ptr, const double* __restrict__ Fn,
                                                const int32_t* __restrict__ fd_ptr, const int32_t* __restrict__ fs_ptr,
                                                const double* __restrict__ F,
                                                const double* __restrict__ b0, const double* __restrict__ load_dev, int mode,
                                                const double* __restrict__ Ru, const ProbDev* __restrict__ pd,
                                                const int32_t* __restrict__ cell_prob, const int* __restrict__ gate,
                                                const double* __restrict__ u, const double* __restrict__ vol,
                                                const double* __restrict__ rc, double mk, double* __restrict__ out,
                                                RowMap rm)
{
    JF_PDL_ENTRY();
    if (gate && *gate) return;
    const double load = *load_dev;
    // one cell per thread, all components, over the row map's cells in warp-uniform rounds
    const int tot = rm.total();
    for (int64_t tw = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); tw < tot; tw += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)tw + (int)(threadIdx.x & 31u);
        const int P = warp_row(rm, v, (int)tw, tot);
        if (v >= tot) continue;
        double r[3];
        if (dim == 2) {
            finish_cell<2>(P, nc, nflux, ni, fo_ptr, fn_ptr, Fn, fd_ptr, fs_ptr, F, b0, load, u, vol, rc, mk, r);
            r[2] = 0.0;
        } else {
            finish_cell<3>(P, nc, nflux, ni, fo_ptr, fn_ptr, Fn, fd_ptr, fs_ptr, F, b0, load, u, vol, rc, mk, r);
        }
        const int K = dim == 2 ? 2 : 3;
        if (mode == 1) {
            const ProbDev& Q = pd[cell_prob[P]];
            const double eps = Q.eps, ieps = Q.ieps;
            for (int k = 0; k < K; k++)  // 1 / eps, formed once per problem
                r[k] = eps == 0.0 ? 0.0 : (r[k] - Ru[(size_t)k * nc + P]) * ieps;
        }
#pragma unroll
        for (int k = 0; k < 3; k++) out[(size_t)k * nc + P] = r[k];
    }
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// Makes the device copy of the load factor equal to c->load (rare: once per load step).  The
// copy is ordered in the call's stream, from pinned memory, so the kernels enqueued after it
// read the new factor.  (A plain cudaMemcpy from pageable memory may return before its DMA
// lands, and kernels on a non-blocking stream do not wait for the legacy stream: under load
// from other contexts they read the old factor.)
int sync_load(jfnk_ctx* c)
{
    if (c->load_on_device == c->load) return JFNK_OK;
    JF_CUDA(c, cudaStreamSynchronize(c->cur));  // an earlier copy from the pinned slot is done
    c->scal_h[0] = c->load;
    JF_CUDA(c, cudaMemcpyAsync(&c->gdev->load, c->scal_h, sizeof(double), cudaMemcpyHostToDevice, c->cur));
    c->load_on_device = c->load;
    return JFNK_OK;
}

int residual_gated(jfnk_ctx* c, const double* u_int, double* out, int mode, const int* gate, int skip)
{
    return residual_bufs(c, u_int, out, mode, gate, c->G, c->T, c->F, c->Fn, nullptr, skip);
}

int residual_bufs(jfnk_ctx* c, const double* u_int, double* out, int mode, const int* gate, double* G, double* T,
                  double* F, double* Fn, const double* load_dev, int skip)
{
    const DevMesh& m = c->dm;
    const double* load = load_dev ? load_dev : (const double*)&c->gdev->load;
    // rows of the problems taking part (compacted for a batch's passes that leave problems
    // out; the maps of SKIP_CYCLE are built at the start of each Arnoldi iteration)
    const bool part = skip != SKIP_NONE && c->nprob > 1 && c->skip_done;
    if (part && skip == SKIP_INACTIVE) {
        const int rc = rowmap_build(c, SKIP_INACTIVE);
        if (rc) return rc;
    }
    const RowMap rcell = part ? rowmap(c, SPACE_CELLS, skip, m.nc) : RowMap{nullptr, nullptr, nullptr, m.nc};
    const RowMap rface = part ? rowmap(c, SPACE_FACES, skip, m.nflux) : RowMap{nullptr, nullptr, nullptr, m.nflux};
    static const char* const kNames[3] = {"grad", "flux", "finish"};
    int sl[3];
    for (int q = 0; q < 3; q++) sl[q] = c->prof.enabled ? c->prof.slot(kNames[q]) : -1;
    jfnk_prof_begin(c, sl[0]);
    const Tuning& tu = c->tune;
#define JF_GRAD_BS(LAW_, BS_)                                                                                   \
    jfnk_launch(c, k_grad<LAW_, BS_>, dim3(rowmap_blocks(c, (const void*)k_grad<LAW_, BS_>, BS_, m.nc, BS_, rcell, 4)),  \
                dim3(BS_), gate, m.nc, m.dim, m.sell_off, m.sell_w, m.sell_nbr, m.sell_l, m.n_slots, u_int, G, T,  \
                c->mat, (const int32_t*)c->cell_prob, (const double*)m.sym_n, m.nsy, rcell, (const double*)c->ul_Gn, \
                (const double*)c->ul_F)
#define JF_GRAD(LAW_)                                     \
    do {                                                  \
        if (tu.grad_bs == 64) JF_GRAD_BS(LAW_, 64);       \
        else if (tu.grad_bs == 256) JF_GRAD_BS(LAW_, 256); \
        else JF_GRAD_BS(LAW_, 128);                       \
    } while (0)
    if (c->law_mode == 0) JF_GRAD(JFNK_LAW_LINEAR);
    else if (c->law_mode == 1) JF_GRAD(JFNK_LAW_NEOHOOKEAN);
    else if (c->law_mode == kLawUpdated) JF_GRAD(kLawUpdated);
    else JF_GRAD(2);
#undef JF_GRAD
#undef JF_GRAD_BS
    JF_LAUNCHED(c);
    jfnk_prof_end(c, sl[0]);
    if (m.nflux > 0) {
        jfnk_prof_begin(c, sl[1]);
#define JF_FLUX_BS(LAW_, BS_, ST_)                                                                                      \
    jfnk_launch(c, k_flux<LAW_, BS_, ST_>, dim3(rowmap_blocks(c, (const void*)k_flux<LAW_, BS_, ST_>, BS_, m.nflux, BS_, rface, 4)), \
                dim3(BS_), gate, m.ni, m.nd, m.nflux, m.nc, m.own, m.nei, m.coef, u_int, (const double*)G, (const double*)T, \
                m.bval, load, m.fn_pos, c->mat, (const int32_t*)c->cell_prob, F, Fn, rface)
#define JF_FLUX(LAW_)                                                        \
    do {                                                                     \
        if (tu.flux_bs == 128) {                                             \
            if (tu.flux_stage) JF_FLUX_BS(LAW_, 128, 1);                     \
            else JF_FLUX_BS(LAW_, 128, 0);                                   \
        } else {                                                             \
            if (tu.flux_stage) JF_FLUX_BS(LAW_, 256, 1);                     \
            else JF_FLUX_BS(LAW_, 256, 0);                                   \
        }                                                                    \
    } while (0)
        if (c->law_mode == 0) JF_FLUX(JFNK_LAW_LINEAR);
        else if (c->law_mode == 1) JF_FLUX(JFNK_LAW_NEOHOOKEAN);
        else if (c->law_mode == kLawUpdated) JF_FLUX(kLawUpdated);
        else JF_FLUX(2);
#undef JF_FLUX
#undef JF_FLUX_BS
        JF_LAUNCHED(c);
        jfnk_prof_end(c, sl[1]);
    }
    jfnk_prof_begin(c, sl[2]);
    jfnk_launch(c, k_finish, dim3(rowmap_blocks(c, (const void*)k_finish, tu.finish_bs, (long)m.nc, tu.finish_bs, rcell)),
                dim3(tu.finish_bs), m.nc, m.nflux, m.ni, m.dim, m.fo_ptr, m.fn_ptr, Fn, m.fd_ptr,
                (const int32_t*)m.fs_ptr, (const double*)F, m.b0,
                load, mode, c->Ru, c->pd, c->cell_prob, gate, u_int, (const double*)m.V,
                (const double*)(c->dyn_on ? c->dyn_rc : nullptr), c->dyn_mk, out, rcell);
    JF_LAUNCHED(c);
    jfnk_prof_end(c, sl[2]);
    return JFNK_OK;
}

int gradient_only(jfnk_ctx* c, const double* u_int, double* Gout)
{
    const DevMesh& m = c->dm;
    jfnk_launch(c, k_grad<JFNK_LAW_LINEAR, 128>, dim3(nblk(m.nc, 128)), dim3(128), (const int*)nullptr, m.nc, m.dim,
                m.sell_off, m.sell_w, m.sell_nbr, m.sell_l, m.n_slots, u_int, Gout, (double*)nullptr, c->mat,
                (const int32_t*)c->cell_prob, (const double*)m.sym_n, m.nsy, RowMap{nullptr, nullptr, nullptr, m.nc},
                (const double*)nullptr, (const double*)nullptr);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int residual(jfnk_ctx* c, const double* u_int, double* out, int mode, int skip)
{
    int rc = sync_load(c);
    if (rc) return rc;
    return residual_gated(c, u_int, out, mode, nullptr, skip);
}

}  // namespace jfnk
