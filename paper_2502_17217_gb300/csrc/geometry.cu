// Device set-up: geometry of the face-addressed mesh (Sec. 2.3), least-squares vectors
// (Eq. leastSquaresGrad), the per-face coefficients of the residual (Eqs. divStressDiscret,
// stressInterp, RhieChow, App. B) and of the approximate Jacobian J~ (Sec. 3.1).
//
// Geometry convention (the paper leaves non-planar faces open): a face is the fan of
// triangles about its point average; its area vector is the sum of the triangle area
// vectors and its centroid the area-weighted mean of the triangle centroids.  A cell is the
// polyhedron bounded by those triangles; its volume and centroid come from the tetrahedra
// joining each triangle to the mean of the cell's face centroids.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cstring>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

__global__ void k_face_geom(int nf, const int32_t* __restrict__ fptr, const int32_t* __restrict__ fpts,
                            const double* __restrict__ pts, double* __restrict__ Sf, double* __restrict__ Cf)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int s0 = fptr[f], n = fptr[f + 1] - s0;
    double ax = 0, ay = 0, az = 0;
    for (int q = 0; q < n; q++) {
        const int p = fpts[s0 + q];
        ax += pts[3 * p]; ay += pts[3 * p + 1]; az += pts[3 * p + 2];
    }
    const double rn = 1.0 / n;
    ax *= rn; ay *= rn; az *= rn;
    double sx = 0, sy = 0, sz = 0, area = 0, mx = 0, my = 0, mz = 0;
    for (int q = 0; q < n; q++) {
        const int p0 = fpts[s0 + q], p1 = fpts[s0 + (q + 1 == n ? 0 : q + 1)];
        const double e0x = pts[3 * p0] - ax, e0y = pts[3 * p0 + 1] - ay, e0z = pts[3 * p0 + 2] - az;
        const double e1x = pts[3 * p1] - ax, e1y = pts[3 * p1 + 1] - ay, e1z = pts[3 * p1 + 2] - az;
        const double tx = 0.5 * (e0y * e1z - e0z * e1y);
        const double ty = 0.5 * (e0z * e1x - e0x * e1z);
        const double tz = 0.5 * (e0x * e1y - e0y * e1x);
        const double m = sqrt(tx * tx + ty * ty + tz * tz);
        sx += tx; sy += ty; sz += tz;
        area += m;
        // triangle centroid relative to a: (e0 + e1) / 3
        mx += m * (e0x + e1x); my += m * (e0y + e1y); mz += m * (e0z + e1z);
    }
    Sf[f] = sx; Sf[nf + f] = sy; Sf[2 * nf + f] = sz;
    const double s = 1.0 / (3.0 * area);
    Cf[f] = ax + mx * s; Cf[nf + f] = ay + my * s; Cf[2 * nf + f] = az + mz * s;
}

__global__ void k_cell_geom(int nc, int nf, const int32_t* __restrict__ ca_ptr, const int32_t* __restrict__ ca_face,
                            const int32_t* __restrict__ fptr, const int32_t* __restrict__ fpts,
                            const double* __restrict__ pts, const double* __restrict__ Cf,
                            double* __restrict__ V, double* __restrict__ C, int32_t* err)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const int a0 = ca_ptr[P], a1 = ca_ptr[P + 1];
    double cx = 0, cy = 0, cz = 0;
    for (int k = a0; k < a1; k++) {
        int f = ca_face[k];
        if (f < 0) f = ~f;
        cx += Cf[f]; cy += Cf[nf + f]; cz += Cf[2 * nf + f];
    }
    const double rk = 1.0 / (a1 - a0);
    cx *= rk; cy *= rk; cz *= rk;
    double vol = 0, mx = 0, my = 0, mz = 0;
    for (int k = a0; k < a1; k++) {
        int f = ca_face[k];
        const double sgn = f < 0 ? -1.0 : 1.0;
        if (f < 0) f = ~f;
        const int s0 = fptr[f], n = fptr[f + 1] - s0;
        double ax = 0, ay = 0, az = 0;
        for (int q = 0; q < n; q++) {
            const int p = fpts[s0 + q];
            ax += pts[3 * p]; ay += pts[3 * p + 1]; az += pts[3 * p + 2];
        }
        const double rn = 1.0 / n;
        ax *= rn; ay *= rn; az *= rn;
        const double hx = ax - cx, hy = ay - cy, hz = az - cz;
        for (int q = 0; q < n; q++) {
            const int p0 = fpts[s0 + q], p1 = fpts[s0 + (q + 1 == n ? 0 : q + 1)];
            const double e0x = pts[3 * p0] - ax, e0y = pts[3 * p0 + 1] - ay, e0z = pts[3 * p0 + 2] - az;
            const double e1x = pts[3 * p1] - ax, e1y = pts[3 * p1 + 1] - ay, e1z = pts[3 * p1 + 2] - az;
            const double tv = sgn * ((e0y * e1z - e0z * e1y) * hx + (e0z * e1x - e0x * e1z) * hy +
                                     (e0x * e1y - e0y * e1x) * hz) / 6.0;
            vol += tv;
            // tetrahedron centroid (apex + a + p0 + p1) / 4, relative to the apex
            mx += tv * (3.0 * hx + e0x + e1x);
            my += tv * (3.0 * hy + e0y + e1y);
            mz += tv * (3.0 * hz + e0z + e1z);
        }
    }
    V[P] = vol;
    const double s = 0.25 / vol;
    C[P] = cx + mx * s; C[nc + P] = cy + my * s; C[2 * nc + P] = cz + mz * s;
    if (!(vol > 0.0)) atomicMax(err, 1);
}

// Least-squares tensor G_P = sum |Gamma| d d / (d.d) over internal faces (the weight w of
// Eq. leastSquaresGrad read as 1/2 on both sums, so the gradient is exact for linear
// fields) and the stored vectors l = |Gamma| G_P^-1 d / (d.d).
// d of a sliced-ELL slot: to the neighbour's centroid, or for a symmetry face (N >= nc) to
// the cell's mirror image, d = 2 delta n with delta = n . (x_f - x_P) (Eq. leastSquaresGrad,
// reading: the mirror neighbour of Eq. symm sits at the reflection of x_P)
__device__ __forceinline__ void slot_d(int P, int N, int f, int nc, int nf, const double* __restrict__ Sf,
                                       const double* __restrict__ Cf, const double* __restrict__ C, double& dx,
                                       double& dy, double& dz)
{
    if (N < nc) {
        dx = C[N] - C[P]; dy = C[nc + N] - C[nc + P]; dz = C[2 * nc + N] - C[2 * nc + P];
        return;
    }
    const double gx = Sf[f], gy = Sf[nf + f], gz = Sf[2 * nf + f];
    const double mg = sqrt(gx * gx + gy * gy + gz * gz);
    const double nx = gx / mg, ny = gy / mg, nz = gz / mg;
    const double delta = nx * (Cf[f] - C[P]) + ny * (Cf[nf + f] - C[nc + P]) + nz * (Cf[2 * nf + f] - C[2 * nc + P]);
    dx = 2.0 * delta * nx; dy = 2.0 * delta * ny; dz = 2.0 * delta * nz;
}

__global__ void k_cell_ls(int nc, int nf, int dim, const int32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_w,
                          const int32_t* __restrict__ sell_nbr, const int32_t* __restrict__ sell_face,
                          const double* __restrict__ Sf, const double* __restrict__ Cf, const double* __restrict__ C,
                          int n_slots, double* __restrict__ sell_l, int32_t* err)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const int s = P >> 5, lane = P & 31, base = sell_off[s], w = sell_w[s];
    double g[6] = {0, 0, 0, 0, 0, 0};  // xx xy xz yy yz zz
    double scale = 0;
    for (int k = 0; k < w; k++) {
        const int slot = base + 32 * k + lane;
        const int N = sell_nbr[slot];
        if (N < 0) break;
        const int f = sell_face[slot];
        double dx, dy, dz;
        slot_d(P, N, f, nc, nf, Sf, Cf, C, dx, dy, dz);
        const double mS = sqrt(Sf[f] * Sf[f] + Sf[nf + f] * Sf[nf + f] + Sf[2 * nf + f] * Sf[2 * nf + f]);
        const double c = mS / (dx * dx + dy * dy + dz * dz);
        g[0] += c * dx * dx; g[1] += c * dx * dy; g[2] += c * dx * dz;
        g[3] += c * dy * dy; g[4] += c * dy * dz; g[5] += c * dz * dz;
        scale += mS;
    }
    double iv[9];
    if (dim == 2) {
        const double det = g[0] * g[3] - g[1] * g[1];
        if (!(fabs(det) > 1e-12 * scale * scale)) { atomicMax(err, 2); return; }
        const double r = 1.0 / det;
        iv[0] = g[3] * r; iv[1] = -g[1] * r; iv[2] = 0;
        iv[3] = -g[1] * r; iv[4] = g[0] * r; iv[5] = 0;
        iv[6] = 0; iv[7] = 0; iv[8] = 0;
    } else {
        const double c00 = g[3] * g[5] - g[4] * g[4];
        const double c01 = g[2] * g[4] - g[1] * g[5];
        const double c02 = g[1] * g[4] - g[2] * g[3];
        const double det = g[0] * c00 + g[1] * c01 + g[2] * c02;
        if (!(fabs(det) > 1e-12 * scale * scale * scale)) { atomicMax(err, 2); return; }
        const double r = 1.0 / det;
        iv[0] = c00 * r; iv[1] = c01 * r; iv[2] = c02 * r;
        iv[3] = c01 * r; iv[4] = (g[0] * g[5] - g[2] * g[2]) * r; iv[5] = (g[1] * g[2] - g[0] * g[4]) * r;
        iv[6] = c02 * r; iv[7] = iv[5]; iv[8] = (g[0] * g[3] - g[1] * g[1]) * r;
    }
    for (int k = 0; k < w; k++) {
        const int slot = base + 32 * k + lane;
        const int N = sell_nbr[slot];
        if (N < 0) break;
        const int f = sell_face[slot];
        double dx, dy, dz;
        slot_d(P, N, f, nc, nf, Sf, Cf, C, dx, dy, dz);
        const double mS = sqrt(Sf[f] * Sf[f] + Sf[nf + f] * Sf[nf + f] + Sf[2 * nf + f] * Sf[2 * nf + f]);
        const double c = mS / (dx * dx + dy * dy + dz * dz);
        sell_l[slot] = c * (iv[0] * dx + iv[1] * dy + iv[2] * dz);
        sell_l[n_slots + slot] = c * (iv[3] * dx + iv[4] * dy + iv[5] * dz);
        sell_l[2 * n_slots + slot] = c * (iv[6] * dx + iv[7] * dy + iv[8] * dz);
    }
}

// Face coefficients of the residual for internal faces [0, ni) and displacement faces
// [ni, ni+nd) (owner side; Gamma points out of the owner):
//   w  = n.(x_N - x_f) / n.(x_N - x_P)                       (Eq. stressInterp)
//   Delta = d / (d.n)                                        (Sec. 2.3.3)
//   kc = alpha Kbar |Delta| |Gamma| / |d|                    (compact Rhie-Chow part)
//   a  = alpha Kbar |Gamma| Delta                            (non-compact Rhie-Chow part)
// Hooke (small strain) folds Gamma . sigma(G) - a . G into three vectors:
//   t_j = sum_i p_i G_ij + sum_i q_i G_ji + r_j tr(G),  p = mu Gamma - a, q = mu Gamma, r = lambda Gamma.
// Neo-Hookean (total Lagrangian) keeps Gamma and a:  t = Gamma . T_f - a . G_f.
// slots: 0 w | 1 kc | 2-4 p (or Gamma) | 5-7 q (or a) | 8-10 r.  J~ gets alpha_pc Kbar |Delta||Gamma|/|d|.
// Symmetry faces [ni + nd, nflux) (Eq. symm; mirror neighbour at d = 2 delta n, Delta = n):
//   slots 0 alpha Kbar | 1 1/delta | 2-4 Gamma | 5-7 n;  J~ gets alpha_pc Kbar |Gamma| / (2 delta)
//   on the n n part of the diagonal block.
__global__ void k_flux_coef(int ni, int nd, int nflux, int nf, int nc, MatDev mat, const int32_t* __restrict__ cell_prob,
                            const int32_t* __restrict__ own, const int32_t* __restrict__ nei,
                            const double* __restrict__ Sf, const double* __restrict__ Cf, const double* __restrict__ C,
                            double* __restrict__ coef, double* __restrict__ jt_c)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nflux) return;
    const int P = own[f];
    // material of the face's problem (both cells of an internal face belong to one problem)
    const int pr = cell_prob[P];
    const int law = mat.law[pr];
    const double mu = mat.mu[pr], lam = mat.lam[pr], aK = mat.aK[pr], aKpc = mat.aKpc[pr];
    const double Gx = Sf[f], Gy = Sf[nf + f], Gz = Sf[2 * nf + f];
    const double mG = sqrt(Gx * Gx + Gy * Gy + Gz * Gz);
    const double nx = Gx / mG, ny = Gy / mG, nz = Gz / mG;
    if (f >= ni + nd) {
        const double delta = nx * (Cf[f] - C[P]) + ny * (Cf[nf + f] - C[nc + P]) + nz * (Cf[2 * nf + f] - C[2 * nc + P]);
        coef[f] = aK;
        coef[nflux + f] = 1.0 / delta;
        coef[2 * nflux + f] = Gx; coef[3 * nflux + f] = Gy; coef[4 * nflux + f] = Gz;
        coef[5 * nflux + f] = nx; coef[6 * nflux + f] = ny; coef[7 * nflux + f] = nz;
        coef[8 * nflux + f] = 0.0; coef[9 * nflux + f] = 0.0; coef[10 * nflux + f] = 0.0;
        jt_c[f] = aKpc * mG / (2.0 * delta);
        (void)mu; (void)lam; (void)law;
        return;
    }
    double dx, dy, dz, w = 1.0;
    if (f < ni) {
        const int N = nei[f];
        dx = C[N] - C[P]; dy = C[nc + N] - C[nc + P]; dz = C[2 * nc + N] - C[2 * nc + P];
        const double ex = C[N] - Cf[f], ey = C[nc + N] - Cf[nf + f], ez = C[2 * nc + N] - Cf[2 * nf + f];
        w = (nx * ex + ny * ey + nz * ez) / (nx * dx + ny * dy + nz * dz);
    } else {
        dx = Cf[f] - C[P]; dy = Cf[nf + f] - C[nc + P]; dz = Cf[2 * nf + f] - C[2 * nc + P];
    }
    const double dn = nx * dx + ny * dy + nz * dz;
    const double Dx = dx / dn, Dy = dy / dn, Dz = dz / dn;
    const double mD = sqrt(Dx * Dx + Dy * Dy + Dz * Dz), md = sqrt(dx * dx + dy * dy + dz * dz);
    const double geo = mD * mG / md;
    coef[f] = w;
    coef[nflux + f] = aK * geo;
    const double ax = aK * mG * Dx, ay = aK * mG * Dy, az = aK * mG * Dz;
    if (law == JFNK_LAW_LINEAR) {
        coef[2 * nflux + f] = mu * Gx - ax;
        coef[3 * nflux + f] = mu * Gy - ay;
        coef[4 * nflux + f] = mu * Gz - az;
        coef[5 * nflux + f] = mu * Gx;
        coef[6 * nflux + f] = mu * Gy;
        coef[7 * nflux + f] = mu * Gz;
        coef[8 * nflux + f] = lam * Gx;
        coef[9 * nflux + f] = lam * Gy;
        coef[10 * nflux + f] = lam * Gz;
    } else {
        coef[2 * nflux + f] = Gx;
        coef[3 * nflux + f] = Gy;
        coef[4 * nflux + f] = Gz;
        coef[5 * nflux + f] = ax;
        coef[6 * nflux + f] = ay;
        coef[7 * nflux + f] = az;
        coef[8 * nflux + f] = 0.0;
        coef[9 * nflux + f] = 0.0;
        coef[10 * nflux + f] = 0.0;
    }
    jt_c[f] = aKpc * geo;
}

// Constant part of the residual: body force f_b Omega_P (Eq. volume_integral) plus the
// traction faces |Gamma| Tbar (Eq. divStressDiscret); the load factor is applied at use.
__global__ void k_cell_b0(int nc, int nf, int ni, int nd, const int32_t* __restrict__ ft_ptr,
                          const double* __restrict__ Sf, const double* __restrict__ bval,
                          const double* __restrict__ V, const double* __restrict__ fb, int dim, double* __restrict__ b0)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    double b[3];
    for (int c = 0; c < 3; c++) b[c] = fb[c * nc + P] * V[P];
    for (int f = ft_ptr[P]; f < ft_ptr[P + 1]; f++) {
        const double mG = sqrt(Sf[f] * Sf[f] + Sf[nf + f] * Sf[nf + f] + Sf[2 * nf + f] * Sf[2 * nf + f]);
        const int k = f - ni;
        for (int c = 0; c < 3; c++) b[c] += mG * bval[(size_t)k * 3 + c];
    }
    if (dim == 2) b[2] = 0.0;
    for (int c = 0; c < 3; c++) b0[c * nc + P] = b[c];
}

__global__ void k_jt_diag(int nc, const int32_t* __restrict__ fo_ptr, const int32_t* __restrict__ fn_ptr,
                          const int32_t* __restrict__ fn_face, const int32_t* __restrict__ fd_ptr,
                          const double* __restrict__ jt_c, const double* __restrict__ vol, double mass,
                          double* __restrict__ diag, double* __restrict__ dinv, float* __restrict__ dinv_f)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    double s = 0;
    for (int f = fo_ptr[P]; f < fo_ptr[P + 1]; f++) s -= jt_c[f];
    for (int k = fn_ptr[P]; k < fn_ptr[P + 1]; k++) s -= jt_c[fn_face[k]];
    for (int f = fd_ptr[P]; f < fd_ptr[P + 1]; f++) s -= jt_c[f];
    s -= mass * vol[P];  // dynamics (Sec. 3.1): -(9/4) rho Omega_P / dt^2, else 0
    diag[P] = s;
    dinv[P] = 1.0 / s;
    dinv_f[P] = (float)(1.0 / s);
}

// Cells with symmetry faces have the 3x3 diagonal block B = diag I - 2 sum_s c_s n_s n_s of J~
// (Sec. 3.1): its inverse for block-Jacobi ([6][nc]: xx xy xz yy yz zz; 2-D keeps the plane
// block and 1/diag in z), the unit normals of the symmetry faces, and for the segregated
// solver the A = -J~ diagonal additions 2 sum_s c_s n_k^2 per component.
__global__ void k_jt_block(int nc, int nf, int ni, int nd, int dim, const int32_t* __restrict__ fs_ptr,
                           const double* __restrict__ Sf, const double* __restrict__ jt_c, const double* __restrict__ diag,
                           double* __restrict__ binv, float* __restrict__ binv_f, double* __restrict__ symd,
                           double* __restrict__ sym_n, int nsy)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    const double d = diag[P];
    double b[6] = {d, 0.0, 0.0, d, 0.0, d};  // xx xy xz yy yz zz
    double sd[3] = {0.0, 0.0, 0.0};
    for (int f = fs_ptr[P]; f < fs_ptr[P + 1]; f++) {
        const double gx = Sf[f], gy = Sf[nf + f], gz = Sf[2 * nf + f];
        const double mg = sqrt(gx * gx + gy * gy + gz * gz);
        const double n[3] = {gx / mg, gy / mg, gz / mg};
        const int s = f - ni - nd;
        for (int k = 0; k < 3; k++) sym_n[(size_t)k * nsy + s] = n[k];
        const double c2 = 2.0 * jt_c[f];
        b[0] -= c2 * n[0] * n[0]; b[1] -= c2 * n[0] * n[1]; b[2] -= c2 * n[0] * n[2];
        b[3] -= c2 * n[1] * n[1]; b[4] -= c2 * n[1] * n[2]; b[5] -= c2 * n[2] * n[2];
        for (int k = 0; k < 3; k++) sd[k] += c2 * n[k] * n[k];
    }
    double iv[6];
    if (dim == 2) {
        const double det = b[0] * b[3] - b[1] * b[1];
        iv[0] = b[3] / det; iv[1] = -b[1] / det; iv[2] = 0.0; iv[3] = b[0] / det; iv[4] = 0.0; iv[5] = 1.0 / d;
    } else {
        const double c00 = b[3] * b[5] - b[4] * b[4], c01 = b[2] * b[4] - b[1] * b[5], c02 = b[1] * b[4] - b[2] * b[3];
        const double det = b[0] * c00 + b[1] * c01 + b[2] * c02;
        const double r = 1.0 / det;
        iv[0] = c00 * r; iv[1] = c01 * r; iv[2] = c02 * r;
        iv[3] = (b[0] * b[5] - b[2] * b[2]) * r; iv[4] = (b[1] * b[2] - b[0] * b[4]) * r; iv[5] = (b[0] * b[3] - b[1] * b[1]) * r;
    }
    for (int q = 0; q < 6; q++) {
        binv[(size_t)q * nc + P] = iv[q];
        binv_f[(size_t)q * nc + P] = (float)iv[q];
    }
    for (int k = 0; k < 3; k++) symd[(size_t)k * nc + P] = sd[k];
}

template <typename T>
static T* upload(jfnk_ctx* c, const std::vector<T>& h)
{
    T* d = (T*)jfnk_dalloc(c, sizeof(T) * (h.empty() ? 1 : h.size()));
    if (d && jfnk_upload(c, d, h.data(), sizeof(T) * h.size())) return nullptr;
    return d;
}

static inline int blocks(long n, int t) { return (int)((n + t - 1) / t); }

int setup_device_mesh(jfnk_ctx* c)
{
    const Topology& t = c->topo;
    DevMesh& m = c->dm;
    m.dim = c->hm.dim;
    m.nc = t.nc; m.ni = t.ni; m.nd = t.nd; m.nsy = t.nsy; m.nt = t.nt; m.nf = t.nf;
    m.nflux = t.ni + t.nd + t.nsy;
    m.n_slots = t.n_slots;
    m.n_slices = (t.nc + 31) / 32;
    m.pts = upload(c, c->hm.pts);
    m.fptr = upload(c, t.fptr);
    m.fpts = upload(c, t.fpts);
    m.own = upload(c, t.own);
    m.nei = upload(c, t.nei);
    m.fo_ptr = upload(c, t.fo_ptr);
    m.fn_ptr = upload(c, t.fn_ptr);
    m.fn_face = upload(c, t.fn_face);
    {
        std::vector<int32_t> pos(std::max(1, t.ni), 0);
        for (int k = 0; k < t.ni; k++) pos[t.fn_face[k]] = k;
        m.fn_pos = upload(c, pos);
    }
    m.fd_ptr = upload(c, t.fd_ptr);
    m.fs_ptr = upload(c, t.fs_ptr);
    m.ft_ptr = upload(c, t.ft_ptr);
    m.ca_ptr = upload(c, t.ca_ptr);
    m.ca_face = upload(c, t.ca_face);
    m.sell_off = upload(c, t.sell_off);
    m.sell_w = upload(c, t.sell_w);
    m.sell_nbr = upload(c, t.sell_nbr);
    m.sell_face = upload(c, t.sell_face);
    m.n2o = upload(c, t.n2o);
    m.bval = upload(c, t.bval);
    const int nc = t.nc, nf = t.nf;
    m.sell_l = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)std::max(1, t.n_slots));
    m.Sf = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nf);
    m.Cf = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nf);
    m.V = (double*)jfnk_dalloc(c, sizeof(double) * (size_t)nc);
    m.C = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nc);
    m.coef = (double*)jfnk_dalloc(c, sizeof(double) * 11 * (size_t)std::max(1, m.nflux));
    m.b0 = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nc);
    m.fb = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nc);
    m.jt_c = (double*)jfnk_dalloc(c, sizeof(double) * (size_t)std::max(1, m.nflux));
    m.jt_diag = (double*)jfnk_dalloc(c, sizeof(double) * (size_t)nc);
    m.jt_dinv = (double*)jfnk_dalloc(c, sizeof(double) * (size_t)nc);
    m.jt_dinv_f = (float*)jfnk_dalloc(c, sizeof(float) * (size_t)nc);
    m.err = (int32_t*)jfnk_dalloc(c, sizeof(int32_t));
    if (t.nsy > 0) {
        m.jt_binv = (double*)jfnk_dalloc(c, sizeof(double) * 6 * (size_t)nc);
        m.jt_binv_f = (float*)jfnk_dalloc(c, sizeof(float) * 6 * (size_t)nc);
        m.seg_symd = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nc);
        m.sym_n = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)t.nsy);
        if (!m.jt_binv || !m.jt_binv_f || !m.seg_symd || !m.sym_n)
            return jfnk_fail(c, JFNK_ENOMEM, "device allocation failed during mesh set-up");
    }
    if (!m.fs_ptr || !m.pts || !m.fptr || !m.fpts || !m.own || !m.nei || !m.fo_ptr || !m.fn_ptr || !m.fn_face || !m.fn_pos || !m.fd_ptr ||
        !m.ft_ptr || !m.ca_ptr || !m.ca_face || !m.sell_off || !m.sell_w || !m.sell_nbr || !m.sell_face || !m.n2o ||
        !m.bval || !m.sell_l || !m.Sf || !m.Cf || !m.V || !m.C || !m.coef || !m.b0 || !m.fb || !m.jt_c ||
        !m.jt_diag || !m.jt_dinv || !m.jt_dinv_f || !m.err)
        return jfnk_fail(c, JFNK_ENOMEM, "device allocation failed during mesh set-up");
    cudaStream_t s = c->stream;
    k_face_geom<<<blocks(nf, 256), 256, 0, s>>>(nf, m.fptr, m.fpts, m.pts, m.Sf, m.Cf);
    JF_LAUNCHED(c);
    k_cell_geom<<<blocks(nc, 256), 256, 0, s>>>(nc, nf, m.ca_ptr, m.ca_face, m.fptr, m.fpts, m.pts, m.Cf, m.V, m.C, m.err);
    JF_LAUNCHED(c);
    k_cell_ls<<<blocks(nc, 128), 128, 0, s>>>(nc, nf, m.dim, m.sell_off, m.sell_w, m.sell_nbr, m.sell_face, m.Sf, m.Cf,
                                              m.C, m.n_slots, m.sell_l, m.err);
    JF_LAUNCHED(c);
    int err = 0;
    JF_CUDA(c, cudaMemcpyAsync(&err, m.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    JF_CUDA(c, cudaStreamSynchronize(s));
    if (err == 1) return jfnk_fail(c, JFNK_EINVAL, "a cell has a non-positive volume");
    if (err == 2) return jfnk_fail(c, JFNK_EINVAL, "singular least-squares tensor: a cell lacks neighbours spanning the space");
    return JFNK_OK;
}

int setup_material_coefficients(jfnk_ctx* c)
{
    DevMesh& m = c->dm;
    cudaStream_t s = c->stream;
    // body force (input order -> internal SoA)
    std::vector<double> fbs((size_t)3 * m.nc, 0.0);
    if (!c->fb_host.empty())
        for (int P = 0; P < m.nc; P++)
            for (int k = 0; k < 3; k++) fbs[(size_t)k * m.nc + P] = c->fb_host[(size_t)c->topo.n2o[P] * 3 + k];
    JF_CUDA(c, cudaMemcpyAsync(m.fb, fbs.data(), sizeof(double) * fbs.size(), cudaMemcpyHostToDevice, s));
    if (m.nflux > 0) {
        k_flux_coef<<<blocks(m.nflux, 256), 256, 0, s>>>(m.ni, m.nd, m.nflux, m.nf, m.nc, c->mat, c->cell_prob, m.own,
                                                         m.nei, m.Sf, m.Cf, m.C, m.coef, m.jt_c);
        JF_LAUNCHED(c);
    }
    k_cell_b0<<<blocks(m.nc, 256), 256, 0, s>>>(m.nc, m.nf, m.ni, m.nd, m.ft_ptr, m.Sf, m.bval, m.V, m.fb, m.dim, m.b0);
    JF_LAUNCHED(c);
    const double mass = c->opt.density > 0 ? 2.25 * c->opt.density / (c->opt.dt * c->opt.dt) : 0.0;
    k_jt_diag<<<blocks(m.nc, 256), 256, 0, s>>>(m.nc, m.fo_ptr, m.fn_ptr, m.fn_face, m.fd_ptr, m.jt_c, m.V, mass,
                                                 m.jt_diag, m.jt_dinv, m.jt_dinv_f);
    JF_LAUNCHED(c);
    if (m.nsy > 0) {
        k_jt_block<<<blocks(m.nc, 256), 256, 0, s>>>(m.nc, m.nf, m.ni, m.nd, m.dim, m.fs_ptr, m.Sf, m.jt_c, m.jt_diag,
                                                     m.jt_binv, m.jt_binv_f, m.seg_symd, m.sym_n, m.nsy);
        JF_LAUNCHED(c);
    }
    JF_CUDA(c, cudaStreamSynchronize(s));
    return JFNK_OK;
}

int update_geometry(jfnk_ctx* c)
{
    DevMesh& m = c->dm;
    cudaStream_t s = c->cur ? c->cur : c->stream;
    const int nc = m.nc, nf = m.nf;
    JF_CUDA(c, cudaMemsetAsync(m.err, 0, sizeof(int32_t), s));
    k_face_geom<<<blocks(nf, 256), 256, 0, s>>>(nf, m.fptr, m.fpts, m.pts, m.Sf, m.Cf);
    JF_LAUNCHED(c);
    k_cell_geom<<<blocks(nc, 256), 256, 0, s>>>(nc, nf, m.ca_ptr, m.ca_face, m.fptr, m.fpts, m.pts, m.Cf, m.V, m.C, m.err);
    JF_LAUNCHED(c);
    k_cell_ls<<<blocks(nc, 128), 128, 0, s>>>(nc, nf, m.dim, m.sell_off, m.sell_w, m.sell_nbr, m.sell_face, m.Sf, m.Cf,
                                              m.C, m.n_slots, m.sell_l, m.err);
    JF_LAUNCHED(c);
    if (m.nflux > 0) {
        k_flux_coef<<<blocks(m.nflux, 256), 256, 0, s>>>(m.ni, m.nd, m.nflux, m.nf, m.nc, c->mat, c->cell_prob, m.own,
                                                         m.nei, m.Sf, m.Cf, m.C, m.coef, m.jt_c);
        JF_LAUNCHED(c);
    }
    k_cell_b0<<<blocks(m.nc, 256), 256, 0, s>>>(m.nc, m.nf, m.ni, m.nd, m.ft_ptr, m.Sf, m.bval, m.V, m.fb, m.dim, m.b0);
    JF_LAUNCHED(c);
    k_jt_diag<<<blocks(m.nc, 256), 256, 0, s>>>(m.nc, m.fo_ptr, m.fn_ptr, m.fn_face, m.fd_ptr, m.jt_c, m.V, 0.0,
                                                 m.jt_diag, m.jt_dinv, m.jt_dinv_f);
    JF_LAUNCHED(c);
    int err = 0;
    JF_CUDA(c, cudaMemcpyAsync(c->scal_h + 2, m.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    JF_CUDA(c, cudaStreamSynchronize(s));
    std::memcpy(&err, c->scal_h + 2, sizeof(int));
    if (err == 1) return jfnk_fail(c, JFNK_EINVAL, "a cell has a non-positive volume in the updated configuration");
    if (err == 2) return jfnk_fail(c, JFNK_EINVAL, "singular least-squares tensor in the updated configuration");
    return JFNK_OK;
}

}  // namespace jfnk
