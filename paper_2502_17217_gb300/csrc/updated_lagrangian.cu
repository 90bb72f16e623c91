// The updated-Lagrangian form of App. A (Eq. momentum_UL) on the device: each load step is
// evaluated on the configuration of the last converged one.  The residual kernels read the
// moved geometry and form the neo-Hookean operator T = j f^-1 sigma(f F_n) (residual.cu,
// k_grad); this file keeps the state between load steps:
//   F_n  [9][nc]  total deformation gradient of the last converged step,
//   u_n  [3][nc]  its displacement, G_n [9][nc] the gradient of u_n on the updated mesh,
//   the reference points (every solve starts from the reference configuration), and the cells
//   around each mesh point.
// At the end of a converged step (ul_advance): every point moves by the mean, over the cells
// sharing it, of the increment extrapolated from the cell centre with the cell gradient,
// du_P + (x_v - x_P) . (grad du)_P (exact for increments linear in space); F_n <- f F_n;
// u_n <- u; the geometry, least-squares vectors, face coefficients, load terms and the
// approximate Jacobian's diagonal are rebuilt from the moved points; G_n is the gradient of
// u_n on the moved mesh.  The unknown stays the total displacement, so the Rhie-Chow term
// acts on it as in the total-Lagrangian form.
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

static inline int nb(long n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_ul_init(int nc, double* __restrict__ F, double* __restrict__ un, double* __restrict__ Gn)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        F[(size_t)q * nc + P] = (q % 4 == 0) ? 1.0 : 0.0;
        Gn[(size_t)q * nc + P] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) un[(size_t)k * nc + P] = 0.0;
}

// pts[v] += mean over the cells P of v of du_P + (x_v - x_P) . (G_P - Gn_P), du = u - un
__global__ void k_ul_points(int np, const int32_t* __restrict__ pc_ptr, const int32_t* __restrict__ pc_cell, int nc,
                            const double* __restrict__ u, const double* __restrict__ un, const double* __restrict__ G,
                            const double* __restrict__ Gn, const double* __restrict__ C, double* __restrict__ pts)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= np) return;
    const int a = pc_ptr[v], b = pc_ptr[v + 1];
    if (a == b) return;
    const double x[3] = {pts[3 * (size_t)v], pts[3 * (size_t)v + 1], pts[3 * (size_t)v + 2]};
    double acc[3] = {0.0, 0.0, 0.0};
    for (int k = a; k < b; k++) {
        const int P = pc_cell[k];
        double r[3];
#pragma unroll
        for (int i = 0; i < 3; i++) r[i] = x[i] - C[(size_t)i * nc + P];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double e = u[(size_t)j * nc + P] - un[(size_t)j * nc + P];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const size_t q = (size_t)(3 * i + j) * nc + P;
                e += r[i] * (G[q] - Gn[q]);
            }
            acc[j] += e;
        }
    }
    const double inv = 1.0 / (double)(b - a);
#pragma unroll
    for (int j = 0; j < 3; j++) pts[3 * (size_t)v + j] += acc[j] * inv;
}

// F_n <- f F_n with f = I + (G - Gn)^T; u_n <- u
__global__ void k_ul_commit(int nc, const double* __restrict__ u, const double* __restrict__ G,
                            const double* __restrict__ Gn, double* __restrict__ F, double* __restrict__ un)
{
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    double f[9], Fn[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const size_t q = (size_t)(3 * j + i) * nc + P;
            f[3 * i + j] = (i == j ? 1.0 : 0.0) + (G[q] - Gn[q]);
        }
#pragma unroll
    for (int q = 0; q < 9; q++) Fn[q] = F[(size_t)q * nc + P];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            F[(size_t)(3 * i + j) * nc + P] = f[3 * i] * Fn[j] + f[3 * i + 1] * Fn[3 + j] + f[3 * i + 2] * Fn[6 + j];
#pragma unroll
    for (int k = 0; k < 3; k++) un[(size_t)k * nc + P] = u[(size_t)k * nc + P];
}

int ul_setup(jfnk_ctx* c)
{
    DevMesh& m = c->dm;
    const Topology& t = c->topo;
    const int nc = m.nc, np = c->hm.np;
    c->ul_pts0 = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)np);
    c->ul_F = (double*)jfnk_dalloc(c, sizeof(double) * 9 * (size_t)nc);
    c->ul_un = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)nc);
    c->ul_Gn = (double*)jfnk_dalloc(c, sizeof(double) * 9 * (size_t)nc);
    // cells around each point (internal cell numbering), each cell once per point
    std::vector<int32_t> mark(np, -1), cnt(np + 1, 0), pairs;
    pairs.reserve((size_t)8 * nc);
    for (int P = 0; P < nc; P++)
        for (int k = t.ca_ptr[P]; k < t.ca_ptr[P + 1]; k++) {
            const int f = t.ca_face[k] < 0 ? ~t.ca_face[k] : t.ca_face[k];
            for (int q = t.fptr[f]; q < t.fptr[f + 1]; q++) {
                const int v = t.fpts[q];
                if (mark[v] == P) continue;
                mark[v] = P;
                cnt[v + 1]++;
                pairs.push_back(v);
                pairs.push_back(P);
            }
        }
    for (int v = 0; v < np; v++) cnt[v + 1] += cnt[v];
    std::vector<int32_t> cell(std::max<size_t>(1, pairs.size() / 2)), fill(cnt.begin(), cnt.end() - 1);
    for (size_t k = 0; k + 1 < pairs.size(); k += 2) cell[fill[pairs[k]]++] = pairs[k + 1];
    c->ul_pc_ptr = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * (size_t)(np + 1));
    c->ul_pc_cell = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * cell.size());
    if (!c->ul_pts0 || !c->ul_F || !c->ul_un || !c->ul_Gn || !c->ul_pc_ptr || !c->ul_pc_cell)
        return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the updated-Lagrangian state failed");
    int rc;
    if ((rc = jfnk_upload(c, c->ul_pc_ptr, cnt.data(), sizeof(int32_t) * cnt.size())) ||
        (rc = jfnk_upload(c, c->ul_pc_cell, cell.data(), sizeof(int32_t) * cell.size())))
        return rc;
    cudaStream_t s = c->cur ? c->cur : c->stream;
    JF_CUDA(c, cudaMemcpyAsync(c->ul_pts0, m.pts, sizeof(double) * 3 * (size_t)np, cudaMemcpyDeviceToDevice, s));
    k_ul_init<<<nb(nc, 256), 256, 0, s>>>(nc, c->ul_F, c->ul_un, c->ul_Gn);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

int ul_reset(jfnk_ctx* c)
{
    DevMesh& m = c->dm;
    cudaStream_t s = c->cur ? c->cur : c->stream;
    JF_CUDA(c, cudaMemcpyAsync(m.pts, c->ul_pts0, sizeof(double) * 3 * (size_t)c->hm.np, cudaMemcpyDeviceToDevice, s));
    k_ul_init<<<nb(m.nc, 256), 256, 0, s>>>(m.nc, c->ul_F, c->ul_un, c->ul_Gn);
    JF_LAUNCHED(c);
    return update_geometry(c);
}

int ul_advance(jfnk_ctx* c)
{
    DevMesh& m = c->dm;
    cudaStream_t s = c->cur ? c->cur : c->stream;
    int rc;
    if ((rc = gradient_only(c, c->u, c->G))) return rc;  // grad u on the mesh of the last step
    k_ul_points<<<nb(c->hm.np, 256), 256, 0, s>>>(c->hm.np, c->ul_pc_ptr, c->ul_pc_cell, m.nc, c->u, c->ul_un, c->G,
                                                  c->ul_Gn, m.C, m.pts);
    JF_LAUNCHED(c);
    k_ul_commit<<<nb(m.nc, 256), 256, 0, s>>>(m.nc, c->u, c->G, c->ul_Gn, c->ul_F, c->ul_un);
    JF_LAUNCHED(c);
    if ((rc = update_geometry(c))) return rc;
    return gradient_only(c, c->ul_un, c->ul_Gn);
}

}  // namespace jfnk

extern "C" int jfnk_set_formulation(jfnk_ctx* c, int formulation)
{
    if (!c) return JFNK_EINVAL;
    if (formulation != JFNK_FORM_TOTAL_LAGRANGIAN && formulation != JFNK_FORM_UPDATED_LAGRANGIAN)
        return jfnk_fail(c, JFNK_EINVAL, "jfnk_set_formulation: JFNK_FORM_TOTAL_LAGRANGIAN or JFNK_FORM_UPDATED_LAGRANGIAN");
    c->form = formulation;
    c->dirty = true;
    return JFNK_OK;
}
