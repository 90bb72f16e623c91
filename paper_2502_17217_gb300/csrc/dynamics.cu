// Time integration of the momentum equation with inertia (Sec. 2.3, Eq. inertia, BDF2 of
// Eq. inertia2), for the same P >= 1 problems as the static path.
//
// The context holds the state of the two previous time levels, u_t, u_{t-1}, v_t, v_{t-1},
// and the acceleration a_t, at rest after set-up.  A time step:
//   c   = [3 (-4 u_t + u_{t-1}) / (2 dt) - 4 v_t + v_{t-1}] / (2 dt), stored as rho c, so the
//         residual's inertia term is -rho Omega_P (9/(4 dt^2) u_P + c_P);
//   u   = u_t + dt v_t + dt^2/2 a_t (the transient-continuation predictor, Eq. predictor);
//   Newton-Krylov (or segregated) solve of R(u) = 0 at full load from that guess (the J~ diagonal carries
//         -(9/4) rho Omega / dt^2, Sec. 3.1, added at set-up);
//   v_{t+1} = (3 u - 4 u_t + u_{t-1}) / (2 dt), a_{t+1} = (3 v_{t+1} - 4 v_t + v_{t-1}) / (2 dt),
//         and the levels shift.
// Density and dt are context options (one value for all problems of a batch).
#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

namespace {

__global__ void k_dyn_begin(size_t n, const double* __restrict__ ut, const double* __restrict__ utm1,
                            const double* __restrict__ vt, const double* __restrict__ vtm1,
                            const double* __restrict__ at, double rho, double dt, double* __restrict__ rc,
                            double* __restrict__ u)
{
    JF_PDL_ENTRY();
    const double i2dt = 1.0 / (2.0 * dt);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double c = (3.0 * (-4.0 * ut[e] + utm1[e]) * i2dt - 4.0 * vt[e] + vtm1[e]) * i2dt;
        rc[e] = rho * c;
        u[e] = ut[e] + dt * vt[e] + 0.5 * dt * dt * at[e];
    }
}

__global__ void k_dyn_end(size_t n, const double* __restrict__ u, double* __restrict__ ut, double* __restrict__ utm1,
                          double* __restrict__ vt, double* __restrict__ vtm1, double* __restrict__ at, double dt)
{
    JF_PDL_ENTRY();
    const double i2dt = 1.0 / (2.0 * dt);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double un = u[e], u0 = ut[e], um = utm1[e], v0 = vt[e], vm = vtm1[e];
        const double vn = (3.0 * un - 4.0 * u0 + um) * i2dt;
        at[e] = (3.0 * vn - 4.0 * v0 + vm) * i2dt;
        utm1[e] = u0;
        ut[e] = un;
        vtm1[e] = v0;
        vt[e] = vn;
    }
}

// out[3 step + k] = u_k at internal cell P
__global__ void k_dyn_probe(const double* __restrict__ u, int nc, int P, double* __restrict__ out)
{
    JF_PDL_ENTRY();
    const int k = threadIdx.x;
    if (k < 3) out[k] = u[(size_t)k * nc + P];
}

inline int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)kRedBlocks * 4); }

}  // namespace

int dynamics_setup(jfnk_ctx* c)
{
    c->dyn_on = c->opt.density > 0.0;
    c->dyn_mk = c->dyn_on ? 2.25 * c->opt.density / (c->opt.dt * c->opt.dt) : 0.0;
    c->dyn_ut = c->dyn_utm1 = c->dyn_vt = c->dyn_vtm1 = c->dyn_at = c->dyn_rc = nullptr;
    if (!c->dyn_on) return JFNK_OK;
    const size_t n = 3 * (size_t)c->dm.nc;
    double** bufs[6] = {&c->dyn_ut, &c->dyn_utm1, &c->dyn_vt, &c->dyn_vtm1, &c->dyn_at, &c->dyn_rc};
    for (auto b : bufs) {
        *b = (double*)jfnk_dalloc(c, sizeof(double) * n);  // zeroed: at rest
        if (!*b) return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the time-integration state failed");
    }
    return JFNK_OK;
}

}  // namespace jfnk

extern "C" int jfnk_dynamic_reset(jfnk_ctx* c)
{
    if (!c) return JFNK_EINVAL;
    if (c->dirty) return jfnk_fail(c, JFNK_ESTATE, "jfnk_dynamic_reset: set the context up first");
    if (!c->dyn_on) return jfnk_fail(c, JFNK_ESTATE, "jfnk_dynamic_reset: options.density is 0 (static context)");
    const int rc = jfnk_use_stream(c, nullptr);
    if (rc) return rc;
    const size_t bytes = sizeof(double) * 3 * (size_t)c->dm.nc;
    double* bufs[6] = {c->dyn_ut, c->dyn_utm1, c->dyn_vt, c->dyn_vtm1, c->dyn_at, c->dyn_rc};
    for (auto b : bufs) JF_CUDA(c, cudaMemsetAsync(b, 0, bytes, c->stream));
    JF_CUDA(c, cudaStreamSynchronize(c->stream));
    return JFNK_OK;
}

// Checkpoint and restart of the time integration: the five state fields in the caller's
// cell order, [5][n_cells][3] (u_t, u_{t-1}, v_t, v_{t-1}, a_t).
extern "C" int jfnk_dynamic_get_state(jfnk_ctx* c, double* state)
{
    if (!c || !state) return JFNK_EINVAL;
    if (c->dirty) return jfnk_fail(c, JFNK_ESTATE, "jfnk_dynamic_get_state: set the context up first");
    if (!c->dyn_on) return jfnk_fail(c, JFNK_ESTATE, "jfnk_dynamic_get_state: options.density is 0 (static context)");
    int rc = jfnk_use_stream(c, nullptr);
    if (rc) return rc;
    const size_t n = 3 * (size_t)c->dm.nc;
    const double* f[5] = {c->dyn_ut, c->dyn_utm1, c->dyn_vt, c->dyn_vtm1, c->dyn_at};
    for (int k = 0; k < 5; k++) {
        if ((rc = jfnk::perm_out(c, f[k], c->ext))) return rc;
        if ((rc = jfnk_download(c, state + k * n, c->ext, sizeof(double) * n))) return rc;
    }
    return JFNK_OK;
}

extern "C" int jfnk_dynamic_set_state(jfnk_ctx* c, const double* state)
{
    if (!c || !state) return JFNK_EINVAL;
    if (c->dirty) return jfnk_fail(c, JFNK_ESTATE, "jfnk_dynamic_set_state: set the context up first");
    if (!c->dyn_on) return jfnk_fail(c, JFNK_ESTATE, "jfnk_dynamic_set_state: options.density is 0 (static context)");
    int rc = jfnk_use_stream(c, nullptr);
    if (rc) return rc;
    const size_t n = 3 * (size_t)c->dm.nc;
    double* f[5] = {c->dyn_ut, c->dyn_utm1, c->dyn_vt, c->dyn_vtm1, c->dyn_at};
    for (int k = 0; k < 5; k++) {
        if ((rc = jfnk_upload(c, c->ext, state + k * n, sizeof(double) * n))) return rc;
        if ((rc = jfnk::perm_in(c, c->ext, f[k]))) return rc;
    }
    JF_CUDA(c, cudaStreamSynchronize(c->stream));
    return JFNK_OK;
}

namespace jfnk {

int solve_dynamic(jfnk_ctx* c, int n_steps, int32_t probe_cell, double* probe, jfnk_stats* st, int method)
{
    if (!c->dyn_on) return jfnk_fail(c, JFNK_ESTATE, "jfnk_solve_dynamic: options.density is 0 (static context)");
    const size_t n = 3 * (size_t)c->dm.nc;
    const int nc = c->dm.nc;
    const double dt = c->opt.dt, rho = c->opt.density;
    int Pint = -1;
    if (probe && probe_cell >= 0) {
        if (probe_cell >= nc) return jfnk_fail(c, JFNK_EINVAL, "jfnk_solve_dynamic: probe cell out of range");
        Pint = c->topo.o2n[probe_cell];
    }
    double* probe_dev = nullptr;
    if (Pint >= 0) JF_CUDA(c, cudaMallocAsync((void**)&probe_dev, sizeof(double) * 3 * (size_t)n_steps, c->cur));
    std::memset(st, 0, sizeof *st);
    int status = JFNK_OK;
    jfnk_stats one;
    for (int step = 0; step < n_steps; step++) {
        jfnk_launch(c, k_dyn_begin, dim3(grid_for(n)), dim3(256), n, (const double*)c->dyn_ut, (const double*)c->dyn_utm1,
                    (const double*)c->dyn_vt, (const double*)c->dyn_vtm1, (const double*)c->dyn_at, rho, dt, c->dyn_rc, c->u);
        JF_LAUNCHED(c);
        status = method == 1 ? segregated(c, 1, &one) : newton(c, 1, &one);
        st->newton_its += one.newton_its;
        st->gmres_its += one.gmres_its;
        st->jv_products += one.jv_products;
        st->residual_evals += one.residual_evals;
        st->reorth_its += one.reorth_its;
        st->arnoldi_cols += one.arnoldi_cols;
        st->reorth_cols += one.reorth_cols;
        st->final_rel_res = std::max(st->final_rel_res, one.final_rel_res);
        st->final_abs_res = one.final_abs_res;
        if (st->n_hist < 64) st->hist[st->n_hist++] = one.final_abs_res;
        if (status != JFNK_OK) break;
        st->load_steps_done++;  // time steps completed
        jfnk_launch(c, k_dyn_end, dim3(grid_for(n)), dim3(256), n, (const double*)c->u, c->dyn_ut, c->dyn_utm1,
                    c->dyn_vt, c->dyn_vtm1, c->dyn_at, dt);
        JF_LAUNCHED(c);
        if (probe_dev) {
            jfnk_launch(c, k_dyn_probe, dim3(1), dim3(32), (const double*)c->u, nc, Pint, probe_dev + 3 * (size_t)step);
            JF_LAUNCHED(c);
        }
    }
    st->status = status;
    if (probe_dev) {
        JF_CUDA(c, cudaMemcpyAsync(probe, probe_dev, sizeof(double) * 3 * (size_t)st->load_steps_done,
                                   cudaMemcpyDeviceToHost, c->cur));
        JF_CUDA(c, cudaFreeAsync(probe_dev, c->cur));
    }
    return status;
}

}  // namespace jfnk
