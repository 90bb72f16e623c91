// The C ABI (include/jfnk_gb300.h): context life cycle, problem definition, hot-path calls,
// inspection and kernel timing.  Argument marshalling and validation only; every step of
// the method runs in the device kernels of the other translation units.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <new>

#include "jfnk_internal.h"

// ------------------------------------------------------------------ helpers
int jfnk_fail(jfnk_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int jfnk_cuda_fail(jfnk_ctx* c, cudaError_t e, const char* what)
{
    std::string m = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return jfnk_fail(c, JFNK_ECUDA, m);
}

void* jfnk_dalloc(jfnk_ctx* c, size_t bytes)
{
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemsetAsync(p, 0, bytes, c->cur ? c->cur : c->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return nullptr;
    }
    c->allocs.push_back(p);
    c->dev_bytes += (int64_t)bytes;
    return p;
}

int jfnk_upload(jfnk_ctx* c, void* dst, const void* src, size_t bytes)
{
    if (!bytes) return JFNK_OK;
    JF_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->cur ? c->cur : c->stream));
    return JFNK_OK;
}

int jfnk_download(jfnk_ctx* c, void* dst, const void* src, size_t bytes)
{
    cudaStream_t s = c->cur ? c->cur : c->stream;
    if (bytes) JF_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    JF_CUDA(c, cudaStreamSynchronize(s));
    return JFNK_OK;
}

int jfnk_use_stream(jfnk_ctx* c, cudaStream_t s)
{
    if (!s) s = c->stream;
    if (c->cur && c->cur != s) {
        // the previous call's work (on its stream) comes before this call's on the device; a
        // stream being captured is left to the caller's ordering
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        JF_CUDA(c, cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            JF_CUDA(c, cudaEventRecord(c->sw_ev, c->cur));
            JF_CUDA(c, cudaStreamWaitEvent(s, c->sw_ev, 0));
        }
    }
    c->cur = s;
    return JFNK_OK;
}

int jfnk::Profiler::slot(const char* name)
{
    for (size_t i = 0; i < slots.size(); i++)
        if (slots[i].name == name) return (int)i;
    slots.push_back(Slot());
    slots.back().name = name;
    return (int)slots.size() - 1;
}

void jfnk_prof_begin(jfnk_ctx* c, int slot)
{
    if (slot < 0 || !c->prof.enabled) return;
    auto& s = c->prof.slots[slot];
    if (s.used + 2 > s.ev.size()) {
        for (int q = 0; q < 64; q++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            s.ev.push_back(e);
        }
    }
    cudaEventRecord(s.ev[s.used], c->cur);
}

void jfnk_prof_end(jfnk_ctx* c, int slot)
{
    if (slot < 0 || !c->prof.enabled) return;
    auto& s = c->prof.slots[slot];
    cudaEventRecord(s.ev[s.used + 1], c->cur);
    s.used += 2;
    s.launches++;
    if (s.used + 2 > 4096) {
        // fold completed pairs into the running total to bound the event pool
        cudaEventSynchronize(s.ev[s.used - 1]);
        for (size_t q = 0; q < s.used; q += 2) {
            float ms = 0;
            cudaEventElapsedTime(&ms, s.ev[q], s.ev[q + 1]);
            s.ms += ms;
        }
        s.used = 0;
    }
}

static void free_device(jfnk_ctx* c)
{
    if (c->cur && c->cur != c->stream) cudaStreamSynchronize(c->cur);  // the last call's stream
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->it_graph) cudaGraphExecDestroy(c->it_graph);
    c->it_graph = nullptr;
    if (c->seg_graph) cudaGraphExecDestroy(c->seg_graph);
    c->seg_graph = nullptr;
    c->seg_slot = c->seg_sbeg = c->seg_scnt = nullptr;
    c->seg_state = nullptr;
    c->load_on_device = -1.0;
    jfnk::mg_release(c);
    jfnk::rowmap_release(c);
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->dev_bytes = 0;
    c->dm = jfnk::DevMesh();
    c->u = c->Ru = c->w = c->R = c->z = c->x = c->bvec = c->wk = c->tmp = c->ext = nullptr;
    c->G = c->T = c->F = c->Fn = c->partials = c->V = nullptr;
    c->Zaug = c->AZaug = c->rprev = c->dcorr = nullptr;
    c->pd = nullptr;
    c->gdev = nullptr;
    c->ul_pts0 = c->ul_F = c->ul_un = c->ul_Gn = nullptr;
    c->ul_pc_ptr = c->ul_pc_cell = nullptr;
    c->ch_beg = nullptr;
    c->ch_len = c->ch_prob = c->pch_beg = c->pch_cnt = c->cell_prob = c->pmask = nullptr;
    c->mat = MatDev{};
    c->n_chunks = 0;
    c->mg_ready = false;
}

static bool valid_options(const jfnk_options* o, std::string& why)
{
    if (o->gmres_restart < 1 || o->gmres_restart > jfnk::kMaxRestart) { why = "gmres_restart must be in [1, 64]"; return false; }
    if (!(o->gmres_eta > 0 && o->gmres_eta < 1)) { why = "gmres_eta must be in (0, 1)"; return false; }
    if (o->gmres_max_restarts < 1) { why = "gmres_max_restarts must be >= 1"; return false; }
    if (!(o->newton_rtol >= 0) || !(o->newton_atol >= 0)) { why = "tolerances must be >= 0"; return false; }
    if (o->pc < JFNK_PC_NONE || o->pc > JFNK_PC_MG) { why = "unknown preconditioner"; return false; }
    if (o->precision != JFNK_PREC_FP64 && o->precision != JFNK_PREC_MIXED) { why = "unknown precision"; return false; }
    if (!(o->jv_eps_scale > 0)) { why = "jv_eps_scale must be > 0"; return false; }
    if (o->mg_coarse_max < 1 || o->mg_coarse_max > 8192) { why = "mg_coarse_max must be in [1, 8192]"; return false; }
    if (o->autotune != 0 && o->autotune != 1) { why = "autotune must be 0 or 1"; return false; }
    if (o->pc_side != 0 && o->pc_side != 1) { why = "pc_side must be 0 (right) or 1 (left)"; return false; }
    if (!(o->seg_inner_tol > 0 && o->seg_inner_tol < 1)) { why = "seg_inner_tol must be in (0, 1)"; return false; }
    if (!(o->density >= 0) || (o->density > 0 && !(o->dt > 0))) { why = "density must be >= 0, and dt > 0 when density > 0"; return false; }
    if (o->seg_max_outer < 1 || o->seg_max_inner < 1) { why = "seg_max_outer and seg_max_inner must be >= 1"; return false; }
    if (o->gmres_aug < 0 || o->gmres_aug > 8 || o->gmres_aug >= o->gmres_restart) {
        why = "gmres_aug must be in [0, min(8, gmres_restart - 1)]";
        return false;
    }
    return true;
}

extern "C" {

void jfnk_default_options(jfnk_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->device = 0;
    o->gmres_restart = 30;
    o->gmres_eta = 1e-3;
    o->gmres_max_restarts = 100;
    o->newton_rtol = 1e-8;
    o->newton_atol = 1e-50;
    o->newton_max_its = 50;
    o->line_search_max = 10;
    o->alpha_residual = 1.0;
    o->alpha_pc = 1.0;
    o->jv_eps_scale = 1e-7;
    o->pc = JFNK_PC_BJACOBI;
    o->precision = JFNK_PREC_FP64;
    o->reorth = 2;
    o->renumber = 1;
    o->mg_max_levels = 25;
    o->mg_coarse_max = 1000;
    o->mg_theta = 0.4;
    o->mg_smooth_sweeps = 2;
    o->mg_smoothed = 1;
    o->autotune = 1;
    o->gmres_aug = 2;
    o->seg_inner_tol = 0.9;
    o->seg_max_outer = 100000;
    o->seg_max_inner = 1000;
    o->density = 0.0;
    o->dt = 0.0;
    o->pc_side = 0;
}

int jfnk_create(jfnk_ctx** out, const jfnk_options* opt)
{
    if (!out) return JFNK_EINVAL;
    *out = nullptr;
    jfnk_ctx* c = new (std::nothrow) jfnk_ctx();
    if (!c) return JFNK_ENOMEM;
    if (opt) c->opt = *opt;
    else jfnk_default_options(&c->opt);
    std::string why;
    if (!valid_options(&c->opt, why)) {
        delete c;
        return JFNK_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->opt.device < 0 || c->opt.device >= ndev) {
        cudaGetLastError();
        delete c;
        return JFNK_ECUDA;
    }
    if (cudaSetDevice(c->opt.device) != cudaSuccess || cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return JFNK_ECUDA;
    }
    if (cudaHostAlloc((void**)&c->gh, sizeof(jfnk::GlobalDev), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->gh_dev, c->gh, 0) != cudaSuccess ||
        cudaMallocHost(&c->scal_h, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(c->stream);
        delete c;
        return JFNK_ENOMEM;
    }
    for (auto& e : c->it_ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->sw_ev, cudaEventDisableTiming);
    // programmatic dependent launch of the hot-path kernels (JFNK_PDL=1).  Off by default: with
    // the iteration replayed as a CUDA graph it measured slower on GB300 (the kernels have no
    // prologue to overlap, and the early-resident blocks only wait); same kernels and results
    // either way
    if (const char* v = getenv("JFNK_PDL")) c->pdl = atoi(v) != 0;
    // a batch's problems whose Krylov cycle is done (or that left the Newton iteration) skip
    // the residual passes and the V-cycle of each Arnoldi iteration (JFNK_SKIP_DONE=0 runs
    // every row every time; the results are the same bit for bit, only the work differs)
    if (const char* v = getenv("JFNK_SKIP_DONE")) c->skip_done = atoi(v) != 0;
    c->cur = c->stream;
    *out = c;
    return JFNK_OK;
}

int jfnk_destroy(jfnk_ctx* c)
{
    if (!c) return JFNK_OK;
    cudaSetDevice(c->opt.device);
    free_device(c);
    for (auto& s : c->prof.slots)
        for (auto e : s.ev) cudaEventDestroy(e);
    for (auto e : c->it_ev)
        if (e) cudaEventDestroy(e);
    if (c->sw_ev) cudaEventDestroy(c->sw_ev);
    if (c->gh) cudaFreeHost(c->gh);
    if (c->ph) cudaFreeHost(c->ph);
    if (c->scal_h) cudaFreeHost(c->scal_h);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return JFNK_OK;
}

const char* jfnk_last_error(const jfnk_ctx* c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

int jfnk_set_options(jfnk_ctx* c, const jfnk_options* opt)
{
    if (!c || !opt) return JFNK_EINVAL;
    std::string why;
    if (!valid_options(opt, why)) return jfnk_fail(c, JFNK_EINVAL, why);
    if (opt->device != c->opt.device) return jfnk_fail(c, JFNK_EINVAL, "the device of a context cannot change");
    c->opt = *opt;
    c->dirty = true;
    return JFNK_OK;
}

int jfnk_set_mesh(jfnk_ctx* c, int dim, int32_t n_points, const double* points, int32_t n_faces, const int32_t* face_ptr,
                  const int32_t* face_pts, const int32_t* owner, int32_t n_internal, const int32_t* neighbour, int32_t n_cells)
{
    if (!c) return JFNK_EINVAL;
    if ((dim != 2 && dim != 3) || n_points <= 0 || n_faces <= 0 || n_cells <= 0 || n_internal < 0 || n_internal > n_faces ||
        !points || !face_ptr || !face_pts || !owner || (n_internal > 0 && !neighbour))
        return jfnk_fail(c, JFNK_EINVAL, "jfnk_set_mesh: invalid sizes or null arrays");
    if (c->is_batch) return jfnk_fail(c, JFNK_ESTATE, "jfnk_set_mesh on a batch context (problems are added with jfnk_batch_add)");
    if (face_ptr[0] != 0) return jfnk_fail(c, JFNK_EINVAL, "face_ptr[0] must be 0");
    for (int32_t f = 0; f < n_faces; f++) {
        if (face_ptr[f + 1] - face_ptr[f] < 3) return jfnk_fail(c, JFNK_EINVAL, "every face needs >= 3 points");
        if (owner[f] < 0 || owner[f] >= n_cells) return jfnk_fail(c, JFNK_EINVAL, "owner index out of range");
        if (f < n_internal && (neighbour[f] < 0 || neighbour[f] >= n_cells || neighbour[f] == owner[f]))
            return jfnk_fail(c, JFNK_EINVAL, "neighbour index out of range or equal to the owner");
    }
    for (int64_t q = 0; q < face_ptr[n_faces]; q++)
        if (face_pts[q] < 0 || face_pts[q] >= n_points) return jfnk_fail(c, JFNK_EINVAL, "face point index out of range");
    jfnk::HostMesh& h = c->hm;
    h.dim = dim; h.np = n_points; h.nf = n_faces; h.ni = n_internal; h.nc = n_cells;
    h.pts.assign(points, points + 3 * (size_t)n_points);
    h.fptr.assign(face_ptr, face_ptr + n_faces + 1);
    h.fpts.assign(face_pts, face_pts + face_ptr[n_faces]);
    h.own.assign(owner, owner + n_faces);
    h.nei.assign(neighbour, neighbour + n_internal);
    h.btype.assign(n_faces - n_internal, JFNK_BC_TRAC);
    h.bval.assign((size_t)(n_faces - n_internal) * 3, 0.0);
    c->fb_host.clear();
    c->have_mesh = true;
    c->dirty = true;
    return JFNK_OK;
}

int jfnk_set_patch(jfnk_ctx* c, int32_t first_face, int32_t n_faces, int bc_type, const double* values)
{
    if (!c) return JFNK_EINVAL;
    if (!c->have_mesh) return jfnk_fail(c, JFNK_ESTATE, "jfnk_set_patch before jfnk_set_mesh");
    if (first_face < c->hm.ni || n_faces < 0 || first_face + n_faces > c->hm.nf)
        return jfnk_fail(c, JFNK_EINVAL, "patch faces must be boundary faces");
    if (bc_type != JFNK_BC_DISP && bc_type != JFNK_BC_TRAC && bc_type != JFNK_BC_SYMM && bc_type != JFNK_BC_EMPTY)
        return jfnk_fail(c, JFNK_EINVAL, "unknown boundary condition type");
    for (int32_t k = 0; k < n_faces; k++) {
        const int b = first_face - c->hm.ni + k;
        c->hm.btype[b] = bc_type;
        for (int q = 0; q < 3; q++) c->hm.bval[(size_t)b * 3 + q] = values ? values[(size_t)k * 3 + q] : 0.0;
    }
    c->dirty = true;
    return JFNK_OK;
}

int jfnk_set_material(jfnk_ctx* c, int law, double p1, double p2)
{
    if (!c) return JFNK_EINVAL;
    if (law == JFNK_LAW_LINEAR || law == JFNK_LAW_STVK) {
        if (!(p1 > 0) || !(p2 > -1.0 && p2 < 0.5))
            return jfnk_fail(c, JFNK_EINVAL, "linear and St. Venant-Kirchhoff laws need E > 0 and -1 < nu < 1/2");
        c->mu = p1 / (2.0 * (1.0 + p2));
        c->lam = p1 * p2 / ((1.0 + p2) * (1.0 - 2.0 * p2));
        c->kappa = c->lam + 2.0 * c->mu / 3.0;
    } else if (law == JFNK_LAW_NEOHOOKEAN) {
        if (!(p1 > 0) || !(p2 > 0)) return jfnk_fail(c, JFNK_EINVAL, "neo-Hookean law needs mu > 0 and kappa > 0");
        c->mu = p1;
        c->kappa = p2;
        c->lam = p2 - 2.0 * p1 / 3.0;
    } else {
        return jfnk_fail(c, JFNK_EINVAL, "unknown material law");
    }
    c->law = law;
    c->p1 = p1;
    c->p2 = p2;
    c->Kbar = 4.0 * c->mu / 3.0 + c->kappa;
    c->have_material = true;
    c->dirty = true;
    return JFNK_OK;
}

int jfnk_set_body_force(jfnk_ctx* c, const double* fb)
{
    if (!c) return JFNK_EINVAL;
    if (!c->have_mesh) return jfnk_fail(c, JFNK_ESTATE, "jfnk_set_body_force before jfnk_set_mesh");
    if (fb) c->fb_host.assign(fb, fb + 3 * (size_t)c->hm.nc);
    else c->fb_host.clear();
    c->dirty = true;
    return JFNK_OK;
}

int jfnk_set_load_factor(jfnk_ctx* c, double lambda)
{
    if (!c) return JFNK_EINVAL;
    if (!std::isfinite(lambda)) return jfnk_fail(c, JFNK_EINVAL, "load factor must be finite");
    c->load = lambda;
    return JFNK_OK;
}

// set-up phase times, printed to stderr when JFNK_VERBOSE is set
struct SetupClock {
    bool on = getenv("JFNK_VERBOSE") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void lap(const char* what)
    {
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[jfnk] set-up %-22s %8.1f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

int jfnk_setup(jfnk_ctx* c)
{
    SetupClock clk;
    if (!c) return JFNK_EINVAL;
    if (c->is_batch ? c->batch.empty() : (!c->have_mesh || !c->have_material))
        return jfnk_fail(c, JFNK_ESTATE, "mesh and material (or batch problems) must be set before set-up");
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return jfnk_cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    free_device(c);
    c->cur = c->stream;
    // problems: the single mesh, or the batch concatenated into one mesh
    std::vector<int32_t> group;
    std::vector<std::array<double, 3>> mats;  // (law, p1, p2) per problem
    if (c->is_batch) {
        jfnk::HostMesh& h = c->hm;
        h = jfnk::HostMesh();
        h.dim = c->batch[0].hm.dim;
        int np = 0, nc = 0, nf = 0, ni = 0;
        for (auto& q : c->batch) { np += q.hm.np; nc += q.hm.nc; nf += q.hm.nf; ni += q.hm.ni; }
        h.np = np; h.nc = nc; h.nf = nf; h.ni = ni;
        // per problem: its first point, cell, internal face and boundary face, and the first
        // entries of its internal and boundary faces' point lists in the union; each problem is
        // then copied on its own host thread (internal faces of all problems first, then the
        // boundary faces, in problem order)
        const int P = (int)c->batch.size();
        std::vector<int64_t> p0(P + 1, 0), c0(P + 1, 0), i0(P + 1, 0), b0(P + 1, 0), ip0(P + 1, 0), bp0(P + 1, 0);
        for (int p = 0; p < P; p++) {
            const jfnk::HostMesh& q = c->batch[p].hm;
            p0[p + 1] = p0[p] + q.np;
            c0[p + 1] = c0[p] + q.nc;
            i0[p + 1] = i0[p] + q.ni;
            b0[p + 1] = b0[p] + (q.nf - q.ni);
            ip0[p + 1] = ip0[p] + q.fptr[q.ni];
            bp0[p + 1] = bp0[p] + (q.fptr[q.nf] - q.fptr[q.ni]);
        }
        const int64_t nbf = b0[P], nip = ip0[P];
        h.pts.resize(3 * (size_t)np);
        h.fptr.resize((size_t)nf + 1);
        h.fpts.resize((size_t)(ip0[P] + bp0[P]));
        h.own.resize(nf);
        h.nei.resize(ni);
        h.btype.resize(nbf);
        h.bval.resize(3 * (size_t)nbf);
        group.resize(nc);
        c->fb_host.assign(3 * (size_t)nc, 0.0);
        c->prob_first_cell.assign(P, 0);
        h.fptr[0] = 0;
        jfnk::host_parallel(P, 1, [&](int lo, int hi) {
            for (int p = lo; p < hi; p++) {
                const jfnk::HostMesh& q = c->batch[p].hm;
                const int32_t poff = (int32_t)p0[p], coff = (int32_t)c0[p];
                c->prob_first_cell[p] = coff;
                std::copy(q.pts.begin(), q.pts.end(), h.pts.begin() + 3 * p0[p]);
                for (int f = 0; f < q.ni; f++) {
                    const int64_t F = i0[p] + f;
                    h.own[F] = q.own[f] + coff;
                    h.nei[F] = q.nei[f] + coff;
                    h.fptr[F + 1] = (int32_t)(ip0[p] + q.fptr[f + 1]);
                }
                for (int k = 0; k < q.fptr[q.ni]; k++) h.fpts[ip0[p] + k] = q.fpts[k] + poff;
                for (int f = q.ni; f < q.nf; f++) {
                    const int64_t B = b0[p] + (f - q.ni), F = ni + B;
                    h.own[F] = q.own[f] + coff;
                    h.btype[B] = q.btype[f - q.ni];
                    for (int k = 0; k < 3; k++) h.bval[3 * B + k] = q.bval[(size_t)(f - q.ni) * 3 + k];
                    h.fptr[F + 1] = (int32_t)(nip + bp0[p] + (q.fptr[f + 1] - q.fptr[q.ni]));
                }
                for (int k = q.fptr[q.ni]; k < q.fptr[q.nf]; k++) h.fpts[nip + bp0[p] + (k - q.fptr[q.ni])] = q.fpts[k] + poff;
                if (!c->batch[p].fb.empty())
                    std::copy(c->batch[p].fb.begin(), c->batch[p].fb.end(), c->fb_host.begin() + 3 * (size_t)coff);
                std::fill(group.begin() + coff, group.begin() + coff + q.nc, (int32_t)p);
            }
        });
        for (int p = 0; p < P; p++) mats.push_back({(double)c->batch[p].law, c->batch[p].p1, c->batch[p].p2});
        c->nprob = (int)c->batch.size();
    } else {
        c->nprob = 1;
        c->prob_first_cell.assign(1, 0);
        mats.push_back({(double)c->law, c->p1, c->p2});
    }
    // material table: law, mu, lambda, kappa, alpha Kbar, alpha_pc Kbar per problem
    const int P = c->nprob;
    c->mat_host.assign(6 * (size_t)P, 0.0);
    int n_lin = 0, n_nh = 0;
    for (int p = 0; p < P; p++) {
        const int law = (int)mats[p][0];
        double mu, lam, kappa;
        if (law == JFNK_LAW_LINEAR || law == JFNK_LAW_STVK) {
            mu = mats[p][1] / (2.0 * (1.0 + mats[p][2]));
            lam = mats[p][1] * mats[p][2] / ((1.0 + mats[p][2]) * (1.0 - 2.0 * mats[p][2]));
            kappa = lam + 2.0 * mu / 3.0;
            n_lin += law == JFNK_LAW_LINEAR;
        } else {
            n_nh++;
            mu = mats[p][1];
            kappa = mats[p][2];
            lam = kappa - 2.0 * mu / 3.0;
        }
        const double Kbar = 4.0 * mu / 3.0 + kappa;
        c->mat_host[p] = law;
        c->mat_host[P + p] = mu;
        c->mat_host[2 * P + p] = lam;
        c->mat_host[3 * P + p] = kappa;
        c->mat_host[4 * P + p] = c->opt.alpha_residual * Kbar;
        c->mat_host[5 * P + p] = c->opt.alpha_pc * Kbar;
    }
    // kernels specialised for all-Hooke (0) and all-neo-Hookean (1); otherwise the law is read
    // per cell (2: mixtures and St. Venant-Kirchhoff)
    c->law_mode = (n_lin == P) ? 0 : (n_nh == P ? 1 : 2);
    clk.lap("problems and materials");
    std::string e = jfnk::build_topology(c->hm, c->opt.renumber != 0, c->topo, c->is_batch ? &group : nullptr);
    if (!e.empty()) return jfnk_fail(c, JFNK_EINVAL, e);
    if (c->form == JFNK_FORM_UPDATED_LAGRANGIAN) {
        if (c->is_batch || c->law_mode != 1 || c->hm.dim != 3 || c->topo.nsy > 0 || c->opt.density > 0)
            return jfnk_fail(c, JFNK_EINVAL,
                             "updated Lagrangian: one neo-Hookean 3-D problem without symmetry faces and without inertia");
        c->law_mode = 3;  // the neo-Hookean operator of the updated-Lagrangian form
    }
    clk.lap("topology (host)");
    const int nc = c->hm.nc;
    // problems' internal cell ranges and the internal cell -> problem map
    std::vector<int32_t> cell_prob(nc, 0);
    c->prob_c0.assign(P, 0);
    c->prob_c1.assign(P, 0);
    for (int i = 0; i < nc; i++) cell_prob[i] = c->is_batch ? group[c->topo.n2o[i]] : 0;
    for (int i = nc - 1; i >= 0; i--) c->prob_c0[cell_prob[i]] = i;
    for (int i = 0; i < nc; i++) c->prob_c1[cell_prob[i]] = i + 1;
    {
        std::vector<int32_t> lawv(P);
        for (int p = 0; p < P; p++) lawv[p] = (int32_t)c->mat_host[p];
        int32_t* dl = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * P);
        double* dm = (double*)jfnk_dalloc(c, sizeof(double) * 5 * (size_t)P);
        c->cell_prob = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * (size_t)nc);
        if (!dl || !dm || !c->cell_prob) return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the material table failed");
        int e;
        if ((e = jfnk_upload(c, dl, lawv.data(), sizeof(int32_t) * P)) ||
            (e = jfnk_upload(c, dm, c->mat_host.data() + P, sizeof(double) * 5 * (size_t)P)) ||
            (e = jfnk_upload(c, c->cell_prob, cell_prob.data(), sizeof(int32_t) * (size_t)nc)))
            return e;
        c->mat = MatDev{dl, dm, dm + P, dm + 2 * (size_t)P, dm + 3 * (size_t)P, dm + 4 * (size_t)P};
    }
    int rc = jfnk::setup_device_mesh(c);
    if (rc) return rc;
    clk.lap("mesh upload, geometry");
    rc = jfnk::setup_material_coefficients(c);
    if (rc) return rc;
    rc = jfnk::build_chunks(c);
    if (rc) return rc;
    clk.lap("coefficients, chunks");
    const size_t v3 = 3 * (size_t)nc;
    double** vecs[] = {&c->u, &c->Ru, &c->w, &c->R, &c->z, &c->x, &c->bvec, &c->wk, &c->tmp, &c->ext};
    for (double** p : vecs) {
        *p = (double*)jfnk_dalloc(c, sizeof(double) * v3);
        if (!*p) return jfnk_fail(c, JFNK_ENOMEM, "device allocation of work vectors failed");
        // a batch's problems that sit a pass out keep their old values: start from zeros
        JF_CUDA(c, cudaMemsetAsync(*p, 0, sizeof(double) * v3, c->stream));
    }
    c->G = (double*)jfnk_dalloc(c, sizeof(double) * 9 * (size_t)nc);
    c->T = (double*)jfnk_dalloc(c, sizeof(double) * (c->law_mode != 0 ? 9 * (size_t)nc : 1));
    c->F = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)std::max(1, c->dm.nflux));
    c->Fn = (double*)jfnk_dalloc(c, sizeof(double) * 3 * (size_t)std::max(1, c->dm.ni));
    c->partials = (double*)jfnk_dalloc(c, sizeof(double) * ((size_t)c->n_chunks * jfnk::kUpdSub + 64) * (jfnk::kMaxRestart + 2));
    c->V_is_float = c->opt.precision == JFNK_PREC_MIXED;
    c->V_ld = (v3 + 63) / 64 * 64;
    const size_t vbytes = (c->V_is_float ? sizeof(float) : sizeof(double)) * c->V_ld * (size_t)(c->opt.gmres_restart + 1);
    c->V = (double*)jfnk_dalloc(c, vbytes);
    c->pd = (jfnk::ProbDev*)jfnk_dalloc(c, sizeof(jfnk::ProbDev) * (size_t)P);
    c->gdev = (jfnk::GlobalDev*)jfnk_dalloc(c, sizeof(jfnk::GlobalDev));
    c->pmask = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * (size_t)P);
    if (c->opt.gmres_aug > 0) {  // loose GMRES: kept corrections, their products, r and d of the last cycle
        c->Zaug = (double*)jfnk_dalloc(c, sizeof(double) * v3 * (size_t)c->opt.gmres_aug);
        c->AZaug = (double*)jfnk_dalloc(c, sizeof(double) * v3 * (size_t)c->opt.gmres_aug);
        c->rprev = (double*)jfnk_dalloc(c, sizeof(double) * v3);
        c->dcorr = (double*)jfnk_dalloc(c, sizeof(double) * v3);
        if (!c->Zaug || !c->AZaug || !c->rprev || !c->dcorr)
            return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the loose-GMRES vectors failed");
    }
    if (!c->G || !c->T || !c->F || !c->Fn || !c->partials || !c->V || !c->pd || !c->gdev || !c->pmask)
        return jfnk_fail(c, JFNK_ENOMEM, "device allocation of solver buffers failed");
    if (c->ph_count < (size_t)P) {
        if (c->ph) cudaFreeHost(c->ph);
        c->ph = nullptr;
        if (cudaMallocHost(&c->ph, sizeof(jfnk::ProbDev) * (size_t)P) != cudaSuccess) {
            c->ph_count = 0;
            return jfnk_fail(c, JFNK_ENOMEM, "pinned host allocation failed");
        }
        c->ph_count = P;
    }
    std::memset(c->ph, 0, sizeof(jfnk::ProbDev) * (size_t)P);
    c->pmask_h_store.assign(P, 0);
    c->pmask_h = c->pmask_h_store.data();
    rc = jfnk::dynamics_setup(c);
    if (rc) return rc;
    if (c->form == JFNK_FORM_UPDATED_LAGRANGIAN && (rc = jfnk::ul_setup(c))) return rc;
    clk.lap("work vectors");
    rc = jfnk::pc_setup(c);
    if (rc) return rc;
    rc = jfnk::rowmap_setup(c);
    if (rc) return rc;
    clk.lap("preconditioner");
    // every upload and zero-fill above is ordered on the context's stream
    JF_CUDA(c, cudaStreamSynchronize(c->stream));
    rc = jfnk::autotune(c);
    if (rc) return rc;
    JF_CUDA(c, cudaStreamSynchronize(c->stream));
    clk.lap("autotune");
    c->dirty = false;
    return JFNK_OK;
}

int jfnk_batch_add(jfnk_ctx* c, const jfnk_ctx* q, int32_t* index)
{
    if (!c || !q) return JFNK_EINVAL;
    if (c->have_mesh) return jfnk_fail(c, JFNK_ESTATE, "jfnk_batch_add on a context that holds a single mesh");
    if (!q->have_mesh || !q->have_material || q->is_batch)
        return jfnk_fail(c, JFNK_ESTATE, "jfnk_batch_add: the problem needs a mesh and a material");
    if (!c->batch.empty() && c->batch[0].hm.dim != q->hm.dim)
        return jfnk_fail(c, JFNK_EINVAL, "jfnk_batch_add: all problems of a batch share the dimension");
    ProblemDef d;
    d.hm = q->hm;
    d.law = q->law;
    d.p1 = q->p1;
    d.p2 = q->p2;
    d.fb = q->fb_host;
    c->batch.push_back(std::move(d));
    c->is_batch = true;
    c->dirty = true;
    if (index) *index = (int32_t)c->batch.size() - 1;
    return JFNK_OK;
}

int jfnk_batch_size(const jfnk_ctx* c)
{
    if (!c) return JFNK_EINVAL;
    return c->is_batch ? (int)c->batch.size() : 1;
}

int jfnk_batch_problem_cells(const jfnk_ctx* c, int32_t index, int32_t* first_cell, int32_t* n_cells)
{
    if (!c) return JFNK_EINVAL;
    const int P = c->is_batch ? (int)c->batch.size() : 1;
    if (index < 0 || index >= P) return JFNK_EINVAL;
    int32_t first = 0;
    for (int p = 0; p < index; p++) first += c->batch[p].hm.nc;
    if (first_cell) *first_cell = first;
    if (n_cells) *n_cells = c->is_batch ? c->batch[index].hm.nc : c->hm.nc;
    return JFNK_OK;
}

int jfnk_batch_stats(const jfnk_ctx* c, jfnk_stats* per_problem)
{
    if (!c || !per_problem) return JFNK_EINVAL;
    if (c->pstats.empty()) return JFNK_ESTATE;
    std::memcpy(per_problem, c->pstats.data(), sizeof(jfnk_stats) * c->pstats.size());
    return JFNK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ hot-path helpers
static int begin_call(jfnk_ctx* c, void* stream)
{
    if (!c) return JFNK_EINVAL;
    if (c->dirty) {
        int rc = jfnk_setup(c);
        if (rc) return rc;
    }
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return jfnk_cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    return jfnk_use_stream(c, (cudaStream_t)stream);
}

static int load_vec(jfnk_ctx* c, const double* src, int mem, double* dst_int)
{
    const size_t bytes = sizeof(double) * 3 * (size_t)c->dm.nc;
    if (mem == JFNK_MEM_HOST) {
        JF_CUDA(c, cudaMemcpyAsync(c->ext, src, bytes, cudaMemcpyHostToDevice, c->cur));
        return jfnk::perm_in(c, c->ext, dst_int);
    }
    return jfnk::perm_in(c, src, dst_int);
}

static int store_vec(jfnk_ctx* c, const double* src_int, int mem, double* dst)
{
    const size_t bytes = sizeof(double) * 3 * (size_t)c->dm.nc;
    if (mem == JFNK_MEM_HOST) {
        int rc = jfnk::perm_out(c, src_int, c->ext);
        if (rc) return rc;
        JF_CUDA(c, cudaMemcpyAsync(dst, c->ext, bytes, cudaMemcpyDeviceToHost, c->cur));
        JF_CUDA(c, cudaStreamSynchronize(c->cur));
        return JFNK_OK;
    }
    return jfnk::perm_out(c, src_int, dst);
}

extern "C" {

int jfnk_residual(jfnk_ctx* c, const double* u, double* R, int mem, void* stream)
{
    int rc = begin_call(c, stream);
    if (rc) return rc;
    if (!u || !R || (mem != JFNK_MEM_HOST && mem != JFNK_MEM_DEVICE)) return jfnk_fail(c, JFNK_EINVAL, "jfnk_residual: bad arguments");
    if ((rc = load_vec(c, u, mem, c->u))) return rc;
    if ((rc = jfnk::residual(c, c->u, c->R, jfnk::OUT_R))) return rc;
    return store_vec(c, c->R, mem, R);
}

int jfnk_jv(jfnk_ctx* c, const double* u, const double* v, double* Jv, int mem, void* stream)
{
    int rc = begin_call(c, stream);
    if (rc) return rc;
    if (!u || !v || !Jv || (mem != JFNK_MEM_HOST && mem != JFNK_MEM_DEVICE)) return jfnk_fail(c, JFNK_EINVAL, "jfnk_jv: bad arguments");
    if ((rc = load_vec(c, u, mem, c->u))) return rc;
    if ((rc = load_vec(c, v, mem, c->z))) return rc;
    if ((rc = jfnk::residual(c, c->u, c->Ru, jfnk::OUT_R))) return rc;
    if ((rc = jfnk::pnorm(c, c->u, 2, false))) return rc;
    if ((rc = jfnk::pnorm(c, c->z, 1, false))) return rc;
    if ((rc = jfnk::perturb(c, c->u, c->z, c->w, false))) return rc;
    if ((rc = jfnk::residual(c, c->w, c->tmp, jfnk::OUT_JV))) return rc;
    return store_vec(c, c->tmp, mem, Jv);
}

int jfnk_precondition(jfnk_ctx* c, const double* v, double* z, int pc, int mem, void* stream)
{
    int rc = begin_call(c, stream);
    if (rc) return rc;
    if (!v || !z || (mem != JFNK_MEM_HOST && mem != JFNK_MEM_DEVICE) || pc < JFNK_PC_NONE || pc > JFNK_PC_MG)
        return jfnk_fail(c, JFNK_EINVAL, "jfnk_precondition: bad arguments");
    if ((rc = load_vec(c, v, mem, c->tmp))) return rc;
    if ((rc = jfnk::pc_apply(c, pc, c->tmp, c->z))) return rc;
    return store_vec(c, c->z, mem, z);
}

int jfnk_solve(jfnk_ctx* c, double* u, int mem, int n_load_steps, jfnk_stats* stats, void* stream)
{
    return jfnk_solve_method(c, u, mem, n_load_steps, stats, stream, 0);
}

}  // extern "C"

extern "C" int jfnk_solve_dynamic(jfnk_ctx* c, double* u, int mem, int n_steps, int32_t probe_cell, double* probe,
                                  int method, jfnk_stats* stats, void* stream)
{
    int rc = begin_call(c, stream);
    if (rc) return rc;
    if (!u || n_steps < 1 || (mem != JFNK_MEM_HOST && mem != JFNK_MEM_DEVICE) || method < 0 || method > 1)
        return jfnk_fail(c, JFNK_EINVAL, "jfnk_solve_dynamic: bad arguments");
    jfnk_stats local;
    jfnk_stats* st = stats ? stats : &local;
    const double saved_load = c->load;
    int status = jfnk::solve_dynamic(c, n_steps, probe_cell, probe, st, method);
    c->load = saved_load;
    if (status == JFNK_ECUDA || status == JFNK_ENOMEM || status == JFNK_ESTATE || status == JFNK_EINVAL) return status;
    if ((rc = store_vec(c, c->u, mem, u))) return rc;
    JF_CUDA(c, cudaStreamSynchronize(c->cur));
    if (status != JFNK_OK) return jfnk_fail(c, status, "a time step's Newton solve failed");
    return JFNK_OK;
}

int jfnk_solve_method(jfnk_ctx* c, double* u, int mem, int n_load_steps, jfnk_stats* stats, void* stream, int method)
{
    int rc = begin_call(c, stream);
    if (rc) return rc;
    if (!u || n_load_steps < 1 || (mem != JFNK_MEM_HOST && mem != JFNK_MEM_DEVICE))
        return jfnk_fail(c, JFNK_EINVAL, "jfnk_solve: bad arguments");
    jfnk_stats local;
    jfnk_stats* st = stats ? stats : &local;
    std::memset(st, 0, sizeof *st);
    if (method == 1 && c->law_mode == 3)
        return jfnk_fail(c, JFNK_ESTATE, "the updated-Lagrangian form is solved by the Newton-Krylov method only");
    if ((rc = load_vec(c, u, mem, c->u))) return rc;
    const double saved_load = c->load;
    int status = method == 1 ? jfnk::segregated(c, n_load_steps, st) : jfnk::newton(c, n_load_steps, st);
    c->load = saved_load;
    if (status == JFNK_ECUDA || status == JFNK_ENOMEM) return status;
    if ((rc = store_vec(c, c->u, mem, u))) return rc;
    JF_CUDA(c, cudaStreamSynchronize(c->cur));
    if (status != JFNK_OK) {
        const char* why = status == JFNK_MAXIT ? "Newton reached the iteration limit"
                        : status == JFNK_LS_FAILED ? "line search found no decrease"
                        : status == JFNK_DIVERGED ? "non-finite residual" : "solve failed";
        return jfnk_fail(c, status, why);
    }
    return JFNK_OK;
}

extern "C" {

int jfnk_get_geometry(jfnk_ctx* c, double* Sf, double* Cf, double* V, double* C)
{
    int rc = begin_call(c, nullptr);
    if (rc) return rc;
    const auto& t = c->topo;
    const int nf = t.nf, nc = t.nc;
    std::vector<double> a((size_t)3 * nf), b((size_t)3 * nf), v(nc), cc((size_t)3 * nc);
    if ((rc = jfnk_download(c, a.data(), c->dm.Sf, sizeof(double) * a.size())) ||
        (rc = jfnk_download(c, b.data(), c->dm.Cf, sizeof(double) * b.size())) ||
        (rc = jfnk_download(c, v.data(), c->dm.V, sizeof(double) * v.size())) ||
        (rc = jfnk_download(c, cc.data(), c->dm.C, sizeof(double) * cc.size())))
        return rc;
    for (int f = 0; f < nf; f++) {
        const int o = t.face_src[f];
        const double sg = t.face_flip[f] ? -1.0 : 1.0;
        for (int k = 0; k < 3; k++) {
            if (Sf) Sf[(size_t)o * 3 + k] = sg * a[(size_t)k * nf + f];
            if (Cf) Cf[(size_t)o * 3 + k] = b[(size_t)k * nf + f];
        }
    }
    for (int P = 0; P < nc; P++) {
        const int o = t.n2o[P];
        if (V) V[o] = v[P];
        for (int k = 0; k < 3; k++)
            if (C) C[(size_t)o * 3 + k] = cc[(size_t)k * nc + P];
    }
    return JFNK_OK;
}

int jfnk_get_gradient(jfnk_ctx* c, double* grad)
{
    int rc = begin_call(c, nullptr);
    if (rc) return rc;
    if (!grad) return jfnk_fail(c, JFNK_EINVAL, "null gradient buffer");
    const int nc = c->dm.nc;
    std::vector<double> g((size_t)9 * nc);
    if ((rc = jfnk_download(c, g.data(), c->G, sizeof(double) * g.size()))) return rc;
    for (int P = 0; P < nc; P++)
        for (int q = 0; q < 9; q++) grad[(size_t)c->topo.n2o[P] * 9 + q] = g[(size_t)q * nc + P];
    return JFNK_OK;
}

int jfnk_get_permutation(jfnk_ctx* c, int32_t* new_to_old)
{
    int rc = begin_call(c, nullptr);
    if (rc) return rc;
    if (!new_to_old) return jfnk_fail(c, JFNK_EINVAL, "null buffer");
    std::copy(c->topo.n2o.begin(), c->topo.n2o.end(), new_to_old);
    return JFNK_OK;
}

int jfnk_profile_enable(jfnk_ctx* c, int enable)
{
    if (!c) return JFNK_EINVAL;
    c->prof.enabled = enable != 0;
    c->prof.detail = enable >= 2;
    return JFNK_OK;
}

int jfnk_profile_get(jfnk_ctx* c, const char* name, double* total_ms, int64_t* launches)
{
    if (!c || !name) return JFNK_EINVAL;
    for (auto& s : c->prof.slots) {
        if (s.name != name) continue;
        if (s.used) {
            cudaEventSynchronize(s.ev[s.used - 1]);
            for (size_t q = 0; q < s.used; q += 2) {
                float ms = 0;
                cudaEventElapsedTime(&ms, s.ev[q], s.ev[q + 1]);
                s.ms += ms;
            }
            s.used = 0;
        }
        if (total_ms) *total_ms = s.ms;
        if (launches) *launches = s.launches;
        return JFNK_OK;
    }
    return jfnk_fail(c, JFNK_EINVAL, std::string("no kernel timed under the name ") + name);
}

int jfnk_profile_reset(jfnk_ctx* c)
{
    if (!c) return JFNK_EINVAL;
    for (auto& s : c->prof.slots) {
        if (s.used) cudaEventSynchronize(s.ev[s.used - 1]);
        s.used = 0;
        s.ms = 0;
        s.launches = 0;
    }
    return JFNK_OK;
}

int jfnk_synchronize(jfnk_ctx* c)
{
    if (!c) return JFNK_EINVAL;
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return jfnk_cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    JF_CUDA(c, cudaStreamSynchronize(c->cur ? c->cur : c->stream));
    return JFNK_OK;
}

int64_t jfnk_launch_count(const jfnk_ctx* c) { return c ? c->launches : 0; }

int64_t jfnk_device_bytes(const jfnk_ctx* c) { return c ? c->dev_bytes : 0; }

}  // extern "C"

extern "C" int jfnk_mg_hierarchy(jfnk_ctx* c, int max_levels, int64_t* rows, int64_t* nnz_a, int64_t* nnz_p)
{
    if (!c || max_levels < 0) return JFNK_EINVAL;
    if (c->dirty) {
        const int rc = jfnk_setup(c);
        if (rc) return rc;
    }
    std::vector<int64_t> r, a, p;
    const int nl = jfnk::mg_hierarchy_info(c, r, a, p);
    for (int l = 0; l < nl && l < max_levels; l++) {
        if (rows) rows[l] = r[l];
        if (nnz_a) nnz_a[l] = a[l];
        if (nnz_p) nnz_p[l] = p[l];
    }
    return nl;
}
