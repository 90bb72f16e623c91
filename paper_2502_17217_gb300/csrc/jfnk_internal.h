// Internal definitions of the GB300 JFNK library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/jfnk_gb300.h"

namespace jfnk {

constexpr int kMaxRestart = 64;   // largest m of GMRES(m)
constexpr int kRedBlocks = 608;   // 4 x 152 SMs: fixed grid of every reduction (deterministic)
constexpr int kRedThreads = 256;

// ------------------------------------------------------------------ host copy of the input
struct HostMesh {
    int dim = 3;
    int np = 0, nf = 0, ni = 0, nc = 0;
    std::vector<double> pts;                 // [np][3]
    std::vector<int32_t> fptr, fpts, own, nei;
    std::vector<int32_t> btype;              // [nf - ni]
    std::vector<double> bval;                // [nf - ni][3]
};

// ------------------------------------------------------------------ host-built topology
// Internal (device) numbering: cells renumbered, faces reordered into
//   [0, ni)                internal faces, sorted by (owner, neighbour), owner < neighbour
//   [ni, ni + nd)          displacement faces, sorted by owner
//   [ni + nd, .. + nsy)    symmetry faces, sorted by owner
//   [.., .. + nt)          traction faces, sorted by owner
//   [.., nf)               empty faces
struct Topology {
    int nc = 0, ni = 0, nd = 0, nsy = 0, nt = 0, ne = 0, nf = 0;
    std::vector<int32_t> n2o, o2n;           // cell permutation
    std::vector<int32_t> face_src;           // new face -> input face
    std::vector<uint8_t> face_flip;          // 1 if the point loop was reversed
    std::vector<int32_t> fptr, fpts;         // reordered (and flipped) face point lists
    std::vector<int32_t> own, nei;           // own [nf], nei [ni]
    std::vector<int32_t> fo_ptr;             // [nc+1] internal faces owned by each cell
    std::vector<int32_t> fn_ptr, fn_face;    // [nc+1], [ni] internal faces whose neighbour is the cell
    std::vector<int32_t> fd_ptr;             // [nc+1] displacement faces (absolute indices)
    std::vector<int32_t> fs_ptr;             // [nc+1] symmetry faces (absolute indices)
    std::vector<int32_t> ft_ptr;             // [nc+1] traction faces (absolute indices)
    std::vector<int32_t> ca_ptr, ca_face;    // all faces of each cell; ~f marks the neighbour side
    // sliced-ELL (32 cells per slice) list of the internal neighbours of each cell, then its
    // symmetry faces (the mirror neighbour, coded nc + symmetry-face index)
    std::vector<int32_t> sell_off, sell_w;   // per slice: first slot, width (slots per lane)
    std::vector<int32_t> sell_nbr, sell_face;// per slot: neighbour cell (-1 = padding), face
    int n_slots = 0;
    std::vector<double> bval;                // [nd + nsy + nt][3] boundary values in new face order
    int bandwidth = 0;
};

// Runs f(lo, hi) over [0, n) in blocks of `grain` on up to 16 host threads (setup_host.cpp);
// each block's results must depend on the block alone, so the outcome does not depend on the
// thread count.
void host_parallel(int n, int grain, const std::function<void(int, int)>& f);

// Builds the topology; returns "" on success or an error message.  With `group` (one entry
// per input cell) the cells of each group stay contiguous, groups in increasing order.
std::string build_topology(const HostMesh& hm, bool rcm, Topology& t, const std::vector<int32_t>* group = nullptr);

// ------------------------------------------------------------------ multigrid hierarchy (host)
struct MgLevelHost {
    int n = 0;
    std::vector<int32_t> rp, col;
    std::vector<double> val;
    std::vector<int32_t> agg;              // aggregate of each row (all but the coarsest level)
    std::vector<int32_t> prp, pcol;        // prolongation to the next level (CSR, n x n_next)
    std::vector<double> pval;
};
// Aggregation hierarchy on A = -J~ given in CSR (plain or smoothed prolongation) and the
// dense inverse of the coarsest matrix; returns "" on success.
std::string mg_build_hierarchy(MgLevelHost&& fine, double theta, int max_levels, int coarse_max, bool smoothed,
                               std::vector<MgLevelHost>& levels, std::vector<double>& inverse);

// ------------------------------------------------------------------ device state
struct DevMesh {
    int dim = 3, nc = 0, ni = 0, nd = 0, nsy = 0, nt = 0, nf = 0, nflux = 0, n_slots = 0, n_slices = 0;
    double* pts = nullptr;
    int32_t *fptr = nullptr, *fpts = nullptr;
    int32_t *own = nullptr, *nei = nullptr;
    int32_t *fo_ptr = nullptr, *fn_ptr = nullptr, *fn_face = nullptr, *fd_ptr = nullptr, *ft_ptr = nullptr;
    int32_t* fs_ptr = nullptr;       // [nc+1] symmetry faces of each cell
    double* sym_n = nullptr;         // [3][nsy] unit outward normals of the symmetry faces
    int32_t* fn_pos = nullptr;       // [ni] position of each internal face in the neighbour-sorted list
    int32_t *ca_ptr = nullptr, *ca_face = nullptr;
    int32_t *sell_off = nullptr, *sell_w = nullptr, *sell_nbr = nullptr, *sell_face = nullptr;
    double* sell_l = nullptr;        // [3][n_slots] least-squares vectors
    double *Sf = nullptr, *Cf = nullptr;   // [3][nf]
    double *V = nullptr, *C = nullptr;     // [nc], [3][nc]
    double* coef = nullptr;          // [11][nflux] face coefficients of the residual
    double* bval = nullptr;          // [nd + nsy + nt][3] boundary values (unscaled)
    double* b0 = nullptr;            // [3][nc] body force + traction (unscaled)
    double* fb = nullptr;            // [3][nc] body force density
    double* jt_c = nullptr;          // [nflux] J~ face coefficients (internal, displacement, symmetry)
    double* jt_diag = nullptr;       // [nc] scalar part of the diagonal blocks
    double* jt_dinv = nullptr;       // [nc] 1 / diag
    float* jt_dinv_f = nullptr;      // [nc]
    // with symmetry faces: inverses of the 3x3 diagonal blocks diag I - 2 sum c n n, [6][nc]
    // (xx xy xz yy yz zz), and the blocks' diagonals in A = -J~ form for the segregated solver
    double* jt_binv = nullptr;
    float* jt_binv_f = nullptr;
    double* seg_symd = nullptr;      // [3][nc] sum 2 c n_k^2
    int32_t* n2o = nullptr;
    int32_t* err = nullptr;          // set-up error word
};

// Chunks of the SoA vectors for per-problem (segmented) reductions: every chunk lies inside
// one problem's range of one displacement component.
constexpr int kChunk = 2048;
constexpr int kChunkThreads = 512;   // kChunk / kChunkThreads = 4 elements per thread
constexpr int kUpdSub = 4;           // sub-blocks per chunk of the basis update / combination
constexpr int kUpdE = kChunk / (kUpdSub * kChunkThreads);  // elements per thread there

// Per-problem scalars of the GMRES cycle and the Newton step, resident on the device.
struct ProbDev {
    int j;            // Arnoldi index of the iteration being built
    int k;            // iterations completed in this cycle
    int done;         // this problem's cycle is finished (converged, breakdown, full, inactive)
    int reorth;       // second Gram-Schmidt pass needed for this column
    int active;       // takes part in the current Newton step
    int n_reorth;     // second passes run (diagnostic)
    unsigned ticket[4];
    double eps;       // Jv step for the current direction
    double unorm;     // |u_p|
    double beta;      // |r_p| at the start of the cycle
    double target;    // eta |b_p|
    double inv;       // 1 / |w_p| (or 1 / beta at the cycle start)
    double wn2;       // |w_p|^2 before orthogonalisation
    double res;       // |g_k| current residual estimate
    double step;      // line-search step s_p
    double nrm;       // output of plain per-problem norms
    double n_cols;    // sum over Arnoldi iterations of the basis vectors projected out (j + 1)
    double n_rcols;   // the same over the iterations that repeated the projection
    double ieps;      // 1 / eps (0 when eps = 0), formed once where eps is set
    double pad2[4];
    double h[kMaxRestart + 1];
    double H[(kMaxRestart + 1) * kMaxRestart];  // column-major: H[i + (m+1) j]
    double g[kMaxRestart + 1];
    double cs[kMaxRestart], sn[kMaxRestart];
    double y[kMaxRestart];
};

// Conjugate-gradient state of one component system of one problem (segregated solver).
struct SegSlot {
    double rr0, rr;   // |r| at the start and now
    double rz;        // r . (preconditioned r)
    double beta, alpha;
    int its;          // CG iterations of this outer iteration
    int done;         // residual reduced enough (or no work)
    unsigned ticket;
    int pad;
};

#ifdef __CUDACC__
// Whether row i (of a multigrid level) belongs to a problem that sits out the current pass of
// a batch: the problem of each row and the per-problem flags.  A problem sits out when it left
// the Newton iteration or (inside the Arnoldi iteration) finished its Krylov cycle.  The
// batch's coarse solve uses it to zero the columns of such problems (their rows hold values of
// an earlier cycle); which rows the kernels visit is the row maps' business (RowMap below).
// prob == nullptr: no problem sits out.
struct ProbSkip {
    const int32_t* prob;
    const ProbDev* pd;
    int cycle = 1;  // 1: also the problems whose Krylov cycle is done (inside the Arnoldi iteration)
    __device__ __forceinline__ bool operator()(int i) const
    {
        if (!prob) return false;
        const ProbDev& P = pd[prob[i]];
        return !P.active || (cycle && P.done);
    }
};

// Rows of one index space (cells, faces, the rows of a multigrid level) that a launch visits.
// Identity (pre == nullptr): rows [0, n).  Compacted (batches, passes that leave problems
// out): the runs of consecutive rows of the problems taking part, concatenated in row order;
// virtual row v of run k (pre[k] <= v < pre[k + 1]) is row first[k] + v - pre[k].  The
// kernels loop over virtual rows with a grid stride, so rows of the problems that sit a pass
// out cost neither a block nor a load, and the rows a pass evaluates are the same as with
// per-row skipping: the results are bitwise equal.
struct RowMap {
    const int32_t* pre = nullptr;    // [runs + 1] rows before each run taking part
    const int32_t* first = nullptr;  // [runs] first row of each run taking part
    const int32_t* hdr = nullptr;    // {runs taking part, rows taking part}
    int n = 0;                       // rows of the space (identity)
    __device__ __forceinline__ int total() const { return pre ? __ldg(hdr + 1) : n; }
    // run of virtual row v (0 <= v < total()), by bisection
    __device__ __forceinline__ int run_of(int v) const
    {
        int lo = 0, hi = __ldg(hdr);
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(pre + mid) <= v) lo = mid;
            else hi = mid;
        }
        return lo;
    }
    __device__ __forceinline__ int row(int v) const
    {
        if (!pre) return v;
        const int k = run_of(v);
        return __ldg(first + k) + (v - __ldg(pre + k));
    }
    // row(v) from a hint k, the run of a virtual row at or before v (v < total()): a few
    // steps forward, else bisection
    __device__ __forceinline__ int row_from(int v, int k) const
    {
        if (!pre) return v;
        if (v >= __ldg(pre + k)) {
#pragma unroll 1
            for (int s = 0; s < 4; s++, k++)
                if (__ldg(pre + k + 1) > v) return __ldg(first + k) + (v - __ldg(pre + k));
        }
        return row(v);
    }
};

// Row of virtual row v for a converged warp whose lanes take rows at or after vw (the
// warp's first row, warp-uniform): lane 0 bisects for vw's run, the lanes step on from it
// (rows of one run are contiguous, so most lanes take no step).  Returns 0 for v >= tot.
__device__ __forceinline__ int warp_row(const RowMap& rm, int v, int vw, int tot)
{
    if (!rm.pre) return v;
    int k = 0;
    if ((threadIdx.x & 31) == 0 && vw < tot) k = rm.run_of(vw);
    k = __shfl_sync(0xffffffffu, k, 0);
    return v < tot ? rm.row_from(v, k) : 0;
}
#endif

// Scalars shared by all problems of a context.
struct GlobalDev {
    int jg;           // index of the lockstep Arnoldi iteration (all active problems share it)
    int all_done;     // every problem's cycle is finished: the iteration's kernels return at once
    int n_active;     // problems whose cycle is still running
    int pad;
    double load;      // load factor read by the residual kernels
};

struct Profiler {
    bool enabled = false;
    bool detail = false;  // also the multigrid's steps inside each V-cycle
    struct Slot {
        std::string name;
        std::vector<cudaEvent_t> ev;   // pairs
        size_t used = 0;
        double ms = 0;
        int64_t launches = 0;
    };
    std::vector<Slot> slots;
    int slot(const char* name);
};

}  // namespace jfnk

namespace jfnk {
// Launch shapes of the tunable kernels (chosen per mesh by the autotuner, autotune.cu):
// cells per block of the gradient and cell-sum passes, faces per block of the face pass and
// whether it stages its owner cells' gradients in shared memory, cells per block of the
// fine-level multigrid kernels.  Results do not depend on them.
struct Tuning {
    int grad_bs = 128, flux_bs = 256, flux_stage = 0, finish_bs = 256, mg_bs = 256;
    int tuned = 0;
};
}  // namespace jfnk

// A problem copied into a batch: mesh, boundary data, material, body force.
struct ProblemDef {
    jfnk::HostMesh hm;
    int law = JFNK_LAW_LINEAR;
    double p1 = 0, p2 = 0;
    std::vector<double> fb;
};

// Per-problem material constants on the device (arrays over problems).
struct MatDev {
    const int32_t* law;
    const double *mu, *lam, *kappa, *aK, *aKpc;
};

struct jfnk_ctx {
    jfnk_options opt;
    std::string err;
    cudaStream_t stream = nullptr;      // context's own stream
    cudaStream_t cur = nullptr;         // stream of the call in progress (or of the last call)
    cudaEvent_t sw_ev = nullptr;        // orders a call after the previous one on another stream
    jfnk::HostMesh hm;
    bool have_mesh = false, have_material = false;
    bool is_batch = false;
    std::vector<ProblemDef> batch;       // problems of a batch, in the order added
    std::vector<int32_t> prob_first_cell;// caller numbering: first cell of each problem
    std::vector<double> mat_host;        // [6][nprob]: law, mu, lam, kappa, Kbar(alpha), Kbar(alpha_pc)
    int law_mode = 0;                    // 0 all Hooke, 1 all neo-Hookean, 2 mixed, 3 neo-Hookean updated Lagrangian
    // updated-Lagrangian form (App. A): formulation flag, and on the device the reference
    // points, the last converged step's total deformation gradient [9][nc], displacement
    // [3][nc] and its gradient on the updated mesh [9][nc], and the point -> cell lists
    int form = 0;
    double *ul_pts0 = nullptr, *ul_F = nullptr, *ul_un = nullptr, *ul_Gn = nullptr;
    int32_t *ul_pc_ptr = nullptr, *ul_pc_cell = nullptr;
    MatDev mat{};                        // device copies
    std::vector<jfnk_stats> pstats;      // per-problem statistics of the last solve
    int32_t* pmask = nullptr;            // device [nprob]
    std::vector<int32_t> pmask_h_store;
    int32_t* pmask_h = nullptr;
    int law = JFNK_LAW_LINEAR;
    double p1 = 0, p2 = 0, mu = 0, lam = 0, kappa = 0, Kbar = 0;
    std::vector<double> fb_host;
    double load = 1.0;
    double load_on_device = -1.0;      // value last copied to gdev->load
    bool dirty = true;
    jfnk::Topology topo;
    jfnk::DevMesh dm;
    // hot-path vectors, internal order, SoA [3][nc] unless noted
    double *u = nullptr, *Ru = nullptr, *w = nullptr, *R = nullptr, *z = nullptr, *x = nullptr;
    double *bvec = nullptr, *wk = nullptr, *tmp = nullptr, *ext = nullptr;
    double *G = nullptr, *T = nullptr;  // [9][nc]
    double* F = nullptr;                 // [3][nflux] face fluxes, owner-sorted
    double* Fn = nullptr;                // [3][ni] the same fluxes, neighbour-sorted
    double* partials = nullptr;          // reduction partials
    double *Zaug = nullptr, *AZaug = nullptr;  // loose GMRES: kept corrections z_l and J z_l, [aug][3][nc]
    double *rprev = nullptr, *dcorr = nullptr;  // residual at the start and correction of the last cycle
    double* V = nullptr;                 // Krylov basis (double or float storage)
    size_t V_ld = 0;                     // stride between basis vectors (elements)
    int V_is_float = 0;
    // problems (P >= 1) in one concatenated index space
    int nprob = 1;
    std::vector<int32_t> prob_c0, prob_c1;   // internal cell range of each problem
    int n_chunks = 0;
    int64_t* ch_beg = nullptr;           // device chunk table
    int32_t *ch_len = nullptr, *ch_prob = nullptr;
    int32_t *pch_beg = nullptr, *pch_cnt = nullptr;  // per problem: first chunk, chunk count
    int32_t* cell_prob = nullptr;        // [nc] problem of each internal cell
    jfnk::ProbDev* pd = nullptr;         // device per-problem scalars [nprob]
    jfnk::ProbDev* ph = nullptr;         // pinned host mirror (header fields only are refreshed)
    jfnk::GlobalDev* gdev = nullptr;     // device global scalars
    jfnk::GlobalDev* gh = nullptr;       // pinned, mapped host mirror
    jfnk::GlobalDev* gh_dev = nullptr;   // device address of the mirror (kernels store to it)
    int pdl = 0;                         // launch hot-path kernels with programmatic serialisation
    int skip_done = 1;                   // batches: problems out of the Arnoldi iteration skip its passes
    size_t ph_count = 0;                 // problems the pinned mirror can hold
    cudaGraphExec_t it_graph = nullptr;  // one captured Arnoldi iteration (replayed for every j)
    cudaEvent_t it_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int use_graphs = 1;
    int64_t graph_kernels = 0;           // kernels in the captured iteration
    double* scal_h = nullptr;            // pinned [16]
    // multigrid (precond.cu owns the hierarchy object)
    void* mgs = nullptr;
    // compacted launches of a batch (rowmap.cu owns the object): runs of rows per problem of
    // every index space, and the runs of the problems taking part in the current pass
    void* rmaps = nullptr;
    int mg_coarse_n = 0;
    bool mg_ready = false;
    int64_t launches = 0;
    int64_t dev_bytes = 0;
    std::vector<void*> allocs;
    jfnk::Profiler prof;
    jfnk::Tuning tune;
    // segregated solver (segregated.cu): chunk -> slot (3 p + component), per-slot chunk ranges
    int32_t *seg_slot = nullptr, *seg_sbeg = nullptr, *seg_scnt = nullptr;
    jfnk::SegSlot* seg_state = nullptr;
    std::vector<jfnk::SegSlot> seg_state_h;
    cudaGraphExec_t seg_graph = nullptr;
    int64_t seg_graph_kernels = 0;
    // dynamics (dynamics.cu): BDF2 history [3][nc] each, rho c of the current step, 9 rho/(4 dt^2)
    bool dyn_on = false;
    double dyn_mk = 0.0;
    double *dyn_ut = nullptr, *dyn_utm1 = nullptr, *dyn_vt = nullptr, *dyn_vtm1 = nullptr, *dyn_at = nullptr;
    double* dyn_rc = nullptr;
};

// ------------------------------------------------------------------ helpers (capi.cu)
// jfnk_solve (method 0: Newton-Krylov) and jfnk_solve_segregated (method 1)
int jfnk_solve_method(jfnk_ctx* c, double* u, int mem, int n_load_steps, jfnk_stats* stats, void* stream, int method);
int jfnk_fail(jfnk_ctx* c, int code, const std::string& msg);
int jfnk_cuda_fail(jfnk_ctx* c, cudaError_t e, const char* what);
// Device memory and host transfers of set-up and inspection calls.  Every one is ordered on
// the stream of the call in progress (the context's own during set-up): the synchronous
// cudaMemcpy / cudaMemset run on the legacy stream, which the context's non-blocking streams
// do not wait for, and a pageable host-to-device cudaMemcpy may return before its data lands.
void* jfnk_dalloc(jfnk_ctx* c, size_t bytes);   // tracked cudaMalloc, zeroed in stream order; nullptr on failure
int jfnk_upload(jfnk_ctx* c, void* dst, const void* src, size_t bytes);    // host (pageable) -> device
int jfnk_download(jfnk_ctx* c, void* dst, const void* src, size_t bytes);  // device -> host; returns when landed
// Makes s (NULL: the context's own stream) the stream of the call in progress; when it differs
// from the previous call's, the previous call's work is ordered before it on the device.
int jfnk_use_stream(jfnk_ctx* c, cudaStream_t s);

#define JF_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return jfnk_cuda_fail(ctx, e_, #call); \
    } while (0)

// Launches kernel k on the call's stream.  With ctx->pdl set, the launch carries the
// programmatic-stream-serialisation attribute: its blocks may be scheduled while the previous
// kernel drains, and the kernel itself (JF_PDL_ENTRY) waits for that kernel's results before
// reading anything.  Inside a captured graph this becomes a programmatic edge.
template <typename... KArgs, typename... Args>
inline cudaError_t jfnk_launch(jfnk_ctx* c, void (*k)(KArgs...), dim3 grid, dim3 block, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c->cur;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = c->pdl ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

#define JF_LAUNCHED(ctx)                                           \
    do {                                                           \
        (ctx)->launches++;                                         \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return jfnk_cuda_fail(ctx, e_, "kernel launch"); \
    } while (0)

// profiling brackets around a launch
void jfnk_prof_begin(jfnk_ctx* c, int slot);
void jfnk_prof_end(jfnk_ctx* c, int slot);

// ------------------------------------------------------------------ module entry points
namespace jfnk {
// geometry.cu: device set-up (geometry, least-squares vectors, coefficients, J~)
int setup_device_mesh(jfnk_ctx* c);
int setup_material_coefficients(jfnk_ctx* c);
// residual.cu
enum ResidualOut { OUT_R = 0, OUT_JV = 1 };
// R(u_int) into `out` (internal order); mode OUT_JV writes (R - Ru) / eps_p with each
// problem's eps_p (and 1 / eps_p) from its ProbDev.
// skip (batches): SKIP_NONE evaluates every row; SKIP_CYCLE (inside the Arnoldi iteration)
// leaves out the rows of problems whose cycle is done or that are not active; SKIP_INACTIVE
// (restarts, cycle ends, line-search trials) those of problems that are not active.  Rows
// left out keep their old contents.
enum SkipMode { SKIP_NONE = 0, SKIP_CYCLE = 1, SKIP_INACTIVE = 2 };
int residual(jfnk_ctx* c, const double* u_int, double* out, int mode, int skip = SKIP_NONE);
int residual_gated(jfnk_ctx* c, const double* u_int, double* out, int mode, const int* gate, int skip = SKIP_NONE);
int sync_load(jfnk_ctx* c);
// load_dev: device address of the load factor the kernels read (nullptr = the context's own,
// kept equal to c->load by sync_load)
int residual_bufs(jfnk_ctx* c, const double* u_int, double* out, int mode, const int* gate, double* G, double* T,
                  double* F, double* Fn, const double* load_dev = nullptr, int skip = SKIP_NONE);
// linalg.cu
// least-squares gradient alone of u_int into Gout [9][nc] (no stress, no gating)
int gradient_only(jfnk_ctx* c, const double* u_int, double* Gout);
// geometry.cu: face and cell geometry, least-squares vectors, face coefficients, the constant
// load part and the approximate Jacobian's diagonal recomputed from the device points (the
// updated-Lagrangian configuration), on the call's stream; JFNK_EINVAL for an inverted cell
int update_geometry(jfnk_ctx* c);
// updated_lagrangian.cu
int ul_setup(jfnk_ctx* c);    // allocations, point -> cell lists, reference state
int ul_reset(jfnk_ctx* c);    // back to the reference configuration
int ul_advance(jfnk_ctx* c);  // the end of a converged load step at displacement c->u
int perm_in(jfnk_ctx* c, const double* ext_aos, double* int_soa);
int build_chunks(jfnk_ctx* c);
int perm_out(jfnk_ctx* c, const double* int_soa, double* ext_aos);
int axpby(jfnk_ctx* c, size_t n, double a, const double* x, double b, const double* y, double* out);
int axpy_dev_scalar(jfnk_ctx* c, size_t n, const double* x, const double* a_dev, const double* y, double* out); // out = y + a x
// per-problem norms: mode 0 -> pd[p].nrm, 1 -> pd[p].eps (Jv step), 2 -> pd[p].unorm,
// 3 -> pd[p].beta and inv; gated = skip problems that are inactive or whose cycle is done
int pnorm(jfnk_ctx* c, const double* x, int mode, bool gated);
int perturb(jfnk_ctx* c, const double* u, const double* z, double* w, bool gated);
int perturb_basis(jfnk_ctx* c, const double* u, double* w);  // w = u + eps V_jg (gated)
int cycle_init(jfnk_ctx* c, const double* r);
int arnoldi_orthogonalise(jfnk_ctx* c, double* w);
int cycle_solution(jfnk_ctx* c, double* out, int ncols);  // out = sum_{i < min(k_p, ncols)} y_i V_i
// loose GMRES (linalg.cu): kept correction l (0 = newest) of `na`, slots in a ring
int aug_store(jfnk_ctx* c, int slot, const double* r);     // slot <- dcorr / |dcorr_p|, (rprev - r) / |dcorr_p|
int aug_load(jfnk_ctx* c, int slot, double* w);            // w <- J z of slot (gated on `all done`)
// x += d for the active problems only
int add_active(jfnk_ctx* c, const double* d, double* x);
int aug_add(jfnk_ctx* c, const int* slots, int na, int ncols, const double* z, double* out);
int line_trial(jfnk_ctx* c, const double* u, const double* x, double* w);       // w = u + s_p x (active)
int accept_masked(jfnk_ctx* c, const int32_t* mask_dev, double* u, const double* w, double* Ru, const double* R);
// precond.cu
int pc_setup(jfnk_ctx* c);
int autotune(jfnk_ctx* c);               // launch shapes for this mesh (autotune.cu)
int segregated(jfnk_ctx* c, int n_load_steps, jfnk_stats* st);  // Sec. 3.1 (segregated.cu)
int dynamics_setup(jfnk_ctx* c);       // history buffers at rest (dynamics.cu)
int solve_dynamic(jfnk_ctx* c, int n_steps, int32_t probe_cell, double* probe, jfnk_stats* st, int method);
bool tuning_valid(const Tuning& t);
// z = P^-1 v (v, z internal SoA double); pc = JFNK_PC_*
int pc_apply(jfnk_ctx* c, int pc, const double* v, double* z);
int pc_apply_any(jfnk_ctx* c, int pc, const void* v, int v_is_float, double* z, const int* gate, int skip = SKIP_NONE);
// eps_formed (optional): asks the multigrid's last sweep to form the following Jv's eps for a
// single problem; set to whether it did (else the caller runs the norm pass)
int pc_apply_dev(jfnk_ctx* c, int pc, const void* vbase, size_t ld, const int* jidx, int v_is_float, double* z,
                 const int* gate, bool* eps_formed = nullptr, int skip = SKIP_NONE);
void mg_release(jfnk_ctx* c);
int mg_hierarchy_info(jfnk_ctx* c, std::vector<int64_t>& rows, std::vector<int64_t>& nnz_a, std::vector<int64_t>& nnz_p);
// rowmap.cu: index spaces of compacted launches (batches with skipping): cells (also the
// finest multigrid level), faces (the residual's flux faces), and multigrid level l >= 1
enum MapSpace { SPACE_CELLS = 0, SPACE_FACES = 1 };
inline int space_of_level(int l) { return l == 0 ? SPACE_CELLS : 1 + l; }
// runs of rows per problem of every space (after the multigrid set-up; nothing for one problem)
int rowmap_setup(jfnk_ctx* c);
void rowmap_release(jfnk_ctx* c);
// compacts the runs of the problems taking part in passes of skip mode `skip` (SKIP_CYCLE or
// SKIP_INACTIVE) on the call's stream; a no-op when the context has no compacted spaces
int rowmap_build(jfnk_ctx* c, int skip);
#ifdef __CUDACC__
// the rows a pass of mode `skip` visits in `space` of n rows (identity unless compacted)
RowMap rowmap(const jfnk_ctx* c, int space, int skip, int n);
// blocks of a grid-stride launch of kernel fn (bs threads, `per_block` units of work each)
// over units_all units: every unit once for identity maps, else at most `waves` times the
// blocks the SMs hold at once (the FP64-bound residual passes measured fastest with 4 waves,
// the latency-bound V-cycle and cell sums with 1)
int rowmap_blocks(jfnk_ctx* c, const void* fn, int bs, long units_all, long per_block, const RowMap& rm, int waves = 1);
#endif
// precond.cu: the problem of every row of multigrid levels >= 1 (host, batches)
const std::vector<std::vector<int32_t>>* mg_level_problems(jfnk_ctx* c);
// solver.cu
int gmres(jfnk_ctx* c, const double* b, double* x, int* its, double* relres, int* status);
int newton(jfnk_ctx* c, int n_load_steps, jfnk_stats* st);
}  // namespace jfnk
