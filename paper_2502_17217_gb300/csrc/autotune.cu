// Launch-shape autotuner of the hot-path kernels.
//
// At set-up (options.autotune = 1) the context times, on its own mesh and device, each
// candidate launch shape of the kernels whose best shape depends on the mesh and the GPU:
//   cells per block of the gradient pass            {64, 128, 256}
//   faces per block of the face pass, with or
//     without shared-memory staging of the owner
//     cells' gradients                              {128, 256} x {direct, staged}
//   cells per block of the cell-sum pass            {128, 256, 512}
//   rows per block of the fine-level multigrid
//     kernels (multigrid preconditioner only)       {128, 256, 512}
// one parameter at a time (coordinate descent from the defaults), each candidate timed with
// CUDA events over a few residual evaluations (V-cycles) after a warm-up, and keeps the
// fastest.  The arithmetic of every kernel is the same for every shape (one thread per cell
// or face, fixed summation order), so the choice changes timing only, never results.
// A batch's passes run over compacted row maps on persistent grids, so a batch is timed that
// way, with every problem taking part (the problems' flags are put back afterwards).
// Choices are cached per (device, mesh sizes, law mix, preconditioner, precision) so that
// contexts set up for the same mesh shape (a serving loop) do not tune again.  Meshes below
// kTuneMinCells keep the defaults: their kernels are launch-bound and the timings noise.
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "jfnk_internal.h"

namespace jfnk {

namespace {

constexpr int kTuneMinCells = 4096;
constexpr int kWarm = 2, kReps = 3, kEvals = 4;

using Key = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_cache_mutex;
std::map<Key, Tuning> g_cache;

Key key_of(const jfnk_ctx* c)
{
    return Key(c->opt.device, c->dm.nc, c->dm.ni, c->dm.nflux, c->law_mode, c->opt.pc, c->opt.precision);
}

// best (minimum over repetitions) mean time of `evals` calls of f, in ms; < 0 on error
template <typename F>
float time_it(jfnk_ctx* c, F f)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float best = -1.f;
    for (int w = 0; w < kWarm; w++)
        if (f()) best = -2.f;
    for (int r = 0; r < kReps && best > -2.f; r++) {
        cudaEventRecord(a, c->cur);
        for (int e = 0; e < kEvals; e++)
            if (f()) best = -2.f;
        cudaEventRecord(b, c->cur);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            best = -2.f;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= kEvals;
        if (best < 0.f || ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace

bool tuning_valid(const Tuning& t)
{
    const bool g = t.grad_bs == 64 || t.grad_bs == 128 || t.grad_bs == 256;
    const bool f = (t.flux_bs == 128 || t.flux_bs == 256) && (t.flux_stage == 0 || t.flux_stage == 1);
    const bool s = t.finish_bs == 128 || t.finish_bs == 256 || t.finish_bs == 512;
    const bool m = t.mg_bs == 128 || t.mg_bs == 256 || t.mg_bs == 512;
    return g && f && s && m;
}

int autotune(jfnk_ctx* c)
{
    c->tune = Tuning();
    if (!c->opt.autotune || c->dm.nc < kTuneMinCells) return JFNK_OK;
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        auto it = g_cache.find(key_of(c));
        if (it != g_cache.end()) {
            c->tune = it->second;
            return JFNK_OK;
        }
    }
    const bool prof = c->prof.enabled;
    c->prof.enabled = false;
    c->cur = c->stream;
    const int64_t launches = c->launches;
    // a batch: every problem takes part in the timed passes (flags `active` and `done` of each
    // problem, zero at set-up, set here and put back at the end)
    const bool mapped = c->rmaps != nullptr && c->ph != nullptr;
    auto set_flags = [&](int active) -> int {
        for (int p = 0; p < c->nprob; p++) {
            c->ph[p].active = active;
            c->ph[p].done = 0;
        }
        for (size_t off : {offsetof(ProbDev, active), offsetof(ProbDev, done)})
            JF_CUDA(c, cudaMemcpy2DAsync((char*)c->pd + off, sizeof(ProbDev), (const char*)c->ph + off, sizeof(ProbDev),
                                         sizeof(int), c->nprob, cudaMemcpyHostToDevice, c->cur));
        JF_CUDA(c, cudaStreamSynchronize(c->cur));
        return JFNK_OK;
    };
    const int skip = mapped ? SKIP_INACTIVE : SKIP_NONE;
    auto res = [&]() { return residual_bufs(c, c->u, c->R, OUT_R, nullptr, c->G, c->T, c->F, c->Fn, nullptr, skip); };
    Tuning& t = c->tune;
    int rc = sync_load(c);
    if (!rc && mapped) rc = set_flags(1);
    // coordinate descent: each parameter over its candidates, the others held
    auto pick = [&](int* field, const int* cand, int n) {
        const int keep = *field;
        float best = -1.f;
        int arg = keep;
        for (int i = 0; i < n && !rc; i++) {
            *field = cand[i];
            const float ms = time_it(c, res);
            if (ms < -1.5f) { rc = jfnk_cuda_fail(c, cudaGetLastError(), "autotune"); break; }
            if (ms >= 0.f && (best < 0.f || ms < best)) { best = ms; arg = cand[i]; }
        }
        *field = rc ? keep : arg;
    };
    const int g_c[] = {64, 128, 256};
    const int s_c[] = {128, 256, 512};
    pick(&t.grad_bs, g_c, 3);
    if (!rc && c->dm.nflux > 0) {
        // the face pass: block size x staging, jointly
        const int fb[] = {128, 256};
        float best = -1.f;
        int bb = t.flux_bs, bs = t.flux_stage;
        for (int i = 0; i < 2 && !rc; i++)
            for (int st = 0; st < 2 && !rc; st++) {
                t.flux_bs = fb[i];
                t.flux_stage = st;
                const float ms = time_it(c, res);
                if (ms < -1.5f) { rc = jfnk_cuda_fail(c, cudaGetLastError(), "autotune"); break; }
                if (ms >= 0.f && (best < 0.f || ms < best)) { best = ms; bb = fb[i]; bs = st; }
            }
        t.flux_bs = bb;
        t.flux_stage = bs;
    }
    if (!rc) pick(&t.finish_bs, s_c, 3);
    if (!rc && c->opt.pc == JFNK_PC_MG && c->mg_ready) {
        const int m_c[] = {128, 256, 512};
        const int keep = t.mg_bs;
        float best = -1.f;
        int arg = keep;
        for (int i = 0; i < 3 && !rc; i++) {
            t.mg_bs = m_c[i];
            const float ms = time_it(c, [&]() { return pc_apply_any(c, JFNK_PC_MG, c->R, 0, c->z, nullptr, skip); });
            if (ms < -1.5f) { rc = jfnk_cuda_fail(c, cudaGetLastError(), "autotune"); break; }
            if (ms >= 0.f && (best < 0.f || ms < best)) { best = ms; arg = m_c[i]; }
        }
        t.mg_bs = rc ? keep : arg;
    }
    if (mapped) {
        const int rc2 = set_flags(0);
        if (!rc) rc = rc2;
    }
    c->prof.enabled = prof;
    c->launches = launches;  // tuning launches are not the caller's work
    if (rc) {
        c->tune = Tuning();
        return rc;
    }
    t.tuned = 1;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    g_cache[key_of(c)] = t;
    return JFNK_OK;
}

}  // namespace jfnk

extern "C" int jfnk_get_tuning(jfnk_ctx* c, int32_t* out, int n)
{
    if (!c || !out || n < 6) return JFNK_EINVAL;
    if (c->dirty) {
        const int rc = jfnk_setup(c);
        if (rc) return rc;
    }
    const jfnk::Tuning& t = c->tune;
    const int32_t v[6] = {t.grad_bs, t.flux_bs, t.flux_stage, t.finish_bs, t.mg_bs, t.tuned};
    std::memcpy(out, v, sizeof v);
    return JFNK_OK;
}

extern "C" int jfnk_set_tuning(jfnk_ctx* c, const int32_t* in, int n)
{
    if (!c || !in || n < 5) return JFNK_EINVAL;
    if (c->dirty) {
        const int rc = jfnk_setup(c);
        if (rc) return rc;
    }
    jfnk::Tuning t;
    t.grad_bs = in[0];
    t.flux_bs = in[1];
    t.flux_stage = in[2];
    t.finish_bs = in[3];
    t.mg_bs = in[4];
    t.tuned = 0;
    if (!jfnk::tuning_valid(t))
        return jfnk_fail(c, JFNK_EINVAL,
                         "jfnk_set_tuning: grad {64,128,256}, flux {128,256}, stage {0,1}, finish {128,256,512}, "
                         "multigrid {128,256,512}");
    c->tune = t;
    if (c->it_graph) {  // the captured iteration holds the old launch shapes
        cudaGraphExecDestroy(c->it_graph);
        c->it_graph = nullptr;
    }
    return JFNK_OK;
}
