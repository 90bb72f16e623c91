// Compacted launches for batches (the union index space of many problems).  Inside the Arnoldi
// iteration the problems whose Krylov cycle is done, and around it the problems that left the
// Newton iteration, sit the residual passes and the V-cycle out.  Rather than launching every
// row and testing each row's problem, every index space (cells, flux faces, the rows of each
// multigrid level) is cut at set-up into runs of consecutive rows of one problem; before a
// pass one block per space compacts the runs of the problems taking part into a prefix table
// (RowMap), and the pass's kernels walk those rows with a grid stride on a grid of the
// blocks the SMs hold at once.  The rows a pass evaluates, and the arithmetic of each, are the
// same as with per-row skipping, so results are bitwise equal; the rows left out cost nothing.
#include <algorithm>
#include <map>
#include <mutex>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace jfnk {

// device table of one space
struct SpaceDev {
    const int32_t *run_first, *run_len, *run_prob;  // runs of rows of one problem, in row order
    int32_t* pre[2];    // per mode (0: SKIP_CYCLE, 1: SKIP_INACTIVE): [nrun + 1] rows before each run taking part
    int32_t* first[2];  // [nrun] first row of each run taking part
    int32_t* hdr[2];    // {runs taking part, rows taking part}
    int nrun;
    int pad;
};

struct RowMaps {
    struct Space {
        int n = 0;       // rows
        bool on = false; // compacted (else identity)
        SpaceDev d{};
    };
    std::vector<Space> sp;
    SpaceDev* dev = nullptr;
    int n_sm = 0;
};

static RowMaps* maps(const jfnk_ctx* c) { return (RowMaps*)c->rmaps; }

// runs of equal problem over rows [0, n) with problem prob(i)
template <typename F>
static void make_runs(int n, F&& prob, std::vector<int32_t>& first, std::vector<int32_t>& len, std::vector<int32_t>& pr)
{
    first.clear();
    len.clear();
    pr.clear();
    for (int i = 0; i < n; i++) {
        const int p = prob(i);
        if (!pr.empty() && pr.back() == p && first.back() + len.back() == i) {
            len.back()++;
        } else {
            first.push_back(i);
            len.push_back(1);
            pr.push_back(p);
        }
    }
}

// One block per space: the runs whose problem takes part (active, and for mode 0 with its
// cycle still running), in row order, with the prefix of their row counts.  Each thread takes
// a consecutive share of the runs: it counts its runs and rows taking part (independent loads),
// the block scans the counts, and the thread writes its runs at their places.
constexpr int kMapThreads = 256;

__global__ void __launch_bounds__(kMapThreads) k_rowmap_build(const SpaceDev* __restrict__ sp, const ProbDev* __restrict__ pd,
                                                              int mode)
{
    JF_PDL_ENTRY();
    const SpaceDev S = sp[blockIdx.x];
    if (!S.pre[mode]) return;  // identity space
    const int n = S.nrun, per = (n + kMapThreads - 1) / kMapThreads;
    const int j0 = min(n, (int)threadIdx.x * per), j1 = min(n, j0 + per);
    auto takes = [&](int j) {
        const ProbDev& P = pd[S.run_prob[j]];
        return P.active && !(mode == 0 && P.done);
    };
    int cnt = 0, rows = 0;
#pragma unroll 4
    for (int j = j0; j < j1; j++)
        if (takes(j)) { cnt++; rows += S.run_len[j]; }
    // exclusive block scan of (cnt, rows)
    __shared__ int wc[kMapThreads / 32], wr[kMapThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int ic = cnt, ir = rows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, ic, o), b = __shfl_up_sync(0xffffffffu, ir, o);
        if (lane >= o) { ic += a; ir += b; }
    }
    if (lane == 31) { wc[wid] = ic; wr[wid] = ir; }
    __syncthreads();
    int bc = 0, br = 0;
    for (int w = 0; w < wid; w++) { bc += wc[w]; br += wr[w]; }
    int k = bc + ic - cnt, r = br + ir - rows;
    for (int j = j0; j < j1; j++)
        if (takes(j)) {
            S.first[mode][k] = S.run_first[j];
            S.pre[mode][k] = r;
            k++;
            r += S.run_len[j];
        }
    if (threadIdx.x == kMapThreads - 1) {  // the last thread ends at the totals
        S.pre[mode][k] = r;
        S.hdr[mode][0] = k;
        S.hdr[mode][1] = r;
    }
}

void rowmap_release(jfnk_ctx* c)
{
    delete maps(c);
    c->rmaps = nullptr;
}

int rowmap_setup(jfnk_ctx* c)
{
    rowmap_release(c);
    if (c->nprob <= 1 || !c->skip_done) return JFNK_OK;
    const int nc = c->dm.nc, P = c->nprob;
    std::vector<int32_t> cell_prob(nc, 0);
    for (int p = 0; p < P; p++)
        for (int i = c->prob_c0[p]; i < c->prob_c1[p]; i++) cell_prob[i] = p;
    auto* R = new RowMaps();
    c->rmaps = R;
    cudaDeviceGetAttribute(&R->n_sm, cudaDevAttrMultiProcessorCount, c->opt.device);
    R->n_sm = std::max(1, R->n_sm);
    const auto* lp = mg_level_problems(c);
    const int nsp = 2 + (lp ? (int)lp->size() : 0);
    R->sp.resize(nsp);
    std::vector<int32_t> first, len, pr;
    for (int s = 0; s < nsp; s++) {
        auto& S = R->sp[s];
        if (s == SPACE_CELLS) {
            S.n = nc;
            make_runs(nc, [&](int i) { return cell_prob[i]; }, first, len, pr);
        } else if (s == SPACE_FACES) {
            S.n = c->dm.nflux;
            const auto& own = c->topo.own;
            make_runs(S.n, [&](int f) { return cell_prob[own[f]]; }, first, len, pr);
        } else {
            const auto& v = (*lp)[s - 2];
            S.n = (int)v.size();
            make_runs(S.n, [&](int i) { return v[i]; }, first, len, pr);
        }
        // problems hold contiguous rows on every level but for stray aggregates: a space cut
        // into many more runs than problems stays on per-row work (identity map)
        const int nrun = (int)first.size();
        S.on = nrun > 0 && nrun <= 8 * P + 64;
        S.d.nrun = S.on ? nrun : 0;
        if (!S.on) continue;
        int32_t* buf = (int32_t*)jfnk_dalloc(c, sizeof(int32_t) * (3 * (size_t)nrun + 2 * (2 * (size_t)nrun + 1) + 4));
        if (!buf) return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the row maps failed");
        std::vector<int32_t> h;
        h.insert(h.end(), first.begin(), first.end());
        h.insert(h.end(), len.begin(), len.end());
        h.insert(h.end(), pr.begin(), pr.end());
        int rc = jfnk_upload(c, buf, h.data(), sizeof(int32_t) * h.size());
        if (rc) return rc;
        S.d.run_first = buf;
        S.d.run_len = buf + nrun;
        S.d.run_prob = buf + 2 * (size_t)nrun;
        int32_t* q = buf + 3 * (size_t)nrun;
        for (int m = 0; m < 2; m++) {
            S.d.pre[m] = q; q += nrun + 1;
            S.d.first[m] = q; q += nrun;
        }
        S.d.hdr[0] = q; S.d.hdr[1] = q + 2;
    }
    std::vector<SpaceDev> tab(nsp);
    for (int s = 0; s < nsp; s++) tab[s] = R->sp[s].d;
    R->dev = (SpaceDev*)jfnk_dalloc(c, sizeof(SpaceDev) * nsp);
    if (!R->dev) return jfnk_fail(c, JFNK_ENOMEM, "device allocation of the row maps failed");
    int rc = jfnk_upload(c, R->dev, tab.data(), sizeof(SpaceDev) * nsp);
    if (rc) return rc;
    if (getenv("JFNK_VERBOSE")) {
        for (int s = 0; s < nsp; s++)
            fprintf(stderr, "[jfnk] row map space %d: %d rows, %d runs%s\n", s, R->sp[s].n, R->sp[s].d.nrun,
                    R->sp[s].on ? "" : " (identity)");
    }
    return JFNK_OK;
}

int rowmap_build(jfnk_ctx* c, int skip)
{
    const RowMaps* R = maps(c);
    if (!R || (skip != SKIP_CYCLE && skip != SKIP_INACTIVE)) return JFNK_OK;
    const int nsp = (int)R->sp.size();
    jfnk_launch(c, k_rowmap_build, dim3(nsp), dim3(kMapThreads), (const SpaceDev*)R->dev, (const ProbDev*)c->pd,
                skip == SKIP_CYCLE ? 0 : 1);
    JF_LAUNCHED(c);
    return JFNK_OK;
}

RowMap rowmap(const jfnk_ctx* c, int space, int skip, int n)
{
    RowMap m;
    m.n = n;
    const RowMaps* R = maps(c);
    if (!R || (skip != SKIP_CYCLE && skip != SKIP_INACTIVE) || space < 0 || space >= (int)R->sp.size()) return m;
    const auto& S = R->sp[space];
    if (!S.on || S.n != n) return m;
    const int md = skip == SKIP_CYCLE ? 0 : 1;
    m.pre = S.d.pre[md];
    m.first = S.d.first[md];
    m.hdr = S.d.hdr[md];
    return m;
}

int rowmap_blocks(jfnk_ctx* c, const void* fn, int bs, long units_all, long per_block, const RowMap& rm, int waves)
{
    const long all = std::max<long>(1, (units_all + per_block - 1) / per_block);
    const RowMaps* R = maps(c);
    if (!rm.pre || !R) return (int)all;
    // blocks resident at once, per kernel and block size (the same on every device of a pool)
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> occ;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = occ.find({fn, bs});
        if (it != occ.end()) per_sm = it->second;
    }
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bs, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = std::max(1, 2048 / bs);
        }
        std::lock_guard<std::mutex> g(mu);
        occ[{fn, bs}] = per_sm;
    }
    return (int)std::min<long>(all, (long)per_sm * R->n_sm * std::max(1, waves));
}

}  // namespace jfnk
