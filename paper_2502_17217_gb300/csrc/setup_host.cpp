// Host-side set-up of the mesh topology: validation, reverse Cuthill-McKee cell numbering,
// face reordering (owner-sorted internal faces with owner < neighbour, boundary faces grouped
// by condition), the cell-to-face lists and the sliced-ELL neighbour table of the gradient
// kernel; plus the aggregation multigrid hierarchy on -J~.  Runs once per mesh (off the hot
// path); everything it builds is uploaded and used by the kernels.
#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <thread>

#include "jfnk_internal.h"

namespace jfnk {

// Host threads of the set-up's parallel loops: the host's cores, at most 16.
static int host_threads()
{
    return std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
}

// Runs f(lo, hi, tid) over [0, n) in blocks of `grain` taken by up to host_threads() threads
// (tid in [0, host_threads()); blocks are handed out in order through an atomic counter, so
// uneven blocks balance).  Each block's results depend on the block alone: the outcome is the
// same for any thread count.  Scratch indexed by tid is private to the block's thread.
template <typename F>
static void parallel_blocks(int n, int grain, F&& f)
{
    const int nblocks = (n + grain - 1) / grain;
    const int nt = std::max(1, std::min(nblocks, host_threads()));
    if (nt <= 1) {
        for (int b = 0; b < nblocks; b++) f(b * grain, std::min(n, (b + 1) * grain), 0);
        return;
    }
    std::atomic<int> next(0);
    auto work = [&](int tid) {
        for (int b = next++; b < nblocks; b = next++) f(b * grain, std::min(n, (b + 1) * grain), tid);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto& t : th) t.join();
}

// Sparse accumulator of one host thread over nco columns: entries stamped with the row being
// formed, so it is cleared once per use, not once per row or block.
struct SparseAcc {
    std::vector<double> acc;
    std::vector<int32_t> mark;
    std::vector<int32_t> list;
    void init(int nco)
    {
        if ((int)acc.size() != nco) {
            acc.assign(nco, 0.0);
            mark.assign(nco, -1);
        }
    }
};

static std::vector<int32_t> rcm_order(int nc, const std::vector<int32_t>& aptr, const std::vector<int32_t>& adj)
{
    // Reverse Cuthill-McKee (Cuthill & McKee 1969; George 1971): breadth-first search from a
    // minimum-degree cell of each component, visiting neighbours by increasing degree (then
    // index), and the final order reversed.  Adjacency in CSR form (aptr, adj).
    std::vector<int32_t> deg(nc);
    for (int i = 0; i < nc; i++) deg[i] = aptr[i + 1] - aptr[i];
    std::vector<int32_t> cand(nc);
    std::iota(cand.begin(), cand.end(), 0);
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return deg[a] < deg[b]; });
    std::vector<char> seen(nc, 0);
    std::vector<int32_t> order;
    order.reserve(nc);
    std::vector<int32_t> nb;
    for (int s : cand) {
        if (seen[s]) continue;
        size_t head = order.size();
        order.push_back(s);
        seen[s] = 1;
        while (head < order.size()) {
            int v = order[head++];
            nb.clear();
            for (int q = aptr[v]; q < aptr[v + 1]; q++)
                if (!seen[adj[q]]) nb.push_back(adj[q]);
            std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
            for (int w : nb) {
                seen[w] = 1;
                order.push_back(w);
            }
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// phase times of the set-up, printed to stderr when JFNK_VERBOSE is set
struct PhaseClock {
    bool on = getenv("JFNK_VERBOSE") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void lap(const char* what)
    {
        if (!on) return;
        const auto n = std::chrono::steady_clock::now();
        fprintf(stderr, "[jfnk]   topology: %-28s %8.1f ms\n", what, std::chrono::duration<double, std::milli>(n - t).count());
        t = n;
    }
};

std::string build_topology(const HostMesh& hm, bool rcm, Topology& t, const std::vector<int32_t>* group)
{
    const int nc = hm.nc, ni = hm.ni, nf = hm.nf;
    PhaseClock clk;
    t = Topology();
    t.nc = nc;
    // --- cell numbering
    if (rcm) {
        // cell adjacency in CSR form, each cell's neighbours in face order
        std::vector<int32_t> aptr(nc + 1, 0), adj(2 * (size_t)ni);
        for (int f = 0; f < ni; f++) { aptr[hm.own[f] + 1]++; aptr[hm.nei[f] + 1]++; }
        for (int i = 0; i < nc; i++) aptr[i + 1] += aptr[i];
        std::vector<int32_t> fill(aptr.begin(), aptr.end() - 1);
        for (int f = 0; f < ni; f++) {
            adj[fill[hm.own[f]]++] = hm.nei[f];
            adj[fill[hm.nei[f]]++] = hm.own[f];
        }
        t.n2o = rcm_order(nc, aptr, adj);
    } else {
        t.n2o.resize(nc);
        std::iota(t.n2o.begin(), t.n2o.end(), 0);
    }
    if (group)
        std::stable_sort(t.n2o.begin(), t.n2o.end(), [&](int a, int b) { return (*group)[a] < (*group)[b]; });
    t.o2n.assign(nc, -1);
    for (int i = 0; i < nc; i++) t.o2n[t.n2o[i]] = i;
    clk.lap("cell numbering");
    // --- face order
    struct FK { int32_t a, b, src; uint8_t flip; };
    std::vector<FK> in(ni);
    for (int f = 0; f < ni; f++) {
        int a = t.o2n[hm.own[f]], b = t.o2n[hm.nei[f]];
        uint8_t flip = 0;
        if (a > b) { std::swap(a, b); flip = 1; }
        in[f] = {a, b, f, flip};
    }
    {
        // order by (a, b, src): bucket by a (counting), then each short bucket by (b, src)
        std::vector<int32_t> cnt(nc + 1, 0);
        for (const FK& k : in) cnt[k.a + 1]++;
        for (int i = 0; i < nc; i++) cnt[i + 1] += cnt[i];
        std::vector<FK> out(ni);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (const FK& k : in) out[fill[k.a]++] = k;  // stable: src ascending within a bucket
        for (int i = 0; i < nc; i++)
            std::sort(out.begin() + cnt[i], out.begin() + cnt[i + 1],
                      [](const FK& x, const FK& y) { return x.b != y.b ? x.b < y.b : x.src < y.src; });
        in.swap(out);
    }
    std::vector<FK> bd[4];  // disp, symm, trac, empty
    for (int f = ni; f < nf; f++) {
        int bt = hm.btype[f - ni];
        int cls = bt == JFNK_BC_DISP ? 0 : (bt == JFNK_BC_SYMM ? 1 : (bt == JFNK_BC_TRAC ? 2 : 3));
        bd[cls].push_back({t.o2n[hm.own[f]], -1, f, 0});
    }
    for (auto& v : bd)
        std::sort(v.begin(), v.end(), [](const FK& x, const FK& y) { return x.a != y.a ? x.a < y.a : x.src < y.src; });
    clk.lap("face order");
    t.ni = ni;
    t.nd = (int)bd[0].size();
    t.nsy = (int)bd[1].size();
    t.nt = (int)bd[2].size();
    t.ne = (int)bd[3].size();
    t.nf = nf;
    std::vector<FK> all;
    all.reserve(nf);
    all.insert(all.end(), in.begin(), in.end());
    for (auto& v : bd) all.insert(all.end(), v.begin(), v.end());
    t.face_src.resize(nf);
    t.face_flip.resize(nf);
    t.own.resize(nf);
    t.nei.resize(ni);
    t.fptr.assign(nf + 1, 0);
    t.fpts.clear();
    t.fpts.reserve(hm.fpts.size());
    for (int f = 0; f < nf; f++) {
        const FK& k = all[f];
        t.face_src[f] = k.src;
        t.face_flip[f] = k.flip;
        t.own[f] = k.a;
        if (f < ni) t.nei[f] = k.b;
        int s0 = hm.fptr[k.src], s1 = hm.fptr[k.src + 1];
        if (!k.flip)
            for (int q = s0; q < s1; q++) t.fpts.push_back(hm.fpts[q]);
        else
            for (int q = s1 - 1; q >= s0; q--) t.fpts.push_back(hm.fpts[q]);
        t.fptr[f + 1] = (int32_t)t.fpts.size();
    }
    int bw = 0;
    for (int f = 0; f < ni; f++) bw = std::max(bw, t.nei[f] - t.own[f]);
    t.bandwidth = bw;
    clk.lap("face arrays");
    // --- per-cell ranges
    auto ranges = [&](int lo, int hi, std::vector<int32_t>& ptr) {
        ptr.assign(nc + 1, 0);
        for (int f = lo; f < hi; f++) ptr[t.own[f] + 1]++;
        for (int P = 0; P < nc; P++) ptr[P + 1] += ptr[P];
        for (int P = 0; P <= nc; P++) ptr[P] += lo;
    };
    ranges(0, ni, t.fo_ptr);
    ranges(ni, ni + t.nd, t.fd_ptr);
    ranges(ni + t.nd, ni + t.nd + t.nsy, t.fs_ptr);
    ranges(ni + t.nd + t.nsy, ni + t.nd + t.nsy + t.nt, t.ft_ptr);
    // neighbour-sorted internal faces
    t.fn_ptr.assign(nc + 1, 0);
    for (int f = 0; f < ni; f++) t.fn_ptr[t.nei[f] + 1]++;
    for (int P = 0; P < nc; P++) t.fn_ptr[P + 1] += t.fn_ptr[P];
    t.fn_face.resize(ni);
    {
        std::vector<int32_t> fill(t.fn_ptr.begin(), t.fn_ptr.end() - 1);
        for (int f = 0; f < ni; f++) t.fn_face[fill[t.nei[f]]++] = f;
    }
    // all faces of each cell (geometry): owner side f, neighbour side ~f, by face index
    t.ca_ptr.assign(nc + 1, 0);
    for (int f = 0; f < nf; f++) {
        t.ca_ptr[t.own[f] + 1]++;
        if (f < ni) t.ca_ptr[t.nei[f] + 1]++;
    }
    for (int P = 0; P < nc; P++) t.ca_ptr[P + 1] += t.ca_ptr[P];
    t.ca_face.resize(t.ca_ptr[nc]);
    {
        std::vector<int32_t> fill(t.ca_ptr.begin(), t.ca_ptr.end() - 1);
        for (int f = 0; f < nf; f++) {
            t.ca_face[fill[t.own[f]]++] = f;
            if (f < ni) t.ca_face[fill[t.nei[f]]++] = ~f;
        }
    }
    clk.lap("cell face lists");
    // sliced ELL of internal neighbours (32 cells per slice), faces in increasing index
    std::vector<int32_t> cnt(nc, 0);
    for (int f = 0; f < ni; f++) { cnt[t.own[f]]++; cnt[t.nei[f]]++; }
    for (int f = ni + t.nd; f < ni + t.nd + t.nsy; f++) cnt[t.own[f]]++;
    const int ns = (nc + 31) / 32;
    t.sell_off.resize(ns + 1);
    t.sell_w.resize(ns);
    int off = 0;
    for (int s = 0; s < ns; s++) {
        int w = 0;
        for (int l = 0; l < 32 && 32 * s + l < nc; l++) w = std::max(w, cnt[32 * s + l]);
        t.sell_off[s] = off;
        t.sell_w[s] = w;
        off += 32 * w;
    }
    t.sell_off[ns] = off;
    t.n_slots = off;
    t.sell_nbr.assign(off, -1);
    t.sell_face.assign(off, -1);
    std::vector<int32_t> k(nc, 0);
    // walk each cell's internal faces in increasing face index: merge owner and neighbour lists
    for (int P = 0; P < nc; P++) {
        int a = t.fo_ptr[P], ae = t.fo_ptr[P + 1];
        int b = t.fn_ptr[P], be = t.fn_ptr[P + 1];
        int s = P / 32, lane = P % 32;
        while (a < ae || b < be) {
            int f, N;
            if (b >= be || (a < ae && a < t.fn_face[b])) { f = a; N = t.nei[a]; a++; }
            else { f = t.fn_face[b]; N = t.own[f]; b++; }
            int slot = t.sell_off[s] + 32 * k[P] + lane;
            t.sell_nbr[slot] = N;
            t.sell_face[slot] = f;
            k[P]++;
        }
        for (int f = t.fs_ptr[P]; f < t.fs_ptr[P + 1]; f++) {  // mirror neighbours
            int slot = t.sell_off[s] + 32 * k[P] + lane;
            t.sell_nbr[slot] = nc + (f - ni - t.nd);
            t.sell_face[slot] = f;
            k[P]++;
        }
    }
    // boundary values in the new face order
    t.bval.assign((size_t)(t.nd + t.nsy + t.nt) * 3, 0.0);
    for (int f = ni; f < ni + t.nd + t.nsy + t.nt; f++)
        for (int c = 0; c < 3; c++) t.bval[(size_t)(f - ni) * 3 + c] = hm.bval[(size_t)(t.face_src[f] - ni) * 3 + c];
    clk.lap("neighbour table, values");
    return "";
}

// ------------------------------------------------------------------ aggregation multigrid
// Aggregation AMG on A = -J~, rows visited in the input cell order:
//   strong(i, j):  -a_ij >= theta * max_k(-a_ik), values within a relative 1e-10 counting as
//                  equal so that rounding does not decide ties;
//   pass 1:        a free row whose strong neighbours are all free starts an aggregate;
//   pass 2:        a remaining row joins the aggregate of its strongest aggregated neighbour
//                  (lowest index among equals), else forms a singleton;
//   P:             piecewise constant, or smoothed P = (I - omega D^-1 A) P_tent with
//                  omega = 4 / (3 rho), rho = max_i sum_j |a_ij| / a_ii (Gershgorin);
//   A_c = P^T A P, until coarse_max rows, max_levels, or < 10% shrink.
static int aggregate(const MgLevelHost& L, double theta, std::vector<int32_t>& agg)
{
    const double tie = 1e-10;
    const int n = L.n;
    agg.assign(n, -1);
    std::vector<char> strong(L.col.size(), 0);
    for (int i = 0; i < n; i++) {
        double mx = 0;
        for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
            if (L.col[q] != i) mx = std::max(mx, -L.val[q]);
        for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
            strong[q] = (L.col[q] != i && mx > 0 && -L.val[q] >= theta * mx * (1.0 - tie));
    }
    int na = 0;
    for (int i = 0; i < n; i++) {
        if (agg[i] >= 0) continue;
        bool ok = true;
        int ns = 0;
        for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
            if (strong[q]) {
                ns++;
                if (agg[L.col[q]] >= 0) ok = false;
            }
        if (!ok || ns == 0) continue;
        agg[i] = na;
        for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
            if (strong[q]) agg[L.col[q]] = na;
        na++;
    }
    for (int i = 0; i < n; i++) {
        if (agg[i] >= 0) continue;
        double mx = 0;
        for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
            if (L.col[q] != i && agg[L.col[q]] >= 0) mx = std::max(mx, -L.val[q]);
        int best = -1;
        if (mx > 0)
            for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
                if (L.col[q] != i && agg[L.col[q]] >= 0 && -L.val[q] >= mx * (1.0 - tie)) { best = L.col[q]; break; }
        agg[i] = best >= 0 ? agg[best] : na++;
    }
    return na;
}

static void smoothed_prolongation(const MgLevelHost& F, const std::vector<int32_t>& agg, int nco, bool smoothed,
                                  std::vector<int32_t>& prp, std::vector<int32_t>& pcol, std::vector<double>& pval)
{
    const int n = F.n;
    prp.assign(n + 1, 0);
    pcol.clear();
    pval.clear();
    if (!smoothed) {
        for (int i = 0; i < n; i++) { pcol.push_back(agg[i]); pval.push_back(1.0); prp[i + 1] = i + 1; }
        return;
    }
    double rho = 0.0;
    std::vector<double> diag(n, 0.0);
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int q = F.rp[i]; q < F.rp[i + 1]; q++) {
            s += std::fabs(F.val[q]);
            if (F.col[q] == i) diag[i] = F.val[q];
        }
        rho = std::max(rho, s / diag[i]);
    }
    const double omega = 4.0 / (3.0 * rho);
    // rows in blocks, each block into its own arrays, then concatenated in row order
    const int grain = 4096, nb = (n + grain - 1) / grain;
    std::vector<std::vector<int32_t>> bcol(nb);
    std::vector<std::vector<double>> bval(nb);
    std::vector<int32_t> len(n, 0);
    std::vector<SparseAcc> scratch(host_threads());
    parallel_blocks(n, grain, [&](int lo, int hi, int tid) {
        SparseAcc& S = scratch[tid];
        S.init(nco);
        auto& acc = S.acc;
        auto& mark = S.mark;
        auto& list = S.list;
        auto& oc = bcol[lo / grain];
        auto& ov = bval[lo / grain];
        for (int i = lo; i < hi; i++) {
            list.clear();
            mark[agg[i]] = i; acc[agg[i]] = 1.0; list.push_back(agg[i]);
            for (int q = F.rp[i]; q < F.rp[i + 1]; q++) {
                const int J = agg[F.col[q]];
                if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; list.push_back(J); }
                acc[J] -= omega * F.val[q] / diag[i];
            }
            std::sort(list.begin(), list.end());
            for (int J : list) { oc.push_back(J); ov.push_back(acc[J]); }
            len[i] = (int32_t)list.size();
        }
    });
    for (int i = 0; i < n; i++) prp[i + 1] = prp[i] + len[i];
    pcol.reserve(prp[n]);
    pval.reserve(prp[n]);
    for (int b = 0; b < nb; b++) {
        pcol.insert(pcol.end(), bcol[b].begin(), bcol[b].end());
        pval.insert(pval.end(), bval[b].begin(), bval[b].end());
    }
}

// A_c = P^T A P, rows with ascending columns
static void galerkin(const MgLevelHost& F, int nco, MgLevelHost& Cl)
{
    const int n = F.n;
    std::vector<int32_t> tp(nco + 1, 0);
    for (int i = 0; i < n; i++)
        for (int q = F.prp[i]; q < F.prp[i + 1]; q++) tp[F.pcol[q] + 1]++;
    for (int J = 0; J < nco; J++) tp[J + 1] += tp[J];
    std::vector<int32_t> tr(F.prp[n]);
    std::vector<double> tv(F.prp[n]);
    {
        std::vector<int32_t> fill(tp.begin(), tp.end() - 1);
        for (int i = 0; i < n; i++)
            for (int q = F.prp[i]; q < F.prp[i + 1]; q++) {
                const int J = F.pcol[q];
                tr[fill[J]] = i;
                tv[fill[J]] = F.pval[q];
                fill[J]++;
            }
    }
    Cl.n = nco;
    Cl.rp.assign(nco + 1, 0);
    Cl.col.clear();
    Cl.val.clear();
    // about 64 blocks of coarse rows: a coarse level has few rows but dense ones (each sums
    // over hundreds of fine rows), so even a small level is split across the threads
    const int grain = std::max(1, std::min(1024, nco / 64)), nb = (nco + grain - 1) / grain;
    std::vector<std::vector<int32_t>> bcol(nb);
    std::vector<std::vector<double>> bval(nb);
    std::vector<int32_t> len(nco, 0);
    std::vector<SparseAcc> scratch(host_threads());
    parallel_blocks(nco, grain, [&](int lo, int hi, int tid) {
        SparseAcc& S = scratch[tid];
        S.init(nco);
        auto& acc = S.acc;
        auto& mark = S.mark;
        auto& list = S.list;
        auto& oc = bcol[lo / grain];
        auto& ov = bval[lo / grain];
        for (int I = lo; I < hi; I++) {
            list.clear();
            for (int t = tp[I]; t < tp[I + 1]; t++) {
                const int i = tr[t];
                const double pI = tv[t];
                for (int k = F.rp[i]; k < F.rp[i + 1]; k++) {
                    const int j = F.col[k];
                    const double a = pI * F.val[k];
                    for (int q = F.prp[j]; q < F.prp[j + 1]; q++) {
                        const int J = F.pcol[q];
                        if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; list.push_back(J); }
                        acc[J] += a * F.pval[q];
                    }
                }
            }
            std::sort(list.begin(), list.end());
            for (int J : list) { oc.push_back(J); ov.push_back(acc[J]); }
            len[I] = (int32_t)list.size();
        }
    });
    for (int I = 0; I < nco; I++) Cl.rp[I + 1] = Cl.rp[I] + len[I];
    Cl.col.reserve(Cl.rp[nco]);
    Cl.val.reserve(Cl.rp[nco]);
    for (int b = 0; b < nb; b++) {
        Cl.col.insert(Cl.col.end(), bcol[b].begin(), bcol[b].end());
        Cl.val.insert(Cl.val.end(), bval[b].begin(), bval[b].end());
    }
}

std::string mg_build_hierarchy(MgLevelHost&& fine, double theta, int max_levels, int coarse_max, bool smoothed,
                               std::vector<MgLevelHost>& levels, std::vector<double>& chol)
{
    levels.clear();
    levels.push_back(std::move(fine));
    const int cap = max_levels > 0 ? max_levels : 25;
    const bool verbose = getenv("JFNK_VERBOSE") != nullptr;
    auto ms_since = [](std::chrono::steady_clock::time_point t0) {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    while ((int)levels.size() < cap && levels.back().n > coarse_max) {
        MgLevelHost& F = levels.back();
        std::vector<int32_t> agg;
        auto t0 = std::chrono::steady_clock::now();
        int nco = aggregate(F, theta, agg);
        const double t_agg = ms_since(t0);
        if (nco > 0.9 * F.n) break;
        F.agg = agg;
        t0 = std::chrono::steady_clock::now();
        smoothed_prolongation(F, agg, nco, smoothed, F.prp, F.pcol, F.pval);
        const double t_p = ms_since(t0);
        MgLevelHost Cl;
        t0 = std::chrono::steady_clock::now();
        galerkin(F, nco, Cl);
        if (verbose)
            fprintf(stderr, "[jfnk]   level %zu -> %d rows: aggregation %.1f ms, prolongation %.1f ms, Galerkin %.1f ms\n",
                    levels.size() - 1, nco, t_agg, t_p, ms_since(t0));
        levels.push_back(std::move(Cl));
    }
    const auto t_inv = std::chrono::steady_clock::now();
    // explicit inverse of the coarsest matrix via its Cholesky factor.  The inner products run
    // with four partial sums (independent chains for the host's FP pipes)
    const MgLevelHost& Lc = levels.back();
    const int n = Lc.n;
    auto dot = [](const double* a, const double* b, int len) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int q = 0;
        for (; q + 3 < len; q += 4) {
            s0 += a[q] * b[q]; s1 += a[q + 1] * b[q + 1]; s2 += a[q + 2] * b[q + 2]; s3 += a[q + 3] * b[q + 3];
        }
        for (; q < len; q++) s0 += a[q] * b[q];
        return (s0 + s1) + (s2 + s3);
    };
    std::vector<double> A((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++)
        for (int q = Lc.rp[i]; q < Lc.rp[i + 1]; q++) A[(size_t)i * n + Lc.col[q]] = Lc.val[q];
    for (int j = 0; j < n; j++) {
        const double* Lj = A.data() + (size_t)j * n;
        const double s = Lj[j] - dot(Lj, Lj, j);
        if (!(s > 0)) {
            char buf[96];
            snprintf(buf, sizeof buf, "coarse multigrid matrix not positive definite at row %d", j);
            return buf;
        }
        const double d = std::sqrt(s);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double* Li = A.data() + (size_t)i * n;
            Li[j] = (Li[j] - dot(Li, Lj, j)) / d;
        }
    }
    // X = (L L^T)^-1 = W^T W with W = L^-1: the columns of W by forward substitution (column c
    // is zero above row c; W is kept transposed, row c of Wt = column c of W, so that the
    // substitution reads rows of L and of Wt contiguously), then the symmetric product, each
    // entry a contiguous dot product over the rows both columns share
    std::vector<double> Wt((size_t)n * n, 0.0);
    parallel_blocks(n, 8, [&](int lo, int hi, int) {
        for (int c = lo; c < hi; c++) {
            double* w = Wt.data() + (size_t)c * n;
            w[c] = 1.0 / A[(size_t)c * n + c];
            for (int i = c + 1; i < n; i++) {
                const double* Li = A.data() + (size_t)i * n;
                w[i] = -dot(Li + c, w + c, i - c) / Li[i];
            }
        }
    });
    chol.assign((size_t)n * n, 0.0);
    parallel_blocks(n, 8, [&](int lo, int hi, int) {
        for (int i = lo; i < hi; i++) {
            const double* wi = Wt.data() + (size_t)i * n;
            for (int j = 0; j <= i; j++) {
                const double t = dot(wi + i, Wt.data() + (size_t)j * n + i, n - i);
                chol[(size_t)i * n + j] = t;
                chol[(size_t)j * n + i] = t;
            }
        }
    });
    if (verbose) fprintf(stderr, "[jfnk]   coarsest %d rows: dense inverse %.1f ms\n", n, ms_since(t_inv));
    return "";
}

}  // namespace jfnk
