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

void host_parallel(int n, int grain, const std::function<void(int, int)>& f)
{
    parallel_blocks(n, grain, [&](int lo, int hi, int) { f(lo, hi); });
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

// Reverse Cuthill-McKee (Cuthill & McKee 1969; George 1971) of the cells [c0, c1), whose
// neighbours all lie in the range: breadth-first search from a minimum-degree cell of each
// component (lowest index among equals), visiting neighbours by increasing degree (then
// index), and the order reversed.  Adjacency in CSR form: cell v's neighbours (cell indices)
// are adj[ap[v - c0] .. ap[v - c0 + 1]); the order (cell indices) is written to out[0, c1 - c0).
static void rcm_range(int c0, int c1, const int32_t* ap, const int32_t* adj, int32_t* out)
{
    const int n = c1 - c0;
    if (n <= 0) return;
    const int32_t* aptr = ap - c0;  // indexed by cell
    auto deg = [&](int v) { return aptr[v + 1] - aptr[v]; };
    // candidates by increasing degree, index order among equals (a counting sort)
    int maxd = 0;
    for (int v = c0; v < c1; v++) maxd = std::max(maxd, deg(v));
    std::vector<int32_t> start(maxd + 2, 0), cand(n);
    for (int v = c0; v < c1; v++) start[deg(v) + 1]++;
    for (int d = 0; d <= maxd; d++) start[d + 1] += start[d];
    for (int v = c0; v < c1; v++) cand[start[deg(v)]++] = v;
    std::vector<char> seen(n, 0);
    int tail = 0;  // the BFS order is built in out[0, tail)
    int32_t nb[64];
    std::vector<int32_t> nbv;
    for (int s : cand) {
        if (seen[s - c0]) continue;
        int head = tail;
        out[tail++] = s;
        seen[s - c0] = 1;
        while (head < tail) {
            const int v = out[head++];
            const int k = aptr[v + 1] - aptr[v];
            int32_t* list = nb;
            if (k > 64) {
                nbv.resize(k);
                list = nbv.data();
            }
            int m = 0;
            for (int q = aptr[v]; q < aptr[v + 1]; q++)
                if (!seen[adj[q] - c0]) list[m++] = adj[q];
            // insertion sort by (degree, index): a handful of neighbours
            for (int a = 1; a < m; a++) {
                const int w = list[a], dw = deg(w);
                int b = a - 1;
                for (; b >= 0 && (deg(list[b]) > dw || (deg(list[b]) == dw && list[b] > w)); b--) list[b + 1] = list[b];
                list[b + 1] = w;
            }
            for (int a = 0; a < m; a++) {
                seen[list[a] - c0] = 1;
                out[tail++] = list[a];
            }
        }
    }
    std::reverse(out, out + n);
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
    // groups that are contiguous, increasing ranges of cells, each with a contiguous range of
    // the internal faces and no face between two groups (the problems of a batch), are
    // renumbered and have their faces ordered each on its own host thread; the results are
    // those of single passes over all cells and faces
    std::vector<int32_t> gfirst, gface;
    bool grouped = group != nullptr;
    {
        if (grouped) {
            for (int i = 0; i < nc && grouped; i++) {
                const int g = (*group)[i];
                if (i == 0 || g != (*group)[i - 1]) {
                    grouped = i == 0 || g > (*group)[i - 1];
                    gfirst.push_back(i);
                }
            }
            gfirst.push_back(nc);
            // face range of each group: faces in group order, each inside its group
            const int ng = (int)gfirst.size() - 1;
            gface.assign(ng + 1, 0);
            int g = 0;
            for (int f = 0; f < ni && grouped; f++) {
                const int a = hm.own[f], b = hm.nei[f];
                while (g < ng && a >= gfirst[g + 1]) gface[++g] = f;
                grouped = a >= gfirst[g] && a < gfirst[g + 1] && b >= gfirst[g] && b < gfirst[g + 1];
            }
            while (g < ng) gface[++g] = ni;
        }
    }
    // --- cell numbering
    if (rcm) {
        t.n2o.resize(nc);
        // cell adjacency in CSR form over cells [c0, c1) from faces [f0, f1)
        auto adjacency = [&](int c0, int c1, int f0, int f1, std::vector<int32_t>& ap, std::vector<int32_t>& adj) {
            ap.assign(c1 - c0 + 1, 0);
            adj.resize(2 * (size_t)(f1 - f0));
            for (int f = f0; f < f1; f++) { ap[hm.own[f] - c0 + 1]++; ap[hm.nei[f] - c0 + 1]++; }
            for (int i = 0; i < c1 - c0; i++) ap[i + 1] += ap[i];
            std::vector<int32_t> fill(ap.begin(), ap.end() - 1);
            for (int f = f0; f < f1; f++) {
                adj[fill[hm.own[f] - c0]++] = hm.nei[f];
                adj[fill[hm.nei[f] - c0]++] = hm.own[f];
            }
        };
        if (grouped) {
            const int ng = (int)gfirst.size() - 1;
            parallel_blocks(ng, 1, [&](int lo, int hi, int) {
                std::vector<int32_t> ap, adj;
                for (int g = lo; g < hi; g++) {
                    adjacency(gfirst[g], gfirst[g + 1], gface[g], gface[g + 1], ap, adj);
                    rcm_range(gfirst[g], gfirst[g + 1], ap.data(), adj.data(), t.n2o.data() + gfirst[g]);
                }
            });
        } else {
            std::vector<int32_t> ap, adj;
            adjacency(0, nc, 0, ni, ap, adj);
            rcm_range(0, nc, ap.data(), adj.data(), t.n2o.data());
            if (group)
                std::stable_sort(t.n2o.begin(), t.n2o.end(), [&](int a, int b) { return (*group)[a] < (*group)[b]; });
        }
    } else {
        t.n2o.resize(nc);
        std::iota(t.n2o.begin(), t.n2o.end(), 0);
        if (group)
            std::stable_sort(t.n2o.begin(), t.n2o.end(), [&](int a, int b) { return (*group)[a] < (*group)[b]; });
    }
    t.o2n.assign(nc, -1);
    for (int i = 0; i < nc; i++) t.o2n[t.n2o[i]] = i;
    clk.lap("cell numbering");
    // --- face order
    struct FK { int32_t a, b, src; uint8_t flip; };
    std::vector<FK> in(ni);
    parallel_blocks(ni, 1 << 16, [&](int lo, int hi, int) {
        for (int f = lo; f < hi; f++) {
            int a = t.o2n[hm.own[f]], b = t.o2n[hm.nei[f]];
            uint8_t flip = 0;
            if (a > b) { std::swap(a, b); flip = 1; }
            in[f] = {a, b, f, flip};
        }
    });
    // stable counting sort of v[f0, f1) by key a in [c0, c1) (src ascending within a key, as
    // stored); with by_b, each key's short bucket then by b (insertion sort, stable)
    auto sort_range = [](std::vector<FK>& v, int f0, int f1, int c0, int c1, bool by_b, std::vector<FK>& tmp) {
        std::vector<int32_t> cnt(c1 - c0 + 1, 0);
        for (int f = f0; f < f1; f++) cnt[v[f].a - c0 + 1]++;
        for (int i = 0; i < c1 - c0; i++) cnt[i + 1] += cnt[i];
        tmp.resize(f1 - f0);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int f = f0; f < f1; f++) tmp[fill[v[f].a - c0]++] = v[f];
        std::copy(tmp.begin(), tmp.end(), v.begin() + f0);
        if (by_b)
            for (int i = 0; i < c1 - c0; i++)
                for (int q = f0 + cnt[i] + 1; q < f0 + cnt[i + 1]; q++) {
                    const FK k = v[q];
                    int r = q - 1;
                    for (; r >= f0 + cnt[i] && v[r].b > k.b; r--) v[r + 1] = v[r];
                    v[r + 1] = k;
                }
    };
    // internal faces by (a, b, src); a group's faces keep their range (the new cell numbers of
    // a group are the group's range)
    if (grouped) {
        const int ng = (int)gfirst.size() - 1;
        parallel_blocks(ng, 1, [&](int lo, int hi, int) {
            std::vector<FK> tmp;
            for (int g = lo; g < hi; g++) sort_range(in, gface[g], gface[g + 1], gfirst[g], gfirst[g + 1], true, tmp);
        });
    } else {
        std::vector<FK> tmp;
        sort_range(in, 0, ni, 0, nc, true, tmp);
    }
    auto by_owner = [&](std::vector<FK>& v) {
        std::vector<FK> tmp;
        sort_range(v, 0, (int)v.size(), 0, nc, false, tmp);
    };
    std::vector<FK> bd[4];  // disp, symm, trac, empty
    for (int f = ni; f < nf; f++) {
        int bt = hm.btype[f - ni];
        int cls = bt == JFNK_BC_DISP ? 0 : (bt == JFNK_BC_SYMM ? 1 : (bt == JFNK_BC_TRAC ? 2 : 3));
        bd[cls].push_back({t.o2n[hm.own[f]], -1, f, 0});
    }
    for (auto& v : bd) by_owner(v);  // (a, src): pushed in src order
    clk.lap("face order");
    t.ni = ni;
    t.nd = (int)bd[0].size();
    t.nsy = (int)bd[1].size();
    t.nt = (int)bd[2].size();
    t.ne = (int)bd[3].size();
    t.nf = nf;
    // face f of the new order: the internal faces, then the boundary classes
    std::vector<const FK*> cls_base(4);
    std::vector<int> cls_first(5, ni);
    for (int c = 0; c < 4; c++) {
        cls_base[c] = bd[c].data();
        cls_first[c + 1] = cls_first[c] + (int)bd[c].size();
    }
    auto key = [&](int f) -> const FK& {
        if (f < ni) return in[f];
        int c = 0;
        while (f >= cls_first[c + 1]) c++;
        return cls_base[c][f - cls_first[c]];
    };
    t.face_src.resize(nf);
    t.face_flip.resize(nf);
    t.own.resize(nf);
    t.nei.resize(ni);
    t.fptr.assign(nf + 1, 0);
    for (int f = 0; f < nf; f++) {
        const FK& k = key(f);
        t.fptr[f + 1] = t.fptr[f] + (hm.fptr[k.src + 1] - hm.fptr[k.src]);
    }
    t.fpts.resize(t.fptr[nf]);
    parallel_blocks(nf, 1 << 16, [&](int lo, int hi, int) {
        for (int f = lo; f < hi; f++) {
            const FK& k = key(f);
            t.face_src[f] = k.src;
            t.face_flip[f] = k.flip;
            t.own[f] = k.a;
            if (f < ni) t.nei[f] = k.b;
            const int s0 = hm.fptr[k.src], s1 = hm.fptr[k.src + 1];
            int32_t* o = t.fpts.data() + t.fptr[f];
            if (!k.flip)
                for (int q = s0; q < s1; q++) *o++ = hm.fpts[q];
            else
                for (int q = s1 - 1; q >= s0; q--) *o++ = hm.fpts[q];
        }
    });
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
    // all faces of each cell (geometry): owner side f, neighbour side ~f, by face index: the
    // cell's owned and neighbouring internal faces merged by index, then its boundary faces
    // (each class owner-sorted, classes in face order)
    std::vector<int32_t> fe_ptr;
    ranges(ni + t.nd + t.nsy + t.nt, nf, fe_ptr);
    t.ca_ptr.assign(nc + 1, 0);
    for (int P = 0; P < nc; P++)
        t.ca_ptr[P + 1] = t.ca_ptr[P] + (t.fo_ptr[P + 1] - t.fo_ptr[P]) + (t.fn_ptr[P + 1] - t.fn_ptr[P]) +
                          (t.fd_ptr[P + 1] - t.fd_ptr[P]) + (t.fs_ptr[P + 1] - t.fs_ptr[P]) +
                          (t.ft_ptr[P + 1] - t.ft_ptr[P]) + (fe_ptr[P + 1] - fe_ptr[P]);
    t.ca_face.resize(t.ca_ptr[nc]);
    parallel_blocks(nc, 1 << 15, [&](int lo, int hi, int) {
        for (int P = lo; P < hi; P++) {
            int32_t* o = t.ca_face.data() + t.ca_ptr[P];
            int a = t.fo_ptr[P], b = t.fn_ptr[P];
            const int ae = t.fo_ptr[P + 1], be = t.fn_ptr[P + 1];
            while (a < ae || b < be) {
                if (b >= be || (a < ae && a < t.fn_face[b])) *o++ = a++;
                else *o++ = ~t.fn_face[b++];
            }
            const std::vector<int32_t>* bp[4] = {&t.fd_ptr, &t.fs_ptr, &t.ft_ptr, &fe_ptr};
            for (const auto* p : bp)
                for (int f = (*p)[P]; f < (*p)[P + 1]; f++) *o++ = f;
        }
    });
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
    // walk each cell's internal faces in increasing face index: merge owner and neighbour lists
    parallel_blocks(nc, 1 << 15, [&](int lo, int hi, int) {
        for (int P = lo; P < hi; P++) {
            int a = t.fo_ptr[P], ae = t.fo_ptr[P + 1];
            int b = t.fn_ptr[P], be = t.fn_ptr[P + 1];
            const int s = P / 32, lane = P % 32;
            int k = 0;
            while (a < ae || b < be) {
                int f, N;
                if (b >= be || (a < ae && a < t.fn_face[b])) { f = a; N = t.nei[a]; a++; }
                else { f = t.fn_face[b]; N = t.own[f]; b++; }
                const int slot = t.sell_off[s] + 32 * k + lane;
                t.sell_nbr[slot] = N;
                t.sell_face[slot] = f;
                k++;
            }
            for (int f = t.fs_ptr[P]; f < t.fs_ptr[P + 1]; f++) {  // mirror neighbours
                const int slot = t.sell_off[s] + 32 * k + lane;
                t.sell_nbr[slot] = nc + (f - ni - t.nd);
                t.sell_face[slot] = f;
                k++;
            }
        }
    });
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
    parallel_blocks(n, 1 << 14, [&](int lo, int hi, int) {
        for (int i = lo; i < hi; i++) {
            double mx = 0;
            for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
                if (L.col[q] != i) mx = std::max(mx, -L.val[q]);
            for (int q = L.rp[i]; q < L.rp[i + 1]; q++)
                strong[q] = (L.col[q] != i && mx > 0 && -L.val[q] >= theta * mx * (1.0 - tie));
        }
    });
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
    // row i of P: the aggregates of i and of its neighbours, ascending, with their weights; two
    // passes over blocks of rows (the entry counts, then the entries at their final places),
    // so that no thread grows arrays of its own
    const int grain = 4096;
    std::vector<SparseAcc> scratch(host_threads());
    auto row = [&](SparseAcc& S, int i) {
        auto& acc = S.acc;
        auto& mark = S.mark;
        auto& list = S.list;
        list.clear();
        mark[agg[i]] = i; acc[agg[i]] = 1.0; list.push_back(agg[i]);
        for (int q = F.rp[i]; q < F.rp[i + 1]; q++) {
            const int J = agg[F.col[q]];
            if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; list.push_back(J); }
            acc[J] -= omega * F.val[q] / diag[i];
        }
        std::sort(list.begin(), list.end());
    };
    parallel_blocks(n, grain, [&](int lo, int hi, int tid) {
        SparseAcc& S = scratch[tid];
        S.init(nco);
        for (int i = lo; i < hi; i++) {
            row(S, i);
            prp[i + 1] = (int32_t)S.list.size();
        }
    });
    for (int i = 0; i < n; i++) prp[i + 1] += prp[i];
    pcol.resize(prp[n]);
    pval.resize(prp[n]);
    for (auto& S : scratch) S.acc.clear(), S.mark.clear();  // stamps restart from a clean state
    parallel_blocks(n, grain, [&](int lo, int hi, int tid) {
        SparseAcc& S = scratch[tid];
        S.init(nco);
        for (int i = lo; i < hi; i++) {
            row(S, i);
            int o = prp[i];
            for (int J : S.list) { pcol[o] = J; pval[o] = S.acc[J]; o++; }
        }
    });
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
