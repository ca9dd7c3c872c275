// gdi_api.cpp -- host side of libgdi.so: the C ABI declared in include/gdi.h.
//
// gdi_create validates the CSR, colours it (greedy first-fit in vertex-id order unless a colouring
// is given), relabels every instance into rank order (colour asc, then splitmix64 of the local
// vertex id asc inside each class), packs each neighbour as
// (local rank | weight-sign bit) and uploads the rank-space CSR once.  gdi_anneal builds the
// per-sweep threshold table on the host (double precision; the GPU never evaluates exp), then
// enqueues the initial-state kernel and the persistent anneal kernel on the caller's stream.
#include "gdi.h"
#include "gdi_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(GDI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count)
    {
        if (count <= n && p) return cudaSuccess;
        release();
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaMalloc((void **)&p, bytes);
        if (e == cudaSuccess) n = count; else p = nullptr;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

}  // namespace

int gdi_set_error(int code, const std::string &msg) { return fail(code, msg); }

namespace {
// splitmix64 finaliser (Steele, Lea, Flood 2014): the in-class rank key
uint64_t splitmix64_host(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
}  // namespace

struct gdi_ctx {
    int device = 0;
    int32_t Q = 0, R = 1, A = 0, B = 1, W = 0;
    int64_t N = 0, nnz = 0;
    int32_t max_n = 0, max_window = 0, max_degree = 0, max_class = 0;
    int32_t path = 0;                        // GDI_PATH_*
    DevBuf<uint8_t> g_packed, g_rflags;
    DevBuf<int16_t> g_tables;
    DevBuf<int32_t> g_gin, g_Gcls, g_err, g_status, g_rhist, g_rties, g_rparams;
    DevBuf<unsigned int> g_bar;
    DevBuf<unsigned long long> g_hfield;
    bool used_grid = false;
    // cost-weighted split of every colour class over the grid path's blocks: window costs (one
    // instance, W >= 1), and the device copy of the bounds for the last block count and cap
    std::vector<int64_t> wcost, wcost_off;
    DevBuf<int32_t> g_wbnd;
    int wbnd_blocks = 0, wbnd_wpc = 0;
    // events around the anneal kernel launches of the last gdi_anneal (none while capturing)
    std::vector<cudaEvent_t> kev;
    int kev_pairs = 0;
    // failure-detection test hook for the next grid-scale anneal (gdi_inject_wait_failure)
    long long inject_limit = 0;
    std::vector<int32_t> num_classes;       // per instance
    DevBuf<int64_t> node_off, row_ptr;
    DevBuf<int32_t> class_off, class_ptr, rank_of;
    DevBuf<uint32_t> col;
    DevBuf<uint16_t> col16;
    DevBuf<int8_t> spins, init_stage, out_stage;
    DevBuf<uint32_t> tab;
    DevBuf<int32_t> tab_off;
    DevBuf<float> temp;
    DevBuf<int32_t> item_order, item_counter;
    // pinned staging of the per-anneal host->device copies, so that an anneal can be captured in
    // a CUDA graph (no pageable copies, no allocation once the buffers exist)
    uint32_t *h_tab = nullptr;
    int32_t *h_off = nullptr;
    float *h_temp = nullptr;
    size_t h_tab_n = 0, h_off_n = 0;
    bool tab_valid = false;
    gdi_schedule tab_sched{};
    int32_t tab_ecap = 0, tab_max_row = 0;
    DevBuf<int32_t> raw_G, final_G, tr_G, err;
    DevBuf<int64_t> raw_cut, final_cut, tr_cut;
    DevBuf<uint64_t> tr_digest;
    int32_t last_sweeps = 0, last_flags = 0, ecap = 0;
    bool annealed = false;
    cudaStream_t stream = nullptr;
    int block = 256;
    int grid_limit = 0;
    int last_grid = 0;
    size_t last_smem = 0;

    GdiDevProblem problem() const
    {
        GdiDevProblem P;
        P.num_instances = Q;
        P.replicas = R;
        P.N = N;
        P.node_off = node_off.p;
        P.class_off = class_off.p;
        P.class_ptr = class_ptr.p;
        P.row_ptr = row_ptr.p;
        P.col = col.p;
        P.col16 = col16.p;
        P.rank_of = rank_of.p;
        P.A = A;
        P.B = B;
        P.W = W;
        P.max_n = max_n;
        P.max_window = max_window;
        P.max_degree = max_degree;
        P.max_class = max_class;
        return P;
    }
    void release()
    {
        node_off.release(); row_ptr.release(); class_off.release(); class_ptr.release();
        rank_of.release(); col.release(); col16.release(); spins.release(); init_stage.release(); out_stage.release();
        tab.release(); tab_off.release(); temp.release(); raw_G.release(); final_G.release(); tr_G.release();
        err.release(); raw_cut.release(); final_cut.release(); tr_cut.release(); tr_digest.release();
        g_packed.release(); g_rflags.release(); g_tables.release(); g_gin.release(); g_Gcls.release();
        g_wbnd.release();
        for (cudaEvent_t ev : kev) cudaEventDestroy(ev);
        kev.clear();
        kev_pairs = 0;
        g_err.release(); g_status.release(); g_rhist.release(); g_rties.release(); g_rparams.release();
        g_bar.release();
        item_order.release(); item_counter.release();
        if (h_tab) cudaFreeHost(h_tab);
        if (h_off) cudaFreeHost(h_off);
        if (h_temp) cudaFreeHost(h_temp);
        h_tab = nullptr; h_off = nullptr; h_temp = nullptr; h_tab_n = h_off_n = 0;
    }
    GdiGridScratch grid_scratch()
    {
        GdiGridScratch X;
        X.packed = g_packed.p;
        X.tables = g_tables.p;
        X.gin = g_gin.p;
        X.Gcls = g_Gcls.p;
        X.bar = g_bar.p;
        X.err = g_err.p;
        X.status = g_status.p;
        X.rhist = g_rhist.p;
        X.rflags = g_rflags.p;
        X.rties = g_rties.p;
        X.rparams = g_rparams.p;
        X.hfield = g_hfield.p;
        X.spin_limit = 1ll << 26;
        X.bar_start = 0;
        return X;
    }
};

namespace {

// ---------------------------------------------------------------------------------------------
// Threshold table.  Metropolis row s holds thr_s(dE) = floor(exp(-dE / T_s) 2^32) for dE = 1, 2, ...
// while it is non-zero (thr = 2^32 for dE <= 0 is implicit); T_s = t0 (t1/t0)^(s/(M-1)).
// Paper row s holds thr for dE = -1, 0, +1: 2^32 - p, 2^31, p with p = floor(P_f,s 2^32) + 1
// (argmin, then the random flip "u <= P_f" of Section 5.2), P_f,s = pf0 (pf1/pf0)^(s/(M-1)).
double sched_at(double v0, double v1, int s, int M)
{
    if (M <= 1 || v0 == v1) return v0;
    return v0 * std::pow(v1 / v0, (double)s / (double)(M - 1));
}

int build_table(const gdi_schedule &S, std::vector<uint32_t> &tab, std::vector<int32_t> &off,
                std::vector<float> &temp, int32_t &ecap, int32_t &max_row)
{
    const int M = S.sweeps;
    tab.clear();
    off.assign((size_t)M + 1, 0);
    temp.assign((size_t)M, 0.f);
    max_row = 0;
    if (S.mode == GDI_METROPOLIS) {
        if (!(S.t0 > 0.0) || !(S.t1 > 0.0) || !std::isfinite(S.t0) || !std::isfinite(S.t1))
            return fail(GDI_ERR_INVALID_ARG, "Metropolis temperatures must be finite and > 0");
        for (int s = 0; s < M; ++s) {
            off[s] = (int32_t)tab.size();
            const double T = sched_at(S.t0, S.t1, s, M);
            temp[(size_t)s] = (float)T;
            for (int64_t E = 1;; ++E) {
                const double t = std::floor(std::exp(-(double)E / T) * 4294967296.0);
                if (t <= 0.0) break;
                if (E > (1 << 22)) return fail(GDI_ERR_OVERFLOW, "temperature too high for the table");
                tab.push_back((uint32_t)t);
            }
            max_row = std::max<int32_t>(max_row, (int32_t)tab.size() - off[s]);
            if (tab.size() > (size_t)1 << 28) return fail(GDI_ERR_OVERFLOW, "threshold table too large");
        }
        off[M] = (int32_t)tab.size();
        ecap = max_row + 1;
        return GDI_OK;
    }
    if (S.mode == GDI_PAPER_PF) {
        if (!(S.pf0 >= 0 && S.pf0 < 0.5 && S.pf1 >= 0 && S.pf1 < 0.5))
            return fail(GDI_ERR_INVALID_ARG, "P_f must lie in [0, 0.5)");
        if (S.pf0 != S.pf1 && (S.pf0 <= 0 || S.pf1 <= 0))
            return fail(GDI_ERR_INVALID_ARG, "a geometric P_f schedule needs pf0, pf1 > 0");
        for (int s = 0; s < M; ++s) {
            off[s] = (int32_t)tab.size();
            const double pf = sched_at(S.pf0, S.pf1, s, M);
            uint64_t p = (uint64_t)std::floor(pf * 4294967296.0) + 1;
            if (p > ((uint64_t)1 << 32)) p = (uint64_t)1 << 32;
            tab.push_back((uint32_t)(((uint64_t)1 << 32) - p));
            tab.push_back(0x80000000u);
            tab.push_back((uint32_t)p);
        }
        off[M] = (int32_t)tab.size();
        max_row = 3;
        ecap = 1;
        return GDI_OK;
    }
    return fail(GDI_ERR_INVALID_ARG, "unknown schedule mode");
}

// ---------------------------------------------------------------------------------------------
// CSR validation: ids inside the instance, no self-loops, no duplicates, weights +-1, symmetric.
int validate_graph(const gdi_graph &g, const std::vector<int64_t> &inst, std::vector<int32_t> &w)
{
    const int64_t N = g.num_vertices;
    if (g.row_ptr[0] != 0) return fail(GDI_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (int64_t v = 0; v < N; ++v)
        if (g.row_ptr[v + 1] < g.row_ptr[v]) return fail(GDI_ERR_INVALID_ARG, "row_ptr not monotone");
    const int64_t nnz = g.row_ptr[N];
    w.resize((size_t)nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        const int32_t x = g.weight ? g.weight[e] : 1;
        if (x != 1 && x != -1) return fail(GDI_ERR_INVALID_ARG, "edge weights must be +1 or -1");
        w[(size_t)e] = x;
    }
    std::vector<int64_t> stamp((size_t)N, -1);
    size_t q = 0;
    for (int64_t v = 0; v < N; ++v) {
        while (inst[q + 1] <= v) ++q;
        for (int64_t e = g.row_ptr[v]; e < g.row_ptr[v + 1]; ++e) {
            const int64_t j = g.col[e];
            if (j < inst[q] || j >= inst[q + 1])
                return fail(GDI_ERR_INVALID_ARG, "neighbour id outside its instance (vertex " + std::to_string(v) + ")");
            if (j == v) return fail(GDI_ERR_SELF_LOOP, "self-loop at vertex " + std::to_string(v));
            if (stamp[(size_t)j] == v)
                return fail(GDI_ERR_DUP_EDGE, "duplicate edge " + std::to_string(v) + "-" + std::to_string(j));
            stamp[(size_t)j] = v;
        }
    }
    // symmetry: per row a sorted copy (by neighbour), then each (v, j, w) must find (j, v, w)
    std::vector<int32_t> sc((size_t)nnz);
    std::vector<int32_t> sw((size_t)nnz);
    std::vector<int64_t> idx;
    for (int64_t v = 0; v < N; ++v) {
        const int64_t e0 = g.row_ptr[v], e1 = g.row_ptr[v + 1];
        idx.resize((size_t)(e1 - e0));
        for (int64_t e = e0; e < e1; ++e) idx[(size_t)(e - e0)] = e;
        std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return g.col[a] < g.col[b]; });
        for (int64_t k = 0; k < e1 - e0; ++k) {
            sc[(size_t)(e0 + k)] = g.col[idx[(size_t)k]];
            sw[(size_t)(e0 + k)] = w[(size_t)idx[(size_t)k]];
        }
    }
    for (int64_t v = 0; v < N; ++v) {
        for (int64_t e = g.row_ptr[v]; e < g.row_ptr[v + 1]; ++e) {
            const int64_t j = sc[(size_t)e];
            const int32_t *b = sc.data() + g.row_ptr[j];
            const int32_t *en = sc.data() + g.row_ptr[j + 1];
            const int32_t *f = std::lower_bound(b, en, (int32_t)v);
            if (f == en || *f != v || sw[(size_t)(f - sc.data())] != sw[(size_t)e])
                return fail(GDI_ERR_NOT_SYMMETRIC, "edge " + std::to_string(v) + "-" + std::to_string(j) +
                                                       " has no mirror with the same weight");
        }
    }
    return GDI_OK;
}

// ---------------------------------------------------------------------------------------------
// Host preprocessing shared by gdi_create and gdi_rank_space: validation, colouring, rank order
// and the rank-space CSR of every instance (instance bounds `inst`, window W for max_window).
struct HostRankSpace {
    std::vector<int32_t> w, color, rank_of, vert_of, class_off, class_ptr, num_classes;
    std::vector<int64_t> rp;
    std::vector<uint32_t> cr;
    int32_t max_n = 0, max_window = 0, max_class = 0, max_degree = 0;
};

int build_rank_space(const gdi_graph *g, const std::vector<int64_t> &inst, int32_t W, HostRankSpace &H)
{
    const int32_t Q = g->num_instances;
    const int64_t N = g->num_vertices;
    int rc = validate_graph(*g, inst, H.w);
    if (rc) return rc;
    const std::vector<int32_t> &w = H.w;

    // colouring: caller's (checked) or greedy first-fit in id order, per instance
    std::vector<int32_t> &color = H.color;
    color.assign((size_t)N, 0);
    if (g->color) {
        for (int64_t v = 0; v < N; ++v) {
            if (g->color[v] < 0) return fail(GDI_ERR_BAD_COLORING, "negative colour");
            color[(size_t)v] = g->color[v];
        }
    } else {
        std::vector<int64_t> mark;
        for (int64_t v = 0; v < N; ++v) {
            const int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
            if ((int64_t)mark.size() < d + 2) mark.resize((size_t)d + 2, -1);
            for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
                const int64_t j = g->col[e];
                if (j < v) {
                    const int32_t c = color[(size_t)j];
                    if (c < d + 2) mark[(size_t)c] = v;
                }
            }
            int32_t c = 0;
            while (mark[(size_t)c] == v) ++c;
            color[(size_t)v] = c;
        }
    }
    for (int64_t v = 0; v < N; ++v)
        for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e)
            if (color[(size_t)g->col[e]] == color[(size_t)v])
                return fail(GDI_ERR_BAD_COLORING, "adjacent vertices share a colour");

    // rank order per instance: counting sort by colour, then inside each class by splitmix64 of
    // the local vertex id
    std::vector<int32_t> &rank_of = H.rank_of, &vert_of = H.vert_of;
    std::vector<int32_t> &class_off = H.class_off, &class_ptr = H.class_ptr;
    rank_of.assign((size_t)N, 0);
    vert_of.assign((size_t)N, 0);
    class_off.assign((size_t)Q + 1, 0);
    class_ptr.clear();
    H.num_classes.assign((size_t)Q, 0);
    for (int32_t q = 0; q < Q; ++q) {
        const int64_t lo = inst[(size_t)q], hi = inst[(size_t)q + 1];
        const int32_t n = (int32_t)(hi - lo);
        int32_t ncol = 0;
        for (int64_t v = lo; v < hi; ++v) ncol = std::max(ncol, color[(size_t)v] + 1);
        if ((int64_t)ncol > (int64_t)n + 1 && ncol > (1 << 24))
            return fail(GDI_ERR_OVERFLOW, "colour values too large");
        std::vector<int32_t> cnt((size_t)ncol + 1, 0);
        for (int64_t v = lo; v < hi; ++v) cnt[(size_t)color[(size_t)v] + 1]++;
        for (int32_t k = 0; k < ncol; ++k) cnt[(size_t)k + 1] += cnt[(size_t)k];
        class_off[(size_t)q] = (int32_t)class_ptr.size();
        int32_t nclass = 0;
        for (int32_t k = 0; k < ncol; ++k) {
            if (cnt[(size_t)k + 1] > cnt[(size_t)k]) {
                class_ptr.push_back(cnt[(size_t)k]);
                const int32_t sz = cnt[(size_t)k + 1] - cnt[(size_t)k];
                H.max_window = std::max(H.max_window, W > 0 ? std::min(W, sz) : sz);
                H.max_class = std::max(H.max_class, sz);
                ++nclass;
            }
        }
        class_ptr.push_back(n);
        H.num_classes[(size_t)q] = nclass;
        for (int64_t v = lo; v < hi; ++v) {
            const int32_t r = cnt[(size_t)color[(size_t)v]]++;
            vert_of[(size_t)(lo + r)] = (int32_t)v;
        }
        // inside a class, ranks follow splitmix64 of the local vertex id (a fixed pseudo-random
        // order, so that heavy vertices spread over windows and blocks)
        {
            std::vector<std::pair<uint64_t, int32_t>> keyed;
            const int32_t *bounds = class_ptr.data() + class_off[(size_t)q];
            for (int32_t k = 0; k < nclass; ++k) {
                const int32_t c0 = bounds[k], c1 = bounds[k + 1];
                keyed.resize((size_t)(c1 - c0));
                for (int32_t r = c0; r < c1; ++r) {
                    const int32_t v = vert_of[(size_t)(lo + r)];
                    keyed[(size_t)(r - c0)] = {splitmix64_host((uint64_t)(v - lo)), v};
                }
                std::sort(keyed.begin(), keyed.end());
                for (int32_t r = c0; r < c1; ++r) vert_of[(size_t)(lo + r)] = keyed[(size_t)(r - c0)].second;
            }
        }
        for (int64_t r = lo; r < hi; ++r) rank_of[(size_t)vert_of[(size_t)r]] = (int32_t)r;
        H.max_n = std::max(H.max_n, n);
    }
    class_off[(size_t)Q] = (int32_t)class_ptr.size();

    // rank-space CSR, neighbour = local rank | weight-sign bit
    std::vector<int64_t> &rp = H.rp;
    std::vector<uint32_t> &cr = H.cr;
    rp.assign((size_t)N + 1, 0);
    cr.assign((size_t)g->row_ptr[N], 0);
    {
        size_t q = 0;
        int64_t e_out = 0;
        for (int64_t r = 0; r < N; ++r) {
            while (inst[q + 1] <= r) ++q;
            const int64_t v = vert_of[(size_t)r];
            rp[(size_t)r] = e_out;
            const int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
            H.max_degree = (int32_t)std::max<int64_t>(H.max_degree, d);
            for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
                const uint32_t lr = (uint32_t)(rank_of[(size_t)g->col[e]] - inst[q]);
                cr[(size_t)e_out++] = lr | (w[(size_t)e] < 0 ? 0x80000000u : 0u);
            }
        }
        rp[(size_t)N] = e_out;
    }
    return GDI_OK;
}

}  // namespace

extern "C" {

int gdi_create(gdi_ctx **out, const gdi_graph *g, const gdi_model *m)
{
    if (!out || !g || !m) return fail(GDI_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (g->num_instances < 1 || g->num_vertices < 1 || !g->row_ptr || !g->col)
        return fail(GDI_ERR_INVALID_ARG, "empty graph or missing CSR arrays");
    if (g->num_instances > 1 && !g->inst_ptr) return fail(GDI_ERR_INVALID_ARG, "inst_ptr required for a batch");
    if (m->A < 0 || m->B < 1 || m->W < 0 || m->replicas < 1)
        return fail(GDI_ERR_INVALID_ARG, "need A >= 0, B >= 1, W >= 0, replicas >= 1");
    if (m->A > (1 << 20) || m->B > (1 << 20)) return fail(GDI_ERR_OVERFLOW, "A or B too large");
    const int32_t Q = g->num_instances;
    const int64_t N = g->num_vertices;
    std::vector<int64_t> inst((size_t)Q + 1);
    if (g->inst_ptr) {
        for (int32_t q = 0; q <= Q; ++q) inst[(size_t)q] = g->inst_ptr[q];
    } else {
        inst[0] = 0;
        inst[1] = N;
    }
    if (inst[0] != 0 || inst[(size_t)Q] != N) return fail(GDI_ERR_INVALID_ARG, "inst_ptr must run from 0 to N");
    for (int32_t q = 0; q < Q; ++q) {
        if (inst[(size_t)q + 1] <= inst[(size_t)q]) return fail(GDI_ERR_INVALID_ARG, "empty instance");
        if (inst[(size_t)q + 1] - inst[(size_t)q] > (1 << 28)) return fail(GDI_ERR_OVERFLOW, "instance over 2^28 vertices");
    }
    if ((int64_t)m->replicas * N > ((int64_t)1 << 40)) return fail(GDI_ERR_OVERFLOW, "replicas * N too large");

    HostRankSpace H;
    int rc = build_rank_space(g, inst, m->W, H);
    if (rc) return rc;
    const std::vector<int32_t> &rank_of = H.rank_of, &class_off = H.class_off, &class_ptr = H.class_ptr;
    const std::vector<int64_t> &rp = H.rp;
    const std::vector<uint32_t> &cr = H.cr;

    gdi_ctx *c = new (std::nothrow) gdi_ctx;
    if (!c) return fail(GDI_ERR_OOM, "host allocation failed");
    cudaGetDevice(&c->device);
    c->Q = Q;
    c->R = m->replicas;
    c->A = m->A;
    c->B = m->B;
    c->W = m->W;
    c->N = N;
    c->nnz = g->row_ptr[N];
    c->num_classes = H.num_classes;
    c->max_n = H.max_n;
    c->max_window = H.max_window;
    c->max_class = H.max_class;
    c->max_degree = H.max_degree;
    // window costs for the grid path's weighted split: a rank costs its degree plus a constant for
    // its threshold and its share of the window sort (both measured as about 12 neighbour reads)
    if (Q == 1 && c->W >= 1) {
        const int32_t nclass = c->num_classes[0];
        c->wcost_off.assign((size_t)nclass + 1, 0);
        for (int32_t k = 0; k < nclass; ++k) {
            const int32_t c0 = class_ptr[(size_t)k], c1 = class_ptr[(size_t)k + 1];
            for (int32_t a = c0; a < c1; a += c->W) {
                const int32_t b = std::min(a + c->W, c1);
                c->wcost.push_back((rp[(size_t)b] - rp[(size_t)a]) + (int64_t)12 * (b - a));
            }
            c->wcost_off[(size_t)k + 1] = (int64_t)c->wcost.size();
        }
    }

    cudaError_t e;
#define GDI_UP(buf, vec)                                                                          \
    do {                                                                                          \
        e = buf.alloc(vec.size());                                                                \
        if (e == cudaSuccess && !vec.empty())                                                     \
            e = cudaMemcpy(buf.p, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice); \
        if (e != cudaSuccess) {                                                                   \
            c->release();                                                                         \
            delete c;                                                                             \
            return e == cudaErrorMemoryAllocation ? fail(GDI_ERR_OOM, "device allocation failed")  \
                                                  : cuda_fail(e, "upload");                       \
        }                                                                                         \
    } while (0)
    GDI_UP(c->node_off, inst);
    GDI_UP(c->row_ptr, rp);
    GDI_UP(c->col, cr);
    if (H.max_n <= 32767) {
        // 16-bit columns for the CTA-resident kernels' neighbour sums (half the CSR bytes)
        std::vector<uint16_t> c16(cr.size());
        for (size_t e = 0; e < cr.size(); ++e)
            c16[e] = (uint16_t)((cr[e] & 0x7FFFu) | ((cr[e] >> 31) << 15));
        GDI_UP(c->col16, c16);
    }
    GDI_UP(c->class_off, class_off);
    GDI_UP(c->class_ptr, class_ptr);
    GDI_UP(c->rank_of, rank_of);
    {
        // work queue order for the CTA path: largest instance (vertices + CSR entries) first
        std::vector<int32_t> order((size_t)Q * c->R);
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
        std::vector<int64_t> work((size_t)Q);
        for (int32_t q = 0; q < Q; ++q)
            work[(size_t)q] = (inst[(size_t)q + 1] - inst[(size_t)q]) + (g->row_ptr[inst[(size_t)q + 1]] - g->row_ptr[inst[(size_t)q]]);
        const int32_t Rr = c->R;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return work[(size_t)(a / Rr)] > work[(size_t)(b / Rr)];
        });
        GDI_UP(c->item_order, order);
    }
#undef GDI_UP
    e = c->spins.alloc((size_t)c->R * (size_t)N);
    if (e == cudaSuccess) e = c->raw_G.alloc((size_t)Q * c->R);
    if (e == cudaSuccess) e = c->final_G.alloc((size_t)Q * c->R);
    if (e == cudaSuccess) e = c->raw_cut.alloc((size_t)Q * c->R);
    if (e == cudaSuccess) e = c->final_cut.alloc((size_t)Q * c->R);
    if (e == cudaSuccess) e = c->err.alloc(4);
    if (e == cudaSuccess) e = c->item_counter.alloc(1);
    if (e != cudaSuccess) {
        c->release();
        delete c;
        return fail(GDI_ERR_OOM, "device allocation failed");
    }
    *out = c;
    return GDI_OK;
}

int gdi_rank_space(const gdi_graph *g, int32_t *vert_of, int64_t *row_ptr, uint32_t *col,
                   int32_t *class_ptr, int32_t *num_classes, int32_t *max_class, int32_t *max_degree)
{
    if (!g || !vert_of || !row_ptr || !col || !class_ptr || !num_classes)
        return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (g->num_instances != 1 || g->num_vertices < 1 || !g->row_ptr || !g->col)
        return fail(GDI_ERR_INVALID_ARG, "gdi_rank_space takes one non-empty graph");
    if (g->num_vertices > (1 << 28)) return fail(GDI_ERR_OVERFLOW, "graph over 2^28 vertices");
    const int64_t N = g->num_vertices;
    std::vector<int64_t> inst = {0, N};
    HostRankSpace H;
    const int rc = build_rank_space(g, inst, 0, H);
    if (rc) return rc;
    std::copy(H.vert_of.begin(), H.vert_of.end(), vert_of);
    std::copy(H.rp.begin(), H.rp.end(), row_ptr);
    std::copy(H.cr.begin(), H.cr.end(), col);
    std::copy(H.class_ptr.begin(), H.class_ptr.end(), class_ptr);
    *num_classes = H.num_classes[0];
    if (max_class) *max_class = H.max_class;
    if (max_degree) *max_degree = H.max_degree;
    return GDI_OK;
}

int gdi_build_table(const gdi_schedule *S, uint32_t *tab, int64_t tab_cap, int64_t *tab_len,
                    int32_t *tab_off, float *temp, int32_t *max_row)
{
    if (!S || !tab_len) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (S->sweeps < 1) return fail(GDI_ERR_INVALID_ARG, "sweeps must be >= 1");
    std::vector<uint32_t> t;
    std::vector<int32_t> off;
    std::vector<float> tp;
    int32_t ecap = 0, mr = 0;
    const int rc = build_table(*S, t, off, tp, ecap, mr);
    if (rc) return rc;
    *tab_len = (int64_t)t.size();
    if (max_row) *max_row = mr;
    if (!tab) return GDI_OK;                     // size query
    if (tab_cap < (int64_t)t.size()) return fail(GDI_ERR_INVALID_ARG, "tab_cap below the table length");
    if (!tab_off || !temp) return fail(GDI_ERR_INVALID_ARG, "null tab_off or temp");
    std::copy(t.begin(), t.end(), tab);
    std::copy(off.begin(), off.end(), tab_off);
    std::copy(tp.begin(), tp.end(), temp);
    return GDI_OK;
}

int gdi_anneal(gdi_ctx *c, const gdi_schedule *S, const gdi_run *run)
{
    if (!c || !S || !run) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (S->sweeps < 1) return fail(GDI_ERR_INVALID_ARG, "sweeps must be >= 1");
    const int32_t s_begin = run->first_sweep;
    const int32_t s_end = run->last_sweep > 0 ? run->last_sweep : S->sweeps;
    if (s_begin < 0 || s_end > S->sweeps || s_begin > s_end)
        return fail(GDI_ERR_INVALID_ARG, "sweep range outside the schedule");
    const bool cont = (run->flags & GDI_FLAG_CONTINUE) != 0;
    if (cont && !c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "GDI_FLAG_CONTINUE before any anneal");
    if (!cont && !run->init_spins && s_begin != 0)
        return fail(GDI_ERR_INVALID_ARG, "a random start must begin at sweep 0");

    // the device table is rebuilt only when the schedule changes (then the previous anneal, which
    // may still read it, is waited for); repeated anneals with one schedule enqueue no copies, so
    // they can be captured in a CUDA graph
    cudaStream_t st = (cudaStream_t)run->stream;
    cudaError_t e = cudaSuccess;
    const bool same = c->tab_valid && c->tab_sched.mode == S->mode && c->tab_sched.t0 == S->t0 &&
                      c->tab_sched.t1 == S->t1 && c->tab_sched.pf0 == S->pf0 &&
                      c->tab_sched.pf1 == S->pf1 && c->tab_sched.sweeps == S->sweeps;
    int32_t ecap = 0, max_row = 0;
    if (same) {
        ecap = c->tab_ecap;
        max_row = c->tab_max_row;
    } else {
        std::vector<uint32_t> tab;
        std::vector<int32_t> off;
        std::vector<float> temp;
        int rc = build_table(*S, tab, off, temp, ecap, max_row);
        if (rc) return rc;
        if (c->annealed) {
            e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
        }
        e = c->tab.alloc(tab.size());
        if (e == cudaSuccess) e = c->tab_off.alloc(off.size());
        if (e == cudaSuccess) e = c->temp.alloc(temp.size());
        if (e != cudaSuccess) return fail(GDI_ERR_OOM, "device allocation failed (table)");
        if (c->h_tab_n < tab.size() || c->h_off_n < off.size()) {
            if (c->h_tab) cudaFreeHost(c->h_tab);
            if (c->h_off) cudaFreeHost(c->h_off);
            if (c->h_temp) cudaFreeHost(c->h_temp);
            c->h_tab = nullptr; c->h_off = nullptr; c->h_temp = nullptr;
            c->h_tab_n = c->h_off_n = 0;
            e = cudaMallocHost((void **)&c->h_tab, std::max<size_t>(tab.size(), 1) * sizeof(uint32_t));
            if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_off, off.size() * sizeof(int32_t));
            if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_temp, off.size() * sizeof(float));
            if (e != cudaSuccess) return fail(GDI_ERR_OOM, "pinned host allocation failed");
            c->h_tab_n = std::max<size_t>(tab.size(), 1);
            c->h_off_n = off.size();
        }
        std::memcpy(c->h_tab, tab.data(), tab.size() * sizeof(uint32_t));
        std::memcpy(c->h_off, off.data(), off.size() * sizeof(int32_t));
        std::memcpy(c->h_temp, temp.data(), temp.size() * sizeof(float));
        e = cudaMemcpyAsync(c->tab.p, c->h_tab, tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->tab_off.p, c->h_off, off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->temp.p, c->h_temp, temp.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { c->tab_valid = false; return cuda_fail(e, "table upload"); }
        c->tab_valid = true;
        c->tab_sched = *S;
        c->tab_ecap = ecap;
        c->tab_max_row = max_row;
    }
    // integer ranges: |B h + 4A - E*| and |G| must stay far below the 2^30 threshold sentinels
    if ((int64_t)c->B * c->max_degree + 4LL * c->A + ecap >= ((int64_t)1 << 29))
        return fail(GDI_ERR_OVERFLOW, "B * max_degree + 4A + E_cap must stay below 2^29");

    const bool trace = (run->flags & GDI_FLAG_TRACE) != 0;
    const size_t items = (size_t)c->Q * c->R;
    if (trace) {
        e = c->tr_digest.alloc(items * S->sweeps);
        if (e == cudaSuccess) e = c->tr_G.alloc(items * S->sweeps);
        if (e == cudaSuccess) e = c->tr_cut.alloc(items * S->sweeps);
        if (e != cudaSuccess) return fail(GDI_ERR_OOM, "device allocation failed (trace)");
        cudaMemsetAsync(c->tr_digest.p, 0, items * S->sweeps * sizeof(uint64_t), st);
        cudaMemsetAsync(c->tr_G.p, 0, items * S->sweeps * sizeof(int32_t), st);
        cudaMemsetAsync(c->tr_cut.p, 0, items * S->sweeps * sizeof(int64_t), st);
    }
    const GdiDevProblem P = c->problem();
    const uint32_t key0 = (uint32_t)run->seed, key1 = (uint32_t)(run->seed >> 32);
    if (!cont) {
        const int8_t *init = nullptr;
        if (run->init_spins) {
            const size_t bytes = (size_t)c->R * (size_t)c->N;
            if (run->init_mem == GDI_MEM_DEVICE) {
                init = run->init_spins;
            } else {
                e = c->init_stage.alloc(bytes);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(c->init_stage.p, run->init_spins, bytes, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) return cuda_fail(e, "init spins upload");
                init = c->init_stage.p;
            }
        }
        int ke = gdi_launch_init(P, c->spins.p, init, init ? 1 : 0, key0, key1, st);
        if (ke) return cuda_fail((cudaError_t)ke, "init kernel");
    }

    GdiDevRun R;
    R.spins = c->spins.p;
    R.tab = c->tab.p;
    R.tab_off = c->tab_off.p;
    R.temp = c->temp.p;
    R.mode = S->mode;
    R.sweeps = S->sweeps;
    R.s_begin = s_begin;
    R.s_end = s_end;
    R.max_row = max_row;
    R.key0 = key0;
    R.key1 = key1;
    R.flags = (trace ? GDI_DEV_TRACE : 0) | ((run->flags & GDI_FLAG_NO_REPAIR) ? GDI_DEV_NO_REPAIR : 0) |
              ((run->flags & GDI_FLAG_RACY) ? GDI_DEV_RACY : 0) |
              ((run->flags & GDI_FLAG_STANDARD) ? GDI_DEV_STANDARD : 0);
    R.raw_G = c->raw_G.p;
    R.final_G = c->final_G.p;
    R.raw_cut = c->raw_cut.p;
    R.final_cut = c->final_cut.p;
    R.tr_digest = trace ? c->tr_digest.p : nullptr;
    R.tr_G = trace ? c->tr_G.p : nullptr;
    R.tr_cut = trace ? c->tr_cut.p : nullptr;
    R.err = c->err.p;
    R.item_order = c->item_order.p;
    R.item_counter = c->item_counter.p;

    size_t need = 0;
    int H = 0;
    gdi_cta_smem_bytes(P, R, c->block, &need, &H);
    int max_optin = 0, sms = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    bool grid = false;
    if ((run->flags & GDI_FLAG_STANDARD) && ((run->flags & GDI_FLAG_RACY) || c->path == GDI_PATH_GRID))
        return fail(GDI_ERR_INVALID_ARG, "GDI_FLAG_STANDARD runs on the CTA-resident path only");
    if (c->path == GDI_PATH_GRID || (run->flags & GDI_FLAG_RACY)) grid = true;
    else if (run->flags & GDI_FLAG_STANDARD) grid = false;
    else if (c->path == GDI_PATH_AUTO && c->Q == 1 && c->W >= 1 && c->max_degree <= 32767) {
        // one instance: the cheaper path by a cost model fitted on GB300 (BA graphs, m = 5, of
        // 2*10^3 to 6.4*10^4 vertices; ER graphs of 800 vertices at mean degree 49 and 1.6*10^4 at
        // 10; 1 to 152 replicas; 100 sweeps).  Per sweep, a CTA-resident block costs about 2 us
        // per colour class + 1.8 ns (blocks of 128 or 256 threads) or 1.2 ns (512, 1024) per
        // (vertex + directed edge), per wave of resident blocks; a grid-scale launch costs about
        // 13 us per colour class (thresholds, sort, chain and barrier) + 0.02 ns per (vertex +
        // edge), per group of 8 replicas.
        int per_sm = 0;
        if (need > (size_t)max_optin || gdi_cta_blocks_per_sm(P, R, c->block, &per_sm) != 0 || per_sm < 1) {
            grid = true;
        } else {
            const double work = (double)c->N + (double)c->nnz;
            const double ncls = (double)c->num_classes[0];
            const int64_t slots = (int64_t)sms * per_sm;
            const double per_work = c->block >= 512 ? 1.2e-9 : 1.8e-9;
            const double cta_s = (double)((c->R + slots - 1) / slots) * (2e-6 * ncls + per_work * work);
            const double grid_s = (double)((c->R + 7) / 8) * (13e-6 * ncls + 0.02e-9 * work);
            grid = grid_s < cta_s;
        }
    }
    // kernel timing events (not while the stream is being captured into a graph)
    GdiKernelTimer timer{nullptr, 0, 0};
    c->kev_pairs = 0;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            const size_t want = 2 * (size_t)std::max(1, (c->R + 7) / 8);
            while (c->kev.size() < want) {
                cudaEvent_t ev;
                if (cudaEventCreate(&ev) != cudaSuccess) break;
                c->kev.push_back(ev);
            }
            if (c->kev.size() >= want) timer = GdiKernelTimer{c->kev.data(), (int)(c->kev.size() / 2), 0};
        }
        cudaGetLastError();
    }
    if (!grid) {
        cudaMemsetAsync(c->item_counter.p, 0, sizeof(int32_t), st);
        cudaMemsetAsync(c->err.p, 0, sizeof(int32_t), st);
        if (need > (size_t)max_optin)
            return fail(GDI_ERR_TOO_LARGE, "instance needs " + std::to_string(need) +
                                               " bytes of shared memory per block (limit " +
                                               std::to_string(max_optin) + "); use one instance with W > 0");
        if (timer.ev) cudaEventRecord(timer.ev[0], st);
        int ke = gdi_launch_cta_anneal(P, R, c->block, c->grid_limit, st, &c->last_grid, &c->last_smem);
        if (ke) return cuda_fail((cudaError_t)ke, "anneal kernel launch");
        if (timer.ev) {
            cudaEventRecord(timer.ev[1], st);
            timer.n = 1;
        }
        c->used_grid = false;
    } else {
        if (c->Q != 1 || c->W < 1)
            return fail(GDI_ERR_TOO_LARGE, "the grid-scale path anneals one instance with a window W >= 1");
        if (c->max_degree > 32767) return fail(GDI_ERR_TOO_LARGE, "degree above 32767 on the grid-scale path");
        int spc = 0, wpc = 0;
        size_t smem = 0;
        const int nblk = c->grid_limit > 0 ? std::min(c->grid_limit, sms) : sms;
        if (gdi_grid_plan(P, max_row, nblk, (size_t)max_optin, &spc, &wpc, &smem) != 0)
            return fail(GDI_ERR_TOO_LARGE, "grid-scale plan needs " + std::to_string(smem) +
                                               " bytes of shared memory per block; use a smaller W");
        const int D = c->max_degree;
        e = c->g_packed.alloc((size_t)c->N);
        if (e == cudaSuccess) e = c->g_rflags.alloc((size_t)c->N);
        if (e == cudaSuccess) e = c->g_tables.alloc((size_t)nblk * 8 * GDI_GRID_TW);
        if (e == cudaSuccess) e = c->g_gin.alloc((size_t)nblk * 8);
        if (e == cudaSuccess) e = c->g_Gcls.alloc(8);
        if (e == cudaSuccess) e = c->g_err.alloc(4);
        if (e == cudaSuccess) e = c->g_status.alloc(16);
        if (e == cudaSuccess) e = c->g_rhist.alloc((size_t)8 * (2 * D + 1));
        if (e == cudaSuccess) e = c->g_rties.alloc((size_t)8 * 152 * 4);
        if (e == cudaSuccess) e = c->g_rparams.alloc(32);
        if (e == cudaSuccess) e = c->g_bar.alloc(4);
        if (e == cudaSuccess && c->W <= 256) e = c->g_hfield.alloc((size_t)2 * c->N);
        if (e != cudaSuccess) return fail(GDI_ERR_OOM, "device allocation failed (grid scratch)");
        cudaMemsetAsync(c->g_err.p, 0, sizeof(int32_t), st);
        cudaMemsetAsync(c->g_status.p, 0, 16 * sizeof(int32_t), st);
        GdiGridScratch X = c->grid_scratch();
        if (c->inject_limit > 0) {               // no barrier can complete: every wait runs out
            X.spin_limit = c->inject_limit;
            X.bar_start = (unsigned int)nblk;
            c->inject_limit = 0;
        }
        const int32_t *wbnd = nullptr;
        if (c->W <= 256 && !c->wcost_off.empty()) {
            if (c->wbnd_blocks != nblk || c->wbnd_wpc != wpc) {
                const int ncls = (int)c->wcost_off.size() - 1;
                std::vector<int32_t> bnd((size_t)ncls * (nblk + 1));
                gdi_grid_window_bounds(c->wcost.data(), c->wcost_off.data(), ncls, nblk, wpc, bnd.data());
                e = c->g_wbnd.alloc(bnd.size());
                if (e == cudaSuccess) e = cudaMemcpy(c->g_wbnd.p, bnd.data(), bnd.size() * sizeof(int32_t),
                                                     cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return cuda_fail(e, "window bounds");
                c->wbnd_blocks = nblk;
                c->wbnd_wpc = wpc;
            }
            wbnd = c->g_wbnd.p;
        }
        int ke = gdi_launch_grid_anneal(P, R, X, c->spins.p, nblk, spc, wpc, smem, wbnd, &timer, st);
        if (ke) return cuda_fail((cudaError_t)ke, "grid anneal launch");
        ke = gdi_launch_grid_finish(P, R, X, c->spins.p, (run->flags & GDI_FLAG_NO_REPAIR) ? 0 : 1, st);
        if (ke) return cuda_fail((cudaError_t)ke, "grid finish kernels");
        c->used_grid = true;
        c->last_grid = nblk;
        c->last_smem = smem;
    }
    c->kev_pairs = timer.n;
    c->stream = st;
    c->annealed = true;
    c->last_sweeps = S->sweeps;
    c->last_flags = run->flags;
    c->ecap = ecap;
    return GDI_OK;
}

static int sync_ctx(gdi_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (c->used_grid) {
        int32_t err = 0;
        e = cudaMemcpy(&err, c->g_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "error word");
        if (err == GDI_DEVERR_TIMEOUT) return fail(GDI_ERR_TIMEOUT, "a grid barrier wait ran out");
        if (err) return fail(GDI_ERR_CUDA, "device error word " + std::to_string(err));
    } else {
        int32_t err = 0;
        e = cudaMemcpy(&err, c->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "error word");
        if (err) return fail(GDI_ERR_CUDA, "device error word " + std::to_string(err));
    }
    return GDI_OK;
}

int gdi_get_spins(gdi_ctx *c, int8_t *out, int32_t out_mem)
{
    if (!c || !out) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    const size_t bytes = (size_t)c->R * (size_t)c->N;
    int8_t *dst = out;
    if (out_mem != GDI_MEM_DEVICE) {
        cudaError_t e = c->out_stage.alloc(bytes);
        if (e != cudaSuccess) return fail(GDI_ERR_OOM, "device allocation failed");
        dst = c->out_stage.p;
    }
    int ke = gdi_launch_gather_spins(c->problem(), c->spins.p, dst, c->stream);
    if (ke) return cuda_fail((cudaError_t)ke, "gather kernel");
    if (out_mem != GDI_MEM_DEVICE) {
        cudaError_t e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "spins download");
    }
    return sync_ctx(c);
}

int gdi_get_results(gdi_ctx *c, int32_t *raw_G, int32_t *final_G, int64_t *raw_cut, int64_t *final_cut)
{
    if (!c) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    int rc = sync_ctx(c);
    if (rc) return rc;
    const size_t items = (size_t)c->Q * c->R;
    cudaError_t e = cudaSuccess;
    if (raw_G && e == cudaSuccess) e = cudaMemcpy(raw_G, c->raw_G.p, items * 4, cudaMemcpyDeviceToHost);
    if (final_G && e == cudaSuccess) e = cudaMemcpy(final_G, c->final_G.p, items * 4, cudaMemcpyDeviceToHost);
    if (raw_cut && e == cudaSuccess) e = cudaMemcpy(raw_cut, c->raw_cut.p, items * 8, cudaMemcpyDeviceToHost);
    if (final_cut && e == cudaSuccess) e = cudaMemcpy(final_cut, c->final_cut.p, items * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "results download");
    return GDI_OK;
}

int gdi_cut(gdi_ctx *c, int32_t instance, int32_t replica, int64_t *cut_out)
{
    if (!c || !cut_out || instance < 0 || instance >= c->Q || replica < 0 || replica >= c->R)
        return fail(GDI_ERR_INVALID_ARG, "bad instance/replica");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    int rc = sync_ctx(c);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(cut_out, c->final_cut.p + (size_t)instance * c->R + replica, 8,
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GDI_OK : cuda_fail(e, "cut download");
}

int gdi_balance(gdi_ctx *c, int32_t instance, int32_t replica, int32_t *raw_G, int32_t *final_G)
{
    if (!c || instance < 0 || instance >= c->Q || replica < 0 || replica >= c->R)
        return fail(GDI_ERR_INVALID_ARG, "bad instance/replica");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    int rc = sync_ctx(c);
    if (rc) return rc;
    const size_t i = (size_t)instance * c->R + replica;
    cudaError_t e = cudaSuccess;
    if (raw_G) e = cudaMemcpy(raw_G, c->raw_G.p + i, 4, cudaMemcpyDeviceToHost);
    if (final_G && e == cudaSuccess) e = cudaMemcpy(final_G, c->final_G.p + i, 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GDI_OK : cuda_fail(e, "balance download");
}

int gdi_get_trace(gdi_ctx *c, uint64_t *digest, int32_t *G, int64_t *cut)
{
    if (!c) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    if (!(c->last_flags & GDI_FLAG_TRACE)) return fail(GDI_ERR_INVALID_ARG, "last anneal had no GDI_FLAG_TRACE");
    int rc = sync_ctx(c);
    if (rc) return rc;
    const size_t cnt = (size_t)c->Q * c->R * c->last_sweeps;
    cudaError_t e = cudaSuccess;
    if (digest) e = cudaMemcpy(digest, c->tr_digest.p, cnt * 8, cudaMemcpyDeviceToHost);
    if (G && e == cudaSuccess) e = cudaMemcpy(G, c->tr_G.p, cnt * 4, cudaMemcpyDeviceToHost);
    if (cut && e == cudaSuccess) e = cudaMemcpy(cut, c->tr_cut.p, cnt * 8, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GDI_OK : cuda_fail(e, "trace download");
}

int gdi_configure(gdi_ctx *c, int32_t path, int32_t block, int32_t grid_limit)
{
    if (!c) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (path < GDI_PATH_AUTO || path > GDI_PATH_GRID) return fail(GDI_ERR_INVALID_ARG, "unknown path");
    if (block != 0 && block != 128 && block != 256 && block != 512 && block != 1024)
        return fail(GDI_ERR_INVALID_ARG, "block must be 0, 128, 256, 512 or 1024");
    if (grid_limit < 0) return fail(GDI_ERR_INVALID_ARG, "grid_limit must be >= 0");
    c->path = path;
    if (block) c->block = block;
    c->grid_limit = grid_limit;
    return GDI_OK;
}

int gdi_autotune(gdi_ctx *c, const gdi_schedule *S, int32_t probe_sweeps, int32_t *block_out,
                 int32_t *grid_out, float *ms_out)
{
    if (!c || !S) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (probe_sweeps < 1 || probe_sweeps > S->sweeps) return fail(GDI_ERR_INVALID_ARG, "probe_sweeps outside the schedule");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune setup");
    gdi_run run{};
    run.seed = 0x5eedULL;
    run.last_sweep = probe_sweeps;
    run.flags = GDI_FLAG_NO_REPAIR;
    run.stream = st;
    // a first probe (also the warm-up) shows which path the current settings take; a CTA block
    // that does not fit leaves the choice to the block-size candidates
    int rc = gdi_anneal(c, S, &run);
    bool grid_path = false;
    if (rc == GDI_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "autotune probe");
        grid_path = c->used_grid;
    } else if (rc == GDI_ERR_TOO_LARGE) {
        rc = GDI_OK;
    }
    if (rc != GDI_OK) {
        cudaStreamSynchronize(st);
        c->stream = nullptr;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(st);
        return rc;
    }
    // candidate launch configurations: (block, grid cap); the grid path ignores the block size
    std::vector<std::pair<int, int>> cand;
    if (grid_path) {
        for (int g : {sms, (sms * 3) / 4, sms / 2}) cand.push_back({c->block, g});
    } else {
        for (int b : {128, 256, 512, 1024})
            for (int g : {0, sms}) cand.push_back({b, g});
    }
    const int keep_block = c->block, keep_grid = c->grid_limit;
    float best = 1e30f;
    int best_b = keep_block, best_g = keep_grid;
    for (const auto &cg : cand) {
        c->block = cg.first;
        c->grid_limit = cg.second;
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && rc == GDI_OK; ++rep) {
            cudaEventRecord(e0, st);
            rc = gdi_anneal(c, S, &run);
            cudaEventRecord(e1, st);
            if (rc != GDI_OK) break;
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep == 1) ms = t;
        }
        if (rc == GDI_ERR_TOO_LARGE) { rc = GDI_OK; continue; }   // a block size that does not fit
        if (rc != GDI_OK) break;
        if (ms < best) { best = ms; best_b = cg.first; best_g = cg.second; }
    }
    cudaStreamSynchronize(st);
    c->stream = nullptr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc != GDI_OK) { c->block = keep_block; c->grid_limit = keep_grid; return rc; }
    c->block = best_b;
    c->grid_limit = best_g;
    if (block_out) *block_out = best_b;
    if (grid_out) *grid_out = best_g;
    if (ms_out) *ms_out = best;
    return GDI_OK;
}

int gdi_last_launch(gdi_ctx *c, int32_t *path, int32_t *grid, int64_t *smem_bytes, int32_t *fallbacks)
{
    if (!c) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    int rc = sync_ctx(c);
    if (rc) return rc;
    if (path) *path = c->used_grid ? GDI_PATH_GRID : GDI_PATH_CTA;
    if (grid) *grid = c->last_grid;
    if (smem_bytes) *smem_bytes = (int64_t)c->last_smem;
    if (fallbacks) {
        *fallbacks = 0;
        if (c->used_grid) {
            int32_t st[16];
            cudaError_t e = cudaMemcpy(st, c->g_status.p, sizeof st, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "status");
            for (int i = 0; i < 8; ++i) *fallbacks += st[i];
        }
    }
    return GDI_OK;
}

int gdi_inject_wait_failure(gdi_ctx *c, int64_t spin_limit)
{
    if (!c || spin_limit < 1) return fail(GDI_ERR_INVALID_ARG, "need a context and spin_limit >= 1");
    c->inject_limit = spin_limit;
    return GDI_OK;
}

int gdi_kernel_time(gdi_ctx *c, float *ms, int32_t *launches)
{
    if (!c || !ms) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (!c->annealed) return fail(GDI_ERR_NOT_ANNEALED, "no anneal yet");
    int rc = sync_ctx(c);
    if (rc) return rc;
    if (c->kev_pairs < 1) return fail(GDI_ERR_NOT_ANNEALED, "the last anneal was not timed (captured into a graph)");
    float total = 0.f;
    for (int i = 0; i < c->kev_pairs; ++i) {
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, c->kev[(size_t)2 * i], c->kev[(size_t)2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "kernel events");
        total += t;
    }
    *ms = total;
    if (launches) *launches = c->kev_pairs;
    return GDI_OK;
}

int gdi_info(gdi_ctx *c, int32_t *num_classes, int32_t *max_degree, int32_t *ecap)
{
    if (!c) return fail(GDI_ERR_INVALID_ARG, "null argument");
    if (num_classes) std::memcpy(num_classes, c->num_classes.data(), c->num_classes.size() * 4);
    if (max_degree) *max_degree = c->max_degree;
    if (ecap) *ecap = c->ecap;
    return GDI_OK;
}

void gdi_destroy(gdi_ctx *c)
{
    if (!c) return;
    if (c->annealed) cudaStreamSynchronize(c->stream);
    c->release();
    delete c;
}

const char *gdi_strerror(int code)
{
    switch (code) {
    case GDI_OK: return "ok";
    case GDI_ERR_INVALID_ARG: return "invalid argument";
    case GDI_ERR_NOT_SYMMETRIC: return "CSR is not symmetric";
    case GDI_ERR_SELF_LOOP: return "self-loop";
    case GDI_ERR_DUP_EDGE: return "duplicate edge";
    case GDI_ERR_BAD_COLORING: return "colouring is not proper";
    case GDI_ERR_OVERFLOW: return "integer range exceeded";
    case GDI_ERR_OOM: return "out of memory";
    case GDI_ERR_CUDA: return "CUDA error";
    case GDI_ERR_TIMEOUT: return "device wait timed out";
    case GDI_ERR_NOT_ANNEALED: return "no anneal has run";
    case GDI_ERR_TOO_LARGE: return "problem too large for the kernels";
    default: return "unknown error";
    }
}

const char *gdi_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
