// C ABI of the GTQA hot path: state management, graph bookkeeping, launch
// sequencing.  Declarations and argument contracts are in include/gtqa.h.
#include "gtqa.h"
#include "gtqa_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace gtqa;

struct gtqa_state {
    int B = 0, n = 0, m = 0;
    int chi = 0, CHI = 0;
    int precision = GTQA_FP64;
    cudaStream_t stream = nullptr;
    double svd_cutoff = 1e-14, eig_cutoff = 1e-13;
    int ncol = 0;
    std::vector<int> colour_off;        // [ncol + 1] ranges in colour_edges
    std::vector<int> h_inst_vbeg;       // [B + 1]
    std::vector<int> h_inst_m;          // [B]
    std::vector<int4> h_edge_info;
    // device buffers
    void* Gamma = nullptr;
    double* lam = nullptr;
    cd* msg[2] = {nullptr, nullptr};
    int cur = 0;
    cd* T = nullptr;
    cd* X = nullptr;
    int4* edge_info = nullptr;
    int4* vert_edges = nullptr;
    int* vert_inst = nullptr;
    int* edge_inst = nullptr;
    double* J = nullptr;
    double* h = nullptr;
    int* colour_edges = nullptr;
    double* disc = nullptr;
    int2* work = nullptr;               // per edge: core-SVD sweeps and rotations of the last gate
    double* stats = nullptr;            // [4]: discarded weight, log fidelity, SVD pairs, SVD rotations
    double* vdelta = nullptr;
    int* inst_vbeg = nullptr;
    int* inst_m = nullptr;
    int* inst_done = nullptr;
    int* inst_iters = nullptr;
    double* inst_dist = nullptr;
    int* flags = nullptr;               // [0] all done, [1] NaN in BP, [2] NaN in marginals
    cd* rho = nullptr;
    int8_t* sign = nullptr;
    int* h_flags = nullptr;             // pinned mirror of flags
    // counters
    long long layers = 0, gates = 0, bp_sweeps = 0, launches = 0;
    // optional profiler: pending event pairs and accumulated figures per kernel class
    bool prof_on = false;
    struct Pending { int kind; cudaEvent_t a, b; long long units; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[GTQA_K_COUNT] = {};
    long long prof_launches[GTQA_K_COUNT] = {};
    long long prof_units[GTQA_K_COUNT] = {};
    int last_iters = 0, not_conv = 0;
    double last_dist = 0.0;
    int sticky = GTQA_OK;
};

namespace {

bool cuda_ok(gtqa_state* s, cudaError_t e) {
    if (e != cudaSuccess) {
        if (s) s->sticky = GTQA_ERR_CUDA;
        return false;
    }
    return true;
}

int launch_check(gtqa_state* s) {
    if (!cuda_ok(s, cudaGetLastError())) return GTQA_ERR_CUDA;
    s->launches += 1;
    return GTQA_OK;
}

cudaEvent_t prof_event(gtqa_state* s) {
    if (!s->pool.empty()) {
        cudaEvent_t e = s->pool.back();
        s->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Bracket one launch with events when the profiler is on.
struct ProfScope {
    gtqa_state* s;
    int kind;
    long long units;
    cudaEvent_t a = nullptr;
    ProfScope(gtqa_state* st, int k, long long u) : s(st), kind(k), units(u) {
        if (s->prof_on) {
            a = prof_event(s);
            if (a) cudaEventRecord(a, s->stream);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = prof_event(s);
        if (!b) return;
        cudaEventRecord(b, s->stream);
        s->pending.push_back({kind, a, b, units});
    }
};

void prof_collect(gtqa_state* s) {
    for (auto& p : s->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            s->prof_ms[p.kind] += ms;
            s->prof_launches[p.kind] += 1;
            s->prof_units[p.kind] += p.units;
        }
        s->pool.push_back(p.a);
        s->pool.push_back(p.b);
    }
    s->pending.clear();
}

template <typename T>
int dalloc(gtqa_state* s, T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        s->sticky = GTQA_ERR_OOM;
        return GTQA_ERR_OOM;
    }
    if (e != cudaSuccess) {
        s->sticky = GTQA_ERR_CUDA;
        return GTQA_ERR_CUDA;
    }
    return GTQA_OK;
}

int storage_chi(int chi) {
    if (chi <= 2) return 2;
    if (chi <= 4) return 4;
    if (chi <= 8) return 8;
    return 0;
}

size_t gamma_elems(const gtqa_state* s) { return (size_t)s->n * 2 * s->CHI * s->CHI * s->CHI; }
size_t msg_elems(const gtqa_state* s) { return (size_t)s->m * 2 * s->CHI * s->CHI; }

GraphView view(const gtqa_state* s) {
    GraphView g;
    g.edge_info = s->edge_info;
    g.vert_edges = s->vert_edges;
    g.vert_inst = s->vert_inst;
    g.edge_inst = s->edge_inst;
    g.J = s->J;
    g.h = s->h;
    g.n = s->n;
    g.m = s->m;
    return g;
}

int grid_for(size_t work, int tpb) {
    size_t b = (work + tpb - 1) / tpb;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Misra-Gries proper edge colouring with at most Delta + 1 colours.
bool misra_gries(int n, int m, const int* edges, std::vector<int>& colour, int& ncol) {
    std::vector<int> deg(n, 0);
    for (int e = 0; e < m; ++e) {
        deg[edges[2 * e]]++;
        deg[edges[2 * e + 1]]++;
    }
    int dmax = 0;
    for (int v = 0; v < n; ++v) dmax = deg[v] > dmax ? deg[v] : dmax;
    const int C = dmax + 1;
    std::vector<int> at((size_t)n * C, -1);     // neighbour reached by colour c
    std::vector<int> atE((size_t)n * C, -1);    // edge id of that colour at v
    colour.assign(m, -1);
    auto is_free = [&](int v, int c) { return at[(size_t)v * C + c] < 0; };
    auto set_col = [&](int e, int c) {
        const int u = edges[2 * e], v = edges[2 * e + 1];
        const int old = colour[e];
        if (old >= 0) {
            at[(size_t)u * C + old] = -1; atE[(size_t)u * C + old] = -1;
            at[(size_t)v * C + old] = -1; atE[(size_t)v * C + old] = -1;
        }
        colour[e] = c;
        if (c >= 0) {
            at[(size_t)u * C + c] = v; atE[(size_t)u * C + c] = e;
            at[(size_t)v * C + c] = u; atE[(size_t)v * C + c] = e;
        }
    };
    // edge lookup u -> list of (nbr, edge)
    std::vector<std::vector<std::pair<int, int>>> adj(n);
    for (int e = 0; e < m; ++e) {
        adj[edges[2 * e]].push_back({edges[2 * e + 1], e});
        adj[edges[2 * e + 1]].push_back({edges[2 * e], e});
    }
    auto edge_of = [&](int u, int v) {
        for (auto& p : adj[u]) if (p.first == v) return p.second;
        return -1;
    };
    for (int e = 0; e < m; ++e) {
        const int u = edges[2 * e], v = edges[2 * e + 1];
        std::vector<int> fan{v};
        std::vector<char> used(n, 0);
        used[v] = 1;
        for (;;) {
            const int last = fan.back();
            int nxt = -1;
            for (int c = 0; c < C && nxt < 0; ++c) {
                if (!is_free(last, c)) continue;
                const int w = at[(size_t)u * C + c];
                if (w >= 0 && !used[w]) nxt = w;
            }
            if (nxt < 0) break;
            fan.push_back(nxt);
            used[nxt] = 1;
        }
        int c = -1, d = -1;
        for (int q = 0; q < C && c < 0; ++q) if (is_free(u, q)) c = q;
        for (int q = 0; q < C && d < 0; ++q) if (is_free(fan.back(), q)) d = q;
        if (c < 0 || d < 0) return false;
        if (!is_free(u, d)) {
            // invert the path from u alternating colours d, c
            std::vector<int> pe;
            int cur = u, col = d;
            while (at[(size_t)cur * C + col] >= 0) {
                const int ed = atE[(size_t)cur * C + col];
                pe.push_back(ed);
                cur = at[(size_t)cur * C + col];
                col = (col == d) ? c : d;
                if ((int)pe.size() > m) return false;
            }
            std::vector<int> pc(pe.size());
            for (size_t i = 0; i < pe.size(); ++i) pc[i] = colour[pe[i]];
            for (size_t i = 0; i < pe.size(); ++i) set_col(pe[i], -1);
            for (size_t i = 0; i < pe.size(); ++i) set_col(pe[i], pc[i] == c ? d : c);
        }
        int widx = -1;
        for (size_t i = 0; i < fan.size() && widx < 0; ++i) {
            if (!is_free(fan[i], d)) continue;
            bool ok = true;
            for (size_t j = 1; j <= i && ok; ++j) {
                const int cj = colour[edge_of(u, fan[j])];
                if (cj < 0 || !is_free(fan[j - 1], cj)) ok = false;
            }
            if (ok) widx = (int)i;
        }
        if (widx < 0) return false;
        for (int j = 0; j < widx; ++j) {
            const int ej = edge_of(u, fan[j + 1]);
            const int cj = colour[ej];
            set_col(ej, -1);
            set_col(edge_of(u, fan[j]), cj);
        }
        set_col(edge_of(u, fan[widx]), d);
    }
    ncol = 0;
    for (int e = 0; e < m; ++e) {
        if (colour[e] < 0) return false;
        ncol = colour[e] + 1 > ncol ? colour[e] + 1 : ncol;
    }
    return true;
}

void free_state(gtqa_state* s) {
    if (!s) return;
    void* ptrs[] = {s->Gamma, s->lam, s->msg[0], s->msg[1], s->T, s->X, s->edge_info, s->vert_edges,
                    s->vert_inst, s->edge_inst, s->J, s->h, s->colour_edges, s->disc, s->stats, s->vdelta,
                    s->inst_vbeg, s->inst_m, s->inst_done, s->inst_iters, s->inst_dist, s->flags, s->rho,
                    s->sign};
    for (void* p : ptrs) if (p) cudaFree(p);
    if (s->work) cudaFree(s->work);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    for (auto& p : s->pending) {
        s->pool.push_back(p.a);
        s->pool.push_back(p.b);
    }
    for (cudaEvent_t e : s->pool) cudaEventDestroy(e);
    delete s;
}

// --------------------------------------------------------------------------
// launch sequences (templated on the storage bond dimension)
// --------------------------------------------------------------------------
template <int CHI, typename TS>
int set_kernel_attrs() {
    static bool done = false;
    if (done) return GTQA_OK;
    cudaError_t e1 = cudaFuncSetAttribute(gate_kernel<CHI, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(GateSmem<CHI>) * GateShape<CHI>::TEAMS));
    cudaError_t e2 = cudaFuncSetAttribute(bp_sweep_kernel<CHI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(BPSmem<CHI>) * BPShape<CHI>::TEAMS));
    if (e1 != cudaSuccess || e2 != cudaSuccess) return GTQA_ERR_CUDA;
    done = true;
    return GTQA_OK;
}

template <int CHI, typename TS>
int trotter_layer_t(gtqa_state* s, double tZ, double tX) {
    if (set_kernel_attrs<CHI, TS>() != GTQA_OK) { s->sticky = GTQA_ERR_CUDA; return GTQA_ERR_CUDA; }
    using GS = GateShape<CHI>;
    GateArgs<TS> a;
    a.Gamma = (C<TS>*)s->Gamma;
    a.lam = s->lam;
    a.g = view(s);
    a.tZ = tZ;
    a.chi = s->chi;
    a.svd_cutoff = s->svd_cutoff;
    a.disc = s->disc;
    a.work = s->work;
    const size_t smem = sizeof(GateSmem<CHI>) * GS::TEAMS;
    for (int c = 0; c < s->ncol; ++c) {
        const int cnt = s->colour_off[c + 1] - s->colour_off[c];
        if (cnt == 0) continue;
        a.edge_list = s->colour_edges + s->colour_off[c];
        a.count = cnt;
        const int grid = (cnt + GS::TEAMS - 1) / GS::TEAMS;
        ProfScope ps(s, GTQA_K_GATE, cnt);
        gate_kernel<CHI, TS><<<grid, GS::TPB, smem, s->stream>>>(a);
        if (launch_check(s)) return GTQA_ERR_CUDA;
    }
    const size_t work = (size_t)s->n * CHI * CHI * CHI;
    {
        ProfScope ps(s, GTQA_K_MIXING, s->n);
        xrot_kernel<CHI, TS><<<grid_for(work, 256), 256, 0, s->stream>>>((C<TS>*)s->Gamma, s->n, tX);
        if (launch_check(s)) return GTQA_ERR_CUDA;
    }
    if (s->m > 0) {
        ProfScope ps(s, GTQA_K_LAYER_STATS, s->m);
        layer_stats_kernel<<<1, 256, 0, s->stream>>>(s->disc, s->work, s->m, (2 * CHI - 1) * CHI, s->stats);
        if (launch_check(s)) return GTQA_ERR_CUDA;
    }
    return GTQA_OK;
}

template <int CHI, typename TS>
int symmetric_t(gtqa_state* s) {
    const size_t work = (size_t)s->n * 2 * CHI * CHI * CHI;
    ProfScope ps(s, GTQA_K_SYMMETRIC, s->n);
    symmetric_kernel<CHI, TS><<<grid_for(work, 256), 256, 0, s->stream>>>((const C<TS>*)s->Gamma, s->lam, view(s), s->T);
    return launch_check(s);
}

template <int CHI, typename TS>
int bp_t(gtqa_state* s, double tol, int max_iter, unsigned flags, int* iters_out, double* dist_out) {
    if (set_kernel_attrs<CHI, TS>() != GTQA_OK) { s->sticky = GTQA_ERR_CUDA; return GTQA_ERR_CUDA; }
    if (symmetric_t<CHI, TS>(s)) return GTQA_ERR_CUDA;
    if (flags & GTQA_BP_WARM_START) {
        const size_t work = msg_elems(s);
        ProfScope ps(s, GTQA_K_WARM_START, s->m);
        warm_start_kernel<CHI><<<grid_for(work, 256), 256, 0, s->stream>>>(s->lam, s->m, s->msg[s->cur]);
        if (launch_check(s)) return GTQA_ERR_CUDA;
    }
    if (!cuda_ok(s, cudaMemsetAsync(s->inst_done, 0, sizeof(int) * s->B, s->stream))) return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaMemsetAsync(s->inst_iters, 0, sizeof(int) * s->B, s->stream))) return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaMemsetAsync(s->flags, 0, sizeof(int) * 4, s->stream))) return GTQA_ERR_CUDA;
    using BS = BPShape<CHI>;
    BPArgs a;
    a.T = s->T;
    a.vdelta = s->vdelta;
    a.inst_done = s->inst_done;
    a.g = view(s);
    ReduceArgs r;
    r.vdelta = s->vdelta;
    r.inst_vbeg = s->inst_vbeg;
    r.inst_m = s->inst_m;
    r.inst_done = s->inst_done;
    r.inst_iters = s->inst_iters;
    r.inst_dist = s->inst_dist;
    r.flags = s->flags;
    r.tol = tol;
    r.max_iter = max_iter;
    r.B = s->B;
    const size_t smem = sizeof(BPSmem<CHI>) * BS::TEAMS;
    const int grid = (s->n + BS::TEAMS - 1) / BS::TEAMS;
    for (int it = 0; it < max_iter; ++it) {
        a.src = s->msg[s->cur];
        a.dst = s->msg[s->cur ^ 1];
        {
            ProfScope ps(s, GTQA_K_BP_SWEEP, s->n);
            bp_sweep_kernel<CHI><<<grid, BS::TPB, smem, s->stream>>>(a);
            if (launch_check(s)) return GTQA_ERR_CUDA;
        }
        {
            ProfScope ps(s, GTQA_K_BP_REDUCE, s->n);
            bp_reduce_kernel<<<1, 256, 0, s->stream>>>(r);
            if (launch_check(s)) return GTQA_ERR_CUDA;
        }
        s->cur ^= 1;
        if (!cuda_ok(s, cudaMemcpyAsync(s->h_flags, s->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s->stream)))
            return GTQA_ERR_CUDA;
        if (!cuda_ok(s, cudaStreamSynchronize(s->stream))) return GTQA_ERR_CUDA;
        if (s->h_flags[1]) { s->sticky = GTQA_ERR_NUMERIC; return GTQA_ERR_NUMERIC; }
        if (s->h_flags[0]) break;
    }
    std::vector<int> iters(s->B), done(s->B);
    std::vector<double> dist(s->B);
    if (!cuda_ok(s, cudaMemcpyAsync(iters.data(), s->inst_iters, sizeof(int) * s->B, cudaMemcpyDeviceToHost, s->stream)))
        return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaMemcpyAsync(dist.data(), s->inst_dist, sizeof(double) * s->B, cudaMemcpyDeviceToHost, s->stream)))
        return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaStreamSynchronize(s->stream))) return GTQA_ERR_CUDA;
    int mi = 0, nc = 0;
    double md = 0.0;
    for (int b = 0; b < s->B; ++b) {
        mi = iters[b] > mi ? iters[b] : mi;
        md = dist[b] > md ? dist[b] : md;
        if (!(dist[b] < tol) && s->h_inst_m[b] > 0) nc++;
    }
    s->last_iters = mi;
    s->bp_sweeps += mi;
    s->last_dist = md;
    s->not_conv = nc;
    if (iters_out) *iters_out = mi;
    if (dist_out) *dist_out = md;
    return nc > 0 ? GTQA_ERR_NOT_CONVERGED : GTQA_OK;
}

template <int CHI, typename TS>
int regauge_t(gtqa_state* s) {
    if (s->m == 0) return GTQA_OK;
    using RS = RGShape<CHI>;
    RGArgs a;
    a.msg = s->msg[s->cur];
    a.X = s->X;
    a.lam = s->lam;
    a.m = s->m;
    a.eig_cutoff = s->eig_cutoff;
    a.svd_cutoff = s->svd_cutoff;
    {
        ProfScope ps(s, GTQA_K_REGAUGE_EDGE, s->m);
        regauge_edge_kernel<CHI><<<(s->m + RS::TEAMS - 1) / RS::TEAMS, RS::TPB, 0, s->stream>>>(a);
        if (launch_check(s)) return GTQA_ERR_CUDA;
    }
    ProfScope ps(s, GTQA_K_REGAUGE_VERTEX, s->n);
    regauge_vertex_kernel<CHI, TS><<<s->n, 128, 0, s->stream>>>(s->T, s->X, view(s), (C<TS>*)s->Gamma);
    return launch_check(s);
}

template <int CHI, typename TS>
int marginals_t(gtqa_state* s) {
    const int warps_per_block = 4;
    ProfScope ps(s, GTQA_K_MARGINALS, s->n);
    marginals_kernel<CHI, TS><<<(s->n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s->stream>>>(
        (const C<TS>*)s->Gamma, s->lam, view(s), s->rho, s->sign, s->flags + 2);
    return launch_check(s);
}

#define GTQA_DISPATCH(s, FN, ...)                                         \
    do {                                                                  \
        switch ((s)->CHI) {                                               \
            case 2: return FN<2, double>((s), ##__VA_ARGS__);             \
            case 4: return FN<4, double>((s), ##__VA_ARGS__);             \
            case 8: return FN<8, double>((s), ##__VA_ARGS__);             \
            default: return GTQA_ERR_UNSUPPORTED;                         \
        }                                                                 \
    } while (0)

int check_state(const gtqa_state* s) {
    if (!s) return GTQA_ERR_INVALID_ARG;
    return s->sticky;
}

int create_impl(int B, const int* n, const int* m, const int* edges, const int* colour, const double* J,
                const double* h, int chi, const gtqa_options* opt, gtqa_state** out) {
    if (!out) return GTQA_ERR_INVALID_ARG;
    *out = nullptr;
    if (B < 1 || !n || !m || !h || chi < 1) return GTQA_ERR_INVALID_ARG;
    if (storage_chi(chi) == 0) return GTQA_ERR_UNSUPPORTED;
    gtqa_options o;
    gtqa_options_init(&o);
    if (opt) o = *opt;
    if (o.precision != GTQA_FP64) return GTQA_ERR_UNSUPPORTED;
    if (o.reserved0 != 0) return GTQA_ERR_INVALID_ARG;
    long long N = 0, Mtot = 0;
    for (int b = 0; b < B; ++b) {
        if (n[b] < 1 || m[b] < 0) return GTQA_ERR_INVALID_ARG;
        N += n[b];
        Mtot += m[b];
    }
    if (N > (1LL << 30) || Mtot > (1LL << 30)) return GTQA_ERR_INVALID_ARG;
    if (Mtot > 0 && (!edges || !J)) return GTQA_ERR_INVALID_ARG;
    // validate and globalise the graph
    std::vector<int> ge((size_t)Mtot * 2), gcol((size_t)Mtot), vinst(N), einst(Mtot);
    std::vector<int> deg(N, 0);
    std::vector<int> vbeg(B + 1, 0), minst(B);
    int ncol = 0;
    {
        long long voff = 0, eoff = 0;
        for (int b = 0; b < B; ++b) {
            vbeg[b] = (int)voff;
            minst[b] = m[b];
            std::vector<long long> keys;
            keys.reserve(m[b]);
            for (int e = 0; e < m[b]; ++e) {
                const int u = edges[2 * (eoff + e)], v = edges[2 * (eoff + e) + 1];
                if (u < 0 || v < 0 || u >= n[b] || v >= n[b] || u == v) return GTQA_ERR_INVALID_ARG;
                if (!std::isfinite(J[eoff + e])) return GTQA_ERR_INVALID_ARG;
                const long long a = u < v ? u : v, c = u < v ? v : u;
                keys.push_back(a * n[b] + c);
                ge[2 * (eoff + e)] = (int)(u + voff);
                ge[2 * (eoff + e) + 1] = (int)(v + voff);
                einst[eoff + e] = b;
                if (++deg[u + voff] > 3 || ++deg[v + voff] > 3) return GTQA_ERR_INVALID_ARG;
            }
            std::vector<long long> sk = keys;
            std::sort(sk.begin(), sk.end());
            for (size_t i = 1; i < sk.size(); ++i) if (sk[i] == sk[i - 1]) return GTQA_ERR_INVALID_ARG;
            for (int a = 0; a < n[b]; ++a) {
                if (!std::isfinite(h[voff + a])) return GTQA_ERR_INVALID_ARG;
                vinst[voff + a] = b;
            }
            // colouring
            if (colour) {
                for (int e = 0; e < m[b]; ++e) {
                    const int c = colour[eoff + e];
                    if (c < 0 || c >= 64) return GTQA_ERR_INVALID_ARG;
                    gcol[eoff + e] = c;
                }
            } else {
                std::vector<int> col;
                int nc = 0;
                if (!misra_gries(n[b], m[b], edges + 2 * eoff, col, nc)) return GTQA_ERR_INVALID_ARG;
                for (int e = 0; e < m[b]; ++e) gcol[eoff + e] = col[e];
            }
            voff += n[b];
            eoff += m[b];
        }
        vbeg[B] = (int)voff;
        // each colour must be a matching
        std::vector<unsigned long long> seen((size_t)N, 0ull);
        for (long long e = 0; e < Mtot; ++e) {
            const unsigned long long bit = 1ull << gcol[e];
            for (int q = 0; q < 2; ++q) {
                const int v = ge[2 * e + q];
                if (seen[v] & bit) return GTQA_ERR_INVALID_ARG;
                seen[v] |= bit;
            }
            ncol = gcol[e] + 1 > ncol ? gcol[e] + 1 : ncol;
        }
    }
    gtqa_state* s = new (std::nothrow) gtqa_state();
    if (!s) return GTQA_ERR_OOM;
    s->B = B;
    s->n = (int)N;
    s->m = (int)Mtot;
    s->chi = chi;
    s->CHI = storage_chi(chi);
    s->precision = o.precision;
    s->stream = (cudaStream_t)o.cuda_stream;
    s->svd_cutoff = o.svd_cutoff > 0 ? o.svd_cutoff : 1e-14;
    s->eig_cutoff = o.eig_cutoff > 0 ? o.eig_cutoff : 1e-13;
    s->ncol = ncol;
    s->h_inst_vbeg = vbeg;
    s->h_inst_m = minst;
    // slots: incident edges in ascending id
    std::vector<int4> vedges(N, make_int4(-1, -1, -1, 0));
    std::vector<int4> einfo(Mtot);
    for (long long e = 0; e < Mtot; ++e) {
        int sl[2];
        for (int q = 0; q < 2; ++q) {
            const int v = ge[2 * e + q];
            int4& ve = vedges[v];
            int k = ve.w;
            if (k == 0) ve.x = (int)e; else if (k == 1) ve.y = (int)e; else ve.z = (int)e;
            sl[q] = k;
            ve.w = k + 1;
        }
        einfo[e] = make_int4(ge[2 * e], ge[2 * e + 1], sl[0], sl[1]);
    }
    s->h_edge_info = einfo;
    std::vector<int> cedges;
    cedges.reserve(Mtot);
    s->colour_off.assign(ncol + 1, 0);
    for (int c = 0; c < ncol; ++c) {
        s->colour_off[c] = (int)cedges.size();
        for (long long e = 0; e < Mtot; ++e) if (gcol[e] == c) cedges.push_back((int)e);
    }
    s->colour_off[ncol] = (int)cedges.size();
    // device allocations
    const int CHI = s->CHI;
    const size_t gel = gamma_elems(s), mel = msg_elems(s);
    const size_t rsz = sizeof(cd);
    int rc = GTQA_OK;
    if ((rc = dalloc(s, (unsigned char**)&s->Gamma, gel * rsz)) ||
        (rc = dalloc(s, &s->lam, (size_t)s->m * CHI)) || (rc = dalloc(s, &s->msg[0], mel)) ||
        (rc = dalloc(s, &s->msg[1], mel)) || (rc = dalloc(s, &s->T, gel)) ||
        (rc = dalloc(s, &s->X, (size_t)s->m * 2 * CHI * CHI)) || (rc = dalloc(s, &s->edge_info, s->m)) ||
        (rc = dalloc(s, &s->vert_edges, s->n)) || (rc = dalloc(s, &s->vert_inst, s->n)) ||
        (rc = dalloc(s, &s->edge_inst, s->m)) || (rc = dalloc(s, &s->J, s->m)) || (rc = dalloc(s, &s->h, s->n)) ||
        (rc = dalloc(s, &s->colour_edges, s->m)) || (rc = dalloc(s, &s->disc, s->m)) ||
        (rc = dalloc(s, &s->work, s->m)) || (rc = dalloc(s, &s->stats, 4)) || (rc = dalloc(s, &s->vdelta, s->n)) ||
        (rc = dalloc(s, &s->inst_vbeg, B + 1)) || (rc = dalloc(s, &s->inst_m, B)) ||
        (rc = dalloc(s, &s->inst_done, B)) || (rc = dalloc(s, &s->inst_iters, B)) ||
        (rc = dalloc(s, &s->inst_dist, B)) || (rc = dalloc(s, &s->flags, 4)) ||
        (rc = dalloc(s, &s->rho, (size_t)s->n * 4)) || (rc = dalloc(s, &s->sign, s->n))) {
        free_state(s);
        return rc;
    }
    if (cudaMallocHost((void**)&s->h_flags, sizeof(int) * 4) != cudaSuccess) {
        free_state(s);
        return GTQA_ERR_OOM;
    }
    // initial state |+>^N: Gamma[a][i][0][0][0] = 1/sqrt(2), lambda_e = (1, 0, ...)
    std::vector<cd> g0(gel, cd{0.0, 0.0});
    const size_t H = (size_t)CHI * CHI * CHI;
    for (long long a = 0; a < N; ++a) {
        g0[a * 2 * H] = cd{M_SQRT1_2, 0.0};
        g0[a * 2 * H + H] = cd{M_SQRT1_2, 0.0};
    }
    std::vector<double> l0((size_t)s->m * CHI, 0.0);
    for (long long e = 0; e < Mtot; ++e) l0[e * CHI] = 1.0;
    std::vector<double> Jv(Mtot), hv(N);
    for (long long e = 0; e < Mtot; ++e) Jv[e] = J[e];
    for (long long a = 0; a < N; ++a) hv[a] = h[a];
    cudaStream_t st = s->stream;
    bool ok = cuda_ok(s, cudaMemcpyAsync(s->Gamma, g0.data(), gel * rsz, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->lam, l0.data(), l0.size() * sizeof(double), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->msg[0], 0, mel * sizeof(cd), st)) &&
              cuda_ok(s, cudaMemsetAsync(s->msg[1], 0, mel * sizeof(cd), st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->edge_info, einfo.data(), sizeof(int4) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->vert_edges, vedges.data(), sizeof(int4) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->vert_inst, vinst.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->edge_inst, einst.data(), sizeof(int) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->J, Jv.data(), sizeof(double) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->h, hv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->colour_edges, cedges.data(), sizeof(int) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->disc, 0, sizeof(double) * (Mtot > 0 ? Mtot : 1), st)) &&
              cuda_ok(s, cudaMemsetAsync(s->stats, 0, sizeof(double) * 4, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->work, 0, sizeof(int2) * (Mtot > 0 ? Mtot : 1), st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->inst_vbeg, vbeg.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->inst_m, minst.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->flags, 0, sizeof(int) * 4, st)) &&
              cuda_ok(s, cudaStreamSynchronize(st));
    if (!ok) {
        free_state(s);
        return GTQA_ERR_CUDA;
    }
    *out = s;
    return GTQA_OK;
}

}  // namespace

extern "C" {

void gtqa_options_init(gtqa_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = GTQA_FP64;
    opt->svd_cutoff = 1e-14;
    opt->eig_cutoff = 1e-13;
    opt->cuda_stream = nullptr;
}

int gtqa_create(int32_t n, int32_t m, const int32_t* edges, const int32_t* colour, const double* J,
                const double* h, int32_t chi, const gtqa_options* opt, gtqa_state** out) {
    return create_impl(1, &n, &m, edges, colour, J, h, chi, opt, out);
}

int gtqa_create_batch(int32_t B, const int32_t* n, const int32_t* m, const int32_t* edges, const int32_t* colour,
                      const double* J, const double* h, int32_t chi, const gtqa_options* opt, gtqa_state** out) {
    return create_impl(B, n, m, edges, colour, J, h, chi, opt, out);
}

int gtqa_trotter_layer(gtqa_state* s, double tau, double dt) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!std::isfinite(tau) || !std::isfinite(dt)) return GTQA_ERR_INVALID_ARG;
    const double tZ = dt * tau, tX = dt * (1.0 - tau);
    rc = [&]() -> int { GTQA_DISPATCH(s, trotter_layer_t, tZ, tX); }();
    if (rc == GTQA_OK) {
        s->layers += 1;
        s->gates += s->m;
    }
    return rc;
}

int gtqa_bp_sweep(gtqa_state* s, double tol, int32_t max_iter, uint32_t flags, int32_t* iters_out,
                  double* dist_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (max_iter < 1 || !(tol >= 0.0) || (flags & ~3u)) return GTQA_ERR_INVALID_ARG;
    rc = [&]() -> int { GTQA_DISPATCH(s, bp_t, tol, max_iter, flags, iters_out, dist_out); }();
    if (rc != GTQA_OK && rc != GTQA_ERR_NOT_CONVERGED) return rc;
    if (flags & GTQA_BP_REGAUGE) {
        int r2 = [&]() -> int { GTQA_DISPATCH(s, regauge_t); }();
        if (r2) return r2;
    }
    return rc;
}

int gtqa_regauge(gtqa_state* s) {
    int rc = check_state(s);
    if (rc) return rc;
    GTQA_DISPATCH(s, regauge_t);
}

int gtqa_marginals(gtqa_state* s, double* rho_out, int8_t* sign_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!rho_out) return GTQA_ERR_INVALID_ARG;
    rc = [&]() -> int { GTQA_DISPATCH(s, marginals_t); }();
    if (rc) return rc;
    if (!cuda_ok(s, cudaMemcpyAsync(rho_out, s->rho, sizeof(cd) * 4 * (size_t)s->n, cudaMemcpyDefault, s->stream)))
        return GTQA_ERR_CUDA;
    if (sign_out &&
        !cuda_ok(s, cudaMemcpyAsync(sign_out, s->sign, (size_t)s->n, cudaMemcpyDefault, s->stream)))
        return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaMemcpyAsync(s->h_flags, s->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s->stream)))
        return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaStreamSynchronize(s->stream))) return GTQA_ERR_CUDA;
    if (s->h_flags[2]) {
        s->sticky = GTQA_ERR_NUMERIC;
        return GTQA_ERR_NUMERIC;
    }
    return GTQA_OK;
}

int gtqa_stats(gtqa_state* s, gtqa_stats_t* out) {
    if (!s || !out) return GTQA_ERR_INVALID_ARG;
    double st[4] = {0.0, 0.0, 0.0, 0.0};
    if (!cuda_ok(s, cudaMemcpyAsync(st, s->stats, sizeof(st), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    out->layers = s->layers;
    out->gates = s->gates;
    out->last_bp_iters = s->last_iters;
    out->not_converged = s->not_conv;
    out->last_bp_dist = s->last_dist;
    out->discarded_weight = st[0];
    out->log_fidelity = st[1];
    out->svd_pairs = (int64_t)st[2];
    out->svd_rotations = (int64_t)st[3];
    out->bp_sweeps = s->bp_sweeps;
    out->launches = s->launches;
    return GTQA_OK;
}

int gtqa_get_state(gtqa_state* s, double* gamma_out, double* lambda_out, double* messages_out) {
    int rc = check_state(s);
    if (rc) return rc;
    const cudaStream_t st = s->stream;
    if (gamma_out && !cuda_ok(s, cudaMemcpyAsync(gamma_out, s->Gamma, gamma_elems(s) * sizeof(cd), cudaMemcpyDefault, st)))
        return GTQA_ERR_CUDA;
    if (lambda_out &&
        !cuda_ok(s, cudaMemcpyAsync(lambda_out, s->lam, sizeof(double) * s->m * s->CHI, cudaMemcpyDefault, st)))
        return GTQA_ERR_CUDA;
    if (messages_out &&
        !cuda_ok(s, cudaMemcpyAsync(messages_out, s->msg[s->cur], msg_elems(s) * sizeof(cd), cudaMemcpyDefault, st)))
        return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaStreamSynchronize(st))) return GTQA_ERR_CUDA;
    return GTQA_OK;
}

int gtqa_set_state(gtqa_state* s, const double* gamma, const double* lambda, const double* messages) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!gamma || !lambda || !messages) return GTQA_ERR_INVALID_ARG;
    const cudaStream_t st = s->stream;
    if (!cuda_ok(s, cudaMemcpyAsync(s->Gamma, gamma, gamma_elems(s) * sizeof(cd), cudaMemcpyDefault, st)) ||
        !cuda_ok(s, cudaMemcpyAsync(s->lam, lambda, sizeof(double) * s->m * s->CHI, cudaMemcpyDefault, st)) ||
        !cuda_ok(s, cudaMemcpyAsync(s->msg[s->cur], messages, msg_elems(s) * sizeof(cd), cudaMemcpyDefault, st)) ||
        !cuda_ok(s, cudaStreamSynchronize(st)))
        return GTQA_ERR_CUDA;
    return GTQA_OK;
}

int gtqa_sizes(const gtqa_state* s, int64_t* n, int64_t* m, int32_t* chi_storage, int32_t* n_colours) {
    if (!s) return GTQA_ERR_INVALID_ARG;
    if (n) *n = s->n;
    if (m) *m = s->m;
    if (chi_storage) *chi_storage = s->CHI;
    if (n_colours) *n_colours = s->ncol;
    return GTQA_OK;
}

int gtqa_edge_colouring(int32_t n, int32_t m, const int32_t* edges, int32_t* colour_out, int32_t* n_colours_out) {
    if (n < 1 || m < 0 || (m > 0 && (!edges || !colour_out))) return GTQA_ERR_INVALID_ARG;
    std::vector<int> deg(n, 0);
    for (int e = 0; e < m; ++e) {
        const int u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return GTQA_ERR_INVALID_ARG;
    }
    std::vector<int> col;
    int nc = 0;
    if (!misra_gries(n, m, edges, col, nc)) return GTQA_ERR_INVALID_ARG;
    for (int e = 0; e < m; ++e) colour_out[e] = col[e];
    if (n_colours_out) *n_colours_out = nc;
    return GTQA_OK;
}

int gtqa_profile(gtqa_state* s, int32_t enable) {
    if (!s) return GTQA_ERR_INVALID_ARG;
    if (!cuda_ok(s, cudaStreamSynchronize(s->stream))) return GTQA_ERR_CUDA;
    prof_collect(s);
    for (int k = 0; k < GTQA_K_COUNT; ++k) {
        s->prof_ms[k] = 0.0;
        s->prof_launches[k] = 0;
        s->prof_units[k] = 0;
    }
    s->prof_on = enable != 0;
    return GTQA_OK;
}

int gtqa_profile_read(gtqa_state* s, int32_t kind, int64_t* launches, double* total_ms, int64_t* units) {
    if (!s || kind < 0 || kind >= GTQA_K_COUNT) return GTQA_ERR_INVALID_ARG;
    if (!cuda_ok(s, cudaStreamSynchronize(s->stream))) return GTQA_ERR_CUDA;
    prof_collect(s);
    if (launches) *launches = s->prof_launches[kind];
    if (total_ms) *total_ms = s->prof_ms[kind];
    if (units) *units = s->prof_units[kind];
    return GTQA_OK;
}

const char* gtqa_profile_name(int32_t kind) {
    static const char* names[GTQA_K_COUNT] = {"gate", "mixing", "layer_stats", "symmetric", "warm_start",
                                              "bp_sweep", "bp_reduce", "regauge_edge", "regauge_vertex",
                                              "marginals"};
    if (kind < 0 || kind >= GTQA_K_COUNT) return nullptr;
    return names[kind];
}

const char* gtqa_strerror(int code) {
    switch (code) {
        case GTQA_OK: return "ok";
        case GTQA_ERR_INVALID_ARG: return "invalid argument";
        case GTQA_ERR_NOT_CONVERGED: return "belief propagation reached max_iter before tol";
        case GTQA_ERR_NUMERIC: return "NaN or Inf detected";
        case GTQA_ERR_OOM: return "device memory allocation failed";
        case GTQA_ERR_CUDA: return "CUDA runtime error";
        case GTQA_ERR_TIMEOUT: return "bounded device wait timed out";
        case GTQA_ERR_UNSUPPORTED: return "chi or precision not supported by this build";
        default: return "unknown error code";
    }
}

void gtqa_destroy(gtqa_state* s) { free_state(s); }

}  // extern "C"
