// C ABI of the GTQA hot path: validation, graph bookkeeping, state management and
// the launches of the persistent annealing kernel.  Contracts are in include/gtqa.h.
#include "gtqa.h"
#include "gtqa_launch.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace gtqa;

// Dispatch on precision mode and phase kernel to the launcher units (compiled in gtqa_units.cu).
// Kept out of gtqa_launch.h: in a unit that sees the launchers' definitions these calls would
// instantiate every kernel set there.
namespace gtqa {
inline bool phase_shape(bool mixed, int pk, int CHI, int v, size_t* sb, int* tpb, int* team) {
    switch (pk) {
        case PK_GATES: return mixed ? PhaseUnit<ModeMixed, PK_GATES>::shape(CHI, v, sb, tpb, team)
                                    : PhaseUnit<ModeFP64, PK_GATES>::shape(CHI, v, sb, tpb, team);
        case PK_BP: return mixed ? PhaseUnit<ModeMixed, PK_BP>::shape(CHI, v, sb, tpb, team)
                                 : PhaseUnit<ModeFP64, PK_BP>::shape(CHI, v, sb, tpb, team);
        default: return mixed ? PhaseUnit<ModeMixed, PK_REGAUGE>::shape(CHI, v, sb, tpb, team)
                              : PhaseUnit<ModeFP64, PK_REGAUGE>::shape(CHI, v, sb, tpb, team);
    }
}
inline cudaError_t phase_prepare(bool mixed, int pk, int CHI, int v, size_t smem, int* bps) {
    switch (pk) {
        case PK_GATES: return mixed ? PhaseUnit<ModeMixed, PK_GATES>::prepare(CHI, v, smem, bps)
                                    : PhaseUnit<ModeFP64, PK_GATES>::prepare(CHI, v, smem, bps);
        case PK_BP: return mixed ? PhaseUnit<ModeMixed, PK_BP>::prepare(CHI, v, smem, bps)
                                 : PhaseUnit<ModeFP64, PK_BP>::prepare(CHI, v, smem, bps);
        default: return mixed ? PhaseUnit<ModeMixed, PK_REGAUGE>::prepare(CHI, v, smem, bps)
                              : PhaseUnit<ModeFP64, PK_REGAUGE>::prepare(CHI, v, smem, bps);
    }
}
inline cudaError_t phase_launch(bool mixed, int pk, int CHI, int v, const Ctx& c, size_t smem, cudaStream_t st) {
    switch (pk) {
        case PK_GATES: return mixed ? PhaseUnit<ModeMixed, PK_GATES>::launch(CHI, v, c, smem, st)
                                    : PhaseUnit<ModeFP64, PK_GATES>::launch(CHI, v, c, smem, st);
        case PK_BP: return mixed ? PhaseUnit<ModeMixed, PK_BP>::launch(CHI, v, c, smem, st)
                                 : PhaseUnit<ModeFP64, PK_BP>::launch(CHI, v, c, smem, st);
        default: return mixed ? PhaseUnit<ModeMixed, PK_REGAUGE>::launch(CHI, v, c, smem, st)
                              : PhaseUnit<ModeFP64, PK_REGAUGE>::launch(CHI, v, c, smem, st);
    }
}

}  // namespace gtqa

struct gtqa_state {
    int B = 0, n = 0, m = 0;
    int chi = 0, CHI = 0;
    int precision = GTQA_FP64;
    cudaStream_t stream = nullptr;
    double svd_cutoff = 1e-14, eig_cutoff = 1e-13;
    int ncol = 0;
    int nblocks = 0;
    size_t smem[PK_COUNT] = {0, 0, 0};   // dynamic shared memory of the three phase kernels
    int shape[PK_COUNT] = {0, 0, 0};     // their launch-shape variants (gtqa_autotune, gtqa_set_shape)
    int tpb[PK_COUNT] = {0, 0, 0};       // threads per block and team size of each kernel's variant
    int team[PK_COUNT] = {0, 0, 0};
    std::vector<int> h_inst_m;
    // device buffers
    void* Gamma = nullptr;
    double* lam = nullptr;
    void* T = nullptr;
    void* msg[2] = {nullptr, nullptr};
    cf* D0 = nullptr;
    cd* t0 = nullptr;
    cd* X = nullptr;
    int4* edge_info = nullptr;
    int4* vert_edges = nullptr;
    int* vert_inst = nullptr;
    double* J = nullptr;
    double* h = nullptr;
    int* colour_edges = nullptr;
    int* colour_off = nullptr;
    int* last_colour = nullptr;
    int* first_colour = nullptr;
    int* iso = nullptr;
    int n_iso = 0;
    int* inst_vbeg = nullptr;
    int* inst_m = nullptr;
    double* acc = nullptr;
    int* inst_done = nullptr;
    int* inst_iters = nullptr;
    double* inst_dist = nullptr;
    double* stats = nullptr;    // [kStats]: discarded weight, log fidelity, gate SVD pairs, gate SVD rotations,
                                // regauge SVD sweeps
    Control* ctl = nullptr;
    cd* rho = nullptr;
    int8_t* sign = nullptr;
    int* flags = nullptr;       // [0]: NaN in marginals
    double* rbuf = nullptr;     // residual / entropy accumulator
    unsigned char* cutbuf = nullptr;   // entropy: per-edge cut mask
    int8_t* xs = nullptr;       // sampling: outcomes [n]
    double* ps = nullptr;       // sampling: outcome probabilities [n]
    int* gate_edge = nullptr;   // arbitrary gates: edge ids grouped by launch, and their matrices
    cd* gate_U = nullptr;
    size_t gate_cap = 0;
    int* sq_vertex = nullptr;   // one-qubit gates: vertices and composed 2x2 matrices
    cd* sq_W = nullptr;
    size_t sq_cap = 0;
    std::vector<int> h_edges;   // endpoints of every edge (2m), for host-side scheduling
    // degree-4 graphs: slots per vertex, all vertex ids, host copies for the gate phases
    int D = 3;
    bool plain = false;         // degree 4 or CHI = 16: the plain kernels
    cd* pscratch = nullptr;     // plain path: per-block tensor buffers in global memory
    cd* dm = nullptr;           // plain path: new - old of every message of a sweep
    int4* vslots4 = nullptr;
    int* allv = nullptr;
    std::vector<int> h_deg, h_cedges, h_coff;
    std::vector<double> h_J, h_h;
    int cur4 = 0;               // message buffer holding the latest messages (degree 4)
    // gtqa_anneal_graph: one captured layer (gates, BP, regauge) whose layer index is read from
    // *kdev, and what it was captured for; with profiling on, events between the launches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int* kdev = nullptr;
    int gK = 0, gmi = 0;
    double gdt = 0.0, gtol = 0.0;
    bool gpending = false;      // a profiled replay whose events are not read yet
    cudaEvent_t gev[4] = {nullptr, nullptr, nullptr, nullptr};
    // host counters
    long long layers = 0, gates = 0, launches = 0;
    int sticky = GTQA_OK;
    long long spin_limit = 1LL << 22;   // polls per grid barrier before GTQA_ERR_TIMEOUT (about a second)
    int bar_extra = 0;                  // test hook: extra arrivals the barrier waits for
    int grid[PK_COUNT] = {0, 0, 0};     // persistent blocks per phase kernel (gtqa_autotune)
    // optional profiler (per launch class)
    bool prof_on = false;
    struct Pending { int kind; cudaEvent_t a, b; long long units; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[GTQA_K_COUNT] = {};
    long long prof_launches[GTQA_K_COUNT] = {};
    long long prof_units[GTQA_K_COUNT] = {};
};

namespace {

constexpr int kStats = 8;   // entries of the device statistics buffer (five in use)

bool cuda_ok(gtqa_state* s, cudaError_t e) {
    if (e != cudaSuccess) {
        if (s) s->sticky = GTQA_ERR_CUDA;
        return false;
    }
    return true;
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

// Grow a pair of state-owned device buffers to hold `need` entries (contents dropped).
template <typename A, typename B>
int grow_pair(gtqa_state* s, A** a, B** b, size_t per_b, size_t& cap, size_t need) {
    if (need <= cap) return GTQA_OK;
    if (*a) cudaFree(*a);
    if (*b) cudaFree(*b);
    *a = nullptr;
    *b = nullptr;
    cap = 0;
    int rc;
    if ((rc = dalloc(s, a, need)) || (rc = dalloc(s, b, need * per_b))) return rc;
    cap = need;
    return GTQA_OK;
}

int storage_chi(int chi) {
    if (chi <= 2) return 2;
    if (chi <= 4) return 4;
    if (chi <= 8) return 8;
    if (chi <= 16) return 16;
    return 0;
}

bool mixed(const gtqa_state* s) { return s->precision == GTQA_MIXED; }
bool f32(const gtqa_state* s) { return s->precision == GTQA_C64; }
// precision selector of the plain kernels: 0 FP64, 1 mixed, 2 complex64
int pm(const gtqa_state* s) { return s->precision == GTQA_FP64 ? 0 : (s->precision == GTQA_MIXED ? 1 : 2); }
// messages held as the absolute m in complex64 (the complex64 mode); the mixed mode holds
// m - m0 on both paths
bool abs32(const gtqa_state* s) { return f32(s); }
bool f32store(const gtqa_state* s) { return s->precision != GTQA_FP64; }
size_t elem_bytes(const gtqa_state* s) { return f32store(s) ? sizeof(cf) : sizeof(cd); }
size_t gamma_elems(const gtqa_state* s) {
    return (size_t)s->n * 2 * s->CHI * s->CHI * s->CHI * (s->D == 4 ? s->CHI : 1);
}
size_t msg_elems(const gtqa_state* s) { return (size_t)s->m * 2 * s->CHI * s->CHI; }

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

// Adds the phase times of the last profiled graph replay (gtqa_anneal_graph) to the profiler's
// classes; waits for that replay.  Returns false on a CUDA error.
bool graph_collect(gtqa_state* s) {
    if (!s->gpending) return true;
    s->gpending = false;
    float ms[3];
    if (!cuda_ok(s, cudaEventSynchronize(s->gev[3]))) return false;
    for (int q = 0; q < 3; ++q)
        if (!cuda_ok(s, cudaEventElapsedTime(&ms[q], s->gev[q], s->gev[q + 1]))) return false;
    const int kinds[3] = {GTQA_K_TROTTER, GTQA_K_BP, GTQA_K_REGAUGE};
    const long long units[3] = {s->m, s->n, s->m};
    for (int q = 0; q < 3; ++q) {
        s->prof_ms[kinds[q]] += ms[q];
        s->prof_launches[kinds[q]] += 1;
        s->prof_units[kinds[q]] += units[q];
    }
    return true;
}

// Drop the captured layer graph: its launches carry the grid sizes and shapes of the capture.
bool drop_graph(gtqa_state* s) {
    const bool ok = graph_collect(s);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->gexec = nullptr;
    s->graph = nullptr;
    return ok;
}

void prof_collect(gtqa_state* s) {
    graph_collect(s);
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

// Edge colouring with Delta colours by a seeded Kempe-chain search (same scheme as the
// input generators): edges in a random order; an edge {u, v} takes a colour free at both
// ends, else the a/b chain from v (a free at u, b free at v) is swapped unless it ends at u,
// else a random Kempe component through u or v is swapped and the edge is tried again.
// Returns false after max_steps attempts (the graph may need Delta + 1 colours).
bool delta_colouring(int n, int m, const int* edges, std::vector<int>& colour, int& ncol) {
    ncol = 0;
    colour.assign(m, 0);
    if (m == 0) return true;
    std::vector<int> deg(n, 0);
    for (int e = 0; e < m; ++e) {
        deg[edges[2 * e]]++;
        deg[edges[2 * e + 1]]++;
    }
    int D = 0;
    for (int v = 0; v < n; ++v) D = deg[v] > D ? deg[v] : D;
    if (D <= 1) {
        ncol = 1;
        return true;
    }
    unsigned long long rs = 0x9e3779b97f4a7c15ull;
    auto rnd = [&](int k) {   // splitmix64, reduced to [0, k)
        rs += 0x9e3779b97f4a7c15ull;
        unsigned long long z = rs;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (int)(z % (unsigned long long)k);
    };
    std::vector<int> at((size_t)n * D, -1), col(m, -1), order(m);
    for (int e = 0; e < m; ++e) order[e] = e;
    for (int e = m - 1; e > 0; --e) std::swap(order[e], order[rnd(e + 1)]);
    auto other = [&](int f, int x) { return edges[2 * f] == x ? edges[2 * f + 1] : edges[2 * f]; };
    auto recolour = [&](const std::vector<int>& fs, int a, int b) {
        for (int f : fs) {
            at[(size_t)edges[2 * f] * D + col[f]] = -1;
            at[(size_t)edges[2 * f + 1] * D + col[f]] = -1;
        }
        for (int f : fs) {
            col[f] = col[f] == a ? b : a;
            at[(size_t)edges[2 * f] * D + col[f]] = f;
            at[(size_t)edges[2 * f + 1] * D + col[f]] = f;
        }
    };
    std::vector<int> path, stack, fu, fv, common;
    std::vector<char> fseen(m, 0), vseen(n, 0);
    const long long limit = 200LL * m + 1000;
    long long steps = 0;
    for (int e : order) {
        const int u = edges[2 * e], v = edges[2 * e + 1];
        int c = -1;
        while (c < 0) {
            if (++steps > limit) return false;
            fu.clear();
            fv.clear();
            common.clear();
            for (int k = 0; k < D; ++k) {
                if (at[(size_t)u * D + k] < 0) fu.push_back(k);
                if (at[(size_t)v * D + k] < 0) fv.push_back(k);
            }
            for (int k : fu)
                if (std::find(fv.begin(), fv.end(), k) != fv.end()) common.push_back(k);
            if (!common.empty()) {
                c = common[rnd((int)common.size())];
                break;
            }
            const int a = fu[rnd((int)fu.size())], b = fv[rnd((int)fv.size())];
            path.clear();
            int x = v, cc = a;
            while (at[(size_t)x * D + cc] >= 0) {
                const int f = at[(size_t)x * D + cc];
                path.push_back(f);
                x = other(f, x);
                cc = cc == a ? b : a;
            }
            if (x != u) {
                recolour(path, a, b);
                c = a;
                break;
            }
            // the whole p/q component through u or v
            const int p = rnd(D);
            int q = rnd(D - 1);
            if (q >= p) ++q;
            path.clear();
            stack.assign(1, rnd(2) ? u : v);
            vseen[stack[0]] = 1;
            std::vector<int> touched(1, stack[0]);
            while (!stack.empty()) {
                const int y = stack.back();
                stack.pop_back();
                for (int k : {p, q}) {
                    const int f = at[(size_t)y * D + k];
                    if (f >= 0 && !fseen[f]) {
                        fseen[f] = 1;
                        path.push_back(f);
                        const int z = other(f, y);
                        if (!vseen[z]) {
                            vseen[z] = 1;
                            touched.push_back(z);
                            stack.push_back(z);
                        }
                    }
                }
            }
            for (int f : path) fseen[f] = 0;
            for (int z : touched) vseen[z] = 0;
            recolour(path, p, q);
        }
        col[e] = c;
        at[(size_t)u * D + c] = e;
        at[(size_t)v * D + c] = e;
    }
    colour = col;
    ncol = D;
    return true;
}

// Fewest colours the library can find: Delta by delta_colouring, else Misra-Gries.
bool misra_gries(int n, int m, const int* edges, std::vector<int>& colour, int& ncol);
bool edge_colouring(int n, int m, const int* edges, std::vector<int>& colour, int& ncol) {
    return delta_colouring(n, m, edges, colour, ncol) || misra_gries(n, m, edges, colour, ncol);
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
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (cudaEvent_t e : s->gev)
        if (e) cudaEventDestroy(e);
    void* ptrs[] = {s->kdev, s->Gamma, s->lam, s->T, s->msg[0], s->msg[1], s->D0, s->t0, s->X, s->edge_info,
                    s->vert_edges, s->vert_inst, s->J, s->h, s->colour_edges, s->colour_off, s->last_colour, s->first_colour,
                    s->iso, s->inst_vbeg, s->inst_m, s->acc, s->inst_done, s->inst_iters, s->inst_dist,
                    s->stats, s->ctl, s->rho, s->sign, s->flags, s->rbuf, s->cutbuf, s->xs, s->ps,
                    s->gate_edge, s->gate_U, s->sq_vertex, s->sq_W, s->vslots4, s->allv, s->pscratch, s->dm};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& p : s->pending) {
        s->pool.push_back(p.a);
        s->pool.push_back(p.b);
    }
    for (cudaEvent_t e : s->pool) cudaEventDestroy(e);
    delete s;
}

// stores the first layer index of a run of graph replays (gtqa_anneal_graph)
__global__ void set_layer_kernel(int* kdev, int k) { *kdev = k; }

Ctx make_ctx(const gtqa_state* s) {
    Ctx c;
    std::memset(&c, 0, sizeof(c));
    c.edge_info = s->edge_info;
    c.vert_edges = s->vert_edges;
    c.vert_inst = s->vert_inst;
    c.J = s->J;
    c.h = s->h;
    c.colour_edges = s->colour_edges;
    c.colour_off = s->colour_off;
    c.last_colour = s->last_colour;
    c.first_colour = s->first_colour;
    c.iso = s->iso;
    c.n_iso = s->n_iso;
    c.ncol = s->ncol;
    c.n = s->n;
    c.m = s->m;
    c.B = s->B;
    c.inst_vbeg = s->inst_vbeg;
    c.inst_m = s->inst_m;
    c.Gamma = s->Gamma;
    c.lam = s->lam;
    c.T = s->T;
    c.msg[0] = s->msg[0];
    c.msg[1] = s->msg[1];
    c.D0 = s->D0;
    c.t0 = s->t0;
    c.X = s->X;
    c.acc = s->acc;
    c.inst_done = s->inst_done;
    c.inst_iters = s->inst_iters;
    c.inst_dist = s->inst_dist;
    c.stats = s->stats;
    c.ctl = s->ctl;
    c.chi = s->chi;
    c.svd_cut = s->svd_cutoff;
    c.eig_cut = s->eig_cutoff;
    c.nblocks = s->nblocks;
    c.bar_expect = s->nblocks + s->bar_extra;
    c.spin_limit = s->spin_limit;
    return c;
}

// Select launch-shape variant v of phase kernel pk: its dynamic shared memory (with the BP
// kernel's per-instance part), the kernel's opt-in shared-memory limit, and a check that a
// block fits on an SM.  GTQA_ERR_UNSUPPORTED for a variant that does not exist or does not
// fit; the state keeps its previous shape then.
int apply_shape(gtqa_state* s, int pk, int v) {
    if (v < 0 || v >= shape_count(pk)) return GTQA_ERR_UNSUPPORTED;
    size_t base = 0;
    int tpb = 0, team = 0, bps = 0;
    if (!phase_shape(mixed(s), pk, s->CHI, v, &base, &tpb, &team)) return GTQA_ERR_UNSUPPORTED;
    const size_t smem = (base + (pk == PK_BP ? bp_instance_smem(s->B) : 0) + 15) / 16 * 16;
    const cudaError_t pe = phase_prepare(mixed(s), pk, s->CHI, v, smem, &bps);
    if (pe != cudaSuccess || bps < 1) {
        cudaGetLastError();
        return (pe == cudaSuccess || pe == cudaErrorInvalidValue) ? GTQA_ERR_UNSUPPORTED : GTQA_ERR_CUDA;
    }
    s->shape[pk] = v;
    s->smem[pk] = smem;
    s->tpb[pk] = tpb;
    s->team[pk] = team;
    return GTQA_OK;
}

// One cooperative launch of a phase kernel.
int run(gtqa_state* s, const Ctx& c0, int pk, int kind, long long units) {
    cudaError_t e;
    Ctx c = c0;
    c.nblocks = s->grid[pk];
    c.bar_expect = s->grid[pk] + s->bar_extra;
    // each phase kernel counts its barrier arrivals separately, so that the counter stays a
    // multiple of that kernel's grid size between its launches (gtqa_set_grid and the
    // autotuner zero it when the size changes)
    c.bar = &s->ctl->bar_pk[pk];
    {
        ProfScope ps(s, kind, units);
        e = phase_launch(mixed(s), pk, s->CHI, s->shape[pk], c, s->smem[pk], s->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->sticky = GTQA_ERR_CUDA;
        return GTQA_ERR_CUDA;
    }
    s->launches += 1;
    return GTQA_OK;
}

// Read the device control block (synchronises) and surface a device-side error.
int read_ctl(gtqa_state* s, Control* out) {
    if (!cuda_ok(s, cudaMemcpyAsync(out, s->ctl, sizeof(Control), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    if (out->err) {
        s->sticky = out->err;
        return out->err;
    }
    return GTQA_OK;
}

int check_state(const gtqa_state* s) {
    if (!s) return GTQA_ERR_INVALID_ARG;
    return s->sticky;
}

int create_impl(int B, const int* n, const int* m, const int* edges, const int* colour, const double* J,
                const double* h, int chi, const gtqa_options* opt, gtqa_state** out) {
    if (!out) return GTQA_ERR_INVALID_ARG;
    *out = nullptr;
    if (B < 1 || B > 4096 || !n || !m || !h || chi < 1) return GTQA_ERR_INVALID_ARG;
    if (storage_chi(chi) == 0) return GTQA_ERR_UNSUPPORTED;
    gtqa_options o;
    gtqa_options_init(&o);
    if (opt) o = *opt;
    if (o.precision != GTQA_FP64 && o.precision != GTQA_MIXED && o.precision != GTQA_C64) return GTQA_ERR_UNSUPPORTED;
    if (o.reserved0 != 0) return GTQA_ERR_INVALID_ARG;
    long long N = 0, Mtot = 0;
    for (int b = 0; b < B; ++b) {
        if (n[b] < 1 || m[b] < 0) return GTQA_ERR_INVALID_ARG;
        N += n[b];
        Mtot += m[b];
    }
    if (N > (1LL << 28) || Mtot > (1LL << 28)) return GTQA_ERR_INVALID_ARG;
    if (Mtot > 0 && (!edges || !J)) return GTQA_ERR_INVALID_ARG;
    std::vector<int> ge((size_t)Mtot * 2), gcol((size_t)Mtot), vinst(N);
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
                if (++deg[u + voff] > 4 || ++deg[v + voff] > 4) return GTQA_ERR_INVALID_ARG;
            }
            std::vector<long long> sk = keys;
            std::sort(sk.begin(), sk.end());
            for (size_t i = 1; i < sk.size(); ++i)
                if (sk[i] == sk[i - 1]) return GTQA_ERR_INVALID_ARG;
            for (int a = 0; a < n[b]; ++a) {
                if (!std::isfinite(h[voff + a])) return GTQA_ERR_INVALID_ARG;
                vinst[voff + a] = b;
            }
            if (colour) {
                for (int e = 0; e < m[b]; ++e) {
                    const int c = colour[eoff + e];
                    if (c < 0 || c >= 64) return GTQA_ERR_INVALID_ARG;
                    gcol[eoff + e] = c;
                }
            } else {
                std::vector<int> col;
                int nc = 0;
                if (!edge_colouring(n[b], m[b], edges + 2 * eoff, col, nc)) return GTQA_ERR_INVALID_ARG;
                for (int e = 0; e < m[b]; ++e) gcol[eoff + e] = col[e];
            }
            voff += n[b];
            eoff += m[b];
        }
        vbeg[B] = (int)voff;
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
    // vertex degree 4 (Sec. V's 4-regular graphs), storage bond dimension 16 or the complex64
    // mode: the plain kernels, one instance
    int Dmax = 0;
    for (long long v = 0; v < N; ++v) Dmax = std::max(Dmax, deg[v]);
    const int Dst = Dmax == 4 ? 4 : 3;
    const bool c64 = o.precision == GTQA_C64;
    const bool plain = Dst == 4 || storage_chi(chi) == 16 || c64;
    const int pmode = o.precision == GTQA_FP64 ? 0 : (o.precision == GTQA_MIXED ? 1 : 2);
    if (plain && (B != 1 || !plain_supported(storage_chi(chi), Dst, pmode)))
        return GTQA_ERR_UNSUPPORTED;
    gtqa_state* s = new (std::nothrow) gtqa_state();
    if (!s) return GTQA_ERR_OOM;
    s->D = Dst;
    s->plain = plain;
    s->B = B;
    s->n = (int)N;
    s->m = (int)Mtot;
    s->chi = chi;
    s->CHI = storage_chi(chi);
    s->precision = o.precision;
    s->stream = (cudaStream_t)o.cuda_stream;
    // relative cut-offs: FP64 defaults, FP32-sized ones in the complex64 mode
    s->svd_cutoff = o.svd_cutoff > 0 ? o.svd_cutoff : (c64 ? 1e-7 : 1e-14);
    s->eig_cutoff = o.eig_cutoff > 0 ? o.eig_cutoff : (c64 ? 1e-6 : 1e-13);
    s->ncol = ncol;
    s->h_inst_m = minst;
    s->h_edges = ge;
    // launch shapes: one resident block per SM for each cooperative phase kernel
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return GTQA_ERR_CUDA;
    }
    for (int pk = 0; pk < PK_COUNT && !s->plain; ++pk) {
        const int src = apply_shape(s, pk, 0);
        if (src != GTQA_OK) {
            delete s;
            return src;
        }
    }
    s->nblocks = sms;
    for (int pk = 0; pk < PK_COUNT; ++pk) s->grid[pk] = sms;
    // slots: incident edges in ascending id; colour of each vertex's last gate
    std::vector<int4> vedges(N, make_int4(-1, -1, -1, 0)), v4(N, make_int4(-1, -1, -1, -1));
    std::vector<int4> einfo(Mtot);
    std::vector<int> lastc(N, -1), firstc(N, -1);
    for (long long e = 0; e < Mtot; ++e) {
        int sl[2];
        for (int q = 0; q < 2; ++q) {
            const int v = ge[2 * e + q];
            int4& ve = vedges[v];
            const int k = ve.w;
            if (k == 0) ve.x = (int)e; else if (k == 1) ve.y = (int)e; else if (k == 2) ve.z = (int)e;
            int4& w4 = v4[v];
            if (k == 0) w4.x = (int)e; else if (k == 1) w4.y = (int)e; else if (k == 2) w4.z = (int)e; else w4.w = (int)e;
            sl[q] = k;
            ve.w = k + 1;
            lastc[v] = std::max(lastc[v], gcol[e]);
            firstc[v] = firstc[v] < 0 ? gcol[e] : std::min(firstc[v], gcol[e]);
        }
        einfo[e] = make_int4(ge[2 * e], ge[2 * e + 1], sl[0], sl[1]);
    }
    std::vector<int> iso;
    for (long long a = 0; a < N; ++a)
        if (vedges[a].w == 0) iso.push_back((int)a);
    s->n_iso = (int)iso.size();
    std::vector<int> cedges;
    cedges.reserve(Mtot);
    std::vector<int> coff(ncol + 1, 0);
    for (int c = 0; c < ncol; ++c) {
        coff[c] = (int)cedges.size();
        for (long long e = 0; e < Mtot; ++e)
            if (gcol[e] == c) cedges.push_back((int)e);
    }
    coff[ncol] = (int)cedges.size();
    if (s->plain) {
        s->h_cedges = cedges;
        s->h_coff = coff;
        s->h_J.assign(J ? J : (const double*)nullptr, J ? J + Mtot : (const double*)nullptr);
        s->h_h.assign(h, h + N);
        s->h_deg.assign(deg.begin(), deg.end());
    }
    const int CHI = s->CHI;
    const size_t gel = gamma_elems(s), mel = msg_elems(s), eb = elem_bytes(s);
    int rc = GTQA_OK;
    if ((rc = dalloc(s, (unsigned char**)&s->Gamma, gel * eb)) || (rc = dalloc(s, (unsigned char**)&s->T, gel * eb)) ||
        (rc = dalloc(s, (unsigned char**)&s->msg[0], mel * eb)) ||
        (rc = dalloc(s, (unsigned char**)&s->msg[1], mel * eb)) || (rc = dalloc(s, &s->lam, (size_t)s->m * CHI)) ||
        (rc = dalloc(s, &s->D0, mixed(s) ? mel : 1)) || (rc = dalloc(s, &s->t0, mixed(s) ? (size_t)2 * s->m : 1)) ||
        (rc = dalloc(s, &s->X, (size_t)s->m * 2 * CHI * CHI)) || (rc = dalloc(s, &s->edge_info, s->m)) ||
        (rc = dalloc(s, &s->vert_edges, s->n)) || (rc = dalloc(s, &s->vert_inst, s->n)) ||
        (rc = dalloc(s, &s->J, s->m)) || (rc = dalloc(s, &s->h, s->n)) || (rc = dalloc(s, &s->colour_edges, s->m)) ||
        (rc = dalloc(s, &s->colour_off, ncol + 1)) || (rc = dalloc(s, &s->last_colour, s->n)) ||
        (rc = dalloc(s, &s->first_colour, s->n)) ||
        (rc = dalloc(s, &s->iso, iso.size())) || (rc = dalloc(s, &s->inst_vbeg, B + 1)) ||
        (rc = dalloc(s, &s->inst_m, B)) || (rc = dalloc(s, &s->acc, 6 * (size_t)B)) ||
        (rc = dalloc(s, &s->inst_done, B)) || (rc = dalloc(s, &s->inst_iters, B)) ||
        (rc = dalloc(s, &s->inst_dist, B)) || (rc = dalloc(s, &s->stats, kStats)) || (rc = dalloc(s, &s->ctl, 1)) || (rc = dalloc(s, &s->kdev, 1)) ||
        (rc = dalloc(s, &s->rho, (size_t)s->n * 4)) || (rc = dalloc(s, &s->sign, s->n)) ||
        (rc = dalloc(s, &s->flags, 4)) || (rc = dalloc(s, &s->rbuf, 1)) ||
        (rc = dalloc(s, &s->cutbuf, std::max(s->m, 1))) || (rc = dalloc(s, &s->xs, s->n)) ||
        (rc = dalloc(s, &s->ps, s->n)) || (s->plain && (rc = dalloc(s, &s->vslots4, s->n))) ||
        (s->plain && (rc = dalloc(s, &s->allv, s->n))) ||
        (s->plain && (rc = dalloc(s, &s->pscratch, plain_scratch_entries(s->CHI, s->D, s->n, s->m)))) ||
        (s->plain && (rc = dalloc(s, &s->dm, (size_t)2 * s->m * CHI * CHI)))) {
        free_state(s);
        return rc;
    }
    if (s->plain) {
        std::vector<int> all(N);
        for (long long a = 0; a < N; ++a) all[a] = (int)a;
        if (!cuda_ok(s, cudaMemcpyAsync(s->vslots4, v4.data(), sizeof(int4) * N, cudaMemcpyHostToDevice, s->stream)) ||
            !cuda_ok(s, cudaMemcpyAsync(s->allv, all.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s->stream)) ||
            !cuda_ok(s, cudaStreamSynchronize(s->stream))) {
            free_state(s);
            return GTQA_ERR_CUDA;
        }
    }
    // |+>^N: Gamma[a][i][0][0][0] = 1/sqrt(2); lambda_e = (1, 0, ...)
    const size_t H = (size_t)CHI * CHI * CHI * (s->D == 4 ? CHI : 1);
    std::vector<unsigned char> g0(gel * eb, 0);
    for (long long a = 0; a < N; ++a) {
        for (int i = 0; i < 2; ++i) {
            const size_t idx = a * 2 * H + i * H;
            if (f32store(s)) reinterpret_cast<cf*>(g0.data())[idx] = cf{(float)M_SQRT1_2, 0.f};
            else reinterpret_cast<cd*>(g0.data())[idx] = cd{M_SQRT1_2, 0.0};
        }
    }
    std::vector<double> l0((size_t)s->m * CHI, 0.0);
    for (long long e = 0; e < Mtot; ++e) l0[e * CHI] = 1.0;
    std::vector<double> Jv(J ? J : (const double*)nullptr, J ? J + Mtot : (const double*)nullptr);
    std::vector<double> hv(h, h + N);
    Control ctl0;
    std::memset(&ctl0, 0, sizeof(ctl0));
    cudaStream_t st = s->stream;
    bool ok = cuda_ok(s, cudaMemcpyAsync(s->Gamma, g0.data(), g0.size(), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->T, 0, gel * eb, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->msg[0], 0, mel * eb, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->msg[1], 0, mel * eb, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->lam, l0.data(), l0.size() * sizeof(double), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->edge_info, einfo.data(), sizeof(int4) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->vert_edges, vedges.data(), sizeof(int4) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->vert_inst, vinst.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->J, Jv.data(), sizeof(double) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->h, hv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->colour_edges, cedges.data(), sizeof(int) * Mtot, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->colour_off, coff.data(), sizeof(int) * (ncol + 1), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->last_colour, lastc.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->first_colour, firstc.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st)) &&
              (iso.empty() || cuda_ok(s, cudaMemcpyAsync(s->iso, iso.data(), sizeof(int) * iso.size(), cudaMemcpyHostToDevice, st))) &&
              cuda_ok(s, cudaMemcpyAsync(s->inst_vbeg, vbeg.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->inst_m, minst.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->stats, 0, sizeof(double) * kStats, st)) &&
              cuda_ok(s, cudaMemcpyAsync(s->ctl, &ctl0, sizeof(Control), cudaMemcpyHostToDevice, st)) &&
              cuda_ok(s, cudaMemsetAsync(s->flags, 0, sizeof(int) * 4, st)) && cuda_ok(s, cudaStreamSynchronize(st));
    if (!ok) {
        free_state(s);
        return GTQA_ERR_CUDA;
    }
    *out = s;
    return GTQA_OK;
}

// messages of the state in complex128 (mixed mode: m0 from lambda plus the stored correction)
int read_messages(gtqa_state* s, int cur, std::vector<cd>& out) {
    const size_t mel = msg_elems(s);
    const int CC = s->CHI * s->CHI;
    out.assign(mel, cd{0.0, 0.0});
    if (!f32store(s)) {
        if (!cuda_ok(s, cudaMemcpyAsync(out.data(), s->msg[cur], mel * sizeof(cd), cudaMemcpyDeviceToHost, s->stream)))
            return GTQA_ERR_CUDA;
        return cuda_ok(s, cudaStreamSynchronize(s->stream)) ? GTQA_OK : GTQA_ERR_CUDA;
    }
    if (abs32(s)) {
        std::vector<cf> d(mel);
        if (!cuda_ok(s, cudaMemcpyAsync(d.data(), s->msg[cur], mel * sizeof(cf), cudaMemcpyDeviceToHost, s->stream)) ||
            !cuda_ok(s, cudaStreamSynchronize(s->stream)))
            return GTQA_ERR_CUDA;
        for (size_t i = 0; i < mel; ++i) out[i] = cd{(double)d[i].x, (double)d[i].y};
        return GTQA_OK;
    }
    std::vector<cf> d(mel);
    std::vector<double> L((size_t)s->m * s->CHI);
    if (!cuda_ok(s, cudaMemcpyAsync(d.data(), s->msg[cur], mel * sizeof(cf), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaMemcpyAsync(L.data(), s->lam, L.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    for (int e = 0; e < s->m; ++e) {
        double sum = 0.0;
        for (int q = 0; q < s->CHI; ++q) sum += L[(size_t)e * s->CHI + q];
        for (int x = 0; x < 2; ++x)
            for (int r = 0; r < CC; ++r) {
                const size_t idx = ((size_t)2 * e + x) * CC + r;
                const int j = r / s->CHI, jp = r % s->CHI;
                double m0 = (j == jp && sum > 0.0) ? L[(size_t)e * s->CHI + j] / sum : 0.0;
                out[idx] = cd{m0 + (double)d[idx].x, (double)d[idx].y};
            }
    }
    return GTQA_OK;
}

// Eq. (apprx_entropy): every thread adds -sum_j lambda^2 log lambda^2 of one cut edge.
__global__ void entropy_kernel(const double* lam, const unsigned char* cut, int m, int chi, double* out) {
    __shared__ double part[8];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (e < m && cut[e]) {
        for (int j = 0; j < chi; ++j) {
            const double p = lam[(size_t)e * chi + j] * lam[(size_t)e * chi + j];
            if (p > 0.0) v -= p * log(p);
        }
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += part[w];
        if (t != 0.0) atomicAdd(out, t);
    }
}

// Smallest eigenpair of the symmetric tridiagonal matrix (a on the diagonal, b below it):
// the eigenvalue by bisection on the Sturm count, the eigenvector by inverse iteration
// with a tridiagonal (Thomas) solve.
void tridiag_min_eigvec(const std::vector<double>& a, const std::vector<double>& b, std::vector<double>& y) {
    const int k = (int)a.size();
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto count_below = [&](double x) {   // eigenvalues < x (Sturm sequence)
        int c = 0;
        double q = a[0] - x;
        if (q < 0) ++c;
        for (int i = 1; i < k; ++i) {
            const double d = q != 0.0 ? q : 1e-300;
            q = a[i] - x - b[i - 1] * b[i - 1] / d;
            if (q < 0) ++c;
        }
        return c;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(mid) >= 1) hi = mid; else lo = mid;
    }
    const double lam = lo - 1e-13 * std::max(1.0, std::fabs(lo));
    y.assign(k, 1.0);
    std::vector<double> d(k), r(k);
    for (int pass = 0; pass < 4; ++pass) {   // (T - lam I) y_new = y
        d[0] = a[0] - lam;
        r[0] = y[0];
        for (int i = 1; i < k; ++i) {
            const double piv = d[i - 1] != 0.0 ? d[i - 1] : 1e-300;
            const double f = b[i - 1] / piv;
            d[i] = a[i] - lam - f * b[i - 1];
            r[i] = y[i] - f * r[i - 1];
        }
        y[k - 1] = r[k - 1] / (d[k - 1] != 0.0 ? d[k - 1] : 1e-300);
        for (int i = k - 2; i >= 0; --i) y[i] = (r[i] - b[i] * y[i + 1]) / (d[i] != 0.0 ? d[i] : 1e-300);
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (double& v : y) v /= nrm;
    }
}

// ---------------------------------------------------------------------------
// degree-4 graphs: host orchestration of the plain kernels of gtqa_deg4.cuh
// ---------------------------------------------------------------------------
PlainArgs d4_args(gtqa_state* s, int cur) {
    PlainArgs a;
    a.Gamma = s->Gamma;
    a.T = s->T;
    a.lam = s->lam;
    a.msg_cur = s->msg[cur];
    a.msg_nxt = s->msg[cur ^ 1];
    a.X = s->X;
    a.dm = s->dm;
    a.scratch = s->pscratch;
    a.vslots = s->vslots4;
    a.edge_info = s->edge_info;
    a.n = s->n;
    a.m = s->m;
    a.acc = s->acc;
    a.warm = 0;
    a.D0 = s->D0;
    a.t0 = s->t0;
    return a;
}

int d4_fail(gtqa_state* s) {
    cudaGetLastError();
    s->sticky = GTQA_ERR_CUDA;
    return GTQA_ERR_CUDA;
}

// exp(-i t X) on every vertex (Sec. II D)
int d4_mixing(gtqa_state* s, double t) {
    if (t == 0.0 || s->n == 0) return GTQA_OK;
    std::vector<double> W(8 * (size_t)s->n);
    const double c = std::cos(t), sn = std::sin(t);
    for (int a = 0; a < s->n; ++a) {
        double* w = &W[8 * (size_t)a];
        w[0] = c; w[1] = 0.0; w[2] = 0.0; w[3] = -sn;
        w[4] = 0.0; w[5] = -sn; w[6] = c; w[7] = 0.0;
    }
    int rc;
    if ((rc = grow_pair(s, &s->sq_vertex, &s->sq_W, 4, s->sq_cap, (size_t)s->n))) return rc;
    if (!cuda_ok(s, cudaMemcpyAsync(s->sq_W, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, s->stream)))
        return GTQA_ERR_CUDA;
    if (plain_single_gates_launch(s->CHI, s->D, pm(s), s->Gamma, s->allv, s->sq_W, s->n, s->stream) != cudaSuccess)
        return d4_fail(s);
    s->launches += 1;
    return GTQA_OK;
}

// Edge gates of U_Z(t_Z) by colour class (App. F; App. E through the whole-side update).
int d4_interaction(gtqa_state* s, double tZ) {
    const int m = s->m;
    if (m == 0) return GTQA_OK;
    std::vector<double> U(32 * (size_t)m, 0.0);
    for (int q = 0; q < m; ++q) {
        const int e = s->h_cedges[q];
        const int a = s->h_edges[2 * (size_t)e], b = s->h_edges[2 * (size_t)e + 1];
        const double ha = s->h_h[a] / s->h_deg[a], hb = s->h_h[b] / s->h_deg[b], Je = s->h_J.empty() ? 0.0 : s->h_J[e];
        for (int ia = 0; ia < 2; ++ia)
            for (int ib = 0; ib < 2; ++ib) {
                const double za = 1.0 - 2.0 * ia, zb = 1.0 - 2.0 * ib;
                const double ph = -tZ * (Je * za * zb + ha * za + hb * zb);
                const int d = 2 * ia + ib;
                U[32 * (size_t)q + 2 * (4 * d + d)] = std::cos(ph);
                U[32 * (size_t)q + 2 * (4 * d + d) + 1] = std::sin(ph);
            }
    }
    int rc;
    if ((rc = grow_pair(s, &s->gate_edge, &s->gate_U, 16, s->gate_cap, (size_t)m))) return rc;
    if (!cuda_ok(s, cudaMemcpyAsync(s->gate_U, U.data(), sizeof(double) * U.size(), cudaMemcpyHostToDevice, s->stream)))
        return GTQA_ERR_CUDA;
    for (int c = 0; c < s->ncol; ++c) {
        cudaError_t e;
        if (s->CHI == 16) {
            Gate16Args g;
            g.Gamma = s->Gamma;
            g.lam = s->lam;
            g.edge_info = s->edge_info;
            g.vslots = s->vslots4;
            g.gate_edge = s->colour_edges + s->h_coff[c];
            g.gate_U = s->gate_U + 16 * (size_t)s->h_coff[c];
            g.scratch = s->pscratch;
            g.count = s->h_coff[c + 1] - s->h_coff[c];
            g.stats = s->stats;
            g.chi = s->chi;
            g.svd_cut = s->svd_cutoff;
            e = ising16_gates_launch(g, pm(s), s->stream);
        } else {
            GenArgs g;
            g.Gamma = s->Gamma;
            g.lam = s->lam;
            g.edge_info = s->edge_info;
            g.vert_edges = s->vslots4;
            g.gate_edge = s->colour_edges + s->h_coff[c];
            g.gate_U = s->gate_U + 16 * (size_t)s->h_coff[c];
            g.count = s->h_coff[c + 1] - s->h_coff[c];
            g.stats = s->stats;
            g.chi = s->chi;
            g.svd_cut = s->svd_cutoff;
            e = plain_general_gates_launch(s->CHI, s->D, pm(s), g, s->stream);
        }
        if (e != cudaSuccess) return d4_fail(s);
        s->launches += 1;
    }
    return GTQA_OK;
}

int d4_trotter(gtqa_state* s, double tZ, double tXpre, double tXpost) {
    int rc;
    if ((rc = d4_mixing(s, tXpre)) || (rc = d4_interaction(s, tZ)) || (rc = d4_mixing(s, tXpost))) return rc;
    s->layers += 1;
    s->gates += s->m;
    return GTQA_OK;
}

int d4_regauge(gtqa_state* s) {
    if (plain_regauge_launch(s->CHI, s->D, pm(s), d4_args(s, s->cur4), s->msg[s->cur4], s->eig_cutoff,
                             s->svd_cutoff, s->stream) != cudaSuccess)
        return d4_fail(s);
    s->launches += 2;
    return GTQA_OK;
}

// Flooding BP (App. B): one launch per sweep; the host reads the trace-norm distance after
// each sweep and stops after the sweep where dist/|E| < tol, or after max_iter sweeps.
int d4_bp(gtqa_state* s, double tol, int max_iter, uint32_t flags, int32_t* iters_out, double* dist_out) {
    int cur = s->cur4;
    PlainArgs a = d4_args(s, cur);
    a.warm = (flags & GTQA_BP_WARM_START) ? 1 : 0;
    a.msg_nxt = s->msg[cur];   // the init kernel writes the warm start where the first sweep reads
    if (s->n > 0 && plain_bp_init_launch(s->CHI, s->D, pm(s), a, s->stream) != cudaSuccess) return d4_fail(s);
    s->launches += 1;
    int it = 0;
    double dist = 0.0;
    bool conv = false;
    for (; it < max_iter;) {
        if (!cuda_ok(s, cudaMemsetAsync(s->acc, 0, sizeof(double), s->stream))) return GTQA_ERR_CUDA;
        PlainArgs w = d4_args(s, cur);
        if (plain_bp_sweep_launch(s->CHI, s->D, pm(s), w, s->stream) != cudaSuccess) return d4_fail(s);
        s->launches += 2;
        double acc = 0.0;
        if (!cuda_ok(s, cudaMemcpyAsync(&acc, s->acc, sizeof(double), cudaMemcpyDeviceToHost, s->stream)) ||
            !cuda_ok(s, cudaStreamSynchronize(s->stream)))
            return GTQA_ERR_CUDA;
        cur ^= 1;
        ++it;
        dist = s->m > 0 ? acc / s->m : 0.0;
        if (!(dist == dist)) {
            s->sticky = GTQA_ERR_NUMERIC;
            return GTQA_ERR_NUMERIC;
        }
        if (dist < tol) {
            conv = true;
            break;
        }
    }
    s->cur4 = cur;
    Control ctl;
    int rc;
    if ((rc = read_ctl(s, &ctl))) return rc;
    ctl.cur = cur;
    ctl.last_iters = it;
    ctl.last_dist = dist;
    ctl.not_conv = conv ? 0 : 1;
    ctl.sweeps_total += it;
    ctl.bp_calls += 1;
    ctl.nc_calls += conv ? 0 : 1;
    if (!cuda_ok(s, cudaMemcpyAsync(s->ctl, &ctl, sizeof(Control), cudaMemcpyHostToDevice, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    if (iters_out) *iters_out = it;
    if (dist_out) *dist_out = dist;
    if ((flags & GTQA_BP_REGAUGE) && (rc = d4_regauge(s))) return rc;
    return conv ? GTQA_OK : GTQA_ERR_NOT_CONVERGED;
}

// Unnormalised residual sum of App. C over the 2m directed bonds, added to s->rbuf.
cudaError_t residual_launch(gtqa_state* s) {
    if (s->plain)
        return plain_residual_launch(s->CHI, s->D, pm(s), s->Gamma, s->lam, s->vslots4, s->n, s->rbuf, s->stream);
    return mixed(s) ? AuxUnit<ModeMixed>::residual(s->CHI, s->Gamma, s->lam, s->vert_edges, s->n, s->rbuf, s->stream)
                    : AuxUnit<ModeFP64>::residual(s->CHI, s->Gamma, s->lam, s->vert_edges, s->n, s->rbuf, s->stream);
}

// The regauge policy (Sec. II C) on the plain path: after the gates of each layer the host
// reads R; BP from the warm start and the regauge run only when R > r_threshold.
int d4_anneal_policy(gtqa_state* s, int k_begin, int k_end, int K, double dt, double tol, int max_iter,
                     double r_threshold) {
    int rc;
    long long reg = 0, skip = 0;
    const double thr_sum = r_threshold * 2.0 * (double)s->m;
    for (int k = k_begin; k <= k_end; ++k) {
        const double tau = (double)k / (double)K;
        if ((rc = d4_trotter(s, dt * tau, 0.0, dt * (1.0 - tau)))) return rc;
        if (!cuda_ok(s, cudaMemsetAsync(s->rbuf, 0, sizeof(double), s->stream))) return GTQA_ERR_CUDA;
        if (residual_launch(s) != cudaSuccess) return d4_fail(s);
        s->launches += 1;
        double sum = 0.0;
        if (!cuda_ok(s, cudaMemcpyAsync(&sum, s->rbuf, sizeof(double), cudaMemcpyDeviceToHost, s->stream)) ||
            !cuda_ok(s, cudaStreamSynchronize(s->stream)))
            return GTQA_ERR_CUDA;
        if (!(sum == sum)) {
            s->sticky = GTQA_ERR_NUMERIC;
            return GTQA_ERR_NUMERIC;
        }
        if (sum > thr_sum) {
            rc = d4_bp(s, tol, max_iter, GTQA_BP_DEFAULT, nullptr, nullptr);
            if (rc && rc != GTQA_ERR_NOT_CONVERGED) return rc;
            ++reg;
        } else {
            ++skip;
        }
    }
    Control ctl;
    if ((rc = read_ctl(s, &ctl))) return rc;
    ctl.regauged += reg;
    ctl.reg_skipped += skip;
    if (!cuda_ok(s, cudaMemcpyAsync(s->ctl, &ctl, sizeof(Control), cudaMemcpyHostToDevice, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    return GTQA_OK;
}

// The three phase launches of layers k_begin..k_end (gtqa_anneal's body).
int anneal_launches(gtqa_state* s, int k_begin, int k_end, int K, double dt, double tol, int max_iter) {
    int rc;
    Ctx c = make_ctx(s);
    c.phases = PH_GATES | PH_BP | PH_WARM | PH_REGAUGE;
    c.Ksched = K;
    c.dt = dt;
    c.tol = tol;
    c.max_iter = max_iter;
    for (int k = k_begin; k <= k_end; ++k) {
        c.k0 = c.k1 = k;
        if ((rc = run(s, c, PK_GATES, GTQA_K_TROTTER, s->m)) || (rc = run(s, c, PK_BP, GTQA_K_BP, s->n)) ||
            (rc = run(s, c, PK_REGAUGE, GTQA_K_REGAUGE, s->m)))
            return rc;
        s->layers += 1;
        s->gates += s->m;
    }
    return GTQA_OK;
}

// Work teams per block of a phase kernel in its current shape (the regauge counts its edge
// teams of CHI^2 threads).
int teams_per_block(const gtqa_state* s, int pk) {
    return s->tpb[pk] / std::max(1, pk == PK_REGAUGE ? s->CHI * s->CHI : s->team[pk]);
}

// Zero the per-kernel barrier counters (stream-ordered, between launches).
int zero_barriers(gtqa_state* s) {
    Control* c = s->ctl;
    return cuda_ok(s, cudaMemsetAsync(&c->bar_pk[0], 0, sizeof(c->bar_pk), s->stream)) ? GTQA_OK : GTQA_ERR_CUDA;
}

// As-soon-as-possible layering of a gate list: a gate goes one launch after the latest earlier
// gate that shares a vertex with it, so gates of one launch have disjoint endpoints and every
// pair of gates sharing a vertex keeps its order.  Returns the number of launches.
int gate_layers(int n, const int* edges, int k, const int32_t* edge, int32_t* layer) {
    std::vector<int> depth(n, 0);
    int nl = 0;
    for (int q = 0; q < k; ++q) {
        const int a = edges[2 * (size_t)edge[q]], b = edges[2 * (size_t)edge[q] + 1];
        const int L = std::max(depth[a], depth[b]);
        layer[q] = L;
        depth[a] = depth[b] = L + 1;
        nl = std::max(nl, L + 1);
    }
    return nl;
}

}  // namespace

extern "C" {

void gtqa_options_init(gtqa_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = GTQA_FP64;
    opt->svd_cutoff = 0.0;   // the precision's default (gtqa_create)
    opt->eig_cutoff = 0.0;
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
    if (s->plain) return d4_trotter(s, dt * tau, 0.0, dt * (1.0 - tau));
    Ctx c = make_ctx(s);
    c.phases = PH_GATES;
    c.k0 = c.k1 = 0;
    c.Ksched = 0;
    c.tZ1 = dt * tau;
    c.tX1 = dt * (1.0 - tau);
    if ((rc = run(s, c, PK_GATES, GTQA_K_TROTTER, s->m))) return rc;
    s->layers += 1;
    s->gates += s->m;
    return GTQA_OK;
}

int gtqa_set_grid(gtqa_state* s, const int32_t* grid) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!grid) return GTQA_ERR_INVALID_ARG;
    for (int pk = 0; pk < PK_COUNT; ++pk)
        if (grid[pk] < 1 || grid[pk] > s->nblocks) return GTQA_ERR_INVALID_ARG;
    if (!drop_graph(s)) return GTQA_ERR_CUDA;
    for (int pk = 0; pk < PK_COUNT; ++pk) s->grid[pk] = grid[pk];
    return zero_barriers(s);
}

int gtqa_set_shape(gtqa_state* s, const int32_t* variant) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!variant) return GTQA_ERR_INVALID_ARG;
    if (s->plain) return GTQA_ERR_UNSUPPORTED;
    for (int pk = 0; pk < PK_COUNT; ++pk)
        if (variant[pk] < 0 || variant[pk] >= shape_count(pk)) return GTQA_ERR_INVALID_ARG;
    if (!drop_graph(s)) return GTQA_ERR_CUDA;
    int old[PK_COUNT];
    for (int pk = 0; pk < PK_COUNT; ++pk) old[pk] = s->shape[pk];
    for (int pk = 0; pk < PK_COUNT; ++pk) {
        if ((rc = apply_shape(s, pk, variant[pk])) != GTQA_OK) {
            for (int q = 0; q < pk; ++q) apply_shape(s, q, old[q]);
            return rc;
        }
    }
    return zero_barriers(s);
}

int gtqa_launch_shape(gtqa_state* s, int32_t* out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!out) return GTQA_ERR_INVALID_ARG;
    if (s->plain) return GTQA_ERR_UNSUPPORTED;
    for (int pk = 0; pk < PK_COUNT; ++pk) {
        out[4 * pk + 0] = s->grid[pk];
        out[4 * pk + 1] = s->shape[pk];
        out[4 * pk + 2] = s->tpb[pk];
        out[4 * pk + 3] = s->team[pk];
    }
    return GTQA_OK;
}

int gtqa_autotune(gtqa_state* s, double tau, double dt, double tol, int32_t max_iter, int32_t* grid_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!std::isfinite(tau) || !std::isfinite(dt) || !(tol >= 0.0) || max_iter < 1) return GTQA_ERR_INVALID_ARG;
    if (s->plain) return GTQA_ERR_UNSUPPORTED;
    // snapshot of everything a layer writes, restored before every timed launch and at the end:
    // in one device buffer when it fits in free device memory, else in host memory
    struct Buf { void* p; size_t bytes; std::vector<unsigned char> h; size_t off; };
    const size_t gel = gamma_elems(s), mel = msg_elems(s), eb = elem_bytes(s);
    std::vector<Buf> bufs = {{s->Gamma, gel * eb, {}}, {s->T, gel * eb, {}}, {s->lam, sizeof(double) * s->m * s->CHI, {}},
                             {s->msg[0], mel * eb, {}}, {s->msg[1], mel * eb, {}},
                             {s->X, sizeof(cd) * s->m * 2 * s->CHI * s->CHI, {}},
                             {s->D0, mixed(s) ? sizeof(cf) * mel : 0, {}}, {s->t0, mixed(s) ? sizeof(cd) * 2 * s->m : 0, {}},
                             {s->stats, sizeof(double) * kStats, {}}, {s->ctl, sizeof(Control), {}},
                             {s->acc, sizeof(double) * 6 * s->B, {}}, {s->inst_done, sizeof(int) * s->B, {}},
                             {s->inst_iters, sizeof(int) * s->B, {}}, {s->inst_dist, sizeof(double) * s->B, {}}};
    size_t total = 0;
    for (auto& b : bufs) {
        b.off = total;
        total += (b.bytes + 255) / 256 * 256;
    }
    struct DevSnap {
        unsigned char* p = nullptr;
        ~DevSnap() { if (p) cudaFree(p); }
    } dev;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && total + (256u << 20) < free_b &&
        cudaMalloc((void**)&dev.p, total) != cudaSuccess) {
        dev.p = nullptr;
    }
    cudaGetLastError();
    for (auto& b : bufs) {
        if (!b.bytes) continue;
        cudaError_t e;
        if (dev.p) {
            e = cudaMemcpyAsync(dev.p + b.off, b.p, b.bytes, cudaMemcpyDeviceToDevice, s->stream);
        } else {
            b.h.resize(b.bytes);
            e = cudaMemcpyAsync(b.h.data(), b.p, b.bytes, cudaMemcpyDeviceToHost, s->stream);
        }
        if (!cuda_ok(s, e)) return GTQA_ERR_CUDA;
    }
    if (!cuda_ok(s, cudaStreamSynchronize(s->stream))) return GTQA_ERR_CUDA;
    // the restored control block holds barrier counts of the snapshot's grid sizes: zero them
    auto restore = [&]() {
        for (auto& b : bufs) {
            if (!b.bytes) continue;
            const cudaError_t e = dev.p ? cudaMemcpyAsync(b.p, dev.p + b.off, b.bytes, cudaMemcpyDeviceToDevice, s->stream)
                                        : cudaMemcpyAsync(b.p, b.h.data(), b.bytes, cudaMemcpyHostToDevice, s->stream);
            if (!cuda_ok(s, e)) return false;
        }
        return zero_barriers(s) == GTQA_OK;
    };
    const long long layers = s->layers, gates = s->gates, launches = s->launches;
    const bool prof = s->prof_on;
    s->prof_on = false;
    Ctx c = make_ctx(s);
    c.k0 = c.k1 = 0;
    c.Ksched = 0;
    c.tZ1 = dt * tau;
    c.tX1 = dt * (1.0 - tau);
    c.tol = tol;
    c.max_iter = max_iter;
    // per phase kernel, every launch-shape variant that fits; per variant, the grid candidates
    // are all SMs and, when the work fits in one round of that variant's teams, fewer blocks in
    // steps of 1/8 and the fewest blocks that still cover the work in one round
    if (!drop_graph(s)) return GTQA_ERR_CUDA;
    const int full = s->nblocks;
    const long long units[PK_COUNT] = {s->m, s->n, s->m};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!cuda_ok(s, cudaEventCreate(&e0)) || !cuda_ok(s, cudaEventCreate(&e1))) return GTQA_ERR_CUDA;
    // median of three timed launches of kernel pk with the state's current grid and shape
    auto time_kernel = [&](int pk, float* med) {
        std::vector<float> ts;
        for (int rep = 0; rep < 3; ++rep) {
            if (!restore()) return GTQA_ERR_CUDA;
            // the phases before the timed one, untimed, so that it sees its real inputs
            Ctx ci = c;
            int r;
            ci.phases = PH_GATES;
            if (pk >= PK_BP && (r = run(s, ci, PK_GATES, GTQA_K_TROTTER, s->m))) return r;
            ci.phases = PH_BP | PH_WARM;
            if (pk >= PK_REGAUGE && (r = run(s, ci, PK_BP, GTQA_K_BP, s->n))) return r;
            ci.phases = pk == PK_GATES ? PH_GATES : (pk == PK_BP ? (PH_BP | PH_WARM) : PH_REGAUGE);
            cudaEventRecord(e0, s->stream);
            if ((r = run(s, ci, pk, pk, units[pk]))) return r;
            cudaEventRecord(e1, s->stream);
            float ms = 0.f;
            if (!cuda_ok(s, cudaEventSynchronize(e1)) || !cuda_ok(s, cudaEventElapsedTime(&ms, e0, e1)))
                return GTQA_ERR_CUDA;
            ts.push_back(ms);
        }
        std::sort(ts.begin(), ts.end());
        *med = ts[1];
        return GTQA_OK;
    };
    rc = GTQA_OK;
    for (int pk = 0; pk < PK_COUNT && rc == GTQA_OK; ++pk) {
        float tbest = 3.0e38f;
        int best_g = s->grid[pk], best_v = s->shape[pk];
        const int keep_g = s->grid[pk], keep_v = s->shape[pk];
        for (int v = 0; v < shape_count(pk) && rc == GTQA_OK; ++v) {
            const int arc = apply_shape(s, pk, v);
            if (arc == GTQA_ERR_UNSUPPORTED) continue;   // does not fit on an SM
            if ((rc = arc) != GTQA_OK) break;
            const int tpb_teams = teams_per_block(s, pk);
            // fewer blocks than SMs only pay when the work fits in one round of teams
            std::vector<int> cand = {full};
            const long long one_round = (units[pk] + tpb_teams - 1) / std::max(1, tpb_teams);
            if (one_round < full) {
                for (int q = 7; q >= 4; --q) cand.push_back(std::max(1, full * q / 8));
                if (one_round >= 1) cand.push_back((int)one_round);
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            for (int g : cand) {
                s->grid[pk] = g;
                float med = 0.f;
                if ((rc = time_kernel(pk, &med)) != GTQA_OK) break;
                if (med < tbest) {
                    tbest = med;
                    best_g = g;
                    best_v = v;
                }
            }
        }
        const int arc = apply_shape(s, pk, rc == GTQA_OK ? best_v : keep_v);
        if (rc == GTQA_OK) rc = arc;
        s->grid[pk] = rc == GTQA_OK ? best_g : keep_g;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const bool ok = restore() && cuda_ok(s, cudaStreamSynchronize(s->stream));
    s->layers = layers;
    s->gates = gates;
    s->launches = launches;
    s->prof_on = prof;
    if (rc != GTQA_OK) return rc;
    if (!ok) return GTQA_ERR_CUDA;
    if (grid_out)
        for (int pk = 0; pk < PK_COUNT; ++pk) grid_out[pk] = s->grid[pk];
    return GTQA_OK;
}

int gtqa_trotter_split(gtqa_state* s, double t_Z, double t_X_pre, double t_X_post) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!std::isfinite(t_Z) || !std::isfinite(t_X_pre) || !std::isfinite(t_X_post)) return GTQA_ERR_INVALID_ARG;
    if (s->plain) return d4_trotter(s, t_Z, t_X_pre, t_X_post);
    Ctx c = make_ctx(s);
    c.phases = PH_GATES;
    c.k0 = c.k1 = 0;
    c.Ksched = 0;
    c.tZ1 = t_Z;
    c.tX1 = t_X_post;
    c.tXpre1 = t_X_pre;
    if ((rc = run(s, c, PK_GATES, GTQA_K_TROTTER, s->m))) return rc;
    s->layers += 1;
    s->gates += s->m;
    return GTQA_OK;
}

int gtqa_bp_sweep(gtqa_state* s, double tol, int32_t max_iter, uint32_t flags, int32_t* iters_out,
                  double* dist_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (max_iter < 1 || !(tol >= 0.0) || (flags & ~3u)) return GTQA_ERR_INVALID_ARG;
    if (s->plain) return d4_bp(s, tol, max_iter, flags, iters_out, dist_out);
    Ctx c = make_ctx(s);
    c.phases = PH_BP | ((flags & GTQA_BP_WARM_START) ? PH_WARM : 0u);
    c.k0 = c.k1 = 0;
    c.tol = tol;
    c.max_iter = max_iter;
    if ((rc = run(s, c, PK_BP, GTQA_K_BP, s->n))) return rc;
    if ((flags & GTQA_BP_REGAUGE) && (rc = run(s, c, PK_REGAUGE, GTQA_K_REGAUGE, s->m))) return rc;
    Control ctl;
    if ((rc = read_ctl(s, &ctl))) return rc;
    if (iters_out) *iters_out = ctl.last_iters;
    if (dist_out) *dist_out = ctl.last_dist;
    if (!(ctl.last_dist == ctl.last_dist)) {
        s->sticky = GTQA_ERR_NUMERIC;
        return GTQA_ERR_NUMERIC;
    }
    return ctl.not_conv > 0 ? GTQA_ERR_NOT_CONVERGED : GTQA_OK;
}

int gtqa_sample(gtqa_state* s, int32_t k, const int32_t* order, const double* u, double tol, int32_t max_iter,
                int8_t* x_out, double* p_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (k < 0 || k > s->n || (k > 0 && (!order || !u)) || !x_out || max_iter < 1 || !(tol >= 0.0))
        return GTQA_ERR_INVALID_ARG;
    std::vector<char> seen(s->n, 0);
    for (int q = 0; q < k; ++q) {
        if (order[q] < 0 || order[q] >= s->n || seen[order[q]] || !(u[q] >= 0.0 && u[q] <= 1.0))
            return GTQA_ERR_INVALID_ARG;
        seen[order[q]] = 1;
    }
    if (!cuda_ok(s, cudaMemsetAsync(s->xs, 0, (size_t)s->n, s->stream))) return GTQA_ERR_CUDA;
    Ctx c = make_ctx(s);
    c.phases = PH_BP | PH_WARM;
    c.k0 = c.k1 = 0;
    c.tol = tol;
    c.max_iter = max_iter;
    for (int q = 0; q < k && s->plain; ++q) {
        if (plain_sample_launch(s->CHI, s->D, pm(s), s->Gamma, s->lam, s->vslots4, order[q], u[q], q, s->xs, s->ps,
                                s->stream) != cudaSuccess)
            return d4_fail(s);
        s->launches += 1;
        // the projection leaves the Vidal gauge: BP from the warm start, then the regauge
        rc = d4_bp(s, tol, max_iter, GTQA_BP_WARM_START | GTQA_BP_REGAUGE, nullptr, nullptr);
        if (rc && rc != GTQA_ERR_NOT_CONVERGED) return rc;
    }
    for (int q = 0; q < k && !s->plain; ++q) {
        const cudaError_t e = mixed(s) ? AuxUnit<ModeMixed>::sample(s->CHI, s->Gamma, s->lam, s->vert_edges, order[q], u[q], q,
                                                             s->xs, s->ps, s->stream)
                                       : AuxUnit<ModeFP64>::sample(s->CHI, s->Gamma, s->lam, s->vert_edges, order[q], u[q], q,
                                                            s->xs, s->ps, s->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->sticky = GTQA_ERR_CUDA;
            return GTQA_ERR_CUDA;
        }
        s->launches += 1;
        // the projection leaves the Vidal gauge: BP from the warm start, then the regauge
        if ((rc = run(s, c, PK_BP, GTQA_K_BP, s->n)) || (rc = run(s, c, PK_REGAUGE, GTQA_K_REGAUGE, s->m))) return rc;
    }
    Control ctl;
    if ((rc = read_ctl(s, &ctl))) return rc;
    if (!cuda_ok(s, cudaMemcpyAsync(x_out, s->xs, (size_t)s->n, cudaMemcpyDeviceToHost, s->stream)) ||
        (p_out && k > 0 && !cuda_ok(s, cudaMemcpyAsync(p_out, s->ps, sizeof(double) * k, cudaMemcpyDeviceToHost, s->stream))) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    return GTQA_OK;
}

int gtqa_apply_gates(gtqa_state* s, int32_t k, const int32_t* edge, const double* U) {
    int rc = check_state(s);
    if (rc) return rc;
    if (s->plain && s->CHI == 16) return GTQA_ERR_UNSUPPORTED;   // a 64 x 64 core per gate
    if (k < 0 || (k > 0 && (!edge || !U))) return GTQA_ERR_INVALID_ARG;
    for (int q = 0; q < k; ++q) {
        if (edge[q] < 0 || edge[q] >= s->m) return GTQA_ERR_INVALID_ARG;
        for (int t = 0; t < 32; ++t)
            if (!std::isfinite(U[32 * (size_t)q + t])) return GTQA_ERR_INVALID_ARG;
    }
    if (k == 0) return GTQA_OK;
    std::vector<int> lay(k);
    const int nl = gate_layers(s->n, s->h_edges.data(), k, edge, lay.data());
    std::vector<int> off(nl + 1, 0);
    for (int q = 0; q < k; ++q) ++off[lay[q] + 1];
    for (int L = 0; L < nl; ++L) off[L + 1] += off[L];
    std::vector<int> fill(off.begin(), off.end() - 1), es(k);
    std::vector<double> Us(32 * (size_t)k);
    for (int q = 0; q < k; ++q) {
        const int pos = fill[lay[q]]++;
        es[pos] = edge[q];
        std::memcpy(&Us[32 * (size_t)pos], U + 32 * (size_t)q, 32 * sizeof(double));
    }
    if ((rc = grow_pair(s, &s->gate_edge, &s->gate_U, 16, s->gate_cap, (size_t)k))) return rc;
    if (!cuda_ok(s, cudaMemcpyAsync(s->gate_edge, es.data(), sizeof(int) * k, cudaMemcpyHostToDevice, s->stream)) ||
        !cuda_ok(s, cudaMemcpyAsync(s->gate_U, Us.data(), sizeof(double) * Us.size(), cudaMemcpyHostToDevice, s->stream)))
        return GTQA_ERR_CUDA;
    for (int L = 0; L < nl; ++L) {
        GenArgs a;
        a.Gamma = s->Gamma;
        a.lam = s->lam;
        a.edge_info = s->edge_info;
        a.vert_edges = s->plain ? s->vslots4 : s->vert_edges;
        a.gate_edge = s->gate_edge + off[L];
        a.gate_U = s->gate_U + 16 * (size_t)off[L];
        a.count = off[L + 1] - off[L];
        a.stats = s->stats;
        a.chi = s->chi;
        a.svd_cut = s->svd_cutoff;
        const cudaError_t e = s->plain    ? plain_general_gates_launch(s->CHI, s->D, pm(s), a, s->stream)
                              : mixed(s) ? GeneralUnit<ModeMixed>::gates(s->CHI, a, s->stream)
                                         : GeneralUnit<ModeFP64>::gates(s->CHI, a, s->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->sticky = GTQA_ERR_CUDA;
            return GTQA_ERR_CUDA;
        }
        s->launches += 1;
    }
    s->gates += k;
    return GTQA_OK;
}

int gtqa_apply_single_qubit_gates(gtqa_state* s, int32_t k, const int32_t* vertex, const double* W) {
    int rc = check_state(s);
    if (rc) return rc;
    if (k < 0 || (k > 0 && (!vertex || !W))) return GTQA_ERR_INVALID_ARG;
    for (int q = 0; q < k; ++q) {
        if (vertex[q] < 0 || vertex[q] >= s->n) return GTQA_ERR_INVALID_ARG;
        for (int t = 0; t < 8; ++t)
            if (!std::isfinite(W[8 * (size_t)q + t])) return GTQA_ERR_INVALID_ARG;
    }
    if (k == 0) return GTQA_OK;
    // gates on one vertex compose in list order: W_total = W_last ... W_first
    using cx = std::complex<double>;
    std::vector<int> slot(s->n, -1), vs;
    std::vector<cx> acc;
    for (int q = 0; q < k; ++q) {
        const int a = vertex[q];
        if (slot[a] < 0) {
            slot[a] = (int)vs.size();
            vs.push_back(a);
            acc.insert(acc.end(), {cx(1, 0), cx(0, 0), cx(0, 0), cx(1, 0)});
        }
        cx* T = &acc[4 * (size_t)slot[a]];
        const double* w = W + 8 * (size_t)q;
        const cx w00(w[0], w[1]), w01(w[2], w[3]), w10(w[4], w[5]), w11(w[6], w[7]);
        const cx t00 = w00 * T[0] + w01 * T[2], t01 = w00 * T[1] + w01 * T[3];
        const cx t10 = w10 * T[0] + w11 * T[2], t11 = w10 * T[1] + w11 * T[3];
        T[0] = t00;
        T[1] = t01;
        T[2] = t10;
        T[3] = t11;
    }
    const int cnt = (int)vs.size();
    std::vector<double> Wd(8 * (size_t)cnt);
    for (size_t t = 0; t < 4 * (size_t)cnt; ++t) {
        Wd[2 * t] = acc[t].real();
        Wd[2 * t + 1] = acc[t].imag();
    }
    if ((rc = grow_pair(s, &s->sq_vertex, &s->sq_W, 4, s->sq_cap, (size_t)cnt))) return rc;
    if (!cuda_ok(s, cudaMemcpyAsync(s->sq_vertex, vs.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s->stream)) ||
        !cuda_ok(s, cudaMemcpyAsync(s->sq_W, Wd.data(), sizeof(double) * Wd.size(), cudaMemcpyHostToDevice, s->stream)))
        return GTQA_ERR_CUDA;
    const cudaError_t e = s->plain ? plain_single_gates_launch(s->CHI, s->D, pm(s), s->Gamma, s->sq_vertex, s->sq_W,
                                                               cnt, s->stream)
                          : mixed(s) ? GeneralUnit<ModeMixed>::single(s->CHI, s->Gamma, s->sq_vertex, s->sq_W, cnt, s->stream)
                                     : GeneralUnit<ModeFP64>::single(s->CHI, s->Gamma, s->sq_vertex, s->sq_W, cnt, s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->sticky = GTQA_ERR_CUDA;
        return GTQA_ERR_CUDA;
    }
    s->launches += 1;
    return GTQA_OK;
}

int gtqa_regauge(gtqa_state* s) {
    int rc = check_state(s);
    if (rc) return rc;
    if (s->plain) return d4_regauge(s);
    Ctx c = make_ctx(s);
    c.phases = PH_REGAUGE;
    c.k0 = c.k1 = 0;
    return run(s, c, PK_REGAUGE, GTQA_K_REGAUGE, s->m);
}

int gtqa_anneal(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol, int32_t max_iter) {
    int rc = check_state(s);
    if (rc) return rc;
    if (K < 1 || k_begin < 1 || k_end < k_begin || k_end > K || !std::isfinite(dt) || !(tol >= 0.0) || max_iter < 1)
        return GTQA_ERR_INVALID_ARG;
    if (s->plain) {
        for (int k = k_begin; k <= k_end; ++k) {
            const double tau = (double)k / (double)K;
            if ((rc = d4_trotter(s, dt * tau, 0.0, dt * (1.0 - tau)))) return rc;
            rc = d4_bp(s, tol, max_iter, GTQA_BP_DEFAULT, nullptr, nullptr);
            if (rc && rc != GTQA_ERR_NOT_CONVERGED) return rc;
        }
        return GTQA_OK;
    }
    return anneal_launches(s, k_begin, k_end, K, dt, tol, max_iter);
}

int gtqa_anneal_policy(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                       int32_t max_iter, double r_threshold) {
    int rc = check_state(s);
    if (rc) return rc;
    if (K < 1 || k_begin < 1 || k_end < k_begin || k_end > K || !std::isfinite(dt) || !(tol >= 0.0) || max_iter < 1 ||
        std::isnan(r_threshold))
        return GTQA_ERR_INVALID_ARG;
    if (s->plain) return d4_anneal_policy(s, k_begin, k_end, K, dt, tol, max_iter, r_threshold);
    Ctx c = make_ctx(s);
    c.Ksched = K;
    c.dt = dt;
    c.tol = tol;
    c.max_iter = max_iter;
    for (int k = k_begin; k <= k_end; ++k) {
        c.k0 = c.k1 = k;
        c.phases = PH_GATES;
        c.rgate = nullptr;
        if ((rc = run(s, c, PK_GATES, GTQA_K_TROTTER, s->m))) return rc;
        // R of App. C (unnormalised sum over the 2m directed bonds) on the device
        if (!cuda_ok(s, cudaMemsetAsync(s->rbuf, 0, sizeof(double), s->stream))) return GTQA_ERR_CUDA;
        const cudaError_t e = residual_launch(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->sticky = GTQA_ERR_CUDA;
            return GTQA_ERR_CUDA;
        }
        s->launches += 1;
        c.rgate = s->rbuf;
        c.rthr_sum = r_threshold * 2.0 * (double)s->m;
        c.phases = PH_BP | PH_WARM;
        if ((rc = run(s, c, PK_BP, GTQA_K_BP, s->n))) return rc;
        c.phases = PH_REGAUGE;
        if ((rc = run(s, c, PK_REGAUGE, GTQA_K_REGAUGE, s->m))) return rc;
        s->layers += 1;
        s->gates += s->m;
    }
    return GTQA_OK;
}

int gtqa_regauge_counts(gtqa_state* s, int64_t* regauged, int64_t* skipped) {
    int rc = check_state(s);
    if (rc) return rc;
    Control ctl;
    if ((rc = read_ctl(s, &ctl))) return rc;
    if (regauged) *regauged = ctl.regauged;
    if (skipped) *skipped = ctl.reg_skipped;
    return GTQA_OK;
}

int gtqa_anneal_graph(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                      int32_t max_iter) {
    int rc = check_state(s);
    if (rc) return rc;
    if (K < 1 || k_begin < 1 || k_end < k_begin || k_end > K || !std::isfinite(dt) || !(tol >= 0.0) || max_iter < 1)
        return GTQA_ERR_INVALID_ARG;
    if (s->plain) return GTQA_ERR_UNSUPPORTED;
    const bool same = s->gexec && s->gK == K && s->gdt == dt && s->gtol == tol && s->gmi == max_iter;
    if (!same) {
        if (!graph_collect(s)) return GTQA_ERR_CUDA;
        if (s->gexec) cudaGraphExecDestroy(s->gexec);
        if (s->graph) cudaGraphDestroy(s->graph);
        s->gexec = nullptr;
        s->graph = nullptr;
        const bool prof = s->prof_on;
        for (cudaEvent_t& e : s->gev)
            if (!e && !cuda_ok(s, cudaEventCreate(&e))) return GTQA_ERR_CUDA;
        // capture on a private stream (the state's own stream may be the legacy default stream)
        cudaStream_t cs = nullptr;
        if (!cuda_ok(s, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) return GTQA_ERR_CUDA;
        const cudaStream_t own = s->stream;
        const long long launches = s->launches;
        s->stream = cs;
        s->prof_on = false;   // the library's per-launch events are replaced by the graph's own
        Ctx c = make_ctx(s);
        c.phases = PH_GATES | PH_BP | PH_WARM | PH_REGAUGE;
        c.Ksched = K;
        c.dt = dt;
        c.tol = tol;
        c.max_iter = max_iter;
        c.kdev = s->kdev;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int lrc = e == cudaSuccess ? GTQA_OK : GTQA_ERR_CUDA;
        const int pks[3] = {PK_GATES, PK_BP, PK_REGAUGE};
        const long long units[3] = {s->m, s->n, s->m};
        // external event nodes around the three launches: every replay re-records them, and they
        // are read when the profiler is on
        for (int q = 0; q < 3 && lrc == GTQA_OK; ++q) {
            if (cudaEventRecordWithFlags(s->gev[q], cs, cudaEventRecordExternal) != cudaSuccess) lrc = GTQA_ERR_CUDA;
            if (lrc == GTQA_OK) lrc = run(s, c, pks[q], pks[q], units[q]);
        }
        if (lrc == GTQA_OK && cudaEventRecordWithFlags(s->gev[3], cs, cudaEventRecordExternal) != cudaSuccess)
            lrc = GTQA_ERR_CUDA;
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cs, &g) : e;
        s->stream = own;
        s->prof_on = prof;
        s->launches = launches;
        cudaStreamDestroy(cs);
        if (lrc == GTQA_OK && e2 == cudaSuccess && g) e = cudaGraphInstantiate(&s->gexec, g, 0);
        else e = e2 != cudaSuccess ? e2 : cudaErrorUnknown;
        if (e != cudaSuccess || lrc != GTQA_OK) {
            if (g) cudaGraphDestroy(g);
            s->gexec = nullptr;
            cudaGetLastError();
            // a failed capture leaves the state usable: nothing was launched
            if (s->sticky == GTQA_ERR_CUDA) s->sticky = GTQA_OK;
            return GTQA_ERR_UNSUPPORTED;
        }
        s->graph = g;
        s->gK = K;
        s->gdt = dt;
        s->gtol = tol;
        s->gmi = max_iter;
    }
    // the captured layer reads its index from *kdev and its regauge stores the next one
    set_layer_kernel<<<1, 1, 0, s->stream>>>(s->kdev, k_begin);
    if (!cuda_ok(s, cudaGetLastError())) return GTQA_ERR_CUDA;
    s->launches += 1;
    for (int k = k_begin; k <= k_end; ++k) {
        // each replay re-records the events: a profiled replay's are read before the next one
        if (!graph_collect(s)) return GTQA_ERR_CUDA;
        if (!cuda_ok(s, cudaGraphLaunch(s->gexec, s->stream))) return GTQA_ERR_CUDA;
        s->layers += 1;
        s->gates += s->m;
        s->launches += 3;
        s->gpending = s->prof_on;
    }
    return GTQA_OK;
}

int gtqa_anneal_ex(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                   int32_t max_iter, int32_t order, const uint8_t* reverse) {
    int rc = check_state(s);
    if (rc) return rc;
    if (K < 1 || k_begin < 1 || k_end < k_begin || k_end > K || !std::isfinite(dt) || !(tol >= 0.0) || max_iter < 1 ||
        (order != GTQA_TROTTER_FIRST && order != GTQA_TROTTER_SYMMETRIC) ||
        (order == GTQA_TROTTER_SYMMETRIC && reverse))
        return GTQA_ERR_INVALID_ARG;
    if (s->plain) {
        for (int k = k_begin; k <= k_end; ++k) {
            const double tau = (double)k / (double)K, tZ = dt * tau, tX = dt * (1.0 - tau);
            const bool rev = reverse && reverse[k - k_begin];
            const double pre = order == GTQA_TROTTER_SYMMETRIC ? 0.5 * tX : (rev ? tX : 0.0);
            const double post = order == GTQA_TROTTER_SYMMETRIC ? 0.5 * tX : (rev ? 0.0 : tX);
            if ((rc = d4_trotter(s, tZ, pre, post))) return rc;
            rc = d4_bp(s, tol, max_iter, GTQA_BP_DEFAULT, nullptr, nullptr);
            if (rc && rc != GTQA_ERR_NOT_CONVERGED) return rc;
        }
        return GTQA_OK;
    }
    Ctx c = make_ctx(s);
    c.phases = PH_GATES | PH_BP | PH_WARM | PH_REGAUGE;
    c.Ksched = 0;
    c.tol = tol;
    c.max_iter = max_iter;
    for (int k = k_begin; k <= k_end; ++k) {
        // the layer's angles are formed here, as in the oracle's product_formula
        const double tau = (double)k / (double)K, tZ = dt * tau, tX = dt * (1.0 - tau);
        const bool rev = reverse && reverse[k - k_begin];
        c.k0 = c.k1 = k;
        c.tZ1 = tZ;
        if (order == GTQA_TROTTER_SYMMETRIC) {
            c.tXpre1 = 0.5 * tX;
            c.tX1 = 0.5 * tX;
        } else {
            c.tXpre1 = rev ? tX : 0.0;
            c.tX1 = rev ? 0.0 : tX;
        }
        if ((rc = run(s, c, PK_GATES, GTQA_K_TROTTER, s->m)) || (rc = run(s, c, PK_BP, GTQA_K_BP, s->n)) ||
            (rc = run(s, c, PK_REGAUGE, GTQA_K_REGAUGE, s->m)))
            return rc;
        s->layers += 1;
        s->gates += s->m;
    }
    return GTQA_OK;
}

int gtqa_entropy(gtqa_state* s, const uint8_t* cut, double* S_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!S_out || (s->m > 0 && !cut)) return GTQA_ERR_INVALID_ARG;
    if (s->m == 0) {
        *S_out = 0.0;
        return GTQA_OK;
    }
    if (!cuda_ok(s, cudaMemcpyAsync(s->cutbuf, cut, (size_t)s->m, cudaMemcpyDefault, s->stream)) ||
        !cuda_ok(s, cudaMemsetAsync(s->rbuf, 0, sizeof(double), s->stream)))
        return GTQA_ERR_CUDA;
    entropy_kernel<<<(s->m + 255) / 256, 256, 0, s->stream>>>(s->lam, s->cutbuf, (int)s->m, s->CHI, s->rbuf);
    if (!cuda_ok(s, cudaGetLastError())) return GTQA_ERR_CUDA;
    s->launches += 1;
    double v = 0.0;
    if (!cuda_ok(s, cudaMemcpyAsync(&v, s->rbuf, sizeof(double), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    *S_out = v;
    return (v == v) ? GTQA_OK : GTQA_ERR_NUMERIC;
}

int gtqa_spectral_bipartition(int32_t n, int32_t m, const int32_t* edges, uint8_t* side_out, uint8_t* cut_out,
                              double* ratio_out) {
    if (n < 2 || m < 0 || (m > 0 && !edges) || !side_out) return GTQA_ERR_INVALID_ARG;
    std::vector<int> deg(n, 0);
    for (int e = 0; e < m; ++e) {
        const int u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return GTQA_ERR_INVALID_ARG;
        ++deg[u];
        ++deg[v];
    }
    std::vector<int> off(n + 1, 0), adj(2 * (size_t)m);
    for (int a = 0; a < n; ++a) off[a + 1] = off[a] + deg[a];
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int e = 0; e < m; ++e) {
            const int u = edges[2 * e], v = edges[2 * e + 1];
            adj[fill[u]++] = v;
            adj[fill[v]++] = u;
        }
    }
    auto laplacian = [&](const std::vector<double>& x, std::vector<double>& y) {
        for (int a = 0; a < n; ++a) {
            double t = deg[a] * x[a];
            for (int q = off[a]; q < off[a + 1]; ++q) t -= x[adj[q]];
            y[a] = t;
        }
    };
    auto project = [&](std::vector<double>& x) {   // remove the constant vector
        double mean = 0.0;
        for (double v : x) mean += v;
        mean /= n;
        for (double& v : x) v -= mean;
    };
    // Lanczos on L = D - A restricted to the complement of the constant vector, with full
    // reorthogonalisation; the Krylov space is the whole complement for n <= 241
    const int kmax = std::min(n - 1, 240);
    std::vector<std::vector<double>> Q;
    Q.reserve(kmax);
    std::vector<double> al, be, w(n);
    std::vector<double> q(n);
    unsigned long long st = 0x9E3779B97F4A7C15ull;
    for (int a = 0; a < n; ++a) {   // deterministic start vector (xorshift64)
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        q[a] = (double)(st >> 11) / 9007199254740992.0 - 0.5;
    }
    project(q);
    double nq = 0.0;
    for (double v : q) nq += v * v;
    nq = std::sqrt(nq);
    if (!(nq > 0.0)) return GTQA_ERR_NUMERIC;
    for (double& v : q) v /= nq;
    for (int j = 0; j < kmax; ++j) {
        Q.push_back(q);
        laplacian(Q[j], w);
        double aj = 0.0;
        for (int a = 0; a < n; ++a) aj += Q[j][a] * w[a];
        al.push_back(aj);
        for (int pass = 0; pass < 2; ++pass) {
            project(w);
            for (int i = 0; i <= j; ++i) {
                double c = 0.0;
                for (int a = 0; a < n; ++a) c += Q[i][a] * w[a];
                for (int a = 0; a < n; ++a) w[a] -= c * Q[i][a];
            }
        }
        double bj = 0.0;
        for (double v : w) bj += v * v;
        bj = std::sqrt(bj);
        if (j + 1 == kmax || bj < 1e-10 * std::max(1.0, std::fabs(aj))) break;
        be.push_back(bj);
        for (int a = 0; a < n; ++a) q[a] = w[a] / bj;
    }
    std::vector<double> y;
    tridiag_min_eigvec(al, be, y);
    std::vector<double> f(n, 0.0);
    for (size_t i = 0; i < y.size(); ++i)
        for (int a = 0; a < n; ++a) f[a] += y[i] * Q[i][a];
    int big = 0;
    for (int a = 1; a < n; ++a)
        if (std::fabs(f[a]) > std::fabs(f[big])) big = a;
    if (f[big] < 0)
        for (double& v : f) v = -v;
    std::vector<int> order(n);
    for (int a = 0; a < n; ++a) order[a] = a;
    std::sort(order.begin(), order.end(), [&](int x, int z) { return f[x] < f[z] || (f[x] == f[z] && x < z); });
    std::vector<char> inA(n, 0);
    long long cutsz = 0, best_s = 1;
    double best = HUGE_VAL;
    for (int sz = 1; sz < n; ++sz) {
        const int u = order[sz - 1];
        int inside = 0;
        for (int qq = off[u]; qq < off[u + 1]; ++qq) inside += inA[adj[qq]];
        cutsz += deg[u] - 2 * inside;
        inA[u] = 1;
        const double r = (double)cutsz / ((double)sz * (double)(n - sz));
        if (r < best) {
            best = r;
            best_s = sz;
        }
    }
    for (int a = 0; a < n; ++a) side_out[a] = 0;
    for (long long i = 0; i < best_s; ++i) side_out[order[i]] = 1;
    if (cut_out)
        for (int e = 0; e < m; ++e) cut_out[e] = side_out[edges[2 * e]] != side_out[edges[2 * e + 1]];
    if (ratio_out) *ratio_out = best;
    return GTQA_OK;
}

int gtqa_residual(gtqa_state* s, double* R_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!R_out) return GTQA_ERR_INVALID_ARG;
    if (!cuda_ok(s, cudaMemsetAsync(s->rbuf, 0, sizeof(double), s->stream))) return GTQA_ERR_CUDA;
    const cudaError_t e = residual_launch(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->sticky = GTQA_ERR_CUDA;
        return GTQA_ERR_CUDA;
    }
    s->launches += 1;
    double sum = 0.0;
    if (!cuda_ok(s, cudaMemcpyAsync(&sum, s->rbuf, sizeof(double), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    *R_out = s->m > 0 ? sum / (2.0 * (double)s->m) : 0.0;
    return (sum == sum) ? GTQA_OK : GTQA_ERR_NUMERIC;
}

int gtqa_marginals(gtqa_state* s, double* rho_out, int8_t* sign_out) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!rho_out) return GTQA_ERR_INVALID_ARG;
    {
        ProfScope ps(s, GTQA_K_MARGINALS, s->n);
        const cudaError_t e =
            s->plain ? plain_marginals_launch(s->CHI, s->D, pm(s), s->Gamma, s->lam, s->vslots4, s->n, s->rho,
                                              s->sign, s->flags, s->stream)
            : mixed(s) ? AuxUnit<ModeMixed>::marginals(s->CHI, s->Gamma, s->lam, s->vert_edges, s->n, s->rho, s->sign,
                                                s->flags, s->stream)
                       : AuxUnit<ModeFP64>::marginals(s->CHI, s->Gamma, s->lam, s->vert_edges, s->n, s->rho, s->sign,
                                               s->flags, s->stream);
        if (!cuda_ok(s, e)) return GTQA_ERR_CUDA;
        s->launches += 1;
    }
    int hf[4] = {0, 0, 0, 0};
    if (!cuda_ok(s, cudaMemcpyAsync(rho_out, s->rho, sizeof(cd) * 4 * (size_t)s->n, cudaMemcpyDefault, s->stream)))
        return GTQA_ERR_CUDA;
    if (sign_out && !cuda_ok(s, cudaMemcpyAsync(sign_out, s->sign, (size_t)s->n, cudaMemcpyDefault, s->stream)))
        return GTQA_ERR_CUDA;
    if (!cuda_ok(s, cudaMemcpyAsync(hf, s->flags, sizeof(hf), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    if (hf[0]) {
        s->sticky = GTQA_ERR_NUMERIC;
        return GTQA_ERR_NUMERIC;
    }
    return GTQA_OK;
}

int gtqa_stats(gtqa_state* s, gtqa_stats_t* out) {
    if (!s || !out) return GTQA_ERR_INVALID_ARG;
    double st[kStats] = {};
    Control ctl;
    if (!cuda_ok(s, cudaMemcpyAsync(st, s->stats, sizeof(st), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaMemcpyAsync(&ctl, s->ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s->stream)) ||
        !cuda_ok(s, cudaStreamSynchronize(s->stream)))
        return GTQA_ERR_CUDA;
    out->layers = s->layers;
    out->gates = s->gates;
    out->last_bp_iters = ctl.last_iters;
    out->not_converged = ctl.not_conv;
    out->last_bp_dist = ctl.last_dist;
    out->discarded_weight = st[0];
    out->log_fidelity = st[1];
    out->svd_pairs = (int64_t)st[2];
    out->svd_rotations = (int64_t)st[3];
    out->bp_sweeps = ctl.sweeps_total;
    out->launches = s->launches;
    out->bp_calls = ctl.bp_calls;
    out->bp_not_converged_calls = ctl.nc_calls;
    out->bp_exact_passes = ctl.exact_passes;
    out->regauge_svd_sweeps = (int64_t)st[4];
    out->gate_svd_sweeps_max = ctl.gate_sw_max;
    out->gate_svd_sweeps32_max = ctl.gate_sw32_max;
    out->regauge_svd_sweeps_max = ctl.reg_sw_max;
    out->regauge_svd_sweeps32_max = ctl.reg_sw32_max;
    return ctl.err ? ctl.err : GTQA_OK;
}

int gtqa_get_state(gtqa_state* s, double* gamma_out, double* lambda_out, double* messages_out) {
    int rc = check_state(s);
    if (rc) return rc;
    Control ctl;
    if ((rc = read_ctl(s, &ctl))) return rc;
    const cudaStream_t st = s->stream;
    const size_t gel = gamma_elems(s), mel = msg_elems(s);
    if (gamma_out) {
        if (!f32store(s)) {
            if (!cuda_ok(s, cudaMemcpyAsync(gamma_out, s->Gamma, gel * sizeof(cd), cudaMemcpyDefault, st)))
                return GTQA_ERR_CUDA;
        } else {
            std::vector<cf> g(gel);
            std::vector<cd> g2(gel);
            if (!cuda_ok(s, cudaMemcpyAsync(g.data(), s->Gamma, gel * sizeof(cf), cudaMemcpyDeviceToHost, st)) ||
                !cuda_ok(s, cudaStreamSynchronize(st)))
                return GTQA_ERR_CUDA;
            for (size_t i = 0; i < gel; ++i) g2[i] = cd{(double)g[i].x, (double)g[i].y};
            if (!cuda_ok(s, cudaMemcpyAsync(gamma_out, g2.data(), gel * sizeof(cd), cudaMemcpyDefault, st)) ||
                !cuda_ok(s, cudaStreamSynchronize(st)))
                return GTQA_ERR_CUDA;
        }
    }
    if (lambda_out &&
        !cuda_ok(s, cudaMemcpyAsync(lambda_out, s->lam, sizeof(double) * s->m * s->CHI, cudaMemcpyDefault, st)))
        return GTQA_ERR_CUDA;
    if (messages_out) {
        std::vector<cd> mm;
        if ((rc = read_messages(s, ctl.cur, mm))) return rc;
        if (!cuda_ok(s, cudaMemcpyAsync(messages_out, mm.data(), mel * sizeof(cd), cudaMemcpyDefault, st)))
            return GTQA_ERR_CUDA;
    }
    if (!cuda_ok(s, cudaStreamSynchronize(st))) return GTQA_ERR_CUDA;
    return GTQA_OK;
}

int gtqa_set_state(gtqa_state* s, const double* gamma, const double* lambda, const double* messages) {
    int rc = check_state(s);
    if (rc) return rc;
    if (!gamma || !lambda || !messages) return GTQA_ERR_INVALID_ARG;
    Control ctl;
    if ((rc = read_ctl(s, &ctl))) return rc;
    const cudaStream_t st = s->stream;
    const size_t gel = gamma_elems(s), mel = msg_elems(s);
    const int CC = s->CHI * s->CHI;
    std::vector<cd> g(gel), mm(mel);
    std::vector<double> L((size_t)s->m * s->CHI);
    if (!cuda_ok(s, cudaMemcpyAsync(g.data(), gamma, gel * sizeof(cd), cudaMemcpyDefault, st)) ||
        !cuda_ok(s, cudaMemcpyAsync(L.data(), lambda, L.size() * sizeof(double), cudaMemcpyDefault, st)) ||
        !cuda_ok(s, cudaMemcpyAsync(mm.data(), messages, mel * sizeof(cd), cudaMemcpyDefault, st)) ||
        !cuda_ok(s, cudaStreamSynchronize(st)))
        return GTQA_ERR_CUDA;
    for (double x : L)
        if (!(x >= 0.0) || !std::isfinite(x)) return GTQA_ERR_INVALID_ARG;
    if (!f32store(s)) {
        if (!cuda_ok(s, cudaMemcpyAsync(s->Gamma, g.data(), gel * sizeof(cd), cudaMemcpyHostToDevice, st)) ||
            !cuda_ok(s, cudaMemcpyAsync(s->msg[ctl.cur], mm.data(), mel * sizeof(cd), cudaMemcpyHostToDevice, st)))
            return GTQA_ERR_CUDA;
    } else if (abs32(s)) {
        std::vector<cf> gf(gel), mf(mel);
        for (size_t i = 0; i < gel; ++i) gf[i] = cf{(float)g[i].x, (float)g[i].y};
        for (size_t i = 0; i < mel; ++i) mf[i] = cf{(float)mm[i].x, (float)mm[i].y};
        if (!cuda_ok(s, cudaMemcpyAsync(s->Gamma, gf.data(), gel * sizeof(cf), cudaMemcpyHostToDevice, st)) ||
            !cuda_ok(s, cudaMemcpyAsync(s->msg[ctl.cur], mf.data(), mel * sizeof(cf), cudaMemcpyHostToDevice, st)) ||
            !cuda_ok(s, cudaStreamSynchronize(st)))
            return GTQA_ERR_CUDA;
    } else {
        std::vector<cf> gf(gel), df(mel);
        for (size_t i = 0; i < gel; ++i) gf[i] = cf{(float)g[i].x, (float)g[i].y};
        for (int e = 0; e < s->m; ++e) {
            double sum = 0.0;
            for (int q = 0; q < s->CHI; ++q) sum += L[(size_t)e * s->CHI + q];
            for (int x = 0; x < 2; ++x)
                for (int r = 0; r < CC; ++r) {
                    const size_t idx = ((size_t)2 * e + x) * CC + r;
                    const int j = r / s->CHI, jp = r % s->CHI;
                    const double m0 = (j == jp && sum > 0.0) ? L[(size_t)e * s->CHI + j] / sum : 0.0;
                    df[idx] = cf{(float)(mm[idx].x - m0), (float)mm[idx].y};
                }
        }
        if (!cuda_ok(s, cudaMemcpyAsync(s->Gamma, gf.data(), gel * sizeof(cf), cudaMemcpyHostToDevice, st)) ||
            !cuda_ok(s, cudaMemcpyAsync(s->msg[ctl.cur], df.data(), mel * sizeof(cf), cudaMemcpyHostToDevice, st)) ||
            !cuda_ok(s, cudaStreamSynchronize(st)))
            return GTQA_ERR_CUDA;
    }
    if (!cuda_ok(s, cudaMemcpyAsync(s->lam, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, st)) ||
        !cuda_ok(s, cudaStreamSynchronize(st)))
        return GTQA_ERR_CUDA;
    return GTQA_OK;
}

int gtqa_gate_layers(int32_t n, int32_t m, const int32_t* edges, int32_t k, const int32_t* edge, int32_t* layer_out,
                     int32_t* n_layers_out) {
    if (n < 1 || m < 0 || k < 0 || (m > 0 && !edges) || (k > 0 && (!edge || !layer_out))) return GTQA_ERR_INVALID_ARG;
    for (int e = 0; e < m; ++e)
        if (edges[2 * e] < 0 || edges[2 * e] >= n || edges[2 * e + 1] < 0 || edges[2 * e + 1] >= n)
            return GTQA_ERR_INVALID_ARG;
    for (int q = 0; q < k; ++q)
        if (edge[q] < 0 || edge[q] >= m) return GTQA_ERR_INVALID_ARG;
    const int nl = gate_layers(n, edges, k, edge, layer_out);
    if (n_layers_out) *n_layers_out = nl;
    return GTQA_OK;
}

int gtqa_max_degree(const gtqa_state* s, int32_t* D_out) {
    if (!s || !D_out) return GTQA_ERR_INVALID_ARG;
    *D_out = s->D;
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
    for (int e = 0; e < m; ++e) {
        const int u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return GTQA_ERR_INVALID_ARG;
    }
    std::vector<int> col;
    int nc = 0;
    if (!edge_colouring(n, m, edges, col, nc)) return GTQA_ERR_INVALID_ARG;
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

int gtqa_debug_barrier(gtqa_state* s, int64_t spin_limit, int32_t extra_arrivals) {
    if (!s || spin_limit < 1 || extra_arrivals < 0 || extra_arrivals > 1) return GTQA_ERR_INVALID_ARG;
    s->spin_limit = spin_limit;
    s->bar_extra = extra_arrivals;
    return GTQA_OK;
}

const char* gtqa_profile_name(int32_t kind) {
    static const char* names[GTQA_K_COUNT] = {"gates_kernel", "bp_kernel", "regauge_kernel", "marginals_kernel"};
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
