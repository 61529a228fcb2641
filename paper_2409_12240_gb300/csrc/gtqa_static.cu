// gtqa_bp_static: belief propagation on caller-owned device buffers without any
// device allocation.  The scratch this BP run needs (the symmetric-gauge tensors,
// the second message buffer, the barrier/control block and the per-run counters)
// lives in one file-scope device array; the caller passes inputs and the output.
//
// Who needs this: callers that cannot call cudaMalloc from this code path, for
// example latency-bound loops that forbid allocation after start-up (cudaMalloc can
// synchronise the device and has no latency bound), or processes whose device memory
// is owned by another allocator (a framework's caching pool), where an allocation by
// this library would fail or fragment that pool.
#include "gtqa.h"
#include "gtqa_launch.h"

#include <cstring>

using namespace gtqa;

namespace {

constexpr int kChi = GTQA_STATIC_CHI;
constexpr int kH = kChi * kChi * kChi;
constexpr int kCC = kChi * kChi;
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
// layout of the scratch array
constexpr size_t kOffT = 0;                                                            // T [n][2][H] complex128
constexpr size_t kOffMsg = align256(kOffT + sizeof(cd) * 2 * kH * (size_t)GTQA_STATIC_MAX_N);   // messages [2m][CC]
constexpr size_t kOffCtl = align256(kOffMsg + sizeof(cd) * kCC * 2 * (size_t)GTQA_STATIC_MAX_M);
constexpr size_t kOffAcc = align256(kOffCtl + sizeof(Control));                         // acc[6], dist[1]
constexpr size_t kOffInt = align256(kOffAcc + sizeof(double) * 7);                      // done, iters, vbeg[2], m
constexpr size_t kOffVinst = align256(kOffInt + sizeof(int) * 8);                       // vert_inst [n] (zeros)
constexpr size_t kBytes = align256(kOffVinst + sizeof(int) * (size_t)GTQA_STATIC_MAX_N);

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_bp_scratch[kBytes];

// Set-up on every call, with the caller's device current: the device address of the
// scratch array (cudaGetSymbolAddress, which allocates nothing) and the BP kernel's
// shared-memory opt-in.  Neither is cached, so a call after a device reset (which reloads
// the module and drops the kernel attribute) still sees the live array and limit.
int setup(void** addr, size_t* smem) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bp_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    size_t base = 0;
    int tpb = 0, bps = 0;
    if (!PhaseUnit<ModeFP64, PK_BP>::shape(kChi, 0, &base, &tpb, nullptr)) return GTQA_ERR_UNSUPPORTED;
    const size_t sm = (base + bp_instance_smem(1) + 15) / 16 * 16;
    if (PhaseUnit<ModeFP64, PK_BP>::prepare(kChi, 0, sm, &bps) != cudaSuccess || bps < 1) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    *addr = p;
    *smem = sm;
    return GTQA_OK;
}

// Checks the caller's index arrays before BP follows them: every vertex has degree 0..3,
// its slots below the degree hold edge ids in [0, m) whose endpoint and slot entries
// name that vertex and slot, and the slots past the degree hold -1; every edge joins two
// distinct vertices in [0, n) with slots in 0..2 that list the edge.  Any violation sets
// *bad.  Only indices already checked to be in range are followed.
__global__ void check_graph(const int4* ve, const int4* ei, int n, int m, int* bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = true;
    if (t < n) {
        const int4 v = ve[t];
        const int es[3] = {v.x, v.y, v.z};
        ok = v.w >= 0 && v.w <= 3;
        for (int k = 0; k < 3 && ok; ++k) {
            if (k >= v.w) {
                ok = es[k] == -1;
            } else if (es[k] < 0 || es[k] >= m) {
                ok = false;
            } else {
                const int4 x = ei[es[k]];
                ok = (x.x == t && x.z == k) || (x.y == t && x.w == k);
            }
        }
    } else if (t < n + m) {
        const int e = t - n;
        const int4 x = ei[e];
        ok = x.x >= 0 && x.x < n && x.y >= 0 && x.y < n && x.x != x.y && x.z >= 0 && x.z < 3 && x.w >= 0 && x.w < 3;
        if (ok) {
            const int4 a = ve[x.x], b = ve[x.y];
            const int sa[3] = {a.x, a.y, a.z}, sb[3] = {b.x, b.y, b.z};
            ok = sa[x.z] == e && sb[x.w] == e;
        }
    }
    if (!ok) atomicOr(bad, 1);
}

bool device_accessible(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int gtqa_bp_static(int32_t n, int32_t m, const int32_t* vert_edges, const int32_t* edge_info,
                              const double* gamma, const double* lambda, double* messages_out, double tol,
                              int32_t max_iter, int32_t* iters_out, double* dist_out, void* cuda_stream) {
    if (n < 1 || m < 1 || n > GTQA_STATIC_MAX_N || m > GTQA_STATIC_MAX_M) return GTQA_ERR_INVALID_ARG;
    if (!vert_edges || !edge_info || !gamma || !lambda || !messages_out || max_iter < 1 || !(tol >= 0.0))
        return GTQA_ERR_INVALID_ARG;
    if (!device_accessible(vert_edges) || !device_accessible(edge_info) || !device_accessible(gamma) ||
        !device_accessible(lambda) || !device_accessible(messages_out))
        return GTQA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    void* base = nullptr;
    size_t smem = 0;
    int rc = setup(&base, &smem);
    if (rc) return rc;
    unsigned char* sc = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // Per-call initialisation of the parts that must start at zero or hold sizes; the
    // array keeps the previous call's contents otherwise.
    const int ints[8] = {0, 0, 0, n, m, 0, 0, 0};   // done, iters, vbeg[0], vbeg[1], m, index check flag
    if (cudaMemsetAsync(sc + kOffCtl, 0, sizeof(Control), st) != cudaSuccess ||
        cudaMemsetAsync(sc + kOffAcc, 0, sizeof(double) * 7, st) != cudaSuccess ||
        cudaMemcpyAsync(sc + kOffInt, ints, sizeof(ints), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(sc + kOffVinst, 0, sizeof(int) * (size_t)n, st) != cudaSuccess) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    // the index arrays are checked on the device before the BP kernel reads through them
    int* bad = reinterpret_cast<int*>(sc + kOffInt) + 5;
    int hbad = 0;
    check_graph<<<(n + m + 255) / 256, 256, 0, st>>>(reinterpret_cast<const int4*>(vert_edges),
                                                     reinterpret_cast<const int4*>(edge_info), n, m, bad);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    if (hbad) return GTQA_ERR_INVALID_ARG;
    Ctx c;
    std::memset(&c, 0, sizeof(c));
    c.edge_info = reinterpret_cast<const int4*>(edge_info);
    c.vert_edges = reinterpret_cast<const int4*>(vert_edges);
    c.vert_inst = reinterpret_cast<const int*>(sc + kOffVinst);
    c.n = n;
    c.m = m;
    c.B = 1;
    c.inst_done = reinterpret_cast<int*>(sc + kOffInt);
    c.inst_iters = reinterpret_cast<int*>(sc + kOffInt) + 1;
    c.inst_vbeg = reinterpret_cast<const int*>(sc + kOffInt) + 2;
    c.inst_m = reinterpret_cast<const int*>(sc + kOffInt) + 4;
    c.acc = reinterpret_cast<double*>(sc + kOffAcc);
    c.inst_dist = reinterpret_cast<double*>(sc + kOffAcc) + 6;
    c.Gamma = const_cast<double*>(gamma);
    c.lam = const_cast<double*>(lambda);
    c.T = sc + kOffT;
    c.msg[0] = messages_out;
    c.msg[1] = sc + kOffMsg;
    c.ctl = reinterpret_cast<Control*>(sc + kOffCtl);
    c.phases = PH_BP | PH_WARM;
    c.tol = tol;
    c.max_iter = max_iter;
    c.nblocks = sms;
    c.bar_expect = sms;
    c.spin_limit = 1LL << 22;
    if (PhaseUnit<ModeFP64, PK_BP>::launch(kChi, 0, c, smem, st) != cudaSuccess) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    Control ctl;
    if (cudaMemcpyAsync(&ctl, sc + kOffCtl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return GTQA_ERR_CUDA;
    }
    if (ctl.err) return ctl.err;
    if (ctl.cur == 1) {   // the last sweep wrote the scratch buffer
        if (cudaMemcpyAsync(messages_out, sc + kOffMsg, sizeof(cd) * kCC * 2 * (size_t)m, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return GTQA_ERR_CUDA;
        }
    }
    if (iters_out) *iters_out = ctl.last_iters;
    if (dist_out) *dist_out = ctl.last_dist;
    if (!(ctl.last_dist == ctl.last_dist)) return GTQA_ERR_NUMERIC;
    return ctl.not_conv > 0 ? GTQA_ERR_NOT_CONVERGED : GTQA_OK;
}
