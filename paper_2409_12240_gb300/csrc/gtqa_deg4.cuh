// Graph tensor networks with vertex degree up to 4 (the random 4-regular graphs of Sec. V).
//
// Layout: Gamma and T are [n][2][CHI][CHI][CHI][CHI] (slot k = k-th incident edge in
// ascending id, stride CHI^(3-k); phantom slots of vertices with fewer edges have dimension 1
// with lambda = e_0); lambda [m][CHI]; messages [2m][CHI][CHI] as in the degree-3 layout.
// Complex128 throughout (the FP64 precision mode).  Same method as the degree-3 path, with
// plain kernels instead of persistent ones:
//   gates    the edge gates (diagonal Ising gates or arbitrary 4x4 gates) go through the
//            whole-side simple update of general_gates_kernel<CHI, 4> (App. E, App. D
//            "Truncation"), one launch per colour class; mixing gates through
//            single_gates_kernel<CHI, 4> (Sec. II D);
//   bp       T = Gamma prod lambda^{1/2} (Eq. (symmetric_gauge)), warm start
//            diag(lambda)/sum(lambda) (Eq. (reconstructed_messages)); one launch per flooding
//            sweep of Eq. (local_consistency), one block per vertex, with the exact trace-norm
//            distance (App. B); the host reads the distance after every sweep;
//   regauge  regauge_edge of the degree-3 path per edge (App. D "Vidal gauge finding"),
//            then the four bond transforms applied to T per vertex;
//   marginals  Eq. (partial_dens) with the environment of Eq. (bp_approx).
#pragma once

#include "gtqa_general.cuh"

namespace gtqa {

struct D4Args {
    void* Gamma;
    void* T;
    double* lam;
    const void* msg_cur;      // incoming and previous outgoing messages
    void* msg_nxt;            // new outgoing messages
    cd* X;                    // regauge transforms [m][2][CHI^2]
    const int4* vslots;       // four slots per vertex (-1 phantom)
    const int4* edge_info;    // (u, v, slot at u, slot at v)
    int n, m;
    double* acc;              // distance accumulator (one double)
    int warm;
};

template <int CHI>
struct D4Shape {
    static constexpr int H = ipow(CHI, 4), H2 = 2 * H, CC = CHI * CHI;
    static constexpr int NT = 16 * CC;     // threads of the sweep kernel: 16 per message entry
};

__device__ __forceinline__ int d4_slot_edge(const int4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// T = Gamma prod_k lambda_k^{1/2}; with warm, the outgoing messages of the vertex are set to
// diag(lambda)/sum(lambda).  One block per vertex.
template <int CHI>
__global__ void d4_bp_init_kernel(D4Args a) {
    using S = D4Shape<CHI>;
    const int v = blockIdx.x;
    __shared__ double sq[4][CHI], m0[4][CHI];
    const int4 sl = a.vslots[v];
    if (threadIdx.x < 4 * CHI) {
        const int k = threadIdx.x / CHI, j = threadIdx.x % CHI;
        const int e = d4_slot_edge(sl, k);
        const double lj = lam_get(a.lam, CHI, e, j);
        sq[k][j] = sqrt(lj);
        double s = 0.0;
        for (int q = 0; q < CHI; ++q) s += lam_get(a.lam, CHI, e, q);
        m0[k][j] = s > 0.0 ? lj / s : 0.0;
    }
    __syncthreads();
    const cd* g = (const cd*)a.Gamma + (size_t)v * S::H2;
    cd* T = (cd*)a.T + (size_t)v * S::H2;
    for (int t = threadIdx.x; t < S::H2; t += blockDim.x) {
        const int r = t % S::H;
        const int j0 = r / (CHI * CHI * CHI), j1 = (r / (CHI * CHI)) % CHI, j2 = (r / CHI) % CHI, j3 = r % CHI;
        T[t] = (sq[0][j0] * sq[1][j1] * sq[2][j2] * sq[3][j3]) * g[t];
    }
    if (a.warm) {
        cd* out = (cd*)a.msg_nxt;   // the buffer the first sweep reads
        for (int t = threadIdx.x; t < 4 * S::CC; t += blockDim.x) {
            const int k = t / S::CC, r = t % S::CC;
            const int e = d4_slot_edge(sl, k);
            if (e < 0) continue;
            const int o = 2 * e + (a.edge_info[e].x == v ? 0 : 1);
            const int j = r / CHI, jp = r % CHI;
            out[(size_t)o * S::CC + r] = cd{j == jp ? m0[k][j] : 0.0, 0.0};
        }
    }
}

// One flooding sweep for one vertex: every outgoing message
//   m_{v->b}[j][j'] = sum T[.., j@s, ..] conj(T[.., j'@s, ..]) prod_{o != s} m_o[x_o][x'_o]
// (Eq. (local_consistency)), divided by its complex trace, and the trace norms of new - old.
template <int CHI>
__global__ void __launch_bounds__(D4Shape<CHI>::NT) d4_bp_sweep_kernel(D4Args a) {
    using S = D4Shape<CHI>;
    constexpr int H2 = S::H2, CC = S::CC, NT = S::NT, TPO = NT / CC;
    extern __shared__ __align__(16) unsigned char d4_smem[];
    cd* T = reinterpret_cast<cd*>(d4_smem);
    cd* P0 = T + H2;
    cd* P1 = P0 + H2;
    cd* min = P1 + H2;      // [4][CC]
    cd* Dm = min + 4 * CC;  // [4][CC] new - old, column-major for the SVD
    __shared__ int es[4], in_idx[4], out_idx[4];
    __shared__ cd itr;
    __shared__ double tn[4];
    __shared__ int flag[4];
    const int v = blockIdx.x, tid = threadIdx.x;
    const cd* src_msg = (const cd*)a.msg_cur;
    cd* dst_msg = (cd*)a.msg_nxt;
    if (tid < 4) {
        const int e = d4_slot_edge(a.vslots[v], tid);
        es[tid] = e;
        tn[tid] = 0.0;
        if (e >= 0) {
            const bool first = a.edge_info[e].x == v;
            out_idx[tid] = 2 * e + (first ? 0 : 1);
            in_idx[tid] = 2 * e + (first ? 1 : 0);
        } else {
            out_idx[tid] = in_idx[tid] = -1;
        }
    }
    for (int t = tid; t < H2; t += NT) T[t] = ((const cd*)a.T)[(size_t)v * H2 + t];
    __syncthreads();
    for (int t = tid; t < 4 * CC; t += NT) {
        const int k = t / CC, r = t % CC;
        min[t] = in_idx[k] >= 0 ? src_msg[(size_t)in_idx[k] * CC + r] : cd{r == 0 ? 1.0 : 0.0, 0.0};
    }
    __syncthreads();
    for (int s = 0; s < 4; ++s) {
        if (es[s] < 0) continue;   // uniform: es is shared
        const cd* src = T;
        cd* dst = P0;
        for (int o = 0; o < 4; ++o) {
            if (o == s) continue;
            const int so = ipow(CHI, 3 - o);
            for (int t = tid; t < H2; t += NT) {
                const int x = (t / so) % CHI, base = t - x * so;
                cd acc = cd{0.0, 0.0};
#pragma unroll
                for (int q = 0; q < CHI; ++q) acc = cfma(src[base + q * so], min[o * CC + q * CHI + x], acc);
                dst[t] = acc;
            }
            __syncthreads();
            src = dst;
            dst = (dst == P0) ? P1 : P0;
        }
        // F[j][j'] = sum over the entries with slot-s index j of conj(T[.. j' ..]) src[.. j ..]
        const int ss = ipow(CHI, 3 - s);
        const int r = tid / TPO, part = tid % TPO;
        const int j = r / CHI, jp = r % CHI;
        constexpr int NTERM = H2 / CHI;
        cd f = cd{0.0, 0.0};
        for (int q = part; q < NTERM; q += TPO) {
            const int t = (q / ss) * (ss * CHI) + (q % ss);
            f = cfmac(T[t + jp * ss], src[t + j * ss], f);
        }
        f.x = group_sum<TPO>(f.x, group_mask<TPO>());
        f.y = group_sum<TPO>(f.y, group_mask<TPO>());
        if (part == 0) Dm[s * CC + r] = f;   // staged; normalised below
        __syncthreads();
        if (tid == 0) {
            cd tr = cd{0.0, 0.0};
            for (int q = 0; q < CHI; ++q) tr = tr + Dm[s * CC + q * CHI + q];
            const double d = tr.x * tr.x + tr.y * tr.y;
            itr = d > 0.0 ? cd{tr.x / d, -tr.y / d} : cd{0.0, 0.0};
        }
        __syncthreads();
        if (tid < CC) {
            const cd mn = Dm[s * CC + tid] * itr;
            const cd mo = src_msg[(size_t)out_idx[s] * CC + tid];
            dst_msg[(size_t)out_idx[s] * CC + tid] = mn;
            Dm[s * CC + tid] = mn - mo;
        }
        __syncthreads();
    }
    // trace norms of the four differences: CHI^2/2 lanes of warp 0 per matrix
    constexpr int GJ = CC / 2;
    if (tid < 4 * GJ) {
        const int s = tid / GJ, g = tid % GJ;
        if (es[s] >= 0) {
            WarpGroup grp{group_mask<GJ>()};
            jacobi_svd<CHI, double, WarpGroup, false>(Dm + s * CC, nullptr, g, grp, group_mask<CHI>(), 1e-15, 60, false);
            if (g < CHI) {
                double c2 = 0.0;
                for (int rr = 0; rr < CHI; ++rr) c2 += norm2(Dm[s * CC + g * CHI + rr]);
                atomicAdd(&tn[s], sqrt(c2));
            }
        }
    }
    __syncthreads();
    if (tid == 0) atomicAdd(a.acc, tn[0] + tn[1] + tn[2] + tn[3]);
}

// Vidal gauge finding, edge part: the degree-3 path's regauge_edge (it reads only the
// edge's two messages and lambda).
template <int CHI>
__global__ void d4_regauge_edge_kernel(Ctx c, int cur) {
    __shared__ RGSm<CHI> sm;
    regauge_edge<CHI, ModeFP64>(c, blockIdx.x, threadIdx.x, 0, cur, sm);
}

// Vidal gauge finding, vertex part: Gamma[.., j@k, ..] = sum_q T[.., q@k, ..] X_k[q][j] for the
// four slots (X of the edge, from this vertex's side; identity on phantom slots).
template <int CHI>
__global__ void d4_regauge_vertex_kernel(D4Args a) {
    using S = D4Shape<CHI>;
    constexpr int H2 = S::H2, CC = S::CC;
    extern __shared__ __align__(16) unsigned char d4_smem[];
    cd* b0 = reinterpret_cast<cd*>(d4_smem);
    cd* b1 = b0 + H2;
    cd* Xs = b1 + H2;   // [4][CC]
    const int v = blockIdx.x;
    const int4 sl = a.vslots[v];
    for (int t = threadIdx.x; t < H2; t += blockDim.x) b0[t] = ((const cd*)a.T)[(size_t)v * H2 + t];
    for (int t = threadIdx.x; t < 4 * CC; t += blockDim.x) {
        const int k = t / CC, r = t % CC;
        const int e = d4_slot_edge(sl, k);
        if (e >= 0) {
            const int side = a.edge_info[e].x == v ? 0 : 1;
            Xs[t] = a.X[((size_t)e * 2 + side) * CC + r];
        } else {
            Xs[t] = cd{(r / CHI == r % CHI) ? 1.0 : 0.0, 0.0};
        }
    }
    __syncthreads();
    cd* cur = b0;
    cd* nxt = b1;
    for (int k = 0; k < 4; ++k) {
        const int st = ipow(CHI, 3 - k);
        for (int t = threadIdx.x; t < H2; t += blockDim.x) {
            const int jk = (t / st) % CHI, base = t - jk * st;
            cd acc = cd{0.0, 0.0};
            for (int q = 0; q < CHI; ++q) acc = cfma(cur[base + q * st], Xs[k * CC + q * CHI + jk], acc);
            nxt[t] = acc;
        }
        __syncthreads();
        cd* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    cd* g = (cd*)a.Gamma + (size_t)v * H2;
    for (int t = threadIdx.x; t < H2; t += blockDim.x) g[t] = cur[t];
}

// rho_a = sum_J Gamma[i, J] conj(Gamma[i', J]) prod_k lambda_k[j_k]^2 / trace (Eqs. (partial_dens),
// (bp_approx)); read-out +1 if rho_a[0][0] > 1/2 (Eq. (rounding_rule)).  One warp per vertex.
template <int CHI>
__global__ void d4_marginals_kernel(const cd* Gamma, const double* lam, const int4* vslots, int n, cd* rho,
                                    int8_t* sign, int* nan_flag) {
    using S = D4Shape<CHI>;
    constexpr int H = S::H;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int v = warp;
    const int4 sl = vslots[v];
    cd acc[4] = {cd{0, 0}, cd{0, 0}, cd{0, 0}, cd{0, 0}};
    for (int r = lane; r < H; r += 32) {
        int rem = r;
        double wgt = 1.0;
        for (int k = 3; k >= 0; --k) {
            const double l = lam_get(lam, CHI, d4_slot_edge(sl, k), rem % CHI);
            wgt *= l * l;
            rem /= CHI;
        }
        const cd g0 = Gamma[(size_t)v * 2 * H + r], g1 = Gamma[(size_t)v * 2 * H + H + r];
        acc[0] = cfmac(g0, wgt * g0, acc[0]);
        acc[1] = cfmac(g1, wgt * g0, acc[1]);
        acc[2] = cfmac(g0, wgt * g1, acc[2]);
        acc[3] = cfmac(g1, wgt * g1, acc[3]);
    }
    for (int q = 0; q < 4; ++q) {
        acc[q].x = group_sum<32>(acc[q].x, 0xffffffffu);
        acc[q].y = group_sum<32>(acc[q].y, 0xffffffffu);
    }
    if (lane == 0) {
        const double tr = acc[0].x + acc[3].x;
        const double it = 1.0 / tr;
        for (int q = 0; q < 4; ++q) rho[(size_t)v * 4 + q] = it * acc[q];
        if (sign) sign[v] = (acc[0].x * it > 0.5) ? 1 : -1;
        if (!(tr == tr) || tr == 0.0) atomicOr(nan_flag, 1);
    }
}

}  // namespace gtqa
