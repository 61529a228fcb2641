// The plain path: graph tensor networks whose vertex tensors are too large or have too many
// bonds for the persistent kernels, or that run every step in FP32.  Shapes built: degree 4
// with CHI <= 4 (the random 4-regular graphs of Sec. V) and degree 3 with CHI = 16 (the largest
// bond dimension of the chi sweep), in complex128 (the FP64 precision mode, R = RC = double) and
// in the mixed mode (complex64 storage and contractions, R = float, with the normalisation,
// trace norms, regauge and the CHI = 16 gate's QR/SVD in RC = double); degree 3 with CHI <= 8 or
// CHI = 16 and degree 4 with CHI <= 4 in complex64 with every step in FP32 (the complex64 mode,
// R = RC = float).  One instance.  The messages hold m itself in FP64 and complex64 and, as on
// the persistent path, delta = m - m0 with m0 = diag(lambda)/sum(lambda) in the mixed mode
// (BP contracts only the delta terms in FP32; the warm-start defect D0 is computed in FP64 and
// stored in complex64, its trace t0 in complex128).
//
// Layout: Gamma and T are [n][2][CHI]^D (slot k = k-th incident edge in ascending id, stride
// CHI^(D-1-k); phantom slots of vertices with fewer edges have dimension 1 with lambda = e_0);
// lambda [m][CHI]; messages [2m][CHI][CHI] as in the persistent path.
// The steps are those of the persistent path, in plain launches:
//   gates    degree 4: general_gates_kernel<CHI, 4> with the diagonal Ising gate (App. E);
//            CHI = 16: ising16_gate_kernel, the per-physical-index QR-reduced simple update
//            with a 2 CHI x 2 CHI core (App. E, App. D "Truncation"); one launch per colour
//            class; mixing gates through single_gates_kernel (Sec. II D);
//   bp       T = Gamma prod lambda^{1/2} (Eq. (symmetric_gauge)), warm start
//            diag(lambda)/sum(lambda) (Eq. (reconstructed_messages)); per flooding sweep of
//            Eq. (local_consistency) one launch over vertices and one over messages for the
//            exact trace-norm distance (App. B); the host reads the distance after every sweep;
//   regauge  per edge the Vidal gauge transforms from the two messages (App. D "Vidal gauge
//            finding"), then per vertex the transforms applied to T;
//   marginals  Eq. (partial_dens) with the environment of Eq. (bp_approx);
//   residual   R of App. C per (vertex, slot), FP64 trace norms (the regauge policy of
//              Sec. II C reads it on the host);
//   sampling   the projection step of Sec. IV A for one vertex, then BP and the regauge.
#pragma once

#include "gtqa_general.cuh"

namespace gtqa {

struct PlainArgs {
    void* Gamma;
    void* T;
    double* lam;
    const void* msg_cur;      // incoming and previous outgoing messages
    void* msg_nxt;            // new outgoing messages
    void* X;                  // regauge transforms [m][2][CHI^2]
    void* dm;                 // [2m][CHI^2]: new - old of every outgoing message of a sweep
    void* scratch;            // per-block tensor buffers when shared memory is too small
    const int4* vslots;       // slots per vertex (x, y, z, w; -1 phantom)
    const int4* edge_info;    // (u, v, slot at u, slot at v)
    int n, m;
    double* acc;              // distance accumulator (one double)
    int warm;
    void* D0;                 // mixed mode: [2m][CHI^2] warm-start defect F(m0) - tr F(m0) m0 (storage type)
    cd* t0;                   // mixed mode: [2m] tr F(m0)
};

template <int CHI, int D, typename R = double>
struct PlainShape {
    static constexpr int H = ipow(CHI, D), H2 = 2 * H, CC = CHI * CHI;
    static constexpr int NT = 16 * CC < 1024 ? 16 * CC : 1024;    // threads of the sweep kernel
    static constexpr int TPO = NT / CC;                           // threads per message entry
    static constexpr bool SMEM = 3 * H2 * (int)sizeof(C<R>) <= 48 * 1024;   // tensor buffers in shared memory
    static constexpr size_t scratch_per_block = SMEM ? 0 : (size_t)3 * H2;   // complex entries
};

__device__ __forceinline__ int plain_slot_edge(const int4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// T = Gamma prod_k lambda_k^{1/2}; with warm, the vertex's outgoing messages are set to
// diag(lambda)/sum(lambda) in msg_nxt (the buffer the first sweep reads).  One block per vertex.
template <int CHI, int D, typename R, typename RC = R>
__global__ void plain_bp_init_kernel(PlainArgs a) {
    using S = PlainShape<CHI, D, R>;
    const int v = blockIdx.x;
    __shared__ RC sq[D][CHI], m0[D][CHI];
    const int4 sl = a.vslots[v];
    if (threadIdx.x < D * CHI) {
        const int k = threadIdx.x / CHI, j = threadIdx.x % CHI;
        const int e = plain_slot_edge(sl, k);
        const RC lj = lam_get(a.lam, CHI, e, j);
        sq[k][j] = sqrt(lj);
        RC s = 0.0;
        for (int q = 0; q < CHI; ++q) s += lam_get(a.lam, CHI, e, q);
        m0[k][j] = s > 0.0 ? lj / s : 0.0;
    }
    __syncthreads();
    const C<R>* g = (const C<R>*)a.Gamma + (size_t)v * S::H2;
    C<R>* T = (C<R>*)a.T + (size_t)v * S::H2;
    for (int t = threadIdx.x; t < S::H2; t += blockDim.x) {
        int r = t % S::H;
        RC f = 1.0;
        for (int k = D - 1; k >= 0; --k) {
            f *= sq[k][r % CHI];
            r /= CHI;
        }
        T[t] = ccast<R>(f * ccast<RC>(g[t]));
    }
    constexpr bool MIX = sizeof(R) != sizeof(RC);
    if (a.warm) {
        // the mixed mode holds delta = m - m0, which the warm start sets to 0
        C<R>* out = (C<R>*)a.msg_nxt;
        for (int t = threadIdx.x; t < D * S::CC; t += blockDim.x) {
            const int k = t / S::CC, r = t % S::CC;
            const int e = plain_slot_edge(sl, k);
            if (e < 0) continue;
            const int o = 2 * e + (a.edge_info[e].x == v ? 0 : 1);
            const int j = r / CHI, jp = r % CHI;
            out[(size_t)o * S::CC + r] = C<R>{(!MIX && j == jp) ? (R)m0[k][j] : (R)0, (R)0};
        }
    }
    if constexpr (MIX) {
        // F0 = F(m0) of every outgoing message in RC from the stored T (so that F(m0 + delta) =
        // F0 + F_delta holds for the T the sweeps contract), kept as D0 = F0 - tr(F0) m0 and t0
        __shared__ C<RC> F0[D][S::CC];
        __shared__ C<RC> tr0[D];
        __syncthreads();   // this block's T is written
        constexpr int NO = S::H / CHI;
        for (int t = threadIdx.x; t < D * S::CC; t += blockDim.x) {
            const int k = t / S::CC, r = t % S::CC;
            if (plain_slot_edge(sl, k) < 0) continue;
            const int j = r / CHI, jp = r % CHI;
            int sk = 1;
            for (int l = D - 1; l > k; --l) sk *= CHI;
            C<RC> f = C<RC>{(RC)0, (RC)0};
            for (int i = 0; i < 2; ++i)
                for (int q = 0; q < NO; ++q) {
                    int rem = q, base = 0, stride = 1;
                    RC w = 1.0;
                    for (int l = D - 1; l >= 0; --l) {
                        if (l != k) {
                            const int idx = rem % CHI;
                            rem /= CHI;
                            w *= m0[l][idx];
                            base += idx * stride;
                        }
                        stride *= CHI;
                    }
                    const C<RC> x = ccast<RC>(T[i * S::H + base + j * sk]), y = ccast<RC>(T[i * S::H + base + jp * sk]);
                    f = cfmac(y, w * x, f);
                }
            F0[k][r] = f;
        }
        __syncthreads();
        if (threadIdx.x < D) {
            C<RC> tr = C<RC>{(RC)0, (RC)0};
            for (int j = 0; j < CHI; ++j) tr = tr + F0[threadIdx.x][j * CHI + j];
            tr0[threadIdx.x] = tr;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < D * S::CC; t += blockDim.x) {
            const int k = t / S::CC, r = t % S::CC;
            const int e = plain_slot_edge(sl, k);
            if (e < 0) continue;
            const int o = 2 * e + (a.edge_info[e].x == v ? 0 : 1);
            const int j = r / CHI, jp = r % CHI;
            C<RC> d = F0[k][r];
            if (j == jp) d = d - m0[k][j] * tr0[k];
            ((C<R>*)a.D0)[(size_t)o * S::CC + r] = ccast<R>(d);
            if (r == 0) a.t0[o] = ccast<double>(tr0[k]);
        }
    }
}

// One flooding sweep for one vertex: every outgoing message
//   m_{v->b}[j][j'] = sum T[.., j@s, ..] conj(T[.., j'@s, ..]) prod_{o != s} m_o[x_o][x'_o]
// (Eq. (local_consistency)), divided by its complex trace; new - old goes to dm for the
// trace-norm kernel.
// R is the storage and contraction type; RC the type of the trace and the normalisation
// (FP64 in the mixed mode).
template <int CHI, int D, typename R, typename RC = R>
__global__ void __launch_bounds__(PlainShape<CHI, D, R>::NT) plain_bp_sweep_kernel(PlainArgs a) {
    using S = PlainShape<CHI, D, R>;
    constexpr int H2 = S::H2, CC = S::CC, NT = S::NT, TPO = S::TPO;
    extern __shared__ __align__(16) unsigned char plain_smem[];
    C<R>* min = reinterpret_cast<C<R>*>(plain_smem);   // [D][CC]
    C<R>* F = min + D * CC;                          // [CC]
    C<R>* T;
    C<R>* P0;
    C<R>* P1;
    if constexpr (S::SMEM) {
        T = F + CC;
        P0 = T + H2;
        P1 = P0 + H2;
    } else {
        T = (C<R>*)a.scratch + (size_t)blockIdx.x * S::scratch_per_block;
        P0 = T + H2;
        P1 = P0 + H2;
    }
    __shared__ int es[4], in_idx[4], out_idx[4];
    __shared__ C<RC> itr;
    // mixed mode (the delta form of the persistent path): the messages hold delta = m - m0 with
    // m0 = diag(lambda)/sum(lambda); mz and md hold m0 and delta of the incoming messages
    constexpr bool MIX = sizeof(R) != sizeof(RC);
    C<R>* mz = min + (D + 1) * CC + (S::SMEM ? 3 * H2 : 0);   // [D][CC], mixed mode only
    C<R>* md = mz + D * CC;                                  // [D][CC], mixed mode only
    __shared__ RC m0d[D][CHI];
    __shared__ C<RC> tau;
    const int v = blockIdx.x, tid = threadIdx.x;
    const C<R>* src_msg = (const C<R>*)a.msg_cur;
    C<R>* dst_msg = (C<R>*)a.msg_nxt;
    if (tid < D) {
        const int e = plain_slot_edge(a.vslots[v], tid);
        es[tid] = e;
        if (e >= 0) {
            const bool first = a.edge_info[e].x == v;
            out_idx[tid] = 2 * e + (first ? 0 : 1);
            in_idx[tid] = 2 * e + (first ? 1 : 0);
        } else {
            out_idx[tid] = in_idx[tid] = -1;
        }
    }
    if (MIX && tid < D * CHI) {
        const int k = tid / CHI, j = tid % CHI;
        const int e = plain_slot_edge(a.vslots[v], k);
        RC sum = 0.0;
        for (int q = 0; q < CHI; ++q) sum += lam_get(a.lam, CHI, e, q);
        m0d[k][j] = sum > 0.0 ? lam_get(a.lam, CHI, e, j) / sum : 0.0;
    }
    for (int t = tid; t < H2; t += NT) T[t] = ((const C<R>*)a.T)[(size_t)v * H2 + t];
    __syncthreads();
    for (int t = tid; t < D * CC; t += NT) {
        const int k = t / CC, r = t % CC;
        if constexpr (MIX) {
            const int j = r / CHI, jp = r % CHI;
            const C<R> dv = in_idx[k] >= 0 ? src_msg[(size_t)in_idx[k] * CC + r] : C<R>{(R)0, (R)0};
            const C<R> zv = C<R>{j == jp ? (R)m0d[k][j] : (R)0, (R)0};
            md[t] = dv;
            mz[t] = zv;
            min[t] = zv + dv;
        } else {
            min[t] = in_idx[k] >= 0 ? src_msg[(size_t)in_idx[k] * CC + r] : C<R>{(R)(r == 0 ? 1 : 0), (R)0};
        }
    }
    __syncthreads();
    if constexpr (MIX) {
        // F(m0 + delta) - F(m0) telescoped over the other slots o_1 < o_2 < ...: chain c takes
        // m0 on the slots before its own, delta on its own and m after it (FP32 contractions);
        // then delta' = (D0 + F_delta - m0 tr F_delta) / (t0 + tr F_delta) in RC
        for (int s = 0; s < D; ++s) {
            if (es[s] < 0) continue;   // uniform: es is shared
            const int ss = ipow(CHI, D - 1 - s);
            constexpr int NTERM = H2 / CHI;
            for (int c = 0; c < D - 1; ++c) {
                const C<R>* src = T;
                C<R>* dst = P0;
                int i = 0;
                for (int o = 0; o < D; ++o) {
                    if (o == s) continue;
                    const C<R>* mo = (i < c ? mz : (i == c ? md : min)) + o * CC;
                    ++i;
                    const int so = ipow(CHI, D - 1 - o);
                    for (int t = tid; t < H2; t += NT) {
                        const int x = (t / so) % CHI, base = t - x * so;
                        C<R> acc = C<R>{(R)0, (R)0};
#pragma unroll 4
                        for (int q = 0; q < CHI; ++q) acc = cfma(src[base + q * so], mo[q * CHI + x], acc);
                        dst[t] = acc;
                    }
                    __syncthreads();
                    src = dst;
                    dst = (dst == P0) ? P1 : P0;
                }
                for (int rr = tid / TPO; rr < CC; rr += NT / TPO) {
                    const int part = tid % TPO;
                    const int j = rr / CHI, jp = rr % CHI;
                    C<R> f = C<R>{(R)0, (R)0};
                    for (int q = part; q < NTERM; q += TPO) {
                        const int t = (q / ss) * (ss * CHI) + (q % ss);
                        f = cfmac(T[t + jp * ss], src[t + j * ss], f);
                    }
                    f.x = group_sum<TPO>(f.x, group_mask<TPO>());
                    f.y = group_sum<TPO>(f.y, group_mask<TPO>());
                    if (part == 0) F[rr] = c == 0 ? f : F[rr] + f;
                }
                __syncthreads();
            }
            const int out = out_idx[s];
            if (tid == 0) {
                C<RC> tr = C<RC>{(RC)0, (RC)0};
                for (int q = 0; q < CHI; ++q) tr = tr + ccast<RC>(F[q * CHI + q]);
                tau = tr;
                const C<RC> den = a.t0[out] + tr;
                const RC d = den.x * den.x + den.y * den.y;
                itr = d > 0.0 ? C<RC>{den.x / d, -den.y / d} : C<RC>{(RC)0, (RC)0};
            }
            __syncthreads();
            for (int r = tid; r < CC; r += NT) {
                const int j = r / CHI, jp = r % CHI;
                C<RC> num = ccast<RC>(((const C<R>*)a.D0)[(size_t)out * CC + r]) + ccast<RC>(F[r]);
                if (j == jp) num = num - m0d[s][j] * tau;
                const C<RC> dn = num * itr;
                const C<RC> dold = ccast<RC>(src_msg[(size_t)out * CC + r]);
                dst_msg[(size_t)out * CC + r] = ccast<R>(dn);
                ((C<R>*)a.dm)[(size_t)out * CC + r] = ccast<R>(dn - dold);
            }
            __syncthreads();
        }
        return;
    }
    for (int s = 0; s < D; ++s) {
        if (es[s] < 0) continue;   // uniform: es is shared
        const C<R>* src = T;
        C<R>* dst = P0;
        for (int o = 0; o < D; ++o) {
            if (o == s) continue;
            const int so = ipow(CHI, D - 1 - o);
            for (int t = tid; t < H2; t += NT) {
                const int x = (t / so) % CHI, base = t - x * so;
                C<R> acc = C<R>{(R)0, (R)0};
#pragma unroll 4
                for (int q = 0; q < CHI; ++q) acc = cfma(src[base + q * so], min[o * CC + q * CHI + x], acc);
                dst[t] = acc;
            }
            __syncthreads();
            src = dst;
            dst = (dst == P0) ? P1 : P0;
        }
        // F[j][j'] = sum over the entries with slot-s index j of conj(T[.. j' ..]) src[.. j ..]
        const int ss = ipow(CHI, D - 1 - s);
        constexpr int NTERM = H2 / CHI;
        for (int rr = tid / TPO; rr < CC; rr += NT / TPO) {
            const int part = tid % TPO;
            const int j = rr / CHI, jp = rr % CHI;
            C<R> f = C<R>{(R)0, (R)0};
            for (int q = part; q < NTERM; q += TPO) {
                const int t = (q / ss) * (ss * CHI) + (q % ss);
                f = cfmac(T[t + jp * ss], src[t + j * ss], f);
            }
            f.x = group_sum<TPO>(f.x, group_mask<TPO>());
            f.y = group_sum<TPO>(f.y, group_mask<TPO>());
            if (part == 0) F[rr] = f;
        }
        __syncthreads();
        if (tid == 0) {
            C<RC> tr = C<RC>{(RC)0, (RC)0};
            for (int q = 0; q < CHI; ++q) tr = tr + ccast<RC>(F[q * CHI + q]);
            const RC d = tr.x * tr.x + tr.y * tr.y;
            itr = d > 0.0 ? C<RC>{tr.x / d, -tr.y / d} : C<RC>{(RC)0, (RC)0};
        }
        __syncthreads();
        for (int r = tid; r < CC; r += NT) {
            const C<RC> mn = ccast<RC>(F[r]) * itr;
            const C<RC> mo = ccast<RC>(src_msg[(size_t)out_idx[s] * CC + r]);
            dst_msg[(size_t)out_idx[s] * CC + r] = ccast<R>(mn);
            ((C<R>*)a.dm)[(size_t)out_idx[s] * CC + r] = ccast<R>(mn - mo);
        }
        __syncthreads();
    }
}

// Trace norm (sum of singular values, one-sided Jacobi in FP64) of every directed message's
// new - old; block = CHI^2 / 2 threads, one message per block; the sum goes to *acc.
template <int CHI, typename R, typename RC = R>
__global__ void plain_trace_norm_kernel(const C<R>* dm, double* acc) {
    constexpr int CC = CHI * CHI;
    __shared__ C<RC> A[CC];
    __shared__ RC tn;
    __shared__ int flag;
    const int g = threadIdx.x;
    for (int t = g; t < CC; t += blockDim.x) A[t] = ccast<RC>(dm[(size_t)blockIdx.x * CC + t]);
    if (g == 0) tn = 0.0;
    __syncthreads();
    BlockGroup grp{&flag};
    jacobi_svd<CHI, RC, BlockGroup, false>(A, nullptr, g, grp, group_mask<CHI>(), (RC)(sizeof(RC) == 8 ? 1e-15 : 1e-6),
                                           60, false);
    __syncthreads();
    if (g < CHI) {
        RC c2 = 0.0;
        for (int r = 0; r < CHI; ++r) c2 += norm2(A[g * CHI + r]);
        atomicAdd(&tn, sqrt(c2));
    }
    __syncthreads();
    if (g == 0) atomicAdd(acc, tn);
}

// Vidal gauge finding, edge part (App. D "Vidal gauge finding"), FP64, block = CHI^2 / 2
// threads: Hermitian eigen-decompositions of m_{a->b} and m_{b->a} (as SVDs; signs from
// v^H A v), principal square roots and pseudo-inverse square roots, the SVD of
// M = (m_{a->b}^{1/2})^T m_{b->a}^{1/2}, lambda = S/||S||, X_a = conj(m_{a->b}^{-1/2}) U ||S||^{1/2}
// and X_b = conj(m_{b->a}^{-1/2}) V^* ||S||^{1/2}.
template <int CHI, typename R, typename RC = R>
__global__ void plain_regauge_edge_kernel(const C<R>* msg, double* lam, C<R>* X, double eig_cut, double svd_cut) {
    constexpr int CC = CHI * CHI;
    __shared__ C<RC> Am[2][CC], Vm[2][CC], sqm[2][CC], isq[2][CC], M[CC], VM[CC];
    __shared__ RC w[2][CHI], sig[CHI], scal[2];
    __shared__ int perm[CHI], flag;
    const int e = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    BlockGroup grp{&flag};
    // mixed mode: the messages hold delta = m - m0, m0 = diag(lambda_e)/sum(lambda_e) (read before
    // this kernel overwrites lambda_e)
    constexpr bool MIX = sizeof(R) != sizeof(RC);
    __shared__ RC m0e[CHI];
    if (MIX && tid < CHI) {
        RC sum = 0.0;
        for (int q = 0; q < CHI; ++q) sum += lam[(size_t)e * CHI + q];
        m0e[tid] = sum > 0.0 ? lam[(size_t)e * CHI + tid] / sum : 0.0;
    }
    if (MIX) __syncthreads();
    for (int t = tid; t < 2 * CC; t += NT) {
        const int x = t / CC, r = t % CC;
        const int row = r % CHI, col = r / CHI;
        const C<R>* mm = msg + (size_t)(2 * e + x) * CC;
        C<RC> v = ccast<RC>(mm[row * CHI + col]), vt = ccast<RC>(mm[col * CHI + row]);
        if (MIX && row == col) {
            v.x += m0e[row];
            vt.x += m0e[row];
        }
        Am[x][col * CHI + row] = C<RC>{(RC)0.5 * (v.x + vt.x), (RC)0.5 * (v.y - vt.y)};
    }
    __syncthreads();
    for (int x = 0; x < 2; ++x)
        jacobi_svd<CHI, RC, BlockGroup, true, sizeof(RC) == 8>(Am[x], Vm[x], tid, grp, group_mask<CHI>(),
                                                                  (RC)(sizeof(RC) == 8 ? 1e-15 : 1e-6), 60, true, nullptr,
                                                                  (RC)(sizeof(RC) == 8 ? 3e-8 : 1e-3));
    __syncthreads();
    for (int t = tid; t < 2 * CHI; t += NT) {
        const int x = t / CHI, k = t % CHI;
        RC n2 = 0.0, sg = 0.0;
        for (int r = 0; r < CHI; ++r) {
            const C<RC> av = Am[x][k * CHI + r], vv = Vm[x][k * CHI + r];
            n2 += norm2(av);
            sg += vv.x * av.x + vv.y * av.y;
        }
        const RC wv = nr_sqrt(n2);
        w[x][k] = sg >= 0.0 ? wv : -wv;
    }
    __syncthreads();
    for (int t = tid; t < 2 * CC; t += NT) {
        const int x = t / CC, r = t % CC;
        const int j = r / CHI, jp = r % CHI;
        RC wmax = 0.0;
        for (int k = 0; k < CHI; ++k) wmax = fmax(wmax, w[x][k]);
        C<RC> s1 = C<RC>{(RC)0, (RC)0}, s2 = C<RC>{(RC)0, (RC)0};
        for (int k = 0; k < CHI; ++k) {
            const RC wk = w[x][k];
            if (!(wk > eig_cut * wmax)) continue;
            const RC is = nr_rsqrt(wk);
            const RC sq = wk * is;
            const C<RC> vv = Vm[x][k * CHI + j] * conj(Vm[x][k * CHI + jp]);
            s1 = cfma(C<RC>{sq, (RC)0}, vv, s1);
            s2 = cfma(C<RC>{is, (RC)0}, vv, s2);
        }
        sqm[x][r] = s1;
        isq[x][r] = s2;
    }
    __syncthreads();
    for (int t = tid; t < CC; t += NT) {
        const int k = t % CHI, l = t / CHI;
        C<RC> acc = C<RC>{(RC)0, (RC)0};
        for (int j = 0; j < CHI; ++j) acc = cfma(sqm[0][j * CHI + k], sqm[1][j * CHI + l], acc);
        M[l * CHI + k] = acc;
    }
    __syncthreads();
    jacobi_svd<CHI, RC, BlockGroup, true, sizeof(RC) == 8>(M, VM, tid, grp, group_mask<CHI>(),
                                                         (RC)(sizeof(RC) == 8 ? 1e-15 : 1e-6), 60, true, nullptr,
                                                         (RC)(sizeof(RC) == 8 ? 3e-8 : 1e-3));
    __syncthreads();
    for (int cc = tid; cc < CHI; cc += NT) {
        RC n2 = 0.0;
        for (int r = 0; r < CHI; ++r) n2 += norm2(M[cc * CHI + r]);
        sig[cc] = nr_sqrt(n2);
    }
    __syncthreads();
    for (int cc = tid; cc < CHI; cc += NT) perm[desc_rank(sig, CHI, cc)] = cc;
    __syncthreads();
    if (tid == 0) {
        RC tot = 0.0;
        for (int cc = 0; cc < CHI; ++cc) tot += sig[cc] * sig[cc];
        const RC nrm = nr_sqrt(tot);
        scal[0] = nrm;
        scal[1] = nr_sqrt(nrm);
        const RC inrm = nrm > 0.0 ? nr_rcp(nrm) : 0.0;
        const RC smax = sig[perm[0]];
        for (int r = 0; r < CHI; ++r) {
            const RC s = sig[perm[r]];
            lam[(size_t)e * CHI + r] = (nrm > 0.0 && s > svd_cut * smax) ? s * inrm : 0.0;
        }
    }
    __syncthreads();
    for (int t = tid; t < 2 * CC; t += NT) {
        const int x = t / CC, r = t % CC;
        const int jpp = r / CHI, j = r % CHI;
        const int pc = perm[j];
        const RC s = sig[pc];
        C<RC> acc = C<RC>{(RC)0, (RC)0};
        const bool kept = scal[0] > 0.0 && s > svd_cut * sig[perm[0]];
        if (kept) {
            for (int jp = 0; jp < CHI; ++jp) {
                const C<RC> u = (x == 0) ? nr_rcp(s) * M[pc * CHI + jp] : conj(VM[pc * CHI + jp]);
                acc = cfma(isq[x][jp * CHI + jpp], u, acc);
            }
            acc = scal[1] * acc;
        }
        X[((size_t)e * 2 + x) * CC + r] = ccast<R>(acc);
    }
}

// Vidal gauge finding, vertex part: Gamma[.., j@k, ..] = sum_q T[.., q@k, ..] X_k[q][j] for every
// slot (X of the edge, from this vertex's side; identity on phantom slots).
template <int CHI, int D, typename R>
__global__ void plain_regauge_vertex_kernel(PlainArgs a) {
    using S = PlainShape<CHI, D, R>;
    constexpr int H2 = S::H2, CC = S::CC;
    extern __shared__ __align__(16) unsigned char plain_smem[];
    C<R>* Xs = reinterpret_cast<C<R>*>(plain_smem);   // [D][CC]
    C<R>* b0;
    C<R>* b1;
    if constexpr (S::SMEM) {
        b0 = Xs + D * CC;
        b1 = b0 + H2;
    } else {
        b0 = (C<R>*)a.scratch + (size_t)blockIdx.x * S::scratch_per_block;
        b1 = b0 + H2;
    }
    const int v = blockIdx.x;
    const int4 sl = a.vslots[v];
    for (int t = threadIdx.x; t < H2; t += blockDim.x) b0[t] = ((const C<R>*)a.T)[(size_t)v * H2 + t];
    for (int t = threadIdx.x; t < D * CC; t += blockDim.x) {
        const int k = t / CC, r = t % CC;
        const int e = plain_slot_edge(sl, k);
        if (e >= 0) {
            const int side = a.edge_info[e].x == v ? 0 : 1;
            Xs[t] = ((const C<R>*)a.X)[((size_t)e * 2 + side) * CC + r];
        } else {
            Xs[t] = C<R>{(R)((r / CHI == r % CHI) ? 1 : 0), (R)0};
        }
    }
    __syncthreads();
    C<R>* cur = b0;
    C<R>* nxt = b1;
    for (int k = 0; k < D; ++k) {
        const int st = ipow(CHI, D - 1 - k);
        for (int t = threadIdx.x; t < H2; t += blockDim.x) {
            const int jk = (t / st) % CHI, base = t - jk * st;
            C<R> acc = C<R>{(R)0, (R)0};
            for (int q = 0; q < CHI; ++q) acc = cfma(cur[base + q * st], Xs[k * CC + q * CHI + jk], acc);
            nxt[t] = acc;
        }
        __syncthreads();
        C<R>* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    C<R>* g = (C<R>*)a.Gamma + (size_t)v * H2;
    for (int t = threadIdx.x; t < H2; t += blockDim.x) g[t] = cur[t];
}

// rho_a = sum_J Gamma[i, J] conj(Gamma[i', J]) prod_k lambda_k[j_k]^2 / trace (Eqs. (partial_dens),
// (bp_approx)); read-out +1 if rho_a[0][0] > 1/2 (Eq. (rounding_rule)).  One warp per vertex.
template <int CHI, int D, typename R>
__global__ void plain_marginals_kernel(const C<R>* Gamma, const double* lam, const int4* vslots, int n, cd* rho,
                                       int8_t* sign, int* nan_flag) {
    constexpr int H = PlainShape<CHI, D, R>::H;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int v = warp;
    const int4 sl = vslots[v];
    cd acc[4] = {cd{0, 0}, cd{0, 0}, cd{0, 0}, cd{0, 0}};
    for (int r = lane; r < H; r += 32) {
        int rem = r;
        double wgt = 1.0;
        for (int k = D - 1; k >= 0; --k) {
            const double l = lam_get(lam, CHI, plain_slot_edge(sl, k), rem % CHI);
            wgt *= l * l;
            rem /= CHI;
        }
        const cd g0 = ccast<double>(Gamma[(size_t)v * 2 * H + r]), g1 = ccast<double>(Gamma[(size_t)v * 2 * H + H + r]);
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

// Residual R of the local-orthogonality condition (App. C) on the plain layout: one block of
// max(CHI^2/2, 1) threads per (vertex, slot) item whose slot holds a bond,
//   D_k[j, j'] = delta_{j j'} [lambda_k[j] > 0] - sum_{i, J \ j_k} Gamma[i, J(j)] conj(Gamma[i, J(j')])
//                prod_{l != k} lambda_l[j_l]^2
// in FP64 (complex64 Gamma is widened), then its trace norm (FP64 one-sided Jacobi), added to
// *out.  The caller divides the sum by 2|E|.
template <int CHI, int D, typename R>
__global__ void plain_residual_kernel(const C<R>* Gamma, const double* lam, const int4* vslots, double* out) {
    constexpr int H = PlainShape<CHI, D, R>::H, CC = CHI * CHI, NO = H / CHI;
    __shared__ cd A[CC];
    __shared__ double tn;
    __shared__ int flag;
    const int v = blockIdx.x / D, k = blockIdx.x % D;
    const int4 sl = vslots[v];
    const int ek = plain_slot_edge(sl, k);
    if (ek < 0) return;   // a phantom slot: the whole block leaves
    const int g = threadIdx.x;
    const C<R>* gv = Gamma + (size_t)v * 2 * H;
    int sk = 1;   // stride of slot k, CHI^(D-1-k)
    for (int l = D - 1; l > k; --l) sk *= CHI;
    for (int r = g; r < CC; r += blockDim.x) {
        const int j = r / CHI, jp = r % CHI;
        cd acc = cd{0.0, 0.0};
        for (int q = 0; q < NO; ++q) {
            // q runs over the indices of the other slots (last slot fastest)
            int rem = q, base = 0, stride = 1;
            double w = 1.0;
            for (int l = D - 1; l >= 0; --l) {
                if (l != k) {
                    const int idx = rem % CHI;
                    rem /= CHI;
                    const double lv = lam_get(lam, CHI, plain_slot_edge(sl, l), idx);
                    w *= lv * lv;
                    base += idx * stride;
                }
                stride *= CHI;
            }
            for (int i = 0; i < 2; ++i) {
                const cd x = ccast<double>(gv[i * H + base + j * sk]), y = ccast<double>(gv[i * H + base + jp * sk]);
                acc = cfmac(y, w * x, acc);
            }
        }
        const double act = (j == jp && lam_get(lam, CHI, ek, j) > 0.0) ? 1.0 : 0.0;
        A[r] = cd{act - acc.x, -acc.y};
    }
    if (g == 0) tn = 0.0;
    __syncthreads();
    BlockGroup grp{&flag};
    jacobi_svd<CHI, double, BlockGroup, false>(A, nullptr, g, grp, group_mask<CHI>(), 1e-15, 60, false);
    __syncthreads();
    if (g < CHI) {
        double c2 = 0.0;
        for (int r = 0; r < CHI; ++r) c2 += norm2(A[g * CHI + r]);
        atomicAdd(&tn, sqrt(c2));
    }
    __syncthreads();
    if (g == 0) atomicAdd(out, tn);
}

// One step of the measurement sampling of Sec. IV A on the plain layout (one warp, vertex a):
// p0 = rho_a[0][0] as in plain_marginals_kernel, the outcome x_a = +1 if u < p0 (else -1) and its
// probability, then the projection of Eq. (projection): the other physical component of
// Gamma_a is zeroed.
template <int CHI, int D, typename R>
__global__ void plain_sample_kernel(C<R>* Gamma, const double* lam, const int4* vslots, int a, double u, int step,
                                    int8_t* x_out, double* p_out) {
    constexpr int H = PlainShape<CHI, D, R>::H;
    const int lane = threadIdx.x & 31;
    const int4 sl = vslots[a];
    C<R>* g = Gamma + (size_t)a * 2 * H;
    double r00 = 0.0, r11 = 0.0;
    for (int r = lane; r < H; r += 32) {
        int rem = r;
        double wgt = 1.0;
        for (int k = D - 1; k >= 0; --k) {
            const double l = lam_get(lam, CHI, plain_slot_edge(sl, k), rem % CHI);
            wgt *= l * l;
            rem /= CHI;
        }
        r00 += wgt * norm2(ccast<double>(g[r]));
        r11 += wgt * norm2(ccast<double>(g[H + r]));
    }
    r00 = group_sum<32>(r00, 0xffffffffu);
    r11 = group_sum<32>(r11, 0xffffffffu);
    const double p0 = r00 / (r00 + r11);
    const int keep = u < p0 ? 0 : 1;
    if (lane == 0) {
        x_out[a] = keep == 0 ? 1 : -1;
        p_out[step] = keep == 0 ? p0 : r11 / (r00 + r11);
    }
    for (int r = lane; r < H; r += 32) g[(1 - keep) * H + r] = C<R>{(R)0, (R)0};
}

// ---------------------------------------------------------------------------
// CHI = 16, degree 3: the simple update of a diagonal gate (App. E) in QR-reduced form, one
// block of 512 threads per edge.  The four blocks A_{x,i}[J, j] = w_x[J] Gamma_x[i][j][J]
// (CHI^2 x CHI) live in global scratch; each gets a Householder QR from a group of 128 threads
// (two rows each) whose sums go through shared memory.  The core
//   M[(i_a r), (i_b r')] = U[(i_a i_b), (i_a i_b)] sum_j R_{a,i_a}[r, j] lambda_j R_{b,i_b}[r', j]
// (2 CHI x 2 CHI) has the same singular values as Theta; one-sided Jacobi (512 threads),
// truncation to chi as in App. D "Truncation", and the new Gamma from the reflectors.
// ---------------------------------------------------------------------------
struct Gate16Args {
    void* Gamma;
    double* lam;
    const int4* edge_info;
    const int4* vslots;
    const int* gate_edge;
    const cd* gate_U;         // [gates][16], diagonal used
    cd* scratch;              // [gates in launch][4][CHI][CHI^2]
    int count;
    double* stats;
    int chi;
    double svd_cut;
};

template <int CHI, typename R>
struct Gate16Sm {
    using CR = C<R>;
    static constexpr int NM = 2 * CHI, NR = CHI * CHI;
    CR M[NM * NM];
    CR V[NM * NM];
    CR vk[4][CHI];
    R st[4][CHI];             // square roots of the reflector coefficients
    R w[2][NR];
    R lab[CHI];
    CR ph[4];
    R sig[NM];
    int perm[NM];
    CR red[4][4][CHI];        // [group][warp][value] partial sums
    int keep, flag, nrot;
};

// sum over the 128 threads of group grp of vals[0..nv) (complex), returned to every thread;
// red is [4 warps][nv]; named barrier 1 + grp
template <int NV, typename CR>
__device__ __forceinline__ void group128_sum(CR (&vals)[NV], int nv, CR (*red)[16], int grp) {
    const int lane = threadIdx.x & 31, wig = (threadIdx.x / 32) & 3;
    for (int q = 0; q < nv; ++q) {
        vals[q].x = group_sum<32>(vals[q].x, 0xffffffffu);
        vals[q].y = group_sum<32>(vals[q].y, 0xffffffffu);
        if (lane == 0) red[wig][q] = vals[q];
    }
    asm volatile("bar.sync %0, 128;" ::"r"(1 + grp) : "memory");
    for (int q = 0; q < nv; ++q) vals[q] = red[0][q] + red[1][q] + red[2][q] + red[3][q];
    asm volatile("bar.sync %0, 128;" ::"r"(1 + grp) : "memory");
}

// TS is the storage type of Gamma, R the arithmetic type: (double, double) is the FP64
// precision mode, (float, float) the complex64 mode (QR, Jacobi SVD and the new Gamma in FP32)
// and (float, double) the mixed mode (FP64 QR and SVD on complex64 Gamma).  lambda is always
// written as float64.
template <int CHI, typename TS, typename R>
__global__ void __launch_bounds__(512, 1) ising16_gate_kernel(Gate16Args c) {
    using CR = C<R>;
    constexpr bool R64 = sizeof(R) == 8;
    constexpr int NM = 2 * CHI, NR = CHI * CHI, H = CHI * CHI * CHI;
    static_assert(NR == 2 * 128, "the 128-thread groups hold two rows each");
    __shared__ Gate16Sm<CHI, R> sm;
    const int tid = threadIdx.x;
    const int e = c.gate_edge[blockIdx.x];
    const int4 ei = c.edge_info[e];
    const int vtx[2] = {ei.x, ei.y};
    const int slot[2] = {ei.z, ei.w};
    int oe[2][2], os[2][2];
    for (int x = 0; x < 2; ++x) {
        const int4 ve = c.vslots[vtx[x]];
        const int es[3] = {ve.x, ve.y, ve.z};
        others_of(slot[x], os[x][0], os[x][1]);
        oe[x][0] = es[os[x][0]];
        oe[x][1] = es[os[x][1]];
    }
    CR* Xg = reinterpret_cast<CR*>(c.scratch) + (size_t)blockIdx.x * 4 * CHI * NR;   // [blk][col][row]
    C<TS>* Gam = (C<TS>*)c.Gamma;
    for (int t = tid; t < 2 * NR; t += 512) {
        const int x = t / NR, J = t % NR;
        sm.w[x][J] = (R)(lam_get(c.lam, CHI, oe[x][0], J / CHI) * lam_get(c.lam, CHI, oe[x][1], J % CHI));
    }
    for (int t = tid; t < CHI; t += 512) sm.lab[t] = (R)c.lam[(size_t)e * CHI + t];
    if (tid < 4) sm.ph[tid] = ccast<R>(c.gate_U[(size_t)blockIdx.x * 16 + 5 * tid]);
    if (tid == 0) sm.nrot = 0;
    __syncthreads();
    for (int t = tid; t < 4 * CHI * NR; t += 512) {
        const int blk = t / (CHI * NR), rem = t % (CHI * NR);
        const int col = rem / NR, row = rem % NR;
        const int x = blk >> 1, i = blk & 1;
        const size_t off = (size_t)vtx[x] * 2 * H + (size_t)i * H + col * sstride<CHI>(slot[x]) +
                           (row / CHI) * sstride<CHI>(os[x][0]) + (row % CHI) * sstride<CHI>(os[x][1]);
        Xg[((size_t)blk * CHI + col) * NR + row] = sm.w[x][row] * ccast<R>(Gam[off]);
    }
    __syncthreads();
    // ---- Householder QR of the four blocks, 128 threads per block, rows l and l + 128 ----
    const int blk = tid / 128, l = tid % 128;
    CR* Xb = Xg + (size_t)blk * CHI * NR;
    for (int k = 0; k < CHI; ++k) {
        CR* Xk = Xb + (size_t)k * NR;
        const CR z = CR{(R)0, (R)0};
        CR x0 = (l >= k) ? Xk[l] : z;
        CR x1 = Xk[l + 128];
        CR nv[1] = {CR{norm2(x0) + norm2(x1), (R)0}};
        group128_sum<1>(nv, 1, sm.red[blk], blk);
        const R nrm = nr_sqrt(nv[0].x);
        const CR xkk = Xk[k];
        const R a2 = norm2(xkk);
        const R ra = a2 > (R)0 ? nr_rsqrt(a2) : (R)0;
        const R axkk = a2 * ra;
        const CR ph = a2 > (R)0 ? CR{xkk.x * ra, xkk.y * ra} : CR{(R)1, (R)0};
        const R stau = nrm > (R)0 ? nr_rsqrt(nrm * (nrm + axkk)) : (R)0;
        const R tau = stau * stau;
        const CR vkk = (axkk + nrm) * ph;
        const CR v0 = (l == k) ? vkk : x0;
        const CR v1 = x1;
        CR d[CHI];
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) {
            d[cc] = z;
            if (cc > k) {
                const CR* Xc = Xb + (size_t)cc * NR;
                d[cc] = cfmac(v0, Xc[l], cfmac(v1, Xc[l + 128], z));
            }
        }
        group128_sum<CHI>(d, CHI, sm.red[blk], blk);
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) {
            if (cc <= k) continue;
            CR* Xc = Xb + (size_t)cc * NR;
            const CR td = tau * d[cc];
            if (l >= k) Xc[l] = Xc[l] - v0 * td;
            Xc[l + 128] = Xc[l + 128] - v1 * td;
        }
        if (l == k) Xk[k] = (-nrm) * ph;
        if (l == 0) {
            sm.vk[blk][k] = vkk;
            sm.st[blk][k] = stau;
        }
        asm volatile("bar.sync %0, 128;" ::"r"(1 + blk) : "memory");
    }
    __syncthreads();
    // ---- core M (column-major NM x NM) with the diagonal gate ----
    for (int t = tid; t < NM * NM; t += 512) {
        const int col = t / NM, row = t % NM;
        const int ia = row / CHI, r = row % CHI, ib = col / CHI, rp = col % CHI;
        const CR* Ra = Xg + (size_t)ia * CHI * NR;          // block (a, ia)
        const CR* Rb = Xg + (size_t)(2 + ib) * CHI * NR;    // block (b, ib)
        CR acc = CR{(R)0, (R)0};
        const int j0 = r > rp ? r : rp;
        for (int j = j0; j < CHI; ++j) acc = cfma(sm.lab[j] * Ra[(size_t)j * NR + r], Rb[(size_t)j * NR + rp], acc);
        sm.M[t] = sm.ph[2 * ia + ib] * acc;
    }
    __syncthreads();
    int nrot = 0;
    BlockGroup grp{&sm.flag};
    const int sweeps = jacobi_svd<NM, R, BlockGroup, true, R64>(sm.M, sm.V, tid, grp, group_mask<NM>(),
                                                                (R)(R64 ? 1e-15 : 1e-6), 60, true, &nrot,
                                                                (R)(R64 ? 3e-8 : 1e-3));
    if (nrot) atomicAdd(&sm.nrot, nrot);
    __syncthreads();
    for (int cc = tid; cc < NM; cc += 512) {
        R s2 = (R)0;
        for (int r = 0; r < NM; ++r) s2 += norm2(sm.M[cc * NM + r]);
        sm.sig[cc] = nr_sqrt(s2);
    }
    __syncthreads();
    for (int cc = tid; cc < NM; cc += 512) sm.perm[desc_rank(sm.sig, NM, cc)] = cc;
    __syncthreads();
    if (tid < NM) {   // lane r holds the r-th largest singular value (NM = 32: one warp)
        const unsigned mk = group_mask<NM>();
        const R sv = sm.sig[sm.perm[tid]];
        const R smax = sm.sig[sm.perm[0]];
        const int cnt = __popc(__ballot_sync(mk, sv > (R)c.svd_cut * smax));
        int keep = cnt < c.chi ? cnt : c.chi;
        if (keep < 1) keep = 1;
        const R s2 = sv * sv;
        const R kept = group_sum<NM>(tid < keep ? s2 : (R)0, mk);
        const R drop = group_sum<NM>(tid < keep ? (R)0 : s2, mk);
        const R inv = kept > (R)0 ? nr_rsqrt(kept) : (R)0;
        if (tid < CHI) c.lam[(size_t)e * CHI + tid] = (tid < keep) ? (double)(sv * inv) : 0.0;
        if (tid == 0) {
            const R tot = kept + drop;
            const R disc = tot > (R)0 ? drop * nr_rcp(tot) : (R)0;
            atomicAdd(&c.stats[0], (double)disc);
            atomicAdd(&c.stats[1], 2.0 * log1p(-(double)disc));   // Eq. (gate_fidelity)
            atomicAdd(&c.stats[2], (double)sweeps * (NM - 1) * (NM / 2));
            atomicAdd(&c.stats[3], (double)sm.nrot);
            sm.keep = keep;
        }
    }
    __syncthreads();
    const int keep = sm.keep;
    // ---- new Gamma: the reflectors of each block applied to U (side a) / V^* (side b) ----
    const int x = blk >> 1, i = blk & 1;
    CR E0[CHI], E1[CHI];
#pragma unroll
    for (int cc = 0; cc < CHI; ++cc) {
        E0[cc] = CR{(R)0, (R)0};
        E1[cc] = CR{(R)0, (R)0};
        if (l < CHI && cc < keep) {
            const int pc = sm.perm[cc];
            const int row = i * CHI + l;
            E0[cc] = (x == 0) ? nr_rcp(sm.sig[pc]) * sm.M[pc * NM + row] : conj(sm.V[pc * NM + row]);
        }
    }
    for (int k = CHI - 1; k >= 0; --k) {
        const R st = sm.st[blk][k];
        const CR* Xk = Xb + (size_t)k * NR;
        const CR v0 = st * ((l == k) ? sm.vk[blk][k] : ((l > k) ? Xk[l] : CR{(R)0, (R)0}));
        const CR v1 = st * Xk[l + 128];
        CR d[CHI];
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) d[cc] = cfmac(v0, E0[cc], cfmac(v1, E1[cc], CR{(R)0, (R)0}));
        group128_sum<CHI>(d, CHI, sm.red[blk], blk);
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) {
            E0[cc] = E0[cc] - v0 * d[cc];
            E1[cc] = E1[cc] - v1 * d[cc];
        }
    }
    const R w0 = sm.w[x][l], w1 = sm.w[x][l + 128];
    const R iw0 = w0 > (R)0 ? nr_rcp(w0) : (R)0, iw1 = w1 > (R)0 ? nr_rcp(w1) : (R)0;
    const size_t base = (size_t)vtx[x] * 2 * H + (size_t)i * H;
    const size_t o0 = (l / CHI) * sstride<CHI>(os[x][0]) + (l % CHI) * sstride<CHI>(os[x][1]);
    const size_t o1 = ((l + 128) / CHI) * sstride<CHI>(os[x][0]) + ((l + 128) % CHI) * sstride<CHI>(os[x][1]);
#pragma unroll
    for (int cc = 0; cc < CHI; ++cc) {
        Gam[base + cc * sstride<CHI>(slot[x]) + o0] = ccast<TS>(iw0 * E0[cc]);
        Gam[base + cc * sstride<CHI>(slot[x]) + o1] = ccast<TS>(iw1 * E1[cc]);
    }
}

}  // namespace gtqa
