// GTQA hot-path kernels (FP64 reference-precision path).
//
// Layout (see gtqa.h): Gamma[n][2][CHI][CHI][CHI] complex, slot k of a vertex is its
// k-th incident edge in ascending id; lambda[m][CHI]; messages[2m][CHI][CHI] with
// row 2e = m_{u->v}, 2e+1 = m_{v->u}.  Phantom slots (degree < 3) have dimension 1:
// lambda = (1, 0, ...), message = e_0 e_0^T, only index 0 of Gamma is used.
#pragma once

#include "gtqa_common.cuh"

namespace gtqa {

struct GraphView {
    const int4* edge_info;   // per edge: u, v, slot of e in u, slot of e in v
    const int4* vert_edges;  // per vertex: edge id at slots 0, 1, 2 (-1 = phantom), degree
    const int* vert_inst;    // instance id of each vertex
    const int* edge_inst;    // instance id of each edge
    const double* J;
    const double* h;
    int n, m;
};

template <int CHI> __host__ __device__ constexpr int slot_stride(int k) {
    return k == 0 ? CHI * CHI : (k == 1 ? CHI : 1);
}
__host__ __device__ inline void other_slots(int s, int& o0, int& o1) {
    o0 = (s == 0) ? 1 : 0;
    o1 = (s == 2) ? 1 : 2;
}
// lambda_e[j] with the phantom convention for e < 0
__device__ __forceinline__ double lam_at(const double* lam, int CHI, int e, int j) {
    return e < 0 ? (j == 0 ? 1.0 : 0.0) : lam[(size_t)e * CHI + j];
}
// directed message indices seen from vertex a on edge e = (u, v)
__device__ __forceinline__ int msg_out(int e, int a, int u) { return 2 * e + (a == u ? 0 : 1); }
__device__ __forceinline__ int msg_in(int e, int a, int u) { return 2 * e + (a == u ? 1 : 0); }

template <int TEAM>
__device__ __forceinline__ void team_sync() {
    if (TEAM <= 32) __syncwarp(group_mask<(TEAM <= 32 ? TEAM : 32)>());
    else __syncthreads();
}

// ===========================================================================
// K2: two-qubit gate + truncation on every edge of one colour class (App. E,
// App. D "Truncation").  QR-reduced form of the paper's dense Theta SVD:
//   X_{a,i}[J, j] = Gamma_a[i, J, j] prod lambda_other(J)      (CHI^2 x CHI, i = 0, 1)
//   X_{a,i} = Q_{a,i} R_{a,i} (Householder), same for b,
//   M[(i_a r), (i_b r')] = w(i_a, i_b) sum_j R_{a,i_a}[r, j] lambda_ab[j] R_{b,i_b}[r', j]
// so Theta = blockdiag(Q_a) M blockdiag(Q_b)^T has the singular values of M.
//   M = U S V^H (one-sided Jacobi), keep the chi largest,
//   Gamma~_a[i, J, j] = (Q_{a,i} U_i)[J, j] / prod lambda_other(J),
//   Gamma~_b[i, J, j] = (Q_{b,i} V^*_i)[J, j] / prod lambda_other(J),  lambda~ = S / ||S||.
// ===========================================================================
template <int CHI>
struct GateShape {
    static constexpr int TEAM = 2 * CHI * CHI;               // = (2CHI)^2 / 2, one Jacobi group
    static constexpr int TPB = TEAM >= 128 ? TEAM : 128;
    static constexpr int TEAMS = TPB / TEAM;
    static constexpr int NM = 2 * CHI;
    static constexpr int NR = CHI * CHI;
    static constexpr int G = NR / 2;                          // threads per QR block
};

template <int CHI>
struct GateSmem {
    cd X[4][CHI][CHI * CHI];   // [block][col][row]; blocks (a,0) (a,1) (b,0) (b,1)
    cd vk[4][CHI];
    double tau[4][CHI];
    cd M[4 * CHI * CHI];
    cd V[4 * CHI * CHI];
    double w[2][CHI * CHI];
    double lab[CHI];
    double sig[2 * CHI];
    int perm[2 * CHI];
    double scal[2];            // 1/norm of kept singular values, keep count
    int flag;
    int nrot;
};

template <typename TS>
struct GateArgs {
    C<TS>* Gamma;
    double* lam;
    const int* edge_list;      // edges of this colour
    int count;
    GraphView g;
    double tZ;
    int chi;
    double svd_cutoff;
    double* disc;              // per edge: discarded weight of this gate
    int2* work;                // per edge: (Jacobi sweeps, rotations) of the core SVD
};

template <int CHI, typename TS>
__global__ void __launch_bounds__(GateShape<CHI>::TPB)
gate_kernel(GateArgs<TS> A) {
    using S = GateShape<CHI>;
    constexpr int NM = S::NM, NR = S::NR, G = S::G, TEAM = S::TEAM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int team = threadIdx.x / TEAM;
    const int tid = threadIdx.x % TEAM;
    GateSmem<CHI>& sm = reinterpret_cast<GateSmem<CHI>*>(smem_raw)[team];
    const int idx = blockIdx.x * S::TEAMS + team;
    if (idx >= A.count) return;
    const int e = A.edge_list[idx];
    const int4 ei = A.g.edge_info[e];
    const int vtx[2] = {ei.x, ei.y};
    const int slot[2] = {ei.z, ei.w};
    int oe[2][2];   // edges at the two other slots of each side
    int os[2][2];   // the other slot indices
    for (int x = 0; x < 2; ++x) {
        const int4 ve = A.g.vert_edges[vtx[x]];
        const int es[3] = {ve.x, ve.y, ve.z};
        other_slots(slot[x], os[x][0], os[x][1]);
        oe[x][0] = es[os[x][0]];
        oe[x][1] = es[os[x][1]];
    }
    // lambda products over the flattened J = (j_o0, j_o1) of each side
    for (int t = tid; t < 2 * NR; t += TEAM) {
        const int x = t / NR, J = t % NR;
        sm.w[x][J] = lam_at(A.lam, CHI, oe[x][0], J / CHI) * lam_at(A.lam, CHI, oe[x][1], J % CHI);
    }
    for (int t = tid; t < CHI; t += TEAM) sm.lab[t] = A.lam[(size_t)e * CHI + t];
    team_sync<TEAM>();
    // X blocks
    for (int t = tid; t < 4 * CHI * NR; t += TEAM) {
        const int blk = t / (CHI * NR), rem = t % (CHI * NR);
        const int col = rem / NR, row = rem % NR;
        const int x = blk >> 1, i = blk & 1;
        const size_t off = (size_t)vtx[x] * (2 * CHI * CHI * CHI) + (size_t)i * CHI * CHI * CHI +
                           col * slot_stride<CHI>(slot[x]) + (row / CHI) * slot_stride<CHI>(os[x][0]) +
                           (row % CHI) * slot_stride<CHI>(os[x][1]);
        const cd gv = ccast<double>(A.Gamma[off]);
        sm.X[blk][col][row] = sm.w[x][row] * gv;
    }
    team_sync<TEAM>();

    // ---- Householder QR of the four CHI^2 x CHI blocks (G threads per block) ----
    const int blk = tid / G, l = tid % G;
    const unsigned gm = group_mask<G>();
    const int r0 = l, r1 = l + G;
    for (int k = 0; k < CHI; ++k) {
        cd* Xk = sm.X[blk][k];
        const cd z = cd{0.0, 0.0};
        const cd x0 = (r0 >= k) ? Xk[r0] : z;
        const cd x1 = (r1 >= k) ? Xk[r1] : z;
        const double nrm2 = group_sum<G>(norm2(x0) + norm2(x1), gm);
        const cd xkk = Xk[k];
        const double nrm = sqrt(nrm2);
        const double axkk = sqrt(norm2(xkk));
        const cd ph = axkk > 0.0 ? cd{xkk.x / axkk, xkk.y / axkk} : cd{1.0, 0.0};
        const double tau = nrm > 0.0 ? 1.0 / (nrm * (nrm + axkk)) : 0.0;
        const cd vkk = (axkk + nrm) * ph;
        const cd v0 = (r0 == k) ? vkk : x0;
        const cd v1 = x1;
        for (int c = k + 1; c < CHI; ++c) {
            cd* Xc = sm.X[blk][c];
            const cd y0 = Xc[r0], y1 = Xc[r1];
            cd d = cfmac(v0, y0, cfmac(v1, y1, z));
            d.x = group_sum<G>(d.x, gm);
            d.y = group_sum<G>(d.y, gm);
            const cd td = tau * d;
            if (r0 >= k) Xc[r0] = y0 - v0 * td;
            Xc[r1] = y1 - v1 * td;
        }
        __syncwarp(gm);
        if (r0 == k) Xk[k] = (-nrm) * ph;   // R diagonal; rows > k keep the reflector
        if (l == 0) {
            sm.vk[blk][k] = vkk;
            sm.tau[blk][k] = tau;
        }
        __syncwarp(gm);
    }
    team_sync<TEAM>();

    // ---- core matrix M (column-major, NM x NM) ----
    const double* Jv = A.g.J;
    const double* hv = A.g.h;
    const int Da = A.g.vert_edges[vtx[0]].w, Db = A.g.vert_edges[vtx[1]].w;
    const double ha = hv[vtx[0]] / Da, hb = hv[vtx[1]] / Db, Je = Jv[e];
    for (int t = tid; t < NM * NM; t += TEAM) {
        const int col = t / NM, row = t % NM;
        const int ia = row / CHI, r = row % CHI, ib = col / CHI, rp = col % CHI;
        cd acc = cd{0.0, 0.0};
        const int j0 = r > rp ? r : rp;
        for (int j = j0; j < CHI; ++j) {
            const cd ra = sm.X[ia][j][r];
            const cd rb = sm.X[2 + ib][j][rp];
            acc = cfma(sm.lab[j] * ra, rb, acc);
        }
        const double za = 1.0 - 2.0 * ia, zb = 1.0 - 2.0 * ib;
        const double phase = -A.tZ * (Je * za * zb + ha * za + hb * zb);
        double sn, cs;
        sincos(phase, &sn, &cs);
        sm.M[t] = cd{cs, sn} * acc;
    }
    team_sync<TEAM>();

    // ---- SVD of M ----
    if (tid == 0) sm.nrot = 0;
    int nrot = 0, sweeps;
    if constexpr (TEAM <= 32) {
        WarpGroup grp{group_mask<TEAM>()};
        sweeps = jacobi_svd<NM, double>(sm.M, sm.V, tid, grp, group_mask<NM>(), 1e-15, 60, true, &nrot);
    } else {
        BlockGroup grp{&sm.flag};
        sweeps = jacobi_svd<NM, double>(sm.M, sm.V, tid, grp, group_mask<NM>(), 1e-15, 60, true, &nrot);
    }
    if (nrot) atomicAdd(&sm.nrot, nrot);
    team_sync<TEAM>();
    if (tid == 0) A.work[e] = make_int2(sweeps, sm.nrot);
    for (int c = tid; c < NM; c += TEAM) {
        double s2 = 0.0;
        for (int r = 0; r < NM; ++r) s2 += norm2(sm.M[c * NM + r]);
        sm.sig[c] = sqrt(s2);
    }
    team_sync<TEAM>();
    for (int c = tid; c < NM; c += TEAM) sm.perm[desc_rank(sm.sig, NM, c)] = c;
    team_sync<TEAM>();
    if (tid == 0) {
        const double smax = sm.sig[sm.perm[0]];
        int cnt = 0;
        double tot = 0.0;
        for (int r = 0; r < NM; ++r) {
            const double s = sm.sig[sm.perm[r]];
            tot += s * s;
            cnt += (s > A.svd_cutoff * smax) ? 1 : 0;
        }
        int keep = cnt < A.chi ? cnt : A.chi;
        if (keep < 1) keep = 1;
        double kept = 0.0, drop = 0.0;
        for (int r = 0; r < NM; ++r) {
            const double s = sm.sig[sm.perm[r]];
            if (r < keep) kept += s * s; else drop += s * s;
        }
        const double inv = kept > 0.0 ? 1.0 / sqrt(kept) : 0.0;
        for (int r = 0; r < CHI; ++r)
            A.lam[(size_t)e * CHI + r] = (r < keep) ? sm.sig[sm.perm[r]] * inv : 0.0;
        A.disc[e] = tot > 0.0 ? drop / tot : 0.0;
        sm.scal[1] = (double)keep;
    }
    team_sync<TEAM>();
    const int keep = (int)sm.scal[1];

    // ---- new Gamma: apply the block reflectors to U (side a) or V^* (side b) ----
    {
        const int x = blk >> 1, i = blk & 1;
        cd E0[CHI], E1[CHI];
#pragma unroll
        for (int c = 0; c < CHI; ++c) {
            E1[c] = cd{0.0, 0.0};
            E0[c] = cd{0.0, 0.0};
            if (r0 < CHI && c < keep) {
                const int pc = sm.perm[c];
                const int row = i * CHI + r0;
                if (x == 0) E0[c] = (1.0 / sm.sig[pc]) * sm.M[pc * NM + row];
                else E0[c] = conj(sm.V[pc * NM + row]);
            }
        }
        for (int k = CHI - 1; k >= 0; --k) {
            const double tau = sm.tau[blk][k];
            const cd v0 = (r0 == k) ? sm.vk[blk][k] : ((r0 > k) ? sm.X[blk][k][r0] : cd{0.0, 0.0});
            const cd v1 = sm.X[blk][k][r1];
#pragma unroll
            for (int c = 0; c < CHI; ++c) {
                cd d = cfmac(v0, E0[c], cfmac(v1, E1[c], cd{0.0, 0.0}));
                d.x = group_sum<G>(d.x, gm);
                d.y = group_sum<G>(d.y, gm);
                const cd td = tau * d;
                E0[c] = E0[c] - v0 * td;
                E1[c] = E1[c] - v1 * td;
            }
        }
        const double w0 = sm.w[x][r0], w1 = sm.w[x][r1];
        const double iw0 = w0 > 0.0 ? 1.0 / w0 : 0.0, iw1 = w1 > 0.0 ? 1.0 / w1 : 0.0;
        const size_t base = (size_t)vtx[x] * (2 * CHI * CHI * CHI) + (size_t)i * CHI * CHI * CHI;
        const int so0 = slot_stride<CHI>(os[x][0]), so1 = slot_stride<CHI>(os[x][1]);
        const int ss = slot_stride<CHI>(slot[x]);
#pragma unroll
        for (int c = 0; c < CHI; ++c) {
            A.Gamma[base + c * ss + (r0 / CHI) * so0 + (r0 % CHI) * so1] = ccast<TS>(iw0 * E0[c]);
            A.Gamma[base + c * ss + (r1 / CHI) * so0 + (r1 % CHI) * so1] = ccast<TS>(iw1 * E1[c]);
        }
    }
}

// ===========================================================================
// K1: mixing gate exp(-i t X) on every vertex (Sec. II D).
// ===========================================================================
template <int CHI, typename TS>
__global__ void xrot_kernel(C<TS>* Gamma, int n, double tX) {
    constexpr int H = CHI * CHI * CHI;
    const size_t total = (size_t)n * H;
    double sn, cs;
    sincos(tX, &sn, &cs);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t a = t / H, r = t % H;
        C<TS>* g = Gamma + a * 2 * H;
        const cd g0 = ccast<double>(g[r]), g1 = ccast<double>(g[H + r]);
        // [[c, -i s], [-i s, c]]
        const cd n0 = cd{cs * g0.x + sn * g1.y, cs * g0.y - sn * g1.x};
        const cd n1 = cd{sn * g0.y + cs * g1.x, -sn * g0.x + cs * g1.y};
        g[r] = ccast<TS>(n0);
        g[H + r] = ccast<TS>(n1);
    }
}

// ===========================================================================
// Symmetric split T_a = Gamma_a prod_b lambda_ba^{1/2}, Eq. (symmetric_gauge).
// ===========================================================================
template <int CHI, typename TS>
__global__ void symmetric_kernel(const C<TS>* Gamma, const double* lam, GraphView g, cd* T) {
    constexpr int H = CHI * CHI * CHI;
    const size_t total = (size_t)g.n * 2 * H;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / (2 * H));
        const int r = (int)(t % H);
        const int4 ve = g.vert_edges[a];
        const int j0 = r / (CHI * CHI), j1 = (r / CHI) % CHI, j2 = r % CHI;
        const double f = sqrt(lam_at(lam, CHI, ve.x, j0)) * sqrt(lam_at(lam, CHI, ve.y, j1)) *
                         sqrt(lam_at(lam, CHI, ve.z, j2));
        T[t] = f * ccast<double>(Gamma[t]);
    }
}

// Warm-start messages m_{a->b} = diag(lambda_ab) / sum(lambda_ab), Eq. (reconstructed_messages)
// with the lambda (not lambda^{1/2}) reading.
template <int CHI>
__global__ void warm_start_kernel(const double* lam, int m, cd* msg) {
    const size_t total = (size_t)m * 2 * CHI * CHI;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t dm = t / (CHI * CHI);
        const int r = (int)(t % (CHI * CHI));
        const size_t e = dm / 2;
        const int j = r / CHI, jp = r % CHI;
        double s = 0.0;
        for (int q = 0; q < CHI; ++q) s += lam[e * CHI + q];
        msg[t] = cd{(j == jp && s > 0.0) ? lam[e * CHI + j] / s : 0.0, 0.0};
    }
}

// ===========================================================================
// K3: one flooding BP sweep (App. B), FP64.  One team per vertex a computes its
// outgoing messages m_{a->b} from T_a and the previous incoming messages,
// Eq. (local_consistency), normalises them to unit trace and adds the trace
// norms ||m_new - m_old||_1 into vdelta[a].
// ===========================================================================
template <int CHI>
struct BPShape {
    static constexpr int TEAM = (2 * CHI * CHI >= 32) ? 2 * CHI * CHI : 32;
    static constexpr int TPB = TEAM >= 128 ? TEAM : 128;
    static constexpr int TEAMS = TPB / TEAM;
};

template <int CHI>
struct BPSmem {
    cd T[2 * CHI * CHI * CHI];
    cd P[2 * CHI * CHI * CHI];
    cd Q[2 * CHI * CHI * CHI];
    cd min[3][CHI * CHI];
    cd mout[3][CHI * CHI];
    cd D[3][CHI * CHI];
    cd DV[3][CHI * CHI];
    double tr[3];
    double dl[3];
};

struct BPArgs {
    const cd* T;
    const cd* src;
    cd* dst;
    double* vdelta;
    const int* inst_done;
    GraphView g;
};

template <int CHI>
__global__ void __launch_bounds__(BPShape<CHI>::TPB)
bp_sweep_kernel(BPArgs A) {
    using S = BPShape<CHI>;
    constexpr int TEAM = S::TEAM, CC = CHI * CHI, H = CHI * CHI * CHI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int team = threadIdx.x / TEAM;
    const int tid = threadIdx.x % TEAM;
    BPSmem<CHI>& sm = reinterpret_cast<BPSmem<CHI>*>(smem_raw)[team];
    const int a = blockIdx.x * S::TEAMS + team;
    if (a >= A.g.n) return;
    const int4 ve = A.g.vert_edges[a];
    const int es[3] = {ve.x, ve.y, ve.z};
    int out_idx[3], in_idx[3];
    for (int k = 0; k < 3; ++k) {
        if (es[k] >= 0) {
            const int u = A.g.edge_info[es[k]].x;
            out_idx[k] = msg_out(es[k], a, u);
            in_idx[k] = msg_in(es[k], a, u);
        } else {
            out_idx[k] = in_idx[k] = -1;
        }
    }
    if (A.inst_done[A.g.vert_inst[a]]) {
        for (int k = 0; k < 3; ++k) {
            if (out_idx[k] < 0) continue;
            for (int t = tid; t < CC; t += TEAM) A.dst[(size_t)out_idx[k] * CC + t] = A.src[(size_t)out_idx[k] * CC + t];
        }
        if (tid == 0) A.vdelta[a] = 0.0;
        return;
    }
    for (int t = tid; t < 2 * H; t += TEAM) sm.T[t] = A.T[(size_t)a * 2 * H + t];
    for (int t = tid; t < 3 * CC; t += TEAM) {
        const int k = t / CC, r = t % CC;
        cd v;
        if (in_idx[k] >= 0) v = A.src[(size_t)in_idx[k] * CC + r];
        else v = cd{r == 0 ? 1.0 : 0.0, 0.0};
        sm.min[k][r] = v;
    }
    team_sync<TEAM>();
    for (int s = 0; s < 3; ++s) {
        if (es[s] < 0) continue;
        int o0, o1;
        other_slots(s, o0, o1);
        const int ss = slot_stride<CHI>(s), s0 = slot_stride<CHI>(o0), s1 = slot_stride<CHI>(o1);
        // P[i][a'][b][j] = sum_a T[i; a@o0, b@o1, j@s] m_o0[a][a']
        for (int t = tid; t < 2 * H; t += TEAM) {
            const int i = t / H, ap = (t / CC) % CHI, b = (t / CHI) % CHI, j = t % CHI;
            cd acc = cd{0.0, 0.0};
            for (int q = 0; q < CHI; ++q)
                acc = cfma(sm.T[i * H + q * s0 + b * s1 + j * ss], sm.min[o0][q * CHI + ap], acc);
            sm.P[t] = acc;
        }
        team_sync<TEAM>();
        // Q[i][a'][b'][j] = sum_b P[i][a'][b][j] m_o1[b][b']
        for (int t = tid; t < 2 * H; t += TEAM) {
            const int i = t / H, ap = (t / CC) % CHI, bp = (t / CHI) % CHI, j = t % CHI;
            cd acc = cd{0.0, 0.0};
            for (int q = 0; q < CHI; ++q)
                acc = cfma(sm.P[i * H + ap * CC + q * CHI + j], sm.min[o1][q * CHI + bp], acc);
            sm.Q[t] = acc;
        }
        team_sync<TEAM>();
        // m[j][j'] = sum_{i,a',b'} Q[i][a'][b'][j] conj(T[i; a'@o0, b'@o1, j'@s])
        for (int t = tid; t < CC; t += TEAM) {
            const int j = t / CHI, jp = t % CHI;
            cd acc = cd{0.0, 0.0};
            for (int i = 0; i < 2; ++i)
                for (int ap = 0; ap < CHI; ++ap)
                    for (int bp = 0; bp < CHI; ++bp)
                        acc = cfmac(sm.T[i * H + ap * s0 + bp * s1 + jp * ss],
                                    sm.Q[i * H + ap * CC + bp * CHI + j], acc);
            sm.mout[s][t] = acc;
        }
        team_sync<TEAM>();
    }
    // unit trace, difference to the previous outgoing message
    if (tid < 3) {
        double tr = 0.0;
        if (es[tid] >= 0)
            for (int j = 0; j < CHI; ++j) tr += sm.mout[tid][j * CHI + j].x;
        sm.tr[tid] = tr;
    }
    team_sync<TEAM>();
    for (int t = tid; t < 3 * CC; t += TEAM) {
        const int k = t / CC, r = t % CC;
        if (es[k] < 0) {
            sm.D[k][r] = cd{0.0, 0.0};
            continue;
        }
        const cd nv = (1.0 / sm.tr[k]) * sm.mout[k][r];
        sm.mout[k][r] = nv;
        A.dst[(size_t)out_idx[k] * CC + r] = nv;
        sm.D[k][r] = nv - A.src[(size_t)out_idx[k] * CC + r];
    }
    team_sync<TEAM>();
    // trace norms: one Jacobi group of CHI*CHI/2 threads per message
    constexpr int GJ = CC / 2;
    if (tid < 3 * GJ) {
        const int k = tid / GJ, g = tid % GJ;
        WarpGroup grp{group_mask<GJ>()};
        jacobi_svd<CHI, double>(sm.D[k], sm.DV[k], g, grp, group_mask<CHI>(), 1e-15, 60, true);
        if (g == 0) {
            double s = 0.0;
            for (int c = 0; c < CHI; ++c) {
                double n2 = 0.0;
                for (int r = 0; r < CHI; ++r) n2 += norm2(sm.D[k][c * CHI + r]);
                s += sqrt(n2);
            }
            sm.dl[k] = s;
        }
    }
    team_sync<TEAM>();
    if (tid == 0) A.vdelta[a] = sm.dl[0] + sm.dl[1] + sm.dl[2];
}

// dist_b = sum_{a in b} vdelta[a] / |E_b|; per-instance stopping rule of App. B.
struct ReduceArgs {
    const double* vdelta;
    const int* inst_vbeg;   // [B+1] vertex ranges of instances
    const int* inst_m;      // [B]
    int* inst_done;
    int* inst_iters;
    double* inst_dist;
    int* flags;             // [0]: all done, [1]: NaN seen
    double tol;
    int max_iter;
    int B;
};

__global__ void bp_reduce_kernel(ReduceArgs A) {
    __shared__ double part[256];
    __shared__ int notdone;
    if (threadIdx.x == 0) notdone = 0;
    __syncthreads();
    for (int b = 0; b < A.B; ++b) {
        if (A.inst_done[b]) continue;   // uniform across the block
        const int beg = A.inst_vbeg[b], end = A.inst_vbeg[b + 1];
        double s = 0.0;
        for (int a = beg + threadIdx.x; a < end; a += blockDim.x) s += A.vdelta[a];
        part[threadIdx.x] = s;
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
            if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double d = A.inst_m[b] > 0 ? part[0] / A.inst_m[b] : 0.0;
            A.inst_dist[b] = d;
            A.inst_iters[b] += 1;
            if (!(d == d)) A.flags[1] = 1;
            if (d < A.tol || A.inst_iters[b] >= A.max_iter || !(d == d)) A.inst_done[b] = 1;
            if (!A.inst_done[b]) notdone = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) A.flags[0] = notdone ? 0 : 1;
}

// ===========================================================================
// K4: Vidal gauge finding (App. D), edge part.  Per edge {a, b} (a = u):
//   m_{a->b} = W_a w_a W_a^H, P_a = m_{a->b}^{1/2}, Pi_a = m_{a->b}^{-1/2} (cut-off pseudo-inverse)
//   M = P_a^T P_b = U S V^H,   X_a = Pi_a^T U ||S||^{1/2},   X_b = Pi_b^T V^* ||S||^{1/2},
//   lambda_ab = S / ||S||.
// X[e][side][j''][j] is applied to slot e of Gamma_side by regauge_vertex_kernel.
// ===========================================================================
template <int CHI>
struct RGShape {
    static constexpr int TEAM = CHI * CHI;   // two Jacobi groups of CHI^2/2
    static constexpr int TPB = TEAM > 32 ? TEAM : 128;   // block-wide teams own their block
    static constexpr int TEAMS = TPB / TEAM;
};

template <int CHI>
struct RGSmem {
    cd Am[2][CHI * CHI];
    cd Vm[2][CHI * CHI];
    double w[2][CHI];
    cd sq[2][CHI * CHI];
    cd isq[2][CHI * CHI];
    cd M[CHI * CHI];
    cd VM[CHI * CHI];
    double sig[CHI];
    int perm[CHI];
    double scal[3];
};

struct RGArgs {
    const cd* msg;
    cd* X;            // [m][2][CHI][CHI]
    double* lam;
    int m;
    double eig_cutoff;
    double svd_cutoff;
};

template <int CHI>
__global__ void __launch_bounds__(RGShape<CHI>::TPB)
regauge_edge_kernel(RGArgs A) {
    using S = RGShape<CHI>;
    constexpr int TEAM = S::TEAM, CC = CHI * CHI, GJ = CC / 2;
    __shared__ RGSmem<CHI> smem_all[S::TEAMS];
    const int team = threadIdx.x / TEAM;
    const int tid = threadIdx.x % TEAM;
    RGSmem<CHI>& sm = smem_all[team];
    const int e = blockIdx.x * S::TEAMS + team;
    if (e >= A.m) return;
    // Hermitian parts of m_{a->b} (side 0) and m_{b->a} (side 1), column-major
    for (int t = tid; t < 2 * CC; t += TEAM) {
        const int x = t / CC, r = t % CC;
        const int row = r % CHI, col = r / CHI;
        const cd* mm = A.msg + (size_t)(2 * e + x) * CC;
        const cd v = mm[row * CHI + col], vt = mm[col * CHI + row];
        sm.Am[x][col * CHI + row] = cd{0.5 * (v.x + vt.x), 0.5 * (v.y - vt.y)};
    }
    team_sync<TEAM>();
    {
        const int x = tid / GJ, g = tid % GJ;
        WarpGroup grp{group_mask<GJ>()};
        jacobi_svd<CHI, double>(sm.Am[x], sm.Vm[x], g, grp, group_mask<CHI>(), 1e-15, 60, true);
    }
    team_sync<TEAM>();
    // eigenvalues: |w_k| = ||(A V)_k||, sign from Re(v_k^H (A V)_k)
    for (int t = tid; t < 2 * CHI; t += TEAM) {
        const int x = t / CHI, k = t % CHI;
        double n2 = 0.0, sg = 0.0;
        for (int r = 0; r < CHI; ++r) {
            const cd av = sm.Am[x][k * CHI + r], vv = sm.Vm[x][k * CHI + r];
            n2 += norm2(av);
            sg += vv.x * av.x + vv.y * av.y;
        }
        const double wv = sqrt(n2);
        sm.w[x][k] = sg >= 0.0 ? wv : -wv;
    }
    team_sync<TEAM>();
    // m^{1/2} and m^{-1/2} (row-major [j][j'])
    for (int t = tid; t < 2 * CC; t += TEAM) {
        const int x = t / CC, r = t % CC;
        const int j = r / CHI, jp = r % CHI;
        double wmax = 0.0;
        for (int k = 0; k < CHI; ++k) wmax = fmax(wmax, sm.w[x][k]);
        cd s1 = cd{0.0, 0.0}, s2 = cd{0.0, 0.0};
        for (int k = 0; k < CHI; ++k) {
            const double wk = sm.w[x][k];
            if (!(wk > A.eig_cutoff * wmax)) continue;
            const double sq = sqrt(wk);
            const cd vv = sm.Vm[x][k * CHI + j] * conj(sm.Vm[x][k * CHI + jp]);
            s1 = cfma(cd{sq, 0.0}, vv, s1);
            s2 = cfma(cd{1.0 / sq, 0.0}, vv, s2);
        }
        sm.sq[x][r] = s1;
        sm.isq[x][r] = s2;
    }
    team_sync<TEAM>();
    // M[k][l] = sum_j P_a[j][k] P_b[j][l], column-major
    for (int t = tid; t < CC; t += TEAM) {
        const int k = t % CHI, l = t / CHI;
        cd acc = cd{0.0, 0.0};
        for (int j = 0; j < CHI; ++j) acc = cfma(sm.sq[0][j * CHI + k], sm.sq[1][j * CHI + l], acc);
        sm.M[l * CHI + k] = acc;
    }
    team_sync<TEAM>();
    if (tid < GJ) {
        WarpGroup grp{group_mask<GJ>()};
        jacobi_svd<CHI, double>(sm.M, sm.VM, tid, grp, group_mask<CHI>(), 1e-15, 60, true);
    }
    team_sync<TEAM>();
    for (int c = tid; c < CHI; c += TEAM) {
        double n2 = 0.0;
        for (int r = 0; r < CHI; ++r) n2 += norm2(sm.M[c * CHI + r]);
        sm.sig[c] = sqrt(n2);
    }
    team_sync<TEAM>();
    for (int c = tid; c < CHI; c += TEAM) sm.perm[desc_rank(sm.sig, CHI, c)] = c;
    team_sync<TEAM>();
    if (tid == 0) {
        double tot = 0.0;
        for (int c = 0; c < CHI; ++c) tot += sm.sig[c] * sm.sig[c];
        const double nrm = sqrt(tot);
        sm.scal[0] = nrm;
        sm.scal[1] = sqrt(nrm);
        const double smax = sm.sig[sm.perm[0]];
        for (int r = 0; r < CHI; ++r) {
            const double s = sm.sig[sm.perm[r]];
            A.lam[(size_t)e * CHI + r] = (nrm > 0.0 && s > A.svd_cutoff * smax) ? s / nrm : 0.0;
        }
    }
    team_sync<TEAM>();
    // X_a[j''][j] = sqrt||S|| sum_j' Pi_a[j'][j''] U[j'][j];  X_b uses conj(V)
    for (int t = tid; t < 2 * CC; t += TEAM) {
        const int x = t / CC, r = t % CC;
        const int jpp = r / CHI, j = r % CHI;
        const int pc = sm.perm[j];
        const double s = sm.sig[pc];
        cd acc = cd{0.0, 0.0};
        const bool kept = sm.scal[0] > 0.0 && s > A.svd_cutoff * sm.sig[sm.perm[0]];
        if (kept) {
            for (int jp = 0; jp < CHI; ++jp) {
                const cd u = (x == 0) ? (1.0 / s) * sm.M[pc * CHI + jp] : conj(sm.VM[pc * CHI + jp]);
                acc = cfma(sm.isq[x][jp * CHI + jpp], u, acc);
            }
            acc = sm.scal[1] * acc;
        }
        A.X[((size_t)e * 2 + x) * CC + r] = acc;
    }
}

// Vertex part: Gamma_a = T_a x_{slot k} X_{e_k, side}, k = 0, 1, 2.
template <int CHI>
struct RVShape {
    static constexpr int TPB = 128;
};

template <int CHI, typename TS>
__global__ void __launch_bounds__(128)
regauge_vertex_kernel(const cd* T, const cd* X, GraphView g, C<TS>* Gamma) {
    constexpr int H = CHI * CHI * CHI, CC = CHI * CHI;
    __shared__ cd buf[2][2 * H];
    __shared__ cd Xs[3][CC];
    const int a = blockIdx.x;
    if (a >= g.n) return;
    const int4 ve = g.vert_edges[a];
    const int es[3] = {ve.x, ve.y, ve.z};
    for (int t = threadIdx.x; t < 2 * H; t += blockDim.x) buf[0][t] = T[(size_t)a * 2 * H + t];
    for (int t = threadIdx.x; t < 3 * CC; t += blockDim.x) {
        const int k = t / CC, r = t % CC;
        cd v;
        if (es[k] >= 0) {
            const int side = (g.edge_info[es[k]].x == a) ? 0 : 1;
            v = X[((size_t)es[k] * 2 + side) * CC + r];
        } else {
            v = cd{(r / CHI == r % CHI) ? 1.0 : 0.0, 0.0};
        }
        Xs[k][r] = v;
    }
    __syncthreads();
    int cur = 0;
    for (int k = 0; k < 3; ++k) {
        const int st = slot_stride<CHI>(k);
        for (int t = threadIdx.x; t < 2 * H; t += blockDim.x) {
            const int jk = (t / st) % CHI;
            const int base = t - jk * st;
            cd acc = cd{0.0, 0.0};
            for (int q = 0; q < CHI; ++q) acc = cfma(buf[cur][base + q * st], Xs[k][q * CHI + jk], acc);
            buf[cur ^ 1][t] = acc;
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int t = threadIdx.x; t < 2 * H; t += blockDim.x) Gamma[(size_t)a * 2 * H + t] = ccast<TS>(buf[cur][t]);
}

// ===========================================================================
// K5: marginals rho_a = sum Gamma Gamma^* prod lambda^2 / tr and read-out.
// ===========================================================================
template <int CHI, typename TS>
__global__ void marginals_kernel(const C<TS>* Gamma, const double* lam, GraphView g, cd* rho, int8_t* sign,
                                 int* nan_flag) {
    constexpr int H = CHI * CHI * CHI;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (warp >= g.n) return;
    const int a = warp;
    const int4 ve = g.vert_edges[a];
    cd acc[4] = {cd{0, 0}, cd{0, 0}, cd{0, 0}, cd{0, 0}};
    for (int r = lane; r < H; r += 32) {
        const int j0 = r / (CHI * CHI), j1 = (r / CHI) % CHI, j2 = r % CHI;
        const double l0 = lam_at(lam, CHI, ve.x, j0), l1 = lam_at(lam, CHI, ve.y, j1), l2 = lam_at(lam, CHI, ve.z, j2);
        const double wgt = (l0 * l0) * (l1 * l1) * (l2 * l2);
        const cd g0 = ccast<double>(Gamma[(size_t)a * 2 * H + r]);
        const cd g1 = ccast<double>(Gamma[(size_t)a * 2 * H + H + r]);
        acc[0] = cfmac(g0, wgt * g0, acc[0]);   // sum conj(g0) g0 -> rho[0][0]
        acc[1] = cfmac(g1, wgt * g0, acc[1]);   // g0 conj(g1) -> rho[0][1]
        acc[2] = cfmac(g0, wgt * g1, acc[2]);   // g1 conj(g0) -> rho[1][0]
        acc[3] = cfmac(g1, wgt * g1, acc[3]);
    }
    for (int q = 0; q < 4; ++q) {
        acc[q].x = group_sum<32>(acc[q].x, 0xffffffffu);
        acc[q].y = group_sum<32>(acc[q].y, 0xffffffffu);
    }
    if (lane == 0) {
        const double tr = acc[0].x + acc[3].x;
        const double it = 1.0 / tr;
        for (int q = 0; q < 4; ++q) rho[(size_t)a * 4 + q] = it * acc[q];
        if (sign) sign[a] = (acc[0].x * it > 0.5) ? 1 : -1;
        if (!(tr == tr) || tr == 0.0) atomicOr(nan_flag, 1);
    }
}

// Per-layer statistics: sums of discarded weights, log gate fidelities
// (Eq. (gate_fidelity)), and the core-SVD work counters (sweeps, rotations).
__global__ void layer_stats_kernel(const double* disc, const int2* work, int m, int pairs_per_sweep,
                                   double* stats) {
    __shared__ double p[4][256];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        const double d = disc[e];
        s0 += d;
        s1 += 2.0 * log1p(-d);
        const int2 w = work[e];
        s2 += (double)w.x * pairs_per_sweep;
        s3 += (double)w.y;
    }
    p[0][threadIdx.x] = s0;
    p[1][threadIdx.x] = s1;
    p[2][threadIdx.x] = s2;
    p[3][threadIdx.x] = s3;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int q = 0; q < 4; ++q) p[q][threadIdx.x] += p[q][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) stats[q] += p[q][0];
}

}  // namespace gtqa
