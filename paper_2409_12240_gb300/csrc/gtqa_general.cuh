// Arbitrary one- and two-qubit gates on the Vidal-gauge network (Sec. II D, App. E).
//
// The Ising gates of the annealing layer are diagonal, so the fused gates kernel splits
// each side by its physical index and keeps a 2 CHI x 2 CHI core.  A general 4 x 4 gate
// mixes the physical indices, so here each side x in {a, b} is reduced as a whole:
//   A_x[J, (i, j)] = w_x[J] Gamma_x[i][j][J]      (CHI^2 x 2 CHI; J = the two other bonds,
//                                                   w_x[J] their lambda weights, j = shared bond)
//   A_x = Q_x R_x                                  (Householder, FP64)
//   M[(i_a, r), (i_b, r')] = sum_{i_a' i_b'} U[(i_a i_b), (i_a' i_b')]
//                            sum_j R_a[r, (i_a', j)] lambda_j R_b[r', (i_b', j)]   (4 CHI x 4 CHI)
//   M = U_s S V^H (one-sided Jacobi, FP64), truncated to chi as in App. D "Truncation",
//   Gamma~_a[i_a][k][J] = (Q_a U_s)[(J), (i_a, k)] / w_a[J] and
//   Gamma~_b[i_b][k][J] = (Q_b conj V)[(J), (i_b, k)] / w_b[J],
// so that Theta' = Q_a M Q_b^T is the gate applied to the two-site tensor of App. E.
// One team of (4 CHI)^2 / 2 threads (the Jacobi layout) per gate; one launch per set of
// gates with disjoint endpoints.  D is the number of bond slots per vertex tensor (3, or 4 for
// degree-4 graphs, where J runs over CHI^3 values); slot k has stride CHI^(D-1-k).
#pragma once

#include "gtqa_anneal.cuh"

namespace gtqa {

struct GenArgs {
    void* Gamma;
    double* lam;
    const int4* edge_info;
    const int4* vert_edges;   // slots of each vertex (x, y, z, and w when D = 4; -1 phantom)
    const int* gate_edge;     // edge of each gate of this launch
    const cd* gate_U;         // [gates][4][4], row 2 i_a + i_b, column 2 i_a' + i_b'
    int count;                // gates in this launch
    double* stats;            // discarded weight, log fidelity, SVD pairs, SVD rotations
    int chi;
    double svd_cut;
};

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int CHI, int D = 3>
struct GenShape {
    static constexpr int NR = ipow(CHI, D - 1);   // rows of A_x
    static constexpr int NC = 2 * CHI;       // columns of A_x: (i, j)
    static constexpr int NM = 4 * CHI;       // order of the core matrix
    static constexpr int G = NR / 2;         // lanes per Householder group (two rows each)
    static constexpr int TEAM = NM * NM / 2; // Jacobi layout: NM/2 pairs x NM rows
};

template <int CHI, int D = 3, typename R = double>
struct GenSm {
    using S = GenShape<CHI, D>;
    C<R> X[2][S::NC][S::NR];   // [side][column (i, j)][row J]; reflectors after the QR
    C<R> vk[2][S::NC];
    R tau[2][S::NC];
    C<R> M[S::NM * S::NM];
    C<R> V[S::NM * S::NM];
    C<R> U[16];
    R w[2][S::NR];
    R lab[CHI];
    R sig[S::NM];
    int perm[S::NM];
    int keep;
    int flag;
    int nrot;
};

template <int CHI, int D, class Mode>
__global__ void __launch_bounds__(GenShape<CHI, D>::TEAM, 1) general_gates_kernel(GenArgs c) {
    using TS = typename Mode::TS;
    using R = typename Mode::RC;   // FP64, or FP32 in the complex64 mode
    using CR = C<R>;
    constexpr bool R64 = sizeof(R) == 8;
    using S = GenShape<CHI, D>;
    constexpr int NR = S::NR, NC = S::NC, NM = S::NM, G = S::G, TEAM = S::TEAM, HV = ipow(CHI, D);
    static_assert(G <= 32, "a Householder group must fit in one warp");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GenSm<CHI, D, R>& sm = *reinterpret_cast<GenSm<CHI, D, R>*>(smem_raw);
    const int g = threadIdx.x;
    if (blockIdx.x >= (unsigned)c.count) return;   // uniform per block
    auto bar = [&]() {
        if constexpr (TEAM <= 32) __syncwarp(group_mask<TEAM>());
        else __syncthreads();
    };
    C<TS>* Gam = (C<TS>*)c.Gamma;
    const int e = c.gate_edge[blockIdx.x];
    const int4 ei = c.edge_info[e];
    const int vtx[2] = {ei.x, ei.y};
    const int slot[2] = {ei.z, ei.w};
    // the D - 1 other slots of each side in ascending order; J = sum_m o_m CHI^(D-2-m)
    int oe[2][D - 1], ost[2][D - 1];
    for (int x = 0; x < 2; ++x) {
        const int4 ve = c.vert_edges[vtx[x]];
        const int es[4] = {ve.x, ve.y, ve.z, D == 4 ? ve.w : -1};
        int m = 0;
        for (int k = 0; k < D; ++k)
            if (k != slot[x]) {
                oe[x][m] = es[k];
                ost[x][m] = ipow(CHI, D - 1 - k);
                ++m;
            }
    }
    auto joff = [&](int x, int J) {   // offset of the other-slot index J inside a vertex tensor
        size_t off = 0;
        for (int m = D - 2; m >= 0; --m) {
            off += (size_t)(J % CHI) * ost[x][m];
            J /= CHI;
        }
        return off;
    };
    for (int t = g; t < 2 * NR; t += TEAM) {
        const int x = t / NR;
        int J = t % NR;
        R w = 1.0;
        for (int m = D - 2; m >= 0; --m) {
            w *= lam_get(c.lam, CHI, oe[x][m], J % CHI);
            J /= CHI;
        }
        sm.w[x][t % NR] = w;
    }
    for (int t = g; t < CHI; t += TEAM) sm.lab[t] = __ldcg(c.lam + (size_t)e * CHI + t);
    for (int t = g; t < 16; t += TEAM) sm.U[t] = ccast<R>(c.gate_U[(size_t)blockIdx.x * 16 + t]);
    bar();
    for (int t = g; t < 2 * NC * NR; t += TEAM) {
        const int x = t / (NC * NR), rem = t % (NC * NR);
        const int col = rem / NR, row = rem % NR;
        const int i = col / CHI, j = col % CHI;
        const size_t off = (size_t)vtx[x] * (2 * HV) + (size_t)i * HV + (size_t)j * ipow(CHI, D - 1 - slot[x]) +
                           joff(x, row);
        sm.X[x][col][row] = sm.w[x][row] * ccast<R>(ldcg(Gam + off));
    }
    bar();

    // ---- Householder QR of A_a and A_b (NR x NC), G lanes per side, two rows per lane ----
    const int l = g % G;
    const int r0 = l, r1 = l + G;
    if (g < 2 * G) {
        const int x = g / G;
        const unsigned gm = group_mask<G>();
        for (int k = 0; k < NC; ++k) {
            CR* Xk = sm.X[x][k];
            const CR z = CR{(R)0, (R)0};
            const CR x0 = (r0 >= k) ? Xk[r0] : z;
            const CR x1 = (r1 >= k) ? Xk[r1] : z;
            const R nrm2 = group_sum<G>(norm2(x0) + norm2(x1), gm);
            const CR xkk = Xk[k];
            const R nrm = nr_sqrt(nrm2);
            const R a2 = norm2(xkk);
            const R ra = a2 > 0.0 ? nr_rsqrt(a2) : 0.0;
            const R axkk = a2 * ra;
            const CR ph = a2 > 0.0 ? CR{xkk.x * ra, xkk.y * ra} : CR{(R)1, (R)0};
            const R tau = nrm > 0.0 ? nr_rcp(nrm * (nrm + axkk)) : 0.0;
            const CR vkk = (axkk + nrm) * ph;
            const CR v0 = (r0 == k) ? vkk : x0;
            const CR v1 = (r1 == k) ? vkk : x1;
            for (int cc = k + 1; cc < NC; ++cc) {
                CR* Xc = sm.X[x][cc];
                const CR y0 = Xc[r0], y1 = Xc[r1];
                CR d = cfmac(v0, y0, cfmac(v1, y1, z));
                d.x = group_sum<G>(d.x, gm);
                d.y = group_sum<G>(d.y, gm);
                const CR td = tau * d;
                if (r0 >= k) Xc[r0] = y0 - v0 * td;
                if (r1 >= k) Xc[r1] = y1 - v1 * td;
            }
            __syncwarp(gm);
            if (r0 == k) Xk[k] = (-nrm) * ph;
            if (r1 == k) Xk[k] = (-nrm) * ph;
            if (l == 0) {
                sm.vk[x][k] = vkk;
                sm.tau[x][k] = tau;
            }
            __syncwarp(gm);
        }
    }
    bar();

    // ---- core matrix M (column-major NM x NM): the gate on the two R factors ----
    for (int t = g; t < NC * NC; t += TEAM) {
        const int r = t % NC, rp = t / NC;
        CR B[2][2];
#pragma unroll
        for (int ia = 0; ia < 2; ++ia)
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                CR acc = CR{(R)0, (R)0};
                for (int j = 0; j < CHI; ++j) {
                    const int ca = ia * CHI + j, cb = ib * CHI + j;
                    if (r <= ca && rp <= cb) acc = cfma(sm.lab[j] * sm.X[0][ca][r], sm.X[1][cb][rp], acc);
                }
                B[ia][ib] = acc;
            }
#pragma unroll
        for (int ia = 0; ia < 2; ++ia)
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                const CR* u = sm.U + (2 * ia + ib) * 4;
                CR acc = u[0] * B[0][0];
                acc = cfma(u[1], B[0][1], acc);
                acc = cfma(u[2], B[1][0], acc);
                acc = cfma(u[3], B[1][1], acc);
                sm.M[(ib * NC + rp) * NM + ia * NC + r] = acc;
            }
    }
    if (g == 0) sm.nrot = 0;
    bar();

    // ---- FP64 one-sided Jacobi SVD of M (FP32 angles, FP64-unitary rotations) ----
    int nrot = 0, sweeps;
    if constexpr (TEAM <= 32) {
        WarpGroup grp{group_mask<TEAM>()};
        sweeps = jacobi_svd<NM, R, WarpGroup, true, R64>(sm.M, sm.V, g, grp, group_mask<NM>(), (R)(R64 ? 1e-15 : 1e-6), 60, true,
                                                               &nrot, (R)(R64 ? 3e-8 : 1e-3));
    } else {
        BlockGroup grp{&sm.flag};
        sweeps = jacobi_svd<NM, R, BlockGroup, true, R64>(sm.M, sm.V, g, grp, group_mask<NM>(), (R)(R64 ? 1e-15 : 1e-6), 60, true,
                                                                &nrot, (R)(R64 ? 3e-8 : 1e-3));
    }
    if (nrot) atomicAdd(&sm.nrot, nrot);
    bar();
    for (int cc = g; cc < NM; cc += TEAM) {
        R s2 = 0.0;
        for (int r = 0; r < NM; ++r) s2 += norm2(sm.M[cc * NM + r]);
        sm.sig[cc] = nr_sqrt(s2);
    }
    bar();
    for (int cc = g; cc < NM; cc += TEAM) sm.perm[desc_rank(sm.sig, NM, cc)] = cc;
    bar();
    if (g == 0) {
        const R smax = sm.sig[sm.perm[0]];
        int cnt = 0;
        R tot = 0.0;
        for (int r = 0; r < NM; ++r) {
            const R s = sm.sig[sm.perm[r]];
            tot += s * s;
            cnt += (s > c.svd_cut * smax) ? 1 : 0;
        }
        int keep = cnt < c.chi ? cnt : c.chi;
        if (keep < 1) keep = 1;
        R kept = 0.0, drop = 0.0;
        for (int r = 0; r < NM; ++r) {
            const R s = sm.sig[sm.perm[r]];
            if (r < keep) kept += s * s; else drop += s * s;
        }
        const R inv = kept > 0.0 ? nr_rsqrt(kept) : 0.0;
        for (int r = 0; r < CHI; ++r) c.lam[(size_t)e * CHI + r] = (r < keep) ? sm.sig[sm.perm[r]] * inv : 0.0;
        const R disc = tot > 0.0 ? drop * nr_rcp(tot) : 0.0;
        atomicAdd(&c.stats[0], disc);
        atomicAdd(&c.stats[1], 2.0 * log1p(-disc));   // Eq. (gate_fidelity)
        atomicAdd(&c.stats[2], (double)sweeps * (NM - 1) * (NM / 2));
        atomicAdd(&c.stats[3], (double)sm.nrot);
        sm.keep = keep;
    }
    bar();
    const int keep = sm.keep;

    // ---- new Gamma: Q_x applied to the kept singular vectors of each (side, physical) block ----
    if (g < 4 * G) {
        const int blk = g / G, x = blk >> 1, i = blk & 1;
        const unsigned gm = group_mask<G>();
        CR E0[CHI], E1[CHI];
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) {
            E0[cc] = CR{(R)0, (R)0};
            E1[cc] = CR{(R)0, (R)0};
            if (cc < keep) {
                const int pc = sm.perm[cc];
                const R is = sm.sig[pc] > 0.0 ? nr_rcp(sm.sig[pc]) : 0.0;
                if (r0 < NC) {
                    const int row = i * NC + r0;
                    E0[cc] = (x == 0) ? is * sm.M[pc * NM + row] : conj(sm.V[pc * NM + row]);
                }
                if (r1 < NC) {
                    const int row = i * NC + r1;
                    E1[cc] = (x == 0) ? is * sm.M[pc * NM + row] : conj(sm.V[pc * NM + row]);
                }
            }
        }
        // H_k = I - tau v v^H applied as I - u u^H with u = sqrt(tau) v, last reflector first
        for (int k = NC - 1; k >= 0; --k) {
            const R st = nr_sqrt(sm.tau[x][k]);
            const CR v0 = st * ((r0 == k) ? sm.vk[x][k] : ((r0 > k) ? sm.X[x][k][r0] : CR{(R)0, (R)0}));
            const CR v1 = st * ((r1 == k) ? sm.vk[x][k] : ((r1 > k) ? sm.X[x][k][r1] : CR{(R)0, (R)0}));
#pragma unroll
            for (int cc = 0; cc < CHI; ++cc) {
                CR d = cfmac(v0, E0[cc], cfmac(v1, E1[cc], CR{(R)0, (R)0}));
                d.x = group_sum<G>(d.x, gm);
                d.y = group_sum<G>(d.y, gm);
                E0[cc] = E0[cc] - v0 * d;
                E1[cc] = E1[cc] - v1 * d;
            }
        }
        const R w0 = sm.w[x][r0], w1 = sm.w[x][r1];
        const R iw0 = w0 > 0.0 ? nr_rcp(w0) : 0.0, iw1 = w1 > 0.0 ? nr_rcp(w1) : 0.0;
        const size_t base = (size_t)vtx[x] * (2 * HV) + (size_t)i * HV;
        const size_t o0 = joff(x, r0), o1 = joff(x, r1);
        const size_t ss = ipow(CHI, D - 1 - slot[x]);
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) {
            Gam[base + cc * ss + o0] = ccast<TS>(iw0 * E0[cc]);
            Gam[base + cc * ss + o1] = ccast<TS>(iw1 * E1[cc]);
        }
    }
}

// One-qubit gates: Gamma~_a[i] = sum_i' W[i][i'] Gamma_a[i'] (Sec. II D); one block per gate,
// all gates of a launch on distinct vertices.
template <int CHI, int D, class Mode>
__global__ void single_gates_kernel(void* Gamma, const int* vertex, const cd* W, int count) {
    using TS = typename Mode::TS;
    constexpr int H = ipow(CHI, D);
    const int q = blockIdx.x;
    if (q >= count) return;
    C<TS>* gm = (C<TS>*)Gamma + (size_t)vertex[q] * 2 * H;
    const cd w00 = W[4 * q], w01 = W[4 * q + 1], w10 = W[4 * q + 2], w11 = W[4 * q + 3];
    for (int r = threadIdx.x; r < H; r += blockDim.x) {
        const cd a0 = ccast<double>(gm[r]), a1 = ccast<double>(gm[H + r]);
        gm[r] = ccast<TS>(cfma(w01, a1, w00 * a0));
        gm[H + r] = ccast<TS>(cfma(w11, a1, w10 * a0));
    }
}

template <int CHI, int D, class Mode>
cudaError_t general_gates_launch_t(const GenArgs& a, cudaStream_t st) {
    constexpr size_t smem = sizeof(GenSm<CHI, D, typename Mode::RC>);
    static bool attr_set = false;   // the attribute is per function; setting it twice is harmless
    if (!attr_set) {
        const cudaError_t e = raise_smem_limit(general_gates_kernel<CHI, D, Mode>, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.count <= 0) return cudaSuccess;
    general_gates_kernel<CHI, D, Mode><<<a.count, GenShape<CHI, D>::TEAM, smem, st>>>(a);
    return cudaGetLastError();
}

template <int CHI, int D, class Mode>
cudaError_t single_gates_launch_t(void* Gamma, const int* vertex, const cd* W, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    single_gates_kernel<CHI, D, Mode><<<count, 64, 0, st>>>(Gamma, vertex, W, count);
    return cudaGetLastError();
}

}  // namespace gtqa
