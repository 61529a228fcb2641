// Persistent annealing kernel: one cooperative launch runs whole GTQA layers.
//
// Phases of one layer (each separated by a bounded grid barrier):
//   gates      for each colour class: simple update + truncation of every edge of
//              that matching (App. E, App. D "Truncation"); the mixing gate
//              exp(-i t_X X) (Sec. II D) is applied to a vertex right after its last
//              gate of the layer, and a leading mixing gate exp(-i t_pre X) (the
//              second-order and reversed first-order product formulas of Sec. V)
//              right before its first gate.
//   bp init    T_a = Gamma_a prod lambda^{1/2} (Eq. (symmetric_gauge)); warm-start
//              messages diag(lambda)/sum(lambda) (Eq. (reconstructed_messages)).
//   bp sweeps  flooding update of every directed message, Eq. (local_consistency),
//              unit-trace normalisation and trace-norm distance (App. B), until
//              dist_b/|E_b| < tol for every instance b or max_iter sweeps.
//   regauge    Vidal gauge finding (App. D): per-edge transforms, then per-vertex
//              application to T.
//
// Layout: Gamma[n][2][CHI][CHI][CHI] (slot k = k-th incident edge, ascending id),
// lambda[m][CHI], messages[2m][CHI][CHI] (2e = m_{u->v}, 2e+1 = m_{v->u}); phantom
// slots (degree < 3) have dimension 1 with lambda = e_0 and message e_0 e_0^T.
//
// Precision modes:
//   FP64   complex128 tensors and messages, FP64 arithmetic throughout.
//   Mixed  complex64 Gamma, T and message corrections; the simple update's QR and
//          SVD, the regauge's eigen/SVD and square roots, and the message
//          normalisation in FP64.  Messages are kept as m = m0 + delta with m0 the
//          warm start (exact, from lambda) and delta in complex64; each sweep
//          contracts only delta in FP32, and the warm-start part F(m0) is contracted
//          once per BP call in FP64.
#pragma once

#include "gtqa_common.cuh"

namespace gtqa {

struct ModeFP64 {
    using TS = double;   // storage of Gamma, T, messages
    using RC = double;   // arithmetic of the SVDs, QRs and gauge roots
    static constexpr bool mixed = false;
};
struct ModeMixed {
    using TS = float;
    using RC = double;
    static constexpr bool mixed = true;
};
// every step in complex64 / FP32 (a reference point for the precision split; plain kernels only)
struct ModeC64 {
    using TS = float;
    using RC = float;
    static constexpr bool mixed = false;
};

enum : unsigned { PH_GATES = 1u, PH_BP = 2u, PH_WARM = 4u, PH_REGAUGE = 8u };

struct Control {
    unsigned long long bar_count;   // grid-barrier arrivals (monotonic), a multiple of the grid between launches
    unsigned long long bar_pk[3];   // the same, one counter per phase kernel (each kernel keeps its grid size)
    int err;
    int cur;                 // message buffer holding the latest messages
    long long sweeps_total;  // sum over BP calls of max-over-instances sweeps
    int last_iters;          // sweeps of the last BP call (max over instances)
    int not_conv;            // instances at max_iter in the last BP call
    double last_dist;        // max over instances of the final dist/|E|
    long long bp_calls;
    long long nc_calls;      // BP calls in which some instance hit max_iter
    long long regauged;      // regauge-policy layers: regauged (BP and gauge finding ran)
    long long reg_skipped;   // and skipped (R at or below the threshold)
    long long exact_passes;  // separate exact-distance passes (bp_exact_pass) run by BP
    int gate_sw_max;         // most FP64 Jacobi sweeps of one gate-core SVD (polish sweeps in the mixed mode)
    int gate_sw32_max;       // mixed mode: most FP32 preconditioning sweeps of one gate-core SVD
    int reg_sw_max;          // the same for the regauge's eigen-decompositions and SVD
    int reg_sw32_max;
};

struct Ctx {
    // graph
    const int4* edge_info;    // u, v, slot in u, slot in v
    const int4* vert_edges;   // edge at slots 0..2 (-1 phantom), degree
    const int* vert_inst;
    const double* J;
    const double* h;
    const int* colour_edges;
    const int* colour_off;    // [ncol + 1]
    const int* last_colour;   // per vertex: colour of its last gate in a layer (-1: none)
    const int* first_colour;  // per vertex: colour of its first gate in a layer (-1: none)
    const int* iso;           // vertices of degree 0
    int n_iso;
    int ncol;
    int n, m, B;
    const int* inst_vbeg;     // [B + 1]
    const int* inst_m;
    // state
    void* Gamma;
    double* lam;
    void* T;
    void* msg[2];
    cf* D0;                   // mixed: warm-start defect F(m0) - tr F(m0) m0, [2m][CHI^2]
    cd* t0;                   // mixed: tr F(m0), [2m]
    cd* X;                    // regauge transforms [m][2][CHI^2]
    double* acc;              // [3][B] per-sweep distance accumulators
    int* inst_done;
    int* inst_iters;
    double* inst_dist;
    double* stats;            // discarded weight, log fidelity, gate SVD pairs and rotations, regauge SVD sweeps
    Control* ctl;
    unsigned long long* bar;  // barrier counter of this launch (null: ctl->bar_count)
    // parameters
    int chi;
    double svd_cut, eig_cut;
    double tol;
    int max_iter;
    unsigned phases;
    int k0, k1, Ksched;       // layers k0..k1 with tau = k/Ksched; Ksched = 0: one layer at (tZ1, tX1)
    int* kdev;                // non-null: one layer, k read from *kdev; the regauge phase stores k + 1
                              // (CUDA-graph replays of one captured layer advance through the anneal)
    double dt, tZ1, tX1;
    double tXpre1;            // Ksched = 0: leading mixing angle of the layer (0: none)
    const double* rgate;      // regauge policy: the residual sum of this layer (null: always regauge)
    double rthr_sum;          // BP and regauge run only if *rgate > rthr_sum
    int nblocks;
    int bar_expect;           // arrivals per grid barrier (= nblocks; larger only in the timeout test)
    long long spin_limit;
};

template <int CHI> __host__ __device__ constexpr int sstride(int k) {
    return k == 0 ? CHI * CHI : (k == 1 ? CHI : 1);
}
__host__ __device__ inline void others_of(int s, int& o0, int& o1) {
    o0 = (s == 0) ? 1 : 0;
    o1 = (s == 2) ? 1 : 2;
}
__device__ __forceinline__ double lam_get(const double* lam, int CHI, int e, int j) {
    return e < 0 ? (j == 0 ? 1.0 : 0.0) : __ldcg(lam + (size_t)e * CHI + j);
}

// Launch shapes of the persistent phase kernels: threads per block and team sizes.  The gate
// team TG (one lane per element pair of the Jacobi SVD of the 2CHI x 2CHI core), the
// regauge-edge team TR and the BP-init team TV are fixed by their algorithms; the block size
// TPB, the BP vertex team TB and the regauge-vertex team TRV come in NSHAPE variants, which
// gtqa_autotune times kernel by kernel.  Variant 0 is the default:
//   CHI <= 4: (TPB, TB, TRV) = (512, 64, 32), (256, 64, 32), (512, 128, 64)
//   CHI  = 8:                  (256, 256, 128), (512, 256, 128), (512, 512, 256)
constexpr int NSHAPE = 3;
template <int CHI, int V = 0> struct Shape {
    static_assert(V >= 0 && V < NSHAPE, "launch-shape variant");
    static constexpr bool BIG = CHI >= 8;
    static constexpr int TPB = V == 0 ? (BIG ? 256 : 512) : (V == 1 ? (BIG ? 512 : 256) : 512);
    static constexpr int TG = 2 * CHI * CHI;                                           // gate team
    static constexpr int TB = V == 2 ? (BIG ? 512 : 128) : (BIG ? 256 : 64);            // BP team (one vertex)
    static constexpr int TR = CHI * CHI;                                               // regauge-edge team
    static constexpr int TV = 32;                                                      // BP-init team (one warp)
    // warps of a block that run the BP init (its per-warp scratch grows as CHI^3)
    static constexpr int NIT = BIG && TPB / 32 > 8 ? 8 : TPB / 32;
    static constexpr int TRV = V == 2 ? (BIG ? 256 : 64) : (BIG ? 128 : 32);           // regauge-vertex team
};

// ===========================================================================
// gates: simple update of one edge (team of 2 CHI^2 threads)
// ===========================================================================
template <int CHI>
struct GateSm {
    cd X[4][CHI][CHI * CHI];   // [block][col][row]: (a,0) (a,1) (b,0) (b,1); reused for staging
    cd vk[4][CHI];
    double tau[4][CHI];        // square roots of the reflector coefficients
    cd M[4 * CHI * CHI];
    cd V[4 * CHI * CHI];
    cd G[4 * CHI * CHI];       // mixed: V^H V, then M V
    cd Vn[4 * CHI * CHI];      // mixed: Newton-Schulz update of V
    cf M32[4 * CHI * CHI];     // mixed: FP32 copy of M for the preconditioning sweeps
    cf V32[4 * CHI * CHI];
    double w[2][CHI * CHI];
    double lab[CHI];
    double sig[2 * CHI];
    double isig[2 * CHI];      // 1 / sig
    cd ph[4];
    int perm[2 * CHI];
    int keep;
    unsigned relmask;          // mixed: columns that decide the polish's stop
    int flag;
    int nrot;
};

template <int CHI, class Mode>
__device__ void gate_edge(const Ctx& c, int e, int tid, int team, GateSm<CHI>& sm, double tZ, double cX, double sX,
                          int colour, bool pre, double cXp, double sXp) {
    using TS = typename Mode::TS;
    constexpr int NM = 2 * CHI, NR = CHI * CHI, G = NR / 2, TEAM = 2 * CHI * CHI;
    C<TS>* Gam = (C<TS>*)c.Gamma;
    const int4 ei = c.edge_info[e];
    const int vtx[2] = {ei.x, ei.y};
    const int slot[2] = {ei.z, ei.w};
    int oe[2][2], os[2][2];
    for (int x = 0; x < 2; ++x) {
        const int4 ve = c.vert_edges[vtx[x]];
        const int es[3] = {ve.x, ve.y, ve.z};
        others_of(slot[x], os[x][0], os[x][1]);
        oe[x][0] = es[os[x][0]];
        oe[x][1] = es[os[x][1]];
    }
    for (int t = tid; t < 2 * NR; t += TEAM) {
        const int x = t / NR, J = t % NR;
        sm.w[x][J] = lam_get(c.lam, CHI, oe[x][0], J / CHI) * lam_get(c.lam, CHI, oe[x][1], J % CHI);
    }
    for (int t = tid; t < CHI; t += TEAM) sm.lab[t] = __ldcg(c.lam + (size_t)e * CHI + t);
    team_bar<TEAM>(team);
    // both physical components of one element per thread, so that the leading mixing
    // gate [[c, -i s], [-i s, c]] can act on a vertex before its first gate of the layer
    for (int t = tid; t < 2 * CHI * NR; t += TEAM) {
        const int x = t / (CHI * NR), rem = t % (CHI * NR);
        const int col = rem / NR, row = rem % NR;
        const size_t off = (size_t)vtx[x] * (2 * CHI * CHI * CHI) + col * sstride<CHI>(slot[x]) +
                           (row / CHI) * sstride<CHI>(os[x][0]) + (row % CHI) * sstride<CHI>(os[x][1]);
        cd g0 = ccast<double>(ldcg(Gam + off));
        cd g1 = ccast<double>(ldcg(Gam + off + CHI * CHI * CHI));
        if (pre && c.first_colour[vtx[x]] == colour) {
            const cd a0 = g0, a1 = g1;
            g0 = cd{cXp * a0.x + sXp * a1.y, cXp * a0.y - sXp * a1.x};
            g1 = cd{sXp * a0.y + cXp * a1.x, -sXp * a0.x + cXp * a1.y};
        }
        sm.X[2 * x][col][row] = sm.w[x][row] * g0;
        sm.X[2 * x + 1][col][row] = sm.w[x][row] * g1;
    }
    team_bar<TEAM>(team);

    // ---- Householder QR of the four CHI^2 x CHI blocks, G threads per block ----
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
        const double nrm = nr_sqrt(nrm2);
        const double a2 = norm2(xkk);
        const double ra = a2 > 0.0 ? nr_rsqrt(a2) : 0.0;
        const double axkk = a2 * ra;
        const cd ph = a2 > 0.0 ? cd{xkk.x * ra, xkk.y * ra} : cd{1.0, 0.0};
        const double stau = nrm > 0.0 ? nr_rsqrt(nrm * (nrm + axkk)) : 0.0;   // sqrt(tau)
        const double tau = stau * stau;
        const cd vkk = (axkk + nrm) * ph;
        const cd v0 = (r0 == k) ? vkk : x0;
        const cd v1 = x1;
        for (int cc = k + 1; cc < CHI; ++cc) {
            cd* Xc = sm.X[blk][cc];
            const cd y0 = Xc[r0], y1 = Xc[r1];
            cd d = cfmac(v0, y0, cfmac(v1, y1, z));
            d.x = group_sum<G>(d.x, gm);
            d.y = group_sum<G>(d.y, gm);
            const cd td = tau * d;
            if (r0 >= k) Xc[r0] = y0 - v0 * td;
            Xc[r1] = y1 - v1 * td;
        }
        __syncwarp(gm);
        if (r0 == k) Xk[k] = (-nrm) * ph;
        if (l == 0) {
            sm.vk[blk][k] = vkk;
            sm.tau[blk][k] = stau;
        }
        __syncwarp(gm);
    }
    team_bar<TEAM>(team);

    // ---- core matrix M (column-major NM x NM); the 4 diagonal gate phases first ----
    if (tid < 4) {
        const int Da = c.vert_edges[vtx[0]].w, Db = c.vert_edges[vtx[1]].w;
        const double ha = c.h[vtx[0]] * nr_rcp((double)Da), hb = c.h[vtx[1]] * nr_rcp((double)Db), Je = c.J[e];
        const double za = 1.0 - 2.0 * (tid >> 1), zb = 1.0 - 2.0 * (tid & 1);
        double sn, cs;
        sincos(-tZ * (Je * za * zb + ha * za + hb * zb), &sn, &cs);
        sm.ph[tid] = cd{cs, sn};
    }
    team_bar<TEAM>(team);
    for (int t = tid; t < NM * NM; t += TEAM) {
        const int col = t / NM, row = t % NM;
        const int ia = row / CHI, r = row % CHI, ib = col / CHI, rp = col % CHI;
        cd acc = cd{0.0, 0.0};
        const int j0 = r > rp ? r : rp;
        for (int j = j0; j < CHI; ++j) acc = cfma(sm.lab[j] * sm.X[ia][j][r], sm.X[2 + ib][j][rp], acc);
        sm.M[t] = sm.ph[2 * ia + ib] * acc;
    }
    if (tid == 0) sm.nrot = 0;
    team_bar<TEAM>(team);
    // rounding-level entries of the core (graded spectra of the early anneal) are zeroed first
    if constexpr (TEAM <= 32) prune_noise<NM>(sm.M, tid, WarpGroup{group_mask<TEAM>()});
    else prune_noise<NM>(sm.M, tid, TeamGroup<TEAM>{team, &sm.flag});

    // ---- SVD of M ----
    // FP64 mode: one-sided Jacobi in FP64 from V = I.
    // Mixed mode: Jacobi sweeps in FP32 on a copy of M give V32; one FP64 Newton-Schulz
    // step V <- V (3I - V^H V)/2 makes it unitary to ~1e-14; the FP64 Jacobi then polishes
    // W = M V (typically two sweeps; the confirming sweep is skipped by the quadratic
    // stop).  The result is an FP64 SVD of M with a fraction of the FP64 instructions.
    int nrot = 0, sweeps, nsteps = 0;
    // FP32 rotation angles with FP64-exact rotations; the confirming sweep is skipped
    // once a sweep's rotations are all below sqrt(tol) (quadratic convergence)
    auto svd64 = [&](bool init_v, double tol, double quad) {
        if constexpr (TEAM <= 32) {
            WarpGroup grp{group_mask<TEAM>()};
            return jacobi_svd<NM, double, WarpGroup, true, true>(sm.M, sm.V, tid, grp, group_mask<NM>(), tol, 60,
                                                                 init_v, &nrot, quad);
        } else {
            TeamGroup<TEAM> grp{team, &sm.flag};
            return jacobi_svd<NM, double, TeamGroup<TEAM>, true, true>(sm.M, sm.V, tid, grp, group_mask<NM>(), tol,
                                                                       60, init_v, &nrot, quad);
        }
    };
    if constexpr (!Mode::mixed) {
        sweeps = svd64(true, 1e-15, 3e-8);
    } else {
        for (int t = tid; t < NM * NM; t += TEAM) sm.M32[t] = ccast<float>(sm.M[t]);
        team_bar<TEAM>(team);
        int sw32;
        if constexpr (TEAM <= 32) {
            WarpGroup grp{group_mask<TEAM>()};
            sw32 = jacobi_svd<NM, float>(sm.M32, sm.V32, tid, grp, group_mask<NM>(), 1e-6f, 40, true, nullptr, 1e-3f);
        } else {
            TeamGroup<TEAM> grp{team, &sm.flag};
            sw32 = jacobi_svd<NM, float>(sm.M32, sm.V32, tid, grp, group_mask<NM>(), 1e-6f, 40, true, nullptr, 1e-3f);
        }
        if (tid == 0) atomicMax(&c.ctl->gate_sw32_max, sw32);
        team_bar<TEAM>(team);
        for (int t = tid; t < NM * NM; t += TEAM) sm.V[t] = ccast<double>(sm.V32[t]);
        team_bar<TEAM>(team);
        // G = V^H V (column-major: G[p][q] at q*NM + p)
        for (int t = tid; t < NM * NM; t += TEAM) {
            const int q = t / NM, p = t % NM;
            cd acc = cd{0.0, 0.0};
            for (int r = 0; r < NM; ++r) acc = cfmac(sm.V[p * NM + r], sm.V[q * NM + r], acc);
            sm.G[t] = acc;
        }
        team_bar<TEAM>(team);
        // Vn = V (1.5 I - 0.5 G)
        for (int t = tid; t < NM * NM; t += TEAM) {
            const int q = t / NM, r = t % NM;
            cd acc = 1.5 * sm.V[q * NM + r];
            for (int p = 0; p < NM; ++p) acc = cfma(-0.5 * sm.V[p * NM + r], sm.G[q * NM + p], acc);
            sm.Vn[t] = acc;
        }
        team_bar<TEAM>(team);
        // W = M Vn into G, then M <- W, V <- Vn
        for (int t = tid; t < NM * NM; t += TEAM) {
            const int q = t / NM, r = t % NM;
            cd acc = cd{0.0, 0.0};
            for (int p = 0; p < NM; ++p) acc = cfma(sm.M[p * NM + r], sm.Vn[q * NM + p], acc);
            sm.G[t] = acc;
        }
        team_bar<TEAM>(team);
        for (int t = tid; t < NM * NM; t += TEAM) {
            sm.M[t] = sm.G[t];
            sm.V[t] = sm.Vn[t];
        }
        team_bar<TEAM>(team);
        if constexpr (TEAM <= 32) {
            WarpGroup grp{group_mask<TEAM>()};
            sweeps = jacobi_polish<NM, decltype(grp), true>(sm.M, sm.V, sm.sig, tid, grp, group_mask<NM>(), 1e-12,
                                                            1e-5, 60, &nrot, c.chi, &sm.relmask, &nsteps);
        } else {
            TeamGroup<TEAM> grp{team, &sm.flag};
            sweeps = jacobi_polish<NM, decltype(grp), true>(sm.M, sm.V, sm.sig, tid, grp, group_mask<NM>(), 1e-12,
                                                            1e-5, 60, &nrot, c.chi, &sm.relmask, &nsteps);
        }
    }
    if (nrot) atomicAdd(&sm.nrot, nrot);
    team_bar<TEAM>(team);
    for (int cc = tid; cc < NM; cc += TEAM) {
        double s2 = 0.0;
        for (int r = 0; r < NM; ++r) s2 += norm2(sm.M[cc * NM + r]);
        const double sv = nr_sqrt(s2);
        sm.sig[cc] = sv;
        sm.isig[cc] = sv > 0.0 ? nr_rcp(sv) : 0.0;
    }
    team_bar<TEAM>(team);
    for (int cc = tid; cc < NM; cc += TEAM) sm.perm[desc_rank(sm.sig, NM, cc)] = cc;
    team_bar<TEAM>(team);
    if (tid < NM) {   // lane r holds the r-th largest singular value
        const unsigned mk = group_mask<NM>();
        const double sv = sm.sig[sm.perm[tid]];
        const double smax = sm.sig[sm.perm[0]];
        const int cnt = __popc(__ballot_sync(mk, sv > c.svd_cut * smax));
        int keep = cnt < c.chi ? cnt : c.chi;
        if (keep < 1) keep = 1;
        const double s2 = sv * sv;
        const double kept = group_sum<NM>(tid < keep ? s2 : 0.0, mk);
        const double drop = group_sum<NM>(tid < keep ? 0.0 : s2, mk);
        const double inv = kept > 0.0 ? nr_rsqrt(kept) : 0.0;
        if (tid < CHI) c.lam[(size_t)e * CHI + tid] = (tid < keep) ? sv * inv : 0.0;
        if (tid == 0) {
            const double tot = kept + drop;
            const double disc = tot > 0.0 ? drop * nr_rcp(tot) : 0.0;
            atomicAdd(&c.stats[0], disc);
            // log of the gate fidelity (1 - disc)^2, Eq. (gate_fidelity); a float log in the mixed mode
            atomicAdd(&c.stats[1], Mode::mixed ? 2.0 * (double)log1pf(-(float)disc) : 2.0 * log1p(-disc));
            // Jacobi pairs examined (the mixed polish runs partial sweeps)
            atomicAdd(&c.stats[2], (double)(Mode::mixed ? nsteps : sweeps * (NM - 1)) * (NM / 2));
            atomicAdd(&c.stats[3], (double)sm.nrot);
            atomicMax(&c.ctl->gate_sw_max, sweeps);
            sm.keep = keep;
        }
    }
    team_bar<TEAM>(team);
    const int keep = sm.keep;

    // ---- new Gamma: reflectors of each block applied to U (side a) / V^* (side b) ----
    // FP64 mode in double, mixed mode in float (the result is stored in complex64).
    using RB = typename Mode::TS;
    C<RB> E0[CHI], E1[CHI];
    const int x = blk >> 1, i = blk & 1;
#pragma unroll
    for (int cc = 0; cc < CHI; ++cc) {
        E0[cc] = C<RB>{(RB)0, (RB)0};
        E1[cc] = C<RB>{(RB)0, (RB)0};
        if (r0 < CHI && cc < keep) {
            const int pc = sm.perm[cc];
            const int row = i * CHI + r0;
            const cd u = (x == 0) ? sm.isig[pc] * sm.M[pc * NM + row] : conj(sm.V[pc * NM + row]);
            E0[cc] = ccast<RB>(u);
        }
    }
    // H_k = I - tau v v^H is applied as I - u u^H with u = sqrt(tau) v (|u| = sqrt 2), so
    // neither factor over- or underflows when the reflector is tiny (matters in float).
    for (int k = CHI - 1; k >= 0; --k) {
        const double st = sm.tau[blk][k];
        const C<RB> v0 = ccast<RB>(st * ((r0 == k) ? sm.vk[blk][k] : ((r0 > k) ? sm.X[blk][k][r0] : cd{0.0, 0.0})));
        const C<RB> v1 = ccast<RB>(st * sm.X[blk][k][r1]);
#pragma unroll
        for (int cc = 0; cc < CHI; ++cc) {
            C<RB> d = cfmac(v0, E0[cc], cfmac(v1, E1[cc], C<RB>{(RB)0, (RB)0}));
            d.x = group_sum<G>(d.x, gm);
            d.y = group_sum<G>(d.y, gm);
            E0[cc] = E0[cc] - v0 * d;
            E1[cc] = E1[cc] - v1 * d;
        }
    }
    const double w0 = sm.w[x][r0], w1 = sm.w[x][r1];
    const RB iw0 = w0 > 0.0 ? (RB)nr_rcp(w0) : (RB)0, iw1 = w1 > 0.0 ? (RB)nr_rcp(w1) : (RB)0;
    team_bar<TEAM>(team);   // everyone is done reading the reflectors in sm.X
    // stage Gamma~ (rounded to storage) in sm.X as [x*2+i][col][row]
#pragma unroll
    for (int cc = 0; cc < CHI; ++cc) {
        sm.X[blk][cc][r0] = ccast<double>(ccast<TS>(iw0 * E0[cc]));
        sm.X[blk][cc][r1] = ccast<double>(ccast<TS>(iw1 * E1[cc]));
    }
    team_bar<TEAM>(team);
    // write back, applying the mixing gate to a vertex after its last gate of the layer
    for (int t = tid; t < 2 * CHI * NR; t += TEAM) {
        const int xx = t / (CHI * NR), rem = t % (CHI * NR);
        const int col = rem / NR, row = rem % NR;
        C<TS> g0 = ccast<TS>(sm.X[2 * xx][col][row]);
        C<TS> g1 = ccast<TS>(sm.X[2 * xx + 1][col][row]);
        if (c.last_colour[vtx[xx]] == colour) {
            const C<TS> a0 = g0, a1 = g1;
            const TS cs = (TS)cX, sn = (TS)sX;
            // [[c, -i s], [-i s, c]]
            g0 = C<TS>{cs * a0.x + sn * a1.y, cs * a0.y - sn * a1.x};
            g1 = C<TS>{sn * a0.y + cs * a1.x, -sn * a0.x + cs * a1.y};
        }
        const size_t base = (size_t)vtx[xx] * (2 * CHI * CHI * CHI);
        const size_t off = col * sstride<CHI>(slot[xx]) + (row / CHI) * sstride<CHI>(os[xx][0]) +
                           (row % CHI) * sstride<CHI>(os[xx][1]);
        Gam[base + off] = g0;
        Gam[base + CHI * CHI * CHI + off] = g1;
    }
}

// mixing gate on one vertex (used for degree-0 vertices only)
template <int CHI, class Mode>
__device__ void mixing_vertex(const Ctx& c, int a, int tid, int TEAM, double cX, double sX) {
    using TS = typename Mode::TS;
    constexpr int H = CHI * CHI * CHI;
    C<TS>* g = (C<TS>*)c.Gamma + (size_t)a * 2 * H;
    for (int r = tid; r < H; r += TEAM) {
        const C<TS> a0 = ldcg(g + r), a1 = ldcg(g + H + r);
        const TS cs = (TS)cX, sn = (TS)sX;
        g[r] = C<TS>{cs * a0.x + sn * a1.y, cs * a0.y - sn * a1.x};
        g[H + r] = C<TS>{sn * a0.y + cs * a1.x, -sn * a0.x + cs * a1.y};
    }
}

// ===========================================================================
// BP init (one warp per vertex): symmetric split, warm start, and in the mixed mode
// the FP64 contraction of the warm start F0 = F(m0, m0), kept as its trace t0 and
// the defect D0 = F0 - t0 m0 (complex64; |D0| is of the order of the corrections).
// ===========================================================================
template <int CHI, class Mode>
__device__ void bp_init_vertex(const Ctx& c, int a, int tid, int cur, bool warm, double* wsm, cd* tsm) {
    using TS = typename Mode::TS;
    constexpr int H = CHI * CHI * CHI, CC = CHI * CHI, TEAM = Shape<CHI>::TV;
    const int4 ve = c.vert_edges[a];
    const int es[3] = {ve.x, ve.y, ve.z};
    // wsm[0 .. 3CHI): lambda^{1/2} per slot; wsm[3CHI .. 6CHI): m0 diagonal per slot;
    // wsm[6CHI .. 6CHI + 3): (sum lambda)^{-1/2} per slot
    if (tid < 3 * CHI) {
        const int k = tid / CHI, j = tid % CHI;
        const double lj = lam_get(c.lam, CHI, es[k], j);
        wsm[tid] = nr_sqrt(lj);
        double s = 0.0;
        for (int q = 0; q < CHI; ++q) s += lam_get(c.lam, CHI, es[k], q);
        wsm[3 * CHI + tid] = s > 0.0 ? lj * nr_rcp(s) : 0.0;
        if (j == 0) wsm[6 * CHI + k] = s > 0.0 ? nr_rsqrt(s) : 0.0;
    }
    __syncwarp();
    const C<TS>* g = (const C<TS>*)c.Gamma + (size_t)a * 2 * H;
    C<TS>* T = (C<TS>*)c.T + (size_t)a * 2 * H;
    // mixed: tsm holds T~ = T prod_k m0_k[j_k]^{1/2} (T as stored, in FP64), so that the warm
    // start's contraction below needs no weights in its inner loop
    const double iso = Mode::mixed ? wsm[6 * CHI] * wsm[6 * CHI + 1] * wsm[6 * CHI + 2] : 0.0;
    for (int t = tid; t < 2 * H; t += TEAM) {
        const int r = t % H;
        const int j0 = r / CC, j1 = (r / CHI) % CHI, j2 = r % CHI;
        const double f = wsm[j0] * wsm[CHI + j1] * wsm[2 * CHI + j2];
        const C<TS> tv = ccast<TS>(f * ccast<double>(ldcg(g + t)));
        T[t] = tv;
        if constexpr (Mode::mixed) tsm[t] = (f * iso) * ccast<double>(tv);
    }
    int out[3];
    for (int s = 0; s < 3; ++s) out[s] = es[s] >= 0 ? 2 * es[s] + (a == c.edge_info[es[s]].x ? 0 : 1) : -1;
    if (warm) {
        for (int t = tid; t < 3 * CC; t += TEAM) {
            const int s = t / CC, r = t % CC;
            if (out[s] < 0) continue;
            const int j = r / CHI, jp = r % CHI;
            if constexpr (!Mode::mixed) ((cd*)c.msg[cur])[(size_t)out[s] * CC + r] = cd{j == jp ? wsm[3 * CHI + s * CHI + j] : 0.0, 0.0};
            else ((cf*)c.msg[cur])[(size_t)out[s] * CC + r] = cf{0.f, 0.f};
        }
    }
    if constexpr (Mode::mixed) {
        __syncwarp();
        // upper triangle (j <= j') of F0 for the 3 outgoing slots, items spread over the warp:
        //   F0_s[j][j'] = sum_{i,p,q} m0_o0[p] m0_o1[q] T[.., j@s, ..] conj(T[.., j'@s, ..])
        //              = (sum T~[.., j@s, ..] conj(T~[.., j'@s, ..])) / (m0_s[j] m0_s[j'])^{1/2},
        // and 0 where m0_s[j] or m0_s[j'] vanishes (T vanishes there too)
        constexpr int NU = CHI * (CHI + 1) / 2;
        cd* F = tsm + 2 * H;   // [3][CC]
        for (int item = tid; item < 3 * NU; item += TEAM) {
            const int s = item / NU;
            int u = item % NU, j = 0;
            while (u >= CHI - j) { u -= CHI - j; ++j; }
            const int jp = j + u;
            if (out[s] < 0) continue;
            int o0, o1;
            others_of(s, o0, o1);
            const int ss = sstride<CHI>(s), s0 = sstride<CHI>(o0), s1 = sstride<CHI>(o1);
            cd f = cd{0.0, 0.0};
            for (int p = 0; p < CHI; ++p) {
                if (wsm[o0 * CHI + p] == 0.0) continue;
                for (int q = 0; q < CHI; ++q) {
                    if (wsm[o1 * CHI + q] == 0.0) continue;
                    for (int ii = 0; ii < 2; ++ii) {
                        const int base = ii * H + p * s0 + q * s1;
                        f = cfmac(tsm[base + jp * ss], tsm[base + j * ss], f);
                    }
                }
            }
            const double d = wsm[3 * CHI + s * CHI + j] * wsm[3 * CHI + s * CHI + jp];
            f = d > 0.0 ? nr_rsqrt(d) * f : cd{0.0, 0.0};
            F[s * CC + j * CHI + jp] = f;
            if (jp != j) F[s * CC + jp * CHI + j] = conj(f);
        }
        __syncwarp();
        for (int t = tid; t < 3 * CC; t += TEAM) {
            const int s = t / CC, r = t % CC;
            if (out[s] < 0) continue;
            const int j = r / CHI, jp = r % CHI;
            double t0 = 0.0;
            for (int q = 0; q < CHI; ++q) t0 += F[s * CC + q * CHI + q].x;
            const double m0 = (j == jp) ? wsm[3 * CHI + s * CHI + j] : 0.0;
            c.D0[(size_t)out[s] * CC + r] = ccast<float>(F[s * CC + r] - cd{t0 * m0, 0.0});
            if (r == 0) c.t0[out[s]] = cd{t0, 0.0};
        }
    }
}

// ===========================================================================
// BP sweep for one vertex: all three outgoing messages at once (team TB).
//
// With T in its natural layout [i][j0][j1][j2] the message out of slot s is
//   F_s[j][j'] = sum T[..j@s..] conj(T[..j'@s..]) x (m_o0 (x) m_o1),        Eq. (local_consistency)
// computed as: first contractions along single slots (shared between the outgoing
// slots), second contractions per slot (Q_s), then the overlap with conj(T).  In the
// mixed mode the incoming messages are m = m0 + delta and only the delta terms are
// contracted (FP32): F_s - F_s(m0) = T x_{o0} delta x_{o1} m + m0_{o0} T x_{o1} delta.
// The per-vertex inputs that do not change during a BP run (T, the warm-start
// diagonals, D0, t0, this vertex's previous outgoing messages) are cached in the
// team's shared memory across sweeps.
// ===========================================================================
template <int CHI, class Mode, int TB>
struct BPSm {
    using TS = typename Mode::TS;
    static constexpr int H2 = 2 * CHI * CHI * CHI, CC = CHI * CHI, NP = Mode::mixed ? 3 : 2;
    // lanes that share one 2 x 2 block of an outgoing message, each summing a slice of the
    // 2 CHI^2 columns: the largest power of two (at most 32 and 2 CHI^2) that keeps all
    // 3 (CHI/2)^2 blocks of the three slots within the team
    static constexpr int fslices() {
        int ns = 1;
        while (2 * ns <= 32 && 2 * ns <= 2 * CC && 3 * (CHI / 2) * (CHI / 2) * 2 * ns <= TB) ns *= 2;
        return ns;
    }
    static constexpr int NS = fslices();
    // FP64 mode: the overlap stage keeps every lane busy instead (FP64 instructions cost per
    // warp, so the fewer per lane the better): NPART lanes per (j, j') split the (i, u) sum
    // and meet by shuffles, or, where that does not divide, the sum in two halves over the
    // physical index i, added at use
    static constexpr int NPART = TB / CC;
    static constexpr bool HALVES = !(TB % CC == 0 && NPART <= 32 && (2 * CHI) % NPART == 0);
    static_assert(CHI % 2 == 0 && 3 * (CHI / 2) * (CHI / 2) * NS <= TB, "BP team too small for the overlap stage");
    // T, P and Q in the natural index order [i][j0][j1][j2] with one padding element after
    // every (i, j0) plane, so that a stride along slot 0 does not map to one bank
    static constexpr int PS = CC + 1, H2P = 2 * CHI * PS;
    C<TS> T[H2P];
    C<TS> P[NP][H2P];    // FP64: T x0 m0, T x1 m1; mixed: T x0 d0, T x1 d1, T x2 d2
    C<TS> Q[3][H2P];     // per outgoing slot
    C<TS> min[3][CC];    // incoming messages (mixed: m0 + delta)
    C<TS> din[3][CC];    // mixed: incoming delta
    C<TS> F[3][CC];      // the outgoing messages before normalisation
    C<TS> F1[Mode::mixed ? 1 : 3][CC];   // FP64 mode with HALVES: the i = 1 half
    C<TS> prev[3][CC];   // outgoing messages of the previous sweep
    C<TS> D[3][CC];      // new - old, for the trace norm
    cf D0f[3][CC];       // mixed: warm-start defect
    float m0f[3][CHI];   // mixed: warm-start diagonals
    cd t0[3];            // mixed: traces of F0
    C<TS> trs[3];        // traces of the outgoing messages (mixed: of the correction terms)
    C<TS> itr[3];        // 1 / trace, formed in FP64
    TS dl[3];
    TS dsum[3];          // one instance: the team's distance summed over the rounds of a sweep
    int es[3], out_idx[3], in_idx[3];
    int cached;          // vertex held in the cache, -1 if none
};

template <int CHI, class Mode, int TB>
__device__ void bp_prepare(const Ctx& c, int a, int tid, int team, int cur, BPSm<CHI, Mode, TB>& sm) {
    using TS = typename Mode::TS;
    using CT = C<TS>;
    constexpr int TEAM = TB, CC = CHI * CHI, H2 = 2 * CHI * CHI * CHI;
    team_bar<TEAM>(team);   // the team may still be reading the previous vertex's cache
    if (tid < 3) {
        const int4 ve = c.vert_edges[a];
        const int e = tid == 0 ? ve.x : (tid == 1 ? ve.y : ve.z);
        sm.es[tid] = e;
        if (e >= 0) {
            const int u = c.edge_info[e].x;
            sm.out_idx[tid] = 2 * e + (a == u ? 0 : 1);
            sm.in_idx[tid] = 2 * e + (a == u ? 1 : 0);
        } else {
            sm.out_idx[tid] = sm.in_idx[tid] = -1;
        }
    }
    const CT* Tg = (const CT*)c.T + (size_t)a * H2;
    for (int t = tid; t < H2; t += TEAM) sm.T[t + t / CC] = ldcg(Tg + t);
    team_bar<TEAM>(team);
    const CT* src = (const CT*)c.msg[cur];
    for (int t = tid; t < 3 * CC; t += TEAM) {
        const int k = t / CC, r = t % CC;
        const int out = sm.out_idx[k];
        sm.prev[k][r] = out >= 0 ? ldcg(src + (size_t)out * CC + r) : CT{(TS)0, (TS)0};
    }
    if constexpr (Mode::mixed) {
        if (tid < 3 * CHI) {
            const int k = tid / CHI, j = tid % CHI;
            double s = 0.0;
            for (int q = 0; q < CHI; ++q) s += lam_get(c.lam, CHI, sm.es[k], q);
            sm.m0f[k][j] = s > 0.0 ? (float)(lam_get(c.lam, CHI, sm.es[k], j) * nr_rcp(s)) : 0.f;
        }
        for (int t = tid; t < 3 * CC; t += TEAM) {
            const int k = t / CC, r = t % CC;
            sm.D0f[k][r] = sm.out_idx[k] >= 0 ? ldcg(c.D0 + (size_t)sm.out_idx[k] * CC + r) : cf{0.f, 0.f};
        }
        if (tid < 3) sm.t0[tid] = sm.out_idx[tid] >= 0 ? ldcg(c.t0 + sm.out_idx[tid]) : cd{1.0, 0.0};
    }
    if (tid == 0) sm.cached = a;
    team_bar<TEAM>(team);
}

// First part of the sweep for vertex a: incoming messages, the contractions, and the
// traces of the three outgoing messages (left in sm.trs).
template <int CHI, class Mode, int TB>
__device__ void bp_front(const Ctx& c, int a, int tid, int team, int cur, BPSm<CHI, Mode, TB>& sm, bool have_pre,
                         C<typename Mode::TS> pre) {
    using TS = typename Mode::TS;
    using CT = C<TS>;
    using SM = BPSm<CHI, Mode, TB>;
    constexpr int TEAM = TB, CC = CHI * CHI, H = CHI * CHI * CHI, H2 = 2 * H;
    // strides in the padded shared-memory layout: slot 0, slot 1 (slot 2 has stride 1), i
    constexpr int S0 = SM::PS, S1 = CHI, HP = CHI * SM::PS;
    if (sm.cached != a) bp_prepare<CHI, Mode, TB>(c, a, tid, team, cur, sm);
    const CT* src = (const CT*)c.msg[cur];
    const CT z = CT{(TS)0, (TS)0};
    // incoming messages (prefetched into `pre` by the caller when have_pre)
    for (int t = tid; t < 3 * CC; t += TEAM) {
        const int k = t / CC, r = t % CC;
        const int in = sm.in_idx[k];
        const CT lv = in >= 0 ? (have_pre ? pre : ldcg(src + (size_t)in * CC + r)) : z;
        if constexpr (!Mode::mixed) {
            sm.min[k][r] = in >= 0 ? lv : CT{(TS)(r == 0 ? 1 : 0), (TS)0};
        } else {
            const int j = r / CHI, jp = r % CHI;
            const CT dv = lv;
            sm.din[k][r] = dv;
            sm.min[k][r] = CT{dv.x + ((j == jp) ? sm.m0f[k][j] : 0.f), dv.y};
        }
    }
    team_bar<TEAM>(team);
    // first contractions along one slot: P_k[.., x@k, ..] = sum_q T[.., q@k, ..] y_k[q][x]
    //   FP64: y = m (k = 0, 1); mixed: y = delta (k = 0, 1, 2)
    constexpr int NP = SM::NP;
    constexpr bool EVEN = H2 % TEAM == 0;   // whole tensors per team pass: slots fixed at compile time
    auto slot_stride = [](int k) { return k == 0 ? S0 : (k == 1 ? S1 : 1); };
    // e: natural index of an element, pe: its padded position
    auto p_elem = [&](int k, int e) {
        const int pe = e + e / CC;
        const int st = slot_stride(k);
        const int x = k == 0 ? (e / CC) % CHI : (k == 1 ? (e / CHI) % CHI : e % CHI);
        const int base = pe - x * st;
        const CT* y = Mode::mixed ? sm.din[k] : sm.min[k];
        CT acc = z;
#pragma unroll
        for (int q = 0; q < CHI; ++q) acc = cfma(sm.T[base + q * st], y[q * CHI + x], acc);
        sm.P[k][pe] = acc;
    };
    if constexpr (EVEN) {
#pragma unroll
        for (int k = 0; k < NP; ++k)
#pragma unroll
            for (int w = 0; w < H2 / TEAM; ++w) p_elem(k, tid + w * TEAM);
    } else {
        for (int t = tid; t < NP * H2; t += TEAM) p_elem(t / H2, t % H2);
    }
    team_bar<TEAM>(team);
    // second contractions per outgoing slot s (natural layout, slot-s index = j):
    //   Q_0[i][j][a][b] = sum_q P_1[i][j][a][q] m_2[q][b]  (+ m0_1[a] P_2[i][j][a][b])
    //   Q_1[i][a][j][b] = sum_q P_0[i][a][j][q] m_2[q][b]  (+ m0_0[a] P_2[i][a][j][b])
    //   Q_2[i][a][b][j] = sum_q P_0[i][a][q][j] m_1[q][b]  (+ m0_0[a] P_1[i][a][b][j])
    auto q_elem = [&](int s, int e) {
        const int pe = e + e / CC;
        const int j0 = (e / CC) % CHI, j1 = (e / CHI) % CHI, j2 = e % CHI;
        CT acc = z;
        if (s == 2) {
#pragma unroll
            for (int q = 0; q < CHI; ++q) acc = cfma(sm.P[0][pe - j1 * S1 + q * S1], sm.min[1][q * CHI + j1], acc);
        } else {
            const CT* Ps = (s == 0) ? sm.P[1] : sm.P[0];
#pragma unroll
            for (int q = 0; q < CHI; ++q) acc = cfma(Ps[pe - j2 + q], sm.min[2][q * CHI + j2], acc);
        }
        if constexpr (Mode::mixed) {
            const float w = (s == 0) ? sm.m0f[1][j1] : sm.m0f[0][j0];
            const CT pv = (s == 2) ? sm.P[1][pe] : sm.P[2][pe];
            acc = acc + w * pv;
        }
        sm.Q[s][pe] = acc;
    };
    if constexpr (EVEN) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (sm.es[s] < 0) continue;
#pragma unroll
            for (int w = 0; w < H2 / TEAM; ++w) q_elem(s, tid + w * TEAM);
        }
    } else {
        for (int t = tid; t < 3 * H2; t += TEAM) {
            const int s = t / H2;
            if (sm.es[s] >= 0) q_elem(s, t % H2);
        }
    }
    team_bar<TEAM>(team);
    // overlaps with conj(T): F_s[j][j'] = sum over the 2 CHI^2 columns (i, u@o0, v@o1) of
    // Q_s[.., j@s, ..] conj(T[.., j'@s, ..]).  Mixed mode: a lane holds a 2 x 2 block of
    // (j, j') over a slice of the columns, so that every element it loads feeds two products;
    // the NS lanes of a block then sum by shuffles.
    if constexpr (Mode::mixed) {
        constexpr int NBJ = CHI / 2, NB = NBJ * NBJ, K = 2 * CC, NS = SM::NS, CPL = K / NS;
        if (tid < 3 * NB * NS) {
            const int s = tid / (NB * NS), rem = tid % (NB * NS);
            const int b = rem / NS, slice = rem % NS;
            const int j0 = 2 * (b / NBJ), jp0 = 2 * (b % NBJ);
            if (sm.es[s] >= 0) {   // the same for the NS lanes of a block
                const int ss = slot_stride(s);
                const int so = s == 0 ? S1 : S0, st2 = s == 2 ? S1 : 1;   // strides of the two other slots
                const CT* Qs = sm.Q[s];
                CT a00 = z, a01 = z, a10 = z, a11 = z;
#pragma unroll
                for (int w = 0; w < CPL; ++w) {
                    const int cl = slice * CPL + w;
                    const int off = (cl / CC) * HP + ((cl / CHI) % CHI) * so + (cl % CHI) * st2;
                    const CT q0 = Qs[off + j0 * ss], q1 = Qs[off + (j0 + 1) * ss];
                    const CT t0 = sm.T[off + jp0 * ss], t1 = sm.T[off + (jp0 + 1) * ss];
                    a00 = cfmac(t0, q0, a00);
                    a01 = cfmac(t1, q0, a01);
                    a10 = cfmac(t0, q1, a10);
                    a11 = cfmac(t1, q1, a11);
                }
                const unsigned gm = group_mask<NS>();
                a00.x = group_sum<NS>(a00.x, gm);
                a00.y = group_sum<NS>(a00.y, gm);
                a01.x = group_sum<NS>(a01.x, gm);
                a01.y = group_sum<NS>(a01.y, gm);
                a10.x = group_sum<NS>(a10.x, gm);
                a10.y = group_sum<NS>(a10.y, gm);
                a11.x = group_sum<NS>(a11.x, gm);
                a11.y = group_sum<NS>(a11.y, gm);
                if (slice == 0) {
                    sm.F[s][j0 * CHI + jp0] = a00;
                    sm.F[s][j0 * CHI + jp0 + 1] = a01;
                    sm.F[s][(j0 + 1) * CHI + jp0] = a10;
                    sm.F[s][(j0 + 1) * CHI + jp0 + 1] = a11;
                }
            }
        }
    } else if constexpr (SM::HALVES) {
        for (int t = tid; t < 2 * 3 * CC; t += TEAM) {
            const int i = t / (3 * CC), rem = t % (3 * CC);
            const int s = rem / CC, r = rem % CC;
            if (sm.es[s] < 0) continue;
            const int j = r / CHI, jp = r % CHI;
            const int ss = slot_stride(s);
            const int so = s == 0 ? S1 : S0, st2 = s == 2 ? S1 : 1;   // strides of the two other slots
            CT acc = z;
#pragma unroll
            for (int u = 0; u < CHI; ++u)
#pragma unroll
                for (int v = 0; v < CHI; ++v) {
                    const int off = i * HP + u * so + v * st2;
                    acc = cfmac(sm.T[off + jp * ss], sm.Q[s][off + j * ss], acc);
                }
            if (i == 0) sm.F[s][r] = acc;
            else sm.F1[s][r] = acc;
        }
    } else {
        constexpr int NPART = SM::NPART, PER = 2 * CHI / NPART;
        const int r = tid / NPART, part = tid % NPART;
        const int j = r / CHI, jp = r % CHI;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (sm.es[s] < 0) continue;
            const int ss = slot_stride(s);
            const int so = s == 0 ? S1 : S0, st2 = s == 2 ? S1 : 1;
            CT acc = z;
#pragma unroll
            for (int h = 0; h < PER; ++h) {
                const int cmb = part * PER + h, i = cmb / CHI, u = cmb % CHI;
#pragma unroll
                for (int v = 0; v < CHI; ++v) {
                    const int off = i * HP + u * so + v * st2;
                    acc = cfmac(sm.T[off + jp * ss], sm.Q[s][off + j * ss], acc);
                }
            }
            acc.x = group_sum<NPART>(acc.x, group_mask<NPART>());
            acc.y = group_sum<NPART>(acc.y, group_mask<NPART>());
            if (part == 0) sm.F[s][r] = acc;
        }
    }
    team_bar<TEAM>(team);
    // traces of the outgoing messages (their reciprocals follow in FP64, bp_trace_rcp)
    if (tid < 3 * CC && tid % CC == 0) {
        const int k = tid / CC;
        CT trs = z;
#pragma unroll
        for (int j = 0; j < CHI; ++j) {
            trs = trs + sm.F[k][j * CHI + j];
            if constexpr (!Mode::mixed && SM::HALVES) trs = trs + sm.F1[k][j * CHI + j];
        }
        sm.trs[k] = trs;
    }
}

// Reciprocals of the complex traces of every team's outgoing messages in FP64 (reading
// R10: messages are divided by their complex trace), one lane per message, by the first
// warp of the block: FP64 instructions cost the same for 1 or 32 active lanes, so one
// warp does this for all teams.  Mixed: the trace is t0 + tr Fd.
template <int CHI, class Mode, int TB>
__device__ void bp_trace_rcp(BPSm<CHI, Mode, TB>* all, int nteams) {
    using TS = typename Mode::TS;
    for (int l = threadIdx.x; l < 3 * nteams; l += 32) {
        BPSm<CHI, Mode, TB>& sm = all[l / 3];
        const int k = l % 3;
        cd tr = ccast<double>(sm.trs[k]);
        if constexpr (Mode::mixed) tr = tr + sm.t0[k];
        const double n2 = norm2(tr);
        // the mixed mode rounds the result to FP32, so one Newton step (relative error ~2^-44) suffices
        const double in2 = n2 > 0.0 ? (Mode::mixed ? nr_rcp1(n2) : nr_rcp(n2)) : 0.0;
        sm.itr[k] = ccast<TS>(cd{tr.x * in2, -tr.y * in2});
    }
}

// Second part: new messages m' = F / tr F (mixed: delta' = (D0 + Fd - m0 tr Fd) / (t0 + tr Fd))
// and the distance of App. B, added to *dacc.
template <int CHI, class Mode, int TB>
__device__ void bp_back(const Ctx& c, int tid, int team, int cur, bool exact, BPSm<CHI, Mode, TB>& sm,
                        double* gacc) {
    using TS = typename Mode::TS;
    using CT = C<TS>;
    constexpr int TEAM = TB, CC = CHI * CHI;
    CT* dst = (CT*)c.msg[cur ^ 1];
    const CT z = CT{(TS)0, (TS)0};
    constexpr int GJ = CC / 2;
    constexpr bool FAST = CC <= 32;   // the elements of one message lie in one warp
    static_assert(3 * GJ <= TEAM && 3 * CHI <= 32 && 3 * CC <= TEAM, "BP team too small");
    TS f2 = (TS)0;
    if (tid < 3 * CC) {
        const int k = tid / CC, r = tid % CC;
        const int out = sm.out_idx[k];
        CT d = z;
        if (out >= 0) {
            const CT itr = sm.itr[k];
            CT f = sm.F[k][r];
            if constexpr (!Mode::mixed && BPSm<CHI, Mode, TB>::HALVES) f = f + sm.F1[k][r];
            CT num = f;
            if constexpr (Mode::mixed) {
                const int j = r / CHI, jp = r % CHI;
                num = sm.D0f[k][r] + f;
                if (j == jp) num = num - sm.m0f[k][j] * sm.trs[k];
            }
            const CT nv = itr * num;
            dst[(size_t)out * CC + r] = nv;
            d = nv - sm.prev[k][r];
            sm.prev[k][r] = nv;
        }
        if (FAST && !exact) f2 = norm2(d);
        else sm.D[k][r] = d;
    }
    // distance of App. B: trace norms ||m_new - m_old||_1 (sum of singular values) when
    // `exact`, else the Frobenius norms, a lower bound that suffices to continue
    if constexpr (FAST) {
        if (!exact) {
            if (tid < 3 * CC) {
                f2 = group_sum<CC>(f2, group_mask<CC>());
                if (tid % CC == 0) {
                    const TS f = sm.out_idx[tid / CC] >= 0 ? nr_sqrt(f2) : (TS)0;
                    if (gacc) atomicAdd(gacc, (double)f);
                    else sm.dsum[tid / CC] += f;
                }
            }
            return;
        }
    }
    team_bar<TEAM>(team);
    if (!exact) {
        if (tid < 32) {
            TS c2 = (TS)0;
            if (tid < 3 * CHI) {
                const int k = tid / CHI, cc = tid % CHI;
#pragma unroll
                for (int r = 0; r < CHI; ++r) c2 += norm2(sm.D[k][cc * CHI + r]);
            }
#pragma unroll
            for (int o = 1; o < CHI; o <<= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
            if (tid < 3 * CHI && tid % CHI == 0) sm.dl[tid / CHI] = nr_sqrt(c2);
        }
    } else if (tid < 3 * GJ) {
        const int k = tid / GJ, g = tid % GJ;
        WarpGroup grp{group_mask<GJ>()};
        jacobi_svd<CHI, TS, WarpGroup, false, !Mode::mixed>(sm.D[k], nullptr, g, grp, group_mask<CHI>(),
                                                             Mode::mixed ? (TS)1e-6 : (TS)1e-15, 60, false, nullptr,
                                                             Mode::mixed ? (TS)1e-3 : (TS)3e-8);
        if (g == 0) {
            TS sacc = (TS)0;
            for (int cc = 0; cc < CHI; ++cc) {
                TS n2 = (TS)0;
                for (int r = 0; r < CHI; ++r) n2 += norm2(sm.D[k][cc * CHI + r]);
                sacc += nr_sqrt(n2);
            }
            sm.dl[k] = sacc;
        }
    }
    team_bar<TEAM>(team);
    if (gacc) {
        if (tid == 0) atomicAdd(gacc, (double)sm.dl[0] + (double)sm.dl[1] + (double)sm.dl[2]);
    } else if (tid < 3) {
        sm.dsum[tid] += sm.dl[tid];
    }
}

// copy a frozen instance's outgoing messages to the other buffer
template <int CHI, class Mode>
__device__ void bp_copy_vertex(const Ctx& c, int a, int tid, int TEAM, int cur) {
    using CT = C<typename Mode::TS>;
    constexpr int CC = CHI * CHI;
    const int4 ve = c.vert_edges[a];
    const int es[3] = {ve.x, ve.y, ve.z};
    const CT* src = (const CT*)c.msg[cur];
    CT* dst = (CT*)c.msg[cur ^ 1];
    for (int k = 0; k < 3; ++k) {
        if (es[k] < 0) continue;
        const int u = c.edge_info[es[k]].x;
        const int out = 2 * es[k] + (a == u ? 0 : 1);
        for (int r = tid; r < CC; r += TEAM) dst[(size_t)out * CC + r] = ldcg(src + (size_t)out * CC + r);
    }
}

// Exact distance of the sweep that wrote msg[cur_new] for the instances with need[b]
// set: trace norms of new - old for every directed message, one group of CHI^2/2
// threads per message (whole block, after a grid barrier).  Accumulates into ex[b].
template <int CHI, class Mode, int TPB>
__device__ void bp_exact_pass(const Ctx& c, int cur_new, const int* need, C<typename Mode::TS>* scratch,
                              double* bacc, double* ex) {
    using TS = typename Mode::TS;
    using CT = C<TS>;
    constexpr int CC = CHI * CHI, GJ = CC / 2, NG = TPB / GJ;
    const int gi = threadIdx.x / GJ, g = threadIdx.x % GJ;
    CT* Dm = scratch + gi * CC;
    const CT* nw = (const CT*)c.msg[cur_new];
    const CT* od = (const CT*)c.msg[cur_new ^ 1];
    if (threadIdx.x == 0) *bacc = 0.0;
    __syncthreads();
    const WarpGroup grp{group_mask<GJ>()};
    double mine = 0.0;
    for (int mi = blockIdx.x * NG + gi; mi < 2 * c.m; mi += c.nblocks * NG) {
        const int inst = c.vert_inst[c.edge_info[mi >> 1].x];
        if (!need[inst]) continue;
        for (int r = g; r < CC; r += GJ) Dm[r] = ldcg(nw + (size_t)mi * CC + r) - ldcg(od + (size_t)mi * CC + r);
        jacobi_svd<CHI, TS, WarpGroup, false, !Mode::mixed>(Dm, nullptr, g, grp, group_mask<CHI>(),
                                                             Mode::mixed ? (TS)1e-6 : (TS)1e-15, 60, false, nullptr,
                                                             Mode::mixed ? (TS)1e-3 : (TS)3e-8);
        if (g == 0) {
            TS sacc = (TS)0;
            for (int cc = 0; cc < CHI; ++cc) {
                TS n2 = (TS)0;
                for (int r = 0; r < CHI; ++r) n2 += norm2(Dm[cc * CHI + r]);
                sacc += nr_sqrt(n2);
            }
            if (c.B == 1) mine += (double)sacc;
            else atomicAdd(ex + inst, (double)sacc);
        }
        grp.sync();
    }
    if (c.B == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if ((threadIdx.x & 31) == 0 && mine != 0.0) atomicAdd(bacc, mine);
        __syncthreads();
        if (threadIdx.x == 0 && *bacc != 0.0) atomicAdd(ex, *bacc);
    }
}

// ===========================================================================
// regauge, edge part (team CHI^2): FP64 eigen/SVD, transforms X_a, X_b and lambda
// ===========================================================================
template <int CHI>
struct RGSm {
    cd Am[2][CHI * CHI];
    cd Vm[2][CHI * CHI];
    double w[2][CHI];
    double wq[2][CHI], wiq[2][CHI];   // w^{1/2} and w^{-1/2} of the kept eigenvalues, else 0
    cd sq[2][CHI * CHI];
    cd isq[2][CHI * CHI];
    cd M[CHI * CHI];
    cd VM[CHI * CHI];
    double sig[CHI];
    double isig[CHI];   // 1 / sig (0 for a zero singular value)
    int perm[CHI];
    double scal[2];
    // mixed mode: scratch of the FP32-preconditioned SVDs
    cf A32[2][CHI * CHI];
    cf V32[2][CHI * CHI];
    cd T1[2][CHI * CHI];
    cd T2[2][CHI * CHI];
    double nrm[2][CHI];
};

template <int CHI, class Mode>
__device__ void regauge_edge(const Ctx& c, int e, int tid, int team, int cur, RGSm<CHI>& sm) {
    constexpr int TEAM = CHI * CHI, CC = CHI * CHI, GJ = CC / 2;
    // Hermitian parts of m_{a->b} (x = 0) and m_{b->a} (x = 1), column-major
    for (int t = tid; t < 2 * CC; t += TEAM) {
        const int x = t / CC, r = t % CC;
        const int row = r % CHI, col = r / CHI;
        cd v, vt;
        if constexpr (!Mode::mixed) {
            const cd* mm = (const cd*)c.msg[cur] + (size_t)(2 * e + x) * CC;
            v = ldcg(mm + row * CHI + col);
            vt = ldcg(mm + col * CHI + row);
        } else {
            const cf* mm = (const cf*)c.msg[cur] + (size_t)(2 * e + x) * CC;
            v = ccast<double>(ldcg(mm + row * CHI + col));
            vt = ccast<double>(ldcg(mm + col * CHI + row));
            if (row == col) {
                double s = 0.0;
                for (int q = 0; q < CHI; ++q) s += __ldcg(c.lam + (size_t)e * CHI + q);
                const double m0 = s > 0.0 ? __ldcg(c.lam + (size_t)e * CHI + row) * nr_rcp(s) : 0.0;
                v.x += m0;
                vt.x += m0;
            }
        }
        sm.Am[x][col * CHI + row] = cd{0.5 * (v.x + vt.x), 0.5 * (v.y - vt.y)};
    }
    team_bar<TEAM>(team);
    {
        // FP64 eigen-decompositions of the two Hermitian messages (the singular values of a
        // Hermitian matrix are the moduli of its eigenvalues); the mixed mode takes the
        // FP32-preconditioned path, whose result is FP64-accurate as well
        const int x = tid / GJ, g = tid % GJ;
        WarpGroup grp{group_mask<GJ>()};
        prune_noise<CHI>(sm.Am[x], g, grp);
        int sw, sw32 = 0;
        if constexpr (Mode::mixed)
            sw = mixed_svd<CHI>(sm.Am[x], sm.Vm[x], sm.A32[x], sm.V32[x], sm.T1[x], sm.T2[x], sm.nrm[x], g, grp,
                                group_mask<CHI>(), 1e-13, 3e-7, nullptr, &sw32);
        else
            sw = jacobi_svd<CHI, double, WarpGroup, true, true>(sm.Am[x], sm.Vm[x], g, grp, group_mask<CHI>(), 1e-15, 60,
                                                                true, nullptr, 3e-8);
        if (g == 0) {
            atomicAdd(&c.stats[4], (double)sw);
            atomicMax(&c.ctl->reg_sw_max, sw);
            atomicMax(&c.ctl->reg_sw32_max, sw32);
        }
    }
    team_bar<TEAM>(team);
    for (int t = tid; t < 2 * CHI; t += TEAM) {
        const int x = t / CHI, k = t % CHI;
        double n2 = 0.0, sg = 0.0;
        for (int r = 0; r < CHI; ++r) {
            const cd av = sm.Am[x][k * CHI + r], vv = sm.Vm[x][k * CHI + r];
            n2 += norm2(av);
            sg += vv.x * av.x + vv.y * av.y;
        }
        const double wv = nr_sqrt(n2);
        sm.w[x][k] = sg >= 0.0 ? wv : -wv;
    }
    team_bar<TEAM>(team);
    // the roots of each eigenvalue once (eigenvalues at or below the cut-off count as zero)
    for (int t = tid; t < 2 * CHI; t += TEAM) {
        const int x = t / CHI, k = t % CHI;
        double wmax = 0.0;
        for (int q = 0; q < CHI; ++q) wmax = fmax(wmax, sm.w[x][q]);
        const double wk = sm.w[x][k];
        const bool kept = wk > c.eig_cut * wmax;
        const double isq = kept ? nr_rsqrt(wk) : 0.0;
        sm.wiq[x][k] = isq;
        sm.wq[x][k] = kept ? wk * isq : 0.0;
    }
    team_bar<TEAM>(team);
    for (int t = tid; t < 2 * CC; t += TEAM) {
        const int x = t / CC, r = t % CC;
        const int j = r / CHI, jp = r % CHI;
        cd s1 = cd{0.0, 0.0}, s2 = cd{0.0, 0.0};
        for (int k = 0; k < CHI; ++k) {
            const double isq = sm.wiq[x][k];
            if (!(isq > 0.0)) continue;
            const double sq = sm.wq[x][k];
            const cd vv = sm.Vm[x][k * CHI + j] * conj(sm.Vm[x][k * CHI + jp]);
            s1 = cfma(cd{sq, 0.0}, vv, s1);
            s2 = cfma(cd{isq, 0.0}, vv, s2);
        }
        sm.sq[x][r] = s1;
        sm.isq[x][r] = s2;
    }
    team_bar<TEAM>(team);
    for (int t = tid; t < CC; t += TEAM) {
        const int k = t % CHI, l = t / CHI;
        cd acc = cd{0.0, 0.0};
        for (int j = 0; j < CHI; ++j) acc = cfma(sm.sq[0][j * CHI + k], sm.sq[1][j * CHI + l], acc);
        sm.M[l * CHI + k] = acc;
    }
    team_bar<TEAM>(team);
    if (tid < GJ) {
        WarpGroup grp{group_mask<GJ>()};
        prune_noise<CHI>(sm.M, tid, grp);
        int sw, sw32 = 0;
        if constexpr (Mode::mixed)
            sw = mixed_svd<CHI>(sm.M, sm.VM, sm.A32[0], sm.V32[0], sm.T1[0], sm.T2[0], sm.nrm[0], tid, grp,
                                group_mask<CHI>(), 1e-13, 3e-7, nullptr, &sw32);
        else
            sw = jacobi_svd<CHI, double, WarpGroup, true, true>(sm.M, sm.VM, tid, grp, group_mask<CHI>(), 1e-15, 60, true,
                                                                nullptr, 3e-8);
        if (tid == 0) {
            atomicAdd(&c.stats[4], (double)sw);
            atomicMax(&c.ctl->reg_sw_max, sw);
            atomicMax(&c.ctl->reg_sw32_max, sw32);
        }
    }
    team_bar<TEAM>(team);
    for (int cc = tid; cc < CHI; cc += TEAM) {
        double n2 = 0.0;
        for (int r = 0; r < CHI; ++r) n2 += norm2(sm.M[cc * CHI + r]);
        const double sv = nr_sqrt(n2);
        sm.sig[cc] = sv;
        sm.isig[cc] = sv > 0.0 ? nr_rcp(sv) : 0.0;
    }
    team_bar<TEAM>(team);
    for (int cc = tid; cc < CHI; cc += TEAM) sm.perm[desc_rank(sm.sig, CHI, cc)] = cc;
    team_bar<TEAM>(team);
    if (tid == 0) {
        double tot = 0.0;
        for (int cc = 0; cc < CHI; ++cc) tot += sm.sig[cc] * sm.sig[cc];
        const double nrm = nr_sqrt(tot);
        sm.scal[0] = nrm;
        sm.scal[1] = nr_sqrt(nrm);
        const double inrm = nrm > 0.0 ? nr_rcp(nrm) : 0.0;
        const double smax = sm.sig[sm.perm[0]];
        for (int r = 0; r < CHI; ++r) {
            const double s = sm.sig[sm.perm[r]];
            c.lam[(size_t)e * CHI + r] = (nrm > 0.0 && s > c.svd_cut * smax) ? s * inrm : 0.0;
        }
    }
    team_bar<TEAM>(team);
    for (int t = tid; t < 2 * CC; t += TEAM) {
        const int x = t / CC, r = t % CC;
        const int jpp = r / CHI, j = r % CHI;
        const int pc = sm.perm[j];
        const double s = sm.sig[pc];
        cd acc = cd{0.0, 0.0};
        const bool kept = sm.scal[0] > 0.0 && s > c.svd_cut * sm.sig[sm.perm[0]];
        if (kept) {
            for (int jp = 0; jp < CHI; ++jp) {
                const cd u = (x == 0) ? sm.isig[pc] * sm.M[pc * CHI + jp] : conj(sm.VM[pc * CHI + jp]);
                acc = cfma(sm.isq[x][jp * CHI + jpp], u, acc);
            }
            acc = sm.scal[1] * acc;
        }
        c.X[((size_t)e * 2 + x) * CC + r] = acc;
    }
}

// regauge, vertex part: Gamma_a = T_a x_slot X (team TV, buffers in shared memory)
template <int CHI, class Mode, int TEAM>
__device__ void regauge_vertex(const Ctx& c, int a, int tid, int team, C<typename Mode::TS>* buf) {
    using TS = typename Mode::TS;
    using CT = C<TS>;
    constexpr int H = CHI * CHI * CHI, CC = CHI * CHI;
    const int4 ve = c.vert_edges[a];
    const int es[3] = {ve.x, ve.y, ve.z};
    CT* b0 = buf;
    CT* b1 = buf + 2 * H;
    CT* Xs = buf + 4 * H;   // [3][CC]
    for (int t = tid; t < 2 * H; t += TEAM) b0[t] = ldcg((const CT*)c.T + (size_t)a * 2 * H + t);
    for (int t = tid; t < 3 * CC; t += TEAM) {
        const int k = t / CC, r = t % CC;
        cd v;
        if (es[k] >= 0) {
            const int side = (c.edge_info[es[k]].x == a) ? 0 : 1;
            v = ldcg(c.X + ((size_t)es[k] * 2 + side) * CC + r);
        } else {
            v = cd{(r / CHI == r % CHI) ? 1.0 : 0.0, 0.0};
        }
        Xs[t] = ccast<TS>(v);
    }
    team_bar<TEAM>(team);
    CT* cur = b0;
    CT* nxt = b1;
    for (int k = 0; k < 3; ++k) {
        const int st = sstride<CHI>(k);
        for (int t = tid; t < 2 * H; t += TEAM) {
            const int jk = (t / st) % CHI;
            const int base = t - jk * st;
            CT acc = CT{(TS)0, (TS)0};
            for (int q = 0; q < CHI; ++q) acc = cfma(cur[base + q * st], Xs[k * CC + q * CHI + jk], acc);
            nxt[t] = acc;
        }
        team_bar<TEAM>(team);
        CT* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    CT* g = (CT*)c.Gamma + (size_t)a * 2 * H;
    for (int t = tid; t < 2 * H; t += TEAM) g[t] = cur[t];
}

// ===========================================================================
// the persistent kernel
// ===========================================================================
template <int CHI, class Mode, unsigned PH, int V = 0>
struct SmemSize {
    using S = Shape<CHI, V>;
    static constexpr int TPB = S::TPB;
    static constexpr size_t gate = sizeof(GateSm<CHI>) * (TPB / S::TG);
    // per-team caches, block sums (64 doubles), scratch of the exact-distance pass
    static constexpr size_t bp = sizeof(BPSm<CHI, Mode, S::TB>) * (TPB / S::TB) + 64 * sizeof(double) +
                                 sizeof(C<typename Mode::TS>) * 2 * TPB;
    static constexpr size_t rg = sizeof(RGSm<CHI>) * (TPB / S::TR);
    static constexpr size_t rv =
        sizeof(C<typename Mode::TS>) * (4 * CHI * CHI * CHI + 3 * CHI * CHI) * (TPB / S::TRV);
    static constexpr size_t init =
        (sizeof(double) * (6 * CHI + 4) + (Mode::mixed ? sizeof(cd) * (2 * CHI * CHI * CHI + 3 * CHI * CHI) : 0)) * S::NIT;
    static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
    // bytes before the per-instance flags (which follow at this offset in the BP kernel)
    static constexpr size_t value = mx(mx((PH & PH_GATES) ? gate : 0, (PH & PH_BP) ? mx(bp, init) : 0),
                                       (PH & PH_REGAUGE) ? mx(rg, rv) : 0) + 16;
};

template <int CHI, class Mode, unsigned PH, int V>
__device__ __forceinline__ void anneal_body(const Ctx& c) {
    using S = Shape<CHI, V>;
    extern __shared__ __align__(16) unsigned char smem[];
    GridBarrier gb = grid_barrier_init(c.bar ? c.bar : &c.ctl->bar_count, &c.ctl->err, (unsigned)c.bar_expect);
    const int nteams_total_g = c.nblocks * (S::TPB / S::TG);
    int cur = *(volatile int*)&c.ctl->cur;
    const int kb = c.kdev ? *(volatile int*)c.kdev : c.k0, ke = c.kdev ? kb : c.k1;
    for (int k = kb; k <= ke; ++k) {
        double tZ, tX;
        if (c.Ksched > 0) {
            const double tau = (double)k / (double)c.Ksched;
            tZ = c.dt * tau;
            tX = c.dt * (1.0 - tau);
        } else {
            tZ = c.tZ1;
            tX = c.tX1;
        }
        double sX, cX;
        sincos(tX, &sX, &cX);
        if constexpr ((PH & PH_GATES) != 0u) {
            const double tXp = c.Ksched > 0 ? 0.0 : c.tXpre1;
            const bool pre = tXp != 0.0;
            double sXp = 0.0, cXp = 1.0, sXi = sX, cXi = cX;
            if (pre) {
                sincos(tXp, &sXp, &cXp);
                sincos(tX + tXp, &sXi, &cXi);   // vertices without gates: both mixing gates at once
            }
            const int team = threadIdx.x / S::TG, tid = threadIdx.x % S::TG;
            GateSm<CHI>& sm = reinterpret_cast<GateSm<CHI>*>(smem)[team];
            const int gteam = team * c.nblocks + blockIdx.x;
            for (int col = 0; col < c.ncol; ++col) {
                const int beg = c.colour_off[col], end = c.colour_off[col + 1];
                for (int idx = beg + gteam; idx < end; idx += nteams_total_g)
                    gate_edge<CHI, Mode>(c, c.colour_edges[idx], tid, team, sm, tZ, cX, sX, col, pre, cXp, sXp);
                if (col == c.ncol - 1)
                    for (int q = gteam; q < c.n_iso; q += nteams_total_g)
                        mixing_vertex<CHI, Mode>(c, c.iso[q], tid, S::TG, cXi, sXi);
                if (!grid_sync(gb, c.spin_limit)) return;
            }
            if (c.ncol == 0) {
                for (int q = gteam; q < c.n_iso; q += nteams_total_g)
                    mixing_vertex<CHI, Mode>(c, c.iso[q], tid, S::TG, cXi, sXi);
                if (!grid_sync(gb, c.spin_limit)) return;
            }
        }
        // regauge policy (Sec. II C): BP and gauge finding only when R exceeds the threshold;
        // every block reads the same value, so the whole grid takes the same branch
        const bool skip_regauge = c.rgate && !(__ldcg(c.rgate) > c.rthr_sum);
        if constexpr ((PH & PH_BP) != 0u) {
            if (skip_regauge) continue;
            {
                static_assert(S::TV == 32, "one warp per BP-init team");
                const int team = threadIdx.x / S::TV, tid = threadIdx.x % S::TV;
                const int gteam = team * c.nblocks + blockIdx.x, nt = c.nblocks * S::NIT;
                double* wsm = reinterpret_cast<double*>(smem) + team * (6 * CHI + 4);
                cd* tsm = reinterpret_cast<cd*>(reinterpret_cast<double*>(smem) + S::NIT * (6 * CHI + 4)) +
                          team * (2 * CHI * CHI * CHI + 3 * CHI * CHI);
                if (team < S::NIT)
                    for (int a = gteam; a < c.n; a += nt)
                        bp_init_vertex<CHI, Mode>(c, a, tid, cur, (c.phases & PH_WARM) != 0, wsm, tsm);
                const int g = blockIdx.x * S::TPB + threadIdx.x;
                for (int b = g; b < c.B; b += c.nblocks * S::TPB) {
                    c.inst_done[b] = 0;   // host-visible copy
                    c.inst_iters[b] = 0;
                    c.inst_dist[b] = 0.0;
                    for (int q = 0; q < 6; ++q) c.acc[q * c.B + b] = 0.0;
                }
                if (!grid_sync(gb, c.spin_limit)) return;
            }
            const int team = threadIdx.x / S::TB, tid = threadIdx.x % S::TB;
            const int tpb_teams = S::TPB / S::TB;
            using CT_ = C<typename Mode::TS>;
            using SMB = BPSm<CHI, Mode, S::TB>;
            SMB& sm = reinterpret_cast<SMB*>(smem)[team];
            double* bsum = reinterpret_cast<double*>(smem + sizeof(SMB) * tpb_teams);
            // every block keeps its own copy of the per-instance state; all blocks take
            // identical decisions from the same accumulators, so one barrier per sweep suffices
            // (two when a sweep's lower bound falls under the threshold and the exact
            // distance is computed afterwards)
            int* done = reinterpret_cast<int*>(smem + SmemSize<CHI, Mode, PH, V>::value);
            int* exnow = done + c.B;   // this sweep computes the exact distance inline
            int* need = exnow + c.B;   // exact distance needed after the sweep
            double* thr = reinterpret_cast<double*>(smem + SmemSize<CHI, Mode, PH, V>::value +
                                                    (3 * sizeof(int) * (size_t)c.B + 7) / 8 * 8);
            double* thr_hi = thr + c.B;                               // bound that lets a sweep continue
            float* thr3 = reinterpret_cast<float*>(thr_hi + c.B);     // inline-exact trigger
            CT_* scratch = reinterpret_cast<CT_*>(bsum + 64);
            const double slack = Mode::mixed ? 1e-5 : 1e-12;   // rounding of the lower bound
            for (int b = threadIdx.x; b < c.B; b += S::TPB) {
                done[b] = 0;
                exnow[b] = c.max_iter == 1;
                need[b] = 0;
                const double t = c.tol * (double)c.inst_m[b];
                thr[b] = t;
                thr_hi[b] = t / (1.0 - slack);
                thr3[b] = (float)(3.0 * t);
            }
            if (tid == 0) sm.cached = -1;   // T and D0 changed in the init phase
            if (tid < 3) sm.dsum[tid] = 0;
            __syncthreads();
            const int gteam = team * c.nblocks + blockIdx.x, nt = c.nblocks * tpb_teams;
            const int inst0 = gteam < c.n ? c.vert_inst[gteam] : 0;   // the first round's vertex
            SMB* all = reinterpret_cast<SMB*>(smem);
            bool have_pre = false;
            CT_ pre = CT_{0, 0};
            int* sflag = reinterpret_cast<int*>(bsum + 48);   // [2]: need | open << 1, per sweep parity
            if (threadIdx.x == 0) sflag[0] = sflag[1] = 0;
            __syncthreads();
            int it = 0;
            for (; it < c.max_iter; ++it) {
                double* acc = c.acc + (size_t)(it % 3) * c.B;
                double* acc_next = c.acc + (size_t)((it + 1) % 3) * c.B;
                double* ex = c.acc + (size_t)(3 + it % 3) * c.B;
                double* ex_next = c.acc + (size_t)(3 + (it + 1) % 3) * c.B;
                for (int b = blockIdx.x * S::TPB + threadIdx.x; b < c.B; b += c.nblocks * S::TPB) {
                    acc_next[b] = 0.0;
                    ex_next[b] = 0.0;
                }
                // rounds of one vertex per team; the block synchronises twice per round
                for (int base = 0; base < c.n; base += nt) {
                    const int a = base + gteam;
                    int inst = 0;
                    bool act = false;
                    if (a < c.n) {
                        inst = base == 0 ? inst0 : c.vert_inst[a];
                        if (done[inst]) bp_copy_vertex<CHI, Mode>(c, a, tid, S::TB, cur);
                        else act = true;
                    }
                    if (act) bp_front<CHI, Mode, S::TB>(c, a, tid, team, cur, sm, base == 0 && have_pre, pre);
                    __syncthreads();
                    if (threadIdx.x < 32) bp_trace_rcp<CHI, Mode, S::TB>(all, tpb_teams);
                    __syncthreads();
                    if (act) bp_back<CHI, Mode, S::TB>(c, tid, team, cur, exnow[inst] != 0, sm, c.B == 1 ? nullptr : acc + inst);
                }
                cur ^= 1;
                // one instance: the first warp sums the teams' distances between the block's
                // barrier and its arrival at the grid barrier
                if (!grid_sync_pre(gb, c.spin_limit, [&]() {
                        if (c.B != 1) return;
                        typename Mode::TS v = 0;
                        for (int q = threadIdx.x; q < 3 * tpb_teams; q += 32) v += all[q / 3].dsum[q % 3];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (threadIdx.x == 0) atomicAdd(acc, (double)v);
                    }))
                    return;
                if (tid < 3) sm.dsum[tid] = 0;   // read by the first warp before the barrier
                // the next sweep's incoming messages of this team's first vertex are loaded
                // now, so that their latency overlaps the decision below
                have_pre = false;
                if (gteam < c.n && sm.cached == gteam && tid < 3 * CHI * CHI) {
                    const int in = sm.in_idx[tid / (CHI * CHI)];
                    if (in >= 0) pre = ldcg((const CT_*)c.msg[cur] + (size_t)in * CHI * CHI + tid % (CHI * CHI));
                    have_pre = true;
                }
                // stopping rule of App. B, per instance, evaluated identically by every block;
                // the raw distance sums are kept and divided by |E| at the end
                const bool last = it + 1 >= c.max_iter;
                int open_local = 0, need_local = 0;
                for (int b = threadIdx.x; b < c.B; b += S::TPB) {
                    if (done[b]) continue;
                    const double dsum = __ldcg(acc + b);
                    bool fin;
                    if (c.inst_m[b] == 0 || !(dsum == dsum)) {
                        fin = true;
                    } else if (exnow[b]) {
                        fin = last || dsum < thr[b];
                    } else if (!last && dsum >= thr_hi[b]) {
                        fin = false;   // the exact distance is at least the bound
                    } else {
                        need[b] = 1;
                        need_local = 1;
                        continue;
                    }
                    if (blockIdx.x == 0) {
                        c.inst_dist[b] = dsum;
                        c.inst_iters[b] = it + 1;
                        if (fin) c.inst_done[b] = 1;
                    }
                    if (fin) done[b] = 1;
                    else open_local = 1;
                    // the next sweep is exact inline when it is the last or when this
                    // sweep came within a factor 3 of the threshold
                    exnow[b] = (it + 2 >= c.max_iter) || (float)dsum < thr3[b];
                }
                // one block barrier for both flags (a word per sweep parity, reset one sweep ahead)
                if (need_local | open_local) atomicOr(&sflag[it & 1], need_local | (open_local << 1));
                __syncthreads();
                const int fl = sflag[it & 1];
                if (threadIdx.x == 0) sflag[(it + 1) & 1] = 0;
                if (fl & 1) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) ++c.ctl->exact_passes;
                    bp_exact_pass<CHI, Mode, S::TPB>(c, cur, need, scratch, bsum + 32, ex);
                    if (!grid_sync(gb, c.spin_limit)) return;
                    for (int b = threadIdx.x; b < c.B; b += S::TPB) {
                        if (!need[b]) continue;
                        need[b] = 0;
                        const double dsum = __ldcg(ex + b);
                        const bool fin = last || dsum < thr[b] || !(dsum == dsum);
                        if (blockIdx.x == 0) {
                            c.inst_dist[b] = dsum;
                            c.inst_iters[b] = it + 1;
                            if (fin) c.inst_done[b] = 1;
                        }
                        if (fin) done[b] = 1;
                        else open_local = 1;
                        exnow[b] = 1;
                    }
                    if (!__syncthreads_or(open_local)) {
                        ++it;
                        break;
                    }
                } else if (!(fl & 2)) {
                    ++it;
                    break;
                }
            }
            __syncthreads();
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                int mi = 0, ncv = 0;
                double md = 0.0;
                for (int b = 0; b < c.B; ++b) {
                    const int mb = c.inst_m[b];
                    c.inst_dist[b] = mb > 0 ? c.inst_dist[b] / (double)mb : 0.0;
                    mi = c.inst_iters[b] > mi ? c.inst_iters[b] : mi;
                    md = c.inst_dist[b] > md ? c.inst_dist[b] : md;
                    if (!(c.inst_dist[b] < c.tol) && c.inst_m[b] > 0) ++ncv;
                }
                c.ctl->last_iters = mi;
                c.ctl->last_dist = md;
                c.ctl->not_conv = ncv;
                c.ctl->sweeps_total += mi;
                c.ctl->bp_calls += 1;
                c.ctl->nc_calls += (ncv > 0) ? 1 : 0;
                c.ctl->cur = cur;
            }
        }
        if constexpr ((PH & PH_REGAUGE) != 0u) {
            if (c.rgate && blockIdx.x == 0 && threadIdx.x == 0) {
                if (skip_regauge) ++c.ctl->reg_skipped;
                else ++c.ctl->regauged;
            }
            if (skip_regauge) continue;
            {
                const int team = threadIdx.x / S::TR, tid = threadIdx.x % S::TR;
                RGSm<CHI>& sm = reinterpret_cast<RGSm<CHI>*>(smem)[team];
                const int gteam = team * c.nblocks + blockIdx.x, nt = c.nblocks * (S::TPB / S::TR);
                for (int e = gteam; e < c.m; e += nt) regauge_edge<CHI, Mode>(c, e, tid, team, cur, sm);
                if (!grid_sync(gb, c.spin_limit)) return;
            }
            {
                using CT = C<typename Mode::TS>;
                const int team = threadIdx.x / S::TRV, tid = threadIdx.x % S::TRV;
                CT* buf = reinterpret_cast<CT*>(smem) + (size_t)team * (4 * CHI * CHI * CHI + 3 * CHI * CHI);
                const int gteam = team * c.nblocks + blockIdx.x, nt = c.nblocks * (S::TPB / S::TRV);
                for (int a = gteam; a < c.n; a += nt) {
                    regauge_vertex<CHI, Mode, S::TRV>(c, a, tid, team, buf);
                    team_bar<S::TRV>(team);
                }
                if (!grid_sync(gb, c.spin_limit)) return;
            }
        }
        // every block read *kdev at entry, before the barriers above
        if constexpr ((PH & PH_REGAUGE) != 0u)
            if (c.kdev && blockIdx.x == 0 && threadIdx.x == 0) *c.kdev = k + 1;
    }
}

// The three phase kernels (one cooperative launch each).
template <int CHI, class Mode, int V>
__global__ void __launch_bounds__(Shape<CHI, V>::TPB, 1) gates_kernel(Ctx c) { anneal_body<CHI, Mode, PH_GATES, V>(c); }
template <int CHI, class Mode, int V>
__global__ void __launch_bounds__(Shape<CHI, V>::TPB, 1) bp_kernel(Ctx c) { anneal_body<CHI, Mode, PH_BP, V>(c); }
template <int CHI, class Mode, int V>
__global__ void __launch_bounds__(Shape<CHI, V>::TPB, 1) regauge_kernel(Ctx c) {
    anneal_body<CHI, Mode, PH_REGAUGE, V>(c);
}

}  // namespace gtqa
