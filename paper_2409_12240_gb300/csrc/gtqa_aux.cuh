// Auxiliary kernels of the persistent path (degree <= 3, CHI in {2, 4, 8}): the marginals
// and read-out (Sec. II B, Eqs. (partial_dens), (bp_approx); Sec. III A, Eq. (rounding_rule)),
// the local-orthogonality residual R (App. C), and one step of the measurement sampling
// (Sec. IV A, Eq. (projection)).  Same layouts and precision modes as the phase kernels.
#pragma once

#include "gtqa_anneal.cuh"

namespace gtqa {

// marginals rho_a = sum Gamma Gamma^* prod lambda^2 / tr and the read-out (one warp per vertex)
template <int CHI, class Mode>
__global__ void marginals_kernel2(const C<typename Mode::TS>* Gamma, const double* lam, const int4* vert_edges, int n,
                                  cd* rho, int8_t* sign, int* nan_flag) {
    constexpr int H = CHI * CHI * CHI;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int a = warp;
    const int4 ve = vert_edges[a];
    cd acc[4] = {cd{0, 0}, cd{0, 0}, cd{0, 0}, cd{0, 0}};
    for (int r = lane; r < H; r += 32) {
        const int j0 = r / (CHI * CHI), j1 = (r / CHI) % CHI, j2 = r % CHI;
        const double l0 = lam_get(lam, CHI, ve.x, j0), l1 = lam_get(lam, CHI, ve.y, j1), l2 = lam_get(lam, CHI, ve.z, j2);
        const double wgt = (l0 * l0) * (l1 * l1) * (l2 * l2);
        const cd g0 = ccast<double>(Gamma[(size_t)a * 2 * H + r]);
        const cd g1 = ccast<double>(Gamma[(size_t)a * 2 * H + H + r]);
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
        for (int q = 0; q < 4; ++q) rho[(size_t)a * 4 + q] = it * acc[q];
        if (sign) sign[a] = (acc[0].x * it > 0.5) ? 1 : -1;
        if (!(tr == tr) || tr == 0.0) atomicOr(nan_flag, 1);
    }
}

// Residual R of the local-orthogonality condition (App. C):
//   R = 1/(2|E|) sum_a sum_{b in da} || delta - sum Gamma_a Gamma_a^* prod_{c != b} lambda_ca^2 ||_1,
// where delta is the identity on the bond indices with lambda > 0 (the padded indices do not
// exist in the state) and the trace norm is the sum of singular values of the C x C
// difference (FP64 Jacobi).  Adds the unnormalised sum over the 2m directed bonds to *out.
// One warp handles IPW consecutive (vertex, slot) items: first the CHI^2 elements of every
// item's matrix, spread over the lanes, then one Jacobi SVD per item on its own group of GJ
// lanes, so that up to 32 lanes share each FP64 instruction of the trace norms.
template <int CHI, class Mode>
__global__ void residual_kernel(const C<typename Mode::TS>* Gamma, const double* lam, const int4* vert_edges, int n,
                                double* out) {
    constexpr int H = CHI * CHI * CHI, CC = CHI * CHI, GJ = CC / 2 > 0 ? CC / 2 : 1, WPB = 8;
    constexpr int IPW = 32 / GJ > 0 ? 32 / GJ : 1;
    static_assert(GJ * IPW <= 32 || IPW == 1, "items of one warp");
    __shared__ cd Dsm[WPB][IPW][CC];
    const int wib = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int item0 = (blockIdx.x * WPB + wib) * IPW;
    if (item0 >= 3 * n) return;   // the whole warp
    for (int t = lane; t < IPW * CC; t += 32) {
        const int q = t / CC, r = t % CC;
        const int item = item0 + q;
        if (item >= 3 * n) continue;
        const int a = item / 3, s = item % 3;
        const int4 ve = vert_edges[a];
        const int es[3] = {ve.x, ve.y, ve.z};
        if (es[s] < 0) continue;
        int o0, o1;
        others_of(s, o0, o1);
        const int ss = sstride<CHI>(s), s0 = sstride<CHI>(o0), s1 = sstride<CHI>(o1);
        const C<typename Mode::TS>* g = Gamma + (size_t)a * 2 * H;
        const int j = r / CHI, jp = r % CHI;
        cd acc = cd{0.0, 0.0};
        for (int i = 0; i < 2; ++i)
            for (int u = 0; u < CHI; ++u) {
                const double lu = lam_get(lam, CHI, es[o0], u);
                for (int v = 0; v < CHI; ++v) {
                    const double lv = lam_get(lam, CHI, es[o1], v);
                    const int base = i * H + u * s0 + v * s1;
                    const cd x = ccast<double>(g[base + j * ss]), y = ccast<double>(g[base + jp * ss]);
                    acc = cfmac(y, (lu * lu * lv * lv) * x, acc);
                }
            }
        const double act = (j == jp && lam_get(lam, CHI, es[s], j) > 0.0) ? 1.0 : 0.0;
        Dsm[wib][q][r] = cd{act - acc.x, -acc.y};
    }
    __syncwarp();
    const int q = lane / GJ, g = lane % GJ, item = item0 + q;
    bool valid = q < IPW && item < 3 * n;
    if (valid) {
        const int4 ve = vert_edges[item / 3];
        const int s = item % 3;
        valid = (s == 0 ? ve.x : (s == 1 ? ve.y : ve.z)) >= 0;
    }
    if (valid) {   // the same for the GJ lanes of an item
        WarpGroup grp{group_mask<GJ>()};
        // FP32 rotation angles with FP64-exact rotations and the quadratic stop, as in the
        // exact trace norms of the BP distance (the singular values stay FP64-accurate)
        jacobi_svd<CHI, double, WarpGroup, false, true>(Dsm[wib][q], nullptr, g, grp, group_mask<CHI>(), 1e-15, 60,
                                                        false, nullptr, 3e-8);
        grp.sync();
        if (g == 0) {
            double sacc = 0.0;
            for (int cc = 0; cc < CHI; ++cc) {
                double n2 = 0.0;
                for (int r = 0; r < CHI; ++r) n2 += norm2(Dsm[wib][q][cc * CHI + r]);
                sacc += nr_sqrt(n2);
            }
            atomicAdd(out, sacc);
        }
    }
}

// One step of the measurement sampling of Sec. IV A for vertex a (one warp): rho_a as in
// marginals_kernel2, the outcome x_a = +1 if u < rho_a[0,0] (else -1), its probability, and
// the projection of Eq. (projection): the other physical component of Gamma_a is zeroed.
template <int CHI, class Mode>
__global__ void sample_kernel(C<typename Mode::TS>* Gamma, const double* lam, const int4* vert_edges, int a, double u,
                              int step, int8_t* x_out, double* p_out) {
    constexpr int H = CHI * CHI * CHI;
    const int lane = threadIdx.x & 31;
    const int4 ve = vert_edges[a];
    C<typename Mode::TS>* g = Gamma + (size_t)a * 2 * H;
    double r00 = 0.0, r11 = 0.0;
    for (int r = lane; r < H; r += 32) {
        const int j0 = r / (CHI * CHI), j1 = (r / CHI) % CHI, j2 = r % CHI;
        const double l0 = lam_get(lam, CHI, ve.x, j0), l1 = lam_get(lam, CHI, ve.y, j1), l2 = lam_get(lam, CHI, ve.z, j2);
        const double wgt = (l0 * l0) * (l1 * l1) * (l2 * l2);
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
    for (int r = lane; r < H; r += 32) g[(1 - keep) * H + r] = C<typename Mode::TS>{0, 0};
}

}  // namespace gtqa
