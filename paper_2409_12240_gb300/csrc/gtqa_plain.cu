// Plain-path kernel instantiations (FP64): degree 4 with CHI in {2, 4}, degree 3 with CHI = 16.
#include "gtqa_launch.h"

namespace gtqa {

namespace {
template <int CHI, int D>
size_t sweep_smem() {
    using S = PlainShape<CHI, D>;
    return sizeof(cd) * ((D + 1) * S::CC + (S::SMEM ? 3 * S::H2 : 0));
}
template <int CHI, int D>
size_t vertex_smem() {
    using S = PlainShape<CHI, D>;
    return sizeof(cd) * (D * S::CC + (S::SMEM ? 2 * S::H2 : 0));
}
template <int CHI, int D>
cudaError_t init_t(const PlainArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    plain_bp_init_kernel<CHI, D><<<a.n, 256, 0, st>>>(a);
    return cudaGetLastError();
}
template <int CHI, int D>
cudaError_t sweep_t(const PlainArgs& a, cudaStream_t st) {
    using S = PlainShape<CHI, D>;
    if (a.n > 0) {
        plain_bp_sweep_kernel<CHI, D><<<a.n, S::NT, sweep_smem<CHI, D>(), st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.m > 0) plain_trace_norm_kernel<CHI><<<2 * a.m, S::CC / 2, 0, st>>>(a.dm, a.acc);
    return cudaGetLastError();
}
template <int CHI, int D>
cudaError_t regauge_t(const PlainArgs& a, const cd* msg, double eig_cut, double svd_cut, cudaStream_t st) {
    using S = PlainShape<CHI, D>;
    if (a.m > 0) {
        plain_regauge_edge_kernel<CHI><<<a.m, S::CC / 2, 0, st>>>(msg, a.lam, a.X, eig_cut, svd_cut);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.n <= 0) return cudaSuccess;
    plain_regauge_vertex_kernel<CHI, D><<<a.n, 256, vertex_smem<CHI, D>(), st>>>(a);
    return cudaGetLastError();
}
template <int CHI, int D>
cudaError_t marg_t(const cd* G, const double* lam, const int4* vs, int n, cd* rho, int8_t* sign, int* flag,
                   cudaStream_t st) {
    const int wpb = 4;
    plain_marginals_kernel<CHI, D><<<(n + wpb - 1) / wpb, 32 * wpb, 0, st>>>(G, lam, vs, n, rho, sign, flag);
    return cudaGetLastError();
}
}  // namespace

#define GTQA_PLAIN_DISPATCH(CALL)                                  \
    if (D == 4 && CHI == 2) return CALL(2, 4);                     \
    if (D == 4 && CHI == 4) return CALL(4, 4);                     \
    if (D == 3 && CHI == 16) return CALL(16, 3);                   \
    return cudaErrorInvalidValue;

bool plain_supported(int CHI, int D) { return (D == 4 && (CHI == 2 || CHI == 4)) || (D == 3 && CHI == 16); }

size_t plain_scratch_entries(int CHI, int D, int n, int m) {
    size_t s = 0;
    if (D == 3 && CHI == 16) {
        s = std::max((size_t)n * PlainShape<16, 3>::scratch_per_block, (size_t)m * 4 * 16 * 256);
    }
    return s;
}

cudaError_t plain_bp_init_launch(int CHI, int D, const PlainArgs& a, cudaStream_t st) {
#define C_(c, d) init_t<c, d>(a, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_bp_sweep_launch(int CHI, int D, const PlainArgs& a, cudaStream_t st) {
#define C_(c, d) sweep_t<c, d>(a, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_regauge_launch(int CHI, int D, const PlainArgs& a, const cd* msg, double eig_cut, double svd_cut,
                                 cudaStream_t st) {
#define C_(c, d) regauge_t<c, d>(a, msg, eig_cut, svd_cut, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_marginals_launch(int CHI, int D, const cd* G, const double* lam, const int4* vs, int n, cd* rho,
                                   int8_t* sign, int* flag, cudaStream_t st) {
#define C_(c, d) marg_t<c, d>(G, lam, vs, n, rho, sign, flag, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_general_gates_launch(int CHI, int D, const GenArgs& a, cudaStream_t st) {
    if (D == 4 && CHI == 2) return general_gates_launch_t<2, 4, ModeFP64>(a, st);
    if (D == 4 && CHI == 4) return general_gates_launch_t<4, 4, ModeFP64>(a, st);
    return cudaErrorInvalidValue;   // CHI = 16: the whole-side core (64 x 64) exceeds one block's Jacobi
}
cudaError_t plain_single_gates_launch(int CHI, int D, void* G, const int* v, const cd* W, int count, cudaStream_t st) {
#define C_(c, d) single_gates_launch_t<c, d, ModeFP64>(G, v, W, count, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t ising16_gates_launch(const Gate16Args& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    ising16_gate_kernel<16><<<a.count, 512, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gtqa
