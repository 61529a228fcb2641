// Degree-4 kernel instantiations (FP64 mode, CHI in {2, 4}).
#include "gtqa_launch.h"

namespace gtqa {

namespace {
template <int CHI>
cudaError_t init_t(const D4Args& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    d4_bp_init_kernel<CHI><<<a.n, 128, 0, st>>>(a);
    return cudaGetLastError();
}
template <int CHI>
cudaError_t sweep_t(const D4Args& a, cudaStream_t st) {
    using S = D4Shape<CHI>;
    if (a.n <= 0) return cudaSuccess;
    const size_t smem = sizeof(cd) * (3 * S::H2 + 8 * S::CC);
    d4_bp_sweep_kernel<CHI><<<a.n, S::NT, smem, st>>>(a);
    return cudaGetLastError();
}
template <int CHI>
cudaError_t regauge_t(const Ctx& c, int cur, const D4Args& a, cudaStream_t st) {
    using S = D4Shape<CHI>;
    if (a.m > 0) {
        d4_regauge_edge_kernel<CHI><<<a.m, CHI * CHI, 0, st>>>(c, cur);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.n <= 0) return cudaSuccess;
    const size_t smem = sizeof(cd) * (2 * S::H2 + 4 * S::CC);
    d4_regauge_vertex_kernel<CHI><<<a.n, 128, smem, st>>>(a);
    return cudaGetLastError();
}
template <int CHI>
cudaError_t marg_t(const cd* G, const double* lam, const int4* vs, int n, cd* rho, int8_t* sign, int* flag,
                   cudaStream_t st) {
    const int wpb = 4;
    d4_marginals_kernel<CHI><<<(n + wpb - 1) / wpb, 32 * wpb, 0, st>>>(G, lam, vs, n, rho, sign, flag);
    return cudaGetLastError();
}
}  // namespace

cudaError_t d4_bp_init_launch(int CHI, const D4Args& a, cudaStream_t st) {
    return CHI == 2 ? init_t<2>(a, st) : (CHI == 4 ? init_t<4>(a, st) : cudaErrorInvalidValue);
}
cudaError_t d4_bp_sweep_launch(int CHI, const D4Args& a, cudaStream_t st) {
    return CHI == 2 ? sweep_t<2>(a, st) : (CHI == 4 ? sweep_t<4>(a, st) : cudaErrorInvalidValue);
}
cudaError_t d4_regauge_launch(int CHI, const Ctx& c, int cur, const D4Args& a, cudaStream_t st) {
    return CHI == 2 ? regauge_t<2>(c, cur, a, st) : (CHI == 4 ? regauge_t<4>(c, cur, a, st) : cudaErrorInvalidValue);
}
cudaError_t d4_marginals_launch(int CHI, const cd* G, const double* lam, const int4* vs, int n, cd* rho,
                                int8_t* sign, int* flag, cudaStream_t st) {
    return CHI == 2 ? marg_t<2>(G, lam, vs, n, rho, sign, flag, st)
                    : (CHI == 4 ? marg_t<4>(G, lam, vs, n, rho, sign, flag, st) : cudaErrorInvalidValue);
}
cudaError_t d4_general_gates_launch(int CHI, const GenArgs& a, cudaStream_t st) {
    return CHI == 2 ? general_gates_launch_t<2, 4, ModeFP64>(a, st)
                    : (CHI == 4 ? general_gates_launch_t<4, 4, ModeFP64>(a, st) : cudaErrorInvalidValue);
}
cudaError_t d4_single_gates_launch(int CHI, void* G, const int* v, const cd* W, int count, cudaStream_t st) {
    return CHI == 2 ? single_gates_launch_t<2, 4, ModeFP64>(G, v, W, count, st)
                    : (CHI == 4 ? single_gates_launch_t<4, 4, ModeFP64>(G, v, W, count, st) : cudaErrorInvalidValue);
}

}  // namespace gtqa
