// Plain-path kernel instantiations.  FP64: degree 4 with CHI in {2, 4}, degree 3 with CHI = 16.
// Complex64 mode (every step in FP32): degree 3 with CHI in {2, 4, 8, 16}, degree 4 with CHI in {2, 4}.
#include "gtqa_launch.h"

namespace gtqa {

namespace {
template <int CHI, int D, typename R>
size_t sweep_smem() {
    using S = PlainShape<CHI, D, R>;
    return sizeof(C<R>) * ((D + 1) * S::CC + (S::SMEM ? 3 * S::H2 : 0));
}
template <int CHI, int D, typename R>
size_t vertex_smem() {
    using S = PlainShape<CHI, D, R>;
    return sizeof(C<R>) * (D * S::CC + (S::SMEM ? 2 * S::H2 : 0));
}
template <int CHI, int D, typename R>
cudaError_t init_t(const PlainArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    plain_bp_init_kernel<CHI, D, R><<<a.n, 256, 0, st>>>(a);
    return cudaGetLastError();
}
template <int CHI, int D, typename R>
cudaError_t sweep_t(const PlainArgs& a, cudaStream_t st) {
    using S = PlainShape<CHI, D, R>;
    if (a.n > 0) {
        plain_bp_sweep_kernel<CHI, D, R><<<a.n, S::NT, sweep_smem<CHI, D, R>(), st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.m > 0) plain_trace_norm_kernel<CHI, R><<<2 * a.m, S::CC / 2, 0, st>>>((const C<R>*)a.dm, a.acc);
    return cudaGetLastError();
}
template <int CHI, int D, typename R>
cudaError_t regauge_t(const PlainArgs& a, const void* msg, double eig_cut, double svd_cut, cudaStream_t st) {
    using S = PlainShape<CHI, D, R>;
    if (a.m > 0) {
        plain_regauge_edge_kernel<CHI, R><<<a.m, S::CC / 2, 0, st>>>((const C<R>*)msg, a.lam, (C<R>*)a.X, eig_cut,
                                                                     svd_cut);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.n <= 0) return cudaSuccess;
    plain_regauge_vertex_kernel<CHI, D, R><<<a.n, 256, vertex_smem<CHI, D, R>(), st>>>(a);
    return cudaGetLastError();
}
template <int CHI, int D, typename R>
cudaError_t marg_t(const void* G, const double* lam, const int4* vs, int n, cd* rho, int8_t* sign, int* flag,
                   cudaStream_t st) {
    const int wpb = 4;
    plain_marginals_kernel<CHI, D, R><<<(n + wpb - 1) / wpb, 32 * wpb, 0, st>>>((const C<R>*)G, lam, vs, n, rho, sign,
                                                                                flag);
    return cudaGetLastError();
}
template <int CHI, int D, typename R>
cudaError_t resid_t(const void* G, const double* lam, const int4* vs, int n, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    plain_residual_kernel<CHI, D, R><<<n * D, PlainShape<CHI, D, R>::CC / 2, 0, st>>>((const C<R>*)G, lam, vs, out);
    return cudaGetLastError();
}
template <int CHI, int D, typename R>
cudaError_t sample_t(void* G, const double* lam, const int4* vs, int a, double u, int step, int8_t* x, double* p,
                     cudaStream_t st) {
    plain_sample_kernel<CHI, D, R><<<1, 32, 0, st>>>((C<R>*)G, lam, vs, a, u, step, x, p);
    return cudaGetLastError();
}
}  // namespace

// CALL(CHI, D, R) for every built shape
#define GTQA_PLAIN_DISPATCH(CALL)                                              \
    if (!f32) {                                                                \
        if (D == 4 && CHI == 2) return CALL(2, 4, double);                     \
        if (D == 4 && CHI == 4) return CALL(4, 4, double);                     \
        if (D == 3 && CHI == 16) return CALL(16, 3, double);                   \
    } else {                                                                   \
        if (D == 3 && CHI == 2) return CALL(2, 3, float);                      \
        if (D == 3 && CHI == 4) return CALL(4, 3, float);                      \
        if (D == 3 && CHI == 8) return CALL(8, 3, float);                      \
        if (D == 3 && CHI == 16) return CALL(16, 3, float);                    \
        if (D == 4 && CHI == 2) return CALL(2, 4, float);                      \
        if (D == 4 && CHI == 4) return CALL(4, 4, float);                      \
    }                                                                          \
    return cudaErrorInvalidValue;

bool plain_supported(int CHI, int D, bool f32) {
    if (!f32) return (D == 4 && (CHI == 2 || CHI == 4)) || (D == 3 && CHI == 16);
    return (D == 3 && (CHI == 2 || CHI == 4 || CHI == 8 || CHI == 16)) || (D == 4 && (CHI == 2 || CHI == 4));
}

size_t plain_scratch_entries(int CHI, int D, int n, int m) {
    // complex entries (sized for complex128; the complex64 mode uses half of each entry)
    if (D == 3 && CHI == 16)
        return std::max((size_t)n * PlainShape<16, 3, double>::scratch_per_block, (size_t)m * 4 * 16 * 256);
    return 0;
}

cudaError_t plain_bp_init_launch(int CHI, int D, bool f32, const PlainArgs& a, cudaStream_t st) {
#define C_(c, d, r) init_t<c, d, r>(a, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_bp_sweep_launch(int CHI, int D, bool f32, const PlainArgs& a, cudaStream_t st) {
#define C_(c, d, r) sweep_t<c, d, r>(a, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_regauge_launch(int CHI, int D, bool f32, const PlainArgs& a, const void* msg, double eig_cut,
                                 double svd_cut, cudaStream_t st) {
#define C_(c, d, r) regauge_t<c, d, r>(a, msg, eig_cut, svd_cut, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_marginals_launch(int CHI, int D, bool f32, const void* G, const double* lam, const int4* vs, int n,
                                   cd* rho, int8_t* sign, int* flag, cudaStream_t st) {
#define C_(c, d, r) marg_t<c, d, r>(G, lam, vs, n, rho, sign, flag, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_residual_launch(int CHI, int D, bool f32, const void* G, const double* lam, const int4* vs, int n,
                                  double* out, cudaStream_t st) {
#define C_(c, d, r) resid_t<c, d, r>(G, lam, vs, n, out, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_sample_launch(int CHI, int D, bool f32, void* G, const double* lam, const int4* vs, int a, double u,
                                int step, int8_t* x, double* p, cudaStream_t st) {
#define C_(c, d, r) sample_t<c, d, r>(G, lam, vs, a, u, step, x, p, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_general_gates_launch(int CHI, int D, bool f32, const GenArgs& a, cudaStream_t st) {
    if (!f32) {
        if (D == 4 && CHI == 2) return general_gates_launch_t<2, 4, ModeFP64>(a, st);
        if (D == 4 && CHI == 4) return general_gates_launch_t<4, 4, ModeFP64>(a, st);
    } else {
        if (D == 3 && CHI == 2) return general_gates_launch_t<2, 3, ModeC64>(a, st);
        if (D == 3 && CHI == 4) return general_gates_launch_t<4, 3, ModeC64>(a, st);
        if (D == 3 && CHI == 8) return general_gates_launch_t<8, 3, ModeC64>(a, st);
        if (D == 4 && CHI == 2) return general_gates_launch_t<2, 4, ModeC64>(a, st);
        if (D == 4 && CHI == 4) return general_gates_launch_t<4, 4, ModeC64>(a, st);
    }
    return cudaErrorInvalidValue;   // CHI = 16: the whole-side core (64 x 64) exceeds one block's Jacobi
}
cudaError_t plain_single_gates_launch(int CHI, int D, bool f32, void* G, const int* v, const cd* W, int count,
                                      cudaStream_t st) {
    if (!f32) {
        if (D == 4 && CHI == 2) return single_gates_launch_t<2, 4, ModeFP64>(G, v, W, count, st);
        if (D == 4 && CHI == 4) return single_gates_launch_t<4, 4, ModeFP64>(G, v, W, count, st);
        if (D == 3 && CHI == 16) return single_gates_launch_t<16, 3, ModeFP64>(G, v, W, count, st);
    } else {
        if (D == 3 && CHI == 2) return single_gates_launch_t<2, 3, ModeC64>(G, v, W, count, st);
        if (D == 3 && CHI == 4) return single_gates_launch_t<4, 3, ModeC64>(G, v, W, count, st);
        if (D == 3 && CHI == 8) return single_gates_launch_t<8, 3, ModeC64>(G, v, W, count, st);
        if (D == 3 && CHI == 16) return single_gates_launch_t<16, 3, ModeC64>(G, v, W, count, st);
        if (D == 4 && CHI == 2) return single_gates_launch_t<2, 4, ModeC64>(G, v, W, count, st);
        if (D == 4 && CHI == 4) return single_gates_launch_t<4, 4, ModeC64>(G, v, W, count, st);
    }
    return cudaErrorInvalidValue;
}
cudaError_t ising16_gates_launch(const Gate16Args& a, bool f32, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (f32) ising16_gate_kernel<16, float><<<a.count, 512, 0, st>>>(a);
    else ising16_gate_kernel<16, double><<<a.count, 512, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gtqa
