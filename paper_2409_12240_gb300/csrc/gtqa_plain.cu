// Plain-path kernel instantiations.  pm selects the precision: 0 FP64 and 1 mixed (complex64
// storage and contractions; FP64 QR/SVD, gauge roots and normalisation), each for degree 4 with
// CHI in {2, 4} and degree 3 with CHI = 16; 2 the complex64 mode (every step in FP32), for
// degree 3 with CHI in {2, 4, 8, 16} and degree 4 with CHI in {2, 4}.
#include "gtqa_launch.h"

namespace gtqa {

namespace {
template <int CHI, int D, typename R, typename RC>
size_t sweep_smem() {
    using S = PlainShape<CHI, D, R>;
    // the mixed mode adds m0 and delta of the incoming messages
    const int mix = sizeof(R) != sizeof(RC) ? 2 * D * S::CC : 0;
    return sizeof(C<R>) * ((D + 1) * S::CC + (S::SMEM ? 3 * S::H2 : 0) + mix);
}
template <int CHI, int D, typename R>
size_t vertex_smem() {
    using S = PlainShape<CHI, D, R>;
    return sizeof(C<R>) * (D * S::CC + (S::SMEM ? 2 * S::H2 : 0));
}
template <int CHI, int D, typename R, typename RC>
cudaError_t init_t(const PlainArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    plain_bp_init_kernel<CHI, D, R, RC><<<a.n, 256, 0, st>>>(a);
    return cudaGetLastError();
}
template <int CHI, int D, typename R, typename RC>
cudaError_t sweep_t(const PlainArgs& a, cudaStream_t st) {
    using S = PlainShape<CHI, D, R>;
    if (a.n > 0) {
        plain_bp_sweep_kernel<CHI, D, R, RC><<<a.n, S::NT, sweep_smem<CHI, D, R, RC>(), st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.m > 0) plain_trace_norm_kernel<CHI, R, RC><<<2 * a.m, S::CC / 2, 0, st>>>((const C<R>*)a.dm, a.acc);
    return cudaGetLastError();
}
template <int CHI, int D, typename R, typename RC>
cudaError_t regauge_t(const PlainArgs& a, const void* msg, double eig_cut, double svd_cut, cudaStream_t st) {
    using S = PlainShape<CHI, D, R>;
    if (a.m > 0) {
        plain_regauge_edge_kernel<CHI, R, RC><<<a.m, S::CC / 2, 0, st>>>((const C<R>*)msg, a.lam, (C<R>*)a.X,
                                                                         eig_cut, svd_cut);
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

// CALL(CHI, D, R, RC) for every built shape: R the storage and contraction type, RC the type
// of the FP64 steps (normalisation, trace norms, the regauge's eigen and SVD)
#define GTQA_PLAIN_DISPATCH(CALL)                                              \
    if (pm == 0) {                                                             \
        if (D == 4 && CHI == 2) return CALL(2, 4, double, double);             \
        if (D == 4 && CHI == 4) return CALL(4, 4, double, double);             \
        if (D == 3 && CHI == 16) return CALL(16, 3, double, double);           \
    } else if (pm == 1) {                                                      \
        if (D == 4 && CHI == 2) return CALL(2, 4, float, double);              \
        if (D == 4 && CHI == 4) return CALL(4, 4, float, double);              \
        if (D == 3 && CHI == 16) return CALL(16, 3, float, double);            \
    } else {                                                                   \
        if (D == 3 && CHI == 2) return CALL(2, 3, float, float);               \
        if (D == 3 && CHI == 4) return CALL(4, 3, float, float);               \
        if (D == 3 && CHI == 8) return CALL(8, 3, float, float);               \
        if (D == 3 && CHI == 16) return CALL(16, 3, float, float);             \
        if (D == 4 && CHI == 2) return CALL(2, 4, float, float);               \
        if (D == 4 && CHI == 4) return CALL(4, 4, float, float);               \
    }                                                                          \
    return cudaErrorInvalidValue;

bool plain_supported(int CHI, int D, int pm) {
    if (pm != 2) return (D == 4 && (CHI == 2 || CHI == 4)) || (D == 3 && CHI == 16);
    return (D == 3 && (CHI == 2 || CHI == 4 || CHI == 8 || CHI == 16)) || (D == 4 && (CHI == 2 || CHI == 4));
}

size_t plain_scratch_entries(int CHI, int D, int n, int m) {
    // complex entries (sized for complex128; the complex64 mode uses half of each entry)
    if (D == 3 && CHI == 16)
        return std::max((size_t)n * PlainShape<16, 3, double>::scratch_per_block, (size_t)m * 4 * 16 * 256);
    return 0;
}

cudaError_t plain_bp_init_launch(int CHI, int D, int pm, const PlainArgs& a, cudaStream_t st) {
#define C_(c, d, r, rc) init_t<c, d, r, rc>(a, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_bp_sweep_launch(int CHI, int D, int pm, const PlainArgs& a, cudaStream_t st) {
#define C_(c, d, r, rc) sweep_t<c, d, r, rc>(a, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_regauge_launch(int CHI, int D, int pm, const PlainArgs& a, const void* msg, double eig_cut,
                                 double svd_cut, cudaStream_t st) {
#define C_(c, d, r, rc) regauge_t<c, d, r, rc>(a, msg, eig_cut, svd_cut, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_marginals_launch(int CHI, int D, int pm, const void* G, const double* lam, const int4* vs, int n,
                                   cd* rho, int8_t* sign, int* flag, cudaStream_t st) {
#define C_(c, d, r, rc) marg_t<c, d, r>(G, lam, vs, n, rho, sign, flag, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_residual_launch(int CHI, int D, int pm, const void* G, const double* lam, const int4* vs, int n,
                                  double* out, cudaStream_t st) {
#define C_(c, d, r, rc) resid_t<c, d, r>(G, lam, vs, n, out, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_sample_launch(int CHI, int D, int pm, void* G, const double* lam, const int4* vs, int a, double u,
                                int step, int8_t* x, double* p, cudaStream_t st) {
#define C_(c, d, r, rc) sample_t<c, d, r>(G, lam, vs, a, u, step, x, p, st)
    GTQA_PLAIN_DISPATCH(C_)
#undef C_
}
cudaError_t plain_general_gates_launch(int CHI, int D, int pm, const GenArgs& a, cudaStream_t st) {
    if (pm == 0) {
        if (D == 4 && CHI == 2) return general_gates_launch_t<2, 4, ModeFP64>(a, st);
        if (D == 4 && CHI == 4) return general_gates_launch_t<4, 4, ModeFP64>(a, st);
    } else if (pm == 1) {
        if (D == 4 && CHI == 2) return general_gates_launch_t<2, 4, ModeMixed>(a, st);
        if (D == 4 && CHI == 4) return general_gates_launch_t<4, 4, ModeMixed>(a, st);
    } else {
        if (D == 3 && CHI == 2) return general_gates_launch_t<2, 3, ModeC64>(a, st);
        if (D == 3 && CHI == 4) return general_gates_launch_t<4, 3, ModeC64>(a, st);
        if (D == 3 && CHI == 8) return general_gates_launch_t<8, 3, ModeC64>(a, st);
        if (D == 4 && CHI == 2) return general_gates_launch_t<2, 4, ModeC64>(a, st);
        if (D == 4 && CHI == 4) return general_gates_launch_t<4, 4, ModeC64>(a, st);
    }
    return cudaErrorInvalidValue;   // CHI = 16: the whole-side core (64 x 64) exceeds one block's Jacobi
}
cudaError_t plain_single_gates_launch(int CHI, int D, int pm, void* G, const int* v, const cd* W, int count,
                                      cudaStream_t st) {
    if (pm == 0) {
        if (D == 4 && CHI == 2) return single_gates_launch_t<2, 4, ModeFP64>(G, v, W, count, st);
        if (D == 4 && CHI == 4) return single_gates_launch_t<4, 4, ModeFP64>(G, v, W, count, st);
        if (D == 3 && CHI == 16) return single_gates_launch_t<16, 3, ModeFP64>(G, v, W, count, st);
    } else if (pm == 1) {
        if (D == 4 && CHI == 2) return single_gates_launch_t<2, 4, ModeMixed>(G, v, W, count, st);
        if (D == 4 && CHI == 4) return single_gates_launch_t<4, 4, ModeMixed>(G, v, W, count, st);
        if (D == 3 && CHI == 16) return single_gates_launch_t<16, 3, ModeMixed>(G, v, W, count, st);
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
cudaError_t ising16_gates_launch(const Gate16Args& a, int pm, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (pm == 0) ising16_gate_kernel<16, double, double><<<a.count, 512, 0, st>>>(a);
    else if (pm == 1) ising16_gate_kernel<16, float, double><<<a.count, 512, 0, st>>>(a);
    else ising16_gate_kernel<16, float, float><<<a.count, 512, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gtqa
