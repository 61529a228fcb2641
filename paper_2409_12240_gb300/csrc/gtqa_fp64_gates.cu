// gates kernel instantiations, fp64 precision mode.
#include "gtqa_launch.h"

namespace gtqa {

namespace {
template <int CHI>
cudaError_t launch_t(const Ctx& c, size_t smem, cudaStream_t st) {
    Ctx copy = c;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)gates_kernel<CHI, ModeFP64>, dim3(c.nblocks), dim3(Shape<CHI>::TPB), args,
                                       smem, st);
}
template <int CHI>
cudaError_t prepare_t(size_t smem, int* bps) {
    cudaError_t e = raise_smem_limit(gates_kernel<CHI, ModeFP64>, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, gates_kernel<CHI, ModeFP64>, Shape<CHI>::TPB, smem);
}
}  // namespace

bool gates_fp64_shape(int CHI, size_t* smem_base, int* tpb) {
    switch (CHI) {
        case 2: *smem_base = SmemSize<2, ModeFP64, PH_GATES>::value; *tpb = Shape<2>::TPB; return true;
        case 4: *smem_base = SmemSize<4, ModeFP64, PH_GATES>::value; *tpb = Shape<4>::TPB; return true;
        case 8: *smem_base = SmemSize<8, ModeFP64, PH_GATES>::value; *tpb = Shape<8>::TPB; return true;
        default: return false;
    }
}

cudaError_t gates_fp64_prepare(int CHI, size_t smem, int* bps) {
    switch (CHI) {
        case 2: return prepare_t<2>(smem, bps);
        case 4: return prepare_t<4>(smem, bps);
        case 8: return prepare_t<8>(smem, bps);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t gates_fp64_launch(int CHI, const Ctx& c, size_t smem, cudaStream_t st) {
    switch (CHI) {
        case 2: return launch_t<2>(c, smem, st);
        case 4: return launch_t<4>(c, smem, st);
        case 8: return launch_t<8>(c, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int CHI>
cudaError_t marg_t(const void* G, const double* lam, const int4* ve, int n, cd* rho, int8_t* sign, int* flag,
                   cudaStream_t st) {
    const int wpb = 4;
    marginals_kernel2<CHI, ModeFP64><<<(n + wpb - 1) / wpb, 32 * wpb, 0, st>>>((const C<typename ModeFP64::TS>*)G, lam, ve, n,
                                                                             rho, sign, flag);
    return cudaGetLastError();
}
}  // namespace

cudaError_t marginals_launch_fp64(int CHI, const void* G, const double* lam, const int4* ve, int n, cd* rho,
                                     int8_t* sign, int* flag, cudaStream_t st) {
    switch (CHI) {
        case 2: return marg_t<2>(G, lam, ve, n, rho, sign, flag, st);
        case 4: return marg_t<4>(G, lam, ve, n, rho, sign, flag, st);
        case 8: return marg_t<8>(G, lam, ve, n, rho, sign, flag, st);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int CHI>
cudaError_t resid_t(const void* G, const double* lam, const int4* ve, int n, double* out, cudaStream_t st) {
    const int wpb = 8;
    residual_kernel<CHI, ModeFP64><<<(3 * n + wpb - 1) / wpb, 32 * wpb, 0, st>>>((const C<typename ModeFP64::TS>*)G, lam, ve, n, out);
    return cudaGetLastError();
}
}  // namespace

cudaError_t residual_launch_fp64(int CHI, const void* G, const double* lam, const int4* ve, int n, double* out,
                                  cudaStream_t st) {
    switch (CHI) {
        case 2: return resid_t<2>(G, lam, ve, n, out, st);
        case 4: return resid_t<4>(G, lam, ve, n, out, st);
        case 8: return resid_t<8>(G, lam, ve, n, out, st);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int CHI>
cudaError_t sample_t(void* G, const double* lam, const int4* ve, int a, double u, int step, int8_t* x, double* p,
                     cudaStream_t st) {
    sample_kernel<CHI, ModeFP64><<<1, 32, 0, st>>>((C<typename ModeFP64::TS>*)G, lam, ve, a, u, step, x, p);
    return cudaGetLastError();
}
}  // namespace

cudaError_t sample_launch_fp64(int CHI, void* G, const double* lam, const int4* ve, int a, double u, int step,
                                int8_t* x, double* p, cudaStream_t st) {
    switch (CHI) {
        case 2: return sample_t<2>(G, lam, ve, a, u, step, x, p, st);
        case 4: return sample_t<4>(G, lam, ve, a, u, step, x, p, st);
        case 8: return sample_t<8>(G, lam, ve, a, u, step, x, p, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gtqa
