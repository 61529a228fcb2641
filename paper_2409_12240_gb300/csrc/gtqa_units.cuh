// Definitions of the launcher units declared in gtqa_launch.h.  Included only by
// gtqa_units.cu, whose explicit instantiations place each (mode, phase) set of kernel
// instantiations in its own object file.
#pragma once

#include <type_traits>

#include "gtqa_launch.h"

namespace gtqa {

// Calls f with the storage bond dimension of the persistent kernels as a compile-time
// constant (2, 4 or 8); any other value is rejected.
template <class R, class F>
R by_chi(int CHI, R bad, F&& f) {
    switch (CHI) {
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default: return bad;
    }
}

constexpr unsigned phase_bits(int PK) { return PK == PK_GATES ? PH_GATES : (PK == PK_BP ? PH_BP : PH_REGAUGE); }

template <int CHI, class Mode, int PK>
constexpr auto phase_kernel() {
    if constexpr (PK == PK_GATES) return gates_kernel<CHI, Mode>;
    else if constexpr (PK == PK_BP) return bp_kernel<CHI, Mode>;
    else return regauge_kernel<CHI, Mode>;
}

template <class Mode, int PK>
bool PhaseUnit<Mode, PK>::shape(int CHI, size_t* smem_base, int* tpb) {
    return by_chi(CHI, false, [&](auto k) {
        constexpr int X = decltype(k)::value;
        *smem_base = SmemSize<X, Mode, phase_bits(PK)>::value;
        *tpb = Shape<X>::TPB;
        return true;
    });
}

template <class Mode, int PK>
cudaError_t PhaseUnit<Mode, PK>::prepare(int CHI, size_t smem, int* bps) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value;
        const cudaError_t e = raise_smem_limit(phase_kernel<X, Mode, PK>(), smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, phase_kernel<X, Mode, PK>(), Shape<X>::TPB, smem);
    });
}

template <class Mode, int PK>
cudaError_t PhaseUnit<Mode, PK>::launch(int CHI, const Ctx& c, size_t smem, cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value;
        Ctx copy = c;
        void* args[] = {&copy};
        return cudaLaunchCooperativeKernel((const void*)phase_kernel<X, Mode, PK>(), dim3(c.nblocks),
                                           dim3(Shape<X>::TPB), args, smem, st);
    });
}

template <class Mode>
cudaError_t AuxUnit<Mode>::marginals(int CHI, const void* G, const double* lam, const int4* ve, int n, cd* rho,
                                     int8_t* sign, int* flag, cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value, WPB = 4;
        marginals_kernel2<X, Mode><<<(n + WPB - 1) / WPB, 32 * WPB, 0, st>>>(
            (const C<typename Mode::TS>*)G, lam, ve, n, rho, sign, flag);
        return cudaGetLastError();
    });
}

template <class Mode>
cudaError_t AuxUnit<Mode>::residual(int CHI, const void* G, const double* lam, const int4* ve, int n, double* out,
                                    cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value, WPB = 8;
        residual_kernel<X, Mode><<<(3 * n + WPB - 1) / WPB, 32 * WPB, 0, st>>>((const C<typename Mode::TS>*)G, lam,
                                                                             ve, n, out);
        return cudaGetLastError();
    });
}

template <class Mode>
cudaError_t AuxUnit<Mode>::sample(int CHI, void* G, const double* lam, const int4* ve, int a, double u, int step,
                                  int8_t* x, double* p, cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value;
        sample_kernel<X, Mode><<<1, 32, 0, st>>>((C<typename Mode::TS>*)G, lam, ve, a, u, step, x, p);
        return cudaGetLastError();
    });
}

template <class Mode>
cudaError_t GeneralUnit<Mode>::gates(int CHI, const GenArgs& a, cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        return general_gates_launch_t<decltype(k)::value, 3, Mode>(a, st);
    });
}

template <class Mode>
cudaError_t GeneralUnit<Mode>::single(int CHI, void* Gamma, const int* vertex, const cd* W, int count,
                                      cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        return single_gates_launch_t<decltype(k)::value, 3, Mode>(Gamma, vertex, W, count, st);
    });
}

}  // namespace gtqa
