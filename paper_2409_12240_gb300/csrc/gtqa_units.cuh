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

// Calls f with the launch-shape variant of phase kernel PK as a compile-time constant.
template <int PK, class R, class F>
R by_shape(int v, R bad, F&& f) {
    switch (v) {
        case 0: return f(std::integral_constant<int, 0>{});
        case 1: return f(std::integral_constant<int, 1>{});
        case 2:
            if constexpr (shape_count(PK) > 2) return f(std::integral_constant<int, 2>{});
            else return bad;
        default: return bad;
    }
}

constexpr unsigned phase_bits(int PK) { return PK == PK_GATES ? PH_GATES : (PK == PK_BP ? PH_BP : PH_REGAUGE); }

template <int CHI, class Mode, int PK, int V>
constexpr auto phase_kernel() {
    if constexpr (PK == PK_GATES) return gates_kernel<CHI, Mode, V>;
    else if constexpr (PK == PK_BP) return bp_kernel<CHI, Mode, V>;
    else return regauge_kernel<CHI, Mode, V>;
}

template <class Mode, int PK>
bool PhaseUnit<Mode, PK>::shape(int CHI, int v, size_t* smem_base, int* tpb, int* team) {
    return by_chi(CHI, false, [&](auto k) {
        constexpr int X = decltype(k)::value;
        return by_shape<PK>(v, false, [&](auto w) {
            constexpr int V = decltype(w)::value;
            using S = Shape<X, V>;
            *smem_base = SmemSize<X, Mode, phase_bits(PK), V>::value;
            *tpb = S::TPB;
            if (team) *team = PK == PK_GATES ? S::TG : (PK == PK_BP ? S::TB : S::TRV);
            return true;
        });
    });
}

template <class Mode, int PK>
cudaError_t PhaseUnit<Mode, PK>::prepare(int CHI, int v, size_t smem, int* bps) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value;
        return by_shape<PK>(v, cudaErrorInvalidValue, [&](auto w) {
            constexpr int V = decltype(w)::value;
            const cudaError_t e = raise_smem_limit(phase_kernel<X, Mode, PK, V>(), smem);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, phase_kernel<X, Mode, PK, V>(),
                                                                 Shape<X, V>::TPB, smem);
        });
    });
}

template <class Mode, int PK>
cudaError_t PhaseUnit<Mode, PK>::launch(int CHI, int v, const Ctx& c, size_t smem, cudaStream_t st) {
    return by_chi(CHI, cudaErrorInvalidValue, [&](auto k) {
        constexpr int X = decltype(k)::value;
        return by_shape<PK>(v, cudaErrorInvalidValue, [&](auto w) {
            constexpr int V = decltype(w)::value;
            Ctx copy = c;
            void* args[] = {&copy};
            return cudaLaunchCooperativeKernel((const void*)phase_kernel<X, Mode, PK, V>(), dim3(c.nblocks),
                                               dim3(Shape<X, V>::TPB), args, smem, st);
        });
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
        // WPB warps per block, each taking IPW (vertex, slot) items (as in residual_kernel)
        constexpr int X = decltype(k)::value, WPB = 8, GJ = X * X / 2, IPW = 32 / GJ > 0 ? 32 / GJ : 1;
        const int warps = (3 * n + IPW - 1) / IPW;
        residual_kernel<X, Mode><<<(warps + WPB - 1) / WPB, 32 * WPB, 0, st>>>((const C<typename Mode::TS>*)G, lam,
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
