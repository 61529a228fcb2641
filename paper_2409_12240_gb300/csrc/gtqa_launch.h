// Host-side launchers of the annealing kernels and the dispatch on precision mode and
// phase kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gtqa_anneal.cuh"
#include "gtqa_aux.cuh"
#include "gtqa_general.cuh"
#include "gtqa_plain.cuh"
#include <algorithm>

namespace gtqa {

enum PhaseKernel { PK_GATES = 0, PK_BP = 1, PK_REGAUGE = 2, PK_COUNT = 3 };

// Launch-shape variants that differ for a phase kernel: the gates kernel depends on the block
// size only, which its third variant would repeat.
constexpr int shape_count(int pk) { return pk == PK_GATES ? 2 : NSHAPE; }

// Shared memory the BP kernel keeps per instance after its fixed part: three int flags
// (padded to 8 bytes), two FP64 thresholds and one float threshold.
inline size_t bp_instance_smem(long long B) { return (12 * (size_t)B + 7) / 8 * 8 + 20 * (size_t)B; }

// Launchers of the persistent phase kernels of one precision mode.  The definitions
// (gtqa_units.cuh) are compiled only in gtqa_units.cu, which the build compiles once per
// (mode, phase) with an explicit instantiation, so the instantiation sets build in
// parallel; every other unit links against them.
// Every call takes the launch-shape variant v (0 .. shape_count(PK) - 1) besides CHI; shape
// also returns the kernel's team size (gate edge, BP vertex or regauge vertex team).
template <class Mode, int PK>
struct PhaseUnit {
    static bool shape(int CHI, int v, size_t* smem_base, int* tpb, int* team);
    static cudaError_t prepare(int CHI, int v, size_t smem, int* blocks_per_sm);
    static cudaError_t launch(int CHI, int v, const Ctx& c, size_t smem, cudaStream_t st);
};

// Marginals, residual and measurement-sampling kernels of one mode (instantiated in the
// gates unit of that mode).
template <class Mode>
struct AuxUnit {
    static cudaError_t marginals(int CHI, const void* Gamma, const double* lam, const int4* vert_edges, int n, cd* rho,
                                 int8_t* sign, int* flag, cudaStream_t st);
    static cudaError_t residual(int CHI, const void* Gamma, const double* lam, const int4* vert_edges, int n,
                                double* out, cudaStream_t st);
    static cudaError_t sample(int CHI, void* Gamma, const double* lam, const int4* vert_edges, int a, double u,
                              int step, int8_t* x, double* p, cudaStream_t st);
};

// Arbitrary two-qubit and one-qubit gate kernels of one mode (degree 3).
template <class Mode>
struct GeneralUnit {
    static cudaError_t gates(int CHI, const GenArgs& a, cudaStream_t st);
    static cudaError_t single(int CHI, void* Gamma, const int* vertex, const cd* W, int count, cudaStream_t st);
};

// the plain path; pm selects the precision: 0 FP64, 1 mixed (degree 4 with CHI in {2, 4},
// degree 3 with CHI = 16 for both) or 2 complex64 (degree 3 with CHI in {2, 4, 8, 16}, degree 4
// with CHI in {2, 4})
bool plain_supported(int CHI, int D, int pm);
size_t plain_scratch_entries(int CHI, int D, int n, int m);
cudaError_t plain_bp_init_launch(int CHI, int D, int pm, const PlainArgs& a, cudaStream_t st);
cudaError_t plain_bp_sweep_launch(int CHI, int D, int pm, const PlainArgs& a, cudaStream_t st);
cudaError_t plain_regauge_launch(int CHI, int D, int pm, const PlainArgs& a, const void* msg, double eig_cut,
                                 double svd_cut, cudaStream_t st);
cudaError_t plain_marginals_launch(int CHI, int D, int pm, const void* Gamma, const double* lam, const int4* vslots,
                                   int n, cd* rho, int8_t* sign, int* flag, cudaStream_t st);
cudaError_t plain_residual_launch(int CHI, int D, int pm, const void* Gamma, const double* lam, const int4* vslots,
                                  int n, double* out, cudaStream_t st);
cudaError_t plain_sample_launch(int CHI, int D, int pm, void* Gamma, const double* lam, const int4* vslots, int a,
                                double u, int step, int8_t* x, double* p, cudaStream_t st);
cudaError_t plain_general_gates_launch(int CHI, int D, int pm, const GenArgs& a, cudaStream_t st);
cudaError_t plain_single_gates_launch(int CHI, int D, int pm, void* Gamma, const int* vertex, const cd* W, int count,
                                      cudaStream_t st);
cudaError_t ising16_gates_launch(const Gate16Args& a, int pm, cudaStream_t st);

}  // namespace gtqa
