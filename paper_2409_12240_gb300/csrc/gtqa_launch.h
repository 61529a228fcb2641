// Host-side launchers of the annealing kernels.  One translation unit per
// (precision mode, phase kernel) so the six instantiation sets compile in parallel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gtqa_anneal.cuh"
#include "gtqa_general.cuh"
#include "gtqa_plain.cuh"
#include <algorithm>

namespace gtqa {

enum PhaseKernel { PK_GATES = 0, PK_BP = 1, PK_REGAUGE = 2, PK_COUNT = 3 };

// Shared memory the BP kernel keeps per instance after its fixed part: three int flags
// (padded to 8 bytes), two FP64 thresholds and one float threshold.
inline size_t bp_instance_smem(long long B) { return (12 * (size_t)B + 7) / 8 * 8 + 20 * (size_t)B; }

#define GTQA_DECLARE_PHASE(MODE, PHASE)                                                                 \
    bool PHASE##_##MODE##_shape(int CHI, size_t* smem_base, int* tpb);                                  \
    cudaError_t PHASE##_##MODE##_prepare(int CHI, size_t smem, int* blocks_per_sm);                      \
    cudaError_t PHASE##_##MODE##_launch(int CHI, const Ctx& c, size_t smem, cudaStream_t st);
GTQA_DECLARE_PHASE(fp64, gates)
GTQA_DECLARE_PHASE(fp64, bp)
GTQA_DECLARE_PHASE(fp64, regauge)
GTQA_DECLARE_PHASE(mixed, gates)
GTQA_DECLARE_PHASE(mixed, bp)
GTQA_DECLARE_PHASE(mixed, regauge)
#undef GTQA_DECLARE_PHASE

cudaError_t sample_launch_fp64(int CHI, void* Gamma, const double* lam, const int4* vert_edges, int a, double u,
                               int step, int8_t* x, double* p, cudaStream_t st);
cudaError_t sample_launch_mixed(int CHI, void* Gamma, const double* lam, const int4* vert_edges, int a, double u,
                                int step, int8_t* x, double* p, cudaStream_t st);
cudaError_t residual_launch_fp64(int CHI, const void* Gamma, const double* lam, const int4* vert_edges, int n,
                                 double* out, cudaStream_t st);
cudaError_t residual_launch_mixed(int CHI, const void* Gamma, const double* lam, const int4* vert_edges, int n,
                                  double* out, cudaStream_t st);
cudaError_t marginals_launch_fp64(int CHI, const void* Gamma, const double* lam, const int4* vert_edges, int n,
                                  cd* rho, int8_t* sign, int* flag, cudaStream_t st);
cudaError_t marginals_launch_mixed(int CHI, const void* Gamma, const double* lam, const int4* vert_edges, int n,
                                   cd* rho, int8_t* sign, int* flag, cudaStream_t st);

cudaError_t general_gates_launch_fp64(int CHI, const GenArgs& a, cudaStream_t st);
cudaError_t general_gates_launch_mixed(int CHI, const GenArgs& a, cudaStream_t st);
cudaError_t single_gates_launch_fp64(int CHI, void* Gamma, const int* vertex, const cd* W, int count, cudaStream_t st);
cudaError_t single_gates_launch_mixed(int CHI, void* Gamma, const int* vertex, const cd* W, int count,
                                      cudaStream_t st);

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

inline bool phase_shape(bool mixed, int pk, int CHI, size_t* sb, int* tpb) {
    switch (pk) {
        case PK_GATES: return mixed ? gates_mixed_shape(CHI, sb, tpb) : gates_fp64_shape(CHI, sb, tpb);
        case PK_BP: return mixed ? bp_mixed_shape(CHI, sb, tpb) : bp_fp64_shape(CHI, sb, tpb);
        default: return mixed ? regauge_mixed_shape(CHI, sb, tpb) : regauge_fp64_shape(CHI, sb, tpb);
    }
}
inline cudaError_t phase_prepare(bool mixed, int pk, int CHI, size_t smem, int* bps) {
    switch (pk) {
        case PK_GATES: return mixed ? gates_mixed_prepare(CHI, smem, bps) : gates_fp64_prepare(CHI, smem, bps);
        case PK_BP: return mixed ? bp_mixed_prepare(CHI, smem, bps) : bp_fp64_prepare(CHI, smem, bps);
        default: return mixed ? regauge_mixed_prepare(CHI, smem, bps) : regauge_fp64_prepare(CHI, smem, bps);
    }
}
inline cudaError_t phase_launch(bool mixed, int pk, int CHI, const Ctx& c, size_t smem, cudaStream_t st) {
    switch (pk) {
        case PK_GATES: return mixed ? gates_mixed_launch(CHI, c, smem, st) : gates_fp64_launch(CHI, c, smem, st);
        case PK_BP: return mixed ? bp_mixed_launch(CHI, c, smem, st) : bp_fp64_launch(CHI, c, smem, st);
        default: return mixed ? regauge_mixed_launch(CHI, c, smem, st) : regauge_fp64_launch(CHI, c, smem, st);
    }
}

}  // namespace gtqa
