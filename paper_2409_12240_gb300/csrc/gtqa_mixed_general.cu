// Arbitrary-gate kernel instantiations, mixed mode.
#include "gtqa_launch.h"

namespace gtqa {

cudaError_t general_gates_launch_mixed(int CHI, const GenArgs& a, cudaStream_t st) {
    switch (CHI) {
        case 2: return general_gates_launch_t<2, 3, ModeMixed>(a, st);
        case 4: return general_gates_launch_t<4, 3, ModeMixed>(a, st);
        case 8: return general_gates_launch_t<8, 3, ModeMixed>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t single_gates_launch_mixed(int CHI, void* Gamma, const int* vertex, const cd* W, int count,
                                      cudaStream_t st) {
    switch (CHI) {
        case 2: return single_gates_launch_t<2, 3, ModeMixed>(Gamma, vertex, W, count, st);
        case 4: return single_gates_launch_t<4, 3, ModeMixed>(Gamma, vertex, W, count, st);
        case 8: return single_gates_launch_t<8, 3, ModeMixed>(Gamma, vertex, W, count, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gtqa
