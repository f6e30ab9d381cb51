// FP32 instantiations of the fused sweep (K = 1, 2, 4 steps per HBM pass).
#include "qla_sweep.cuh"

namespace qla {

cudaError_t launch_sweep_f32(int K, const SweepArgs &a, int nfam, cudaStream_t st) {
    switch (K) {
        case 1: return launch_sweep_t<float, 1, 1, 8>(a, nfam, st);
        case 2: return launch_sweep_t<float, 2, 1, 8>(a, nfam, st);
        case 4: return launch_sweep_t<float, 4, 2, 8>(a, nfam, st);
        default: return cudaErrorInvalidValue;
    }
}

int sweep_strip_width() { return W_IN; }

int sweep_occupancy_f32(int K) {
    switch (K) {
        case 1: return occupancy_t<float, 1, 1, 8>();
        case 2: return occupancy_t<float, 2, 1, 8>();
        case 4: return occupancy_t<float, 4, 2, 8>();
        default: return 1;
    }
}

bool sweep_supported(int precision, int K) {
    if (precision == 0) return K == 1 || K == 2 || K == 4;
    return K == 1 || K == 2;
}

}  // namespace qla
