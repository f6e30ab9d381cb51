// FP64 instantiations of the fused sweep (correctness mode; K = 1, 2).
#include "qla_sweep.cuh"

namespace qla {

cudaError_t launch_sweep_f64(int K, const SweepArgs &a, int nfam, cudaStream_t st) {
    switch (K) {
        case 1: return launch_sweep_modes<double, 1, 4, 1>(a, nfam, st);
        case 2: return launch_sweep_modes<double, 2, 4, 2>(a, nfam, st);
        default: return cudaErrorInvalidValue;
    }
}

int sweep_occupancy_f64(int K, int interleaved) {
    switch (K) {
        case 1: return occupancy_modes<double, 1, 4, 1>(interleaved);
        case 2: return occupancy_modes<double, 2, 4, 2>(interleaved);
        default: return 1;
    }
}

}  // namespace qla
