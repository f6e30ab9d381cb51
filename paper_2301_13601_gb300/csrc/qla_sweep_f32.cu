// FP32 instantiations of the fused sweep (K = 1, 2, 4 steps per HBM pass).
#include "qla_sweep.cuh"

namespace qla {

// (K, rows per iteration R, column pipelines per thread NY): shared memory is
// 112 KB for K = 1, 2 (two CTAs per SM) and 224 KB for K = 4.
cudaError_t launch_sweep_f32(int K, const SweepArgs &a, int nfam, cudaStream_t st) {
    switch (K) {
        case 1: return launch_sweep_modes<float, 1, 8, 1>(a, nfam, st);
        case 2: return launch_sweep_modes<float, 2, 4, 2>(a, nfam, st);
        case 4: return launch_sweep_modes<float, 4, 4, 2>(a, nfam, st);
        default: return cudaErrorInvalidValue;
    }
}

int sweep_strip_width() { return W_IN; }

bool sweep_supported(int precision, int K) {
    if (precision == 0) return K == 1 || K == 2 || K == 4;
    return K == 1 || K == 2;
}

int sweep_block_rows(int precision, int K) {
    if (precision == 0) return K == 1 ? 8 : 4;  // the FP32 instantiations above
    return 4;                                   // FP64 (qla_sweep_f64.cu)
}

SweepSplit make_sweep_split(int Nx, int Ny, int K, int R, int tma) {
    SweepSplit s;
    s.Nx = Nx;
    s.Ny = Ny;
    s.w_valid = W_IN - 8 * K;
    // seam layout: the seam strip, then strips over the Nx - W_IN + 8K columns between
    s.seam = tma && Nx % 8 == 0 && Nx >= W_IN && K >= 2 ? 1 : 0;
    s.nsx = s.seam ? 1 + (Nx - W_IN + 8 * K + s.w_valid - 1) / s.w_valid : (Nx + s.w_valid - 1) / s.w_valid;
    s.warm = 8 * K + R * (K - 1);
    return s;
}

int sweep_occupancy_f32(int K, int interleaved) {
    switch (K) {
        case 1: return occupancy_modes<float, 1, 8, 1>(interleaved);
        case 2: return occupancy_modes<float, 2, 4, 2>(interleaved);
        case 4: return occupancy_modes<float, 4, 4, 2>(interleaved);
        default: return 1;
    }
}

}  // namespace qla
