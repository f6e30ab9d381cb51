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

int sweep_block_rows(int precision, int K) {
    if (precision == 0) return K == 1 ? 8 : 4;  // the FP32 instantiations above
    return 4;                                   // FP64 (qla_sweep_f64.cu)
}

// Cost of a row of a strip that copies with cp.async, in sixteenths of a row
// of a TMA strip: measured on GB300 by the throughput of the balanced split
// (site-updates/s) against the weight. 8192^2, K = 2: 54.5 G at 16, 62.9 G at
// 20, 74.0 G at 26, 80.3 G at 32, 79.6 G at 40, 77.2 G at 48. K = 4 (one CTA
// per SM): 4096^2 45.5 G at 16, 55.3 G at 26, 54.1 G at 32, 51.7 G at 40;
// 2048^2 40.3 G at 26, 39.0 G at 32.
static int slow_strip_row_cost(int K) { return K >= 4 ? 26 : 32; }

SweepSplit make_sweep_split(int Nx, int Ny, int K, int R, int fp32) {
    SweepSplit s;
    s.Nx = Nx;
    s.Ny = Ny;
    s.w_in = W_IN;
    s.w_valid = W_IN - 8 * K;
    s.nsx = (Nx + s.w_valid - 1) / s.w_valid;
    s.warm = 8 * K + R * (K - 1);
    s.w_slow = slow_strip_row_cost(K);
    s.tma = fp32 && Nx % 8 == 0 ? 1 : 0;
    s.cost_total = 0;
    for (int i = 0; i < s.nsx; ++i) s.cost_total += s.strip_cost(i);
    return s;
}

bool sweep_supported(int precision, int K) {
    if (precision == 0) return K == 1 || K == 2 || K == 4;
    return K == 1 || K == 2;
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
