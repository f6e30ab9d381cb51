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

// Balanced-split weights, measured on GB300 (8192^2, 2 steps per pass, two
// CTAs per SM; per-CTA start and end times by globaltimer, equal shares): the
// seam strip's shares ran 1.10x (TM) and 1.19x (TE) as long per row as the
// others; the first 152 TM CTAs (one per SM) 731.7 us against 806.9 us for
// the second 152; the TE CTAs started over 256 us as the TM CTAs finished.
// Throughput against the weights (G site-updates/s): equal shares 80.5; seam
// rows 18, 19: 81.2; + older 3: 81.3; + start-order slope 6: 83.7, 8: 83.1,
// 11: 82.3, 16: 80.9; older 5 with slope 8: 82.7.
constexpr int kSeamRowCost[2] = {18, 19};  // sixteenths, TM, TE
constexpr int kOlderShare64 = 3;           // profile 1
constexpr int kStartOrderSlope64 = 6;      // profile 2

SweepSplit make_sweep_split(int Nx, int Ny, int K, int R, int tma, int fam, int layer, int layers) {
    SweepSplit s;
    s.Nx = Nx;
    s.Ny = Ny;
    s.w_valid = W_IN - 8 * K;
    // seam layout: the seam strip, then strips over the Nx - W_IN + 8K columns between
    s.seam = tma && Nx % 8 == 0 && Nx >= W_IN && K >= 2 ? 1 : 0;
    s.nsx = s.seam ? 1 + (Nx - W_IN + 8 * K + s.w_valid - 1) / s.w_valid : (Nx + s.w_valid - 1) / s.w_valid;
    s.warm = 8 * K + R * (K - 1);
    s.w_seam = kSeamRowCost[fam ? 1 : 0];
    s.profile = layers == 2 && layer == 1 ? 2 : 1;
    s.p64 = s.profile == 2 ? kStartOrderSlope64 : kOlderShare64;
    s.K = K;
    s.R = R;
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
