// Internal declarations shared by the CUDA translation units of libqla.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qla.h"

namespace qla {

// Coefficient pair planes: NPAIR planes of [Ny][Nx] pairs, element type =
// state precision. The angle a is a collision angle (Eq. 24) or an effective
// potential angle b (Eq. 25, scaled by 1/2 when interleaved (Eq. 28) and by
// 1/2 again for the unitary potentials).
// A collision pair is (x = tan(a/2), y = sin(a)) in FP32 with the printed
// potentials (three-shear form) and (x = cos(a) - 1, y = sin(a)) otherwise; a
// potential pair is (cos(b) - 1, sin(b)). FP32 pairs of the (cos - 1, sin)
// form that are rotations (collisions and the unitary potentials) are tuned
// for orthogonality. Signs of the operators are applied by the kernels.
// The order puts the two planes that the sweep copies together next to each
// other: (V_X, C_X) for the x-pass and (C_Y, V_Y) for the y-pass of a family.
enum CoefPair {
    P_TM_VX = 0,  // beta_2 (V_X row q4)
    P_TM_C = 1,   // theta_2 (x and y collisions of the TM family)
    P_TM_VY = 2,  // beta_3 (V_Y row q3)
    P_TE_VX = 3,  // beta_0 (V_X row q5)
    P_TE_CX = 4,  // theta_1 (C_X pair q1, q5)
    P_TE_CY = 5,  // theta_0 (C_Y pair q0, q5)
    P_TE_VY = 6,  // beta_1 (V_Y row q5)
    NPAIR = 7
};
constexpr int NCOEF = 2 * NPAIR;  // scalars per site

// The six components split into two families that never couple (every
// operator of Eq. 17-22 acts inside one of them):
//   TM: hub q2, x-partner q4, y-partner q3   (E_z polarisation)
//   TE: hub q5, x-partner q1, y-partner q0   (E_y polarisation)
// In both families the first streaming group (S_14 along x, S_03 along y)
// moves the partner and the second (S_25) moves the hub.
struct Family {
    int h, px, py;            // state planes
    int cx, cy, vx, vy;       // coefficient pair planes
    float sgx, sgy;           // collision orientation: C is h' = h + (m h + sg sin p)
    float tx, ty;             // potential orientation: target' = ... + t sin source
    int vx_hub, vy_hub;       // 1 if the potential row targets the hub, 0 if the partner
};

// Strips and balanced split of a pass. The row units u = strip * Ny + y of
// a family (nsx strips, Ny rows each) are shared among the G CTAs of the
// family's grid layer in shares of estimated cost; a CTA sweeps its units as
// one segment per strip it touches. Cost, in sixteenths of a row: 16 per row
// (w_seam per row of the seam strip, which issues more TMA copies: its state
// and coefficient boxes are two-half views and its coefficient levels come in
// separate boxes) and 16 * warm at each strip's start (the warm-up rows a
// segment that starts there sweeps in addition). Without the seam layout
// (FP64; FP32 with K = 1, Nx not a multiple of 8, or Nx < W_IN) no strip copies
// with TMA and every row costs the same. Share sizes (profile):
//   0: equal;
//   1: (G even) shares b < G/2 larger by p64/64 and the others smaller by as
//      much: the first G/2 CTAs of a launch are the first on their SMs, and
//      the warp schedulers favour the older of two resident CTAs;
//   2: decreasing linearly from 1 + p64/64 to 1 - p64/64 times the mean, taken
//      in the order the CTAs start (the last family layer of a launch: its
//      CTAs start as the previous layer's finish, over a spread of times).
struct SweepSplit {
    int Nx, Ny;
    int w_valid;  // output columns per strip
    int nsx;      // strips
    int warm;     // warm-up rows of a segment: 8K + R (K - 1)
    int seam;     // the seam layout (SweepArgs::seam)
    int w_seam;   // cost of a row of the seam strip (sixteenths)
    int profile;  // share sizes (above)
    int p64;
    int K, R;     // steps per pass, rows per iteration

    __host__ __device__ long long strip0_cost() const {
        return 16LL * warm + (long long)(seam ? w_seam : 16) * Ny;
    }
    __host__ __device__ long long cost_total() const {
        return strip0_cost() + (long long)(nsx - 1) * 16 * (Ny + warm);
    }
    // The row unit at cost position c (0 <= c <= cost_total(); a position
    // inside a strip's warm-up maps to the strip's first row): monotonic, so
    // shares [unit(c_b), unit(c_{b+1})) for increasing c_b tile the nsx * Ny
    // units exactly.
    __host__ __device__ long long unit_of_cost(long long c) const {
        const long long c0 = strip0_cost();
        if (c < c0) {
            const long long r = c - 16LL * warm;
            return r <= 0 ? 0 : r / (seam ? w_seam : 16);
        }
        const long long per = 16LL * (Ny + warm);
        const long long s = 1 + (c - c0) / per;
        if (s >= nsx) return (long long)nsx * Ny;
        const long long r = c - c0 - (s - 1) * per - 16LL * warm;  // cost into strip s's rows
        return s * Ny + (r <= 0 ? 0 : r / 16);
    }
    // Cost position where share b of G begins (the profile's weights summed
    // over the shares before b, as a fraction num / den of the total).
    __host__ __device__ long long share_begin(int b, int G) const {
        long long num = b, den = G;
        if (profile == 1 && G % 2 == 0 && G <= 4096) {
            const long long H = G / 2;
            num = b <= H ? b * (64LL + p64) : H * (64LL + p64) + (b - H) * (64LL - p64);
            den = 64LL * G;
        } else if (profile == 2 && G >= 2 && G <= 4096) {
            num = 64LL * (G - 1) * b + (long long)p64 * b * (G - b);
            den = 64LL * G * (G - 1);
        }
        return unit_of_cost(cost_total() / den * num + cost_total() % den * num / den);
    }

    // Columns of strip s, as circular intervals mod Nx: it reads w_in columns
    // from *rd (its halo of 4K columns either side included) and writes *ow
    // columns from *o0 (the sweep kernel's strip geometry, SweepArgs::seam).
    __host__ __device__ void strip_cols(int s, int w_in, int *rd, int *o0, int *ow) const {
        const int h = 4 * K;
        int r, o, w;
        if (!seam) {
            o = s * w_valid;
            w = Nx - o < w_valid ? Nx - o : w_valid;
            r = o - h;
        } else if (s == 0) {
            r = Nx - w_in / 2;
            o = r + h;
            w = w_in - 2 * h;
        } else {
            o = w_in / 2 - h + (s - 1) * w_valid;
            const int hi = Nx - w_in / 2 + h;
            w = (o + w_valid < hi ? o + w_valid : hi) - o;
            r = o - h < Nx - w_in ? o - h : Nx - w_in;
        }
        *rd = ((r % Nx) + Nx) % Nx;
        *o0 = ((o % Nx) + Nx) % Nx;
        *ow = w;
    }
    // Whether [a, a + la) and [b, b + lb) meet on a circle of n points
    // (0 <= a, b < n; la, lb >= 1; a length >= n is the whole circle).
    __host__ __device__ static bool circ_meet(int a, int la, int b, int lb, int n) {
        if (la >= n || lb >= n) return true;
        const int ba = b >= a ? b - a : b - a + n;
        const int ab = a >= b ? a - b : a - b + n;
        return ba < la || ab < lb;
    }
    // Whether the shares of units [b0, b1) and [d0, d1) of consecutive passes
    // must be ordered: one writes a cell that the other reads (on the same
    // state buffer, the later pass's read after the earlier pass's write, or
    // its write after the earlier pass's read). A segment writes rows
    // [y0, y1) of its strip's output columns and reads rows [y0 - 4K,
    // y1 + 4K + R - 1) of its input columns (level 0 is fed from y0 - 4K and
    // its last R-row block starts at y1 + 4K - 1 at the latest); both
    // directions are covered by rows [y0 - 4K - R, y1 + 4K + R) against the
    // other's rows, and input columns against output columns either way.
    __host__ __device__ bool shares_touch(long long b0, long long b1, long long d0, long long d1, int w_in) const {
        for (long long u = b0; u < b1;) {
            const int s = int(u / Ny);
            const int y0 = int(u - (long long)s * Ny);
            const int y1 = (long long)(Ny - y0) < b1 - u ? Ny : y0 + int(b1 - u);
            u += y1 - y0;
            int rs, os, ws;
            strip_cols(s, w_in, &rs, &os, &ws);
            const int wl = y1 - y0 + 8 * K + 2 * R;
            const int ws0 = (((y0 - 4 * K - R) % Ny) + Ny) % Ny;
            for (long long v = d0; v < d1;) {
                const int t = int(v / Ny);
                const int z0 = int(v - (long long)t * Ny);
                const int z1 = (long long)(Ny - z0) < d1 - v ? Ny : z0 + int(d1 - v);
                v += z1 - z0;
                if (!circ_meet(ws0, wl, z0, z1 - z0, Ny)) continue;
                int rt, ot, wt;
                strip_cols(t, w_in, &rt, &ot, &wt);
                if (circ_meet(rs, w_in, ot, wt, Nx) || circ_meet(rt, w_in, os, ws, Nx)) return true;
            }
        }
        return false;
    }
};

// The strips and split of one family layer of a pass of K steps (R rows per
// iteration) over an Nx x Ny lattice; tma: the pass may copy with TMA (FP32
// with its tensor maps); fam: the layer's family (0 = TM, 1 = TE); layer,
// layers: the layer's index and the pass's number of family layers (1, 2).
SweepSplit make_sweep_split(int Nx, int Ny, int K, int R, int tma, int fam = 0, int layer = 0, int layers = 1);
// Rows per iteration R of the sweep instantiated for (precision, K).
int sweep_block_rows(int precision, int K);

struct SweepArgs {
    const void *q_in;   // [6][Ny][Nx]
    void *q_out;        // [6][Ny][Nx]
    const void *coef;   // [NCOEF][Ny][Nx]
    int Nx, Ny;
    int w_valid;        // output columns per strip
    int chunk;          // output rows per tile (tiled grid); 0: balanced split over `ctas` CTAs per family
    int ctas;           // balanced split: CTAs per family
    // Strip layout. 0: strip s reads input columns [s w_valid - 4K, + W_IN)
    // (the first and the last strip wrap around x). 1 (the seam layout, FP32
    // with TMA, Nx >= W_IN, a multiple of 8): strip 0 straddles the periodic
    // seam, reading columns [Nx - W_IN/2, Nx) and [0, W_IN/2) and writing the
    // w_valid in their middle; strips s >= 1 cover the outputs between,
    // strip s from column W_IN/2 - 4K + (s - 1) w_valid, the last one's input
    // moved left to end at Nx at the latest (it writes only its own columns).
    int seam;
    // Balanced split, last of two family layers: a counter (zero between
    // launches) from which the layer's CTAs take their share index in the
    // order they start; null: share = blockIdx.x.
    unsigned *order;
    int interleaved;    // 1: Eq. 28, 0: Eq. 23
    int unitary;        // 1: unitary potentials
    int vec;            // 1: 16-byte vector access is legal (Nx multiple of 16/sizeof(T))
    int fam0;           // first family index handled by blockIdx.z = 0 (0 = TM, 1 = TE)
    int *error;         // device flag set when a bounded wait of the TMA copy path runs out (null: no TMA)
};

// Sweep kernel launcher: one fused pass of K time steps over the lattice.
// Returns cudaSuccess or the launch error.
cudaError_t launch_sweep_f32(int K, const SweepArgs &a, int nfam, cudaStream_t st);
cudaError_t launch_sweep_f64(int K, const SweepArgs &a, int nfam, cudaStream_t st);
bool sweep_supported(int precision, int K);
// Persistent form of the balanced split (qla_sweep_persist.cu): `passes`
// passes of K steps in one cooperative launch of a.ctas CTAs (at most
// kPersistMaxCtas), CTA b sweeping share b of each of the nfam families in
// turn, ordered by the per-share pass counters done[nfam][a.ctas] (their
// values before the launch all <= base). FP32 with tensor maps and the seam
// layout only: cudaErrorNotSupported otherwise.
constexpr int kPersistMaxCtas = 4096;
cudaError_t launch_sweep_persistent_f32(int K, const SweepArgs &a, int nfam, int passes, unsigned base,
                                        unsigned *done, cudaStream_t st);
bool sweep_persistent_supported(int precision, int K);
int sweep_strip_width();  // input columns per strip (halo included)
int sweep_occupancy_f32(int K, int interleaved);  // resident CTAs per SM
int sweep_occupancy_f64(int K, int interleaved);

// Coefficients (Eq. 24-25) from the device index planes n[3][Ny][Nx] (double).
cudaError_t launch_coefficients(const double *n, void *coef, int Nx, int Ny, double delta,
                                int precision, int interleaved, int unitary, cudaStream_t st);
// Pulse initial condition into state (precision-typed) [6][Ny][Nx].
cudaError_t launch_init_pulse(void *q, int Nx, int Ny, int precision, int pol, double x0,
                              double sigma, double amp, cudaStream_t st);
// Conversions between a double/float staging buffer and the state.
cudaError_t launch_convert(const void *src, int src_double, void *dst, int dst_double, size_t n,
                           cudaStream_t st);

// Diagnostics: partial reductions into scratch, then a single-block final pass.
struct DiagResult {
    double energy_sum;   // sum over sites of Q.Q
    double div_sq_sum;
    double div_max;
    double b_max;
    unsigned long long nonfinite;
    unsigned long long pad[3];
};
int diag_blocks(int Nx, int Ny);
size_t diag_scratch_bytes(int Nx, int Ny);
cudaError_t launch_diagnostics(const void *q, int precision, int Nx, int Ny, void *scratch,
                               DiagResult *out_dev, cudaStream_t st);
// div D statistics in the DiagResult fields div_sq_sum, div_max and b_max
// (= max |D|); index: the FP64 fields n_x, n_y, n_z [3][Ny][Nx].
cudaError_t launch_divD(const void *q, int precision, const double *index, int Nx, int Ny, void *scratch,
                        DiagResult *out_dev, cudaStream_t st);


// ---------------------------------------------------------------------------
// Surrogate building blocks (BF16 tensor-core convolution and friends).
// ---------------------------------------------------------------------------
struct ConvArgs {
    const void *x;        // BF16 [nimg][H][W][cin]
    const void *w;        // BF16 packed [9][cin/8][nout][8]
    const float *bias;    // [nout] or null
    int nimg, H, W;       // images of H x W (each periodic)
    int epi;              // QLA_EPI_*
    const void *aux0;     // GELU: BF16 residual or null; DGRAD: FP32 g_in or null; QUPDATE: FP32 q_in [nimg][6][H][W]
    const void *zprev;    // DGRAD: BF16 pre-activation [nimg][H][W][nout]
    void *out0;           // GELU: BF16 z or null; LINEAR: FP32; DGRAD: FP32 g; QUPDATE: FP32 q_out [nimg][6][H][W]
    void *out1;           // GELU: BF16 activation; DGRAD: BF16 dz
    float scale;          // QUPDATE
    int *error;           // set to 1 when a bounded wait runs out
};
// Supported (cin, nout): (16, 64), (64, 64), (64, 16).
bool conv_supported(int cin, int nout);
cudaError_t launch_conv(int cin, int nout, const ConvArgs &a, cudaStream_t st);

// Weight gradient of a 3x3 circular conv on the tensor cores: per-CTA partial
// sums part[cta][9][nt][64] of sum_p g[p][n] x[p + tap][c]; x BF16 [..][cs]
// (cs = 16 or 64), g BF16 [..][nt] (nt = 64 or 16). *grid_out = CTAs used.
struct WgradArgs {
    const void *x;
    int cs;
    const void *g;
    int nt;
    int nimg, H, W;
    float *part;
    int *error;
};
int wgrad_grid(const WgradArgs &a);
cudaError_t launch_wgrad_tc(const WgradArgs &a, int *grid_out, cudaStream_t st);

// Weight packing modes: plain, adjoint (transpose + 180-degree flip), and
// plain with the input channels of the surrogate's first layer
// (packed c: 0-5 -> logical c, 6-11 -> logical c-6, 12-14 -> logical c-6, 15 -> 0).
enum PackMode { PACK_PLAIN = 0, PACK_ADJOINT = 1, PACK_TIED_INPUT = 2 };
cudaError_t launch_pack_weights(const float *w, int nout, int cin, int nout_pad, int cin_pad, int mode,
                                void *packed, cudaStream_t st);

// One operator of the step (qla_debug_apply), in place on `state` or, for a
// streaming op, from `state` into `spare` (*swapped set).
cudaError_t debug_apply(int op, int precision, void *state, void *spare, const void *coef, int Nx, int Ny, int unitary,
                        cudaStream_t st, bool *swapped);

}  // namespace qla

// Access to a QLA context from other parts of the library (the surrogate
// rollout advances a context's state and hands steps back to it).
namespace qla {
struct CtxView {
    int Nx, Ny, precision;
    cudaStream_t stream;
    void *cur_state;     // current state [6][Ny][Nx]
    void *spare_state;   // the other state buffer (free between steps)
    int has_state;
    int families;        // QLA_FAMILIES_BOTH, QLA_FAMILY_TM or QLA_FAMILY_TE
};
bool ctx_view(qla_ctx *c, CtxView *v);
// The spare buffer, now holding the state `steps` steps later, becomes current.
void ctx_commit_spare(qla_ctx *c, long long steps);
// The current buffer was advanced in place by `steps` steps (step count only).
void ctx_add_steps(qla_ctx *c, long long steps);
}  // namespace qla

