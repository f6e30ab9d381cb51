// 3x3 convolution with circular padding on BF16 NHWC activations, as an
// implicit GEMM on the tcgen05 tensor cores with FP32 accumulation in TMEM.
//
// Activations hold nimg images of H x W stacked ([nimg][H][W][C]); each image
// is periodic on its own. One tile = 128 consecutive pixels of one image row
// (M = 128), all output channels, K = 9 taps x input channels. Input rows
// (130 pixels with the x halo, CIN channels) are staged once each in the
// interleaved K-major layout, so the three x taps are shifted windows of the
// same row (no swizzle: any 16-byte aligned start is a valid operand). Each
// staged input row is multiplied once per (x tap, 16-channel slice) against
// the weights of all three y taps at once (N = 3 NOUT), accumulating into the
// TMEM accumulators of the three output rows it feeds. All 9 taps of the
// packed weights stay resident in shared memory. One thread issues the MMAs;
// the epilogue warps (32 TMEM lanes each) run the fused epilogue:
//   EPI_GELU      z = acc + b;  act = GELU(z) (+ residual);  stores act and, if asked, z (BF16)
//   EPI_LINEAR    out = acc + b (FP32, NOUT channels)
//   EPI_DGRAD     g = acc + g_in (FP32);  dz = BF16(g * GELU'(z_prev))
//   EPI_QUPDATE   q_out[c] = q_in[c] + scale * (acc + b)[c], c < 6, FP32 planes [nimg][6][H][W]
// GELU is the tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
#include <cuda_bf16.h>
#include <math.h>

#include "../../include/qla_surrogate.h"
#include "qla_internal.h"
#include "qla_tc.cuh"

namespace qla {

enum ConvEpi { EPI_GELU = QLA_EPI_GELU, EPI_LINEAR = QLA_EPI_LINEAR, EPI_DGRAD = QLA_EPI_DGRAD, EPI_QUPDATE = QLA_EPI_QUPDATE };


// GELU (tanh form) with the hardware tanh approximation (tanh.approx.f32,
// relative error about 2^-11, below the BF16 resolution of the outputs).
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float gelu_f(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.7978845608028654f * 0.044715f;  // sqrt(2/pi), sqrt(2/pi) 0.044715
    const float t = tanh_fast(x * fmaf(k1, x * x, k0));
    const float hx = 0.5f * x;
    return fmaf(hx, t, hx);
}

__device__ __forceinline__ float gelu_grad(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.7978845608028654f * 0.044715f;
    const float x2 = x * x;
    const float t = tanh_fast(x * fmaf(k1, x2, k0));
    // d/dx [0.5 x (1 + t)] = 0.5 (1 + t) + 0.5 x (1 - t^2) (k0 + 3 k1 x^2)
    return fmaf(0.5f * x * fmaf(-t, t, 1.0f), fmaf(3.0f * k1, x2, k0), 0.5f * (1.0f + t));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t bf2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Shared memory: a ring of NS halo rows, As[c][slot][130 px][16 B] (c = 8-channel
// chunk), then the packed weights of all nine taps, Bs[kx][c][ky][n][16 B]
// (the three y taps consecutive along N), then one staging buffer per epilogue
// warp for its BF16 output rows (32 pixels x one column half).
template <int CCH, int NOUT>
struct ConvLayout {
    static constexpr int HALO_PX = 130;
    // Ring depth; even, so that a slot is always released by the same epilogue group.
    static constexpr int NS = CCH >= 8 && NOUT >= 64 ? 8 : (CCH >= 8 ? 6 : 8);
    static_assert(NS % 2 == 0, "ring slots alternate between the two epilogue groups");
    static constexpr int A_BYTES = CCH * NS * HALO_PX * 16;
    static constexpr int B_BYTES = 9 * CCH * NOUT * 16;
    static constexpr int A_OFF = 0;
    static constexpr int B_OFF = ((A_BYTES + 1023) / 1024) * 1024;
    static constexpr int STG_OFF = B_OFF + B_BYTES;
    static constexpr int STG_STRIDE = (NOUT < 32 ? NOUT : 32) * 2 + 16;  // bytes per pixel: an odd number of 16 B units
    static constexpr int STG_BYTES = 8 * 32 * STG_STRIDE;
    static constexpr int SMEM = STG_OFF + STG_BYTES;
    // At least half of an SM's shared memory, so one CTA per SM owns all of TMEM.
    static constexpr int SMEM_LAUNCH = SMEM > 116 * 1024 ? SMEM : 116 * 1024;
    static constexpr int TMEM_COLS = 512;
    static constexpr int NB = TMEM_COLS / NOUT;  // output-row accumulators (NOUT columns each)
};

constexpr int CONV_EPI_WARPS = 8;
constexpr int CONV_MMA_WARP = 8;
constexpr int CONV_LOAD_WARP = 9;
constexpr int CONV_THREADS = 320;
constexpr uint32_t CONV_WAIT_TRIES = 1u << 22;

__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(tc::smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(tc::smem_addr(bar))
                 : "memory");
}

// Stores BF16 outputs of one column half of a warp's 32 pixels: vals[c] holds
// channels cb0 + 8c .. cb0 + 8c + 7 of this lane's pixel p_w0 + lane. The
// values pass through the warp's staging buffer so that the global stores are
// runs of NC * 2 bytes per pixel (whole sectors) instead of 16-byte pieces of
// 32 different pixels per instruction.
template <int NC, int NOUT, int STRIDE>
__device__ __forceinline__ void store_half_bf16(uint8_t *stg, const uint4 (&vals)[NC / 8], __nv_bfloat16 *out,
                                                size_t p_w0, int cb0, int lane) {
    constexpr int CH = NC / 8;  // 16-byte chunks per pixel
#pragma unroll
    for (int c = 0; c < CH; ++c) *reinterpret_cast<uint4 *>(stg + lane * STRIDE + c * 16) = vals[c];
    __syncwarp();
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        const int idx = 32 * k + lane, pp = idx / CH, cc = idx % CH;
        const uint4 w = *reinterpret_cast<const uint4 *>(stg + pp * STRIDE + cc * 16);
        *reinterpret_cast<uint4 *>(out + (p_w0 + pp) * NOUT + cb0 + 8 * cc) = w;
    }
    __syncwarp();
}

// Segment walker shared by all roles: the CTA's rows, ordered (image, column
// block, row), split into runs of consecutive rows of one column block.
struct ConvSeg {
    int img, x0, y_s, len;
};
__host__ __device__ __forceinline__ ConvSeg conv_segment(long long u0, long long u_end, int H, int TPR) {
    ConvSeg g;
    g.y_s = int(u0 % H);
    const long long t2 = u0 / H;
    g.x0 = int(t2 % TPR) * 128;
    g.img = int(t2 / TPR);
    const long long end = (u0 - g.y_s + H) < u_end ? (u0 - g.y_s + H) : u_end;
    g.len = int(end - u0);
    return g;
}

// ---------------------------------------------------------------------------
// The MMA issue schedule, shared by the kernel's MMA warp and by the host-side
// enumeration (qla_conv_schedule) that tests/test_conv_schedule.py checks.
// Input row j of a run of `len` output rows (ring row r) feeds output rows
// j - ky (ky = 0..2); output row `on` = o_run + j owns accumulator block
// b0 = (-on) mod NB of the TMEM ring, so the rows it feeds are consecutive
// blocks and one MMA covers them (split in two where the ring wraps).
// ---------------------------------------------------------------------------
struct ConvMma {
    int kx, k2;      // x tap, 16-channel slice
    int ka, kb;      // y taps ka..kb in one MMA (N = (kb - ka + 1) NOUT)
    int blk;         // accumulator block of y tap ka
    int acc;         // 0: the first MMA of a new accumulator (accumulation off)
    uint32_t a_off;  // A descriptor start, 16-byte units from the row's ring slot
    uint32_t b_off;  // B descriptor start, 16-byte units from the weights
};

__host__ __device__ __forceinline__ int conv_block(long long on, int NB) { return int((NB - on % NB) % NB); }

// The MMAs of input row j: the y taps whose output row lies inside the run,
// split where the block ring wraps, the first MMA of a new accumulator (x tap
// 0, first slice, ky = 0) alone with accumulation off.
template <int CCH, int NOUT, int NS, int HP, class F>
__host__ __device__ __forceinline__ void conv_row_mmas(int j, int len, int b0, F &&emit) {
    constexpr int NB = 512 / NOUT;
    const int k_lo = j - len + 1 > 0 ? j - len + 1 : 0;
    const int k_hi = j < 2 ? j : 2;
    const int wrap = NB - b0;  // first ky whose block wraps to 0
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
        for (int k2 = 0; k2 < CCH / 2; ++k2) {
            const bool first = kx == 0 && k2 == 0;
            for (int ka = k_lo; ka <= k_hi;) {
                int kb = k_hi;
                if (ka < wrap && wrap <= kb) kb = wrap - 1;
                if (first && ka == 0) kb = 0;
                const int blk = b0 + ka < NB ? b0 + ka : b0 + ka - NB;
                emit(ConvMma{kx, k2, ka, kb, blk, (first && ka == 0) ? 0 : 1, uint32_t((2 * k2) * NS * HP + kx),
                             uint32_t((kx * CCH + 2 * k2) * 3 * NOUT + ka * NOUT)});
                ka = kb + 1;
            }
        }
    }
}

// Before the MMAs of input row j: a new accumulator (j < len) reuses the block
// of output row on - NB, so the MMA warp waits for that row's epilogue on
// acc_empty[b0], phase parity (on / NB + 1) & 1. Returns false if no wait.
__host__ __device__ __forceinline__ bool conv_row_acc_wait(int j, int len, long long on, int NB, uint32_t *parity) {
    *parity = uint32_t(((on / NB) + 1) & 1);
    return j < len && on >= NB;
}

// After the MMAs of input row j: output row on - 2 has all its taps; its
// block is committed to acc_full (-1: none yet).
__host__ __device__ __forceinline__ int conv_row_done_block(int j, long long on, int NB) {
    return j >= 2 ? conv_block(on - 2, NB) : -1;
}

// Walks the CTA's rows in the order of every role: for each run, input rows
// j = 0 .. len + 1 (ring row g + j, output row o + j); row(sg, j, r, on)
// returns false to stop.
template <class F>
__host__ __device__ __forceinline__ void conv_walk_rows(long long u_begin, long long u_end, int H, int TPR, F &&row) {
    long long g = 0, o = 0;
    for (long long u0 = u_begin; u0 < u_end;) {
        const ConvSeg sg = conv_segment(u0, u_end, H, TPR);
        for (int j = 0; j < sg.len + 2; ++j)
            if (!row(sg, j, g + j, o + j)) return;
        g += sg.len + 2;
        o += sg.len;
        u0 += sg.len;
    }
}

// Persistent, warp-specialised conv kernel (320 threads = 10 warps). Work =
// rows of 128-pixel column blocks, ordered (image, column block, row); each CTA
// takes a contiguous range and walks down its column blocks with a ring of
// halo rows in shared memory, so every input row is loaded once per block.
//   warp 9 (loader)   cp.async of each halo row into the ring; arrival on
//                     full[slot] when its copies land; waits on empty[slot]
//   warp 8 (MMA)      per input row, one lane issues the 3 x CCH/2 MMAs (x tap,
//                     16-channel slice) whose N = 3 NOUT columns are the
//                     accumulators of the three output rows the row feeds,
//                     then releases the row (empty[slot]) and commits acc_full
//                     of the output row it completes
//   warps 0-7 (epilogue) wait acc_full, tcgen05.ld, fused epilogue, stores;
//                     arrive on acc_empty, and on empty[slot] of the centre
//                     row (a residual equal to the input is read from the
//                     ring), so a row is free after its MMAs and its
//                     epilogue (edge rows of a run get their arrival at the
//                     run's start and end)
// TMEM holds NB = 512 / NOUT accumulators in a ring; output row o (counted
// over the CTA's runs) owns block (-o) mod NB, so the rows j, j-1, j-2 that
// input row j feeds are consecutive blocks and one MMA covers them (split in
// two where the ring wraps). Every wait is bounded; a timeout sets the error
// flag and the role stops, and the others time out in turn, so the kernel
// always ends.
template <int CCH, int NOUT>
__global__ void __launch_bounds__(CONV_THREADS, 1) conv3x3_tc_kernel(const ConvArgs a) {
    using L = ConvLayout<CCH, NOUT>;
    constexpr int CIN = 8 * CCH;
    constexpr int NS = L::NS;
    constexpr int HP = L::HALO_PX;
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NB = L::NB;
    __shared__ uint64_t full_bar[NS], empty_bar[NS], accf_bar[NB], acce_bar[NB], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ float bias_s[64];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int TPR = W / 128;
    const long long T = (long long)a.nimg * TPR * H;
    const long long u_begin = T * blockIdx.x / gridDim.x;
    const long long u_end = T * (blockIdx.x + 1) / gridDim.x;
    uint8_t *As = smem + L::A_OFF;
    uint8_t *Bs = smem + L::B_OFF;

    {
        const uint4 *src = static_cast<const uint4 *>(a.w);
        for (int i = tid; i < 9 * CCH * NOUT; i += CONV_THREADS) {  // [t][c][n] -> [kx][c][ky][n]
            const int n = i % NOUT, c = (i / NOUT) % CCH, t = i / (NOUT * CCH);
            const int ky = t / 3, kx = t - 3 * ky;
            cp_async16(Bs + (((kx * CCH + c) * 3 + ky) * NOUT + n) * 16, src + i);
        }
        cp_async_commit();
        if (tid < 64) bias_s[tid] = (a.bias && tid < NOUT && a.epi != EPI_DGRAD) ? a.bias[tid] : 0.0f;
    }
    if (warp == CONV_MMA_WARP) tc::tmem_alloc(&tmem_base_s, L::TMEM_COLS);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full_bar[s], 32);
            tc::mbar_init(&empty_bar[s], 1 + CONV_EPI_WARPS / 2);
        }
        for (int b = 0; b < NB; ++b) {
            tc::mbar_init(&accf_bar[b], 1);
            tc::mbar_init(&acce_bar[b], CONV_EPI_WARPS / 2);
        }
        tc::mbar_init(&done_bar, 1);
        tc::fence_mbar_init();
    }
    cp_async_wait_0();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_s;

    if (warp == CONV_LOAD_WARP) {
        // ---------------- loader ----------------
        const __nv_bfloat16 *xg = static_cast<const __nv_bfloat16 *>(a.x);
        long long g = 0;  // running row counter (ring position)
        bool ok = true;
        for (long long u0 = u_begin; u0 < u_end && ok;) {
            const ConvSeg sg = conv_segment(u0, u_end, H, TPR);
            const __nv_bfloat16 *ximg = xg + (size_t)sg.img * H * W * CIN;
            for (int j = 0; j < sg.len + 2 && ok; ++j, ++g) {
                const int slot = int(g % NS);
                if (g >= NS && !tc::mbar_wait(&empty_bar[slot], uint32_t((g / NS - 1) & 1), CONV_WAIT_TRIES)) {
                    ok = false;
                    break;
                }
                int yy = (sg.y_s - 1 + j) % H;
                yy = yy < 0 ? yy + H : yy;
                const __nv_bfloat16 *row = ximg + (size_t)yy * W * CIN;
                for (int i = lane; i < CCH * HP; i += 32) {
                    const int c = i % CCH, px = i / CCH;
                    int xx = sg.x0 + px - 1;
                    xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
                    cp_async16(As + ((c * NS + slot) * HP + px) * 16, row + (size_t)xx * CIN + 8 * c);
                }
                cp_async_arrive_noinc(&full_bar[slot]);
            }
            u0 += sg.len;
        }
        cp_async_wait_0();
        if (!ok && lane == 0) atomicExch(a.error, 1);
    } else if (warp == CONV_MMA_WARP) {
        // ---------------- MMA issuer ----------------
        // Input row j of a run feeds output rows j - ky (ky = 0..2) through
        // the weights of y tap ky; those rows' accumulators are the blocks
        // b0, b0 + 1, b0 + 2 (mod NB), b0 = block of output row j. The first
        // MMA of a new accumulator (x tap 0, first slice, ky = 0) runs alone
        // with accumulation off; the rest add to what is there.
        constexpr uint32_t IDESC1 = tc::make_idesc_bf16(128, NOUT);
        constexpr uint32_t IDESC2 = tc::make_idesc_bf16(128, 2 * NOUT);
        constexpr uint32_t IDESC3 = tc::make_idesc_bf16(128, 3 * NOUT);
        constexpr uint32_t A_LBO = NS * HP * 16, A_SBO = 128;
        constexpr uint32_t B_LBO = 3 * NOUT * 16, B_SBO = 128;
        const uint64_t ad0 = tc::make_desc(tc::smem_addr(As), A_LBO, A_SBO);
        const uint64_t bd0 = tc::make_desc(tc::smem_addr(Bs), B_LBO, B_SBO);
        const uint32_t a_lo0 = uint32_t(ad0), a_hi = uint32_t(ad0 >> 32);
        const uint32_t b_lo0 = uint32_t(bd0), b_hi = uint32_t(bd0 >> 32);
        bool ok = true;
        conv_walk_rows(u_begin, u_end, H, TPR, [&](const ConvSeg &sg, int j, long long r, long long on) {
            const int b0 = conv_block(on, NB);
            if (!tc::mbar_wait(&full_bar[r % NS], uint32_t((r / NS) & 1), CONV_WAIT_TRIES)) ok = false;
            uint32_t par = 0;
            if (ok && conv_row_acc_wait(j, sg.len, on, NB, &par) && !tc::mbar_wait(&acce_bar[b0], par, CONV_WAIT_TRIES))
                ok = false;
            if (!ok) return false;
            tc::fence_after_sync();
            if (lane == 0) {
                const uint32_t a_row = a_lo0 + uint32_t(int(r % NS) * HP);  // (slot * HP * 16) >> 4
                conv_row_mmas<CCH, NOUT, NS, HP>(j, sg.len, b0, [&](const ConvMma &m) {
                    const uint32_t idesc = m.kb == m.ka ? IDESC1 : (m.kb == m.ka + 1 ? IDESC2 : IDESC3);
                    tc::mma_bf16_lohi(tmem + uint32_t(m.blk * NOUT), a_row + m.a_off, a_hi, b_lo0 + m.b_off, b_hi,
                                      idesc, uint32_t(m.acc));
                });
                tc::mma_commit(&empty_bar[r % NS]);  // the tensor cores are done with row r
                const int bd = conv_row_done_block(j, on, NB);
                if (bd >= 0) tc::mma_commit(&accf_bar[bd]);  // output row on - 2
            }
            __syncwarp();
            return true;
        });
        if (lane == 0) {
            tc::mma_commit(&done_bar);  // tracks every MMA issued above
            if (!tc::mbar_wait(&done_bar, 0u, CONV_WAIT_TRIES)) ok = false;
        }
        __syncwarp();
        if (!ok && lane == 0) atomicExch(a.error, 1);
    } else {
        // ---------------- epilogue ----------------
        // Two groups of four warps (grp = warp / 4) take alternate output rows
        // (o mod 2), so the epilogues of two rows overlap; each warp covers its
        // TMEM lane quarter and all NOUT columns. Ring rows are released by the
        // group of the output row they are the centre of (edge rows: the group
        // of the neighbouring output row), so a slot is always released by the
        // same group and its arrivals come in order.
        const int q = warp & 3, grp = warp >> 2;
        const int m = 32 * q + lane;
        uint8_t *stg = smem + L::STG_OFF + warp * 32 * L::STG_STRIDE;  // this warp's staging buffer
        constexpr int NC = NOUT < 32 ? NOUT : 32;
        constexpr int NCB = NOUT >= 64 ? 2 : 1;
        const bool res_smem = a.epi == EPI_GELU && a.aux0 != nullptr && a.aux0 == a.x && CIN == NOUT;
        long long o = 0, g = 0;
        bool ok = true;
        for (long long u0 = u_begin; u0 < u_end && ok;) {
            const ConvSeg sg = conv_segment(u0, u_end, H, TPR);
            const long long o_seg = o;
            __syncwarp();
            if (lane == 0 && int((o_seg - 1) & 1) == grp) mbar_arrive(&empty_bar[g % NS]);  // first halo row
            // q update (the surrogate's last layer, NOUT = 16): the FP32 input
            // state of this group's rows is loaded one of its rows ahead, before
            // the wait for the row's accumulator, so that the load latency overlaps
            // the wait and the previous row's epilogue (issued after the wait it was
            // exposed once per row). Other widths load it after the wait.
            constexpr bool QPRE = NOUT == 16;
            constexpr int NQ = QPRE ? 6 : 1;
            const size_t qP = (size_t)H * W;
            bool qup = false;
            const float *qi = nullptr;
            float qv[NQ];
            auto qload = [&](int i, float (&dst)[NQ]) {
                const size_t pix = (size_t)(sg.y_s + i) * W + sg.x0 + m;
#pragma unroll
                for (int c = 0; c < NQ; ++c) dst[c] = qi[c * qP + pix];
            };
            if constexpr (QPRE) {
                qup = a.epi == EPI_QUPDATE;
                if (qup) {
                    qi = static_cast<const float *>(a.aux0) + (size_t)sg.img * 6 * qP;
                    const int i_first = int(((long long)grp - o_seg) & 1);  // first i with (o_seg + i) mod 2 == grp
                    if (i_first < sg.len) qload(i_first, qv);
                }
            }
            for (int i = 0; i < sg.len; ++i, ++o) {
                if (int(o & 1) != grp) continue;
                float qn[NQ];
                bool q_more = false;
                if constexpr (QPRE) {
                    q_more = qup && i + 2 < sg.len;
                    if (q_more) qload(i + 2, qn);
                }
                const int b = int((NB - o % NB) % NB);
                if (!tc::mbar_wait(&accf_bar[b], uint32_t((o / NB) & 1), CONV_WAIT_TRIES)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
#pragma unroll 1
                for (int cbi = 0; cbi < NCB; ++cbi) {
                    const int cb0 = 32 * cbi;
                    const int y = sg.y_s + i;
                    const size_t p = ((size_t)sg.img * H + y) * W + sg.x0 + m;
                    float v[32];
                    const uint32_t ta = tmem + uint32_t(b * NOUT + cb0) + (uint32_t(32 * q) << 16);
                    if constexpr (NC == 32) tc::tmem_ld32(ta, v);
                    else tc::tmem_ld16(ta, v);
#pragma unroll
                    for (int k = 0; k < NC; ++k) v[k] += bias_s[cb0 + k];
                    if (a.epi == EPI_GELU) {
                        const uint4 *rp =
                            res_smem ? reinterpret_cast<const uint4 *>(
                                           As + (((cb0 / 8) * NS + int((g + i + 1) % NS)) * HP + m + 1) * 16)
                            : a.aux0 ? reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(a.aux0) +
                                                                       p * NOUT + cb0)
                                     : nullptr;
                        const int rstride = res_smem ? NS * HP : 1;  // uint4 steps between 8-channel chunks
                        uint4 av[NC / 8], zv[NC / 8];
#pragma unroll
                        for (int c4 = 0; c4 < NC / 8; ++c4) {
                            float g8[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) g8[k] = gelu_f(v[8 * c4 + k]);
                            if (rp) {
                                const uint4 w4 = rp[c4 * rstride];
                                const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    g8[2 * k] += __uint_as_float(ww[k] << 16);
                                    g8[2 * k + 1] += __uint_as_float(ww[k] & 0xffff0000u);
                                }
                            }
                            av[c4] = make_uint4(bf2(g8[0], g8[1]), bf2(g8[2], g8[3]), bf2(g8[4], g8[5]),
                                                bf2(g8[6], g8[7]));
                            const float *z = v + 8 * c4;
                            zv[c4] = make_uint4(bf2(z[0], z[1]), bf2(z[2], z[3]), bf2(z[4], z[5]), bf2(z[6], z[7]));
                        }
                        // Staged stores measured faster for the first layer (59.6 vs 63.8 us at
                        // 1024^2) and with z also stored (73.9 vs 141 us), slower for a hidden
                        // layer storing only the activation (99.0 vs 96.1 us).
                        if (CCH < 8 || a.out0) {
                            store_half_bf16<NC, NOUT, L::STG_STRIDE>(stg, av, static_cast<__nv_bfloat16 *>(a.out1),
                                                                     p - lane, cb0, lane);
                            if (a.out0)
                                store_half_bf16<NC, NOUT, L::STG_STRIDE>(
                                    stg, zv, static_cast<__nv_bfloat16 *>(a.out0), p - lane, cb0, lane);
                        } else {
                            uint4 *ao = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out1) + p * NOUT + cb0);
#pragma unroll
                            for (int c4 = 0; c4 < NC / 8; ++c4) ao[c4] = av[c4];
                        }
                    } else if (a.epi == EPI_LINEAR) {
                        float4 *op = reinterpret_cast<float4 *>(static_cast<float *>(a.out0) + p * NOUT + cb0);
#pragma unroll
                        for (int k = 0; k < NC / 4; ++k)
                            op[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    } else if (a.epi == EPI_DGRAD) {
                        const float4 *gin = a.aux0 ? reinterpret_cast<const float4 *>(
                                                         static_cast<const float *>(a.aux0) + p * NOUT + cb0)
                                                   : nullptr;
                        float4 *go = reinterpret_cast<float4 *>(static_cast<float *>(a.out0) + p * NOUT + cb0);
                        const uint4 *zp = reinterpret_cast<const uint4 *>(
                            static_cast<const __nv_bfloat16 *>(a.zprev) + p * NOUT + cb0);
                        uint4 dzv[NC / 8];
#pragma unroll
                        for (int c4 = 0; c4 < NC / 8; ++c4) {
                            float g8[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) g8[k] = v[8 * c4 + k];
                            if (gin) {
                                const float4 g0 = gin[2 * c4], g1 = gin[2 * c4 + 1];
                                g8[0] += g0.x; g8[1] += g0.y; g8[2] += g0.z; g8[3] += g0.w;
                                g8[4] += g1.x; g8[5] += g1.y; g8[6] += g1.z; g8[7] += g1.w;
                            }
                            go[2 * c4] = make_float4(g8[0], g8[1], g8[2], g8[3]);
                            go[2 * c4 + 1] = make_float4(g8[4], g8[5], g8[6], g8[7]);
                            const uint4 z4 = zp[c4];
                            const uint32_t zz[4] = {z4.x, z4.y, z4.z, z4.w};
                            float d[8];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                d[2 * k] = g8[2 * k] * gelu_grad(__uint_as_float(zz[k] << 16));
                                d[2 * k + 1] = g8[2 * k + 1] * gelu_grad(__uint_as_float(zz[k] & 0xffff0000u));
                            }
                            dzv[c4] = make_uint4(bf2(d[0], d[1]), bf2(d[2], d[3]), bf2(d[4], d[5]), bf2(d[6], d[7]));
                        }
                        store_half_bf16<NC, NOUT, L::STG_STRIDE>(stg, dzv, static_cast<__nv_bfloat16 *>(a.out1),
                                                                 p - lane, cb0, lane);
                    } else if (cb0 == 0) {  // EPI_QUPDATE: channels 0..5
                        const size_t pix = (size_t)y * W + sg.x0 + m;
                        float *qo = static_cast<float *>(a.out0) + (size_t)sg.img * 6 * qP;
                        if constexpr (QPRE) {
#pragma unroll
                            for (int c = 0; c < 6; ++c) qo[c * qP + pix] = qv[c] + a.scale * v[c];
                        } else {
                            const float *qin = static_cast<const float *>(a.aux0) + (size_t)sg.img * 6 * qP;
#pragma unroll
                            for (int c = 0; c < 6; ++c) qo[c * qP + pix] = qin[c * qP + pix] + a.scale * v[c];
                        }
                    }
                }
                if (q_more) {
#pragma unroll
                    for (int c = 0; c < NQ; ++c) qv[c] = qn[c];
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&acce_bar[b]);
                    mbar_arrive(&empty_bar[(g + i + 1) % NS]);  // centre row of output row i
                }
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0 && int((o_seg + sg.len) & 1) == grp)
                mbar_arrive(&empty_bar[(g + sg.len + 1) % NS]);  // last halo row
            g += sg.len + 2;
            u0 += sg.len;
        }
        if (!ok && lane == 0) atomicExch(a.error, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == CONV_MMA_WARP) tc::tmem_dealloc(tmem, L::TMEM_COLS);
}

template <int CCH, int NOUT>
cudaError_t launch_conv_t(const ConvArgs &a, cudaStream_t st) {
    using L = ConvLayout<CCH, NOUT>;
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<CCH, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L::SMEM_LAUNCH);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long rows = (long long)a.nimg * a.H * (a.W / 128);
    const int grid = rows < sms ? int(rows) : sms;
    conv3x3_tc_kernel<CCH, NOUT><<<grid, CONV_THREADS, L::SMEM_LAUNCH, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores:
//   dW[n][c][ky][kx] = sum_p g[p][n] x[p + (ky-1, kx-1)][c]
// as D[m][n] = sum_k A[m][k] B[n][k] with K = pixels and both operands
// MN-major (NHWC rows give 8 consecutive channels per 16 bytes). A rows are
// (ky, c) for two consecutive halo rows stacked in M = 128 (ky = 0, 1 in one
// tile; ky = 2 and an unused half in the other); kx is a 16-byte shift of the
// start address along K. Six accumulator tiles (2 row pairs x 3 kx) of N = NT
// columns stay in TMEM for all of a CTA's rows; at the end each CTA writes its
// partial sums [9][NT][64] (FP32), reduced over CTAs in a fixed order later.
// The x ring has one mirror slot after the last, a copy of slot 0, so that two
// consecutive rows are always adjacent in memory. Source x may have 16 or 64
// channels (16: the other chunks stay zero).
// ---------------------------------------------------------------------------
template <int NT>
struct WgradLayout {
    static constexpr int HP = 130;
    static constexpr int NSX = 6;
    static constexpr int XSLOT = 8 * HP * 16;
    static constexpr int X_BYTES = (NSX + 1) * XSLOT;
    static constexpr int NSG = 4;
    static constexpr int GSLOT = (NT / 8) * 128 * 16;
    static constexpr int G_OFF = ((X_BYTES + 1023) / 1024) * 1024;
    static constexpr int SMEM = G_OFF + NSG * GSLOT;
    static constexpr int TMEM_COLS = NT == 64 ? 512 : 128;  // 6 tiles x NT columns
};

template <int CS, int NT>
__global__ void __launch_bounds__(CONV_THREADS, 1) wgrad_tc_kernel(const WgradArgs a) {
    using L = WgradLayout<NT>;
    constexpr int NSX = L::NSX, NSG = L::NSG, HP = L::HP;
    constexpr int CCS = CS / 8;  // source chunks per pixel
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t xf_bar[NSX], xe_bar[NSX], gf_bar[NSG], ge_bar[NSG], done_bar;
    __shared__ uint32_t tmem_base_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int TPR = W / 128;
    const long long T = (long long)a.nimg * TPR * H;
    const long long u_begin = T * blockIdx.x / gridDim.x;
    const long long u_end = T * (blockIdx.x + 1) / gridDim.x;
    uint8_t *Xs = smem;
    uint8_t *Gs = smem + L::G_OFF;

    for (int i = tid; i < L::X_BYTES / 16; i += CONV_THREADS) reinterpret_cast<uint4 *>(Xs)[i] = make_uint4(0, 0, 0, 0);
    if (warp == CONV_MMA_WARP) tc::tmem_alloc(&tmem_base_s, L::TMEM_COLS);
    if (tid == 0) {
        for (int s = 0; s < NSX; ++s) {
            tc::mbar_init(&xf_bar[s], 32);
            tc::mbar_init(&xe_bar[s], 1);
        }
        for (int s = 0; s < NSG; ++s) {
            tc::mbar_init(&gf_bar[s], 32);
            tc::mbar_init(&ge_bar[s], 1);
        }
        tc::mbar_init(&done_bar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_s;

    if (warp == CONV_LOAD_WARP) {
        const __nv_bfloat16 *xg = static_cast<const __nv_bfloat16 *>(a.x);
        const __nv_bfloat16 *gg = static_cast<const __nv_bfloat16 *>(a.g);
        long long gx = 0, gn = 0;
        bool ok = true;
        auto load_x = [&](const ConvSeg &sg, int j) -> bool {
            const int slot = int(gx % NSX);
            if (gx >= NSX && !tc::mbar_wait(&xe_bar[slot], uint32_t((gx / NSX - 1) & 1), CONV_WAIT_TRIES)) return false;
            int yy = (sg.y_s - 1 + j) % H;
            yy = yy < 0 ? yy + H : yy;
            const __nv_bfloat16 *row = xg + ((size_t)sg.img * H + yy) * W * CS;
            for (int i = lane; i < CCS * HP; i += 32) {
                const int c = i % CCS, px = i / CCS;
                int xx = sg.x0 + px - 1;
                xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
                const __nv_bfloat16 *src = row + (size_t)xx * CS + 8 * c;
                cp_async16(Xs + ((slot * 8 + c) * HP + px) * 16, src);
                if (slot == 0) cp_async16(Xs + ((NSX * 8 + c) * HP + px) * 16, src);
            }
            cp_async_arrive_noinc(&xf_bar[slot]);
            ++gx;
            return true;
        };
        auto load_g = [&](const ConvSeg &sg, int i) -> bool {
            const int slot = int(gn % NSG);
            if (gn >= NSG && !tc::mbar_wait(&ge_bar[slot], uint32_t((gn / NSG - 1) & 1), CONV_WAIT_TRIES)) return false;
            const __nv_bfloat16 *row = gg + (((size_t)sg.img * H + sg.y_s + i) * W + sg.x0) * NT;
            for (int k = lane; k < (NT / 8) * 128; k += 32) {
                const int c = k % (NT / 8), px = k / (NT / 8);
                cp_async16(Gs + slot * L::GSLOT + (c * 128 + px) * 16, row + (size_t)px * NT + 8 * c);
            }
            cp_async_arrive_noinc(&gf_bar[slot]);
            ++gn;
            return true;
        };
        for (long long u0 = u_begin; u0 < u_end && ok;) {
            const ConvSeg sg = conv_segment(u0, u_end, H, TPR);
            ok = load_x(sg, 0) && load_x(sg, 1);
            for (int i = 0; i < sg.len && ok; ++i) ok = load_x(sg, i + 2) && load_g(sg, i);
            u0 += sg.len;
        }
        cp_async_wait_0();
        if (!ok && lane == 0) atomicExch(a.error, 1);
    } else if (warp == CONV_MMA_WARP) {
        constexpr uint32_t IDESC = tc::make_idesc_bf16(128, NT) | (1u << 15) | (1u << 16);  // A, B MN-major
        const uint32_t x_base = tc::smem_addr(Xs), g_base = tc::smem_addr(Gs);
        // MN-major, no swizzle: a core matrix is 8 k-rows x 16 B (8 channels);
        // the leading byte offset steps along K (128 B: the next 8 pixels), the
        // stride byte offset along M/N (the next 8-channel chunk).
        constexpr uint32_t A_LBO = 128, A_SBO = HP * 16;
        constexpr uint32_t B_LBO = 128, B_SBO = 128 * 16;
        const uint64_t ad0 = tc::make_desc(x_base, A_LBO, A_SBO), bd0 = tc::make_desc(g_base, B_LBO, B_SBO);
        const uint32_t a_lo0 = uint32_t(ad0), a_hi = uint32_t(ad0 >> 32);
        const uint32_t b_lo0 = uint32_t(bd0), b_hi = uint32_t(bd0 >> 32);
        long long gx = 0, gn = 0;
        bool ok = true, first = true;
        for (long long u0 = u_begin; u0 < u_end && ok;) {
            const ConvSeg sg = conv_segment(u0, u_end, H, TPR);
            for (int i = 0; i < sg.len && ok; ++i, ++gn) {
                for (int j = (i == 0 ? 0 : 2); j < 3; ++j) {
                    const long long r = gx + i + j;
                    if (!tc::mbar_wait(&xf_bar[r % NSX], uint32_t((r / NSX) & 1), CONV_WAIT_TRIES)) ok = false;
                }
                if (!tc::mbar_wait(&gf_bar[gn % NSG], uint32_t((gn / NSG) & 1), CONV_WAIT_TRIES)) ok = false;
                if (!ok) break;
                tc::fence_after_sync();
                if (lane == 0) {
                    const uint32_t s0 = uint32_t((gx + i) % NSX), s2 = uint32_t((gx + i + 2) % NSX);
                    const uint32_t g_lo = b_lo0 + uint32_t(gn % NSG) * (L::GSLOT >> 4);
                    const uint32_t a0_lo = a_lo0 + s0 * 8 * HP, a1_lo = a_lo0 + s2 * 8 * HP;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) {
                            const uint32_t acc = (first && kk == 0) ? 0u : 1u;
                            tc::mma_bf16_lohi(tmem + kx * NT, a0_lo + kx + 16 * kk, a_hi, g_lo + 16 * kk, b_hi, IDESC,
                                              acc);
                            tc::mma_bf16_lohi(tmem + (3 + kx) * NT, a1_lo + kx + 16 * kk, a_hi, g_lo + 16 * kk, b_hi,
                                              IDESC, acc);
                        }
                    }
                    tc::mma_commit(&ge_bar[gn % NSG]);
                    tc::mma_commit(&xe_bar[(gx + i) % NSX]);
                    if (i == sg.len - 1) {
                        tc::mma_commit(&xe_bar[(gx + i + 1) % NSX]);
                        tc::mma_commit(&xe_bar[(gx + i + 2) % NSX]);
                    }
                }
                first = false;
                __syncwarp();
            }
            gx += sg.len + 2;
            u0 += sg.len;
        }
        if (lane == 0) tc::mma_commit(&done_bar);
        __syncwarp();
        if (!ok && lane == 0) atomicExch(a.error, 1);
    }
    if (warp < CONV_EPI_WARPS) {
        // epilogue: partial sums of this CTA
        const bool ok = tc::mbar_wait(&done_bar, 0u, CONV_WAIT_TRIES);
        if (!ok && lane == 0) atomicExch(a.error, 1);
        tc::fence_after_sync();
        const int q = warp & 3, half = warp >> 2;
        const int m = 32 * q + lane;
        const int c = m & 63;
        float *part = a.part + (size_t)blockIdx.x * 9 * NT * 64;
        if (ok && (NT == 64 || half == 0)) {
            for (int pr = 0; pr < 2; ++pr) {
                const int ky = 2 * pr + (m >> 6);
                for (int kx = 0; kx < 3; ++kx) {
                    float v[32];
                    if (NT == 64) {
                        tc::tmem_ld32(tmem + (pr * 3 + kx) * NT + 32 * half + (uint32_t(32 * q) << 16), v);
                        if (ky <= 2) {
                            float *o = part + ((size_t)(ky * 3 + kx) * NT + 32 * half) * 64 + c;
#pragma unroll
                            for (int k = 0; k < 32; ++k) o[k * 64] = v[k];
                        }
                    } else {
                        tc::tmem_ld32(tmem + (pr * 3 + kx) * NT + (uint32_t(32 * q) << 16), v);  // 16 used
                        if (ky <= 2) {
                            float *o = part + ((size_t)(ky * 3 + kx) * NT) * 64 + c;
#pragma unroll
                            for (int k = 0; k < 16; ++k) o[k * 64] = v[k];
                        }
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == CONV_MMA_WARP) tc::tmem_dealloc(tmem, L::TMEM_COLS);
}

template <int CS, int NT>
cudaError_t launch_wgrad_t(const WgradArgs &a, int grid, cudaStream_t st) {
    using L = WgradLayout<NT>;
    cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<CS, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L::SMEM);
    if (e != cudaSuccess) return e;
    wgrad_tc_kernel<CS, NT><<<grid, CONV_THREADS, L::SMEM, st>>>(a);
    return cudaGetLastError();
}

int wgrad_grid(const WgradArgs &a) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long rows = (long long)a.nimg * a.H * (a.W / 128);
    return rows < sms ? int(rows) : sms;
}

cudaError_t launch_wgrad_tc(const WgradArgs &a, int *grid_out, cudaStream_t st) {
    const int grid = wgrad_grid(a);
    if (grid_out) *grid_out = grid;
    if (a.cs == 64 && a.nt == 64) return launch_wgrad_t<64, 64>(a, grid, st);
    if (a.cs == 16 && a.nt == 64) return launch_wgrad_t<16, 64>(a, grid, st);
    if (a.cs == 64 && a.nt == 16) return launch_wgrad_t<64, 16>(a, grid, st);
    return cudaErrorInvalidValue;
}

bool conv_supported(int cin, int nout) {
    return (cin == 16 && nout == 64) || (cin == 64 && nout == 64) || (cin == 64 && nout == 16);
}

cudaError_t launch_conv(int cin, int nout, const ConvArgs &a, cudaStream_t st) {
    if (cin == 16 && nout == 64) return launch_conv_t<2, 64>(a, st);
    if (cin == 64 && nout == 64) return launch_conv_t<8, 64>(a, st);
    if (cin == 64 && nout == 16) return launch_conv_t<8, 16>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace qla

extern "C" qla_status qla_conv3x3_bf16(const void *x, int nimg, int H, int W, int cin, const void *w_packed,
                                       const float *bias, int nout, int epilogue, const void *aux0, const void *zprev,
                                       void *out0, void *out1, float scale, int *error_flag, void *stream) {
    if (!x || !w_packed || !error_flag || nimg < 1 || H < 1 || W < 128 || W % 128 != 0) return QLA_EINVAL;
    if ((long long)nimg * H * W > (1LL << 31) - 1) return QLA_EINVAL;
    if (!qla::conv_supported(cin, nout)) return QLA_EUNSUPPORTED;
    if (epilogue < 0 || epilogue > 3) return QLA_EINVAL;
    if (epilogue != qla::EPI_GELU && !out0) return QLA_EINVAL;
    if ((epilogue == qla::EPI_GELU || epilogue == qla::EPI_DGRAD) && !out1) return QLA_EINVAL;
    if (epilogue == qla::EPI_DGRAD && !zprev) return QLA_EINVAL;
    if (epilogue == qla::EPI_QUPDATE && (!aux0 || nout < 6)) return QLA_EINVAL;
    qla::ConvArgs a;
    a.x = x;
    a.w = w_packed;
    a.bias = bias;
    a.nimg = nimg;
    a.H = H;
    a.W = W;
    a.epi = epilogue;
    a.aux0 = aux0;
    a.zprev = zprev;
    a.out0 = out0;
    a.out1 = out1;
    a.scale = scale;
    a.error = error_flag;
    const cudaError_t e = qla::launch_conv(cin, nout, a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QLA_OK : QLA_ECUDA;
}

// ---------------------------------------------------------------------------
// Weight packing: FP32 w[nout][cin][3][3] -> BF16 [9][cin_pad/8][nout_pad][8]
// (the B operand layout of conv3x3_tc_kernel), zero-padded.
//   PACK_PLAIN       packed[t][c][n] = w[n][c][t]
//   PACK_ADJOINT     the input-gradient convolution of w: w'[c][n][ky][kx] =
//                    w[n][c][2-ky][2-kx] (packed outputs = w's inputs)
//   PACK_TIED_INPUT  as PLAIN, but packed input channels 0-5 and 6-11 both
//                    read logical 0-5 (high and low BF16 parts of the same
//                    field) and 12-14 read logical 6-8
// ---------------------------------------------------------------------------
namespace qla {

__global__ void pack_conv_weights_kernel(const float *__restrict__ w, int nout, int cin, int nout_pad, int cin_pad,
                                         int mode, __nv_bfloat16 *__restrict__ out) {
    const int total = 9 * cin_pad * nout_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int j = i % 8;
        const int n = (i / 8) % nout_pad;
        const int chunk = (i / (8 * nout_pad)) % (cin_pad / 8);
        const int t = i / (8 * nout_pad * (cin_pad / 8));
        int c = chunk * 8 + j;
        const int ky = t / 3, kx = t % 3;
        float v = 0.0f;
        if (mode == PACK_ADJOINT) {
            // packed output channel n ranges over the original inputs, packed input c over the original outputs
            if (n < cin && c < nout) v = w[((size_t(c) * cin + n) * 3 + (2 - ky)) * 3 + (2 - kx)];
        } else {
            if (mode == PACK_TIED_INPUT) c = c < 6 ? c : (c < 15 ? c - 6 : cin);
            if (n < nout && c < cin) v = w[((size_t(n) * cin + c) * 3 + ky) * 3 + kx];
        }
        out[i] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_pack_weights(const float *w, int nout, int cin, int nout_pad, int cin_pad, int mode,
                                void *packed, cudaStream_t st) {
    const int total = 9 * cin_pad * nout_pad;
    pack_conv_weights_kernel<<<(total + 255) / 256, 256, 0, st>>>(w, nout, cin, nout_pad, cin_pad, mode,
                                                                  static_cast<__nv_bfloat16 *>(packed));
    return cudaGetLastError();
}

}  // namespace qla

extern "C" qla_status qla_pack_conv_weights(const float *w, int nout, int cin, int nout_pad, int cin_pad,
                                            int transpose_flip, void *packed, void *stream) {
    if (!w || !packed || nout < 1 || cin < 1 || cin_pad % 8 != 0 || nout_pad % 8 != 0) return QLA_EINVAL;
    if (!transpose_flip && (nout > nout_pad || cin > cin_pad)) return QLA_EINVAL;
    if (transpose_flip && (cin > nout_pad || nout > cin_pad)) return QLA_EINVAL;
    const cudaError_t e = qla::launch_pack_weights(w, nout, cin, nout_pad, cin_pad,
                                                   transpose_flip ? qla::PACK_ADJOINT : qla::PACK_PLAIN, packed,
                                                   static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QLA_OK : QLA_ECUDA;
}

namespace qla {
namespace {

// Host-side walk of one CTA's MMA warp (the same helpers the kernel calls).
template <int CCH, int NOUT>
long long conv_schedule_t(int nimg, int H, int W, int grid, int cta, int *rec, long long cap) {
    using L = ConvLayout<CCH, NOUT>;
    constexpr int NB = L::NB, NS = L::NS, HP = L::HALO_PX;
    const int TPR = W / 128;
    const long long T = (long long)nimg * TPR * H;
    const long long u_begin = T * cta / grid, u_end = T * (cta + 1) / grid;
    long long n = 0;
    auto put = [&](int type, long long r, long long on, int j, int len, int a, int b, int c, int d, int e, int f,
                   uint32_t g, uint32_t h) {
        if (n < cap) {
            int *p = rec + n * QLA_CONV_SCHEDULE_FIELDS;
            const int v[QLA_CONV_SCHEDULE_FIELDS] = {type, int(r), int(on), j, len, a, b, c, d, e, f, int(g), int(h), 0};
            for (int k = 0; k < QLA_CONV_SCHEDULE_FIELDS; ++k) p[k] = v[k];
        }
        ++n;
    };
    conv_walk_rows(u_begin, u_end, H, TPR, [&](const ConvSeg &sg, int j, long long r, long long on) {
        const int b0 = conv_block(on, NB);
        uint32_t par = 0;
        if (conv_row_acc_wait(j, sg.len, on, NB, &par)) put(2, r, on, j, sg.len, b0, int(par), 0, 0, 0, 0, 0, 0);
        conv_row_mmas<CCH, NOUT, NS, HP>(j, sg.len, b0, [&](const ConvMma &m) {
            put(0, r, on, j, sg.len, m.kx, m.k2, m.ka, m.kb, m.blk, m.acc, m.a_off, m.b_off);
        });
        put(3, r, on, j, sg.len, int(r % NS), 0, 0, 0, 0, 0, 0, 0);
        const int bd = conv_row_done_block(j, on, NB);
        if (bd >= 0) put(1, r, on, j, sg.len, bd, 0, 0, 0, 0, 0, 0, 0);
        return true;
    });
    return n;
}

}  // namespace
}  // namespace qla

extern "C" qla_status qla_conv_schedule(int cin, int nout, int nimg, int H, int W, int grid, int cta, int *records,
                                        long long capacity, long long *count) {
    if (!count || nimg < 1 || H < 1 || W < 128 || W % 128 != 0 || grid < 1 || cta < 0 || cta >= grid ||
        capacity < 0 || (capacity > 0 && !records) || (long long)nimg * H * (W / 128) > (1LL << 30))
        return QLA_EINVAL;
    long long n;
    if (cin == 16 && nout == 64) n = qla::conv_schedule_t<2, 64>(nimg, H, W, grid, cta, records, capacity);
    else if (cin == 64 && nout == 64) n = qla::conv_schedule_t<8, 64>(nimg, H, W, grid, cta, records, capacity);
    else if (cin == 64 && nout == 16) n = qla::conv_schedule_t<8, 16>(nimg, H, W, grid, cta, records, capacity);
    else return QLA_EUNSUPPORTED;
    *count = n;
    return QLA_OK;
}
