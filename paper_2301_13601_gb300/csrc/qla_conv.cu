// 3x3 convolution with circular padding on BF16 NHWC activations, as an
// implicit GEMM on the tcgen05 tensor cores with FP32 accumulation in TMEM.
//
// One tile = 128 consecutive pixels of one image row (M = 128), all output
// channels (N = NOUT), K = 9 taps x input channels. The CTA stages the 3-row
// halo block (3 x 130 pixels x CIN channels) once per tile in the interleaved
// K-major layout, so the nine taps are nine shifted windows of the same block
// (no swizzle: any 16-byte aligned start is a valid operand). All 9 taps of the
// packed weights stay resident in shared memory. One thread issues the MMAs;
// the 128 threads (4 warps x 32 TMEM lanes) run the fused epilogue:
//   EPI_GELU      z = acc + b;  act = GELU(z) (+ residual);  stores z, act (BF16)
//   EPI_LINEAR    out = acc + b (FP32, NOUT channels)
//   EPI_DGRAD     g = acc + g_in (FP32);  dz = BF16(g * GELU'(z_prev))
//   EPI_QUPDATE   q_out[c] = q_in[c] + scale * (acc + b)[c], c < 6, SoA FP32 planes
// GELU is the tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
#include <cuda_bf16.h>
#include <math.h>

#include "../../include/qla_surrogate.h"
#include "qla_tc.cuh"

namespace qla {

enum ConvEpi { EPI_GELU = QLA_EPI_GELU, EPI_LINEAR = QLA_EPI_LINEAR, EPI_DGRAD = QLA_EPI_DGRAD, EPI_QUPDATE = QLA_EPI_QUPDATE };

struct ConvArgs {
    const __nv_bfloat16 *x;      // [H][W][8*CCH]
    const __nv_bfloat16 *w;      // packed [9][CCH][NOUT][8]
    const float *bias;           // [NOUT] or null
    int H, W;
    int epi;
    const void *aux0;            // GELU: residual act (BF16 [H][W][NOUT]) or null; DGRAD: g_in FP32 [H][W][NOUT] or null;
                                 // QUPDATE: q_in FP32 [6][H][W]
    const __nv_bfloat16 *zprev;  // DGRAD: pre-activation of the previous layer (BF16 [H][W][NOUT]) or null
    void *out0;                  // GELU: z (BF16) ; LINEAR: FP32 ; DGRAD: g FP32 ; QUPDATE: q_out FP32 [6][H][W]
    void *out1;                  // GELU: act (BF16) ; DGRAD: dz (BF16)
    float scale;                 // QUPDATE
    int *error;                  // set when a bounded wait runs out
};

__device__ __forceinline__ float gelu_f(float x) {
    const float k = 0.7978845608028654f;  // sqrt(2/pi)
    return 0.5f * x * (1.0f + tanhf(k * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad(float x) {
    const float k = 0.7978845608028654f;
    const float u = k * (x + 0.044715f * x * x * x);
    const float t = tanhf(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * x * x);
}

template <int CCH, int NOUT>
struct ConvLayout {
    static constexpr int HALO_PX = 130;
    static constexpr int A_BYTES = CCH * 3 * HALO_PX * 16;
    static constexpr int B_BYTES = 9 * CCH * NOUT * 16;
    static constexpr int A_OFF = 0;
    static constexpr int B_OFF = ((A_BYTES + 1023) / 1024) * 1024;
    // 160 KB floor: every operand window a descriptor can address, under either
    // reading of its two byte offsets, stays inside the allocation.
    static constexpr int SMEM = B_OFF + B_BYTES > 160 * 1024 ? B_OFF + B_BYTES : 160 * 1024;
    static constexpr int TMEM_COLS = NOUT < 32 ? 32 : NOUT;
};

template <int CCH, int NOUT>
__global__ void __launch_bounds__(128, 1) conv3x3_tc_kernel(const ConvArgs a) {
    using L = ConvLayout<CCH, NOUT>;
    constexpr int CIN = 8 * CCH;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int tiles_per_row = W / 128;
    const int ntiles = H * tiles_per_row;
    uint8_t *As = smem + L::A_OFF;
    uint8_t *Bs = smem + L::B_OFF;

    // weights: all taps, resident for the CTA's lifetime
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.w);
        uint4 *dst = reinterpret_cast<uint4 *>(Bs);
        for (int i = tid; i < 9 * CCH * NOUT; i += 128) dst[i] = src[i];
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base_s, L::TMEM_COLS);
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr uint32_t IDESC = tc::make_idesc_bf16(128, NOUT);
    const uint32_t a_base = tc::smem_addr(As), b_base = tc::smem_addr(Bs);
    constexpr uint32_t A_LBO = 3 * L::HALO_PX * 16, A_SBO = 128;
    constexpr uint32_t B_LBO = NOUT * 16, B_SBO = 128;
    uint32_t phase = 0;
    bool ok = true;
    int failed = 0;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int y = tile / tiles_per_row;
        const int x0 = (tile % tiles_per_row) * 128;
        // ---- stage the 3 x 130 pixel halo block: As[c][r][px][8 bf16] ----
        for (int i = tid; i < CCH * 3 * L::HALO_PX; i += 128) {
            const int px = i % L::HALO_PX;
            const int cr = i / L::HALO_PX;
            const int r = cr % 3, c = cr / 3;
            int yy = y + r - 1;
            yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
            int xx = x0 + px - 1;
            xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
            const uint4 v = *reinterpret_cast<const uint4 *>(a.x + (size_t(yy) * W + xx) * CIN + 8 * c);
            *reinterpret_cast<uint4 *>(As + ((c * 3 + r) * L::HALO_PX + px) * 16) = v;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // ---- MMAs: 9 taps x CCH/2 K-steps of 16 ----
        if (tid == 0) {
            uint32_t acc = 0;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
#pragma unroll
                for (int k2 = 0; k2 < CCH / 2; ++k2) {
                    const uint64_t ad =
                        tc::make_desc(a_base + (((2 * k2) * 3 + ky) * L::HALO_PX + kx) * 16, A_LBO, A_SBO);
                    const uint64_t bd = tc::make_desc(b_base + ((t * CCH + 2 * k2) * NOUT) * 16, B_LBO, B_SBO);
                    tc::mma_bf16(tmem, ad, bd, IDESC, acc);
                    acc = 1;
                }
            }
            tc::mma_commit(&mbar);
        }
        __syncwarp();
        if (!tc::mbar_wait(&mbar, phase, 1u << 22)) {
            ok = false;
            if (lane == 0) atomicExch(a.error, 1);
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // ---- epilogue: thread = pixel x0 + tid (TMEM lane tid) ----
        const size_t p = size_t(y) * W + x0 + tid;
        const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll
        for (int cb = 0; cb < NOUT; cb += 32) {
            float v[32];
            if constexpr (NOUT >= 32) {
                tc::tmem_ld32(trow + cb, v);
            } else {
                float v16[32];
                tc::tmem_ld32(trow + cb, v16);  // columns beyond NOUT are allocated (32) and ignored
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = v16[i];
            }
            constexpr int NC = NOUT < 32 ? NOUT : 32;
            if (a.bias && a.epi != EPI_DGRAD) {
#pragma unroll
                for (int i = 0; i < NC; ++i) v[i] += a.bias[cb + i];
            }
            if (a.epi == EPI_GELU) {
                __nv_bfloat16 *zo = static_cast<__nv_bfloat16 *>(a.out0) + p * NOUT + cb;
                __nv_bfloat16 *ao = static_cast<__nv_bfloat16 *>(a.out1) + p * NOUT + cb;
                const __nv_bfloat16 *res = a.aux0 ? static_cast<const __nv_bfloat16 *>(a.aux0) + p * NOUT + cb : nullptr;
#pragma unroll
                for (int i = 0; i < NC; i += 2) {
                    float g0 = gelu_f(v[i]), g1 = gelu_f(v[i + 1]);
                    if (res) {
                        const __nv_bfloat162 r2 = *reinterpret_cast<const __nv_bfloat162 *>(res + i);
                        g0 += __bfloat162float(r2.x);
                        g1 += __bfloat162float(r2.y);
                    }
                    *reinterpret_cast<__nv_bfloat162 *>(zo + i) = __floats2bfloat162_rn(v[i], v[i + 1]);
                    *reinterpret_cast<__nv_bfloat162 *>(ao + i) = __floats2bfloat162_rn(g0, g1);
                }
            } else if (a.epi == EPI_LINEAR) {
                float *o = static_cast<float *>(a.out0) + p * NOUT + cb;
#pragma unroll
                for (int i = 0; i < NC; i += 4) *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            } else if (a.epi == EPI_DGRAD) {
                const float *gin = a.aux0 ? static_cast<const float *>(a.aux0) + p * NOUT + cb : nullptr;
                float *go = static_cast<float *>(a.out0) + p * NOUT + cb;
                __nv_bfloat16 *dz = static_cast<__nv_bfloat16 *>(a.out1) + p * NOUT + cb;
                const __nv_bfloat16 *zp = a.zprev + p * NOUT + cb;
#pragma unroll
                for (int i = 0; i < NC; i += 2) {
                    float g0 = v[i], g1 = v[i + 1];
                    if (gin) {
                        g0 += gin[i];
                        g1 += gin[i + 1];
                    }
                    go[i] = g0;
                    go[i + 1] = g1;
                    const __nv_bfloat162 z2 = *reinterpret_cast<const __nv_bfloat162 *>(zp + i);
                    *reinterpret_cast<__nv_bfloat162 *>(dz + i) = __floats2bfloat162_rn(
                        g0 * gelu_grad(__bfloat162float(z2.x)), g1 * gelu_grad(__bfloat162float(z2.y)));
                }
            } else {  // EPI_QUPDATE: channels 0..5 of the first column block
                if (cb == 0) {
                    const size_t P = size_t(H) * W;
                    const float *qi = static_cast<const float *>(a.aux0);
                    float *qo = static_cast<float *>(a.out0);
#pragma unroll
                    for (int c = 0; c < 6; ++c) qo[c * P + p] = qi[c * P + p] + a.scale * v[c];
                }
            }
        }
        tc::fence_before_sync();
        failed = __syncthreads_or(!ok);  // smem and TMEM free for the next tile; uniform exit on a timeout
        tc::fence_after_sync();
        if (failed) break;
    }
    if (failed) tc::mbar_wait(&mbar, phase ^ 1u, 1u << 22);  // let a late MMA finish before TMEM is freed
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
}

template <int CCH, int NOUT>
cudaError_t launch_conv_t(const ConvArgs &a, cudaStream_t st) {
    using L = ConvLayout<CCH, NOUT>;
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<CCH, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = a.H * (a.W / 128);
    const int grid = ntiles < sms ? ntiles : sms;
    conv3x3_tc_kernel<CCH, NOUT><<<grid, 128, L::SMEM, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv(int cin_chunks, int nout, const ConvArgs &a, cudaStream_t st) {
    if (cin_chunks == 2 && nout == 64) return launch_conv_t<2, 64>(a, st);
    if (cin_chunks == 8 && nout == 64) return launch_conv_t<8, 64>(a, st);
    if (cin_chunks == 8 && nout == 16) return launch_conv_t<8, 16>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace qla

extern "C" qla_status qla_conv3x3_bf16(const void *x, int H, int W, int cin, const void *w_packed, const float *bias,
                                       int nout, int epilogue, const void *aux0, const void *zprev, void *out0,
                                       void *out1, float scale, int *error_flag, void *stream) {
    if (!x || !w_packed || !out0 || !error_flag || H < 1 || W < 128 || W % 128 != 0) return QLA_EINVAL;
    if (!((cin == 16 && nout == 64) || (cin == 64 && nout == 64) || (cin == 64 && nout == 16))) return QLA_EUNSUPPORTED;
    if (epilogue < 0 || epilogue > 3) return QLA_EINVAL;
    if ((epilogue == qla::EPI_GELU || epilogue == qla::EPI_DGRAD) && !out1) return QLA_EINVAL;
    if (epilogue == qla::EPI_DGRAD && !zprev) return QLA_EINVAL;
    if (epilogue == qla::EPI_QUPDATE && (!aux0 || nout < 6)) return QLA_EINVAL;
    qla::ConvArgs a;
    a.x = static_cast<const __nv_bfloat16 *>(x);
    a.w = static_cast<const __nv_bfloat16 *>(w_packed);
    a.bias = bias;
    a.H = H;
    a.W = W;
    a.epi = epilogue;
    a.aux0 = aux0;
    a.zprev = static_cast<const __nv_bfloat16 *>(zprev);
    a.out0 = out0;
    a.out1 = out1;
    a.scale = scale;
    a.error = error_flag;
    const cudaError_t e = qla::launch_conv(cin / 8, nout, a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QLA_OK : QLA_ECUDA;
}

// ---------------------------------------------------------------------------
// Weight packing: FP32 w[nout][cin][3][3] -> BF16 [9][cin_pad/8][nout_pad][8]
// (the B operand layout of conv3x3_tc_kernel). With transpose_flip the packed
// operand is the adjoint convolution (input-gradient) of w:
// w'[c][n][ky][kx] = w[n][c][2-ky][2-kx].
// ---------------------------------------------------------------------------
namespace qla {

__global__ void pack_conv_weights_kernel(const float *__restrict__ w, int nout, int cin, int nout_pad, int cin_pad,
                                         int transpose_flip, __nv_bfloat16 *__restrict__ out) {
    const int total = 9 * cin_pad * nout_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int j = i % 8;
        const int n = (i / 8) % nout_pad;
        const int chunk = (i / (8 * nout_pad)) % (cin_pad / 8);
        const int t = i / (8 * nout_pad * (cin_pad / 8));
        const int c = chunk * 8 + j;
        const int ky = t / 3, kx = t % 3;
        float v = 0.0f;
        if (!transpose_flip) {
            if (n < nout && c < cin) v = w[((size_t(n) * cin + c) * 3 + ky) * 3 + kx];
        } else {
            // packed output channel n ranges over the original inputs, packed input c over the original outputs
            if (n < cin && c < nout) v = w[((size_t(c) * cin + n) * 3 + (2 - ky)) * 3 + (2 - kx)];
        }
        out[i] = __float2bfloat16_rn(v);
    }
}

}  // namespace qla

extern "C" qla_status qla_pack_conv_weights(const float *w, int nout, int cin, int nout_pad, int cin_pad,
                                            int transpose_flip, void *packed, void *stream) {
    if (!w || !packed || nout < 1 || cin < 1 || cin_pad % 8 != 0 || nout_pad % 8 != 0) return QLA_EINVAL;
    if (!transpose_flip && (nout > nout_pad || cin > cin_pad)) return QLA_EINVAL;
    if (transpose_flip && (cin > nout_pad || nout > cin_pad)) return QLA_EINVAL;
    const int total = 9 * cin_pad * nout_pad;
    qla::pack_conv_weights_kernel<<<(total + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w, nout, cin, nout_pad, cin_pad, transpose_flip, static_cast<__nv_bfloat16 *>(packed));
    return cudaGetLastError() == cudaSuccess ? QLA_OK : QLA_ECUDA;
}
