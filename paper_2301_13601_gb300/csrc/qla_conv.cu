// 3x3 convolution with circular padding on BF16 NHWC activations, as an
// implicit GEMM on the tcgen05 tensor cores with FP32 accumulation in TMEM.
//
// Activations hold nimg images of H x W stacked ([nimg][H][W][C]); each image
// is periodic on its own. One tile = 128 consecutive pixels of one image row
// (M = 128), all output
// channels (N = NOUT), K = 9 taps x input channels. The CTA stages the 3-row
// halo block (3 x 130 pixels x CIN channels) once per tile in the interleaved
// K-major layout, so the nine taps are nine shifted windows of the same block
// (no swizzle: any 16-byte aligned start is a valid operand). All 9 taps of the
// packed weights stay resident in shared memory. One thread issues the MMAs;
// the 128 threads (4 warps x 32 TMEM lanes) run the fused epilogue:
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
// chunk), then the packed weights of all nine taps, Bs[t][c][n][16 B].
template <int CCH, int NOUT>
struct ConvLayout {
    static constexpr int HALO_PX = 130;
    static constexpr int NS = 5;  // rows y-1..y+1 for the MMA of row y, y+2 waiting, y+3 loading
    static constexpr int A_BYTES = CCH * NS * HALO_PX * 16;
    static constexpr int B_BYTES = 9 * CCH * NOUT * 16;
    static constexpr int A_OFF = 0;
    static constexpr int B_OFF = ((A_BYTES + 1023) / 1024) * 1024;
    static constexpr int SMEM = B_OFF + B_BYTES;
    static constexpr int ACC_COLS = NOUT < 32 ? 32 : NOUT;  // TMEM columns of one accumulator
    static constexpr int TMEM_COLS = 2 * ACC_COLS;          // two accumulators
};

// Persistent conv kernel. Work = rows of 128-pixel column blocks, ordered
// (image, column block, row); each CTA takes a contiguous range and walks down
// its column blocks with a rolling window of halo rows, so every input row is
// loaded once per block. Per output row y (256 threads = 8 warps):
//   a) cp.async row y+3 into the ring (its slot was last read by the MMA of y-1)
//   b) wait for row y+2, fence, barrier
//   c) one thread issues the 9 x CCH/2 MMAs of row y+1 into the other accumulator
//   d) all wait for the MMAs of row y, then run the fused epilogue of row y
// so loads, tensor-core work and epilogue of three rows overlap.
// Epilogue: warp w reads TMEM lanes 32 (w % 4)... (its pixels) and the column
// half w / 4 (32 channels); for NOUT = 16 only warps 0-3 work.
template <int CCH, int NOUT>
__global__ void __launch_bounds__(256, 1) conv3x3_tc_kernel(const ConvArgs a) {
    using L = ConvLayout<CCH, NOUT>;
    constexpr int CIN = 8 * CCH;
    constexpr int NS = L::NS;
    constexpr int HP = L::HALO_PX;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
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
    const __nv_bfloat16 *xg = static_cast<const __nv_bfloat16 *>(a.x);

    {
        const uint4 *src = static_cast<const uint4 *>(a.w);
        for (int i = tid; i < 9 * CCH * NOUT; i += 256) cp_async16(Bs + i * 16, src + i);
        cp_async_commit();
        if (tid < 64) bias_s[tid] = (a.bias && tid < NOUT && a.epi != EPI_DGRAD) ? a.bias[tid] : 0.0f;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base_s, L::TMEM_COLS);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::fence_mbar_init();
    }
    cp_async_wait_0();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr uint32_t IDESC = tc::make_idesc_bf16(128, NOUT);
    const uint32_t a_base = tc::smem_addr(As), b_base = tc::smem_addr(Bs);
    constexpr uint32_t A_LBO = NS * HP * 16, A_SBO = 128;
    constexpr uint32_t B_LBO = NOUT * 16, B_SBO = 128;
    uint32_t ph[2] = {0u, 0u};
    int issued[2] = {0, 0}, waited[2] = {0, 0};
    bool failed = false;

    // epilogue role
    const int q = warp & 3, half = warp >> 2;
    const bool epi_on = (NOUT >= 64) || half == 0;
    const int m = 32 * q + lane;  // pixel within the column block (TMEM lane)
    const int cb0 = (NOUT >= 64 ? 32 * half : 0);
    const bool res_smem = a.epi == EPI_GELU && a.aux0 != nullptr && a.aux0 == a.x && CIN == NOUT;

    for (long long u0 = u_begin; u0 < u_end && !failed;) {
        // segment: consecutive rows of one column block of one image
        const int y_s = int(u0 % H);
        const long long t2 = u0 / H;
        const int cbk = int(t2 % TPR);
        const int img = int(t2 / TPR);
        const long long seg_end = (u0 - y_s + H) < u_end ? (u0 - y_s + H) : u_end;
        const int y_e = y_s + int(seg_end - u0) - 1;
        const int x0 = cbk * 128;
        const __nv_bfloat16 *ximg = xg + (size_t)img * H * W * CIN;
        // rows are addressed relative to y_s - 1: slot(r) = (r - y_s + 1) % NS
        auto load_row = [&](int r) {
            int yy = r % H;
            yy = yy < 0 ? yy + H : yy;
            const int slot = (r - y_s + 1) % NS;
            const __nv_bfloat16 *row = ximg + (size_t)yy * W * CIN;
            for (int i = tid; i < CCH * HP; i += 256) {
                const int px = i % HP, c = i / HP;
                int xx = x0 + px - 1;
                xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
                cp_async16(As + ((c * NS + slot) * HP + px) * 16, row + (size_t)xx * CIN + 8 * c);
            }
        };
        auto issue_mma = [&](int y, int acc) {
            const uint32_t d = tmem + acc * L::ACC_COLS;
            uint32_t accum = 0;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int slot = (y - 1 + ky - y_s + 1) % NS;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int t = ky * 3 + kx;
#pragma unroll
                    for (int k2 = 0; k2 < CCH / 2; ++k2) {
                        const uint64_t ad =
                            tc::make_desc(a_base + (((2 * k2) * NS + slot) * HP + kx) * 16, A_LBO, A_SBO);
                        const uint64_t bd = tc::make_desc(b_base + ((t * CCH + 2 * k2) * NOUT) * 16, B_LBO, B_SBO);
                        tc::mma_bf16(d, ad, bd, IDESC, accum);
                        accum = 1;
                    }
                }
            }
            tc::mma_commit(&mbar[acc]);
        };
        // prologue: rows y_s-1 .. y_s+1, then y_s+2
        load_row(y_s - 1);
        load_row(y_s);
        load_row(y_s + 1);
        cp_async_commit();
        if (y_s + 1 <= y_e) load_row(y_s + 2);
        cp_async_commit();
        cp_async_wait_1();
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) issue_mma(y_s, y_s & 1);
        issued[y_s & 1]++;
        for (int y = y_s; y <= y_e; ++y) {
            if (y + 2 <= y_e) load_row(y + 3);
            cp_async_commit();
            cp_async_wait_1();
            tc::fence_proxy_async();
            tc::fence_before_sync();
            if (__syncthreads_or(failed ? 1 : 0)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            if (y + 1 <= y_e) {
                if (tid == 0) issue_mma(y + 1, (y + 1) & 1);
                issued[(y + 1) & 1]++;
            }
            const int acc = y & 1;
            __syncwarp();
            if (!tc::mbar_wait(&mbar[acc], ph[acc], 1u << 22)) {
                failed = true;
                if (lane == 0) atomicExch(a.error, 1);
            }
            ph[acc] ^= 1u;
            waited[acc]++;
            tc::fence_after_sync();
            if (!epi_on || failed) continue;
            // ---- fused epilogue of row y: pixel p, channels cb0 .. cb0+31 ----
            const size_t p = ((size_t)img * H + y) * W + x0 + m;
            float v[32];
            tc::tmem_ld32(tmem + acc * L::ACC_COLS + cb0 + (uint32_t(32 * q) << 16), v);
            constexpr int NC = NOUT < 32 ? NOUT : 32;
#pragma unroll
            for (int i = 0; i < NC; ++i) v[i] += bias_s[cb0 + i];
            if (a.epi == EPI_GELU) {
                float r[32];
                if (res_smem) {
                    const int slot = (y - y_s + 1) % NS;
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        const uint4 w4 = *reinterpret_cast<const uint4 *>(
                            As + (((cb0 / 8 + c4) * NS + slot) * HP + m + 1) * 16);
                        const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            r[8 * c4 + 2 * k] = __uint_as_float(ww[k] << 16);
                            r[8 * c4 + 2 * k + 1] = __uint_as_float(ww[k] & 0xffff0000u);
                        }
                    }
                } else if (a.aux0) {
                    const uint4 *rp = reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(a.aux0) +
                                                                      p * NOUT + cb0);
#pragma unroll
                    for (int c4 = 0; c4 < NC / 8; ++c4) {
                        const uint4 w4 = rp[c4];
                        const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            r[8 * c4 + 2 * k] = __uint_as_float(ww[k] << 16);
                            r[8 * c4 + 2 * k + 1] = __uint_as_float(ww[k] & 0xffff0000u);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) r[i] = 0.0f;
                }
                uint4 *ao = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out1) + p * NOUT + cb0);
#pragma unroll
                for (int c4 = 0; c4 < NC / 8; ++c4) {
                    float g[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) g[k] = gelu_f(v[8 * c4 + k]) + r[8 * c4 + k];
                    ao[c4] = make_uint4(bf2(g[0], g[1]), bf2(g[2], g[3]), bf2(g[4], g[5]), bf2(g[6], g[7]));
                }
                if (a.out0) {
                    uint4 *zo = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out0) + p * NOUT + cb0);
#pragma unroll
                    for (int c4 = 0; c4 < NC / 8; ++c4) {
                        const float *z = v + 8 * c4;
                        zo[c4] = make_uint4(bf2(z[0], z[1]), bf2(z[2], z[3]), bf2(z[4], z[5]), bf2(z[6], z[7]));
                    }
                }
            } else if (a.epi == EPI_LINEAR) {
                float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out0) + p * NOUT + cb0);
#pragma unroll
                for (int i = 0; i < NC / 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            } else if (a.epi == EPI_DGRAD) {
                const float4 *gin =
                    a.aux0 ? reinterpret_cast<const float4 *>(static_cast<const float *>(a.aux0) + p * NOUT + cb0)
                           : nullptr;
                float4 *go = reinterpret_cast<float4 *>(static_cast<float *>(a.out0) + p * NOUT + cb0);
                const uint4 *zp =
                    reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(a.zprev) + p * NOUT + cb0);
                uint4 *dz = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out1) + p * NOUT + cb0);
#pragma unroll
                for (int c4 = 0; c4 < NC / 8; ++c4) {
                    float g[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) g[k] = v[8 * c4 + k];
                    if (gin) {
                        const float4 g0 = gin[2 * c4], g1 = gin[2 * c4 + 1];
                        g[0] += g0.x; g[1] += g0.y; g[2] += g0.z; g[3] += g0.w;
                        g[4] += g1.x; g[5] += g1.y; g[6] += g1.z; g[7] += g1.w;
                    }
                    go[2 * c4] = make_float4(g[0], g[1], g[2], g[3]);
                    go[2 * c4 + 1] = make_float4(g[4], g[5], g[6], g[7]);
                    const uint4 z4 = zp[c4];
                    const uint32_t zz[4] = {z4.x, z4.y, z4.z, z4.w};
                    float d[8];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        d[2 * k] = g[2 * k] * gelu_grad(__uint_as_float(zz[k] << 16));
                        d[2 * k + 1] = g[2 * k + 1] * gelu_grad(__uint_as_float(zz[k] & 0xffff0000u));
                    }
                    dz[c4] = make_uint4(bf2(d[0], d[1]), bf2(d[2], d[3]), bf2(d[4], d[5]), bf2(d[6], d[7]));
                }
            } else if (cb0 == 0) {  // EPI_QUPDATE: channels 0..5
                const size_t P = (size_t)H * W;
                const size_t pix = (size_t)y * W + x0 + m;
                const float *qi = static_cast<const float *>(a.aux0) + (size_t)img * 6 * P;
                float *qo = static_cast<float *>(a.out0) + (size_t)img * 6 * P;
#pragma unroll
                for (int c = 0; c < 6; ++c) qo[c * P + pix] = qi[c * P + pix] + a.scale * v[c];
            }
        }
        if (__syncthreads_or(failed ? 1 : 0)) failed = true;  // uniform exit after a segment
        u0 = seg_end;
    }
    // drain: let outstanding copies and MMAs finish (bounded) before TMEM is freed
    cp_async_wait_0();
    for (int b = 0; b < 2; ++b) {
        while (waited[b] < issued[b]) {
            if (!tc::mbar_wait(&mbar[b], ph[b], 1u << 22) && lane == 0) atomicExch(a.error, 1);
            ph[b] ^= 1u;
            waited[b]++;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
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
    const long long rows = (long long)a.nimg * a.H * (a.W / 128);
    const int grid = rows < sms ? int(rows) : sms;
    conv3x3_tc_kernel<CCH, NOUT><<<grid, 256, L::SMEM, st>>>(a);
    return cudaGetLastError();
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
