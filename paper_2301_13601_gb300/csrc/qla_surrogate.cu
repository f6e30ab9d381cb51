// Learned time-stepping surrogate: a 6-layer residual CNN that advances the
// six fields of the QLA state (Sec. 4 scattering problem) by K QLA steps per
// call, Q_{t+K} = Q_t + s * f([Q_t, n_x, n_y, n_z]):
//   a0 = GELU(conv0(x0));  a_l = a_{l-1} + GELU(conv_l(a_{l-1})), l = 1..4;
//   f  = conv5(a4)   (3x3 circular convolutions, 64 hidden channels).
// The forward and input-gradient convolutions run on the tcgen05 tensor cores
// (qla_conv.cu), and so do the weight gradients (pixels as the reduction
// dimension, per-CTA partial sums reduced in a fixed order); the optimiser
// is Adam on FP32 master weights that are re-packed to BF16 after every
// update. The input x0 carries each field as two BF16 parts
// (high and low) that share first-layer weights, so the network sees the
// FP32 state to about 16 significant bits, plus n in BF16.
//
// The rollout advances a QLA context by calls of the network, checks the
// energy (Eq. 27) after each call and falls back to K plain QLA steps from the
// unchanged state when the relative drift exceeds the tolerance.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/qla_surrogate.h"
#include "qla_internal.h"

namespace qla {
namespace sg {

constexpr int NL = 6;
constexpr int HID = 64;
constexpr int CIN[NL] = {9, 64, 64, 64, 64, 64};    // logical input channels
constexpr int CINP[NL] = {16, 64, 64, 64, 64, 64};  // packed input channels
constexpr int NOUT[NL] = {64, 64, 64, 64, 64, 6};   // logical output channels
constexpr int NOUTP[NL] = {64, 64, 64, 64, 64, 16};
constexpr int X0C = 16;                              // x0 channels: Q hi (6), Q lo (6), n (3), 0
constexpr int BIAS_BLOCKS = 256;                     // pixel splits of the bias-gradient reduction
constexpr int RED_BLOCKS = 512;                      // partial sums of the loss reductions

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// ---- input: FP32 planes -> BF16 NHWC x0 ----------------------------------
__global__ void input_pack_kernel(const float *__restrict__ q, const float *__restrict__ n, int nimg, long long P,
                                  uint4 *__restrict__ x0) {
    const long long NP = nimg * P;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP; p += (long long)gridDim.x * blockDim.x) {
        const long long img = p / P, pix = p - img * P;
        const float *qi = q + img * 6 * P + pix;
        const float *ni = n + img * 3 * P + pix;
        float hi[6], lo[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float f = qi[c * P];
            hi[c] = __bfloat162float(__float2bfloat16_rn(f));
            lo[c] = f - hi[c];
        }
        const float n0 = ni[0], n1 = ni[P], n2 = ni[2 * P];
        x0[2 * p] = make_uint4(pack_bf2(hi[0], hi[1]), pack_bf2(hi[2], hi[3]), pack_bf2(hi[4], hi[5]),
                               pack_bf2(lo[0], lo[1]));
        x0[2 * p + 1] = make_uint4(pack_bf2(lo[2], lo[3]), pack_bf2(lo[4], lo[5]), pack_bf2(n0, n1),
                                   pack_bf2(n2, 0.0f));
    }
}

// ---- reductions (fixed order: deterministic) -----------------------------
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// part[b] = sum over this block's elements of (t - q)^2
__global__ void dq_sumsq_kernel(const float *__restrict__ qt, const float *__restrict__ qin, long long n,
                                double *__restrict__ part) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = double(qt[i]) - double(qin[i]);
        acc += d * d;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// part[b] = sum over this block's elements of q^2: FP32 squares summed per
// thread (a few dozen terms), FP64 across threads and blocks. Accurate to
// ~1e-6 relative, ample for a drift check at 1e-3; a non-finite element makes
// the sum non-finite.
__global__ void sumsq_kernel(const float *__restrict__ q, long long n, double *__restrict__ part) {
    float acc = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fmaf(q[i], q[i], acc);
    const double s = block_sum(double(acc));
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void finalize_kernel(const double *__restrict__ part, int nb, double *__restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) *out = s;
}

// Loss L = sum (s*f - dQ)^2 / sum dQ^2 over the batch; writes dL/df as BF16
// [NP][16] (channels 6-15 zero) and partial sums of the numerator.
__global__ void loss_grad_kernel(const float *__restrict__ f, const float *__restrict__ qin,
                                 const float *__restrict__ qt, int nimg, long long P, float scale,
                                 const double *__restrict__ den, uint4 *__restrict__ g6, double *__restrict__ part) {
    const double d = *den > 1e-300 ? *den : 1e-300;
    const float inv = float(2.0 * scale / d);
    const long long NP = nimg * P;
    double acc = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP; p += (long long)gridDim.x * blockDim.x) {
        const long long img = p / P, pix = p - img * P;
        const float4 f0 = *reinterpret_cast<const float4 *>(f + p * 16);
        const float2 f1 = *reinterpret_cast<const float2 *>(f + p * 16 + 4);
        const float fv[6] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y};
        float g[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const long long k = (img * 6 + c) * P + pix;
            const float dq = qt[k] - qin[k];
            const float r = scale * fv[c] - dq;
            acc += double(r) * double(r);
            g[c] = r * inv;
        }
        g6[2 * p] = make_uint4(pack_bf2(g[0], g[1]), pack_bf2(g[2], g[3]), pack_bf2(g[4], g[5]), 0u);
        g6[2 * p + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ---- bias gradient: partial sums of g over pixel ranges -------------------
// 16-byte loads: NT/8 threads per pixel, 256 / (NT/8) pixels per pass.
template <int NT>
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ g, long long NP, float *__restrict__ bpart) {
    constexpr int TPP = NT / 8;       // threads per pixel
    constexpr int PPB = 256 / TPP;    // pixels per pass
    __shared__ float sh[PPB][NT + 1];
    const int c8 = threadIdx.x % TPP, pl = threadIdx.x / TPP;
    const long long per = (NP + gridDim.x - 1) / gridDim.x;
    const long long b = blockIdx.x * per, e = b + per < NP ? b + per : NP;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long p = b + pl; p < e; p += PPB) {
        const uint4 v = *reinterpret_cast<const uint4 *>(g + p * NT + 8 * c8);
        acc[0] += bf_lo(v.x); acc[1] += bf_hi(v.x); acc[2] += bf_lo(v.y); acc[3] += bf_hi(v.y);
        acc[4] += bf_lo(v.z); acc[5] += bf_hi(v.z); acc[6] += bf_lo(v.w); acc[7] += bf_hi(v.w);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[pl][8 * c8 + k] = acc[k];
    __syncthreads();
    if (threadIdx.x < NT) {
        float t = 0.0f;
        for (int k = 0; k < PPB; ++k) t += sh[k][threadIdx.x];
        bpart[size_t(blockIdx.x) * NT + threadIdx.x] = t;
    }
}

// Sum the per-CTA partials part[S][9][NT][CT] and bias partials bpart[SB][NT]
// in a fixed order into the logical gradient layout gw[n][c][ky][kx], gb[n];
// tied: packed input channels c and c+6 (c < 6) both belong to logical c,
// packed 12-14 to logical 6-8.
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int S, const float *__restrict__ bpart, int SB,
                                    int NT, int CT, int nout, int cin, int tied, float *__restrict__ gw,
                                    float *__restrict__ gb) {
    const int total = nout * cin * 9;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) {
        // c fastest: consecutive threads read consecutive partials
        const int c = i % cin, n = (i / cin) % nout, t = i / (cin * nout);
        const int c1 = tied ? (c < 6 ? c : c + 6) : c;
        const int c2 = (tied && c < 6) ? c + 6 : -1;
        float acc = 0.0f;
        for (int s = 0; s < S; ++s) {
            const float *o = part + ((size_t(s) * 9 + t) * NT + n) * CT;
            acc += o[c1];
            if (c2 >= 0) acc += o[c2];
        }
        gw[(n * cin + c) * 9 + t] = acc;
    } else if (i < total + nout) {
        const int n = i - total;
        float acc = 0.0f;
        for (int s = 0; s < SB; ++s) acc += bpart[size_t(s) * NT + n];
        gb[n] = acc;
    }
}

// ---- Adam on the flat FP32 parameter vector --------------------------------
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr_t, float b1, float b2, float eps_t) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr_t * mi / (sqrtf(vi) + eps_t);
    }
}

__global__ void pad_bias_kernel(const float *__restrict__ b, int n, int npad, float *__restrict__ out) {
    const int i = threadIdx.x;
    if (i < npad) out[i] = i < n ? b[i] : 0.0f;
}

}  // namespace sg
}  // namespace qla

using namespace qla;
using namespace qla::sg;

struct qla_surrogate {
    qla_surrogate_config cfg{};
    int dev = 0;
    int sms = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long P = 0, NP = 0;
    void *arena = nullptr;
    long long nparam = 0;
    long long off_w[NL] = {}, off_b[NL] = {};
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    void *wf[NL] = {}, *wb[NL] = {};
    float *bpad[NL] = {};
    void *x0 = nullptr, *z[5] = {}, *act[5] = {}, *g6 = nullptr, *dz[2] = {};
    float *fout = nullptr, *da[2] = {};
    float *wpart = nullptr, *bpart = nullptr;
    double *red = nullptr, *scal = nullptr;  // scal[0] = sum dQ^2, scal[1] = sum residual^2
    int *err = nullptr;
    double *host_scal = nullptr;  // pinned [4]: loss sums, rollout energies (two slots)
    int *host_err = nullptr;      // pinned
    float *qspec = nullptr;       // third state buffer of a one-image surrogate (speculative rollout calls)
    cudaEvent_t ev[2] = {nullptr, nullptr};  // rollout: a call's energy has reached the host
    bool packed = false;
    long long adam_t = 0;
    qla_status sticky = QLA_OK;
    std::string msg;
};

namespace {

qla_status sfail(qla_surrogate *s, qla_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (s) {
        if ((st == QLA_ECUDA || st == QLA_ETIMEOUT) && s->sticky == QLA_OK) s->sticky = st;
        s->msg = buf;
    }
    return st;
}

#define SG_CUDA(s, call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return sfail((s), QLA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

qla_status enter(qla_surrogate *s) {
    if (!s) return QLA_EINVAL;
    if (s->sticky != QLA_OK) return s->sticky;
    if (cudaSetDevice(s->dev) != cudaSuccess) return sfail(s, QLA_ECUDA, "cudaSetDevice failed");
    return QLA_OK;
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

int grid_for(long long n, int block, int sms) {
    long long g = (n + block - 1) / block;
    const long long cap = (long long)sms * 8;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

qla_status conv(qla_surrogate *s, int cin, int nout, const void *x, const void *w, const float *bias, int epi,
                const void *aux0, const void *zprev, void *out0, void *out1, float scale, cudaStream_t st) {
    ConvArgs a;
    a.x = x;
    a.w = w;
    a.bias = bias;
    a.nimg = s->cfg.nimg;
    a.H = s->cfg.H;
    a.W = s->cfg.W;
    a.epi = epi;
    a.aux0 = aux0;
    a.zprev = zprev;
    a.out0 = out0;
    a.out1 = out1;
    a.scale = scale;
    a.error = s->err;
    SG_CUDA(s, launch_conv(cin, nout, a, st));
    return QLA_OK;
}

qla_status repack(qla_surrogate *s, cudaStream_t st) {
    for (int l = 0; l < NL; ++l) {
        const float *w = s->params + s->off_w[l];
        SG_CUDA(s, launch_pack_weights(w, NOUT[l], CIN[l], NOUTP[l], CINP[l], l == 0 ? PACK_TIED_INPUT : PACK_PLAIN,
                                       s->wf[l], st));
        if (l > 0 && s->wb[l])
            SG_CUDA(s, launch_pack_weights(w, NOUT[l], CIN[l], CINP[l], NOUTP[l], PACK_ADJOINT, s->wb[l], st));
        pad_bias_kernel<<<1, 64, 0, st>>>(s->params + s->off_b[l], NOUT[l], NOUTP[l], s->bpad[l]);
        SG_CUDA(s, cudaGetLastError());
    }
    s->packed = true;
    return QLA_OK;
}

qla_status pack_input(qla_surrogate *s, const float *q, const float *n, cudaStream_t st) {
    input_pack_kernel<<<grid_for(s->NP, 256, s->sms), 256, 0, st>>>(q, n, s->cfg.nimg, s->P,
                                                                    static_cast<uint4 *>(s->x0));
    SG_CUDA(s, cudaGetLastError());
    return QLA_OK;
}

// Inference: q_out = q_in + s f (activations ping-pong through act[0], act[1]).
qla_status forward_infer(qla_surrogate *s, const float *q_in, const float *n, float *q_out, cudaStream_t st) {
    qla_status r = pack_input(s, q_in, n, st);
    if (r != QLA_OK) return r;
    r = conv(s, CINP[0], NOUTP[0], s->x0, s->wf[0], s->bpad[0], QLA_EPI_GELU, nullptr, nullptr, nullptr, s->act[0],
             1.0f, st);
    for (int l = 1; l < 5 && r == QLA_OK; ++l) {
        const void *in = s->act[(l - 1) & 1];
        r = conv(s, HID, HID, in, s->wf[l], s->bpad[l], QLA_EPI_GELU, in, nullptr, nullptr, s->act[l & 1], 1.0f, st);
    }
    if (r != QLA_OK) return r;
    return conv(s, HID, NOUTP[5], s->act[0], s->wf[5], s->bpad[5], QLA_EPI_QUPDATE, q_in, nullptr, q_out, nullptr,
                s->cfg.out_scale, st);
}

// Training forward: keeps z_l and a_l; f (FP32 [NP][16]) into fout.
qla_status forward_train(qla_surrogate *s, const float *q_in, const float *n, cudaStream_t st) {
    qla_status r = pack_input(s, q_in, n, st);
    if (r != QLA_OK) return r;
    r = conv(s, CINP[0], NOUTP[0], s->x0, s->wf[0], s->bpad[0], QLA_EPI_GELU, nullptr, nullptr, s->z[0], s->act[0],
             1.0f, st);
    for (int l = 1; l < 5 && r == QLA_OK; ++l)
        r = conv(s, HID, HID, s->act[l - 1], s->wf[l], s->bpad[l], QLA_EPI_GELU, s->act[l - 1], nullptr, s->z[l],
                 s->act[l], 1.0f, st);
    if (r != QLA_OK) return r;
    return conv(s, HID, NOUTP[5], s->act[4], s->wf[5], s->bpad[5], QLA_EPI_LINEAR, nullptr, nullptr, s->fout,
                nullptr, 1.0f, st);
}

// Weight and bias gradient of layer l: x = the layer's input (cs channels),
// g = dL/dz of the layer (nt channels).
qla_status wgrad(qla_surrogate *s, int l, const void *x, int cs, const void *g, int nt, cudaStream_t st) {
    WgradArgs w;
    w.x = x;
    w.cs = cs;
    w.g = g;
    w.nt = nt;
    w.nimg = s->cfg.nimg;
    w.H = s->cfg.H;
    w.W = s->cfg.W;
    w.part = s->wpart;
    w.error = s->err;
    int S = 0;
    SG_CUDA(s, launch_wgrad_tc(w, &S, st));
    if (nt == 64)
        bias_grad_kernel<64><<<BIAS_BLOCKS, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(g), s->NP, s->bpart);
    else
        bias_grad_kernel<16><<<BIAS_BLOCKS, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(g), s->NP, s->bpart);
    SG_CUDA(s, cudaGetLastError());
    const int total = NOUT[l] * CIN[l] * 9 + NOUT[l];
    wgrad_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(s->wpart, S, s->bpart, BIAS_BLOCKS, nt, 64, NOUT[l],
                                                             CIN[l], l == 0 ? 1 : 0, s->grads + s->off_w[l],
                                                             s->grads + s->off_b[l]);
    SG_CUDA(s, cudaGetLastError());
    return QLA_OK;
}

// Loss and gradient of L = sum (s f - (q_t - q_in))^2 / sum (q_t - q_in)^2.
qla_status loss_and_grad(qla_surrogate *s, const float *q_in, const float *n, const float *q_t, cudaStream_t st) {
    if (!s->packed) {
        qla_status r = repack(s, st);
        if (r != QLA_OK) return r;
    }
    qla_status r = forward_train(s, q_in, n, st);
    if (r != QLA_OK) return r;
    const long long nq = s->NP * 6;
    dq_sumsq_kernel<<<RED_BLOCKS, 256, 0, st>>>(q_t, q_in, nq, s->red);
    finalize_kernel<<<1, 256, 0, st>>>(s->red, RED_BLOCKS, s->scal);
    loss_grad_kernel<<<RED_BLOCKS, 256, 0, st>>>(s->fout, q_in, q_t, s->cfg.nimg, s->P, s->cfg.out_scale, s->scal,
                                                 static_cast<uint4 *>(s->g6), s->red);
    finalize_kernel<<<1, 256, 0, st>>>(s->red, RED_BLOCKS, s->scal + 1);
    SG_CUDA(s, cudaGetLastError());
    // layer 5: dgrad into da_4 (a_4 feeds only layer 5), dz_4 = da_4 GELU'(z_4)
    r = conv(s, NOUTP[5], HID, s->g6, s->wb[5], nullptr, QLA_EPI_DGRAD, nullptr, s->z[4], s->da[0], s->dz[0], 1.0f,
             st);
    if (r == QLA_OK) r = wgrad(s, 5, s->act[4], HID, s->g6, 16, st);
    // layers 4..1: da_{l-1} = da_l + dgrad_l(dz_l); dz_{l-1} = da_{l-1} GELU'(z_{l-1})
    int cur = 0;
    for (int l = 4; l >= 1 && r == QLA_OK; --l) {
        r = conv(s, HID, HID, s->dz[cur], s->wb[l], nullptr, QLA_EPI_DGRAD, s->da[cur], s->z[l - 1], s->da[cur ^ 1],
                 s->dz[cur ^ 1], 1.0f, st);
        if (r == QLA_OK) r = wgrad(s, l, s->act[l - 1], HID, s->dz[cur], HID, st);
        cur ^= 1;
    }
    if (r == QLA_OK) r = wgrad(s, 0, s->x0, X0C, s->dz[cur], HID, st);
    return r;
}

qla_status check_err(qla_surrogate *s, cudaStream_t st) {
    SG_CUDA(s, cudaMemcpyAsync(s->host_err, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA(s, cudaStreamSynchronize(st));
    if (*s->host_err) return sfail(s, QLA_ETIMEOUT, "a tensor-core wait ran out of its limit");
    return QLA_OK;
}

// splitmix64 and Box-Muller: deterministic host-side initial weights
uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double normal(uint64_t &st) {
    const double u1 = (double(splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = double(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

}  // namespace

extern "C" {

long long qla_surrogate_param_count(void) {
    long long n = 0;
    for (int l = 0; l < NL; ++l) n += (long long)NOUT[l] * CIN[l] * 9 + NOUT[l];
    return n;
}

qla_status qla_surrogate_create(const qla_surrogate_config *cfg, qla_surrogate **out) {
    if (!cfg || !out) return QLA_EINVAL;
    *out = nullptr;
    const qla_surrogate_config c = *cfg;
    if (c.nimg < 1 || c.H < 1 || c.W < 128 || c.W % 128 != 0 || c.K < 1) return QLA_EINVAL;
    if ((long long)c.nimg * c.H * c.W > (1LL << 31) - 1) return QLA_EINVAL;
    if (!(c.out_scale > 0.0f) || !isfinite(c.out_scale)) return QLA_EINVAL;
    qla_surrogate *s = new qla_surrogate();
    s->cfg = c;
    s->P = (long long)c.H * c.W;
    s->NP = s->P * c.nimg;
    cudaGetDevice(&s->dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->dev);
    if (c.stream) {
        s->stream = static_cast<cudaStream_t>(c.stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return QLA_ECUDA;
        }
        s->own_stream = true;
    }
    long long off = 0;
    for (int l = 0; l < NL; ++l) {
        s->off_w[l] = off;
        off += (long long)NOUT[l] * CIN[l] * 9;
        s->off_b[l] = off;
        off += NOUT[l];
    }
    s->nparam = off;
    const bool train = c.train != 0;
    const size_t NP = size_t(s->NP);
    std::vector<size_t> sizes;
    auto add = [&](size_t b) { sizes.push_back(al(b)); };
    add(s->nparam * 4);  // params
    add(train ? s->nparam * 4 : 0);
    add(train ? s->nparam * 4 : 0);
    add(train ? s->nparam * 4 : 0);
    for (int l = 0; l < NL; ++l) add(size_t(9) * CINP[l] * NOUTP[l] * 2);                        // wf
    for (int l = 0; l < NL; ++l) add(train && l > 0 ? size_t(9) * CINP[l] * NOUTP[l] * 2 : 0);   // wb
    for (int l = 0; l < NL; ++l) add(64 * 4);                                                    // bpad
    add(NP * X0C * 2);                                                                           // x0
    for (int l = 0; l < 5; ++l) add(train ? NP * HID * 2 : 0);                                   // z
    for (int l = 0; l < 5; ++l) add((train || l < 2) ? NP * HID * 2 : 0);                        // act
    add(train ? NP * 16 * 2 : 0);                                                                // g6
    for (int k = 0; k < 2; ++k) add(train ? NP * HID * 2 : 0);                                   // dz
    add(train ? NP * 16 * 4 : 0);                                                                // fout
    for (int k = 0; k < 2; ++k) add(train ? NP * HID * 4 : 0);                                   // da
    add(train ? size_t(s->sms) * 9 * HID * HID * 4 : 0);                                         // wpart (per CTA)
    add(train ? size_t(BIAS_BLOCKS) * HID * 4 : 0);                                              // bpart
    add(RED_BLOCKS * 8);                                                                         // red
    add(4 * 8);                                                                                  // scal
    add(sizeof(int));                                                                            // err
    add(c.nimg == 1 ? size_t(6) * size_t(s->P) * 4 : 0);                                         // qspec
    size_t total = 0;
    for (size_t b : sizes) total += b;
    if (cudaMalloc(&s->arena, total) != cudaSuccess) {
        cudaGetLastError();
        qla_surrogate_destroy(s);
        return QLA_ENOMEM;
    }
    char *p = static_cast<char *>(s->arena);
    size_t k = 0;
    auto take = [&]() -> void * {
        void *r = sizes[k] ? p : nullptr;
        p += sizes[k++];
        return r;
    };
    s->params = static_cast<float *>(take());
    s->grads = static_cast<float *>(take());
    s->adam_m = static_cast<float *>(take());
    s->adam_v = static_cast<float *>(take());
    for (int l = 0; l < NL; ++l) s->wf[l] = take();
    for (int l = 0; l < NL; ++l) s->wb[l] = take();
    for (int l = 0; l < NL; ++l) s->bpad[l] = static_cast<float *>(take());
    s->x0 = take();
    for (int l = 0; l < 5; ++l) s->z[l] = take();
    for (int l = 0; l < 5; ++l) s->act[l] = take();
    s->g6 = take();
    for (int j = 0; j < 2; ++j) s->dz[j] = take();
    s->fout = static_cast<float *>(take());
    for (int j = 0; j < 2; ++j) s->da[j] = static_cast<float *>(take());
    s->wpart = static_cast<float *>(take());
    s->bpart = static_cast<float *>(take());
    s->red = static_cast<double *>(take());
    s->scal = static_cast<double *>(take());
    s->err = static_cast<int *>(take());
    s->qspec = static_cast<float *>(take());
    if (cudaMallocHost(&s->host_scal, 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&s->host_err, sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        qla_surrogate_destroy(s);
        return QLA_ENOMEM;
    }
    if (cudaMemsetAsync(s->arena, 0, total, s->stream) != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess) {
        qla_surrogate_destroy(s);
        return QLA_ECUDA;
    }
    *out = s;
    return QLA_OK;
}

qla_status qla_surrogate_init_params(qla_surrogate *s, unsigned long long seed) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    std::vector<float> h(size_t(s->nparam), 0.0f);
    uint64_t st = seed * 0x2545F4914F6CDD1Dull + 1;
    for (int l = 0; l < NL; ++l) {
        const double sd = sqrt(2.0 / (9.0 * CIN[l])) * (l == NL - 1 ? 0.1 : 1.0);
        for (long long i = 0; i < (long long)NOUT[l] * CIN[l] * 9; ++i) h[size_t(s->off_w[l] + i)] = float(sd * normal(st));
    }
    return qla_surrogate_set_params(s, h.data());
}

qla_status qla_surrogate_set_params(qla_surrogate *s, const float *host) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    if (!host) return sfail(s, QLA_EINVAL, "set_params: NULL");
    for (long long i = 0; i < s->nparam; ++i)
        if (!isfinite(host[i])) return sfail(s, QLA_EINVAL, "set_params: non-finite value at %lld", i);
    SG_CUDA(s, cudaMemcpyAsync(s->params, host, size_t(s->nparam) * 4, cudaMemcpyHostToDevice, s->stream));
    if (s->adam_m) {
        SG_CUDA(s, cudaMemsetAsync(s->adam_m, 0, size_t(s->nparam) * 4, s->stream));
        SG_CUDA(s, cudaMemsetAsync(s->adam_v, 0, size_t(s->nparam) * 4, s->stream));
    }
    s->adam_t = 0;
    r = repack(s, s->stream);
    if (r != QLA_OK) return r;
    SG_CUDA(s, cudaStreamSynchronize(s->stream));
    return QLA_OK;
}

qla_status qla_surrogate_get_params(qla_surrogate *s, float *host) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    if (!host) return sfail(s, QLA_EINVAL, "get_params: NULL");
    SG_CUDA(s, cudaMemcpyAsync(host, s->params, size_t(s->nparam) * 4, cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(s, cudaStreamSynchronize(s->stream));
    return QLA_OK;
}

qla_status qla_surrogate_forward(qla_surrogate *s, const float *q_in, const float *n, float *q_out) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    if (!q_in || !n || !q_out) return sfail(s, QLA_EINVAL, "forward: NULL pointer");
    if (!s->packed) {
        r = repack(s, s->stream);
        if (r != QLA_OK) return r;
    }
    return forward_infer(s, q_in, n, q_out, s->stream);
}

qla_status qla_surrogate_loss_grad(qla_surrogate *s, const float *q_in, const float *n, const float *q_target,
                                   double *loss, float *grad_host) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    if (!s->grads) return sfail(s, QLA_ESTATE, "loss_grad: created without training buffers");
    if (!q_in || !n || !q_target) return sfail(s, QLA_EINVAL, "loss_grad: NULL pointer");
    r = loss_and_grad(s, q_in, n, q_target, s->stream);
    if (r != QLA_OK) return r;
    if (loss) SG_CUDA(s, cudaMemcpyAsync(s->host_scal, s->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (grad_host)
        SG_CUDA(s, cudaMemcpyAsync(grad_host, s->grads, size_t(s->nparam) * 4, cudaMemcpyDeviceToHost, s->stream));
    if (loss || grad_host) {
        r = check_err(s, s->stream);
        if (r != QLA_OK) return r;
    }
    if (loss) *loss = s->host_scal[1] / (s->host_scal[0] > 1e-300 ? s->host_scal[0] : 1e-300);
    return QLA_OK;
}

qla_status qla_surrogate_adam_step(qla_surrogate *s, float lr, float beta1, float beta2, float eps) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    if (!s->grads) return sfail(s, QLA_ESTATE, "adam_step: created without training buffers");
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return sfail(s, QLA_EINVAL, "adam_step: bad hyper-parameters");
    s->adam_t += 1;
    const double bc1 = 1.0 - pow(double(beta1), double(s->adam_t));
    const double bc2 = 1.0 - pow(double(beta2), double(s->adam_t));
    const float lr_t = float(lr * sqrt(bc2) / bc1);
    const float eps_t = float(eps * sqrt(bc2));
    adam_kernel<<<grid_for(s->nparam, 256, s->sms), 256, 0, s->stream>>>(s->params, s->grads, s->adam_m, s->adam_v,
                                                                          s->nparam, lr_t, beta1, beta2, eps_t);
    SG_CUDA(s, cudaGetLastError());
    return repack(s, s->stream);
}

qla_status qla_surrogate_train_step(qla_surrogate *s, const float *q_in, const float *n, const float *q_target,
                                    float lr, double *loss) {
    qla_status r = qla_surrogate_loss_grad(s, q_in, n, q_target, loss, nullptr);
    if (r != QLA_OK) return r;
    return qla_surrogate_adam_step(s, lr, 0.9f, 0.999f, 1e-8f);
}

qla_status qla_surrogate_synchronize(qla_surrogate *s) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    return check_err(s, s->stream);
}

qla_status qla_surrogate_rollout(qla_surrogate *s, qla_ctx *ctx, const float *n, int calls, double drift_tol,
                                 int drift_mode, double energy_ref, qla_rollout_stats *stats) {
    qla_status r = enter(s);
    if (r != QLA_OK) return r;
    CtxView v;
    const bool serial = (drift_mode & QLA_ROLLOUT_SERIAL) != 0;
    const int mode = drift_mode & ~QLA_ROLLOUT_SERIAL;
    if (!ctx || !n || calls < 0 || !(drift_tol >= 0.0) || !ctx_view(ctx, &v) ||
        (mode != QLA_DRIFT_PER_CALL && mode != QLA_DRIFT_FROM_START))
        return sfail(s, QLA_EINVAL, "rollout: bad argument");
    if (v.precision != QLA_FP32) return sfail(s, QLA_EUNSUPPORTED, "rollout: the context must be FP32");
    if (v.families != QLA_FAMILIES_BOTH)  // the network writes all six components
        return sfail(s, QLA_EUNSUPPORTED, "rollout: the context must advance both families");
    if (s->cfg.nimg != 1 || v.Nx != s->cfg.W || v.Ny != s->cfg.H)
        return sfail(s, QLA_EINVAL, "rollout: lattice %dx%d does not match the surrogate's %dx%d (one image)", v.Nx,
                     v.Ny, s->cfg.W, s->cfg.H);
    if (!v.has_state) return sfail(s, QLA_ESTATE, "rollout: the context has no state");
    SG_CUDA(s, cudaStreamSynchronize(s->stream));  // pending surrogate work (weights) before the context's stream
    if (!s->packed) {
        r = repack(s, v.stream);
        if (r != QLA_OK) return r;
    }
    const cudaStream_t st = v.stream;
    const double sites = double(v.Nx) * v.Ny;
    // Eq. 27 energy (mean over sites of Q.Q) of a state: one light reduction
    // (the full diagnostics add div B and compensated FP64 sums, which the
    // drift check does not need and which cost more than the check), its
    // result and the error flag copied to pinned host slot `slot`.
    auto launch_energy = [&](const void *q, int slot) -> qla_status {
        sumsq_kernel<<<RED_BLOCKS, 256, 0, st>>>(static_cast<const float *>(q), 6LL * v.Nx * v.Ny, s->red);
        finalize_kernel<<<1, 256, 0, st>>>(s->red, RED_BLOCKS, s->scal + 2 + slot);
        SG_CUDA(s, cudaGetLastError());
        SG_CUDA(s, cudaMemcpyAsync(s->host_scal + 2 + slot, s->scal + 2 + slot, sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
        SG_CUDA(s, cudaMemcpyAsync(s->host_err, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SG_CUDA(s, cudaEventRecord(s->ev[slot], st));
        return QLA_OK;
    };
    auto read_energy = [&](int slot, double *e, bool *finite) -> qla_status {
        SG_CUDA(s, cudaEventSynchronize(s->ev[slot]));
        if (*s->host_err) return sfail(s, QLA_ETIMEOUT, "rollout: a tensor-core wait ran out of its limit");
        *e = s->host_scal[2 + slot] / sites;
        *finite = isfinite(*e) != 0;
        return QLA_OK;
    };
    auto energy = [&](const void *q, double *e, bool *finite) -> qla_status {
        qla_status rr = launch_energy(q, 0);
        return rr == QLA_OK ? read_energy(0, e, finite) : rr;
    };
    qla_rollout_stats stt{};
    bool fin = true;
    double e_start = 0.0;
    r = energy(v.cur_state, &e_start, &fin);
    if (r != QLA_OK) return r;
    if (!fin || !(e_start > 0.0)) return sfail(s, QLA_ESTATE, "rollout: initial state has no finite energy");
    stt.energy_ref = (mode == QLA_DRIFT_FROM_START && energy_ref > 0.0 && isfinite(energy_ref)) ? energy_ref : e_start;
    double e_cur = e_start;  // energy of the current state (reference of the per-call check)
    // the decision on one proposal of energy e (updates the statistics)
    auto accept = [&](double e, bool finite) {
        const double ref = mode == QLA_DRIFT_PER_CALL ? e_cur : stt.energy_ref;
        const double drift = fabs(e / ref - 1.0);
        stt.calls += 1;
        if (finite && drift <= drift_tol) {
            stt.surrogate_calls += 1;
            if (drift > stt.max_drift) stt.max_drift = drift;
            e_cur = e;
            return true;
        }
        stt.fallback_calls += 1;
        return false;
    };
    // K plain QLA steps from the context's current state after a rejection
    auto fallback = [&]() -> qla_status {
        qla_status rr = qla_step(ctx, s->cfg.K);
        if (rr != QLA_OK) return sfail(s, rr, "rollout: fallback qla_step failed: %s", qla_last_error(ctx));
        if (mode == QLA_DRIFT_PER_CALL) {
            bool f2 = true;
            ctx_view(ctx, &v);
            rr = energy(v.cur_state, &e_cur, &f2);
        }
        return rr;
    };
    if (serial) {
        for (int k = 0; k < calls; ++k) {
            ctx_view(ctx, &v);
            r = forward_infer(s, static_cast<const float *>(v.cur_state), n, static_cast<float *>(v.spare_state), st);
            if (r != QLA_OK) return r;
            double e = 0.0;
            r = energy(v.spare_state, &e, &fin);
            if (r != QLA_OK) return r;
            if (accept(e, fin)) {
                ctx_commit_spare(ctx, s->cfg.K);
            } else {
                r = fallback();
                if (r != QLA_OK) return r;
            }
        }
    } else {
        // Three state buffers: the context's two (A, B) and the surrogate's
        // qspec. `cur` holds the accepted state, `pend` the proposal of the
        // call being decided, `next` the speculative proposal computed from
        // `pend`; each is one of the three. The context's own current buffer
        // is brought up to date (sync_ctx) before a fallback and at the end.
        float *const A = static_cast<float *>(v.cur_state), *const B = static_cast<float *>(v.spare_state);
        float *const X = s->qspec;
        float *cur = A;
        long long pending_steps = 0;  // accepted steps not yet counted by the context
        auto free_buf = [&](const float *a, const float *b) { return (A != a && A != b) ? A : (B != a && B != b) ? B : X; };
        auto sync_ctx = [&]() -> qla_status {
            ctx_view(ctx, &v);
            if (cur == v.cur_state) {
                ctx_add_steps(ctx, pending_steps);
            } else {
                if (cur == X)
                    SG_CUDA(s, cudaMemcpyAsync(v.spare_state, X, sizeof(float) * 6 * size_t(v.Nx) * v.Ny,
                                               cudaMemcpyDeviceToDevice, st));
                ctx_commit_spare(ctx, pending_steps);
            }
            pending_steps = 0;
            ctx_view(ctx, &v);
            cur = static_cast<float *>(v.cur_state);
            return QLA_OK;
        };
        auto launch_call = [&](const float *src, float *dst, int slot) -> qla_status {
            qla_status rr = forward_infer(s, src, n, dst, st);
            return rr == QLA_OK ? launch_energy(dst, slot) : rr;
        };
        float *pend = nullptr;
        int slot = 0;
        for (int k = 0; k < calls; ++k) {
            if (!pend) {  // (re)start the pipeline from the accepted state
                pend = free_buf(cur, nullptr);
                slot = 0;
                r = launch_call(cur, pend, slot);
                if (r != QLA_OK) return r;
            }
            float *next = nullptr;
            if (k + 1 < calls) {  // the next call, on the assumption that this one is accepted
                next = free_buf(cur, pend);
                r = launch_call(pend, next, slot ^ 1);
                if (r != QLA_OK) return r;
            }
            double e = 0.0;
            r = read_energy(slot, &e, &fin);
            if (r != QLA_OK) return r;
            if (accept(e, fin)) {
                cur = pend;
                pending_steps += s->cfg.K;
                pend = next;
                slot ^= 1;
            } else {
                SG_CUDA(s, cudaStreamSynchronize(st));  // the speculative call is discarded
                r = sync_ctx();
                if (r != QLA_OK) return r;
                r = fallback();
                if (r != QLA_OK) return r;
                ctx_view(ctx, &v);
                cur = static_cast<float *>(v.cur_state);
                pend = nullptr;
            }
        }
        r = sync_ctx();
        if (r != QLA_OK) return r;
    }
    ctx_view(ctx, &v);
    r = energy(v.cur_state, &stt.energy_final, &fin);
    if (r != QLA_OK) return r;
    if (stats) *stats = stt;
    return QLA_OK;
}

qla_status qla_surrogate_info(const qla_surrogate *s, long long *nparam, long long *flops_per_call) {
    if (!s) return QLA_EINVAL;
    if (nparam) *nparam = s->nparam;
    if (flops_per_call) {
        long long macs = 0;
        for (int l = 0; l < NL; ++l) macs += 9LL * CINP[l] * NOUTP[l];
        *flops_per_call = 2 * macs * s->NP;
    }
    return QLA_OK;
}

const char *qla_surrogate_last_error(const qla_surrogate *s) { return s ? s->msg.c_str() : "NULL surrogate"; }

void qla_surrogate_destroy(qla_surrogate *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->arena) cudaFree(s->arena);
    if (s->host_scal) cudaFreeHost(s->host_scal);
    if (s->host_err) cudaFreeHost(s->host_err);
    for (cudaEvent_t e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
