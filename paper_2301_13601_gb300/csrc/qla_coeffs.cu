// Set-up kernels: rotation/potential coefficients (Eq. 24-25), the pulse
// initial condition and precision conversions.
#include <math.h>

#include "qla_internal.h"

namespace qla {

namespace {

// FP32 rotation pair (t, s) for the three-shear collision of the sweep:
// t = tan(a / 2) rounded to FP32, and s the FP32 value nearest to
// 2t / (1 + t^2), the sine of the angle 2 atan(t) that t represents exactly.
// The three shears (determinant exactly 1) are then a rotation to within one
// rounding of s, and the angle differs from a by at most half an ulp of t.
__device__ void shear_pair_f32(double ang, float &tf, float &sf) {
    tf = (float)tan(0.5 * ang);
    const double t = (double)tf;
    sf = (float)(2.0 * t / (1.0 + t * t));
}

// FP32 (cos(a) - 1, sin(a)) pair chosen among FP32 values within a few ulps of
// the correctly rounded ones so that (1 + m)^2 + s^2 - 1 (evaluated exactly in
// FP64: every term is a product of two FP32 values) is as small as possible:
// each rotation then keeps the energy (Eq. 27) to ~1e-13, with the angle
// changed by a few ulps of m and s at most.
__device__ void tuned_pair_f32(double ang, float &mf, float &sf) {
    const double sh = sin(0.5 * ang);
    const double m = -2.0 * sh * sh;  // cos(ang) - 1 without cancellation
    const double s = sin(ang);
    const float m0 = (float)m, s0 = (float)s;
    if (!(fabsf(m0) >= 1e-30f) || !(fabsf(s0) >= 1e-30f)) {  // zero or denormal: keep the rounded values
        mf = m0;
        sf = s0;
        return;
    }
    const int mi = __float_as_int(m0), si = __float_as_int(s0);
    double best = 1e300;
    int bdm = 0, bds = 0;
    for (int dm = -4; dm <= 4; ++dm) {
        const float mc = __int_as_float(mi + dm);
        for (int ds = -2; ds <= 2; ++ds) {
            const float sc = __int_as_float(si + ds);
            const double dmc = (double)mc, dsc = (double)sc;
            const double e = fabs(2.0 * dmc + dmc * dmc + dsc * dsc);
            const int cost = abs(dm) + abs(ds);
            if (e < best || (e == best && cost < abs(bdm) + abs(bds))) {
                best = e;
                bdm = dm;
                bds = ds;
            }
        }
    }
    mf = __int_as_float(mi + bdm);
    sf = __int_as_float(si + bds);
}

// How a pair is stored (see CoefPair and rot in the sweep): a collision of the
// three-shear form (FP32 with the printed potentials: (tan(a/2), sin a)), a
// rotation of the (cos - 1, sin) form (FP32: tuned for orthogonality) or a
// printed potential row (cos a - 1, sin a). FP64 stores (cos a - 1, sin a)
// for all.
enum PairKind { PK_SHEAR, PK_ROTATION, PK_PRINTED_V };

template <typename T>
__device__ void store_pair(T *coef, size_t P, int pair, size_t i, double ang, PairKind kind) {
    T *dst = coef + 2 * (size_t(pair) * P + i);
    if constexpr (sizeof(T) == 4) {
        float xf, sf;
        if (kind == PK_SHEAR) {
            shear_pair_f32(ang, xf, sf);
        } else if (kind == PK_ROTATION) {
            tuned_pair_f32(ang, xf, sf);
        } else {
            const double sh = sin(0.5 * ang);
            xf = (float)(-2.0 * sh * sh);
            sf = (float)sin(ang);
        }
        dst[0] = xf;
        dst[1] = sf;
    } else {
        const double sh = sin(0.5 * ang);
        dst[0] = -2.0 * sh * sh;
        dst[1] = sin(ang);
    }
}

// One thread per site. n: [3][Ny][Nx] double (n_x, n_y, n_z).
template <typename T>
__global__ void coef_kernel(const double *__restrict__ n, T *__restrict__ coef, int Nx, int Ny, double delta,
                            int interleaved, int unitary) {
    const size_t P = size_t(Nx) * size_t(Ny);
    const double *nx = n, *ny = n + P, *nz = n + 2 * P;
    // effective potential angle: halved when interleaved (Eq. 28), halved
    // again for the unitary pair rotation
    const double vscale = (interleaved ? 0.5 : 1.0) * (unitary ? 0.5 : 1.0);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x) {
        const int y = int(i / Nx), x = int(i % Nx);
        const int xp = x + 1 == Nx ? 0 : x + 1, xm = x == 0 ? Nx - 1 : x - 1;
        const int yp = y + 1 == Ny ? 0 : y + 1, ym = y == 0 ? Ny - 1 : y - 1;
        const size_t r = size_t(y) * Nx;
        const double vnx = nx[i], vny = ny[i], vnz = nz[i];
        // Eq. 24
        const double th0 = delta / (4.0 * vnx), th1 = delta / (4.0 * vny), th2 = delta / (4.0 * vnz);
        // Eq. 25 with central differences over lattice spacing delta
        const double dny_dx = (ny[r + xp] - ny[r + xm]) / (2.0 * delta);
        const double dnx_dy = (nx[size_t(yp) * Nx + x] - nx[size_t(ym) * Nx + x]) / (2.0 * delta);
        const double dnz_dx = (nz[r + xp] - nz[r + xm]) / (2.0 * delta);
        const double dnz_dy = (nz[size_t(yp) * Nx + x] - nz[size_t(ym) * Nx + x]) / (2.0 * delta);
        const double b0 = delta * delta * dny_dx / (vny * vny);
        const double b1 = delta * delta * dnx_dy / (vnx * vnx);
        const double b2 = delta * delta * dnz_dx / (vnz * vnz);
        const double b3 = delta * delta * dnz_dy / (vnz * vnz);
        const PairKind ck = unitary ? PK_ROTATION : PK_SHEAR;
        const PairKind vk = unitary ? PK_ROTATION : PK_PRINTED_V;
        store_pair<T>(coef, P, P_TM_C, i, th2, ck);
        store_pair<T>(coef, P, P_TE_CX, i, th1, ck);
        store_pair<T>(coef, P, P_TE_CY, i, th0, ck);
        store_pair<T>(coef, P, P_TM_VX, i, b2 * vscale, vk);
        store_pair<T>(coef, P, P_TM_VY, i, b3 * vscale, vk);
        store_pair<T>(coef, P, P_TE_VX, i, b0 * vscale, vk);
        store_pair<T>(coef, P, P_TE_VY, i, b1 * vscale, vk);
    }
}

// g(x) = amp exp(-d^2/(2 sigma^2)), d the periodic minimum-image x - x0;
// E_z: q2 = g, q4 = -g; E_y: q1 = g, q5 = g; other components 0.
template <typename T>
__global__ void pulse_kernel(T *__restrict__ q, int Nx, int Ny, int pol, double x0, double sigma, double amp) {
    const size_t P = size_t(Nx) * size_t(Ny);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < P; i += size_t(gridDim.x) * blockDim.x) {
        const int x = int(i % Nx);
        double d = double(x) - x0;
        d -= double(Nx) * floor(d / double(Nx) + 0.5);
        const double g = amp * exp(-d * d / (2.0 * sigma * sigma));
        T v[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (pol == 0) {
            v[2] = T(g);
            v[4] = T(-g);
        } else {
            v[1] = T(g);
            v[5] = T(g);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) q[size_t(c) * P + i] = v[c];
    }
}

template <typename S, typename D>
__global__ void convert_kernel(const S *__restrict__ src, D *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        dst[i] = D(src[i]);
}

int grid_for(size_t n, int block) {
    size_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return int(g);
}

}  // namespace

cudaError_t launch_coefficients(const double *n, void *coef, int Nx, int Ny, double delta, int precision,
                                int interleaved, int unitary, cudaStream_t st) {
    const size_t P = size_t(Nx) * size_t(Ny);
    const int B = 256;
    if (precision == 0)
        coef_kernel<float><<<grid_for(P, B), B, 0, st>>>(n, static_cast<float *>(coef), Nx, Ny, delta,
                                                          interleaved, unitary);
    else
        coef_kernel<double><<<grid_for(P, B), B, 0, st>>>(n, static_cast<double *>(coef), Nx, Ny, delta,
                                                           interleaved, unitary);
    return cudaGetLastError();
}

cudaError_t launch_init_pulse(void *q, int Nx, int Ny, int precision, int pol, double x0, double sigma,
                              double amp, cudaStream_t st) {
    const size_t P = size_t(Nx) * size_t(Ny);
    const int B = 256;
    if (precision == 0)
        pulse_kernel<float><<<grid_for(P, B), B, 0, st>>>(static_cast<float *>(q), Nx, Ny, pol, x0, sigma, amp);
    else
        pulse_kernel<double><<<grid_for(P, B), B, 0, st>>>(static_cast<double *>(q), Nx, Ny, pol, x0, sigma, amp);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void *src, int src_double, void *dst, int dst_double, size_t n, cudaStream_t st) {
    const int B = 256;
    const int G = grid_for(n, B);
    if (src_double && dst_double)
        convert_kernel<double, double><<<G, B, 0, st>>>(static_cast<const double *>(src), static_cast<double *>(dst), n);
    else if (src_double)
        convert_kernel<double, float><<<G, B, 0, st>>>(static_cast<const double *>(src), static_cast<float *>(dst), n);
    else if (dst_double)
        convert_kernel<float, double><<<G, B, 0, st>>>(static_cast<const float *>(src), static_cast<double *>(dst), n);
    else
        convert_kernel<float, float><<<G, B, 0, st>>>(static_cast<const float *>(src), static_cast<float *>(dst), n);
    return cudaGetLastError();
}

}  // namespace qla
