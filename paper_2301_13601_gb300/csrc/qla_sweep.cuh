// Fused collide-stream-potential sweep: K full QLA time steps per HBM pass.
//
// Method (arXiv 2301.13601): one time step is U_X, U_Y, V_X, V_Y (Eq. 23) or
// the interleaved form with V' after the first and the last eight operators of
// each direction (Eq. 28). U_X (Eq. 18) acts right to left as
//   C+, S-G1, C, S+G1, C+, S+G2, C, S-G2, | C, S+G1, C+, S-G1, C, S-G2, C+, S+G2
// where G1 = S_14 and G2 = S_25 (Eq. 17 collisions); U_Y (Eq. 20) is the same
// with C_Y, G1 = S_03, along y. S^{+} sets q(r) <- q(r+1), S^{-} q(r) <- q(r-1).
//
// GPU design:
//  * The six components form two families that never couple (TM: q2 hub, q4
//    x-partner, q3 y-partner; TE: q5 hub, q1 x-partner, q0 y-partner). Every
//    x-operator acts on (hub, x-partner) and every y-operator on
//    (hub, y-partner). One CTA advances one family of one tile.
//  * A tile is a strip of W_IN = 256 columns (each lane of a warp holds 8
//    consecutive columns) swept downwards over a chunk of rows. The strip
//    carries a 4K-column halo on each side (a step has dependency radius 4
//    along each axis); its central W_IN - 8K columns are written.
//  * Per time level j = 0..K-1 and per block of R rows, an x-pass (one warp
//    per row; shifts are register renames plus one warp shuffle) runs in
//    place on a shared-memory row buffer, then a y-pass streams each column
//    through a register pipeline: the eight y-shifts become eight saved
//    registers per column, output trails input by 4 rows, and no y-halo is
//    recomputed. The y-pass of level j writes level j+1's row buffer (double
//    buffered) or, for the last level, global memory.
//  * Level 0 rows are fetched one iteration ahead with cp.async.
//  * Rotations use the (cos-1, sin) form h' = h + (m h + s p): one rounding at
//    the scale of h per output, and coefficients whose FP32 norm error is
//    minimised at creation.
#pragma once

#include "qla_internal.h"

namespace qla {

constexpr int LANE_COLS = 8;
constexpr int W_IN = 32 * LANE_COLS;

struct SweepParams {
    SweepArgs a;
    Family fam[2];
};

template <typename T>
struct Ar;
template <>
struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};
template <>
struct Ar<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
};

// Collision C (DAG = false) or its transpose (DAG = true) on (h, p), with
// m = cos(theta) - 1 and s = orientation * sin(theta):
//   C:  h' = h + (m h + s p),   p' = p + (m p - s h)
template <bool DAG, typename T>
__device__ __forceinline__ void rot(T &h, T &p, T m, T s) {
    using A = Ar<T>;
    const T sg = DAG ? -s : s;
    const T u = A::fma(m, h, A::mul(sg, p));
    const T v = A::fma(m, p, -A::mul(sg, h));
    h = A::add(h, u);
    p = A::add(p, v);
}

// Potential row: target' = target + (c target + s source) with
// s = orientation * sin(b), c = cos(b) - 1; the unitary variant also rotates the
// source: source' = source + (c source - s target).
template <typename T>
__device__ __forceinline__ void vop(T &target, T &source, T s, T c, bool unitary) {
    using A = Ar<T>;
    const T t2 = A::add(target, A::fma(c, target, A::mul(s, source)));
    if (unitary) source = A::add(source, A::fma(c, source, -A::mul(s, target)));
    target = t2;
}

template <typename T>
__device__ __forceinline__ void vop_pair(T &h, T &p, T s, T c, bool target_is_hub, bool unitary) {
    if (target_is_hub) vop(h, p, s, c, unitary);
    else vop(p, h, s, c, unitary);
}

// a(x) <- a(x-1) across the warp's 8*32 columns
template <typename T>
__device__ __forceinline__ void shift_from_left(T (&a)[LANE_COLS]) {
    const T edge = __shfl_up_sync(0xffffffffu, a[LANE_COLS - 1], 1);
#pragma unroll
    for (int j = LANE_COLS - 1; j > 0; --j) a[j] = a[j - 1];
    a[0] = edge;
}

// a(x) <- a(x+1)
template <typename T>
__device__ __forceinline__ void shift_from_right(T (&a)[LANE_COLS]) {
    const T edge = __shfl_down_sync(0xffffffffu, a[0], 1);
#pragma unroll
    for (int j = 0; j < LANE_COLS - 1; ++j) a[j] = a[j + 1];
    a[LANE_COLS - 1] = edge;
}

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// 8 consecutive (periodic) elements of a global row starting at column c0.
template <typename T>
__device__ __forceinline__ void gload8(T (&v)[LANE_COLS], const T *__restrict__ row, int c0, int Nx, bool vec) {
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(row + c0));
            int c1 = c0 + 4;
            if (c1 >= Nx) c1 -= Nx;
            const float4 b = __ldg(reinterpret_cast<const float4 *>(row + c1));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int c = c0 + 2 * k;
                c = c >= Nx ? c - Nx * (c / Nx) : c;
                const double2 d = __ldg(reinterpret_cast<const double2 *>(row + c));
                v[2 * k] = d.x;
                v[2 * k + 1] = d.y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < LANE_COLS; ++j) v[j] = __ldg(row + (c0 + j) % Nx);
    }
}

template <typename T>
__device__ __forceinline__ void sload8(T (&v)[LANE_COLS], const T *p) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        const float4 b = *reinterpret_cast<const float4 *>(p + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 d = *reinterpret_cast<const double2 *>(p + 2 * k);
            v[2 * k] = d.x;
            v[2 * k + 1] = d.y;
        }
    }
}

template <typename T>
__device__ __forceinline__ void sstore8(T *p, const T (&v)[LANE_COLS]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) *reinterpret_cast<double2 *>(p + 2 * k) = make_double2(v[2 * k], v[2 * k + 1]);
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Register pipeline of the y-pass for one column of one level.
template <typename T>
struct YPipe {
    T S2, S4, S6, S8, S10, S12, S14, S16;  // one saved value per y-shift
    T m1, s1, m2, s2, m3, s3;              // collision coefficients of rows R-1, R-2, R-3
    T d0, d1, d2, d3;                      // x-partner delayed by 4 rows
    __device__ __forceinline__ void zero() {
        S2 = S4 = S6 = S8 = S10 = S12 = S14 = S16 = T(0);
        m1 = s1 = m2 = s2 = m3 = s3 = T(0);
        d0 = d1 = d2 = d3 = T(0);
    }
};

template <typename T, int K, int NY, int R>
struct SweepCfg {
    static constexpr int NT = W_IN * K / NY;
    static constexpr int NWARP = NT / 32;
    static constexpr size_t SMEM = size_t(K) * 2 * 3 * R * W_IN * sizeof(T);
    static_assert(W_IN * K % NY == 0, "tasks must divide");
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
};

template <typename T, int K, int NY, int R>
__global__ void __launch_bounds__(SweepCfg<T, K, NY, R>::NT, 1) sweep_kernel(const SweepParams prm) {
    using Cfg = SweepCfg<T, K, NY, R>;
    constexpr int NT = Cfg::NT;
    constexpr int NWARP = Cfg::NWARP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const buf = reinterpret_cast<T *>(smem_raw);

    const SweepArgs &A = prm.a;
    Family F = prm.fam[0];
    if (A.fam0 + int(blockIdx.z) == 1) F = prm.fam[1];
    const int Nx = A.Nx, Ny = A.Ny;
    const size_t P = size_t(Nx) * size_t(Ny);
    const T *__restrict__ qin = static_cast<const T *>(A.q_in);
    T *__restrict__ qout = static_cast<T *>(A.q_out);
    const T *__restrict__ coef = static_cast<const T *>(A.coef);
    const bool vec = A.vec != 0;
    const bool inter = A.interleaved != 0;
    const bool unit = A.unitary != 0;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    const int xs0 = blockIdx.x * A.w_valid;   // first output column of the strip
    const int xbase = xs0 - 4 * K;            // global column of strip column 0 (may be < 0)
    const int yb = blockIdx.y * A.chunk;
    const int ye = min(yb + A.chunk, Ny);
    const int F0 = yb - 4 * K;                // first row fed to level 0
    const int nit = (ye - yb + 8 * K + R - 1) / R + K - 1;

    auto bufrow = [&](int j, int half, int comp, int ir) -> T * {
        return buf + ((size_t(((j * 2 + half) * 3 + comp) * R + ir)) * W_IN);
    };
    // first row handled by level j in iteration it
    auto arow = [&](int j, int it) { return F0 + (it - j) * R - 4 * j; };
    auto active = [&](int j, int it) { return it >= j && arow(j, it) <= ye - 1 + 4 * (K - j); };

    for (int i = tid; i < K * 2 * 3 * R * W_IN; i += NT) buf[i] = T(0);

    auto plane_of = [&](int comp) { return comp == 0 ? F.h : (comp == 1 ? F.px : F.py); };

    auto load0 = [&](int it, int half) {
        const int row0 = arow(0, it);
        if (vec) {
            constexpr int EPC = 16 / sizeof(T);
            constexpr int CH = W_IN / EPC;
            for (int q = tid; q < 3 * R * CH; q += NT) {
                const int k = q % CH;
                const int rc = q / CH;
                const int ir = rc % R;
                const int comp = rc / R;
                const int grow = wrapi(row0 + ir, Ny);
                const int gcol = wrapi(xbase + k * EPC, Nx);
                const T *src = qin + size_t(plane_of(comp)) * P + size_t(grow) * Nx + gcol;
                cp_async16(bufrow(0, half, comp, ir) + k * EPC, src);
            }
        } else {
            for (int q = tid; q < 3 * R * W_IN; q += NT) {
                const int c = q % W_IN;
                const int rc = q / W_IN;
                const int ir = rc % R;
                const int comp = rc / R;
                const int grow = wrapi(row0 + ir, Ny);
                const int gcol = wrapi(xbase + c, Nx);
                const T *src = qin + size_t(plane_of(comp)) * P + size_t(grow) * Nx + gcol;
                cp_async_small<sizeof(T)>(bufrow(0, half, comp, ir) + c, src);
            }
        }
        cp_async_commit();
    };

    __syncthreads();  // zeroed buffers before the async copies land
    load0(0, 0);
    cp_async_wait_all();
    __syncthreads();

    YPipe<T> yp[NY];
#pragma unroll
    for (int u = 0; u < NY; ++u) yp[u].zero();

    const T sgx = T(F.sgx), sgy = T(F.sgy), tx = T(F.tx), ty = T(F.ty);
    const bool vxh = F.vx_hub != 0, vyh = F.vy_hub != 0;

    for (int it = 0; it < nit; ++it) {
        const int cur = it & 1;
        if (it + 1 < nit && active(0, it + 1)) load0(it + 1, cur ^ 1);

        // ---- phase 1: x-pass, one warp per (level, row) -------------------
        for (int task = warp; task < K * R; task += NWARP) {
            const int j = task / R;
            const int ir = task % R;
            if (!active(j, it)) continue;
            T *rh = bufrow(j, cur, 0, ir) + LANE_COLS * lane;
            T *rp = bufrow(j, cur, 1, ir) + LANE_COLS * lane;
            const int grow = wrapi(arow(j, it) + ir, Ny);
            const int gc0 = wrapi(xbase + LANE_COLS * lane, Nx);
            const size_t roff = size_t(grow) * Nx;
            T m[LANE_COLS], s[LANE_COLS], h[LANE_COLS], p[LANE_COLS];
            gload8(m, coef + size_t(F.cxm) * P + roff, gc0, Nx, vec);
            gload8(s, coef + size_t(F.cxs) * P + roff, gc0, Nx, vec);
            sload8(h, rh);
            sload8(p, rp);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) s[c] *= sgx;
            // ops 1-8
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true>(h[c], p[c], m[c], s[c]);
            shift_from_left(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false>(h[c], p[c], m[c], s[c]);
            shift_from_right(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true>(h[c], p[c], m[c], s[c]);
            shift_from_right(h);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false>(h[c], p[c], m[c], s[c]);
            shift_from_left(h);
            T vs[LANE_COLS], vc[LANE_COLS];
            if (inter) {
                gload8(vs, coef + size_t(F.vxs) * P + roff, gc0, Nx, vec);
                gload8(vc, coef + size_t(F.vxc) * P + roff, gc0, Nx, vec);
#pragma unroll
                for (int c = 0; c < LANE_COLS; ++c) {
                    vs[c] *= tx;
                    vop_pair(h[c], p[c], vs[c], vc[c], vxh, unit);
                }
            }
            // ops 9-16
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false>(h[c], p[c], m[c], s[c]);
            shift_from_right(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true>(h[c], p[c], m[c], s[c]);
            shift_from_left(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false>(h[c], p[c], m[c], s[c]);
            shift_from_left(h);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true>(h[c], p[c], m[c], s[c]);
            shift_from_right(h);
            if (inter) {
#pragma unroll
                for (int c = 0; c < LANE_COLS; ++c) vop_pair(h[c], p[c], vs[c], vc[c], vxh, unit);
            }
            sstore8(rh, h);
            sstore8(rp, p);
        }
        __syncthreads();

        // ---- phase 2: y-pass, one thread per (level, column) --------------
#pragma unroll
        for (int u = 0; u < NY; ++u) {
            const int task = tid + u * NT;
            const int j = task / W_IN;
            const int c = task % W_IN;
            if (!active(j, it)) continue;
            YPipe<T> &Y = yp[u];
            const int gcol = wrapi(xbase + c, Nx);
            const T *hin = bufrow(j, cur, 0, 0) + c;
            const T *pxin = bufrow(j, cur, 1, 0) + c;
            const T *pyin = bufrow(j, cur, 2, 0) + c;
            const bool last = (j == K - 1);
            T *hout = last ? nullptr : bufrow(j + 1, cur ^ 1, 0, 0) + c;
            T *pxout = last ? nullptr : bufrow(j + 1, cur ^ 1, 1, 0) + c;
            T *pyout = last ? nullptr : bufrow(j + 1, cur ^ 1, 2, 0) + c;
            const bool col_ok = last && c >= 4 * K && c < 4 * K + A.w_valid && xs0 + (c - 4 * K) < Nx;
            const int gx = xs0 + (c - 4 * K);
            const T *cym = coef + size_t(F.cym) * P + gcol;
            const T *cys = coef + size_t(F.cys) * P + gcol;
            const T *vys = coef + size_t(F.vys) * P + gcol;
            const T *vyc = coef + size_t(F.vyc) * P + gcol;
            const T *vxs = coef + size_t(F.vxs) * P + gcol;
            const T *vxc = coef + size_t(F.vxc) * P + gcol;
            const int a0 = arow(j, it);
#pragma unroll
            for (int ir = 0; ir < R; ++ir) {
                const int rin = a0 + ir;
                const size_t o0 = size_t(wrapi(rin, Ny)) * Nx;
                const size_t o2 = size_t(wrapi(rin - 2, Ny)) * Nx;
                const size_t o4 = size_t(wrapi(rin - 4, Ny)) * Nx;
                const T m0 = __ldg(cym + o0);
                const T s0 = __ldg(cys + o0) * sgy;
                T h = hin[ir * W_IN];
                T p = pyin[ir * W_IN];
                const T px0 = pxin[ir * W_IN];
                rot<true>(h, p, m0, s0);                    // op 1  C+   (row R)
                { const T t = Y.S2; Y.S2 = p; p = t; }      // op 2  p <- p(r-1)
                rot<false>(h, p, m0, s0);                   // op 3  C    (row R)
                { const T t = Y.S4; Y.S4 = h; h = t; }      // op 4  p <- p(r+1): now row R-1
                rot<true>(h, p, Y.m1, Y.s1);                // op 5  C+   (row R-1)
                { const T t = Y.S6; Y.S6 = p; p = t; }      // op 6  h <- h(r+1): now row R-2
                rot<false>(h, p, Y.m2, Y.s2);               // op 7  C    (row R-2)
                { const T t = Y.S8; Y.S8 = h; h = t; }      // op 8  h <- h(r-1)
                if (inter) {
                    const T vs = __ldg(vys + o2) * ty, vc = __ldg(vyc + o2);
                    vop_pair(h, p, vs, vc, vyh, unit);      // V_Y' (row R-2)
                }
                rot<false>(h, p, Y.m2, Y.s2);               // op 9  C    (row R-2)
                { const T t = Y.S10; Y.S10 = h; h = t; }    // op 10 p <- p(r+1): now row R-3
                rot<true>(h, p, Y.m3, Y.s3);                // op 11 C+   (row R-3)
                { const T t = Y.S12; Y.S12 = p; p = t; }    // op 12 p <- p(r-1)
                rot<false>(h, p, Y.m3, Y.s3);               // op 13 C    (row R-3)
                { const T t = Y.S14; Y.S14 = h; h = t; }    // op 14 h <- h(r-1)
                rot<true>(h, p, Y.m3, Y.s3);                // op 15 C+   (row R-3)
                { const T t = Y.S16; Y.S16 = p; p = t; }    // op 16 h <- h(r+1): now row R-4
                T px = Y.d3;
                Y.d3 = Y.d2; Y.d2 = Y.d1; Y.d1 = Y.d0; Y.d0 = px0;
                if (inter) {
                    const T vs = __ldg(vys + o4) * ty, vc = __ldg(vyc + o4);
                    vop_pair(h, p, vs, vc, vyh, unit);      // V_Y' (row R-4)
                } else {
                    const T xs = __ldg(vxs + o4) * tx, xc = __ldg(vxc + o4);
                    vop_pair(h, px, xs, xc, vxh, unit);     // V_X  (row R-4)
                    const T vs = __ldg(vys + o4) * ty, vc = __ldg(vyc + o4);
                    vop_pair(h, p, vs, vc, vyh, unit);      // V_Y  (row R-4)
                }
                Y.m3 = Y.m2; Y.s3 = Y.s2;
                Y.m2 = Y.m1; Y.s2 = Y.s1;
                Y.m1 = m0;   Y.s1 = s0;
                if (!last) {
                    hout[ir * W_IN] = h;
                    pxout[ir * W_IN] = px;
                    pyout[ir * W_IN] = p;
                } else {
                    const int rout = rin - 4;
                    if (col_ok && rout >= yb && rout < ye) {
                        const size_t o = size_t(rout) * Nx + gx;
                        qout[size_t(F.h) * P + o] = h;
                        qout[size_t(F.px) * P + o] = px;
                        qout[size_t(F.py) * P + o] = p;
                    }
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
}

template <typename T, int K, int NY, int R>
int occupancy_t() {
    using Cfg = SweepCfg<T, K, NY, R>;
    cudaFuncSetAttribute(sweep_kernel<T, K, NY, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::SMEM));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, K, NY, R>, Cfg::NT, Cfg::SMEM) !=
        cudaSuccess)
        n = 1;
    cudaGetLastError();
    return n < 1 ? 1 : n;
}

template <typename T, int K, int NY, int R>
cudaError_t launch_sweep_t(const SweepArgs &a, int nfam, cudaStream_t st) {
    using Cfg = SweepCfg<T, K, NY, R>;
    static int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(sweep_kernel<T, K, NY, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Cfg::SMEM));
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    SweepParams prm;
    prm.a = a;
    // TM: hub q2, x-partner q4, y-partner q3.
    //   C_X on (q2,q4): q2' = c q2 - s q4 -> orientation -1; V_X row q4 <- -sin b2 q2 (partner, -1)
    //   C_Y on (q2,q3): q2' = c q2 + s q3 -> orientation +1; V_Y row q3 <- +sin b3 q2 (partner, +1)
    prm.fam[0] = Family{2, 4, 3, C_TM_M, C_TM_S, C_TM_M, C_TM_S, C_TM_VXS, C_TM_VXC, C_TM_VYS, C_TM_VYC,
                        -1.f, +1.f, -1.f, +1.f, 0, 0};
    // TE: hub q5, x-partner q1, y-partner q0.
    //   C_X on (q1,q5): q5' = s q1 + c q5 -> orientation +1; V_X row q5 <- +sin b0 q1 (hub, +1)
    //   C_Y on (q0,q5): q5' = -s q0 + c q5 -> orientation -1; V_Y row q5 <- -sin b1 q0 (hub, -1)
    prm.fam[1] = Family{5, 1, 0, C_TE_XM, C_TE_XS, C_TE_YM, C_TE_YS, C_TE_VXS, C_TE_VXC, C_TE_VYS, C_TE_VYC,
                        +1.f, -1.f, +1.f, -1.f, 1, 1};
    const int nsx = (a.Nx + a.w_valid - 1) / a.w_valid;
    const int ncy = (a.Ny + a.chunk - 1) / a.chunk;
    dim3 grid(nsx, ncy, nfam);
    sweep_kernel<T, K, NY, R><<<grid, Cfg::NT, Cfg::SMEM, st>>>(prm);
    return cudaGetLastError();
}

}  // namespace qla
