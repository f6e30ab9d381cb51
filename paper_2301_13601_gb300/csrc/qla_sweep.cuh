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
//    (hub, y-partner). One CTA advances one family of one tile; the family,
//    the step order and the potential variant are compile-time parameters.
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
//  * No compute phase touches global memory for its inputs: the y-pass
//    coefficients of an iteration are copied into shared memory while the
//    x-pass of that iteration runs, and the x-pass coefficients and next
//    level-0 rows while the y-pass of the previous iteration runs. The copies
//    are TMA tile loads where the strip does not wrap around x (one box per
//    R-row block, or per coefficient plane for all levels; mbarrier
//    completion), per-lane cp.async elsewhere. (A bulk L2 prefetch two
//    iterations ahead was measured to cost 18% on top of this staging and is
//    not used.)
//  * In FP32 with the printed potentials a collision is three shears
//    (h += t p, p -= s h, h += t p with t = tan(theta/2): three FMAs, the
//    determinant exactly 1); otherwise the (cos-1, sin) form
//    h' = h + (m h + s p), one rounding at the scale of each output, with FP32
//    pairs tuned at creation for orthogonality. Coefficients are stored as
//    pairs of the form the kernel uses (see rot).
#pragma once

#include <cuda.h>
#include <string.h>

#include <type_traits>

#include "qla_internal.h"
#include "qla_tc.cuh"

namespace qla {

constexpr int LANE_COLS = 8;
constexpr int W_IN = 32 * LANE_COLS;

// Global nanosecond timer (bounds the waits on other CTAs' progress).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Progress counters written by other CTAs: acquire loads and release stores
// at GPU scope.
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Tensor maps for the TMA loads of one FP32 pass: the input state viewed as
// [6][Ny][Nx/8][8] floats with the 32-byte swizzle and the coefficient pairs
// as [7][Ny][Nx/8][16] floats with the 64-byte swizzle. One box row (8 x 32,
// resp. 16 x 32) is one 256-column strip row, landing in exactly the
// XOR-swizzled layout of the shared row buffers (swz below).
struct SweepMaps {
    CUtensorMap state;     // one row of one component (blocks that wrap around y)
    CUtensorMap state_r1;  // R rows of 1 component
    CUtensorMap state_r2;  // R rows of 2 adjacent components
    CUtensorMap state_r3;  // R rows of 3 adjacent components
    CUtensorMap coef;      // one row of one pair plane
    CUtensorMap coef_r;    // R rows of one pair plane
    // The pair planes as [7][Ny / (R + 4)][R + 4][Nx/8][16] floats: one box
    // (16 x 32 x R x K x n) holds the R-row blocks of all K levels of an
    // iteration, which start R + 4 rows apart, of n adjacent planes (n = 1, 2);
    // valid when merged != 0 (K > 1 and Ny a multiple of R + 4).
    CUtensorMap coef_m1;
    CUtensorMap coef_m2;
    // The seam strip (SweepArgs::seam) reads columns [Nx - 128, Nx) and
    // [0, 128). These views see a row as two 128-column halves, half 0 at
    // column 0 and half 1 at column Nx - 128 ({e, 16, 2, Ny, planes}, the half
    // stride (Nx - 128) elements), so one box brings both halves. They land
    // swapped (global columns 0..127 first): the kernel addresses the seam
    // strip's shared rows at column c ^ 128.
    CUtensorMap seam_state;     // one row of one component
    CUtensorMap seam_state_r1;  // R rows of 1, 2, 3 adjacent components
    CUtensorMap seam_state_r2;
    CUtensorMap seam_state_r3;
    CUtensorMap seam_coef;      // one row of one pair plane
    CUtensorMap seam_coef_r;    // R rows of one pair plane
};

struct SweepParams {
    SweepArgs a;
    SweepMaps m;
    int tma;
    int merged;
    int tiles_fastest;  // grid x runs over the row tiles of a strip (else over the strips of a tile row)
    SweepSplit split[2];  // per family layer (blockIdx.z): strips and balanced split (a.chunk == 0)
};

template <typename T>
struct Ar;
template <>
struct Ar<float> {
    using T2 = float2;
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};
template <>
struct Ar<double> {
    using T2 = double2;
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
};

// Compile-time description of a family (see qla_internal.h).
//   TM: hub q2, x-partner q4, y-partner q3.
//     C_X on (q2,q4): q2' = c q2 - s q4 -> orientation -1; V_X row q4 <- -sin b2 q2 (partner, -1)
//     C_Y on (q2,q3): q2' = c q2 + s q3 -> orientation +1; V_Y row q3 <- +sin b3 q2 (partner, +1)
//   TE: hub q5, x-partner q1, y-partner q0.
//     C_X on (q1,q5): q5' = s q1 + c q5 -> orientation +1; V_X row q5 <- +sin b0 q1 (hub, +1)
//     C_Y on (q0,q5): q5' = -s q0 + c q5 -> orientation -1; V_Y row q5 <- -sin b1 q0 (hub, -1)
template <int FAM>
struct Fam;
// State planes sit in the shared row buffers in plane order, so that the
// family's planes that are adjacent in global memory arrive in one TMA box:
// SH, SPX, SPY are the buffer slots of the hub and the partners, and the
// state boxes are (first plane, planes, first slot) per box (n1 = 0: none).
template <>
struct Fam<0> {
    static constexpr int H = 2, PX = 4, PY = 3;
    static constexpr int CX = P_TM_C, CY = P_TM_C, VX = P_TM_VX, VY = P_TM_VY;
    static constexpr int SGX = -1, SGY = +1, TX = -1, TY = +1;
    static constexpr bool VX_HUB = false, VY_HUB = false;
    static constexpr int SH = 0, SPY = 1, SPX = 2;  // planes 2, 3, 4
    static constexpr int B0 = 2, N0 = 3, B1 = 0, N1 = 0;
    static constexpr int plane_of_slot(int slot) { return 2 + slot; }
};
template <>
struct Fam<1> {
    static constexpr int H = 5, PX = 1, PY = 0;
    static constexpr int CX = P_TE_CX, CY = P_TE_CY, VX = P_TE_VX, VY = P_TE_VY;
    static constexpr int SGX = +1, SGY = -1, TX = +1, TY = -1;
    static constexpr bool VX_HUB = true, VY_HUB = true;
    static constexpr int SPY = 0, SPX = 1, SH = 2;  // planes 0, 1, 5
    static constexpr int B0 = 0, N0 = 2, B1 = 5, N1 = 1;
    static constexpr int plane_of_slot(int slot) { return slot < 2 ? slot : 5; }
};

// Collision C (DAG = false) or its transpose (DAG = true) on (h, p) with
// orientation SG: the rotation h' = c h + SG s p, p' = -SG s h + c p by the
// angle theta (c = cos theta, s = sin theta).
//  * SHEAR = false: pair (m, s) with m = cos(theta) - 1:
//      h' = h + (m h + SG s p),   p' = p + (m p - SG s h)
//    (one rounding at the scale of each output; six instructions).
//  * SHEAR = true (FP32 with the printed potentials): pair (t, s) with
//    t = tan(theta / 2), as three shears
//      h1 = h + SG t p,  p' = p - SG s h1,  h' = h1 + SG t p'
//    (three FMAs). Each shear has determinant exactly 1 whatever the rounding
//    of t and s, so the rotation cannot scale the energy (Eq. 27) coherently;
//    s is stored as the FP32 value nearest to 2t / (1 + t^2), which makes the
//    shears a rotation to within one rounding of s, and the small remaining
//    asymmetry biases the energy with opposite signs in C and its transpose,
//    which alternate in Eq. 18 and Eq. 20.
template <bool DAG, int SG, bool SHEAR, typename T>
__device__ __forceinline__ void rot(T &h, T &p, T m, T s) {
    using A = Ar<T>;
    constexpr bool pos = (SG > 0) != DAG;
    if constexpr (SHEAR) {
        const T t = m;
        h = pos ? A::fma(t, p, h) : A::fma(-t, p, h);
        p = pos ? A::fma(-s, h, p) : A::fma(s, h, p);
        h = pos ? A::fma(t, p, h) : A::fma(-t, p, h);
    } else {
        const T sp = A::mul(s, p);
        const T sh = A::mul(s, h);
        const T u = pos ? A::fma(m, h, sp) : A::fma(m, h, -sp);
        const T v = pos ? A::fma(m, p, -sh) : A::fma(m, p, sh);
        h = A::add(h, u);
        p = A::add(p, v);
    }
}

// Collision form of a configuration: three shears in FP32 with the printed
// potentials; the (cos - 1, sin) form in FP64, and in FP32 with the unitary
// potentials, where every operator is an exact rotation and the tuned pairs
// keep the energy (Eq. 27) to FP32 rounding over 1e4 steps.
template <typename T, bool UNIT>
constexpr bool shear_collisions() {
    return std::is_same<T, float>::value && !UNIT;
}

// Potential row: target' = target + (c target + TAU s source), c = cos(b) - 1,
// s = sin(b); the unitary variant also rotates the source:
// source' = source + (c source - TAU s target).
template <int TAU, bool UNIT, typename T>
__device__ __forceinline__ void vop(T &target, T &source, T s, T c) {
    using A = Ar<T>;
    const T ss = A::mul(s, source);
    const T t2 = A::add(target, TAU > 0 ? A::fma(c, target, ss) : A::fma(c, target, -ss));
    if (UNIT) {
        const T st = A::mul(s, target);
        source = A::add(source, TAU > 0 ? A::fma(c, source, -st) : A::fma(c, source, st));
    }
    target = t2;
}

template <int TAU, bool HUB, bool UNIT, typename T>
__device__ __forceinline__ void vop_pair(T &h, T &p, T s, T c) {
    if (HUB) vop<TAU, UNIT>(h, p, s, c);
    else vop<TAU, UNIT>(p, h, s, c);
}

// Magnitude bits of a coefficient (zero for +0 and -0 only).
template <typename T>
__device__ __forceinline__ unsigned nzbits(T v) {
    if constexpr (sizeof(T) == 4) {
        return __float_as_uint(v) & 0x7fffffffu;
    } else {
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
        return unsigned(b) | unsigned(b >> 32);
    }
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
__device__ __forceinline__ int wrap_down(int v, int n) {
    while (v >= n) v -= n;
    return v;
}
__device__ __forceinline__ int wrap_up(int v, int n) {
    while (v < 0) v += n;
    return v;
}

// Shared rows hold W_IN elements of type E. 16-byte chunks are XOR-swizzled
// within groups of eight chunks (chunk c is stored at c ^ ((c >> 3) & MASK))
// so that both access patterns are free of bank conflicts: a lane reading its
// 8 consecutive columns with 16-byte loads, and a warp reading 32
// consecutive columns one element per thread.
template <typename E>
__device__ __forceinline__ int swz(int e) {
    constexpr int EPC = 16 / int(sizeof(E));
    constexpr int MASK = sizeof(E) == 4 ? 1 : (sizeof(E) == 8 ? 3 : 7);
    const int chunk = e / EPC;
    return (chunk ^ ((chunk >> 3) & MASK)) * EPC + (e % EPC);
}

// The 8 consecutive columns of lane `lane` of a shared row.
template <typename T>
__device__ __forceinline__ void sload8(T (&v)[LANE_COLS], const T *row, int lane) {
    const int c0 = LANE_COLS * lane;
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(row + swz<T>(c0));
        const float4 b = *reinterpret_cast<const float4 *>(row + swz<T>(c0 + 4));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 d = *reinterpret_cast<const double2 *>(row + swz<T>(c0 + 2 * k));
            v[2 * k] = d.x;
            v[2 * k + 1] = d.y;
        }
    }
}

template <typename T>
__device__ __forceinline__ void sstore8(T *row, int lane, const T (&v)[LANE_COLS]) {
    const int c0 = LANE_COLS * lane;
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(row + swz<T>(c0)) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(row + swz<T>(c0 + 4)) = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            *reinterpret_cast<double2 *>(row + swz<T>(c0 + 2 * k)) = make_double2(v[2 * k], v[2 * k + 1]);
    }
}

// 8 coefficient pairs (x = m, y = s) of lane `lane` from a shared pair row.
template <typename T>
__device__ __forceinline__ void sload8pair(T (&m)[LANE_COLS], T (&s)[LANE_COLS], const typename Ar<T>::T2 *row,
                                           int lane) {
    using T2 = typename Ar<T>::T2;
    const int c0 = LANE_COLS * lane;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = *reinterpret_cast<const float4 *>(row + swz<T2>(c0 + 2 * k));
            m[2 * k] = v.x;
            s[2 * k] = v.y;
            m[2 * k + 1] = v.z;
            s[2 * k + 1] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < LANE_COLS; ++k) {
            const double2 v = row[swz<T2>(c0 + k)];
            m[k] = v.x;
            s[k] = v.y;
        }
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

// One box by TMA: the box at (0, c1, c2, c3) of `map` into `dst`, completing
// its bytes on the mbarrier.
__device__ __forceinline__ void tma_row(void *dst, const CUtensorMap *map, int c1, int c2, int c3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::smem_addr(bar))
        : "memory");
}
// The box at (0, c1, c2, c3, c4) of a five-dimensional `map` into `dst`.
__device__ __forceinline__ void tma_box5(void *dst, const CUtensorMap *map, int c1, int c2, int c3, int c4,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];\n" ::"r"(tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(tc::smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Copies the strip's 256 columns of one global row into a (swizzled) shared
// row: lane l copies strip columns 8l .. 8l+7. xb: wrapped global column of
// strip column 0; nowrap: the strip lies inside [0, Nx).
template <typename E>
__device__ __forceinline__ void copy_strip_row(E *dst, const E *grow, int xb, int Nx, bool nowrap, bool vec,
                                               int lane) {
    constexpr int EPC = 16 / int(sizeof(E));
    const int c0 = LANE_COLS * lane;
    if (vec) {
#pragma unroll
        for (int k = 0; k < LANE_COLS / EPC; ++k) {
            const int sc = c0 + k * EPC;
            const int gc = nowrap ? xb + sc : wrap_down(xb + sc, Nx);
            cp_async16(dst + swz<E>(sc), grow + gc);
        }
    } else {
#pragma unroll
        for (int e = 0; e < LANE_COLS; ++e) {
            const int sc = c0 + e;
            cp_async_small<sizeof(E)>(dst + swz<E>(sc), grow + wrap_down(xb + sc, Nx));
        }
    }
}

template <typename T, int K, int R, bool INTER>
struct SweepLayout {
    using T2 = typename Ar<T>::T2;
    static constexpr int NYS = INTER ? 2 : 3;  // y-pass pairs: C_Y, V_Y (+ V_X for Eq. 23)
    static constexpr int NXS = INTER ? 2 : 1;  // x-pass pairs: C_X (+ V_X for Eq. 28)
    static constexpr size_t STATE = size_t(K) * 2 * 3 * R * W_IN * sizeof(T);
    static constexpr size_t YST = size_t(K) * NYS * R * W_IN * sizeof(T2);
    static constexpr size_t XST = size_t(K) * NXS * R * W_IN * sizeof(T2);
    static constexpr size_t BAR_OFF = STATE + YST + XST;  // mbarriers of the two TMA copy groups
    static constexpr size_t ORD_OFF = BAR_OFF + 16;       // the CTA's share index (start order)
    static constexpr size_t SMEM = ORD_OFF + 16;
};

template <typename T, int K, int R, int NY>
struct SweepCfg {
    static constexpr int NT = W_IN * K / NY;
    // two resident CTAs per SM when the block is small and its shared memory allows it
    static constexpr int MINB =
        (sizeof(T) == 4 && NT <= 256 && SweepLayout<T, K, R, true>::SMEM <= 114 * 1024) ? 2 : 1;
    static constexpr int NWARP = NT / 32;
    static_assert(W_IN * K % NY == 0, "tasks must divide");
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    static_assert(K * R <= NWARP * 4, "x-pass row tasks per warp");
};

template <typename T>
struct YPipe {
    T S2, S4, S6, S8, S10, S12, S14, S16;  // one saved value per y-shift
    T m1, s1, m2, s2, m3, s3;              // collision coefficients of rows R-1, R-2, R-3
    T d0, d1, d2, d3;                      // x-partner delayed by 4 rows
    T vc1, vs1, vc2, vs2, vc3, vs3, vc4, vs4;  // V_Y pair of rows R-1 .. R-4
    T wc1, ws1, wc2, ws2, wc3, ws3, wc4, ws4;  // V_X pair of rows R-1 .. R-4 (Eq. 23 only)
    __device__ __forceinline__ void zero() {
        S2 = S4 = S6 = S8 = S10 = S12 = S14 = S16 = T(0);
        m1 = s1 = m2 = s2 = m3 = s3 = T(0);
        d0 = d1 = d2 = d3 = T(0);
        vc1 = vs1 = vc2 = vs2 = vc3 = vs3 = vc4 = vs4 = T(0);
        wc1 = ws1 = wc2 = ws2 = wc3 = ws3 = wc4 = ws4 = T(0);
    }
};

// One tile: output rows [yb, ye) of a strip, level 0 fed from yb - 4K.
// Returns true (uniformly over the CTA) if the error flag is set (a bounded
// copy wait ran out); the CTA's copy barriers are then left as they are and
// the caller stops.
// TMA_ONLY: the caller guarantees TMA copies for every strip (the seam
// layout); the per-lane copy path is compiled out, and a strip that could not
// copy with TMA sets the error flag instead.
template <typename T, int K, int R, int NY, bool INTER, bool UNIT, int FAM, bool TMA_ONLY = false>
__device__ __forceinline__ bool sweep_body(const SweepArgs &A, int strip, int yb, int ye, unsigned char *smem_raw,
                                           const SweepMaps *M = nullptr, bool merged = false,
                                           bool swap = false) {
    using Cfg = SweepCfg<T, K, R, NY>;
    using L = SweepLayout<T, K, R, INTER>;
    using T2 = typename Ar<T>::T2;
    using Fm = Fam<FAM>;
    constexpr int NT = Cfg::NT;
    constexpr int NWARP = Cfg::NWARP;
    constexpr int NYS = L::NYS, NXS = L::NXS;
    constexpr bool SHR = shear_collisions<T, UNIT>();
    // coefficient stash slots, in the order of the pair planes (so that a
    // group's planes arrive in one TMA box): x-pass (Eq. 28) V_X then C_X,
    // (Eq. 23) C_X; y-pass C_Y, V_Y (+ V_X for Eq. 23)
    constexpr int XS_C = INTER ? 1 : 0, XS_V = 0;
    static_assert(!INTER || (Fm::VX + 1 == Fm::CX && Fm::CY + 1 == Fm::VY), "pair planes of a copy group adjacent");

    T *const buf = reinterpret_cast<T *>(smem_raw);
    T2 *const yst = reinterpret_cast<T2 *>(smem_raw + L::STATE);
    T2 *const xst = reinterpret_cast<T2 *>(smem_raw + L::STATE + L::YST);

    const int Nx = A.Nx, Ny = A.Ny;
    const int P = Nx * Ny;  // < 2^31 (checked on the host)
    // swap: read A.q_out and write A.q_in (the odd passes of a persistent launch)
    const T *__restrict__ qin = static_cast<const T *>(swap ? A.q_out : A.q_in);
    T *__restrict__ qout = static_cast<T *>(swap ? const_cast<void *>(A.q_in) : A.q_out);
    const T2 *__restrict__ cpairs = static_cast<const T2 *>(A.coef);
    const bool vec = A.vec != 0;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // strip geometry (SweepArgs::seam): xbase = global column of strip column
    // 0 (may be < 0), [o_lo, o_hi) = the global columns the strip writes
    constexpr int HALF_W = W_IN / 2;
    const bool seam_strip = A.seam && strip == 0;
    int xbase, o_lo, o_hi;
    if (!A.seam) {
        o_lo = strip * A.w_valid;
        o_hi = min(o_lo + A.w_valid, Nx);
        xbase = o_lo - 4 * K;
    } else if (seam_strip) {
        xbase = Nx - HALF_W;  // writes strip columns [4K, W_IN - 4K), wrapped
        o_lo = o_hi = 0;
    } else {
        o_lo = HALF_W - 4 * K + (strip - 1) * A.w_valid;
        o_hi = min(o_lo + A.w_valid, Nx - HALF_W + 4 * K);
        xbase = min(o_lo - 4 * K, Nx - W_IN);
    }
    const int xb = wrapi(xbase, Nx);
    const bool nowrap = xbase >= 0 && xbase + W_IN <= Nx;
    // the seam strip's shared rows hold its two halves swapped (see SweepMaps):
    // strip column c sits at c ^ 128, i.e. lane l's 8 columns at lane l ^ 16's
    const int sl = seam_strip ? lane ^ (HALF_W / LANE_COLS) : lane;
    const int scx = seam_strip ? HALF_W : 0;
    const int F0 = yb - 4 * K;                // first row fed to level 0
    const int nit = (ye - yb + 8 * K + R - 1) / R + K - 1;

    auto bufrow = [&](int j, int half, int comp, int ir) -> T * {
        return buf + ((((j * 2 + half) * 3 + comp) * R + ir) * W_IN);
    };
    // coefficient stashes: [slot][level K-1 .. 0][R rows], the order of a
    // merged TMA box (level K-1's block has the lowest global rows)
    auto ystrow = [&](int j, int slot, int ir) -> T2 * { return yst + (((slot * K + K - 1 - j) * R + ir) * W_IN); };
    auto xstrow = [&](int j, int slot, int ir) -> T2 * { return xst + (((slot * K + K - 1 - j) * R + ir) * W_IN); };
    // first (unwrapped) row handled by level j in iteration it
    auto arow = [&](int j, int it) { return F0 + (it - j) * R - 4 * j; };
    auto active = [&](int j, int it) { return it >= j && arow(j, it) <= ye - 1 + 4 * (K - j); };
    // wrapped global row of row ir of level j in iteration it, from the
    // wrapped first level-0 row of the current iteration (no division)
    int itcur = 0, r0w = wrapi(F0, Ny);
    auto growof = [&](int j, int it, int ir) {
        return wrap_down(wrap_up(r0w + (it - itcur) * R - j * (R + 4) + ir, Ny), Ny);
    };

    const T2 *const pCX = cpairs + size_t(Fm::CX) * P;
    const T2 *const pCY = cpairs + size_t(Fm::CY) * P;
    const T2 *const pVX = cpairs + size_t(Fm::VX) * P;
    const T2 *const pVY = cpairs + size_t(Fm::VY) * P;

    // Row segments copied per iteration are spread over the warps; a warp
    // copies one 256-column row segment per task (each lane 8 columns).
    // level-0 state rows for iteration it (3 components x R rows)
    auto copy_state0 = [&](int it, int half) {
        for (int task = warp; task < 3 * R; task += NWARP) {
            const int slot = task / R, ir = task % R;
            const T *src = qin + size_t(Fm::plane_of_slot(slot)) * P + size_t(growof(0, it, ir)) * Nx;
            copy_strip_row(bufrow(0, half, slot, ir), src, xb, Nx, nowrap, vec, lane);
        }
    };
    // x-pass coefficient rows of iteration it, all active levels
    auto copy_xstash = [&](int it) {
        for (int task = warp; task < K * NXS * R; task += NWARP) {
            const int j = task / (NXS * R), rem = task % (NXS * R);
            const int slot = rem / R, ir = rem % R;
            if (!active(j, it)) continue;
            const T2 *plane = slot == XS_C ? pCX : pVX;
            copy_strip_row(xstrow(j, slot, ir), plane + size_t(growof(j, it, ir)) * Nx, xb, Nx, nowrap, vec, lane);
        }
    };
    // y-pass coefficient rows of iteration it
    auto copy_ystash = [&](int it) {
        for (int task = warp; task < K * NYS * R; task += NWARP) {
            const int j = task / (NYS * R), rem = task % (NYS * R);
            const int slot = rem / R, ir = rem % R;
            const T2 *plane = slot == 0 ? pCY : (slot == 1 ? pVY : pVX);
            copy_strip_row(ystrow(j, slot, ir), plane + size_t(growof(j, it, ir)) * Nx, xb, Nx, nowrap, vec, lane);
        }
    };

    // TMA path (FP32, a strip that does not wrap around x, 8-column aligned).
    // Group X (x-pass coefficients of every active level and the level-0 state
    // rows) and group Y (y-pass coefficients) each complete on one mbarrier.
    // A box carries whole R-row blocks: of all K levels and of the group's
    // adjacent pair planes at once (V_X, C_X resp. C_Y, V_Y with Eq. 28), and of
    // the family's adjacent state planes (TM: one box of 3 planes; TE: 2 + 1).
    // An iteration then issues 3 (TM) or 4 (TE) loads, by lane 0 of as many
    // warps: measured on GB300, each issue holds its warp for hundreds of
    // cycles, so the number of issues, not the bytes, is what costs.
    uint64_t *const tbar = reinterpret_cast<uint64_t *>(smem_raw + L::BAR_OFF);
    bool use_tma = false;
    if constexpr (std::is_same<T, float>::value)
        use_tma = M != nullptr && ((nowrap && (xb & 7) == 0) || seam_strip) && (tc::smem_addr(smem_raw) & 1023u) == 0;
    if constexpr (TMA_ONLY) {
        if (!use_tma) {  // uniform over the CTA
            if (A.error) atomicExch(A.error, 1);
            return true;
        }
        use_tma = true;
    }
    uint32_t tph_x = 0, tph_y = 0;
    constexpr uint32_t SROW = W_IN * sizeof(T), CROW = W_IN * sizeof(T2);
    // the R rows of a block (level j) of one pair plane: one box, or R one-row
    // boxes where the block wraps around y
    auto tma_block = [&](void *dst, int j, int it, int plane, uint64_t *bar) {
        const int r0 = growof(j, it, 0);
        if (seam_strip) {
            if (r0 + R <= Ny) {
                tma_box5(dst, &M->seam_coef_r, 0, 0, r0, plane, bar);
            } else {
                for (int ir = 0; ir < R; ++ir)
                    tma_box5(static_cast<unsigned char *>(dst) + ir * CROW, &M->seam_coef, 0, 0, growof(j, it, ir),
                             plane, bar);
            }
        } else if (r0 + R <= Ny) {
            tma_row(dst, &M->coef_r, xb >> 3, r0, plane, bar);
        } else {
            for (int ir = 0; ir < R; ++ir)
                tma_row(static_cast<unsigned char *>(dst) + ir * CROW, &M->coef, xb >> 3, growof(j, it, ir), plane,
                        bar);
        }
    };
    // the blocks of n adjacent pair planes (stash slots slot0..) for all K
    // levels: one merged box where they neither wrap around y nor straddle a
    // group of R + 4 rows, else one box (or R one-row boxes) per level and plane
    const bool merge_ok = merged && K > 1 && !seam_strip;
    auto tma_planes = [&](bool ystash, int slot0, int n, int it, int plane0, uint64_t *bar) {
        const int r_top = growof(K - 1, it, 0);
        const int b0 = r_top % (R + 4);
        if (merge_ok && r_top + (K - 1) * (R + 4) + R <= Ny && b0 <= 4) {
            T2 *const top = ystash ? ystrow(K - 1, slot0, 0) : xstrow(K - 1, slot0, 0);
            tma_box5(top, n == 2 ? &M->coef_m2 : &M->coef_m1, xb >> 3, b0, r_top / (R + 4), plane0, bar);
        } else {
            for (int q = 0; q < n; ++q)
                for (int j = 0; j < K; ++j)
                    tma_block(ystash ? ystrow(j, slot0 + q, 0) : xstrow(j, slot0 + q, 0), j, it, plane0 + q, bar);
        }
    };
    // level-0 state rows: planes p0 .. p0 + n - 1 into buffer slots s0 ..
    auto tma_state = [&](int it, int half, int p0, int n, int s0, uint64_t *bar) {
        const int r0 = growof(0, it, 0);
        if (seam_strip) {
            if (r0 + R <= Ny) {
                const CUtensorMap *map = n == 3 ? &M->seam_state_r3 : (n == 2 ? &M->seam_state_r2 : &M->seam_state_r1);
                tma_box5(bufrow(0, half, s0, 0), map, 0, 0, r0, p0, bar);
            } else {
                for (int q = 0; q < n; ++q)
                    for (int ir = 0; ir < R; ++ir)
                        tma_box5(bufrow(0, half, s0 + q, ir), &M->seam_state, 0, 0, growof(0, it, ir), p0 + q, bar);
            }
        } else if (r0 + R <= Ny) {
            const CUtensorMap *map = n == 3 ? &M->state_r3 : (n == 2 ? &M->state_r2 : &M->state_r1);
            tma_row(bufrow(0, half, s0, 0), map, xb >> 3, r0, p0, bar);
        } else {
            for (int q = 0; q < n; ++q)
                for (int ir = 0; ir < R; ++ir)
                    tma_row(bufrow(0, half, s0 + q, ir), &M->state, xb >> 3, growof(0, it, ir), p0 + q, bar);
        }
    };
    constexpr int NSB = Fm::N1 > 0 ? 2 : 1;  // state boxes of the family
    auto tma_group_x = [&](int it, bool with_state, int half) {
        // every level's blocks are loaded (an inactive level's are not read)
        const uint32_t row_bytes = uint32_t(K * NXS) * CROW + (with_state ? 3u * SROW : 0u);
        if (tid == 0) mbar_arrive_expect_tx(&tbar[0], uint32_t(R) * row_bytes);
        const int ntask = 1 + (with_state ? NSB : 0);
        for (int t = warp + NWARP * lane; t < ntask; t += 32 * NWARP) {
            if (t == 0) {
                if constexpr (INTER) tma_planes(false, XS_V, 2, it, Fm::VX, &tbar[0]);
                else tma_planes(false, XS_C, 1, it, Fm::CX, &tbar[0]);
            } else if (t == 1) {
                tma_state(it, half, Fm::B0, Fm::N0, 0, &tbar[0]);
            } else {
                tma_state(it, half, Fm::B1, Fm::N1, Fm::N0, &tbar[0]);
            }
        }
    };
    auto tma_group_y = [&](int it) {
        if (tid == 0) mbar_arrive_expect_tx(&tbar[1], uint32_t(R * K * NYS) * CROW);
        constexpr int ntask = INTER ? 1 : 2;
        for (int t = warp + NWARP * lane; t < ntask; t += 32 * NWARP) {
            if (t == 0) tma_planes(true, 0, 2, it, Fm::CY, &tbar[1]);  // C_Y, V_Y
            else tma_planes(true, 2, 1, it, Fm::VX, &tbar[1]);         // V_X (Eq. 23)
        }
    };
    // bounded wait for a copy group (the warp sleeps until the copies land; at
    // most 2 s): a timeout sets the error flag (the results of the launch are
    // then invalid) instead of hanging
    auto tma_wait = [&](int b, uint32_t ph) {
        if (!tc::mbar_wait_suspended(&tbar[b], ph, 1000000u, 2000000000ull) && A.error) atomicExch(A.error, 1);
    };

    for (int i = tid; i < int(L::STATE / sizeof(T)); i += NT) buf[i] = T(0);

    // ---- y-pass tasks: fixed (level, column) per thread slot ---------------
    // Only the last slot can hold the last level (tasks are ordered by level).
    constexpr int LVL = 2 * 3 * R * W_IN;   // elements of one level's state buffers
    constexpr int HALF = 3 * R * W_IN;      // one half (3 components x R rows)
    constexpr int YSLOT = K * R * W_IN;     // one y-stash slot (all levels)
    int yj[NY];
    const T *st_base[NY];
    const T2 *ys_base[NY];
#pragma unroll
    for (int u = 0; u < NY; ++u) {
        const int task = tid + u * NT;
        yj[u] = task / W_IN;
        const int c = task % W_IN;
        st_base[u] = buf + yj[u] * LVL + swz<T>(c ^ scx);
        ys_base[u] = yst + (K - 1 - yj[u]) * R * W_IN + swz<T2>(c ^ scx);
    }
    const int c_last = (tid + (NY - 1) * NT) % W_IN;
    const bool last_is_final = yj[NY - 1] == K - 1;  // uniform per warp
    const int gcol = xbase + c_last;
    const bool col_ok = seam_strip ? (c_last >= 4 * K && c_last < W_IN - 4 * K) : (gcol >= o_lo && gcol < o_hi);
    const int gx = gcol >= Nx ? gcol - Nx : gcol;
    T *const qo_h = qout + size_t(Fm::H) * P + gx;
    T *const qo_px = qout + size_t(Fm::PX) * P + gx;
    T *const qo_py = qout + size_t(Fm::PY) * P + gx;

    // Generic writes of shared memory that a TMA load later overwrites (the
    // zeroing here, the x-pass's in-place level-0 rows) are fenced to the async
    // proxy by their writers before the barrier that precedes the issue. Rows
    // that threads only read are reused after a barrier alone.
    if (use_tma) tc::fence_proxy_async();
    if (use_tma && tid == 0) {
        tc::mbar_init(&tbar[0], 1);
        tc::mbar_init(&tbar[1], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();  // zeroed buffers before the async copies land
    if (use_tma) {
        tma_group_x(0, true, 0);  // waited for in the first x-pass
    } else {
        copy_state0(0, 0);
        copy_xstash(0);
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();

    YPipe<T> yp[NY];
#pragma unroll
    for (int u = 0; u < NY; ++u) yp[u].zero();
    bool vy_prev_on = false;  // the previous iteration's V_Y' pairs were nonzero for the warp

    for (int it = 0; it < nit; ++it) {
        const int cur = it & 1;
        if (use_tma) {
            tma_group_y(it);
        } else {
            copy_ystash(it);
            cp_async_commit();
        }

        // ---- phase 1: x-pass, one warp per (level, row) -------------------
        for (int task = warp; task < K * R; task += NWARP) {
            const int j = task / R, ir = task % R;
            if (!active(j, it)) continue;
            if (use_tma) {
                tma_wait(0, tph_x);
                tc::fence_after_sync();
            }
            T *rh = bufrow(j, cur, Fm::SH, ir);
            T *rp = bufrow(j, cur, Fm::SPX, ir);
            T m[LANE_COLS], s[LANE_COLS], h[LANE_COLS], p[LANE_COLS];
            sload8pair(m, s, xstrow(j, XS_C, ir), sl);
            sload8(h, rh, sl);
            sload8(p, rp, sl);
            constexpr int SG = Fm::SGX;
            // ops 1-8
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_left(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_right(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_right(h);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_left(h);
            // V_X' is the identity where the potential angle is zero, i.e.
            // wherever the index field is locally uniform (most of a lattice
            // holding compact objects): a warp whose 256 columns all have zero
            // pairs skips both applications (the result is unchanged but for
            // the sign of a zero).
            T vc[LANE_COLS], vs[LANE_COLS];
            bool vx_on = false;
            if constexpr (INTER) {
                sload8pair(vc, vs, xstrow(j, XS_V, ir), sl);
                unsigned nz = 0;
#pragma unroll
                for (int c = 0; c < LANE_COLS; ++c) nz |= nzbits(vc[c]) | nzbits(vs[c]);
                vx_on = __any_sync(0xffffffffu, nz != 0u);
                if (vx_on) {
#pragma unroll
                    for (int c = 0; c < LANE_COLS; ++c)
                        vop_pair<Fm::TX, Fm::VX_HUB, UNIT>(h[c], p[c], vs[c], vc[c]);
                }
            }
            // ops 9-16
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_right(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_left(p);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<false, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_left(h);
#pragma unroll
            for (int c = 0; c < LANE_COLS; ++c) rot<true, SG, SHR>(h[c], p[c], m[c], s[c]);
            shift_from_right(h);
            if constexpr (INTER) {
                if (vx_on) {
#pragma unroll
                    for (int c = 0; c < LANE_COLS; ++c)
                        vop_pair<Fm::TX, Fm::VX_HUB, UNIT>(h[c], p[c], vs[c], vc[c]);
                }
            }
            sstore8(rh, sl, h);
            sstore8(rp, sl, p);
            if (use_tma && j == 0) tc::fence_proxy_async();  // level-0 rows are TMA targets again later
        }
        if (use_tma) {
            tph_x ^= 1u;
        } else {
            cp_async_wait_all();
        }
        __syncthreads();

        // next iteration's x-pass coefficients and level-0 rows land while the
        // y-pass runs
        if (use_tma) {
            if (it + 1 < nit) tma_group_x(it + 1, active(0, it + 1), cur ^ 1);
        } else {
            if (it + 1 < nit) {
                copy_xstash(it + 1);
                if (active(0, it + 1)) copy_state0(it + 1, cur ^ 1);
            }
            cp_async_commit();
        }

        // ---- phase 2: y-pass, one thread per (level, column) --------------
        // The NY column pipelines of a thread advance row by row together so
        // that their independent dependency chains interleave. A pipeline runs
        // even in iterations where its level is inactive (before its first or
        // after its last needed row): those rows are never read by a later
        // level nor written to global memory, and running unconditionally
        // keeps the loop-carried pipeline registers free of merge copies.
        const int hin = cur * HALF, hout = (cur ^ 1) * HALF;
        const int rout0 = arow(yj[NY - 1], it) - 4;  // first output row of the last slot
        if (use_tma) {  // the y-pass coefficients of all levels have landed
            tma_wait(1, tph_y);
            tc::fence_after_sync();
        }
        // V_Y' skip (Eq. 28): the applications of this iteration use the V_Y
        // pairs of the previous iteration's rows and of this one's; when all
        // of them are zero for the warp (a locally uniform index field) the
        // V_Y' rows, their loads and the delay line are skipped (the delay
        // line then holds zeros already).
        bool vy_on = true;
        if constexpr (INTER) {
            unsigned nz = 0;
#pragma unroll
            for (int u = 0; u < NY; ++u)
#pragma unroll
                for (int ir = 0; ir < R; ++ir) {
                    const T2 v = ys_base[u][YSLOT + ir * W_IN];
                    nz |= nzbits(v.x) | nzbits(v.y);
                }
            const bool cur_on = __any_sync(0xffffffffu, nz != 0u);
            vy_on = cur_on || vy_prev_on;
            vy_prev_on = cur_on;
        }
        auto rows = [&](auto final_tag, auto von_tag) {
            constexpr bool FINAL = decltype(final_tag)::value;
            constexpr bool VON = decltype(von_tag)::value;  // V_Y' applied (always for Eq. 23)
#pragma unroll
            for (int ir = 0; ir < R; ++ir) {
#pragma unroll
                for (int u = 0; u < NY; ++u) {
                    YPipe<T> &Y = yp[u];
                    constexpr int SG = Fm::SGY;
                    const T *in = st_base[u] + hin;
                    const T2 *ys = ys_base[u];
                    const T2 cy = ys[ir * W_IN];
                    const T2 vy = VON ? ys[YSLOT + ir * W_IN] : T2{T(0), T(0)};
                    const T m0 = cy.x, s0 = cy.y;
                    T h = in[(Fm::SH * R + ir) * W_IN];
                    T p = in[(Fm::SPY * R + ir) * W_IN];
                    const T px0 = in[(Fm::SPX * R + ir) * W_IN];
                    rot<true, SG, SHR>(h, p, m0, s0);                // op 1  C+   (row R)
                    { const T t = Y.S2; Y.S2 = p; p = t; }      // op 2  p <- p(r-1)
                    rot<false, SG, SHR>(h, p, m0, s0);               // op 3  C    (row R)
                    { const T t = Y.S4; Y.S4 = h; h = t; }      // op 4  p <- p(r+1): now row R-1
                    rot<true, SG, SHR>(h, p, Y.m1, Y.s1);            // op 5  C+   (row R-1)
                    { const T t = Y.S6; Y.S6 = p; p = t; }      // op 6  h <- h(r+1): now row R-2
                    rot<false, SG, SHR>(h, p, Y.m2, Y.s2);           // op 7  C    (row R-2)
                    { const T t = Y.S8; Y.S8 = h; h = t; }      // op 8  h <- h(r-1)
                    if constexpr (INTER && VON)
                        vop_pair<Fm::TY, Fm::VY_HUB, UNIT>(h, p, Y.vs2, Y.vc2);  // V_Y' (row R-2)
                    rot<false, SG, SHR>(h, p, Y.m2, Y.s2);           // op 9  C    (row R-2)
                    { const T t = Y.S10; Y.S10 = h; h = t; }    // op 10 p <- p(r+1): now row R-3
                    rot<true, SG, SHR>(h, p, Y.m3, Y.s3);            // op 11 C+   (row R-3)
                    { const T t = Y.S12; Y.S12 = p; p = t; }    // op 12 p <- p(r-1)
                    rot<false, SG, SHR>(h, p, Y.m3, Y.s3);           // op 13 C    (row R-3)
                    { const T t = Y.S14; Y.S14 = h; h = t; }    // op 14 h <- h(r-1)
                    rot<true, SG, SHR>(h, p, Y.m3, Y.s3);            // op 15 C+   (row R-3)
                    { const T t = Y.S16; Y.S16 = p; p = t; }    // op 16 h <- h(r+1): now row R-4
                    T px = Y.d3;
                    Y.d3 = Y.d2; Y.d2 = Y.d1; Y.d1 = Y.d0; Y.d0 = px0;
                    if constexpr (INTER) {
                        if constexpr (VON) vop_pair<Fm::TY, Fm::VY_HUB, UNIT>(h, p, Y.vs4, Y.vc4);  // V_Y' (row R-4)
                    } else {
                        vop_pair<Fm::TX, Fm::VX_HUB, UNIT>(h, px, Y.ws4, Y.wc4);  // V_X  (row R-4)
                        vop_pair<Fm::TY, Fm::VY_HUB, UNIT>(h, p, Y.vs4, Y.vc4);   // V_Y  (row R-4)
                        const T2 vx = ys[2 * YSLOT + ir * W_IN];
                        Y.wc4 = Y.wc3; Y.ws4 = Y.ws3; Y.wc3 = Y.wc2; Y.ws3 = Y.ws2;
                        Y.wc2 = Y.wc1; Y.ws2 = Y.ws1; Y.wc1 = vx.x; Y.ws1 = vx.y;
                    }
                    Y.m3 = Y.m2; Y.s3 = Y.s2;
                    Y.m2 = Y.m1; Y.s2 = Y.s1;
                    Y.m1 = m0;   Y.s1 = s0;
                    if constexpr (VON) {
                        Y.vc4 = Y.vc3; Y.vs4 = Y.vs3; Y.vc3 = Y.vc2; Y.vs3 = Y.vs2;
                        Y.vc2 = Y.vc1; Y.vs2 = Y.vs1; Y.vc1 = vy.x; Y.vs1 = vy.y;
                    }
                    if (FINAL && u == NY - 1) {
                        const int rout = rout0 + ir;
                        if (col_ok && rout >= yb && rout < ye) {
                            const size_t o = size_t(rout) * Nx;
                            qo_h[o] = h;
                            qo_px[o] = px;
                            qo_py[o] = p;
                        }
                    } else {
                        T *out = const_cast<T *>(st_base[u]) + LVL + hout;  // level j+1, other half
                        out[(Fm::SH * R + ir) * W_IN] = h;
                        out[(Fm::SPX * R + ir) * W_IN] = px;
                        out[(Fm::SPY * R + ir) * W_IN] = p;
                    }
                }
            }
        };
        using tru = std::integral_constant<bool, true>;
        using fls = std::integral_constant<bool, false>;
        if (last_is_final) {
            if (vy_on) rows(tru(), tru());
            else rows(tru(), fls());
        } else {
            if (vy_on) rows(fls(), tru());
            else rows(fls(), fls());
        }
        itcur = it + 1;
        r0w = wrap_down(r0w + R, Ny);
        if (use_tma) {
            tph_y ^= 1u;
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
    }
    // every copy issued was waited for: the barriers are idle unless a wait
    // ran out (here or in another CTA; the pass's results are then invalid)
    const bool failed = A.error && __syncthreads_or(*reinterpret_cast<volatile int *>(A.error) != 0);
    if (use_tma && !failed && tid == 0) {
        tc::mbar_inval(&tbar[0]);
        tc::mbar_inval(&tbar[1]);
    }
    return failed;
}

template <typename T, int K, int R, int NY, bool INTER, bool UNIT>
__global__ void __launch_bounds__(SweepCfg<T, K, R, NY>::NT, SweepCfg<T, K, R, NY>::MINB)
    sweep_kernel(const __grid_constant__ SweepParams prm) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const SweepMaps *maps = prm.tma ? &prm.m : nullptr;
    const int Ny = prm.a.Ny;
    int u, u1;  // this CTA's row units [u, u1) (nsx * Ny < 2^31, checked on the host)
    if (prm.a.chunk <= 0) {
        const SweepSplit &sp = prm.split[blockIdx.z];
        int b = blockIdx.x;
        if (sp.profile == 2 && prm.a.order) {  // share index = start order
            int *const ord = reinterpret_cast<int *>(smem_raw + SweepLayout<T, K, R, INTER>::ORD_OFF);
            if (threadIdx.x == 0) {
                const unsigned k = atomicAdd(prm.a.order, 1u);
                if (k + 1 == gridDim.x) atomicExch(prm.a.order, 0u);  // the last to start: zero for the next launch
                *ord = int(k % gridDim.x);
            }
            __syncthreads();
            b = *ord;
        }
        u = int(sp.share_begin(b, gridDim.x));
        u1 = int(sp.share_begin(b + 1, gridDim.x));
    } else {
        const int strip = prm.tiles_fastest ? blockIdx.y : blockIdx.x;
        const int chunk = prm.tiles_fastest ? blockIdx.x : blockIdx.y;
        u = strip * Ny + chunk * prm.a.chunk;
        u1 = min(u + prm.a.chunk, (strip + 1) * Ny);
    }
    while (u < u1) {
        const int s = u / Ny;
        const int y0 = u - s * Ny;
        const int y1 = min(Ny, y0 + (u1 - u));
        const bool failed =
            prm.a.fam0 + int(blockIdx.z) != 0
                ? sweep_body<T, K, R, NY, INTER, UNIT, 1>(prm.a, s, y0, y1, smem_raw, maps, prm.merged != 0)
                : sweep_body<T, K, R, NY, INTER, UNIT, 0>(prm.a, s, y0, y1, smem_raw, maps, prm.merged != 0);
        if (failed) break;
        u += y1 - y0;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return EncodeTiledFn(nullptr);
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor maps of one FP32 pass (see SweepMaps); false when TMA cannot be used
// (Nx not a multiple of 8, no encoder), in which case the kernel copies with
// cp.async. *merged: the merged-level coefficient maps are valid.
inline bool make_sweep_maps(const SweepArgs &a, int K, int R, SweepMaps &m, int *merged) {
    const EncodeTiledFn fn = encode_tiled_fn();
    *merged = 0;
    if (!fn || a.Nx % 8 != 0) return false;
    const cuuint64_t Nx = cuuint64_t(a.Nx), Ny = cuuint64_t(a.Ny);
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    const cuuint64_t sdim[4] = {8, Nx / 8, Ny, 6};
    const cuuint64_t sstr[3] = {32, Nx * 4, Nx * Ny * 4};
    auto state_map = [&](CUtensorMap *map, cuuint32_t rows, cuuint32_t comps) {
        const cuuint32_t box[4] = {8, 32, rows, comps};
        return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(a.q_in), sdim, sstr, box, one,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!state_map(&m.state, 1, 1) || !state_map(&m.state_r1, cuuint32_t(R), 1) ||
        !state_map(&m.state_r2, cuuint32_t(R), 2) || !state_map(&m.state_r3, cuuint32_t(R), 3))
        return false;
    const cuuint64_t cdim[4] = {16, Nx / 8, Ny, cuuint64_t(NPAIR)};
    const cuuint64_t cstr[3] = {64, Nx * 8, Nx * Ny * 8};
    auto coef_map = [&](CUtensorMap *map, cuuint32_t rows) {
        const cuuint32_t box[4] = {16, 32, rows, 1};
        return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(a.coef), cdim, cstr, box, one,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!coef_map(&m.coef, 1) || !coef_map(&m.coef_r, cuuint32_t(R))) return false;
    const cuuint64_t G = cuuint64_t(R + 4);
    if (K > 1 && Ny % G == 0) {
        const cuuint64_t mdim[5] = {16, Nx / 8, G, Ny / G, cuuint64_t(NPAIR)};
        const cuuint64_t mstr[4] = {64, Nx * 8, G * Nx * 8, Nx * Ny * 8};
        auto merged_map = [&](CUtensorMap *map, cuuint32_t planes) {
            const cuuint32_t box[5] = {16, 32, cuuint32_t(R), cuuint32_t(K), planes};
            return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(a.coef), mdim, mstr, box, one,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        *merged = (merged_map(&m.coef_m1, 1) && merged_map(&m.coef_m2, 2)) ? 1 : 0;
    }
    if (a.seam) {
        if (a.Nx < W_IN) return false;
        const cuuint64_t half = cuuint64_t(W_IN / 2);
        const cuuint64_t hdim[5] = {8, half / 8, 2, Ny, 6};
        const cuuint64_t hstr[4] = {32, (Nx - half) * 4, Nx * 4, Nx * Ny * 4};
        auto seam_state = [&](CUtensorMap *map, cuuint32_t rows, cuuint32_t comps) {
            const cuuint32_t box[5] = {8, cuuint32_t(half / 8), 2, rows, comps};
            return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(a.q_in), hdim, hstr, box, one,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        if (!seam_state(&m.seam_state, 1, 1) || !seam_state(&m.seam_state_r1, cuuint32_t(R), 1) ||
            !seam_state(&m.seam_state_r2, cuuint32_t(R), 2) || !seam_state(&m.seam_state_r3, cuuint32_t(R), 3))
            return false;
        const cuuint64_t hcdim[5] = {16, half / 8, 2, Ny, cuuint64_t(NPAIR)};
        const cuuint64_t hcstr[4] = {64, (Nx - half) * 8, Nx * 8, Nx * Ny * 8};
        auto seam_coef = [&](CUtensorMap *map, cuuint32_t rows) {
            const cuuint32_t box[5] = {16, cuuint32_t(half / 8), 2, rows, 1};
            return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(a.coef), hcdim, hcstr, box, one,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        if (!seam_coef(&m.seam_coef, 1) || !seam_coef(&m.seam_coef_r, cuuint32_t(R))) return false;
    }
    return true;
}

template <typename T, int K, int R, int NY, bool INTER, bool UNIT>
int occupancy_t() {
    using Cfg = SweepCfg<T, K, R, NY>;
    using L = SweepLayout<T, K, R, INTER>;
    cudaFuncSetAttribute(sweep_kernel<T, K, R, NY, INTER, UNIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(L::SMEM));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, K, R, NY, INTER, UNIT>, Cfg::NT,
                                                      L::SMEM) != cudaSuccess)
        n = 1;
    cudaGetLastError();
    return n < 1 ? 1 : n;
}

template <typename T, int K, int R, int NY, bool INTER, bool UNIT>
cudaError_t launch_sweep_t(const SweepArgs &a, int nfam, cudaStream_t st) {
    using Cfg = SweepCfg<T, K, R, NY>;
    using L = SweepLayout<T, K, R, INTER>;
    static int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(sweep_kernel<T, K, R, NY, INTER, UNIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(L::SMEM));
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    SweepParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.a = a;
    // strips: the seam layout wherever the pass copies with TMA
    const bool try_tma = std::is_same<T, float>::value && a.error != nullptr;
    for (int z = 0; z < nfam; ++z) prm.split[z] = make_sweep_split(a.Nx, a.Ny, K, R, try_tma, a.fam0 + z, z, nfam);
    prm.a.seam = prm.split[0].seam;
    if constexpr (std::is_same<T, float>::value)
        prm.tma = (a.error != nullptr && make_sweep_maps(prm.a, K, R, prm.m, &prm.merged)) ? 1 : 0;
    if (!prm.tma && prm.a.seam) {  // no tensor maps: every strip copies with cp.async
        for (int z = 0; z < nfam; ++z) prm.split[z] = make_sweep_split(a.Nx, a.Ny, K, R, 0, a.fam0 + z, z, nfam);
        prm.a.seam = 0;
    }
    const int nsx = prm.split[0].nsx;
    if ((long long)nsx * a.Ny >= (1LL << 31)) return cudaErrorInvalidValue;
    if (a.chunk <= 0) {
        // balanced: a.ctas CTAs per family (one per resident slot), each one
        // equal share of its family's rows: no tail wave, and the warm-up
        // rows once per share and strip instead of once per tile
        if (a.ctas < 1) return cudaErrorInvalidValue;
        sweep_kernel<T, K, R, NY, INTER, UNIT><<<dim3(unsigned(a.ctas), 1, nfam), Cfg::NT, L::SMEM, st>>>(prm);
        return cudaGetLastError();
    }
    const int ncy = (a.Ny + a.chunk - 1) / a.chunk;
    // CTA order. One 224 KB CTA per SM (K = 4): the tiles of a strip in a row,
    // so that a tile's warm-up rows were just read by its neighbour above
    // (8192^2: 58.6 vs 55.0 G site-updates/s). Two CTAs per SM: the strips of
    // a tile row in a row (equal or better there). Families stay in separate
    // halves of the grid: two resident CTAs of different families (different
    // code) ran 13% slower.
    prm.tiles_fastest = K >= 4 ? 1 : 0;
    const dim3 grid = prm.tiles_fastest ? dim3(ncy, nsx, nfam) : dim3(nsx, ncy, nfam);
    sweep_kernel<T, K, R, NY, INTER, UNIT><<<grid, Cfg::NT, L::SMEM, st>>>(prm);
    return cudaGetLastError();
}

// Dispatch on the step order and the potential variant.
template <typename T, int K, int R, int NY>
cudaError_t launch_sweep_modes(const SweepArgs &a, int nfam, cudaStream_t st) {
    if (a.interleaved) {
        return a.unitary ? launch_sweep_t<T, K, R, NY, true, true>(a, nfam, st)
                         : launch_sweep_t<T, K, R, NY, true, false>(a, nfam, st);
    }
    return a.unitary ? launch_sweep_t<T, K, R, NY, false, true>(a, nfam, st)
                     : launch_sweep_t<T, K, R, NY, false, false>(a, nfam, st);
}

template <typename T, int K, int R, int NY>
int occupancy_modes(int interleaved) {
    return interleaved ? occupancy_t<T, K, R, NY, true, false>() : occupancy_t<T, K, R, NY, false, false>();
}

}  // namespace qla
