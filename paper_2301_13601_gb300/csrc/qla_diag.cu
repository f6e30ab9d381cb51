// Diagnostics reduction: energy (Eq. 27), div B statistics and a non-finite
// count in one pass over the state, reduced in FP64 with Neumaier-compensated
// sums in a fixed order (the result depends only on the lattice size, not on
// scheduling).
//
// Pass 1 (diag_partial): block b takes rows b, b + G, b + 2G, ...; every
// thread keeps compensated sums of its per-row sums; the block combines its
// threads in a fixed tree and writes one partial record to scratch.
// Pass 2 (diag_final): one block combines the G partials in a fixed tree.
#include <math.h>

#include "qla_internal.h"

namespace qla {

namespace {

constexpr int DIAG_THREADS = 256;

struct CSum {
    double s, c;
    __device__ __forceinline__ void add(double v) {
        const double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ void merge(const CSum &o) {
        add(o.s);
        c += o.c;
    }
};

struct Partial {
    double e_s, e_c, d_s, d_c, dmax, bmax;
    unsigned long long nonfinite;
    unsigned long long pad;
};

template <typename T>
__device__ __forceinline__ bool finite_val(T v) {
    return isfinite(v);
}

__device__ __forceinline__ void merge_into(Partial &a, const Partial &b) {
    CSum es{a.e_s, a.e_c}, ds{a.d_s, a.d_c};
    es.merge(CSum{b.e_s, b.e_c});
    ds.merge(CSum{b.d_s, b.d_c});
    a.e_s = es.s; a.e_c = es.c; a.d_s = ds.s; a.d_c = ds.c;
    a.dmax = fmax(a.dmax, b.dmax);
    a.bmax = fmax(a.bmax, b.bmax);
    a.nonfinite += b.nonfinite;
}

// The block's threads combined in a fixed tree; thread 0 writes the record.
__device__ __forceinline__ void block_reduce_write(const Partial &mine, Partial *__restrict__ part) {
    __shared__ Partial sh[DIAG_THREADS];
    sh[threadIdx.x] = mine;
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            Partial a = sh[threadIdx.x];
            merge_into(a, sh[threadIdx.x + w]);
            sh[threadIdx.x] = a;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) diag_partial(const T *__restrict__ q, int Nx, int Ny,
                                                             Partial *__restrict__ part) {
    const size_t P = size_t(Nx) * size_t(Ny);
    const T *q3 = q + 3 * P, *q4 = q + 4 * P;
    CSum e{0.0, 0.0}, d{0.0, 0.0};
    double dmax = 0.0, b2max = 0.0;
    unsigned long long nf = 0;
    for (int y = blockIdx.x; y < Ny; y += gridDim.x) {
        const int yp = y + 1 == Ny ? 0 : y + 1, ym = y == 0 ? Ny - 1 : y - 1;
        const size_t r = size_t(y) * Nx;
        // A thread's sites of one row (at most ceil(Nx / DIAG_THREADS) terms of
        // equal sign) are summed plainly in FP64; the row sums enter the
        // compensated sums. The FP64 pipe is the bound of this kernel, so
        // per-site work is kept to the squares and one add per sum.
        double erow = 0.0, drow = 0.0;
        for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
            const size_t i = r + x;
            double sq[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const T v = q[size_t(c) * P + i];
                if (!finite_val(v)) ++nf;
                const double dv = double(v);
                sq[c] = dv * dv;
            }
            const double b2 = sq[3] + sq[4] + sq[5];
            erow += (sq[0] + sq[1] + sq[2]) + b2;
            b2max = fmax(b2max, b2);
            const int xp = x + 1 == Nx ? 0 : x + 1, xm = x == 0 ? Nx - 1 : x - 1;
            const double dv = 0.5 * (double(q3[r + xp]) - double(q3[r + xm])) +
                              0.5 * (double(q4[size_t(yp) * Nx + x]) - double(q4[size_t(ym) * Nx + x]));
            drow = fma(dv, dv, drow);
            dmax = fmax(dmax, fabs(dv));
        }
        e.add(erow);
        d.add(drow);
    }
    const double bmax = sqrt(b2max);  // sqrt is monotonic: the max of the site norms
    block_reduce_write(Partial{e.s, e.c, d.s, d.c, dmax, bmax, nf, 0ull}, part);
}

// Exact FP32 -> FP64 conversion on the integer pipe (this kernel is bound by
// GB300's FP64 pipe, which also executes the hardware conversion): zero and
// normal values by rebiasing the exponent and widening the mantissa; subnormal,
// infinite and NaN values take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned e = (u >> 23) & 0xffu;
    const bool zero = (u << 1) == 0u;
    if (zero || e - 1u < 254u) {
        const unsigned mag = zero ? 0u : (((e + 896u) << 20) | ((u >> 3) & 0xfffffu));
        return __hiloint2double(int((u & 0x80000000u) | mag), zero ? 0 : int(u << 29));
    }
    return double(v);
}

// FP32 state: the same sums and maxima as the generic kernel below, with the
// FP64 pipe doing only what needs FP64: a site's squares are summed as an
// exact-product float pair and enter the FP64 row sum by two additions (sites
// with values beyond 2^+-60, where FP32 squares could overflow or lose their
// error term, take FP64 squares instead), the divergence is formed in FP64
// as (q3(x+1) - q3(x-1)) + (q4(y+1) - q4(y-1)) with the factors 1/2 and 1/4
// applied to the reduced max and sum (exact scalings), and the site norms |B|^2
// are screened in FP32: a site's FP64 norm is computed only when its FP32 norm
// (relative error below 2^-22) reaches the running maximum lowered by 2^-20,
// so no site whose FP64 norm exceeds the maximum is skipped. max |div| is kept
// as the bit pattern of a non-negative double (integer order = numeric order;
// NaN excluded, as fmax would).
__global__ void __launch_bounds__(DIAG_THREADS) diag_partial_f32(const float *__restrict__ q, int Nx, int Ny,
                                                                 Partial *__restrict__ part) {
    const size_t P = size_t(Nx) * size_t(Ny);
    const float *q3 = q + 3 * P, *q4 = q + 4 * P;
    CSum e{0.0, 0.0}, d{0.0, 0.0};
    unsigned long long dmax_bits = 0;
    double b2max = 0.0;
    float b2thr = 0.0f;
    unsigned long long nf = 0;
    for (int y = blockIdx.x; y < Ny; y += gridDim.x) {
        const int yp = y + 1 == Ny ? 0 : y + 1, ym = y == 0 ? Ny - 1 : y - 1;
        const size_t r = size_t(y) * Nx;
        double erow = 0.0, drow = 0.0;
        for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
            const size_t i = r + x;
            float v[6];
            bool ff = true;  // every |v| zero or in [2^-60, 2^60): FP32 squares and their errors are exact
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                v[c] = q[size_t(c) * P + i];
                if (!isfinite(v[c])) ++nf;
                const unsigned ua = __float_as_uint(v[c]) & 0x7fffffffu;
                ff = ff && (ua == 0u || ua - 0x21800000u < 0x3c000000u);
            }
            if (ff) {
                // the site's sum of squares as an unevaluated float pair: each
                // square is p + e exactly (e by FMA), the p are added by TwoSum,
                // the low parts in FP32 (relative error ~2^-47 of the site value,
                // unbiased); two FP64 additions enter it into the row sum
                // (intrinsics: no contraction of a product into the TwoSum)
                float hi = __fmul_rn(v[0], v[0]), lo = __fmaf_rn(v[0], v[0], -hi);
#pragma unroll
                for (int c = 1; c < 6; ++c) {
                    const float pc = __fmul_rn(v[c], v[c]);
                    const float ec = __fmaf_rn(v[c], v[c], -pc);
                    const float sc = __fadd_rn(hi, pc);
                    const float bb = __fsub_rn(sc, hi);
                    const float tc = __fadd_rn(__fsub_rn(hi, __fsub_rn(sc, bb)), __fsub_rn(pc, bb));
                    lo = __fadd_rn(lo, __fadd_rn(tc, ec));
                    hi = sc;
                }
                erow = (erow + f2d_exact(hi)) + f2d_exact(lo);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const double dv = f2d_exact(v[c]);
                    erow = fma(dv, dv, erow);
                }
            }
            const float b2f = fmaf(v[3], v[3], fmaf(v[4], v[4], v[5] * v[5]));
            if (!(b2f < b2thr)) {  // candidate for the maximum (also when b2f is inf or NaN)
                const double d3 = f2d_exact(v[3]), d4 = f2d_exact(v[4]), d5 = f2d_exact(v[5]);
                const double b2 = (d3 * d3 + d4 * d4) + d5 * d5;
                if (b2 > b2max) {
                    b2max = b2;
                    b2thr = __double2float_rd(b2 * (1.0 - 0x1p-20));
                }
            }
            const int xp = x + 1 == Nx ? 0 : x + 1, xm = x == 0 ? Nx - 1 : x - 1;
            const double dv = (f2d_exact(q3[r + xp]) - f2d_exact(q3[r + xm])) +
                              (f2d_exact(q4[size_t(yp) * Nx + x]) - f2d_exact(q4[size_t(ym) * Nx + x]));
            drow = fma(dv, dv, drow);
            const unsigned long long ab = static_cast<unsigned long long>(__double_as_longlong(dv)) &
                                          0x7fffffffffffffffull;
            if (ab <= 0x7ff0000000000000ull && ab > dmax_bits) dmax_bits = ab;
        }
        e.add(erow);
        d.add(0.25 * drow);
    }
    const double dmax = 0.5 * __longlong_as_double(static_cast<long long>(dmax_bits));
    block_reduce_write(Partial{e.s, e.c, d.s, d.c, dmax, sqrt(b2max), nf, 0ull}, part);
}

// Divergence of D (Sec. 4.2): D = (n_x q0, n_y q1, n_z q2) for the diagonal
// dielectric eps_i = n_i^2 (Eq. 15: q_i = n_i E_i), central differences in
// lattice units; the same partition and trees as diag_partial. The record's
// div fields hold sum div^2 and max |div|, its B field max |D|; the energy
// fields are zero.
template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) divD_partial(const T *__restrict__ q, const double *__restrict__ idx,
                                                             int Nx, int Ny, Partial *__restrict__ part) {
    const size_t P = size_t(Nx) * size_t(Ny);
    const T *q0 = q, *q1 = q + P, *q2 = q + 2 * P;
    const double *nx = idx, *ny = idx + P, *nz = idx + 2 * P;
    CSum d{0.0, 0.0};
    double dmax = 0.0, d2max = 0.0;
    unsigned long long nf = 0;
    for (int y = blockIdx.x; y < Ny; y += gridDim.x) {
        const int yp = y + 1 == Ny ? 0 : y + 1, ym = y == 0 ? Ny - 1 : y - 1;
        const size_t r = size_t(y) * Nx;
        double drow = 0.0;
        for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
            const size_t i = r + x;
            const int xp = x + 1 == Nx ? 0 : x + 1, xm = x == 0 ? Nx - 1 : x - 1;
            const size_t ixp = r + xp, ixm = r + xm, iyp = size_t(yp) * Nx + x, iym = size_t(ym) * Nx + x;
            const double dv = 0.5 * (nx[ixp] * double(q0[ixp]) - nx[ixm] * double(q0[ixm])) +
                              0.5 * (ny[iyp] * double(q1[iyp]) - ny[iym] * double(q1[iym]));
            drow = fma(dv, dv, drow);
            dmax = fmax(dmax, fabs(dv));
            const double dx = nx[i] * double(q0[i]), dy = ny[i] * double(q1[i]), dz = nz[i] * double(q2[i]);
            d2max = fmax(d2max, dx * dx + dy * dy + dz * dz);
            if (!finite_val(q0[i]) || !finite_val(q1[i]) || !finite_val(q2[i])) ++nf;
        }
        d.add(drow);
    }
    block_reduce_write(Partial{0.0, 0.0, d.s, d.c, dmax, sqrt(d2max), nf, 0ull}, part);
}

__global__ void __launch_bounds__(DIAG_THREADS) diag_final(const Partial *__restrict__ part, int n,
                                                           DiagResult *__restrict__ out) {
    CSum e{0.0, 0.0}, d{0.0, 0.0};
    double dmax = 0.0, bmax = 0.0;
    unsigned long long nf = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Partial p = part[i];
        e.merge(CSum{p.e_s, p.e_c});
        d.merge(CSum{p.d_s, p.d_c});
        dmax = fmax(dmax, p.dmax);
        bmax = fmax(bmax, p.bmax);
        nf += p.nonfinite;
    }
    __shared__ Partial sh[DIAG_THREADS];
    sh[threadIdx.x] = Partial{e.s, e.c, d.s, d.c, dmax, bmax, nf, 0ull};
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            Partial a = sh[threadIdx.x];
            const Partial b = sh[threadIdx.x + w];
            CSum es{a.e_s, a.e_c}, ds{a.d_s, a.d_c};
            es.merge(CSum{b.e_s, b.e_c});
            ds.merge(CSum{b.d_s, b.d_c});
            a.e_s = es.s; a.e_c = es.c; a.d_s = ds.s; a.d_c = ds.c;
            a.dmax = fmax(a.dmax, b.dmax);
            a.bmax = fmax(a.bmax, b.bmax);
            a.nonfinite += b.nonfinite;
            sh[threadIdx.x] = a;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const Partial a = sh[0];
        out->energy_sum = a.e_s + a.e_c;
        out->div_sq_sum = a.d_s + a.d_c;
        out->div_max = a.dmax;
        out->b_max = a.bmax;
        out->nonfinite = a.nonfinite;
    }
}

}  // namespace

int diag_blocks(int Nx, int Ny) {
    (void)Nx;
    return Ny < 4 * 152 ? Ny : 4 * 152;
}

size_t diag_scratch_bytes(int Nx, int Ny) {
    return size_t(diag_blocks(Nx, Ny)) * sizeof(Partial) + 256;
}

cudaError_t launch_diagnostics(const void *q, int precision, int Nx, int Ny, void *scratch, DiagResult *out_dev,
                               cudaStream_t st) {
    const int G = diag_blocks(Nx, Ny);
    Partial *part = static_cast<Partial *>(scratch);
    if (precision == 0)
        diag_partial_f32<<<G, DIAG_THREADS, 0, st>>>(static_cast<const float *>(q), Nx, Ny, part);
    else
        diag_partial<double><<<G, DIAG_THREADS, 0, st>>>(static_cast<const double *>(q), Nx, Ny, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, DIAG_THREADS, 0, st>>>(part, G, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_divD(const void *q, int precision, const double *index, int Nx, int Ny, void *scratch,
                        DiagResult *out_dev, cudaStream_t st) {
    const int G = diag_blocks(Nx, Ny);
    Partial *part = static_cast<Partial *>(scratch);
    if (precision == 0)
        divD_partial<float><<<G, DIAG_THREADS, 0, st>>>(static_cast<const float *>(q), index, Nx, Ny, part);
    else
        divD_partial<double><<<G, DIAG_THREADS, 0, st>>>(static_cast<const double *>(q), index, Nx, Ny, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, DIAG_THREADS, 0, st>>>(part, G, out_dev);
    return cudaGetLastError();
}

}  // namespace qla

// ---------------------------------------------------------------------------
// Allocation-free diagnostics (qla_diagnostics_noalloc in include/qla.h).
//
// Some callers cannot allocate device memory at the point where they need
// the diagnostics: an application that hands all of the GPU's memory to its
// own allocator up front (a framework's caching pool, a fixed budget per job)
// and forbids cudaMalloc afterwards, or a monitoring loop that must not block
// on the allocator or fail with out-of-memory halfway through a long run. This variant
// runs the same two reduction kernels as the context-based diagnostics, but
// keeps their scratch (the per-block partial records and the final result) in
// the file-scope device array below instead of memory from cudaMalloc.
//
// The array is reserved in every GPU that loads the library, for the life of
// the process. All calls share it and it keeps the previous call's contents:
// every record a call reads is written earlier in the same call, so nothing
// has to be cleared, but two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it.
// ---------------------------------------------------------------------------
#include <limits.h>

#include "../../include/qla.h"

namespace qla {
namespace {

constexpr int NOALLOC_ROWS_PER_BLOCK = 4;
constexpr int NOALLOC_MAX_PARTIALS = 4096;  // lattices of at most 4096 * 4 = 16384 rows
struct NoallocScratch {
    Partial part[NOALLOC_MAX_PARTIALS];
    DiagResult result;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of the array on the current device. In host code the
// symbol g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up on every call: a cached address would go stale after a device
// reset or a re-created primary context, when the module reloads elsewhere.
// The first call on a device may load the module: make it before any stream
// capture.
cudaError_t noalloc_scratch(NoallocScratch **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<NoallocScratch *>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace qla

extern "C" qla_status qla_diagnostics_noalloc(const void *q, int precision, int Nx, int Ny, void *stream,
                                              qla_diag *out) {
    using namespace qla;
    if (!q || !out || Nx < 1 || Ny < 1 || (long long)Nx * (long long)Ny > INT_MAX ||
        (precision != QLA_FP32 && precision != QLA_FP64))
        return QLA_EINVAL;
    const int G = (Ny + NOALLOC_ROWS_PER_BLOCK - 1) / NOALLOC_ROWS_PER_BLOCK;
    if (G > NOALLOC_MAX_PARTIALS) return QLA_EINVAL;  // Ny above 16384: the static scratch is too small
    NoallocScratch *s = nullptr;
    if (noalloc_scratch(&s) != cudaSuccess) {
        cudaGetLastError();
        return QLA_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == QLA_FP32)
        diag_partial_f32<<<G, DIAG_THREADS, 0, st>>>(static_cast<const float *>(q), Nx, Ny, s->part);
    else
        diag_partial<double><<<G, DIAG_THREADS, 0, st>>>(static_cast<const double *>(q), Nx, Ny, s->part);
    if (cudaGetLastError() != cudaSuccess) return QLA_ECUDA;
    diag_final<<<1, DIAG_THREADS, 0, st>>>(s->part, G, &s->result);
    if (cudaGetLastError() != cudaSuccess) return QLA_ECUDA;
    DiagResult r;
    if (cudaMemcpyAsync(&r, &s->result, sizeof(r), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return QLA_ECUDA;
    }
    out->energy = r.energy_sum / (double(Nx) * double(Ny));
    out->div_l2_sq = r.div_sq_sum;
    out->div_max = r.div_max;
    out->b_max = r.b_max;
    out->nonfinite = (long long)r.nonfinite;
    return r.nonfinite ? QLA_ENONFINITE : QLA_OK;
}
