// Single operators of one QLA step on the context's state (qla_debug_apply):
// the collisions C_X, C_Y (Eq. 17, Eq. 19) and their transposes, the eight
// one-cell streaming shifts of Eq. 18 and Eq. 20, and the potentials V_X, V_Y
// (Eq. 21-22). They evaluate each operator with the same per-site arithmetic
// and coefficient pairs as the fused sweep (rot, vop_pair in qla_sweep.cuh),
// one thread per site, so that each factor of the step can be compared on its
// own with a reference of that operator.
#include "../../include/qla.h"
#include "qla_sweep.cuh"

namespace qla {
namespace {

constexpr int DBG_THREADS = 256;

template <bool DAG, int SG, bool SHR, typename T>
__device__ __forceinline__ void rot_pair(T *q, const typename Ar<T>::T2 *cp, long long P, long long i, int hub,
                                         int partner, int plane) {
    const typename Ar<T>::T2 c = cp[plane * P + i];
    T h = q[hub * P + i], p = q[partner * P + i];
    rot<DAG, SG, SHR>(h, p, c.x, c.y);
    q[hub * P + i] = h;
    q[partner * P + i] = p;
}

// C_X (axis 0) or C_Y (axis 1) on both families, or their transposes.
template <int AXIS, bool DAG, bool SHR, typename T>
__global__ void __launch_bounds__(DBG_THREADS) collide_kernel(T *q, const typename Ar<T>::T2 *cp, long long P) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        if (AXIS == 0) {
            rot_pair<DAG, Fam<0>::SGX, SHR>(q, cp, P, i, Fam<0>::H, Fam<0>::PX, Fam<0>::CX);
            rot_pair<DAG, Fam<1>::SGX, SHR>(q, cp, P, i, Fam<1>::H, Fam<1>::PX, Fam<1>::CX);
        } else {
            rot_pair<DAG, Fam<0>::SGY, SHR>(q, cp, P, i, Fam<0>::H, Fam<0>::PY, Fam<0>::CY);
            rot_pair<DAG, Fam<1>::SGY, SHR>(q, cp, P, i, Fam<1>::H, Fam<1>::PY, Fam<1>::CY);
        }
    }
}

template <int TAU, bool HUB, bool UNIT, typename T>
__device__ __forceinline__ void pot_pair(T *q, const typename Ar<T>::T2 *cp, long long P, long long i, int hub,
                                         int partner, int plane) {
    const typename Ar<T>::T2 c = cp[plane * P + i];  // (cos b - 1, sin b)
    T h = q[hub * P + i], p = q[partner * P + i];
    vop_pair<TAU, HUB, UNIT>(h, p, c.y, c.x);
    q[hub * P + i] = h;
    q[partner * P + i] = p;
}

// V_X (axis 0) or V_Y (axis 1) on both families, as one application in the
// context's step (its pair planes hold that application's angles).
template <int AXIS, bool UNIT, typename T>
__global__ void __launch_bounds__(DBG_THREADS) potential_kernel(T *q, const typename Ar<T>::T2 *cp, long long P) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        if (AXIS == 0) {
            pot_pair<Fam<0>::TX, Fam<0>::VX_HUB, UNIT>(q, cp, P, i, Fam<0>::H, Fam<0>::PX, Fam<0>::VX);
            pot_pair<Fam<1>::TX, Fam<1>::VX_HUB, UNIT>(q, cp, P, i, Fam<1>::H, Fam<1>::PX, Fam<1>::VX);
        } else {
            pot_pair<Fam<0>::TY, Fam<0>::VY_HUB, UNIT>(q, cp, P, i, Fam<0>::H, Fam<0>::PY, Fam<0>::VY);
            pot_pair<Fam<1>::TY, Fam<1>::VY_HUB, UNIT>(q, cp, P, i, Fam<1>::H, Fam<1>::PY, Fam<1>::VY);
        }
    }
}

// Streaming: components ca and cb move by one cell along the axis
// (dir = +1: q(r) <- q(r + e); dir = -1: q(r) <- q(r - e), periodic); the
// other four are copied unchanged. Out of place.
template <typename T>
__global__ void __launch_bounds__(DBG_THREADS) stream_kernel(const T *__restrict__ in, T *__restrict__ out, int Nx,
                                                             int Ny, int ca, int cb, int axis, int dir) {
    const long long P = (long long)Nx * Ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 6 * P;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i / P);
        const long long s = i - c * P;
        int y = int(s / Nx), x = int(s - (long long)y * Nx);
        if (c == ca || c == cb) {
            if (axis == 0) x = x + dir < 0 ? Nx - 1 : (x + dir >= Nx ? 0 : x + dir);
            else y = y + dir < 0 ? Ny - 1 : (y + dir >= Ny ? 0 : y + dir);
        }
        out[i] = in[c * P + (long long)y * Nx + x];
    }
}

template <typename T>
cudaError_t apply_t(int op, void *state, void *spare, const void *coef, int Nx, int Ny, int unitary, cudaStream_t st,
                    bool *swapped) {
    using T2 = typename Ar<T>::T2;
    T *q = static_cast<T *>(state);
    const T2 *cp = static_cast<const T2 *>(coef);
    const long long P = (long long)Nx * Ny;
    const int blocks = int(std::min<long long>((P + DBG_THREADS - 1) / DBG_THREADS, 152LL * 16));
    *swapped = false;
    switch (op) {
        case QLA_OP_CX:
        case QLA_OP_CX_T:
        case QLA_OP_CY:
        case QLA_OP_CY_T: {
            // the collision form of the context's configuration (see rot)
            const bool shear = shear_collisions<T, false>() && !unitary;
            const int k = (op == QLA_OP_CX ? 0 : op == QLA_OP_CX_T ? 1 : op == QLA_OP_CY ? 2 : 3) + (shear ? 4 : 0);
            switch (k) {
                case 0: collide_kernel<0, false, false><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                case 1: collide_kernel<0, true, false><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                case 2: collide_kernel<1, false, false><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                case 3: collide_kernel<1, true, false><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                case 4: collide_kernel<0, false, true><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                case 5: collide_kernel<0, true, true><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                case 6: collide_kernel<1, false, true><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
                default: collide_kernel<1, true, true><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P); break;
            }
            break;
        }
        case QLA_OP_VX:
            if (unitary) potential_kernel<0, true><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P);
            else potential_kernel<0, false><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P);
            break;
        case QLA_OP_VY:
            if (unitary) potential_kernel<1, true><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P);
            else potential_kernel<1, false><<<blocks, DBG_THREADS, 0, st>>>(q, cp, P);
            break;
        default: {
            // streaming ops QLA_OP_S14_XP .. QLA_OP_S25_YM: (components, axis, direction)
            static const int table[8][4] = {{1, 4, 0, +1}, {1, 4, 0, -1}, {2, 5, 0, +1}, {2, 5, 0, -1},
                                            {0, 3, 1, +1}, {0, 3, 1, -1}, {2, 5, 1, +1}, {2, 5, 1, -1}};
            const int *t = table[op - QLA_OP_S14_XP];
            const int sb = int(std::min<long long>((6 * P + DBG_THREADS - 1) / DBG_THREADS, 152LL * 16));
            stream_kernel<T><<<sb, DBG_THREADS, 0, st>>>(q, static_cast<T *>(spare), Nx, Ny, t[0], t[1], t[2], t[3]);
            *swapped = true;
        }
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t debug_apply(int op, int precision, void *state, void *spare, const void *coef, int Nx, int Ny, int unitary,
                        cudaStream_t st, bool *swapped) {
    return precision == QLA_FP64 ? apply_t<double>(op, state, spare, coef, Nx, Ny, unitary, st, swapped)
                                 : apply_t<float>(op, state, spare, coef, Nx, Ny, unitary, st, swapped);
}

}  // namespace qla
