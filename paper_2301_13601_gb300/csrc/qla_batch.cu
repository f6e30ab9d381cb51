// Batched QLA: many independent lattices (of uneven sizes) advanced by one
// persistent kernel, replayed as a CUDA graph.
//
// Work items are (instance, pass, family, tile) with a tile one strip x chunk
// of one family (see qla_sweep.cuh). Items are numbered pass-major: every item
// of pass p precedes every item of pass p + 1, so a CTA that takes an item of
// pass p + 1 can rely on all items of pass p having been taken by running
// CTAs, which never wait on later passes: the queue cannot deadlock. Before
// starting an item of pass p > 0 a CTA waits until all tiles of pass p - 1 of
// the same (instance, family) are complete (a counter per pair, incremented
// after a fence). The wait is bounded by a time limit after which the kernel
// records QLA_ETIMEOUT, stops taking items and returns.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/qla.h"
#include "qla_sweep.cuh"

namespace qla {

struct BatchInst {
    void *q[2];
    const void *coef;
    int Nx, Ny, w_valid, chunk, nsx, ncy, tiles, passes, vec;
    int tma, merged;  // tensor maps encoded (see BatchMaps); merged-level coefficient map encoded
    int seam;         // the seam strip layout (SweepArgs::seam)
};

// TMA tensor maps of one instance (as SweepParams, for both state buffers),
// kept in device memory and read by the TMA unit from there.
struct BatchMaps {
    SweepMaps m[2];  // per state buffer holding the input
};

struct BatchSched {
    const BatchInst *inst;           // sorted by passes, descending
    const BatchMaps *maps;           // [ninst], same order
    int ninst;
    int maxpass;
    const long long *pass_start;     // [maxpass + 1]
    const int *active_count;         // [maxpass]: instances with passes > p (a prefix of inst)
    const long long *tile_prefix;    // [ninst + 1]: prefix sums of 2 * tiles
    unsigned long long *next;        // work counter
    unsigned int *done;              // [2 * ninst] completed tiles per (instance, family)
    int *cur;                        // [ninst] state buffer holding the input of pass 0
    int *error;                      // set to 1 on a wait timeout
    long long timeout_ns;
    unsigned int withhold;           // test hook: extra completions a dependency waits for (0 normally)
};

template <typename T, int K, int R, int NY, bool INTER, bool UNIT>
__global__ void __launch_bounds__(SweepCfg<T, K, R, NY>::NT, SweepCfg<T, K, R, NY>::MINB)
    batch_kernel(const BatchSched S) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // stop, instance, pass, family, strip, chunk: after the sweep's layout in
    // the dynamic allocation (a static array would shift the 1024-byte aligned
    // dynamic base by a whole kilobyte)
    using L = SweepLayout<T, K, R, INTER>;
    int *const sh = reinterpret_cast<int *>(smem_raw + L::SMEM);
    for (;;) {
        if (threadIdx.x == 0) {
            int stop = 0, inst = 0, pass = 0, fam = 0, tile = 0;
            const unsigned long long g = atomicAdd(S.next, 1ull);
            const unsigned long long total = (unsigned long long)S.pass_start[S.maxpass];
            if (g >= total || *(volatile int *)S.error) {
                stop = 1;
            } else {
                int lo = 0, hi = S.maxpass;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if ((unsigned long long)S.pass_start[mid] <= g) lo = mid;
                    else hi = mid;
                }
                pass = lo;
                const long long r = (long long)g - S.pass_start[pass];
                lo = 0;
                hi = S.active_count[pass];
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (S.tile_prefix[mid] <= r) lo = mid;
                    else hi = mid;
                }
                inst = lo;
                const int rr = int(r - S.tile_prefix[inst]);
                const int tiles = S.inst[inst].tiles;
                fam = rr / tiles;
                tile = rr % tiles;
                if (pass > 0) {
                    const unsigned int target = (unsigned int)pass * (unsigned int)tiles + S.withhold;
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire_u32(&S.done[2 * inst + fam]) < target) {
                        if (*(volatile int *)S.error) {  // another CTA gave up: stop as well
                            stop = 1;
                            break;
                        }
                        if ((long long)(global_ns() - t0) > S.timeout_ns) {
                            atomicExch(S.error, 1);
                            stop = 1;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
            }
            sh[0] = stop;
            sh[1] = inst;
            sh[2] = pass;
            sh[3] = fam;
            sh[4] = tile % S.inst[inst].nsx;
            sh[5] = tile / S.inst[inst].nsx;
        }
        __syncthreads();
        if (sh[0]) break;
        const int inst = sh[1], pass = sh[2], fam = sh[3], strip = sh[4], chunk = sh[5];
        const BatchInst &I = S.inst[inst];
        const int par = (S.cur[inst] + pass) & 1;
        SweepArgs a;
        a.q_in = I.q[par];
        a.q_out = I.q[par ^ 1];
        a.coef = I.coef;
        a.Nx = I.Nx;
        a.Ny = I.Ny;
        a.w_valid = I.w_valid;
        a.chunk = I.chunk;
        a.ctas = 0;
        a.seam = I.seam;
        a.interleaved = INTER ? 1 : 0;
        a.unitary = UNIT ? 1 : 0;
        a.vec = I.vec;
        a.fam0 = 0;
        a.error = S.error;  // a TMA wait that runs out stops the batch like a dependency timeout
        const BatchMaps *M = I.tma ? &S.maps[inst] : nullptr;
        // the input rows were written by other CTAs (generic proxy) and are
        // read here by TMA loads (async proxy)
        asm volatile("fence.proxy.async;\n" ::: "memory");
        const int yb = chunk * I.chunk, ye = min(yb + I.chunk, I.Ny);
        const bool failed =
            fam == 0 ? sweep_body<T, K, R, NY, INTER, UNIT, 0>(a, strip, yb, ye, smem_raw, M ? &M->m[par] : nullptr,
                                                               I.merged != 0)
                     : sweep_body<T, K, R, NY, INTER, UNIT, 1>(a, strip, yb, ye, smem_raw, M ? &M->m[par] : nullptr,
                                                               I.merged != 0);
        if (failed) break;  // the error flag is set: every CTA stops at its next work item
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&S.done[2 * inst + fam], 1u);
        }
    }
}

// After a run every instance has advanced `passes` passes: flip its parity.
__global__ void batch_flip(const BatchInst *inst, int *cur, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cur[i] ^= (inst[i].passes & 1);
}

constexpr int kBatchRows = 4;  // rows per iteration of the batch's sweep configurations (K = 2 and 4)

// dynamic shared memory of the batch kernel: the sweep's layout + 6 scheduler words
template <int K, int R, bool INTER>
constexpr size_t batch_smem() {
    return SweepLayout<float, K, R, INTER>::SMEM + 32;
}

// Sets the shared-memory attribute and returns the persistent grid size
// (SMs x resident CTAs); called before stream capture.
template <int K, int R, int NY, bool INTER, bool UNIT>
cudaError_t prepare_batch_t(int sms, int *grid) {
    using Cfg = SweepCfg<float, K, R, NY>;
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<float, K, R, NY, INTER, UNIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(batch_smem<K, R, INTER>()));
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel<float, K, R, NY, INTER, UNIT>, Cfg::NT,
                                                      batch_smem<K, R, INTER>());
    if (e != cudaSuccess) return e;
    *grid = sms * (occ < 1 ? 1 : occ);
    return cudaSuccess;
}

template <int K, int R, int NY, bool INTER, bool UNIT>
cudaError_t launch_batch_t(const BatchSched &S, int grid, cudaStream_t st) {
    using Cfg = SweepCfg<float, K, R, NY>;
    batch_kernel<float, K, R, NY, INTER, UNIT><<<grid, Cfg::NT, batch_smem<K, R, INTER>(), st>>>(S);
    return cudaGetLastError();
}

// mode dispatch: op(integral constants) for the four (interleaved, unitary) variants
template <int K, int R, int NY>
cudaError_t batch_modes(bool inter, bool unit, int sms, int *grid, const BatchSched *S, cudaStream_t st) {
    if (S == nullptr) {
        if (inter) return unit ? prepare_batch_t<K, R, NY, true, true>(sms, grid) : prepare_batch_t<K, R, NY, true, false>(sms, grid);
        return unit ? prepare_batch_t<K, R, NY, false, true>(sms, grid) : prepare_batch_t<K, R, NY, false, false>(sms, grid);
    }
    if (inter) return unit ? launch_batch_t<K, R, NY, true, true>(*S, *grid, st) : launch_batch_t<K, R, NY, true, false>(*S, *grid, st);
    return unit ? launch_batch_t<K, R, NY, false, true>(*S, *grid, st) : launch_batch_t<K, R, NY, false, false>(*S, *grid, st);
}

// S == nullptr: prepare (attribute + grid size); otherwise launch with *grid CTAs.
cudaError_t batch_dispatch(int K, bool inter, bool unit, int sms, int *grid, const BatchSched *S, cudaStream_t st) {
    switch (K) {
        case 2: return batch_modes<2, kBatchRows, 2>(inter, unit, sms, grid, S, st);
        case 4: return batch_modes<4, kBatchRows, 2>(inter, unit, sms, grid, S, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qla

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct qla_batch {
    int n = 0;
    int K = 4;
    int dev = 0;
    int sms = 152;
    bool inter = true, unit = false;
    cudaStream_t stream = nullptr;
    std::vector<qla::BatchInst> inst;  // sorted order
    std::vector<int> order;            // order[k] = user index of sorted instance k
    std::vector<int> slot;             // slot[user index] = sorted position
    std::vector<int> cur;              // host copy of the parities
    std::vector<void *> allocs;
    qla::BatchInst *d_inst = nullptr;
    qla::BatchMaps *d_maps = nullptr;
    long long *d_pass_start = nullptr;
    int *d_active = nullptr;
    long long *d_tile_prefix = nullptr;
    unsigned long long *d_next = nullptr;
    unsigned int *d_done = nullptr;
    int *d_cur = nullptr;
    int *d_error = nullptr;
    void *d_scratch = nullptr;
    qla::DiagResult *d_diag = nullptr;
    qla::DiagResult *h_diag = nullptr;
    int maxpass = 0;
    int grid = 0;
    long long total_items = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long timeout_ns = 4000000000LL;  // per dependency wait
    unsigned int withhold = 0;
    std::string msg;
};

namespace {

template <typename P>
cudaError_t dalloc(qla_batch *b, P **p, size_t bytes) {
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e == cudaSuccess) {
        b->allocs.push_back(v);
        *p = static_cast<P *>(v);
    }
    return e;
}

// Rows per tile in the batch. Measured on the 64-lattice workload (sides
// 256-2048, 4 steps per pass), site-updates/s: 512 rows 52.5 G, 768 and 1024
// rows 53.3 G, 2048 rows 50.1 G.
int auto_batch_chunk(int Ny) {
    int ch = std::min(Ny, 768);
    return std::max(1, ch);
}

}  // namespace

extern "C" {

qla_status qla_batch_create(int count, const qla_instance_desc *descs, const qla_options *opt, qla_batch **out) {
    if (!out || count < 1 || !descs) return QLA_EINVAL;
    *out = nullptr;
    qla_options o;
    qla_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != QLA_FP32 || o.families != QLA_FAMILIES_BOTH) return QLA_EUNSUPPORTED;
    const int K = o.steps_per_pass > 0 ? o.steps_per_pass : 4;
    if (K != 2 && K != 4) return QLA_EUNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        const qla_instance_desc &d = descs[i];
        if (d.Nx < 4 || d.Ny < 1 || d.Nx % 4 != 0 || (long long)d.Nx * d.Ny > 2147483647LL) return QLA_EINVAL;
        if (!d.n_x || !d.n_y || !d.n_z || !(d.delta > 0.0) || !(d.delta <= 0.5)) return QLA_EINVAL;
        if (d.nsteps < 0 || d.nsteps % K != 0) return QLA_EINVAL;
        const size_t P = size_t(d.Nx) * d.Ny;
        const double *nn[3] = {d.n_x, d.n_y, d.n_z};
        for (int k = 0; k < 3; ++k)
            for (size_t s = 0; s < P; ++s)
                if (!(nn[k][s] > 0.0) || !std::isfinite(nn[k][s])) return QLA_EINVAL;
    }
    qla_batch *b = new qla_batch();
    auto bail = [&](qla_status s) {
        qla_batch_destroy(b);
        return s;
    };
    b->n = count;
    b->K = K;
    b->inter = o.sequence == QLA_SEQ_INTERLEAVED;
    b->unit = o.potential == QLA_POT_UNITARY;
    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) return bail(QLA_ECUDA);
        b->dev = o.device;
    } else if (cudaGetDevice(&b->dev) != cudaSuccess) {
        return bail(QLA_ECUDA);
    }
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(QLA_ECUDA);

    // sort by number of passes, descending (active instances of a pass are a prefix)
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int a, int c) { return descs[a].nsteps > descs[c].nsteps; });
    b->slot.resize(count);
    for (int k = 0; k < count; ++k) b->slot[b->order[k]] = k;
    b->inst.resize(count);
    b->cur.assign(count, 0);
    const int W = qla::sweep_strip_width();
    size_t scratch_max = 0;
    for (int k = 0; k < count; ++k) {
        const qla_instance_desc &d = descs[b->order[k]];
        qla::BatchInst &I = b->inst[k];
        const size_t P = size_t(d.Nx) * d.Ny;
        I.Nx = d.Nx;
        I.Ny = d.Ny;
        I.w_valid = W - 8 * K;
        I.chunk = d.chunk_rows > 0 ? std::min(d.chunk_rows, d.Ny) : auto_batch_chunk(d.Ny);
        I.ncy = (d.Ny + I.chunk - 1) / I.chunk;
        I.passes = int(d.nsteps / K);
        I.vec = 1;
        float *q0, *q1, *coef;
        double *idx;
        if (dalloc(b, &q0, 6 * P * 4) != cudaSuccess || dalloc(b, &q1, 6 * P * 4) != cudaSuccess ||
            dalloc(b, &coef, size_t(qla::NCOEF) * P * 4) != cudaSuccess || dalloc(b, &idx, 3 * P * 8) != cudaSuccess) {
            cudaGetLastError();
            return bail(QLA_ENOMEM);
        }
        I.q[0] = q0;
        I.q[1] = q1;
        I.coef = coef;
        const double *nn[3] = {d.n_x, d.n_y, d.n_z};
        for (int c = 0; c < 3; ++c)
            if (cudaMemcpyAsync(idx + c * P, nn[c], P * 8, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
                return bail(QLA_ECUDA);
        if (qla::launch_coefficients(idx, coef, d.Nx, d.Ny, d.delta, 0, b->inter ? 1 : 0, b->unit ? 1 : 0, b->stream) !=
            cudaSuccess)
            return bail(QLA_ECUDA);
        if (cudaMemsetAsync(q0, 0, 6 * P * 4, b->stream) != cudaSuccess ||
            cudaMemsetAsync(q1, 0, 6 * P * 4, b->stream) != cudaSuccess)
            return bail(QLA_ECUDA);
        if (d.pulse_polarization == QLA_POL_EZ || d.pulse_polarization == QLA_POL_EY) {
            if (!(d.pulse_sigma > 0.0)) return bail(QLA_EINVAL);
            if (qla::launch_init_pulse(q0, d.Nx, d.Ny, 0, d.pulse_polarization, d.pulse_x0, d.pulse_sigma,
                                       d.pulse_amplitude, b->stream) != cudaSuccess)
                return bail(QLA_ECUDA);
        }
        scratch_max = std::max(scratch_max, qla::diag_scratch_bytes(d.Nx, d.Ny));
        // the index fields are only needed for the coefficients
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bail(QLA_ECUDA);
        cudaFree(idx);
        b->allocs.pop_back();
    }
    // TMA tensor maps of every instance (both state buffers) and its strips:
    // the seam layout where TMA applies (every strip copies with TMA); an
    // instance whose maps cannot be encoded copies with cp.async in the plain
    // layout
    std::vector<qla::BatchMaps> maps(count);
    for (int k = 0; k < count; ++k) {
        qla::BatchInst &I = b->inst[k];
        I.seam = qla::make_sweep_split(I.Nx, I.Ny, K, qla::kBatchRows, 1).seam;
        bool ok = true;
        for (int par = 0; par < 2 && ok; ++par) {
            qla::SweepArgs a;
            memset(&a, 0, sizeof(a));
            a.q_in = I.q[par];
            a.coef = I.coef;
            a.Nx = I.Nx;
            a.Ny = I.Ny;
            a.w_valid = I.w_valid;
            a.chunk = I.chunk;
            a.seam = I.seam;
            int merged = 0;
            memset(&maps[k].m[par], 0, sizeof(qla::SweepMaps));
            ok = qla::make_sweep_maps(a, K, qla::kBatchRows, maps[k].m[par], &merged);
            if (par == 0) I.merged = merged;
        }
        I.tma = ok ? 1 : 0;
        const qla::SweepSplit sp = qla::make_sweep_split(I.Nx, I.Ny, K, qla::kBatchRows, I.tma);
        I.seam = sp.seam;
        I.nsx = sp.nsx;
        I.tiles = I.nsx * I.ncy;
    }
    // schedule tables
    b->maxpass = b->inst[0].passes;
    std::vector<long long> tile_prefix(count + 1, 0);
    for (int k = 0; k < count; ++k) tile_prefix[k + 1] = tile_prefix[k] + 2LL * b->inst[k].tiles;
    std::vector<long long> pass_start(b->maxpass + 1, 0);
    std::vector<int> active(std::max(1, b->maxpass), 0);
    for (int p = 0; p < b->maxpass; ++p) {
        int a = 0;
        while (a < count && b->inst[a].passes > p) ++a;
        active[p] = a;
        pass_start[p + 1] = pass_start[p] + tile_prefix[a];
    }
    b->total_items = pass_start[b->maxpass];
    if (dalloc(b, &b->d_inst, sizeof(qla::BatchInst) * count) != cudaSuccess ||
        dalloc(b, &b->d_maps, sizeof(qla::BatchMaps) * count) != cudaSuccess ||
        dalloc(b, &b->d_pass_start, sizeof(long long) * (b->maxpass + 1)) != cudaSuccess ||
        dalloc(b, &b->d_active, sizeof(int) * active.size()) != cudaSuccess ||
        dalloc(b, &b->d_tile_prefix, sizeof(long long) * (count + 1)) != cudaSuccess ||
        dalloc(b, &b->d_next, 64) != cudaSuccess || dalloc(b, &b->d_done, sizeof(unsigned) * 2 * count) != cudaSuccess ||
        dalloc(b, &b->d_cur, sizeof(int) * count) != cudaSuccess || dalloc(b, &b->d_error, 64) != cudaSuccess ||
        dalloc(b, &b->d_scratch, scratch_max + 512) != cudaSuccess)
        return bail(QLA_ENOMEM);
    b->d_diag = reinterpret_cast<qla::DiagResult *>(static_cast<char *>(b->d_scratch) + ((scratch_max + 255) / 256) * 256);
    if (cudaMallocHost(reinterpret_cast<void **>(&b->h_diag), sizeof(qla::DiagResult)) != cudaSuccess)
        return bail(QLA_ENOMEM);
    if (cudaMemcpy(b->d_inst, b->inst.data(), sizeof(qla::BatchInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_maps, maps.data(), sizeof(qla::BatchMaps) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_pass_start, pass_start.data(), sizeof(long long) * pass_start.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_active, active.data(), sizeof(int) * active.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tile_prefix, tile_prefix.data(), sizeof(long long) * tile_prefix.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_cur, 0, sizeof(int) * count) != cudaSuccess)
        return bail(QLA_ECUDA);
    if (qla::batch_dispatch(b->K, b->inter, b->unit, b->sms, &b->grid, nullptr, nullptr) != cudaSuccess)
        return bail(QLA_ECUDA);
    *out = b;
    return QLA_OK;
}

qla_status qla_batch_run(qla_batch *b) {
    if (!b) return QLA_EINVAL;
    if (cudaSetDevice(b->dev) != cudaSuccess) return QLA_ECUDA;
    if (!b->exec) {
        qla::BatchSched S;
        S.inst = b->d_inst;
        S.maps = b->d_maps;
        S.ninst = b->n;
        S.maxpass = b->maxpass;
        S.pass_start = b->d_pass_start;
        S.active_count = b->d_active;
        S.tile_prefix = b->d_tile_prefix;
        S.next = b->d_next;
        S.done = b->d_done;
        S.cur = b->d_cur;
        S.error = b->d_error;
        S.timeout_ns = b->timeout_ns;
        S.withhold = b->withhold;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return QLA_ECUDA;
        cudaError_t e = cudaMemsetAsync(b->d_next, 0, 64, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * 2 * b->n, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_error, 0, 64, b->stream);
        if (e == cudaSuccess && b->maxpass > 0)
            e = qla::batch_dispatch(b->K, b->inter, b->unit, b->sms, &b->grid, &S, b->stream);
        if (e == cudaSuccess) {
            qla::batch_flip<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_inst, b->d_cur, b->n);
            e = cudaGetLastError();
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->msg = std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
            return QLA_ECUDA;
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            b->msg = "graph instantiation failed";
            return QLA_ECUDA;
        }
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return QLA_ECUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, b->d_error, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return QLA_ECUDA;
    for (int k = 0; k < b->n; ++k) b->cur[k] ^= (b->inst[k].passes & 1);
    if (err) {
        b->msg = "a dependency wait or a TMA copy wait timed out";
        return QLA_ETIMEOUT;
    }
    return QLA_OK;
}

qla_status qla_batch_get_fields_f32(qla_batch *b, int i, float *q) {
    if (!b || i < 0 || i >= b->n || !q) return QLA_EINVAL;
    if (cudaSetDevice(b->dev) != cudaSuccess) return QLA_ECUDA;
    const int k = b->slot[i];
    const qla::BatchInst &I = b->inst[k];
    const size_t P = size_t(I.Nx) * I.Ny;
    if (cudaMemcpyAsync(q, I.q[b->cur[k]], 6 * P * 4, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return QLA_ECUDA;
    return QLA_OK;
}

qla_status qla_batch_diagnostics(qla_batch *b, int i, qla_diag *out) {
    if (!b || i < 0 || i >= b->n || !out) return QLA_EINVAL;
    if (cudaSetDevice(b->dev) != cudaSuccess) return QLA_ECUDA;
    const int k = b->slot[i];
    const qla::BatchInst &I = b->inst[k];
    if (qla::launch_diagnostics(I.q[b->cur[k]], 0, I.Nx, I.Ny, b->d_scratch, b->d_diag, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->h_diag, b->d_diag, sizeof(qla::DiagResult), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return QLA_ECUDA;
    out->energy = b->h_diag->energy_sum / (double(I.Nx) * I.Ny);
    out->div_l2_sq = b->h_diag->div_sq_sum;
    out->div_max = b->h_diag->div_max;
    out->b_max = b->h_diag->b_max;
    out->nonfinite = (long long)b->h_diag->nonfinite;
    return out->nonfinite ? QLA_ENONFINITE : QLA_OK;
}

qla_status qla_batch_info(const qla_batch *b, long long *total_items, int *steps_per_pass, long long *site_updates) {
    if (!b) return QLA_EINVAL;
    if (total_items) *total_items = b->total_items;
    if (steps_per_pass) *steps_per_pass = b->K;
    if (site_updates) {
        long long s = 0;
        for (const auto &I : b->inst) s += (long long)I.Nx * I.Ny * I.passes * b->K;
        *site_updates = s;
    }
    return QLA_OK;
}

qla_status qla_batch_set_wait_limit(qla_batch *b, long long timeout_ns, int withhold) {
    if (!b || timeout_ns <= 0 || withhold < 0) return QLA_EINVAL;
    b->timeout_ns = timeout_ns;
    b->withhold = (unsigned int)withhold;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    return QLA_OK;
}

const char *qla_batch_last_error(const qla_batch *b) { return b ? b->msg.c_str() : "NULL batch"; }

void qla_batch_destroy(qla_batch *b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *p : b->allocs) cudaFree(p);
    if (b->h_diag) cudaFreeHost(b->h_diag);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
