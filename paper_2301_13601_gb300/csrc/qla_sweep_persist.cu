// Persistent form of the balanced FP32 sweep: every full pass of one
// qla_step call in one cooperative launch.
//
// In the per-pass form every pass of K fused steps (Eq. 28 / Eq. 23) ends at a
// kernel boundary, where each CTA waits for the slowest CTA of the pass and
// then for the next launch to start. Here CTA b keeps share b of each
// advanced family for all the passes of the launch, one family after the
// other. Before pass p >= 1 of a family it waits only for the shares of that
// family whose pass p - 1 wrote cells that share b reads, or read cells that
// share b overwrites: its halo neighbours along its strip and in the strips
// beside it (SweepSplit::shares_touch). Each CTA publishes its progress in a per-share
// pass counter (release store at GPU scope after its pass; the waiting CTA
// reads it with acquire loads). A cooperative launch guarantees that all CTAs
// (one per resident slot) run at once, so every wait ends; each is also bounded
// in time (2 s, global timer), after which the CTA sets the error flag and
// stops, and the other CTAs stop at their next wait.
//
// The arithmetic of a pass is the per-pass kernel's (the same sweep_body), so
// both forms give bit-identical states.
#include "qla_sweep.cuh"

namespace qla {

struct SweepPersistParams {
    SweepParams s;     // the pass's arguments, splits and the maps of the even passes (input s.a.q_in)
    SweepMaps m_odd;   // tensor maps of the odd passes (input and output buffers swapped)
    int passes;        // passes of K steps in this launch
    int nfam;          // family layers advanced: the CTA sweeps share blockIdx.x of each
    unsigned base;     // pass counters reached by the earlier launches on these counters
    unsigned *done;    // [nfam][gridDim.x] passes each share has completed (monotonic across launches)
    unsigned withhold;           // test hook: extra passes every wait demands (0 normally)
    unsigned long long wait_ns;  // limit of one pass's waits
};

// A CTA's dependency lists, after the sweep's shared memory: per family up to
// kPersistDeps share indices and their count (more than that: the CTA waits
// for every share of the family).
constexpr int kPersistDeps = 64;
constexpr size_t kPersistSmemExtra = 2 * kPersistDeps * sizeof(unsigned short) + 2 * sizeof(int);
constexpr unsigned long long kPersistWaitNs = 2000000000ull;  // default wait limit

template <typename T, int K, int R, int NY, bool INTER, bool UNIT>
__global__ void __launch_bounds__(SweepCfg<T, K, R, NY>::NT, SweepCfg<T, K, R, NY>::MINB)
    sweep_persistent_kernel(const __grid_constant__ SweepPersistParams pp) {
    using Cfg = SweepCfg<T, K, R, NY>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const SweepParams &prm = pp.s;
    const int G = int(gridDim.x), b = int(blockIdx.x), tid = int(threadIdx.x);
    const int Ny = prm.a.Ny;
    using L = SweepLayout<T, K, R, INTER>;
    unsigned short *const deps = reinterpret_cast<unsigned short *>(smem_raw + L::SMEM);
    int *const ndeps = reinterpret_cast<int *>(smem_raw + L::SMEM + 2 * kPersistDeps * sizeof(unsigned short));

    // the shares of each family that must have finished a pass before share
    // b of that family starts the next one (each thread tests every NT-th)
    if (tid < 2) ndeps[tid] = 0;
    __syncthreads();
    for (int f = 0; f < pp.nfam; ++f) {
        const SweepSplit &sp = prm.split[f];
        const long long b0 = sp.share_begin(b, G), b1 = sp.share_begin(b + 1, G);
        for (int d = tid; d < G; d += Cfg::NT) {
            if (d != b && sp.shares_touch(b0, b1, sp.share_begin(d, G), sp.share_begin(d + 1, G), W_IN)) {
                const int k = atomicAdd(&ndeps[f], 1);
                if (k < kPersistDeps) deps[f * kPersistDeps + k] = (unsigned short)d;
            }
        }
    }
    __syncthreads();

    // The families never couple (Eq. 17-22), so each runs all its passes in
    // turn: the CTAs of an SM then run one family's code at a time (with the
    // families alternating per pass, two resident CTAs often ran different
    // code: 62.1 against 83.5 G site-updates/s at 8192^2).
    for (int f = 0; f < pp.nfam; ++f) {
        for (int p = 0; p < pp.passes; ++p) {
            // even passes read q_in and write q_out, odd passes the other way
            const bool odd = (p & 1) != 0;
            const SweepMaps *maps = odd ? &pp.m_odd : &prm.m;
            if (p > 0) {
                // thread t waits for dependency t (t, t + NT, ... of all the
                // family's shares when the list overflowed)
                const unsigned target = pp.base + unsigned(p) + pp.withhold;
                const int n = ndeps[f];
                const bool all = n > kPersistDeps;
                int stop = 0;
                const unsigned long long t0 = global_ns();
                for (int k = tid; k < (all ? G : n) && !stop; k += Cfg::NT) {
                    const unsigned *cnt = pp.done + f * G + (all ? k : int(deps[f * kPersistDeps + k]));
                    while (int(ld_acquire_u32(cnt) - target) < 0) {
                        if (*(volatile int *)prm.a.error) {  // another CTA gave up: stop as well
                            stop = 1;
                            break;
                        }
                        if (global_ns() - t0 > pp.wait_ns) {
                            atomicExch(prm.a.error, 1);
                            stop = 1;
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                if (__syncthreads_or(stop)) return;
                // the input rows were written by other CTAs (generic proxy)
                // and are read here by TMA loads (async proxy)
                asm volatile("fence.proxy.async;\n" ::: "memory");
            }
            const SweepSplit &sp = prm.split[f];
            int u = int(sp.share_begin(b, G));  // nsx * Ny < 2^31 (checked on the host)
            const int u1 = int(sp.share_begin(b + 1, G));
            while (u < u1) {
                const int s = u / Ny;
                const int y0 = u - s * Ny;
                const int y1 = min(Ny, y0 + (u1 - u));
                const bool failed =
                    prm.a.fam0 + f != 0
                        ? sweep_body<T, K, R, NY, INTER, UNIT, 1, true>(prm.a, s, y0, y1, smem_raw, maps,
                                                                        prm.merged != 0, odd)
                        : sweep_body<T, K, R, NY, INTER, UNIT, 0, true>(prm.a, s, y0, y1, smem_raw, maps,
                                                                        prm.merged != 0, odd);
                if (failed) return;  // the error flag is set: the other CTAs stop at their next wait
                u += y1 - y0;
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                st_release_u32(pp.done + f * G + b, pp.base + unsigned(p) + 1u);
            }
        }
    }
}

template <typename T, int K, int R, int NY, bool INTER, bool UNIT>
cudaError_t launch_persistent_t(const SweepArgs &a, int nfam, int passes, unsigned base, unsigned *done,
                                unsigned withhold, unsigned long long wait_ns, cudaStream_t st) {
    using Cfg = SweepCfg<T, K, R, NY>;
    using L = SweepLayout<T, K, R, INTER>;
    auto kern = sweep_persistent_kernel<T, K, R, NY, INTER, UNIT>;
    static int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_dev != dev) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L::SMEM + kPersistSmemExtra));
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    if (a.ctas < 1 || a.ctas > kPersistMaxCtas || nfam < 1 || nfam > 2 || passes < 1 || !done ||
        !a.error)
        return cudaErrorInvalidValue;
    SweepPersistParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.s.a = a;
    pp.s.a.order = nullptr;  // share index = blockIdx.x
    // one layer's split per family: CTA b sweeps share b of each family in turn
    for (int z = 0; z < nfam; ++z) pp.s.split[z] = make_sweep_split(a.Nx, a.Ny, K, R, 1, a.fam0 + z, 0, 1);
    pp.s.a.seam = pp.s.split[0].seam;
    if (!pp.s.a.seam || (long long)pp.s.split[0].nsx * a.Ny >= (1LL << 31)) return cudaErrorNotSupported;
    SweepArgs odd = pp.s.a;
    odd.q_in = a.q_out;
    odd.q_out = const_cast<void *>(a.q_in);
    int merged_odd = 0;
    if (!make_sweep_maps(pp.s.a, K, R, pp.s.m, &pp.s.merged) || !make_sweep_maps(odd, K, R, pp.m_odd, &merged_odd) ||
        merged_odd != pp.s.merged)
        return cudaErrorNotSupported;
    pp.s.tma = 1;
    pp.passes = passes;
    pp.nfam = nfam;
    pp.base = base;
    pp.done = done;
    pp.withhold = withhold;
    pp.wait_ns = wait_ns;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(a.ctas), 1, 1);
    cfg.blockDim = dim3(unsigned(Cfg::NT), 1, 1);
    cfg.dynamicSmemBytes = L::SMEM + kPersistSmemExtra;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, pp);
}

// The launch with its waits' test hook (qla_set_wait_limit): withhold extra
// passes demanded by every wait, each pass's waits limited to wait_ns.
cudaError_t launch_sweep_persistent_hooked_f32(int K, const SweepArgs &a, int nfam, int passes, unsigned base,
                                               unsigned *done, unsigned withhold, unsigned long long wait_ns,
                                               cudaStream_t st) {
    if (K != 2) return cudaErrorNotSupported;
    if (a.interleaved) {
        return a.unitary
                   ? launch_persistent_t<float, 2, 4, 2, true, true>(a, nfam, passes, base, done, withhold, wait_ns, st)
                   : launch_persistent_t<float, 2, 4, 2, true, false>(a, nfam, passes, base, done, withhold, wait_ns,
                                                                      st);
    }
    return a.unitary
               ? launch_persistent_t<float, 2, 4, 2, false, true>(a, nfam, passes, base, done, withhold, wait_ns, st)
               : launch_persistent_t<float, 2, 4, 2, false, false>(a, nfam, passes, base, done, withhold, wait_ns, st);
}

cudaError_t launch_sweep_persistent_f32(int K, const SweepArgs &a, int nfam, int passes, unsigned base,
                                        unsigned *done, cudaStream_t st) {
    return launch_sweep_persistent_hooked_f32(K, a, nfam, passes, base, done, 0u, kPersistWaitNs, st);
}

bool sweep_persistent_supported(int precision, int K) { return precision == 0 && K == 2; }

}  // namespace qla
