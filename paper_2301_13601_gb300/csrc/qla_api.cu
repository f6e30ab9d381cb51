// C ABI of libqla: context management, argument validation, buffer
// ownership, pass scheduling and error reporting (declared in include/qla.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/qla.h"
#include "qla_internal.h"

namespace qla {
// The persistent launch with the test hook of its waits (qla_sweep_persist.cu).
cudaError_t launch_sweep_persistent_hooked_f32(int K, const SweepArgs &a, int nfam, int passes, unsigned base,
                                               unsigned *done, unsigned withhold, unsigned long long wait_ns,
                                               cudaStream_t st);
}  // namespace qla

struct qla_ctx {
    int Nx = 0, Ny = 0;
    double delta = 0.0;
    qla_options opt{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool own_mem = false;
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    void *coef = nullptr;
    double *index = nullptr;
    void *scratch = nullptr;
    qla::DiagResult *diag_dev = nullptr;
    qla::DiagResult *diag_host = nullptr;
    int *sweep_err = nullptr;       // device flag: a bounded wait of the sweep's TMA copies ran out
    unsigned *share_order = nullptr;  // device counter: start order of the balanced split's last layer
    int *sweep_err_host = nullptr;  // pinned
    size_t esize = 4;
    int K = 4;
    int chunk = 0;
    int ctas[5] = {0, 0, 0, 0, 0};  // balanced split (chunk == 0): CTAs per family of a pass of K steps
    bool persistent = false;        // passes of K steps in one cooperative launch per qla_step (QLA_LAUNCH_*)
    unsigned *pass_done = nullptr;  // device [2][kPersistMaxCtas]: passes completed per share (persistent form)
    unsigned pass_epoch = 0;        // passes the persistent launches have completed (the counters' base)
    long long wait_ns = 2000000000LL;  // limit of a persistent pass's waits for its neighbours
    unsigned withhold = 0;             // test hook: extra passes every such wait demands
    long long steps = 0;
    bool has_state = false;
    qla_status sticky = QLA_OK;
    std::string msg;
};

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kPassCounterBytes = 2 * size_t(qla::kPersistMaxCtas) * sizeof(unsigned);

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

qla_status fail(qla_ctx *c, qla_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) {
        if (s == QLA_ECUDA || s == QLA_ETIMEOUT) {
            if (c->sticky == QLA_OK) {
                c->sticky = s;
                c->msg = buf;
            }
        } else {
            c->msg = buf;
        }
    }
    return s;
}

#define QLA_CUDA(ctx, expr)                                                                       \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess)                                                                    \
            return fail((ctx), QLA_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(_e));        \
    } while (0)

qla_status enter(qla_ctx *c) {
    if (!c) return QLA_EINVAL;
    if (c->sticky != QLA_OK) return c->sticky;
    cudaError_t e = cudaSetDevice(c->dev);
    if (e != cudaSuccess) return fail(c, QLA_ECUDA, "cudaSetDevice(%d): %s", c->dev, cudaGetErrorString(e));
    return QLA_OK;
}

qla_status validate_sizes(int Nx, int Ny) {
    if (Nx < 1 || Ny < 1) return QLA_EINVAL;
    if ((long long)Nx * (long long)Ny > 2147483647LL) return QLA_EINVAL;
    return QLA_OK;
}

void resolve_options(const qla_options *in, qla_options *out) {
    qla_default_options(out);
    if (in) *out = *in;
}

size_t elem_size(const qla_options &o) { return o.precision == QLA_FP64 ? 8 : 4; }

int sm_count(int dev) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    return n;
}

// Default steps per pass. FP32 with the balanced split: K = 2 (two CTAs per
// SM, 112 KB of shared memory each). Measured on GB300 (three-cylinder
// workload, site-updates/s, K = 2 vs K = 4): 6144^2 79.6 G vs 62.6 G; 4096^2
// 72.8 G vs 51.5 G; 3072^2 66.7 G vs 48.5 G; 2048^2 50.8 G vs 37.3 G; 1024^2
// 24.6 G vs 21.6 G; 768^2 17.5 G vs 13.6 G; 512^2 8.5 G vs 7.2 G; 256^2 2.4 G
// vs 2.1 G. With fixed tiles (chunk_rows > 0) the second resident CTA paid
// only from 2^25 sites up (tiles of 192 and 1024 rows: 8192^2 64.3 G vs
// 55.1 G, 4096^2 42.6-44.4 G vs 43.4-44.0 G, 1024^2 19.9 G vs 25.4 G).
int default_steps_per_pass(int precision, int Nx, int Ny, int chunk_rows) {
    if (precision == QLA_FP64) return 2;
    return chunk_rows == 0 || (long long)Nx * Ny >= (1LL << 25) ? 2 : 4;
}

// CTAs per family of the balanced split of a pass of K steps: one per
// resident slot (SMs x CTAs per SM), at most one per row unit.
int balanced_ctas(int Nx, int Ny, int K, int prec, int interleaved, int sms) {
    const int occ = prec ? qla::sweep_occupancy_f64(K, interleaved) : qla::sweep_occupancy_f32(K, interleaved);
    const qla::SweepSplit sp = qla::make_sweep_split(Nx, Ny, K, qla::sweep_block_rows(prec, K), prec ? 0 : 1);
    return int(std::min((long long)sms * occ, (long long)sp.nsx * Ny));
}

// Whether the context's passes of K steps can take the persistent launch form:
// FP32, the balanced split, K instantiated for it, the seam layout (Nx a
// multiple of 8, at least 256 columns) and at most kPersistMaxCtas shares.
bool persistent_applies(const qla_ctx *c) {
    return c->opt.precision == QLA_FP32 && c->chunk == 0 && qla::sweep_persistent_supported(0, c->K) &&
           c->Nx % 8 == 0 && c->Nx >= qla::sweep_strip_width() && c->ctas[c->K] >= 1 &&
           c->ctas[c->K] <= qla::kPersistMaxCtas;
}

// Whether component `comp` (Eq. 15 order) belongs to a family the context
// advances: TM = (q2, q3, q4), TE = (q0, q1, q5).
bool family_has(const qla_ctx *c, int comp) {
    if (c->opt.families == QLA_FAMILIES_BOTH) return true;
    const bool tm = comp >= 2 && comp <= 4;
    return c->opt.families == QLA_FAMILY_TM ? tm : !tm;
}

qla_status launch_pass(qla_ctx *c, int K) {
    qla::SweepArgs a{};
    a.q_in = c->state[c->cur];
    a.q_out = c->state[c->cur ^ 1];
    a.coef = c->coef;
    a.Nx = c->Nx;
    a.Ny = c->Ny;
    a.w_valid = qla::sweep_strip_width() - 8 * K;
    a.chunk = c->chunk;
    a.ctas = c->ctas[K];
    a.order = c->share_order;
    a.interleaved = c->opt.sequence == QLA_SEQ_INTERLEAVED ? 1 : 0;
    a.unitary = c->opt.potential == QLA_POT_UNITARY ? 1 : 0;
    a.vec = (c->Nx % int(16 / c->esize)) == 0 ? 1 : 0;
    // one CTA grid layer per advanced family (TM = family 0, TE = family 1);
    // the planes of a family that is not advanced stay zero in both buffers
    const int nfam = c->opt.families == QLA_FAMILIES_BOTH ? 2 : 1;
    a.fam0 = c->opt.families == QLA_FAMILY_TE ? 1 : 0;
    a.error = c->sweep_err;
    cudaError_t e = c->opt.precision == QLA_FP64 ? qla::launch_sweep_f64(K, a, nfam, c->stream)
                                                  : qla::launch_sweep_f32(K, a, nfam, c->stream);
    if (e != cudaSuccess) return fail(c, QLA_ECUDA, "sweep launch (K=%d): %s", K, cudaGetErrorString(e));
    c->cur ^= 1;
    return QLA_OK;
}

// `passes` passes of K = c->K steps in one cooperative launch. *refused: the
// device did not take the launch (nothing ran; the caller falls back to one
// launch per pass).
qla_status launch_persistent(qla_ctx *c, int passes, bool *refused) {
    *refused = false;
    const int K = c->K;
    qla::SweepArgs a{};
    a.q_in = c->state[c->cur];
    a.q_out = c->state[c->cur ^ 1];
    a.coef = c->coef;
    a.Nx = c->Nx;
    a.Ny = c->Ny;
    a.w_valid = qla::sweep_strip_width() - 8 * K;
    a.chunk = 0;
    a.ctas = c->ctas[K];
    a.order = nullptr;
    a.interleaved = c->opt.sequence == QLA_SEQ_INTERLEAVED ? 1 : 0;
    a.unitary = c->opt.potential == QLA_POT_UNITARY ? 1 : 0;
    a.vec = (c->Nx % int(16 / c->esize)) == 0 ? 1 : 0;
    const int nfam = c->opt.families == QLA_FAMILIES_BOTH ? 2 : 1;
    a.fam0 = c->opt.families == QLA_FAMILY_TE ? 1 : 0;
    a.error = c->sweep_err;
    const cudaError_t e = qla::launch_sweep_persistent_hooked_f32(K, a, nfam, passes, c->pass_epoch, c->pass_done,
                                                                  c->withhold, (unsigned long long)c->wait_ns,
                                                                  c->stream);
    if (e == cudaErrorNotSupported || e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        *refused = true;
        return QLA_OK;
    }
    if (e != cudaSuccess) return fail(c, QLA_ECUDA, "persistent sweep launch (K=%d): %s", K, cudaGetErrorString(e));
    c->pass_epoch += unsigned(passes);
    if (passes & 1) c->cur ^= 1;
    return QLA_OK;
}

// After a stream synchronisation: report a sweep whose TMA copy wait ran out.
qla_status check_sweep_error(qla_ctx *c) {
    QLA_CUDA(c, cudaMemcpyAsync(c->sweep_err_host, c->sweep_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QLA_CUDA(c, cudaStreamSynchronize(c->stream));
    if (*c->sweep_err_host) return fail(c, QLA_ETIMEOUT, "a sweep's wait for its row copies ran out of its limit");
    return QLA_OK;
}

qla_status run_diag(qla_ctx *c) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (!c->has_state) return fail(c, QLA_ESTATE, "no state set (call qla_init_pulse or qla_set_fields)");
    cudaError_t e = qla::launch_diagnostics(c->state[c->cur], c->opt.precision == QLA_FP64 ? 1 : 0, c->Nx, c->Ny,
                                            c->scratch, c->diag_dev, c->stream);
    if (e != cudaSuccess) return fail(c, QLA_ECUDA, "diagnostics launch: %s", cudaGetErrorString(e));
    QLA_CUDA(c, cudaMemcpyAsync(c->diag_host, c->diag_dev, sizeof(qla::DiagResult), cudaMemcpyDeviceToHost,
                                c->stream));
    return check_sweep_error(c);
}

}  // namespace

extern "C" {

void qla_default_options(qla_options *opt) {
    if (!opt) return;
    opt->precision = QLA_FP32;
    opt->sequence = QLA_SEQ_INTERLEAVED;
    opt->potential = QLA_POT_PAPER;
    opt->steps_per_pass = 0;
    opt->chunk_rows = 0;
    opt->device = -1;
    opt->stream = nullptr;
    opt->families = QLA_FAMILIES_BOTH;
    opt->launch = QLA_LAUNCH_AUTO;
}

qla_status qla_query_buffer_sizes(int Nx, int Ny, const qla_options *opt, qla_buffer_sizes *out) {
    if (!out || validate_sizes(Nx, Ny) != QLA_OK) return QLA_EINVAL;
    qla_options o;
    resolve_options(opt, &o);
    if (o.precision != QLA_FP32 && o.precision != QLA_FP64) return QLA_EINVAL;
    const size_t P = size_t(Nx) * size_t(Ny);
    const size_t es = elem_size(o);
    out->state_bytes = round_up(6 * P * es, kAlign);
    out->coeff_bytes = round_up(size_t(qla::NCOEF) * P * es, kAlign);
    out->index_bytes = round_up(3 * P * sizeof(double), kAlign);
    out->scratch_bytes = round_up(qla::diag_scratch_bytes(Nx, Ny), kAlign) + round_up(sizeof(qla::DiagResult), kAlign) +
                         kAlign +  // sweep error flag, share-order counter
                         kPassCounterBytes;  // per-share pass counters of the persistent launch form
    return QLA_OK;
}

qla_status qla_create(int Nx, int Ny, const double *n_x, const double *n_y, const double *n_z, double delta,
                      const qla_options *opt, const qla_device_buffers *buffers, qla_ctx **out) {
    if (!out) return QLA_EINVAL;
    *out = nullptr;
    if (validate_sizes(Nx, Ny) != QLA_OK || !n_x || !n_y || !n_z) return QLA_EINVAL;
    if (!(delta > 0.0) || !(delta <= 0.5) || !std::isfinite(delta)) return QLA_EINVAL;
    qla_options o;
    resolve_options(opt, &o);
    if (o.precision != QLA_FP32 && o.precision != QLA_FP64) return QLA_EINVAL;
    if (o.sequence != QLA_SEQ_INTERLEAVED && o.sequence != QLA_SEQ_PLAIN) return QLA_EINVAL;
    if (o.potential != QLA_POT_PAPER && o.potential != QLA_POT_UNITARY) return QLA_EINVAL;
    if (o.families != QLA_FAMILIES_BOTH && o.families != QLA_FAMILY_TM && o.families != QLA_FAMILY_TE)
        return QLA_EINVAL;
    if (o.steps_per_pass < 0 || o.chunk_rows < 0) return QLA_EINVAL;
    if (o.launch != QLA_LAUNCH_AUTO && o.launch != QLA_LAUNCH_PER_PASS && o.launch != QLA_LAUNCH_PERSISTENT)
        return QLA_EINVAL;
    if (o.steps_per_pass > 0 && !qla::sweep_supported(o.precision, o.steps_per_pass)) return QLA_EUNSUPPORTED;
    const size_t P = size_t(Nx) * size_t(Ny);
    const double *nn[3] = {n_x, n_y, n_z};
    for (int k = 0; k < 3; ++k)
        for (size_t i = 0; i < P; ++i)
            if (!(nn[k][i] > 0.0) || !std::isfinite(nn[k][i])) return QLA_EINVAL;

    qla_ctx *c = new qla_ctx();
    c->Nx = Nx;
    c->Ny = Ny;
    c->delta = delta;
    c->opt = o;
    c->esize = elem_size(o);
    auto bail = [&](qla_status s) {
        qla_destroy(c);
        return s;
    };
    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) return bail(QLA_ECUDA);
        c->dev = o.device;
    } else if (cudaGetDevice(&c->dev) != cudaSuccess) {
        return bail(QLA_ECUDA);
    }
    if (cudaFree(nullptr) != cudaSuccess) return bail(QLA_ECUDA);  // context up
    if (o.stream) {
        c->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(QLA_ECUDA);
        c->own_stream = true;
    }
    qla_buffer_sizes bs;
    qla_query_buffer_sizes(Nx, Ny, &o, &bs);
    if (buffers) {
        if (!buffers->state[0] || !buffers->state[1] || !buffers->coeff || !buffers->index || !buffers->scratch)
            return bail(QLA_EINVAL);
        const void *ps[5] = {buffers->state[0], buffers->state[1], buffers->coeff, buffers->index, buffers->scratch};
        for (const void *p : ps)
            if ((reinterpret_cast<uintptr_t>(p) % kAlign) != 0) return bail(QLA_EINVAL);
        c->state[0] = buffers->state[0];
        c->state[1] = buffers->state[1];
        c->coef = buffers->coeff;
        c->index = static_cast<double *>(buffers->index);
        c->scratch = buffers->scratch;
    } else {
        c->own_mem = true;
        if (cudaMalloc(&c->state[0], bs.state_bytes) != cudaSuccess ||
            cudaMalloc(&c->state[1], bs.state_bytes) != cudaSuccess ||
            cudaMalloc(&c->coef, bs.coeff_bytes) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void **>(&c->index), bs.index_bytes) != cudaSuccess ||
            cudaMalloc(&c->scratch, bs.scratch_bytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(QLA_ENOMEM);
        }
    }
    c->diag_dev = reinterpret_cast<qla::DiagResult *>(static_cast<char *>(c->scratch) +
                                                      round_up(qla::diag_scratch_bytes(Nx, Ny), kAlign));
    c->sweep_err = reinterpret_cast<int *>(reinterpret_cast<char *>(c->diag_dev) +
                                           round_up(sizeof(qla::DiagResult), kAlign));
    if (cudaMallocHost(reinterpret_cast<void **>(&c->diag_host), sizeof(qla::DiagResult)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&c->sweep_err_host), sizeof(int)) != cudaSuccess)
        return bail(QLA_ENOMEM);
    // the sweep error flag and, 64 bytes on in the same slot, the share-order counter
    c->share_order = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(c->sweep_err) + 64);
    if (cudaMemsetAsync(c->sweep_err, 0, kAlign, c->stream) != cudaSuccess) return bail(QLA_ECUDA);
    c->pass_done = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(c->sweep_err) + kAlign);
    if (cudaMemsetAsync(c->pass_done, 0, kPassCounterBytes, c->stream) != cudaSuccess) return bail(QLA_ECUDA);
    for (int k = 0; k < 3; ++k)
        if (cudaMemcpyAsync(c->index + size_t(k) * P, nn[k], P * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess)
            return bail(QLA_ECUDA);
    if (qla::launch_coefficients(c->index, c->coef, Nx, Ny, delta, o.precision,
                                 o.sequence == QLA_SEQ_INTERLEAVED ? 1 : 0, o.potential == QLA_POT_UNITARY ? 1 : 0,
                                 c->stream) != cudaSuccess)
        return bail(QLA_ECUDA);
    if (cudaMemsetAsync(c->state[0], 0, bs.state_bytes, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->state[1], 0, bs.state_bytes, c->stream) != cudaSuccess)
        return bail(QLA_ECUDA);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(QLA_ECUDA);
    c->K = o.steps_per_pass > 0 ? o.steps_per_pass : default_steps_per_pass(o.precision, Nx, Ny, o.chunk_rows);
    c->chunk = o.chunk_rows > 0 ? std::min(o.chunk_rows, Ny) : 0;
    if (c->chunk == 0)
        for (int k = 1; k <= 4; ++k)
            if (qla::sweep_supported(o.precision, k))
                c->ctas[k] = balanced_ctas(Nx, Ny, k, o.precision == QLA_FP64 ? 1 : 0,
                                           o.sequence == QLA_SEQ_INTERLEAVED ? 1 : 0, sm_count(c->dev));
    // QLA_LAUNCH_AUTO: one launch per pass, measured the faster form (the persistent one on GB300, 8192^2,
    // 2 steps per pass, site-updates/s: both families 62.1 G with the families alternating per pass against
    // 83.5 G; TM alone 161.2 against 164.6 G; TE alone 166.2 against 163.5 G)
    c->persistent = o.launch == QLA_LAUNCH_PERSISTENT && persistent_applies(c);
    c->has_state = true;  // zero state
    *out = c;
    return QLA_OK;
}

qla_status qla_init_pulse(qla_ctx *c, int polarization, double x0, double sigma, double amplitude) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if ((polarization != QLA_POL_EZ && polarization != QLA_POL_EY) || !(sigma > 0.0) || !std::isfinite(x0) ||
        !std::isfinite(sigma) || !std::isfinite(amplitude))
        return fail(c, QLA_EINVAL, "qla_init_pulse: invalid argument");
    if ((polarization == QLA_POL_EZ && c->opt.families == QLA_FAMILY_TE) ||
        (polarization == QLA_POL_EY && c->opt.families == QLA_FAMILY_TM))
        return fail(c, QLA_EINVAL, "qla_init_pulse: the pulse's family is not advanced by this context");
    cudaError_t e = qla::launch_init_pulse(c->state[c->cur], c->Nx, c->Ny, c->opt.precision == QLA_FP64 ? 1 : 0,
                                           polarization, x0, sigma, amplitude, c->stream);
    if (e != cudaSuccess) return fail(c, QLA_ECUDA, "pulse launch: %s", cudaGetErrorString(e));
    c->steps = 0;
    c->has_state = true;
    return QLA_OK;
}

qla_status qla_set_fields(qla_ctx *c, const double *q) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (!q) return fail(c, QLA_EINVAL, "qla_set_fields: NULL");
    const size_t P = size_t(c->Nx) * size_t(c->Ny);
    std::vector<float> tmp(c->opt.precision == QLA_FP64 ? 0 : P);
    for (int comp = 0; comp < 6; ++comp) {
        if (!family_has(c, comp)) continue;
        const double *src = q + comp * P;
        if (c->opt.precision == QLA_FP64) {
            QLA_CUDA(c, cudaMemcpyAsync(static_cast<double *>(c->state[c->cur]) + comp * P, src, P * 8,
                                        cudaMemcpyHostToDevice, c->stream));
        } else {
            QLA_CUDA(c, cudaStreamSynchronize(c->stream));  // tmp is reused per plane
            for (size_t i = 0; i < P; ++i) tmp[i] = float(src[i]);
            QLA_CUDA(c, cudaMemcpyAsync(static_cast<float *>(c->state[c->cur]) + comp * P, tmp.data(), P * 4,
                                        cudaMemcpyHostToDevice, c->stream));
        }
    }
    QLA_CUDA(c, cudaStreamSynchronize(c->stream));
    c->steps = 0;
    c->has_state = true;
    return QLA_OK;
}

qla_status qla_set_fields_f32(qla_ctx *c, const float *q) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (!q) return fail(c, QLA_EINVAL, "qla_set_fields_f32: NULL");
    const size_t P = size_t(c->Nx) * size_t(c->Ny);
    if (c->opt.precision == QLA_FP32) {
        if (c->opt.families == QLA_FAMILIES_BOTH) {
            QLA_CUDA(c, cudaMemcpyAsync(c->state[c->cur], q, 6 * P * 4, cudaMemcpyHostToDevice, c->stream));
        } else {
            for (int comp = 0; comp < 6; ++comp)
                if (family_has(c, comp))
                    QLA_CUDA(c, cudaMemcpyAsync(static_cast<float *>(c->state[c->cur]) + comp * P, q + comp * P,
                                                P * 4, cudaMemcpyHostToDevice, c->stream));
        }
    } else {
        std::vector<double> tmp(P);
        for (int comp = 0; comp < 6; ++comp) {
            if (!family_has(c, comp)) continue;
            for (size_t i = 0; i < P; ++i) tmp[i] = double(q[comp * P + i]);
            QLA_CUDA(c, cudaMemcpyAsync(static_cast<double *>(c->state[c->cur]) + comp * P, tmp.data(), P * 8,
                                        cudaMemcpyHostToDevice, c->stream));
            QLA_CUDA(c, cudaStreamSynchronize(c->stream));
        }
    }
    c->steps = 0;
    c->has_state = true;
    return QLA_OK;
}

qla_status qla_step(qla_ctx *c, long long nsteps) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (nsteps < 0) return fail(c, QLA_EINVAL, "qla_step: nsteps < 0");
    if (!c->has_state) return fail(c, QLA_ESTATE, "qla_step: no state");
    long long left = nsteps;
    // the full passes in cooperative launches (at most 2^20 passes each)
    while (c->persistent && left >= c->K) {
        const int passes = int(std::min(left / c->K, 1LL << 20));
        bool refused = false;
        s = launch_persistent(c, passes, &refused);
        if (s != QLA_OK) return s;
        if (refused) {  // from now on one launch per pass
            c->persistent = false;
            break;
        }
        left -= (long long)passes * c->K;
        c->steps += (long long)passes * c->K;
    }
    while (left > 0) {
        int k = c->K;
        while (k > 1 && (k > left || !qla::sweep_supported(c->opt.precision, k))) --k;
        s = launch_pass(c, k);
        if (s != QLA_OK) return s;
        left -= k;
        c->steps += k;
    }
    return QLA_OK;
}

qla_status qla_diagnostics(qla_ctx *c, qla_diag *out) {
    if (!out) return fail(c, QLA_EINVAL, "qla_diagnostics: NULL");
    qla_status s = run_diag(c);
    if (s != QLA_OK) return s;
    const qla::DiagResult &r = *c->diag_host;
    out->energy = r.energy_sum / (double(c->Nx) * double(c->Ny));
    out->div_l2_sq = r.div_sq_sum;
    out->div_max = r.div_max;
    out->b_max = r.b_max;
    out->nonfinite = (long long)r.nonfinite;
    if (r.nonfinite) return fail(c, QLA_ENONFINITE, "state holds %llu non-finite values", r.nonfinite);
    return QLA_OK;
}

qla_status qla_energy(qla_ctx *c, double *energy) {
    if (!energy) return fail(c, QLA_EINVAL, "qla_energy: NULL");
    qla_diag d;
    qla_status s = qla_diagnostics(c, &d);
    if (s != QLA_OK && s != QLA_ENONFINITE) return s;
    *energy = d.energy;
    return s;
}

qla_status qla_divB(qla_ctx *c, double *l2_sq_sum, double *max_abs, double *max_absB) {
    qla_diag d;
    qla_status s = qla_diagnostics(c, &d);
    if (s != QLA_OK && s != QLA_ENONFINITE) return s;
    if (l2_sq_sum) *l2_sq_sum = d.div_l2_sq;
    if (max_abs) *max_abs = d.div_max;
    if (max_absB) *max_absB = d.b_max;
    return s;
}

qla_status qla_divD(qla_ctx *c, double *l2_sq_sum, double *max_abs, double *max_absD) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (!c->has_state) return fail(c, QLA_ESTATE, "no state set (call qla_init_pulse or qla_set_fields)");
    cudaError_t e = qla::launch_divD(c->state[c->cur], c->opt.precision == QLA_FP64 ? 1 : 0, c->index, c->Nx, c->Ny,
                                     c->scratch, c->diag_dev, c->stream);
    if (e != cudaSuccess) return fail(c, QLA_ECUDA, "div D launch: %s", cudaGetErrorString(e));
    QLA_CUDA(c, cudaMemcpyAsync(c->diag_host, c->diag_dev, sizeof(qla::DiagResult), cudaMemcpyDeviceToHost,
                                c->stream));
    s = check_sweep_error(c);
    if (s != QLA_OK) return s;
    if (l2_sq_sum) *l2_sq_sum = c->diag_host->div_sq_sum;
    if (max_abs) *max_abs = c->diag_host->div_max;
    if (max_absD) *max_absD = c->diag_host->b_max;
    return c->diag_host->nonfinite ? QLA_ENONFINITE : QLA_OK;
}

qla_status qla_get_fields(qla_ctx *c, double *q) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (!q) return fail(c, QLA_EINVAL, "qla_get_fields: NULL");
    const size_t n = 6 * size_t(c->Nx) * size_t(c->Ny);
    if (c->opt.precision == QLA_FP64) {
        QLA_CUDA(c, cudaMemcpyAsync(q, c->state[c->cur], n * 8, cudaMemcpyDeviceToHost, c->stream));
        QLA_CUDA(c, cudaStreamSynchronize(c->stream));
    } else {
        std::vector<float> tmp(n);
        QLA_CUDA(c, cudaMemcpyAsync(tmp.data(), c->state[c->cur], n * 4, cudaMemcpyDeviceToHost, c->stream));
        QLA_CUDA(c, cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < n; ++i) q[i] = double(tmp[i]);
    }
    return QLA_OK;
}

qla_status qla_get_fields_f32(qla_ctx *c, float *q) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (!q) return fail(c, QLA_EINVAL, "qla_get_fields_f32: NULL");
    const size_t n = 6 * size_t(c->Nx) * size_t(c->Ny);
    if (c->opt.precision == QLA_FP32) {
        QLA_CUDA(c, cudaMemcpyAsync(q, c->state[c->cur], n * 4, cudaMemcpyDeviceToHost, c->stream));
        QLA_CUDA(c, cudaStreamSynchronize(c->stream));
    } else {
        std::vector<double> tmp(n);
        QLA_CUDA(c, cudaMemcpyAsync(tmp.data(), c->state[c->cur], n * 8, cudaMemcpyDeviceToHost, c->stream));
        QLA_CUDA(c, cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < n; ++i) q[i] = float(tmp[i]);
    }
    return QLA_OK;
}

qla_status qla_debug_apply(qla_ctx *c, int op, int count) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    if (op < QLA_OP_CX || op > QLA_OP_VY || count < 0) return fail(c, QLA_EINVAL, "qla_debug_apply: bad op or count");
    if (!c->has_state) return fail(c, QLA_ESTATE, "qla_debug_apply: no state");
    for (int k = 0; k < count; ++k) {
        bool swapped = false;
        const cudaError_t e = qla::debug_apply(op, c->opt.precision, c->state[c->cur], c->state[c->cur ^ 1], c->coef,
                                               c->Nx, c->Ny, c->opt.potential == QLA_POT_UNITARY ? 1 : 0, c->stream,
                                               &swapped);
        if (e != cudaSuccess) return fail(c, QLA_ECUDA, "qla_debug_apply: %s", cudaGetErrorString(e));
        if (swapped) c->cur ^= 1;
    }
    return QLA_OK;
}

void *qla_state_device_ptr(qla_ctx *c) { return c ? c->state[c->cur] : nullptr; }

qla_status qla_synchronize(qla_ctx *c) {
    qla_status s = enter(c);
    if (s != QLA_OK) return s;
    QLA_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_sweep_error(c);
}

long long qla_step_count(const qla_ctx *c) { return c ? c->steps : -1; }

qla_status qla_get_config(const qla_ctx *c, int *steps_per_pass, int *chunk_rows, int *precision) {
    if (!c) return QLA_EINVAL;
    if (steps_per_pass) *steps_per_pass = c->K;
    if (chunk_rows) *chunk_rows = c->chunk;
    if (precision) *precision = c->opt.precision;
    return QLA_OK;
}

namespace {
qla_status write_split(const qla::SweepSplit &sp, int ctas, long long *bounds, int capacity) {
    if (ctas < 1 || !bounds || capacity < ctas + 1) return QLA_EINVAL;
    for (int b = 0; b <= ctas; ++b) bounds[b] = sp.share_begin(b, ctas);
    return QLA_OK;
}
}  // namespace

qla_status qla_sweep_split(int Nx, int Ny, int precision, int steps_per_pass, int ctas, int family, int layers,
                           long long *bounds, int capacity) {
    if (Nx < 1 || Ny < 1 || (precision != QLA_FP32 && precision != QLA_FP64)) return QLA_EINVAL;
    if ((family != QLA_FAMILY_TM && family != QLA_FAMILY_TE) || (layers != 1 && layers != 2)) return QLA_EINVAL;
    if (!qla::sweep_supported(precision, steps_per_pass)) return QLA_EUNSUPPORTED;
    const int prec = precision == QLA_FP64 ? 1 : 0;
    const int fam = family == QLA_FAMILY_TE ? 1 : 0;
    const qla::SweepSplit sp = qla::make_sweep_split(Nx, Ny, steps_per_pass, qla::sweep_block_rows(prec, steps_per_pass),
                                                     prec ? 0 : 1, fam, layers == 2 ? fam : 0, layers);
    if ((long long)sp.nsx * Ny >= (1LL << 31)) return QLA_EINVAL;
    return write_split(sp, ctas, bounds, capacity);
}

qla_status qla_get_sweep_split(const qla_ctx *c, int steps_per_pass, int family, int *ctas, long long *bounds,
                               int capacity) {
    if (!c || !ctas) return QLA_EINVAL;
    if (family != QLA_FAMILY_TM && family != QLA_FAMILY_TE) return QLA_EINVAL;
    if (!qla::sweep_supported(c->opt.precision, steps_per_pass)) return QLA_EUNSUPPORTED;
    const bool advanced = c->opt.families == QLA_FAMILIES_BOTH || c->opt.families == family;
    *ctas = c->chunk > 0 || !advanced ? 0 : c->ctas[steps_per_pass];
    if (*ctas == 0 || !bounds) return QLA_OK;
    // the persistent form sweeps one layer's split per family
    const bool one_layer = c->opt.families != QLA_FAMILIES_BOTH || (c->persistent && steps_per_pass == c->K);
    return qla_sweep_split(c->Nx, c->Ny, c->opt.precision, steps_per_pass, *ctas, family, one_layer ? 1 : 2, bounds,
                           capacity);
}

qla_status qla_sweep_dependencies(int Nx, int Ny, int steps_per_pass, int ctas, int family, int share, int *deps,
                                  int capacity, int *count) {
    if (Nx < 1 || Ny < 1 || !deps || !count || capacity < 0) return QLA_EINVAL;
    if (family != QLA_FAMILY_TM && family != QLA_FAMILY_TE) return QLA_EINVAL;
    if (ctas < 1 || ctas > qla::kPersistMaxCtas || share < 0 || share >= ctas) return QLA_EINVAL;
    if (!qla::sweep_persistent_supported(0, steps_per_pass)) return QLA_EUNSUPPORTED;
    const qla::SweepSplit sp = qla::make_sweep_split(Nx, Ny, steps_per_pass, qla::sweep_block_rows(0, steps_per_pass),
                                                     1, family == QLA_FAMILY_TE ? 1 : 0, 0, 1);
    if (!sp.seam) return QLA_EUNSUPPORTED;
    if ((long long)sp.nsx * Ny >= (1LL << 31)) return QLA_EINVAL;
    const long long b0 = sp.share_begin(share, ctas), b1 = sp.share_begin(share + 1, ctas);
    int n = 0;
    for (int d = 0; d < ctas; ++d) {
        if (d == share ||
            !sp.shares_touch(b0, b1, sp.share_begin(d, ctas), sp.share_begin(d + 1, ctas), qla::sweep_strip_width()))
            continue;
        if (n >= capacity) return QLA_EINVAL;
        deps[n++] = d;
    }
    *count = n;
    return QLA_OK;
}

qla_status qla_set_wait_limit(qla_ctx *c, long long timeout_ns, int withhold) {
    if (!c || timeout_ns <= 0 || withhold < 0) return QLA_EINVAL;
    c->wait_ns = timeout_ns;
    c->withhold = unsigned(withhold);
    return QLA_OK;
}

qla_status qla_get_launch(const qla_ctx *c, int *launch) {
    if (!c || !launch) return QLA_EINVAL;
    *launch = c->persistent ? QLA_LAUNCH_PERSISTENT : QLA_LAUNCH_PER_PASS;
    return QLA_OK;
}

const char *qla_last_error(const qla_ctx *c) { return c ? c->msg.c_str() : "NULL context"; }

const char *qla_status_string(qla_status s) {
    switch (s) {
        case QLA_OK: return "QLA_OK";
        case QLA_EINVAL: return "QLA_EINVAL";
        case QLA_ENOMEM: return "QLA_ENOMEM";
        case QLA_ECUDA: return "QLA_ECUDA";
        case QLA_ETIMEOUT: return "QLA_ETIMEOUT";
        case QLA_ENONFINITE: return "QLA_ENONFINITE";
        case QLA_EUNSUPPORTED: return "QLA_EUNSUPPORTED";
        case QLA_ESTATE: return "QLA_ESTATE";
    }
    return "unknown";
}

void qla_destroy(qla_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->own_mem) {
        cudaFree(c->state[0]);
        cudaFree(c->state[1]);
        cudaFree(c->coef);
        cudaFree(c->index);
        cudaFree(c->scratch);
    }
    if (c->diag_host) cudaFreeHost(c->diag_host);
    if (c->sweep_err_host) cudaFreeHost(c->sweep_err_host);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

}  // extern "C"

namespace qla {

bool ctx_view(qla_ctx *c, CtxView *v) {
    if (!c || !v) return false;
    v->Nx = c->Nx;
    v->Ny = c->Ny;
    v->precision = c->opt.precision;
    v->stream = c->stream;
    v->cur_state = c->state[c->cur];
    v->spare_state = c->state[c->cur ^ 1];
    v->has_state = c->has_state ? 1 : 0;
    v->families = c->opt.families;
    return true;
}

void ctx_commit_spare(qla_ctx *c, long long steps) {
    c->cur ^= 1;
    c->steps += steps;
}

void ctx_add_steps(qla_ctx *c, long long steps) { c->steps += steps; }

}  // namespace qla
