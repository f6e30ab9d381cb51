/* Learned time-stepping surrogate for the QLA: BF16 tensor-core convolution
 * building blocks (tcgen05, FP32 accumulation in tensor memory).
 *
 * The surrogate advances the fields of the 2D anisotropic-dielectric scattering
 * problem (Sec. 4) by K QLA steps per call: Q_{t+K} = Q_t + s * f([Q_t, n]).
 * The paper has no learned component; the network only approximates the map
 * that the QLA step (Eq. 28) iterated K times defines, and plain QLA stays its
 * fallback and the reference its error and energy (Eq. 27) are measured against.
 *
 * Conventions: activations are BF16 in NHWC order ([H][W][C], C contiguous)
 * on a periodic H x W lattice (circular padding, as the QLA lattice); all
 * pointers are DEVICE pointers owned by the caller, 16-byte aligned; `stream`
 * is a cudaStream_t (NULL = legacy default stream). Calls are asynchronous
 * on the stream; argument errors are returned before any launch.
 */
#ifndef QLA_SURROGATE_H
#define QLA_SURROGATE_H

#include "qla.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Epilogues of qla_conv3x3_bf16. acc = sum_{ky,kx,c} w[n][c][ky][kx] x[y+ky-1][x+kx-1][c]. */
enum {
    QLA_EPI_GELU = 0,    /* z = acc + b; out0 = BF16(z) (NULL: not stored); out1 = BF16(GELU(z) + aux0) (aux0: BF16 residual or NULL) */
    QLA_EPI_LINEAR = 1,  /* out0 = FP32 (acc + b), [H][W][nout] */
    QLA_EPI_DGRAD = 2,   /* g = acc + aux0 (FP32 [H][W][nout] or NULL); out0 = g (FP32); out1 = BF16(g * GELU'(zprev)) */
    QLA_EPI_QUPDATE = 3  /* out0[i][c][y][x] = aux0[i][c][y][x] + scale * (acc + b)[c], c < 6 (FP32 [nimg][6][H][W]) */
};

/* One 3x3 circular convolution as an implicit GEMM on the tensor cores, over
 * nimg images of H x W stacked in memory, each periodic on its own.
 * x: BF16 [nimg][H][W][cin]; w_packed: BF16 [9][cin/8][nout][8] (qla_pack_conv_weights);
 * bias: FP32 [nout] or NULL (ignored by QLA_EPI_DGRAD); GELU is the tanh form.
 * Supported (cin, nout): (16, 64), (64, 64), (64, 16); W a multiple of 128.
 * error_flag: device int set to 1 if the kernel's bounded wait for its tensor
 * core work ran out (the outputs are then invalid); the caller zeroes it.
 * Errors: QLA_EINVAL (NULL pointer, bad size or epilogue operands),
 * QLA_EUNSUPPORTED (channel pair), QLA_ECUDA (launch failure). */
qla_status qla_conv3x3_bf16(const void *x, int nimg, int H, int W, int cin, const void *w_packed, const float *bias,
                            int nout, int epilogue, const void *aux0, const void *zprev, void *out0, void *out1,
                            float scale, int *error_flag, void *stream);

/* The MMA issue schedule of one CTA of qla_conv3x3_bf16 (cin, nout as there;
 * the CTA takes rows [T cta / grid, T (cta + 1) / grid) of the T = nimg H W/128
 * (image, column block, row) items), enumerated on the host by the same code
 * the kernel's MMA warp runs; for tests. No GPU is touched. Each record is
 * QLA_CONV_SCHEDULE_FIELDS ints [type, r, on, j, len, a, b, c, d, e, f, g, h, 0]
 * with r the ring row, on the output row fed by y tap 0, j the input row of
 * the run of len output rows, and per type:
 *   0 MMA: a = x tap, b = 16-channel slice, c..d = y taps ka..kb, e = first
 *     accumulator block, f = accumulate flag, g = A start and h = B start
 *     (16-byte units from the ring slot and the packed weights);
 *   1 accumulator of output row on - 2 complete: a = its block;
 *   2 wait for the epilogue of the block's previous row before the row's MMAs:
 *     a = block, b = phase parity;
 *   3 the row's ring slot released by the tensor cores: a = slot.
 * At most `capacity` records are written to `records` (host); *count gets the
 * total. Errors: QLA_EINVAL (sizes, W not a multiple of 128, cta out of range,
 * NULL count), QLA_EUNSUPPORTED (channel pair). */
#define QLA_CONV_SCHEDULE_FIELDS 14
qla_status qla_conv_schedule(int cin, int nout, int nimg, int H, int W, int grid, int cta, int *records,
                             long long capacity, long long *count);

/* Pack FP32 weights w[nout][cin][3][3] (device) into the BF16 B-operand layout
 * [9][cin_pad/8][nout_pad][8], zero-padded. transpose_flip != 0 packs the
 * adjoint (input-gradient) convolution instead, w'[c][n][ky][kx] =
 * w[n][c][2-ky][2-kx], whose output channels are w's inputs (then cin <=
 * nout_pad and nout <= cin_pad). Errors: QLA_EINVAL. */
qla_status qla_pack_conv_weights(const float *w, int nout, int cin, int nout_pad, int cin_pad, int transpose_flip,
                                 void *packed, void *stream);


/* ---------------------------------------------------------------------------
 * The surrogate network and its training and rollout.
 *
 * f is a 6-layer residual CNN with 64 hidden channels and GELU:
 *   a0 = GELU(conv0(x0)); a_l = a_{l-1} + GELU(conv_l(a_{l-1})), l = 1..4;
 *   f = conv5(a4) (6 output channels); Q_{t+K} = Q_t + out_scale * f.
 * x0 holds, per site, the six state components (each as a high and a low
 * BF16 part that share first-layer weights) and n_x, n_y, n_z.
 * Parameters are one FP32 vector, layer by layer: W_l [nout][cin][3][3] then
 * b_l [nout], with (cin, nout) = (9, 64), (64, 64) x 4, (64, 6); first-layer
 * input channels are Q0..Q5, n_x, n_y, n_z. Fields are FP32 device planes:
 * Q as [nimg][6][H][W] (the QLA state layout), n as [nimg][3][H][W].
 * ------------------------------------------------------------------------- */
typedef struct qla_surrogate qla_surrogate;

typedef struct {
    int nimg;          /* images per call (training batch); 1 for a rollout */
    int H, W;          /* lattice (Ny, Nx); W a multiple of 128 */
    int K;             /* QLA steps that one call stands for (rollout; multiple of the context's steps per pass) */
    float out_scale;   /* s > 0 */
    int train;         /* nonzero: allocate gradient, optimiser and activation buffers for training */
    void *stream;      /* cudaStream_t for forward and training calls; NULL: the surrogate creates its own */
} qla_surrogate_config;

typedef struct {
    long long calls;            /* surrogate calls attempted */
    long long surrogate_calls;  /* accepted (energy drift within tolerance) */
    long long fallback_calls;   /* replaced by K plain QLA steps */
    double energy_ref;          /* Eq. 27 energy (mean of Q.Q) at the start */
    double energy_final;
    double max_drift;           /* largest drift among accepted calls */
} qla_rollout_stats;

/* Number of FP32 parameters (156422). */
long long qla_surrogate_param_count(void);

/* Create a surrogate on the current device. Errors: QLA_EINVAL, QLA_ENOMEM, QLA_ECUDA. */
qla_status qla_surrogate_create(const qla_surrogate_config *cfg, qla_surrogate **out);

/* He-normal weights from a seed (host splitmix64 + Box-Muller), zero biases,
 * last layer scaled by 0.1; resets the optimiser. Synchronous. */
qla_status qla_surrogate_init_params(qla_surrogate *s, unsigned long long seed);

/* Copy the parameter vector from / to host memory (param_count floats).
 * set_params rejects non-finite values (QLA_EINVAL) and resets the optimiser.
 * Synchronous. */
qla_status qla_surrogate_set_params(qla_surrogate *s, const float *host);
qla_status qla_surrogate_get_params(qla_surrogate *s, float *host);

/* q_out = q_in + s f([q_in, n]) for all nimg images (device pointers; q_out
 * must not alias q_in). Asynchronous on the surrogate's stream. */
qla_status qla_surrogate_forward(qla_surrogate *s, const float *q_in, const float *n, float *q_out);

/* Loss L = sum (s f - (q_target - q_in))^2 / sum (q_target - q_in)^2 over the
 * batch, and its gradient with respect to the parameters (kept on the device
 * for qla_surrogate_adam_step). loss and grad_host (param_count floats) may be
 * NULL; if either is given the call synchronises. Needs train != 0
 * (QLA_ESTATE otherwise); QLA_ETIMEOUT if a tensor-core wait ran out. */
qla_status qla_surrogate_loss_grad(qla_surrogate *s, const float *q_in, const float *n, const float *q_target,
                                   double *loss, float *grad_host);

/* One Adam update (bias-corrected) of the FP32 master weights with the last
 * gradient, then re-packing of the BF16 operands. Asynchronous. */
qla_status qla_surrogate_adam_step(qla_surrogate *s, float lr, float beta1, float beta2, float eps);

/* loss_grad followed by adam_step(lr, 0.9, 0.999, 1e-8). */
qla_status qla_surrogate_train_step(qla_surrogate *s, const float *q_in, const float *n, const float *q_target,
                                    float lr, double *loss);

/* Wait for the surrogate's stream; QLA_ETIMEOUT if a tensor-core wait ran out. */
qla_status qla_surrogate_synchronize(qla_surrogate *s);

/* Energy checks of qla_surrogate_rollout. */
enum {
    QLA_DRIFT_PER_CALL = 0,    /* |E(proposal) / E(state the call starts from) - 1| */
    QLA_DRIFT_FROM_START = 1,  /* |E(proposal) / E_ref - 1|, E_ref fixed for the whole rollout */
    QLA_ROLLOUT_SERIAL = 16    /* flag (OR into drift_mode): no speculative next call (see below) */
};

/* Advance an FP32 QLA context by `calls` x K steps with the network. After each
 * call the energy (Eq. 27, mean of Q.Q) of the proposed state is computed
 * (FP32 squares, FP64 sums: ~1e-6 relative); if it is non-finite or its drift
 * (drift_mode) exceeds drift_tol, the
 * proposal is discarded and K plain QLA steps (qla_step) are taken from the
 * unchanged state instead. With QLA_DRIFT_FROM_START, energy_ref > 0 sets
 * E_ref (e.g. the energy at the start of an earlier rollout segment);
 * otherwise E_ref is measured on the context's state at the start.
 * n: device FP32 [3][Ny][Nx]. The surrogate must have nimg == 1 and the
 * context's lattice, and the context must advance both polarisation families
 * (QLA_EUNSUPPORTED otherwise: the network writes all six components). Runs
 * on the context's stream; synchronous.
 * Speculation: while the host reads a call's energy, the next call's network
 * pass is already running on the proposal (in a third state buffer the
 * surrogate holds), so the GPU does not wait for the host between accepted
 * calls; after a rejection the speculative pass is discarded. The states,
 * decisions and statistics are those of the serial loop, which
 * QLA_ROLLOUT_SERIAL in drift_mode selects (tests compare the two bit for
 * bit). */
qla_status qla_surrogate_rollout(qla_surrogate *s, qla_ctx *ctx, const float *n, int calls, double drift_tol,
                                 int drift_mode, double energy_ref, qla_rollout_stats *stats);

/* Parameter count and tensor-core FLOPs of one forward call (padded channels). */
qla_status qla_surrogate_info(const qla_surrogate *s, long long *nparam, long long *flops_per_call);

const char *qla_surrogate_last_error(const qla_surrogate *s);
void qla_surrogate_destroy(qla_surrogate *s);

#ifdef __cplusplus
}
#endif

#endif /* QLA_SURROGATE_H */
