/* Learned time-stepping surrogate for the QLA: BF16 tensor-core convolution
 * building blocks (tcgen05, FP32 accumulation in tensor memory).
 *
 * The surrogate advances the fields of the 2D anisotropic-dielectric scattering
 * problem (Sec. 4) by K QLA steps per call: Q_{t+K} = Q_t + s * f([Q_t, n]).
 * The paper has no learned component; the network only approximates the map
 * that the QLA step (Eq. 28) iterated K times defines, and plain QLA stays its
 * fallback and the judge of its error and energy (Eq. 27).
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
    QLA_EPI_GELU = 0,    /* z = acc + b; out0 = BF16(z); out1 = BF16(GELU(z) + aux0) (aux0: BF16 residual or NULL) */
    QLA_EPI_LINEAR = 1,  /* out0 = FP32 (acc + b), [H][W][nout] */
    QLA_EPI_DGRAD = 2,   /* g = acc + aux0 (FP32 [H][W][nout] or NULL); out0 = g (FP32); out1 = BF16(g * GELU'(zprev)) */
    QLA_EPI_QUPDATE = 3  /* out0[c][y][x] = aux0[c][y][x] + scale * (acc + b)[c], c < 6 (FP32 planes [6][H][W]) */
};

/* One 3x3 circular convolution as an implicit GEMM on the tensor cores.
 * x: BF16 [H][W][cin]; w_packed: BF16 [9][cin/8][nout][8] (qla_pack_conv_weights);
 * bias: FP32 [nout] or NULL (ignored by QLA_EPI_DGRAD); GELU is the tanh form.
 * Supported (cin, nout): (16, 64), (64, 64), (64, 16); W a multiple of 128.
 * error_flag: device int set to 1 if the kernel's bounded wait for its tensor
 * core work ran out (the outputs are then invalid); the caller zeroes it.
 * Errors: QLA_EINVAL (NULL pointer, bad size or epilogue operands),
 * QLA_EUNSUPPORTED (channel pair), QLA_ECUDA (launch failure). */
qla_status qla_conv3x3_bf16(const void *x, int H, int W, int cin, const void *w_packed, const float *bias, int nout,
                            int epilogue, const void *aux0, const void *zprev, void *out0, void *out1, float scale,
                            int *error_flag, void *stream);

/* Pack FP32 weights w[nout][cin][3][3] (device) into the BF16 B-operand layout
 * [9][cin_pad/8][nout_pad][8], zero-padded. transpose_flip != 0 packs the
 * adjoint (input-gradient) convolution instead, w'[c][n][ky][kx] =
 * w[n][c][2-ky][2-kx], whose output channels are w's inputs (then cin <=
 * nout_pad and nout <= cin_pad). Errors: QLA_EINVAL. */
qla_status qla_pack_conv_weights(const float *w, int nout, int cin, int nout_pad, int cin_pad, int transpose_flip,
                                 void *packed, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QLA_SURROGATE_H */
