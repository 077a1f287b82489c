/*
 * lic_student.h -- the learned form: a distilled student synthesis net that
 * the decoder can run in place of g_s (liblic.so, same library as lic.h).
 *
 * The paper's decoder is g_s of the factorized / hyperprior codec
 * (Sec. III-A, III-B, Fig. 1), four transposed convolutions with IGDN
 * between them; the decoder side is its heavier half (Sec. V).  The student
 * keeps the interface of g_s -- y_hat (M channels at 1/16 resolution) in,
 * the 3-channel reconstruction out -- and replaces it with four transposed
 * convolutions 5x5 / stride 2 (pad 2, output padding 1),
 *     M -> C -> C -> C -> 3, ReLU after the first three, no IGDN,
 * trained by mean squared error against the teacher's g_s output on random
 * crops, with Adam (Kingma & Ba 2015, Algorithm 1).  The paper trains no
 * network; the student is a form built on its decoder, not one of its
 * results.
 *
 * Every step -- the crop gather, the forward pass, the loss, the backward
 * pass (input gradient = the strided convolution with the same weights,
 * masked by the ReLU; weight gradient = a reduction over batch x pixels;
 * bias gradient = a per-channel sum) and the Adam update -- runs in the
 * library's CUDA kernels, float32, with fixed reduction orders (results do
 * not depend on the launch).  The LIC_BF16 form stores the 64-channel
 * layers' activations and output gradients in bf16 and runs their forward
 * pass, input gradients and weight gradients on tcgen05 (bf16 x bf16 ->
 * float32 sums).  Conventions (return codes, streams, NCHW) are those of
 * lic.h.
 */
#ifndef LIC_STUDENT_H
#define LIC_STUDENT_H

#include <stdint.h>

#include "lic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lic_student lic_student;

/* Largest number of crops in one training batch. */
#define LIC_STUDENT_MAX_BATCH 64

typedef struct {
    int precision;   /* LIC_FP32, or LIC_BF16 (C = 64, M a multiple of 64): bf16 tensor-core form */
    int max_batch;   /* crops per training step, 1 .. LIC_STUDENT_MAX_BATCH */
    int crop;        /* crop side in output pixels, a multiple of 16, >= 32 */
    float lr, beta1, beta2, eps;   /* Adam hyper-parameters */
    int halo;        /* latent rows/columns of context around each crop, 0 .. 8 */
    int reserved[3];               /* must be 0 */
} lic_student_options;

/* Create a student with M latent channels and C hidden channels from the
 * host float32 parameters `init` (copied):
 *   student.deconv{0..3}.weight [Cin, Cout, 5, 5] (transposed-conv layout),
 *   student.deconv{0..3}.bias   [Cout],    channels M -> C -> C -> C -> 3.
 * C and M must be multiples of 16.  Adam moments start at zero, step 0.
 * Returns LIC_E_INVALID_ARG for a missing or mis-sized tensor or bad
 * options, LIC_E_OOM when device memory runs out. */
int lic_student_create(const lic_weights *init, int M, int C, const lic_student_options *opt, lic_student **out);
void lic_student_destroy(lic_student *student);

/* Loss and gradients of one training batch, without an update.
 * yhat_pool: device NCHW [P, M, Hy, Wy]; xhat_pool: device NCHW
 * [P, 3, 16 Hy, 16 Wy], the teacher's g_s output for that pool (both
 * caller-owned, read only).  crops: host int32 [B, 3] of (frame, row, col)
 * in latent units.  Crop b runs the student on the L-square latent window
 * at (row, col) of frame `frame`, L = crop/16 + 2 halo, and compares the
 * central crop-square of its output with the target window at
 * (16 (row + halo), 16 (col + halo)): with halo > 0 the student sees the
 * latents around the crop that the teacher's output there depends on.
 * Every window must lie inside the pool (else LIC_E_INVALID_ARG, nothing
 * launched).  B <= max_batch.  The loss is mean((student(y) - x)^2) over
 * the B x 3 x crop x crop target values; when `loss` is non-null the call
 * waits for the stream and writes it there (host float). */
int lic_student_grad(lic_student *student, const float *yhat_pool, const float *xhat_pool, int P, int Hy, int Wy,
                     const int32_t *crops, int B, float *loss, void *stream);

/* lic_student_grad, then one Adam step of every parameter (t += 1):
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
int lic_student_step(lic_student *student, const float *yhat_pool, const float *xhat_pool, int P, int Hy, int Wy,
                     const int32_t *crops, int B, float *loss, void *stream);

/* What lic_student_read copies. */
typedef enum {
    LIC_STUDENT_PARAM = 0,   /* current weights / biases */
    LIC_STUDENT_GRAD = 1,    /* gradients of the last lic_student_grad/step */
    LIC_STUDENT_ADAM_M = 2,  /* Adam first moment */
    LIC_STUDENT_ADAM_V = 3   /* Adam second moment */
} lic_student_what;

/* Copy the named tensor (names as in lic_student_create) to the host
 * float32 buffer `dst` of `numel` elements (must equal the tensor's size).
 * Synchronous (waits for the device). */
int lic_student_read(lic_student *student, const char *name, int what, float *dst, int64_t numel);

/* Diagnostics: the post-ReLU activation h_layer (layer 1..3) of the last
 * lic_student_grad/step batch, NHWC [B, 16 L/2^(4-layer), same, C] float32,
 * copied to the host buffer dst of numel elements (must equal that size for
 * the batch's B).  layer 0 is the gathered y_hat window, NHWC [B, L, L, M].
 * Values stored in bf16 (the BF16 form) are widened exactly.  Synchronous. */
int lic_student_read_activation(lic_student *student, int layer, float *dst, int64_t numel);

/* Diagnostics: dz_layer (layer 0..3), the loss gradient with respect to the
 * pre-activation output of transposed conv `layer` in the last batch (the
 * backward pass of the chain rule above), NHWC [B, 16 L/2^(3-layer), same,
 * Cout] float32, as stored (bf16 values widened exactly), into dst of numel
 * elements (must equal that size).  Synchronous. */
int lic_student_read_output_grad(lic_student *student, int layer, float *dst, int64_t numel);

/* Adam steps taken so far, or a negative LIC_E_*. */
int64_t lic_student_steps(const lic_student *student);

/* Inference: y_hat NCHW [B, M, Hy, Wy] (device or host) -> the student's
 * reconstruction NCHW [B, 3, 16 Hy, 16 Wy] (device or host), before the
 * [0, 1] clamp.  Stream-ordered for device buffers. */
int lic_student_forward(lic_student *student, const float *yhat, int B, int Hy, int Wy, float *x, void *stream);

/* Measurement, as lic_profile_enable / lic_profile_report /
 * lic_launch_count of lic.h, for the launches the student issues (training
 * and inference, also when a codec runs it). */
int lic_student_profile_enable(lic_student *student, int enable);
int lic_student_profile_report(lic_student *student, char *buf, int cap);
int64_t lic_student_launch_count(const lic_student *student);

/* Decode with the student in place of g_s.  `student` NULL restores g_s.
 * The student must have the codec's M.  The codec keeps a reference; the
 * student must outlive its use by the codec.
 * checked = 0: lic_decode and lic_synthesis run the student only.
 * checked = 1: lic_decode runs both nets, measures each frame's PSNR of the
 *   student's clamped, cropped output against the teacher's, and returns the
 *   student's frame where that PSNR >= min_psnr_db, the teacher's frame
 *   (the fallback) otherwise; lic_synthesis runs the student only. */
int lic_codec_set_student(lic_codec *codec, lic_student *student, float min_psnr_db, int checked);

/* Statistics of checked decoding since lic_codec_set_student: frames
 * checked and frames that fell back to the teacher (either may be NULL);
 * and the per-frame PSNR (dB) of the last checked lic_decode into
 * `last_psnr` (up to `cap` values; NULL to skip).  Waits for the device.
 * Returns the number of frames of the last checked decode (>= 0). */
int lic_codec_student_report(lic_codec *codec, int64_t *frames, int64_t *fallbacks, float *last_psnr, int cap);

#ifdef __cplusplus
}
#endif

#endif /* LIC_STUDENT_H */
