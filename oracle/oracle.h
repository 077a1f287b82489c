/*
 * FP64 CPU reference ("oracle") of the learned-image-codec chain that
 * arXiv 2208.01641 pipelines (factorized prior [1], scale hyperprior [2]).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this code; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * Every routine is the plain definition, written out loop by loop in double
 * precision; no blocking, fusion or reordering.  The paper itself prints no
 * equations (Sec. III names x, y, y_hat, z, g_a, g_s, h_a, h_s only), so each
 * function names the published definition it restates and the reading taken
 * where those are silent.
 *
 * Layout: all images are NCHW, row-major, double.
 */
#ifndef LIC_ORACLE_H
#define LIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- transforms (Sec. III-A/B: g_a, g_s, h_a, h_s) ---- */

/* Zero-padded 2-D convolution (cross-correlation), pad = k/2, stride s.
 * y[b,o,i,j] = bias[o] + sum_{c,u,v} w[o,c,u,v] * x[b,c, s*i+u-k/2, s*j+v-k/2]
 * x: B x Cin x H x W; w: Cout x Cin x k x k; y: B x Cout x ceil(H/s) x ceil(W/s). */
void orc_conv2d(const double *x, int B, int Cin, int H, int W,
                const double *w, const double *bias, int Cout, int k, int s,
                double *y);

/* Transposed convolution, kernel k, stride s, pad k/2, output padding s-1
 * (output size s*H x s*W):
 * y[b,o, s*a+u-k/2, s*c+v-k/2] += w[i,o,u,v] * x[b,i,a,c]  (+ bias[o])
 * x: B x Cin x H x W; w: Cin x Cout x k x k. */
void orc_deconv2d(const double *x, int B, int Cin, int H, int W,
                  const double *w, const double *bias, int Cout, int k, int s,
                  double *y);

/* Weight gradient of the transposed convolution orc_deconv2d (same k, s,
 * pad k/2): dw[i,o,u,v] = sum_{b,a,c} x[b,i,a,c] * g[b,o, s*a+u-k/2, s*c+v-k/2]
 * over output positions inside the s*H x s*W output.  x: B x Cin x H x W,
 * g: B x Cout x sH x sW, dw: Cin x Cout x k x k (overwritten). */
void orc_deconv2d_wgrad(const double *x, int B, int Cin, int H, int W, const double *g, int Cout,
                        int k, int s, double *dw);

/* GDN (Ballé et al. [9]) in place, per pixel:
 *   inverse == 0: x_i <- x_i / sqrt(beta_i + sum_j gamma[i,j] x_j^2)
 *   inverse == 1: x_i <- x_i * sqrt(beta_i + sum_j gamma[i,j] x_j^2)   (IGDN) */
void orc_gdn(double *x, int B, int C, int H, int W,
             const double *beta, const double *gamma, int inverse);

/* 1DN (the paper's variant C, ref. [6]), read as GDN without channel mixing,
 * in place, per element: x_i <- x_i / sqrt(beta_i + gamma_i x_i^2), or
 * x_i * sqrt(.) when inverse.  gamma has C entries. */
void orc_norm1d(double *x, int B, int C, int H, int W,
                const double *beta, const double *gamma, int inverse);

void orc_relu(double *x, int64_t n);
void orc_abs(double *x, int64_t n);

/* ---- entropy models ---- */

/* Factorized entropy bottleneck, Ballé 2018 [2] appendix 6.1: per channel a
 * cumulative c(x) = sigmoid(h5(x)) of a 1-3-3-3-3-1 monotone net.
 * Per-channel parameter block, ORC_EB_PARAMS doubles, in this order:
 *   H0[3x1] H1[3x3] H2[3x3] H3[3x3] H4[1x3]   (row-major, out x in)
 *   b0[3] b1[3] b2[3] b3[3] b4[1]
 *   a0[3] a1[3] a2[3] a3[3]                                               */
#define ORC_EB_PARAMS 58
double orc_eb_logits(const double *p, double x);

/* A probability table for one symbol alphabet: support [-lo, hi] plus an
 * escape symbol at index lo+hi+1; cdf has n+1 entries, n = lo+hi+2. */
typedef struct {
    int lo, hi, n;
    uint32_t *cdf; /* owned by the caller of the builder */
} orc_table;

/* Quantized 16-bit CDF from a pmf over n symbols (escape last). */
int orc_quantize_pmf(const double *p, int n, uint32_t *cdf);

/* Median (float), tails and likelihoods of one channel of the entropy
 * bottleneck before frequency quantization: pm[s + lo] = c(m+s+1/2) -
 * c(m+s-1/2) for s in [-lo, hi], and pm[lo+hi+1] = c(m-lo-1/2) + 1 -
 * c(m+hi+1/2), the escape mass of both tails.  cap = capacity of pm.
 * Returns n = lo+hi+2, or -1 (support above 4096 symbols, or above cap). */
int orc_eb_pmf(const double *p, float *median, int *lo, int *hi, double *pm, int cap);

/* Median (float) and tails of channel c of the entropy bottleneck, and its
 * quantized table.  cdf must hold 4097 entries.  Returns 0 or -1 if the
 * support exceeds 4096 symbols. */
int orc_eb_table(const double *p, float *median, int *lo, int *hi, uint32_t *cdf);

/* The 64 scales of the Gaussian conditional, log-spaced 0.11 .. 256. */
void orc_scale_table(float T[64]);
/* Gaussian table k (zero mean, scale T[k]); cdf must hold 4097 entries. */
int orc_gauss_table(int k, int *c, uint32_t *cdf);
double orc_gauss_ztau(void);

/* ---- quantization and scale index ---- */

/* s = rint(fl32(y - mu)) saturated to +-2^30; NaN -> 0. mu may be NULL (0). */
void orc_quantize(const float *y, int B, int C, int HW, const float *mu, int32_t *s);
/* y_hat = fl32(s + mu) (mu NULL: y_hat = s). */
void orc_dequantize(const int32_t *s, int B, int C, int HW, const float *mu, float *yhat);
/* idx = smallest k with T[k] >= max(sigma, T[0]); sigma > T[63] or NaN -> 63. */
void orc_scale_index(const float *sigma, int64_t n, const float T[64], uint8_t *idx);

/* ---- interleaved rANS (Duda 2013, Giesen 2014 interleaving) ---- */

/* Encode n symbols of one substream with 32 interleaved states.
 * tab_of[i] selects tabs[] for symbol i.  Writes the stream (decoder order)
 * into words[0..*nwords).  cap = capacity of words.  Returns 0 or -1. */
int orc_rans_encode(const int32_t *s, const int32_t *tab_of, int n,
                    const orc_table *tabs, uint16_t *words, int64_t cap,
                    int64_t *nwords, int64_t lane_words[32], double lane_bits[32]);

/* Decode n symbols; reads at most nwords words.  Returns 0 or -1 (corrupt). */
int orc_rans_decode(const uint16_t *words, int64_t nwords, int n,
                    const int32_t *tab_of, const orc_table *tabs, int32_t *s);

/* ---- format 2: escape payloads outside the rANS words, resume records ---- */

/* Encode n symbols into one format-2 substream (layout in oracle.c) of
 * *len words (cap = capacity of out), and, with S > 0, its resume records
 * (35 u32 each, rec_cap u32 of room) every S groups of 32 symbols.  The
 * lane statistics are as for orc_rans_encode (escape nibbles counted as
 * bits of their lane).  Returns 0 or -1. */
int orc_rans2_encode(const int32_t *s, const int32_t *tab_of, int n, const orc_table *tabs, int S,
                     uint16_t *out, int64_t cap, int64_t *len, uint32_t *rec, int64_t rec_cap,
                     int64_t *nrec, int64_t lane_words[32], double lane_bits[32]);

/* Decode groups [g0, g1) of a format-2 substream of L words: from its
 * initial states (rec NULL, g0 = 0) or from the resume record of group g0.
 * Returns 0 or -1 (corrupt). */
int orc_rans2_decode_range(const uint16_t *w, int64_t L, int n, const int32_t *tab_of, const orc_table *tabs,
                           const uint32_t *rec, int g0, int g1, int32_t *s);

#ifdef __cplusplus
}
#endif
#endif
