/*
 * FP64 CPU reference of the codec chain.  TEST INFRASTRUCTURE ONLY: see
 * oracle.h.  Built with -O2 -ffp-contract=off (no fused multiply-add, no
 * fast-math) so that the table builders follow IEEE double step by step.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Transforms                                                               */
/* ------------------------------------------------------------------------ */

/* Strided convolution; Ballé 2017 [1] g_a uses 5x5 stride 2, the hyper
 * analysis of [2] also 3x3 stride 1.  Zero padding of k/2 on every side. */
void orc_conv2d(const double *x, int B, int Cin, int H, int W,
                const double *w, const double *bias, int Cout, int k, int s,
                double *y)
{
    int p = k / 2;
    int Ho = (H + 2 * p - k) / s + 1, Wo = (W + 2 * p - k) / s + 1;
    for (int b = 0; b < B; b++) {
#pragma omp parallel for schedule(static)
        for (int o = 0; o < Cout; o++) {
            double *yo = y + ((int64_t)b * Cout + o) * Ho * Wo;
            for (int i = 0; i < Ho; i++)
                for (int j = 0; j < Wo; j++) {
                    double acc = bias ? bias[o] : 0.0;
                    for (int c = 0; c < Cin; c++) {
                        const double *xc = x + ((int64_t)b * Cin + c) * H * W;
                        const double *wc = w + ((int64_t)o * Cin + c) * k * k;
                        for (int u = 0; u < k; u++) {
                            int r = s * i + u - p;
                            if (r < 0 || r >= H) continue;
                            for (int v = 0; v < k; v++) {
                                int q = s * j + v - p;
                                if (q < 0 || q >= W) continue;
                                acc += wc[u * k + v] * xc[r * W + q];
                            }
                        }
                    }
                    yo[i * Wo + j] = acc;
                }
        }
    }
}

/* Transposed convolution as the scatter that defines it: every input sample
 * x[a,c] adds w[.,.,u,v]*x[a,c] at output (s*a+u-p, s*c+v-p).  Output
 * padding s-1 makes the output exactly s*H x s*W (the synthesis transforms
 * of [1], [2] mirror the analysis strides). */
void orc_deconv2d(const double *x, int B, int Cin, int H, int W,
                  const double *w, const double *bias, int Cout, int k, int s,
                  double *y)
{
    int p = k / 2;
    int Ho = s * H, Wo = s * W;
    for (int b = 0; b < B; b++) {
#pragma omp parallel for schedule(static)
        for (int o = 0; o < Cout; o++) {
            double *yo = y + ((int64_t)b * Cout + o) * Ho * Wo;
            for (int64_t t = 0; t < (int64_t)Ho * Wo; t++)
                yo[t] = bias ? bias[o] : 0.0;
            for (int c = 0; c < Cin; c++) {
                const double *xc = x + ((int64_t)b * Cin + c) * H * W;
                const double *wc = w + ((int64_t)c * Cout + o) * k * k;
                for (int a = 0; a < H; a++)
                    for (int e = 0; e < W; e++) {
                        double xv = xc[a * W + e];
                        for (int u = 0; u < k; u++) {
                            int r = s * a + u - p;
                            if (r < 0 || r >= Ho) continue;
                            for (int v = 0; v < k; v++) {
                                int q = s * e + v - p;
                                if (q < 0 || q >= Wo) continue;
                                yo[r * Wo + q] += wc[u * k + v] * xv;
                            }
                        }
                    }
            }
        }
    }
}

/* The derivative of the transposed convolution's scatter with respect to
 * each weight: every (input sample, tap) pair that the forward pass added
 * contributes x * g at the same output position. */
void orc_deconv2d_wgrad(const double *x, int B, int Cin, int H, int W, const double *g, int Cout,
                        int k, int s, double *dw)
{
    int p = k / 2;
    int Ho = s * H, Wo = s * W;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Cin; i++)
        for (int o = 0; o < Cout; o++)
            for (int u = 0; u < k; u++)
                for (int v = 0; v < k; v++) {
                    double acc = 0.0;
                    for (int b = 0; b < B; b++) {
                        const double *xi = x + ((int64_t)b * Cin + i) * H * W;
                        const double *go = g + ((int64_t)b * Cout + o) * Ho * Wo;
                        for (int a = 0; a < H; a++) {
                            int r = s * a + u - p;
                            if (r < 0 || r >= Ho) continue;
                            for (int c = 0; c < W; c++) {
                                int q = s * c + v - p;
                                if (q < 0 || q >= Wo) continue;
                                acc += xi[a * W + c] * go[r * Wo + q];
                            }
                        }
                    }
                    dw[(((int64_t)i * Cout + o) * k + u) * k + v] = acc;
                }
}

/* GDN / IGDN, Ballé, Laparra, Simoncelli [9]: a per-pixel divisive
 * normalisation over channels. */
void orc_gdn(double *x, int B, int C, int H, int W,
             const double *beta, const double *gamma, int inverse)
{
    int64_t HW = (int64_t)H * W;
    for (int b = 0; b < B; b++) {
        double *xb = x + (int64_t)b * C * HW;
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < HW; t++) {
            double *v = (double *)malloc(sizeof(double) * C);
            for (int j = 0; j < C; j++) v[j] = xb[j * HW + t];
            for (int i = 0; i < C; i++) {
                double norm = beta[i];
                for (int j = 0; j < C; j++) norm += gamma[i * C + j] * v[j] * v[j];
                double r = sqrt(norm);
                xb[i * HW + t] = inverse ? v[i] * r : v[i] / r;
            }
            free(v);
        }
    }
}

void orc_norm1d(double *x, int B, int C, int H, int W,
                const double *beta, const double *gamma, int inverse)
{
    int64_t HW = (int64_t)H * W;
    for (int b = 0; b < B; b++)
        for (int c = 0; c < C; c++) {
            double *xc = x + ((int64_t)b * C + c) * HW;
            for (int64_t t = 0; t < HW; t++) {
                double r = sqrt(beta[c] + gamma[c] * xc[t] * xc[t]);
                xc[t] = inverse ? xc[t] * r : xc[t] / r;
            }
        }
}

void orc_relu(double *x, int64_t n)
{
    for (int64_t i = 0; i < n; i++) if (x[i] < 0.0) x[i] = 0.0;
}

void orc_abs(double *x, int64_t n)
{
    for (int64_t i = 0; i < n; i++) x[i] = fabs(x[i]);
}

/* ------------------------------------------------------------------------ */
/* Entropy bottleneck (factorized prior): Ballé 2018 [2], appendix 6.1      */
/* ------------------------------------------------------------------------ */

static double softplus(double x)
{
    return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* h_0 = x; h_k = softplus(H_k) h_{k-1} + b_k, plus tanh(a_k)*tanh(h_k) for
 * k < 5; the cumulative is sigmoid(h_5).  Returns h_5 (the logit). */
double orc_eb_logits(const double *p, double x)
{
    static const int f[6] = {1, 3, 3, 3, 3, 1};
    const double *Hm[5], *bv[5], *av[4];
    int off = 0;
    for (int k = 0; k < 5; k++) { Hm[k] = p + off; off += f[k + 1] * f[k]; }
    for (int k = 0; k < 5; k++) { bv[k] = p + off; off += f[k + 1]; }
    for (int k = 0; k < 4; k++) { av[k] = p + off; off += f[k + 1]; }
    double h[3] = {x, 0.0, 0.0};
    for (int k = 0; k < 5; k++) {
        double g[3];
        for (int i = 0; i < f[k + 1]; i++) {
            double acc = 0.0;
            for (int j = 0; j < f[k]; j++) acc += softplus(Hm[k][i * f[k] + j]) * h[j];
            acc += bv[k][i];
            if (k < 4) acc += tanh(av[k][i]) * tanh(acc);
            g[i] = acc;
        }
        for (int i = 0; i < f[k + 1]; i++) h[i] = g[i];
    }
    return h[0];
}

/* Bisection for the point where the logit reaches `target` (the logit is
 * monotone increasing): [-1e6, 1e6], 200 halvings, returns the upper end. */
static double eb_solve(const double *p, double target)
{
    double lo = -1e6, hi = 1e6;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (orc_eb_logits(p, mid) < target) lo = mid; else hi = mid;
    }
    return hi;
}

#define TAIL_MASS 1e-9

int orc_eb_pmf(const double *p, float *median, int *lo, int *hi, double *pm, int cap)
{
    double tq = log((TAIL_MASS / 2) / (1.0 - TAIL_MASS / 2)); /* logit(tau/2) */
    float med = (float)eb_solve(p, 0.0);
    double m = (double)med;
    double qlo = eb_solve(p, tq), qhi = eb_solve(p, -tq);
    double l = ceil(m - qlo), h = ceil(qhi - m);
    if (l < 0) l = 0;
    if (h < 0) h = 0;
    if (l + h + 2 > 4096) return -1;
    int L = (int)l, Hh = (int)h, n = L + Hh + 2;
    if (n > cap) return -1;
    for (int s = -L; s <= Hh; s++) {
        /* likelihood of the unit bin around m+s, with the sign flip that
         * evaluates the difference on the side where the sigmoid is small */
        double lower = orc_eb_logits(p, m + s - 0.5);
        double upper = orc_eb_logits(p, m + s + 0.5);
        double sg = (lower + upper > 0.0) ? -1.0 : 1.0;
        pm[s + L] = fabs(sigmoid(sg * upper) - sigmoid(sg * lower));
    }
    pm[n - 1] = sigmoid(orc_eb_logits(p, m - L - 0.5))
              + sigmoid(-orc_eb_logits(p, m + Hh + 0.5));
    *median = med; *lo = L; *hi = Hh;
    return n;
}

int orc_eb_table(const double *p, float *median, int *lo, int *hi, uint32_t *cdf)
{
    double *pm = (double *)malloc(sizeof(double) * 4096);
    int n = orc_eb_pmf(p, median, lo, hi, pm, 4096);
    int rc = n < 0 ? -1 : orc_quantize_pmf(pm, n, cdf);
    free(pm);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Frequency quantization to a 16-bit CDF                                    */
/* ------------------------------------------------------------------------ */

/* Reading (the paper is silent): f_i = max(1, floor(65536 p_i + 1/2)); a
 * positive deficit goes to the largest f (lowest index on ties); a surplus
 * is taken, min(f_i - 1, rest) at a time, from the symbols in order of
 * decreasing f (ties by increasing index). */
static const uint32_t *g_sort_f;
static int cmp_desc_f(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    if (g_sort_f[i] != g_sort_f[j]) return g_sort_f[i] > g_sort_f[j] ? -1 : 1;
    return i < j ? -1 : (i > j);
}

int orc_quantize_pmf(const double *p, int n, uint32_t *cdf)
{
    if (n < 1 || n > 4096) return -1;
    uint32_t *f = (uint32_t *)malloc(sizeof(uint32_t) * n);
    int64_t sum = 0;
    for (int i = 0; i < n; i++) {
        double q = floor(p[i] * 65536.0 + 0.5);
        f[i] = q < 1.0 ? 1u : (uint32_t)q;
        sum += f[i];
    }
    int64_t D = 65536 - sum;
    if (D > 0) {
        int best = 0;
        for (int i = 1; i < n; i++) if (f[i] > f[best]) best = i;
        f[best] += (uint32_t)D;
    } else if (D < 0) {
        int *ord = (int *)malloc(sizeof(int) * n);
        for (int i = 0; i < n; i++) ord[i] = i;
        g_sort_f = f;
        qsort(ord, n, sizeof(int), cmp_desc_f);
        int64_t rest = -D;
        while (rest > 0) {
            for (int t = 0; t < n && rest > 0; t++) {
                int i = ord[t];
                int64_t take = (int64_t)f[i] - 1;
                if (take > rest) take = rest;
                f[i] -= (uint32_t)take;
                rest -= take;
            }
        }
        free(ord);
    }
    cdf[0] = 0;
    for (int i = 0; i < n; i++) cdf[i + 1] = cdf[i] + f[i];
    free(f);
    return cdf[n] == 65536 ? 0 : -1;
}

/* ------------------------------------------------------------------------ */
/* Gaussian conditional (scale hyperprior [2])                                */
/* ------------------------------------------------------------------------ */

void orc_scale_table(float T[64])
{
    double la = log(0.11), lb = log(256.0);
    for (int k = 0; k < 64; k++)
        T[k] = (float)exp(la + (double)k * (lb - la) / 63.0);
}

/* Standard normal CDF */
static double Phi(double x) { return 0.5 * erfc(-x * M_SQRT1_2); }

/* z with Phi(-z) = tau/2, by bisection on [-40, 0] (200 halvings, upper end). */
double orc_gauss_ztau(void)
{
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (Phi(mid) < TAIL_MASS / 2) lo = mid; else hi = mid;
    }
    return -hi;
}

/* N(0, sigma^2) convolved with U(-1/2, 1/2), on the integers |s| <= c with
 * c = ceil(sigma z_tau); the two tails form the escape symbol. */
int orc_gauss_table(int k, int *cout, uint32_t *cdf)
{
    float T[64];
    orc_scale_table(T);
    double sg = (double)T[k];
    double z = orc_gauss_ztau();
    int c = (int)ceil(sg * z);
    int n = 2 * c + 2;
    if (n > 4096) return -1;
    double *pm = (double *)malloc(sizeof(double) * n);
    for (int s = -c; s <= c; s++) {
        double a = fabs((double)s);
        pm[s + c] = Phi((0.5 - a) / sg) - Phi((-0.5 - a) / sg);
    }
    pm[n - 1] = 2.0 * Phi((-(double)c - 0.5) / sg);
    int rc = orc_quantize_pmf(pm, n, cdf);
    free(pm);
    *cout = c;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Quantization and scale index                                              */
/* ------------------------------------------------------------------------ */

#define SYM_LIMIT 1073741824.0f /* 2^30 */

void orc_quantize(const float *y, int B, int C, int HW, const float *mu, int32_t *s)
{
    for (int b = 0; b < B; b++)
        for (int c = 0; c < C; c++)
            for (int t = 0; t < HW; t++) {
                int64_t i = ((int64_t)b * C + c) * HW + t;
                float d = mu ? y[i] - mu[c] : y[i];   /* float subtraction */
                float r = rintf(d);                    /* ties to even */
                if (r != r) r = 0.0f;
                if (r > SYM_LIMIT) r = SYM_LIMIT;
                if (r < -SYM_LIMIT) r = -SYM_LIMIT;
                s[i] = (int32_t)r;
            }
}

void orc_dequantize(const int32_t *s, int B, int C, int HW, const float *mu, float *yhat)
{
    for (int b = 0; b < B; b++)
        for (int c = 0; c < C; c++)
            for (int t = 0; t < HW; t++) {
                int64_t i = ((int64_t)b * C + c) * HW + t;
                yhat[i] = mu ? (float)s[i] + mu[c] : (float)s[i];
            }
}

void orc_scale_index(const float *sigma, int64_t n, const float T[64], uint8_t *idx)
{
    for (int64_t i = 0; i < n; i++) {
        float v = sigma[i];
        if (v != v) { idx[i] = 63; continue; }
        if (v < T[0]) v = T[0];
        int k = 0;
        while (k < 63 && T[k] < v) k++;   /* linear scan */
        idx[i] = (uint8_t)k;
    }
}

/* ------------------------------------------------------------------------ */
/* rANS: 32-bit state in [2^16, 2^32), 16-bit words, 16-bit probabilities    */
/* ------------------------------------------------------------------------ */

#define RANS_L 65536u

typedef struct {
    uint16_t *w;
    int64_t n, cap;
    int overflow;
} wbuf;

static void put_word(wbuf *b, uint16_t v)
{
    if (b->n >= b->cap) { b->overflow = 1; return; }
    b->w[b->n++] = v;
}

/* Encode (start, f) on state *x: renormalise (at most one word), then
 * x <- floor(x/f)*2^16 + (x mod f) + start. */
static void rans_put(uint32_t *x, uint32_t start, uint32_t f, wbuf *b, int64_t *cnt)
{
    uint64_t xv = *x;
    if (xv >= ((uint64_t)f << 16)) {
        put_word(b, (uint16_t)(xv & 0xFFFF));
        xv >>= 16;
        (*cnt)++;
    }
    xv = (xv / f) * 65536u + (xv % f) + start;
    *x = (uint32_t)xv;
}

/* Symbol mapping: value s in [-lo, hi] -> index s+lo; otherwise the escape
 * index lo+hi+1 with payload v (zigzag of the overflow), sent as a nibble
 * count-1 and then the nibbles, least significant first, each uniform. */
static int nibbles_of(uint32_t v)
{
    int nn = 1;
    while (nn < 8 && (v >> (4 * nn)) != 0) nn++;
    return nn;
}

int orc_rans_encode(const int32_t *s, const int32_t *tab_of, int n,
                    const orc_table *tabs, uint16_t *words, int64_t cap,
                    int64_t *nwords, int64_t lane_words[32], double lane_bits[32])
{
    uint32_t x[32];
    wbuf b = {words, 0, cap, 0};
    for (int l = 0; l < 32; l++) {
        x[l] = RANS_L;
        if (lane_words) lane_words[l] = 0;
        if (lane_bits) lane_bits[l] = 0.0;
    }
    int64_t dummy[32];
    int64_t *lw = lane_words ? lane_words : dummy;
    for (int i = n - 1; i >= 0; i--) {
        int l = i % 32;
        const orc_table *t = &tabs[tab_of[i]];
        int esc = t->lo + t->hi + 1;
        int sym;
        uint32_t v = 0;
        if (s[i] >= -t->lo && s[i] <= t->hi) {
            sym = s[i] + t->lo;
        } else {
            sym = esc;
            if (s[i] > t->hi) v = 2u * (uint32_t)(s[i] - t->hi - 1);
            else v = 2u * (uint32_t)(-s[i] - t->lo - 1) + 1u;
        }
        if (sym == esc) {
            int nn = nibbles_of(v);
            for (int j = nn - 1; j >= 0; j--)
                rans_put(&x[l], 4096u * ((v >> (4 * j)) & 15u), 4096u, &b, &lw[l]);
            rans_put(&x[l], 4096u * (uint32_t)(nn - 1), 4096u, &b, &lw[l]);
            if (lane_bits) lane_bits[l] += 4.0 * (nn + 1);
        }
        uint32_t st = t->cdf[sym], f = t->cdf[sym + 1] - t->cdf[sym];
        rans_put(&x[l], st, f, &b, &lw[l]);
        if (lane_bits) lane_bits[l] += -log2((double)f / 65536.0);
    }
    for (int l = 31; l >= 0; l--) {
        put_word(&b, (uint16_t)(x[l] >> 16));
        put_word(&b, (uint16_t)(x[l] & 0xFFFF));
    }
    if (b.overflow) return -1;
    /* reverse: the decoder reads in the opposite order of emission */
    for (int64_t i = 0, j = b.n - 1; i < j; i++, j--) {
        uint16_t tmp = words[i]; words[i] = words[j]; words[j] = tmp;
    }
    *nwords = b.n;
    return 0;
}

typedef struct {
    const uint16_t *w;
    int64_t n, pos;
    int bad;
} rbuf;

static uint32_t take_word(rbuf *r)
{
    if (r->pos >= r->n) { r->bad = 1; return 0; }
    return r->w[r->pos++];
}

/* Decode one symbol of a 16-bit CDF: the slot x mod 2^16 selects the symbol
 * (cdf[sym] <= slot < cdf[sym+1]); x <- f*(x >> 16) + slot - start; refill
 * one word when x falls below 2^16. */
static int rans_get(uint32_t *x, const uint32_t *cdf, int n, rbuf *r)
{
    uint32_t slot = *x & 0xFFFF;
    int sym = 0;
    while (sym + 1 < n && cdf[sym + 1] <= slot) sym++;  /* linear search */
    uint32_t st = cdf[sym], f = cdf[sym + 1] - cdf[sym];
    uint32_t xv = f * (*x >> 16) + slot - st;
    if (xv < RANS_L) xv = (xv << 16) | take_word(r);
    *x = xv;
    return sym;
}

static uint32_t rans_get_nibble(uint32_t *x, rbuf *r)
{
    uint32_t slot = *x & 0xFFFF;
    uint32_t nib = slot / 4096u;
    uint32_t xv = 4096u * (*x >> 16) + slot - 4096u * nib;
    if (xv < RANS_L) xv = (xv << 16) | take_word(r);
    *x = xv;
    return nib;
}

int orc_rans_decode(const uint16_t *words, int64_t nwords, int n,
                    const int32_t *tab_of, const orc_table *tabs, int32_t *s)
{
    rbuf r = {words, nwords, 0, 0};
    uint32_t x[32];
    for (int l = 0; l < 32; l++) {
        uint32_t lo = take_word(&r);
        uint32_t hi = take_word(&r);
        x[l] = lo | (hi << 16);
    }
    if (r.bad) return -1;
    for (int i = 0; i < n; i++) {
        int l = i % 32;
        const orc_table *t = &tabs[tab_of[i]];
        int esc = t->lo + t->hi + 1;
        int sym = rans_get(&x[l], t->cdf, t->n, &r);
        if (sym < esc) {
            s[i] = sym - t->lo;
        } else {
            uint32_t nn = rans_get_nibble(&x[l], &r) + 1;
            if (nn > 8) return -1;
            uint32_t v = 0;
            for (uint32_t j = 0; j < nn; j++) v |= rans_get_nibble(&x[l], &r) << (4 * j);
            int64_t val = (v & 1u) ? -(int64_t)t->lo - 1 - (int64_t)(v >> 1)
                                   : (int64_t)t->hi + 1 + (int64_t)(v >> 1);
            if (val > 1073741824LL || val < -1073741824LL) return -1;
            s[i] = (int32_t)val;
        }
        if (r.bad) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* rANS substreams, format 2: escape payloads outside the rANS words and     */
/* optional resume records (the decoder-adaptive form)                       */
/* ------------------------------------------------------------------------ */

/* Substream layout (16-bit words, little endian), L words in all:
 *   w[0], w[1]          nw, the number of rANS words (low half first)
 *   w[2 .. 2+nw)        the rANS words exactly as format 1 would order them
 *                       (32 initial states, then renormalisation words in
 *                       symbol order), except that an escape is the escape
 *                       symbol alone: its payload is not in this section
 *   payload nibbles     from w[2+nw] on: escape k's n_k nibbles of v (the
 *                       zigzag overflow, least significant first) at nibble
 *                       positions Q_k .. Q_k+n_k-1, Q_k = sum of n_i, i < k;
 *                       nibble j sits in word j/4 at bits 4 (j mod 4)
 *   count nibbles       from the last word backwards: n_k - 1 for escape k is
 *                       nibble k, in word L-1-k/4 at bits 4 (k mod 4)
 *   with 2 + nw + ceil(np/4) + ceil(ne/4) = L (ne escapes, np payload nibbles).
 * Resume record for group G (symbols 32G .. 32G+31), 35 u32: the index P of
 * the next rANS word at the start of group G (relative to w[2]), the escapes
 * E and payload nibbles Q before group G, and the 32 lane states then.  With
 * spacing S > 0 there is one record for each G = S, 2S, ... below the group
 * count. */

static void put_nibble(uint16_t *base, int64_t j, uint32_t v)
{
    base[j >> 2] = (uint16_t)(base[j >> 2] | ((v & 15u) << (4 * (j & 3))));
}

static uint32_t get_nibble(const uint16_t *base, int64_t j)
{
    return ((uint32_t)base[j >> 2] >> (4 * (j & 3))) & 15u;
}

int orc_rans2_encode(const int32_t *s, const int32_t *tab_of, int n, const orc_table *tabs, int S,
                     uint16_t *out, int64_t cap, int64_t *len, uint32_t *rec, int64_t rec_cap,
                     int64_t *nrec, int64_t lane_words[32], double lane_bits[32])
{
    int ngroups = (n + 31) / 32;
    int64_t nr = (S > 0 && ngroups > 0) ? (ngroups - 1) / S : 0;
    if (nr * 35 > rec_cap) return -1;
    /* symbols, escapes and their payloads in symbol order */
    int *sym = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    uint32_t *pay = (uint32_t *)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    int *nib = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    int64_t ne = 0, np = 0;
    for (int i = 0; i < n; i++) {
        const orc_table *t = &tabs[tab_of[i]];
        nib[i] = 0;
        if (s[i] >= -t->lo && s[i] <= t->hi) {
            sym[i] = s[i] + t->lo;
        } else {
            sym[i] = t->lo + t->hi + 1;
            pay[i] = s[i] > t->hi ? 2u * (uint32_t)(s[i] - t->hi - 1) : 2u * (uint32_t)(-s[i] - t->lo - 1) + 1u;
            nib[i] = nibbles_of(pay[i]);
            ne++;
            np += nib[i];
        }
    }
    /* the rANS words: symbols from last to first, state i mod 32; records
     * keep each lane's state after its group G was encoded */
    uint16_t *tmp = (uint16_t *)malloc(sizeof(uint16_t) * ((int64_t)n + 64));
    wbuf b = {tmp, 0, (int64_t)n + 64, 0};
    uint32_t x[32];
    int64_t dummy[32];
    int64_t *lw = lane_words ? lane_words : dummy;
    for (int l = 0; l < 32; l++) {
        x[l] = RANS_L;
        lw[l] = 0;
        if (lane_bits) lane_bits[l] = 0.0;
    }
    int64_t esc_after = 0, nib_after = 0;   /* escapes / nibbles in the groups encoded so far */
    for (int i = n - 1; i >= 0; i--) {
        int l = i % 32;
        const orc_table *t = &tabs[tab_of[i]];
        uint32_t st = t->cdf[sym[i]], f = t->cdf[sym[i] + 1] - t->cdf[sym[i]];
        rans_put(&x[l], st, f, &b, &lw[l]);
        if (lane_bits) lane_bits[l] += -log2((double)f / 65536.0) + (nib[i] ? 4.0 * (nib[i] + 1) : 0.0);
        if (nib[i]) {
            esc_after++;
            nib_after += nib[i];
        }
        if (l == 0 && S > 0 && i / 32 > 0 && (i / 32) % S == 0) {
            int64_t r = (i / 32) / S - 1;   /* record of group G = i / 32 */
            uint32_t *R = rec + 35 * r;
            R[0] = (uint32_t)b.n;           /* words emitted for groups >= G; made relative below */
            R[1] = (uint32_t)(ne - esc_after);
            R[2] = (uint32_t)(np - nib_after);
            for (int k = 0; k < 32; k++) R[3 + k] = x[k];
        }
    }
    for (int l = 31; l >= 0; l--) {
        put_word(&b, (uint16_t)(x[l] >> 16));
        put_word(&b, (uint16_t)(x[l] & 0xFFFF));
    }
    int64_t nw = b.n;
    int64_t L = 2 + nw + (np + 3) / 4 + (ne + 3) / 4;
    int rc = 0;
    if (b.overflow || L > cap) {
        rc = -1;
    } else {
        memset(out, 0, sizeof(uint16_t) * L);
        out[0] = (uint16_t)(nw & 0xFFFF);
        out[1] = (uint16_t)(nw >> 16);
        for (int64_t k = 0; k < nw; k++) out[2 + k] = tmp[nw - 1 - k];   /* decoder order */
        uint16_t *pw = out + 2 + nw;
        int64_t q = 0, e = 0;
        for (int i = 0; i < n; i++) {
            if (!nib[i]) continue;
            for (int j = 0; j < nib[i]; j++) put_nibble(pw, q++, pay[i] >> (4 * j));
            /* count nibbles grow from the last word backwards */
            out[L - 1 - (e >> 2)] = (uint16_t)(out[L - 1 - (e >> 2)] | ((uint32_t)(nib[i] - 1) << (4 * (e & 3))));
            e++;
        }
        for (int64_t r = 0; r < nr; r++) rec[35 * r] = (uint32_t)(nw - rec[35 * r]);   /* P: words before G */
        *len = L;
        *nrec = nr;
    }
    free(tmp);
    free(sym);
    free(pay);
    free(nib);
    return rc;
}

/* Decode groups [g0, g1) of a format-2 substream of n symbols.  rec = NULL
 * starts at group 0 from the stream's initial states; otherwise from that
 * record (g0 is its group).  Every read is bounded; returns 0, or -1 for a
 * stream this coder cannot have written.  When the decode reaches the last
 * symbol, the section sizes must add up to the substream length exactly. */
int orc_rans2_decode_range(const uint16_t *w, int64_t L, int n, const int32_t *tab_of, const orc_table *tabs,
                           const uint32_t *rec, int g0, int g1, int32_t *s)
{
    if (L < 2) return -1;
    int64_t nw = (int64_t)w[0] | ((int64_t)w[1] << 16);
    if (nw < 64 || 2 + nw > L) return -1;
    rbuf r = {w + 2, nw, 0, 0};
    uint32_t x[32];
    int64_t e = 0, q = 0;
    if (!rec) {
        if (g0 != 0) return -1;
        for (int l = 0; l < 32; l++) {
            uint32_t lo = take_word(&r);
            uint32_t hi = take_word(&r);
            x[l] = lo | (hi << 16);
        }
    } else {
        r.pos = rec[0];
        e = rec[1];
        q = rec[2];
        for (int l = 0; l < 32; l++) x[l] = rec[3 + l];
        if (r.pos < 64 || r.pos > nw) return -1;
    }
    if (r.bad) return -1;
    const uint16_t *pw = w + 2 + nw;
    int64_t wa = L - 2 - nw;   /* words after the rANS section: payload, then counts from the end */
    int i_end = 32 * g1 < n ? 32 * g1 : n;
    for (int i = 32 * g0; i < i_end; i++) {
        int l = i % 32;
        const orc_table *t = &tabs[tab_of[i]];
        int esc = t->lo + t->hi + 1;
        int sym = rans_get(&x[l], t->cdf, t->n, &r);
        if (r.bad) return -1;
        if (sym < esc) {
            s[i] = sym - t->lo;
            continue;
        }
        /* count nibble e from the end, then its payload nibbles from q on */
        if (e / 4 >= wa) return -1;
        uint32_t nn = ((uint32_t)w[L - 1 - e / 4] >> (4 * (e % 4)) & 15u) + 1;
        e++;
        if ((q + (int64_t)nn - 1) / 4 >= wa) return -1;
        uint32_t v = 0;
        for (uint32_t j = 0; j < nn; j++) v |= get_nibble(pw, q + j) << (4 * j);
        q += nn;
        int64_t val = (v & 1u) ? -(int64_t)t->lo - 1 - (int64_t)(v >> 1) : (int64_t)t->hi + 1 + (int64_t)(v >> 1);
        if (val > 1073741824LL || val < -1073741824LL) return -1;
        s[i] = (int32_t)val;
    }
    if (i_end == n && (r.pos != nw || 2 + nw + (q + 3) / 4 + (e + 3) / 4 != L)) return -1;
    return 0;
}
