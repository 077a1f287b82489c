/*
 * lic.h -- C ABI of the B300 learned-image-codec library (liblic.so).
 *
 * The library runs the encode/decode chain of the two learned image codecs
 * that arXiv 2208.01641 pipelines -- the factorized prior (Ballé et al. 2017,
 * the paper's [1]) and the scale hyperprior (Ballé et al. 2018, [2]) -- on one
 * GPU (Sec. III-A, III-B and Fig. 1 of the paper):
 *
 *   encoder:  x -> g_a -> y -> Q -> rANS            (factorized, Sec. III-A)
 *             y -> h_a -> z -> Q -> rANS,  z_hat -> h_s -> scales -> index
 *                                                   (hyperprior, Sec. III-B)
 *   decoder:  rANS^-1 -> Q^-1 -> g_s -> x_hat       (hyperprior: z first, then
 *             h_s -> scales -> index, then y: the 4-stage order of Sec. III-B)
 *
 * Every step runs in the library's own CUDA kernels for sm_103a; there is no
 * CPU fallback.  The paper's CPU-thread pipeline, zero-copy and pooling are
 * replaced by an all-device chain (see the design notes).
 *
 * Conventions
 *  - Return value: LIC_OK (0) or a negative LIC_E_* code.  No exception or
 *    abort crosses this boundary.
 *  - Streams: `stream` is a cudaStream_t passed as void*.  Calls are
 *    stream-ordered and return once the work is enqueued, except where a
 *    host buffer must be filled (stated per call).
 *  - Errors found by kernels (corrupt bitstream, bounded waits that ran out)
 *    are latched in a per-codec device status word; lic_sync() waits for the
 *    stream and returns (and clears) the latched status.
 *  - Frames are float32, NCHW (B x 3 x H x W), values in [0, 1].  A frame
 *    pointer may be device memory or host memory (pinned or pageable); the
 *    library detects which and stages host memory through its own device
 *    buffers.
 *  - Stage tensors exchanged by the diagnostic calls are NCHW as well.
 *  - Thread safety: one codec must not be used by two host threads at once.
 */
#ifndef LIC_H
#define LIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LIC_OK 0
#define LIC_E_INVALID_ARG (-1)
#define LIC_E_UNSUPPORTED (-2)
#define LIC_E_OOM (-3)
#define LIC_E_CORRUPT_STREAM (-4)
#define LIC_E_TIMEOUT (-5)
#define LIC_E_CUDA (-6)
#define LIC_E_BUSY (-7)   /* too many requests / batches outstanding */

typedef enum { LIC_FACTORIZED = 0, LIC_HYPERPRIOR = 1 } lic_kind;
/* LIC_FP32: every step float32-accurate (tensor-core convs in 3xTF32).
 * LIC_BF16: the precision form -- the convolutions of g_a and g_s take bf16
 * activations and weights with float32 accumulation; GDN / IGDN norms, h_a,
 * h_s, the scales and the scale index stay float32, so encoder and decoder
 * derive identical indices. */
/* LIC_FP8: as LIC_BF16, with e4m3 activations (stored as x * 16, saturating)
 * and e4m3 weights scaled per output channel wherever a layer has a multiple
 * of 128 input channels (the 192-channel input of g_s stays bf16). */
typedef enum { LIC_FP32 = 0, LIC_BF16 = 1, LIC_FP8 = 2 } lic_precision;

/* Convolution implementation: LIC_CONV_AUTO picks the tcgen05 tensor-core
 * kernels where they exist and the CUDA-core (SIMT) kernels elsewhere;
 * LIC_CONV_SIMT forces the CUDA-core kernels everywhere. */
typedef enum { LIC_CONV_AUTO = 0, LIC_CONV_SIMT = 1 } lic_conv_impl;

/* One named host float32 parameter tensor.  Names and shapes:
 *   g_a.conv{0..3}.{weight [Cout,Cin,5,5], bias [Cout]}     3->N->N->N->M
 *   g_a.gdn{0..2}.{beta [N], gamma [N,N]}
 *   g_s.deconv{0..3}.{weight [Cin,Cout,5,5], bias [Cout]}   M->N->N->N->3
 *   g_s.igdn{0..2}.{beta [N], gamma [N,N]}
 *   hyperprior only:
 *   h_a.conv0 [N,M,3,3], h_a.conv1 [N,N,5,5], h_a.conv2 [N,N,5,5] (+ .bias)
 *   h_s.deconv0 [N,N,5,5], h_s.deconv1 [N,N,5,5] (transposed-conv layout),
 *   h_s.conv2 [M,N,3,3] (+ .bias)
 *   entropy bottleneck over C channels (C = M factorized, N hyperprior):
 *   eb.H0 [C,3,1] eb.H1..H3 [C,3,3] eb.H4 [C,1,3], eb.b0..b3 [C,3],
 *   eb.b4 [C,1], eb.a0..a3 [C,3]   (Ballé 2018 appendix 6.1)            */
typedef struct {
    const char *name;
    const float *data;   /* host memory; copied by lic_codec_create */
    int64_t numel;
} lic_param;

typedef struct {
    const lic_param *params;
    int count;
} lic_weights;

typedef struct {
    int precision;   /* lic_precision (LIC_BF16 needs the tensor-core kernels) */
    int band_rows;   /* latent rows per y substream; 0 -> 16 (a value >= the
                        latent height makes each y plane one substream) */
    int conv_impl;   /* lic_conv_impl */
    int norm;        /* lic_norm: the normalisation between the g_a / g_s layers */
    int format;      /* lic_format: the substream format; 0 -> LIC_FORMAT_1 */
    int resume_groups; /* LIC_FORMAT_2: a resume record every this many groups
                        of 32 symbols of a substream (0: none) */
    int reserved[2]; /* 0 */
} lic_options;

/* Substream formats (the container's version field; the paper integrates
 * CompressAI's coder and defines none).  Both code the same symbols with the
 * same 32 interleaved rANS states per substream.
 * LIC_FORMAT_1: an escape's payload is coded as uniform 4-bit rANS symbols
 *   after it, inside the interleaved words.
 * LIC_FORMAT_2: the escape symbol alone is rANS-coded; payload nibbles follow
 *   the rANS words and count nibbles grow from the substream's end, so a
 *   decoder resolves all escapes of a group of 32 at once (the
 *   decoder-adaptive, higher-throughput coder the paper names as future
 *   work, Sec. VII).  With resume_groups = S > 0 the encoder also writes, in
 *   a trailer after the substreams, a resume record every S groups (the next
 *   word's position, escape and payload positions, the 32 lane states); a
 *   decoder set up with the same S decodes the segments between records in
 *   parallel, any other decoder of the format (or one given a stream whose
 *   records were stripped, lic_strip_resume_records) decodes each substream
 *   from its start.  A codec encodes and decodes its own format only. */
typedef enum { LIC_FORMAT_1 = 1, LIC_FORMAT_2 = 2 } lic_format;

/* LIC_NORM_GDN: GDN / IGDN of Ballé et al. (the paper's [9]), gamma [C,C].
 * LIC_NORM_1DN: the cheaper activation of the paper's variant C (Sec. IV-C,
 * its ref. [6]), read as GDN without channel mixing:
 * y_i = x_i / sqrt(beta_i + gamma_i x_i^2) (inverse: x_i * sqrt(.)), with
 * per-channel gamma [C] under the same parameter names. */
typedef enum { LIC_NORM_GDN = 0, LIC_NORM_1DN = 1 } lic_norm;

typedef struct lic_codec lic_codec;

/* A batch of frame bitstreams laid out back to back -- the strings the
 * paper's encoder hands to its decoder (Sec. III-B: the z string, then the
 * y string, per frame).  Frame i occupies bytes [offsets[i], offsets[i] +
 * sizes[i]) of `data`.  Each frame is one self-describing container (magic
 * "LIC1", see the design notes):
 *   'LIC1' u16 version (1 or 2, the lic_format), u16 kind, u16 N, u16 M,
 *   u32 H, u32 W, u32 Hp, u32 Wp, u16 R, u16 S (format 2: resume-record
 *   spacing, else 0), u32 nsub, u32 off[nsub+1] (16-bit word offsets),
 *   u16 payload[off[nsub]], then (format 2, S > 0) the resume records, 140
 *   bytes each                                           (little endian)
 * A batch made by lic_encode is library-owned (owner != NULL) and stays
 * valid until lic_bitstreams_release; a batch a caller assembles from its
 * own memory has owner = NULL and is never touched by the library beyond
 * the call it is passed to.  Every frame of a batch has the same size. */
typedef struct {
    int count;                 /* frames */
    int on_device;             /* 1: data and d_offsets are device pointers */
    const uint8_t *data;       /* containers back to back */
    const int64_t *offsets;    /* host, count+1 byte offsets (sizes are
                                  offsets[i+1]-offsets[i] minus alignment
                                  padding: use sizes[]) */
    const int64_t *sizes;      /* host, count sizes in bytes */
    const int64_t *d_offsets;  /* device copy of offsets (on_device only) */
    const int64_t *d_sizes;    /* device copy of sizes (on_device only) */
    int H, W;                  /* original frame size of every frame; 0, 0:
                                  lic_decode reads it from frame 0's header */
    void *owner;               /* library batch this view belongs to, or NULL */
} lic_bitstreams;

/* ---------------------------------------------------------------------- */
/* Codec lifetime                                                          */
/* ---------------------------------------------------------------------- */

/* Create a codec of `kind` with N transform channels and M latent channels
 * on the current CUDA device -- the factorized-prior codec of the paper's
 * [1] (Sec. III-A, the "factorized" rows of Tables 2-4) or the scale
 * hyperprior of [2] (Sec. III-B, the "hyper" rows).  The weights are
 * validated (every name above present with the right numel), copied,
 * re-laid-out for the kernels, and the entropy-model CDF tables are built
 * once on the host in FP64 (the factorized entropy bottleneck of [2] app.
 * 6.1 and the 64-scale Gaussian conditional of [2]) and uploaded.  opts may
 * be NULL (defaults).  *out is owned by the caller (lic_codec_destroy).
 * Errors: INVALID_ARG (bad kind/N/M/weights), UNSUPPORTED (table support
 * above 4096 symbols, N or M not a multiple of 32, N > 256), OOM, CUDA. */
int lic_codec_create(int kind, int N, int M, const lic_weights *weights,
                     const lic_options *opts, lic_codec **out);

/* Free every device and host resource of the codec (synchronizes the
 * device first), including every bitstream batch it still owns.  NULL is
 * accepted. */
void lic_codec_destroy(lic_codec *codec);

/* Wait for `stream`, then return and clear the status latched by kernels
 * since the previous lic_sync: LIC_OK, LIC_E_CORRUPT_STREAM or
 * LIC_E_TIMEOUT (or LIC_E_CUDA if the stream itself failed).  (No
 * counterpart in the paper, whose stages report nothing back.) */
int lic_sync(lic_codec *codec, void *stream);

/* ---------------------------------------------------------------------- */
/* Encode / decode                                                         */
/* ---------------------------------------------------------------------- */

/* Encode B frames (B x 3 x H x W float32, device or host memory): the
 * encoder of the paper's Fig. 1 / Sec. III-A (x -> g_a -> y -> Q -> rANS)
 * and, for the hyperprior, Sec. III-B (y -> h_a -> z -> Q -> rANS, z_hat ->
 * h_s -> scales -> index).  The frames are replicate-padded on the
 * bottom/right to multiples of 64 internally.  On return *out describes a
 * library-owned batch: data, d_offsets and d_sizes on the device (valid in
 * stream order), offsets and sizes on the host (pinned; valid once the
 * stream has synchronized), H and W, and the owner handle.  The batch stays
 * valid until lic_bitstreams_release (or lic_codec_destroy), whatever is
 * encoded meanwhile; released batches' buffers are pooled and reused by
 * later encodes (the paper's memory pooling, Sec. III-D).  At most 64
 * batches may be unreleased at once.  Errors: INVALID_ARG (B < 1, H or W <
 * 1, null pointers), BUSY (64 batches unreleased), OOM, CUDA. */
int lic_encode(lic_codec *codec, const float *frames, int B, int H, int W,
               lic_bitstreams *out, void *stream);

/* Return a batch made by lic_encode or lic_encode_latents to the codec's
 * pool and clear *bs (owner = NULL, count = 0).  The buffers may be
 * overwritten by the next encode on this codec, on any stream: release a
 * batch once every call that reads it has been enqueued on the stream the
 * next encode will use, or has completed.  Host-only, never waits.  Errors:
 * INVALID_ARG (not a live batch of this codec; releasing twice is an
 * error, and a cleared struct is accepted as a no-op). */
int lic_bitstreams_release(lic_codec *codec, lic_bitstreams *bs);

/* Decode in->count frames into `frames` (count x 3 x H x W float32, device
 * or host memory; a host destination makes the call wait for the stream):
 * the decoder of Sec. III-B in the order of its 4-stage pipeline -- z
 * first, then h_s -> scales -> index, then y, then g_s (Fig. 1) -- or, for
 * the factorized codec, rANS^-1 -> Q^-1 -> g_s (Sec. III-A).  H x W is the
 * batch's frame size: in->H, in->W, or, when those are 0, frame 0's header
 * (a device-resident batch then costs one small synchronous copy).  in may
 * live on the device (on_device = 1, e.g. the output of lic_encode) or on
 * the host.  Headers are validated on the device against (kind, N, M, H,
 * W); a mismatch or a corrupt substream is latched as LIC_E_CORRUPT_STREAM
 * (read it with lic_sync) and the frames of a corrupt stream are left
 * unspecified.  The entropy decoder bounds every read; a corrupt stream
 * never faults the device.  Errors: INVALID_ARG (null pointers, count < 1),
 * CORRUPT_STREAM returned at once (nothing launched) when H, W are taken
 * from a frame-0 header that is not a valid container header, OOM, CUDA. */
int lic_decode(lic_codec *codec, const lic_bitstreams *in, float *frames, void *stream);

/* Copy a device-resident batch (in->on_device = 1, e.g. from lic_encode)
 * to host memory after waiting for `stream` (the strings leave the GPU, as
 * the paper's encoder sends them, Sec. III-B and V-B): bytes [0, offsets[count]) of
 * in->data, so frame i starts at dst + offsets[i] and is sizes[i] bytes.
 * dst_cap is the capacity of dst.  Returns the bytes copied (>= 0) or
 * INVALID_ARG (capacity too small, not a device batch) / CUDA. */
int64_t lic_bitstreams_download(const lic_bitstreams *in, uint8_t *dst, int64_t dst_cap,
                                void *stream);

/* Parse the header of one host-resident frame container: original size
 * and kind (the project's container; the paper defines no format).
 * Returns INVALID_ARG / CORRUPT_STREAM on a bad header. */
int lic_decoded_shape(const uint8_t *frame, int64_t size, int *kind, int *H, int *W);

/* Host-only: copy one format-2 frame container without its resume records
 * (the trailer dropped and the header's record spacing set to 0): what a
 * sender transmits to a decoder that will not use them.  A frame without
 * records is copied unchanged.  out may equal frame.  *out_size receives the
 * new size; out_cap is out's capacity (the input size suffices).  Errors:
 * INVALID_ARG (null pointers, capacity), CORRUPT_STREAM (not a container of
 * either format, or a size that does not match its header). */
int lic_strip_resume_records(const uint8_t *frame, int64_t size, uint8_t *out, int64_t out_cap,
                             int64_t *out_size);

/* ---------------------------------------------------------------------- */
/* Stage-level calls (tests, diagnostics, custom pipelines)                */
/* All tensors NCHW; device or host memory unless stated.                  */
/* ---------------------------------------------------------------------- */

/* Intermediate tensors of the most recent lic_encode / lic_decode. */
typedef enum {
    LIC_T_Y = 0,      /* float32 B x M x Hp/16 x Wp/16, encoder latent y    */
    LIC_T_SY = 1,     /* int32, quantized y symbols (encoder or decoder)    */
    LIC_T_Z = 2,      /* float32 B x N x Hp/64 x Wp/64, hyper latent z      */
    LIC_T_SZ = 3,     /* int32, quantized z symbols                         */
    LIC_T_SIGMA = 4,  /* float32 B x M x Hp/16 x Wp/16, h_s scales          */
    LIC_T_IDX = 5,    /* uint8, scale-table index                           */
    LIC_T_XPRE = 6,   /* float32 B x 3 x Hp x Wp, decoder output before
                         clamp and crop                                     */
    LIC_T_YHAT = 7    /* float32 B x M x Hp/16 x Wp/16, the decoder's
                         dequantized y_hat (g_s input; after lic_decode or
                         lic_decode_latents)                                */
} lic_tensor;

/* Copy intermediate `which` of the last call into dst (NCHW); `count`
 * receives the element count (dst may be NULL to query it).  Errors:
 * INVALID_ARG if the tensor does not exist for this codec/last call. */
int lic_read_tensor(lic_codec *codec, int which, void *dst, int64_t *count,
                    void *stream);

/* y = g_a(pad(frames)): B x M x Hp/16 x Wp/16 float32 (the analysis
 * transform of [1], Sec. III-A).  Errors: INVALID_ARG, OOM, CUDA. */
int lic_analysis(lic_codec *codec, const float *frames, int B, int H, int W,
                 float *y, void *stream);
/* x = g_s(y_hat), unclamped: B x 3 x 16Hy x 16Wy float32 (the synthesis
 * transform of [1], Sec. III-A; the student replaces it when one is set).
 * Errors: INVALID_ARG, OOM, CUDA. */
int lic_synthesis(lic_codec *codec, const float *yhat, int B, int Hy, int Wy,
                  float *x, void *stream);
/* z = h_a(y) (hyperprior): B x N x Hy/4 x Wy/4 (the hyper analysis of
 * [2], Sec. III-B).  Errors: INVALID_ARG (factorized codec), OOM, CUDA. */
int lic_hyper_analysis(lic_codec *codec, const float *y, int B, int Hy, int Wy,
                       float *z, void *stream);
/* sigma = h_s(z_hat) and idx = scale index of sigma (hyperprior):
 * B x M x 4Hz x 4Wz float32 and uint8 (idx may be NULL) -- the hyper
 * synthesis of [2] that both encoder and decoder run (Sec. III-B), and the
 * index into the 64-scale Gaussian table.  Errors: INVALID_ARG, OOM, CUDA. */
int lic_hyper_synthesis(lic_codec *codec, const float *zhat, int B, int Hz, int Wz,
                        float *sigma, uint8_t *idx, void *stream);

/* Entropy-code given integer symbols (device int32/uint8, NCHW) into frame
 * containers, exactly as lic_encode does after quantization (the rANS
 * stage of Sec. III-A/B, which the paper runs on CPU threads): s_y is
 * B x M x Hy x Wy; idx (hyperprior) the same shape; s_z (hyperprior)
 * B x N x Hy/4 x Wy/4.  H, W are the original frame size recorded in the
 * headers (Hp = 16 Hy, Wp = 16 Wy).  Output, ownership and errors as for
 * lic_encode; INVALID_ARG also for a symbol pointer not in device memory. */
int lic_encode_latents(lic_codec *codec, const int32_t *s_y, const uint8_t *idx,
                       const int32_t *s_z, int B, int H, int W, int Hy, int Wy,
                       lic_bitstreams *out, void *stream);

/* Working memory of lic_encode_latents_noalloc: a fixed array compiled into
 * the library, present on every device that loads it until the process
 * exits. */
#define LIC_NOALLOC_SCRATCH_BYTES (32ll << 20)

/* lic_encode_latents without any allocation (the paper has no counterpart:
 * it is an interface for callers that cannot allocate device memory when
 * they encode -- a real-time thread that must not stall in cudaMalloc or
 * cudaFree, which wait on the device; a host that gives all device memory
 * to its own fixed-budget allocator; a plugin handed buffers by its host).
 * Produces the same frame containers as lic_encode_latents, byte for byte,
 * from the same inputs (device pointers, NCHW, as there).  Outputs are the
 * caller's device buffers:
 *   data      containers, frame i at byte d_layout[i]; data_cap bytes, at
 *             least B * (36 + 4 (nsub+1) + 2 nsub c + 16) (the worst case for
 *             escapes in every symbol; nsub substreams per frame, n_max
 *             symbols in the longest; c = 10 n_max + 64 words in format 1,
 *             8 + 2 ceil((n_max + 64) / 2) + 2 (n_max + 1 + n_max / 8 + 1 +
 *             35 r) in format 2 with r = its records per substream plus 1,
 *             0 without records), else INVALID_ARG;
 *   d_layout  2B+1 int64: byte offsets of the frames [0..B] followed by
 *             their sizes [B+1..2B].
 * Working memory comes from one array of LIC_NOALLOC_SCRATCH_BYTES inside
 * the library; a batch needing more (about 2 nsub (10 n_max + 64) B bytes)
 * returns UNSUPPORTED before anything is launched.  The call allocates
 * nothing and calls no allocating routine.  Its first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All
 * calls share the one array and it keeps the previous call's contents
 * (none of which a call reads), so calls whose work overlaps on the GPU --
 * on two streams, or from two host threads -- race and corrupt each other:
 * order them on one stream or synchronize between them.  Stream-ordered;
 * returns once the work is enqueued. */
int lic_encode_latents_noalloc(lic_codec *codec, const int32_t *s_y, const uint8_t *idx,
                               const int32_t *s_z, int B, int H, int W, int Hy, int Wy,
                               uint8_t *data, int64_t data_cap, int64_t *d_layout,
                               void *stream);

/* Entropy-decode the symbols of in->count frames (device int32 outputs,
 * NCHW; s_z ignored for the factorized codec); the frame size comes from in
 * as for lic_decode.  The hyperprior path runs h_s on the decoded z to
 * obtain the indices of y, as the decoder must (stages 1-3 of the 4-stage
 * decoder, Sec. III-B).  Errors as for lic_decode. */
int lic_decode_latents(lic_codec *codec, const lic_bitstreams *in,
                       int32_t *s_y, int32_t *s_z, void *stream);

/* ---------------------------------------------------------------------- */
/* Host-only: entropy-model tables (no GPU needed)                         */
/* ---------------------------------------------------------------------- */

/* Build the quantized 16-bit CDF tables exactly as lic_codec_create does
 * (the entropy models of [2]: app. 6.1 for the bottleneck, Sec. 3 for the
 * Gaussian conditional; the paper's codecs use them through CompressAI).
 * Factorized entropy bottleneck over C channels from the eb.* parameters
 * (pass weights with the eb.* entries; C from eb.H0's numel / 3), then, if
 * gauss != 0, the 64 Gaussian tables.  Table t has support [-lo[t], hi[t]]
 * plus an escape symbol; its cdf occupies cdf[start[t] .. start[t]+n[t]]
 * (n[t]+1 entries, n[t] = lo[t]+hi[t]+2).  medians[c] is the float32 median
 * of channel c.  Capacities: tables <= max_tables, cdf entries <= cdf_cap.
 * Returns the number of tables written (>= 0) or a negative LIC_E_*. */
int lic_build_tables(const lic_weights *weights, int gauss, int max_tables,
                     int64_t cdf_cap, float *medians, int32_t *lo, int32_t *hi,
                     int64_t *start, uint32_t *cdf);

/* The 64 scales of the Gaussian conditional (0.11 .. 256, log-spaced; the
 * scale table of [2] as the hyperprior codec of Sec. III-B indexes it). */
void lic_scale_table(float T[64]);

/* ---------------------------------------------------------------------- */
/* Measurement                                                             */
/* ---------------------------------------------------------------------- */

/* Measurement hooks (no counterpart in the paper; they time the chain the
 * way its Tables 2-4 report fps, per stage).
 * enable = 1: start recording a CUDA event pair around every kernel launch
 * the codec issues (on the stream it is given), discarding earlier records;
 * enable = 0: stop recording.  Recording adds a small gap between launches,
 * and the sub-pixel phases of a transposed convolution, which otherwise run
 * side by side on auxiliary streams, run one after another so that each
 * record times one launch; time the chain without it. */
int lic_profile_enable(lic_codec *codec, int enable);

/* Write the records as JSON into buf: a list of {"name", "launches", "ms",
 * "flop", "bytes"} aggregated by launch name, where flop and bytes are the
 * algorithmic work of those launches (2 x multiply-adds of the definition;
 * bytes of the inputs read once, outputs written once and weights).  Waits
 * for the recorded events.  Returns the string length (excluding the
 * terminator; buf may be NULL to query it) or a negative code. */
int lic_profile_report(lic_codec *codec, char *buf, int cap);

/* Kernel launches issued by this codec since it was created. */
int64_t lic_launch_count(lic_codec *codec);

/* Device memory the codec holds now, in bytes: weights, tables, grow-only
 * workspaces and pooled bitstream batches, counted at each allocation the
 * codec makes (not from the device's free memory, which other users of the
 * GPU move).  Returns the byte count or INVALID_ARG. */
int64_t lic_codec_device_bytes(const lic_codec *codec);

/* Device memory, in bytes, that lic_encode + lic_decode of B frames of
 * H x W (device frames, no student) make the codec's workspaces and one
 * bitstream batch reach, computed from the geometry without allocating
 * (the weights and tables, already held, are not included).  For
 * admission decisions before a workload is first run.  Returns the byte
 * count or INVALID_ARG. */
int64_t lic_codec_workspace_bytes(const lic_codec *codec, int B, int H, int W);

/* The dense rate of the current device's tensor pipe, measured (no
 * counterpart in the paper; the roofline context of the convolution
 * kernels): every SM issues `iters` (1 .. 1e6) tcgen05 MMAs of M = 128,
 * N = 256 back to back into one tensor-memory accumulator, operands resident
 * in shared memory; kind 0 = tf32 (K = 8 per MMA), 1 = bf16 (K = 16), 2 =
 * e4m3 (K = 32).  *tflops = 2 M N K iters SMs / the launch's CUDA-event
 * time.  Allocates a 4-byte status word and a stream, synchronizes.  Errors:
 * INVALID_ARG, TIMEOUT (a bounded wait ran out), CUDA. */
int lic_probe_mma_rate(int kind, int iters, double *tflops);

/* Diagnostics of the failure path (no counterpart in the paper): one GPU
 * thread waits, through the same
 * bounded wait the tensor-core pipelines use, on a barrier that nothing
 * arrives at; after limit_cycles (1 .. 4e9 SM clock cycles) it gives up and
 * latches the codec's timeout status, so the next lic_sync returns
 * LIC_E_TIMEOUT (and clears it) while the context stays usable.  No hang,
 * no fault.  Stream-ordered. */
int lic_test_bounded_wait(lic_codec *codec, int64_t limit_cycles, void *stream);

/* Human-readable message for an error code. */
const char *lic_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LIC_H */
