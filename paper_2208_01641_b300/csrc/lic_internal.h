// Internal declarations of liblic: device data structures, kernel launchers
// and the codec object.  Not part of the public ABI (include/lic.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/lic.h"

namespace lic {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

// Bits of the per-codec device status word (latched by kernels, read and
// cleared by lic_sync).
enum : uint32_t {
    ST_CORRUPT = 1u,   // a bitstream failed a check in the entropy decoder
    ST_TIMEOUT = 2u,   // a bounded wait ran out
};

#define LIC_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            lic::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return _e == cudaErrorMemoryAllocation ? LIC_E_OOM : LIC_E_CUDA; \
        }                                                    \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// ---------------------------------------------------------------------------
// device / pinned buffers, pointer kinds
// ---------------------------------------------------------------------------

// Device bytes allocated through dev_malloc / DevBuf while an AllocScope is
// active on this thread are added to (and bytes freed subtracted from) its
// counter: every public entry point of a codec opens one on the codec's own
// counter, so a codec knows what it holds without asking the device (whose
// free memory other users of the GPU move).
extern thread_local int64_t *g_alloc_sink;
struct AllocScope {
    int64_t *prev;
    explicit AllocScope(int64_t *sink) : prev(g_alloc_sink) { g_alloc_sink = sink; }
    ~AllocScope() { g_alloc_sink = prev; }
    AllocScope(const AllocScope &) = delete;
    AllocScope &operator=(const AllocScope &) = delete;
};
inline cudaError_t dev_malloc(void **p, size_t n) {
    cudaError_t e = cudaMalloc(p, n);
    if (e == cudaSuccess && g_alloc_sink) *g_alloc_sink += (int64_t)n;
    return e;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            cudaFree(p);
            if (g_alloc_sink) *g_alloc_sink -= (int64_t)bytes;
        }
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes) return cudaSuccess;
        release();
        cudaError_t e = dev_malloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

struct HostPinned {
    void *p = nullptr;
    size_t bytes = 0;
    ~HostPinned() { if (p) cudaFreeHost(p); }
    cudaError_t ensure(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocHost(&p, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
};

inline bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// launch counting and optional CUDA-event timing of every launch
// ---------------------------------------------------------------------------

struct Profiler {
    struct Rec {
        std::string name;
        cudaEvent_t a, b;
        double flop, bytes;
        int launches;
    };
    bool on = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    int64_t launches = 0;
    ~Profiler() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
    cudaEvent_t next_event() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void enable(bool en) {
        if (en) {
            recs.clear();
            used = 0;
        }
        on = en;
    }
    // count nlaunch launches made by f(); with recording on, bracket them
    // with an event pair on st
    template <typename F>
    void run(const std::string &name, double flop, double bytes, int nlaunch, cudaStream_t st, F &&f) {
        launches += nlaunch;
        if (!on) {
            f();
            return;
        }
        cudaEvent_t a = next_event(), b = next_event();
        cudaEventRecord(a, st);
        f();
        cudaEventRecord(b, st);
        recs.push_back({name, a, b, flop, bytes, nlaunch});
    }
    // JSON list of {"name", "launches", "ms", "flop", "bytes"} aggregated by
    // name in first-seen order; returns the length or a negative LIC_E_*
    int report(char *buf, int cap) {
        struct Agg {
            int launches = 0;
            double ms = 0, flop = 0, bytes = 0;
        };
        std::vector<std::string> order;
        std::map<std::string, Agg> agg;
        for (auto &r : recs) {
            LIC_CUDA_TRY(cudaEventSynchronize(r.b));
            float ms = 0;
            LIC_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
            if (!agg.count(r.name)) order.push_back(r.name);
            Agg &g = agg[r.name];
            g.launches += r.launches;
            g.ms += ms;
            g.flop += r.flop;
            g.bytes += r.bytes;
        }
        std::string js = "[";
        char tmp[512];
        for (size_t i = 0; i < order.size(); ++i) {
            const Agg &g = agg[order[i]];
            snprintf(tmp, sizeof(tmp),
                     "%s{\"name\": \"%s\", \"launches\": %d, \"ms\": %.6f, \"flop\": %.6e, \"bytes\": %.6e}",
                     i ? ", " : "", order[i].c_str(), g.launches, g.ms, g.flop, g.bytes);
            js += tmp;
        }
        js += "]";
        if (buf && cap > 0) {
            size_t n = std::min((size_t)cap - 1, js.size());
            memcpy(buf, js.data(), n);
            buf[n] = 0;
        }
        return (int)js.size();
    }
};

// ---------------------------------------------------------------------------
// the learned form's student net (student.cu), as the codec uses it
// ---------------------------------------------------------------------------

}  // namespace lic
struct lic_student;
namespace lic {
// the codec's device status word (ST_* bits; api.cu)
uint32_t *codec_status_ptr(lic_codec *cd);
// latent channels M of the student
int student_channels(const lic_student *s);
// NHWC y_hat [B][Hy][Wy][M] -> NHWC [B][16Hy][16Wy][3], stream-ordered
int student_forward_nhwc(lic_student *s, const float *yhat, int B, int Hy, int Wy, float *out, cudaStream_t st);
// per-frame PSNR of clamp(xs) against clamp(xt) over the H x W crop of the
// Hp x Wp NHWC frames; frames with PSNR >= thr get xs copied into xt;
// counts[0] += B, counts[1] += frames below thr.  part: B * 64 doubles.
void launch_student_check(const float *xs, float *xt, int B, int Hp, int Wp, int H, int W, float thr, double *part,
                          float *psnr, int *pass, long long *counts, cudaStream_t st);

// ---------------------------------------------------------------------------
// entropy tables (host build, tables.cpp)
// ---------------------------------------------------------------------------

struct HostTables {
    std::vector<float> medians;     // per entropy-bottleneck channel
    std::vector<int32_t> lo, hi;    // per table
    std::vector<int64_t> start;     // per table, into cdf
    std::vector<uint32_t> cdf;      // concatenated, n+1 entries per table
    int n_eb = 0;                   // tables [0, n_eb) are the bottleneck's
    int n_gauss = 0;                // tables [n_eb, n_eb+64) Gaussian
};

// Build the factorized-bottleneck tables from per-channel parameter blocks
// (58 doubles per channel) and, optionally, the 64 Gaussian tables.
// Returns 0 or a negative LIC_E_* code.
int build_tables(const std::vector<double> &eb_params, int channels, bool gauss, HostTables *out);
void scale_table(float T[64]);

// ---------------------------------------------------------------------------
// conv descriptor shared by the conv kernels
// ---------------------------------------------------------------------------

enum InXform : int { IN_NONE = 0, IN_ABS = 1, IN_SQUARE = 2 };
// EPI_MASK (CUDA-core kernel only): keep the sum where gdn_x (same layout
// as the output) is positive, else 0 -- the ReLU's backward pass.
enum Epi : int { EPI_NONE = 0, EPI_RELU = 1, EPI_GDN = 2, EPI_IGDN = 3, EPI_MASK = 4 };
// Storage of an activation tensor: float32, bf16, or e4m3 holding x / scale.
enum DType : int { DT_F32 = 0, DT_BF16 = 1, DT_E4M3 = 2 };

constexpr int MAX_TAPS = 25;

// One implicit-GEMM convolution over NHWC float32 tensors.
//  GEMM row r = (b, i, j) over a Gh x Gw grid; input pixel of tap t is
//  (s*i + du[t], s*j + dv[t]) of a Hi x Wi input (zero outside); the result
//  goes to output pixel (oym*i + oyo, oxm*j + oxo) of a Ho x Wo output.
//  Weights: [Cout][T][Cin] float32 (K index = t*Cin + c).
struct ConvDesc {
    const float *in;
    float *out;
    const float *w;
    const float *bias;     // [Cout] or null
    const float *gdn_x;    // EPI_GDN/IGDN: x that the norm divides, NHWC with Cout channels
    uint32_t *status;      // device status word (bounded waits that run out set ST_TIMEOUT)
    // GDN / IGDN fused into the epilogue of this convolution (tensor-core
    // kernel only): 0 none, 1 GDN, 2 IGDN; gdn_w is the tc::TcWeights of gamma
    // ([C][1][C]), gdn_beta its beta.
    int fuse_gdn;              // 3: 1DN, 4: inverse 1DN (per-channel, gdn_gamma)
    const float *gdn_beta;
    const void *gdn_w;
    const float *gdn_gamma;
    // precision forms: storage of the input and output activations; e4m3
    // tensors hold x / scale (in_scale, out_scale)
    int in_dt, out_dt;
    float in_scale, out_scale;
    int B, Hi, Wi, Cin;
    int Gh, Gw, s;
    int Ho, Wo, Cout;
    int oym, oyo, oxm, oxo;
    // output row stride in elements (0: Cout) and first output channel, for
    // a launch that computes a column slice of a wider layer (tensor cores)
    int out_stride, out_coff;
    // the output is read once, soon (tensor-core kernels store it evict-first in L2)
    int out_stream;
    // split-K scratch (FP32 tensor-core kernel, Cout = 128, no fused norm): part
    // holds B * part_frame_floats floats; null: no split
    float *part;
    int64_t part_frame_floats;
    // g_a conv0 as a 1x1 GEMM of K = FRAME_K over its (Hp/2) x (Wp/2) output
    // pixels: non-null, the kernel builds each A row from this padded frame
    // [B][Hp][Wp][4] (device, 16-byte aligned, channel 3 zero; see
    // launch_frame_pad4), K index 4 (5u + v) + c, and `in` is not read (the
    // persistent FP32 kernel, Cout = 128, only)
    const float *frame;
    int T;
    int8_t du[MAX_TAPS], dv[MAX_TAPS];
    int in_xform, epi;
    // quantisation fused into the epilogue of a float32 output (tensor-core
    // kernels; launch_conv_simt and the low-precision kernels ignore it):
    // q_mode 1: q_sym[b][c][hw] = rint(fl32(y - q_mu[c])) (q_mu may be null),
    //   saturated to +-2^30, NaN -> 0, and, if q_hat, q_hat (NHWC, q_C
    //   channels) = fl32(s + q_mu[c]); q_mode 2: q_idx[b][c][hw] = the scale
    //   index of y (smallest k with q_tab[k] >= max(y, q_tab[0]), NaN or above
    //   q_tab[63] -> 63; q_tab = the 64 scales in device memory).  c counts
    //   the whole layer's q_C channels (out_coff included); hw the output
    //   pixel within its frame.
    int q_mode;
    int32_t *q_sym;
    float *q_hat;
    const float *q_mu;
    uint8_t *q_idx;
    const float *q_tab;
    int q_C;
};

void launch_conv_simt(const ConvDesc &d, cudaStream_t st);

// Transposed conv 5x5 / stride 2 (pad 2, output padding 1) to at most 4
// output channels, all four sub-pixel phases in one launch (the last layer
// of g_s).  in: NHWC [B][Hi][Wi][Cin] (Cin % 32 == 0); w: [Cin][5][5][4]
// (output channel padded to 4); out: NHWC [B][2Hi][2Wi][Cout].
void launch_deconv_small(const float *in, int B, int Hi, int Wi, int Cin, const float *w, const float *bias,
                         int Cout, float *out, cudaStream_t st);

// The same transposed conv in two passes, the first on the tensor cores: C
// ([B][Hi][Wi][deconv_scatter_stride(Cout)], from a 1x1 GEMM) holds every input
// position's 25 * Cout tap contributions; this sums them into out (NHWC
// [B][2Hi][2Wi][Cout]) and adds the bias.  Each C entry lands in exactly one
// output pixel; the sum order per pixel is fixed.
//
// Column layout: input position (mi, ni) is neighbour (du, dv) in {-1, 0, 1}^2
// of the output quad (2m .. 2m+1, 2n .. 2n+1) with m = mi - du, n = ni - dv,
// and feeds its pixel (2m + py, 2n + px) through tap u = py + 2 - 2du, v = px
// + 2 - 2dv (py < scatter_n(du), px < scatter_n(dv)).  The columns come as nine
// blocks in (du, dv) order, block (du, dv) holding (py, px, o) at (py *
// scatter_n(dv) + px) * Cout + o, each padded to a multiple of 4 floats: the
// second pass reads a quad's contributions as whole 16-byte runs.
__host__ __device__ constexpr int scatter_n(int d) { return d < 0 ? 1 : 2; }
__host__ __device__ constexpr int scatter_block(int du, int dv, int cout) {
    return (scatter_n(du) * scatter_n(dv) * cout + 3) / 4 * 4;
}
__host__ __device__ constexpr int scatter_offset(int du, int dv, int cout) {
    int off = 0;
    for (int a = -1; a <= 1; ++a)
        for (int c = -1; c <= 1; ++c) {
            if (a == du && c == dv) return off;
            off += scatter_block(a, c, cout);
        }
    return off;
}
constexpr int deconv_scatter_stride(int cout) { return scatter_offset(2, 2, cout); }   // all nine blocks
void launch_deconv_gather(const float *C, int B, int Hi, int Wi, int Cout, const float *bias, float *out,
                          cudaStream_t st);

// ---------------------------------------------------------------------------
// elementwise / layout kernels (layout.cu)
// ---------------------------------------------------------------------------

// frames NCHW [B][3][H][W] -> NHWC [B][Hp][Wp][3], replicate padding
void launch_pad_pack(const float *frames, int B, int H, int W, int Hp, int Wp, float *out,
                     cudaStream_t st);
// NHWC [B][Hp][Wp][3] -> NCHW [B][3][H][W], clamped to [0, 1]
void launch_crop_unpack(const float *x, int B, int Hp, int Wp, int H, int W, float *frames,
                        cudaStream_t st);
// generic NHWC <-> NCHW float32 / int32 conversions
void launch_nhwc_to_nchw(const float *in, int B, int H, int W, int C, float *out, cudaStream_t st);
void launch_nchw_to_nhwc(const float *in, int B, int C, int H, int W, float *out, cudaStream_t st);

// s = rint(fl32(y - mu[c])) (mu may be null), saturated to +-2^30, NaN -> 0.
// y NHWC [B][HW][C] -> s NCHW [B][C][HW]; if yhat != null also writes the
// dequantized value fl32(s + mu[c]) in NHWC.
void launch_quantize(const float *y, int B, int HW, int C, const float *mu, int32_t *s,
                     float *yhat, cudaStream_t st);
// idx = smallest k with T[k] >= max(sigma, T[0]); NaN / > T[63] -> 63.
// sigma NHWC [B][HW][C] -> idx NCHW [B][C][HW]; sigma_nchw (optional) copy.
// 1DN / inverse 1DN on NHWC [P][C] float32: out = x * rsqrt(beta + gamma x^2)
// (inverse: * sqrt).
void launch_norm1d(const float *in, int64_t P, int C, const float *beta, const float *gamma, int inverse,
                   float *out, cudaStream_t st);
// float32 -> bf16 (round to nearest even), n elements.
void launch_to_bf16(const float *in, int64_t n, void *out, cudaStream_t st);

// The first layer of g_a as a plain GEMM: NHWC 3-channel [B][Hp][Wp][3] ->
// the rows of its 5x5 / stride-2 patches [B][Hp/2][Wp/2][PATCH_K], K index
// (5u + v) * 3 + c, zero-padded from 75 to PATCH_K.
constexpr int PATCH_K = 96;
// The same layer over the padded frame with 4 channels (ConvDesc::frame): K
// index 4 (5u + v) + c, zero-padded from 100 to FRAME_K.
constexpr int FRAME_K = 128;
// frames [B][3][H][W] (device) -> [B][Hp][Wp][4], replicate-padded as
// launch_pad_pack pads, channel 3 zero.
void launch_frame_pad4(const float *frames, int B, int H, int W, int Hp, int Wp, float *out, cudaStream_t st);
void launch_patch_pack(const float *x, int B, int Hp, int Wp, float *out, cudaStream_t st);
// The same patches straight from the caller's frames [B][3][H][W] (device),
// replicate-padded to Hp x Wp on the fly (as launch_pad_pack pads).
void launch_frame_patch(const float *frames, int B, int H, int W, int Hp, int Wp, float *out, cudaStream_t st);
// Copies the 64 scales into the constant bank of the current device (once
// per device, at codec creation).
cudaError_t upload_scale_table();
void launch_scale_index(const float *sigma, int B, int HW, int C, uint8_t *idx,
                        float *sigma_nchw, cudaStream_t st);

// ---------------------------------------------------------------------------
// entropy coder (rans.cu)
// ---------------------------------------------------------------------------

// Slot lookup: for table t, lut[t * LUT_N + j] (j = 0 .. 256) is the symbol
// whose CDF interval holds slot 256 j (entry 256: the last symbol), so the
// symbol of a slot lies in [lut[slot >> 8], lut[(slot >> 8) + 1]].
constexpr int LUT_N = 257;

struct DevTables {
    const uint32_t *cdf;
    const int64_t *start;
    const int32_t *lo, *hi;
    const uint16_t *lut;
    int n_eb;        // bottleneck tables: table c for channel c
    int gauss_base;  // first Gaussian table (or -1)
    // format 2: the 64 Gaussian tables as the kernels hold them in shared
    // memory (build_gauss_image), copied there with 16-byte loads; null when
    // the codec has no Gaussian tables
    const void *gimg;
};

// The shared-memory image of the 64 Gaussian tables for the format-2
// kernels, in bytes: int32 lo[64], n[64] (symbols incl. the escape), cs[64]
// (first entry of each CDF below), then RANS2_GAUSS_CDF_CAP 16-bit CDF
// entries (each table's n entries, its final 2^16 implied), then the 64
// slot lookups (LUT_N 16-bit entries each).  Multiple of 16 bytes.
constexpr int RANS2_GIMG_HDR = 3 * 64 * 4;

// Geometry of the substreams of one frame (identical for every frame).
struct StreamGeom {
    int kind;
    int N, M;
    int Hy, Wy;      // y latent
    int Hz, Wz;      // z latent (hyperprior)
    int R;           // band rows
    int nbands;
    int nz;          // z substreams per frame (N or 0)
    int nsub;        // substreams per frame
    int H, W, Hp, Wp;
    int64_t header_bytes;  // 36 + 4 (nsub + 1)
    int64_t cap_words;     // scratch words per substream, max over substreams
    // substream format: 1 = escape nibbles inside the rANS words; 2 = escape
    // payloads after them and optional resume records every S groups of 32
    // symbols (decoder-adaptive parallel decoding)
    int version;
    int S;
    // format 2: records per z substream, per full y band, per last y band,
    // and per frame (all substreams); the scratch layout of one substream in
    // 16-bit words: meta (nw, ne, np, nr as u32) at 0, the rANS words
    // right-aligned in [8, 8 + cap_r), then cap_p32 u32 of payload nibbles,
    // cap_c32 u32 of count nibbles and 35 u32 per resume record
    int nr_z, nr_full, nr_last;
    int64_t rec_per_frame;
    int64_t cap_r, cap_p32, cap_c32;
    // worst-case bytes of one frame container
    int64_t frame_cap;
};

StreamGeom make_geom(int kind, int N, int M, int H, int W, int Hp, int Wp, int R, int version = 1, int S = 0);

// Encoder: symbols NCHW (s_y [B][M][Hy][Wy], idx same, s_z [B][N][Hz][Wz])
// -> per substream words in scratch (decoder order, right-aligned) + counts.
void launch_rans_encode(const StreamGeom &g, int B, const DevTables &t, const int32_t *s_y,
                        const uint8_t *idx, const int32_t *s_z, uint16_t *scratch,
                        int64_t *counts, cudaStream_t st);
// Containers: scans, headers and payload copy into data (frames 16-byte
// aligned); offsets [B+1] and sizes [B] on the device.
void launch_rans_compact(const StreamGeom &g, int B, const uint16_t *scratch,
                         const int64_t *counts, int64_t *sub_off, int64_t *frame_bytes,
                         int64_t *offsets, uint8_t *data, cudaStream_t st);

// The per-frame scan of substream lengths (counts, in 16-bit words) into
// offsets and frame sizes (header + 2 * words + trailer_bytes), and the
// frames' 16-byte aligned placement (offsets [B+1], then sizes [B]).
void launch_rans_scan(const StreamGeom &g, int B, const int64_t *counts, int64_t *sub_off, int64_t *frame_bytes,
                      int64_t trailer_bytes, cudaStream_t st);
void launch_frame_place(int B, const int64_t *frame_bytes, int64_t *offsets, cudaStream_t st);

// Entries of the 64 Gaussian CDFs (without each table's final 2^16) that the
// format-2 kernels stage in shared memory; a codec whose tables exceed it
// cannot use format 2.
constexpr int RANS2_GAUSS_CDF_CAP = 27200;
constexpr int RANS2_GIMG_CDF_BYTES = RANS2_GIMG_HDR + 2 * RANS2_GAUSS_CDF_CAP;   // header + CDFs
constexpr int RANS2_GIMG_BYTES = RANS2_GIMG_CDF_BYTES + 2 * 64 * LUT_N;           // + slot lookups
static_assert(RANS2_GIMG_CDF_BYTES % 16 == 0 && RANS2_GIMG_BYTES % 16 == 0, "16-byte copies");
// Host: the image of Gaussian tables [first, first + 64) of ht (with their
// slot lookups lut, LUT_N entries per table); false if they do not fit.
bool build_gauss_image(const HostTables &ht, int first, const std::vector<uint16_t> &lut, std::vector<uint8_t> *img);

// Format 2 (rans2.cu): the same roles as the three calls above, for
// substreams whose escape payloads follow the rANS words (g.version == 2).
// The encoder fills each substream's scratch (layout in StreamGeom) and
// counts[] with the substream's length in words; the compaction writes the
// containers and the resume-record trailer; the decoder runs one warp per
// segment between resume records (one per substream without records).
void launch_rans2_encode(const StreamGeom &g, int B, const DevTables &t, const int32_t *s_y, const uint8_t *idx,
                         const int32_t *s_z, uint16_t *scratch, int64_t *counts, cudaStream_t st);
void launch_rans2_compact(const StreamGeom &g, int B, const uint16_t *scratch, const int64_t *counts,
                          int64_t *sub_off, int64_t *frame_bytes, int64_t *offsets, uint8_t *data, cudaStream_t st);
void launch_rans2_decode(const StreamGeom &g, int B, int part, const DevTables &t, const uint8_t *data,
                         const int64_t *offsets, const int64_t *sizes, const uint8_t *idx, const float *med,
                         int32_t *s_out, float *hat_out, uint32_t *status, cudaStream_t st);

// Either format, by g.version.
void launch_entropy_encode(const StreamGeom &g, int B, const DevTables &t, const int32_t *s_y, const uint8_t *idx,
                           const int32_t *s_z, uint16_t *scratch, int64_t *counts, cudaStream_t st);
void launch_entropy_compact(const StreamGeom &g, int B, const uint16_t *scratch, const int64_t *counts,
                            int64_t *sub_off, int64_t *frame_bytes, int64_t *offsets, uint8_t *data,
                            cudaStream_t st);
void launch_entropy_decode(const StreamGeom &g, int B, int part, const DevTables &t, const uint8_t *data,
                           const int64_t *offsets, const int64_t *sizes, const uint8_t *idx, const float *med,
                           int32_t *s_out, float *hat_out, uint32_t *status, cudaStream_t st);
// Decoder: validates headers, decodes the z substreams (part 0) or the y
// substreams (part 1).  z: s_z NCHW + zhat NHWC (fl32(s + med)).  y: s_y
// NCHW + yhat NHWC (factorized: fl32(s + med); hyperprior: s).
void launch_rans_decode(const StreamGeom &g, int B, int part, const DevTables &t,
                        const uint8_t *data, const int64_t *offsets, const int64_t *sizes,
                        const uint8_t *idx, const float *med, int32_t *s_out, float *hat_out,
                        uint32_t *status, cudaStream_t st);

// Read-only view of a codec's entropy-coding state, for entry points that
// live outside api.cu.
struct CodecEntropyView {
    int kind, N, M, R;
    int version, S;  // substream format and resume-record spacing
    int device;      // the CUDA device the codec (and its tables) lives on
    DevTables tables;
};
int codec_entropy_view(const lic_codec *codec, CodecEntropyView *out);

}  // namespace lic
