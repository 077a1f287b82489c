// Layout, quantization and scale-index kernels (all HBM-bound, elementwise).
//
//  * pad/pack: the codec input is replicate-padded on the bottom/right to
//    multiples of 64 (the four stride-2 stages of g_a and two of h_a) and
//    turned from NCHW into the NHWC layout of the conv kernels.
//  * crop/unpack: clamp the reconstruction to [0, 1], crop, back to NCHW.
//  * quantize (Sec. III-A: "quantization of y with a channel-wise mean"):
//    s = rint(fl32(y - mu_c)), round half to even, in float32.
//  * scale index (the Gaussian conditional of [2]): the smallest of the 64
//    table scales that is >= max(sigma, 0.11).
#include <cuda_bf16.h>

#include "lic_internal.h"

namespace lic {
namespace {

__constant__ float c_scales[64];

__global__ void pad_pack_kernel(const float *__restrict__ f, int B, int H, int W, int Hp, int Wp,
                                float *__restrict__ out) {
    int64_t n = (int64_t)B * Hp * Wp;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(p % Wp);
        int y = (int)((p / Wp) % Hp);
        int b = (int)(p / ((int64_t)Wp * Hp));
        int ys = min(y, H - 1), xs = min(x, W - 1);
        const float *src = f + (int64_t)b * 3 * H * W + (int64_t)ys * W + xs;
        out[p * 3 + 0] = src[0];
        out[p * 3 + 1] = src[(int64_t)H * W];
        out[p * 3 + 2] = src[2 * (int64_t)H * W];
    }
}

// frames [B][3][H][W] -> [B][Hp][Wp][4] (channel 3 zero), replicate-padded:
// one thread per pixel, three plane reads and one 16-byte store, both
// coalesced across the warp
__global__ void frame_pad4_kernel(const float *__restrict__ f, int B, int H, int W, int Hp, int Wp,
                                  float4 *__restrict__ out) {
    const int64_t n = (int64_t)B * Hp * Wp, HW = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % Wp);
        const int y = (int)((p / Wp) % Hp);
        const int64_t b = p / ((int64_t)Wp * Hp);
        const float *src = f + b * 3 * HW + (int64_t)min(y, H - 1) * W + min(x, W - 1);
        out[p] = make_float4(__ldg(src), __ldg(src + HW), __ldg(src + 2 * HW), 0.f);
    }
}

// Patches of a 5x5 / stride-2 convolution of a 3-channel Hp x Wp image:
// row (b, i, j) of the output holds, at K index k = (5u + v) * 3 + c, the
// input value x[b][2i + u - 2][2j + v - 2][c] (0 outside the image), and 0
// for k >= 75.  A block makes PP_COLS consecutive rows of one output image
// row: it stages the 5 input rows they read (zero-filled outside the
// image) in shared memory, then writes the rows as contiguous float4s.
// PLANAR: x is the caller's frames [B][3][H][W], replicate-padded to Hp x Wp
// on the fly (the padded value at (y, x) is frame[min(y, H-1)][min(x, W-1)]);
// otherwise x is the padded NHWC image [B][Hp][Wp][3].
constexpr int PP_COLS = 64, PP_T = 240;   // 10 rows x 24 float4 columns per pass
constexpr int PP_IN_COLS = 2 * PP_COLS + 3;   // input columns 2 j0 - 2 .. 2 j0 + 2 PP_COLS

template <bool PLANAR>
__global__ void __launch_bounds__(PP_T) patch_pack_kernel(const float *__restrict__ x, int H, int W, int Hp, int Wp,
                                                          float *__restrict__ out) {
    __shared__ float tile[5][PP_IN_COLS * 3];
    const int Ho = Hp / 2, Wo = Wp / 2;
    const int j0 = blockIdx.x * PP_COLS, i = blockIdx.y, b = blockIdx.z;
    for (int e = threadIdx.x; e < 5 * PP_IN_COLS * 3; e += PP_T) {
        if (PLANAR) {   // consecutive threads read consecutive columns of one plane
            const int r = e / (PP_IN_COLS * 3), c = (e / PP_IN_COLS) % 3, col = e % PP_IN_COLS;
            const int y = 2 * i - 2 + r, xx = 2 * j0 - 2 + col;
            tile[r][col * 3 + c] = (y >= 0 && y < Hp && xx >= 0 && xx < Wp)
                                       ? x[(((int64_t)b * 3 + c) * H + min(y, H - 1)) * W + min(xx, W - 1)]
                                       : 0.f;
        } else {
            const int r = e / (PP_IN_COLS * 3), rem = e % (PP_IN_COLS * 3);
            const int y = 2 * i - 2 + r, xx = 2 * j0 - 2 + rem / 3;
            tile[r][rem] = (y >= 0 && y < Hp && xx >= 0 && xx < Wp)
                               ? x[(((int64_t)b * Hp + y) * Wp + xx) * 3 + rem % 3]
                               : 0.f;
        }
    }
    __syncthreads();
    const int cols = min(PP_COLS, Wo - j0);
    float4 *dst = reinterpret_cast<float4 *>(out + (((int64_t)b * Ho + i) * Wo + j0) * PATCH_K);
    // this thread's four K indices, fixed: their offsets in the tile (output column 0)
    constexpr int Q = PATCH_K / 4;
    const int q = threadIdx.x % Q, r0 = threadIdx.x / Q;
    int off[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int k = 4 * q + m, t = k / 3, c = k % 3;
        off[m] = k < 75 ? (t / 5) * (PP_IN_COLS * 3) + (t % 5) * 3 + c : -1;
    }
    const float *tf = &tile[0][0];
    for (int jr = r0; jr < cols; jr += PP_T / Q) {
        float v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = off[m] >= 0 ? tf[off[m] + 6 * jr] : 0.f;
        dst[jr * Q + q] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

__global__ void crop_unpack_kernel(const float *__restrict__ x, int B, int Hp, int Wp, int H, int W,
                                   float *__restrict__ f) {
    // one thread per pixel: its 3 channels are one 12-byte read, and each
    // channel plane is written coalesced across the warp
    const int64_t n = (int64_t)B * H * W, HW = (int64_t)H * W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(e % W);
        const int yy = (int)((e / W) % H);
        const int64_t b = e / HW;
        const float *src = x + ((b * Hp + yy) * Wp + xx) * 3;
        float *dst = f + b * 3 * HW + (int64_t)yy * W + xx;
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[c * HW] = fminf(fmaxf(src[c], 0.f), 1.f);
    }
}

// 32 x 32 tiled transposes between [B][P][C] (NHWC, P = H*W) and [B][C][P].
template <typename Fn>
__device__ __forceinline__ void tile_nhwc_to_nchw(int B, int P, int C, Fn fn) {
    // blockIdx.x: tile of P, blockIdx.y: tile of C, blockIdx.z: batch; 32x8 threads
    __shared__ float tile[32][33];
    (void)B;
    int b = blockIdx.z;
    int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    float v[4];   // the four loads in flight together, then the shared stores
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = p0 + threadIdx.y + 8 * k, c = c0 + threadIdx.x;
        fn.load(b, p, c, p < P && c < C, v[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) tile[threadIdx.y + 8 * k][threadIdx.x] = v[k];
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        int c = c0 + r, p = p0 + threadIdx.x;
        if (c < C && p < P) fn.store(b, p, c, tile[threadIdx.x][r]);
    }
}

struct CopyF {
    const float *in;
    float *out;
    int P, C;
    __device__ void load(int b, int p, int c, bool ok, float &v) const {
        v = ok ? in[((int64_t)b * P + p) * C + c] : 0.f;
    }
    __device__ void store(int b, int p, int c, float v) const { out[((int64_t)b * C + c) * P + p] = v; }
};

__global__ void nhwc_to_nchw_kernel(CopyF fn, int B) { tile_nhwc_to_nchw(B, fn.P, fn.C, fn); }

__global__ void nchw_to_nhwc_kernel(const float *__restrict__ in, int B, int C, int P, float *__restrict__ out) {
    __shared__ float tile[32][33];
    int b = blockIdx.z;
    int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        int c = c0 + r, p = p0 + threadIdx.x;
        tile[r][threadIdx.x] = (c < C && p < P) ? in[((int64_t)b * C + c) * P + p] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        int p = p0 + r, c = c0 + threadIdx.x;
        if (c < C && p < P) out[((int64_t)b * P + p) * C + c] = tile[threadIdx.x][r];
    }
}

__device__ __forceinline__ int32_t quantize_one(float y, float mu) {
    float d = __fsub_rn(y, mu);
    float r = rintf(d);
    if (r != r) r = 0.f;
    r = fminf(fmaxf(r, -1073741824.f), 1073741824.f);
    return (int32_t)r;
}

struct QuantF {
    const float *y;
    const float *mu;
    int32_t *s;
    float *yhat;
    int P, C;
    __device__ void load(int b, int p, int c, bool ok, float &v) const {
        if (!ok) { v = 0.f; return; }
        int64_t i = ((int64_t)b * P + p) * C + c;
        float m = mu ? mu[c] : 0.f;
        int32_t q = quantize_one(y[i], m);
        if (yhat) yhat[i] = __fadd_rn(__int2float_rn(q), m);
        v = __int_as_float(q);
    }
    __device__ void store(int b, int p, int c, float v) const {
        s[((int64_t)b * C + c) * P + p] = __float_as_int(v);
    }
};

__global__ void quantize_kernel(QuantF fn, int B) { tile_nhwc_to_nchw(B, fn.P, fn.C, fn); }

// tab: the 64 scales, in shared memory (the threads of a warp probe different
// entries; constant memory would serialise those reads)
// smallest k with scales[k] >= sg (scales increasing), else 63.  The scales
// are log-spaced (0.11 .. 256 in 63 steps): log(sg / 0.11) over the step
// lands within one of k, and comparisons with the table itself settle it.
__device__ __forceinline__ uint8_t index_one(float sg, const float *tab) {
    if (sg != sg) return 63;
    sg = fmaxf(sg, tab[0]);
    if (sg > tab[63]) return 63;
    constexpr float kPerLog = 8.1266f;   // 63 / ln(256 / 0.11)
    int k = (int)ceilf(__logf(sg * (1.f / 0.11f)) * kPerLog);
    k = min(max(k, 0), 63);
    while (k < 63 && tab[k] < sg) ++k;
    while (k > 0 && tab[k - 1] >= sg) --k;
    return (uint8_t)k;
}

struct IndexF {
    const float *sigma;
    uint8_t *idx;
    float *sig_nchw;
    int P, C;
    const float *tab;   // shared-memory copy of the scales
    __device__ void load(int b, int p, int c, bool ok, float &v) const {
        v = ok ? sigma[((int64_t)b * P + p) * C + c] : 0.f;
    }
    __device__ void store(int b, int p, int c, float v) const {
        int64_t o = ((int64_t)b * C + c) * P + p;
        idx[o] = index_one(v, tab);
        if (sig_nchw) sig_nchw[o] = v;
    }
};

__global__ void index_kernel(IndexF fn, int B) {
    __shared__ float tab[64];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if (t < 64) tab[t] = c_scales[t];
    __syncthreads();
    fn.tab = tab;
    tile_nhwc_to_nchw(B, fn.P, fn.C, fn);
}

// The same indices when P % 4 == 0, four pixels per thread: a block (32 x 8
// threads) reads a 128-pixel x 32-channel tile of sigma with coalesced rows,
// then each thread writes the indices of 4 consecutive pixels of one channel
// as one 4-byte word (a warp: 128 contiguous bytes of a channel's plane).
constexpr int IX_P = 128;
__global__ void __launch_bounds__(256) index4_kernel(const float *__restrict__ sigma, int P, int C,
                                                     uint8_t *__restrict__ idx) {
    __shared__ float tab[64];
    __shared__ float tile[IX_P][33];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
    if (t < 64) tab[t] = c_scales[t];
    const int b = blockIdx.z, p0 = blockIdx.x * IX_P, c0 = blockIdx.y * 32;
    // all sixteen loads in flight before the first shared store
    float v[IX_P / 8];
#pragma unroll
    for (int k = 0; k < IX_P / 8; ++k) {
        const int p = p0 + ty + 8 * k, c = c0 + tx;
        v[k] = (p < P && c < C) ? sigma[((int64_t)b * P + p) * C + c] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < IX_P / 8; ++k) tile[ty + 8 * k][tx] = v[k];
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int c = c0 + r, p = p0 + 4 * tx;
        if (c >= C || p >= P) continue;
        const uint32_t w = (uint32_t)index_one(tile[4 * tx][r], tab) |
                           ((uint32_t)index_one(tile[4 * tx + 1][r], tab) << 8) |
                           ((uint32_t)index_one(tile[4 * tx + 2][r], tab) << 16) |
                           ((uint32_t)index_one(tile[4 * tx + 3][r], tab) << 24);
        *reinterpret_cast<uint32_t *>(idx + ((int64_t)b * C + c) * P + p) = w;
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g < 148 * 32 ? (g < 1 ? 1 : g) : 148 * 32);
}

dim3 tile_grid(int B, int P, int C) { return dim3((P + 31) / 32, (C + 31) / 32, B); }

}  // namespace

cudaError_t upload_scale_table() {
    float T[64];
    scale_table(T);
    return cudaMemcpyToSymbol(c_scales, T, sizeof(T));
}

__global__ void norm1d_kernel(const float *__restrict__ in, int64_t n, int C, const float *__restrict__ beta,
                              const float *__restrict__ gamma, int inverse, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const float x = in[i];
        const float v = fmaf(gamma[c], x * x, beta[c]);
        out[i] = inverse ? x * sqrtf(v) : x * rsqrtf(v);
    }
}

void launch_norm1d(const float *in, int64_t P, int C, const float *beta, const float *gamma, int inverse,
                   float *out, cudaStream_t st) {
    norm1d_kernel<<<grid_for(P * C), 256, 0, st>>>(in, P * C, C, beta, gamma, inverse, out);
}

__global__ void to_bf16_kernel(const float *__restrict__ in, int64_t n, __nv_bfloat16 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

void launch_to_bf16(const float *in, int64_t n, void *out, cudaStream_t st) {
    to_bf16_kernel<<<grid_for(n), 256, 0, st>>>(in, n, static_cast<__nv_bfloat16 *>(out));
}

void launch_pad_pack(const float *frames, int B, int H, int W, int Hp, int Wp, float *out, cudaStream_t st) {
    pad_pack_kernel<<<grid_for((int64_t)B * Hp * Wp), 256, 0, st>>>(frames, B, H, W, Hp, Wp, out);
}

void launch_frame_pad4(const float *frames, int B, int H, int W, int Hp, int Wp, float *out, cudaStream_t st) {
    frame_pad4_kernel<<<grid_for((int64_t)B * Hp * Wp), 256, 0, st>>>(frames, B, H, W, Hp, Wp,
                                                                      reinterpret_cast<float4 *>(out));
}

void launch_patch_pack(const float *x, int B, int Hp, int Wp, float *out, cudaStream_t st) {
    const dim3 grid((unsigned)((Wp / 2 + PP_COLS - 1) / PP_COLS), (unsigned)(Hp / 2), (unsigned)B);
    patch_pack_kernel<false><<<grid, PP_T, 0, st>>>(x, Hp, Wp, Hp, Wp, out);
}

void launch_frame_patch(const float *frames, int B, int H, int W, int Hp, int Wp, float *out, cudaStream_t st) {
    const dim3 grid((unsigned)((Wp / 2 + PP_COLS - 1) / PP_COLS), (unsigned)(Hp / 2), (unsigned)B);
    patch_pack_kernel<true><<<grid, PP_T, 0, st>>>(frames, H, W, Hp, Wp, out);
}

void launch_crop_unpack(const float *x, int B, int Hp, int Wp, int H, int W, float *frames, cudaStream_t st) {
    crop_unpack_kernel<<<grid_for((int64_t)B * H * W), 256, 0, st>>>(x, B, Hp, Wp, H, W, frames);
}

void launch_nhwc_to_nchw(const float *in, int B, int H, int W, int C, float *out, cudaStream_t st) {
    CopyF fn{in, out, H * W, C};
    nhwc_to_nchw_kernel<<<tile_grid(B, H * W, C), dim3(32, 8), 0, st>>>(fn, B);
}

void launch_nchw_to_nhwc(const float *in, int B, int C, int H, int W, float *out, cudaStream_t st) {
    nchw_to_nhwc_kernel<<<tile_grid(B, H * W, C), dim3(32, 8), 0, st>>>(in, B, C, H * W, out);
}

void launch_quantize(const float *y, int B, int HW, int C, const float *mu, int32_t *s, float *yhat,
                     cudaStream_t st) {
    QuantF fn{y, mu, s, yhat, HW, C};
    quantize_kernel<<<tile_grid(B, HW, C), dim3(32, 8), 0, st>>>(fn, B);
}

void launch_scale_index(const float *sigma, int B, int HW, int C, uint8_t *idx, float *sigma_nchw,
                        cudaStream_t st) {
    if (!sigma_nchw && HW % 4 == 0 && (reinterpret_cast<uintptr_t>(idx) & 3) == 0) {
        index4_kernel<<<dim3((HW + IX_P - 1) / IX_P, (C + 31) / 32, B), dim3(32, 8), 0, st>>>(sigma, HW, C, idx);
        return;
    }
    IndexF fn{sigma, idx, sigma_nchw, HW, C, nullptr};
    index_kernel<<<tile_grid(B, HW, C), dim3(32, 8), 0, st>>>(fn, B);
}

}  // namespace lic
