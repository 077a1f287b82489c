// The learned form (include/lic_student.h): a distilled student synthesis
// net -- four transposed convolutions 5x5 / stride 2, M -> C -> C -> C -> 3,
// ReLU after the first three -- trained on the GPU against the teacher's g_s
// (the decoder transform of the paper's Sec. III-A/B) and run by the
// decoder in its place.
//
// Notation: h_0 = y_hat crop, z_l = deconv_l(h_l) (l = 0..3), h_{l+1} =
// ReLU(z_l), out = z_3.  Loss L = mean((out - x)^2).  Backward pass, by the
// chain rule: dz_3 = 2 (out - x) / n; for l = 3..0
//   dW_l[i][o][u][v] = sum_{b,a,c} h_l[b,a,c,i] dz_l[b, 2a+u-2, 2c+v-2, o]
//   db_l[o]          = sum over dz_l's positions of dz_l[., o]
//   dz_{l-1}         = conv5x5/2(dz_l; W_l) * [h_l > 0]     (l > 0)
// where conv5x5/2 with the transposed conv's own weight array is its
// adjoint.  Then one Adam step (Kingma & Ba 2015, Algorithm 1).
//
// Layout: activations and gradients NHWC float32; the master weights keep
// the transposed-conv layout [Cin][Cout][5][5] and are re-laid out after
// every update into (a) the four sub-pixel phase matrices [Cout][T][Cin] of
// the forward pass, (b) the conv matrix [Cin][25][Cout] of the input
// gradient, (c) [Cin][25][4] for the 3-channel last layer.
//
// Every reduction has a fixed order (split-K partials summed in split
// order), so results do not depend on timing.
//
// Precision LIC_BF16 (the training form the task configures): the three
// 64-channel transposed convs and the input gradients through them run on
// the tcgen05 bf16 kernel (bf16 operands, float32 accumulation); y_hat,
// h_1, h_2 and dz_0..dz_2 are stored in bf16, h_3, the output and dz_3 in
// float32; the 3-channel layer, the weight and bias gradients and Adam stay
// float32 on CUDA cores (reading the bf16 tensors), master weights float32.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/lic_student.h"
#include "conv_tc.h"
#include "lic_internal.h"

namespace lic {
namespace {

constexpr int NL = 4;
// taps of sub-pixel phase ph = 2 py + px: (0,0) 9, (0,1) 6, (1,0) 6, (1,1) 4;
// and the first tap of each phase in the forward matrices
__host__ __device__ constexpr int ph_taps(int ph) { return ph == 0 ? 9 : (ph == 3 ? 4 : 6); }
__host__ __device__ constexpr int ph_off(int ph) { return ph == 0 ? 0 : (ph == 1 ? 9 : (ph == 2 ? 15 : 21)); }

struct Crops {
    int n;
    int f[LIC_STUDENT_MAX_BATCH], r[LIC_STUDENT_MAX_BATCH], c[LIC_STUDENT_MAX_BATCH];
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ld(const float *p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void st(float *p, int64_t i, float v) { p[i] = v; }
__device__ __forceinline__ void st(__nv_bfloat16 *p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }
// four consecutive values starting at a 4-aligned index
__device__ __forceinline__ float4 ld4(const float *p, int64_t i) { return *reinterpret_cast<const float4 *>(p + i); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p, int64_t i) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p + i);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}

// y_hat crops: pool NCHW [P][M][Hy][Wy] -> h0 NHWC [B][lc][lc][M]
template <typename TO>
__global__ void gather_yhat_kernel(const float *__restrict__ pool, int M, int Hy, int Wy, Crops cr, int lc,
                                   TO *__restrict__ h0) {
    const int64_t n = (int64_t)cr.n * lc * lc * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % M);
        int64_t pos = e / M;
        const int c = (int)(pos % lc);
        pos /= lc;
        const int r = (int)(pos % lc);
        const int b = (int)(pos / lc);
        st(h0, e, pool[(((int64_t)cr.f[b] * M + ch) * Hy + cr.r[b] + r) * Wy + cr.c[b] + c]);
    }
}

constexpr int RED_T = 256;
constexpr int BG_BLOCKS = 4 * 148;   // blocks of a bias-gradient reduction

// out NHWC [B][S][S][3] (the net's output on the latent windows) against
// the target crops of xpool NCHW [P][3][Hx][Wx]: inside the loss square
// [o, o + crop)^2, dz = (2/n) (out - x), outside dz = 0; per block the
// float64 sum of (out - x)^2 over its loss pixels (fixed tree)
__global__ void __launch_bounds__(RED_T) mse_grad_kernel(const float *__restrict__ out,
                                                         const float *__restrict__ xpool, int Hx, int Wx, Crops cr,
                                                         int S, int o, int crop, float two_over_n,
                                                         float *__restrict__ dz, double *__restrict__ part) {
    __shared__ double red[RED_T];
    const int64_t npix = (int64_t)cr.n * S * S;
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)RED_T + threadIdx.x; p < npix; p += (int64_t)gridDim.x * RED_T) {
        const int x = (int)(p % S);
        const int y = (int)((p / S) % S);
        const int b = (int)(p / ((int64_t)S * S));
        const bool in = y >= o && y < o + crop && x >= o && x < o + crop;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float d = 0.f;
            if (in) {
                const float t =
                    xpool[(((int64_t)cr.f[b] * 3 + k) * Hx + 16 * cr.r[b] + y) * Wx + 16 * cr.c[b] + x];
                d = out[p * 3 + k] - t;
            }
            dz[p * 3 + k] = two_over_n * d;
            acc += (double)d * (double)d;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_T / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// loss = (sum of the block partials, in block order) / n
__global__ void __launch_bounds__(RED_T) mse_final_kernel(const double *__restrict__ part, int nblk, double n,
                                                          float *__restrict__ loss) {
    __shared__ double red[RED_T];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += RED_T) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_T / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] / n);
}

// per-channel sums of an NHWC tensor [P][C] (C <= RED_T): block z sums the
// pixels [z*per, (z+1)*per) into part[z][C]
template <typename TX>
__global__ void __launch_bounds__(RED_T) chan_sum_kernel(const TX *__restrict__ x, int64_t P, int C, int64_t per,
                                                         float *__restrict__ part) {
    __shared__ float red[RED_T];
    const int G = RED_T / C;          // pixel lanes
    const int g = threadIdx.x / C, c = threadIdx.x % C;
    float acc = 0.f;
    if (g < G) {
        const int64_t p0 = blockIdx.x * per, p1 = min(P, p0 + per);
        for (int64_t p = p0 + g; p < p1; p += G) acc += ld(x, p * C + c);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int q = 0; q < G; ++q) s += red[q * C + threadIdx.x];
        part[(int64_t)blockIdx.x * C + threadIdx.x] = s;
    }
}

// out[c] = sum over z of part[z][c]: block c, thread t sums z = t, t + RED_T,
// ... in order, then a fixed tree over the threads
__global__ void __launch_bounds__(RED_T) chan_sum_final_kernel(const float *__restrict__ part, int nz, int C,
                                                               float *__restrict__ out) {
    __shared__ float red[RED_T];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int z = threadIdx.x; z < nz; z += RED_T) s += part[(int64_t)z * C + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = RED_T / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// Weight gradient of a transposed conv 5x5 / 2 as a GEMM: rows i (input
// channel), columns n = tap * Cout + o, K = the B*H*W input pixels, split
// over gridDim.z slices of kper pixels.  x: NHWC [B][H][W][Cin] (Cin % 4 == 0);
// dz: NHWC [B][2H][2W][Cout].  part[z][Cin][25*Cout].
constexpr int WG_BM = 64, WG_BN = 64, WG_BK = 16, WG_NT = 256;

template <bool VEC, typename TX, typename TD>   // VEC: Cout % 64 == 0, one tap per column tile, 4-wide loads
__global__ void __launch_bounds__(WG_NT) wgrad_kernel(const TX *__restrict__ x, const TD *__restrict__ dz, int B,
                                                      int H, int W, int Cin, int Cout, int64_t kper,
                                                      float *__restrict__ part) {
    __shared__ __align__(16) float As[WG_BK][WG_BM];
    __shared__ __align__(16) float Bs[WG_BK][WG_BN];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int i0 = blockIdx.y * WG_BM, n0 = blockIdx.x * WG_BN;
    const int N = 25 * Cout;
    const int64_t HW = (int64_t)H * W, P = (int64_t)B * HW;
    const int64_t k_begin = blockIdx.z * kper, k_end = min(P, k_begin + kper);
    const int Ho = 2 * H, Wo = 2 * W;
    const int lp = tid / 16, lq = tid % 16;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int64_t k0 = k_begin; k0 < k_end; k0 += WG_BK) {
        const int64_t p = k0 + lp;
        const bool pv = p < k_end;
        int b = 0, a = 0, c = 0;
        if (pv) {
            b = (int)(p / HW);
            const int rem = (int)(p % HW);
            a = rem / W;
            c = rem % W;
        }
        float4 va = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pv && i0 + 4 * lq < Cin) va = ld4(x, p * Cin + i0 + 4 * lq);
        *reinterpret_cast<float4 *>(&As[lp][4 * lq]) = va;
        if (VEC) {
            const int tap = n0 / Cout, o0 = n0 % Cout;
            const int yo = 2 * a + tap / 5 - 2, xo = 2 * c + tap % 5 - 2;
            float4 vb = make_float4(0.f, 0.f, 0.f, 0.f);
            if (pv && yo >= 0 && yo < Ho && xo >= 0 && xo < Wo)
                vb = ld4(dz, (((int64_t)b * Ho + yo) * Wo + xo) * Cout + o0 + 4 * lq);
            *reinterpret_cast<float4 *>(&Bs[lp][4 * lq]) = vb;
        } else {
#pragma unroll
            for (int r = 0; r < (WG_BK * WG_BN) / WG_NT; ++r) {
                const int e = tid + r * WG_NT;
                const int kk = e / WG_BN, nn = e % WG_BN;
                const int64_t pp = k0 + kk;
                const int n = n0 + nn;
                float vb = 0.f;
                if (pp < k_end && n < N) {
                    const int tap = n / Cout, o = n % Cout;
                    const int bb = (int)(pp / HW);
                    const int rem = (int)(pp % HW);
                    const int yo = 2 * (rem / W) + tap / 5 - 2, xo = 2 * (rem % W) + tap % 5 - 2;
                    if (yo >= 0 && yo < Ho && xo >= 0 && xo < Wo) vb = ld(dz, (((int64_t)bb * Ho + yo) * Wo + xo) * Cout + o);
                }
                Bs[kk][nn] = vb;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < WG_BK; ++kk) {
            const float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ii = i0 + ty * 4 + i;
        if (ii >= Cin) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < N) part[((int64_t)blockIdx.z * Cin + ii) * N + n] = acc[i][j];
        }
    }
}

// Weight gradient of the 3-channel last layer (float32 h and dz):
// dW[i][o][u][v] = sum_{b,a,c} h[b,a,c,i] dz[b, 2a+u-2, 2c+v-2, o].  Per
// pixel that is a 64 x 75 outer product of h's channels with dz's 5 x 5 x 3
// window, so the kernel is bound by FMA issue.  A work unit is 2 input rows
// x 128 columns x 64 input channels of one frame: the dz rows it touches go
// to shared memory as a zero-padded strip (7 rows x 260 columns x 3), h in
// chunks of 64 pixels; both are double-buffered and fetched with cp.async one
// chunk ahead, so the loads overlap the FMAs.  Warp u (0..4) owns the 15
// window values of tap row u -- contiguous in the strip -- and each lane 8
// channels (4 ig .. 4 ig + 3 and 32 + 4 ig ..: a quarter warp's 16-byte
// loads cover 128 contiguous bytes) x those 15 values for every fourth pixel
// of a chunk (lane = 8 pixel slot + ig): a pixel step is 2 x 16-byte h loads and 15
// strip values for 120 FMAs.  The four pixel slots are added by shuffles at
// the end, and block z's sums go to part[z][i][(5u+v)*3 + o]
// (wgrad_reduce_kernel adds the blocks in order).
constexpr int W3_TR = 2, W3_TC = 128, W3_PC = 64, W3_T = 160, W3_BLOCKS = 2 * 148;
constexpr int W3_SR = 2 * W3_TR + 3, W3_SP = (2 * W3_TC + 4) * 3;   // strip rows, row pitch (floats)
constexpr int W3_CPU = W3_TR * (W3_TC / W3_PC);                      // chunks per unit

__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// global -> shared without registers; bytes past src_bytes (0 or all) are zero-filled
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sh_addr(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sh_addr(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__global__ void __launch_bounds__(W3_T, 2) wgrad3_kernel(const float *__restrict__ h, const float *__restrict__ dz,
                                                         int B, int H, int W, int Cin, int per_block,
                                                         float *__restrict__ part) {
    extern __shared__ __align__(16) float w3_smem[];
    float *strip = w3_smem;                        // [2][W3_SR * W3_SP]
    float *hs = w3_smem + 2 * W3_SR * W3_SP;       // [2][W3_PC][64]
    const int tid = threadIdx.x, u = tid >> 5, lane = tid & 31, ig = lane & 7, ps = lane >> 3;
    const int tiles_x = (W + W3_TC - 1) / W3_TC, rows = (H + W3_TR - 1) / W3_TR, ichunks = (Cin + 63) / 64;
    const int nunits = tiles_x * rows * B * ichunks;
    const int Ho = 2 * H, Wo = 2 * W;
    const int u_begin = blockIdx.x * per_block, u_end = min(nunits, u_begin + per_block);
    float acc[8][15];
    for (int ic = 0; ic < ichunks; ++ic) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int k = 0; k < 15; ++k) acc[i][k] = 0.f;
        // this chunk's units: un0, un0 + ichunks, ... below u_end (units interleave the channel chunks)
        const int un0 = u_begin + ((ic - u_begin % ichunks) % ichunks + ichunks) % ichunks;
        const int nu = un0 < u_end ? (u_end - 1 - un0) / ichunks + 1 : 0;
        const int jobs = nu * W3_CPU;
        // unit k's frame and corner
        auto unit = [&](int k, int *b, int *a0, int *c0) {
            int r = (un0 + k * ichunks) / ichunks;
            const int tx = r % tiles_x;
            r /= tiles_x;
            *a0 = (r % rows) * W3_TR;
            *b = r / rows;
            *c0 = tx * W3_TC;
        };
        // issue job j's loads: its h chunk, and the unit's strip when j opens a unit
        auto issue = [&](int j) {
            if (j < jobs) {
                int b, a0, c0;
                unit(j / W3_CPU, &b, &a0, &c0);
                const int c = j % W3_CPU, rr = c / (W3_TC / W3_PC), cc = (c % (W3_TC / W3_PC)) * W3_PC;
                if (c == 0) {
                    float *sb = strip + ((j / W3_CPU) & 1) * (W3_SR * W3_SP);
                    for (int e = tid; e < W3_SR * W3_SP; e += W3_T) {
                        const int sr = e / W3_SP, rem = e % W3_SP;
                        const int y = 2 * a0 - 2 + sr, x = 2 * c0 - 2 + rem / 3;
                        const bool ok = y >= 0 && y < Ho && x >= 0 && x < Wo;
                        cp_async4(sb + e, ok ? dz + (((int64_t)b * Ho + y) * Wo + x) * 3 + rem % 3 : dz, ok);
                    }
                }
                float *hb = hs + (j & 1) * (W3_PC * 64);
                const int a = a0 + rr, n = (a < H) ? max(0, min(W3_PC, W - c0 - cc)) : 0;
                for (int e = tid; e < W3_PC * 16; e += W3_T) {
                    const int px = e >> 4, q = e & 15, ch = 64 * ic + 4 * q;
                    const bool ok = px < n && ch < Cin;
                    cp_async16(hb + px * 64 + 4 * q,
                               ok ? h + (((int64_t)b * H + a) * W + c0 + cc + px) * Cin + ch : h, ok);
                }
            }
            cp_async_commit();   // an empty group past the last job keeps the wait count uniform
        };
        issue(0);
        for (int j = 0; j < jobs; ++j) {
            issue(j + 1);
            cp_async_wait1();    // job j's group has landed (this thread's copies)
            __syncthreads();     // ... and every thread's
            int b, a0, c0;
            unit(j / W3_CPU, &b, &a0, &c0);
            const int c = j % W3_CPU, rr = c / (W3_TC / W3_PC), cc = (c % (W3_TC / W3_PC)) * W3_PC;
            const int n = (a0 + rr < H) ? max(0, min(W3_PC, W - c0 - cc)) : 0;
            const float *hb = hs + (j & 1) * (W3_PC * 64);
            // window of pixel (a0 + rr, c0 + cc + px), tap row u: strip row 2 rr + u, columns 2 (cc + px) ..
            const float *wrow = strip + ((j / W3_CPU) & 1) * (W3_SR * W3_SP) + (2 * rr + u) * W3_SP + 2 * cc * 3;
            for (int px = ps; px < n; px += 4) {
                const float4 h0 = *reinterpret_cast<const float4 *>(hb + px * 64 + 4 * ig);
                const float4 h1 = *reinterpret_cast<const float4 *>(hb + px * 64 + 32 + 4 * ig);
                const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
                const float *wp = wrow + 6 * px;   // 8-byte aligned: 15 values as 7 pairs + 1
                float w[15];
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    const float2 t = *reinterpret_cast<const float2 *>(wp + 2 * k);
                    w[2 * k] = t.x;
                    w[2 * k + 1] = t.y;
                }
                w[14] = wp[14];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int k = 0; k < 15; ++k) acc[i][k] = fmaf(hv[i], w[k], acc[i][k]);
            }
            __syncthreads();     // job j's buffers are free for job j + 2's loads
        }
        // the four pixel slots of a channel group, then one store per (i, k)
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int k = 0; k < 15; ++k) {
                float v = acc[i][k];
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                acc[i][k] = v;
            }
        if (ps == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int ci = 64 * ic + (i < 4 ? 4 * ig + i : 32 + 4 * ig + i - 4);
                if (ci < Cin)
#pragma unroll
                    for (int k = 0; k < 15; ++k) part[((int64_t)blockIdx.x * Cin + ci) * 75 + 15 * u + k] = acc[i][k];
            }
        }
        __syncthreads();
    }
}
constexpr int W3_SMEM = (2 * W3_SR * W3_SP + 2 * W3_PC * 64) * 4;

// Input gradient through the 3-channel last layer and the ReLU before it:
// dz_prev[b,a,c,i] = [h[b,a,c,i] > 0] sum_{u,v,o} dz[b, 2a+u-2, 2c+v-2, o]
// W[i][o][u][v] -- the stride-2 conv with the transposed conv's weights, its
// adjoint.  Per pixel a 75 x 64 matrix-vector product, so the kernel is
// bound by FMA issue.  The weights sit in shared memory as [k][i] (k =
// (5u+v)*3+o); a work unit is the same 2 x 128 block of pixels as in
// wgrad3_kernel with the same double-buffered dz strip, and each thread
// computes 8 consecutive pixels of a row x 8 channels (4 ig .. 4 ig + 3 and
// 32 + 4 ig .. 32 + 4 ig + 3): per k, 8 strip values (a warp's four pixel
// groups: four broadcast addresses) and 2 x 16-byte weight loads for 64 FMAs.
// The mask and the store (float32 or bf16, as the activation before it is
// stored) follow in the epilogue.
constexpr int D3_T = 256;
constexpr int D3_SMEM = (2 * W3_SR * W3_SP + 75 * 64) * 4;

template <typename TO>
__global__ void __launch_bounds__(D3_T, 2) dgrad3_kernel(const float *__restrict__ dz, const float *__restrict__ wd,
                                                        const float *__restrict__ h, int B, int H, int W,
                                                        int per_block, TO *__restrict__ out) {
    extern __shared__ __align__(16) float d3_smem[];
    float *strip = d3_smem;                       // [2][W3_SR * W3_SP]
    float *ws = d3_smem + 2 * W3_SR * W3_SP;      // [75][64]
    const int tid = threadIdx.x, lane = tid & 31, ig = lane & 7;
    const int pg = (tid >> 5) * 4 + (lane >> 3);   // pixel group 0..31: row pg / 16, columns 8 (pg % 16) ..
    const int tiles_x = (W + W3_TC - 1) / W3_TC, rows = (H + W3_TR - 1) / W3_TR;
    const int nunits = tiles_x * rows * B;
    const int Ho = 2 * H, Wo = 2 * W;
    const int u_begin = blockIdx.x * per_block, u_end = min(nunits, u_begin + per_block);
    // weights: wd [64][25][3] (i, tap, o) -> ws[k][i], k = tap * 3 + o
    for (int e = tid; e < 75 * 64; e += D3_T) ws[(e % 75) * 64 + e / 75] = wd[e];
    auto unit = [&](int un, int *b, int *a0, int *c0) {
        int r = un;
        const int tx = r % tiles_x;
        r /= tiles_x;
        *a0 = (r % rows) * W3_TR;
        *b = r / rows;
        *c0 = tx * W3_TC;
    };
    auto issue = [&](int un, int slot) {
        if (un < u_end) {
            int b, a0, c0;
            unit(un, &b, &a0, &c0);
            float *sb = strip + slot * (W3_SR * W3_SP);
            for (int e = tid; e < W3_SR * W3_SP; e += D3_T) {
                const int sr = e / W3_SP, rem = e % W3_SP;
                const int y = 2 * a0 - 2 + sr, x = 2 * c0 - 2 + rem / 3;
                const bool ok = y >= 0 && y < Ho && x >= 0 && x < Wo;
                cp_async4(sb + e, ok ? dz + (((int64_t)b * Ho + y) * Wo + x) * 3 + rem % 3 : dz, ok);
            }
        }
        cp_async_commit();
    };
    const int rr = pg / 16, cq = (pg % 16) * 8;   // the thread's row and first column within a unit
    issue(u_begin, 0);
    for (int un = u_begin; un < u_end; ++un) {
        const int slot = (un - u_begin) & 1;
        issue(un + 1, slot ^ 1);
        cp_async_wait1();
        __syncthreads();   // the strip (and, the first time, the weights) are in place
        int b, a0, c0;
        unit(un, &b, &a0, &c0);
        const int a = a0 + rr;
        float acc[8][8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[j][i] = 0.f;
        // pixel j = column c0 + cq + j: window element (u, v, o) at strip row 2 rr + u, column 2 (cq + j) + v
        const float *sb = strip + slot * (W3_SR * W3_SP) + 2 * rr * W3_SP + 2 * cq * 3;
#pragma unroll 1
        for (int u = 0; u < 5; ++u) {
#pragma unroll 1
            for (int vo = 0; vo < 15; ++vo) {
                const int k = u * 15 + vo;
                const float4 w0 = *reinterpret_cast<const float4 *>(ws + k * 64 + 4 * ig);
                const float4 w1 = *reinterpret_cast<const float4 *>(ws + k * 64 + 32 + 4 * ig);
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                const float *xp = sb + u * W3_SP + vo;
                float xv[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) xv[j] = xp[6 * j];
#pragma unroll
                for (int j = 0; j < 8; ++j)
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[j][i] = fmaf(xv[j], wv[i], acc[j][i]);
            }
        }
        if (a < H) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + cq + j;
                if (c >= W) break;
                const int64_t o = (((int64_t)b * H + a) * W + c) * 64;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int ch = half * 32 + 4 * ig;
                    const float4 m = ld4(h, o + ch);
                    const float v0 = m.x > 0.f ? acc[j][4 * half] : 0.f, v1 = m.y > 0.f ? acc[j][4 * half + 1] : 0.f;
                    const float v2 = m.z > 0.f ? acc[j][4 * half + 2] : 0.f, v3 = m.w > 0.f ? acc[j][4 * half + 3] : 0.f;
                    st(out, o + ch, v0);
                    st(out, o + ch + 1, v1);
                    st(out, o + ch + 2, v2);
                    st(out, o + ch + 3, v3);
                }
            }
        }
        __syncthreads();   // this strip slot is free for the unit after next
    }
}

void dgrad3_plan(int B, int H, int W, int *blocks, int *per_block) {
    const int nunits = ((W + W3_TC - 1) / W3_TC) * ((H + W3_TR - 1) / W3_TR) * B;
    *per_block = (nunits + W3_BLOCKS - 1) / W3_BLOCKS;
    *blocks = (nunits + *per_block - 1) / *per_block;
}

// blocks of wgrad3_kernel and the units each takes (2 rows x 128 columns x
// 64 channels); the grid is a fixed count, so the sums do not depend on the device
void wgrad3_plan(int B, int H, int W, int Cin, int *blocks, int *per_block) {
    const int nunits = ((W + W3_TC - 1) / W3_TC) * ((H + W3_TR - 1) / W3_TR) * B * ((Cin + 63) / 64);
    *per_block = (nunits + W3_BLOCKS - 1) / W3_BLOCKS;
    *blocks = (nunits + *per_block - 1) / *per_block;
}

// dW[i][o][u][v] = sum over z of part[z][i][(u*5+v)*Cout + o], in a fixed
// order: a block takes 32 consecutive (i, column) entries; thread (g, t) adds
// slices z = g, g + 8, ... in order, then the 8 group sums are added as a
// fixed tree.  Eight loads in flight per entry instead of one chain of nz.
constexpr int WR_G = 8;
__global__ void __launch_bounds__(32 * WR_G) wgrad_reduce_kernel(const float *__restrict__ part, int nz, int Cin,
                                                                 int Cout, float *__restrict__ dw) {
    __shared__ float red[WR_G][33];
    const int N = 25 * Cout;
    const int t = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t ne = (int64_t)Cin * N, e = blockIdx.x * (int64_t)32 + t;
    float s = 0.f;
    if (e < ne)
        for (int z = g; z < nz; z += WR_G) s += part[(int64_t)z * ne + e];
    red[g][t] = s;
    __syncthreads();
    if (g == 0 && e < ne) {
        const float a = (red[0][t] + red[1][t]) + (red[2][t] + red[3][t]);
        const float b = (red[4][t] + red[5][t]) + (red[6][t] + red[7][t]);
        const int i = (int)(e / N), n = (int)(e % N);
        dw[((int64_t)i * Cout + n % Cout) * 25 + n / Cout] = a + b;
    }
}
inline unsigned wgrad_reduce_grid(int64_t ne) { return (unsigned)((ne + 31) / 32); }

// Adam over the flat parameter vector; c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int64_t n, float lr, float b1, float b2, float c1, float c2,
                            float eps) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

struct RepackArgs {
    const float *w[NL];
    float *wf[NL];   // forward phase matrices (layers with > 4 outputs) or null
    float *wd[NL];   // input-gradient conv matrix (layers 1..3) or null
    __nv_bfloat16 *wfb[NL], *wdb[NL];   // bf16 copies of the same (precision LIC_BF16) or null
    float *ws;       // last layer [Cin][25][4]
    int cin[NL], cout[NL];
    int64_t start[NL + 1];
};

// master [Cin][Cout][5][5] -> the layouts the kernels read.  Output row
// Y = 2m + py takes tap u of input row m + (py + 2 - u)/2 when u = py mod 2:
// phase (u & 1, v & 1), tap index (u >> 1) * (3 or 2) + (v >> 1).
__global__ void repack_kernel(RepackArgs a) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= a.start[NL]) return;
    int l = 0;
    while (l < NL - 1 && idx >= a.start[l + 1]) ++l;
    const int64_t e = idx - a.start[l];
    const int Cin = a.cin[l], Cout = a.cout[l];
    const int v = (int)(e % 5), u = (int)((e / 5) % 5);
    const int o = (int)((e / 25) % Cout);
    const int i = (int)(e / (25 * (int64_t)Cout));
    const float wv = a.w[l][e];
    const int ph = (u & 1) * 2 + (v & 1);
    const int t = (u >> 1) * ((v & 1) ? 2 : 3) + (v >> 1);
    const int64_t fi = (int64_t)ph_off(ph) * Cout * Cin + ((int64_t)o * ph_taps(ph) + t) * Cin + i;
    const int64_t di = ((int64_t)i * 25 + u * 5 + v) * Cout + o;
    if (a.wf[l]) a.wf[l][fi] = wv;
    if (a.wfb[l]) a.wfb[l][fi] = __float2bfloat16_rn(wv);
    if (a.wd[l]) a.wd[l][di] = wv;
    if (a.wdb[l]) a.wdb[l][di] = __float2bfloat16_rn(wv);
    if (l == NL - 1 && a.ws) a.ws[((int64_t)i * 25 + u * 5 + v) * 4 + o] = wv;
}

// per frame: float64 sum over its H x W x 3 cropped values of
// (clamp(xs) - clamp(xt))^2; grid (blocks, B); part[b][block]
__global__ void __launch_bounds__(RED_T) frame_sse_kernel(const float *__restrict__ xs, const float *__restrict__ xt,
                                                          int Hp, int Wp, int H, int W, double *__restrict__ part) {
    __shared__ double red[RED_T];
    const int b = blockIdx.y;
    const int64_t n = (int64_t)H * W;
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)RED_T + threadIdx.x; p < n; p += (int64_t)gridDim.x * RED_T) {
        const int y = (int)(p / W), x = (int)(p % W);
        const int64_t q = (((int64_t)b * Hp + y) * Wp + x) * 3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float d = fminf(fmaxf(xs[q + k], 0.f), 1.f) - fminf(fmaxf(xt[q + k], 0.f), 1.f);
            acc += (double)d * (double)d;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_T / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = red[0];
}

// per frame PSNR = 10 log10(1 / mse); pass[b] = PSNR >= thr; the counters
// (frames, fallbacks) advance
__global__ void frame_psnr_kernel(const double *__restrict__ part, int nblk, int B, double n, float thr,
                                  float *__restrict__ psnr, int *__restrict__ pass, long long *__restrict__ counts) {
    const int b = threadIdx.x;
    bool fail = false;
    if (b < B) {
        double s = 0.0;
        for (int i = 0; i < nblk; ++i) s += part[(int64_t)b * nblk + i];
        const double mse = s / n;
        const float q = mse > 0.0 ? (float)(10.0 * log10(1.0 / mse)) : INFINITY;
        psnr[b] = q;
        pass[b] = q >= thr;
        fail = !(q >= thr);
    }
    const int nfail = __syncthreads_count(fail);
    if (b == 0) {
        counts[0] += B;
        counts[1] += nfail;
    }
}

// frames that passed take the student's output
__global__ void frame_select_kernel(const float *__restrict__ xs, float *__restrict__ xt, int64_t per_frame, int B,
                                    const int *__restrict__ pass) {
    const int64_t n = per_frame * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (pass[e / per_frame]) xt[e] = xs[e];
}

int grid_for(int64_t n, int t) { return (int)std::min<int64_t>((n + t - 1) / t, 148 * 16); }

}  // namespace
}  // namespace lic

struct lic_student {
    int M = 0, C = 0;
    lic_student_options opt{};
    bool bf16 = false;
    int device = 0;
    int cin[4] = {}, cout[4] = {};
    int64_t woff[4] = {}, boff[4] = {}, nparam = 0;
    lic::DevBuf param, grad, adam_m, adam_v;
    // float32 re-layouts (CUDA-core kernels) and bf16 ones with their tensor maps (tcgen05 kernel)
    lic::DevBuf wf[4], wd[4], ws, wfb[4], wdb[4];
    lic::tc::TmaMap fmap[4][4], dmap[4];
    // training workspace (max_batch crops)
    lic::DevBuf h[4], out, dz[4], part, lpart, loss, bpart, status;
    // inference workspace
    lic::DevBuf ih[4], iout;
    int64_t t = 0;
    int last_B = 0;
    bool launch_failed = false;
    lic::Profiler pf;
};

namespace lic {
namespace {

int64_t wsize(const lic_student *s, int l) { return (int64_t)s->cin[l] * s->cout[l] * 25; }

// storage bytes per element of h_l / dz_l (l = 0..3)
int act_bytes(const lic_student *s, int l) { return (s->bf16 && l < NL - 1) ? 2 : 4; }

template <typename F>
void timed(lic_student *s, const std::string &name, double flop, double bytes, int n, cudaStream_t st, F &&f) {
    s->pf.run(name, flop, bytes, n, st, f);
}

int ensure_e(DevBuf &b, int64_t n, int elem) {
    LIC_CUDA_TRY(b.ensure((size_t)std::max<int64_t>(n, 1) * elem));
    return LIC_OK;
}

int ensure_f(DevBuf &b, int64_t n) { return ensure_e(b, n, 4); }

int repack(lic_student *s, cudaStream_t st) {
    RepackArgs a{};
    a.start[0] = 0;
    for (int l = 0; l < NL; ++l) {
        a.w[l] = s->param.as<float>() + s->woff[l];
        a.wf[l] = s->wf[l].as<float>();
        a.wd[l] = s->wd[l].as<float>();
        a.wfb[l] = s->wfb[l].as<__nv_bfloat16>();
        a.wdb[l] = s->wdb[l].as<__nv_bfloat16>();
        a.cin[l] = s->cin[l];
        a.cout[l] = s->cout[l];
        a.start[l + 1] = a.start[l] + wsize(s, l);
    }
    a.ws = s->ws.as<float>();
    const int64_t n = a.start[NL];
    timed(s, "student.repack", 0, 12.0 * n, 1, st,
          [&] { repack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a); });
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

// taps of sub-pixel phase (py, px) of a transposed conv 5x5 / 2 into d
void phase_taps(ConvDesc &d, int py, int px) {
    int t = 0;
    for (int u = py; u < 5; u += 2)
        for (int v = px; v < 5; v += 2) {
            d.du[t] = (int8_t)((py + 2 - u) / 2);
            d.dv[t] = (int8_t)((px + 2 - v) / 2);
            ++t;
        }
    d.T = t;
}

// one transposed conv (l < 3: four phase launches + ReLU, on the bf16
// tensor-core kernel or the CUDA-core kernel; l == 3: the small-Cout
// kernel) from h (NHWC, Hi x Wi) into out
void forward_layer(lic_student *s, int l, const void *in, int B, int Hi, int Wi, void *out, cudaStream_t st) {
    const int Cin = s->cin[l], Cout = s->cout[l];
    const double flop = 2.0 * B * Hi * Wi * (double)Cin * Cout * 25;
    const double bytes = (double)B * Hi * Wi * Cin * act_bytes(s, l) +
                         4.0 * B * Hi * Wi * Cout * act_bytes(s, l + 1 < NL ? l + 1 : NL - 1) +
                         4.0 * wsize(s, l) * (s->bf16 ? 2 : 4) / 4.0;
    const float *bias = s->param.as<float>() + s->boff[l];
    if (l == NL - 1) {
        timed(s, "student.deconv3", flop, bytes, 1, st, [&] {
            launch_deconv_small(static_cast<const float *>(in), B, Hi, Wi, Cin, s->ws.as<float>(), bias, Cout,
                                static_cast<float *>(out), st);
        });
        return;
    }
    const bool tc = s->bf16;
    timed(s, "student.deconv" + std::to_string(l) + (tc ? ":tc" : ""), flop, bytes, 4, st, [&] {
        for (int ph = 0; ph < 4; ++ph) {
            const int py = ph >> 1, px = ph & 1;
            ConvDesc d{};
            d.in = static_cast<const float *>(in);
            d.out = static_cast<float *>(out);
            d.bias = bias;
            d.status = s->status.as<uint32_t>();
            d.B = B;
            d.Hi = Hi;
            d.Wi = Wi;
            d.Cin = Cin;
            d.Gh = Hi;
            d.Gw = Wi;
            d.s = 1;
            d.Ho = 2 * Hi;
            d.Wo = 2 * Wi;
            d.Cout = Cout;
            d.oym = 2;
            d.oyo = py;
            d.oxm = 2;
            d.oxo = px;
            phase_taps(d, py, px);
            d.in_xform = IN_NONE;
            d.epi = EPI_RELU;
            d.in_scale = d.out_scale = 1.f;
            if (tc) {
                d.in_dt = DT_BF16;
                d.out_dt = (l == NL - 2) ? DT_F32 : DT_BF16;
                if (!tc::launch_lp_map(d, s->fmap[l][ph], st)) s->launch_failed = true;
            } else {
                d.w = s->wf[l].as<float>() + (int64_t)ph_off(ph) * Cout * Cin;
                d.in_dt = d.out_dt = DT_F32;
                launch_conv_simt(d, st);
            }
        }
    });
}

// the student on NHWC y_hat [B][Hy][Wy][M] (stored as h_0) into NHWC out
// [B][16Hy][16Wy][3], activations in hbuf[1..3]
void forward_all(lic_student *s, const void *h0, int B, int Hy, int Wy, DevBuf *hbuf, float *out, cudaStream_t st) {
    const void *in = h0;
    int H = Hy, W = Wy;
    for (int l = 0; l < NL; ++l) {
        void *o = l < NL - 1 ? hbuf[l + 1].p : out;
        forward_layer(s, l, in, B, H, W, o, st);
        in = o;
        H *= 2;
        W *= 2;
    }
}

// latent side of one training window: the crop's latents plus the halo
int window_lat(const lic_student *s) { return s->opt.crop / 16 + 2 * s->opt.halo; }

int check_crops(const lic_student *s, const float *yp, const float *xp, int P, int Hy, int Wy, const int32_t *crops,
                int B, Crops *cr) {
    const int lc = window_lat(s);
    if (!yp || !xp || !crops || P < 1 || B < 1 || B > s->opt.max_batch || Hy < lc || Wy < lc) return LIC_E_INVALID_ARG;
    if (!is_device_ptr(yp) || !is_device_ptr(xp)) return LIC_E_INVALID_ARG;
    cr->n = B;
    for (int b = 0; b < B; ++b) {
        const int f = crops[3 * b], r = crops[3 * b + 1], c = crops[3 * b + 2];
        if (f < 0 || f >= P || r < 0 || c < 0 || r + lc > Hy || c + lc > Wy) return LIC_E_INVALID_ARG;
        cr->f[b] = f;
        cr->r[b] = r;
        cr->c[b] = c;
    }
    return LIC_OK;
}

template <typename TX, typename TD>
void launch_wgrad(bool vec, dim3 grid, cudaStream_t st, const void *x, const void *dz, int B, int H, int Cin,
                  int Cout, int64_t kper, float *part) {
    if (vec)
        wgrad_kernel<true, TX, TD><<<grid, WG_NT, 0, st>>>(static_cast<const TX *>(x), static_cast<const TD *>(dz), B,
                                                           H, H, Cin, Cout, kper, part);
    else
        wgrad_kernel<false, TX, TD><<<grid, WG_NT, 0, st>>>(static_cast<const TX *>(x), static_cast<const TD *>(dz),
                                                            B, H, H, Cin, Cout, kper, part);
}

// forward, loss and every gradient of one batch
int grad_pass(lic_student *s, const float *yp, const float *xp, int P, int Hy, int Wy, const int32_t *crops, int B,
              cudaStream_t st) {
    Crops cr{};
    int rc = check_crops(s, yp, xp, P, Hy, Wy, crops, B, &cr);
    if (rc) return rc;
    s->last_B = B;
    s->launch_failed = false;
    const int lc = window_lat(s), S = 16 * lc, M = s->M;
    // gather
    const int64_t ny = (int64_t)B * lc * lc * M;
    timed(s, "student.gather", 0, (4.0 + act_bytes(s, 0)) * ny, 1, st, [&] {
        if (s->bf16)
            gather_yhat_kernel<<<grid_for(ny, 256), 256, 0, st>>>(yp, M, Hy, Wy, cr, lc, s->h[0].as<__nv_bfloat16>());
        else
            gather_yhat_kernel<<<grid_for(ny, 256), 256, 0, st>>>(yp, M, Hy, Wy, cr, lc, s->h[0].as<float>());
    });
    // forward
    forward_all(s, s->h[0].p, B, lc, lc, s->h, s->out.as<float>(), st);
    // loss and dz_3
    const int64_t npix = (int64_t)B * S * S;
    const int nblk = grid_for(npix, RED_T);
    const double n = 3.0 * B * s->opt.crop * s->opt.crop;   // values inside the loss squares
    timed(s, "student.mse", 3.0 * n, 12.0 * n, 2, st, [&] {
        mse_grad_kernel<<<nblk, RED_T, 0, st>>>(s->out.as<float>(), xp, 16 * Hy, 16 * Wy, cr, S, 16 * s->opt.halo,
                                                s->opt.crop, (float)(2.0 / n), s->dz[3].as<float>(),
                                                s->lpart.as<double>());
        mse_final_kernel<<<1, RED_T, 0, st>>>(s->lpart.as<double>(), nblk, n, s->loss.as<float>());
    });
    // backward, l = 3 .. 0
    int H = S / 2;   // h_3 resolution
    for (int l = NL - 1; l >= 0; --l) {
        const int Cin = s->cin[l], Cout = s->cout[l];
        const bool xb = act_bytes(s, l) == 2, db = act_bytes(s, l) == 2 && l < NL - 1;
        const void *hl = s->h[l].p;
        const void *dzl = s->dz[l].p;
        const int64_t P_in = (int64_t)B * H * H;      // pixels of h_l
        const int64_t P_out = 4 * P_in;               // pixels of dz_l
        // bias gradient: pixel slices sized so that about 4 x 148 blocks run
        {
            const int64_t per = std::max<int64_t>(64, (P_out + BG_BLOCKS - 1) / BG_BLOCKS);
            const int nz = (int)((P_out + per - 1) / per);
            timed(s, "student.bgrad" + std::to_string(l), (double)P_out * Cout, 4.0 * P_out * Cout, 2, st, [&] {
                if (db)
                    chan_sum_kernel<<<nz, RED_T, 0, st>>>(static_cast<const __nv_bfloat16 *>(dzl), P_out, Cout, per,
                                                          s->bpart.as<float>());
                else
                    chan_sum_kernel<<<nz, RED_T, 0, st>>>(static_cast<const float *>(dzl), P_out, Cout, per,
                                                          s->bpart.as<float>());
                chan_sum_final_kernel<<<Cout, RED_T, 0, st>>>(s->bpart.as<float>(), nz, Cout,
                                                              s->grad.as<float>() + s->boff[l]);
            });
        }
        // weight gradient, BF16 form: the tcgen05 kernel over pixel slices, then the slices in order
        if (s->bf16 && l < NL - 1) {
            const double flop = 2.0 * P_in * (double)Cin * Cout * 25;
            const double bytes = P_in * (double)Cin * 2 + P_out * (double)Cout * 2 + 4.0 * wsize(s, l);
            const int ns = tc::wgrad_bf16_slices(B, H, H);
            timed(s, "student.wgrad" + std::to_string(l) + ":tc", flop, bytes, 2, st, [&] {
                float *part = s->part.as<float>();
                if (!tc::launch_wgrad_bf16(hl, dzl, B, H, H, Cin, part, s->status.as<uint32_t>(), st))
                    s->launch_failed = true;
                const int64_t ne = (int64_t)Cin * 25 * Cout;
                wgrad_reduce_kernel<<<wgrad_reduce_grid(ne), 32 * WR_G, 0, st>>>(part, ns, Cin, Cout,
                                                                                  s->grad.as<float>() + s->woff[l]);
            });
        } else if (l == NL - 1) {
            // the 3-channel layer: float32 outer products over dz windows staged in shared memory
            const double flop = 2.0 * P_in * (double)Cin * Cout * 25;
            const double bytes = P_in * (double)Cin * 4 + P_out * (double)Cout * 4 + 4.0 * wsize(s, l);
            int nb = 0, per = 0;
            wgrad3_plan(B, H, H, Cin, &nb, &per);
            timed(s, "student.wgrad" + std::to_string(l), flop, bytes, 2, st, [&] {
                float *part = s->part.as<float>();
                wgrad3_kernel<<<nb, W3_T, W3_SMEM, st>>>(static_cast<const float *>(hl), static_cast<const float *>(dzl),
                                                   B, H, H, Cin, per, part);
                const int64_t ne = (int64_t)Cin * 25 * Cout;
                wgrad_reduce_kernel<<<wgrad_reduce_grid(ne), 32 * WR_G, 0, st>>>(part, nb, Cin, Cout,
                                                                                  s->grad.as<float>() + s->woff[l]);
            });
        } else
        // weight gradient: split K so that the grid covers the SMs a few times
        {
            const int N = 25 * Cout;
            const int tn = (N + WG_BN - 1) / WG_BN, tm = (Cin + WG_BM - 1) / WG_BM;
            int64_t splits = std::max<int64_t>(1, (4 * 148) / (tn * tm));
            int64_t kper = (P_in + splits - 1) / splits;
            kper = std::max<int64_t>(WG_BK, (kper + WG_BK - 1) / WG_BK * WG_BK);
            splits = (P_in + kper - 1) / kper;
            const double flop = 2.0 * P_in * (double)Cin * Cout * 25;
            const double bytes = P_in * (double)Cin * act_bytes(s, l) + P_out * (double)Cout * act_bytes(s, l) +
                                 4.0 * wsize(s, l);
            timed(s, "student.wgrad" + std::to_string(l), flop, bytes, 2, st, [&] {
                dim3 grid(tn, tm, (unsigned)splits);
                const bool vec = Cout % WG_BN == 0;
                float *part = s->part.as<float>();
                if (xb && db)
                    launch_wgrad<__nv_bfloat16, __nv_bfloat16>(vec, grid, st, hl, dzl, B, H, Cin, Cout, kper, part);
                else if (!xb && !db)
                    launch_wgrad<float, float>(vec, grid, st, hl, dzl, B, H, Cin, Cout, kper, part);
                else
                    s->launch_failed = true;
                const int64_t ne = (int64_t)Cin * N;
                wgrad_reduce_kernel<<<wgrad_reduce_grid(ne), 32 * WR_G, 0, st>>>(
                    part, (int)splits, Cin, Cout, s->grad.as<float>() + s->woff[l]);
            });
        }
        // input gradient through the ReLU: dz_{l-1} = conv5x5/2(dz_l; W_l) * [h_l > 0]
        if (l > 0) {
            const double flop = 2.0 * P_in * (double)Cin * Cout * 25;
            const double bytes = P_out * (double)Cout * act_bytes(s, l) + 2.0 * P_in * Cin * act_bytes(s, l - 1) +
                                 4.0 * wsize(s, l);
            const bool tc = s->bf16 && l < NL - 1;
            if (l == NL - 1 && Cin == 64) {
                int nb = 0, per = 0;
                dgrad3_plan(B, H, H, &nb, &per);
                timed(s, "student.dgrad" + std::to_string(l), flop, bytes, 1, st, [&] {
                    if (act_bytes(s, l - 1) == 2)
                        dgrad3_kernel<<<nb, D3_T, D3_SMEM, st>>>(static_cast<const float *>(dzl), s->wd[l].as<float>(),
                                                                 static_cast<const float *>(hl), B, H, H, per,
                                                                 s->dz[l - 1].as<__nv_bfloat16>());
                    else
                        dgrad3_kernel<<<nb, D3_T, D3_SMEM, st>>>(static_cast<const float *>(dzl), s->wd[l].as<float>(),
                                                                 static_cast<const float *>(hl), B, H, H, per,
                                                                 s->dz[l - 1].as<float>());
                });
            } else
            timed(s, "student.dgrad" + std::to_string(l) + (tc ? ":tc" : ""), flop, bytes, 1, st, [&] {
                ConvDesc d{};
                d.in = static_cast<const float *>(dzl);
                d.out = static_cast<float *>(s->dz[l - 1].p);
                d.bias = nullptr;
                d.gdn_x = static_cast<const float *>(hl);
                d.status = s->status.as<uint32_t>();
                d.B = B;
                d.Hi = 2 * H;
                d.Wi = 2 * H;
                d.Cin = Cout;
                d.Gh = H;
                d.Gw = H;
                d.s = 2;
                d.Ho = H;
                d.Wo = H;
                d.Cout = Cin;
                d.oym = 1;
                d.oxm = 1;
                d.T = 25;
                for (int u = 0; u < 5; ++u)
                    for (int v = 0; v < 5; ++v) {
                        d.du[u * 5 + v] = (int8_t)(u - 2);
                        d.dv[u * 5 + v] = (int8_t)(v - 2);
                    }
                d.in_xform = IN_NONE;
                d.epi = EPI_MASK;
                d.in_scale = d.out_scale = 1.f;
                d.out_dt = act_bytes(s, l - 1) == 2 ? DT_BF16 : DT_F32;
                if (tc) {
                    d.in_dt = DT_BF16;
                    if (!tc::launch_lp_map(d, s->dmap[l], st)) s->launch_failed = true;
                } else {
                    d.in_dt = DT_F32;
                    d.w = s->wd[l].as<float>();
                    launch_conv_simt(d, st);
                }
            });
        }
        H /= 2;
    }
    LIC_CUDA_TRY(cudaGetLastError());
    return s->launch_failed ? LIC_E_UNSUPPORTED : LIC_OK;
}

int check_status(lic_student *s) {
    uint32_t v = 0;
    LIC_CUDA_TRY(cudaMemcpy(&v, s->status.p, 4, cudaMemcpyDeviceToHost));
    if (v) {
        LIC_CUDA_TRY(cudaMemset(s->status.p, 0, 4));
        return LIC_E_TIMEOUT;
    }
    return LIC_OK;
}

int read_loss(lic_student *s, float *loss, cudaStream_t st) {
    if (!loss) return LIC_OK;
    LIC_CUDA_TRY(cudaMemcpyAsync(loss, s->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st));
    LIC_CUDA_TRY(cudaStreamSynchronize(st));
    return check_status(s);
}

cudaStream_t SS(void *p) { return static_cast<cudaStream_t>(p); }

}  // namespace

// used by the codec (api.cu)
int student_channels(const lic_student *s) { return s ? s->M : 0; }

int student_forward_nhwc(lic_student *s, const float *yhat, int B, int Hy, int Wy, float *out, cudaStream_t st) {
    const int64_t p1 = (int64_t)B * 2 * Hy * 2 * Wy;
    int rc;
    if ((rc = ensure_e(s->ih[1], p1 * s->C, act_bytes(s, 1))) || (rc = ensure_e(s->ih[2], 4 * p1 * s->C, act_bytes(s, 2))) ||
        (rc = ensure_e(s->ih[3], 16 * p1 * s->C, act_bytes(s, 3))))
        return rc;
    const void *h0 = yhat;
    if (s->bf16) {
        const int64_t ny = (int64_t)B * Hy * Wy * s->M;
        if ((rc = ensure_e(s->ih[0], ny, 2))) return rc;
        timed(s, "student.to_bf16", 0, 6.0 * ny, 1, st, [&] { launch_to_bf16(yhat, ny, s->ih[0].p, st); });
        h0 = s->ih[0].p;
    }
    s->launch_failed = false;
    forward_all(s, h0, B, Hy, Wy, s->ih, out, st);
    LIC_CUDA_TRY(cudaGetLastError());
    return s->launch_failed ? LIC_E_UNSUPPORTED : LIC_OK;
}

void launch_student_check(const float *xs, float *xt, int B, int Hp, int Wp, int H, int W, float thr, double *part,
                          float *psnr, int *pass, long long *counts, cudaStream_t st) {
    const int nblk = 64;
    frame_sse_kernel<<<dim3(nblk, B), RED_T, 0, st>>>(xs, xt, Hp, Wp, H, W, part);
    frame_psnr_kernel<<<1, ((B + 31) / 32) * 32, 0, st>>>(part, nblk, B, 3.0 * H * W, thr, psnr, pass, counts);
    const int64_t per = (int64_t)Hp * Wp * 3;
    frame_select_kernel<<<grid_for(per * B, 256), 256, 0, st>>>(xs, xt, per, B, pass);
}

}  // namespace lic

using namespace lic;

int lic_student_create(const lic_weights *init, int M, int C, const lic_student_options *opt, lic_student **out) {
    if (!init || !opt || !out || M < 16 || C < 16 || M % 16 || C % 16 || C > RED_T) return LIC_E_INVALID_ARG;
    *out = nullptr;
    if ((opt->precision != LIC_FP32 && opt->precision != LIC_BF16) || opt->max_batch < 1 ||
        opt->max_batch > LIC_STUDENT_MAX_BATCH || opt->crop < 32 || opt->crop % 16 || opt->halo < 0 ||
        opt->halo > 8 || !(opt->lr > 0.f) ||
        !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f) || !(opt->eps > 0.f))
        return LIC_E_INVALID_ARG;
    // the bf16 tensor-core kernel takes 64-channel chunks and 64 outputs
    if (opt->precision == LIC_BF16 && (C != 64 || M % 64)) return LIC_E_UNSUPPORTED;
    for (int r : opt->reserved)
        if (r) return LIC_E_INVALID_ARG;
    auto s = new (std::nothrow) lic_student();
    if (!s) return LIC_E_OOM;
    s->M = M;
    s->C = C;
    s->opt = *opt;
    s->bf16 = opt->precision == LIC_BF16;
    cudaGetDevice(&s->device);
    const int ch[5] = {M, C, C, C, 3};
    std::vector<float> host;
    for (int l = 0; l < NL; ++l) {
        s->cin[l] = ch[l];
        s->cout[l] = ch[l + 1];
        s->woff[l] = s->nparam;
        s->nparam += wsize(s, l);
        s->boff[l] = s->nparam;
        s->nparam += s->cout[l];
    }
    host.assign((size_t)s->nparam, 0.f);
    auto fail = [&](int rc) {
        delete s;
        return rc;
    };
    for (int l = 0; l < NL; ++l) {
        const std::string base = "student.deconv" + std::to_string(l);
        for (int which = 0; which < 2; ++which) {
            const std::string name = base + (which ? ".bias" : ".weight");
            const int64_t want = which ? s->cout[l] : wsize(s, l);
            const float *src = nullptr;
            for (int i = 0; i < init->count; ++i)
                if (init->params[i].name && name == init->params[i].name) {
                    if (init->params[i].numel != want || !init->params[i].data) return fail(LIC_E_INVALID_ARG);
                    src = init->params[i].data;
                }
            if (!src) return fail(LIC_E_INVALID_ARG);
            memcpy(host.data() + (which ? s->boff[l] : s->woff[l]), src, (size_t)want * sizeof(float));
        }
    }
    int rc;
    const int64_t np = s->nparam;
    if ((rc = ensure_f(s->param, np)) || (rc = ensure_f(s->grad, np)) || (rc = ensure_f(s->adam_m, np)) ||
        (rc = ensure_f(s->adam_v, np)))
        return fail(rc);
    if (cudaMemcpy(s->param.p, host.data(), np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->grad.p, 0, np * sizeof(float)) != cudaSuccess ||
        cudaMemset(s->adam_m.p, 0, np * sizeof(float)) != cudaSuccess ||
        cudaMemset(s->adam_v.p, 0, np * sizeof(float)) != cudaSuccess)
        return fail(LIC_E_CUDA);
    for (int l = 0; l < NL - 1; ++l) {
        if (!s->bf16) {
            if ((rc = ensure_f(s->wf[l], wsize(s, l)))) return fail(rc);
            continue;
        }
        if ((rc = ensure_e(s->wfb[l], wsize(s, l), 2))) return fail(rc);
        for (int ph = 0; ph < 4; ++ph) {
            const void *base = s->wfb[l].as<__nv_bfloat16>() + (int64_t)ph_off(ph) * s->cout[l] * s->cin[l];
            if (!tc::make_bf16_weight_map(&s->fmap[l][ph], base, s->cout[l], ph_taps(ph) * s->cin[l]))
                return fail(LIC_E_UNSUPPORTED);
        }
    }
    for (int l = 1; l < NL; ++l) {
        if (s->bf16 && l < NL - 1) {
            if ((rc = ensure_e(s->wdb[l], wsize(s, l), 2))) return fail(rc);
            if (!tc::make_bf16_weight_map(&s->dmap[l], s->wdb[l].p, s->cin[l], 25 * s->cout[l]))
                return fail(LIC_E_UNSUPPORTED);
        } else if ((rc = ensure_f(s->wd[l], wsize(s, l)))) {
            return fail(rc);
        }
    }
    if ((rc = ensure_f(s->ws, (int64_t)s->cin[3] * 25 * 4))) return fail(rc);
    if (cudaMemset(s->ws.p, 0, s->ws.bytes) != cudaSuccess) return fail(LIC_E_CUDA);
    // training workspace
    const int Bm = opt->max_batch, S = 16 * window_lat(s);
    int64_t side = S / 16;
    if ((rc = ensure_e(s->h[0], Bm * side * side * M, act_bytes(s, 0)))) return fail(rc);
    for (int l = 1; l < NL; ++l) {
        side *= 2;
        if ((rc = ensure_e(s->h[l], Bm * side * side * C, act_bytes(s, l)))) return fail(rc);
    }
    side = S / 16;
    int64_t part_max = 0;
    for (int l = 0; l < NL; ++l) {
        side *= 2;   // dz_l lives at layer l's output resolution
        if ((rc = ensure_e(s->dz[l], Bm * side * side * s->cout[l], act_bytes(s, l)))) return fail(rc);
        const int N = 25 * s->cout[l];
        const int tiles = ((N + WG_BN - 1) / WG_BN) * ((s->cin[l] + WG_BM - 1) / WG_BM);
        const int64_t P_in = Bm * (side / 2) * (side / 2);
        const int64_t splits = std::min<int64_t>(std::max<int64_t>(1, (4 * 148) / tiles), (P_in + WG_BK - 1) / WG_BK);
        part_max = std::max<int64_t>(part_max, (splits + 1) * (int64_t)s->cin[l] * N);
        if (l == NL - 1) {   // the 3-channel layer's blocks
            int nb = 0, per = 0;
            wgrad3_plan(Bm, (int)(side / 2), (int)(side / 2), s->cin[l], &nb, &per);
            part_max = std::max<int64_t>(part_max, (int64_t)W3_BLOCKS * s->cin[l] * N);
        }
        if (s->bf16 && l < NL - 1)   // the tensor-core weight gradient's slices, for any batch up to Bm
            for (int b = 1; b <= Bm; ++b)
                part_max = std::max<int64_t>(part_max, (int64_t)tc::wgrad_bf16_slices(b, (int)(side / 2),
                                                                                      (int)(side / 2)) *
                                                           s->cin[l] * N);
    }
    if ((rc = ensure_f(s->out, (int64_t)Bm * S * S * 3)) || (rc = ensure_f(s->part, part_max)) ||
        (rc = ensure_f(s->bpart, (int64_t)(BG_BLOCKS + 1) * RED_T)) ||
        (rc = ensure_f(s->loss, 1)))
        return fail(rc);
    if (s->lpart.ensure(sizeof(double) * 148 * 16) != cudaSuccess || s->status.ensure(16) != cudaSuccess)
        return fail(LIC_E_OOM);
    cudaMemset(s->status.p, 0, 16);
    if (cudaFuncSetAttribute(wgrad3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, W3_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(dgrad3_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, D3_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(dgrad3_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, D3_SMEM) !=
            cudaSuccess)
        return fail(LIC_E_CUDA);
    if ((rc = repack(s, 0))) return fail(rc);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(LIC_E_CUDA);
    *out = s;
    return LIC_OK;
}

void lic_student_destroy(lic_student *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    delete s;
}

int lic_student_grad(lic_student *s, const float *yp, const float *xp, int P, int Hy, int Wy, const int32_t *crops,
                     int B, float *loss, void *stream) {
    if (!s) return LIC_E_INVALID_ARG;
    cudaStream_t st = SS(stream);
    int rc = grad_pass(s, yp, xp, P, Hy, Wy, crops, B, st);
    if (rc) return rc;
    return read_loss(s, loss, st);
}

int lic_student_step(lic_student *s, const float *yp, const float *xp, int P, int Hy, int Wy, const int32_t *crops,
                     int B, float *loss, void *stream) {
    if (!s) return LIC_E_INVALID_ARG;
    cudaStream_t st = SS(stream);
    int rc = grad_pass(s, yp, xp, P, Hy, Wy, crops, B, st);
    if (rc) return rc;
    s->t += 1;
    const double b1 = s->opt.beta1, b2 = s->opt.beta2;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)s->t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)s->t)));
    const int64_t n = s->nparam;
    timed(s, "student.adam", 12.0 * n, 28.0 * n, 1, st, [&] {
        adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->param.as<float>(), s->adam_m.as<float>(),
                                                                 s->adam_v.as<float>(), s->grad.as<float>(), n,
                                                                 s->opt.lr, s->opt.beta1, s->opt.beta2, c1, c2,
                                                                 s->opt.eps);
    });
    LIC_CUDA_TRY(cudaGetLastError());
    if ((rc = repack(s, st))) return rc;
    return read_loss(s, loss, st);
}

int lic_student_read(lic_student *s, const char *name, int what, float *dst, int64_t numel) {
    if (!s || !name || !dst || what < 0 || what > 3) return LIC_E_INVALID_ARG;
    const DevBuf *src[4] = {&s->param, &s->grad, &s->adam_m, &s->adam_v};
    for (int l = 0; l < NL; ++l) {
        const std::string base = "student.deconv" + std::to_string(l);
        int64_t off = -1, n = 0;
        if (base + ".weight" == name) {
            off = s->woff[l];
            n = wsize(s, l);
        } else if (base + ".bias" == name) {
            off = s->boff[l];
            n = s->cout[l];
        }
        if (off < 0) continue;
        if (n != numel) return LIC_E_INVALID_ARG;
        LIC_CUDA_TRY(cudaDeviceSynchronize());
        LIC_CUDA_TRY(cudaMemcpy(dst, src[what]->as<float>() + off, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
        return LIC_OK;
    }
    return LIC_E_INVALID_ARG;
}

namespace {
// n values of a float32 or bf16 device tensor -> host float32 (synchronous)
int copy_widened(const void *src, bool bf16, float *dst, int64_t n) {
    LIC_CUDA_TRY(cudaDeviceSynchronize());
    if (!bf16) {
        LIC_CUDA_TRY(cudaMemcpy(dst, src, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
        return LIC_OK;
    }
    std::vector<uint16_t> raw((size_t)n);
    LIC_CUDA_TRY(cudaMemcpy(raw.data(), src, (size_t)n * 2, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t u = (uint32_t)raw[i] << 16;
        memcpy(dst + i, &u, 4);
    }
    return LIC_OK;
}
}  // namespace

int lic_student_read_activation(lic_student *s, int layer, float *dst, int64_t numel) {
    if (!s || !dst || layer < 0 || layer > 3 || s->last_B < 1) return LIC_E_INVALID_ARG;
    const int64_t side = (int64_t)((16 * window_lat(s)) >> (4 - layer));
    const int ch = layer == 0 ? s->M : s->C;
    if (numel != (int64_t)s->last_B * side * side * ch) return LIC_E_INVALID_ARG;
    return copy_widened(s->h[layer].p, act_bytes(s, layer) == 2, dst, numel);
}

int lic_student_read_output_grad(lic_student *s, int layer, float *dst, int64_t numel) {
    if (!s || !dst || layer < 0 || layer > 3 || s->last_B < 1) return LIC_E_INVALID_ARG;
    const int64_t side = (int64_t)((16 * window_lat(s)) >> (3 - layer));
    if (numel != (int64_t)s->last_B * side * side * s->cout[layer]) return LIC_E_INVALID_ARG;
    return copy_widened(s->dz[layer].p, act_bytes(s, layer) == 2, dst, numel);
}

int64_t lic_student_steps(const lic_student *s) { return s ? s->t : LIC_E_INVALID_ARG; }

int lic_student_forward(lic_student *s, const float *yhat, int B, int Hy, int Wy, float *x, void *stream) {
    if (!s || !yhat || !x || B < 1 || Hy < 1 || Wy < 1) return LIC_E_INVALID_ARG;
    cudaStream_t st = SS(stream);
    const int64_t ny = (int64_t)B * s->M * Hy * Wy, nx = (int64_t)B * 3 * 256 * Hy * Wy;
    int rc;
    if ((rc = ensure_f(s->iout, 2 * nx + ny))) return rc;
    const bool dy = is_device_ptr(yhat), dx = is_device_ptr(x);
    float *nhwc_y = s->iout.as<float>() + 2 * nx;   // y_hat NHWC
    const float *ysrc = yhat;
    float *stage = s->iout.as<float>() + nx;        // NCHW staging next to the NHWC output
    if (!dy) {
        LIC_CUDA_TRY(cudaMemcpyAsync(stage, yhat, (size_t)ny * sizeof(float), cudaMemcpyHostToDevice, st));
        ysrc = stage;
    }
    timed(s, "student.nchw_to_nhwc", 0, 8.0 * ny, 1, st,
          [&] { launch_nchw_to_nhwc(ysrc, B, s->M, Hy, Wy, nhwc_y, st); });
    if ((rc = student_forward_nhwc(s, nhwc_y, B, Hy, Wy, s->iout.as<float>(), st))) return rc;
    float *dst = dx ? x : stage;
    timed(s, "student.nhwc_to_nchw", 0, 8.0 * nx, 1, st,
          [&] { launch_nhwc_to_nchw(s->iout.as<float>(), B, 16 * Hy, 16 * Wy, 3, dst, st); });
    if (!dx) {
        LIC_CUDA_TRY(cudaMemcpyAsync(x, stage, (size_t)nx * sizeof(float), cudaMemcpyDeviceToHost, st));
        LIC_CUDA_TRY(cudaStreamSynchronize(st));
        if ((rc = check_status(s))) return rc;
    }
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

int lic_student_profile_enable(lic_student *s, int enable) {
    if (!s) return LIC_E_INVALID_ARG;
    s->pf.enable(enable != 0);
    return LIC_OK;
}

int lic_student_profile_report(lic_student *s, char *buf, int cap) {
    return s ? s->pf.report(buf, cap) : LIC_E_INVALID_ARG;
}

int64_t lic_student_launch_count(const lic_student *s) { return s ? s->pf.launches : LIC_E_INVALID_ARG; }
