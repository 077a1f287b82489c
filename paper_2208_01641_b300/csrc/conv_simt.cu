// CUDA-core (SIMT) implicit-GEMM convolution over NHWC float32 tensors.
//
// One kernel serves every conv-like step of the chain through ConvDesc:
//   * strided 5x5 convolutions of g_a and h_a (Ballé 2017 [1], 2018 [2]),
//   * 3x3 stride-1 convolutions of h_a / h_s,
//   * each of the four sub-pixel phases of a 5x5 stride-2 transposed
//     convolution (g_s, h_s): output pixels (2m+py, 2n+px) of one phase form
//     a stride-1 convolution of the input with a 3x3, 3x2, 2x3 or 2x2 subset
//     of the taps,
//   * the GDN / IGDN normalisation of [9] as a 1x1 "convolution" of x^2 with
//     gamma plus beta, whose epilogue multiplies x by rsqrt(norm) (GDN) or
//     sqrt(norm) (IGDN).
// Every output element is one float32 sum over K = T * Cin in a fixed order
// (taps, then channels), so results do not depend on the batch position or
// the launch.  This is the exact FP32 path the tensor-core kernels are
// measured against, and it runs the layers those kernels do not cover.
#include <cuda_bf16.h>

#include "lic_internal.h"

namespace lic {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ float xform(float v, int mode) {
    return mode == IN_ABS ? fabsf(v) : (mode == IN_SQUARE ? v * v : v);
}

template <bool VEC>
__global__ void __launch_bounds__(NT) conv_simt_kernel(const ConvDesc d) {
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t rows = (int64_t)d.B * d.Gh * d.Gw;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int K = d.T * d.Cin;

    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    // the pixel this thread loads in the vectorised path
    const int lp = tid / 4, lq = tid % 4;
    int lb = 0, li = 0, lj = 0;
    bool lvalid = false;
    {
        int64_t r = row0 + lp;
        if (r < rows) {
            lvalid = true;
            lb = (int)(r / ((int64_t)d.Gh * d.Gw));
            int rem = (int)(r % ((int64_t)d.Gh * d.Gw));
            li = rem / d.Gw;
            lj = rem % d.Gw;
        }
    }

    for (int k0 = 0; k0 < K; k0 += BK) {
        // ---- A tile: BM pixels x BK of K ----
        if (VEC) {
            const int t = k0 / d.Cin, c0 = k0 % d.Cin;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lvalid) {
                int yi = d.s * li + d.du[t], xi = d.s * lj + d.dv[t];
                if (yi >= 0 && yi < d.Hi && xi >= 0 && xi < d.Wi) {
                    const float *p = d.in + (((int64_t)lb * d.Hi + yi) * d.Wi + xi) * d.Cin + c0 + 4 * lq;
                    v = *reinterpret_cast<const float4 *>(p);
                }
            }
            As[4 * lq + 0][lp] = xform(v.x, d.in_xform);
            As[4 * lq + 1][lp] = xform(v.y, d.in_xform);
            As[4 * lq + 2][lp] = xform(v.z, d.in_xform);
            As[4 * lq + 3][lp] = xform(v.w, d.in_xform);
        } else {
#pragma unroll
            for (int r = 0; r < (BM * BK) / NT; ++r) {
                int e = tid + r * NT;
                int p = e / BK, kk = e % BK;
                int k = k0 + kk;
                float v = 0.f;
                int64_t rr = row0 + p;
                if (k < K && rr < rows) {
                    int t = k / d.Cin, c = k % d.Cin;
                    int b = (int)(rr / ((int64_t)d.Gh * d.Gw));
                    int rem = (int)(rr % ((int64_t)d.Gh * d.Gw));
                    int i = rem / d.Gw, j = rem % d.Gw;
                    int yi = d.s * i + d.du[t], xi = d.s * j + d.dv[t];
                    if (yi >= 0 && yi < d.Hi && xi >= 0 && xi < d.Wi)
                        v = d.in[(((int64_t)b * d.Hi + yi) * d.Wi + xi) * d.Cin + c];
                }
                As[kk][p] = xform(v, d.in_xform);
            }
        }
        // ---- B tile: BK of K x BN output channels (weights [Cout][K]) ----
        if (VEC) {
            const int n = n0 + tid / 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n < d.Cout) v = *reinterpret_cast<const float4 *>(d.w + (int64_t)n * K + k0 + 4 * lq);
            Bs[4 * lq + 0][tid / 4] = v.x;
            Bs[4 * lq + 1][tid / 4] = v.y;
            Bs[4 * lq + 2][tid / 4] = v.z;
            Bs[4 * lq + 3][tid / 4] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < (BN * BK) / NT; ++r) {
                int e = tid + r * NT;
                int nn = e / BK, kk = e % BK;
                int n = n0 + nn, k = k0 + kk;
                Bs[kk][nn] = (n < d.Cout && k < K) ? d.w[(int64_t)n * K + k] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }

    // ---- epilogue ----
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = row0 + ty * 4 + i;
        if (r >= rows) continue;
        int b = (int)(r / ((int64_t)d.Gh * d.Gw));
        int rem = (int)(r % ((int64_t)d.Gh * d.Gw));
        int gi = rem / d.Gw, gj = rem % d.Gw;
        int oy = d.oym * gi + d.oyo, ox = d.oxm * gj + d.oxo;
        int64_t opix = ((int64_t)b * d.Ho + oy) * d.Wo + ox;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx * 4 + j;
            if (n >= d.Cout) continue;
            float v = acc[i][j] + (d.bias ? d.bias[n] : 0.f);
            if (d.epi == EPI_RELU) {
                v = fmaxf(v, 0.f);
            } else if (d.epi == EPI_GDN) {
                v = d.gdn_x[opix * d.Cout + n] * rsqrtf(v);
            } else if (d.epi == EPI_IGDN) {
                v = d.gdn_x[opix * d.Cout + n] * sqrtf(v);
            } else if (d.epi == EPI_MASK) {
                v = d.gdn_x[opix * d.Cout + n] > 0.f ? v : 0.f;
            }
            if (d.out_dt == DT_BF16)
                reinterpret_cast<__nv_bfloat16 *>(d.out)[opix * d.Cout + n] = __float2bfloat16_rn(v);
            else
                d.out[opix * d.Cout + n] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Transposed conv to <= 4 channels (the last layer of g_s).  Input position
// (m, n) feeds output pixels (2m + py, 2n + px) through tap u = py + 2 - 2 du
// of input row m + du (du in {-1, 0, 1}, valid when 0 <= u <= 4), likewise
// for columns: all four phases at (m, n) read only the 3 x 3 neighbourhood
// of (m, n).  A thread owns a 2 x 2 block of input positions -- 16 output
// pixels -- so its 4 x 4 input neighbourhood and every (broadcast) weight
// load are shared by four positions; the kernel is bound by FMA issue.
constexpr int DS_TR = 8, DS_TC = 64, DS_CH = 8, DS_THREADS = 128;
constexpr int DS_PITCH = DS_TC + 4;   // row pitch in floats

template <int COUT>
__global__ void __launch_bounds__(DS_THREADS) deconv_small_kernel(const float *__restrict__ in, int B, int Hi,
                                                                  int Wi, int Cin, const float *__restrict__ w,
                                                                  const float *__restrict__ bias,
                                                                  float *__restrict__ out) {
    __shared__ float xs[DS_CH][DS_TR + 2][DS_PITCH];
    __shared__ __align__(16) float ws[DS_CH][25][4];
    const int tid = threadIdx.x;
    const int tr = tid / 32, tc = tid % 32;      // positions (m0 + 2tr + a, n0 + 2tc + c)
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * DS_TR, n0 = blockIdx.x * DS_TC;
    float acc[2][2][2][2][COUT];                 // [a][c][py][px][o]
#pragma unroll
    for (int i = 0; i < 2 * 2 * 2 * 2 * COUT; ++i) (&acc[0][0][0][0][0])[i] = 0.f;

    for (int c0 = 0; c0 < Cin; c0 += DS_CH) {
        // input tile with a one-pixel halo, zero outside the image
        for (int e = tid; e < (DS_TR + 2) * (DS_TC + 2) * (DS_CH / 4); e += DS_THREADS) {
            const int q = e % (DS_CH / 4);
            const int pos = e / (DS_CH / 4);
            const int rr = pos / (DS_TC + 2), cc = pos % (DS_TC + 2);
            const int yi = m0 - 1 + rr, xi = n0 - 1 + cc;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (yi >= 0 && yi < Hi && xi >= 0 && xi < Wi)
                v = *reinterpret_cast<const float4 *>(in + (((int64_t)b * Hi + yi) * Wi + xi) * Cin + c0 + 4 * q);
            xs[4 * q + 0][rr][cc] = v.x;
            xs[4 * q + 1][rr][cc] = v.y;
            xs[4 * q + 2][rr][cc] = v.z;
            xs[4 * q + 3][rr][cc] = v.w;
        }
        for (int e = tid; e < DS_CH * 25; e += DS_THREADS) {
            const float4 v = *reinterpret_cast<const float4 *>(w + ((int64_t)(c0 + e / 25) * 25 + e % 25) * 4);
            *reinterpret_cast<float4 *>(&ws[e / 25][e % 25][0]) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < DS_CH; ++c) {
            float x[4][4];   // neighbourhood rows m0+2tr-1 .. +2, cols n0+2tc-1 .. +2
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) x[r][q] = xs[c][2 * tr + r][2 * tc + q];
#pragma unroll
            for (int py = 0; py < 2; ++py)
#pragma unroll
                for (int du = -1; du <= 1; ++du) {
                    const int u = py + 2 - 2 * du;
                    if (u < 0 || u > 4) continue;
#pragma unroll
                    for (int px = 0; px < 2; ++px)
#pragma unroll
                        for (int dv = -1; dv <= 1; ++dv) {
                            const int v = px + 2 - 2 * dv;
                            if (v < 0 || v > 4) continue;
                            const float4 wv = *reinterpret_cast<const float4 *>(&ws[c][u * 5 + v][0]);
                            const float wk[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                            for (int a = 0; a < 2; ++a)
#pragma unroll
                                for (int cc = 0; cc < 2; ++cc) {
                                    const float xv = x[1 + a + du][1 + cc + dv];
#pragma unroll
                                    for (int o = 0; o < COUT; ++o)
                                        acc[a][cc][py][px][o] = fmaf(xv, wk[o], acc[a][cc][py][px][o]);
                                }
                        }
                }
        }
        __syncthreads();
    }
    const int Ho = 2 * Hi, Wo = 2 * Wi;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int m = m0 + 2 * tr + a, n = n0 + 2 * tc + cc;
            if (m >= Hi || n >= Wi) continue;
#pragma unroll
            for (int py = 0; py < 2; ++py)
#pragma unroll
                for (int px = 0; px < 2; ++px) {
                    float *o = out + (((int64_t)b * Ho + 2 * m + py) * Wo + 2 * n + px) * COUT;
#pragma unroll
                    for (int k = 0; k < COUT; ++k) o[k] = acc[a][cc][py][px][k] + __ldg(bias + k);
                }
        }
}


// Second pass of the two-pass form (see launch_deconv_gather).  A block takes
// one row m of output quads (2m .. 2m+1, 2n .. 2n+1) for GQ_W consecutive n.
// Row m - 1 of C feeds the quads only through its (du = -1) blocks, row m
// through its (du = 0) blocks and row m + 1 through its (du = 1) blocks, each a
// contiguous run of every position's record: the block copies those three runs
// of the GQ_W + 2 positions it touches into a shared-memory record per position
// (coalesced 16-byte loads, zeros outside the grid; every C entry is read once),
// then thread t adds, in (du, dv) order, position n + dv's (du, dv) block to
// its quad's pixels (16-byte shared loads: the record pitch spreads a quarter
// warp over all 32 banks), adds the bias and writes the quad's two rows.
constexpr int GQ_W = 128;

template <int COUT>
__global__ void __launch_bounds__(GQ_W) deconv_gather_kernel(const float *__restrict__ C, int B, int Hi, int Wi,
                                                             const float *__restrict__ bias,
                                                             float *__restrict__ out) {
    constexpr int S = deconv_scatter_stride(COUT);
    extern __shared__ __align__(16) float rec[];   // [GQ_W + 2][S]: position n0 - 1 + k at k
    const int t = threadIdx.x, n0 = blockIdx.x * GQ_W, m = blockIdx.y, b = blockIdx.z;
    // every load of the three runs in flight before the first shared store
    constexpr int IT = ((GQ_W + 2) * (S / 4) + GQ_W - 1) / GQ_W;   // float4s a thread copies, at most
    float4 v[IT];
    int dst[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = t + i * GQ_W;   // float4 e of the block's (GQ_W + 2) x S / 4, row-part by row-part
        dst[i] = -1;
        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        int du = -1, base = 0;
        for (; du < 1; ++du) {        // the row part e falls in
            const int cnt = (GQ_W + 2) * ((scatter_offset(du + 1, -1, COUT) - scatter_offset(du, -1, COUT)) / 4);
            if (e < base + cnt) break;
            base += cnt;
        }
        const int off = scatter_offset(du, -1, COUT);
        const int nf = (scatter_offset(du + 1, -1, COUT) - off) / 4;
        const int r = e - base;
        if (r >= (GQ_W + 2) * nf) continue;   // past the last part
        const int k = r / nf, j = r % nf, ni = n0 - 1 + k, mi = m + du;
        dst[i] = k * S + off + 4 * j;
        if (mi >= 0 && mi < Hi && ni >= 0 && ni < Wi)
            v[i] = __ldcs(reinterpret_cast<const float4 *>(C + (((int64_t)b * Hi + mi) * Wi + ni) * S + off) + j);
    }
#pragma unroll
    for (int i = 0; i < IT; ++i)
        if (dst[i] >= 0) *reinterpret_cast<float4 *>(rec + dst[i]) = v[i];
    __syncthreads();
    const int n = n0 + t;
    if (n >= Wi) return;
    float acc[2][2][COUT];
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
        for (int px = 0; px < 2; ++px)
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[py][px][o] = 0.f;
#pragma unroll
    for (int du = -1; du <= 1; ++du) {
#pragma unroll
        for (int dv = -1; dv <= 1; ++dv) {
            const int nb = scatter_block(du, dv, COUT) / 4, npx = scatter_n(dv);
            const float4 *src = reinterpret_cast<const float4 *>(rec + (t + 1 + dv) * S + scatter_offset(du, dv, COUT));
            float blk[16];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j < nb) {
                    const float4 v = src[j];
                    blk[4 * j] = v.x;
                    blk[4 * j + 1] = v.y;
                    blk[4 * j + 2] = v.z;
                    blk[4 * j + 3] = v.w;
                }
            }
#pragma unroll
            for (int py = 0; py < scatter_n(du); ++py)
#pragma unroll
                for (int px = 0; px < npx; ++px)
#pragma unroll
                    for (int o = 0; o < COUT; ++o) acc[py][px][o] += blk[(py * npx + px) * COUT + o];
        }
    }
    const int Ho = 2 * Hi, Wo = 2 * Wi;
#pragma unroll
    for (int py = 0; py < 2; ++py) {
        float *dst = out + (((int64_t)b * Ho + 2 * m + py) * Wo + 2 * n) * COUT;
#pragma unroll
        for (int px = 0; px < 2; ++px)
#pragma unroll
            for (int o = 0; o < COUT; ++o) dst[px * COUT + o] = __ldg(bias + o) + acc[py][px][o];
    }
}

template <int COUT>
void gather_launch(const float *C, int B, int Hi, int Wi, const float *bias, float *out, cudaStream_t st) {
    const int smem = (GQ_W + 2) * deconv_scatter_stride(COUT) * (int)sizeof(float);
    static const bool attr =
        cudaFuncSetAttribute(deconv_gather_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
        cudaSuccess;
    (void)attr;
    const dim3 grid((unsigned)((Wi + GQ_W - 1) / GQ_W), (unsigned)Hi, (unsigned)B);
    deconv_gather_kernel<COUT><<<grid, GQ_W, smem, st>>>(C, B, Hi, Wi, bias, out);
}
}  // namespace

void launch_deconv_gather(const float *C, int B, int Hi, int Wi, int Cout, const float *bias, float *out,
                          cudaStream_t st) {
    if ((int64_t)B * Hi * Wi == 0) return;
    switch (Cout) {
        case 1: gather_launch<1>(C, B, Hi, Wi, bias, out, st); break;
        case 2: gather_launch<2>(C, B, Hi, Wi, bias, out, st); break;
        case 3: gather_launch<3>(C, B, Hi, Wi, bias, out, st); break;
        default: gather_launch<4>(C, B, Hi, Wi, bias, out, st); break;
    }
}

void launch_deconv_small(const float *in, int B, int Hi, int Wi, int Cin, const float *w, const float *bias, int Cout,
                         float *out, cudaStream_t st) {
    dim3 grid((Wi + DS_TC - 1) / DS_TC, (Hi + DS_TR - 1) / DS_TR, B);
    switch (Cout) {
        case 1: deconv_small_kernel<1><<<grid, DS_THREADS, 0, st>>>(in, B, Hi, Wi, Cin, w, bias, out); break;
        case 2: deconv_small_kernel<2><<<grid, DS_THREADS, 0, st>>>(in, B, Hi, Wi, Cin, w, bias, out); break;
        case 3: deconv_small_kernel<3><<<grid, DS_THREADS, 0, st>>>(in, B, Hi, Wi, Cin, w, bias, out); break;
        default: deconv_small_kernel<4><<<grid, DS_THREADS, 0, st>>>(in, B, Hi, Wi, Cin, w, bias, out); break;
    }
}

void launch_conv_simt(const ConvDesc &d, cudaStream_t st) {
    const int64_t rows = (int64_t)d.B * d.Gh * d.Gw;
    if (rows == 0) return;
    dim3 grid((unsigned)((rows + BM - 1) / BM), (unsigned)((d.Cout + BN - 1) / BN));
    const bool vec = (d.Cin % BK) == 0 && ((d.T * d.Cin) % BK) == 0;
    if (vec)
        conv_simt_kernel<true><<<grid, NT, 0, st>>>(d);
    else
        conv_simt_kernel<false><<<grid, NT, 0, st>>>(d);
}

}  // namespace lic
