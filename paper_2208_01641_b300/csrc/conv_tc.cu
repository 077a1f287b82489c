// Tensor-core (tcgen05) implicit-GEMM convolution for sm_103a, FP32-accurate
// through 3xTF32.
//
// The conv-like steps of g_a, g_s, h_a, h_s (Ballé 2017 [1], 2018 [2]) and the
// channel sums of GDN / IGDN [9] are dense contractions: GEMM rows are output
// pixels, columns output channels, K = taps x input channels.  One CTA owns
// a tile of 128 output pixels x all Cout channels:
//
//   warp 0      TMA producer: per K chunk (one tap, 32 input channels) a
//               128 x 32 float32 activation box and the 32-wide slices of
//               the split weights (hi, lo), 128-byte swizzled, into a stage
//   warp 1      allocates TMEM; one lane issues, per 8-wide K step,
//               D += Ahi*Bhi + Ahi*Blo + Alo*Bhi (kind::tf32) and commits each
//               stage back to the producer
//   warps 2..9  split each activation box in place into TF32 hi and lo parts
//               (x = hi + lo, both TF32-exact), fold partial sums (below),
//               then run the epilogue (bias, ReLU or GDN / IGDN)
//
// Dropping only Alo*Blo leaves a relative product error of about 2^-21.
//
// Accumulation: the tensor core adds each MMA's products into the TMEM
// accumulator with truncation, so one accumulator taking all K steps of a
// 3200-long reduction drifts toward zero by ~1e-5 relative.  The K chunks are
// therefore summed in groups of FOLD: each group into one of two TMEM partial
// buffers (ping-pong), and the epilogue warps fold every finished partial
// into a float32 master sum in registers with round-to-nearest adds, one
// group behind the MMAs so the folds overlap the main loop.
//
// The activation boxes are plain tiled TMA loads with out-of-range zero fill,
// which implements the zero padding of the convolution:
//   * stride 2: the NHWC input viewed as (2C, W/2, 2, H/2, B) -- an input
//     pixel pair shares one "row" of 2C values, and rows of one parity are
//     contiguous -- so input (2i + du, 2j + dv) for an R x Wt block of
//     outputs is one box at (wp*C + c0, j0 + (dv >> 1), du & 1, i0 + (du >> 1), b);
//   * stride 1 (3x3 convs, sub-pixel phases of the transposed convs):
//     (C, W, H, B) at (c0, j0 + dv, i0 + du, b);
//   * 1x1 (GDN): (C, rows) at (c0, p0).
// Every wait on an mbarrier is bounded; a wait that runs out latches
// ST_TIMEOUT in the codec status word and the CTA winds down.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "conv_tc.h"

namespace lic {
namespace tc {
namespace {

constexpr int BLOCK_M = 128;
constexpr int KCH = 32;                          // K chunk: 32 float32 = one 128-byte swizzle row
constexpr int A_BYTES = BLOCK_M * KCH * 4;       // 16 KB
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr int FOLD = 8;                          // K chunks per TMEM partial sum
constexpr int EPI_WARPS = 8;
constexpr int EPI_THREADS = EPI_WARPS * 32;

// MODE_IM2COL: inputs with few channels (the 3-channel frame into g_a): the
// epilogue warps gather each 128 x 32 slice of the im2col matrix (K index
// t * Cin + c, zero past T * Cin) straight from global memory, split it and
// write it swizzled into the stage; TMA brings only the weights.
// MODE_TAPS (persistent kernel, g_a conv0 over the padded 4-channel frame):
// K index 4 t + c, tap t = 5u + v; a K chunk is eight taps, each one TMA box
// of the 128 pixels' 4 channels (2 KB) through the stride-2 view, stacked in
// the no-swizzle K-major layout (8-row core matrices 128 bytes apart, taps
// 2 KB apart), so no patch rows exist in HBM.
enum Mode : int { MODE_S2 = 0, MODE_S1 = 1, MODE_FLAT = 2, MODE_IM2COL = 3, MODE_TAPS = 4 };
constexpr int TAP_BYTES = BLOCK_M * 16;   // one tap's box: 128 pixels x 4 float32

struct Params {
    float *out;
    const float *bias;
    const float *gdn_x;
    uint32_t *status;
    int mode, T, Cin, cpt;        // cpt: K chunks per tap
    int Gh, Gw, R, Wt, tiles_x, tiles_y, B;
    int64_t rows;                 // MODE_FLAT: total pixels
    int Ho, Wo, Cout;
    int oym, oyo, oxm, oxo;
    int epi, in_xform;
    const float *in;              // MODE_IM2COL: NHWC input
    int Hi, Wi, s;                // MODE_IM2COL: input size, stride
    int fuse_gdn;                 // 0, 1 (GDN) or 2 (IGDN) applied after bias
    int out_dt;                   // DType of the output
    int ostride, ocoff;           // output: elements per pixel, first channel (a column slice of a wider layer)
    float out_inv_scale;          // e4m3 output: stored = x * out_inv_scale
    float in_scale;               // e4m3 input: x = stored * in_scale
    const float *w_scale;         // e4m3 weights: per output channel
    const float *gdn_beta;
    const float *gdn_gamma;       // fuse_gdn 3 / 4 (1DN): per-channel gamma
    int kchunks;
    uint32_t tmem_cols;
    int ntiles;                   // conv_tcx_kernel: tiles of the launch
    int ksplit;                   // conv_tcx_kernel: K slices a tile is cut into (1: none)
    int out_stream;               // conv_tcx_kernel: output read once soon after; evict it from L2 first
    int8_t du[MAX_TAPS], dv[MAX_TAPS];
    // quantisation fused into the epilogue (see ConvDesc)
    int q_mode, q_C;
    int32_t *q_sym;
    float *q_hat;
    const float *q_mu;
    uint8_t *q_idx;
    const float *q_tab;
};

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// n arrivals at once (completes a phase that expects n)
__device__ __forceinline__ void mbar_arrive_n(uint64_t *bar, uint32_t n) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the phase did not complete within WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = WAIT_CYCLES) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1, int c2,
                                            int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6, %7}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

// Tensor stores from a 128-byte-swizzled shared-memory box (bulk groups of
// the issuing thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tm, const void *src, int c0, int c1) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1)
                 : "memory");
}

__device__ __forceinline__ void tma_store_5d(const CUtensorMap *tm, const void *src, int c0, int c1, int c2, int c3,
                                             int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(tm)),
        "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

// The same with an L2 cache policy (createpolicy: evict-first for output that
// is read once, so it does not displace weights and activations other
// launches reuse)
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tma_store_2d_hint(const CUtensorMap *tm, const void *src, int c0, int c1, uint64_t pol) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%2, %3}], [%1], %4;" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the committed stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the committed stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Warpgroup register budgets (every thread of the warpgroup executes these)
template <int N>
__device__ __forceinline__ void reg_release() { asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N)); }
template <int N>
__device__ __forceinline__ void reg_claim() { asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N)); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// A operand from tensor memory (lanes = rows, one 32-bit column per K element)
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])),
        "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])),
        "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])),
        "r"(__float_as_uint(v[23])), "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])),
        "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])),
        "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 columns at each of two TMEM addresses of this thread's lane, one wait for both
__device__ __forceinline__ void tmem_ld32x2(uint32_t ta, uint32_t tb, float *va, float *vb) {
    uint32_t r[32], q[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
          "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]),
          "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]),
          "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(q[i]);
    }
}

// 16 columns at each of two TMEM addresses of this thread's lane, one wait for both
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float *va, float *vb) {
    uint32_t r[16], q[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
          "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(q[i]);
    }
}

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16_f(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// Four floats -> four e4m3 bytes (round to nearest even, saturating), first in the low byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

// Store NV consecutive channels (NV % 16 == 0) of one pixel, element offset
// `off`, in the output storage type.
template <int NV>
__device__ __forceinline__ void store_row(const float *v, void *out, int64_t off, int dt, float inv_scale) {
    if (dt == DT_BF16) {
        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(out) + off);
#pragma unroll
        for (int q = 0; q < NV / 8; ++q)
            dst[q] = make_uint4(pack_bf16_f(v[8 * q], v[8 * q + 1]), pack_bf16_f(v[8 * q + 2], v[8 * q + 3]),
                                pack_bf16_f(v[8 * q + 4], v[8 * q + 5]), pack_bf16_f(v[8 * q + 6], v[8 * q + 7]));
    } else if (dt == DT_E4M3) {
        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(out) + off);
#pragma unroll
        for (int q = 0; q < NV / 16; ++q) {
            const float *w = v + 16 * q;
            dst[q] = make_uint4(
                pack_e4m3x4(w[0] * inv_scale, w[1] * inv_scale, w[2] * inv_scale, w[3] * inv_scale),
                pack_e4m3x4(w[4] * inv_scale, w[5] * inv_scale, w[6] * inv_scale, w[7] * inv_scale),
                pack_e4m3x4(w[8] * inv_scale, w[9] * inv_scale, w[10] * inv_scale, w[11] * inv_scale),
                pack_e4m3x4(w[12] * inv_scale, w[13] * inv_scale, w[14] * inv_scale, w[15] * inv_scale));
        }
    } else {
        float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + off);
#pragma unroll
        for (int q = 0; q < NV / 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

// ---- quantisation fused into an epilogue: the same arithmetic as the
// separate quantisation and scale-index kernels (layout.cu), so both decide
// every integer identically ----

__device__ __forceinline__ int32_t fq_symbol(float y, float mu) {
    const float d = __fsub_rn(y, mu);
    float r = rintf(d);
    if (r != r) r = 0.f;
    r = fminf(fmaxf(r, -1073741824.f), 1073741824.f);
    return (int32_t)r;
}

// The smallest k with tab[k] >= max(sg, tab[0]) (NaN or above tab[63]: 63):
// the scales are log-spaced (0.11 .. 256 in 63 steps), so log(sg / 0.11)
// over the step puts k within one of the answer, and comparisons with the
// table itself settle it -- the same k as a binary search of the table.
__device__ __forceinline__ uint8_t fq_index(float sg, const float *tab) {
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

// Channels c .. c+NV-1 (whole-layer numbering) of output pixel hw of frame b
// (NHWC pixel index opix for q_hat); tab: the scales in shared memory.
// QM 1: symbols (and q_hat), 2: scale indices.
template <int QM, int NV>
__device__ __forceinline__ void fused_quant_m(const Params &p, const float *v, int b, int64_t hw, int64_t HW, int c,
                                              int64_t opix, const float *tab) {
    const int64_t o0 = ((int64_t)b * p.q_C + c) * HW + hw;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int cc = c + j;
        const int64_t o = o0 + (int64_t)j * HW;
        if constexpr (QM == 1) {
            const float mu = p.q_mu ? __ldg(p.q_mu + cc) : 0.f;
            const int32_t sy = fq_symbol(v[j], mu);
            p.q_sym[o] = sy;
            if (p.q_hat) p.q_hat[opix * p.q_C + cc] = __fadd_rn(__int2float_rn(sy), mu);
        } else {
            p.q_idx[o] = fq_index(v[j], tab);
        }
    }
}

template <int NV>
__device__ __forceinline__ void fused_quant(const Params &p, const float *v, int b, int64_t hw, int64_t HW, int c,
                                            int64_t opix, const float *tab) {
    if (p.q_mode == 1) fused_quant_m<1, NV>(p, v, b, hw, HW, c, opix, tab);
    else fused_quant_m<2, NV>(p, v, b, hw, HW, c, opix, tab);
}

// Four consecutive per-channel parameters (16-byte aligned; the launch checks
// it) through the read-only path.
__device__ __forceinline__ float4 ld_param4(const float *src) { return __ldg(reinterpret_cast<const float4 *>(src)); }

// Divisive normalisation of one value: y / sqrt(n) (GDN) or y * sqrt(n)
// (inverse GDN).  n >= beta > 0, so sqrt(n) = n * rsqrt(n); both forms go
// through rsqrtf, which keeps the epilogue's loops free of the IEEE square
// root's slow-path branch.
template <bool INV>
__device__ __forceinline__ float norm_apply(float y, float n) {
    const float r = rsqrtf(n);
    return INV ? y * (n * r) : y * r;
}

// master[i] = norm_apply(master[i], n[i] + beta[i]) for NV channels
template <int NV, bool INV>
__device__ __forceinline__ void norm_n(float *master, const float *n, const float *beta) {
#pragma unroll
    for (int q = 0; q < NV / 4; ++q) {
        const float4 b = ld_param4(beta + 4 * q);
        master[4 * q + 0] = norm_apply<INV>(master[4 * q + 0], n[4 * q + 0] + b.x);
        master[4 * q + 1] = norm_apply<INV>(master[4 * q + 1], n[4 * q + 1] + b.y);
        master[4 * q + 2] = norm_apply<INV>(master[4 * q + 2], n[4 * q + 2] + b.z);
        master[4 * q + 3] = norm_apply<INV>(master[4 * q + 3], n[4 * q + 3] + b.w);
    }
}

// Per-channel (diagonal) norm of NV channels: y = master + bias (bias may be
// null), master = norm_apply(y, beta + gamma y^2)
template <int NV, bool INV>
__device__ __forceinline__ void norm_diag(float *master, const float *bias, const float *gamma, const float *beta) {
#pragma unroll
    for (int q = 0; q < NV / 4; ++q) {
        const float4 bi = bias ? ld_param4(bias + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 g = ld_param4(gamma + 4 * q), be = ld_param4(beta + 4 * q);
        const float bb[4] = {bi.x, bi.y, bi.z, bi.w}, gg[4] = {g.x, g.y, g.z, g.w}, ee[4] = {be.x, be.y, be.z, be.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float y = master[4 * q + e] + bb[e];
            master[4 * q + e] = norm_apply<INV>(y, fmaf(gg[e], y * y, ee[e]));
        }
    }
}

// master[i] += bias[i] for NV channels
template <int NV>
__device__ __forceinline__ void add_bias(float *master, const float *bias) {
#pragma unroll
    for (int q = 0; q < NV / 4; ++q) {
        const float4 b = ld_param4(bias + 4 * q);
        master[4 * q] += b.x; master[4 * q + 1] += b.y; master[4 * q + 2] += b.z; master[4 * q + 3] += b.w;
    }
}

// The ReLU's backward pass: zero v[i] wherever the activation m (same layout
// and storage type as the output, dt) is not positive.
template <int NV>
__device__ __forceinline__ void mask_row(float *v, const void *m, int64_t off, int dt) {
    if (dt == DT_BF16) {
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(m) + off);
#pragma unroll
        for (int q = 0; q < NV / 8; ++q) {
            const uint4 u = __ldg(src + q);
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t h = (w[j >> 1] >> (16 * (j & 1))) & 0xffffu;
                if ((h & 0x8000u) || !(h & 0x7fffu)) v[8 * q + j] = 0.f;
            }
        }
    } else {
        const float4 *src = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(m) + off);
#pragma unroll
        for (int q = 0; q < NV / 4; ++q) {
            const float4 u = __ldg(src + q);
            if (!(u.x > 0.f)) v[4 * q] = 0.f;
            if (!(u.y > 0.f)) v[4 * q + 1] = 0.f;
            if (!(u.z > 0.f)) v[4 * q + 2] = 0.f;
            if (!(u.w > 0.f)) v[4 * q + 3] = 0.f;
        }
    }
}

// Round to TF32 (10 stored mantissa bits), to nearest, ties away from zero:
// add half of the 13 dropped bits to the magnitude, then clear them.  Same
// result as cvt.rna.tf32.f32 for finite values, at integer-ALU rate.
// x with its low 13 mantissa bits cleared: the TF32 value the tensor core
// takes an FP32 operand for
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;            // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1u << 46;            // descriptor version
    d |= (uint64_t)2u << 61;            // SWIZZLE_128B
    return d;
}

// The same for the no-swizzle K-major layout of MODE_TAPS: 8-row core
// matrices (8 x 16 bytes, contiguous) 128 bytes apart along M (stride byte
// offset), taps TAP_BYTES apart along K (leading byte offset).
__device__ __forceinline__ uint64_t sdesc_taps(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((TAP_BYTES >> 4) & 0x3FFFu) << 16;   // leading byte offset: the next tap
    d |= (uint64_t)(128u >> 4) << 32;                    // stride byte offset: the next 8 pixels
    d |= (uint64_t)1u << 46;                             // descriptor version; layout type 0: no swizzle
    return d;
}

// One thread waits on a barrier that nothing arrives at, through the same
// bounded wait as the kernels' pipelines; when it gives up it latches
// ST_TIMEOUT, as a stalled pipeline would.
__global__ void wait_probe_kernel(uint32_t *status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    fence_barrier_init();
    if (!mbar_wait(&bar, 0, limit)) atomicOr(status, ST_TIMEOUT);
    mbar_arrive(&bar);   // complete the phase before the block exits
}

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                       // D: f32
           | (2u << 7) | (2u << 10)        // A, B: tf32
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// ------------------------------------------------------------------ kernel

//
// Fused GDN / IGDN (p.fuse_gdn): once the convolution sum y of the tile is
// complete, its channel norm  n_i = beta_i + sum_j gamma_ij y_j^2  is a second
// GEMM of y^2 (128 pixels x C) with gamma^T.  The epilogue warps write y^2,
// split into TF32 hi / lo, into the (now idle) stage buffers as the A
// operand, the producer loads gamma's hi / lo slices as B, and the MMA lane
// accumulates n (K = C, short enough for one TMEM accumulator) in HALF
// passes of two 32-channel chunks each.  The output is y * rsqrt(n) (GDN) or
// y * sqrt(n) (IGDN); y itself never reaches global memory.
// ATM (Cout = 128): the split A operand lives in TMEM instead of shared
// memory (tcgen05.mma with A from tensor memory).  A stage then holds only
// the float32 box and the weights (48 KB), so four stages fit and buffer
// more MMA work against the latency of TMA plus the split; TMEM holds two
// partial sums (2 x 128 columns) and a hi / lo A slot per stage (4 x 64).
// QM: quantisation fused into the plain (no GDN) epilogue -- 0 none, 1 symbols
// (q_sym, q_hat), 2 scale indices (q_idx) -- with the arithmetic of the
// separate kernels, so both decide every integer identically.
template <int STAGES, int HALF, int QM = 0>  // HALF: 32-column blocks per epilogue thread (Cout = 64 * HALF)
__global__ void __launch_bounds__(64 + EPI_THREADS, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                      const __grid_constant__ CUtensorMap tmBh,
                                                                      const __grid_constant__ CUtensorMap tmBl,
                                                                      const __grid_constant__ CUtensorMap tmGh,
                                                                      const __grid_constant__ CUtensorMap tmGl,
                                                                      const __grid_constant__ Params p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int COUT = 64 * HALF;
    constexpr int B_BYTES = COUT * KCH * 4;
    constexpr bool ATM = (HALF == 2);
    constexpr int A_STAGE_BYTES = ATM ? A_BYTES : 2 * A_BYTES;
    constexpr int STAGE_BYTES = A_STAGE_BYTES + 2 * B_BYTES;
    static_assert(!ATM || 2 * COUT + STAGES * 2 * KCH <= 512, "TMEM budget");
    // fused GDN: ATM runs the norm GEMM as one pass over all COUT/32 chunks
    // (one per stage and A slot); otherwise HALF passes of two chunks
    constexpr int GPASS = ATM ? 1 : HALF;
    constexpr int GCH = ATM ? COUT / KCH : 2;
    static_assert(!ATM || GCH <= STAGES, "one stage per norm chunk");
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *full = bars, *conv = bars + STAGES, *empty = bars + 2 * STAGES;
    uint64_t *pfull = bars + 3 * STAGES, *pempty = pfull + 2;
    uint64_t *gdn_full = pempty + 2, *gdn_ready = gdn_full + 1, *mma_done = gdn_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gdn_full + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int groups = (p.kchunks + FOLD - 1) / FOLD;
    __shared__ float s_qtab[QM == 2 ? 64 : 1];   // fused scale index: the 64 scales
    if (QM == 2 && threadIdx.x < 64) s_qtab[threadIdx.x] = p.q_tab[threadIdx.x];

    int b = 0, i0 = 0, j0 = 0;
    int64_t p0 = 0;
    if (p.mode == MODE_FLAT) {
        p0 = (int64_t)blockIdx.x * BLOCK_M;
    } else {   // S2, S1 and IM2COL tile the output grid the same way
        int t = blockIdx.x;
        const int tx = t % p.tiles_x;
        t /= p.tiles_x;
        const int ty = t % p.tiles_y;
        b = t / p.tiles_y;
        i0 = ty * p.R;
        j0 = tx * p.Wt;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], EPI_THREADS);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&pfull[q], 1);
            mbar_init(&pempty[q], EPI_THREADS);
        }
        mbar_init(gdn_full, 1);
        mbar_init(gdn_ready, EPI_THREADS);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, p.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto stage_a = [&](int s) { return smem + s * STAGE_BYTES; };
    auto stage_alo = [&](int s) { return smem + s * STAGE_BYTES + A_BYTES; };   // !ATM only
    auto stage_bh = [&](int s) { return smem + s * STAGE_BYTES + A_STAGE_BYTES; };
    auto stage_bl = [&](int s) { return smem + s * STAGE_BYTES + A_STAGE_BYTES + B_BYTES; };
    // ATM: TMEM columns of the hi / lo A slot of stage s
    auto slot_hi = [&](int s) { return tmem + (uint32_t)(2 * COUT + s * 2 * KCH); };
    auto slot_lo = [&](int s) { return tmem + (uint32_t)(2 * COUT + s * 2 * KCH + KCH); };
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(p.status, ST_TIMEOUT);
    };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint32_t tx_bytes = (p.mode == MODE_IM2COL ? 0 : A_BYTES) + 2 * B_BYTES;
            int issued = 0;
            for (int kc = 0; kc < p.kchunks && !*abort_flag; ++kc) {
                const int s = kc % STAGES;
                const uint32_t ph = (kc / STAGES) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1)) {
                    fail();
                    break;
                }
                const int t = kc / p.cpt;
                const int c0 = (kc % p.cpt) * KCH;
                mbar_expect_tx(&full[s], tx_bytes);
                if (p.mode == MODE_S2) {
                    const int du = p.du[t], dv = p.dv[t];
                    tma_load_5d(stage_a(s), &tmA, &full[s], (dv & 1) * p.Cin + c0, j0 + (dv >> 1), du & 1,
                                i0 + (du >> 1), b);
                } else if (p.mode == MODE_S1) {
                    tma_load_4d(stage_a(s), &tmA, &full[s], c0, j0 + p.dv[t], i0 + p.du[t], b);
                } else if (p.mode == MODE_FLAT) {
                    tma_load_2d(stage_a(s), &tmA, &full[s], c0, (int)p0);
                }
                tma_load_2d(stage_bh(s), &tmBh, &full[s], kc * KCH, 0);
                tma_load_2d(stage_bl(s), &tmBl, &full[s], kc * KCH, 0);
                issued = kc + 1;
            }
            // gamma slices for the fused norm: pass h uses stages 0 and 1 once
            // the MMAs that read them (main loop, then pass h-1) are done
            for (int h = 0; (p.fuse_gdn == 1 || p.fuse_gdn == 2) && h < GPASS && !*abort_flag; ++h) {
                if (!mbar_wait(mma_done, h & 1)) {
                    fail();
                    break;
                }
                mbar_expect_tx(gdn_full, 2 * GCH * B_BYTES);
                for (int c = 0; c < GCH; ++c) {
                    const int chunk = ATM ? c : (c == 0 ? h : HALF + h);
                    tma_load_2d(stage_bh(c), &tmGh, gdn_full, chunk * KCH, 0);
                    tma_load_2d(stage_bl(c), &tmGl, gdn_full, chunk * KCH, 0);
                }
            }
            if (*abort_flag) {  // wait (bounded) for loads still in flight
                for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; ++kc)
                    mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(BLOCK_M, COUT);
            for (int kc = 0; kc < p.kchunks; ++kc) {
                const int s = kc % STAGES;
                const int g = kc / FOLD, q = g & 1;
                const uint32_t dt = tmem + (uint32_t)(q * COUT);
                if (kc % FOLD == 0 && g >= 2) {  // partial buffer q must have been folded
                    if (*abort_flag || !mbar_wait(&pempty[q], ((g >> 1) - 1) & 1)) {
                        fail();
                        break;
                    }
                }
                if (*abort_flag || !mbar_wait(&conv[s], (kc / STAGES) & 1)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t bh = smem_u32(stage_bh(s)), bl = smem_u32(stage_bl(s));
                if constexpr (ATM) {
#pragma unroll
                    for (int kk = 0; kk < KCH / 8; ++kk) {
                        const uint32_t off = kk * 32;   // 8 tf32 along K: 32 bytes in smem, 8 columns in TMEM
                        const uint64_t dbh = sdesc(bh + off), dbl = sdesc(bl + off);
                        mma_tf32_ts(dt, slot_hi(s) + 8 * kk, dbh, idesc, (kc % FOLD != 0 || kk > 0) ? 1u : 0u);
                        mma_tf32_ts(dt, slot_hi(s) + 8 * kk, dbl, idesc, 1u);
                        mma_tf32_ts(dt, slot_lo(s) + 8 * kk, dbh, idesc, 1u);
                    }
                } else {
                    const uint32_t ah = smem_u32(stage_a(s)), al = smem_u32(stage_alo(s));
#pragma unroll
                    for (int kk = 0; kk < KCH / 8; ++kk) {
                        const uint32_t off = kk * 32;  // 8 tf32 = 32 bytes along K inside the swizzle row
                        const uint64_t dah = sdesc(ah + off), dal = sdesc(al + off);
                        const uint64_t dbh = sdesc(bh + off), dbl = sdesc(bl + off);
                        mma_tf32(dt, dah, dbh, idesc, (kc % FOLD != 0 || kk > 0) ? 1u : 0u);
                        mma_tf32(dt, dah, dbl, idesc, 1u);
                        mma_tf32(dt, dal, dbh, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
                if (kc % FOLD == FOLD - 1 || kc == p.kchunks - 1) mma_commit(&pfull[q]);
            }
            mma_commit(mma_done);   // phase 0: the main loop's MMAs are complete
            for (int h = 0; (p.fuse_gdn == 1 || p.fuse_gdn == 2) && h < GPASS; ++h) {
                if (*abort_flag || !mbar_wait(gdn_ready, h & 1) || !mbar_wait(gdn_full, h & 1)) {
                    fail();
                    break;
                }
                tc_fence_after();
                // All terms are positive and the accumulator truncates each addition by up to a
                // unit in its last place: a pass's small products (hi x lo, lo x hi, ~2^-11 of the
                // sum) go in before its large ones (hi x hi), while the accumulator is smaller
#pragma unroll
                for (int part = 0; part < 2; ++part) {
#pragma unroll
                    for (int c = 0; c < GCH; ++c) {
                        const uint32_t bh = smem_u32(stage_bh(c)), bl = smem_u32(stage_bl(c));
#pragma unroll
                        for (int kk = 0; kk < KCH / 8; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint64_t dbh = sdesc(bh + off), dbl = sdesc(bl + off);
                            const uint32_t acc = (h > 0 || part > 0 || c > 0 || kk > 0) ? 1u : 0u;
                            if constexpr (ATM) {
                                if (part == 0) {
                                    mma_tf32_ts(tmem, slot_hi(c) + 8 * kk, dbl, idesc, acc);
                                    mma_tf32_ts(tmem, slot_lo(c) + 8 * kk, dbh, idesc, 1u);
                                } else {
                                    mma_tf32_ts(tmem, slot_hi(c) + 8 * kk, dbh, idesc, 1u);
                                }
                            } else {
                                const uint64_t dah = sdesc(smem_u32(stage_a(c)) + off);
                                if (part == 0) {
                                    mma_tf32(tmem, dah, dbl, idesc, acc);
                                    mma_tf32(tmem, sdesc(smem_u32(stage_alo(c)) + off), dbh, idesc, 1u);
                                } else {
                                    mma_tf32(tmem, dah, dbh, idesc, 1u);
                                }
                            }
                        }
                    }
                }
                mma_commit(mma_done);   // phase h + 1
            }
        }
    } else {
        // ---------------- split, fold and epilogue (warps 2..9) ----------------
        const int et = threadIdx.x - 64;   // 0..255
        const int quarter = warp & 3;      // TMEM lanes 32*quarter ..
        const int half = (warp - 2) >> 2;  // column half
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * HALF * 32);
        float master[HALF * 32];
#pragma unroll
        for (int i = 0; i < HALF * 32; ++i) master[i] = 0.f;
        int folded = 0;
        bool ok = true;
        auto fold = [&](int g) {
            if (!ok) return;
            if (!mbar_wait(&pfull[g & 1], (g >> 1) & 1)) {
                fail();
                ok = false;
                return;
            }
            tc_fence_after();
            if constexpr (HALF == 2) {   // both 32-column slices in one TMEM round trip
                float v[32], w[32];
                tmem_ld32x2(lane_base + (uint32_t)((g & 1) * COUT), lane_base + (uint32_t)((g & 1) * COUT + 32), v, w);
#pragma unroll
                for (int i = 0; i < 32; ++i) master[i] += v[i];
#pragma unroll
                for (int i = 0; i < 32; ++i) master[32 + i] += w[i];
            } else {   // (three slices: one at a time, the registers are short)
#pragma unroll
                for (int h = 0; h < HALF; ++h) {
                    float v[32];
                    tmem_ld32(lane_base + (uint32_t)((g & 1) * COUT + h * 32), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) master[h * 32 + i] += v[i];
                }
            }
            tc_fence_before();
            mbar_arrive(&pempty[g & 1]);
        };
        for (int kc = 0; kc < p.kchunks && ok; ++kc) {
            const int s = kc % STAGES;
            // MODE_IM2COL (ATM): gather this chunk's A values from global memory
            // first, overlapping the weights' TMA; slot s is written only after
            // full[s] shows the stage (and so the slot) is free again
            float gv[16];
            if (ATM && p.mode == MODE_IM2COL) {
                const int m = quarter * 32 + lane;
                const int gi = i0 + m / p.Wt, gj = j0 + m % p.Wt;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int k = kc * KCH + 16 * half + e;
                    const int t = k / p.Cin, c = k - t * p.Cin;
                    float x = 0.f;
                    if (t < p.T) {
                        const int yi = p.s * gi + p.du[t], xi = p.s * gj + p.dv[t];
                        if (yi >= 0 && yi < p.Hi && xi >= 0 && xi < p.Wi)
                            x = __ldg(p.in + (((int64_t)b * p.Hi + yi) * p.Wi + xi) * p.Cin + c);
                    }
                    gv[e] = x;
                }
            }
            if (*abort_flag || !mbar_wait(&full[s], (kc / STAGES) & 1)) {
                fail();
                ok = false;
                break;
            }
            float4 *a = reinterpret_cast<float4 *>(stage_a(s));
            float4 *alo = reinterpret_cast<float4 *>(stage_alo(s));
            if constexpr (ATM) {
                // row m = this thread's TMEM lane, columns [16 * hc, 16 * hc + 16) of the chunk
                const int m = quarter * 32 + lane, hc = half;
                float v[16], hv[16], lv[16];
                if (p.mode == MODE_IM2COL) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = gv[e];
                } else {
                    const uint8_t *row = stage_a(s) + m * 128;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 f = *reinterpret_cast<const float4 *>(row + (((4 * hc + q) ^ (m & 7)) << 4));
                        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
                    }
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float x = v[e];
                    if (p.in_xform == IN_ABS) x = fabsf(x);
                    else if (p.in_xform == IN_SQUARE) x = x * x;
                    hv[e] = tf32_rna(x);
                    lv[e] = tf32_rna(x - hv[e]);
                }
                tmem_st16(slot_hi(s) + ((uint32_t)(quarter * 32) << 16) + 16 * hc, hv);
                tmem_st16(slot_lo(s) + ((uint32_t)(quarter * 32) << 16) + 16 * hc, lv);
                tmem_st_wait();
                tc_fence_before();
            } else if (p.mode == MODE_IM2COL) {
                // row m of the tile, 16 consecutive K entries [kc*32 + 16*kh, +16)
                const int m = et >> 1, kh = et & 1;
                const int gi = i0 + m / p.Wt, gj = j0 + m % p.Wt;
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int k = kc * KCH + 16 * kh + e;
                    const int t = k / p.Cin, c = k - t * p.Cin;
                    float x = 0.f;
                    if (t < p.T) {
                        const int yi = p.s * gi + p.du[t], xi = p.s * gj + p.dv[t];
                        if (yi >= 0 && yi < p.Hi && xi >= 0 && xi < p.Wi)
                            x = __ldg(p.in + (((int64_t)b * p.Hi + yi) * p.Wi + xi) * p.Cin + c);
                    }
                    v[e] = x;
                }
                uint8_t *ah = reinterpret_cast<uint8_t *>(a), *al = reinterpret_cast<uint8_t *>(alo);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 hv, lv;
                    hv.x = tf32_rna(v[4 * q + 0]); lv.x = tf32_rna(v[4 * q + 0] - hv.x);
                    hv.y = tf32_rna(v[4 * q + 1]); lv.y = tf32_rna(v[4 * q + 1] - hv.y);
                    hv.z = tf32_rna(v[4 * q + 2]); lv.z = tf32_rna(v[4 * q + 2] - hv.z);
                    hv.w = tf32_rna(v[4 * q + 3]); lv.w = tf32_rna(v[4 * q + 3] - hv.w);
                    const int off = m * 128 + (((4 * kh + q) ^ (m & 7)) << 4);
                    *reinterpret_cast<float4 *>(ah + off) = hv;
                    *reinterpret_cast<float4 *>(al + off) = lv;
                }
            } else
#pragma unroll
            for (int q = 0; q < A_BYTES / 16 / EPI_THREADS; ++q) {
                // the raw value serves as A_hi (the MMA takes it as trunc(x)); only
                // A_lo = x - trunc(x), exact, is written, and a transformed input back
                const int idx = et + q * EPI_THREADS;
                float4 v = a[idx];
                if (p.in_xform != IN_NONE) {
                    if (p.in_xform == IN_ABS) {
                        v.x = fabsf(v.x); v.y = fabsf(v.y); v.z = fabsf(v.z); v.w = fabsf(v.w);
                    } else {
                        v.x *= v.x; v.y *= v.y; v.z *= v.z; v.w *= v.w;
                    }
                    a[idx] = v;
                }
                alo[idx] = make_float4(v.x - tf32_trunc(v.x), v.y - tf32_trunc(v.y), v.z - tf32_trunc(v.z),
                                       v.w - tf32_trunc(v.w));
            }
            fence_proxy_async();
            mbar_arrive(&conv[s]);
            // mid-way through group g, the MMAs of group g-1 are done: fold it
            if (kc % FOLD == FOLD / 2 && kc / FOLD >= 1 && folded < kc / FOLD) fold(folded++);
        }
        while (ok && folded < groups) fold(folded++);
        const int cbase = half * HALF * 32;
        if (ok && p.fuse_gdn >= 3) {
            // 1DN / inverse 1DN: per-channel, y * rsqrt(beta + gamma y^2) or y * sqrt(.)
#pragma unroll
            for (int h = 0; h < HALF; ++h) {
                const int c = cbase + 32 * h;
                if (p.fuse_gdn == 3) norm_diag<32, false>(master + 32 * h, p.bias + c, p.gdn_gamma + c, p.gdn_beta + c);
                else norm_diag<32, true>(master + 32 * h, p.bias + c, p.gdn_gamma + c, p.gdn_beta + c);
            }
        }
        if (ok && (p.fuse_gdn == 1 || p.fuse_gdn == 2)) {
            // y = conv + bias, then the norm GEMM on y^2 (see above)
#pragma unroll
            for (int h = 0; h < HALF; ++h) add_bias<32>(master + 32 * h, p.bias + cbase + 32 * h);
            const int m = quarter * 32 + lane;
            if constexpr (ATM) {
                // this thread's chunks (HALF of them) -> TMEM A slots HALF*half + h, its lane
                const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
#pragma unroll
                for (int h = 0; h < HALF; ++h) {
                    float hv[32], lv[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float sq = master[h * 32 + i] * master[h * 32 + i];
                        hv[i] = tf32_rna(sq);
                        lv[i] = tf32_rna(sq - hv[i]);
                    }
                    const int slot = HALF * half + h;
                    tmem_st16(slot_hi(slot) + lane_off, hv);
                    tmem_st16(slot_hi(slot) + lane_off + 16, hv + 16);
                    tmem_st16(slot_lo(slot) + lane_off, lv);
                    tmem_st16(slot_lo(slot) + lane_off + 16, lv + 16);
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(gdn_ready);
            }
#pragma unroll
            for (int h = 0; h < (ATM ? 0 : HALF); ++h) {
                if (h > 0 && (*abort_flag || !mbar_wait(mma_done, h & 1))) {
                    fail();
                    ok = false;
                    break;
                }
                // chunk h of this half -> stage `half` (A: hi, Alo: lo), row m, 128-byte swizzle
                uint8_t *ahi = stage_a(half), *alo = stage_alo(half);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float4 v, hv, lv;
                    v.x = master[h * 32 + 4 * u + 0]; v.y = master[h * 32 + 4 * u + 1];
                    v.z = master[h * 32 + 4 * u + 2]; v.w = master[h * 32 + 4 * u + 3];
                    v.x *= v.x; v.y *= v.y; v.z *= v.z; v.w *= v.w;
                    // truncation split, as for the activations: y^2 itself is the hi operand
                    hv = v;
                    lv.x = v.x - tf32_trunc(v.x); lv.y = v.y - tf32_trunc(v.y);
                    lv.z = v.z - tf32_trunc(v.z); lv.w = v.w - tf32_trunc(v.w);
                    const int off = m * 128 + ((u ^ (m & 7)) << 4);
                    *reinterpret_cast<float4 *>(ahi + off) = hv;
                    *reinterpret_cast<float4 *>(alo + off) = lv;
                }
                fence_proxy_async();
                tc_fence_before();
                mbar_arrive(gdn_ready);
            }
            if (ok && (*abort_flag || !mbar_wait(mma_done, GPASS & 1))) {
                fail();
                ok = false;
            }
            if (ok) {
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < 2 * HALF; ++h) {   // 16 columns at a time
                    float v[16];
                    tmem_ld16(lane_base + (uint32_t)(h * 16), v);
                    if (p.fuse_gdn == 1) norm_n<16, false>(master + h * 16, v, p.gdn_beta + cbase + h * 16);
                    else norm_n<16, true>(master + h * 16, v, p.gdn_beta + cbase + h * 16);
                }
            }
        }
        if (ok && !*abort_flag) {
            const int m = quarter * 32 + lane;
            bool valid;
            int64_t opix;
            if (p.mode == MODE_FLAT) {
                valid = p0 + m < p.rows;
                opix = p0 + m;
            } else {
                const int r = m / p.Wt, w = m % p.Wt;
                const int gi = i0 + r, gj = j0 + w;
                valid = gi < p.Gh && gj < p.Gw;
                opix = ((int64_t)b * p.Ho + p.oym * gi + p.oyo) * p.Wo + p.oxm * gj + p.oxo;
            }
            if (valid && p.fuse_gdn) {
                store_row<HALF * 32>(master, p.out, opix * p.ostride + p.ocoff + cbase, p.out_dt, p.out_inv_scale);
            } else if (valid) {
                float *dst = p.out + opix * p.ostride + p.ocoff + cbase;
                const int64_t HW = (int64_t)p.Ho * p.Wo;
                const int fb = (int)(opix / HW);
                const int64_t hw = opix - (int64_t)fb * HW;
#pragma unroll
                for (int q = 0; q < HALF * 8; ++q) {
                    float4 o;
                    float *op = reinterpret_cast<float *>(&o);
                    float4 xg = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (p.epi == EPI_GDN || p.epi == EPI_IGDN)
                        xg = *reinterpret_cast<const float4 *>(p.gdn_x + opix * p.ostride + p.ocoff + cbase + 4 * q);
                    const float *xp = reinterpret_cast<const float *>(&xg);
                    const float4 b4 = ld_param4(p.bias + cbase + 4 * q);
                    const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float y = master[4 * q + e] + bb[e];
                        if (p.epi == EPI_RELU) y = fmaxf(y, 0.f);
                        else if (p.epi == EPI_GDN) y = norm_apply<false>(xp[e], y);
                        else if (p.epi == EPI_IGDN) y = norm_apply<true>(xp[e], y);
                        op[e] = y;
                    }
                    reinterpret_cast<float4 *>(dst)[q] = o;
                    if constexpr (QM == 1) {
                        fused_quant_m<1, 4>(p, op, fb, hw, HW, p.ocoff + cbase + 4 * q, opix, s_qtab);
                    } else if constexpr (QM == 2) {
                        fused_quant_m<2, 4>(p, op, fb, hw, HW, p.ocoff + cbase + 4 * q, opix, s_qtab);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
}



// ------------------------------------------------------------------ persistent FP32 kernel (Cout = 128)
//
// conv_tcx_kernel: the Cout = 128 FP32 convolutions (fused GDN / IGDN, 1DN,
// bias, ReLU) as a persistent, warp-specialised kernel: one CTA per SM over
// tiles blockIdx.x + k gridDim.x, the same arithmetic as conv_tc_kernel
// (3xTF32, FOLD-chunk partial sums folded into float32 registers), organised
// around four measurements on this part (timestamps and micro-benchmarks):
//   * a one-tile-per-CTA schedule paid ~2 us of start-up, ~1 us between CTAs
//     and ~2.4 us of output stores per 128-pixel tile, and its epilogue
//     (last fold, y^2, norm GEMM, normalisation, output: ~7.4 us) left the
//     tensor pipe idle;
//   * a TF32 MMA of 128 x 128 x 8 takes ~63 ns and one of 128 x 256 x 8 ~73
//     ns: the instruction, not the multiply-adds, sets the pace at N = 128;
//   * the MMA takes an FP32 operand as TF32 by clearing its low 13 mantissa
//     bits;
//   * with A split by eight epilogue warps between their other work, the
//     split paced the main loop.
// Hence:
//   * one 3-stage load ring runs across tiles; a stage holds A (raw, serving
//     as A_hi), A_lo, B_hi, B_lo (16 KB each, 128-byte swizzled);
//   * per 8-wide K step two MMAs: A_hi x [B_hi | B_lo] (N = 256: one
//     descriptor spans the adjacent B areas; the two halves of the partial
//     sum accumulate apart and the fold adds them) and A_lo x B_hi (N = 128,
//     into the second half, with the other small product: the accumulator
//     truncates each addition by up to a unit in its last place, so the half
//     that holds the large products drifts half as far when it takes one
//     addition per K step instead of two; the norm GEMM likewise); with
//     256-column partials the two ping-pong buffers fill TMEM, so A is read
//     from shared memory;
//   * the split only writes A_lo = x - trunc(x), exact in FP32 (the MMA's
//     own truncation of it costs at most 2^-20 of a product);
//   * the fused norm's gamma rides the ring as two entries of two
//     [gamma_hi | gamma_lo] chunks; y^2 goes into the columns of the tile's
//     last (already folded) partial, each thread writing exactly the columns
//     it read; the norm result is one more ping-pong group;
//   * six warps only split, eight epilogue warps fold each partial as it
//     completes and finish a tile while the next one streams through the
//     ring, so the tensor pipe waits only for a tile's last fold and y^2;
//     the output leaves through a 32 KB staging buffer as two TMA stores of
//     64 channels;
//   * registers move from the producer / MMA / split warpgroups (72 a
//     thread) to the epilogue warpgroups (184) with setmaxnreg; the shares
//     add up to the 64 K registers the block is launched with;
//   * the fold reads a partial's two halves with one TMEM round trip (the
//     tile's last fold is on the tensor pipe's critical path);
//   * split K (ksplit > 1, launches without a fused norm): the work units are
//     (tile, K slice) pairs; a slice stores its folded partial sums raw and
//     tcx_splitk_sum_kernel adds the slices, the bias and ReLU;
//   * resident weights (NB > 0: 1x1 GEMMs of at most four K chunks whose
//     stored columns lie below NB, i.e. the tap contributions of a transposed
//     conv to three channels): the first NB rows of B_hi and B_lo are loaded
//     once per CTA and stay in shared memory (96 KB at NB = 96), so the ring
//     carries A alone (32 KB a stage) instead of re-streaming 128 KB of
//     constants a tile; the
//     products go as three N = NB MMAs (hi x hi into the first half, hi x lo
//     and lo x hi into the second) so the partial sums keep their layout.
//   warp 0       TMA producer            warp 1      TMEM allocation, MMA issue
//   warps 2..7   split A                 warps 8..15 fold, bias / norm, output
//                                                    (TMEM lanes 32 (warp % 4) ..)
constexpr int TCX_THREADS = 512, TCX_SPLIT = 192, TCX_EPI = 256;

// TAPS: MODE_TAPS only (g_a conv0 over the padded 4-channel frame); NB > 0: weights resident (MODE_FLAT)
template <int STAGES, bool TAPS, int NB = 0>
__global__ void __launch_bounds__(TCX_THREADS, 1) conv_tcx_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                       const __grid_constant__ CUtensorMap tmBh,
                                                                       const __grid_constant__ CUtensorMap tmBl,
                                                                       const __grid_constant__ CUtensorMap tmGh,
                                                                       const __grid_constant__ CUtensorMap tmGl,
                                                                       const __grid_constant__ CUtensorMap tmO,
                                                                       const __grid_constant__ Params p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int COUT = 128, HALF = 2;
    constexpr int AREA = A_BYTES;                     // 128 rows x 128 bytes
    constexpr bool BRES = NB > 0;
    // a stage: A (split in place to hi), A lo, and unless the weights are resident B hi, B lo
    constexpr int STAGE_BYTES = (BRES ? 2 : 4) * AREA;
    constexpr int RES_AREA = NB * KCH * 4;            // one resident weight slice: NB rows x 128 bytes
    constexpr int RES_CH = 4;                         // K chunks the resident weights hold at most
    constexpr int GCH = COUT / KCH;                   // gamma chunks of the norm GEMM
    constexpr int NGE = GCH / 2;                      // gamma entries: two chunks ([hi | lo] each) per stage
    static_assert(NGE <= STAGES, "the gamma entries fit the ring at once");
    static_assert(COUT * KCH * 4 == AREA, "a weight slice fills one area");
    static_assert(NB % 16 == 0 && NB <= COUT, "N = NB is an MMA shape; its slices keep 1024-byte swizzle atoms");
    // [resident weights: RES_CH x (B hi, B lo)] [ring] [output staging]
    uint8_t *ring = smem + (BRES ? RES_CH * 2 * RES_AREA : 0);
    uint8_t *otile = ring + STAGES * STAGE_BYTES;     // two output boxes of 32 channels
    uint64_t *bars = reinterpret_cast<uint64_t *>(otile + 2 * AREA);
    uint64_t *full = bars, *conv = bars + STAGES, *empty = bars + 2 * STAGES;
    uint64_t *pfull = bars + 3 * STAGES, *pempty = pfull + 2, *ebar = pempty + 2, *ready = ebar + 1;
    uint64_t *done = ready + 1;   // the epilogue warps' last TMEM access is behind them
    // gamma entry ge's loads, one phase per tile: full[s] then counts stage s's K chunks alone,
    // every one of which the split warps wait for, so none of their waits runs ahead of a phase
    // (a gamma load on full[s], which only the MMA waits for, could let a split warp's parity wait
    // on that stage pass before it)
    uint64_t *gfull = done + 1;
    uint64_t *bfull = gfull + NGE;   // the resident weights have landed (NB > 0)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bfull + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const bool gdn = !BRES && (p.fuse_gdn == 1 || p.fuse_gdn == 2);   // (never with ksplit > 1)
    // work units u = tile * ksplit + slice; slice q covers K chunks [kbegin(q), kbegin(q + 1))
    const int nunits = p.ntiles * p.ksplit;
    auto kbegin = [&](int q) { return (int)((int64_t)q * p.kchunks / p.ksplit); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], TCX_SPLIT);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&pfull[q], 1);
            mbar_init(&pempty[q], TCX_EPI);
        }
        mbar_init(ebar, TCX_EPI);
        mbar_init(ready, TCX_EPI);
        mbar_init(done, TCX_EPI);
        for (int ge = 0; ge < NGE; ++ge) mbar_init(&gfull[ge], 1);
        mbar_init(bfull, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    __shared__ float s_qtab[64];   // fused scale index: the 64 scales
    if (p.q_mode == 2 && threadIdx.x < 64) s_qtab[threadIdx.x] = p.q_tab[threadIdx.x];
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto area = [&](int s, int a) { return ring + s * STAGE_BYTES + a * AREA; };
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(p.status, ST_TIMEOUT);
    };
    auto origin = [&](int tile, int &b, int &i0, int &j0, int64_t &p0) {
        b = i0 = j0 = 0;
        p0 = (int64_t)tile * BLOCK_M;
        if (p.mode != MODE_FLAT) {
            const int tx = tile % p.tiles_x, t = tile / p.tiles_x;
            i0 = (t % p.tiles_y) * p.R;
            j0 = tx * p.Wt;
            b = t / p.tiles_y;
        }
    };

    if (warp < 8) reg_release<72>();   // warpgroups 0, 1; the epilogue's take the rest
    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint32_t tx_bytes = BRES ? AREA : (p.mode == MODE_IM2COL ? 0 : AREA) + 2 * AREA;
            uint32_t v = 0;
            // bit s / ge: parity of the last phase issued on full[s] / gfull[ge]; whether one was
            uint32_t fph = 0, fis = 0, gph = 0, gis = 0;
            int tk = 0;
            bool ok = true, bis = false;   // bis: the resident weights' load was issued
            if (BRES && blockIdx.x < nunits) {
                // NB rows of every K chunk's B hi and B lo, once: one phase of bfull
                mbar_expect_tx(bfull, (uint32_t)(p.kchunks * 2 * RES_AREA));
                for (int kc = 0; kc < p.kchunks; ++kc) {
                    tma_load_2d(smem + kc * 2 * RES_AREA, &tmBh, bfull, kc * KCH, 0);
                    tma_load_2d(smem + kc * 2 * RES_AREA + RES_AREA, &tmBl, bfull, kc * KCH, 0);
                }
                bis = true;
            }
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++tk) {
                const int tile = u / p.ksplit, kc0 = kbegin(u % p.ksplit), nk = kbegin(u % p.ksplit + 1) - kc0;
                int b, i0, j0;
                int64_t p0;
                origin(tile, b, i0, j0, p0);
                for (int e = 0; e < nk + (gdn ? NGE : 0); ++e, ++v) {   // ring entries of the unit
                    const int s = v % STAGES;
                    if (*abort_flag || !mbar_wait(&empty[s], ((v / STAGES) & 1) ^ 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    if (e < nk) {
                        const int kc = kc0 + e;
                        const int t = kc / p.cpt;
                        const int c0 = (kc % p.cpt) * KCH;
                        mbar_expect_tx(&full[s], tx_bytes);
                        if (p.mode == MODE_S2) {
                            const int du = p.du[t], dv = p.dv[t];
                            tma_load_5d(area(s, 0), &tmA, &full[s], (dv & 1) * p.Cin + c0, j0 + (dv >> 1), du & 1,
                                        i0 + (du >> 1), b);
                        } else if (p.mode == MODE_S1) {
                            tma_load_4d(area(s, 0), &tmA, &full[s], c0, j0 + p.dv[t], i0 + p.du[t], b);
                        } else if (p.mode == MODE_FLAT) {
                            tma_load_2d(area(s, 0), &tmA, &full[s], c0, (int)p0);
                        } else if (TAPS) {
                            // taps 8 kc .. 8 kc + 7 (past tap 24 its box again: finite values
                            // against zero weights) at pixel (2i + u - 2, 2j + v - 2)
#pragma unroll 1
                            for (int j = 0; j < KCH / 4; ++j) {
                                const int tt = min(kc * (KCH / 4) + j, 24), du = tt / 5 - 2, dv = tt % 5 - 2;
                                tma_load_5d(area(s, 0) + j * TAP_BYTES, &tmA, &full[s], (dv & 1) * 4, j0 + (dv >> 1),
                                            du & 1, i0 + (du >> 1), b);
                            }
                        }
                        if constexpr (!BRES) {
                            tma_load_2d(area(s, 2), &tmBh, &full[s], kc * KCH, 0);
                            tma_load_2d(area(s, 3), &tmBl, &full[s], kc * KCH, 0);
                        }
                        if (fis >> s & 1) fph ^= 1u << s;
                        fis |= 1u << s;
                    } else {   // gamma entry ge: chunks 2 ge, 2 ge + 1 as [hi | lo] pairs
                        const int ge = e - nk;
                        mbar_expect_tx(&gfull[ge], 4 * AREA);
                        for (int j = 0; j < 2; ++j) {
                            tma_load_2d(area(s, 2 * j), &tmGh, &gfull[ge], (2 * ge + j) * KCH, 0);
                            tma_load_2d(area(s, 2 * j + 1), &tmGl, &gfull[ge], (2 * ge + j) * KCH, 0);
                        }
                        gph = (gph & ~(1u << ge)) | (uint32_t)(tk & 1) << ge;
                        gis |= 1u << ge;
                    }
                }
            }
            if (!ok) {   // wait (bounded) for the last phase issued on every load barrier
                for (int s = 0; s < STAGES; ++s)
                    if (fis >> s & 1) mbar_wait(&full[s], fph >> s & 1);
                for (int ge = 0; ge < NGE; ++ge)
                    if (gis >> ge & 1) mbar_wait(&gfull[ge], gph >> ge & 1);
                if (bis) mbar_wait(bfull, 0);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idw = idesc_tf32(BLOCK_M, 2 * COUT), idn = idesc_tf32(BLOCK_M, COUT);
            uint32_t v = 0, g = 0;   // ring entry, partial-buffer group
            bool ok = true;
            int tk = 0;
            if (BRES && blockIdx.x < nunits) {   // the resident weights, before the first MMA
                if (*abort_flag || !mbar_wait(bfull, 0)) {
                    fail();
                    ok = false;
                }
                tc_fence_after();
            }
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++tk) {
                const int kc0 = kbegin(u % p.ksplit), kc1 = kbegin(u % p.ksplit + 1);
                // the previous tile's norm GEMM read its y^2 from the buffer this tile's
                // first group writes: let it complete first
                if (gdn && tk > 0 && (*abort_flag || !mbar_wait(&pfull[(g - 1) & 1], ((g - 1) >> 1) & 1))) {
                    fail();
                    ok = false;
                    break;
                }
                for (int kc = kc0; kc < kc1; ++kc, ++v) {
                    const int s = v % STAGES;
                    const bool first = (kc - kc0) % FOLD == 0;
                    const bool last = (kc - kc0) % FOLD == FOLD - 1 || kc == kc1 - 1;
                    const uint32_t q = g & 1;
                    if (first && g >= 2 && (*abort_flag || !mbar_wait(&pempty[q], ((g >> 1) - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    if (*abort_flag || !mbar_wait(&conv[s], (v / STAGES) & 1)) {   // A split into hi / lo
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + q * 2 * COUT;
                    const uint32_t ah = smem_u32(area(s, 0)), al = smem_u32(area(s, 1));
                    if constexpr (BRES) {
                        // chunk kc's resident slices; the same products and order as the
                        // wide form, as N = NB MMAs into the two halves of the partial
                        const uint32_t wh = smem_u32(smem + kc * 2 * RES_AREA), wl = wh + RES_AREA;
                        const uint32_t idb = idesc_tf32(BLOCK_M, NB);
#pragma unroll
                        for (int kk = 0; kk < KCH / 8; ++kk) {
                            const uint64_t da = sdesc(ah + kk * 32), dh = sdesc(wh + kk * 32);
                            const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
                            mma_tf32(dt, da, dh, idb, acc);                             // A hi x B hi
                            mma_tf32(dt + COUT, da, sdesc(wl + kk * 32), idb, acc);     // A hi x B lo
                            mma_tf32(dt + COUT, sdesc(al + kk * 32), dh, idb, 1u);      // A lo x B hi
                        }
                    } else if constexpr (!TAPS) {
                        const uint32_t bh = smem_u32(area(s, 2));
#pragma unroll
                        for (int kk = 0; kk < KCH / 8; ++kk) {
                            const uint64_t db = sdesc(bh + kk * 32);
                            mma_tf32(dt, sdesc(ah + kk * 32), db, idw, (!first || kk > 0) ? 1u : 0u);   // [hi | lo]
                            mma_tf32(dt + COUT, sdesc(al + kk * 32), db, idn, 1u);   // A lo x B hi: small, second half
                        }
                    } else {
                        // the last chunk's data is its first K step (tap 24 and a zero one)
                        const uint32_t bh = smem_u32(area(s, 2));
                        const int ksteps = kc == kc1 - 1 ? 1 : KCH / 8;
                        for (int kk = 0; kk < ksteps; ++kk) {
                            const uint64_t db = sdesc(bh + kk * 32);
                            mma_tf32(dt, sdesc_taps(ah + kk * 2 * TAP_BYTES), db, idw, (!first || kk > 0) ? 1u : 0u);
                            mma_tf32(dt + COUT, sdesc_taps(al + kk * 2 * TAP_BYTES), db, idn, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                    if (last) {
                        mma_commit(&pfull[q]);
                        ++g;
                    }
                }
                if (!ok || !gdn) continue;
                // the norm GEMM into buffer g & 1; y^2 sits in the other (the tile's last group's)
                const uint32_t q = g & 1;
                if (*abort_flag || (g >= 2 && !mbar_wait(&pempty[q], ((g >> 1) - 1) & 1)) ||
                    !mbar_wait(ready, tk & 1)) {
                    fail();
                    ok = false;
                    continue;
                }
                const uint32_t dt = tmem + q * 2 * COUT, ysl = tmem + (q ^ 1) * 2 * COUT;
#pragma unroll
                for (int c = 0; c < GCH; ++c) {
                    const uint32_t ve = v + c / 2;
                    const int s = ve % STAGES;
                    if (c % 2 == 0) {
                        if (*abort_flag || !mbar_wait(&gfull[c / 2], tk & 1)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    const uint32_t bh = smem_u32(area(s, 2 * (c % 2)));
#pragma unroll
                    for (int kk = 0; kk < KCH / 8; ++kk) {
                        const uint64_t db = sdesc(bh + kk * 32);
                        mma_tf32_ts(dt, ysl + KCH * c + 8 * kk, db, idw, (c > 0 || kk > 0) ? 1u : 0u);
                        mma_tf32_ts(dt + COUT, ysl + COUT + KCH * c + 8 * kk, db, idn, 1u);   // small: second half
                    }
                    if (c % 2 == 1) {   // the entry's two chunks are issued: back to the producer
                        mbar_arrive_n(&conv[s], TCX_SPLIT);   // one conv phase per ring entry
                        mma_commit(&empty[s]);
                    }
                }
                if (!ok) continue;
                mma_commit(&pfull[q]);
                ++g;
                v += NGE;
            }
        }
    } else if (warp < 8) {
        // ---------------- split (warps 2..7) ----------------
        const int st = threadIdx.x - 64;   // 0 .. TCX_SPLIT - 1
        uint32_t v = 0, fph = 0;   // bit s: parity of stage s's next K-chunk phase on full[s]
        bool ok = true;
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const int nk = kbegin(u % p.ksplit + 1) - kbegin(u % p.ksplit);
            for (int kc = 0; kc < nk; ++kc, ++v) {
                const int s = v % STAGES;
                if (*abort_flag || !mbar_wait(&full[s], fph >> s & 1)) {
                    fail();
                    ok = false;
                    break;
                }
                fph ^= 1u << s;
                // The MMA reads an FP32 operand as TF32 by dropping its low 13 mantissa
                // bits (checked on this part), so the raw activation serves as A_hi and
                // only A_lo = x - trunc(x), exact in FP32, is written (elementwise, the
                // swizzled layout kept); a transformed input (|x|, x^2) is written back
                float4 *ah = reinterpret_cast<float4 *>(area(s, 0)), *al = reinterpret_cast<float4 *>(area(s, 1));
                for (int idx = st; idx < AREA / 16; idx += TCX_SPLIT) {
                    float4 f = ah[idx];
                    if (p.in_xform != IN_NONE) {
                        if (p.in_xform == IN_ABS) {
                            f.x = fabsf(f.x); f.y = fabsf(f.y); f.z = fabsf(f.z); f.w = fabsf(f.w);
                        } else {
                            f.x *= f.x; f.y *= f.y; f.z *= f.z; f.w *= f.w;
                        }
                        ah[idx] = f;
                    }
                    al[idx] = make_float4(f.x - tf32_trunc(f.x), f.y - tf32_trunc(f.y), f.z - tf32_trunc(f.z),
                                          f.w - tf32_trunc(f.w));
                }
                fence_proxy_async();
                mbar_arrive(&conv[s]);
            }
            if (gdn) v += NGE;
        }
    } else {
        // ---------------- fold, bias / norm, output (warps 8..15) ----------------
        reg_claim<184>();
        const int et = threadIdx.x - 256;
        const int quarter = warp & 3, half = (warp - 8) >> 2;
        const int m = quarter * 32 + lane;                 // this thread's TMEM lane / tile row
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int cbase = half * HALF * 32;                // this thread's output channels
        uint32_t g = 0, eph = 0;
        bool ok = true;
        float master[HALF * 32];
        auto esync = [&]() {
            if (!ok) return;
            mbar_arrive(ebar);
            if (!mbar_wait(ebar, eph & 1)) {
                fail();
                ok = false;
            }
            ++eph;
        };
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const int tile = u / p.ksplit, sl = u % p.ksplit;
            const int groups = (kbegin(sl + 1) - kbegin(sl) + FOLD - 1) / FOLD;
            int b, i0, j0;
            int64_t p0;
            origin(tile, b, i0, j0, p0);
#pragma unroll
            for (int i = 0; i < HALF * 32; ++i) master[i] = 0.f;
            // every partial sum of the unit into master, as its group completes
            for (int k = 0; k < groups && ok; ++k, ++g) {
                if (*abort_flag || !mbar_wait(&pfull[g & 1], (g >> 1) & 1)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + lane_off + (g & 1) * 2 * COUT + cbase;
#pragma unroll
                for (int h = 0; h < HALF; ++h) {   // both halves of the partial, one TMEM round trip
                    float x[32], xl[32];
                    tmem_ld32x2(base + 32 * h, base + COUT + 32 * h, x, xl);
#pragma unroll
                    for (int i = 0; i < 32; ++i) master[h * 32 + i] += x[i];
#pragma unroll
                    for (int i = 0; i < 32; ++i) master[h * 32 + i] += xl[i];
                }
                tc_fence_before();
                mbar_arrive(&pempty[g & 1]);
            }
            if (!ok) break;
#pragma unroll
            for (int h = 0; h < (p.ksplit > 1 ? 0 : HALF); ++h) {   // a K slice leaves bias and ReLU to the sum
                const int c = cbase + 32 * h;
                if (p.fuse_gdn == 3) norm_diag<32, false>(master + 32 * h, p.bias + c, p.gdn_gamma + c, p.gdn_beta + c);
                else if (p.fuse_gdn == 4) norm_diag<32, true>(master + 32 * h, p.bias + c, p.gdn_gamma + c, p.gdn_beta + c);
                else add_bias<32>(master + 32 * h, p.bias + c);
            }
            if (p.epi == EPI_RELU && p.ksplit == 1) {
#pragma unroll
                for (int i = 0; i < HALF * 32; ++i) master[i] = fmaxf(master[i], 0.f);
            }
            if (gdn) {
                // y^2 of this thread's chunks c = HALF half + h into the buffer of the
                // tile's last group (folded above; the MMA warp writes it again only
                // after the norm GEMM has completed): hi at column 32 c, lo at COUT + 32 c,
                // the columns this thread has read
                const uint32_t ysl = tmem + lane_off + ((g - 1) & 1) * 2 * COUT;
#pragma unroll
                for (int h = 0; h < HALF; ++h) {
                    const uint32_t slot = ysl + KCH * (HALF * half + h);
                    // hi is y^2 itself (the MMA takes it as trunc(y^2)), lo the exact rest
                    float hv[32], lv[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float sq = master[32 * h + i] * master[32 * h + i];
                        hv[i] = sq;
                        lv[i] = sq - tf32_trunc(sq);
                    }
                    tmem_st32(slot, hv);
                    tmem_st32(slot + COUT, lv);
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(ready);
                if (*abort_flag || !mbar_wait(&pfull[g & 1], (g >> 1) & 1)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + lane_off + (g & 1) * 2 * COUT + cbase;
#pragma unroll
                for (int h = 0; h < 2 * HALF; ++h) {
                    float n[16], nl[16];
                    tmem_ld16x2(base + 16 * h, base + COUT + 16 * h, n, nl);
#pragma unroll
                    for (int i = 0; i < 16; ++i) n[i] += nl[i];
                    if (p.fuse_gdn == 1) norm_n<16, false>(master + h * 16, n, p.gdn_beta + cbase + h * 16);
                    else norm_n<16, true>(master + h * 16, n, p.gdn_beta + cbase + h * 16);
                }
                tc_fence_before();
                mbar_arrive(&pempty[g & 1]);
                ++g;
            }
            if (BRES || p.out_dt == DT_F32) {   // (the resident-weights form is launched for float32 only)
                // the output in two halves of 64 channels (threads of half 0, then 1)
#pragma unroll
                for (int ph = 0; ph < 2; ++ph) {
                    if (et == 0) bulk_wait_read();   // the previous store has read the staging boxes
                    esync();
                    if (ok && half == ph) {
#pragma unroll
                        for (int h = 0; h < HALF; ++h) {
                            uint8_t *row = otile + h * AREA + m * 128;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                *reinterpret_cast<float4 *>(row + ((q ^ (m & 7)) << 4)) =
                                    make_float4(master[32 * h + 4 * q], master[32 * h + 4 * q + 1],
                                                master[32 * h + 4 * q + 2], master[32 * h + 4 * q + 3]);
                        }
                        fence_proxy_async();
                        if (p.q_mode && p.ksplit == 1) {
                            // quantisation fused: this thread's pixel, read back from the rows
                            // it has just staged (no registers held for it)
                            bool valid;
                            int64_t opix;
                            if (p.mode == MODE_FLAT) {
                                valid = p0 + m < p.rows;
                                opix = p0 + m;
                            } else {
                                const int gi = i0 + m / p.Wt, gj = j0 + m % p.Wt;
                                valid = gi < p.Gh && gj < p.Gw;
                                opix = ((int64_t)b * p.Ho + p.oym * gi + p.oyo) * p.Wo + p.oxm * gj + p.oxo;
                            }
                            if (valid) {
                                const int64_t HW = (int64_t)p.Ho * p.Wo;
                                const int fb = (int)(opix / HW);
#pragma unroll 1
                                for (int u = 0; u < HALF * 8; ++u) {
                                    const int h = u >> 3, q = u & 7;
                                    const float4 v4 = *reinterpret_cast<const float4 *>(otile + h * AREA + m * 128 +
                                                                                        ((q ^ (m & 7)) << 4));
                                    const float v[4] = {v4.x, v4.y, v4.z, v4.w};
                                    fused_quant<4>(p, v, fb, opix - (int64_t)fb * HW, HW, p.ocoff + cbase + 32 * h + 4 * q,
                                                   opix, s_qtab);
                                }
                            }
                        }
                    }
                    esync();
                    if (ok && et == 0 && !*abort_flag) {
                        for (int bx = 0; bx < HALF; ++bx) {
                            const int co = HALF * 32 * ph + 32 * bx;
                            if (p.ksplit > 1) {   // partial sums: rows (slice * ntiles + tile) * 128 ..
                                tma_store_2d(&tmO, otile + bx * AREA, co, (sl * p.ntiles + tile) * BLOCK_M);
                                continue;
                            }
                            if (p.mode == MODE_FLAT && co >= p.ostride - p.ocoff) continue;   // narrow output
                            if (p.mode == MODE_FLAT && p.out_stream)
                                tma_store_2d_hint(&tmO, otile + bx * AREA, co, (int)p0, policy_evict_first());
                            else if (p.mode == MODE_FLAT) tma_store_2d(&tmO, otile + bx * AREA, co, (int)p0);
                            else tma_store_5d(&tmO, otile + bx * AREA, p.oxo * p.ostride + co, j0, p.oyo, i0, b);
                        }
                        bulk_commit();
                    }
                }
            } else {
                // bf16: one 128-byte box row of 64 channels per half; e4m3: one box row
                // of all 128 channels (the halves write its two 64-byte parts)
                const bool e4 = p.out_dt == DT_E4M3;
                if (et == 0) bulk_wait_read();
                esync();
                if (ok) {
                    uint8_t *row = otile + (e4 ? 0 : half) * AREA + m * 128;
                    if (!e4) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            *reinterpret_cast<uint4 *>(row + ((q ^ (m & 7)) << 4)) = make_uint4(
                                pack_bf16_f(master[8 * q], master[8 * q + 1]),
                                pack_bf16_f(master[8 * q + 2], master[8 * q + 3]),
                                pack_bf16_f(master[8 * q + 4], master[8 * q + 5]),
                                pack_bf16_f(master[8 * q + 6], master[8 * q + 7]));
                    } else {
                        const float sc = p.out_inv_scale;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float *w = master + 16 * q;
                            *reinterpret_cast<uint4 *>(row + (((4 * half + q) ^ (m & 7)) << 4)) = make_uint4(
                                pack_e4m3x4(w[0] * sc, w[1] * sc, w[2] * sc, w[3] * sc),
                                pack_e4m3x4(w[4] * sc, w[5] * sc, w[6] * sc, w[7] * sc),
                                pack_e4m3x4(w[8] * sc, w[9] * sc, w[10] * sc, w[11] * sc),
                                pack_e4m3x4(w[12] * sc, w[13] * sc, w[14] * sc, w[15] * sc));
                        }
                    }
                    fence_proxy_async();
                }
                esync();
                if (ok && et == 0 && !*abort_flag) {
                    for (int bx = 0; bx < (e4 ? 1 : 2); ++bx) {
                        const int co = 64 * bx;
                        if (p.mode == MODE_FLAT) tma_store_2d(&tmO, otile + bx * AREA, co, (int)p0);
                        else tma_store_5d(&tmO, otile + bx * AREA, p.oxo * p.ostride + co, j0, p.oyo, i0, b);
                    }
                    bulk_commit();
                }
            }
        }
        if (et == 0) bulk_wait_all();
        tc_fence_before();
        mbar_arrive(done);
    }

    // TMEM is released once the epilogue warps are past their last access
    // (bounded: a stalled pipeline has latched its status already)
    if (warp == 1) {
        __syncwarp();
        mbar_wait(done, 0);
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------ BF16 kernel
//
// The BF16 precision form: activations between BF16 layers are bf16 NHWC in
// HBM, weights bf16, the MMA is kind::f16 (BF16 x BF16 -> FP32 in TMEM).  A
// K chunk is 64 channels (one 128-byte swizzle row), so TMA feeds the MMA
// directly and the eight epilogue warps only fold partial sums.  Anything
// that decides an integer or normalises stays FP32: the fused GDN / IGDN
// norm is the same 3xTF32 GEMM on the FP32 sum as in the FP32 kernel.

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                       // D: f32
           | (1u << 7) | (1u << 10)        // A, B: bf16
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// e4m3 x e4m3 -> f32 (kind::f8f6f4, formats 0 = E4M3)
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

constexpr int AB_BYTES = BLOCK_M * 128;   // one 128-byte row per pixel: 64 bf16 or 128 e4m3 channels
constexpr int KCB = 64;                   // bf16 per K chunk (weights built for the BF16 form)
constexpr int KC8 = 128;                  // e4m3 per K chunk

// EB: bytes per element (2: bf16, kind::f16; 1: e4m3, kind::f8f6f4).  A K
// chunk is one 128-byte row either way, fed by 4 MMAs of 32 bytes of K.
template <int STAGES, int HALF, int EB>
__global__ void __launch_bounds__(64 + EPI_THREADS, 1) conv_lp_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                        const __grid_constant__ CUtensorMap tmB,
                                                                        const __grid_constant__ CUtensorMap tmGh,
                                                                        const __grid_constant__ CUtensorMap tmGl,
                                                                        const __grid_constant__ Params p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int COUT = 64 * HALF;
    constexpr int KCE = 128 / EB;              // elements per K chunk
    constexpr int BB_BYTES = COUT * 128;
    constexpr int STAGE_BYTES = AB_BYTES + BB_BYTES;
    // Fused GDN / IGDN: the norm GEMM of y^2 (TF32 hi / lo, A from TMEM slots
    // after the two partial buffers) with gamma (hi / lo slices by TMA into the
    // idle stages).  Cout = 128: one pass over its 4 chunks (gamma hi in the A
    // area, lo in the B area of stages 0..3).  Cout = 192: three passes of two
    // chunks (two TMEM slot pairs after the 384 partial columns; gamma hi / lo
    // of chunk j in the B areas of stages 2j / 2j + 1).
    constexpr bool NORM = HALF >= 2;
    constexpr int GPASS = HALF == 3 ? 3 : 1;   // norm passes
    constexpr int GCP = HALF == 3 ? 2 : COUT / KCH;   // tf32 chunks per pass
    constexpr int GB = COUT * KCH * 4;         // bytes of one gamma chunk (hi or lo)
    static_assert(HALF != 2 || (GCP <= STAGES && GB <= AB_BYTES && GB <= BB_BYTES), "norm operands fit the stages");
    static_assert(HALF != 3 || (2 * GCP <= STAGES && GB <= BB_BYTES && 2 * COUT + GCP * 2 * KCH <= 512),
                  "norm operands fit the stages and TMEM");
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *full = bars, *empty = bars + STAGES;
    uint64_t *pfull = bars + 2 * STAGES, *pempty = pfull + 2;
    uint64_t *gdn_full = pempty + 2, *gdn_ready = gdn_full + 1, *mma_done = gdn_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gdn_full + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int groups = (p.kchunks + FOLD - 1) / FOLD;
    int b = 0, i0 = 0, j0 = 0;
    {
        int t = blockIdx.x;
        const int tx = t % p.tiles_x;
        t /= p.tiles_x;
        const int ty = t % p.tiles_y;
        b = t / p.tiles_y;
        i0 = ty * p.R;
        j0 = tx * p.Wt;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&pfull[q], 1);
            mbar_init(&pempty[q], EPI_THREADS);
        }
        mbar_init(gdn_full, 1);
        mbar_init(gdn_ready, EPI_THREADS);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, p.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto stage_a = [&](int s) { return smem + s * STAGE_BYTES; };
    auto stage_b = [&](int s) { return smem + s * STAGE_BYTES + AB_BYTES; };
    // norm A operand (y^2 hi / lo) in TMEM after the two partial buffers
    auto slot_hi = [&](int c) { return tmem + (uint32_t)(2 * COUT + c * 2 * KCH); };
    auto slot_lo = [&](int c) { return tmem + (uint32_t)(2 * COUT + c * 2 * KCH + KCH); };
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(p.status, ST_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kc = 0; kc < p.kchunks && !*abort_flag; ++kc) {
                const int s = kc % STAGES;
                if (!mbar_wait(&empty[s], ((kc / STAGES) & 1) ^ 1)) {
                    fail();
                    break;
                }
                const int t = kc / p.cpt;
                const int c0 = (kc % p.cpt) * KCE;
                mbar_expect_tx(&full[s], AB_BYTES + BB_BYTES);
                if (p.mode == MODE_S2) {
                    const int du = p.du[t], dv = p.dv[t];
                    tma_load_5d(stage_a(s), &tmA, &full[s], (dv & 1) * p.Cin + c0, j0 + (dv >> 1), du & 1,
                                i0 + (du >> 1), b);
                } else {
                    tma_load_4d(stage_a(s), &tmA, &full[s], c0, j0 + p.dv[t], i0 + p.du[t], b);
                }
                tma_load_2d(stage_b(s), &tmB, &full[s], kc * KCE, 0);
                issued = kc + 1;
            }
            for (int h = 0; NORM && (p.fuse_gdn == 1 || p.fuse_gdn == 2) && h < GPASS && !*abort_flag; ++h) {
                // pass h's gamma once the MMAs reading the stages (main loop, then pass h-1) are done
                if (!mbar_wait(mma_done, h & 1)) {
                    fail();
                    break;
                }
                mbar_expect_tx(gdn_full, 2 * GCP * GB);
                for (int c = 0; c < GCP; ++c) {
                    const int chunk = h * GCP + c;
                    uint8_t *dh = HALF == 3 ? stage_b(2 * c) : stage_a(c);
                    uint8_t *dl = HALF == 3 ? stage_b(2 * c + 1) : stage_b(c);
                    tma_load_2d(dh, &tmGh, gdn_full, chunk * KCH, 0);
                    tma_load_2d(dl, &tmGl, gdn_full, chunk * KCH, 0);
                }
            }
            if (*abort_flag) {
                for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; ++kc)
                    mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = EB == 2 ? idesc_bf16(BLOCK_M, COUT) : idesc_e4m3(BLOCK_M, COUT);
            for (int kc = 0; kc < p.kchunks; ++kc) {
                const int s = kc % STAGES;
                const int g = kc / FOLD, q = g & 1;
                const uint32_t dt = tmem + (uint32_t)(q * COUT);
                if (kc % FOLD == 0 && g >= 2) {
                    if (*abort_flag || !mbar_wait(&pempty[q], ((g >> 1) - 1) & 1)) {
                        fail();
                        break;
                    }
                }
                if (*abort_flag || !mbar_wait(&full[s], (kc / STAGES) & 1)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t a = smem_u32(stage_a(s)), bb = smem_u32(stage_b(s));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of K per MMA
                    if constexpr (EB == 2)
                        mma_bf16(dt, sdesc(a + kk * 32), sdesc(bb + kk * 32), idesc,
                                 (kc % FOLD != 0 || kk > 0) ? 1u : 0u);
                    else
                        mma_e4m3(dt, sdesc(a + kk * 32), sdesc(bb + kk * 32), idesc,
                                 (kc % FOLD != 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
                if (kc % FOLD == FOLD - 1 || kc == p.kchunks - 1) mma_commit(&pfull[q]);
            }
            mma_commit(mma_done);   // commit 0: the main loop
            for (int h = 0; NORM && (p.fuse_gdn == 1 || p.fuse_gdn == 2) && h < GPASS; ++h) {
                const uint32_t idt = idesc_tf32(BLOCK_M, COUT);
                if (*abort_flag || !mbar_wait(gdn_ready, h & 1) || !mbar_wait(gdn_full, h & 1)) {
                    fail();
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < GCP; ++c) {
                    const uint32_t gh = smem_u32(HALF == 3 ? stage_b(2 * c) : stage_a(c));
                    const uint32_t gl = smem_u32(HALF == 3 ? stage_b(2 * c + 1) : stage_b(c));
#pragma unroll
                    for (int kk = 0; kk < KCH / 8; ++kk) {
                        const uint64_t dgh = sdesc(gh + kk * 32), dgl = sdesc(gl + kk * 32);
                        mma_tf32_ts(tmem, slot_hi(c) + 8 * kk, dgh, idt, (h > 0 || c > 0 || kk > 0) ? 1u : 0u);
                        mma_tf32_ts(tmem, slot_hi(c) + 8 * kk, dgl, idt, 1u);
                        mma_tf32_ts(tmem, slot_lo(c) + 8 * kk, dgh, idt, 1u);
                    }
                }
                mma_commit(mma_done);   // commit h + 1: norm pass h
            }
        }
    } else {
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const uint32_t lane_base = tmem + lane_off + (uint32_t)(half * HALF * 32);
        const int cbase = half * HALF * 32;
        float master[HALF * 32];
#pragma unroll
        for (int i = 0; i < HALF * 32; ++i) master[i] = 0.f;
        bool ok = true;
        for (int g = 0; g < groups && ok; ++g) {
            if (*abort_flag || !mbar_wait(&pfull[g & 1], (g >> 1) & 1)) {
                fail();
                ok = false;
                break;
            }
            tc_fence_after();
            if constexpr (HALF == 2) {   // both 32-column slices in one TMEM round trip
                float v[32], w[32];
                tmem_ld32x2(lane_base + (uint32_t)((g & 1) * COUT), lane_base + (uint32_t)((g & 1) * COUT + 32), v, w);
#pragma unroll
                for (int i = 0; i < 32; ++i) master[i] += v[i];
#pragma unroll
                for (int i = 0; i < 32; ++i) master[32 + i] += w[i];
            } else {   // (three slices: one at a time, the registers are short)
#pragma unroll
                for (int h = 0; h < HALF; ++h) {
                    float v[32];
                    tmem_ld32(lane_base + (uint32_t)((g & 1) * COUT + h * 32), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) master[h * 32 + i] += v[i];
                }
            }
            tc_fence_before();
            mbar_arrive(&pempty[g & 1]);
        }
#pragma unroll
        for (int h = 0; h < HALF; ++h) {
            float *mh = master + 32 * h;
            if constexpr (EB == 1) {   // undo the e4m3 scales: x = stored * in_scale, w = stored * w_scale[o]
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 w = ld_param4(p.w_scale + cbase + 32 * h + 4 * q);
                    mh[4 * q] *= w.x * p.in_scale; mh[4 * q + 1] *= w.y * p.in_scale;
                    mh[4 * q + 2] *= w.z * p.in_scale; mh[4 * q + 3] *= w.w * p.in_scale;
                }
            }
            if (p.bias) add_bias<32>(mh, p.bias + cbase + 32 * h);
        }
        if (ok && p.fuse_gdn >= 3) {   // 1DN / inverse 1DN, per channel
#pragma unroll
            for (int h = 0; h < HALF; ++h) {
                const int c = cbase + 32 * h;
                if (p.fuse_gdn == 3) norm_diag<32, false>(master + 32 * h, nullptr, p.gdn_gamma + c, p.gdn_beta + c);
                else norm_diag<32, true>(master + 32 * h, nullptr, p.gdn_gamma + c, p.gdn_beta + c);
            }
        }
        if (ok && NORM && (p.fuse_gdn == 1 || p.fuse_gdn == 2)) {
            // pass g: this thread's chunks among [g GCP, (g+1) GCP) -> slots chunk - g GCP
#pragma unroll
            for (int g = 0; g < GPASS; ++g) {
                if (!ok) break;
                if (g > 0 && (*abort_flag || !mbar_wait(mma_done, g & 1))) {   // pass g-1 read the slots
                    fail();
                    ok = false;
                    break;
                }
#pragma unroll
                for (int h = 0; h < HALF; ++h) {
                    const int chunk = HALF * half + h;
                    if (chunk / GCP != g) continue;
                    const int slot = chunk - g * GCP;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {   // 16 columns at a time
                        float hv[16], lv[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float y = master[h * 32 + 16 * q + i];
                            const float sq = y * y;
                            hv[i] = tf32_rna(sq);
                            lv[i] = tf32_rna(sq - hv[i]);
                        }
                        tmem_st16(slot_hi(slot) + lane_off + 16 * q, hv);
                        tmem_st16(slot_lo(slot) + lane_off + 16 * q, lv);
                    }
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(gdn_ready);
            }
            if (!ok || *abort_flag || !mbar_wait(mma_done, GPASS & 1)) {
                fail();
                ok = false;
            } else {
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < 2 * HALF; ++h) {   // 16 columns at a time
                    float v[16];
                    tmem_ld16(lane_base + (uint32_t)(h * 16), v);
                    if (p.fuse_gdn == 1) norm_n<16, false>(master + h * 16, v, p.gdn_beta + cbase + h * 16);
                    else norm_n<16, true>(master + h * 16, v, p.gdn_beta + cbase + h * 16);
                }
            }
        }
        if (ok && !*abort_flag) {
            const int m = quarter * 32 + lane;
            const int r = m / p.Wt, w = m % p.Wt;
            const int gi = i0 + r, gj = j0 + w;
            if (gi < p.Gh && gj < p.Gw) {
                const int64_t opix = ((int64_t)b * p.Ho + p.oym * gi + p.oyo) * p.Wo + p.oxm * gj + p.oxo;
                if (p.epi == EPI_RELU) {
#pragma unroll
                    for (int i = 0; i < HALF * 32; ++i) master[i] = fmaxf(master[i], 0.f);
                } else if (p.epi == EPI_MASK) {
                    mask_row<HALF * 32>(master, p.gdn_x, opix * p.ostride + p.ocoff + cbase, p.out_dt);
                }
                store_row<HALF * 32>(master, p.out, opix * p.ostride + p.ocoff + cbase, p.out_dt, p.out_inv_scale);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
}

// ------------------------------------------------------------------ host

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

bool make_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
              const uint32_t *box, CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
              CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t gd[5], gs[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i > 0) gs[i - 1] = strides_bytes[i - 1];
    }
    CUresult r = fn(m, dt, rank, const_cast<void *>(base), gd, gs, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Round a float to TF32 (10 mantissa bits), nearest, ties away from zero.
uint32_t tf32_rna_host(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u & ~0x1fffu;  // inf / nan: truncate
    u += 0x1000u;                                                // half of the dropped 13 bits
    return u & ~0x1fffu;
}

// Cout = 128: A in TMEM, 4 stages of 48 KB; Cout = 192: A in shared memory,
// 2 stages of 80 KB.
int stages_for(int Cout) { return Cout == 128 ? 4 : 2; }

int smem_bytes(int stages, int Cout) {
    const int a = Cout == 128 ? A_BYTES : 2 * A_BYTES;
    return stages * (a + 2 * Cout * KCH * 4) + 256 + 1024;
}

template <int STAGES, int HALF, int QM = 0>
void launch_kernel(unsigned grid, int smem, cudaStream_t st, const CUtensorMap &a, const CUtensorMap &bh,
                   const CUtensorMap &bl, const CUtensorMap &gh, const CUtensorMap &gl, const Params &p) {
    if constexpr (HALF == 3 && QM == 0) {   // Cout = 192: Q(y) fused (tc_fuses_quant)
        if (p.q_mode == 1) return launch_kernel<STAGES, HALF, 1>(grid, smem, st, a, bh, bl, gh, gl, p);
    }
    cudaFuncSetAttribute(conv_tc_kernel<STAGES, HALF, QM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    conv_tc_kernel<STAGES, HALF, QM><<<grid, 64 + EPI_THREADS, smem, st>>>(a, bh, bl, gh, gl, p);
}


// Split-K sums of conv_tcx_kernel (ksplit > 1): slice q of tile t left its
// 128 x 128 partial sums at rows (q * ntiles + t) * 128 .. of part; one thread
// adds the slices of four channels of one tile row in slice order, then the
// bias and ReLU, and writes them where the fused store would have (FLAT rows,
// or pixel (i, j) of the tile's R x Wt block at output (i oym + oyo, j oxm + oxo)).
__global__ void __launch_bounds__(256) tcx_splitk_sum_kernel(const float4 *__restrict__ part, const Params p) {
    __shared__ float s_qtab[64];   // fused scale index: the 64 scales
    if (p.q_mode == 2 && threadIdx.x < 64) s_qtab[threadIdx.x] = p.q_tab[threadIdx.x];
    __syncthreads();
    const int64_t rows = (int64_t)p.ntiles * BLOCK_M;
    const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (idx >= rows * 32) return;
    const int c4 = (int)(idx % 32);
    const int64_t row = idx / 32;
    const int tile = (int)(row / BLOCK_M), m = (int)(row % BLOCK_M);
    int64_t o;
    int64_t opix;
    if (p.mode == MODE_FLAT) {
        if (row >= p.rows) return;
        opix = row;
    } else {
        const int tx = tile % p.tiles_x, t = tile / p.tiles_x;
        const int i = (t % p.tiles_y) * p.R + m / p.Wt, j = tx * p.Wt + m % p.Wt, b = t / p.tiles_y;
        if (i >= p.Gh || j >= p.Gw) return;
        opix = ((int64_t)b * p.Ho + (int64_t)i * p.oym + p.oyo) * p.Wo + (int64_t)j * p.oxm + p.oxo;
    }
    o = opix * p.ostride;
    float4 acc = part[idx];
    for (int q = 1; q < p.ksplit; ++q) {
        const float4 x = part[q * rows * 32 + idx];
        acc.x += x.x;
        acc.y += x.y;
        acc.z += x.z;
        acc.w += x.w;
    }
    const float4 bb = __ldg(reinterpret_cast<const float4 *>(p.bias) + c4);
    acc.x += bb.x;
    acc.y += bb.y;
    acc.z += bb.z;
    acc.w += bb.w;
    if (p.epi == EPI_RELU) {
        acc.x = fmaxf(acc.x, 0.f);
        acc.y = fmaxf(acc.y, 0.f);
        acc.z = fmaxf(acc.z, 0.f);
        acc.w = fmaxf(acc.w, 0.f);
    }
    *reinterpret_cast<float4 *>(p.out + o + p.ocoff + 4 * c4) = acc;
    if (p.q_mode) {
        const int64_t HW = (int64_t)p.Ho * p.Wo;
        const int fb = (int)(opix / HW);
        const float v[4] = {acc.x, acc.y, acc.z, acc.w};
        fused_quant<4>(p, v, fb, opix - (int64_t)fb * HW, HW, p.ocoff + 4 * c4, opix, s_qtab);
    }
}

// ------------------------------------------------------------------ persistent low-precision kernel (Cout = 128)
//
// conv_lpx_kernel: conv_lp_kernel's Cout = 128 arithmetic (bf16 or e4m3
// operands by TMA straight into the MMA, FOLD-chunk partial sums folded into
// float32 registers, the fused norm as a 3xTF32 GEMM on the FP32 sum) with
// conv_tcx_kernel's schedule: one CTA per SM over tiles blockIdx.x + k
// gridDim.x, one load ring across tiles (six 32 KB stages: A, B), gamma hi /
// lo of the norm's four 32-channel chunks as four more ring entries, y^2 in
// four TMEM slots of its own (so the next tile's first group never waits for
// the norm GEMM), the norm result as one more ping-pong group, and eight
// epilogue warps that finish a tile -- scales, bias or norm, output through a
// 32 KB staging buffer by TMA store -- while the next one streams through.
//   warp 0  TMA producer     warp 1  TMEM allocation, MMA issue
//   warps 2..9  fold, scales / bias / norm, output (TMEM lanes 32 (warp % 4) ..)
template <int STAGES, int EB>
__global__ void __launch_bounds__(64 + EPI_THREADS, 1) conv_lpx_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                       const __grid_constant__ CUtensorMap tmB,
                                                                       const __grid_constant__ CUtensorMap tmGh,
                                                                       const __grid_constant__ CUtensorMap tmGl,
                                                                       const __grid_constant__ CUtensorMap tmO,
                                                                       const __grid_constant__ Params p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int COUT = 128, HALF = 2;
    constexpr int AREA = AB_BYTES;                 // 128 rows x 128 bytes
    constexpr int STAGE_BYTES = 2 * AREA;          // A, B (or gamma hi, lo)
    constexpr int GCH = COUT / KCH;                // gamma chunks of the norm GEMM
    static_assert(COUT * 128 == AREA && COUT * KCH * 4 == AREA, "weight slices and gamma chunks fill an area");
    uint8_t *otile = smem + STAGES * STAGE_BYTES;  // two output boxes
    uint64_t *bars = reinterpret_cast<uint64_t *>(otile + 2 * AREA);
    uint64_t *full = bars, *empty = bars + STAGES;
    uint64_t *pfull = bars + 2 * STAGES, *pempty = pfull + 2, *ebar = pempty + 2, *ready = ebar + 1, *done = ready + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int groups = (p.kchunks + FOLD - 1) / FOLD;
    const bool gdn = p.fuse_gdn == 1 || p.fuse_gdn == 2;
    const int entries = p.kchunks + (gdn ? GCH : 0);
    constexpr int KCE = 128 / EB;                  // elements per K chunk

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&pfull[q], 1);
            mbar_init(&pempty[q], EPI_THREADS);
        }
        mbar_init(ebar, EPI_THREADS);
        mbar_init(ready, EPI_THREADS);
        mbar_init(done, EPI_THREADS);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto area = [&](int s, int a) { return smem + s * STAGE_BYTES + a * AREA; };
    // y^2 of norm chunk c (hi, lo) in TMEM after the two partial buffers
    auto slot_hi = [&](int c) { return tmem + (uint32_t)(2 * COUT + c * 2 * KCH); };
    auto slot_lo = [&](int c) { return tmem + (uint32_t)(2 * COUT + c * 2 * KCH + KCH); };
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(p.status, ST_TIMEOUT);
    };
    auto origin = [&](int tile, int &b, int &i0, int &j0) {
        const int tx = tile % p.tiles_x, t = tile / p.tiles_x;
        i0 = (t % p.tiles_y) * p.R;
        j0 = tx * p.Wt;
        b = t / p.tiles_y;
    };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t v = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < p.ntiles && ok; tile += gridDim.x) {
                int b, i0, j0;
                origin(tile, b, i0, j0);
                for (int kc = 0; kc < entries; ++kc, ++v) {
                    const int s = v % STAGES;
                    if (*abort_flag || !mbar_wait(&empty[s], ((v / STAGES) & 1) ^ 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], 2 * AREA);
                    if (kc < p.kchunks) {
                        const int t = kc / p.cpt;
                        const int c0 = (kc % p.cpt) * KCE;
                        if (p.mode == MODE_S2) {
                            const int du = p.du[t], dv = p.dv[t];
                            tma_load_5d(area(s, 0), &tmA, &full[s], (dv & 1) * p.Cin + c0, j0 + (dv >> 1), du & 1,
                                        i0 + (du >> 1), b);
                        } else {
                            tma_load_4d(area(s, 0), &tmA, &full[s], c0, j0 + p.dv[t], i0 + p.du[t], b);
                        }
                        tma_load_2d(area(s, 1), &tmB, &full[s], kc * KCE, 0);
                    } else {   // gamma chunk kc - kchunks: hi, lo
                        tma_load_2d(area(s, 0), &tmGh, &full[s], (kc - p.kchunks) * KCH, 0);
                        tma_load_2d(area(s, 1), &tmGl, &full[s], (kc - p.kchunks) * KCH, 0);
                    }
                }
            }
            if (!ok) {
                for (uint32_t u = v > STAGES ? v - STAGES : 0; u < v; ++u) mbar_wait(&full[u % STAGES], (u / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = EB == 2 ? idesc_bf16(BLOCK_M, COUT) : idesc_e4m3(BLOCK_M, COUT);
            const uint32_t idt = idesc_tf32(BLOCK_M, COUT);
            uint32_t v = 0, g = 0;
            bool ok = true;
            int tk = 0;
            for (int tile = blockIdx.x; tile < p.ntiles && ok; tile += gridDim.x, ++tk) {
                for (int kc = 0; kc < entries; ++kc, ++v) {
                    const int s = v % STAGES;
                    const bool norm = kc >= p.kchunks;
                    const bool first = norm ? kc == p.kchunks : kc % FOLD == 0;
                    const bool last = norm ? kc == entries - 1 : (kc % FOLD == FOLD - 1 || kc == p.kchunks - 1);
                    const uint32_t q = g & 1;
                    if (first && g >= 2 && (*abort_flag || !mbar_wait(&pempty[q], ((g >> 1) - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    if (first && norm && (*abort_flag || !mbar_wait(ready, tk & 1))) {   // y^2 written
                        fail();
                        ok = false;
                        break;
                    }
                    if (*abort_flag || !mbar_wait(&full[s], (v / STAGES) & 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + q * COUT;
                    const uint32_t a = smem_u32(area(s, 0)), bb = smem_u32(area(s, 1));
                    if (!norm) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of K per MMA
                            if constexpr (EB == 2)
                                mma_bf16(dt, sdesc(a + kk * 32), sdesc(bb + kk * 32), idesc, (!first || kk > 0) ? 1u : 0u);
                            else
                                mma_e4m3(dt, sdesc(a + kk * 32), sdesc(bb + kk * 32), idesc, (!first || kk > 0) ? 1u : 0u);
                        }
                    } else {
                        const int c = kc - p.kchunks;
#pragma unroll
                        for (int kk = 0; kk < KCH / 8; ++kk) {
                            const uint64_t dgh = sdesc(a + kk * 32), dgl = sdesc(bb + kk * 32);
                            mma_tf32_ts(dt, slot_hi(c) + 8 * kk, dgh, idt, (!first || kk > 0) ? 1u : 0u);
                            mma_tf32_ts(dt, slot_hi(c) + 8 * kk, dgl, idt, 1u);
                            mma_tf32_ts(dt, slot_lo(c) + 8 * kk, dgh, idt, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                    if (last) {
                        mma_commit(&pfull[q]);
                        ++g;
                    }
                }
            }
        }
    } else {
        // ---------------- fold, scales / bias / norm, output (warps 2..9) ----------------
        const int et = threadIdx.x - 64;
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int cbase = half * HALF * 32;
        uint32_t g = 0, eph = 0;
        bool ok = true;
        float master[HALF * 32];
        auto esync = [&]() {
            if (!ok) return;
            mbar_arrive(ebar);
            if (!mbar_wait(ebar, eph & 1)) {
                fail();
                ok = false;
            }
            ++eph;
        };
        int tk = 0;
        for (int tile = blockIdx.x; tile < p.ntiles && ok; tile += gridDim.x, ++tk) {
            int b, i0, j0;
            origin(tile, b, i0, j0);
#pragma unroll
            for (int i = 0; i < HALF * 32; ++i) master[i] = 0.f;
            for (int k = 0; k < groups && ok; ++k, ++g) {
                if (*abort_flag || !mbar_wait(&pfull[g & 1], (g >> 1) & 1)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + lane_off + (g & 1) * COUT + cbase;
                static_assert(HALF == 2, "one TMEM round trip per partial");
                {
                    float x[32], w[32];
                    tmem_ld32x2(base, base + 32, x, w);
#pragma unroll
                    for (int i = 0; i < 32; ++i) master[i] += x[i];
#pragma unroll
                    for (int i = 0; i < 32; ++i) master[32 + i] += w[i];
                }
                tc_fence_before();
                mbar_arrive(&pempty[g & 1]);
            }
            if (!ok) break;
#pragma unroll
            for (int h = 0; h < HALF; ++h) {
                float *mh = master + 32 * h;
                const int c = cbase + 32 * h;
                if constexpr (EB == 1) {   // undo the e4m3 scales: x = stored * in_scale, w = stored * w_scale[o]
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 w = ld_param4(p.w_scale + c + 4 * q);
                        mh[4 * q] *= w.x * p.in_scale; mh[4 * q + 1] *= w.y * p.in_scale;
                        mh[4 * q + 2] *= w.z * p.in_scale; mh[4 * q + 3] *= w.w * p.in_scale;
                    }
                }
                if (p.bias) add_bias<32>(mh, p.bias + c);
                if (p.fuse_gdn == 3) norm_diag<32, false>(mh, nullptr, p.gdn_gamma + c, p.gdn_beta + c);
                else if (p.fuse_gdn == 4) norm_diag<32, true>(mh, nullptr, p.gdn_gamma + c, p.gdn_beta + c);
            }
            if (p.epi == EPI_RELU) {
#pragma unroll
                for (int i = 0; i < HALF * 32; ++i) master[i] = fmaxf(master[i], 0.f);
            }
            if (gdn) {
                // y^2 of this thread's chunks c = HALF half + h into their slots (hi is y^2
                // itself, the MMA taking it as trunc(y^2); lo the exact rest)
#pragma unroll
                for (int h = 0; h < HALF; ++h) {
                    const int c = HALF * half + h;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        float hv[16], lv[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float sq = master[32 * h + 16 * q + i] * master[32 * h + 16 * q + i];
                            hv[i] = sq;
                            lv[i] = sq - tf32_trunc(sq);
                        }
                        tmem_st16(slot_hi(c) + lane_off + 16 * q, hv);
                        tmem_st16(slot_lo(c) + lane_off + 16 * q, lv);
                    }
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(ready);
                if (*abort_flag || !mbar_wait(&pfull[g & 1], (g >> 1) & 1)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + lane_off + (g & 1) * COUT + cbase;
#pragma unroll
                for (int h = 0; h < 2 * HALF; h += 2) {   // two 16-column slices per TMEM round trip
                    float n[16], n2[16];
                    tmem_ld16x2(base + 16 * h, base + 16 * (h + 1), n, n2);
                    if (p.fuse_gdn == 1) {
                        norm_n<16, false>(master + h * 16, n, p.gdn_beta + cbase + h * 16);
                        norm_n<16, false>(master + (h + 1) * 16, n2, p.gdn_beta + cbase + (h + 1) * 16);
                    } else {
                        norm_n<16, true>(master + h * 16, n, p.gdn_beta + cbase + h * 16);
                        norm_n<16, true>(master + (h + 1) * 16, n2, p.gdn_beta + cbase + (h + 1) * 16);
                    }
                }
                tc_fence_before();
                mbar_arrive(&pempty[g & 1]);
                ++g;
            }
            if (p.out_dt == DT_F32) {
                // two halves of 64 channels (threads of half 0, then 1)
#pragma unroll
                for (int ph = 0; ph < 2; ++ph) {
                    if (et == 0) bulk_wait_read();
                    esync();
                    if (ok && half == ph) {
#pragma unroll
                        for (int h = 0; h < HALF; ++h) {
                            uint8_t *row = otile + h * AREA + m * 128;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                *reinterpret_cast<float4 *>(row + ((q ^ (m & 7)) << 4)) =
                                    make_float4(master[32 * h + 4 * q], master[32 * h + 4 * q + 1],
                                                master[32 * h + 4 * q + 2], master[32 * h + 4 * q + 3]);
                        }
                        fence_proxy_async();
                    }
                    esync();
                    if (ok && et == 0 && !*abort_flag) {
                        for (int bx = 0; bx < HALF; ++bx)
                            tma_store_5d(&tmO, otile + bx * AREA, p.oxo * p.ostride + HALF * 32 * ph + 32 * bx, j0,
                                         p.oyo, i0, b);
                        bulk_commit();
                    }
                }
            } else {
                const bool e4 = p.out_dt == DT_E4M3;
                if (et == 0) bulk_wait_read();
                esync();
                if (ok) {
                    uint8_t *row = otile + (e4 ? 0 : half) * AREA + m * 128;
                    if (!e4) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            *reinterpret_cast<uint4 *>(row + ((q ^ (m & 7)) << 4)) = make_uint4(
                                pack_bf16_f(master[8 * q], master[8 * q + 1]),
                                pack_bf16_f(master[8 * q + 2], master[8 * q + 3]),
                                pack_bf16_f(master[8 * q + 4], master[8 * q + 5]),
                                pack_bf16_f(master[8 * q + 6], master[8 * q + 7]));
                    } else {
                        const float sc = p.out_inv_scale;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float *w = master + 16 * q;
                            *reinterpret_cast<uint4 *>(row + (((4 * half + q) ^ (m & 7)) << 4)) = make_uint4(
                                pack_e4m3x4(w[0] * sc, w[1] * sc, w[2] * sc, w[3] * sc),
                                pack_e4m3x4(w[4] * sc, w[5] * sc, w[6] * sc, w[7] * sc),
                                pack_e4m3x4(w[8] * sc, w[9] * sc, w[10] * sc, w[11] * sc),
                                pack_e4m3x4(w[12] * sc, w[13] * sc, w[14] * sc, w[15] * sc));
                        }
                    }
                    fence_proxy_async();
                }
                esync();
                if (ok && et == 0 && !*abort_flag) {
                    for (int bx = 0; bx < (e4 ? 1 : 2); ++bx)
                        tma_store_5d(&tmO, otile + bx * AREA, p.oxo * p.ostride + 64 * bx, j0, p.oyo, i0, b);
                    bulk_commit();
                }
            }
        }
        if (et == 0) bulk_wait_all();
        tc_fence_before();
        mbar_arrive(done);
    }

    if (warp == 1) {
        __syncwarp();
        mbar_wait(done, 0);
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

bool is_flat(const ConvDesc &d) {
    return d.T == 1 && d.du[0] == 0 && d.dv[0] == 0 && d.s == 1 && d.Gh == d.Hi && d.Gw == d.Wi && d.oym == 1 &&
           d.oxm == 1 && d.Ho == d.Hi && d.Wo == d.Wi;
}

int sm_count() {
    static int n = 0;
    if (n <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

// The output of a conv_tcx_kernel launch as a tensor map for its 32-channel
// boxes.  Grid modes: output pixel (b, oym * gi + oyo, oxm * gj + oxo),
// channel c, of a row stride of ostride elements from channel ocoff, viewed
// as (oxm * ostride - ocoff, Gw, oym, Gh, B) -- the x phase merged into the
// channel dimension -- so a tile is one box at (oxo * ostride + 32 k, j0, oyo,
// i0, b); boxes past Gw or Gh are clipped by the store.  MODE_FLAT: (ostride
// - ocoff, rows) at (32 k, p0).
bool make_out_map(CUtensorMap *m, const ConvDesc &d, const Params &p) {
    // a box row is 128 bytes: 32 floats, 64 bf16 or 128 e4m3 channels
    const uint64_t es = p.out_dt == DT_BF16 ? 2 : (p.out_dt == DT_E4M3 ? 1 : 4);
    const CUtensorMapDataType dt = p.out_dt == DT_BF16   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                   : p.out_dt == DT_E4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint32_t inner = (uint32_t)(128 / es);
    const uint64_t os = (uint64_t)p.ostride;
    void *base = reinterpret_cast<uint8_t *>(d.out) + (uint64_t)p.ocoff * es;
    if (p.mode == MODE_FLAT) {
        const uint64_t dims[2] = {os - p.ocoff, (uint64_t)p.rows};
        const uint64_t strides[1] = {os * es};
        const uint32_t box[2] = {inner, BLOCK_M};
        return make_map(m, base, 2, dims, strides, box, dt);
    }
    const uint64_t dims[5] = {(uint64_t)p.oxm * os - p.ocoff, (uint64_t)d.Gw, (uint64_t)p.oym, (uint64_t)d.Gh,
                              (uint64_t)d.B};
    const uint64_t strides[4] = {(uint64_t)p.oxm * os * es, (uint64_t)d.Wo * os * es, (uint64_t)p.oym * d.Wo * os * es,
                                 (uint64_t)d.Ho * d.Wo * os * es};
    const uint32_t box[5] = {inner, (uint32_t)p.Wt, 1, (uint32_t)p.R, 1};
    return make_map(m, base, 5, dims, strides, box, dt);
}

// Choose the R x Wt output block (R * Wt = 128) with the least padding.
void pick_tile(int Gh, int Gw, int *R, int *Wt) {
    double best = 1e30;
    for (int wt = 128; wt >= 4; wt /= 2) {
        const int r = BLOCK_M / wt;
        const double area = (double)((Gw + wt - 1) / wt * wt) * ((Gh + r - 1) / r * r);
        if (area < best - 1e-9) {
            best = area;
            *R = r;
            *Wt = wt;
        }
    }
}

}  // namespace

TcWeights::~TcWeights() {
    if (hi) cudaFree(hi);
    if (lo) cudaFree(lo);
    if (wb) cudaFree(wb);
    if (w8) cudaFree(w8);
    if (w8scale) cudaFree(w8scale);
    delete[] reinterpret_cast<CUtensorMap *>(maps);
    delete reinterpret_cast<CUtensorMap *>(bmap);
    delete reinterpret_cast<CUtensorMap *>(w8map);
}

namespace {
uint16_t bf16_rne_host(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// e4m3 copy of w / s[o], s[o] = max_k |w[o][k]| / 448 (per output channel),
// laid out [Cout][T][cin8] with each tap's channels zero-padded to a
// multiple of 128 (one K chunk): the kernel then reads whole chunks, and
// whatever the activation box holds past the real channels meets zeros.
void build_weights_e4m3(const float *w, int Cout, int T, int Cin, TcWeights *out) {
    if (Cin % 16 || (Cout != 128 && Cout != 192) || !encode_fn()) return;
    const int cin8 = (Cin + KC8 - 1) / KC8 * KC8;
    const int64_t K0 = (int64_t)T * Cin, K = (int64_t)T * cin8;
    std::vector<uint8_t> v((size_t)Cout * K, 0);
    std::vector<float> sc(Cout);
    for (int o = 0; o < Cout; ++o) {
        float mx = 0.f;
        for (int64_t k = 0; k < K0; ++k) mx = std::max(mx, std::fabs(w[o * K0 + k]));
        sc[o] = mx > 0.f ? mx / 448.f : 1.f;
        for (int t = 0; t < T; ++t)
            for (int c = 0; c < Cin; ++c)
                v[o * K + (int64_t)t * cin8 + c] =
                    (uint8_t)__nv_cvt_float_to_fp8(w[o * K0 + (int64_t)t * Cin + c] / sc[o], __NV_SATFINITE, __NV_E4M3);
    }
    out->cin8 = cin8;
    if (dev_malloc(&out->w8, v.size()) != cudaSuccess) return;
    if (dev_malloc((void **)&out->w8scale, Cout * sizeof(float)) != cudaSuccess) return;
    if (cudaMemcpy(out->w8, v.data(), v.size(), cudaMemcpyHostToDevice) != cudaSuccess) return;
    if (cudaMemcpy(out->w8scale, sc.data(), Cout * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return;
    CUtensorMap *m = new CUtensorMap;
    const uint64_t dims[2] = {(uint64_t)K, (uint64_t)Cout};
    const uint64_t strides[1] = {(uint64_t)K};
    const uint32_t box[2] = {KC8, (uint32_t)Cout};
    if (!make_map(m, out->w8, 2, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_UINT8)) {
        delete m;
        return;
    }
    out->w8map = m;
    out->f8valid = true;
}

void build_weights_bf16(const float *w, int Cout, int T, int Cin, TcWeights *out) {
    if (Cin % KCB || (Cout != 128 && Cout != 192) || !encode_fn()) return;
    const int64_t K = (int64_t)T * Cin;
    std::vector<uint16_t> v((size_t)Cout * K);
    for (size_t e = 0; e < v.size(); ++e) v[e] = bf16_rne_host(w[e]);
    if (dev_malloc(&out->wb, v.size() * 2) != cudaSuccess) return;
    if (cudaMemcpy(out->wb, v.data(), v.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return;
    CUtensorMap *m = new CUtensorMap;
    const uint64_t dims[2] = {(uint64_t)K, (uint64_t)Cout};
    const uint64_t strides[1] = {(uint64_t)K * 2};
    const uint32_t box[2] = {KCB, (uint32_t)Cout};
    if (!make_map(m, out->wb, 2, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16)) {
        delete m;
        return;
    }
    out->bmap = m;
    out->bvalid = true;
}
}  // namespace

void build_weights(const float *w, int Cout, int T, int Cin, TcWeights *out) {
    out->Cout = Cout;
    out->T = T;
    out->Cin = Cin;
    out->valid = false;
    build_weights_bf16(w, Cout, T, Cin, out);
    build_weights_e4m3(w, Cout, T, Cin, out);
    if ((Cout != 128 && Cout != 192) || stages_for(Cout) < 2) return;
    // Cin % 32 != 0: the im2col path, K = T * Cin zero-padded to a chunk multiple
    out->im2col = Cin % KCH != 0;
    if (out->im2col && (Cin > 4 || T * Cin > 8 * KCH)) return;
    if (!encode_fn()) return;
    const int64_t K0 = (int64_t)T * Cin;
    const int64_t K = (K0 + KCH - 1) / KCH * KCH;
    std::vector<uint32_t> hi((size_t)Cout * K, 0u), lo((size_t)Cout * K, 0u);
    for (int64_t o = 0; o < Cout; ++o)
        for (int64_t k = 0; k < K0; ++k) {
            const float x = w[o * K0 + k];
            const uint32_t h = tf32_rna_host(x);
            float hf;
            memcpy(&hf, &h, 4);
            hi[o * K + k] = h;
            lo[o * K + k] = tf32_rna_host(x - hf);
        }
    if (dev_malloc(&out->hi, hi.size() * 4) != cudaSuccess) return;
    if (dev_malloc(&out->lo, lo.size() * 4) != cudaSuccess) return;
    if (cudaMemcpy(out->hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return;
    if (cudaMemcpy(out->lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return;
    CUtensorMap *maps = new CUtensorMap[2];
    const uint64_t dims[2] = {(uint64_t)K, (uint64_t)Cout};
    const uint64_t strides[1] = {(uint64_t)K * 4};
    const uint32_t box[2] = {KCH, (uint32_t)Cout};
    if (!make_map(&maps[0], out->hi, 2, dims, strides, box) || !make_map(&maps[1], out->lo, 2, dims, strides, box)) {
        delete[] maps;
        return;
    }
    out->maps = maps;
    out->Kpad = (int)K;
    out->Npad = Cout;
    out->valid = true;
}

// The epilogues read per-channel parameters (bias, norm beta / gamma) four at a time.
bool params_aligned(const ConvDesc &d) {
    auto a16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    return a16(d.bias) && a16(d.gdn_beta) && a16(d.gdn_gamma);
}

int split_k(const ConvDesc &d, const TcWeights &w) {
    // Only the small grids of the hyper transforms profit: a tile walks its K
    // chunks one after another, so a layer of a few tiles a frame leaves most SMs
    // idle.  The slice count fills 148 SMs for a batch of 8 frames (fixed numbers,
    // not the device's: the arithmetic must not depend on where it runs), keeps
    // six or more K chunks a slice, and keeps the partial sums within the
    // scratch the caller gives a frame.
    if (!d.part || d.part_frame_floats <= 0 || !w.valid || w.im2col) return 1;
    if (d.Cout != 128 || d.fuse_gdn || d.in_dt != DT_F32 || d.out_dt != DT_F32) return 1;
    if (d.epi != EPI_NONE && d.epi != EPI_RELU) return 1;
    const int ostride = d.out_stride > 0 ? d.out_stride : d.Cout;
    if (ostride - d.out_coff < d.Cout || ostride % 4 || d.out_coff % 4) return 1;
    if (is_flat(d) || (d.s != 1 && d.s != 2)) return 1;
    int R, Wt;
    pick_tile(d.Gh, d.Gw, &R, &Wt);
    const int64_t tpf = (int64_t)((d.Gw + Wt - 1) / Wt) * ((d.Gh + R - 1) / R);
    const int nk = d.T * (d.Cin / KCH);
    int64_t q = 148 / (8 * tpf);
    q = std::min<int64_t>(q, nk / 6);
    q = std::min<int64_t>(q, 8);
    q = std::min<int64_t>(q, d.part_frame_floats / (tpf * BLOCK_M * 128));
    // partial-sum rows are 32-bit TMA coordinates (2^31 rows would be a terabyte of scratch)
    if (q > 1 && q * tpf * d.B * BLOCK_M >= ((int64_t)1 << 31)) return 1;
    return (int)std::max<int64_t>(q, 1);
}

bool can_run(const ConvDesc &d, const TcWeights &w) {
    if (!w.valid || d.Cin != w.Cin || d.T != w.T || d.Cout != w.Cout || !d.bias || !d.status) return false;
    if (!params_aligned(d)) return false;
    if ((reinterpret_cast<uintptr_t>(d.in) & 15) || (reinterpret_cast<uintptr_t>(d.out) & 15)) return false;
    if ((d.epi == EPI_GDN || d.epi == EPI_IGDN) && !d.gdn_x) return false;
    if (d.in_dt != DT_F32 || (d.out_dt != DT_F32 && !d.fuse_gdn)) return false;
    if (d.fuse_gdn >= 3 && (!d.gdn_beta || !d.gdn_gamma || d.epi != EPI_NONE)) return false;
    if (d.fuse_gdn == 1 || d.fuse_gdn == 2) {
        const TcWeights *g = static_cast<const TcWeights *>(d.gdn_w);
        if (!g || !g->valid || g->T != 1 || g->Cin != d.Cout || g->Cout != d.Cout || !d.gdn_beta) return false;
        if (d.epi != EPI_NONE) return false;
    }
    if (d.out_stride > 0 && d.out_stride - d.out_coff < d.Cout) {
        // a narrow output (the leading out_stride - out_coff channels of each row are
        // stored): the persistent kernel's clipped FLAT store only
        if (d.Cout != 128 || !is_flat(d) || w.im2col || d.fuse_gdn || d.out_dt != DT_F32) return false;
        if (d.epi != EPI_NONE && d.epi != EPI_RELU) return false;
        if (d.out_stride - d.out_coff <= 0 || (d.out_stride * 4) % 16 || (d.out_coff * 4) % 16) return false;
    }
    if (w.im2col) return d.epi != EPI_GDN && d.epi != EPI_IGDN && d.in_xform == IN_NONE && d.oym == 1 && d.oxm == 1;

    if (is_flat(d)) return true;
    if (d.s == 2) return (d.Hi % 2 == 0) && (d.Wi % 2 == 0) && d.oym == 1 && d.oxm == 1;
    return d.s == 1;
}

bool tc_fuses_quant(const ConvDesc &d) {
    // Cout = 192 runs one tile per CTA, an epilogue nothing overlaps: it takes
    // the symbols (about as fast as the separate kernel) but not the scale
    // index (its searches there cost more than the separate integer kernel)
    return d.q_mode != 0 && (d.Cout == 128 || (d.Cout == 192 && d.q_mode == 1)) &&
           (d.epi == EPI_NONE || d.epi == EPI_RELU) && d.fuse_gdn == 0 && d.out_dt == DT_F32;
}

bool launch(const ConvDesc &d, const TcWeights &w, cudaStream_t st) {
    Params p{};
    p.ksplit = 1;
    p.out = d.out;
    p.bias = d.bias;
    p.gdn_x = d.gdn_x;
    p.status = d.status;
    p.T = d.T;
    p.Cin = d.Cin;
    p.cpt = d.Cin / KCH;
    p.kchunks = d.T * p.cpt;
    p.in = d.in;
    p.Hi = d.Hi;
    p.Wi = d.Wi;
    p.s = d.s;
    p.Gh = d.Gh;
    p.Gw = d.Gw;
    p.B = d.B;
    p.Ho = d.Ho;
    p.Wo = d.Wo;
    p.Cout = d.Cout;
    p.oym = d.oym;
    p.oyo = d.oyo;
    p.oxm = d.oxm;
    p.oxo = d.oxo;
    p.epi = d.epi;
    p.in_xform = d.in_xform;
    p.fuse_gdn = d.fuse_gdn;
    p.gdn_beta = d.gdn_beta;
    p.gdn_gamma = d.gdn_gamma;
    p.out_dt = d.out_dt;
    p.ostride = d.out_stride > 0 ? d.out_stride : d.Cout;
    p.out_stream = d.out_stream;
    p.ocoff = d.out_coff;
    p.out_inv_scale = d.out_scale > 0.f ? 1.f / d.out_scale : 1.f;
    p.tmem_cols = 512;  // partial sums (+ A slots when Cout = 128)
    // fused quantisation: the persistent Cout = 128 kernel and its split-K sum,
    // and symbols in the one-tile-per-CTA Cout = 192 kernel (tc_fuses_quant)
    if (d.out_dt == DT_F32 && tc_fuses_quant(d)) {
        p.q_mode = d.q_mode;
        p.q_C = d.q_C;
        p.q_sym = d.q_sym;
        p.q_hat = d.q_hat;
        p.q_mu = d.q_mu;
        p.q_idx = d.q_idx;
        p.q_tab = d.q_tab;
    }
    for (int t = 0; t < d.T; ++t) {
        p.du[t] = d.du[t];
        p.dv[t] = d.dv[t];
    }
    CUtensorMap tmA;
    unsigned grid;
    const uint64_t C = (uint64_t)d.Cin;
    if (w.im2col) {
        p.mode = MODE_IM2COL;
        p.cpt = 1;
        p.kchunks = w.Kpad / KCH;
        pick_tile(d.Gh, d.Gw, &p.R, &p.Wt);
        p.tiles_x = (d.Gw + p.Wt - 1) / p.Wt;
        p.tiles_y = (d.Gh + p.R - 1) / p.R;
        grid = (unsigned)(p.tiles_x * p.tiles_y * d.B);
        tmA = reinterpret_cast<const CUtensorMap *>(w.maps)[0];   // unused in this mode
    } else if (d.frame) {
        // g_a conv0 over the padded 4-channel frame [B][2 Hi][2 Wi][4], viewed as pixel pairs
        // (8, Wp / 2, 2, Hp / 2, B); one tap's box: 4 channels of an R x Wt block
        if (d.Cout != 128 || d.Cin != FRAME_K || d.T != 1 || !is_flat(d) || (reinterpret_cast<uintptr_t>(d.frame) & 15))
            return false;
        p.mode = MODE_TAPS;
        pick_tile(d.Gh, d.Gw, &p.R, &p.Wt);
        p.tiles_x = (d.Gw + p.Wt - 1) / p.Wt;
        p.tiles_y = (d.Gh + p.R - 1) / p.R;
        grid = (unsigned)(p.tiles_x * p.tiles_y * d.B);
        const uint64_t Wp = 2ull * d.Wi, Hp = 2ull * d.Hi;
        const uint64_t dims[5] = {8, Wp / 2, 2, Hp / 2, (uint64_t)d.B};
        const uint64_t strides[4] = {32, Wp * 16, 2 * Wp * 16, Hp * Wp * 16};
        const uint32_t box[5] = {4, (uint32_t)p.Wt, 1, (uint32_t)p.R, 1};
        if (!make_map(&tmA, d.frame, 5, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE))
            return false;
    } else if (is_flat(d)) {
        p.mode = MODE_FLAT;
        p.rows = (int64_t)d.B * d.Hi * d.Wi;
        const uint64_t dims[2] = {C, (uint64_t)p.rows};
        const uint64_t strides[1] = {C * 4};
        const uint32_t box[2] = {KCH, BLOCK_M};
        if (!make_map(&tmA, d.in, 2, dims, strides, box)) return false;
        grid = (unsigned)((p.rows + BLOCK_M - 1) / BLOCK_M);
    } else {
        pick_tile(d.Gh, d.Gw, &p.R, &p.Wt);
        p.tiles_x = (d.Gw + p.Wt - 1) / p.Wt;
        p.tiles_y = (d.Gh + p.R - 1) / p.R;
        grid = (unsigned)(p.tiles_x * p.tiles_y * d.B);
        if (d.s == 2) {
            p.mode = MODE_S2;
            const uint64_t dims[5] = {2 * C, (uint64_t)d.Wi / 2, 2, (uint64_t)d.Hi / 2, (uint64_t)d.B};
            const uint64_t strides[4] = {2 * C * 4, (uint64_t)d.Wi * C * 4, 2ull * d.Wi * C * 4,
                                         (uint64_t)d.Hi * d.Wi * C * 4};
            const uint32_t box[5] = {KCH, (uint32_t)p.Wt, 1, (uint32_t)p.R, 1};
            if (!make_map(&tmA, d.in, 5, dims, strides, box)) return false;
        } else {
            p.mode = MODE_S1;
            const uint64_t dims[4] = {C, (uint64_t)d.Wi, (uint64_t)d.Hi, (uint64_t)d.B};
            const uint64_t strides[3] = {C * 4, (uint64_t)d.Wi * C * 4, (uint64_t)d.Hi * d.Wi * C * 4};
            const uint32_t box[4] = {KCH, (uint32_t)p.Wt, (uint32_t)p.R, 1};
            if (!make_map(&tmA, d.in, 4, dims, strides, box)) return false;
        }
    }
    if (grid == 0) return true;
    const CUtensorMap *maps = reinterpret_cast<const CUtensorMap *>(w.maps);
    // without fusion the gamma maps are unused: pass the weight maps
    const CUtensorMap *gmaps = (d.fuse_gdn == 1 || d.fuse_gdn == 2)
                                   ? reinterpret_cast<const CUtensorMap *>(static_cast<const TcWeights *>(d.gdn_w)->maps)
                                   : maps;
    CUtensorMap tmO;
    const int ks = split_k(d, w);
    bool omap;
    if (ks > 1) {
        // the slices' partial sums: [ks][grid * 128][128] floats at d.part
        const uint64_t dims[2] = {128, (uint64_t)ks * grid * BLOCK_M};
        const uint64_t strides[1] = {128 * 4};
        const uint32_t box[2] = {32, BLOCK_M};
        omap = make_map(&tmO, d.part, 2, dims, strides, box);
    } else {
        omap = make_out_map(&tmO, d, p);
    }
    if (d.Cout == 128 && (d.epi == EPI_NONE || d.epi == EPI_RELU) && p.mode != MODE_IM2COL && omap) {
        // persistent, one CTA per SM (conv_tcx_kernel)
        constexpr int STAGES = 3;
        p.ntiles = (int)grid;
        p.ksplit = ks;
        const unsigned pgrid = std::min<unsigned>(grid * ks, (unsigned)sm_count());
        // a 1x1 GEMM of at most four K chunks that stores at most 96 columns (the 84 tap
        // contribution columns of g_s's last transposed conv): its weights' first 96 rows
        // stay resident in shared memory and the ring carries A alone
        constexpr int NBR = 96;
        if (p.mode == MODE_FLAT && ks == 1 && d.fuse_gdn == 0 && p.q_mode == 0 && d.out_dt == DT_F32 &&
            p.kchunks >= 1 && p.kchunks * KCH == w.Kpad && p.kchunks <= 4 && w.Npad == 128 &&
            p.ostride - p.ocoff <= NBR) {
            CUtensorMap rbh, rbl;
            const uint64_t dims[2] = {(uint64_t)w.Kpad, (uint64_t)w.Npad};
            const uint64_t strides[1] = {(uint64_t)w.Kpad * 4};
            const uint32_t box[2] = {KCH, NBR};
            if (make_map(&rbh, w.hi, 2, dims, strides, box) && make_map(&rbl, w.lo, 2, dims, strides, box)) {
                const int smem_r = 4 * 2 * NBR * KCH * 4 + STAGES * 2 * A_BYTES + 2 * A_BYTES + 256 + 1024;
                cudaFuncSetAttribute(conv_tcx_kernel<STAGES, false, NBR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_r);
                conv_tcx_kernel<STAGES, false, NBR><<<pgrid, TCX_THREADS, smem_r, st>>>(tmA, rbh, rbl, rbh, rbl, tmO, p);
                return true;
            }
        }
        const int smem = STAGES * 4 * A_BYTES + 2 * A_BYTES + 256 + 1024;
        if (p.mode == MODE_TAPS) {
            cudaFuncSetAttribute(conv_tcx_kernel<STAGES, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            conv_tcx_kernel<STAGES, true>
                <<<pgrid, TCX_THREADS, smem, st>>>(tmA, maps[0], maps[1], gmaps[0], gmaps[1], tmO, p);
        } else {
            cudaFuncSetAttribute(conv_tcx_kernel<STAGES, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            conv_tcx_kernel<STAGES, false>
                <<<pgrid, TCX_THREADS, smem, st>>>(tmA, maps[0], maps[1], gmaps[0], gmaps[1], tmO, p);
        }
        if (ks > 1) {
            const int64_t n = (int64_t)grid * BLOCK_M * 32;
            tcx_splitk_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4 *>(d.part),
                                                                               p);
        }
        return true;
    }
    if (ks > 1) return false;   // not reached: split_k admits only launches of the persistent kernel
    if (p.mode == MODE_TAPS) return false;   // not reached: the caller builds this form for the persistent kernel
    if (p.ostride - p.ocoff < d.Cout) return false;   // a narrow output needs the clipped TMA store
    const int smem = smem_bytes(stages_for(d.Cout), d.Cout);
    if (d.Cout == 128)
        launch_kernel<4, 2>(grid, smem, st, tmA, maps[0], maps[1], gmaps[0], gmaps[1], p);
    else
        launch_kernel<2, 3>(grid, smem, st, tmA, maps[0], maps[1], gmaps[0], gmaps[1], p);
    return true;
}

namespace {
// launch shapes the low-precision kernel handles (weights aside)
bool lp_shape_ok(const ConvDesc &d) {
    const bool e4 = d.in_dt == DT_E4M3;
    if (d.in_dt != DT_BF16 && !e4) return false;
    if (d.Cout != 64 && d.Cout != 128 && d.Cout != 192) return false;
    if (d.Cout == 64 && e4) return false;
    if (!d.status || (reinterpret_cast<uintptr_t>(d.in) & 15) || (reinterpret_cast<uintptr_t>(d.out) & 15))
        return false;
    if (!params_aligned(d)) return false;
    if (d.epi != EPI_NONE && d.epi != EPI_RELU && d.epi != EPI_MASK) return false;
    if (d.epi == EPI_MASK && (!d.gdn_x || (reinterpret_cast<uintptr_t>(d.gdn_x) & 15) ||
                              (d.out_dt != DT_BF16 && d.out_dt != DT_F32)))
        return false;
    if (d.in_xform != IN_NONE) return false;
    if (d.Cin % (e4 ? 16 : KCB)) return false;   // e4m3: weights padded to whole chunks, see build_weights_e4m3
    if (d.fuse_gdn >= 3 && (!d.gdn_beta || !d.gdn_gamma)) return false;
    if (d.fuse_gdn == 1 || d.fuse_gdn == 2) {
        const TcWeights *g = static_cast<const TcWeights *>(d.gdn_w);
        if ((d.Cout != 128 && d.Cout != 192) || !g || !g->valid || g->T != 1 || g->Cin != d.Cout ||
            g->Cout != d.Cout || !d.gdn_beta)
            return false;
    }
    if (d.s == 2) return (d.Hi % 2 == 0) && (d.Wi % 2 == 0) && d.oym == 1 && d.oxm == 1;
    return d.s == 1;
}

template <int STAGES, int HALF, int EB>
void launch_lp_kernel(unsigned grid, cudaStream_t st, const CUtensorMap &a, const CUtensorMap &b,
                      const CUtensorMap &gh, const CUtensorMap &gl, const Params &p) {
    const int smem = STAGES * (AB_BYTES + 64 * HALF * 128) + 256 + 1024;
    cudaFuncSetAttribute(conv_lp_kernel<STAGES, HALF, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    conv_lp_kernel<STAGES, HALF, EB><<<grid, 64 + EPI_THREADS, smem, st>>>(a, b, gh, gl, p);
}
}  // namespace

bool can_run_lp(const ConvDesc &d, const TcWeights &w) {
    const bool e4 = d.in_dt == DT_E4M3;
    if (!lp_shape_ok(d) || (e4 ? !w.f8valid : !w.bvalid) || d.Cin != w.Cin || d.T != w.T || d.Cout != w.Cout)
        return false;
    return d.bias != nullptr;
}

bool can_run_lp_map(const ConvDesc &d) { return d.in_dt == DT_BF16 && lp_shape_ok(d); }

bool make_bf16_weight_map(TmaMap *m, const void *w, int Cout, int K) {
    if (!m || !w || K % KCB || (reinterpret_cast<uintptr_t>(w) & 15) || !encode_fn()) return false;
    if (Cout != 64 && Cout != 128 && Cout != 192) return false;
    const uint64_t dims[2] = {(uint64_t)K, (uint64_t)Cout};
    const uint64_t strides[1] = {(uint64_t)K * 2};
    const uint32_t box[2] = {KCB, (uint32_t)Cout};
    static_assert(sizeof(TmaMap) == sizeof(CUtensorMap), "TmaMap holds one CUtensorMap");
    return make_map(reinterpret_cast<CUtensorMap *>(m), w, 2, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
}

namespace {
// cpt: K chunks per tap (Cin / 64 for bf16; the padded e4m3 width / 128)
bool launch_lp_impl(const ConvDesc &d, const CUtensorMap &bm, const float *w_scale, int cpt, cudaStream_t st) {
    const bool e4 = d.in_dt == DT_E4M3;
    const int EBY = e4 ? 1 : 2;
    Params p{};
    p.ksplit = 1;
    p.out = d.out;
    p.bias = d.bias;
    p.gdn_x = d.gdn_x;
    p.status = d.status;
    p.T = d.T;
    p.Cin = d.Cin;
    p.cpt = cpt;
    p.kchunks = d.T * p.cpt;
    p.Gh = d.Gh;
    p.Gw = d.Gw;
    p.B = d.B;
    p.Ho = d.Ho;
    p.Wo = d.Wo;
    p.Cout = d.Cout;
    p.oym = d.oym;
    p.oyo = d.oyo;
    p.oxm = d.oxm;
    p.oxo = d.oxo;
    p.epi = d.epi;
    p.fuse_gdn = d.fuse_gdn;
    p.gdn_beta = d.gdn_beta;
    p.gdn_gamma = d.gdn_gamma;
    p.out_dt = d.out_dt;
    p.ostride = d.out_stride > 0 ? d.out_stride : d.Cout;
    p.ocoff = d.out_coff;
    p.out_inv_scale = d.out_scale > 0.f ? 1.f / d.out_scale : 1.f;
    p.in_scale = d.in_scale > 0.f ? d.in_scale : 1.f;
    p.w_scale = w_scale;
    p.tmem_cols = d.Cout == 64 ? 128 : 512;   // two partial buffers (+ norm operands when Cout = 128)
    for (int t = 0; t < d.T; ++t) {
        p.du[t] = d.du[t];
        p.dv[t] = d.dv[t];
    }
    pick_tile(d.Gh, d.Gw, &p.R, &p.Wt);
    p.tiles_x = (d.Gw + p.Wt - 1) / p.Wt;
    p.tiles_y = (d.Gh + p.R - 1) / p.R;
    const unsigned grid = (unsigned)(p.tiles_x * p.tiles_y * d.B);
    const uint64_t C = (uint64_t)d.Cin, E = (uint64_t)EBY;
    const CUtensorMapDataType dt = e4 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const uint32_t kce = 128 / EBY;
    CUtensorMap tmA;
    if (d.s == 2) {
        p.mode = MODE_S2;
        const uint64_t dims[5] = {2 * C, (uint64_t)d.Wi / 2, 2, (uint64_t)d.Hi / 2, (uint64_t)d.B};
        const uint64_t strides[4] = {2 * C * E, (uint64_t)d.Wi * C * E, 2ull * d.Wi * C * E,
                                     (uint64_t)d.Hi * d.Wi * C * E};
        const uint32_t box[5] = {kce, (uint32_t)p.Wt, 1, (uint32_t)p.R, 1};
        if (!make_map(&tmA, d.in, 5, dims, strides, box, dt)) return false;
    } else {
        p.mode = MODE_S1;
        const uint64_t dims[4] = {C, (uint64_t)d.Wi, (uint64_t)d.Hi, (uint64_t)d.B};
        const uint64_t strides[3] = {C * E, (uint64_t)d.Wi * C * E, (uint64_t)d.Hi * d.Wi * C * E};
        const uint32_t box[4] = {kce, (uint32_t)p.Wt, (uint32_t)p.R, 1};
        if (!make_map(&tmA, d.in, 4, dims, strides, box, dt)) return false;
    }
    if (grid == 0) return true;
    const bool gemm_norm = d.fuse_gdn == 1 || d.fuse_gdn == 2;
    const CUtensorMap *g = gemm_norm ? reinterpret_cast<const CUtensorMap *>(
                                            static_cast<const TcWeights *>(d.gdn_w)->maps)
                                      : &bm;
    const CUtensorMap &gh = g[0];
    const CUtensorMap &gl = gemm_norm ? g[1] : g[0];
    // a narrow output (the leading ostride - ocoff channels of each pixel stored) needs the
    // persistent kernel's clipped TMA stores
    const bool narrow = p.ostride - p.ocoff < d.Cout;
    if (narrow && (d.Cout != 128 || (d.epi != EPI_NONE && d.epi != EPI_RELU))) return false;
    if (d.Cout == 64) {
        // 4 stages (99.6 KB of shared memory, 128 TMEM columns): two CTAs share an SM, so one
        // CTA's epilogue overlaps the other's main loop on these short-K launches
        launch_lp_kernel<4, 1, 2>(grid, st, tmA, bm, gh, gl, p);
    } else if (d.Cout == 128) {
        CUtensorMap tmO;
        const bool omap = (d.epi == EPI_NONE || d.epi == EPI_RELU) && make_out_map(&tmO, d, p);
        if (narrow && !omap) return false;
        if (omap) {
            // persistent, one CTA per SM: six stages of 32 KB + half the output tile
            constexpr int ST = 6;
            const int smem = ST * 2 * AB_BYTES + 2 * AB_BYTES + 256 + 1024;
            p.ntiles = (int)grid;
            const unsigned pgrid = std::min<unsigned>(grid, (unsigned)sm_count());
            if (e4) {
                cudaFuncSetAttribute(conv_lpx_kernel<ST, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                conv_lpx_kernel<ST, 1><<<pgrid, 64 + EPI_THREADS, smem, st>>>(tmA, bm, gh, gl, tmO, p);
            } else {
                cudaFuncSetAttribute(conv_lpx_kernel<ST, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
                conv_lpx_kernel<ST, 2><<<pgrid, 64 + EPI_THREADS, smem, st>>>(tmA, bm, gh, gl, tmO, p);
            }
        } else if (e4) {
            launch_lp_kernel<6, 2, 1>(grid, st, tmA, bm, gh, gl, p);
        } else {
            launch_lp_kernel<6, 2, 2>(grid, st, tmA, bm, gh, gl, p);
        }
    } else {
        if (e4)
            launch_lp_kernel<5, 3, 1>(grid, st, tmA, bm, gh, gl, p);
        else
            launch_lp_kernel<5, 3, 2>(grid, st, tmA, bm, gh, gl, p);
    }
    return true;
}
}  // namespace

bool launch_lp(const ConvDesc &d, const TcWeights &w, cudaStream_t st) {
    const bool e4 = d.in_dt == DT_E4M3;
    return launch_lp_impl(d, *reinterpret_cast<const CUtensorMap *>(e4 ? w.w8map : w.bmap), w.w8scale,
                          e4 ? w.cin8 / KC8 : d.Cin / KCB, st);
}

bool launch_lp_map(const ConvDesc &d, const TmaMap &bmap, cudaStream_t st) {
    if (!can_run_lp_map(d)) return false;
    return launch_lp_impl(d, *reinterpret_cast<const CUtensorMap *>(&bmap), nullptr, d.Cin / KCB, st);
}

void launch_wait_probe(uint32_t *status, long long limit_cycles, cudaStream_t st) {
    wait_probe_kernel<<<1, 1, 0, st>>>(status, limit_cycles);
}

namespace {

// ------------------------------------------------------------------ weight gradient (bf16)
//
// wgrad_tc_kernel: the weight gradient of a transposed conv 5x5 / stride 2
// (pad 2) whose input x (NHWC [B][H][W][Cin], Cin = 64 CB) and output
// gradient dz (NHWC [B][2H][2W][64]) are stored in bf16,
//     dW[i][o][u][v] = sum_{b,a,c} x[b,a,c,i] dz[b, 2a+u-2, 2c+v-2, o],
// as GEMMs over K = the input pixels on tcgen05 (kind::f16, bf16 x bf16 ->
// float32 in TMEM).  The rows of an MMA are a pair of taps x the 64 output
// channels (tap 2j in TMEM lanes 0..63, tap 2j+1 in 64..127; the thirteenth
// pair loads tap 24 twice and drops its second half), the columns the Cin
// input channels.  Both operands are activation boxes as TMA lands them --
// one pixel per 128-byte swizzled row, channels contiguous -- read as
// MN-major matrices: a K step of 16 pixels is 2048 bytes, the 64-channel
// blocks (the two taps of A, the CB blocks of B) lie one box (8 KB) apart,
// 8-pixel groups 1024 bytes apart.  dz of tap (u, v) over a block of input
// pixels (a, c) is one box of the pixel-pair view (2*64, W, 2, H, B) of dz
// at ((v-2) & 1) * 64, c + ((v-2) >> 1), (u-2) & 1, a + ((u-2) >> 1), b):
// positions outside the output grid come back zero-filled and add nothing,
// as they add nothing to the sum; so do the zero-filled pixels past H or W.
// Work units (pair j, slice z of 64-pixel tiles) run over a persistent grid;
// unit (j, z) stores its sums at part[z][i][tap * 64 + o], and the caller adds
// the slices in slice order (fixed, so results do not depend on the launch).
//   warp 0      TMA producer (a stage = one tile: CB x-boxes + two dz boxes)
//   warp 1      TMEM allocation; one lane issues the MMAs
//   warps 2..5  epilogue (TMEM lanes 32 (warp % 4) ..): two accumulators
//               alternate, so a unit's store overlaps the next unit's MMAs
// Every wait is bounded; one that runs out latches ST_TIMEOUT and the CTA
// winds down after its copies and MMAs in flight have landed.
constexpr int WG_KP = 64;                  // input pixels per stage (one tile, R x Wt)
constexpr int WG_BOX = WG_KP * 128;        // bytes of one 64-channel box
constexpr int WG_PAIRS = 13;               // tap pairs (25 taps)
constexpr int WG_THREADS = 192;
constexpr int WG_UNITS_TARGET = 2 * 148;   // work units aimed at (a constant: the split never depends on the device)

struct WgParams {
    float *part;
    uint32_t *status;
    int R, Wt, tiles_x, tiles_y, ntiles, tps, units;
};

// kind::f16 with both operands MN-major (bits 15 and 16: A and B transposed)
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
    return idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// MN-major shared-memory descriptor, 128-byte swizzle: 64-element blocks
// along M / N `lbo` bytes apart, 8-row groups along K 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;  // leading byte offset: between 64-element MN blocks
    d |= (uint64_t)(1024u >> 4) << 32;            // stride byte offset: between 8-row K groups
    d |= (uint64_t)1u << 46;                      // descriptor version
    d |= (uint64_t)2u << 61;                      // SWIZZLE_128B
    return d;
}

template <int CB, int STAGES>
__global__ void __launch_bounds__(WG_THREADS, 1) wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                                 const __grid_constant__ CUtensorMap tmD,
                                                                 const __grid_constant__ WgParams p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int CIN = 64 * CB;
    constexpr int STAGE = (CB + 2) * WG_BOX;
    constexpr uint32_t ACC = CIN <= 64 ? 64 : 256;     // TMEM columns between the two accumulators
    constexpr uint32_t TCOLS = CIN <= 64 ? 128 : 512;
    constexpr int N = 25 * 64;                          // columns of a part row
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE);
    uint64_t *full = bars, *empty = bars + STAGES, *tfull = bars + 2 * STAGES, *tempty = tfull + 2;
    uint64_t *drained = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drained + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&tfull[q], 1);
            mbar_init(&tempty[q], 128);
        }
        mbar_init(drained, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(p.status, ST_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, issued = 0;   // stages filled by this CTA, across its units
            for (int u = blockIdx.x; u < p.units && !*abort_flag; u += gridDim.x) {
                const int j = u % WG_PAIRS, z = u / WG_PAIRS;
                const int taps[2] = {2 * j, min(2 * j + 1, 24)};
                const int k1 = min(p.ntiles, (z + 1) * p.tps);
                for (int k = z * p.tps; k < k1; ++k, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1)) {
                        fail();
                        break;
                    }
                    int t = k;
                    const int tx = t % p.tiles_x;
                    t /= p.tiles_x;
                    const int ty = t % p.tiles_y, b = t / p.tiles_y;
                    const int a0 = ty * p.R, c0 = tx * p.Wt;
                    uint8_t *st = smem + s * STAGE;
                    mbar_expect_tx(&full[s], STAGE);
#pragma unroll
                    for (int cb = 0; cb < CB; ++cb) tma_load_4d(st + cb * WG_BOX, &tmX, &full[s], 64 * cb, c0, a0, b);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int du = taps[h] / 5 - 2, dv = taps[h] % 5 - 2;
                        tma_load_5d(st + (CB + h) * WG_BOX, &tmD, &full[s], (dv & 1) * 64, c0 + (dv >> 1), du & 1,
                                    a0 + (du >> 1), b);
                    }
                    issued = it + 1;
                }
            }
            if (*abort_flag) {   // let the copies in flight land before the CTA exits
                for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; ++kc)
                    mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_mn(128, CIN);
            int it = 0, n = 0;   // stages consumed, units done
            for (int u = blockIdx.x; u < p.units; u += gridDim.x, ++n) {
                const int z = u / WG_PAIRS;
                const int k0 = z * p.tps, k1 = min(p.ntiles, k0 + p.tps);
                const int q = n & 1;
                if (n >= 2 && (*abort_flag || !mbar_wait(&tempty[q], ((n >> 1) - 1) & 1))) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + q * ACC;
                bool ok = true;
                for (int k = k0; k < k1; ++k, ++it) {
                    const int s = it % STAGES;
                    if (*abort_flag || !mbar_wait(&full[s], (it / STAGES) & 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xb = smem_u32(smem + s * STAGE), db = xb + CB * WG_BOX;
#pragma unroll
                    for (int kk = 0; kk < WG_KP / 16; ++kk)
                        mma_bf16(dt, sdesc_mn(db + kk * 2048, WG_BOX), sdesc_mn(xb + kk * 2048, WG_BOX), idesc,
                                 (k > k0 || kk > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[q]);
            }
            mma_commit(drained);   // arrives once every MMA issued above has completed
        }
    } else {
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;   // TMEM lane = GEMM row (tap half, output channel)
        const int h = m >> 6, o = m & 63;
        int n = 0;
        for (int u = blockIdx.x; u < p.units; u += gridDim.x, ++n) {
            const int j = u % WG_PAIRS, z = u / WG_PAIRS;
            const int q = n & 1;
            if (*abort_flag || !mbar_wait(&tfull[q], (n >> 1) & 1)) {
                fail();
                break;
            }
            tc_fence_after();
            const int tap = 2 * j + h;
            float *dst = p.part + (int64_t)z * CIN * N + tap * 64 + o;
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + q * ACC;
#pragma unroll 1
            for (int c = 0; c < CIN; c += 32) {
                float v[32];
                tmem_ld32(ta + c, v);
                if (tap < 25) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) dst[(int64_t)(c + i) * N] = v[i];   // a warp: 32 consecutive o
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[q]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        if (!mbar_wait(drained, 0)) {   // TMEM is released only after the MMAs are done
            atomicOr(p.status, ST_TIMEOUT);
            mbar_wait(drained, 0);
        }
        tmem_dealloc(tmem, TCOLS);
    }
}

// 64-pixel tiles R x Wt of an H x W grid, the fewest padded pixels (ties: wider)
void wgrad_tile(int H, int W, int *R, int *Wt) {
    double best = 1e30;
    for (int wt = 64; wt >= 8; wt /= 2) {
        const int r = WG_KP / wt;
        const double area = (double)((W + wt - 1) / wt * wt) * ((H + r - 1) / r * r);
        if (area < best - 1e-9) {
            best = area;
            *R = r;
            *Wt = wt;
        }
    }
}

void wgrad_plan(int B, int H, int W, WgParams *p) {
    wgrad_tile(H, W, &p->R, &p->Wt);
    p->tiles_x = (W + p->Wt - 1) / p->Wt;
    p->tiles_y = (H + p->R - 1) / p->R;
    p->ntiles = p->tiles_x * p->tiles_y * B;
    int ns = std::max(1, std::min(p->ntiles, (WG_UNITS_TARGET + WG_PAIRS - 1) / WG_PAIRS));
    p->tps = (p->ntiles + ns - 1) / ns;
    ns = (p->ntiles + p->tps - 1) / p->tps;
    p->units = ns * WG_PAIRS;
}

template <int CB, int STAGES>
bool launch_wgrad_cb(const CUtensorMap &tmX, const CUtensorMap &tmD, const WgParams &p, cudaStream_t st) {
    // stages, barriers, alignment, and 16 KB of slack past the last stage
    const int smem = STAGES * (CB + 2) * WG_BOX + 256 + 1024 + 16384;
    if (cudaFuncSetAttribute(wgrad_tc_kernel<CB, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return false;
    const unsigned grid = (unsigned)std::min(p.units, sm_count());
    wgrad_tc_kernel<CB, STAGES><<<grid, WG_THREADS, smem, st>>>(tmX, tmD, p);
    return true;
}

}  // namespace

int wgrad_bf16_slices(int B, int H, int W) {
    WgParams p{};
    wgrad_plan(B, H, W, &p);
    return p.units / WG_PAIRS;
}

bool launch_wgrad_bf16(const void *x, const void *dz, int B, int H, int W, int Cin, float *part, uint32_t *status,
                       cudaStream_t st) {
    if ((Cin != 64 && Cin != 128 && Cin != 192) || B < 1 || H < 1 || W < 1 || !x || !dz || !part ||
        (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(dz) & 15))
        return false;
    WgParams p{};
    wgrad_plan(B, H, W, &p);
    p.part = part;
    p.status = status;
    const uint64_t C = (uint64_t)Cin, E = 2;
    CUtensorMap tmX, tmD;
    {
        const uint64_t dims[4] = {C, (uint64_t)W, (uint64_t)H, (uint64_t)B};
        const uint64_t strides[3] = {C * E, (uint64_t)W * C * E, (uint64_t)H * W * C * E};
        const uint32_t box[4] = {64, (uint32_t)p.Wt, (uint32_t)p.R, 1};
        if (!make_map(&tmX, x, 4, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16)) return false;
    }
    {
        // dz [B][2H][2W][64] as (2 * 64, W, 2, H, B): a pixel pair per row of 128 values, rows of one parity
        const uint64_t row = 2ull * W * 64 * E;
        const uint64_t dims[5] = {128, (uint64_t)W, 2, (uint64_t)H, (uint64_t)B};
        const uint64_t strides[4] = {128 * E, row, 2 * row, 2ull * H * row};
        const uint32_t box[5] = {64, (uint32_t)p.Wt, 1, (uint32_t)p.R, 1};
        if (!make_map(&tmD, dz, 5, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16)) return false;
    }
    if (Cin == 64) return launch_wgrad_cb<1, 8>(tmX, tmD, p, st);
    if (Cin == 128) return launch_wgrad_cb<2, 6>(tmX, tmD, p, st);
    return launch_wgrad_cb<3, 5>(tmX, tmD, p, st);
}

// ------------------------------------------------------------------ MMA rate probe
//
// The dense rate of the tensor pipe, measured: every CTA (one per SM) issues
// `iters` tcgen05 MMAs of M = 128, N = 256 back to back into one TMEM
// accumulator, A (128 x 128 B) and B (256 x 128 B) resident in shared memory,
// the K step cycling over the four 32-byte quarters of the swizzled row.
// KIND 0: kind::tf32 (K = 8 per MMA), 1: kind::f16 with bf16 (K = 16),
// 2: kind::f8f6f4 with e4m3 (K = 32).  The operands hold 1.0 in their format.
template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_rate_kernel(int iters, uint32_t *status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bar;
    const uint32_t one = KIND == 0 ? 0x3f800000u : (KIND == 1 ? 0x3f803f80u : 0x38383838u);
    uint32_t *w = reinterpret_cast<uint32_t *>(smem);
    for (int i = threadIdx.x; i < (128 + 256) * 128 / 4; i += blockDim.x) w[i] = one;
    fence_proxy_async();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    if (threadIdx.x < 32) tmem_alloc(&tslot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t dt = tslot;
    if (threadIdx.x == 0) {
        const uint32_t a = smem_u32(smem), b = a + 128 * 128;
        const uint32_t idesc = KIND == 0 ? idesc_tf32(128, 256) : (KIND == 1 ? idesc_bf16(128, 256) : idesc_e4m3(128, 256));
        for (int i = 0; i < iters; ++i) {
            const uint32_t kk = (uint32_t)(i & 3) * 32;
            if (KIND == 0) mma_tf32(dt, sdesc(a + kk), sdesc(b + kk), idesc, i > 0 ? 1u : 0u);
            else if (KIND == 1) mma_bf16(dt, sdesc(a + kk), sdesc(b + kk), idesc, i > 0 ? 1u : 0u);
            else mma_e4m3(dt, sdesc(a + kk), sdesc(b + kk), idesc, i > 0 ? 1u : 0u);
        }
        mma_commit(&bar);
        // the MMAs must have finished before TMEM is released: one more bounded
        // wait after a first one that ran out
        if (!mbar_wait(&bar, 0)) {
            atomicOr(status, ST_TIMEOUT);
            mbar_wait(&bar, 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(dt, 256);
}

int mma_rate(int kind, int iters, double *tflops) {
    if (kind < 0 || kind > 2 || iters < 1 || iters > 1000000 || !tflops) return LIC_E_INVALID_ARG;
    int dev = 0, sms = 0;
    LIC_CUDA_TRY(cudaGetDevice(&dev));
    LIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // more shared memory than two CTAs could share: one CTA per SM
    const int smem = 160 * 1024;
    auto kern = kind == 0 ? mma_rate_kernel<0> : (kind == 1 ? mma_rate_kernel<1> : mma_rate_kernel<2>);
    LIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    uint32_t *status = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LIC_OK;
    float ms = 0.f;
    uint32_t hs = 0;
    if (cudaMalloc(&status, 4) != cudaSuccess || cudaMemset(status, 0, 4) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = LIC_E_CUDA;
    } else {
        kern<<<sms, 128, smem, st>>>(iters / 10 + 1, status);   // warm-up
        cudaEventRecord(e0, st);
        kern<<<sms, 128, smem, st>>>(iters, status);
        cudaEventRecord(e1, st);
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = LIC_E_CUDA;
        else if (hs)
            rc = LIC_E_TIMEOUT;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (status) cudaFree(status);
    if (rc) return rc;
    const double k = kind == 0 ? 8.0 : (kind == 1 ? 16.0 : 32.0);
    *tflops = 2.0 * 128.0 * 256.0 * k * (double)iters * sms / (ms * 1e-3) / 1e12;
    return LIC_OK;
}

}  // namespace tc
}  // namespace lic
