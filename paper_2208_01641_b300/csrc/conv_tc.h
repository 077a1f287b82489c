// Tensor-core (tcgen05) implicit-GEMM convolution: interface used by the
// layer runner.  The kernels live in conv_tc.cu.
#pragma once

#include "lic_internal.h"

namespace lic {
namespace tc {

// Weights of one GEMM launch, split for 3xTF32 (w = hi + lo, both exactly
// representable in TF32) and laid out as the B operand of the kernel.
struct TcWeights {
    void *hi = nullptr, *lo = nullptr;
    void *maps = nullptr;   // two CUtensorMap (hi, lo), host copies passed as kernel parameters
    void *wb = nullptr;     // bf16 copy [Cout][K] for the BF16 form
    void *bmap = nullptr;   // its CUtensorMap
    bool bvalid = false;
    void *w8 = nullptr;     // e4m3 copy [Cout][K] of w / scale[o] for the FP8 form
    void *w8map = nullptr;  // its CUtensorMap
    float *w8scale = nullptr;   // device, per output channel
    bool f8valid = false;
    int Cout = 0, T = 0, Cin = 0, Npad = 0, Kpad = 0;
    int cin8 = 0;           // e4m3 copy: Cin zero-padded to a multiple of 128 (one K chunk per 128 channels)
    bool im2col = false;    // few input channels: A gathered by the kernel, K zero-padded
    bool valid = false;
    TcWeights() = default;
    TcWeights(const TcWeights &) = delete;
    TcWeights &operator=(const TcWeights &) = delete;
    ~TcWeights();
};

// Build the tensor-core copy of weights [Cout][T][Cin] (host float32).
// Leaves valid = false when the shape is not handled by the kernels.
void build_weights(const float *w, int Cout, int T, int Cin, TcWeights *out);

// Whether the tensor-core kernel handles this launch.
bool can_run(const ConvDesc &d, const TcWeights &w);

// Launches the kernel; false (nothing launched) if a tensor map could not be
// encoded, in which case the caller runs the CUDA-core kernel instead.
bool launch(const ConvDesc &d, const TcWeights &w, cudaStream_t st);

// Whether launch() applies d.q_mode in the epilogue: the persistent Cout = 128
// kernel and its split-K sum (symbols or scale indices), the one-tile-per-CTA
// Cout = 192 kernel (symbols only: its epilogue, which nothing overlaps, ran
// the scale-index searches slower than the separate integer kernel).
bool tc_fuses_quant(const ConvDesc &d);

// The K slices launch() cuts each 128-pixel tile into (1: none).  Above 1 it
// runs a second kernel that adds the slices' partial sums in slice order.  The
// count depends on the layer and the frame size only (never on the batch, the
// buffers or the device), so a frame gets the same arithmetic in any batch.
int split_k(const ConvDesc &d, const TcWeights &w);

// Precision forms: bf16 or e4m3 activations in (d.in_dt), any storage out.
bool can_run_lp(const ConvDesc &d, const TcWeights &w);
bool launch_lp(const ConvDesc &d, const TcWeights &w, cudaStream_t st);

// Storage of one tensor map (a CUtensorMap, passed to kernels by value).
struct alignas(64) TmaMap {
    unsigned char raw[128];
};

// bf16 weights [Cout][K] in device memory (Cout 64, 128 or 192; K a multiple
// of 64; 16-byte aligned) -> the kernel's B-operand tensor map.
bool make_bf16_weight_map(TmaMap *m, const void *w, int Cout, int K);

// The bf16 kernel with caller-made weight maps (weights that change on the
// device, e.g. during training): Cout 64, 128 or 192; epilogues none, ReLU
// or EPI_MASK (d.gdn_x = the activation, stored like the output); d.bias
// may be null.  false = not launched.
bool can_run_lp_map(const ConvDesc &d);

// Weight gradient of a transposed conv 5x5 / stride 2 (pad 2) with bf16
// operands on tcgen05: x NHWC [B][H][W][Cin] (Cin 64, 128 or 192), dz NHWC
// [B][2H][2W][64], both device, 16-byte aligned.  Writes the float32 sums of
// wgrad_bf16_slices(B, H, W) pixel slices into part[z][Cin][25 * 64] (column
// tap * 64 + o, tap = 5u + v); the caller adds the slices in order.  false =
// not launched (shape or tensor map not handled).
int wgrad_bf16_slices(int B, int H, int W);
bool launch_wgrad_bf16(const void *x, const void *dz, int B, int H, int W, int Cin, float *part, uint32_t *status,
                       cudaStream_t st);

// The bounded mbarrier wait of the kernels, on a barrier nothing arrives at:
// gives up after limit_cycles and latches ST_TIMEOUT in *status.
void launch_wait_probe(uint32_t *status, long long limit_cycles, cudaStream_t st);

// Dense tensor-pipe rate (TFLOP/s) of back-to-back MMAs of M = 128, N = 256
// on every SM: kind 0 tf32, 1 bf16, 2 e4m3.  Synchronizes; LIC_OK or LIC_E_*.
int mma_rate(int kind, int iters, double *tflops);
bool launch_lp_map(const ConvDesc &d, const TmaMap &bmap, cudaStream_t st);

}  // namespace tc
}  // namespace lic
