// Tensor-core (tcgen05) implicit-GEMM convolution -- not built yet; every
// launch is reported as unsupported so the CUDA-core kernels run.
#include "conv_tc.h"

namespace lic {
namespace tc {

TcWeights::~TcWeights() {
    if (hi) cudaFree(hi);
    if (lo) cudaFree(lo);
}

void build_weights(const float *, int Cout, int T, int Cin, TcWeights *out) {
    out->Cout = Cout;
    out->T = T;
    out->Cin = Cin;
    out->valid = false;
}

bool can_run(const ConvDesc &, const TcWeights &) { return false; }

void launch(const ConvDesc &, const TcWeights &, cudaStream_t) {}

}  // namespace tc
}  // namespace lic
