// lic_encode_latents_noalloc: the entropy encoder without any allocation.
//
// Some callers cannot allocate device memory at the moment they need to
// encode: a real-time capture or streaming thread must not stall on
// cudaMalloc / cudaFree (cudaFree waits for every running kernel on the
// device), a host process may hand the GPU's memory to a fixed-budget
// allocator and leave nothing for a library to grab, and a plugin may be
// handed device buffers by its host with no allocator of its own.  For them
// this entry point runs the same rANS encode and container kernels as
// lic_encode_latents, with the caller's input and output buffers, and keeps
// its working memory (per-substream word buffers, word counts and offsets)
// in one fixed-size array compiled into the library instead of buffers it
// would allocate.
#include <cuda_runtime.h>

#include <atomic>

#include "lic_internal.h"

// The working memory of every call on a device: LIC_NOALLOC_SCRATCH_BYTES,
// resident for as long as the library is loaded on that device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LIC_NOALLOC_SCRATCH_BYTES];

namespace lic {
namespace {

constexpr int kMaxDevices = 64;
// Per device, the array's device address, published once found.  Two host
// threads may both look it up the first time; they store the same value.
// The cache assumes the module stays loaded: after cudaDeviceReset the
// library's device code is loaded afresh and these addresses are stale.
std::atomic<void *> g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
int scratch_address(int dev, void **ptr) {
    if (dev < 0 || dev >= kMaxDevices) return LIC_E_UNSUPPORTED;
    void *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return LIC_E_CUDA;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *ptr = p;
    return LIC_OK;
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int64_t align256(int64_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace lic

using namespace lic;

extern "C" int lic_encode_latents_noalloc(lic_codec *codec, const int32_t *s_y, const uint8_t *idx,
                                          const int32_t *s_z, int B, int H, int W, int Hy, int Wy, uint8_t *data,
                                          int64_t data_cap, int64_t *d_layout, void *stream) {
    CodecEntropyView v;
    if (codec_entropy_view(codec, &v) != LIC_OK) return LIC_E_INVALID_ARG;
    if (!s_y || !data || !d_layout || B < 1 || H < 1 || W < 1 || Hy < 1 || Wy < 1) return LIC_E_INVALID_ARG;
    if (v.kind == LIC_HYPERPRIOR && (!idx || !s_z || Hy % 4 || Wy % 4)) return LIC_E_INVALID_ARG;
    // The kernels store 32-bit container words into data and 64-bit offsets
    // into d_layout, and read every input on the device: a host pointer or a
    // misaligned output is refused here rather than faulting a kernel.
    if (!is_device_ptr(s_y) || !is_device_ptr(data) || !is_device_ptr(d_layout) ||
        (v.kind == LIC_HYPERPRIOR && (!is_device_ptr(idx) || !is_device_ptr(s_z))))
        return LIC_E_INVALID_ARG;
    if (!aligned(s_y, 4) || !aligned(data, 16) || !aligned(d_layout, 8) ||
        (v.kind == LIC_HYPERPRIOR && !aligned(s_z, 4)))
        return LIC_E_INVALID_ARG;
    // the codec's tables live on its own device: the call must run there
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LIC_E_CUDA;
    if (dev != v.device) return LIC_E_INVALID_ARG;
    const StreamGeom g = make_geom(v.kind, v.N, v.M, H, W, 16 * Hy, 16 * Wy, v.R, v.version, v.S);
    const int64_t subs = (int64_t)B * g.nsub;
    // scratch carve-up: words | counts | sub_off | frame_bytes
    const int64_t words_bytes = align256(subs * g.cap_words * (int64_t)sizeof(uint16_t));
    const int64_t counts_bytes = align256(subs * (int64_t)sizeof(int64_t));
    const int64_t frame_bytes = align256((int64_t)B * (int64_t)sizeof(int64_t));
    const int64_t need = words_bytes + 2 * counts_bytes + frame_bytes;
    if (need > (int64_t)LIC_NOALLOC_SCRATCH_BYTES) return LIC_E_UNSUPPORTED;
    // every frame is placed at a 16-byte aligned offset; worst-case sizes
    if (data_cap < (int64_t)B * g.frame_cap) return LIC_E_INVALID_ARG;
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc != LIC_OK) return rc;
    unsigned char *p = static_cast<unsigned char *>(base);
    uint16_t *words = reinterpret_cast<uint16_t *>(p);
    int64_t *counts = reinterpret_cast<int64_t *>(p + words_bytes);
    int64_t *sub_off = reinterpret_cast<int64_t *>(p + words_bytes + counts_bytes);
    int64_t *fbytes = reinterpret_cast<int64_t *>(p + words_bytes + 2 * counts_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // No scratch word needs clearing: each kernel reads only what an earlier
    // kernel of this call wrote (the encoder writes every count and the
    // words it counts; the scan writes every offset and frame size).
    launch_entropy_encode(g, B, v.tables, s_y, idx, s_z, words, counts, st);
    launch_entropy_compact(g, B, words, counts, sub_off, fbytes, d_layout, data, st);
    return cudaGetLastError() == cudaSuccess ? LIC_OK : LIC_E_CUDA;
}
