// Interleaved rANS entropy coder on the GPU (integer kernels).
//
// The paper runs CompressAI's CPU entropy coder (Sec. IV-B) and calls
// entropy coding the CPU-intensive part of the codec (Sec. III-A).  Here it
// runs on the device: every substream (one z channel, or one band of R
// latent rows of one y channel) is coded by one warp whose 32 lanes are the
// 32 interleaved rANS states of that substream (Giesen's interleaving of
// Duda's rANS).  Symbol i of a substream belongs to state i mod 32.
//
// Coder: state x in [2^16, 2^32), 16-bit renormalisation words, 16-bit CDFs.
//   encode(start, f): if x >= f * 2^16 emit x & 0xffff, x >>= 16;
//                     x = floor(x / f) * 2^16 + x mod f + start
//   decode: slot = x & 0xffff -> symbol with cdf[s] <= slot < cdf[s+1];
//           x = f * (x >> 16) + slot - start; if x < 2^16 refill one word.
// A value outside a table's support is sent as the escape symbol followed by
// uniform 4-bit symbols on the same state: (nibble count - 1), then the
// nibbles of zigzag(overflow), least significant first.
//
// Word order (the format): the encoder walks the symbols from last to first;
// inside a group of 32 symbols lane 31 emits first.  After the last symbol
// the states flush from lane 31 down to 0, high half then low half.  The
// substream is the emitted sequence reversed, so a decoder reads 32 initial
// states (lane 0 first, low half first) and then words in symbol order.  The
// warp reproduces that order exactly with ballots (one word per lane at
// most) or, in groups holding an escape, with a suffix sum of word counts.
#include "lic_internal.h"

namespace lic {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS = 4;
constexpr int MAX_WORDS_PER_SYMBOL = 10;  // escape + count nibble + 8 nibbles
constexpr uint32_t RANS_L = 1u << 16;

struct SubInfo {
    const int32_t *sym;   // first symbol of the substream
    const uint8_t *idx;   // per-symbol scale index (hyperprior y) or null
    int n;                // symbols
    int table;            // fixed table (z, factorized y) when idx is null
    int c;                // channel
    int p0;               // first latent pixel (row0 * width) in the plane
    bool is_z;
};

__device__ __forceinline__ SubInfo sub_info(const StreamGeom &g, int b, int q, const int32_t *s_y,
                                            const uint8_t *idx, const int32_t *s_z, const DevTables &t) {
    SubInfo si;
    if (q < g.nz) {
        int HWz = g.Hz * g.Wz;
        si.sym = s_z ? s_z + ((int64_t)b * g.N + q) * HWz : nullptr;
        si.idx = nullptr;
        si.n = HWz;
        si.table = q;
        si.c = q;
        si.p0 = 0;
        si.is_z = true;
    } else {
        int qq = q - g.nz;
        int c = qq / g.nbands, band = qq % g.nbands;
        int r0 = band * g.R;
        int rows = min(g.R, g.Hy - r0);
        int64_t plane = ((int64_t)b * g.M + c) * g.Hy * g.Wy;
        si.p0 = r0 * g.Wy;
        si.sym = s_y ? s_y + plane + si.p0 : nullptr;
        si.idx = (g.kind == LIC_HYPERPRIOR && idx) ? idx + plane + si.p0 : nullptr;
        si.n = rows * g.Wy;
        si.table = (g.kind == LIC_HYPERPRIOR) ? -1 : c;
        si.c = c;
        si.is_z = false;
    }
    return si;
}

__device__ __forceinline__ int nibble_count(uint32_t v) {
    int nn = 1;
    while (nn < 8 && (v >> (4 * nn)) != 0u) ++nn;
    return nn;
}

// One encode step; returns true (and the word) when it renormalised.
__device__ __forceinline__ bool enc_put(uint32_t &x, uint32_t start, uint32_t f, uint16_t &word) {
    bool emit = x >= (f << 16);
    if (emit) {
        word = (uint16_t)(x & 0xffffu);
        x >>= 16;
    }
    uint32_t q = x / f;
    x = (q << 16) + (x - q * f) + start;
    return emit;
}

__global__ void __launch_bounds__(WARPS * 32) rans_encode_kernel(const StreamGeom g, int B, const DevTables t,
                                                                 const int32_t *__restrict__ s_y,
                                                                 const uint8_t *__restrict__ idx,
                                                                 const int32_t *__restrict__ s_z,
                                                                 uint16_t *__restrict__ scratch,
                                                                 int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (warp >= (int64_t)B * g.nsub) return;
    const int b = (int)(warp / g.nsub), q = (int)(warp % g.nsub);
    const SubInfo si = sub_info(g, b, q, s_y, idx, s_z, t);
    const int64_t cap = g.cap_words;
    uint16_t *out = scratch + warp * cap;  // emitted word k -> out[cap - 1 - k]
    uint32_t x = RANS_L;
    int64_t E = 0;

    const int ngroups = (si.n + 31) / 32;
    for (int grp = ngroups - 1; grp >= 0; --grp) {
        const int i = grp * 32 + lane;
        const bool active = i < si.n;
        int tab = 0, lo = 0, hi = 0, sym = 0, esc = 0;
        uint32_t v = 0;
        int32_t s = 0;
        if (active) {
            s = si.sym[i];
            tab = si.idx ? t.gauss_base + si.idx[i] : si.table;
            lo = t.lo[tab];
            hi = t.hi[tab];
            esc = lo + hi + 1;
            if (s >= -lo && s <= hi) {
                sym = s + lo;
            } else {
                sym = esc;
                v = (s > hi) ? 2u * (uint32_t)(s - hi - 1) : 2u * (uint32_t)(-s - lo - 1) + 1u;
            }
        }
        const bool is_esc = active && sym == esc;
        if (!__any_sync(FULL, is_esc)) {
            // fast path: at most one word per lane; lanes above come first
            uint16_t w = 0;
            bool emit = false;
            if (active) {
                const uint32_t *cdf = t.cdf + t.start[tab];
                uint32_t st = cdf[sym], f = cdf[sym + 1] - st;
                emit = enc_put(x, st, f, w);
            }
            unsigned m = __ballot_sync(FULL, emit);
            if (emit) {
                int before = __popc(m & ~((2u << lane) - 1u));  // lanes > lane
                out[cap - 1 - (E + before)] = w;
            }
            E += __popc(m);
        } else {
            uint16_t w[MAX_WORDS_PER_SYMBOL];
            int cnt = 0;
            if (active) {
                if (is_esc) {
                    int nn = nibble_count(v);
                    for (int j = nn - 1; j >= 0; --j)
                        if (enc_put(x, 4096u * ((v >> (4 * j)) & 15u), 4096u, w[cnt])) ++cnt;
                    if (enc_put(x, 4096u * (uint32_t)(nn - 1), 4096u, w[cnt])) ++cnt;
                }
                const uint32_t *cdf = t.cdf + t.start[tab];
                uint32_t st = cdf[sym], f = cdf[sym + 1] - st;
                if (enc_put(x, st, f, w[cnt])) ++cnt;
            }
            // suffix sum over lanes: words of lanes > lane come first
            int incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int o = __shfl_down_sync(FULL, incl, d);
                if (lane + d < 32) incl += o;
            }
            int before = incl - cnt;
            int total = __shfl_sync(FULL, incl, 0);
            for (int j = 0; j < cnt; ++j) out[cap - 1 - (E + before + j)] = w[j];
            E += total;
        }
    }
    // flush: lane 31 first, high half then low half
    int64_t k = E + 2 * (31 - lane);
    out[cap - 1 - k] = (uint16_t)(x >> 16);
    out[cap - 2 - k] = (uint16_t)(x & 0xffffu);
    E += 64;
    if (lane == 0) counts[warp] = E;
}

// Per frame: exclusive scan of substream word counts, frame size in bytes.
__global__ void rans_scan_kernel(const StreamGeom g, const int64_t *__restrict__ counts,
                                 int64_t *__restrict__ sub_off, int64_t *__restrict__ frame_bytes,
                                 int64_t trailer_bytes) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < g.nsub; base += blockDim.x) {
        int q = base + threadIdx.x;
        int64_t v = q < g.nsub ? counts[(int64_t)b * g.nsub + q] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            int64_t o = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0;
            __syncthreads();
            part[threadIdx.x] += o;
            __syncthreads();
        }
        if (q < g.nsub) sub_off[(int64_t)b * g.nsub + q] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) frame_bytes[b] = g.header_bytes + 2 * carry + trailer_bytes;
}

// Frame placement: 16-byte aligned starts.  offsets has B+1 entries, then
// sizes (B entries) follow it in the same allocation.
__global__ void frame_place_kernel(int B, const int64_t *__restrict__ frame_bytes, int64_t *__restrict__ offsets) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t o = 0;
    for (int b = 0; b < B; ++b) {
        offsets[b] = o;
        offsets[B + 1 + b] = frame_bytes[b];
        o += (frame_bytes[b] + 15) / 16 * 16;
    }
    offsets[B] = o;
}

__global__ void __launch_bounds__(WARPS * 32) rans_write_kernel(const StreamGeom g, int B,
                                                                const uint16_t *__restrict__ scratch,
                                                                const int64_t *__restrict__ counts,
                                                                const int64_t *__restrict__ sub_off,
                                                                const int64_t *__restrict__ offsets,
                                                                uint8_t *__restrict__ data) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (warp >= (int64_t)B * g.nsub) return;
    const int b = (int)(warp / g.nsub), q = (int)(warp % g.nsub);
    uint8_t *frame = data + offsets[b];
    uint32_t *hdr = reinterpret_cast<uint32_t *>(frame);
    const int64_t nw = counts[warp];
    const int64_t off = sub_off[warp];
    if (q == 0 && lane == 0) {
        hdr[0] = 0x3143494Cu;  // "LIC1"
        hdr[1] = 1u | ((uint32_t)g.kind << 16);
        hdr[2] = (uint32_t)g.N | ((uint32_t)g.M << 16);
        hdr[3] = (uint32_t)g.H;
        hdr[4] = (uint32_t)g.W;
        hdr[5] = (uint32_t)g.Hp;
        hdr[6] = (uint32_t)g.Wp;
        hdr[7] = (uint32_t)g.R;
        hdr[8] = (uint32_t)g.nsub;
    }
    if (lane == 0) {
        hdr[9 + q] = (uint32_t)off;
        if (q == g.nsub - 1) hdr[9 + g.nsub] = (uint32_t)(off + nw);
    }
    uint16_t *dst = reinterpret_cast<uint16_t *>(frame + g.header_bytes) + off;
    const uint16_t *src = scratch + warp * g.cap_words + (g.cap_words - nw);
    for (int64_t k = lane; k < nw; k += 32) dst[k] = src[k];
}

__device__ __forceinline__ uint32_t rd_u32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__device__ __forceinline__ int find_symbol(const uint32_t *cdf, int n, uint32_t slot, const uint16_t *lut) {
    // largest s in [0, n) with cdf[s] <= slot (cdf[0] = 0, cdf[n] = 2^16),
    // searched between the symbols of the 256-slot bucket's two ends
    const int j = (int)(slot >> 8);
    int lo = lut[j], hi = min((int)lut[j + 1], n - 1);
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cdf[mid] <= slot) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Decoder: DEC_WARPS substreams per block.  The per-symbol table data sits
// in shared memory: for the Gaussian scale tables (hyperprior y) the slot
// lookups and (lo, symbol count, CDF start) of all 64 tables, staged once per
// block; for a substream with one fixed table (z, factorized y) that table's
// slot lookup in the warp's own row.  The next group's scale indices are
// loaded a group ahead.
constexpr int DEC_WARPS = 8;
constexpr int NGAUSS = 64;

__global__ void __launch_bounds__(DEC_WARPS * 32) rans_decode_kernel(const StreamGeom g, int B, int part,
                                                                 const DevTables t,
                                                                 const uint8_t *__restrict__ data,
                                                                 const int64_t *__restrict__ offsets,
                                                                 const int64_t *__restrict__ sizes,
                                                                 const uint8_t *__restrict__ idx,
                                                                 const float *__restrict__ med,
                                                                 int32_t *__restrict__ s_out,
                                                                 float *__restrict__ hat_out,
                                                                 uint32_t *__restrict__ status) {
    __shared__ uint16_t s_glut[NGAUSS * LUT_N];
    __shared__ int32_t s_glo[NGAUSS], s_gnt[NGAUSS];
    __shared__ int64_t s_gstart[NGAUSS];
    __shared__ uint16_t s_wlut[DEC_WARPS][LUT_N];
    // escape walk of a group: every lane's state after its symbol, read by all lanes
    __shared__ uint32_t s_ex[DEC_WARPS][32];
    const bool gauss = part == 1 && g.kind == LIC_HYPERPRIOR && t.gauss_base >= 0;
    if (gauss) {
        for (int e = threadIdx.x; e < NGAUSS * LUT_N; e += blockDim.x)
            s_glut[e] = t.lut[(int64_t)t.gauss_base * LUT_N + e];
        for (int e = threadIdx.x; e < NGAUSS; e += blockDim.x) {
            const int tab = t.gauss_base + e;
            s_glo[e] = t.lo[tab];
            s_gnt[e] = t.lo[tab] + t.hi[tab] + 2;
            s_gstart[e] = t.start[tab];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nq = part == 0 ? g.nz : g.nsub - g.nz;
    const int64_t warp = (int64_t)blockIdx.x * DEC_WARPS + wib;
    if (warp >= (int64_t)B * nq) return;
    const int b = (int)(warp / nq);
    const int q = (int)(warp % nq) + (part == 0 ? 0 : g.nz);

    // ---- header checks (bounded, never trust the stream) ----
    const int64_t fsize = sizes[b];
    const uint8_t *frame = data + offsets[b];
    bool bad = (offsets[b] & 1) != 0 || fsize < g.header_bytes;
    if (!bad) {
        bad = rd_u32(frame) != 0x3143494Cu || rd_u32(frame + 4) != (1u | ((uint32_t)g.kind << 16)) ||
              rd_u32(frame + 8) != ((uint32_t)g.N | ((uint32_t)g.M << 16)) ||
              rd_u32(frame + 12) != (uint32_t)g.H || rd_u32(frame + 16) != (uint32_t)g.W ||
              rd_u32(frame + 20) != (uint32_t)g.Hp || rd_u32(frame + 24) != (uint32_t)g.Wp ||
              rd_u32(frame + 28) != (uint32_t)g.R || rd_u32(frame + 32) != (uint32_t)g.nsub;
    }
    int64_t w0 = 0, w1 = 0;
    if (!bad) {
        int64_t avail = (fsize - g.header_bytes) / 2;
        w0 = rd_u32(frame + 36 + 4 * (int64_t)q);
        w1 = rd_u32(frame + 36 + 4 * (int64_t)(q + 1));
        int64_t wend = rd_u32(frame + 36 + 4 * (int64_t)g.nsub);
        bad = w1 < w0 || w1 > wend || wend > avail || (w1 - w0) < 64;
    }
    if (bad) {
        if (lane == 0) atomicOr(status, ST_CORRUPT);
        return;
    }
    const uint16_t *words = reinterpret_cast<const uint16_t *>(frame + g.header_bytes) + w0;
    const int64_t nw = w1 - w0;

    const SubInfo si = sub_info(g, b, q, nullptr, idx, nullptr, t);
    const int C = si.is_z ? g.N : g.M;
    const int HW = si.is_z ? g.Hz * g.Wz : g.Hy * g.Wy;
    int32_t *sdst = s_out + ((int64_t)b * C + si.c) * HW + si.p0;
    float *hdst = hat_out ? hat_out + ((int64_t)b * HW + si.p0) * C + si.c : nullptr;
    const float mu = (si.is_z || g.kind == LIC_FACTORIZED) ? med[si.c] : 0.f;

    // a substream with one table: its parameters in registers, its lookup in the warp's row
    int lo_f = 0, nt_f = 2;
    const uint32_t *cdf_f = t.cdf;
    const bool per_symbol = si.idx != nullptr;
    if ((per_symbol && !gauss) || (!per_symbol && si.table < 0)) {   // no table for these symbols
        if (lane == 0) atomicOr(status, ST_CORRUPT);
        return;
    }
    if (!per_symbol) {
        lo_f = t.lo[si.table];
        nt_f = lo_f + t.hi[si.table] + 2;
        cdf_f = t.cdf + t.start[si.table];
        for (int e = lane; e < LUT_N; e += 32) s_wlut[wib][e] = t.lut[(int64_t)si.table * LUT_N + e];
        __syncwarp();
    }

    uint32_t x = (uint32_t)words[2 * lane] | ((uint32_t)words[2 * lane + 1] << 16);
    int64_t pos = 64;
    bool corrupt = false;
    const int ngroups = (si.n + 31) / 32;
    int next_k = (per_symbol && lane < si.n) ? si.idx[lane] : 0;
    for (int grp = 0; grp < ngroups; ++grp) {
        const int i = grp * 32 + lane;
        const bool active = i < si.n;
        const int k = next_k;
        if (per_symbol) next_k = (i + 32 < si.n) ? si.idx[i + 32] : 0;   // a group ahead
        int lo = 0, nt = 2, sym = 0;
        bool need = false;
        if (active) {
            const uint32_t *cdf;
            const uint16_t *lut;
            if (per_symbol) {
                lo = s_glo[k];
                nt = s_gnt[k];
                cdf = t.cdf + s_gstart[k];
                lut = s_glut + k * LUT_N;
            } else {
                lo = lo_f;
                nt = nt_f;
                cdf = cdf_f;
                lut = s_wlut[wib];
            }
            uint32_t slot = x & 0xffffu;
            sym = find_symbol(cdf, nt, slot, lut);
            uint32_t st = cdf[sym], f = cdf[sym + 1] - st;
            x = f * (x >> 16) + slot - st;
            need = x < RANS_L;
        }
        const bool is_esc = active && sym == nt - 1;
        int32_t val = sym - lo;
        if (!__any_sync(FULL, is_esc)) {
            unsigned m = __ballot_sync(FULL, need);
            if (need) {
                int64_t p = pos + __popc(m & ((1u << lane) - 1u));
                if (p < nw) x = (x << 16) | words[p]; else corrupt = true;
            }
            pos += __popc(m);
        } else {
            // an escape's nibbles sit between its own word and the next lane's:
            // lanes between two escapes read their words in parallel (rank
            // among the renormalising lanes of the segment).  The nibbles are
            // uniform 4-bit symbols, and decoding one leaves the renormalisation
            // test (state < 2^16) to the state's high half h alone: h >> 4 without
            // a renormalisation; after one, the next three steps cannot
            // renormalise and the fourth sees the same h.  So the words an escape
            // consumes follow from its state when it starts (its count nibble
            // gives the number of steps): the walk over the escapes only adds
            // those counts, and the escape lanes then decode their nibbles at
            // once, each checking the count it predicted.
            const unsigned m_need = __ballot_sync(FULL, need);
            const unsigned m_esc = __ballot_sync(FULL, is_esc);
            // one lane walks the escapes in order: lane e's symbol word sits after the
            // renormalising lanes below it and the nibble words of the escapes below it
            s_ex[wib][lane] = x;
            __syncwarp();
            // every lane runs the same walk (no divergence): escape e's symbol word sits
            // after the renormalising lanes below it and the nibble words of the escapes
            // below it; each lane keeps what it needs
            int32_t W = 0, wb = 0, ewords = 0;
            for (unsigned m = m_esc; m; m &= m - 1u) {
                const int e = __ffs(m) - 1;
                const uint32_t xe = s_ex[wib][e];
                uint32_t h, low;
                if ((m_need >> e) & 1u) {   // its word becomes the state's low half
                    const int64_t P = pos + __popc(m_need & ((1u << e) - 1u)) + W;
                    low = P < nw ? words[P] : 0u;
                    if (P >= nw) corrupt = true;
                    h = xe;
                } else {
                    low = xe & 0xffffu;
                    h = xe >> 16;
                }
                const int steps = (int)(low >> 12) + 2;
                const int j0 = (h >= 16u) + (h >= 256u) + (h >= 4096u);
                const int w = steps > j0 ? (steps - 1 - j0) / 4 + 1 : 0;
                if (e == lane) {
                    wb = W;   // an escape lane: the nibble words before its own
                    ewords = w;
                } else if (e < lane) {
                    wb = W + w;   // a lane above escape e
                }
                W += w;
            }
            const int64_t psym = pos + __popc(m_need & ((1u << lane) - 1u)) + wb;
            if (need) {
                if (psym < nw) x = (x << 16) | words[psym]; else corrupt = true;
            }
            const int64_t epos = psym + (need ? 1 : 0);   // escape lanes: their nibbles' first word
            pos += __popc(m_need) + W;
            __syncwarp();   // s_ex is rewritten by the next group
            if (is_esc && !corrupt) {
                int64_t p = epos;
                uint32_t v = 0, nn = 0;
                for (int j = -1; j < (int)nn && !corrupt; ++j) {
                    uint32_t slot = x & 0xffffu;
                    uint32_t nib = slot >> 12;
                    x = 4096u * (x >> 16) + slot - 4096u * nib;
                    if (x < RANS_L) {
                        if (p < nw) x = (x << 16) | words[p]; else corrupt = true;
                        ++p;
                    }
                    if (j < 0) {
                        nn = nib + 1;
                        if (nn > 8) corrupt = true;
                    } else {
                        v |= nib << (4 * j);
                    }
                }
                // a state below 2^16 here (no stream this coder wrote) breaks the count
                if (p - epos != ewords) corrupt = true;
                int64_t r = (v & 1u) ? -(int64_t)lo - 1 - (int64_t)(v >> 1)
                                     : (int64_t)(nt - 2 - lo) + 1 + (int64_t)(v >> 1);
                if (r > 1073741824LL || r < -1073741824LL) corrupt = true;
                val = (int32_t)r;
            }
        }
        if (__any_sync(FULL, corrupt)) {
            if (lane == 0) atomicOr(status, ST_CORRUPT);
            return;
        }
        if (active) {
            sdst[i] = val;
            if (hdst) hdst[(int64_t)i * C] = __fadd_rn(__int2float_rn(val), mu);
        }
    }
}

int64_t blocks_for(int64_t warps) { return (warps + WARPS - 1) / WARPS; }

}  // namespace

StreamGeom make_geom(int kind, int N, int M, int H, int W, int Hp, int Wp, int R, int version, int S) {
    StreamGeom g{};
    g.kind = kind;
    g.N = N;
    g.M = M;
    g.H = H;
    g.W = W;
    g.Hp = Hp;
    g.Wp = Wp;
    g.Hy = Hp / 16;
    g.Wy = Wp / 16;
    g.Hz = Hp / 64;
    g.Wz = Wp / 64;
    g.R = R;
    g.nbands = (g.Hy + R - 1) / R;
    g.nz = kind == LIC_HYPERPRIOR ? N : 0;
    g.nsub = g.nz + M * g.nbands;
    g.header_bytes = 36 + 4 * (int64_t)(g.nsub + 1);
    int64_t nmax = (int64_t)std::min(R, g.Hy) * g.Wy;
    if (kind == LIC_HYPERPRIOR) nmax = std::max<int64_t>(nmax, (int64_t)g.Hz * g.Wz);
    g.version = version == 2 ? 2 : 1;
    g.S = g.version == 2 && S > 0 ? S : 0;
    auto nrec = [&](int64_t n) -> int {
        const int64_t ng = (n + 31) / 32;
        return (g.S > 0 && ng > 0) ? (int)((ng - 1) / g.S) : 0;
    };
    const int last_rows = g.Hy - (g.nbands - 1) * R;
    g.nr_z = kind == LIC_HYPERPRIOR ? nrec((int64_t)g.Hz * g.Wz) : 0;
    g.nr_full = nrec((int64_t)std::min(R, g.Hy) * g.Wy);
    g.nr_last = nrec((int64_t)last_rows * g.Wy);
    g.rec_per_frame = (int64_t)g.nz * g.nr_z + (int64_t)M * ((int64_t)(g.nbands - 1) * g.nr_full + g.nr_last);
    if (g.version == 1) {
        g.cap_words = MAX_WORDS_PER_SYMBOL * nmax + 64;
        g.cap_r = g.cap_p32 = g.cap_c32 = 0;
    } else {
        // at most one rANS word per symbol plus the flush; 8 payload nibbles and one
        // count nibble per escape; the records of the longest substream
        const int64_t nr_max = (g.S > 0) ? ((nmax + 31) / 32 - 1) / g.S + 1 : 0;
        g.cap_r = (nmax + 64 + 1) / 2 * 2;
        g.cap_p32 = nmax + 1;
        g.cap_c32 = nmax / 8 + 1;
        g.cap_words = 8 + g.cap_r + 2 * (g.cap_p32 + g.cap_c32 + 35 * nr_max);
    }
    // every frame starts 16-byte aligned; format 2 adds its record trailer (at most the
    // records' scratch, which cap_words holds)
    g.frame_cap = g.header_bytes + 2 * (int64_t)g.nsub * g.cap_words + 16;
    return g;
}

void launch_rans_encode(const StreamGeom &g, int B, const DevTables &t, const int32_t *s_y, const uint8_t *idx,
                        const int32_t *s_z, uint16_t *scratch, int64_t *counts, cudaStream_t st) {
    int64_t warps = (int64_t)B * g.nsub;
    rans_encode_kernel<<<(unsigned)blocks_for(warps), WARPS * 32, 0, st>>>(g, B, t, s_y, idx, s_z, scratch, counts);
}

void launch_rans_scan(const StreamGeom &g, int B, const int64_t *counts, int64_t *sub_off, int64_t *frame_bytes,
                      int64_t trailer_bytes, cudaStream_t st) {
    rans_scan_kernel<<<B, 1024, 0, st>>>(g, counts, sub_off, frame_bytes, trailer_bytes);
}

void launch_frame_place(int B, const int64_t *frame_bytes, int64_t *offsets, cudaStream_t st) {
    frame_place_kernel<<<1, 32, 0, st>>>(B, frame_bytes, offsets);
}

void launch_rans_compact(const StreamGeom &g, int B, const uint16_t *scratch, const int64_t *counts,
                         int64_t *sub_off, int64_t *frame_bytes, int64_t *offsets, uint8_t *data,
                         cudaStream_t st) {
    launch_rans_scan(g, B, counts, sub_off, frame_bytes, 0, st);
    launch_frame_place(B, frame_bytes, offsets, st);
    int64_t warps = (int64_t)B * g.nsub;
    rans_write_kernel<<<(unsigned)blocks_for(warps), WARPS * 32, 0, st>>>(g, B, scratch, counts, sub_off, offsets,
                                                                          data);
}

void launch_entropy_encode(const StreamGeom &g, int B, const DevTables &t, const int32_t *s_y, const uint8_t *idx,
                           const int32_t *s_z, uint16_t *scratch, int64_t *counts, cudaStream_t st) {
    if (g.version == 2) launch_rans2_encode(g, B, t, s_y, idx, s_z, scratch, counts, st);
    else launch_rans_encode(g, B, t, s_y, idx, s_z, scratch, counts, st);
}

void launch_entropy_compact(const StreamGeom &g, int B, const uint16_t *scratch, const int64_t *counts,
                            int64_t *sub_off, int64_t *frame_bytes, int64_t *offsets, uint8_t *data,
                            cudaStream_t st) {
    if (g.version == 2) launch_rans2_compact(g, B, scratch, counts, sub_off, frame_bytes, offsets, data, st);
    else launch_rans_compact(g, B, scratch, counts, sub_off, frame_bytes, offsets, data, st);
}

void launch_entropy_decode(const StreamGeom &g, int B, int part, const DevTables &t, const uint8_t *data,
                           const int64_t *offsets, const int64_t *sizes, const uint8_t *idx, const float *med,
                           int32_t *s_out, float *hat_out, uint32_t *status, cudaStream_t st) {
    if (g.version == 2) launch_rans2_decode(g, B, part, t, data, offsets, sizes, idx, med, s_out, hat_out, status, st);
    else launch_rans_decode(g, B, part, t, data, offsets, sizes, idx, med, s_out, hat_out, status, st);
}

void launch_rans_decode(const StreamGeom &g, int B, int part, const DevTables &t, const uint8_t *data,
                        const int64_t *offsets, const int64_t *sizes, const uint8_t *idx, const float *med,
                        int32_t *s_out, float *hat_out, uint32_t *status, cudaStream_t st) {
    int nq = part == 0 ? g.nz : g.nsub - g.nz;
    int64_t warps = (int64_t)B * nq;
    if (warps == 0) return;
    const unsigned blocks = (unsigned)((warps + DEC_WARPS - 1) / DEC_WARPS);
    rans_decode_kernel<<<blocks, DEC_WARPS * 32, 0, st>>>(g, B, part, t, data, offsets, sizes, idx, med, s_out,
                                                          hat_out, status);
}

}  // namespace lic
