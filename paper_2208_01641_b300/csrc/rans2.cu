// Interleaved rANS, substream format 2: escape payloads outside the rANS
// words, and resume records for decoder-adaptive parallel decoding.
//
// The paper names higher-performance entropy coders as the next step for its
// pipeline (Sec. VII).  Format 1 (rans.cu) codes an escape as the escape
// symbol followed by uniform 4-bit rANS symbols on the same state, so a
// decoder must walk every escape of a group in turn to find where the next
// lane's word lies; one warp per 16-row band keeps enough warps busy, at the
// price of one 32-state flush per band.  Format 2 keeps the same coder (32
// interleaved states, state in [2^16, 2^32), 16-bit words, 16-bit CDFs) but
// codes an escape as the escape symbol alone: its payload nibbles go to a
// section after the rANS words and its nibble count to a section that grows
// from the substream's end.  Every group of 32 symbols then decodes in one
// step, escapes resolved together by prefix sums, and a whole latent plane
// can be one substream (one flush per plane).  Optional resume records every
// S groups (the next word's position, the escape and payload positions and
// the 32 lane states) sit in a trailer after the substreams; a decoder may
// start a warp at each record or ignore them, and a sender may strip them.
//
// Substream (16-bit words, L in all): u32 nw; nw rANS words in decoder order
// (32 initial states, then renormalisation words in symbol order); payload
// nibbles (escape k's nibbles of its zigzag overflow, least significant
// first, at nibble positions Q_k.., 4 per word from bit 0); count nibbles
// (n_k - 1 of escape k in word L-1-k/4 at bits 4 (k mod 4)).  Record (35 u32,
// stored as 70 little-endian words): P (next rANS word index at the start
// of group G, relative to the rANS section), E (escapes before G), Q
// (payload nibbles before G), the 32 lane states there.
#include "lic_internal.h"

namespace lic {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t RANS_L = 1u << 16;
constexpr int ENC_WARPS = 8;
constexpr int DEC_WARPS = 8;
constexpr int NG = 64;          // Gaussian scale tables
constexpr int REC = 35;         // u32 per resume record
constexpr int FIX_CDF = 4096;   // a single table's entries (without the final 2^16)
constexpr int FIX_LUT = 264;    // LUT_N rounded up to 8

// dynamic shared memory: the Gaussian image (whole for the decoder, without
// the slot lookups for the encoder), or one fixed table per decoder warp
constexpr size_t FIXED_SMEM = (size_t)DEC_WARPS * (FIX_CDF + FIX_LUT) * 2;
constexpr size_t DEC_SMEM = RANS2_GIMG_BYTES > FIXED_SMEM ? RANS2_GIMG_BYTES : FIXED_SMEM;
constexpr size_t ENC_SMEM = RANS2_GIMG_CDF_BYTES;

// One substream of a frame: what it codes and where its records go.
struct Sub {
    bool is_z;
    int c;          // channel
    int n;          // symbols
    int p0;         // first symbol's index in the channel's plane
    int table;      // fixed table (z, factorized y) or -1 (per-symbol scale index)
    int nr;         // resume records
    int64_t rbase;  // records of the frame's earlier substreams
};

__device__ __forceinline__ Sub sub_of(const StreamGeom &g, int q) {
    Sub s;
    if (q < g.nz) {
        s.is_z = true;
        s.c = q;
        s.n = g.Hz * g.Wz;
        s.p0 = 0;
        s.table = q;
        s.nr = g.nr_z;
        s.rbase = (int64_t)q * g.nr_z;
    } else {
        const int qq = q - g.nz;
        const int c = qq / g.nbands, band = qq % g.nbands;
        const int r0 = band * g.R;
        s.is_z = false;
        s.c = c;
        s.n = min(g.R, g.Hy - r0) * g.Wy;
        s.p0 = r0 * g.Wy;
        s.table = g.kind == LIC_HYPERPRIOR ? -1 : c;
        s.nr = band == g.nbands - 1 ? g.nr_last : g.nr_full;
        const int64_t perch = (int64_t)(g.nbands - 1) * g.nr_full + g.nr_last;
        s.rbase = (int64_t)g.nz * g.nr_z + (int64_t)c * perch + (int64_t)band * g.nr_full;
    }
    return s;
}

// Records of a frame whose substreams carry one every S groups (S = 0: none).
__device__ __forceinline__ int64_t recs_per_frame(const StreamGeom &g, int S) {
    if (S <= 0) return 0;
    auto nrec = [&](int64_t n) -> int64_t {
        const int64_t ng = (n + 31) / 32;
        return ng > 0 ? (ng - 1) / S : 0;
    };
    const int last_rows = g.Hy - (g.nbands - 1) * g.R;
    return (int64_t)g.nz * nrec((int64_t)g.Hz * g.Wz) +
           (int64_t)g.M * ((int64_t)(g.nbands - 1) * nrec((int64_t)g.R * g.Wy) + nrec((int64_t)last_rows * g.Wy));
}

// Exclusive prefix sum (over lower lanes) and total of nn in [1, 8] on the
// lanes of mask `me` (0 elsewhere): nn - 1 has three bits, each counted by a
// ballot, so the sums take three ballots and popcounts instead of a scan.
__device__ __forceinline__ void nibble_prefix(unsigned me, int nn, bool esc, int lane, int &excl, int &total) {
    const unsigned lt = (1u << lane) - 1u;
    const int m1 = esc ? nn - 1 : 0;
    const unsigned b0 = __ballot_sync(0xffffffffu, m1 & 1), b1 = __ballot_sync(0xffffffffu, m1 & 2),
                   b2 = __ballot_sync(0xffffffffu, m1 & 4);
    excl = __popc(me & lt) + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
    total = __popc(me) + __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
}

__device__ __forceinline__ int nibble_count(uint32_t v) {
    int nn = 1;
    while (nn < 8 && (v >> (4 * nn)) != 0u) ++nn;
    return nn;
}

__device__ __forceinline__ bool enc_put(uint32_t &x, uint32_t start, uint32_t f, uint16_t &word) {
    const bool emit = x >= (f << 16);
    if (emit) {
        word = (uint16_t)(x & 0xffffu);
        x >>= 16;
    }
    const uint32_t q = x / f;
    x = (q << 16) + (x - q * f) + start;
    return emit;
}

// The first `bytes` of the Gaussian image (a multiple of 16) into shared
// memory, 16 bytes a thread at a time; every thread of the block takes part.
__device__ __forceinline__ void stage_image(const DevTables &t, uint8_t *sm, int bytes) {
    const uint4 *src = reinterpret_cast<const uint4 *>(t.gimg);
    uint4 *dst = reinterpret_cast<uint4 *>(sm);
    for (int e = threadIdx.x; e < bytes / 16; e += blockDim.x) dst[e] = src[e];
    __syncthreads();
}

// A table's view for one symbol: lo, symbol count n (escape = n - 1) and its
// CDF, 16-bit in shared memory (entry n = 2^16 implied) or 32-bit in global.
struct Tab {
    int lo, n;
    const uint16_t *cs;
    const uint32_t *cg;
    __device__ __forceinline__ uint32_t at(int i) const {
        return cs ? (i < n ? (uint32_t)cs[i] : 65536u) : cg[i];
    }
};

// ------------------------------------------------------------------ encoder

__global__ void __launch_bounds__(ENC_WARPS * 32) rans2_encode_kernel(const StreamGeom g, int B, const DevTables t,
                                                                      const int32_t *__restrict__ s_y,
                                                                      const uint8_t *__restrict__ idx,
                                                                      const int32_t *__restrict__ s_z,
                                                                      uint16_t *__restrict__ scratch,
                                                                      int64_t *__restrict__ counts) {
    extern __shared__ __align__(16) uint8_t e_sm[];
    __shared__ uint32_t s_pay[ENC_WARPS][64];
    __shared__ uint32_t s_cnt[ENC_WARPS][8];
    const bool staged = g.kind == LIC_HYPERPRIOR && t.gimg != nullptr && idx != nullptr;
    if (staged) stage_image(t, e_sm, RANS2_GIMG_CDF_BYTES);
    const int32_t *s_lo = reinterpret_cast<const int32_t *>(e_sm), *s_n = s_lo + NG, *s_cs = s_lo + 2 * NG;
    const uint16_t *e_cdf = reinterpret_cast<const uint16_t *>(e_sm + RANS2_GIMG_HDR);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // two warps per substream: role 0 packs the escape nibbles (pass 1), role 1
    // writes the rANS words and the records (pass 2); neither needs the other
    const int64_t gw = (int64_t)blockIdx.x * ENC_WARPS + wib;
    if (gw >= 2 * (int64_t)B * g.nsub) return;
    const int role = (int)(gw & 1);
    const int64_t warp = gw >> 1;
    const int b = (int)(warp / g.nsub), q = (int)(warp % g.nsub);
    const Sub si = sub_of(g, q);
    const int64_t plane = si.is_z ? ((int64_t)b * g.N + si.c) * g.Hz * g.Wz : ((int64_t)b * g.M + si.c) * g.Hy * g.Wy;
    const int32_t *sym = (si.is_z ? s_z : s_y) + plane + si.p0;
    const uint8_t *ix = si.table < 0 ? idx + plane + si.p0 : nullptr;
    uint16_t *base = scratch + warp * g.cap_words;
    uint32_t *meta = reinterpret_cast<uint32_t *>(base);
    uint16_t *rw = base + 8;
    uint32_t *pay = reinterpret_cast<uint32_t *>(base + 8 + g.cap_r);
    uint32_t *cnt = pay + g.cap_p32;
    uint32_t *rec = cnt + g.cap_c32;
    // the table of a symbol: fixed, or by its scale index (from the staged image; global
    // memory only if a codec had no image, which format-2 hyperprior codecs always have)
    Tab fixed{0, 2, nullptr, t.cdf};
    if (si.table >= 0) {
        fixed.lo = t.lo[si.table];
        fixed.n = fixed.lo + t.hi[si.table] + 2;
        fixed.cg = t.cdf + t.start[si.table];
    }
    const int ngroups = (si.n + 31) / 32;

    // symbols and scale indices by blocks of 4 groups (128 symbols): lane l holds
    // symbols 4l .. 4l+3 of a block (one 16-byte load where aligned) and their
    // indices in one word; a group's value comes by shuffle
    const bool sym_al = (reinterpret_cast<uintptr_t>(sym) & 15) == 0;
    auto ld_sblk = [&](int b4) -> int4 {
        const int i0 = 128 * b4 + 4 * lane;
        if (b4 >= 0 && sym_al && i0 + 3 < si.n) return *reinterpret_cast<const int4 *>(sym + i0);
        int4 v = make_int4(0, 0, 0, 0);
        if (b4 >= 0) {
            if (i0 < si.n) v.x = sym[i0];
            if (i0 + 1 < si.n) v.y = sym[i0 + 1];
            if (i0 + 2 < si.n) v.z = sym[i0 + 2];
            if (i0 + 3 < si.n) v.w = sym[i0 + 3];
        }
        return v;
    };
    auto ld_kblk = [&](int b4) -> uint32_t {
        const int i0 = 128 * b4 + 4 * lane;
        if (!ix || b4 < 0) return 0u;
        if (i0 + 3 < si.n) return *reinterpret_cast<const uint32_t *>(ix + i0);
        uint32_t v = 0;
        for (int e = 0; e < 4; ++e)
            if (i0 + e < si.n) v |= (uint32_t)ix[i0 + e] << (8 * e);
        return v;
    };
    auto sym_of = [&](const int4 &bl, int grp) -> int32_t {
        const int src = 8 * (grp & 3) + (lane >> 2);
        const int a = __shfl_sync(FULL, bl.x, src), b2 = __shfl_sync(FULL, bl.y, src);
        const int c = __shfl_sync(FULL, bl.z, src), d = __shfl_sync(FULL, bl.w, src);
        const int e = lane & 3;
        return e == 0 ? a : (e == 1 ? b2 : (e == 2 ? c : d));
    };
    auto k_of = [&](uint32_t bl, int grp) -> int {
        return (int)((__shfl_sync(FULL, bl, 8 * (grp & 3) + (lane >> 2)) >> (8 * (lane & 3))) & 0xffu);
    };
    auto tab_k = [&](int k) -> Tab {
        if (si.table >= 0) return fixed;
        if (staged) return Tab{s_lo[k], s_n[k], e_cdf + s_cs[k], nullptr};
        const int tab = t.gauss_base + k;
        return Tab{t.lo[tab], t.lo[tab] + t.hi[tab] + 2, nullptr, t.cdf + t.start[tab]};
    };

    // What a lane codes for its symbol in group grp of block data (sb, kb): the
    // coding interval (start, f) of the symbol or of the escape, and for an
    // escape its payload v and nibble count nn (0 otherwise).  Independent of
    // the rANS state, so a block's four groups are looked up together.
    auto lookup = [&](const int4 &sbl, uint32_t kbl, int grp, uint32_t &st, uint32_t &f, uint32_t &v, int &nn) {
        const int i = grp * 32 + lane;
        const int32_t s = sym_of(sbl, grp);
        const int k = k_of(kbl, grp);
        st = 0;
        f = 0;
        v = 0;
        nn = 0;
        if (i < si.n) {
            const Tab tb = tab_k(k);
            const int hi = tb.n - 2 - tb.lo;
            int c = s + tb.lo;
            if (s < -tb.lo || s > hi) {
                c = tb.n - 1;
                v = s > hi ? 2u * (uint32_t)(s - hi - 1) : 2u * (uint32_t)(-s - tb.lo - 1) + 1u;
                nn = nibble_count(v);
            }
            st = tb.at(c);
            f = tb.at(c + 1) - st;
        }
    };

    // ---- pass 1, forward: escape payload and count nibbles in symbol order ----
    const int nblk = (ngroups + 3) >> 2;
    if (role == 0) {
    int64_t ne = 0, np = 0;
    uint32_t pay_carry = 0, cnt_carry = 0;
    int4 sb = ld_sblk(0), sb_next = ld_sblk(1);
    uint32_t kb = ld_kblk(0), kb_next = ld_kblk(1);
    for (int bk = 0; bk < nblk; ++bk) {
        if (bk > 0) {
            sb = sb_next;
            kb = kb_next;
            sb_next = ld_sblk(bk + 1);
            kb_next = ld_kblk(bk + 1);
        }
        uint32_t v4[4];
        int nn4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t st, f;
            lookup(sb, kb, 4 * bk + h, st, f, v4[h], nn4[h]);
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const bool esc = nn4[h] > 0;
            const int nn = nn4[h];
            const uint32_t v = v4[h];
            const unsigned me = __ballot_sync(FULL, esc);
            if (!me) continue;
            int excl, T;
            nibble_prefix(me, nn, esc, lane, excl, T);
            const int rk = __popc(me & ((1u << lane) - 1u)), te = __popc(me);
            // payload nibbles, staged per u32 unit from unit np / 8 (its earlier nibbles
            // carried): an escape's nn nibbles touch two units at most
            s_pay[wib][lane] = 0u;
            s_pay[wib][lane + 32] = 0u;
            __syncwarp();
            if (lane == 0) s_pay[wib][0] = pay_carry;
            __syncwarp();
            const int p0 = (int)(np & 7);
            if (esc) {
                const int o = p0 + excl, sh = 4 * (o & 7);
                atomicOr(&s_pay[wib][o >> 3], v << sh);
                if (sh && (o & 7) + nn > 8) atomicOr(&s_pay[wib][(o >> 3) + 1], v >> (32 - sh));
            }
            // count nibbles, likewise from unit ne / 8
            if (lane < 8) s_cnt[wib][lane] = 0u;
            __syncwarp();
            if (lane == 0) s_cnt[wib][0] = cnt_carry;
            __syncwarp();
            const int c0 = (int)(ne & 7);
            if (esc) {
                const int p = c0 + rk;
                atomicOr(&s_cnt[wib][p >> 3], (uint32_t)(nn - 1) << (4 * (p & 7)));
            }
            __syncwarp();
            const int pend = p0 + T, cend = c0 + te;
            const int64_t U0 = np >> 3, C0 = ne >> 3;
            for (int u = lane; u < (pend + 7) >> 3; u += 32) pay[U0 + u] = s_pay[wib][u];
            if (lane < ((cend + 7) >> 3)) cnt[C0 + lane] = s_cnt[wib][lane];
            pay_carry = (pend & 7) ? s_pay[wib][pend >> 3] : 0u;
            cnt_carry = (cend & 7) ? s_cnt[wib][cend >> 3] : 0u;
            __syncwarp();
            ne += te;
            np += T;
        }
    }

    if (lane == 0) {
        meta[1] = (uint32_t)ne;
        meta[2] = (uint32_t)np;
    }
    return;
    }

    // ---- pass 2, backward: the rANS words (at most one per lane and group) ----
    const int64_t cap = g.cap_r;   // emitted word k -> rw[cap - 1 - k]
    uint32_t x = RANS_L;
    int64_t E = 0, e_ge = 0, q_ge = 0;
    int4 sb = ld_sblk(nblk - 1), sb_next = ld_sblk(nblk - 2);
    uint32_t kb = ld_kblk(nblk - 1), kb_next = ld_kblk(nblk - 2);
    for (int bk = nblk - 1; bk >= 0; --bk) {
        if (bk < nblk - 1) {
            sb = sb_next;
            kb = kb_next;
            sb_next = ld_sblk(bk - 1);
            kb_next = ld_kblk(bk - 1);
        }
        uint32_t st4[4], f4[4];
        int nn4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t v;
            lookup(sb, kb, 4 * bk + h, st4[h], f4[h], v, nn4[h]);
        }
#pragma unroll
        for (int h = 3; h >= 0; --h) {
            const int grp = 4 * bk + h;
            if (grp >= ngroups) continue;
            const int i = grp * 32 + lane;
            uint16_t w = 0;
            const bool emit = i < si.n && enc_put(x, st4[h], f4[h], w);
            const unsigned m = __ballot_sync(FULL, emit);
            if (emit) rw[cap - 1 - (E + __popc(m & ~((2u << lane) - 1u)))] = w;   // lanes above come first
            E += __popc(m);
            const unsigned me = __ballot_sync(FULL, nn4[h] > 0);
            if (me) {
                int sum = nn4[h];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(FULL, sum, d);
                e_ge += __popc(me);
                q_ge += sum;
            }
            if (g.S > 0 && grp > 0 && grp % g.S == 0) {   // decoder state at the start of group grp
                uint32_t *R = rec + (int64_t)REC * (grp / g.S - 1);
                R[3 + lane] = x;
                if (lane == 0) {
                    R[0] = (uint32_t)E;      // words of groups >= grp: the compaction makes them P
                    R[1] = (uint32_t)e_ge;   // escapes of groups >= grp
                    R[2] = (uint32_t)q_ge;   // payload nibbles of groups >= grp
                }
            }
        }
    }
    // flush: lane 31 first, high half then low half
    const int64_t k = E + 2 * (31 - lane);
    rw[cap - 1 - k] = (uint16_t)(x >> 16);
    rw[cap - 2 - k] = (uint16_t)(x & 0xffffu);
    E += 64;
    if (lane == 0) {
        meta[0] = (uint32_t)E;
        meta[3] = (uint32_t)si.nr;
    }
}

// Each substream's length in words, once both of its encoder warps are done.
__global__ void rans2_len_kernel(const StreamGeom g, int B, const uint16_t *__restrict__ scratch,
                                 int64_t *__restrict__ counts) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= (int64_t)B * g.nsub) return;
    const uint32_t *meta = reinterpret_cast<const uint32_t *>(scratch + u * g.cap_words);
    counts[u] = 2 + (int64_t)meta[0] + ((int64_t)meta[2] + 3) / 4 + ((int64_t)meta[1] + 3) / 4;
}

// ------------------------------------------------------------------ compaction

__global__ void __launch_bounds__(ENC_WARPS * 32) rans2_write_kernel(const StreamGeom g, int B,
                                                                     const uint16_t *__restrict__ scratch,
                                                                     const int64_t *__restrict__ counts,
                                                                     const int64_t *__restrict__ sub_off,
                                                                     const int64_t *__restrict__ offsets,
                                                                     uint8_t *__restrict__ data) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * ENC_WARPS + (threadIdx.x >> 5);
    if (warp >= (int64_t)B * g.nsub) return;
    const int b = (int)(warp / g.nsub), q = (int)(warp % g.nsub);
    uint8_t *frame = data + offsets[b];
    uint32_t *hdr = reinterpret_cast<uint32_t *>(frame);
    const int64_t L = counts[warp];
    const int64_t off = sub_off[warp];
    if (q == 0 && lane == 0) {
        hdr[0] = 0x3143494Cu;  // "LIC1"
        hdr[1] = 2u | ((uint32_t)g.kind << 16);
        hdr[2] = (uint32_t)g.N | ((uint32_t)g.M << 16);
        hdr[3] = (uint32_t)g.H;
        hdr[4] = (uint32_t)g.W;
        hdr[5] = (uint32_t)g.Hp;
        hdr[6] = (uint32_t)g.Wp;
        hdr[7] = (uint32_t)g.R | ((uint32_t)g.S << 16);
        hdr[8] = (uint32_t)g.nsub;
    }
    if (lane == 0) {
        hdr[9 + q] = (uint32_t)off;
        if (q == g.nsub - 1) hdr[9 + g.nsub] = (uint32_t)(off + L);
    }
    const uint16_t *base = scratch + warp * g.cap_words;
    const uint32_t *meta = reinterpret_cast<const uint32_t *>(base);
    const int64_t nw = meta[0], ne = meta[1], np = meta[2];
    const int nr = (int)meta[3];
    const uint16_t *rw = base + 8 + (g.cap_r - nw);
    const uint16_t *pw = base + 8 + g.cap_r;
    const uint16_t *cw = pw + 2 * g.cap_p32;
    const uint32_t *rec = reinterpret_cast<const uint32_t *>(cw + 2 * g.cap_c32);
    uint16_t *dst = reinterpret_cast<uint16_t *>(frame + g.header_bytes) + off;
    if (lane == 0) {
        dst[0] = (uint16_t)(nw & 0xffff);
        dst[1] = (uint16_t)(nw >> 16);
    }
    for (int64_t k = lane; k < nw; k += 32) dst[2 + k] = rw[k];
    const int64_t npw = (np + 3) / 4, ncw = (ne + 3) / 4;
    for (int64_t k = lane; k < npw; k += 32) dst[2 + nw + k] = pw[k];
    for (int64_t k = lane; k < ncw; k += 32) dst[L - 1 - k] = cw[k];
    // the resume records, after every substream of the frame (16-bit halves: the trailer
    // need not be 4-byte aligned)
    const int64_t fsize = offsets[B + 1 + b];
    uint16_t *trail = reinterpret_cast<uint16_t *>(frame + (fsize - 4 * REC * g.rec_per_frame));
    const int64_t rbase = sub_of(g, q).rbase;
    for (int r = 0; r < nr; ++r) {
        const uint32_t *R = rec + (int64_t)REC * r;
        uint32_t v;
        if (lane < 3) v = lane == 0 ? (uint32_t)(nw - R[0]) : (lane == 1 ? (uint32_t)(ne - R[1]) : (uint32_t)(np - R[2]));
        uint16_t *o = trail + 2 * REC * (rbase + r);
        if (lane < 3) {
            o[2 * lane] = (uint16_t)(v & 0xffff);
            o[2 * lane + 1] = (uint16_t)(v >> 16);
        }
        const uint32_t s = R[3 + lane];
        o[6 + 2 * lane] = (uint16_t)(s & 0xffff);
        o[7 + 2 * lane] = (uint16_t)(s >> 16);
    }
}

// ------------------------------------------------------------------ decoder

__device__ __forceinline__ uint32_t rd_u32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__device__ __forceinline__ uint32_t rd_w32(const uint16_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 16); }

// largest s in [0, n) with cdf[s] <= slot, between the 256-slot bucket's ends
__device__ __forceinline__ int find_sym(const uint16_t *cdf, int n, uint32_t slot, const uint16_t *lut) {
    const int j = (int)(slot >> 8);
    int lo = lut[j], hi = min((int)lut[j + 1], n - 1);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint32_t)cdf[mid] <= slot) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(DEC_WARPS * 32) rans2_decode_kernel(const StreamGeom g, int B, int part,
                                                                      const DevTables t,
                                                                      const uint8_t *__restrict__ data,
                                                                      const int64_t *__restrict__ offsets,
                                                                      const int64_t *__restrict__ sizes,
                                                                      const uint8_t *__restrict__ idx,
                                                                      const float *__restrict__ med,
                                                                      int32_t *__restrict__ s_out,
                                                                      float *__restrict__ hat_out,
                                                                      uint32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t d_raw[];
    const bool gauss = part == 1 && g.kind == LIC_HYPERPRIOR && t.gauss_base >= 0;
    const bool staged = gauss && t.gimg != nullptr;
    if (staged) stage_image(t, d_raw, RANS2_GIMG_BYTES);
    const int32_t *s_lo = reinterpret_cast<const int32_t *>(d_raw), *s_n = s_lo + NG, *s_cs = s_lo + 2 * NG;
    const uint16_t *gcdf = reinterpret_cast<const uint16_t *>(d_raw + RANS2_GIMG_HDR);
    const uint16_t *glut = reinterpret_cast<const uint16_t *>(d_raw + RANS2_GIMG_CDF_BYTES);
    uint16_t *d_sm = reinterpret_cast<uint16_t *>(d_raw);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // warp -> (frame, substream, segment between resume records)
    const int64_t per_z = g.nr_z + 1;
    const int64_t per_ch = (int64_t)(g.nbands - 1) * (g.nr_full + 1) + (g.nr_last + 1);
    const int64_t nseg = part == 0 ? (int64_t)g.nz * per_z : (int64_t)g.M * per_ch;
    const int64_t warp = (int64_t)blockIdx.x * DEC_WARPS + wib;
    if (warp >= (int64_t)B * nseg) return;
    const int b = (int)(warp / nseg);
    const int64_t j = warp % nseg;
    int q, seg;
    if (part == 0) {
        q = (int)(j / per_z);
        seg = (int)(j % per_z);
    } else {
        const int c = (int)(j / per_ch);
        const int64_t rem = j % per_ch;
        const int64_t bq = rem / (g.nr_full + 1);
        const int band = bq < g.nbands - 1 ? (int)bq : g.nbands - 1;
        seg = (int)(rem - (int64_t)band * (g.nr_full + 1));
        q = g.nz + c * g.nbands + band;
    }
    const Sub si = sub_of(g, q);

    // ---- header and substream bounds (never trust the stream) ----
    // The stream's own record spacing decides how it is decoded: with the
    // spacing this decoder was set up for, one warp per segment from the
    // records; with another (none, or stripped), each substream from its start
    // by its segment-0 warp, the other warps leaving at once.
    const int64_t fsize = sizes[b];
    const uint8_t *frame = data + offsets[b];
    bool bad = (offsets[b] & 1) != 0 || fsize < g.header_bytes;
    int s_stream = 0;
    if (!bad) {
        s_stream = (int)(rd_u32(frame + 28) >> 16);
        bad = rd_u32(frame) != 0x3143494Cu || rd_u32(frame + 4) != (2u | ((uint32_t)g.kind << 16)) ||
              rd_u32(frame + 8) != ((uint32_t)g.N | ((uint32_t)g.M << 16)) || rd_u32(frame + 12) != (uint32_t)g.H ||
              rd_u32(frame + 16) != (uint32_t)g.W || rd_u32(frame + 20) != (uint32_t)g.Hp ||
              rd_u32(frame + 24) != (uint32_t)g.Wp || (rd_u32(frame + 28) & 0xffffu) != (uint32_t)g.R ||
              rd_u32(frame + 32) != (uint32_t)g.nsub;
    }
    const bool use_rec = !bad && g.S > 0 && s_stream == g.S;
    if (!bad && seg > 0 && !use_rec) return;
    int64_t w0 = 0, w1 = 0;
    if (!bad) {
        w0 = rd_u32(frame + 36 + 4 * (int64_t)q);
        w1 = rd_u32(frame + 36 + 4 * (int64_t)(q + 1));
        const int64_t wend = rd_u32(frame + 36 + 4 * (int64_t)g.nsub);
        bad = w1 < w0 + 66 || w1 > wend || w1 - w0 > (1ll << 30) ||
              g.header_bytes + 2 * wend + 4 * REC * recs_per_frame(g, s_stream) != fsize;
    }
    const uint16_t *sw = reinterpret_cast<const uint16_t *>(frame + g.header_bytes) + w0;
    const int64_t L = w1 - w0;
    int64_t nw = 0;
    if (!bad) {
        nw = rd_w32(sw);
        bad = nw < 64 || 2 + nw > L;
    }
    if (bad || (gauss && (!staged || !idx)) || (!gauss && si.table < 0)) {
        if (lane == 0) atomicOr(status, ST_CORRUPT);
        return;
    }
    const uint16_t *rws = sw + 2;                 // rANS section
    const int64_t wa = L - 2 - nw;               // payload + count words
    const int nw32 = (int)nw, wa32 = (int)wa;
    const uint16_t *pws = sw + 2 + nw;           // payload section (forward)
    const uint16_t *cend = sw + L - 1;           // count word j at cend[-j]
    const uint16_t *trail = reinterpret_cast<const uint16_t *>(frame + g.header_bytes) + rd_u32(frame + 36 + 4 * (int64_t)g.nsub);

    // ---- the table(s) of this substream ----
    const uint16_t *cdf_f = nullptr, *lut_f = nullptr;
    int lo_f = 0, n_f = 2;
    if (!gauss) {
        uint16_t *mine = d_sm + (size_t)wib * (FIX_CDF + FIX_LUT);
        lo_f = t.lo[si.table];
        n_f = lo_f + t.hi[si.table] + 2;
        if (n_f > FIX_CDF) {   // not reached: tables hold at most 4096 symbols
            if (lane == 0) atomicOr(status, ST_CORRUPT);
            return;
        }
        const uint32_t *src = t.cdf + t.start[si.table];
        for (int e = lane; e < n_f; e += 32) mine[e] = (uint16_t)src[e];
        for (int e = lane; e < LUT_N; e += 32) mine[FIX_CDF + e] = t.lut[(int64_t)si.table * LUT_N + e];
        __syncwarp();
        cdf_f = mine;
        lut_f = mine + FIX_CDF;
    }

    // ---- start: the stream's initial states, or resume record seg - 1 ----
    const int ngroups = (si.n + 31) / 32;
    const int nr = use_rec ? si.nr : 0;   // records of this substream that this warp follows
    const int g0 = seg * g.S;
    const int g1 = seg < nr ? (seg + 1) * g.S : ngroups;
    uint32_t x;
    int pos, er, qp;   // substreams hold fewer than 2^31 words
    if (seg == 0) {
        x = rd_w32(rws + 2 * lane);
        pos = 64;
        er = 0;
        qp = 0;
    } else {
        const uint16_t *R = trail + 2 * REC * (si.rbase + seg - 1);
        pos = (int)rd_w32(R);
        er = (int)rd_w32(R + 2);
        qp = (int)rd_w32(R + 4);
        x = rd_w32(R + 6 + 2 * lane);
        if (pos < 64 || pos > nw || er < 0 || qp < 0) {
            if (lane == 0) atomicOr(status, ST_CORRUPT);
            return;
        }
    }
    // register windows: rANS words [wb, wb + 96), payload words [pb, pb + 96),
    // count words (from the end) [cb, cb + 64), one word per lane and chunk
    auto ldr = [&](int k) -> uint32_t { return k < nw32 ? rws[k] : 0u; };
    auto ldp = [&](int k) -> uint32_t { return k < wa32 ? pws[k] : 0u; };
    auto ldc = [&](int k) -> uint32_t { return k < wa32 ? cend[-k] : 0u; };
    int wb = pos & ~31, pb = (qp >> 2) & ~31, cb = (er >> 2) & ~31;
    // (the last chunk of each window is the one in flight: shuffles read only the others,
    // and it is waited for when the window moves on)
    uint32_t r0 = ldr(wb + lane), r1 = ldr(wb + 32 + lane), r2 = ldr(wb + 64 + lane);
    uint32_t p0 = ldp(pb + lane), p1 = ldp(pb + 32 + lane), p2 = ldp(pb + 64 + lane), p3 = ldp(pb + 96 + lane);
    uint32_t k0 = ldc(cb + lane), k1 = ldc(cb + 32 + lane);

    const int C = si.is_z ? g.N : g.M;
    const int HW = si.is_z ? g.Hz * g.Wz : g.Hy * g.Wy;
    int32_t *sdst = s_out + ((int64_t)b * C + si.c) * HW + si.p0;
    float *hdst = hat_out ? hat_out + ((int64_t)b * HW + si.p0) * C + si.c : nullptr;
    const float mu = (si.is_z || g.kind == LIC_FACTORIZED) ? med[si.c] : 0.f;
    const int64_t plane = ((int64_t)b * g.M + si.c) * g.Hy * g.Wy;
    const uint8_t *ix = gauss ? idx + plane + si.p0 : nullptr;
    bool corrupt = false;
    // scale indices by blocks of 4 groups: lane l holds symbols 4l .. 4l+3 of a block in
    // one word (the plane and the substream start are 16-byte aligned), the next block
    // loaded a block ahead
    auto ld_blk = [&](int b4) -> uint32_t {
        const int i0 = 128 * b4 + 4 * lane;
        if (!ix) return 0u;
        if (i0 + 3 < si.n) return *reinterpret_cast<const uint32_t *>(ix + i0);
        uint32_t v = 0;
        for (int e = 0; e < 4; ++e)
            if (i0 + e < si.n) v |= (uint32_t)ix[i0 + e] << (8 * e);
        return v;
    };
    uint32_t blk = ld_blk(g0 >> 2), blk_next = ld_blk((g0 >> 2) + 1);
    for (int grp = g0; grp < g1; ++grp) {
        const int i = grp * 32 + lane;
        const bool active = i < si.n;
        if (grp > g0 && (grp & 3) == 0) {
            blk = blk_next;
            blk_next = ld_blk((grp >> 2) + 1);
        }
        const int kk = (int)((__shfl_sync(FULL, blk, 8 * (grp & 3) + (lane >> 2)) >> (8 * (lane & 3))) & 0xffu);
        int lo = lo_f, n = n_f, sym = 0;
        bool need = false;
        if (active) {
            const uint16_t *cdf = cdf_f, *lut = lut_f;
            if (gauss) {
                lo = s_lo[kk];
                n = s_n[kk];
                cdf = gcdf + s_cs[kk];
                lut = glut + kk * LUT_N;
            }
            const uint32_t slot = x & 0xffffu;
            sym = find_sym(cdf, n, slot, lut);
            const uint32_t st = cdf[sym], f = (sym + 1 < n ? (uint32_t)cdf[sym + 1] : 65536u) - st;
            x = f * (x >> 16) + slot - st;
            need = x < RANS_L;
        }
        // renormalisation words: rank among the renormalising lanes
        const unsigned m = __ballot_sync(FULL, need);
        const int p = pos + __popc(m & ((1u << lane) - 1u));
        const int dr = need ? p - wb : 0;   // < 64: the first two chunks
        const uint32_t ra = __shfl_sync(FULL, r0, dr & 31), rb = __shfl_sync(FULL, r1, dr & 31);
        const uint32_t wv = dr < 32 ? ra : rb;
        if (need) {
            if (p < nw32) x = (x << 16) | wv;
            else corrupt = true;
        }
        pos += __popc(m);
        if (pos - wb >= 32) {
            wb += 32;
            r0 = r1;
            r1 = r2;
            r2 = ldr(wb + 64 + lane);
        }
        // escapes: counts from the end, payloads from the front, all at once
        const bool esc = active && sym == n - 1;
        int32_t val = sym - lo;
        const unsigned me = __ballot_sync(FULL, esc);
        if (me) {
            const int rk = __popc(me & ((1u << lane) - 1u));
            const int e = er + rk;
            const int dc = esc ? (e >> 2) - cb : 0;   // < 40
            uint32_t cw = __shfl_sync(FULL, k0, dc & 31);
            if (__any_sync(FULL, dc >= 32)) {
                const uint32_t c1v = __shfl_sync(FULL, k1, dc & 31);
                if (dc >= 32) cw = c1v;
            }
            int nn = esc ? (int)((cw >> (4 * (e & 3))) & 15u) + 1 : 0;
            if (esc && ((e >> 2) >= wa32 || nn > 8)) corrupt = true;
            nn = min(nn, 8);
            int excl, T;
            nibble_prefix(me, nn, esc, lane, excl, T);
            const int qo = qp + excl;
            if (esc && ((qo + nn - 1) >> 2) >= wa32) corrupt = true;
            // an escape's nibbles lie in three consecutive payload words at most
            const int dp = esc ? (qo >> 2) - pb : 0;   // + 2 < 96: the first three chunks
            const bool far = __any_sync(FULL, dp + 2 >= 64);
            uint64_t span = 0;
#pragma unroll
            for (int h = 0; h < 3; ++h) {
                const int d = dp + h;
                const uint32_t a = __shfl_sync(FULL, p0, d & 31), b2 = __shfl_sync(FULL, p1, d & 31);
                uint32_t wd = d < 32 ? a : b2;
                if (far) {
                    const uint32_t c2 = __shfl_sync(FULL, p2, d & 31);
                    if (d >= 64) wd = c2;
                }
                span |= (uint64_t)wd << (16 * h);
            }
            const uint32_t v = (uint32_t)((span >> (4 * (qo & 3))) & ((nn >= 8) ? 0xffffffffull : ((1ull << (4 * nn)) - 1ull)));
            if (esc) {
                const int64_t r = (v & 1u) ? -(int64_t)lo - 1 - (int64_t)(v >> 1)
                                           : (int64_t)(n - 2 - lo) + 1 + (int64_t)(v >> 1);
                if (r > 1073741824LL || r < -1073741824LL) corrupt = true;
                val = (int32_t)r;
            }
            er += __popc(me);
            qp += T;
            while ((qp >> 2) - pb >= 32) {
                pb += 32;
                p0 = p1;
                p1 = p2;
                p2 = p3;
                p3 = ldp(pb + 96 + lane);
            }
            if ((er >> 2) - cb >= 32) {
                cb += 32;
                k0 = k1;
                k1 = ldc(cb + 32 + lane);
            }
        }
        if (active) {
            sdst[i] = val;
            if (hdst) hdst[(int64_t)i * C] = __fadd_rn(__int2float_rn(val), mu);
        }
    }
    // ---- corruption found on the way (every read above is bounded, so decoding on
    // after it is safe), then the segment must end where the next record or the
    // substream says ----
    if (__any_sync(FULL, corrupt)) {
        if (lane == 0) atomicOr(status, ST_CORRUPT);
        return;
    }
    bool ok;
    if (seg < nr) {
        const uint16_t *R = trail + 2 * REC * (si.rbase + seg);
        ok = rd_w32(R) == (uint32_t)pos && rd_w32(R + 2) == (uint32_t)er && rd_w32(R + 4) == (uint32_t)qp &&
             rd_w32(R + 6 + 2 * lane) == x;
    } else {
        ok = pos == nw32 && 2 + nw + (qp + 3) / 4 + (er + 3) / 4 == L;
    }
    if (!__all_sync(FULL, ok) && lane == 0) atomicOr(status, ST_CORRUPT);
}

int64_t blocks_for(int64_t warps, int per) { return (warps + per - 1) / per; }

}  // namespace

bool build_gauss_image(const HostTables &ht, int first, const std::vector<uint16_t> &lut, std::vector<uint8_t> *img) {
    img->assign(RANS2_GIMG_BYTES, 0);
    int32_t *lo = reinterpret_cast<int32_t *>(img->data()), *n = lo + NG, *cs = lo + 2 * NG;
    uint16_t *cdf = reinterpret_cast<uint16_t *>(img->data() + RANS2_GIMG_HDR);
    uint16_t *lt = reinterpret_cast<uint16_t *>(img->data() + RANS2_GIMG_CDF_BYTES);
    if ((int)ht.lo.size() < first + NG || lut.size() < (size_t)(first + NG) * LUT_N) return false;
    int acc = 0;
    for (int k = 0; k < NG; ++k) {
        const int tab = first + k;
        lo[k] = ht.lo[tab];
        n[k] = ht.lo[tab] + ht.hi[tab] + 2;
        cs[k] = acc;
        if (acc + n[k] > RANS2_GAUSS_CDF_CAP) return false;
        for (int e = 0; e < n[k]; ++e) cdf[acc + e] = (uint16_t)ht.cdf[ht.start[tab] + e];   // < 2^16 below entry n
        acc += n[k];
        for (int e = 0; e < LUT_N; ++e) lt[k * LUT_N + e] = lut[(size_t)tab * LUT_N + e];
    }
    return true;
}

namespace {

// dynamic shared memory above the default is opted into once per device
void allow_smem(const void *kernel, size_t bytes, bool *done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    if (!done[dev]) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        done[dev] = true;
    }
}

bool g_enc_smem[64], g_dec_smem[64];

}  // namespace

void launch_rans2_encode(const StreamGeom &g, int B, const DevTables &t, const int32_t *s_y, const uint8_t *idx,
                         const int32_t *s_z, uint16_t *scratch, int64_t *counts, cudaStream_t st) {
    const int64_t warps = 2 * (int64_t)B * g.nsub;
    if (warps == 0) return;
    const bool gauss = g.kind == LIC_HYPERPRIOR && t.gauss_base >= 0 && idx != nullptr;
    const size_t smem = gauss ? ENC_SMEM : 0;
    allow_smem((const void *)rans2_encode_kernel, ENC_SMEM, g_enc_smem);
    rans2_encode_kernel<<<(unsigned)blocks_for(warps, ENC_WARPS), ENC_WARPS * 32, smem, st>>>(g, B, t, s_y, idx, s_z,
                                                                                             scratch, counts);
    const int64_t subs = (int64_t)B * g.nsub;
    rans2_len_kernel<<<(unsigned)((subs + 255) / 256), 256, 0, st>>>(g, B, scratch, counts);
}

void launch_rans2_compact(const StreamGeom &g, int B, const uint16_t *scratch, const int64_t *counts,
                          int64_t *sub_off, int64_t *frame_bytes, int64_t *offsets, uint8_t *data, cudaStream_t st) {
    launch_rans_scan(g, B, counts, sub_off, frame_bytes, 4 * REC * g.rec_per_frame, st);
    launch_frame_place(B, frame_bytes, offsets, st);
    const int64_t warps = (int64_t)B * g.nsub;
    rans2_write_kernel<<<(unsigned)blocks_for(warps, ENC_WARPS), ENC_WARPS * 32, 0, st>>>(g, B, scratch, counts,
                                                                                         sub_off, offsets, data);
}

void launch_rans2_decode(const StreamGeom &g, int B, int part, const DevTables &t, const uint8_t *data,
                         const int64_t *offsets, const int64_t *sizes, const uint8_t *idx, const float *med,
                         int32_t *s_out, float *hat_out, uint32_t *status, cudaStream_t st) {
    const int64_t per = part == 0 ? (int64_t)g.nz * (g.nr_z + 1)
                                  : (int64_t)g.M * ((int64_t)(g.nbands - 1) * (g.nr_full + 1) + g.nr_last + 1);
    const int64_t warps = (int64_t)B * per;
    if (warps == 0) return;
    allow_smem((const void *)rans2_decode_kernel, DEC_SMEM, g_dec_smem);
    rans2_decode_kernel<<<(unsigned)blocks_for(warps, DEC_WARPS), DEC_WARPS * 32, DEC_SMEM, st>>>(
        g, B, part, t, data, offsets, sizes, idx, med, s_out, hat_out, status);
}

}  // namespace lic
