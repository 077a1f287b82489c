// The C ABI (include/lic.h): codec object, weight re-layout, workspace, and
// the encode / decode chains of the factorized-prior [1] and
// scale-hyperprior [2] codecs in the order of the paper's Fig. 1 and
// Sec. III-A/B, all on one CUDA stream.
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/lic_serve.h"
#include "../../include/lic_student.h"
#include "conv_tc.h"
#include "lic_internal.h"

namespace lic {

static thread_local char g_last_error[512];
thread_local int64_t *g_alloc_sink = nullptr;

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

namespace {


// One GEMM launch of a layer: a full convolution, or one sub-pixel phase of
// a transposed convolution.
struct ConvOp {
    DevBuf w;     // [Cout][T][Cin] float32
    tc::TcWeights tcw;  // tensor-core operand copy (built when the op qualifies)
    // g_a conv0's patch GEMM over the padded 4-channel frame (ConvDesc::frame):
    // [Cout][FRAME_K], K index 4 (5u + v) + c (built for Cin = 3, Cout = 128)
    tc::TcWeights tcw4;
    // Cout the tensor-core kernels take only in slices (Cout not 128 or 192,
    // e.g. M = 320): one operand copy per column slice of 192 or 128 channels
    std::vector<std::unique_ptr<tc::TcWeights>> parts;
    std::vector<int> part_off;
    int T = 0;
    int8_t du[MAX_TAPS] = {}, dv[MAX_TAPS] = {};
    int py = 0, px = 0;
};

struct Layer {
    std::string name;
    bool deconv = false;
    int Cin = 0, Cout = 0, k = 0, stride = 1;
    int in_xform = IN_NONE, epi = EPI_NONE;
    DevBuf bias;
    DevBuf w_small;  // transposed conv to <= 4 channels: [Cin][5][5][4]
    // ... and as a 1x1 GEMM from Cin channels to 128 columns: the 25 * Cout tap
    // contributions of an input position (column (u * 5 + v) * Cout + o, zero
    // beyond), summed per output pixel by launch_deconv_gather
    tc::TcWeights w_scatter;
    DevBuf zero_bias;
    int in_dt = DT_F32, out_dt = DT_F32;   // activation storage of this layer (precision forms)
    float in_scale = 1.f, out_scale = 1.f;   // e4m3 tensors hold x / scale
    std::vector<std::unique_ptr<ConvOp>> ops;
    // a 1x1 GEMM over packed patches standing for a k x k conv of def_cin
    // channels: its algorithmic work is that conv's (K = k * k * def_cin), and
    // the input it reads is the frame, whose bytes the packing launch counts
    int def_cin = 0, def_k = 0;
};

struct Gdn {
    std::string name;
    int C = 0;
    bool inverse = false;
    bool diag = false;   // 1DN: per-channel gamma, no channel mixing
    DevBuf gamma;  // [C][1][C]
    DevBuf beta;
    tc::TcWeights tcw;
};

}  // namespace
}  // namespace lic

struct lic_codec {
    int kind = 0, N = 0, M = 0;
    lic_options opt{};
    int device = 0;
    // transforms
    lic::Layer ga[4], gs[4], ha[3], hs[3];
    // g_a conv0 as a GEMM over its 5x5 patches (tensor-core path), A loaded by
    // TMA: tap by tap from the padded 4-channel frame (Cout = 128, the tap
    // form), else from patch rows packed in HBM
    lic::Layer ga0p;
    bool use_patch = false;
    // while analysis runs ga0p on the persistent FP32 kernel: the padded 4-channel
    // frame it builds its A rows from (no patch rows in HBM)
    const float *frame_src = nullptr;
    lic::Gdn gdn[3], igdn[3];
    // entropy models
    lic::HostTables ht;
    lic::DevBuf cdf, start, lo, hi, med, lut, gimg, scales;
    // whether the last analysis / hyper analysis fused Q(y) / Q(z) into their epilogues
    bool q_y_fused = false, q_z_fused = false;
    lic::DevTables dt{};
    lic::DevBuf status;
    // workspace
    lic::DevBuf xin, patches, act0, act1, y, s_y, h1, h2, z, s_z, zhat, g1, g2, sigma, idx, yhat, xpre;
    lic::DevBuf scratch, counts, sub_off, frame_bytes, stage_in, stage_out, in_data, in_offs;
    // encoded batches: containers + offsets/sizes (device and pinned host),
    // handed out by encode, pooled on release (grow-only buffers)
    struct Batch {
        lic::DevBuf data, offs;
        lic::HostPinned h_offs;
        bool live = false;
    };
    std::vector<std::unique_ptr<Batch>> batches;
    // device bytes this codec holds (lic::AllocScope of every entry point)
    int64_t device_bytes = 0;
    // measurement
    lic::Profiler pf;
    // the four sub-pixel phases of a transposed conv write disjoint pixels:
    // phases 1..3 run on these streams, forked from and joined to the caller's
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
    ~lic_codec() {
        for (int i = 0; i < 3; ++i) {
            if (aux[i]) cudaStreamDestroy(aux[i]);
            if (ev_join[i]) cudaEventDestroy(ev_join[i]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
    // learned form: the student that replaces g_s (not owned)
    lic_student *student = nullptr;
    float stu_thr = 0.f;
    int stu_checked = 0, stu_lastB = 0;
    lic::DevBuf xstu, stu_part, stu_psnr, stu_pass, stu_counts;
    // last call (for lic_read_tensor)
    int last_B = 0, last_Hp = 0, last_Wp = 0;
    bool have_y = false, have_sy = false, have_z = false, have_sz = false, have_sigma = false, have_idx = false,
         have_xpre = false, have_yhat = false;
};

namespace lic {
namespace {


void atomic_status(const lic_codec *cd, uint32_t bits) {
    // a launch that could not be made (host side): latch it like a kernel would
    uint32_t cur = 0;
    cudaMemcpy(&cur, cd->status.p, 4, cudaMemcpyDeviceToHost);
    cur |= bits;
    cudaMemcpy(cd->status.p, &cur, 4, cudaMemcpyHostToDevice);
}

// Every kernel launch goes through here: counts it and, when profiling is
// on, brackets it with CUDA events on its stream.
template <typename F>
void timed(lic_codec *cd, const std::string &name, double flop, double bytes, int nlaunch, cudaStream_t st, F &&f) {
    cd->pf.run(name, flop, bytes, nlaunch, st, f);
}

using ParamMap = std::map<std::string, std::pair<const float *, int64_t>>;

int get_param(const ParamMap &pm, const std::string &name, int64_t numel, const float **out) {
    auto it = pm.find(name);
    if (it == pm.end() || it->second.first == nullptr || it->second.second != numel) {
        snprintf(g_last_error, sizeof(g_last_error), "parameter %s missing or of wrong size (want %lld)",
                 name.c_str(), (long long)numel);
        return LIC_E_INVALID_ARG;
    }
    *out = it->second.first;
    return LIC_OK;
}

int upload(DevBuf &b, const void *src, size_t bytes) {
    LIC_CUDA_TRY(b.ensure(bytes));
    LIC_CUDA_TRY(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
    return LIC_OK;
}

// Column slices of a [Cout][T][Cin] weight matrix for the tensor-core
// kernels when Cout is not one of their widths: Cout = 192 a + 128 b.
void build_parts(ConvOp &op, const float *r, int Cout, int Cin) {
    if (Cout == 128 || Cout == 192 || Cout % 64) return;
    for (int a = Cout / 192; a >= 0; --a) {
        if ((Cout - 192 * a) % 128) continue;
        const int64_t K = (int64_t)op.T * Cin;
        int off = 0;
        for (int j = 0; j < a + (Cout - 192 * a) / 128; ++j) {
            const int w = j < a ? 192 : 128;
            auto tw = std::make_unique<tc::TcWeights>();
            tc::build_weights(r + off * K, w, op.T, Cin, tw.get());
            op.parts.push_back(std::move(tw));
            op.part_off.push_back(off);
            off += w;
        }
        return;
    }
}

// conv weight [Cout][Cin][k][k] -> [Cout][k*k][Cin]; taps (u - k/2, v - k/2)
int make_conv(Layer &L, const ParamMap &pm, const std::string &name, int Cin, int Cout, int k, int stride,
              int in_xform, int epi) {
    L.name = name;
    L.deconv = false;
    L.Cin = Cin;
    L.Cout = Cout;
    L.k = k;
    L.stride = stride;
    L.in_xform = in_xform;
    L.epi = epi;
    const float *w, *b;
    int rc = get_param(pm, name + ".weight", (int64_t)Cout * Cin * k * k, &w);
    if (rc) return rc;
    rc = get_param(pm, name + ".bias", Cout, &b);
    if (rc) return rc;
    auto op = std::make_unique<ConvOp>();
    op->T = k * k;
    std::vector<float> r((size_t)Cout * k * k * Cin);
    for (int o = 0; o < Cout; ++o)
        for (int c = 0; c < Cin; ++c)
            for (int u = 0; u < k; ++u)
                for (int v = 0; v < k; ++v)
                    r[((size_t)o * k * k + u * k + v) * Cin + c] = w[(((size_t)o * Cin + c) * k + u) * k + v];
    for (int u = 0; u < k; ++u)
        for (int v = 0; v < k; ++v) {
            op->du[u * k + v] = (int8_t)(u - k / 2);
            op->dv[u * k + v] = (int8_t)(v - k / 2);
        }
    if ((rc = upload(op->w, r.data(), r.size() * sizeof(float)))) return rc;
    tc::build_weights(r.data(), Cout, op->T, Cin, &op->tcw);
    build_parts(*op, r.data(), Cout, Cin);
    L.ops.push_back(std::move(op));
    return upload(L.bias, b, Cout * sizeof(float));
}

// transposed conv weight [Cin][Cout][k][k] (k = 5, stride 2, pad 2, output
// padding 1) -> four sub-pixel phases.  Output row Y = 2m + py receives
// input row a = m + (py + 2 - u) / 2 through tap u whenever u = py (mod 2).
int make_deconv(Layer &L, const ParamMap &pm, const std::string &name, int Cin, int Cout, int epi) {
    const int k = 5;
    L.name = name;
    L.deconv = true;
    L.Cin = Cin;
    L.Cout = Cout;
    L.k = k;
    L.stride = 2;
    L.in_xform = IN_NONE;
    L.epi = epi;
    const float *w, *b;
    int rc = get_param(pm, name + ".weight", (int64_t)Cin * Cout * k * k, &w);
    if (rc) return rc;
    rc = get_param(pm, name + ".bias", Cout, &b);
    if (rc) return rc;
    if (Cout <= 4 && Cin % 32 == 0) {
        std::vector<float> r((size_t)Cin * 25 * 4, 0.f);
        for (int c = 0; c < Cin; ++c)
            for (int o = 0; o < Cout; ++o)
                for (int u = 0; u < k; ++u)
                    for (int v = 0; v < k; ++v)
                        r[(((size_t)c * 25) + u * 5 + v) * 4 + o] = w[(((size_t)c * Cout + o) * k + u) * k + v];
        if ((rc = upload(L.w_small, r.data(), r.size() * sizeof(float)))) return rc;
        // the two-pass form needs 25 * Cout floats of scratch a position, which the
        // codec's activation buffers hold when Cin >= 128; the choice depends on
        // the model only, so every batch size decodes through the same arithmetic
        if (Cin >= 128) {
            // GEMM column of (du, dv, py, px, o): the neighbour-class layout of
            // launch_deconv_gather (lic_internal.h); padding columns stay zero
            std::vector<float> ws((size_t)128 * Cin, 0.f), zb(128, 0.f);
            for (int du = -1; du <= 1; ++du)
                for (int dv = -1; dv <= 1; ++dv)
                    for (int py = 0; py < scatter_n(du); ++py)
                        for (int px = 0; px < scatter_n(dv); ++px)
                            for (int o = 0; o < Cout; ++o) {
                                const int u = py + 2 - 2 * du, v = px + 2 - 2 * dv;
                                const size_t col = (size_t)scatter_offset(du, dv, Cout) +
                                                   (size_t)(py * scatter_n(dv) + px) * Cout + o;
                                for (int c = 0; c < Cin; ++c)
                                    ws[col * Cin + c] = w[(((size_t)c * Cout + o) * k + u) * k + v];
                            }
            tc::build_weights(ws.data(), 128, 1, Cin, &L.w_scatter);
            if ((rc = upload(L.zero_bias, zb.data(), zb.size() * sizeof(float)))) return rc;
        }
    }
    for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px) {
            auto op = std::make_unique<ConvOp>();
            op->py = py;
            op->px = px;
            std::vector<int> us, vs;
            for (int u = py; u < k; u += 2) us.push_back(u);
            for (int v = px; v < k; v += 2) vs.push_back(v);
            op->T = (int)(us.size() * vs.size());
            std::vector<float> r((size_t)Cout * op->T * Cin);
            int t = 0;
            for (int u : us)
                for (int v : vs) {
                    op->du[t] = (int8_t)((py + 2 - u) / 2);
                    op->dv[t] = (int8_t)((px + 2 - v) / 2);
                    for (int o = 0; o < Cout; ++o)
                        for (int c = 0; c < Cin; ++c)
                            r[((size_t)o * op->T + t) * Cin + c] = w[(((size_t)c * Cout + o) * k + u) * k + v];
                    ++t;
                }
            if ((rc = upload(op->w, r.data(), r.size() * sizeof(float)))) return rc;
            tc::build_weights(r.data(), Cout, op->T, Cin, &op->tcw);
            build_parts(*op, r.data(), Cout, Cin);
            L.ops.push_back(std::move(op));
        }
    return upload(L.bias, b, Cout * sizeof(float));
}

// g_a conv0 (Cin * 25 <= PATCH_K) as a 1x1 convolution over its packed
// patches: weights [Cout][PATCH_K], the conv's [Cout][25][Cin] order
// flattened and zero-padded, the same K order the gathering kernel uses, so
// results are unchanged
int make_patch_layer(Layer &P, const Layer &L, const ParamMap &pm) {
    const int Cout = L.Cout, Cin = L.Cin, k = L.k;
    if (L.deconv || Cin * k * k > PATCH_K || L.stride != 2 || k != 5) return LIC_E_UNSUPPORTED;
    const float *w, *b;
    int rc = get_param(pm, L.name + ".weight", (int64_t)Cout * Cin * k * k, &w);
    if (rc) return rc;
    if ((rc = get_param(pm, L.name + ".bias", Cout, &b))) return rc;
    P.name = L.name;
    P.deconv = false;
    P.Cin = PATCH_K;
    P.Cout = Cout;
    P.k = 1;
    P.stride = 1;
    P.in_xform = IN_NONE;
    P.epi = L.epi;
    P.in_dt = DT_F32;
    P.out_dt = L.out_dt;
    P.in_scale = 1.f;
    P.out_scale = L.out_scale;
    P.def_cin = Cin;
    P.def_k = k;
    auto op = std::make_unique<ConvOp>();
    op->T = 1;
    std::vector<float> r((size_t)Cout * PATCH_K, 0.f);
    for (int o = 0; o < Cout; ++o)
        for (int u = 0; u < k; ++u)
            for (int v = 0; v < k; ++v)
                for (int c = 0; c < Cin; ++c)
                    r[(size_t)o * PATCH_K + (u * k + v) * Cin + c] = w[(((size_t)o * Cin + c) * k + u) * k + v];
    if ((rc = upload(op->w, r.data(), r.size() * sizeof(float)))) return rc;
    tc::build_weights(r.data(), Cout, 1, PATCH_K, &op->tcw);
    if (!op->tcw.valid) return LIC_E_UNSUPPORTED;
    if (Cin == 3 && Cout == 128) {   // the same weights for the padded 4-channel frame (K = 4 t + c)
        std::vector<float> r4((size_t)Cout * FRAME_K, 0.f);
        for (int o = 0; o < Cout; ++o)
            for (int u = 0; u < k; ++u)
                for (int v = 0; v < k; ++v)
                    for (int c = 0; c < Cin; ++c)
                        r4[(size_t)o * FRAME_K + 4 * (u * k + v) + c] = w[(((size_t)o * Cin + c) * k + u) * k + v];
        tc::build_weights(r4.data(), Cout, 1, FRAME_K, &op->tcw4);
    }
    P.ops.clear();
    P.ops.push_back(std::move(op));
    return upload(P.bias, b, Cout * sizeof(float));
}

int make_gdn(Gdn &G, const ParamMap &pm, const std::string &name, int C, bool inverse, bool diag) {
    G.name = name;
    G.C = C;
    G.inverse = inverse;
    G.diag = diag;
    const float *beta, *gamma;
    int rc = get_param(pm, name + ".beta", C, &beta);
    if (rc) return rc;
    const int64_t ng = diag ? C : (int64_t)C * C;
    rc = get_param(pm, name + ".gamma", ng, &gamma);
    if (rc) return rc;
    if ((rc = upload(G.gamma, gamma, (size_t)ng * sizeof(float)))) return rc;
    if (!diag) tc::build_weights(gamma, C, 1, C, &G.tcw);
    return upload(G.beta, beta, C * sizeof(float));
}

// ---------------------------------------------------------------------------
// running layers
// ---------------------------------------------------------------------------

ConvDesc op_desc(const lic_codec *cd, const Layer &L, const ConvOp &op, const float *in, int B, int Hi, int Wi,
                 float *out, int Ho, int Wo) {
    ConvDesc d{};
    d.in = in;
    d.out = out;
    d.w = op.w.as<float>();
    d.bias = L.bias.as<float>();
    d.gdn_x = nullptr;
    d.status = cd->status.as<uint32_t>();
    d.B = B;
    d.Hi = Hi;
    d.Wi = Wi;
    d.Cin = L.Cin;
    d.Ho = Ho;
    d.Wo = Wo;
    d.Cout = L.Cout;
    d.T = op.T;
    for (int t = 0; t < op.T; ++t) {
        d.du[t] = op.du[t];
        d.dv[t] = op.dv[t];
    }
    d.in_xform = L.in_xform;
    d.epi = L.epi;
    d.in_dt = L.in_dt;
    d.out_dt = L.out_dt;
    d.in_scale = L.in_scale;
    d.out_scale = L.out_scale;
    if (L.deconv) {
        d.Gh = Hi;
        d.Gw = Wi;
        d.s = 1;
        d.oym = 2;
        d.oyo = op.py;
        d.oxm = 2;
        d.oxo = op.px;
    } else {
        d.Gh = Ho;
        d.Gw = Wo;
        d.s = L.stride;
        d.oym = 1;
        d.oyo = 0;
        d.oxm = 1;
        d.oxo = 0;
    }
    if (L.def_cin > 0 && cd->frame_src) {
        d.frame = cd->frame_src;
        d.Cin = FRAME_K;
    }
    return d;
}

// One GEMM launch of a layer; with G, the GDN / IGDN that follows the layer
// runs in the same launch (the caller has checked that it can).
// Split-K scratch a layer's launches may use: B * frame_floats floats at p,
// frame_floats fixed by the frame size (never by the buffer's capacity)
struct SplitScratch {
    float *p = nullptr;
    int64_t frame_floats = 0;
};

// Quantisation a layer's epilogue is asked to fuse (ConvDesc q_*), and
// whether every launch of the layer did (else the caller runs the separate
// kernel).
struct QFuse {
    int mode = 0;
    int32_t *sym = nullptr;
    float *hat = nullptr;
    const float *mu = nullptr;
    uint8_t *idx = nullptr;
    const float *tab = nullptr;
    int C = 0;
    bool done = false;
};

void run_op(const lic_codec *cd, const Layer &L, const ConvOp &op, const float *in, int B, int Hi, int Wi,
            float *out, int Ho, int Wo, cudaStream_t st, const Gdn *G = nullptr, int out_dt = -1,
            SplitScratch sk = {}, QFuse *qf = nullptr) {
    ConvDesc d = op_desc(cd, L, op, in, B, Hi, Wi, out, Ho, Wo);
    d.part = sk.p;
    d.part_frame_floats = sk.p ? sk.frame_floats : 0;
    bool q_ok = false;   // set where a launch applies the fused quantisation
    if (qf && qf->mode && !G) {
        d.q_mode = qf->mode;
        d.q_sym = qf->sym;
        d.q_hat = qf->hat;
        d.q_mu = qf->mu;
        d.q_idx = qf->idx;
        d.q_tab = qf->tab;
        d.q_C = qf->C;
    }
    if (out_dt >= 0) {   // the caller wants this storage instead of the layer's own
        d.out_dt = out_dt;
        d.out_scale = 1.f;
    }
    // algorithmic work of the definition: 2 x multiply-adds; bytes = the
    // input read once (a transposed conv's phases share it), the output
    // written once, the weights, at the storage size of each
    const double rows = (double)B * d.Gh * d.Gw;
    const double esz_in = d.in_dt == DT_F32 ? 4.0 : (d.in_dt == DT_BF16 ? 2.0 : 1.0);
    const int odt = out_dt >= 0 ? out_dt : d.out_dt;
    const double esz_out = odt == DT_F32 ? 4.0 : (odt == DT_BF16 ? 2.0 : 1.0);
    double kdef = (double)d.T * d.Cin;
    double in_bytes = esz_in * B * Hi * Wi * d.Cin / (L.deconv ? (double)L.ops.size() : 1.0);
    if (L.def_cin > 0) {   // patch GEMM: the k x k conv it stands for; the frame read is the packing's
        kdef = (double)L.def_k * L.def_k * L.def_cin;
        in_bytes = 0.0;
    }
    double flop = 2.0 * rows * d.Cout * kdef;
    const double bytes = in_bytes + esz_out * rows * d.Cout + esz_in * d.Cout * kdef;
    std::string nm = L.name + (L.deconv ? ".p" + std::to_string(2 * op.py + op.px) : std::string());
    if (G) {
        d.fuse_gdn = G->diag ? (G->inverse ? 4 : 3) : (G->inverse ? 2 : 1);
        d.gdn_beta = G->beta.as<float>();
        d.gdn_w = &G->tcw;
        d.gdn_gamma = G->gamma.as<float>();
        flop += G->diag ? 4.0 * rows * G->C : 2.0 * rows * G->C * G->C;
        nm += "+" + G->name.substr(G->name.find('.') + 1);
    }
    if (!op.parts.empty() && !G) {
        // column slices on the tensor cores, each writing its channels of the full-width output
        std::vector<ConvDesc> ds;
        bool ok = cd->opt.conv_impl != LIC_CONV_SIMT || d.in_dt != DT_F32;
        for (size_t j = 0; j < op.parts.size() && ok; ++j) {
            ConvDesc dp = d;
            dp.part = nullptr;
            dp.Cout = op.parts[j]->Cout;
            dp.out_coff = op.part_off[j];
            dp.out_stride = d.Cout;
            dp.bias = d.bias + op.part_off[j];
            ok = d.in_dt != DT_F32 ? tc::can_run_lp(dp, *op.parts[j]) : tc::can_run(dp, *op.parts[j]);
            ds.push_back(dp);
        }
        if (ok) {
            nm += d.in_dt == DT_F32 ? ":tc" : (d.in_dt == DT_E4M3 ? ":e4m3" : ":bf16");
            bool all = true;
            timed(const_cast<lic_codec *>(cd), nm, flop, bytes, (int)ds.size(), st, [&] {
                for (size_t j = 0; j < ds.size(); ++j) {
                    const bool done = d.in_dt != DT_F32 ? tc::launch_lp(ds[j], *op.parts[j], st)
                                                        : tc::launch(ds[j], *op.parts[j], st);
                    if (!done) atomic_status(cd, ST_TIMEOUT);
                    all = all && done;
                }
            });
            bool fq = d.in_dt == DT_F32 && d.q_mode;
            for (const ConvDesc &dp : ds) fq = fq && tc::tc_fuses_quant(dp);
            if (qf) qf->done = qf->mode && fq && all;
            return;
        }
    }
    if (d.in_dt != DT_F32) {   // precision forms: checked at codec creation
        nm += d.in_dt == DT_E4M3 ? ":e4m3" : ":bf16";
        timed(const_cast<lic_codec *>(cd), nm, flop, bytes, 1, st, [&] {
            if (!tc::launch_lp(d, op.tcw, st)) atomic_status(cd, ST_TIMEOUT);
        });
        if (qf) qf->done = false;   // the low-precision kernels leave quantisation to the caller
        return;
    }
    const tc::TcWeights &tw = d.frame ? op.tcw4 : op.tcw;
    const bool use_tc = cd->opt.conv_impl != LIC_CONV_SIMT && tc::can_run(d, tw);
    if (use_tc && !tc::tc_fuses_quant(d)) d.q_mode = 0;
    if (use_tc && d.q_mode) nm += d.q_mode == 1 ? "+q" : "+index";
    nm += use_tc ? ":tc" : ":simt";
    const int nl = use_tc && tc::split_k(d, tw) > 1 ? 2 : 1;   // split K: + the sum of the slices
    timed(const_cast<lic_codec *>(cd), nm, flop, bytes, nl, st, [&] {
        q_ok = use_tc && tc::launch(d, tw, st);
        if (!q_ok && d.frame) atomic_status(cd, ST_TIMEOUT);   // not reached: analysis checked the form
        else if (!q_ok) launch_conv_simt(d, st);
    });
    if (qf) qf->done = qf->mode && d.q_mode && q_ok && d.out_dt == DT_F32;
}

// Every GEMM launch of a layer.  The phases of a transposed conv are
// independent (disjoint output pixels, shared input): phase k > 0 runs on
// auxiliary stream k - 1, so the small launches of h_s and of the first
// g_s layers fill the GPU together instead of one after another.
void run_ops(const lic_codec *cd, const Layer &L, const float *in, int B, int Hi, int Wi, float *out, int Ho, int Wo,
             cudaStream_t st, const Gdn *G, int out_dt = -1, SplitScratch sk = {}, QFuse *qf = nullptr) {
    const int n = (int)L.ops.size();
    // while launches are being timed one by one (lic_profile_enable) the phases run in
    // sequence, so that each launch's event pair brackets that launch alone
    const bool fork = n > 1 && n <= 4 && cd->ev_fork && cd->aux[n - 2] && !cd->pf.on;
    if (fork) {
        cudaEventRecord(cd->ev_fork, st);
        for (int k = 1; k < n; ++k) cudaStreamWaitEvent(cd->aux[k - 1], cd->ev_fork, 0);
    }
    // split K only for a single launch: the phases of a transposed conv already
    // fill the GPU together (slicing them measured slower)
    // fused quantisation only for a layer of one launch (a convolution, not the phases
    // of a transposed one)
    if (qf) qf->done = false;
    for (int k = 0; k < n; ++k)
        run_op(cd, L, *L.ops[k], in, B, Hi, Wi, out, Ho, Wo, (fork && k > 0) ? cd->aux[k - 1] : st, G, out_dt,
               n == 1 ? sk : SplitScratch{}, n == 1 ? qf : nullptr);
    if (fork) {
        for (int k = 1; k < n; ++k) {
            cudaEventRecord(cd->ev_join[k - 1], cd->aux[k - 1]);
            cudaStreamWaitEvent(st, cd->ev_join[k - 1], 0);
        }
    }
}

void run_layer(const lic_codec *cd, const Layer &L, const float *in, int B, int Hi, int Wi, float *out,
               cudaStream_t st, int out_dt = -1, const DevBuf *scratch = nullptr, SplitScratch sk = {},
               QFuse *qf = nullptr) {
    if (qf) qf->done = false;
    int Ho, Wo;
    if (L.deconv) {
        Ho = 2 * Hi;
        Wo = 2 * Wi;
    } else {
        int p = L.k / 2;
        Ho = (Hi + 2 * p - L.k) / L.stride + 1;
        Wo = (Wi + 2 * p - L.k) / L.stride + 1;
    }
    if (L.deconv && L.w_small.p) {
        const double flop = 2.0 * B * Ho * Wo * L.Cout * L.Cin * 6.25;
        const double bytes = 4.0 * ((double)B * Hi * Wi * L.Cin + (double)B * Ho * Wo * L.Cout + 25.0 * L.Cout * L.Cin);
        // two passes (the layer's tensor-core weights exist when Cin >= 128): the tap
        // contributions of every input position by a tensor-core 1x1 GEMM (128 columns,
        // the leading 25 * Cout stored) into the scratch buffer (an activation buffer
        // of Cin >= 128 channels), then their per-pixel sums
        const int cs = deconv_scatter_stride(L.Cout);
        const size_t need = (size_t)B * Hi * Wi * cs * sizeof(float);
        // the precision forms hand this layer bf16 activations: the tap GEMM then runs on the
        // bf16 kernel (bf16 x bf16 -> float32 contributions), the gather as in FP32
        const bool lp = L.in_dt == DT_BF16;
        if (scratch && L.w_scatter.valid && cd->opt.conv_impl != LIC_CONV_SIMT &&
            (L.in_dt == DT_F32 || (lp && L.w_scatter.bvalid))) {
            if (!scratch->p || scratch->bytes < need) {   // not reached: the buffers hold Cin >= 128 channels
                atomic_status(cd, ST_TIMEOUT);
                return;
            }
            float *cbuf = scratch->as<float>();
            ConvDesc d{};
            d.in = in;
            d.out = cbuf;
            d.bias = L.zero_bias.as<float>();
            d.status = cd->status.as<uint32_t>();
            d.B = B;
            d.Hi = d.Gh = d.Ho = Hi;
            d.Wi = d.Gw = d.Wo = Wi;
            d.Cin = L.Cin;
            d.Cout = 128;
            d.T = 1;
            d.s = 1;
            d.oym = d.oxm = 1;
            d.in_xform = IN_NONE;
            d.epi = EPI_NONE;
            d.in_dt = lp ? DT_BF16 : DT_F32;
            d.out_dt = DT_F32;
            d.in_scale = d.out_scale = 1.f;
            d.out_stream = 1;
            d.out_stride = cs;
            if (lp ? tc::can_run_lp(d, L.w_scatter) : tc::can_run(d, L.w_scatter)) {
                const double rows = (double)B * Hi * Wi;
                const double esz = lp ? 2.0 : 4.0;
                // algorithmic bytes: the input and weights for the GEMM, the output for
                // the gather (the tap contributions in between are this build's staging)
                timed(const_cast<lic_codec *>(cd), L.name + (lp ? ":bf16" : ":tc"), flop,
                      esz * (rows * L.Cin + 25.0 * L.Cout * L.Cin), 1, st, [&] {
                          const bool done = lp ? tc::launch_lp(d, L.w_scatter, st) : tc::launch(d, L.w_scatter, st);
                          if (!done) atomic_status(cd, ST_TIMEOUT);
                      });
                timed(const_cast<lic_codec *>(cd), L.name + ".gather", 0.0, 4.0 * (double)B * Ho * Wo * L.Cout, 1, st,
                      [&] { launch_deconv_gather(cbuf, B, Hi, Wi, L.Cout, L.bias.as<float>(), out, st); });
                return;
            }
        }
        if (L.in_dt != DT_F32) {   // not reached: a bf16 input is set only where the two-pass form runs
            atomic_status(cd, ST_TIMEOUT);
            return;
        }
        timed(const_cast<lic_codec *>(cd), L.name + ":small", flop, bytes, 1, st, [&] {
            launch_deconv_small(in, B, Hi, Wi, L.Cin, L.w_small.as<float>(), L.bias.as<float>(), L.Cout, out, st);
        });
        return;
    }
    run_ops(cd, L, in, B, Hi, Wi, out, Ho, Wo, st, nullptr, out_dt, sk, qf);
}

void run_gdn(const lic_codec *cd, const Gdn &G, const float *in, int B, int H, int W, float *out, cudaStream_t st) {
    if (G.diag) {
        const int64_t P = (int64_t)B * H * W;
        timed(const_cast<lic_codec *>(cd), G.name + ":1dn", 4.0 * P * G.C, 8.0 * P * G.C, 1, st, [&] {
            launch_norm1d(in, P, G.C, G.beta.as<float>(), G.gamma.as<float>(), G.inverse ? 1 : 0, out, st);
        });
        return;
    }
    ConvDesc d{};
    d.in = in;
    d.out = out;
    d.w = G.gamma.as<float>();
    d.bias = G.beta.as<float>();
    d.gdn_x = in;
    d.status = cd->status.as<uint32_t>();
    d.B = B;
    d.Hi = H;
    d.Wi = W;
    d.Cin = G.C;
    d.Gh = H;
    d.Gw = W;
    d.s = 1;
    d.Ho = H;
    d.Wo = W;
    d.Cout = G.C;
    d.oym = 1;
    d.oxm = 1;
    d.T = 1;
    d.in_xform = IN_SQUARE;
    d.epi = G.inverse ? EPI_IGDN : EPI_GDN;
    const double rows = (double)B * H * W;
    const bool use_tc = cd->opt.conv_impl != LIC_CONV_SIMT && tc::can_run(d, G.tcw);
    timed(const_cast<lic_codec *>(cd), G.name + (use_tc ? ":tc" : ":simt"), 2.0 * rows * G.C * G.C,
          4.0 * (2.0 * rows * G.C + (double)G.C * G.C), 1, st, [&] {
              if (!use_tc || !tc::launch(d, G.tcw, st)) launch_conv_simt(d, st);
          });
}

int out_size(const Layer &L, int Hi, int Wi, int *Ho, int *Wo) {
    if (L.deconv) {
        *Ho = 2 * Hi;
        *Wo = 2 * Wi;
    } else {
        const int p = L.k / 2;
        *Ho = (Hi + 2 * p - L.k) / L.stride + 1;
        *Wo = (Wi + 2 * p - L.k) / L.stride + 1;
    }
    return 0;
}

// A layer followed by GDN / IGDN, ping-ponging between buffers a and b;
// returns the buffer holding the result.  One fused tensor-core launch per
// GEMM (writing the buffer that is not the input) when every launch of the
// layer qualifies; else the layer into that buffer and a separate
// normalisation into the other one (which may be the consumed input).
float *run_layer_gdn(const lic_codec *cd, const Layer &L, const Gdn &G, const float *in, int B, int Hi, int Wi,
                     float *a, float *b, cudaStream_t st) {
    float *other = (in == a) ? b : a;
    float *out = other;
    int Ho, Wo;
    out_size(L, Hi, Wi, &Ho, &Wo);
    bool fuse = cd->opt.conv_impl != LIC_CONV_SIMT && !L.w_small.p && !L.ops.empty();
    for (auto &op : L.ops) {
        if (!fuse) break;
        ConvDesc d = op_desc(cd, L, *op, in, B, Hi, Wi, out, Ho, Wo);
        d.fuse_gdn = G.diag ? (G.inverse ? 4 : 3) : (G.inverse ? 2 : 1);
        d.gdn_beta = G.beta.as<float>();
        d.gdn_w = &G.tcw;
        d.gdn_gamma = G.gamma.as<float>();
        fuse = d.in_dt != DT_F32 ? tc::can_run_lp(d, op->tcw) : tc::can_run(d, d.frame ? op->tcw4 : op->tcw);
    }
    if (fuse) {
        run_ops(cd, L, in, B, Hi, Wi, out, Ho, Wo, st, &G);
        return out;
    }
    float *norm_out = (other == a) ? b : a;
    if (L.out_dt != DT_F32) {
        // precision form with a norm the low-precision kernel cannot fuse (Cout 192): the
        // convolution in float32, the norm in float32, then the next layer's storage
        run_layer(cd, L, in, B, Hi, Wi, other, st, DT_F32);
        run_gdn(cd, G, other, B, Ho, Wo, norm_out, st);
        const int64_t n = (int64_t)B * Ho * Wo * L.Cout;
        timed(const_cast<lic_codec *>(cd), G.name + ":to_bf16", 0, 6.0 * n, 1, st,
              [&] { launch_to_bf16(norm_out, n, other, st); });
        return other;
    }
    run_layer(cd, L, in, B, Hi, Wi, other, st);
    run_gdn(cd, G, other, B, Ho, Wo, norm_out, st);
    return norm_out;
}

int pad64(int v) { return (v + 63) / 64 * 64; }

// g_a conv0 runs in the tap form (the padded 4-channel frame, each tap TMA-loaded)
// when its weights were built for it (Cin = 3, Cout = 128, tensor-core path)
bool frame_form(const lic_codec *cd) {
    return cd->use_patch && !cd->ga0p.ops.empty() && cd->ga0p.ops[0]->tcw4.valid;
}

// The grow-only workspace of a batch of B frames padded to Hp x Wp, as a
// list of (buffer, bytes) handed to need(): ensure_workspace allocates it,
// lic_codec_workspace_bytes adds it up without allocating.
template <typename F>
int workspace_plan(lic_codec *cd, int B, int Hp, int Wp, F &&need) {
    const int N = cd->N, M = cd->M;
    const int64_t Hy = Hp / 16, Wy = Wp / 16, Hz = Hp / 64, Wz = Wp / 64;
    const int64_t big = (int64_t)B * (Hp / 2) * (Wp / 2) * N;
    int rc = 0;
    auto f = [&](DevBuf &b, int64_t n, int64_t elem) {
        if (!rc) rc = need(b, n * elem + 256);
    };
    if (!cd->use_patch) f(cd->xin, (int64_t)B * Hp * Wp * 3, 4);   // else unused
    // the patch rows, or (the tap form of g_a conv0) the frame padded to 4 channels
    if (cd->use_patch && frame_form(cd)) f(cd->patches, (int64_t)B * Hp * Wp * 4, 4);
    else if (cd->use_patch) f(cd->patches, (int64_t)B * (Hp / 2) * (Wp / 2) * PATCH_K, 4);
    f(cd->act0, big, 4);
    f(cd->act1, big, 4);
    f(cd->y, (int64_t)B * Hy * Wy * M, 4);
    f(cd->s_y, (int64_t)B * Hy * Wy * M, 4);
    f(cd->yhat, (int64_t)B * Hy * Wy * M, 4);
    f(cd->xpre, (int64_t)B * Hp * Wp * 3, 4);
    if (cd->kind == LIC_HYPERPRIOR) {
        f(cd->h1, (int64_t)B * Hy * Wy * N, 4);
        f(cd->h2, (int64_t)B * (Hy / 2) * (Wy / 2) * N, 4);
        f(cd->z, (int64_t)B * Hz * Wz * N, 4);
        f(cd->s_z, (int64_t)B * Hz * Wz * N, 4);
        f(cd->zhat, (int64_t)B * Hz * Wz * N, 4);
        f(cd->g1, (int64_t)B * (Hy / 2) * (Wy / 2) * N, 4);
        f(cd->g2, (int64_t)B * Hy * Wy * N, 4);
        f(cd->sigma, (int64_t)B * Hy * Wy * M, 4);
        f(cd->idx, (int64_t)B * Hy * Wy * M, 1);
    }
    return rc;
}

// Working memory of the entropy encoder, then the batch's own buffers
// (bb: the pooled batch being filled; its data holds worst-case containers).
template <typename F>
int entropy_plan(lic_codec *cd, const StreamGeom &g, int B, lic_codec::Batch *bb, F &&need) {
    const int64_t subs = (int64_t)B * g.nsub;
    int rc = 0;
    auto f = [&](DevBuf &b, int64_t n, int64_t elem) {
        if (!rc) rc = need(b, n * elem + 256);
    };
    f(cd->scratch, subs * g.cap_words, 2);
    f(cd->counts, subs, 8);
    f(cd->sub_off, subs, 8);
    f(cd->frame_bytes, B, 8);
    f(bb->offs, 2 * (int64_t)B + 1, 8);
    f(bb->data, (int64_t)B * g.frame_cap, 1);
    return rc;
}

int ensure_buf(DevBuf &b, int64_t n) {
    LIC_CUDA_TRY(b.ensure((size_t)n));
    return LIC_OK;
}

int ensure_workspace(lic_codec *cd, int B, int Hp, int Wp) {
    return workspace_plan(cd, B, Hp, Wp, ensure_buf);
}

// At most this many encoded batches may be unreleased at once per codec.
constexpr int kMaxLiveBatches = 64;

// A free pooled batch sized for B frames of geometry g (not yet marked
// live), or null with *rc set.
lic_codec::Batch *acquire_batch(lic_codec *cd, const StreamGeom &g, int B, int *rc) {
    lic_codec::Batch *bb = nullptr;
    int live = 0;
    for (auto &p : cd->batches) {
        if (p->live) ++live;
        else if (!bb) bb = p.get();
    }
    if (!bb) {
        if (live >= kMaxLiveBatches) {
            *rc = LIC_E_BUSY;
            return nullptr;
        }
        cd->batches.push_back(std::make_unique<lic_codec::Batch>());
        bb = cd->batches.back().get();
    }
    if ((*rc = entropy_plan(cd, g, B, bb, ensure_buf))) return nullptr;
    if (bb->h_offs.ensure((2 * (size_t)B + 1) * sizeof(int64_t)) != cudaSuccess) {
        *rc = LIC_E_OOM;
        return nullptr;
    }
    return bb;
}

cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

// ---- the transforms ----

// g_a: frames (device [B][3][Hf][Wf], replicate-padded to Hp x Wp) -> y (NHWC);
// 4 x conv5x5/2 with GDN after the first three
void analysis(lic_codec *cd, const float *frames, int B, int Hf, int Wf, int Hp, int Wp, cudaStream_t st) {
    float *a = cd->act0.as<float>(), *b = cd->act1.as<float>();
    int H = Hp, W = Wp;
    const float *in = cd->xin.as<float>();
    int first = 0;
    if (cd->use_patch && frame_form(cd)) {
        // the frame padded once with 4 channels (into the patch buffer); the persistent FP32
        // kernel loads each tap of the patch rows by TMA
        // algorithmic bytes: the frame read once
        float *f4 = cd->patches.as<float>();
        timed(cd, "frame_pad4", 0, 12.0 * B * Hf * Wf, 1, st,
              [&] { launch_frame_pad4(frames, B, Hf, Wf, Hp, Wp, f4, st); });
        cd->frame_src = f4;
        in = run_layer_gdn(cd, cd->ga0p, cd->gdn[0], f4, B, Hp / 2, Wp / 2, a, b, st);
        cd->frame_src = nullptr;
        H /= 2;
        W /= 2;
        first = 1;
    } else if (cd->use_patch) {
        // the first layer's patches straight from the frames (no padded copy)
        // algorithmic bytes: the frame read once (the patch rows are this build's staging)
        timed(cd, "patch_pack", 0, 12.0 * B * Hf * Wf, 1, st,
              [&] { launch_frame_patch(frames, B, Hf, Wf, Hp, Wp, cd->patches.as<float>(), st); });
        in = run_layer_gdn(cd, cd->ga0p, cd->gdn[0], cd->patches.as<float>(), B, Hp / 2, Wp / 2, a, b, st);
        H /= 2;
        W /= 2;
        first = 1;
    } else {
        timed(cd, "pad_pack", 0, 12.0 * B * ((double)Hf * Wf + (double)Hp * Wp), 1, st,
              [&] { launch_pad_pack(frames, B, Hf, Wf, Hp, Wp, cd->xin.as<float>(), st); });
    }
    for (int i = first; i < 3; ++i) {
        in = run_layer_gdn(cd, cd->ga[i], cd->gdn[i], in, B, H, W, a, b, st);
        H /= 2;
        W /= 2;
    }
    // y, and Q(y) in the same epilogue: s = rint(y) (hyperprior) or rint(fl32(y - median))
    QFuse q;
    q.mode = 1;
    q.sym = cd->s_y.as<int32_t>();
    q.mu = cd->kind == LIC_FACTORIZED ? cd->med.as<float>() : nullptr;
    q.C = cd->M;
    run_layer(cd, cd->ga[3], in, B, H, W, cd->y.as<float>(), st, -1, nullptr, {}, &q);
    cd->q_y_fused = q.done;
}

// Split-K scratch of the hyper transforms: act0, free while they run, holds
// (Hp / 2) (Wp / 2) N floats a frame for frames of Hp x Wp = 16 Hy x 16 Wy
SplitScratch hyper_scratch(lic_codec *cd, int B, int Hy, int Wy) {
    SplitScratch sk;
    sk.frame_floats = 64LL * Hy * Wy * cd->N;
    if (cd->act0.p && cd->act0.bytes >= (size_t)B * sk.frame_floats * sizeof(float)) sk.p = cd->act0.as<float>();
    else atomic_status(cd, ST_TIMEOUT);   // not reached: ensure_workspace sized act0 for these frames
    return sk;
}

// h_a: y -> z; conv3x3/1 on |y| + ReLU, conv5x5/2 + ReLU, conv5x5/2
// (with Q(z) and z_hat in the last layer's epilogue: s_z = rint(fl32(z - median)),
// z_hat = fl32(s_z + median); the caller quantises where the epilogue could not)
void hyper_analysis(lic_codec *cd, const float *y, int B, int Hy, int Wy, cudaStream_t st) {
    const SplitScratch sk = hyper_scratch(cd, B, Hy, Wy);
    run_layer(cd, cd->ha[0], y, B, Hy, Wy, cd->h1.as<float>(), st, -1, nullptr, sk);
    run_layer(cd, cd->ha[1], cd->h1.as<float>(), B, Hy, Wy, cd->h2.as<float>(), st, -1, nullptr, sk);
    QFuse q;
    q.mode = 1;
    q.sym = cd->s_z.as<int32_t>();
    q.hat = cd->zhat.as<float>();
    q.mu = cd->med.as<float>();
    q.C = cd->N;
    run_layer(cd, cd->ha[2], cd->h2.as<float>(), B, Hy / 2, Wy / 2, cd->z.as<float>(), st, -1, nullptr, sk, &q);
    cd->q_z_fused = q.done;
}

// h_s: z_hat -> sigma; deconv+ReLU, deconv+ReLU, conv3x3+ReLU; then the index
void hyper_synthesis(lic_codec *cd, const float *zhat, int B, int Hz, int Wz, cudaStream_t st) {
    const SplitScratch sk = hyper_scratch(cd, B, 4 * Hz, 4 * Wz);
    run_layer(cd, cd->hs[0], zhat, B, Hz, Wz, cd->g1.as<float>(), st, -1, nullptr, sk);
    run_layer(cd, cd->hs[1], cd->g1.as<float>(), B, 2 * Hz, 2 * Wz, cd->g2.as<float>(), st, -1, nullptr, sk);
    // sigma, and its scale index in the same epilogue
    QFuse q;
    q.mode = 2;
    q.idx = cd->idx.as<uint8_t>();
    q.tab = cd->scales.as<float>();
    q.C = cd->M;
    run_layer(cd, cd->hs[2], cd->g2.as<float>(), B, 4 * Hz, 4 * Wz, cd->sigma.as<float>(), st, -1, nullptr, sk, &q);
    if (!q.done) {
        const double n = 16.0 * B * Hz * Wz * cd->M;
        timed(cd, "scale_index", 0, 5 * n, 1, st, [&] {
            launch_scale_index(cd->sigma.as<float>(), B, 16 * Hz * Wz, cd->M, cd->idx.as<uint8_t>(), nullptr, st);
        });
    }
}

// g_s: y_hat (NHWC) -> xpre (NHWC, 3 channels); deconvs with IGDN between
void teacher_synthesis(lic_codec *cd, const float *yhat, int B, int Hy, int Wy, cudaStream_t st) {
    float *a = cd->act0.as<float>(), *b = cd->act1.as<float>();
    int H = Hy, W = Wy;
    const float *in = yhat;
    if (cd->gs[0].in_dt == DT_BF16) {   // precision forms: g_s takes y_hat as bf16
        const int64_t n = (int64_t)B * Hy * Wy * cd->M;
        timed(cd, "to_bf16", 0, 6.0 * n, 1, st, [&] { launch_to_bf16(yhat, n, a, st); });
        in = a;
    }
    for (int i = 0; i < 3; ++i) {
        in = run_layer_gdn(cd, cd->gs[i], cd->igdn[i], in, B, H, W, a, b, st);
        H *= 2;
        W *= 2;
    }
    // the contributions of g_s's last layer go to the activation buffer its input is not in
    // (when it is large enough: 128 floats a position)
    run_layer(cd, cd->gs[3], in, B, H, W, cd->xpre.as<float>(), st, -1, in == a ? &cd->act1 : &cd->act0);
}

// g_s, or the student in its place when one is set
int synthesis(lic_codec *cd, const float *yhat, int B, int Hy, int Wy, cudaStream_t st) {
    if (cd->student) {
        AllocScope not_ours(nullptr);   // the student's buffers are its own
        return student_forward_nhwc(cd->student, yhat, B, Hy, Wy, cd->xpre.as<float>(), st);
    }
    teacher_synthesis(cd, yhat, B, Hy, Wy, st);
    return LIC_OK;
}

// checked decoding: both nets, per-frame PSNR of the student against the
// teacher, the teacher's frame wherever the student falls below the bar
int checked_synthesis(lic_codec *cd, int B, int Hp, int Wp, int H, int W, cudaStream_t st) {
    if (B > 1024) return LIC_E_INVALID_ARG;
    teacher_synthesis(cd, cd->yhat.as<float>(), B, Hp / 16, Wp / 16, st);
    LIC_CUDA_TRY(cd->xstu.ensure((size_t)B * Hp * Wp * 3 * sizeof(float)));
    LIC_CUDA_TRY(cd->stu_part.ensure((size_t)B * 64 * sizeof(double)));
    LIC_CUDA_TRY(cd->stu_psnr.ensure((size_t)B * sizeof(float)));
    LIC_CUDA_TRY(cd->stu_pass.ensure((size_t)B * sizeof(int)));
    int rc;
    {
        AllocScope not_ours(nullptr);   // the student's buffers are its own
        rc = student_forward_nhwc(cd->student, cd->yhat.as<float>(), B, Hp / 16, Wp / 16, cd->xstu.as<float>(), st);
    }
    if (rc) return rc;
    timed(cd, "student_check", 0, 24.0 * B * Hp * Wp, 3, st, [&] {
        launch_student_check(cd->xstu.as<float>(), cd->xpre.as<float>(), B, Hp, Wp, H, W, cd->stu_thr,
                             cd->stu_part.as<double>(), cd->stu_psnr.as<float>(), cd->stu_pass.as<int>(),
                             cd->stu_counts.as<long long>(), st);
    });
    cd->stu_lastB = B;
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

void fill_out(lic_codec::Batch *bb, int B, int H, int W, lic_bitstreams *out) {
    int64_t *h = static_cast<int64_t *>(bb->h_offs.p);
    const int64_t *d = bb->offs.as<int64_t>();
    out->count = B;
    out->on_device = 1;
    out->data = bb->data.as<uint8_t>();
    out->offsets = h;
    out->sizes = h + B + 1;
    out->d_offsets = d;
    out->d_sizes = d + B + 1;
    out->H = H;
    out->W = W;
    out->owner = bb;
}

int entropy_encode(lic_codec *cd, const StreamGeom &g, int B, const int32_t *s_y, const uint8_t *idx,
                   const int32_t *s_z, lic_bitstreams *out, cudaStream_t st) {
    int rc = LIC_OK;
    lic_codec::Batch *bb = acquire_batch(cd, g, B, &rc);
    if (!bb) return rc;
    const double nsym = (double)B * ((double)g.M * g.Hy * g.Wy + (double)g.nz * g.Hz * g.Wz);
    timed(cd, "rans_encode", 0, 5 * nsym, g.version == 2 ? 2 : 1, st, [&] {   // format 2: + the length sum
        launch_entropy_encode(g, B, cd->dt, s_y, idx, s_z, cd->scratch.as<uint16_t>(), cd->counts.as<int64_t>(), st);
    });
    timed(cd, "rans_compact", 0, 0, 3, st, [&] {
        launch_entropy_compact(g, B, cd->scratch.as<uint16_t>(), cd->counts.as<int64_t>(), cd->sub_off.as<int64_t>(),
                               cd->frame_bytes.as<int64_t>(), bb->offs.as<int64_t>(), bb->data.as<uint8_t>(), st);
    });
    LIC_CUDA_TRY(cudaMemcpyAsync(bb->h_offs.p, bb->offs.p, (2 * (size_t)B + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    LIC_CUDA_TRY(cudaGetLastError());
    bb->live = true;
    fill_out(bb, B, g.H, g.W, out);
    return LIC_OK;
}

// The frame size of a batch: in->H, in->W, else frame 0's header (copied
// from the device when the batch lives there).
int batch_frame_size(const lic_bitstreams *in, int *H, int *W, cudaStream_t st) {
    if (in->H > 0 && in->W > 0) {
        *H = in->H;
        *W = in->W;
        return LIC_OK;
    }
    if (in->H != 0 || in->W != 0 || !in->data) return LIC_E_INVALID_ARG;
    uint8_t head[36];
    int64_t off = 0, size = 0;
    if (in->on_device) {
        if (!in->d_offsets || !in->d_sizes) return LIC_E_INVALID_ARG;
        LIC_CUDA_TRY(cudaStreamSynchronize(st));
        LIC_CUDA_TRY(cudaMemcpy(&off, in->d_offsets, 8, cudaMemcpyDeviceToHost));
        LIC_CUDA_TRY(cudaMemcpy(&size, in->d_sizes, 8, cudaMemcpyDeviceToHost));
        if (off < 0) return LIC_E_INVALID_ARG;
        if (size < 36) return LIC_E_CORRUPT_STREAM;
        LIC_CUDA_TRY(cudaMemcpy(head, in->data + off, 36, cudaMemcpyDeviceToHost));
    } else {
        if (!in->offsets || !in->sizes) return LIC_E_INVALID_ARG;
        off = in->offsets[0];
        size = in->sizes[0];
        if (off < 0) return LIC_E_INVALID_ARG;
        if (size < 36) return LIC_E_CORRUPT_STREAM;
        memcpy(head, in->data + off, 36);
    }
    int kind = 0;
    if (lic_decoded_shape(head, 36, &kind, H, W) != LIC_OK || *H < 1 || *W < 1) return LIC_E_CORRUPT_STREAM;
    return LIC_OK;
}

// Bring a bitstream batch onto the device: returns device data/offsets/sizes.
int stage_bitstreams(lic_codec *cd, const lic_bitstreams *in, const uint8_t **data, const int64_t **offs,
                     const int64_t **sizes, cudaStream_t st) {
    const int B = in->count;
    if (in->on_device) {
        if (!in->d_offsets || !in->d_sizes || !in->data) return LIC_E_INVALID_ARG;
        *data = in->data;
        *offs = in->d_offsets;
        *sizes = in->d_sizes;
        return LIC_OK;
    }
    if (!in->offsets || !in->sizes || !in->data) return LIC_E_INVALID_ARG;
    std::vector<int64_t> ho(2 * (size_t)B + 1);
    int64_t o = 0;
    for (int b = 0; b < B; ++b) {
        if (in->sizes[b] < 0) return LIC_E_INVALID_ARG;
        ho[b] = o;
        ho[B + 1 + b] = in->sizes[b];
        o += (in->sizes[b] + 15) / 16 * 16;
    }
    ho[B] = o;
    LIC_CUDA_TRY(cd->in_data.ensure((size_t)o + 16));
    LIC_CUDA_TRY(cd->in_offs.ensure(ho.size() * sizeof(int64_t)));
    for (int b = 0; b < B; ++b)
        if (in->sizes[b] > 0)
            LIC_CUDA_TRY(cudaMemcpyAsync(cd->in_data.as<uint8_t>() + ho[b], in->data + in->offsets[b],
                                         (size_t)in->sizes[b], cudaMemcpyHostToDevice, st));
    LIC_CUDA_TRY(cudaMemcpyAsync(cd->in_offs.p, ho.data(), ho.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    // the host vector dies here: make the copy complete before returning
    LIC_CUDA_TRY(cudaStreamSynchronize(st));
    *data = cd->in_data.as<uint8_t>();
    *offs = cd->in_offs.as<int64_t>();
    *sizes = cd->in_offs.as<int64_t>() + B + 1;
    return LIC_OK;
}

// Entropy decoding of a batch (and, for the hyperprior, h_s in between);
// leaves s_y / yhat (and s_z / zhat / sigma / idx) in the workspace.
int entropy_decode(lic_codec *cd, const lic_bitstreams *in, int H, int W, cudaStream_t st) {
    const int B = in->count;
    const int Hp = pad64(H), Wp = pad64(W);
    int rc = ensure_workspace(cd, B, Hp, Wp);
    if (rc) return rc;
    const uint8_t *data;
    const int64_t *offs, *sizes;
    if ((rc = stage_bitstreams(cd, in, &data, &offs, &sizes, st))) return rc;
    StreamGeom g = make_geom(cd->kind, cd->N, cd->M, H, W, Hp, Wp, cd->opt.band_rows, cd->opt.format, cd->opt.resume_groups);
    uint32_t *status = cd->status.as<uint32_t>();
    if (cd->kind == LIC_HYPERPRIOR) {
        timed(cd, "rans_decode_z", 0, 8.0 * B * g.nz * g.Hz * g.Wz, 1, st, [&] {
            launch_entropy_decode(g, B, 0, cd->dt, data, offs, sizes, nullptr, cd->med.as<float>(),
                               cd->s_z.as<int32_t>(), cd->zhat.as<float>(), status, st);
        });
        hyper_synthesis(cd, cd->zhat.as<float>(), B, g.Hz, g.Wz, st);
    }
    timed(cd, "rans_decode_y", 0, 9.0 * B * g.M * g.Hy * g.Wy, 1, st, [&] {
        launch_entropy_decode(g, B, 1, cd->dt, data, offs, sizes,
                           cd->kind == LIC_HYPERPRIOR ? cd->idx.as<uint8_t>() : nullptr, cd->med.as<float>(),
                           cd->s_y.as<int32_t>(), cd->yhat.as<float>(), status, st);
    });
    cd->last_B = B;
    cd->last_Hp = Hp;
    cd->last_Wp = Wp;
    cd->have_y = false;
    cd->have_sy = true;
    cd->have_z = false;
    cd->have_sz = cd->kind == LIC_HYPERPRIOR;
    cd->have_sigma = cd->have_idx = cd->kind == LIC_HYPERPRIOR;
    cd->have_xpre = false;
    cd->have_yhat = true;
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

int copy_in(lic_codec *cd, DevBuf &stage, const void *src, size_t bytes, const void **dev, cudaStream_t st) {
    if (is_device_ptr(src)) {
        *dev = src;
        return LIC_OK;
    }
    LIC_CUDA_TRY(stage.ensure(bytes));
    LIC_CUDA_TRY(cudaMemcpyAsync(stage.p, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = stage.p;
    return LIC_OK;
}

}  // namespace
}  // namespace lic

namespace lic {
int codec_entropy_view(const lic_codec *cd, CodecEntropyView *out) {
    if (!cd || !out) return LIC_E_INVALID_ARG;
    out->kind = cd->kind;
    out->N = cd->N;
    out->M = cd->M;
    out->R = cd->opt.band_rows;
    out->version = cd->opt.format;
    out->S = cd->opt.resume_groups;
    out->device = cd->device;
    out->tables = cd->dt;
    return LIC_OK;
}
}  // namespace lic

using namespace lic;

extern "C" {

const char *lic_strerror(int code) {
    switch (code) {
        case LIC_OK: return "ok";
        case LIC_E_INVALID_ARG: return g_last_error[0] ? g_last_error : "invalid argument";
        case LIC_E_UNSUPPORTED: return "unsupported configuration";
        case LIC_E_OOM: return "out of device memory";
        case LIC_E_CORRUPT_STREAM: return "corrupt bitstream";
        case LIC_E_TIMEOUT: return "device wait timed out";
        case LIC_E_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
        case LIC_E_BUSY: return "busy: too many requests in flight";
        default: return "unknown error";
    }
}

void lic_scale_table(float T[64]) { lic::scale_table(T); }

static int pack_eb(const ParamMap &pm, int C, std::vector<double> *out) {
    static const int f[6] = {1, 3, 3, 3, 3, 1};
    std::vector<const float *> H(5), b(5), a(4);
    for (int k = 0; k < 5; ++k) {
        int rc = get_param(pm, "eb.H" + std::to_string(k), (int64_t)C * f[k + 1] * f[k], &H[k]);
        if (rc) return rc;
        rc = get_param(pm, "eb.b" + std::to_string(k), (int64_t)C * f[k + 1], &b[k]);
        if (rc) return rc;
        if (k < 4 && (rc = get_param(pm, "eb.a" + std::to_string(k), (int64_t)C * f[k + 1], &a[k]))) return rc;
    }
    out->assign((size_t)C * 58, 0.0);
    for (int c = 0; c < C; ++c) {
        double *p = out->data() + (size_t)c * 58;
        for (int k = 0; k < 5; ++k)
            for (int e = 0; e < f[k + 1] * f[k]; ++e) *p++ = H[k][(size_t)c * f[k + 1] * f[k] + e];
        for (int k = 0; k < 5; ++k)
            for (int e = 0; e < f[k + 1]; ++e) *p++ = b[k][(size_t)c * f[k + 1] + e];
        for (int k = 0; k < 4; ++k)
            for (int e = 0; e < f[k + 1]; ++e) *p++ = a[k][(size_t)c * f[k + 1] + e];
    }
    return LIC_OK;
}

static ParamMap param_map(const lic_weights *w) {
    ParamMap pm;
    for (int i = 0; i < w->count; ++i)
        if (w->params[i].name) pm[w->params[i].name] = {w->params[i].data, w->params[i].numel};
    return pm;
}

int lic_build_tables(const lic_weights *weights, int gauss, int max_tables, int64_t cdf_cap, float *medians,
                     int32_t *lo, int32_t *hi, int64_t *start, uint32_t *cdf) {
    if (!weights || !weights->params) return LIC_E_INVALID_ARG;
    ParamMap pm = param_map(weights);
    auto it = pm.find("eb.H0");
    if (it == pm.end() || it->second.second % 3 != 0) return LIC_E_INVALID_ARG;
    int C = (int)(it->second.second / 3);
    std::vector<double> P;
    int rc = pack_eb(pm, C, &P);
    if (rc) return rc;
    HostTables t;
    if ((rc = build_tables(P, C, gauss != 0, &t))) return rc;
    int nt = (int)t.lo.size();
    if (nt > max_tables || (int64_t)t.cdf.size() > cdf_cap) return LIC_E_INVALID_ARG;
    if (medians) memcpy(medians, t.medians.data(), C * sizeof(float));
    memcpy(lo, t.lo.data(), nt * sizeof(int32_t));
    memcpy(hi, t.hi.data(), nt * sizeof(int32_t));
    memcpy(start, t.start.data(), nt * sizeof(int64_t));
    memcpy(cdf, t.cdf.data(), t.cdf.size() * sizeof(uint32_t));
    return nt;
}

int lic_codec_create(int kind, int N, int M, const lic_weights *weights, const lic_options *opts, lic_codec **out) {
    g_last_error[0] = 0;
    if (!out || !weights || !weights->params) return LIC_E_INVALID_ARG;
    *out = nullptr;
    if (kind != LIC_FACTORIZED && kind != LIC_HYPERPRIOR) return LIC_E_INVALID_ARG;
    if (N <= 0 || M <= 0) return LIC_E_INVALID_ARG;
    if (N % 32 || M % 32 || N > 256 || M > 512) return LIC_E_UNSUPPORTED;
    auto cd = std::make_unique<lic_codec>();
    cd->kind = kind;
    cd->N = N;
    cd->M = M;
    if (opts) cd->opt = *opts;
    if (cd->opt.band_rows <= 0) cd->opt.band_rows = 16;
    if (cd->opt.format == 0) cd->opt.format = LIC_FORMAT_1;
    if (cd->opt.format != LIC_FORMAT_1 && cd->opt.format != LIC_FORMAT_2) return LIC_E_INVALID_ARG;
    if (cd->opt.resume_groups < 0 || cd->opt.resume_groups > 65535 ||
        (cd->opt.format == LIC_FORMAT_1 && cd->opt.resume_groups != 0))
        return LIC_E_INVALID_ARG;
    if (cd->opt.reserved[0] || cd->opt.reserved[1]) return LIC_E_INVALID_ARG;
    if (cd->opt.norm != LIC_NORM_GDN && cd->opt.norm != LIC_NORM_1DN) return LIC_E_INVALID_ARG;
    if (cd->opt.precision < LIC_FP32 || cd->opt.precision > LIC_FP8) return LIC_E_UNSUPPORTED;
    if (cd->opt.precision != LIC_FP32 && cd->opt.conv_impl == LIC_CONV_SIMT) return LIC_E_UNSUPPORTED;
    AllocScope scope(&cd->device_bytes);
    LIC_CUDA_TRY(cudaGetDevice(&cd->device));
    for (int i = 0; i < 3; ++i) {
        LIC_CUDA_TRY(cudaStreamCreateWithFlags(&cd->aux[i], cudaStreamNonBlocking));
        LIC_CUDA_TRY(cudaEventCreateWithFlags(&cd->ev_join[i], cudaEventDisableTiming));
    }
    LIC_CUDA_TRY(cudaEventCreateWithFlags(&cd->ev_fork, cudaEventDisableTiming));
    LIC_CUDA_TRY(upload_scale_table());
    {
        float T[64];
        scale_table(T);   // the scale index fused into h_s's epilogue reads them from here
        int rc0 = upload(cd->scales, T, sizeof(T));
        if (rc0) return rc0;
    }
    ParamMap pm = param_map(weights);
    int rc;
    const int ch[5] = {3, N, N, N, M};
    for (int i = 0; i < 4; ++i) {
        if ((rc = make_conv(cd->ga[i], pm, "g_a.conv" + std::to_string(i), ch[i], ch[i + 1], 5, 2, IN_NONE, EPI_NONE)))
            return rc;
        if ((rc = make_deconv(cd->gs[i], pm, "g_s.deconv" + std::to_string(i), ch[4 - i], ch[3 - i], EPI_NONE)))
            return rc;
    }
    for (int i = 0; i < 3; ++i) {
        const bool diag = cd->opt.norm == LIC_NORM_1DN;
        if ((rc = make_gdn(cd->gdn[i], pm, "g_a.gdn" + std::to_string(i), N, false, diag))) return rc;
        if ((rc = make_gdn(cd->igdn[i], pm, "g_s.igdn" + std::to_string(i), N, true, diag))) return rc;
    }
    if (kind == LIC_HYPERPRIOR) {
        if ((rc = make_conv(cd->ha[0], pm, "h_a.conv0", M, N, 3, 1, IN_ABS, EPI_RELU))) return rc;
        if ((rc = make_conv(cd->ha[1], pm, "h_a.conv1", N, N, 5, 2, IN_NONE, EPI_RELU))) return rc;
        if ((rc = make_conv(cd->ha[2], pm, "h_a.conv2", N, N, 5, 2, IN_NONE, EPI_NONE))) return rc;
        if ((rc = make_deconv(cd->hs[0], pm, "h_s.deconv0", N, N, EPI_RELU))) return rc;
        if ((rc = make_deconv(cd->hs[1], pm, "h_s.deconv1", N, N, EPI_RELU))) return rc;
        if ((rc = make_conv(cd->hs[2], pm, "h_s.conv2", N, M, 3, 1, IN_NONE, EPI_RELU))) return rc;
    }
    if (cd->opt.precision != LIC_FP32) {
        // Low-precision activations flow g_a conv0 -> conv1 -> conv2 -> conv3
        // and y_hat -> g_s deconv0 -> deconv1 -> deconv2; y and the input of
        // the last (CUDA-core) layer of g_s stay float32.  FP8: e4m3 wherever
        // the consumer has a multiple of 128 input channels, bf16 otherwise.
        const bool f8 = cd->opt.precision == LIC_FP8;
        const float S = 1.f / 16.f;   // e4m3 activation scale: |x| <= 448 * S = 28 representable
        auto lp_in = [&](Layer &L) {
            if (f8 && L.Cin % 64 == 0) {
                L.in_dt = DT_E4M3;
                L.in_scale = S;
            } else {
                L.in_dt = DT_BF16;
            }
        };
        auto lp_out_for = [&](Layer &L, const Layer &next) {
            L.out_dt = next.in_dt;
            L.out_scale = next.in_scale;
        };
        for (int i = 1; i < 4; ++i) lp_in(cd->ga[i]);
        for (int i = 0; i < 3; ++i) lp_in(cd->gs[i]);
        cd->gs[0].in_dt = DT_BF16;   // y_hat is converted to bf16 once
        cd->gs[0].in_scale = 1.f;
        // the last layer of g_s: bf16 input where its two-pass form runs on the tensor cores
        // (N >= 128; the bf16 tap GEMM), float32 for the CUDA-core form
        if (cd->gs[3].w_scatter.bvalid) cd->gs[3].in_dt = DT_BF16;
        for (int i = 0; i < 3; ++i) lp_out_for(cd->ga[i], cd->ga[i + 1]);
        for (int i = 0; i < 3; ++i) lp_out_for(cd->gs[i], cd->gs[i + 1]);
        auto check = [&](const Layer &L) {
            for (auto &op : L.ops) {
                bool ok = L.in_dt == DT_E4M3 ? op->tcw.f8valid : op->tcw.bvalid;
                if (!ok && !op->parts.empty()) {
                    ok = true;
                    for (auto &pt : op->parts) ok = ok && (L.in_dt == DT_E4M3 ? pt->f8valid : pt->bvalid);
                }
                if (!ok) return false;
            }
            return true;
        };
        for (int i = 1; i < 4; ++i)
            if (!check(cd->ga[i])) return LIC_E_UNSUPPORTED;
        for (int i = 0; i < 3; ++i)
            if (!check(cd->gs[i])) return LIC_E_UNSUPPORTED;
        for (int i = 0; i < 3; ++i)
            if ((!cd->gdn[i].diag && (!cd->gdn[i].tcw.valid || !cd->igdn[i].tcw.valid)) || (N != 128 && N != 192))
                return LIC_E_UNSUPPORTED;
        // a norm the low-precision kernels cannot fuse runs unfused and hands the next layer
        // bf16: no e4m3 input may follow one (the kernels fuse at 128 and 192 channels)
        for (int i = 0; i < 3; ++i) {
            const bool fusable = cd->gdn[i].diag || N == 128 || N == 192;
            if (!fusable && (cd->ga[i + 1].in_dt == DT_E4M3 || (i < 2 && cd->gs[i + 1].in_dt == DT_E4M3)))
                return LIC_E_UNSUPPORTED;
        }
        if (!cd->ga[0].ops[0]->tcw.valid) return LIC_E_UNSUPPORTED;
    }
    // tensor-core path: g_a conv0 over packed patches (same arithmetic, TMA-fed)
    if (cd->opt.conv_impl != LIC_CONV_SIMT) cd->use_patch = make_patch_layer(cd->ga0p, cd->ga[0], pm) == LIC_OK;
    // entropy models: the bottleneck codes y (factorized) or z (hyperprior)
    const int C = kind == LIC_FACTORIZED ? M : N;
    std::vector<double> P;
    if ((rc = pack_eb(pm, C, &P))) return rc;
    if ((rc = build_tables(P, C, kind == LIC_HYPERPRIOR, &cd->ht))) return rc;

    if ((rc = upload(cd->cdf, cd->ht.cdf.data(), cd->ht.cdf.size() * 4))) return rc;
    if ((rc = upload(cd->start, cd->ht.start.data(), cd->ht.start.size() * 8))) return rc;
    if ((rc = upload(cd->lo, cd->ht.lo.data(), cd->ht.lo.size() * 4))) return rc;
    if ((rc = upload(cd->hi, cd->ht.hi.data(), cd->ht.hi.size() * 4))) return rc;
    if ((rc = upload(cd->med, cd->ht.medians.data(), cd->ht.medians.size() * 4))) return rc;
    {
        // slot lookup of every table (see LUT_N)
        const size_t nt = cd->ht.lo.size();
        std::vector<uint16_t> lut(nt * LUT_N);
        for (size_t t = 0; t < nt; ++t) {
            const int n = cd->ht.lo[t] + cd->ht.hi[t] + 2;
            const uint32_t *c = cd->ht.cdf.data() + cd->ht.start[t];
            int s = 0;
            for (int j = 0; j < LUT_N - 1; ++j) {
                const uint32_t slot = 256u * (uint32_t)j;
                while (s < n - 1 && c[s + 1] <= slot) ++s;
                lut[t * LUT_N + j] = (uint16_t)s;
            }
            lut[t * LUT_N + LUT_N - 1] = (uint16_t)(n - 1);
        }
        if ((rc = upload(cd->lut, lut.data(), lut.size() * sizeof(uint16_t)))) return rc;
        if (cd->opt.format == LIC_FORMAT_2 && kind == LIC_HYPERPRIOR) {
            // the format-2 kernels' shared-memory image of the Gaussian tables
            std::vector<uint8_t> img;
            if (!build_gauss_image(cd->ht, C, lut, &img)) return LIC_E_UNSUPPORTED;
            if ((rc = upload(cd->gimg, img.data(), img.size()))) return rc;
        }
    }
    cd->dt.gimg = cd->gimg.p;
    cd->dt.lut = cd->lut.as<uint16_t>();
    cd->dt.cdf = cd->cdf.as<uint32_t>();
    cd->dt.start = cd->start.as<int64_t>();
    cd->dt.lo = cd->lo.as<int32_t>();
    cd->dt.hi = cd->hi.as<int32_t>();
    cd->dt.n_eb = C;
    cd->dt.gauss_base = kind == LIC_HYPERPRIOR ? C : -1;
    LIC_CUDA_TRY(cd->status.ensure(256));
    LIC_CUDA_TRY(cudaMemset(cd->status.p, 0, 256));
    LIC_CUDA_TRY(cudaDeviceSynchronize());
    *out = cd.release();
    return LIC_OK;
}

void lic_codec_destroy(lic_codec *codec) {
    if (!codec) return;
    cudaDeviceSynchronize();
    delete codec;
}

int lic_sync(lic_codec *cd, void *stream) {
    if (!cd) return LIC_E_INVALID_ARG;
    LIC_CUDA_TRY(cudaStreamSynchronize(S(stream)));
    uint32_t st = 0;
    LIC_CUDA_TRY(cudaMemcpy(&st, cd->status.p, 4, cudaMemcpyDeviceToHost));
    if (st) LIC_CUDA_TRY(cudaMemset(cd->status.p, 0, 4));
    if (st & ST_CORRUPT) return LIC_E_CORRUPT_STREAM;
    if (st & ST_TIMEOUT) return LIC_E_TIMEOUT;
    return LIC_OK;
}

int lic_encode(lic_codec *cd, const float *frames, int B, int H, int W, lic_bitstreams *out, void *stream) {
    if (!cd || !frames || !out || B < 1 || H < 1 || W < 1) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    cudaStream_t st = S(stream);
    const int Hp = pad64(H), Wp = pad64(W);
    int rc = ensure_workspace(cd, B, Hp, Wp);
    if (rc) return rc;
    const void *src;
    if ((rc = copy_in(cd, cd->stage_in, frames, (size_t)B * 3 * H * W * sizeof(float), &src, st))) return rc;
    analysis(cd, static_cast<const float *>(src), B, H, W, Hp, Wp, st);
    const int Hy = Hp / 16, Wy = Wp / 16;
    StreamGeom g = make_geom(cd->kind, cd->N, cd->M, H, W, Hp, Wp, cd->opt.band_rows, cd->opt.format, cd->opt.resume_groups);
    // Q(y), Q(z) and the scale index run in the epilogues that produce y, z and sigma
    // (q_*_fused); the separate kernels only where those launches could not
    if (!cd->q_y_fused) {
        timed(cd, "quantize_y", 0, 8.0 * B * Hy * Wy * cd->M, 1, st, [&] {
            launch_quantize(cd->y.as<float>(), B, Hy * Wy, cd->M,
                            cd->kind == LIC_FACTORIZED ? cd->med.as<float>() : nullptr, cd->s_y.as<int32_t>(), nullptr,
                            st);
        });
    }
    if (cd->kind == LIC_HYPERPRIOR) {
        hyper_analysis(cd, cd->y.as<float>(), B, Hy, Wy, st);
        if (!cd->q_z_fused) {
            timed(cd, "quantize_z", 0, 12.0 * B * g.Hz * g.Wz * cd->N, 1, st, [&] {
                launch_quantize(cd->z.as<float>(), B, g.Hz * g.Wz, cd->N, cd->med.as<float>(),
                                cd->s_z.as<int32_t>(), cd->zhat.as<float>(), st);
            });
        }
        hyper_synthesis(cd, cd->zhat.as<float>(), B, g.Hz, g.Wz, st);
    }
    if ((rc = entropy_encode(cd, g, B, cd->s_y.as<int32_t>(), cd->idx.as<uint8_t>(), cd->s_z.as<int32_t>(), out, st)))
        return rc;
    cd->last_B = B;
    cd->last_Hp = Hp;
    cd->last_Wp = Wp;
    cd->have_y = cd->have_sy = true;
    cd->have_z = cd->have_sz = cd->have_sigma = cd->have_idx = cd->kind == LIC_HYPERPRIOR;
    cd->have_xpre = cd->have_yhat = false;
    return LIC_OK;
}

int lic_encode_latents(lic_codec *cd, const int32_t *s_y, const uint8_t *idx, const int32_t *s_z, int B, int H, int W,
                       int Hy, int Wy, lic_bitstreams *out, void *stream) {
    if (!cd || !s_y || !out || B < 1 || H < 1 || W < 1 || Hy < 1 || Wy < 1) return LIC_E_INVALID_ARG;
    if (cd->kind == LIC_HYPERPRIOR && (!idx || !s_z || Hy % 4 || Wy % 4)) return LIC_E_INVALID_ARG;
    if (!is_device_ptr(s_y) || (idx && !is_device_ptr(idx)) || (s_z && !is_device_ptr(s_z))) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    StreamGeom g = make_geom(cd->kind, cd->N, cd->M, H, W, 16 * Hy, 16 * Wy, cd->opt.band_rows, cd->opt.format,
                             cd->opt.resume_groups);
    return entropy_encode(cd, g, B, s_y, idx, s_z, out, S(stream));
}

int lic_bitstreams_release(lic_codec *cd, lic_bitstreams *bs) {
    if (!cd || !bs) return LIC_E_INVALID_ARG;
    if (!bs->owner) return bs->count == 0 ? LIC_OK : LIC_E_INVALID_ARG;
    for (auto &p : cd->batches)
        if (p.get() == bs->owner) {
            if (!p->live) return LIC_E_INVALID_ARG;
            p->live = false;
            *bs = lic_bitstreams{};
            return LIC_OK;
        }
    return LIC_E_INVALID_ARG;
}

int lic_decode_latents(lic_codec *cd, const lic_bitstreams *in, int32_t *s_y, int32_t *s_z, void *stream) {
    if (!cd || !in || !s_y || in->count < 1) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    cudaStream_t st = S(stream);
    int H = 0, W = 0;
    int rc = batch_frame_size(in, &H, &W, st);
    if (rc) return rc;
    if ((rc = entropy_decode(cd, in, H, W, st))) return rc;
    const int B = in->count, Hp = pad64(H), Wp = pad64(W);
    const int64_t ny = (int64_t)B * cd->M * (Hp / 16) * (Wp / 16);
    LIC_CUDA_TRY(cudaMemcpyAsync(s_y, cd->s_y.p, ny * 4, cudaMemcpyDefault, st));
    if (cd->kind == LIC_HYPERPRIOR && s_z) {
        const int64_t nz = (int64_t)B * cd->N * (Hp / 64) * (Wp / 64);
        LIC_CUDA_TRY(cudaMemcpyAsync(s_z, cd->s_z.p, nz * 4, cudaMemcpyDefault, st));
    }
    return LIC_OK;
}

int lic_decode(lic_codec *cd, const lic_bitstreams *in, float *frames, void *stream) {
    if (!cd || !in || !frames || in->count < 1) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    cudaStream_t st = S(stream);
    int H = 0, W = 0;
    int rc = batch_frame_size(in, &H, &W, st);
    if (rc) return rc;
    if ((rc = entropy_decode(cd, in, H, W, st))) return rc;
    const int B = in->count, Hp = pad64(H), Wp = pad64(W);
    rc = (cd->student && cd->stu_checked) ? checked_synthesis(cd, B, Hp, Wp, H, W, st)
                                          : synthesis(cd, cd->yhat.as<float>(), B, Hp / 16, Wp / 16, st);
    if (rc) return rc;
    cd->have_xpre = true;
    const size_t bytes = (size_t)B * 3 * H * W * sizeof(float);
    if (is_device_ptr(frames)) {
        timed(cd, "crop_unpack", 0, 24.0 * B * H * W, 1, st,
              [&] { launch_crop_unpack(cd->xpre.as<float>(), B, Hp, Wp, H, W, frames, st); });
    } else {
        LIC_CUDA_TRY(cd->stage_out.ensure(bytes));
        timed(cd, "crop_unpack", 0, 24.0 * B * H * W, 1, st,
              [&] { launch_crop_unpack(cd->xpre.as<float>(), B, Hp, Wp, H, W, cd->stage_out.as<float>(), st); });
        LIC_CUDA_TRY(cudaMemcpyAsync(frames, cd->stage_out.p, bytes, cudaMemcpyDeviceToHost, st));
        LIC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

int64_t lic_codec_device_bytes(const lic_codec *cd) { return cd ? cd->device_bytes : LIC_E_INVALID_ARG; }

int64_t lic_codec_workspace_bytes(const lic_codec *cd, int B, int H, int W) {
    if (!cd || B < 1 || H < 1 || W < 1) return LIC_E_INVALID_ARG;
    lic_codec *c = const_cast<lic_codec *>(cd);   // the plans only name the buffers
    const int Hp = pad64(H), Wp = pad64(W);
    int64_t total = 0;
    auto add = [&](DevBuf &, int64_t n) {
        total += n;
        return 0;
    };
    workspace_plan(c, B, Hp, Wp, add);
    lic_codec::Batch probe;
    entropy_plan(c, make_geom(cd->kind, cd->N, cd->M, H, W, Hp, Wp, cd->opt.band_rows, cd->opt.format, cd->opt.resume_groups), B, &probe, add);
    return total;
}

int64_t lic_bitstreams_download(const lic_bitstreams *in, uint8_t *dst, int64_t dst_cap, void *stream) {
    if (!in || !dst || !in->on_device || !in->offsets || in->count < 1) return LIC_E_INVALID_ARG;
    LIC_CUDA_TRY(cudaStreamSynchronize(S(stream)));
    const int64_t n = in->offsets[in->count];
    if (n > dst_cap || n < 0) return LIC_E_INVALID_ARG;
    LIC_CUDA_TRY(cudaMemcpy(dst, in->data, (size_t)n, cudaMemcpyDeviceToHost));
    return n;
}

int lic_profile_enable(lic_codec *cd, int enable) {
    if (!cd) return LIC_E_INVALID_ARG;
    cd->pf.enable(enable != 0);
    return LIC_OK;
}

int lic_profile_report(lic_codec *cd, char *buf, int cap) { return cd ? cd->pf.report(buf, cap) : LIC_E_INVALID_ARG; }

int64_t lic_launch_count(lic_codec *cd) { return cd ? cd->pf.launches : LIC_E_INVALID_ARG; }

int lic_probe_mma_rate(int kind, int iters, double *tflops) { return tc::mma_rate(kind, iters, tflops); }

int lic_test_bounded_wait(lic_codec *cd, int64_t limit_cycles, void *stream) {
    if (!cd || limit_cycles < 1 || limit_cycles > 4000000000LL) return LIC_E_INVALID_ARG;
    timed(cd, "wait_probe", 0, 0, 1, S(stream),
          [&] { tc::launch_wait_probe(cd->status.as<uint32_t>(), (long long)limit_cycles, S(stream)); });
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

}  // extern "C"

namespace lic {
uint32_t *codec_status_ptr(lic_codec *cd) { return cd->status.as<uint32_t>(); }
}  // namespace lic

extern "C" {

int lic_codec_set_student(lic_codec *cd, lic_student *student, float min_psnr_db, int checked) {
    if (!cd || (student && student_channels(student) != cd->M) || (checked != 0 && checked != 1))
        return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    if (student && checked && !(min_psnr_db == min_psnr_db)) return LIC_E_INVALID_ARG;
    LIC_CUDA_TRY(cudaDeviceSynchronize());
    LIC_CUDA_TRY(cd->stu_counts.ensure(2 * sizeof(long long)));
    LIC_CUDA_TRY(cudaMemset(cd->stu_counts.p, 0, 2 * sizeof(long long)));
    cd->student = student;
    cd->stu_thr = min_psnr_db;
    cd->stu_checked = student ? checked : 0;
    cd->stu_lastB = 0;
    cd->have_xpre = false;
    return LIC_OK;
}

int lic_codec_student_report(lic_codec *cd, int64_t *frames, int64_t *fallbacks, float *last_psnr, int cap) {
    if (!cd || cap < 0) return LIC_E_INVALID_ARG;
    LIC_CUDA_TRY(cudaDeviceSynchronize());
    long long c[2] = {0, 0};
    if (cd->stu_counts.p) LIC_CUDA_TRY(cudaMemcpy(c, cd->stu_counts.p, sizeof(c), cudaMemcpyDeviceToHost));
    if (frames) *frames = c[0];
    if (fallbacks) *fallbacks = c[1];
    const int n = std::min(cap, cd->stu_lastB);
    if (last_psnr && n > 0) LIC_CUDA_TRY(cudaMemcpy(last_psnr, cd->stu_psnr.p, n * sizeof(float), cudaMemcpyDeviceToHost));
    return cd->stu_lastB;
}

int lic_decoded_shape(const uint8_t *f, int64_t size, int *kind, int *H, int *W) {
    if (!f || size < 36) return LIC_E_INVALID_ARG;
    if (memcmp(f, "LIC1", 4) != 0) return LIC_E_CORRUPT_STREAM;
    uint16_t ver, k;
    uint32_t h, w;
    memcpy(&ver, f + 4, 2);
    memcpy(&k, f + 6, 2);
    memcpy(&h, f + 12, 4);
    memcpy(&w, f + 16, 4);
    if ((ver != 1 && ver != 2) || k > 1) return LIC_E_CORRUPT_STREAM;
    if (kind) *kind = k;
    if (H) *H = (int)h;
    if (W) *W = (int)w;
    return LIC_OK;
}

int lic_strip_resume_records(const uint8_t *f, int64_t size, uint8_t *out, int64_t out_cap, int64_t *out_size) {
    if (!f || !out || !out_size || size < 36 || out_cap < 0) return LIC_E_INVALID_ARG;
    int kind = 0, H = 0, W = 0;
    if (lic_decoded_shape(f, size, &kind, &H, &W) != LIC_OK) return LIC_E_CORRUPT_STREAM;
    uint16_t ver = 0, S = 0;
    uint32_t nsub = 0, wend = 0;
    memcpy(&ver, f + 4, 2);
    memcpy(&S, f + 30, 2);
    memcpy(&nsub, f + 32, 4);
    const int64_t head = 36 + 4 * ((int64_t)nsub + 1);
    if (head > size) return LIC_E_CORRUPT_STREAM;
    memcpy(&wend, f + 36 + 4 * (int64_t)nsub, 4);
    const int64_t body = head + 2 * (int64_t)wend;
    if (body > size || (ver == 1 && body != size) || (ver == 2 && S == 0 && body != size)) return LIC_E_CORRUPT_STREAM;
    if (ver == 2 && S > 0 && (size - body) % 140 != 0) return LIC_E_CORRUPT_STREAM;
    if (out_cap < body) return LIC_E_INVALID_ARG;
    if (out != f) memmove(out, f, (size_t)body);
    if (ver == 2) out[30] = out[31] = 0;
    *out_size = body;
    return LIC_OK;
}

// ---- stage calls ----

// copy a device NHWC float tensor into dst (NCHW, device or host)
static int emit_nchw(lic_codec *cd, const float *src, int B, int H, int W, int C, void *dst, cudaStream_t st) {
    const size_t bytes = (size_t)B * C * H * W * sizeof(float);
    if (is_device_ptr(dst)) {
        timed(cd, "to_nchw", 0, 8.0 * B * H * W * C, 1, st,
              [&] { launch_nhwc_to_nchw(src, B, H, W, C, static_cast<float *>(dst), st); });
    } else {
        LIC_CUDA_TRY(cd->stage_out.ensure(bytes));
        timed(cd, "to_nchw", 0, 8.0 * B * H * W * C, 1, st,
              [&] { launch_nhwc_to_nchw(src, B, H, W, C, cd->stage_out.as<float>(), st); });
        LIC_CUDA_TRY(cudaMemcpyAsync(dst, cd->stage_out.p, bytes, cudaMemcpyDeviceToHost, st));
        LIC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    LIC_CUDA_TRY(cudaGetLastError());
    return LIC_OK;
}

static int ingest_nchw(lic_codec *cd, const float *src, int B, int C, int H, int W, float *dst_nhwc, cudaStream_t st) {
    const void *dev;
    int rc = copy_in(cd, cd->stage_in, src, (size_t)B * C * H * W * sizeof(float), &dev, st);
    if (rc) return rc;
    timed(cd, "to_nhwc", 0, 8.0 * B * H * W * C, 1, st,
          [&] { launch_nchw_to_nhwc(static_cast<const float *>(dev), B, C, H, W, dst_nhwc, st); });
    return LIC_OK;
}

int lic_analysis(lic_codec *cd, const float *frames, int B, int H, int W, float *y, void *stream) {
    if (!cd || !frames || !y || B < 1 || H < 1 || W < 1) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    cudaStream_t st = S(stream);
    const int Hp = pad64(H), Wp = pad64(W);
    int rc = ensure_workspace(cd, B, Hp, Wp);
    if (rc) return rc;
    const void *src;
    if ((rc = copy_in(cd, cd->stage_in, frames, (size_t)B * 3 * H * W * sizeof(float), &src, st))) return rc;
    analysis(cd, static_cast<const float *>(src), B, H, W, Hp, Wp, st);
    return emit_nchw(cd, cd->y.as<float>(), B, Hp / 16, Wp / 16, cd->M, y, st);
}

int lic_synthesis(lic_codec *cd, const float *yhat, int B, int Hy, int Wy, float *x, void *stream) {
    if (!cd || !yhat || !x || B < 1 || Hy < 1 || Wy < 1) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    cudaStream_t st = S(stream);
    int rc = ensure_workspace(cd, B, 16 * Hy, 16 * Wy);
    if (rc) return rc;
    if ((rc = ingest_nchw(cd, yhat, B, cd->M, Hy, Wy, cd->yhat.as<float>(), st))) return rc;
    if ((rc = synthesis(cd, cd->yhat.as<float>(), B, Hy, Wy, st))) return rc;
    return emit_nchw(cd, cd->xpre.as<float>(), B, 16 * Hy, 16 * Wy, 3, x, st);
}

int lic_hyper_analysis(lic_codec *cd, const float *y, int B, int Hy, int Wy, float *z, void *stream) {
    if (!cd || !y || !z || B < 1 || Hy < 4 || Wy < 4 || Hy % 4 || Wy % 4) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    if (cd->kind != LIC_HYPERPRIOR) return LIC_E_INVALID_ARG;
    cudaStream_t st = S(stream);
    int rc = ensure_workspace(cd, B, 16 * Hy, 16 * Wy);
    if (rc) return rc;
    if ((rc = ingest_nchw(cd, y, B, cd->M, Hy, Wy, cd->y.as<float>(), st))) return rc;
    hyper_analysis(cd, cd->y.as<float>(), B, Hy, Wy, st);
    return emit_nchw(cd, cd->z.as<float>(), B, Hy / 4, Wy / 4, cd->N, z, st);
}

int lic_hyper_synthesis(lic_codec *cd, const float *zhat, int B, int Hz, int Wz, float *sigma, uint8_t *idx,
                        void *stream) {
    if (!cd || !zhat || !sigma || B < 1 || Hz < 1 || Wz < 1) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    if (cd->kind != LIC_HYPERPRIOR) return LIC_E_INVALID_ARG;
    cudaStream_t st = S(stream);
    int rc = ensure_workspace(cd, B, 64 * Hz, 64 * Wz);
    if (rc) return rc;
    if ((rc = ingest_nchw(cd, zhat, B, cd->N, Hz, Wz, cd->zhat.as<float>(), st))) return rc;
    hyper_synthesis(cd, cd->zhat.as<float>(), B, Hz, Wz, st);
    if ((rc = emit_nchw(cd, cd->sigma.as<float>(), B, 4 * Hz, 4 * Wz, cd->M, sigma, st))) return rc;
    if (idx) {
        const size_t n = (size_t)B * cd->M * 16 * Hz * Wz;
        LIC_CUDA_TRY(cudaMemcpyAsync(idx, cd->idx.p, n, cudaMemcpyDefault, st));
        LIC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return LIC_OK;
}

int lic_read_tensor(lic_codec *cd, int which, void *dst, int64_t *count, void *stream) {
    if (!cd) return LIC_E_INVALID_ARG;
    AllocScope scope(&cd->device_bytes);
    cudaStream_t st = S(stream);
    const int B = cd->last_B, Hp = cd->last_Hp, Wp = cd->last_Wp;
    const int Hy = Hp / 16, Wy = Wp / 16, Hz = Hp / 64, Wz = Wp / 64;
    int64_t n = 0;
    bool ok = false;
    switch (which) {
        case LIC_T_Y: n = (int64_t)B * cd->M * Hy * Wy; ok = cd->have_y; break;
        case LIC_T_SY: n = (int64_t)B * cd->M * Hy * Wy; ok = cd->have_sy; break;
        case LIC_T_Z: n = (int64_t)B * cd->N * Hz * Wz; ok = cd->have_z; break;
        case LIC_T_SZ: n = (int64_t)B * cd->N * Hz * Wz; ok = cd->have_sz; break;
        case LIC_T_SIGMA: n = (int64_t)B * cd->M * Hy * Wy; ok = cd->have_sigma; break;
        case LIC_T_IDX: n = (int64_t)B * cd->M * Hy * Wy; ok = cd->have_idx; break;
        case LIC_T_XPRE: n = (int64_t)B * 3 * Hp * Wp; ok = cd->have_xpre; break;
        case LIC_T_YHAT: n = (int64_t)B * cd->M * Hy * Wy; ok = cd->have_yhat; break;
        default: return LIC_E_INVALID_ARG;
    }
    if (!ok || B == 0) return LIC_E_INVALID_ARG;
    if (count) *count = n;
    if (!dst) return LIC_OK;
    switch (which) {
        case LIC_T_Y: return emit_nchw(cd, cd->y.as<float>(), B, Hy, Wy, cd->M, dst, st);
        case LIC_T_Z: return emit_nchw(cd, cd->z.as<float>(), B, Hz, Wz, cd->N, dst, st);
        case LIC_T_SIGMA: return emit_nchw(cd, cd->sigma.as<float>(), B, Hy, Wy, cd->M, dst, st);
        case LIC_T_XPRE: return emit_nchw(cd, cd->xpre.as<float>(), B, Hp, Wp, 3, dst, st);
        case LIC_T_YHAT: return emit_nchw(cd, cd->yhat.as<float>(), B, Hy, Wy, cd->M, dst, st);
        case LIC_T_SY: LIC_CUDA_TRY(cudaMemcpyAsync(dst, cd->s_y.p, n * 4, cudaMemcpyDefault, st)); break;
        case LIC_T_SZ: LIC_CUDA_TRY(cudaMemcpyAsync(dst, cd->s_z.p, n * 4, cudaMemcpyDefault, st)); break;
        case LIC_T_IDX: LIC_CUDA_TRY(cudaMemcpyAsync(dst, cd->idx.p, n, cudaMemcpyDefault, st)); break;
    }
    LIC_CUDA_TRY(cudaStreamSynchronize(st));
    return LIC_OK;
}

}  // extern "C"
