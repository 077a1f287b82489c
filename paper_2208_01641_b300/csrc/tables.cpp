// Host-side FP64 construction of the entropy-model CDF tables, once per
// codec.  Compiled with -ffp-contract=off and without fast-math so that
// every step is a rounded IEEE double operation in the order written.
//
//  * Factorized entropy bottleneck (Ballé 2018 [2], appendix 6.1): per
//    channel a cumulative sigmoid(f(x)) with f a 1-3-3-3-3-1 net whose
//    matrices pass through softplus and whose hidden layers add
//    tanh(a) * tanh(h).  Median and tail quantiles (tail mass 1e-9) are
//    found by bisection; the pmf of the integers around the median plus an
//    escape symbol holding the tails is quantized to 16 bits.
//  * Gaussian conditional ([2]): 64 scales log-spaced over [0.11, 256]; the
//    pmf of a zero-mean Gaussian of that scale convolved with a unit box,
//    over |s| <= ceil(scale * z), Phi(-z) = 1e-9 / 2, plus the escape.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <vector>

#include "lic_internal.h"

namespace lic {
namespace {

constexpr double kTail = 1e-9;
constexpr int kMaxSymbols = 4096;
constexpr uint32_t kTotal = 1u << 16;

double softplus(double v) { return v > 0.0 ? v + std::log1p(std::exp(-v)) : std::log1p(std::exp(v)); }
double sigmoid(double v) { return 1.0 / (1.0 + std::exp(-v)); }

// One channel of the bottleneck: parameters laid out as H0..H4 (out x in,
// row-major), b0..b4, a0..a3.
class Bottleneck {
  public:
    explicit Bottleneck(const double *p) {
        static const int widths[6] = {1, 3, 3, 3, 3, 1};
        const double *q = p;
        for (int k = 0; k < 5; ++k) {
            layers_[k].in = widths[k];
            layers_[k].out = widths[k + 1];
            for (int e = 0; e < widths[k + 1] * widths[k]; ++e) layers_[k].w[e] = softplus(q[e]);
            q += widths[k + 1] * widths[k];
        }
        for (int k = 0; k < 5; ++k) {
            for (int e = 0; e < widths[k + 1]; ++e) layers_[k].b[e] = q[e];
            q += widths[k + 1];
        }
        for (int k = 0; k < 4; ++k) {
            for (int e = 0; e < widths[k + 1]; ++e) layers_[k].ta[e] = std::tanh(q[e]);
            q += widths[k + 1];
        }
    }

    double logit(double x) const {
        std::array<double, 3> cur{x, 0.0, 0.0};
        for (int k = 0; k < 5; ++k) {
            const Layer &L = layers_[k];
            std::array<double, 3> nxt{};
            for (int o = 0; o < L.out; ++o) {
                double v = 0.0;
                for (int i = 0; i < L.in; ++i) v += L.w[o * L.in + i] * cur[i];
                v += L.b[o];
                if (k < 4) v += L.ta[o] * std::tanh(v);
                nxt[o] = v;
            }
            cur = nxt;
        }
        return cur[0];
    }

    // smallest representable "upper end" of a bisection for logit(x) = t
    double solve(double t) const {
        double a = -1e6, b = 1e6;
        for (int it = 0; it < 200; ++it) {
            double m = 0.5 * (a + b);
            (logit(m) < t ? a : b) = m;
        }
        return b;
    }

  private:
    struct Layer {
        int in = 1, out = 1;
        double w[9] = {}, b[3] = {}, ta[3] = {};
    };
    Layer layers_[5];
};

double normal_cdf(double v) { return 0.5 * std::erfc(-v * M_SQRT1_2); }

double gauss_z() {
    double a = -40.0, b = 0.0;
    for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (a + b);
        (normal_cdf(m) < kTail / 2 ? a : b) = m;
    }
    return -b;
}

// 16-bit frequencies: round each probability to the nearest count (at
// least 1), then give a shortfall to the most probable symbol, or take an
// excess from the most probable symbols first (down to 1 each).
bool quantize(const std::vector<double> &pmf, std::vector<uint32_t> *cdf) {
    const int n = static_cast<int>(pmf.size());
    if (n < 1 || n > kMaxSymbols) return false;
    std::vector<uint32_t> f(n);
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        double r = std::floor(pmf[i] * 65536.0 + 0.5);
        f[i] = r < 1.0 ? 1u : static_cast<uint32_t>(r);
        total += f[i];
    }
    int64_t diff = static_cast<int64_t>(kTotal) - total;
    if (diff > 0) {
        int arg = static_cast<int>(std::max_element(f.begin(), f.end()) - f.begin());
        f[arg] += static_cast<uint32_t>(diff);
    } else if (diff < 0) {
        std::vector<int> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return f[a] > f[b]; });
        int64_t excess = -diff;
        while (excess > 0) {
            for (int i : order) {
                if (excess == 0) break;
                int64_t give = std::min<int64_t>(f[i] - 1, excess);
                f[i] -= static_cast<uint32_t>(give);
                excess -= give;
            }
        }
    }
    cdf->assign(n + 1, 0);
    for (int i = 0; i < n; ++i) (*cdf)[i + 1] = (*cdf)[i] + f[i];
    return (*cdf)[n] == kTotal;
}

void append(HostTables *t, int lo, int hi, const std::vector<uint32_t> &cdf) {
    t->lo.push_back(lo);
    t->hi.push_back(hi);
    t->start.push_back(static_cast<int64_t>(t->cdf.size()));
    t->cdf.insert(t->cdf.end(), cdf.begin(), cdf.end());
}

}  // namespace

void scale_table(float T[64]) {
    const double a = std::log(0.11), b = std::log(256.0);
    for (int k = 0; k < 64; ++k) T[k] = static_cast<float>(std::exp(a + static_cast<double>(k) * (b - a) / 63.0));
}

int build_tables(const std::vector<double> &eb_params, int channels, bool gauss, HostTables *out) {
    HostTables t;
    const double t_lo = std::log((kTail / 2) / (1.0 - kTail / 2));
    for (int c = 0; c < channels; ++c) {
        Bottleneck net(eb_params.data() + static_cast<size_t>(c) * 58);
        float med = static_cast<float>(net.solve(0.0));
        double m = static_cast<double>(med);
        double lo = std::ceil(m - net.solve(t_lo));
        double hi = std::ceil(net.solve(-t_lo) - m);
        lo = std::max(lo, 0.0);
        hi = std::max(hi, 0.0);
        if (lo + hi + 2 > kMaxSymbols) return LIC_E_UNSUPPORTED;
        int L = static_cast<int>(lo), H = static_cast<int>(hi);
        std::vector<double> pmf;
        pmf.reserve(L + H + 2);
        for (int s = -L; s <= H; ++s) {
            double a = net.logit(m + s - 0.5), b = net.logit(m + s + 0.5);
            double flip = (a + b > 0.0) ? -1.0 : 1.0;
            pmf.push_back(std::fabs(sigmoid(flip * b) - sigmoid(flip * a)));
        }
        pmf.push_back(sigmoid(net.logit(m - L - 0.5)) + sigmoid(-net.logit(m + H + 0.5)));
        std::vector<uint32_t> cdf;
        if (!quantize(pmf, &cdf)) return LIC_E_UNSUPPORTED;
        t.medians.push_back(med);
        append(&t, L, H, cdf);
    }
    t.n_eb = channels;
    if (gauss) {
        float T[64];
        scale_table(T);
        const double z = gauss_z();
        for (int k = 0; k < 64; ++k) {
            const double sd = static_cast<double>(T[k]);
            const int c = static_cast<int>(std::ceil(sd * z));
            if (2 * c + 2 > kMaxSymbols) return LIC_E_UNSUPPORTED;
            std::vector<double> pmf;
            pmf.reserve(2 * c + 2);
            for (int s = -c; s <= c; ++s) {
                double a = std::fabs(static_cast<double>(s));
                pmf.push_back(normal_cdf((0.5 - a) / sd) - normal_cdf((-0.5 - a) / sd));
            }
            pmf.push_back(2.0 * normal_cdf((-static_cast<double>(c) - 0.5) / sd));
            std::vector<uint32_t> cdf;
            if (!quantize(pmf, &cdf)) return LIC_E_UNSUPPORTED;
            append(&t, c, c, cdf);
        }
        t.n_gauss = 64;
    }
    *out = std::move(t);
    return LIC_OK;
}

}  // namespace lic
