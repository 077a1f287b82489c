// The serving form (include/lic_serve.h): per-resolution buckets of frame
// requests, a dispatcher thread that forms batches and issues them to the
// lanes (codec + stream) of their bucket, each lane's encode+decode chain
// replayed as a CUDA graph, and completion callbacks that turn finished
// batches into results.  This is the paper's frame pipeline (task FIFOs and
// a control thread per GPU workload, Sec. III-A) with all stages on the GPU:
// the overlap the paper gets between CPU and GPU stages of successive frames
// comes here from batches of several lanes and buckets in flight at once.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lic_serve.h"
#include "lic_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    int stream_id;
    const float *frame;
    float *decoded;
    double t_submit;
};

struct Bucket;

struct Lane {
    lic_server *srv = nullptr;
    Bucket *bucket = nullptr;
    lic_codec *codec = nullptr;
    cudaStream_t stream = nullptr;
    float *in = nullptr, *out = nullptr;     // device slabs, max_batch frames each
    uint32_t *status_host = nullptr;         // pinned: the codec's status word after each batch
    std::vector<cudaGraphExec_t> graphs;     // [b - 1]: encode+decode of b frames
    lic_bitstreams last{};                   // view of the last batch: its sizes (pinned, written by the chain)
    bool busy = false;
    std::vector<Request> batch;
    double t_start = 0;
};

struct Bucket {
    int H = 0, W = 0;
    std::deque<Request> q;
    std::vector<std::unique_ptr<Lane>> lanes;
    int64_t bytes = 0;
};

}  // namespace

struct lic_server {
    int kind = 0, N = 0, M = 0;
    std::vector<std::string> names;
    std::vector<std::vector<float>> data;
    lic_options copt{};
    bool has_copt = false;
    lic_server_options opt{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;                       // queues, lanes' busy flags, results, counters
    std::condition_variable work_cv;     // dispatcher: new request, lane idle, stop
    std::condition_variable done_cv;     // pollers: new result
    std::mutex prep_mu;                  // one bucket preparation at a time
    std::map<std::pair<int, int>, std::unique_ptr<Bucket>> buckets;
    std::deque<lic_server_result> done;
    uint64_t next_ticket = 0;
    int64_t pending = 0;
    lic_server_stats st{};
    bool stop = false;
    std::thread dispatcher;
};

namespace {

double now_ms(const lic_server *s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

size_t frame_floats(const Bucket *b) { return (size_t)3 * b->H * b->W; }

void destroy_lane(Lane *L) {
    for (cudaGraphExec_t g : L->graphs)
        if (g) cudaGraphExecDestroy(g);
    L->graphs.clear();
    if (L->codec) lic_codec_destroy(L->codec);
    if (L->in) cudaFree(L->in);
    if (L->out) cudaFree(L->out);
    if (L->status_host) cudaFreeHost(L->status_host);
    if (L->stream) cudaStreamDestroy(L->stream);
    L->codec = nullptr;
    L->in = L->out = nullptr;
    L->status_host = nullptr;
    L->stream = nullptr;
}

// The device part of one batch of b frames: encode, decode, then the codec's
// status word to the host and cleared (so each batch reports its own).  The
// batch goes back to the codec's pool once its decode is enqueued: the next
// chain on this lane (same stream) reuses the same buffers, so every graph
// of the lane is captured over one batch buffer.  The view stays in
// L->last for the sizes the completion callback reads.
int chain(Lane *L, int b) {
    const Bucket *B = L->bucket;
    lic_bitstreams bs{};
    int rc = lic_encode(L->codec, L->in, b, B->H, B->W, &bs, L->stream);
    if (rc) return rc;
    L->last = bs;
    rc = lic_decode(L->codec, &bs, L->out, L->stream);
    const int rr = lic_bitstreams_release(L->codec, &bs);
    if (rc) return rc;
    if (rr) return rr;
    uint32_t *dev_status = lic::codec_status_ptr(L->codec);
    if (cudaMemcpyAsync(L->status_host, dev_status, 4, cudaMemcpyDeviceToHost, L->stream) != cudaSuccess ||
        cudaMemsetAsync(dev_status, 0, 4, L->stream) != cudaSuccess)
        return LIC_E_CUDA;
    return LIC_OK;
}

int status_code(uint32_t s) {
    if (s & lic::ST_CORRUPT) return LIC_E_CORRUPT_STREAM;
    if (s & lic::ST_TIMEOUT) return LIC_E_TIMEOUT;
    return LIC_OK;
}

void finish(lic_server *s, Lane *L, int status) {
    std::vector<lic_server_result> res;
    const double t = now_ms(s);
    const int n = (int)L->batch.size();
    for (int i = 0; i < n; ++i) {
        const Request &r = L->batch[i];
        lic_server_result x{};
        x.ticket = r.ticket;
        x.stream_id = r.stream_id;
        x.status = status;
        x.H = L->bucket->H;
        x.W = L->bucket->W;
        x.batch = n;
        // the chain's offsets land in the codec's pinned array: b + 1 offsets, then b sizes
        x.bytes = (status == LIC_OK && L->last.offsets) ? L->last.offsets[n + 1 + i] : 0;
        x.t_submit_ms = r.t_submit;
        x.t_start_ms = L->t_start;
        x.t_done_ms = t;
        res.push_back(x);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &x : res) s->done.push_back(x);
        s->pending -= n;
        s->st.completed += n;
        L->batch.clear();
        L->busy = false;
    }
    s->work_cv.notify_all();
    s->done_cv.notify_all();
}

void CUDART_CB on_done(void *p) {
    Lane *L = static_cast<Lane *>(p);
    finish(L->srv, L, status_code(*L->status_host));
}

// issue the lane's current batch (called without the lock; the lane is busy)
void issue(lic_server *s, Lane *L) {
    const Bucket *B = L->bucket;
    const int b = (int)L->batch.size();
    const size_t fs = frame_floats(B);
    int rc = LIC_OK;
    L->t_start = now_ms(s);
    for (int i = 0; i < b && !rc; ++i)
        if (cudaMemcpyAsync(L->in + i * fs, L->batch[i].frame, fs * sizeof(float), cudaMemcpyDefault, L->stream) !=
            cudaSuccess)
            rc = LIC_E_CUDA;
    bool replay = false;
    if (!rc) {
        if (s->opt.graphs && (int)L->graphs.size() >= b && L->graphs[b - 1]) {
            rc = cudaGraphLaunch(L->graphs[b - 1], L->stream) == cudaSuccess ? LIC_OK : LIC_E_CUDA;
            replay = true;
        } else {
            rc = chain(L, b);
        }
    }
    for (int i = 0; i < b && !rc; ++i)
        if (L->batch[i].decoded &&
            cudaMemcpyAsync(L->batch[i].decoded, L->out + i * fs, fs * sizeof(float), cudaMemcpyDefault,
                            L->stream) != cudaSuccess)
            rc = LIC_E_CUDA;
    if (!rc && cudaLaunchHostFunc(L->stream, on_done, L) != cudaSuccess) rc = LIC_E_CUDA;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.batches += 1;
        if (replay && !rc) s->st.graph_replays += 1;
    }
    if (rc) {
        cudaStreamSynchronize(L->stream);
        finish(s, L, rc);
    }
}

void dispatch_loop(lic_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool launched = false, any_busy = false, any_queued = false;
        double deadline = -1.0;
        for (auto &kv : s->buckets) {
            Bucket *B = kv.second.get();
            for (auto &lp : B->lanes) any_busy |= lp->busy;
            while (!B->q.empty()) {
                any_queued = true;
                Lane *idle = nullptr;
                for (auto &lp : B->lanes)
                    if (!lp->busy) {
                        idle = lp.get();
                        break;
                    }
                if (!idle) break;
                const int n = (int)std::min<size_t>(B->q.size(), (size_t)s->opt.max_batch);
                const double due = B->q.front().t_submit + s->opt.max_wait_ms;
                if (n < s->opt.max_batch && now_ms(s) < due && !s->stop) {
                    deadline = deadline < 0 ? due : std::min(deadline, due);
                    break;
                }
                idle->batch.assign(B->q.begin(), B->q.begin() + n);
                B->q.erase(B->q.begin(), B->q.begin() + n);
                idle->busy = true;
                lk.unlock();
                issue(s, idle);
                lk.lock();
                launched = true;
            }
        }
        if (launched) continue;
        if (s->stop && !any_queued && !any_busy) break;
        if (deadline >= 0) {
            const auto when = s->t0 + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double, std::milli>(deadline));
            s->work_cv.wait_until(lk, when);
        } else {
            s->work_cv.wait(lk);
        }
    }
}

// Create the lane's codec only (weights and tables, no workspace yet).
int make_lane_codec(lic_server *s, Bucket *B, Lane *L) {
    L->srv = s;
    L->bucket = B;
    std::vector<lic_param> ps(s->names.size());
    for (size_t i = 0; i < ps.size(); ++i) {
        ps[i].name = s->names[i].c_str();
        ps[i].data = s->data[i].data();
        ps[i].numel = (int64_t)s->data[i].size();
    }
    lic_weights w{ps.data(), (int)ps.size()};
    return lic_codec_create((lic_kind)s->kind, s->N, s->M, &w, s->has_copt ? &s->copt : nullptr, &L->codec);
}

size_t slab_bytes(const lic_server *s, const Bucket *B) {
    return (size_t)s->opt.max_batch * frame_floats(B) * sizeof(float);
}

// Device bytes the lane holds: its codec's own count and its two slabs.
int64_t lane_bytes(const lic_server *s, const Lane *L) {
    const int64_t c = L->codec ? lic_codec_device_bytes(L->codec) : 0;
    return (c > 0 ? c : 0) + (L->in ? 2 * (int64_t)slab_bytes(s, L->bucket) : 0);
}

// Slabs, a first pass at the largest batch (every workspace reaches its
// final size), then one graph per batch size.
int make_lane(lic_server *s, Bucket *B, Lane *L) {
    int rc = LIC_OK;
    if (!L->codec && (rc = make_lane_codec(s, B, L))) return rc;
    const size_t bytes = slab_bytes(s, B);
    LIC_CUDA_TRY(cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking));
    LIC_CUDA_TRY(cudaMalloc(&L->in, bytes));
    LIC_CUDA_TRY(cudaMalloc(&L->out, bytes));
    LIC_CUDA_TRY(cudaMallocHost(&L->status_host, 16));
    LIC_CUDA_TRY(cudaMemsetAsync(L->in, 0, bytes, L->stream));
    if ((rc = chain(L, s->opt.max_batch))) return rc;
    LIC_CUDA_TRY(cudaStreamSynchronize(L->stream));
    if ((rc = status_code(*L->status_host))) return rc;
    if (s->opt.graphs) {
        L->graphs.assign(s->opt.max_batch, nullptr);
        for (int b = 1; b <= s->opt.max_batch; ++b) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) break;
            const int crc = chain(L, b);
            const cudaError_t e = cudaStreamEndCapture(L->stream, &g);
            if (crc || e != cudaSuccess || !g) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                L->graphs.assign(s->opt.max_batch, nullptr);   // this lane runs eagerly
                break;
            }
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                cudaGetLastError();
                L->graphs.assign(s->opt.max_batch, nullptr);
                break;
            }
            L->graphs[b - 1] = ex;
        }
    }
    return LIC_OK;
}

// Create the bucket of H x W frames (outside the server lock; prep_mu held).
// Admission by HBM budget: the first lane's codec is created (weights and
// tables), then the bucket's cost is estimated from the geometry -- per
// lane, those weights, the workspaces and one bitstream batch that
// encode + decode of max_batch frames reach (lic_codec_workspace_bytes), and
// the two frame slabs -- and checked against the budget before any
// workspace is allocated.  Once built, the bucket is charged what its lanes'
// codecs counted at each allocation plus the slabs: the device's free
// memory, which other users of the GPU move, enters neither figure.
int prepare_locked(lic_server *s, int H, int W) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->buckets.count({H, W})) return LIC_OK;
    }
    auto B = std::make_unique<Bucket>();
    B->H = H;
    B->W = W;
    int64_t held = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        held = s->st.device_bytes;
    }
    auto refuse = [&](int rc) {
        for (auto &L : B->lanes) destroy_lane(L.get());
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc == LIC_E_OOM) s->st.refused_budget += 1;
        return rc;
    };
    B->lanes.push_back(std::make_unique<Lane>());
    int rc = make_lane_codec(s, B.get(), B->lanes[0].get());
    if (rc) return refuse(rc);
    const int64_t ws = lic_codec_workspace_bytes(B->lanes[0]->codec, s->opt.max_batch, H, W);
    if (ws < 0) return refuse((int)ws);
    const int64_t per_lane = lic_codec_device_bytes(B->lanes[0]->codec) + ws + 2 * (int64_t)slab_bytes(s, B.get());
    if (held + (int64_t)s->opt.lanes * per_lane > s->opt.hbm_budget) return refuse(LIC_E_OOM);
    for (int l = 0; l < s->opt.lanes && !rc; ++l) {
        if (l > 0) B->lanes.push_back(std::make_unique<Lane>());
        rc = make_lane(s, B.get(), B->lanes[l].get());
    }
    if (rc) return refuse(rc);
    B->bytes = 0;
    for (auto &L : B->lanes) B->bytes += lane_bytes(s, L.get());
    if (held + B->bytes > s->opt.hbm_budget) return refuse(LIC_E_OOM);
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.device_bytes += B->bytes;
    s->st.buckets += 1;
    s->buckets[{H, W}] = std::move(B);
    return LIC_OK;
}

}  // namespace

extern "C" {

int lic_server_create(lic_kind kind, int N, int M, const lic_weights *weights, const lic_options *codec_opt,
                      const lic_server_options *opt, lic_server **out) {
    if (!weights || !opt || !out || !weights->params || weights->count < 1) return LIC_E_INVALID_ARG;
    *out = nullptr;
    if (opt->max_batch < 1 || opt->max_batch > 64 || opt->lanes < 1 || opt->lanes > 8 || opt->max_pending < 1 ||
        !(opt->max_wait_ms >= 0.0) || opt->hbm_budget <= 0 || (opt->graphs != 0 && opt->graphs != 1))
        return LIC_E_INVALID_ARG;
    for (int r : opt->reserved)
        if (r) return LIC_E_INVALID_ARG;
    if (kind != LIC_FACTORIZED && kind != LIC_HYPERPRIOR) return LIC_E_INVALID_ARG;
    for (int i = 0; i < weights->count; ++i)
        if (!weights->params[i].name || !weights->params[i].data || weights->params[i].numel < 0)
            return LIC_E_INVALID_ARG;
    auto s = new (std::nothrow) lic_server();
    if (!s) return LIC_E_OOM;
    s->kind = kind;
    s->N = N;
    s->M = M;
    if (codec_opt) {
        s->copt = *codec_opt;
        s->has_copt = true;
    }
    s->opt = *opt;
    for (int i = 0; i < weights->count; ++i) {
        s->names.emplace_back(weights->params[i].name);
        s->data.emplace_back(weights->params[i].data, weights->params[i].data + weights->params[i].numel);
    }
    cudaGetDevice(&s->device);
    s->t0 = Clock::now();
    s->dispatcher = std::thread(dispatch_loop, s);
    *out = s;
    return LIC_OK;
}

void lic_server_destroy(lic_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->work_cv.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    for (auto &kv : s->buckets)
        for (auto &L : kv.second->lanes) {
            if (L->stream) cudaStreamSynchronize(L->stream);
            destroy_lane(L.get());
        }
    delete s;
}

int lic_server_prepare(lic_server *s, int H, int W) {
    if (!s || H < 1 || W < 1) return LIC_E_INVALID_ARG;
    std::lock_guard<std::mutex> pk(s->prep_mu);
    return prepare_locked(s, H, W);
}

int lic_server_submit(lic_server *s, int stream_id, const float *frame, int H, int W, float *decoded,
                      uint64_t *ticket) {
    if (!s || !frame || H < 1 || W < 1) return LIC_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return LIC_E_INVALID_ARG;
        if (s->pending >= s->opt.max_pending) {
            s->st.refused_busy += 1;
            return LIC_E_BUSY;
        }
    }
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        have = s->buckets.count({H, W}) != 0;
    }
    if (!have) {
        const int rc = lic_server_prepare(s, H, W);
        if (rc) return rc;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->pending >= s->opt.max_pending) {
            s->st.refused_busy += 1;
            return LIC_E_BUSY;
        }
        Request r{s->next_ticket++, stream_id, frame, decoded, now_ms(s)};
        if (ticket) *ticket = r.ticket;
        s->buckets[{H, W}]->q.push_back(r);
        s->pending += 1;
        s->st.submitted += 1;
    }
    s->work_cv.notify_all();
    return LIC_OK;
}

int lic_server_poll(lic_server *s, lic_server_result *out, int cap, double wait_ms) {
    if (!s || cap < 0 || (cap > 0 && !out)) return LIC_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->done_cv.wait_for(lk, std::chrono::duration<double, std::milli>(wait_ms), [&] { return !s->done.empty(); });
    int n = 0;
    while (n < cap && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

int lic_server_drain(lic_server *s, double timeout_ms) {
    if (!s) return LIC_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->done_cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                        [&] { return s->pending == 0; });
    return ok ? LIC_OK : LIC_E_TIMEOUT;
}

int lic_server_stats_get(lic_server *s, lic_server_stats *out) {
    if (!s || !out) return LIC_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return LIC_OK;
}

double lic_server_clock_ms(lic_server *s) { return s ? now_ms(s) : -1.0; }

}  // extern "C"
