// Serving loop: render requests from many simulated agents against one scene
// kept resident on the device (the simulator's agents render views while they
// walk, Sec. IV-B data collection).
//
// Continuous batching: a worker thread owns `lanes` render lanes, each a
// stream with its own work buffers over the shared scene. Whenever a lane is
// free it admits the oldest waiting requests, as many as fit its sort-buffer
// budget (estimated (tile, Gaussian) pairs, pixels x pairs-per-pixel) and its
// camera limit, and launches them as one batched render. Requests that arrive
// while the other lanes are busy join the next launch, and the launches of
// different lanes overlap on the device. A request completes when its lane's
// completion event fires; its latency is measured from submission.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "ngs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    ngs_camera cam;
    float *image;
    Clock::time_point t_submit;
    int tries = 0;       // launches that overflowed a work buffer with this request
};

// launches a request may take part in that overflow a work buffer before it
// is failed (each overflow re-plans the lane from the counted pairs)
constexpr int kMaxCapacityRetries = 3;

struct Lane {
    ngs_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request> reqs;
};

}  // namespace

struct ngs_server {
    ngs_ctx *parent = nullptr;
    int device = 0;
    ngs_server_config cfg{};
    std::vector<Lane> lanes;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    bool stop = false;
    uint64_t next_ticket = 1;
    // completion records, indexed by ticket - 1: 0 pending, 1 done, 2 failed
    std::vector<uint8_t> state;
    std::vector<float> latency_ms;
    int64_t submitted = 0, completed = 0, failed = 0, launches = 0, requeued = 0;
    double mpix = 0.0;
    Clock::time_point t_first, t_last;
    bool any = false;
    ngs_status worker_error = NGS_OK;
};

namespace {

double pixels_of(const ngs_camera &c) { return (double)c.width * (double)c.height; }

void finish_lane(ngs_server *s, Lane &l) {
    const ngs_status st = ngs_synchronize(l.ctx, l.stream);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    if (st == NGS_ERR_CAPACITY) {
        // the launch overflowed a work buffer: the lane's planner has taken the
        // pair densities the device counted, admission follows it, and the
        // requests go back to the front of the queue in their order
        s->cfg.pairs_per_pixel = std::max(s->cfg.pairs_per_pixel, ngs::ctx_pairs_per_pixel(l.ctx));
        for (auto it = l.reqs.rbegin(); it != l.reqs.rend(); ++it) {
            Request r = *it;
            if (++r.tries > kMaxCapacityRetries) {
                s->state[(size_t)(r.ticket - 1)] = 2;
                ++s->failed;
            } else {
                s->pending.push_front(r);
                ++s->requeued;
            }
        }
        l.reqs.clear();
        l.busy = false;
        s->cv.notify_all();
        return;
    }
    for (const Request &r : l.reqs) {
        const size_t i = (size_t)(r.ticket - 1);
        if (st == NGS_OK) {
            s->state[i] = 1;
            s->latency_ms[i] =
                (float)std::chrono::duration<double, std::milli>(now - r.t_submit).count();
            ++s->completed;
            s->mpix += pixels_of(r.cam) * 1e-6;
        } else {
            s->state[i] = 2;
            ++s->failed;
        }
    }
    s->t_last = now;
    l.reqs.clear();
    l.busy = false;
    s->cv.notify_all();
}

void launch_lane(ngs_server *s, Lane &l) {
    // admission: oldest first, within the camera limit and the pair budget
    {
        std::lock_guard<std::mutex> lock(s->mu);
        double budget = 0.0;
        while (!s->pending.empty() && (int)l.reqs.size() < s->cfg.max_cams) {
            const Request &r = s->pending.front();
            const double est = s->cfg.pairs_per_pixel * pixels_of(r.cam);
            if (!l.reqs.empty() && budget + est > (double)s->cfg.pair_budget) break;
            budget += est;
            l.reqs.push_back(r);
            s->pending.pop_front();
        }
    }
    if (l.reqs.empty()) return;
    std::vector<ngs_camera> cams(l.reqs.size());
    std::vector<float *> imgs(l.reqs.size());
    for (size_t i = 0; i < l.reqs.size(); ++i) {
        cams[i] = l.reqs[i].cam;
        imgs[i] = l.reqs[i].image;
    }
    ngs_status st = ngs_render(l.ctx, cams.data(), (int32_t)cams.size(), imgs.data(), l.stream);
    if (st != NGS_OK) {
        std::lock_guard<std::mutex> lock(s->mu);
        for (const Request &r : l.reqs) {
            s->state[(size_t)(r.ticket - 1)] = 2;
            ++s->failed;
        }
        l.reqs.clear();
        s->cv.notify_all();
        return;
    }
    cudaEventRecord(l.done, l.stream);
    l.busy = true;
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->launches;
}

void worker_main(ngs_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        for (Lane &l : s->lanes) {
            if (l.busy && cudaEventQuery(l.done) == cudaSuccess) {
                finish_lane(s, l);
                progressed = true;
            }
        }
        for (Lane &l : s->lanes) {
            if (!l.busy) {
                launch_lane(s, l);
                progressed |= l.busy;
            }
        }
        std::unique_lock<std::mutex> lock(s->mu);
        bool idle = true;
        for (const Lane &l : s->lanes) idle = idle && !l.busy;
        if (s->stop && s->pending.empty() && idle) break;
        if (!progressed) {
            if (idle && s->pending.empty())
                s->cv.wait_for(lock, std::chrono::milliseconds(2));
            else
                s->cv.wait_for(lock, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" {

NGS_API ngs_status ngs_server_start(ngs_ctx *ctx, const ngs_server_config *cfg,
                                    ngs_server **out) {
    if (!ctx || !out) return NGS_ERR_INVALID_ARG;
    *out = nullptr;
    ngs_server_config c{};
    if (cfg) c = *cfg;
    if (c.lanes <= 0) c.lanes = 2;
    if (c.max_cams <= 0) c.max_cams = 64;
    if (c.pairs_per_pixel <= 0) c.pairs_per_pixel = 48.0;
    if (c.lanes > 8 || c.max_cams > 1024) return NGS_ERR_INVALID_ARG;
    ngs_server *s = new ngs_server();
    s->parent = ctx;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return NGS_ERR_CUDA;
    }
    s->lanes.resize(c.lanes);
    for (Lane &l : s->lanes) {
        ngs_status st = ngs::lane_create(ctx, c.lane_record_capacity, c.lane_pair_capacity, &l.ctx);
        if (st == NGS_OK && (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
                             cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess))
            st = NGS_ERR_CUDA;
        if (st != NGS_OK) {
            s->cfg = c;
            ngs_server_stop(s);
            return st;
        }
    }
    if (c.pair_budget <= 0) c.pair_budget = (int64_t)1 << 29;
    s->cfg = c;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return NGS_OK;
}

NGS_API ngs_status ngs_server_submit(ngs_server *s, const ngs_camera *cam, float *d_image,
                                     uint64_t *ticket) {
    if (!s || !cam || !d_image || !ticket) return NGS_ERR_INVALID_ARG;
    if (cam->width <= 0 || cam->height <= 0 || !(cam->fx > 0) || !(cam->fy > 0) || cam->tau < 0)
        return NGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return NGS_ERR_INVALID_ARG;
    Request r{s->next_ticket++, *cam, d_image, Clock::now(), 0};
    if (!s->any) {
        s->t_first = r.t_submit;
        s->any = true;
    }
    s->state.push_back(0);
    s->latency_ms.push_back(0.f);
    s->pending.push_back(r);
    ++s->submitted;
    *ticket = r.ticket;
    s->cv.notify_all();
    return NGS_OK;
}

NGS_API ngs_status ngs_server_poll(ngs_server *s, uint64_t ticket, int32_t *done,
                                   double *latency_ms) {
    if (!s || !done) return NGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return NGS_ERR_INVALID_ARG;
    const uint8_t st = s->state[(size_t)(ticket - 1)];
    *done = st != 0;
    if (latency_ms) *latency_ms = s->latency_ms[(size_t)(ticket - 1)];
    return st == 2 ? NGS_ERR_CUDA : NGS_OK;
}

NGS_API ngs_status ngs_server_wait_all(ngs_server *s, int32_t timeout_ms) {
    if (!s) return NGS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    const auto until = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (s->completed + s->failed < s->submitted) {
        if (s->cv.wait_until(lock, until) == std::cv_status::timeout &&
            s->completed + s->failed < s->submitted)
            return NGS_ERR_DEVICE_TIMEOUT;
    }
    return s->failed ? NGS_ERR_CUDA : NGS_OK;
}

NGS_API ngs_status ngs_server_stats(ngs_server *s, ngs_serving_stats *out) {
    if (!s || !out) return NGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    std::vector<float> lat;
    lat.reserve((size_t)s->completed);
    for (size_t i = 0; i < s->state.size(); ++i)
        if (s->state[i] == 1) lat.push_back(s->latency_ms[i]);
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) -> double {
        if (lat.empty()) return 0.0;
        const size_t k = (size_t)std::min<double>(lat.size() - 1, p * (lat.size() - 1) + 0.5);
        return lat[k];
    };
    double sum = 0.0;
    for (float v : lat) sum += v;
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->launches = s->launches;
    out->requeued = s->requeued;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->mean_ms = lat.empty() ? 0.0 : sum / lat.size();
    out->max_ms = lat.empty() ? 0.0 : lat.back();
    out->mpix = s->mpix;
    out->span_s = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    return NGS_OK;
}

NGS_API ngs_status ngs_server_stop(ngs_server *s) {
    if (!s) return NGS_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Lane &l : s->lanes) {
        if (l.stream) cudaStreamSynchronize(l.stream);
        if (l.done) cudaEventDestroy(l.done);
        if (l.stream) cudaStreamDestroy(l.stream);
        if (l.ctx) ngs_destroy(l.ctx);
    }
    delete s;
    return NGS_OK;
}

}  // extern "C"
