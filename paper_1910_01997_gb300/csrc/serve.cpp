// Serving loop: keyframe solves from many camera streams, continuously batched.
//
// Requests arrive from any host thread (sgn_server_submit only takes a lock).  A server thread owns
// every CUDA call: it admits queued requests when their plan workspace fits the free part of the
// caller's device arena (admission by free HBM), uploads and prepares their frames on the copy
// stream (overlapping the solve in flight), groups everything uploaded since the last launch into
// an epoch that runs as one persistent batch launch on the compute stream (requests that arrive
// while an epoch runs join the next one), copies each result back on the copy stream and stamps its
// latency (submit -> result in host memory).  Arena space is released when a request completes or
// is cancelled.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sgn.h"
#include "sgn_internal.h"

namespace sgn {
PlanParams plan_params(const sgn_plan* p);
void plan_mark_solved(sgn_plan* p);
}  // namespace sgn

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// First-fit allocator over [0, size) in kAlign units.
class Arena {
   public:
    void reset(size_t size) {
        free_.clear();
        free_.push_back({0, size});
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + sgn::kAlign - 1) / sgn::kAlign * sgn::kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                it->first += bytes;
                it->second -= bytes;
                if (it->second == 0) free_.erase(it);
                used_ += bytes;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + sgn::kAlign - 1) / sgn::kAlign * sgn::kAlign;
        used_ -= bytes;
        auto it = free_.begin();
        while (it != free_.end() && it->first < off) ++it;
        it = free_.insert(it, {off, bytes});
        if (it != free_.begin()) {  // merge with the previous block
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
                it = prev;
            }
        }
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
    }
    size_t used() const { return used_; }

   private:
    std::list<std::pair<size_t, size_t>> free_;
    size_t used_ = 0;
};

enum class Stage { Queued, Uploading, InEpoch, Reading, Done };

struct Job {
    sgn_request req;
    std::vector<const float*> frame_ptrs;
    std::vector<double> poses;
    Stage stage = Stage::Queued;
    bool cancelled = false;
    sgn_plan* plan = nullptr;
    size_t off = 0, bytes = 0;
    cudaEvent_t uploaded = nullptr, done = nullptr;
    int epoch = -1;
    Clock::time_point t_submit, t_admit;
    sgn_status result = SGN_OK;
    int overtaken = 0;       // later requests admitted while this one waited for arena memory
    uint64_t admit_seq = 0;  // admission order (1, 2, ...); 0 until admitted
};

// A request that does not fit the free arena yet lets at most this many later requests pass it;
// then nothing behind it is admitted until it fits (the requests in flight finish and free their
// memory), so that a large request cannot be starved by a stream of small ones.
constexpr int kMaxOvertake = 8;

struct Epoch {
    std::vector<Job*> jobs;
    cudaEvent_t done = nullptr;
    int slot = 0;  // device table buffer
};

}  // namespace

struct sgn_server {
    // configuration
    char* arena_base = nullptr;
    size_t arena_bytes = 0;
    int max_slots = 0;
    int chunk = 64;
    cudaStream_t compute = nullptr, copy = nullptr;
    int device = -1;
    // device tables (two buffers so that two epochs can be in flight)
    char* tables[2] = {nullptr, nullptr};
    size_t table_bytes = 0;
    int max_items = 0;
    int sms = 0;  // multiprocessors of the device (the launch grid is sms x resident blocks)
    uint64_t admitted = 0;  // requests admitted so far (server thread)
    bool table_busy[2] = {false, false};
    std::vector<sgn::PlanParams> h_plans;
    std::vector<sgn::WorkItem> h_items;
    // state shared with submitters
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> incoming;
    std::vector<sgn_completion> completed;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> pending{0};
    std::vector<uint64_t> cancel_tags;
    // owned by the server thread
    Arena arena;
    std::deque<Job*> queued;
    std::vector<Job*> uploading;
    std::deque<Epoch> epochs;
    std::vector<Job*> reading;
    std::thread worker;
    // statistics (under mu)
    std::vector<double> latencies;
    uint64_t residuals_done = 0, completed_count = 0, epochs_launched = 0, rejected = 0, admission_waits = 0;
    size_t peak_arena = 0;
    Clock::time_point t_first, t_last;
    bool have_first = false;
    std::string error;
};

namespace {

sgn_status srv_error(sgn_status st, const std::string& m) { return sgn::record_error(st, m.c_str()); }

bool event_done(cudaEvent_t e) {
    const cudaError_t r = cudaEventQuery(e);
    if (r == cudaErrorNotReady) return false;
    return true;  // done, or an error that the completion path reports
}

void finish_job(sgn_server* s, Job* j, sgn_status st) {
    const auto now = Clock::now();
    const double lat = ms_between(j->t_submit, now);
    if (j->plan) sgn_plan_destroy(j->plan);
    j->plan = nullptr;
    if (j->bytes) s->arena.release(j->off, j->bytes);
    j->bytes = 0;
    if (j->uploaded) cudaEventDestroy(j->uploaded);
    if (j->done) cudaEventDestroy(j->done);
    j->uploaded = j->done = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        sgn_completion c{};
        c.tag = j->req.tag;
        c.status = j->cancelled ? SGN_ERR_STATE : st;
        c.latency_ms = lat;
        c.queue_ms = ms_between(j->t_submit, j->t_admit.time_since_epoch().count() ? j->t_admit : now);
        c.admit_seq = j->admit_seq;
        c.cancelled = j->cancelled ? 1 : 0;
        s->completed.push_back(c);
        if (!j->cancelled && st == SGN_OK) {
            s->latencies.push_back(lat);
            const sgn_plan_desc& d = j->req.desc;
            s->residuals_done += uint64_t(d.width / d.patch) * (d.height / d.patch) * d.patch * d.patch *
                                 uint64_t(j->req.num_frames) * uint64_t(j->req.iters);
            s->completed_count++;
            if (!s->have_first) {
                s->t_first = j->t_submit;
                s->have_first = true;
            }
            s->t_last = now;
        }
    }
    s->pending.fetch_sub(1);
    s->cv.notify_all();
    delete j;
}

// Create the request's plan in its arena slot and enqueue its uploads on the copy stream.
sgn_status start_upload(sgn_server* s, Job* j) {
    const sgn_request& r = j->req;
    sgn_status st = sgn_plan_create(&r.desc, &j->plan);
    if (st != SGN_OK) return st;
    if ((st = sgn_plan_bind(j->plan, s->arena_base + j->off, j->bytes, s->copy)) != SGN_OK) return st;
    if ((st = sgn_set_intrinsics(j->plan, r.intrinsics[0], r.intrinsics[1], r.intrinsics[2], r.intrinsics[3])) != SGN_OK)
        return st;
    const size_t pitch = size_t(r.desc.width) * sizeof(float);
    if ((st = sgn_set_keyframe(j->plan, r.keyframe, pitch, SGN_HOST)) != SGN_OK) return st;
    if ((st = sgn_set_frames(j->plan, r.num_frames, j->frame_ptrs.data(), pitch, SGN_HOST, j->poses.data())) != SGN_OK)
        return st;
    if ((st = sgn_init_surfels(j->plan, r.inv_depth0, r.normal0, r.state0, SGN_HOST)) != SGN_OK) return st;
    if (cudaEventCreateWithFlags(&j->uploaded, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(j->uploaded, s->copy) != cudaSuccess)
        return srv_error(SGN_ERR_CUDA, "server: upload event");
    j->stage = Stage::Uploading;
    return SGN_OK;
}

// One persistent batch launch over the jobs on the compute stream, after their uploads.
sgn_status launch_epoch(sgn_server* s, std::vector<Job*>& jobs, Epoch* ep) {
    int slot = s->table_busy[0] ? 1 : 0;
    s->h_plans.clear();
    s->h_items.clear();
    for (size_t i = 0; i < jobs.size(); ++i) {
        Job* j = jobs[i];
        s->h_plans.push_back(sgn::plan_params(j->plan));
        const int S = s->h_plans.back().S;
        for (int f = 0; f < S; f += s->chunk) s->h_items.push_back(sgn::WorkItem{int(i), f, std::min(s->chunk, S - f), 0});
        if (cudaStreamWaitEvent(s->compute, j->uploaded, 0) != cudaSuccess) return srv_error(SGN_ERR_CUDA, "server: wait upload");
    }
    std::stable_sort(s->h_items.begin(), s->h_items.end(), [&](const sgn::WorkItem& a, const sgn::WorkItem& b) {
        const sgn::PlanParams& pa = s->h_plans[a.plan];
        const sgn::PlanParams& pb = s->h_plans[b.plan];
        if (sgn::batch_kind(pa) != sgn::batch_kind(pb)) return sgn::batch_kind(pa) < sgn::batch_kind(pb);  // one launch per kind
        if (pa.P != pb.P) return pa.P > pb.P;  // one solver variant at a time (see the batch work list)
        return double(a.count) * pa.P * pa.P * pa.F > double(b.count) * pb.P * pb.P * pb.F;
    });
    if (int(s->h_items.size()) > s->max_items) return srv_error(SGN_ERR_ADMISSION, "server: work list overflow");
    char* base = s->tables[slot];
    const size_t plans_bytes = size_t(s->max_slots) * sizeof(sgn::PlanParams);
    char* items = base + plans_bytes;
    int* counter = reinterpret_cast<int*>(items + size_t(s->max_items) * sizeof(sgn::WorkItem));
    if (cudaMemcpyAsync(base, s->h_plans.data(), s->h_plans.size() * sizeof(sgn::PlanParams), cudaMemcpyHostToDevice,
                        s->compute) != cudaSuccess ||
        cudaMemcpyAsync(items, s->h_items.data(), s->h_items.size() * sizeof(sgn::WorkItem), cudaMemcpyHostToDevice,
                        s->compute) != cudaSuccess)
        return srv_error(SGN_ERR_CUDA, "server: table upload");
    int fmax = 1;
    for (const sgn::PlanParams& pp : s->h_plans) fmax = std::max(fmax, pp.F);
    // one persistent launch per solver kind present (items sorted by kind), each with its own counter
    int begin = 0;
    for (int k = 0; k < sgn::kBatchKinds; ++k) {
        int end = begin;
        while (end < int(s->h_items.size()) && sgn::batch_kind(s->h_plans[s->h_items[end].plan]) == k) ++end;
        if (end == begin) continue;
        const int grid = s->sms * std::max(1, sgn::batch_blocks_per_sm(k, 0, 256, fmax));
        const int le = sgn::launch_gn_batch(k, reinterpret_cast<const sgn::PlanParams*>(base),
                                            reinterpret_cast<const sgn::WorkItem*>(items) + begin, end - begin, counter + k,
                                            jobs[0]->req.iters, 0, grid, 256, fmax, s->compute);
        if (le) return srv_error(SGN_ERR_CUDA, std::string("server: batch launch: ") + cudaGetErrorString(cudaError_t(le)));
        sgn::count_launch();
        begin = end;
    }
    if (cudaEventCreateWithFlags(&ep->done, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ep->done, s->compute) != cudaSuccess)
        return srv_error(SGN_ERR_CUDA, "server: epoch event");
    ep->jobs = jobs;
    ep->slot = slot;
    s->table_busy[slot] = true;
    for (Job* j : jobs) {
        j->stage = Stage::InEpoch;
        sgn::plan_mark_solved(j->plan);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->epochs_launched++;
    return SGN_OK;
}

// Enqueue the result copies of a finished epoch's job on the copy stream.
sgn_status start_read(sgn_server* s, Job* j, cudaEvent_t epoch_done) {
    const sgn_request& r = j->req;
    if (cudaStreamWaitEvent(s->copy, epoch_done, 0) != cudaSuccess) return srv_error(SGN_ERR_CUDA, "server: wait epoch");
    sgn_status st = sgn_read_surfels(j->plan, r.inv_depth, r.normal, r.cost, r.nres, r.status, SGN_HOST);
    if (st != SGN_OK) return st;
    if (cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(j->done, s->copy) != cudaSuccess)
        return srv_error(SGN_ERR_CUDA, "server: read event");
    j->stage = Stage::Reading;
    return SGN_OK;
}

void server_loop(sgn_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        bool idle = true;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (!s->incoming.empty()) {
                s->queued.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
            for (uint64_t tag : s->cancel_tags) {
                for (Job* j : s->queued)
                    if (j->req.tag == tag) j->cancelled = true;
                for (Job* j : s->uploading)
                    if (j->req.tag == tag) j->cancelled = true;
                for (Epoch& ep : s->epochs)
                    for (Job* j : ep.jobs)
                        if (j->req.tag == tag) j->cancelled = true;
                for (Job* j : s->reading)
                    if (j->req.tag == tag) j->cancelled = true;
            }
            s->cancel_tags.clear();
            if (s->stop.load() && s->queued.empty() && s->uploading.empty() && s->epochs.empty() && s->reading.empty())
                break;
        }
        // cancelled before admission: complete immediately
        for (auto it = s->queued.begin(); it != s->queued.end();) {
            if ((*it)->cancelled) {
                finish_job(s, *it, SGN_ERR_STATE);
                it = s->queued.erase(it);
                idle = false;
            } else {
                ++it;
            }
        }
        // admission: FIFO; a later request may pass one that does not fit yet, at most kMaxOvertake
        // times per waiting request, after which admission stops at that request until it fits
        std::vector<Job*> waiting;
        for (auto it = s->queued.begin(); it != s->queued.end();) {
            Job* j = *it;
            if (!s->arena.alloc(j->bytes, &j->off)) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->admission_waits++;
                }
                if (j->overtaken >= kMaxOvertake) break;
                waiting.push_back(j);
                ++it;
                continue;
            }
            for (Job* w : waiting) ++w->overtaken;
            j->admit_seq = ++s->admitted;
            j->t_admit = Clock::now();
            sgn_status st = start_upload(s, j);
            it = s->queued.erase(it);
            idle = false;
            if (st != SGN_OK) {
                finish_job(s, j, st);
                continue;
            }
            s->uploading.push_back(j);
            std::lock_guard<std::mutex> lk(s->mu);
            s->peak_arena = std::max(s->peak_arena, s->arena.used());
        }
        // epochs: everything uploaded so far runs in the next launch (at most two in flight)
        if (!s->uploading.empty() && int(s->epochs.size()) < 2 && !(s->table_busy[0] && s->table_busy[1])) {
            std::vector<Job*> ready;
            int items = 0;
            for (auto it = s->uploading.begin(); it != s->uploading.end();) {
                const sgn::PlanParams pp = sgn::plan_params((*it)->plan);
                const int n = (pp.S + s->chunk - 1) / s->chunk;
                if (int(ready.size()) >= s->max_slots || items + n > s->max_items ||
                    (!ready.empty() && (*it)->req.iters != ready[0]->req.iters)) {
                    ++it;
                    continue;
                }
                items += n;
                ready.push_back(*it);
                it = s->uploading.erase(it);
            }
            if (!ready.empty()) {
                s->epochs.emplace_back();
                sgn_status st = launch_epoch(s, ready, &s->epochs.back());
                idle = false;
                if (st != SGN_OK) {
                    s->epochs.pop_back();
                    for (Job* j : ready) finish_job(s, j, st);
                }
            }
        }
        // finished epochs: queue the result copies
        while (!s->epochs.empty() && event_done(s->epochs.front().done)) {
            Epoch ep = s->epochs.front();
            s->epochs.pop_front();
            const cudaError_t e = cudaEventQuery(ep.done);
            for (Job* j : ep.jobs) {
                sgn_status st = e == cudaSuccess ? start_read(s, j, ep.done) : srv_error(SGN_ERR_CUDA, "server: epoch failed");
                if (st != SGN_OK) {
                    finish_job(s, j, st);
                    continue;
                }
                s->reading.push_back(j);
            }
            s->table_busy[ep.slot] = false;
            cudaEventDestroy(ep.done);
            idle = false;
        }
        // finished reads: complete
        for (auto it = s->reading.begin(); it != s->reading.end();) {
            if (event_done((*it)->done)) {
                const cudaError_t e = cudaEventQuery((*it)->done);
                finish_job(s, *it, e == cudaSuccess ? SGN_OK : SGN_ERR_CUDA);
                it = s->reading.erase(it);
                idle = false;
            } else {
                ++it;
            }
        }
        if (idle) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace

extern "C" {

sgn_status sgn_server_create(void* d_arena, size_t arena_bytes, int max_slots, int max_surfels_per_epoch,
                             void* compute_stream, void* copy_stream, sgn_server** out) {
    if (!out || !d_arena) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: arena/out is NULL");
    *out = nullptr;
    if (reinterpret_cast<uintptr_t>(d_arena) % sgn::kAlign) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: arena must be 256-byte aligned");
    if (max_slots < 1 || max_slots > 4096) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: max_slots outside [1, 4096]");
    if (max_surfels_per_epoch < 1) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: max_surfels_per_epoch < 1");
    if (!compute_stream || !copy_stream || compute_stream == copy_stream)
        return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: needs two distinct non-default streams");
    sgn_server* s = new sgn_server();
    s->max_slots = max_slots;
    s->max_items = max_surfels_per_epoch / s->chunk + max_slots;
    s->table_bytes = (size_t(max_slots) * sizeof(sgn::PlanParams) + size_t(s->max_items) * sizeof(sgn::WorkItem) +
                      sgn::kBatchKinds * sizeof(int) + sgn::kAlign - 1) / sgn::kAlign * sgn::kAlign;
    if (arena_bytes < 4 * s->table_bytes) {
        delete s;
        return srv_error(SGN_ERR_WORKSPACE_TOO_SMALL, "server: arena too small for its launch tables");
    }
    s->arena_base = static_cast<char*>(d_arena);
    s->tables[0] = s->arena_base;
    s->tables[1] = s->arena_base + s->table_bytes;
    s->arena_base += 2 * s->table_bytes;
    s->arena_bytes = arena_bytes - 2 * s->table_bytes;
    s->arena.reset(s->arena_bytes);
    s->compute = static_cast<cudaStream_t>(compute_stream);
    s->copy = static_cast<cudaStream_t>(copy_stream);
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return srv_error(SGN_ERR_CUDA, "server: cudaGetDevice");
    }
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    s->worker = std::thread(server_loop, s);
    *out = s;
    return SGN_OK;
}

sgn_status sgn_server_submit(sgn_server* s, const sgn_request* r) {
    if (!s || !r) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: NULL argument");
    const sgn_plan_desc& d = r->desc;
    sgn_plan* probe = nullptr;
    sgn_status st = sgn_plan_create(&d, &probe);  // validates the description
    if (st != SGN_OK) return st;
    size_t bytes = 0;
    sgn_plan_workspace_bytes(probe, &bytes);
    sgn_plan_destroy(probe);
    if (r->num_frames < 1 || r->num_frames > d.max_frames || !r->frames || !r->poses || !r->keyframe || !r->inv_depth0 ||
        !r->normal0 || !r->state0 || r->iters < 0 || r->iters > 100000)
        return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: incomplete request");
    if (bytes > s->arena_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->rejected++;
        return srv_error(SGN_ERR_ADMISSION, "server: request needs more device memory than the whole arena");
    }
    if (s->stop.load()) return srv_error(SGN_ERR_STATE, "server: shutting down");
    Job* j = new Job();
    j->req = *r;
    j->frame_ptrs.assign(r->frames, r->frames + r->num_frames);
    j->poses.assign(r->poses, r->poses + 12 * r->num_frames);
    j->req.frames = nullptr;
    j->req.poses = nullptr;
    j->bytes = bytes;
    j->t_submit = Clock::now();
    s->pending.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->incoming.push_back(j);
    }
    s->cv.notify_all();
    return SGN_OK;
}

sgn_status sgn_server_cancel(sgn_server* s, uint64_t tag) {
    if (!s) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    for (Job* j : s->incoming)
        if (j->req.tag == tag) j->cancelled = true;
    s->cancel_tags.push_back(tag);
    s->cv.notify_all();
    return SGN_OK;
}

sgn_status sgn_server_poll(sgn_server* s, sgn_completion* out, int max, int* n) {
    if (!s || !n || (max > 0 && !out)) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const int k = std::min<int>(max, int(s->completed.size()));
    for (int i = 0; i < k; ++i) out[i] = s->completed[i];
    s->completed.erase(s->completed.begin(), s->completed.begin() + k);
    *n = k;
    return SGN_OK;
}

sgn_status sgn_server_drain(sgn_server* s, uint64_t timeout_ns) {
    if (!s) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server is NULL");
    const auto t0 = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    while (s->pending.load() > 0) {
        if (timeout_ns && uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count()) >= timeout_ns)
            return srv_error(SGN_ERR_TIMEOUT, "server: drain deadline passed");
        s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    return SGN_OK;
}

sgn_status sgn_server_stats(sgn_server* s, sgn_serving_stats* out) {
    if (!s || !out) return srv_error(SGN_ERR_INVALID_ARGUMENT, "server: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->completed = s->completed_count;
    out->epochs = s->epochs_launched;
    out->rejected = s->rejected;
    out->admission_waits = s->admission_waits;
    out->peak_arena_bytes = s->peak_arena;
    out->residuals = s->residuals_done;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, size_t(f * (v.size() - 1) + 0.5))]; };
        out->latency_p50_ms = q(0.50);
        out->latency_p99_ms = q(0.99);
        out->latency_max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->latency_mean_ms = sum / v.size();
        out->busy_seconds = ms_between(s->t_first, s->t_last) / 1e3;
    }
    return SGN_OK;
}

sgn_status sgn_server_destroy(sgn_server* s) {
    if (!s) return SGN_OK;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return SGN_OK;
}

}  // extern "C"
