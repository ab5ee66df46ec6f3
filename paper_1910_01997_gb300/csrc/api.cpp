// Host runtime behind the C ABI of include/sgn.h: argument validation, workspace layout, uploads,
// kernel launches, synchronisation, checkpoints and batches.  No device memory is allocated here.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "sgn.h"
#include "sgn_internal.h"

using sgn::PlanParams;
using sgn::WorkItem;

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

sgn_status fail(sgn_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

sgn_status cuda_fail(int err, const char* what) {
    return fail(SGN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(static_cast<cudaError_t>(err)));
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Makes the plan's device current for the duration of a call and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (dev < 0) return;
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct Layout {
    size_t kf, tex, raw, id0, n0, state0, id, n, cost, nres, status, depth, sidx, disc, zbuf, total;
    int kf_pitch, tex_pitch, raw_pitch;
    long long tex_plane, raw_plane;
};

Layout make_layout(const sgn_plan_desc& d, int S, int disc_n) {
    Layout L{};
    const size_t W = size_t(d.width), H = size_t(d.height);
    L.kf_pitch = int(round_up(W, 64));
    L.tex_pitch = int(round_up(W, 32));
    L.raw_pitch = int(round_up(W, 64));
    L.tex_plane = (long long)H * L.tex_pitch;
    L.raw_plane = (long long)H * L.raw_pitch;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = round_up(off + bytes, sgn::kAlign);
        return o;
    };
    L.kf = take(H * L.kf_pitch * sizeof(float));
    L.tex = take(size_t(d.max_frames) * L.tex_plane * sgn::texel_bytes(d.image_dtype));
    L.raw = take(size_t(d.max_frames) * L.raw_plane * sizeof(float));
    L.id0 = take(size_t(S) * sizeof(float));
    L.n0 = take(size_t(S) * 3 * sizeof(float));
    L.state0 = take(size_t(S));
    L.id = take(size_t(S) * sizeof(float));
    L.n = take(size_t(S) * 3 * sizeof(float));
    L.cost = take(size_t(S) * sizeof(float));
    L.nres = take(size_t(S) * sizeof(int32_t));
    L.status = take(size_t(S));
    L.depth = take(W * H * sizeof(float));
    L.sidx = take(W * H * sizeof(int32_t));
    if (disc_n > 0) {  // circular surfels: pixel table and the depth buffer of the disc render
        L.disc = take(size_t(disc_n) * 2 * sizeof(int));
        L.zbuf = take(W * H * sizeof(unsigned long long));
    }
    L.total = off;
    return L;
}

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

sgn_status check_pose(const double* T) {
    if (!T) return fail(SGN_ERR_INVALID_ARGUMENT, "pose pointer is NULL");
    if (!finite_all(T, 12)) return fail(SGN_ERR_INVALID_ARGUMENT, "pose has non-finite entries");
    double worst = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d = 0.0;
            for (int k = 0; k < 3; ++k) d += T[4 * k + i] * T[4 * k + j];
            worst = std::max(worst, std::fabs(d - (i == j ? 1.0 : 0.0)));
        }
    const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                       T[2] * (T[4] * T[9] - T[5] * T[8]);
    if (worst > 1e-6 || det <= 0.0) return fail(SGN_ERR_INVALID_ARGUMENT, "pose rotation is not a rotation (|R^T R - I| = %g, det = %g)", worst, det);
    return SGN_OK;
}

}  // namespace

namespace sgn {
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
sgn_status record_error(sgn_status st, const char* message) {
    g_last_error = message;
    return st;
}
}  // namespace sgn

struct sgn_plan {
    sgn_plan_desc desc{};
    int TX = 0, TY = 0, S = 0;
    Layout L{};
    bool have_K = false;
    double fx = 0, fy = 0, cx = 0, cy = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
    cudaEvent_t done = nullptr;
    bool kf_set = false;
    bool frame_set[sgn::kMaxFrames] = {};
    double T[sgn::kMaxFrames][12] = {};
    int F = 0;
    bool surfels_set = false;
    bool state_pending = false;  // initial surfels uploaded, working state not derived yet
    bool depth_valid = false;
    int lanes = 0, block = 256;
    std::vector<int> disc;                // circular surfels: pixel offsets (x, y) from the tile origin
    bool staging = false;                 // stage texel boxes in shared memory (TMA)
    alignas(64) unsigned char tmap[sgn::kTensorMapBytes] = {};
    bool tmap_ok = false;                 // tmap describes the bound workspace's texel planes
};

struct sgn_batch {
    int max_plans = 0;
    std::vector<sgn_plan*> plans;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
    int variant = 0;
    int chunk = 64;
    bool dirty = true;
    int n_items = 0;
    int kind_begin[sgn::kBatchKinds + 1] = {0, 0, 0, 0};  // work-list range of each solver kind
    std::vector<PlanParams> h_plans;
    std::vector<WorkItem> h_items;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_iters = -1;
    int graph_grid = 0;  // blocks of the fixed-damping launch
    int graph_frames = 0;  // largest frame count the captured launch sizes its scratch for
    cudaEvent_t done = nullptr;
    std::vector<cudaEvent_t> plan_events;
};

namespace {

int default_lanes(int P) { return P == 4 ? 8 : (P == 8 ? 16 : 32); }

bool mapping_supported(int P, int G) {
    return (P == 4 && (G == 8 || G == 16)) || (P == 8 && (G == 8 || G == 16 || G == 32)) || (P == 16 && G == 32);
}

PlanParams make_params(const sgn_plan* p) {
    PlanParams pp{};
    const sgn_plan_desc& d = p->desc;
    pp.W = d.width;
    pp.H = d.height;
    pp.P = d.patch;
    pp.TX = p->TX;
    pp.TY = p->TY;
    pp.S = p->S;
    pp.F = p->F;
    pp.dtype = d.image_dtype;
    pp.fx = float(p->fx);
    pp.fy = float(p->fy);
    pp.cx = float(p->cx);
    pp.cy = float(p->cy);
    pp.fx_lo = float(p->fx - double(pp.fx));
    pp.fy_lo = float(p->fy - double(pp.fy));
    pp.cx_lo = float(p->cx - double(pp.cx));
    pp.cy_lo = float(p->cy - double(pp.cy));
    pp.ifx = float(1.0 / p->fx);
    pp.ify = float(1.0 / p->fy);
    pp.huber_k = d.huber_k;
    pp.lm_lambda = d.lm_lambda;
    pp.fp64_cond = d.fp64_cond > 0 ? float(std::min(d.fp64_cond, 3.0e38)) : 0.0f;
    pp.optimize_normal = d.optimize_normal;
    pp.min_residuals = d.min_residuals;
    pp.lm_adaptive = d.lm_adaptive;
    char* b = p->ws;
    const Layout& L = p->L;
    pp.kf = reinterpret_cast<const float*>(b + L.kf);
    pp.kf_pitch = L.kf_pitch;
    pp.tex = b + L.tex;
    pp.tex_pitch = L.tex_pitch;
    pp.tex_plane = L.tex_plane;
    pp.id0 = reinterpret_cast<const float*>(b + L.id0);
    pp.n0 = reinterpret_cast<const float*>(b + L.n0);
    pp.state0 = reinterpret_cast<const uint8_t*>(b + L.state0);
    pp.id = reinterpret_cast<float*>(b + L.id);
    pp.n = reinterpret_cast<float*>(b + L.n);
    pp.cost = reinterpret_cast<float*>(b + L.cost);
    pp.nres = reinterpret_cast<int32_t*>(b + L.nres);
    pp.status = reinterpret_cast<uint8_t*>(b + L.status);
    pp.depth = reinterpret_cast<float*>(b + L.depth);
    pp.sidx = reinterpret_cast<int32_t*>(b + L.sidx);
    pp.stage_err = sgn::stage_error_word();
    pp.radius = d.surfel_radius;
    pp.disc_n = int(p->disc.size() / 2);
    pp.disc = pp.disc_n ? reinterpret_cast<const int*>(b + L.disc) : nullptr;
    pp.zbuf = pp.disc_n ? reinterpret_cast<unsigned long long*>(b + L.zbuf) : nullptr;
    for (int f = 0; f < p->F; ++f) {
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                const double v = p->T[f][4 * i + j];
                pp.frames[f].R[3 * i + j] = float(v);
                pp.frames[f].R_lo[3 * i + j] = float(v - double(float(v)));
            }
            const double v = p->T[f][4 * i + 3];
            pp.frames[f].t[i] = float(v);
            pp.frames[f].t_lo[i] = float(v - double(float(v)));
        }
    }
    return pp;
}

sgn_status require_bound(const sgn_plan* p) {
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    if (!p->ws) return fail(SGN_ERR_NOT_BOUND, "plan has no workspace; call sgn_plan_bind first");
    return SGN_OK;
}

sgn_status require_ready(const sgn_plan* p) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (!p->have_K) return fail(SGN_ERR_STATE, "intrinsics not set");
    if (!p->kf_set) return fail(SGN_ERR_STATE, "keyframe not set");
    if (p->F < 1) return fail(SGN_ERR_STATE, "no frames in use; call sgn_set_frame(s) / sgn_set_num_frames");
    for (int f = 0; f < p->F; ++f)
        if (!p->frame_set[f]) return fail(SGN_ERR_STATE, "frame slot %d in use but not set", f);
    if (!p->surfels_set) return fail(SGN_ERR_STATE, "surfels not initialised");
    return SGN_OK;
}

// The square tile mapping of plain launches covers every tile exactly once (checked at compile
// time on ragged tile grids for every block shape).
constexpr bool square_mapping_is_bijective(int TX, int TY, int groups) {
    int seen[13 * 11] = {};
    const int blocks = sgn::square_blocks(TX, TY, groups);
    for (int b = 0; b < blocks; ++b)
        for (int g = 0; g < groups; ++g) {
            const int s = sgn::square_surfel(TX, TY, groups, b, g);
            if (s >= TX * TY) return false;
            if (s >= 0) ++seen[s];
        }
    for (int s = 0; s < TX * TY; ++s)
        if (seen[s] != 1) return false;
    return true;
}
constexpr bool square_mapping_checks() {
    for (int groups = 2; groups <= 32; groups *= 2)
        for (int TX = 1; TX <= 13; TX += 3)
            for (int TY = 1; TY <= 11; TY += 2)
                if (!square_mapping_is_bijective(TX, TY, groups)) return false;
    return true;
}
static_assert(square_mapping_checks(), "square tile mapping");

cudaMemcpyKind kind_to_device(sgn_mem m) { return m == SGN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind kind_from_device(sgn_mem m) { return m == SGN_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

// A call's stream-ordered transfers: device-side ones go out as one copy kernel (a single graph
// node instead of one memcpy node per range), host-side ones, or any range the device cannot
// address directly, as one cudaMemcpy(2D)Async each.
struct Transfers {
    sgn::CopyJob job[sgn::kMaxCopyJobs];
    int n = 0;
    void add(void* dst, const void* src, size_t bytes) { add_rows(dst, bytes, src, bytes, bytes, 1); }
    void add_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row_bytes, int rows) {
        if (row_bytes == 0 || rows <= 0) return;
        job[n++] = sgn::CopyJob{dst, src, dpitch, spitch, row_bytes, rows};
    }
    static bool device_accessible(const void* q) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
               (a.type == cudaMemoryTypeHost && a.devicePointer == q);
    }
    cudaError_t issue(sgn_mem mem, cudaMemcpyKind kind, cudaStream_t st) const {
        bool kernel = mem == SGN_DEVICE;
        for (int i = 0; kernel && i < n; ++i) kernel = device_accessible(job[i].dst) && device_accessible(job[i].src);
        if (kernel) {
            const int e = sgn::launch_copy_jobs(job, n, st);
            if (e == cudaSuccess && n > 0) sgn::count_launch();
            return cudaError_t(e);
        }
        for (int i = 0; i < n; ++i) {
            const sgn::CopyJob& j = job[i];
            const cudaError_t e = j.rows == 1 ? cudaMemcpyAsync(j.dst, j.src, j.row_bytes, kind, st)
                                              : cudaMemcpy2DAsync(j.dst, j.dpitch, j.src, j.spitch, j.row_bytes, j.rows, kind, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

sgn_status sync_event(cudaEvent_t ev, cudaStream_t stream, uint64_t timeout_ns) {
    cudaError_t e = cudaEventRecord(ev, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned spin = 0;; ++spin) {
        e = cudaEventQuery(ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "asynchronous CUDA error");
        if (timeout_ns) {
            const auto dt = std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0);
            if (uint64_t(dt.count()) >= timeout_ns) return fail(SGN_ERR_TIMEOUT, "sync deadline passed");
        }
        if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CUDA error");
    return SGN_OK;
}

}  // namespace

extern "C" {

sgn_status sgn_plan_desc_default(sgn_plan_desc* d, int width, int height, int patch, int max_frames) {
    if (!d) return fail(SGN_ERR_INVALID_ARGUMENT, "desc is NULL");
    std::memset(d, 0, sizeof *d);
    d->width = width;
    d->height = height;
    d->patch = patch;
    d->max_frames = max_frames;
    d->image_dtype = SGN_F32;
    d->huber_k = 9.0f / 255.0f;
    d->lm_lambda = 1e-3f;
    d->fp64_cond = 1e6;
    d->optimize_normal = 1;
    d->min_residuals = 8;
    d->lm_adaptive = 0;
    d->surfel_radius = 0.0f;
    return SGN_OK;
}

sgn_status sgn_plan_create(const sgn_plan_desc* d, sgn_plan** out) {
    if (!d || !out) return fail(SGN_ERR_INVALID_ARGUMENT, "desc/out is NULL");
    *out = nullptr;
    if (d->patch != 4 && d->patch != 8 && d->patch != 16) return fail(SGN_ERR_INVALID_ARGUMENT, "patch must be 4, 8 or 16 (got %d)", d->patch);
    if (d->width < 8 || d->height < 8 || d->width > 16384 || d->height > 16384)
        return fail(SGN_ERR_INVALID_ARGUMENT, "image size %dx%d outside [8, 16384]", d->width, d->height);
    if (d->width < d->patch || d->height < d->patch) return fail(SGN_ERR_INVALID_ARGUMENT, "image smaller than one tile");
    if (d->max_frames < 1 || d->max_frames > SGN_MAX_FRAMES)
        return fail(SGN_ERR_INVALID_ARGUMENT, "max_frames must be in [1, %d]", SGN_MAX_FRAMES);
    if (!(d->image_dtype >= SGN_F32 && d->image_dtype <= SGN_BF16G))
        return fail(SGN_ERR_INVALID_ARGUMENT, "unknown image dtype %d", int(d->image_dtype));
    if (!(d->huber_k > 0.0f) || !std::isfinite(d->huber_k)) return fail(SGN_ERR_INVALID_ARGUMENT, "huber_k must be positive and finite");
    if (!(d->lm_lambda >= 0.0f) || !std::isfinite(d->lm_lambda)) return fail(SGN_ERR_INVALID_ARGUMENT, "lm_lambda must be >= 0 and finite");
    if (std::isnan(d->fp64_cond)) return fail(SGN_ERR_INVALID_ARGUMENT, "fp64_cond is NaN");
    if (d->optimize_normal != 0 && d->optimize_normal != 1) return fail(SGN_ERR_INVALID_ARGUMENT, "optimize_normal must be 0 or 1");
    if (d->min_residuals < 0) return fail(SGN_ERR_INVALID_ARGUMENT, "min_residuals must be >= 0");
    if (d->lm_adaptive != 0 && d->lm_adaptive != 1) return fail(SGN_ERR_INVALID_ARGUMENT, "lm_adaptive must be 0 or 1");
    std::vector<int> disc;
    if (d->surfel_radius != 0.0f && d->lm_adaptive)
        return fail(SGN_ERR_INVALID_ARGUMENT, "circular surfels use the fixed damping (lm_adaptive = 0)");
    if (d->surfel_radius != 0.0f) {
        if (!(d->surfel_radius >= 0.5f) || !(d->surfel_radius <= 16.0f))
            return fail(SGN_ERR_INVALID_ARGUMENT, "surfel_radius must be 0 (tiles) or in [0.5, 16]");
        const int n = sgn::disc_pixels(d->patch, d->surfel_radius, nullptr);
        if (n < 1) return fail(SGN_ERR_INVALID_ARGUMENT, "surfel_radius %g covers more than %d pixels", double(d->surfel_radius), sgn::kMaxDiscPixels);
        disc.resize(size_t(2) * n);
        sgn::disc_pixels(d->patch, d->surfel_radius, disc.data());
    }
    sgn_plan* p = new (std::nothrow) sgn_plan();
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "out of host memory");
    p->desc = *d;
    p->TX = d->width / d->patch;
    p->TY = d->height / d->patch;
    p->S = p->TX * p->TY;
    p->disc = std::move(disc);
    p->L = make_layout(*d, p->S, int(p->disc.size() / 2));
    p->lanes = p->disc.empty() ? default_lanes(d->patch) : 32;
    *out = p;
    return SGN_OK;
}

sgn_status sgn_plan_destroy(sgn_plan* p) {
    if (!p) return SGN_OK;
    if (p->done) {
        DeviceGuard g(p->device);
        cudaEventDestroy(p->done);
    }
    delete p;
    return SGN_OK;
}

sgn_status sgn_plan_num_surfels(const sgn_plan* p, int* n) {
    if (!p || !n) return fail(SGN_ERR_INVALID_ARGUMENT, "plan/out is NULL");
    *n = p->S;
    return SGN_OK;
}

sgn_status sgn_plan_workspace_bytes(const sgn_plan* p, size_t* bytes) {
    if (!p || !bytes) return fail(SGN_ERR_INVALID_ARGUMENT, "plan/out is NULL");
    *bytes = p->L.total;
    return SGN_OK;
}

sgn_status sgn_plan_set_mapping(sgn_plan* p, int lanes_per_surfel, int block_threads) {
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    const int G = lanes_per_surfel ? lanes_per_surfel : (p->disc.empty() ? default_lanes(p->desc.patch) : 32);
    const int B = block_threads ? block_threads : 256;
    if (!p->disc.empty() && lanes_per_surfel && G != 32)
        return fail(SGN_ERR_INVALID_ARGUMENT, "circular surfels use 32 lanes per surfel");
    if (p->disc.empty() && !mapping_supported(p->desc.patch, G))
        return fail(SGN_ERR_INVALID_ARGUMENT, "%d lanes per surfel not supported for %dx%d tiles", G, p->desc.patch, p->desc.patch);
    if (B == 512) {
        if (!p->disc.empty() || p->desc.lm_adaptive || p->staging || G * 4 != p->desc.patch * p->desc.patch)
            return fail(SGN_ERR_INVALID_ARGUMENT, "512-thread blocks need square surfels with 4 pixels per lane and fixed damping");
    } else if (B < 32 || B > 256 || B % 32) {
        return fail(SGN_ERR_INVALID_ARGUMENT, "block_threads must be a multiple of 32 in [32, 256], or 512");
    }
    p->lanes = G;
    p->block = B;
    return SGN_OK;
}

sgn_status sgn_plan_set_staging(sgn_plan* p, int enabled) {
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    if (enabled != 0 && enabled != 1) return fail(SGN_ERR_INVALID_ARGUMENT, "enabled must be 0 or 1");
    if (enabled && p->block > 256) return fail(SGN_ERR_INVALID_ARGUMENT, "staging needs blocks of at most 256 threads");
    p->staging = enabled != 0;
    return SGN_OK;
}

sgn_status sgn_staging_timeouts(uint32_t* count) {
    if (!count) return fail(SGN_ERR_INVALID_ARGUMENT, "count is NULL");
    unsigned int* w = sgn::stage_error_word();
    if (!w) return fail(SGN_ERR_CUDA, "staging error counter unavailable");
    const cudaError_t e = cudaMemcpy(count, w, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the staging timeout counter");
    return SGN_OK;
}

sgn_status sgn_plan_bind(sgn_plan* p, void* ws, size_t bytes, void* stream) {
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    if (!ws) return fail(SGN_ERR_INVALID_ARGUMENT, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % sgn::kAlign) return fail(SGN_ERR_INVALID_ARGUMENT, "workspace must be 256-byte aligned");
    if (bytes < p->L.total) return fail(SGN_ERR_WORKSPACE_TOO_SMALL, "workspace %zu bytes < %zu needed", bytes, p->L.total);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaPointerAttributes attr{};
    e = cudaPointerGetAttributes(&attr, ws);
    if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(SGN_ERR_INVALID_ARGUMENT, "workspace is not device memory");
    }
    if (attr.device != dev) return fail(SGN_ERR_INVALID_ARGUMENT, "workspace is on device %d, current device is %d", attr.device, dev);
    if (p->done && p->device != dev) {
        DeviceGuard g(p->device);
        cudaEventDestroy(p->done);
        p->done = nullptr;
    }
    if (!p->done) {
        e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    p->ws = static_cast<char*>(ws);
    p->ws_bytes = bytes;
    p->tmap_ok = false;
    p->stream = static_cast<cudaStream_t>(stream);
    p->device = dev;
    p->kf_set = false;
    p->surfels_set = false;
    for (bool& b : p->frame_set) b = false;
    p->F = 0;
    const size_t npx = size_t(p->desc.width) * p->desc.height;
    e = cudaMemsetAsync(p->ws + p->L.depth, 0, npx * sizeof(float), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ws + p->L.sidx, 0xff, npx * sizeof(int32_t), p->stream);
    if (e == cudaSuccess && !p->disc.empty())  // the plan owns the host table, which outlives the copy
        e = cudaMemcpyAsync(p->ws + p->L.disc, p->disc.data(), p->disc.size() * sizeof(int), cudaMemcpyHostToDevice,
                            p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the depth map");
    p->depth_valid = true;
    return SGN_OK;
}

sgn_status sgn_set_intrinsics(sgn_plan* p, double fx, double fy, double cx, double cy) {
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    if (!(fx > 0) || !(fy > 0) || !std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(cx) || !std::isfinite(cy))
        return fail(SGN_ERR_INVALID_ARGUMENT, "intrinsics must be finite with fx, fy > 0");
    p->fx = fx;
    p->fy = fy;
    p->cx = cx;
    p->cy = cy;
    p->have_K = true;
    return SGN_OK;
}

sgn_status sgn_set_keyframe(sgn_plan* p, const float* img, size_t pitch, sgn_mem mem) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    const int W = p->desc.width, H = p->desc.height;
    if (!img) return fail(SGN_ERR_INVALID_ARGUMENT, "keyframe pointer is NULL");
    if (mem != SGN_HOST && mem != SGN_DEVICE) return fail(SGN_ERR_INVALID_ARGUMENT, "bad memory kind");
    if (pitch < size_t(W) * sizeof(float) || pitch % sizeof(float)) return fail(SGN_ERR_INVALID_ARGUMENT, "keyframe pitch %zu invalid for width %d", pitch, W);
    DeviceGuard g(p->device);
    Transfers t;
    t.add_rows(p->ws + p->L.kf, size_t(p->L.kf_pitch) * sizeof(float), img, pitch, size_t(W) * sizeof(float), H);
    const cudaError_t e = t.issue(mem, kind_to_device(mem), p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "keyframe upload");
    p->kf_set = true;
    return SGN_OK;
}

sgn_status sgn_set_frames(sgn_plan* p, int n, const float* const* imgs, size_t pitch, sgn_mem mem, const double* T) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    const int W = p->desc.width, H = p->desc.height;
    if (n < 1 || n > p->desc.max_frames) return fail(SGN_ERR_INVALID_ARGUMENT, "frame count %d outside [1, %d]", n, p->desc.max_frames);
    if (!imgs || !T) return fail(SGN_ERR_INVALID_ARGUMENT, "images/poses pointer is NULL");
    if (mem != SGN_HOST && mem != SGN_DEVICE) return fail(SGN_ERR_INVALID_ARGUMENT, "bad memory kind");
    if (pitch < size_t(W) * sizeof(float) || pitch % sizeof(float)) return fail(SGN_ERR_INVALID_ARGUMENT, "frame pitch %zu invalid for width %d", pitch, W);
    for (int i = 0; i < n; ++i) {
        if (!imgs[i]) return fail(SGN_ERR_INVALID_ARGUMENT, "frame %d pointer is NULL", i);
        if ((st = check_pose(T + 12 * i)) != SGN_OK) return st;
    }
    DeviceGuard g(p->device);
    const float* src[sgn::kMaxFrames];
    size_t sp[sgn::kMaxFrames];
    for (int i = 0; i < n; ++i) {
        if (mem == SGN_HOST) {
            char* dst = p->ws + p->L.raw + size_t(i) * p->L.raw_plane * sizeof(float);
            cudaError_t e = cudaMemcpy2DAsync(dst, size_t(p->L.raw_pitch) * sizeof(float), imgs[i], pitch,
                                              size_t(W) * sizeof(float), H, cudaMemcpyHostToDevice, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "frame upload");
            src[i] = reinterpret_cast<const float*>(dst);
            sp[i] = size_t(p->L.raw_pitch);
        } else {
            src[i] = imgs[i];
            sp[i] = pitch / sizeof(float);
        }
    }
    PlanParams pp = make_params(p);
    int e = sgn::launch_prep_frames(pp, src, sp, 0, n, p->stream);
    if (e) return cuda_fail(e, "frame preparation launch");
    sgn::count_launch();
    for (int i = 0; i < n; ++i) {
        std::memcpy(p->T[i], T + 12 * i, sizeof(double) * 12);
        p->frame_set[i] = true;
    }
    p->F = n;
    return SGN_OK;
}

sgn_status sgn_set_frame(sgn_plan* p, int slot, const float* img, size_t pitch, sgn_mem mem, const double* T) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    const int W = p->desc.width, H = p->desc.height;
    if (slot < 0 || slot >= p->desc.max_frames) return fail(SGN_ERR_INVALID_ARGUMENT, "slot %d outside [0, %d)", slot, p->desc.max_frames);
    if (!img) return fail(SGN_ERR_INVALID_ARGUMENT, "frame pointer is NULL");
    if (mem != SGN_HOST && mem != SGN_DEVICE) return fail(SGN_ERR_INVALID_ARGUMENT, "bad memory kind");
    if (pitch < size_t(W) * sizeof(float) || pitch % sizeof(float)) return fail(SGN_ERR_INVALID_ARGUMENT, "frame pitch %zu invalid for width %d", pitch, W);
    if ((st = check_pose(T)) != SGN_OK) return st;
    DeviceGuard g(p->device);
    const float* src = img;
    size_t sp = pitch / sizeof(float);
    if (mem == SGN_HOST) {
        char* dst = p->ws + p->L.raw + size_t(slot) * p->L.raw_plane * sizeof(float);
        cudaError_t e = cudaMemcpy2DAsync(dst, size_t(p->L.raw_pitch) * sizeof(float), img, pitch, size_t(W) * sizeof(float),
                                          H, cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "frame upload");
        src = reinterpret_cast<const float*>(dst);
        sp = size_t(p->L.raw_pitch);
    }
    PlanParams pp = make_params(p);
    int e = sgn::launch_prep_frames(pp, &src, &sp, slot, 1, p->stream);
    if (e) return cuda_fail(e, "frame preparation launch");
    sgn::count_launch();
    std::memcpy(p->T[slot], T, sizeof(double) * 12);
    p->frame_set[slot] = true;
    if (slot + 1 > p->F) p->F = slot + 1;
    return SGN_OK;
}

sgn_status sgn_set_num_frames(sgn_plan* p, int n) {
    if (!p) return fail(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    if (n < 1 || n > p->desc.max_frames) return fail(SGN_ERR_INVALID_ARGUMENT, "frame count %d outside [1, %d]", n, p->desc.max_frames);
    for (int f = 0; f < n; ++f)
        if (!p->frame_set[f]) return fail(SGN_ERR_STATE, "frame slot %d not set", f);
    p->F = n;
    return SGN_OK;
}

sgn_status sgn_init_surfels(sgn_plan* p, const float* id, const float* n, const uint8_t* state, sgn_mem mem) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (!id || !n || !state) return fail(SGN_ERR_INVALID_ARGUMENT, "surfel pointer is NULL");
    if (mem != SGN_HOST && mem != SGN_DEVICE) return fail(SGN_ERR_INVALID_ARGUMENT, "bad memory kind");
    const size_t S = size_t(p->S);
    if (mem == SGN_HOST) {
        for (size_t s = 0; s < S; ++s) {
            if (state[s] > SGN_STATE_TO_SEED) return fail(SGN_ERR_INVALID_ARGUMENT, "surfel %zu has unknown state %d", s, int(state[s]));
            if (state[s] == SGN_STATE_VALID) {
                const float nn = n[3 * s] * n[3 * s] + n[3 * s + 1] * n[3 * s + 1] + n[3 * s + 2] * n[3 * s + 2];
                if (!(id[s] > 0.0f) || !std::isfinite(id[s]) || !(std::fabs(nn - 1.0f) < 1e-3f))
                    return fail(SGN_ERR_INVALID_ARGUMENT, "valid surfel %zu needs a positive finite inverse depth and a unit normal", s);
            }
        }
    }
    DeviceGuard g(p->device);
    Transfers t;
    t.add(p->ws + p->L.id0, id, S * sizeof(float));
    t.add(p->ws + p->L.n0, n, 3 * S * sizeof(float));
    t.add(p->ws + p->L.state0, state, S);
    const cudaError_t e = t.issue(mem, kind_to_device(mem), p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "surfel upload");
    // The working state is derived from the initial surfels on first need (sgn_solve rebuilds it
    // itself, so a solve right after the upload launches nothing extra).
    p->surfels_set = true;
    p->state_pending = true;
    p->depth_valid = false;
    return SGN_OK;
}

static sgn_status ensure_state(sgn_plan* p) {
    if (!p->state_pending) return SGN_OK;
    PlanParams pp = make_params(p);
    int le = sgn::launch_init_state(pp, p->stream);
    if (le) return cuda_fail(le, "surfel initialisation launch");
    sgn::count_launch();
    p->state_pending = false;
    return SGN_OK;
}

sgn_status sgn_seed_surfels(sgn_plan* p) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (!p->have_K) return fail(SGN_ERR_STATE, "intrinsics not set");
    if (!p->surfels_set) return fail(SGN_ERR_STATE, "surfels not initialised");
    DeviceGuard g(p->device);
    PlanParams pp = make_params(p);
    int e = sgn::launch_seed(pp, p->stream);
    if (e) return cuda_fail(e, "seeding launch");
    sgn::count_launch();
    p->state_pending = false;
    p->depth_valid = false;
    return SGN_OK;
}

static sgn_status run_mode(sgn_plan* p, int iters, int mode) {
    sgn_status st = require_ready(p);
    if (st != SGN_OK) return st;
    if (iters < 0 || iters > 100000) return fail(SGN_ERR_INVALID_ARGUMENT, "iters %d outside [0, 100000]", iters);
    DeviceGuard g(p->device);
    if (mode == sgn::kModeRun && (st = ensure_state(p)) != SGN_OK) return st;
    PlanParams pp = make_params(p);
    if (p->staging && !p->tmap_ok) {
        if (!pp.stage_err) return fail(SGN_ERR_CUDA, "staging error counter unavailable");
        const int te = sgn::encode_texel_map(p->tmap, pp, p->desc.max_frames);
        if (te) return cuda_fail(te, "encoding the texel TMA descriptor");
        p->tmap_ok = true;
    }
    const bool disc = !p->disc.empty();
    int e = sgn::launch_gn(pp, iters, mode, p->lanes, p->block, p->stream, p->staging && !disc ? p->tmap : nullptr);
    if (e) return cuda_fail(e, "Gauss-Newton launch");
    sgn::count_launch();
    if (disc) {  // overlapping discs: the depth map is their depth-buffered render (Sec. 2.2)
        if ((e = sgn::launch_render_discs(pp, p->stream))) return cuda_fail(e, "disc render launch");
        sgn::count_launch(2);
    }
    p->state_pending = false;  // a solve writes the whole working state
    p->depth_valid = true;
    return SGN_OK;
}

sgn_status sgn_run(sgn_plan* p, int iters) { return run_mode(p, iters, sgn::kModeRun); }
sgn_status sgn_solve(sgn_plan* p, int iters) { return run_mode(p, iters, sgn::kModeSolve); }

// Transfers of the surfel arrays and of the depth map into t (the map is rendered first when it is
// stale).  Either group may be absent (all its pointers NULL).
static sgn_status queue_results(sgn_plan* p, float* id, float* n, float* cost, int32_t* nres, uint8_t* status,
                                float* inv_depth, int32_t* sidx, bool surfels, bool map, Transfers& t) {
    sgn_status st;
    if (surfels) {
        if (!p->surfels_set) return fail(SGN_ERR_STATE, "surfels not initialised");
        if ((st = ensure_state(p)) != SGN_OK) return st;
        const size_t S = size_t(p->S);
        if (id) t.add(id, p->ws + p->L.id, S * sizeof(float));
        if (n) t.add(n, p->ws + p->L.n, 3 * S * sizeof(float));
        if (cost) t.add(cost, p->ws + p->L.cost, S * sizeof(float));
        if (nres) t.add(nres, p->ws + p->L.nres, S * sizeof(int32_t));
        if (status) t.add(status, p->ws + p->L.status, S);
    }
    if (map) {
        if (!p->depth_valid) {
            if (!p->have_K || !p->surfels_set) return fail(SGN_ERR_STATE, "depth map needs intrinsics and surfels");
            if ((st = ensure_state(p)) != SGN_OK) return st;
            PlanParams pp = make_params(p);
            int e = p->disc.empty() ? sgn::launch_render_depth(pp, p->stream) : sgn::launch_render_discs(pp, p->stream);
            if (e) return cuda_fail(e, "depth render launch");
            sgn::count_launch(p->disc.empty() ? 1 : 2);
            p->depth_valid = true;
        }
        const size_t npx = size_t(p->desc.width) * p->desc.height;
        if (inv_depth) t.add(inv_depth, p->ws + p->L.depth, npx * sizeof(float));
        if (sidx) t.add(sidx, p->ws + p->L.sidx, npx * sizeof(int32_t));
    }
    return SGN_OK;
}

sgn_status sgn_read_surfels(sgn_plan* p, float* id, float* n, float* cost, int32_t* nres, uint8_t* status, sgn_mem mem) {
    return sgn_read_results(p, id, n, cost, nres, status, nullptr, nullptr, mem);
}

sgn_status sgn_read_depth_map(sgn_plan* p, float* inv_depth, int32_t* sidx, sgn_mem mem) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (mem != SGN_HOST && mem != SGN_DEVICE) return fail(SGN_ERR_INVALID_ARGUMENT, "bad memory kind");
    DeviceGuard g(p->device);
    Transfers t;
    if ((st = queue_results(p, nullptr, nullptr, nullptr, nullptr, nullptr, inv_depth, sidx, false, true, t)) != SGN_OK)
        return st;
    const cudaError_t e = t.issue(mem, kind_from_device(mem), p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "depth map readback");
    return SGN_OK;
}

sgn_status sgn_read_results(sgn_plan* p, float* id, float* n, float* cost, int32_t* nres, uint8_t* status,
                            float* inv_depth, int32_t* sidx, sgn_mem mem) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (mem != SGN_HOST && mem != SGN_DEVICE) return fail(SGN_ERR_INVALID_ARGUMENT, "bad memory kind");
    DeviceGuard g(p->device);
    Transfers t;
    const bool map = inv_depth || sidx;
    if ((st = queue_results(p, id, n, cost, nres, status, inv_depth, sidx, true, map, t)) != SGN_OK) return st;
    const cudaError_t e = t.issue(mem, kind_from_device(mem), p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "result readback");
    return SGN_OK;
}

sgn_status sgn_sync(sgn_plan* p, uint64_t timeout_ns) {
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    DeviceGuard g(p->device);
    return sync_event(p->done, p->stream, timeout_ns);
}

sgn_status sgn_state_bytes(const sgn_plan* p, size_t* bytes) {
    if (!p || !bytes) return fail(SGN_ERR_INVALID_ARGUMENT, "plan/out is NULL");
    *bytes = size_t(p->S) * (sizeof(float) * 5 + sizeof(int32_t) + 1);
    return SGN_OK;
}

sgn_status sgn_export_state(sgn_plan* p, void* host, size_t bytes) {
    size_t need = 0;
    sgn_state_bytes(p, &need);
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (!host || bytes < need) return fail(SGN_ERR_INVALID_ARGUMENT, "state buffer NULL or smaller than %zu bytes", need);
    char* h = static_cast<char*>(host);
    const size_t S = size_t(p->S);
    if ((st = sgn_read_surfels(p, reinterpret_cast<float*>(h), reinterpret_cast<float*>(h + 4 * S),
                               reinterpret_cast<float*>(h + 16 * S), reinterpret_cast<int32_t*>(h + 20 * S),
                               reinterpret_cast<uint8_t*>(h + 24 * S), SGN_HOST)) != SGN_OK)
        return st;
    return sgn_sync(p, 0);
}

sgn_status sgn_import_state(sgn_plan* p, const void* host, size_t bytes) {
    size_t need = 0;
    sgn_state_bytes(p, &need);
    sgn_status st = require_bound(p);
    if (st != SGN_OK) return st;
    if (!host || bytes < need) return fail(SGN_ERR_INVALID_ARGUMENT, "state buffer NULL or smaller than %zu bytes", need);
    DeviceGuard g(p->device);
    const char* h = static_cast<const char*>(host);
    const size_t S = size_t(p->S);
    const cudaMemcpyKind k = cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(p->ws + p->L.id, h, 4 * S, k, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->ws + p->L.n, h + 4 * S, 12 * S, k, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->ws + p->L.cost, h + 16 * S, 4 * S, k, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->ws + p->L.nres, h + 20 * S, 4 * S, k, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->ws + p->L.status, h + 24 * S, S, k, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state import");
    p->surfels_set = true;
    p->state_pending = false;
    p->depth_valid = false;
    return sgn_sync(p, 0);
}

// ------------------------------------------------------------------------------------------ batches

sgn_status sgn_batch_create(int max_plans, sgn_batch** out) {
    if (!out) return fail(SGN_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (max_plans < 1 || max_plans > 65536) return fail(SGN_ERR_INVALID_ARGUMENT, "max_plans outside [1, 65536]");
    sgn_batch* b = new (std::nothrow) sgn_batch();
    if (!b) return fail(SGN_ERR_INVALID_ARGUMENT, "out of host memory");
    b->max_plans = max_plans;
    *out = b;
    return SGN_OK;
}

static void batch_drop_graph(sgn_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_iters = -1;
}

sgn_status sgn_batch_add(sgn_batch* b, sgn_plan* p) {
    if (!b || !p) return fail(SGN_ERR_INVALID_ARGUMENT, "batch/plan is NULL");
    if (int(b->plans.size()) >= b->max_plans) return fail(SGN_ERR_INVALID_ARGUMENT, "batch is full (%d plans)", b->max_plans);
    b->plans.push_back(p);
    b->dirty = true;
    return SGN_OK;
}

sgn_status sgn_batch_clear(sgn_batch* b) {
    if (!b) return fail(SGN_ERR_INVALID_ARGUMENT, "batch is NULL");
    b->plans.clear();
    b->dirty = true;
    return SGN_OK;
}

static size_t batch_items_upper(const sgn_batch* b) {
    size_t n = 0;
    for (const sgn_plan* p : b->plans) {
        n += (size_t(p->S) + b->chunk - 1) / b->chunk;
        if (b->variant == 2 && p->disc.empty() && !p->desc.lm_adaptive)  // square items of a fixed-damping plan
            n += size_t(sgn::square_items(p->desc.patch, p->desc.width / p->desc.patch, p->desc.height / p->desc.patch));
    }
    return n;
}

static size_t batch_ws_need(const sgn_batch* b, size_t* off_items, size_t* off_counter) {
    const size_t tbl = round_up(size_t(b->max_plans) * sizeof(PlanParams), sgn::kAlign);
    const size_t items = round_up(std::max<size_t>(1, batch_items_upper(b)) * sizeof(WorkItem), sgn::kAlign);
    if (off_items) *off_items = tbl;
    if (off_counter) *off_counter = tbl + items;
    return tbl + items + sgn::kAlign;
}

sgn_status sgn_batch_workspace_bytes(const sgn_batch* b, size_t* bytes) {
    if (!b || !bytes) return fail(SGN_ERR_INVALID_ARGUMENT, "batch/out is NULL");
    *bytes = batch_ws_need(b, nullptr, nullptr);
    return SGN_OK;
}

sgn_status sgn_batch_set_schedule(sgn_batch* b, int variant, int chunk) {
    if (!b) return fail(SGN_ERR_INVALID_ARGUMENT, "batch is NULL");
    if (variant < 0 || variant > 2) return fail(SGN_ERR_INVALID_ARGUMENT, "variant must be 0, 1 or 2");
    if (chunk < 1 || chunk > 65536) return fail(SGN_ERR_INVALID_ARGUMENT, "chunk outside [1, 65536]");
    if (b->variant != variant || b->chunk != chunk) {
        b->variant = variant;
        b->chunk = chunk;
        b->dirty = true;
        batch_drop_graph(b);
    }
    return SGN_OK;
}

sgn_status sgn_batch_bind(sgn_batch* b, void* ws, size_t bytes, void* stream) {
    if (!b || !ws) return fail(SGN_ERR_INVALID_ARGUMENT, "batch/workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % sgn::kAlign) return fail(SGN_ERR_INVALID_ARGUMENT, "workspace must be 256-byte aligned");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (!b->done) {
        e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    batch_drop_graph(b);
    b->ws = static_cast<char*>(ws);
    b->ws_bytes = bytes;
    b->stream = static_cast<cudaStream_t>(stream);
    b->device = dev;
    b->dirty = true;
    return SGN_OK;
}

sgn_status sgn_batch_run(sgn_batch* b, int iters) {
    if (!b) return fail(SGN_ERR_INVALID_ARGUMENT, "batch is NULL");
    if (!b->ws) return fail(SGN_ERR_NOT_BOUND, "batch has no workspace; call sgn_batch_bind");
    if (b->plans.empty()) return fail(SGN_ERR_STATE, "batch has no plans");
    if (iters < 0 || iters > 100000) return fail(SGN_ERR_INVALID_ARGUMENT, "iters %d outside [0, 100000]", iters);
    size_t off_items = 0, off_counter = 0;
    const size_t need = batch_ws_need(b, &off_items, &off_counter);
    if (b->ws_bytes < need) return fail(SGN_ERR_WORKSPACE_TOO_SMALL, "batch workspace %zu bytes < %zu needed", b->ws_bytes, need);
    for (sgn_plan* p : b->plans) {
        sgn_status st = require_ready(p);
        if (st != SGN_OK) return st;
        if (p->device != b->device) return fail(SGN_ERR_INVALID_ARGUMENT, "plan and batch are on different devices");
    }
    DeviceGuard g(b->device);
    cudaError_t e;
    // Order the batch after each plan's uploads and preparations.
    std::vector<cudaStream_t> streams;
    for (sgn_plan* p : b->plans)
        if (p->stream != b->stream && std::find(streams.begin(), streams.end(), p->stream) == streams.end())
            streams.push_back(p->stream);
    while (b->plan_events.size() < streams.size()) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        b->plan_events.push_back(ev);
    }
    for (size_t i = 0; i < streams.size(); ++i) {
        if ((e = cudaEventRecord(b->plan_events[i], streams[i])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(b->stream, b->plan_events[i], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    }
    // Plan table and work list: refreshed every run (poses, frame counts and options may change);
    // items are (plan, surfel range) chunks ordered by decreasing cost (largest first).
    b->h_plans.resize(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); ++i) b->h_plans[i] = make_params(b->plans[i]);
    if (b->dirty) {
        b->h_items.clear();
        for (size_t i = 0; i < b->plans.size(); ++i) {
            const sgn_plan* p = b->plans[i];
            if (b->variant == 2 && sgn::batch_kind(b->h_plans[i]) == sgn::kBatchFixed) {
                // square items: one block's square of tiles each (count = its surfels, for the order)
                const PlanParams& pp = b->h_plans[i];
                const int groups = 256 / sgn::lanes_for_patch(2, pp.P);
                const int n = sgn::square_items(pp.P, pp.TX, pp.TY);
                for (int q = 0; q < n; ++q) {
                    int cnt = 0;
                    for (int g = 0; g < groups; ++g) cnt += sgn::square_surfel(pp.TX, pp.TY, groups, q, g) >= 0;
                    b->h_items.push_back(WorkItem{int(i), q, cnt, 0});
                }
                continue;
            }
            for (int f = 0; f < p->S; f += b->chunk)
                b->h_items.push_back(WorkItem{int(i), f, std::min(b->chunk, p->S - f), 0});
        }
        // Items of one solver kind form one contiguous range (one launch per kind).  Items of one
        // patch size run the same code path: grouping them (largest patch first) keeps the warps of an
        // SM on one solver variant at a time; within a group, largest cost first.
        auto kind_of = [&](const WorkItem& w) { return sgn::batch_kind(b->h_plans[w.plan]); };
        std::stable_sort(b->h_items.begin(), b->h_items.end(), [&](const WorkItem& a, const WorkItem& c) {
            const sgn_plan* pa = b->plans[a.plan];
            const sgn_plan* pc = b->plans[c.plan];
            if (kind_of(a) != kind_of(c)) return kind_of(a) < kind_of(c);
            if (pa->desc.patch != pc->desc.patch) return pa->desc.patch > pc->desc.patch;
            const double ca = double(a.count) * pa->desc.patch * pa->desc.patch * std::max(1, pa->F);
            const double cc = double(c.count) * pc->desc.patch * pc->desc.patch * std::max(1, pc->F);
            return ca > cc;
        });
        b->n_items = int(b->h_items.size());
        for (int k = 0; k <= sgn::kBatchKinds; ++k) b->kind_begin[k] = 0;
        for (const WorkItem& w : b->h_items) b->kind_begin[kind_of(w) + 1]++;
        for (int k = 0; k < sgn::kBatchKinds; ++k) b->kind_begin[k + 1] += b->kind_begin[k];
        batch_drop_graph(b);  // the captured launches hold the item counts
        e = cudaMemcpyAsync(b->ws + off_items, b->h_items.data(), b->h_items.size() * sizeof(WorkItem),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "work list upload");
        b->dirty = false;
    }
    e = cudaMemcpyAsync(b->ws, b->h_plans.data(), b->h_plans.size() * sizeof(PlanParams), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "plan table upload");
    // The persistent launch (counter reset + kernel) is captured once per iteration count and
    // replayed as a CUDA graph.
    int fmax = 1;
    for (const PlanParams& pp : b->h_plans) fmax = std::max(fmax, pp.F);
    if (!b->exec || b->graph_iters != iters || b->graph_frames != fmax) {
        batch_drop_graph(b);
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        int grids[sgn::kBatchKinds] = {0, 0, 0};
        for (int k = 0; k < sgn::kBatchKinds; ++k) {
            if (b->kind_begin[k + 1] == b->kind_begin[k]) continue;
            const int per_sm = sgn::batch_blocks_per_sm(k, b->variant, 256, fmax);
            if (per_sm <= 0) return fail(SGN_ERR_CUDA, "batch kernel cannot be resident");
            grids[k] = sms * per_sm;
        }
        b->graph_grid = grids[sgn::kBatchFixed];
        cudaStream_t cap = b->stream;
        bool own = false;
        if (cap == nullptr || cap == cudaStreamLegacy) {
            if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "capture stream");
            own = true;
        }
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            if (own) cudaStreamDestroy(cap);
            return cuda_fail(e, "cudaStreamBeginCapture");
        }
        // one persistent launch per solver kind present, each over its range of the work list with its
        // own counter (the launches run one after another on the stream)
        int le = 0;
        for (int k = 0; k < sgn::kBatchKinds && !le; ++k) {
            const int n = b->kind_begin[k + 1] - b->kind_begin[k];
            if (n == 0) continue;
            le = sgn::launch_gn_batch(k, reinterpret_cast<const PlanParams*>(b->ws),
                                      reinterpret_cast<const WorkItem*>(b->ws + off_items) + b->kind_begin[k], n,
                                      reinterpret_cast<int*>(b->ws + off_counter) + k, iters, b->variant, grids[k], 256,
                                      fmax, cap);
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        if (own) cudaStreamDestroy(cap);
        if (le) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le, "batch kernel capture");
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        b->graph = graph;
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
            batch_drop_graph(b);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        b->graph_iters = iters;
        b->graph_frames = fmax;
    }
    if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    int kinds = 0;
    for (int k = 0; k < sgn::kBatchKinds; ++k) kinds += b->kind_begin[k + 1] > b->kind_begin[k];
    sgn::count_launch(uint64_t(kinds));
    // circular surfels may overlap: each such plan's depth map is the depth-buffered render of its
    // solved discs (Sec. 2.2), launched here with the plan's current parameters
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (b->plans[i]->disc.empty()) continue;
        const int le = sgn::launch_render_discs(b->h_plans[i], b->stream);
        if (le) return cuda_fail(le, "disc render launch");
        sgn::count_launch(2);
    }
    // Later work on each plan's stream (reads) waits for the batch.
    if ((e = cudaEventRecord(b->done, b->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (cudaStream_t s : streams)
        if ((e = cudaStreamWaitEvent(s, b->done, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    for (sgn_plan* p : b->plans) {
        p->depth_valid = true;
        p->state_pending = false;
    }
    return SGN_OK;
}

sgn_status sgn_batch_sync(sgn_batch* b, uint64_t timeout_ns) {
    if (!b) return fail(SGN_ERR_INVALID_ARGUMENT, "batch is NULL");
    if (!b->ws) return fail(SGN_ERR_NOT_BOUND, "batch has no workspace");
    DeviceGuard g(b->device);
    return sync_event(b->done, b->stream, timeout_ns);
}

sgn_status sgn_batch_destroy(sgn_batch* b) {
    if (!b) return SGN_OK;
    DeviceGuard g(b->device);
    batch_drop_graph(b);
    if (b->done) cudaEventDestroy(b->done);
    for (cudaEvent_t ev : b->plan_events) cudaEventDestroy(ev);
    delete b;
    return SGN_OK;
}

const char* sgn_last_error(void) { return g_last_error.c_str(); }
uint64_t sgn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
int sgn_abi_version(void) { return SGN_ABI_VERSION; }

}  // extern "C"

namespace sgn {
PlanParams plan_params(const sgn_plan* p) { return make_params(p); }
bool plan_ready(const sgn_plan* p) { return require_ready(p) == SGN_OK; }
// After a batched solve of this plan: the working state and depth map are those of a solve.
void plan_mark_solved(sgn_plan* p) {
    p->state_pending = false;
    p->depth_valid = true;
}
cudaStream_t plan_stream(const sgn_plan* p) { return p->stream; }
void plan_shape(const sgn_plan* p, int* W, int* H, int* P, int* F, int* dtype) {
    *W = p->desc.width;
    *H = p->desc.height;
    *P = p->desc.patch;
    *F = p->F;
    *dtype = p->desc.image_dtype;
}
cudaStream_t batch_stream(const sgn_batch* b) { return b->stream; }
// Shape of a batch for tuning caches: plan count and a hash of the (W, H, P, F, dtype) multiset.
std::string batch_signature(const sgn_batch* b) {
    std::vector<std::string> shapes;
    for (const sgn_plan* p : b->plans) {
        std::ostringstream o;
        o << p->desc.width << 'x' << p->desc.height << 'p' << p->desc.patch << 'f' << p->F << 'd' << p->desc.image_dtype;
        shapes.push_back(o.str());
    }
    std::sort(shapes.begin(), shapes.end());
    uint64_t h = 1469598103934665603ull;  // FNV-1a
    for (const std::string& s : shapes)
        for (char c : s + ";") h = (h ^ uint8_t(c)) * 1099511628211ull;
    std::ostringstream o;
    o << b->plans.size() << "plans-" << std::hex << h;
    return o.str();
}
}  // namespace sgn
