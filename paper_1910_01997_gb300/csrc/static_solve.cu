// sgn_solve_static: the whole keyframe solve (frame preparation, seeding, Gauss-Newton iterations,
// final cost, depth map) for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc or any allocator at the point where they solve: real-time
// loops that must not take the allocator's locks or risk an out-of-memory failure mid-run, and host
// frameworks or plugins that hand out only the buffers they own and forbid any allocation of their
// components.  Those callers pass their inputs
// and outputs as device pointers; the one intermediate this path needs, the packed frame texels,
// goes to the fixed array below.
//
// The array is a file-scope __device__ object of SGN_STATIC_SCRATCH_BYTES: every GPU that loads this
// library holds it until the process exits.  All calls share it and it keeps the last call's
// contents; every call rewrites the texels it reads (nothing needs to start at zero), so calls that
// run one after another are independent, but calls whose work overlaps on the GPU (other streams,
// other host threads) race on it.  In host code the array's name is only a host-side stand-in, not a
// device address: the address is looked up with cudaGetSymbolAddress once per device, by the first
// call on that device with the device current, so that first call should come before any stream
// capture.  This path calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "sgn.h"
#include "sgn_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[SGN_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

sgn_status error(sgn_status st, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return sgn::record_error(st, buf);
}

// Device address of the scratch array on the current device (looked up once per device).
sgn_status scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr)
            return error(SGN_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return SGN_OK;
}

// Can the kernels, running on device `dev`, use p directly?  Memory of device `dev` or managed
// memory; another GPU's memory is refused (the kernels would need peer access to it).
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

bool is_rotation(const double* T) {
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(T[i])) return false;
    double worst = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d = 0.0;
            for (int k = 0; k < 3; ++k) d += T[4 * k + i] * T[4 * k + j];
            worst = std::fmax(worst, std::fabs(d - (i == j ? 1.0 : 0.0)));
        }
    const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                       T[2] * (T[4] * T[9] - T[5] * T[8]);
    return worst <= 1e-6 && det > 0.0;
}

}  // namespace

extern "C" sgn_status sgn_solve_static(const sgn_plan_desc* d, const double intrinsics[4], const float* keyframe,
                                       size_t keyframe_pitch_bytes, int num_frames, const float* const* frames,
                                       size_t frame_pitch_bytes, const double* poses, const float* inv_depth0,
                                       const float* normal0, const uint8_t* state0, int iters, float* inv_depth,
                                       float* normal, float* cost, int32_t* nres, uint8_t* status, float* depth_map,
                                       int32_t* surfel_index, void* cuda_stream) {
    // ---- host-side validation (nothing is enqueued on failure)
    if (!d || !intrinsics || !frames || !poses) return error(SGN_ERR_INVALID_ARGUMENT, "desc/intrinsics/frames/poses is NULL");
    if (d->patch != 4 && d->patch != 8 && d->patch != 16) return error(SGN_ERR_INVALID_ARGUMENT, "patch must be 4, 8 or 16");
    if (d->width < 8 || d->height < 8 || d->width > 16384 || d->height > 16384 || d->width < d->patch || d->height < d->patch)
        return error(SGN_ERR_INVALID_ARGUMENT, "image size %dx%d not supported", d->width, d->height);
    if (!(d->image_dtype >= SGN_F32 && d->image_dtype <= SGN_BF16G))
        return error(SGN_ERR_INVALID_ARGUMENT, "unknown image dtype");
    if (!(d->huber_k > 0.0f) || !std::isfinite(d->huber_k) || !(d->lm_lambda >= 0.0f) || !std::isfinite(d->lm_lambda) ||
        std::isnan(d->fp64_cond) || (d->optimize_normal != 0 && d->optimize_normal != 1) || d->min_residuals < 0 ||
        (d->lm_adaptive != 0 && d->lm_adaptive != 1) || d->surfel_radius != 0.0f)
        return error(SGN_ERR_INVALID_ARGUMENT, "invalid solver options in desc");
    if (num_frames < 1 || num_frames > SGN_MAX_FRAMES) return error(SGN_ERR_INVALID_ARGUMENT, "num_frames outside [1, %d]", SGN_MAX_FRAMES);
    if (iters < 0 || iters > 100000) return error(SGN_ERR_INVALID_ARGUMENT, "iters outside [0, 100000]");
    const double fx = intrinsics[0], fy = intrinsics[1], cx = intrinsics[2], cy = intrinsics[3];
    if (!(fx > 0) || !(fy > 0) || !std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(cx) || !std::isfinite(cy))
        return error(SGN_ERR_INVALID_ARGUMENT, "intrinsics must be finite with fx, fy > 0");
    const int W = d->width, H = d->height, P = d->patch, F = num_frames;
    if (keyframe_pitch_bytes < size_t(W) * 4 || keyframe_pitch_bytes % 4 || frame_pitch_bytes < size_t(W) * 4 || frame_pitch_bytes % 4)
        return error(SGN_ERR_INVALID_ARGUMENT, "pitches must be multiples of 4 bytes and at least 4 W");
    for (int f = 0; f < F; ++f) {
        if (!frames[f]) return error(SGN_ERR_INVALID_ARGUMENT, "frame %d pointer is NULL", f);
        if (!is_rotation(poses + 12 * f)) return error(SGN_ERR_INVALID_ARGUMENT, "pose %d is not a finite rigid motion", f);
    }
    const void* dev_ptrs[] = {keyframe, inv_depth0, normal0, state0, inv_depth, normal, cost, nres, status, depth_map, surfel_index};
    for (const void* p : dev_ptrs)
        if (!p) return error(SGN_ERR_INVALID_ARGUMENT, "an input or output pointer is NULL (all are required)");
    const int tex_pitch = (W + 31) / 32 * 32;
    const size_t need = size_t(F) * H * tex_pitch * sgn::texel_bytes(d->image_dtype);
    if (need > SGN_STATIC_SCRATCH_BYTES)
        return error(SGN_ERR_WORKSPACE_TOO_SMALL,
                     "%d frames of %dx%d texels need %zu bytes; the static scratch holds %u (use a plan with a workspace)",
                     F, W, H, need, unsigned(SGN_STATIC_SCRATCH_BYTES));
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return error(SGN_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return error(SGN_ERR_INVALID_ARGUMENT, "device ordinal %d not supported", dev);
    for (const void* p : dev_ptrs)
        if (!on_device(p, dev))
            return error(SGN_ERR_INVALID_ARGUMENT, "inputs and outputs must be memory of the current device (%d)", dev);
    for (int f = 0; f < F; ++f)
        if (!on_device(frames[f], dev)) return error(SGN_ERR_INVALID_ARGUMENT, "frame %d is not memory of the current device", f);
    void* scratch = nullptr;
    sgn_status st = scratch_address(dev, &scratch);
    if (st != SGN_OK) return st;

    // ---- plan parameters over the caller's buffers and the static texel planes
    sgn::PlanParams pp{};
    pp.W = W;
    pp.H = H;
    pp.P = P;
    pp.TX = W / P;
    pp.TY = H / P;
    pp.S = pp.TX * pp.TY;
    pp.F = F;
    pp.dtype = d->image_dtype;
    pp.fx = float(fx);
    pp.fy = float(fy);
    pp.cx = float(cx);
    pp.cy = float(cy);
    pp.fx_lo = float(fx - double(pp.fx));
    pp.fy_lo = float(fy - double(pp.fy));
    pp.cx_lo = float(cx - double(pp.cx));
    pp.cy_lo = float(cy - double(pp.cy));
    pp.ifx = float(1.0 / fx);
    pp.ify = float(1.0 / fy);
    pp.huber_k = d->huber_k;
    pp.lm_lambda = d->lm_lambda;
    pp.fp64_cond = d->fp64_cond > 0 ? float(std::fmin(d->fp64_cond, 3.0e38)) : 0.0f;
    pp.optimize_normal = d->optimize_normal;
    pp.min_residuals = d->min_residuals;
    pp.lm_adaptive = d->lm_adaptive;
    pp.radius = 0.0f;  // tiles only: circular surfels need a pixel table and a depth buffer
    pp.kf = keyframe;
    pp.kf_pitch = int(keyframe_pitch_bytes / 4);
    pp.tex = scratch;
    pp.tex_pitch = tex_pitch;
    pp.tex_plane = (long long)H * tex_pitch;
    pp.id0 = inv_depth0;
    pp.n0 = normal0;
    pp.state0 = state0;
    pp.id = inv_depth;
    pp.n = normal;
    pp.cost = cost;
    pp.nres = nres;
    pp.status = status;
    pp.depth = depth_map;
    pp.sidx = surfel_index;
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                const double v = poses[12 * f + 4 * i + j];
                pp.frames[f].R[3 * i + j] = float(v);
                pp.frames[f].R_lo[3 * i + j] = float(v - double(float(v)));
            }
            const double v = poses[12 * f + 4 * i + 3];
            pp.frames[f].t[i] = float(v);
            pp.frames[f].t_lo[i] = float(v - double(float(v)));
        }

    // ---- enqueue: clear the map (pixels outside full tiles keep 0 / -1), prepare frames, solve
    const cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t npx = size_t(W) * H;
    if ((e = cudaMemsetAsync(depth_map, 0, npx * sizeof(float), stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(surfel_index, 0xff, npx * sizeof(int32_t), stream)) != cudaSuccess)
        return error(SGN_ERR_CUDA, "clearing the depth map: %s", cudaGetErrorString(e));
    size_t pitches[SGN_MAX_FRAMES];
    for (int f = 0; f < F; ++f) pitches[f] = frame_pitch_bytes / 4;
    int le = sgn::launch_prep_frames(pp, frames, pitches, 0, F, stream);
    if (le) return error(SGN_ERR_CUDA, "frame preparation launch: %s", cudaGetErrorString(cudaError_t(le)));
    const int lanes = P == 4 ? 8 : (P == 8 ? 16 : 32);
    le = sgn::launch_gn(pp, iters, sgn::kModeSolve, lanes, 256, stream);
    if (le) return error(SGN_ERR_CUDA, "Gauss-Newton launch: %s", cudaGetErrorString(cudaError_t(le)));
    sgn::count_launch(2);
    return SGN_OK;
}
