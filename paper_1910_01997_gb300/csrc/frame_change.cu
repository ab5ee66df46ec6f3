// Reference-frame change of surfels (Sec. 2.5, Eq. 10) and the depth-buffered render of free surfels
// (Sec. 2.2: Eq. 3 per pixel, Eq. 4 coverage, nearest surfel kept).
//
// A free surfel is the pixel u_s where its point projects in its reference frame, its inverse depth
// id_s along r_s = K^-1 (u_s, 1) (z = 1) and its unit normal n.  The render replaces the depth buffer
// of a graphics pipeline by a 64-bit atomic maximum per pixel on the key
// (bits of id_u) << 32 | ~surfel index: positive floats order like their bit patterns, so the
// largest inverse depth (the nearest surfel) wins, and for equal inverse depths the larger ~index,
// i.e. the lower index.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "sgn.h"
#include "sgn_internal.h"

namespace {

struct Cam {
    float fx, fy, cx, cy, ifx, ify;
};

struct Pose {
    float R[9], t[3];
};

sgn_status error(sgn_status st, const char* fmt, ...) {
    char buf[320];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return sgn::record_error(st, buf);
}

bool make_cam(const double k[4], Cam* c) {
    if (!k) return false;
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(k[i])) return false;
    if (!(k[0] > 0) || !(k[1] > 0)) return false;
    *c = Cam{float(k[0]), float(k[1]), float(k[2]), float(k[3]), float(1.0 / k[0]), float(1.0 / k[1])};
    return true;
}

bool make_pose(const double* T, Pose* p) {
    if (!T) return false;
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
    if (!(worst <= 1e-6) || !(det > 0.0)) return false;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) p->R[3 * i + j] = float(T[4 * i + j]);
        p->t[i] = float(T[4 * i + 3]);
    }
    return true;
}

bool on_device(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Eq. 10: p1 = R r_s / id_s + t, n1 = R n, u1 = pi(K p1), id1 = 1 / p1_z.
__global__ void __launch_bounds__(256) k_transfer_surfels(const Cam cam, const Pose T, int n,
                                                          const float2* __restrict__ u, const float* __restrict__ id,
                                                          const float* __restrict__ nrm, float2* __restrict__ u_out,
                                                          float* __restrict__ id_out, float* __restrict__ n_out,
                                                          uint8_t* __restrict__ valid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 us = u[i];
    const float ids = id[i];
    const float r0x = (us.x - cam.cx) * cam.ifx, r0y = (us.y - cam.cy) * cam.ify;
    const float inv = 1.0f / ids;
    const float px = r0x * inv, py = r0y * inv, pz = inv;
    float p1[3], n1[3];
    const float nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p1[k] = fmaf(T.R[3 * k], px, fmaf(T.R[3 * k + 1], py, fmaf(T.R[3 * k + 2], pz, T.t[k])));
        n1[k] = fmaf(T.R[3 * k], nx, fmaf(T.R[3 * k + 1], ny, T.R[3 * k + 2] * nz));
    }
    const bool ok = ids > 0.0f && isfinite(ids) && p1[2] > 0.0f && isfinite(p1[2]);
    const float iz = 1.0f / p1[2];
    u_out[i] = ok ? make_float2(fmaf(cam.fx, p1[0] * iz, cam.cx), fmaf(cam.fy, p1[1] * iz, cam.cy)) : make_float2(0.f, 0.f);
    id_out[i] = ok ? iz : 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) n_out[3 * i + k] = ok ? n1[k] : 0.0f;
    valid[i] = ok ? 1 : 0;
}

// The lanes of one warp draw surfel i: they sweep the pixel box around its disc of radius r.  Eq. 3
// is taken in the tile-local form id_u = id_s (1 + ((r_u - r_s) . n) / (r_s . n)), which has no
// cancellation for pixels near the surfel's centre.
__device__ __forceinline__ void draw_surfel(const Cam& cam, int W, int H, float2 us, float ids, float nx, float ny,
                                            float nz, float radius, int i, int lane, unsigned long long* zbuf) {
    const float rsx = (us.x - cam.cx) * cam.ifx, rsy = (us.y - cam.cy) * cam.ify;
    const float rsn = fmaf(rsx, nx, fmaf(rsy, ny, nz));
    const float inv_rsn = 1.0f / rsn;
    if (!(ids > 0.0f) || !isfinite(ids) || !isfinite(inv_rsn)) return;
    // pixel box; clamped in float first so that far-off surfels do not overflow the integer range
    const float bx0 = fmaxf(floorf(us.x - radius), 0.0f), bx1 = fminf(ceilf(us.x + radius), float(W - 1));
    const float by0 = fmaxf(floorf(us.y - radius), 0.0f), by1 = fminf(ceilf(us.y + radius), float(H - 1));
    if (!(bx0 <= bx1) || !(by0 <= by1)) return;
    const int x0 = int(bx0), y0 = int(by0), bw = int(bx1) - x0 + 1, bh = int(by1) - y0 + 1;
    const float r2 = radius * radius;
    const unsigned lo = ~unsigned(i);
    for (int k = lane; k < bw * bh; k += 32) {
        const int x = x0 + k % bw, y = y0 + k / bw;
        const float dx = float(x) - us.x, dy = float(y) - us.y;
        if (!(fmaf(dx, dx, dy * dy) < r2)) continue;
        const float e = fmaf(dx * cam.ifx, nx, dy * cam.ify * ny) * inv_rsn;
        const float v = fmaf(ids, e, ids);
        if (!(v > 0.0f) || !isfinite(v)) continue;
        const unsigned long long key = (static_cast<unsigned long long>(__float_as_uint(v)) << 32) | lo;
        atomicMax(zbuf + size_t(y) * W + x, key);
    }
}

// One warp per free surfel.
__global__ void __launch_bounds__(256) k_render_surfels(const Cam cam, int W, int H, int n, const float2* __restrict__ u,
                                                        const float* __restrict__ id, const float* __restrict__ nrm,
                                                        const uint8_t* __restrict__ valid, float radius,
                                                        unsigned long long* __restrict__ zbuf) {
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (i >= n || !valid[i]) return;
    draw_surfel(cam, W, H, u[i], id[i], nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2], radius, i, lane, zbuf);
}

// One warp per surfel of a plan with circular surfels: centre = tile centre, drawn unless EMPTY or
// UNSEEDED.  The same draw as k_render_surfels, so the map equals the render of the plan's surfels
// as free surfels.
__global__ void __launch_bounds__(256) k_render_plan_discs(const Cam cam, const __grid_constant__ sgn::PlanParams pp) {
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (s >= pp.S) return;
    const int st = pp.status[s] & 0x3f;
    if (st == SGN_SURFEL_EMPTY || st == SGN_SURFEL_UNSEEDED) return;
    const float half = 0.5f * float(pp.P - 1);
    const float2 us = make_float2(float((s % pp.TX) * pp.P) + half, float((s / pp.TX) * pp.P) + half);
    draw_surfel(cam, pp.W, pp.H, us, pp.id[s], pp.n[3 * s], pp.n[3 * s + 1], pp.n[3 * s + 2], pp.radius, s, lane,
                pp.zbuf);
}

__global__ void __launch_bounds__(256) k_resolve_depth(int npx, const unsigned long long* __restrict__ zbuf,
                                                       float* __restrict__ depth, int32_t* __restrict__ sidx) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npx) return;
    const unsigned long long key = zbuf[k];
    depth[k] = key ? __uint_as_float(unsigned(key >> 32)) : 0.0f;
    sidx[k] = key ? int(~unsigned(key & 0xffffffffu)) : -1;
}

}  // namespace

extern "C" sgn_status sgn_transfer_surfels(const double intrinsics[4], const double T_kf1_kf0[12], int n,
                                           const float* u, const float* inv_depth, const float* normal, float* u_out,
                                           float* inv_depth_out, float* normal_out, uint8_t* valid, void* stream) {
    Cam cam;
    Pose T;
    if (!make_cam(intrinsics, &cam)) return error(SGN_ERR_INVALID_ARGUMENT, "intrinsics must be finite with fx, fy > 0");
    if (!make_pose(T_kf1_kf0, &T)) return error(SGN_ERR_INVALID_ARGUMENT, "T_kf1_kf0 is not a finite rigid motion");
    if (n < 0) return error(SGN_ERR_INVALID_ARGUMENT, "n < 0");
    if (n == 0) return SGN_OK;
    const void* ptrs[] = {u, inv_depth, normal, u_out, inv_depth_out, normal_out, valid};
    for (const void* p : ptrs)
        if (!p || !on_device(p)) return error(SGN_ERR_INVALID_ARGUMENT, "surfel arrays must be non-NULL device memory");
    if (reinterpret_cast<uintptr_t>(u) % 8 || reinterpret_cast<uintptr_t>(u_out) % 8)
        return error(SGN_ERR_INVALID_ARGUMENT, "u and u_out must be 8-byte aligned (float pairs)");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_transfer_surfels<<<(n + 255) / 256, 256, 0, st>>>(cam, T, n, reinterpret_cast<const float2*>(u), inv_depth, normal,
                                                        reinterpret_cast<float2*>(u_out), inv_depth_out, normal_out, valid);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return error(SGN_ERR_CUDA, "transfer launch: %s", cudaGetErrorString(e));
    sgn::count_launch();
    return SGN_OK;
}

extern "C" sgn_status sgn_render_surfels(const double intrinsics[4], int width, int height, int n, const float* u,
                                         const float* inv_depth, const float* normal, const uint8_t* valid, float radius,
                                         uint64_t* zbuffer, float* inv_depth_map, int32_t* surfel_index, void* stream) {
    Cam cam;
    if (!make_cam(intrinsics, &cam)) return error(SGN_ERR_INVALID_ARGUMENT, "intrinsics must be finite with fx, fy > 0");
    if (width < 1 || height < 1 || width > 16384 || height > 16384)
        return error(SGN_ERR_INVALID_ARGUMENT, "image size %dx%d not supported", width, height);
    if (n < 0) return error(SGN_ERR_INVALID_ARGUMENT, "n < 0");
    if (!(radius > 0.0f) || !(radius <= 1024.0f)) return error(SGN_ERR_INVALID_ARGUMENT, "radius must be in (0, 1024]");
    const void* maps[] = {zbuffer, inv_depth_map, surfel_index};
    for (const void* p : maps)
        if (!p || !on_device(p)) return error(SGN_ERR_INVALID_ARGUMENT, "zbuffer and output maps must be non-NULL device memory");
    if (n > 0) {
        const void* ptrs[] = {u, inv_depth, normal, valid};
        for (const void* p : ptrs)
            if (!p || !on_device(p)) return error(SGN_ERR_INVALID_ARGUMENT, "surfel arrays must be non-NULL device memory");
        if (reinterpret_cast<uintptr_t>(u) % 8) return error(SGN_ERR_INVALID_ARGUMENT, "u must be 8-byte aligned (float pairs)");
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t npx = size_t(width) * height;
    cudaError_t e = cudaMemsetAsync(zbuffer, 0, npx * sizeof(uint64_t), st);
    if (e != cudaSuccess) return error(SGN_ERR_CUDA, "clearing the depth buffer: %s", cudaGetErrorString(e));
    if (n > 0) {
        k_render_surfels<<<(n + 7) / 8, 256, 0, st>>>(cam, width, height, n, reinterpret_cast<const float2*>(u), inv_depth,
                                                      normal, valid, radius, reinterpret_cast<unsigned long long*>(zbuffer));
        if ((e = cudaGetLastError()) != cudaSuccess) return error(SGN_ERR_CUDA, "render launch: %s", cudaGetErrorString(e));
    }
    k_resolve_depth<<<int((npx + 255) / 256), 256, 0, st>>>(int(npx), reinterpret_cast<const unsigned long long*>(zbuffer),
                                                             inv_depth_map, surfel_index);
    if ((e = cudaGetLastError()) != cudaSuccess) return error(SGN_ERR_CUDA, "resolve launch: %s", cudaGetErrorString(e));
    sgn::count_launch(n > 0 ? 2 : 1);
    return SGN_OK;
}

namespace sgn {

int disc_pixels(int P, float radius, int* out_xy) {
    const double c = 0.5 * (P - 1), r = double(radius);
    const int lo = int(std::floor(c - r)) - 1, hi = int(std::ceil(c + r)) + 1;
    int n = 0;
    for (int y = lo; y <= hi; ++y)
        for (int x = lo; x <= hi; ++x) {
            const double dx = x - c, dy = y - c;
            if (!(std::sqrt(dx * dx + dy * dy) < r)) continue;
            if (n == kMaxDiscPixels) return -1;
            if (out_xy) {
                out_xy[2 * n] = x;
                out_xy[2 * n + 1] = y;
            }
            ++n;
        }
    return n;
}

int launch_render_discs(const PlanParams& pp, void* stream) {
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t npx = size_t(pp.W) * pp.H;
    cudaError_t e = cudaMemsetAsync(pp.zbuf, 0, npx * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return int(e);
    const Cam cam{pp.fx, pp.fy, pp.cx, pp.cy, pp.ifx, pp.ify};
    if (pp.S > 0) k_render_plan_discs<<<(pp.S + 7) / 8, 256, 0, st>>>(cam, pp);
    if ((e = cudaGetLastError()) != cudaSuccess) return int(e);
    k_resolve_depth<<<int((npx + 255) / 256), 256, 0, st>>>(int(npx), pp.zbuf, pp.depth, pp.sidx);
    return int(cudaGetLastError());
}

}  // namespace sgn
