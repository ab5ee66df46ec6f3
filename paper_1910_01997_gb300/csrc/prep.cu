// Frame preparation, surfel initialisation/seeding and depth-map rendering kernels, and the
// dtype dispatch of the Gauss-Newton launcher.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "sgn_internal.h"

namespace sgn {

int launch_gn_f32(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap);
int launch_gn_f16(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap);
int launch_gn_bf16(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap);
int launch_gn_f16g(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap);
int launch_gn_bf16g(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap);

int launch_gn(const PlanParams& pp, int iters, int mode, int lanes_per_surfel, int block_threads, void* stream,
              const void* tmap) {
    switch (pp.dtype) {
        case SGN_F32: return launch_gn_f32(pp, iters, mode, lanes_per_surfel, block_threads, stream, tmap);
        case SGN_F16: return launch_gn_f16(pp, iters, mode, lanes_per_surfel, block_threads, stream, tmap);
        case SGN_BF16: return launch_gn_bf16(pp, iters, mode, lanes_per_surfel, block_threads, stream, tmap);
        case SGN_F16G: return launch_gn_f16g(pp, iters, mode, lanes_per_surfel, block_threads, stream, tmap);
        case SGN_BF16G: return launch_gn_bf16g(pp, iters, mode, lanes_per_surfel, block_threads, stream, tmap);
        default: return int(cudaErrorInvalidValue);
    }
}

// ------------------------------------------------------------------------------ staging support

namespace {
__device__ unsigned int g_stage_err;  // staging waits that timed out, all plans of this process
constexpr int kMaxDevices = 64;
unsigned int* g_stage_err_addr[kMaxDevices] = {};
std::mutex g_stage_mutex;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}  // namespace

unsigned int* stage_error_word() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    if (!g_stage_err_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_stage_err) != cudaSuccess) return nullptr;
        g_stage_err_addr[dev] = static_cast<unsigned int*>(p);
    }
    return g_stage_err_addr[dev];
}

// The texel planes as a 3-D tensor of 32-bit (FP32 texels) or 16-bit (FP16/BF16 texels) elements,
// 4 per texel: (4 W, H, planes) with byte strides (4 tex_pitch e, tex_plane 4 e); box
// (4 box_w, box_h, 1).  Boxes reaching outside the image are filled with zeros.
int encode_texel_map(void* tmap, const PlanParams& pp, int planes) {
    {
        std::lock_guard<std::mutex> lock(g_stage_mutex);
        if (!g_encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return int(e != cudaSuccess ? e : cudaErrorNotSupported);
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    const bool f32 = pp.dtype == SGN_F32;
    const cuuint64_t esize = f32 ? 4 : 2;
    const cuuint64_t dims[3] = {cuuint64_t(4) * pp.W, cuuint64_t(pp.H), cuuint64_t(planes)};
    const cuuint64_t strides[2] = {cuuint64_t(pp.tex_pitch) * 4 * esize, cuuint64_t(pp.tex_plane) * 4 * esize};
    const cuuint32_t box[3] = {cuuint32_t(4 * box_w(pp.P, pp.dtype)), cuuint32_t(box_h(pp.P)), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = g_encode(static_cast<CUtensorMap*>(tmap), f32 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                                3, const_cast<void*>(pp.tex), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? int(cudaSuccess) : int(cudaErrorInvalidValue);
}

// ------------------------------------------------------------------------------ frame preparation

struct PrepArgs {
    const float* src[kMaxFrames];
    long long src_pitch[kMaxFrames];  // floats
    void* dst;
    long long plane;                  // texels per frame plane
    int tex_pitch;                    // texels per row
    int W, H, first, dtype;
};

// Intensity as stored in the texel type (FP32 in SGN_F32, SGN_F16G and SGN_BF16G; rounded to FP16 / BF16
// in SGN_F16 / SGN_BF16).
__device__ __forceinline__ float stored(float v, int dtype) {
    if (dtype == SGN_F16) return __half2float(__float2half_rn(v));
    if (dtype == SGN_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    return v;
}

// Intensity + central-difference gradient (the grad I of Eq. 8), packed as one texel per pixel:
// (gx, gy, I, I(x + 1, y)) in FP32 (the right neighbour's intensity fills the fourth word, so that a
// bilinear sample blends intensity pairs; 0 past the last column), (gx, gy, I, 0) in FP16/BF16, or
// (gx, gy) then I for the G formats.  The gradient is taken from the intensities
// as stored, so that with FP16/BF16 texels it is the exact central difference of the stored image
// (half the difference of two values on the storage grid fits the storage mantissa); the G formats
// round the FP32 central difference to their gradient type.  Border rows/columns get a zero gradient; the
// validity rule of the warp never samples them.
__global__ void __launch_bounds__(256) k_prep_frames(const __grid_constant__ PrepArgs a) {
    const int f = blockIdx.z;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const long long sp = a.src_pitch[f];
    const float* row = a.src[f] + (long long)y * sp;
    const int dt = a.dtype;
    const float I = stored(__ldg(row + x), dt);
    const float gx = (x >= 1 && x <= a.W - 2) ? 0.5f * (stored(__ldg(row + x + 1), dt) - stored(__ldg(row + x - 1), dt)) : 0.0f;
    const float gy = (y >= 1 && y <= a.H - 2) ? 0.5f * (stored(__ldg(row + x + sp), dt) - stored(__ldg(row + x - sp), dt)) : 0.0f;
    const long long o = (long long)(a.first + f) * a.plane + (long long)y * a.tex_pitch + x;
    if (a.dtype == SGN_F32) {
        const float Ir = x + 1 < a.W ? __ldg(row + x + 1) : 0.0f;
        static_cast<float4*>(a.dst)[o] = make_float4(gx, gy, I, Ir);
    } else if (a.dtype == SGN_F16) {
        __half2 lo = __floats2half2_rn(gx, gy), hi = __floats2half2_rn(I, 0.0f);
        uint2 v;
        v.x = *reinterpret_cast<unsigned*>(&lo);
        v.y = *reinterpret_cast<unsigned*>(&hi);
        static_cast<uint2*>(a.dst)[o] = v;
    } else if (a.dtype == SGN_BF16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(gx, gy), hi = __floats2bfloat162_rn(I, 0.0f);
        uint2 v;
        v.x = *reinterpret_cast<unsigned*>(&lo);
        v.y = *reinterpret_cast<unsigned*>(&hi);
        static_cast<uint2*>(a.dst)[o] = v;
    } else if (a.dtype == SGN_F16G) {
        __half2 g = __floats2half2_rn(gx, gy);
        static_cast<uint2*>(a.dst)[o] = make_uint2(*reinterpret_cast<unsigned*>(&g), __float_as_uint(I));
    } else {
        __nv_bfloat162 g = __floats2bfloat162_rn(gx, gy);
        static_cast<uint2*>(a.dst)[o] = make_uint2(*reinterpret_cast<unsigned*>(&g), __float_as_uint(I));
    }
}

int launch_prep_frames(const PlanParams& pp, const float* const* src, const size_t* src_pitch_floats, int first,
                       int count, void* stream) {
    if (count <= 0) return cudaSuccess;
    PrepArgs a{};
    for (int i = 0; i < count; ++i) {
        a.src[i] = src[i];
        a.src_pitch[i] = (long long)src_pitch_floats[i];
    }
    a.dst = const_cast<void*>(pp.tex);
    a.plane = pp.tex_plane;
    a.tex_pitch = pp.tex_pitch;
    a.W = pp.W;
    a.H = pp.H;
    a.first = first;
    a.dtype = pp.dtype;
    dim3 block(32, 8), grid((pp.W + 31) / 32, (pp.H + 7) / 8, count);
    k_prep_frames<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return int(cudaGetLastError());
}

// ------------------------------------------------------------------------------ device copies

struct CopyArgs {
    CopyJob job[kMaxCopyJobs];
    int n;
};

// blockIdx.z: job; blockIdx.y: rows (grid-stride); x: the row's 16-byte words (grid-stride), or its
// 4-byte words / bytes when the job's addresses and pitches do not allow wider accesses.
__global__ void __launch_bounds__(256) k_copy_jobs(const __grid_constant__ CopyArgs a) {
    const CopyJob& j = a.job[blockIdx.z];
    const uintptr_t al = reinterpret_cast<uintptr_t>(j.dst) | reinterpret_cast<uintptr_t>(j.src) | j.dpitch | j.spitch;
    const size_t x0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x, xs = size_t(gridDim.x) * blockDim.x;
    for (int r = blockIdx.y; r < j.rows; r += gridDim.y) {
        char* d = static_cast<char*>(j.dst) + size_t(r) * j.dpitch;
        const char* s = static_cast<const char*>(j.src) + size_t(r) * j.spitch;
        size_t done = 0;
        if ((al & 15) == 0) {
            const size_t n16 = j.row_bytes / 16;
            for (size_t i = x0; i < n16; i += xs)
                reinterpret_cast<uint4*>(d)[i] = __ldg(reinterpret_cast<const uint4*>(s) + i);
            done = n16 * 16;
        } else if ((al & 3) == 0) {
            const size_t n4 = j.row_bytes / 4;
            for (size_t i = x0; i < n4; i += xs)
                reinterpret_cast<unsigned*>(d)[i] = __ldg(reinterpret_cast<const unsigned*>(s) + i);
            done = n4 * 4;
        }
        for (size_t i = done + x0; i < j.row_bytes; i += xs) d[i] = s[i];
    }
}

int launch_copy_jobs(const CopyJob* jobs, int n, void* stream) {
    if (n <= 0) return cudaSuccess;
    if (n > kMaxCopyJobs) return cudaErrorInvalidValue;
    CopyArgs a{};
    size_t widest = 1;
    int rows = 1;
    for (int i = 0; i < n; ++i) {
        a.job[i] = jobs[i];
        widest = std::max(widest, (jobs[i].row_bytes + 15) / 16);
        rows = std::max(rows, jobs[i].rows);
    }
    a.n = n;
    const unsigned gx = unsigned(std::min<size_t>((widest + 255) / 256, 1024));
    const unsigned gy = unsigned(std::min(rows, 4096));
    k_copy_jobs<<<dim3(gx, gy, n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return int(cudaGetLastError());
}

// ------------------------------------------------------------------------------ surfel state

// Initial working state from the initial surfels.  With seed != 0 every TO_SEED surfel is seeded
// from its 8-connected VALID neighbours (Sec. 2.3): mean of Eq. 3 at its centre ray against each
// neighbour's plane, normalised sum of the neighbours' camera-facing normals.
__global__ void __launch_bounds__(256) k_init_state(const __grid_constant__ PlanParams pp, int seed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= pp.S) return;
    const int st0 = pp.state0[s];
    float id = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;
    int status = SGN_SURFEL_EMPTY;
    if (st0 == SGN_STATE_VALID) {
        id = pp.id0[s];
        nx = pp.n0[3 * s];
        ny = pp.n0[3 * s + 1];
        nz = pp.n0[3 * s + 2];
        status = SGN_SURFEL_OK;
    } else if (st0 == SGN_STATE_TO_SEED) {
        status = SGN_SURFEL_UNSEEDED;
        if (seed) {
            const int TX = pp.TX, P = pp.P;
            const int tx = s % TX, ty = s / TX;
            const float half = 0.5f * float(P - 1);
            const float rx = (float(tx * P) + half - pp.cx) * pp.ifx, ry = (float(ty * P) + half - pp.cy) * pp.ify;
            float sid = 0.0f, snx = 0.0f, sny = 0.0f, snz = 0.0f;
            int cid = 0, cn = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int qx = tx + dx, qy = ty + dy;
                    if ((dx == 0 && dy == 0) || qx < 0 || qy < 0 || qx >= TX || qy >= pp.TY) continue;
                    const int q = qy * TX + qx;
                    if (pp.state0[q] != SGN_STATE_VALID) continue;
                    const float rqx = (float(qx * P) + half - pp.cx) * pp.ifx;
                    const float rqy = (float(qy * P) + half - pp.cy) * pp.ify;
                    const float qnx = pp.n0[3 * q], qny = pp.n0[3 * q + 1], qnz = pp.n0[3 * q + 2];
                    const float rqn = rqx * qnx + rqy * qny + qnz;
                    const float v = pp.id0[q] * (rx * qnx + ry * qny + qnz) / rqn;
                    if (isfinite(v) && v > 0.0f) {
                        sid += v;
                        ++cid;
                    }
                    const float sg = rqn < 0.0f ? 1.0f : -1.0f;
                    snx += sg * qnx;
                    sny += sg * qny;
                    snz += sg * qnz;
                    ++cn;
                }
            const float len = sqrtf(snx * snx + sny * sny + snz * snz);
            if (cid > 0 && cn > 0 && len >= 1e-6f) {
                id = sid / float(cid);
                nx = snx / len;
                ny = sny / len;
                nz = snz / len;
                status = SGN_SURFEL_OK | SGN_SURFEL_SEEDED;
            }
        }
    }
    pp.id[s] = id;
    pp.n[3 * s] = nx;
    pp.n[3 * s + 1] = ny;
    pp.n[3 * s + 2] = nz;
    pp.cost[s] = 0.0f;
    pp.nres[s] = 0;
    pp.status[s] = uint8_t(status);
}

int launch_seed(const PlanParams& pp, void* stream) {
    const int block = 256, grid = (pp.S + block - 1) / block;
    if (grid) k_init_state<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(pp, 1);
    return int(cudaGetLastError());
}

int launch_init_state(const PlanParams& pp, void* stream) {
    const int block = 256, grid = (pp.S + block - 1) / block;
    if (grid) k_init_state<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(pp, 0);
    return int(cudaGetLastError());
}

// ------------------------------------------------------------------------------ depth map

// Per-pixel inverse depth of Eq. 3 from the current surfels (tiles do not overlap, so each pixel
// of a full tile belongs to its tile's surfel), and the generating surfel index (Sec. 2.2).
__global__ void __launch_bounds__(256) k_render_depth(const __grid_constant__ PlanParams pp) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int P = pp.P;
    if (x >= pp.TX * P || y >= pp.TY * P) return;
    const int tx = x / P, ty = y / P, s = ty * pp.TX + tx;
    const int st = pp.status[s] & 0x3f;
    float v = 0.0f;
    int idx = -1;
    if (st != SGN_SURFEL_EMPTY && st != SGN_SURFEL_UNSEEDED) {
        const float half = 0.5f * float(P - 1);
        const float rsx = (float(tx * P) + half - pp.cx) * pp.ifx, rsy = (float(ty * P) + half - pp.cy) * pp.ify;
        const float nx = pp.n[3 * s], ny = pp.n[3 * s + 1], nz = pp.n[3 * s + 2], ids = pp.id[s];
        const float e = ((float(x - tx * P) - half) * pp.ifx * nx + (float(y - ty * P) - half) * pp.ify * ny) /
                        (rsx * nx + rsy * ny + nz);
        const float idu = fmaf(ids, e, ids);
        if (idu > 0.0f && isfinite(idu)) {
            v = idu;
            idx = s;
        }
    }
    pp.depth[(size_t)y * pp.W + x] = v;
    pp.sidx[(size_t)y * pp.W + x] = idx;
}

int launch_render_depth(const PlanParams& pp, void* stream) {
    dim3 block(32, 8), grid((pp.TX * pp.P + 31) / 32, (pp.TY * pp.P + 7) / 8);
    if (grid.x && grid.y) k_render_depth<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(pp);
    return int(cudaGetLastError());
}

}  // namespace sgn
