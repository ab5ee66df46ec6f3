// Internal definitions shared by the host runtime (api.cpp) and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include "sgn.h"

#if defined(__CUDACC__)
#define SGN_HD __host__ __device__
#else
#define SGN_HD
#endif

namespace sgn {

constexpr int kMaxFrames = SGN_MAX_FRAMES;
constexpr size_t kAlign = 256;

// Pose of one observing frame (Eq. 6): X_frame = R X_keyframe + t, R row-major.  Each entry is
// the double-precision value split into a float pair, value = hi + lo (used where a tile centre is
// projected precisely); the kernels' per-pixel arithmetic uses hi alone.
struct FramePose {
    float R[9];
    float t[3];
    float R_lo[9];
    float t_lo[3];
};

// Per surfel and frame: the tile centre projected at the reference inverse depth in double-float
// arithmetic, U_ref = (X_int + X_frac, Y_int + Y_frac), with the centre point q_ref = R r_s + t id_ref,
// 1 / q_ref_z and e = (fx (t_x q_z - q_x t_z), fy (t_y q_z - q_y t_z)) for the per-iteration update.
constexpr int kRefWords = 10;
// Per surfel and frame, the Gauss-Newton kernels keep in shared memory the kRefWords reference words
// (padded to 12) and the frame's local projective map of the current pass (24 words, 16-byte
// aligned): kFrameWords floats per frame.  A group's scratch holds F frames plus 4 words of padding,
// so that the groups of a warp read different shared-memory banks.
constexpr int kMapOffset = 12;
constexpr int kMapWords = 24;
constexpr int kFrameWords = kMapOffset + kMapWords;
SGN_HD constexpr int group_scratch_words(int F) { return F * kFrameWords + 4; }

// Surfels of a plain launch by block: a block's `groups` surfels are an sqx x sqy square of
// neighbouring tiles (sqx = 2, 2, 4, 4, 8 for 2, 4, 8, 16, 32 groups), so that the warped footprints
// that the SM's resident blocks gather overlap and stay in its L1 cache across iterations (a row
// strip of the same tiles covers more texels).  Squares past the right or bottom tile edge have
// groups without a tile (-1).
SGN_HD constexpr int square_w(int groups) { return groups >= 32 ? 8 : groups >= 8 ? 4 : groups >= 2 ? 2 : 1; }
SGN_HD constexpr int square_blocks(int TX, int TY, int groups) {
    const int sqx = square_w(groups), sqy = groups / sqx;
    return ((TX + sqx - 1) / sqx) * ((TY + sqy - 1) / sqy);
}
SGN_HD constexpr int square_surfel(int TX, int TY, int groups, int block, int group) {
    const int sqx = square_w(groups), sqy = groups / sqx;
    const int nsx = (TX + sqx - 1) / sqx;
    const int x = (block % nsx) * sqx + group % sqx, y = (block / nsx) * sqy + group / sqx;
    return x < TX && y < TY ? y * TX + x : -1;
}

// Everything a kernel needs to solve the surfels of one keyframe problem.
// Lives in kernel parameters (plain launch) or in a device table (batched launch); kernels
// copy it to shared memory before use.
struct PlanParams {
    // geometry
    int W, H, P, TX, TY, S;
    int F;              // frames in use
    int dtype;          // sgn_dtype
    float fx, fy, cx, cy;
    float fx_lo, fy_lo, cx_lo, cy_lo;  // double value = float pair (fx + fx_lo, ...)
    float ifx, ify;     // 1 / fx, 1 / fy
    // options
    float huber_k;
    float lm_lambda;
    float fp64_cond;    // <= 0: never route to FP64
    int optimize_normal;
    int min_residuals;
    int lm_adaptive;    // Marquardt schedule (see sgn_plan_desc)
    // device buffers (inside the plan's workspace)
    const float* kf;            // keyframe intensity, H rows of kf_pitch floats
    int kf_pitch;
    const void* tex;            // frame texels: F planes of H rows of tex_pitch texels
    int tex_pitch;              // texels per row
    long long tex_plane;        // texels per frame plane
    const float* id0;           // initial surfels (S), normals SoA (3 x S), states (S)
    const float* n0;
    const uint8_t* state0;
    float* id;                  // working / result surfels
    float* n;                   // SoA 3 x S
    float* cost;
    int32_t* nres;
    uint8_t* status;
    float* depth;               // W x H, tightly packed
    int32_t* sidx;
    unsigned int* stage_err;    // device counter of staging waits that timed out (library-wide)
    // circular surfels (radius > 0): the disc's pixels as (x, y) offsets from the tile origin,
    // disc_n pairs; a depth buffer of W x H keys for the render of the discs
    float radius;
    int disc_n;
    const int* disc;
    unsigned long long* zbuf;
    FramePose frames[kMaxFrames];
};

// 32-bit words of a PlanParams up to and including the poses of its first F frames (the part a kernel
// copies into shared memory).
static_assert(sizeof(PlanParams) % 4 == 0 && sizeof(FramePose) % 4 == 0, "plan params are copied as words");
SGN_HD constexpr int plan_words(int F) {
    return int((offsetof(PlanParams, frames) + size_t(F < 0 ? 0 : (F > kMaxFrames ? kMaxFrames : F)) * sizeof(FramePose)) / 4);
}

// ---- shared-memory staging of frame texels
// Each (surfel, frame) stages a box of texels around the tile centre's reference projection
// U_ref = (X_int + X_frac, Y_int + Y_frac): rows Y_int - R .. Y_int + R + 1 and columns from
// X_int - R (rounded down to even for 8-byte texels, so that a TMA row starts on 16 bytes) over
// box_w texels.  R = P / 2 + 1 leaves a margin of at least one pixel around the footprint of a P x P
// tile at unit scale; samples outside the box read global memory.
SGN_HD constexpr int box_radius(int P) { return P / 2 + 1; }
SGN_HD constexpr int box_h(int P) { return 2 * box_radius(P) + 2; }
SGN_HD constexpr int box_w(int P, int dtype) { return dtype == SGN_F32 ? 2 * box_radius(P) + 2 : 2 * box_radius(P) + 4; }
SGN_HD constexpr int box_bytes(int P, int dtype) { return box_w(P, dtype) * box_h(P) * (dtype == SGN_F32 ? 16 : 8); }
SGN_HD constexpr int box_stride(int P, int dtype) { return (box_bytes(P, dtype) + 127) / 128 * 128; }
constexpr int kStageSlots = 2;  // boxes in flight per surfel (double buffering)
constexpr int kTensorMapBytes = 128;

// Circular surfels: at most this many pixels per disc (radius up to about 12.7).
constexpr int kMaxDiscPixels = 512;
// Pixels (x, y offsets from the tile origin, row-major) strictly within `radius` of the tile centre
// ((P - 1) / 2, (P - 1) / 2) (Eq. 4); returns the count (or -1 when more than kMaxDiscPixels).
int disc_pixels(int P, float radius, int* out_xy);
// Depth-buffered render of a plan's circular surfels (tile centres, status not EMPTY/UNSEEDED) into
// pp.depth / pp.sidx using pp.zbuf.  Returns cudaError_t cast to int.
int launch_render_discs(const PlanParams& pp, void* stream);

// Encodes the TMA descriptor of a plan's texel planes (planes frames of H rows, 4 components per
// texel) with the staging box of patch P into tmap (kTensorMapBytes, 64-byte aligned host memory).
// Returns cudaError_t cast to int.
int encode_texel_map(void* tmap, const PlanParams& pp, int planes);
// Device address of the library-wide staging timeout counter on the current device (nullptr on error).
unsigned int* stage_error_word();

// Texel element sizes per dtype.
inline int texel_bytes(int dtype) { return dtype == SGN_F32 ? 16 : 8; }

// Kernel modes of the Gauss-Newton kernel.
enum GnMode : int {
    kModeRun = 0,     // continue from the working state (id, n, status)
    kModeSolve = 1,   // seed from the initial surfels, then iterate (whole path)
};

// Launchers (defined in the .cu files). All return cudaError_t cast to int.
int launch_prep_frames(const PlanParams& pp, const float* const* src, const size_t* src_pitch_floats, int first,
                       int count, void* stream);
// tmap: host copy of the texel TMA descriptor (encode_texel_map), or nullptr for direct gathers.
int launch_gn(const PlanParams& pp, int iters, int mode, int lanes_per_surfel, int block_threads, void* stream,
              const void* tmap = nullptr);
int launch_seed(const PlanParams& pp, void* stream);

// Device-side copies (stream-ordered like cudaMemcpyAsync, but up to kMaxCopyJobs ranges in one
// kernel launch): job j copies `rows` rows of `row_bytes` bytes from src (row stride spitch bytes)
// to dst (row stride dpitch bytes).  Both sides must be device-accessible.
struct CopyJob {
    void* dst;
    const void* src;
    size_t dpitch, spitch, row_bytes;
    int rows;
};
constexpr int kMaxCopyJobs = 8;
int launch_copy_jobs(const CopyJob* jobs, int n, void* stream);
int launch_init_state(const PlanParams& pp, void* stream);
int launch_render_depth(const PlanParams& pp, void* stream);

// Batched persistent execution (batch.cu).
struct WorkItem {
    int plan;     // index into the plan table
    int first;    // first surfel
    int count;    // number of surfels
    int pad;
};
// Solver kinds of batched execution: one persistent kernel per kind present in a batch, each over a
// contiguous range of the work list.
enum BatchKind : int {
    kBatchFixed = 0,     // square surfels, fixed damping
    kBatchAdaptive = 1,  // square surfels, Marquardt schedule (lm_adaptive)
    kBatchDisc = 2,      // circular surfels (surfel_radius > 0)
    kBatchKinds = 3
};
inline int batch_kind(const PlanParams& pp) { return pp.disc_n > 0 ? kBatchDisc : (pp.lm_adaptive ? kBatchAdaptive : kBatchFixed); }
// variant (fixed damping only; the other kinds use variant 0): lanes per surfel P4->8, P8->16,
// P16->32 (0) or P4->16, P8->32, P16->32 (1); circular surfels take one warp per surfel.
// max_frames: the largest frame count of the batch's plans (sizes the shared-memory scratch).
int launch_gn_batch(int kind, const PlanParams* d_plans, const WorkItem* d_items, int n_items, int* d_counter, int iters,
                    int variant, int grid, int block_threads, int max_frames, void* stream);
int batch_blocks_per_sm(int kind, int variant, int block_threads, int max_frames);
int lanes_for_patch(int variant, int P);
// Square items of a fixed-damping plan under schedule variant 2 (a block's square of tiles each).
int square_items(int P, int TX, int TY);

void count_launch(uint64_t n = 1);
// Sets the calling thread's sgn_last_error() message and returns st.
sgn_status record_error(sgn_status st, const char* message);

}  // namespace sgn
