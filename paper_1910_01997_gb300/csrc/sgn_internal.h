// Internal definitions shared by the host runtime (api.cpp) and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include "sgn.h"

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
    FramePose frames[kMaxFrames];
};

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
int launch_gn(const PlanParams& pp, int iters, int mode, int lanes_per_surfel, int block_threads, void* stream);
int launch_seed(const PlanParams& pp, void* stream);
int launch_init_state(const PlanParams& pp, void* stream);
int launch_render_depth(const PlanParams& pp, void* stream);

// Batched persistent execution (batch.cu).
struct WorkItem {
    int plan;     // index into the plan table
    int first;    // first surfel
    int count;    // number of surfels
    int pad;
};
// variant 0: lanes per surfel P4->8, P8->16, P16->32; variant 1: P4->16, P8->32, P16->32.
int launch_gn_batch(const PlanParams* d_plans, const WorkItem* d_items, int n_items, int* d_counter, int iters,
                    int variant, int grid, int block_threads, void* stream);
int batch_blocks_per_sm(int variant, int block_threads);
int lanes_for_patch(int variant, int P);

void count_launch(uint64_t n = 1);
// Sets the calling thread's sgn_last_error() message and returns st.
sgn_status record_error(sgn_status st, const char* message);

}  // namespace sgn
