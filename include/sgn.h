/*
 * sgn.h -- C ABI of libsgn, a CUDA (sm_103a) implementation of per-surfel Gauss-Newton
 * photometric optimisation for dense monocular depth and normal estimation
 * ("Dense monocular SLAM by direct surfel optimization", Sec. 2).
 *
 * Model.  A keyframe of W x H pixels is cut into P x P tiles; tile s = ty * (W / P) + tx
 * (row-major, full tiles only) is surfel s.  A surfel is a plane given by its inverse depth
 * id_s along the ray r_s = K^-1 (u_s, 1) of the tile centre u_s = (tx P + (P-1)/2,
 * ty P + (P-1)/2) and its unit normal n_s, both in keyframe camera coordinates (Sec. 2.1,
 * Eq. 1).  Pixel centres sit at integer coordinates.  Observing frames n = 0..F-1 come with
 * the pose T = [R | t] (row-major 3 x 4, doubles) that maps keyframe points into frame
 * coordinates.  The library minimises, per surfel, the Huber-normed photometric error of
 * Eq. 5 over the tile's pixels warped into every frame through the plane (Eq. 6), by
 * Levenberg-Marquardt damped Gauss-Newton steps on (two tangent directions of n_s, id_s)
 * (Eqs. 7-9, Sec. 2.4), seeds new surfels from their neighbours (Sec. 2.3) and renders the
 * per-pixel inverse depth of Eq. 3 (Sec. 2.2).
 *
 * Memory.  The caller owns all memory.  A plan describes one keyframe problem; the caller
 * asks sgn_plan_workspace_bytes() for the device workspace size, allocates it (any
 * allocator) and binds it with a CUDA stream.  libsgn allocates no device memory.  Host
 * pointers passed in stay owned by the caller; copies from/to host memory are enqueued on
 * the bound stream (page-locked host memory makes them asynchronous), so host buffers must
 * stay valid until sgn_sync() returns.  Device pointers passed in must stay valid until
 * the work that reads them has run (sgn_sync() or a stream synchronisation).
 *
 * Errors.  Every call returns an sgn_status.  Arguments are validated on the host before
 * anything is enqueued; a rejected call changes nothing.  Asynchronous CUDA errors surface
 * as SGN_ERR_CUDA at the next call that checks the stream (sgn_sync, reads).  A
 * human-readable message for the last failure of the calling thread is available from
 * sgn_last_error().  Per-surfel numerical outcomes are status codes, not errors.
 *
 * Threads.  A plan (and a batch) must be used by one host thread at a time.
 */
#ifndef SGN_H
#define SGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGN_MAX_FRAMES 16
#define SGN_ABI_VERSION 4

typedef enum {
    SGN_OK = 0,
    SGN_ERR_INVALID_ARGUMENT = -1,   /* a size, pointer, pitch, pose or option is not acceptable */
    SGN_ERR_NOT_BOUND = -2,          /* the plan has no workspace/stream yet */
    SGN_ERR_WORKSPACE_TOO_SMALL = -3,
    SGN_ERR_CUDA = -4,               /* a CUDA runtime call or kernel failed */
    SGN_ERR_TIMEOUT = -5,            /* sgn_sync deadline passed, or a device-side wait gave up */
    SGN_ERR_ADMISSION = -6,          /* a request does not fit the memory budget */
    SGN_ERR_STATE = -7               /* call out of order (e.g. run before intrinsics/frames) */
} sgn_status;

/* Frame texel storage (intensity I and central-difference gradient gx, gy of each pixel):
 *   SGN_F32   16-byte texel, all three in FP32;
 *   SGN_F16   8-byte texel, all three in FP16 (the gradient is the central difference of the FP16 image);
 *   SGN_BF16  8-byte texel, all three in BF16 (likewise);
 *   SGN_F16G  8-byte texel, gradient in FP16 and intensity in FP32 (the gradient is the central
 *             difference of the FP32 image, rounded to FP16);
 *   SGN_BF16G 8-byte texel, gradient in BF16 and intensity in FP32.
 * The residual of Eq. 5 is a difference of intensities, so rounding the stored intensity moves the
 * cost minimum itself, while a rounded gradient only perturbs the Jacobian (Eq. 8); the G formats
 * keep the 8-byte texel of the reduced-precision formats with the intensity exact. */
typedef enum { SGN_F32 = 0, SGN_F16 = 1, SGN_BF16 = 2, SGN_F16G = 3, SGN_BF16G = 4 } sgn_dtype;
typedef enum { SGN_HOST = 0, SGN_DEVICE = 1 } sgn_mem;              /* where a pointer points */

/* Surfel input states (sgn_init_surfels). */
enum { SGN_STATE_EMPTY = 0, SGN_STATE_VALID = 1, SGN_STATE_TO_SEED = 2 };

/* Per-surfel result status: low 6 bits = outcome, high bits = flags. */
enum {
    SGN_SURFEL_OK = 0,               /* last iteration took a step (or no iterations were run) */
    SGN_SURFEL_EMPTY = 1,            /* not a surfel */
    SGN_SURFEL_UNSEEDED = 2,         /* TO_SEED but no VALID neighbour gave a value */
    SGN_SURFEL_UNDERDETERMINED = 3,  /* last iteration had fewer than min_residuals valid samples */
    SGN_SURFEL_SINGULAR = 4,         /* damped normal matrix not positive definite */
    SGN_SURFEL_STEP_REJECTED = 5,    /* step gave id_s <= 0 or a non-finite value; kept old values */
    SGN_SURFEL_SEEDED = 0x40,        /* parameters came from neighbour seeding */
    SGN_SURFEL_FP64 = 0x80           /* at least one normal-equation solve ran in FP64 */
};

typedef struct {
    int width, height;        /* keyframe and frame size, pixels; >= 8 and <= 16384 */
    int patch;                /* P: 4, 8 or 16 */
    int max_frames;           /* frame slots, 1..SGN_MAX_FRAMES */
    sgn_dtype image_dtype;    /* storage of frame intensity + gradient texels */
    float huber_k;            /* Huber threshold on intensity residuals (intensities in [0,1]); default 9/255 */
    float lm_lambda;          /* Marquardt damping: H + lm_lambda diag(m, m, H33), m = (H11+H22)/2; default 1e-3 */
    double fp64_cond;         /* solve in FP64 when cond2 of the Jacobi-scaled H exceeds this; <= 0: never; default 1e6 */
    int optimize_normal;      /* 1; 0 = depth-only ablation (d id_u / d n := 0, Sec. 4.4) */
    int min_residuals;        /* fewer valid samples than this: no update; default 8 */
    int lm_adaptive;          /* 0 (default): fixed damping lm_lambda.  1: Marquardt schedule starting at
                                 lm_lambda: a step is kept when the mean Huber cost over valid samples
                                 decreases (lambda / 10), otherwise dropped (lambda x 10); a singular system
                                 or an unusable step counts as dropped; lambda stays in [1e-7, 1e7]; one
                                 extra cost evaluation per solve.  Such plans run without texel staging,
                                 with square surfels (in a batch or a server: their own persistent
                                 launch, with the lane mapping of schedule variant 0) */
    float surfel_radius;      /* 0 (default): surfel s is its P x P tile.  In [0.5, 16]: surfel s is the set
                                 of pixels whose centre lies strictly within this radius of its tile centre
                                 (the paper's circular surfel, Eq. 4; at most 512 pixels); discs of
                                 neighbouring tiles may overlap, and the depth map is then the
                                 depth-buffered render of the discs (Sec. 2.2, as sgn_render_surfels).
                                 Such plans use 32 lanes per surfel (in a batch or a server: their own
                                 persistent launch) and cannot be solved by sgn_solve_static */
} sgn_plan_desc;

typedef struct sgn_plan sgn_plan;     /* opaque, host side */
typedef struct sgn_batch sgn_batch;   /* opaque, host side */

/* Fill *desc with the defaults above for the given size. */
sgn_status sgn_plan_desc_default(sgn_plan_desc* desc, int width, int height, int patch, int max_frames);

/* Create / destroy a plan.  Creation validates desc and allocates host memory only. */
sgn_status sgn_plan_create(const sgn_plan_desc* desc, sgn_plan** out);
sgn_status sgn_plan_destroy(sgn_plan* plan);

/* Number of surfels S = (W / P) * (H / P). */
sgn_status sgn_plan_num_surfels(const sgn_plan* plan, int* num_surfels);

/* Device workspace bytes the plan needs (256-byte aligned base required). */
sgn_status sgn_plan_workspace_bytes(const sgn_plan* plan, size_t* bytes);

/* Kernel mapping of sgn_run / sgn_solve: lanes per surfel (P=4: 8 or 16; P=8: 8, 16 or 32;
 * P=16: 32) and threads per block (multiple of 32 in [32, 256], or 512 for square surfels with
 * 4 pixels per lane (P=8 at 16 lanes), fixed damping and no staging: a block then solves an
 * 8 x 4 square of tiles); 0 selects the default (P=4: 8, P=8: 16, P=16: 32 lanes; 256 threads).
 * Results do not depend on the mapping beyond floating-point summation order. */
sgn_status sgn_plan_set_mapping(sgn_plan* plan, int lanes_per_surfel, int block_threads);

/* Bind a device workspace (>= sgn_plan_workspace_bytes, 256-byte aligned) and a CUDA stream
 * (cudaStream_t; NULL = legacy default stream) on the current device.  Clears the depth map.
 * May be called again to move the plan to another workspace/stream (state is not kept). */
sgn_status sgn_plan_bind(sgn_plan* plan, void* d_workspace, size_t bytes, void* cuda_stream);

/* Pinhole intrinsics, pixels (Eq. 2: r_u = K^-1 (u_x, u_y, 1)).  fx, fy > 0, finite. */
sgn_status sgn_set_intrinsics(sgn_plan* plan, double fx, double fy, double cx, double cy);

/* Keyframe intensity I_kf (Eq. 5): W x H floats, rows pitch_bytes apart (>= 4 W). */
sgn_status sgn_set_keyframe(sgn_plan* plan, const float* img, size_t pitch_bytes, sgn_mem mem);

/* Observing frame `slot` (0 <= slot < max_frames): W x H float intensities, rows pitch_bytes
 * apart, and its pose T_f_kf (12 doubles, row-major [R | t], keyframe -> frame, Eq. 6;
 * R must be a rotation to 1e-6).  Enqueues the frame preparation (central-difference
 * gradients, packed intensity+gradient texels in the plan's image_dtype). */
sgn_status sgn_set_frame(sgn_plan* plan, int slot, const float* img, size_t pitch_bytes, sgn_mem mem,
                         const double T_f_kf[12]);

/* Frames 0..n-1 at once (one preparation launch): imgs[i] as in sgn_set_frame, poses 12 n doubles. */
sgn_status sgn_set_frames(sgn_plan* plan, int n, const float* const* imgs, size_t pitch_bytes, sgn_mem mem,
                          const double* T_f_kf);

/* Number of frames used by the cost (Omega of Eq. 5): 1..max_frames, each must have been set. */
sgn_status sgn_set_num_frames(sgn_plan* plan, int n);

/* Initial surfels: inverse depth (S floats), unit normals (3 S floats, xyz per surfel) and
 * states (S bytes, SGN_STATE_*).  Values of non-VALID surfels are ignored. */
sgn_status sgn_init_surfels(sgn_plan* plan, const float* inv_depth, const float* normal, const uint8_t* state,
                            sgn_mem mem);

/* Sec. 2.3 neighbour seeding, one pass: every TO_SEED surfel takes the mean of Eq. 3 at its
 * centre ray over its 8-connected VALID neighbours (as given to sgn_init_surfels) and the
 * normalised sum of their camera-facing normals.  Enqueued on the stream. */
sgn_status sgn_seed_surfels(sgn_plan* plan);

/* Sec. 2.4: `iters` damped Gauss-Newton iterations on every surfel, continuing from the
 * current state, then one evaluation at the returned parameters giving the cost (the
 * surfel's "last residual", Sec. 2.1) and the valid-sample count; also renders the
 * per-pixel inverse depth map (Eq. 3).  iters >= 0.  Enqueued on the stream. */
sgn_status sgn_run(sgn_plan* plan, int iters);

/* The whole path in one launch: seeding (from the initial surfels), `iters` iterations,
 * final cost and the depth map.  Equivalent to sgn_seed_surfels + sgn_run. */
sgn_status sgn_solve(sgn_plan* plan, int iters);

/* Enqueue copies of the current surfels: inverse depth (S), normal (3 S), cost (S), valid
 * samples (S), status (S).  Any pointer may be NULL.  Valid after sgn_sync. */
sgn_status sgn_read_surfels(sgn_plan* plan, float* inv_depth, float* normal, float* cost, int32_t* nres,
                            uint8_t* status, sgn_mem mem);

/* Enqueue copies of the per-pixel inverse depth (W x H floats, 0 where no surfel) and the
 * generating surfel index (W x H int32, -1 where none), tightly packed rows (Sec. 2.2). */
sgn_status sgn_read_depth_map(sgn_plan* plan, float* inv_depth, int32_t* surfel_index, sgn_mem mem);

/* sgn_read_surfels and sgn_read_depth_map in one call: the surfels (Sec. 2.1: inverse depth,
 * normal, last cost, valid samples, status) and the per-pixel inverse depth and surfel index
 * (Sec. 2.2), layouts as there.  Any pointer may be NULL.  With SGN_DEVICE memory every transfer
 * of the call is one copy kernel; with SGN_HOST one cudaMemcpyAsync per array.  Valid after
 * sgn_sync. */
sgn_status sgn_read_results(sgn_plan* plan, float* inv_depth, float* normal, float* cost, int32_t* nres,
                            uint8_t* status, float* depth_map, int32_t* surfel_index, sgn_mem mem);

/* Wait for the plan's stream; timeout_ns = 0 waits forever.  SGN_ERR_TIMEOUT if the
 * deadline passes (the work keeps running), SGN_ERR_CUDA on an asynchronous error. */
sgn_status sgn_sync(sgn_plan* plan, uint64_t timeout_ns);

/* Surfel state snapshot (checkpoint/resume): bytes needed, then copy to/from host memory.
 * Export is synchronous (the stream is synchronised).  Importing the exported bytes and
 * running k more iterations equals running them without the snapshot, bit for bit. */
sgn_status sgn_state_bytes(const sgn_plan* plan, size_t* bytes);
sgn_status sgn_export_state(sgn_plan* plan, void* host, size_t bytes);
sgn_status sgn_import_state(sgn_plan* plan, const void* host, size_t bytes);

/* ---- one solve that allocates nothing --------------------------------------------------- */

/* The paper has no counterpart to this call; it serves callers that must not allocate device
 * memory where they solve: real-time loops that may not take the allocator's locks or fail with
 * out-of-memory mid-run, and host frameworks or plugins that hand out only the buffers they own
 * (and forbid their components any allocation of their own).
 *
 * sgn_solve_static runs the same work as sgn_set_frames + sgn_init_surfels + sgn_solve + the reads,
 * enqueued on cuda_stream, without a plan or workspace: every input and output is a caller-owned
 * DEVICE pointer (all required; keyframe W x H floats with keyframe_pitch_bytes rows; frames[] is a
 * host array of num_frames device pointers with frame_pitch_bytes rows; surfel arrays as in
 * sgn_init_surfels / sgn_read_surfels; depth_map and surfel_index W x H, tightly packed) except
 * desc, intrinsics (fx, fy, cx, cy) and poses (12 doubles per frame), which are host memory read
 * during the call.  The packed frame texels go to a fixed device array of SGN_STATIC_SCRATCH_BYTES
 * that the library owns: num_frames * height * round_up(width, 32) * (16 for FP32, 8 for FP16/BF16
 * texels) must fit, else SGN_ERR_WORKSPACE_TOO_SMALL.  Every GPU that loads the library holds that
 * array until the process exits.  All calls share it and it keeps the last call's contents; calls in
 * sequence are independent (each rewrites what it reads), but calls whose work overlaps on the GPU
 * race on it.  The first call on a device looks the array's address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  No cudaMalloc, cudaFree or
 * other allocating routine is called. */
#define SGN_STATIC_SCRATCH_BYTES (32u << 20)
sgn_status sgn_solve_static(const sgn_plan_desc* desc, const double intrinsics[4], const float* keyframe,
                            size_t keyframe_pitch_bytes, int num_frames, const float* const* frames,
                            size_t frame_pitch_bytes, const double* poses, const float* inv_depth0,
                            const float* normal0, const uint8_t* state0, int iters, float* inv_depth, float* normal,
                            float* cost, int32_t* nres, uint8_t* status, float* depth_map, int32_t* surfel_index,
                            void* cuda_stream);

/* ---- batches: many keyframe plans in one persistent launch --------------------------- */

/* A batch groups up to max_plans bound plans (any sizes, patches, frame counts, dtypes, options).
 * sgn_batch_run runs, for every plan, the same work as sgn_solve, in one persistent kernel per
 * solver kind present (square surfels with fixed damping; the Marquardt schedule; circular
 * surfels, whose depth maps are then rendered per plan) over a device work list of (plan, surfel
 * range) items, on `cuda_stream`.  The batch needs a small device workspace of its own
 * (sgn_batch_workspace_bytes, after adding the plans). */
sgn_status sgn_batch_create(int max_plans, sgn_batch** out);
sgn_status sgn_batch_add(sgn_batch* batch, sgn_plan* plan);
sgn_status sgn_batch_clear(sgn_batch* batch);
sgn_status sgn_batch_workspace_bytes(const sgn_batch* batch, size_t* bytes);
sgn_status sgn_batch_bind(sgn_batch* batch, void* d_workspace, size_t bytes, void* cuda_stream);
/* Schedule of the persistent launches: variant 0 maps P=4/8/16 surfels to 8/16/32 lanes and
 * variant 1 to 16/32/32 lanes, each warp taking work items of `chunk` surfels (1..65536) in tile
 * order; variant 2 maps as variant 0 but each block takes a square of neighbouring tiles of one
 * plan at a time (the block of a plain launch; `chunk` then applies to the other kinds only).  The
 * schedule applies to fixed-damping plans; the other kinds keep their own mapping with chunk-sized
 * items.  Defaults 0 and 64. */
sgn_status sgn_batch_set_schedule(sgn_batch* batch, int variant, int chunk);
sgn_status sgn_batch_run(sgn_batch* batch, int iters);
sgn_status sgn_batch_sync(sgn_batch* batch, uint64_t timeout_ns);
sgn_status sgn_batch_destroy(sgn_batch* batch);

/* ---- serving: continuous batching of keyframe solves from many camera streams ------------ */

typedef struct sgn_server sgn_server;   /* opaque, host side */

/* One keyframe solve request.  All pointers are host memory (page-locked memory makes the copies
 * asynchronous) and must stay valid until the request's completion is returned by sgn_server_poll;
 * desc/intrinsics/poses/frames[] (the pointer array) are copied at submission. */
typedef struct {
    sgn_plan_desc desc;          /* size, patch, frame slots, texel type, options */
    double intrinsics[4];        /* fx, fy, cx, cy */
    const float* keyframe;       /* W x H, tightly packed */
    int num_frames;              /* 1..desc.max_frames */
    const float* const* frames;  /* num_frames pointers to W x H images */
    const double* poses;         /* 12 per frame, keyframe -> frame */
    const float* inv_depth0;     /* initial surfels as in sgn_init_surfels */
    const float* normal0;
    const uint8_t* state0;
    int iters;                   /* Gauss-Newton iterations (sgn_solve) */
    float* inv_depth;            /* results as in sgn_read_surfels (S, 3 S, S, S, S) */
    float* normal;
    float* cost;
    int32_t* nres;
    uint8_t* status;
    uint64_t tag;                /* caller's identifier, returned in the completion */
} sgn_request;

typedef struct {
    uint64_t tag;
    sgn_status status;   /* SGN_OK, SGN_ERR_CUDA, SGN_ERR_STATE (cancelled) ... */
    int cancelled;
    double latency_ms;   /* submission -> results in host memory */
    double queue_ms;     /* submission -> admission */
    uint64_t admit_seq;  /* admission order (1, 2, ...); 0 if never admitted */
} sgn_completion;

typedef struct {
    uint64_t completed, epochs, rejected, admission_waits, residuals;
    size_t peak_arena_bytes;
    double latency_p50_ms, latency_p99_ms, latency_max_ms, latency_mean_ms;
    double busy_seconds; /* first submission -> last completion */
} sgn_serving_stats;

/* Start a server over a caller-owned device arena (256-byte aligned) that bounds the device memory
 * of the requests in flight (admission by free memory): each admitted request takes its plan
 * workspace (sgn_plan_workspace_bytes) from the arena until it completes; a request larger than the
 * arena is refused at submission with SGN_ERR_ADMISSION, one that does not fit yet waits.
 * Admission is first come, first served, except that later requests may pass one that does not
 * fit yet; each waiting request is passed at most 8 times, after which nothing behind it is
 * admitted until it fits (so no request waits indefinitely behind a stream of smaller ones).
 * compute_stream runs the batched solves, copy_stream the uploads, frame preparation and result
 * copies (two distinct non-default streams of the current device).  An epoch = one persistent batch
 * launch over every request uploaded since the previous launch, at most max_slots requests and
 * max_surfels_per_epoch surfels (plus one work item per request); up to two epochs are in flight.
 * A server thread makes all CUDA calls. */
sgn_status sgn_server_create(void* d_arena, size_t arena_bytes, int max_slots, int max_surfels_per_epoch,
                             void* compute_stream, void* copy_stream, sgn_server** out);
/* Queue a request (thread-safe; no CUDA call in the caller's thread). */
sgn_status sgn_server_submit(sgn_server* server, const sgn_request* request);
/* Cancel by tag: a request not yet finished completes with cancelled = 1 (its results are not
 * written if it had not run yet; if it already ran, they may be). */
sgn_status sgn_server_cancel(sgn_server* server, uint64_t tag);
/* Take up to max completions (in completion order). */
sgn_status sgn_server_poll(sgn_server* server, sgn_completion* out, int max, int* n);
/* Wait until every submitted request has completed; timeout_ns = 0 waits forever. */
sgn_status sgn_server_drain(sgn_server* server, uint64_t timeout_ns);
sgn_status sgn_server_stats(sgn_server* server, sgn_serving_stats* out);
/* Finish the requests in flight, then stop the server thread. */
sgn_status sgn_server_destroy(sgn_server* server);

/* ---- reference-frame change and surfel render (Sec. 2.5, Sec. 2.2) ------------------------ */

/* A free surfel is the pixel u_s = (x, y) where its point projects in its reference frame, its
 * inverse depth id_s along the ray r_s = K^-1 (u_s, 1) (z = 1), and its unit normal n = (x, y, z).
 * A plan's surfel s is the free surfel at its tile centre (tx P + (P-1)/2, ty P + (P-1)/2). */

/* Sec. 2.5, Eq. 10: express n free surfels of reference frame kf0 in reference frame kf1.
 * T_kf1_kf0: host array of 12 doubles, row-major [R | t] mapping kf0 coordinates to kf1
 * coordinates (a finite rigid motion, else SGN_ERR_INVALID_ARGUMENT).  For each surfel
 * p1 = R r_s / id_s + t, n1 = R n, u1 = pi(K p1) and id1 = 1 / p1_z; valid[i] = 1, or 0 (all
 * outputs 0) when id_s <= 0 or p1 lies behind the new camera.  Device arrays: u, u_out 2n floats
 * (8-byte aligned), inv_depth, inv_depth_out n floats, normal, normal_out 3n floats, valid n
 * bytes; inputs and outputs must not overlap.  FP32 arithmetic.  Asynchronous on `stream`
 * (cudaStream_t, may be NULL); n = 0 is a no-op. */
sgn_status sgn_transfer_surfels(const double intrinsics[4], const double T_kf1_kf0[12], int n, const float* u,
                                const float* inv_depth, const float* normal, float* u_out, float* inv_depth_out,
                                float* normal_out, uint8_t* valid, void* stream);

/* Sec. 2.2: depth-buffered render of n free surfels of radius `radius` pixels (0 < radius <= 1024)
 * into a width x height map.  A surfel covers the pixels whose centre lies strictly within the
 * radius of u_s (Eq. 4); at a covered pixel its inverse depth is Eq. 3 along its own ray, drawn
 * when positive.  The nearest surfel (largest inverse depth) is kept; equal inverse depths go to
 * the lower index.  inv_depth_map (floats) and surfel_index (int32) get 0 and -1 where no surfel
 * is drawn.  zbuffer: caller scratch of width * height uint64 (device).  Surfels with
 * valid[i] == 0 are skipped.  Surfel arrays as for sgn_transfer_surfels (device; may be NULL
 * when n = 0).  FP32 arithmetic; asynchronous on `stream`. */
sgn_status sgn_render_surfels(const double intrinsics[4], int width, int height, int n, const float* u,
                              const float* inv_depth, const float* normal, const uint8_t* valid, float radius,
                              uint64_t* zbuffer, float* inv_depth_map, int32_t* surfel_index, void* stream);

/* ---- autotuning -------------------------------------------------------------------------- */

/* Choose the plan's kernel mapping (lanes per surfel x threads per block, as in
 * sgn_plan_set_mapping) by timing sgn_solve(plan, iters) for every supported mapping on the bound
 * stream (one warm-up and three timed runs each; the plan is left with the working state of a
 * solve).  cache_path (may be NULL) names a text file of earlier results keyed by GPU name and
 * problem shape; a hit skips the timing, a miss appends a line.  Synchronises the stream. */
sgn_status sgn_plan_autotune(sgn_plan* plan, int iters, const char* cache_path, int* lanes_per_surfel,
                             int* block_threads);

/* Choose the batch schedule (variant x surfels per work item, as in sgn_batch_set_schedule) by
 * timing sgn_batch_run(batch, iters) for variants {0, 1} x chunks {8, 16, 32, 64, 128, 256}.
 * Schedules whose work list does not fit the bound workspace are skipped: bind a workspace sized
 * at chunk 8 to try them all.  Cache as for sgn_plan_autotune. */
sgn_status sgn_batch_autotune(sgn_batch* batch, int iters, const char* cache_path, int* variant, int* chunk);

/* Shared-memory staging of frame texels (default off).  With staging, each surfel's Gauss-Newton
 * evaluation reads the bilinear taps from boxes of texels around the projection of its tile centre,
 * copied into shared memory by the tensor memory accelerator two boxes ahead of use; taps outside a
 * box read global memory.  Results are identical with and without staging (same texels, same
 * arithmetic); it changes only where the taps come from.  Without staging the taps are read through
 * the L1 cache, which keeps a surfel's footprint across iterations, whereas the boxes are fetched
 * again on every pass; on one GB300 at 640x480 staging is the slower of the two.  enabled: 1 or 0. */
sgn_status sgn_plan_set_staging(sgn_plan* plan, int enabled);

/* Number of staging waits on the current device that ran out of time (about one second each) since
 * the library was loaded.  A surfel whose wait runs out reads its texels from global memory for
 * the rest of the launch, so results stay correct; a non-zero count means the GPU stalled.
 * Synchronous (a 4-byte device-to-host copy). */
sgn_status sgn_staging_timeouts(uint32_t* count);

/* ---- introspection --------------------------------------------------------------------- */

/* Diagnostic: the FP64 route of the damped normal-equation solve of Sec. 2.4 (the step of Eq. 7
 * with Levenberg-Marquardt damping), run on n given systems exactly as the Gauss-Newton kernels run
 * it (Cramer's rule, one component per lane of a 16-lane group): (H + lambda diag(m, m, H33)) delta
 * = -g, m = (H11 + H22) / 2.  H6: n x 6 floats, the upper triangle (H11, H12, H13, H22, H23, H33)
 * row by row; g3: n x 3 floats; delta: n x 3 floats out; pd: n int32 out, 1 when the damped matrix
 * is positive definite (its leading principal minors are positive in FP64), else 0 (delta is then
 * meaningless).  All arrays are device pointers; enqueued on `stream` (cudaStream_t, may be NULL);
 * n = 0 is a no-op; NULL arrays with n > 0, n < 0 or lambda not >= 0 give
 * SGN_ERR_INVALID_ARGUMENT. */
sgn_status sgn_check_fp64_solve(const float* H6, const float* g3, double lambda, int n, float* delta, int32_t* pd,
                                void* stream);

/* Message for the calling thread's last failed call ("" if none). */
const char* sgn_last_error(void);

/* Number of kernels libsgn has launched in this process (all plans and batches). */
uint64_t sgn_launch_count(void);

/* ABI version (SGN_ABI_VERSION). */
int sgn_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SGN_H */
