"""Python binding of libsgn: per-surfel Gauss-Newton photometric optimisation on the GPU.

The binding only marshals arguments: every step of the computation runs in the CUDA kernels of
``libsgn.so`` (built in-tree for sm_103a by ``paper_1910_01997_gb300/build.py``).  PyTorch supplies
device memory and CUDA streams.  If the library is missing, importing this package fails.

Functions carry the names of the C ABI in ``include/sgn.h``; a non-OK status raises ``SgnError``.
``Plan`` and ``Batch`` wrap a plan/batch together with its torch-allocated workspace.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1910_01997_gb300/build.py` "
                      "(nvcc, sm_103a); there is no fallback implementation")
_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------------------------------- constants
SGN_OK, SGN_ERR_INVALID_ARGUMENT, SGN_ERR_NOT_BOUND, SGN_ERR_WORKSPACE_TOO_SMALL = 0, -1, -2, -3
SGN_ERR_CUDA, SGN_ERR_TIMEOUT, SGN_ERR_ADMISSION, SGN_ERR_STATE = -4, -5, -6, -7
SGN_F32, SGN_F16, SGN_BF16, SGN_F16G, SGN_BF16G = 0, 1, 2, 3, 4
SGN_HOST, SGN_DEVICE = 0, 1
SGN_STATE_EMPTY, SGN_STATE_VALID, SGN_STATE_TO_SEED = 0, 1, 2
SGN_SURFEL_OK, SGN_SURFEL_EMPTY, SGN_SURFEL_UNSEEDED = 0, 1, 2
SGN_SURFEL_UNDERDETERMINED, SGN_SURFEL_SINGULAR, SGN_SURFEL_STEP_REJECTED = 3, 4, 5
SGN_SURFEL_SEEDED, SGN_SURFEL_FP64 = 0x40, 0x80
SGN_MAX_FRAMES = 16
DTYPES = {"f32": SGN_F32, "f16": SGN_F16, "bf16": SGN_BF16, "f16g": SGN_F16G, "bf16g": SGN_BF16G}


class sgn_plan_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("patch", ctypes.c_int),
                ("max_frames", ctypes.c_int), ("image_dtype", ctypes.c_int), ("huber_k", ctypes.c_float),
                ("lm_lambda", ctypes.c_float), ("fp64_cond", ctypes.c_double), ("optimize_normal", ctypes.c_int),
                ("min_residuals", ctypes.c_int), ("lm_adaptive", ctypes.c_int), ("surfel_radius", ctypes.c_float)]


class sgn_request(ctypes.Structure):
    _fields_ = [("desc", sgn_plan_desc), ("intrinsics", ctypes.c_double * 4), ("keyframe", ctypes.c_void_p),
                ("num_frames", ctypes.c_int), ("frames", ctypes.c_void_p), ("poses", ctypes.c_void_p),
                ("inv_depth0", ctypes.c_void_p), ("normal0", ctypes.c_void_p), ("state0", ctypes.c_void_p),
                ("iters", ctypes.c_int), ("inv_depth", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("cost", ctypes.c_void_p), ("nres", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("tag", ctypes.c_uint64)]


class sgn_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("cancelled", ctypes.c_int),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("admit_seq", ctypes.c_uint64)]


class sgn_serving_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("epochs", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("admission_waits", ctypes.c_uint64), ("residuals", ctypes.c_uint64),
                ("peak_arena_bytes", ctypes.c_size_t), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double),
                ("latency_mean_ms", ctypes.c_double), ("busy_seconds", ctypes.c_double)]


class SgnError(RuntimeError):
    def __init__(self, status: int, func: str):
        self.status = status
        msg = _lib.sgn_last_error().decode(errors="replace")
        super().__init__(f"{func} failed with status {status}: {msg}")


_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_SIGS = {
    "sgn_plan_desc_default": [ctypes.POINTER(sgn_plan_desc), _I, _I, _I, _I],
    "sgn_plan_create": [ctypes.POINTER(sgn_plan_desc), ctypes.POINTER(_P)],
    "sgn_plan_destroy": [_P],
    "sgn_plan_num_surfels": [_P, ctypes.POINTER(_I)],
    "sgn_plan_workspace_bytes": [_P, ctypes.POINTER(_SZ)],
    "sgn_plan_set_mapping": [_P, _I, _I],
    "sgn_plan_bind": [_P, _P, _SZ, _P],
    "sgn_set_intrinsics": [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double],
    "sgn_set_keyframe": [_P, _P, _SZ, _I],
    "sgn_set_frame": [_P, _I, _P, _SZ, _I, _P],
    "sgn_set_frames": [_P, _I, _P, _SZ, _I, _P],
    "sgn_set_num_frames": [_P, _I],
    "sgn_init_surfels": [_P, _P, _P, _P, _I],
    "sgn_seed_surfels": [_P],
    "sgn_run": [_P, _I],
    "sgn_solve": [_P, _I],
    "sgn_read_surfels": [_P, _P, _P, _P, _P, _P, _I],
    "sgn_read_depth_map": [_P, _P, _P, _I],
    "sgn_read_results": [_P, _P, _P, _P, _P, _P, _P, _P, _I],
    "sgn_sync": [_P, ctypes.c_uint64],
    "sgn_state_bytes": [_P, ctypes.POINTER(_SZ)],
    "sgn_export_state": [_P, _P, _SZ],
    "sgn_import_state": [_P, _P, _SZ],
    "sgn_solve_static": [ctypes.POINTER(sgn_plan_desc), _P, _P, _SZ, _I, _P, _SZ, _P, _P, _P, _P, _I,
                         _P, _P, _P, _P, _P, _P, _P, _P],
    "sgn_plan_autotune": [_P, _I, ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "sgn_server_create": [_P, _SZ, _I, _I, _P, _P, ctypes.POINTER(_P)],
    "sgn_server_submit": [_P, ctypes.POINTER(sgn_request)],
    "sgn_server_cancel": [_P, ctypes.c_uint64],
    "sgn_server_poll": [_P, ctypes.POINTER(sgn_completion), _I, ctypes.POINTER(_I)],
    "sgn_server_drain": [_P, ctypes.c_uint64],
    "sgn_server_stats": [_P, ctypes.POINTER(sgn_serving_stats)],
    "sgn_server_destroy": [_P],
    "sgn_batch_autotune": [_P, _I, ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "sgn_batch_create": [_I, ctypes.POINTER(_P)],
    "sgn_batch_add": [_P, _P],
    "sgn_batch_clear": [_P],
    "sgn_batch_workspace_bytes": [_P, ctypes.POINTER(_SZ)],
    "sgn_batch_bind": [_P, _P, _SZ, _P],
    "sgn_batch_set_schedule": [_P, _I, _I],
    "sgn_batch_run": [_P, _I],
    "sgn_batch_sync": [_P, ctypes.c_uint64],
    "sgn_batch_destroy": [_P],
    "sgn_check_fp64_solve": [_P, _P, ctypes.c_double, _I, _P, _P, _P],
    "sgn_plan_set_staging": [_P, _I],
    "sgn_transfer_surfels": [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _I, _P, _P, _P, _P, _P,
                             _P, _P, _P],
    "sgn_render_surfels": [ctypes.POINTER(ctypes.c_double), _I, _I, _I, _P, _P, _P, _P, ctypes.c_float, _P, _P, _P, _P],
    "sgn_staging_timeouts": [ctypes.POINTER(ctypes.c_uint32)],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int
_lib.sgn_last_error.restype = ctypes.c_char_p
_lib.sgn_last_error.argtypes = []
_lib.sgn_launch_count.restype = ctypes.c_uint64
_lib.sgn_launch_count.argtypes = []
_lib.sgn_abi_version.restype = ctypes.c_int
_lib.sgn_abi_version.argtypes = []


def _call(name, *args):
    st = getattr(_lib, name)(*args)
    if st != SGN_OK:
        raise SgnError(st, name)
    return st


def _status(name, *args) -> int:
    """Call without raising; returns the sgn_status."""
    return getattr(_lib, name)(*args)


# ------------------------------------------------------------------------------- C-ABI functions

def sgn_plan_desc_default(width, height, patch, max_frames) -> sgn_plan_desc:
    d = sgn_plan_desc()
    _call("sgn_plan_desc_default", ctypes.byref(d), width, height, patch, max_frames)
    return d


def sgn_plan_create(desc: sgn_plan_desc) -> int:
    h = _P()
    _call("sgn_plan_create", ctypes.byref(desc), ctypes.byref(h))
    return h.value


def sgn_plan_destroy(plan):
    _call("sgn_plan_destroy", plan)


def sgn_plan_num_surfels(plan) -> int:
    n = _I()
    _call("sgn_plan_num_surfels", plan, ctypes.byref(n))
    return n.value


def sgn_plan_workspace_bytes(plan) -> int:
    n = _SZ()
    _call("sgn_plan_workspace_bytes", plan, ctypes.byref(n))
    return n.value


def sgn_plan_set_mapping(plan, lanes_per_surfel, block_threads):
    _call("sgn_plan_set_mapping", plan, lanes_per_surfel, block_threads)


def sgn_plan_set_staging(plan, enabled):
    _call("sgn_plan_set_staging", plan, int(enabled))


def sgn_plan_bind(plan, d_workspace, nbytes, cuda_stream):
    _call("sgn_plan_bind", plan, d_workspace, nbytes, cuda_stream)


def sgn_set_intrinsics(plan, fx, fy, cx, cy):
    _call("sgn_set_intrinsics", plan, fx, fy, cx, cy)


def sgn_set_keyframe(plan, ptr, pitch_bytes, mem):
    _call("sgn_set_keyframe", plan, ptr, pitch_bytes, mem)


def sgn_set_frame(plan, slot, ptr, pitch_bytes, mem, pose_ptr):
    _call("sgn_set_frame", plan, slot, ptr, pitch_bytes, mem, pose_ptr)


def sgn_set_frames(plan, n, ptrs_ptr, pitch_bytes, mem, poses_ptr):
    _call("sgn_set_frames", plan, n, ptrs_ptr, pitch_bytes, mem, poses_ptr)


def sgn_set_num_frames(plan, n):
    _call("sgn_set_num_frames", plan, n)


def sgn_init_surfels(plan, id_ptr, n_ptr, state_ptr, mem):
    _call("sgn_init_surfels", plan, id_ptr, n_ptr, state_ptr, mem)


def sgn_seed_surfels(plan):
    _call("sgn_seed_surfels", plan)


def sgn_run(plan, iters):
    _call("sgn_run", plan, iters)


def sgn_solve(plan, iters):
    _call("sgn_solve", plan, iters)


def sgn_read_surfels(plan, id_ptr, n_ptr, cost_ptr, nres_ptr, status_ptr, mem):
    _call("sgn_read_surfels", plan, id_ptr, n_ptr, cost_ptr, nres_ptr, status_ptr, mem)


def sgn_read_depth_map(plan, depth_ptr, sidx_ptr, mem):
    _call("sgn_read_depth_map", plan, depth_ptr, sidx_ptr, mem)


def sgn_read_results(plan, id_ptr, n_ptr, cost_ptr, nres_ptr, status_ptr, depth_ptr, sidx_ptr, mem):
    _call("sgn_read_results", plan, id_ptr, n_ptr, cost_ptr, nres_ptr, status_ptr, depth_ptr, sidx_ptr, mem)


def sgn_sync(plan, timeout_ns=0):
    _call("sgn_sync", plan, timeout_ns)


def sgn_state_bytes(plan) -> int:
    n = _SZ()
    _call("sgn_state_bytes", plan, ctypes.byref(n))
    return n.value


def sgn_export_state(plan, host_ptr, nbytes):
    _call("sgn_export_state", plan, host_ptr, nbytes)


def sgn_import_state(plan, host_ptr, nbytes):
    _call("sgn_import_state", plan, host_ptr, nbytes)


SGN_STATIC_SCRATCH_BYTES = 32 << 20


def sgn_solve_static(desc, intrinsics_ptr, keyframe_ptr, keyframe_pitch_bytes, num_frames, frame_ptrs_ptr,
                     frame_pitch_bytes, poses_ptr, inv_depth0_ptr, normal0_ptr, state0_ptr, iters, inv_depth_ptr,
                     normal_ptr, cost_ptr, nres_ptr, status_ptr, depth_map_ptr, surfel_index_ptr, cuda_stream):
    """Whole-path solve that allocates nothing (see include/sgn.h): device pointers in and out, frame
    texels in the library's fixed device scratch.  For callers that must not allocate device memory."""
    _call("sgn_solve_static", ctypes.byref(desc), intrinsics_ptr, keyframe_ptr, keyframe_pitch_bytes, num_frames,
          frame_ptrs_ptr, frame_pitch_bytes, poses_ptr, inv_depth0_ptr, normal0_ptr, state0_ptr, iters, inv_depth_ptr,
          normal_ptr, cost_ptr, nres_ptr, status_ptr, depth_map_ptr, surfel_index_ptr, cuda_stream)


def sgn_plan_autotune(plan, iters, cache_path=None):
    a, b = _I(), _I()
    _call("sgn_plan_autotune", plan, int(iters), None if cache_path is None else str(cache_path).encode(),
          ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def sgn_batch_autotune(batch, iters, cache_path=None):
    a, b = _I(), _I()
    _call("sgn_batch_autotune", batch, int(iters), None if cache_path is None else str(cache_path).encode(),
          ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def sgn_batch_create(max_plans) -> int:
    h = _P()
    _call("sgn_batch_create", max_plans, ctypes.byref(h))
    return h.value


def sgn_batch_add(batch, plan):
    _call("sgn_batch_add", batch, plan)


def sgn_batch_clear(batch):
    _call("sgn_batch_clear", batch)


def sgn_batch_workspace_bytes(batch) -> int:
    n = _SZ()
    _call("sgn_batch_workspace_bytes", batch, ctypes.byref(n))
    return n.value


def sgn_batch_bind(batch, d_workspace, nbytes, cuda_stream):
    _call("sgn_batch_bind", batch, d_workspace, nbytes, cuda_stream)


def sgn_batch_set_schedule(batch, variant, chunk):
    _call("sgn_batch_set_schedule", batch, variant, chunk)


def sgn_batch_run(batch, iters):
    _call("sgn_batch_run", batch, iters)


def sgn_batch_sync(batch, timeout_ns=0):
    _call("sgn_batch_sync", batch, timeout_ns)


def sgn_batch_destroy(batch):
    _call("sgn_batch_destroy", batch)


def sgn_server_create(d_arena, arena_bytes, max_slots, max_surfels_per_epoch, compute_stream, copy_stream) -> int:
    h = _P()
    _call("sgn_server_create", d_arena, arena_bytes, max_slots, max_surfels_per_epoch, compute_stream, copy_stream,
          ctypes.byref(h))
    return h.value


def sgn_server_submit(server, request: sgn_request):
    _call("sgn_server_submit", server, ctypes.byref(request))


def sgn_server_cancel(server, tag):
    _call("sgn_server_cancel", server, tag)


def sgn_server_poll(server, max_n=1024):
    buf = (sgn_completion * max_n)()
    n = _I()
    _call("sgn_server_poll", server, buf, max_n, ctypes.byref(n))
    return [buf[i] for i in range(n.value)]


def sgn_server_drain(server, timeout_ns=0):
    _call("sgn_server_drain", server, timeout_ns)


def sgn_server_stats(server) -> sgn_serving_stats:
    st = sgn_serving_stats()
    _call("sgn_server_stats", server, ctypes.byref(st))
    return st


def sgn_server_destroy(server):
    _call("sgn_server_destroy", server)


def sgn_last_error() -> str:
    return _lib.sgn_last_error().decode(errors="replace")


def sgn_launch_count() -> int:
    return int(_lib.sgn_launch_count())


def sgn_abi_version() -> int:
    return int(_lib.sgn_abi_version())


def _doubles(values, n):
    a = (ctypes.c_double * n)(*[float(v) for v in np.asarray(values, dtype=np.float64).reshape(-1)])
    if len(np.asarray(values).reshape(-1)) != n:
        raise ValueError(f"expected {n} values")
    return a


def _dev(t, dtype, shape):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype} and shape {tuple(shape)}")
    return t.data_ptr()


def sgn_transfer_surfels(intrinsics, T_kf1_kf0, u, inv_depth, normal, stream=None):
    """Sec. 2.5, Eq. 10 on CUDA tensors u (n, 2), inv_depth (n,), normal (n, 3) (float32).
    Returns dict(u, inv_depth, normal, valid) of new CUDA tensors (enqueued on the stream)."""
    import torch

    n = int(inv_depth.shape[0])
    out = dict(u=torch.empty(n, 2, device=u.device), inv_depth=torch.empty(n, device=u.device),
               normal=torch.empty(n, 3, device=u.device), valid=torch.empty(n, dtype=torch.uint8, device=u.device))
    s = torch.cuda.current_stream() if stream is None else stream
    _call("sgn_transfer_surfels", _doubles(intrinsics, 4), _doubles(T_kf1_kf0, 12), n,
          _dev(u, torch.float32, (n, 2)), _dev(inv_depth, torch.float32, (n,)), _dev(normal, torch.float32, (n, 3)),
          out["u"].data_ptr(), out["inv_depth"].data_ptr(), out["normal"].data_ptr(), out["valid"].data_ptr(), s.cuda_stream)
    return out


def sgn_render_surfels(intrinsics, width, height, u, inv_depth, normal, valid, radius, zbuffer=None, stream=None):
    """Sec. 2.2 depth-buffered render of free surfels (CUDA tensors as for sgn_transfer_surfels) of
    the given radius.  Returns (inverse-depth map (H, W) float32, surfel index (H, W) int32)."""
    import torch

    n = int(inv_depth.shape[0])
    dev = u.device
    if zbuffer is None:
        zbuffer = torch.empty(height * width, dtype=torch.int64, device=dev)
    inv = torch.empty(height, width, device=dev)
    sidx = torch.empty(height, width, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream() if stream is None else stream
    _call("sgn_render_surfels", _doubles(intrinsics, 4), int(width), int(height), n, _dev(u, torch.float32, (n, 2)),
          _dev(inv_depth, torch.float32, (n,)), _dev(normal, torch.float32, (n, 3)), _dev(valid, torch.uint8, (n,)),
          float(radius), _dev(zbuffer, torch.int64, (height * width,)), inv.data_ptr(), sidx.data_ptr(), s.cuda_stream)
    return inv, sidx


def sgn_staging_timeouts() -> int:
    n = ctypes.c_uint32()
    _call("sgn_staging_timeouts", ctypes.byref(n))
    return int(n.value)


def sgn_check_fp64_solve(H6, g3, lam, stream=None):
    """The FP64 route of the damped solve on the systems of the float32 CUDA tensors H6 (n, 6) and
    g3 (n, 3) (diagnostic).  Returns (delta (n, 3) float32, positive definite (n,) bool) on the GPU."""
    import torch

    n = int(H6.shape[0]) if isinstance(H6, torch.Tensor) and H6.dim() == 2 else -1
    delta = torch.empty(max(n, 0), 3, device=H6.device)
    pd = torch.empty(max(n, 0), dtype=torch.int32, device=H6.device)
    s = torch.cuda.current_stream() if stream is None else stream
    _call("sgn_check_fp64_solve", _dev(H6, torch.float32, (n, 6)), _dev(g3, torch.float32, (n, 3)), float(lam), n,
          delta.data_ptr(), pd.data_ptr(), s.cuda_stream)
    s.synchronize()
    return delta, pd != 0


# ------------------------------------------------------------------------------- helpers


def _torch():
    import torch

    return torch


def _ptr_and_mem(a):
    """(pointer, sgn_mem, keepalive) for a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            a = np.ascontiguousarray(a)
        return a.ctypes.data, SGN_HOST, a
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), (SGN_DEVICE if a.is_cuda else SGN_HOST), a
    raise TypeError(f"expected a numpy array or torch tensor, got {type(a)}")


def _as(a, np_dtype, torch_dtype):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np_dtype)
    return a.to(torch_dtype).contiguous()


class Plan:
    """A plan plus its device workspace (a torch uint8 tensor) on the current CUDA device/stream."""

    def __init__(self, width, height, patch, max_frames, image_dtype="f32", *, huber_k=9.0 / 255.0,
                 lm_lambda=1e-3, fp64_cond=1e6, optimize_normal=True, min_residuals=8, lm_adaptive=False,
                 surfel_radius=0.0, stream=None,
                 lanes_per_surfel=0, block_threads=0, staging=False):
        torch = _torch()
        d = sgn_plan_desc_default(width, height, patch, max_frames)
        d.image_dtype = DTYPES[image_dtype] if isinstance(image_dtype, str) else int(image_dtype)
        d.huber_k, d.lm_lambda, d.fp64_cond = huber_k, lm_lambda, fp64_cond
        d.optimize_normal, d.min_residuals = int(bool(optimize_normal)), min_residuals
        d.lm_adaptive = int(bool(lm_adaptive))
        d.surfel_radius = float(surfel_radius)
        self.desc = d
        self.handle = sgn_plan_create(d)
        self.W, self.H, self.P = width, height, patch
        self.S = sgn_plan_num_surfels(self.handle)
        if lanes_per_surfel or block_threads:
            sgn_plan_set_mapping(self.handle, lanes_per_surfel, block_threads)
        if staging:
            sgn_plan_set_staging(self.handle, 1)
        nbytes = sgn_plan_workspace_bytes(self.handle)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        sgn_plan_bind(self.handle, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        self._keep = []

    def close(self):
        if getattr(self, "handle", None):
            sgn_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # inputs
    def set_intrinsics(self, fx, fy, cx, cy):
        sgn_set_intrinsics(self.handle, float(fx), float(fy), float(cx), float(cy))

    def set_keyframe(self, img):
        img = _as(img, np.float32, _torch().float32)
        ptr, mem, keep = _ptr_and_mem(img)
        self._keep.append(keep)
        sgn_set_keyframe(self.handle, ptr, self.W * 4, mem)

    def set_frames(self, frames, poses):
        """frames: (F, H, W) float32 array/tensor or a list of (H, W); poses: (F, 3, 4) keyframe->frame."""
        torch = _torch()
        if isinstance(frames, (list, tuple)):
            frames = [_as(f, np.float32, torch.float32) for f in frames]
        else:
            frames = [_as(frames[i], np.float32, torch.float32) for i in range(len(frames))]
        info = [_ptr_and_mem(f) for f in frames]
        mems = {m for _, m, _ in info}
        if len(mems) != 1:
            raise ValueError("frames must all be host arrays or all device tensors")
        ptrs = (ctypes.c_void_p * len(info))(*[p for p, _, _ in info])
        T = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(len(info), 12))
        self._keep.extend([k for _, _, k in info] + [ptrs, T])
        sgn_set_frames(self.handle, len(info), ctypes.cast(ptrs, ctypes.c_void_p), self.W * 4, mems.pop(),
                       T.ctypes.data)

    def set_frame(self, slot, img, pose):
        img = _as(img, np.float32, _torch().float32)
        ptr, mem, keep = _ptr_and_mem(img)
        T = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
        self._keep.extend([keep, T])
        sgn_set_frame(self.handle, slot, ptr, self.W * 4, mem, T.ctypes.data)

    def set_num_frames(self, n):
        sgn_set_num_frames(self.handle, n)

    def autotune(self, iters, cache_path=None):
        """Time the supported kernel mappings of sgn_solve and keep the fastest (C++ autotuner)."""
        return sgn_plan_autotune(self.handle, iters, cache_path)

    def init_surfels(self, inv_depth, normal, state):
        torch = _torch()
        a = _as(inv_depth, np.float32, torch.float32)
        b = _as(normal, np.float32, torch.float32)
        c = _as(state, np.uint8, torch.uint8)
        (pa, ma, ka), (pb, mb, kb), (pc, mc, kc) = map(_ptr_and_mem, (a, b, c))
        if len({ma, mb, mc}) != 1:
            raise ValueError("surfel arrays must share one memory kind")
        self._keep.extend([ka, kb, kc])
        sgn_init_surfels(self.handle, pa, pb, pc, ma)

    # work
    def seed(self):
        sgn_seed_surfels(self.handle)

    def run(self, iters):
        sgn_run(self.handle, int(iters))

    def solve(self, iters):
        sgn_solve(self.handle, int(iters))

    def sync(self, timeout_ns=0):
        sgn_sync(self.handle, timeout_ns)
        self._keep.clear()

    # outputs
    def read_surfels(self, device=False):
        """Returns dict(id (S,), n (S, 3), cost (S,), nres (S,), status (S,)) as numpy (synchronises)
        or, with device=True, as CUDA tensors (enqueued, no synchronisation)."""
        torch = _torch()
        S = self.S
        if device:
            out = dict(id=torch.empty(S, device="cuda"), n=torch.empty(S, 3, device="cuda"),
                       cost=torch.empty(S, device="cuda"), nres=torch.empty(S, dtype=torch.int32, device="cuda"),
                       status=torch.empty(S, dtype=torch.uint8, device="cuda"))
            sgn_read_surfels(self.handle, *[out[k].data_ptr() for k in ("id", "n", "cost", "nres", "status")],
                             SGN_DEVICE)
            return out
        out = dict(id=np.empty(S, np.float32), n=np.empty((S, 3), np.float32), cost=np.empty(S, np.float32),
                   nres=np.empty(S, np.int32), status=np.empty(S, np.uint8))
        sgn_read_surfels(self.handle, *[out[k].ctypes.data for k in ("id", "n", "cost", "nres", "status")], SGN_HOST)
        self.sync()
        return out

    def read_depth_map(self):
        inv = np.empty((self.H, self.W), np.float32)
        sidx = np.empty((self.H, self.W), np.int32)
        sgn_read_depth_map(self.handle, inv.ctypes.data, sidx.ctypes.data, SGN_HOST)
        self.sync()
        return inv, sidx

    def export_state(self) -> bytes:
        n = sgn_state_bytes(self.handle)
        buf = ctypes.create_string_buffer(n)
        sgn_export_state(self.handle, ctypes.addressof(buf), n)
        return buf.raw

    def import_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        sgn_import_state(self.handle, ctypes.addressof(buf), len(data))


class Batch:
    """A batch of bound plans run by one persistent, graph-captured launch."""

    def __init__(self, max_plans, stream=None):
        self.handle = sgn_batch_create(max_plans)
        self.plans = []
        self.workspace = None
        self.stream = stream if stream is not None else _torch().cuda.current_stream()

    def add(self, plan: Plan):
        sgn_batch_add(self.handle, plan.handle)
        self.plans.append(plan)
        self.workspace = None

    def clear(self):
        sgn_batch_clear(self.handle)
        self.plans = []
        self.workspace = None

    def set_schedule(self, variant, chunk):
        sgn_batch_set_schedule(self.handle, variant, chunk)
        self.workspace = None

    def _bind(self):
        torch = _torch()
        n = sgn_batch_workspace_bytes(self.handle)
        self.workspace = torch.empty(n, dtype=torch.uint8, device="cuda")
        sgn_batch_bind(self.handle, self.workspace.data_ptr(), n, self.stream.cuda_stream)

    def run(self, iters):
        if self.workspace is None or self.workspace.numel() < sgn_batch_workspace_bytes(self.handle):
            self._bind()
        sgn_batch_run(self.handle, int(iters))

    def sync(self, timeout_ns=0):
        sgn_batch_sync(self.handle, timeout_ns)

    def autotune(self, iters, cache_path=None):
        """Bind a workspace large enough for every schedule, then time the schedules (C++ autotuner)."""
        torch = _torch()
        n = 0
        for v in (0, 2):  # the larger work list of the schedules tried (chunk 8)
            sgn_batch_set_schedule(self.handle, v, 8)
            n = max(n, sgn_batch_workspace_bytes(self.handle))
        self.workspace = torch.empty(n, dtype=torch.uint8, device="cuda")
        sgn_batch_bind(self.handle, self.workspace.data_ptr(), n, self.stream.cuda_stream)
        return sgn_batch_autotune(self.handle, iters, cache_path)

    def close(self):
        if getattr(self, "handle", None):
            sgn_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop over a torch-allocated device arena, with its own compute and copy streams.

    submit() takes host inputs (numpy or page-locked torch CPU tensors) and returns the tag; the
    request's output arrays are allocated page-locked here and returned by poll() together with the
    completion record once the request has finished."""

    def __init__(self, arena_bytes, max_slots=256, max_surfels_per_epoch=2_000_000):
        torch = _torch()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        self.compute = torch.cuda.Stream()
        self.copy = torch.cuda.Stream()
        self.handle = sgn_server_create(self.arena.data_ptr(), int(arena_bytes), max_slots, max_surfels_per_epoch,
                                        self.compute.cuda_stream, self.copy.cuda_stream)
        self._live = {}
        self._next = 1

    def submit(self, W, H, P, cam, keyframe, frames, poses, id0, n0, state, iters, image_dtype="f32",
               max_frames=None, tag=None, **opts):
        torch = _torch()
        F = len(frames)
        d = sgn_plan_desc_default(W, H, P, max_frames or F)
        d.image_dtype = DTYPES[image_dtype] if isinstance(image_dtype, str) else int(image_dtype)
        for k, v in opts.items():
            setattr(d, k, v)
        S = (W // P) * (H // P)

        def pinned(a, dtype):
            if isinstance(a, torch.Tensor):
                return a.contiguous()
            return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).pin_memory()

        ins = dict(kf=pinned(keyframe, np.float32), frames=[pinned(f, np.float32) for f in frames],
                   id0=pinned(id0, np.float32), n0=pinned(n0, np.float32), st0=pinned(state, np.uint8))
        outs = dict(id=torch.empty(S).pin_memory(), n=torch.empty(S, 3).pin_memory(), cost=torch.empty(S).pin_memory(),
                    nres=torch.empty(S, dtype=torch.int32).pin_memory(), status=torch.empty(S, dtype=torch.uint8).pin_memory())
        fptrs = (ctypes.c_void_p * F)(*[f.data_ptr() for f in ins["frames"]])
        T = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(F, 12))
        if tag is None:
            tag = self._next
            self._next += 1
        r = sgn_request()
        r.desc = d
        for i, c in enumerate(cam):
            r.intrinsics[i] = float(c)
        r.keyframe, r.num_frames, r.frames, r.poses = ins["kf"].data_ptr(), F, ctypes.cast(fptrs, ctypes.c_void_p).value, T.ctypes.data
        r.inv_depth0, r.normal0, r.state0 = ins["id0"].data_ptr(), ins["n0"].data_ptr(), ins["st0"].data_ptr()
        r.iters = int(iters)
        r.inv_depth, r.normal, r.cost = outs["id"].data_ptr(), outs["n"].data_ptr(), outs["cost"].data_ptr()
        r.nres, r.status, r.tag = outs["nres"].data_ptr(), outs["status"].data_ptr(), tag
        self._live[tag] = (ins, outs, fptrs, T, r)
        sgn_server_submit(self.handle, r)
        return tag

    def cancel(self, tag):
        sgn_server_cancel(self.handle, tag)

    def poll(self):
        """[(completion, outputs as numpy arrays)] of requests finished since the last poll."""
        out = []
        for c in sgn_server_poll(self.handle):
            ins, outs, *_ = self._live.pop(c.tag)
            out.append((c, {k: v.numpy().copy() for k, v in outs.items()}))
        return out

    def drain(self, timeout_ns=0):
        sgn_server_drain(self.handle, timeout_ns)

    def stats(self):
        st = sgn_server_stats(self.handle)
        return {f: getattr(st, f) for f, _ in sgn_serving_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            sgn_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
