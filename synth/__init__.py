"""Seeded synthetic piecewise-planar scenes: the input generator.

This module is shared by the tests, the benchmark and the smoke check.  It holds
none of the surfel method's arithmetic: it builds textured planes and rectangles,
camera poses and noise from a seed, renders images by ray casting (``scene.c``),
and reports per-tile ground truth (the primitive seen through a tile's centre
ray, and its depth) together with the perturbed initial surfel parameters that
the method starts from.

The paper evaluates on recorded 640x480 monocular sequences (Sec. 4); these
scenes stand in for them with the same image sizes and a piecewise-planar scene
structure (Sec. 2.1 models the scene as planar patches).

Conventions
-----------
* World coordinates = keyframe camera coordinates (x right, y down, z forward).
* A pose ``T`` (3x4, row-major ``[R | t]``) maps keyframe points into a camera:
  ``X_cam = R X_kf + t``.  The keyframe's own pose is the identity.
* Pixel centres are at integer coordinates; ``K = [[fx,0,cx],[0,fy,cy],[0,0,1]]``
  with ``fx = fy = 0.875 W``, ``cx = (W-1)/2``, ``cy = (H-1)/2``.
* Tile ``s = ty * (W // P) + tx`` covers pixels ``[tx P, tx P + P - 1] x
  [ty P, ty P + P - 1]``; its centre is ``(tx P + (P-1)/2, ty P + (P-1)/2)``.
* Surfel state codes: 0 empty, 1 valid (has initial parameters), 2 to be seeded.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

PRIM_DTYPE = np.dtype(
    [
        ("kind", np.int32), ("pad_", np.int32), ("n", np.float64, 3), ("d", np.float64),
        ("o", np.float64, 3), ("e1", np.float64, 3), ("e2", np.float64, 3),
        ("half1", np.float64), ("half2", np.float64), ("cell", np.float64),
        ("bright", np.float64), ("contrast", np.float64), ("seed", np.uint64),
    ],
    align=True,
)
assert PRIM_DTYPE.itemsize == 160

EMPTY, VALID, TO_SEED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to this file (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "scene.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
             src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.synth_render.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_render.restype = None
            lib.synth_shade_points.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, ctypes.c_long, dp,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_shade_points.restype = None
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------------------------
# geometry helpers (scene construction only)

def rot_axis_angle(axis, angle: float) -> np.ndarray:
    """Rodrigues rotation matrix for a unit axis and an angle in radians."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * k + (1 - np.cos(angle)) * (k @ k)


def rot_x(deg: float) -> np.ndarray:
    return rot_axis_angle([1, 0, 0], np.deg2rad(deg))


def rot_y(deg: float) -> np.ndarray:
    return rot_axis_angle([0, 1, 0], np.deg2rad(deg))


def pose(R, t) -> np.ndarray:
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _perp_axes(n):
    n = _unit(n)
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = _unit(np.cross(n, a))
    e2 = np.cross(n, e1)
    return e1, e2


def _prim(kind, n, point, e1, e2, half1, half2, cell, rng):
    p = np.zeros((), dtype=PRIM_DTYPE)
    n = _unit(n)
    p["kind"] = kind
    p["n"] = n
    p["d"] = float(n @ point)
    p["o"] = point
    p["e1"] = e1
    p["e2"] = e2
    p["half1"] = half1
    p["half2"] = half2
    p["cell"] = cell
    p["bright"] = rng.uniform(0.35, 0.65)
    p["contrast"] = rng.uniform(0.5, 0.7)
    p["seed"] = np.uint64(rng.integers(0, 2**63 - 1))
    return p


def intrinsics(W: int, H: int) -> tuple:
    f = 0.875 * W
    return (f, f, (W - 1) / 2.0, (H - 1) / 2.0)


class Scene:
    """Primitives + intrinsics + poses (index 0 is the keyframe, identity pose)."""

    def __init__(self, prims: np.ndarray, W: int, H: int, poses: list, name: str):
        self.prims = np.ascontiguousarray(prims, dtype=PRIM_DTYPE)
        self.W, self.H = int(W), int(H)
        self.cam = np.array(intrinsics(W, H), dtype=np.float64)
        self.poses = [np.ascontiguousarray(p, dtype=np.float64) for p in poses]
        self.name = name

    @property
    def K(self) -> np.ndarray:
        fx, fy, cx, cy = self.cam
        return np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1.0]])

    def render(self, idx: int, noise: np.ndarray | None = None):
        """Point-sampled image of camera ``idx`` (float32 HxW), primitive ids, depths."""
        lib = _load()
        W, H = self.W, self.H
        img = np.empty((H, W), np.float32)
        pid = np.empty((H, W), np.int32)
        dep = np.empty((H, W), np.float64)
        nz = None if noise is None else np.ascontiguousarray(noise, dtype=np.float64)
        lib.synth_render(_ptr(self.prims), len(self.prims), _dp(self.cam), _dp(self.poses[idx]), W, H,
                         _ptr(nz), _ptr(img), _ptr(pid), _ptr(dep))
        return img, pid, dep

    def shade(self, idx: int, xy: np.ndarray):
        """Noise-free continuous intensity of camera ``idx`` at pixel positions ``xy`` (N x 2)."""
        lib = _load()
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        out = np.empty(len(xy))
        pid = np.empty(len(xy), np.int32)
        dep = np.empty(len(xy))
        lib.synth_shade_points(_ptr(self.prims), len(self.prims), _dp(self.cam), _dp(self.poses[idx]),
                               len(xy), _dp(xy), _ptr(out), _ptr(pid), _ptr(dep))
        return out, pid, dep


# ----------------------------------------------------------------------------------------------
# scene families

def planes_scene(seed: int, W: int = 160, H: int = 120) -> Scene:
    """Three textured planes, normals within 40 deg of the optical axis, depth 1.5-3 m.

    Observing cameras: t = (0.05, 0, 0) with R = R_y(2 deg); t = (0, 0.05, 0) with R = R_x(-2 deg).
    """
    rng = np.random.default_rng([seed, 1])
    fx = intrinsics(W, H)[0]
    prims = []
    for _ in range(3):
        tilt = np.deg2rad(rng.uniform(0, 40))
        az = rng.uniform(0, 2 * np.pi)
        n = np.array([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), -np.cos(tilt)])
        z0 = rng.uniform(1.5, 3.0)
        px = rng.uniform(-0.3, 0.3) * W / fx * z0
        py = rng.uniform(-0.3, 0.3) * H / fx * z0
        point = np.array([px, py, z0])
        e1, e2 = _perp_axes(n)
        cell = 0.25 * (160.0 / W)
        prims.append(_prim(0, n, point, e1, e2, 0, 0, cell, rng))
    poses = [pose(np.eye(3), [0, 0, 0]), pose(rot_y(2.0), [0.05, 0, 0]), pose(rot_x(-2.0), [0, 0.05, 0])]
    return Scene(np.array(prims), W, H, poses, f"planes{W}x{H}s{seed}")


def smooth_trajectory(rng, n_frames: int, step: float = 0.025, max_rot_deg: float = 1.0) -> list:
    """Keyframe->camera poses of a sum-of-sines path; frame 0 is the keyframe.

    Positions and rotation vectors are sums of three sines per axis, rescaled so that
    the mean camera step is ``step`` metres and the largest step rotation is
    ``max_rot_deg`` degrees.
    """
    tau = np.arange(n_frames + 1, dtype=np.float64)

    def sines():
        out = np.zeros((len(tau), 3))
        for ax in range(3):
            for _ in range(3):
                w = rng.uniform(0.05, 0.35)
                ph = rng.uniform(0, 2 * np.pi)
                amp = rng.uniform(0.5, 1.0)
                out[:, ax] += amp * np.sin(w * tau + ph)
        return out - out[0]

    pos = sines()
    pos[:, 2] *= 0.5  # mostly sideways motion, as a hand-held camera scanning a room
    steps = np.linalg.norm(np.diff(pos, axis=0), axis=1)
    pos *= step / max(steps.mean(), 1e-12)
    rv = sines()
    rsteps = np.linalg.norm(np.diff(rv, axis=0), axis=1)
    rv *= np.deg2rad(max_rot_deg) * rng.uniform(0.6, 1.0) / max(rsteps.max(), 1e-12)
    poses = []
    for i in range(len(tau)):
        ang = np.linalg.norm(rv[i])
        Rwc = np.eye(3) if ang == 0 else rot_axis_angle(rv[i] / ang, ang)
        C = pos[i]
        R = Rwc.T
        poses.append(pose(R, -R @ C))
    return poses


def room_scene(seed: int, W: int = 640, H: int = 480, n_frames: int = 5, n_quads: int = 20) -> Scene:
    """Box room (6 walls, about 6 m wide, 3 m high, front wall 4.2-4.8 m ahead) plus
    ``n_quads`` textured rectangles (0.3-1 m sides, 1-4 m deep, tilted up to 60 deg)."""
    rng = np.random.default_rng([seed, 2])
    fx = intrinsics(W, H)[0]
    cell = 0.1 * (640.0 / W)
    prims = []
    xl, xr = -rng.uniform(2.7, 3.3), rng.uniform(2.7, 3.3)
    yt, yb = -rng.uniform(1.3, 1.7), rng.uniform(1.3, 1.7)
    zf, zb = rng.uniform(4.2, 4.8), -rng.uniform(1.0, 1.5)
    ex, ey, ez = np.eye(3)
    walls = [
        (ez * -1, np.array([0, 0, zf]), ex, ey),   # front
        (ez, np.array([0, 0, zb]), ex, ey),        # back
        (ex, np.array([xl, 0, 0]), ez, ey),        # left
        (-ex, np.array([xr, 0, 0]), ez, ey),       # right
        (ey, np.array([0, yt, 0]), ex, ez),        # ceiling
        (-ey, np.array([0, yb, 0]), ex, ez),       # floor
    ]
    for n, pt, e1, e2 in walls:
        prims.append(_prim(0, n, pt, e1, e2, 0, 0, cell, rng))
    for _ in range(n_quads):
        z = rng.uniform(1.0, 4.0)
        u = rng.uniform(0.1, W - 1.1)
        v = rng.uniform(0.1, H - 1.1)
        c = np.array([(u - (W - 1) / 2) / fx * z, (v - (H - 1) / 2) / fx * z, z])
        tilt = np.deg2rad(rng.uniform(0, 60))
        az = rng.uniform(0, 2 * np.pi)
        n = np.array([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), -np.cos(tilt)])
        e1, e2 = _perp_axes(n)
        rot = rng.uniform(0, np.pi)
        e1, e2 = np.cos(rot) * e1 + np.sin(rot) * e2, -np.sin(rot) * e1 + np.cos(rot) * e2
        prims.append(_prim(1, n, c, e1, e2, rng.uniform(0.15, 0.5), rng.uniform(0.15, 0.5), cell, rng))
    poses = smooth_trajectory(rng, n_frames)
    return Scene(np.array(prims), W, H, poses, f"room{W}x{H}s{seed}")


# ----------------------------------------------------------------------------------------------
# problems: images + ground truth + initial surfels


class Problem:
    """One keyframe solve: images, poses, intrinsics, initial surfels and ground truth.

    Arrays: ``keyframe`` (H, W) float32, ``frames`` (F, H, W) float32, ``poses`` (F, 3, 4)
    float64 keyframe->frame, ``id0`` (S,), ``n0`` (S, 3) initial inverse depth and unit
    normal (zeros where the state is not VALID), ``state`` (S,) uint8, ``gt_id`` (S,),
    ``gt_n`` (S, 3), ``tile_prim`` (S,) primitive seen by every pixel of the tile and by
    its centre ray, or -1 if the tile straddles primitives.
    """

    def __init__(self, **kw):
        self.__dict__.update(kw)

    @property
    def S(self) -> int:
        return len(self.state)

    @property
    def F(self) -> int:
        return len(self.frames)

    def residuals_per_iteration(self) -> int:
        return self.S * self.P * self.P * self.F


def render_set(scene: Scene, noise_sigma: float, seed: int, idx: list) -> dict:
    """Noisy renders {camera index: (image, primitive ids)} for the given cameras (0 = keyframe)."""
    out = {}
    for i in idx:
        nz = None
        if noise_sigma > 0:
            nz = np.random.default_rng([seed, 4, i]).normal(0.0, noise_sigma, size=(scene.H, scene.W))
        img, pid, _ = scene.render(i, nz)
        out[i] = (img, pid)
    return out


def make_problem(scene: Scene, P: int, *, noise_sigma: float = 0.0, seed_frac: float = 0.0,
                 depth_perturb: float = 0.1, normal_perturb_deg: float = 10.0, seed: int = 0,
                 frames: list | None = None, rendered: dict | None = None, init_seed: int | None = None) -> Problem:
    """Render the keyframe and observing frames and draw the initial surfels.

    Valid tiles start from ground truth with inverse depth scaled by U[1-d, 1+d] and the
    normal rotated by U[0, normal_perturb_deg] about a random perpendicular axis.  A
    ``seed_frac`` share of tiles (seeded choice) is marked TO_SEED instead.
    """
    rng = np.random.default_rng([seed if init_seed is None else init_seed, 3])
    W, H = scene.W, scene.H
    idx = list(range(1, len(scene.poses))) if frames is None else list(frames)
    if rendered is None:
        rendered = render_set(scene, noise_sigma, seed, [0] + idx)
    kf, kf_pid = rendered[0]
    fr = np.stack([rendered[i][0] for i in idx])
    poses = np.stack([scene.poses[i] for i in idx])
    TX, TY = W // P, H // P
    S = TX * TY
    ty, tx = np.divmod(np.arange(S), TX)
    cx = tx * P + (P - 1) / 2.0
    cy = ty * P + (P - 1) / 2.0
    _, cpid, cdep = scene.shade(0, np.stack([cx, cy], 1))
    gt_id = 1.0 / cdep
    gt_n = scene.prims["n"][np.maximum(cpid, 0)].copy()
    fx, fy, ccx, ccy = scene.cam
    rays = np.stack([(cx - ccx) / fx, (cy - ccy) / fy, np.ones(S)], 1)
    flip = np.einsum("ij,ij->i", gt_n, rays) > 0
    gt_n[flip] *= -1
    tiles = kf_pid[: TY * P, : TX * P].reshape(TY, P, TX, P).transpose(0, 2, 1, 3).reshape(S, P * P)
    same = (tiles == tiles[:, :1]).all(1) & (tiles[:, 0] == cpid) & (cpid >= 0)
    tile_prim = np.where(same, cpid, -1).astype(np.int32)

    state = np.full(S, VALID, np.uint8)
    state[cpid < 0] = EMPTY
    if seed_frac > 0:
        pick = rng.permutation(S)[: int(round(seed_frac * S))]
        state[pick] = np.where(state[pick] == VALID, TO_SEED, state[pick])
    id0 = np.zeros(S)
    n0 = np.zeros((S, 3))
    v = state == VALID
    nv = int(v.sum())
    id0[v] = gt_id[v] * (1.0 + rng.uniform(-depth_perturb, depth_perturb, nv))
    # rotate each normal by U[0, max] degrees about a random axis perpendicular to it (Rodrigues)
    axis = rng.normal(size=(nv, 3))
    g = gt_n[v]
    axis -= np.einsum("ij,ij->i", axis, g)[:, None] * g
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(0.0, normal_perturb_deg, nv))
    n = g * np.cos(ang)[:, None] + np.cross(axis, g) * np.sin(ang)[:, None]
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[np.einsum("ij,ij->i", n, rays[v]) > 0] *= -1
    n0[v] = n
    return Problem(W=W, H=H, P=P, cam=scene.cam.copy(), keyframe=kf, frames=fr, poses=poses, id0=id0,
                   n0=n0, state=state, gt_id=gt_id, gt_n=gt_n, tile_prim=tile_prim, scene=scene,
                   frame_index=idx, noise_sigma=noise_sigma)


# ----------------------------------------------------------------------------------------------
# named workloads


def tiny_problem(seed: int = 0, noise_sigma: float = 0.0, **kw) -> Problem:
    """160x120, three planes, two observing frames, 4x4 surfels (1200), all valid."""
    return make_problem(planes_scene(seed), 4, noise_sigma=noise_sigma, seed=seed, **kw)


def room_problem(seed: int = 0, W: int = 640, H: int = 480, F: int = 5, P: int = 8,
                 noise_sigma: float = 0.01, seed_frac: float = 0.2, **kw) -> Problem:
    """Box room + 20 rectangles, keyframe = frame 0, observing frames 1..F, P x P surfels."""
    return make_problem(room_scene(seed, W, H, F), P, noise_sigma=noise_sigma, seed_frac=seed_frac,
                        seed=seed, **kw)


def ring_scene(seed: int, W: int = 320, H: int = 240, n_frames: int = 6, radius: float = 0.12,
               cell: float = 0.25) -> Scene:
    """Two tilted textured planes about 2 m ahead, seen from ``n_frames`` cameras spaced on a
    ring of ``radius`` metres around the optical axis, each turned to look at (0, 0, 2).

    Baselines in every direction make the plane normals well observable; this scene serves
    the convergence checks, not the benchmark."""
    rng = np.random.default_rng([seed, 5])
    prims = []
    for side in (-1, 1):
        tilt = np.deg2rad(rng.uniform(15, 30))
        az = rng.uniform(0, 2 * np.pi)
        n = np.array([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), -np.cos(tilt)])
        point = np.array([side * 0.3, 0.0, rng.uniform(1.8, 2.2)])
        e1, e2 = _perp_axes(n)
        prims.append(_prim(0, n, point, e1, e2, 0, 0, cell * (320.0 / W), rng))
    poses = [pose(np.eye(3), [0, 0, 0])]
    target = np.array([0, 0, 2.0])
    for k in range(n_frames):
        a = 2 * np.pi * k / n_frames + rng.uniform(0, 0.3)
        C = radius * np.array([np.cos(a), np.sin(a), 0.0])
        z = _unit(target - C)
        x = _unit(np.cross([0, 1.0, 0], z))
        y = np.cross(z, x)
        Rwc = np.stack([x, y, z], 1)
        R = Rwc.T
        poses.append(pose(R, -R @ C))
    return Scene(np.array(prims), W, H, poses, f"ring{W}x{H}s{seed}")


def ring_problem(seed: int = 0, P: int = 16, noise_sigma: float = 0.0, **kw) -> Problem:
    return make_problem(ring_scene(seed), P, noise_sigma=noise_sigma, seed=seed, **kw)


def batch_problems(seed: int = 0, n: int = 64, scenes: int = 16, max_frames: int = 8) -> list:
    """Many keyframe problems of uneven size for batched execution: resolutions drawn from
    {320x240, 640x480, 1280x720, 1920x1080}, patch sizes from {4, 8, 16}, 2..max_frames observing
    frames, 20 % seeded tiles, noise sigma 0.01.  `scenes` box-room scenes are rendered once (with
    max_frames observing frames) and shared by the n problems, which differ in patch size, frame
    count, seeded tiles and initial perturbation."""
    rng = np.random.default_rng([seed, 6])
    sizes = [(320, 240), (640, 480), (1280, 720), (1920, 1080)]
    scene_list = []
    for k in range(scenes):
        W, H = sizes[k % len(sizes)]
        sc = room_scene(1000 + 31 * seed + k, W, H, max_frames)
        scene_list.append((sc, render_set(sc, 0.01, 1000 + k, list(range(max_frames + 1)))))
    out = []
    for j in range(n):
        sc, rendered = scene_list[int(rng.integers(len(scene_list)))]
        P = int(rng.choice([4, 8, 16]))
        F = int(rng.integers(2, max_frames + 1))
        out.append(make_problem(sc, P, noise_sigma=0.01, seed_frac=0.2, seed=1000 + j, frames=list(range(1, F + 1)),
                                rendered=rendered, init_seed=5000 + j))
    return out
