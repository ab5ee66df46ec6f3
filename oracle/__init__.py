"""FP64 CPU oracle of the per-surfel Gauss-Newton photometric optimisation (Sec. 2.1-2.4).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg may import this package; the CUDA library never does, and this package never
imports the CUDA library.  The arithmetic lives in ``surfel_gn.c`` (plain C, double
precision, one function per step of the paper); this file only marshals arguments.

Pins (tests/test_oracle_*.py): every step is checked against closed forms, finite
differences, library routines (numpy eigen/linear solvers) or brute force.  The
values of the Huber threshold k, the damping lambda and min_residuals are
conventions the paper does not give (parity unpinned for those values).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# surfel input states and output status codes (same meaning as the library's, defined here independently)
EMPTY_STATE, VALID_STATE, TO_SEED_STATE = 0, 1, 2
OK, EMPTY, UNSEEDED, UNDERDETERMINED, SINGULAR, STEP_REJECTED = 0, 1, 2, 3, 4, 5
SEEDED_FLAG = 0x40


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to this file (gcc -O2, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "surfel_gn.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("huber_k", ctypes.c_double), ("lm_lambda", ctypes.c_double),
                ("optimize_normal", ctypes.c_int), ("min_residuals", ctypes.c_int), ("lm_adaptive", ctypes.c_int),
                ("radius", ctypes.c_double)]


def params(huber_k: float = 9.0 / 255.0, lm_lambda: float = 1e-3, optimize_normal: bool = True,
           min_residuals: int = 8, lm_adaptive: bool = False, radius: float = 0.0) -> Params:
    return Params(huber_k, lm_lambda, int(bool(optimize_normal)), int(min_residuals), int(bool(lm_adaptive)),
                  float(radius))


_D = ctypes.POINTER(ctypes.c_double)
_V = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_SO lets the mutation test load a deliberately broken copy of the oracle.
            path = os.environ.get("ORACLE_SO") or build()
            lib = ctypes.CDLL(path)
            c_d, c_i = ctypes.c_double, ctypes.c_int
            sig = {
                "orc_gradients": (None, [c_i, c_i, _D, _D, _D]),
                "orc_bilinear": (c_d, [c_i, _D, c_d, c_d]),
                "orc_huber": (None, [c_d, c_d, _D, _D]),
                "orc_ray": (None, [c_d, c_d, c_d, c_d, c_d, c_d, _D]),
                "orc_inv_depth": (c_d, [_D, _D, c_d, _D]),
                "orc_inv_depth_derivative": (None, [_D, _D, c_d, _D, _D, _D]),
                "orc_warp": (c_d, [c_d, c_d, c_d, c_d, _D, _D, c_d, _D, _D]),
                "orc_tangent_basis": (None, [_D, _D, _D]),
                "orc_cholesky_solve3": (c_i, [_D, _D, _D]),
                "orc_problem_create": (_V, [c_i, c_i, c_i, c_d, c_d, c_d, c_d, _V, c_i, _V, _D]),
                "orc_problem_destroy": (None, [_V]),
                "orc_eval_surfel": (None, [_V, ctypes.POINTER(Params), c_i, c_d, _D, _D, _D, _D,
                                           ctypes.POINTER(c_i), _D, _D, _D]),
                "orc_damped_step": (c_i, [_D, _D, c_d, c_i, _D]),
                "orc_apply_step": (None, [_D, c_d, _D, _D, _D]),
                "orc_gauss_newton": (c_i, [_V, ctypes.POINTER(Params), c_i, c_i, _D, _D, _V, _D, _V, _V, _V, _V, _V, _V]),
                "orc_problem_create_planes": (_V, [c_i, c_i, c_i, c_d, c_d, c_d, c_d, _V, c_i, _D, _D, _D, _D]),
                "orc_seed": (None, [_V, _D, _D, _V, _D, _D, _V]),
                "orc_depth_map": (None, [_V, _D, _D, _V, _D, _V]),
                "orc_cost_grid": (None, [_V, ctypes.POINTER(Params), c_i, ctypes.c_long, _D, _D, _D, _V]),
                "orc_transfer_surfels": (None, [_D, _D, c_i, _D, _D, _D, _D, _D, _D, _V]),
                "orc_render_surfels": (None, [_D, c_i, c_i, c_i, _D, _D, _D, _V, c_d, _D, _V, _V]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _v(a):
    return None if a is None else a.ctypes.data_as(_V)


def _vec(x, n=3):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


# ------------------------------------------------------------------------------ per-step functions


def transfer_surfels(cam, T, u, inv_depth, normal):
    """Sec. 2.5, Eq. 10: free surfels (pixel u_s (n, 2), inverse depth (n,), normal (n, 3)) of
    reference frame kf0 expressed in kf1, T (3, 4) mapping kf0 to kf1 coordinates.  Returns
    (u, inv_depth, normal, valid)."""
    cam = np.ascontiguousarray(cam, dtype=np.float64).reshape(4)
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(12)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 2)
    idv = np.ascontiguousarray(inv_depth, dtype=np.float64).reshape(-1)
    nv = np.ascontiguousarray(normal, dtype=np.float64).reshape(-1, 3)
    n = len(idv)
    uo, io, no, valid = np.empty((n, 2)), np.empty(n), np.empty((n, 3)), np.empty(n, np.uint8)
    _load().orc_transfer_surfels(_d(cam), _d(T), n, _d(u), _d(idv), _d(nv), _d(uo), _d(io), _d(no), _v(valid))
    return uo, io, no, valid


def render_surfels(cam, W, H, u, inv_depth, normal, valid, radius, with_second=False):
    """Sec. 2.2 depth-buffered render of free surfels of radius ``radius`` (Eq. 3, Eq. 4).
    Returns (inv_depth (H, W), surfel index (H, W)[, runner-up inverse depth (H, W)])."""
    cam = np.ascontiguousarray(cam, dtype=np.float64).reshape(4)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 2)
    idv = np.ascontiguousarray(inv_depth, dtype=np.float64).reshape(-1)
    nv = np.ascontiguousarray(normal, dtype=np.float64).reshape(-1, 3)
    valid = np.ascontiguousarray(valid, dtype=np.uint8).reshape(-1)
    inv, sidx = np.empty((H, W)), np.empty((H, W), np.int32)
    second = np.empty((H, W)) if with_second else None
    _load().orc_render_surfels(_d(cam), int(W), int(H), len(idv), _d(u), _d(idv), _d(nv), _v(valid), float(radius),
                               _d(inv), _v(sidx), _v(second))
    return (inv, sidx, second) if with_second else (inv, sidx)


def gradients(img):
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    gx, gy = np.empty_like(img), np.empty_like(img)
    _load().orc_gradients(W, H, _d(img), _d(gx), _d(gy))
    return gx, gy


def bilinear(img, x, y):
    img = np.ascontiguousarray(img, dtype=np.float64)
    return _load().orc_bilinear(img.shape[1], _d(img), float(x), float(y))


def huber(r, k):
    rho, w = ctypes.c_double(), ctypes.c_double()
    _load().orc_huber(float(r), float(k), ctypes.byref(rho), ctypes.byref(w))
    return rho.value, w.value


def ray(cam, ux, uy):
    r = np.empty(3)
    _load().orc_ray(*map(float, cam), float(ux), float(uy), _d(r))
    return r


def inv_depth(r_u, r_s, id_s, n):
    r_u, r_s, n = _vec(r_u), _vec(r_s), _vec(n)
    return _load().orc_inv_depth(_d(r_u), _d(r_s), float(id_s), _d(n))


def inv_depth_derivative(r_u, r_s, id_s, n):
    r_u, r_s, n = _vec(r_u), _vec(r_s), _vec(n)
    dn, did = np.empty(3), ctypes.c_double()
    _load().orc_inv_depth_derivative(_d(r_u), _d(r_s), float(id_s), _d(n), _d(dn), ctypes.byref(did))
    return dn, did.value


def warp(cam, T, r_u, id_u):
    """Returns (u_p (2,), d u_p / d id_u (2,), q_z)."""
    T = _vec(T, 12)
    r_u = _vec(r_u)
    up, du = np.empty(2), np.empty(2)
    qz = _load().orc_warp(*map(float, cam), _d(T), _d(r_u), float(id_u), _d(up), _d(du))
    return up, du, qz


def tangent_basis(n):
    n = _vec(n)
    t1, t2 = np.empty(3), np.empty(3)
    _load().orc_tangent_basis(_d(n), _d(t1), _d(t2))
    return t1, t2


def cholesky_solve3(A6, b):
    A6, b = _vec(A6, 6), _vec(b)
    x = np.empty(3)
    ok = _load().orc_cholesky_solve3(_d(A6), _d(b), _d(x))
    return (x if ok else None)


def damped_step(H6, g, lm_lambda, optimize_normal=True):
    H6, g = _vec(H6, 6), _vec(g)
    d = np.empty(3)
    ok = _load().orc_damped_step(_d(H6), _d(g), float(lm_lambda), int(bool(optimize_normal)), _d(d))
    return (d if ok else None)


def apply_step(n, id_s, delta):
    n, delta = _vec(n), _vec(delta)
    n_out, id_out = np.empty(3), ctypes.c_double()
    _load().orc_apply_step(_d(n), float(id_s), _d(delta), _d(n_out), ctypes.byref(id_out))
    return n_out, id_out.value


def sym3(h6):
    a = np.asarray(h6)
    return np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])


def sym4(h10):
    M = np.zeros((4, 4))
    k = 0
    for i in range(4):
        for j in range(i, 4):
            M[i, j] = M[j, i] = h10[k]
            k += 1
    return M


# ------------------------------------------------------------------------------ whole problem


class Problem:
    """Oracle copy of one keyframe problem (images, gradients, poses) in double precision."""

    def __init__(self, W, H, P, cam, keyframe, frames, poses):
        lib = _load()
        self.W, self.H, self.P = int(W), int(H), int(P)
        self.cam = tuple(float(c) for c in cam)
        kf = np.ascontiguousarray(keyframe, dtype=np.float32)
        fr = np.ascontiguousarray(frames, dtype=np.float32)
        ps = np.ascontiguousarray(poses, dtype=np.float64)
        self.F = fr.shape[0]
        self.S = (self.W // self.P) * (self.H // self.P)
        self._h = lib.orc_problem_create(self.W, self.H, self.P, *self.cam, _v(kf), self.F, _v(fr), _d(ps))

    @classmethod
    def from_synth(cls, prob):
        return cls(prob.W, prob.H, prob.P, prob.cam, prob.keyframe, prob.frames, prob.poses)

    @classmethod
    def from_planes(cls, W, H, P, cam, keyframe, I, gx, gy, poses):
        """Problem whose frame intensity and gradient planes (F, H, W) are given, not computed."""
        self = cls.__new__(cls)
        lib = _load()
        self.W, self.H, self.P = int(W), int(H), int(P)
        self.cam = tuple(float(c) for c in cam)
        kf = np.ascontiguousarray(keyframe, dtype=np.float32)
        I, gx, gy = (np.ascontiguousarray(a, dtype=np.float64) for a in (I, gx, gy))
        ps = np.ascontiguousarray(poses, dtype=np.float64)
        self.F = I.shape[0]
        self.S = (self.W // self.P) * (self.H // self.P)
        self._h = lib.orc_problem_create_planes(self.W, self.H, self.P, *self.cam, _v(kf), self.F, _d(I), _d(gx),
                                                _d(gy), _d(ps))
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_problem_destroy(h)
            self._h = None

    def eval_surfel(self, prm: Params, s: int, id_s: float, n):
        n = _vec(n)
        H, g, H4, g4 = np.empty(6), np.empty(3), np.empty(10), np.empty(4)
        E, mg = ctypes.c_double(), ctypes.c_double()
        cnt = ctypes.c_int()
        _load().orc_eval_surfel(self._h, ctypes.byref(prm), int(s), float(id_s), _d(n), _d(H), _d(g),
                                ctypes.byref(E), ctypes.byref(cnt), ctypes.byref(mg), _d(H4), _d(g4))
        return dict(H=H, g=g, E=E.value, cnt=cnt.value, margin=mg.value, H4=H4, g4=g4)

    def cost_grid(self, prm: Params, s: int, ids, normals):
        """Huber cost (Eq. 5) and valid-sample count of surfel s at each candidate (id, n)."""
        ids = np.ascontiguousarray(ids, dtype=np.float64).reshape(-1)
        normals = np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, 3)
        E, cnt = np.empty(len(ids)), np.empty(len(ids), np.int32)
        _load().orc_cost_grid(self._h, ctypes.byref(prm), int(s), len(ids), _d(ids), _d(normals), _d(E), _v(cnt))
        return E, cnt

    def seed(self, id0, n0, state):
        id_in = np.ascontiguousarray(id0, dtype=np.float64)
        n_in = np.ascontiguousarray(n0, dtype=np.float64).reshape(-1)
        st = np.ascontiguousarray(state, dtype=np.uint8)
        id_out, n_out, status = np.empty(self.S), np.empty(3 * self.S), np.empty(self.S, np.uint8)
        _load().orc_seed(self._h, _d(id_in), _d(n_in), _v(st), _d(id_out), _d(n_out), _v(status))
        return id_out, n_out.reshape(-1, 3), status

    def gauss_newton(self, prm: Params, iters: int, id_s, n, status, nthreads: int = 0, diagnostics=True):
        id_s = np.array(id_s, dtype=np.float64, copy=True)
        n = np.array(n, dtype=np.float64, copy=True).reshape(-1)
        status = np.array(status, dtype=np.uint8, copy=True)
        cost, nres = np.empty(self.S), np.empty(self.S, np.int32)
        margin = np.empty(self.S) if diagnostics else None
        H_last = np.empty(6 * self.S) if diagnostics else None
        path_n = np.empty(self.S) if diagnostics else None
        path_id = np.empty(self.S) if diagnostics else None
        dmargin = np.empty(self.S) if diagnostics else None
        used = _load().orc_gauss_newton(self._h, ctypes.byref(prm), int(iters), int(nthreads), _d(id_s), _d(n),
                                        _v(status), _d(cost), _v(nres), _v(margin), _v(H_last), _v(path_n),
                                        _v(path_id), _v(dmargin))
        out = dict(id=id_s, n=n.reshape(-1, 3), status=status, cost=cost, nres=nres, threads=used)
        if diagnostics:
            out["margin"] = margin
            out["H_last"] = H_last.reshape(-1, 6)
            out["path_n"] = path_n
            out["path_id"] = path_id
            out["decision_margin"] = dmargin
        return out

    def depth_map(self, id_s, n, status):
        id_s = np.ascontiguousarray(id_s, dtype=np.float64)
        n = np.ascontiguousarray(n, dtype=np.float64).reshape(-1)
        status = np.ascontiguousarray(status, dtype=np.uint8)
        inv = np.empty(self.W * self.H)
        sidx = np.empty(self.W * self.H, np.int32)
        _load().orc_depth_map(self._h, _d(id_s), _d(n), _v(status), _d(inv), _v(sidx))
        return inv.reshape(self.H, self.W), sidx.reshape(self.H, self.W)

    def solve(self, prm: Params, iters: int, id0, n0, state, nthreads: int = 0, depth_map=True):
        """The whole path: seeding (Sec. 2.3), Gauss-Newton (Sec. 2.4), final cost, depth map (Sec. 2.2)."""
        id_s, n, status = self.seed(id0, n0, state)
        out = self.gauss_newton(prm, iters, id_s, n, status, nthreads)
        if depth_map and prm.radius > 0:
            # circular surfels may overlap: the depth-buffered render of the discs (Sec. 2.2)
            TX = self.W // self.P
            s = np.arange(self.S)
            u = np.stack([(s % TX) * self.P + (self.P - 1) / 2.0, (s // TX) * self.P + (self.P - 1) / 2.0], 1)
            st = out["status"] & 0x3F
            drawn = ((st != EMPTY) & (st != UNSEEDED)).astype(np.uint8)
            out["inv_depth"], out["sidx"] = render_surfels(self.cam, self.W, self.H, u, out["id"], out["n"], drawn,
                                                           prm.radius)
        elif depth_map:
            out["inv_depth"], out["sidx"] = self.depth_map(out["id"], out["n"], out["status"])
        out["seeded_id"], out["seeded_n"], out["seeded_status"] = id_s, n, status
        return out
