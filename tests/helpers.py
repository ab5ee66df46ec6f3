"""Shared test helpers: run a synthetic problem through the CUDA library and through the oracle,
and compare the two."""
from __future__ import annotations

import numpy as np

import oracle
import synth


def gpu_solve(prob, iters, dtype="f32", lanes=0, block=0, steps=None, **opts):
    """Whole path through the C ABI (upload, prep, seeding, iterations, readback)."""
    import paper_1910_01997_gb300 as sgn

    plan = sgn.Plan(prob.W, prob.H, prob.P, prob.F, dtype, lanes_per_surfel=lanes, block_threads=block, **opts)
    plan.set_intrinsics(*prob.cam)
    plan.set_keyframe(prob.keyframe)
    plan.set_frames(prob.frames, prob.poses)
    plan.init_surfels(prob.id0, prob.n0, prob.state)
    if steps is None:
        plan.solve(iters)
    else:
        steps(plan)
    out = plan.read_surfels()
    out["inv_depth"], out["sidx"] = plan.read_depth_map()
    out["plan"] = plan
    return out


def oracle_params(**opts):
    keep = {k: opts[k] for k in ("huber_k", "lm_lambda", "optimize_normal", "min_residuals", "lm_adaptive", "radius")
            if k in opts}
    return oracle.params(**keep)


def with_frames(prob, frames):
    """Copy of a problem with other frame intensities (e.g. rounded to a storage type)."""
    return synth.Problem(**{**prob.__dict__, "frames": np.asarray(frames, np.float32)})


def oracle_solve(prob, iters, **opts):
    ob = oracle.Problem.from_synth(prob)
    out = ob.solve(oracle_params(**opts), iters, prob.id0, prob.n0, prob.state)
    out["problem"] = ob
    return out


# The FP32 rounding scale of the kernel's inputs: the GPU starts from float32(id0), float32(n0), a
# relative change of at most 2^-24 per value; the stability test perturbs the oracle's initial values
# by twice that (one FP32 ulp, relative).  The FP32 error of each later step is covered separately
# by the path x condition-number criterion of oracle_stable.
FP32_INPUT_EPS = 2.0 ** -23


def round_bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even) and back, in numpy."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def quantize(frames, dtype):
    if dtype == "f16":
        return np.asarray(frames, np.float32).astype(np.float16).astype(np.float32)
    if dtype == "bf16":
        return round_bf16(frames)
    return np.asarray(frames, np.float32)


MANTISSA_BITS = {"f32": 23, "f16": 10, "bf16": 7}
# Texel formats: the type their intensity and their gradient are stored in.
INTENSITY_TYPE = {"f32": "f32", "f16": "f16", "bf16": "bf16", "f16g": "f32", "bf16g": "f32"}
GRADIENT_TYPE = {"f32": "f32", "f16": "f16", "bf16": "bf16", "f16g": "f16", "bf16g": "bf16"}


def ulp(x, dtype):
    """Unit in the last place of x in the given storage type."""
    x = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(x, 1e-30)))
    return np.exp2(e - MANTISSA_BITS[dtype])


def stored_planes(frames, dtype):
    """Intensity and central-difference gradient planes as a texel format stores them: intensities
    in the format's intensity type, gradients as half differences of the stored intensities (in
    FP32, where they are exact for FP16/BF16 intensities) rounded to the format's gradient type,
    zero on the border rows/columns.  Computed here in numpy from the inputs."""
    Iq = quantize(frames, INTENSITY_TYPE[dtype]).astype(np.float32)
    gx = np.zeros_like(Iq)
    gy = np.zeros_like(Iq)
    gx[:, :, 1:-1] = np.float32(0.5) * (Iq[:, :, 2:] - Iq[:, :, :-2])
    gy[:, 1:-1, :] = np.float32(0.5) * (Iq[:, 2:, :] - Iq[:, :-2, :])
    gt = GRADIENT_TYPE[dtype]
    return Iq.astype(np.float64), quantize(gx, gt).astype(np.float64), quantize(gy, gt).astype(np.float64)


def oracle_solve_planes(prob, planes, iters, **opts):
    ob = oracle.Problem.from_planes(prob.W, prob.H, prob.P, prob.cam, prob.keyframe, *planes, prob.poses)
    out = ob.solve(oracle_params(**opts), iters, prob.id0, prob.n0, prob.state)
    out["problem"] = ob
    return out


# A surfel is stable when every re-run of the oracle stays within this fraction of the tolerance: the
# GPU is one more sample of the same rounding-scale perturbations, and over the compared surfels of
# the full-size workloads its deviation stays within three times the largest re-run deviation for
# all but a few in ten thousand surfels.
STABLE_FRACTION = 1.0 / 3.0


def oracle_stable(prob, iters, tol_depth, tol_deg, base, dtype="f32", eps=FP32_INPUT_EPS, seeds=(1, 2, 3),
                  planes=None, step_seeds=(11, 12), frac_tol=STABLE_FRACTION, **opts):
    """Surfels whose oracle result after `iters` iterations is a stable function of the inputs.

    The oracle alone is re-run with the initial parameters perturbed by a relative eps (default: one
    FP32 ulp, the rounding the GPU's inputs undergo) and the frame data perturbed at the rounding
    scale of the format's intensity type (uniform +-ulp/2 per pixel for each seed; for FP32 +-2 ulp,
    standing for the FP32 arithmetic of a sample), plus, for the reduced-precision formats, once on
    the intensity and gradient planes as that format stores them; and, with step_seeds, re-run one
    iteration at a time with its parameters rounded to FP32 and perturbed by FP32_STEP_EPS (relative)
    after every iteration.  With `planes` (intensity and gradient planes given to the
    oracle) those planes are perturbed by +-2 FP32 ulp.  A surfel is stable when every re-run keeps
    its status and stays within frac_tol (a third) of the tolerance of the unperturbed result, and when the path its
    parameters travel over the iterations, times the condition number of its scaled normal
    equations and 1e-6 (the relative FP32 error of one step), stays below that fraction of the tolerance:
    element-by-element parity is only defined there.
    """
    prm = oracle_params(**opts)
    stable = np.ones(prob.S, bool)
    kappa = scaled_cond(base["H_last"]) if prm.optimize_normal else np.ones(prob.S)
    with np.errstate(invalid="ignore"):
        stable &= (base["path_n"] * kappa * 1e-6 <= frac_tol * tol_deg) & (base["path_id"] * kappa * 1e-6 <= frac_tol * tol_depth)
    problems = []
    for k in seeds:
        rng = np.random.default_rng([k, 77])
        if planes is not None:
            pl = [a + 2.0 * ulp(a, "f32") * rng.uniform(-1, 1, a.shape) for a in planes]
            problems.append((k, oracle.Problem.from_planes(prob.W, prob.H, prob.P, prob.cam, prob.keyframe, *pl,
                                                           prob.poses)))
        else:
            itype = INTENSITY_TYPE[dtype]
            scale = 2.0 if itype == "f32" else 0.5
            frames = prob.frames + scale * ulp(prob.frames, itype) * rng.uniform(-1, 1, prob.frames.shape)
            problems.append((k, oracle.Problem(prob.W, prob.H, prob.P, prob.cam, prob.keyframe, frames, prob.poses)))
    if planes is None and dtype != "f32":
        problems.append((99, oracle.Problem.from_planes(prob.W, prob.H, prob.P, prob.cam, prob.keyframe,
                                                        *stored_planes(prob.frames, dtype), prob.poses)))
    for k, ob in problems:
        rng = np.random.default_rng([k, 78])
        id1 = prob.id0 * (1.0 + eps * rng.standard_normal(prob.S))
        n1 = prob.n0 + eps * rng.standard_normal(prob.n0.shape)
        n1 /= np.maximum(np.linalg.norm(n1, axis=1, keepdims=True), 1e-30)
        p = ob.solve(prm, iters, id1, n1, prob.state, depth_map=False)
        stable &= (p["status"] == base["status"])
        stable &= np.abs(p["id"] / np.where(base["id"] != 0, base["id"], 1.0) - 1.0) <= frac_tol * tol_depth
        stable &= angle_deg(p["n"], base["n"]) <= frac_tol * tol_deg
    if step_seeds and not prm.lm_adaptive:
        # the parameters perturbed after every iteration (the rounding of the GPU's FP32 state)
        if planes is not None:
            ob = oracle.Problem.from_planes(prob.W, prob.H, prob.P, prob.cam, prob.keyframe, *planes, prob.poses)
        else:
            ob = oracle.Problem.from_synth(prob)
        for k in step_seeds:
            p = oracle_perturbed_steps(ob, prm, iters, prob.id0, prob.n0, prob.state, np.random.default_rng([k, 79]),
                                       FP32_STEP_EPS)
            # each iteration's FP32 sums (relative error ~1e-6) move its step by up to that much
            # times the scaled condition number of the iteration's normal equations
            stable &= (p["step_err_n"] * 1e-6 <= frac_tol * tol_deg) & (p["step_err_id"] * 1e-6 <= frac_tol * tol_depth)
            stable &= (p["status"] == base["status"])
            stable &= np.abs(p["id"] / np.where(base["id"] != 0, base["id"], 1.0) - 1.0) <= frac_tol * tol_depth
            stable &= angle_deg(p["n"], base["n"]) <= frac_tol * tol_deg
    return stable


# Relative perturbation of the parameters after every iteration in the stability re-runs: the GPU keeps
# id_s and n in FP32, so each update rounds them (half an ulp) on top of the FP32 error of the step
# itself (a few ulps); two ulps stand for both.
FP32_STEP_EPS = 2.0 ** -22


def oracle_perturbed_steps(ob, prm, iters, id0, n0, state, rng, rel):
    """The oracle's seeding and Gauss-Newton iterations one at a time, with the parameters rounded to
    FP32 and multiplied by (1 + rel u), u uniform in [-1, 1], after every iteration (the normal
    renormalised): the oracle's result under a per-iteration perturbation at the FP32 rounding scale.
    Also returns, per surfel, the sum over the iterations of each step's size (normal rotation in
    degrees, relative inverse-depth change) times the scaled condition number of that iteration's
    normal equations ("step_err_n", "step_err_id"): the first-order growth of an FP32 relative error
    in the sums of one iteration through its solve."""
    id_s, n, status = ob.seed(id0, n0, state)
    p = None
    err_n, err_id = np.zeros(len(id_s)), np.zeros(len(id_s))
    for _ in range(iters):
        p = ob.gauss_newton(prm, 1, id_s, n, status, diagnostics=True)
        kap = scaled_cond(p["H_last"]) if prm.optimize_normal else np.ones(len(id_s))
        with np.errstate(invalid="ignore"):
            err_n += np.nan_to_num(p["path_n"] * kap, nan=np.inf)
            err_id += np.nan_to_num(p["path_id"] * kap, nan=np.inf)
        id_s = p["id"].astype(np.float32).astype(np.float64) * (1.0 + rel * rng.uniform(-1, 1, len(p["id"])))
        n = p["n"].astype(np.float32).astype(np.float64) * (1.0 + rel * rng.uniform(-1, 1, p["n"].shape))
        n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-30)
        status = p["status"]
    if p is None:
        p = ob.gauss_newton(prm, 0, id_s, n, status, diagnostics=False)
    else:  # parameters of the last iteration, unperturbed
        p = ob.gauss_newton(prm, 0, p["id"], p["n"], p["status"], diagnostics=False)
    p["step_err_n"], p["step_err_id"] = err_n, err_id
    return p


def scaled_cond(H6):
    """2-norm condition numbers of the Jacobi-scaled (unit-diagonal) 3x3 normal matrices."""
    H = np.stack([np.asarray(H6)[:, i] for i in (0, 1, 2, 1, 3, 4, 2, 4, 5)], 1).reshape(-1, 3, 3)
    d = np.einsum("nii->ni", H)
    good = (d > 0).all(1)
    out = np.full(len(H), np.inf)
    if good.any():
        sq = np.sqrt(d[good])
        S = H[good] / (sq[:, :, None] * sq[:, None, :])
        w = np.linalg.eigvalsh(S)
        out[good] = w[:, -1] / np.maximum(w[:, 0], 1e-300)
    return out


def angle_deg(a, b):
    """Angle between unit normals, sign-invariant (Eq. 3 does not see the sign of n)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    return np.rad2deg(np.arccos(np.clip(np.abs(np.einsum("...i,...i->...", a, b)), 0.0, 1.0)))


def tangent_min_eig(H6):
    """Smallest eigenvalue of the 2x2 tangent block of packed 3x3 normal matrices."""
    H6 = np.asarray(H6, np.float64)
    a, b, c = H6[:, 0], H6[:, 1], H6[:, 3]
    tr, det = a + c, a * c - b * b
    return 0.5 * (tr - np.sqrt(np.maximum(tr * tr - 4 * det, 0.0)))


def compare(prob, g, o, margin_px=1e-3, min_normal_eig=None, stable=None):
    """Per-surfel errors of the GPU result against the oracle.

    Compared set: status OK in both (low bits) and no sample of the oracle within margin_px of a
    validity bound (a bound the FP32 and FP64 paths may decide differently); optionally, the
    oracle's normal equations determine the normal well (smallest tangent eigenvalue of the last
    iteration >= min_normal_eig) and the oracle result is stable (see oracle_stable).  Returns errors over the compared set and over all surfels
    usable in both, with counts of each exclusion.
    """
    gs, os_ = g["status"] & 0x3F, o["status"] & 0x3F
    usable = (gs == 0) & (os_ == 0)
    margin_ok = o["margin"] > margin_px
    cmp = usable & margin_ok
    excl = dict(status=int((~((gs == 0) & (os_ == 0)) & (os_ != oracle.EMPTY)).sum()),
                margin=int((usable & ~margin_ok).sum()))
    if stable is not None:
        excl["unstable"] = int((cmp & ~stable).sum())
        cmp &= stable
    if min_normal_eig is not None:
        lam = tangent_min_eig(o["H_last"])
        well = lam >= min_normal_eig
        excl["ill_posed"] = int((cmp & ~well).sum())
        cmp &= well
    rel = np.abs(g["id"].astype(np.float64) / o["id"] - 1.0)
    ang = angle_deg(g["n"], o["n"])
    st = dict(n=int(cmp.sum()), n_usable=int(usable.sum()), excluded=excl,
              status_mismatch=int((gs != os_).sum()))  # outcome codes; the high bits are route flags
    for name, m in (("", cmp), ("all_", usable)):
        if m.any():
            st[name + "depth_max"] = float(rel[m].max())
            st[name + "depth_p99"] = float(np.percentile(rel[m], 99))
            st[name + "depth_med"] = float(np.median(rel[m]))
            st[name + "ang_max"] = float(ang[m].max())
            st[name + "ang_p99"] = float(np.percentile(ang[m], 99))
            st[name + "ang_med"] = float(np.median(ang[m]))
    st["rel"], st["ang"], st["mask"] = rel, ang, cmp
    return st


def gt_errors(prob, out):
    """Quality of a solve against the scene's ground truth: per-pixel inverse depth of the returned
    depth map vs the renderer's (noise-free keyframe, pixels of tiles that see one primitive and
    whose own primitive is that one), and per-surfel normal angle vs the primitive's normal."""
    _, pid, dep = prob.scene.render(0)
    sidx = out["sidx"]
    m = sidx >= 0
    tp = np.full(sidx.shape, -1)
    tp[m] = prob.tile_prim[sidx[m]]
    m &= (tp >= 0) & (pid == tp) & np.isfinite(dep) & (dep > 0)
    rel = np.abs(out["inv_depth"][m] * dep[m] - 1.0)
    ok = ((out["status"] & 0x3F) == 0) & (prob.tile_prim >= 0)
    ang = angle_deg(out["n"][ok], prob.gt_n[ok])
    return dict(pixels=int(m.sum()), depth_rel_median=float(np.median(rel)), depth_rel_p90=float(np.quantile(rel, 0.9)),
                surfels=int(ok.sum()), normal_deg_median=float(np.median(ang)), normal_deg_p90=float(np.quantile(ang, 0.9)))
