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
    keep = {k: opts[k] for k in ("huber_k", "lm_lambda", "optimize_normal", "min_residuals") if k in opts}
    return oracle.params(**keep)


def oracle_solve(prob, iters, **opts):
    ob = oracle.Problem.from_synth(prob)
    out = ob.solve(oracle_params(**opts), iters, prob.id0, prob.n0, prob.state)
    out["problem"] = ob
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


def compare(prob, g, o, margin_px=1e-3, min_normal_eig=None):
    """Per-surfel errors of the GPU result against the oracle.

    Compared set: status OK in both (low bits) and no sample of the oracle within margin_px of a
    validity bound (a bound the FP32 and FP64 paths may decide differently); optionally, the
    oracle's normal equations determine the normal well (smallest tangent eigenvalue of the last
    iteration >= min_normal_eig).  Returns errors over the compared set and over all surfels
    usable in both, with counts of each exclusion.
    """
    gs, os_ = g["status"] & 0x3F, o["status"] & 0x3F
    usable = (gs == 0) & (os_ == 0)
    margin_ok = o["margin"] > margin_px
    cmp = usable & margin_ok
    excl = dict(status=int((~((gs == 0) & (os_ == 0)) & (os_ != oracle.EMPTY)).sum()),
                margin=int((usable & ~margin_ok).sum()))
    if min_normal_eig is not None:
        lam = tangent_min_eig(o["H_last"])
        well = lam >= min_normal_eig
        excl["ill_posed"] = int((cmp & ~well).sum())
        cmp &= well
    rel = np.abs(g["id"].astype(np.float64) / o["id"] - 1.0)
    ang = angle_deg(g["n"], o["n"])
    st = dict(n=int(cmp.sum()), n_usable=int(usable.sum()), excluded=excl,
              status_mismatch=int((g["status"] != o["status"]).sum()))
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
