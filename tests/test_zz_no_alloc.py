"""sgn_solve_static: the whole keyframe solve for callers that must not allocate device memory
(real-time loops that may not take allocator locks or fail with out-of-memory mid-run, frameworks
that own every buffer).

It runs through the C ABI with device inputs and outputs only, its frame texels in the library's
fixed device scratch, and must give the result of the plan-based solve, within the tolerances the
parity tests use, on two calls in a row (the second reuses the scratch the first left behind).
This file is collected last on purpose.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import synth
from helpers import angle_deg, gpu_solve

pytestmark = pytest.mark.gpu

TOL = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tolerances.json")))["parity"]


def _static_solve(prob, iters, dtype):
    import torch

    import paper_1910_01997_gb300 as sgn

    dev = torch.device("cuda")
    S, W, H = prob.S, prob.W, prob.H
    desc = sgn.sgn_plan_desc_default(W, H, prob.P, prob.F)
    desc.image_dtype = sgn.DTYPES[dtype]
    kf = torch.from_numpy(prob.keyframe).to(dev)
    frames = torch.from_numpy(prob.frames).to(dev)
    frame_ptrs = (ctypes.c_void_p * prob.F)(*[frames[i].data_ptr() for i in range(prob.F)])
    poses = np.ascontiguousarray(prob.poses.reshape(prob.F, 12), dtype=np.float64)
    intr = np.ascontiguousarray(prob.cam, dtype=np.float64)
    id0 = torch.from_numpy(prob.id0.astype(np.float32)).to(dev)
    n0 = torch.from_numpy(prob.n0.astype(np.float32)).to(dev)
    st0 = torch.from_numpy(prob.state).to(dev)
    out = dict(id=torch.empty(S, device=dev), n=torch.empty(S, 3, device=dev), cost=torch.empty(S, device=dev),
               nres=torch.empty(S, dtype=torch.int32, device=dev), status=torch.empty(S, dtype=torch.uint8, device=dev),
               inv_depth=torch.empty(H, W, device=dev), sidx=torch.empty(H, W, dtype=torch.int32, device=dev))
    stream = torch.cuda.current_stream()
    sgn.sgn_solve_static(desc, intr.ctypes.data, kf.data_ptr(), W * 4, prob.F, ctypes.cast(frame_ptrs, ctypes.c_void_p),
                         W * 4, poses.ctypes.data, id0.data_ptr(), n0.data_ptr(), st0.data_ptr(), iters,
                         out["id"].data_ptr(), out["n"].data_ptr(), out["cost"].data_ptr(), out["nres"].data_ptr(),
                         out["status"].data_ptr(), out["inv_depth"].data_ptr(), out["sidx"].data_ptr(),
                         stream.cuda_stream)
    stream.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_static_solve_matches_plan_solve_twice_in_a_row():
    cases = [(synth.room_problem(0), "f32"), (synth.tiny_problem(1, noise_sigma=0.01, seed_frac=0.2), "f16")]
    for prob, dtype in cases:
        got = _static_solve(prob, 10, dtype)
        ref = gpu_solve(prob, 10, dtype=dtype)
        tol = TOL["f32"]
        assert np.mean(got["status"] != ref["status"]) < 0.01
        m = ((got["status"] & 0x3F) == 0) & ((ref["status"] & 0x3F) == 0)
        assert m.sum() > 0.5 * prob.S
        assert np.abs(got["id"][m] / ref["id"][m] - 1).max() <= tol["depth_rel"]
        assert angle_deg(got["n"][m], ref["n"][m]).max() <= tol["normal_deg"]
        assert np.allclose(got["cost"][m], ref["cost"][m], rtol=1e-4, atol=1e-7)
        px = (got["sidx"] >= 0) & (ref["sidx"] >= 0)
        assert np.mean((got["sidx"] >= 0) != (ref["sidx"] >= 0)) < 0.01
        assert np.abs(got["inv_depth"][px] / ref["inv_depth"][px] - 1).max() <= 10 * tol["depth_rel"]
        # outside full tiles the map is cleared
        assert np.all(got["sidx"][(prob.H // prob.P) * prob.P:, :] == -1)


def test_static_solve_rejects_problems_larger_than_the_scratch():
    import torch

    import paper_1910_01997_gb300 as sgn

    W, H, F = 4096, 2048, 8
    need = F * H * W * 16
    assert need > sgn.SGN_STATIC_SCRATCH_BYTES
    desc = sgn.sgn_plan_desc_default(W, H, 8, F)
    dummy = torch.zeros(16, device="cuda")
    ptrs = (ctypes.c_void_p * F)(*[dummy.data_ptr()] * F)
    poses = np.tile(np.eye(3, 4).reshape(1, 12), (F, 1)).astype(np.float64)
    intr = np.array([3584.0, 3584.0, 2047.5, 1023.5])
    p = dummy.data_ptr()
    st = sgn._status("sgn_solve_static", ctypes.byref(desc), intr.ctypes.data, p, W * 4, F,
                     ctypes.cast(ptrs, ctypes.c_void_p), W * 4, poses.ctypes.data, p, p, p, 10, p, p, p, p, p, p, p, 0)
    assert st == sgn.SGN_ERR_WORKSPACE_TOO_SMALL
    assert "static scratch" in sgn.sgn_last_error()
