"""The plan calls are capturable: uploads from device memory, frame preparation, the solve and the
device-to-device reads recorded into a CUDA graph replay to the eager result."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_captured_step_replays_to_the_eager_result():
    import torch

    import paper_1910_01997_gb300 as sgn

    prob = synth.room_problem(9)
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = sgn.Plan(prob.W, prob.H, prob.P, prob.F, stream=stream)
        plan.set_intrinsics(*prob.cam)
        kf = torch.from_numpy(prob.keyframe).to(dev)
        frames = torch.from_numpy(prob.frames).to(dev)
        id0 = torch.from_numpy(prob.id0.astype(np.float32)).to(dev)
        n0 = torch.from_numpy(prob.n0.astype(np.float32)).to(dev)
        st0 = torch.from_numpy(prob.state).to(dev)
        out = [torch.empty(prob.S, device=dev), torch.empty(prob.S, 3, device=dev), torch.empty(prob.S, device=dev),
               torch.empty(prob.S, dtype=torch.int32, device=dev), torch.empty(prob.S, dtype=torch.uint8, device=dev)]

        def step():
            plan.set_keyframe(kf)
            plan.set_frames([frames[i] for i in range(prob.F)], prob.poses)
            plan.init_surfels(id0, n0, st0)
            plan.solve(10)
            sgn.sgn_read_surfels(plan.handle, *[t.data_ptr() for t in out], sgn.SGN_DEVICE)

        step()
        stream.synchronize()
        eager = [t.clone() for t in out]
        for t in out:
            t.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        for _ in range(3):
            g.replay()
        stream.synchronize()
    for a, b in zip(eager, out):
        assert torch.equal(a, b)
