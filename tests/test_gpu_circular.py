"""Circular surfels (option surfel_radius, Eq. 4) on the GPU against the oracle."""
import numpy as np
import pytest

import synth
from helpers import gpu_solve, oracle_solve
from test_gpu_parity import _check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P,radius", [(8, 5.0), (16, 10.0), (16, 12.0), (4, 3.0)])
def test_circular_parity(P, radius):
    """Surfel-by-surfel parity at the FP32 tolerances (overlapping discs around the tile centres)."""
    prob = synth.room_problem(21, W=320, H=240, F=4, P=P)
    g, o = gpu_solve(prob, 10, surfel_radius=radius), oracle_solve(prob, 10, radius=radius)
    # 3-px discs of 28 pixels are less well determined: fewer surfels are stable at the rounding scale
    _check(prob, g, o, "f32", f"disc P{P} r{radius}", 10, frac="noisy_small" if P == 4 else "disc", radius=radius)


def test_circular_depth_map_is_the_render_of_the_discs():
    """The plan's depth map equals the depth-buffered render (sgn_render_surfels) of its solved
    surfels at the tile centres, bit for bit (same draw), and it covers the overlap of the discs."""
    import torch

    import paper_1910_01997_gb300 as sgn

    prob = synth.room_problem(22)
    g = gpu_solve(prob, 10, surfel_radius=5.0)
    TX = prob.W // prob.P
    s = np.arange(prob.S)
    u = np.stack([(s % TX) * prob.P + 3.5, (s // TX) * prob.P + 3.5], 1).astype(np.float32)
    st = g["status"] & 0x3F
    drawn = ((st != 1) & (st != 2)).astype(np.uint8)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    inv, sidx = sgn.sgn_render_surfels(prob.cam, prob.W, prob.H, t(u), t(g["id"].astype(np.float32)),
                                       t(g["n"].astype(np.float32)), t(drawn), 5.0)
    torch.cuda.synchronize()
    assert np.array_equal(sidx.cpu().numpy(), g["sidx"])
    assert np.array_equal(inv.cpu().numpy(), g["inv_depth"])
    assert (g["sidx"] >= 0).mean() > 0.9


def test_circular_rejected_where_unsupported():
    import paper_1910_01997_gb300 as sgn

    prob = synth.room_problem(23, W=160, H=120, F=2)
    with pytest.raises(sgn.SgnError):
        sgn.Plan(prob.W, prob.H, 8, 2, surfel_radius=40.0)  # more than 512 pixels
    pl = sgn.Plan(prob.W, prob.H, 8, 2, surfel_radius=5.0)
    b = sgn.Batch(2)
    b.add(pl)  # circular surfels run in their own persistent launch of a batch (test_gpu_batch)
    with pytest.raises(sgn.SgnError):
        sgn.sgn_plan_set_mapping(pl.handle, 16, 256)
