"""Depth-only ablation (Sec. 4.4: d id_u / d n set to zero, only the inverse depth optimised),
quantified against the synthetic scenes' ground truth on the GPU path."""
import pytest

import synth
from helpers import gpu_solve, gt_errors

pytestmark = pytest.mark.gpu


def _both(prob, iters=10):
    full = gt_errors(prob, gpu_solve(prob, iters))
    depth_only = gt_errors(prob, gpu_solve(prob, iters, optimize_normal=False))
    print("full", full)
    print("depth-only", depth_only)
    return full, depth_only


def test_normal_estimation_improves_reconstruction_where_normals_are_observable():
    """Ring scene (baselines in every direction, 16x16 surfels, initial normals 0-10 deg off, initial
    inverse depth +-10 %): optimising the normal recovers it and the per-pixel inverse depth across
    each tile; depth-only keeps the initial normal, so pixels away from the tile centre stay off."""
    full, depth_only = _both(synth.ring_problem(0, P=16))
    assert full["normal_deg_median"] < 0.25 * depth_only["normal_deg_median"]
    assert full["depth_rel_median"] < 0.5 * depth_only["depth_rel_median"]
    assert full["depth_rel_p90"] < depth_only["depth_rel_p90"]


def test_ablation_on_the_benchmark_workload_is_reported():
    """640x480 room, 8x8 surfels, 2.5 cm steps: normals are weakly observable here (see the design
    notes), so only sanity is asserted; the numbers are printed and reported by the benchmark."""
    full, depth_only = _both(synth.room_problem(0))
    for r in (full, depth_only):
        assert r["pixels"] > 100_000 and r["depth_rel_median"] < 0.05
