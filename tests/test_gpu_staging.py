"""Shared-memory (TMA) staging of frame texels: the staged kernel reads the same texels as the direct
gathers and does the same arithmetic, so its results equal those of the unstaged kernel bit for bit;
and every staged run of the suite completes its waits (no timeout)."""
import numpy as np
import pytest

import synth
from helpers import gpu_solve

pytestmark = pytest.mark.gpu

KEYS = ("id", "n", "cost", "nres", "status", "inv_depth", "sidx")


def _same(a, b):
    for k in KEYS:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_staged_equals_direct_gathers_8x8(dtype, lanes):
    prob = synth.room_problem(7)
    _same(gpu_solve(prob, 10, dtype=dtype, lanes=lanes, staging=True), gpu_solve(prob, 10, dtype=dtype, lanes=lanes))


@pytest.mark.parametrize("patch,lanes", [(4, 8), (4, 16), (16, 32)])
def test_staged_equals_direct_gathers_other_patches(patch, lanes):
    prob = synth.room_problem(8, P=patch, F=3)
    for dtype in ("f32", "f16"):
        _same(gpu_solve(prob, 6, dtype=dtype, lanes=lanes, staging=True), gpu_solve(prob, 6, dtype=dtype, lanes=lanes))


def test_staged_edge_cases():
    """One frame (both boxes in flight hold the same frame), zero iterations (the final pass alone),
    block of 128 threads, and a run continued from an earlier solve."""
    prob = synth.room_problem(9, F=1)
    for iters in (0, 1, 3):
        _same(gpu_solve(prob, iters, staging=True), gpu_solve(prob, iters))
    prob = synth.room_problem(9, F=4)
    _same(gpu_solve(prob, 5, block=128, staging=True), gpu_solve(prob, 5, block=128))

    def steps(plan):
        plan.solve(2)
        plan.run(3)

    _same(gpu_solve(prob, 0, steps=steps, staging=True), gpu_solve(prob, 0, steps=steps))


def test_no_staging_timeouts():
    import paper_1910_01997_gb300 as sgn

    gpu_solve(synth.room_problem(0), 10, staging=True)
    assert sgn.sgn_staging_timeouts() == 0
