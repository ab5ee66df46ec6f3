"""GPU (CUDA, through the C ABI) against the FP64 oracle on a full-size, well-conditioned workload:
the ring scene at 640x480 (two tilted textured planes seen from five cameras on a 12 cm ring, so
that the baselines span every direction and surfel normals are observable), 20 % of the tiles seeded
from their neighbours, 10 iterations (Sec. 2.3-2.4)."""
import json
import os

import numpy as np
import pytest

import synth
from helpers import compare, gpu_solve, oracle_solve, oracle_stable

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = json.load(open(os.path.join(HERE, "tolerances.json")))
WELL = TOL["well_posed"]
FRAC = WELL["min_stable_frac"]

# (patch, image noise sigma): 8x8 tiles on noise-free renders (normals converge to about 1 degree of
# the true planes), 16x16 tiles with the benchmark's sigma = 0.01 noise
RING_CASES = [(8, 0.0), (16, 0.01)]


def ring_problem_640(P, noise):
    return synth.make_problem(synth.ring_scene(0, 640, 480, 5), P, noise_sigma=noise, seed_frac=0.2, seed=0)


def _stats(prob, g, o, dtype, frac_key):
    tol = TOL["parity"][dtype]
    stable = oracle_stable(prob, 10, tol["depth_rel"], tol["normal_deg"], o, dtype=dtype)
    st = compare(prob, g, o, margin_px=WELL["margin_px"], stable=stable)
    print(f"ring {prob.W}x{prob.H} P{prob.P} sigma {prob.noise_sigma} {dtype} vs FP64 oracle",
          {k: v for k, v in st.items() if k not in ("rel", "ang", "mask")})
    return tol, st, FRAC[frac_key]


@pytest.mark.parametrize("P,noise", RING_CASES)
def test_ring_parity_f32(P, noise):
    """FP32 texels: depth within 1e-4 and normal within 0.01 deg of the FP64 oracle at the maximum over
    the compared surfels (at least 90 % of the usable ones), and the 99th percentile over every usable
    surfel within twice those bounds."""
    prob = ring_problem_640(P, noise)
    g, o = gpu_solve(prob, 10), oracle_solve(prob, 10)
    tol, st, min_frac = _stats(prob, g, o, "f32", "ring")
    assert st["n"] >= min_frac * st["n_usable"], (st["n"], st["n_usable"], st["excluded"])
    assert st["depth_max"] <= tol["depth_rel"] and st["ang_max"] <= tol["normal_deg"], (st["depth_max"], st["ang_max"])
    assert st["all_depth_p99"] <= 2 * tol["depth_rel"] and st["all_ang_p99"] <= 2 * tol["normal_deg"], \
        (st["all_depth_p99"], st["all_ang_p99"])
    assert (g["status"] != o["status"]).sum() <= max(5, 0.01 * prob.S)


@pytest.mark.parametrize("dtype", ["f16g", "bf16g"])
@pytest.mark.parametrize("P,noise", RING_CASES)
def test_ring_reduced_precision_gradients(P, noise, dtype):
    """Gradients stored in FP16/BF16 next to the FP32 intensity (8-byte texels, FP32 residuals and
    accumulation): within 1e-3 and 0.1 deg of the FP64 oracle run on the original frames, at the
    maximum over the oracle-stable surfels (at least 65 % of the usable ones) and, within twice
    that, at the 99th percentile over all usable surfels."""
    prob = ring_problem_640(P, noise)
    g, o = gpu_solve(prob, 10, dtype=dtype), oracle_solve(prob, 10)
    tol, st, min_frac = _stats(prob, g, o, dtype, "ring_reduced")
    assert st["n"] >= min_frac * st["n_usable"], (st["n"], st["n_usable"], st["excluded"])
    assert st["depth_max"] <= tol["depth_rel"] and st["ang_max"] <= tol["normal_deg"], (st["depth_max"], st["ang_max"])
    assert st["all_depth_p99"] <= 2 * tol["depth_rel"] and st["all_ang_p99"] <= 2 * tol["normal_deg"], \
        (st["all_depth_p99"], st["all_ang_p99"])


@pytest.mark.xfail(strict=True, reason="FP16/BF16 intensities move the photometric cost minimum itself: against the "
                                       "FP64 oracle the normals move by a median 0.37 deg (FP16) / 3.0 deg (BF16) on "
                                       "the 8x8 noise-free ring and 0.12 / 0.94 deg on the 16x16 noisy ring, so 0.1 deg "
                                       "holds on under half of the surfels (the stated reduced-precision bound is not met with "
                                       "reduced-precision images; the G formats meet it)")
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("P,noise", RING_CASES)
def test_ring_reduced_precision_images(P, noise, dtype):
    """Intensity and gradient both stored in FP16/BF16: the stated reduced-precision bound (1e-3,
    0.1 deg against the FP64 oracle on the original frames) on at least half of the usable surfels."""
    prob = ring_problem_640(P, noise)
    g, o = gpu_solve(prob, 10, dtype=dtype), oracle_solve(prob, 10)
    tol, st, min_frac = _stats(prob, g, o, dtype, "reduced_images")
    assert st["n"] >= min_frac * st["n_usable"], (st["n"], st["n_usable"], st["excluded"])
    assert st["depth_max"] <= tol["depth_rel"] and st["ang_max"] <= tol["normal_deg"], (st["depth_max"], st["ang_max"])
