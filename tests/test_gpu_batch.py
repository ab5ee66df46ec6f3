"""Batched persistent execution: many keyframes (uneven sizes, patches, frame counts, texel types)
in one graph-captured launch give the results of the plain per-keyframe launch."""
import numpy as np
import pytest

import synth
from helpers import gpu_solve, oracle_solve, oracle_solve_planes, stored_planes

pytestmark = pytest.mark.gpu


def _problems():
    return [
        ("f32", synth.tiny_problem(3, noise_sigma=0.01, seed_frac=0.2)),
        ("f32", synth.room_problem(4)),
        ("f16", synth.make_problem(synth.room_scene(5, 320, 240, 3), 16, noise_sigma=0.01, seed_frac=0.2, seed=5)),
        ("bf16", synth.make_problem(synth.room_scene(6, 320, 240, 7), 4, noise_sigma=0.01, seed_frac=0.2, seed=6)),
        ("f32", synth.make_problem(synth.room_scene(7, 157, 113, 2), 8, noise_sigma=0.01, seed_frac=0.2, seed=7)),
    ]


def _plan(prob, dtype, **opts):
    import paper_1910_01997_gb300 as sgn

    plan = sgn.Plan(prob.W, prob.H, prob.P, prob.F, dtype, **opts)
    plan.set_intrinsics(*prob.cam)
    plan.set_keyframe(prob.keyframe)
    plan.set_frames(prob.frames, prob.poses)
    plan.init_surfels(prob.id0, prob.n0, prob.state)
    return plan


@pytest.mark.parametrize("variant,chunk", [(0, 64), (1, 64), (0, 7), (2, 64), (2, 7)])
def test_batch_matches_plain(variant, chunk):
    """Each keyframe solved in the mix equals the oracle (and so the plain launch) within the
    parity tolerances, on the surfels where the comparison is defined (see test_gpu_parity)."""
    import paper_1910_01997_gb300 as sgn
    from test_gpu_parity import _check

    probs = _problems()
    plans = [_plan(p, dt) for dt, p in probs]
    batch = sgn.Batch(len(plans))
    for pl in plans:
        batch.add(pl)
    batch.set_schedule(variant, chunk)
    launches = sgn.sgn_launch_count()
    batch.run(10)
    batch.sync()
    assert sgn.sgn_launch_count() == launches + 1  # one persistent launch for all keyframes
    for (dt, prob), pl in zip(probs, plans):
        got = pl.read_surfels()
        ref = gpu_solve(prob, 10, dtype=dt)
        assert np.mean(got["status"] != ref["status"]) < 0.02
        inv, sidx = pl.read_depth_map()
        assert np.mean((sidx >= 0) != (ref["sidx"] >= 0)) < 0.02
        if dt == "f32":
            frac = "room" if prob.W >= 640 else "noisy_small"
            _check(prob, got, oracle_solve(prob, 10), "f32", f"batch {prob.W}x{prob.H} P{prob.P}", 10, frac=frac)
        else:
            planes = stored_planes(prob.frames, dt)
            _check(prob, got, oracle_solve_planes(prob, planes, 10), "f32", f"batch {dt} {prob.W}x{prob.H} P{prob.P}",
                   10, frac="noisy_small" if prob.P == 4 else "room", planes=planes)


def test_batch_with_adaptive_and_circular_plans():
    """Plans with the Marquardt schedule (Sec. 2.4) and with circular surfels (Sec. 2.1, Eq. 4) join a
    batch beside fixed-damping square surfels: one persistent launch per solver kind, and each plan's
    surfels equal the oracle within the parity tolerances (and its depth map is the render of its
    discs)."""
    import paper_1910_01997_gb300 as sgn
    from test_gpu_parity import _check

    cases = [
        ("f32", dict(), synth.room_problem(60, W=320, H=240, F=4, P=8)),
        ("f32", dict(lm_adaptive=True), synth.room_problem(61, W=320, H=240, F=4, P=8)),
        ("f16g", dict(lm_adaptive=True), synth.room_problem(62, W=640, H=480, F=3, P=8)),
        ("f32", dict(surfel_radius=5.0), synth.room_problem(63, W=320, H=240, F=4, P=8)),
        ("f16g", dict(surfel_radius=10.0), synth.room_problem(64, W=320, H=240, F=3, P=16)),
    ]
    plans = [_plan(p, dt, **o) for dt, o, p in cases]
    batch = sgn.Batch(len(plans))
    for pl in plans:
        batch.add(pl)
    launches = sgn.sgn_launch_count()
    batch.run(10)
    batch.sync()
    # fixed, adaptive and circular launches, plus a render (memset-free: 2 kernels) per circular plan
    assert sgn.sgn_launch_count() == launches + 3 + 2 * 2
    for (dt, o, prob), pl in zip(cases, plans):
        got = pl.read_surfels()
        got["inv_depth"], got["sidx"] = pl.read_depth_map()
        plain = gpu_solve(prob, 10, dtype=dt, **o)
        assert np.mean(got["status"] != plain["status"]) < 0.02
        if "surfel_radius" in o:
            assert np.array_equal(got["sidx"] >= 0, plain["sidx"] >= 0) or np.mean((got["sidx"] >= 0) != (plain["sidx"] >= 0)) < 0.01
        oo = dict(radius=o["surfel_radius"]) if "surfel_radius" in o else dict(o)
        if dt == "f32":
            ref = oracle_solve(prob, 10, **oo)
            planes = None
        else:
            planes = stored_planes(prob.frames, dt)
            ref = oracle_solve_planes(prob, planes, 10, **oo)
        also = ref["decision_margin"] > 1e-4 if o.get("lm_adaptive") else None
        # 320x240 keyframes at sigma 0.01: the small noisy workloads' fraction
        frac = "noisy_small"
        _check(prob, got, ref, "f32", f"batch {dt} {o} {prob.W}x{prob.H} P{prob.P}", 10, frac=frac, planes=planes,
               also_stable=also, **oo)


def test_batch_graph_replay_is_deterministic():
    import paper_1910_01997_gb300 as sgn

    probs = _problems()[:3]
    plans = [_plan(p, dt) for dt, p in probs]
    batch = sgn.Batch(len(plans))
    for pl in plans:
        batch.add(pl)
    batch.run(6)
    first = [pl.read_surfels() for pl in plans]
    for _ in range(3):  # replays of the captured graph
        batch.run(6)
    batch.sync()
    for a, pl in zip(first, plans):
        b = pl.read_surfels()
        for k in ("id", "n", "cost", "nres", "status"):
            assert np.array_equal(a[k], b[k])


def test_autotuners_choose_valid_schedules_and_use_the_cache(tmp_path):
    import paper_1910_01997_gb300 as sgn

    cache = tmp_path / "tune.txt"
    probs = _problems()[:3]
    plans = [_plan(p, dt) for dt, p in probs]
    lanes, block = plans[1].autotune(4, cache)
    assert lanes in (8, 16, 32) and block in (128, 256)
    assert cache.read_text().count("plan|") == 1
    assert plans[1].autotune(4, cache) == (lanes, block)  # cache hit
    assert cache.read_text().count("plan|") == 1
    batch = sgn.Batch(len(plans))
    for pl in plans:
        batch.add(pl)
    variant, chunk = batch.autotune(4, cache)
    assert variant in (0, 1, 2) and chunk in (8, 16, 32, 64, 128, 256)
    assert batch.autotune(4, cache) == (variant, chunk)
    assert cache.read_text().count("batch|") == 1
    batch.run(4)
    batch.sync()
