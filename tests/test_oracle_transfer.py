"""Pins of the oracle's reference-frame change (Sec. 2.5, Eq. 10) and depth-buffered surfel render
(Sec. 2.2, Eq. 3, Eq. 4) to closed forms, brute force and the scene's own ray caster (CPU only)."""
import numpy as np

import oracle
import synth


def _rot(axis, deg):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    t = np.radians(deg)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K


def _tile_surfels(prob):
    """Ground-truth free surfels at the tile centres of tiles that see one primitive."""
    TX = prob.W // prob.P
    s = np.flatnonzero(prob.tile_prim >= 0)
    u = np.stack([(s % TX) * prob.P + (prob.P - 1) / 2.0, (s // TX) * prob.P + (prob.P - 1) / 2.0], 1)
    return s, u, prob.gt_id[s], prob.gt_n[s]


def test_transfer_identity_and_round_trip():
    prob = synth.tiny_problem(0)
    s, u, idv, n = _tile_surfels(prob)
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    uo, io, no, valid = oracle.transfer_surfels(prob.cam, I, u, idv, n)
    assert valid.all()
    assert np.abs(uo - u).max() < 1e-9 and np.abs(io / idv - 1).max() < 1e-12 and np.abs(no - n).max() < 1e-15
    R = _rot([0.3, -1.0, 0.2], 7.0)
    t = np.array([0.12, -0.05, 0.3])
    T = np.hstack([R, t[:, None]])
    Ti = np.hstack([R.T, (-R.T @ t)[:, None]])
    u1, i1, n1, v1 = oracle.transfer_surfels(prob.cam, T, u, idv, n)
    u2, i2, n2, v2 = oracle.transfer_surfels(prob.cam, Ti, u1, i1, n1)
    assert v1.all() and v2.all()
    assert np.abs(u2 - u).max() < 1e-8 and np.abs(i2 / idv - 1).max() < 1e-11 and np.abs(n2 - n).max() < 1e-12


def test_transfer_lands_on_the_scene_surface():
    """A ground-truth surfel moved into frame f (Eq. 10) sits where the scene's ray caster, looking
    from camera f through the new pixel u1, hits the same primitive at depth 1 / id1; its normal is
    the primitive's normal in frame f coordinates."""
    prob = synth.tiny_problem(0)
    s, u, idv, n = _tile_surfels(prob)
    for f, cam_idx in enumerate(prob.frame_index):
        u1, i1, n1, valid = oracle.transfer_surfels(prob.cam, prob.poses[f], u, idv, n)
        inside = valid.astype(bool) & (u1[:, 0] > 0) & (u1[:, 0] < prob.W - 1) & (u1[:, 1] > 0) & (u1[:, 1] < prob.H - 1)
        assert inside.sum() > 0.8 * len(s)
        _, pid, dep = prob.scene.shade(cam_idx, u1[inside])
        hit = pid == prob.tile_prim[s][inside]
        assert hit.mean() > 0.95
        assert np.abs(i1[inside][hit] * dep[hit] - 1).max() < 1e-9
        R = prob.poses[f][:, :3]
        world_n = prob.scene.prims["n"][prob.tile_prim[s][inside][hit]]
        assert np.abs(np.abs(np.einsum("ij,ij->i", n1[inside][hit], world_n @ R.T)) - 1).max() < 1e-12


def test_render_fronto_parallel_disc_is_exact():
    """One fronto-parallel surfel: every pixel centre strictly inside radius r (brute-force lattice
    count) gets id_u = id_s, every other pixel nothing."""
    cam = (140.0, 140.0, 79.5, 59.5)
    for cx, cy, r in ((40.0, 30.0, 5.0), (40.3, 30.7, 4.5), (0.5, 0.5, 6.0), (158.2, 10.0, 3.2)):
        inv, sidx = oracle.render_surfels(cam, 160, 120, [[cx, cy]], [0.4], [[0.0, 0.0, -1.0]], [1], r)
        yy, xx = np.mgrid[0:120, 0:160]
        inside = np.hypot(xx - cx, yy - cy) < r
        assert np.array_equal(sidx == 0, inside)
        assert np.all(inv[inside] == 0.4) and np.all(inv[~inside] == 0.0)


def test_render_points_lie_on_their_surfel_plane():
    rng = np.random.default_rng(3)
    cam = (140.0, 140.0, 79.5, 59.5)
    n = rng.normal(size=(30, 3))
    n[:, 2] = -np.abs(n[:, 2]) - 1.0
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    u = rng.uniform([0, 0], [160, 120], (30, 2))
    idv = rng.uniform(0.2, 1.0, 30)
    inv, sidx = oracle.render_surfels(cam, 160, 120, u, idv, n, np.ones(30, np.uint8), 9.0)
    yy, xx = np.mgrid[0:120, 0:160]
    m = sidx >= 0
    s = sidx[m]
    r_u = np.stack([(xx[m] - cam[2]) / cam[0], (yy[m] - cam[3]) / cam[1], np.ones(m.sum())], 1)
    r_s = np.stack([(u[s, 0] - cam[2]) / cam[0], (u[s, 1] - cam[3]) / cam[1], np.ones(m.sum())], 1)
    lhs = np.einsum("ij,ij->i", r_u / inv[m][:, None], n[s])
    rhs = np.einsum("ij,ij->i", r_s / idv[s][:, None], n[s])
    assert np.abs(lhs / rhs - 1).max() < 1e-12


def test_render_depth_buffer_keeps_the_nearest_and_breaks_ties_low():
    cam = (140.0, 140.0, 79.5, 59.5)
    fp = [[0.0, 0.0, -1.0]] * 3
    # surfel 1 is nearer than surfel 0; surfel 2 ties with surfel 1 and has the higher index
    u = [[50.0, 50.0], [54.0, 50.0], [54.0, 50.0]]
    inv, sidx, second = oracle.render_surfels(cam, 160, 120, u, [0.3, 0.5, 0.5], fp, [1, 1, 1], 6.0, with_second=True)
    yy, xx = np.mgrid[0:120, 0:160]
    in0 = np.hypot(xx - 50, yy - 50) < 6
    in1 = np.hypot(xx - 54, yy - 50) < 6
    assert np.all(sidx[in1] == 1) and np.all(inv[in1] == 0.5)
    assert np.all(sidx[in0 & ~in1] == 0) and np.all(inv[in0 & ~in1] == 0.3)
    assert np.all(second[in1 & ~in0] == 0.5) and np.all(second[in1 & in0] == 0.5)
    assert np.all(second[in0 & ~in1] == 0.0)
    # invalid surfels and surfels facing away draw nothing
    inv, sidx = oracle.render_surfels(cam, 160, 120, u, [0.3, 0.5, 0.5], fp, [0, 0, 0], 6.0)
    assert (sidx < 0).all()
    # plane seen edge-on (it contains the surfel's ray, r_s . n = 0): Eq. 3 is undefined, nothing drawn
    inv, sidx = oracle.render_surfels(cam, 160, 120, [[79.5, 59.5]], [0.3], [[0.0, 1.0, 0.0]], [1], 6.0)
    assert (sidx < 0).all()


def test_transfer_then_render_matches_ray_casting():
    """Ground-truth surfels of the keyframe moved into frame f and rendered there: wherever the
    drawn surfel lies on the primitive the frame's ray caster sees at that pixel, the rendered inverse
    depth equals 1 / depth of the ray caster."""
    prob = synth.tiny_problem(1)
    s, u, idv, n = _tile_surfels(prob)
    for f, cam_idx in enumerate(prob.frame_index):
        u1, i1, n1, valid = oracle.transfer_surfels(prob.cam, prob.poses[f], u, idv, n)
        inv, sidx = oracle.render_surfels(prob.cam, prob.W, prob.H, u1, i1, n1, valid, prob.P / 2.0)
        _, pid, dep = prob.scene.render(cam_idx)
        m = sidx >= 0
        m[m] &= prob.tile_prim[s][sidx[m]] == pid[m]
        assert m.sum() > 0.5 * prob.W * prob.H
        assert np.abs(inv[m] * dep[m] - 1).max() < 1e-9
