"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks one step of the oracle against what the paper and the mathematics fix:
closed forms, exactness properties, finite differences of an independently pinned
function, library routines (numpy/scipy) or brute force.  A plausible slip anywhere in the
oracle (dropped term, wrong sign, wrong index, transposed operand) fails at least one of
them.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = json.load(open(os.path.join(HERE, "tolerances.json")))
PRM = oracle.params()
RNG = np.random.default_rng(1234)


def _rand_unit(rng, facing=None):
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    if facing is not None and v @ facing > 0:
        v = -v
    return v


def _tile_ray(p, s):
    TX = p.W // p.P
    tx, ty = s % TX, s // TX
    return oracle.ray(p.cam, tx * p.P + (p.P - 1) / 2, ty * p.P + (p.P - 1) / 2)


# ------------------------------------------------------------------------------------------ image terms


def test_gradients_are_exact_on_linear_images():
    """Central differences reproduce the slope of a linear image; borders are zero."""
    H, W = 9, 13
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = 0.3 + 0.02 * x - 0.05 * y
    gx, gy = oracle.gradients(img)
    assert np.allclose(gx[:, 1:-1], 0.02, atol=1e-15) and np.allclose(gy[1:-1, :], -0.05, atol=1e-15)
    assert np.all(gx[:, [0, -1]] == 0) and np.all(gy[[0, -1], :] == 0)
    q = RNG.normal(size=(H, W))
    gx, gy = oracle.gradients(q)
    assert np.allclose(gx[:, 1:-1], (q[:, 2:] - q[:, :-2]) / 2)  # definition on random data
    assert np.allclose(gy[1:-1, :], (q[2:, :] - q[:-2, :]) / 2)


def test_bilinear_reproduces_bilinear_functions():
    H, W = 7, 8
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    f = lambda X, Y: 0.1 + 0.3 * X - 0.2 * Y + 0.05 * X * Y
    img = f(x, y)
    for _ in range(50):
        X, Y = RNG.uniform(0, W - 1.0001), RNG.uniform(0, H - 1.0001)
        assert abs(oracle.bilinear(img, X, Y) - f(X, Y)) < 1e-13
    assert oracle.bilinear(img, 3.0, 4.0) == img[4, 3]
    # a tap-weight slip would break symmetry: sample a delta image
    d = np.zeros((4, 4))
    d[1, 2] = 1.0
    assert abs(oracle.bilinear(d, 1.25, 1.5) - 0.25 * 0.5) < 1e-15   # x weight 0.25 toward column 2
    assert abs(oracle.bilinear(d, 2.0, 0.75) - 0.75) < 1e-15


def test_huber_norm_and_weight():
    k = 0.05
    for r in (-0.2, -0.05, -0.01, 0.0, 0.03, 0.05, 0.5):
        rho, w = oracle.huber(r, k)
        want = 0.5 * r * r if abs(r) <= k else k * abs(r) - 0.5 * k * k
        assert abs(rho - want) < 1e-15
        h = 1e-7
        if abs(abs(r) - k) > 1e-6:  # IRLS weight: rho'(r) = w r
            d = (oracle.huber(r + h, k)[0] - oracle.huber(r - h, k)[0]) / (2 * h)
            assert abs(d - w * r) < 1e-8
    a, b = oracle.huber(k - 1e-12, k)[0], oracle.huber(k + 1e-12, k)[0]
    assert abs(a - b) < 1e-12  # continuous at the threshold


# ------------------------------------------------------------------------------------------ geometry


def test_ray_is_inverse_intrinsics():
    cam = synth.intrinsics(640, 480)
    K = np.array([[cam[0], 0, cam[2]], [0, cam[1], cam[3]], [0, 0, 1.0]])
    for _ in range(10):
        u = RNG.uniform(0, 640, 2)
        assert np.allclose(oracle.ray(cam, *u), np.linalg.solve(K, [u[0], u[1], 1.0]), rtol=1e-14, atol=1e-15)


def test_inverse_depth_lies_on_surfel_plane():
    """Eq. 3 is the ray-plane intersection: n . (r_u / id_u - r_s / id_s) = 0."""
    for _ in range(100):
        r_s = np.r_[RNG.uniform(-0.5, 0.5, 2), 1.0]
        r_u = r_s + np.r_[RNG.uniform(-0.05, 0.05, 2), 0.0]
        n = _rand_unit(RNG, facing=r_s)
        ids = RNG.uniform(0.2, 1.0)
        idu = oracle.inv_depth(r_u, r_s, ids, n)
        assert abs(n @ (r_u / idu - r_s / ids)) < 1e-12
    # fronto-parallel plane: every ray has the same inverse depth (z = 1 rays)
    assert abs(oracle.inv_depth([0.3, -0.2, 1], [0.01, 0.02, 1], 0.5, [0, 0, -1]) - 0.5) < 1e-15


def test_inverse_depth_derivative_matches_fd_and_invariants():
    h = 1e-7
    for _ in range(30):
        r_s = np.r_[RNG.uniform(-0.5, 0.5, 2), 1.0]
        r_u = r_s + np.r_[RNG.uniform(-0.05, 0.05, 2), 0.0]
        n = _rand_unit(RNG, facing=r_s)
        ids = RNG.uniform(0.2, 1.0)
        dn, did = oracle.inv_depth_derivative(r_u, r_s, ids, n)
        fd = np.array([(oracle.inv_depth(r_u, r_s, ids, n + h * e) - oracle.inv_depth(r_u, r_s, ids, n - h * e))
                       / (2 * h) for e in np.eye(3)])
        assert np.allclose(dn, fd, rtol=1e-6, atol=1e-9)
        fdi = (oracle.inv_depth(r_u, r_s, ids + h, n) - oracle.inv_depth(r_u, r_s, ids - h, n)) / (2 * h)
        assert abs(did - fdi) < 1e-7 * max(1, abs(did))
        assert abs(did - oracle.inv_depth(r_u, r_s, ids, n) / ids) < 1e-12   # d id_u / d id_s = id_u / id_s
        assert abs(dn @ n) < 1e-12 * max(1.0, np.linalg.norm(dn))           # scale invariance in n
        dn0, _ = oracle.inv_depth_derivative(r_s, r_s, ids, n)
        assert np.linalg.norm(dn0) < 1e-14                                    # centre ray does not move


def test_warp_equals_plane_homography_and_fd():
    """u_p of Eq. 6 equals the plane-induced homography K (R + c t n^T) K^-1 u, c = id_s / (r_s . n)."""
    cam = synth.intrinsics(640, 480)
    K = np.array([[cam[0], 0, cam[2]], [0, cam[1], cam[3]], [0, 0, 1.0]])
    for _ in range(30):
        R = synth.rot_axis_angle(RNG.normal(size=3), np.deg2rad(RNG.uniform(0, 5)))
        t = RNG.uniform(-0.1, 0.1, 3)
        T = synth.pose(R, t)
        us = RNG.uniform(50, 590), RNG.uniform(50, 430)
        r_s = oracle.ray(cam, *us)
        n = _rand_unit(RNG, facing=r_s)
        if n @ r_s > -0.3:
            continue
        ids = RNG.uniform(0.25, 1.0)
        u = np.array([us[0] + RNG.uniform(-8, 8), us[1] + RNG.uniform(-8, 8), 1.0])
        r_u = oracle.ray(cam, u[0], u[1])
        idu = oracle.inv_depth(r_u, r_s, ids, n)
        up, du, qz = oracle.warp(cam, T, r_u, idu)
        c = ids / (r_s @ n)
        Hm = K @ (R + c * np.outer(t, n)) @ np.linalg.inv(K)
        hh = Hm @ u
        assert qz > 0
        assert np.allclose(up, hh[:2] / hh[2], rtol=0, atol=1e-9)
        h = 1e-7
        fd = (oracle.warp(cam, T, r_u, idu + h)[0] - oracle.warp(cam, T, r_u, idu - h)[0]) / (2 * h)
        assert np.allclose(du, fd, rtol=1e-6, atol=1e-6)
    # closed form: fronto-parallel plane, pure x translation -> u_p = u + (fx t_x id, 0)
    T = synth.pose(np.eye(3), [0.07, 0, 0])
    r_u = oracle.ray(cam, 100.0, 200.0)
    up, du, _ = oracle.warp(cam, T, r_u, 0.4)
    assert np.allclose(up, [100.0 + cam[0] * 0.07 * 0.4, 200.0], atol=1e-10)
    assert np.allclose(du, [cam[0] * 0.07, 0.0], atol=1e-9)


def test_tangent_basis_is_orthonormal():
    for n in [_rand_unit(RNG) for _ in range(200)] + [np.array([0, 0, -1.0]), np.array([0, 0, 1.0]),
                                                       np.array([1e-9, 0, -1.0]) / np.linalg.norm([1e-9, 0, -1.0])]:
        t1, t2 = oracle.tangent_basis(n)
        B = np.stack([t1, t2, n])
        assert np.allclose(B @ B.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(t1, t2), n, atol=1e-12)


def test_cholesky_solve_matches_numpy():
    for _ in range(50):
        A = RNG.normal(size=(3, 3))
        A = A @ A.T + 0.1 * np.eye(3)
        b = RNG.normal(size=3)
        x = oracle.cholesky_solve3([A[0, 0], A[0, 1], A[0, 2], A[1, 1], A[1, 2], A[2, 2]], b)
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    assert oracle.cholesky_solve3([1, 2, 0, 1, 0, 1], [1, 1, 1]) is None   # indefinite
    assert oracle.cholesky_solve3([0, 0, 0, 0, 0, 0], [1, 1, 1]) is None


def test_damped_step_definition_and_rotation_invariance():
    for _ in range(20):
        J = RNG.normal(size=(40, 3)) * np.array([1e-2, 2e-2, 1.0])
        Hm = J.T @ J
        g = J.T @ RNG.normal(size=40)
        H6 = [Hm[0, 0], Hm[0, 1], Hm[0, 2], Hm[1, 1], Hm[1, 2], Hm[2, 2]]
        lam = 1e-2
        m = 0.5 * (Hm[0, 0] + Hm[1, 1])
        want = np.linalg.solve(Hm + lam * np.diag([m, m, Hm[2, 2]]), -g)
        d = oracle.damped_step(H6, g, lam)
        assert np.allclose(d, want, rtol=1e-10)
        # rotating the tangent basis by phi rotates the step by phi: the normal update is unchanged
        phi = RNG.uniform(0, 2 * np.pi)
        Q = np.eye(3)
        Q[:2, :2] = [[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]]
        Hr, gr = Q.T @ Hm @ Q, Q.T @ g
        dr = oracle.damped_step([Hr[0, 0], Hr[0, 1], Hr[0, 2], Hr[1, 1], Hr[1, 2], Hr[2, 2]], gr, lam)
        assert np.allclose(Q @ dr, d, rtol=1e-9, atol=1e-15)
    # depth-only: scalar step on id_s
    d = oracle.damped_step([0, 0, 0, 0, 0, 4.0], [0, 0, 2.0], 0.5, optimize_normal=False)
    assert np.allclose(d, [0, 0, -2.0 / (1.5 * 4.0)])


def test_apply_step_moves_in_tangent_plane():
    n = _rand_unit(RNG)
    t1, t2 = oracle.tangent_basis(n)
    n2, id2 = oracle.apply_step(n, 0.5, [0.1, -0.2, 0.01])
    v = n + 0.1 * t1 - 0.2 * t2
    assert np.allclose(n2, v / np.linalg.norm(v), atol=1e-15) and abs(id2 - 0.51) < 1e-15


# ------------------------------------------------------------------------------------------ analytic scene


def _single_plane_tiles(p, limit=40):
    return [s for s in range(p.S) if p.tile_prim[s] >= 0][:: max(1, p.S // limit)][:limit]


def test_residual_is_zero_at_ground_truth_in_analytic_mode():
    """At the true plane, Eq. 6 maps every tile pixel onto the same scene point: the
    continuous (noise-free, unsampled) images agree exactly where the point is visible."""
    for p in (synth.tiny_problem(0), synth.ring_problem(0, P=16)):
        sc = p.scene
        checked = 0
        for s in _single_plane_tiles(p):
            r_s = _tile_ray(p, s)
            TX = p.W // p.P
            tx, ty = s % TX, s // TX
            for py in range(0, p.P, 3):
                for px in range(0, p.P, 3):
                    u = (tx * p.P + px, ty * p.P + py)
                    r_u = oracle.ray(p.cam, *u)
                    idu = oracle.inv_depth(r_u, r_s, p.gt_id[s], p.gt_n[s])
                    Ikf, pid_kf, _ = sc.shade(0, np.array([u], float))
                    for f, T in zip(p.frame_index, p.poses):
                        up, _, qz = oracle.warp(p.cam, T.reshape(-1), r_u, idu)
                        If, pid, _ = sc.shade(f, up[None])
                        if pid[0] != p.tile_prim[s] or pid_kf[0] != p.tile_prim[s]:
                            continue  # occluded in the frame
                        assert abs(If[0] - Ikf[0]) < 1e-9, (s, u, f)
                        checked += 1
        assert checked > 100


def test_jacobian_chain_matches_finite_differences_in_analytic_mode():
    """Full chain of Eqs. 7-9 (d I/d u_p . d u_p/d id_u . d id_u/d theta) against central
    differences of the analytic residual in theta = (step along t1, step along t2, id_s)."""
    p = synth.ring_problem(0, P=16)
    sc = p.scene
    worst = 0.0
    for s in _single_plane_tiles(p, 12):
        r_s = _tile_ray(p, s)
        n0, id0 = p.n0[s], p.id0[s]
        t1, t2 = oracle.tangent_basis(n0)
        TX = p.W // p.P
        u = ((s % TX) * p.P + 2, (s // TX) * p.P + 11)
        r_u = oracle.ray(p.cam, *u)
        Ikf = sc.shade(0, np.array([u], float))[0][0]

        def residual(theta, f):
            n, ids = oracle.apply_step(n0, id0, theta)
            idu = oracle.inv_depth(r_u, r_s, ids, n)
            up, _, _ = oracle.warp(p.cam, p.poses[f].reshape(-1), r_u, idu)
            return sc.shade(p.frame_index[f], up[None])[0][0] - Ikf

        for f in range(p.F):
            idu = oracle.inv_depth(r_u, r_s, id0, n0)
            up, du, _ = oracle.warp(p.cam, p.poses[f].reshape(-1), r_u, idu)
            hp = 1e-5
            ga = np.array([(sc.shade(p.frame_index[f], (up + hp * e)[None])[0][0] -
                            sc.shade(p.frame_index[f], (up - hp * e)[None])[0][0]) / (2 * hp) for e in np.eye(2)])
            dn, did = oracle.inv_depth_derivative(r_u, r_s, id0, n0)
            J = (ga @ du) * np.array([dn @ t1, dn @ t2, did])
            h = 1e-6
            fd = np.array([(residual(h * e, f) - residual(-h * e, f)) / (2 * h) for e in np.eye(3)])
            err = np.linalg.norm(J - fd) / np.linalg.norm(fd)
            worst = max(worst, err)
    assert worst < 1e-6, worst


# ------------------------------------------------------------------------------------------ normal equations


def _linear_problem(F=2, keyframe=None, T_list=None, P=8, W=48, H=40):
    """Frames that are exactly linear images (exact in float32), so that the interpolated
    central-difference gradient is the exact derivative of the sampled image."""
    cam = synth.intrinsics(W, H)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    coefs = [(0.25, 2.0 ** -7, 2.0 ** -8), (0.5, -2.0 ** -8, 2.0 ** -7), (0.375, 2.0 ** -7, 2.0 ** -7)]
    frames = np.stack([a + b * x + c * y for a, b, c in coefs[:F]]).astype(np.float32)
    if T_list is None:
        T_list = [synth.pose(synth.rot_axis_angle([0.3, 1, 0.2], np.deg2rad(1.0)), [0.06, 0.01, 0.02]),
                  synth.pose(synth.rot_axis_angle([1, -0.2, 0.1], np.deg2rad(-0.8)), [-0.02, 0.05, -0.01]),
                  synth.pose(np.eye(3), [0.03, -0.03, 0.0])][:F]
    if keyframe is None:
        keyframe = (0.4 + 0.1 * np.sin(x / 3.0) * np.cos(y / 4.0)).astype(np.float32)
    return cam, oracle.Problem(W, H, P, cam, keyframe, frames, np.stack(T_list)), frames, T_list


def _theta_fd(ob, prm, s, id0, n0, h, fn):
    out = []
    for e in np.eye(3):
        n_p, i_p = oracle.apply_step(n0, id0, h * e)
        n_m, i_m = oracle.apply_step(n0, id0, -h * e)
        out.append((fn(ob.eval_surfel(prm, s, i_p, n_p)) - fn(ob.eval_surfel(prm, s, i_m, n_m))) / (2 * h))
    return np.array(out)


def test_normal_equation_gradient_is_cost_gradient_on_linear_images():
    """g = sum w J r equals the gradient of the Huber cost of Eq. 5 when image gradients are exact."""
    cam, ob, _, _ = _linear_problem()
    for k in (1e9, 0.02):  # quadratic and Huber regimes
        prm = oracle.params(huber_k=k)
        for s in (7, 14, 22):
            r_s = oracle.ray(cam, (s % 6) * 8 + 3.5, (s // 6) * 8 + 3.5)
            n0 = _rand_unit(RNG, facing=r_s)
            n0 = n0 if n0 @ r_s < -0.6 else np.array([0.1, -0.05, -1]) / np.linalg.norm([0.1, -0.05, -1])
            e = ob.eval_surfel(prm, s, 0.5, n0)
            assert e["cnt"] > 0 and e["margin"] > 1e-3
            fd = _theta_fd(ob, prm, s, 0.5, n0, 1e-6, lambda q: q["E"])
            assert np.allclose(e["g"], fd, rtol=1e-5, atol=1e-9 * np.abs(e["g"]).max()), (k, s, e["g"], fd)


def test_normal_matrix_is_cost_hessian_at_zero_residual():
    """At parameters where every residual vanishes, sum J J^T is the exact Hessian of the cost."""
    W, H, P = 48, 40, 8
    cam = synth.intrinsics(W, H)
    K = np.array([[cam[0], 0, cam[2]], [0, cam[1], cam[3]], [0, 0, 1.0]])
    T = synth.pose(synth.rot_axis_angle([0.3, 1, 0.2], np.deg2rad(1.0)), [0.06, 0.01, 0.02])
    s = 14
    r_s = oracle.ray(cam, (s % 6) * 8 + 3.5, (s // 6) * 8 + 3.5)
    n_star = np.array([0.2, -0.1, -1.0]) / np.linalg.norm([0.2, -0.1, -1.0])
    id_star = 0.5
    # keyframe made consistent with the linear frame through the plane homography (numpy)
    c = id_star / (r_s @ n_star)
    Hm = K @ (T[:, :3] + c * np.outer(T[:, 3], n_star)) @ np.linalg.inv(K)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    hh = np.einsum("ij,jhw->ihw", Hm, np.stack([x, y, np.ones_like(x)]))
    xp, yp = hh[0] / hh[2], hh[1] / hh[2]
    a, b, cc = 0.25, 2.0 ** -7, 2.0 ** -8
    kf = (a + b * xp + cc * yp).astype(np.float64)
    _, ob, _, _ = _linear_problem(F=1, keyframe=kf.astype(np.float32), T_list=[T])
    prm = oracle.params(huber_k=1e9)
    e = ob.eval_surfel(prm, s, id_star, n_star)
    assert e["cnt"] == P * P
    h = 2e-4
    Hfd = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            vals = []
            for si, sj in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
                d = np.zeros(3)
                d[i] += si * h
                d[j] += sj * h
                n2, i2 = oracle.apply_step(n_star, id_star, d)
                vals.append(ob.eval_surfel(prm, s, i2, n2)["E"])
            Hfd[i, j] = (vals[0] - vals[1] - vals[2] + vals[3]) / (4 * h * h)
    Hm3 = oracle.sym3(e["H"])
    scale = np.sqrt(np.outer(np.diag(Hm3), np.diag(Hm3)))
    assert np.all(np.abs(Hm3 - Hfd) <= 2e-4 * scale), (Hm3, Hfd)


def test_tangent_step_equals_four_dof_min_norm_step():
    """The 3-parameter tangent solve equals the min-norm solve over (n in R^3, id_s)
    (the 4x4 J^T J is singular along (n, 0)), mapped back through the tangent basis."""
    p = synth.tiny_problem(0)
    ob = oracle.Problem.from_synth(p)
    for s in _single_plane_tiles(p, 10):
        e = ob.eval_surfel(PRM, s, p.id0[s], p.n0[s])
        H4 = oracle.sym4(e["H4"])
        assert abs(np.linalg.eigvalsh(H4)[0]) < 1e-10 * np.abs(H4).max()
        d4 = -np.linalg.pinv(H4, rcond=1e-14) @ e["g4"]
        d3 = oracle.damped_step(e["H"], e["g"], 0.0)
        t1, t2 = oracle.tangent_basis(p.n0[s])
        mapped = np.r_[d3[0] * t1 + d3[1] * t2, d3[2]]
        assert np.allclose(mapped, d4, rtol=1e-6, atol=1e-9 * np.abs(d4).max())


# ------------------------------------------------------------------------------------------ whole method


def test_seeding_is_exact_on_a_single_plane():
    """Sec. 2.3: where the surface is one plane, neighbour seeding returns that plane."""
    prims = synth.ring_scene(0).prims[:1].copy()
    sc = synth.Scene(prims, 160, 120, synth.ring_scene(0).poses[:2], "one-plane")
    p = synth.make_problem(sc, 8, seed_frac=0.3, depth_perturb=0.0, normal_perturb_deg=0.0, seed=3)
    ob = oracle.Problem.from_synth(p)
    ids, ns, st = ob.seed(p.id0, p.n0, p.state)
    seeded = (st & oracle.SEEDED_FLAG) != 0
    assert seeded.sum() > 20
    assert np.allclose(ids[seeded], p.gt_id[seeded], rtol=1e-12)
    assert np.allclose(ns[seeded], p.gt_n[seeded], atol=1e-12)
    # valid tiles pass through unchanged; TO_SEED tiles without VALID neighbours are UNSEEDED
    v = p.state == synth.VALID
    assert np.all(ids[v] == p.id0[v]) and np.all(st[v] == oracle.OK)
    state = np.full(p.S, synth.TO_SEED, np.uint8)
    _, _, st2 = ob.seed(p.id0, p.n0, state)
    assert np.all(st2 == oracle.UNSEEDED)


def test_seeding_turns_neighbour_normals_to_face_the_camera():
    prims = synth.ring_scene(0).prims[:1].copy()
    sc = synth.Scene(prims, 64, 64, synth.ring_scene(0).poses[:2], "one-plane")
    p = synth.make_problem(sc, 8, depth_perturb=0.0, normal_perturb_deg=0.0, seed=1)
    ob = oracle.Problem.from_synth(p)
    state = p.state.copy()
    state[27] = synth.TO_SEED
    n0 = p.n0.copy()
    n0[[18, 20, 34, 36]] *= -1  # flipped representatives of the same planes
    ids, ns, st = ob.seed(p.id0, n0, state)
    assert st[27] == oracle.OK | oracle.SEEDED_FLAG
    assert np.allclose(ns[27], p.gt_n[27], atol=1e-12) and abs(ids[27] / p.gt_id[27] - 1) < 1e-12


def test_depth_map_matches_ray_casting_at_ground_truth():
    """Sec. 2.2 / Eq. 3 per pixel, against the renderer's own ray-plane depths."""
    p = synth.ring_problem(0, P=16)
    ob = oracle.Problem.from_synth(p)
    status = np.where(p.tile_prim >= 0, oracle.OK, oracle.EMPTY).astype(np.uint8)
    inv, sidx = ob.depth_map(p.gt_id, p.gt_n, status)
    _, pid, depth = p.scene.render(0)
    TX = p.W // p.P
    for s in np.where(p.tile_prim >= 0)[0]:
        tx, ty = s % TX, s // TX
        sl = np.s_[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16]
        assert np.all(sidx[sl] == s)
        assert np.allclose(inv[sl], 1.0 / depth[sl], rtol=1e-12)
    assert np.all(sidx[np.isin(sidx, np.where(p.tile_prim < 0)[0])] == -1)


def test_no_motion_gives_zero_jacobian():
    """R = I, t = 0: u_p = u whatever the plane, so every Jacobian row vanishes (closed form)."""
    p = synth.tiny_problem(0)
    poses = np.stack([synth.pose(np.eye(3), [0, 0, 0])] * 2)
    ob = oracle.Problem(p.W, p.H, p.P, p.cam, p.keyframe, p.frames, poses)
    ref = oracle.Problem.from_synth(p)
    for s in _single_plane_tiles(p, 20):
        e = ob.eval_surfel(PRM, s, p.id0[s], p.n0[s])
        e_ref = ref.eval_surfel(PRM, s, p.id0[s], p.n0[s])
        assert e["cnt"] > 0
        assert np.abs(e["H"]).max() < 1e-20 * np.abs(e_ref["H"]).max()
        assert np.abs(e["g"]).max() < 1e-9 * max(np.abs(e_ref["g"]).max(), 1e-12)


def test_min_residuals_gives_underdetermined():
    p = synth.tiny_problem(0)
    ob = oracle.Problem.from_synth(p)
    out = ob.gauss_newton(oracle.params(min_residuals=33), 3, p.id0, p.n0, np.zeros(p.S, np.uint8))
    assert np.all(out["status"] == oracle.UNDERDETERMINED) and np.all(out["id"] == p.id0)
    st = np.zeros(p.S, np.uint8)
    st[:5] = oracle.EMPTY
    st[5:9] = oracle.UNSEEDED
    out = ob.gauss_newton(PRM, 3, p.id0, p.n0, st)
    assert np.all(out["status"][:5] == oracle.EMPTY) and np.all(out["status"][5:9] == oracle.UNSEEDED)
    assert np.all(out["nres"][:9] == 0)


def _consistent_linear_problem(id_star, n_star, s):
    """One linear frame and a keyframe made consistent with it through the plane (id_star,
    n_star) of tile s (plane homography in numpy)."""
    W, H = 48, 40
    cam = synth.intrinsics(W, H)
    K = np.array([[cam[0], 0, cam[2]], [0, cam[1], cam[3]], [0, 0, 1.0]])
    T = synth.pose(synth.rot_axis_angle([0.3, 1, 0.2], np.deg2rad(1.0)), [0.06, 0.01, 0.02])
    r_s = oracle.ray(cam, (s % 6) * 8 + 3.5, (s // 6) * 8 + 3.5)
    c = id_star / (r_s @ n_star)
    Hm = K @ (T[:, :3] + c * np.outer(T[:, 3], n_star)) @ np.linalg.inv(K)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    hh = np.einsum("ij,jhw->ihw", Hm, np.stack([x, y, np.ones_like(x)]))
    kf = 0.25 + 2.0 ** -7 * hh[0] / hh[2] + 2.0 ** -8 * hh[1] / hh[2]
    return _linear_problem(F=1, keyframe=kf.astype(np.float32), T_list=[T])


def test_depth_only_keeps_normals_and_finds_the_1d_minimum():
    """Depth-only ablation (Sec. 4.4): d id_u / d n := 0 leaves n untouched; on exact-gradient
    images the fixed point is the minimiser of the cost along id_s (scalar search)."""
    from scipy.optimize import minimize_scalar

    s = 14
    n_star = np.array([0.2, -0.1, -1.0]) / np.linalg.norm([0.2, -0.1, -1.0])
    cam, ob, _, _ = _consistent_linear_problem(0.5, n_star, s)
    r_s = oracle.ray(cam, (s % 6) * 8 + 3.5, (s // 6) * 8 + 3.5)
    for k, tilt in ((1e9, 0.0), (0.02, 4.0), (1e9, 6.0)):
        prm = oracle.params(huber_k=k, optimize_normal=False)
        axis = np.cross(n_star, [1.0, 0, 0])
        n_fix = synth.rot_axis_angle(axis, np.deg2rad(tilt)) @ n_star
        n0 = np.tile(n_fix, (ob.S, 1))
        id0 = np.full(ob.S, 0.46)
        out = ob.gauss_newton(prm, 30, id0, n0, np.zeros(ob.S, np.uint8))
        assert np.all(out["n"] == n0)
        assert out["status"][s] == oracle.OK
        res = minimize_scalar(lambda v: ob.eval_surfel(prm, s, v, n_fix)["E"], bounds=(0.4, 0.6),
                              method="bounded", options={"xatol": 1e-12})
        assert abs(out["id"][s] / res.x - 1) < 1e-6, (tilt, out["id"][s], res.x)
        if tilt == 0.0:
            assert abs(out["id"][s] / 0.5 - 1) < 1e-6   # exact plane: zero residual at id_star


def test_noise_free_views_converge_to_ground_truth():
    """Noise-free rendered views, init +-10% inverse depth / up to 10 deg normal: single-plane
    tiles converge to the true plane within the sampling bias (bounds in tolerances.json)."""
    t = TOL["convergence_ring"]
    for seed in (0, 1):
        p = synth.ring_problem(seed, P=16)
        ob = oracle.Problem.from_synth(p)
        out = ob.solve(PRM, t["iterations"], p.id0, p.n0, p.state)
        ok = ((out["status"] & 0x3F) == oracle.OK) & (p.tile_prim >= 0)
        assert ok.sum() > 0.85 * (p.tile_prim >= 0).sum()
        rel = np.abs(out["id"][ok] / p.gt_id[ok] - 1)
        ang = np.rad2deg(np.arccos(np.clip(np.abs(np.einsum("ij,ij->i", out["n"][ok], p.gt_n[ok])), 0, 1)))
        assert np.median(rel) < t["depth_rel_median"] and np.percentile(rel, 90) < t["depth_rel_p90"]
        assert np.median(ang) < t["normal_deg_median"] and np.percentile(ang, 90) < t["normal_deg_p90"]
        # the representation stays camera-facing
        rs = np.stack([_tile_ray(p, s) for s in range(p.S)])
        assert np.all(np.einsum("ij,ij->i", out["n"][ok], rs[ok]) < 0)


def test_gauss_newton_minimiser_matches_brute_force_scan():
    """Scan inverse depth +-10% x a 10 deg normal cone around the truth on the Huber cost; the
    Gauss-Newton fixed point lies within one fine grid cell (0.1 % / 0.25 deg) of the scan's minimum."""
    p = synth.ring_problem(0, P=16)
    ob = oracle.Problem.from_synth(p)
    out = ob.gauss_newton(PRM, 40, p.id0, p.n0, np.zeros(p.S, np.uint8))

    def cone(n_c, max_deg, step_deg):
        t1, t2 = oracle.tangent_basis(n_c)
        k = int(round(max_deg / step_deg))
        a = np.deg2rad(np.arange(-k, k + 1) * step_deg)
        A, B = [q.ravel() for q in np.meshgrid(a, a, indexing="ij")]
        keep = np.hypot(A, B) <= np.deg2rad(max_deg) + 1e-12
        v = n_c[None] + np.tan(A[keep])[:, None] * t1 + np.tan(B[keep])[:, None] * t2
        return v / np.linalg.norm(v, axis=1, keepdims=True)

    def scan(s, id_c, n_c, id_span, id_steps, max_deg, step_deg):
        N = cone(n_c, max_deg, step_deg)
        ids = id_c * (1 + np.linspace(-id_span, id_span, id_steps))
        E, _ = ob.cost_grid(PRM, s, np.repeat(ids, len(N)), np.tile(N, (len(ids), 1)))
        k = int(np.argmin(E))
        return ids[k // len(N)], N[k % len(N)], E[k]

    tiles = [s for s in _single_plane_tiles(p, 60) if (out["status"][s] & 0x3F) == oracle.OK][::3][:8]
    d_ang, d_id = [], []
    for s in tiles:
        i1, n1, _ = scan(s, p.gt_id[s], p.gt_n[s], 0.10, 41, 10.0, 1.0)          # whole domain, coarse
        i2, n2, e2 = scan(s, i1, n1, 0.01, 21, 2.0, 0.25)                       # refine around the best
        ids, ns = out["id"][s], out["n"][s]
        # Gauss-Newton reaches a cost no worse than the best grid point (0.1 % allows for the
        # sampled-gradient approximation in J) ...
        assert ob.eval_surfel(PRM, s, ids, ns)["E"] <= e2 * (1 + 1e-3), s
        d_id.append(abs(ids / i2 - 1))
        d_ang.append(np.rad2deg(np.arccos(min(1.0, abs(ns @ n2)))))
    # ... and sits at the scan's minimum: within one cell typically, a few cells along the
    # elongated valley of the weakest-observed normal direction at worst.
    assert np.median(d_id) <= 0.001 and max(d_id) <= 0.002
    assert np.median(d_ang) <= 0.25 and max(d_ang) <= 1.5


def test_adaptive_lm_never_raises_the_mean_cost_and_converges():
    """Marquardt schedule (option): accepted steps only lower the mean Huber cost, so the returned
    mean cost is at most the initial one for every surfel; on the noise-free ring views it reaches
    the same accuracy as the fixed damping, also from an initial lambda far too large for it."""
    t = TOL["convergence_ring"]
    p = synth.ring_problem(0, P=16)
    ob = oracle.Problem.from_synth(p)
    prm0 = oracle.params(lm_adaptive=True)
    start = ob.solve(prm0, 0, p.id0, p.n0, p.state)
    for lam, iters in ((1e-3, t["iterations"]), (1e3, t["iterations"] + 15)):
        prm = oracle.params(lm_adaptive=True, lm_lambda=lam)
        out = ob.solve(prm, iters, p.id0, p.n0, p.state)
        live = (start["nres"] >= 8) & (out["nres"] >= 8)
        mean0 = start["cost"][live] / start["nres"][live]
        mean1 = out["cost"][live] / out["nres"][live]
        assert np.all(mean1 <= mean0 * (1 + 1e-12))
        assert np.mean(mean1 < mean0) > 0.9
        ok = ((out["status"] & 0x3F) == oracle.OK) & (p.tile_prim >= 0)
        assert ok.sum() > 0.85 * (p.tile_prim >= 0).sum()
        rel = np.abs(out["id"][ok] / p.gt_id[ok] - 1)
        ang = np.rad2deg(np.arccos(np.clip(np.abs(np.einsum("ij,ij->i", out["n"][ok], p.gt_n[ok])), 0, 1)))
        assert np.median(rel) < t["depth_rel_median"] and np.percentile(rel, 90) < t["depth_rel_p90"]
        assert np.median(ang) < t["normal_deg_median"] and np.percentile(ang, 90) < t["normal_deg_p90"]
    # where steps move samples across the image border the valid-sample set changes: the schedule
    # compares the mean cost, so it still never rises
    q = synth.room_problem(3, W=320, H=240, F=3, seed_frac=0.0)
    oq = oracle.Problem.from_synth(q)
    s0 = oq.solve(prm0, 0, q.id0, q.n0, q.state)
    s1 = oq.solve(oracle.params(lm_adaptive=True), 10, q.id0, q.n0, q.state)
    live = (s0["nres"] >= 8) & (s1["nres"] >= 8)
    assert np.sum(s0["nres"][live] != s1["nres"][live]) > 20
    assert np.all(s1["cost"][live] / s1["nres"][live] <= s0["cost"][live] / s0["nres"][live] * (1 + 1e-12))
    # a fixed damping of 1e3 barely moves in the same number of iterations
    fixed = ob.solve(oracle.params(lm_lambda=1e3), t["iterations"] + 15, p.id0, p.n0, p.state)
    okf = ((fixed["status"] & 0x3F) == oracle.OK) & (p.tile_prim >= 0)
    angf = np.rad2deg(np.arccos(np.clip(np.abs(np.einsum("ij,ij->i", fixed["n"][okf], p.gt_n[okf])), 0, 1)))
    assert np.median(angf) > 5 * t["normal_deg_median"]


def test_circular_surfel_pixels_and_cost_gradient():
    """Circular surfels (radius option, Eq. 4): an interior surfel with every sample valid uses
    exactly the pixels strictly inside the radius of its tile centre (brute-force lattice count, F
    samples each), and on exact (linear) frames g is still the gradient of its Huber cost."""
    cam, ob, _, _ = _linear_problem(W=64, H=56)
    TX = 64 // 8
    for radius in (3.0, 4.2, 6.5, np.sqrt(6.5)):  # sqrt(6.5): pixels at (0.5, 2.5) sit on the boundary
        prm = oracle.params(huber_k=1e9, radius=radius)
        s = 3 * TX + 3  # tile (3, 3): centre (27.5, 27.5), the disc stays inside the image
        ux, uy = 3 * 8 + 3.5, 3 * 8 + 3.5
        yy, xx = np.mgrid[0:56, 0:64]
        count = int((np.sqrt((xx - ux) * (xx - ux) + (yy - uy) * (yy - uy)) < radius).sum())
        r_s = oracle.ray(cam, ux, uy)
        n0 = np.array([0.1, -0.05, -1.0]) / np.linalg.norm([0.1, -0.05, -1.0])
        e = ob.eval_surfel(prm, s, 0.5, n0)
        assert e["cnt"] == 2 * count and e["margin"] > 1e-3
        fd = _theta_fd(ob, prm, s, 0.5, n0, 1e-6, lambda q: q["E"])
        assert np.allclose(e["g"], fd, rtol=1e-5, atol=1e-9 * np.abs(e["g"]).max()), (radius, e["g"], fd)
    # the smallest disc: the four pixels nearest to the (half-integer) centre
    d = ob.eval_surfel(oracle.params(huber_k=1e9, radius=0.75), s, 0.5, n0)
    assert d["cnt"] == 2 * 4


def test_circular_surfels_converge_and_render():
    """Noise-free ring views with discs of radius 10 around 16-px tile centres (overlapping): the
    solve reaches the same accuracy as with tiles, and the depth map is the depth-buffered render
    of the discs, so every drawn pixel lies on the plane of the surfel that drew it."""
    t = TOL["convergence_ring"]
    p = synth.ring_problem(0, P=16)
    ob = oracle.Problem.from_synth(p)
    out = ob.solve(oracle.params(radius=10.0), t["iterations"], p.id0, p.n0, p.state)
    ok = ((out["status"] & 0x3F) == oracle.OK) & (p.tile_prim >= 0)
    assert ok.sum() > 0.85 * (p.tile_prim >= 0).sum()
    rel = np.abs(out["id"][ok] / p.gt_id[ok] - 1)
    ang = np.rad2deg(np.arccos(np.clip(np.abs(np.einsum("ij,ij->i", out["n"][ok], p.gt_n[ok])), 0, 1)))
    assert np.median(rel) < t["depth_rel_median"] and np.median(ang) < t["normal_deg_median"]
    sidx = out["sidx"]
    m = sidx >= 0
    yy, xx = np.mgrid[0:p.H, 0:p.W]
    s = sidx[m]
    TX = p.W // p.P
    ux, uy = (s % TX) * 16 + 7.5, (s // TX) * 16 + 7.5
    assert np.all(np.hypot(xx[m] - ux, yy[m] - uy) < 10.0)
    cam = p.cam
    r_u = np.stack([(xx[m] - cam[2]) / cam[0], (yy[m] - cam[3]) / cam[1], np.ones(m.sum())], 1)
    r_s = np.stack([(ux - cam[2]) / cam[0], (uy - cam[3]) / cam[1], np.ones(m.sum())], 1)
    nn = out["n"][s]
    assert np.allclose(np.einsum("ij,ij->i", r_u / out["inv_depth"][m][:, None], nn),
                       np.einsum("ij,ij->i", r_s / out["id"][s][:, None], nn), rtol=1e-10)
    assert m.mean() > 0.9  # radius 10 > 16 / sqrt(2): discs cover the tiled area
