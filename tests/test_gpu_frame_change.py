"""Reference-frame change (Sec. 2.5, Eq. 10) and depth-buffered surfel render (Sec. 2.2) on the GPU,
through the C ABI, against the FP64 oracle on the same inputs."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _surfels(prob):
    """The valid surfels of a problem as free surfels at their tile centres (float32)."""
    TX = prob.W // prob.P
    s = np.flatnonzero(prob.state == synth.VALID)
    u = np.stack([(s % TX) * prob.P + (prob.P - 1) / 2.0, (s // TX) * prob.P + (prob.P - 1) / 2.0], 1)
    return u.astype(np.float32), prob.id0[s].astype(np.float32), prob.n0[s].astype(np.float32)


def _gpu_transfer(cam, T, u, idv, n):
    import torch

    import paper_1910_01997_gb300 as sgn

    out = sgn.sgn_transfer_surfels(cam, T, torch.from_numpy(u).cuda(), torch.from_numpy(idv).cuda(),
                                   torch.from_numpy(n).cuda())
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _gpu_render(cam, W, H, u, idv, n, valid, radius):
    import torch

    import paper_1910_01997_gb300 as sgn

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    inv, sidx = sgn.sgn_render_surfels(cam, W, H, t(u), t(idv), t(n), t(valid.astype(np.uint8)), radius)
    torch.cuda.synchronize()
    return inv.cpu().numpy(), sidx.cpu().numpy()


def test_transfer_parity():
    prob = synth.room_problem(0)
    u, idv, n = _surfels(prob)
    for f in range(prob.F):
        g = _gpu_transfer(prob.cam, prob.poses[f], u, idv, n)
        ou, oi, on, ov = oracle.transfer_surfels(prob.cam, prob.poses[f], u, idv, n)
        assert np.array_equal(g["valid"], ov)
        v = ov.astype(bool)
        assert v.sum() > 0.9 * len(v)
        assert np.abs(g["u"][v] - ou[v]).max() < 2e-3
        assert np.abs(g["inv_depth"][v] / oi[v] - 1).max() < 2e-6
        assert np.abs(g["normal"][v] - on[v]).max() < 2e-6


def test_transfer_edge_cases():
    cam = (140.0, 140.0, 79.5, 59.5)
    u = np.array([[10, 10], [80, 60], [80, 60], [150, 110]], np.float32)
    idv = np.array([0.5, -0.2, 0.0, 0.25], np.float32)
    n = np.tile(np.array([0, 0, -1], np.float32), (4, 1))
    T = np.hstack([np.eye(3), np.array([[0.0], [0.0], [-3.0]])])  # surfel 3 (4 m away) stays in front
    g = _gpu_transfer(cam, T, u, idv, n)
    assert g["valid"].tolist() == [0, 0, 0, 1]  # behind the camera, negative and zero inverse depth
    assert np.all(g["inv_depth"][:3] == 0) and np.all(g["u"][:3] == 0)
    assert abs(g["inv_depth"][3] - 1.0) < 1e-6
    import paper_1910_01997_gb300 as sgn
    import torch

    bad = np.hstack([2 * np.eye(3), np.zeros((3, 1))])
    with pytest.raises(sgn.SgnError):
        sgn.sgn_transfer_surfels(cam, bad, torch.zeros(1, 2).cuda(), torch.ones(1).cuda(), torch.zeros(1, 3).cuda())
    empty = sgn.sgn_transfer_surfels(cam, T, torch.zeros(0, 2).cuda(), torch.zeros(0).cuda(), torch.zeros(0, 3).cuda())
    assert empty["valid"].numel() == 0


def _boundary_pixels(W, H, u, valid, radius, eps):
    """Pixels whose centre lies within eps of some valid surfel's disc boundary."""
    amb = np.zeros((H, W), bool)
    for (x, y), v in zip(u.astype(np.float64), valid):
        if not v:
            continue
        x0, x1 = max(int(np.floor(x - radius - 1)), 0), min(int(np.ceil(x + radius + 1)), W - 1)
        y0, y1 = max(int(np.floor(y - radius - 1)), 0), min(int(np.ceil(y + radius + 1)), H - 1)
        if x0 > x1 or y0 > y1:
            continue
        yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        amb[y0:y1 + 1, x0:x1 + 1] |= np.abs(np.hypot(xx - x, yy - y) - radius) < eps
    return amb


def _check_render(cam, W, H, u, idv, n, valid, radius):
    g_inv, g_sidx = _gpu_render(cam, W, H, u, idv, n, valid, radius)
    o_inv, o_sidx, o_second = oracle.render_surfels(cam, W, H, u, idv, n, valid, radius, with_second=True)
    amb = _boundary_pixels(W, H, u, valid, radius, 1e-3)
    # coverage: same pixels drawn, except at disc boundaries within FP32 rounding
    assert np.array_equal((g_sidx >= 0) & ~amb, (o_sidx >= 0) & ~amb)
    both = (g_sidx >= 0) & (o_sidx >= 0) & ~amb
    # FP32 error of Eq. 3 in the form id_s (1 + e), e = ((r_u - r_s) . n) / (r_s . n), relative to
    # id_u: about eps (1 + (|dx n_x| / fx + |dy n_y| / fy) / |r_s . n|) / |1 + e| (it grows where
    # the plane is seen edge-on), for the oracle's nearest surfel at each pixel
    yy, xx = np.mgrid[0:H, 0:W]
    s = o_sidx[both]
    us = u.astype(np.float64)[s]
    dx, dy = xx[both] - us[:, 0], yy[both] - us[:, 1]
    nn = n.astype(np.float64)[s]
    rsn = (us[:, 0] - cam[2]) / cam[0] * nn[:, 0] + (us[:, 1] - cam[3]) / cam[1] * nn[:, 1] + nn[:, 2]
    terms = np.abs(dx * nn[:, 0]) / cam[0] + np.abs(dy * nn[:, 1]) / cam[1]
    one_e = o_inv[both] / idv.astype(np.float64)[s]
    bound = 1e-6 + 8 * 6e-8 * (1 + terms / np.abs(rsn)) / np.abs(one_e)
    # a unique nearest surfel: ahead of the runner-up by more than twice that error
    u_mask = (o_inv[both] - o_second[both]) > (2 * bound + 1e-5) * o_inv[both]
    unique = np.zeros_like(both)
    unique[both] = u_mask
    assert np.array_equal(g_sidx[unique], o_sidx[unique])
    rel = np.abs(g_inv[both] / o_inv[both] - 1)
    assert np.all(rel[u_mask] <= bound[u_mask]), (rel[u_mask] / bound[u_mask]).max()
    # near ties: the GPU keeps one of the tied surfels, whose value is within the tie of the nearest
    assert np.all(rel[~u_mask] <= 2 * (1e-5 + 2 * bound[~u_mask]))
    return int(both.sum()), int(unique.sum()), int(amb.sum())


def test_render_parity_transferred_room_surfels():
    """The benchmark room's surfels moved into each observing frame and rendered there as discs of
    the tile's area (radius 8 / sqrt(pi)) and of radius 6 (overlapping neighbours)."""
    prob = synth.room_problem(0)
    u, idv, n = _surfels(prob)
    for f in (0, prob.F - 1):
        ou, oi, on, ov = oracle.transfer_surfels(prob.cam, prob.poses[f], u, idv, n)
        for radius in (8 / np.sqrt(np.pi), 6.0):
            both, unique, amb = _check_render(prob.cam, prob.W, prob.H, ou.astype(np.float32), oi.astype(np.float32),
                                              on.astype(np.float32), ov, radius)
            print(f"frame {f} radius {radius:.2f}: drawn in both {both}, unique winner {unique}, boundary {amb}")
            assert both > 0.5 * prob.W * prob.H and unique > 0.9 * both


def test_render_edge_cases():
    cam = (140.0, 140.0, 79.5, 59.5)
    W, H = 160, 120
    rng = np.random.default_rng(5)
    k = 50
    u = np.concatenate([rng.uniform(-20, 180, (k, 2)), [[-500.0, 30.0], [1e9, 1e9], [79.5, 59.5]]]).astype(np.float32)
    idv = np.concatenate([rng.uniform(0.2, 1.0, k), [0.5, 0.5, 0.5]]).astype(np.float32)
    nn = rng.normal(size=(k + 3, 3))
    nn[:, 2] = -np.abs(nn[:, 2]) - 1
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    nn = nn.astype(np.float32)
    valid = np.ones(k + 3, np.uint8)
    valid[::7] = 0  # skipped
    for radius in (0.3, 2.5, 12.0, 100.0):
        _check_render(cam, W, H, u, idv, nn, valid, radius)
    # nothing to draw: every pixel empty
    g_inv, g_sidx = _gpu_render(cam, W, H, u, idv, nn, np.zeros(k + 3, np.uint8), 5.0)
    assert (g_sidx == -1).all() and (g_inv == 0).all()
    import paper_1910_01997_gb300 as sgn
    import torch

    z = torch.zeros(0).cuda()
    inv, sidx = sgn.sgn_render_surfels(cam, W, H, z.reshape(0, 2), z, z.reshape(0, 3), torch.zeros(0, dtype=torch.uint8).cuda(), 3.0)
    assert (sidx == -1).all()
    with pytest.raises(sgn.SgnError):
        sgn.sgn_render_surfels(cam, W, H, z.reshape(0, 2), z, z.reshape(0, 3), torch.zeros(0, dtype=torch.uint8).cuda(), -1.0)
