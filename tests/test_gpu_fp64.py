"""FP64 route of the normal-equation solve (GPU through the C ABI against numpy and the FP64 oracle).

Surfels whose Jacobi-scaled normal matrix has a 2-norm condition number above `fp64_cond` solve the
damped system in FP64 (Cramer's rule, one component per lane); the others solve it in FP32."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import compare, gpu_solve, oracle_solve, oracle_stable

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = json.load(open(os.path.join(HERE, "tolerances.json")))
FP64_FLAG = 0x80


def _random_systems(rng, n, log_cond_max=10.0, indefinite=False):
    """Symmetric 3x3 normal matrices D S D (S unit-diagonal-ish with a log-uniform condition number,
    D a diagonal scale over five decades) and right-hand sides, rounded to float32."""
    Q, _ = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    ev = np.stack([np.ones(n), 10.0 ** rng.uniform(-log_cond_max / 2, 0, n), 10.0 ** -rng.uniform(0, log_cond_max, n)], 1)
    if indefinite:
        ev[:, 2] = -rng.uniform(0.05, 0.5, n)
    S = np.einsum("nij,nj,nkj->nik", Q, ev, Q)
    d = 10.0 ** rng.uniform(-1, 4, (n, 3))
    H = S * d[:, :, None] * d[:, None, :]
    H6 = np.stack([H[:, 0, 0], H[:, 0, 1], H[:, 0, 2], H[:, 1, 1], H[:, 1, 2], H[:, 2, 2]], 1).astype(np.float32)
    g3 = (rng.normal(size=(n, 3)) * d).astype(np.float32)
    return H6, g3


def _damped(H6, lam):
    H = H6.astype(np.float64)
    A = np.empty((len(H), 3, 3))
    idx = [(0, 0, 0), (0, 1, 1), (0, 2, 2), (1, 1, 3), (1, 2, 4), (2, 2, 5)]
    for i, j, k in idx:
        A[:, i, j] = A[:, j, i] = H[:, k]
    m = 0.5 * (H[:, 0] + H[:, 3])
    A[:, 0, 0] += lam * m
    A[:, 1, 1] += lam * m
    A[:, 2, 2] += lam * H[:, 5]
    return A


def test_fp64_solve_matches_numpy():
    """The FP64 route of the damped solve (Cramer's rule, one component per lane of a group) on
    random systems with scaled condition numbers up to 1e10 over five decades of diagonal scale, at
    the default damping and at the smallest damping of the Marquardt schedule, against numpy's FP64
    solve of the same float32 inputs: within FP32 rounding of the result plus 1e4 cond x 2^-53 in the
    Jacobi-scaled variables; damped matrices with a clearly negative eigenvalue are reported as not
    positive definite."""
    import torch

    import paper_1910_01997_gb300 as sgn

    rng = np.random.default_rng(11)
    n = 20000
    H6, g3 = _random_systems(rng, n)
    worst = 0.0
    for lam in (1e-3, 1e-7):
        delta, pd = sgn.sgn_check_fp64_solve(torch.from_numpy(H6).cuda(), torch.from_numpy(g3).cuda(), lam)
        delta, pd = delta.cpu().numpy().astype(np.float64), pd.cpu().numpy()
        A = _damped(H6, lam)
        dsc = np.sqrt(np.einsum("nii->ni", A))
        S = A / (dsc[:, :, None] * dsc[:, None, :])
        w = np.linalg.eigvalsh(S)
        posdef = w[:, 0] > 1e-11
        assert posdef.mean() > 0.95 and pd[posdef].all()
        assert not pd[w[:, 0] < -1e-9].any()
        x = np.linalg.solve(A[posdef], -g3.astype(np.float64)[posdef, :, None])[:, :, 0]
        cond = w[posdef, 2] / w[posdef, 0]
        err = np.linalg.norm((delta[posdef] - x) * dsc[posdef], axis=1) / np.linalg.norm(x * dsc[posdef], axis=1)
        # Cramer's rule is not backward stable: its forward error grows faster than cond x 2^-53
        # (up to ~4e3 cond x 2^-53 on these systems), still far below the FP32 route's cond x 2^-24
        bound = 2.0**-22 + 1e4 * 2.0**-53 * cond
        assert np.all(err <= bound), (lam, (err / bound).max())
        worst = max(worst, (err / bound).max())
        print("lambda", lam, "cond max", cond.max(), "max err / bound", (err / bound).max())
    # indefinite systems (one negative eigenvalue): not positive definite
    H6n, g3n = _random_systems(rng, 4096, log_cond_max=4.0, indefinite=True)
    wn = np.linalg.eigvalsh(_damped(H6n, 1e-3))
    neg = wn[:, 0] < -1e-3 * np.abs(wn).max(1)
    _, pdn = sgn.sgn_check_fp64_solve(torch.from_numpy(H6n).cuda(), torch.from_numpy(g3n).cuda(), 1e-3)
    assert neg.sum() > 2000 and not pdn.cpu().numpy()[neg].any()
    # an odd count (the last warp's second group idle) gives the same results, and the argument checks
    d_all, _ = sgn.sgn_check_fp64_solve(torch.from_numpy(H6[:4]).cuda(), torch.from_numpy(g3[:4]).cuda(), 1e-3)
    d1, p1 = sgn.sgn_check_fp64_solve(torch.from_numpy(H6[:3]).cuda(), torch.from_numpy(g3[:3]).cuda(), 1e-3)
    assert np.array_equal(d1.cpu().numpy(), d_all.cpu().numpy()[:3]) and p1.cpu().numpy().all()
    with pytest.raises(sgn.SgnError):
        sgn._call("sgn_check_fp64_solve", 0, 0, 1e-3, 5, 0, 0, None)
    with pytest.raises(sgn.SgnError):
        sgn._call("sgn_check_fp64_solve", 0, 0, -1.0, 0, 0, 0, None)


def _scaled_cond(H6):
    """2-norm condition number of the unit-diagonal (Jacobi-scaled) symmetric 3x3 matrix (numpy FP64)."""
    H = np.array([[H6[0], H6[1], H6[2]], [H6[1], H6[3], H6[4]], [H6[2], H6[4], H6[5]]])
    d = np.sqrt(np.diag(H))
    S = H / np.outer(d, d)
    w = np.linalg.eigvalsh(S)
    return np.inf if w[0] <= 0 else w[-1] / w[0]


def test_route_follows_the_condition_number():
    """One iteration from given surfels: a surfel's first solve runs in FP64 exactly when the scaled
    condition number of its normal matrix (numpy eigenvalues of the oracle's FP64 matrix at the
    same parameters) exceeds the threshold; surfels within 5 % of the threshold, or with a sample
    on the validity bound, may go either way."""
    prob = synth.room_problem(6, seed_frac=0.0)
    op = oracle.Problem.from_synth(prob)
    prm = oracle.params()
    live = np.flatnonzero(prob.state == synth.VALID)
    cond = np.full(prob.S, np.nan)
    margin = np.zeros(prob.S)
    for s in live:
        e = op.eval_surfel(prm, int(s), float(np.float32(prob.id0[s])), prob.n0[s].astype(np.float32).astype(np.float64))
        if e["cnt"] >= 8 and np.all(np.isfinite(e["H"])) and min(e["H"][0], e["H"][3], e["H"][5]) > 0:
            cond[s] = _scaled_cond(e["H"])
            margin[s] = e["margin"]
    ok = np.isfinite(cond)
    assert ok.sum() > 2000
    for quantile in (0.7, 0.98):
        thr = float(np.quantile(cond[ok], quantile))
        g = gpu_solve(prob, 1, fp64_cond=thr)
        routed = (g["status"] & FP64_FLAG) != 0
        clear = ok & (np.abs(np.log(cond / thr)) > np.log(1.05)) & (margin > TOL["well_posed"]["margin_px"])
        assert clear.sum() > 0.8 * ok.sum()
        wrong = clear & (routed != (cond > thr))
        assert wrong.sum() == 0, (cond[wrong][:10], routed[wrong][:10], thr)
        assert abs(routed[clear].mean() - (1 - quantile)) < 0.1
    # no route at all when disabled
    assert not ((gpu_solve(prob, 1, fp64_cond=0.0)["status"] & FP64_FLAG) != 0).any()


def test_all_solves_in_fp64_match_oracle():
    """fp64_cond = 1 routes every positive-definite system: full-size parity of the FP64 solve with
    the FP64 oracle at the FP32 tolerances."""
    prob = synth.room_problem(5)
    g, o = gpu_solve(prob, 10, fp64_cond=1.0), oracle_solve(prob, 10)
    tol = TOL["parity"]["f32"]
    stable = oracle_stable(prob, 10, tol["depth_rel"], tol["normal_deg"], o, dtype="f32")
    st = compare(prob, g, o, margin_px=TOL["well_posed"]["margin_px"], stable=stable)
    print("all-FP64", {k: v for k, v in st.items() if k not in ("rel", "ang", "mask", "stable")})
    ok = (g["status"] & 0x3F) == 0
    assert ((g["status"][ok] & FP64_FLAG) != 0).mean() > 0.99
    assert st["n"] >= TOL["well_posed"]["min_stable_frac"]["room"] * st["n_usable"]
    assert st["depth_max"] <= tol["depth_rel"] and st["ang_max"] <= tol["normal_deg"], (st["depth_max"], st["ang_max"])
