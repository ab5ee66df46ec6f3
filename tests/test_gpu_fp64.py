"""FP64 route of the normal-equation solve (GPU through the C ABI against numpy and the FP64 oracle).

Surfels whose Jacobi-scaled normal matrix has a 2-norm condition number above `fp64_cond` solve the
damped system in FP64 (a square-root-free Cholesky factorisation); the others solve it in FP32."""
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


def _ulp_distance(a, b):
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_fp64_reciprocal_within_one_ulp_of_division():
    """The pivot reciprocal (hardware estimate + series correction) against IEEE 1/x over the
    whole exponent range of the pivots (positive normal doubles)."""
    import torch

    import paper_1910_01997_gb300 as sgn

    rng = np.random.default_rng(7)
    n = 1 << 20
    x = np.ldexp(1.0 + rng.random(n), rng.integers(-1000, 1000, n))
    x[:8] = [1.0, 2.0, 0.5, 3.0, 1.0 - 2.0**-53, 1.0 + 2.0**-52, 2.0**-1000, 1.5 * 2.0**1000]
    r = sgn.sgn_check_fp64_reciprocal(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    d = _ulp_distance(r, ref)
    assert d.max() <= 1, (x[d.argmax()], r[d.argmax()], ref[d.argmax()])
    assert np.mean(d == 0) > 0.99
    for bad in (-1, ):
        with pytest.raises(sgn.SgnError):
            sgn._call("sgn_check_fp64_reciprocal", 0, 0, bad, None)


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
    assert st["n"] >= TOL["well_posed"]["min_stable_frac"]["f32"] * st["n_usable"]
    assert st["depth_max"] <= tol["depth_rel"] and st["ang_max"] <= tol["normal_deg"], (st["depth_max"], st["ang_max"])
