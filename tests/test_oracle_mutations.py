"""The oracle's pins must catch plausible mistakes (CPU only).

Each case compiles a copy of the oracle with one planted mistake (a dropped term, a wrong
sign, a wrong index or a transposed operand) and runs the pin suite against it in a
subprocess; the suite has to fail.  The mistakes are planted in the oracle only.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "surfel_gn.c")

MUTANTS = {
    "drop 1/id_u^2 in dq/d id_u": (
        "dq[i] = -(T[4 * i + 0] * r_u[0] + T[4 * i + 1] * r_u[1] + T[4 * i + 2] * r_u[2]) / (id_u * id_u);",
        "dq[i] = -(T[4 * i + 0] * r_u[0] + T[4 * i + 1] * r_u[1] + T[4 * i + 2] * r_u[2]) / id_u;"),
    "wrong sign in Eq. 9": (
        "d_dn[i] = r_u[i] / psn - run * p_s[i] / (psn * psn);",
        "d_dn[i] = r_u[i] / psn + run * p_s[i] / (psn * psn);"),
    "r_u and p_s swapped as printed in Eq. 9": (
        "d_dn[i] = r_u[i] / psn - run * p_s[i] / (psn * psn);",
        "d_dn[i] = p_s[i] / run - psn * r_u[i] / (run * run);"),
    "transposed rotation in the warp": (
        "q[i] = T[4 * i + 0] * p_u[0] + T[4 * i + 1] * p_u[1] + T[4 * i + 2] * p_u[2] + T[4 * i + 3];",
        "q[i] = T[0 + i] * p_u[0] + T[4 + i] * p_u[1] + T[8 + i] * p_u[2] + T[4 * i + 3];"),
    "bilinear weights swapped": (
        "return (1.0 - ay) * ((1.0 - ax) * v00 + ax * v10) + ay * ((1.0 - ax) * v01 + ax * v11);",
        "return (1.0 - ax) * ((1.0 - ay) * v00 + ay * v10) + ax * ((1.0 - ay) * v01 + ay * v11);"),
    "forward-difference gradient": (
        "gx[i] = (x >= 1 && x <= W - 2) ? 0.5 * (img[i + 1] - img[i - 1]) : 0.0;",
        "gx[i] = (x >= 1 && x <= W - 2) ? (img[i + 1] - img[i]) : 0.0;"),
    "Huber weight not applied to g": (
        "for (int a = 0; a < 3; ++a) g[a] += w * J[a] * r;",
        "for (int a = 0; a < 3; ++a) g[a] += J[a] * r;"),
    "tangent directions swapped in J": (
        "double Jt[3] = {dot3(d_dn, t1), dot3(d_dn, t2), d_did};",
        "double Jt[3] = {dot3(d_dn, t2), dot3(d_dn, t1), d_did};"),
    "damping not rotation invariant": (
        "double A[6] = {H[0] + lambda * m, H[1], H[2], H[3] + lambda * m, H[4], H[5] + lambda * H[5]};",
        "double A[6] = {H[0] + lambda * H[0], H[1], H[2], H[3] + lambda * H[0], H[4], H[5] + lambda * H[5]};"),
    "step sign flipped": (
        "double rhs[3] = {-g[0], -g[1], -g[2]};",
        "double rhs[3] = {g[0], g[1], g[2]};"),
    "seeding without camera-facing flip": (
        "double sgn = dot3(nq, r_q) < 0.0 ? 1.0 : -1.0;",
        "double sgn = 1.0;"),
    "seeding against the wrong tile ray": (
        "double v = orc_inv_depth(r_new, r_q, id_in[q], nq);",
        "double v = orc_inv_depth(r_q, r_new, id_in[q], nq);"),
    "tile centre off by half a pixel": (
        "double ux = tx * pb->P + 0.5 * (pb->P - 1), uy = ty * pb->P + 0.5 * (pb->P - 1);",
        "double ux = tx * pb->P + 0.5 * pb->P, uy = ty * pb->P + 0.5 * pb->P;"),
    "adaptive schedule accepts a cost increase": (
        "accept = cnt2 >= prm->min_residuals && E2 * cnt < E * cnt2;",
        "accept = cnt2 >= prm->min_residuals && E2 * cnt > E * cnt2;"),
    "adaptive schedule inverted": (
        "lambda = fmax(lambda / 10.0, 1e-7);", "lambda = fmin(lambda * 10.0, 1e7);"),
    "adaptive schedule compares total instead of mean cost": (
        "accept = cnt2 >= prm->min_residuals && E2 * cnt < E * cnt2;",
        "accept = cnt2 >= prm->min_residuals && E2 < E;"),
    "circular surfel boundary inclusive": (
        "if (rad > 0.0 && !(sqrt((ux - ucx) * (ux - ucx) + (uy - ucy) * (uy - ucy)) < rad)) continue;",
        "if (rad > 0.0 && !(sqrt((ux - ucx) * (ux - ucx) + (uy - ucy) * (uy - ucy)) <= rad)) continue;"),
    "circular surfel centred on the tile corner": (
        "const double ucx = tx * P + 0.5 * (P - 1), ucy = ty * P + 0.5 * (P - 1), rad = prm->radius;",
        "const double ucx = tx * P, ucy = ty * P, rad = prm->radius;"),
    # reference-frame change and depth-buffered render (pinned by test_oracle_transfer.py)
    "frame change with transposed rotation": (
        "p1[k] = T[4 * k] * p0[0] + T[4 * k + 1] * p0[1] + T[4 * k + 2] * p0[2] + T[4 * k + 3];",
        "p1[k] = T[k] * p0[0] + T[4 + k] * p0[1] + T[8 + k] * p0[2] + T[4 * k + 3];", "transfer"),
    "frame change without translation": (
        "p1[k] = T[4 * k] * p0[0] + T[4 * k + 1] * p0[1] + T[4 * k + 2] * p0[2] + T[4 * k + 3];",
        "p1[k] = T[4 * k] * p0[0] + T[4 * k + 1] * p0[1] + T[4 * k + 2] * p0[2];", "transfer"),
    "frame change leaves the normal unrotated": (
        "n1[k] = T[4 * k] * n_in[3 * i] + T[4 * k + 1] * n_in[3 * i + 1] + T[4 * k + 2] * n_in[3 * i + 2];",
        "n1[k] = n_in[3 * i + k];", "transfer"),
    "new inverse depth taken as the depth": (
        "id_out[i] = ok ? 1.0 / p1[2] : 0.0;", "id_out[i] = ok ? p1[2] : 0.0;", "transfer"),
    "render keeps the farthest surfel": (
        "if (v > inv_depth[k]) {", "if (sidx[k] < 0 || v < inv_depth[k]) {", "transfer"),
    "render ties go to the higher index": (
        "if (v > inv_depth[k]) {", "if (v >= inv_depth[k]) {", "transfer"),
    "render radius test inclusive": (
        "if (!(sqrt(dx * dx + dy * dy) < radius)) continue;",
        "if (!(sqrt(dx * dx + dy * dy) <= radius)) continue;", "transfer"),
}
PIN_FILES = {None: "test_oracle_pins.py", "transfer": "test_oracle_transfer.py"}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(name, tmp_path):
    old, new, *which = MUTANTS[name]
    pins = PIN_FILES[which[0] if which else None]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           str(mut), "-o", str(so), "-lm"])
    env = dict(os.environ, ORACLE_SO=str(so), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
