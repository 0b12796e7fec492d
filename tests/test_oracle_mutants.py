"""The pins in test_oracle_pins.py must catch plausible transcription
mistakes.  Each case below plants one mistake in a copy of the oracle's C
source (on the CPU, in a temporary directory), builds it, and runs the pin
suite against it: the suite must fail for every mutant."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "pn_oracle.c")
INC = os.path.join(ROOT, "oracle", "pn_oracle_accel.inc")

MUTANTS = [
    ("Eq.6 line 2: 5/(4 r_j1) -> 4/(4 r_j1)",
     "4.0 / rij + 5.0 / (4.0 * rj1) + ri1_2", "4.0 / rij + 4.0 / (4.0 * rj1) + ri1_2"),
    ("Eq.6 line 4: sign of the -7/2 term",
     "kadd3(&pn, -3.5 * G * G * mj * M / rj1_3", "kadd3(&pn, 3.5 * G * G * mj * M / rj1_3"),
    ("Eq.6 line 5: coefficient 3 -> 4",
     "kadd3(&pn, g5 * 3.0 * dot(vj, xi1), vi);", "kadd3(&pn, g5 * 4.0 * dot(vj, xi1), vi);"),
    ("Eq.6 line 6: square dropped", "1.5 * vj_nij * vj_nij", "1.5 * vj_nij"),
    ("Eq.6 line 7: v_ij -> v_i",
     "kadd3(&pn, G * mj / rij_3 * dot(xij, w), vij);", "kadd3(&pn, G * mj / rij_3 * dot(xij, w), vi);"),
    ("Eq.6 line 1: 5 G^2 m_i M -> 4",
     "kadd3(&pn, 5.0 * G * G * mi * M / ri1_4, xi1);", "kadd3(&pn, 4.0 * G * G * mi * M / ri1_4, xi1);"),
    ("Eq.5: 4GM (v.x) v -> 3GM",
     "kadd3(&pn, 4.0 * G * M / ri1_3 * vi_xi1, vi);", "kadd3(&pn, 3.0 * G * M / ri1_3 * vi_xi1, vi);"),
    ("Eq.2: 5GM/r -> 4GM/r", "(5.0 * G * M / r1j - 2.0", "(4.0 * G * M / r1j - 2.0"),
    ("Eq.3 line 1: 4 G^2 m_j^2 -> 3",
     "kadd3(&pn, 4.0 * G * G * mj * mj / r1j_4, x1j);", "kadd3(&pn, 3.0 * G * G * mj * mj / r1j_4, x1j);"),
    ("Eq.3: r_1j^2/(4 r_jk^3) sign", "+ r1j_2 / (4.0 * rjk_3)), x1j);", "- r1j_2 / (4.0 * rjk_3)), x1j);"),
    ("Eq.3: -7/2 -> -3",
     "kadd3(&acc, -3.5 * G * G * mj * mk / (rjk_3 * r1j), xjk);",
     "kadd3(&acc, -3.0 * G * G * mj * mk / (rjk_3 * r1j), xjk);"),
    ("Eq.3: k = j dropped from the velocity-replacement sum",
     "        if (k == j)\n            continue;\n        const REAL r1k_2", "        const REAL r1k_2"),
    ("softening on a hole-star separation (star equation)",
     "const REAL rj1 = SQRT(dot(xj1, xj1));", "const REAL rj1 = SQRT(dot(xj1, xj1) + e2);"),
    ("softening on a hole-star separation (hole equation)",
     "const REAL r1k = SQRT(r1k_2);", "const REAL r1k = SQRT(r1k_2 + e2);"),
    ("Eq.7: 6 v_i^2 -> 7 v_i^2", "0.25 * gmm * (6.0 * vi2", "0.25 * gmm * (7.0 * vi2"),
    ("Eq.7: i = j term of the last double sum dropped twice",
     "kadd(&ePN, 0.5 * o[3]);", "kadd(&ePN, o[3]);"),
    ("Eq.7: -7 v_1.v_i -> -6", "0.5 * gmm * (3.0 * v1_2 - 7.0", "0.5 * gmm * (3.0 * v1_2 - 6.0"),
    ("Eq.8: star-star factor 1/2 dropped",
     "kadd3(&s_p, -0.5 * gmm, w);", "kadd3(&s_p, -1.0 * gmm, w);"),
    ("integrator: no velocity prediction",
     "vp[q] = vel_mode == 0 ? vh[q] + h * a[q] : vh[q];", "vp[q] = vel_mode == 0 ? vh[q] : vh[q];"),
    ("jerk: velocity tangent (the a_j of Appendix A) dropped",
     "return orc_accel_jvp(n, x, v, m, G, inv_c2, eps, v, a, 0.0, 0.0, jerk);",
     "return orc_accel_jvp(n, x, v, m, G, inv_c2, eps, v, v, 0.0, 0.0, jerk);"),
    ("Hermite corrector: dt^2/12 -> dt^2/10 in the velocity",
     "dt2 / 12.0 * (j0[q] - j1[q]);", "dt2 / 10.0 * (j0[q] - j1[q]);"),
    ("trajectory derivative: KDK velocity prediction dropped",
     "vp[q] = vel_mode == 0 ? vh[q] + 0.5 * dt * ac[q] : vh[q];", "vp[q] = vh[q];"),
    ("trajectory derivative: hole-mass perturbation dropped",
     "mc[0] = m[0] + I * (h * dM);", "mc[0] = m[0];"),
    ("Hermite: a single evaluate-correct pass",
     "for (int pass = 0; pass < 2 && rc == 0; ++pass)", "for (int pass = 0; pass < 1 && rc == 0; ++pass)"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    src, inc = open(SRC).read(), open(INC).read()
    assert old in src or old in inc, f"mutation site vanished: {name}"
    c = tmp_path / "mutant.c"
    so = tmp_path / "mutant.so"
    if old in src:
        src = src.replace(old, new, 1)
    else:
        inc = inc.replace(old, new, 1)
    c.write_text(src)
    (tmp_path / os.path.basename(INC)).write_text(inc)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(so), str(c), "-lm"], check=True)
    env = dict(os.environ, PN_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
