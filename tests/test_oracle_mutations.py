"""The pins catch plausible mistakes in the checker.

Each case copies the checker's source, plants one mistake of the kind that
slips into a hand-written model (a dropped term, a flipped sign, a swapped
operand or index, a wrong weight), builds it on the side, and runs the pin
tests against it: at least one pin must fail.  The checker's own source is
left untouched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle")

MUTATIONS = {
    "drop drag": ("dx[3 + i] = b3[i] * acc - drag * v[i];", "dx[3 + i] = b3[i] * acc;"),
    "gravity sign": ("dx[5] = dx[5] - P.g;", "dx[5] = dx[5] + P.g;"),
    "body z transposed": ("b3[0] = T(2.0) * (x * z + w * y);", "b3[0] = T(2.0) * (x * z - w * y);"),
    "q' = [0, w] o q": ("hamilton(q, wq, qd);", "hamilton(wq, q, qd);"),
    "gyroscopic sign": ("cross(om, Iw, gyro);", "cross(Iw, om, gyro);"),
    "drop gyroscopic term": ("dx[10 + i] = (u[1 + i] - gyro[i]) / P.J[i];", "dx[10 + i] = u[1 + i] / P.J[i];"),
    "inertia index": ("dx[10 + i] = (u[1 + i] - gyro[i]) / P.J[i];", "dx[10 + i] = (u[1 + i] - gyro[i]) / P.J[(i + 1) % 3];"),
    "rotor lag sign": ("dx[13 + i] = (w[i] - Om[i]) / P.tau_m;", "dx[13 + i] = (Om[i] - w[i]) / P.tau_m;"),
    "RK4 weight": ("(k1[i] + T(2.0) * k2[i] + T(2.0) * k3[i] + k4[i])", "(k1[i] + T(2.0) * k2[i] + k3[i] + T(2.0) * k4[i])"),
    "yaw row sign": ("u[3] = T(r) * (f[0] - f[1] + f[2] - f[3]);", "u[3] = T(r) * (-f[0] + f[1] - f[2] + f[3]);"),
    "attitude error order": ("hamilton(qc, qd, qe);", "hamilton(qd, qc, qe);"),
    "Shepperd sign": ("q[1] = (R[2][1] - R[1][2]) * k;", "q[1] = (R[1][2] - R[2][1]) * k;"),
    "no acceleration clamp": ("const T a = clampv(ar, -val(P.a_max), val(P.a_max));", "const T a = ar;"),
    "rate loop sign": ("(wdes - om[i]);", "(om[i] - wdes);"),
    "attitude gain x1": ("const T wdes = T(2.0) * P.katt[i] * qe[1 + i];", "const T wdes = P.katt[i] * qe[1 + i];"),
    "PID derivative sign": ("+ P.kI[i] * xi[i] - P.kD[i] * wdot[i]);", "+ P.kI[i] * xi[i] + P.kD[i] * wdot[i]);"),
    "PID integrator sign": ("x[NX + i] + T(h) * e[i]", "x[NX + i] - T(h) * e[i]"),
    "PID integral index": ("P.kI[i] * xi[i]", "P.kI[i] * xi[(i + 1) % 3]"),
    "PID no anti-windup": ("xn[NX + i] = clampv(x[NX + i] + T(h) * e[i], -lim, lim);", "xn[NX + i] = x[NX + i] + T(h) * e[i];"),
    # car and fixed-wing models (vehicles.hpp)
    "car curvature factor": ("vehicles.hpp", "T(2.0) * cross / (dist * ld)", "cross / (dist * ld)"),
    "car no look-ahead floor": ("vehicles.hpp", "val(dist) > P.veh[4] ? dist : T(P.veh[4])", "dist"),
    "heading rotation sign": ("vehicles.hpp", "dx[6] = -s * turn;", "dx[6] = s * turn;"),
    "fixed-wing turn rate": ("vehicles.hpp", "P.g * tan(x[10]) / v", "P.g * x[10] / v"),
    "fixed-wing altitude loop": ("vehicles.hpp", "T(P.veh[4]) * (u[1] - x[2])", "T(P.veh[4]) * (x[2] - u[1])"),
    "fixed-wing course error": ("vehicles.hpp", "atan2(cross, dot)", "atan2(dot, cross)"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    entry = MUTATIONS[name]
    fname, old, new = entry if len(entry) == 3 else ("quad_model.hpp", *entry)
    work = tmp_path / "oracle"
    shutil.copytree(SRC, work, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    model = work / fname
    text = model.read_text()
    assert text.count(old) == 1, f"mutation anchor not unique for {name!r}"
    model.write_text(text.replace(old, new))
    lib = work / "liboracle_mutant.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                    str(work / "oracle.cpp"), "-o", str(lib)], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pid.py"),
                        os.path.join(ROOT, "tests", "test_oracle_vehicles.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutation {name!r}:\n{r.stdout[-2000:]}"
