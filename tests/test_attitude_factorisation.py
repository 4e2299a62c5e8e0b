"""The device controller forms the desired attitude's quaternion without the matrix: in the
heading frame the desired body z axis (A, B, F_z)/|F| equals Rx(phi) Ry(theta) e3, so
R_des = Rz(psi) Rx(phi) Ry(theta), and q_d is the product of the three half-angle quaternions,
each taken from an unnormalised (cos, sin) pair and normalised once at the end.

These CPU tests check that construction, restated in FP64 numpy, against the definition of
R_des (body z along the force, body y = z x (cos psi, sin psi, 0) normalised, x = y x z) and
against the checker's Shepperd conversion of that matrix, over all headings, both signs of
F_z and near-vertical and near-horizontal forces.  The GPU parity tests then hold the kernel to
the checker.
"""
import numpy as np

import oracle


def half_angle_qd(F, psi):
    c, s, c2, s2 = np.cos(psi), np.sin(psi), np.cos(psi / 2), np.sin(psi / 2)
    A = c * F[0] + s * F[1]
    B = c * F[1] - s * F[0]
    N = np.sqrt(B * B + F[2] * F[2])
    M = np.sqrt(A * A + N * N)
    X = (N + F[2], -B) if F[2] >= 0 else (-B, N - F[2])
    Y = (M + N, A)
    P = np.array([X[0] * Y[0], X[1] * Y[0], X[0] * Y[1], X[1] * Y[1]])
    Q = np.array([c2 * P[0] - s2 * P[3], c2 * P[1] - s2 * P[2], c2 * P[2] + s2 * P[1], c2 * P[3] + s2 * P[0]])
    return Q / np.linalg.norm(Q)


def rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def r_des(F, psi):
    zd = F / np.linalg.norm(F)
    yd = np.cross(zd, [np.cos(psi), np.sin(psi), 0.0])
    yd /= np.linalg.norm(yd)
    return np.stack([np.cross(yd, zd), yd, zd], axis=1)


def forces(rng, n):
    F = rng.normal(size=(n, 3)) * rng.choice([0.1, 1.0, 30.0], size=(n, 1))
    F[: n // 4, 2] = -np.abs(F[: n // 4, 2])                  # pointing down
    F[n // 4: n // 2, 2] = np.abs(F[n // 4: n // 2, 2]) + 9.81  # hover-like
    F[n // 2: n // 2 + 50, 0:2] *= 1e-6                        # near vertical, up
    F[n // 2 + 50: n // 2 + 100, 0:2] *= 1e-6
    F[n // 2 + 50: n // 2 + 100, 2] = -np.abs(F[n // 2 + 50: n // 2 + 100, 2])  # near vertical, down
    F[n // 2 + 100: n // 2 + 150, 2] *= 1e-6                   # near horizontal
    return F


def test_half_angle_quaternion_is_the_desired_rotation():
    rng = np.random.default_rng(5)
    F = forces(rng, 4000)
    psi = rng.uniform(-np.pi, np.pi, len(F))
    for f, p in zip(F, psi):
        np.testing.assert_allclose(rot(half_angle_qd(f, p)), r_des(f, p), atol=1e-12)


def test_half_angle_quaternion_matches_shepperd_up_to_sign():
    rng = np.random.default_rng(6)
    F = forces(rng, 2000)
    psi = rng.uniform(-np.pi, np.pi, len(F))
    for f, p in zip(F, psi):
        a = half_angle_qd(f, p)
        b = oracle.shepperd(r_des(f, p))
        assert min(np.abs(a - b).max(), np.abs(a + b).max()) < 1e-12, (f, p, a, b)
