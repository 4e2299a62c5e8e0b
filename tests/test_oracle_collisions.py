"""Pins of the checker's collision test (CPU only).

The checker decides, by brute force over all pairs, which live agents are
closer than the sum of their radii (Sec. III-A: colliding agents are marked
dead and excluded).  It is pinned to scipy's KD-tree pair search, to hand-made
cases at and around the threshold, and to its own subset mode.
"""
import numpy as np
from scipy.spatial import cKDTree

from paper_2308_12698_b300 import workload as W


def test_matches_kdtree_pair_search(orc):
    rng = np.random.default_rng(3)
    p = rng.uniform(0, 20, (4000, 3)).astype(np.float32)
    r = np.full(4000, 0.225, np.float32)
    got = orc.collisions(p, r, np.ones(4000))
    pairs = cKDTree(p.astype(np.float64)).query_pairs(0.45, output_type="ndarray")
    d = np.linalg.norm(p[pairs[:, 0]].astype(np.float64) - p[pairs[:, 1]], axis=1)
    # pairs within 1e-6 of the threshold may round either way in FP32; there are none here
    assert np.all(np.abs(d - 0.45) > 1e-6)
    ref = np.zeros(4000, np.uint8)
    ref[pairs.ravel()] = 1
    assert got.sum() > 50
    np.testing.assert_array_equal(got, ref)


def test_hand_cases(orc):
    r = np.float32(0.25)
    p = np.array([[0, 0, 0], [0.5, 0, 0],          # exactly r_i + r_j apart: not a collision (strict <)
                  [10, 0, 0], [10.49, 0, 0],       # just inside
                  [20, 0, 0], [20, 0.3, 0.4],      # 0.5 apart along a diagonal: not a collision
                  [30, 0, 0]], np.float32)         # alone
    got = orc.collisions(p, np.full(7, r), np.ones(7))
    np.testing.assert_array_equal(got, [0, 0, 1, 1, 0, 0, 0])


def test_unequal_radii_and_dead_agents(orc):
    p = np.array([[0, 0, 0], [0.7, 0, 0], [5, 0, 0], [5.2, 0, 0], [9, 0, 0], [9, 0.1, 0]], np.float32)
    r = np.array([0.5, 0.3, 0.1, 0.05, 0.2, 0.2], np.float32)
    alive = np.array([1, 1, 1, 1, 1, 0], np.uint8)
    # 0.7 < 0.8; 0.2 > 0.15; agent 5 is dead, so agent 4 has nobody to hit and 5 is not marked
    np.testing.assert_array_equal(orc.collisions(p, r, alive), [1, 1, 0, 0, 0, 0])


def test_subset_mode_equals_full(orc):
    wl = W.collision_field(3000)
    r = np.full(wl.n, wl.groups[0]["L"], np.float32)
    full = orc.collisions(wl.x0[:, 0:3], r, np.ones(wl.n))
    idx = np.random.default_rng(1).choice(wl.n, 300, replace=False)
    np.testing.assert_array_equal(orc.collisions(wl.x0[:, 0:3], r, np.ones(wl.n), idx=idx), full[idx])
    assert 0 < full.sum() < wl.n
