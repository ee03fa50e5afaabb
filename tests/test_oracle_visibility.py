"""Pins of the oracle's visibility filter (Sec. 3.2 "Filtering"): the largest
ray weight T (1 - exp(-sigma delta)) per leaf, by closed forms and invariants."""
import math

import numpy as np

from paper_2103_14024_gb300 import synth as S


def _cam_through(eye, target, W=1, H=1):
    # a 1x1 camera whose single pixel ray passes through ``target``
    return S.make_cameras([S.look_at(eye, target)], W, H, 1.0)


def test_single_leaf_weight_closed_form(oracle_mod):
    D, h = 3, 2.0 / 8
    m = S.morton_encode(np.array([4]), np.array([4]), np.array([4]), D)
    sc = S.Scene(D, (-1.0, -1.0, -1.0), 2.0, 0, m, np.array([7.0], np.float32), np.zeros((1, 1, 3), np.float32))
    t = oracle_mod.build_sparse(sc)
    centre = np.array([-1 + 4.5 * h] * 3)
    cams = _cam_through(centre + np.array([0.0, 0.0, 3.0]), centre)
    w = oracle_mod.visibility(t, cams)
    assert w[0] == __import__("pytest").approx(1 - math.exp(-7.0 * h), abs=1e-12)


def test_occluded_leaf_weight(oracle_mod):
    # two voxels on one line of sight: the far one is seen through the near one
    D, h = 3, 2.0 / 8
    m = S.morton_encode(np.array([4, 4]), np.array([4, 4]), np.array([5, 4]), D)
    order = np.argsort(m)
    sig = np.array([3.0, 9.0], np.float32)[order]
    sc = S.Scene(D, (-1.0, -1.0, -1.0), 2.0, 0, m[order], sig, np.zeros((2, 1, 3), np.float32))
    t = oracle_mod.build_sparse(sc)
    x = -1 + 4.5 * h
    cams = _cam_through(np.array([x, x, 3.0]), np.array([x, x, 0.0]))     # looks down -z: z=5 first
    w = oracle_mod.visibility(t, cams)
    near, far = (0, 1) if m[order][0] == m[0] else (1, 0)
    a_near = 1 - math.exp(-3.0 * h)
    assert w[near] == __import__("pytest").approx(a_near, abs=1e-12)
    assert w[far] == __import__("pytest").approx((1 - a_near) * (1 - math.exp(-9.0 * h)), abs=1e-12)


def test_weights_bounded_and_unseen_zero(oracle_mod):
    sc = S.scene_random(3, 5, 1, p_occ=0.4, sigma_mu=2.0)
    t = oracle_mod.build_sparse(sc)
    cams = S.make_cameras(S.orbit_c2ws(6, radius=3.0), 24, 24, 20.0)
    w = oracle_mod.visibility(t, cams)
    assert np.all(w >= 0) and np.all(w <= 1)
    # a leaf is seen iff some ray composites it (the render's touched set)
    seen = np.zeros(sc.n, bool)
    for c in cams:
        seen |= oracle_mod.render_cams(t, c[None], want_touched=True)["touched"].astype(bool)
    assert np.array_equal(w > 0, seen)
    # early stop can only lower weights (later segments are never composited)
    assert np.all(oracle_mod.visibility(t, cams, gamma=0.05) <= w + 1e-15)


def test_prune_keeps_renders_of_the_filter_views(oracle_mod):
    sc = S.scene_random(4, 5, 1, p_occ=0.4, sigma_mu=2.0)
    t = oracle_mod.build_sparse(sc)
    cams = S.make_cameras(S.orbit_c2ws(4, radius=3.0), 20, 20, 18.0)
    w = oracle_mod.visibility(t, cams)
    small = oracle_mod.prune(sc, w, 1e-300)        # drop only leaves no ray composites
    assert 0 < small.n < sc.n
    tp = oracle_mod.build_sparse(small)
    a = oracle_mod.render_cams(t, cams)["rgb"]
    b = oracle_mod.render_cams(tp, cams)["rgb"]
    assert np.abs(a - b).max() <= 1e-12
