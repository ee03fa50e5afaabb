"""Pins of the oracle's renderer: ray/voxel intersection (Sec. 3.2
"Rendering") against brute force, compositing (Eq. 1, background term of
App. B.3.2) against closed forms, invariants and a dense fine-step marcher."""
import math

import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))
C1 = math.sqrt(3.0 / (4.0 * math.pi))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _slab(o, d, lo, hi):
    """[t_in, t_out) of the ray o + t d inside the half-open box [lo, hi) (fp64)."""
    tin, tout = -math.inf, math.inf
    for a in range(3):
        if d[a] == 0.0:
            if o[a] < lo[a] or o[a] >= hi[a]:
                return math.inf, -math.inf
        else:
            t0 = (lo[a] - o[a]) / d[a]
            t1 = (hi[a] - o[a]) / d[a]
            tin, tout = max(tin, min(t0, t1)), min(tout, max(t0, t1))
    return tin, tout


def _bruteforce_segments(sc, o, d, near=0.0, far=1e30):
    """Slab-intersect every kept voxel; sort by entry."""
    o = o.astype(np.float64)
    d = d.astype(np.float64)
    ln = float(np.linalg.norm(d))
    h = sc.bbox_size / sc.res
    lo = np.array(sc.bbox_lo, dtype=np.float64)
    btin, btout = _slab(o, d, lo, lo + sc.bbox_size)
    tn, tf = max(near / ln, btin), min(far / ln, btout)
    x, y, z = S.morton_decode(sc.morton, sc.depth)
    segs = []
    for i in range(sc.n):
        vlo = lo + np.array([x[i], y[i], z[i]], dtype=np.float64) * h
        a, b = _slab(o, d, vlo, vlo + h)
        a, b = max(a, tn), min(b, tf)
        if b - a > 1e-12:
            segs.append((a, i, b))
    segs.sort()
    return segs


@pytest.mark.parametrize("seed,D", [(1, 2), (2, 3), (3, 4), (4, 5)])
def test_traversal_equals_bruteforce(oracle_mod, seed, D):
    sc = S.scene_random(seed, D, 0, p_occ=0.35)
    t = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(seed + 100, 60, radius=3.0, spread=0.9)
    for r in range(o.shape[0]):
        leaf, t0, t1, dl = oracle_mod.trace_ray(t, o[r], d[r])
        keep = (leaf >= 0) & (t1 - t0 > 1e-12)
        bf = _bruteforce_segments(sc, o[r], d[r])
        assert [s[1] for s in bf] == list(leaf[keep])
        if bf:
            assert np.allclose([s[0] for s in bf], t0[keep], atol=1e-12)
            assert np.allclose([s[2] for s in bf], t1[keep], atol=1e-12)
        # segments tile [t_in, t_out] contiguously; delta = world length
        if leaf.size:
            assert np.all(t1[:-1] <= t0[1:] + 1e-15) and np.all(t0[1:] - t1[:-1] < 1e-12)
            assert np.allclose(dl, (t1 - t0) * np.linalg.norm(d[r].astype(np.float64)), rtol=1e-14)


def test_traversal_degenerate_rays_on_faces(oracle_mod):
    # rays parallel to axes lying exactly on voxel faces / edges
    sc = S.scene_random(7, 4, 0, p_occ=0.4)
    t = oracle_mod.build_sparse(sc)
    h = np.float32(sc.bbox_size / sc.res)
    lo = np.float32(sc.bbox_lo[0])
    rays = []
    for k in range(0, 17, 3):
        for j in range(0, 17, 5):
            on_k, on_j = lo + np.float32(k) * h, lo + np.float32(j) * h
            rays.append(((on_k, on_j, 3.0), (0.0, 0.0, -1.0)))
            rays.append(((on_k, 3.0, on_j), (0.0, -1.0, 0.0)))
            rays.append(((-3.0, on_k, on_j + np.float32(0.3) * h), (1.0, 0.0, 0.0)))
            rays.append(((on_k, -3.0, -3.0), (0.0, 1.0, 1.0)))    # diagonal in a face plane
            rays.append(((-3.0, -3.0, -3.0 + float(on_k) + 1.0), (1.0, 1.0, 1.0)))
    for o, d in rays:
        o = np.array(o, np.float32)
        d = np.array(d, np.float32)
        leaf, t0, t1, dl = oracle_mod.trace_ray(t, o, d)
        keep = (leaf >= 0) & (t1 - t0 > 1e-12)
        bf = _bruteforce_segments(sc, o, d)
        assert [s[1] for s in bf] == list(leaf[keep]), (o, d)


def _single_voxel_scene(D, xyz, sigma, sh, lo=(-1.0, -1.0, -1.0), size=2.0):
    m = S.morton_encode(*[np.array([v]) for v in xyz], D)
    sh = np.asarray(sh, np.float32).reshape(1, -1, 3)
    deg = int(math.isqrt(sh.shape[1])) - 1
    return S.Scene(D, lo, size, deg, m, np.array([sigma], np.float32), sh)


def test_single_leaf_closed_forms(oracle_mod):
    D = 3
    h = 2.0 / 8
    k0 = np.array([[0.7, -1.1, 0.3]], np.float32)
    sc = _single_voxel_scene(D, (3, 4, 5), 5.5, k0)
    t = oracle_mod.build_sparse(sc)
    c = sigmoid(k0[0].astype(np.float64) * Y00)
    centre = np.array([-1 + 3.5 * h, -1 + 4.5 * h, -1 + 5.5 * h])
    # axis-aligned through the centre: chord = h
    o = np.array([[centre[0], centre[1], 5.0]], np.float32)
    d = np.array([[0, 0, -2.0]], np.float32)
    r = oracle_mod.render_rays(t, o, d)["rgb"][0]
    assert np.allclose(r, c * (1 - math.exp(-5.5 * h)), atol=1e-14)
    # main diagonal through the centre (passes exactly through two corners): chord = h sqrt 3
    o = (centre - 3.0).astype(np.float32)[None]
    d = np.array([[1.0, 1.0, 1.0]], np.float32)
    r = oracle_mod.render_rays(t, o, d)["rgb"][0]
    assert np.allclose(r, c * (1 - math.exp(-5.5 * h * math.sqrt(3))), atol=1e-14)
    # generic rays: analytic chord by the slab formula
    o, d = S.random_rays(3, 200, radius=3.0, spread=0.2)
    res = oracle_mod.render_rays(t, o, d)["rgb"]
    vlo = np.array([-1 + 3 * h, -1 + 4 * h, -1 + 5 * h])
    for i in range(o.shape[0]):
        a, b = _slab(o[i].astype(np.float64), d[i].astype(np.float64), vlo, vlo + h)
        L = max(0.0, b - a) * float(np.linalg.norm(d[i].astype(np.float64)))
        assert np.allclose(res[i], c * (1 - math.exp(-5.5 * L)), atol=1e-13)


def test_two_leaf_closed_form(oracle_mod):
    D = 3
    h = 2.0 / 8
    m = S.morton_encode(np.array([2, 3]), np.array([4, 4]), np.array([4, 4]), D)
    k = np.array([[[0.4, 1.2, -0.8]], [[-1.5, 0.1, 2.0]]], np.float32)
    sig = np.array([3.0, 9.0], np.float32)
    sc = S.Scene(D, (-1.0, -1.0, -1.0), 2.0, 0, m, sig, k)
    t = oracle_mod.build_sparse(sc)
    o = np.array([[-4.0, -1 + 4.5 * h, -1 + 4.5 * h]], np.float32)
    d = np.array([[1.0, 0, 0]], np.float32)
    for bg in ((0.0, 0.0, 0.0), (1.0, 0.5, 0.25)):
        r = oracle_mod.render_rays(t, o, d, bg=bg)
        c1 = sigmoid(k[0, 0].astype(np.float64) * Y00)
        c2 = sigmoid(k[1, 0].astype(np.float64) * Y00)
        a1, a2 = 1 - math.exp(-3.0 * h), 1 - math.exp(-9.0 * h)
        exp = c1 * a1 + (1 - a1) * c2 * a2 + (1 - a1) * (1 - a2) * np.array(bg)
        assert np.allclose(r["rgb"][0], exp, atol=1e-14)
        assert r["t_final"][0] == pytest.approx((1 - a1) * (1 - a2), abs=1e-15)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6])
def test_uniform_full_tree_independent_of_depth(oracle_mod, D):
    k = np.array([[0.9, -0.4, 0.1]], np.float32)
    sig = 1.7
    sc = S.scene_uniform(D, sig, k)
    t = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(40 + D, 300, radius=2.5, spread=1.2)
    res = oracle_mod.render_rays(t, o, d, near=0.3, far=5.0)["rgb"]
    c = sigmoid(k[0].astype(np.float64) * Y00)
    for i in range(o.shape[0]):
        od, dd = o[i].astype(np.float64), d[i].astype(np.float64)
        ln = float(np.linalg.norm(dd))
        a, b = _slab(od, dd, np.full(3, -1.0), np.full(3, 1.0))
        a, b = max(a, 0.3 / ln), min(b, 5.0 / ln)
        L = max(0.0, b - a) * ln
        assert np.allclose(res[i], c * (1 - math.exp(-sig * L)), atol=1e-12)


def test_degree0_opaque_gives_sigmoid(oracle_mod):
    sc = S.scene_tiny().replace(sigma=np.full(S.scene_tiny().n, 1e6, np.float32))
    t = oracle_mod.build_sparse(sc)
    cams = S.cameras_tiny("generic")
    r = oracle_mod.render_cams(t, cams)
    hit = r["t_final"][0] < 0.5
    assert hit.sum() > 100
    o, d = oracle_mod.cam_rays(cams)
    first = np.array([oracle_mod.trace_ray(t, o[i], d[i])[0] for i in np.flatnonzero(hit.ravel())],
                     dtype=object)
    rgb = r["rgb"][0].reshape(-1, 3)[hit.ravel()]
    for j, segs in enumerate(first):
        lf = segs[segs >= 0][0]
        assert np.allclose(rgb[j], sigmoid(sc.sh[lf, 0].astype(np.float64) * Y00), atol=1e-12)


def test_weights_sum_and_background(oracle_mod):
    sc = S.scene_random(5, 4, 2, p_occ=0.4)
    sc0 = sc.replace(sh=np.zeros_like(sc.sh))                 # every colour = sigmoid(0) = 1/2
    t = oracle_mod.build_sparse(sc0)
    o, d = S.random_rays(8, 500, radius=3.0, spread=1.5)
    r0 = oracle_mod.render_rays(t, o, d, bg=(0, 0, 0))
    r1 = oracle_mod.render_rays(t, o, d, bg=(1, 1, 1))
    sw = 2.0 * r0["rgb"][:, 0]
    TN = r1["rgb"][:, 0] - r0["rgb"][:, 0]
    assert np.all(sw <= 1 + 1e-12) and np.all(sw >= 0)
    assert np.allclose(sw + TN, 1.0, atol=1e-12)
    assert np.allclose(TN, r0["t_final"], atol=1e-12)
    # rays that miss the box return the background exactly
    om = np.array([[5.0, 5.0, 5.0]] * 3, np.float32)
    dm = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.2], [1.0, 1.0, 1.0]], np.float32)
    rm = oracle_mod.render_rays(t, om, dm, bg=(0.2, 0.3, 0.4))
    assert np.array_equal(rm["rgb"], np.tile([0.2, 0.3, 0.4], (3, 1)))
    assert np.all(rm["t_final"] == 1.0)


def test_early_stop(oracle_mod):
    sc = S.scene_random(6, 4, 1, p_occ=0.6, sigma_mu=2.5)
    t = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(9, 400, radius=3.0, spread=0.5)
    full = oracle_mod.render_rays(t, o, d)
    g = 0.05
    st = oracle_mod.render_rays(t, o, d, gamma=g)
    # stopped rays end just below gamma; the colour differs by at most T_stop * max|c - bg|
    stopped = st["n_seg"] < full["n_seg"]
    assert stopped.any()
    assert np.all(st["t_final"][stopped] < g)
    assert np.all(np.abs(st["rgb"] - full["rgb"]).max(axis=1) <= st["t_final"] + 1e-12)
    assert np.array_equal(st["rgb"][~stopped], full["rgb"][~stopped])


def test_axis_permutation_symmetry(oracle_mod):
    sc = S.scene_random(15, 4, 0, p_occ=0.4)
    x, y, z = S.morton_decode(sc.morton, sc.depth)
    m2 = S.morton_encode(y, x, z, sc.depth)
    order = np.argsort(m2)
    sc2 = sc.replace(morton=m2[order], sigma=sc.sigma[order], sh=sc.sh[order])
    t1, t2 = oracle_mod.build_sparse(sc), oracle_mod.build_sparse(sc2)
    o, d = S.random_rays(10, 400, radius=3.0, spread=1.0)
    r1 = oracle_mod.render_rays(t1, o, d)["rgb"]
    r2 = oracle_mod.render_rays(t2, o[:, [1, 0, 2]], d[:, [1, 0, 2]])["rgb"]
    assert np.allclose(r1, r2, atol=1e-13)


def test_dense_fine_step_marcher_converges(oracle_mod):
    # Piecewise-constant field sampled at N midpoints per ray (SH degree 2 in
    # its Cartesian form): the quadrature error is O(sigma * step) at each
    # boundary a sample straddles, so it must shrink about as 1 / N.
    sc = S.scene_random(16, 3, 2, p_occ=0.4, sigma_mu=0.5, sigma_s=0.5)
    t = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(11, 25, radius=3.0, spread=0.7)
    ref = oracle_mod.render_rays(t, o, d)["rgb"]
    R, h = sc.res, sc.bbox_size / sc.res
    lo = np.array(sc.bbox_lo)
    dense = -np.ones((R, R, R), dtype=np.int64)
    x, y, z = S.morton_decode(sc.morton, sc.depth)
    dense[x, y, z] = np.arange(sc.n)
    c2 = 0.5 * math.sqrt(15.0 / math.pi)

    def march(i, N):
        od, dd = o[i].astype(np.float64), d[i].astype(np.float64)
        ln = float(np.linalg.norm(dd))
        ux, uy, uz = dd / ln
        Y = np.array([Y00, C1 * uy, C1 * uz, C1 * ux,
                      c2 * ux * uy, c2 * uy * uz, 0.25 * math.sqrt(5.0 / math.pi) * (3 * uz * uz - 1),
                      c2 * ux * uz, 0.25 * math.sqrt(15.0 / math.pi) * (ux * ux - uy * uy)])
        a, b = _slab(od, dd, lo, lo + sc.bbox_size)
        if not a < b:
            return np.zeros(3)
        ts = a + (np.arange(N) + 0.5) * (b - a) / N
        p = od[None] + ts[:, None] * dd[None]
        q = np.clip(np.floor((p - lo) / h).astype(int), 0, R - 1)
        lf = dense[q[:, 0], q[:, 1], q[:, 2]]
        sig = np.where(lf >= 0, sc.sigma[np.maximum(lf, 0)].astype(np.float64), 0.0)
        col = sigmoid(np.einsum("nkc,k->nc", sc.sh[np.maximum(lf, 0)].astype(np.float64), Y))
        x_ = sig * (b - a) / N * ln
        T = np.exp(-np.concatenate([[0.0], np.cumsum(x_)[:-1]]))
        return ((T * (1 - np.exp(-x_)))[:, None] * col).sum(axis=0)

    e1 = np.array([np.abs(march(i, 4000) - ref[i]).max() for i in range(o.shape[0])])
    e2 = np.array([np.abs(march(i, 64000) - ref[i]).max() for i in range(o.shape[0])])
    assert e2.max() <= 1e-4
    assert (e2 <= e1 + 1e-9).all()
    assert e1.sum() > 1e-4, "the rays must cross boundaries for the rate to mean anything"
    assert e2.sum() <= e1.sum() / 8.0  # 16 times the samples: about 16 times smaller


def test_camera_ray_fp32_expression(oracle_mod):
    cams = np.concatenate([S.cameras_tiny("generic"), S.cameras_tiny("axis")])
    o, d = oracle_mod.cam_rays(cams)
    f = np.float32
    k = 0
    for c in cams:
        W, H = int(c["width"]), int(c["height"])
        j, i = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        xc = ((i.astype(f) + f(0.5)) - c["cx"]) / c["fx"]
        yc = -(((j.astype(f) + f(0.5)) - c["cy"]) / c["fy"])
        M = c["c2w"]
        for r in range(3):
            dr = ((M[r, 0] * xc) + (M[r, 1] * yc)) - M[r, 2]
            assert np.array_equal(d[k:k + W * H, r], dr.ravel().astype(f))
            assert np.all(o[k:k + W * H, r] == M[r, 3])
        # the central rays look at the origin
        k += W * H


def test_camera_rays_project_back_to_their_pixels(oracle_mod):
    """Pinhole geometry of the camera rays (reading R2: looks along its -z
    axis, image rows grow downwards): a point on the ray of pixel (i, j),
    taken into the camera frame with the inverse of the camera's rotation and
    projected with the focal lengths and principal point, lands on the pixel
    centre (i + 0.5, j + 0.5); the ray of the principal point is the camera's
    -z axis; the orbit cameras' central rays pass through the origin."""
    for cams in (S.cameras_tiny("generic"), S.cameras_main(3), S.cameras_train(n=3)):
        o, d = oracle_mod.cam_rays(cams)
        k = 0
        for c in cams:
            W, H = int(c["width"]), int(c["height"])
            M = c["c2w"].astype(np.float64)
            R, ctr = M[:, :3], M[:, 3]
            assert np.allclose(R.T @ R, np.eye(3), atol=1e-6)           # a rotation
            j, i = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
            oo, dd = o[k:k + W * H].astype(np.float64), d[k:k + W * H].astype(np.float64)
            assert np.allclose(oo, ctr)
            q = (dd * 3.0) @ R                                            # R^T (p - centre), p = o + 3 d
            u = c["cx"] + c["fx"] * q[:, 0] / -q[:, 2]
            v = c["cy"] - c["fy"] * q[:, 1] / -q[:, 2]
            assert np.all(q[:, 2] < 0)                                    # in front of the camera
            assert np.abs(u - (i.ravel() + 0.5)).max() < 1e-3
            assert np.abs(v - (j.ravel() + 0.5)).max() < 1e-3
            k += W * H
        # the ray through the principal point is the -z axis of the camera
        c = cams[0]
        cam1 = c.copy()
        cam1["cx"], cam1["cy"] = 0.5, 0.5                                 # pixel (0, 0) at the principal point
        _, d0 = oracle_mod.cam_rays(np.array([cam1]))
        assert np.allclose(d0[0], -c["c2w"][:, 2], atol=1e-7)
    # orbit cameras look at the origin: the central pixel's ray passes it closely
    for cams in (S.cameras_main(4), S.cameras_train(n=4)):
        o, d = oracle_mod.cam_rays(cams)
        n = int(cams[0]["width"]) * int(cams[0]["height"])
        for v_ in range(len(cams)):
            W, H = int(cams[v_]["width"]), int(cams[v_]["height"])
            r = v_ * n + (H // 2) * W + W // 2
            oo, dd = o[r].astype(np.float64), d[r].astype(np.float64)
            dd /= np.linalg.norm(dd)
            miss = np.linalg.norm(np.cross(-oo, dd))                      # distance of the origin from the ray
            assert miss < 4.0 / min(float(cams[v_]["fx"]), float(cams[v_]["fy"])) * 1.5


def test_render_cams_equals_render_rays(oracle_mod):
    sc = S.scene_tiny()
    t = oracle_mod.build_sparse(sc)
    cams = S.cameras_tiny("axis")
    r = oracle_mod.render_cams(t, cams, bg=(0.1, 0.2, 0.3))
    o, d = oracle_mod.cam_rays(cams)
    rr = oracle_mod.render_rays(t, o, d, near=float(cams[0]["near"]), far=float(cams[0]["far"]),
                                bg=(0.1, 0.2, 0.3))
    assert np.array_equal(r["rgb"].reshape(-1, 3), rr["rgb"])
    idx = np.array([5, 100, 2000, 4095])
    rp = oracle_mod.render_pixels(t, cams, np.zeros(4), idx % 64, idx // 64, bg=(0.1, 0.2, 0.3))
    assert np.array_equal(rp["rgb"], rr["rgb"][idx])
