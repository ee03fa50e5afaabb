"""Cell index (per-voxel leaf / empty box, the library's replacement for the
child-array descent when locating cells), in its dense and brick layouts: the
entries against their definition from the occupied voxels alone, and renders,
counts, gradients, visibility weights and batched renders bit-identical with
either layout and without an index."""
import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pot():
    import torch
    assert torch.cuda.is_available()
    import paper_2103_14024_gb300 as P
    P.lib()
    return P


CUBE_MAX = 63   # largest cube half-extent the index records


def _expected_index(sc, cubes=True):
    """Entry of every voxel [x][y][z] from the occupied Morton codes: the leaf
    rank; for an empty voxel, with l the coarsest level whose block around the
    voxel holds no occupied voxel (the empty child of an existing node) and
    dist its Chebyshev distance to the nearest occupied voxel (scipy, capped
    at CUBE_MAX + 1): the cube code -(3 + 2e), e = dist - 1, if 2e + 2 > 2^(D-l),
    else the node code -(2 + 2l)."""
    from scipy import ndimage
    D, R = sc.depth, 1 << sc.depth
    g = np.arange(R, dtype=np.uint64)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    m = S.morton_encode(x.ravel(), y.ravel(), z.ravel(), D).astype(np.uint64)
    occ = np.sort(sc.morton.astype(np.uint64))
    out = np.zeros(m.shape, np.int64)
    level = np.full(m.shape, -1, np.int64)
    for l in range(1, D + 1):
        sh = np.uint64(3 * (D - l))
        inside = np.isin(m >> sh, np.unique(occ >> sh))
        level[(level < 0) & ~inside] = l
    empty = level > 0
    out[~empty] = np.searchsorted(occ, m[~empty])
    grid_empty = empty.reshape(R, R, R)
    if grid_empty.all():
        dist = np.full(grid_empty.shape, CUBE_MAX + 1)
    else:
        dist = np.minimum(ndimage.distance_transform_cdt(grid_empty, metric="chessboard"), CUBE_MAX + 1)
    e = dist.ravel()[empty] - 1
    lv = level[empty]
    cube = (2 * e + 2 > (1 << (D - lv))) & cubes
    out[empty] = np.where(cube, -(3 + 2 * e), -(2 + 2 * lv))
    return out.reshape(R, R, R).astype(np.int32)


def _expected_brick_index(sc):
    """Entry of every voxel in the brick layout: inside a 4^3 brick that holds an
    occupied voxel, the leaf rank or the node code of the voxel's empty node
    (level D-1 or D; no cubes there);
    for every voxel of a brick without one, the brick's code: with l the coarsest
    level whose block around the brick is empty and db the brick's Chebyshev
    distance in bricks to the nearest brick holding an occupied voxel (capped at
    CUBE_MAX + 1), the cube -(3 + 2e), e = min(4 (db - 1), CUBE_MAX), if
    2e + 2 > 2^(D-l), else the node -(2 + 2l)."""
    from scipy import ndimage
    D, R = sc.depth, 1 << sc.depth
    dense = _expected_index(sc, cubes=False)
    B = R // 4
    x, y, z = (a.astype(np.int64) for a in S.morton_decode(sc.morton, D))
    held = np.zeros((B, B, B), bool)
    held[x // 4, y // 4, z // 4] = True
    if held.any():
        db = np.minimum(ndimage.distance_transform_cdt(~held, metric="chessboard"), CUBE_MAX + 1)
    else:
        db = np.full(held.shape, CUBE_MAX + 1)
    occ_b = np.unique(sc.morton.astype(np.uint64) >> np.uint64(6))      # Morton codes of held bricks
    g = np.arange(B, dtype=np.uint64)
    bx, by, bz = np.meshgrid(g, g, g, indexing="ij")
    mb = S.morton_encode(bx.ravel(), by.ravel(), bz.ravel(), D - 2).astype(np.uint64)
    level = np.full(mb.shape, -1, np.int64)
    for l in range(1, D - 1):
        sh = np.uint64(3 * (D - 2 - l))
        inside = np.isin(mb >> sh, np.unique(occ_b >> sh))
        level[(level < 0) & ~inside] = l
    level = level.reshape(B, B, B)
    e = np.minimum(4 * (db - 1), CUBE_MAX)
    code = np.where(2 * e + 2 > (1 << (D - np.maximum(level, 0))), -(3 + 2 * e), -(2 + 2 * level))
    out = np.repeat(np.repeat(np.repeat(code, 4, 0), 4, 1), 4, 2).astype(np.int32)
    keep = np.repeat(np.repeat(np.repeat(held, 4, 0), 4, 1), 4, 2)
    out[keep] = dense[keep]
    return out


@pytest.mark.parametrize("seed,D,p_occ", [(81, 3, 0.2), (82, 4, 0.05), (83, 5, 0.3), (84, 6, 0.02),
                                          (85, 7, 0.01), (86, 8, 0.002), (80, 7, 0.0)])
def test_brick_index_entries_match_definition(pot, seed, D, p_occ):
    sc = S.scene_random(seed, D, 1, p_occ=p_occ)
    if p_occ == 0.0:   # one occupied voxel in a corner: distances past the cap
        sc = S.scene_random(seed, D, 1, p_occ=0.01)
        keep = np.argmin(sc.morton)
        sc = sc.replace(morton=sc.morton[keep:keep + 1], sigma=sc.sigma[keep:keep + 1], sh=sc.sh[keep:keep + 1])
    t = pot.Tree.from_scene(sc)
    t.set_cell_index("brick")
    info = t.info()
    held = np.unique(sc.morton.astype(np.uint64) >> np.uint64(6)).shape[0]
    assert info["index_kind"] == 3 and info["index_bytes"] == 4 * (8 ** (D - 2) + 64 * held)
    assert np.array_equal(t.export_cell_index(), _expected_brick_index(sc))


@pytest.mark.parametrize("seed,D,p_occ", [(81, 1, 0.5), (82, 2, 0.3), (83, 3, 0.2), (84, 4, 0.05),
                                          (85, 5, 0.3), (86, 6, 0.02), (87, 7, 0.01), (80, 7, 0.0)])
def test_index_entries_match_definition(pot, seed, D, p_occ):
    sc = S.scene_random(seed, D, 1, p_occ=p_occ)
    if p_occ == 0.0:   # one occupied voxel in a corner: distances past the cap
        sc = S.scene_random(seed, D, 1, p_occ=0.01)
        keep = np.argmin(sc.morton)
        sc = sc.replace(morton=sc.morton[keep:keep + 1], sigma=sc.sigma[keep:keep + 1], sh=sc.sh[keep:keep + 1])
    t = pot.Tree.from_scene(sc)
    info = t.info()
    assert info["index_kind"] == 2 and info["index_bytes"] == 4 * max(64, 8 ** D)
    assert np.array_equal(t.export_cell_index(), _expected_index(sc))


def test_index_depth_10(pot, oracle_mod):
    """The largest indexed depth (1024^3 voxels, 4.3 GB): sampled entries against
    their definition (Chebyshev distance by brute force over the occupied voxels,
    node level from Morton prefixes), and renders through the tree against the
    oracle."""
    import torch
    D, R = 10, 1024
    rng = np.random.default_rng(10)
    # clusters of occupied voxels so that distances vary from 1 past the cap
    centres = rng.integers(40, R - 40, size=(40, 3))
    pts = (centres[:, None, :] + rng.integers(-6, 7, size=(40, 60, 3))).reshape(-1, 3)
    m = np.unique(S.morton_encode(pts[:, 0].astype(np.uint64), pts[:, 1].astype(np.uint64),
                                  pts[:, 2].astype(np.uint64), D))
    n = m.shape[0]
    sc = S.Scene(depth=D, bbox_lo=(-1.0, -1.0, -1.0), bbox_size=2.0, sh_degree=1, morton=m.astype(np.uint64),
                 sigma=rng.uniform(50.0, 400.0, n).astype(np.float32),
                 sh=rng.normal(size=(n, 4, 3)).astype(np.float32))
    t = pot.Tree.from_scene(sc)
    held = np.unique(sc.morton >> np.uint64(6)).shape[0]
    assert t.info()["index_kind"] == 3                     # depth 10: bricks by default
    assert t.info()["index_bytes"] == 4 * (8 ** (D - 2) + 64 * held)
    t.set_cell_index("dense")
    assert t.info()["index_kind"] == 2 and t.info()["index_bytes"] == 4 * 8 ** D
    idx = t.export_cell_index(device="cuda")
    x, y, z = (a.astype(np.int64) for a in S.morton_decode(sc.morton, D))
    occ = np.stack([x, y, z], 1)
    # sample voxels: near the clusters, and anywhere
    near = (occ[rng.integers(0, n, 3000)] + rng.integers(-70, 71, size=(3000, 3))).clip(0, R - 1)
    anyw = rng.integers(0, R, size=(1000, 3))
    q = np.concatenate([near, anyw])
    got = idx[torch.from_numpy(q[:, 0]).cuda(), torch.from_numpy(q[:, 1]).cuda(),
              torch.from_numpy(q[:, 2]).cuda()].cpu().numpy()
    mq = S.morton_encode(q[:, 0].astype(np.uint64), q[:, 1].astype(np.uint64), q[:, 2].astype(np.uint64), D)
    for k in range(q.shape[0]):
        pos = np.searchsorted(sc.morton, mq[k])
        if pos < n and sc.morton[pos] == mq[k]:
            assert got[k] == pos
            continue
        dist = min(int(np.abs(occ - q[k]).max(1).min()), CUBE_MAX + 1)
        level = next(l for l in range(1, D + 1)
                     if not np.any((sc.morton >> np.uint64(3 * (D - l))) == (mq[k] >> np.uint64(3 * (D - l)))))
        e = dist - 1
        want = -(3 + 2 * e) if 2 * e + 2 > (1 << (D - level)) else -(2 + 2 * level)
        assert got[k] == want, (q[k], got[k], want)
    del idx
    # rays aimed at occupied voxels, against the oracle
    h = 2.0 / R
    tgt = (-1.0 + (occ[rng.integers(0, n, 300)] + 0.5) * h).astype(np.float32)
    o = np.repeat(np.float32([[0.1, -3.5, 0.4]]), 300, axis=0)
    d = (tgt - o).astype(np.float32)
    og, dg = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    rgb = pot.render_rays(t, og, dg).cpu().numpy()
    ref = oracle_mod.render_rays(oracle_mod.build_sparse(sc), o, d)["rgb"]
    assert np.abs(rgb - ref).max() <= 1e-4
    t.set_cell_index("brick")
    assert np.array_equal(pot.render_rays(t, og, dg).cpu().numpy(), rgb)
    pot.check()


def test_index_empty_and_single_leaf_trees(pot):
    sc = S.scene_random(88, 4, 0, p_occ=0.3)
    for n in (0, 1):
        s = sc.replace(morton=sc.morton[:n], sigma=sc.sigma[:n], sh=sc.sh[:n])
        t = pot.Tree.from_scene(s)
        assert np.array_equal(t.export_cell_index(), _expected_index(s))
        t.set_cell_index("brick")
        assert np.array_equal(t.export_cell_index(), _expected_brick_index(s))


def test_index_toggle_and_limits(pot, oracle_mod):
    sc = S.scene_random(89, 5, 2, p_occ=0.3)
    t = pot.Tree.from_scene(sc)
    full = t.info()
    t.set_cell_index(False)
    t.set_cell_index(False)                       # idempotent
    off = t.info()
    assert off["index_bytes"] == 0 and off["bytes"] == full["bytes"] - full["index_bytes"]
    with pytest.raises(pot.PotError) as e:
        t.export_cell_index()
    assert e.value.status == pot.POT_ERR_INVALID_ARG
    t.set_cell_index(True)
    assert t.info() == full
    t.set_cell_index("brick")
    assert t.info()["index_kind"] == 3 and 0 < t.info()["index_bytes"]
    t.set_cell_index("dense")
    assert t.info() == full
    assert pot.lib().pot_tree_set_cell_index(t.handle, 4, None) == pot.POT_ERR_INVALID_ARG
    import torch
    for D, kind in ((11, 3), (12, 0)):
        # depth 11: a brick index (the dense one would take 4 * 8^11 bytes);
        # depth 12: none, cells found by the descent
        R = 1 << D
        m = S.morton_encode(np.array([5, 1000, R - 1], np.uint64), np.array([7, 3, R - 1], np.uint64),
                            np.array([9, 1500, 0], np.uint64), D)
        order = np.argsort(m)
        deep = S.Scene(depth=D, bbox_lo=(-1.0, -1.0, -1.0), bbox_size=2.0, sh_degree=0,
                       morton=m[order].astype(np.uint64), sigma=np.float32([5000.0, 6000.0, 7000.0]),
                       sh=np.zeros((3, 1, 3), np.float32))
        td = pot.Tree.from_scene(deep)
        info = td.info()
        assert info["index_kind"] == kind
        assert info["index_bytes"] == (4 * (8 ** (D - 2) + 64 * 3) if kind else 0)
        with pytest.raises(pot.PotError) as e:
            td.set_cell_index("dense")
        assert e.value.status == pot.POT_ERR_UNSUPPORTED
        if kind == 0:
            with pytest.raises(pot.PotError) as e:
                td.set_cell_index(True)
            assert e.value.status == pot.POT_ERR_UNSUPPORTED
        # rays aimed at the three leaves
        h = 2.0 / R
        vox = np.array([[5, 7, 9], [1000, 3, 1500], [R - 1, R - 1, 0]], np.float64)
        centres = (-1.0 + (vox + 0.5) * h).astype(np.float32)
        o = np.repeat(centres + np.float32([0.0, 0.0, 3.0]), 11, axis=0)
        jitter = (S.uniform(5, 1, np.arange(33 * 2, dtype=np.uint64)).reshape(33, 2) - 0.5) * 4e-4 * (2048 / R)
        d = np.concatenate([jitter, -np.ones((33, 1))], 1).astype(np.float32)
        og, dg = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
        rgb = pot.render_rays(td, og, dg).cpu().numpy()
        ref = oracle_mod.render_rays(oracle_mod.build_sparse(deep), o, d)["rgb"]
        assert np.abs(rgb - ref).max() <= 1e-4
        assert float(ref.max()) > 0.1
        if kind:
            td.set_cell_index(False)
            assert np.array_equal(pot.render_rays(td, og, dg).cpu().numpy(), rgb)
        td.free()
    pot.check()


def _both(pot, t, fn):
    """fn(tree) with its default cell index, without one, and (depth >= 3) with
    the brick layout; the default index is restored afterwards."""
    a = fn(t)
    t.set_cell_index(False)
    c = None
    try:
        b = fn(t)
        if t.info()["depth"] >= 3:
            t.set_cell_index("brick")
            c = fn(t)
    finally:
        t.set_cell_index(True)
    return a, b, c


def _edge_rays(sc):
    h = np.float32(sc.bbox_size / sc.res)
    lo = np.float32(sc.bbox_lo[0])
    o, d = [], []
    for k in range(0, sc.res + 1, max(1, sc.res // 8)):
        a = lo + np.float32(k) * h
        o += [(a, a, 3.0), (a, 3.0, a), (-3.0, a, a), (a, -3.0, -3.0)]
        d += [(0, 0, -1), (0, -1, 0), (1, 0, 0), (0, 1, 1)]
    return np.array(o, np.float32), np.array(d, np.float32)


@pytest.mark.parametrize("seed,D,deg,dtype", [(91, 2, 0, "f32"), (92, 4, 1, "f16"), (93, 5, 3, "f32"),
                                              (94, 6, 2, "bf16"), (95, 7, 3, "f32"), (96, 8, 1, "f16")])
@pytest.mark.parametrize("gamma", [0.0, 1e-3])
def test_renders_bit_identical(pot, seed, D, deg, dtype, gamma):
    import torch
    sc = S.scene_random(seed, D, deg, p_occ=0.3, sigma_mu=2.0)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    o, d = S.random_rays(seed, 20000, radius=3.0, spread=1.0)
    eo, ed = _edge_rays(sc)
    o = torch.from_numpy(np.concatenate([o, eo])).cuda()
    d = torch.from_numpy(np.concatenate([d, ed])).cuda()
    cams = S.make_cameras(S.orbit_c2ws(5, radius=3.0, elevation_deg=25.0), 61, 47, 50.0)
    n = o.shape[0]

    def run(tree):
        seg = torch.zeros(n, dtype=torch.int32, device="cuda")
        touched = torch.zeros(max(1, sc.n), dtype=torch.uint8, device="cuda")
        rgb, tf = pot.render_rays(tree, o, d, near=0.3, far=8.0, bg=(0.1, 0.2, 0.3), gamma=gamma,
                                  want_t_final=True, seg_count=seg, leaf_touched=touched)
        img, itf = pot.render(tree, cams, gamma=gamma, bg=(0.5, 0.5, 0.5), want_t_final=True)
        return rgb, tf, seg, touched, img, itf

    a, b, c = _both(pot, t, run)
    for other in (b, c):
        if other is not None:
            for x, y in zip(a, other):
                assert torch.equal(x, y)
    pot.check()


def test_backward_and_visibility_bit_identical(pot):
    import torch
    sc = S.scene_random(97, 6, 3, p_occ=0.3, sigma_mu=2.0)
    t = pot.Tree.from_scene(sc)
    o, d = S.random_rays(97, 30000, radius=3.0, spread=1.0)
    o, d = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    g = torch.from_numpy(S.uniform(97, 5, np.arange(3 * o.shape[0], dtype=np.uint64)).astype(np.float32)
                         .reshape(-1, 3) - 0.5).cuda()
    cams = S.make_cameras(S.orbit_c2ws(4, radius=3.0), 48, 40, 40.0)

    def run(tree):
        rgb = pot.render_rays(tree, o, d, gamma=1e-3)
        gs, gsh = pot.render_backward(tree, o, d, g, rgb_fwd=rgb, gamma=1e-3)
        w = pot.visibility(tree, cams, gamma=1e-3)
        return gs, gsh, w

    a, b, c = _both(pot, t, run)
    # gradients are sums of float reductions whose order varies from run to
    # run; the maxima of the visibility weights do not depend on the order
    for other in (b, c):
        for x, y in zip(a[:2], other[:2]):
            assert torch.allclose(x, y, rtol=1e-5, atol=1e-6)
        assert torch.equal(a[2], other[2])
    pot.check()


def test_batch_mixes_trees_with_and_without_index(pot):
    import torch
    trees = [pot.Tree.from_scene(S.scene_random(98 + i, 5 + i, 2, p_occ=0.3), dtype="f16") for i in range(4)]
    trees[1].set_cell_index(False)
    trees[3].set_cell_index("brick")
    cams = [S.make_cameras([S.look_at((4 * np.cos(a), 4 * np.sin(a), 1.5))], 40 + 7 * i, 30 + 5 * i, 40.0,
                           near=1.0, far=8.0)[0] for i, a in enumerate(np.linspace(0, 5, 6))]
    outs = [torch.full((int(c["height"]), int(c["width"]), 3), -1.0, device="cuda") for c in cams]
    items = [(trees[i % 4], c, out, (0.0, 0.0, 0.0), 1e-3, None) for i, (c, out) in enumerate(zip(cams, outs))]
    pot.render_batch(items)
    for i, (c, out) in enumerate(zip(cams, outs)):
        tr = trees[i % 4]
        kind = {0: "none", 2: "dense", 3: "brick"}[tr.info()["index_kind"]]
        alone = pot.render(tr, c[None], gamma=1e-3)[0]
        assert torch.equal(out, alone)
        tr.set_cell_index(False)
        assert torch.equal(out, pot.render(tr, c[None], gamma=1e-3)[0])
        tr.set_cell_index(kind)
    pot.check()
