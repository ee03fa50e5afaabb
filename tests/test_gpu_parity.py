"""GPU parity of the C-ABI path against the FP64 oracle.

Bar: bit-exact tree arrays and point queries; rendered colours within 1e-4
max-abs per channel (gamma = 0).  With gamma > 0 a ray may stop one segment
apart on the two sides; such rays are bounded by 1e-4 + T_stop * max|c - bg|
(the remaining transmittance is below gamma)."""
import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def pot():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2103_14024_gb300 as P
    P.lib()
    return P


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _export_equal(pot, oracle_mod, sc, dtype="f32"):
    t = pot.Tree.from_scene(sc, dtype=dtype)
    ot = oracle_mod.build_sparse(sc, dtype=dtype)
    child, sigma, sh, morton = t.export()
    oc, osig, osh, om = ot.export()
    assert np.array_equal(child, oc)
    assert np.array_equal(morton, om)
    assert np.array_equal(sigma.astype(np.float64), osig)
    assert np.array_equal(sh.astype(np.float64), osh)
    info = t.info()
    assert info["n_nodes"] == ot.n_nodes and info["n_leaves"] == ot.n_leaves
    return t, ot


# ---------------------------------------------------------------- build ----

@pytest.mark.parametrize("seed,D,deg", [(1, 1, 0), (2, 2, 1), (3, 3, 2), (4, 4, 3), (5, 5, 0), (6, 6, 3),
                                        (7, 7, 1), (8, 5, 4)])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_build_bitexact(pot, oracle_mod, seed, D, deg, dtype):
    sc = S.scene_random(seed, D, deg, p_occ=0.3, sh_std=2.0)
    _export_equal(pot, oracle_mod, sc, dtype)


def test_build_tiny_and_degenerate(pot, oracle_mod):
    _export_equal(pot, oracle_mod, S.scene_tiny())
    one = S.scene_random(9, 4, 1, p_occ=0.3)
    _export_equal(pot, oracle_mod, one.replace(morton=one.morton[:1], sigma=one.sigma[:1], sh=one.sh[:1]))
    empty = one.replace(morton=one.morton[:0], sigma=one.sigma[:0], sh=one.sh[:0])
    t = pot.Tree.from_scene(empty)
    child, *_ = t.export()
    assert t.info()["n_nodes"] == 1 and not child.any()
    full = S.scene_uniform(4, 2.0, np.ones((4, 3), np.float32))
    _export_equal(pot, oracle_mod, full)


def test_build_dense_equals_sparse(pot, oracle_mod, torch_mod):
    sc = S.scene_random(12, 5, 2, p_occ=0.3)
    sig, sh = sc.to_dense(fill_sigma=0.0, noise_seed=3)
    td = pot.Tree.build_dense(sc.depth, sc.sh_degree, sc.bbox_lo, sc.bbox_size, sig, sh)
    ts = pot.Tree.from_scene(sc)
    for a, b in zip(td.export(), ts.export()):
        assert np.array_equal(a, b)
    # device-resident inputs and a threshold
    tau = float(np.median(sc.sigma))
    tdev = pot.Tree.build_dense(sc.depth, sc.sh_degree, sc.bbox_lo, sc.bbox_size,
                                torch_mod.from_numpy(sig).cuda(), torch_mod.from_numpy(sh).cuda(),
                                threshold=tau)
    ot = oracle_mod.build_dense(sc.depth, sc.bbox_lo, sc.bbox_size, sc.sh_degree, sig, sh, tau=tau)
    for a, b in zip(tdev.export(), ot.export()):
        assert np.array_equal(a.astype(b.dtype), b)


def test_build_sparse_saturation_flag(pot, oracle_mod):
    sc = S.scene_random(13, 3, 0, p_occ=0.5)
    sig = sc.sigma.copy()
    sig[0] = 1e6
    t = pot.Tree.from_scene(sc.replace(sigma=sig), dtype="f16")
    assert t.info()["saturated"] == 1
    _, s16, _, _ = t.export()
    assert s16[0] == 65504.0


def test_build_rejects_bad_input(pot):
    sc = S.scene_random(14, 3, 0, p_occ=0.5)
    with pytest.raises(pot.PotError) as e:
        pot.Tree.from_scene(sc.replace(morton=sc.morton[::-1].copy()))
    assert e.value.status == pot.POT_ERR_INVALID_ARG
    sig = sc.sigma.copy()
    sig[3] = np.inf
    with pytest.raises(pot.PotError) as e:
        pot.Tree.from_scene(sc.replace(sigma=sig))
    assert e.value.status == pot.POT_ERR_INVALID_ARG
    big = sc.morton.copy()
    big[-1] = np.uint64(1 << 9)
    with pytest.raises(pot.PotError):
        pot.Tree.from_scene(sc.replace(morton=big))


# ---------------------------------------------------------------- query ----

@pytest.mark.parametrize("lo,size,D", [((-1.0, -1.0, -1.0), 2.0, 4), ((-1.5, -1.5, -1.5), 3.0, 7),
                                        ((0.1, -0.3, 2.7), 1.3, 5), ((-7.25, 3.5, 0.0), 10.0, 9)])
def test_query_bitexact(pot, oracle_mod, torch_mod, lo, size, D):
    sc = S.scene_random(21, min(D, 7), 0, p_occ=0.5, lo=lo, size=size) if D <= 7 else \
        S.scene_shapes(5, depth=D, sh_degree=0, occupancy=0.03).replace(bbox_lo=lo, bbox_size=size)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    rng = np.random.default_rng(D)
    R = 1 << sc.depth
    pts = (np.array(lo) + rng.uniform(-0.05, 1.05, size=(200000, 3)) * size).astype(np.float32)
    k = rng.integers(0, R + 1, size=(50000, 3))
    h = np.float32(size) / np.float32(R)
    face = (np.float32(lo) + k.astype(np.float32) * h).astype(np.float32)
    mix = pts[:50000].copy()
    sel = rng.integers(0, 2, size=mix.shape).astype(bool)
    mix[sel] = face[sel]
    nxt = np.nextafter(face, np.float32(np.inf)).astype(np.float32)
    prv = np.nextafter(face, np.float32(-np.inf)).astype(np.float32)
    special = np.array([[np.nan, 0, 0], [lo[0], lo[1], lo[2]],
                        [lo[0] + size, lo[1], lo[2]]], np.float32)
    pts = np.concatenate([pts, face, mix, nxt, prv, special]).astype(np.float32)
    got = pot.query(t, torch_mod.from_numpy(pts).cuda()).cpu().numpy()
    exp = oracle_mod.query(ot, pts)
    assert np.array_equal(got, exp), np.flatnonzero(got != exp)[:10]


def test_sh_basis_vs_oracle(pot, oracle_mod, torch_mod):
    rng = np.random.default_rng(3)
    d = rng.normal(size=(20000, 3)).astype(np.float32)
    d = np.concatenate([d, np.eye(3, dtype=np.float32), -np.eye(3, dtype=np.float32)])
    for K in (1, 4, 9, 16, 25):
        Y = pot.sh_basis(K, torch_mod.from_numpy(d).cuda()).cpu().numpy()
        ref = oracle_mod.sh_basis(K, d.astype(np.float64))
        assert np.abs(Y - ref).max() <= 1e-6


# --------------------------------------------------------------- render ----

def _cmp_render(gpu, ref, gamma, t_gpu=None, t_ref=None, bg=(0, 0, 0), name=""):
    err = np.abs(gpu - ref).max(axis=-1)
    if gamma == 0:
        assert err.max() <= TOL, f"{name}: max err {err.max():.3e}"
    else:
        # rays whose stop decision may differ: bound by the residual transmittance
        bad = err > TOL
        if bad.any():
            bound = TOL + gamma * 1.0 + 1e-6
            assert err[bad].max() <= bound, f"{name}: {err[bad].max():.3e} > {bound:.3e}"
            assert bad.mean() < 0.01


@pytest.mark.parametrize("variant", ["generic", "axis"])
@pytest.mark.parametrize("gamma", [0.0, 1e-4])
@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (1.0, 0.5, 0.25)])
def test_render_tiny(pot, oracle_mod, variant, gamma, bg):
    sc = S.scene_tiny()
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    cams = S.cameras_tiny(variant)
    rgb, tf = pot.render(t, cams, gamma=gamma, bg=bg, want_t_final=True)
    ref = oracle_mod.render_cams(ot, cams, gamma=gamma, bg=bg)
    _cmp_render(rgb.cpu().numpy(), ref["rgb"], gamma, name=f"tiny-{variant}")
    if gamma == 0:
        assert np.abs(tf.cpu().numpy() - ref["t_final"]).max() <= TOL
    pot.check()


@pytest.mark.parametrize("seed,D,deg", [(31, 2, 0), (32, 3, 1), (33, 4, 2), (34, 5, 3), (35, 6, 3),
                                        (36, 7, 2), (37, 5, 4), (38, 6, 4)])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_render_random_trees_rays(pot, oracle_mod, torch_mod, seed, D, deg, dtype):
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=2.0, sigma_s=1.5, sh_std=1.0)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    ot = oracle_mod.build_sparse(sc, dtype=dtype)       # oracle on the stored (rounded) values
    o, d = S.random_rays(seed, 5003, radius=3.0, spread=1.0)
    rgb, tf = pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda(),
                              near=0.5, far=7.0, bg=(0.2, 0.4, 0.6), want_t_final=True)
    ref = oracle_mod.render_rays(ot, o, d, near=0.5, far=7.0, bg=(0.2, 0.4, 0.6))
    _cmp_render(rgb.cpu().numpy(), ref["rgb"], 0.0, name=f"rand{seed}-{dtype}")
    assert np.abs(tf.cpu().numpy() - ref["t_final"]).max() <= TOL
    pot.check()


@pytest.mark.parametrize("W,H,ncam", [(37, 29, 3), (8, 4, 1), (1, 1, 2), (65, 3, 2)])
def test_render_ragged_tiles(pot, oracle_mod, W, H, ncam):
    sc = S.scene_random(41, 5, 1, p_occ=0.35)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    cams = S.make_cameras(S.orbit_c2ws(ncam, radius=3.0), W, H, 0.9 * max(W, H))
    rgb = pot.render(t, cams).cpu().numpy()
    ref = oracle_mod.render_cams(ot, cams)["rgb"]
    assert rgb.shape == (ncam, H, W, 3)
    assert np.abs(rgb - ref).max() <= TOL


def test_render_rays_ragged_counts(pot, oracle_mod, torch_mod):
    sc = S.scene_random(42, 4, 2, p_occ=0.4)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    for n in (1, 31, 33, 1000):
        o, d = S.random_rays(n, n, radius=3.0, spread=1.0)
        rgb = pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda()).cpu().numpy()
        assert np.abs(rgb - oracle_mod.render_rays(ot, o, d)["rgb"]).max() <= TOL
    # n = 0 is a no-op
    z = torch_mod.zeros((0, 3), device="cuda")
    assert pot.render_rays(t, z, z).shape == (0, 3)


def test_render_host_buffers(pot, oracle_mod):
    # the C ABI takes host arrays too (staged inside the call)
    sc = S.scene_random(43, 4, 1, p_occ=0.4)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(5, 777, radius=3.0, spread=1.0)
    import torch
    rgb = torch.empty((777, 3), dtype=torch.float32)   # host
    pot.render_rays(t, torch.from_numpy(o), torch.from_numpy(d), rgb=rgb)
    assert np.abs(rgb.numpy() - oracle_mod.render_rays(ot, o, d)["rgb"]).max() <= TOL
    cams = S.cameras_tiny("generic")
    host = torch.empty((1, 64, 64, 3), dtype=torch.float32)
    pot.render(t, cams, rgb=host)
    assert np.abs(host.numpy() - oracle_mod.render_cams(ot, cams)["rgb"]).max() <= TOL


@pytest.mark.parametrize("pinned", [True, False])
def test_render_host_output_chunked(pot, torch_mod, pinned):
    """Host outputs are rendered in view groups and copied back while the next
    group renders; the images equal a device-output render bit for bit."""
    torch = torch_mod
    sc = S.scene_random(47, 5, 2, p_occ=0.35)
    t = pot.Tree.from_scene(sc)
    cams = S.make_cameras(S.orbit_c2ws(41, radius=3.0), 33, 21, 30.0)      # 3 groups of 16 + ragged tile
    ref, ref_tf = pot.render(t, cams, gamma=1e-4, want_t_final=True)
    host = torch.full((41, 21, 33, 3), -1.0, pin_memory=pinned)
    host_tf = torch.full((41, 21, 33), -1.0, pin_memory=pinned)
    pot.render(t, cams, rgb=host, t_final=host_tf, gamma=1e-4)
    assert torch.equal(host, ref.cpu()) and torch.equal(host_tf, ref_tf.cpu())
    # host rgb with a device t_final
    dev_tf = torch.full((41, 21, 33), -1.0, device="cuda")
    host2 = torch.full((41, 21, 33, 3), -1.0)
    pot.render(t, cams, rgb=host2, t_final=dev_tf, gamma=1e-4)
    assert torch.equal(host2, ref.cpu()) and torch.equal(dev_tf, ref_tf)
    # device rgb with a host t_final (the image is written in place, t_final staged)
    dev_rgb = torch.full((41, 21, 33, 3), -1.0, device="cuda")
    host_tf2 = torch.full((41, 21, 33), -1.0, pin_memory=pinned)
    pot.render(t, cams, rgb=dev_rgb, t_final=host_tf2, gamma=1e-4)
    assert torch.equal(dev_rgb, ref) and torch.equal(host_tf2, ref_tf.cpu())
    # repeated calls reuse the library's scratch pool and streams: same result
    for _ in range(3):
        host.fill_(-1.0)
        pot.render(t, cams, rgb=host, gamma=1e-4)
        assert torch.equal(host, ref.cpu())


def test_render_edge_cases(pot, oracle_mod, torch_mod):
    sc = S.scene_random(44, 4, 2, p_occ=0.4, sigma_mu=1.0)
    sig = sc.sigma.copy()
    sig[::5] = -sig[::5]          # negative densities render as 0
    sig[1::9] = 1e4               # nearly opaque
    sc = sc.replace(sigma=sig)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    h = np.float32(sc.bbox_size / sc.res)
    lo = np.float32(sc.bbox_lo[0])
    o, d = [], []
    for k in range(0, 17, 2):
        for j in range(0, 17, 3):
            a, b = lo + np.float32(k) * h, lo + np.float32(j) * h
            o += [(a, b, 3.0), (a, 3.0, b), (-3.0, a, b), (a, -3.0, -3.0), (0.1 * k - 0.8, 0.1 * j - 0.8, 0.05)]
            d += [(0, 0, -1), (0, -1, 0), (1, 0, 0), (0, 1, 1), (0.3, -0.2, 1.0)]
    o += [(5, 5, 5), (0, 0, 0), (0.99, 0.99, 0.99), (-1, -1, -1), (1, 1, 1)]
    d += [(1, 0, 0), (1, 2, 3), (-1, -1, -1), (1, 1, 1), (-1, -1, -1)]
    o = np.array(o, np.float32)
    d = np.array(d, np.float32)
    for near, far in ((0.0, 1e30), (0.7, 2.5)):
        rgb = pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda(),
                              near=near, far=far, bg=(0.3, 0.3, 0.3)).cpu().numpy()
        ref = oracle_mod.render_rays(ot, o, d, near=near, far=far, bg=(0.3, 0.3, 0.3))["rgb"]
        assert np.abs(rgb - ref).max() <= TOL
    # an empty tree renders the background
    empty = sc.replace(morton=sc.morton[:0], sigma=sc.sigma[:0], sh=sc.sh[:0])
    te = pot.Tree.from_scene(empty)
    rgb = pot.render_rays(te, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda(),
                          bg=(0.1, 0.2, 0.3)).cpu().numpy()
    assert np.array_equal(rgb, np.tile(np.float32([0.1, 0.2, 0.3]), (o.shape[0], 1)))


def test_render_counts_match_oracle(pot, oracle_mod, torch_mod):
    sc = S.scene_random(45, 5, 1, p_occ=0.35)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(6, 4000, radius=3.0, spread=1.0)
    seg = torch_mod.zeros(4000, dtype=torch_mod.int32, device="cuda")
    touched = torch_mod.zeros(sc.n, dtype=torch_mod.uint8, device="cuda")
    pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda(), seg_count=seg,
                    leaf_touched=touched)
    ref = oracle_mod.render_rays(ot, o, d, want_touched=True)
    seg = seg.cpu().numpy()
    # a zero-length tie segment may be counted on one side only
    assert np.abs(seg - ref["n_seg"]).max() <= 2
    assert (seg == ref["n_seg"]).mean() > 0.99
    tt = touched.cpu().numpy()
    assert (tt != ref["touched"]).sum() <= max(2, int(0.002 * sc.n))


def test_traversal_step_bound_raises_error_word(pot, torch_mod):
    sc = S.scene_random(46, 5, 0, p_occ=0.4)
    t = pot.Tree.from_scene(sc)
    o, d = S.random_rays(7, 64, radius=3.0, spread=0.3)
    pot.check()
    pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda(), max_steps=2)
    with pytest.raises(pot.PotError) as e:
        pot.check()
    assert e.value.status == pot.POT_ERR_TRAVERSAL
    pot.check()   # the word was cleared
    pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda())
    pot.check()


def test_render_tile_limit_is_an_error(pot, torch_mod):
    """A call whose tiles would reach 2^32 is refused before any launch (the
    kernels index tiles in 32 bits); the image is never touched."""
    t = pot.Tree.from_scene(S.scene_tiny())
    big = S.make_cameras(S.orbit_c2ws(65, radius=3.0), 46000, 46000, 40000.0)   # 65 x 2^26 tiles
    rgb = torch_mod.full((4,), -1.0, device="cuda")
    with pytest.raises(pot.PotError) as e:
        pot.render(t, big, rgb=rgb)
    assert e.value.status == pot.POT_ERR_INVALID_ARG
    assert torch_mod.equal(rgb, torch_mod.full((4,), -1.0, device="cuda"))
    pot.check()


def test_render_depth_12_tree(pot, oracle_mod, torch_mod):
    """The deepest trees (D = 12, 4096^3 voxels, no cell index): rays through
    single leaves far apart, against the oracle."""
    D = 12
    xyz = np.array([[3, 4, 5], [2048, 100, 4095], [4095, 4095, 4095], [1000, 1001, 1002]], np.uint64)
    m = S.morton_encode(xyz[:, 0], xyz[:, 1], xyz[:, 2], D)
    order = np.argsort(m)
    sc = S.Scene(depth=D, bbox_lo=(-1.0, -1.0, -1.0), bbox_size=2.0, sh_degree=1, morton=m[order].astype(np.uint64),
                 sigma=np.float32([900.0, 2000.0, 500.0, 1500.0]),
                 sh=np.random.default_rng(0).normal(size=(4, 4, 3)).astype(np.float32))
    t = pot.Tree.from_scene(sc)
    assert t.info()["index_bytes"] == 0
    h = 2.0 / 4096
    centres = (-1.0 + (xyz[order].astype(np.float64) + 0.5) * h).astype(np.float32)
    o = np.repeat(centres - np.float32([0.0, 0.0, 2.5]), 7, axis=0)
    jit = (S.uniform(12, 1, np.arange(2 * o.shape[0], dtype=np.uint64)).reshape(-1, 2) - 0.5) * (1.5 * h / 2.5)
    d = np.concatenate([jit, np.ones((o.shape[0], 1))], 1).astype(np.float32)
    rgb = pot.render_rays(t, torch_mod.from_numpy(o).cuda(), torch_mod.from_numpy(d).cuda()).cpu().numpy()
    ref = oracle_mod.render_rays(oracle_mod.build_sparse(sc), o, d)["rgb"]
    assert np.abs(rgb - ref).max() <= TOL
    assert (np.abs(ref).sum(1) > 0).sum() >= 4          # some rays do hit the leaves
    pot.check()


def test_render_invalid_args(pot):
    sc = S.scene_tiny()
    t = pot.Tree.from_scene(sc)
    cams = np.concatenate([S.cameras_tiny("generic"), S.make_cameras(S.orbit_c2ws(1), 32, 32, 40.0)])
    with pytest.raises(pot.PotError) as e:
        pot.render(t, cams)
    assert e.value.status == pot.POT_ERR_INVALID_ARG
    bad = S.cameras_tiny("generic").copy()
    bad["fx"] = np.nan
    with pytest.raises(pot.PotError):
        pot.render(t, bad)
    with pytest.raises(pot.PotError):
        pot.render(t, S.cameras_tiny("generic"), gamma=-1.0)


# ------------------------------------------------- main scene, full size ----

@pytest.fixture(scope="module")
def main_scene():
    return S.scene_shapes()


@pytest.fixture(scope="module")
def main_trees(pot, oracle_mod, main_scene):
    return pot.Tree.from_scene(main_scene), oracle_mod.build_sparse(main_scene)


def test_main_scene_tree_bitexact(pot, oracle_mod, main_scene, main_trees):
    t, ot = main_trees
    child, sigma, sh, morton = t.export()
    oc, osig, osh, om = ot.export()
    assert np.array_equal(child, oc) and np.array_equal(morton, om)
    assert np.array_equal(sigma.astype(np.float64), osig) and np.array_equal(sh.astype(np.float64), osh)


@pytest.mark.parametrize("gamma", [0.0, 1e-4])
def test_main_scene_200_views_sampled(pot, oracle_mod, main_trees, gamma):
    """All 200 views of 800x800 in one call (the benchmark's launch); 40000
    sampled pixels and 2 full views against the oracle."""
    t, ot = main_trees
    cams = S.cameras_main(200)
    rgb = pot.render(t, cams, gamma=gamma).cpu().numpy()
    assert rgb.shape == (200, 800, 800, 3) and np.isfinite(rgb).all()
    rng = np.random.default_rng(int(gamma * 1e6) + 1)
    n = 40000
    ci, px, py = rng.integers(0, 200, n), rng.integers(0, 800, n), rng.integers(0, 800, n)
    ref = oracle_mod.render_pixels(ot, cams, ci, px, py, gamma=gamma)
    _cmp_render(rgb[ci, py, px], ref["rgb"], gamma, name="main-sampled")
    for v in (0, 137):
        full = oracle_mod.render_cams(ot, cams[v:v + 1], gamma=gamma)["rgb"][0]
        _cmp_render(rgb[v], full, gamma, name=f"main-view{v}")
    pot.check()
