"""Pins of the oracle's tree construction (Sec. 3.2 "Filtering": kept voxels
become leaves at the deepest level, the tree is empty elsewhere), point
queries (exact voxel membership) and fp16 / bf16 rounding."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S


def _walk_paths(child, D):
    """Independent check: (level, prefix) of every node and Morton code of every leaf, by DFS."""
    node_lp = {0: (0, 0)}
    leaf_code = {}
    stack = [0]
    while stack:
        n = stack.pop()
        l, p = node_lp[n]
        for s in range(8):
            c = int(child[n, s])
            if c > 0:
                assert c not in node_lp, "node reached twice"
                assert l + 1 < D, "internal node below depth D-1"
                node_lp[c] = (l + 1, (p << 3) | s)
                stack.append(c)
            elif c < 0:
                assert l == D - 1, "leaf above the deepest level"
                leaf_code[-c - 1] = (p << 3) | s
    return node_lp, leaf_code


@pytest.mark.parametrize("seed,D,deg", [(1, 1, 0), (2, 2, 1), (3, 3, 2), (4, 4, 3), (5, 5, 1), (6, 6, 0)])
def test_structure_invariants(oracle_mod, seed, D, deg):
    sc = S.scene_random(seed, D, deg, p_occ=0.3)
    t = oracle_mod.build_sparse(sc)
    child, sigma, sh, morton = t.export()
    assert t.n_leaves == sc.n
    node_lp, leaf_code = _walk_paths(child, D)
    # every node reachable, every node has >= 1 child (except an empty root)
    assert len(node_lp) == t.n_nodes
    for n in range(t.n_nodes):
        if n != 0 or sc.n > 0:
            assert (child[n] != 0).any()
    # leaf index = rank of Morton code among kept voxels; codes strictly increasing
    assert sorted(leaf_code) == list(range(sc.n))
    assert all(leaf_code[i] == int(sc.morton[i]) for i in range(sc.n))
    assert np.all(np.diff(morton.astype(np.int64)) > 0) if sc.n > 1 else True
    # breadth-first order: sorted by (level, prefix) equals index order
    order = sorted(node_lp, key=lambda n: node_lp[n])
    assert order == list(range(t.n_nodes))
    # a node exists iff it has a kept descendant: count prefixes directly
    for l in range(D):
        prefixes = set(int(m) >> (3 * (D - l)) for m in sc.morton)
        have = sum(1 for n in node_lp.values() if n[0] == l)
        assert have == (len(prefixes) if sc.n > 0 else (1 if l == 0 else 0))
    # values copied through
    assert np.array_equal(sigma, sc.sigma.astype(np.float64))
    assert np.array_equal(sh, sc.sh.astype(np.float64))


def test_every_voxel_lookup_bruteforce(oracle_mod):
    sc = S.scene_random(11, 4, 0, p_occ=0.4)
    t = oracle_mod.build_sparse(sc)
    D, R = sc.depth, sc.res
    h = sc.bbox_size / R
    rank = {int(m): i for i, m in enumerate(sc.morton)}
    xs = np.arange(R)
    X, Y, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    pts = np.stack([sc.bbox_lo[0] + (X + 0.5) * h, sc.bbox_lo[1] + (Y + 0.5) * h,
                    sc.bbox_lo[2] + (Z + 0.5) * h], axis=-1).reshape(-1, 3)
    got = oracle_mod.query(t, pts)
    codes = S.morton_encode(X.ravel(), Y.ravel(), Z.ravel(), D)
    exp = np.array([rank.get(int(c), -1) for c in codes])
    assert np.array_equal(got, exp)


def test_dense_equals_sparse_and_threshold(oracle_mod):
    sc = S.scene_random(12, 4, 2, p_occ=0.3)
    sig, sh = sc.to_dense(fill_sigma=0.0, noise_seed=5)
    td = oracle_mod.build_dense(sc.depth, sc.bbox_lo, sc.bbox_size, sc.sh_degree, sig, sh, tau=0.0)
    ts = oracle_mod.build_sparse(sc)
    for x, y in zip(td.export(), ts.export()):
        assert np.array_equal(x, y)
    # a voxel at exactly tau is dropped
    x0, y0, z0 = S.morton_decode(sc.morton[:1], sc.depth)
    sig2 = sig.copy()
    sig2[x0[0], y0[0], z0[0]] = 0.0
    t2 = oracle_mod.build_dense(sc.depth, sc.bbox_lo, sc.bbox_size, sc.sh_degree, sig2, sh, tau=0.0)
    assert t2.n_leaves == sc.n - 1
    # threshold: keep sigma > tau only
    tau = float(np.median(sc.sigma))
    tt = oracle_mod.build_dense(sc.depth, sc.bbox_lo, sc.bbox_size, sc.sh_degree, sig, sh, tau=tau)
    assert tt.n_leaves == int((sc.sigma > tau).sum())


def test_invalid_inputs(oracle_mod):
    sc = S.scene_random(13, 3, 0, p_occ=0.5)
    bad = sc.replace(morton=sc.morton[::-1].copy())
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.build_sparse(bad)
    sig, sh = sc.to_dense()
    sig[1, 1, 1] = np.nan
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.build_dense(sc.depth, sc.bbox_lo, sc.bbox_size, 0, sig, sh)


def test_empty_tree(oracle_mod):
    sc = S.scene_random(14, 3, 0, p_occ=0.0)
    sc = sc.replace(morton=sc.morton[:0], sigma=sc.sigma[:0], sh=sc.sh[:0])
    t = oracle_mod.build_sparse(sc)
    child, *_ = t.export()
    assert t.n_nodes == 1 and t.n_leaves == 0 and not child.any()
    assert np.all(oracle_mod.query(t, np.zeros((4, 3), np.float32)) == -1)


def _exact_voxel(p, lo, size, D):
    """Exact rational voxel index of fp32 coordinate p, or None outside [lo, lo+size)."""
    P, L, Sz = Fraction(float(p)), Fraction(float(lo)), Fraction(float(size))
    if P < L or P >= L + Sz:
        return None
    return int((P - L) * (1 << D) // Sz)


@pytest.mark.parametrize("lo,size,D", [((-1.0, -1.0, -1.0), 2.0, 4), ((-1.5, -1.5, -1.5), 3.0, 6),
                                        ((0.1, -0.3, 2.7), 1.3, 5)])
def test_query_exact_membership(oracle_mod, lo, size, D):
    sc = S.scene_random(21, D, 0, p_occ=0.5, lo=lo, size=size)
    t = oracle_mod.build_sparse(sc)
    rank = {int(m): i for i, m in enumerate(sc.morton)}
    rng = np.random.default_rng(D)
    n = 3000
    pts = (np.array(lo) + rng.uniform(-0.05, 1.05, size=(n, 3)) * size).astype(np.float32)
    # points exactly on faces, edges and corners
    R = 1 << D
    k = rng.integers(0, R + 1, size=(600, 3))
    h = np.float32(size) / np.float32(R)
    face = (np.float32(lo) + k.astype(np.float32) * h).astype(np.float32)
    mix = pts[:600].copy()
    sel = rng.integers(0, 2, size=(600, 3)).astype(bool)
    mix[sel] = face[sel]
    # one ulp below / above faces (includes subnormals next to a face at 0)
    nxt = np.nextafter(face, np.float32(np.inf)).astype(np.float32)
    prv = np.nextafter(face, np.float32(-np.inf)).astype(np.float32)
    pts = np.concatenate([pts, face, mix, nxt, prv]).astype(np.float32)
    got = oracle_mod.query(t, pts)
    for i in range(pts.shape[0]):
        q = [_exact_voxel(pts[i, a], np.float32(lo[a]), np.float32(size), D) for a in range(3)]
        if any(v is None for v in q):
            exp = -2
        else:
            exp = rank.get(int(S.morton_encode(q[0], q[1], q[2], D)), -1)
        assert got[i] == exp, (pts[i], q)


def test_f16_rounding_matches_numpy(oracle_mod):
    rng = np.random.default_rng(0)
    bits = np.concatenate([
        rng.integers(0, 2 ** 32, size=400000, dtype=np.uint64).astype(np.uint32),
        # exponents within the binary16 range and its subnormals
        (rng.integers(0x33000000, 0x477FE000, size=400000, dtype=np.uint64)).astype(np.uint32),
    ])
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) <= 65504.0)]
    # exact halfway cases between binary16 neighbours
    h = np.arange(0, 0x7BFF, dtype=np.uint16).view(np.float16).astype(np.float64)
    mids = ((h[:-1] + h[1:]) / 2).astype(np.float32)
    x = np.concatenate([x, mids, -mids])
    got, ovf = oracle_mod.round_values(x, "f16")
    assert not ovf
    assert np.array_equal(got.view(np.uint32), x.astype(np.float16).astype(np.float32).view(np.uint32))


def test_f16_saturation(oracle_mod):
    got, ovf = oracle_mod.round_values(np.array([65519.0, 65520.0, -1e6, 3e38], np.float32), "f16")
    assert ovf
    assert got.tolist() == [65504.0, 65504.0, -65504.0, 65504.0]


def test_bf16_rounding_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, size=800000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < 3.38e38)]
    # exact ties (lower 16 bits 0x8000)
    tb = (rng.integers(0, 2 ** 16, size=20000, dtype=np.uint64).astype(np.uint32) << 16) | 0x8000
    t = tb.view(np.float32)
    x = np.concatenate([x, t[np.isfinite(t) & (np.abs(t) < 3.38e38)]])
    got, ovf = oracle_mod.round_values(x, "bf16")
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_stored_values_rounded(oracle_mod):
    sc = S.scene_random(31, 3, 1, p_occ=0.5, sh_std=3.0)
    for dt in ("f16", "bf16"):
        t = oracle_mod.build_sparse(sc, dtype=dt)
        _, sigma, sh, _ = t.export()
        s_ref, _ = oracle_mod.round_values(sc.sigma, dt)
        h_ref, _ = oracle_mod.round_values(sc.sh, dt)
        assert np.array_equal(sigma, s_ref.astype(np.float64))
        assert np.array_equal(sh, h_ref.astype(np.float64))


@pytest.mark.parametrize("seed,depth,deg", [(1004, 5, 1), (1006, 6, 3), (1001, 7, 2)])
def test_scene_generator_torch_form_equals_numpy_form(seed, depth, deg):
    """The torch form of the shapes generator (used where the serving trees are
    generated on the device) gives the numpy form's leaves bit for bit, so the
    oracle may be given either."""
    torch = pytest.importorskip("torch")
    a = S.scene_shapes(seed, depth=depth, sh_degree=deg)
    b = S.scene_shapes_torch(seed, depth=depth, sh_degree=deg, device="cpu")
    assert np.array_equal(a.morton, b.morton.numpy().view(np.uint64))
    assert np.array_equal(a.sigma.view(np.uint32), b.sigma.numpy().view(np.uint32))
    assert np.array_equal(a.sh.view(np.uint32), b.sh.numpy().view(np.uint32))
