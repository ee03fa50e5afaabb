"""Pins of the oracle's SH codebook quantisation (App. B.2, median cut per SH
basis function): a plain recursive restatement on small inputs, balanced box
sizes, identity when every point gets its own box, box means, and the direct
float64 -> float16 rounding of the codebook entries."""
import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S


def _recursive_median_cut(P, bits):
    """The definition written out as recursion (slow; small inputs)."""
    P = np.asarray(P, np.float32)

    def split(idx, level):
        if level == bits:
            return [idx]
        if len(idx) < 2:
            return split(idx, level + 1) + split(idx[:0], level + 1)
        v = P[idx].astype(np.float64)
        ext = v.max(axis=0) - v.min(axis=0)
        a = int(np.argmax(ext))
        srt = sorted(idx, key=lambda i: (float(P[i, a]), int(i)))
        m = len(srt) // 2
        return split(np.array(srt[:m], np.int64), level + 1) + split(np.array(srt[m:], np.int64), level + 1)

    boxes = split(np.arange(P.shape[0], dtype=np.int64), 0)
    book = np.zeros((len(boxes), 3), np.float16)
    codes = np.zeros(P.shape[0], np.uint16)
    for j, b in enumerate(boxes):
        if len(b):
            acc = np.zeros(3)
            for i in b:
                acc = acc + P[i].astype(np.float64)
            book[j] = (acc / len(b)).astype(np.float16)
            codes[b] = j
    return book, codes


@pytest.mark.parametrize("n,bits", [(1, 3), (7, 3), (50, 4), (333, 6), (1000, 5), (64, 6)])
def test_matches_recursive_definition(oracle_mod, n, bits):
    rng = np.random.default_rng(n + bits)
    P = rng.normal(size=(n, 3)).astype(np.float32)
    P[: n // 5] = P[0]                       # repeated points (ties on every axis)
    b1, c1 = oracle_mod.median_cut(P, bits)
    b2, c2 = _recursive_median_cut(P, bits)
    assert np.array_equal(b1.view(np.uint16), b2.view(np.uint16)) and np.array_equal(c1, c2)


def test_balanced_boxes_and_means(oracle_mod):
    rng = np.random.default_rng(3)
    P = rng.uniform(-2, 2, size=(5000, 3)).astype(np.float32)
    book, codes = oracle_mod.median_cut(P, 8)
    counts = np.bincount(codes, minlength=256)
    assert set(counts.tolist()) <= {5000 // 256, 5000 // 256 + 1}
    for j in range(0, 256, 17):
        m = P[codes == j].astype(np.float64).mean(axis=0)
        assert np.allclose(book[j].astype(np.float64), m, rtol=1e-3, atol=1e-3)


def test_identity_when_boxes_outnumber_points(oracle_mod):
    rng = np.random.default_rng(4)
    P = rng.normal(size=(100, 3)).astype(np.float32)
    book, codes = oracle_mod.median_cut(P, 8)        # 256 boxes >= 100 points
    assert len(set(codes.tolist())) == 100
    assert np.array_equal(book[codes], P.astype(np.float16))


def test_entries_round_once_from_float64(oracle_mod):
    # float64 -> float16 must be one rounding (a float32 detour can differ)
    x = np.array([[1.0 + 2 ** -11 + 2 ** -30, 0.5, -0.25]], np.float64)
    P = x.astype(np.float32)
    book, _ = oracle_mod.median_cut(P, 1)
    assert book[0, 0] == np.float64(P[0, 0]).astype(np.float16)


def test_quantize_scene_values(oracle_mod):
    sc = S.scene_random(5, 4, 2, p_occ=0.5)
    q, books, codes = oracle_mod.quantize_scene(sc, 6)
    assert books.shape == (sc.sh_dim, 64, 3) and codes.shape == (sc.n, sc.sh_dim)
    for k in range(sc.sh_dim):
        assert np.array_equal(q.sh[:, k, :], books[k][codes[:, k]].astype(np.float32))
    assert np.array_equal(q.sigma, sc.sigma)          # sigma kept as it is (App. B.2)
