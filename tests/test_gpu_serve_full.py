"""Serving workload at its own sizes: the depth-9 and depth-10 serving trees
(SH degree 3, fp16 leaves, ~4 M and ~32 M leaves) rendered through
pot_render_batch with 1920 x 1080 and 800 x 800 requests in one call, checked
against the FP64 oracle of the same (fp16-rounded) trees on sampled pixels.

The GPU trees are generated on the device by the torch form of the scene
generator; the oracle gets the same leaves copied to the host (the generator
is shared input code, and its torch form equals the numpy form, checked in
tests/test_oracle_tree.py)."""
import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch
    assert torch.cuda.is_available()
    import paper_2103_14024_gb300 as pot
    pot.lib()
    out = []
    for i, (D, deg) in enumerate(S.SERVE_TREES):
        if D < 9:
            continue
        sc = S.scene_shapes_torch(1004 + i, depth=D, sh_degree=deg, device="cuda")
        tree = pot.Tree.build_sparse(D, deg, sc.bbox_lo, sc.bbox_size, sc.morton, sc.sigma, sc.sh, dtype="f16")
        host = S.Scene(D, sc.bbox_lo, sc.bbox_size, deg, sc.morton.cpu().numpy().view(np.uint64),
                       sc.sigma.cpu().numpy(), sc.sh.cpu().numpy())
        del sc
        torch.cuda.empty_cache()
        out.append((D, tree, oracle_mod.build_sparse(host, dtype="f16")))
        del host
    return pot, torch, out


def _cam(W, H, az, el):
    eye = (4.0 * np.cos(el) * np.cos(az), 4.0 * np.cos(el) * np.sin(az), 4.0 * np.sin(el))
    return S.make_cameras([S.look_at(eye)], W, H, 1111.0 * W / 800.0, near=2.0, far=6.0)[0]


@pytest.mark.parametrize("gamma", [0.0, 1e-4])
def test_serving_trees_full_size_vs_oracle(env, oracle_mod, gamma):
    pot, torch, trees = env
    reqs = []
    for D, tree, otree in trees:
        for W, H in ((1920, 1080), (800, 800)):
            reqs.append((D, tree, otree, _cam(W, H, 0.3 + 0.7 * len(reqs), np.radians(15.0 + 9.0 * len(reqs)))))
    outs = [torch.full((int(c["height"]), int(c["width"]), 3), -1.0, device="cuda") for *_, c in reqs]
    pot.render_batch([(tree, c, o, (0.0, 0.0, 0.0), gamma, None) for (_, tree, _, c), o in zip(reqs, outs)])
    torch.cuda.synchronize()
    pot.check()
    rng = np.random.default_rng(17)
    for k, ((D, tree, otree, c), o) in enumerate(zip(reqs, outs)):
        W, H = int(c["width"]), int(c["height"])
        img = o.cpu().numpy()
        assert (img >= 0).all()
        # sampled pixels: uniform over the image plus a dense 32 x 32 block at the centre
        n = 6000
        px = rng.integers(0, W, n)
        py = rng.integers(0, H, n)
        by, bx = np.mgrid[H // 2 - 16:H // 2 + 16, W // 2 - 16:W // 2 + 16]
        px = np.concatenate([px, bx.ravel()])
        py = np.concatenate([py, by.ravel()])
        ref = oracle_mod.render_pixels(otree, c[None], np.zeros_like(px), px, py, gamma=gamma)
        got = img[py, px]
        err = np.abs(got - ref["rgb"]).max(axis=1)
        hit = ref["n_seg"] > 0
        assert hit.sum() > 500, f"request {k}: too few sampled pixels see the object"
        if gamma == 0.0:
            assert err.max() <= TOL, f"depth {D} {W}x{H}: max err {err.max():.3e}"
        else:
            # a ray may stop one segment apart on the two sides: bounded by gamma * max|c - bg| <= gamma
            assert err.max() <= TOL + gamma
            assert (err > TOL).mean() < 0.01
    # the same requests alone through pot_render give the same images bit for bit
    for (D, tree, otree, c), o in zip(reqs, outs):
        alone = pot.render(tree, c[None], gamma=gamma)[0]
        assert torch.equal(alone, o)
