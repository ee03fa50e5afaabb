"""Serving path on the GPU: pot_render_batch (mixed trees, SH degrees, dtypes
and resolutions in one call) renders every request bit-identically to
rendering it alone with pot_render, and the continuous-batching server
delivers the same images under a Poisson request stream."""
import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import paper_2103_14024_gb300 as pot
    pot.lib()
    specs = [(5, 1, "f16", 2001), (6, 2, "f16", 2002), (7, 3, "f16", 2003), (8, 3, "f16", 2004),
             (6, 3, "f32", 2005), (5, 0, "bf16", 2006), (5, 4, "f32", 2007)]
    scenes = [S.scene_shapes(seed, depth=D, sh_degree=deg) for D, deg, _, seed in specs]
    trees = [pot.Tree.from_scene(sc, dtype=dt) for sc, (_, _, dt, _) in zip(scenes, specs)]
    return pot, torch, trees, scenes, specs


def _requests(n, n_trees, seed=11):
    ids = np.arange(n, dtype=np.uint64)
    tree = (S.uniform(seed, 1, ids) * n_trees).astype(int)
    res = [(64, 64), (96, 80), (128, 128), (200, 120), (37, 53)]
    pick = (S.uniform(seed, 2, ids) * len(res)).astype(int)
    az = S.uniform(seed, 3, ids) * 2 * np.pi
    cams = []
    for i in range(n):
        W, H = res[pick[i]]
        eye = (4 * np.cos(0.5) * np.cos(az[i]), 4 * np.cos(0.5) * np.sin(az[i]), 4 * np.sin(0.5))
        cams.append(S.make_cameras([S.look_at(eye)], W, H, 1.2 * W, near=2.0, far=6.0)[0])
    return tree, cams


def test_batch_bitidentical_to_alone(env):
    pot, torch, trees, scenes, specs = env
    tree_idx, cams = _requests(30, len(trees))
    outs = [torch.full((int(c["height"]), int(c["width"]), 3), -1.0, device="cuda") for c in cams]
    tfs = [torch.full((int(c["height"]), int(c["width"])), -1.0, device="cuda") for c in cams]
    bgs = [(0.1 * (i % 3), 0.2, 0.3) for i in range(len(cams))]
    items = [(trees[t], c, o, bg, 1e-4, tf) for t, c, o, bg, tf in zip(tree_idx, cams, outs, bgs, tfs)]
    pot.render_batch(items)
    torch.cuda.synchronize()
    for t, c, o, bg, tf in zip(tree_idx, cams, outs, bgs, tfs):
        alone, tf_alone = pot.render(trees[t], c[None], bg=bg, gamma=1e-4, want_t_final=True)
        assert torch.equal(o, alone[0]), "batch differs from alone"
        assert torch.equal(tf, tf_alone[0])
    pot.check()


def test_batch_vs_oracle(env, oracle_mod):
    pot, torch, trees, scenes, specs = env
    tree_idx, cams = _requests(6, len(trees), seed=12)
    for t, c in zip(tree_idx, cams):
        out = torch.empty((int(c["height"]), int(c["width"]), 3), device="cuda")
        pot.render_batch([(trees[t], c, out, (0.0, 0.0, 0.0), 0.0, None)])
        ot = oracle_mod.build_sparse(scenes[t], dtype=specs[t][2])
        ref = oracle_mod.render_cams(ot, c[None])["rgb"][0]
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-4


def test_server_results_same_alone_and_in_the_mix(env):
    from paper_2103_14024_gb300.serve import RenderServer, Request, summarize
    pot, torch, trees, scenes, specs = env
    tree_idx, cams = _requests(80, len(trees), seed=13)
    arrival = np.cumsum(-np.log(1 - S.uniform(13, 9, np.arange(80, dtype=np.uint64))) / 2000.0)
    budget = sum(t.info()["bytes"] for t in trees) + 2_000_000          # tight: forces admission waits
    results = {}
    for mode in ("batch", "alone"):
        reqs = [Request(i, float(arrival[i]), int(tree_idx[i]), cams[i]) for i in range(80)]
        srv = RenderServer(trees, hbm_budget_bytes=budget, streams=3, gamma=1e-4)
        srv.run(reqs, mode=mode)
        torch.cuda.synchronize()
        s = summarize(reqs)
        assert s["requests"] == 80 and s["rejected"] == 0 and s["p99_ms"] >= s["p50_ms"] > 0
        results[mode] = [r.rgb.clone() for r in reqs]
    for a, b, t, c in zip(results["batch"], results["alone"], tree_idx, cams):
        assert torch.equal(a, b)
        assert torch.equal(a, pot.render(trees[t], c[None], gamma=1e-4)[0])
    pot.check()
