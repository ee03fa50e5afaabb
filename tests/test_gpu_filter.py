"""Visibility filtering (Sec. 3.2 "Filtering") on the GPU against the oracle:
per-leaf max ray weights within 1e-4, pruning bit-exact (both sides get the
same scores, so the threshold decision is shared), renders of the filter views
unchanged when only never-composited leaves are dropped, and the size/error
trade-off of tau_w on the main scene (also written to $POT_REPORT_DIR/filter.json when that is set)."""
import json
import math
import os

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


@pytest.mark.parametrize("seed,D,deg,dtype", [(71, 4, 1, "f32"), (72, 5, 2, "f32"), (73, 6, 3, "f16"),
                                              (74, 5, 4, "bf16")])
@pytest.mark.parametrize("gamma", [0.0, 0.02])
def test_visibility_vs_oracle(pot, oracle_mod, seed, D, deg, dtype, gamma):
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=2.0)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    ot = oracle_mod.build_sparse(sc, dtype=dtype)
    cams = S.make_cameras(S.orbit_c2ws(5, radius=3.0), 40, 36, 35.0)
    w = pot.visibility(t, cams, gamma=gamma).cpu().numpy()
    ref = oracle_mod.visibility(ot, cams, gamma=gamma)
    err = np.abs(w - ref)
    if gamma == 0.0:
        assert err.max() <= 1e-4
    else:   # a ray may stop one segment apart on the two sides
        assert (err > 1e-4).mean() < 0.002 and err.max() <= 1e-4 + gamma
    assert np.all(w >= 0) and np.all(w <= 1)


def test_visibility_accumulates_by_max(pot):
    import torch
    sc = S.scene_random(74, 5, 1, p_occ=0.35)
    t = pot.Tree.from_scene(sc)
    c1 = S.make_cameras(S.orbit_c2ws(2, radius=3.0), 32, 32, 30.0)
    c2 = S.make_cameras(S.orbit_c2ws(3, radius=3.0, elevation_deg=-20), 32, 32, 30.0)
    a = pot.visibility(t, c1)
    b = pot.visibility(t, c2)
    acc = pot.visibility(t, c2, max_weight=a.clone())
    assert torch.equal(acc, torch.maximum(a, b))


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_prune_bitexact(pot, oracle_mod, dtype):
    sc = S.scene_random(75, 6, 2, p_occ=0.35, sigma_mu=2.0)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    cams = S.make_cameras(S.orbit_c2ws(4, radius=3.0), 48, 48, 40.0)
    w = pot.visibility(t, cams)
    scores = w.cpu().numpy()
    for thr in (1e-30, 1e-3, 0.05, 2.0):
        tp = t.prune(w, thr)
        ref = oracle_mod.build_sparse(oracle_mod.prune(sc, scores, thr), dtype=dtype)
        a, b = tp.export(), ref.export()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
        assert np.array_equal(a[1].astype(np.float64), b[1]) and np.array_equal(a[2].astype(np.float64), b[2])
        assert tp.info()["n_leaves"] == int((scores >= thr).sum())


def test_prune_unseen_keeps_filter_view_renders(pot):
    import torch
    sc = S.scene_random(76, 6, 3, p_occ=0.4, sigma_mu=2.5)
    t = pot.Tree.from_scene(sc)
    cams = S.make_cameras(S.orbit_c2ws(6, radius=3.0), 64, 48, 50.0)
    w = pot.visibility(t, cams, gamma=1e-4)
    tp = t.prune(w, 1e-30)
    assert tp.info()["n_leaves"] < t.info()["n_leaves"]
    a = pot.render(t, cams, gamma=1e-4)
    b = pot.render(tp, cams, gamma=1e-4)
    assert torch.equal(a, b)


def test_filter_main_scene_tradeoff(pot):
    """Filter the main tree with the 100 training views, then render the 200
    evaluation views with the filtered trees: leaves kept and image error
    against the unfiltered tree, per tau_w."""
    import torch
    scene = S.scene_shapes()
    t = pot.Tree.from_scene(scene)
    train = S.cameras_train(n=100)
    w = pot.visibility(t, train, gamma=1e-4)
    evalc = S.cameras_main(200)
    ref = pot.render(t, evalc, gamma=1e-4)
    n0 = t.info()["n_leaves"]
    rep = {"leaves": n0, "bytes": t.info()["bytes"], "seen_by_training_views": int((w > 0).sum().item())}
    for tau in (1e-3, 1e-2):
        tp = t.prune(w, tau)
        img = pot.render(tp, evalc, gamma=1e-4)
        err = (img - ref).abs()
        mse = float((err ** 2).mean().item())
        rep[f"tau_w={tau}"] = {"leaves": tp.info()["n_leaves"], "bytes": tp.info()["bytes"],
                               "max_abs_vs_unfiltered": float(err.max().item()),
                               "psnr_vs_unfiltered_db": 10 * math.log10(1.0 / mse) if mse > 0 else float("inf")}
        tp.free()
    print(json.dumps(rep, indent=1))
    out_dir = os.environ.get("POT_REPORT_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "filter.json"), "w") as f:
            json.dump(rep, f, indent=1)
    assert rep["tau_w=0.001"]["leaves"] <= n0
    pot.check()
