"""Codebook quantisation (App. B.2) on the GPU path against the oracle: the
quantised tree's stored values equal the oracle's median cut bit for bit, its
renders match the oracle on those values within 1e-4, it batches and filters
like other trees, and on the main scene its size and image error against the
float32 tree are recorded (also in $POT_REPORT_DIR/codebook.json when set)."""
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


@pytest.mark.parametrize("seed,D,deg,bits,dtype", [(81, 4, 1, 4, "f32"), (82, 5, 2, 6, "f32"),
                                                    (83, 6, 3, 8, "f16"), (84, 3, 0, 16, "f32"),
                                                    (85, 4, 4, 5, "f32")])
def test_quantized_values_bitexact(pot, oracle_mod, seed, D, deg, bits, dtype):
    sc = S.scene_random(seed, D, deg, p_occ=0.4, sigma_mu=2.0)
    base = oracle_mod.build_sparse(sc, dtype=dtype)
    _, bs, bh, _ = base.export()              # the stored values the quantiser reads
    src = sc.replace(sigma=bs.astype(np.float32), sh=bh.astype(np.float32))
    q_ref, books, codes = oracle_mod.quantize_scene(src, bits)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    tq = t.quantize(bits)
    info = tq.info()
    assert info["leaf_dtype"] == 3 and info["n_leaves"] == sc.n
    child, sig, sh, morton = tq.export()
    c0, _, _, m0 = t.export()
    assert np.array_equal(child, c0) and np.array_equal(morton, m0)
    assert np.array_equal(sig, q_ref.sigma) and np.array_equal(sh, q_ref.sh)


def test_quantized_render_vs_oracle(pot, oracle_mod):
    import torch
    sc = S.scene_random(85, 6, 3, p_occ=0.35, sigma_mu=2.0)
    t = pot.Tree.from_scene(sc).quantize(10)
    _, sig, sh, _ = t.export()
    ot = oracle_mod.build_sparse(sc.replace(sigma=sig, sh=sh))
    cams = S.make_cameras(S.orbit_c2ws(3, radius=3.0), 48, 40, 40.0)
    rgb = pot.render(t, cams).cpu().numpy()
    assert np.abs(rgb - oracle_mod.render_cams(ot, cams)["rgb"]).max() <= 1e-4
    o, d = S.random_rays(5, 3000, radius=3.0, spread=0.9)
    r = pot.render_rays(t, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()).cpu().numpy()
    assert np.abs(r - oracle_mod.render_rays(ot, o, d)["rgb"]).max() <= 1e-4
    # batch and filtering accept the quantised tree
    out = torch.empty((40, 48, 3), device="cuda")
    pot.render_batch([(t, cams[0], out, (0.0, 0.0, 0.0), 0.0, None)])
    assert torch.equal(out, pot.render(t, cams[:1])[0])
    w = pot.visibility(t, cams)
    assert float(w.max().item()) > 0
    with pytest.raises(pot.PotError):
        pot.render_backward(t, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                            torch.zeros((3000, 3), device="cuda"))


def test_codebook_main_scene(pot):
    import torch
    scene = S.scene_shapes()
    t = pot.Tree.from_scene(scene)
    cams = S.cameras_main(200)
    ref = pot.render(t, cams, gamma=1e-4)
    tq = t.quantize(16)
    img = pot.render(tq, cams, gamma=1e-4)
    err = (img - ref).abs()
    mse = float((err ** 2).mean().item())
    rep = {"bits": 16, "leaves": t.info()["n_leaves"], "bytes_f32_tree": t.info()["bytes"],
           "bytes_quantised_tree": tq.info()["bytes"], "leaf_bytes": tq.info()["leaf_bytes"],
           "max_abs_vs_f32": float(err.max().item()),
           "psnr_vs_f32_db": 10 * math.log10(1.0 / mse) if mse > 0 else float("inf")}
    print(json.dumps(rep, indent=1))
    out_dir = os.environ.get("POT_REPORT_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "codebook.json"), "w") as f:
            json.dump(rep, f, indent=1)
    assert rep["psnr_vs_f32_db"] > 30
    pot.check()
