"""GPU parity of the differentiation path (App. B.3.2) and the optimiser step
(Sec. 3.3) against the FP64 oracle; MSE loss; pixel-ray generation; the
torch.autograd.Function; a short optimisation run.

Gradient bar: max |gpu - oracle| <= 1e-4 x max |oracle| per array (float
atomics make the GPU summation order non-deterministic)."""
import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def pot():
    import torch
    assert torch.cuda.is_available()
    import paper_2103_14024_gb300 as P
    P.lib()
    return P


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _close(gpu, ref, name):
    scale = max(float(np.abs(ref).max()), 1e-12)
    err = float(np.abs(gpu - ref).max())
    assert err <= REL * scale, f"{name}: max err {err:.3e} vs scale {scale:.3e}"


@pytest.mark.parametrize("seed,D,deg", [(51, 3, 0), (52, 4, 1), (53, 5, 2), (54, 5, 3), (55, 6, 3), (56, 5, 4)])
@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.9)])
def test_backward_vs_oracle(pot, oracle_mod, torch_mod, seed, D, deg, bg):
    torch = torch_mod
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    sig = sc.sigma.copy()
    sig[::11] = -sig[::11]                     # some non-positive densities (zero gradient)
    sc = sc.replace(sigma=sig)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(seed, 3001, radius=3.0, spread=0.9)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(o.shape[0], 3)).astype(np.float32)
    og, od, gg = (torch.from_numpy(a).cuda() for a in (o, d, g))
    rgb = pot.render_rays(t, og, od, bg=bg, near=0.2, far=8.0)
    gs, gh = pot.render_backward(t, og, od, gg, rgb_fwd=rgb, bg=bg, near=0.2, far=8.0)
    rs, rh = oracle_mod.backward_rays(ot, o, d, g.astype(np.float64), near=0.2, far=8.0, bg=bg)
    _close(gs.cpu().numpy(), rs, "grad_sigma")
    _close(gh.cpu().numpy(), rh, "grad_sh")
    assert np.all(gs.cpu().numpy()[sig <= 0] == 0)
    # the two-pass variant (forward colour recomputed in the kernel) agrees
    gs2, gh2 = pot.render_backward(t, og, od, gg, rgb_fwd=None, bg=bg, near=0.2, far=8.0)
    _close(gs2.cpu().numpy(), rs, "grad_sigma (two-pass)")
    _close(gh2.cpu().numpy(), rh, "grad_sh (two-pass)")
    pot.check()


@pytest.mark.parametrize("gamma", [0.0, 1e-4])
def test_backward_vs_oracle_main_depth5(pot, oracle_mod, torch_mod, gamma):
    """The optimisation benchmark's setting on a depth-5 copy of the main scene
    (32^3 grid, SH degree 3): a perturbed copy (SH + N(0, 0.3), sigma x
    U(0.5, 1.5)) seen through training cameras on the upper hemisphere (800 x
    800, near 2, far 6), upstream gradient = the MSE gradient against the
    target tree's colours; GPU gradients against the oracle's, 1e-4 x max.
    With gamma > 0 a ray may stop one segment apart on the two sides, so only
    rays whose segment counts agree (decided before either backward) are used."""
    torch = torch_mod
    target_sc = S.scene_shapes(depth=5, sh_degree=3)
    sc = S.perturbed(target_sc, 1003)
    cams = S.cameras_train(n=100)[::25]
    o_all, d_all = oracle_mod.cam_rays(cams)
    pick = np.random.default_rng(5).choice(o_all.shape[0], 30000, replace=False)
    o, d = np.ascontiguousarray(o_all[pick]), np.ascontiguousarray(d_all[pick])
    ot, ot_target = oracle_mod.build_sparse(sc), oracle_mod.build_sparse(target_sc)
    fwd = oracle_mod.render_rays(ot, o, d, near=2.0, far=6.0, gamma=gamma)
    target = oracle_mod.render_rays(ot_target, o, d, near=2.0, far=6.0, gamma=gamma)["rgb"]
    t = pot.Tree.from_scene(sc)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    seg = torch.zeros(o.shape[0], dtype=torch.int32, device="cuda")
    touched = torch.zeros(t.info()["n_leaves"], dtype=torch.uint8, device="cuda")
    pot.render_rays(t, og, od, gamma=gamma, near=2.0, far=6.0, seg_count=seg, leaf_touched=touched)
    keep = seg.cpu().numpy() == fwd["n_seg"]
    if gamma == 0.0:
        assert keep.all()
    assert keep.mean() > 0.99 and (fwd["n_seg"][keep] > 0).sum() > 5000
    o, d = np.ascontiguousarray(o[keep]), np.ascontiguousarray(d[keep])
    g = (2.0 / (3 * o.shape[0])) * (fwd["rgb"][keep] - target[keep])       # MSE gradient (oracle colours)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    gg = torch.from_numpy(g.astype(np.float32)).cuda()
    gs, gh = pot.render_backward(t, og, od, gg, gamma=gamma, near=2.0, far=6.0)
    rs, rh = oracle_mod.backward_rays(ot, o, d, g.astype(np.float32).astype(np.float64), near=2.0, far=6.0,
                                      gamma=gamma)
    assert float(np.abs(rs).max()) > 0 and float(np.abs(rh).max()) > 0
    _close(gs.cpu().numpy(), rs, "grad_sigma")
    _close(gh.cpu().numpy(), rh, "grad_sh")
    pot.check()
    t.free()


def test_backward_vs_gpu_finite_differences(pot, torch_mod):
    """The adjoint against central differences of the GPU render itself, on a
    depth-5 copy of the main scene: L = sum over rays of <g, C>, each sampled
    leaf value moved by +-eps through pot_tree_set_values."""
    torch = torch_mod
    sc = S.scene_shapes(depth=5, sh_degree=3)
    t = pot.Tree.from_scene(sc)
    cams = S.make_cameras(S.orbit_c2ws(3, radius=4.0), 48, 48, 60.0, near=2.0, far=6.0)
    o, d = pot.camera_rays(cams)
    g = torch.from_numpy(np.random.default_rng(9).normal(size=(o.shape[0], 3)).astype(np.float32)).cuda()
    gs, gh = pot.render_backward(t, o, d, g, near=2.0, far=6.0)
    sig0 = torch.from_numpy(sc.sigma.astype(np.float32)).cuda()
    sh0 = torch.from_numpy(sc.sh.astype(np.float32)).cuda()

    def loss(sig, sh):
        t.set_values(sig, sh)
        return float((pot.render_rays(t, o, d, near=2.0, far=6.0).double() * g.double()).sum().item())

    checked = 0
    for which, grad in (("sigma", gs), ("sh", gh)):
        flat = grad.reshape(-1).abs()
        for idx in torch.topk(flat, 4).indices.tolist():
            sig, sh = sig0.clone(), sh0.clone()
            base = (sig if which == "sigma" else sh).reshape(-1)
            x = float(base[idx].item())
            if which == "sigma" and x < 1.0:
                continue
            eps = 1e-3 * max(1.0, abs(x))
            base[idx] = x + eps
            lp = loss(sig, sh)
            base[idx] = x - eps
            lm = loss(sig, sh)
            fd = (lp - lm) / (2 * eps)
            an = float(grad.reshape(-1)[idx].item())
            assert abs(fd - an) <= 2e-2 * abs(an) + 1e-3, (which, idx, fd, an)
            checked += 1
    t.set_values(sig0, sh0)
    assert checked >= 6
    pot.check()


@pytest.mark.parametrize("seed,D,deg,dtype", [(61, 4, 1, "f32"), (62, 5, 3, "f32"), (63, 5, 2, "f16")])
def test_mse_backward_fused(pot, oracle_mod, torch_mod, seed, D, deg, dtype):
    """pot_render_mse_backward = pot_render_rays + pot_loss_mse + pot_render_backward in one
    launch; its gradients also against the oracle's, with the oracle's own MSE gradient."""
    torch = torch_mod
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    ot = oracle_mod.build_sparse(sc, dtype=dtype)
    o, d = S.random_rays(seed, 2503, radius=3.0, spread=0.9)
    target = np.random.default_rng(seed).uniform(size=(o.shape[0], 3)).astype(np.float32)
    og, od, tg = (torch.from_numpy(a).cuda() for a in (o, d, target))
    bg = (0.2, 0.3, 0.4)
    rgb = torch.full((o.shape[0], 3), -1.0, device="cuda")
    loss, gs, gh = pot.render_mse_backward(t, og, od, tg, rgb=rgb, bg=bg, gamma=1e-3, near=0.2, far=8.0)
    ref_rgb = pot.render_rays(t, og, od, bg=bg, gamma=1e-3, near=0.2, far=8.0)
    assert torch.equal(rgb, ref_rgb)                       # the same walk and arithmetic
    ref_loss, g = pot.loss_mse(ref_rgb, tg)
    assert abs(float(loss.item()) - float(ref_loss.item())) <= 1e-5 * float(ref_loss.item())
    rs_, rh_ = pot.render_backward(t, og, od, g, rgb_fwd=ref_rgb, bg=bg, gamma=1e-3, near=0.2, far=8.0)
    assert torch.allclose(gs, rs_, rtol=1e-5, atol=1e-7) and torch.allclose(gh, rh_, rtol=1e-5, atol=1e-7)
    # against the oracle (gamma = 0: no stop decision to share): its colour, its MSE
    # gradient 2 (C - target) / (3 n), its adjoint
    loss, gs, gh = pot.render_mse_backward(t, og, od, tg, bg=bg, near=0.2, far=8.0)
    ref = oracle_mod.render_rays(ot, o, d, near=0.2, far=8.0, bg=bg)["rgb"]
    g64 = 2.0 * (ref - target.astype(np.float64)) / (3 * o.shape[0])
    rs, rh = oracle_mod.backward_rays(ot, o, d, g64, near=0.2, far=8.0, bg=bg)
    _close(gs.cpu().numpy(), rs, "fused grad_sigma")
    _close(gh.cpu().numpy(), rh, "fused grad_sh")
    assert abs(float(loss.item()) - float(((ref - target) ** 2).mean())) <= 1e-4 * float(((ref - target) ** 2).mean())
    # an empty tree: background colour, loss only
    empty = sc.replace(morton=sc.morton[:0], sigma=sc.sigma[:0], sh=sc.sh[:0])
    te = pot.Tree.from_scene(empty, dtype=dtype)
    le, _, _ = pot.render_mse_backward(te, og, od, tg, bg=bg)
    assert abs(float(le.item()) - float(((np.float32(bg) - target) ** 2).mean())) <= 1e-5
    pot.check()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_backward_low_precision_trees(pot, oracle_mod, torch_mod, dtype):
    torch = torch_mod
    sc = S.scene_random(56, 5, 3, p_occ=0.35, sigma_mu=1.5)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    ot = oracle_mod.build_sparse(sc, dtype=dtype)
    o, d = S.random_rays(56, 2000, radius=3.0, spread=0.9)
    g = np.random.default_rng(1).normal(size=(2000, 3)).astype(np.float32)
    gs, gh = pot.render_backward(t, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                                 torch.from_numpy(g).cuda())
    rs, rh = oracle_mod.backward_rays(ot, o, d, g.astype(np.float64))
    _close(gs.cpu().numpy(), rs, f"grad_sigma {dtype}")
    _close(gh.cpu().numpy(), rh, f"grad_sh {dtype}")


def test_backward_tiny_with_early_stop(pot, oracle_mod, torch_mod):
    torch = torch_mod
    sc = S.scene_tiny()
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    cams = S.cameras_tiny("generic")
    o, d = oracle_mod.cam_rays(cams)
    g = np.random.default_rng(2).normal(size=o.shape).astype(np.float32)
    for gamma in (0.0, 0.05):
        gs, gh = pot.render_backward(t, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                                     torch.from_numpy(g).cuda(), gamma=gamma)
        rs, rh = oracle_mod.backward_rays(ot, o, d, g.astype(np.float64), gamma=gamma)
        _close(gs.cpu().numpy(), rs, f"tiny grad_sigma gamma={gamma}")
        _close(gh.cpu().numpy(), rh, f"tiny grad_sh gamma={gamma}")


@pytest.mark.parametrize("kind", ["sgd", "rmsprop", "adam"])
@pytest.mark.parametrize("deg,rem", [(2, 0), (3, 0), (3, 1), (1, 2)])
def test_step_vs_oracle(pot, oracle_mod, torch_mod, kind, deg, rem):
    """deg 2: padded SH records (27 of 28 floats); deg 3 / 1: unpadded records,
    with the leaf count a multiple of 4 (16-byte update path) or not."""
    torch = torch_mod
    sc = S.scene_random(57, 4, deg, p_occ=0.4)
    n = sc.n - (sc.n % 4) + rem if sc.n % 4 >= rem else sc.n - (sc.n % 4) - 4 + rem
    sc = sc.replace(morton=sc.morton[:n], sigma=sc.sigma[:n], sh=sc.sh[:n])
    assert sc.n % 4 == rem
    t = pot.Tree.from_scene(sc)
    L, K = sc.n, sc.sh_dim
    rng = np.random.default_rng(3)
    x_s = sc.sigma.astype(np.float64)
    x_h = sc.sh.astype(np.float64).reshape(L, -1)
    v_s, v_h = np.zeros(L), np.zeros_like(x_h)
    m_s, m_h = np.zeros(L), np.zeros_like(x_h)
    opt = pot.LeafOptimizer(t, kind, lr_sigma=0.05, lr_sh=0.02)
    for it in range(1, 4):
        gs = rng.normal(size=L).astype(np.float32)
        gh = rng.normal(size=(L, K, 3)).astype(np.float32)
        opt.step(torch.from_numpy(gs).cuda(), torch.from_numpy(gh).cuda())
        g_s, g_h = gs.astype(np.float64), gh.astype(np.float64).reshape(L, -1)
        if kind == "sgd":
            x_s, x_h = oracle_mod.step_sgd(x_s, g_s, 0.05), oracle_mod.step_sgd(x_h, g_h, 0.02)
        elif kind == "rmsprop":
            x_s, v_s = oracle_mod.step_rmsprop(x_s, g_s, v_s, 0.05)
            x_h, v_h = oracle_mod.step_rmsprop(x_h, g_h, v_h, 0.02)
        else:
            x_s, m_s, v_s = oracle_mod.step_adam(x_s, g_s, m_s, v_s, it, 0.05)
            x_h, m_h, v_h = oracle_mod.step_adam(x_h, g_h, m_h, v_h, it, 0.02)
    _, sig, sh, _ = t.export()
    assert np.abs(sig - x_s).max() <= 1e-5 * max(1.0, np.abs(x_s).max())
    assert np.abs(sh.reshape(L, -1) - x_h).max() <= 1e-5 * max(1.0, np.abs(x_h).max())


def test_step_rejects_low_precision_tree(pot, torch_mod):
    sc = S.scene_random(58, 3, 0, p_occ=0.5)
    t = pot.Tree.from_scene(sc, dtype="f16")
    gs = torch_mod.zeros(sc.n, device="cuda")
    gh = torch_mod.zeros((sc.n, 1, 3), device="cuda")
    with pytest.raises(pot.PotError) as e:
        pot.step(t, gs, gh, None, "sgd")
    assert e.value.status == pot.POT_ERR_UNSUPPORTED


def test_loss_mse(pot, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(4)
    for n in (1, 1000, 70001):
        a = rng.uniform(size=(n, 3)).astype(np.float32)
        b = rng.uniform(size=(n, 3)).astype(np.float32)
        loss, grad = pot.loss_mse(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
        ref = ((a.astype(np.float64) - b) ** 2).mean()
        assert abs(float(loss.item()) - ref) <= 1e-5 * ref + 1e-9
        assert np.abs(grad.cpu().numpy() - 2 * (a.astype(np.float64) - b) / (3 * n)).max() <= 1e-6 / n + 1e-12


def test_camera_rays_bitexact(pot, oracle_mod, torch_mod):
    cams = np.concatenate([S.cameras_train(n=3, width=40, height=30)])
    o, d = pot.camera_rays(cams)
    ro, rd = oracle_mod.cam_rays(cams)
    assert np.array_equal(o.cpu().numpy(), ro) and np.array_equal(d.cpu().numpy(), rd)
    pix = torch_mod.tensor([0, 5, 1200, 3599, 2 * 1200 + 7], dtype=torch_mod.int64, device="cuda")
    o2, d2 = pot.camera_rays(cams, pixels=pix)
    idx = pix.cpu().numpy()
    assert np.array_equal(d2.cpu().numpy(), rd[idx]) and np.array_equal(o2.cpu().numpy(), ro[idx])
    bad = torch_mod.tensor([3600], dtype=torch_mod.int64, device="cuda")
    with pytest.raises(pot.PotError):
        pot.camera_rays(cams, pixels=bad)


def test_autograd_function(pot, torch_mod):
    torch = torch_mod
    sc = S.scene_random(59, 4, 1, p_occ=0.4)
    t = pot.Tree.from_scene(sc)
    o, d = S.random_rays(9, 500, radius=3.0, spread=0.9)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    sp = torch.zeros(sc.n, device="cuda", requires_grad=True)
    hp = torch.zeros((sc.n, sc.sh_dim, 3), device="cuda", requires_grad=True)
    target = torch.rand((500, 3), device="cuda")
    rgb = pot.render_rays_diff(t, sp, hp, og, od)
    loss = ((rgb - target) ** 2).mean()
    loss.backward()
    g = (2 * (rgb.detach() - target) / rgb.numel()).contiguous()
    gs, gh = pot.render_backward(t, og, od, g, rgb_fwd=rgb.detach())
    assert torch.allclose(sp.grad, gs, rtol=1e-4, atol=1e-7)
    assert torch.allclose(hp.grad, gh, rtol=1e-4, atol=1e-7)


def test_short_optimisation_reduces_loss(pot, torch_mod):
    """Fit a perturbed copy of a tree to renders of the original (Sec. 3.3)."""
    torch = torch_mod
    target_scene = S.scene_random(60, 5, 2, p_occ=0.35, sigma_mu=2.0, sh_std=0.7)
    start = S.perturbed(target_scene, 61, sh_noise=0.3)
    tgt = pot.Tree.from_scene(target_scene)
    t = pot.Tree.from_scene(start)
    cams = S.make_cameras(S.hemisphere_c2ws(62, 12, radius=3.0), 48, 48, 45.0)
    all_o, all_d = pot.camera_rays(cams)
    target = pot.render_rays(tgt, all_o, all_d)
    opt = pot.LeafOptimizer(t, "adam", lr_sigma=0.05, lr_sh=0.02)
    gen = torch.Generator(device="cuda").manual_seed(0)
    losses = []
    for it in range(60):
        idx = torch.randint(0, all_o.shape[0], (8192,), device="cuda", generator=gen)
        o, d, y = all_o[idx].contiguous(), all_d[idx].contiguous(), target[idx].contiguous()
        rgb = pot.render_rays(t, o, d)
        loss, g = pot.loss_mse(rgb, y)
        gs, gh = pot.render_backward(t, o, d, g, rgb_fwd=rgb)
        opt.step(gs, gh)
        losses.append(float(loss.item()))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5]), losses[:5] + losses[-5:]
    pot.check()
