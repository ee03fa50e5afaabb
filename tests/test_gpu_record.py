"""GPU parity of the recorded-segment training path (App. B.3.2 derivatives,
Sec. 3.3): pot_render_rays_record renders exactly what pot_render_rays renders
and records every composited leaf segment (ray, leaf, delta_i, T_i, P_i);
pot_render_backward_recorded differentiates the records one by one.

Checks: colours and transmittances bit-identical to pot_render_rays; the
records against the oracle's segment lists with T_i and P_i composited from
them (Eq. 1); gradients against the oracle's (1e-4 x max) and against the
walking backward (the same per-segment terms, summed in another order); the
overflow fallback; argument checks; the autograd Function with records."""
import ctypes as C

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


def _close(gpu, ref, name, rel=REL):
    scale = max(float(np.abs(ref).max()), 1e-12)
    err = float(np.abs(gpu - ref).max())
    assert err <= rel * scale, f"{name}: max err {err:.3e} vs scale {scale:.3e}"


def _records_by_ray(rec_np, used, n):
    """Records of each ray, in slot order (= compositing order), as a dict ray -> float32 [m, 8]."""
    r = rec_np[:used]
    ray = r[:, 0].view(np.int32)
    live = ray >= 0
    out = {}
    idx = np.nonzero(live)[0]
    order = idx[np.argsort(ray[idx], kind="stable")]
    rs = ray[order]
    bounds = np.flatnonzero(np.diff(rs)) + 1
    for grp in np.split(order, bounds):
        if len(grp):
            out[int(ray[grp[0]])] = r[grp]
    assert all(0 <= k < n for k in out)
    return out


@pytest.mark.parametrize("seed,D,deg,dtype", [(71, 4, 0, "f32"), (72, 5, 1, "f32"), (73, 5, 3, "f32"),
                                              (74, 6, 2, "f16"), (75, 5, 4, "bf16")])
@pytest.mark.parametrize("gamma", [0.0, 1e-3])
def test_record_forward_equals_render_rays(pot, torch_mod, seed, D, deg, dtype, gamma):
    """Colours and final transmittances bit-identical to pot_render_rays; one
    record per composited segment (the counting render's per-ray counts)."""
    torch = torch_mod
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    o, d = S.random_rays(seed, 4001, radius=3.0, spread=0.9)   # ragged: 4001 = 125 tiles + 1 ray
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    bg = (0.1, 0.5, 0.9)
    ref, ref_t = pot.render_rays(t, og, od, bg=bg, gamma=gamma, near=0.2, far=8.0, want_t_final=True)
    recs = pot.SegmentRecords.for_rays(o.shape[0], 32)
    rgb, tf = pot.render_rays_record(t, og, od, recs, bg=bg, gamma=gamma, near=0.2, far=8.0, want_t_final=True)
    assert torch.equal(rgb, ref) and torch.equal(tf, ref_t)
    assert not recs.overflowed()
    used = recs.used()
    assert used % pot.SEGMENT_BLOCK == 0 and used <= recs.capacity
    seg = torch.zeros(o.shape[0], dtype=torch.int32, device="cuda")
    touched = torch.zeros(t.info()["n_leaves"], dtype=torch.uint8, device="cuda")
    pot.render_rays(t, og, od, bg=bg, gamma=gamma, near=0.2, far=8.0, seg_count=seg, leaf_touched=touched)
    by_ray = _records_by_ray(recs.records.cpu().numpy(), used, o.shape[0])
    counts = np.zeros(o.shape[0], dtype=np.int64)
    for k, v in by_ray.items():
        counts[k] = v.shape[0]
    assert np.array_equal(counts, seg.cpu().numpy().astype(np.int64))
    assert counts.sum() > 1000
    pot.check()


@pytest.mark.parametrize("seed,D,deg", [(81, 4, 1), (82, 5, 3)])
def test_records_vs_oracle_segments(pot, oracle_mod, torch_mod, seed, D, deg):
    """Each ray's records against the oracle's segment list (leaf ids exact,
    lengths to 1e-5 relative), with T_i and P_i composited in float64 from the
    oracle's segments (Eq. 1; ReLU on sigma; sigmoid of the SH expansion),
    T_i to 2e-5 relative and P_i to 2e-5 (fp32 products of up to ~60 factors)."""
    torch = torch_mod
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(seed, 600, radius=3.0, spread=0.9)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    recs = pot.SegmentRecords(600 * 64 + 64 * pot.SEGMENT_BLOCK)
    pot.render_rays_record(t, og, od, recs, near=0.2, far=8.0)
    by_ray = _records_by_ray(recs.records.cpu().numpy(), recs.used(), o.shape[0])
    K = sc.sh_dim
    sig64, sh64 = sc.sigma.astype(np.float64), sc.sh.astype(np.float64)
    checked = 0
    for r in range(o.shape[0]):
        leaf, _, _, dl = oracle_mod.trace_ray(ot, o[r], d[r], near=0.2, far=8.0)
        keep = (leaf >= 0) & (dl > 0)
        leaf, dl = leaf[keep], dl[keep]
        got = by_ray.get(r, np.zeros((0, 8), np.float32))
        assert got.shape[0] == leaf.shape[0], r
        if not leaf.shape[0]:
            continue
        assert np.array_equal(got[:, 1].view(np.int32).astype(np.int64), leaf), r
        assert np.allclose(got[:, 2], dl, rtol=1e-5, atol=1e-9), r
        dn = d[r].astype(np.float64) / np.linalg.norm(d[r].astype(np.float64))
        Y = oracle_mod.sh_basis(K, dn[None])[0]
        T, P = 1.0, np.zeros(3)
        for i, (lf, de) in enumerate(zip(leaf, dl)):
            assert abs(got[i, 3] - T) <= 2e-5 * T + 1e-6, (r, i)
            assert np.all(np.abs(got[i, 4:7] - P) <= 2e-5), (r, i)
            e = np.exp(-max(sig64[lf], 0.0) * de)
            c = 1.0 / (1.0 + np.exp(-(Y @ sh64[lf])))
            P = P + T * (1.0 - e) * c
            T *= e
        checked += 1
    assert checked > 100
    pot.check()


@pytest.mark.parametrize("seed,D,deg,dtype", [(91, 3, 0, "f32"), (92, 4, 1, "f32"), (93, 5, 2, "f32"),
                                              (94, 5, 3, "f32"), (95, 6, 3, "f16"), (96, 5, 4, "bf16")])
@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.9)])
def test_backward_recorded_vs_oracle(pot, oracle_mod, torch_mod, seed, D, deg, dtype, bg):
    torch = torch_mod
    sc = S.scene_random(seed, D, deg, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    sig = sc.sigma.copy()
    sig[::11] = -sig[::11]                     # some non-positive densities (zero gradient)
    sc = sc.replace(sigma=sig)
    t = pot.Tree.from_scene(sc, dtype=dtype)
    ot = oracle_mod.build_sparse(sc, dtype=dtype)
    o, d = S.random_rays(seed, 3001, radius=3.0, spread=0.9)
    g = np.random.default_rng(seed).normal(size=(o.shape[0], 3)).astype(np.float32)
    g[::7] = 0.0                               # rays without an upstream gradient
    og, od, gg = (torch.from_numpy(a).cuda() for a in (o, d, g))
    recs = pot.SegmentRecords.for_rays(o.shape[0], 32)
    rgb = pot.render_rays_record(t, og, od, recs, bg=bg, near=0.2, far=8.0)
    gs, gh = pot.render_backward_recorded(t, og, od, gg, rgb, recs, bg=bg, near=0.2, far=8.0)
    assert not recs.overflowed()
    rs, rh = oracle_mod.backward_rays(ot, o, d, g.astype(np.float64), near=0.2, far=8.0, bg=bg)
    _close(gs.cpu().numpy(), rs, "grad_sigma")
    _close(gh.cpu().numpy(), rh, "grad_sh")
    assert np.all(gs.cpu().numpy()[sig <= 0] == 0)
    # the walking backward: the same per-segment terms, another summation order
    ws, wh = pot.render_backward(t, og, od, gg, rgb_fwd=rgb, bg=bg, near=0.2, far=8.0)
    _close(gs.cpu().numpy(), ws.cpu().numpy(), "grad_sigma vs walking", rel=1e-5)
    _close(gh.cpu().numpy(), wh.cpu().numpy(), "grad_sh vs walking", rel=1e-5)
    pot.check()


@pytest.mark.parametrize("capacity", [0, 128, 1000])
def test_backward_recorded_overflow_falls_back(pot, oracle_mod, torch_mod, capacity):
    """Too few slots: the forward's colours stay exact, the overflow flag is
    set, and the backward's walking fallback gives the oracle's gradients."""
    torch = torch_mod
    sc = S.scene_random(97, 5, 2, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    t = pot.Tree.from_scene(sc)
    ot = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(97, 5000, radius=3.0, spread=0.9)
    g = np.random.default_rng(97).normal(size=(o.shape[0], 3)).astype(np.float32)
    og, od, gg = (torch.from_numpy(a).cuda() for a in (o, d, g))
    recs = pot.SegmentRecords(capacity)
    rgb = pot.render_rays_record(t, og, od, recs, gamma=1e-3, near=0.2, far=8.0)
    assert torch.equal(rgb, pot.render_rays(t, og, od, gamma=1e-3, near=0.2, far=8.0))
    assert recs.overflowed()
    gs, gh = pot.render_backward_recorded(t, og, od, gg, rgb, recs, gamma=1e-3, near=0.2, far=8.0)
    ws, wh = pot.render_backward(t, og, od, gg, rgb_fwd=rgb, gamma=1e-3, near=0.2, far=8.0)
    _close(gs.cpu().numpy(), ws.cpu().numpy(), "fallback grad_sigma vs walking", rel=1e-5)
    _close(gh.cpu().numpy(), wh.cpu().numpy(), "fallback grad_sh vs walking", rel=1e-5)
    # gamma = 0 against the oracle
    rgb = pot.render_rays_record(t, og, od, recs, near=0.2, far=8.0)
    gs, gh = pot.render_backward_recorded(t, og, od, gg, rgb, recs, near=0.2, far=8.0)
    rs, rh = oracle_mod.backward_rays(ot, o, d, g.astype(np.float64), near=0.2, far=8.0)
    _close(gs.cpu().numpy(), rs, "fallback grad_sigma")
    _close(gh.cpu().numpy(), rh, "fallback grad_sh")
    pot.check()


@pytest.mark.parametrize("gamma", [0.0, 1e-4])
def test_backward_recorded_main_depth5(pot, torch_mod, gamma):
    """The optimisation benchmark's setting on a depth-5 copy of the main scene
    (perturbed tree, training cameras, 30 000 random pixels, MSE upstream
    gradient): recorded gradients against the walking backward's."""
    torch = torch_mod
    target_sc = S.scene_shapes(depth=5, sh_degree=3)
    sc = S.perturbed(target_sc, 1003)
    cams = S.cameras_train(n=100)[::10]
    o_all, d_all = pot.camera_rays(cams)
    pick = torch.from_numpy(np.sort(np.random.default_rng(6).choice(o_all.shape[0], 30000, replace=False))).cuda()
    o, d = o_all[pick].contiguous(), d_all[pick].contiguous()
    t, tt = pot.Tree.from_scene(sc), pot.Tree.from_scene(target_sc)
    target = pot.render_rays(tt, o, d, gamma=gamma, near=2.0, far=6.0)
    recs = pot.SegmentRecords.for_rays(o.shape[0])
    rgb = pot.render_rays_record(t, o, d, recs, gamma=gamma, near=2.0, far=6.0)
    _, g = pot.loss_mse(rgb, target)
    gs, gh = pot.render_backward_recorded(t, o, d, g, rgb, recs, gamma=gamma, near=2.0, far=6.0)
    assert not recs.overflowed()
    ws, wh = pot.render_backward(t, o, d, g, rgb_fwd=rgb, gamma=gamma, near=2.0, far=6.0)
    assert float(ws.abs().max()) > 0 and float(wh.abs().max()) > 0
    _close(gs.cpu().numpy(), ws.cpu().numpy(), "grad_sigma vs walking", rel=1e-5)
    _close(gh.cpu().numpy(), wh.cpu().numpy(), "grad_sh vs walking", rel=1e-5)
    pot.check()


@pytest.mark.parametrize("cells", ["none", "brick"])
def test_record_path_without_dense_index(pot, torch_mod, cells):
    """The recording forward and the recorded backward on a tree located by
    the child-array descent (no cell index: the walker's ancestor stack in
    dynamic shared memory) and by the brick layout of the index: colours
    bit-identical to pot_render_rays, gradients equal to the walking
    backward's."""
    torch = torch_mod
    sc = S.scene_random(88, 6, 3, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
    t = pot.Tree.from_scene(sc)
    t.set_cell_index(cells)
    o, d = S.random_rays(88, 3001, radius=3.0, spread=0.9)
    g = np.random.default_rng(88).normal(size=(o.shape[0], 3)).astype(np.float32)
    og, od, gg = (torch.from_numpy(a).cuda() for a in (o, d, g))
    ref = pot.render_rays(t, og, od, gamma=1e-3, near=0.2, far=8.0)
    recs = pot.SegmentRecords.for_rays(o.shape[0], 32)
    rgb = pot.render_rays_record(t, og, od, recs, gamma=1e-3, near=0.2, far=8.0)
    assert torch.equal(rgb, ref) and not recs.overflowed()
    gs, gh = pot.render_backward_recorded(t, og, od, gg, rgb, recs, gamma=1e-3, near=0.2, far=8.0)
    ws, wh = pot.render_backward(t, og, od, gg, rgb_fwd=rgb, gamma=1e-3, near=0.2, far=8.0)
    assert float(ws.abs().max()) > 0
    _close(gs.cpu().numpy(), ws.cpu().numpy(), f"grad_sigma vs walking ({cells})", rel=1e-5)
    _close(gh.cpu().numpy(), wh.cpu().numpy(), f"grad_sh vs walking ({cells})", rel=1e-5)
    pot.check()


def test_record_path_empty_tree_and_misses(pot, torch_mod):
    """An empty tree: background colours, no records, zero gradients; rays
    that miss a non-empty tree add no records either."""
    torch = torch_mod
    sc = S.scene_random(89, 4, 1, p_occ=0.35)
    empty = sc.replace(morton=sc.morton[:0], sigma=sc.sigma[:0], sh=sc.sh[:0])
    te = pot.Tree.from_scene(empty)
    o, d = S.random_rays(89, 500, radius=3.0, spread=0.9)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    recs = pot.SegmentRecords.for_rays(500, 8)
    bg = (0.25, 0.5, 0.75)
    rgb = pot.render_rays_record(te, og, od, recs, bg=bg, near=0.2, far=8.0)
    assert torch.equal(rgb, torch.tensor(bg, device="cuda").expand(500, 3))
    assert recs.used() == 0 and not recs.overflowed()
    gs, gh = pot.render_backward_recorded(te, og, od, torch.ones_like(rgb), rgb, recs, bg=bg, near=0.2, far=8.0)
    assert gs.numel() == 0 and gh.numel() == 0
    t = pot.Tree.from_scene(sc)
    away = torch.tensor([[0.0, 0.0, 1.0]], device="cuda").expand(500, 3).contiguous()
    orig = torch.tensor([[0.0, 0.0, 5.0]], device="cuda").expand(500, 3).contiguous()   # pointing away
    pot.render_rays_record(t, orig, away, recs, near=0.0, far=8.0)
    assert recs.used() == 0
    pot.check()


def test_recorded_autograd(pot, torch_mod):
    """render_rays_diff with records: the gradients of the walking autograd path."""
    torch = torch_mod
    sc = S.scene_random(98, 5, 3, p_occ=0.35)
    t = pot.Tree.from_scene(sc)
    o, d = S.random_rays(98, 2000, radius=3.0, spread=0.9)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    target = torch.rand((2000, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    grads = []
    for records in (None, pot.SegmentRecords.for_rays(2000, 32)):
        ps = torch.zeros(sc.n, device="cuda", requires_grad=True)
        ph = torch.zeros((sc.n, sc.sh_dim, 3), device="cuda", requires_grad=True)
        rgb = pot.render_rays_diff(t, ps, ph, og, od, bg=(0.2, 0.2, 0.2), gamma=1e-4, near=0.2, far=8.0,
                                   records=records)
        ((rgb - target) ** 2).mean().backward()
        grads.append((ps.grad.cpu().numpy(), ph.grad.cpu().numpy()))
    _close(grads[1][0], grads[0][0], "autograd grad_sigma", rel=1e-5)
    _close(grads[1][1], grads[0][1], "autograd grad_sh", rel=1e-5)


def test_record_argument_checks(pot, torch_mod):
    """Rejected before any launch: host arrays, a misaligned record buffer, a
    negative capacity, a codebook tree; n = 0 clears the state and is a no-op."""
    torch = torch_mod
    L = pot.lib()
    sc = S.scene_random(99, 4, 1, p_occ=0.35)
    t = pot.Tree.from_scene(sc)
    o, d = S.random_rays(99, 64, radius=3.0, spread=0.9)
    og, od = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    rgb = torch.empty((64, 3), device="cuda")
    recs = pot.SegmentRecords(4096)
    opts = pot._opts(near=0.2, far=8.0)
    P = pot._ptr

    def call(o_=og, d_=od, rgb_=rgb, rec=P(recs.records), cap=recs.capacity, state=P(recs.state), tree=t):
        return L.pot_render_rays_record(tree.handle, 64, P(o_), P(d_), C.byref(opts), P(rgb_), None, rec, cap,
                                        state, pot._stream())

    assert call() == pot.POT_OK
    torch.cuda.synchronize()
    assert call(o_=o) == 1                                        # host origins
    assert call(rgb_=np.zeros((64, 3), np.float32)) == 1           # host output
    host_state = recs.state.cpu()
    assert call(state=P(host_state)) == 1                         # host state
    assert call(rec=C.c_void_p(recs.records.data_ptr() + 4)) == 1  # misaligned records
    assert call(cap=-1) == 1
    cb = t.quantize(bits=8)
    assert call(tree=cb) == 6                                     # POT_ERR_UNSUPPORTED
    gg = torch.zeros((64, 3), device="cuda")
    gs = torch.zeros(sc.n, device="cuda")
    gh = torch.zeros((sc.n, sc.sh_dim, 3), device="cuda")
    st = L.pot_render_backward_recorded(t.handle, 64, P(og), P(od), P(gg), P(o), C.byref(opts), P(recs.records),
                                        recs.capacity, P(recs.state), P(gs), P(gh), pot._stream())
    assert st == 1                                                # host rgb_fwd
    # grad_sh rows are added in 16-byte vectors (3K = 12 floats here): a
    # misaligned gradient array is refused by every backward before any launch
    t3 = pot.Tree.from_scene(S.scene_random(99, 4, 1, p_occ=0.35))
    gh_buf = torch.zeros(t3.info()["n_leaves"] * 12 + 4, device="cuda")
    bad = C.c_void_p(gh_buf.data_ptr() + 4)
    st = L.pot_render_backward_recorded(t3.handle, 64, P(og), P(od), P(gg), P(rgb), C.byref(opts), P(recs.records),
                                        recs.capacity, P(recs.state), P(gs), bad, pot._stream())
    assert st == 1
    assert L.pot_render_backward(t3.handle, 64, P(og), P(od), P(gg), P(rgb), C.byref(opts), P(gs), bad,
                                 pot._stream()) == 1
    loss = torch.zeros(1, device="cuda")
    assert L.pot_render_mse_backward(t3.handle, 64, P(og), P(od), P(gg), C.byref(opts), None, P(loss), P(gs), bad,
                                     pot._stream()) == 1
    recs.state.fill_(7)
    assert L.pot_render_rays_record(t.handle, 0, None, None, C.byref(opts), None, None, P(recs.records),
                                    recs.capacity, P(recs.state), pot._stream()) == pot.POT_OK
    assert recs.state.cpu().tolist() == [0, 0]
    pot.check()


def test_backward_recorded_slot_order(pot):
    """The per-record backward visiting the records in slot order
    (POT_SEGBWD_ORDER=0, read once per process, so it runs in a child
    process) against the walking backward."""
    import os
    import subprocess
    import sys
    code = r'''
import numpy as np, torch
import paper_2103_14024_gb300 as pot
from paper_2103_14024_gb300 import synth as S
sc = S.scene_random(93, 5, 3, p_occ=0.35, sigma_mu=1.5, sigma_s=1.0, sh_std=0.8)
t = pot.Tree.from_scene(sc)
o, d = S.random_rays(93, 3001, radius=3.0, spread=0.9)
g = np.random.default_rng(93).normal(size=(o.shape[0], 3)).astype(np.float32)
og, od, gg = (torch.from_numpy(a).cuda() for a in (o, d, g))
recs = pot.SegmentRecords.for_rays(o.shape[0], 32)
rgb = pot.render_rays_record(t, og, od, recs, gamma=1e-3, near=0.2, far=8.0)
gs, gh = pot.render_backward_recorded(t, og, od, gg, rgb, recs, gamma=1e-3, near=0.2, far=8.0)
ws, wh = pot.render_backward(t, og, od, gg, rgb_fwd=rgb, gamma=1e-3, near=0.2, far=8.0)
es = float((gs - ws).abs().max() / ws.abs().max()); eh = float((gh - wh).abs().max() / wh.abs().max())
assert not recs.overflowed() and es <= 1e-5 and eh <= 1e-5, (es, eh)
pot.check()
print("ok")
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, POT_SEGBWD_ORDER="0")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
