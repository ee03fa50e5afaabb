"""Pins of the oracle's analytic derivatives (App. B.3.2) against central
finite differences and single-leaf closed forms, and of the optimiser steps
against torch.optim (CPU, float64)."""
import math

import numpy as np
import pytest

from paper_2103_14024_gb300 import synth as S

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def _loss(oracle_mod, sc, o, d, g, bg, gamma=0.0):
    t = oracle_mod.build_sparse(sc)
    return float((oracle_mod.render_rays(t, o, d, bg=bg, gamma=gamma)["rgb"] * g).sum())


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.9)])
def test_gradient_vs_finite_differences(oracle_mod, bg):
    sc = S.scene_random(3, 4, 2, p_occ=0.5, sigma_mu=0.8, sigma_s=0.5, sh_std=0.7)
    o, d = S.random_rays(4, 6, radius=3.0, spread=0.4)
    rng = np.random.default_rng(0)
    g = rng.normal(size=(o.shape[0], 3))
    t = oracle_mod.build_sparse(sc)
    gs, gh = oracle_mod.backward_rays(t, o, d, g, bg=bg)
    touched = np.flatnonzero(np.abs(gs) > 0)
    assert touched.size > 10
    # finite differences in float64: perturb the oracle's leaf values through a
    # float64 scene copy (values are passed as float32, so use steps that are
    # exactly representable relative to the values)
    picks = rng.choice(touched, size=min(12, touched.size), replace=False)
    for L in picks:
        for kind in ("sigma", "sh"):
            for trial in range(2 if kind == "sh" else 1):
                j = int(rng.integers(0, sc.sh_dim)) if kind == "sh" else 0
                c = int(rng.integers(0, 3)) if kind == "sh" else 0
                base = float(sc.sigma[L]) if kind == "sigma" else float(sc.sh[L, j, c])
                hstep = 2.0 ** -12 * max(1.0, abs(base))

                def f(val):
                    s2 = sc.replace(sigma=sc.sigma.copy(), sh=sc.sh.copy())
                    if kind == "sigma":
                        s2.sigma[L] = val
                    else:
                        s2.sh[L, j, c] = val
                    return _loss(oracle_mod, s2, o, d, g, bg)

                # values are exactly representable in fp32 (base +- 2^-12 * scale)
                fp, fm = f(np.float32(base + hstep)), f(np.float32(base - hstep))
                h2 = float(np.float32(base + hstep)) - float(np.float32(base - hstep))
                fd = (fp - fm) / h2
                an = gs[L] if kind == "sigma" else gh[L, j, c]
                assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (kind, L, j, c, fd, an)


def test_single_leaf_gradient_closed_form(oracle_mod):
    D, h = 3, 2.0 / 8
    k = np.array([[[0.7, -0.2, 1.3]]], np.float32)
    m = S.morton_encode(np.array([4]), np.array([4]), np.array([4]), D)
    sc = S.Scene(D, (-1.0, -1.0, -1.0), 2.0, 0, m, np.array([3.0], np.float32), k)
    t = oracle_mod.build_sparse(sc)
    o = np.array([[-1 + 4.5 * h, -1 + 4.5 * h, 4.0]], np.float32)
    d = np.array([[0.0, 0.0, -1.0]], np.float32)
    g = np.array([[1.0, -2.0, 0.5]])
    gs, gh = oracle_mod.backward_rays(t, o, d, g)
    c = 1 / (1 + np.exp(-k[0, 0].astype(np.float64) * Y00))
    delta = h
    dC_dsigma = c * delta * math.exp(-3.0 * delta)              # bg = 0
    w = 1 - math.exp(-3.0 * delta)
    dC_dk = w * c * (1 - c) * Y00
    assert gs[0] == pytest.approx(float((g[0] * dC_dsigma).sum()), abs=1e-14)
    assert np.allclose(gh[0, 0], g[0] * dC_dk, atol=1e-14)


def test_relu_zero_gradient_for_nonpositive_sigma(oracle_mod):
    sc = S.scene_random(8, 3, 1, p_occ=0.7)
    sig = sc.sigma.copy()
    sig[::3] = -np.abs(sig[::3])
    sig[1::7] = 0.0
    sc = sc.replace(sigma=sig)
    t = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(12, 100, radius=3.0, spread=0.5)
    gs, gh = oracle_mod.backward_rays(t, o, d, np.ones((100, 3)))
    assert np.all(gs[sig <= 0] == 0)
    assert np.abs(gs[sig > 0]).sum() > 0
    # a non-positive sigma renders as 0: fully transparent, no colour contribution
    r = oracle_mod.render_rays(t, o, d)
    sc2 = sc.replace(sigma=np.maximum(sig, 0))
    r2 = oracle_mod.render_rays(oracle_mod.build_sparse(sc2), o, d)
    assert np.array_equal(r["rgb"], r2["rgb"])


def test_rmsprop_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(5)]
    p = torch.nn.Parameter(torch.tensor(x0, dtype=torch.float64))
    opt = torch.optim.RMSprop([p], lr=0.1, alpha=0.99, eps=1e-8)
    x, v = x0.copy(), np.zeros(50)
    for g in grads:
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        x, v = oracle_mod.step_rmsprop(x, g, v, lr=0.1, alpha=0.99, eps=1e-8)
    assert np.allclose(x, p.detach().numpy(), rtol=0, atol=1e-12)


def test_adam_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x0 = rng.normal(size=40)
    grads = [rng.normal(size=40) for _ in range(6)]
    p = torch.nn.Parameter(torch.tensor(x0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    x, m, v = x0.copy(), np.zeros(40), np.zeros(40)
    for s, g in enumerate(grads, 1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        x, m, v = oracle_mod.step_adam(x, g, m, v, s, lr=0.05)
    assert np.allclose(x, p.detach().numpy(), rtol=0, atol=1e-12)


def test_sgd_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    x0 = np.linspace(-1, 1, 9)
    g = np.cos(x0)
    p = torch.nn.Parameter(torch.tensor(x0, dtype=torch.float64))
    opt = torch.optim.SGD([p], lr=0.3)
    p.grad = torch.tensor(g, dtype=torch.float64)
    opt.step()
    assert np.allclose(oracle_mod.step_sgd(x0, g, 0.3), p.detach().numpy(), atol=1e-15)


def test_gradient_vs_finite_differences_with_early_stop(oracle_mod):
    """gamma > 0 (Sec. 3.2 early stop): segments after the stop neither shade
    nor receive gradient.  Central differences of the oracle's render, only
    for perturbations that leave every ray's stop segment where it was."""
    sc = S.scene_random(21, 4, 1, p_occ=0.6, sigma_mu=2.5, sigma_s=0.5, sh_std=0.7)
    o, d = S.random_rays(22, 40, radius=3.0, spread=0.4)
    gamma, bg = 0.05, (0.2, 0.4, 0.6)
    g = np.random.default_rng(1).normal(size=(o.shape[0], 3))
    t = oracle_mod.build_sparse(sc)
    base = oracle_mod.render_rays(t, o, d, bg=bg, gamma=gamma)
    full = oracle_mod.render_rays(t, o, d, bg=bg, gamma=0.0)
    assert (base["n_seg"] < full["n_seg"]).sum() >= 5           # some rays do stop early
    gs, gh = oracle_mod.backward_rays(t, o, d, g, bg=bg, gamma=gamma)
    rng = np.random.default_rng(2)
    touched = np.flatnonzero(np.abs(gs) > 0)
    checked = 0
    for L in rng.choice(touched, size=min(16, touched.size), replace=False):
        for kind in ("sigma", "sh"):
            j, c = (int(rng.integers(0, sc.sh_dim)), int(rng.integers(0, 3))) if kind == "sh" else (0, 0)
            val = float(sc.sigma[L]) if kind == "sigma" else float(sc.sh[L, j, c])
            hstep = 2.0 ** -14 * max(1.0, abs(val))
            outs = []
            for v in (np.float32(val + hstep), np.float32(val - hstep)):
                s2 = sc.replace(sigma=sc.sigma.copy(), sh=sc.sh.copy())
                if kind == "sigma":
                    s2.sigma[L] = v
                else:
                    s2.sh[L, j, c] = v
                outs.append(oracle_mod.render_rays(oracle_mod.build_sparse(s2), o, d, bg=bg, gamma=gamma))
            if not all(np.array_equal(r["n_seg"], base["n_seg"]) for r in outs):
                continue                                         # a stop decision moved: not differentiable here
            h2 = float(np.float32(val + hstep)) - float(np.float32(val - hstep))
            fd = float(((outs[0]["rgb"] - outs[1]["rgb"]) * g).sum()) / h2
            an = gs[L] if kind == "sigma" else gh[L, j, c]
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (kind, L, j, c, fd, an)
            checked += 1
    assert checked >= 16


@pytest.mark.parametrize("gamma", [0.0, 0.05])
def test_gradient_vs_autograd_of_compositing(oracle_mod, gamma):
    """The analytic two-pass derivatives (App. B.3.2) against torch float64
    automatic differentiation of the compositing sum (Eq. 1 with the ReLU on
    sigma, the sigmoid of the SH expansion and the background term) over the
    oracle's own segment lists."""
    torch = pytest.importorskip("torch")
    sc = S.scene_random(23, 4, 2, p_occ=0.5, sigma_mu=1.5, sigma_s=0.8, sh_std=0.7)
    sig = sc.sigma.copy()
    sig[::9] = -np.abs(sig[::9])                                 # some non-positive densities
    sc = sc.replace(sigma=sig)
    t = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(24, 30, radius=3.0, spread=0.4)
    bg = (0.1, 0.5, 0.9)
    g = np.random.default_rng(3).normal(size=(o.shape[0], 3))
    gs, gh = oracle_mod.backward_rays(t, o, d, g, bg=bg, gamma=gamma)
    sigma = torch.tensor(sc.sigma.astype(np.float64), requires_grad=True)
    sh = torch.tensor(sc.sh.astype(np.float64), requires_grad=True)
    loss = torch.zeros((), dtype=torch.float64)
    for r in range(o.shape[0]):
        leaf, _, _, dl = oracle_mod.trace_ray(t, o[r], d[r])
        dn = d[r].astype(np.float64) / np.linalg.norm(d[r].astype(np.float64))
        Y = torch.tensor(oracle_mod.sh_basis(sc.sh_dim, dn[None])[0])
        T = torch.ones((), dtype=torch.float64)
        C = torch.zeros(3, dtype=torch.float64)
        for lf, de in zip(leaf, dl):
            if lf < 0 or de <= 0:
                continue
            a = 1.0 - torch.exp(-torch.relu(sigma[lf]) * de)
            col = torch.sigmoid(Y @ sh[lf])
            C = C + T * a * col
            T = T * (1.0 - a)
            if gamma > 0 and float(T.detach()) < gamma:
                break
        C = C + T * torch.tensor(bg, dtype=torch.float64)
        loss = loss + (C * torch.tensor(g[r])).sum()
    loss.backward()
    assert np.abs(sigma.grad.numpy()).max() > 0
    assert np.allclose(gs, sigma.grad.numpy(), rtol=1e-9, atol=1e-12)
    assert np.allclose(gh, sh.grad.numpy(), rtol=1e-9, atol=1e-12)
