#!/usr/bin/env python3
"""Benchmark of the PlenOctree per-ray render path on GB300.

One step = ``pot_render`` of the main workload: a depth-9 octree (512^3
effective grid) over [-1.5, 1.5]^3 holding ~4.05 M leaves with SH degree 3,
rendered from 200 orbit cameras of 800 x 800 (128 M rays), early stop at
T < 1e-4 (the configuration the paper's synthetic-scene FPS is quoted on,
Sec. 4.1 / Table 1, with synthetic content).

Prints one JSON line (rank 0).  ``value`` is whole-job Mrays/s with the tree
resident in HBM; ``e2e`` is the same metric through the C ABI with the cameras
and the output image in host memory (copies inside the timed region).
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s @800^2 SH-3 (200 views, depth-9 octree, gamma 1e-4)"
UNIT = "Mrays/s"
N_VIEWS, W, H, GAMMA = 200, 800, 800, 1e-4

# Per-launch counters of the render kernel from ncu captures (metrics
# gpu__time_duration, dram__bytes_read/write, lts__t_bytes, smsp__inst_executed,
# l1tex__data_pipe_lsu_wavefronts and its fraction of peak, smsp__issue_active)
# of one 16-view group of the benchmark launch (the 200-view launch renders
# 12.5 such groups, and every counter grows with the groups rendered).  Used only while the kernel sources still
# hash to ``sha``; a changed kernel reports null until it is captured again.
NCU_VIEWS = 16
SHA = "df117c6dfe79ca1d"
NCU_PROFILE = {
    "f32": {"sha": SHA, "dram_read": 1968329728, "dram_write": 106194176,
             "lts_bytes": 28113234944, "warp_inst": 3258636500,
             "l1_wavefronts": 939874052, "l1_pct": 82.33,
             "issue_pct": 72.04, "ncu_ms": 3.6316},
    "f16": {"sha": SHA, "dram_read": 592667392, "dram_write": 102915840,
             "lts_bytes": 14323976192, "warp_inst": 3431872882,
             "l1_wavefronts": 629640129, "l1_pct": 60.18,
             "issue_pct": 83.05, "ncu_ms": 3.3277},
    "bf16": {"sha": SHA, "dram_read": 613072128, "dram_write": 103311616,
             "lts_bytes": 14361677088, "warp_inst": 3431863482,
             "l1_wavefronts": 629176102, "l1_pct": 57.25,
             "issue_pct": 79.09, "ncu_ms": 3.495},
    "cb16": {"sha": SHA, "dram_read": 5433897472, "dram_write": 100167936,
             "lts_bytes": 80758678112, "warp_inst": 3999652230,
             "l1_wavefronts": 1547808887, "l1_pct": 72.23,
             "issue_pct": 47.13, "ncu_ms": 6.8142},
    "f32-descent": {"sha": SHA, "dram_read": 1519985920, "dram_write": 104544512,
             "lts_bytes": 28638647616, "warp_inst": 4770991233,
             "l1_wavefronts": 1052478544, "l1_pct": 61.03,
             "issue_pct": 70.13, "ncu_ms": 5.4848},
    "f32-brick": {"sha": SHA, "dram_read": 1599089152, "dram_write": 103660288,
             "lts_bytes": 26551277472, "warp_inst": 3495248667,
             "l1_wavefronts": 963427507, "l1_pct": 79.18,
             "issue_pct": 72.52, "ncu_ms": 3.8703},
    "f16-brick": {"sha": SHA, "dram_read": 394305536, "dram_write": 101286144,
             "lts_bytes": 13219991296, "warp_inst": 3669975306,
             "l1_wavefronts": 655773496, "l1_pct": 58.08,
             "issue_pct": 82.22, "ncu_ms": 3.5903},
}


# the files compiled into the render kernel (a change anywhere else in the
# library leaves its DRAM counters valid)
KERNEL_SOURCES = ("csrc/pot_device.cuh", "csrc/pot_internal.h", "csrc/pot_render.cuh", "csrc/pot_render_f32.cu",
                  "csrc/pot_render_f16.cu", "csrc/pot_render_bf16.cu", "csrc/pot_render_cb16.cu")


def kernel_sha() -> str:
    """Hash of the render kernel's sources and the public header, comments and
    white space left out (a change of wording does not change the kernel)."""
    import re
    h = hashlib.sha256()
    files = [os.path.join(ROOT, "paper_2103_14024_gb300", f) for f in KERNEL_SOURCES]
    for f in files + [os.path.join(ROOT, "include", "pot.h")]:
        with open(f, encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        src = " ".join(src.split())
        h.update(os.path.basename(f).encode())
        h.update(src.encode())
    return h.hexdigest()[:16]


def max_over_ranks(torch, dist, value: float, device) -> float:
    """Max of a per-rank float over the process group (identity without one)."""
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, rays_per_rank_step: int, wall_max: float, steps: int) -> float:
    """Whole-job Mrays/s when every rank renders the same number of rays per step:
    the rays all ranks rendered per step / the slowest rank's step time."""
    return world * rays_per_rank_step / (wall_max / steps) / 1e6


def view_slice(rank: int, world: int, n_views: int):
    """Views [start, end) that ``rank`` renders when the cameras are partitioned:
    contiguous, balanced (sizes differ by at most one), disjoint, covering all
    views; contiguous so that a rank's neighbouring views share leaves in L2."""
    return n_views * rank // world, n_views * (rank + 1) // world


def job_rays_per_step(partition: str, world: int, n_views: int, rays_per_view: int) -> int:
    """Rays the whole job renders per step: each ray once when the views are
    partitioned, once per rank when every rank renders all of them."""
    return n_views * rays_per_view * (world if partition == "replicate" else 1)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_rays(cams, views, every):
    """Pixel indices of a bounded sample: every ``every``-th pixel of ``views``."""
    import numpy as np
    ci, px, py = [], [], []
    for v in views:
        idx = np.arange(0, W * H, every)
        ci.append(np.full(idx.shape, v))
        px.append(idx % W)
        py.append(idx // W)
    return np.concatenate(ci), np.concatenate(px), np.concatenate(py)


def run_oracle_timing(scene, cams, views, every, steps=1, chunk_views=8):
    """Times the oracle (as it stands) on the bounded sample, ``chunk_views`` views per call so
    that host memory stays small; returns (rays/s, rays per step, seconds, threads)."""
    from oracle import oracle
    ot = oracle.build_sparse(scene)
    n, dt = 0, 0.0
    for _ in range(steps):
        for c in range(0, len(views), chunk_views):
            ci, px, py = oracle_sample_rays(cams, views[c:c + chunk_views], every)
            t0 = time.perf_counter()
            oracle.render_pixels(ot, cams, ci, px, py, gamma=GAMMA)
            dt += time.perf_counter() - t0
            n += ci.shape[0]
    return n / dt, n // steps, dt, oracle.num_threads()


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from paper_2103_14024_gb300 import synth
    scene = synth.scene_shapes()
    cams = synth.cameras_main(N_VIEWS, W, H)
    views = [0]
    every = 1
    for _ in range(args.warmup):
        run_oracle_timing(scene, cams, views, every)
    rate, n, dt, thr = run_oracle_timing(scene, cams, views, every, steps=args.steps)
    value = rate / 1e6
    sample = f"{n} rays per step (all pixels of view 0 of 200), {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3),
        "higher_is_better": True, "scaling": "weak" if args.partition == "replicate" else "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(scene, "f32"),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(scene, dtype, views=N_VIEWS):
    return {"workload": "main plain render: depth-9 octree (512^3) over [-1.5,1.5]^3, union of 8 seeded "
                        f"spheres/boxes, SH degree 3, {views} orbit views of 800x800, gamma 1e-4",
            "leaves": int(scene.n), "views": views, "width": W, "height": H, "rays_per_step": views * W * H,
            "sh_degree": 3, "leaf_dtype": dtype, "gamma": GAMMA,
            "l2": "no flush: inputs and outputs larger than L2 (tree >= 0.4 GB read, 1.54 GB of rgb written per step)"}


def algorithmic_bytes(pot, torch, tree, cams, dtype, leaf_bytes):
    """Per-launch algorithmic bytes: sum over views of (distinct leaves composited in the view) x leaf
    record bytes (the HBM floor), plus the rgb output; also the touched bytes (every composited leaf
    segment) for the L2 view.  Counted with the library's counting launch, outside the timed region."""
    n_leaves = tree.info()["n_leaves"]
    touched = torch.zeros(n_leaves, dtype=torch.uint8, device="cuda")
    seg = torch.zeros((1, H, W), dtype=torch.int32, device="cuda")
    rgb = torch.empty((1, H, W, 3), dtype=torch.float32, device="cuda")
    uniq, segs, hits = 0, 0, 0
    for v in range(len(cams)):
        touched.zero_()
        pot.render(tree, cams[v:v + 1], rgb=rgb, gamma=GAMMA, seg_count=seg, leaf_touched=touched)
        uniq += int(touched.sum().item())
        segs += int(seg.sum().item())
        hits += int((seg > 0).sum().item())
    rays = len(cams) * W * H
    out_bytes = 12 * rays
    return {"unique_leaves": uniq, "leaf_segments": segs, "hbm_bytes": uniq * leaf_bytes + out_bytes,
            "touched_bytes": segs * leaf_bytes + out_bytes, "rays": rays, "hit_rays": hits}


KERNEL_TYPE = {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16", "cb16": "cb16"}
ISSUE_SLOTS_PER_SM_CYCLE = 4      # one warp instruction per cycle from each of an SM's 4 schedulers


def measured_units(variant, sha, launch_ms, n_views, sm_mhz, l2_peak, hbm_peak):
    """Each hardware unit's share of its peak for the render launch just timed,
    from the committed ncu counters of this kernel version (scaled from the
    captured 16 views to ``n_views``) over the CUDA-event launch time: DRAM
    bytes (against the HBM copy peak), L2 bytes (against the library's own L2
    read probe), warp instructions issued (against 4 per SM per cycle at the
    clock sampled during the run), and the L1 data pipe's wavefronts (ncu's own
    fraction of peak).  None when this kernel version has not been captured."""
    prof = NCU_PROFILE.get(variant)
    if not prof or prof.get("sha") != sha:
        return None
    scale = n_views / NCU_VIEWS
    t = launch_ms * 1e-3
    sms = 152
    out = {"source": f"ncu counters of a {NCU_VIEWS}-view launch of this kernel version, x {scale:g}"}
    dram = (prof["dram_read"] + prof["dram_write"]) * scale
    out["dram"] = {"bytes_per_launch": round(dram), "achieved_gbs": round(dram / t / 1e9, 1), "peak_gbs": hbm_peak,
                   "frac": round(dram / t / 1e9 / hbm_peak, 4)}
    if l2_peak:
        l2 = prof["lts_bytes"] * scale
        out["l2"] = {"bytes_per_launch": round(l2), "achieved_gbs": round(l2 / t / 1e9, 1),
                     "peak_gbs": round(l2_peak, 1), "peak_source": "pot_probe_l2_read, 32 MiB, measured here",
                     "frac": round(l2 / t / 1e9 / l2_peak, 4)}
    inst = prof["warp_inst"] * scale
    if sm_mhz:
        peak_i = sms * ISSUE_SLOTS_PER_SM_CYCLE * sm_mhz * 1e6
        out["issue"] = {"warp_inst_per_launch": round(inst), "achieved_ginst_s": round(inst / t / 1e9, 1),
                        "peak_ginst_s": round(peak_i / 1e9, 1), "frac": round(inst / t / peak_i, 4)}
    out["l1_data_pipe"] = {"wavefronts_per_launch": round(prof["l1_wavefronts"] * scale),
                           "frac": round(prof["l1_pct"] / 100.0, 4), "frac_source": "ncu pct_of_peak (capture)"}
    fr = {k: v["frac"] for k, v in out.items() if isinstance(v, dict) and "frac" in v}
    out["binding"] = max(fr, key=fr.get)
    return out


def train_measure(pot, torch, synth, scene, target_tree, args, barrier):
    """Direct octree optimisation (Sec. 3.3): fit a perturbed copy of the main tree
    (SH + N(0, 0.3), sigma x U(0.5, 1.5)) to renders of the main tree from 100
    training views of 800x800 on the upper hemisphere; batches of random rays,
    MSE, backward, optimiser step.  Reports the backward kernel alone and the
    whole step in Mrays/s."""
    cams = synth.cameras_train(n=args.train_views)
    all_o, all_d = pot.camera_rays(cams)
    target = pot.render_rays(target_tree, all_o, all_d, gamma=GAMMA, near=2.0, far=6.0)
    tree = pot.Tree.from_scene(synth.perturbed(scene, 1003))
    # held-out views (other hemisphere cameras) for the fit's PSNR against the target tree
    held = synth.cameras_train(seed=1005, n=args.train_eval_views)
    held_target = pot.render(target_tree, held, gamma=GAMMA)

    def held_psnr():
        mse = float(((pot.render(tree, held, gamma=GAMMA) - held_target) ** 2).mean().item())
        return round(10.0 * math.log10(1.0 / mse), 3) if mse > 0 else float("inf")

    psnr0 = held_psnr()
    n_tiles_total = len(cams) * (W // 4) * (H // 8)
    lane = torch.arange(32, device="cuda")
    info = tree.info()
    L, K = info["n_leaves"], info["sh_dim"]
    opt = pot.LeafOptimizer(tree, args.train_opt, lr_sigma=args.train_lr_sigma, lr_sh=args.train_lr_sh)
    gs = torch.zeros(L, dtype=torch.float32, device="cuda")
    gh = torch.zeros((L, K, 3), dtype=torch.float32, device="cuda")
    B = args.train_batch
    loss_buf = torch.zeros(1, dtype=torch.float32, device="cuda")
    records = pot.SegmentRecords.for_rays(B) if args.train_record and not args.train_fused else None
    gen = torch.Generator(device="cuda").manual_seed(1003)
    parts = ("batch", "forward", "mse", "zero", "backward", "optimizer")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)]
    losses, t_parts = [], {k: [] for k in parts}
    n_total = args.train_steps + 3
    for it in range(n_total):
        ev[0].record()
        if args.train_batch_mode == "tiles":
            # B / 32 random 4 x 8 pixel tiles of the training views, one tile per warp
            tl = torch.randint(0, n_tiles_total, (B // 32,), device="cuda", generator=gen)
            view, rem = tl // ((W // 4) * (H // 8)), tl % ((W // 4) * (H // 8))
            px = (rem % (W // 4))[:, None] * 4 + lane % 4
            py = (rem // (W // 4))[:, None] * 8 + lane // 4
            idx = ((view[:, None] * H + py) * W + px).reshape(-1)
        else:
            idx = torch.randint(0, all_o.shape[0], (B,), device="cuda", generator=gen)
            if args.train_sort:   # same random rays, in view / row / column order: coherent warps
                idx = torch.sort(idx).values
        o, d, y = all_o[idx], all_d[idx], target[idx]
        ev[1].record()
        if args.train_fused:   # render + MSE + backward in one launch
            ev[2].record()
            ev[3].record()
            gs.zero_()
            gh.zero_()
            ev[4].record()
            loss, _, _ = pot.render_mse_backward(tree, o, d, y, grad_sigma=gs, grad_sh=gh, loss=loss_buf,
                                                 gamma=GAMMA, near=2.0, far=6.0)
        else:
            if records is not None:
                rgb = pot.render_rays_record(tree, o, d, records, gamma=GAMMA, near=2.0, far=6.0)
            else:
                rgb = pot.render_rays(tree, o, d, gamma=GAMMA, near=2.0, far=6.0)
            ev[2].record()
            loss, g = pot.loss_mse(rgb, y)
            ev[3].record()
            gs.zero_()
            gh.zero_()
            ev[4].record()
            if records is not None:
                pot.render_backward_recorded(tree, o, d, g, rgb, records, grad_sigma=gs, grad_sh=gh, gamma=GAMMA,
                                             near=2.0, far=6.0)
            else:
                pot.render_backward(tree, o, d, g, rgb_fwd=rgb, grad_sigma=gs, grad_sh=gh, gamma=GAMMA, near=2.0,
                                    far=6.0)
        ev[5].record()
        opt.step(gs, gh)
        ev[6].record()
        torch.cuda.synchronize()
        losses.append(float(loss.item()))
        if it >= 3:
            for k, name in enumerate(parts):
                t_parts[name].append(ev[k].elapsed_time(ev[k + 1]))
    t_bwd = t_parts["backward"]
    t_step = [sum(v) for v in zip(*t_parts.values())]
    ab = None if args.train_fused else record_ab(pot, torch, tree, o, d, y, B, L, K)
    # the last batch's leaf counts (a counting forward, outside the timed loop) for the
    # backward's roofline: every distinct leaf's record read once and its gradient row
    # (1 + 3K floats) read and written once from DRAM; the rays' origins, directions,
    # upstream gradients and forward colours read once
    seg = torch.zeros(B, dtype=torch.int32, device="cuda")
    touched = torch.zeros(L, dtype=torch.uint8, device="cuda")
    pot.render_rays(tree, o, d, gamma=GAMMA, near=2.0, far=6.0, seg_count=seg, leaf_touched=touched)
    uniq, segs = int(touched.sum().item()), int(seg.sum().item())
    leaf_b, grad_b = int(info["leaf_bytes"]), 4 * (1 + 3 * K)
    bwd_bytes = uniq * (leaf_b + 2 * grad_b) + B * 4 * (3 + 3 + 3 + 3)
    bwd_l2 = segs * (leaf_b + grad_b) + B * 4 * 12
    psnr1 = held_psnr()
    pot.check()
    tree.free()
    mb, ms = sum(t_bwd) / len(t_bwd), sum(t_step) / len(t_step)
    hbm_peak, hbm_kind = measured_peaks()
    return {"workload": f"fit a perturbed main tree to {args.train_views} training views of 800x800 (hemisphere), MSE",
            "rays_per_batch": B, "optimizer": args.train_opt, "lr_sigma": args.train_lr_sigma,
            "lr_sh": args.train_lr_sh, "steps": args.train_steps,
            "bwd_mrays_s": round(B / (mb * 1e-3) / 1e6, 2), "bwd_ms": round(mb, 4),
            "bwd_roofline": {"bound": "hbm", "algorithmic_bytes": bwd_bytes,
                             "achieved": round(bwd_bytes / (mb * 1e-3) / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
                             "frac": round(bwd_bytes / (mb * 1e-3) / 1e9 / hbm_peak, 4),
                             "peak_source": f"hbm_gbs of {hbm_kind}",
                             "unique_leaves": uniq, "leaf_segments": segs,
                             "touched_bytes": bwd_l2,
                             "touched_gbs": round(bwd_l2 / (mb * 1e-3) / 1e9, 1),
                             "bytes": "distinct leaves x (record + 2 x gradient row) + rays x 48 B; touched = "
                                      "segments x (record + gradient row) + rays x 48 B"},
            "bwd_launch": ("pot_render_mse_backward: colour walk + MSE + gradient walk" if args.train_fused
                           else "pot_render_backward_recorded: the forward's recorded segments sorted by leaf, "
                                "one thread per record, runs of a leaf merged in the warp" if records is not None
                           else "pot_render_backward with the forward colour given"),
            "record_ab": ab,
            "step_mrays_s": round(B / (ms * 1e-3) / 1e6, 2), "step_ms": round(ms, 4),
            "batch": (f"{B // 32} random 4x8-pixel tiles of the training views, one per warp"
                      if args.train_batch_mode == "tiles" else
                      f"{B} random pixels of the training views" + (", sorted by view and pixel"
                                                                    if args.train_sort else "")),
            "step_parts": ("random batch" + (" sorted by pixel" if args.train_sort else "") +
                           " + gather (torch), " +
                           ("zero grads (torch), fused forward + MSE + backward (one launch), "
                            if args.train_fused else
                            "forward recording its segments, MSE, zero grads (torch), backward over the records, "
                            if records is not None else "forward, MSE, zero grads (torch), backward, ") +
                           "optimiser step"),
            "parts_ms": {k: round(sum(v) / len(v), 4) for k, v in t_parts.items()},
            "loss_first": round(losses[0], 6), "loss_last": round(losses[-1], 6),
            "heldout_psnr_db": {"before": psnr0, "after": psnr1,
                                "views": f"{args.train_eval_views} held-out hemisphere views of 800x800 against "
                                         "the target tree's renders"}}


def record_ab(pot, torch, tree, o, d, y, B, L, K, reps=10):
    """The two training pairs on one batch (CUDA events, mean of ``reps`` after a
    warm-up call): pot_render_rays + pot_render_backward (the backward walks
    every ray again) against pot_render_rays_record + pot_render_backward_recorded
    (one thread per recorded segment); and their gradients on that batch, which
    must agree to float-atomic summation order."""
    records = pot.SegmentRecords.for_rays(B)
    gs = torch.zeros(L, dtype=torch.float32, device="cuda")
    gh = torch.zeros((L, K, 3), dtype=torch.float32, device="cuda")

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    kw = dict(gamma=GAMMA, near=2.0, far=6.0)
    rgb = pot.render_rays(tree, o, d, **kw)
    _, g = pot.loss_mse(rgb, y)
    out = {"forward_ms": round(timed(lambda: pot.render_rays(tree, o, d, rgb=rgb, **kw)), 4),
           "forward_record_ms": round(timed(lambda: pot.render_rays_record(tree, o, d, records, rgb=rgb, **kw)), 4)}
    out["backward_walk_ms"] = round(timed(lambda: pot.render_backward(tree, o, d, g, rgb_fwd=rgb, grad_sigma=gs,
                                                                      grad_sh=gh, **kw)), 4)
    out["backward_recorded_ms"] = round(timed(lambda: pot.render_backward_recorded(tree, o, d, g, rgb, records,
                                                                                   grad_sigma=gs, grad_sh=gh, **kw)), 4)
    out["records_used"] = records.used()
    out["records_capacity"] = records.capacity
    out["records_overflow"] = records.overflowed()
    gs.zero_()
    gh.zero_()
    pot.render_backward_recorded(tree, o, d, g, rgb, records, grad_sigma=gs, grad_sh=gh, **kw)
    ws, wh = pot.render_backward(tree, o, d, g, rgb_fwd=rgb, **kw)
    out["recorded_vs_walk"] = {
        "grad_sigma_max_rel": float((gs - ws).abs().max() / ws.abs().max().clamp_min(1e-30)),
        "grad_sh_max_rel": float((gh - wh).abs().max() / wh.abs().max().clamp_min(1e-30)),
        "bar": "max |recorded - walking| / max |walking| (float atomics: summation order only)"}
    del records
    return out


def serve_measure(pot, torch, synth, args):
    """Continuous-batching server: 4 resident fp16 trees (depth 7/8/9/10, SH degree
    1/2/3/3), Poisson arrivals, resolutions from {256^2, 512^2, 800^2, 1920x1080};
    p50/p99 latency (arrival -> completion event) and rays/s, batched (requests of
    up to 800x800 on a high-priority stream) vs one request at a time; plus a burst
    (all requests at t = 0) for throughput."""
    import numpy as np
    from paper_2103_14024_gb300.serve import RenderServer, Request, summarize
    trees = []
    for i, (D, deg) in enumerate(synth.SERVE_TREES):
        sc = synth.scene_shapes_torch(1004 + i, depth=D, sh_degree=deg, device="cuda")
        trees.append(pot.Tree.build_sparse(D, deg, sc.bbox_lo, sc.bbox_size, sc.morton, sc.sigma, sc.sh,
                                           dtype="f16"))
        del sc
    torch.cuda.empty_cache()
    resident = sum(t.info()["bytes"] for t in trees)
    budget = resident + (1 << 30)      # 1 GiB of in-flight outputs on top of the resident trees
    arrival, tree_idx, cams = synth.serve_requests(1004, args.serve_requests, rate_hz=args.serve_rate)
    out = {"trees": [{"depth": D, "sh_degree": deg, "leaves": int(t.info()["n_leaves"]),
                      "bytes": int(t.info()["bytes"])} for (D, deg), t in zip(synth.SERVE_TREES, trees)],
           "rate_hz": args.serve_rate, "hbm_budget_bytes": int(budget)}
    # warm the kernels (one launch per tree group) outside the measurement
    warm = [Request(i, 0.0, int(tree_idx[i]), cams[i]) for i in range(min(8, len(cams)))]
    RenderServer(trees, budget).run(warm, mode="batch")
    torch.cuda.synchronize()
    for label, arr in (("poisson", arrival), ("burst", np.zeros_like(arrival))):
        for mode in ("batch", "alone"):
            reqs = [Request(i, float(arr[i]), int(tree_idx[i]), cams[i]) for i in range(len(cams))]
            srv = RenderServer(trees, budget, streams=3, gamma=GAMMA, priority_pixels=args.serve_priority_pixels)
            torch.cuda.synchronize()
            base = torch.cuda.memory_allocated()
            torch.cuda.reset_peak_memory_stats()
            srv.run(reqs, mode=mode, on_done=lambda r: None)   # each image consumed (dropped) when done
            torch.cuda.synchronize()
            out[f"{label}_{mode}"] = summarize(reqs)
            out[f"{label}_{mode}"]["peak_output_bytes"] = int(torch.cuda.max_memory_allocated() - base)
    pot.check()
    for t in trees:
        t.free()
    return out


def pinned_d2h_gbs(torch, host):
    """Copy rate (GB/s) from device memory into the pinned host buffer ``host``
    (one warm-up copy, then one timed with CUDA events); None if it cannot be
    measured."""
    try:
        dev = torch.empty(host.shape, dtype=host.dtype, device="cuda")
        host.copy_(dev, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        host.copy_(dev, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        nbytes = host.numel() * host.element_size()
        del dev
        return round(nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1)
    except Exception:  # noqa: BLE001
        return None


def time_steps(torch, fn, steps, warmup, barrier):
    """W untimed steps, then K steps bracketed by barrier + synchronize; returns (host wall
    seconds, per-step CUDA-event ms, CUDA-event seconds from the first step's start to the
    last step's end)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = time.perf_counter()
    for s, e in evs:
        s.record()
        fn()
        e.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    per = [s.elapsed_time(e) for s, e in evs]
    return wall, per, evs[0][0].elapsed_time(evs[-1][1]) * 1e-3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "bf16", "cb16"])
    ap.add_argument("--variants", default="f16,bf16,cb16,f32-descent,f32-brick,f16-brick",
                    help="extra leaf dtypes to time ('' for none); '<dtype>-descent' = that tree without its "
                         "cell index (cells located by descending the child array); '<dtype>-brick' = with the "
                         "brick layout of the cell index instead of the dense one; '<dtype>-batch' = the views "
                         "rendered as a pot_render_batch work list of one item per view")
    ap.add_argument("--cells", default="default", choices=["default", "descent", "brick"],
                    help="cell index of the main measurement's tree: its default layout, none (descend the "
                         "child array) or the brick layout")
    ap.add_argument("--partition", default="views", choices=["views", "replicate"],
                    help="N > 1: split the views across the ranks (each ray once, strong scaling) or let "
                         "every rank render all of them (weak scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--train-steps", type=int, default=200)
    ap.add_argument("--train-batch", type=int, default=1 << 18)
    ap.add_argument("--train-sort", type=int, default=1,
                    help="1: order each random ray batch by view and pixel before rendering (the sum of the "
                         "gradients does not depend on the order)")
    ap.add_argument("--train-record", type=int, default=1,
                    help="1: the forward records its segments and the backward differentiates the records "
                         "(pot_render_rays_record / pot_render_backward_recorded); 0: the backward walks the rays")
    ap.add_argument("--train-fused", type=int, default=0,
                    help="1: pot_render_mse_backward (render, loss and gradients in one launch); "
                         "0: pot_render_rays + pot_loss_mse + pot_render_backward")
    ap.add_argument("--train-views", type=int, default=100,
                    help="training views the ray batches are drawn from (100 in the benchmark; fewer for "
                         "profiler captures)")
    ap.add_argument("--train-eval-views", type=int, default=8, help="held-out views for the fit's PSNR")
    ap.add_argument("--train-batch-mode", default="rays", choices=["rays", "tiles"],
                    help="rays: random pixels; tiles: random 4x8-pixel tiles (32 neighbouring rays per warp)")
    ap.add_argument("--train-opt", default="rmsprop", choices=["sgd", "rmsprop", "adam"])
    ap.add_argument("--train-lr-sigma", type=float, default=1.0)
    ap.add_argument("--train-lr-sh", type=float, default=1e-2)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--serve-rate", type=float, default=300.0)
    ap.add_argument("--serve-priority-pixels", type=int, default=800 * 800,
                    help="requests of at most this many pixels go to a high-priority stream (0: none)")
    ap.add_argument("--views", type=int, default=N_VIEWS,
                    help="cameras per step (a smaller case for profiler captures; the benchmark uses 200)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import paper_2103_14024_gb300 as pot
    from paper_2103_14024_gb300 import synth

    rank, local, world = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()

    def barrier():
        if dist is not None:
            dist.barrier()

    scene = synth.scene_shapes()
    all_cams = synth.cameras_main(N_VIEWS, W, H)[:args.views]
    # N > 1: each rank renders a contiguous slice of the views (strong scaling,
    # every ray once) or, with --partition replicate, all of them (weak scaling);
    # no exchange on the data path either way
    if args.partition == "views" and world > 1:
        v0, v1 = view_slice(rank, world, len(all_cams))
    else:
        v0, v1 = 0, len(all_cams)
    cams = all_cams[v0:v1]
    ccams = pot.make_cameras(cams)
    rays = len(cams) * W * H
    job_rays = job_rays_per_step(args.partition, world, len(all_cams), W * H)
    scaling = "weak" if args.partition == "replicate" else "strong"

    def measure(variant, e2e=False):
        dtype, _, mode = variant.partition("-")
        if dtype == "cb16":     # median-cut SH codebooks (2^16 entries per basis) of the f32 tree
            t32 = pot.Tree.from_scene(scene, dtype="f32")
            tree = t32.quantize(16)
            t32.free()
        else:
            tree = pot.Tree.from_scene(scene, dtype=dtype)
        if mode == "descent":
            tree.set_cell_index(False)
        elif mode == "brick":
            tree.set_cell_index("brick")
        info = tree.info()
        rgb = torch.empty((len(cams), H, W, 3), dtype=torch.float32, device="cuda")
        if mode == "batch":     # the same views as a work list of one item per view (pot_render_batch)
            items = [(tree, cams[i], rgb[i], (0.0, 0.0, 0.0), GAMMA, None) for i in range(len(cams))]

            def step():
                pot.render_batch(items)
        else:
            def step():
                pot.render(tree, ccams, rgb=rgb, gamma=GAMMA)

        l0 = pot.launch_count()
        with ClockSampler(dev_index) as clk:
            _, per, wall = time_steps(torch, step, args.steps, args.warmup, barrier)   # device (event) time
        launches = (pot.launch_count() - l0)
        launches_timed = launches * args.steps // (args.steps + args.warmup)
        pot.check()
        res = {"tree": tree, "info": info, "wall": wall, "per": per, "clk": clk.summary(),
               "launches": launches_timed}
        if e2e:
            host = torch.empty((len(cams), H, W, 3), dtype=torch.float32, pin_memory=True)

            def step_e2e():
                pot.render(tree, ccams, rgb=host, gamma=GAMMA)   # host output: D2H + sync inside

            ke = max(5, args.steps // 2)
            wall_e, _, _ = time_steps(torch, step_e2e, ke, 2, barrier)   # host wall clock: end to end
            res["e2e_wall"] = wall_e / ke
            res["d2h_gbs"] = pinned_d2h_gbs(torch, host)
            del host
        return res

    main_key = args.dtype if args.cells == "default" else f"{args.dtype}-{args.cells}"
    main_res = measure(main_key, e2e=not args.no_e2e)
    leaf_bytes = int(main_res["info"]["leaf_bytes"])
    alg = algorithmic_bytes(pot, torch, main_res["tree"], cams, args.dtype, leaf_bytes)

    # whole-job time: max over ranks of the timed region; value = the rays all
    # ranks rendered per step / that time
    wall = max_over_ranks(torch, dist, main_res["wall"], "cuda")
    ms_per_step = 1e3 * wall / args.steps
    value = job_rays / (wall / args.steps) / 1e6
    avg_launch_ms = sum(main_res["per"]) / len(main_res["per"])
    peak, peak_kind = measured_peaks()
    achieved = alg["hbm_bytes"] / (avg_launch_ms * 1e-3) / 1e9
    sha = kernel_sha()
    l2_peak = None
    if rank == 0:
        try:
            l2_peak = pot.probe_l2_read(32 << 20, 200)
        except Exception:  # noqa: BLE001
            l2_peak = None
    units = measured_units(main_key, sha, avg_launch_ms, len(cams), main_res["clk"].get("sm_mhz"), l2_peak, peak)
    traffic = units["dram"]["bytes_per_launch"] if units else None

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "ms_per_step_median": round(sorted(main_res["per"])[len(main_res["per"]) // 2], 3),
        "scaling": scaling, "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": dict(workload_config(scene, args.dtype, len(all_cams)),
                       cell_index_bytes=int(main_res["info"]["index_bytes"]),
                       cell_index={0: "none", 2: "dense", 3: "brick"}[int(main_res["info"]["index_kind"])],
                       partition=(f"views split across {world} ranks (rank 0: views {v0}..{v1 - 1})"
                                  if args.partition == "views" and world > 1 else
                                  f"every rank renders all {len(all_cams)} views" if world > 1 else "one GPU")),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"hbm_gbs of {peak_kind}",
                     "algorithmic_bytes_per_launch": alg["hbm_bytes"],
                     "kernel": f"render_kernel<16,{KERNEL_TYPE[args.dtype]},cams>",
                     "avg_launch_ms": round(avg_launch_ms, 3)},
        "gpu_launches": int(main_res["launches"]),
        "clocks": main_res["clk"],
    }
    if units:
        line["roofline"]["measured_units"] = units
    if l2_peak:
        line["roofline"]["l2_probe_gbs"] = round(l2_peak, 1)
    line["roofline"]["touched_bytes_per_launch"] = alg["touched_bytes"]
    if rank == 0:
        line["counts"] = {"unique_leaves_summed_over_views": alg["unique_leaves"],
                          "leaf_segments": alg["leaf_segments"],
                          "mean_leaf_segments_per_ray": round(alg["leaf_segments"] / rays, 3),
                          "hit_fraction": round(alg["hit_rays"] / rays, 4),
                          "mean_leaf_segments_per_hit_ray": round(alg["leaf_segments"] / max(1, alg["hit_rays"]), 3)}
    if not args.no_e2e:
        e2e_wall = max_over_ranks(torch, dist, main_res["e2e_wall"], "cuda")
        e2e_value = job_rays / e2e_wall / 1e6
        n_job_views = job_rays // (W * H)
        line["e2e"] = {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 80 * n_job_views,
                       "d2h_bytes_per_step": 12 * job_rays,
                       "pinned_d2h_gbs": main_res.get("d2h_gbs"),
                       "d2h_note": "device-to-pinned-host copy rate of this box for an image-sized buffer "
                                   "(one copy, CUDA events); the end-to-end number follows it"}
    variants = {}
    # per-GPU characteristics (other leaf types, training, serving) are measured at N = 1 only
    extras = world == 1
    for vd in [v for v in args.variants.split(",") if v and v != main_key and extras]:
        r = measure(vd)
        w = r["wall"]
        vb = algorithmic_bytes(pot, torch, r["tree"], cams, vd.partition("-")[0], int(r["info"]["leaf_bytes"]))
        avg = sum(r["per"]) / len(r["per"])
        vunits = measured_units(vd, sha, avg, len(cams), r["clk"].get("sm_mhz"), l2_peak, peak)
        variants[vd] = {"value": round(rays / (w / args.steps) / 1e6, 3),
                        "ms_per_step": round(1e3 * w / args.steps, 3),
                        "roofline": {"bound": "hbm", "achieved": round(vb["hbm_bytes"] / (avg * 1e-3) / 1e9, 1),
                                     "peak": peak, "unit": "GB/s",
                                     "frac": round(vb["hbm_bytes"] / (avg * 1e-3) / 1e9 / peak, 4),
                                     "traffic": (vunits["dram"]["bytes_per_launch"] if vunits else None),
                                     "measured_units": vunits},
                        "clocks": r["clk"], "leaf_bytes": int(r["info"]["leaf_bytes"]),
                        "cell_index_bytes": int(r["info"]["index_bytes"]),
                        "cell_index": {0: "none", 2: "dense", 3: "brick"}[int(r["info"]["index_kind"])]}
        r["tree"].free()
    if variants:
        line["variants"] = variants
    if not args.no_train and extras:
        line["train"] = train_measure(pot, torch, synth, scene, main_res["tree"], args, barrier)
    if not args.no_serve and extras:
        line["serve"] = serve_measure(pot, torch, synth, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        views = list(range(0, N_VIEWS, 2))     # 100 of the 200 views, all pixels: ~10-20 s of CPU work
        rate, n, dt, thr = run_oracle_timing(scene, synth.cameras_main(N_VIEWS, W, H), views, 1)
        line["cpu_baseline"] = {"value": round(rate / 1e6, 4), "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": f"all pixels of views 0,2,...,198 of 200 ({n} rays, {dt:.1f} s on "
                                          f"{thr} threads)"}
        # the same oracle on one thread, all pixels of view 0
        from oracle import oracle
        oracle.set_num_threads(1)
        try:
            rate1, n1, dt1, _ = run_oracle_timing(scene, synth.cameras_main(N_VIEWS, W, H), [0], 1)
        finally:
            oracle.set_num_threads(thr)
        line["cpu_baseline"]["value_1_thread"] = round(rate1 / 1e6, 4)
        line["cpu_baseline"]["sample_1_thread"] = f"all pixels of view 0 ({n1} rays, {dt1:.1f} s)"
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
