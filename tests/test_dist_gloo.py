"""The multi-rank path of bench.py on CPU (world size 2, gloo): the views are
split into contiguous slices, one per rank, and each rank renders its own
slice with no exchange on the data path; the only collective is the max over
ranks of the timed region, from which the whole-job value is computed.  The
reference arm runs on rank 0 only.  The renderer of a rank is stood in for by
the CPU oracle here (the GPU path is tested on one GPU)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wall = 1.0 + 0.5 * rank                      # rank 1 is the slowest
    m = bench.max_over_ranks(torch, dist, wall, "cpu")
    v = bench.job_value(world, 1000, m, 10)
    out.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]
    # 2 ranks x 1000 rays per step / (1.5 s / 10 steps) = 13333 rays/s
    assert all(abs(r[2] - 2 * 1000 / 0.15 / 1e6) < 1e-12 for r in res)


def test_reference_arm_only_on_rank_zero():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_view_slices_partition_the_views():
    sys.path.insert(0, ROOT)
    import bench
    for n in (1, 2, 7, 25, 200):
        for world in range(1, 9):
            sl = [bench.view_slice(r, world, n) for r in range(world)]
            assert sl[0][0] == 0 and sl[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))        # contiguous, disjoint
            sizes = [e - s for s, e in sl]
            assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n    # balanced, complete
    # every ray once when partitioned, once per rank when replicated
    assert bench.job_rays_per_step("views", 8, 200, 640000) == 200 * 640000
    assert bench.job_rays_per_step("replicate", 8, 200, 640000) == 8 * 200 * 640000
    assert bench.job_rays_per_step("views", 1, 200, 640000) == bench.job_rays_per_step("replicate", 1, 200, 640000)


def _slice_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle
    from paper_2103_14024_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_num_threads(1)
    scene = synth.scene_random(91, 5, 1, p_occ=0.3, sigma_mu=2.0)
    cams = synth.make_cameras(synth.orbit_c2ws(5, radius=3.0), 24, 16, 20.0)
    v0, v1 = bench.view_slice(rank, world, len(cams))
    mine = oracle.render_cams(oracle.build_sparse(scene), cams[v0:v1], gamma=1e-4)["rgb"]
    parts = [None] * world
    dist.all_gather_object(parts, (v0, v1, np.asarray(mine)))
    if rank == 0:
        parts.sort(key=lambda p: p[0])
        out.put(np.concatenate([p[2] for p in parts], axis=0))
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_render_equals_one_rank():
    """Two ranks each render their slice of 5 views; the views put back together
    equal the render of all 5 views by one rank, bit for bit."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import oracle
    from paper_2103_14024_gb300 import synth
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_slice_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    joined = q.get(timeout=300)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    scene = synth.scene_random(91, 5, 1, p_occ=0.3, sigma_mu=2.0)
    cams = synth.make_cameras(synth.orbit_c2ws(5, radius=3.0), 24, 16, 20.0)
    whole = oracle.render_cams(oracle.build_sparse(scene), cams, gamma=1e-4)["rgb"]
    assert joined.shape == whole.shape == (5, 16, 24, 3)
    assert np.array_equal(joined, whole)
    assert float(np.abs(whole).max()) > 0.0     # the views see the scene


def _grad_worker(rank, world, port, out):
    """One rank of data-parallel optimisation: the oracle's gradients of the
    MSE (mean over this rank's rays) of its share of the batch, then the
    library's all-reduce."""
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_2103_14024_gb300 as pot
    from oracle import oracle as O
    from paper_2103_14024_gb300 import synth as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = S.scene_random(58, 4, 2, p_occ=0.35)
    ot = O.build_sparse(sc)
    o, d = S.random_rays(58, 600, radius=3.0, spread=0.9)
    target = np.random.default_rng(58).uniform(size=(600, 3))
    lo, hi = rank * 600 // world, (rank + 1) * 600 // world
    col = O.render_rays(ot, o[lo:hi], d[lo:hi], near=0.2, far=8.0)["rgb"]
    g = 2.0 * (col - target[lo:hi]) / (3 * (hi - lo))           # MSE over this rank's rays
    gs, gh = O.backward_rays(ot, o[lo:hi], d[lo:hi], g, near=0.2, far=8.0)
    gs_t = torch.from_numpy(gs.astype(np.float32))
    gh_t = torch.from_numpy(gh.astype(np.float32))
    pot.allreduce_leaf_grads(gs_t, gh_t, "mean")
    out.put((rank, gs_t.numpy(), gh_t.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_data_parallel_gradients_equal_one_rank(oracle_mod):
    """Data-parallel optimisation (the ray batch split across 2 ranks, the tree
    replicated): after the all-reduce every rank holds the gradient of the
    whole batch's mean loss, the one-process gradient of all 600 rays."""
    import numpy as np
    import torch.multiprocessing as mp
    from paper_2103_14024_gb300 import synth as S
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda r: r[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = S.scene_random(58, 4, 2, p_occ=0.35)
    ot = oracle_mod.build_sparse(sc)
    o, d = S.random_rays(58, 600, radius=3.0, spread=0.9)
    target = np.random.default_rng(58).uniform(size=(600, 3))
    col = oracle_mod.render_rays(ot, o, d, near=0.2, far=8.0)["rgb"]
    rs, rh = oracle_mod.backward_rays(ot, o, d, 2.0 * (col - target) / (3 * 600), near=0.2, far=8.0)
    for _, gs, gh in res:
        assert np.abs(gs - rs).max() <= 1e-6 * np.abs(rs).max()
        assert np.abs(gh - rh).max() <= 1e-6 * np.abs(rh).max()
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])   # replicas stay equal


def test_allreduce_without_process_group_is_a_no_op():
    import torch
    sys.path.insert(0, ROOT)
    import paper_2103_14024_gb300 as pot
    a, b = torch.ones(3), torch.ones(2, 4)
    pot.allreduce_leaf_grads(a, b)
    assert a.tolist() == [1.0, 1.0, 1.0] and float(b.sum()) == 8.0
    with pytest.raises(ValueError):
        pot.allreduce_leaf_grads(a, b, op="max")
