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
