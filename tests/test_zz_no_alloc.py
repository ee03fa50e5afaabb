"""pot_render_noalloc: the camera render for callers that cannot allocate GPU
memory (an embedding application that owns all GPU memory on a fixed budget,
allocator hooks that refuse library allocations, a frame loop that cannot
afford an allocator call).  Its scratch is a fixed array inside libpot.so.

Checked through the C ABI against pot_render (the allocating entry point) on
two calls in a row, so the second call runs on the scratch the first one
left behind.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    import paper_2103_14024_gb300 as pot
    L = pot.lib()
    fn = L.pot_render_noalloc
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return pot, torch, fn


def _noalloc(env, tree, cams, gamma=0.0, bg=(0.0, 0.0, 0.0)):
    pot, torch, fn = env
    carr = pot.make_cameras(cams)
    n = len(carr)
    H, W = carr[0].height, carr[0].width
    rgb = torch.full((n, H, W, 3), -1.0, dtype=torch.float32, device="cuda")
    tf = torch.full((n, H, W), -1.0, dtype=torch.float32, device="cuda")
    opts = pot._opts(bg, gamma)
    st = fn(tree.handle, carr, n, C.byref(opts), C.c_void_p(rgb.data_ptr()), C.c_void_p(tf.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pot.POT_OK, pot.last_error()
    return rgb, tf


def test_noalloc_matches_pot_render_on_consecutive_calls(env):
    pot, torch, _ = env
    from paper_2103_14024_gb300 import synth as S
    scene = S.scene_random(77, 6, 3, p_occ=0.3, sigma_mu=2.0)
    tree = pot.Tree.from_scene(scene)
    calls = [
        (S.make_cameras(S.orbit_c2ws(5, radius=3.0), 37, 29, 40.0), 0.0, (0.0, 0.0, 0.0)),
        (S.make_cameras(S.orbit_c2ws(3, radius=3.5, elevation_deg=-20.0), 64, 48, 70.0), 1e-4,
         (0.2, 0.5, 0.1)),
    ]
    for cams, gamma, bg in calls:
        rgb, tf = _noalloc(env, tree, cams, gamma, bg)
        ref, ref_tf = pot.render(tree, cams, gamma=gamma, bg=bg, want_t_final=True)
        torch.cuda.synchronize()
        assert float((rgb - ref).abs().max()) <= TOL
        assert float((tf - ref_tf).abs().max()) <= TOL
        assert bool((rgb >= 0).all())
    pot.check()
    tree.free()


def test_noalloc_rejects_more_than_its_scratch_holds(env):
    pot, torch, fn = env
    from paper_2103_14024_gb300 import synth as S
    tree = pot.Tree.from_scene(S.scene_tiny())
    cams = S.make_cameras(S.orbit_c2ws(1025), 8, 8, 10.0)
    carr = pot.make_cameras(cams)
    rgb = torch.empty((1025, 8, 8, 3), dtype=torch.float32, device="cuda")
    st = fn(tree.handle, carr, 1025, None, C.c_void_p(rgb.data_ptr()), None,
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pot.POT_ERR_INVALID_ARG
    assert "1024" in pot.last_error()
    host = np.zeros((1, 64, 64, 3), np.float32)
    one = pot.make_cameras(S.cameras_tiny("generic"))
    st = fn(tree.handle, one, 1, None, C.c_void_p(host.ctypes.data), None,
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pot.POT_ERR_INVALID_ARG


def test_noalloc_refuses_host_count_arrays(env):
    """The counting outputs are written by the kernel, so host arrays are refused
    before any launch, as pot_render refuses them."""
    pot, torch, fn = env
    from paper_2103_14024_gb300 import synth as S
    tree = pot.Tree.from_scene(S.scene_tiny())
    one = pot.make_cameras(S.cameras_tiny("generic"))
    rgb = torch.empty((1, 64, 64, 3), dtype=torch.float32, device="cuda")
    seg_h = np.zeros((1, 64, 64), np.int32)
    touched_h = np.zeros(tree.info()["n_leaves"], np.uint8)
    seg_d = torch.zeros((1, 64, 64), dtype=torch.int32, device="cuda")
    touched_d = torch.zeros(tree.info()["n_leaves"], dtype=torch.uint8, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seg, touched in ((seg_h.ctypes.data, touched_d.data_ptr()), (seg_d.data_ptr(), touched_h.ctypes.data),
                         (seg_h.ctypes.data, touched_h.ctypes.data)):
        opts = pot._opts((0.0, 0.0, 0.0), 0.0)
        opts.seg_count = seg
        opts.leaf_touched = touched
        st = fn(tree.handle, one, 1, C.byref(opts), C.c_void_p(rgb.data_ptr()), None, stream)
        assert st == pot.POT_ERR_INVALID_ARG
        assert "device memory" in pot.last_error()
    torch.cuda.synchronize()
    assert not seg_h.any() and not touched_h.any()
    # device arrays are accepted and give pot_render's counts
    opts = pot._opts((0.0, 0.0, 0.0), 0.0)
    opts.seg_count = seg_d.data_ptr()
    opts.leaf_touched = touched_d.data_ptr()
    st = fn(tree.handle, one, 1, C.byref(opts), C.c_void_p(rgb.data_ptr()), None, stream)
    assert st == pot.POT_OK, pot.last_error()
    seg_r = torch.zeros_like(seg_d)
    touched_r = torch.zeros_like(touched_d)
    pot.render(tree, S.cameras_tiny("generic"), seg_count=seg_r, leaf_touched=touched_r)
    torch.cuda.synchronize()
    assert torch.equal(seg_d, seg_r) and torch.equal(touched_d, touched_r)
    pot.check()
    tree.free()


def test_noalloc_python_wrapper(env):
    pot, torch, _ = env
    from paper_2103_14024_gb300 import synth as S
    tree = pot.Tree.from_scene(S.scene_random(77, 5, 2, p_occ=0.3))
    cams = S.make_cameras(S.orbit_c2ws(3, radius=3.0), 40, 24, 35.0)
    ref, ref_tf = pot.render(tree, cams, gamma=1e-3, bg=(0.2, 0.1, 0.0), want_t_final=True)
    rgb = torch.full_like(ref, -1.0)
    tf = torch.full_like(ref_tf, -1.0)
    out = pot.render_noalloc(tree, cams, rgb, t_final=tf, gamma=1e-3, bg=(0.2, 0.1, 0.0))
    torch.cuda.synchronize()
    assert out is rgb and torch.equal(rgb, ref) and torch.equal(tf, ref_tf)
    pot.check()
    tree.free()
