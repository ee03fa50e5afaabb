"""GB300 PlenOctree renderer: Python binding of ``libpot.so``.

Argument marshalling only: every step of the render path runs in the CUDA
kernels of ``libpot.so`` (sources in ``csrc/``, C ABI in ``include/pot.h``).
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
library is missing, every call raises.

Method: PlenOctrees for Real-time Rendering of Neural Radiance Fields
(Yu et al., ICCV 2021), Sec. 3.2 (octree rendering and conversion), Eq. 1
(quadrature), App. B.1 (real SH basis), App. B.3 (derivatives).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpot.so")

POT_OK, POT_ERR_INVALID_ARG, POT_ERR_OOM, POT_ERR_CUDA, POT_ERR_TRAVERSAL, POT_ERR_BUDGET, \
    POT_ERR_UNSUPPORTED = range(7)
DTYPES = {"f32": 0, "f16": 1, "bf16": 2, "cb16": 3}
_STATUS = {0: "POT_OK", 1: "POT_ERR_INVALID_ARG", 2: "POT_ERR_OOM", 3: "POT_ERR_CUDA",
           4: "POT_ERR_TRAVERSAL", 5: "POT_ERR_BUDGET", 6: "POT_ERR_UNSUPPORTED"}


class PotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class BuildDesc(C.Structure):
    _fields_ = [("depth", C.c_int32), ("sh_degree", C.c_int32), ("leaf_dtype", C.c_int32),
                ("sigma_threshold", C.c_float), ("bbox_lo", C.c_float * 3), ("bbox_size", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("c2w", (C.c_float * 4) * 3), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("near", C.c_float),
                ("far", C.c_float)]


class RenderOpts(C.Structure):
    _fields_ = [("bg", C.c_float * 3), ("gamma", C.c_float), ("near", C.c_float), ("far", C.c_float),
                ("flags", C.c_uint32), ("max_steps", C.c_int32), ("seg_count", C.c_void_p),
                ("leaf_touched", C.c_void_p)]


class RenderItem(C.Structure):
    _fields_ = [("tree", C.c_void_p), ("cam", Camera), ("bg", C.c_float * 3), ("gamma", C.c_float),
                ("rgb", C.c_void_p), ("t_final", C.c_void_p)]


class StepDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lr_sigma", C.c_float), ("lr_sh", C.c_float), ("alpha", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("step", C.c_int32)]


OPTIMIZERS = {"sgd": 0, "rmsprop": 1, "adam": 2}


class TreeInfo(C.Structure):
    _fields_ = [("depth", C.c_int32), ("sh_degree", C.c_int32), ("sh_dim", C.c_int32),
                ("leaf_dtype", C.c_int32), ("n_nodes", C.c_int64), ("n_leaves", C.c_int64),
                ("bytes", C.c_int64), ("leaf_bytes", C.c_int64), ("bbox_lo", C.c_float * 3),
                ("bbox_size", C.c_float), ("saturated", C.c_int32), ("device", C.c_int32),
                ("index_bytes", C.c_int64), ("index_kind", C.c_int32)]


CELLS = {"none": 0, "default": 1, "dense": 2, "brick": 3}


assert C.sizeof(Camera) == 80

_lib = None
_lock = threading.Lock()

_p = C.c_void_p
_SIGS = {
    "pot_build": [_p, _p, _p, _p, _p],
    "pot_build_sparse": [_p, C.c_int64, _p, _p, _p, _p, _p],
    "pot_tree_get_info": [_p, _p],
    "pot_tree_export": [_p, _p, _p, _p, _p, _p],
    "pot_tree_set_values": [_p, _p, _p, _p],
    "pot_tree_free": [_p],
    "pot_tree_set_cell_index": [_p, C.c_int32, _p],
    "pot_tree_export_cell_index": [_p, _p, _p],
    "pot_query": [_p, C.c_int64, _p, _p, _p],
    "pot_sh_basis": [C.c_int32, C.c_int64, _p, _p, _p],
    "pot_render": [_p, _p, C.c_int32, _p, _p, _p, _p],
    "pot_render_noalloc": [_p, _p, C.c_int32, _p, _p, _p, _p],
    "pot_render_rays": [_p, C.c_int64, _p, _p, _p, _p, _p, _p],
    "pot_check": [_p],
    "pot_render_backward": [_p, C.c_int64, _p, _p, _p, _p, _p, _p, _p, _p],
    "pot_render_mse_backward": [_p, C.c_int64, _p, _p, _p, _p, _p, _p, _p, _p, _p],
    "pot_render_rays_record": [_p, C.c_int64, _p, _p, _p, _p, _p, _p, C.c_int64, _p, _p],
    "pot_render_backward_recorded": [_p, C.c_int64, _p, _p, _p, _p, _p, _p, C.c_int64, _p, _p, _p, _p],
    "pot_step": [_p, _p, _p, _p, _p, _p],
    "pot_loss_mse": [C.c_int64, _p, _p, _p, _p, _p],
    "pot_camera_rays": [_p, C.c_int32, C.c_int64, _p, _p, _p, _p],
    "pot_render_batch": [_p, C.c_int32, _p],
    "pot_visibility": [_p, _p, C.c_int32, _p, _p, _p],
    "pot_tree_prune": [_p, _p, C.c_float, _p, _p],
    "pot_tree_quantize": [_p, C.c_int32, _p, _p],
    "pot_probe_l2_read": [C.c_int64, C.c_int32, _p, _p],
}


def lib():
    """The loaded ``libpot.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.pot_last_error.restype = C.c_char_p
            L.pot_last_error.argtypes = []
            L.pot_version.restype = C.c_int32
            L.pot_launch_count.restype = C.c_int64
            L.pot_step_state_floats.restype = C.c_int64
            L.pot_step_state_floats.argtypes = [_p, C.c_int32]
            _lib = L
    return _lib


def _check(st: int):
    if st != POT_OK:
        raise PotError(st, lib().pot_last_error().decode(errors="replace"))


def last_error() -> str:
    return lib().pot_last_error().decode(errors="replace")


def launch_count() -> int:
    return int(lib().pot_launch_count())


def probe_l2_read(nbytes: int = 32 << 20, reps: int = 200, stream=None) -> float:
    """``pot_probe_l2_read``: L2 read bandwidth (GB/s) over an L2-resident buffer."""
    out = C.c_double(0.0)
    _check(lib().pot_probe_l2_read(int(nbytes), int(reps), C.byref(out), _stream(stream)))
    return float(out.value)


# ----------------------------------------------------------------------------
# pointers: torch tensors (any device) or numpy arrays (host)
# ----------------------------------------------------------------------------

def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    # torch.Tensor
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(x.data_ptr())


def _stream(stream=None):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _as_np(x, dtype):
    return np.ascontiguousarray(x, dtype=dtype)


def make_cameras(cams_np) -> C.Array:
    """ctypes array of Camera from a numpy structured array with the synth.CAMERA_DTYPE layout."""
    cams_np = np.ascontiguousarray(cams_np)
    arr = (Camera * len(cams_np))()
    C.memmove(arr, cams_np.ctypes.data, 80 * len(cams_np))
    return arr


def _opts(bg=(0.0, 0.0, 0.0), gamma=0.0, near=0.0, far=3.0e38, seg_count=None, leaf_touched=None,
          max_steps=0):
    o = RenderOpts()
    o.max_steps = max_steps
    o.bg[0], o.bg[1], o.bg[2] = bg
    o.gamma = gamma
    o.near = near
    o.far = far
    o.flags = 0
    o.seg_count = None if seg_count is None else seg_count.data_ptr()
    o.leaf_touched = None if leaf_touched is None else leaf_touched.data_ptr()
    return o


# ----------------------------------------------------------------------------
# trees
# ----------------------------------------------------------------------------

class Tree:
    """A PlenOctree resident on the GPU (owned by libpot)."""

    def __init__(self, handle):
        self._h = handle

    def __del__(self):
        self.free()

    def free(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            lib().pot_tree_free(h)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("tree was freed")
        return self._h

    @staticmethod
    def _desc(depth, sh_degree, dtype, bbox_lo, bbox_size, threshold=0.0):
        d = BuildDesc()
        d.depth, d.sh_degree, d.leaf_dtype = depth, sh_degree, DTYPES[dtype]
        d.sigma_threshold = threshold
        for a in range(3):
            d.bbox_lo[a] = bbox_lo[a]
        d.bbox_size = bbox_size
        return d

    @classmethod
    def build_sparse(cls, depth, sh_degree, bbox_lo, bbox_size, morton, sigma, sh, dtype="f32",
                     stream=None) -> "Tree":
        """``pot_build_sparse``; arrays are numpy (host) or torch tensors (any device)."""
        d = cls._desc(depth, sh_degree, dtype, bbox_lo, bbox_size)
        if isinstance(morton, np.ndarray):
            morton = _as_np(morton, np.uint64)
            sigma = _as_np(sigma, np.float32)
            sh = _as_np(sh, np.float32)
        n = int(morton.shape[0])
        out = C.c_void_p()
        _check(lib().pot_build_sparse(C.byref(d), n, _ptr(morton), _ptr(sigma), _ptr(sh), C.byref(out),
                                      _stream(stream)))
        return cls(out.value)

    @classmethod
    def from_scene(cls, scene, dtype="f32", stream=None) -> "Tree":
        return cls.build_sparse(scene.depth, scene.sh_degree, scene.bbox_lo, scene.bbox_size,
                                scene.morton, scene.sigma, scene.sh, dtype=dtype, stream=stream)

    @classmethod
    def build_dense(cls, depth, sh_degree, bbox_lo, bbox_size, sigma, sh, threshold=0.0, dtype="f32",
                    stream=None) -> "Tree":
        """``pot_build`` from dense grids sigma [R,R,R], sh [R,R,R,K,3] indexed [x][y][z]."""
        d = cls._desc(depth, sh_degree, dtype, bbox_lo, bbox_size, threshold)
        if isinstance(sigma, np.ndarray):
            sigma = _as_np(sigma, np.float32)
            sh = _as_np(sh, np.float32)
        out = C.c_void_p()
        _check(lib().pot_build(C.byref(d), _ptr(sigma), _ptr(sh), C.byref(out), _stream(stream)))
        return cls(out.value)

    def info(self) -> dict:
        i = TreeInfo()
        _check(lib().pot_tree_get_info(self.handle, C.byref(i)))
        return {f: (list(getattr(i, f)) if f == "bbox_lo" else getattr(i, f)) for f, _ in TreeInfo._fields_}

    def export(self, stream=None):
        """Canonical arrays (numpy): child [N,8] int32, sigma [L] f32, sh [L,K,3] f32, morton [L] u64."""
        inf = self.info()
        N, L, K = inf["n_nodes"], inf["n_leaves"], inf["sh_dim"]
        child = np.zeros((N, 8), np.int32)
        sigma = np.zeros(L, np.float32)
        sh = np.zeros((L, K, 3), np.float32)
        morton = np.zeros(L, np.uint64)
        _check(lib().pot_tree_export(self.handle, _ptr(child), _ptr(sigma), _ptr(sh), _ptr(morton),
                                     _stream(stream)))
        return child, sigma, sh, morton

    def set_cell_index(self, enable=True, stream=None):
        """``pot_tree_set_cell_index``: free (False / "none") the cell index that replaces the
        child-array descent when locating cells, or build it: True / "default" (the layout for
        the tree's depth), "dense" (one entry per voxel, depth <= 10) or "brick" (one entry per
        4^3 brick plus the entries of bricks holding a leaf, depth 3..11)."""
        mode = CELLS[enable] if isinstance(enable, str) else (1 if enable else 0)
        _check(lib().pot_tree_set_cell_index(self.handle, mode, _stream(stream)))

    def export_cell_index(self, device=None, stream=None):
        """``pot_tree_export_cell_index``: int32 [R, R, R] indexed [x][y][z]: leaf index; for an
        empty voxel -(2 + 2 l) (inside the empty node of level l) or -(3 + 2 e) (every voxel within
        Chebyshev distance e is empty).  numpy by default; a torch tensor on ``device`` if given."""
        R = 1 << self.info()["depth"]
        if device is None:
            out = np.zeros((R, R, R), np.int32)
        else:
            import torch
            out = torch.empty((R, R, R), dtype=torch.int32, device=device)
        _check(lib().pot_tree_export_cell_index(self.handle, _ptr(out), _stream(stream)))
        return out

    def set_values(self, sigma, sh, stream=None):
        _check(lib().pot_tree_set_values(self.handle, _ptr(sigma), _ptr(sh), _stream(stream)))

    def quantize(self, bits: int = 16, stream=None) -> "Tree":
        """``pot_tree_quantize``: median-cut SH codebooks of 2^bits entries per basis function (App. B.2)."""
        out = C.c_void_p()
        _check(lib().pot_tree_quantize(self.handle, int(bits), C.byref(out), _stream(stream)))
        return Tree(out.value)

    def prune(self, score, threshold: float, stream=None) -> "Tree":
        """``pot_tree_prune``: a new tree of the leaves with score >= threshold (Sec. 3.2 "Filtering")."""
        out = C.c_void_p()
        _check(lib().pot_tree_prune(self.handle, _ptr(score), float(threshold), C.byref(out), _stream(stream)))
        return Tree(out.value)


# ----------------------------------------------------------------------------
# calls
# ----------------------------------------------------------------------------

def query(tree: Tree, xyz, out=None, stream=None):
    """``pot_query``: leaf index per point (torch int32 tensor on the points' device)."""
    import torch
    n = int(xyz.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=xyz.device)
    _check(lib().pot_query(tree.handle, n, _ptr(xyz), _ptr(out), _stream(stream)))
    return out


def sh_basis(K: int, dirs, out=None, stream=None):
    import torch
    n = int(dirs.shape[0])
    if out is None:
        out = torch.empty((n, K), dtype=torch.float32, device=dirs.device)
    _check(lib().pot_sh_basis(K, n, _ptr(dirs), _ptr(out), _stream(stream)))
    return out


def render(tree: Tree, cams, rgb=None, t_final=None, bg=(0.0, 0.0, 0.0), gamma=0.0, want_t_final=False,
           seg_count=None, leaf_touched=None, max_steps=0, device="cuda", stream=None):
    """``pot_render``: rgb [n_cams, H, W, 3] float32 (torch, on ``device`` unless given)."""
    import torch
    carr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    n = len(carr)
    H, W = (carr[0].height, carr[0].width) if n else (0, 0)
    if rgb is None:
        rgb = torch.empty((n, H, W, 3), dtype=torch.float32, device=device)
    if want_t_final and t_final is None:
        t_final = torch.empty((n, H, W), dtype=torch.float32, device=rgb.device if hasattr(rgb, "device") else device)
    o = _opts(bg, gamma, seg_count=seg_count, leaf_touched=leaf_touched, max_steps=max_steps)
    _check(lib().pot_render(tree.handle, carr, n, C.byref(o), _ptr(rgb), _ptr(t_final), _stream(stream)))
    return (rgb, t_final) if want_t_final else rgb


def render_noalloc(tree: Tree, cams, rgb, t_final=None, bg=(0.0, 0.0, 0.0), gamma=0.0, max_steps=0, stream=None):
    """``pot_render_noalloc``: as ``render`` into caller-allocated device tensors, with no GPU
    allocation inside the call (at most 1024 cameras; calls that overlap on the GPU must be
    serialised by the caller, since they share the library's fixed scratch)."""
    carr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    o = _opts(bg, gamma, max_steps=max_steps)
    _check(lib().pot_render_noalloc(tree.handle, carr, len(carr), C.byref(o), _ptr(rgb), _ptr(t_final),
                                    _stream(stream)))
    return rgb


def render_rays(tree: Tree, origins, dirs, rgb=None, t_final=None, bg=(0.0, 0.0, 0.0), gamma=0.0,
                near=0.0, far=3.0e38, want_t_final=False, seg_count=None, leaf_touched=None, max_steps=0,
                stream=None):
    """``pot_render_rays``: rgb [n, 3] float32 on the rays' device."""
    import torch
    n = int(origins.shape[0])
    dev = origins.device if hasattr(origins, "device") else "cpu"
    if rgb is None:
        rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    if want_t_final and t_final is None:
        t_final = torch.empty(n, dtype=torch.float32, device=dev)
    o = _opts(bg, gamma, near, far, seg_count=seg_count, leaf_touched=leaf_touched, max_steps=max_steps)
    _check(lib().pot_render_rays(tree.handle, n, _ptr(origins), _ptr(dirs), C.byref(o), _ptr(rgb),
                                 _ptr(t_final), _stream(stream)))
    return (rgb, t_final) if want_t_final else rgb


def check(stream=None):
    """``pot_check``: synchronise and raise on a device-side traversal error."""
    _check(lib().pot_check(_stream(stream)))


# ----------------------------------------------------------------------------
# differentiation and optimisation (App. B.3, Sec. 3.3)
# ----------------------------------------------------------------------------

def render_backward(tree: Tree, origins, dirs, grad_rgb, rgb_fwd=None, grad_sigma=None, grad_sh=None,
                    bg=(0.0, 0.0, 0.0), gamma=0.0, near=0.0, far=3.0e38, stream=None):
    """``pot_render_backward``: accumulates into (and returns) grad_sigma [L], grad_sh [L, K, 3]."""
    import torch
    inf = tree.info()
    L, K = inf["n_leaves"], inf["sh_dim"]
    dev = origins.device
    if grad_sigma is None:
        grad_sigma = torch.zeros(L, dtype=torch.float32, device=dev)
    if grad_sh is None:
        grad_sh = torch.zeros((L, K, 3), dtype=torch.float32, device=dev)
    o = _opts(bg, gamma, near, far)
    _check(lib().pot_render_backward(tree.handle, int(origins.shape[0]), _ptr(origins), _ptr(dirs), _ptr(grad_rgb),
                                     _ptr(rgb_fwd), C.byref(o), _ptr(grad_sigma), _ptr(grad_sh), _stream(stream)))
    return grad_sigma, grad_sh


def render_mse_backward(tree: Tree, origins, dirs, target, grad_sigma=None, grad_sh=None, rgb=None, loss=None,
                        bg=(0.0, 0.0, 0.0), gamma=0.0, near=0.0, far=3.0e38, stream=None):
    """``pot_render_mse_backward``: renders the rays, writes the MSE against ``target`` to ``loss``
    (a 1-element device tensor) and accumulates its gradients; returns (loss, grad_sigma, grad_sh)."""
    import torch
    inf = tree.info()
    L, K = inf["n_leaves"], inf["sh_dim"]
    dev = origins.device
    if grad_sigma is None:
        grad_sigma = torch.zeros(L, dtype=torch.float32, device=dev)
    if grad_sh is None:
        grad_sh = torch.zeros((L, K, 3), dtype=torch.float32, device=dev)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
    o = _opts(bg, gamma, near, far)
    _check(lib().pot_render_mse_backward(tree.handle, int(origins.shape[0]), _ptr(origins), _ptr(dirs),
                                         _ptr(target), C.byref(o), _ptr(rgb), _ptr(loss), _ptr(grad_sigma),
                                         _ptr(grad_sh), _stream(stream)))
    return loss, grad_sigma, grad_sh


SEGMENT_RECORD_BYTES = 32
SEGMENT_BLOCK = 128


class SegmentRecords:
    """Device buffer of ``pot_render_rays_record``: ``capacity`` records of 32 bytes
    (viewed as float32 [capacity, 8]) and the two-int64 state (slots handed out,
    overflow flag)."""

    def __init__(self, capacity: int, device="cuda"):
        import torch
        self.capacity = int(capacity)
        self.records = torch.empty((max(self.capacity, 1), 8), dtype=torch.float32, device=device)
        self.state = torch.zeros(2, dtype=torch.int64, device=device)

    @classmethod
    def for_rays(cls, n_rays: int, segments_per_ray: int = 64, device="cuda") -> "SegmentRecords":
        """A buffer for ``n_rays`` rays of up to ``segments_per_ray`` composited leaf
        segments on average, plus one block of slots per resident warp."""
        return cls(int(n_rays) * int(segments_per_ray) + 152 * 64 * SEGMENT_BLOCK, device=device)

    def used(self) -> int:
        """Slots handed out by the last recording forward (synchronises)."""
        return int(self.state[0].item())

    def overflowed(self) -> bool:
        """Whether the last recording forward ran out of slots (synchronises)."""
        return bool(self.state[1].item())


def render_rays_record(tree: Tree, origins, dirs, records: SegmentRecords, rgb=None, t_final=None,
                       bg=(0.0, 0.0, 0.0), gamma=0.0, near=0.0, far=3.0e38, want_t_final=False, stream=None):
    """``pot_render_rays_record``: the colours of ``render_rays`` (rgb [n, 3]) and a record per
    composited leaf segment in ``records``."""
    import torch
    n = int(origins.shape[0])
    if rgb is None:
        rgb = torch.empty((n, 3), dtype=torch.float32, device=origins.device)
    if want_t_final and t_final is None:
        t_final = torch.empty(n, dtype=torch.float32, device=origins.device)
    o = _opts(bg, gamma, near, far)
    _check(lib().pot_render_rays_record(tree.handle, n, _ptr(origins), _ptr(dirs), C.byref(o), _ptr(rgb),
                                        _ptr(t_final), _ptr(records.records), records.capacity,
                                        _ptr(records.state), _stream(stream)))
    return (rgb, t_final) if want_t_final else rgb


def render_backward_recorded(tree: Tree, origins, dirs, grad_rgb, rgb_fwd, records: SegmentRecords,
                             grad_sigma=None, grad_sh=None, bg=(0.0, 0.0, 0.0), gamma=0.0, near=0.0, far=3.0e38,
                             stream=None):
    """``pot_render_backward_recorded``: the gradients of ``render_backward`` from the records of the
    ``render_rays_record`` call that produced ``rgb_fwd``; accumulates into (and returns) grad_sigma [L],
    grad_sh [L, K, 3]."""
    import torch
    inf = tree.info()
    L, K = inf["n_leaves"], inf["sh_dim"]
    dev = origins.device
    if grad_sigma is None:
        grad_sigma = torch.zeros(L, dtype=torch.float32, device=dev)
    if grad_sh is None:
        grad_sh = torch.zeros((L, K, 3), dtype=torch.float32, device=dev)
    o = _opts(bg, gamma, near, far)
    _check(lib().pot_render_backward_recorded(tree.handle, int(origins.shape[0]), _ptr(origins), _ptr(dirs),
                                              _ptr(grad_rgb), _ptr(rgb_fwd), C.byref(o), _ptr(records.records),
                                              records.capacity, _ptr(records.state), _ptr(grad_sigma),
                                              _ptr(grad_sh), _stream(stream)))
    return grad_sigma, grad_sh


def step_state_floats(tree: Tree, kind: str) -> int:
    return int(lib().pot_step_state_floats(tree.handle, OPTIMIZERS[kind]))


def step(tree: Tree, grad_sigma, grad_sh, state=None, kind="rmsprop", lr_sigma=1e-2, lr_sh=1e-2, alpha=0.99,
         beta1=0.9, beta2=0.999, eps=1e-8, step_index=1, stream=None):
    """``pot_step``: one optimiser step on the tree's leaf values (float32 trees)."""
    d = StepDesc(OPTIMIZERS[kind], lr_sigma, lr_sh, alpha, beta1, beta2, eps, step_index)
    _check(lib().pot_step(tree.handle, C.byref(d), _ptr(grad_sigma), _ptr(grad_sh), _ptr(state), _stream(stream)))


def loss_mse(rgb, target, grad=None, want_grad=True, stream=None):
    """``pot_loss_mse``: (loss [1] tensor, grad [n,3] or None)."""
    import torch
    n = int(rgb.shape[0])
    loss = torch.empty(1, dtype=torch.float32, device=rgb.device)
    if want_grad and grad is None:
        grad = torch.empty_like(rgb)
    _check(lib().pot_loss_mse(n, _ptr(rgb), _ptr(target), _ptr(grad if want_grad else None), _ptr(loss),
                              _stream(stream)))
    return loss, grad


def camera_rays(cams, pixels=None, n=None, device="cuda", stream=None):
    """``pot_camera_rays``: (origins, dirs) [n,3] for global pixel indices (int64 tensor) or all pixels."""
    import torch
    carr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    if pixels is not None:
        n = int(pixels.shape[0])
        device = pixels.device
    elif n is None:
        n = len(carr) * carr[0].width * carr[0].height
    o = torch.empty((n, 3), dtype=torch.float32, device=device)
    d = torch.empty((n, 3), dtype=torch.float32, device=device)
    _check(lib().pot_camera_rays(carr, len(carr), n, _ptr(pixels), _ptr(o), _ptr(d), _stream(stream)))
    return o, d


def _autograd_fn():
    import torch

    class RenderRaysFn(torch.autograd.Function):
        """rgb = render(tree, rays); gradients flow to two placeholder tensors
        standing for the tree's sigma [L] and SH [L,K,3] (their values are the
        tree's; the tree itself is updated by ``step`` or ``Tree.set_values``)."""

        @staticmethod
        def forward(ctx, sigma_param, sh_param, tree, origins, dirs, bg, gamma, near, far, records):
            if records is None:
                rgb = render_rays(tree, origins, dirs, bg=bg, gamma=gamma, near=near, far=far)
            else:
                rgb = render_rays_record(tree, origins, dirs, records, bg=bg, gamma=gamma, near=near, far=far)
            ctx.save_for_backward(origins, dirs, rgb)
            ctx.tree = tree
            ctx.records = records
            ctx.cfg = (bg, gamma, near, far)
            ctx.shapes = (sigma_param.shape, sh_param.shape)
            return rgb

        @staticmethod
        def backward(ctx, grad_rgb):
            o, d, rgb = ctx.saved_tensors
            bg, gamma, near, far = ctx.cfg
            if ctx.records is None:
                gs, gh = render_backward(ctx.tree, o, d, grad_rgb.contiguous(), rgb_fwd=rgb, bg=bg, gamma=gamma,
                                         near=near, far=far)
            else:
                gs, gh = render_backward_recorded(ctx.tree, o, d, grad_rgb.contiguous(), rgb, ctx.records, bg=bg,
                                                  gamma=gamma, near=near, far=far)
            return (gs.reshape(ctx.shapes[0]), gh.reshape(ctx.shapes[1]), None, None, None, None, None, None, None,
                    None)

    return RenderRaysFn


_RenderRaysFn = None


def render_rays_diff(tree: Tree, sigma_param, sh_param, origins, dirs, bg=(0.0, 0.0, 0.0), gamma=0.0, near=0.0,
                     far=3.0e38, records: "SegmentRecords | None" = None):
    """Differentiable ``render_rays`` (torch.autograd.Function around pot_render_rays / pot_render_backward;
    with ``records``, around pot_render_rays_record / pot_render_backward_recorded: the buffer keeps this
    forward's records until its backward, so give each live forward its own buffer)."""
    global _RenderRaysFn
    if _RenderRaysFn is None:
        _RenderRaysFn = _autograd_fn()
    return _RenderRaysFn.apply(sigma_param, sh_param, tree, origins, dirs, tuple(bg), float(gamma), float(near),
                               float(far), records)


def allreduce_leaf_grads(grad_sigma, grad_sh, op="mean", group=None):
    """The exchange of data-parallel octree optimisation (Sec. 3.3 with the ray
    batch split across ranks, the tree replicated on every rank): each rank
    holds the leaf gradients of its part of the batch; after one all-reduce
    per array every rank holds the gradient of the whole batch, so identical
    optimiser steps keep the replicas equal.  ``op="mean"``: the ranks'
    gradients are averaged, which is the gradient of the whole batch's mean
    loss when every rank's loss is the mean over an equal share of the rays
    (``pot_loss_mse``); ``op="sum"`` for summed losses.  In place; nothing to
    do without an initialised process group of more than one rank."""
    import torch.distributed as dist
    if op not in ("mean", "sum"):
        raise ValueError("op must be 'mean' or 'sum'")
    if not dist.is_available() or not dist.is_initialized():
        return
    world = dist.get_world_size(group)
    if world == 1:
        return
    for g in (grad_sigma, grad_sh):
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
        if op == "mean":
            g.div_(world)


class LeafOptimizer:
    """Owns the optimiser state of ``pot_step`` for one float32 tree.  With
    ``data_parallel=True`` (a process group initialised, one rank per GPU,
    every rank holding the same tree) each step first averages the ranks'
    gradients with ``allreduce_leaf_grads``."""

    def __init__(self, tree: Tree, kind="rmsprop", lr_sigma=1e-2, lr_sh=1e-2, alpha=0.99, beta1=0.9, beta2=0.999,
                 eps=1e-8, data_parallel=False, group=None):
        import torch
        self.tree, self.kind = tree, kind
        self.hp = dict(lr_sigma=lr_sigma, lr_sh=lr_sh, alpha=alpha, beta1=beta1, beta2=beta2, eps=eps)
        nst = step_state_floats(tree, kind)
        self.state = torch.zeros(max(nst, 1), dtype=torch.float32, device="cuda")
        self.t = 0
        self.data_parallel, self.group = data_parallel, group

    def step(self, grad_sigma, grad_sh, stream=None):
        if self.data_parallel:
            allreduce_leaf_grads(grad_sigma, grad_sh, "mean", self.group)
        self.t += 1
        step(self.tree, grad_sigma, grad_sh, self.state, self.kind, step_index=self.t, stream=stream, **self.hp)


def render_batch(items, stream=None):
    """``pot_render_batch``: items = [(tree, camera record, rgb tensor [H,W,3], bg, gamma, t_final or None)]."""
    arr = (RenderItem * len(items))()
    for k, (tree, cam, rgb, bg, gamma, tf) in enumerate(items):
        r = arr[k]
        r.tree = tree.handle
        C.memmove(C.byref(r.cam), np.ascontiguousarray(cam).ctypes.data, 80)
        r.bg[0], r.bg[1], r.bg[2] = bg
        r.gamma = gamma
        r.rgb = rgb.data_ptr()
        r.t_final = None if tf is None else tf.data_ptr()
    _check(lib().pot_render_batch(arr, len(items), _stream(stream)))


def visibility(tree: Tree, cams, max_weight=None, gamma=0.0, stream=None):
    """``pot_visibility``: per-leaf max ray weight over the cameras' pixels (accumulates by max)."""
    import torch
    carr = cams if isinstance(cams, C.Array) else make_cameras(cams)
    if max_weight is None:
        max_weight = torch.zeros(tree.info()["n_leaves"], dtype=torch.float32, device="cuda")
    o = _opts((0.0, 0.0, 0.0), gamma)
    _check(lib().pot_visibility(tree.handle, carr, len(carr), C.byref(o), _ptr(max_weight), _stream(stream)))
    return max_weight
