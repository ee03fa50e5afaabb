"""Python access to the FP64 CPU oracle (``pot_oracle.c``) plus the optimiser
step, restated in numpy.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  The product
path (the ``paper_2103_14024_gb300`` package and its CUDA library) never
imports it, and this module never imports the product path.

Parity of every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, brute force, library special cases).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pot_oracle.c")
_LIB = os.path.join(_HERE, "libpot_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_p = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_dbl = C.c_double


def _declare(L):
    L.oracle_build_sparse.restype = _p
    L.oracle_build_sparse.argtypes = [C.c_int, _p, C.c_float, C.c_int, C.c_int, _i64, _p, _p, _p,
                                      C.POINTER(C.c_int)]
    L.oracle_build_dense.restype = _p
    L.oracle_build_dense.argtypes = [C.c_int, _p, C.c_float, C.c_int, C.c_int, C.c_float, _p, _p,
                                     C.POINTER(C.c_int)]
    L.oracle_tree_free.argtypes = [_p]
    L.oracle_tree_n_nodes.restype = _i64
    L.oracle_tree_n_nodes.argtypes = [_p]
    L.oracle_tree_n_leaves.restype = _i64
    L.oracle_tree_n_leaves.argtypes = [_p]
    L.oracle_tree_export.argtypes = [_p, _p, _p, _p, _p]
    L.oracle_round_values.restype = C.c_int
    L.oracle_round_values.argtypes = [C.c_int, _i64, _p, _p]
    L.oracle_query.argtypes = [_p, _i64, _p, _p]
    L.oracle_trace_ray.restype = C.c_int
    L.oracle_trace_ray.argtypes = [_p, _p, _p, _dbl, _dbl, C.c_int, _p, _p, _p, _p]
    L.oracle_sh_basis.argtypes = [C.c_int, _i64, _p, _p]
    L.oracle_num_threads.restype = C.c_int
    L.oracle_set_num_threads.argtypes = [C.c_int]
    L.oracle_render_rays.argtypes = [_p, _i64, _p, _p, _dbl, _dbl, _p, _dbl, _p, _p, _p, _p]
    L.oracle_cam_rays.argtypes = [_p, C.c_int, _p, _p]
    L.oracle_render_cams.argtypes = [_p, _p, C.c_int, _p, _dbl, _p, _p, _p, _p]
    L.oracle_render_pixels.argtypes = [_p, _p, _i64, _p, _p, _p, _p, _dbl, _p, _p, _p]
    L.oracle_backward_rays.argtypes = [_p, _i64, _p, _p, _dbl, _dbl, _p, _dbl, _p, _p, _p]
    L.oracle_visibility.argtypes = [_p, _p, C.c_int, _dbl, _p]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


DTYPES = {"f32": 0, "f16": 1, "bf16": 2}


class OTree:
    """An oracle tree (FP64 leaf values, canonical arrays)."""

    def __init__(self, handle, depth, lo, size, sh_degree):
        self._h = handle
        self.depth = depth
        self.bbox_lo = tuple(float(v) for v in lo)
        self.bbox_size = float(size)
        self.sh_degree = sh_degree
        self.K = (sh_degree + 1) ** 2

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            lib().oracle_tree_free(h)

    @property
    def n_nodes(self) -> int:
        return int(lib().oracle_tree_n_nodes(self._h))

    @property
    def n_leaves(self) -> int:
        return int(lib().oracle_tree_n_leaves(self._h))

    def export(self):
        """(child int32 [N,8], sigma f64 [L], sh f64 [L,K,3], morton u64 [L])."""
        N, L = self.n_nodes, self.n_leaves
        child = np.zeros((N, 8), dtype=np.int32)
        sigma = np.zeros(L, dtype=np.float64)
        sh = np.zeros((L, self.K, 3), dtype=np.float64)
        morton = np.zeros(L, dtype=np.uint64)
        lib().oracle_tree_export(self._h, _ptr(child), _ptr(sigma), _ptr(sh), _ptr(morton))
        return child, sigma, sh, morton


class OracleError(ValueError):
    pass


def build_sparse(scene, dtype: str = "f32") -> OTree:
    lo = _c(scene.bbox_lo, np.float32)
    m = _c(scene.morton, np.uint64)
    s = _c(scene.sigma, np.float32)
    h = _c(scene.sh, np.float32)
    err = C.c_int(0)
    t = lib().oracle_build_sparse(scene.depth, _ptr(lo), C.c_float(scene.bbox_size), scene.sh_degree,
                                  DTYPES[dtype], m.shape[0], _ptr(m), _ptr(s), _ptr(h), C.byref(err))
    if not t:
        raise OracleError(f"oracle_build_sparse failed ({err.value})")
    return OTree(t, scene.depth, scene.bbox_lo, scene.bbox_size, scene.sh_degree)


def build_dense(depth, lo, size, sh_degree, sigma, sh, tau: float = 0.0, dtype: str = "f32") -> OTree:
    lo32 = _c(lo, np.float32)
    s = _c(sigma, np.float32)
    h = _c(sh, np.float32)
    err = C.c_int(0)
    t = lib().oracle_build_dense(depth, _ptr(lo32), C.c_float(size), sh_degree, DTYPES[dtype],
                                 C.c_float(tau), _ptr(s), _ptr(h), C.byref(err))
    if not t:
        raise OracleError(f"oracle_build_dense failed ({err.value})")
    return OTree(t, depth, lo, size, sh_degree)


def round_values(x, dtype: str):
    """fp16 / bf16 rounding of stored leaf values; returns (float32 values, overflow flag)."""
    x = _c(x, np.float32)
    out = np.empty_like(x)
    ovf = lib().oracle_round_values(DTYPES[dtype], x.size, _ptr(x), _ptr(out))
    return out, bool(ovf)


def query(tree: OTree, xyz) -> np.ndarray:
    xyz = _c(xyz, np.float32).reshape(-1, 3)
    out = np.empty(xyz.shape[0], dtype=np.int32)
    lib().oracle_query(tree._h, xyz.shape[0], _ptr(xyz), _ptr(out))
    return out


def trace_ray(tree: OTree, o, d, near=0.0, far=1e30):
    """Segments of one ray: (leaf int64 [n] (-1 empty), t0, t1, delta (world length))."""
    o = _c(o, np.float32)
    d = _c(d, np.float32)
    cap = 3 * (1 << tree.depth) + 16
    leaf = np.empty(cap, dtype=np.int64)
    t0, t1, dl = (np.empty(cap) for _ in range(3))
    n = lib().oracle_trace_ray(tree._h, _ptr(o), _ptr(d), near, far, cap, _ptr(leaf), _ptr(t0),
                               _ptr(t1), _ptr(dl))
    return leaf[:n].copy(), t0[:n].copy(), t1[:n].copy(), dl[:n].copy()


def sh_basis(K: int, dirs) -> np.ndarray:
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    Y = np.empty((dirs.shape[0], K))
    lib().oracle_sh_basis(K, dirs.shape[0], _ptr(dirs), _ptr(Y))
    return Y


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def render_rays(tree: OTree, o, d, near=0.0, far=1e30, bg=(0.0, 0.0, 0.0), gamma=0.0,
                want_touched=False):
    """Returns dict(rgb f64 [n,3], t_final [n], n_seg int32 [n], touched uint8 [L] or None)."""
    o = _c(o, np.float32).reshape(-1, 3)
    d = _c(d, np.float32).reshape(-1, 3)
    n = o.shape[0]
    rgb = np.zeros((n, 3))
    tf = np.zeros(n)
    ns = np.zeros(n, dtype=np.int32)
    touched = np.zeros(tree.n_leaves, dtype=np.uint8) if want_touched else None
    bgv = _c(bg, np.float64)
    lib().oracle_render_rays(tree._h, n, _ptr(o), _ptr(d), near, far, _ptr(bgv), gamma, _ptr(rgb),
                             _ptr(tf), _ptr(ns), _ptr(touched))
    return {"rgb": rgb, "t_final": tf, "n_seg": ns, "touched": touched}


def cam_rays(cams):
    """fp32 (origins, directions) of every pixel, [n_cams*H*W, 3] each (row-major pixels)."""
    cams = np.ascontiguousarray(cams)
    n = int(sum(int(c["width"]) * int(c["height"]) for c in cams))
    o = np.empty((n, 3), dtype=np.float32)
    d = np.empty((n, 3), dtype=np.float32)
    lib().oracle_cam_rays(_ptr(cams), len(cams), _ptr(o), _ptr(d))
    return o, d


def render_cams(tree: OTree, cams, bg=(0.0, 0.0, 0.0), gamma=0.0, want_touched=False):
    """rgb f64 [n_cams, H, W, 3] (all cameras the same size), t_final, n_seg, touched."""
    cams = np.ascontiguousarray(cams)
    nc = len(cams)
    H, W = int(cams[0]["height"]), int(cams[0]["width"])
    assert all(int(c["height"]) == H and int(c["width"]) == W for c in cams)
    rgb = np.zeros((nc, H, W, 3))
    tf = np.zeros((nc, H, W))
    ns = np.zeros((nc, H, W), dtype=np.int32)
    touched = np.zeros(tree.n_leaves, dtype=np.uint8) if want_touched else None
    bgv = _c(bg, np.float64)
    lib().oracle_render_cams(tree._h, _ptr(cams), nc, _ptr(bgv), gamma, _ptr(rgb), _ptr(tf), _ptr(ns),
                             _ptr(touched))
    return {"rgb": rgb, "t_final": tf, "n_seg": ns, "touched": touched}


def render_pixels(tree: OTree, cams, cam_idx, px, py, bg=(0.0, 0.0, 0.0), gamma=0.0):
    cams = np.ascontiguousarray(cams)
    ci = _c(cam_idx, np.int32)
    x = _c(px, np.int32)
    y = _c(py, np.int32)
    n = ci.shape[0]
    rgb = np.zeros((n, 3))
    tf = np.zeros(n)
    ns = np.zeros(n, dtype=np.int32)
    bgv = _c(bg, np.float64)
    lib().oracle_render_pixels(tree._h, _ptr(cams), n, _ptr(ci), _ptr(x), _ptr(y), _ptr(bgv), gamma,
                               _ptr(rgb), _ptr(tf), _ptr(ns))
    return {"rgb": rgb, "t_final": tf, "n_seg": ns}


def backward_rays(tree: OTree, o, d, grad_rgb, near=0.0, far=1e30, bg=(0.0, 0.0, 0.0), gamma=0.0):
    """(grad_sigma f64 [L], grad_sh f64 [L,K,3]) of sum(grad_rgb * rgb)."""
    o = _c(o, np.float32).reshape(-1, 3)
    d = _c(d, np.float32).reshape(-1, 3)
    g = _c(grad_rgb, np.float64).reshape(-1, 3)
    gs = np.zeros(tree.n_leaves)
    gh = np.zeros((tree.n_leaves, tree.K, 3))
    bgv = _c(bg, np.float64)
    lib().oracle_backward_rays(tree._h, o.shape[0], _ptr(o), _ptr(d), near, far, _ptr(bgv), gamma,
                               _ptr(g), _ptr(gs), _ptr(gh))
    return gs, gh


def visibility(tree: OTree, cams, gamma=0.0):
    """Largest ray weight T (1 - exp(-sigma delta)) each leaf receives over all
    pixels of ``cams`` (Sec. 3.2 "Filtering"); float64 [n_leaves]."""
    cams = np.ascontiguousarray(cams)
    out = np.zeros(tree.n_leaves)
    lib().oracle_visibility(tree._h, _ptr(cams), len(cams), gamma, _ptr(out))
    return out


def prune(scene, scores, threshold):
    """The scene restricted to the voxels whose score >= threshold (the leaves of
    the filtered octree, Sec. 3.2 "Filtering"), in their Morton order."""
    keep = np.asarray(scores) >= threshold
    return scene.replace(morton=scene.morton[keep], sigma=scene.sigma[keep], sh=scene.sh[keep])


# ----------------------------------------------------------------------------
# Optimiser step (Sec. 3.3 fine-tunes leaf values by gradient descent on the
# NeRF loss; the step rules below are the textbook definitions)
# ----------------------------------------------------------------------------

def step_sgd(x, g, lr):
    """x <- x - lr g."""
    return x - lr * g


def step_rmsprop(x, g, v, lr, alpha=0.99, eps=1e-8):
    """v <- alpha v + (1 - alpha) g^2;  x <- x - lr g / (sqrt(v) + eps)."""
    v = alpha * v + (1.0 - alpha) * g * g
    return x - lr * g / (np.sqrt(v) + eps), v


def step_adam(x, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) with bias correction; ``step`` counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return x - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------------------------
# SH codebook quantisation (App. B.2): median cut per SH basis function
# ----------------------------------------------------------------------------

def median_cut(points, bits: int):
    """Median-cut quantisation (Heckbert) of float32 points [n, 3] into 2^bits
    boxes, every box split at every level: the split axis is the box's longest
    extent (ties: lowest channel); the box's points are ordered by (value on
    that axis, point index) and split at floor(n/2); boxes of fewer than two
    points keep them and get an empty sibling.  Returns (codebook float16
    [2^bits, 3] = the fp64 mean of each box in box order rounded once to fp16,
    0 for empty boxes; codes uint16 [n])."""
    P = np.asarray(points, dtype=np.float32)
    n = P.shape[0]
    order = np.arange(n, dtype=np.int64)
    starts = np.array([0], dtype=np.int64)
    ends = np.array([n], dtype=np.int64)
    for _ in range(bits):
        sizes = ends - starts
        box_of = np.repeat(np.arange(starts.shape[0]), sizes)
        vals = P[order].astype(np.float64)
        big = sizes >= 2
        # per-box extents (boxes with >= 1 point)
        nz = sizes > 0
        mx = np.full((starts.shape[0], 3), -np.inf)
        mn = np.full((starts.shape[0], 3), np.inf)
        if n:
            mx[nz] = np.maximum.reduceat(vals, starts[nz], axis=0)
            mn[nz] = np.minimum.reduceat(vals, starts[nz], axis=0)
        axis = np.argmax(np.where(nz[:, None], mx - mn, -1.0), axis=1)
        key = vals[np.arange(n), axis[box_of]] if n else vals[:, 0]
        # sort inside boxes that split: by (box, value on the box's axis, point index)
        key = np.where(big[box_of], key, 0.0)
        perm = np.lexsort((order, key, box_of))
        order = order[perm]
        mids = starts + sizes // 2
        mids = np.where(big, mids, ends)
        new_s = np.stack([starts, mids], axis=1).reshape(-1)
        new_e = np.stack([mids, ends], axis=1).reshape(-1)
        starts, ends = new_s, new_e
    C = starts.shape[0]
    codebook = np.zeros((C, 3), dtype=np.float16)
    codes = np.zeros(n, dtype=np.uint16)
    for j in range(C):
        s, e = starts[j], ends[j]
        if e > s:
            idx = order[s:e]
            acc = np.zeros(3)
            for i in idx:                       # sequential fp64 sum in box order
                acc = acc + P[i].astype(np.float64)
            codebook[j] = (acc / (e - s)).astype(np.float16)
            codes[idx] = j
    return codebook, codes


def quantize_scene(scene, bits: int):
    """The scene with each SH basis function's RGB coefficients replaced by their
    median-cut codebook entries (float16) and sigma kept as it is (App. B.2),
    i.e. the values a quantised tree stores; also the codebooks and codes."""
    K = scene.sh_dim
    sh = np.empty_like(scene.sh)
    books, codes = [], []
    for k in range(K):
        cb, cd = median_cut(scene.sh[:, k, :], bits)
        sh[:, k, :] = cb[cd].astype(np.float32)
        books.append(cb)
        codes.append(cd)
    return scene.replace(sh=sh), np.stack(books), np.stack(codes, axis=1)
