"""Seeded synthetic inputs for the PlenOctree render path: scenes and cameras.

This module produces *inputs only*.  It holds none of the rendering arithmetic
(no ray generation, traversal, spherical harmonics or compositing): it emits
occupied voxels with their density and SH coefficients, and pinhole cameras as
fp32 camera-to-world matrices.  Both the CUDA path and the CPU oracle consume
exactly the arrays produced here.

Random numbers are counter based: every value is a SplitMix64 hash of
(seed, stream, voxel Morton code), so a voxel's value does not depend on the
order in which voxels are generated, and a tree at depth 9 can be produced
sparsely without ever materialising the dense 512^3 grid.  SplitMix64 is the
published mixing function of Steele, Lea and Flood ("Fast splittable
pseudorandom number generators", OOPSLA 2014).

Voxel Morton code (input format of ``pot_build_sparse``): bits of the integer
voxel coordinates interleaved with x most significant in each triple,
``m = sum_b x_b << (3b+2) | y_b << (3b+1) | z_b << 3b``.

Scene shapes follow the workloads of the paper's experiments (Sec. 4.1: 800x800
views of objects occupying a few percent of a 512^3 grid, SH degree 3, Table 1)
with synthetic content in place of the NeRF-synthetic dataset.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_U64 = np.uint64
_GOLDEN = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 counters."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
        return z ^ (z >> _U64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    k = splitmix64(np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)], dtype=np.uint64))
    return k[0]


def hash_u64(seed: int, stream: int, codes: np.ndarray) -> np.ndarray:
    """64 random bits per counter, keyed by (seed, stream)."""
    codes = np.asarray(codes, dtype=np.uint64)
    return splitmix64(codes ^ _stream_key(seed, stream))


def uniform(seed: int, stream: int, codes: np.ndarray) -> np.ndarray:
    """U[0,1) float64 from the top 53 bits of the hash."""
    h = hash_u64(seed, stream, codes)
    return (h >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_pair(seed: int, stream: int, codes: np.ndarray):
    """Two independent N(0,1) float64 arrays per counter (Box-Muller on one 64-bit hash)."""
    h = hash_u64(seed, stream, codes)
    u1 = ((h >> _U64(32)).astype(np.float64) + 0.5) * (1.0 / 4294967296.0)   # (0,1)
    u2 = (h & _U64(0xFFFFFFFF)).astype(np.float64) * (1.0 / 4294967296.0)     # [0,1)
    r = np.sqrt(-2.0 * np.log(u1))
    a = 2.0 * math.pi * u2
    return r * np.cos(a), r * np.sin(a)


# ----------------------------------------------------------------------------
# Morton codes (input format)
# ----------------------------------------------------------------------------

def morton_encode(x, y, z, depth: int) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    m = np.zeros(np.broadcast(x, y, z).shape, dtype=np.uint64)
    one = _U64(1)
    for b in range(depth):
        bb = _U64(b)
        m |= ((x >> bb) & one) << _U64(3 * b + 2)
        m |= ((y >> bb) & one) << _U64(3 * b + 1)
        m |= ((z >> bb) & one) << _U64(3 * b)
    return m


def morton_decode(m, depth: int):
    m = np.asarray(m, dtype=np.uint64)
    x = np.zeros(m.shape, dtype=np.int64)
    y = np.zeros(m.shape, dtype=np.int64)
    z = np.zeros(m.shape, dtype=np.int64)
    one = _U64(1)
    for b in range(depth):
        x |= (((m >> _U64(3 * b + 2)) & one).astype(np.int64)) << b
        y |= (((m >> _U64(3 * b + 1)) & one).astype(np.int64)) << b
        z |= (((m >> _U64(3 * b)) & one).astype(np.int64)) << b
    return x, y, z


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    """A sparse set of occupied voxels, sorted by Morton code (strictly increasing).

    sigma: float32 [n];  sh: float32 [n, K, 3] (basis-major, RGB innermost).
    """
    depth: int
    bbox_lo: tuple
    bbox_size: float
    sh_degree: int
    morton: np.ndarray
    sigma: np.ndarray
    sh: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.morton.shape[0])

    @property
    def sh_dim(self) -> int:
        return (self.sh_degree + 1) ** 2

    @property
    def res(self) -> int:
        return 1 << self.depth

    def to_dense(self, fill_sigma: float = 0.0, noise_seed: int | None = None):
        """Dense grids sigma[R][R][R] and sh[R][R][R][K][3] indexed [x][y][z].

        Unoccupied voxels get ``fill_sigma`` and, if ``noise_seed`` is given,
        random SH values (a build must ignore them).
        """
        R = self.res
        sig = np.full((R, R, R), fill_sigma, dtype=np.float32)
        sh = np.zeros((R, R, R, self.sh_dim, 3), dtype=np.float32)
        if noise_seed is not None:
            allc = np.arange(R ** 3, dtype=np.uint64)
            a, b = normal_pair(noise_seed, 7, allc)
            sh += (a.reshape(R, R, R, 1, 1)).astype(np.float32)
        x, y, z = morton_decode(self.morton, self.depth)
        sig[x, y, z] = self.sigma
        sh[x, y, z] = self.sh
        return sig, sh

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


def _sort_unique(codes: np.ndarray) -> np.ndarray:
    return np.unique(np.asarray(codes, dtype=np.uint64))


def sh_coeffs(seed: int, codes: np.ndarray, sh_degree: int, std_fn) -> np.ndarray:
    """SH coefficients [n, K, 3]; coefficient (l, m, c) ~ N(0, std_fn(l))."""
    K = (sh_degree + 1) ** 2
    n = codes.shape[0]
    out = np.empty((n, K, 3), dtype=np.float32)
    flat = [(k, c) for k in range(K) for c in range(3)]
    for p in range(0, len(flat), 2):
        z0, z1 = normal_pair(seed, 1000 + p // 2, codes)
        for zz, idx in ((z0, p), (z1, p + 1)):
            if idx >= len(flat):
                break
            k, c = flat[idx]
            l = int(math.isqrt(k))
            out[:, k, c] = (zz * std_fn(l)).astype(np.float32)
    return out


def scene_tiny(seed: int = 1000) -> Scene:
    """Tiny plain render scene: a 32^3 grid over [-1,1]^3 (depth 5); a ball of
    radius 0.5 (test at voxel centres) with sigma = 20; SH degree 0 with RGB
    coefficients ~ U(-2, 2) per leaf."""
    D = 5
    R = 1 << D
    lo, size = (-1.0, -1.0, -1.0), 2.0
    idx = np.arange(R, dtype=np.float64)
    c = lo[0] + (idx + 0.5) * (size / R)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    occ = (X * X + Y * Y + Z * Z) < 0.25
    xi, yi, zi = np.nonzero(occ)
    codes = _sort_unique(morton_encode(xi, yi, zi, D))
    sigma = np.full(codes.shape, 20.0, dtype=np.float32)
    sh = np.empty((codes.shape[0], 1, 3), dtype=np.float32)
    for ch in range(3):
        sh[:, 0, ch] = (uniform(seed, 10 + ch, codes) * 4.0 - 2.0).astype(np.float32)
    return Scene(D, lo, size, 0, codes, sigma, sh, name="tiny")


def _shapes(seed: int, n_shapes: int = 8):
    ids = np.arange(n_shapes, dtype=np.uint64)
    centers = np.stack([uniform(seed, 20 + a, ids) * 1.8 - 0.9 for a in range(3)], axis=1)
    radius = uniform(seed, 24, ids) * 0.2 + 0.2                      # spheres
    half = np.stack([uniform(seed, 25 + a, ids) * 0.2 + 0.15 for a in range(3)], axis=1)  # boxes
    return centers, radius, half


def _occupied_codes(depth, lo, size, centers, radius, half, scale):
    """Morton codes of voxels whose centre lies in the union of the scaled shapes."""
    R = 1 << depth
    h = size / R
    codes = []
    for i in range(centers.shape[0]):
        c = centers[i]
        ext = (radius[i] if i % 2 == 0 else half[i].max()) * scale
        lo_i = np.clip(np.floor((c - ext - lo[0]) / h - 0.5).astype(int), 0, R - 1)
        hi_i = np.clip(np.ceil((c + ext - lo[0]) / h + 0.5).astype(int), 0, R - 1)
        ax = [np.arange(lo_i[a], hi_i[a] + 1) for a in range(3)]
        pc = [lo[a] + (ax[a] + 0.5) * h for a in range(3)]
        X, Y, Z = np.meshgrid(pc[0], pc[1], pc[2], indexing="ij")
        if i % 2 == 0:
            m = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 < (radius[i] * scale) ** 2
        else:
            hs = half[i] * scale
            m = (np.abs(X - c[0]) < hs[0]) & (np.abs(Y - c[1]) < hs[1]) & (np.abs(Z - c[2]) < hs[2])
        xi, yi, zi = np.nonzero(m)
        codes.append(morton_encode(xi + lo_i[0], yi + lo_i[1], zi + lo_i[2], depth))
    if not codes:
        return np.zeros(0, dtype=np.uint64)
    return _sort_unique(np.concatenate(codes))


def scene_shapes(seed: int = 1001, depth: int = 9, sh_degree: int = 3,
                 occupancy: float = 0.03, name: str = "main") -> Scene:
    """Main plain render scene: over [-1.5,1.5]^3, the union of 8 seeded shapes
    (even index: sphere, odd: axis-aligned box) with centres ~ U(-0.9,0.9)^3,
    uniformly rescaled so that the occupied fraction of voxel centres is
    ``occupancy`` (3 % gives about 4.0 M leaves at depth 9).  sigma ~
    lognormal(mu=3, s=1) per leaf; SH coefficient of degree l ~ N(0, 0.5/(l+1))
    (standard deviation)."""
    lo, size = (-1.5, -1.5, -1.5), 3.0
    centers, radius, half = _shapes(seed)
    # bisection of the scale on a coarse grid, then the final grid
    coarse = min(depth, 7)
    target = occupancy * (1 << (3 * coarse))
    s_lo, s_hi = 0.2, 4.0
    for _ in range(40):
        s_mid = 0.5 * (s_lo + s_hi)
        n = _occupied_codes(coarse, lo, size, centers, radius, half, s_mid).shape[0]
        if n < target:
            s_lo = s_mid
        else:
            s_hi = s_mid
    scale = 0.5 * (s_lo + s_hi)
    codes = _occupied_codes(depth, lo, size, centers, radius, half, scale)
    z0, _ = normal_pair(seed, 30, codes)
    sigma = np.exp(3.0 + 1.0 * z0).astype(np.float32)
    sh = sh_coeffs(seed, codes, sh_degree, lambda l: 0.5 / (l + 1))
    return Scene(depth, lo, size, sh_degree, codes, sigma, sh, name=name)


def scene_random(seed: int, depth: int, sh_degree: int, p_occ: float = 0.3,
                 lo=(-1.0, -1.0, -1.0), size: float = 2.0, clustered: bool = True,
                 sigma_mu: float = 1.5, sigma_s: float = 1.0, sh_std: float = 1.0) -> Scene:
    """Random tiny tree for tests: each voxel occupied with probability p_occ
    (``clustered`` makes occupancy follow coarse 2x2x2-blocks so that the tree
    has empty nodes at several levels), sigma lognormal, SH ~ N(0, sh_std)."""
    R = 1 << depth
    allc = np.arange(R ** 3, dtype=np.uint64)
    if clustered and depth >= 2:
        block = allc >> _U64(3 * min(2, depth - 1))
        u = uniform(seed, 40, block)
        keep_block = u < min(1.0, 2.0 * p_occ)
        u2 = uniform(seed, 41, allc)
        occ = keep_block & (u2 < 0.5 + 0.5 * p_occ)
    else:
        occ = uniform(seed, 41, allc) < p_occ
    codes = allc[occ]
    z0, _ = normal_pair(seed, 42, codes)
    sigma = np.exp(sigma_mu + sigma_s * z0).astype(np.float32)
    sh = sh_coeffs(seed, codes, sh_degree, lambda l: sh_std)
    return Scene(depth, tuple(float(v) for v in lo), float(size), sh_degree, codes, sigma, sh,
                 name=f"random{seed}")


def scene_uniform(depth: int, sigma: float, sh: np.ndarray, lo=(-1.0, -1.0, -1.0),
                  size: float = 2.0) -> Scene:
    """Every voxel occupied with the same density and SH coefficients [K,3]."""
    R = 1 << depth
    codes = np.arange(R ** 3, dtype=np.uint64)
    sh = np.asarray(sh, dtype=np.float32)
    K = sh.shape[0]
    deg = int(math.isqrt(K)) - 1
    return Scene(depth, tuple(float(v) for v in lo), float(size), deg, codes,
                 np.full(codes.shape, sigma, dtype=np.float32),
                 np.broadcast_to(sh, (codes.shape[0], K, 3)).copy(), name="uniform")


def perturbed(scene: Scene, seed: int, sh_noise: float = 0.3,
              sigma_lo: float = 0.5, sigma_hi: float = 1.5) -> Scene:
    """Start point of octree optimisation: sh += N(0, sh_noise), sigma *= U(lo, hi)."""
    codes = scene.morton
    sh = scene.sh.astype(np.float64).copy()
    K = scene.sh_dim
    flat = [(k, c) for k in range(K) for c in range(3)]
    for p in range(0, len(flat), 2):
        z0, z1 = normal_pair(seed, 2000 + p // 2, codes)
        for zz, idx in ((z0, p), (z1, p + 1)):
            if idx < len(flat):
                k, c = flat[idx]
                sh[:, k, c] += zz * sh_noise
    f = uniform(seed, 2100, codes) * (sigma_hi - sigma_lo) + sigma_lo
    return scene.replace(sigma=(scene.sigma.astype(np.float64) * f).astype(np.float32),
                         sh=sh.astype(np.float32), name=scene.name + "-perturbed")


# ----------------------------------------------------------------------------
# Cameras (inputs: fp32 camera-to-world matrices and intrinsics)
# ----------------------------------------------------------------------------

CAMERA_DTYPE = np.dtype([
    ("c2w", np.float32, (3, 4)),
    ("fx", np.float32), ("fy", np.float32), ("cx", np.float32), ("cy", np.float32),
    ("width", np.int32), ("height", np.int32),
    ("near", np.float32), ("far", np.float32),
])


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world [3,4] (float64): columns right, up, back (= -forward), eye.
    The camera looks along its -z axis (OpenGL / NeRF-Blender convention)."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(fwd, upv))) > 0.999999:
        upv = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, upv)
    right /= np.linalg.norm(right)
    cup = np.cross(right, fwd)
    m = np.zeros((3, 4))
    m[:, 0], m[:, 1], m[:, 2], m[:, 3] = right, cup, -fwd, eye
    return m


def make_cameras(c2ws, width, height, focal, near=0.0, far=1e30, cx=None, cy=None) -> np.ndarray:
    c2ws = list(c2ws)
    cams = np.zeros(len(c2ws), dtype=CAMERA_DTYPE)
    for i, m in enumerate(c2ws):
        cams[i]["c2w"] = np.asarray(m, dtype=np.float32)
    cams["fx"] = focal
    cams["fy"] = focal
    cams["cx"] = width * 0.5 if cx is None else cx
    cams["cy"] = height * 0.5 if cy is None else cy
    cams["width"] = width
    cams["height"] = height
    cams["near"] = near
    cams["far"] = far
    return cams


def orbit_c2ws(n: int, radius: float = 4.0, elevation_deg: float = 30.0):
    el = math.radians(elevation_deg)
    out = []
    for k in range(n):
        az = 2.0 * math.pi * k / n
        eye = (radius * math.cos(el) * math.cos(az), radius * math.cos(el) * math.sin(az),
               radius * math.sin(el))
        out.append(look_at(eye))
    return out


def hemisphere_c2ws(seed: int, n: int, radius: float = 4.0):
    """n views uniform on the upper hemisphere (z >= 0) at ``radius``, looking at the origin."""
    ids = np.arange(n, dtype=np.uint64)
    z = uniform(seed, 50, ids)
    phi = uniform(seed, 51, ids) * 2.0 * math.pi
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return [look_at((radius * r[i] * math.cos(phi[i]), radius * r[i] * math.sin(phi[i]),
                     radius * z[i])) for i in range(n)]


def cameras_tiny(variant: str = "generic") -> np.ndarray:
    """One 64x64 camera at distance 4 looking at the origin, focal 80 px."""
    if variant == "generic":
        v = np.array([1.0, 0.7, 0.5])
        eye = 4.0 * v / np.linalg.norm(v)
    elif variant == "axis":
        eye = (0.0, 0.0, 4.0)
    else:
        raise ValueError(variant)
    return make_cameras([look_at(eye)], 64, 64, 80.0)


def cameras_main(n: int = 200, width: int = 800, height: int = 800) -> np.ndarray:
    """Orbit views: azimuth 2 pi k / n, elevation 30 deg, radius 4, focal 1111 px,
    near 2, far 6."""
    return make_cameras(orbit_c2ws(n), width, height, 1111.0, near=2.0, far=6.0)


def cameras_train(seed: int = 1003, n: int = 100, width: int = 800, height: int = 800) -> np.ndarray:
    return make_cameras(hemisphere_c2ws(seed, n), width, height, 1111.0, near=2.0, far=6.0)


def random_rays(seed: int, n: int, radius: float = 4.0, spread: float = 0.6):
    """Random rays (origin on a sphere, aimed near the origin; directions not unit)."""
    ids = np.arange(n, dtype=np.uint64)
    z = uniform(seed, 60, ids) * 2.0 - 1.0
    phi = uniform(seed, 61, ids) * 2.0 * math.pi
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    o = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1) * radius
    tgt = np.stack([uniform(seed, 62 + a, ids) * 2.0 - 1.0 for a in range(3)], axis=1) * spread
    d = (tgt - o) * (0.5 + uniform(seed, 65, ids))[:, None]
    return o.astype(np.float32), d.astype(np.float32)


# ----------------------------------------------------------------------------
# The same generators evaluated with torch on a GPU (for trees with tens of
# millions of leaves).  Integer hashing is bit-identical to the numpy path;
# the float transforms (log, cos, exp) may differ in the last ulp.
# ----------------------------------------------------------------------------

def _t_consts(torch, device):
    def s64(v):
        return torch.tensor(v - (1 << 64) if v >= (1 << 63) else v, dtype=torch.int64, device=device)
    return s64(0x9E3779B97F4A7C15), s64(0xBF58476D1CE4E5B9), s64(0x94D049BB133111EB)


def _t_srl(x, k):
    """Logical right shift of int64 tensors holding uint64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _t_splitmix64(torch, x):
    g, m1, m2 = _t_consts(torch, x.device)
    z = x + g
    z = (z ^ _t_srl(z, 30)) * m1
    z = (z ^ _t_srl(z, 27)) * m2
    return z ^ _t_srl(z, 31)


def _t_hash(torch, seed, stream, codes):
    key = int(_stream_key(seed, stream))
    key = key - (1 << 64) if key >= (1 << 63) else key
    return _t_splitmix64(torch, codes ^ key)


def t_uniform(torch, seed, stream, codes):
    h = _t_hash(torch, seed, stream, codes)
    return _t_srl(h, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def t_normal_pair(torch, seed, stream, codes):
    h = _t_hash(torch, seed, stream, codes)
    u1 = (_t_srl(h, 32).to(torch.float64) + 0.5) * (1.0 / 4294967296.0)
    u2 = (h & 0xFFFFFFFF).to(torch.float64) * (1.0 / 4294967296.0)
    r = torch.sqrt(-2.0 * torch.log(u1))
    a = 2.0 * math.pi * u2
    return r * torch.cos(a), r * torch.sin(a)


def _t_morton(torch, x, y, z, depth):
    m = torch.zeros_like(x)
    for b in range(depth):
        m |= ((x >> b) & 1) << (3 * b + 2)
        m |= ((y >> b) & 1) << (3 * b + 1)
        m |= ((z >> b) & 1) << (3 * b)
    return m


def scene_shapes_torch(seed: int = 1001, depth: int = 9, sh_degree: int = 3, occupancy: float = 0.03,
                       device="cuda", name: str = "main") -> Scene:
    """``scene_shapes`` evaluated on a GPU; morton / sigma / sh are torch tensors
    (morton as int64 bit patterns) on ``device``."""
    import torch
    lo, size = (-1.5, -1.5, -1.5), 3.0
    centers, radius, half = _shapes(seed)
    coarse = min(depth, 7)
    target = occupancy * (1 << (3 * coarse))
    s_lo, s_hi = 0.2, 4.0
    for _ in range(40):
        s_mid = 0.5 * (s_lo + s_hi)
        n = _occupied_codes(coarse, lo, size, centers, radius, half, s_mid).shape[0]
        if n < target:
            s_lo = s_mid
        else:
            s_hi = s_mid
    scale = 0.5 * (s_lo + s_hi)
    R = 1 << depth
    h = size / R
    codes = []
    for i in range(centers.shape[0]):
        c = centers[i]
        ext = (radius[i] if i % 2 == 0 else half[i].max()) * scale
        lo_i = np.clip(np.floor((c - ext - lo[0]) / h - 0.5).astype(int), 0, R - 1)
        hi_i = np.clip(np.ceil((c + ext - lo[0]) / h + 0.5).astype(int), 0, R - 1)
        ax = [torch.arange(int(lo_i[a]), int(hi_i[a]) + 1, device=device, dtype=torch.int64) for a in range(3)]
        for xs in torch.split(ax[0], 64):
            X, Y, Z = torch.meshgrid(xs, ax[1], ax[2], indexing="ij")
            px = lo[0] + (X.to(torch.float64) + 0.5) * h
            py = lo[1] + (Y.to(torch.float64) + 0.5) * h
            pz = lo[2] + (Z.to(torch.float64) + 0.5) * h
            if i % 2 == 0:
                m = (px - c[0]) ** 2 + (py - c[1]) ** 2 + (pz - c[2]) ** 2 < (radius[i] * scale) ** 2
            else:
                hs = half[i] * scale
                m = ((px - c[0]).abs() < hs[0]) & ((py - c[1]).abs() < hs[1]) & ((pz - c[2]).abs() < hs[2])
            codes.append(_t_morton(torch, X[m], Y[m], Z[m], depth))
    codes = torch.unique(torch.cat(codes)) if codes else torch.zeros(0, dtype=torch.int64, device=device)
    z0, _ = t_normal_pair(torch, seed, 30, codes)
    sigma = torch.exp(3.0 + z0).to(torch.float32)
    K = (sh_degree + 1) ** 2
    sh = torch.empty((codes.shape[0], K, 3), dtype=torch.float32, device=device)
    flat = [(k, c) for k in range(K) for c in range(3)]
    for p in range(0, len(flat), 2):
        z0, z1 = t_normal_pair(torch, seed, 1000 + p // 2, codes)
        for zz, idx in ((z0, p), (z1, p + 1)):
            if idx < len(flat):
                k, c = flat[idx]
                sh[:, k, c] = (zz * (0.5 / (int(math.isqrt(k)) + 1))).to(torch.float32)
    return Scene(depth, lo, size, sh_degree, codes, sigma, sh, name=name)


# ----------------------------------------------------------------------------
# Serving workload: Poisson arrivals of render requests on resident trees
# ----------------------------------------------------------------------------

SERVE_TREES = ((7, 1), (8, 2), (9, 3), (10, 3))            # (depth, SH degree), fp16 leaves
SERVE_RESOLUTIONS = ((256, 256), (512, 512), (800, 800), (1920, 1080))


def serve_requests(seed: int, n: int, rate_hz: float = 300.0, n_trees: int = 4):
    """n requests: arrival times (s) of a Poisson process of ``rate_hz``, a tree
    index, and one camera each (random orbit position at radius 4, elevation
    10..50 degrees, looking at the origin; focal 1111 px scaled with width)."""
    ids = np.arange(n, dtype=np.uint64)
    gaps = -np.log(1.0 - uniform(seed, 70, ids)) / rate_hz
    arrival = np.cumsum(gaps) - gaps[0]
    tree = (uniform(seed, 71, ids) * n_trees).astype(np.int64)
    res = (uniform(seed, 72, ids) * len(SERVE_RESOLUTIONS)).astype(np.int64)
    az = uniform(seed, 73, ids) * 2.0 * math.pi
    el = np.radians(10.0 + 40.0 * uniform(seed, 74, ids))
    cams = []
    for i in range(n):
        W, H = SERVE_RESOLUTIONS[res[i]]
        eye = (4.0 * math.cos(el[i]) * math.cos(az[i]), 4.0 * math.cos(el[i]) * math.sin(az[i]),
               4.0 * math.sin(el[i]))
        cams.append(make_cameras([look_at(eye)], W, H, 1111.0 * W / 800.0, near=2.0, far=6.0)[0])
    return arrival, tree, cams
