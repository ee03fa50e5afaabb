// pot_build.cu -- tree construction on the device (Sec. 3.2 "Filtering": the
// kept voxels become leaves at the deepest level, the tree is empty elsewhere).
//
// Input: the kept voxels' Morton codes in ascending order (given, or compacted
// from a dense grid).  For each level l = D-1 .. 0 the parents' codes are the
// children's codes >> 3; a scan of "first child of its parent" flags ranks the
// distinct parents, which are the level's nodes in ascending Morton prefix.
// Breadth-first offsets of the levels then give every node's index, and one
// pass per level writes child[node][slot].
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <vector>

#include "pot_device.cuh"
#include "pot_internal.h"

namespace pot {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Inclusive scan of one value per thread across the block; returns the
// thread's inclusive prefix and writes the block total to *total.
__device__ int block_scan_incl(int v, int *total)
{
    __shared__ int warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v += warp_tot[wid - 1];
    *total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return v;
}

__global__ void scan_tile_totals(const int *in, int64_t n, int *totals)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    int tot;
    block_scan_incl(s, &tot);
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

// prefix: inclusive scan of the tile totals (NULL for a single tile)
__global__ void scan_tiles(const int *in, int *out, int64_t n, const int *prefix)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
        v[k] = s;
    }
    int tot;
    int incl = block_scan_incl(s, &tot);
    int off = incl - s + ((prefix && blockIdx.x > 0) ? prefix[blockIdx.x - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) out[base + k] = v[k] + off;
}

cudaError_t scan_inclusive_impl(const int *in, int *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        count_launch();
        return cudaGetLastError();
    }
    int *tot = nullptr;
    cudaError_t e = cudaMallocAsync(&tot, sizeof(int) * 2 * tiles, s);
    if (e != cudaSuccess) return e;
    scan_tile_totals<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, tot);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_inclusive_impl(tot, tot + tiles, tiles, s);
    if (e == cudaSuccess) {
        scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, tot + tiles);
        count_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(tot, s);
    return e;
}

unsigned grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > (1 << 20)) b = 1 << 20;  // grid-stride loops cover the rest
    return (unsigned)(b < 1 ? 1 : b);
}

// ---- sparse input validation ---------------------------------------------
__global__ void k_validate(int depth, int64_t n, const uint64_t *codes, const float *sigma,
                           unsigned *flags)
{
    const uint64_t lim = 1ull << (3 * depth);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = codes[i];
        if (c >= lim || (i > 0 && c <= codes[i - 1])) atomicOr(flags, 1u);
        if (!isfinite(sigma[i])) atomicOr(flags, 2u);
    }
}

// ---- levels ---------------------------------------------------------------
__global__ void k_heads(int64_t m, const uint64_t *c, int *head)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || (c[i] >> 3) != (c[i - 1] >> 3)) ? 1 : 0;
}

// rank := inclusive count - 1; the first child of each parent writes the parent's code
__global__ void k_parents(int64_t m, const uint64_t *c, int *rank, uint64_t *parent_codes)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = rank[i] - 1;
        rank[i] = r;
        if (i == 0 || (c[i] >> 3) != (c[i - 1] >> 3)) parent_codes[r] = c[i] >> 3;
    }
}

// child[(off_parent + rank[i]) * 8 + (c[i] & 7)] = leaf or node index of entry i
__global__ void k_children(int64_t m, const uint64_t *c, const int *rank, int32_t *child,
                           int64_t off_parent, int64_t off_self, int leaves)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = leaves ? (int32_t)(-(i + 1)) : (int32_t)(off_self + i);
        child[(off_parent + rank[i]) * 8 + (int64_t)(c[i] & 7u)] = v;
    }
}

// ---- leaf packing ---------------------------------------------------------
template <typename T>
__device__ __forceinline__ T to_store(float x, unsigned *flags);

template <>
__device__ __forceinline__ float to_store<float>(float x, unsigned *)
{
    return x;
}

template <>
__device__ __forceinline__ __half to_store<__half>(float x, unsigned *flags)
{
    __half h = __float2half_rn(x);
    if (__hisinf(h) && isfinite(x)) {
        atomicOr(flags, 4u);
        h = __float2half_rn(x > 0.f ? 65504.f : -65504.f);
    }
    return h;
}

template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float x, unsigned *flags)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    if (__hisinf(b) && isfinite(x)) {
        atomicOr(flags, 4u);
        b = __ushort_as_bfloat16(x > 0.f ? (unsigned short)0x7F7F : (unsigned short)0xFF7F);
    }
    return b;
}

template <typename T>
__device__ __forceinline__ float from_store(T x);
template <>
__device__ __forceinline__ float from_store<float>(float x)
{
    return x;
}
template <>
__device__ __forceinline__ float from_store<__half>(__half x)
{
    return __half2float(x);
}
template <>
__device__ __forceinline__ float from_store<__nv_bfloat16>(__nv_bfloat16 x)
{
    return __bfloat162float(x);
}

template <typename T>
__global__ void k_pack(int64_t n, int K, int stride, const float *sigma, const float *sh, T *sig_out,
                       T *sh_out, unsigned *flags)
{
    const int row = 3 * K;
    const int64_t total = n * (int64_t)stride;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = j / stride;
        const int e = (int)(j - i * stride);
        sh_out[j] = e < row ? to_store<T>(sh[i * row + e], flags) : to_store<T>(0.f, flags);
        if (e == 0) sig_out[i] = to_store<T>(sigma[i], flags);
    }
}

template <typename T>
__global__ void k_unpack(int64_t n, int K, int stride, const T *sig_in, const T *sh_in, float *sigma,
                         float *sh)
{
    const int row = 3 * K;
    const int64_t total = n * (int64_t)row;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = j / row;
        const int e = (int)(j - i * row);
        if (sh) sh[j] = from_store<T>(sh_in[i * stride + e]);
        if (sigma && e == 0) sigma[i] = from_store<T>(sig_in[i]);
    }
}

// codebook leaves -> canonical float32 arrays
__global__ void k_unpack_cb16(int64_t n, int K, int stride, const float *sig_in, const uint16_t *codes,
                              const __half *book, float *sigma, float *sh)
{
    const int64_t total = n * (int64_t)K;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = j / K;
        const int k = (int)(j - i * K);
        const uint16_t code = codes[i * stride + k];
        const __half *e = book + ((int64_t)k * kCodebookEntries + code) * 4;
        if (sh)
            for (int c = 0; c < 3; ++c) sh[(i * K + k) * 3 + c] = __half2float(e[c]);
        if (sigma && k == 0) sigma[i] = sig_in[i];
    }
}

// ---- dense compaction -----------------------------------------------------
__device__ __forceinline__ void morton_decode3(uint64_t m, int depth, int64_t &x, int64_t &y, int64_t &z)
{
    x = y = z = 0;
    for (int b = 0; b < depth; ++b) {
        x |= (int64_t)((m >> (3 * b + 2)) & 1u) << b;
        y |= (int64_t)((m >> (3 * b + 1)) & 1u) << b;
        z |= (int64_t)((m >> (3 * b)) & 1u) << b;
    }
}

__global__ void k_dense_flags(int depth, float tau, const float *sigma, int *flag, unsigned *flags)
{
    const int64_t R = 1ll << depth;
    const int64_t total = R * R * R;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < total;
         m += (int64_t)gridDim.x * blockDim.x) {
        int64_t x, y, z;
        morton_decode3((uint64_t)m, depth, x, y, z);
        const float s = sigma[(x * R + y) * R + z];
        if (!isfinite(s)) atomicOr(flags, 2u);
        flag[m] = s > tau ? 1 : 0;
    }
}

__global__ void k_dense_gather(int depth, int K, const float *sigma, const float *sh, const int *incl,
                               uint64_t *codes, float *sig_out, float *sh_out)
{
    const int64_t R = 1ll << depth;
    const int64_t total = R * R * R;
    const int row = 3 * K;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < total;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int prev = m > 0 ? incl[m - 1] : 0;
        if (incl[m] == prev) continue;
        int64_t x, y, z;
        morton_decode3((uint64_t)m, depth, x, y, z);
        const int64_t v = (x * R + y) * R + z;
        codes[prev] = (uint64_t)m;
        sig_out[prev] = sigma[v];
        for (int e = 0; e < row; ++e) sh_out[(int64_t)prev * row + e] = sh[v * row + e];
    }
}

// Cell index entry of every voxel: a root descent of the child array (the
// query's rule), written in the index's brick order so that stores coalesce.
__global__ void k_cell_index(int D, const int32_t *child, int32_t *cells)
{
    const int nb = D > 2 ? D - 2 : 0;
    const uint32_t R = 1u << D, bmask = (1u << nb) - 1u;
    const int64_t n = cell_index_entries(D);
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t in = (uint32_t)o & 63u, brick = (uint32_t)(o >> 6);
        const uint32_t x = ((brick >> (2 * nb)) << 2) | (in >> 4);
        const uint32_t y = (((brick >> nb) & bmask) << 2) | ((in >> 2) & 3u);
        const uint32_t z = ((brick & bmask) << 2) | (in & 3u);
        int32_t v = -1;  // entries of voxels outside a grid smaller than one brick are never read
        if (x < R && y < R && z < R) {
            int32_t node = 0;
            for (int l = 0; l < D; ++l) {
                const int b = D - 1 - l;
                const int slot = (int)((((x >> b) & 1u) << 2) | (((y >> b) & 1u) << 1) | ((z >> b) & 1u));
                const int32_t c = child[(int64_t)node * 8 + slot];
                if (c > 0 && l < D - 1) {
                    node = c;
                    continue;
                }
                // an empty slot of a level-l node is an empty level-(l+1) node
                v = c < 0 ? -c - 1 : cell_code_node(l + 1, D);
                break;
            }
        }
        cells[o] = v;
    }
}

// Chebyshev distance transform of the occupied voxels, capped at
// kCellCubeMax + 1, in three passes along x, y, z of an x-major uint8 grid
// f (0 = occupied): f'(v) = min over |k| <= kCellCubeMax of max(|k|, f(v + k e_axis)).
// The L-infinity distance separates into these 1-D passes; values beyond the
// cap stay at the cap, a lower bound, which is all the renderer needs.
constexpr int kDistCap = kCellCubeMax + 1;

__global__ void k_dist_init(int D, const int32_t *cells, uint8_t *f)
{
    const int64_t n = 1ll << (3 * D);
    const uint32_t m = (1u << D) - 1u;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(v >> (2 * D)), y = (uint32_t)(v >> D) & m, z = (uint32_t)v & m;
        f[v] = cells[cell_index_offset(x, y, z, D)] >= 0 ? 0 : (uint8_t)kDistCap;
    }
}

__global__ void k_dist_pass(int D, int axis, const uint8_t *in, uint8_t *out)
{
    const int64_t n = 1ll << (3 * D);
    const int R = 1 << D;
    const int shift = D * (2 - axis);  // x: 2D, y: D, z: 0
    const int64_t stride = 1ll << shift;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)((v >> shift) & (R - 1));
        int best = in[v];
        for (int k = 1; k < best && k <= kCellCubeMax; ++k) {
            if (c - k >= 0) best = min(best, max(k, (int)in[v - k * stride]));
            if (c + k < R) best = min(best, max(k, (int)in[v + k * stride]));
        }
        out[v] = (uint8_t)best;
    }
}

// Empty entries become cubes where the cube's half-extent e = distance - 1
// is at least half the empty node's size (2e + 2 > 2^(D-l)).
__global__ void k_dist_apply(int D, const uint8_t *f, int32_t *cells)
{
    const int64_t n = 1ll << (3 * D);
    const uint32_t m = (1u << D) - 1u;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(v >> (2 * D)), y = (uint32_t)(v >> D) & m, z = (uint32_t)v & m;
        int32_t &c = cells[cell_index_offset(x, y, z, D)];
        if (c >= 0) continue;
        const int level = cell_code_node_level(c, D);
        const int e = (int)f[v] - 1;
        if (2 * e + 2 > (1 << (D - level))) c = cell_code_cube(e);
    }
}

// Index entries in x-major voxel order (export), from either layout.
__global__ void k_cell_index_export(int D, const int32_t *cells, const int32_t *btab, int32_t *out)
{
    const int64_t n = 1ll << (3 * D);
    const uint32_t m = (1u << D) - 1u;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(v >> (2 * D)), y = (uint32_t)(v >> D) & m, z = (uint32_t)v & m;
        if (btab) {
            const int32_t b = btab[brick_of(x, y, z, D)];
            out[v] = cell_code_public(b >= 0 ? cells[((int64_t)b << 6) | in_brick(x, y, z)] : b, D);
        } else {
            out[v] = cell_code_public(cells[cell_index_offset(x, y, z, D)], D);
        }
    }
}

// ---- brick layout -----------------------------------------------------------
// Per 4^3 brick (x-major over the (2^(D-2))^3 brick grid): the descent of the
// child array along the brick's path.  A brick holding a leaf is an existing
// node of level D - 2: its node index (> 0) is recorded and its distance seed
// is 0; otherwise the empty node of level l around it, cell_code_node(l), and
// the seed is the cap.
__global__ void k_brick_classify(int D, const int32_t *child, int32_t *node_or_code, uint8_t *dist)
{
    const int nb = D - 2;
    const int64_t n = brick_count(D);
    const uint32_t m = (1u << nb) - 1u;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t bx = (uint32_t)(b >> (2 * nb)), by = (uint32_t)(b >> nb) & m, bz = (uint32_t)b & m;
        int32_t node = 0, code = 0;
        for (int l = 0; l < nb; ++l) {
            const int bit = nb - 1 - l;
            const int slot = (int)((((bx >> bit) & 1u) << 2) | (((by >> bit) & 1u) << 1) | ((bz >> bit) & 1u));
            const int32_t c = child[(int64_t)node * 8 + slot];
            if (c > 0) {
                node = c;
                continue;
            }
            code = cell_code_node(l + 1, D);  // an empty slot of a level-l node
            break;
        }
        node_or_code[b] = code ? code : node;
        dist[b] = code ? (uint8_t)kDistCap : 0;
    }
}

__global__ void k_brick_flags(int64_t n, const int32_t *node_or_code, int *flags)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x)
        flags[b] = node_or_code[b] > 0 ? 1 : 0;
}

// Brick codes and the entries of bricks holding a leaf.  A brick at
// Chebyshev distance db (in bricks, capped) from the nearest brick with a leaf
// has no leaf within 4 (db - 1) voxels of any of its voxels, so the cube of
// that half-extent centred on any of them is empty; it replaces the empty node
// where it is larger (the dense layout's rule).  Inside a brick with a leaf,
// each voxel is a leaf or lies in an empty node of level D - 1 or D.
__global__ void k_brick_fill(int D, const int32_t *child, const int32_t *node_or_code, const int *ids,
                             const uint8_t *dist, int32_t *btab, int32_t *bricks)
{
    const int64_t n = brick_count(D);
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = node_or_code[b];
        if (v > 0) {
            const int32_t id = ids[b] - 1;
            btab[b] = id;
            int32_t *out = bricks + ((int64_t)id << 6);
            for (int in = 0; in < 64; ++in) {
                const int x = in >> 4, y = (in >> 2) & 3, z = in & 3;
                const int s1 = ((x >> 1) << 2) | ((y >> 1) << 1) | (z >> 1);
                const int32_t c = child[(int64_t)v * 8 + s1];
                int32_t e;
                if (c > 0) {
                    const int32_t c2 = child[(int64_t)c * 8 + (((x & 1) << 2) | ((y & 1) << 1) | (z & 1))];
                    e = c2 < 0 ? -c2 - 1 : cell_code_node(D, D);
                } else {
                    e = cell_code_node(D - 1, D);
                }
                out[in] = e;
            }
        } else {
            const int level = cell_code_node_level(v, D);
            const int eb = min(4 * ((int)dist[b] - 1), kCellCubeMax);
            btab[b] = (2 * eb + 2 > (1 << (D - level))) ? cell_code_cube(eb) : v;
        }
    }
}

}  // namespace

cudaError_t export_cell_index(const pot_tree *t, int32_t *out, cudaStream_t s)
{
    const int D = t->desc.depth;
    const int64_t n = 1ll << (3 * D);
    const int64_t want = (n + 255) / 256;
    k_cell_index_export<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, s>>>(D, t->cells, t->btab, out);
    count_launch();
    return cudaGetLastError();
}

void free_cell_index(pot_tree *t)
{
    if (t->cells) cudaFree(t->cells);
    if (t->btab) cudaFree(t->btab);
    t->cells = nullptr;
    t->btab = nullptr;
    t->n_bricks = 0;
    t->cell_kind = POT_CELLS_NONE;
    t->index_bytes = 0;
}

namespace {

cudaError_t build_brick_index(pot_tree *t, cudaStream_t s)
{
    const int D = t->desc.depth;
    if (D < kBrickIndexMinDepth || D > kBrickIndexMaxDepth) return cudaErrorNotSupported;
    const int64_t n = brick_count(D);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t want = (n + 255) / 256, cap = (int64_t)sms * 16;
    const unsigned g = (unsigned)(want < cap ? want : cap);
    int32_t *node_or_code = nullptr, *btab = nullptr, *bricks = nullptr;
    int *flags = nullptr, *ids = nullptr;
    uint8_t *d0 = nullptr, *d1 = nullptr;
    e = cudaMallocAsync(&node_or_code, sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&flags, sizeof(int) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&ids, sizeof(int) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d0, (size_t)n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d1, (size_t)n, s);
    int last_id = 0;
    if (e == cudaSuccess) {
        k_brick_classify<<<g, 256, 0, s>>>(D, t->child, node_or_code, d0);
        // Chebyshev distance in bricks to the nearest brick holding a leaf (capped)
        k_dist_pass<<<g, 256, 0, s>>>(D - 2, 0, d0, d1);
        k_dist_pass<<<g, 256, 0, s>>>(D - 2, 1, d1, d0);
        k_dist_pass<<<g, 256, 0, s>>>(D - 2, 2, d0, d1);
        k_brick_flags<<<g, 256, 0, s>>>(n, node_or_code, flags);
        count_launch(5);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_inclusive_impl(flags, ids, n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_id, ids + (n - 1), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const int64_t nb = last_id;
    if (e == cudaSuccess) e = cudaMalloc(&btab, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bricks, sizeof(int32_t) * 64 * (nb > 0 ? nb : 1));
    if (e == cudaSuccess) {
        k_brick_fill<<<g, 256, 0, s>>>(D, t->child, node_or_code, ids, d1, btab, bricks);
        count_launch();
        e = cudaGetLastError();
    }
    if (node_or_code) cudaFreeAsync(node_or_code, s);
    if (flags) cudaFreeAsync(flags, s);
    if (ids) cudaFreeAsync(ids, s);
    if (d0) cudaFreeAsync(d0, s);
    if (d1) cudaFreeAsync(d1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        if (btab) cudaFree(btab);
        if (bricks) cudaFree(bricks);
        return e;
    }
    t->btab = btab;
    t->cells = bricks;
    t->n_bricks = nb;
    t->cell_kind = POT_CELLS_BRICK;
    t->index_bytes = (int64_t)sizeof(int32_t) * (n + 64 * nb);
    return cudaSuccess;
}

}  // namespace

cudaError_t build_cell_index(pot_tree *t, int kind, cudaStream_t s)
{
    if (kind == POT_CELLS_BRICK) return build_brick_index(t, s);
    const int D = t->desc.depth;
    if (D > kCellIndexMaxDepth) return cudaErrorNotSupported;
    const int64_t n = cell_index_entries(D);
    int32_t *cells = nullptr;
    cudaError_t e = cudaMalloc(&cells, sizeof(int32_t) * n);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const int64_t want = (n + 255) / 256, cap = (int64_t)sms * 16;
        k_cell_index<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(D, t->child, cells);
        count_launch();
        e = cudaGetLastError();
    }
    // empty cubes from the distance transform (two R^3 byte grids, freed here)
    const int64_t nv = 1ll << (3 * D);
    uint8_t *f0 = nullptr, *f1 = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&f0, (size_t)nv, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&f1, (size_t)nv, s);
    if (e == cudaSuccess) {
        const int64_t want = (nv + 255) / 256, cap = (int64_t)sms * 16;
        const unsigned g = (unsigned)(want < cap ? want : cap);
        k_dist_init<<<g, 256, 0, s>>>(D, cells, f0);
        k_dist_pass<<<g, 256, 0, s>>>(D, 0, f0, f1);
        k_dist_pass<<<g, 256, 0, s>>>(D, 1, f1, f0);
        k_dist_pass<<<g, 256, 0, s>>>(D, 2, f0, f1);
        k_dist_apply<<<g, 256, 0, s>>>(D, f1, cells);
        count_launch(5);
        e = cudaGetLastError();
    }
    if (f0) cudaFreeAsync(f0, s);
    if (f1) cudaFreeAsync(f1, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        cudaFree(cells);
        return e;
    }
    t->cells = cells;
    t->btab = nullptr;
    t->n_bricks = 0;
    t->cell_kind = POT_CELLS_DENSE;
    t->index_bytes = (int64_t)sizeof(int32_t) * n;
    return cudaSuccess;
}

cudaError_t scan_inclusive(const int *in, int *out, int64_t n, cudaStream_t s);

cudaError_t scan_inclusive(const int *in, int *out, int64_t n, cudaStream_t s)
{
    return scan_inclusive_impl(in, out, n, s);
}

cudaError_t validate_sparse(int depth, int64_t n, const uint64_t *d_codes, const float *d_sigma,
                            unsigned int *d_flags, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_validate<<<grid_for(n, 256), 256, 0, s>>>(depth, n, d_codes, d_sigma, d_flags);
    count_launch();
    return cudaGetLastError();
}

cudaError_t build_levels_and_children(pot_tree *t, int64_t n, const uint64_t *d_codes, cudaStream_t s,
                                      unsigned int *, int *status)
{
    const int D = t->desc.depth;
    *status = 0;
    cudaError_t e = cudaSuccess;
    if (n == 0) {
        t->n_nodes = 1;
        e = cudaMalloc(&t->child, sizeof(int32_t) * 8);
        if (e == cudaSuccess) e = cudaMemsetAsync(t->child, 0, sizeof(int32_t) * 8, s);
        return e;
    }
    // per level l (0..D): codes and, for l >= 1, the rank of each entry's parent
    std::vector<uint64_t *> codes(D + 1, nullptr);
    std::vector<int *> rank(D + 1, nullptr);
    std::vector<int64_t> cnt(D + 1, 0);
    codes[D] = const_cast<uint64_t *>(d_codes);
    cnt[D] = n;
    for (int l = D - 1; l >= 0 && e == cudaSuccess; --l) {
        const int64_t m = cnt[l + 1];
        e = cudaMallocAsync(&rank[l + 1], sizeof(int) * m, s);
        if (e != cudaSuccess) break;
        k_heads<<<grid_for(m, 256), 256, 0, s>>>(m, codes[l + 1], rank[l + 1]);
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = scan_inclusive(rank[l + 1], rank[l + 1], m, s);
        int np = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&np, rank[l + 1] + (m - 1), sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        cnt[l] = np;
        e = cudaMallocAsync(&codes[l], sizeof(uint64_t) * (np > 0 ? np : 1), s);
        if (e != cudaSuccess) break;
        k_parents<<<grid_for(m, 256), 256, 0, s>>>(m, codes[l + 1], rank[l + 1], codes[l]);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && cnt[0] != 1) *status = 1;  // cannot happen for valid codes
    std::vector<int64_t> off(D + 1, 0);
    for (int l = 1; l <= D; ++l) off[l] = off[l - 1] + cnt[l - 1];
    const int64_t N = off[D];
    if (e == cudaSuccess && N >= (int64_t)0x7FFFFFFF) *status = 2;
    if (e == cudaSuccess && *status == 0) {
        t->n_nodes = N;
        e = cudaMalloc(&t->child, sizeof(int32_t) * 8 * N);
        if (e == cudaSuccess) e = cudaMemsetAsync(t->child, 0, sizeof(int32_t) * 8 * N, s);
        for (int l = 0; l < D && e == cudaSuccess; ++l) {
            const int64_t m = cnt[l + 1];
            k_children<<<grid_for(m, 256), 256, 0, s>>>(m, codes[l + 1], rank[l + 1], t->child, off[l],
                                                        off[l + 1], l + 1 == D);
            count_launch();
            e = cudaGetLastError();
        }
    }
    for (int l = 0; l <= D; ++l) {
        if (l < D && codes[l]) cudaFreeAsync(codes[l], s);
        if (rank[l]) cudaFreeAsync(rank[l], s);
    }
    return e;
}

cudaError_t pack_leaves(pot_tree *t, const float *d_sigma, const float *d_sh, unsigned int *d_flags,
                        cudaStream_t s)
{
    const int64_t n = t->n_leaves;
    const int64_t sig_bytes = ((n * t->elem_bytes + 255) / 256) * 256;
    const int64_t sh_bytes = n * t->stride * t->elem_bytes;
    cudaError_t e = cudaSuccess;
    if (!t->sigma) e = cudaMalloc(&t->sigma, sig_bytes > 0 ? sig_bytes : 256);
    if (e == cudaSuccess && !t->sh) e = cudaMalloc(&t->sh, sh_bytes > 0 ? sh_bytes : 256);
    if (e != cudaSuccess || n == 0) return e;
    const unsigned g = grid_for(n * t->stride, 256);
    switch (t->desc.leaf_dtype) {
    case POT_F32:
        k_pack<float><<<g, 256, 0, s>>>(n, t->K, t->stride, d_sigma, d_sh, (float *)t->sigma,
                                         (float *)t->sh, d_flags);
        break;
    case POT_F16:
        k_pack<__half><<<g, 256, 0, s>>>(n, t->K, t->stride, d_sigma, d_sh, (__half *)t->sigma,
                                          (__half *)t->sh, d_flags);
        break;
    default:
        k_pack<__nv_bfloat16><<<g, 256, 0, s>>>(n, t->K, t->stride, d_sigma, d_sh,
                                                 (__nv_bfloat16 *)t->sigma, (__nv_bfloat16 *)t->sh,
                                                 d_flags);
        break;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t export_leaves(const pot_tree *t, float *d_sigma, float *d_sh, cudaStream_t s)
{
    const int64_t n = t->n_leaves;
    if (n == 0 || (!d_sigma && !d_sh)) return cudaSuccess;
    const unsigned g = grid_for(n * 3 * t->K, 256);
    if (t->desc.leaf_dtype == POT_CB16) {
        k_unpack_cb16<<<g, 256, 0, s>>>(n, t->K, t->stride, (const float *)t->sigma, (const uint16_t *)t->sh,
                                        (const __half *)t->codebook, d_sigma, d_sh);
        count_launch();
        return cudaGetLastError();
    }
    switch (t->desc.leaf_dtype) {
    case POT_F32:
        k_unpack<float><<<g, 256, 0, s>>>(n, t->K, t->stride, (const float *)t->sigma,
                                           (const float *)t->sh, d_sigma, d_sh);
        break;
    case POT_F16:
        k_unpack<__half><<<g, 256, 0, s>>>(n, t->K, t->stride, (const __half *)t->sigma,
                                            (const __half *)t->sh, d_sigma, d_sh);
        break;
    default:
        k_unpack<__nv_bfloat16><<<g, 256, 0, s>>>(n, t->K, t->stride, (const __nv_bfloat16 *)t->sigma,
                                                   (const __nv_bfloat16 *)t->sh, d_sigma, d_sh);
        break;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t compact_dense(int depth, float tau, const float *d_sigma, const float *d_sh, int K,
                          uint64_t **d_codes, float **d_sig_out, float **d_sh_out, int64_t *n_out,
                          unsigned int *d_flags, cudaStream_t s)
{
    const int64_t total = 1ll << (3 * depth);
    int *incl = nullptr;
    cudaError_t e = cudaMallocAsync(&incl, sizeof(int) * total, s);
    if (e != cudaSuccess) return e;
    k_dense_flags<<<grid_for(total, 256), 256, 0, s>>>(depth, tau, d_sigma, incl, d_flags);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_inclusive(incl, incl, total, s);
    int n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, incl + (total - 1), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        *n_out = n;
        e = cudaMallocAsync(d_codes, sizeof(uint64_t) * (n > 0 ? n : 1), s);
        if (e == cudaSuccess) e = cudaMallocAsync(d_sig_out, sizeof(float) * (n > 0 ? n : 1), s);
        if (e == cudaSuccess) e = cudaMallocAsync(d_sh_out, sizeof(float) * 3 * K * (int64_t)(n > 0 ? n : 1), s);
    }
    if (e == cudaSuccess && n > 0) {
        k_dense_gather<<<grid_for(total, 256), 256, 0, s>>>(depth, K, d_sigma, d_sh, incl, *d_codes,
                                                            *d_sig_out, *d_sh_out);
        count_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(incl, s);
    return e;
}

}  // namespace pot
