// pot_render.cuh -- forward render kernel of the PlenOctree path (sm_103a).
//
// One warp renders one tile of 32 rays at a time (4 x 8 pixels of a camera,
// or 32 consecutive explicit rays); warps take tiles from a global counter
// until none is left (persistent grid, one wave of resident blocks).  Per ray:
//   a1 pinhole ray (fp32 expression of the public header)
//   a2 clip to the tree box and to [near, far]
//   a3 locate the cell: one load from the tree's cell index (leaf, or the
//      empty box around the voxel; two loads in the brick layout), or, for
//      trees without one, a descent of the child array from the deepest
//      ancestor the new voxel shares with the previous one (ancestor stack in
//      shared memory)
//   a4 exit time of the cell (double-float plane crossings, the earliest of
//      three chosen with selects); an empty node of any size is crossed in one
//      step (Sec. 3.2 "Rendering")
//   a5 leaf fetch: sigma and the SH record in 32-byte (or 16-byte) vector loads
//   a6 colour: sigmoid of the SH dot product, basis evaluated once per ray
//      because it is constant along the ray (App. B.3.2)
//   a7 composite: w = T (1 - exp(-max(sigma,0) delta)), C += w c (Eq. 1)
//   a8 stop once T < gamma (Sec. 3.2), add T * bg (App. B.3.2), store.
#pragma once

#include "pot_device.cuh"
#include "pot_internal.h"

namespace pot {

constexpr int kBlock = 256;
#ifndef POT_RENDER_MIN_BLOCKS
#define POT_RENDER_MIN_BLOCKS 4  // resident blocks per SM the register budget is cut for (64 registers)
#endif
#ifndef POT_PREFETCH
// prefetch the next cell's leaf into L1 before shading the current one (helped
// while leaves streamed from DRAM; with neighbouring views sharing L2 it costs
// 1-2 %, so it is off)
#define POT_PREFETCH 0
#endif


// One ray's walk through the octree (a2-a4) as resumable state: begin() sets
// the ray up (clip, locate, first descent), step() advances one cell and calls
// vis(leaf, delta, Y) for a leaf segment of positive length (Y: the SH basis at
// the ray direction), returning false once the walk is over (vis returned
// true, far clip, or the ray left the box).  The next cell is located and its
// leaf prefetched before vis runs on the current one.
template <int K, typename T>
struct Walker {
    float d[3];
    // per-ray constants in shared memory, one float4 per axis (A = lo - o as hi
    // + lo parts, 1/d, the locate margin), 12 registers fewer across the walk;
    // a thread's three float4 are 12 words apart from the next thread's, so the
    // 16-byte loads of 8 consecutive threads hit distinct banks
    float4 *st;
    __device__ __forceinline__ float Ahi(int a) const { return st[a].x; }
    __device__ __forceinline__ float Alo(int a) const { return st[a].y; }
    __device__ __forceinline__ float rd(int a) const { return st[a].z; }
    __device__ __forceinline__ float margin(int a) const { return st[a].w; }
    float len;
    // the per-ray SH basis lives in shared memory (this thread's part of the
    // block's array), not in 16 registers: that lets 4 blocks (32 warps) reside per SM
    float *ysm;
    __device__ __forceinline__ SmemY<K, kBlock> Y() const { return {ysm}; }
    df t, tout;
    int q[3];
    // cell: the box the ray is in, cshape >= 0: the cube of half-extent cshape
    // centred on voxel q (a leaf is the cube of extent 0); cshape < 0: the
    // aligned octree node of 2^(-cshape - 1) voxels per axis around q
    int leaf, cshape, lvl_valid, step_i;

    // a3: the cell of voxel nq: one load from the cell index when the tree
    // has one, else a descent from the deepest ancestor nq shares with voxel
    // pq (whose path the stack holds up to lvl_valid)
    __device__ __forceinline__ void descend(const RenderParams &p, int32_t *stk, const int nq[3], const int pq[3],
                                            int &out_leaf, int &out_shape)
    {
        const int D = p.depth;
        if (p.cells) {
            const uint32_t bk = brick_of((uint32_t)nq[0], (uint32_t)nq[1], (uint32_t)nq[2], D);
            const uint32_t in = in_brick((uint32_t)nq[0], (uint32_t)nq[1], (uint32_t)nq[2]);
            int v;
            if (p.btab) {  // brick layout: the brick's code, or its stored entries
                const int b = __ldg(p.btab + bk);
                v = b >= 0 ? __ldg(p.cells + (((int64_t)b << 6) | in)) : b;
            } else {
                v = __ldg(p.cells + ((bk << 6) | in));
            }
            out_leaf = v >= 0 ? v : -1;
            out_shape = v >= 0 ? 0 : v + kShapeBias;  // stored as the cell shape - 64
            return;
        }
        const unsigned diff = (unsigned)((nq[0] ^ pq[0]) | (nq[1] ^ pq[1]) | (nq[2] ^ pq[2]));
        const int lc = diff ? D - 32 + __clz(diff) : D - 1;  // level of the common ancestor
        int l = min(lc, lvl_valid);
        int node = stk[l * kBlock];
        out_leaf = -1;
        out_shape = 0;
        for (; l < D; ++l) {
            const int b = D - 1 - l;
            const int s = (((nq[0] >> b) & 1) << 2) | (((nq[1] >> b) & 1) << 1) | ((nq[2] >> b) & 1);
            const int c = __ldg(p.child + (int64_t)node * 8 + s);
            if (c > 0 && l < D - 1) {
                node = c;
                stk[(l + 1) * kBlock] = c;
                continue;
            }
            if (c < 0) out_leaf = -c - 1;
            else out_shape = -(D - l);  // empty node of level l + 1: 2^(D-l-1) voxels per axis
            break;
        }
        lvl_valid = min(l, D - 1);
    }

    __device__ __forceinline__ bool begin(const RenderParams &p, int32_t *stk, const T *sig_arr, const T *sh_arr,
                                          const float o[3], const float dir[3], float near, float far)
    {
        const int R = p.R;
        const float h = p.h, invh = p.invh;
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = dir[a];
        len = sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
        if (!(len > 0.f) || !(len < 3.0e38f)) return false;
        const float invlen = __frcp_rn(len);
        {
            float Yt[K];
            sh_basis<K>(d[0] * invlen, d[1] * invlen, d[2] * invlen, Yt);
            SmemY<K, kBlock>::store(ysm, Yt);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float ah, al;
            two_sum(p.lo[a], -o[a], ah, al);
            st[a].x = ah;
            st[a].y = al;
            st[a].z = d[a] != 0.f ? __frcp_rn(d[a]) : 0.f;
        }
        // a2: clip range in units of the ray parameter t (position o + t d)
        df tin = {near * invlen, 0.f};
        tout = {far * invlen, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] == 0.f) {
                float s, e;
                two_sum(o[a], -p.lo[a], s, e);
                const bool inside = (s > 0.f || (s == 0.f && e >= 0.f)) && (s < p.size || (s == p.size && e < 0.f));
                if (!inside) return false;
            } else {
                df t0 = cross_time(0, h, Ahi(a), Alo(a), d[a], rd(a));
                df t1 = cross_time(R, h, Ahi(a), Alo(a), d[a], rd(a));
                if (d[a] < 0.f) {
                    df tmp = t0;
                    t0 = t1;
                    t1 = tmp;
                }
                if (df_lt(tin, t0)) tin = t0;
                if (df_lt(t1, tout)) tout = t1;
            }
        }
        if (!df_lt(tin, tout)) return false;
        // error bound of the fp32 voxel-coordinate estimate, in voxels
#pragma unroll
        for (int a = 0; a < 3; ++a)
            st[a].w = (fabsf(tout.hi * d[a]) + fabsf(Ahi(a))) * invh * 3.8146973e-6f + 1e-6f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int v = locate_axis(tin, d[a], Ahi(a), Alo(a), h, invh, margin(a));
            q[a] = min(max(v, 0), R - 1);
        }
        lvl_valid = 0;
        if (!p.cells) stk[0] = 0;  // the stack exists only for trees without a cell index
        descend(p, stk, q, q, leaf, cshape);
        if (POT_PREFETCH && leaf >= 0) prefetch_leaf<K, T>(sig_arr, sh_arr, leaf);
        t = tin;
        step_i = 0;
        return true;
    }

    template <typename Visitor>
    __device__ __forceinline__ bool step(const RenderParams &p, int32_t *stk, const T *sig_arr, const T *sh_arr,
                                         Visitor &vis)
    {
        const int D = p.depth;
        const int R = p.R;
        const float h = p.h, invh = p.invh;
        // a4: exit of the current cell [qb, qb + sz) per axis
        const int sz = cshape >= 0 ? 2 * cshape + 1 : 1 << (-cshape - 1);
        int qb[3];
        df texit = {__int_as_float(0x7f800000), 0.f};
        int ax = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            qb[a] = cshape >= 0 ? q[a] - cshape : q[a] & ~(sz - 1);
            // the exit plane's crossing, every step and without branches:
            // recomputing it costs fewer issued instructions than branching on
            // whether it moved (lanes of a warp cross different axes); it is
            // finite for d = 0 (1/d is stored as 0) and then never chosen
            const int k = d[a] > 0.f ? qb[a] + sz : qb[a];
            const df c = cross_time(k, h, Ahi(a), Alo(a), d[a], rd(a));
            const bool earlier = d[a] != 0.f && df_lt(c, texit);
            texit.hi = earlier ? c.hi : texit.hi;
            texit.lo = earlier ? c.lo : texit.lo;
            ax = earlier ? a : ax;
        }
        const bool last = !df_lt(texit, tout);
        const df tend = last ? tout : texit;
        const float dt = df_sub(tend, t);

        // next voxel and its cell, fetched ahead of shading the current leaf:
        // the exit axis steps one cell; the other axes are located at t_exit
        // within the current cell's face (a one-voxel cell keeps them) and
        // never move backwards.  A leaf's entry time is the crossing time of
        // its own face plane whichever box the ray crossed before it, so the
        // leaf segments do not depend on how empty space was stepped over.
        // (few branches: each potentially divergent branch costs issue slots)
        const bool capped = !last && step_i >= p.step_cap;
        if (capped) *p.err = 1u;  // device error word: a plain store, no branch around an atomic
        int nq[3] = {q[0], q[1], q[2]};
        int nleaf = -1, nshape = 0;
        bool outside = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int stepped = d[a] > 0.f ? qb[a] + sz : qb[a] - 1;
            nq[a] = a == ax ? stepped : nq[a];
            outside = outside || (a == ax && (stepped < 0 || stepped >= R));
        }
        const bool stop = last || capped || outside;
        if (sz > 1 && !stop) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a != ax && d[a] != 0.f) {
                    // within the cell and the grid (a cube may reach past the grid)
                    int v = locate_axis(texit, d[a], Ahi(a), Alo(a), h, invh, margin(a));
                    v = min(max(v, max(qb[a], 0)), min(qb[a] + sz, R) - 1);
                    nq[a] = d[a] > 0.f ? max(v, q[a]) : min(v, q[a]);
                }
            }
        }
        if (!stop) {
            descend(p, stk, nq, q, nleaf, nshape);
            if (POT_PREFETCH && nleaf >= 0) prefetch_leaf<K, T>(sig_arr, sh_arr, nleaf);
        }
        if (leaf >= 0 && dt > 0.f) {
            if (vis(leaf, dt * len, Y())) return false;
        }
        if (stop) return false;
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] = nq[a];
        leaf = nleaf;
        cshape = nshape;
        if (df_lt(t, texit)) t = texit;
        ++step_i;
        return true;
    }
};

// Per-thread scratch of a walk in shared memory: the SH basis (SmemY, rows
// 0..K-1) and the walker's per-ray constants (rows K..K+11) of one
// [K + 12][kBlock] float array, and the ancestor stack [kMaxDepth][kBlock] in
// dynamic shared memory, which a launch provides (walk_smem_bytes) only when
// some tree of it has no cell index; without it the space goes to L1.
// Declared once per kernel.
#define POT_WALK_SHARED(K)                                          \
    extern __shared__ int32_t walk_stack_sh[];                      \
    __shared__ float4 walk_y_sh[kBlock * SmemY<K, kBlock>::kRow4];   \
    __shared__ float4 walk_st_sh[kBlock * 3];                       \
    int32_t *stk = walk_stack_sh + threadIdx.x;                     \
    float *ysm = reinterpret_cast<float *>(walk_y_sh + threadIdx.x * SmemY<K, kBlock>::kRow4); \
    float4 *wst = walk_st_sh + 3 * threadIdx.x;                     \
    (void)ysm;                                                      \
    (void)wst;

inline size_t walk_smem_bytes(bool need_stack)
{
    return need_stack ? sizeof(int32_t) * kMaxDepth * kBlock : 0;
}

// Grid of a persistent walk kernel: one wave of resident blocks (SMs x blocks
// per SM for this kernel and shared memory), no more blocks than tiles need.
template <typename Fn>
cudaError_t persistent_grid(Fn fn, size_t smem, int64_t n_tiles, int max_blocks, unsigned *grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (n_tiles + (kBlock / 32) - 1) / (kBlock / 32);
    if (blocks > need) blocks = need;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    *grid = (unsigned)blocks;
    return cudaSuccess;
}

// The whole walk of one ray.
template <int K, typename T, typename Visitor>
__device__ __forceinline__ void walk_ray(const RenderParams &p, const T *sig_arr, const T *sh_arr,
                                         int32_t *stk, float *ysm, float4 *wst, const float o[3], const float d[3],
                                         float near, float far, Visitor &vis)
{
    Walker<K, T> w;
    w.ysm = ysm;
    w.st = wst;
    if (!w.begin(p, stk, sig_arr, sh_arr, o, d, near, far)) return;
    while (w.step(p, stk, sig_arr, sh_arr, vis)) {
    }
}

// a5-a8 for one leaf segment: fetch, colour, composite, early stop.
template <int K, typename T, bool COUNT>
struct ShadeVisitor {
    const T *sig_arr;
    const T *sh_arr;
    uint8_t *touched;
    float gamma;
    float col[3];
    float Tr;
    int nseg;
    const void *cb;  // codebook (cb16 leaves only)
    template <typename YT>
    __device__ __forceinline__ bool operator()(int leaf, float delta, const YT &Y)
    {
        const float sig = fmaxf(Store<T>::load_sigma(sig_arr, leaf), 0.f);
        float x[3];
        leaf_colour_dot<K, T>(sh_arr, leaf, Y, x, cb);
        const float e = __expf(-sig * delta);  // transmittance of the segment
        const float w = Tr * (1.f - e);
#pragma unroll
        for (int c = 0; c < 3; ++c) col[c] = fmaf(w, sigmoidf_(x[c]), col[c]);
        Tr *= e;
        if (COUNT) {
            ++nseg;
            touched[leaf] = 1;
        }
        return Tr < gamma;  // a8 early stop (gamma = 0 never stops)
    }
};

// Ray (origin, direction, clip range, output index) of slot `slot` (0..31) of
// tile `tile`: kTileW x kTileH pixels of a camera (tiles interleaved over groups of
// adjacent cameras) or 32 consecutive explicit rays.  False for slots outside
// the image or past the last ray.
template <bool CAMS>
__device__ __forceinline__ bool tile_ray(const RenderParams &p, unsigned long long tile, int slot, float o[3],
                                         float d[3], float &near, float &far, int64_t &ray)
{
    if (CAMS) {
        // tiles of a group of G consecutive cameras are interleaved: the same
        // tile of each camera of the group in turn, so neighbouring views
        // (which touch nearly the same leaves) share L1/L2
        // 32-bit arithmetic: the host keeps tile counts below 2^32
        const uint32_t tl = (uint32_t)tile;
        const uint32_t G = (uint32_t)p.view_group;
        const uint32_t per_group = (uint32_t)p.tiles_per_cam * G;
        const uint32_t group = tl / per_group;
        const uint32_t in_group = tl - group * per_group;
        const uint32_t gsize = min(G, (uint32_t)p.n_cams - group * G);
        const int64_t cam = (int64_t)(group * G + in_group % gsize);
        const uint32_t rem = in_group / gsize;
        const int ty = (int)(rem / (uint32_t)p.tiles_x);
        const int tx = (int)(rem - (uint32_t)ty * (uint32_t)p.tiles_x);
        const int i = tx * kTileW + (slot % kTileW);
        const int j = ty * kTileH + (slot / kTileW);
        if (i >= p.W || j >= p.H) return false;
        ray = (cam * p.H + j) * p.W + i;
        const pot_camera *c = p.cams + cam;
        // a1: pixel ray, each operation rounded once in the stated order
        const float xc = __fdiv_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), c->cx), c->fx);
        const float yc = -__fdiv_rn(__fsub_rn(__fadd_rn((float)j, 0.5f), c->cy), c->fy);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            d[r] = __fsub_rn(__fadd_rn(__fmul_rn(c->c2w[r][0], xc), __fmul_rn(c->c2w[r][1], yc)), c->c2w[r][2]);
            o[r] = c->c2w[r][3];
        }
        near = c->near;
        far = c->far;
        return true;
    }
    ray = (int64_t)tile * 32 + slot;
    if (ray >= p.n_rays) return false;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        o[r] = __ldg(p.ray_o + 3 * ray + r);
        d[r] = __ldg(p.ray_d + 3 * ray + r);
    }
    near = p.near;
    far = p.far;
    return true;
}

template <int K, typename T, bool COUNT>
__device__ __forceinline__ void store_ray(const RenderParams &p, int64_t ray, const ShadeVisitor<K, T, COUNT> &v)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) p.rgb[3 * ray + c] = fmaf(v.Tr, p.bg[c], v.col[c]);
    if (p.t_final) p.t_final[ray] = v.Tr;
    if (COUNT) p.seg_count[ray] = v.nseg;
}

// Forward render, one tile per warp at a time: the warp takes the next tile
// once all 32 of its rays are done.
template <int K, typename T, bool CAMS, bool COUNT>
__global__ void __launch_bounds__(kBlock, POT_RENDER_MIN_BLOCKS) render_kernel(const RenderParams p)
{
    POT_WALK_SHARED(K)
    const int lane = threadIdx.x & 31;
    const T *sig_arr = static_cast<const T *>(p.sigma);
    const T *sh_arr = static_cast<const T *>(p.sh);
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(p.tile_counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= (unsigned long long)p.n_tiles) break;
        float o[3], d[3], near, far;
        int64_t ray;
        if (tile_ray<CAMS>(p, tile, lane, o, d, near, far, ray)) {
            ShadeVisitor<K, T, COUNT> v{sig_arr, sh_arr, p.leaf_touched, p.gamma, {0.f, 0.f, 0.f}, 1.f, 0,
                                        p.codebook};
            walk_ray<K, T>(p, sig_arr, sh_arr, stk, ysm, wst, o, d, near, far, v);
            store_ray<K, T, COUNT>(p, ray, v);
        }
    }
}

template <typename T>
cudaError_t launch_render_t(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                            int max_blocks)
{
    using Fn = void (*)(const RenderParams);
    Fn fn = nullptr;
#define POT_PICK(KK)                                                                            \
    if (K == KK)                                                                                \
        fn = cams ? (count ? render_kernel<KK, T, true, true> : render_kernel<KK, T, true, false>) \
                  : (count ? render_kernel<KK, T, false, true> : render_kernel<KK, T, false, false>);
    POT_PICK(1)
    POT_PICK(4)
    POT_PICK(9)
    POT_PICK(16)
    POT_PICK(25)
#undef POT_PICK
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = walk_smem_bytes(p.cells == nullptr);
    unsigned grid = 0;
    cudaError_t e = persistent_grid(fn, smem, p.n_tiles, max_blocks, &grid);
    if (e != cudaSuccess) return e;
    fn<<<grid, kBlock, smem, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pot
