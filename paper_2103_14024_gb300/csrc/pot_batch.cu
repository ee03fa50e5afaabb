// pot_batch.cu -- one launch renders many requests: different trees, cameras,
// resolutions and outputs (the work list of a continuous-batching server).
//
// The host groups the items by (SH coefficients, leaf dtype); each group is one
// launch.  Every item contributes tiles of kTileW x kTileH pixels (as pot_render);
// warps take tiles from one counter and find their item by binary search over
// the items' first-tile offsets.  The per-ray code (walk + shading) is the
// same as pot_render's, so a request renders bit-identically alone or in a mix.
#include <algorithm>
#include <vector>

#include "pot_render.cuh"

namespace pot {

namespace {

struct BatchItem {
    const int32_t *child;
    const int32_t *cells;
    const int32_t *btab;
    const void *sigma;
    const void *sh;
    const void *codebook;
    int depth, R;
    float lo[3];
    float size, h, invh;
    float bg[3];
    float gamma;
    int W, H, tiles_x;
    int64_t tile_begin;
    float *rgb;
    float *t_final;
    pot_camera cam;
};

struct BatchParams {
    const BatchItem *items;
    int n_items;
    int64_t n_tiles;
    unsigned long long *tile_counter;
    unsigned int *err;
};

template <int K, typename T>
__global__ void __launch_bounds__(kBlock, POT_RENDER_MIN_BLOCKS) batch_kernel(const BatchParams bp)
{
    POT_WALK_SHARED(K)
    const int lane = threadIdx.x & 31;
    // short blocks: every warp renders one tile and the block ends, so a
    // launch frees its SM slots tile by tile and launches of higher-priority
    // streams (small requests) start between them
    {
        const unsigned long long tile = (unsigned long long)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
        if (tile >= (unsigned long long)bp.n_tiles) return;
        // item owning the tile: the last item with tile_begin <= tile, by a
        // warp-wide search -- each round the 32 lanes test 32 evenly spaced
        // items of [lo, hi] at once and the range shrinks to one stride (one
        // round up to 32 items, two up to 1024), instead of a chain of
        // dependent loads of a binary search.  items[lo].tile_begin <= tile
        // holds throughout (item 0 begins at tile 0).
        int lo = 0, hi = bp.n_items - 1;
        while (hi > lo) {
            const int stride = (hi - lo + 32) / 32;
            const int cand = lo + lane * stride;
            const bool ok = cand <= hi && bp.items[cand].tile_begin <= (int64_t)tile;
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            lo += (31 - __clz(m)) * stride;
            hi = min(hi, lo + stride - 1);
        }
        const BatchItem &it = bp.items[lo];
        const int64_t rem = (int64_t)tile - it.tile_begin;
        const int ty = (int)(rem / it.tiles_x);
        const int tx = (int)(rem - (int64_t)ty * it.tiles_x);
        const int i = tx * kTileW + (lane % kTileW);
        const int j = ty * kTileH + (lane / kTileW);
        if (i < it.W && j < it.H) {
            RenderParams p;
            p.child = it.child;
            p.cells = it.cells;
            p.btab = it.btab;
            p.depth = it.depth;
            p.R = it.R;
            p.lo[0] = it.lo[0];
            p.lo[1] = it.lo[1];
            p.lo[2] = it.lo[2];
            p.size = it.size;
            p.h = it.h;
            p.invh = it.invh;
            p.step_cap = 3 * it.R + 16;
            p.err = bp.err;
            const pot_camera *c = &it.cam;
            float o[3], d[3];
            const float xc = __fdiv_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), c->cx), c->fx);
            const float yc = -__fdiv_rn(__fsub_rn(__fadd_rn((float)j, 0.5f), c->cy), c->fy);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                d[r] = __fsub_rn(__fadd_rn(__fmul_rn(c->c2w[r][0], xc), __fmul_rn(c->c2w[r][1], yc)),
                                 c->c2w[r][2]);
                o[r] = c->c2w[r][3];
            }
            const T *sig_arr = static_cast<const T *>(it.sigma);
            const T *sh_arr = static_cast<const T *>(it.sh);
            ShadeVisitor<K, T, false> v{sig_arr, sh_arr, nullptr, it.gamma, {0.f, 0.f, 0.f}, 1.f, 0, it.codebook};
            walk_ray<K, T>(p, sig_arr, sh_arr, stk, ysm, wst, o, d, c->near, c->far, v);
            const int64_t px = (int64_t)j * it.W + i;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) it.rgb[3 * px + ch] = fmaf(v.Tr, it.bg[ch], v.col[ch]);
            if (it.t_final) it.t_final[px] = v.Tr;
        }
    }
}

template <typename T>
cudaError_t launch_batch_t(const BatchParams &bp, int K, bool need_stack, cudaStream_t s)
{
    using Fn = void (*)(const BatchParams);
    Fn fn = K == 1 ? batch_kernel<1, T> : K == 4 ? batch_kernel<4, T> : K == 9 ? batch_kernel<9, T>
          : K == 16 ? batch_kernel<16, T> : K == 25 ? batch_kernel<25, T> : nullptr;
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = walk_smem_bytes(need_stack);
    const int64_t blocks = (bp.n_tiles + kBlock / 32 - 1) / (kBlock / 32);
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)(blocks > 0 ? blocks : 1);
    fn<<<grid, kBlock, smem, s>>>(bp);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

// items: host array of n validated requests; groups by (K, dtype), stages the
// descriptors and one counter per group in a single stream-ordered buffer.
cudaError_t launch_render_batch(const pot_render_item *items, int n, cudaStream_t s, unsigned int *err)
{
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto key = [&](int i) { return items[i].tree->K * 4 + items[i].tree->desc.leaf_dtype; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });
    std::vector<BatchItem> desc(n);
    std::vector<int> group_start;
    int64_t tiles = 0;
    for (int k = 0; k < n; ++k) {
        const pot_render_item &r = items[order[k]];
        if (k == 0 || key(order[k]) != key(order[k - 1])) {
            group_start.push_back(k);
            tiles = 0;
        }
        const pot_tree *t = r.tree;
        BatchItem &b = desc[k];
        b.child = t->child;
        b.cells = t->cells;
        b.btab = t->btab;
        b.sigma = t->sigma;
        b.sh = t->sh;
        b.codebook = t->codebook;
        b.depth = t->desc.depth;
        b.R = 1 << t->desc.depth;
        for (int a = 0; a < 3; ++a) b.lo[a] = t->desc.bbox_lo[a];
        b.size = t->desc.bbox_size;
        b.h = t->h;
        b.invh = 1.0f / t->h;
        for (int c = 0; c < 3; ++c) b.bg[c] = r.bg[c];
        b.gamma = r.gamma;
        b.W = r.cam.width;
        b.H = r.cam.height;
        b.tiles_x = (b.W + kTileW - 1) / kTileW;
        b.tile_begin = tiles;
        b.rgb = r.rgb;
        b.t_final = r.t_final;
        b.cam = r.cam;
        tiles += (int64_t)b.tiles_x * ((b.H + kTileH - 1) / kTileH);
    }
    group_start.push_back(n);
    const int groups = (int)group_start.size() - 1;
    const size_t cnt_bytes = 256;
    const size_t bytes = cnt_bytes + sizeof(BatchItem) * (size_t)n;
    void *buf = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&buf, bytes, pool, s);
    if (e != cudaSuccess) return e;
    char *cb = static_cast<char *>(buf);
    BatchItem *d_items = reinterpret_cast<BatchItem *>(cb + cnt_bytes);
    e = cudaMemsetAsync(cb, 0, cnt_bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, desc.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice, s);
    for (int g = 0; g < groups && e == cudaSuccess; ++g) {
        const int a = group_start[g], b = group_start[g + 1];
        const BatchItem &last = desc[b - 1];
        BatchParams bp;
        bp.items = d_items + a;
        bp.n_items = b - a;
        bp.n_tiles = last.tile_begin + (int64_t)last.tiles_x * ((last.H + kTileH - 1) / kTileH);
        bp.tile_counter = reinterpret_cast<unsigned long long *>(cb) + g;
        bp.err = err;
        const pot_tree *t = items[order[a]].tree;
        bool need_stack = false;  // some tree of the group without a cell index
        for (int k = a; k < b; ++k) need_stack = need_stack || desc[k].cells == nullptr;
        switch (t->desc.leaf_dtype) {
        case POT_F32: e = launch_batch_t<float>(bp, t->K, need_stack, s); break;
        case POT_F16: e = launch_batch_t<__half>(bp, t->K, need_stack, s); break;
        case POT_CB16: e = launch_batch_t<cb16>(bp, t->K, need_stack, s); break;
        default: e = launch_batch_t<__nv_bfloat16>(bp, t->K, need_stack, s); break;
        }
    }
    cudaFreeAsync(buf, s);
    return e;
}

}  // namespace pot
