// pot_record.cu -- forward render of explicit rays that records every
// composited leaf segment (ray, leaf, delta_i, T_i, P_i) for the per-record
// backward of App. B.3.2 (training batches, Sec. 3.3).
//
// The walk and the compositing are the render kernel's (Walker, ShadeVisitor),
// so colours, transmittances and early-stop points are bit-identical to
// pot_render_rays.  The walk loop is warp-synchronous: after every step the
// warp counts, with one ballot, the lanes that composited a segment and
// writes their records to consecutive slots of a block of POT_SEGMENT_BLOCK
// slots that the warp reserved from the buffer's counter (one atomic per
// block, not per segment).  The record of one segment is two 16-byte stores;
// the lanes of a step write one contiguous span.
#include "pot_render.cuh"
#include "pot_segments_internal.h"

#ifndef POT_RECORD_MIN_BLOCKS
#define POT_RECORD_MIN_BLOCKS 3  // resident blocks per SM: 80 registers, no spills (64 registers spill 28 bytes)
#endif

namespace pot {

namespace {

// The render's shading of a segment, keeping what the backward needs of it:
// T_i and P_i (the transmittance and the composited colour in front of it).
template <int K, typename T>
struct RecordVisitor {
    ShadeVisitor<K, T, false> sv;
    bool has;
    int leaf;
    float delta, T0, P0[3];
    template <typename YT>
    __device__ __forceinline__ bool operator()(int l, float dl, const YT &Y)
    {
        has = true;
        leaf = l;
        delta = dl;
        T0 = sv.Tr;
#pragma unroll
        for (int c = 0; c < 3; ++c) P0[c] = sv.col[c];
        return sv(l, dl, Y);
    }
};

template <int K, typename T>
__global__ void __launch_bounds__(kBlock, POT_RECORD_MIN_BLOCKS)
    record_kernel(const RenderParams p, const SegmentBuffer sb)
{
    POT_WALK_SHARED(K)
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const T *sig_arr = static_cast<const T *>(p.sigma);
    const T *sh_arr = static_cast<const T *>(p.sh);
    // this warp's block of slots [base, base + kSegBlock), of which `fill` are
    // used; warp-uniform (every lane holds the same values).  fill = kSegBlock
    // with base = -1: no block yet.  dead: the buffer is full, record nothing.
    long long base = -1;
    int fill = kSegBlock;
    bool dead = false;
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(p.tile_counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= (unsigned long long)p.n_tiles) break;
        const int64_t ray = (int64_t)tile * 32 + lane;
        RecordVisitor<K, T> v;
        v.sv = ShadeVisitor<K, T, false>{sig_arr, sh_arr, nullptr, p.gamma, {0.f, 0.f, 0.f}, 1.f, 0, nullptr};
        v.has = false;
        Walker<K, T> w;
        w.ysm = ysm;
        w.st = wst;
        bool alive = false;
        if (ray < p.n_rays) {
            float o[3], d[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                o[r] = __ldg(p.ray_o + 3 * ray + r);
                d[r] = __ldg(p.ray_d + 3 * ray + r);
            }
            alive = w.begin(p, stk, sig_arr, sh_arr, o, d, p.near, p.far);
        }
        while (__any_sync(0xffffffffu, alive)) {
            v.has = false;
            if (alive) alive = w.step(p, stk, sig_arr, sh_arr, v);
            const unsigned m = __ballot_sync(0xffffffffu, v.has);
            if (m == 0u || dead) continue;
            const int nseg = __popc(m);
            const int pos = fill + __popc(m & below);  // this lane's place, counted from the block's start
            long long slot;
            if (fill + nseg <= kSegBlock) {
                slot = base + pos;  // fill < kSegBlock: the block is a reserved one
                fill += nseg;
            } else {
                // the block is full after the first kSegBlock - fill lanes:
                // the rest go to a new block
                unsigned long long nb = 0;
                if (lane == 0) nb = atomicAdd(sb.state, (unsigned long long)kSegBlock);
                nb = __shfl_sync(0xffffffffu, nb, 0);
                const bool fits = nb + (unsigned long long)kSegBlock <= (unsigned long long)sb.capacity;
                slot = pos < kSegBlock ? base + pos : (fits ? (long long)nb + (pos - kSegBlock) : -1ll);
                if (fits) {
                    base = (long long)nb;
                    fill = fill + nseg - kSegBlock;
                } else {
                    dead = true;
                    base = -1;
                    fill = kSegBlock;
                    if (lane == 0) sb.state[1] = 1ull;
                }
            }
            if (v.has && slot >= 0) {
                float4 *r = sb.rec + 2 * slot;
                r[0] = make_float4(__int_as_float((int)ray), __int_as_float(v.leaf), v.delta, v.T0);
                r[1] = make_float4(v.P0[0], v.P0[1], v.P0[2], 0.f);
            }
        }
        if (ray < p.n_rays) store_ray<K, T, false>(p, ray, v.sv);
    }
    // the slots of the last block that this warp did not use
    if (base >= 0)
        for (int j = fill + lane; j < kSegBlock; j += 32)
            sb.rec[2 * (base + j)] = make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
}

template <typename T>
cudaError_t launch_record_t(const RenderParams &p, const SegmentBuffer &sb, int K, cudaStream_t s)
{
    using Fn = void (*)(const RenderParams, const SegmentBuffer);
    Fn fn = K == 1 ? record_kernel<1, T> : K == 4 ? record_kernel<4, T> : K == 9 ? record_kernel<9, T>
          : K == 16 ? record_kernel<16, T> : K == 25 ? record_kernel<25, T> : nullptr;
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = walk_smem_bytes(p.cells == nullptr);
    unsigned grid = 0;
    cudaError_t e = persistent_grid(fn, smem, p.n_tiles, 0, &grid);
    if (e != cudaSuccess) return e;
    fn<<<grid, kBlock, smem, s>>>(p, sb);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_record(const RenderParams &p, const SegmentBuffer &sb, int dtype, int K, cudaStream_t s)
{
    switch (dtype) {
    case POT_F32: return launch_record_t<float>(p, sb, K, s);
    case POT_F16: return launch_record_t<__half>(p, sb, K, s);
    case POT_BF16: return launch_record_t<__nv_bfloat16>(p, sb, K, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pot
