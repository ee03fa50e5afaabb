// pot_backward.cu -- analytic derivatives of the render (App. B.3.2), the
// optimiser step on the leaves (Sec. 3.3), the MSE loss of a ray batch (Sec. 3,
// NeRF loss) and pixel-ray generation for training batches.
//
// Backward, per ray (replaying the forward walk, so segments and the early-
// stop point are the forward's):
//   c_i = S(x_i),  x_i = sum_k k_{i,k} Y_k,  w_i = T_i (1 - e^{-sigma_i delta_i})
//   dC/dx_i      = w_i c_i (1 - c_i)                         (colour derivative, chain rule)
//   dC/dk_{i,k}  = dC/dx_i Y_k                               (basis constant along the ray)
//   dC/dsigma_i  = delta_i [ c_i T_{i+1} - S_i ],  S_i = sum_{k>i} w_k c_k + T_N bg
//                = delta_i [ c_i T_{i+1} - (C - sum_{k<=i} w_k c_k) ]
// i.e. the paper's two passes: the composited colour C (the forward output,
// or a first in-kernel pass) minus a running prefix.  Zero for sigma <= 0.
// Gradients of L = sum_rays <dL/dC, C> are scattered with float reductions
// (16-byte vector reductions where the row allows).  With POT_BWD_AGG, lanes
// of a warp that composite the same leaf in the same step first sum their
// contributions with warp shuffles (warp-aggregated atomics) and one lane per
// leaf issues the reductions.
#include <cmath>

#include "pot_render.cuh"
#include "pot_segments_internal.h"

#ifndef POT_BWD_AGG
// warp-aggregated gradient scatter (lanes sharing a leaf reduce by shuffles
// first).  Off: measured slower on 2^18-ray batches of the main tree, both for
// random pixels (1.28 vs 0.86 ms) and for random 4 x 8 pixel tiles, whose
// lanes do share leaves (0.75 vs 0.53 ms): the match and the 49-value shuffle
// tree cost more than the float reductions they save.
#define POT_BWD_AGG 0
#endif

namespace pot {

namespace {

__device__ __forceinline__ void red_add(float *a, float v)
{
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(a), "f"(v) : "memory");
}

__device__ __forceinline__ void red_add4(float *a, float x, float y, float z, float w)
{
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(x), "f"(y), "f"(z),
                 "f"(w)
                 : "memory");
}

// The terms of one leaf segment (App. B.3.2), given T_i (Tr) and the colour
// composited in front of it (prefix): the colour derivative gx_c =
// dL/dC_c w c_c (1 - c_c) (times Y_k for coefficient k) and the density
// derivative gsd (0 for sigma <= 0); Tr and prefix move past the segment.
// Returns whether sigma > 0.  The same operations as the forward's shading.
template <int K, typename T, typename YT>
__device__ __forceinline__ bool segment_terms(const T *sig_arr, const T *sh_arr, int leaf, float delta, const YT &Y,
                                              const float g[3], const float ctot[3], float prefix[3], float &Tr,
                                              float gx[3], float &gsd)
{
    const float sraw = Store<T>::load_sigma(sig_arr, leaf);
    const float sig = fmaxf(sraw, 0.f);
    float x[3];
    leaf_sh_dot<K, T>(sh_arr, leaf, Y, x, nullptr);
    const float e = __expf(-sig * delta);  // same operations as the forward
    const float w = Tr * (1.f - e);
    const float Tn = Tr * e;
    float gs = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float col = sigmoidf_(x[c]);
        prefix[c] = fmaf(w, col, prefix[c]);
        gx[c] = g[c] * w * col * (1.f - col);
        gs = fmaf(g[c], fmaf(col, Tn, -(ctot[c] - prefix[c])), gs);
    }
    gsd = sraw > 0.f ? gs * delta : 0.f;  // zero for sigma <= 0 (same leaf: same sign)
    Tr = Tn;
    return sraw > 0.f;
}

template <int K, typename T>
struct GradVisitor {
    const T *sig_arr;
    const T *sh_arr;
    float gamma;
    float g[3];       // dL/dC of the ray
    float ctot[3];    // C of the ray (background included)
    float prefix[3];  // sum over composited segments of w c
    float Tr;
    float *grad_sigma;
    float *grad_sh;
    template <typename YT>
    __device__ __forceinline__ bool operator()(int leaf, float delta, const YT &Y)
    {
        float gx[3], gsd;
        const bool pos = segment_terms<K, T>(sig_arr, sh_arr, leaf, delta, Y, g, ctot, prefix, Tr, gx, gsd);
        float *row = grad_sh + (int64_t)leaf * (3 * K);
#if POT_BWD_AGG
        // lanes compositing the same leaf: sum over the group with a shuffle
        // tree over its members (ranked by lane); the lowest lane scatters
        const unsigned act = __activemask();
        const unsigned grp = __match_any_sync(act, leaf);
        const unsigned shared_lanes = __ballot_sync(act, __popc(grp) > 1);
        if (shared_lanes) {
            const int lane = threadIdx.x & 31;
            if (grp != (1u << lane)) {
                const int n = __popc(grp);
                const int rank = __popc(grp & ((1u << lane) - 1u));
                const int nmax = (int)__reduce_max_sync(shared_lanes, (unsigned)n);
                float v[3 * K];
#pragma unroll
                for (int j = 0; j < 3 * K; ++j) v[j] = gx[j % 3] * Y[j / 3];
                for (int o = 1; o < nmax; o <<= 1) {
                    const bool has = rank + o < n;
                    const int src = has ? (int)__fns(grp, (unsigned)lane, o + 1) : lane;
#pragma unroll
                    for (int j = 0; j < 3 * K; ++j) {
                        const float t = __shfl_sync(shared_lanes, v[j], src);
                        if (has) v[j] += t;
                    }
                    const float t = __shfl_sync(shared_lanes, gsd, src);
                    if (has) gsd += t;
                }
                if (rank == 0) {
                    if ((3 * K) % 4 == 0) {
#pragma unroll
                        for (int j = 0; j < 3 * K; j += 4) red_add4(row + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 3 * K; ++j) red_add(row + j, v[j]);
                    }
                    if (pos) red_add(grad_sigma + leaf, gsd);
                }
                return Tr < gamma;
            }
        }
#endif
        if ((3 * K) % 4 == 0) {
#pragma unroll
            for (int j = 0; j < 3 * K; j += 4)
                red_add4(row + j, gx[j % 3] * Y[j / 3], gx[(j + 1) % 3] * Y[(j + 1) / 3],
                         gx[(j + 2) % 3] * Y[(j + 2) / 3], gx[(j + 3) % 3] * Y[(j + 3) / 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 3 * K; ++j) red_add(row + j, gx[j % 3] * Y[j / 3]);
        }
        if (pos) red_add(grad_sigma + leaf, gsd);
        return Tr < gamma;
    }
};

struct BackwardParams {
    RenderParams r;
    const float *grad_rgb;
    const float *rgb_fwd;  // NULL: computed by a first pass
    float *grad_sigma;
    float *grad_sh;
    // fused MSE mode: dL/dC = mse_scale (C - target), L += sum (C - target)^2 mse_scale / 2
    const float *target;
    float *loss;
    float *rgb_out;        // optional copy of C
    float mse_scale;
    // non-null: the kernel runs only if *run_if != 0 (the walking backward as
    // the fallback of the per-record backward, whose records overflowed)
    const unsigned long long *run_if;
};

// What the backward kernel is given per ray.
enum BackwardMode { kGradAndColour = 0, kGrad = 1, kMseTarget = 2 };

#ifndef POT_BACKWARD_MIN_BLOCKS
// resident blocks per SM: 2 (112 registers); 3 blocks (80 registers, no
// spills) and 4 (64, small spills) measured slower on 2^18-ray batches of the
// main tree: 0.96 and 1.39 ms against 0.80 ms for random pixels
#define POT_BACKWARD_MIN_BLOCKS 2
#endif

// MODE kGradAndColour: dL/dC and C given; kGrad: dL/dC given, C from a first
// walk; kMseTarget: C from a first walk, then dL/dC of the MSE against the
// target, the loss summed per warp into *loss, C optionally written out.
template <int K, typename T, int MODE>
__global__ void __launch_bounds__(kBlock, POT_BACKWARD_MIN_BLOCKS) backward_kernel(const BackwardParams bp)
{
    POT_WALK_SHARED(K)
    const RenderParams &p = bp.r;
    if (bp.run_if && *bp.run_if == 0ull) return;
    const int lane = threadIdx.x & 31;
    const T *sig_arr = static_cast<const T *>(p.sigma);
    const T *sh_arr = static_cast<const T *>(p.sh);
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(p.tile_counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= (unsigned long long)p.n_tiles) break;
        const int64_t ray = (int64_t)tile * 32 + lane;
        float lsum = 0.f;  // this ray's squared error (MSE mode)
        if (ray < p.n_rays) {
            float o[3], d[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                o[r] = __ldg(p.ray_o + 3 * ray + r);
                d[r] = __ldg(p.ray_d + 3 * ray + r);
            }
            GradVisitor<K, T> gv;
            gv.sig_arr = sig_arr;
            gv.sh_arr = sh_arr;
            gv.gamma = p.gamma;
            gv.Tr = 1.f;
            gv.grad_sigma = bp.grad_sigma;
            gv.grad_sh = bp.grad_sh;
#pragma unroll
            for (int c = 0; c < 3; ++c) gv.prefix[c] = 0.f;
            if (MODE == kGradAndColour) {
#pragma unroll
                for (int c = 0; c < 3; ++c) gv.ctot[c] = __ldg(bp.rgb_fwd + 3 * ray + c);
            } else {
                ShadeVisitor<K, T, false> sv{sig_arr, sh_arr, nullptr, p.gamma, {0.f, 0.f, 0.f}, 1.f, 0, nullptr};
                walk_ray<K, T>(p, sig_arr, sh_arr, stk, ysm, wst, o, d, p.near, p.far, sv);
#pragma unroll
                for (int c = 0; c < 3; ++c) gv.ctot[c] = fmaf(sv.Tr, p.bg[c], sv.col[c]);
            }
            if (MODE == kMseTarget) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float r = gv.ctot[c] - __ldg(bp.target + 3 * ray + c);
                    lsum = fmaf(r, r, lsum);
                    gv.g[c] = bp.mse_scale * r;
                    if (bp.rgb_out) bp.rgb_out[3 * ray + c] = gv.ctot[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) gv.g[c] = __ldg(bp.grad_rgb + 3 * ray + c);
            }
            if (gv.g[0] != 0.f || gv.g[1] != 0.f || gv.g[2] != 0.f)
                walk_ray<K, T>(p, sig_arr, sh_arr, stk, ysm, wst, o, d, p.near, p.far, gv);
        }
        if (MODE == kMseTarget) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if (lane == 0 && lsum != 0.f) atomicAdd(bp.loss, 0.5f * bp.mse_scale * lsum);
        }
    }
}

template <typename T>
cudaError_t launch_backward_t(const BackwardParams &bp, int K, int mode, cudaStream_t s)
{
    using Fn = void (*)(const BackwardParams);
    Fn fn = nullptr;
#define POT_PICK(KK)                                                                              \
    if (K == KK)                                                                                  \
        fn = mode == kGradAndColour ? backward_kernel<KK, T, kGradAndColour>                      \
             : mode == kGrad        ? backward_kernel<KK, T, kGrad>                               \
                                    : backward_kernel<KK, T, kMseTarget>;
    POT_PICK(1)
    POT_PICK(4)
    POT_PICK(9)
    POT_PICK(16)
    POT_PICK(25)
#undef POT_PICK
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = walk_smem_bytes(bp.r.cells == nullptr);
    unsigned grid = 0;
    cudaError_t e = persistent_grid(fn, smem, bp.r.n_tiles, 0, &grid);
    if (e != cudaSuccess) return e;
    fn<<<grid, kBlock, smem, s>>>(bp);
    count_launch();
    return cudaGetLastError();
}

// ---- gradients from recorded segments ---------------------------------------
// One thread per record of pot_render_rays_record: the record gives the leaf,
// delta_i, T_i and P_i, the ray gives dL/dC, C and the SH basis at its
// direction; GradVisitor then does exactly the per-segment work of the walking
// backward (same operations, so the same per-segment terms bit for bit).

// The per-ray SH basis in registers (the interface of SmemY).
template <int K>
struct RegY {
    float v[K];
    __device__ __forceinline__ float operator[](int k) const { return v[k]; }
    __device__ __forceinline__ void fetch(float *yv, int k0, int k1) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (k >= k0 && k <= k1) yv[k] = v[k];
    }
};

struct SegBackwardParams {
    SegmentBuffer sb;
    int64_t n_rays;    // records naming a ray or leaf outside these ranges are skipped
    int64_t n_leaves;
    // non-null: visit the records in the order perm[0 .. *n_perm) (by bin of
    // leaves, so that the reductions of neighbouring threads meet the same
    // gradient rows in L2); null: in slot order
    const unsigned *perm;
    const unsigned *n_perm;
    const void *sigma;
    const void *sh;
    const float *ray_d;
    const float *grad_rgb;
    const float *rgb_fwd;
    float *grad_sigma;
    float *grad_sh;
};

#ifndef POT_SEGBWD_MIN_BLOCKS
// resident blocks per SM: 3 (at most 80 registers, no spills; 4 blocks spill 12 bytes at 64)
#define POT_SEGBWD_MIN_BLOCKS 3
#endif

// The sum of v over the lanes of each run of adjacent lanes (run0: this
// lane's run starts there), complete in the run's last lane (a scan within
// runs).
__device__ __forceinline__ float run_sum(float v, int lane, int run0)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane - d >= run0) v += t;
    }
    return v;
}

// Whole warps step over the records together.  Lanes next to each other
// that hold records of the same leaf (records in leaf order, or neighbouring
// rays of one forward step in slot order) form a run: the run's terms are
// summed with shuffles and its last lane issues the float reductions, so a
// leaf's row gets one set of reductions per warp and step instead of one per
// record.
template <int K, typename T>
__global__ void __launch_bounds__(kBlock, POT_SEGBWD_MIN_BLOCKS) segment_backward_kernel(const SegBackwardParams q)
{
    if (q.sb.state[1] != 0ull) return;  // the records overflowed: the walking backward runs instead
    const unsigned long long handed = q.sb.state[0];
    const int64_t used = q.perm ? (int64_t)*q.n_perm
                       : handed < (unsigned long long)q.sb.capacity ? (int64_t)handed : q.sb.capacity;
    const int lane = threadIdx.x & 31;
    const T *sig_arr = static_cast<const T *>(q.sigma);
    const T *sh_arr = static_cast<const T *>(q.sh);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); k0 < used; k0 += stride) {
        const int64_t k = k0 + lane;
        int leaf = -1;  // -1: no terms on this lane
        float gx[3] = {0.f, 0.f, 0.f}, gsd = 0.f;
        RegY<K> Y;
#pragma unroll
        for (int j = 0; j < K; ++j) Y.v[j] = 0.f;
        if (k < used) {
            const int64_t i = q.perm ? (int64_t)q.perm[k] : k;
            const float4 a = __ldg(q.sb.rec + 2 * i);
            const int ray = __float_as_int(a.x), lf = __float_as_int(a.y);
            // unused slots (ray -1) and records naming a ray or leaf out of range are skipped
            if (ray >= 0 && ray < q.n_rays && lf >= 0 && lf < q.n_leaves) {
                float g[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) g[c] = __ldg(q.grad_rgb + 3 * (int64_t)ray + c);
                if (g[0] != 0.f || g[1] != 0.f || g[2] != 0.f) {
                    const float4 b4 = __ldg(q.sb.rec + 2 * i + 1);
                    float ctot[3], prefix[3] = {b4.x, b4.y, b4.z}, d[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) ctot[c] = __ldg(q.rgb_fwd + 3 * (int64_t)ray + c);
#pragma unroll
                    for (int c = 0; c < 3; ++c) d[c] = __ldg(q.ray_d + 3 * (int64_t)ray + c);
                    // the basis exactly as the walk computes it (Walker::begin)
                    const float len = sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
                    const float invlen = __frcp_rn(len);
                    sh_basis<K>(d[0] * invlen, d[1] * invlen, d[2] * invlen, Y.v);
                    float Tr = a.w;
                    segment_terms<K, T>(sig_arr, sh_arr, lf, a.z, Y, g, ctot, prefix, Tr, gx, gsd);
                    leaf = lf;
                }
            }
        }
        const int prev = __shfl_up_sync(0xffffffffu, leaf, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || leaf != prev);
        float *row = q.grad_sh + (int64_t)(leaf < 0 ? 0 : leaf) * (3 * K);
        if (heads == 0xffffffffu) {  // no two adjacent lanes share a leaf: reductions per lane
            if (leaf >= 0) {
                if ((3 * K) % 4 == 0) {
#pragma unroll
                    for (int j = 0; j < 3 * K; j += 4)
                        red_add4(row + j, gx[j % 3] * Y[j / 3], gx[(j + 1) % 3] * Y[(j + 1) / 3],
                                 gx[(j + 2) % 3] * Y[(j + 2) / 3], gx[(j + 3) % 3] * Y[(j + 3) / 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 3 * K; ++j) red_add(row + j, gx[j % 3] * Y[j / 3]);
                }
                if (gsd != 0.f) red_add(q.grad_sigma + leaf, gsd);
            }
            continue;
        }
        const int run0 = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // last head at or before this lane
        const bool tail = leaf >= 0 && (lane == 31 || ((heads >> (lane + 1)) & 1u));
        if ((3 * K) % 4 == 0) {
#pragma unroll
            for (int j = 0; j < 3 * K; j += 4) {
                const float v0 = run_sum(gx[j % 3] * Y[j / 3], lane, run0);
                const float v1 = run_sum(gx[(j + 1) % 3] * Y[(j + 1) / 3], lane, run0);
                const float v2 = run_sum(gx[(j + 2) % 3] * Y[(j + 2) / 3], lane, run0);
                const float v3 = run_sum(gx[(j + 3) % 3] * Y[(j + 3) / 3], lane, run0);
                if (tail) red_add4(row + j, v0, v1, v2, v3);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 3 * K; ++j) {
                const float v = run_sum(gx[j % 3] * Y[j / 3], lane, run0);
                if (tail) red_add(row + j, v);
            }
        }
        const float gs = run_sum(gsd, lane, run0);
        if (tail && gs != 0.f) red_add(q.grad_sigma + leaf, gs);
    }
}

template <typename T>
cudaError_t launch_segment_backward_t(const SegBackwardParams &q, int K, cudaStream_t s)
{
    using Fn = void (*)(const SegBackwardParams);
    Fn fn = K == 1 ? segment_backward_kernel<1, T> : K == 4 ? segment_backward_kernel<4, T>
          : K == 9 ? segment_backward_kernel<9, T> : K == 16 ? segment_backward_kernel<16, T>
          : K == 25 ? segment_backward_kernel<25, T> : nullptr;
    if (!fn) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0);
    if (e != cudaSuccess) return e;
    // one wave of resident blocks, no more than the slots could need
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (q.sb.capacity + kBlock - 1) / kBlock;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    fn<<<(unsigned)blocks, kBlock, 0, s>>>(q);
    count_launch();
    return cudaGetLastError();
}

// ---- recorded segments in leaf order ----------------------------------------
// The records are visited sorted by leaf (a counting sort: records per leaf,
// a scan, the record numbers scattered to their leaf's range): a leaf's
// records are then adjacent, so the per-record kernel merges them within a
// warp, and neighbouring threads reduce into neighbouring gradient rows.

struct SegBinParams {
    SegBackwardParams s;
    const unsigned *start;  // [n_bins + 1] first sorted position of each leaf
    unsigned *count;        // [n_bins] records per leaf
    unsigned *cursor;       // [n_bins] scatter cursors
    unsigned *perm;         // [capacity] record numbers in leaf order
    unsigned *tile_sum;     // [ceil(n_bins / kScanTile)] scan partials
    int64_t n_bins;         // = n_leaves
};

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;  // counts per scan block
static_assert(kScanTile == kSegScanTile, "scan tile of the scratch layout");

// A record's leaf, or -1 for an unused slot or one naming an out-of-range ray
// or leaf.
__device__ __forceinline__ int record_leaf(const SegBackwardParams &q, int64_t i, int64_t used)
{
    if (i >= used) return -1;
    const float4 a = __ldg(q.sb.rec + 2 * i);
    const int ray = __float_as_int(a.x), leaf = __float_as_int(a.y);
    if (ray < 0 || ray >= q.n_rays || leaf < 0 || leaf >= q.n_leaves) return -1;
    return leaf;
}

__device__ __forceinline__ int64_t records_used(const SegmentBuffer &sb)
{
    const unsigned long long handed = sb.state[0];
    return handed < (unsigned long long)sb.capacity ? (int64_t)handed : sb.capacity;
}

// Pass 1 (SCATTER = false): records per leaf.  Pass 2 (SCATTER = true): each
// record's number to its leaf's range of perm.  Whole warps step together so
// that lanes with the same leaf (neighbouring rays of one step) share one
// atomic, found with a match.
template <bool SCATTER>
__global__ void __launch_bounds__(kBlock) leaf_pass_kernel(const SegBinParams q)
{
    if (q.s.sb.state[1] != 0ull) return;
    const int64_t used = records_used(q.s.sb);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < used; i0 += stride) {
        const int64_t i = i0 + lane;
        const int b = record_leaf(q.s, i, used);
        const unsigned m = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(m) - 1;
        if (!SCATTER) {
            if (b >= 0 && lane == leader) atomicAdd(q.count + b, (unsigned)__popc(m));
        } else {
            unsigned base = 0;
            if (b >= 0 && lane == leader) base = atomicAdd(q.cursor + b, (unsigned)__popc(m));
            base = __shfl_sync(m, base, leader);
            if (b >= 0) q.perm[q.start[b] + base + __popc(m & ((1u << lane) - 1u))] = (unsigned)i;
        }
    }
}

// Exclusive scan of one value per thread over a block of kScanBlock threads;
// *total = the block's sum.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned *total)
{
    __shared__ unsigned warp_sum[kScanBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned w = warp_sum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        warp_sum[lane] = w;
    }
    __syncthreads();
    *total = warp_sum[kScanBlock / 32 - 1];
    return (wid ? warp_sum[wid - 1] : 0u) + incl - v;
}

// Scan step 1: the sum of each tile of kScanTile counts.
__global__ void __launch_bounds__(kScanBlock) scan_tile_sums_kernel(const SegBinParams q)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned v = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u)
        if (base + u < q.n_bins) v += q.count[base + u];
    unsigned total;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) q.tile_sum[blockIdx.x] = total;
}

// Scan step 2 (one block): the tile sums become the tiles' exclusive offsets;
// start[n_bins] = the number of records.
__global__ void __launch_bounds__(kScanBlock) scan_tile_offsets_kernel(const SegBinParams q, int64_t n_tiles)
{
    const int64_t per = (n_tiles + kScanBlock - 1) / kScanBlock;
    const int64_t lo = threadIdx.x * per, hi = min(lo + per, n_tiles);
    unsigned v = 0;
    for (int64_t t = lo; t < hi; ++t) v += q.tile_sum[t];
    unsigned total;
    unsigned run = block_exclusive_scan(v, &total);
    for (int64_t t = lo; t < hi; ++t) {
        const unsigned c = q.tile_sum[t];
        q.tile_sum[t] = run;
        run += c;
    }
    if (threadIdx.x == 0) const_cast<unsigned *>(q.start)[q.n_bins] = total;
}

// Scan step 3: each leaf's first sorted position; cursors cleared.
__global__ void __launch_bounds__(kScanBlock) scan_apply_kernel(const SegBinParams q)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned c[kScanItems], v = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        c[u] = base + u < q.n_bins ? q.count[base + u] : 0u;
        v += c[u];
    }
    unsigned total;
    unsigned run = block_exclusive_scan(v, &total) + q.tile_sum[blockIdx.x];
    unsigned *start = const_cast<unsigned *>(q.start);
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        if (base + u < q.n_bins) {
            start[base + u] = run;
            q.cursor[base + u] = 0u;
        }
        run += c[u];
    }
}

template <typename T>
cudaError_t launch_leaf_order_t(const SegBinParams &q, int K, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // count and scatter passes: a few waves of blocks over the slots (grid-stride)
    int64_t blocks = (q.s.sb.capacity + kBlock - 1) / kBlock;
    if (blocks > 8 * (int64_t)sms) blocks = 8 * (int64_t)sms;
    if (blocks < 1) blocks = 1;
    const int64_t n_tiles = (q.n_bins + kScanTile - 1) / kScanTile;
    leaf_pass_kernel<false><<<(unsigned)blocks, kBlock, 0, s>>>(q);
    scan_tile_sums_kernel<<<(unsigned)n_tiles, kScanBlock, 0, s>>>(q);
    scan_tile_offsets_kernel<<<1, kScanBlock, 0, s>>>(q, n_tiles);
    scan_apply_kernel<<<(unsigned)n_tiles, kScanBlock, 0, s>>>(q);
    leaf_pass_kernel<true><<<(unsigned)blocks, kBlock, 0, s>>>(q);
    count_launch(5);
    // the per-record kernel over the records in leaf order
    SegBackwardParams sq = q.s;
    sq.perm = q.perm;
    sq.n_perm = q.start + q.n_bins;
    return launch_segment_backward_t<T>(sq, K, s);
}

// ---- optimiser step on the leaves ------------------------------------------
struct StepParams {
    int64_t L;
    int K3;      // 3K
    int stride;  // SH record stride (elements)
    float lr_sigma, lr_sh, alpha, beta1, beta2, eps;
    float bc1, bc2;  // Adam bias corrections 1 - beta^t
};

// One parameter's update; m and v are its optimiser state (v unused by SGD,
// m only by Adam).
template <int KIND>
__device__ __forceinline__ float step_one(const StepParams &sp, float x, float g, float lr, float &m, float &v)
{
    if (KIND == POT_SGD) {
        x -= lr * g;
    } else if (KIND == POT_RMSPROP) {
        v = sp.alpha * v + (1.f - sp.alpha) * g * g;
        x -= lr * g / (sqrtf(v) + sp.eps);
    } else {
        m = sp.beta1 * m + (1.f - sp.beta1) * g;
        v = sp.beta2 * v + (1.f - sp.beta2) * g * g;
        x -= (lr / sp.bc1) * m / (sqrtf(v) / sqrtf(sp.bc2) + sp.eps);
    }
    return x;
}

// State of value j (public order: sigma part, then SH part): RMSprop v at
// state[j]; Adam m at state[j], v at state[N + j].
template <int KIND>
__device__ __forceinline__ void load_state(const float *state, int64_t N, int64_t j, float &m, float &v)
{
    if (KIND == POT_RMSPROP) v = state[j];
    if (KIND == POT_ADAM) {
        m = state[j];
        v = state[N + j];
    }
}
template <int KIND>
__device__ __forceinline__ void store_state(float *state, int64_t N, int64_t j, float m, float v)
{
    if (KIND == POT_RMSPROP) state[j] = v;
    if (KIND == POT_ADAM) {
        state[j] = m;
        state[N + j] = v;
    }
}

// FLAT: the SH records have no padding (stride == 3K), so the public
// gradient index is the record index and no division is needed.
template <int KIND, bool FLAT>
__global__ void k_step(StepParams sp, float *sigma, float *sh, const float *gs, const float *gsh, float *state)
{
    const int64_t N = sp.L * (1 + sp.K3);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        float *param;
        float g, lr;
        if (j < sp.L) {
            param = sigma + j;
            g = gs[j];
            lr = sp.lr_sigma;
        } else {
            const int64_t jj = j - sp.L;
            if (FLAT) {
                param = sh + jj;
            } else {
                const int64_t i = jj / sp.K3;
                param = sh + i * sp.stride + (jj - i * sp.K3);
            }
            g = gsh[jj];
            lr = sp.lr_sh;
        }
        float m = 0.f, v = 0.f;
        load_state<KIND>(state, N, j, m, v);
        *param = step_one<KIND>(sp, *param, g, lr, m, v);
        store_state<KIND>(state, N, j, m, v);
    }
}

// The same update with 16-byte accesses for the SH part (unpadded records,
// L a multiple of 4, 16-byte aligned arrays): the step streams ~5 arrays of
// L (1 + 3K) floats and is bound by HBM.
template <int KIND>
__global__ void k_step_vec(StepParams sp, float *sigma, float4 *sh4, const float *gs, const float4 *gsh4,
                           float *state)
{
    const int64_t N = sp.L * (1 + sp.K3);
    const int64_t n4 = sp.L * sp.K3 / 4;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < sp.L + n4;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (j < sp.L) {
            float m = 0.f, v = 0.f;
            load_state<KIND>(state, N, j, m, v);
            sigma[j] = step_one<KIND>(sp, sigma[j], gs[j], sp.lr_sigma, m, v);
            store_state<KIND>(state, N, j, m, v);
        } else {
            const int64_t u = j - sp.L;
            float4 x = sh4[u];
            const float4 g = gsh4[u];
            float4 *m4 = nullptr, *v4 = nullptr;  // Adam m, v / RMSprop v (in m4)
            if (KIND != POT_SGD) m4 = reinterpret_cast<float4 *>(state + sp.L) + u;
            if (KIND == POT_ADAM) v4 = reinterpret_cast<float4 *>(state + N + sp.L) + u;
            float4 m = make_float4(0.f, 0.f, 0.f, 0.f), v = m;
            if (KIND == POT_RMSPROP) v = *m4;
            if (KIND == POT_ADAM) {
                m = *m4;
                v = *v4;
            }
            x.x = step_one<KIND>(sp, x.x, g.x, sp.lr_sh, m.x, v.x);
            x.y = step_one<KIND>(sp, x.y, g.y, sp.lr_sh, m.y, v.y);
            x.z = step_one<KIND>(sp, x.z, g.z, sp.lr_sh, m.z, v.z);
            x.w = step_one<KIND>(sp, x.w, g.w, sp.lr_sh, m.w, v.w);
            sh4[u] = x;
            if (KIND == POT_RMSPROP) *m4 = v;
            if (KIND == POT_ADAM) {
                *m4 = m;
                *v4 = v;
            }
        }
    }
}

// ---- MSE loss of a ray batch: L = mean over n*3 of (rgb - target)^2 --------
__global__ void k_mse(int64_t n3, const float *rgb, const float *target, float *grad, float *loss)
{
    __shared__ float part[kBlock / 32];
    const float scale = 2.f / (float)n3;
    float acc = 0.f;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n3; j += (int64_t)gridDim.x * blockDim.x) {
        const float r = rgb[j] - target[j];
        acc = fmaf(r, r, acc);
        if (grad) grad[j] = scale * r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kBlock / 32; ++w) s += part[w];
        atomicAdd(loss, s / (float)n3);
    }
}

// ---- pixel rays (the camera expression of the public header) ----------------
__global__ void k_camera_rays(const pot_camera *cams, int n_cams, int64_t per_cam, int W, int64_t n,
                              const int64_t *pixels, float *o, float *d)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = pixels ? pixels[k] : k;
        int64_t cam = pix / per_cam;
        if (cam < 0 || cam >= n_cams) cam = cam < 0 ? 0 : n_cams - 1;  // guarded by the host check
        const int64_t rem = pix - cam * per_cam;
        const int j = (int)(rem / W), i = (int)(rem - (int64_t)j * W);
        const pot_camera *c = cams + cam;
        const float xc = __fdiv_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), c->cx), c->fx);
        const float yc = -__fdiv_rn(__fsub_rn(__fadd_rn((float)j, 0.5f), c->cy), c->fy);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            d[3 * k + r] = __fsub_rn(__fadd_rn(__fmul_rn(c->c2w[r][0], xc), __fmul_rn(c->c2w[r][1], yc)),
                                     c->c2w[r][2]);
            o[3 * k + r] = c->c2w[r][3];
        }
    }
}

__global__ void k_pixel_range(int64_t n, const int64_t *pixels, int64_t total, unsigned *flag)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (pixels[k] < 0 || pixels[k] >= total) atomicOr(flag, 1u);
}

unsigned grid_n(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t launch_backward(const RenderParams &r, const float *grad_rgb, const float *rgb_fwd, float *grad_sigma,
                            float *grad_sh, int dtype, int K, cudaStream_t s)
{
    BackwardParams bp{r, grad_rgb, rgb_fwd, grad_sigma, grad_sh, nullptr, nullptr, nullptr, 0.f};
    const int mode = rgb_fwd ? kGradAndColour : kGrad;
    switch (dtype) {
    case POT_F32: return launch_backward_t<float>(bp, K, mode, s);
    case POT_F16: return launch_backward_t<__half>(bp, K, mode, s);
    default: return launch_backward_t<__nv_bfloat16>(bp, K, mode, s);
    }
}

cudaError_t launch_mse_backward(const RenderParams &r, const float *target, float *rgb_out, float *loss,
                                float *grad_sigma, float *grad_sh, int dtype, int K, cudaStream_t s)
{
    BackwardParams bp{r, nullptr, nullptr, grad_sigma, grad_sh, target, loss, rgb_out,
                      2.f / (3.f * (float)r.n_rays)};
    switch (dtype) {
    case POT_F32: return launch_backward_t<float>(bp, K, kMseTarget, s);
    case POT_F16: return launch_backward_t<__half>(bp, K, kMseTarget, s);
    default: return launch_backward_t<__nv_bfloat16>(bp, K, kMseTarget, s);
    }
}

cudaError_t launch_backward_recorded(const RenderParams &r, int64_t n_leaves, const SegmentBuffer &sb,
                                     const SegmentBins *bins, const float *grad_rgb, const float *rgb_fwd,
                                     float *grad_sigma, float *grad_sh, int dtype, int K, cudaStream_t s)
{
    SegBackwardParams q{sb,      r.n_rays,   n_leaves, nullptr,    nullptr,   r.sigma,
                        r.sh,    r.ray_d,    grad_rgb, rgb_fwd,    grad_sigma, grad_sh};
    cudaError_t e;
    if (bins) {
        const SegBinParams bq{q, bins->start, bins->count, bins->cursor, bins->perm, bins->tile_sum, bins->n_bins};
        switch (dtype) {
        case POT_F32: e = launch_leaf_order_t<float>(bq, K, s); break;
        case POT_F16: e = launch_leaf_order_t<__half>(bq, K, s); break;
        case POT_BF16: e = launch_leaf_order_t<__nv_bfloat16>(bq, K, s); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (dtype) {
        case POT_F32: e = launch_segment_backward_t<float>(q, K, s); break;
        case POT_F16: e = launch_segment_backward_t<__half>(q, K, s); break;
        case POT_BF16: e = launch_segment_backward_t<__nv_bfloat16>(q, K, s); break;
        default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    // the fallback: every ray walked again, only if the records overflowed
    BackwardParams bp{r, grad_rgb, rgb_fwd, grad_sigma, grad_sh, nullptr, nullptr, nullptr, 0.f, sb.state + 1};
    switch (dtype) {
    case POT_F32: return launch_backward_t<float>(bp, K, kGradAndColour, s);
    case POT_F16: return launch_backward_t<__half>(bp, K, kGradAndColour, s);
    default: return launch_backward_t<__nv_bfloat16>(bp, K, kGradAndColour, s);
    }
}

cudaError_t launch_step(pot_tree *t, int kind, float lr_sigma, float lr_sh, float alpha, float beta1, float beta2,
                        float eps, int step, const float *gs, const float *gsh, float *state, cudaStream_t s)
{
    StepParams sp;
    sp.L = t->n_leaves;
    sp.K3 = 3 * t->K;
    sp.stride = t->stride;
    sp.lr_sigma = lr_sigma;
    sp.lr_sh = lr_sh;
    sp.alpha = alpha;
    sp.beta1 = beta1;
    sp.beta2 = beta2;
    sp.eps = eps;
    sp.bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
    sp.bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
    if (sp.L == 0) return cudaSuccess;
    const unsigned g = grid_n(sp.L * (1 + sp.K3));
    float *sig = static_cast<float *>(t->sigma);
    float *sh = static_cast<float *>(t->sh);
    const bool flat = sp.stride == sp.K3;
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    const bool vec = flat && sp.L % 4 == 0 && a16(sh) && a16(gsh) && (kind == POT_SGD || a16(state));
    const unsigned gv = grid_n(sp.L + sp.L * sp.K3 / 4);
#define POT_STEP(KIND)                                                                           \
    if (vec) k_step_vec<KIND><<<gv, 256, 0, s>>>(sp, sig, reinterpret_cast<float4 *>(sh), gs,    \
                                                  reinterpret_cast<const float4 *>(gsh), state); \
    else if (flat) k_step<KIND, true><<<g, 256, 0, s>>>(sp, sig, sh, gs, gsh, state);            \
    else k_step<KIND, false><<<g, 256, 0, s>>>(sp, sig, sh, gs, gsh, state);
    if (kind == POT_SGD) {
        POT_STEP(POT_SGD)
    } else if (kind == POT_RMSPROP) {
        POT_STEP(POT_RMSPROP)
    } else {
        POT_STEP(POT_ADAM)
    }
#undef POT_STEP
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mse(int64_t n, const float *rgb, const float *target, float *grad, float *loss, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess || n == 0) return e;
    k_mse<<<grid_n(3 * n), kBlock, 0, s>>>(3 * n, rgb, target, grad, loss);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_camera_rays(const pot_camera *d_cams, int n_cams, int W, int H, int64_t n, const int64_t *pixels,
                               float *o, float *d, unsigned *d_flag, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (pixels) {
        k_pixel_range<<<grid_n(n), 256, 0, s>>>(n, pixels, (int64_t)n_cams * W * H, d_flag);
        count_launch();
    }
    k_camera_rays<<<grid_n(n), 256, 0, s>>>(d_cams, n_cams, (int64_t)W * H, W, n, pixels, o, d);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pot
