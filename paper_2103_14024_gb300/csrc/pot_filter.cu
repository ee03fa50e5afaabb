// pot_filter.cu -- visibility filtering (Sec. 3.2 "Filtering"): the largest
// ray weight each leaf receives over the pixels of a set of cameras, and the
// leaf compaction used to rebuild a tree from the leaves that pass a threshold.
#include "pot_render.cuh"

namespace pot {

namespace {

// Ray weight w = T (1 - e^{-sigma delta}) of each composited leaf, with the
// forward's transmittance arithmetic and early stop; max kept per leaf
// (non-negative floats order like their bit patterns).
template <typename T>
struct MaxWeightVisitor {
    const T *sig_arr;
    float gamma;
    float Tr;
    float *max_w;
    template <typename YT>
    __device__ __forceinline__ bool operator()(int leaf, float delta, const YT &)
    {
        const float sig = fmaxf(Store<T>::load_sigma(sig_arr, leaf), 0.f);
        const float e = __expf(-sig * delta);
        const float w = Tr * (1.f - e);
        atomicMax(reinterpret_cast<int *>(max_w + leaf), __float_as_int(fmaxf(w, 0.f)));
        Tr *= e;
        return Tr < gamma;
    }
};

template <int K, typename T>
__global__ void __launch_bounds__(kBlock, POT_RENDER_MIN_BLOCKS) visibility_kernel(const RenderParams p, float *max_w)
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
        if (tile_ray<true>(p, tile, lane, o, d, near, far, ray)) {
            MaxWeightVisitor<T> v{sig_arr, p.gamma, 1.f, max_w};
            walk_ray<K, T>(p, sig_arr, sh_arr, stk, ysm, wst, o, d, near, far, v);
        }
    }
}

template <typename T>
cudaError_t launch_visibility_t(const RenderParams &p, int K, float *max_w, cudaStream_t s)
{
    using Fn = void (*)(const RenderParams, float *);
    Fn fn = K == 1 ? visibility_kernel<1, T> : K == 4 ? visibility_kernel<4, T> : K == 9 ? visibility_kernel<9, T>
          : K == 16 ? visibility_kernel<16, T> : K == 25 ? visibility_kernel<25, T> : nullptr;
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = walk_smem_bytes(p.cells == nullptr);
    unsigned grid = 0;
    cudaError_t e = persistent_grid(fn, smem, p.n_tiles, 0, &grid);
    if (e != cudaSuccess) return e;
    fn<<<grid, kBlock, smem, s>>>(p, max_w);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
__device__ __forceinline__ float widen(T x);
template <>
__device__ __forceinline__ float widen<float>(float x)
{
    return x;
}
template <>
__device__ __forceinline__ float widen<__half>(__half x)
{
    return __half2float(x);
}
template <>
__device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 x)
{
    return __bfloat162float(x);
}

__global__ void k_keep_flags(int64_t n, const float *score, float threshold, int *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = score[i] >= threshold ? 1 : 0;
}

template <typename T>
__global__ void k_compact(int64_t n, int K3, int stride, const int *incl, const uint64_t *morton, const T *sigma,
                          const T *sh, uint64_t *codes, float *sig_out, float *sh_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int prev = i > 0 ? incl[i - 1] : 0;
        if (incl[i] == prev) continue;
        codes[prev] = morton[i];
        sig_out[prev] = widen<T>(sigma[i]);
        for (int e = 0; e < K3; ++e) sh_out[(int64_t)prev * K3 + e] = widen<T>(sh[i * stride + e]);
    }
}

unsigned grid_f(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

}  // namespace

cudaError_t scan_inclusive(const int *in, int *out, int64_t n, cudaStream_t s);

cudaError_t launch_visibility(const RenderParams &p, const pot_tree *t, float *max_w, cudaStream_t s)
{
    switch (t->desc.leaf_dtype) {
    case POT_F32: return launch_visibility_t<float>(p, t->K, max_w, s);
    case POT_F16: return launch_visibility_t<__half>(p, t->K, max_w, s);
    case POT_CB16: return launch_visibility_t<cb16>(p, t->K, max_w, s);
    default: return launch_visibility_t<__nv_bfloat16>(p, t->K, max_w, s);
    }
}

cudaError_t compact_kept_leaves(const pot_tree *t, const float *score, float threshold, uint64_t **codes,
                                float **sig_out, float **sh_out, int64_t *n_keep, cudaStream_t s)
{
    const int64_t n = t->n_leaves;
    int *incl = nullptr;
    cudaError_t e = cudaMallocAsync(&incl, sizeof(int) * (n > 0 ? n : 1), s);
    if (e != cudaSuccess) return e;
    int keep = 0;
    if (n > 0) {
        k_keep_flags<<<grid_f(n), 256, 0, s>>>(n, score, threshold, incl);
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = scan_inclusive(incl, incl, n, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&keep, incl + (n - 1), sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    const int K3 = 3 * t->K;
    if (e == cudaSuccess) e = cudaMallocAsync(codes, sizeof(uint64_t) * (keep > 0 ? keep : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(sig_out, sizeof(float) * (keep > 0 ? keep : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(sh_out, sizeof(float) * K3 * (int64_t)(keep > 0 ? keep : 1), s);
    if (e == cudaSuccess && keep > 0) {
        switch (t->desc.leaf_dtype) {
        case POT_F32:
            k_compact<float><<<grid_f(n), 256, 0, s>>>(n, K3, t->stride, incl, t->morton, (const float *)t->sigma,
                                                       (const float *)t->sh, *codes, *sig_out, *sh_out);
            break;
        case POT_F16:
            k_compact<__half><<<grid_f(n), 256, 0, s>>>(n, K3, t->stride, incl, t->morton, (const __half *)t->sigma,
                                                        (const __half *)t->sh, *codes, *sig_out, *sh_out);
            break;
        default:
            k_compact<__nv_bfloat16><<<grid_f(n), 256, 0, s>>>(n, K3, t->stride, incl, t->morton,
                                                               (const __nv_bfloat16 *)t->sigma,
                                                               (const __nv_bfloat16 *)t->sh, *codes, *sig_out,
                                                               *sh_out);
            break;
        }
        count_launch();
        e = cudaGetLastError();
    }
    *n_keep = keep;
    cudaFreeAsync(incl, s);
    return e;
}

}  // namespace pot
