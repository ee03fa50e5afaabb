// pot_query.cu -- point -> leaf lookups and the SH basis at given directions.
#include "pot_device.cuh"
#include "pot_internal.h"

namespace pot {

namespace {

struct QueryParams {
    const int32_t *child;
    int depth, R;
    float lo[3];
    float h, invh;
};

// Exact voxel membership per axis, then a descent from the root.
__global__ void k_query(QueryParams q, int64_t n, const float *xyz, int32_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int v[3];
        bool outside = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] = voxel_exact(xyz[3 * i + a], q.lo[a], q.h, q.invh, q.R);
            outside |= (v[a] < 0 || v[a] >= q.R);
        }
        if (outside) {
            out[i] = -2;
            continue;
        }
        int32_t node = 0, res = -1;
        for (int l = 0; l < q.depth; ++l) {
            const int b = q.depth - 1 - l;
            const int s = (((v[0] >> b) & 1) << 2) | (((v[1] >> b) & 1) << 1) | ((v[2] >> b) & 1);
            const int32_t c = __ldg(q.child + (int64_t)node * 8 + s);
            if (c > 0 && l < q.depth - 1) {
                node = c;
                continue;
            }
            res = c < 0 ? -c - 1 : -1;
            break;
        }
        out[i] = res;
    }
}

template <int K>
__global__ void k_sh_basis(int64_t n, const float *dirs, float *Y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = dirs[3 * i], y = dirs[3 * i + 1], z = dirs[3 * i + 2];
        const float len = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
        const float il = __frcp_rn(len);
        float v[K];
        sh_basis<K>(x * il, y * il, z * il, v);
#pragma unroll
        for (int k = 0; k < K; ++k) Y[i * K + k] = v[k];
    }
}

unsigned grid1(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > (1 << 20) ? (1 << 20) : b));
}

}  // namespace

cudaError_t launch_query(const pot_tree *t, int64_t n, const float *xyz, int32_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    QueryParams q;
    q.child = t->child;
    q.depth = t->desc.depth;
    q.R = 1 << t->desc.depth;
    for (int a = 0; a < 3; ++a) q.lo[a] = t->desc.bbox_lo[a];
    q.h = t->h;
    q.invh = 1.0f / t->h;
    k_query<<<grid1(n), 256, 0, s>>>(q, n, xyz, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sh_basis(int K, int64_t n, const float *dirs, float *Y, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    switch (K) {
    case 1: k_sh_basis<1><<<grid1(n), 256, 0, s>>>(n, dirs, Y); break;
    case 4: k_sh_basis<4><<<grid1(n), 256, 0, s>>>(n, dirs, Y); break;
    case 9: k_sh_basis<9><<<grid1(n), 256, 0, s>>>(n, dirs, Y); break;
    case 16: k_sh_basis<16><<<grid1(n), 256, 0, s>>>(n, dirs, Y); break;
    case 25: k_sh_basis<25><<<grid1(n), 256, 0, s>>>(n, dirs, Y); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace pot
