// pot_probe.cu -- measurement kernel for the render path's L2 roofline.
//
// The render kernel's leaf reads are served mostly by L2 (neighbouring views
// share leaves there); to state how close it runs to L2 bandwidth, the
// library measures that bandwidth itself with a read-only kernel over an
// L2-resident buffer: every thread streams 16-byte loads that bypass L1
// (ld.global.cg) over the whole buffer `reps` times; the loaded words are
// folded into one value per thread so the loads cannot be dropped.
#include <cstdio>

#include "pot_internal.h"

namespace pot {
namespace {

__global__ void k_l2_read(const uint4 *__restrict__ buf, int64_t n16, int reps, uint32_t *sink)
{
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;  // practically never true; keeps the loads live
}

__global__ void k_fill(uint4 *buf, int64_t n16)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 7), 0x55u, (uint32_t)(i * 2654435761u));
}

}  // namespace
}  // namespace pot

using namespace pot;

extern "C" pot_status pot_probe_l2_read(int64_t bytes, int32_t reps, double *gbs, pot_stream stream)
{
    if (!gbs || bytes < (1 << 20) || bytes > (1ll << 30) || reps < 1 || reps > 10000) {
        set_last_error("pot_probe_l2_read: bytes in [1 MiB, 1 GiB], reps in [1, 10000], gbs not NULL");
        return POT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n16 = bytes / 16;
    int dev = 0, sms = 0;
    uint4 *buf = nullptr;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&buf, (size_t)n16 * 16);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned grid = (unsigned)(sms > 0 ? sms * 8 : 1216);
    if (e == cudaSuccess) {
        k_fill<<<grid, 256, 0, s>>>(buf, n16);
        k_l2_read<<<grid, 256, 0, s>>>(buf, n16, 2, sink);  // warm: the buffer is now in L2
        count_launch(2);
        e = cudaEventRecord(e0, s);
    }
    if (e == cudaSuccess) {
        k_l2_read<<<grid, 256, 0, s>>>(buf, n16, reps, sink);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "pot_probe_l2_read: %s", cudaGetErrorString(e));
        cudaGetLastError();
        set_last_error(msg);
        return POT_ERR_CUDA;
    }
    *gbs = (double)n16 * 16.0 * reps / (ms * 1e-3) / 1e9;
    return POT_OK;
}
