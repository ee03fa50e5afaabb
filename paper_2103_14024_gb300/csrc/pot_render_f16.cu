// Forward render kernels with __half leaf storage (fp32 arithmetic).
#include "pot_render.cuh"

namespace pot {
cudaError_t launch_render_f16(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                             int max_blocks)
{
    return launch_render_t<__half>(p, K, cams, count, s, max_blocks);
}
}  // namespace pot
