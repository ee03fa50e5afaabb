// Forward render kernels for codebook-quantised leaves (fp32 arithmetic).
#include "pot_render.cuh"

namespace pot {
cudaError_t launch_render_cb16(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                               int max_blocks)
{
    return launch_render_t<cb16>(p, K, cams, count, s, max_blocks);
}
}  // namespace pot
