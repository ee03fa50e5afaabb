// Forward render kernels with __nv_bfloat16 leaf storage (fp32 arithmetic).
#include "pot_render.cuh"

namespace pot {
cudaError_t launch_render_bf16(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                             int max_blocks)
{
    return launch_render_t<__nv_bfloat16>(p, K, cams, count, s, max_blocks);
}
}  // namespace pot
