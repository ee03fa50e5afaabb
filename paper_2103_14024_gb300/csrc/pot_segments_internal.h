// pot_segments_internal.h -- launches of the recorded-segment forward and
// backward (pot_record.cu, pot_backward.cu).
#pragma once

#include "../../include/pot_segments.h"
#include "pot_internal.h"

namespace pot {

// One record: { ray, leaf, delta, T_i } and { P_i[3], unused } as two 16-byte halves.
constexpr int kSegBlock = POT_SEGMENT_BLOCK;
static_assert(POT_SEGMENT_RECORD_BYTES == 2 * sizeof(float4), "a record is two float4");

struct SegmentBuffer {
    float4 *rec;                  // [capacity][2]
    int64_t capacity;
    unsigned long long *state;    // [0] slots handed out, [1] overflow
};

// Forward of explicit rays (p.ray_o / p.ray_d, p.n_rays) that records its segments.
cudaError_t launch_render_record(const RenderParams &p, const SegmentBuffer &sb, int dtype, int K, cudaStream_t s);

// Scratch of the per-record backward in leaf order (a counting sort of the
// records by leaf); count zeroed by the caller.
constexpr int kSegScanTile = 4096;  // counts per block of the scan
struct SegmentBins {
    unsigned *count;     // [n_bins]
    unsigned *start;     // [n_bins + 1]
    unsigned *cursor;    // [n_bins]
    unsigned *perm;      // [capacity]
    unsigned *tile_sum;  // [ceil(n_bins / kSegScanTile)]
    int64_t n_bins;      // = the tree's leaves
};

// Gradients from the records, one thread per record with float reductions,
// visiting the records in leaf order (bins) or in slot order (null); then the walking
// backward over all rays, which runs only when the records overflowed (both
// decide on the GPU).
cudaError_t launch_backward_recorded(const RenderParams &r, int64_t n_leaves, const SegmentBuffer &sb,
                                     const SegmentBins *bins, const float *grad_rgb, const float *rgb_fwd,
                                     float *grad_sigma, float *grad_sh, int dtype, int K, cudaStream_t s);

}  // namespace pot
