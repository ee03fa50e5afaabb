/*
 * pot_segments.h -- recorded ray segments: the training form of the forward
 * and backward pair of libpot.so (App. B.3.2 derivatives, Sec. 3.3 direct
 * octree optimisation).  Conventions (grid, SH, rays, errors, streams) are
 * those of pot.h.
 *
 * pot_render_backward replays every ray's walk through the octree to find
 * its segments again.  The derivative of one segment (App. B.3.2) needs only
 * a few values the forward has at hand when it composites the segment:
 *
 *   leaf i, its length delta_i, the transmittance in front of it
 *   T_i = prod_{k<i} exp(-max(sigma_k,0) delta_k), and the colour composited
 *   in front of it P_i = sum_{k<i} w_k c_k, w_k = T_k (1 - exp(-max(sigma_k,0) delta_k)),
 *
 * together with the ray's composited colour C (background included), its
 * upstream gradient dL/dC and its direction (for the SH basis):
 *
 *   c_i = S(x_i), x_i = sum_k k_{i,k} Y_k(d),  T_{i+1} = T_i exp(-max(sigma_i,0) delta_i)
 *   dL/dk_{i,k} = sum_c dL/dC_c w_i c_{i,c} (1 - c_{i,c}) Y_k
 *   dL/dsigma_i = delta_i sum_c dL/dC_c [ c_{i,c} T_{i+1} - (C_c - P_{i,c} - w_i c_{i,c}) ]   (0 for sigma_i <= 0)
 *
 * so pot_render_rays_record writes one record per composited segment and
 * pot_render_backward_recorded differentiates the records independently of
 * one another (one thread per record), without walking the rays again.  It
 * visits the records sorted by leaf: threads next to each other that hold
 * records of the same leaf sum their terms first, and one of them adds the
 * sum to the leaf's gradient row.
 *
 * Record buffer (caller-owned device memory):
 *   records   capacity x POT_SEGMENT_RECORD_BYTES bytes, 16-byte aligned.  A
 *             record is { int32 ray; int32 leaf; float delta; float T_i;
 *             float P_i[3]; uint32 unused }; ray = -1 marks an unused slot.
 *             The forward hands out slots in blocks of POT_SEGMENT_BLOCK to
 *             each warp, so a ray's records are in compositing order but the
 *             records of different rays interleave, and up to
 *             POT_SEGMENT_BLOCK - 1 slots per resident warp stay unused.
 *   seg_state int64[2], device memory, written by the forward (it clears them
 *             first): [0] slots handed out, [1] nonzero when the records did
 *             not fit in `capacity` (the forward's colours are still exact).
 * Sizing: about (mean leaf segments per ray) x n slots, plus one partly used
 * block of POT_SEGMENT_BLOCK slots per resident warp of the recording kernel
 * (3 blocks of 8 warps per SM: 3,648 warps on a 152-SM GB300); when the
 * records overflow, pot_render_backward_recorded detects it on the GPU and
 * computes the gradients by the walking backward instead (same result, no
 * host synchronisation).  A buffer holds one forward's records: reuse it only
 * after that forward's backward has been issued.
 */
#ifndef POT_SEGMENTS_H
#define POT_SEGMENTS_H

#include "pot.h"

#ifdef __cplusplus
extern "C" {
#endif

#define POT_SEGMENT_RECORD_BYTES 32
#define POT_SEGMENT_BLOCK 128

/* pot_render_rays (Eq. 1, Sec. 3.2 rendering and early stop) that also
 * records every composited leaf segment (see above).  Same arguments and
 * results as pot_render_rays, plus the record buffer; everything in device
 * memory (host arrays give POT_ERR_INVALID_ARG before any launch).
 * n < 2^31; 0 <= capacity < 2^31; opts->seg_count / leaf_touched must be NULL.
 * Asynchronous on `stream`.                                                  */
pot_status pot_render_rays_record(const pot_tree *tree, int64_t n, const float *origins, const float *dirs,
                                  const pot_render_opts *opts, float *rgb, float *t_final, void *records,
                                  int64_t capacity, int64_t *seg_state, pot_stream stream);

/* The gradients of pot_render_backward (App. B.3.2) from the records of the
 * pot_render_rays_record call that rendered the same rays with the same
 * tree values and opts: accumulates (+=) dL/dsigma into grad_sigma [L] and
 * dL/dk into grad_sh [L][K][3] (float32, caller-zeroed; 16-byte aligned when
 * 3K is a multiple of 4, else POT_ERR_INVALID_ARG).  grad_rgb [n][3] is
 * dL/dC; rgb_fwd [n][3] is that call's colour output (background included).
 * origins / dirs are that call's rays (the directions give the SH basis; both
 * are used by the walking backward when the records overflowed).  All device
 * memory.  Launches on `stream`: the sort of the records by leaf (count,
 * scan, scatter), the per-record kernel, then the walking backward; each
 * reads seg_state on the GPU and returns at once when the other one applies.
 * Scratch from the library's pool: 4 bytes per record slot plus about 12
 * bytes per leaf of the tree.  Float atomics make the summation order, and
 * so the last bits of the gradients, vary from call to call (as in
 * pot_render_backward).                                                      */
pot_status pot_render_backward_recorded(const pot_tree *tree, int64_t n, const float *origins, const float *dirs,
                                        const float *grad_rgb, const float *rgb_fwd, const pot_render_opts *opts,
                                        const void *records, int64_t capacity, const int64_t *seg_state,
                                        float *grad_sigma, float *grad_sh, pot_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* POT_SEGMENTS_H */
