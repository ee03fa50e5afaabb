// pot_internal.h -- types shared by the library's host code and kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pot.h"

struct pot_tree {
    int device;
    pot_build_desc desc;
    int K;              // SH coefficients per channel
    int stride;         // elements per padded SH record
    int elem_bytes;     // 4 (f32) or 2 (f16 / bf16)
    int64_t n_nodes;
    int64_t n_leaves;
    float h;            // voxel edge, bbox_size / 2^D (exact)
    int32_t *child;     // [n_nodes][8]
    void *sigma;        // [n_leaves]          leaf dtype
    void *sh;           // [n_leaves][stride]  leaf dtype
    uint64_t *morton;   // [n_leaves]
    int64_t bytes;
    int saturated;
    void *codebook;     // POT_CB16: [K][65536][4] fp16
    int cb_bits;        // POT_CB16: codebook entries used per basis function = 2^cb_bits
    int32_t *cells;     // cell index: dense (cell_index_entries(D) int32) or the brick entries, or null
    int32_t *btab;      // brick index: one code per 4^3 brick (brick_count(D) int32), else null
    int64_t n_bricks;   // brick index: bricks stored entry by entry (those holding a leaf)
    int cell_kind;      // POT_CELLS_NONE / _DENSE / _BRICK
    int64_t index_bytes;
};

#ifndef POT_TILE_W
#define POT_TILE_W 4  // pixels per tile row: a warp renders POT_TILE_W x (32 / POT_TILE_W) pixels
#endif

namespace pot {

constexpr int kTileW = POT_TILE_W;
constexpr int kTileH = 32 / POT_TILE_W;

// Everything a render launch needs; passed by value.
struct RenderParams {
    const int32_t *child;
    const int32_t *cells;  // cell index (dense, or the stored bricks' entries), or null (descend the child array)
    const int32_t *btab;   // brick index: code per 4^3 brick (>= 0: stored brick number), or null (dense)
    const void *sigma;
    const void *sh;
    const void *codebook;  // POT_CB16 trees
    int depth;
    int R;
    float lo[3];
    float size;
    float h;
    float invh;
    float bg[3];
    float gamma;
    int step_cap;
    // ray source: cameras (tiles of kTileW x kTileH pixels) or explicit rays (32 per tile)
    const pot_camera *cams;
    int n_cams;
    int view_group;     // tiles are interleaved over groups of this many consecutive cameras
    int W, H;
    int tiles_x;
    int64_t tiles_per_cam;
    const float *ray_o;
    const float *ray_d;
    int64_t n_rays;
    float near, far;
    int64_t n_tiles;
    // outputs
    float *rgb;
    float *t_final;
    int32_t *seg_count;
    uint8_t *leaf_touched;
    // scratch
    unsigned long long *tile_counter;
    unsigned int *err;
};

// Launches (defined in pot_render_*.cu); return the CUDA error of the launch.
cudaError_t launch_render_f32(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                              int max_blocks);
cudaError_t launch_render_f16(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                              int max_blocks);
cudaError_t launch_render_bf16(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                               int max_blocks);
cudaError_t launch_render_cb16(const RenderParams &p, int K, bool cams, bool count, cudaStream_t s,
                               int max_blocks);

// Build / query / export helpers (pot_build.cu, pot_query.cu).
cudaError_t build_levels_and_children(pot_tree *t, int64_t n, const uint64_t *d_codes, cudaStream_t s,
                                      unsigned int *d_flags, int *status);
cudaError_t validate_sparse(int depth, int64_t n, const uint64_t *d_codes, const float *d_sigma,
                            unsigned int *d_flags, cudaStream_t s);
cudaError_t compact_dense(int depth, float tau, const float *d_sigma, const float *d_sh, int K,
                          uint64_t **d_codes, float **d_sig_out, float **d_sh_out, int64_t *n_out,
                          unsigned int *d_flags, cudaStream_t s);
cudaError_t pack_leaves(pot_tree *t, const float *d_sigma, const float *d_sh, unsigned int *d_flags,
                        cudaStream_t s);
cudaError_t export_leaves(const pot_tree *t, float *d_sigma, float *d_sh, cudaStream_t s);
cudaError_t build_cell_index(pot_tree *t, int kind, cudaStream_t s);  // allocates the index of that kind and fills it
void free_cell_index(pot_tree *t);
cudaError_t export_cell_index(const pot_tree *t, int32_t *out, cudaStream_t s);  // [R][R][R] x-major
cudaError_t launch_query(const pot_tree *t, int64_t n, const float *xyz, int32_t *out, cudaStream_t s);
cudaError_t launch_sh_basis(int K, int64_t n, const float *dirs, float *Y, cudaStream_t s);

cudaError_t launch_backward(const RenderParams &r, const float *grad_rgb, const float *rgb_fwd, float *grad_sigma,
                            float *grad_sh, int dtype, int K, cudaStream_t s);
cudaError_t launch_mse_backward(const RenderParams &r, const float *target, float *rgb_out, float *loss,
                                float *grad_sigma, float *grad_sh, int dtype, int K, cudaStream_t s);
cudaError_t launch_step(pot_tree *t, int kind, float lr_sigma, float lr_sh, float alpha, float beta1, float beta2,
                        float eps, int step, const float *gs, const float *gsh, float *state, cudaStream_t s);
cudaError_t launch_mse(int64_t n, const float *rgb, const float *target, float *grad, float *loss, cudaStream_t s);
cudaError_t launch_camera_rays(const pot_camera *d_cams, int n_cams, int W, int H, int64_t n, const int64_t *pixels,
                               float *o, float *d, unsigned *d_flag, cudaStream_t s);

cudaError_t launch_visibility(const RenderParams &p, const pot_tree *t, float *max_w, cudaStream_t s);
cudaError_t compact_kept_leaves(const pot_tree *t, const float *score, float threshold, uint64_t **codes,
                                float **sig_out, float **sh_out, int64_t *n_keep, cudaStream_t s);
cudaError_t quantize_tree(const pot_tree *t, int bits, pot_tree *q, cudaStream_t s);
cudaError_t launch_render_batch(const pot_render_item *items, int n, cudaStream_t s, unsigned int *err);

// cameras interleaved per tile group in camera renders (POT_VIEW_GROUP overrides)
int render_view_group(int n_cams);

unsigned int *device_error_word();   // per-device word raised by kernels
cudaError_t scratch_pool(cudaMemPool_t *out);  // the library's pool of stream-ordered scratch
void set_last_error(const char *msg); // message returned by pot_last_error on this thread
void count_launch(int n = 1);

}  // namespace pot
