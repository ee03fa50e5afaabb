// pot_noalloc.cu -- pot_render_noalloc: the camera render for callers that
// must not allocate GPU memory.
//
// Who needs it: applications that embed this renderer and own every byte of
// GPU memory themselves -- a viewer or engine running against a fixed memory
// budget, or a host process whose allocator hooks reject allocations made by
// third-party libraries -- and frame loops that cannot afford an allocator
// call (a pool growth or an implicit synchronisation) in the middle of a frame.
// pot_render allocates a small stream-ordered scratch buffer on every call
// (the warps' tile counter and a device copy of the cameras); this entry point
// takes that scratch from a fixed array compiled into the library instead.
//
// The array: kNoallocScratchBytes bytes in a file-scope __device__ variable.
// Every GPU that loads the library holds it until the process exits.  It fits
// a 256-byte tile-counter slot and kNoallocMaxCams camera records.
//
// Host code cannot use the array's name as a device address (on the host it is
// only a stand-in symbol), so the first call on each device, with that device
// current, asks the runtime for the array's device address
// (cudaGetSymbolAddress) and caches it; later calls reuse it.  Make that first
// call before any stream capture on that device.
//
// All calls share the one array, and it keeps whatever the last call left in
// it; the tile counter is cleared at the start of every call.  Calls whose
// work overlaps on the GPU (different streams, or another host thread) race on
// the array and may corrupt each other's output: serialise them.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pot_device.cuh"
#include "pot_internal.h"

namespace pot {

constexpr int kNoallocMaxCams = 1024;
constexpr size_t kNoallocCamOffset = 256;
constexpr size_t kNoallocScratchBytes = kNoallocCamOffset + sizeof(pot_camera) * kNoallocMaxCams;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch on the current device (looked up once
// per device), or nullptr with *err set.
static unsigned char *noalloc_scratch_address(cudaError_t *err)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = static_cast<unsigned char *>(p);
    }
    return addr[dev];
}

}  // namespace pot

using namespace pot;

namespace {

pot_status na_fail(pot_status st, const char *msg)
{
    set_last_error(msg);
    return st;
}

pot_status na_cuda(cudaError_t e, const char *where)
{
    cudaGetLastError();
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    set_last_error(buf);
    return POT_ERR_CUDA;
}

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

pot_status pot_render_noalloc(const pot_tree *t, const pot_camera *cams, int32_t n_cams,
                              const pot_render_opts *opts, float *rgb, float *t_final, pot_stream stream)
{
    if (!t) return na_fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n_cams < 0) return na_fail(POT_ERR_INVALID_ARG, "n_cams < 0");
    if (n_cams == 0) return POT_OK;
    if (n_cams > kNoallocMaxCams)
        return na_fail(POT_ERR_INVALID_ARG,
                       "pot_render_noalloc renders at most 1024 cameras per call (its fixed scratch holds "
                       "1024 camera records); split the cameras over several calls");
    if (!cams || !rgb) return na_fail(POT_ERR_INVALID_ARG, "NULL cams or rgb");
    if (on_device(cams)) return na_fail(POT_ERR_INVALID_ARG, "cams must be in host memory");
    if (!on_device(rgb) || (t_final && !on_device(t_final)))
        return na_fail(POT_ERR_INVALID_ARG, "rgb and t_final must be device memory (nothing is staged)");
    if (opts) {
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(opts->bg[c])) return na_fail(POT_ERR_INVALID_ARG, "bg must be finite");
        if (!(opts->gamma >= 0.f) || !std::isfinite(opts->gamma))
            return na_fail(POT_ERR_INVALID_ARG, "gamma must be finite and >= 0");
        if (opts->flags != 0 || opts->max_steps < 0)
            return na_fail(POT_ERR_INVALID_ARG, "opts.flags must be 0 and max_steps >= 0");
        if ((opts->seg_count == nullptr) != (opts->leaf_touched == nullptr))
            return na_fail(POT_ERR_INVALID_ARG, "seg_count and leaf_touched go together");
        // the kernel writes through these: host arrays are refused before any launch
        if (opts->seg_count && (!on_device(opts->seg_count) || !on_device(opts->leaf_touched)))
            return na_fail(POT_ERR_INVALID_ARG, "seg_count / leaf_touched must be device memory");
    }
    const int W = cams[0].width, H = cams[0].height;
    if (W <= 0 || H <= 0 || (int64_t)W * H > (1ll << 31)) return na_fail(POT_ERR_INVALID_ARG, "bad image size");
    for (int c = 0; c < n_cams; ++c) {
        const pot_camera &k = cams[c];
        bool ok = k.width == W && k.height == H && std::isfinite(k.fx) && std::isfinite(k.fy) &&
                  std::isfinite(k.cx) && std::isfinite(k.cy) && k.fx != 0.f && k.fy != 0.f &&
                  !std::isnan(k.near) && !std::isnan(k.far) && k.near >= 0.f;
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 4; ++q) ok = ok && std::isfinite(k.c2w[r][q]);
        if (!ok) return na_fail(POT_ERR_INVALID_ARG, "cameras must share width/height and be finite");
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return na_cuda(cudaGetLastError(), "cudaGetDevice");
    if (prev != t->device && cudaSetDevice(t->device) != cudaSuccess)
        return na_cuda(cudaGetLastError(), "cudaSetDevice");
    struct Restore {
        int dev, prev;
        ~Restore()
        {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{t->device, prev};

    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    unsigned char *scratch = noalloc_scratch_address(&e);
    if (!scratch) return na_cuda(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    unsigned int *err_word = device_error_word();
    if (!err_word) return na_fail(POT_ERR_CUDA, "device error word unavailable");

    // the tile counter must start at zero; the cameras overwrite the last call's
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kNoallocCamOffset, cams, sizeof(pot_camera) * n_cams,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return na_cuda(e, "scratch set-up");

    RenderParams p;
    memset(&p, 0, sizeof(p));
    p.child = t->child;
    p.cells = t->cells;
    p.btab = t->btab;
    p.sigma = t->sigma;
    p.sh = t->sh;
    p.codebook = t->codebook;
    p.depth = t->desc.depth;
    p.R = 1 << t->desc.depth;
    for (int a = 0; a < 3; ++a) p.lo[a] = t->desc.bbox_lo[a];
    p.size = t->desc.bbox_size;
    p.h = t->h;
    p.invh = 1.0f / t->h;
    p.step_cap = 3 * p.R + 16;
    if (opts) {
        for (int c = 0; c < 3; ++c) p.bg[c] = opts->bg[c];
        p.gamma = opts->gamma;
        p.seg_count = opts->seg_count;
        p.leaf_touched = opts->leaf_touched;
        if (opts->max_steps > 0 && opts->max_steps < p.step_cap) p.step_cap = opts->max_steps;
    }
    p.err = err_word;
    p.cams = reinterpret_cast<const pot_camera *>(scratch + kNoallocCamOffset);
    p.W = W;
    p.H = H;
    p.n_cams = n_cams;
    p.view_group = render_view_group(n_cams);
    p.tiles_x = (W + kTileW - 1) / kTileW;
    p.tiles_per_cam = (int64_t)p.tiles_x * ((H + kTileH - 1) / kTileH);
    if (p.tiles_per_cam * ((int64_t)n_cams + 16) >= (1ll << 32))
        return na_fail(POT_ERR_INVALID_ARG, "too many pixels in one call (tiles must stay below 2^32)");
    p.n_tiles = p.tiles_per_cam * n_cams;
    p.rgb = rgb;
    p.t_final = t_final;
    p.tile_counter = reinterpret_cast<unsigned long long *>(scratch);
    const bool count = p.seg_count != nullptr;
    switch (t->desc.leaf_dtype) {
    case POT_F32: e = launch_render_f32(p, t->K, true, count, s, 0); break;
    case POT_F16: e = launch_render_f16(p, t->K, true, count, s, 0); break;
    case POT_CB16: e = launch_render_cb16(p, t->K, true, count, s, 0); break;
    default: e = launch_render_bf16(p, t->K, true, count, s, 0); break;
    }
    if (e != cudaSuccess) return na_cuda(e, "render launch");
    return POT_OK;
}

}  // extern "C"
