// pot_api.cu -- the C ABI of libpot.so: argument checks, host/device staging,
// error reporting, tree lifetime, and the launches.  Every numeric step runs in
// the kernels of pot_build.cu, pot_query.cu and pot_render_*.cu.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "pot_device.cuh"
#include "pot_internal.h"
#include "pot_segments_internal.h"

namespace pot {

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Raised (bit 0) by a render whose traversal hit its step bound.
__device__ unsigned int g_error_word;

unsigned int *device_error_word()
{
    static std::mutex mu;
    static unsigned int *ptr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<unsigned int *>(p);
    }
    return ptr[dev];
}

int render_view_group(int n_cams)
{
    static int g = [] {
        const char *e = std::getenv("POT_VIEW_GROUP");
        const int v = e ? std::atoi(e) : 16;
        return v >= 1 ? v : 1;
    }();
    return n_cams < g ? (n_cams > 0 ? n_cams : 1) : g;
}

}  // namespace pot

using namespace pot;

namespace {

thread_local char g_msg[512] = "";

pot_status fail(pot_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

pot_status cuda_fail(cudaError_t e, const char *where)
{
    cudaGetLastError();  // clear a sticky launch error of this thread
    return fail(e == cudaErrorMemoryAllocation ? POT_ERR_OOM : POT_ERR_CUDA, "%s: %s (%d)", where,
                cudaGetErrorString(e), (int)e);
}

#define POT_CUDA(call, where)                              \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Stream-ordered scratch of the library comes from a memory pool per device
// that keeps up to 1 GiB of freed memory for the next call; the default pool
// returns freed memory at every synchronisation, so each host-output render
// re-mapped its staging buffers (about 9 ms per 200-view call).
cudaError_t pot::scratch_pool(cudaMemPool_t *out)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = 1ull << 30;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

namespace {

// Stream-ordered temporary device buffer (from the library's scratch pool).
struct Tmp {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~Tmp()
    {
        if (p) cudaFreeAsync(p, s);
    }
    cudaError_t alloc(size_t bytes, cudaStream_t st)
    {
        s = st;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = scratch_pool(&pool);
        if (e != cudaSuccess) return e;
        return cudaMallocFromPoolAsync(&p, bytes > 0 ? bytes : 16, pool, st);
    }
};

// A device view of an input array that may live in host memory.
cudaError_t stage_in(const void *src, size_t bytes, Tmp &tmp, cudaStream_t s, const void **out)
{
    if (!src || is_device_ptr(src)) {
        *out = src;
        return cudaSuccess;
    }
    cudaError_t e = tmp.alloc(bytes, s);
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(tmp.p, src, bytes, cudaMemcpyHostToDevice, s);
    *out = tmp.p;
    return e;
}

// A device destination for an output that may live in host memory; finish()
// copies back and synchronises when needed.
struct Out {
    void *user = nullptr;
    size_t bytes = 0;
    Tmp tmp;
    bool host = false;
    cudaError_t bind(void *dst, size_t n, cudaStream_t s, void **dev)
    {
        user = dst;
        bytes = n;
        host = dst && !is_device_ptr(dst);
        if (!host) {
            *dev = dst;
            return cudaSuccess;
        }
        cudaError_t e = tmp.alloc(n, s);
        *dev = tmp.p;
        return e;
    }
    cudaError_t finish(cudaStream_t s)
    {
        if (!host || !bytes) return cudaSuccess;
        return cudaMemcpyAsync(user, tmp.p, bytes, cudaMemcpyDeviceToHost, s);
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int elem_bytes(int dtype) { return dtype == POT_F32 ? 4 : 2; }

int stride_for(int dtype, int K)
{
    return dtype == POT_F32 ? sh_stride<float>(K) : sh_stride<__half>(K);
}

pot_status check_desc(const pot_build_desc *d, int max_depth)
{
    if (!d) return fail(POT_ERR_INVALID_ARG, "desc is NULL");
    if (d->depth < 1 || d->depth > max_depth)
        return fail(POT_ERR_INVALID_ARG, "depth %d outside 1..%d", d->depth, max_depth);
    if (d->sh_degree < 0 || d->sh_degree > 4)
        return fail(POT_ERR_INVALID_ARG, "sh_degree %d outside 0..4", d->sh_degree);
    if (d->leaf_dtype < POT_F32 || d->leaf_dtype > POT_BF16)
        return fail(POT_ERR_INVALID_ARG, "leaf_dtype %d unknown", d->leaf_dtype);
    if (!(d->bbox_size > 0.f) || !std::isfinite(d->bbox_size))
        return fail(POT_ERR_INVALID_ARG, "bbox_size must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->bbox_lo[a])) return fail(POT_ERR_INVALID_ARG, "bbox_lo must be finite");
    if (!std::isfinite(d->sigma_threshold)) return fail(POT_ERR_INVALID_ARG, "sigma_threshold not finite");
    return POT_OK;
}

pot_tree *new_tree(const pot_build_desc *d, int dev)
{
    pot_tree *t = new (std::nothrow) pot_tree();
    if (!t) return nullptr;
    t->device = dev;
    t->desc = *d;
    t->K = (d->sh_degree + 1) * (d->sh_degree + 1);
    t->stride = stride_for(d->leaf_dtype, t->K);
    t->elem_bytes = elem_bytes(d->leaf_dtype);
    t->h = std::ldexp(d->bbox_size, -d->depth);
    return t;
}

void destroy_tree(pot_tree *t)
{
    if (!t) return;
    DeviceGuard g(t->device);
    cudaDeviceSynchronize();
    cudaFree(t->child);
    cudaFree(t->sigma);
    cudaFree(t->sh);
    cudaFree(t->morton);
    cudaFree(t->codebook);
    free_cell_index(t);
    delete t;
}

// Cell index layout a tree of depth D gets by default: dense up to depth 9
// (537 MB at D = 9; one load per cell), bricks for depths 10 and 11 (the
// dense layout would take 4.3 GB at D = 10 and cannot be built beyond).
int default_cell_kind(int D)
{
    if (D <= kDenseDefaultMaxDepth) return POT_CELLS_DENSE;
    if (D >= kBrickIndexMinDepth && D <= kBrickIndexMaxDepth) return POT_CELLS_BRICK;
    return POT_CELLS_NONE;
}

// Gives a new tree its default cell index.  A device too full for it leaves
// the tree without one (cells are then found by descending the child array);
// any other failure is returned.
cudaError_t attach_cell_index(pot_tree *t, cudaStream_t s)
{
    const int kind = default_cell_kind(t->desc.depth);
    if (kind == POT_CELLS_NONE) return cudaSuccess;
    cudaError_t e = build_cell_index(t, kind, s);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) t->bytes += t->index_bytes;
    return e;
}

// Shared tail of both builds: codes, sigma, sh are device arrays of n kept voxels.
pot_status finish_build(const pot_build_desc *desc, int64_t n, const uint64_t *d_codes,
                        const float *d_sigma, const float *d_sh, unsigned *d_flags, pot_tree **out,
                        cudaStream_t s)
{
    int dev = 0;
    POT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    pot_tree *t = new_tree(desc, dev);
    if (!t) return fail(POT_ERR_OOM, "host allocation failed");
    t->n_leaves = n;
    cudaError_t e = cudaMalloc(&t->morton, sizeof(uint64_t) * (n > 0 ? n : 1));
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(t->morton, d_codes, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    int status = 0;
    if (e == cudaSuccess) e = build_levels_and_children(t, n, d_codes, s, d_flags, &status);
    if (e == cudaSuccess && status == 0) e = pack_leaves(t, d_sigma, d_sh, d_flags, s);
    unsigned flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        destroy_tree(t);
        return cuda_fail(e, "pot_build");
    }
    if (status != 0) {
        destroy_tree(t);
        return fail(POT_ERR_UNSUPPORTED, "tree too large (%d)", status);
    }
    t->saturated = (flags & 4u) ? 1 : 0;
    t->bytes = t->n_nodes * 32 + n * 8 + ((n * t->elem_bytes + 255) / 256) * 256 +
               n * (int64_t)t->stride * t->elem_bytes;
    e = attach_cell_index(t, s);
    if (e != cudaSuccess) {
        destroy_tree(t);
        return cuda_fail(e, "cell index");
    }
    *out = t;
    return POT_OK;
}

pot_status tile_limit_error()
{
    return fail(POT_ERR_INVALID_ARG, "too many pixels in one call (tiles must stay below 2^32): split the cameras");
}

pot_status check_opts(const pot_render_opts *o)
{
    if (!o) return POT_OK;
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(o->bg[c])) return fail(POT_ERR_INVALID_ARG, "bg must be finite");
    if (!(o->gamma >= 0.f) || !std::isfinite(o->gamma))
        return fail(POT_ERR_INVALID_ARG, "gamma must be finite and >= 0");
    if (o->flags != 0) return fail(POT_ERR_INVALID_ARG, "opts.flags must be 0");
    if (o->max_steps < 0) return fail(POT_ERR_INVALID_ARG, "max_steps < 0");
    if ((o->seg_count == nullptr) != (o->leaf_touched == nullptr))
        return fail(POT_ERR_INVALID_ARG, "seg_count and leaf_touched go together");
    if (o->seg_count && (!is_device_ptr(o->seg_count) || !is_device_ptr(o->leaf_touched)))
        return fail(POT_ERR_INVALID_ARG, "seg_count / leaf_touched must be device memory");
    return POT_OK;
}

// The gradient kernels add whole 16-byte vectors to grad_sh rows when a row
// (3K floats) is a multiple of 4 floats.
bool grad_sh_aligned(const pot_tree *t, const float *grad_sh)
{
    return (3 * t->K) % 4 != 0 || ((uintptr_t)grad_sh & 15u) == 0;
}

void fill_tree_params(RenderParams &p, const pot_tree *t, const pot_render_opts *o)
{
    std::memset(&p, 0, sizeof(p));
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
    if (o) {
        for (int c = 0; c < 3; ++c) p.bg[c] = o->bg[c];
        p.gamma = o->gamma;
        p.seg_count = o->seg_count;
        p.leaf_touched = o->leaf_touched;
        if (o->max_steps > 0 && o->max_steps < p.step_cap) p.step_cap = o->max_steps;
    }
    p.err = device_error_word();
}

cudaError_t launch_render(const RenderParams &p, const pot_tree *t, bool cams, cudaStream_t s)
{
    const bool count = p.seg_count != nullptr;
    switch (t->desc.leaf_dtype) {
    case POT_F32: return launch_render_f32(p, t->K, cams, count, s, 0);
    case POT_F16: return launch_render_f16(p, t->K, cams, count, s, 0);
    case POT_CB16: return launch_render_cb16(p, t->K, cams, count, s, 0);
    default: return launch_render_bf16(p, t->K, cams, count, s, 0);
    }
}

// Per-device stream for device->host copies that overlap rendering.
// Library-owned streams per device: 0 = copies of host outputs, 1 = second
// render stream of host-output renders.
cudaError_t aux_stream(int which, cudaStream_t *out)
{
    static std::mutex mu;
    static cudaStream_t st[2][64] = {{nullptr}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!st[which][dev]) {
        e = cudaStreamCreateWithFlags(&st[which][dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *out = st[which][dev];
    return cudaSuccess;
}

// Camera render into host memory: the cameras are rendered in chunks (one view
// group each) into two device staging buffers; the copy of chunk c to the host
// runs on a second stream while chunk c + 1 renders.  Returns after the last
// copy has completed.  p.tile_counter points at one zeroed counter per chunk.
pot_status render_to_host(RenderParams p, const pot_tree *t, const pot_camera *d_cams, int n_cams, float *rgb,
                          float *t_final, cudaStream_t s)
{
    // view groups render alternately on s and a second stream (so one group's
    // last tiles overlap the next group's first) into two staging buffers,
    // whose copies to the host run on a copy stream while later groups render
    const int64_t per_cam = (int64_t)p.W * p.H;
    const int chunk = render_view_group(n_cams);
    const int n_chunks = (n_cams + chunk - 1) / chunk;
    const bool rgb_dev = is_device_ptr(rgb);
    const bool tf_dev = t_final && is_device_ptr(t_final);
    cudaStream_t cs, rs[2];
    POT_CUDA(aux_stream(0, &cs), "copy stream");
    POT_CUDA(aux_stream(1, &rs[1]), "render stream");
    rs[0] = s;
    Tmp stage[2], stage_tf[2];
    cudaEvent_t rendered[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr}, start = nullptr;
    struct Events {
        cudaEvent_t *a, *b, *c;
        ~Events()
        {
            for (int i = 0; i < 2; ++i) {
                if (a[i]) cudaEventDestroy(a[i]);
                if (b[i]) cudaEventDestroy(b[i]);
            }
            if (*c) cudaEventDestroy(*c);
        }
    } guard{rendered, copied, &start};
    for (int i = 0; i < 2; ++i) {
        POT_CUDA(cudaEventCreateWithFlags(&rendered[i], cudaEventDisableTiming), "event");
        POT_CUDA(cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming), "event");
        if (!rgb_dev) POT_CUDA(stage[i].alloc(sizeof(float) * 3 * per_cam * chunk, s), "alloc stage");
        if (t_final && !tf_dev) POT_CUDA(stage_tf[i].alloc(sizeof(float) * per_cam * chunk, s), "alloc stage");
    }
    // the second render stream starts after everything queued on s so far
    // (tile counters, cameras, staging allocations)
    POT_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming), "event");
    POT_CUDA(cudaEventRecord(start, s), "record");
    POT_CUDA(cudaStreamWaitEvent(rs[1], start, 0), "wait start");
    for (int c = 0; c < n_chunks; ++c) {
        const int b = c & 1;
        const int c0 = c * chunk, nc = std::min(chunk, n_cams - c0);
        if (c >= 2) POT_CUDA(cudaStreamWaitEvent(rs[b], copied[b], 0), "wait copy");
        RenderParams q = p;
        q.cams = d_cams + c0;
        q.n_cams = nc;
        q.view_group = nc;
        q.n_tiles = p.tiles_per_cam * nc;
        q.rgb = rgb_dev ? rgb + 3 * per_cam * c0 : static_cast<float *>(stage[b].p);
        q.t_final = !t_final ? nullptr : (tf_dev ? t_final + per_cam * c0 : static_cast<float *>(stage_tf[b].p));
        q.tile_counter = p.tile_counter + c;
        POT_CUDA(launch_render(q, t, true, rs[b]), "render");
        POT_CUDA(cudaEventRecord(rendered[b], rs[b]), "record");
        POT_CUDA(cudaStreamWaitEvent(cs, rendered[b], 0), "wait render");
        if (!rgb_dev)
            POT_CUDA(cudaMemcpyAsync(rgb + 3 * per_cam * c0, stage[b].p, sizeof(float) * 3 * per_cam * nc,
                                     cudaMemcpyDeviceToHost, cs),
                     "copy rgb");
        if (t_final && !tf_dev)
            POT_CUDA(cudaMemcpyAsync(t_final + per_cam * c0, stage_tf[b].p, sizeof(float) * per_cam * nc,
                                     cudaMemcpyDeviceToHost, cs),
                     "copy t_final");
        POT_CUDA(cudaEventRecord(copied[b], cs), "record");
    }
    // the staging buffers are released on s: make s wait for the last copies
    // (which follow every render of both streams)
    for (int b = 0; b < 2 && b < n_chunks; ++b) POT_CUDA(cudaStreamWaitEvent(s, copied[b], 0), "wait copy");
    POT_CUDA(cudaStreamSynchronize(s), "sync");
    return POT_OK;
}

}  // namespace

void pot::set_last_error(const char *msg) { snprintf(g_msg, sizeof(g_msg), "%s", msg); }

extern "C" {

int32_t pot_version(void) { return 1; }

const char *pot_last_error(void) { return g_msg; }

int64_t pot_launch_count(void) { return g_launches.load(); }

pot_status pot_build_sparse(const pot_build_desc *desc, int64_t n, const uint64_t *morton,
                            const float *sigma, const float *sh, pot_tree **out, pot_stream stream)
{
    pot_status st = check_desc(desc, 12);
    if (st != POT_OK) return st;
    if (!out) return fail(POT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > 0x7FFFFFFE) return fail(POT_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
    if (n > 0 && (!morton || !sigma || !sh)) return fail(POT_ERR_INVALID_ARG, "NULL input array");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = (desc->sh_degree + 1) * (desc->sh_degree + 1);
    Tmp tm, ts, th, tf;
    const void *dm, *ds, *dh;
    POT_CUDA(stage_in(morton, sizeof(uint64_t) * n, tm, s, &dm), "stage morton");
    POT_CUDA(stage_in(sigma, sizeof(float) * n, ts, s, &ds), "stage sigma");
    POT_CUDA(stage_in(sh, sizeof(float) * 3 * K * n, th, s, &dh), "stage sh");
    POT_CUDA(tf.alloc(sizeof(unsigned), s), "alloc flags");
    POT_CUDA(cudaMemsetAsync(tf.p, 0, sizeof(unsigned), s), "memset");
    unsigned *d_flags = static_cast<unsigned *>(tf.p);
    POT_CUDA(validate_sparse(desc->depth, n, (const uint64_t *)dm, (const float *)ds, d_flags, s),
             "validate");
    unsigned flags = 0;
    POT_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy flags");
    POT_CUDA(cudaStreamSynchronize(s), "sync");
    if (flags & 1u)
        return fail(POT_ERR_INVALID_ARG, "morton codes must be strictly increasing and < 8^depth");
    if (flags & 2u) return fail(POT_ERR_INVALID_ARG, "sigma contains NaN or Inf");
    return finish_build(desc, n, (const uint64_t *)dm, (const float *)ds, (const float *)dh, d_flags, out, s);
}

pot_status pot_build(const pot_build_desc *desc, const float *sigma, const float *sh, pot_tree **out,
                     pot_stream stream)
{
    pot_status st = check_desc(desc, 10);
    if (st != POT_OK) return st;
    if (!out) return fail(POT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!sigma || !sh) return fail(POT_ERR_INVALID_ARG, "NULL input array");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = (desc->sh_degree + 1) * (desc->sh_degree + 1);
    const int64_t vox = 1ll << (3 * desc->depth);
    Tmp ts, th, tf;
    const void *ds, *dh;
    POT_CUDA(stage_in(sigma, sizeof(float) * vox, ts, s, &ds), "stage sigma");
    POT_CUDA(stage_in(sh, sizeof(float) * 3 * K * vox, th, s, &dh), "stage sh");
    POT_CUDA(tf.alloc(sizeof(unsigned), s), "alloc flags");
    POT_CUDA(cudaMemsetAsync(tf.p, 0, sizeof(unsigned), s), "memset");
    unsigned *d_flags = static_cast<unsigned *>(tf.p);
    uint64_t *codes = nullptr;
    float *csig = nullptr, *csh = nullptr;
    int64_t n = 0;
    cudaError_t e = compact_dense(desc->depth, desc->sigma_threshold, (const float *)ds, (const float *)dh,
                                  K, &codes, &csig, &csh, &n, d_flags, s);
    Tmp fc, fs, fh;  // released after the build
    fc.p = codes;
    fc.s = s;
    fs.p = csig;
    fs.s = s;
    fh.p = csh;
    fh.s = s;
    if (e != cudaSuccess) return cuda_fail(e, "compact");
    unsigned flags = 0;
    POT_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy flags");
    POT_CUDA(cudaStreamSynchronize(s), "sync");
    if (flags & 2u) return fail(POT_ERR_INVALID_ARG, "sigma contains NaN or Inf");
    return finish_build(desc, n, codes, csig, csh, d_flags, out, s);
}

pot_status pot_tree_get_info(const pot_tree *t, pot_tree_info *info)
{
    if (!t || !info) return fail(POT_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->depth = t->desc.depth;
    info->sh_degree = t->desc.sh_degree;
    info->sh_dim = t->K;
    info->leaf_dtype = t->desc.leaf_dtype;
    info->n_nodes = t->n_nodes;
    info->n_leaves = t->n_leaves;
    info->bytes = t->bytes;
    // cb16: float32 sigma + uint16 codes
    info->leaf_bytes = t->desc.leaf_dtype == POT_CB16 ? 4 + 2 * (int64_t)t->stride
                                                       : (int64_t)t->elem_bytes * (1 + t->stride);
    for (int a = 0; a < 3; ++a) info->bbox_lo[a] = t->desc.bbox_lo[a];
    info->bbox_size = t->desc.bbox_size;
    info->saturated = t->saturated;
    info->index_bytes = t->index_bytes;
    info->index_kind = t->cell_kind;
    info->device = t->device;
    return POT_OK;
}

pot_status pot_tree_export(const pot_tree *t, int32_t *child, float *sigma, float *sh, uint64_t *morton,
                           pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->n_leaves;
    if (child)
        POT_CUDA(cudaMemcpyAsync(child, t->child, sizeof(int32_t) * 8 * t->n_nodes, cudaMemcpyDefault, s),
                 "export child");
    if (morton && n)
        POT_CUDA(cudaMemcpyAsync(morton, t->morton, sizeof(uint64_t) * n, cudaMemcpyDefault, s),
                 "export morton");
    Out os, oh;
    void *dsig = nullptr, *dsh = nullptr;
    POT_CUDA(os.bind(sigma, sizeof(float) * n, s, &dsig), "bind sigma");
    POT_CUDA(oh.bind(sh, sizeof(float) * 3 * t->K * n, s, &dsh), "bind sh");
    POT_CUDA(export_leaves(t, (float *)dsig, (float *)dsh, s), "export leaves");
    POT_CUDA(os.finish(s), "copy sigma");
    POT_CUDA(oh.finish(s), "copy sh");
    POT_CUDA(cudaStreamSynchronize(s), "sync");
    return POT_OK;
}

pot_status pot_tree_set_values(pot_tree *t, const float *sigma, const float *sh, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (t->n_leaves == 0) return POT_OK;
    if (!sigma || !sh) return fail(POT_ERR_INVALID_ARG, "NULL input array");
    if (t->desc.leaf_dtype == POT_CB16) return fail(POT_ERR_UNSUPPORTED, "codebook leaves are read-only");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->n_leaves;
    Tmp ts, th, tf;
    const void *ds, *dh;
    POT_CUDA(stage_in(sigma, sizeof(float) * n, ts, s, &ds), "stage sigma");
    POT_CUDA(stage_in(sh, sizeof(float) * 3 * t->K * n, th, s, &dh), "stage sh");
    POT_CUDA(tf.alloc(sizeof(unsigned), s), "alloc flags");
    POT_CUDA(cudaMemsetAsync(tf.p, 0, sizeof(unsigned), s), "memset");
    POT_CUDA(pack_leaves(t, (const float *)ds, (const float *)dh, (unsigned *)tf.p, s), "pack");
    unsigned flags = 0;
    POT_CUDA(cudaMemcpyAsync(&flags, tf.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy flags");
    POT_CUDA(cudaStreamSynchronize(s), "sync");
    if (flags & 4u) t->saturated = 1;
    return POT_OK;
}

pot_status pot_tree_free(pot_tree *t)
{
    destroy_tree(t);
    return POT_OK;
}

pot_status pot_tree_export_cell_index(const pot_tree *t, int32_t *out, pot_stream stream)
{
    if (!t || !out) return fail(POT_ERR_INVALID_ARG, "NULL tree or out");
    if (!t->cells) return fail(POT_ERR_INVALID_ARG, "tree has no cell index");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Out oo;
    void *dout;
    POT_CUDA(oo.bind(out, sizeof(int32_t) * ((size_t)1 << (3 * t->desc.depth)), s, &dout), "bind out");
    POT_CUDA(export_cell_index(t, static_cast<int32_t *>(dout), s), "export cell index");
    POT_CUDA(oo.finish(s), "copy out");
    if (oo.host) POT_CUDA(cudaStreamSynchronize(s), "sync");
    return POT_OK;
}

pot_status pot_tree_set_cell_index(pot_tree *t, int32_t enable, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (enable < 0 || enable > 3) return fail(POT_ERR_INVALID_ARG, "enable must be 0, 1, 2 or 3");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int D = t->desc.depth;
    const int kind = enable == 1 ? default_cell_kind(D) : enable;
    if (enable == 1 && kind == POT_CELLS_NONE)
        return fail(POT_ERR_UNSUPPORTED, "no cell index for depth %d", D);
    if (kind == t->cell_kind) return POT_OK;
    if (kind == POT_CELLS_DENSE && D > kCellIndexMaxDepth)
        return fail(POT_ERR_UNSUPPORTED, "no dense cell index for depth %d (at most %d)", D, kCellIndexMaxDepth);
    if (kind == POT_CELLS_BRICK && (D < kBrickIndexMinDepth || D > kBrickIndexMaxDepth))
        return fail(POT_ERR_UNSUPPORTED, "no brick cell index for depth %d (%d..%d)", D, kBrickIndexMinDepth,
                    kBrickIndexMaxDepth);
    if (t->cell_kind != POT_CELLS_NONE) {
        POT_CUDA(cudaDeviceSynchronize(), "sync");
        t->bytes -= t->index_bytes;
        free_cell_index(t);
    }
    if (kind == POT_CELLS_NONE) return POT_OK;
    cudaError_t e = build_cell_index(t, kind, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(POT_ERR_OOM, "cell index: device full");
    }
    POT_CUDA(e, "cell index");
    t->bytes += t->index_bytes;
    return POT_OK;
}

pot_status pot_query(const pot_tree *t, int64_t n, const float *xyz, int32_t *leaf_out, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return fail(POT_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return POT_OK;
    if (!xyz || !leaf_out) return fail(POT_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Tmp tx;
    const void *dx;
    POT_CUDA(stage_in(xyz, sizeof(float) * 3 * n, tx, s, &dx), "stage xyz");
    Out oo;
    void *dout;
    POT_CUDA(oo.bind(leaf_out, sizeof(int32_t) * n, s, &dout), "bind out");
    POT_CUDA(launch_query(t, n, (const float *)dx, (int32_t *)dout, s), "query");
    POT_CUDA(oo.finish(s), "copy out");
    if (oo.host) POT_CUDA(cudaStreamSynchronize(s), "sync");
    return POT_OK;
}

pot_status pot_sh_basis(int32_t K, int64_t n, const float *dirs, float *Y, pot_stream stream)
{
    if (K != 1 && K != 4 && K != 9 && K != 16 && K != 25)
        return fail(POT_ERR_INVALID_ARG, "K must be 1, 4, 9, 16 or 25");
    if (n < 0) return fail(POT_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return POT_OK;
    if (!dirs || !Y) return fail(POT_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    Tmp td;
    const void *dd;
    POT_CUDA(stage_in(dirs, sizeof(float) * 3 * n, td, s, &dd), "stage dirs");
    Out oy;
    void *dy;
    POT_CUDA(oy.bind(Y, sizeof(float) * K * n, s, &dy), "bind Y");
    POT_CUDA(launch_sh_basis(K, n, (const float *)dd, (float *)dy, s), "sh_basis");
    POT_CUDA(oy.finish(s), "copy Y");
    if (oy.host) POT_CUDA(cudaStreamSynchronize(s), "sync");
    return POT_OK;
}

pot_status pot_render(const pot_tree *t, const pot_camera *cams, int32_t n_cams, const pot_render_opts *opts,
                      float *rgb, float *t_final, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n_cams < 0) return fail(POT_ERR_INVALID_ARG, "n_cams < 0");
    if (n_cams == 0) return POT_OK;
    if (!cams || !rgb) return fail(POT_ERR_INVALID_ARG, "NULL cams or rgb");
    if (is_device_ptr(cams)) return fail(POT_ERR_INVALID_ARG, "cams must be in host memory");
    pot_status st = check_opts(opts);
    if (st != POT_OK) return st;
    const int W = cams[0].width, H = cams[0].height;
    if (W <= 0 || H <= 0 || (int64_t)W * H > (1ll << 31))
        return fail(POT_ERR_INVALID_ARG, "bad image size %dx%d", W, H);
    for (int c = 0; c < n_cams; ++c) {
        const pot_camera &k = cams[c];
        if (k.width != W || k.height != H)
            return fail(POT_ERR_INVALID_ARG, "all cameras of one call must share width and height");
        bool ok = std::isfinite(k.fx) && std::isfinite(k.fy) && std::isfinite(k.cx) && std::isfinite(k.cy) &&
                  k.fx != 0.f && k.fy != 0.f && !std::isnan(k.near) && !std::isnan(k.far) && k.near >= 0.f;
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 4; ++q) ok = ok && std::isfinite(k.c2w[r][q]);
        if (!ok) return fail(POT_ERR_INVALID_ARG, "camera %d has non-finite or invalid parameters", c);
    }
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npix = (int64_t)n_cams * W * H;
    Tmp scratch;
    // tile counters (one per launch: a host-memory output renders in chunks), then the cameras
    const size_t cam_off = ((sizeof(unsigned long long) * (size_t)(n_cams + 1) + 255) / 256) * 256;
    POT_CUDA(scratch.alloc(cam_off + sizeof(pot_camera) * n_cams, s), "alloc scratch");
    char *sp = static_cast<char *>(scratch.p);
    POT_CUDA(cudaMemsetAsync(sp, 0, cam_off, s), "memset");
    POT_CUDA(cudaMemcpyAsync(sp + cam_off, cams, sizeof(pot_camera) * n_cams, cudaMemcpyHostToDevice, s),
             "copy cams");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.W = W;
    p.H = H;
    p.tiles_x = (W + kTileW - 1) / kTileW;
    p.tiles_per_cam = (int64_t)p.tiles_x * ((H + kTileH - 1) / kTileH);
    if (p.tiles_per_cam * ((int64_t)n_cams + 16) >= (1ll << 32))
        return tile_limit_error();
    p.tile_counter = reinterpret_cast<unsigned long long *>(sp);
    const pot_camera *d_cams = reinterpret_cast<const pot_camera *>(sp + cam_off);
    const bool host_out = !is_device_ptr(rgb) || (t_final && !is_device_ptr(t_final));
    if (host_out) return render_to_host(p, t, d_cams, n_cams, rgb, t_final, s);
    p.cams = d_cams;
    p.n_cams = n_cams;
    p.view_group = render_view_group(n_cams);
    p.n_tiles = p.tiles_per_cam * n_cams;
    p.rgb = rgb;
    p.t_final = t_final;
    POT_CUDA(launch_render(p, t, true, s), "render");
    (void)npix;
    return POT_OK;
}

pot_status pot_render_rays(const pot_tree *t, int64_t n, const float *origins, const float *dirs,
                           const pot_render_opts *opts, float *rgb, float *t_final, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return fail(POT_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return POT_OK;
    if (!origins || !dirs || !rgb) return fail(POT_ERR_INVALID_ARG, "NULL array");
    pot_status st = check_opts(opts);
    if (st != POT_OK) return st;
    const float near = opts ? opts->near : 0.f, far = opts ? opts->far : 3.0e38f;
    if (!(near >= 0.f) || std::isnan(far)) return fail(POT_ERR_INVALID_ARG, "bad near / far");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Tmp to, td, scratch;
    const void *dor, *ddr;
    POT_CUDA(stage_in(origins, sizeof(float) * 3 * n, to, s, &dor), "stage origins");
    POT_CUDA(stage_in(dirs, sizeof(float) * 3 * n, td, s, &ddr), "stage dirs");
    POT_CUDA(scratch.alloc(sizeof(unsigned long long), s), "alloc scratch");
    POT_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(unsigned long long), s), "memset");
    Out orgb, otf;
    void *drgb, *dtf = nullptr;
    POT_CUDA(orgb.bind(rgb, sizeof(float) * 3 * n, s, &drgb), "bind rgb");
    if (t_final) POT_CUDA(otf.bind(t_final, sizeof(float) * n, s, &dtf), "bind t_final");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.ray_o = (const float *)dor;
    p.ray_d = (const float *)ddr;
    p.n_rays = n;
    p.near = near;
    p.far = far;
    p.n_tiles = (n + 31) / 32;
    p.rgb = (float *)drgb;
    p.t_final = (float *)dtf;
    p.tile_counter = static_cast<unsigned long long *>(scratch.p);
    POT_CUDA(launch_render(p, t, false, s), "render_rays");
    POT_CUDA(orgb.finish(s), "copy rgb");
    POT_CUDA(otf.finish(s), "copy t_final");
    if (orgb.host || otf.host) POT_CUDA(cudaStreamSynchronize(s), "sync");
    return POT_OK;
}

pot_status pot_visibility(const pot_tree *t, const pot_camera *cams, int32_t n_cams, const pot_render_opts *opts,
                          float *max_weight, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n_cams < 0) return fail(POT_ERR_INVALID_ARG, "n_cams < 0");
    if (n_cams == 0 || t->n_leaves == 0) return POT_OK;
    if (!cams || !max_weight) return fail(POT_ERR_INVALID_ARG, "NULL cams or max_weight");
    if (is_device_ptr(cams)) return fail(POT_ERR_INVALID_ARG, "cams must be in host memory");
    if (!is_device_ptr(max_weight)) return fail(POT_ERR_INVALID_ARG, "max_weight must be device memory");
    pot_status st = check_opts(opts);
    if (st != POT_OK) return st;
    if (opts && opts->seg_count) return fail(POT_ERR_INVALID_ARG, "counting outputs are not used here");
    const int W = cams[0].width, H = cams[0].height;
    for (int c = 0; c < n_cams; ++c)
        if (cams[c].width != W || cams[c].height != H || W <= 0 || H <= 0 || !(cams[c].near >= 0.f) ||
            !std::isfinite(cams[c].fx) || !std::isfinite(cams[c].fy) || cams[c].fx == 0.f || cams[c].fy == 0.f)
            return fail(POT_ERR_INVALID_ARG, "camera %d invalid or of another size", c);
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Tmp scratch;
    const size_t cam_off = 256;
    POT_CUDA(scratch.alloc(cam_off + sizeof(pot_camera) * n_cams, s), "alloc scratch");
    char *sp = static_cast<char *>(scratch.p);
    POT_CUDA(cudaMemsetAsync(sp, 0, cam_off, s), "memset");
    POT_CUDA(cudaMemcpyAsync(sp + cam_off, cams, sizeof(pot_camera) * n_cams, cudaMemcpyHostToDevice, s), "copy cams");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.cams = reinterpret_cast<const pot_camera *>(sp + cam_off);
    p.n_cams = n_cams;
    p.view_group = render_view_group(n_cams);
    p.W = W;
    p.H = H;
    p.tiles_x = (W + kTileW - 1) / kTileW;
    p.tiles_per_cam = (int64_t)p.tiles_x * ((H + kTileH - 1) / kTileH);
    if (p.tiles_per_cam * ((int64_t)n_cams + 16) >= (1ll << 32))
        return tile_limit_error();
    p.n_tiles = p.tiles_per_cam * n_cams;
    p.tile_counter = reinterpret_cast<unsigned long long *>(sp);
    POT_CUDA(launch_visibility(p, t, max_weight, s), "visibility");
    return POT_OK;
}

pot_status pot_tree_prune(const pot_tree *t, const float *score, float threshold, pot_tree **out, pot_stream stream)
{
    if (!t || !out) return fail(POT_ERR_INVALID_ARG, "NULL tree or out");
    *out = nullptr;
    if (std::isnan(threshold)) return fail(POT_ERR_INVALID_ARG, "threshold is NaN");
    if (t->n_leaves > 0 && (!score || !is_device_ptr(score)))
        return fail(POT_ERR_INVALID_ARG, "score must be device memory");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *codes = nullptr;
    float *sig = nullptr, *sh = nullptr;
    int64_t n = 0;
    cudaError_t e = compact_kept_leaves(t, score, threshold, &codes, &sig, &sh, &n, s);
    Tmp fc, fs, fh, tf;
    fc.p = codes;
    fc.s = s;
    fs.p = sig;
    fs.s = s;
    fh.p = sh;
    fh.s = s;
    if (e != cudaSuccess) return cuda_fail(e, "prune");
    POT_CUDA(tf.alloc(sizeof(unsigned), s), "alloc flags");
    POT_CUDA(cudaMemsetAsync(tf.p, 0, sizeof(unsigned), s), "memset");
    return finish_build(&t->desc, n, codes, sig, sh, static_cast<unsigned *>(tf.p), out, s);
}

pot_status pot_tree_quantize(const pot_tree *t, int32_t bits, pot_tree **out, pot_stream stream)
{
    if (!t || !out) return fail(POT_ERR_INVALID_ARG, "NULL tree or out");
    *out = nullptr;
    if (bits < 1 || bits > 16) return fail(POT_ERR_INVALID_ARG, "bits must be in 1..16");
    if (t->desc.leaf_dtype == POT_CB16) return fail(POT_ERR_UNSUPPORTED, "tree is already quantised");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    pot_tree *q = new (std::nothrow) pot_tree();
    if (!q) return fail(POT_ERR_OOM, "host allocation failed");
    *q = *t;
    q->desc.leaf_dtype = POT_CB16;
    q->stride = cb_stride(t->K);
    q->elem_bytes = 2;
    q->child = nullptr;
    q->sigma = nullptr;
    q->sh = nullptr;
    q->morton = nullptr;
    q->codebook = nullptr;
    q->cells = nullptr;
    q->btab = nullptr;
    q->n_bricks = 0;
    q->cell_kind = POT_CELLS_NONE;
    q->index_bytes = 0;
    cudaError_t e = cudaMalloc(&q->child, sizeof(int32_t) * 8 * t->n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&q->morton, sizeof(uint64_t) * (t->n_leaves > 0 ? t->n_leaves : 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->child, t->child, sizeof(int32_t) * 8 * t->n_nodes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && t->n_leaves > 0)
        e = cudaMemcpyAsync(q->morton, t->morton, sizeof(uint64_t) * t->n_leaves, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = quantize_tree(t, bits, q, s);
    if (e != cudaSuccess) {
        destroy_tree(q);
        return cuda_fail(e, "quantize");
    }
    const int64_t n = t->n_leaves;
    q->bytes = q->n_nodes * 32 + n * 8 + ((n * 4 + 255) / 256) * 256 + n * (int64_t)q->stride * 2 +
               (int64_t)t->K * 65536 * 8;
    e = attach_cell_index(q, s);
    if (e != cudaSuccess) {
        destroy_tree(q);
        return cuda_fail(e, "cell index");
    }
    *out = q;
    return POT_OK;
}

pot_status pot_render_batch(const pot_render_item *items, int32_t n_items, pot_stream stream)
{
    if (n_items < 0) return fail(POT_ERR_INVALID_ARG, "n_items < 0");
    if (n_items == 0) return POT_OK;
    if (!items) return fail(POT_ERR_INVALID_ARG, "items is NULL");
    int dev = 0;
    POT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    for (int i = 0; i < n_items; ++i) {
        const pot_render_item &r = items[i];
        if (!r.tree || r.tree->device != dev) return fail(POT_ERR_INVALID_ARG, "item %d: NULL tree or other device", i);
        const pot_camera &k = r.cam;
        bool ok = k.width > 0 && k.height > 0 && (int64_t)k.width * k.height <= (1ll << 31) && std::isfinite(k.fx) &&
                  std::isfinite(k.fy) && std::isfinite(k.cx) && std::isfinite(k.cy) && k.fx != 0.f && k.fy != 0.f &&
                  !std::isnan(k.near) && !std::isnan(k.far) && k.near >= 0.f;
        for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 4; ++q) ok = ok && std::isfinite(k.c2w[a][q]);
        for (int c = 0; c < 3; ++c) ok = ok && std::isfinite(r.bg[c]);
        ok = ok && r.gamma >= 0.f && std::isfinite(r.gamma);
        if (!ok) return fail(POT_ERR_INVALID_ARG, "item %d: invalid camera, bg or gamma", i);
        if (!r.rgb || !is_device_ptr(r.rgb) || (r.t_final && !is_device_ptr(r.t_final)))
            return fail(POT_ERR_INVALID_ARG, "item %d: rgb / t_final must be device memory", i);
    }
    unsigned int *err = device_error_word();
    if (!err) return fail(POT_ERR_CUDA, "device error word unavailable");
    POT_CUDA(launch_render_batch(items, n_items, (cudaStream_t)stream, err), "render_batch");
    return POT_OK;
}

pot_status pot_render_backward(const pot_tree *t, int64_t n, const float *origins, const float *dirs,
                               const float *grad_rgb, const float *rgb_fwd, const pot_render_opts *opts,
                               float *grad_sigma, float *grad_sh, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return fail(POT_ERR_INVALID_ARG, "n < 0");
    if (n == 0 || t->n_leaves == 0) return POT_OK;
    if (!origins || !dirs || !grad_rgb || !grad_sigma || !grad_sh)
        return fail(POT_ERR_INVALID_ARG, "NULL array");
    if (!is_device_ptr(origins) || !is_device_ptr(dirs) || !is_device_ptr(grad_rgb) ||
        !is_device_ptr(grad_sigma) || !is_device_ptr(grad_sh) || (rgb_fwd && !is_device_ptr(rgb_fwd)))
        return fail(POT_ERR_INVALID_ARG, "pot_render_backward takes device arrays only");
    pot_status st = check_opts(opts);
    if (st != POT_OK) return st;
    if (opts && opts->seg_count) return fail(POT_ERR_INVALID_ARG, "counting outputs are not used by the backward");
    if (t->desc.leaf_dtype == POT_CB16) return fail(POT_ERR_UNSUPPORTED, "no gradients for codebook leaves");
    if (!grad_sh_aligned(t, grad_sh)) return fail(POT_ERR_INVALID_ARG, "grad_sh must be 16-byte aligned");
    const float near = opts ? opts->near : 0.f, far = opts ? opts->far : 3.0e38f;
    if (!(near >= 0.f) || std::isnan(far)) return fail(POT_ERR_INVALID_ARG, "bad near / far");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Tmp scratch;
    POT_CUDA(scratch.alloc(sizeof(unsigned long long), s), "alloc scratch");
    POT_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(unsigned long long), s), "memset");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.ray_o = origins;
    p.ray_d = dirs;
    p.n_rays = n;
    p.near = near;
    p.far = far;
    p.n_tiles = (n + 31) / 32;
    p.tile_counter = static_cast<unsigned long long *>(scratch.p);
    POT_CUDA(launch_backward(p, grad_rgb, rgb_fwd, grad_sigma, grad_sh, t->desc.leaf_dtype, t->K, s), "backward");
    return POT_OK;
}

pot_status pot_render_mse_backward(const pot_tree *t, int64_t n, const float *origins, const float *dirs,
                                   const float *target, const pot_render_opts *opts, float *rgb, float *loss,
                                   float *grad_sigma, float *grad_sh, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return fail(POT_ERR_INVALID_ARG, "n < 0");
    if (!loss || !is_device_ptr(loss)) return fail(POT_ERR_INVALID_ARG, "loss must be device memory");
    if (n == 0) return POT_OK;
    const bool leaves = t->n_leaves > 0;
    if (!origins || !dirs || !target || (leaves && (!grad_sigma || !grad_sh)))
        return fail(POT_ERR_INVALID_ARG, "NULL array");
    if (!is_device_ptr(origins) || !is_device_ptr(dirs) || !is_device_ptr(target) ||
        (leaves && (!is_device_ptr(grad_sigma) || !is_device_ptr(grad_sh))) || (rgb && !is_device_ptr(rgb)))
        return fail(POT_ERR_INVALID_ARG, "pot_render_mse_backward takes device arrays only");
    pot_status st = check_opts(opts);
    if (st != POT_OK) return st;
    if (opts && opts->seg_count) return fail(POT_ERR_INVALID_ARG, "counting outputs are not used by the backward");
    if (t->desc.leaf_dtype == POT_CB16) return fail(POT_ERR_UNSUPPORTED, "no gradients for codebook leaves");
    if (leaves && !grad_sh_aligned(t, grad_sh)) return fail(POT_ERR_INVALID_ARG, "grad_sh must be 16-byte aligned");
    const float near = opts ? opts->near : 0.f, far = opts ? opts->far : 3.0e38f;
    if (!(near >= 0.f) || std::isnan(far)) return fail(POT_ERR_INVALID_ARG, "bad near / far");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Tmp scratch;
    POT_CUDA(scratch.alloc(sizeof(unsigned long long), s), "alloc scratch");
    POT_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(unsigned long long), s), "memset");
    POT_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s), "memset loss");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.ray_o = origins;
    p.ray_d = dirs;
    p.n_rays = n;
    p.near = near;
    p.far = far;
    p.n_tiles = (n + 31) / 32;
    p.tile_counter = static_cast<unsigned long long *>(scratch.p);
    POT_CUDA(launch_mse_backward(p, target, rgb, loss, grad_sigma, grad_sh, t->desc.leaf_dtype, t->K, s),
             "mse backward");
    return POT_OK;
}

namespace {

// Checks shared by the two recorded-segment entry points.
pot_status check_segment_buffer(const void *records, int64_t capacity, const int64_t *seg_state)
{
    if (capacity < 0 || capacity > INT32_MAX) return fail(POT_ERR_INVALID_ARG, "capacity must be in [0, 2^31)");
    if (!seg_state || !is_device_ptr(seg_state)) return fail(POT_ERR_INVALID_ARG, "seg_state must be device memory");
    if (capacity > 0 && (!records || !is_device_ptr(records)))
        return fail(POT_ERR_INVALID_ARG, "records must be device memory");
    if (((uintptr_t)records & 15u) != 0 || ((uintptr_t)seg_state & 7u) != 0)
        return fail(POT_ERR_INVALID_ARG, "records must be 16-byte and seg_state 8-byte aligned");
    return POT_OK;
}

}  // namespace

pot_status pot_render_rays_record(const pot_tree *t, int64_t n, const float *origins, const float *dirs,
                                  const pot_render_opts *opts, float *rgb, float *t_final, void *records,
                                  int64_t capacity, int64_t *seg_state, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0 || n > INT32_MAX) return fail(POT_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    pot_status st = check_segment_buffer(records, capacity, seg_state);
    if (st != POT_OK) return st;
    if (n > 0 && (!origins || !dirs || !rgb)) return fail(POT_ERR_INVALID_ARG, "NULL array");
    if (n > 0 && (!is_device_ptr(origins) || !is_device_ptr(dirs) || !is_device_ptr(rgb) ||
                  (t_final && !is_device_ptr(t_final))))
        return fail(POT_ERR_INVALID_ARG, "pot_render_rays_record takes device arrays only");
    st = check_opts(opts);
    if (st != POT_OK) return st;
    if (opts && opts->seg_count) return fail(POT_ERR_INVALID_ARG, "counting outputs are not used when recording");
    if (t->desc.leaf_dtype == POT_CB16) return fail(POT_ERR_UNSUPPORTED, "no gradients for codebook leaves");
    const float near = opts ? opts->near : 0.f, far = opts ? opts->far : 3.0e38f;
    if (!(near >= 0.f) || std::isnan(far)) return fail(POT_ERR_INVALID_ARG, "bad near / far");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    POT_CUDA(cudaMemsetAsync(seg_state, 0, 2 * sizeof(int64_t), s), "clear seg_state");
    if (n == 0) return POT_OK;
    Tmp scratch;
    POT_CUDA(scratch.alloc(sizeof(unsigned long long), s), "alloc scratch");
    POT_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(unsigned long long), s), "memset");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.ray_o = origins;
    p.ray_d = dirs;
    p.n_rays = n;
    p.near = near;
    p.far = far;
    p.n_tiles = (n + 31) / 32;
    p.rgb = rgb;
    p.t_final = t_final;
    p.tile_counter = static_cast<unsigned long long *>(scratch.p);
    const SegmentBuffer sb{static_cast<float4 *>(records), capacity, reinterpret_cast<unsigned long long *>(seg_state)};
    POT_CUDA(launch_render_record(p, sb, t->desc.leaf_dtype, t->K, s), "render_rays_record");
    return POT_OK;
}

pot_status pot_render_backward_recorded(const pot_tree *t, int64_t n, const float *origins, const float *dirs,
                                        const float *grad_rgb, const float *rgb_fwd, const pot_render_opts *opts,
                                        const void *records, int64_t capacity, const int64_t *seg_state,
                                        float *grad_sigma, float *grad_sh, pot_stream stream)
{
    if (!t) return fail(POT_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0 || n > INT32_MAX) return fail(POT_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    pot_status st = check_segment_buffer(records, capacity, seg_state);
    if (st != POT_OK) return st;
    if (n == 0 || t->n_leaves == 0) return POT_OK;
    if (!origins || !dirs || !grad_rgb || !rgb_fwd || !grad_sigma || !grad_sh)
        return fail(POT_ERR_INVALID_ARG, "NULL array");
    if (!is_device_ptr(origins) || !is_device_ptr(dirs) || !is_device_ptr(grad_rgb) || !is_device_ptr(rgb_fwd) ||
        !is_device_ptr(grad_sigma) || !is_device_ptr(grad_sh))
        return fail(POT_ERR_INVALID_ARG, "pot_render_backward_recorded takes device arrays only");
    st = check_opts(opts);
    if (st != POT_OK) return st;
    if (opts && opts->seg_count) return fail(POT_ERR_INVALID_ARG, "counting outputs are not used by the backward");
    if (t->desc.leaf_dtype == POT_CB16) return fail(POT_ERR_UNSUPPORTED, "no gradients for codebook leaves");
    if (!grad_sh_aligned(t, grad_sh)) return fail(POT_ERR_INVALID_ARG, "grad_sh must be 16-byte aligned");
    const float near = opts ? opts->near : 0.f, far = opts ? opts->far : 3.0e38f;
    if (!(near >= 0.f) || std::isnan(far)) return fail(POT_ERR_INVALID_ARG, "bad near / far");
    DeviceGuard g(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    Tmp scratch;  // tile counter of the walking fallback
    POT_CUDA(scratch.alloc(sizeof(unsigned long long), s), "alloc scratch");
    POT_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(unsigned long long), s), "memset");
    RenderParams p;
    fill_tree_params(p, t, opts);
    if (!p.err) return fail(POT_ERR_CUDA, "device error word unavailable");
    p.ray_o = origins;
    p.ray_d = dirs;
    p.n_rays = n;
    p.near = near;
    p.far = far;
    p.n_tiles = (n + 31) / 32;
    p.tile_counter = static_cast<unsigned long long *>(scratch.p);
    const SegmentBuffer sb{static_cast<float4 *>(const_cast<void *>(records)), capacity,
                           reinterpret_cast<unsigned long long *>(const_cast<int64_t *>(seg_state))};
    // scratch of the bin order: bins of 2^bb leaves (count, start, cursor)
    // and the records' numbers in bin order
    // POT_SEGBWD_ORDER (read once): 1 (default) visits the records in leaf
    // order, 0 in slot order (no sort; as fast when a batch's rays are
    // already neighbours, e.g. whole pixel tiles)
    static const bool direct = [] {
        const char *e = std::getenv("POT_SEGBWD_ORDER");
        return e && std::atoi(e) == 0;
    }();
    // scratch of the leaf order: count, start, cursor per leaf, the scan's
    // tile sums and the records' numbers in leaf order
    const int64_t nl = t->n_leaves;
    const int64_t n_tiles = (nl + kSegScanTile - 1) / kSegScanTile;
    Tmp bin_mem;
    SegmentBins bins{};
    if (!direct) {
        POT_CUDA(bin_mem.alloc(sizeof(unsigned) * (size_t)(3 * nl + 1 + n_tiles + capacity), s), "alloc sort");
        unsigned *base = static_cast<unsigned *>(bin_mem.p);
        bins = SegmentBins{base, base + nl, base + 2 * nl + 1, base + 3 * nl + 1 + n_tiles, base + 3 * nl + 1, nl};
        POT_CUDA(cudaMemsetAsync(bins.count, 0, sizeof(unsigned) * (size_t)nl, s), "clear counts");
    }
    POT_CUDA(launch_backward_recorded(p, t->n_leaves, sb, direct ? nullptr : &bins, grad_rgb, rgb_fwd, grad_sigma,
                                      grad_sh, t->desc.leaf_dtype, t->K, s),
             "backward_recorded");
    return POT_OK;
}

int64_t pot_step_state_floats(const pot_tree *t, int32_t kind)
{
    if (!t) return -1;
    const int64_t per = t->n_leaves * (1 + 3 * (int64_t)t->K);
    if (kind == POT_SGD) return 0;
    if (kind == POT_RMSPROP) return per;
    if (kind == POT_ADAM) return 2 * per;
    return -1;
}

pot_status pot_step(pot_tree *t, const pot_step_desc *d, const float *grad_sigma, const float *grad_sh, float *state,
                    pot_stream stream)
{
    if (!t || !d) return fail(POT_ERR_INVALID_ARG, "NULL tree or desc");
    if (t->desc.leaf_dtype != POT_F32) return fail(POT_ERR_UNSUPPORTED, "pot_step needs a float32 tree");
    if (d->kind < POT_SGD || d->kind > POT_ADAM) return fail(POT_ERR_INVALID_ARG, "unknown optimiser kind");
    if (!std::isfinite(d->lr_sigma) || !std::isfinite(d->lr_sh) || !std::isfinite(d->eps))
        return fail(POT_ERR_INVALID_ARG, "learning rates and eps must be finite");
    if (d->kind == POT_ADAM && d->step < 1) return fail(POT_ERR_INVALID_ARG, "Adam step counts from 1");
    if (t->n_leaves == 0) return POT_OK;
    if (!grad_sigma || !grad_sh || (d->kind != POT_SGD && !state)) return fail(POT_ERR_INVALID_ARG, "NULL array");
    if (!is_device_ptr(grad_sigma) || !is_device_ptr(grad_sh) || (state && !is_device_ptr(state)))
        return fail(POT_ERR_INVALID_ARG, "pot_step takes device arrays only");
    DeviceGuard g(t->device);
    POT_CUDA(launch_step(t, d->kind, d->lr_sigma, d->lr_sh, d->alpha, d->beta1, d->beta2, d->eps, d->step, grad_sigma,
                         grad_sh, state, (cudaStream_t)stream),
             "step");
    return POT_OK;
}

pot_status pot_loss_mse(int64_t n, const float *rgb, const float *target, float *grad_rgb, float *loss,
                        pot_stream stream)
{
    if (n < 0 || !loss) return fail(POT_ERR_INVALID_ARG, "bad n or NULL loss");
    if (n > 0 && (!rgb || !target)) return fail(POT_ERR_INVALID_ARG, "NULL array");
    if (!is_device_ptr(loss) || (n > 0 && (!is_device_ptr(rgb) || !is_device_ptr(target))) ||
        (grad_rgb && !is_device_ptr(grad_rgb)))
        return fail(POT_ERR_INVALID_ARG, "pot_loss_mse takes device arrays only");
    POT_CUDA(launch_mse(n, rgb, target, grad_rgb, loss, (cudaStream_t)stream), "loss");
    return POT_OK;
}

pot_status pot_camera_rays(const pot_camera *cams, int32_t n_cams, int64_t n, const int64_t *pixels, float *origins,
                           float *dirs, pot_stream stream)
{
    if (n_cams <= 0 || !cams || n < 0) return fail(POT_ERR_INVALID_ARG, "bad cameras or n");
    if (n == 0) return POT_OK;
    if (is_device_ptr(cams)) return fail(POT_ERR_INVALID_ARG, "cams must be in host memory");
    if (!origins || !dirs || !is_device_ptr(origins) || !is_device_ptr(dirs) || (pixels && !is_device_ptr(pixels)))
        return fail(POT_ERR_INVALID_ARG, "pixels / origins / dirs must be device memory");
    const int W = cams[0].width, H = cams[0].height;
    for (int c = 0; c < n_cams; ++c)
        if (cams[c].width != W || cams[c].height != H || W <= 0 || H <= 0)
            return fail(POT_ERR_INVALID_ARG, "cameras must share a positive width and height");
    if (!pixels && n > (int64_t)n_cams * W * H) return fail(POT_ERR_INVALID_ARG, "n exceeds the cameras' pixels");
    cudaStream_t s = (cudaStream_t)stream;
    Tmp scratch;
    const size_t cam_off = 256;
    POT_CUDA(scratch.alloc(cam_off + sizeof(pot_camera) * n_cams, s), "alloc scratch");
    char *sp = static_cast<char *>(scratch.p);
    POT_CUDA(cudaMemsetAsync(sp, 0, sizeof(unsigned), s), "memset");
    POT_CUDA(cudaMemcpyAsync(sp + cam_off, cams, sizeof(pot_camera) * n_cams, cudaMemcpyHostToDevice, s), "copy cams");
    POT_CUDA(launch_camera_rays(reinterpret_cast<const pot_camera *>(sp + cam_off), n_cams, W, H, n, pixels, origins,
                                dirs, reinterpret_cast<unsigned *>(sp), s),
             "camera rays");
    if (pixels) {
        unsigned flag = 0;
        POT_CUDA(cudaMemcpyAsync(&flag, sp, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy flag");
        POT_CUDA(cudaStreamSynchronize(s), "sync");
        if (flag) return fail(POT_ERR_INVALID_ARG, "a pixel index lies outside the cameras");
    }
    return POT_OK;
}

pot_status pot_check(pot_stream stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    POT_CUDA(cudaStreamSynchronize(s), "sync");
    unsigned int *w = device_error_word();
    if (!w) return fail(POT_ERR_CUDA, "device error word unavailable");
    unsigned v = 0;
    POT_CUDA(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost), "read error word");
    if (v) {
        POT_CUDA(cudaMemset(w, 0, sizeof(v)), "clear error word");
        return fail(POT_ERR_TRAVERSAL, "a ray exceeded its traversal step bound (word 0x%x)", v);
    }
    return POT_OK;
}

}  // extern "C"
