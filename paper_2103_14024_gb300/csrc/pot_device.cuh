// pot_device.cuh -- device helpers of the PlenOctree render path (sm_103a).
//
// Geometry is fp32 throughout.  Plane-crossing times and plane-side tests use
// error-free transformations (TwoSum, TwoProd via fma) so that a crossing time
// is known to about 2^-46 relative and a segment length delta = t_exit - t to
// about 2^-24 of delta itself.  Plain fp32 times would carry an absolute error
// of about one ulp of t (~5e-7 at t ~ 4), which, multiplied by densities in the
// thousands, would move a pixel by more than 1e-4.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pot {

constexpr int kMaxDepth = 12;

// ------------------------------------------------------------------------
// cell index: for every voxel of the 2^D grid, the leaf that holds it (>= 0),
// or, for an empty voxel, the empty box a ray may cross in one step: the
// empty octree node of level l around the voxel (2^(D-l) voxels per axis,
// aligned), or the cube of (2e+1)^3 voxels centred on it, all empty (e < the
// voxel's Chebyshev distance to the nearest leaf).  Locating a cell (the
// octree descent of Sec. 3.2 "Rendering") becomes one 4-byte load (dense
// layout) or two (brick layout), and empty space is crossed in steps of
// whichever box is larger.  Dense entries are stored in 4x4x4 bricks (bricks
// ordered x, y, z; inside a brick x, y, z), so that a 128-byte line covers
// 2x4x4 voxels; the brick layout keeps one code per brick and stores the 64
// entries only of bricks that hold a leaf.
// ------------------------------------------------------------------------
constexpr int kCellIndexMaxDepth = 10;   // dense layout: 4 * 8^10 bytes = 4.3 GB
constexpr int kBrickIndexMaxDepth = 11;  // brick layout: 4 * 8^9 bytes of brick codes at D = 11
constexpr int kBrickIndexMinDepth = 3;
constexpr int kDenseDefaultMaxDepth = 9;  // deeper trees get the brick layout by default
constexpr int kCellCubeMax = 63;         // largest cube half-extent e the build looks for

// Stored form of an empty entry: the walker's cell shape minus 64 (cube of
// half-extent e: shape e; node of level l: shape -(1 + D - l)), so that the
// walker decodes it with one addition; the public form (export) is
// -(2 + 2 l) / -(3 + 2 e).
constexpr int kShapeBias = 64;
__host__ __device__ __forceinline__ int32_t cell_code_node(int level, int D) { return -(1 + D - level) - kShapeBias; }
__host__ __device__ __forceinline__ int32_t cell_code_cube(int e) { return e - kShapeBias; }
__host__ __device__ __forceinline__ int cell_code_node_level(int32_t v, int D) { return D + 1 + (v + kShapeBias); }
__host__ __device__ __forceinline__ int32_t cell_code_public(int32_t v, int D)
{
    if (v >= 0) return v;
    const int s = v + kShapeBias;
    return s >= 0 ? -(3 + 2 * s) : -(2 + 2 * (D + 1 + s));
}

// 4^3 bricks of the grid, ordered x, y, z; inside a brick x, y, z.
__host__ __device__ __forceinline__ uint32_t brick_of(uint32_t x, uint32_t y, uint32_t z, int D)
{
    const int nb = D > 2 ? D - 2 : 0;  // log2 of bricks per axis
    return ((x >> 2) << (2 * nb)) | ((y >> 2) << nb) | (z >> 2);
}
__host__ __device__ __forceinline__ uint32_t in_brick(uint32_t x, uint32_t y, uint32_t z)
{
    return ((x & 3u) << 4) | ((y & 3u) << 2) | (z & 3u);
}
// Entry of voxel (x, y, z) in the dense layout (D <= 10).
__host__ __device__ __forceinline__ uint32_t cell_index_offset(uint32_t x, uint32_t y, uint32_t z, int D)
{
    return (brick_of(x, y, z, D) << 6) | in_brick(x, y, z);
}
__host__ __device__ __forceinline__ int64_t brick_count(int D) { return D > 2 ? 1ll << (3 * (D - 2)) : 1; }

// Entries of the index of a depth-D tree (at least one brick).
__host__ __device__ __forceinline__ int64_t cell_index_entries(int D)
{
    const int64_t n = 1ll << (3 * D);
    return n < 64 ? 64 : n;
}

// ------------------------------------------------------------------------
// error-free transformations
// ------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (a - b) rounded once: hi parts cancel exactly when close.
__device__ __forceinline__ float df_sub(df a, df b)
{
    return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

// a < b, decided as (a.hi - b.hi) + (a.lo - b.lo) < 0 would be (the sign of a
// rounded sum is the sign of the exact sum), with one addition fewer.
__device__ __forceinline__ bool df_lt(df a, df b) { return __fsub_rn(a.hi, b.hi) < __fsub_rn(b.lo, a.lo); }

// Time t at which o + t d crosses plane k of one axis, i.e.
// (lo + k h - o) / d, with A = lo - o given exactly as Ahi + Alo and rd = 1/d.
__device__ __forceinline__ df cross_time(int k, float h, float Ahi, float Alo, float d, float rd)
{
    float p, pe;
    two_prod((float)k, h, p, pe);
    float s, e;
    two_sum(Ahi, p, s, e);
    float rest = __fadd_rn(__fadd_rn(Alo, pe), e);
    float t = __fmul_rn(s, rd);
    float r = __fadd_rn(__fmaf_rn(-t, d, s), rest);
    return {t, __fmul_rn(r, rd)};
}

// (o + t d) - (lo + k h) on one axis, to ~2^-46 relative: only its sign is used.
__device__ __forceinline__ float pos_minus_plane(df t, float d, float Ahi, float Alo, int k, float h)
{
    float p1, e1;
    two_prod(t.hi, d, p1, e1);
    float p2, e2;
    two_prod((float)k, h, p2, e2);
    float s, es;
    two_sum(p1, -Ahi, s, es);
    float s2, es2;
    two_sum(s, -p2, s2, es2);
    float rest = __fsub_rn(__fadd_rn(__fadd_rn(es, es2), __fadd_rn(e1, __fmul_rn(t.lo, d))),
                           __fadd_rn(Alo, e2));
    return __fadd_rn(s2, rest);
}

// Voxel index on one axis of the point o + t d; a point on a face goes to the
// side the ray is heading (d < 0: lower voxel).  ``margin`` bounds the error of
// the fp32 estimate in voxel units; only near a face is the exact test run.
__device__ __forceinline__ int locate_axis(df t, float d, float Ahi, float Alo, float h, float invh,
                                           float margin)
{
    float ug = __fmul_rn(__fmaf_rn(t.hi, d, -Ahi), invh);
    float kn = rintf(ug);
    float fr = __fsub_rn(ug, kn);
    int k = (int)kn;
    if (fabsf(fr) > margin) return fr > 0.f ? k : k - 1;
    float v = pos_minus_plane(t, d, Ahi, Alo, k, h);
    if (v > 0.f) return k;
    if (v < 0.f) return k - 1;
    return d < 0.f ? k - 1 : k;
}

// Exact sign of (p - lo) - k h for fp32 p, lo, h and an integer k (|k| < 2^24):
// the four exact terms are summed into a non-overlapping expansion whose most
// significant non-zero component carries the sign.
__device__ __forceinline__ int sign_point_minus_plane(float p, float lo, int k, float h)
{
    float s1, e1;
    two_sum(p, -lo, s1, e1);
    float q1, q0;
    two_prod((float)k, h, q1, q0);
    float Q, a0, a1, a2, b0, b1, b2, b3;
    two_sum(-q0, e1, Q, a0);
    two_sum(Q, s1, a2, a1);
    two_sum(-q1, a0, Q, b0);
    two_sum(Q, a1, Q, b1);
    two_sum(Q, a2, b3, b2);
    if (b3 != 0.f) return b3 > 0.f ? 1 : -1;
    if (b2 != 0.f) return b2 > 0.f ? 1 : -1;
    if (b1 != 0.f) return b1 > 0.f ? 1 : -1;
    if (b0 != 0.f) return b0 > 0.f ? 1 : -1;
    return 0;
}

// Exact voxel coordinate of p on one axis, or -1 / R when outside [lo, lo + R h).
__device__ __forceinline__ int voxel_exact(float p, float lo, float h, float invh, int R)
{
    if (!(p == p)) return -1;
    float g = floorf(__fmul_rn(__fsub_rn(p, lo), invh));
    int k = (int)fminf(fmaxf(g, -1.f), (float)R);
    for (int it = 0; it < 4 && k >= 0 && sign_point_minus_plane(p, lo, k, h) < 0; ++it) --k;
    for (int it = 0; it < 4 && k < R && sign_point_minus_plane(p, lo, k + 1, h) >= 0; ++it) ++k;
    if (k < 0) return -1;
    if (k >= R) return R;
    return k;
}

// ------------------------------------------------------------------------
// real spherical harmonics, degree <= 4 (App. B.1), polynomial form
// ------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846;

constexpr double csqrt_iter(double x, double g, int n)
{
    return n == 0 ? g : csqrt_iter(x, 0.5 * (g + x / g), n - 1);
}
constexpr double csqrt(double x) { return csqrt_iter(x, x > 1.0 ? x : 1.0, 64); }

// Constants of the real basis: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
// Legendre polynomial's leading factor, reduced to Cartesian monomials of the
// unit direction (x, y, z); every sign is + (Condon-Shortley phase cancelled by
// the (-1)^m of the real basis).
struct ShC {
    static constexpr float c0 = (float)(0.5 * csqrt(1.0 / kPi));
    static constexpr float c1 = (float)csqrt(3.0 / (4.0 * kPi));
    static constexpr float c2a = (float)(0.5 * csqrt(15.0 / kPi));
    static constexpr float c2b = (float)(0.25 * csqrt(5.0 / kPi));
    static constexpr float c2c = (float)(0.25 * csqrt(15.0 / kPi));
    static constexpr float c3a = (float)(0.25 * csqrt(35.0 / (2.0 * kPi)));
    static constexpr float c3b = (float)(0.5 * csqrt(105.0 / kPi));
    static constexpr float c3c = (float)(0.25 * csqrt(21.0 / (2.0 * kPi)));
    static constexpr float c3d = (float)(0.25 * csqrt(7.0 / kPi));
    static constexpr float c3e = (float)(0.25 * csqrt(105.0 / kPi));
    // degree 4: sqrt(2) N_4^|m| times the leading factor of P_4^|m|, with
    // (1 - z^2)^(|m|/2) cos / sin(|m| phi) written as Re / Im (x + i y)^|m|
    static constexpr float c4a = (float)(0.75 * csqrt(35.0 / kPi));          // |m| = 4, sin
    static constexpr float c4b = (float)(0.75 * csqrt(35.0 / (2.0 * kPi)));  // |m| = 3
    static constexpr float c4c = (float)(0.75 * csqrt(5.0 / kPi));           // |m| = 2, sin
    static constexpr float c4d = (float)(0.75 * csqrt(5.0 / (2.0 * kPi)));   // |m| = 1
    static constexpr float c4e = (float)(0.1875 * csqrt(1.0 / kPi));         // m = 0
    static constexpr float c4f = (float)(0.375 * csqrt(5.0 / kPi));          // |m| = 2, cos
    static constexpr float c4g = (float)(0.1875 * csqrt(35.0 / kPi));        // |m| = 4, cos
};

template <int K>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    Y[0] = ShC::c0;
    if (K > 1) {
        Y[1] = ShC::c1 * y;
        Y[2] = ShC::c1 * z;
        Y[3] = ShC::c1 * x;
    }
    if (K > 4) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = ShC::c2a * x * y;
        Y[5] = ShC::c2a * y * z;
        Y[6] = ShC::c2b * (3.f * zz - 1.f);
        Y[7] = ShC::c2a * x * z;
        Y[8] = ShC::c2c * (xx - yy);
        if (K > 9) {
            Y[9] = ShC::c3a * y * (3.f * xx - yy);
            Y[10] = ShC::c3b * x * y * z;
            Y[11] = ShC::c3c * y * (5.f * zz - 1.f);
            Y[12] = ShC::c3d * z * (5.f * zz - 3.f);
            Y[13] = ShC::c3c * x * (5.f * zz - 1.f);
            Y[14] = ShC::c3e * z * (xx - yy);
            Y[15] = ShC::c3a * x * (xx - 3.f * yy);
            if (K > 16) {
                // z-polynomials in homogeneous form (x^2 + y^2 + z^2 = 1):
                // 7z^2 - 3 = 4z^2 - 3 rho, 7z^2 - 1 = 6z^2 - rho,
                // 35z^4 - 30z^2 + 3 = 8z^4 - 24 z^2 rho + 3 rho^2 (rho = x^2 + y^2),
                // which avoids the cancellation of the large coefficients in fp32
                const float rho = xx + yy;
                const float a3 = 4.f * zz - 3.f * rho, a1 = 6.f * zz - rho;
                Y[16] = ShC::c4a * x * y * (xx - yy);
                Y[17] = ShC::c4b * y * z * (3.f * xx - yy);
                Y[18] = ShC::c4c * x * y * a1;
                Y[19] = ShC::c4d * y * z * a3;
                Y[20] = ShC::c4e * (zz * (8.f * zz - 24.f * rho) + 3.f * rho * rho);
                Y[21] = ShC::c4d * x * z * a3;
                Y[22] = ShC::c4f * (xx - yy) * a1;
                Y[23] = ShC::c4b * x * z * (xx - 3.f * yy);
                Y[24] = ShC::c4g * (xx * (xx - 3.f * yy) - yy * (3.f * xx - yy));
            }
        }
    }
}

// ------------------------------------------------------------------------
// leaf storage: sigma [L] and SH records [L][stride] (16-byte aligned rows)
// ------------------------------------------------------------------------
template <typename T>
struct Store;

template <>
struct Store<float> {
    static constexpr int kVec = 4;  // elements per 16-byte load
    __device__ static __forceinline__ float load_sigma(const float *s, int64_t i) { return __ldg(s + i); }
    __device__ static __forceinline__ void unpack(uint4 r, float *f)
    {
        f[0] = __uint_as_float(r.x);
        f[1] = __uint_as_float(r.y);
        f[2] = __uint_as_float(r.z);
        f[3] = __uint_as_float(r.w);
    }
};

template <>
struct Store<__half> {
    static constexpr int kVec = 8;
    __device__ static __forceinline__ float load_sigma(const __half *s, int64_t i)
    {
        return __half2float(__ldg(s + i));
    }
    __device__ static __forceinline__ void unpack(uint4 r, float *f)
    {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __half2 h2 = *reinterpret_cast<const __half2 *>(&w[j]);
            float2 v = __half22float2(h2);
            f[2 * j] = v.x;
            f[2 * j + 1] = v.y;
        }
    }
};

template <>
struct Store<__nv_bfloat16> {
    static constexpr int kVec = 8;
    __device__ static __forceinline__ float load_sigma(const __nv_bfloat16 *s, int64_t i)
    {
        return __bfloat162float(__ldg(s + i));
    }
    __device__ static __forceinline__ void unpack(uint4 r, float *f)
    {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            f[2 * j] = __uint_as_float(w[j] << 16);
            f[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
        }
    }
};

// Codebook-quantised leaves (App. B.2): sigma kept as it is, float32 [L]; per
// leaf one uint16 code per SH basis function, the record padded to 16 bytes;
// per basis function a codebook of 65536 entries of 4 fp16 (R, G, B, 0).
struct cb16 {
};
constexpr int kCodebookEntries = 65536;

template <>
struct Store<cb16> {
    static constexpr int kVec = 8;  // codes per 16-byte load
    __device__ static __forceinline__ float load_sigma(const cb16 *s, int64_t i)
    {
        return __ldg(reinterpret_cast<const float *>(s) + i);
    }
};

// Elements per padded SH record for K coefficients per channel.
template <typename T>
__host__ __device__ constexpr int sh_stride(int K)
{
    return (3 * K + Store<T>::kVec - 1) / Store<T>::kVec * Store<T>::kVec;
}
// codebook leaves: K codes (uint16) per record
__host__ __device__ constexpr int cb_stride(int K) { return (K + 7) / 8 * 8; }

#ifndef POT_FFMA2
// SH dot product of 16-bit leaves as packed fp32 FMAs (sm_100) on pairs of
// adjacent record elements (measured +1.2 % fp16, +1.6 % bf16; -1.3 % for
// float32 leaves, which keep scalar FMAs)
#define POT_FFMA2 1
#endif
#ifndef POT_LDG256
// read SH records with 32-byte loads where a record is a whole number of 32-byte
// units (K = 16 in every type; K = 9 and 4 in fp16 / bf16): half the load
// instructions, and fewer L1 wavefronts for the divergent gathers
#define POT_LDG256 1
#endif

// An 8-byte read-only load that does not allocate in L1 (codebook gathers:
// random entries of 16 L2-resident codebooks, rarely re-read from L1).
__device__ __forceinline__ uint2 ldg_no_l1(const uint2 *p)
{
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// One 32-byte read-only load (sm_100 and later; p 32-byte aligned) that does
// not allocate in L1: an SH record is read once per leaf segment and rarely
// again from L1 (one sector in five hits there), while filling L1 with it
// costs data-pipe wavefronts, which bound the kernel with float32 leaves.
// (Measured on the main workload: f32 leaves 2178 -> 2771 Mrays/s, f16 leaves
// 3007 -> 3042; L1 data-pipe wavefronts -30 % for f32.)
__device__ __forceinline__ void ldg256(const void *p, uint4 &a, uint4 &b)
{
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
        : "l"(p));
}

// The per-ray SH basis in shared memory, one row of float4 per thread (a
// leaf's 3K coefficients meet the basis in a few 16-byte loads instead of K
// 4-byte ones: fewer issued instructions, which bind the walk).
template <int K, int THREADS>
struct SmemY {
    // this thread's row of a [THREADS][kRow4] float4 array; an odd number of
    // float4 per row keeps the 16-byte loads of 8 consecutive threads on
    // distinct banks
    static constexpr int kRow4 = ((K + 3) / 4) | 1;
    const float *base;
    __device__ __forceinline__ float operator[](int k) const { return base[k]; }
    // yv[k] = Y_k for k0 <= k <= k1 (constant bounds once unrolled), in 16-byte loads
    __device__ __forceinline__ void fetch(float *yv, int k0, int k1) const
    {
#pragma unroll
        for (int q = k0 / 4; q <= k1 / 4; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(base)[q];
            if (4 * q + 0 >= k0 && 4 * q + 0 <= k1) yv[4 * q + 0] = v.x;
            if (4 * q + 1 >= k0 && 4 * q + 1 <= k1) yv[4 * q + 1] = v.y;
            if (4 * q + 2 >= k0 && 4 * q + 2 <= k1) yv[4 * q + 2] = v.z;
            if (4 * q + 3 >= k0 && 4 * q + 3 <= k1) yv[4 * q + 3] = v.w;
        }
    }
    __device__ __forceinline__ static void store(float *row, const float *Yt)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) row[k] = Yt[k];
    }
};

// x_c = sum_k sh[k][c] Y_k for the three channels of one leaf.  The record
// is read in chunks of 96 bytes (three 32-byte or six 16-byte loads; for
// K = 16 a chunk meets whole float4 of the basis) to bound live registers;
// each chunk fetches the basis values it multiplies.
template <int K, typename T, typename YT>
__device__ __forceinline__ void leaf_sh_dot(const T *sh, int64_t leaf, const YT &Y, float *x, const void *)
{
    constexpr int V = Store<T>::kVec;
    constexpr int N = 3 * K;
    constexpr int NV = (N + V - 1) / V;  // 16-byte units per record
    constexpr bool WIDE = POT_LDG256 && NV % 2 == 0;
    constexpr int CH = 6;                // 16-byte units per chunk (96 bytes: the basis in whole float4)
    const uint4 *p = reinterpret_cast<const uint4 *>(sh + leaf * (int64_t)(NV * V));
    x[0] = x[1] = x[2] = 0.f;
    constexpr bool PACKED = POT_FFMA2 && sizeof(T) == 2;
    float2 acc01 = make_float2(0.f, 0.f), acc12 = acc01, acc20 = acc01;
#pragma unroll
    for (int v0 = 0; v0 < NV; v0 += CH) {
        uint4 raw[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            if (v0 + j < NV) {
                if (WIDE) {
                    if (j % 2 == 0) ldg256(p + v0 + j, raw[j], raw[j + 1]);
                } else {
                    raw[j] = __ldg(p + v0 + j);
                }
            }
        }
        const int e_hi = min((v0 + CH) * V, N) - 1;
        float yv[K + 1];
        Y.fetch(yv, v0 * V / 3, PACKED ? min(e_hi / 3 + 1, K - 1) : e_hi / 3);  // a pair may reach k + 1
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            if (v0 + j < NV) {
                float f[V];
                Store<T>::unpack(raw[j], f);
                if constexpr (PACKED) {
                // element pairs (idx, idx+1), idx even, as packed FMAs: with k = idx / 3 the
                // pair is (k: R, G), (k: B, k+1: R) or (k: G, B) -- three accumulator pairs
#pragma unroll
                for (int e = 0; e < V; e += 2) {
                    const int idx = (v0 + j) * V + e;
                    if (idx + 1 < N) {
                        const int k = idx / 3, c = idx % 3;
                        const float2 a = make_float2(f[e], f[e + 1]);
                        if (c == 0) acc01 = __ffma2_rn(a, make_float2(yv[k], yv[k]), acc01);
                        else if (c == 1) acc12 = __ffma2_rn(a, make_float2(yv[k], yv[k]), acc12);
                        else acc20 = __ffma2_rn(a, make_float2(yv[k], yv[k + 1]), acc20);
                    } else if (idx < N) {
                        x[idx % 3] = fmaf(f[e], yv[idx / 3], x[idx % 3]);  // odd 3K: last element alone
                    }
                }
                } else {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const int idx = (v0 + j) * V + e;
                    if (idx < N) x[idx % 3] = fmaf(f[e], yv[idx / 3], x[idx % 3]);
                }
                }
            }
        }
    }
    if constexpr (PACKED) {
        x[0] = __fadd_rn(x[0], __fadd_rn(acc01.x, acc20.y));
        x[1] = __fadd_rn(x[1], __fadd_rn(acc01.y, acc12.x));
        x[2] = __fadd_rn(x[2], __fadd_rn(acc20.x, acc12.y));
    }
}

// Codebook leaves: x_c = sum_k codebook[k][code_k][c] Y_k.
template <int K, typename YT>
__device__ __forceinline__ void leaf_sh_dot_cb(const cb16 *sh, int64_t leaf, const YT &Y, float *x, const void *cb)
{
    constexpr int NV = (K + 7) / 8;
    const uint4 *p = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint16_t *>(sh) + leaf * (int64_t)(NV * 8));
    const uint2 *book = static_cast<const uint2 *>(cb);
    uint4 raw[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) raw[v] = __ldg(p + v);  // (one 32-byte load here measured 11 % slower)
    uint2 e[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint4 r = raw[k / 8];
        const uint32_t w = (k % 8) / 2 == 0 ? r.x : (k % 8) / 2 == 1 ? r.y : (k % 8) / 2 == 2 ? r.z : r.w;
        const uint32_t code = (k & 1) ? (w >> 16) : (w & 0xFFFFu);
        e[k] = ldg_no_l1(book + (int64_t)k * kCodebookEntries + code);
    }
    x[0] = x[1] = x[2] = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float2 rg = __half22float2(*reinterpret_cast<const __half2 *>(&e[k].x));
        const float b = __half2float(__ushort_as_half((unsigned short)(e[k].y & 0xFFFFu)));
        x[0] = fmaf(rg.x, Y[k], x[0]);
        x[1] = fmaf(rg.y, Y[k], x[1]);
        x[2] = fmaf(b, Y[k], x[2]);
    }
}

template <int K, typename T, typename YT>
__device__ __forceinline__ void leaf_colour_dot(const T *sh, int64_t leaf, const YT &Y, float *x, const void *cb)
{
    if constexpr (std::is_same<T, cb16>::value) leaf_sh_dot_cb<K>(sh, leaf, Y, x, cb);
    else leaf_sh_dot<K, T>(sh, leaf, Y, x, cb);
}

// Ask L1 for the lines of one leaf (SH record and sigma) ahead of its use.
template <int K, typename T>
__device__ __forceinline__ void prefetch_leaf(const T *sig, const T *sh, int64_t leaf)
{
    if constexpr (std::is_same<T, cb16>::value) return;
    else {
    constexpr int bytes = sh_stride<T>(K) * (int)sizeof(T);
    const char *r = reinterpret_cast<const char *>(sh + leaf * (int64_t)sh_stride<T>(K));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(r));
    if (bytes > 16) asm volatile("prefetch.global.L1 [%0];" ::"l"(r + bytes - 1));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(sig + leaf));
    }
}

// 1 / (1 + e^-x); x is clamped at -80 (sigmoid < 2e-35) so the divisor stays
// below 2^126, where the fast division is accurate to 2 ulp.
__device__ __forceinline__ float sigmoidf_(float x) { return __fdividef(1.f, 1.f + __expf(-fmaxf(x, -80.f))); }

}  // namespace pot
