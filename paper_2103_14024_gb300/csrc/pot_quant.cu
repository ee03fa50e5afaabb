// pot_quant.cu -- codebook quantisation of a tree's SH coefficients
// (App. B.2): for each SH basis function, median cut of the leaves' RGB
// coefficients into 2^bits boxes; the codebook entry of a box is the mean of
// its points (float64 sum in box order, rounded once to float16); each leaf
// stores one uint16 code per basis function; sigma is kept as it is (stored as
// float32, which holds the source tree's values exactly whatever its dtype).
//
// Median cut, every box split at every level: the split axis is the box's
// longest extent (ties: lowest channel); the box's points are ordered by
// (value on that axis, leaf index) and split at floor(n/2); a box of fewer
// than two points keeps them and gets an empty sibling.  Host code (an offline
// step, like the paper's conversion); the basis functions run on threads.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "pot_device.cuh"
#include "pot_internal.h"

namespace pot {

namespace {

// binary16 nearest to x (ties to even), rounded once from double; |x| >= 65520 -> inf
uint16_t half_from_double(double x)
{
    if (std::isnan(x)) return 0x7E00;
    const uint16_t sign = std::signbit(x) ? 0x8000 : 0;
    const double a = std::fabs(x);
    if (a >= 65520.0) return sign | 0x7C00;
    if (a < std::ldexp(1.0, -14)) {  // subnormal range: quantum 2^-24
        const double r = std::nearbyint(a * 16777216.0);
        return sign | (uint16_t)r;  // r == 1024 is the smallest normal, same bits
    }
    int e;
    std::frexp(a, &e);  // a = f 2^e, f in [0.5, 1)
    e -= 1;             // a in [2^e, 2^(e+1))
    double r = std::nearbyint(std::ldexp(a, 10 - e));  // in [1024, 2048]
    if (r == 2048.0) {
        r = 1024.0;
        e += 1;
    }
    return sign | (uint16_t)((e + 15) << 10) | (uint16_t)((int)r - 1024);
}

// points: n x 3 floats (stride 3K, offset 3k) -> codebook [C][4] halves, codes [n]
void median_cut(const float *pts, int64_t n, int64_t stride, int bits, uint16_t *book, uint16_t *codes)
{
    std::vector<int32_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    std::vector<int64_t> starts{0}, ends{n};
    for (int level = 0; level < bits; ++level) {
        std::vector<int64_t> ns, ne;
        ns.reserve(2 * starts.size());
        ne.reserve(2 * starts.size());
        for (size_t b = 0; b < starts.size(); ++b) {
            const int64_t s = starts[b], e = ends[b];
            if (e - s < 2) {
                ns.push_back(s);
                ne.push_back(e);
                ns.push_back(e);
                ne.push_back(e);
                continue;
            }
            double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t j = s; j < e; ++j)
                for (int c = 0; c < 3; ++c) {
                    const double v = pts[(int64_t)order[j] * stride + c];
                    mn[c] = std::min(mn[c], v);
                    mx[c] = std::max(mx[c], v);
                }
            int axis = 0;
            for (int c = 1; c < 3; ++c)
                if (mx[c] - mn[c] > mx[axis] - mn[axis]) axis = c;
            std::sort(order.begin() + s, order.begin() + e, [&](int32_t a, int32_t b2) {
                const float va = pts[(int64_t)a * stride + axis], vb = pts[(int64_t)b2 * stride + axis];
                return va < vb || (va == vb && a < b2);
            });
            const int64_t m = s + (e - s) / 2;
            ns.push_back(s);
            ne.push_back(m);
            ns.push_back(m);
            ne.push_back(e);
        }
        starts.swap(ns);
        ends.swap(ne);
    }
    const int64_t C = (int64_t)starts.size();
    for (int64_t j = 0; j < C; ++j) {
        const int64_t s = starts[j], e = ends[j];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t q = s; q < e; ++q) {
            for (int c = 0; c < 3; ++c) acc[c] = acc[c] + (double)pts[(int64_t)order[q] * stride + c];
            codes[order[q]] = (uint16_t)j;
        }
        for (int c = 0; c < 3; ++c) book[j * 4 + c] = e > s ? half_from_double(acc[c] / (double)(e - s)) : 0;
        book[j * 4 + 3] = 0;
    }
}

}  // namespace

// Builds a POT_CB16 copy of tree t (structure shared by value); *out is new.
cudaError_t quantize_tree(const pot_tree *t, int bits, pot_tree *q, cudaStream_t s)
{
    const int64_t L = t->n_leaves;
    const int K = t->K;
    std::vector<float> sig(L > 0 ? L : 1), sh((size_t)(L > 0 ? L : 1) * 3 * K);
    float *dsig = nullptr, *dsh = nullptr;
    cudaError_t e = cudaSuccess;
    if (L > 0) {
        e = cudaMallocAsync(&dsig, sizeof(float) * L, s);
        if (e == cudaSuccess) e = cudaMallocAsync(&dsh, sizeof(float) * 3 * K * L, s);
        if (e == cudaSuccess) e = export_leaves(t, dsig, dsh, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sig.data(), dsig, sizeof(float) * L, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sh.data(), dsh, sizeof(float) * 3 * K * L, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (dsig) cudaFreeAsync(dsig, s);
        if (dsh) cudaFreeAsync(dsh, s);
        if (e != cudaSuccess) return e;
    }
    const int stride = cb_stride(K);
    std::vector<uint16_t> book((size_t)K * kCodebookEntries * 4, 0);
    std::vector<uint16_t> codes((size_t)(L > 0 ? L : 1) * stride, 0);
    std::vector<std::vector<uint16_t>> per_k(K, std::vector<uint16_t>(L > 0 ? L : 1));
    {
        std::vector<std::thread> th;
        for (int k = 0; k < K; ++k)
            th.emplace_back([&, k] {
                median_cut(sh.data() + 3 * k, L, 3 * K, bits, book.data() + (size_t)k * kCodebookEntries * 4,
                           per_k[k].data());
            });
        for (auto &x : th) x.join();
    }
    for (int64_t i = 0; i < L; ++i)
        for (int k = 0; k < K; ++k) codes[(size_t)i * stride + k] = per_k[k][i];
    q->saturated = t->saturated;
    q->cb_bits = bits;
    const int64_t sig_bytes = ((L * 4 + 255) / 256) * 256;
    e = cudaMalloc(&q->sigma, sig_bytes > 0 ? sig_bytes : 256);
    if (e == cudaSuccess) e = cudaMalloc(&q->sh, sizeof(uint16_t) * stride * (L > 0 ? L : 1));
    if (e == cudaSuccess) e = cudaMalloc(&q->codebook, sizeof(uint16_t) * book.size());
    if (e == cudaSuccess && L > 0) e = cudaMemcpyAsync(q->sigma, sig.data(), sizeof(float) * L, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && L > 0)
        e = cudaMemcpyAsync(q->sh, codes.data(), sizeof(uint16_t) * stride * L, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->codebook, book.data(), sizeof(uint16_t) * book.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace pot
