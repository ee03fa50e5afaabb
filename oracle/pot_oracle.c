/*
 * pot_oracle.c -- FP64 CPU oracle of the PlenOctree render path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  It shares no code, header or
 * table with the CUDA path; the two agree only through the conventions written
 * out below (and in the public header's prose).
 *
 * What it computes (PlenOctrees, Yu et al., ICCV 2021):
 *   - tree construction: the kept voxels become leaves at the deepest level and
 *     the tree is empty elsewhere (Sec. 3.2 "Filtering");
 *   - ray/voxel intersection: the ray is cut at every voxel boundary of the
 *     octree into segments of constant density and colour; one empty node of
 *     any size is one segment (Sec. 3.2 "Rendering");
 *   - colour of a leaf: the sigmoid of the real-SH expansion evaluated at the
 *     ray direction (Sec. 3.1, NeRF-SH colour equation; SH basis of App. B.1);
 *   - compositing: NeRF quadrature over the segments (Eq. 1) with the
 *     background as a final segment (App. B.3.2), density passed through
 *     max(.,0) (App. B.3, end), early stop when transmittance < gamma
 *     (Sec. 3.2 "Rendering");
 *   - the analytic derivatives of App. B.3.2 (colour derivative = weight;
 *     density derivative with the dense suffix sum), chain rule through the
 *     sigmoid and the SH basis.
 *
 * Everything is float64 except two input conventions that are defined as
 * fp32 functions (the paper does not define a camera or a point->voxel rule):
 *   1. the pixel ray (origin, unnormalised direction) of a pinhole camera, an
 *      exact IEEE fp32 expression (see cam_ray_f32), so that both sides trace
 *      the very same line;
 *   2. fp16 / bf16 rounding of stored leaf values (round to nearest even,
 *      saturating at the largest finite value).
 *
 * Conventions:
 *   Morton code  m = sum_b x_b<<(3b+2) | y_b<<(3b+1) | z_b<<3b
 *   child slot at a node of level l: (x_bit<<2)|(y_bit<<1)|z_bit, bit D-1-l
 *   node order   breadth first, root = 0, each level by ascending Morton prefix
 *   child[n][s]  0 = empty, >0 = node index, <0 = -(leaf+1); leaf = rank of the
 *                voxel's Morton code among kept voxels
 *   voxel k on an axis = [lo + k h, lo + (k+1) h), h = size / 2^D (exact);
 *   a ray position exactly on a face belongs to the voxel the ray is heading
 *   into (direction 0 counts as upward).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* Tree                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct otree {
    int depth;
    int K; /* SH coefficients per channel, (lmax+1)^2 */
    double lo[3];
    double size;
    double h;
    int64_t n_nodes;
    int64_t n_leaves;
    int32_t *child;   /* [n_nodes][8] */
    double *sigma;    /* [n_leaves]   */
    double *sh;       /* [n_leaves][K][3] */
    uint64_t *morton; /* [n_leaves]   */
} otree;

void oracle_tree_free(otree *t)
{
    if (!t) return;
    free(t->child);
    free(t->sigma);
    free(t->sh);
    free(t->morton);
    free(t);
}

int64_t oracle_tree_n_nodes(const otree *t) { return t->n_nodes; }
int64_t oracle_tree_n_leaves(const otree *t) { return t->n_leaves; }

void oracle_tree_export(const otree *t, int32_t *child, double *sigma, double *sh, uint64_t *morton)
{
    if (child) memcpy(child, t->child, sizeof(int32_t) * 8 * (size_t)t->n_nodes);
    if (sigma) memcpy(sigma, t->sigma, sizeof(double) * (size_t)t->n_leaves);
    if (sh) memcpy(sh, t->sh, sizeof(double) * 3 * (size_t)t->K * (size_t)t->n_leaves);
    if (morton) memcpy(morton, t->morton, sizeof(uint64_t) * (size_t)t->n_leaves);
}

/* --- fp16 / bf16 rounding of stored values (round to nearest even) ------- */

static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* binary16 value nearest to x (ties to even), as a float; overflow saturates
 * to +-65504 and raises *ovf. */
static float round_f16(float x, int *ovf)
{
    double ax = fabs((double)x);
    double s = x < 0 ? -1.0 : 1.0;
    if (ax == 0.0) return x;
    /* quantum of the binade containing ax; subnormal quantum 2^-24 */
    int e;
    frexp(ax, &e);            /* ax = f * 2^e, f in [0.5,1) */
    int ue = e - 1;           /* ax in [2^ue, 2^(ue+1)) */
    if (ue < -14) ue = -14;
    double q = ldexp(1.0, ue - 10);
    double m = ax / q;        /* exact: ax is a float, q a power of two */
    double r = nearbyint(m);  /* default rounding mode: ties to even */
    double v = r * q;
    if (v > 65504.0) { if (ovf) *ovf = 1; v = 65504.0; }
    return (float)(s * v);
}

static float round_bf16(float x, int *ovf)
{
    uint32_t b = bits_from_f32(x);
    uint32_t lsb = (b >> 16) & 1u;
    uint32_t r = b + 0x7FFFu + lsb;
    r &= 0xFFFF0000u;
    float y = f32_from_bits(r);
    if (isinf(y) && !isinf(x)) {
        if (ovf) *ovf = 1;
        y = f32_from_bits((b & 0x80000000u) | 0x7F7F0000u);
    }
    return y;
}

int oracle_round_values(int dtype, int64_t n, const float *in, float *out)
{
    int ovf = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (dtype == 1) out[i] = round_f16(in[i], &ovf);
        else if (dtype == 2) out[i] = round_bf16(in[i], &ovf);
        else out[i] = in[i];
    }
    return ovf;
}

/* --- construction -------------------------------------------------------- */

typedef struct { int32_t c[8]; } tnode;

/* Leaves exist only at depth D; a node exists iff it has a kept descendant.
 * Insertion from the root creates each node on first use; a breadth-first
 * pass with slots in ascending order then numbers the nodes (this yields the
 * level-by-level, ascending-Morton-prefix order). */
otree *oracle_build_sparse(int depth, const float lo[3], float size, int sh_degree, int dtype,
                           int64_t n, const uint64_t *morton, const float *sigma, const float *sh,
                           int *err)
{
    *err = ORC_OK;
    if (depth < 1 || depth > 12 || sh_degree < 0 || sh_degree > 4 || !(size > 0) || n < 0 ||
        dtype < 0 || dtype > 2) {
        *err = ORC_EINVAL;
        return NULL;
    }
    const int D = depth;
    const uint64_t ncodes = 1ull << (3 * D);
    for (int64_t i = 0; i < n; ++i) {
        if (morton[i] >= ncodes || (i > 0 && morton[i] <= morton[i - 1]) || !isfinite(sigma[i])) {
            *err = ORC_EINVAL;
            return NULL;
        }
    }
    const int K = (sh_degree + 1) * (sh_degree + 1);
    otree *t = (otree *)calloc(1, sizeof(otree));
    t->depth = D;
    t->K = K;
    for (int a = 0; a < 3; ++a) t->lo[a] = (double)lo[a];
    t->size = (double)size;
    t->h = ldexp((double)size, -D);
    t->n_leaves = n;

    size_t cap = 1024, nn = 1;
    tnode *tn = (tnode *)calloc(cap, sizeof(tnode));
    for (int64_t i = 0; i < n; ++i) {
        uint64_t m = morton[i];
        size_t u = 0;
        for (int l = 0; l < D - 1; ++l) {
            int s = (int)((m >> (3 * (D - 1 - l))) & 7u);
            if (tn[u].c[s] == 0) {
                if (nn == cap) {
                    cap *= 2;
                    tn = (tnode *)realloc(tn, cap * sizeof(tnode));
                }
                memset(&tn[nn], 0, sizeof(tnode));
                tn[u].c[s] = (int32_t)nn;
                ++nn;
            }
            u = (size_t)tn[u].c[s];
        }
        tn[u].c[m & 7u] = (int32_t)(-(i + 1));
    }
    /* breadth-first renumbering */
    int32_t *newidx = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc(nn * sizeof(int32_t));
    t->child = (int32_t *)calloc(8 * nn, sizeof(int32_t));
    size_t qh = 0, qt = 0;
    queue[qt++] = 0;
    newidx[0] = 0;
    int32_t next = 1;
    while (qh < qt) {
        int32_t u = queue[qh++];
        int32_t nu = newidx[u];
        for (int s = 0; s < 8; ++s) {
            int32_t c = tn[u].c[s];
            if (c > 0) {
                newidx[c] = next++;
                queue[qt++] = c;
                t->child[8 * (size_t)nu + s] = newidx[c];
            } else {
                t->child[8 * (size_t)nu + s] = c; /* 0 or -(leaf+1) */
            }
        }
    }
    t->n_nodes = (int64_t)nn;
    free(newidx);
    free(queue);
    free(tn);

    t->sigma = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    t->sh = (double *)malloc(sizeof(double) * 3 * (size_t)K * (size_t)(n > 0 ? n : 1));
    t->morton = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    int ovf = 0;
    for (int64_t i = 0; i < n; ++i) {
        t->morton[i] = morton[i];
        float s = sigma[i];
        if (dtype == 1) s = round_f16(s, &ovf);
        if (dtype == 2) s = round_bf16(s, &ovf);
        t->sigma[i] = (double)s;
        for (int j = 0; j < 3 * K; ++j) {
            float v = sh[(size_t)i * 3 * K + j];
            if (dtype == 1) v = round_f16(v, &ovf);
            if (dtype == 2) v = round_bf16(v, &ovf);
            t->sh[(size_t)i * 3 * K + j] = (double)v;
        }
    }
    return t;
}

static uint64_t morton3(int64_t x, int64_t y, int64_t z, int D)
{
    uint64_t m = 0;
    for (int b = 0; b < D; ++b) {
        m |= (uint64_t)((x >> b) & 1) << (3 * b + 2);
        m |= (uint64_t)((y >> b) & 1) << (3 * b + 1);
        m |= (uint64_t)((z >> b) & 1) << (3 * b);
    }
    return m;
}

typedef struct { uint64_t m; int64_t idx; } mpair;
static int cmp_mpair(const void *a, const void *b)
{
    uint64_t x = ((const mpair *)a)->m, y = ((const mpair *)b)->m;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Dense grid sigma[R][R][R], sh[R][R][R][K][3], indexed [x][y][z]: a voxel is
 * kept iff sigma > tau. */
otree *oracle_build_dense(int depth, const float lo[3], float size, int sh_degree, int dtype,
                          float tau, const float *sigma, const float *sh, int *err)
{
    *err = ORC_OK;
    if (depth < 1 || depth > 11 || sh_degree < 0 || sh_degree > 4) {
        *err = ORC_EINVAL;
        return NULL;
    }
    const int64_t R = 1ll << depth;
    const int K = (sh_degree + 1) * (sh_degree + 1);
    int64_t nk = 0;
    for (int64_t v = 0; v < R * R * R; ++v) {
        if (!isfinite(sigma[v])) { *err = ORC_EINVAL; return NULL; }
        if (sigma[v] > tau) ++nk;
    }
    mpair *pr = (mpair *)malloc(sizeof(mpair) * (size_t)(nk > 0 ? nk : 1));
    int64_t c = 0;
    for (int64_t x = 0; x < R; ++x)
        for (int64_t y = 0; y < R; ++y)
            for (int64_t z = 0; z < R; ++z) {
                int64_t v = (x * R + y) * R + z;
                if (sigma[v] > tau) {
                    pr[c].m = morton3(x, y, z, depth);
                    pr[c].idx = v;
                    ++c;
                }
            }
    qsort(pr, (size_t)nk, sizeof(mpair), cmp_mpair);
    uint64_t *ms = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk > 0 ? nk : 1));
    float *ss = (float *)malloc(sizeof(float) * (size_t)(nk > 0 ? nk : 1));
    float *hs = (float *)malloc(sizeof(float) * 3 * (size_t)K * (size_t)(nk > 0 ? nk : 1));
    for (int64_t i = 0; i < nk; ++i) {
        ms[i] = pr[i].m;
        ss[i] = sigma[pr[i].idx];
        memcpy(hs + (size_t)i * 3 * K, sh + (size_t)pr[i].idx * 3 * K, sizeof(float) * 3 * K);
    }
    otree *t = oracle_build_sparse(depth, lo, size, sh_degree, dtype, nk, ms, ss, hs, err);
    free(pr);
    free(ms);
    free(ss);
    free(hs);
    return t;
}

/* --- point -> voxel ------------------------------------------------------ */

/* Index of the voxel containing coordinate p on one axis: the k with
 * lo + k h <= p < lo + (k+1) h; a point on a face goes to the side the ray is
 * heading (dir < 0 -> lower voxel).  The quotient (p - lo) / h only proposes
 * k (it can round across a face when p is within ~1e-16 of it, e.g. a tiny p
 * next to a face at 0); the decision compares p with the face positions
 * lo + k h, which are exact in fp64 for fp32 lo and size (both sides of the
 * comparison are exact, so the comparison is). */
static int64_t voxel_coord(double p, double lo, double h, double dir)
{
    int64_t q = (int64_t)floor((p - lo) / h);
    for (int it = 0; it < 4 && p < lo + (double)q * h; ++it) --q;
    for (int it = 0; it < 4 && p >= lo + (double)(q + 1) * h; ++it) ++q;
    if (dir < 0 && p == lo + (double)q * h) q -= 1;
    return q;
}

/* Descend to the deepest existing node containing voxel q.  Returns the leaf
 * index (>= 0) or -1 (empty); *lvl = level of the cell (D for a leaf, l for an
 * empty child of a level-(l-1) node). */
static int64_t descend(const otree *t, const int64_t q[3], int *lvl)
{
    const int D = t->depth;
    int64_t node = 0;
    for (int l = 0; l < D; ++l) {
        int b = D - 1 - l;
        int s = (int)((((q[0] >> b) & 1) << 2) | (((q[1] >> b) & 1) << 1) | ((q[2] >> b) & 1));
        int32_t c = t->child[8 * node + s];
        if (c == 0) { *lvl = l + 1; return -1; }
        if (c < 0) { *lvl = D; return (int64_t)(-c) - 1; }
        node = c;
    }
    *lvl = D; /* unreachable for a well formed tree */
    return -1;
}

/* leaf index, -1 for empty space inside the box, -2 outside the box. */
void oracle_query(const otree *t, int64_t n, const float *xyz, int32_t *out)
{
    const int64_t R = 1ll << t->depth;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t q[3];
        int outside = 0;
        for (int a = 0; a < 3; ++a) {
            double p = (double)xyz[3 * i + a];
            if (!(p >= t->lo[a] && p < t->lo[a] + t->size)) outside = 1;
            else {
                q[a] = voxel_coord(p, t->lo[a], t->h, 1.0);
                if (q[a] >= R) q[a] = R - 1; /* not reachable for p < lo + size */
            }
        }
        if (outside) { out[i] = -2; continue; }
        int lvl;
        out[i] = (int32_t)descend(t, q, &lvl);
    }
}

/* ------------------------------------------------------------------------ */
/* Ray / voxel intersection (Sec. 3.2 "Rendering")                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t leaf; /* -1: empty cell */
    double t0, t1;
    double delta; /* world length */
} oseg;

/* Cut the ray o + t d, restricted to the box and to world distances
 * [near, far] along it, into cells of the octree.  Segments of zero length
 * are dropped.  Returns the number of segments written (<= cap). */
static int trace(const otree *t, const double o[3], const double d[3], double near, double far,
                 oseg *seg, int cap)
{
    const int D = t->depth;
    const int64_t R = 1ll << D;
    const double h = t->h;
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(len > 0)) return 0;
    double tin = near / len, tout = far / len;
    for (int a = 0; a < 3; ++a) {
        double lo = t->lo[a], hi = t->lo[a] + t->size;
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] >= hi) return 0;
        } else {
            double t0 = (lo - o[a]) / d[a], t1 = (hi - o[a]) / d[a];
            if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
            if (t0 > tin) tin = t0;
            if (t1 < tout) tout = t1;
        }
    }
    if (!(tin < tout)) return 0;

    int64_t q[3];
    for (int a = 0; a < 3; ++a) {
        q[a] = voxel_coord(o[a] + tin * d[a], t->lo[a], h, d[a]);
        if (q[a] < 0) q[a] = 0;
        if (q[a] > R - 1) q[a] = R - 1;
    }
    double tc = tin;
    int ns = 0;
    for (int64_t step = 0; step < 3 * R + 8; ++step) {
        int lvl;
        int64_t leaf = descend(t, q, &lvl);
        int64_t sz = 1ll << (D - lvl);
        int64_t qb[3];
        double tb[3], texit = INFINITY;
        for (int a = 0; a < 3; ++a) {
            qb[a] = q[a] & ~(sz - 1);
            if (d[a] > 0) tb[a] = (t->lo[a] + (double)(qb[a] + sz) * h - o[a]) / d[a];
            else if (d[a] < 0) tb[a] = (t->lo[a] + (double)qb[a] * h - o[a]) / d[a];
            else tb[a] = INFINITY;
            if (tb[a] < texit) texit = tb[a];
        }
        double tend = texit < tout ? texit : tout;
        if (tend > tc && ns < cap) {
            seg[ns].leaf = leaf;
            seg[ns].t0 = tc;
            seg[ns].t1 = tend;
            seg[ns].delta = (tend - tc) * len;
            ++ns;
        }
        if (texit >= tout) break;
        int leaves_box = 0;
        for (int a = 0; a < 3; ++a) {
            if (tb[a] == texit) {
                q[a] = d[a] > 0 ? qb[a] + sz : qb[a] - 1;
                if (q[a] < 0 || q[a] >= R) leaves_box = 1;
            } else {
                int64_t v = voxel_coord(o[a] + texit * d[a], t->lo[a], h, d[a]);
                if (v < qb[a]) v = qb[a];
                if (v > qb[a] + sz - 1) v = qb[a] + sz - 1;
                q[a] = v;
            }
        }
        if (leaves_box) break;
        if (texit > tc) tc = texit;
    }
    return ns;
}

int oracle_trace_ray(const otree *t, const float o32[3], const float d32[3], double near, double far,
                     int cap, int64_t *leaf, double *t0, double *t1, double *delta)
{
    double o[3] = {o32[0], o32[1], o32[2]}, d[3] = {d32[0], d32[1], d32[2]};
    oseg *s = (oseg *)malloc(sizeof(oseg) * (size_t)(cap > 0 ? cap : 1));
    int n = trace(t, o, d, near, far, s, cap);
    for (int i = 0; i < n; ++i) {
        leaf[i] = s[i].leaf;
        t0[i] = s[i].t0;
        t1[i] = s[i].t1;
        delta[i] = s[i].delta;
    }
    free(s);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics (App. B.1)                                       */
/* ------------------------------------------------------------------------ */

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Associated Legendre P_l^m(x), m >= 0, with the Condon-Shortley phase. */
static double legendre_p(int l, int m, double x)
{
    double pmm = 1.0;
    double sx = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * sx;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = ((2.0 * ll - 1.0) * x * pm1 - (double)(ll + m - 1) * pmm) / (double)(ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

/* Y_k at the unit direction u, k = l^2 + l + m, for k < K.  Complex
 * Y_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta) e^{i m phi};
 * real basis: sqrt2 (-1)^m Im Y_l^|m| (m<0), Y_l^0, sqrt2 (-1)^m Re Y_l^m (m>0);
 * theta is the polar angle from +z, phi = atan2(y, x). */
static void sh_basis(int K, const double u[3], double *Y)
{
    double ct = u[2];
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double phi = atan2(u[1], u[0]);
    for (int l = 0; l * l < K; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double P = legendre_p(l, am, ct);
            double sgn = (am & 1) ? -1.0 : 1.0;
            double v;
            if (m < 0) v = M_SQRT2 * sgn * N * P * sin(am * phi);
            else if (m == 0) v = N * P;
            else v = M_SQRT2 * sgn * N * P * cos(am * phi);
            Y[l * l + l + m] = v;
        }
    }
}

void oracle_sh_basis(int K, int64_t n, const double *dirs, double *Y)
{
    for (int64_t i = 0; i < n; ++i) {
        const double *d = dirs + 3 * i;
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double u[3] = {d[0] / len, d[1] / len, d[2] / len};
        sh_basis(K, u, Y + (size_t)K * i);
    }
}

/* ------------------------------------------------------------------------ */
/* Compositing (Eq. 1; background term of App. B.3.2)                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    double bg[3];
    double gamma;
} oopts;

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static void leaf_color(const otree *t, int64_t leaf, const double *Y, double c[3])
{
    const double *k = t->sh + (size_t)leaf * 3 * t->K;
    for (int ch = 0; ch < 3; ++ch) {
        double x = 0.0;
        for (int j = 0; j < t->K; ++j) x += k[3 * j + ch] * Y[j];
        c[ch] = sigmoid(x);
    }
}

/* Renders one ray.  Outputs rgb, final transmittance, the number of leaf
 * segments composited and, if touched != NULL, marks composited leaves. */
static void render_one(const otree *t, const double o[3], const double d[3], double near, double far,
                       const oopts *op, oseg *buf, int cap, double rgb[3], double *tfinal,
                       int32_t *nseg, uint8_t *touched)
{
    int ns = trace(t, o, d, near, far, buf, cap);
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[25];
    if (len > 0) {
        double u[3] = {d[0] / len, d[1] / len, d[2] / len};
        sh_basis(t->K, u, Y);
    }
    double T = 1.0, C[3] = {0, 0, 0};
    int32_t nl = 0;
    for (int i = 0; i < ns; ++i) {
        if (buf[i].leaf < 0) continue;
        double sig = t->sigma[buf[i].leaf];
        if (sig < 0) sig = 0;
        double x = sig * buf[i].delta;
        double alpha = -expm1(-x);
        double c[3];
        leaf_color(t, buf[i].leaf, Y, c);
        double w = T * alpha;
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * c[ch];
        T *= exp(-x);
        ++nl;
        if (touched) touched[buf[i].leaf] = 1;
        if (op->gamma > 0 && T < op->gamma) break;
    }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch] + T * op->bg[ch];
    if (tfinal) *tfinal = T;
    if (nseg) *nseg = nl;
}

static int seg_cap(const otree *t) { return 3 * (1 << t->depth) + 16; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Rays given as fp32 origins and (not necessarily unit) directions. */
void oracle_render_rays(const otree *t, int64_t n, const float *o32, const float *d32, double near,
                        double far, const double bg[3], double gamma, double *rgb, double *tfinal,
                        int32_t *nseg, uint8_t *touched)
{
    oopts op = {{bg[0], bg[1], bg[2]}, gamma};
    int cap = seg_cap(t);
#pragma omp parallel
    {
        oseg *buf = (oseg *)malloc(sizeof(oseg) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double o[3] = {o32[3 * i], o32[3 * i + 1], o32[3 * i + 2]};
            double d[3] = {d32[3 * i], d32[3 * i + 1], d32[3 * i + 2]};
            render_one(t, o, d, near, far, &op, buf, cap, rgb + 3 * i, tfinal ? tfinal + i : NULL,
                       nseg ? nseg + i : NULL, touched);
        }
        free(buf);
    }
}

/* ------------------------------------------------------------------------ */
/* Pinhole camera (input convention, fp32)                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    float c2w[3][4];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near, far;
} ocam;

/* Ray through the centre of pixel (i = column, j = row).  Every operation is
 * one IEEE fp32 operation in the order written (compiled without contraction):
 *   xc = ((float(i) + 0.5) - cx) / fx,   yc = -(((float(j) + 0.5) - cy) / fy),   zc = -1
 *   d_r = (c2w[r][0]*xc + c2w[r][1]*yc) - c2w[r][2]      (r = 0,1,2)
 *   o_r = c2w[r][3]                                                         */
static void cam_ray_f32(const ocam *c, int i, int j, float o[3], float d[3])
{
    float xc = (((float)i + 0.5f) - c->cx) / c->fx;
    float yc = -((((float)j + 0.5f) - c->cy) / c->fy);
    for (int r = 0; r < 3; ++r) {
        float a = c->c2w[r][0] * xc;
        float b = c->c2w[r][1] * yc;
        float s = a + b;
        d[r] = s - c->c2w[r][2];
        o[r] = c->c2w[r][3];
    }
}

void oracle_cam_rays(const ocam *cams, int n_cams, float *o, float *d)
{
    int64_t k = 0;
    for (int c = 0; c < n_cams; ++c)
        for (int j = 0; j < cams[c].height; ++j)
            for (int i = 0; i < cams[c].width; ++i, ++k) cam_ray_f32(&cams[c], i, j, o + 3 * k, d + 3 * k);
}

/* Renders whole cameras: rgb [cam][row][col][3], tfinal/nseg [cam][row][col]. */
void oracle_render_cams(const otree *t, const ocam *cams, int n_cams, const double bg[3], double gamma,
                        double *rgb, double *tfinal, int32_t *nseg, uint8_t *touched)
{
    oopts op = {{bg[0], bg[1], bg[2]}, gamma};
    int cap = seg_cap(t);
    int64_t base = 0;
    for (int c = 0; c < n_cams; ++c) {
        const ocam *cam = &cams[c];
        const int W = cam->width, H = cam->height;
#pragma omp parallel
        {
            oseg *buf = (oseg *)malloc(sizeof(oseg) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
            for (int j = 0; j < H; ++j) {
                for (int i = 0; i < W; ++i) {
                    float o32[3], d32[3];
                    cam_ray_f32(cam, i, j, o32, d32);
                    double o[3] = {o32[0], o32[1], o32[2]}, d[3] = {d32[0], d32[1], d32[2]};
                    int64_t p = base + (int64_t)j * W + i;
                    render_one(t, o, d, cam->near, cam->far, &op, buf, cap, rgb + 3 * p,
                               tfinal ? tfinal + p : NULL, nseg ? nseg + p : NULL, touched);
                }
            }
            free(buf);
        }
        base += (int64_t)W * H;
    }
}

/* Renders a list of pixels (camera index, column, row): rgb [n][3]. */
void oracle_render_pixels(const otree *t, const ocam *cams, int64_t n, const int32_t *cam_idx,
                          const int32_t *px, const int32_t *py, const double bg[3], double gamma,
                          double *rgb, double *tfinal, int32_t *nseg)
{
    oopts op = {{bg[0], bg[1], bg[2]}, gamma};
    int cap = seg_cap(t);
#pragma omp parallel
    {
        oseg *buf = (oseg *)malloc(sizeof(oseg) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < n; ++k) {
            const ocam *cam = &cams[cam_idx[k]];
            float o32[3], d32[3];
            cam_ray_f32(cam, px[k], py[k], o32, d32);
            double o[3] = {o32[0], o32[1], o32[2]}, d[3] = {d32[0], d32[1], d32[2]};
            render_one(t, o, d, cam->near, cam->far, &op, buf, cap, rgb + 3 * k,
                       tfinal ? tfinal + k : NULL, nseg ? nseg + k : NULL, NULL);
        }
        free(buf);
    }
}

/* ------------------------------------------------------------------------ */
/* Visibility filtering (Sec. 3.2 "Filtering")                                */
/* ------------------------------------------------------------------------ */

/* For every leaf, the largest ray weight w_i = T_i (1 - exp(-sigma_i delta_i))
 * it receives over all pixels of the cameras (compositing as in render_one,
 * early stop included); 0 for leaves no ray composites.  max_w [n_leaves]. */
void oracle_visibility(const otree *t, const ocam *cams, int n_cams, double gamma, double *max_w)
{
    int cap = seg_cap(t);
    for (int64_t i = 0; i < t->n_leaves; ++i) max_w[i] = 0.0;
    for (int c = 0; c < n_cams; ++c) {
        const ocam *cam = &cams[c];
        const int W = cam->width, H = cam->height;
#pragma omp parallel
        {
            oseg *buf = (oseg *)malloc(sizeof(oseg) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
            for (int j = 0; j < H; ++j) {
                for (int i = 0; i < W; ++i) {
                    float o32[3], d32[3];
                    cam_ray_f32(cam, i, j, o32, d32);
                    double o[3] = {o32[0], o32[1], o32[2]}, d[3] = {d32[0], d32[1], d32[2]};
                    int ns = trace(t, o, d, cam->near, cam->far, buf, cap);
                    double T = 1.0;
                    for (int k = 0; k < ns; ++k) {
                        if (buf[k].leaf < 0) continue;
                        double sig = t->sigma[buf[k].leaf];
                        if (sig < 0) sig = 0;
                        double x = sig * buf[k].delta;
                        double w = T * (-expm1(-x));
                        double *dst = max_w + buf[k].leaf;
#pragma omp critical(visibility)
                        {
                            if (w > *dst) *dst = w;
                        }
                        T *= exp(-x);
                        if (gamma > 0 && T < gamma) break;
                    }
                }
            }
            free(buf);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Analytic derivatives (App. B.3.2)                                          */
/* ------------------------------------------------------------------------ */

/* Accumulates dL/dsigma [n_leaves] and dL/dsh [n_leaves][K][3] for
 * L = sum_rays <grad_rgb, C>, where C is the composited colour including the
 * background.  Per segment i with weight w_i = T_i (1 - exp(-sigma_i delta_i)):
 *   dC/dc_i = w_i;  dc/dx = c (1 - c);  dx/dk_j = Y_j
 *   dC/dsigma_i = delta_i [ c_i T_{i+1} - sum_{k>i} w_k c_k ],   the sum running
 *   over later segments and the background (w_N = T_N, c_N = bg); zero when
 *   the stored sigma is <= 0 (density passed through max(., 0)).
 * The suffix sum is evaluated directly (quadratic in the segment count). */
void oracle_backward_rays(const otree *t, int64_t n, const float *o32, const float *d32, double near,
                          double far, const double bg[3], double gamma, const double *grad_rgb,
                          double *grad_sigma, double *grad_sh)
{
    int cap = seg_cap(t);
    const int K = t->K;
#pragma omp parallel
    {
        oseg *buf = (oseg *)malloc(sizeof(oseg) * (size_t)cap);
        double *Ti = (double *)malloc(sizeof(double) * (size_t)(cap + 1));
        double *wi = (double *)malloc(sizeof(double) * (size_t)cap);
        double *ci = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
        int64_t *li = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *di = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n; ++r) {
            double o[3] = {o32[3 * r], o32[3 * r + 1], o32[3 * r + 2]};
            double d[3] = {d32[3 * r], d32[3 * r + 1], d32[3 * r + 2]};
            int ns = trace(t, o, d, near, far, buf, cap);
            double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double Y[25];
            if (len > 0) {
                double u[3] = {d[0] / len, d[1] / len, d[2] / len};
                sh_basis(K, u, Y);
            }
            /* forward pass over leaf segments, as in render_one */
            int N = 0;
            double T = 1.0;
            for (int i = 0; i < ns; ++i) {
                if (buf[i].leaf < 0) continue;
                double sig = t->sigma[buf[i].leaf];
                if (sig < 0) sig = 0;
                double x = sig * buf[i].delta;
                Ti[N] = T;
                wi[N] = T * (-expm1(-x));
                leaf_color(t, buf[i].leaf, Y, ci + 3 * N);
                li[N] = buf[i].leaf;
                di[N] = buf[i].delta;
                T *= exp(-x);
                ++N;
                if (gamma > 0 && T < gamma) break;
            }
            Ti[N] = T;
            const double *g = grad_rgb + 3 * r;
            for (int i = 0; i < N; ++i) {
                int64_t L = li[i];
                /* colour and SH coefficients */
                for (int ch = 0; ch < 3; ++ch) {
                    double c = ci[3 * i + ch];
                    double gx = g[ch] * wi[i] * c * (1.0 - c);
                    for (int j = 0; j < K; ++j) {
#pragma omp atomic
                        grad_sh[((size_t)L * K + j) * 3 + ch] += gx * Y[j];
                    }
                }
                /* density */
                if (t->sigma[L] > 0) {
                    double gs = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        double suffix = Ti[N] * bg[ch];
                        for (int k = i + 1; k < N; ++k) suffix += wi[k] * ci[3 * k + ch];
                        gs += g[ch] * di[i] * (ci[3 * i + ch] * Ti[i + 1] - suffix);
                    }
#pragma omp atomic
                    grad_sigma[L] += gs;
                }
            }
        }
        free(buf);
        free(Ti);
        free(wi);
        free(ci);
        free(li);
        free(di);
    }
}
