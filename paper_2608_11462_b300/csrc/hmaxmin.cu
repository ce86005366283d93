// hmaxmin.cu -- hierarchical maximin enumeration for the Vecchia preconditioner
// (the ordering of Sec. 2.2 / Fig. 1 that the factor conditions on).
//
// An exact maximin ordering picks, step by step, the point farthest from all points
// picked before; it is inherently sequential.  This ordering keeps its defining
// property level by level instead: over a dyadic grid of the bounding square, the
// points picked up to level L are one representative per non-empty level-L cell, so
// the points first picked at level L are spaced about one cell width apart and about
// that far from everything picked before.  Definition (the oracle restates it):
//   * square box of side E = max(x extent, y extent) at (xmin, ymin); level-30 integer
//     coordinates ix = min(floor((x - xmin) * (2^30 / E)), 2^30 - 1) and likewise iy;
//     the level-L cell of a point is (ix >> (30 - L), iy >> (30 - L));
//   * the representative of a level-L cell is the representative of its parent cell if
//     that point lies in the cell, otherwise the point of the cell nearest the cell
//     centre (x - cx)^2 + (y - cy)^2 in FP64 without FMA, ties to the smaller index;
//     the root's is the point nearest the centre of the square;
//   * the level of a point is the first L at which it represents its cell (31 if it
//     never does: points sharing a level-30 cell);
//   * points are enumerated by (level, SplitMix64(seed, index) >> 7, index).
#include <algorithm>
#include <climits>
#include <cmath>

#include "geom.cuh"
#include "phs_internal.cuh"

namespace phs {
namespace {

constexpr int kHL = 30;  // finest grid level

struct HParams {
    double xmin, ymin, E, scale;
};

__global__ void h_bbox_partial(const double2 *x, int64_t n, double4 *part) {
    __shared__ double4 red[256];
    double4 b = make_double4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 p = x[i];
        b.x = fmin(b.x, p.x);
        b.y = fmax(b.y, p.x);
        b.z = fmin(b.z, p.y);
        b.w = fmax(b.w, p.y);
    }
    red[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double4 c = red[threadIdx.x + o];
            double4 &a = red[threadIdx.x];
            a.x = fmin(a.x, c.x);
            a.y = fmax(a.y, c.y);
            a.z = fmin(a.z, c.z);
            a.w = fmax(a.w, c.w);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void h_bbox_final(const double4 *part, int np, HParams *prm) {
    double4 b = part[0];
    for (int i = 1; i < np; ++i) {
        b.x = fmin(b.x, part[i].x);
        b.y = fmax(b.y, part[i].y);
        b.z = fmin(b.z, part[i].z);
        b.w = fmax(b.w, part[i].w);
    }
    HParams h;
    h.xmin = b.x;
    h.ymin = b.z;
    h.E = fmax(b.y - b.x, b.w - b.z);
    if (!(h.E > 0)) h.E = 1.0;
    h.scale = 1073741824.0 / h.E;  // 2^30 / E
    *prm = h;
}

__global__ void h_keys(const double2 *x, int64_t n, const HParams *prm, uint64_t *key, int *idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const HParams h = *prm;
    const long long lim = (1ll << kHL) - 1;
    long long ix = (long long)floor(__dmul_rn(__dsub_rn(x[i].x, h.xmin), h.scale));
    long long iy = (long long)floor(__dmul_rn(__dsub_rn(x[i].y, h.ymin), h.scale));
    ix = ix < 0 ? 0 : (ix > lim ? lim : ix);
    iy = iy < 0 ? 0 : (iy > lim ? lim : iy);
    key[i] = morton((uint32_t)ix, (uint32_t)iy);
    idx[i] = (int)i;
}

__global__ void h_pos(const int *idx, int64_t n, int *pos) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) pos[idx[p]] = (int)p;
}

// first point of each level-L cell (points sorted by key)
__global__ void h_flags(const uint64_t *key, int64_t n, int shift, int *flag) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    flag[p] = (p == 0 || (key[p] >> shift) != (key[p - 1] >> shift)) ? 1 : 0;
}

// squared distance of each point to its level-L cell centre; per cell minimum (as bits)
__global__ void h_dist(const double2 *x, const uint64_t *key, const int *idx, const int *segx, const int *flag,
                       int64_t n, int L, const HParams *prm, double *d2, unsigned long long *segd) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const HParams h = *prm;
    const uint64_t pre = key[p] >> (2 * (kHL - L));
    const double w = ldexp(h.E, -L);
    const double cx = __dadd_rn(h.xmin, __dmul_rn((double)compact_bits(pre) + 0.5, w));
    const double cy = __dadd_rn(h.ymin, __dmul_rn((double)compact_bits(pre >> 1) + 0.5, w));
    const double2 q = x[idx[p]];
    const double dx = __dsub_rn(q.x, cx), dy = __dsub_rn(q.y, cy);
    const double d = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    d2[p] = d;
    const int seg = segx[p] + flag[p] - 1;
    atomicMin(&segd[seg], (unsigned long long)__double_as_longlong(d));
}
// smallest caller index among the points at the cell minimum
__global__ void h_argmin(const int *idx, const int *segx, const int *flag, const double *d2, int64_t n,
                         const unsigned long long *segd, int *segi) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int seg = segx[p] + flag[p] - 1;
    if ((unsigned long long)__double_as_longlong(d2[p]) == segd[seg]) atomicMin(&segi[seg], idx[p]);
}
// representative of each point's level-L cell (sorted positions); first-pick levels
__global__ void h_resolve(const uint64_t *key, const int *segx, const int *flag, const int *segi, const int *pos,
                          int64_t n, int L, const int *rep_prev, int *rep, unsigned char *lvl) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int shift = 2 * (kHL - L);
    int r;
    if (L > 0 && (key[rep_prev[p]] >> shift) == (key[p] >> shift)) {
        r = rep_prev[p];
    } else {
        r = pos[segi[segx[p] + flag[p] - 1]];
    }
    rep[p] = r;
    if (r == (int)p && lvl[p] == 255) lvl[p] = (unsigned char)L;
}

__host__ __device__ __forceinline__ uint64_t h_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// enumeration keys by caller index: (level, SplitMix64 >> 7)
__global__ void h_order_keys(const int *idx, const unsigned char *lvl, int64_t n, uint64_t seed, uint64_t *k2,
                             int *o) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = idx[p];
    const uint64_t L = lvl[p] == 255 ? (uint64_t)(kHL + 1) : (uint64_t)lvl[p];
    k2[i] = (L << 57) | (h_splitmix64(seed, (uint64_t)i) >> 7);
    o[i] = i;
}
__global__ void h_fill_u64(unsigned long long *a, int64_t n, unsigned long long v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}
__global__ void h_fill_i32(int *a, int64_t n, int v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

}  // namespace

void hmaxmin_order_dev(const double2 *x, int64_t n, uint64_t seed, int *order_out, cudaStream_t s) {
    if (n <= 0) return;
    const int nbb = (int)std::min<int64_t>(296, blocks_for(n, 256));
    DBuf<double4> part(nbb);
    DBuf<HParams> prm(1);
    h_bbox_partial<<<nbb, 256, 0, s>>>(x, n, part.get());
    PHS_LAUNCH_CHECK();
    h_bbox_final<<<1, 1, 0, s>>>(part.get(), nbb, prm.get());
    PHS_LAUNCH_CHECK();
    DBuf<uint64_t> key(n);
    DBuf<int> idx(n), pos(n), flag(n), segx(n), segi(n), repa(n), repb(n);
    DBuf<double> d2(n);
    DBuf<unsigned long long> segd(n);
    DBuf<unsigned char> lvl(n);
    h_keys<<<blocks_for(n, 256), 256, 0, s>>>(x, n, prm.get(), key.get(), idx.get());
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(key.get(), idx.get(), n, 2 * kHL, s);
    h_pos<<<blocks_for(n, 256), 256, 0, s>>>(idx.get(), n, pos.get());
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaMemsetAsync(lvl.get(), 0xFF, n, s));
    int *rep_prev = repa.get(), *rep = repb.get();
    for (int L = 0; L <= kHL; ++L) {
        h_flags<<<blocks_for(n, 256), 256, 0, s>>>(key.get(), n, 2 * (kHL - L), flag.get());
        PHS_LAUNCH_CHECK();
        exclusive_scan_i32(flag.get(), segx.get(), n, s);
        h_fill_u64<<<blocks_for(n, 256), 256, 0, s>>>(segd.get(), n, ~0ull);
        PHS_LAUNCH_CHECK();
        h_fill_i32<<<blocks_for(n, 256), 256, 0, s>>>(segi.get(), n, INT_MAX);
        PHS_LAUNCH_CHECK();
        h_dist<<<blocks_for(n, 256), 256, 0, s>>>(x, key.get(), idx.get(), segx.get(), flag.get(), n, L, prm.get(),
                                                  d2.get(), segd.get());
        PHS_LAUNCH_CHECK();
        h_argmin<<<blocks_for(n, 256), 256, 0, s>>>(idx.get(), segx.get(), flag.get(), d2.get(), n, segd.get(),
                                                    segi.get());
        PHS_LAUNCH_CHECK();
        h_resolve<<<blocks_for(n, 256), 256, 0, s>>>(key.get(), segx.get(), flag.get(), segi.get(), pos.get(), n, L,
                                                     rep_prev, rep, lvl.get());
        PHS_LAUNCH_CHECK();
        std::swap(rep_prev, rep);
    }
    DBuf<uint64_t> k2(n);
    h_order_keys<<<blocks_for(n, 256), 256, 0, s>>>(idx.get(), lvl.get(), n, seed, k2.get(), order_out);
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(k2.get(), order_out, n, 62, s);
}

}  // namespace phs
