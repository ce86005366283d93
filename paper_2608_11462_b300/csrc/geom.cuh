// geom.cuh -- quadtree geometry helpers shared by the tree, FMM and evaluation kernels.
#pragma once
#include <stdint.h>
#include <cmath>

#include "phs_internal.cuh"

namespace phs {

// four doubles (bounding boxes: xmin, xmax, ymin, ymax in x, y, z, w)
struct __align__(16) Dbl4 {
    double x, y, z, w;
};


__host__ __device__ __forceinline__ uint64_t spread_bits(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
__host__ __device__ __forceinline__ uint32_t compact_bits(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}
// Morton key: x bits at even positions, y bits at odd positions; child quadrant q = key & 3
__host__ __device__ __forceinline__ uint64_t morton(uint32_t ix, uint32_t iy) {
    return spread_bits(ix) | (spread_bits(iy) << 1);
}
__host__ __device__ __forceinline__ void demorton(uint64_t key, int &ix, int &iy) {
    ix = (int)compact_bits(key);
    iy = (int)compact_bits(key >> 1);
}

// x 2^e for positive normal x and a normal result: exact, by the exponent field alone
// (no FP64 arithmetic on the device)
__host__ __device__ __forceinline__ double pow2_scaled(double x, int e) {
#ifdef __CUDA_ARCH__
    return __hiloint2double(__double2hiint(x) + (e << 20), __double2loint(x));
#else
    return std::ldexp(x, e);
#endif
}

// box of level l in the root [-R, R]^2: width 2R/2^l, centre -R + (i + 1/2) * width.
// Dividing by a power of two is exact, so the scaled forms equal the quotients.
__host__ __device__ __forceinline__ double box_width(double R, int l) { return pow2_scaled(2.0 * R, -l); }
__host__ __device__ __forceinline__ double box_centre(double R, double w, int i) { return -R + (i + 0.5) * w; }

// centre (cx, cy) and width w of box b; centres from the tree's table when it has one
__device__ __forceinline__ void box_geom(const TreeView &tv, int b, double &cx, double &cy, double &w) {
    w = box_width(tv.R, tv.level[b]);
    if (tv.ctr) {
        const double2 c = tv.ctr[b];
        cx = c.x;
        cy = c.y;
    } else {
        int ix, iy;
        demorton(tv.key[b], ix, iy);
        cx = box_centre(tv.R, w, ix);
        cy = box_centre(tv.R, w, iy);
    }
}
// the same and 1 / w = (1 / 2R) 2^l, the correctly rounded quotient 1.0 / w
__device__ __forceinline__ void box_geom_iw(const TreeView &tv, int b, double &cx, double &cy, double &w,
                                            double &iw) {
    box_geom(tv, b, cx, cy, w);
    iw = pow2_scaled(tv.rinv2, tv.level[b]);
}

// index of the box at (l, ix, iy), or -1 if it does not exist
__device__ __forceinline__ int find_box(const TreeView &tv, int l, int ix, int iy) {
    if (l < 0 || l > tv.depth) return -1;
    const int lim = 1 << l;
    if (ix < 0 || iy < 0 || ix >= lim || iy >= lim) return -1;
    const uint64_t key = morton((uint32_t)ix, (uint32_t)iy);
    int lo = tv.lvl_off[l], hi = tv.lvl_off[l + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (tv.key[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < tv.lvl_off[l + 1] && tv.key[lo] == key) ? lo : -1;
}

// deepest existing box of level <= l containing cell (l, ix, iy), or -1 if out of range
__device__ __forceinline__ int find_deepest(const TreeView &tv, int l, int ix, int iy) {
    const int lim = 1 << l;
    if (ix < 0 || iy < 0 || ix >= lim || iy >= lim) return -1;
    if (l > tv.depth) {
        ix >>= (l - tv.depth);
        iy >>= (l - tv.depth);
        l = tv.depth;
    }
    for (int ll = l; ll >= 0; --ll) {
        int b = find_box(tv, ll, ix >> (l - ll), iy >> (l - ll));
        if (b >= 0) return b;
    }
    return -1;
}

// boxes (l1, x1, y1) and (l2, x2, y2) with l1 <= l2 touch or overlap (closed squares)
__device__ __forceinline__ bool boxes_touch(int l1, int x1, int y1, int l2, int x2, int y2) {
    const int d = l2 - l1;
    const long long lox = (long long)x1 << d, hix = (long long)(x1 + 1) << d;
    const long long loy = (long long)y1 << d, hiy = (long long)(y1 + 1) << d;
    return x2 <= hix && x2 + 1 >= lox && y2 <= hiy && y2 + 1 >= loy;
}

/* Direct-interaction source ranges of box b ("near" set), for targets inside b.
 *
 * With the adaptive lists of Carrier, Greengard & Rokhlin, a target in box b
 * receives through the FMM (M2L on V lists, then L2L) every source outside:
 *   - b itself and the full subtrees of its same-level neighbours (U and W lists),
 *   - coarser leaves touching b (U list),
 *   - the X list of b and of each ancestor a: coarser leaves c that touch
 *     parent(a) but not a (folded into direct sums instead of P2L).
 * Each emitted range [start, end) is a contiguous run of Morton-sorted points.
 * emit(start, end) is called once per range; ranges never overlap. */
template <typename Emit>
__device__ void enumerate_near(const TreeView &tv, int b, Emit &&emit) {
    const int l = tv.level[b];
    int bx, by;
    demorton(tv.key[b], bx, by);
    emit(tv.start[b], tv.end[b]);
    int coarse[8];
    int nco = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
            if (dx == 0 && dy == 0) continue;
            const int nx = bx + dx, ny = by + dy;
            if (nx < 0 || ny < 0 || nx >= (1 << l) || ny >= (1 << l)) continue;
            int c = find_box(tv, l, nx, ny);
            if (c >= 0) {
                emit(tv.start[c], tv.end[c]);
            } else if (l >= 1) {
                int d = find_deepest(tv, l - 1, nx >> 1, ny >> 1);
                if (d >= 0 && tv.nchild[d] == 0) {
                    bool dup = false;
                    for (int i = 0; i < nco; ++i) dup |= coarse[i] == d;
                    if (!dup) {
                        coarse[nco++] = d;
                        emit(tv.start[d], tv.end[d]);
                    }
                }
            }
        }
    // X lists of b and its ancestors
    int a = b;
    while (a >= 0 && tv.level[a] >= 2) {
        const int la = tv.level[a];
        int ax, ay;
        demorton(tv.key[a], ax, ay);
        const int pa = tv.parent[a];
        int px, py;
        demorton(tv.key[pa], px, py);
        const int lp = la - 1;
        nco = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy) {
                if (dx == 0 && dy == 0) continue;
                const int nx = px + dx, ny = py + dy;
                if (nx < 0 || ny < 0 || nx >= (1 << lp) || ny >= (1 << lp)) continue;
                int c = find_box(tv, lp, nx, ny);
                int cand = -1;
                if (c >= 0) {
                    if (tv.nchild[c] == 0) cand = c;
                } else if (lp >= 1) {
                    int d = find_deepest(tv, lp - 1, nx >> 1, ny >> 1);
                    if (d >= 0 && tv.nchild[d] == 0) {
                        bool dup = false;
                        for (int i = 0; i < nco; ++i) dup |= coarse[i] == d;
                        if (!dup) {
                            coarse[nco++] = d;
                            cand = d;
                        }
                    }
                }
                if (cand >= 0) {
                    int cx, cy;
                    demorton(tv.key[cand], cx, cy);
                    if (!boxes_touch(tv.level[cand], cx, cy, la, ax, ay)) emit(tv.start[cand], tv.end[cand]);
                }
            }
        a = pa;
    }
}

}  // namespace phs
