// maximin.cu -- dyadic maximin-type enumerations for the Vecchia preconditioner
// (the ordering of Sec. 2.2 / Fig. 1 that the factor conditions on).
//
// An exact maximin ordering picks, step by step, the point farthest from all points
// picked before; it is inherently sequential.  Both orderings here work over a dyadic
// grid of the bounding square: a square box of side E = max(x extent, y extent) at
// (xmin, ymin); level-30 integer coordinates ix = min(floor((x - xmin) * (2^30 / E)),
// 2^30 - 1) and likewise iy; the level-L cell of a point is (ix >> (30 - L),
// iy >> (30 - L)), of side c_L = E 2^-L.  Points are kept sorted by the Morton key of
// (ix, iy), so every cell is a contiguous run.  Squared distances are FP64
// dx*dx + dy*dy with one rounding per operation (no FMA), as in the oracle.
//
// Hierarchical maximin (hmaxmin_order_dev; the oracle restates it):
//   * the representative of a level-L cell is the representative of its parent cell if
//     that point lies in the cell, otherwise the point of the cell nearest the cell
//     centre, ties to the smaller index; the root's is the point nearest the centre of
//     the square;
//   * the level of a point is the first L at which it represents its cell (31 if it
//     never does: points sharing a level-30 cell);
//   * points are enumerated by (level, SplitMix64(seed, index) >> 7, index).
//
// Approximate maximin (amaxmin_order_dev; the oracle restates it): batches of points,
// each point of a batch at least half as far from the points taken before as the
// farthest point not yet taken.
//   * the first point is the one nearest the square's centre; l2[i] is the squared
//     distance of point i to the taken set;
//   * for L = 0..30, passes repeat while an untaken point has l2 >= c_L^2 (a
//     candidate): per level-L cell the candidate with the largest l2 (ties to the
//     smaller index) is eligible; eligible points are taken in (l2 descending, index)
//     order unless an already accepted point of the pass is closer than c_L; the pass
//     appends them in that order and lowers l2 by their distances;
//   * untaken points after level 30 (coincident points) follow by (l2 desc, index).
//   The greedy choice within a pass is the lexicographically first independent set of
//   the conflict graph, found here in parallel rounds: an eligible point is accepted once
//   every conflicting eligible point of higher priority is rejected, and rejected as soon
//   as one of them is accepted.  Two points closer than c_L lie in adjacent cells, and at
//   level L every untaken point has l2 < 4 c_L^2 (level L - 1 left none at or above
//   c_{L-1}^2), so conflicts are looked up in the 3 x 3 and distance updates in the 5 x 5
//   block of cells around a point.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "geom.cuh"
#include "phs_internal.cuh"

namespace phs {
namespace {

constexpr int kHL = 30;  // finest grid level

struct HParams {
    double xmin, ymin, E, scale;
};

__global__ void h_bbox_partial(const double2 *x, int64_t n, Dbl4 *part) {
    __shared__ Dbl4 red[256];
    Dbl4 b = Dbl4{INFINITY, -INFINITY, INFINITY, -INFINITY};
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
            const Dbl4 c = red[threadIdx.x + o];
            Dbl4 &a = red[threadIdx.x];
            a.x = fmin(a.x, c.x);
            a.y = fmax(a.y, c.y);
            a.z = fmin(a.z, c.z);
            a.w = fmax(a.w, c.w);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void h_bbox_final(const Dbl4 *part, int np, HParams *prm) {
    Dbl4 b = part[0];
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
    SBuf<Dbl4> part(nbb, s);
    SBuf<HParams> prm(1, s);
    h_bbox_partial<<<nbb, 256, 0, s>>>(x, n, part.get());
    PHS_LAUNCH_CHECK();
    h_bbox_final<<<1, 1, 0, s>>>(part.get(), nbb, prm.get());
    PHS_LAUNCH_CHECK();
    SBuf<uint64_t> key(n, s);
    SBuf<int> idx(n, s), pos(n, s), flag(n, s), segx(n, s), segi(n, s), repa(n, s), repb(n, s);
    SBuf<double> d2(n, s);
    SBuf<unsigned long long> segd(n, s);
    SBuf<unsigned char> lvl(n, s);
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
    SBuf<uint64_t> k2(n, s);
    h_order_keys<<<blocks_for(n, 256), 256, 0, s>>>(idx.get(), lvl.get(), n, seed, k2.get(), order_out);
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(k2.get(), order_out, n, 62, s);
}


// ============================================================================ approximate maximin
namespace {

constexpr int kDiffBits = 53;                                 // l2 rank within a pass
constexpr uint64_t kDiffMask = (1ull << kDiffBits) - 1;
constexpr int kMaxPass = (1 << (64 - kDiffBits)) - 2;        // passes 1..kMaxPass; ~0 = tail

struct AStat {
    unsigned long long maxbits;  // largest l2 (as bits) over untaken points
    int taken;                   // taken points
    int cand;                    // candidates of the pass
    int undecided;               // eligible points still undecided after a round
    unsigned long long root_d2;  // squared distance of the nearest point to the centre
    int root_arg;                // its caller index
};

__device__ __forceinline__ double a_d2(double2 a, double2 b) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}
__device__ __forceinline__ unsigned long long a_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
// one atomicAdd per warp
__device__ __forceinline__ void a_warp_count(int *ctr, bool pred) {
    const unsigned b = __ballot_sync(0xffffffffu, pred);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, __popc(b));
}

__global__ void a_gather(const double2 *x, const int *idx, int64_t n, double2 *xs) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) xs[p] = x[idx[p]];
}
__global__ void a_centre_d2(const double2 *xs, int64_t n, const HParams *prm, double *d2, AStat *st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const HParams h = *prm;
    const double2 c = make_double2(__dadd_rn(h.xmin, 0.5 * h.E), __dadd_rn(h.ymin, 0.5 * h.E));
    const double d = a_d2(xs[p], c);
    d2[p] = d;
    // one atomic per full warp: the warp's smallest distance (bits of a non-negative
    // double order like the values)
    unsigned long long m = a_bits(d);
    if (__activemask() == 0xffffffffu) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
            m = q < m ? q : m;
        }
        if ((threadIdx.x & 31) == 0) atomicMin(&st->root_d2, m);
    } else {
        atomicMin(&st->root_d2, m);
    }
}
__global__ void a_centre_arg(const int *idx, const double *d2, int64_t n, AStat *st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && a_bits(d2[p]) == st->root_d2) atomicMin(&st->root_arg, idx[p]);
}
// l2 = distance to the first point, which takes enumeration key 0
__global__ void a_root(const double2 *xs, const int *pos, int64_t n, const AStat *st, double *l2,
                       unsigned char *taken, uint64_t *keysel) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int r = pos[st->root_arg];
    l2[p] = a_d2(xs[p], xs[r]);
    taken[p] = p == r;
    keysel[p] = 0;
}
// largest untaken l2 and the taken count
__global__ void a_stats(const double *l2, const unsigned char *taken, int64_t n, AStat *st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long m = 0;
    bool t = false;
    if (p < n) {
        t = taken[p];
        if (!t) m = a_bits(l2[p]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
        m = q > m ? q : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&st->maxbits, m);
    a_warp_count(&st->taken, t);
}
__global__ void a_seg_keys(const uint64_t *key, const int *flag, const int *segx, int64_t n, int shift,
                           uint64_t *segkey) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && flag[p]) segkey[segx[p]] = key[p] >> shift;
}
// segment ids of the 5 x 5 block of level-L cells around each segment (-1: empty/outside)
// Finer levels: the cells of one coarse cell (level Lc, key >> cs) are a contiguous run of
// the sorted cell keys, which dir[coarse] = (first, end) delimits; each lookup searches
// that run only.
__global__ void a_seg_dir(const uint64_t *segkey, int nseg, int cs, int2 *dir) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const uint64_t c = segkey[sg] >> cs;
    if (sg == 0 || (segkey[sg - 1] >> cs) != c) dir[c].x = sg;
    if (sg == nseg - 1 || (segkey[sg + 1] >> cs) != c) dir[c].y = sg + 1;
}
__global__ void a_seg_nbrs(const uint64_t *segkey, int nseg, int L, const int2 *dir, int cs, int *nb) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const uint64_t pre = segkey[sg];
    const int cx = (int)compact_bits(pre), cy = (int)compact_bits(pre >> 1);
    const int side = 1 << L;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            const int qx = cx + dx, qy = cy + dy;
            int found = -1;
            if (qx >= 0 && qy >= 0 && qx < side && qy < side) {
                const uint64_t q = morton((uint32_t)qx, (uint32_t)qy);
                const int2 r = dir[q >> cs];
                int lo = r.x, hi = r.y;  // first segkey >= q within the coarse cell's run
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (segkey[mid] < q) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < nseg && segkey[lo] == q) found = lo;
            }
            nb[(int64_t)sg * 25 + (dy + 2) * 5 + (dx + 2)] = found;
        }
}
// the same 5 x 5 block through a dense table of the level's cells (tab[cell] = segment
// or -1), for levels whose grid is small enough to tabulate
__global__ void a_seg_table(const uint64_t *segkey, int nseg, int *tab) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg < nseg) tab[segkey[sg]] = sg;
}
__global__ void a_seg_nbrs_tab(const uint64_t *segkey, int nseg, int L, const int *tab, int *nb) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const uint64_t pre = segkey[sg];
    const int cx = (int)compact_bits(pre), cy = (int)compact_bits(pre >> 1);
    const int side = 1 << L;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            const int qx = cx + dx, qy = cy + dy;
            const bool in = qx >= 0 && qy >= 0 && qx < side && qy < side;
            nb[(int64_t)sg * 25 + (dy + 2) * 5 + (dx + 2)] = in ? tab[morton((uint32_t)qx, (uint32_t)qy)] : -1;
        }
}
// cells with a point accepted in the pass within their 5 x 5 block
__global__ void a_near_acc(int nseg, const int *nb, const signed char *status, unsigned char *nacc) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    unsigned char any = 0;
    for (int k = 0; k < 25; ++k) {
        const int t = nb[(int64_t)sg * 25 + k];
        if (t >= 0 && status[t] == 2) any = 1;
    }
    nacc[sg] = any;
}
__global__ void a_pass_reset(int nseg, unsigned long long *segbest, int *segarg) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg < nseg) {
        segbest[sg] = 0;
        segarg[sg] = INT_MAX;
    }
}
__device__ __forceinline__ int a_seg(const int *segx, const int *flag, int64_t p) { return segx[p] + flag[p] - 1; }
__global__ void a_cand(const double *l2, const unsigned char *taken, const int *segx, const int *flag, int64_t n,
                       double c2, unsigned long long *segbest, AStat *st) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool c = false;
    int sg = -1;
    unsigned long long v = 0;  // l2 bits of a candidate (positive), 0 otherwise
    if (p < n) {
        sg = a_seg(segx, flag, p);
        if (!taken[p] && l2[p] >= c2) {
            c = true;
            v = a_bits(l2[p]);
        }
    }
    // A cell's points are consecutive positions, so the lanes of one cell form a run of
    // the warp: a segmented max over each run, then one atomic per cell and warp from the
    // run's first lane.  After the step with offset o a lane holds the maximum over the
    // next 2o lanes of its run.
    const unsigned grp = __match_any_sync(0xffffffffu, sg);
    const int last = 31 - __clz(grp);
    unsigned long long mx = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long q = __shfl_down_sync(0xffffffffu, mx, o);
        if (lane + o <= last) mx = q > mx ? q : mx;
    }
    if (mx != 0 && lane == __ffs(grp) - 1) atomicMax(&segbest[sg], mx);
    a_warp_count(&st->cand, c);
}
__global__ void a_cand_arg(const double *l2, const unsigned char *taken, const int *segx, const int *flag,
                           const int *idx, int64_t n, double c2, const unsigned long long *segbest, int *segarg) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || taken[p] || !(l2[p] >= c2)) return;
    const int sg = a_seg(segx, flag, p);
    if (a_bits(l2[p]) == segbest[sg]) atomicMin(&segarg[sg], idx[p]);
}
// status: 0 no eligible point, 1 undecided, 2 accepted, 3 rejected
__global__ void a_elig(int nseg, const unsigned long long *segbest, const int *segarg, const int *pos, int *elig,
                       signed char *status) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const bool e = segbest[sg] != 0;
    elig[sg] = e ? pos[segarg[sg]] : -1;
    status[sg] = e ? 1 : 0;
}
// one round of the parallel greedy: decide each undecided eligible point whose
// conflicting higher-priority neighbours are decided
__global__ void a_mis(int nseg, const int *nb, const int *elig, const double *l2, const int *idx,
                      const double2 *xs, double c2, signed char *status, AStat *st) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    bool still = false;
    if (sg < nseg && status[sg] == 1) {
        const int e = elig[sg];
        const double le = l2[e];
        const int ie = idx[e];
        const double2 xe = xs[e];
        bool acc = false, wait = false;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const int t = nb[(int64_t)sg * 25 + (dy + 2) * 5 + (dx + 2)];
                if (t < 0) continue;
                const signed char stt = ((volatile signed char *)status)[t];
                if (stt != 1 && stt != 2) continue;
                const int f = elig[t];
                const double lf = l2[f];
                const bool higher = lf > le || (lf == le && idx[f] < ie);
                if (!higher || !(a_d2(xe, xs[f]) < c2)) continue;
                if (stt == 2) acc = true;
                else wait = true;
            }
        if (acc) status[sg] = 3;
        else if (!wait) status[sg] = 2;
        else still = true;
    }
    a_warp_count(&st->undecided, still);
}
// accepted points are taken; their enumeration key is (pass, l2 descending) -- the
// caller index breaks ties through the stable final sort
__global__ void a_accept(int nseg, const int *elig, const signed char *status, const double *l2, double c2,
                         uint64_t pass, unsigned char *taken, uint64_t *keysel) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg || status[sg] != 2) return;
    const int e = elig[sg];
    uint64_t diff = a_bits(l2[e]) - a_bits(c2);  // l2 in [c2, 4 c2): below 2^53
    if (diff > kDiffMask) diff = kDiffMask;
    taken[e] = 1;
    keysel[e] = (pass << kDiffBits) | (kDiffMask - diff);
}
// lower l2 of untaken points by the points accepted in the pass (5 x 5 cells)
__global__ void a_update(const double2 *xs, const unsigned char *taken, const int *segx, const int *flag, int64_t n,
                         const int *nb, const int *elig, const signed char *status, const unsigned char *nacc,
                         double *l2) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int sg = a_seg(segx, flag, p);
    if (!nacc[sg] || taken[p]) return;
    const double2 xp = xs[p];
    double best = l2[p];
    const int *row = nb + (int64_t)sg * 25;
    for (int k = 0; k < 25; ++k) {
        const int t = row[k];
        if (t < 0 || status[t] != 2) continue;
        const double d = a_d2(xp, xs[elig[t]]);
        if (d < best) best = d;
    }
    l2[p] = best;
}
// final keys in caller order: taken points by (pass, l2 desc), the tail last
__global__ void a_final_keys(const int *pos, const unsigned char *taken, const uint64_t *keysel, int64_t n,
                             uint64_t *k, int *v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = pos[i];
    k[i] = taken[p] ? keysel[p] : ~0ull;
    v[i] = (int)i;
}
__global__ void a_tail_keys(const int *order, const int *pos, const double *l2, int64_t t0, int64_t cnt, uint64_t *k) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < cnt) k[j] = ~a_bits(l2[pos[order[t0 + j]]]);
}

}  // namespace

void amaxmin_order_dev(const double2 *x, int64_t n, int *order_out, cudaStream_t s) {
    if (n <= 0) return;
    PHS_REQUIRE(n < INT_MAX, PHS_ERR_INVALID_ARG, "too many points for the approximate maximin ordering");
    const unsigned nb256 = blocks_for(n, 256);
    const int nbb = (int)std::min<int64_t>(296, nb256);
    SBuf<Dbl4> part(nbb, s);
    SBuf<HParams> prm(1, s);
    h_bbox_partial<<<nbb, 256, 0, s>>>(x, n, part.get());
    PHS_LAUNCH_CHECK();
    h_bbox_final<<<1, 1, 0, s>>>(part.get(), nbb, prm.get());
    PHS_LAUNCH_CHECK();
    SBuf<uint64_t> key(n, s), keysel(n, s);
    SBuf<int> idx(n, s), pos(n, s), flag(n, s), segx(n, s);
    SBuf<double2> xs(n, s);
    SBuf<double> l2(n, s);
    SBuf<unsigned char> taken(n, s);
    SBuf<AStat> st(1, s);
    h_keys<<<nb256, 256, 0, s>>>(x, n, prm.get(), key.get(), idx.get());
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(key.get(), idx.get(), n, 2 * kHL, s);
    h_pos<<<nb256, 256, 0, s>>>(idx.get(), n, pos.get());
    PHS_LAUNCH_CHECK();
    a_gather<<<nb256, 256, 0, s>>>(x, idx.get(), n, xs.get());
    PHS_LAUNCH_CHECK();
    AStat hs{};
    hs.root_d2 = ~0ull;
    hs.root_arg = INT_MAX;
    PHS_CUDA(cudaMemcpyAsync(st.get(), &hs, sizeof(AStat), cudaMemcpyHostToDevice, s));
    a_centre_d2<<<nb256, 256, 0, s>>>(xs.get(), n, prm.get(), l2.get(), st.get());
    PHS_LAUNCH_CHECK();
    a_centre_arg<<<nb256, 256, 0, s>>>(idx.get(), l2.get(), n, st.get());
    PHS_LAUNCH_CHECK();
    a_root<<<nb256, 256, 0, s>>>(xs.get(), pos.get(), n, st.get(), l2.get(), taken.get(), keysel.get());
    PHS_LAUNCH_CHECK();
    HParams h{};
    PHS_CUDA(cudaMemcpyAsync(&h, prm.get(), sizeof(HParams), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));

    // per-cell buffers (a level has at most n cells), stream-ordered scratch sized once
    SBuf<uint64_t> segkey(n, s);
    SBuf<unsigned long long> segbest(n, s);
    SBuf<int> segarg(n, s), elig(n, s), nbr((size_t)n * 25, s);
    SBuf<signed char> status(n, s);
    // levels whose 4^L cells number at most max(16 n, 4^8), and at most 4^11, look their
    // neighbour cells up in a dense table; finer levels search the sorted cell keys within
    // the run of one coarse cell (stream-ordered scratch, sized once)
    const int64_t tab_cap = std::min<int64_t>(1ll << 22, std::max<int64_t>(16 * n, 1ll << 16));
    SBuf<int> celltab(tab_cap, s);
    SBuf<int2> dirtab(tab_cap, s);
    SBuf<unsigned char> nacc(n, s);
    uint64_t pass = 0;
    auto read_stat = [&]() {
        PHS_CUDA(cudaMemcpyAsync(&hs, st.get(), sizeof(AStat), cudaMemcpyDeviceToHost, s));
        PHS_CUDA(cudaStreamSynchronize(s));
    };
    auto level_c2 = [&](int L) {
        const double cL = std::ldexp(h.E, -L);
        return cL * cL;
    };
    for (int L = 0; L <= kHL; ++L) {
        // jump over levels without candidates: one statistics read per level that has work
        PHS_CUDA(cudaMemsetAsync(st.get(), 0, offsetof(AStat, cand), s));
        a_stats<<<nb256, 256, 0, s>>>(l2.get(), taken.get(), n, st.get());
        PHS_LAUNCH_CHECK();
        read_stat();
        if (hs.taken >= n) break;
        double maxl2;
        std::memcpy(&maxl2, &hs.maxbits, sizeof(double));
        while (L <= kHL && !(maxl2 >= level_c2(L))) ++L;
        if (L > kHL) break;
        const double c2 = level_c2(L);
        // level-L cells: segments of the Morton order and their 5 x 5 neighbourhoods
        const int shift = 2 * (kHL - L);
        h_flags<<<nb256, 256, 0, s>>>(key.get(), n, shift, flag.get());
        PHS_LAUNCH_CHECK();
        const int nseg = (int)exclusive_scan_i32(flag.get(), segx.get(), n, s);
        const unsigned sb = blocks_for(nseg, 256);
        a_seg_keys<<<nb256, 256, 0, s>>>(key.get(), flag.get(), segx.get(), n, shift, segkey.get());
        PHS_LAUNCH_CHECK();
        const int64_t ncell = 1ll << (2 * L);
        if (ncell <= tab_cap) {
            PHS_CUDA(cudaMemsetAsync(celltab.get(), 0xFF, (size_t)ncell * sizeof(int), s));
            a_seg_table<<<sb, 256, 0, s>>>(segkey.get(), nseg, celltab.get());
            PHS_LAUNCH_CHECK();
            a_seg_nbrs_tab<<<sb, 256, 0, s>>>(segkey.get(), nseg, L, celltab.get(), nbr.get());
        } else {
            // coarse directory at the finest tabulated level
            int Lc = 0;
            while (Lc < L && (1ll << (2 * (Lc + 1))) <= tab_cap) ++Lc;
            const int cs = 2 * (L - Lc);
            const int64_t ncoarse = 1ll << (2 * Lc);
            PHS_CUDA(cudaMemsetAsync(dirtab.get(), 0, (size_t)ncoarse * sizeof(int2), s));  // empty runs
            a_seg_dir<<<sb, 256, 0, s>>>(segkey.get(), nseg, cs, dirtab.get());
            PHS_LAUNCH_CHECK();
            a_seg_nbrs<<<sb, 256, 0, s>>>(segkey.get(), nseg, L, dirtab.get(), cs, nbr.get());
        }
        PHS_LAUNCH_CHECK();
        for (;;) {
            // a pass: candidates, one eligible point per cell, then rounds of the parallel
            // greedy (each decides at least the highest-priority undecided point; rounds
            // after the last change change nothing).  The candidate count is read together
            // with the undecided count after the first two rounds: an empty pass leaves no
            // eligible point and ends the level.
            a_pass_reset<<<sb, 256, 0, s>>>(nseg, segbest.get(), segarg.get());
            PHS_LAUNCH_CHECK();
            PHS_CUDA(cudaMemsetAsync(&st.get()->cand, 0, sizeof(int), s));
            a_cand<<<nb256, 256, 0, s>>>(l2.get(), taken.get(), segx.get(), flag.get(), n, c2, segbest.get(),
                                         st.get());
            PHS_LAUNCH_CHECK();
            a_cand_arg<<<nb256, 256, 0, s>>>(l2.get(), taken.get(), segx.get(), flag.get(), idx.get(), n, c2,
                                             segbest.get(), segarg.get());
            PHS_LAUNCH_CHECK();
            a_elig<<<sb, 256, 0, s>>>(nseg, segbest.get(), segarg.get(), pos.get(), elig.get(), status.get());
            PHS_LAUNCH_CHECK();
            int rounds = 0;
            for (;;) {
                for (int k = 0; k < (rounds == 0 ? 2 : 1); ++k) {
                    PHS_CUDA(cudaMemsetAsync(&st.get()->undecided, 0, sizeof(int), s));
                    a_mis<<<sb, 256, 0, s>>>(nseg, nbr.get(), elig.get(), l2.get(), idx.get(), xs.get(), c2,
                                             status.get(), st.get());
                    PHS_LAUNCH_CHECK();
                    ++rounds;
                }
                read_stat();
                if (hs.cand == 0 || hs.undecided == 0) break;
                PHS_REQUIRE(rounds <= nseg + 1, PHS_ERR_CUDA, "approximate maximin: independent set did not settle");
            }
            if (hs.cand == 0) break;
            ++pass;
            PHS_REQUIRE((int64_t)pass <= kMaxPass, PHS_ERR_INVALID_ARG, "approximate maximin: too many passes");
            a_accept<<<sb, 256, 0, s>>>(nseg, elig.get(), status.get(), l2.get(), c2, pass, taken.get(),
                                        keysel.get());
            PHS_LAUNCH_CHECK();
            a_near_acc<<<sb, 256, 0, s>>>(nseg, nbr.get(), status.get(), nacc.get());
            PHS_LAUNCH_CHECK();
            a_update<<<nb256, 256, 0, s>>>(xs.get(), taken.get(), segx.get(), flag.get(), n, nbr.get(), elig.get(),
                                           status.get(), nacc.get(), l2.get());
            PHS_LAUNCH_CHECK();
        }
    }
    // one stable sort by (pass, l2 descending) over caller indices; the tail (never a
    // candidate) keeps key ~0 and is then ordered by l2 descending
    SBuf<uint64_t> fk(n, s);
    a_final_keys<<<nb256, 256, 0, s>>>(pos.get(), taken.get(), keysel.get(), n, fk.get(), order_out);
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(fk.get(), order_out, n, 64, s);
    PHS_CUDA(cudaMemsetAsync(&st.get()->taken, 0, sizeof(int), s));
    a_stats<<<nb256, 256, 0, s>>>(l2.get(), taken.get(), n, st.get());
    PHS_LAUNCH_CHECK();
    read_stat();
    const int64_t ntail = n - hs.taken;
    if (ntail > 1) {
        SBuf<uint64_t> tk(ntail, s);
        a_tail_keys<<<blocks_for(ntail, 256), 256, 0, s>>>(order_out, pos.get(), l2.get(), hs.taken, ntail, tk.get());
        PHS_LAUNCH_CHECK();
        radix_sort_pairs(tk.get(), order_out + hs.taken, ntail, 64, s);
    }
}

}  // namespace phs
