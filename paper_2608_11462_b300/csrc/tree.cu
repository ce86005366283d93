// tree.cu -- normalisation (Eq. 2.1), Morton sort and adaptive quadtree with FMM lists (Sec. 2.1).
#include <algorithm>
#include <cmath>

#include "geom.cuh"
#include "phs_internal.cuh"

namespace phs {
namespace {

constexpr int BB_T = 256;
struct BBox {
    double xmin, xmax, ymin, ymax;
};

__global__ void bbox_partial(const double *pts, int64_t n, BBox *part) {
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * BB_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * BB_T) {
        double x = pts[2 * i], y = pts[2 * i + 1];
        bad |= !isfinite(x) || !isfinite(y);
        xmin = fmin(xmin, x); xmax = fmax(xmax, x);
        ymin = fmin(ymin, y); ymax = fmax(ymax, y);
    }
    __shared__ BBox sh[BB_T];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) sbad = 1;
    sh[threadIdx.x] = BBox{xmin, xmax, ymin, ymax};
    __syncthreads();
    for (int o = BB_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            BBox a = sh[threadIdx.x], b = sh[threadIdx.x + o];
            sh[threadIdx.x] = BBox{fmin(a.xmin, b.xmin), fmax(a.xmax, b.xmax), fmin(a.ymin, b.ymin), fmax(a.ymax, b.ymax)};
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        BBox r = sh[0];
        if (sbad) r.xmin = NAN;
        part[blockIdx.x] = r;
    }
}

// x' = (x - c) * rho (two roundings, no fusion), Morton key at level kMaxLevel
__global__ void normalize_keys(const double *pts, int64_t n, double cx, double cy, double rho, double R,
                               double2 *xn, uint64_t *keys, int *idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = __dmul_rn(__dsub_rn(pts[2 * i], cx), rho);
    double y = __dmul_rn(__dsub_rn(pts[2 * i + 1], cy), rho);
    xn[i] = make_double2(x, y);
    const double scale = (double)(1 << kMaxLevel) / (2.0 * R);
    long long ix = (long long)floor((x + R) * scale), iy = (long long)floor((y + R) * scale);
    const long long lim = (1ll << kMaxLevel) - 1;
    ix = ix < 0 ? 0 : (ix > lim ? lim : ix);
    iy = iy < 0 ? 0 : (iy > lim ? lim : iy);
    keys[i] = morton((uint32_t)ix, (uint32_t)iy);
    idx[i] = (int)i;
}

__global__ void gather_sorted(const double2 *xn, const int *idx, int64_t n, double2 *xs, int *perm, int *iperm) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int i = idx[p];
    xs[p] = xn[i];
    perm[p] = i;
    iperm[i] = (int)p;
}

__global__ void find_duplicates(const double2 *xs, const uint64_t *keys, int64_t n, int *flag) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 a = xs[p];
    for (int64_t q = p + 1; q < n && keys[q] == keys[p]; ++q) {
        const double2 b = xs[q];
        if (a.x == b.x && a.y == b.y) { atomicExch(flag, 1); return; }
    }
}

__device__ __forceinline__ int64_t lower_bound_key(const uint64_t *k, int64_t lo, int64_t hi, uint64_t v) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (k[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void split_count(const uint64_t *pkeys, int b0, int nb, int l, int leaf_cap, const int *start,
                            const int *end, const uint64_t *bkey, int *nchild) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int b = b0 + i;
    int s = start[b], e = end[b];
    int c = 0;
    if (e - s > leaf_cap && l < kMaxLevel) {
        const int shift = 2 * (kMaxLevel - l - 1);
        int64_t prev = s;
        for (int q = 0; q < 4; ++q) {
            int64_t nxt = q == 3 ? e : lower_bound_key(pkeys, prev, e, ((bkey[b] << 2) | (uint64_t)(q + 1)) << shift);
            c += nxt > prev;
            prev = nxt;
        }
    }
    nchild[b] = c;
}

__global__ void split_emit(const uint64_t *pkeys, int b0, int nb, int l, const int *nchild, const int *coff,
                           int child0, int *start, int *end, uint64_t *bkey, int *parent, int *child,
                           int *level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int b = b0 + i;
    if (nchild[b] == 0) { child[b] = -1; return; }
    const int s = start[b], e = end[b];
    const int shift = 2 * (kMaxLevel - l - 1);
    int slot = child0 + coff[i];
    child[b] = slot;
    int64_t prev = s;
    for (int q = 0; q < 4; ++q) {
        int64_t nxt = q == 3 ? e : lower_bound_key(pkeys, prev, e, ((bkey[b] << 2) | (uint64_t)(q + 1)) << shift);
        if (nxt > prev) {
            start[slot] = (int)prev;
            end[slot] = (int)nxt;
            bkey[slot] = (bkey[b] << 2) | (uint64_t)q;
            parent[slot] = b;
            level[slot] = l + 1;
            child[slot] = -1;
            ++slot;
        }
        prev = nxt;
    }
}

__global__ void leaf_flags(const int *nchild, int nbox, int *flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox) flag[b] = nchild[b] == 0;
}
__global__ void leaf_emit(const int *nchild, const int *off, int nbox, int *leaf_box) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox && nchild[b] == 0) leaf_box[off[b]] = b;
}
__global__ void point_leaf_fill(const int *leaf_box, int nleaf, const int *start, const int *end, int *pl) {
    int i = blockIdx.x;
    if (i >= nleaf) return;
    int b = leaf_box[i];
    for (int p = start[b] + threadIdx.x; p < end[b]; p += blockDim.x) pl[p] = i;
}

// V list (M2L sources) of box b: children of the parent's neighbours that do not touch b
template <bool FILL>
__global__ void vlist_kernel(TreeView tv, int nbox, int *cnt, const int *off, int *src, unsigned char *cls) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int l = tv.level[b];
    int c = 0;
    if (l >= 2) {
        int bx, by, px, py;
        demorton(tv.key[b], bx, by);
        const int P = tv.parent[b];
        demorton(tv.key[P], px, py);
        int o = FILL ? off[b] : 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy) {
                int C = find_box(tv, l - 1, px + dx, py + dy);
                if (C < 0 || tv.nchild[C] == 0) continue;
                for (int ch = tv.child[C]; ch < tv.child[C] + tv.nchild[C]; ++ch) {
                    int cx, cy;
                    demorton(tv.key[ch], cx, cy);
                    int ddx = cx - bx, ddy = cy - by;
                    if (ddx > 1 || ddx < -1 || ddy > 1 || ddy < -1) {
                        if (FILL) {
                            src[o + c] = ch;
                            cls[o + c] = (unsigned char)((ddx + 3) * 7 + (ddy + 3));
                        }
                        ++c;
                    }
                }
            }
    }
    if (!FILL) cnt[b] = c;
}

// near lists of every box (leaves: the P2P lists; all boxes: direct parts of target
// evaluation); the pair count covers leaves only
// The fill pass writes only inside the box's counted slice [off[b], off[b+1]) and
// counts in pairs[1] every box whose enumeration disagrees with the count pass, so a
// disagreement becomes an error at plan creation instead of a write past the list.
template <bool FILL>
__global__ void nearlist_kernel(TreeView tv, int nbox, int *cnt, const int *off, int2 *rng,
                                unsigned long long *pairs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int c = 0;
    const int o = FILL ? off[b] : 0;
    const int cap = FILL ? off[b + 1] - o : 0;
    long long np = 0;
    const int nt = tv.end[b] - tv.start[b];
    enumerate_near(tv, b, [&](int s, int e) {
        if (FILL && c < cap) rng[o + c] = make_int2(s, e);
        np += (long long)nt * (e - s);
        ++c;
    });
    if (!FILL) {
        cnt[b] = c;
    } else {
        if (c != cap) atomicAdd(pairs + 1, 1ull);
        if (tv.nchild[b] == 0) atomicAdd(pairs, (unsigned long long)np);
    }
}

// Symmetric near field (see Tree::sym_*): a near range of leaf b is either b itself, or
// the points of a box disjoint from b, entirely before or after b in Morton order; each
// leaf inside a range after b receives one gather offset.
__global__ void sym_count(TreeView tv, const int *leaf_box, int nleaf, const int *near_off, const int2 *near_rng,
                          const int *point_leaf, int *up_len, int *gcnt, int *maxleaf, unsigned long long *pairs,
                          uint64_t *cost_key, int *cost_val) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nleaf) return;
    const int b = leaf_box[li];
    const int e = tv.end[b];
    const long long nt = e - tv.start[b];
    atomicMax(maxleaf, (int)nt);
    int len = 0, nr = 0;
    for (int r = near_off[b]; r < near_off[b + 1]; ++r) {
        const int2 rg = near_rng[r];
        if (rg.x < e) continue;  // b itself or before b
        len += rg.y - rg.x;
        ++nr;
        for (int j = rg.x; j < rg.y;) {
            const int d = point_leaf[j];
            atomicAdd(&gcnt[d], 1);
            j = tv.end[leaf_box[d]];
        }
    }
    up_len[li] = len;
    atomicMax(&maxleaf[1], nr);
    atomicAdd(&pairs[0], (unsigned long long)(nt * nt));
    atomicAdd(&pairs[1], (unsigned long long)(nt * len));
    // processing order of the near-field blocks: decreasing pair count
    const unsigned long long work = (unsigned long long)(nt * (nt + len));
    cost_key[li] = 0xFFFFFFFFull - (work > 0xFFFFFFFFull ? 0xFFFFFFFFull : work);
    cost_val[li] = li;
}
__global__ void sym_fill(TreeView tv, const int *leaf_box, int nleaf, const int *near_off, const int2 *near_rng,
                         const int *point_leaf, const int *slot, const int *goff, int *gcur, int *gbase) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nleaf) return;
    const int b = leaf_box[li];
    const int e = tv.end[b];
    int base = slot[li];
    for (int r = near_off[b]; r < near_off[b + 1]; ++r) {
        const int2 rg = near_rng[r];
        if (rg.x < e) continue;
        for (int j = rg.x; j < rg.y;) {
            const int d = point_leaf[j];
            const int db = leaf_box[d];
            gbase[goff[d] + atomicAdd(&gcur[d], 1)] = base + (tv.start[db] - rg.x);
            j = tv.end[db];
        }
        base += rg.y - rg.x;
    }
}
// ascending offsets per leaf: a fixed summation order in the gather
// by a radix sort of (leaf, offset) keys: a leaf beside a dense cluster receives thousands
// of offsets, so any per-leaf quadratic sort on one thread stalls the plan
__global__ void sym_keys(const int *goff, int nleaf, const int *gbase, uint64_t *key) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nleaf) return;
    for (int a = goff[d]; a < goff[d + 1]; ++a) key[a] = ((uint64_t)d << 31) | (uint32_t)gbase[a];
}
__global__ void sym_unkey(const uint64_t *key, int64_t ng, int *gbase) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ng) gbase[i] = (int)(key[i] & 0x7FFFFFFFull);
}

__global__ void count_sum(const int *cnt, int n, unsigned long long *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(out, (unsigned long long)cnt[i]);
}

}  // namespace

TreeView tree_view(const Tree &t) {
    TreeView v;
    v.start = t.start.get(); v.end = t.end.get(); v.parent = t.parent.get(); v.child = t.child.get();
    v.nchild = t.nchild.get(); v.level = t.level.get(); v.key = t.key.get(); v.lvl_off = t.lvl_dev.get();
    v.ctr = t.ctr.get();
    v.depth = t.depth; v.R = t.R;
    v.rinv2 = 1.0 / (2.0 * t.R);
    return v;
}

__global__ void box_centres_kernel(TreeView tv, int nbox, double2 *ctr) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int ix, iy;
    demorton(tv.key[b], ix, iy);
    const double w = box_width(tv.R, tv.level[b]);
    ctr[b] = make_double2(box_centre(tv.R, w, ix), box_centre(tv.R, w, iy));
}

void build_points_and_tree(const double *pts_dev, int64_t n, double halfwidth, int leaf_cap, PointSet &ps,
                           Tree &tree, cudaStream_t s) {
    PHS_REQUIRE(n >= 1 && n < (1ll << 30), PHS_ERR_INVALID_ARG, "point count out of range");
    PHS_REQUIRE(leaf_cap >= 4 && leaf_cap <= 4096, PHS_ERR_INVALID_ARG, "leaf_cap must be in [4, 4096]");
    PHS_REQUIRE(halfwidth > 0 && std::isfinite(halfwidth), PHS_ERR_INVALID_ARG, "domain half-width must be > 0");
    // ---- bounding box and frame
    const int nbb = (int)std::min<int64_t>(592, blocks_for(n, BB_T));
    SBuf<BBox> part(nbb, s);
    bbox_partial<<<nbb, BB_T, 0, s>>>(pts_dev, n, part.get());
    PHS_LAUNCH_CHECK();
    std::vector<BBox> hp(nbb);
    PHS_CUDA(cudaMemcpyAsync(hp.data(), part.get(), nbb * sizeof(BBox), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    double xmin = hp[0].xmin, xmax = hp[0].xmax, ymin = hp[0].ymin, ymax = hp[0].ymax;
    bool bad = false;
    for (auto &v : hp) {
        bad |= std::isnan(v.xmin);
        xmin = std::min(xmin, v.xmin); xmax = std::max(xmax, v.xmax);
        ymin = std::min(ymin, v.ymin); ymax = std::max(ymax, v.ymax);
    }
    PHS_REQUIRE(!bad, PHS_ERR_INVALID_ARG, "non-finite point coordinate");
    Frame fr;
    fr.cx = (xmin + xmax) * 0.5;
    fr.cy = (ymin + ymax) * 0.5;
    const double h = std::max(xmax - xmin, ymax - ymin) * 0.5;
    PHS_REQUIRE(h > 0 || n == 1, PHS_ERR_DUPLICATE_POINTS, "all points coincide");
    fr.rho = h > 0 ? halfwidth / h : 1.0;
    fr.hw = halfwidth;
    ps.n = n;
    ps.frame = fr;
    // root box: [-R, R]^2 with a hair of slack for the rounding of (x - c) * rho
    const double R = halfwidth * (1.0 + 1e-12);
    tree.R = R;
    tree.n = n;
    tree.leaf_cap = leaf_cap;
    // ---- Morton sort
    SBuf<double2> xn(n, s);
    SBuf<uint64_t> keys(n, s);
    SBuf<int> idx(n, s);
    normalize_keys<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, fr.cx, fr.cy, fr.rho, R, xn.get(), keys.get(),
                                                       idx.get());
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(keys.get(), idx.get(), n, 2 * kMaxLevel, s);
    ps.xs.alloc(n);
    ps.perm.alloc(n);
    ps.iperm.alloc(n);
    gather_sorted<<<blocks_for(n, 256), 256, 0, s>>>(xn.get(), idx.get(), n, ps.xs.get(), ps.perm.get(),
                                                     ps.iperm.get());
    PHS_LAUNCH_CHECK();
    {
        SBuf<int> flag(1, s);
        PHS_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int), s));
        find_duplicates<<<blocks_for(n, 256), 256, 0, s>>>(ps.xs.get(), keys.get(), n, flag.get());
        PHS_LAUNCH_CHECK();
        int hf = 0;
        PHS_CUDA(cudaMemcpyAsync(&hf, flag.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        PHS_CUDA(cudaStreamSynchronize(s));
        PHS_REQUIRE(hf == 0, PHS_ERR_DUPLICATE_POINTS, "two input points coincide");
    }
    // ---- levels
    const int64_t cap64 = 1 + 4 * (int64_t)kMaxLevel * (n / (leaf_cap + 1) + 1);
    PHS_REQUIRE(cap64 < (1ll << 31), PHS_ERR_INVALID_ARG, "tree too large");
    const int cap = (int)cap64;
    tree.start.alloc(cap); tree.end.alloc(cap); tree.parent.alloc(cap); tree.child.alloc(cap);
    tree.nchild.alloc(cap); tree.level.alloc(cap); tree.key.alloc(cap);
    {
        int zero = 0, nn = (int)n, neg = -1;
        uint64_t z64 = 0;
        PHS_CUDA(cudaMemcpyAsync(tree.start.get(), &zero, sizeof(int), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(tree.end.get(), &nn, sizeof(int), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(tree.parent.get(), &neg, sizeof(int), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(tree.level.get(), &zero, sizeof(int), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(tree.key.get(), &z64, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaStreamSynchronize(s));
    }
    tree.lvl_off.assign(1, 0);
    tree.lvl_off.push_back(1);
    SBuf<int> coff(cap, s);
    int l = 0;
    for (;; ++l) {
        const int b0 = tree.lvl_off[l], nb = tree.lvl_off[l + 1] - b0;
        split_count<<<blocks_for(nb, 256), 256, 0, s>>>(keys.get(), b0, nb, l, leaf_cap, tree.start.get(),
                                                        tree.end.get(), tree.key.get(), tree.nchild.get());
        PHS_LAUNCH_CHECK();
        int64_t tot = exclusive_scan_i32(tree.nchild.get() + b0, coff.get(), nb, s);
        PHS_REQUIRE(tree.lvl_off[l + 1] + tot <= cap, PHS_ERR_CUDA, "tree capacity exceeded");
        split_emit<<<blocks_for(nb, 256), 256, 0, s>>>(keys.get(), b0, nb, l, tree.nchild.get(), coff.get(),
                                                       tree.lvl_off[l + 1], tree.start.get(), tree.end.get(),
                                                       tree.key.get(), tree.parent.get(), tree.child.get(),
                                                       tree.level.get());
        PHS_LAUNCH_CHECK();
        if (tot == 0) break;
        tree.lvl_off.push_back(tree.lvl_off[l + 1] + (int)tot);
    }
    tree.depth = l;
    tree.nbox = tree.lvl_off[l + 1];
    // nchild of the deepest level was written by split_count (all zero)
    // ---- leaves
    {
        SBuf<int> flag(tree.nbox, s), off(tree.nbox, s);
        leaf_flags<<<blocks_for(tree.nbox, 256), 256, 0, s>>>(tree.nchild.get(), tree.nbox, flag.get());
        PHS_LAUNCH_CHECK();
        tree.nleaf = (int)exclusive_scan_i32(flag.get(), off.get(), tree.nbox, s);
        tree.leaf_box.alloc(tree.nleaf);
        leaf_emit<<<blocks_for(tree.nbox, 256), 256, 0, s>>>(tree.nchild.get(), off.get(), tree.nbox,
                                                             tree.leaf_box.get());
        PHS_LAUNCH_CHECK();
        tree.point_leaf.alloc(n);
        point_leaf_fill<<<tree.nleaf, 128, 0, s>>>(tree.leaf_box.get(), tree.nleaf, tree.start.get(), tree.end.get(),
                                                    tree.point_leaf.get());
        PHS_LAUNCH_CHECK();
    }
    // ---- lists
    tree.lvl_dev.alloc(tree.lvl_off.size());
    PHS_CUDA(cudaMemcpyAsync(tree.lvl_dev.get(), tree.lvl_off.data(), tree.lvl_off.size() * sizeof(int),
                             cudaMemcpyHostToDevice, s));
    tree.ctr.alloc(tree.nbox);
    box_centres_kernel<<<blocks_for(tree.nbox, 256), 256, 0, s>>>(tree_view(tree), tree.nbox, tree.ctr.get());
    PHS_LAUNCH_CHECK();
    TreeView tv = tree_view(tree);
    {
        SBuf<int> cnt(tree.nbox, s);
        tree.v_off.alloc(tree.nbox + 1);
        vlist_kernel<false><<<blocks_for(tree.nbox, 128), 128, 0, s>>>(tv, tree.nbox, cnt.get(), nullptr, nullptr,
                                                                       nullptr);
        PHS_LAUNCH_CHECK();
        int64_t tot = exclusive_scan_i32(cnt.get(), tree.v_off.get(), tree.nbox, s);
        int t32 = (int)tot;
        PHS_CUDA(cudaMemcpyAsync(tree.v_off.get() + tree.nbox, &t32, sizeof(int), cudaMemcpyHostToDevice, s));
        tree.v_src.alloc(std::max<int64_t>(tot, 1));
        tree.v_cls.alloc(std::max<int64_t>(tot, 1));
        vlist_kernel<true><<<blocks_for(tree.nbox, 128), 128, 0, s>>>(tv, tree.nbox, nullptr, tree.v_off.get(),
                                                                      tree.v_src.get(), tree.v_cls.get());
        PHS_LAUNCH_CHECK();
        tree.m2l_pairs = tot;
    }
    {
        SBuf<int> cnt(tree.nbox, s);
        SBuf<unsigned long long> pairs(2, s);  // [0] leaf pair count, [1] boxes whose fill disagreed
        PHS_CUDA(cudaMemsetAsync(pairs.get(), 0, 2 * sizeof(unsigned long long), s));
        tree.near_off.alloc(tree.nbox + 1);
        nearlist_kernel<false><<<blocks_for(tree.nbox, 128), 128, 0, s>>>(tv, tree.nbox, cnt.get(), nullptr, nullptr,
                                                                          nullptr);
        PHS_LAUNCH_CHECK();
        int64_t tot = exclusive_scan_i32(cnt.get(), tree.near_off.get(), tree.nbox, s);
        int t32 = (int)tot;
        PHS_CUDA(cudaMemcpyAsync(tree.near_off.get() + tree.nbox, &t32, sizeof(int), cudaMemcpyHostToDevice, s));
        tree.near_rng.alloc(std::max<int64_t>(tot, 1));
        nearlist_kernel<true><<<blocks_for(tree.nbox, 128), 128, 0, s>>>(tv, tree.nbox, nullptr, tree.near_off.get(),
                                                                         tree.near_rng.get(), pairs.get());
        PHS_LAUNCH_CHECK();
        unsigned long long hp2[2] = {0, 0};
        PHS_CUDA(cudaMemcpyAsync(hp2, pairs.get(), sizeof(hp2), cudaMemcpyDeviceToHost, s));
        PHS_CUDA(cudaStreamSynchronize(s));
        PHS_REQUIRE(hp2[1] == 0, PHS_ERR_CUDA, "near-list fill pass disagreed with its count pass");
        tree.near_pairs = (int64_t)hp2[0];
    }
    {
        const int nl = tree.nleaf;
        SBuf<int> up_len(nl, s), gcnt(nl, s), gcur(nl, s), mx(2, s);
        SBuf<uint64_t> ckey(nl, s);
        tree.p2p_order.alloc(nl);
        SBuf<unsigned long long> prs(2, s);
        PHS_CUDA(cudaMemsetAsync(prs.get(), 0, 2 * sizeof(unsigned long long), s));
        PHS_CUDA(cudaMemsetAsync(gcnt.get(), 0, nl * sizeof(int), s));
        PHS_CUDA(cudaMemsetAsync(gcur.get(), 0, nl * sizeof(int), s));
        PHS_CUDA(cudaMemsetAsync(mx.get(), 0, 2 * sizeof(int), s));
        sym_count<<<blocks_for(nl, 128), 128, 0, s>>>(tv, tree.leaf_box.get(), nl, tree.near_off.get(),
                                                      tree.near_rng.get(), tree.point_leaf.get(), up_len.get(),
                                                      gcnt.get(), mx.get(), prs.get(), ckey.get(),
                                                      tree.p2p_order.get());
        PHS_LAUNCH_CHECK();
        radix_sort_pairs(ckey.get(), tree.p2p_order.get(), nl, 32, s);
        tree.sym_slot.alloc(nl + 1);
        tree.sym_goff.alloc(nl + 1);
        tree.sym_total = exclusive_scan_i32(up_len.get(), tree.sym_slot.get(), nl, s);
        const int64_t ng = exclusive_scan_i32(gcnt.get(), tree.sym_goff.get(), nl, s);
        PHS_REQUIRE(tree.sym_total < (1ll << 31), PHS_ERR_INVALID_ARG, "near field too large for 32-bit slots");
        const int tails[2] = {(int)tree.sym_total, (int)ng};
        PHS_CUDA(cudaMemcpyAsync(tree.sym_slot.get() + nl, &tails[0], sizeof(int), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(tree.sym_goff.get() + nl, &tails[1], sizeof(int), cudaMemcpyHostToDevice, s));
        tree.sym_gbase.alloc(std::max<int64_t>(ng, 1));
        sym_fill<<<blocks_for(nl, 128), 128, 0, s>>>(tv, tree.leaf_box.get(), nl, tree.near_off.get(),
                                                     tree.near_rng.get(), tree.point_leaf.get(), tree.sym_slot.get(),
                                                     tree.sym_goff.get(), gcur.get(), tree.sym_gbase.get());
        PHS_LAUNCH_CHECK();
        if (ng > 1) {
            SBuf<uint64_t> gkey(ng, s);
            SBuf<int> gval(ng, s);
            sym_keys<<<blocks_for(nl, 128), 128, 0, s>>>(tree.sym_goff.get(), nl, tree.sym_gbase.get(), gkey.get());
            PHS_LAUNCH_CHECK();
            int lb = 1;
            while ((1ll << lb) < nl) ++lb;
            radix_sort_pairs(gkey.get(), gval.get(), ng, 31 + lb, s);
            sym_unkey<<<blocks_for(ng, 256), 256, 0, s>>>(gkey.get(), ng, tree.sym_gbase.get());
            PHS_LAUNCH_CHECK();
        }
        unsigned long long hp[2];
        int hm[2];
        PHS_CUDA(cudaMemcpyAsync(hm, mx.get(), sizeof(hm), cudaMemcpyDeviceToHost, s));
        PHS_CUDA(cudaMemcpyAsync(hp, prs.get(), sizeof(hp), cudaMemcpyDeviceToHost, s));
        PHS_CUDA(cudaStreamSynchronize(s));
        tree.max_leaf = hm[0];
        tree.max_up_ranges = hm[1];
        tree.sym_ok = tree.max_leaf <= kP2PThreads && tree.max_up_ranges < kMaxUpRanges;
        tree.p2p_self_pairs = (int64_t)hp[0];
        tree.p2p_upper_pairs = (int64_t)hp[1];
    }
}

}  // namespace phs
