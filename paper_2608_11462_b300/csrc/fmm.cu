// fmm.cu -- 2D fast multipole method for the PHS matvec (Sec. 2.1) through the
// Hadamard/low-rank identity (Eq. 2.6):  M t = sum_l D_{u_l} M_core D_{v_l} t.
//
// Log core (even k): complex outgoing/incoming expansions (Eqs. 2.13-2.15) with
// box-width scaled coefficients, so the translation operators are level
// invariant:  a~_k = a_k / w^k,  b~_l = b_l w^l  (w = box width at the level).
//   P2M  a_0 = sum q,  a~_k = -sum q zeta^k / k,           zeta = (z - c)/w
//   M2M  a~'_l = -a_0 d^l / l + sum_{k<=l} a~_k 2^-k d^(l-k) C(l-1,k-1)   (d = child offset / w_parent)
//   M2L  b~_0 = a_0 (log w + log(-o)) + sum_k a~_k (-1)^k o^-k
//        b~_l = -a_0 / (l o^l) + o^-l sum_k a~_k (-1)^k C(l+k-1,k-1) o^-k (o = source offset / w)
//   L2L  b~'_m = sum_{l>=m} b~_l C(l,m) d^(l-m) 2^-m
//   L2P  Re sum_l b~_l v^l,  v = (z - c)/w
// The near field (U, W and folded X lists) is summed directly with the full phi,
// which equals the Hadamard sum restricted to those pairs.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "geom.cuh"
#include "hadamard.cuh"
#include "phs_internal.cuh"

namespace phs {

// ---------------------------------------------------------------- complex helpers
template <typename T> struct C2T;
template <> struct C2T<double> { using type = double2; };
template <> struct C2T<float> { using type = float2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ void cfma(C &acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

constexpr int kMaxNd = 10;
constexpr int kMaxP = 61;


// ---------------------------------------------------------------- operators (host)
// layout: slot s in [0,4) M2M quadrant, [4,8) L2L quadrant, [8,57) M2L class (dx+3)*7+(dy+3)
constexpr int kSlots = 57;
static std::vector<std::complex<long double>> build_ops(int P) {
    using cx = std::complex<long double>;
    std::vector<cx> ops((size_t)kSlots * P * P, cx(0, 0));
    auto at = [&](int s, int r, int c) -> cx & { return ops[((size_t)s * P + r) * P + c]; };
    // binomials up to 2P
    std::vector<std::vector<long double>> C(2 * P + 1, std::vector<long double>(2 * P + 1, 0));
    for (int a = 0; a <= 2 * P; ++a) {
        C[a][0] = 1;
        for (int b = 1; b <= a; ++b) C[a][b] = C[a - 1][b - 1] + (b <= a - 1 ? C[a - 1][b] : 0);
    }
    for (int q = 0; q < 4; ++q) {
        cx d((q & 1) ? 0.25L : -0.25L, (q & 2) ? 0.25L : -0.25L);
        // M2M
        at(q, 0, 0) = 1;
        for (int l = 1; l < P; ++l) {
            at(q, l, 0) = -std::pow(d, l) / (long double)l;
            for (int k = 1; k <= l; ++k)
                at(q, l, k) = std::pow(0.5L, (long double)k) * std::pow(d, l - k) * C[l - 1][k - 1];
        }
        // L2L
        for (int m = 0; m < P; ++m)
            for (int l = m; l < P; ++l) at(4 + q, m, l) = C[l][m] * std::pow(d, l - m) * std::pow(0.5L, (long double)m);
    }
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy) {
            if (std::abs(dx) <= 1 && std::abs(dy) <= 1) continue;
            const int s = 8 + (dx + 3) * 7 + (dy + 3);
            cx o((long double)dx, (long double)dy);
            cx io = 1.0L / o;
            at(s, 0, 0) = std::log(-o);
            for (int l = 1; l < P; ++l) at(s, l, 0) = -std::pow(io, l) / (long double)l;
            for (int l = 0; l < P; ++l)
                for (int k = 1; k < P; ++k) {
                    long double sg = (k % 2) ? -1.0L : 1.0L;
                    at(s, l, k) = sg * C[l + k - 1][k - 1] * std::pow(io, l + k);
                }
        }
    return ops;
}

// ---------------------------------------------------------------- kernels
constexpr int FMM_T = 256;
constexpr int OUT_PER_T = 3;  // nd * P <= 768

template <typename T>
__global__ void p2m_kernel(TreeView tv, const int *leaf_box, const double2 *xs, const double *t, int power, int nd,
                           int P, typename C2T<T>::type *mp) {
    using C = typename C2T<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *pw = reinterpret_cast<C *>(smem_raw);        // [32][P]
    T *qs = reinterpret_cast<T *>(pw + 32 * P);     // [32][nd]
    const int b = leaf_box[blockIdx.x];
    double cx, cy, w, iw;
    box_geom_iw(tv, b, cx, cy, w, iw);
    const int s = tv.start[b], e = tv.end[b];
    C acc[OUT_PER_T];
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) acc[i].x = acc[i].y = T(0);
    const int nout = nd * P;
    for (int j0 = s; j0 < e; j0 += 32) {
        if (threadIdx.x < 32) {
            const int j = j0 + threadIdx.x;
            C z1;
            C zk;
            zk.x = T(1); zk.y = T(0);
            double v[kMaxNd];
            if (j < e) {
                const double2 xj = xs[j];
                z1.x = T((xj.x - cx) * iw);
                z1.y = T((xj.y - cy) * iw);
                had_v(power, (xj.x - cx) * iw, (xj.y - cy) * iw, v);  // leaf-local densities
                const double tj = t[j];
                for (int d = 0; d < nd; ++d) qs[threadIdx.x * nd + d] = T(v[d] * tj);
            } else {
                z1.x = z1.y = T(0);
                for (int d = 0; d < nd; ++d) qs[threadIdx.x * nd + d] = T(0);
            }
            for (int k = 0; k < P; ++k) {
                pw[threadIdx.x * P + k] = zk;
                zk = cmul(zk, z1);
            }
        }
        __syncthreads();
        const int jn = min(32, e - j0);
#pragma unroll
        for (int i = 0; i < OUT_PER_T; ++i) {
            const int o = threadIdx.x + i * FMM_T;
            if (o < nout) {
                const int d = o / P, k = o - d * P;
                C a = acc[i];
                for (int jj = 0; jj < jn; ++jj) {
                    const T q = qs[jj * nd + d];
                    const C z = pw[jj * P + k];
                    a.x += q * z.x;
                    a.y += q * z.y;
                }
                acc[i] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) {
        const int o = threadIdx.x + i * FMM_T;
        if (o < nout) {
            const int d = o / P, k = o - d * P;
            C a = acc[i];
            if (k > 0) {
                const T sc = T(-1) / T(k);
                a.x *= sc;
                a.y *= sc;
            }
            mp[((size_t)b * nd + d) * P + k] = a;
        }
    }
}

// Box-local Hadamard factors: densities v_b and factors u_a are evaluated in the
// coordinates of the box they belong to, (z - c)/w.  Moving between frames mixes them
// with small level-invariant matrices (rows = new index, columns = old index):
//   slot cls (0..48):  v_l(z + o)       = sum_b S[l][b] v_b(z)    (M2L, o = source offset)
//   slot 49 + q:       v_l(z/2 + d_q)   = sum_b Rv[l][b] v_b(z)   (M2M, child quadrant q)
//   slot 53 + q:       u_l(z/2 + d_q)   = sum_a Ru[l][a] u_a(z)   (L2L)
// With these, every far-field term is O(1) in box units instead of |x|^2 / |x - y|^2.
constexpr int kMixSlots = 57;

// M2M: parents of level l (all non-leaf boxes of that level)
template <typename T>
__global__ void m2m_kernel(TreeView tv, int b0, int nd, int P, const typename C2T<T>::type *ops, const T *mix,
                           typename C2T<T>::type *mp) {
    using C = typename C2T<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);  // [nd][P] child multipole
    C *sh = sm + nd * P;                       // [nd][P] shifted to the parent centre
    const int b = b0 + blockIdx.x;
    const int nc = tv.nchild[b];
    if (nc == 0) return;
    const int nout = nd * P;
    C acc[OUT_PER_T];
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) acc[i].x = acc[i].y = T(0);
    for (int c = tv.child[b]; c < tv.child[b] + nc; ++c) {
        for (int i = threadIdx.x; i < nout; i += blockDim.x) sm[i] = mp[(size_t)c * nout + i];
        __syncthreads();
        const int q = (int)(tv.key[c] & 3);
        const C *A = ops + (size_t)q * P * P;
        const T *Rv = mix + (size_t)(49 + q) * nd * nd;
#pragma unroll
        for (int i = 0; i < OUT_PER_T; ++i) {
            const int o = threadIdx.x + i * FMM_T;
            if (o < nout) {
                const int d = o / P, l = o - d * P;
                C a;
                a.x = a.y = T(0);
                for (int k = 0; k <= l; ++k) cfma(a, A[l * P + k], sm[d * P + k]);
                sh[o] = a;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < OUT_PER_T; ++i) {
            const int o = threadIdx.x + i * FMM_T;
            if (o < nout) {
                const int d = o / P, l = o - d * P;
                C a = acc[i];
                for (int bb = 0; bb < nd; ++bb) {
                    const T r = Rv[d * nd + bb];
                    a.x += r * sh[bb * P + l].x;
                    a.y += r * sh[bb * P + l].y;
                }
                acc[i] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) {
        const int o = threadIdx.x + i * FMM_T;
        if (o < nout) mp[(size_t)b * nout + o] = acc[i];
    }
}

// M2L over V lists for boxes [b0, b0 + gridDim.x)
template <typename T>
__global__ void m2l_kernel(TreeView tv, int b0, const int *v_off, const int *v_src, const unsigned char *v_cls, int nd,
                           int P, int power, const typename C2T<T>::type *ops, const T *mix,
                           const typename C2T<T>::type *mp, typename C2T<T>::type *lc) {
    using C = typename C2T<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *src_m = reinterpret_cast<C *>(smem_raw);  // [nd][P] source multipole (source-local densities)
    C *sm = src_m + nd * P;                      // [nd][P] densities re-expressed about the target centre
    const int b = b0 + blockIdx.x;
    const int nout = nd * P;
    const double wb = box_width(tv.R, tv.level[b]);
    const T logw = T(log(wb));
    C acc[OUT_PER_T];
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) acc[i].x = acc[i].y = T(0);
    for (int v = v_off[b]; v < v_off[b + 1]; ++v) {
        const int src = v_src[v];
        for (int i = threadIdx.x; i < nout; i += blockDim.x) src_m[i] = mp[(size_t)src * nout + i];
        __syncthreads();
        const T *S = mix + (size_t)v_cls[v] * nd * nd;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int d = o / P, k = o - d * P;
            C a;
            a.x = a.y = T(0);
            for (int bb = 0; bb < nd; ++bb) {
                const T s = S[d * nd + bb];
                a.x += s * src_m[bb * P + k].x;
                a.y += s * src_m[bb * P + k].y;
            }
            sm[o] = a;
        }
        __syncthreads();
        const C *A = ops + (size_t)(8 + v_cls[v]) * P * P;
#pragma unroll
        for (int i = 0; i < OUT_PER_T; ++i) {
            const int o = threadIdx.x + i * FMM_T;
            if (o < nout) {
                const int d = o / P, l = o - d * P;
                C a = acc[i];
                const C *Ar = A + l * P;
                const C *mv = sm + d * P;
                for (int k = 0; k < P; ++k) cfma(a, Ar[k], mv[k]);
                if (l == 0) a.x += mv[0].x * logw;
                acc[i] = a;
            }
        }
        __syncthreads();
    }
    // |x - y|^{2m} = w^{2m} |x~ - y~|^{2m} in box units
    T wpow = T(1);
    for (int i = 0; i < power; ++i) wpow *= T(wb);
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) {
        const int o = threadIdx.x + i * FMM_T;
        if (o < nout) {
            C a = acc[i];
            a.x *= wpow;
            a.y *= wpow;
            lc[(size_t)b * nout + o] = a;
        }
    }
}

// L2L: boxes of one level receive their parent's local expansion
template <typename T>
__global__ void l2l_kernel(TreeView tv, int b0, int nd, int P, const typename C2T<T>::type *ops, const T *mix,
                           typename C2T<T>::type *lc) {
    using C = typename C2T<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);  // [nd][P] parent local expansions
    C *sh = sm + nd * P;                       // [nd][P] shifted to the child centre
    const int b = b0 + blockIdx.x;
    const int par = tv.parent[b];
    const int nout = nd * P;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) sm[i] = lc[(size_t)par * nout + i];
    __syncthreads();
    const int q = (int)(tv.key[b] & 3);
    const C *A = ops + (size_t)(4 + q) * P * P;
    const T *Ru = mix + (size_t)(53 + q) * nd * nd;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int d = o / P, m = o - d * P;
        C a;
        a.x = a.y = T(0);
        for (int l = m; l < P; ++l) cfma(a, A[m * P + l], sm[d * P + l]);
        sh[o] = a;
    }
    __syncthreads();
    // child factor a collects parent factor l through u_l(z/2 + d_q) = sum_a Ru[l][a] u_a(z)
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int a_ = o / P, m = o - a_ * P;
        C a = lc[(size_t)b * nout + o];
        for (int l = 0; l < nd; ++l) {
            const T r = Ru[l * nd + a_];
            a.x += r * sh[l * P + m].x;
            a.y += r * sh[l * P + m].y;
        }
        lc[(size_t)b * nout + o] = a;
    }
}

// L2P + Hadamard combination: y_i += sum_d u_d(x_i) Re L_d(x_i)
template <typename T>
__global__ void l2p_kernel(TreeView tv, const int *leaf_box, const double2 *xs, int power, int nd, int P,
                           const typename C2T<T>::type *lc, double *y) {
    using C = typename C2T<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int b = leaf_box[blockIdx.x];
    const int nout = nd * P;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) sm[i] = lc[(size_t)b * nout + i];
    __syncthreads();
    double cx, cy, w, iw;
    box_geom_iw(tv, b, cx, cy, w, iw);
    for (int j = tv.start[b] + threadIdx.x; j < tv.end[b]; j += blockDim.x) {
        const double2 xj = xs[j];
        C v;
        v.x = T((xj.x - cx) * iw);
        v.y = T((xj.y - cy) * iw);
        double u[kMaxNd];
        had_u(power, (xj.x - cx) * iw, (xj.y - cy) * iw, u);  // leaf-local factors
        double sum = 0.0;
        for (int d = 0; d < nd; ++d) {
            const C *L = sm + d * P;
            C h = L[P - 1];
            for (int l = P - 2; l >= 0; --l) {
                C t2 = cmul(h, v);
                h.x = t2.x + L[l].x;
                h.y = t2.y + L[l].y;
            }
            sum += u[d] * (double)h.x;
        }
        y[j] += sum;
    }
}

// ---------------------------------------------------------------- FP64 upward / downward passes
// The same arithmetic as the templated kernels above, arranged for the FP64 pipe: every
// thread of a block has work, dependent chains are short, and the children of a parent
// are processed together (two block barriers instead of twelve).
constexpr int UD_T = 256;    // P2M threads at most
constexpr int UD_MAX = 1024;  // M2M / L2L threads at most
// Block sizes that leave no lane idle where the work is (a warp instruction on the FP64
// pipe costs the same with one lane as with 32): the fewest rounds of at most `cap`
// threads over `items`, each round rounded up to whole warps.
static int even_threads(int items, int cap) {
    const int rounds = (items + cap - 1) / cap;
    return std::max(32, ((items + rounds - 1) / rounds + 31) / 32 * 32);
}
// P2M: one thread per output (nd P of them, at most three rounds) and four per point of
// a chunk of blockDim / 4 points; M2M / L2L: one thread per (child, density, row pair)
static int p2m_threads(int nd, int P) { return even_threads(nd * P, UD_T); }
static int shift_threads(int nd, int P) { return even_threads(4 * nd * ((P + 1) / 2), UD_MAX); }
__device__ double g_neg_inv_k[kMaxP];  // -1/k for 1 <= k < kMaxP (host division, correctly rounded)

// P2M: chunks of blockDim / 4 points (at most 64); four threads per point build the powers zeta^k, each a
// quarter of k from its own starting power; then one thread per output (d, k) sums the
// chunk.  a_0 = sum q, a_k = -sum q zeta^k / k (box-width scaled, fmm.cu header).
template <int ND>  // density count (static, so the Hadamard factors stay in registers)
__global__ void __launch_bounds__(UD_T) p2m64_kernel(TreeView tv, const int *leaf_box, const double2 *xs,
                                                    const double *t, int power, int P, double2 *mp) {
    constexpr int nd = ND;
    extern __shared__ double2 p2m_sm[];
    double2 *pw = p2m_sm;                                 // [64][P]
    double *qs = reinterpret_cast<double *>(pw + 64 * P);  // [64][nd]
    const int b = leaf_box[blockIdx.x];
    double cx, cy, w, iw;
    box_geom_iw(tv, b, cx, cy, w, iw);
    const int s = tv.start[b], e = tv.end[b];
    const int nout = nd * P;
    const int Q = (P + 3) / 4;
    double2 acc[OUT_PER_T];
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) acc[i] = make_double2(0.0, 0.0);
    const int CH = blockDim.x >> 2;  // points per chunk (at most 64)
    for (int j0 = s; j0 < e; j0 += CH) {
        const int jn = min(CH, e - j0);
        {
            const int jp = threadIdx.x >> 2, q = threadIdx.x & 3;
            if (jp < jn) {
                const double2 xj = xs[j0 + jp];
                const double2 z = make_double2((xj.x - cx) * iw, (xj.y - cy) * iw);
                double2 zk = make_double2(1.0, 0.0), base = z;
                for (int e2 = q * Q; e2 > 0; e2 >>= 1) {
                    if (e2 & 1) zk = cmul(zk, base);
                    base = cmul(base, base);
                }
                const int k1 = min(P, (q + 1) * Q);
                for (int k = q * Q; k < k1; ++k) {
                    pw[jp * P + k] = zk;
                    zk = cmul(zk, z);
                }
                if (q == 0) {
                    double v[kMaxNd];
                    had_v(power, z.x, z.y, v);
                    const double tj = t[j0 + jp];
                    for (int d = 0; d < nd; ++d) qs[jp * nd + d] = v[d] * tj;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < OUT_PER_T; ++i) {
            const int o = threadIdx.x + i * (int)blockDim.x;
            if (o < nout) {
                const int d = o / P, k = o - d * P;
                double2 a = acc[i];
                for (int jj = 0; jj < jn; ++jj) {
                    const double q = qs[jj * nd + d];
                    const double2 z = pw[jj * P + k];
                    a.x = fma(q, z.x, a.x);
                    a.y = fma(q, z.y, a.y);
                }
                acc[i] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < OUT_PER_T; ++i) {
        const int o = threadIdx.x + i * (int)blockDim.x;
        if (o < nout) {
            const int d = o / P, k = o - d * P;
            double2 a = acc[i];
            if (k > 0) {
                const double sc = g_neg_inv_k[k];  // -1/k, correctly rounded (no FP64 division)
                a.x *= sc;
                a.y *= sc;
            }
            mp[((size_t)b * nd + d) * P + k] = a;
        }
    }
}

// M2M for the parents of one level: all children load and shift at once.  The shift of
// quadrant q factors as e^{i th_q l} R[l][k] e^{-i th_q k} with a real lower-triangular
// core R common to the four quadrants, so the O(P^2) part is real x complex (2 FMA per
// entry instead of 4).  Each thread takes row pairs (l, P-1-l) to balance the triangle;
// then the parent sums the children through the frame changes Rv (mix slots 49 + q).
__global__ void __launch_bounds__(UD_MAX) m2m64_kernel(TreeView tv, int b0, int nd, int P, const double *R,
                                                    const double2 *ph, const double *mix, double2 *mp) {
    extern __shared__ double2 m2m_sm[];
    const int b = b0 + blockIdx.x;
    const int nc = tv.nchild[b];
    if (nc == 0) return;
    const int nout = nd * P, c0 = tv.child[b];
    double2 *ch = m2m_sm, *sh = m2m_sm + 4 * nout;
    for (int i = threadIdx.x; i < nc * nout; i += (int)blockDim.x) {
        const int c = i / nout, k = (i - c * nout) % P;
        const double2 a = mp[(size_t)c0 * nout + i], e = ph[(size_t)(tv.key[c0 + c] & 3) * P + k];
        ch[i] = make_double2(fma(a.x, e.x, a.y * e.y), fma(a.y, e.x, -a.x * e.y));  // a e^{-i th k}
    }
    __syncthreads();
    const int half = (P + 1) / 2;
    for (int it = threadIdx.x; it < nc * nd * half; it += (int)blockDim.x) {
        const int c = it / (nd * half), r = it - c * nd * half, d = r / half, p = r - d * half;
        const double2 *ephq = ph + (size_t)(tv.key[c0 + c] & 3) * P;
        const double2 *src = ch + c * nout + d * P;
        for (int h = 0; h < 2; ++h) {
            const int l = h == 0 ? p : P - 1 - p;
            if (h == 1 && l == p) break;
            const double *Rr = R + (size_t)l * P;
            double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
            int k = 0;
            for (; k + 1 <= l; k += 2) {
                const double r0 = Rr[k], r1 = Rr[k + 1];
                const double2 m0 = src[k], m1 = src[k + 1];
                ax = fma(r0, m0.x, ax);
                ay = fma(r0, m0.y, ay);
                bx = fma(r1, m1.x, bx);
                by = fma(r1, m1.y, by);
            }
            if (k <= l) {
                const double r0 = Rr[k];
                const double2 m0 = src[k];
                ax = fma(r0, m0.x, ax);
                ay = fma(r0, m0.y, ay);
            }
            const double zx = ax + bx, zy = ay + by;
            const double2 e = ephq[l];  // z e^{i th l}
            sh[c * nout + d * P + l] = make_double2(fma(zx, e.x, -zy * e.y), fma(zx, e.y, zy * e.x));
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += (int)blockDim.x) {
        const int d = o / P, l = o - d * P;
        double ax = 0.0, ay = 0.0;
        for (int c = 0; c < nc; ++c) {
            const double *Rv = mix + (size_t)(49 + (tv.key[c0 + c] & 3)) * nd * nd + d * nd;
            for (int bb = 0; bb < nd; ++bb) {
                const double r = Rv[bb];
                if (r != 0.0) {
                    const double2 v = sh[c * nout + bb * P + l];
                    ax = fma(r, v.x, ax);
                    ay = fma(r, v.y, ay);
                }
            }
        }
        mp[(size_t)b * nout + o] = make_double2(ax, ay);
    }
}

// L2L for the parents of one level: the parent's local expansion loads once, takes each
// child's phase e^{i th_q l}, shifts through the real upper-triangular core (rows m
// paired with P-1-m: sum over l >= m), takes e^{-i th_q m}, and mixes through Ru (mix
// slots 53 + q) into the child's local expansion.
__global__ void __launch_bounds__(UD_MAX) l2l64_kernel(TreeView tv, int b0, int nd, int P, const double *R,
                                                    const double2 *ph, const double *mix, double2 *lc) {
    extern __shared__ double2 l2l_sm[];
    const int b = b0 + blockIdx.x;
    const int nc = tv.nchild[b];
    if (nc == 0) return;
    const int nout = nd * P, c0 = tv.child[b];
    double2 *y = l2l_sm, *sh = l2l_sm + 4 * nout;
    for (int i = threadIdx.x; i < nc * nout; i += (int)blockDim.x) {
        const int c = i / nout, o = i - c * nout, l = o % P;
        const double2 v = lc[(size_t)b * nout + o], e = ph[(size_t)(tv.key[c0 + c] & 3) * P + l];
        y[i] = make_double2(fma(v.x, e.x, -v.y * e.y), fma(v.x, e.y, v.y * e.x));  // b e^{i th l}
    }
    __syncthreads();
    const int half = (P + 1) / 2;
    for (int it = threadIdx.x; it < nc * nd * half; it += (int)blockDim.x) {
        const int c = it / (nd * half), r = it - c * nd * half, d = r / half, p = r - d * half;
        const double2 *ephq = ph + (size_t)(tv.key[c0 + c] & 3) * P;
        const double2 *src = y + c * nout + d * P;
        for (int h = 0; h < 2; ++h) {
            const int m = h == 0 ? p : P - 1 - p;
            if (h == 1 && m == p) break;
            const double *Rr = R + (size_t)m * P;
            double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
            int l = m;
            for (; l + 1 < P; l += 2) {
                const double r0 = Rr[l], r1 = Rr[l + 1];
                const double2 v0 = src[l], v1 = src[l + 1];
                ax = fma(r0, v0.x, ax);
                ay = fma(r0, v0.y, ay);
                bx = fma(r1, v1.x, bx);
                by = fma(r1, v1.y, by);
            }
            if (l < P) {
                const double r0 = Rr[l];
                const double2 v0 = src[l];
                ax = fma(r0, v0.x, ax);
                ay = fma(r0, v0.y, ay);
            }
            const double zx = ax + bx, zy = ay + by;
            const double2 e = ephq[m];  // z e^{-i th m}
            sh[c * nout + d * P + m] = make_double2(fma(zx, e.x, zy * e.y), fma(zy, e.x, -zx * e.y));
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < nc * nout; it += (int)blockDim.x) {
        const int c = it / nout, o = it - c * nout, a_ = o / P, m = o - a_ * P;
        const double *Ru = mix + (size_t)(53 + (tv.key[c0 + c] & 3)) * nd * nd;
        double2 acc = lc[(size_t)(c0 + c) * nout + o];
        for (int l = 0; l < nd; ++l) {
            const double r = Ru[l * nd + a_];
            if (r != 0.0) {
                const double2 v = sh[c * nout + l * P + m];
                acc.x = fma(r, v.x, acc.x);
                acc.y = fma(r, v.y, acc.y);
            }
        }
        lc[(size_t)(c0 + c) * nout + o] = acc;
    }
}

// L2P with the powers z^k shared by the densities: thread per point, P steps of one
// complex product (4 FP64) and, per density, two FMAs on the real part (Re(L_d(z)) is all
// the Hadamard combination sum_d u_d Re(L_d(z)) needs), against 4 FP64 per density and
// step for separate complex Horner recurrences.  |z| <= sqrt(2)/2 inside the leaf, so the
// direct sum of the powers is as accurate as Horner's rule.
constexpr int L2P_T = 64;
template <int ND>
__global__ void __launch_bounds__(L2P_T) l2p64_kernel(TreeView tv, const int *leaf_box, const double2 *xs,
                                                     int power, int P, const double2 *lc, double *y) {
    extern __shared__ double2 l2p_sm[];
    const int b = leaf_box[blockIdx.x];
    const int nout = ND * P;
    for (int i = threadIdx.x; i < nout; i += L2P_T) l2p_sm[i] = lc[(size_t)b * nout + i];
    __syncthreads();
    double cx, cy, w, iw;
    box_geom_iw(tv, b, cx, cy, w, iw);
    const int s = tv.start[b], e = tv.end[b];
    for (int j = s + threadIdx.x; j < e; j += L2P_T) {
        const double2 xj = xs[j];
        const double vx = (xj.x - cx) * iw, vy = (xj.y - cy) * iw;
        double u[kMaxNd];
        had_u(power, vx, vy, u);
        double acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = 0.0;
        double zx = 1.0, zy = 0.0;
        for (int k = 0; k < P; ++k) {
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const double2 L = l2p_sm[d * P + k];
                acc[d] = fma(L.x, zx, fma(-L.y, zy, acc[d]));
            }
            const double nx = fma(zx, vx, -zy * vy);
            zy = fma(zx, vy, zy * vx);
            zx = nx;
        }
        double sum = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) sum = fma(u[d], acc[d], sum);
        y[j] += sum;
    }
}

// near field: y_i = sum_{j in near(leaf(i)), j != i} phi(|x_i - x_j|) t_j  (full phi, Eq. 1.2)
template <typename T, int K>
__device__ __forceinline__ T phi_r2(T r2) {
    if (K == 1) return sqrt(r2);
    if (K == 2) return T(0.5) * r2 * log(r2);
    if (K == 3) return r2 * sqrt(r2);
    if (K == 4) return T(0.5) * r2 * r2 * log(r2);
    return r2 * r2 * sqrt(r2);
}
template <>
__device__ __forceinline__ float phi_r2<float, 2>(float r2) { return 0.5f * r2 * __logf(r2); }
template <>
__device__ __forceinline__ float phi_r2<float, 4>(float r2) { return 0.5f * r2 * r2 * __logf(r2); }

// Table-driven natural logarithm in FP64, after P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic"
// (ACM TOMS 16(4), 1990):  x = 2^e m with m in [1, 2);  F_j = 1 + j/2048 is the grid
// point nearest m;  log x = e log 2 + log F_j + log(1 + r),  r = m/F_j - 1 (one FMA
// with the tabulated 1/F_j), |r| < 2^-12, log(1 + r) ~ r - r^2/2 + r^3/3 (truncation
// below 2^-50).  e log 2 comes from a table over biased exponents 768..1026 (smaller
// exponents clamp: there x < 2^-255 and x log x vanishes to 1e-74).  x = 0 returns a
// finite value, so x log x is 0 there.  FP64 work: 4 DFMA + 1 DADD.
constexpr int kLogTab = 2049;
constexpr int kExpLo = 768, kExpTab = 259;
__device__ double2 g_logtab[kLogTab];  // (log F_j, 1/F_j)
__device__ double g_eln2[kExpTab];     // (e - 1023) log 2 for biased e = kExpLo + i

__device__ __forceinline__ double tab_log(double x, const double2 *tab, const double *eln2) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int j = (((hi >> 8) & 0xfff) + 1) >> 1;
    const int ei = min(max((hi >> 20) - kExpLo, 0), kExpTab - 1);
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
    const double2 fj = tab[j];
    const double r = fma(m, fj.y, -1.0);
    double c = fma(r, 0.33333333333333333, -0.5);
    c = fma(c, r, 1.0);
    return fma(c, r, fj.x + eln2[ei]);
}

constexpr int P2P_T = kP2PThreads;

template <typename T, int K>
struct UsesLogTab {
    static constexpr bool value = sizeof(T) == 8 && (K % 2 == 0);
};

// Near field of one leaf per block iteration (persistent blocks: the logarithm tables
// load once per block).  G threads share a target (power of two <= 32) so small
// leaves keep the block busy.  For the FP64 log kernel the sum is sum_j r^2 log(r^2) t_j,
// halved once at the end (phi = r^2 log r = r^2 log(r^2) / 2, r^k log r likewise).
template <typename T, int K>
__global__ void __launch_bounds__(P2P_T) p2p_kernel(TreeView tv, int nleaf, const int *leaf_box, const int *near_off,
                                                   const int2 *near_rng, const double2 *xs, const double *t,
                                                   double *y) {
    __shared__ T sx[P2P_T], sy[P2P_T], st[P2P_T];
    extern __shared__ double2 logtab_sm[];  // [kLogTab] (log F, 1/F), then [kExpTab] e log 2
    constexpr bool kTab = UsesLogTab<T, K>::value;
    const double *eln2 = reinterpret_cast<const double *>(logtab_sm + kLogTab);
    if (kTab) {
        for (int i = threadIdx.x; i < kLogTab; i += P2P_T) logtab_sm[i] = g_logtab[i];
        for (int i = threadIdx.x; i < kExpTab; i += P2P_T)
            reinterpret_cast<double *>(logtab_sm + kLogTab)[i] = g_eln2[i];
        __syncthreads();
    }
    for (int li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const int b = leaf_box[li];
        double cx, cy, w;
        box_geom(tv, b, cx, cy, w);
        const int s = tv.start[b], e = tv.end[b];
        const int nt = e - s;
        int G = 1;
        while (G < 32 && nt * G * 2 <= P2P_T) G <<= 1;
        const int tpp = P2P_T / G;
        const int sub = threadIdx.x & (G - 1);
        for (int i0 = s; i0 < e; i0 += tpp) {
            const int i = i0 + threadIdx.x / G;
            T xi = 0, yi = 0;
            if (i < e) {
                const double2 p = xs[i];
                xi = T(p.x - cx);
                yi = T(p.y - cy);
            }
            T acc = 0;
            for (int r = near_off[b]; r < near_off[b + 1]; ++r) {
                const int2 rg = near_rng[r];
                for (int j0 = rg.x; j0 < rg.y; j0 += P2P_T) {
                    const int j = j0 + threadIdx.x;
                    __syncthreads();
                    if (j < rg.y) {
                        const double2 p = xs[j];
                        sx[threadIdx.x] = T(p.x - cx);
                        sy[threadIdx.x] = T(p.y - cy);
                        st[threadIdx.x] = T(t[j]);
                    }
                    __syncthreads();
                    const int jn = min(P2P_T, rg.y - j0);
                    for (int jj = sub; jj < jn; jj += G) {
                        const T dx = xi - sx[jj], dy = yi - sy[jj];
                        const T r2 = fma(dy, dy, dx * dx);
                        if constexpr (kTab) {
                            const double L = tab_log(r2, logtab_sm, eln2);
                            const double f = K == 2 ? r2 * L : (r2 * r2) * L;
                            acc = fma(f, st[jj], acc);
                        } else {
                            if (r2 > T(0)) acc += phi_r2<T, K>(r2) * st[jj];
                        }
                    }
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (sub == 0 && i < e) y[i] = kTab ? 0.5 * (double)acc : (double)acc;
        }
    }
}

// phi(r) up to the factor 1/2 of the log kernels (applied once per sum), from
// r^2 = a_i + a_j - 2 (x_i x_j + y_i y_j) with a = x^2 + y^2 of coordinates
// centred on the target leaf (mx = -2 x_i, my = -2 y_i kept per row, a_j per column):
// one DADD and two DFMA instead of two DADD, a DMUL and a DFMA.  The cancellation error
// is at most eps (a_i + a_j), small beside every term of the sum; a self pair may give a
// tiny non-zero r^2 instead of 0, whose contribution (r^2 log r^2) is below 1e-17.
// For odd k the square root turns that absolute error into eps (a_i + a_j) / (2 r) in
// r -- large for close pairs, and a self pair would get r ~ 1e-8 w instead of 0 -- so
// odd k forms r^2 from the differences (x_i = -mx / 2 exactly).
template <int K, bool kTab>
__device__ __forceinline__ double phi_sym_a(double mx, double my, double ai, double xj, double yj, double aj,
                                            const double2 *tab, const double *eln2) {
    if constexpr (kTab) {
        const double r2 = fma(mx, xj, fma(my, yj, ai + aj));
        const double L = tab_log(r2, tab, eln2);
        return K == 2 ? r2 * L : (r2 * r2) * L;
    } else {
        const double dx = fma(-0.5, mx, -xj), dy = fma(-0.5, my, -yj);
        return phi_r2<double, K>(fma(dx, dx, dy * dy));
    }
}

// Symmetric FP64 near field: every pair of points in different leaves is evaluated once.
// Leaf b sums its own box (rows only) and each near range R after it in Morton order:
// rows into y, columns (sum_{i in b} phi_ij t_i, accumulated systolically across the
// lanes that share a source, then summed over the warps in a fixed order) into the
// scratch slot of (b, R).
// Ranges before b arrive through p2p_gather from the slots of the earlier leaves, which
// holds because the near relation is symmetric (its complement, the V-list relation,
// is).  One pass per leaf: the plan enables this path only when every leaf has at most
// P2P_T points.

template <int K>
__global__ void __launch_bounds__(P2P_T) p2p_sym_kernel(TreeView tv, int nleaf, const int *leaf_box,
                                                       const int *order, int *ticket, const int *near_off,
                                                       const int2 *near_rng, const int *slot_off, const double2 *xs,
                                                       const double *t, double *y, double *scratch) {
    __shared__ double sx[P2P_T], sy[P2P_T], sa[P2P_T], st[P2P_T];
    __shared__ double colp[P2P_T / 32][P2P_T];
    __shared__ int2 ups[kMaxUpRanges];  // (start, prefix length) of the ranges after the leaf
    __shared__ int nup, next_leaf;
    extern __shared__ double2 logtab_sm[];
    constexpr bool kTab = (K % 2 == 0);
    const double *eln2 = reinterpret_cast<const double *>(logtab_sm + kLogTab);
    if (kTab) {
        for (int i = threadIdx.x; i < kLogTab; i += P2P_T) logtab_sm[i] = g_logtab[i];
        for (int i = threadIdx.x; i < kExpTab; i += P2P_T)
            reinterpret_cast<double *>(logtab_sm + kLogTab)[i] = g_eln2[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double scale = kTab ? 0.5 : 1.0;  // r^k log r = r^k log(r^2) / 2
    for (;;) {
        // dynamic schedule over the leaves in decreasing cost order
        if (threadIdx.x == 0) next_leaf = atomicAdd(ticket, 1);
        __syncthreads();
        const int oi = next_leaf;
        if (oi >= nleaf) break;
        const int li = order[oi];
        const int b = leaf_box[li];
        double cx, cy, w;
        box_geom(tv, b, cx, cy, w);
        const int s = tv.start[b], e = tv.end[b];
        const int nt = e - s;
        int G = 1;
        while (G < 32 && nt * G * 2 <= P2P_T) G <<= 1;
        const int sub = threadIdx.x & (G - 1);
        const int i = s + threadIdx.x / G;
        const bool act = i < e;
        // warps without an active target skip the arithmetic (warp-uniform)
        const int nwarp = (nt * G + 31) >> 5;
        const bool wact = warp < nwarp;
        double mx = 0, my = 0, ai = 0, ti = 0;
        if (act) {
            const double2 p = xs[i];
            const double xi = p.x - cx, yi = p.y - cy;
            mx = -2.0 * xi;
            my = -2.0 * yi;
            ai = fma(yi, yi, xi * xi);
            ti = t[i];
        }
        // own box (rows only) and the list of ranges after the leaf
        if (threadIdx.x == 0) {
            int n = 0, pre = 0;
            for (int r = near_off[b]; r < near_off[b + 1]; ++r) {
                const int2 rg = near_rng[r];
                if (rg.x >= e && n < kMaxUpRanges - 1) {  // the plan guarantees fewer
                    ups[n++] = make_int2(rg.x, pre);
                    pre += rg.y - rg.x;
                }
            }
            nup = n;
            ups[n] = make_int2(0, pre);  // total length
        }
        if (threadIdx.x < nt) {
            const double2 p = xs[s + threadIdx.x];
            const double xj = p.x - cx, yj = p.y - cy;
            sx[threadIdx.x] = xj;
            sy[threadIdx.x] = yj;
            sa[threadIdx.x] = fma(yj, yj, xj * xj);
            st[threadIdx.x] = t[s + threadIdx.x];
        }
        __syncthreads();
        double acc = 0;
        if (wact) {
            const int nk = (nt + G - 1) / G;
            for (int k = 0; k < nk; ++k) {
                const int jj = k * G + sub;
                const bool v = jj < nt;
                const int jc = v ? jj : 0;
                const double f = v ? phi_sym_a<K, kTab>(mx, my, ai, sx[jc], sy[jc], sa[jc], logtab_sm, eln2) : 0.0;
                acc = fma(f, st[jc], acc);
            }
        }
        const int nu = nup, tot = ups[nu].y;
        const int slot = slot_off[li];
        int r0 = 0;  // range of the chunk's first column (advances monotonically)
        for (int c0 = 0; c0 < tot; c0 += P2P_T) {
            __syncthreads();
            {
                const int g = c0 + threadIdx.x;
                if (g < tot) {
                    int r = r0;
                    while (ups[r + 1].y <= g) ++r;
                    const int j = ups[r].x + (g - ups[r].y);
                    const double2 p = xs[j];
                    const double xj = p.x - cx, yj = p.y - cy;
                    sx[threadIdx.x] = xj;
                    sy[threadIdx.x] = yj;
                    sa[threadIdx.x] = fma(yj, yj, xj * xj);
                    st[threadIdx.x] = t[j];
                }
            }
            while (r0 + 1 < nu && ups[r0 + 1].y <= c0 + P2P_T) ++r0;
            __syncthreads();
            const int jn = min(P2P_T, tot - c0);
            if (wact) {
                // systolic column sums: the S = 32/G lanes of a sub-group (same sub) take the
                // columns of a tile in rotation, step k: lane u on column (k + u) mod S, and
                // pass the running column sum to lane u - 1, so after S steps lane u holds
                // the sum of column u over the sub-group's targets (one FMA per pair)
                const int S = 32 / G, u = lane / G;
                for (int t0 = 0; t0 < jn; t0 += 32) {
                    double cs = 0.0;
                    for (int k = 0; k < S; ++k) {
                        const int jj = t0 + ((k + u) & (S - 1)) * G + sub;
                        const bool v = jj < jn;
                        const int jc = v ? jj : 0;
                        const double f = v ? phi_sym_a<K, kTab>(mx, my, ai, sx[jc], sy[jc], sa[jc], logtab_sm, eln2)
                                           : 0.0;
                        acc = fma(f, st[jc], acc);
                        cs = fma(f, ti, cs);
                        cs = __shfl_sync(0xffffffffu, cs, (lane + G) & 31);
                    }
                    const int jo = t0 + u * G + sub;
                    if (jo < jn) colp[warp][jo] = cs;
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < jn; q += P2P_T) {
                double sum = 0;
                for (int w2 = 0; w2 < nwarp; ++w2) sum += colp[w2][q];
                scratch[slot + c0 + q] = scale * sum;
            }
        }
        if (wact) {
            for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (sub == 0 && act) y[i] = scale * acc;
        }
        __syncthreads();
    }
}

// y_j += the column sums of the earlier leaves whose near ranges contain j's leaf
// (ascending slot order: deterministic)
__global__ void p2p_gather(TreeView tv, const int *leaf_box, const int *point_leaf, const int *goff,
                           const int *gbase, int64_t n, const double *scratch, double *y) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int d = point_leaf[j];
    const int o = (int)j - tv.start[leaf_box[d]];
    double sum = 0;
    for (int p = goff[d]; p < goff[d + 1]; ++p) sum += scratch[gbase[p] + o];
    y[j] += sum;
}

// exact O(n^2) product, FP64
template <int K>
__global__ void dense_kernel(const double2 *x, int64_t n, const double *t, double *out) {
    __shared__ double sx[256], sy[256], st[256];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double xi = 0, yi = 0;
    if (i < n) { xi = x[i].x; yi = x[i].y; }
    double acc = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 256) {
        __syncthreads();
        if (j0 + threadIdx.x < n) {
            sx[threadIdx.x] = x[j0 + threadIdx.x].x;
            sy[threadIdx.x] = x[j0 + threadIdx.x].y;
            st[threadIdx.x] = t[j0 + threadIdx.x];
        }
        __syncthreads();
        const int jn = (int)min((int64_t)256, n - j0);
        for (int jj = 0; jj < jn; ++jj) {
            const double dx = xi - sx[jj], dy = yi - sy[jj];
            const double r2 = dx * dx + dy * dy;
            if (r2 > 0) acc += phi_r2<double, K>(r2) * st[jj];
        }
    }
    if (i < n) out[i] = acc;
}

template <typename T>
typename C2T<T>::type *mp_buf(Fmm &f);
template <>
double2 *mp_buf<double>(Fmm &f) { return f.mp64.get(); }
template <>
float2 *mp_buf<float>(Fmm &f) { return f.mp32.get(); }
template <typename T>
typename C2T<T>::type *lc_buf(Fmm &f);
template <>
double2 *lc_buf<double>(Fmm &f) { return f.lc64.get(); }
template <>
float2 *lc_buf<float>(Fmm &f) { return f.lc32.get(); }
template <typename T>
const typename C2T<T>::type *ops_buf(const Fmm &f);
template <>
const double2 *ops_buf<double>(const Fmm &f) { return f.ops64.get(); }
template <>
const float2 *ops_buf<float>(const Fmm &f) { return f.ops32.get(); }

template <typename T>
const T *mix_buf(const Fmm &f);
template <>
const double *mix_buf<double>(const Fmm &f) { return f.mix64.get(); }
template <>
const float *mix_buf<float>(const Fmm &f) { return f.mix32.get(); }

template <typename T>
static int P_of(const Fmm &f) { return sizeof(T) == 8 ? f.P : f.P32; }

// host copies of the Hadamard factor lists (same definitions as had_u / had_v)
static void host_had(int power, long double x, long double y, long double *u, long double *v) {
    const long double a = x * x + y * y;
    if (power == 0) {
        u[0] = v[0] = 1;
    } else if (power == 2) {
        v[0] = 1; v[1] = a; v[2] = x; v[3] = y;
        u[0] = a; u[1] = 1; u[2] = -2 * x; u[3] = -2 * y;
    } else {
        v[0] = 1; v[1] = a * a; v[2] = x; v[3] = y; v[4] = a * x; v[5] = a * y; v[6] = x * x; v[7] = x * y;
        v[8] = y * y;
        u[0] = a * a; u[1] = 1; u[2] = -4 * a * x; u[3] = -4 * a * y; u[4] = -4 * x; u[5] = -4 * y;
        u[6] = 4 * x * x + 2 * a; u[7] = 8 * x * y; u[8] = 4 * y * y + 2 * a;
    }
}

// Frame-change matrices of the factor lists (see kMixSlots): G with f_l(alpha z + beta) =
// sum_b G[l][b] f_b(z), solved exactly (the lists span affinely closed polynomial spaces)
// by least squares on a 7 x 7 grid in long double.
static std::vector<long double> build_mix(int power, int nd) {
    std::vector<long double> out((size_t)kMixSlots * nd * nd, 0.0L);
    auto solve = [&](bool use_u, long double alpha, long double bx, long double by, long double *dst) {
        const int N = 49;
        std::vector<long double> F0((size_t)N * nd), F1((size_t)N * nd);
        long double u[10], v[10];
        for (int i = 0; i < N; ++i) {
            const long double zx = -0.6L + 0.2L * (i % 7), zy = -0.6L + 0.2L * (i / 7);
            host_had(power, zx, zy, u, v);
            for (int b = 0; b < nd; ++b) F0[(size_t)i * nd + b] = use_u ? u[b] : v[b];
            host_had(power, alpha * zx + bx, alpha * zy + by, u, v);
            for (int b = 0; b < nd; ++b) F1[(size_t)i * nd + b] = use_u ? u[b] : v[b];
        }
        // normal equations (F0' F0) X = F0' F1, X[b][l] = G[l][b]
        std::vector<long double> A((size_t)nd * nd, 0), Bm((size_t)nd * nd, 0);
        for (int i = 0; i < N; ++i)
            for (int r = 0; r < nd; ++r)
                for (int c = 0; c < nd; ++c) {
                    A[(size_t)r * nd + c] += F0[(size_t)i * nd + r] * F0[(size_t)i * nd + c];
                    Bm[(size_t)r * nd + c] += F0[(size_t)i * nd + r] * F1[(size_t)i * nd + c];
                }
        for (int c = 0; c < nd; ++c) {  // Gauss-Jordan with partial pivoting
            int piv = c;
            for (int r = c + 1; r < nd; ++r)
                if (std::fabs(A[(size_t)r * nd + c]) > std::fabs(A[(size_t)piv * nd + c])) piv = r;
            for (int j = 0; j < nd; ++j) {
                std::swap(A[(size_t)c * nd + j], A[(size_t)piv * nd + j]);
                std::swap(Bm[(size_t)c * nd + j], Bm[(size_t)piv * nd + j]);
            }
            const long double d = A[(size_t)c * nd + c];
            for (int j = 0; j < nd; ++j) {
                A[(size_t)c * nd + j] /= d;
                Bm[(size_t)c * nd + j] /= d;
            }
            for (int r = 0; r < nd; ++r) {
                if (r == c) continue;
                const long double fct = A[(size_t)r * nd + c];
                if (fct == 0) continue;
                for (int j = 0; j < nd; ++j) {
                    A[(size_t)r * nd + j] -= fct * A[(size_t)c * nd + j];
                    Bm[(size_t)r * nd + j] -= fct * Bm[(size_t)c * nd + j];
                }
            }
        }
        for (int l = 0; l < nd; ++l)
            for (int b = 0; b < nd; ++b) {
                long double g = Bm[(size_t)b * nd + l];
                dst[(size_t)l * nd + b] = std::fabs(g) < 1e-15L ? 0.0L : g;
            }
    };
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy)
            solve(false, 1.0L, (long double)dx, (long double)dy, out.data() + (size_t)((dx + 3) * 7 + (dy + 3)) * nd * nd);
    for (int q = 0; q < 4; ++q) {
        const long double bx = (q & 1) ? 0.25L : -0.25L, by = (q & 2) ? 0.25L : -0.25L;
        solve(false, 0.5L, bx, by, out.data() + (size_t)(49 + q) * nd * nd);
        solve(true, 0.5L, bx, by, out.data() + (size_t)(53 + q) * nd * nd);
    }
    return out;
}

template <typename T>
static void ensure_bufs(Fmm &f, const Tree &t) {
    const size_t sz = (size_t)t.nbox * f.nd * P_of<T>(f);
    if (sizeof(T) == 8) {
        if (f.mp64.n != sz) { f.mp64.alloc(sz); f.lc64.alloc(sz); }
    } else {
        if (f.mp32.n != sz) { f.mp32.alloc(sz); f.lc32.alloc(sz); }
    }
}

// dynamic shared memory of the FP64 passes exceeds 48 KB for nd = 9, P = 61 (M2M: 8 nd P
// complex values, 70 KB)
static void set_pass_smem_limits() {
    once_per_device(4, [] {
    const int lim = 100 * 1024;
    PHS_CUDA(cudaFuncSetAttribute(p2m64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    PHS_CUDA(cudaFuncSetAttribute(p2m64_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    PHS_CUDA(cudaFuncSetAttribute(p2m64_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    PHS_CUDA(cudaFuncSetAttribute(m2m64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    PHS_CUDA(cudaFuncSetAttribute(l2l64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    });
}

template <typename T>
static void upward(Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, typename C2T<T>::type *mp,
                   const typename C2T<T>::type *ops, int P, cudaStream_t s, bool ff = false) {
    using C = typename C2T<T>::type;
    TreeView tv = tree_view(t);
    const int nd = f.nd;
    const size_t esz = (size_t)nd * P * sizeof(C);
    if constexpr (sizeof(T) == 8) {
        set_pass_smem_limits();
        const size_t sm = (size_t)64 * P * sizeof(double2) + (size_t)64 * nd * sizeof(double);
        if (ff) p2m_ff_launch(f, t, ps, tv_sorted, mp, s);
        else if (nd == 4) p2m64_kernel<4><<<t.nleaf, p2m_threads(nd, P), sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, P, mp);
        else if (nd == 9) p2m64_kernel<9><<<t.nleaf, p2m_threads(nd, P), sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, P, mp);
        else p2m64_kernel<1><<<t.nleaf, p2m_threads(nd, P), sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, P, mp);
        PHS_LAUNCH_CHECK();
        for (int l = t.depth - 1; l >= 0; --l) {
            const int b0 = t.lvl_off[l], nb = t.lvl_off[l + 1] - b0;
            if (nb > 0 && ff) m2m_ff_launch(f, t, b0, nb, mp, s);
            else if (nb > 0)
                m2m64_kernel<<<nb, shift_threads(nd, P), 8 * esz, s>>>(tv, b0, nd, P, f.shift_r.get(), f.shift_ph.get(), mix_buf<T>(f),
                                                       mp);
            PHS_LAUNCH_CHECK();
        }
        return;
    }
    const size_t p2m_smem = 32 * P * sizeof(C) + 32 * nd * sizeof(T);
    p2m_kernel<T><<<t.nleaf, FMM_T, p2m_smem, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, nd, P, mp);
    PHS_LAUNCH_CHECK();
    for (int l = t.depth - 1; l >= 0; --l) {
        const int b0 = t.lvl_off[l], nb = t.lvl_off[l + 1] - b0;
        if (nb > 0) m2m_kernel<T><<<nb, FMM_T, 2 * esz, s>>>(tv, b0, nd, P, ops, mix_buf<T>(f), mp);
        PHS_LAUNCH_CHECK();
    }
}
template <typename T>
static void m2l_pass(Fmm &f, const Tree &t, typename C2T<T>::type *mp, typename C2T<T>::type *lc,
                     const typename C2T<T>::type *ops, int P, cudaStream_t s) {
    using C = typename C2T<T>::type;
    if constexpr (sizeof(T) == 8) {
        if (f.tc && P == f.P) {
            m2l_tc_pass(f, t, mp, lc, s);
            return;
        }
    }
    const size_t esz = (size_t)f.nd * P * sizeof(C);
    PHS_CUDA(cudaMemsetAsync(lc, 0, (size_t)t.nbox * esz, s));
    if (t.depth >= 2) {
        const int b0 = t.lvl_off[2], nb = t.nbox - b0;
        if (nb > 0)
            m2l_kernel<T><<<nb, FMM_T, 2 * esz, s>>>(tree_view(t), b0, t.v_off.get(), t.v_src.get(), t.v_cls.get(), f.nd,
                                                 P, f.power, ops, mix_buf<T>(f), mp, lc);
        PHS_LAUNCH_CHECK();
    }
}
template <typename T>
static void downward(Fmm &f, const Tree &t, typename C2T<T>::type *lc, const typename C2T<T>::type *ops, int P,
                     cudaStream_t s, bool ff = false) {
    using C = typename C2T<T>::type;
    const size_t esz = (size_t)f.nd * P * sizeof(C);
    if constexpr (sizeof(T) == 8) {
        set_pass_smem_limits();
        // parents of levels 2 .. depth-1 pass their local expansions to levels 3 .. depth
        for (int l = 2; l < t.depth; ++l) {
            const int b0 = t.lvl_off[l], nb = t.lvl_off[l + 1] - b0;
            if (nb > 0 && ff) l2l_ff_launch(f, t, b0, nb, lc, s);
            else if (nb > 0)
                l2l64_kernel<<<nb, shift_threads(f.nd, P), 8 * esz, s>>>(tree_view(t), b0, f.nd, P, f.shift_r.get() + (size_t)P * P,
                                                       f.shift_ph.get(), mix_buf<T>(f), lc);
            PHS_LAUNCH_CHECK();
        }
        return;
    }
    for (int l = 3; l <= t.depth; ++l) {
        const int b0 = t.lvl_off[l], nb = t.lvl_off[l + 1] - b0;
        if (nb > 0) l2l_kernel<T><<<nb, FMM_T, 2 * esz, s>>>(tree_view(t), b0, f.nd, P, ops, mix_buf<T>(f), lc);
        PHS_LAUNCH_CHECK();
    }
}

__global__ void d2f_kernel(const double2 *in, float2 *out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void f2d_kernel(const float2 *in, double2 *out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

// upward pass, M2L and downward pass (local expansions of every box) in one precision
template <typename T>
static void far_field(Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, cudaStream_t s,
                      Timers *tm, bool ff = false) {
    ensure_bufs<T>(f, t);
    const int P = P_of<T>(f);
    if (tm) tm->begin(s);
    upward<T>(f, t, ps, tv_sorted, mp_buf<T>(f), ops_buf<T>(f), P, s, ff);
    if (tm) tm->end(T_UP, s);
    if (tm) tm->begin(s);
    m2l_pass<T>(f, t, mp_buf<T>(f), lc_buf<T>(f), ops_buf<T>(f), P, s);
    if (tm) tm->end(T_M2L, s);
    if (tm) tm->begin(s);
    downward<T>(f, t, lc_buf<T>(f), ops_buf<T>(f), P, s, ff);
    if (tm) tm->end(T_DOWN, s);
}

// FP64 upward/downward passes around an FP32 M2L of the same order
static void far_field_m2l32(Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, cudaStream_t s,
                            Timers *tm) {
    ensure_bufs<double>(f, t);
    const size_t sz = (size_t)t.nbox * f.nd * f.P;
    if (f.mpx32.n != sz) { f.mpx32.alloc(sz); f.lcx32.alloc(sz); }
    if (tm) tm->begin(s);
    upward<double>(f, t, ps, tv_sorted, f.mp64.get(), f.ops64.get(), f.P, s);
    d2f_kernel<<<blocks_for((int64_t)sz, 256), 256, 0, s>>>(f.mp64.get(), f.mpx32.get(), sz);
    PHS_LAUNCH_CHECK();
    if (tm) tm->end(T_UP, s);
    if (tm) tm->begin(s);
    m2l_pass<float>(f, t, f.mpx32.get(), f.lcx32.get(), f.ops32p.get(), f.P, s);
    if (tm) tm->end(T_M2L, s);
    if (tm) tm->begin(s);
    f2d_kernel<<<blocks_for((int64_t)sz, 256), 256, 0, s>>>(f.lcx32.get(), f.lc64.get(), sz);
    PHS_LAUNCH_CHECK();
    downward<double>(f, t, f.lc64.get(), f.ops64.get(), f.P, s);
    if (tm) tm->end(T_DOWN, s);
}

template <typename T, int K>
static void p2p_launch(const Tree &t, const PointSet &ps, const double *tv_sorted, double *y, cudaStream_t s) {
    const size_t smem = UsesLogTab<T, K>::value ? kLogTab * sizeof(double2) + kExpTab * sizeof(double) : 0;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        int dev = 0, nsm = 0, per = 0;
        PHS_CUDA(cudaGetDevice(&dev));
        PHS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        PHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, p2p_kernel<T, K>, P2P_T, smem));
        grid_cap = std::max(1, nsm * std::max(per, 1));
    }
    const int grid = std::min(t.nleaf, grid_cap);
    p2p_kernel<T, K><<<grid, P2P_T, smem, s>>>(tree_view(t), t.nleaf, t.leaf_box.get(), t.near_off.get(),
                                               t.near_rng.get(), ps.xs.get(), tv_sorted, y);
    PHS_LAUNCH_CHECK();
}

// (log F_j, 1/F_j), F_j = 1 + j/2048, and e log 2 for the table-driven logarithm
static void upload_log_tables() {
    std::vector<double2> tab(kLogTab);
    for (int j = 0; j < kLogTab; ++j) {
        const long double F = 1.0L + (long double)j / 2048.0L;
        tab[j] = make_double2((double)std::log(F), (double)(1.0L / F));
    }
    std::vector<double> el(kExpTab);
    for (int i = 0; i < kExpTab; ++i) el[i] = (double)((long double)(kExpLo + i - 1023) * std::log(2.0L));
    PHS_CUDA(cudaMemcpyToSymbol(g_logtab, tab.data(), kLogTab * sizeof(double2)));
    PHS_CUDA(cudaMemcpyToSymbol(g_eln2, el.data(), kExpTab * sizeof(double)));
    std::vector<double> ik(kMaxP, 0.0);
    for (int k = 1; k < (int)ik.size(); ++k) ik[k] = -1.0 / k;
    PHS_CUDA(cudaMemcpyToSymbol(g_neg_inv_k, ik.data(), ik.size() * sizeof(double)));
}
template <int K>
static void p2p_sym_launch(Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, double *y,
                           cudaStream_t s) {
    const size_t smem = (K % 2 == 0) ? kLogTab * sizeof(double2) + kExpTab * sizeof(double) : 0;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        int dev = 0, nsm = 0, per = 0;
        PHS_CUDA(cudaGetDevice(&dev));
        PHS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        PHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, p2p_sym_kernel<K>, P2P_T, smem));
        grid_cap = std::max(1, nsm * std::max(per, 1));
    }
    if (f.sym_scratch.n < (size_t)std::max<int64_t>(t.sym_total, 1)) f.sym_scratch.alloc(std::max<int64_t>(t.sym_total, 1));
    if (!f.p2p_ticket.get()) f.p2p_ticket.alloc(1);
    PHS_CUDA(cudaMemsetAsync(f.p2p_ticket.get(), 0, sizeof(int), s));
    p2p_sym_kernel<K><<<std::min(t.nleaf, grid_cap), P2P_T, smem, s>>>(
        tree_view(t), t.nleaf, t.leaf_box.get(), t.p2p_order.get(), f.p2p_ticket.get(), t.near_off.get(),
        t.near_rng.get(), t.sym_slot.get(), ps.xs.get(), tv_sorted, y, f.sym_scratch.get());
    PHS_LAUNCH_CHECK();
    p2p_gather<<<blocks_for(ps.n, 256), 256, 0, s>>>(tree_view(t), t.leaf_box.get(), t.point_leaf.get(),
                                                     t.sym_goff.get(), t.sym_gbase.get(), ps.n, f.sym_scratch.get(), y);
    PHS_LAUNCH_CHECK();
}

template <typename T>
static void p2p_dispatch(Fmm &f, int k, const Tree &t, const PointSet &ps, const double *tv_sorted, double *y,
                         cudaStream_t s) {
    if (sizeof(T) == 8 && t.sym_ok) {
        switch (k) {
            case 1: p2p_sym_launch<1>(f, t, ps, tv_sorted, y, s); return;
            case 2: p2p_sym_launch<2>(f, t, ps, tv_sorted, y, s); return;
            case 3: p2p_sym_launch<3>(f, t, ps, tv_sorted, y, s); return;
            case 4: p2p_sym_launch<4>(f, t, ps, tv_sorted, y, s); return;
            default: p2p_sym_launch<5>(f, t, ps, tv_sorted, y, s); return;
        }
    }
    switch (k) {
        case 1: p2p_launch<T, 1>(t, ps, tv_sorted, y, s); break;
        case 2: p2p_launch<T, 2>(t, ps, tv_sorted, y, s); break;
        case 3: p2p_launch<T, 3>(t, ps, tv_sorted, y, s); break;
        case 4: p2p_launch<T, 4>(t, ps, tv_sorted, y, s); break;
        default: p2p_launch<T, 5>(t, ps, tv_sorted, y, s); break;
    }
}

// mode 4: the near field in float-float on the FP32 pipe (nearfield_ff.cu) with the
// symmetric schedule; trees with a leaf of more than 128 points keep the FP64 kernel
static void p2p_ff_dispatch(Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, double *y,
                            cudaStream_t s) {
    if (!t.sym_ok) {
        p2p_dispatch<double>(f, f.k, t, ps, tv_sorted, y, s);
        return;
    }
    if (f.sym_scratch.n < (size_t)std::max<int64_t>(t.sym_total, 1)) f.sym_scratch.alloc(std::max<int64_t>(t.sym_total, 1));
    if (!f.p2p_ticket.get()) f.p2p_ticket.alloc(1);
    p2p_sym_ff(t, ps, f.k, tv_sorted, y, f.sym_scratch.get(), f.p2p_ticket.get(), s);
    p2p_gather<<<blocks_for(ps.n, 256), 256, 0, s>>>(tree_view(t), t.leaf_box.get(), t.point_leaf.get(),
                                                     t.sym_goff.get(), t.sym_gbase.get(), ps.n, f.sym_scratch.get(), y);
    PHS_LAUNCH_CHECK();
}

template <typename T>
static void l2p_pass(Fmm &f, const Tree &t, const PointSet &ps, double *y, cudaStream_t s, bool ff = false) {
    using C = typename C2T<T>::type;
    if constexpr (sizeof(T) == 8) {
        if (ff) {
            l2p_ff_launch(f, t, ps, f.lc64.get(), y, s);
            return;
        }
        const size_t sm = (size_t)f.nd * f.P * sizeof(double2);  // at most 9 x 61 x 16 B
        const TreeView tv = tree_view(t);
        if (f.nd == 4) l2p64_kernel<4><<<t.nleaf, L2P_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), f.power, f.P, f.lc64.get(), y);
        else if (f.nd == 9) l2p64_kernel<9><<<t.nleaf, L2P_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), f.power, f.P, f.lc64.get(), y);
        else l2p64_kernel<1><<<t.nleaf, L2P_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), f.power, f.P, f.lc64.get(), y);
        PHS_LAUNCH_CHECK();
        return;
    }
    l2p_kernel<T><<<t.nleaf, 128, (size_t)f.nd * P_of<T>(f) * sizeof(C), s>>>(
        tree_view(t), t.leaf_box.get(), ps.xs.get(), f.power, f.nd, P_of<T>(f), lc_buf<T>(f), y);
    PHS_LAUNCH_CHECK();
}

Fmm::~Fmm() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
}

// buffers of the near field, allocated on s before the near field forks onto the side
// stream (so the stream-ordered allocation precedes every use)
static void p2p_prepare(Fmm &f, const Tree &t) {
    if (!t.sym_ok) return;
    if (f.sym_scratch.n < (size_t)std::max<int64_t>(t.sym_total, 1)) f.sym_scratch.alloc(std::max<int64_t>(t.sym_total, 1));
    if (!f.p2p_ticket.get()) f.p2p_ticket.alloc(1);
    if (!f.side) {
        PHS_CUDA(cudaStreamCreateWithFlags(&f.side, cudaStreamNonBlocking));
        PHS_CUDA(cudaEventCreateWithFlags(&f.ev_fork, cudaEventDisableTiming));
        PHS_CUDA(cudaEventCreateWithFlags(&f.ev_join, cudaEventDisableTiming));
    }
}

void fmm_apply(Fmm &f, const Tree &t, const PointSet &ps, const double *t_sorted, double *y, int mode, cudaStream_t s,
               Timers *tm) {
    PHS_REQUIRE(mode >= 0 && mode <= 4, PHS_ERR_INVALID_ARG, "precision mode must be 0..4");
    f.far_valid = false;  // the expansion buffers are about to hold this apply's far field
    PHS_REQUIRE(f.log_core || mode == 0 || mode == 4, PHS_ERR_INVALID_ARG, "odd spline orders run in precision 0 or 4");
    // near field on the side stream (it writes y; the far field's L2P adds to y after the
    // join).  With phase timing on it stays on s, so each phase's events time that phase
    // alone; the arithmetic and its order are the same either way.
    p2p_prepare(f, t);
    const bool fork = f.side && !(tm && tm->enabled);
    cudaStream_t ns = fork ? f.side : s;
    if (fork) {
        PHS_CUDA(cudaEventRecord(f.ev_fork, s));
        PHS_CUDA(cudaStreamWaitEvent(f.side, f.ev_fork, 0));
    }
    if (tm) tm->begin(ns);
    if (mode == 0) p2p_dispatch<double>(f, f.k, t, ps, t_sorted, y, ns);
    else if (mode == 4) p2p_ff_dispatch(f, t, ps, t_sorted, y, ns);
    else p2p_dispatch<float>(f, f.k, t, ps, t_sorted, y, ns);
    if (tm) tm->end(T_P2P, ns);
    if (fork) PHS_CUDA(cudaEventRecord(f.ev_join, f.side));
    if (!f.log_core) {
        // odd k: distance-kernel far field by Chebyshev interpolation in FP64
        cheb_far_field(f, t, ps, t_sorted, s, tm);
        if (fork) PHS_CUDA(cudaStreamWaitEvent(s, f.ev_join, 0));
        if (tm) tm->begin(s);
        cheb_l2p_apply(f, t, ps, y, s);
        if (tm) tm->end(T_DOWN, s);
        return;
    }
    if (mode <= 1 || mode == 4) far_field<double>(f, t, ps, t_sorted, s, tm, mode == 4 && f.ff_passes);
    else if (mode == 2) far_field_m2l32(f, t, ps, t_sorted, s, tm);
    else far_field<float>(f, t, ps, t_sorted, s, tm);
    if (fork) PHS_CUDA(cudaStreamWaitEvent(s, f.ev_join, 0));
    if (tm) tm->begin(s);
    if (mode == 3) l2p_pass<float>(f, t, ps, y, s);
    else l2p_pass<double>(f, t, ps, y, s, mode == 4 && f.ff_passes);
    if (tm) tm->end(T_DOWN, s);
}

// The level-invariant operator tables depend only on the order and the Hadamard power:
// built once per process in long double and reused by every plan.
static std::mutex g_table_mu;
static const std::vector<std::complex<long double>> &ops_cached(int P) {
    static std::map<int, std::vector<std::complex<long double>>> cache;
    std::lock_guard<std::mutex> g(g_table_mu);
    auto it = cache.find(P);
    if (it == cache.end()) it = cache.emplace(P, build_ops(P)).first;
    return it->second;
}
static const std::vector<long double> &mix_cached(int power, int nd) {
    static std::map<int, std::vector<long double>> cache;
    std::lock_guard<std::mutex> g(g_table_mu);
    auto it = cache.find(power);
    if (it == cache.end()) it = cache.emplace(power, build_mix(power, nd)).first;
    return it->second;
}

// The device forms of the level-invariant tables, also per order and per process: the
// operators in FP64 and FP32, and the real shift cores of M2M/L2L with their phases
// (R[l][k] = A_0[l][k] e^{-i th_0 (l - k)} for quadrant 0, checked real and equal for the
// other quadrants; th_q the quadrant's angle).
struct DevTables {
    std::vector<double2> o64;
    std::vector<float2> o32;
    std::vector<double> R;    // [2][P][P]: M2M, L2L
    std::vector<float2> Rff;  // the same split into hi + lo floats (float-float passes)
    std::vector<float4> phff; // ph split into hi + lo floats
    std::vector<double2> ph;  // [4][P]: e^{i th_q k}
    std::vector<long double> re, im;  // the operators split for the tensor-core setup
};
static std::mutex g_dev_tables_mu;
static const DevTables &dev_tables_cached(int P) {
    const auto &ops = ops_cached(P);
    static std::map<int, DevTables> cache;
    std::lock_guard<std::mutex> g(g_dev_tables_mu);
    auto it = cache.find(P);
    if (it != cache.end()) return it->second;
    DevTables d;
    d.o64.resize(ops.size());
    d.o32.resize(ops.size());
    d.re.resize(ops.size());
    d.im.resize(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        d.o64[i] = make_double2((double)ops[i].real(), (double)ops[i].imag());
        d.o32[i] = make_float2((float)ops[i].real(), (float)ops[i].imag());
        d.re[i] = ops[i].real();
        d.im[i] = ops[i].imag();
    }
    d.R.assign((size_t)2 * P * P, 0.0);
    d.Rff.assign((size_t)2 * P * P, make_float2(0.f, 0.f));
    d.ph.resize((size_t)4 * P);
    d.phff.resize((size_t)4 * P);
    for (int q = 0; q < 4; ++q) {
        const long double th = std::atan2((long double)((q & 2) ? 0.25L : -0.25L), (long double)((q & 1) ? 0.25L : -0.25L));
        for (int k = 0; k < P; ++k) {
            const long double a = th * k;
            d.ph[(size_t)q * P + k] = make_double2((double)std::cos(a), (double)std::sin(a));
            const long double c = std::cos(a), sn = std::sin(a);
            const float ch = (float)c, sh = (float)sn;
            d.phff[(size_t)q * P + k] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(sn - (long double)sh));
        }
        for (int t2 = 0; t2 < 2; ++t2)
            for (int r = 0; r < P; ++r)
                for (int c2 = 0; c2 < P; ++c2) {
                    const std::complex<long double> A = ops[((size_t)(4 * t2 + q) * P + r) * P + c2];
                    // M2M: row l = r, col k = c2, phase e^{i th (l - k)}; L2L: row m = r, col l = c2,
                    // phase e^{i th (l - m)}
                    const long double ang = t2 == 0 ? th * (r - c2) : th * (c2 - r);
                    const std::complex<long double> v = A * std::polar(1.0L, -ang);
                    const long double mag = std::abs(A);
                    PHS_REQUIRE(std::fabs(v.imag()) <= 1e-12L * std::max(mag, 1e-300L) + 1e-300L, PHS_ERR_INVALID_ARG,
                                "shift operator does not factor through a real core");
                    double &dst = d.R[((size_t)t2 * P + r) * P + c2];
                    if (q == 0) {
                        dst = (double)v.real();
                        const float hi = (float)v.real();
                        d.Rff[((size_t)t2 * P + r) * P + c2] = make_float2(hi, (float)(v.real() - (long double)hi));
                    }
                    else
                        PHS_REQUIRE(std::fabs((long double)dst - v.real()) <= 1e-12L * std::max(mag, 1e-300L) + 1e-300L,
                                    PHS_ERR_INVALID_ARG, "shift cores differ between quadrants");
                }
    }
    return cache.emplace(P, std::move(d)).first->second;
}

void fmm_setup(Fmm &f, int k, int p, int p32, int cheb_q, int tensor_m2l, const Tree &t, cudaStream_t s) {
    PHS_REQUIRE(k >= 1 && k <= 5, PHS_ERR_INVALID_ARG, "k must be in 1..5");
    PHS_REQUIRE(p >= 2 && p + 1 <= kMaxP, PHS_ERR_INVALID_ARG, "fmm_order must be in 2..60");
    PHS_REQUIRE(p32 >= 2 && p32 + 1 <= kMaxP, PHS_ERR_INVALID_ARG, "FP32 fmm order must be in 2..60");
    f.k = k;
    f.p = p;
    f.P = p + 1;
    f.p32 = p32;
    f.P32 = p32 + 1;
    f.log_core = (k % 2 == 0);
    f.power = f.log_core ? k : k - 1;
    f.nd = f.power == 0 ? 1 : (f.power == 2 ? 4 : 9);
    PHS_REQUIRE(f.nd * f.P <= FMM_T * OUT_PER_T, PHS_ERR_INVALID_ARG, "fmm_order too large for this spline order");
    const DevTables &dt = dev_tables_cached(f.P);
    const DevTables &dtf = dev_tables_cached(f.P32);
    const std::vector<double2> &o64 = dt.o64;
    const std::vector<float2> &o32 = dtf.o32, &o32p = dt.o32;
    f.ops64.alloc(o64.size());
    f.ops32.alloc(o32.size());
    f.ops32p.alloc(o32p.size());
    PHS_CUDA(cudaMemcpyAsync(f.ops64.get(), o64.data(), o64.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.ops32.get(), o32.data(), o32.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.ops32p.get(), o32p.data(), o32p.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    f.shift_r.alloc(dt.R.size());
    f.shift_ph.alloc(dt.ph.size());
    f.shift_rff.alloc(dt.Rff.size());
    f.shift_phff.alloc(dt.phff.size());
    PHS_CUDA(cudaMemcpyAsync(f.shift_phff.get(), dt.phff.data(), dt.phff.size() * sizeof(float4),
                             cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.shift_r.get(), dt.R.data(), dt.R.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.shift_rff.get(), dt.Rff.data(), dt.Rff.size() * sizeof(float2), cudaMemcpyHostToDevice,
                             s));
    PHS_CUDA(cudaMemcpyAsync(f.shift_ph.get(), dt.ph.data(), dt.ph.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    {
        const auto &mx = mix_cached(f.power, f.nd);
        std::vector<double> m64(mx.size());
        std::vector<float> m32(mx.size());
        std::vector<float2> mff(mx.size());
        for (size_t i = 0; i < mx.size(); ++i) {
            m64[i] = (double)mx[i];
            m32[i] = (float)mx[i];
            mff[i] = make_float2(m32[i], (float)(mx[i] - (long double)m32[i]));
        }
        f.mixff.alloc(mff.size());
        PHS_CUDA(cudaMemcpyAsync(f.mixff.get(), mff.data(), mff.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
        f.mix64.alloc(m64.size());
        f.mix32.alloc(m32.size());
        PHS_CUDA(cudaMemcpyAsync(f.mix64.get(), m64.data(), m64.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(f.mix32.get(), m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        f.tc = false;
        if (tensor_m2l && f.log_core && m2l_tc_supported(f.nd, f.P)) m2l_tc_setup(f, dt.re, dt.im, mx, s);
    }
    PHS_CUDA(cudaStreamSynchronize(s));
    once_per_device(1, upload_log_tables);
    once_per_device(2, upload_ff_tables);
    // the compressed M2L truncates at a fifth of the accuracy the order was chosen for
    // (q = the smallest order with 5.83^-(q-1) <= eps), capped at rank 80: 80 of 256 at q = 16
    if (!f.log_core)
        cheb_setup(f, cheb_q, 0.2 * std::pow(5.83, -(double)(cheb_q - 1)), tensor_m2l == 2, mix_cached(f.power, f.nd),
                   s);
    m2l_tc_count(f, t, s);
}

// ---------------------------------------------------------------- evaluation at targets
// Per target: the deepest box containing it, the direct sum over that box's near set
// (the same construction as the leaf lists), and the far field from that box's local
// expansion (complex log expansion or Chebyshev interpolant).  Targets outside the
// root box are summed directly over all sources.
__global__ void eval_box_kernel(TreeView tv, const double2 *tgt, int64_t m, int *box_of) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double2 y = tgt[i];
    const double R = tv.R;
    if (!(y.x >= -R && y.x <= R && y.y >= -R && y.y <= R)) {
        box_of[i] = -1;
        return;
    }
    const int L = tv.depth;
    const double wl = box_width(R, L);
    long long ix = (long long)floor((y.x + R) / wl), iy = (long long)floor((y.y + R) / wl);
    const long long lim = (1ll << L) - 1;
    ix = ix < 0 ? 0 : (ix > lim ? lim : ix);
    iy = iy < 0 ? 0 : (iy > lim ? lim : iy);
    box_of[i] = find_deepest(tv, L, (int)ix, (int)iy);
}

// direct part from the precomputed near list of the target's box: a warp per target, the
// lanes striding over each range, one fixed-order shuffle reduction at the end.  A target
// between clusters lies in a coarse box whose near list holds a large share of all
// points, so the work per target varies by orders of magnitude; a thread per target left
// those sums on a few SMs' FP64 pipes.
constexpr int EVAL_T = 128;
template <int K>
__global__ void __launch_bounds__(EVAL_T) eval_near_kernel(const double2 *xs, const double *w, const double2 *tgt,
                                                           int64_t m, const int *box_of, const int *near_off,
                                                           const int2 *near_rng, double *out) {
    const int64_t i = (int64_t)blockIdx.x * (EVAL_T / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= m) return;  // whole warps leave together
    const int b = box_of[i];
    if (b < 0) {
        if (lane == 0) out[i] = 0.0;
        return;
    }
    const double2 y = tgt[i];
    double acc = 0.0;
    for (int r = near_off[b]; r < near_off[b + 1]; ++r) {
        const int2 rg = near_rng[r];
        for (int j = rg.x + lane; j < rg.y; j += 32) {
            const double dx = y.x - xs[j].x, dy = y.y - xs[j].y;
            const double r2 = dx * dx + dy * dy;
            if (r2 > 0) acc += phi_r2<double, K>(r2) * w[j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = acc;
}

__global__ void eval_far_log_kernel(TreeView tv, const double2 *tgt, int64_t m, const int *box_of, int power, int nd,
                                    int P, const double2 *lc, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int b = box_of[i];
    if (b < 0 || tv.level[b] < 2) return;
    const double2 y = tgt[i];
    double cx, cy, bw;
    box_geom(tv, b, cx, cy, bw);
    double2 v = make_double2((y.x - cx) / bw, (y.y - cy) / bw);
    double u[kMaxNd];
    had_u(power, v.x, v.y, u);  // factors local to the box
    const double2 *Lb = lc + (size_t)b * nd * P;
    double acc = 0.0;
    for (int d = 0; d < nd; ++d) {
        const double2 *Ld = Lb + d * P;
        double2 h = Ld[P - 1];
        for (int l = P - 2; l >= 0; --l) {
            double2 t2 = cmul(h, v);
            h.x = t2.x + Ld[l].x;
            h.y = t2.y + Ld[l].y;
        }
        acc += u[d] * h.x;
    }
    out[i] += acc;
}

// direct sum over all sources for targets outside the root box: blockIdx.y = target,
// blockIdx.x = a chunk of the sources, so one target spreads over many SMs; per-chunk
// partial sums are added in chunk order by eval_outside_sum (deterministic)
constexpr int kOutsideChunk = 4096;
template <int K>
__global__ void eval_outside_kernel(const double2 *xs, int64_t n, const double *w, const double2 *tgt,
                                    const int *out_idx, double *partial) {
    const int64_t i = out_idx[blockIdx.y];
    const double2 y = tgt[i];
    const int64_t j0 = (int64_t)blockIdx.x * kOutsideChunk, j1 = min(n, j0 + kOutsideChunk);
    double acc = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const double dx = y.x - xs[j].x, dy = y.y - xs[j].y;
        const double r2 = dx * dx + dy * dy;
        if (r2 > 0) acc += phi_r2<double, K>(r2) * w[j];
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}
__global__ void eval_outside_sum(const int *out_idx, int nout, int nchunk, const double *partial, double *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nout) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += partial[(size_t)q * nchunk + c];
    out[out_idx[q]] = acc;
}

template <int K>
static void eval_launch(Fmm &f, const Tree &t, const PointSet &ps, const double *w_sorted, const double2 *tgt, int64_t m,
                        double *out, cudaStream_t s) {
    SBuf<int> box_of(std::max<int64_t>(m, 1), s);
    TreeView tv = tree_view(t);
    eval_box_kernel<<<blocks_for(m, 128), 128, 0, s>>>(tv, tgt, m, box_of.get());
    PHS_LAUNCH_CHECK();
    eval_near_kernel<K><<<blocks_for(m, EVAL_T / 32), EVAL_T, 0, s>>>(ps.xs.get(), w_sorted, tgt, m, box_of.get(),
                                                                     t.near_off.get(), t.near_rng.get(), out);
    PHS_LAUNCH_CHECK();
    if (f.log_core) {
        eval_far_log_kernel<<<blocks_for(m, 128), 128, 0, s>>>(tv, tgt, m, box_of.get(), f.power, f.nd, f.P,
                                                               f.lc64.get(), out);
        PHS_LAUNCH_CHECK();
    } else {
        cheb_eval_far_launch(f, t, tgt, box_of.get(), m, out, s);
    }
    // targets outside the root box
    std::vector<int> hb(m);
    PHS_CUDA(cudaMemcpyAsync(hb.data(), box_of.get(), m * sizeof(int), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    std::vector<int> outside;
    for (int64_t i = 0; i < m; ++i)
        if (hb[i] < 0) outside.push_back((int)i);
    if (!outside.empty()) {
        SBuf<int> oi(outside.size(), s);
        PHS_CUDA(cudaMemcpyAsync(oi.get(), outside.data(), outside.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        const int nchunk = (int)((ps.n + kOutsideChunk - 1) / kOutsideChunk);
        const int nout = (int)outside.size(), batch = 65535;  // grid y limit
        SBuf<double> part((size_t)nchunk * std::min(nout, batch), s);
        for (int q0 = 0; q0 < nout; q0 += batch) {
            const int nq = std::min(batch, nout - q0);
            eval_outside_kernel<K><<<dim3((unsigned)nchunk, (unsigned)nq), 256, 0, s>>>(ps.xs.get(), ps.n, w_sorted,
                                                                                        tgt, oi.get() + q0, part.get());
            PHS_LAUNCH_CHECK();
            eval_outside_sum<<<blocks_for(nq, 128), 128, 0, s>>>(oi.get() + q0, nq, nchunk, part.get(), out);
            PHS_LAUNCH_CHECK();
        }
        PHS_CUDA(cudaStreamSynchronize(s));
    }
}

void fmm_eval64(Fmm &f, const Tree &t, const PointSet &ps, const double *w_sorted, const double2 *tgt, int64_t m,
                double *out, cudaStream_t s, Timers *tm, bool far_ready) {
    if (!far_ready) {
        if (f.log_core) far_field<double>(f, t, ps, w_sorted, s, nullptr);
        else cheb_far_field(f, t, ps, w_sorted, s, nullptr);
    }
    if (tm) tm->begin(s);
    switch (f.k) {
        case 1: eval_launch<1>(f, t, ps, w_sorted, tgt, m, out, s); break;
        case 2: eval_launch<2>(f, t, ps, w_sorted, tgt, m, out, s); break;
        case 3: eval_launch<3>(f, t, ps, w_sorted, tgt, m, out, s); break;
        case 4: eval_launch<4>(f, t, ps, w_sorted, tgt, m, out, s); break;
        default: eval_launch<5>(f, t, ps, w_sorted, tgt, m, out, s); break;
    }
    if (tm) tm->end(T_EVAL, s);
}

void dense_matvec64(const double2 *x, int64_t n, int k, const double *t, double *out, cudaStream_t s) {
    const unsigned nb = blocks_for(n, 256);
    switch (k) {
        case 1: dense_kernel<1><<<nb, 256, 0, s>>>(x, n, t, out); break;
        case 2: dense_kernel<2><<<nb, 256, 0, s>>>(x, n, t, out); break;
        case 3: dense_kernel<3><<<nb, 256, 0, s>>>(x, n, t, out); break;
        case 4: dense_kernel<4><<<nb, 256, 0, s>>>(x, n, t, out); break;
        default: dense_kernel<5><<<nb, 256, 0, s>>>(x, n, t, out); break;
    }
    PHS_LAUNCH_CHECK();
}

}  // namespace phs
