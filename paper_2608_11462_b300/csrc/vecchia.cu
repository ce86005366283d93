// vecchia.cu -- Vecchia sparse inverse-Cholesky preconditioner (Sec. 2.2, Eq. 2.19, Fig. 1):
// enumeration, previous-point neighbour search, per-point local Cholesky factors,
// the transposed factor and the apply z = U~ (U~' r).
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "geom.cuh"
#include "ff.cuh"
#include "phs_internal.cuh"

namespace phs {
namespace {

// SplitMix64 output i for a seed (Steele, Lea & Flood 2014)
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void rand_keys(int64_t n, uint64_t seed, uint64_t *keys, int *vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = splitmix64(seed, (uint64_t)i);
    vals[i] = (int)i;
}

// squared distance with two roundings per product and one for the sum (no FMA)
__device__ __forceinline__ double sqd(double2 a, double2 b) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__global__ void ranks_from_order(const int *order, int64_t n, int *rank) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) rank[order[r]] = (int)r;
}

__global__ void gather_xy(const double2 *x, const int *idx, int64_t n, double2 *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[idx[i]];
}

// ---------------------------------------------------------------- neighbour grid
// G x G cells of width cw over the bounding square at (x0, y0); points are sorted by
// (cell, rank), so a run of cells along a grid row is one contiguous range.
struct Grid {
    double x0, y0, cw, inv;
    int G;
};

__global__ void knn_bbox_partial(const double2 *x, int64_t n, Dbl4 *part) {
    __shared__ Dbl4 red[256];
    Dbl4 b = Dbl4{INFINITY, -INFINITY, INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        b.x = fmin(b.x, v.x);
        b.y = fmax(b.y, v.x);
        b.z = fmin(b.z, v.y);
        b.w = fmax(b.w, v.y);
    }
    red[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const Dbl4 c = red[threadIdx.x + o];
            Dbl4 &d = red[threadIdx.x];
            d.x = fmin(d.x, c.x);
            d.y = fmax(d.y, c.y);
            d.z = fmin(d.z, c.z);
            d.w = fmax(d.w, c.w);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void knn_grid_final(const Dbl4 *part, int np, int G, Grid *g) {
    Dbl4 b = part[0];
    for (int i = 1; i < np; ++i) {
        b.x = fmin(b.x, part[i].x);
        b.y = fmax(b.y, part[i].y);
        b.z = fmin(b.z, part[i].z);
        b.w = fmax(b.w, part[i].w);
    }
    const double ext = fmax(b.y - b.x, b.w - b.z);
    Grid h;
    h.G = G;
    h.cw = ext > 0 ? ext / G * (1.0 + 1e-12) : 1.0;
    h.inv = 1.0 / h.cw;
    h.x0 = b.x;
    h.y0 = b.z;
    *g = h;
}
__device__ __forceinline__ int grid_coord(double v, double v0, const Grid &g) {
    return min(max((int)floor((v - v0) * g.inv), 0), g.G - 1);
}

__global__ void grid_keys(const double2 *x, const int *rank, int64_t n, const Grid *gp, uint64_t *keys, int *vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Grid g = *gp;
    const int cx = grid_coord(x[i].x, g.x0, g), cy = grid_coord(x[i].y, g.y0, g);
    keys[i] = ((uint64_t)(cy * g.G + cx) << 32) | (uint64_t)(uint32_t)rank[i];
    vals[i] = (int)i;
}

__global__ void cell_starts(const uint64_t *keys, int64_t n, int ncell, int *start) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    const uint64_t v = (uint64_t)c << 32;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    start[c] = (int)lo;
}

__global__ void cell_payload(const uint64_t *keys, const int *vals, const double2 *x, int64_t n, double2 *xc, int *rc) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    xc[s] = x[vals[s]];
    rc[s] = (int)(keys[s] & 0xffffffffu);
}

constexpr int KNN_MAXM = 64;

__device__ __forceinline__ bool key_less(unsigned long long ad, int aq, unsigned long long bd, int bq) {
    return ad < bd || (ad == bd && aq < bq);
}

// The m smallest (d2, rank) keys seen so far, sorted, spread over the warp: entry k in
// lane k (e0) and, for m > 32, entry 32 + k in lane k (e1).  Squared distances are
// non-negative, so their bit patterns order as unsigned integers and no comparison
// runs on the FP64 pipe.
struct WarpTopM {
    unsigned long long d0 = ~0ull, d1 = ~0ull;
    int q0 = INT_MAX, q1 = INT_MAX;
    unsigned long long td = ~0ull;  // entry m - 1 once m entries are held, else "infinity"
    int tq = INT_MAX;
    int cnt = 0;                    // entries held (at most m), warp-uniform

    // one candidate per lane (valid lanes only); inserts those below the threshold
    __device__ __forceinline__ void offer(bool valid, unsigned long long cd, int cq, int m, int lane) {
        const unsigned full = 0xffffffffu;
        unsigned mask = __ballot_sync(full, valid && key_less(cd, cq, td, tq));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const unsigned long long vd = __shfl_sync(full, cd, src);
            const int vq = __shfl_sync(full, cq, src);
            if (!key_less(vd, vq, td, tq)) continue;
            // entry k becomes entry k - 1 if the candidate precedes that, else the candidate
            // if it precedes entry k, else stays
            const unsigned long long pd = __shfl_up_sync(full, d0, 1);
            const int pq = __shfl_up_sync(full, q0, 1);
            if (m > 32) {
                unsigned long long pd1 = __shfl_up_sync(full, d1, 1);
                int pq1 = __shfl_up_sync(full, q1, 1);
                const unsigned long long ld = __shfl_sync(full, d0, 31);
                const int lq = __shfl_sync(full, q0, 31);
                if (lane == 0) {
                    pd1 = ld;
                    pq1 = lq;
                }
                if (key_less(vd, vq, pd1, pq1)) {
                    d1 = pd1;
                    q1 = pq1;
                } else if (key_less(vd, vq, d1, q1)) {
                    d1 = vd;
                    q1 = vq;
                }
            }
            if (lane > 0 && key_less(vd, vq, pd, pq)) {
                d0 = pd;
                q0 = pq;
            } else if (key_less(vd, vq, d0, q0)) {
                d0 = vd;
                q0 = vq;
            }
            cnt = min(cnt + 1, m);
            if (cnt == m) {
                td = __shfl_sync(full, m > 32 ? d1 : d0, (m - 1) & 31);
                tq = __shfl_sync(full, m > 32 ? q1 : q0, (m - 1) & 31);
            }
        }
    }
    __device__ __forceinline__ unsigned long long entry_d(int k) const {
        return __shfl_sync(0xffffffffu, k >= 32 ? d1 : d0, k & 31);
    }
};

// Warp per rank r: the min(m, r) nearest points of smaller rank, by (d2, rank).  Small
// ranks scan all previous points; the others walk square rings of grid cells around
// the query until the held need-th distance is below the distance to the ring's outside.
// Points sit in cells sorted by rank, so each of a ring's cells contributes the prefix of
// its range below r (a binary search); 32 such ranges at a time are concatenated by a
// warp scan of their lengths so that every distance batch is full of admissible points.
__global__ void knn_kernel(const double2 *x_by_rank, int64_t n, int m, int brute, const Grid *gp, const int *cstart,
                           const double2 *xc, const int *rc, const int *order, int *nbr_ell) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t r64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r64 >= n) return;
    const int r = (int)r64;
    const double2 p = x_by_rank[r];
    const int need = min(m, r);
    WarpTopM top;
    if (need > 0 && r <= brute) {
        for (int base = 0; base < r; base += 32) {
            const int q = base + lane;
            const bool valid = q < r;
            const unsigned long long cd = valid ? (unsigned long long)__double_as_longlong(sqd(p, x_by_rank[q])) : ~0ull;
            top.offer(valid, cd, q, m, lane);
        }
    } else if (need > 0) {
        const Grid g = *gp;
        const int cx0 = grid_coord(p.x, g.x0, g), cy0 = grid_coord(p.y, g.y0, g);
        for (int k = 0;; ++k) {
            const int xa = cx0 - k, xb = cx0 + k, ya = cy0 - k, yb = cy0 + k;
            // cell j of ring k (8k cells; 1 for k = 0): the top row, the bottom row, then
            // the two ends of each row between.  A cell's points are sorted by rank, so
            // those before r (the only admissible ones) are a prefix of its range.
            const int nr = k == 0 ? 1 : 8 * k;
            for (int g0 = 0; g0 < nr; g0 += 32) {
                int st = 0, len = 0;
                const int j = g0 + lane;
                if (j < nr) {
                    int dx = 0, dy = 0;
                    if (k > 0) {
                        if (j < 2 * k + 1) {
                            dy = -k;
                            dx = j - k;
                        } else if (j < 4 * k + 2) {
                            dy = k;
                            dx = j - (3 * k + 1);
                        } else {
                            const int t2 = j - (4 * k + 2);
                            dy = 1 - k + (t2 >> 1);
                            dx = (t2 & 1) ? k : -k;
                        }
                    }
                    const int cx = cx0 + dx, cy = cy0 + dy;
                    if (cx >= 0 && cx < g.G && cy >= 0 && cy < g.G) {
                        const int c = cy * g.G + cx;
                        const int a0 = cstart[c];
                        int lo = a0, hi = cstart[c + 1];
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (rc[mid] < r) lo = mid + 1;
                            else hi = mid;
                        }
                        st = a0;
                        len = lo - a0;
                    }
                }
                int off = len;  // inclusive scan of the range lengths
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(full, off, o);
                    if (lane >= o) off += v;
                }
                const int total = __shfl_sync(full, off, 31);
                off -= len;  // exclusive
                for (int t = 0; t < total; t += 32) {
                    const int e = t + lane;
                    int lo = 0;  // last range with off <= e
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int c = lo + step;
                        const int oc = __shfl_sync(full, off, c & 31);
                        if (c < 32 && oc <= e) lo = c;
                    }
                    const int pos = __shfl_sync(full, st, lo) + (e - __shfl_sync(full, off, lo));
                    bool valid = e < total;
                    int q = INT_MAX;
                    double2 c = p;
                    if (valid) {
                        q = rc[pos];
                        valid = q < r;
                        c = xc[pos];
                    }
                    const unsigned long long cd = valid ? (unsigned long long)__double_as_longlong(sqd(p, c)) : ~0ull;
                    top.offer(valid, cd, q, m, lane);
                }
            }
            if (xa <= 0 && ya <= 0 && xb >= g.G - 1 && yb >= g.G - 1) break;
            if (top.cnt >= need) {
                double dm = INFINITY;
                if (xa > 0) dm = fmin(dm, p.x - (g.x0 + xa * g.cw));
                if (xb < g.G - 1) dm = fmin(dm, (g.x0 + (xb + 1) * g.cw) - p.x);
                if (ya > 0) dm = fmin(dm, p.y - (g.y0 + ya * g.cw));
                if (yb < g.G - 1) dm = fmin(dm, (g.y0 + (yb + 1) * g.cw) - p.y);
                if (dm > 0 && dm * dm * (1.0 - 1e-12) > __longlong_as_double((long long)top.entry_d(need - 1))) break;
            }
        }
    }
    const int i = order[r];
    if (lane < m) nbr_ell[(int64_t)lane * n + i] = lane < top.cnt ? order[top.q0] : -1;
    if (lane + 32 < m) nbr_ell[(int64_t)(lane + 32) * n + i] = lane + 32 < top.cnt ? order[top.q1] : -1;
}

// ---------------------------------------------------------------- Matern covariance, K(0) = 1
// In terms of q = (alpha r)^2 / 4 the ascending series of K_0 and K_1 (DLMF 10.31.1-2)
// need neither a square root nor a division:
//   a K_1(a) = 1 + q (log(q) S_1(q) - P_1(q)),   K_0(a) = -(log(q)/2 + gamma) S_0(q) + H_0(q),
//   S_1 = sum q^k / (k!(k+1)!),  P_1 = sum (psi(k+1) + psi(k+2)) q^k / (k!(k+1)!),
//   S_0 = sum q^k / (k!)^2,      H_0 = sum H_k q^k / (k!)^2.
// The coefficients are tabulated (host, long double) and the sums run in Horner form
// with as many terms as q needs (relative truncation below 1e-16 for q <= 1, a <= 2).
// For a > 2 the trapezoidal rule with step 1/4 on K_nu(a) = int_0^inf exp(-a cosh t)
// cosh(nu t) dt (DLMF 10.32.9) uses tabulated cosh(j/4).
constexpr int kSerTerms = 14;
constexpr int kCoshTab = 64;
__constant__ double c_s1[kSerTerms], c_p1[kSerTerms], c_s0[kSerTerms], c_h0[kSerTerms], c_cosh[kCoshTab];

// terms for a truncation below 1e-16 relative: q^n / (n!)^2 at the bound of each class.
// The class bounds are powers of two, so q < 2^k is a compare of the high words (q > 0),
// which keeps these decisions off the FP64 pipe.
__device__ __forceinline__ int ser_terms(double q) {
    const int hi = __double2hiint(q);
    return hi < 0x3ED00000 ? 3 : (hi < 0x3F100000 ? 4 : (hi < 0x3F900000 ? 6 : (hi < 0x3FC00000 ? 9 : kSerTerms)));
}
// Table-driven FP64 logarithm for the series (P. T. P. Tang, ACM TOMS 16(4), 1990):
// x = 2^e m, F_j = 1 + j/2048 nearest m, log x = e log 2 + log F_j + log(1 + r) with
// r = m/F_j - 1 (|r| < 2^-12) and a three-term log(1 + r); exponents below 2^-255 clamp
// (there q log q vanishes).  Tables in global memory, read through the read-only cache.
constexpr int kVLogTab = 2049, kVExpLo = 768, kVExpTab = 259;
__device__ double2 g_vlogtab[kVLogTab];  // (log F_j, 1/F_j)
__device__ double g_veln2[kVExpTab];     // (e - 1023) log 2 for biased e = kVExpLo + i

__device__ __forceinline__ double vtab_log(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int j = (((hi >> 8) & 0xfff) + 1) >> 1;
    const int ei = min(max((hi >> 20) - kVExpLo, 0), kVExpTab - 1);
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
    const double2 fj = __ldg(&g_vlogtab[j]);
    const double r = fma(m, fj.y, -1.0);
    double c = fma(r, 0.33333333333333333, -0.5);
    c = fma(c, r, 1.0);
    return fma(c, r, fj.x + __ldg(&g_veln2[ei]));
}

// float-float forms for the precision-4 factor (factor_kernel_ff): the same series with
// the coefficients split into hi + lo floats and the logarithm of ff.cuh (ff_log)
__constant__ float2 c_s1f[kSerTerms], c_p1f[kSerTerms], c_s0f[kSerTerms], c_h0f[kSerTerms];
__device__ float g_vf_rcp[256];
__device__ float2 g_vf_tlog[256], g_vf_eln2[256];

__device__ __forceinline__ ffa::F2 horner_ff(const float2 *c, int nt, ffa::F2 q) {
    ffa::F2 v{c[nt - 1].x, c[nt - 1].y};
    for (int k = nt - 2; k >= 0; --k) v = ffa::ff_add(ffa::ff_mul(v, q), ffa::F2{c[k].x, c[k].y});
    return v;
}

__device__ __forceinline__ double horner(const double *c, int nt, double q) {
    double v = c[nt - 1];
    for (int k = nt - 2; k >= 0; --k) v = fma(v, q, c[k]);
    return v;
}

// (K_0(a), a K_1(a)) by quadrature for a > 2
__device__ __forceinline__ void bessel_quad(double a, double &k0, double &ak1) {
    double s0 = 0.5 * exp(-a), s1 = s0;
    for (int j = 1; j < kCoshTab; ++j) {
        const double ch = c_cosh[j];
        const double e = exp(-a * ch);
        s0 += e;
        s1 += e * ch;
        if (e * ch < 1e-19 * s0) break;
    }
    k0 = 0.25 * s0;
    ak1 = a * 0.25 * s1;
}

// Matern with K(0) = 1 as a function of q = (alpha r)^2 / 4 (q > 0); NUC selects
// nu = 0.5, 1, 1.5, 2, 2.5 at compile time
template <int NUC>
__device__ __forceinline__ double matern_q(double q) {
    if (NUC == 0 || NUC == 2 || NUC == 4) {
        const double a = 2.0 * sqrt(q), e = exp(-a);
        if (NUC == 0) return e;
        if (NUC == 2) return (1.0 + a) * e;
        return (1.0 + a + a * a / 3.0) * e;
    }
    double k0, ak1;
    if (__double2hiint(q) < 0x3FF00000) {  // q < 1
        const int nt = ser_terms(q);
        const double lq = vtab_log(q);
        ak1 = fma(q, fma(lq, horner(c_s1, nt, q), -horner(c_p1, nt, q)), 1.0);
        if (NUC == 1) return ak1;
        k0 = fma(-(0.5 * lq + 0.57721566490153286061), horner(c_s0, nt, q), horner(c_h0, nt, q));
    } else {
        bessel_quad(2.0 * sqrt(q), k0, ak1);
        if (NUC == 1) return ak1;
    }
    return 2.0 * q * k0 + ak1;  // nu = 2: a^2 K_2(a) / 2 = a^2 K_0(a) / 2 + a K_1(a)
}

static void upload_bessel_tables() {
    long double s1[kSerTerms], p1[kSerTerms], s0[kSerTerms], h0[kSerTerms];
    const long double eg = 0.57721566490153286060651209008240243L;
    long double fk = 1, fk1 = 1, H = 0;  // k!, (k+1)!, H_k
    for (int k = 0; k < kSerTerms; ++k) {
        if (k > 0) {
            fk *= k;
            H += 1.0L / k;
        }
        fk1 = fk * (k + 1);
        s1[k] = 1.0L / (fk * fk1);
        p1[k] = (-2 * eg + 2 * H + 1.0L / (k + 1)) * s1[k];
        s0[k] = 1.0L / (fk * fk);
        h0[k] = H * s0[k];
    }
    double d[4][kSerTerms], ch[kCoshTab];
    for (int k = 0; k < kSerTerms; ++k) {
        d[0][k] = (double)s1[k];
        d[1][k] = (double)p1[k];
        d[2][k] = (double)s0[k];
        d[3][k] = (double)h0[k];
    }
    for (int j = 0; j < kCoshTab; ++j) ch[j] = (double)std::cosh(0.25L * j);
    std::vector<double2> lt(kVLogTab);
    for (int j = 0; j < kVLogTab; ++j) {
        const long double F = 1.0L + (long double)j / 2048.0L;
        lt[j] = make_double2((double)std::log(F), (double)(1.0L / F));
    }
    std::vector<double> el(kVExpTab);
    for (int i = 0; i < kVExpTab; ++i) el[i] = (double)((long double)(kVExpLo + i - 1023) * std::log(2.0L));
    PHS_CUDA(cudaMemcpyToSymbol(g_vlogtab, lt.data(), kVLogTab * sizeof(double2)));
    PHS_CUDA(cudaMemcpyToSymbol(g_veln2, el.data(), kVExpTab * sizeof(double)));
    PHS_CUDA(cudaMemcpyToSymbol(c_s1, d[0], sizeof(d[0])));
    PHS_CUDA(cudaMemcpyToSymbol(c_p1, d[1], sizeof(d[1])));
    PHS_CUDA(cudaMemcpyToSymbol(c_s0, d[2], sizeof(d[2])));
    PHS_CUDA(cudaMemcpyToSymbol(c_h0, d[3], sizeof(d[3])));
    PHS_CUDA(cudaMemcpyToSymbol(c_cosh, ch, sizeof(ch)));
    float2 f[4][kSerTerms];
    for (int k = 0; k < kSerTerms; ++k) {
        const long double src[4] = {s1[k], p1[k], s0[k], h0[k]};
        for (int t = 0; t < 4; ++t) {
            const float h = (float)src[t];
            f[t][k] = make_float2(h, (float)(src[t] - (long double)h));
        }
    }
    PHS_CUDA(cudaMemcpyToSymbol(c_s1f, f[0], sizeof(f[0])));
    PHS_CUDA(cudaMemcpyToSymbol(c_p1f, f[1], sizeof(f[1])));
    PHS_CUDA(cudaMemcpyToSymbol(c_s0f, f[2], sizeof(f[2])));
    PHS_CUDA(cudaMemcpyToSymbol(c_h0f, f[3], sizeof(f[3])));
    std::vector<float> frc;
    std::vector<float2> ftl, fel;
    ffa::ff_log_tables(frc, ftl, fel);
    PHS_CUDA(cudaMemcpyToSymbol(g_vf_rcp, frc.data(), 256 * sizeof(float)));
    PHS_CUDA(cudaMemcpyToSymbol(g_vf_tlog, ftl.data(), 256 * sizeof(float2)));
    PHS_CUDA(cudaMemcpyToSymbol(g_vf_eln2, fel.data(), 256 * sizeof(float2)));
}

// The Matern entry in float-float from the float-float scaled squared distance q: the
// series of nu = 1 and nu = 2 (the thin-plate and k = 4 preconditioners) for q < 1, the
// FP64 form otherwise (the other smoothness values and q >= 1), then split.
template <int NUC>
__device__ __forceinline__ ffa::F2 matern_ff(ffa::F2 q) {
    using ffa::F2;
    if constexpr (NUC == 1 || NUC == 3) {
        if (q.h < 1.0f && q.h > 1e-30f) {
            const float qh = q.h;
            const int nt = qh < 0x1p-18f ? 3 : (qh < 0x1p-14f ? 4 : (qh < 0x1p-6f ? 6 : (qh < 0x1p-3f ? 9 : kSerTerms)));
            const F2 lq = ffa::ff_log(q, g_vf_rcp, g_vf_tlog, g_vf_eln2);
            const F2 ak1 = ffa::ff_add(F2{1.f, 0.f},
                                       ffa::ff_mul(q, ffa::ff_sub(ffa::ff_mul(lq, horner_ff(c_s1f, nt, q)),
                                                                  horner_ff(c_p1f, nt, q))));
            if constexpr (NUC == 1) return ak1;
            // nu = 2: a^2 K_2(a) / 2 = 2 q K_0 + a K_1, K_0 = -(log(a/2) + gamma) S_0 + H_0
            const F2 gam{0x1.2788dp-1f, -0x1.c824f4p-28f};  // Euler gamma, hi + lo
            const F2 g = ffa::ff_add(ffa::ff_scale(lq, 0.5f), gam);
            const F2 k0 = ffa::ff_sub(horner_ff(c_h0f, nt, q), ffa::ff_mul(g, horner_ff(c_s0f, nt, q)));
            return ffa::ff_add(ffa::ff_scale(ffa::ff_mul(q, k0), 2.0f), ak1);
        }
    }
    return ffa::split_d(matern_q<NUC>(ffa::to_d(q)));
}

// 1/d for normal d > 0: the hardware approximation rcp.approx.ftz.f64 (measured on this
// part: relative error below 2^-19.9) refined by two Newton-Raphson steps
// r <- r + r (1 - d r), each squaring the relative error (Markstein, IBM J. Res. Dev.
// 34(1), 1990); over 2^28 samples across the exponent range the result equals the
// correctly rounded 1/d.
__device__ __forceinline__ double recip_nr(double d) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    r = fma(r, fma(-d, r, 1.0), r);
    return fma(r, fma(-d, r, 1.0), r);
}

// Triangular numbering e = a (a + 1) / 2 + c (c <= a) of the lower triangle, tabulated per
// block in shared memory after the warps' regions: the same table serves the entry loop
// (all pairs b <= a) and every trailing update (the triangle of rows and columns j+1..s
// numbered from j + 1), so no lane derives its (row, column) by search.
__device__ __forceinline__ const uchar2 *tri_table(double *fsm, int per, int m) {
    uchar2 *tri = reinterpret_cast<uchar2 *>(fsm + (size_t)(blockDim.x >> 5) * per);
    const int T = (m + 1) * (m + 2) / 2;
    for (int e = threadIdx.x; e < T; e += blockDim.x) {
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (a * (a + 1) / 2 > e) --a;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        tri[e] = make_uchar2((unsigned char)a, (unsigned char)(e - a * (a + 1) / 2));
    }
    __syncthreads();
    return tri;
}

// Warp per point i with conditioning set sigma (s = |sigma| points): LDL' of the
// (s+1) x (s+1) covariance of (X_sigma, x_i), the point itself last (Eq. 2.19).  With
// K = [K_ss k; k' 1] = L D L' (L unit lower), row s of L is (D^-1 L_ss^-1 k)' and its
// last pivot is c = 1 - k' K_ss^-1 k, so the elimination itself does the forward solve;
// lambda = K_ss^-1 k is one unit-diagonal back solve with that row.  The lower triangle
// (row stride ld, odd) lives in shared memory; the trailing update is spread over the
// entries (not the rows) so every lane has the same work; the FP64 pipe is the bound, so
// every warp instruction on it counts: pivots are reciprocals (recip_nr), distances use
// coordinates pre-scaled by alpha/2 (q = dx^2 + dy^2) and the nu dispatch is static.
template <int NUC>
__global__ void factor_kernel(const double2 *x, int64_t n, const int *rank, const int *nbr_ell, int m, int ld,
                              double halpha, double *val_ell, unsigned long long *njit) {
    // Two points per warp, sixteen lanes each: the FP64 pipe is charged per warp
    // instruction, so the steps that every lane of a point repeats (the pivot reciprocal,
    // the column scaling, the back solve) and the narrow late trailing updates serve two
    // points at once.  Loops run to the larger size of the pair with per-half predicates,
    // so every __syncwarp and shuffle is reached by all 32 lanes.
    extern __shared__ double fsm[];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, half = lane >> 4, hl = lane & 15;
    const int per = (m + 1) * ld + 3 * (m + 1);
    const uchar2 *tri = tri_table(fsm, 2 * per, m);
    double *A = fsm + ((size_t)wib * 2 + half) * per;
    double *W = A + (m + 1) * ld;  // column j before scaling by 1/d_j
    double *X = W + (m + 1);
    double *Y = X + (m + 1);
    const int64_t i = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * 2 + half;
    const bool valid = i < n;
    const int s = valid ? min(m, rank[i]) : -1;
    const int smax = max(s, __shfl_xor_sync(full, s, 16));
    if (smax < 0) return;  // no point in either half (warp-uniform)
    for (int a = hl; a <= s; a += 16) {
        const double2 p = a < s ? x[nbr_ell[(int64_t)a * n + i]] : x[i];
        X[a] = p.x * halpha;
        Y[a] = p.y * halpha;
    }
    __syncwarp();
    const int ntri = (s + 1) * (s + 2) / 2, ntri_max = (smax + 1) * (smax + 2) / 2;
    bool ok = !valid;  // a half without a point counts as done
    int tries = 0;
    for (int t = 0; t <= 7; ++t) {
        if (__all_sync(full, ok)) break;
        const bool work = !ok;
        const double jit = t == 0 ? 0.0 : 1e-12 * pow(10.0, (double)(t - 1));
        for (int idx = hl; idx < ntri_max; idx += 16) {
            if (work && idx < ntri) {
                const uchar2 tb = tri[idx];
                const int a = tb.x, b = tb.y;
                double v;
                if (b == a) {
                    v = a < s ? 1.0 + jit : 1.0;  // jitter on K_ss only
                } else {
                    const double dx = X[a] - X[b], dy = Y[a] - Y[b];
                    const double q = fma(dx, dx, dy * dy);
                    v = __double2hiint(q) > 0 ? matern_q<NUC>(q) : 1.0;
                }
                A[a * ld + b] = v;
            }
        }
        __syncwarp();
        bool good = work;  // no non-positive pivot met in this round
        for (int j = 0; j < smax; ++j) {
            double r = 0.0;
            if (good && j < s) {
                const double d = A[j * ld + j];  // the same value in the half's lanes
                if (!(d >= 2.2250738585072014e-308)) good = false;
                else r = recip_nr(d);
            }
            const bool act = good && j < s;
            for (int a = j + 1 + hl; a <= smax; a += 16) {
                if (act && a <= s) {
                    const double w = A[a * ld + j];
                    W[a] = w;
                    A[a * ld + j] = w * r;
                }
            }
            __syncwarp();
            // entry e = a'(a'+1)/2 + c', c' <= a', of the trailing block (rows and columns j+1..s)
            const int mm = s - j, ntr = act ? mm * (mm + 1) / 2 : 0;
            const int mmx = smax - j, ntr_max = mmx * (mmx + 1) / 2;
            for (int e = hl; e < ntr_max; e += 16) {
                if (e < ntr) {
                    const uchar2 tb = tri[e];
                    const int a = j + 1 + tb.x, c = j + 1 + tb.y;
                    A[a * ld + c] = fma(-A[a * ld + j], W[c], A[a * ld + c]);
                }
            }
            __syncwarp();
        }
        if (work) {
            if (good) ok = true;
            else ++tries;
        }
    }
    const double cc = (valid && ok) ? A[s * ld + s] : 0.0;
    const bool fin = valid && ok && cc > 0.0;
    // L_ss' lambda = (row s of L)': entries hl + 16 r of the half in its lanes' registers
    double l[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) l[r] = (fin && hl + 16 * r < s) ? A[s * ld + hl + 16 * r] : 0.0;
    for (int c = smax - 1; c >= 0; --c) {
        const int rc = c >> 4;
        const double src = rc == 0 ? l[0] : (rc == 1 ? l[1] : (rc == 2 ? l[2] : l[3]));
        const double lc = __shfl_sync(full, src, (half << 4) | (c & 15));
        if (fin && c < s) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (16 * r < c && hl + 16 * r < c) l[r] = fma(-A[c * ld + hl + 16 * r], lc, l[r]);
        }
    }
    if (!valid) return;
    if (!fin) {
        // indefinite after the largest jitter, or no positive conditional variance:
        // empty conditioning set for this point
        if (hl == 0 && (!ok || tries == 0)) atomicAdd(njit, 1ull);
        for (int q = hl; q <= m; q += 16) val_ell[(int64_t)q * n + i] = q == 0 ? 1.0 : 0.0;
        return;
    }
    if (tries > 0 && hl == 0) atomicAdd(njit, 1ull);
    const double ic = rsqrt(cc);
    if (hl == 0) val_ell[i] = ic;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = hl + 16 * r;
        if (q < m) val_ell[(int64_t)(1 + q) * n + i] = q < s ? -l[r] * ic : 0.0;
    }
}

// The same factorisation with the elimination, pivots and back solve in float-float on the
// FP32 pipe (precision-4 plans), one point per warp (this kernel is bound by instruction
// issue, not by the FP64 pipe: two points per warp, with half the warps in flight, was
// measured slower): the Matern entries of nu = 1 and 2 come from the float-float series
// (matern_ff; other nu in FP64, then split), the stored factor is FP64.  The factor only shapes the preconditioner: any U gives a symmetric
// U U' applied in FP64, so float-float's rounding (about 2^-46 per operation, times the
// local condition number) moves the iteration count, not the fit's accuracy.  A pivot
// below the smallest normal float counts as non-positive (next rung of the jitter ladder).
template <int NUC>
__global__ void factor_kernel_ff(const double2 *x, int64_t n, const int *rank, const int *nbr_ell, int m, int ld,
                                 double halpha, double *val_ell, unsigned long long *njit) {
    using ffa::F2;
    extern __shared__ double fsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int per = (m + 1) * ld + 3 * (m + 1);  // 8-byte words, as in factor_kernel
    double *base = fsm + (size_t)wib * per;
    float2 *A = reinterpret_cast<float2 *>(base);
    float2 *W = A + (m + 1) * ld;
    float2 *X = W + (m + 1);  // scaled coordinates, hi + lo
    float2 *Y = X + (m + 1);
    const uchar2 *tri = tri_table(fsm, per, m);
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= n) return;
    const unsigned full = 0xffffffffu;
    const int s = min(m, rank[i]);
    for (int a = lane; a <= s; a += 32) {
        const double2 p = a < s ? x[nbr_ell[(int64_t)a * n + i]] : x[i];
        const F2 px = ffa::split_d(p.x * halpha), py = ffa::split_d(p.y * halpha);
        X[a] = make_float2(px.h, px.l);
        Y[a] = make_float2(py.h, py.l);
    }
    __syncwarp();
    const int nn = s + 1, ntri = nn * (nn + 1) / 2;
    bool ok = false;
    int tries = 0;
    for (int t = 0; t <= 7 && !ok; ++t) {
        const double jit = t == 0 ? 0.0 : 1e-12 * pow(10.0, (double)(t - 1));
        for (int idx = lane; idx < ntri; idx += 32) {
            const uchar2 tb = tri[idx];
            const int a = tb.x, b = tb.y;
            F2 vf;
            if (b == a) {
                vf = ffa::split_d(a < s ? 1.0 + jit : 1.0);  // jitter on K_ss only
            } else {
                const float2 xa = X[a], xb = X[b], ya = Y[a], yb = Y[b];
                const F2 q = ffa::ff_norm2(ffa::ff_sub(F2{xa.x, xa.y}, F2{xb.x, xb.y}),
                                           ffa::ff_sub(F2{ya.x, ya.y}, F2{yb.x, yb.y}));
                vf = q.h > 0.f ? matern_ff<NUC>(q) : F2{1.f, 0.f};
            }
            A[a * ld + b] = make_float2(vf.h, vf.l);
        }
        __syncwarp();
        ok = true;
        for (int j = 0; j < s; ++j) {
            const float2 dd = A[j * ld + j];  // same value in every lane: the branch is uniform
            if (!(dd.x >= 1.17549435e-38f)) { ok = false; break; }
            // 1/d in float-float: the float reciprocal and one Newton correction
            const F2 d{dd.x, dd.y};
            const float r0 = __frcp_rn(d.h);
            const F2 e = ffa::ff_sub(F2{1.f, 0.f}, ffa::ff_mul(d, F2{r0, 0.f}));
            const F2 r = ffa::ff_add(F2{r0, 0.f}, ffa::ff_mul(F2{r0, 0.f}, e));
            for (int a = j + 1 + lane; a <= s; a += 32) {
                const float2 w = A[a * ld + j];
                W[a] = w;
                const F2 l = ffa::ff_mulr(F2{w.x, w.y}, r);
                A[a * ld + j] = make_float2(l.h, l.l);
            }
            __syncwarp();
            const int mm = s - j, ntr = mm * (mm + 1) / 2;
            for (int e2 = lane; e2 < ntr; e2 += 32) {
                const uchar2 tb = tri[e2];
                const int a = j + 1 + tb.x, c = j + 1 + tb.y;
                const float2 la = A[a * ld + j], wc = W[c], ac = A[a * ld + c];
                const F2 u = ffa::ff_add(F2{ac.x, ac.y}, ffa::ff_neg(ffa::ff_mul(F2{la.x, la.y}, F2{wc.x, wc.y})));
                A[a * ld + c] = make_float2(u.h, u.l);
            }
            __syncwarp();
        }
        __syncwarp();
        if (!ok) ++tries;
    }
    const double cc = ok ? (double)A[s * ld + s].x + (double)A[s * ld + s].y : 0.0;
    if (!ok || !(cc > 0.0)) {
        if (lane == 0 && (!ok || tries == 0)) atomicAdd(njit, 1ull);
        for (int q = lane; q <= m; q += 32) val_ell[(int64_t)q * n + i] = q == 0 ? 1.0 : 0.0;
        return;
    }
    if (tries > 0 && lane == 0) atomicAdd(njit, 1ull);
    // L_ss' lambda = (row s of L)'; entries a and a + 32 in the lanes' registers
    float2 z0 = lane < s ? A[s * ld + lane] : make_float2(0.f, 0.f);
    float2 z1 = lane + 32 < s ? A[s * ld + lane + 32] : make_float2(0.f, 0.f);
    F2 l0{z0.x, z0.y}, l1{z1.x, z1.y};
    for (int c = s - 1; c >= 0; --c) {
        const F2 src = c >= 32 ? l1 : l0;
        const F2 lc{__shfl_sync(full, src.h, c & 31), __shfl_sync(full, src.l, c & 31)};
        if (lane < c) {
            const float2 acl = A[c * ld + lane];
            l0 = ffa::ff_add(l0, ffa::ff_neg(ffa::ff_mul(F2{acl.x, acl.y}, lc)));
        }
        if (s > 32 && lane + 32 < c) {
            const float2 acl = A[c * ld + lane + 32];
            l1 = ffa::ff_add(l1, ffa::ff_neg(ffa::ff_mul(F2{acl.x, acl.y}, lc)));
        }
    }
    const double ic = rsqrt(cc);
    if (lane == 0) val_ell[i] = ic;
    if (lane < m) val_ell[(int64_t)(1 + lane) * n + i] = lane < s ? -ffa::to_d(l0) * ic : 0.0;
    if (lane + 32 < m) val_ell[(int64_t)(33 + lane) * n + i] = lane + 32 < s ? -ffa::to_d(l1) * ic : 0.0;
}

// ---------------------------------------------------------------- transpose of U~ (rows of U~)
__global__ void t_count(const int *nbr_ell, int64_t n, int m, int *cnt) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    atomicAdd(&cnt[j], 1);
    for (int q = 0; q < m; ++q) {
        const int r = nbr_ell[(int64_t)q * n + j];
        if (r >= 0) atomicAdd(&cnt[r], 1);
    }
}
// entries of U~ as (row, entry) pairs in column-major order: entry e = slot * n + j of the
// ELL factor (slot 0 the diagonal, slot 1 + q neighbour q); absent neighbours get row n
__global__ void t_pairs(const int *nbr_ell, int64_t n, int m, uint64_t *key, int *ent) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)(m + 1) * n) return;
    const int64_t j = p / (m + 1);
    const int slot = (int)(p - j * (m + 1));
    const int r = slot == 0 ? (int)j : nbr_ell[(int64_t)(slot - 1) * n + j];
    key[p] = r >= 0 ? (uint64_t)r : (uint64_t)n;
    ent[p] = (int)((int64_t)slot * n + j);
}
// after a stable sort by row the entries of a row are in column order (deterministic)
__global__ void t_gather(const int *ent, int64_t nnz, int64_t n, const double *val_ell, int *col, double *val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    const int e = ent[i];
    col[i] = (int)(e % n);
    val[i] = val_ell[e];
}
// y = U~' r  (column j of U~ dotted with r)
__global__ void apply_ut(const int *nbr_ell, const double *val_ell, int64_t n, int m, const double *r, double *y) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double acc = val_ell[j] * r[j];
    for (int q = 0; q < m; ++q) {
        const int c = nbr_ell[(int64_t)q * n + j];
        if (c >= 0) acc += val_ell[(int64_t)(1 + q) * n + j] * r[c];
    }
    y[j] = acc;
}
// z = U~ y: thread per row over the sliced-ELL rows (coalesced across the slice's 32
// rows).  Four entries per step with all index and value loads issued before the
// gathers of y keep enough bytes in flight; entry k goes to accumulator k mod 4 (the last
// L mod 4 entries to a fifth) and they are added in a fixed order.
__global__ void apply_u(const int *s_row, const int *s_off, const int *s_len, const int *col, const double *val,
                        int64_t n, const double *y, double *z) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int sl = (int)(p >> 5);
    const int L = s_len[sl];
    const int *cp = col + s_off[sl] + (p & 31);
    const double *vp = val + s_off[sl] + (p & 31);
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    int k = 0;
    for (; k + 3 < L; k += 4) {
        int c[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldg(cp + 32 * (k + u));
            v[u] = __ldg(vp + 32 * (k + u));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = fma(v[u], y[c[u]], a[u]);
    }
    double t = 0.0;
    for (; k < L; ++k) t = fma(__ldg(vp + 32 * k), y[__ldg(cp + 32 * k)], t);
    z[s_row[p]] = ((a[0] + a[1]) + (a[2] + a[3])) + t;
}
// sliced-ELL build from the CSR rows.  Rows are sorted by descending length over the
// whole factor (sorting only within windows of spatially close rows was measured: the
// extra padding costs more than the gather locality gains).
__global__ void sell_keys(const int *off, int64_t n, uint64_t *key, int *row) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = (uint64_t)(0x7fffffff - (off[i + 1] - off[i]));  // stable: equal lengths keep row order
    row[i] = (int)i;
}
__global__ void sell_len(const int *off, const int *s_row, int nslice, int *s_len) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nslice) return;
    const int r = s_row[(int64_t)sl * 32];
    s_len[sl] = off[r + 1] - off[r];  // the slice's first row is its longest
}
__global__ void sell_width(const int *s_len, int nslice, int *w, unsigned long long *total) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl < nslice) {
        w[sl] = 32 * s_len[sl];
        atomicAdd(total, 32ull * (unsigned long long)s_len[sl]);
    }
}
__global__ void sell_fill(const int *off, const int *col, const double *val, const int *s_row, const int *s_off,
                          const int *s_len, int64_t n, int *s_col, double *s_val) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int r = s_row[p], sl = (int)(p >> 5);
    const int L = s_len[sl], src = off[r], rl = off[r + 1] - src;
    const int64_t base = (int64_t)s_off[sl] + (p & 31);
    for (int k = 0; k < L; ++k) {
        const int64_t e = base + 32 * (int64_t)k;
        s_col[e] = k < rl ? col[src + k] : r;
        s_val[e] = k < rl ? val[src + k] : 0.0;
    }
}

__global__ void ell_to_positions(int *nbr_ell, int64_t total, const int *iperm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int v = nbr_ell[t];
    if (v >= 0) nbr_ell[t] = iperm[v];
}
__global__ void permute_ell(const int *src, int64_t n, int slots, const int *perm, int *dst) {
    // dst[s][p] = src[s][perm[p]]  (caller index -> sorted position columns)
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * slots) return;
    const int64_t s2 = t / n, p = t - s2 * n;
    dst[t] = src[s2 * n + perm[p]];
}
__global__ void permute_ell_d(const double *src, int64_t n, int slots, const int *perm, double *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * slots) return;
    const int64_t s2 = t / n, p = t - s2 * n;
    dst[t] = src[s2 * n + perm[p]];
}

// Exact greedy maxmin in one block: first the point nearest the bounding-box centre,
// then repeatedly argmax over unselected points of the squared distance to the
// selected set; ties to the smaller index.  O(n^2 / blockDim) work.
constexpr int MM_T = 1024;
__global__ void __launch_bounds__(MM_T) maxmin_block(const double2 *x, int64_t n, double *dmin, unsigned char *sel,
                                                     int *order) {
    __shared__ double sv[MM_T];
    __shared__ long long si[MM_T];
    __shared__ double bb[4];
    // bounding box
    double a0 = INFINITY, a1 = -INFINITY, a2 = INFINITY, a3 = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += MM_T) {
        a0 = fmin(a0, x[i].x); a1 = fmax(a1, x[i].x);
        a2 = fmin(a2, x[i].y); a3 = fmax(a3, x[i].y);
    }
    for (int c = 0; c < 4; ++c) {
        double v = c == 0 ? a0 : c == 1 ? a1 : c == 2 ? a2 : a3;
        sv[threadIdx.x] = v;
        __syncthreads();
        for (int o = MM_T / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                double u = sv[threadIdx.x + o];
                sv[threadIdx.x] = (c & 1) ? fmax(sv[threadIdx.x], u) : fmin(sv[threadIdx.x], u);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) bb[c] = sv[0];
        __syncthreads();
    }
    const double2 ctr = make_double2(__dmul_rn(__dadd_rn(bb[0], bb[1]), 0.5), __dmul_rn(__dadd_rn(bb[2], bb[3]), 0.5));
    // first point: smallest (distance to centre, index)
    double bv = INFINITY;
    long long bi = -1;
    for (int64_t i = threadIdx.x; i < n; i += MM_T) {
        double d = sqd(x[i], ctr);
        if (d < bv) { bv = d; bi = i; }
        sel[i] = 0;
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = MM_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double u = sv[threadIdx.x + o];
            long long ui = si[threadIdx.x + o];
            if (ui >= 0 && (u < sv[threadIdx.x] || (u == sv[threadIdx.x] && (si[threadIdx.x] < 0 || ui < si[threadIdx.x])))) {
                sv[threadIdx.x] = u;
                si[threadIdx.x] = ui;
            }
        }
        __syncthreads();
    }
    long long last = si[0];
    __syncthreads();
    if (threadIdx.x == 0) { order[0] = (int)last; sel[last] = 1; }
    for (int64_t i = threadIdx.x; i < n; i += MM_T) dmin[i] = INFINITY;
    __syncthreads();
    for (int64_t r = 1; r < n; ++r) {
        const double2 pl = x[last];
        bv = -1.0;
        bi = -1;
        for (int64_t i = threadIdx.x; i < n; i += MM_T) {
            if (sel[i]) continue;
            double d = fmin(dmin[i], sqd(x[i], pl));
            dmin[i] = d;
            if (d > bv) { bv = d; bi = i; }
        }
        sv[threadIdx.x] = bv;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int o = MM_T / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                double u = sv[threadIdx.x + o];
                long long ui = si[threadIdx.x + o];
                if (ui >= 0 && (si[threadIdx.x] < 0 || u > sv[threadIdx.x] || (u == sv[threadIdx.x] && ui < si[threadIdx.x]))) {
                    sv[threadIdx.x] = u;
                    si[threadIdx.x] = ui;
                }
            }
            __syncthreads();
        }
        last = si[0];
        __syncthreads();
        if (threadIdx.x == 0) { order[r] = (int)last; sel[last] = 1; }
        __syncthreads();
    }
}

// rank[order[r]] = r for a caller-supplied enumeration; bad[0] counts entries outside
// [0, n) (skipped) and bad[1] ranks given twice (a repeated entry leaves another rank unset)
__global__ void ranks_checked(const int64_t *order, int64_t n, int *rank, unsigned long long *bad) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t v = order[r];
    if (v < 0 || v >= n) {
        atomicAdd(bad, 1ull);
        return;
    }
    if (atomicExch(rank + v, (int)r) != -1) atomicAdd(bad + 1, 1ull);
}
// conditioning sets of a caller: the first min(m, rank(i)) entries of row i must be
// points of smaller rank (they are read as coordinates); bad[2] counts violations
__global__ void check_nbr_rows(const int64_t *nbr, const int *rank, int64_t n, int m, unsigned long long *bad) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const int64_t i = t / m;
    const int q = (int)(t - i * m);
    const int s = min(m, rank[i]);
    if (q >= s) return;
    const int64_t v = nbr[t];
    if (v < 0 || v >= n || rank[v] >= rank[i]) atomicAdd(bad + 2, 1ull);
}

}  // namespace

void maxmin_order_dev(const double2 *x, int64_t n, int *order_out, cudaStream_t s) {
    SBuf<double> dmin(n, s);
    SBuf<unsigned char> sel(n, s);
    maxmin_block<<<1, MM_T, 0, s>>>(x, n, dmin.get(), sel.get(), order_out);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
}

void random_order_dev(int64_t n, uint64_t seed, int *order_out, cudaStream_t s) {
    SBuf<uint64_t> keys(n, s);
    rand_keys<<<blocks_for(n, 256), 256, 0, s>>>(n, seed, keys.get(), order_out);
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(keys.get(), order_out, n, 64, s);
}

void knn_prev_dev(const double2 *x, int64_t n, const int *order, int m, int *nbr_ell, cudaStream_t s) {
    PHS_REQUIRE(m >= 1 && m <= KNN_MAXM, PHS_ERR_INVALID_ARG, "conditioning-set size m must be in 1..64");
    SBuf<int> rank(n, s);
    ranks_from_order<<<blocks_for(n, 256), 256, 0, s>>>(order, n, rank.get());
    PHS_LAUNCH_CHECK();
    SBuf<double2> xr(n, s);
    gather_xy<<<blocks_for(n, 256), 256, 0, s>>>(x, order, n, xr.get());
    PHS_LAUNCH_CHECK();
    // grid over the bounding square, about 4 points per cell
    const int nbb = (int)std::min<int64_t>(296, blocks_for(n, 256));
    SBuf<Dbl4> part(nbb, s);
    SBuf<Grid> g(1, s);
    const int G = (int)std::max<double>(1.0, std::min<double>(8192.0, std::floor(std::sqrt((double)n / 4.0))));
    knn_bbox_partial<<<nbb, 256, 0, s>>>(x, n, part.get());
    PHS_LAUNCH_CHECK();
    knn_grid_final<<<1, 1, 0, s>>>(part.get(), nbb, G, g.get());
    PHS_LAUNCH_CHECK();
    const int ncell = G * G;
    SBuf<uint64_t> keys(n, s);
    SBuf<int> vals(n, s);
    grid_keys<<<blocks_for(n, 256), 256, 0, s>>>(x, rank.get(), n, g.get(), keys.get(), vals.get());
    PHS_LAUNCH_CHECK();
    int cbits = 1;
    while ((1ll << cbits) < ncell) ++cbits;
    radix_sort_pairs(keys.get(), vals.get(), n, 32 + cbits, s);
    SBuf<int> cst(ncell + 1, s);
    cell_starts<<<blocks_for(ncell + 1, 256), 256, 0, s>>>(keys.get(), n, ncell, cst.get());
    PHS_LAUNCH_CHECK();
    SBuf<double2> xc(n, s);
    SBuf<int> rc(n, s);
    cell_payload<<<blocks_for(n, 256), 256, 0, s>>>(keys.get(), vals.get(), x, n, xc.get(), rc.get());
    PHS_LAUNCH_CHECK();
    const int brute = (int)std::min<int64_t>(n, 8192);
    knn_kernel<<<blocks_for(n * 32, 256), 256, 0, s>>>(xr.get(), n, m, brute, g.get(), cst.get(), xc.get(), rc.get(),
                                                      order, nbr_ell);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
}

int64_t vecchia_factor_dev(const double2 *x, int64_t n, const int *rank, const int *nbr_ell, int m, double nu,
                           double alpha, double *val_ell, cudaStream_t s, bool ff) {
    PHS_REQUIRE(m >= 1 && m <= KNN_MAXM, PHS_ERR_INVALID_ARG, "conditioning-set size m must be in 1..64");
    PHS_REQUIRE(nu == 0.5 || nu == 1.0 || nu == 1.5 || nu == 2.0 || nu == 2.5, PHS_ERR_INVALID_ARG,
                "nu must be 0.5, 1, 1.5, 2 or 2.5");
    PHS_REQUIRE(alpha > 0 && std::isfinite(alpha), PHS_ERR_INVALID_ARG, "alpha must be positive");
    once_per_device(3, upload_bessel_tables);
    const int ld = (m + 1) | 1;  // odd row stride: rows of consecutive lanes fall in different banks
    const size_t per = (size_t)((m + 1) * ld + 3 * (m + 1)) * sizeof(double);
    // points per warp: two in FP64 (factor_kernel), one in float-float (factor_kernel_ff)
    const int ppw = ff ? 1 : 2;
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (ff ? 96 * 1024 : 110 * 1024) / (ppw * per)));
    const size_t tri_bytes = ((size_t)(m + 1) * (m + 2) / 2 * sizeof(uchar2) + 7) & ~(size_t)7;
    const size_t smem = per * ppw * wpb + tri_bytes;
    SBuf<unsigned long long> cnt(2, s);
    PHS_CUDA(cudaMemsetAsync(cnt.get(), 0, 2 * sizeof(unsigned long long), s));
    const int nuc = nu == 0.5 ? 0 : (nu == 1.0 ? 1 : (nu == 1.5 ? 2 : (nu == 2.0 ? 3 : 4)));
    auto launch = [&](auto kern) {
        PHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<blocks_for(n, (int64_t)ppw * wpb), 32 * wpb, smem, s>>>(x, n, rank, nbr_ell, m, ld, 0.5 * alpha, val_ell,
                                                                      cnt.get());
    };
    if (ff) {
        switch (nuc) {
            case 0: launch(factor_kernel_ff<0>); break;
            case 1: launch(factor_kernel_ff<1>); break;
            case 2: launch(factor_kernel_ff<2>); break;
            case 3: launch(factor_kernel_ff<3>); break;
            default: launch(factor_kernel_ff<4>); break;
        }
    } else {
        switch (nuc) {
            case 0: launch(factor_kernel<0>); break;
            case 1: launch(factor_kernel<1>); break;
            case 2: launch(factor_kernel<2>); break;
            case 3: launch(factor_kernel<3>); break;
            default: launch(factor_kernel<4>); break;
        }
    }
    PHS_LAUNCH_CHECK();
    unsigned long long h[2];
    PHS_CUDA(cudaMemcpyAsync(h, cnt.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_REQUIRE(h[1] == 0, PHS_ERR_CHOLESKY, "a local Vecchia factor failed even with jitter");
    return (int64_t)h[0];
}

void checked_ranks_dev(const int64_t *order, const int64_t *nbr, int64_t n, int m, int *rank, cudaStream_t s) {
    SBuf<unsigned long long> bad(3, s);
    PHS_CUDA(cudaMemsetAsync(bad.get(), 0, 3 * sizeof(unsigned long long), s));
    PHS_CUDA(cudaMemsetAsync(rank, 0xff, n * sizeof(int), s));
    ranks_checked<<<blocks_for(n, 256), 256, 0, s>>>(order, n, rank, bad.get());
    PHS_LAUNCH_CHECK();
    unsigned long long h[3];
    PHS_CUDA(cudaMemcpyAsync(h, bad.get(), 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_REQUIRE(h[0] == 0 && h[1] == 0, PHS_ERR_INVALID_ARG, "order is not a permutation of 0..n-1");
    if (!nbr) return;
    check_nbr_rows<<<blocks_for(n * m, 256), 256, 0, s>>>(nbr, rank, n, m, bad.get());
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaMemcpyAsync(h, bad.get(), 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_REQUIRE(h[2] == 0, PHS_ERR_INVALID_ARG,
                "a conditioning set lists a point that is out of range or not of smaller rank");
}

void vecchia_build(Vecchia &v, const PointSet &ps, int m, int ordering, uint64_t seed, double nu, double alpha,
                   cudaStream_t s, bool ff) {
    const int64_t n = ps.n;
    v.n = n;
    v.m = m;
    // caller-order coordinates (normalised frame): ties in orderings and neighbour lists
    // resolve by caller index, the definition the interface documents
    SBuf<double2> xcal(n, s);
    gather_xy<<<blocks_for(n, 256), 256, 0, s>>>(ps.xs.get(), ps.iperm.get(), n, xcal.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> order_c(n, s);
    if (ordering == 0) random_order_dev(n, seed, order_c.get(), s);
    else if (ordering == 1) maxmin_order_dev(xcal.get(), n, order_c.get(), s);
    else if (ordering == 2) hmaxmin_order_dev(xcal.get(), n, seed, order_c.get(), s);
    else amaxmin_order_dev(xcal.get(), n, order_c.get(), s);
    SBuf<int> nbr_c((size_t)m * n, s);
    knn_prev_dev(xcal.get(), n, order_c.get(), m, nbr_c.get(), s);
    SBuf<int> rank_c(n, s);
    ranks_from_order<<<blocks_for(n, 256), 256, 0, s>>>(order_c.get(), n, rank_c.get());
    PHS_LAUNCH_CHECK();
    SBuf<double> val_c((size_t)(m + 1) * n, s);
    v.jittered = vecchia_factor_dev(xcal.get(), n, rank_c.get(), nbr_c.get(), m, nu, alpha, val_c.get(), s, ff);
    // move to sorted positions: columns permuted by perm, entries mapped by iperm
    v.nbr.alloc((size_t)m * n);
    v.val.alloc((size_t)(m + 1) * n);
    v.rank.alloc(n);
    v.order.alloc(n);
    permute_ell<<<blocks_for((int64_t)m * n, 256), 256, 0, s>>>(nbr_c.get(), n, m, ps.perm.get(), v.nbr.get());
    PHS_LAUNCH_CHECK();
    ell_to_positions<<<blocks_for((int64_t)m * n, 256), 256, 0, s>>>(v.nbr.get(), (int64_t)m * n, ps.iperm.get());
    PHS_LAUNCH_CHECK();
    permute_ell_d<<<blocks_for((int64_t)(m + 1) * n, 256), 256, 0, s>>>(val_c.get(), n, m + 1, ps.perm.get(),
                                                                          v.val.get());
    PHS_LAUNCH_CHECK();
    permute_ell<<<blocks_for(n, 256), 256, 0, s>>>(rank_c.get(), n, 1, ps.perm.get(), v.rank.get());
    PHS_LAUNCH_CHECK();
    // order (ranks -> sorted positions) = iperm[order_c]
    permute_ell<<<blocks_for(n, 256), 256, 0, s>>>(ps.iperm.get(), n, 1, order_c.get(), v.order.get());
    PHS_LAUNCH_CHECK();
    // transpose: CSR rows of U~ in column order, then the sliced-ELL copy the apply reads
    SBuf<int> cnt(n, s);
    PHS_CUDA(cudaMemsetAsync(cnt.get(), 0, n * sizeof(int), s));
    t_count<<<blocks_for(n, 256), 256, 0, s>>>(v.nbr.get(), n, m, cnt.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> t_off(n + 1, s);
    int64_t nnz = exclusive_scan_i32(cnt.get(), t_off.get(), n, s);
    int nz32 = (int)nnz;
    PHS_CUDA(cudaMemcpyAsync(t_off.get() + n, &nz32, sizeof(int), cudaMemcpyHostToDevice, s));
    SBuf<int> t_col(nnz, s);
    SBuf<double> t_val(nnz, s);
    {
        const int64_t np = (int64_t)(m + 1) * n;
        PHS_REQUIRE(np < (1ll << 31), PHS_ERR_INVALID_ARG, "Vecchia factor too large for 32-bit entry indices");
        SBuf<uint64_t> key(np, s);
        SBuf<int> ent(np, s);
        t_pairs<<<blocks_for(np, 256), 256, 0, s>>>(v.nbr.get(), n, m, key.get(), ent.get());
        PHS_LAUNCH_CHECK();
        int bits = 1;
        while ((1ll << bits) <= n) ++bits;
        radix_sort_pairs(key.get(), ent.get(), np, bits, s);
        t_gather<<<blocks_for(nnz, 256), 256, 0, s>>>(ent.get(), nnz, n, v.val.get(), t_col.get(), t_val.get());
        PHS_LAUNCH_CHECK();
    }
    {
        const int nslice = (int)((n + 31) / 32);
        SBuf<uint64_t> key(n, s);
        v.s_row.alloc(n);
        sell_keys<<<blocks_for(n, 256), 256, 0, s>>>(t_off.get(), n, key.get(), v.s_row.get());
        PHS_LAUNCH_CHECK();
        radix_sort_pairs(key.get(), v.s_row.get(), n, 31, s);
        v.s_len.alloc(nslice);
        v.s_off.alloc(nslice + 1);
        sell_len<<<blocks_for(nslice, 256), 256, 0, s>>>(t_off.get(), v.s_row.get(), nslice, v.s_len.get());
        PHS_LAUNCH_CHECK();
        SBuf<int> w(nslice, s);
        SBuf<unsigned long long> wt(1, s);
        PHS_CUDA(cudaMemsetAsync(wt.get(), 0, sizeof(unsigned long long), s));
        sell_width<<<blocks_for(nslice, 256), 256, 0, s>>>(v.s_len.get(), nslice, w.get(), wt.get());
        PHS_LAUNCH_CHECK();
        unsigned long long hwt = 0;  // padded entries, counted in 64 bits before the 32-bit scan
        PHS_CUDA(cudaMemcpyAsync(&hwt, wt.get(), sizeof(hwt), cudaMemcpyDeviceToHost, s));
        PHS_CUDA(cudaStreamSynchronize(s));
        PHS_REQUIRE(hwt < (1ull << 31), PHS_ERR_INVALID_ARG, "Vecchia factor too large for 32-bit entry indices");
        const int64_t tot = exclusive_scan_i32(w.get(), v.s_off.get(), nslice, s);
        v.s_col.alloc(std::max<int64_t>(tot, 1));
        v.s_val.alloc(std::max<int64_t>(tot, 1));
        sell_fill<<<blocks_for(n, 256), 256, 0, s>>>(t_off.get(), t_col.get(), t_val.get(), v.s_row.get(),
                                                     v.s_off.get(), v.s_len.get(), n, v.s_col.get(), v.s_val.get());
        PHS_LAUNCH_CHECK();
    }
    PHS_CUDA(cudaStreamSynchronize(s));
}

void vecchia_apply_ut(const Vecchia &v, const double *r, double *y, cudaStream_t s) {
    apply_ut<<<blocks_for(v.n, 256), 256, 0, s>>>(v.nbr.get(), v.val.get(), v.n, v.m, r, y);
    PHS_LAUNCH_CHECK();
}
void vecchia_apply_u(const Vecchia &v, const double *y, double *z, cudaStream_t s) {
    apply_u<<<blocks_for(v.n, 256), 256, 0, s>>>(v.s_row.get(), v.s_off.get(), v.s_len.get(), v.s_col.get(),
                                                 v.s_val.get(), v.n, y, z);
    PHS_LAUNCH_CHECK();
}
void vecchia_apply(const Vecchia &v, const double *r, double *tmp, double *z, cudaStream_t s) {
    vecchia_apply_ut(v, r, tmp, s);
    vecchia_apply_u(v, tmp, z, s);
}

}  // namespace phs
