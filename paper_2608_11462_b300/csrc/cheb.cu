// cheb.cu -- far field of the distance kernel |x - y| (odd k: r^k = r * r^{k-1}, Eq. 2.6
// with the distance core kernel of Sec. 4) by Chebyshev interpolation on every box.
//
// The paper names the distance-kernel FMM as future work and gives no expansions; this
// file uses tensor-product Chebyshev interpolation (kernel-independent FMM):
//   nodes       xb_m = cos((2m+1) pi / (2q)), m = 0..q-1, per axis; box node (m1, m2)
//   basis       S(xb, t) = 1/q + (2/q) sum_{k=1}^{q-1} T_k(xb) T_k(t)  (= Lagrange basis)
//   P2M         W[m] = sum_j q_j S(xb_m1, s_j1) S(xb_m2, s_j2),  s_j = (x_j - c)/h
//   M2M / L2L   child nodes sit at +-1/2 + xb/2 in the parent frame
//   M2L         L_t[m] += h * sum_n |xb_m - xb_n - 2 o| W_s[n]  (o = source offset in
//               box widths; |x - y| is homogeneous, so one matrix K_o per offset class
//               serves every level after scaling by the half-width h), applied in
//               compressed form: the 40 matrices share a target basis U (left singular
//               vectors of [K_o ...]) and a source basis V (right singular vectors of
//               [K_o; ...]; U = V by symmetry), truncated where the singular values fall below lr_eps times
//               the largest, so K_o ~ U C_o V' and an interaction costs rt x rs instead
//               of (q^2)^2: W~ = V' W once per source box, L~ += C_o (S_o W~) per
//               V-list entry, L = U L~ once per target box
//   L2P         pot(x) = sum_m S(xb_m1, s1) S(xb_m2, s2) L[m]
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "geom.cuh"
#include "hadamard.cuh"
#include "phs_internal.cuh"

namespace phs {

constexpr int kChebMaxQ = 16;
// rank cap of the compressed M2L: the tensor-core form keeps 6 digit diagonals of its
// output columns in 512 TMEM columns (6 x 80); at q = 16 the 81st singular value is
// 8.3e-13 of the largest, so the cap costs no accuracy the interpolation has
constexpr int kChebMaxRank = 80;
constexpr int CHEB_T = 256;

namespace {

__device__ __forceinline__ void box_center_h(const TreeView &tv, int b, double &cx, double &cy, double &h) {
    double w;
    box_geom(tv, b, cx, cy, w);
    h = 0.5 * w;
}

// S(xb_m, t) for m = 0..q-1 (Tn[k*q + m] = T_k(xb_m))
__device__ __forceinline__ void cheb_basis(double t, int q, const double *Tn, double *S) {
    double Tk[kChebMaxQ];
    Tk[0] = 1.0;
    if (q > 1) Tk[1] = t;
    for (int k = 2; k < q; ++k) Tk[k] = 2.0 * t * Tk[k - 1] - Tk[k - 2];
    const double iq = 1.0 / q;
    for (int m = 0; m < q; ++m) {
        double s = 0.0;
        for (int k = 1; k < q; ++k) s += Tn[k * q + m] * Tk[k];
        S[m] = iq + 2.0 * iq * s;
    }
}

// P2M on leaves: W[b][d][m1*q+m2]
__global__ void cheb_p2m(TreeView tv, const int *leaf_box, const double2 *xs, const double *t, int power, int nd, int q,
                         const double *Tn_g, double *W) {
    __shared__ double Tn[kChebMaxQ * kChebMaxQ];
    __shared__ double S1[32][kChebMaxQ], S2[32][kChebMaxQ], qd[32][10];
    for (int i = threadIdx.x; i < q * q; i += blockDim.x) Tn[i] = Tn_g[i];
    const int b = leaf_box[blockIdx.x];
    double cx, cy, h;
    box_center_h(tv, b, cx, cy, h);
    const double ih = 1.0 / h;
    const int s = tv.start[b], e = tv.end[b];
    const int qq = q * q;
    const int m = threadIdx.x;  // node index (q*q <= 256)
    const int m1 = m / q, m2 = m - (m / q) * q;
    double acc[10];
    for (int d = 0; d < nd; ++d) acc[d] = 0.0;
    __syncthreads();
    for (int j0 = s; j0 < e; j0 += 32) {
        if (threadIdx.x < 32) {
            const int j = j0 + threadIdx.x;
            if (j < e) {
                const double2 p = xs[j];
                cheb_basis(fmin(1.0, fmax(-1.0, (p.x - cx) * ih)), q, Tn, S1[threadIdx.x]);
                cheb_basis(fmin(1.0, fmax(-1.0, (p.y - cy) * ih)), q, Tn, S2[threadIdx.x]);
                double v[10];
                had_v(power, 0.5 * (p.x - cx) * ih, 0.5 * (p.y - cy) * ih, v);  // box-local densities
                const double tj = t[j];
                for (int d = 0; d < nd; ++d) qd[threadIdx.x][d] = v[d] * tj;
            } else {
                for (int d = 0; d < nd; ++d) qd[threadIdx.x][d] = 0.0;
                for (int k = 0; k < q; ++k) S1[threadIdx.x][k] = S2[threadIdx.x][k] = 0.0;
            }
        }
        __syncthreads();
        if (m < qq) {
            const int jn = min(32, e - j0);
            for (int jj = 0; jj < jn; ++jj) {
                const double sv = S1[jj][m1] * S2[jj][m2];
                for (int d = 0; d < nd; ++d) acc[d] += qd[jj][d] * sv;
            }
        }
        __syncthreads();
    }
    if (m < qq)
        for (int d = 0; d < nd; ++d) W[((size_t)b * nd + d) * qq + m] = acc[d];
}

// separable 2D application of the 1D child-node matrices A[sx], A[sy]:
// out[m1][m2] (+)= sum_{a,c} Ax(m1,a) Ay(m2,c) in[a][c], with TRANS selecting A' (L2L)
template <bool TRANS>
__device__ __forceinline__ double sep_apply(const double *Ax, const double *Ay, const double *in, double *tmp, int q,
                                            int m1, int m2, bool active) {
    // tmp[a][m2] = sum_c Ay(m2, c) in[a][c]
    const int qq = q * q;
    for (int idx = threadIdx.x; idx < qq; idx += blockDim.x) {
        const int a = idx / q, mm2 = idx - a * q;
        double s = 0.0;
        for (int c = 0; c < q; ++c) s += (TRANS ? Ay[c * q + mm2] : Ay[mm2 * q + c]) * in[a * q + c];
        tmp[idx] = s;
    }
    __syncthreads();
    double r = 0.0;
    if (active)
        for (int a = 0; a < q; ++a) r += (TRANS ? Ax[a * q + m1] : Ax[m1 * q + a]) * tmp[a * q + m2];
    __syncthreads();
    return r;
}

// M2M for the non-leaf boxes of one level; A holds [2][q][q]: A[s][m][m'] = S(xb_m, s*1 - 1/2 + xb_m'/2).
// Densities are box-local: each interpolated child density is mixed into the parent's
// through Rv (mix slot 49 + quadrant, see fmm.cu).
__global__ void cheb_m2m(TreeView tv, int b0, int nd, int q, const double *A, const double *mix, double *W) {
    __shared__ double in[kChebMaxQ * kChebMaxQ], tmp[kChebMaxQ * kChebMaxQ];
    extern __shared__ double ich[];  // [nd][q*q] interpolated child densities
    const int b = b0 + blockIdx.x;
    const int nc = tv.nchild[b];
    if (nc == 0) return;
    const int qq = q * q;
    const int m = threadIdx.x, m1 = m / q, m2 = m % q;
    const bool active = m < qq;
    double acc[10];
    for (int d = 0; d < nd; ++d) acc[d] = 0.0;
    for (int c = tv.child[b]; c < tv.child[b] + nc; ++c) {
        const int quad = (int)(tv.key[c] & 3);
        const double *Ax = A + (size_t)(quad & 1) * qq, *Ay = A + (size_t)((quad >> 1) & 1) * qq;
        for (int d = 0; d < nd; ++d) {
            for (int i = threadIdx.x; i < qq; i += blockDim.x) in[i] = W[((size_t)c * nd + d) * qq + i];
            __syncthreads();
            const double r = sep_apply<false>(Ax, Ay, in, tmp, q, m1, m2, active);
            if (active) ich[d * qq + m] = r;
        }
        const double *Rv = mix + (size_t)(49 + quad) * nd * nd;
        if (active)
            for (int l = 0; l < nd; ++l)
                for (int bb = 0; bb < nd; ++bb) acc[l] += Rv[l * nd + bb] * ich[bb * qq + m];
        __syncthreads();
    }
    if (active)
        for (int l = 0; l < nd; ++l) W[((size_t)b * nd + l) * qq + m] = acc[l];
}

// L2L for one level: interpolate each parent factor's potential to the child nodes,
// then mix into the child's factors through Ru (mix slot 53 + quadrant)
__global__ void cheb_l2l(TreeView tv, int b0, int nd, int q, const double *A, const double *mix, double *L) {
    __shared__ double in[kChebMaxQ * kChebMaxQ], tmp[kChebMaxQ * kChebMaxQ];
    extern __shared__ double ipar[];  // [nd][q*q]
    const int b = b0 + blockIdx.x;
    const int par = tv.parent[b];
    const int qq = q * q;
    const int m = threadIdx.x, m1 = m / q, m2 = m % q;
    const bool active = m < qq;
    const int quad = (int)(tv.key[b] & 3);
    const double *Ax = A + (size_t)(quad & 1) * qq, *Ay = A + (size_t)((quad >> 1) & 1) * qq;
    for (int d = 0; d < nd; ++d) {
        for (int i = threadIdx.x; i < qq; i += blockDim.x) in[i] = L[((size_t)par * nd + d) * qq + i];
        __syncthreads();
        const double r = sep_apply<true>(Ax, Ay, in, tmp, q, m1, m2, active);
        if (active) ipar[d * qq + m] = r;
    }
    const double *Ru = mix + (size_t)(53 + quad) * nd * nd;
    if (active)
        for (int a = 0; a < nd; ++a) {
            double s = 0.0;
            for (int l = 0; l < nd; ++l) s += Ru[l * nd + a] * ipar[l * qq + m];
            L[((size_t)b * nd + a) * qq + m] += s;
        }
}

// local potential of box b at point (x, y) for density d
__device__ __forceinline__ double cheb_l2p_point(const double *Lb, int q, const double *Tn, double sx, double sy) {
    double S1[kChebMaxQ], S2[kChebMaxQ];
    cheb_basis(sx, q, Tn, S1);
    cheb_basis(sy, q, Tn, S2);
    double r = 0.0;
    for (int a = 0; a < q; ++a) {
        double s = 0.0;
        for (int c = 0; c < q; ++c) s += S2[c] * Lb[a * q + c];
        r += S1[a] * s;
    }
    return r;
}

__global__ void cheb_l2p(TreeView tv, const int *leaf_box, const double2 *xs, int power, int nd, int q,
                         const double *Tn_g, const double *L, double *y) {
    extern __shared__ double lsm[];  // [nd][q*q] then Tn
    const int b = leaf_box[blockIdx.x];
    const int qq = q * q;
    double *Tn = lsm + nd * qq;
    for (int i = threadIdx.x; i < nd * qq; i += blockDim.x) lsm[i] = L[(size_t)b * nd * qq + i];
    for (int i = threadIdx.x; i < qq; i += blockDim.x) Tn[i] = Tn_g[i];
    __syncthreads();
    double cx, cy, h;
    box_center_h(tv, b, cx, cy, h);
    const double ih = 1.0 / h;
    for (int j = tv.start[b] + threadIdx.x; j < tv.end[b]; j += blockDim.x) {
        const double2 p = xs[j];
        const double sx = fmin(1.0, fmax(-1.0, (p.x - cx) * ih)), sy = fmin(1.0, fmax(-1.0, (p.y - cy) * ih));
        double S1[kChebMaxQ], S2[kChebMaxQ];
        cheb_basis(sx, q, Tn, S1);
        cheb_basis(sy, q, Tn, S2);
        double u[10];
        had_u(power, 0.5 * sx, 0.5 * sy, u);  // box-local factors
        double sum = 0.0;
        for (int d = 0; d < nd; ++d) {
            const double *Lb = lsm + d * qq;
            double r = 0.0;
            for (int a = 0; a < q; ++a) {
                double s = 0.0;
                for (int c = 0; c < q; ++c) s += S2[c] * Lb[a * q + c];
                r += S1[a] * s;
            }
            sum += u[d] * r;
        }
        y[j] += sum;
    }
}

// W~[b][d][j] = sum_n V[n][j] W[b][d][n]  (boxes b0.., all densities)
__global__ void cheb_compress(int b0, int nd, int qq, int rs, const double *V, const double *W, double *Wc) {
    extern __shared__ double wsh[];  // [nd][qq]
    const int b = b0 + blockIdx.x;
    for (int i = threadIdx.x; i < nd * qq; i += blockDim.x) wsh[i] = W[(size_t)b * nd * qq + i];
    __syncthreads();
    for (int o = threadIdx.x; o < nd * rs; o += blockDim.x) {
        const int d = o / rs, jj = o - d * rs;
        double acc = 0.0;
        for (int n = 0; n < qq; ++n) acc = fma(V[(size_t)n * rs + jj], wsh[d * qq + n], acc);
        Wc[((size_t)b * nd + d) * rs + jj] = acc;
    }
}

// L~_t[d][i] = sum over the V list of sum_j C[cls][i][j] (S[cls] W~_src)[d][j]  (C stored as C')
__global__ void cheb_m2l_lr(int b0, const int *v_off, const int *v_src, const unsigned char *v_cls, int nd, int rt,
                            int rs, const double *C, const double *mix, const double *Wc, double *Lc) {
    extern __shared__ double csm[];  // [nd][rs] source, then [nd][rs] mixed
    const int b = b0 + blockIdx.x;
    double *wmx = csm + nd * rs;
    double acc[10];
    for (int d = 0; d < nd; ++d) acc[d] = 0.0;
    const int i = threadIdx.x;
    for (int v = v_off[b]; v < v_off[b + 1]; ++v) {
        const int src = v_src[v];
        for (int o = threadIdx.x; o < nd * rs; o += blockDim.x) csm[o] = Wc[(size_t)src * nd * rs + o];
        __syncthreads();
        const double *S = mix + (size_t)v_cls[v] * nd * nd;
        for (int o = threadIdx.x; o < nd * rs; o += blockDim.x) {
            const int l = o / rs, jj = o - l * rs;
            double sacc = 0.0;
            for (int bb = 0; bb < nd; ++bb) sacc = fma(S[l * nd + bb], csm[bb * rs + jj], sacc);
            wmx[o] = sacc;
        }
        __syncthreads();
        if (i < rt) {
            const double *Cc = C + (size_t)v_cls[v] * rs * rt + i;  // C' [rs][rt]: coalesced over i
            for (int jj = 0; jj < rs; ++jj) {
                const double cv = Cc[(size_t)jj * rt];
                for (int d = 0; d < nd; ++d) acc[d] = fma(cv, wmx[d * rs + jj], acc[d]);
            }
        }
        __syncthreads();
    }
    if (i < rt)
        for (int d = 0; d < nd; ++d) Lc[((size_t)b * nd + d) * rt + i] = acc[d];
}

// L[b][d][m] = sc_b sum_i U[m][i] L~[b][d][i], sc_b = h w^power (the homogeneity scaling; U stored as U')
__global__ void cheb_expand(TreeView tv, int b0, int nd, int qq, int rt, int power, const double *U, const double *Lc,
                            double *L) {
    extern __shared__ double lsh[];  // [nd][rt]
    const int b = b0 + blockIdx.x;
    for (int o = threadIdx.x; o < nd * rt; o += blockDim.x) lsh[o] = Lc[(size_t)b * nd * rt + o];
    __syncthreads();
    const double w = box_width(tv.R, tv.level[b]);
    double sc = 0.5 * w;
    for (int k = 0; k < power; ++k) sc *= w;
    for (int o = threadIdx.x; o < nd * qq; o += blockDim.x) {
        const int d = o / qq, m = o - d * qq;
        double acc = 0.0;
        for (int k = 0; k < rt; ++k) acc = fma(U[(size_t)k * qq + m], lsh[d * rt + k], acc);  // U' [rt][qq]
        L[((size_t)b * nd + d) * qq + m] = sc * acc;
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
// R of a Householder QR of the column-major m x n matrix M (m >= n): column j's reflector
// v = a - alpha e_j (alpha = -sign(a_j) |a|) is applied to the columns right of j, spread
// over threads by column.  Backward stable: the singular values of R are those of M to
// within eps ||M||, which is what lets the truncation below reach 1e-12 (forming M'M
// first would square the condition and stop near 1e-8).
static std::vector<double> householder_r(int m, int n, std::vector<double> M) {
    const int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    for (int j = 0; j < n; ++j) {
        double *a = M.data() + (size_t)j * m;
        double nrm2 = 0.0;
        for (int i = j; i < m; ++i) nrm2 += a[i] * a[i];
        if (nrm2 == 0.0) continue;
        const double nrm = std::sqrt(nrm2), aj = a[j];
        const double alpha = aj > 0 ? -nrm : nrm;
        a[j] = aj - alpha;
        const double vv = nrm2 - aj * aj + a[j] * a[j];  // |v|^2
        auto update = [&](int k0, int k1) {
            for (int k = k0; k < k1; ++k) {
                double *c = M.data() + (size_t)k * m;
                double d = 0.0;
                for (int i = j; i < m; ++i) d += a[i] * c[i];
                const double fct = 2.0 * d / vv;
                for (int i = j; i < m; ++i) c[i] -= fct * a[i];
            }
        };
        const int rest = n - j - 1;
        if (rest >= 4 * nth) {
            std::vector<std::thread> th;
            const int per = (rest + nth - 1) / nth;
            for (int t = 0; t < nth; ++t) {
                const int k0 = j + 1 + t * per, k1 = std::min(n, k0 + per);
                if (k0 < k1) th.emplace_back(update, k0, k1);
            }
            for (auto &x : th) x.join();
        } else {
            update(j + 1, n);
        }
        a[j] = alpha;
    }
    std::vector<double> R((size_t)n * n, 0.0);  // column-major, upper triangle
    for (int k = 0; k < n; ++k)
        for (int i = 0; i <= k; ++i) R[(size_t)k * n + i] = M[(size_t)k * m + i];
    return R;
}

// Right singular vectors of the n x n column-major R by one-sided (Hestenes) Jacobi:
// column pairs of R are rotated until orthogonal, the rotations accumulated in V (which
// stays orthogonal to rounding whatever the stopping point).  On return the columns of V
// (column-major) are sorted by the norms of R's columns, the singular values, returned
// in s in decreasing order.  Pairs whose smaller column is below 1e-13 of the largest
// norm are left alone: such columns are truncated anyway and rotating rounding noise
// against rounding noise does not converge.
static void jacobi_right(int n, std::vector<double> &R, std::vector<double> &V, std::vector<double> &s) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto col2 = [&](const double *c) {
        double a = 0.0;
        for (int i = 0; i < n; ++i) a += c[i] * c[i];
        return a;
    };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double top = 0.0;
        for (int k = 0; k < n; ++k) top = std::max(top, col2(R.data() + (size_t)k * n));
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double *a = R.data() + (size_t)p * n, *b = R.data() + (size_t)q * n;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < n; ++i) {
                    al += a[i] * a[i];
                    be += b[i] * b[i];
                    ga += a[i] * b[i];
                }
                if (std::min(al, be) < 1e-26 * top || std::fabs(ga) <= 1e-14 * std::sqrt(al * be)) continue;
                rotated = true;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < n; ++i) {
                    const double x = a[i], y = b[i];
                    a[i] = c * x - sn * y;
                    b[i] = sn * x + c * y;
                }
                double *va = V.data() + (size_t)p * n, *vb = V.data() + (size_t)q * n;
                for (int i = 0; i < n; ++i) {
                    const double x = va[i], y = vb[i];
                    va[i] = c * x - sn * y;
                    vb[i] = sn * x + c * y;
                }
            }
        if (!rotated) break;
    }
    std::vector<double> nrm(n);
    for (int k = 0; k < n; ++k) nrm[k] = std::sqrt(col2(R.data() + (size_t)k * n));
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
    std::vector<double> Vs((size_t)n * n);
    s.resize(n);
    for (int c = 0; c < n; ++c) {
        s[c] = nrm[idx[c]];
        std::copy(V.begin() + (size_t)idx[c] * n, V.begin() + (size_t)(idx[c] + 1) * n, Vs.begin() + (size_t)c * n);
    }
    V.swap(Vs);
}

struct ChebLowRank {
    int rt = 0, rs = 0;
    // U' [rt][qq] | V [qq][rs] | C_o' [49][rs][rt]: each laid out so the kernel's threads
    // (over m in cheb_expand, over j in cheb_compress, over i in cheb_m2l_lr) read
    // consecutive addresses
    std::vector<double> buf;
};

// Shared bases of the 40 M2L matrices A_o[m][n] = K[o][n][m] (target m, source n).  The
// source basis V is the leading right singular vectors of the stacked [A_o; ...]
// (Householder R, then one-sided Jacobi), truncated where the singular values fall
// below eps times the largest.  The target basis is the leading left singular vectors
// of [A_o ...]; since A_o' = A_{-o} (|x_m - x_n - 2o| = |x_n - x_m + 2o|) and the offset
// set is symmetric, [A_o ...]' is the same stack with its blocks reordered, so U = V.
// C_o = U' A_o V.  Built once per (q, eps).
static std::vector<double> cheb_dense_ops(int q);
static const ChebLowRank &cheb_lowrank(int q, double eps) {
    static std::mutex mu;
    static std::map<std::pair<int, double>, ChebLowRank> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find({q, eps});
    if (it != cache.end()) return it->second;
    const std::vector<double> K = cheb_dense_ops(q);
    const int qq = q * q;
    std::vector<int> cls;
    for (int c = 0; c < 49; ++c) {
        const int dx = c / 7 - 3, dy = c % 7 - 3;
        if (std::abs(dx) > 1 || std::abs(dy) > 1) cls.push_back(c);
    }
    const int rows = (int)cls.size() * qq;
    std::vector<double> St((size_t)rows * qq);  // column n: (class, target m) rows
    for (size_t ci = 0; ci < cls.size(); ++ci) {
        const double *Kc = K.data() + (size_t)cls[ci] * qq * qq;  // Kc[n * qq + m] = A_o[m][n]
        for (int n = 0; n < qq; ++n)
            std::copy(Kc + (size_t)n * qq, Kc + (size_t)(n + 1) * qq, St.begin() + (size_t)n * rows + ci * qq);
    }
    std::vector<double> R = householder_r(rows, qq, std::move(St));
    std::vector<double> Vc, sv;
    jacobi_right(qq, R, Vc, sv);
    int r = 0;
    while (r < qq && sv[r] > eps * sv[0]) ++r;
    r = std::max(1, std::min(r, kChebMaxRank));
    ChebLowRank lr;
    lr.rt = lr.rs = r;
    lr.buf.assign((size_t)2 * qq * r + (size_t)49 * r * r, 0.0);
    double *Ut = lr.buf.data(), *V = Ut + (size_t)qq * r, *Ct = V + (size_t)qq * r;
    for (int m = 0; m < qq; ++m)
        for (int i = 0; i < r; ++i) Ut[(size_t)i * qq + m] = V[(size_t)m * r + i] = Vc[(size_t)i * qq + m];
    const double *U = V;  // the same basis, [qq][r]
    std::vector<double> AV((size_t)qq * r);
    for (int c : cls) {
        const double *Kc = K.data() + (size_t)c * qq * qq;
        std::fill(AV.begin(), AV.end(), 0.0);  // AV = A_o V
        for (int n = 0; n < qq; ++n)
            for (int m = 0; m < qq; ++m) {
                const double k = Kc[(size_t)n * qq + m];
                for (int j = 0; j < r; ++j) AV[(size_t)m * r + j] += k * V[(size_t)n * r + j];
            }
        double *Cc = Ct + (size_t)c * r * r;  // C_o = U' AV, stored transposed: Cc[j][i]
        for (int m = 0; m < qq; ++m)
            for (int i = 0; i < r; ++i) {
                const double u = U[(size_t)m * r + i];
                for (int j = 0; j < r; ++j) Cc[(size_t)j * r + i] += u * AV[(size_t)m * r + j];
            }
    }
    return cache.emplace(std::make_pair(q, eps), std::move(lr)).first->second;
}

static long double cheb_node(int q, int m) {
    const long double pi = 3.141592653589793238462643383279502884L;
    return std::cos((2 * m + 1) * pi / (2.0L * q));
}

// The dense M2L operators K[cls][n][m] = |xb_m - xb_n - 2 o| (source node n, target node
// m, offset o of class cls in box units), input of the low-rank build only.
static std::vector<double> cheb_dense_ops(int q) {
    const int qq = q * q;
    std::vector<long double> xb(q);
    for (int m = 0; m < q; ++m) xb[m] = cheb_node(q, m);
    std::vector<double> K((size_t)49 * qq * qq, 0.0);
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy) {
            if (std::abs(dx) <= 1 && std::abs(dy) <= 1) continue;
            const int cls = (dx + 3) * 7 + (dy + 3);
            double *Kc = K.data() + (size_t)cls * qq * qq;
            for (int n = 0; n < qq; ++n)
                for (int m = 0; m < qq; ++m) {
                    const long double ex = xb[m / q] - xb[n / q] - 2.0L * dx;
                    const long double ey = xb[m % q] - xb[n % q] - 2.0L * dy;
                    Kc[(size_t)n * qq + m] = (double)std::sqrt(ex * ex + ey * ey);
                }
        }
    return K;
}

// The device tables of one order, built once per process: Tn [q][q] (T_k at the nodes) |
// A [2][q][q] (the basis at the child nodes of either half).
static const std::vector<double> &cheb_dev_tables(int q) {
    static std::mutex mu;
    static std::map<int, std::vector<double>> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(q);
    if (it != cache.end()) return it->second;
    const int qq = q * q;
    const long double pi = 3.141592653589793238462643383279502884L;
    auto S = [&](int m, long double t) {
        long double Tk0 = 1, Tk1 = t, s = 0;
        for (int k = 1; k < q; ++k) {
            long double Tm = std::cos(k * (2 * m + 1) * pi / (2.0L * q));
            s += Tm * Tk1;
            long double Tk2 = 2 * t * Tk1 - Tk0;
            Tk0 = Tk1;
            Tk1 = Tk2;
        }
        return 1.0L / q + 2.0L / q * s;
    };
    std::vector<double> buf((size_t)3 * qq, 0.0);
    for (int k = 0; k < q; ++k)
        for (int m = 0; m < q; ++m) buf[k * q + m] = (double)std::cos(k * (2 * m + 1) * pi / (2.0L * q));
    for (int sgn = 0; sgn < 2; ++sgn)
        for (int m = 0; m < q; ++m)
            for (int mp = 0; mp < q; ++mp)
                buf[qq + (size_t)sgn * qq + m * q + mp] =
                    (double)S(m, (sgn ? 0.5L : -0.5L) + 0.5L * cheb_node(q, mp));
    return cache.emplace(q, std::move(buf)).first->second;
}

void cheb_setup(Fmm &f, int q, double lr_eps, bool tensor, const std::vector<long double> &mix, cudaStream_t s) {
    PHS_REQUIRE(q >= 3 && q <= kChebMaxQ, PHS_ERR_INVALID_ARG, "Chebyshev order must be in 3..16");
    f.cheb_q = q;
    const std::vector<double> &buf = cheb_dev_tables(q);  // cheb64: Tn [q*q] | A [2][q][q]
    f.cheb64.alloc(buf.size());
    PHS_CUDA(cudaMemcpyAsync(f.cheb64.get(), buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    const ChebLowRank &lr = cheb_lowrank(q, lr_eps);
    f.cheb_rt = lr.rt;
    f.cheb_rs = lr.rs;
    PHS_REQUIRE(lr.rt <= 256 && lr.rs <= 256, PHS_ERR_INVALID_ARG, "compressed M2L rank above 256");
    f.cheb_lr.alloc(lr.buf.size());
    PHS_CUDA(cudaMemcpyAsync(f.cheb_lr.get(), lr.buf.data(), lr.buf.size() * sizeof(double), cudaMemcpyHostToDevice,
                             s));
    PHS_CUDA(cudaStreamSynchronize(s));
    f.ctc = false;
    if (tensor && cheb_tc_supported(f.nd, lr.rs, lr.rt))
        cheb_tc_setup(f, lr.buf.data() + (size_t)2 * q * q * lr.rt, mix, s);
}

void cheb_far_field(Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, cudaStream_t s, Timers *tm) {
    const int q = f.cheb_q, qq = q * q, nd = f.nd;
    const size_t sz = (size_t)t.nbox * nd * qq;
    if (f.cw64.n != sz) {
        f.cw64.alloc(sz);
        f.cl64.alloc(sz);
    }
    const double *Tn = f.cheb64.get(), *A = Tn + qq;
    TreeView tv = tree_view(t);
    if (tm) tm->begin(s);
    cheb_p2m<<<t.nleaf, CHEB_T, 0, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, nd, q, Tn,
                                        f.cw64.get());
    PHS_LAUNCH_CHECK();
    for (int l = t.depth - 1; l >= 0; --l) {
        const int b0 = t.lvl_off[l], nb = t.lvl_off[l + 1] - b0;
        if (nb > 0)
            cheb_m2m<<<nb, CHEB_T, (size_t)nd * qq * sizeof(double), s>>>(tv, b0, nd, q, A, f.mix64.get(),
                                                                          f.cw64.get());
        PHS_LAUNCH_CHECK();
    }
    if (tm) tm->end(T_UP, s);
    if (tm) tm->begin(s);
    PHS_CUDA(cudaMemsetAsync(f.cl64.get(), 0, sz * sizeof(double), s));
    if (t.depth >= 2) {
        const int b0 = t.lvl_off[2], nb = t.nbox - b0;
        const int rt = f.cheb_rt, rs = f.cheb_rs;
        if (f.cwc64.n != (size_t)t.nbox * nd * rs) f.cwc64.alloc((size_t)t.nbox * nd * rs);
        if (f.clc64.n != (size_t)t.nbox * nd * rt) f.clc64.alloc((size_t)t.nbox * nd * rt);
        const double *U = f.cheb_lr.get(), *V = U + (size_t)qq * rt, *C = V + (size_t)qq * rs;
        if (nb > 0) {
            cheb_compress<<<nb, CHEB_T, (size_t)nd * qq * sizeof(double), s>>>(b0, nd, qq, rs, V, f.cw64.get(),
                                                                               f.cwc64.get());
            PHS_LAUNCH_CHECK();
            if (f.ctc) {
                cheb_m2l_tc_pass(f, t, b0, f.cwc64.get(), f.clc64.get(), s);
            } else {
                const int thr = std::max(32, (rt + 31) / 32 * 32);
                cheb_m2l_lr<<<nb, thr, 2 * (size_t)nd * rs * sizeof(double), s>>>(
                    b0, t.v_off.get(), t.v_src.get(), t.v_cls.get(), nd, rt, rs, C, f.mix64.get(), f.cwc64.get(),
                    f.clc64.get());
                PHS_LAUNCH_CHECK();
            }
            cheb_expand<<<nb, CHEB_T, (size_t)nd * rt * sizeof(double), s>>>(tv, b0, nd, qq, rt, f.power, U,
                                                                             f.clc64.get(), f.cl64.get());
            PHS_LAUNCH_CHECK();
        }
    }
    if (tm) tm->end(T_M2L, s);
    if (tm) tm->begin(s);
    for (int l = 3; l <= t.depth; ++l) {
        const int b0 = t.lvl_off[l], nb = t.lvl_off[l + 1] - b0;
        if (nb > 0)
            cheb_l2l<<<nb, CHEB_T, (size_t)nd * qq * sizeof(double), s>>>(tv, b0, nd, q, A, f.mix64.get(),
                                                                          f.cl64.get());
        PHS_LAUNCH_CHECK();
    }
    if (tm) tm->end(T_DOWN, s);
}

void cheb_l2p_apply(Fmm &f, const Tree &t, const PointSet &ps, double *y, cudaStream_t s) {
    const int q = f.cheb_q, qq = q * q;
    cheb_l2p<<<t.nleaf, 128, (size_t)(f.nd * qq + qq) * sizeof(double), s>>>(
        tree_view(t), t.leaf_box.get(), ps.xs.get(), f.power, f.nd, q, f.cheb64.get(), f.cl64.get(), y);
    PHS_LAUNCH_CHECK();
}

// far-field part of the interpolant at normalised targets (distance kernel):
// out[i] += sum_d u_d(y_i) pot_d(y_i) from the local expansion of box_of[i] (if level >= 2)
__global__ void cheb_eval_far(TreeView tv, const double2 *tgt, const int *box_of, int64_t m, int power, int nd, int q,
                              const double *Tn, const double *L, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int b = box_of[i];
    if (b < 0 || tv.level[b] < 2) return;
    double cx, cy, h;
    box_center_h(tv, b, cx, cy, h);
    const double2 y = tgt[i];
    const double sx = fmin(1.0, fmax(-1.0, (y.x - cx) / h)), sy = fmin(1.0, fmax(-1.0, (y.y - cy) / h));
    double u[10];
    had_u(power, 0.5 * (y.x - cx) / h, 0.5 * (y.y - cy) / h, u);  // box-local factors
    const int qq = q * q;
    double acc = 0.0;
    for (int d = 0; d < nd; ++d) acc += u[d] * cheb_l2p_point(L + ((size_t)b * nd + d) * qq, q, Tn, sx, sy);
    out[i] += acc;
}

void cheb_eval_far_launch(Fmm &f, const Tree &t, const double2 *tgt, const int *box_of, int64_t m, double *out,
                          cudaStream_t s) {
    cheb_eval_far<<<blocks_for(m, 128), 128, 0, s>>>(tree_view(t), tgt, box_of, m, f.power, f.nd, f.cheb_q,
                                                      f.cheb64.get(), f.cl64.get(), out);
    PHS_LAUNCH_CHECK();
}

}  // namespace phs
