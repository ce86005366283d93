/*
 * phs_oracle.c -- plain, slow, obviously-correct CPU FP64 reference for the
 * polyharmonic-spline (PHS) interpolation path of Geoga & O'Neil,
 * "Linear-cost Polyharmonic Spline Interpolation of Arbitrary Degree".
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path, and it never calls it.
 *
 * Every routine is the plain definition written out in FP64 with no blocking,
 * fusion or reordering beyond what the definition states.  Build flags must
 * include -ffp-contract=off so that squared distances are dx*dx + dy*dy with
 * two roundings (no fused multiply-add); neighbour lists and orderings are
 * compared bit-exactly against the GPU path, which uses the same arithmetic.
 *
 * Points are row-major n x 2 arrays (x, y).  Indices are int64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* PHS radial function, Eq. (1.2): phi(r) = r^k (k odd), r^k log r (k even).
 * phi(0) = 0 for every k >= 1 (the limit of r^k log r). */
double or_phi(int k, double r)
{
    if (r == 0.0) return 0.0;
    double p = 1.0;
    for (int i = 0; i < k; ++i) p *= r;
    if (k % 2 == 0) return p * log(r);
    return p;
}

static double sqdist(const double *a, const double *b)
{
    double dx = a[0] - b[0];
    double dy = a[1] - b[1];
    return dx * dx + dy * dy;
}

/* Dense kernel matrix M_{ij} = phi(|x_i - x_j|), Eq. (1.3).  out is n x n row-major. */
void or_dense_matrix(int64_t n, const double *x, int k, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            out[i * n + j] = or_phi(k, sqrt(sqdist(x + 2 * i, x + 2 * j)));
}

/* Dense product out = M t, M as in Eq. (1.3); O(n^2), summed in index order. */
void or_dense_matvec(int64_t n, const double *x, int k, const double *t, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            s += or_phi(k, sqrt(sqdist(x + 2 * i, x + 2 * j))) * t[j];
        out[i] = s;
    }
}

/* Kernel part of the interpolant, Eq. (1.1): out_i = sum_j w_j phi(|x_j - y_i|)
 * for m target points y. */
void or_dense_eval(int64_t n, const double *x, const double *w, int k,
                   int64_t m, const double *y, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            s += w[j] * or_phi(k, sqrt(sqdist(y + 2 * i, x + 2 * j)));
        out[i] = s;
    }
}

/* The scale of that sum's rounding: out_i = sum_j |w_j phi(|x_j - y_i|)|, the sum of the
 * absolute values of its terms (the error bound of any summation order is relative to
 * it; the sums of an interpolant cancel heavily). */
void or_dense_eval_abs(int64_t n, const double *x, const double *w, int k,
                       int64_t m, const double *y, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            s += fabs(w[j] * or_phi(k, sqrt(sqdist(y + 2 * i, x + 2 * j))));
        out[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the i-th output (i = 0, 1, ...)
 * of the generator seeded with `seed`.  Counter-based: state_i = seed + (i+1)*gamma. */
uint64_t or_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t key; int64_t idx; } keyidx_t;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx_t *p = (const keyidx_t *)a, *q = (const keyidx_t *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

/* Random enumeration of the points (Sec. 3, the paper's choice): order[r] is
 * the point of rank r, ranks sorted by (splitmix64(seed, i), i). */
void or_random_order(int64_t n, uint64_t seed, int64_t *order)
{
    keyidx_t *a = (keyidx_t *)malloc(sizeof(keyidx_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].key = or_splitmix64(seed, (uint64_t)i); a[i].idx = i; }
    qsort(a, (size_t)n, sizeof(keyidx_t), cmp_keyidx);
    for (int64_t r = 0; r < n; ++r) order[r] = a[r].idx;
    free(a);
}

/* Exact maxmin enumeration, O(n^2) greedy.  First point: the one nearest to the
 * bounding-box centre ((min+max)/2 per axis); then repeatedly the unselected
 * point whose squared distance to the selected set is largest.  Ties go to the
 * smallest input index.  dmin_out (optional) receives the squared distance at
 * which each rank was selected (rank 0: +inf). */
void or_maxmin_order(int64_t n, const double *x, int64_t *order, double *dmin_out)
{
    if (n <= 0) return;
    double xmin = x[0], xmax = x[0], ymin = x[1], ymax = x[1];
    for (int64_t i = 1; i < n; ++i) {
        if (x[2 * i] < xmin) xmin = x[2 * i];
        if (x[2 * i] > xmax) xmax = x[2 * i];
        if (x[2 * i + 1] < ymin) ymin = x[2 * i + 1];
        if (x[2 * i + 1] > ymax) ymax = x[2 * i + 1];
    }
    double c[2] = {(xmin + xmax) * 0.5, (ymin + ymax) * 0.5};
    int64_t first = 0;
    double best = sqdist(x, c);
    for (int64_t i = 1; i < n; ++i) {
        double d = sqdist(x + 2 * i, c);
        if (d < best) { best = d; first = i; }
    }
    double *dmin = (double *)malloc(sizeof(double) * (size_t)n);
    char *sel = (char *)calloc((size_t)n, 1);
    order[0] = first; sel[first] = 1;
    if (dmin_out) dmin_out[0] = INFINITY;
    for (int64_t i = 0; i < n; ++i) dmin[i] = sqdist(x + 2 * i, x + 2 * first);
    for (int64_t r = 1; r < n; ++r) {
        int64_t arg = -1; double dv = -1.0;
        for (int64_t i = 0; i < n; ++i)
            if (!sel[i] && dmin[i] > dv) { dv = dmin[i]; arg = i; }
        order[r] = arg; sel[arg] = 1;
        if (dmin_out) dmin_out[r] = dv;
        for (int64_t i = 0; i < n; ++i) {
            double d = sqdist(x + 2 * i, x + 2 * arg);
            if (d < dmin[i]) dmin[i] = d;
        }
    }
    free(dmin); free(sel);
}

/* Conditioning sets sigma(j), Sec. 2.2 and Sec. 3: for the point of rank r,
 * the min(m, r) points of smaller rank nearest to it, listed by increasing
 * (squared distance, rank).  nbr is n x m, indexed by POINT (not rank), entries
 * are point indices, unused slots are -1.  Brute force. */
void or_knn_prev(int64_t n, const double *x, const int64_t *order, int m, int64_t *nbr)
{
#pragma omp parallel
    {
        double *bd = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
        int64_t *br = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < n; ++r) {
            int64_t i = order[r];
            int cnt = 0;
            for (int64_t q = 0; q < r; ++q) {
                double d = sqdist(x + 2 * i, x + 2 * order[q]);
                /* (d, q) is lexicographically after the current worst: skip */
                if (cnt == m && !(d < bd[m - 1] || (d == bd[m - 1] && q < br[m - 1]))) continue;
                int pos = cnt < m ? cnt : m - 1;
                while (pos > 0 && (d < bd[pos - 1] || (d == bd[pos - 1] && q < br[pos - 1]))) {
                    bd[pos] = bd[pos - 1]; br[pos] = br[pos - 1]; --pos;
                }
                bd[pos] = d; br[pos] = q;
                if (cnt < m) ++cnt;
            }
            for (int s = 0; s < m; ++s) nbr[i * m + s] = s < cnt ? order[br[s]] : -1;
        }
        free(bd); free(br);
    }
}

/* ------------------------------------------------------------------ */
/* Modified Bessel function K_1(x), x > 0.
 * x <= 2: the ascending series DLMF 10.31.1 with n = 1,
 *   K_1(x) = 1/x + ln(x/2) I_1(x) - (x/4) sum_k [psi(k+1)+psi(k+2)] (x^2/4)^k / (k!(k+1)!),
 *   I_1(x) = (x/2) sum_k (x^2/4)^k / (k!(k+1)!),  psi(k+1) = -gamma + H_k.
 * x > 2: the integral DLMF 10.32.9, K_1(x) = int_0^inf exp(-x cosh t) cosh t dt,
 *   by the trapezoidal rule (exponentially convergent for this analytic,
 *   doubly-exponentially decaying integrand). */
double or_bessel_k1(double x)
{
    const double euler_gamma = 0.57721566490153286060651209;
    if (x <= 2.0) {
        double q = 0.25 * x * x;
        double term = 1.0;            /* (x^2/4)^k / (k!(k+1)!) */
        double hk = 0.0;              /* H_k */
        double s_i = 0.0, s_psi = 0.0;
        for (int k = 0; k < 60; ++k) {
            if (k > 0) { term *= q / ((double)k * (double)(k + 1)); hk += 1.0 / k; }
            double psi1 = -euler_gamma + hk;             /* psi(k+1) */
            double psi2 = psi1 + 1.0 / (double)(k + 1);  /* psi(k+2) */
            s_i += term;
            s_psi += (psi1 + psi2) * term;
            if (term < 1e-22 * s_i) break;
        }
        double i1 = 0.5 * x * s_i;
        return 1.0 / x + log(0.5 * x) * i1 - 0.25 * x * s_psi;
    }
    double h = 1.0 / 64.0, s = 0.0;
    for (int j = 0; ; ++j) {
        double t = j * h;
        double ch = cosh(t);
        double f = exp(-x * ch) * ch;
        s += (j == 0 ? 0.5 : 1.0) * f;
        if (j > 0 && f < 1e-30 * s) break;
        if (j > 4000) break;
    }
    return h * s;
}

/* Modified Bessel function K_0(x), x > 0: DLMF 10.31.2 for x <= 2,
 *   K_0(x) = -(ln(x/2) + gamma) I_0(x) + sum_{k>=1} H_k (x^2/4)^k / (k!)^2,
 *   I_0(x) = sum_k (x^2/4)^k / (k!)^2,
 * and the trapezoidal rule on DLMF 10.32.9, K_0(x) = int_0^inf exp(-x cosh t) dt, for x > 2. */
double or_bessel_k0(double x)
{
    const double euler_gamma = 0.57721566490153286060651209;
    if (x <= 2.0) {
        double q = 0.25 * x * x, term = 1.0, hk = 0.0, s_i = 1.0, s_h = 0.0;
        for (int k = 1; k < 60; ++k) {
            term *= q / ((double)k * (double)k);
            hk += 1.0 / k;
            s_i += term;
            s_h += hk * term;
            if (term < 1e-22 * s_i) break;
        }
        return -(log(0.5 * x) + euler_gamma) * s_i + s_h;
    }
    double h = 1.0 / 64.0, s = 0.0;
    for (int j = 0; ; ++j) {
        double f = exp(-x * cosh(j * h));
        s += (j == 0 ? 0.5 : 1.0) * f;
        if (j > 0 && f < 1e-30 * s) break;
        if (j > 4000) break;
    }
    return h * s;
}

/* Matern covariance with unit variance, Sec. 2.2:
 *   K(r) = 2^{1-nu}/Gamma(nu) (alpha r)^nu K_nu(alpha r),  K(0) = 1.
 * Implemented for nu = 1 (alpha r K_1(alpha r)), the paper's choice, nu = 2
 * ((alpha r)^2 K_2(alpha r) / 2 with K_2 = K_0 + (2/x) K_1, DLMF 10.29.1), and
 * the half-integer cases nu = 0.5, 1.5, 2.5 where K_nu is elementary. */
double or_matern(double nu, double alpha, double r)
{
    double a = alpha * r;
    if (a == 0.0) return 1.0;
    if (nu == 0.5) return exp(-a);
    if (nu == 1.5) return (1.0 + a) * exp(-a);
    if (nu == 2.5) return (1.0 + a + a * a / 3.0) * exp(-a);
    if (nu == 1.0) return a * or_bessel_k1(a);
    if (nu == 2.0) return 0.5 * a * a * or_bessel_k0(a) + a * or_bessel_k1(a);
    return NAN;
}

/* Plain Cholesky A = L L^T in place (lower triangle of an s x s row-major
 * matrix).  Returns 0 on success, -1 if a pivot is not positive. */
static int chol_inplace(int s, double *A)
{
    for (int j = 0; j < s; ++j) {
        double d = A[j * s + j];
        for (int k = 0; k < j; ++k) d -= A[j * s + k] * A[j * s + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[j * s + j] = d;
        for (int i = j + 1; i < s; ++i) {
            double v = A[i * s + j];
            for (int k = 0; k < j; ++k) v -= A[i * s + k] * A[j * s + k];
            A[i * s + j] = v / d;
        }
    }
    return 0;
}

/* Vecchia factor, Eq. (2.19) and Fig. 1.  For the point i of rank r with
 * conditioning set sigma = nbr[i][0..s-1], s = min(m, r):
 *   lambda = K(X_sigma, X_sigma)^{-1} K(X_sigma, x_i),  c^2 = K(0) - K(x_i, X_sigma)^T lambda,
 * and column i of the sparse upper "reverse" inverse-Cholesky factor U~
 * (Sigma^{-1} ~= U~ U~^T) holds 1/c at row i and -lambda/c at rows sigma.
 * diag[i] = 1/c, offd[i*m + q] = -lambda_q / c (0 for unused slots).
 * If a local Cholesky fails, the diagonal of K_sigma,sigma is raised by
 * jitter_base * 10^t, t = 0..6, until it succeeds; if it still fails (or the
 * conditional variance is not positive) the point keeps an empty conditioning
 * set (column 1/sqrt(K(0)) e_i).  Returns the number of points that needed
 * jitter or the fallback. */
int64_t or_vecchia_factor(int64_t n, const double *x, const int64_t *order, const int64_t *nbr,
                          int m, double nu, double alpha, double jitter_base,
                          double *diag, double *offd)
{
    int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = r;
    int64_t njit = 0, fail = 0;
#pragma omp parallel reduction(+ : njit, fail)
    {
        double *A = (double *)malloc(sizeof(double) * (size_t)(m * m + 1));
        double *kv = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        double *y = (double *)malloc(sizeof(double) * (size_t)(m + 1));
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int s = (int)(rank[i] < m ? rank[i] : m);
            const int64_t *sg = nbr + i * m;
            int ok = -1;
            const double k0 = or_matern(nu, alpha, 0.0);
            for (int t = 0; t <= 7 && ok != 0; ++t) {
                double jit = t == 0 ? 0.0 : jitter_base * pow(10.0, t - 1);
                for (int a = 0; a < s; ++a)
                    for (int b = 0; b < s; ++b)
                        A[a * s + b] = or_matern(nu, alpha, sqrt(sqdist(x + 2 * sg[a], x + 2 * sg[b])))
                                       + (a == b ? jit : 0.0);
                ok = chol_inplace(s, A);
                if (ok == 0 && t > 0) ++njit;
            }
            if (ok != 0) {
                ++njit;
                diag[i] = 1.0 / sqrt(k0);
                for (int q = 0; q < m; ++q) offd[i * m + q] = 0.0;
                continue;
            }
            for (int a = 0; a < s; ++a) kv[a] = or_matern(nu, alpha, sqrt(sqdist(x + 2 * sg[a], x + 2 * i)));
            /* forward solve L y = k */
            for (int a = 0; a < s; ++a) {
                double v = kv[a];
                for (int b = 0; b < a; ++b) v -= A[a * s + b] * y[b];
                y[a] = v / A[a * s + a];
            }
            double c2 = or_matern(nu, alpha, 0.0);
            for (int a = 0; a < s; ++a) c2 -= y[a] * y[a];
            /* back solve L^T lambda = y (lambda overwrites y) */
            for (int a = s - 1; a >= 0; --a) {
                double v = y[a];
                for (int b = a + 1; b < s; ++b) v -= A[b * s + a] * y[b];
                y[a] = v / A[a * s + a];
            }
            if (!(c2 > 0.0)) {
                ++njit;
                diag[i] = 1.0 / sqrt(k0);
                for (int q = 0; q < m; ++q) offd[i * m + q] = 0.0;
                continue;
            }
            double c = sqrt(c2);
            diag[i] = 1.0 / c;
            for (int q = 0; q < m; ++q) offd[i * m + q] = q < s ? -y[q] / c : 0.0;
        }
        free(A); free(kv); free(y);
    }
    free(rank);
    return fail ? -1 : njit;
}

/* Preconditioner product z = U~ (U~^T r), Fig. 1 / Sec. 2.2, with U~ stored by
 * columns as produced by or_vecchia_factor. */
void or_vecchia_apply(int64_t n, const int64_t *nbr, int m, const double *diag,
                      const double *offd, const double *r, double *z)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        double v = diag[i] * r[i];
        for (int q = 0; q < m; ++q)
            if (nbr[i * m + q] >= 0) v += offd[i * m + q] * r[nbr[i * m + q]];
        y[i] = v;
    }
    for (int64_t i = 0; i < n; ++i) z[i] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        z[i] += diag[i] * y[i];
        for (int q = 0; q < m; ++q)
            if (nbr[i * m + q] >= 0) z[nbr[i * m + q]] += offd[i * m + q] * y[i];
    }
    free(y);
}
