// krylov.cu -- GMRES on the kernel matrix alone (the comparison of Sec. 3.1) and the
// preconditioner-range tuner (the parameter search of Sec. 2.2), on a plan.
//
// GMRES (Sec. 3.1): M c = b with M_ij = phi(|x_i - x_j|), no polynomial block, solved by
// restarted GMRES with the plan's Vecchia factor S~^{-1} = U~ U~' as a RIGHT
// preconditioner: minimise ||b - M U~ U~' y|| over the Krylov space of M U~ U~', so the
// residual GMRES minimises is the true residual of M c = b and the stopping rule
// ||b - M c|| <= max(tol ||b||, atol) (relative and absolute tolerances, Sec. 3.1) needs
// no preconditioned norm.  Arnoldi runs on the device with classical Gram-Schmidt and
// one reorthogonalisation (two passes of V'w, w -= V h); the (j + 2) x (j + 1)
// Hessenberg least-squares problem is reduced by Givens rotations on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "plan.cuh"

namespace phs {
namespace {

constexpr int KR_T = 256;
constexpr int KR_B = 592;  // 4 blocks per SM on 148 SMs
constexpr int KR_CH = 8;   // basis vectors per register chunk
constexpr int kMaxRestart = 128;

// part[b * kMaxRestart + q] = this block's share of V_q . w, q < k (V: [k][n])
__global__ void vdots_partial(const double *V, int k, int64_t n, const double *w, double *part) {
    __shared__ double sh[KR_T];
    for (int q0 = 0; q0 < k; q0 += KR_CH) {
        const int nq = min(KR_CH, k - q0);
        double acc[KR_CH];
#pragma unroll
        for (int q = 0; q < KR_CH; ++q) acc[q] = 0.0;
        for (int64_t j = (int64_t)blockIdx.x * KR_T + threadIdx.x; j < n; j += (int64_t)gridDim.x * KR_T) {
            const double wj = w[j];
#pragma unroll
            for (int q = 0; q < KR_CH; ++q)
                if (q < nq) acc[q] = fma(V[(int64_t)(q0 + q) * n + j], wj, acc[q]);
        }
        for (int q = 0; q < nq; ++q) {
            sh[threadIdx.x] = acc[q];
            __syncthreads();
            for (int o = KR_T / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) part[blockIdx.x * kMaxRestart + q0 + q] = sh[0];
            __syncthreads();
        }
    }
}
// out[q] = sum over the blocks of part[.][q], fixed order (block q)
__global__ void vdots_final(const double *part, int nblk, double *out) {
    __shared__ double sh[KR_T];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += KR_T) s += part[b * kMaxRestart + q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = KR_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}
// w += sign * sum_q h[q] V_q
__global__ void vcombine(double *w, const double *V, const double *h, int k, int64_t n, double sign) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double a = w[j];
        for (int q = 0; q < k; ++q) a = fma(sign * h[q], V[(int64_t)q * n + j], a);
        w[j] = a;
    }
}
// dst = src / sqrt(*nrm2)
__global__ void vscale_inv_sqrt(const double *src, const double *nrm2, int64_t n, double *dst) {
    const double a = 1.0 / sqrt(nrm2[0]);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = src[j] * a;
}
__global__ void vsub(const double *a, const double *b, int64_t n, double *out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = a[j] - b[j];
}
__global__ void vzero(double *a, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        a[j] = 0.0;
}
__global__ void vaxpy(double *y, const double *x, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        y[j] += x[j];
}

// out[0..k-1] = V[0..k-1]' w (device)
void vdots(const double *V, int k, int64_t n, const double *w, double *part, double *out, cudaStream_t s) {
    vdots_partial<<<KR_B, KR_T, 0, s>>>(V, k, n, w, part);
    PHS_LAUNCH_CHECK();
    vdots_final<<<k, KR_T, 0, s>>>(part, KR_B, out);
    PHS_LAUNCH_CHECK();
}

}  // namespace

// Right-preconditioned restarted GMRES in sorted order: b_s, x_s (x_s overwritten, x0 = 0).
// A cycle ends when its Givens residual estimate is <= stop (or after `restart`
// iterations); check_true restarts until the recomputed residual meets stop, otherwise
// the solve ends at the first estimate that does.  Returns the iteration count; *res =
// ||b - M x|| recomputed at the end, *restarts the number of cycles, *est the last
// estimate.
int gmres_solve(phs_plan *pl, const double *b_s, double *x_s, int restart, double stop, int maxiter, int precision,
                bool check_true, double *res, double *est, int *restarts, MvTimes *mvt, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    const int m = std::max(1, std::min(restart, kMaxRestart - 1));
    const unsigned gb = (unsigned)std::min<int64_t>(KR_B, blocks_for(n, 256));
    SBuf<double> V((size_t)(m + 1) * n, s), z(n, s), tmp(n, s), w(n, s);
    SBuf<double> part((size_t)KR_B * kMaxRestart, s), dev(3 * kMaxRestart + 8, s);
    std::vector<double> hh(3 * kMaxRestart + 8);
    double *hA = dev.get(), *hB = dev.get() + kMaxRestart, *nrm = dev.get() + 2 * kMaxRestart;
    vzero<<<gb, 256, 0, s>>>(x_s, n);
    PHS_LAUNCH_CHECK();
    // r0 = b
    PHS_CUDA(cudaMemcpyAsync(w.get(), b_s, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    vdots(w.get(), 1, n, w.get(), part.get(), nrm, s);
    double beta = std::sqrt(read_scalar(pl, nrm, s));
    int it = 0, cycles = 0;
    double g_est = beta;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    while (beta > stop && it < maxiter && (check_true || g_est > stop)) {
        ++cycles;
        vscale_inv_sqrt<<<gb, 256, 0, s>>>(w.get(), nrm, n, V.get());
        PHS_LAUNCH_CHECK();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m && it < maxiter; ++j) {
            double *Vj = V.get() + (size_t)j * n;
            vecchia_apply(pl->vec, Vj, tmp.get(), z.get(), s);
            if (mvt) mvt->begin(s);
            matvec_user_sorted(pl, z.get(), w.get(), precision, s);
            if (mvt) mvt->end(s);
            // classical Gram-Schmidt, twice
            vdots(V.get(), j + 1, n, w.get(), part.get(), hA, s);
            vcombine<<<gb, 256, 0, s>>>(w.get(), V.get(), hA, j + 1, n, -1.0);
            PHS_LAUNCH_CHECK();
            vdots(V.get(), j + 1, n, w.get(), part.get(), hB, s);
            vcombine<<<gb, 256, 0, s>>>(w.get(), V.get(), hB, j + 1, n, -1.0);
            PHS_LAUNCH_CHECK();
            vdots(w.get(), 1, n, w.get(), part.get(), nrm, s);
            PHS_CUDA(cudaMemcpyAsync(hh.data(), dev.get(), (2 * kMaxRestart + 1) * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
            PHS_CUDA(cudaStreamSynchronize(s));
            ++it;
            double *col = &H[(size_t)j * (m + 1)];
            for (int q = 0; q <= j; ++q) col[q] = hh[q] + hh[kMaxRestart + q];
            const double hn = std::sqrt(hh[2 * kMaxRestart]);
            col[j + 1] = hn;
            // previous rotations, then a new one zeroing col[j + 1]
            for (int q = 0; q < j; ++q) {
                const double a = cs[q] * col[q] + sn[q] * col[q + 1];
                col[q + 1] = -sn[q] * col[q] + cs[q] * col[q + 1];
                col[q] = a;
            }
            const double r = std::hypot(col[j], col[j + 1]);
            cs[j] = r > 0 ? col[j] / r : 1.0;
            sn[j] = r > 0 ? col[j + 1] / r : 0.0;
            col[j] = r;
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            g_est = std::fabs(g[j + 1]);
            if (g_est <= stop || !(hn > 0.0)) {
                ++j;
                break;
            }
            if (j + 1 < m + 1) {
                vscale_inv_sqrt<<<gb, 256, 0, s>>>(w.get(), nrm, n, V.get() + (size_t)(j + 1) * n);
                PHS_LAUNCH_CHECK();
            }
        }
        // y = R^{-1} g over the j columns, x += U~ U~' (V y)
        for (int q = j - 1; q >= 0; --q) {
            double a = g[q];
            for (int c = q + 1; c < j; ++c) a -= H[(size_t)c * (m + 1) + q] * y[c];
            y[q] = a / H[(size_t)q * (m + 1) + q];
        }
        PHS_CUDA(cudaMemcpyAsync(hA, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, s));
        vzero<<<gb, 256, 0, s>>>(w.get(), n);
        PHS_LAUNCH_CHECK();
        vcombine<<<gb, 256, 0, s>>>(w.get(), V.get(), hA, j, n, 1.0);
        PHS_LAUNCH_CHECK();
        vecchia_apply(pl->vec, w.get(), tmp.get(), z.get(), s);
        vaxpy<<<gb, 256, 0, s>>>(x_s, z.get(), n);
        PHS_LAUNCH_CHECK();
        // true residual r = b - M x, the next cycle's start
        if (mvt) mvt->begin(s);
        matvec_user_sorted(pl, x_s, z.get(), precision, s);
        if (mvt) mvt->end(s);
        vsub<<<gb, 256, 0, s>>>(b_s, z.get(), n, w.get());
        PHS_LAUNCH_CHECK();
        vdots(w.get(), 1, n, w.get(), part.get(), nrm, s);
        beta = std::sqrt(read_scalar(pl, nrm, s));
    }
    *res = beta;
    *est = g_est;
    *restarts = cycles;
    return it;
}

}  // namespace phs

using namespace phs;

extern "C" phs_status phs_gmres(phs_plan_t pl, const double *b_dev, double *c_dev, int restart, int check_true,
                                phs_fit_info *info, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pl && b_dev && c_dev && b_dev != c_dev, PHS_ERR_INVALID_ARG, "bad arguments");
    PHS_REQUIRE(restart >= 1 && restart < kMaxRestart, PHS_ERR_INVALID_ARG, "restart must be in 1..127");
    cudaStream_t s = (cudaStream_t)stream;
    AllocScope scope(s, &pl->dev_bytes);
    pl->last_stream = s;
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = pl->ps.n;
    const phs_options &o = pl->opt;
    const int precision = o.precision == 4 ? 4 : 0;
    double *bs = W(pl, 7), *xs = W(pl, 8);
    to_sorted(pl, b_dev, bs, 1.0, s);
    SBuf<double> part((size_t)KR_B * kMaxRestart, s), nb(1, s);
    vdots(bs, 1, n, bs, part.get(), nb.get(), s);
    const double bnrm = std::sqrt(read_scalar(pl, nb.get(), s));
    const double stop = std::max(o.tol * bnrm, o.atol);
    MvTimes mvt;
    double res = 0, est = 0;
    int cycles = 0;
    const int iters = gmres_solve(pl, bs, xs, restart, stop, o.maxiter, precision, check_true != 0, &res, &est,
                                  &cycles, &mvt, s);
    to_caller(pl, xs, c_dev, 1.0, s);
    PHS_CUDA(cudaStreamSynchronize(s));
    int n_mv = 0;
    const double ms_mv = mvt.resolve(&n_mv);
    m2l_tc_check(pl->fmm, s);
    const bool converged = check_true ? res <= stop : est <= stop;
    if (info) {
        info->iters = iters;
        info->outer_iters = cycles;
        info->converged = converged ? 1 : 0;
        info->jittered = (int)pl->vec.jittered;
        info->rel_res_recursive = bnrm > 0 ? est / bnrm : 0.0;
        info->rel_res_true = bnrm > 0 ? res / bnrm : 0.0;
        info->ms_plan = pl->ms_plan;
        info->ms_fit = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->ms_matvec_avg = n_mv ? (float)(ms_mv / n_mv) : 0.0f;
    }
    if (!converged) throw Error{PHS_ERR_NOT_CONVERGED, "GMRES did not reach the tolerance"};
    PHS_CATCH
}

// ---------------------------------------------------------------- preconditioner tuning
// Sec. 2.2 tunes two quantities, the domain the points are scaled into and the Matern
// inverse range alpha, by a gradient-free search on PCG's cost.  The Vecchia factor sees
// the points only through alpha |x_i - x_j| in the normalised frame, and the projected
// operator Q_perp' M Q_perp only scales under the map of Eq. (2.1), so scaling the domain
// by c and alpha by 1/c leaves the preconditioned iteration unchanged: the pair acts
// through its product, and a search over alpha at the plan's domain covers both.  The
// search runs PCG fits on a seeded random subsample: a grid of alpha0 * 10^(i/4),
// i = -8..4 (alpha0 the options' value, so the result is never worse on the subsample),
// then golden-section refinement between the best grid point's neighbours.  The cost of
// a trial is its PCG iteration count plus log10(final residual / tolerance) in [-1, 0],
// which orders trials of equal count by how far past the tolerance they ended; a trial
// that does not converge costs maxiter + 1.
namespace phs {
namespace {
__global__ void gather_rows2(const double *pts, const double *f, const int *idx, int64_t m, double *pts_out,
                             double *f_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j = idx[i];
    pts_out[2 * i] = pts[2 * j];
    pts_out[2 * i + 1] = pts[2 * j + 1];
    f_out[i] = f[j];
}
}  // namespace
}  // namespace phs

extern "C" phs_status phs_tune_alpha(const double *pts_dev, const double *f_dev, int64_t n, int k, int poly_degree,
                                     int fmm_order, int vecchia_m, const phs_options *opt, int64_t n_sample,
                                     double *alpha_out, int *iters_out, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && f_dev && alpha_out && n > 0, PHS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    phs_options o;
    if (opt) o = *opt;
    else phs_options_default(&o, k);
    PHS_REQUIRE(o.alpha > 0 && std::isfinite(o.alpha), PHS_ERR_INVALID_ARG, "alpha must be positive");
    const int64_t ns = (n_sample <= 0 || n_sample >= n) ? n : n_sample;
    SBuf<double> sp(2 * ns, s), sf(ns, s), w(ns, s), beta(16, s);
    if (ns < n) {
        SBuf<int> ord(n, s);
        random_order_dev(n, o.seed ^ 0x9e3779b97f4a7c15ull, ord.get(), s);
        gather_rows2<<<blocks_for(ns, 256), 256, 0, s>>>(pts_dev, f_dev, ord.get(), ns, sp.get(), sf.get());
        PHS_LAUNCH_CHECK();
    } else {
        PHS_CUDA(cudaMemcpyAsync(sp.get(), pts_dev, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PHS_CUDA(cudaMemcpyAsync(sf.get(), f_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    phs_plan_t pl = nullptr;
    phs_status st = phs_plan_create(sp.get(), ns, k, poly_degree, fmm_order, vecchia_m, &o, stream, &pl);
    if (st != PHS_OK) return st;
    struct Closer {
        phs_plan_t p;
        ~Closer() { phs_plan_destroy(p); }
    } closer{pl};
    const double a0 = o.alpha;
    auto cost = [&](double alpha, int *iters) -> double {
        plan_set_alpha(pl, alpha, s);
        phs_fit_info inf{};
        const phs_status fs = phs_fit(pl, sf.get(), w.get(), beta.get(), &inf, stream);
        if (fs != PHS_OK && fs != PHS_ERR_NOT_CONVERGED) throw Error{fs, phs_last_error()};
        *iters = inf.iters;
        if (!inf.converged) return o.maxiter + 1.0;
        const double frac = std::log10(std::max(inf.rel_res_recursive, 1e-300) / o.tol);
        return inf.iters + std::min(0.0, std::max(-1.0, frac));
    };
    double best_a = a0, best_c = 1e300;
    int best_it = 0, best_i = 0;
    for (int i = -8; i <= 4; ++i) {
        const double a = a0 * std::pow(10.0, i / 4.0);
        int it = 0;
        const double c = cost(a, &it);
        if (c < best_c || (c == best_c && std::abs(i) < std::abs(best_i))) {
            best_c = c;
            best_a = a;
            best_it = it;
            best_i = i;
        }
    }
    // golden section on log alpha between the neighbours of the best grid point
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double lo = std::log(best_a) - std::log(10.0) / 4.0, hi = std::log(best_a) + std::log(10.0) / 4.0;
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    int it1 = 0, it2 = 0;
    double c1 = cost(std::exp(x1), &it1), c2 = cost(std::exp(x2), &it2);
    for (int r = 0; r < 6; ++r) {
        if (c1 < best_c) { best_c = c1; best_a = std::exp(x1); best_it = it1; }
        if (c2 < best_c) { best_c = c2; best_a = std::exp(x2); best_it = it2; }
        if (c1 <= c2) {
            hi = x2; x2 = x1; c2 = c1; it2 = it1;
            x1 = hi - gr * (hi - lo);
            c1 = cost(std::exp(x1), &it1);
        } else {
            lo = x1; x1 = x2; c1 = c2; it1 = it2;
            x2 = lo + gr * (hi - lo);
            c2 = cost(std::exp(x2), &it2);
        }
    }
    if (c1 < best_c) { best_c = c1; best_a = std::exp(x1); best_it = it1; }
    if (c2 < best_c) { best_c = c2; best_a = std::exp(x2); best_it = it2; }
    *alpha_out = best_a;
    if (iters_out) *iters_out = best_it;
    PHS_CATCH
}
