// abi.cu -- the C ABI (include/phs.h): plans, the preconditioned CG solve of
// Eq. (2.5) on the Q_perp complement, evaluation, and stand-alone building blocks.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "plan.cuh"

namespace phs {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
const char *last_error() { return g_err.c_str(); }
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------- timers
static thread_local std::vector<cudaEvent_t> g_pool;
void ev_put(cudaEvent_t e) { g_pool.push_back(e); }
cudaEvent_t ev_get() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    PHS_CUDA(cudaEventCreate(&e));
    return e;
}

static std::mutex g_pin_mu;
static std::vector<double *> g_pin_free;
double *pinned_block() {
    std::lock_guard<std::mutex> g(g_pin_mu);
    if (g_pin_free.empty()) {
        double *chunk = nullptr;
        PHS_CUDA(cudaMallocHost((void **)&chunk, 64 * 64 * sizeof(double)));
        for (int i = 63; i >= 0; --i) g_pin_free.push_back(chunk + 64 * i);
    }
    double *b = g_pin_free.back();
    g_pin_free.pop_back();
    return b;
}
void pinned_release(double *b) {
    std::lock_guard<std::mutex> g(g_pin_mu);
    g_pin_free.push_back(b);
}

}  // namespace phs

phs_plan::~phs_plan() {
    if (hscal) phs::pinned_release(hscal);
}

namespace phs {

void Timers::begin(cudaStream_t s) {
    if (!enabled) return;
    cudaEvent_t a = ev_get();
    cudaEventRecord(a, s);
    stack.push_back(a);
}
void Timers::end(int phase, cudaStream_t s) {
    if (!enabled || stack.empty()) return;
    cudaEvent_t a = stack.back();
    stack.pop_back();
    cudaEvent_t b = ev_get();
    cudaEventRecord(b, s);
    pending.push_back(EvRec{a, b, phase});
    if (pending.size() > 8192) resolve();
}
void Timers::resolve() {
    for (auto &p : pending) {
        cudaEventSynchronize(p.b);
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        this->ms[p.phase] += ms;
        calls[p.phase] += 1;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    pending.clear();
}
Timers::~Timers() {
    for (auto &p : pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
}

namespace {

constexpr int RED_T = 256;
constexpr int RED_B = 592;  // 4 blocks per SM on 148 SMs
constexpr int MAXS = 10;

// partial dot products: out[b*cnt + i] = sum over this block's stride of a_i . b_i
struct DotSet {
    const double *a[12];
    const double *b[12];
    int cnt;
};
__global__ void dots_partial(DotSet ds, int64_t n, double *part) {
    double acc[12];
    for (int i = 0; i < ds.cnt; ++i) acc[i] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * RED_T + threadIdx.x; j < n; j += (int64_t)gridDim.x * RED_T)
        for (int i = 0; i < ds.cnt; ++i) acc[i] += ds.a[i][j] * ds.b[i][j];
    __shared__ double sh[RED_T];
    for (int i = 0; i < ds.cnt; ++i) {
        sh[threadIdx.x] = acc[i];
        __syncthreads();
        for (int o = RED_T / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 12 + i] = sh[0];
        __syncthreads();
    }
}
// fixed-order final sum of the partials: out[i] = sum_b part[b][i]
// out[i] = sum over the nblk block partials of value i; block i, RED_T threads: thread t
// sums partials t, t + RED_T, ... and a fixed shared-memory tree adds the threads, so the
// order is the same on every call (one dependent chain over all partials took ~50 us)
__global__ void dots_final(const double *part, int nblk, double *out) {
    const int i = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += RED_T) s += part[b * 12 + i];
    __shared__ double sh[RED_T];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
}

// monomials 1, x, y, x^2, xy, y^2, ... (graded lexicographic), Eq. (1.3)
__device__ __forceinline__ void monomials(int deg, double x, double y, double *v) {
    int s = 0;
    for (int d = 0; d <= deg; ++d)
        for (int b = 0; b <= d; ++b) {
            const int a = d - b;
            double t = 1.0;
            for (int i = 0; i < a; ++i) t *= x;
            for (int i = 0; i < b; ++i) t *= y;
            v[s++] = t;
        }
}
__global__ void build_B(const double2 *xs, int64_t n, int deg, int S, double *B) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double v[MAXS];
    monomials(deg, xs[j].x, xs[j].y, v);
    for (int s = 0; s < S; ++s) B[(int64_t)s * n + j] = v[s];
}
// Gram partials G_ab = sum_j B_a B_b (upper triangle, packed)
__global__ void gram_partial(const double *B, int64_t n, int S, double *part) {
    double acc[MAXS * (MAXS + 1) / 2];
    const int np = S * (S + 1) / 2;
    for (int i = 0; i < np; ++i) acc[i] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * RED_T + threadIdx.x; j < n; j += (int64_t)gridDim.x * RED_T) {
        double v[MAXS];
        for (int s = 0; s < S; ++s) v[s] = B[(int64_t)s * n + j];
        int t = 0;
        for (int a = 0; a < S; ++a)
            for (int b = a; b < S; ++b) acc[t++] += v[a] * v[b];
    }
    __shared__ double sh[RED_T];
    for (int i = 0; i < np; ++i) {
        sh[threadIdx.x] = acc[i];
        __syncthreads();
        for (int o = RED_T / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 64 + i] = sh[0];
        __syncthreads();
    }
}
// one thread: G = R'R (Cholesky, R upper), status[0] = 0 on success
__global__ void gram_chol(const double *part, int nblk, int S, double *Rout, int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double G[MAXS][MAXS];
    int t = 0;
    for (int a = 0; a < S; ++a)
        for (int b = a; b < S; ++b) {
            double s = 0.0;
            for (int k = 0; k < nblk; ++k) s += part[k * 64 + t];
            G[a][b] = G[b][a] = s;
            ++t;
        }
    double Rm[MAXS][MAXS] = {};
    for (int j = 0; j < S; ++j) {
        double d = G[j][j];
        for (int k = 0; k < j; ++k) d -= Rm[k][j] * Rm[k][j];
        if (!(d > 0.0)) { status[0] = 1; return; }
        Rm[j][j] = sqrt(d);
        for (int i = j + 1; i < S; ++i) {
            double v = G[j][i];
            for (int k = 0; k < j; ++k) v -= Rm[k][j] * Rm[k][i];
            Rm[j][i] = v / Rm[j][j];
        }
    }
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) Rout[a * S + b] = Rm[a][b];
    status[0] = 0;
}
// rows q = b R^{-1} (in place on B, column-major [S][n])
__global__ void apply_rinv(double *B, int64_t n, int S, const double *Rm) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double q[MAXS];
    for (int c = 0; c < S; ++c) {
        double v = B[(int64_t)c * n + j];
        for (int i = 0; i < c; ++i) v -= q[i] * Rm[i * S + c];
        q[c] = v / Rm[c * S + c];
    }
    for (int c = 0; c < S; ++c) B[(int64_t)c * n + j] = q[c];
}
// R = R2 R1 (both upper triangular)
__global__ void mul_upper(const double *R2, const double *R1, int S, double *Rout) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            double s = 0.0;
            for (int k = 0; k < S; ++k) s += R2[a * S + k] * R1[k * S + b];
            Rout[a * S + b] = s;
        }
}
// Q-coefficient partials: part[b][s] = sum Q_s . v
__global__ void qt_partial(const double *Q, int S, int64_t n, const double *v, double *part) {
    double acc[MAXS];
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * RED_T + threadIdx.x; j < n; j += (int64_t)gridDim.x * RED_T) {
        const double vj = v[j];
        for (int s = 0; s < S; ++s) acc[s] += Q[(int64_t)s * n + j] * vj;
    }
    __shared__ double sh[RED_T];
    for (int s = 0; s < S; ++s) {
        sh[threadIdx.x] = acc[s];
        __syncthreads();
        for (int o = RED_T / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 12 + s] = sh[0];
        __syncthreads();
    }
}
// out = sign * (v - Q c); optional partial of dot(other, out)
__global__ void proj_apply(const double *Q, int S, int64_t n, const double *c, const double *v, double sign,
                           double *out, const double *other, double *part) {
    double acc = 0.0;
    double cc[MAXS];
    for (int s = 0; s < S; ++s) cc[s] = c[s];
    for (int64_t j = (int64_t)blockIdx.x * RED_T + threadIdx.x; j < n; j += (int64_t)gridDim.x * RED_T) {
        double x = v[j];
        for (int s = 0; s < S; ++s) x -= Q[(int64_t)s * n + j] * cc[s];
        x *= sign;
        out[j] = x;
        if (other) acc += other[j] * x;
    }
    if (!part) return;
    __shared__ double sh[RED_T];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * 12] = sh[0];
}
__global__ void gather_vec(const double *src, const int *idx, int64_t n, double *dst) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = src[idx[j]];
}
__global__ void gather_scaled(const double *src, const int *idx, int64_t n, double scale, double *dst) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = src[idx[j]] * scale;
}
__global__ void scatter_scaled(const double *src, const int *idx, int64_t n, double scale, double *dst) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[idx[j]] = src[j] * scale;
}
__global__ void axpy_k(double *y, const double *x, int64_t n, double a) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) y[j] += a * x[j];
}
__global__ void scale_k(double *y, int64_t n, double a) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) y[j] *= a;
}
__global__ void zero_k(double *y, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) y[j] = 0.0;
}
// flag[0] = 1 if a and b differ in any bit (flag zeroed by the caller)
__global__ void differ_k(const double *a, const double *b, int64_t n, int *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool d = i < n && __double_as_longlong(a[i]) != __double_as_longlong(b[i]);
    if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) *flag = 1;
}
__global__ void sub_k(double *out, const double *a, const double *b, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = a[j] - b[j];
}
// R beta = c  (upper triangular, one thread)
__global__ void tri_solve(const double *Rm, int S, const double *c, double *beta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double b[MAXS];
    for (int i = S - 1; i >= 0; --i) {
        double v = c[i];
        for (int j = i + 1; j < S; ++j) v -= Rm[i * S + j] * b[j];
        b[i] = v / Rm[i * S + i];
    }
    for (int i = 0; i < S; ++i) beta[i] = b[i];
}
// normalise targets and add the polynomial part: out += sum_s beta_s P_s(y')
__global__ void norm_targets(const double *tgt, int64_t m, double cx, double cy, double rho, double2 *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    out[i] = make_double2(__dmul_rn(__dsub_rn(tgt[2 * i], cx), rho), __dmul_rn(__dsub_rn(tgt[2 * i + 1], cy), rho));
}
__global__ void add_poly(const double2 *y, int64_t m, int deg, int S, const double *beta, double *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double v[MAXS];
    monomials(deg, y[i].x, y[i].y, v);
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += beta[q] * v[q];
    out[i] += s;
}
// low-rank correction of the frame change, Eq. (2.1): partials of v_l . t and y -= log(rho) * u . c
__global__ void had_dots(const double2 *xs, const double *t, int64_t n, int power, double *part) {
    const int nd = power == 2 ? 4 : 10;
    double acc[10] = {};
    for (int64_t j = (int64_t)blockIdx.x * RED_T + threadIdx.x; j < n; j += (int64_t)gridDim.x * RED_T) {
        const double x = xs[j].x, y = xs[j].y, a = x * x + y * y, tj = t[j];
        double v[10];
        if (power == 2) { v[0] = 1; v[1] = a; v[2] = x; v[3] = y; }
        else { v[0] = 1; v[1] = a * a; v[2] = a; v[3] = x; v[4] = y; v[5] = a * x; v[6] = a * y; v[7] = x * x; v[8] = x * y; v[9] = y * y; }
        for (int d = 0; d < nd; ++d) acc[d] += v[d] * tj;
    }
    __shared__ double sh[RED_T];
    for (int d = 0; d < nd; ++d) {
        sh[threadIdx.x] = acc[d];
        __syncthreads();
        for (int o = RED_T / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 12 + d] = sh[0];
        __syncthreads();
    }
}
__global__ void had_correct(const double2 *xs, int64_t n, int power, const double *c, double lr, double *y) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double x = xs[j].x, yy = xs[j].y, a = x * x + yy * yy;
    double u[10];
    int nd;
    if (power == 2) { nd = 4; u[0] = a; u[1] = 1; u[2] = -2 * x; u[3] = -2 * yy; }
    else { nd = 10; u[0] = a * a; u[1] = 1; u[2] = 2 * a; u[3] = -4 * a * x; u[4] = -4 * a * yy; u[5] = -4 * x; u[6] = -4 * yy; u[7] = 4 * x * x; u[8] = 8 * x * yy; u[9] = 4 * yy * yy; }
    double s = 0.0;
    for (int d = 0; d < nd; ++d) s += u[d] * c[d];
    y[j] -= lr * s;
}
__global__ void to_i64(const int *src, int64_t n, int64_t *dst) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = src[j];
}
__global__ void from_i64(const int64_t *src, int64_t n, int *dst) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = (int)src[j];
}
__global__ void ell_to_rows_i64(const int *ell, int64_t n, int m, int64_t *rows) {
    // rows[i*m + q] = ell[q*n + i]
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const int64_t i = t / m, q = t - i * m;
    rows[t] = ell[q * n + i];
}
__global__ void rows_to_ell_i32(const int64_t *rows, int64_t n, int m, int *ell) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const int64_t i = t / m, q = t - i * m;
    ell[q * n + i] = (int)rows[t];
}
__global__ void ell_to_rows_d(const double *ell, int64_t n, int m, int slot0, double *rows) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const int64_t i = t / m, q = t - i * m;
    rows[t] = ell[(q + slot0) * n + i];
}
__global__ void pts_to_d2(const double *p, int64_t n, double2 *out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = make_double2(p[2 * j], p[2 * j + 1]);
}

// ---------------------------------------------------------------- PCG steps, one or many plans
// The PCG vector operations (projection of the matvec, CG update, preconditioner
// projection, p update) are written once as bodies parameterised by the block's
// coordinates and applied to a table of plans: blockIdx.y selects the plan and
// blockIdx.x / gridDim.x play the roles they have in a one-plan launch (RED_B blocks of
// RED_T threads per plan).  The single-plan solve uses a table of one, the serving
// engine a table of the active jobs, so a job's arithmetic -- and its result -- does
// not depend on which other jobs share the launch.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = RED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}
// coefficients B' v, this block's share: part[bx * 12 + c]
__device__ void b_coef_body(const double *B, int S, int64_t n, const double *v, double *part, int bx, int gx) {
    __shared__ double sh[RED_T];
    double acc[MAXS];
    for (int c = 0; c < S; ++c) acc[c] = 0.0;
    for (int64_t j = (int64_t)bx * RED_T + threadIdx.x; j < n; j += (int64_t)gx * RED_T) {
        const double vj = v[j];
        for (int c = 0; c < S; ++c) acc[c] = fma(B[(int64_t)c * n + j], vj, acc[c]);
    }
    for (int c = 0; c < S; ++c) {
        const double t = block_sum(acc[c], sh);
        if (threadIdx.x == 0) part[bx * 12 + c] = t;
    }
}
// out = sum of the RED_B partials of value i, fixed order
__device__ void b_final_body(const double *part, int i, double *out) {
    __shared__ double sh[RED_T];
    double sacc = 0.0;
    for (int b = threadIdx.x; b < RED_B; b += RED_T) sacc += part[b * 12 + i];
    const double t = block_sum(sacc, sh);
    if (threadIdx.x == 0) out[0] = t;
}
// out = sign (v - B c); if other, this block's share of other . out in part[bx * 12]
__device__ void b_proj_body(const double *B, int S, int64_t n, const double *c, const double *v, double sign,
                            double *out, const double *other, double *part, int bx, int gx) {
    __shared__ double sh[RED_T];
    double cc[MAXS];
    for (int q = 0; q < S; ++q) cc[q] = c[q];
    double acc = 0.0;
    for (int64_t j = (int64_t)bx * RED_T + threadIdx.x; j < n; j += (int64_t)gx * RED_T) {
        double xv = v[j];
        for (int q = 0; q < S; ++q) xv = fma(-B[(int64_t)q * n + j], cc[q], xv);
        xv *= sign;
        out[j] = xv;
        if (other) acc = fma(other[j], xv, acc);
    }
    if (!other) return;
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[bx * 12] = t;
}

template <int N>
__global__ void bk_coef(BTable<N> t, int stage) {
    // stage 0: Q' y (matvec projection); 1: the preconditioner's projection coefficients
    // (plain: Q' t2; low-rank: G' r)
    const BJob &j = t.j[blockIdx.y];
    const bool lr = stage == 1 && j.lowrank;
    const double *B = lr ? j.G : j.Q;
    const double *v = stage == 0 ? j.W + 4 * j.n : (lr ? j.W : j.W + 6 * j.n);
    b_coef_body(B, j.S, j.n, v, j.part, blockIdx.x, gridDim.x);
}
template <int N>
__global__ void bk_final(BTable<N> t, int cnt, int out_off) {
    // value i = blockIdx.x; cnt < 0: the plan's S values
    const BJob &j = t.j[blockIdx.y];
    const int nv = cnt < 0 ? j.S : cnt;
    if ((int)blockIdx.x >= nv) return;
    b_final_body(j.part, blockIdx.x, j.scal + out_off + blockIdx.x);
}
template <int N>
__global__ void bk_proj(BTable<N> t, int stage) {
    // stage 0: q = sign P y and partial p . q; 1: z = t2 - B c (B = Q or G)
    const BJob &j = t.j[blockIdx.y];
    const int64_t n = j.n;
    if (stage == 0)
        b_proj_body(j.Q, j.S, n, j.scal + 16, j.W + 4 * n, j.sign, j.W + 3 * n, j.W + 2 * n, j.part, blockIdx.x,
                    gridDim.x);
    else
        b_proj_body(j.lowrank ? j.G : j.Q, j.S, n, j.scal + 16, j.W + 6 * n, 1.0, j.W + n, nullptr, nullptr,
                    blockIdx.x, gridDim.x);
}
// x += alpha p, r -= alpha q, partial r . r; alpha = rz / pq
template <int N>
__global__ void bk_cg_update(BTable<N> t) {
    __shared__ double sh[RED_T];
    const BJob &j = t.j[blockIdx.y];
    const int64_t n = j.n;
    double *r = j.W;
    const double *p = j.W + 2 * n, *q = j.W + 3 * n;
    const double alpha = j.scal[0] / j.scal[1];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RED_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_T) {
        j.x[i] = fma(alpha, p[i], j.x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double tt = block_sum(acc, sh);
    if (threadIdx.x == 0) j.part[blockIdx.x * 12] = tt;
}
// partials of W[a] . W[b] into part[bx * 12 + slot]
template <int N>
__global__ void bk_dot(BTable<N> t, int a, int b, int slot) {
    __shared__ double sh[RED_T];
    const BJob &j = t.j[blockIdx.y];
    const int64_t n = j.n;
    const double *u = j.W + a * n, *v = j.W + b * n;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RED_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_T)
        acc = fma(u[i], v[i], acc);
    const double tt = block_sum(acc, sh);
    if (threadIdx.x == 0) j.part[blockIdx.x * 12 + slot] = tt;
}
// p = z + (rz_new / rz) p (rz = rz_new follows in a separate launch, bk_copy)
template <int N>
__global__ void bk_p_update(BTable<N> t) {
    const BJob &j = t.j[blockIdx.y];
    const int64_t n = j.n;
    double *p = j.W + 2 * n;
    const double *z = j.W + n;
    const double beta = j.scal[3] / j.scal[0];
    for (int64_t i = (int64_t)blockIdx.x * RED_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_T)
        p[i] = fma(beta, p[i], z[i]);
}
template <int N>
__global__ void bk_copy(BTable<N> t, int from, int to) {
    const BJob &j = t.j[blockIdx.x];
    if (threadIdx.x == 0) j.scal[to] = j.scal[from];
}
// out[k] = scal_k[off] for the table's plans
template <int N>
__global__ void bk_gather(BTable<N> t, int off, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < t.nj) out[k] = t.j[k].scal[off];
}
// r = rhs, x = 0 (the start of a solve); p = z after the first preconditioner application
template <int N>
__global__ void bk_start(BTable<N> t) {
    const BJob &j = t.j[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * RED_T + threadIdx.x; i < j.n; i += (int64_t)gridDim.x * RED_T) {
        j.x[i] = 0.0;
        j.W[i] = j.rhs[i];
    }
}
template <int N>
__global__ void bk_p_from_z(BTable<N> t) {
    const BJob &j = t.j[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * RED_T + threadIdx.x; i < j.n; i += (int64_t)gridDim.x * RED_T)
        j.W[2 * j.n + i] = j.W[j.n + i];
}

// uniform points on [0,1)^2 for the leaf-capacity tuner: coordinates from SplitMix64 of
// (seed, 2i) and (seed, 2i + 1), 53 bits each
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void tune_points(int64_t n, uint64_t seed, double *pts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n) return;
    const uint64_t z = mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    pts[i] = (double)(z >> 11) * 0x1.0p-53;
}

}  // namespace

// ---------------------------------------------------------------- plan helpers
double *W(phs_plan *pl, int i) { return pl->work.get() + (size_t)i * pl->ps.n; }

void dots(phs_plan *pl, std::initializer_list<std::pair<const double *, const double *>> prs, double *out,
                 cudaStream_t s) {
    DotSet ds;
    ds.cnt = 0;
    for (auto &pr : prs) {
        ds.a[ds.cnt] = pr.first;
        ds.b[ds.cnt] = pr.second;
        ++ds.cnt;
    }
    dots_partial<<<RED_B, RED_T, 0, s>>>(ds, pl->ps.n, pl->part.get());
    PHS_LAUNCH_CHECK();
    dots_final<<<ds.cnt, RED_T, 0, s>>>(pl->part.get(), RED_B, out);
    PHS_LAUNCH_CHECK();
}

// out = sign * P v  (P = I - Q Q'); if other != null, dot(other, out) -> *dot_out
void project(phs_plan *pl, const double *v, double sign, double *out, const double *other, double *dot_out,
                    cudaStream_t s) {
    const int64_t n = pl->ps.n;
    double *coef = pl->scal.get() + 16;
    qt_partial<<<RED_B, RED_T, 0, s>>>(pl->Q.get(), pl->S, n, v, pl->part.get());
    PHS_LAUNCH_CHECK();
    dots_final<<<pl->S, RED_T, 0, s>>>(pl->part.get(), RED_B, coef);
    PHS_LAUNCH_CHECK();
    proj_apply<<<RED_B, RED_T, 0, s>>>(pl->Q.get(), pl->S, n, coef, v, sign, out, other,
                                        other ? pl->part.get() + 8 * 0 : nullptr);
    PHS_LAUNCH_CHECK();
    if (other) {
        dots_final<<<1, RED_T, 0, s>>>(pl->part.get(), RED_B, dot_out);
        PHS_LAUNCH_CHECK();
    }
}

void matvec_norm(phs_plan *pl, const double *t, double *y, int precision, cudaStream_t s) {
    fmm_apply(pl->fmm, pl->tree, pl->ps, t, y, precision, s, &pl->tm);
}

// The expansion buffers now hold the FP64 far field of the caller-order coefficients w
// (scaled and sorted as phs_eval does); keep a copy of w to recognise it.
void remember_far_field(phs_plan *pl, const double *w_dev, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    if (pl->fmm.far_w.n != (size_t)n) pl->fmm.far_w.alloc(n);
    PHS_CUDA(cudaMemcpyAsync(pl->fmm.far_w.get(), w_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    pl->fmm.far_valid = true;
}
// whether the expansion buffers hold the FP64 far field of w (bitwise the same w)
static bool far_field_of(phs_plan *pl, const double *w_dev, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    if (!pl->fmm.far_valid || pl->fmm.far_w.n != (size_t)n) return false;
    int *flag = reinterpret_cast<int *>(pl->scal.get() + 63);
    PHS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    differ_k<<<blocks_for(n, 256), 256, 0, s>>>(w_dev, pl->fmm.far_w.get(), n, flag);
    PHS_LAUNCH_CHECK();
    int h = 1;
    PHS_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    return h == 0;
}

double read_scalar(phs_plan *pl, const double *dev, cudaStream_t s) {
    PHS_CUDA(cudaMemcpyAsync(pl->hscal, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    return pl->hscal[0];
}

// y = M t with M the kernel matrix of the CALLER's points (Eq. 1.3), vectors in sorted
// order: M' of the normalised points gives rho^k M + log(rho) [r'^k] for even k (Eq. 2.1
// generalised), so M t = rho^-k (M' t - log(rho) U(V' t)) with the Hadamard factors of
// [r'^k]; for odd k the log term is absent.
void matvec_user_sorted(phs_plan *pl, const double *ts, double *y, int precision, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    matvec_norm(pl, ts, y, precision, s);
    const double rho = pl->ps.frame.rho;
    if (pl->k % 2 == 0) {
        const int power = pl->k;
        had_dots<<<RED_B, RED_T, 0, s>>>(pl->ps.xs.get(), ts, n, power, pl->part.get());
        PHS_LAUNCH_CHECK();
        dots_final<<<power == 2 ? 4 : 10, RED_T, 0, s>>>(pl->part.get(), RED_B, pl->scal.get() + 32);
        PHS_LAUNCH_CHECK();
        had_correct<<<blocks_for(n, 256), 256, 0, s>>>(pl->ps.xs.get(), n, power, pl->scal.get() + 32, std::log(rho), y);
        PHS_LAUNCH_CHECK();
    }
    scale_k<<<blocks_for(n, 256), 256, 0, s>>>(y, n, std::pow(rho, -(double)pl->k));
    PHS_LAUNCH_CHECK();
}
// dst[p] = scale * src[perm[p]] (caller order -> sorted order)
void to_sorted(phs_plan *pl, const double *src, double *dst, double scale, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    gather_scaled<<<blocks_for(n, 256), 256, 0, s>>>(src, pl->ps.perm.get(), n, scale, dst);
    PHS_LAUNCH_CHECK();
}
// dst[perm[p]] = scale * src[p] (sorted order -> caller order)
void to_caller(phs_plan *pl, const double *src, double *dst, double scale, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    scatter_scaled<<<blocks_for(n, 256), 256, 0, s>>>(src, pl->ps.perm.get(), n, scale, dst);
    PHS_LAUNCH_CHECK();
}

// Preconditioner of the projected system, r in range(P):
//   plain:    z = P S~^{-1} r                       (S~^{-1} = U~ U~')
//   low-rank: z = S~^{-1} r - G (G' r)              (the inverse of Q_perp' S~ Q_perp on range(P))
// With G = S~^{-1} Q Rc^{-1} and Rc'Rc = Q' S~^{-1} Q, G G' = S~^{-1} Q (Q' S~^{-1} Q)^{-1} Q' S~^{-1},
// the Schur complement term of block elimination on [S~ B; B' 0], and Q'z = 0 by construction.
// Both forms cost one reduction over S basis vectors and one update pass after the factor apply.
void precond(phs_plan *pl, const double *r, double *z, double *tmp, double *tmp2, cudaStream_t s) {
    pl->tm.begin(s);
    vecchia_apply(pl->vec, r, tmp, tmp2, s);
    pl->tm.end(T_PRECOND, s);
    if (!pl->lowrank) {
        project(pl, tmp2, 1.0, z, nullptr, nullptr, s);
        return;
    }
    const int64_t n = pl->ps.n;
    double *coef = pl->scal.get() + 16;
    qt_partial<<<RED_B, RED_T, 0, s>>>(pl->G.get(), pl->S, n, r, pl->part.get());
    PHS_LAUNCH_CHECK();
    dots_final<<<pl->S, RED_T, 0, s>>>(pl->part.get(), RED_B, coef);
    PHS_LAUNCH_CHECK();
    proj_apply<<<RED_B, RED_T, 0, s>>>(pl->G.get(), pl->S, n, coef, tmp2, 1.0, z, nullptr, nullptr);
    PHS_LAUNCH_CHECK();
}

// G = U~ (U~' Q) Rc^{-1} with Rc the Cholesky factor of C = (U~' Q)'(U~' Q) = Q' S~^{-1} Q
// (symmetric by construction).  Work vectors 0..S-1 hold U~' Q.
void build_lowrank(phs_plan *pl, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    const int S = pl->S;
    PHS_REQUIRE(S <= MAXS, PHS_ERR_INVALID_ARG, "too many polynomial terms for the low-rank term");
    pl->G.alloc((size_t)S * n);
    double *Y = W(pl, 0);
    for (int c = 0; c < S; ++c) vecchia_apply_ut(pl->vec, pl->Q.get() + (size_t)c * n, Y + (size_t)c * n, s);
    SBuf<double> Rc((size_t)S * S, s);
    SBuf<int> st(1, s);
    gram_partial<<<RED_B, RED_T, 0, s>>>(Y, n, S, pl->part.get());
    PHS_LAUNCH_CHECK();
    gram_chol<<<1, 1, 0, s>>>(pl->part.get(), RED_B, S, Rc.get(), st.get());
    PHS_LAUNCH_CHECK();
    for (int c = 0; c < S; ++c) vecchia_apply_u(pl->vec, Y + (size_t)c * n, pl->G.get() + (size_t)c * n, s);
    apply_rinv<<<blocks_for(n, 256), 256, 0, s>>>(pl->G.get(), n, S, Rc.get());
    PHS_LAUNCH_CHECK();
    int hs = 0;
    PHS_CUDA(cudaMemcpyAsync(&hs, st.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_REQUIRE(hs == 0, PHS_ERR_CHOLESKY, "Q' S~^{-1} Q is not positive definite");
    pl->lowrank = true;
}

// Rebuild the plan's preconditioner for a new Matern inverse range (the tuner's step):
// enumeration, conditioning sets and local factors (Sec. 2.2), and the low-rank term if
// the plan uses it.  The tree, FMM and QR do not depend on alpha.
void plan_set_alpha(phs_plan *pl, double alpha, cudaStream_t s) {
    PHS_REQUIRE(alpha > 0 && std::isfinite(alpha), PHS_ERR_INVALID_ARG, "alpha must be positive");
    pl->opt.alpha = alpha;
    vecchia_build(pl->vec, pl->ps, pl->m, pl->opt.ordering, pl->opt.seed, pl->opt.nu, alpha, s,
                  pl->opt.precision == 4);
    pl->lowrank = false;
    if (pl->opt.precond_lowrank) build_lowrank(pl, s);
    PHS_CUDA(cudaStreamSynchronize(s));
}

// PCG on sign * P M' P x = rhs (rhs in range(P)), x0 = 0.  Returns iterations; *relres = ||r||/||rhs||.
// Work vectors used: 0..6.
double MvTimes::resolve(int *count) {
    double tot = 0;
    for (auto &p : ev) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) tot += ms;
        ev_put(p.first);
        ev_put(p.second);
    }
    *count = (int)ev.size();
    ev.clear();
    return tot;
}
MvTimes::~MvTimes() {
    for (auto &p : ev) {
        ev_put(p.first);
        ev_put(p.second);
    }
}

template <int N>
static void steps_matvec_update(const BTable<N> &t, cudaStream_t s) {
    const dim3 g(RED_B, t.nj);
    bk_coef<N><<<g, RED_T, 0, s>>>(t, 0);
    PHS_LAUNCH_CHECK();
    bk_final<N><<<dim3(MAXS, t.nj), RED_T, 0, s>>>(t, -1, 16);
    PHS_LAUNCH_CHECK();
    bk_proj<N><<<g, RED_T, 0, s>>>(t, 0);
    PHS_LAUNCH_CHECK();
    bk_final<N><<<dim3(1, t.nj), RED_T, 0, s>>>(t, 1, 1);
    PHS_LAUNCH_CHECK();
    bk_cg_update<N><<<g, RED_T, 0, s>>>(t);
    PHS_LAUNCH_CHECK();
    bk_final<N><<<dim3(1, t.nj), RED_T, 0, s>>>(t, 1, 2);
    PHS_LAUNCH_CHECK();
}
template <int N>
static void steps_zproj(const BTable<N> &t, cudaStream_t s) {
    const dim3 g(RED_B, t.nj);
    bk_coef<N><<<g, RED_T, 0, s>>>(t, 1);
    PHS_LAUNCH_CHECK();
    bk_final<N><<<dim3(MAXS, t.nj), RED_T, 0, s>>>(t, -1, 16);
    PHS_LAUNCH_CHECK();
    bk_proj<N><<<g, RED_T, 0, s>>>(t, 1);
    PHS_LAUNCH_CHECK();
}
template <int N>
static void steps_pupdate(const BTable<N> &t, cudaStream_t s) {
    const dim3 g(RED_B, t.nj);
    bk_dot<N><<<g, RED_T, 0, s>>>(t, 0, 1, 0);
    PHS_LAUNCH_CHECK();
    bk_final<N><<<dim3(1, t.nj), RED_T, 0, s>>>(t, 1, 3);
    PHS_LAUNCH_CHECK();
    bk_p_update<N><<<g, RED_T, 0, s>>>(t);
    PHS_LAUNCH_CHECK();
    bk_copy<N><<<t.nj, 32, 0, s>>>(t, 3, 0);
    PHS_LAUNCH_CHECK();
}
template <int N>
static void steps_start(const BTable<N> &t, cudaStream_t s) {
    // after z = P S~^-1 r: p = z, rz and rr into scal 4 and 5, rz into scal 0
    const dim3 g(RED_B, t.nj);
    bk_p_from_z<N><<<g, RED_T, 0, s>>>(t);
    PHS_LAUNCH_CHECK();
    bk_dot<N><<<g, RED_T, 0, s>>>(t, 0, 1, 0);
    PHS_LAUNCH_CHECK();
    bk_dot<N><<<g, RED_T, 0, s>>>(t, 0, 0, 1);
    PHS_LAUNCH_CHECK();
    bk_final<N><<<dim3(2, t.nj), RED_T, 0, s>>>(t, 2, 4);
    PHS_LAUNCH_CHECK();
    bk_copy<N><<<t.nj, 32, 0, s>>>(t, 4, 0);
    PHS_LAUNCH_CHECK();
}

BJob bjob_of(phs_plan *pl, const double *rhs, double *x) {
    BJob b;
    b.n = pl->ps.n;
    b.S = pl->S;
    b.lowrank = pl->lowrank ? 1 : 0;
    b.sign = (double)pl->sign;
    b.Q = pl->Q.get();
    b.G = pl->lowrank ? pl->G.get() : nullptr;
    b.W = pl->work.get();
    b.x = x;
    b.rhs = rhs;
    b.part = pl->part.get();
    b.scal = pl->scal.get();
    return b;
}
void batch_matvec_update(const BatchTable &t, cudaStream_t s) { steps_matvec_update(t, s); }
void batch_zproj(const BatchTable &t, cudaStream_t s) { steps_zproj(t, s); }
void batch_pupdate(const BatchTable &t, cudaStream_t s) { steps_pupdate(t, s); }
void batch_gather(const BatchTable &t, int off, double *out_dev, cudaStream_t s) {
    bk_gather<kMaxBatch><<<1, kMaxBatch, 0, s>>>(t, off, out_dev);
    PHS_LAUNCH_CHECK();
}

// The start of PCG on one plan: x = 0, r = rhs, z = P S~^-1 r, p = z, rz; returns r . r
// (synchronises s).  Work vectors 0..6.
double pcg_start(phs_plan *pl, const double *rhs, double *x, cudaStream_t s) {
    BTable<1> t;
    t.nj = 1;
    t.j[0] = bjob_of(pl, rhs, x);
    const int64_t n = pl->ps.n;
    bk_start<1><<<dim3(RED_B, 1), RED_T, 0, s>>>(t);
    PHS_LAUNCH_CHECK();
    pl->tm.begin(s);
    vecchia_apply(pl->vec, W(pl, 0), W(pl, 5), W(pl, 6), s);
    pl->tm.end(T_PRECOND, s);
    steps_zproj(t, s);
    steps_start(t, s);
    (void)n;
    return read_scalar(pl, pl->scal.get() + 5, s);
}

// PCG on sign * P M' P x = rhs (rhs in range(P)), x0 = 0.  Returns iterations; *rr_final
// the last recursive r . r.  Work vectors 0..6.  The vector operations are the table
// steps above with a table of one plan (the serving engine runs the same steps on many).
static int pcg(phs_plan *pl, const double *rhs, double *x, double tol_abs, int maxiter, int precision,
               double *rr_final, cudaStream_t s, MvTimes *mvt) {
    BTable<1> t;
    t.nj = 1;
    t.j[0] = bjob_of(pl, rhs, x);
    double rr = pcg_start(pl, rhs, x, s);
    int it = 0;
    while (std::sqrt(rr) > tol_abs && it < maxiter) {
        if (mvt) mvt->begin(s);
        matvec_norm(pl, W(pl, 2), W(pl, 4), precision, s);
        if (mvt) mvt->end(s);
        pl->tm.begin(s);
        steps_matvec_update(t, s);
        pl->tm.end(T_VEC, s);
        rr = read_scalar(pl, pl->scal.get() + 2, s);
        ++it;
        if (std::sqrt(rr) <= tol_abs) break;
        pl->tm.begin(s);
        vecchia_apply(pl->vec, W(pl, 0), W(pl, 5), W(pl, 6), s);
        pl->tm.end(T_PRECOND, s);
        pl->tm.begin(s);
        steps_zproj(t, s);
        steps_pupdate(t, s);
        pl->tm.end(T_VEC, s);
    }
    *rr_final = rr;
    return it;
}

// The start of a fit (Eq. 2.5): f to sorted order (work vector 7), rhs = sign P f (work
// vector 8), the norms and the stopping threshold; synchronises s.  When P f vanishes to
// rounding (f in span(B)) the solution is w = 0 and x (work vector 9) is zeroed.
FitStart fit_begin(phs_plan *pl, const double *f_dev, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    pl->fmm.far_valid = false;  // the fit's applies (some replayed from graphs) overwrite the expansions
    const phs_options &o = pl->opt;
    double *fs = W(pl, 7), *rhs = W(pl, 8), *x = W(pl, 9);
    double *sc = pl->scal.get();
    gather_vec<<<blocks_for(n, 256), 256, 0, s>>>(f_dev, pl->ps.perm.get(), n, fs);
    PHS_LAUNCH_CHECK();
    project(pl, fs, (double)pl->sign, rhs, rhs, sc + 6, s);
    const double rr0 = read_scalar(pl, sc + 6, s);
    dots(pl, {{fs, fs}}, sc + 9, s);
    FitStart st;
    st.fnrm = std::sqrt(read_scalar(pl, sc + 9, s));
    st.nrm0 = std::sqrt(rr0);
    st.stop = std::max(o.tol * st.nrm0, o.atol);
    st.trivial = st.nrm0 <= 1e-14 * st.fnrm || st.nrm0 == 0.0;
    if (st.trivial) {
        zero_k<<<blocks_for(n, 256), 256, 0, s>>>(x, n);
        PHS_LAUNCH_CHECK();
    }
    return st;
}

// FP64 iterative refinement around inner solves with the reduced-precision operator
// (precision 1-4).  Begin: x = 0 (work vector 9), d = rhs (work vector 11, the first
// correction's right-hand side).
void fit_refine_begin(phs_plan *pl, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    zero_k<<<blocks_for(n, 256), 256, 0, s>>>(W(pl, 9), n);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaMemcpyAsync(W(pl, 11), W(pl, 8), n * sizeof(double), cudaMemcpyDeviceToDevice, s));
}
// After an inner solve left its correction dx in work vector 8: x += dx, then the true
// residual in FP64, d = sign P (f - M' x) (work vector 11); returns ||d|| (synchronises).
double fit_refine_step(phs_plan *pl, cudaStream_t s) {
    const int64_t n = pl->ps.n;
    double *x = W(pl, 9), *y = W(pl, 10), *d = W(pl, 11);
    axpy_k<<<blocks_for(n, 256), 256, 0, s>>>(x, W(pl, 8), n, 1.0);
    PHS_LAUNCH_CHECK();
    matvec_norm(pl, x, y, 0, s);
    sub_k<<<blocks_for(n, 256), 256, 0, s>>>(y, W(pl, 7), y, n);
    PHS_LAUNCH_CHECK();
    project(pl, y, (double)pl->sign, d, d, pl->scal.get() + 7, s);
    return std::sqrt(read_scalar(pl, pl->scal.get() + 7, s));
}
// Modes 1-3 solve each correction to inner_tol of the current residual; mode 4 (float-
// float near field) is accurate enough that each inner solve aims at the final tolerance.
double refine_inner_tol(const phs_options &o, double res, double stop) {
    return o.precision == 4 ? 0.5 * stop : std::max(o.inner_tol * res, 0.5 * stop);
}
int refine_inner_maxiter(const phs_options &o, int iters_done) {
    return std::min(o.maxiter - iters_done, o.precision == 4 ? o.maxiter : 100);
}

// The end of a fit from x (work vector 9) and f (work vector 7): beta from
// R beta = Q'(f - M' x) (Eq. 2.5), the true residual ||P (f - M' x)||^2 (returned), and
// w = rho^k x in caller order; synchronises s.  After a refinement step on the same x
// (refined = true) work vector 10 already holds M' x - f from that step's FP64 matvec,
// the same product bit for bit, and it is not formed again.
double fit_end(phs_plan *pl, double *w_dev, double *beta_dev, cudaStream_t s, bool refined) {
    const int64_t n = pl->ps.n;
    double *fs = W(pl, 7), *x = W(pl, 9), *y = W(pl, 10), *d = W(pl, 11);
    double *sc = pl->scal.get();
    // the low-rank preconditioner keeps the iterates in range(P) only up to rounding
    if (pl->lowrank) project(pl, x, 1.0, x, nullptr, nullptr, s);
    if (!refined || pl->lowrank) {
        matvec_norm(pl, x, y, 0, s);
        sub_k<<<blocks_for(n, 256), 256, 0, s>>>(y, fs, y, n);
        PHS_LAUNCH_CHECK();
    }
    qt_partial<<<RED_B, RED_T, 0, s>>>(pl->Q.get(), pl->S, n, y, pl->part.get());
    PHS_LAUNCH_CHECK();
    dots_final<<<pl->S, RED_T, 0, s>>>(pl->part.get(), RED_B, sc + 40);
    PHS_LAUNCH_CHECK();
    tri_solve<<<1, 1, 0, s>>>(pl->R.get(), pl->S, sc + 40, beta_dev);
    PHS_LAUNCH_CHECK();
    project(pl, y, 1.0, d, d, sc + 8, s);
    const double rr_true = read_scalar(pl, sc + 8, s);
    scatter_scaled<<<blocks_for(n, 256), 256, 0, s>>>(x, pl->ps.perm.get(), n, std::pow(pl->ps.frame.rho, (double)pl->k),
                                                       w_dev);
    PHS_LAUNCH_CHECK();
    // the last apply of every fit path is the FP64 operator on x (above, or the refinement
    // step whose product this reuses): the expansion buffers hold the far field of this w
    remember_far_field(pl, w_dev, s);
    PHS_CUDA(cudaStreamSynchronize(s));
    return rr_true;
}

}  // namespace phs

using namespace phs;

static int min_degree(int k) { return k % 2 == 0 ? k / 2 : (k - 1) / 2; }
static int cpd_sign(int k) {
    if (k % 2 == 1) return ((k + 1) / 2) % 2 ? -1 : 1;
    return (k / 2 + 1) % 2 ? -1 : 1;
}

// Leaf capacity chosen by measurement: for the (device, k, floor(log2 n), precision,
// m2l_tensor) of a plan created with leaf_cap <= 0, time the FMM matvec on
// min(max(n, 4096), 131072) synthetic uniform points at each capacity of kLeafCaps (one
// warm-up and two timed applies, CUDA events) and keep the fastest; once per process.
static const int kLeafCaps[] = {32, 48, 64, 96, 128};
static int autotune_leaf_cap(int k, int64_t n, const phs_options &o, cudaStream_t s) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int>, int> cache;
    int dev = 0;
    PHS_CUDA(cudaGetDevice(&dev));
    int bucket = 0;
    while ((int64_t)1 << (bucket + 1) <= n) ++bucket;
    const auto key = std::make_tuple(dev, k, bucket, o.precision, o.m2l_tensor);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int64_t nt = std::min<int64_t>(std::max<int64_t>(n, 4096), 131072);
    SBuf<double> pts(2 * nt, s), t(nt, s), y(nt, s);
    tune_points<<<blocks_for(2 * nt, 256), 256, 0, s>>>(nt, 0x5eedull + (uint64_t)bucket, pts.get());
    PHS_LAUNCH_CHECK();
    tune_points<<<blocks_for(nt, 256), 256, 0, s>>>(nt / 2, 0xfeedull, t.get());
    PHS_LAUNCH_CHECK();
    cudaEvent_t e0 = ev_get(), e1 = ev_get();
    int best = 64;
    float best_ms = 1e30f;
    for (int cap : kLeafCaps) {
        phs_options ot = o;
        ot.leaf_cap = cap;
        phs_plan_t pl = nullptr;
        if (phs_plan_create(pts.get(), nt, k, -1, 0, 1, &ot, (phs_stream_t)s, &pl) != PHS_OK) continue;
        float ms = 0;
        const int mp = o.precision == 4 && k % 2 == 0 ? 4 : 0;  // the operator the fit iterates with
        bool ok = phs_matvec(pl, t.get(), y.get(), mp, (phs_stream_t)s) == PHS_OK;
        PHS_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < 2 && ok; ++r) ok = phs_matvec(pl, t.get(), y.get(), mp, (phs_stream_t)s) == PHS_OK;
        PHS_CUDA(cudaEventRecord(e1, s));
        PHS_CUDA(cudaEventSynchronize(e1));
        PHS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        phs_plan_destroy(pl);
        if (ok && ms < best_ms) {
            best_ms = ms;
            best = cap;
        }
    }
    ev_put(e0);
    ev_put(e1);
    cache[key] = best;
    return best;
}

extern "C" {

void phs_options_default(phs_options *o, int k) {
    std::memset(o, 0, sizeof(*o));
    o->precision = 0;
    o->tol = 1e-8;
    o->atol = 0.0;
    o->maxiter = 200;
    o->leaf_cap = 64;
    o->ordering = 3;
    // Matern smoothness k/2: its leading non-analytic term is r^k (log r), the PHS kernel
    o->nu = 0.5 * (k < 1 ? 2 : k);
    o->alpha = k >= 4 ? 0.5 : 0.35;
    o->domain_halfwidth = k >= 4 ? 1.0 : 0.25;
    o->seed = 1;
    o->fmm_eps = 1e-11;
    o->inner_tol = 1e-4;
    o->max_refine = 8;
    o->m2l_tensor = 1;
    o->precond_lowrank = 0;
}

const char *phs_last_error(void) { return phs::last_error(); }

int64_t phs_kernel_launches(void) { return (int64_t)phs::g_launches.load(); }

phs_status phs_plan_create(const double *pts_dev, int64_t n, int k, int poly_degree, int fmm_order, int vecchia_m,
                           const phs_options *opt, phs_stream_t stream, phs_plan_t *out) {
    PHS_TRY
    PHS_REQUIRE(out != nullptr && pts_dev != nullptr, PHS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    PHS_REQUIRE(k >= 1 && k <= 5, PHS_ERR_INVALID_ARG, "k must be in 1..5");
    const int deg = poly_degree < 0 ? min_degree(k) : poly_degree;
    PHS_REQUIRE(deg >= min_degree(k) && deg <= 3, PHS_ERR_INVALID_ARG, "poly_degree below the minimum for k, or > 3");
    const int S = (deg + 1) * (deg + 2) / 2;
    PHS_REQUIRE(n > S, PHS_ERR_INVALID_ARG, "need more points than polynomial terms");
    PHS_REQUIRE(vecchia_m >= 1 && vecchia_m <= 64, PHS_ERR_INVALID_ARG, "vecchia_m must be in 1..64");
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    phs_plan *pl = new phs_plan();
    pl->last_stream = s;
    try {
        AllocScope scope(s, &pl->dev_bytes);
        pl->k = k;
        pl->deg = deg;
        pl->S = S;
        pl->m = vecchia_m;
        if (opt) pl->opt = *opt;
        else phs_options_default(&pl->opt, k);
        const phs_options &o = pl->opt;
        PHS_REQUIRE(o.tol > 0 && o.maxiter >= 1 && o.precision >= 0 && o.precision <= 4, PHS_ERR_INVALID_ARG,
                    "bad solver options");
        PHS_REQUIRE(k % 2 == 0 || o.precision == 0 || o.precision == 4, PHS_ERR_INVALID_ARG,
                    "odd spline orders run in precision 0 or 4");
        PHS_REQUIRE(o.ordering >= 0 && o.ordering <= 3, PHS_ERR_INVALID_ARG, "ordering must be 0, 1, 2 or 3");
        int p = fmm_order;
        if (p <= 0) {
            PHS_REQUIRE(o.fmm_eps > 0 && o.fmm_eps < 1, PHS_ERR_INVALID_ARG, "fmm_eps must be in (0,1)");
            p = (int)std::ceil(std::log(o.fmm_eps) / std::log(0.55));
            p = std::max(4, std::min(p, 60));
        }
        pl->p = p;
        pl->sign = cpd_sign(k);
        if (o.leaf_cap <= 0) pl->opt.leaf_cap = autotune_leaf_cap(k, n, o, s);
        pl->hscal = pinned_block();
        build_points_and_tree(pts_dev, n, o.domain_halfwidth, pl->opt.leaf_cap, pl->ps, pl->tree, s);
        // Chebyshev order for the distance kernel: interpolation error ~ 5.83^-q at the
        // V-list separation (Bernstein ellipse of a unit gap), q in [6, 16]
        const double eps_q = fmm_order > 0 ? std::pow(0.55, fmm_order) : o.fmm_eps;
        const int cq = std::max(6, std::min(16, (int)std::ceil(std::log(eps_q) / std::log(1.0 / 5.83)) + 1));
        PHS_REQUIRE(o.m2l_tensor >= 0 && o.m2l_tensor <= 2, PHS_ERR_INVALID_ARG, "m2l_tensor must be 0, 1 or 2");
        fmm_setup(pl->fmm, k, p, std::min(p, 24), cq, o.m2l_tensor, pl->tree, s);
        // thin QR of B by two rounds of Cholesky QR (Q has orthonormal columns, R upper)
        pl->Q.alloc((size_t)S * n);
        pl->R.alloc((size_t)S * S * 3);
        pl->part.alloc((size_t)RED_B * 64);
        pl->scal.alloc(64);
        build_B<<<blocks_for(n, 256), 256, 0, s>>>(pl->ps.xs.get(), n, deg, S, pl->Q.get());
        PHS_LAUNCH_CHECK();
        SBuf<int> st(1, s);
        for (int round = 0; round < 2; ++round) {
            gram_partial<<<RED_B, RED_T, 0, s>>>(pl->Q.get(), n, S, pl->part.get());
            PHS_LAUNCH_CHECK();
            gram_chol<<<1, 1, 0, s>>>(pl->part.get(), RED_B, S, pl->R.get() + (size_t)(round + 1) * S * S, st.get());
            PHS_LAUNCH_CHECK();
            int hs = 0;
            PHS_CUDA(cudaMemcpyAsync(&hs, st.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
            PHS_CUDA(cudaStreamSynchronize(s));
            PHS_REQUIRE(hs == 0, PHS_ERR_INVALID_ARG, "polynomial block is rank deficient for these points");
            apply_rinv<<<blocks_for(n, 256), 256, 0, s>>>(pl->Q.get(), n, S, pl->R.get() + (size_t)(round + 1) * S * S);
            PHS_LAUNCH_CHECK();
        }
        mul_upper<<<1, 1, 0, s>>>(pl->R.get() + 2 * S * S, pl->R.get() + S * S, S, pl->R.get());
        PHS_LAUNCH_CHECK();
        // Vecchia preconditioner
        vecchia_build(pl->vec, pl->ps, vecchia_m, o.ordering, o.seed, o.nu, o.alpha, s, o.precision == 4);
        pl->work.alloc((size_t)12 * n);
        if (o.precond_lowrank) build_lowrank(pl, s);
        PHS_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        delete pl;
        throw;
    }
    pl->ms_plan = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = pl;
    PHS_CATCH
}

phs_status phs_plan_destroy(phs_plan_t plan) {
    PHS_TRY
    if (plan) {
        // the plan's work was issued on its last call's stream (calls on a plan are ordered)
        cudaStreamSynchronize(plan->last_stream);
        delete plan;
    }
    PHS_CATCH
}

phs_status phs_matvec(phs_plan_t pl, const double *t_dev, double *out_dev, int precision, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pl && t_dev && out_dev && t_dev != out_dev, PHS_ERR_INVALID_ARG, "bad arguments");
    PHS_REQUIRE(precision >= 0 && precision <= 4, PHS_ERR_INVALID_ARG, "precision must be 0..4");
    cudaStream_t s = (cudaStream_t)stream;
    AllocScope scope(s, &pl->dev_bytes);
    pl->last_stream = s;
    double *ts = W(pl, 8), *y = W(pl, 9);
    to_sorted(pl, t_dev, ts, 1.0, s);
    pl->tm.begin(s);
    matvec_user_sorted(pl, ts, y, precision, s);
    pl->tm.end(T_TOTAL, s);
    to_caller(pl, y, out_dev, 1.0, s);
    PHS_CATCH
}

phs_status phs_fit(phs_plan_t pl, const double *f_dev, double *w_dev, double *beta_dev, phs_fit_info *info,
                   phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pl && f_dev && w_dev && beta_dev, PHS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    AllocScope scope(s, &pl->dev_bytes);
    pl->last_stream = s;
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = pl->ps.n;
    const phs_options &o = pl->opt;
    double *rhs = W(pl, 8), *x = W(pl, 9);
    const FitStart st = fit_begin(pl, f_dev, s);
    const double nrm0 = st.nrm0, stop = st.stop;
    MvTimes mvt;
    int iters = 0, outer = 0;
    double rr = nrm0 * nrm0;
    bool converged = false;
    if (st.trivial) {
        converged = true;
    } else if (fit_precision(pl) == 0) {
        iters = pcg(pl, rhs, x, stop, o.maxiter, 0, &rr, s, &mvt);
        converged = std::sqrt(rr) <= stop;
    } else {
        // FP64 iterative refinement around inner PCG solves with the reduced-precision
        // operator.  Modes 1-3 (plain FP32 pieces) solve each correction to inner_tol;
        // mode 4 (float-float) is accurate enough that its first inner solve aims at the
        // final tolerance; if the FP64 residual still misses it, the corrections run with
        // the FP64 operator (inner_precision).
        fit_refine_begin(pl, s);
        double res = nrm0;
        while (outer < o.max_refine && iters < o.maxiter) {
            double rri = 0;
            const double itol = refine_inner_tol(o, res, stop);
            int it = pcg(pl, W(pl, 11), W(pl, 8), itol, refine_inner_maxiter(o, iters), inner_precision(pl, outer), &rri,
                         s, &mvt);
            iters += it;
            ++outer;
            res = fit_refine_step(pl, s);
            rr = res * res;
            if (res <= stop) { converged = true; break; }
            if (it == 0) break;
        }
    }
    const double rr_true = fit_end(pl, w_dev, beta_dev, s, outer > 0);
    int n_mv = 0;
    const double ms_mv = mvt.resolve(&n_mv);
    m2l_tc_check(pl->fmm, s);
    if (info) {
        info->iters = iters;
        info->outer_iters = outer;
        info->converged = converged ? 1 : 0;
        info->jittered = (int)pl->vec.jittered;
        info->rel_res_recursive = nrm0 > 0 ? std::sqrt(rr) / nrm0 : 0.0;
        info->rel_res_true = nrm0 > 0 ? std::sqrt(rr_true) / nrm0 : 0.0;
        info->ms_plan = pl->ms_plan;
        info->ms_fit = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->ms_matvec_avg = n_mv ? (float)(ms_mv / n_mv) : 0.0f;
    }
    if (!converged) throw phs::Error{PHS_ERR_NOT_CONVERGED, "PCG did not reach the tolerance"};
    PHS_CATCH
}

phs_status phs_eval(phs_plan_t pl, const double *w_dev, const double *beta_dev, const double *tgt_dev, int64_t m,
                    double *out_dev, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pl && w_dev && beta_dev && out_dev && (tgt_dev || m == 0) && m >= 0, PHS_ERR_INVALID_ARG,
                "bad arguments");
    if (m == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    AllocScope scope(s, &pl->dev_bytes);
    pl->last_stream = s;
    const int64_t n = pl->ps.n;
    double *ws = W(pl, 8);
    // w' = rho^-k w_user in sorted order
    gather_scaled<<<blocks_for(n, 256), 256, 0, s>>>(w_dev, pl->ps.perm.get(), n, std::pow(pl->ps.frame.rho, -(double)pl->k),
                                                      ws);
    PHS_LAUNCH_CHECK();
    SBuf<double2> yn(m, s);
    const Frame &fr = pl->ps.frame;
    norm_targets<<<blocks_for(m, 256), 256, 0, s>>>(tgt_dev, m, fr.cx, fr.cy, fr.rho, yn.get());
    PHS_LAUNCH_CHECK();
    // the far field of this w may be in place already (the end of its fit, or an earlier
    // evaluation of it): then only the evaluation at the targets runs
    const bool ready = far_field_of(pl, w_dev, s);
    fmm_eval64(pl->fmm, pl->tree, pl->ps, ws, yn.get(), m, out_dev, s, &pl->tm, ready);
    if (!ready) remember_far_field(pl, w_dev, s);
    add_poly<<<blocks_for(m, 256), 256, 0, s>>>(yn.get(), m, pl->deg, pl->S, beta_dev, out_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    m2l_tc_check(pl->fmm, s);
    PHS_CATCH
}

phs_status phs_fit_predict_host(const double *pts_host, const double *f_host, int64_t n, const double *tgt_host,
                                int64_t m, int k, int poly_degree, int fmm_order, int vecchia_m, const phs_options *opt,
                                double *w_host, double *beta_host, double *pred_host, phs_fit_info *info,
                                phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_host && f_host && n > 0 && m >= 0 && (tgt_host || m == 0), PHS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double> pts(2 * n, s), f(n, s), w(n, s), beta(16, s), tgt(std::max<int64_t>(2 * m, 1), s),
        pred(std::max<int64_t>(m, 1), s);
    PHS_CUDA(cudaMemcpyAsync(pts.get(), pts_host, 2 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.get(), f_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
    if (m) PHS_CUDA(cudaMemcpyAsync(tgt.get(), tgt_host, 2 * m * sizeof(double), cudaMemcpyHostToDevice, s));
    phs_plan_t pl = nullptr;
    phs_status st = phs_plan_create(pts.get(), n, k, poly_degree, fmm_order, vecchia_m, opt, stream, &pl);
    if (st != PHS_OK) return st;
    phs_fit_info inf{};
    st = phs_fit(pl, f.get(), w.get(), beta.get(), &inf, stream);
    if (st != PHS_OK && st != PHS_ERR_NOT_CONVERGED) {
        std::string msg = phs_last_error();
        phs_plan_destroy(pl);
        phs::set_error(msg);
        return st;
    }
    const phs_status fit_st = st;
    if (m) {
        st = phs_eval(pl, w.get(), beta.get(), tgt.get(), m, pred.get(), stream);
        if (st != PHS_OK) {
            std::string msg = phs_last_error();
            phs_plan_destroy(pl);
            phs::set_error(msg);
            return st;
        }
    }
    if (w_host) PHS_CUDA(cudaMemcpyAsync(w_host, w.get(), n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (beta_host) PHS_CUDA(cudaMemcpyAsync(beta_host, beta.get(), pl->S * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (pred_host && m) PHS_CUDA(cudaMemcpyAsync(pred_host, pred.get(), m * sizeof(double), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    if (info) *info = inf;
    phs_plan_destroy(pl);
    if (fit_st != PHS_OK) {
        phs::set_error("PCG did not reach the tolerance");
        return fit_st;
    }
    PHS_CATCH
}

phs_status phs_plan_frame(phs_plan_t pl, double *frame_host, int64_t *sizes_host) {
    PHS_TRY
    PHS_REQUIRE(pl, PHS_ERR_INVALID_ARG, "null plan");
    if (frame_host) {
        frame_host[0] = pl->ps.frame.cx;
        frame_host[1] = pl->ps.frame.cy;
        frame_host[2] = pl->ps.frame.rho;
        frame_host[3] = pl->ps.frame.hw;
    }
    if (sizes_host) {
        sizes_host[0] = pl->ps.n;
        sizes_host[1] = pl->k;
        sizes_host[2] = pl->S;
        sizes_host[3] = pl->p;
        sizes_host[4] = pl->fmm.nd;
        sizes_host[5] = pl->tree.nbox;
        sizes_host[6] = pl->tree.nleaf;
        sizes_host[7] = pl->tree.depth;
    }
    PHS_CATCH
}

phs_status phs_plan_vecchia(phs_plan_t pl, int64_t *order_host, int64_t *nbr_host) {
    PHS_TRY
    PHS_REQUIRE(pl, PHS_ERR_INVALID_ARG, "null plan");
    const int64_t n = pl->ps.n;
    const int m = pl->m;
    if (order_host) {
        // caller index of rank r = perm[order_pos[r]]
        std::vector<int> ho(n), hp(n);
        PHS_CUDA(cudaMemcpy(ho.data(), pl->vec.order.get(), n * sizeof(int), cudaMemcpyDeviceToHost));
        PHS_CUDA(cudaMemcpy(hp.data(), pl->ps.perm.get(), n * sizeof(int), cudaMemcpyDeviceToHost));
        for (int64_t r = 0; r < n; ++r) order_host[r] = hp[ho[r]];
    }
    if (nbr_host) {
        std::vector<int> ell((size_t)m * n), hp(n);
        PHS_CUDA(cudaMemcpy(ell.data(), pl->vec.nbr.get(), ell.size() * sizeof(int), cudaMemcpyDeviceToHost));
        PHS_CUDA(cudaMemcpy(hp.data(), pl->ps.perm.get(), n * sizeof(int), cudaMemcpyDeviceToHost));
        for (int64_t p = 0; p < n; ++p)
            for (int q = 0; q < m; ++q) {
                const int v = ell[(size_t)q * n + p];
                nbr_host[(int64_t)hp[p] * m + q] = v >= 0 ? hp[v] : -1;
            }
    }
    PHS_CATCH
}

phs_status phs_plan_vecchia_factor(phs_plan_t pl, double *diag_host, double *offd_host) {
    PHS_TRY
    PHS_REQUIRE(pl, PHS_ERR_INVALID_ARG, "null plan");
    const int64_t n = pl->ps.n;
    const int m = pl->m;
    std::vector<double> val((size_t)(m + 1) * n);
    std::vector<int> hp(n);
    PHS_CUDA(cudaMemcpy(val.data(), pl->vec.val.get(), val.size() * sizeof(double), cudaMemcpyDeviceToHost));
    PHS_CUDA(cudaMemcpy(hp.data(), pl->ps.perm.get(), n * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t p = 0; p < n; ++p) {
        if (diag_host) diag_host[hp[p]] = val[p];
        if (offd_host)
            for (int q = 0; q < m; ++q) offd_host[(int64_t)hp[p] * m + q] = val[(size_t)(1 + q) * n + p];
    }
    PHS_CATCH
}

phs_status phs_plan_precond(phs_plan_t pl, const double *r_dev, double *z_dev, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pl && r_dev && z_dev, PHS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    AllocScope scope(s, &pl->dev_bytes);
    pl->last_stream = s;
    const int64_t n = pl->ps.n;
    double *rs = W(pl, 8), *zs = W(pl, 9);
    gather_vec<<<blocks_for(n, 256), 256, 0, s>>>(r_dev, pl->ps.perm.get(), n, rs);
    PHS_LAUNCH_CHECK();
    double *t1 = W(pl, 10), *t2 = W(pl, 11);
    project(pl, rs, 1.0, t1, nullptr, nullptr, s);
    precond(pl, t1, zs, rs, t2, s);
    scatter_scaled<<<blocks_for(n, 256), 256, 0, s>>>(zs, pl->ps.perm.get(), n, 1.0, z_dev);
    PHS_LAUNCH_CHECK();
    PHS_CATCH
}

phs_status phs_plan_work(phs_plan_t pl, int64_t *counts_host) {
    PHS_TRY
    PHS_REQUIRE(pl && counts_host, PHS_ERR_INVALID_ARG, "bad arguments");
    counts_host[0] = pl->tree.near_pairs;
    counts_host[1] = pl->tree.m2l_pairs;
    PHS_CATCH
}

phs_status phs_plan_memory(phs_plan_t pl, int64_t *bytes_host) {
    PHS_TRY
    PHS_REQUIRE(pl && bytes_host, PHS_ERR_INVALID_ARG, "bad arguments");
    *bytes_host = pl->dev_bytes;
    PHS_CATCH
}

phs_status phs_plan_kernel_work(phs_plan_t pl, int64_t *counts_host) {
    PHS_TRY
    PHS_REQUIRE(pl && counts_host, PHS_ERR_INVALID_ARG, "bad arguments");
    const Tree &t = pl->tree;
    const bool sym = t.sym_ok;
    counts_host[0] = sym ? t.p2p_self_pairs + t.p2p_upper_pairs : t.near_pairs;
    counts_host[1] = sym ? t.p2p_upper_pairs : 0;
    counts_host[2] = pl->fmm.tc_steps;
    counts_host[3] = pl->fmm.tc_tiles;
    counts_host[4] = pl->fmm.tc ? m2l_tc_mmas_per_step() : 0;
    counts_host[5] = pl->fmm.tc ? (int64_t)128 * pl->fmm.tc_npad * 16 : 0;
    PHS_CATCH
}

phs_status phs_plan_set_wait_limit(phs_plan_t pl, int64_t ns, int probe) {
    PHS_TRY
    PHS_REQUIRE(pl && ns >= 0 && (probe == 0 || probe == 1), PHS_ERR_INVALID_ARG, "bad arguments");
    pl->fmm.tc_wait_ns = (uint64_t)ns;
    pl->fmm.tc_probe = probe;
    PHS_CATCH
}

phs_status phs_plan_set_timing(phs_plan_t pl, int enabled) {
    PHS_TRY
    PHS_REQUIRE(pl, PHS_ERR_INVALID_ARG, "null plan");
    pl->tm.resolve();
    pl->tm.enabled = enabled != 0;
    pl->tm.reset();
    PHS_CATCH
}

phs_status phs_plan_timing(phs_plan_t pl, double *ms_host, int64_t *calls_host) {
    PHS_TRY
    PHS_REQUIRE(pl, PHS_ERR_INVALID_ARG, "null plan");
    pl->tm.resolve();
    for (int i = 0; i < 8; ++i) {
        if (ms_host) ms_host[i] = pl->tm.ms[i];
        if (calls_host) calls_host[i] = pl->tm.calls[i];
    }
    PHS_CATCH
}

phs_status phs_dense_matvec(const double *pts_dev, int64_t n, int k, const double *t_dev, double *out_dev,
                            phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && t_dev && out_dev && n >= 0 && k >= 1 && k <= 5, PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double2> x(n, s);
    pts_to_d2<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, x.get());
    PHS_LAUNCH_CHECK();
    dense_matvec64(x.get(), n, k, t_dev, out_dev, s);
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_CATCH
}

phs_status phs_random_order(int64_t n, uint64_t seed, int64_t *order_dev, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(order_dev && n >= 0 && n < (1ll << 31), PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<int> o(n, s);
    random_order_dev(n, seed, o.get(), s);
    to_i64<<<blocks_for(n, 256), 256, 0, s>>>(o.get(), n, order_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_CATCH
}

phs_status phs_maxmin_order(const double *pts_dev, int64_t n, int64_t *order_dev, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && order_dev && n >= 0 && n < (1ll << 31), PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double2> x(n, s);
    pts_to_d2<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, x.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> o(n, s);
    maxmin_order_dev(x.get(), n, o.get(), s);
    to_i64<<<blocks_for(n, 256), 256, 0, s>>>(o.get(), n, order_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_CATCH
}

phs_status phs_hmaxmin_order(const double *pts_dev, int64_t n, uint64_t seed, int64_t *order_dev,
                             phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && order_dev && n >= 0 && n < (1ll << 31), PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double2> x(n, s);
    pts_to_d2<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, x.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> o(n, s);
    hmaxmin_order_dev(x.get(), n, seed, o.get(), s);
    to_i64<<<blocks_for(n, 256), 256, 0, s>>>(o.get(), n, order_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_CATCH
}

phs_status phs_amaxmin_order(const double *pts_dev, int64_t n, int64_t *order_dev, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && order_dev && n >= 0 && n < (1ll << 31) - 1, PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double2> x(n, s);
    pts_to_d2<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, x.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> o(n, s);
    amaxmin_order_dev(x.get(), n, o.get(), s);
    to_i64<<<blocks_for(n, 256), 256, 0, s>>>(o.get(), n, order_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_CATCH
}

phs_status phs_knn_prev(const double *pts_dev, int64_t n, const int64_t *order_dev, int m, int64_t *nbr_dev,
                        phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && order_dev && nbr_dev && n >= 0 && n < (1ll << 31) && m >= 1 && m <= 64,
                PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double2> x(n, s);
    pts_to_d2<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, x.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> o(n, s), ell((size_t)m * n, s);
    from_i64<<<blocks_for(n, 256), 256, 0, s>>>(order_dev, n, o.get());
    PHS_LAUNCH_CHECK();
    knn_prev_dev(x.get(), n, o.get(), m, ell.get(), s);
    ell_to_rows_i64<<<blocks_for((int64_t)m * n, 256), 256, 0, s>>>(ell.get(), n, m, nbr_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    PHS_CATCH
}

phs_status phs_vecchia_factor(const double *pts_dev, int64_t n, const int64_t *order_dev, const int64_t *nbr_dev, int m,
                              double nu, double alpha, double *diag_dev, double *offd_dev, int64_t *jittered_host,
                              phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && order_dev && nbr_dev && diag_dev && offd_dev && n >= 0 && m >= 1 && m <= 64,
                PHS_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return PHS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SBuf<double2> x(n, s);
    pts_to_d2<<<blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, x.get());
    PHS_LAUNCH_CHECK();
    SBuf<int> rank(n, s), ell((size_t)m * n, s);
    checked_ranks_dev(order_dev, nbr_dev, n, m, rank.get(), s);
    rows_to_ell_i32<<<blocks_for((int64_t)m * n, 256), 256, 0, s>>>(nbr_dev, n, m, ell.get());
    PHS_LAUNCH_CHECK();
    SBuf<double> val((size_t)(m + 1) * n, s);
    int64_t nj = vecchia_factor_dev(x.get(), n, rank.get(), ell.get(), m, nu, alpha, val.get(), s);
    PHS_CUDA(cudaMemcpyAsync(diag_dev, val.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ell_to_rows_d<<<blocks_for((int64_t)m * n, 256), 256, 0, s>>>(val.get(), n, m, 1, offd_dev);
    PHS_LAUNCH_CHECK();
    PHS_CUDA(cudaStreamSynchronize(s));
    if (jittered_host) *jittered_host = nj;
    PHS_CATCH
}

}  // extern "C"
