// plan.cuh -- the plan object behind the C ABI and the solver helpers shared by the
// files that run solves on it (abi.cu: PCG fit, evaluation; krylov.cu: GMRES, tuning).
#pragma once
#include <initializer_list>
#include <utility>
#include <vector>

#include "phs_internal.cuh"

// A plan: one point set with its tree, FMM tables, polynomial QR and Vecchia factor, and
// the work vectors of its solves.  Vectors inside are in sorted (Morton) order.
struct phs_plan {
    // device bytes held by the plan's buffers (first member: destroyed last, after every
    // buffer that counts into it)
    int64_t dev_bytes = 0;
    cudaStream_t last_stream = nullptr;  // stream of the plan's most recent call
    int k = 2, S = 3, deg = 1, m = 30, p = 20;
    phs_options opt{};
    phs::PointSet ps;
    phs::Tree tree;
    phs::Fmm fmm;
    phs::Vecchia vec;
    phs::DBuf<double> Q;      // [S][n] sorted order
    phs::DBuf<double> R;      // S x S upper triangular, row-major
    phs::DBuf<double> G;      // [S][n] S~^{-1} Q Rc^{-1}, Rc'Rc = Q' S~^{-1} Q (low-rank preconditioner term)
    bool lowrank = false;
    phs::DBuf<double> work;   // 12 work vectors of n
    phs::DBuf<double> part;   // reduction partials
    phs::DBuf<double> scal;   // device scalars
    double *hscal = nullptr;  // pinned host mirror (64 doubles from phs::pinned_block)
    phs::Timers tm;
    float ms_plan = 0;
    int sign = 1;             // sign * Q_perp' M Q_perp is positive definite
    ~phs_plan();
};

namespace phs {

// 64 pinned host doubles from a process-wide pool (never returned to the CUDA driver, so a
// plan's destruction does not synchronise the device through cudaFreeHost)
double *pinned_block();
void pinned_release(double *b);

// work vector i (n doubles; 12 of them)
double *W(phs_plan *pl, int i);
// out[q] = a_q . b_q for the pairs given (deterministic two-level reductions), on the device
void dots(phs_plan *pl, std::initializer_list<std::pair<const double *, const double *>> prs, double *out,
          cudaStream_t s);
// out = sign * P v (P = I - Q Q'); if other != null, dot(other, out) -> *dot_out (device)
void project(phs_plan *pl, const double *v, double sign, double *out, const double *other, double *dot_out,
             cudaStream_t s);
// y = M' t in the normalised frame (FMM), sorted order
void matvec_norm(phs_plan *pl, const double *t, double *y, int precision, cudaStream_t s);
// y = M t with the caller's kernel matrix, sorted order
void matvec_user_sorted(phs_plan *pl, const double *ts, double *y, int precision, cudaStream_t s);
// caller order <-> sorted order, times a scale
void to_sorted(phs_plan *pl, const double *src, double *dst, double scale, cudaStream_t s);
void to_caller(phs_plan *pl, const double *src, double *dst, double scale, cudaStream_t s);
// one device double to the host (synchronises s)
double read_scalar(phs_plan *pl, const double *dev, cudaStream_t s);
// preconditioner of the projected system (Sec. 2.2): z from r in range(P); tmp, tmp2 scratch
void precond(phs_plan *pl, const double *r, double *z, double *tmp, double *tmp2, cudaStream_t s);
// the low-rank (Schur complement) preconditioner term of the plan (Sec. 2.2)
void build_lowrank(phs_plan *pl, cudaStream_t s);
// rebuild the Vecchia preconditioner for a new Matern inverse range (synchronises s)
void plan_set_alpha(phs_plan *pl, double alpha, cudaStream_t s);
// restarted right-preconditioned GMRES on M c = b in sorted order (krylov.cu)
int gmres_solve(phs_plan *pl, const double *b_s, double *x_s, int restart, double stop, int maxiter, int precision,
                bool check_true, double *res, double *est, int *restarts, struct MvTimes *mvt, cudaStream_t s);
// ---- a fit in pieces (abi.cu): begin, the PCG iterations, end
struct FitStart {
    double nrm0, fnrm, stop;  // ||P f||, ||f||, max(tol ||P f||, atol)
    bool trivial;             // P f vanishes to rounding: w = 0 (x already zeroed)
};
FitStart fit_begin(phs_plan *pl, const double *f_dev, cudaStream_t s);
double fit_end(phs_plan *pl, double *w_dev, double *beta_dev, cudaStream_t s, bool refined);
// refinement (precision 1-4): x = 0, d = rhs; one step x += dx, d = sign P(f - M' x) in
// FP64, returning ||d||; the inner solves run PCG with rhs = work vector 11, x = 8
void fit_refine_begin(phs_plan *pl, cudaStream_t s);
double fit_refine_step(phs_plan *pl, cudaStream_t s);
// The arithmetic a fit runs in.  Precision 4 with odd k solves with the FP64 operator:
// the distance-kernel far field (FP64) dominates there, so the float-float near field
// saves under a tenth of a matvec, less than the Krylov restart a refinement step costs
// on those ill-conditioned systems.
inline int fit_precision(const phs_plan *pl) { return pl->opt.precision == 4 && pl->k % 2 ? 0 : pl->opt.precision; }
// The operator of a refinement's inner solve: precision 4 runs its first solve in
// float-float; when the FP64 residual check after it fails, the operator's rounding is
// what remains, so the corrections use the FP64 operator.  Modes 1-3 keep theirs.
inline int inner_precision(const phs_plan *pl, int outer) {
    const int fp = fit_precision(pl);
    return fp == 4 && outer > 0 ? 0 : fp;
}
double refine_inner_tol(const phs_options &o, double res, double stop);
int refine_inner_maxiter(const phs_options &o, int iters_done);

// ---- PCG steps on a table of plans (abi.cu).  Each step runs RED_B x RED_T blocks per
// plan with blockIdx.y selecting the plan, the same arithmetic as on a one-plan table,
// so a plan's iterates do not depend on the other plans of the table.
struct BJob {
    int64_t n;
    int S, lowrank;
    double sign;
    const double *Q, *G;  // projection basis; the low-rank term's basis (or null)
    double *W;            // work vectors: r 0, z 1, p 2, q 3, y 4, t1 5, t2 6
    double *x;            // iterate
    const double *rhs;    // right-hand side (read by the start step)
    double *part;         // reduction partials [RED_B][12]
    double *scal;         // device scalars: 0 rz, 1 pq, 2 rr, 3 rz_new, 4-5 start, 16.. coefficients
};
template <int N>
struct BTable {
    int nj;
    BJob j[N];
};
constexpr int kMaxBatch = 96;  // plans per table (passed by value: 96 x 88 bytes of parameters)
using BatchTable = BTable<kMaxBatch>;
BJob bjob_of(phs_plan *pl, const double *rhs, double *x);
// the start of PCG on one plan (x = 0, r = rhs, z, p, rz); returns r . r (synchronises s)
double pcg_start(phs_plan *pl, const double *rhs, double *x, cudaStream_t s);
// after y = M' p (work vector 4) of every plan: q = sign P y, p . q, x, r and r . r (scal 2)
void batch_matvec_update(const BatchTable &t, cudaStream_t s);
// after t2 = S~^-1 r (work vector 6): z = P t2 (or the low-rank form)
void batch_zproj(const BatchTable &t, cudaStream_t s);
// rz_new = r . z, p = z + (rz_new / rz) p, rz = rz_new
void batch_pupdate(const BatchTable &t, cudaStream_t s);
// out[k] = scal_k[off] (device)
void batch_gather(const BatchTable &t, int off, double *out_dev, cudaStream_t s);

// pooled CUDA events of the calling thread
cudaEvent_t ev_get();
void ev_put(cudaEvent_t e);
// Matvec timing of a solve: an event pair around each matvec on the solve's stream,
// resolved once after the solve's final synchronisation (no synchronisation per matvec).
struct MvTimes {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    void begin(cudaStream_t s) {
        ev.emplace_back(ev_get(), ev_get());
        cudaEventRecord(ev.back().first, s);
    }
    void end(cudaStream_t s) { cudaEventRecord(ev.back().second, s); }
    // sum of the recorded intervals in ms (the stream must have passed them); recycles the events
    double resolve(int *count);
    ~MvTimes();
};

}  // namespace phs
