/*
 * phs.h -- C ABI of a B300 (sm_103a) implementation of linear-cost
 * polyharmonic-spline (PHS) interpolation after Geoga & O'Neil,
 * "Linear-cost Polyharmonic Spline Interpolation of Arbitrary Degree".
 *
 * Problem (Sec. 1, Eqs. 1.1-1.3): given points x_j in R^2 and values f_j, find
 * weights w and polynomial coefficients beta with
 *     [ M  B ] [ w    ]   [ f ]
 *     [ B' 0 ] [ beta ] = [ 0 ],   M_ij = phi(|x_i - x_j|),  B_js = P_s(x_j),
 * phi(r) = r^k (k odd) or r^k log r (k even), so that
 *     f^(y) = sum_s beta_s P_s(y) + sum_j w_j phi(|x_j - y|).
 * The solve follows Sec. 2: points are mapped to a square domain (Eq. 2.1),
 * PCG runs on Q_perp' M Q_perp (Eq. 2.5) with M applied by a 2D fast multipole
 * method through the Hadamard/low-rank identity (Eq. 2.6) and the Vecchia
 * sparse inverse-Cholesky preconditioner of a Matern covariance (Sec. 2.2,
 * Eq. 2.19, Fig. 1).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees or retains them past the call.  Pointers named *_host
 *    are host pointers (pinned memory gives asynchronous copies).
 *  - Points are row-major n x 2 arrays of double (x0, y0, x1, y1, ...).
 *  - Vectors are double, indexed in the caller's point order.
 *  - All work is enqueued on `stream` (0 = legacy default stream).  Calls that
 *    return host-visible results (info structs, host outputs) synchronise it.
 *  - Errors are returned as phs_status; no exception crosses the ABI.  A
 *    human-readable message for the most recent failing call on the calling
 *    host thread is available from phs_last_error().
 *  - A plan may be used from one stream at a time: a call on another stream must
 *    not start before the previous call's work on the plan has completed.
 *  - Device memory: a plan's state and the temporaries of every call come from a
 *    stream-ordered memory pool the library creates per device on first use
 *    (cudaMallocFromPoolAsync / cudaFreeAsync on the call's stream), so creating,
 *    using and destroying plans never synchronises the device the way
 *    cudaMalloc / cudaFree do; the pool keeps up to 1 GB of freed blocks for reuse
 *    and returns the rest.  phs_plan_memory reports a plan's bytes.
 *    phs_dense_matvec_noalloc uses no pool (see its entry).
 */
#ifndef PHS_B300_H
#define PHS_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *phs_stream_t; /* == cudaStream_t */
typedef struct phs_plan *phs_plan_t;

typedef enum {
    PHS_OK = 0,
    PHS_ERR_INVALID_ARG = 1,      /* bad size, k, degree, option, or non-finite input */
    PHS_ERR_DUPLICATE_POINTS = 2, /* two input points coincide exactly */
    PHS_ERR_OOM = 3,              /* device allocation failed */
    PHS_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed */
    PHS_ERR_NOT_CONVERGED = 5,    /* PCG reached maxiter above tolerance (results still written) */
    PHS_ERR_CHOLESKY = 6,         /* a local Vecchia factor failed even after jitter, or the
                                     S x S matrix Q' S~^{-1} Q of the low-rank term did */
    PHS_ERR_TIMEOUT = 7           /* a bounded device wait expired (see phs_plan_set_wait_limit) */
} phs_status;

/* Solver options (defaults from phs_options_default). */
typedef struct {
    int precision;          /* FMM arithmetic inside the CG iterations:
                               0: FP64 throughout (plain PCG);
                               1: FP32 near field, FP64 far field;
                               2: FP32 near field and FP32 M2L, FP64 elsewhere;
                               3: FP32 throughout (order min(p, 24));
                               4: near field, P2M, M2M, L2L, L2P (even k) and the local
                                  factorisations of the preconditioner in float-float (hi +
                                  lo FP32, about 2^-46 per operation) on the FP32 pipe, M2L
                                  as m2l_tensor.  Odd k fits with 4 run the FP64 operator
                                  (phs_matvec with 4 applies the float-float near field).
                               Modes 1-4 run inside FP64 iterative refinement: the
                               outer residual uses the FP64 FMM; residuals, inner
                               products, projection and preconditioner stay FP64.  Modes
                               1-3 do not converge on large clustered sets (the projected
                               system amplifies FP32 rounding); mode 4 does.  Odd k: 0 or 4.
                               Modes 1-4 need |t| < 1e37 in the vectors they multiply. */
    double tol;             /* stop when ||r_k|| <= max(tol*||Q_perp' f||, atol); default 1e-8 */
    double atol;            /* default 0 */
    int maxiter;            /* PCG iterations (precision 0) or total inner iterations; default 200 */
    int leaf_cap;           /* quadtree leaf capacity s (the near-field tile: a leaf's points
                               are the rows of its direct-sum tiles); default 64.  <= 0: the
                               capacity of {32, 48, 64, 96, 128} whose FMM matvec is fastest,
                               timed once per process for each (device, k, floor(log2 n),
                               precision, m2l_tensor) on synthetic uniform points */
    int ordering;           /* Vecchia enumeration: 0 random (Sec. 3), 1 exact maxmin (single
                               block, O(n^2): small n), 2 hierarchical maximin (phs_hmaxmin_order),
                               3 dyadic approximate maximin (phs_amaxmin_order; the default: on
                               the clustered 1M-point TPS set 14 PCG iterations against 16 for
                               2 and 23 for 0) */
    double nu;              /* Matern smoothness: 0.5, 1, 1.5, 2 or 2.5; default k/2, whose
                               leading non-analytic term is the PHS kernel (nu = 1 for the
                               thin-plate spline, Sec. 2.2, Eq. 2.17) */
    double alpha;           /* Matern inverse range in the NORMALISED frame; default 0.35 (k<=3), 0.5 (k>=4) */
    double domain_halfwidth;/* points are mapped into [-h, h]^2; default 0.25 (k<=3), 1 (k>=4) */
    uint64_t seed;          /* random enumeration seed */
    double fmm_eps;         /* FMM truncation target used when fmm_order <= 0; default 1e-11 */
    double inner_tol;       /* precision 1-3: relative tolerance of each inner solve; default 1e-4
                               (precision 4 aims each inner solve at the final tolerance) */
    int max_refine;         /* precision 1-4: maximum refinement steps; default 8 */
    int m2l_tensor;         /* 1 (default): the log kernel's (even k) multipole-to-local
                               translations (Sec. 2.1, Eq. 2.14) run on the tensor cores in
                               exact fixed point (bf16 digit planes, about 1e-12 relative);
                               the distance kernel's (odd k) compressed M2L in FP64.  2: the
                               distance kernel's too (about 2e-12 relative to its FP64 form;
                               its rounding is not symmetric at the 1e-14 level, which the CG
                               fit of ill-conditioned odd-k systems does not tolerate -- the
                               100,000-point cubic set then does not converge -- so meant for
                               phs_matvec and phs_gmres).  0: both in FP64 on the CUDA cores.
                               A bounded device wait of a tensor-core path that expires is
                               reported as PHS_ERR_TIMEOUT by the next phs_fit or phs_eval
                               (phs_matvec is asynchronous). */
    int precond_lowrank;    /* 1: the preconditioner is the inverse of Q_perp' S~ Q_perp
                               on range(P) (S~^{-1} = U U' the Vecchia factor), i.e.
                               S~^{-1} r - G (B' G)^{-1} G' r with G = S~^{-1} B -- the low-rank
                               (Schur complement) term of Sec. 2.2, built once per plan and
                               applied at the cost of the projection it replaces; 0 (default):
                               the plain Q_perp' S~^{-1} Q_perp that the paper runs (on the
                               clustered 1M-point TPS workload the low-rank form takes one
                               iteration more; on 4k-40k points one fewer). */
} phs_options;

typedef struct {
    int iters;              /* PCG iterations (all inner iterations for precision 1) */
    int outer_iters;        /* refinement steps (precision 1), else 0 */
    int converged;          /* 1 if the stopping rule was met */
    int jittered;           /* Vecchia local factors that needed diagonal jitter */
    double rel_res_recursive; /* final recursive residual / ||Q_perp' f|| */
    double rel_res_true;      /* ||Q_perp'(f - M w)|| / ||Q_perp' f|| with an FP64 FMM matvec */
    float ms_plan;          /* plan creation wall time (set by phs_plan_create) */
    float ms_fit;           /* phs_fit wall time */
    float ms_matvec_avg;    /* average FMM matvec time inside the fit */
} phs_fit_info;

/* Fill *opt with the defaults for spline order k. */
void phs_options_default(phs_options *opt, int k);

/* Thread-local message of the last failing call ("" if none). */
const char *phs_last_error(void);

/* Number of CUDA kernel launches this library has issued in this process
 * (all threads, all plans); differences of two readings count the launches of
 * the calls between them. */
int64_t phs_kernel_launches(void);

/*
 * Build a plan for n points (Sec. 2, setup phase):
 *   normalisation to [-h,h]^2 (Eq. 2.1), Morton sort and adaptive quadtree with
 *   FMM interaction lists (Sec. 2.1), thin QR of B (Eq. 2.4), Vecchia
 *   enumeration, conditioning sets and local factors (Sec. 2.2, Eq. 2.19).
 * pts_dev:     n x 2 device array, caller order.  Must be finite and distinct.
 * k:           spline order, 1..5 (Eq. 1.2).
 * poly_degree: total degree of the polynomial block; >= k/2 (even k) or (k-1)/2
 *              (odd k), <= 3.  -1 selects the minimum.
 * fmm_order:   number of expansion terms p (Sec. 2.1, Eqs. 2.12-2.15); <= 0 picks
 *              p from opt->fmm_eps.  At most 60.
 * vecchia_m:   conditioning-set size m (Sec. 2.2), 1..64.
 * opt:         NULL for phs_options_default(k).
 * On success *out receives the plan (free with phs_plan_destroy).  The call
 * synchronises `stream`.
 */
phs_status phs_plan_create(const double *pts_dev, int64_t n, int k, int poly_degree,
                           int fmm_order, int vecchia_m, const phs_options *opt,
                           phs_stream_t stream, phs_plan_t *out);

/* out = M t in the caller's frame and order, M_ij = phi(|x_i - x_j|) (Eq. 1.3),
 * by the FMM of Sec. 2.1 applied through Eq. (2.6).  precision selects the
 * arithmetic as in phs_options.precision (0 = FP64 FMM, 0..4; odd k: 0 or 4).
 * t_dev, out_dev: n doubles on the device (may not alias). */
phs_status phs_matvec(phs_plan_t plan, const double *t_dev, double *out_dev, int precision,
                      phs_stream_t stream);

/* Solve the augmented system (Eq. 1.3) by the sequence of Eq. (2.5) with
 * Vecchia-preconditioned CG.  f_dev: n values (caller order).  w_dev: n weights
 * in the caller's frame.  beta_dev: S coefficients of the monomials
 * 1, x, y, x^2, xy, y^2, ... evaluated in the plan's NORMALISED frame
 * (x' = (x - c) * rho, see phs_plan_frame).  info may be NULL.  Synchronises. */
phs_status phs_fit(phs_plan_t plan, const double *f_dev, double *w_dev, double *beta_dev,
                   phs_fit_info *info, phs_stream_t stream);

/* Evaluate the interpolant (Eq. 1.1) at m targets (m x 2 device array, caller
 * frame) with the FMM for the kernel part; w_dev/beta_dev as returned by
 * phs_fit.  out_dev: m values.  The plan keeps a device copy of the w whose FP64
 * far field (multipole and local expansions) it last built, at the end of
 * phs_fit or in an earlier phs_eval; when w_dev equals it bit for bit the
 * upward pass, M2L and downward pass are skipped and only the target-side
 * evaluation runs.  The result then agrees with a recomputed far field to
 * rounding (the fit built it from its own scaling of the same weights).
 * phs_matvec, a new fit or a tensor-core wait timeout clears the record.
 * Synchronises `stream`. */
phs_status phs_eval(phs_plan_t plan, const double *w_dev, const double *beta_dev,
                    const double *tgt_dev, int64_t m, double *out_dev, phs_stream_t stream);

/* End-to-end fit and prediction from HOST buffers: copies points/values in,
 * builds a plan, fits, evaluates at the targets and copies w, beta and the
 * predictions out.  Any output pointer may be NULL.  Synchronises. */
phs_status phs_fit_predict_host(const double *pts_host, const double *f_host, int64_t n,
                                const double *tgt_host, int64_t m, int k, int poly_degree,
                                int fmm_order, int vecchia_m, const phs_options *opt,
                                double *w_host, double *beta_host, double *pred_host,
                                phs_fit_info *info, phs_stream_t stream);

/* Releases every device buffer the plan owns (resource management, no counterpart in the
 * paper).  Synchronises the stream of the plan's most recent call first (that stream
 * must still exist), then returns the buffers to the memory pool without synchronising
 * the device; NULL is accepted and does nothing; the handle is invalid afterwards. */
phs_status phs_plan_destroy(phs_plan_t plan);

/* Solve M c = b for the kernel matrix ALONE (no polynomial block; the preconditioning
 * comparison of Sec. 3.1) by restarted GMRES with the plan's Vecchia factor U~ U~' as a
 * right preconditioner, so the residual it minimises is ||b - M c||.  b_dev, c_dev: n
 * doubles, caller order (may not alias).  Tolerance stop = max(tol ||b||, atol) with the
 * plan's tol and atol; maxiter bounds the total iterations; restart: Krylov vectors per
 * cycle, 1..127 (the basis takes restart + 1 vectors of n doubles from the memory pool).
 * A cycle ends when its least-squares residual estimate is <= stop.  check_true = 0
 * stops there (the iteration count a GMRES library reports); check_true = 1 recomputes
 * ||b - M c|| and restarts until it meets stop (it can stall near rounding, about
 * eps ||M|| ||c||, for ill-conditioned M).  The FMM runs in FP64 (plan precision 0..3)
 * or with the float-float near field (precision 4).  info (may be NULL): iters = GMRES
 * iterations, outer_iters = cycles, rel_res_recursive = the last estimate / ||b||,
 * rel_res_true = the recomputed ||b - M c|| / ||b||, ms_matvec_avg as for phs_fit.
 * Returns PHS_ERR_NOT_CONVERGED (c still written) when maxiter is reached first.
 * Synchronises. */
phs_status phs_gmres(phs_plan_t plan, const double *b_dev, double *c_dev, int restart, int check_true,
                     phs_fit_info *info, phs_stream_t stream);

/* Choose the Matern inverse range alpha of the Vecchia preconditioner for these points
 * and values by a gradient-free search on PCG's iteration count (the tuning of Sec. 2.2).
 * The domain scaling and alpha enter the preconditioned iteration only through their
 * product, so the search is over alpha at the domain of opt (domain_halfwidth).  Trials
 * are full plans and fits on a seeded random subsample of n_sample points (<= 0 or >= n:
 * all points): alpha0 * 10^(i/4), i = -8..4, with alpha0 = opt->alpha, then six steps of
 * golden-section search around the best; a trial costs its iteration count plus
 * log10(final residual / tol) in [-1, 0].  *alpha_out receives the best alpha (never
 * worse on the subsample than alpha0), *iters_out (may be NULL) its iteration count.
 * pts_dev, f_dev: as phs_plan_create and phs_fit; other arguments as phs_plan_create.
 * Synchronises. */
phs_status phs_tune_alpha(const double *pts_dev, const double *f_dev, int64_t n, int k, int poly_degree,
                          int fmm_order, int vecchia_m, const phs_options *opt, int64_t n_sample,
                          double *alpha_out, int *iters_out, phs_stream_t stream);

/* ---- inspection (small host copies; synchronise) --------------------------- */
/* frame[0..3] = (centre_x, centre_y, rho, halfwidth); sizes[0..7] = (n, k, S, p,
 * nd, n_boxes, n_leaves, depth). */
phs_status phs_plan_frame(phs_plan_t plan, double *frame_host, int64_t *sizes_host);
/* Enumeration and conditioning sets built by the plan: order_host[r] = caller
 * index of rank r (n entries); nbr_host: n x m caller indices, -1 padded, by
 * increasing (squared distance, rank).  Either pointer may be NULL. */
phs_status phs_plan_vecchia(phs_plan_t plan, int64_t *order_host, int64_t *nbr_host);
/* Vecchia factor columns (Fig. 1): diag_host[i] = 1/c_i, offd_host[i*m+q] = -lambda_q/c_i
 * (caller order, slots aligned with phs_plan_vecchia's nbr). */
phs_status phs_plan_vecchia_factor(phs_plan_t plan, double *diag_host, double *offd_host);
/* z = Q_perp-projected preconditioner P U~ U~' P r (Sec. 2.2); caller order. */
phs_status phs_plan_precond(phs_plan_t plan, const double *r_dev, double *z_dev,
                            phs_stream_t stream);
/* Direct-interaction pair count of the tree (P2P work per matvec) and V-list
 * translation count (M2L work per matvec): counts_host[0..1]. */
phs_status phs_plan_work(phs_plan_t plan, int64_t *counts_host);
/* Device bytes held by the plan (tree, lists, expansions, operators, QR, Vecchia factor,
 * work vectors; not the temporaries of calls in flight): *bytes_host. */
phs_status phs_plan_memory(phs_plan_t plan, int64_t *bytes_host);
/* Work of one FP64 matvec per kernel, for roofline accounting (host array of 6):
 *   [0] point pairs the near-field kernel evaluates (own leaf: all ordered pairs;
 *       pairs across leaves once on the symmetric path, both orders otherwise),
 *   [1] of those, pairs that also feed a column sum (symmetric path),
 *   [2] tensor-core M2L steps (offset class x 48-column K chunk, summed over the
 *       16-box tiles; 0 when the M2L runs on the CUDA cores),
 *   [3] tensor-core M2L tiles,
 *   [4] digit-plane products per step (plane pairs x 16-deep K slices; the pass issues
 *       them as fewer tcgen05.mma, each spanning several B planes along N),
 *   [5] multiply-adds of one product (M * N * K, N = output columns padded to 16). */
phs_status phs_plan_kernel_work(phs_plan_t plan, int64_t *counts_host);
/* Diagnostics and test hook of the tensor-core M2L's bounded waits (no counterpart in
 * the paper).  ns: wall-time limit of each pipeline wait in the pass's main loop (0
 * restores the default of 2 s); every wait also gives up after ns / 4 polls, so it ends
 * even if the device timer stalls.  probe = 1 makes each block of the later passes wait
 * first on a barrier that nothing completes, so that wait always expires: the block
 * issues no work, and the pass flags the plan.  A wait that expires makes every block
 * of the pass stop issuing work; the multiply-adds and copies already issued are still
 * waited for (with the fixed 2 s limit) before the kernel exits, so the device and the
 * plan stay usable, and the next phs_fit or phs_eval on the plan returns
 * PHS_ERR_TIMEOUT (phs_matvec is asynchronous and does not check).  probe = 0 and
 * ns = 0 restore normal operation. */
phs_status phs_plan_set_wait_limit(phs_plan_t plan, int64_t ns, int probe);
/* Per-phase device timing of the most recent phs_fit / phs_matvec calls, in ms,
 * measured with CUDA events on the plan's stream when enabled (0/1).  While enabled the
 * near field runs on the plan's stream instead of beside the far field on a second
 * stream, so each phase's events time that phase alone (results are bit-identical).
 * ms_host[0..7] = (p2p, m2l, upward, downward, precond, vector, eval, total);
 * calls_host[0..7] = launches timed per phase. */
phs_status phs_plan_set_timing(phs_plan_t plan, int enabled);
phs_status phs_plan_timing(phs_plan_t plan, double *ms_host, int64_t *calls_host);

/* ---- stand-alone building blocks (device pointers, caller order) ----------- */
/* out = M t with an exact O(n^2) all-pairs sum in FP64 (Eq. 1.3). */
phs_status phs_dense_matvec(const double *pts_dev, int64_t n, int k, const double *t_dev,
                            double *out_dev, phs_stream_t stream);
/* The same exact product as phs_dense_matvec without allocating device memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- real-time loops that must not hit the implicit device synchronisation
 * of cudaMalloc/cudaFree, and applications that hand all device memory to their own
 * pool.  The points are staged in a fixed device array inside the library (65,536
 * points, 1 MiB, kept by every GPU that loads the library until the process exits);
 * n > 65536 returns PHS_ERR_INVALID_ARG.  The first call on a device, made with that
 * device current, looks up that array's address (cudaGetSymbolAddress) and keeps it
 * for the life of the process; make that first call before any stream capture, and do
 * not use the library across a cudaDeviceReset of that device (the address would be
 * stale).  All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Asynchronous on `stream`, unlike phs_dense_matvec, which synchronises before it
 * returns: pts_dev, t_dev and out_dev must stay valid, and out_dev unread, until the
 * stream has reached this work. */
phs_status phs_dense_matvec_noalloc(const double *pts_dev, int64_t n, int k, const double *t_dev,
                                    double *out_dev, phs_stream_t stream);

/* Random enumeration (Sec. 3): order_dev[r] = index of rank r, ranks sorted by
 * (SplitMix64(seed, i), i), SplitMix64 output i = mix(seed + (i+1)*0x9E3779B97F4A7C15). */
phs_status phs_random_order(int64_t n, uint64_t seed, int64_t *order_dev, phs_stream_t stream);
/* Exact maxmin enumeration of the given points: first the point nearest the
 * bounding-box centre, then repeatedly the point farthest from the selected
 * set; ties to the smaller index.  Squared distances dx*dx+dy*dy, no FMA. */
phs_status phs_maxmin_order(const double *pts_dev, int64_t n, int64_t *order_dev,
                            phs_stream_t stream);
/* Hierarchical maximin enumeration (parallel, O(n log n)): over a dyadic grid of the
 * bounding square (side E = larger extent, level-30 cell coordinates
 * ix = min(floor((x - xmin) * (2^30 / E)), 2^30 - 1)), each level-L cell is represented
 * by its parent cell's representative if that lies in it, else by its point nearest the
 * cell centre ((x-cx)^2 + (y-cy)^2 in FP64 without FMA, ties to the smaller index); a
 * point's level is the first level at which it represents its cell (31 if never), and
 * points are enumerated by (level, SplitMix64(seed, i) >> 7, i).  The points first
 * picked at level L are one per cell, about a cell width from everything earlier: the
 * spacing property of an exact maxmin ordering, level by level. */
phs_status phs_hmaxmin_order(const double *pts_dev, int64_t n, uint64_t seed, int64_t *order_dev,
                             phs_stream_t stream);
/* Dyadic approximate maximin enumeration (parallel): the first point is the one nearest
 * the centre of the bounding square (side E as above, ties to the smaller index); l2 is
 * each point's squared distance to the points taken so far.  For L = 0..30 (cell side
 * c = E 2^-L, level-L cells as above), passes repeat while an untaken point has
 * l2 >= c^2: in each cell the such point with the largest l2 (ties to the smaller index)
 * is eligible; eligible points are visited by (l2 descending, index) and accepted unless
 * an accepted point of the same pass is closer than c; the pass appends them in that
 * order.  Points never accepted (coincident ones) follow by (l2 descending, index).
 * Every point, when appended, is at least half as far from the points before it as the
 * farthest point still to come (an exact maxmin order: equally far).  Squared distances
 * dx*dx+dy*dy without FMA.  n < 2^31 - 1; the device buffers are the caller's. */
phs_status phs_amaxmin_order(const double *pts_dev, int64_t n, int64_t *order_dev, phs_stream_t stream);
/* Conditioning sets (Sec. 2.2): for the point of rank r (order_dev as above) the
 * min(m, r) points of smaller rank nearest to it, by (squared distance
 * dx*dx+dy*dy without FMA, rank); nbr_dev is n x m int64, -1 padded. */
phs_status phs_knn_prev(const double *pts_dev, int64_t n, const int64_t *order_dev, int m,
                        int64_t *nbr_dev, phs_stream_t stream);
/* Vecchia factor columns (Eq. 2.19, Fig. 1) for conditioning sets nbr_dev
 * (n x m int64, -1 padded) of a Matern(nu, alpha) covariance with K(0) = 1:
 * diag_dev[i] = 1/c_i, offd_dev[i*m+q] = -lambda_q / c_i.  order_dev (n int64)
 * must be a permutation of 0..n-1, and the first min(m, rank(i)) entries of row i
 * of nbr_dev points of smaller rank; otherwise PHS_ERR_INVALID_ARG (checked on the
 * device before any coordinate is read).  nu in {0.5, 1, 1.5, 2, 2.5}, alpha > 0.
 * A local Cholesky that fails (a pivot that is not positive) is retried with
 * diagonal jitter 1e-12 * 10^(t-1) on the conditioning block, t = 1..7 (up to 1e-6);
 * if it still fails, or the conditional variance c is not positive, that point gets
 * an empty conditioning set (diag = 1, offd = 0).  *jittered_host (may be NULL)
 * receives how many points needed either.  Synchronises. */
phs_status phs_vecchia_factor(const double *pts_dev, int64_t n, const int64_t *order_dev,
                              const int64_t *nbr_dev, int m, double nu, double alpha,
                              double *diag_dev, double *offd_dev, int64_t *jittered_host,
                              phs_stream_t stream);

/* ---- serving: continuous batching of many interpolation requests ------------- */
/* A server owns a scheduler thread and setup_threads host worker threads on the device
 * current at phs_server_create.  Requests arrive through phs_server_submit from any host
 * thread at any time.  A request is admitted while fewer than max_active are in setup or
 * in PCG and the memory it reserves fits memory_budget (an a-priori estimate, replaced
 * by the plan's measured bytes plus a quarter once its plan exists; a request larger
 * than the budget still runs, alone).  Each admitted job keeps its plan (tree, FMM
 * tables, QR, Vecchia factor -- Sec. 2) and its PCG state (Eq. 2.5) on the device until
 * it finishes.  Every scheduler tick advances all active jobs by one PCG iteration: each
 * job's FMM matvec and Vecchia apply run on its own stream, and the vector operations of
 * all jobs run as shared launches, one device-to-host copy of the residuals per tick.
 * A job computes exactly what phs_fit followed by phs_eval computes for it (same steps,
 * same arithmetic), alone or in any mix; precision 1-4 jobs run phs_fit's FP64
 * refinement around their inner solves (odd k: precision 0 or 4).  No counterpart in the
 * paper: the serving and batched forms of its solve. */
typedef struct phs_server *phs_server_t;
typedef struct {
    int64_t memory_budget;  /* device bytes the admitted jobs may reserve; <= 0: half the free memory */
    int max_active;         /* jobs in setup or PCG at once, 1..96; <= 0: 32 */
    int setup_threads;      /* host threads building plans and finishing jobs, 1..64; <= 0: 4 */
} phs_server_config;

/* cfg may be NULL (defaults).  Allocates the engine's stream and two small buffers. */
phs_status phs_server_create(const phs_server_config *cfg, phs_server_t *out);
/* Queue one request: points (n x 2), values (n) and targets (m x 2) are HOST arrays,
 * copied before the call returns; k, poly_degree, fmm_order, vecchia_m and opt as for
 * phs_plan_create (NULL: phs_options_default(k)).
 * *job_id receives the request's id.  Thread-safe; does not wait for the GPU. */
phs_status phs_server_submit(phs_server_t server, const double *pts_host, const double *f_host, int64_t n,
                             const double *tgt_host, int64_t m, int k, int poly_degree, int fmm_order,
                             int vecchia_m, const phs_options *opt, int64_t *job_id);
/* Block until the job finishes, then copy its results to host arrays (any may be NULL):
 * w (n), beta (S, normalised frame as phs_fit), predictions at the targets (m), info
 * (as phs_fit's; ms_fit is the time from the end of setup to completion), and
 * times_host[0..3] = submission, admission, end of setup and completion, in seconds
 * since phs_server_create.  Returns the job's status (PHS_ERR_NOT_CONVERGED with results,
 * or the error that ended it).  A job's results can be collected once. */
phs_status phs_server_wait(phs_server_t server, int64_t job_id, double *w_host, double *beta_host,
                           double *pred_host, phs_fit_info *info, double *times_host);
/* stats_host[0..7] = (ticks, job-iterations run in ticks, most jobs in one tick, most
 * bytes reserved at once, the budget, jobs completed, requests waiting for admission,
 * bytes reserved now). */
phs_status phs_server_stats(phs_server_t server, int64_t *stats_host);
/* Finish every submitted job, stop the threads and release the server.  Results not
 * collected are discarded. */
phs_status phs_server_destroy(phs_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* PHS_B300_H */
