// phs_internal.cuh -- shared declarations of the CUDA implementation (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <exception>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "../../include/phs.h"

namespace phs {

// ---------------------------------------------------------------- errors
struct Error {
    phs_status code;
    std::string msg;
};
void set_error(const std::string &msg);
const char *last_error();

#define PHS_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            throw ::phs::Error{e_ == cudaErrorMemoryAllocation ? PHS_ERR_OOM : PHS_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_)};    \
        }                                                                               \
    } while (0)
// every kernel launch in the library is followed by PHS_LAUNCH_CHECK(), which also
// counts it (phs_kernel_launches)
void count_launch();
void count_launches(int64_t k);  // k launches at once (kernels of a replayed graph)
#define PHS_LAUNCH_CHECK()        \
    do {                          \
        ::phs::count_launch();    \
        PHS_CUDA(cudaGetLastError()); \
    } while (0)
#define PHS_REQUIRE(cond, code, msg)                                                    \
    do {                                                                                \
        if (!(cond)) throw ::phs::Error{code, msg};                                     \
    } while (0)

// every extern "C" entry point wraps its body in PHS_TRY ... PHS_CATCH: library errors
// return their code, host allocation failures PHS_ERR_OOM, any other C++ exception
// PHS_ERR_CUDA, each with its message for phs_last_error(); success clears the message
#define PHS_TRY try {
#define PHS_CATCH                                                        \
    }                                                                    \
    catch (const ::phs::Error &e) {                                      \
        ::phs::set_error(e.msg);                                         \
        return e.code;                                                   \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        ::phs::set_error("host allocation failed");                      \
        return PHS_ERR_OOM;                                              \
    }                                                                    \
    catch (const std::exception &e) {                                    \
        ::phs::set_error(e.what());                                      \
        return PHS_ERR_CUDA;                                             \
    }                                                                    \
    ::phs::set_error("");                                                \
    return PHS_OK;

inline unsigned blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- device buffers
// Allocation context of the calling thread.  While an AllocScope is alive (the plan
// entry points open one), DBuf allocations come from the library's stream-ordered memory
// pool on the scope's stream and are counted into the scope's byte counter, so creating
// and destroying plans never triggers the implicit device synchronisation of
// cudaMalloc/cudaFree.  A pooled buffer is released in stream order: on the stream of
// the scope active at release, else on a library-owned stream of the device (used after
// the caller's work on the buffer is known to be complete, as in phs_plan_destroy).
// Outside any scope DBuf falls back to cudaMalloc/cudaFree.
struct AllocCtx {
    bool on = false;
    cudaStream_t s = nullptr;
    int64_t *bytes = nullptr;
};
AllocCtx &alloc_ctx();
struct AllocScope {
    AllocCtx prev;
    AllocScope(cudaStream_t s, int64_t *bytes) : prev(alloc_ctx()) { alloc_ctx() = AllocCtx{true, s, bytes}; }
    ~AllocScope() { alloc_ctx() = prev; }
    AllocScope(const AllocScope &) = delete;
    AllocScope &operator=(const AllocScope &) = delete;
};
void dbuf_alloc(void **p, size_t bytes, bool *pooled, int64_t **acct);
// run fn once per (device, id) in this process, under a lock (constant tables, function
// attributes); ids: 1 log tables, 2 float-float tables, 3 Bessel tables, 4 pass limits
void once_per_device(int id, const std::function<void()> &fn);
void dbuf_free(void *p, size_t bytes, bool pooled, int64_t *acct);

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    bool pooled = false;
    int64_t *acct = nullptr;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), pooled(o.pooled), acct(o.acct) {
        o.p = nullptr;
        o.n = 0;
        o.acct = nullptr;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; pooled = o.pooled; acct = o.acct;
            o.p = nullptr; o.n = 0; o.acct = nullptr;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count) dbuf_alloc((void **)&p, count * sizeof(T), &pooled, &acct);
        n = count;
    }
    void release() {
        if (p) dbuf_free(p, n * sizeof(T), pooled, acct);
        p = nullptr;
        n = 0;
        pooled = false;
        acct = nullptr;
    }
    T *get() const { return p; }
};

// Stream-ordered scratch from the library's memory pool of the current device (created on
// first use, keeping up to 1 GB of freed blocks for reuse): allocation and release are
// ordered on the stream that uses the buffer, so neither synchronises the device the way
// cudaMalloc / cudaFree do.  For temporaries whose every use is on one stream.
cudaMemPool_t scratch_pool();
template <typename T>
struct SBuf {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    SBuf(size_t count, cudaStream_t stream) : s(stream) {
        if (count) PHS_CUDA(cudaMallocFromPoolAsync((void **)&p, count * sizeof(T), scratch_pool(), s));
    }
    SBuf(const SBuf &) = delete;
    SBuf &operator=(const SBuf &) = delete;
    ~SBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    T *get() const { return p; }
};

// ---------------------------------------------------------------- primitives (sort_scan.cu)
// exclusive scan of int32 counts; returns total (synchronises stream)
int64_t exclusive_scan_i32(const int *in, int *out, int64_t n, cudaStream_t s);
// stable LSD radix sort of (key, value) pairs on the low `bits` bits of key
void radix_sort_pairs(uint64_t *keys, int *vals, int64_t n, int bits, cudaStream_t s);

// ---------------------------------------------------------------- tree (tree.cu)
constexpr int kMaxLevel = 20;  // quadtree levels 0..kMaxLevel

struct Frame {
    double cx = 0, cy = 0, rho = 1, hw = 0.25;  // x' = (x - c) * rho in [-hw, hw]^2
};

struct Tree {
    int64_t n = 0;
    int leaf_cap = 64;
    int depth = 0;                   // deepest level present
    int nbox = 0, nleaf = 0;
    double R = 0.25;                 // root box [-R, R]^2
    std::vector<int> lvl_off;        // boxes of level l: [lvl_off[l], lvl_off[l+1])
    DBuf<int> lvl_dev;               // device copy of lvl_off
    DBuf<int> start, end, parent, child, nchild, level;
    DBuf<uint64_t> key;              // Morton key of the box at its own level
    DBuf<double2> ctr;               // box centres
    DBuf<int> leaf_box;              // leaf list
    DBuf<int> point_leaf;            // leaf index of each (sorted) point
    DBuf<int> v_off, v_src;          // V (M2L) lists per box (CSR)
    DBuf<unsigned char> v_cls;       // offset class (dx+3)*7 + (dy+3)
    DBuf<int> near_off;              // near (direct) ranges per box (CSR)
    DBuf<int2> near_rng;
    int64_t near_pairs = 0, m2l_pairs = 0;
    // symmetric near field: leaf li writes the column sums of its near ranges after it
    // (Morton order) to scratch [sym_slot[li], ...); leaf d gathers its share from the
    // slots of earlier leaves, starting at the offsets sym_gbase[sym_goff[d] .. sym_goff[d+1])
    bool sym_ok = false;             // every leaf fits one P2P pass (<= kP2PThreads points)
    int64_t p2p_self_pairs = 0, p2p_upper_pairs = 0;  // pairs in own leaves / ranges after a leaf
    int max_leaf = 0, max_up_ranges = 0;
    int64_t sym_total = 0;
    DBuf<int> sym_slot, sym_goff, sym_gbase;
    DBuf<int> p2p_order;             // leaves by decreasing near-field pair count
};
constexpr int kP2PThreads = 128;     // threads of a near-field block
constexpr int kMaxUpRanges = 256;    // near ranges after a leaf that one block holds

struct PointSet {
    int64_t n = 0;
    Frame frame;
    DBuf<double2> xs;  // normalised coordinates, Morton order
    DBuf<int> perm;    // perm[p] = caller index of sorted position p
    DBuf<int> iperm;   // iperm[i] = sorted position of caller index i
};

// normalise caller points, Morton-sort them and build the adaptive quadtree + lists
void build_points_and_tree(const double *pts_dev, int64_t n, double halfwidth, int leaf_cap,
                           PointSet &ps, Tree &tree, cudaStream_t s);
// device view of the tree for kernels
struct TreeView {
    const int *start, *end, *parent, *child, *nchild, *level;
    const uint64_t *key;
    const int *lvl_off;  // device copy
    const double2 *ctr;  // box centres (null while the tree is being built)
    int depth;
    double R;
    double rinv2;        // 1 / (2R), correctly rounded
};
TreeView tree_view(const Tree &t);

// ---------------------------------------------------------------- FMM (fmm.cu)
struct FmmOps;  // translation operators for one precision
struct Fmm {
    int k = 2, p = 20, P = 21, nd = 4;  // P = p + 1 coefficients (FP64 expansions)
    int p32 = 20, P32 = 21;             // FP32 expansions
    int power = 2;                      // r^{power} Hadamard factor, 0 for k = 1
    bool log_core = true;               // log kernel (even k) or distance kernel (odd k)
    // expansions (complex, [box][nd][P]); double and float variants allocated on demand
    DBuf<double2> mp64, lc64;
    DBuf<float2> mp32, lc32;
    DBuf<double2> ops64;  // M2M[4], L2L[4], M2L[49] (P x P each)
    // M2M/L2L of quadrant q = e^{i th_q l} R[l][k] e^{-i th_q k} (offset d_q = |d| e^{i th_q}):
    // the real shift cores [2][P][P] (M2M, L2L) and the phases e^{i th_q k} [4][P]
    DBuf<double> shift_r;
    DBuf<double2> shift_ph;
    DBuf<float2> shift_rff;  // shift_r split into hi + lo floats
    DBuf<float4> shift_phff; // shift_ph split into hi + lo floats
    DBuf<float2> ops32;   // same for the FP32 order P32
    DBuf<float2> ops32p, mpx32, lcx32;  // FP32 copies at the FP64 order (FP32 M2L mode)
    DBuf<double> mix64;                 // box-local Hadamard frame changes [57][nd][nd]
    DBuf<float> mix32;
    DBuf<float2> mixff;                 // mix64 split into hi + lo floats
    DBuf<int> lvl_off_dev;
    // Chebyshev (distance kernel) data
    int cheb_q = 0;                      // nodes per dimension
    int cheb_rt = 0, cheb_rs = 0;        // ranks of the compressed M2L (target, source bases)
    DBuf<double> cheb64;                 // Tn [q][q] | A [2][q][q]
    DBuf<double> cheb_lr;                // compressed M2L: U' [rt][q*q] | V [q*q][rs] | C' [49][rs][rt]
    DBuf<double> cwc64, clc64;           // compressed weights [box][nd][rs], potentials [box][nd][rt]
    // its M2L on the tensor cores (cheb_tc.cu)
    bool ctc = false;
    int ctc_npad = 0, ctc_nch = 0;       // output columns (rank rounded up to 16), K chunks of 32
    DBuf<uint16_t> ctc_b;                // operator digit planes (bf16 bits)
    DBuf<int> ctc_F;                     // column exponents [rt]
    DBuf<int> ctc_mexp;                  // per-box exponent bound of the compressed weights
    DBuf<double> cw64, cl64;             // weights/potentials at nodes [box][nd][q*q]
    // tensor-core M2L of the log kernel (m2l_tc.cu)
    bool tc = false;                     // use it for the FP64 far field
    bool ff_passes = true;               // precision 4: P2M and L2P in float-float too
    int tc_npad = 0, tc_nch = 0;         // output columns (P rounded up to 16), K chunks
    DBuf<uint16_t> tc_b;                 // operator digit planes (bf16 bits)
    DBuf<int> tc_F;                      // column exponents [P]
    DBuf<int> tc_S;                      // integer frame changes [49][nd][nd]
    DBuf<int> tc_gexp;                   // log2 bound of the frame-change row growth [49][nd]
    DBuf<int2> tc_off;                   // nd = 4: class offsets (ox, oy)
    DBuf<int> tc_mexp;                   // per-box exponent bound of the multipoles
    DBuf<int> tc_tgt;                    // M2L targets (levels >= 2) by (level, child position, box)
    // The FP64 far field held in the expansion buffers is that of the caller-order
    // coefficients far_w (set by the end of a fit, whose last apply is the FP64 operator on
    // the solution, and by an evaluation); any FMM apply clears it
    bool far_valid = false;
    DBuf<double> far_w;
    int tc_tgt_nbox = -1;                // box count of the tree tc_tgt was built for
    DBuf<int> tc_err;                    // device status (nonzero: a bounded wait expired)
    uint64_t tc_wait_ns = 0;             // main-loop wait limit of the pass (0: the 2 s default)
    int tc_probe = 0;                    // test hook: make the pass's first wait expire
    int64_t tc_steps = 0, tc_tiles = 0;  // work of one pass (m2l_tc_count)
    DBuf<double> sym_scratch;            // column sums of the symmetric near field
    DBuf<int> p2p_ticket;                // next leaf of the near-field blocks (reset per launch)
    // the near field runs on a second stream, overlapping the upward pass, M2L and L2L,
    // and joins before L2P adds the far field into y (created on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Fmm() = default;
    Fmm(const Fmm &) = delete;
    Fmm &operator=(const Fmm &) = delete;
    ~Fmm();
};
// tensor_m2l: 1 runs the FP64 M2L of the log kernel on the tensor cores (m2l_tc.cu), 2
// the distance kernel's compressed M2L too (cheb_tc.cu), 0 neither
void fmm_setup(Fmm &f, int k, int p, int p32, int cheb_q, int tensor_m2l, const Tree &t, cudaStream_t s);
// tensor-core M2L (m2l_tc.cu): setup from the class operators (slots 8 + cls of the
// level-invariant operator table, [57][P][P] complex) and the frame changes ([57][nd][nd]);
// the pass writes lc for every box (zero where the interaction list is empty)
bool m2l_tc_supported(int nd, int P);
void m2l_tc_setup(Fmm &f, const std::vector<long double> &ops_re, const std::vector<long double> &ops_im,
                  const std::vector<long double> &mix, cudaStream_t s);
// (rewrites the multipoles mp in place as per-box fixed point: the upward pass is done)
void m2l_tc_pass(Fmm &f, const Tree &t, double2 *mp, double2 *lc, cudaStream_t s);
// steps and tiles of one pass over this tree (sets f.tc_steps, f.tc_tiles)
void m2l_tc_count(Fmm &f, const Tree &t, cudaStream_t s);
int m2l_tc_mmas_per_step();
// throws PHS_ERR_TIMEOUT if a tensor-core wait expired since the last check (synchronises s)
void m2l_tc_check(Fmm &f, cudaStream_t s);
// integer frame changes (slots 0..48 of the mix table) and their growth bound, shared
// by the tensor-core M2L passes (m2l_tc.cu)
void tc_integer_frames(int nd, const std::vector<long double> &mix, std::vector<int> &S, std::vector<int> &gexp);
// distance-kernel far field (cheb.cu)
// q Chebyshev nodes per axis; the M2L operators compressed to relative accuracy lr_eps
// (rank at most 80); tensor: its M2L on the tensor cores where supported (cheb_tc.cu)
void cheb_setup(Fmm &f, int q, double lr_eps, bool tensor, const std::vector<long double> &mix, cudaStream_t s);
// the compressed M2L on the tensor cores (cheb_tc.cu): setup from the transposed class
// operators C' [49][rs][rt]; the pass writes the compressed potentials of boxes b0..
// (overwritten) and rewrites the compressed weights wc in place as per-box fixed point
bool cheb_tc_supported(int nd, int rs, int rt);
void cheb_tc_setup(Fmm &f, const double *Ct, const std::vector<long double> &mix, cudaStream_t s);
void cheb_m2l_tc_pass(Fmm &f, const Tree &t, int b0, double *wc, double *lc, cudaStream_t s);
void cheb_far_field(Fmm &f, const Tree &t, const PointSet &ps, const double *t_sorted, cudaStream_t s,
                    struct Timers *tm);
void cheb_l2p_apply(Fmm &f, const Tree &t, const PointSet &ps, double *y, cudaStream_t s);
void cheb_eval_far_launch(Fmm &f, const Tree &t, const double2 *tgt, const int *box_of, int64_t m, double *out,
                          cudaStream_t s);
// near field in float-float arithmetic on the FP32 pipe (nearfield_ff.cu), symmetric
// schedule: rows into y, column sums of the ranges after each leaf into scratch (the
// caller adds them with p2p_gather); needs t.sym_ok.  upload_ff_tables() loads its
// logarithm tables on the current device (once per plan).
void p2p_sym_ff(const Tree &t, const PointSet &ps, int k, const double *tv_sorted, double *y, double *scratch,
                int *ticket, cudaStream_t s);
void upload_ff_tables();
// float-float P2M and L2P of the log-kernel far field (farfield_ff.cu): the same FP64
// expansion layout as the FP64 passes ([box][d][k] complex coefficients), per-point
// arithmetic on the FP32 pipe; P2M overwrites every leaf's mp, L2P adds into y.
void p2m_ff_launch(const Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, double2 *mp,
                   cudaStream_t s);
void l2p_ff_launch(const Fmm &f, const Tree &t, const PointSet &ps, const double2 *lc, double *y, cudaStream_t s);
// float-float M2M (parents b0 .. b0+nb-1 from their children's mp) and L2L (those parents
// into their children's lc); the phases and frame changes in FP64, the triangular core
// in float-float
void m2m_ff_launch(const Fmm &f, const Tree &t, int b0, int nb, double2 *mp, cudaStream_t s);
void l2l_ff_launch(const Fmm &f, const Tree &t, int b0, int nb, double2 *lc, cudaStream_t s);
// y = M' t for sorted-order vectors in the normalised frame (M' of the normalised points)
// mode 0: FP64 throughout; 1: FP32 near field + FP64 far field; 2: FP32 near field and
// FP32 M2L inside FP64 upward/downward passes; 3: FP32 throughout (order p32);
// 4: float-float near field, P2M, M2M, L2L and L2P on the FP32 pipe + M2L as configured
void fmm_apply(Fmm &f, const Tree &t, const PointSet &ps, const double *t_sorted, double *y_sorted, int mode,
               cudaStream_t s, struct Timers *tm);
// evaluate sum_j w_j phi(|x_j - y|) at normalised targets (after an FMM upward/downward
// pass on w, skipped when far_ready: the expansion buffers already hold w's FP64 far
// field), out written (overwritten) for m targets
void fmm_eval64(Fmm &f, const Tree &t, const PointSet &ps, const double *w_sorted,
                const double2 *tgt_norm, int64_t m, double *out, cudaStream_t s, struct Timers *tm,
                bool far_ready = false);
// exact all-pairs product out = M t (points in any order, FP64)
void dense_matvec64(const double2 *x, int64_t n, int k, const double *t, double *out, cudaStream_t s);

// ---------------------------------------------------------------- timers
// Per-phase device time from CUDA events recorded on the launching stream; events
// are resolved lazily (resolve()) so timing adds no host synchronisation.
struct EvRec {
    cudaEvent_t a, b;
    int phase;
};
struct Timers {
    bool enabled = false;
    double ms[8] = {0};
    int64_t calls[8] = {0};
    std::vector<cudaEvent_t> stack;
    std::vector<EvRec> pending;
    void begin(cudaStream_t s);
    void end(int phase, cudaStream_t s);
    void resolve();
    void reset() { for (int i = 0; i < 8; ++i) { ms[i] = 0; calls[i] = 0; } }
    ~Timers();
};
enum { T_P2P = 0, T_M2L = 1, T_UP = 2, T_DOWN = 3, T_PRECOND = 4, T_VEC = 5, T_EVAL = 6, T_TOTAL = 7 };

// ---------------------------------------------------------------- Vecchia (vecchia.cu)
struct Vecchia {
    int m = 0;
    int64_t n = 0;
    DBuf<int> rank;       // rank of sorted position p
    DBuf<int> order;      // order[r] = sorted position of rank r
    DBuf<int> nbr;        // ELL [m][n] sorted positions of neighbours (-1 pad)
    DBuf<double> val;     // ELL [m+1][n]: slot 0 = 1/c, slot 1+q = -lambda_q/c
    // rows of U~ (for z = U~ y) as sliced ELL: rows sorted by length (descending, stable),
    // slices of 32 consecutive sorted rows padded to the slice's longest row and stored
    // column-major (entry k of sorted position p at s_off[p/32] + 32 k + p%32), each row's
    // entries in column order; padding has value 0
    DBuf<int> s_row;   // row of sorted position p
    DBuf<int> s_off;   // first entry of each slice
    DBuf<int> s_len;   // entries per row of each slice
    DBuf<int> s_col;
    DBuf<double> s_val;
    int64_t jittered = 0;
};
void random_order_dev(int64_t n, uint64_t seed, int *order_out, cudaStream_t s);
void maxmin_order_dev(const double2 *x, int64_t n, int *order_out, cudaStream_t s);
// maximin.cu
void hmaxmin_order_dev(const double2 *x, int64_t n, uint64_t seed, int *order_out, cudaStream_t s);
void amaxmin_order_dev(const double2 *x, int64_t n, int *order_out, cudaStream_t s);
void knn_prev_dev(const double2 *x, int64_t n, const int *order, int m, int *nbr_ell, cudaStream_t s);
int64_t vecchia_factor_dev(const double2 *x, int64_t n, const int *rank, const int *nbr_ell, int m,
                           double nu, double alpha, double *val_ell, cudaStream_t s, bool ff = false);
// rank[order[r]] = r for a caller's enumeration (int64, any device buffer), checking that
// order is a permutation and, if nbr (n x m int64 rows) is given, that the first
// min(m, rank(i)) entries of row i are points of smaller rank; PHS_ERR_INVALID_ARG otherwise
void checked_ranks_dev(const int64_t *order, const int64_t *nbr, int64_t n, int m, int *rank, cudaStream_t s);
void vecchia_build(Vecchia &v, const PointSet &ps, int m, int ordering, uint64_t seed, double nu,
                   double alpha, cudaStream_t s, bool ff = false);
// z = U~ (U~' r) (sorted order)
void vecchia_apply(const Vecchia &v, const double *r, double *tmp, double *z, cudaStream_t s);
// the two halves of z = U (U' r): y = U' r and z = U y
void vecchia_apply_ut(const Vecchia &v, const double *r, double *y, cudaStream_t s);
void vecchia_apply_u(const Vecchia &v, const double *y, double *z, cudaStream_t s);

}  // namespace phs
