// farfield_ff.cu -- the per-point passes of the log-kernel FMM (Sec. 2.1) in float-float
// arithmetic on the FP32 pipe, for precision 4: P2M (outgoing expansions of the leaves,
// Eq. 2.14, with the Hadamard charges of Eq. 2.6) and L2P (evaluation of the incoming
// expansions, Eq. 2.15, combined with the Hadamard factors).  They read and write the
// same FP64 expansions as the FP64 passes (fmm.cu p2m64_kernel / l2p64_kernel), so M2M,
// M2L and L2L are unchanged; only the per-point arithmetic moves to hi + lo floats
// (about 2^-46 per operation, ff.cuh).  Their rounding enters the expansion coefficients,
// so it reaches the matvec as a smooth far-field perturbation, not as the pairwise noise
// the preconditioned system amplifies.
//
// P2M, per leaf: z_j = (x_j - c)/w, q_{d,j} = v_d(z_j) t_j; a~_0 = sum_j q, a~_k = -sum_j q
// z^k / k.  Points in chunks of 64: four threads per point build the powers z^k (a
// quarter each, started by binary powering) into shared memory, then each thread owns
// outputs (d, k) and sums over the chunk.
// L2P, per point of a leaf: y += sum_d u_d(v) Re sum_k b~_{d,k} v^k, v = (x - c)/w, the
// leaf's coefficients split once into hi + lo in shared memory.
#include <algorithm>

#include "ff.cuh"
#include "geom.cuh"
#include "hadamard.cuh"
#include "phs_internal.cuh"

namespace phs {
namespace {
using namespace ffa;

constexpr int PF_T = 256;   // P2M threads per leaf
constexpr int PF_OUT = 3;   // outputs per thread: nd P <= 768
constexpr int LF_T = 128;   // L2P threads per leaf
constexpr int kFfMaxNd = 10;

template <int ND>
__global__ void __launch_bounds__(PF_T) p2m_ff_kernel(TreeView tv, const int *leaf_box, const double2 *xs,
                                                      const double *t, int power, int P, double2 *mp) {
    extern __shared__ float4 pf_sm[];
    float4 *pw = pf_sm;                                          // [64][P] powers, hi + lo parts
    float2 *qs = reinterpret_cast<float2 *>(pw + (size_t)64 * P);  // [64][ND] charges
    const int b = leaf_box[blockIdx.x];
    double cx, cy, w;
    box_geom(tv, b, cx, cy, w);
    const double iw = 1.0 / w;
    const int s = tv.start[b], e = tv.end[b];
    const int nout = ND * P;
    const int Q = (P + 3) / 4;
    C4 acc[PF_OUT];
#pragma unroll
    for (int i = 0; i < PF_OUT; ++i) acc[i] = {F2{0.f, 0.f}, F2{0.f, 0.f}};
    for (int j0 = s; j0 < e; j0 += 64) {
        const int jn = min(64, e - j0);
        {
            const int jp = threadIdx.x >> 2, q = threadIdx.x & 3;
            if (jp < jn) {
                const double2 xj = xs[j0 + jp];
                const double zx = (xj.x - cx) * iw, zy = (xj.y - cy) * iw;
                const C4 z = c4_of(make_double2(zx, zy));
                C4 zk = {F2{1.f, 0.f}, F2{0.f, 0.f}}, base = z;
                for (int e2 = q * Q; e2 > 0; e2 >>= 1) {
                    if (e2 & 1) zk = c4_mul(zk, base);
                    base = c4_mul(base, base);
                }
                const int k1 = min(P, (q + 1) * Q);
                for (int k = q * Q; k < k1; ++k) {
                    pw[jp * P + k] = c4_pack(zk);
                    zk = c4_mul(zk, z);
                }
                if (q == 0) {
                    double v[kFfMaxNd];
                    had_v(power, zx, zy, v);
                    const double tj = t[j0 + jp];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const F2 qd = split_d(v[d] * tj);
                        qs[jp * ND + d] = make_float2(qd.h, qd.l);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PF_OUT; ++i) {
            const int o = threadIdx.x + i * PF_T;
            if (o < nout) {
                const int d = o / P, k = o - d * P;
                C4 a = acc[i];
                for (int jj = 0; jj < jn; ++jj) {
                    const float2 qv = qs[jj * ND + d];
                    const C4 z = c4_unpack(pw[jj * P + k]);
                    const F2 qf{qv.x, qv.y};
                    ff_acc(a.re, ff_mul(qf, z.re));
                    ff_acc(a.im, ff_mul(qf, z.im));
                }
                acc[i] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PF_OUT; ++i) {
        const int o = threadIdx.x + i * PF_T;
        if (o < nout) {
            const int d = o / P, k = o - d * P;
            double ax = to_d(acc[i].re), ay = to_d(acc[i].im);
            if (k > 0) {
                const double sc = -1.0 / k;
                ax *= sc;
                ay *= sc;
            }
            mp[((size_t)b * ND + d) * P + k] = make_double2(ax, ay);
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(LF_T) l2p_ff_kernel(TreeView tv, const int *leaf_box, const double2 *xs, int power,
                                                      int P, const double2 *lc, double *y) {
    extern __shared__ float4 lf_sm[];  // [ND][P] coefficients, hi + lo parts
    const int b = leaf_box[blockIdx.x];
    const int nout = ND * P;
    for (int i = threadIdx.x; i < nout; i += LF_T) lf_sm[i] = c4_pack(c4_of(lc[(size_t)b * nout + i]));
    __syncthreads();
    double cx, cy, w;
    box_geom(tv, b, cx, cy, w);
    const double iw = 1.0 / w;
    const int s = tv.start[b], e = tv.end[b];
    for (int j = s + threadIdx.x; j < e; j += LF_T) {
        const double2 xj = xs[j];
        const double vx = (xj.x - cx) * iw, vy = (xj.y - cy) * iw;
        double u[kFfMaxNd];
        had_u(power, vx, vy, u);
        F2 acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = F2{0.f, 0.f};
        const C4 v = c4_of(make_double2(vx, vy));
        C4 zk = {F2{1.f, 0.f}, F2{0.f, 0.f}};
        for (int k = 0; k < P; ++k) {
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const C4 L = c4_unpack(lf_sm[d * P + k]);
                ff_acc(acc[d], ff_mul(L.re, zk.re));
                ff_acc(acc[d], ff_neg(ff_mul(L.im, zk.im)));
            }
            zk = c4_mul(zk, v);
        }
        double sum = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) sum = fma(u[d], to_d(acc[d]), sum);
        y[j] += sum;
    }
}

}  // namespace

void p2m_ff_launch(const Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, double2 *mp,
                   cudaStream_t s) {
    const int P = f.P, nd = f.nd;
    PHS_REQUIRE(nd * P <= PF_T * PF_OUT, PHS_ERR_INVALID_ARG, "float-float P2M: nd * P above 768");
    const size_t sm = (size_t)64 * P * sizeof(float4) + (size_t)64 * nd * sizeof(float2);
    once_per_device(5, [] {
        const int lim = 100 * 1024;
        PHS_CUDA(cudaFuncSetAttribute(p2m_ff_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        PHS_CUDA(cudaFuncSetAttribute(p2m_ff_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        PHS_CUDA(cudaFuncSetAttribute(p2m_ff_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    });
    const TreeView tv = tree_view(t);
    if (nd == 4) p2m_ff_kernel<4><<<t.nleaf, PF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, P, mp);
    else if (nd == 9) p2m_ff_kernel<9><<<t.nleaf, PF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, P, mp);
    else p2m_ff_kernel<1><<<t.nleaf, PF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, f.power, P, mp);
    PHS_LAUNCH_CHECK();
}

void l2p_ff_launch(const Fmm &f, const Tree &t, const PointSet &ps, const double2 *lc, double *y, cudaStream_t s) {
    const int P = f.P, nd = f.nd;
    const size_t sm = (size_t)nd * P * sizeof(float4);
    const TreeView tv = tree_view(t);
    if (nd == 4) l2p_ff_kernel<4><<<t.nleaf, LF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), f.power, P, lc, y);
    else if (nd == 9) l2p_ff_kernel<9><<<t.nleaf, LF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), f.power, P, lc, y);
    else l2p_ff_kernel<1><<<t.nleaf, LF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), f.power, P, lc, y);
    PHS_LAUNCH_CHECK();
}

}  // namespace phs
