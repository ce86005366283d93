// farfield_ff.cu -- the upward and downward passes of the log-kernel FMM (Sec. 2.1) in
// float-float arithmetic on the FP32 pipe, for precision 4: P2M (outgoing expansions of
// the leaves, Eq. 2.14, with the Hadamard charges of Eq. 2.6), M2M and L2L (the shifts of
// Sec. 2.1 through their real triangular cores) and L2P (evaluation of the incoming
// expansions, Eq. 2.15, combined with the Hadamard factors).  They read and write the
// same FP64 expansions as the FP64 passes (fmm.cu p2m64_kernel, m2m64_kernel,
// l2l64_kernel, l2p64_kernel), so the M2L is unchanged; the bulk arithmetic moves to hi +
// lo floats (about 2^-46 per operation, ff.cuh).  Their rounding enters the expansion
// coefficients, so it reaches the matvec as a smooth far-field perturbation, not as the
// pairwise noise the preconditioned system amplifies.
//
// P2M, per leaf: z_j = (x_j - c)/w, q_{d,j} = v_d(z_j) t_j; a~_0 = sum_j q, a~_k = -sum_j q
// z^k / k.  Points in chunks of 64: one thread per point forms z (FP64, then split) and
// the charges (float-float), four threads per point build the powers z^k (a quarter
// each, started by binary powering) into shared memory, then each thread owns outputs
// (d, k) and sums over the chunk.  FP64 work is a few instructions per point: the FP64
// pipe has 1/64 of the FP32 pipe's rate on this part.
// L2P, per point of a leaf: y += sum_d u_d(v) Re sum_k b~_{d,k} v^k, v = (x - c)/w, the
// leaf's coefficients split once into hi + lo in shared memory, the Hadamard factors
// and the combination in float-float.
#include <algorithm>

#include "ff.cuh"
#include "geom.cuh"
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
                                                      const double *t, int P, double2 *mp) {
    extern __shared__ float4 pf_sm[];
    float4 *pw = pf_sm;                                              // [64][P] powers, hi + lo parts
    float4 *zs = pw + (size_t)64 * P;                                // [64] scaled coordinates
    float2 *qs = reinterpret_cast<float2 *>(zs + 64);                // [64][ND] charges
    const int b = leaf_box[blockIdx.x];
    double cx, cy, w, iw;
    box_geom_iw(tv, b, cx, cy, w, iw);
    const int s = tv.start[b], e = tv.end[b];
    const int nout = ND * P;
    const int Q = (P + 3) / 4;
    C4 acc[PF_OUT];
#pragma unroll
    for (int i = 0; i < PF_OUT; ++i) acc[i] = {F2{0.f, 0.f}, F2{0.f, 0.f}};
    for (int j0 = s; j0 < e; j0 += 64) {
        const int jn = min(64, e - j0);
        // one thread per point: the scaled coordinates (FP64, then split) and the
        // Hadamard charges v_d(z) t_j in float-float
        if (threadIdx.x < jn) {
            const double2 xj = xs[j0 + threadIdx.x];
            const C4 z = c4_of(make_double2((xj.x - cx) * iw, (xj.y - cy) * iw));
            zs[threadIdx.x] = c4_pack(z);
            F2 v[ND];
            had_v_ff<ND>(z.re, z.im, v);
            const F2 tj = split_d(t[j0 + threadIdx.x]);
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const F2 qd = ff_mulr(v[d], tj);
                qs[threadIdx.x * ND + d] = make_float2(qd.h, qd.l);
            }
        }
        __syncthreads();
        {  // four threads per point: powers z^k, a quarter of k each
            const int jp = threadIdx.x >> 2, q = threadIdx.x & 3;
            if (jp < jn) {
                const C4 z = c4_unpack(zs[jp]);
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
            C4 a = acc[i];
            if (k > 0) {  // times -1/k, the reciprocal in float-float (one Newton correction)
                const float kf = (float)k, h = __frcp_rn(kf);
                const F2 nr{-h, -h * __fmaf_rn(-h, kf, 1.f)};
                a = {ff_mul(a.re, nr), ff_mul(a.im, nr)};
            }
            mp[((size_t)b * ND + d) * P + k] = make_double2(to_d(a.re), to_d(a.im));
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(LF_T) l2p_ff_kernel(TreeView tv, const int *leaf_box, const double2 *xs, int P,
                                                      const double2 *lc, double *y) {
    extern __shared__ float4 lf_sm[];  // [ND][P] coefficients, hi + lo parts
    const int b = leaf_box[blockIdx.x];
    const int nout = ND * P;
    for (int i = threadIdx.x; i < nout; i += LF_T) lf_sm[i] = c4_pack(c4_of(lc[(size_t)b * nout + i]));
    __syncthreads();
    double cx, cy, w, iw;
    box_geom_iw(tv, b, cx, cy, w, iw);
    const int s = tv.start[b], e = tv.end[b];
    for (int j = s + threadIdx.x; j < e; j += LF_T) {
        const double2 xj = xs[j];
        const C4 v = c4_of(make_double2((xj.x - cx) * iw, (xj.y - cy) * iw));
        F2 acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = F2{0.f, 0.f};
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
        // sum_d u_d(v) Re L_d(v) in float-float; one FP64 add into y
        F2 u[ND];
        had_u_ff<ND>(v.re, v.im, u);
        F2 sum{0.f, 0.f};
#pragma unroll
        for (int d = 0; d < ND; ++d) ff_acc(sum, ff_mul(u[d], acc[d]));
        y[j] += to_d(sum);
    }
}

// complex conjugate
__device__ __forceinline__ C4 c4_conj(C4 a) { return {a.re, ff_neg(a.im)}; }

// M2M for the parents of one level, as fmm.cu m2m64_kernel: each child's multipole (FP64,
// split once) takes the phase e^{-i th_q k}, passes through the real lower-triangular core
// R (row l: sum over k <= l) with two interleaved accumulator pairs, takes e^{i th_q l},
// and the parent sums the children through the frame changes -- all in float-float, with
// the phases, core and frame changes pre-split; one conversion to FP64 per output.
__global__ void __launch_bounds__(PF_T) m2m_ff_kernel(TreeView tv, int b0, int nd, int P, const float2 *R,
                                                      const float4 *ph, const float2 *mix, double2 *mp) {
    extern __shared__ float4 mf_sm[];
    const int b = b0 + blockIdx.x;
    const int nc = tv.nchild[b];
    if (nc == 0) return;
    const int nout = nd * P, c0 = tv.child[b];
    float4 *ch = mf_sm;               // [4][nd][P] rotated children
    float4 *sh = mf_sm + 4 * nout;    // [4][nd][P] shifted
    float4 *phs = sh + 4 * nout;      // [4][P] phases
    float2 *Rs = reinterpret_cast<float2 *>(phs + 4 * P);  // [P][P] core
    float2 *mxs = Rs + P * P;         // [4][nd][nd] frame changes of the quadrants
    // the tables every step reads, staged once per block (the loops below would
    // otherwise wait on L2 at each dependent step)
    for (int i = threadIdx.x; i < 4 * P; i += PF_T) phs[i] = ph[i];
    for (int i = threadIdx.x; i < P * P; i += PF_T) Rs[i] = R[i];
    for (int i = threadIdx.x; i < 4 * nd * nd; i += PF_T) mxs[i] = mix[(size_t)49 * nd * nd + i];
    __syncthreads();
    for (int i = threadIdx.x; i < nc * nout; i += PF_T) {
        const int c = i / nout, k = (i - c * nout) % P;
        const C4 a = c4_of(mp[(size_t)c0 * nout + i]);
        const C4 e = c4_unpack(phs[(tv.key[c0 + c] & 3) * P + k]);
        ch[i] = c4_pack(c4_mul(a, c4_conj(e)));  // a e^{-i th k}
    }
    __syncthreads();
    const int half = (P + 1) / 2;
    for (int it = threadIdx.x; it < nc * nd * half; it += PF_T) {
        const int c = it / (nd * half), r = it - c * nd * half, d = r / half, p = r - d * half;
        const float4 *ephq = phs + (tv.key[c0 + c] & 3) * P;
        const float4 *src = ch + c * nout + d * P;
        for (int h = 0; h < 2; ++h) {
            const int l = h == 0 ? p : P - 1 - p;
            if (h == 1 && l == p) break;
            const float2 *Rr = Rs + l * P;
            F2 ax{0.f, 0.f}, ay{0.f, 0.f}, bx{0.f, 0.f}, by{0.f, 0.f};
            int k = 0;
            for (; k + 1 <= l; k += 2) {
                const float2 r0 = Rr[k], r1 = Rr[k + 1];
                const C4 m0 = c4_unpack(src[k]), m1 = c4_unpack(src[k + 1]);
                ff_acc(ax, ff_mul(F2{r0.x, r0.y}, m0.re));
                ff_acc(ay, ff_mul(F2{r0.x, r0.y}, m0.im));
                ff_acc(bx, ff_mul(F2{r1.x, r1.y}, m1.re));
                ff_acc(by, ff_mul(F2{r1.x, r1.y}, m1.im));
            }
            if (k <= l) {
                const float2 r0 = Rr[k];
                const C4 m0 = c4_unpack(src[k]);
                ff_acc(ax, ff_mul(F2{r0.x, r0.y}, m0.re));
                ff_acc(ay, ff_mul(F2{r0.x, r0.y}, m0.im));
            }
            const C4 z{ff_add(ax, bx), ff_add(ay, by)};
            sh[c * nout + d * P + l] = c4_pack(c4_mul(z, c4_unpack(ephq[l])));  // z e^{i th l}
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += PF_T) {
        const int d = o / P, l = o - d * P;
        F2 ax{0.f, 0.f}, ay{0.f, 0.f};
        for (int c = 0; c < nc; ++c) {
            const float2 *Rv = mxs + (tv.key[c0 + c] & 3) * nd * nd + d * nd;
            for (int bb = 0; bb < nd; ++bb) {
                const float2 r = Rv[bb];
                if (r.x != 0.f) {
                    const C4 v = c4_unpack(sh[c * nout + bb * P + l]);
                    ff_acc(ax, ff_mul(F2{r.x, r.y}, v.re));
                    ff_acc(ay, ff_mul(F2{r.x, r.y}, v.im));
                }
            }
        }
        mp[(size_t)b * nout + o] = make_double2(to_d(ax), to_d(ay));
    }
}

// L2L for the parents of one level, as fmm.cu l2l64_kernel: the parent's local expansion
// (split once) takes each child's phase e^{i th_q l}, passes through the real
// upper-triangular core (row m: sum over l >= m), takes e^{-i th_q m}, and mixes through
// the frame changes -- in float-float -- into the child's FP64 local expansion.
__global__ void __launch_bounds__(PF_T) l2l_ff_kernel(TreeView tv, int b0, int nd, int P, const float2 *R,
                                                      const float4 *ph, const float2 *mix, double2 *lc) {
    extern __shared__ float4 lf2_sm[];
    const int b = b0 + blockIdx.x;
    const int nc = tv.nchild[b];
    if (nc == 0) return;
    const int nout = nd * P, c0 = tv.child[b];
    float4 *y = lf2_sm;                 // [4][nd][P] rotated copies, then [nd][P] the parent's
    float4 *sh = lf2_sm + 5 * nout;     // [4][nd][P] shifted
    float4 *phs = sh + 4 * nout;        // [4][P] phases
    float2 *Rs = reinterpret_cast<float2 *>(phs + 4 * P);  // [P][P] core
    float2 *mxs = Rs + P * P;           // [4][nd][nd] frame changes of the quadrants
    for (int i = threadIdx.x; i < 4 * P; i += PF_T) phs[i] = ph[i];
    for (int i = threadIdx.x; i < P * P; i += PF_T) Rs[i] = R[i];
    for (int i = threadIdx.x; i < 4 * nd * nd; i += PF_T) mxs[i] = mix[(size_t)53 * nd * nd + i];
    for (int i = threadIdx.x; i < nout; i += PF_T) y[4 * nout + i] = c4_pack(c4_of(lc[(size_t)b * nout + i]));
    __syncthreads();
    for (int i = threadIdx.x; i < nc * nout; i += PF_T) {
        const int c = i / nout, o = i - c * nout, l = o % P;
        const C4 v = c4_unpack(y[4 * nout + o]);
        y[i] = c4_pack(c4_mul(v, c4_unpack(phs[(tv.key[c0 + c] & 3) * P + l])));  // b e^{i th l}
    }
    __syncthreads();
    const int half = (P + 1) / 2;
    for (int it = threadIdx.x; it < nc * nd * half; it += PF_T) {
        const int c = it / (nd * half), r = it - c * nd * half, d = r / half, p = r - d * half;
        const float4 *ephq = phs + (tv.key[c0 + c] & 3) * P;
        const float4 *src = y + c * nout + d * P;
        for (int h = 0; h < 2; ++h) {
            const int m = h == 0 ? p : P - 1 - p;
            if (h == 1 && m == p) break;
            const float2 *Rr = Rs + m * P;
            F2 ax{0.f, 0.f}, ay{0.f, 0.f}, bx{0.f, 0.f}, by{0.f, 0.f};
            int l = m;
            for (; l + 1 < P; l += 2) {
                const float2 r0 = Rr[l], r1 = Rr[l + 1];
                const C4 v0 = c4_unpack(src[l]), v1 = c4_unpack(src[l + 1]);
                ff_acc(ax, ff_mul(F2{r0.x, r0.y}, v0.re));
                ff_acc(ay, ff_mul(F2{r0.x, r0.y}, v0.im));
                ff_acc(bx, ff_mul(F2{r1.x, r1.y}, v1.re));
                ff_acc(by, ff_mul(F2{r1.x, r1.y}, v1.im));
            }
            if (l < P) {
                const float2 r0 = Rr[l];
                const C4 v0 = c4_unpack(src[l]);
                ff_acc(ax, ff_mul(F2{r0.x, r0.y}, v0.re));
                ff_acc(ay, ff_mul(F2{r0.x, r0.y}, v0.im));
            }
            const C4 z{ff_add(ax, bx), ff_add(ay, by)};
            sh[c * nout + d * P + m] = c4_pack(c4_mul(z, c4_conj(c4_unpack(ephq[m]))));  // z e^{-i th m}
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < nc * nout; it += PF_T) {
        const int c = it / nout, o = it - c * nout, a_ = o / P, m = o - a_ * P;
        const float2 *Ru = mxs + (tv.key[c0 + c] & 3) * nd * nd;
        F2 ax{0.f, 0.f}, ay{0.f, 0.f};
        for (int l = 0; l < nd; ++l) {
            const float2 r = Ru[l * nd + a_];
            if (r.x != 0.f) {
                const C4 v = c4_unpack(sh[c * nout + l * P + m]);
                ff_acc(ax, ff_mul(F2{r.x, r.y}, v.re));
                ff_acc(ay, ff_mul(F2{r.x, r.y}, v.im));
            }
        }
        double2 &dst = lc[(size_t)(c0 + c) * nout + o];
        dst = make_double2(dst.x + to_d(ax), dst.y + to_d(ay));
    }
}

}  // namespace

// shared memory of the shift kernels beyond their expansion buffers: phases, core, frame changes
static size_t shift_tables_smem(const Fmm &f) {
    return (size_t)4 * f.P * sizeof(float4) + (size_t)f.P * f.P * sizeof(float2) + (size_t)4 * f.nd * f.nd * sizeof(float2);
}

void m2m_ff_launch(const Fmm &f, const Tree &t, int b0, int nb, double2 *mp, cudaStream_t s) {
    // [4][nd][P] rotated + [4][nd][P] shifted (float4) + the tables: at most 112 KB (nd 9, P 61)
    const size_t sm = (size_t)8 * f.nd * f.P * 16 + shift_tables_smem(f);
    once_per_device(6, [] {
        const int lim = 128 * 1024;
        PHS_CUDA(cudaFuncSetAttribute(m2m_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        PHS_CUDA(cudaFuncSetAttribute(l2l_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    });
    m2m_ff_kernel<<<nb, PF_T, sm, s>>>(tree_view(t), b0, f.nd, f.P, f.shift_rff.get(), f.shift_phff.get(),
                                       f.mixff.get(), mp);
    PHS_LAUNCH_CHECK();
}

void l2l_ff_launch(const Fmm &f, const Tree &t, int b0, int nb, double2 *lc, cudaStream_t s) {
    const size_t sm = (size_t)9 * f.nd * f.P * 16 + shift_tables_smem(f);  // and the parent's split local expansion
    once_per_device(6, [] {
        const int lim = 128 * 1024;
        PHS_CUDA(cudaFuncSetAttribute(m2m_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        PHS_CUDA(cudaFuncSetAttribute(l2l_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    });
    l2l_ff_kernel<<<nb, PF_T, sm, s>>>(tree_view(t), b0, f.nd, f.P, f.shift_rff.get() + (size_t)f.P * f.P,
                                       f.shift_phff.get(), f.mixff.get(), lc);
    PHS_LAUNCH_CHECK();
}

void p2m_ff_launch(const Fmm &f, const Tree &t, const PointSet &ps, const double *tv_sorted, double2 *mp,
                   cudaStream_t s) {
    const int P = f.P, nd = f.nd;
    PHS_REQUIRE(nd * P <= PF_T * PF_OUT, PHS_ERR_INVALID_ARG, "float-float P2M: nd * P above 768");
    const size_t sm = (size_t)64 * P * sizeof(float4) + 64 * sizeof(float4) + (size_t)64 * nd * sizeof(float2);
    once_per_device(5, [] {
        const int lim = 100 * 1024;
        PHS_CUDA(cudaFuncSetAttribute(p2m_ff_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        PHS_CUDA(cudaFuncSetAttribute(p2m_ff_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        PHS_CUDA(cudaFuncSetAttribute(p2m_ff_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    });
    const TreeView tv = tree_view(t);
    if (nd == 4) p2m_ff_kernel<4><<<t.nleaf, PF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, P, mp);
    else if (nd == 9) p2m_ff_kernel<9><<<t.nleaf, PF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, P, mp);
    else p2m_ff_kernel<1><<<t.nleaf, PF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), tv_sorted, P, mp);
    PHS_LAUNCH_CHECK();
}

void l2p_ff_launch(const Fmm &f, const Tree &t, const PointSet &ps, const double2 *lc, double *y, cudaStream_t s) {
    const int P = f.P, nd = f.nd;
    const size_t sm = (size_t)nd * P * sizeof(float4);
    const TreeView tv = tree_view(t);
    if (nd == 4) l2p_ff_kernel<4><<<t.nleaf, LF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), P, lc, y);
    else if (nd == 9) l2p_ff_kernel<9><<<t.nleaf, LF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), P, lc, y);
    else l2p_ff_kernel<1><<<t.nleaf, LF_T, sm, s>>>(tv, t.leaf_box.get(), ps.xs.get(), P, lc, y);
    PHS_LAUNCH_CHECK();
}

}  // namespace phs
