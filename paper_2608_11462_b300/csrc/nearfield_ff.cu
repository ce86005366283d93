// nearfield_ff.cu -- the near field of the PHS matvec (the direct sums over adjacent
// leaves of Sec. 2.1) in float-float arithmetic on the FP32 pipe.
//
// Every value is an unevaluated sum hi + lo of two floats (about 48 significant bits),
// built from error-free transformations: TwoSum (Knuth) for sums and the FMA form of
// Dekker's TwoProd for products.  On the B300 the FP32 pipe executes 64 times as many
// operations per clock as the FP64 pipe, so a pair in float-float (about 100 FP32-pipe
// instructions) costs less than the 10 FP64 instructions of the FP64 kernel, while each
// term keeps a relative error near 2^-46 instead of plain FP32's 2^-24.  That matters:
// in the Vecchia-preconditioned norm the projected system amplifies the near field's
// rounding by about 10^7 (its small eigenvalues belong to oscillating vectors whose
// near-field sums cancel), so plain FP32 sums do not converge (mode 1) while
// float-float sums do.
//
// Per pair (i, j): leaf-centred coordinates as hi + lo; dx, dy by TwoSum; s = r^2 =
// dx^2 + dy^2 by TwoProd; for even k the logarithm of s by an exact-reduction table
// method (after Tang, "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 1990): s_hi = 2^e m, m in [1, 2); j = the top 8
// bits of m's fraction; R_j = 1/(1 + (j + 1/2)/256) rounded to 9 significant bits, so
// u = m R_j - 1 is exact in one FMA (|u| < 2^-8.4, 24 significant bits); log s_hi =
// e log 2 - log R_j + log(1 + u) with the first two from hi + lo tables and
// log(1 + u) = u - u^2/2 + u^3 (1/3 - u/4 + u^2/5) (u^2 as TwoProd, truncation below
// 2^-50); log(s_hi + s_lo) adds s_lo / s_hi.  For odd k the square root r = sqrt(s) is
// refined from the approximate reciprocal square root by one correction in float-float.
// phi = r^k log r = s^(k/2) log(s) / 2 (even k) or r^k (odd k) follows by float-float
// products; the factor 1/2 is applied once per sum.  Row and column sums accumulate in
// float-float (TwoSum of the high parts, low parts added).
//
// The schedule is the symmetric one of the FP64 kernel (fmm.cu, p2p_sym_kernel): each
// leaf sums its own box (rows) and the near ranges after it in Morton order (rows and,
// systolically across the lanes sharing a source, columns into the scratch slot of the
// (leaf, range) pair); p2p_gather adds the column sums of earlier leaves.
#include <cmath>
#include <vector>

#include "ff.cuh"
#include "geom.cuh"
#include "phs_internal.cuh"

namespace phs {
namespace {
using namespace ffa;

constexpr int NF_T = kP2PThreads;
constexpr int kFfTab = 256;  // table cells of the mantissa (top 8 fraction bits)
constexpr int kFfExp = 256;  // biased FP32 exponents

__device__ float g_ff_rcp[kFfTab];    // R_j, 9 significant bits
__device__ float2 g_ff_tlog[kFfTab];  // -log R_j as (hi, lo)
__device__ float2 g_ff_eln2[kFfExp];  // (e - 127) log 2 as (hi, lo), e the biased exponent

// r = sqrt(s.h + s.l): r0 from the approximate reciprocal square root, then one
// correction (s - r0^2) / (2 r0) with s - r0^2 formed exactly by an FMA
__device__ __forceinline__ F2 ff_sqrt(F2 s) {
    if (!(s.h > 0.0f)) return {0.0f, 0.0f};
    const float y = rsqrt_approx(s.h);
    const float r0 = __fmul_rn(s.h, y);
    const float d = __fadd_rn(__fmaf_rn(-r0, r0, s.h), s.l);
    const float c = __fmul_rn(__fmul_rn(d, 0.5f), y);
    return fast_two_sum(r0, c);
}

// phi(r) (times 2 for even k) of the pair with squared distance s
template <int K>
__device__ __forceinline__ F2 ff_phi(F2 s, const float *rcp, const float2 *tlog, const float2 *eln2) {
    if constexpr (K % 2 == 0) {
        const F2 L = ff_log(s, rcp, tlog, eln2);
        if constexpr (K == 2) return ff_mul(s, L);
        else return ff_mul(ff_mul(s, s), L);
    } else {
        const F2 r = ff_sqrt(s);
        if constexpr (K == 1) return r;
        else if constexpr (K == 3) return ff_mul(s, r);
        else return ff_mul(ff_mul(s, s), r);
    }
}

template <int K>
__global__ void __launch_bounds__(NF_T) p2p_sym_ff_kernel(TreeView tv, int nleaf, const int *leaf_box,
                                                          const int *order, int *ticket, const int *near_off,
                                                          const int2 *near_rng, const int *slot_off,
                                                          const double2 *xs, const double *t, double *y,
                                                          double *scratch) {
    __shared__ float4 sxy[NF_T];  // (x hi, x lo, y hi, y lo) about the target leaf's centre
    __shared__ float2 st[NF_T];   // t hi, lo
    __shared__ float2 colp[NF_T / 32][NF_T];
    __shared__ int2 ups[kMaxUpRanges];
    __shared__ int nup, next_leaf;
    __shared__ float rcp[kFfTab];
    __shared__ float2 tlog[kFfTab];
    __shared__ float2 eln2[kFfExp];
    if constexpr (K % 2 == 0) {
        for (int i = threadIdx.x; i < kFfTab; i += NF_T) {
            rcp[i] = g_ff_rcp[i];
            tlog[i] = g_ff_tlog[i];
        }
        for (int i = threadIdx.x; i < kFfExp; i += NF_T) eln2[i] = g_ff_eln2[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double scale = (K % 2 == 0) ? 0.5 : 1.0;  // r^k log r = r^k log(r^2) / 2
    for (;;) {
        if (threadIdx.x == 0) next_leaf = atomicAdd(ticket, 1);
        __syncthreads();
        const int oi = next_leaf;
        if (oi >= nleaf) break;
        const int li = order[oi];
        const int b = leaf_box[li];
        double cx, cy, w;
        box_geom(tv, b, cx, cy, w);
        const int s = tv.start[b], e = tv.end[b];
        const int nt = e - s;
        int G = 1;
        while (G < 32 && nt * G * 2 <= NF_T) G <<= 1;
        const int sub = threadIdx.x & (G - 1);
        const int i = s + threadIdx.x / G;
        const bool act = i < e;
        const int nwarp = (nt * G + 31) >> 5;
        const bool wact = warp < nwarp;
        F2 xi{0.f, 0.f}, yi{0.f, 0.f}, ti{0.f, 0.f};
        if (act) {
            const double2 p = xs[i];
            xi = split_d(p.x - cx);
            yi = split_d(p.y - cy);
            ti = split_d(t[i]);
        }
        if (threadIdx.x == 0) {
            int n = 0, pre = 0;
            for (int r = near_off[b]; r < near_off[b + 1]; ++r) {
                const int2 rg = near_rng[r];
                if (rg.x >= e && n < kMaxUpRanges - 1) {
                    ups[n++] = make_int2(rg.x, pre);
                    pre += rg.y - rg.x;
                }
            }
            nup = n;
            ups[n] = make_int2(0, pre);
        }
        if (threadIdx.x < nt) {
            const double2 p = xs[s + threadIdx.x];
            const F2 a = split_d(p.x - cx), c = split_d(p.y - cy), tt = split_d(t[s + threadIdx.x]);
            sxy[threadIdx.x] = make_float4(a.h, a.l, c.h, c.l);
            st[threadIdx.x] = make_float2(tt.h, tt.l);
        }
        __syncthreads();
        F2 acc{0.f, 0.f};
        if (wact) {
            const int nk = (nt + G - 1) / G;
            for (int k = 0; k < nk; ++k) {
                const int jj = k * G + sub;
                if (jj < nt) {
                    const float4 q = sxy[jj];
                    const float2 tj = st[jj];
                    const F2 sq = ff_norm2(ff_sub(xi, F2{q.x, q.y}), ff_sub(yi, F2{q.z, q.w}));
                    const F2 f = ff_phi<K>(sq, rcp, tlog, eln2);
                    ff_acc(acc, ff_mul(f, F2{tj.x, tj.y}));
                }
            }
        }
        const int nu = nup, tot = ups[nu].y;
        const int slot = slot_off[li];
        int r0 = 0;
        for (int c0 = 0; c0 < tot; c0 += NF_T) {
            __syncthreads();
            {
                const int g = c0 + threadIdx.x;
                if (g < tot) {
                    int r = r0;
                    while (ups[r + 1].y <= g) ++r;
                    const int j = ups[r].x + (g - ups[r].y);
                    const double2 p = xs[j];
                    const F2 a = split_d(p.x - cx), c = split_d(p.y - cy), tt = split_d(t[j]);
                    sxy[threadIdx.x] = make_float4(a.h, a.l, c.h, c.l);
                    st[threadIdx.x] = make_float2(tt.h, tt.l);
                }
            }
            while (r0 + 1 < nu && ups[r0 + 1].y <= c0 + NF_T) ++r0;
            __syncthreads();
            const int jn = min(NF_T, tot - c0);
            if (wact) {
                // systolic column sums as in the FP64 kernel: lane u of a sub-group takes
                // column (k + u) mod S at step k and passes its running sum to lane u - 1
                const int S = 32 / G, u = lane / G;
                for (int t0 = 0; t0 < jn; t0 += 32) {
                    F2 cs{0.f, 0.f};
                    for (int k = 0; k < S; ++k) {
                        const int jj = t0 + ((k + u) & (S - 1)) * G + sub;
                        if (jj < jn) {
                            const float4 q = sxy[jj];
                            const float2 tj = st[jj];
                            const F2 sq = ff_norm2(ff_sub(xi, F2{q.x, q.y}), ff_sub(yi, F2{q.z, q.w}));
                            const F2 f = ff_phi<K>(sq, rcp, tlog, eln2);
                            ff_acc(acc, ff_mul(f, F2{tj.x, tj.y}));
                            ff_acc(cs, ff_mul(f, ti));
                        }
                        cs.h = __shfl_sync(0xffffffffu, cs.h, (lane + G) & 31);
                        cs.l = __shfl_sync(0xffffffffu, cs.l, (lane + G) & 31);
                    }
                    const int jo = t0 + u * G + sub;
                    if (jo < jn) colp[warp][jo] = make_float2(cs.h, cs.l);
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < jn; q += NF_T) {
                double sum = 0;
                for (int w2 = 0; w2 < nwarp; ++w2) sum += (double)colp[w2][q].x + (double)colp[w2][q].y;
                scratch[slot + c0 + q] = scale * sum;
            }
        }
        if (wact) {
            double a = to_d(acc);
            for (int o = G >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (sub == 0 && act) y[i] = scale * a;
        }
        __syncthreads();
    }
}

}  // namespace

// R_j, -log R_j and e log 2 for the logarithm, loaded on the current device
void upload_ff_tables() {
    std::vector<float> rc;
    std::vector<float2> tl, el;
    ffa::ff_log_tables(rc, tl, el);
    PHS_CUDA(cudaMemcpyToSymbol(g_ff_rcp, rc.data(), kFfTab * sizeof(float)));
    PHS_CUDA(cudaMemcpyToSymbol(g_ff_tlog, tl.data(), kFfTab * sizeof(float2)));
    PHS_CUDA(cudaMemcpyToSymbol(g_ff_eln2, el.data(), kFfExp * sizeof(float2)));
}

namespace {

template <int K>
void launch_ff(const Tree &t, const PointSet &ps, const double *tv_sorted, double *y, double *scratch, int *ticket,
               cudaStream_t s) {
    static int grid_cap = 0;
    if (grid_cap == 0) {
        int dev = 0, nsm = 0, per = 0;
        PHS_CUDA(cudaGetDevice(&dev));
        PHS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        PHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, p2p_sym_ff_kernel<K>, NF_T, 0));
        grid_cap = std::max(1, nsm * std::max(per, 1));
    }
    p2p_sym_ff_kernel<K><<<std::min(t.nleaf, grid_cap), NF_T, 0, s>>>(
        tree_view(t), t.nleaf, t.leaf_box.get(), t.p2p_order.get(), ticket, t.near_off.get(), t.near_rng.get(),
        t.sym_slot.get(), ps.xs.get(), tv_sorted, y, scratch);
    PHS_LAUNCH_CHECK();
}

}  // namespace

void p2p_sym_ff(const Tree &t, const PointSet &ps, int k, const double *tv_sorted, double *y, double *scratch,
                int *ticket, cudaStream_t s) {
    PHS_REQUIRE(t.sym_ok, PHS_ERR_INVALID_ARG, "the float-float near field needs leaves of at most 128 points");
    PHS_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int), s));
    switch (k) {
        case 1: launch_ff<1>(t, ps, tv_sorted, y, scratch, ticket, s); break;
        case 2: launch_ff<2>(t, ps, tv_sorted, y, scratch, ticket, s); break;
        case 3: launch_ff<3>(t, ps, tv_sorted, y, scratch, ticket, s); break;
        case 4: launch_ff<4>(t, ps, tv_sorted, y, scratch, ticket, s); break;
        default: launch_ff<5>(t, ps, tv_sorted, y, scratch, ticket, s); break;
    }
}

}  // namespace phs
