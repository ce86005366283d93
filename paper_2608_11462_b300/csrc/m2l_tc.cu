// m2l_tc.cu -- multipole-to-local translations of the log-kernel FMM (Sec. 2.1,
// Eqs. 2.13-2.15) on the 5th-generation tensor cores.
//
// For a target box t the M2L is a sum over its interaction (V) list, one source per
// offset class c:
//     b_t[d][l] = sum_c sum_k T_c[l][k] * (S_c a_src(c))[d][k]  (+ log w * sum_c (S_c a)[d][0] at l = 0)
// with T_c the level-invariant class operator (box units) and S_c the integer frame
// change of the box-local Hadamard densities.  Written over all classes this is one
// dense contraction per tile of targets:  D[rows][l] = sum_(c,k') A_c[rows][k'] B_c[k'][l],
// rows = (density d, re/im, target), k' = (coefficient k, re/im), which runs on the
// tensor cores exactly in fixed point:
//   * every input is an integer X (|X| <= 2^47) times a power of two: A rows share the
//     per-target exponent E_t, B columns the per-column exponent F_l; the factor 2^floor(k/2)
//     moves from B to A so both operands are flat in k;
//   * X is split into six balanced base-256 digits (each in [-128, 128], exact in bf16);
//   * digit planes i of A and j of B with i + j <= 5 are multiplied by tcgen05.mma and
//     accumulated per diagonal g = i + j in FP32 in tensor memory.  All products are
//     integers and every diagonal sum stays far below 2^24 for the digit statistics of
//     this operator, so the accumulation is exact; the dropped planes i + j >= 6 weigh
//     below 2^-48 of the operands;
//   * the epilogue recombines sum_g D_g 256^(5-g) in integer arithmetic and scales it
//     once per output in FP64.
// Complex products use the real form: row (re) = [Re a_k, -Im a_k], row (im) =
// [Im a_k, Re a_k] against column l = [Re T_lk, Im T_lk].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <cuda_bf16.h>
#include <vector>

#include "geom.cuh"
#include "phs_internal.cuh"
#include "tc.cuh"

namespace phs {

constexpr int TC_M = 128;                    // rows per tile (one TMEM lane each)
constexpr int TC_KC = 48;                    // K columns per step
constexpr int TC_KCC = TC_KC / 2;            // complex coefficients per step
constexpr int TC_SW4 = 12, TC_SW9 = 11;      // staging warps (nd = 4, nd = 9); one more warp issues the MMAs
template <int ND>
__host__ __device__ constexpr int tc_staging_warps() { return ND == 4 ? TC_SW4 : TC_SW9; }
template <int ND>
__host__ __device__ constexpr int tc_threads() { return 32 * (tc_staging_warps<ND>() + 1); }
constexpr int TC_A_PLANE = TC_M * TC_KC * 2; // bytes of one A digit plane

bool m2l_tc_supported(int nd, int P) { return (nd == 4 || nd == 9) && P <= 64; }

struct TcArgs {
    TreeView tv;
    const int *tgt;           // target boxes, 16 per tile in list order
    int ntgt;
    const int *v_off, *v_src;
    const unsigned char *v_cls;
    int P, npad, nch, power;
    const longlong2 *mpx;     // multipoles in per-box fixed point (tc_fixed_kernel)
    double2 *lc;
    const int *mexp, *gexp, *S, *F;
    const int2 *off;          // nd = 4: offset (ox, oy) of each class in box units
    const uint16_t *bplanes;  // [49][nch][NPL][npad x 48], core-matrix order
    int *err;
    uint64_t wait_ns;         // limit of the pipeline waits of the main loop
    int probe;                // nonzero: the issuer first waits on a barrier nothing completes
};

// One warp per box: the exponent bound mexp = max over (b, k, re/im) of the exponent of
// |a_b[k]| 2^floor(k/2) (so |a_b[k]| 2^floor(k/2) < 2^mexp), then the box's multipoles are
// rewritten in place as integers X = round(a_b[k] 2^(53 - mexp + floor(k/2))), |X| <= 2^53.
// A target later needs them at its own finer scale: one rounding right shift.
__global__ void tc_fixed_kernel(double2 *mp, int nbox, int nd, int P, int *mexp) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= nbox) return;
    const int lane = threadIdx.x & 31;
    double2 *mb = mp + (size_t)b * nd * P;
    int m = -100000;
    for (int i = lane; i < nd * P; i += 32) {
        const int k = i % P;
        const double2 v = mb[i];
        const int ex = (int)(((unsigned long long)__double_as_longlong(v.x) >> 52) & 0x7FF);
        const int ey = (int)(((unsigned long long)__double_as_longlong(v.y) >> 52) & 0x7FF);
        if (ex) m = max(m, ex - 1023 + 1 + (k >> 1));
        if (ey) m = max(m, ey - 1023 + 1 + (k >> 1));
    }
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) mexp[b] = m;
    longlong2 *xb = reinterpret_cast<longlong2 *>(mb);
    for (int i = lane; i < nd * P; i += 32) {
        const int k = i % P;
        const double2 v = mb[i];
        const int sh = 53 - m + (k >> 1);
        xb[i] = make_longlong2(to_fixed(v.x, sh), to_fixed(v.y, sh));
    }
}

template <int ND>
struct TcLayout {
    static constexpr int TPB = TC_M / (2 * ND);  // targets per tile
    int bplane, bstep;
    size_t off_B, off_vsrc, off_vsh, off_cflag, off_clist, off_E, off_lsum, off_mbar, off_misc, off_coff, total;
    __host__ __device__ TcLayout(int npad) {
        bplane = npad * TC_KC * 2;
        bstep = TC_NPL * bplane;
        off_B = (size_t)2 * TC_NPL * TC_A_PLANE;
        off_vsrc = off_B + (size_t)2 * bstep;
        off_vsh = off_vsrc + (size_t)TPB * TC_NCLS * 4;
        off_cflag = off_vsh + (((size_t)TPB * TC_NCLS + 15) & ~(size_t)15);
        off_clist = off_cflag + TC_NCLS * 4;
        off_E = off_clist + TC_NCLS * 4;                 // [TPB][ND] row exponents, then [TPB] minimum
        off_lsum = (off_E + (size_t)TPB * (ND + 1) * 4 + 7) & ~(size_t)7;
        off_mbar = off_lsum + (size_t)TPB * ND * 8;
        off_misc = off_mbar + 7 * 8;
        off_coff = off_misc + 16;                        // [49] class offsets (nd = 4)
        total = off_coff + (size_t)TC_NCLS * 8;
    }
};

// staging item -> (target, coefficient); for 16-box tiles a warp spans 8 targets x 4
// coefficients (bank-conflict-free shared stores), otherwise targets run fastest
template <int TPB>
__device__ __forceinline__ void item_of(int it, int &ti, int &kk) {
    if constexpr (TPB == 16) {
        ti = (it & 7) | (((it >> 3) / TC_KCC) << 3);
        kk = (it >> 3) % TC_KCC;
    } else {
        ti = it % TPB;
        kk = it / TPB;
    }
}

// Warp roles: warps 0 .. NSW-1 stage A (one mbarrier arrival per thread on full[u] when
// buffer u is written), warp NSW (lane 0) copies B by TMA bulk copies and issues the MMAs,
// committing to empty[u] when they have read buffer u.  No block-wide barrier inside the
// loop; every wait is bounded and a timeout ends all roles through the abort flag.
template <int ND>
__global__ void __launch_bounds__(tc_threads<ND>(), 1) m2l_tc_kernel(TcArgs a) {
    using L = TcLayout<ND>;
    constexpr int TPB = L::TPB;
    constexpr int NSW = tc_staging_warps<ND>();
    constexpr int TC_T = tc_threads<ND>();
    constexpr int NST = NSW * 32;  // staging threads
    extern __shared__ __align__(1024) unsigned char sm[];
    const L lay(a.npad);
    unsigned char *Abuf = sm;
    unsigned char *Bbuf = sm + lay.off_B;
    int *vsrc = reinterpret_cast<int *>(sm + lay.off_vsrc);
    unsigned char *vsh = sm + lay.off_vsh;  // [TPB][49] shift from the source's scale to the target's
    int *cflag = reinterpret_cast<int *>(sm + lay.off_cflag);
    int *clist = reinterpret_cast<int *>(sm + lay.off_clist);
    int *Et = reinterpret_cast<int *>(sm + lay.off_E);
    long long *lsum = reinterpret_cast<long long *>(sm + lay.off_lsum);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + lay.off_mbar);  // empty[2], bfull[2], done, full[2]
    uint32_t *misc = reinterpret_cast<uint32_t *>(sm + lay.off_misc);  // tmem base, ncls, abort
    int2 *coff = reinterpret_cast<int2 *>(sm + lay.off_coff);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tb0 = blockIdx.x * TPB;  // first list position of the tile
    const int nt = min(TPB, a.ntgt - tb0);

    // ---- prologue: interaction lists of the tile, exponents, zeroed operand buffers
    for (int i = tid; i < TPB * TC_NCLS; i += TC_T) vsrc[i] = -1;
    for (int i = tid; i < TC_NCLS; i += TC_T) {
        cflag[i] = 0;
        coff[i] = ND == 4 ? a.off[i] : make_int2(0, 0);
    }
    for (int i = tid; i < TPB * ND; i += TC_T) lsum[i] = 0;
    {
        uint4 *z = reinterpret_cast<uint4 *>(Abuf);
        const int n16 = 2 * TC_NPL * TC_A_PLANE / 16;
        for (int i = tid; i < n16; i += TC_T) z[i] = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        for (int i = 0; i < 5; ++i) tc::mbar_init(&mbar[i], 1);
        tc::mbar_init(&mbar[5], NST);
        tc::mbar_init(&mbar[6], NST);
        tc::fence_mbar_init();
        misc[2] = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&misc[0], 512);
        tc::tmem_relinquish();
    }
    __syncthreads();
    // row exponents: |(S_c a)_d[k] 2^floor(k/2)| < 2^(E[t][d] - 1) over the interaction
    // list; one warp per target, lanes over its list
    for (int ti = warp; ti < nt; ti += TC_T / 32) {
        const int b = a.tgt[tb0 + ti];
        const int v0 = a.v_off[b], v1 = a.v_off[b + 1];
        int e[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) e[d] = -100000;
        for (int v = v0 + lane; v < v1; v += 32) {
            const int c = a.v_cls[v], src = a.v_src[v];
            vsrc[ti * TC_NCLS + c] = src;
            const int me = a.mexp[src];
#pragma unroll
            for (int d = 0; d < ND; ++d) e[d] = max(e[d], me + a.gexp[c * ND + d]);
            cflag[c] = 1;
        }
        int emin = 1 << 30;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            for (int o = 16; o; o >>= 1) e[d] = max(e[d], __shfl_xor_sync(0xffffffffu, e[d], o));
            if (lane == 0) Et[ti * ND + d] = e[d] + 1;
            emin = min(emin, e[d] + 1);
        }
        if (lane == 0) Et[TPB * ND + ti] = emin;
        // emin >= mexp[src] + 1 for every source of the list, so the shift is >= 1
        for (int v = v0 + lane; v < v1; v += 32)
            vsh[ti * TC_NCLS + a.v_cls[v]] = (unsigned char)min(emin - a.mexp[a.v_src[v]], 63);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
        int n = 0;
        for (int c = 0; c < TC_NCLS; ++c)
            if (cflag[c]) clist[n++] = c;
        misc[1] = (uint32_t)n;
    }
    __syncthreads();
    const uint32_t tmem = misc[0];
    const int nsteps = (int)misc[1] * a.nch;
    const int pl_per_mma = 256 / a.npad;  // B planes per MMA: N = planes x npad <= 256
    const uint64_t adesc0 = tc::make_desc_kmajor(tc::smem_u32(Abuf), 128, (TC_KC / 8) * 128);
    const uint64_t bdesc0 = tc::make_desc_kmajor(tc::smem_u32(Bbuf), 128, (TC_KC / 8) * 128);
    // one staging item per staging thread and step when TPB x 24 == NST: its sources for
    // the next step are prefetched into registers
    constexpr bool kPrefetch = TPB * TC_KCC == NST;
    longlong2 mpre[ND];
    int emin_r = 0, dsh_r[ND];  // the item's exponents (fixed target), kept in registers
    if constexpr (kPrefetch) {
        int ti, kk;
        item_of<TPB>(tid, ti, kk);
        if (tid < NST && ti < nt) {
            emin_r = Et[TPB * ND + ti];
#pragma unroll
            for (int d = 0; d < ND; ++d) dsh_r[d] = Et[ti * ND + d] - emin_r;
        }
        if (nsteps > 0 && tid < NST) {
            const int k0 = kk;  // step 0: first K chunk of the first class
            const int src0 = (ti < nt && k0 < a.P) ? vsrc[ti * TC_NCLS + clist[0]] : -1;
            if (src0 >= 0) {
#pragma unroll
                for (int b = 0; b < ND; ++b) mpre[b] = a.mpx[((size_t)src0 * ND + b) * a.P + k0];
            }
        }
    }
    uint32_t inited = 0;     // accumulators written at least once (issuer)
    int bpend[2] = {-1, -1};  // parity of an operator copy not yet waited for (issuer)
    const bool issuer = warp == NSW && lane == 0;
    auto copy_b = [&](int s2) {
        const int u2 = s2 & 1;
        const int c2 = clist[s2 / a.nch], h2 = s2 % a.nch;
        bpend[u2] = (s2 >> 1) & 1;
        tc::mbar_arrive_expect_tx(&mbar[2 + u2], (uint32_t)lay.bstep);
        tc::bulk_g2s(Bbuf + (size_t)u2 * lay.bstep,
                     reinterpret_cast<const unsigned char *>(a.bplanes) + ((size_t)c2 * a.nch + h2) * lay.bstep,
                     (uint32_t)lay.bstep, &mbar[2 + u2]);
    };

    // ---- main loop: one step = (class, K chunk)
    if (warp < NSW) {
        for (int s = 0; s < nsteps; ++s) {
            const int u = s & 1;
            const int c = clist[s / a.nch], h = s % a.nch;
            if (misc[2]) break;
            if (s >= 2 && !tc::mbar_wait(&mbar[u], (uint32_t)(((s >> 1) - 1) & 1), a.wait_ns)) {
                misc[2] = 1;
                break;
            }
            // stage A: item = (coefficient kk, target ti); rows (2d + part) * TPB + ti.  With
            // TPB = 16 a warp covers 8 targets x 4 coefficients, so its 32 stores of a plane
            // hit 32 different banks.
            unsigned char *Au = Abuf + (size_t)u * TC_NPL * TC_A_PLANE;
            const int *Sc = a.S + c * ND * ND;
            const int2 cls_off = coff[c];
            for (int it = tid; it < TPB * TC_KCC; it += NST) {
                int ti, kk;
                item_of<TPB>(it, ti, kk);
                const int k = h * TC_KCC + kk;
                const int src = (ti < nt && k < a.P) ? vsrc[ti * TC_NCLS + c] : -1;
                const uint32_t colb = (uint32_t)((kk >> 2) * 128 + (kk & 3) * 4);  // byte offset of column 2kk in a row
                longlong2 m[ND];
                if constexpr (kPrefetch) {
    #pragma unroll
                    for (int b = 0; b < ND; ++b) m[b] = mpre[b];
                    // the next step's sources load while this step converts
                    if (s + 1 < nsteps) {
                        const int c1 = clist[(s + 1) / a.nch], k1 = ((s + 1) % a.nch) * TC_KCC + kk;
                        const int src1 = (ti < nt && k1 < a.P) ? vsrc[ti * TC_NCLS + c1] : -1;
                        if (src1 >= 0) {
    #pragma unroll
                            for (int b = 0; b < ND; ++b) mpre[b] = a.mpx[((size_t)src1 * ND + b) * a.P + k1];
                        }
                    }
                } else if (src >= 0) {
    #pragma unroll
                    for (int b = 0; b < ND; ++b) m[b] = a.mpx[((size_t)src * ND + b) * a.P + k];
                }
                if (src < 0) {
                    for (int g2 = 0; g2 < 2 * ND; ++g2) {
                        const int row = g2 * TPB + ti;
                        const uint32_t off = (uint32_t)((row >> 3) * (TC_KC / 8) * 128 + (row & 7) * 16) + colb;
    #pragma unroll
                        for (int i = 0; i < TC_NPL; ++i) *reinterpret_cast<uint32_t *>(Au + i * TC_A_PLANE + off) = 0u;
                    }
                    continue;
                }
                // nd = 4: the sources (|X| <= 2^53) mix exactly at their own scale (row sums
                // of |S| are at most 1 + 6 + 6 + 18 = 31, so |y| < 2^58) and each row rounds
                // once, by the shift to the target's finest scale plus its own.  nd = 9 (row
                // sums up to 2^10): the sources first come to the finest row scale (one
                // rounding shift), then mix, then each row rounds to its own exponent.
                constexpr bool kOneShift = ND == 4;
                const int emin = kPrefetch ? emin_r : Et[TPB * ND + ti];
                const int sh2 = vsh[ti * TC_NCLS + c];
                const int s0 = kOneShift ? sh2 : 0;  // shift still owed to the finest row scale
                long long xr[ND], xi[ND];
#pragma unroll
                for (int b = 0; b < ND; ++b) {
                    xr[b] = kOneShift ? m[b].x : rshift_round(m[b].x, sh2);
                    xi[b] = kOneShift ? m[b].y : rshift_round(m[b].y, sh2);
                }
                long long yrs[ND], yis[ND];
                if constexpr (ND == 4) {
                    // v = [1, a, x, y] (a = x^2 + y^2) about the target centre: S = I plus
                    // row 1 = (|o|^2, ., 2 ox, 2 oy), row 2 = (ox, ...), row 3 = (oy, ...)
                    const int2 o = cls_off;
                    const long long o2 = (long long)o.x * o.x + (long long)o.y * o.y;
                    yrs[0] = xr[0];
                    yis[0] = xi[0];
                    yrs[1] = xr[1] + 2ll * o.x * xr[2] + 2ll * o.y * xr[3] + o2 * xr[0];
                    yis[1] = xi[1] + 2ll * o.x * xi[2] + 2ll * o.y * xi[3] + o2 * xi[0];
                    yrs[2] = xr[2] + (long long)o.x * xr[0];
                    yis[2] = xi[2] + (long long)o.x * xi[0];
                    yrs[3] = xr[3] + (long long)o.y * xr[0];
                    yis[3] = xi[3] + (long long)o.y * xi[0];
                } else {
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        long long yr = 0, yi = 0;
#pragma unroll
                        for (int b = 0; b < ND; ++b) {
                            const int sv = Sc[d * ND + b];
                            if (sv) {
                                yr += (long long)sv * xr[b];
                                yi += (long long)sv * xi[b];
                            }
                        }
                        yrs[d] = yr;
                        yis[d] = yi;
                    }
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const int dsh = kPrefetch ? dsh_r[d] : Et[ti * ND + d] - emin;
                    // shifts of 63 round |y| < 2^58 to 0, as every larger one would
                    if (k == 0) lsum[ti * ND + d] += s0 + dsh > 0 ? rshift_round(yrs[d], min(s0 + dsh, 63)) : yrs[d];
                    const int s1 = min(s0 + TC_GB + dsh, 63);
                    const long long yr = rshift_round(yrs[d], s1);
                    const long long yi = rshift_round(yis[d], s1);
                    float dr[TC_NPL], di[TC_NPL];
                    digits_f(yr, dr);
                    digits_f(yi, di);
                    const int row_re = (2 * d) * TPB + ti, row_im = row_re + TPB;
                    const uint32_t off_re = (uint32_t)((row_re >> 3) * (TC_KC / 8) * 128 + (row_re & 7) * 16) + colb;
                    const uint32_t off_im = (uint32_t)((row_im >> 3) * (TC_KC / 8) * 128 + (row_im & 7) * 16) + colb;
    #pragma unroll
                    for (int i = 0; i < TC_NPL; ++i) {
                        *reinterpret_cast<uint32_t *>(Au + i * TC_A_PLANE + off_re) = pack_bf16(dr[i], -di[i]);
                        *reinterpret_cast<uint32_t *>(Au + i * TC_A_PLANE + off_im) = pack_bf16(di[i], dr[i]);
                    }
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&mbar[5 + u]);
        }
    } else if (issuer && nsteps > 0) {
        // test of the timeout path: before anything is issued, wait (bounded) for the
        // "done" barrier, which only this thread's final commit completes, so the wait
        // expires, the pass aborts, and the drain below finds no work in flight
        if (a.probe && !tc::mbar_wait(&mbar[4], 0, a.wait_ns)) misc[2] = 1;
        if (!misc[2]) {
            copy_b(0);
            if (nsteps > 1) copy_b(1);
        }
        for (int s = 0; s < nsteps; ++s) {
            const int u = s & 1;
            if (misc[2]) break;
            if (!tc::mbar_wait(&mbar[5 + u], (uint32_t)((s >> 1) & 1), a.wait_ns) ||
                !tc::mbar_wait(&mbar[2 + u], (uint32_t)((s >> 1) & 1), a.wait_ns)) {
                misc[2] = 1;
                break;
            }
            bpend[u] = -1;
            tc::fence_after_sync();
            // descriptor start addresses advance by (byte offset >> 4) in the low field
            const uint64_t au = adesc0 + (uint64_t)((u * TC_NPL * TC_A_PLANE) >> 4);
            const uint64_t bu = bdesc0 + (uint64_t)((u * lay.bstep) >> 4);
            // The B digit planes lie one after another along N and the accumulators of the
            // diagonals one after another along the TMEM columns, so a single MMA of A plane
            // i against B planes j0 .. j0 + nj - 1 (N = nj x npad <= 256) adds each product
            // A_i B_j to its own diagonal i + j.  Plane i = 0 comes first, and its MMAs cover
            // every diagonal once, so an MMA's diagonals are all fresh or all accumulated.
#pragma unroll 1
            for (int ks = 0; ks < TC_KC / 16; ++ks) {
#pragma unroll
                for (int i = 0; i < TC_NPL; ++i) {
                    const uint64_t ad = au + (uint64_t)((i * TC_A_PLANE + ks * 256) >> 4);
                    for (int j0 = 0; j0 < TC_NPL - i; j0 += pl_per_mma) {
                        const int nj = min(pl_per_mma, TC_NPL - i - j0);
                        const int g = i + j0;
                        const uint64_t bd = bu + (uint64_t)((j0 * lay.bplane + ks * 256) >> 4);
                        tc::mma_bf16(tmem + (uint32_t)(g * a.npad), ad, bd, tc::idesc_bf16_f32(TC_M, nj * a.npad),
                                     (inited >> g) & 1);
                        inited |= ((1u << nj) - 1) << g;
                    }
                }
            }
            tc::mma_commit(&mbar[u]);
            // the operator of step s + 1 goes into the buffer step s - 1 read
            if (s >= 1 && s + 1 < nsteps) {
                if (!tc::mbar_wait(&mbar[u ^ 1], (uint32_t)(((s - 1) >> 1) & 1), a.wait_ns)) {
                    misc[2] = 1;
                    break;
                }
                copy_b(s + 1);
            }
        }
    }
    // Drain: whatever the main loop's limit, the MMAs issued and the operator copies in
    // flight are waited for with the fixed 2 s limit before TMEM is released and the CTA
    // exits, so an early give-up never leaves asynchronous work behind.
    __syncthreads();
    const bool aborted = misc[2] != 0;
    bool ok = !aborted;
    if (nsteps > 0) {
        if (issuer) tc::mma_commit(&mbar[4]);
        ok = tc::mbar_wait(&mbar[4], 0, TC_TIMEOUT_NS) && ok;
    }
    if (issuer) {  // operator copies still in flight after an abort land before the CTA exits
        for (int u = 0; u < 2; ++u)
            if (bpend[u] >= 0 && !tc::mbar_wait(&mbar[2 + u], (uint32_t)bpend[u], TC_TIMEOUT_NS)) ok = false;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) atomicExch(a.err, 1);
    __syncthreads();
    ok = !misc[2] && ok;
    tc::fence_after_sync();

    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, 16-column chunks w / 4, w / 4 + WQ, ...
    constexpr int WQ = (TC_T / 32) / 4;  // epilogue warps per TMEM lane quadrant
    if (ok && warp < 4 * WQ) {
        const int q = warp & 3, cg = warp >> 2;
        const int r = 32 * q + lane;
        const int grp = r / TPB, ti = r - grp * TPB;
        const bool valid = grp < 2 * ND && ti < nt;
        const int d = grp >> 1, part = grp & 1;
        int E = 0;
        double logw = 0, wpow = 1, l0 = 0;
        double2 *dst = nullptr;
        if (valid) {
            const int b = a.tgt[tb0 + ti];
            const double w = box_width(a.tv.R, a.tv.level[b]);
            logw = log(w);
            for (int i = 0; i < a.power; ++i) wpow *= w;
            E = Et[ti * ND + d];
            l0 = ldexp((double)lsum[ti * ND + d], E - TC_QB - TC_GB);
            dst = a.lc + ((size_t)b * ND + d) * a.P;
        }
        for (int chk = cg; chk < a.npad / 16; chk += WQ) {
            uint32_t v[TC_NPL][16];
            if (nsteps > 0) {
#pragma unroll
                for (int g = 0; g < TC_NPL; ++g)
                    tc::tmem_ld16_nowait(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * a.npad + chk * 16), v[g]);
                tc::tmem_wait_ld();
            }
            if (valid) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int l = chk * 16 + j;
                    if (l < a.P) {
                        double val = 0;
                        if (nsteps > 0) {
                            long long dg[TC_NPL];
#pragma unroll
                            for (int g = 0; g < TC_NPL; ++g)
                                dg[g] = (long long)__float2int_rn(__uint_as_float(v[g][j]));
                            const long long hi = (dg[0] << 16) + (dg[1] << 8) + dg[2];
                            const long long lo = (dg[3] << 16) + (dg[4] << 8) + dg[5];
                            val = ldexp(fma((double)hi, 16777216.0, (double)lo),
                                        E + a.F[l] - (2 * TC_QB - TC_DB * (TC_NPL - 1)));
                            if (l == 0 && part == 0) val += logw * l0;
                        }
                        val *= wpow;
                        if (part == 0) dst[l].x = val;
                        else dst[l].y = val;
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- host side
static inline uint16_t bf16_bits_of_int(int v) {
    const float f = (float)v;  // |v| <= 128: exact in bf16
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

// Integer frame changes (slots 0..48 of the mix table) and their growth bound (the rows
// of a target convert at the finest row scale, so the largest growth may add at most 10
// bits to the 52-bit converted sources: |y| < 2^62).  Shared with the distance kernel's
// tensor-core M2L (cheb_tc.cu).
void tc_integer_frames(int nd, const std::vector<long double> &mix, std::vector<int> &S, std::vector<int> &gexp) {
    S.assign((size_t)TC_NCLS * nd * nd, 0);
    gexp.assign((size_t)TC_NCLS * nd, 0);
    for (int c = 0; c < TC_NCLS; ++c) {
        for (int d = 0; d < nd; ++d) {
            long long rs = 0;
            for (int b = 0; b < nd; ++b) {
                const long double v = mix[((size_t)c * nd + d) * nd + b];
                const long long iv = std::llround(v);
                PHS_REQUIRE(std::fabs(v - (long double)iv) < 1e-6L, PHS_ERR_INVALID_ARG,
                            "tensor-core M2L: frame change is not integral");
                S[((size_t)c * nd + d) * nd + b] = (int)iv;
                rs += std::llabs(iv);
            }
            int g = 0;
            while ((1ll << g) < std::max(rs, 1ll)) ++g;
            PHS_REQUIRE(g <= 10, PHS_ERR_INVALID_ARG, "tensor-core M2L: frame-change growth above 2^10");
            gexp[(size_t)c * nd + d] = g;
        }
    }
}

struct TcHostTables {
    std::vector<uint16_t> B;
    std::vector<int> F, S, gexp;
    std::vector<int2> off;
};
static TcHostTables build_tc_tables(int P, int nd, const std::vector<long double> &ops_re,
                                    const std::vector<long double> &ops_im, const std::vector<long double> &mix);

void m2l_tc_setup(Fmm &f, const std::vector<long double> &ops_re, const std::vector<long double> &ops_im,
                  const std::vector<long double> &mix, cudaStream_t s) {
    const int P = f.P, nd = f.nd;
    PHS_REQUIRE(m2l_tc_supported(nd, P), PHS_ERR_INVALID_ARG, "tensor-core M2L needs nd in {4, 9} and P <= 64");
    f.tc_npad = (P + 15) / 16 * 16;
    f.tc_nch = (2 * P + TC_KC - 1) / TC_KC;
    // the tables depend on (P, nd) only: built once per process
    static std::mutex mu;
    static std::map<std::pair<int, int>, TcHostTables> cache;
    const TcHostTables *tab;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find({P, nd});
        if (it == cache.end()) it = cache.emplace(std::make_pair(P, nd), build_tc_tables(P, nd, ops_re, ops_im, mix)).first;
        tab = &it->second;
    }
    f.tc_off.alloc(TC_NCLS);
    f.tc_b.alloc(tab->B.size());
    f.tc_F.alloc(P);
    f.tc_S.alloc(tab->S.size());
    f.tc_gexp.alloc(tab->gexp.size());
    f.tc_err.alloc(1);
    PHS_CUDA(cudaMemcpyAsync(f.tc_off.get(), tab->off.data(), TC_NCLS * sizeof(int2), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.tc_b.get(), tab->B.data(), tab->B.size() * 2, cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.tc_F.get(), tab->F.data(), P * sizeof(int), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.tc_S.get(), tab->S.data(), tab->S.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.tc_gexp.get(), tab->gexp.data(), tab->gexp.size() * sizeof(int), cudaMemcpyHostToDevice,
                             s));
    PHS_CUDA(cudaMemsetAsync(f.tc_err.get(), 0, sizeof(int), s));
    PHS_CUDA(cudaStreamSynchronize(s));
    f.tc = true;
}

static TcHostTables build_tc_tables(int P, int nd, const std::vector<long double> &ops_re,
                                    const std::vector<long double> &ops_im, const std::vector<long double> &mix) {
    TcHostTables out;
    const int npad = (P + 15) / 16 * 16, nch = (2 * P + TC_KC - 1) / TC_KC;
    auto opv = [&](const std::vector<long double> &o, int c, int l, int k) -> long double {
        return o[((size_t)(8 + c) * P + l) * P + k];
    };
    auto valid_cls = [](int c) {
        const int dx = c / 7 - 3, dy = c % 7 - 3;
        return std::abs(dx) > 1 || std::abs(dy) > 1;
    };
    // column exponents: |T_c[l][k] 2^-floor(k/2)| < 2^F_l over all classes
    std::vector<int> F(P, -100000);
    for (int c = 0; c < TC_NCLS; ++c) {
        if (!valid_cls(c)) continue;
        for (int l = 0; l < P; ++l)
            for (int k = 0; k < P; ++k)
                for (int part = 0; part < 2; ++part) {
                    const long double v = (part ? opv(ops_im, c, l, k) : opv(ops_re, c, l, k)) / std::ldexp(1.0L, k >> 1);
                    if (v == 0) continue;
                    int e;
                    std::frexp(v, &e);
                    F[l] = std::max(F[l], e);
                }
    }
    const size_t plane = (size_t)npad * TC_KC;
    std::vector<uint16_t> B((size_t)TC_NCLS * nch * TC_NPL * plane, 0);
    for (int c = 0; c < TC_NCLS; ++c) {
        if (!valid_cls(c)) continue;
        for (int h = 0; h < nch; ++h)
            for (int l = 0; l < P; ++l)
                for (int kc = 0; kc < TC_KC; ++kc) {
                    const int kp = h * TC_KC + kc, k = kp >> 1, part = kp & 1;
                    if (k >= P) continue;
                    const long double v = (part ? opv(ops_im, c, l, k) : opv(ops_re, c, l, k)) / std::ldexp(1.0L, k >> 1);
                    long long X = std::llround(std::ldexp(v, TC_QB - F[l]));
                    int dig[TC_NPL];
                    for (int i = TC_NPL - 1; i >= 1; --i) {
                        const int q = (int)((X + 128) & 255) - 128;
                        dig[i] = q;
                        X = (X - q) >> TC_DB;
                    }
                    dig[0] = (int)X;
                    PHS_REQUIRE(std::abs(dig[0]) <= 128, PHS_ERR_INVALID_ARG, "tensor-core M2L: operator digit overflow");
                    const size_t boff = (size_t)l / 8 * (TC_KC / 8) * 64 + (size_t)kc / 8 * 64 + (l % 8) * 8 + kc % 8;
                    for (int j = 0; j < TC_NPL; ++j)
                        B[(((size_t)c * nch + h) * TC_NPL + j) * plane + boff] = bf16_bits_of_int(dig[j]);
                }
    }
    std::vector<int> S, gexp;
    tc_integer_frames(nd, mix, S, gexp);
    // nd = 4: the frame change has the closed form of [1, a, x, y] shifted by o = (ox, oy)
    std::vector<int2> off(TC_NCLS, make_int2(0, 0));
    if (nd == 4) {
        for (int c = 0; c < TC_NCLS; ++c) {
            if (!valid_cls(c)) continue;
            const int *Sm = S.data() + (size_t)c * 16;
            const int ox = Sm[2 * 4 + 0], oy = Sm[3 * 4 + 0];
            const int want[16] = {1, 0, 0, 0, ox * ox + oy * oy, 1, 2 * ox, 2 * oy, ox, 0, 1, 0, oy, 0, 0, 1};
            for (int i = 0; i < 16; ++i)
                PHS_REQUIRE(Sm[i] == want[i], PHS_ERR_INVALID_ARG, "tensor-core M2L: unexpected frame change");
            off[c] = make_int2(ox, oy);
        }
    }
    out.B = std::move(B);
    out.F = std::move(F);
    out.S = std::move(S);
    out.gexp = std::move(gexp);
    out.off = std::move(off);
    return out;
}

template <int ND>
static void launch_tc(Fmm &f, const Tree &t, double2 *mp, double2 *lc, int b0, cudaStream_t s) {
    const TcLayout<ND> lay(f.tc_npad);
    static bool attr_set = false;
    if (!attr_set) {
        PHS_CUDA(cudaFuncSetAttribute(m2l_tc_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448));
        attr_set = true;
    }
    PHS_REQUIRE(lay.total <= 232448, PHS_ERR_INVALID_ARG, "tensor-core M2L: shared memory layout too large");
    TcArgs a;
    a.tv = tree_view(t);
    a.tgt = f.tc_tgt.get();
    a.ntgt = t.nbox - b0;
    a.v_off = t.v_off.get();
    a.v_src = t.v_src.get();
    a.v_cls = t.v_cls.get();
    a.P = f.P;
    a.npad = f.tc_npad;
    a.nch = f.tc_nch;
    a.power = f.power;
    a.mpx = reinterpret_cast<const longlong2 *>(mp);
    a.lc = lc;
    a.mexp = f.tc_mexp.get();
    a.gexp = f.tc_gexp.get();
    a.S = f.tc_S.get();
    a.F = f.tc_F.get();
    a.off = f.tc_off.get();
    a.bplanes = f.tc_b.get();
    a.err = f.tc_err.get();
    a.wait_ns = f.tc_wait_ns > 0 ? f.tc_wait_ns : TC_TIMEOUT_NS;
    a.probe = f.tc_probe;
    const unsigned grid = (unsigned)((a.ntgt + TcLayout<ND>::TPB - 1) / TcLayout<ND>::TPB);
    m2l_tc_kernel<ND><<<grid, tc_threads<ND>(), lay.total, s>>>(a);
    PHS_LAUNCH_CHECK();
}

// Tile order of the M2L targets (the boxes of levels >= 2): by level, then by the box's
// position within its parent (the low two bits of its Morton key), then by box index.
// The V list of a box is the children of its parent's neighbours that are not its own
// neighbours, so in a refined neighbourhood its offset classes depend only on that
// position: 16 targets of one position share one class set (27 classes) where 16
// consecutive boxes (all four positions) span the union of 40, and each tile step
// stages and multiplies rows of every target in the tile.
__global__ void tc_tgt_keys(const int *level, const uint64_t *key, int b0, int nbox, uint64_t *k, int *v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbox - b0) return;
    const int b = b0 + i;
    k[i] = ((uint64_t)level[b] << 33) | ((key[b] & 3ull) << 31) | (uint64_t)b;
    v[i] = b;
}
static void tc_build_targets(Fmm &f, const Tree &t, int b0, bool force, cudaStream_t s) {
    if (!force && f.tc_tgt_nbox == t.nbox) return;
    const int n = t.nbox - b0;
    f.tc_tgt.alloc(std::max(n, 1));
    DBuf<uint64_t> k(std::max(n, 1));
    tc_tgt_keys<<<blocks_for(n, 256), 256, 0, s>>>(t.level.get(), t.key.get(), b0, t.nbox, k.get(), f.tc_tgt.get());
    PHS_LAUNCH_CHECK();
    radix_sort_pairs(k.get(), f.tc_tgt.get(), n, 38, s);
    PHS_CUDA(cudaStreamSynchronize(s));
    f.tc_tgt_nbox = t.nbox;
}

void m2l_tc_pass(Fmm &f, const Tree &t, double2 *mp, double2 *lc, cudaStream_t s) {
    const int b0 = t.depth >= 2 ? t.lvl_off[2] : t.nbox;
    const size_t esz = (size_t)f.nd * f.P * sizeof(double2);
    if (b0 > 0) PHS_CUDA(cudaMemsetAsync(lc, 0, (size_t)b0 * esz, s));
    if (b0 >= t.nbox) return;
    tc_build_targets(f, t, b0, false, s);  // built by m2l_tc_count for each new tree
    if (f.tc_mexp.n < (size_t)t.nbox) f.tc_mexp.alloc(t.nbox);
    tc_fixed_kernel<<<blocks_for(t.nbox, 8), 256, 0, s>>>(mp, t.nbox, f.nd, f.P, f.tc_mexp.get());
    PHS_LAUNCH_CHECK();
    if (f.nd == 4) launch_tc<4>(f, t, mp, lc, b0, s);
    else launch_tc<9>(f, t, mp, lc, b0, s);
}

// classes present per tile (the steps the pass will take)
__global__ void tc_count_kernel(const int *v_off, const unsigned char *v_cls, const int *tgt, int ntgt, int tpb,
                                unsigned long long *steps) {
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    const int tb0 = tile * tpb;
    if (tb0 >= ntgt) return;
    unsigned long long m = 0;
    for (int i = tb0; i < min(tb0 + tpb, ntgt); ++i) {
        const int b = tgt[i];
        for (int v = v_off[b]; v < v_off[b + 1]; ++v) m |= 1ull << v_cls[v];
    }
    atomicAdd(steps, (unsigned long long)__popcll(m));
}

// digit-plane products of 128 x npad x 16 per step (plane pairs i + j <= 5, three K slices)
int m2l_tc_mmas_per_step() { return (TC_KC / 16) * TC_NPL * (TC_NPL + 1) / 2; }

void m2l_tc_count(Fmm &f, const Tree &t, cudaStream_t s) {
    f.tc_steps = f.tc_tiles = 0;
    if (!f.tc || t.depth < 2) return;
    const int b0 = t.lvl_off[2];
    const int tpb = f.nd == 4 ? TcLayout<4>::TPB : TcLayout<9>::TPB;
    const int ntile = (t.nbox - b0 + tpb - 1) / tpb;
    if (ntile <= 0) return;
    tc_build_targets(f, t, b0, true, s);
    DBuf<unsigned long long> cnt(1);
    PHS_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(unsigned long long), s));
    tc_count_kernel<<<blocks_for(ntile, 128), 128, 0, s>>>(t.v_off.get(), t.v_cls.get(), f.tc_tgt.get(), t.nbox - b0,
                                                           tpb, cnt.get());
    PHS_LAUNCH_CHECK();
    unsigned long long h = 0;
    PHS_CUDA(cudaMemcpyAsync(&h, cnt.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    f.tc_steps = (int64_t)h * f.tc_nch;
    f.tc_tiles = ntile;
}

void m2l_tc_check(Fmm &f, cudaStream_t s) {
    if ((!f.tc && !f.ctc) || !f.tc_err.get()) return;
    int h = 0;
    PHS_CUDA(cudaMemcpyAsync(&h, f.tc_err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    PHS_CUDA(cudaStreamSynchronize(s));
    if (h) {
        PHS_CUDA(cudaMemsetAsync(f.tc_err.get(), 0, sizeof(int), s));
        f.far_valid = false;  // the expansions of that apply are incomplete: no evaluation reuses them
        throw Error{PHS_ERR_TIMEOUT, "tensor-core M2L: a bounded wait expired"};
    }
}

}  // namespace phs
