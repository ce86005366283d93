// cheb_tc.cu -- the compressed M2L of the distance-kernel FMM (cheb.cu: odd k, the r factor
// of r^k = r * r^{k-1}, Eq. 2.6) on the 5th-generation tensor cores in exact fixed point,
// by the scheme of the log kernel's M2L (m2l_tc.cu).
//
// For a target box t the compressed translation is a sum over its interaction list, one
// source per offset class c:
//     L~_t[d][i] = sum_c sum_j C_c[i][j] (S_c W~_src(c))[d][j]
// with C_c the class operator in the shared rank-r basis (level-invariant; the box-size
// scaling is applied by cheb_expand) and S_c the integer frame change of the box-local
// Hadamard densities.  Over a tile of targets it is one dense real contraction,
// D[rows][i] = sum_(c,j) A_c[rows][j] B_c[j][i], rows = (density d, target), run exactly:
//   * every input is an integer X (|X| <= 2^47) times a power of two: the rows of a
//     target share its exponent E_(t,d) over its list, the columns of B the per-column
//     exponent F_i over all classes;
//   * X is split into six balanced base-256 digits (exact in bf16), plane pairs with
//     i + j <= 5 are multiplied by tcgen05.mma and accumulated per diagonal in FP32 in
//     tensor memory (6 diagonals x 80 columns fit its 512), exactly;
//   * the epilogue recombines the diagonals in integers and scales once in FP64.
// The products are exact, so the translation keeps the symmetry of the FP64 form
// (U = V, C_{-o} = C_o'), which the conjugate-gradient solve of these ill-conditioned
// systems needs; its error is the final rounding and the dropped planes (below 2^-48).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "phs_internal.cuh"
#include "tc.cuh"

namespace phs {

constexpr int CT_M = 128;                     // rows per tile (one TMEM lane each)
constexpr int CT_KC = 32;                     // K columns (compressed coefficients j) per step
constexpr int CT_KP = CT_KC / 2;              // column pairs per step: a staging item writes two
constexpr int CT_A_PLANE = CT_M * CT_KC * 2;  // bytes of one A digit plane
constexpr int CT_NSW = 12;                    // staging warps; one more warp issues the MMAs
constexpr int CT_T = 32 * (CT_NSW + 1);
constexpr int CT_NST = CT_NSW * 32;
constexpr int CT_MAXN = 80;                   // output columns: 6 diagonals x 80 <= 512 TMEM columns

template <int ND>
__host__ __device__ constexpr int ct_tpb() { return CT_M / ND; }  // targets per tile: 128, 32, 14

struct CtArgs {
    int b0, nbox;
    const int *v_off, *v_src;
    const unsigned char *v_cls;
    int rs, rt, npad, nch;
    const long long *wx;      // compressed weights in per-box fixed point [box][nd][rs]
    const int *mexp, *gexp, *S, *F;
    const uint16_t *bplanes;  // [49][nch][NPL][npad x CT_KC], core-matrix order
    double *lc;               // compressed potentials [box][nd][rt]
    int *err;
    uint64_t wait_ns;
    int probe;
};

template <int ND>
struct CtLayout {
    static constexpr int TPB = ct_tpb<ND>();
    int bplane, bstep;
    size_t off_B, off_vsrc, off_vsh, off_cflag, off_clist, off_E, off_mbar, off_misc, total;
    __host__ __device__ CtLayout(int npad) {
        bplane = npad * CT_KC * 2;
        bstep = TC_NPL * bplane;
        off_B = (size_t)2 * TC_NPL * CT_A_PLANE;
        off_vsrc = off_B + (size_t)2 * bstep;
        off_vsh = off_vsrc + (size_t)TPB * TC_NCLS * 4;
        off_cflag = off_vsh + (((size_t)TPB * TC_NCLS + 15) & ~(size_t)15);
        off_clist = off_cflag + TC_NCLS * 4;
        off_E = off_clist + TC_NCLS * 4;  // [TPB][ND] row exponents, then [TPB] minimum
        off_mbar = (off_E + (size_t)TPB * (ND + 1) * 4 + 7) & ~(size_t)7;
        off_misc = off_mbar + 7 * 8;
        total = off_misc + 16;
    }
};

// staging item -> (target, column pair); when TPB is a multiple of 8 a warp covers 8
// targets x 4 column pairs, whose 32 four-byte stores of a plane hit 32 different banks
template <int TPB>
__device__ __forceinline__ void ct_item(int it, int &ti, int &kk) {
    if constexpr (TPB % 8 == 0) {
        const int g = it >> 5, l = it & 31;
        ti = (l & 7) + 8 * (g % (TPB / 8));
        kk = (l >> 3) + 4 * (g / (TPB / 8));
    } else {
        ti = it % TPB;
        kk = it / TPB;
    }
}

// One warp per box: mexp = max exponent of |W~[b][.][.]| (|W~| < 2^mexp), then the box's
// compressed weights are rewritten in place as integers X = round(W~ 2^(53 - mexp)).
__global__ void ct_fixed_kernel(double *w, int b0, int nbox, int nd, int rs, int *mexp) {
    const int b = b0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= nbox) return;
    const int lane = threadIdx.x & 31;
    double *wb = w + (size_t)b * nd * rs;
    int m = -100000;
    for (int i = lane; i < nd * rs; i += 32) {
        const int e = (int)(((unsigned long long)__double_as_longlong(wb[i]) >> 52) & 0x7FF);
        if (e) m = max(m, e - 1023 + 1);
    }
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) mexp[b] = m;
    long long *xb = reinterpret_cast<long long *>(wb);
    for (int i = lane; i < nd * rs; i += 32) xb[i] = to_fixed(wb[i], 53 - m);
}

// Warp roles as in m2l_tc_kernel: warps 0 .. CT_NSW-1 stage A (one mbarrier arrival per
// thread on full[u] when buffer u is written), warp CT_NSW (lane 0) copies B by bulk
// copies and issues the MMAs, committing to empty[u] when they have read buffer u.  Every
// wait is bounded; a timeout ends all roles through the abort flag, and the drain waits
// (with the fixed 2 s limit) for the work in flight before TMEM is released.
template <int ND>
__global__ void __launch_bounds__(CT_T, 1) cheb_m2l_tc_kernel(CtArgs a) {
    using L = CtLayout<ND>;
    constexpr int TPB = L::TPB;
    extern __shared__ __align__(1024) unsigned char sm[];
    const L lay(a.npad);
    unsigned char *Abuf = sm;
    unsigned char *Bbuf = sm + lay.off_B;
    int *vsrc = reinterpret_cast<int *>(sm + lay.off_vsrc);
    unsigned char *vsh = sm + lay.off_vsh;  // [TPB][49] shift from the source's scale to the target's
    int *cflag = reinterpret_cast<int *>(sm + lay.off_cflag);
    int *clist = reinterpret_cast<int *>(sm + lay.off_clist);
    int *Et = reinterpret_cast<int *>(sm + lay.off_E);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + lay.off_mbar);  // empty[2], bfull[2], done, full[2]
    uint32_t *misc = reinterpret_cast<uint32_t *>(sm + lay.off_misc);  // tmem base, ncls, abort

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tb0 = a.b0 + blockIdx.x * TPB;
    const int nt = min(TPB, a.nbox - tb0);

    // ---- prologue: interaction lists of the tile, exponents, zeroed operand buffers (the
    // rows past ND x TPB are never staged and stay zero)
    for (int i = tid; i < TPB * TC_NCLS; i += CT_T) vsrc[i] = -1;
    for (int i = tid; i < TC_NCLS; i += CT_T) cflag[i] = 0;
    {
        uint4 *z = reinterpret_cast<uint4 *>(Abuf);
        const int n16 = 2 * TC_NPL * CT_A_PLANE / 16;
        for (int i = tid; i < n16; i += CT_T) z[i] = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        for (int i = 0; i < 5; ++i) tc::mbar_init(&mbar[i], 1);
        tc::mbar_init(&mbar[5], CT_NST);
        tc::mbar_init(&mbar[6], CT_NST);
        tc::fence_mbar_init();
        misc[2] = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&misc[0], 512);
        tc::tmem_relinquish();
    }
    __syncthreads();
    // row exponents: |(S_c W~)_d[j]| < 2^(E[t][d] - 1) over the interaction list
    for (int ti = tid; ti < nt; ti += CT_T) {
        const int b = tb0 + ti;
        int e[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) e[d] = -100000;
        for (int v = a.v_off[b]; v < a.v_off[b + 1]; ++v) {
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
            Et[ti * ND + d] = e[d] + 1;
            emin = min(emin, e[d] + 1);
        }
        Et[TPB * ND + ti] = emin;
        // emin >= mexp[src] + 1 for every source of the list, so the shift is >= 1
        for (int v = a.v_off[b]; v < a.v_off[b + 1]; ++v)
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
    const uint64_t adesc0 = tc::make_desc_kmajor(tc::smem_u32(Abuf), 128, (CT_KC / 8) * 128);
    const uint64_t bdesc0 = tc::make_desc_kmajor(tc::smem_u32(Bbuf), 128, (CT_KC / 8) * 128);
    uint32_t inited = 0;      // accumulators written at least once (issuer)
    int bpend[2] = {-1, -1};  // parity of an operator copy not yet waited for (issuer)
    const bool issuer = warp == CT_NSW && lane == 0;
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
    if (warp < CT_NSW) {
        for (int s = 0; s < nsteps; ++s) {
            const int u = s & 1;
            const int c = clist[s / a.nch], h = s % a.nch;
            if (misc[2]) break;
            if (s >= 2 && !tc::mbar_wait(&mbar[u], (uint32_t)(((s >> 1) - 1) & 1), a.wait_ns)) {
                misc[2] = 1;
                break;
            }
            unsigned char *Au = Abuf + (size_t)u * TC_NPL * CT_A_PLANE;
            const int *Sc = a.S + c * ND * ND;
            for (int it = tid; it < TPB * CT_KP; it += CT_NST) {
                int ti, kk;
                ct_item<TPB>(it, ti, kk);
                const int j0 = h * CT_KC + 2 * kk;
                const int src = (ti < nt && j0 < a.rs) ? vsrc[ti * TC_NCLS + c] : -1;
                if (src < 0) {
                    for (int d = 0; d < ND; ++d) {
                        const uint32_t off = tc::kmajor_offset(d * TPB + ti, 2 * kk, CT_KC);
#pragma unroll
                        for (int i = 0; i < TC_NPL; ++i) *reinterpret_cast<uint32_t *>(Au + i * CT_A_PLANE + off) = 0u;
                    }
                    continue;
                }
                const bool two = j0 + 1 < a.rs;
                // sources come to the finest row scale of the target (one rounding shift),
                // mix exactly in integers, and each row rounds once to its own exponent
                const int emin = Et[TPB * ND + ti];
                const int sh2 = vsh[ti * TC_NCLS + c];
                long long x0[ND], x1[ND];
#pragma unroll
                for (int b = 0; b < ND; ++b) {
                    const long long *wp = a.wx + ((size_t)src * ND + b) * a.rs + j0;
                    x0[b] = rshift_round(wp[0], sh2);
                    x1[b] = two ? rshift_round(wp[1], sh2) : 0ll;
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    long long y0 = 0, y1 = 0;
#pragma unroll
                    for (int b = 0; b < ND; ++b) {
                        const int sv = Sc[d * ND + b];
                        if (sv) {
                            y0 += (long long)sv * x0[b];
                            y1 += (long long)sv * x1[b];
                        }
                    }
                    const int dsh = Et[ti * ND + d] - emin;
                    float g0[TC_NPL], g1[TC_NPL];
                    digits_f(rshift_round(y0, TC_GB + dsh), g0);
                    digits_f(rshift_round(y1, TC_GB + dsh), g1);
                    const uint32_t off = tc::kmajor_offset(d * TPB + ti, 2 * kk, CT_KC);
#pragma unroll
                    for (int i = 0; i < TC_NPL; ++i)
                        *reinterpret_cast<uint32_t *>(Au + i * CT_A_PLANE + off) = pack_bf16(g0[i], g1[i]);
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
            const uint64_t au = adesc0 + (uint64_t)((u * TC_NPL * CT_A_PLANE) >> 4);
            const uint64_t bu = bdesc0 + (uint64_t)((u * lay.bstep) >> 4);
            // one MMA per A plane i and run of B planes j0 .. j0 + nj - 1 (consecutive along N,
            // N = nj x npad <= 256): each product lands on its diagonal i + j; plane i = 0
            // covers every diagonal first, so an MMA's diagonals are all fresh or all summed
#pragma unroll 1
            for (int ks = 0; ks < CT_KC / 16; ++ks) {
#pragma unroll
                for (int i = 0; i < TC_NPL; ++i) {
                    const uint64_t ad = au + (uint64_t)((i * CT_A_PLANE + ks * 256) >> 4);
                    for (int j0 = 0; j0 < TC_NPL - i; j0 += pl_per_mma) {
                        const int nj = min(pl_per_mma, TC_NPL - i - j0);
                        const int g = i + j0;
                        const uint64_t bd = bu + (uint64_t)((j0 * lay.bplane + ks * 256) >> 4);
                        tc::mma_bf16(tmem + (uint32_t)(g * a.npad), ad, bd, tc::idesc_bf16_f32(CT_M, nj * a.npad),
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
    // flight are waited for with the fixed 2 s limit before TMEM is released.
    __syncthreads();
    const bool aborted = misc[2] != 0;
    bool ok = !aborted;
    if (nsteps > 0) {
        if (issuer) tc::mma_commit(&mbar[4]);
        ok = tc::mbar_wait(&mbar[4], 0, TC_TIMEOUT_NS) && ok;
    }
    if (issuer) {
        for (int u = 0; u < 2; ++u)
            if (bpend[u] >= 0 && !tc::mbar_wait(&mbar[2 + u], (uint32_t)bpend[u], TC_TIMEOUT_NS)) ok = false;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) atomicExch(a.err, 1);
    __syncthreads();
    ok = !misc[2] && ok;
    tc::fence_after_sync();

    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, 16-column chunks w / 4, w / 4 + WQ, ...
    constexpr int WQ = (CT_T / 32) / 4;
    if (ok && warp < 4 * WQ) {
        const int q = warp & 3, cg = warp >> 2;
        const int r = 32 * q + lane;
        const int d = r / TPB, ti = r - d * TPB;
        const bool valid = d < ND && ti < nt;
        const int E = valid ? Et[ti * ND + d] : 0;
        double *dst = valid ? a.lc + ((size_t)(tb0 + ti) * ND + d) * a.rt : nullptr;
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
                    if (l < a.rt) {
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
                        }
                        dst[l] = val;
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
static inline uint16_t ct_bf16_bits(int v) {
    const float f = (float)v;  // |v| <= 128: exact in bf16
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

struct CtHostTables {
    std::vector<uint16_t> B;
    std::vector<int> F;
};

// Digit planes of B_c[j][i] = C_c[i][j] (C stored transposed, Ct[c][j][i]) with the
// column exponents F_i = max over (c, j) of the exponent of |C_c[i][j]|.
static CtHostTables build_ct_tables(int rs, int rt, int npad, int nch, const double *Ct) {
    auto valid_cls = [](int c) {
        const int dx = c / 7 - 3, dy = c % 7 - 3;
        return std::abs(dx) > 1 || std::abs(dy) > 1;
    };
    CtHostTables out;
    std::vector<int> F(rt, -100000);
    for (int c = 0; c < TC_NCLS; ++c) {
        if (!valid_cls(c)) continue;
        for (int j = 0; j < rs; ++j)
            for (int i = 0; i < rt; ++i) {
                const double v = Ct[((size_t)c * rs + j) * rt + i];
                if (v == 0) continue;
                int e;
                std::frexp(v, &e);
                F[i] = std::max(F[i], e);
            }
    }
    const size_t plane = (size_t)npad * CT_KC;
    std::vector<uint16_t> B((size_t)TC_NCLS * nch * TC_NPL * plane, 0);
    for (int c = 0; c < TC_NCLS; ++c) {
        if (!valid_cls(c)) continue;
        for (int h = 0; h < nch; ++h)
            for (int i = 0; i < rt; ++i)
                for (int kc = 0; kc < CT_KC; ++kc) {
                    const int j = h * CT_KC + kc;
                    if (j >= rs) continue;
                    long long X = std::llround(std::ldexp(Ct[((size_t)c * rs + j) * rt + i], TC_QB - F[i]));
                    int dig[TC_NPL];
                    for (int p = TC_NPL - 1; p >= 1; --p) {
                        const int qd = (int)((X + 128) & 255) - 128;
                        dig[p] = qd;
                        X = (X - qd) >> TC_DB;
                    }
                    dig[0] = (int)X;
                    PHS_REQUIRE(std::abs(dig[0]) <= 128, PHS_ERR_INVALID_ARG,
                                "distance-kernel tensor-core M2L: operator digit overflow");
                    // element (row i, column kc) of a K-major core-matrix tile
                    const size_t boff = (size_t)i / 8 * (CT_KC / 8) * 64 + (size_t)kc / 8 * 64 + (i % 8) * 8 + kc % 8;
                    for (int p = 0; p < TC_NPL; ++p)
                        B[(((size_t)c * nch + h) * TC_NPL + p) * plane + boff] = ct_bf16_bits(dig[p]);
                }
    }
    out.B = std::move(B);
    out.F = std::move(F);
    return out;
}

bool cheb_tc_supported(int nd, int rs, int rt) {
    return (nd == 1 || nd == 4 || nd == 9) && rs <= CT_MAXN && rt <= CT_MAXN && rs >= 2 && rt >= 1;
}

void cheb_tc_setup(Fmm &f, const double *Ct, const std::vector<long double> &mix, cudaStream_t s) {
    const int rs = f.cheb_rs, rt = f.cheb_rt, nd = f.nd;
    PHS_REQUIRE(cheb_tc_supported(nd, rs, rt), PHS_ERR_INVALID_ARG,
                "distance-kernel tensor-core M2L needs nd in {1, 4, 9} and ranks <= 80");
    f.ctc_npad = (rt + 15) / 16 * 16;
    f.ctc_nch = (rs + CT_KC - 1) / CT_KC;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, CtHostTables> cache;  // the operators depend on (q, ranks) only
    const CtHostTables *tab;
    {
        std::lock_guard<std::mutex> g(mu);
        const auto key = std::make_tuple(f.cheb_q, rs, rt);
        auto it = cache.find(key);
        if (it == cache.end()) it = cache.emplace(key, build_ct_tables(rs, rt, f.ctc_npad, f.ctc_nch, Ct)).first;
        tab = &it->second;
    }
    std::vector<int> S, gexp;
    tc_integer_frames(nd, mix, S, gexp);
    f.ctc_b.alloc(tab->B.size());
    f.ctc_F.alloc(rt);
    f.tc_S.alloc(S.size());
    f.tc_gexp.alloc(gexp.size());
    f.tc_err.alloc(1);
    PHS_CUDA(cudaMemcpyAsync(f.ctc_b.get(), tab->B.data(), tab->B.size() * 2, cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.ctc_F.get(), tab->F.data(), rt * sizeof(int), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.tc_S.get(), S.data(), S.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemcpyAsync(f.tc_gexp.get(), gexp.data(), gexp.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    PHS_CUDA(cudaMemsetAsync(f.tc_err.get(), 0, sizeof(int), s));
    PHS_CUDA(cudaStreamSynchronize(s));
    f.ctc = true;
}

template <int ND>
static void launch_ct(Fmm &f, const Tree &t, int b0, double *wc, double *lc, cudaStream_t s) {
    const CtLayout<ND> lay(f.ctc_npad);
    static bool attr_set = false;
    if (!attr_set) {
        PHS_CUDA(cudaFuncSetAttribute(cheb_m2l_tc_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448));
        attr_set = true;
    }
    PHS_REQUIRE(lay.total <= 232448, PHS_ERR_INVALID_ARG, "distance-kernel tensor-core M2L: shared memory too large");
    CtArgs a;
    a.b0 = b0;
    a.nbox = t.nbox;
    a.v_off = t.v_off.get();
    a.v_src = t.v_src.get();
    a.v_cls = t.v_cls.get();
    a.rs = f.cheb_rs;
    a.rt = f.cheb_rt;
    a.npad = f.ctc_npad;
    a.nch = f.ctc_nch;
    a.wx = reinterpret_cast<const long long *>(wc);
    a.mexp = f.ctc_mexp.get();
    a.gexp = f.tc_gexp.get();
    a.S = f.tc_S.get();
    a.F = f.ctc_F.get();
    a.bplanes = f.ctc_b.get();
    a.lc = lc;
    a.err = f.tc_err.get();
    a.wait_ns = f.tc_wait_ns > 0 ? f.tc_wait_ns : TC_TIMEOUT_NS;
    a.probe = f.tc_probe;
    const int nb = t.nbox - b0;
    const unsigned grid = (unsigned)((nb + CtLayout<ND>::TPB - 1) / CtLayout<ND>::TPB);
    cheb_m2l_tc_kernel<ND><<<grid, CT_T, lay.total, s>>>(a);
    PHS_LAUNCH_CHECK();
}

// boxes b0 .. nbox-1: lc[b][d][i] = L~ (overwritten); wc (compressed weights, FP64) is
// rewritten in place as per-box fixed point
void cheb_m2l_tc_pass(Fmm &f, const Tree &t, int b0, double *wc, double *lc, cudaStream_t s) {
    if (b0 >= t.nbox) return;
    if (f.ctc_mexp.n < (size_t)t.nbox) f.ctc_mexp.alloc(t.nbox);
    const int nb = t.nbox - b0;
    ct_fixed_kernel<<<blocks_for(nb, 8), 256, 0, s>>>(wc, b0, t.nbox, f.nd, f.cheb_rs, f.ctc_mexp.get());
    PHS_LAUNCH_CHECK();
    if (f.nd == 4) launch_ct<4>(f, t, b0, wc, lc, s);
    else if (f.nd == 9) launch_ct<9>(f, t, b0, wc, lc, s);
    else launch_ct<1>(f, t, b0, wc, lc, s);
}

}  // namespace phs
