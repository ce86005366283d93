// ff.cuh -- float-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// (about 48 significant bits), built from error-free transformations -- TwoSum (Knuth)
// for sums and the FMA form of Dekker's TwoProd for products -- with explicit roundings
// so the compiler neither contracts nor reorders them.  Shared by the float-float near
// field and the float-float P2M / L2P.
#pragma once
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

namespace phs {
namespace ffa {

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// (a.h + a.l)(b.h + b.l) without the lo*lo term; the result's lo is not renormalised
__device__ __forceinline__ F2 ff_mul(F2 a, F2 b) {
    F2 p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return p;
}
__device__ __forceinline__ F2 ff_sub(F2 a, F2 b) {
    F2 s = two_sum(a.h, -b.h);
    s.l = __fadd_rn(s.l, __fsub_rn(a.l, b.l));
    return s;
}
__device__ __forceinline__ void ff_acc(F2 &acc, F2 v) {
    const F2 s = two_sum(acc.h, v.h);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, v.l));
}
__device__ __forceinline__ F2 split_d(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double to_d(F2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// complex float-float: (re, im) each hi + lo
struct C4 {
    F2 re, im;
};
// a + b with the result renormalised (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ F2 ff_add(F2 a, F2 b) {
    F2 s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ F2 ff_neg(F2 a) { return {-a.h, -a.l}; }
// (a.re + i a.im)(b.re + i b.im), renormalised parts
__device__ __forceinline__ C4 c4_mul(C4 a, C4 b) {
    return {ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__device__ __forceinline__ C4 c4_of(double2 z) { return {split_d(z.x), split_d(z.y)}; }
__device__ __forceinline__ float4 c4_pack(C4 a) { return make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }
__device__ __forceinline__ C4 c4_unpack(float4 v) { return {F2{v.x, v.y}, F2{v.z, v.w}}; }

// a b renormalised (|lo| <= ulp(hi) / 2), for products that feed further products
__device__ __forceinline__ F2 ff_mulr(F2 a, F2 b) {
    const F2 p = ff_mul(a, b);
    return fast_two_sum(p.h, p.l);
}
// s a power of two: exact
__device__ __forceinline__ F2 ff_scale(F2 a, float s) { return {a.h * s, a.l * s}; }

// The Hadamard factors of hadamard.cuh (had_v, had_u) in float-float, from float-float
// box-local coordinates; ND = 1, 4, 9 for the powers 0, 2, 4 of |x_i - x_j|.
template <int ND>
__device__ __forceinline__ void had_v_ff(F2 x, F2 y, F2 *v) {
    const F2 one{1.f, 0.f};
    v[0] = one;
    if constexpr (ND == 4) {
        v[1] = ff_add(ff_mulr(x, x), ff_mulr(y, y));
        v[2] = x;
        v[3] = y;
    } else if constexpr (ND == 9) {
        const F2 xx = ff_mulr(x, x), yy = ff_mulr(y, y), a = ff_add(xx, yy);
        v[1] = ff_mulr(a, a);
        v[2] = x;
        v[3] = y;
        v[4] = ff_mulr(a, x);
        v[5] = ff_mulr(a, y);
        v[6] = xx;
        v[7] = ff_mulr(x, y);
        v[8] = yy;
    }
}
template <int ND>
__device__ __forceinline__ void had_u_ff(F2 x, F2 y, F2 *u) {
    const F2 one{1.f, 0.f};
    if constexpr (ND == 1) {
        u[0] = one;
    } else if constexpr (ND == 4) {
        u[0] = ff_add(ff_mulr(x, x), ff_mulr(y, y));
        u[1] = one;
        u[2] = ff_scale(x, -2.f);
        u[3] = ff_scale(y, -2.f);
    } else {
        const F2 xx = ff_mulr(x, x), yy = ff_mulr(y, y), a = ff_add(xx, yy);
        u[0] = ff_mulr(a, a);
        u[1] = one;
        u[2] = ff_scale(ff_mulr(a, x), -4.f);
        u[3] = ff_scale(ff_mulr(a, y), -4.f);
        u[4] = ff_scale(x, -4.f);
        u[5] = ff_scale(y, -4.f);
        u[6] = ff_add(ff_scale(xx, 4.f), ff_scale(a, 2.f));
        u[7] = ff_scale(ff_mulr(x, y), 8.f);
        u[8] = ff_add(ff_scale(yy, 4.f), ff_scale(a, 2.f));
    }
}

// s = dx^2 + dy^2, renormalised so that |s.l| <= ulp(s.h) / 2
__device__ __forceinline__ F2 ff_norm2(F2 dx, F2 dy) {
    F2 px = two_prod(dx.h, dx.h);
    px.l = __fmaf_rn(2.0f * dx.h, dx.l, px.l);
    F2 py = two_prod(dy.h, dy.h);
    py.l = __fmaf_rn(2.0f * dy.h, dy.l, py.l);
    F2 s = two_sum(px.h, py.h);
    s.l = __fadd_rn(s.l, __fadd_rn(px.l, py.l));
    return fast_two_sum(s.h, s.l);
}

// log(s.h + s.l) for s > 0 with absolute error about 2^-46 max(1, |log s|); s = 0 (a
// point paired with itself) returns a finite value, so s log s is 0 there
__device__ __forceinline__ F2 ff_log(F2 s, const float *rcp, const float2 *tlog, const float2 *eln2) {
    const unsigned bits = __float_as_uint(s.h);
    const int j = (int)((bits >> 15) & 0xffu);
    const float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    const float2 E = eln2[(bits >> 23) & 0xffu];  // s >= +0 by construction; the mask keeps the index in range
    const float2 T = tlog[j];
    const float u = __fmaf_rn(m, rcp[j], -1.0f);  // exact
    const F2 p2 = two_prod(u, u);
    float q = __fmaf_rn(u, 0.2f, -0.25f);
    q = __fmaf_rn(u, q, 0.333333343f);
    const float tail = __fmul_rn(__fmul_rn(u, p2.h), q);  // u^3 (1/3 - u/4 + u^2/5)
    const F2 h = fast_two_sum(u, -0.5f * p2.h);            // |u| >= u^2 / 2
    const float lo1p = __fadd_rn(h.l, __fsub_rn(tail, 0.5f * p2.l));
    const F2 a = two_sum(E.x, T.x);
    const F2 b = two_sum(a.h, h.h);
    float lo = __fadd_rn(__fadd_rn(E.y, T.y), lo1p);
    lo = __fadd_rn(lo, __fadd_rn(a.l, b.l));
    // log(s.h + s.l) = log(s.h) + s.l / s.h + O(2^-48)
    lo = __fmaf_rn(s.l, rcp_approx(fmaxf(s.h, 1e-30f)), lo);
    return {b.h, lo};
}

// The tables of ff_log (host side): R_j (1/c_j rounded to 9 significant bits, c_j the
// centre of the j-th of 256 mantissa cells), -log R_j and (e - 127) log 2 for the biased
// FP32 exponents e, each logarithm split into hi + lo floats.
inline void ff_log_tables(std::vector<float> &rc, std::vector<float2> &tl, std::vector<float2> &el) {
    rc.resize(256);
    tl.resize(256);
    el.resize(256);
    for (int j = 0; j < 256; ++j) {
        const long double c = 1.0L + ((long double)j + 0.5L) / 256.0L;
        // 1/c rounded to 9 significant bits: 1/c in (1/2, 1), so a multiple of 2^-9
        const long double r = std::nearbyint(512.0L / c) / 512.0L;
        rc[j] = (float)r;
        const long double v = -std::log(r);
        const float h = (float)v;
        tl[j] = make_float2(h, (float)(v - (long double)h));
    }
    for (int be = 0; be < 256; ++be) {
        const long double v = (long double)(be - 127) * std::log(2.0L);
        const float h = (float)v;
        el[be] = make_float2(h, (float)(v - (long double)h));
    }
}

}  // namespace ffa
}  // namespace phs
