// ff.cuh -- float-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// (about 48 significant bits), built from error-free transformations -- TwoSum (Knuth)
// for sums and the FMA form of Dekker's TwoProd for products -- with explicit roundings
// so the compiler neither contracts nor reorders them.  Shared by the float-float near
// field and the float-float P2M / L2P.
#pragma once
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

}  // namespace ffa
}  // namespace phs
