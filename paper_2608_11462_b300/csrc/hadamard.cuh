// hadamard.cuh -- the separable factors of the Hadamard identity (Eq. 2.6): with
// [|x_i - x_j|^power] = sum_l u_l(x_i) v_l(x_j), M = M_core o [r^power] is applied as
// sum_l D_{u_l} M_core D_{v_l}.  Evaluated in box-local scaled coordinates by every pass
// that forms charges (P2M) or combines potentials (L2P), for both cores.
#pragma once

namespace phs {

// Hadamard factors of [|x_i - x_j|^power] (Sec. 2): u_l(x_i) v_l(x_j) summed over l.
// power 2: rank 4.  power 4: rank 9 (|x|^2 |y|^2 folds into the quadratic monomials,
// so the separable rank is 9 rather than the 10 terms of the plain expansion).
__device__ __forceinline__ void had_v(int power, double x, double y, double *v) {
    const double a = x * x + y * y;
    if (power == 0) {
        v[0] = 1.0;
    } else if (power == 2) {
        v[0] = 1.0; v[1] = a; v[2] = x; v[3] = y;
    } else {
        v[0] = 1.0; v[1] = a * a; v[2] = x; v[3] = y; v[4] = a * x; v[5] = a * y;
        v[6] = x * x; v[7] = x * y; v[8] = y * y;
    }
}
__device__ __forceinline__ void had_u(int power, double x, double y, double *u) {
    const double a = x * x + y * y;
    if (power == 0) {
        u[0] = 1.0;
    } else if (power == 2) {
        u[0] = a; u[1] = 1.0; u[2] = -2.0 * x; u[3] = -2.0 * y;
    } else {
        u[0] = a * a; u[1] = 1.0; u[2] = -4.0 * a * x; u[3] = -4.0 * a * y; u[4] = -4.0 * x; u[5] = -4.0 * y;
        u[6] = 4.0 * x * x + 2.0 * a; u[7] = 8.0 * x * y; u[8] = 4.0 * y * y + 2.0 * a;
    }
}
}  // namespace phs
