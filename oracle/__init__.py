"""CPU FP64 oracle for polyharmonic-spline (PHS) interpolation (Geoga & O'Neil).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never calls it; the two meet only through the seeded
input generators in ``synth.py``.

What it computes, each function citing the passage it follows:

* ``normalize``           -- the affine map to a square domain (Sec. 2, Eq. 2.1
                             and the domain choices of Sec. 2.2).
* ``poly_basis``          -- the polynomial block B of Eq. (1.3).
* ``dense_*``             -- the kernel matrix M, M t and the interpolant,
                             Eqs. (1.1)-(1.3), by their O(n^2) definitions
                             (row by row for sampled rows; ``dense_eval_abs``
                             the sums of absolute terms, their rounding scale).
* ``solve_augmented``     -- the augmented system (1.3) by LU with partial
                             pivoting (a library primitive).
* ``solve_qperp``         -- the same system by the sequence (2.5) with an
                             explicit complete QR and a Cholesky factor.
* ``random_order``, ``maxmin_order``, ``hmaxmin_order``, ``amaxmin_order``, ``knn_prev``,
  ``vecchia_factor``,
  ``vecchia_apply``       -- the Vecchia preconditioner of Sec. 2.2 (Eq. 2.19,
                             Fig. 1) with brute-force neighbour search.
* ``projected_precond``   -- the preconditioner of the projected system, with or
                             without the low-rank (Schur complement) term that
                             Sec. 2.2 discusses and sets aside.
* ``pcg``                 -- preconditioned CG on Q_perp^T M Q_perp (Sec. 2,
                             after Eq. 2.5; Sec. 2.2) with a dense matvec.
* ``gmres``               -- restarted GMRES with the Vecchia factor as right
                             preconditioner on M c = b, the kernel matrix alone
                             (the comparison of Sec. 3.1), dense matvec.

The FMM of Sec. 2.1 is not restated here: it approximates M t, whose plain
definition ``dense_matvec`` is the oracle for it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i64, u64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
        P = ctypes.c_void_p
        L.or_phi.restype = d
        L.or_phi.argtypes = [i32, d]
        L.or_dense_matrix.argtypes = [i64, P, i32, P]
        L.or_dense_matvec.argtypes = [i64, P, i32, P, P]
        L.or_dense_eval.argtypes = [i64, P, P, i32, i64, P, P]
        L.or_dense_eval_abs.argtypes = [i64, P, P, i32, i64, P, P]
        L.or_splitmix64.restype = u64
        L.or_splitmix64.argtypes = [u64, u64]
        L.or_random_order.argtypes = [i64, u64, P]
        L.or_maxmin_order.argtypes = [i64, P, P, P]
        L.or_knn_prev.argtypes = [i64, P, P, i32, P]
        L.or_bessel_k1.restype = d
        L.or_bessel_k1.argtypes = [d]
        L.or_bessel_k0.restype = d
        L.or_bessel_k0.argtypes = [d]
        L.or_matern.restype = d
        L.or_matern.argtypes = [d, d, d]
        L.or_vecchia_factor.restype = i64
        L.or_vecchia_factor.argtypes = [i64, P, P, P, i32, d, d, d, P, P]
        L.or_vecchia_apply.argtypes = [i64, P, i32, P, P, P, P]
        _LIB = L
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# frame and polynomial block
def normalize(points, halfwidth: float = 0.25):
    """Map points into [-halfwidth, halfwidth]^2 (Sec. 2: scale invariance, Eq. 2.1;
    Sec. 2.2: [-1/4,1/4]^2 for k = 2, [-1,1]^2 for k = 4).

    centre c = (min + max)/2 per axis, rho = halfwidth / (max(extent_x, extent_y)/2),
    x' = (x - c) * rho.  Returns (x', c, rho)."""
    x = _f64(points).reshape(-1, 2)
    lo = x.min(axis=0)
    hi = x.max(axis=0)
    c = (lo + hi) * 0.5
    h = max(hi[0] - lo[0], hi[1] - lo[1]) * 0.5
    if not h > 0:
        raise ValueError("all points coincide")
    rho = halfwidth / h
    return (x - c) * rho, c, rho


def min_poly_degree(k: int) -> int:
    """Smallest polynomial degree that makes phi conditionally positive definite:
    k/2 for even k, (k-1)/2 for odd k (Sec. 1, Eq. 1.3)."""
    return k // 2 if k % 2 == 0 else (k - 1) // 2


def cpd_sign(k: int) -> int:
    """Sign s with s * Q_perp^T M Q_perp positive definite.  The paper states
    Q_perp^T M Q_perp > 0 for the thin-plate case (Sec. 1); for general k the
    classical result is that (-1)^ceil(k/2) r^k (odd k) and (-1)^(k/2+1) r^k log r
    (even k) are conditionally positive definite of the minimal order."""
    return (-1) ** ((k + 1) // 2) if k % 2 == 1 else (-1) ** (k // 2 + 1)


def n_poly(deg: int) -> int:
    return (deg + 1) * (deg + 2) // 2


def poly_basis(x, deg: int) -> np.ndarray:
    """B_{j,s} = P_s(x_j): the total-degree monomials up to `deg`, graded
    lexicographic order 1, x, y, x^2, xy, y^2, ... (Eq. 1.3)."""
    x = _f64(x).reshape(-1, 2)
    cols = []
    for d in range(deg + 1):
        for b in range(d + 1):
            a = d - b
            cols.append(x[:, 0] ** a * x[:, 1] ** b)
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# dense kernel matrix, Eqs. (1.1)-(1.3)
def phi(k: int, r: float) -> float:
    return lib().or_phi(int(k), float(r))


def dense_matrix(x, k: int) -> np.ndarray:
    x = _f64(x).reshape(-1, 2)
    n = x.shape[0]
    out = np.empty((n, n), dtype=np.float64)
    lib().or_dense_matrix(n, _p(x), int(k), _p(out))
    return out


def dense_matvec(x, k: int, t) -> np.ndarray:
    x = _f64(x).reshape(-1, 2)
    t = _f64(t)
    out = np.empty(x.shape[0], dtype=np.float64)
    lib().or_dense_matvec(x.shape[0], _p(x), int(k), _p(t), _p(out))
    return out


def dense_eval(x, w, k: int, y) -> np.ndarray:
    x = _f64(x).reshape(-1, 2)
    y = _f64(y).reshape(-1, 2)
    w = _f64(w)
    out = np.empty(y.shape[0], dtype=np.float64)
    lib().or_dense_eval(x.shape[0], _p(x), _p(w), int(k), y.shape[0], _p(y), _p(out))
    return out


def dense_eval_abs(x, w, k: int, y) -> np.ndarray:
    """sum_j |w_j phi(|x_j - y|)|: the scale against which the rounding of dense_eval's
    sums (any summation order, any fast method) is measured."""
    x = _f64(x).reshape(-1, 2)
    y = _f64(y).reshape(-1, 2)
    w = _f64(w)
    out = np.empty(y.shape[0], dtype=np.float64)
    lib().or_dense_eval_abs(x.shape[0], _p(x), _p(w), int(k), y.shape[0], _p(y), _p(out))
    return out


def interpolant(x, w, beta, k: int, deg: int, y) -> np.ndarray:
    """f^(y) = sum_s beta_s P_s(y) + sum_j w_j phi(|x_j - y|), Eq. (1.1)."""
    return poly_basis(y, deg) @ _f64(beta) + dense_eval(x, w, k, y)


# --------------------------------------------------------------------------
# direct solves of the augmented system
def solve_augmented(x, f, k: int, deg: int):
    """[M B; B^T 0][w; beta] = [f; 0], Eq. (1.3), by LU with partial pivoting."""
    x = _f64(x).reshape(-1, 2)
    n = x.shape[0]
    M = dense_matrix(x, k)
    B = poly_basis(x, deg)
    S = B.shape[1]
    A = np.zeros((n + S, n + S))
    A[:n, :n] = M
    A[:n, n:] = B
    A[n:, :n] = B.T
    rhs = np.concatenate([_f64(f), np.zeros(S)])
    sol = np.linalg.solve(A, rhs)
    return sol[:n], sol[n:]


def solve_qperp(x, f, k: int, deg: int):
    """The sequence (2.5): Q_perp^T M Q_perp u = Q_perp^T f, w = Q_perp u,
    R beta = Q^T (f - M w), with B = QR and [Q Q_perp] orthogonal."""
    x = _f64(x).reshape(-1, 2)
    f = _f64(f)
    M = dense_matrix(x, k)
    B = poly_basis(x, deg)
    S = B.shape[1]
    Qc, Rc = np.linalg.qr(B, mode="complete")
    Q, Qp, R = Qc[:, :S], Qc[:, S:], Rc[:S, :]
    sg = cpd_sign(k)
    Mp = sg * (Qp.T @ M @ Qp)
    L = np.linalg.cholesky(Mp)
    u = np.linalg.solve(L.T, np.linalg.solve(L, sg * (Qp.T @ f)))
    w = Qp @ u
    beta = np.linalg.solve(R, Q.T @ (f - M @ w))
    return w, beta


# --------------------------------------------------------------------------
# Vecchia preconditioner, Sec. 2.2
def splitmix64(seed: int, i: int) -> int:
    return int(lib().or_splitmix64(ctypes.c_uint64(seed), ctypes.c_uint64(i)))


def random_order(n: int, seed: int) -> np.ndarray:
    """order[r] = point of rank r; ranks sorted by (splitmix64(seed, i), i)."""
    out = np.empty(n, dtype=np.int64)
    lib().or_random_order(n, ctypes.c_uint64(seed), _p(out))
    return out


def maxmin_order(x):
    """Exact greedy maxmin enumeration; returns (order, squared selection distances)."""
    x = _f64(x).reshape(-1, 2)
    n = x.shape[0]
    out = np.empty(n, dtype=np.int64)
    dm = np.empty(n, dtype=np.float64)
    lib().or_maxmin_order(n, _p(x), _p(out), _p(dm))
    return out, dm


def hmaxmin_order(x, seed: int):
    """Hierarchical maximin enumeration, restated from its definition level by level
    (the spacing property of maxmin enumeration kept per dyadic level of the bounding
    square, for the ordering of Sec. 2.2):
    level-30 cell coordinates ix = min(floor((x - xmin) * (2^30 / E)), 2^30 - 1) with E
    the larger extent; a level-L cell (ix >> (30 - L), iy >> (30 - L)) is represented by
    its parent's representative when that lies in it, else by its point nearest the cell
    centre ((x - cx)^2 + (y - cy)^2 in FP64, one rounding per operation, ties to the
    smaller index); a point's level is the first level at which it represents its cell
    (31 if never); the enumeration sorts by (level, splitmix64(seed, i) >> 7, i).
    Returns (order, level)."""
    x = _f64(x).reshape(-1, 2)
    n = x.shape[0]
    idx = np.arange(n)
    xmin, ymin = x[:, 0].min(), x[:, 1].min()
    E = max(x[:, 0].max() - xmin, x[:, 1].max() - ymin)
    if not E > 0:
        E = 1.0
    scale = 2.0 ** 30 / E
    lim = 2 ** 30 - 1
    ix = np.clip(np.floor((x[:, 0] - xmin) * scale), 0, lim).astype(np.int64)
    iy = np.clip(np.floor((x[:, 1] - ymin) * scale), 0, lim).astype(np.int64)
    level = np.full(n, 31, dtype=np.int64)
    rep = None
    for L in range(31):
        cx_i, cy_i = ix >> (30 - L), iy >> (30 - L)
        cell = cx_i * (1 << 31) + cy_i
        w = np.ldexp(E, -L)
        dx = x[:, 0] - (xmin + (cx_i + 0.5) * w)
        dy = x[:, 1] - (ymin + (cy_i + 0.5) * w)
        d2 = dx * dx + dy * dy
        o = np.lexsort((idx, d2, cell))          # by cell, then distance, then index
        first = np.ones(n, dtype=bool)
        first[1:] = cell[o][1:] != cell[o][:-1]
        ucell, best = cell[o][first], o[first]   # the nearest point of each cell
        nearest = best[np.searchsorted(ucell, cell)]
        rep = nearest if rep is None else np.where(cell[rep] == cell, rep, nearest)
        newly = (rep == idx) & (level == 31)
        level[newly] = L
    h = np.array([splitmix64(seed, int(i)) >> 7 for i in range(n)], dtype=np.uint64)
    order = np.lexsort((idx, h, level))
    return order.astype(np.int64), level


def amaxmin_order(x):
    """Dyadic approximate maximin enumeration (for the ordering of Sec. 2.2), restated
    from its definition.  An exact maxmin order appends, one at a time, the point
    farthest from those already taken; this one appends whole batches, each point of a
    batch at least half as far from the points already taken as the farthest remaining
    one, so it can be built in parallel.  Definition:

    * E, xmin, ymin and the level-30 integer coordinates ix, iy as in hmaxmin_order;
      c_L = E 2^-L and the level-L cell of a point (ix >> (30 - L), iy >> (30 - L));
    * the first point is the one nearest the square's centre (xmin + E/2, ymin + E/2),
      ties to the smaller index; l2[i] = squared distance of i to the taken points
      (FP64, dx*dx + dy*dy with one rounding per operation);
    * for L = 0, 1, ..., 30, passes repeat while some untaken point has l2 >= c_L^2
      (a candidate): in each level-L cell the candidate with the largest l2 (ties to the
      smaller index) is eligible; eligible points are visited by (l2 descending, index)
      and each is accepted unless an accepted point of the same pass lies at squared
      distance < c_L^2; the accepted points are appended in that visiting order and
      l2 is lowered by their distances;
    * points still untaken after level 30 (coincident points) follow by (l2 descending,
      index).

    Returns (order, level, l2 at selection); the first point has level -1 and l2 = inf,
    the tail level 31."""
    from scipy.spatial import cKDTree

    x = _f64(x).reshape(-1, 2)
    n = x.shape[0]
    idx = np.arange(n)
    xmin, ymin = x[:, 0].min(), x[:, 1].min()
    E = max(x[:, 0].max() - xmin, x[:, 1].max() - ymin)
    if not E > 0:
        E = 1.0
    scale = 2.0 ** 30 / E
    lim = 2 ** 30 - 1
    ix = np.clip(np.floor((x[:, 0] - xmin) * scale), 0, lim).astype(np.int64)
    iy = np.clip(np.floor((x[:, 1] - ymin) * scale), 0, lim).astype(np.int64)

    def d2_to(p):
        dx = x[:, 0] - p[0]
        dy = x[:, 1] - p[1]
        return dx * dx + dy * dy

    d2c = d2_to((xmin + 0.5 * E, ymin + 0.5 * E))
    root = int(np.lexsort((idx, d2c))[0])
    taken = np.zeros(n, dtype=bool)
    taken[root] = True
    order, level, l2sel = [root], [-1], [np.inf]
    l2 = d2_to(x[root])
    for L in range(31):
        cL = np.ldexp(E, -L)
        c2 = cL * cL
        sh = 30 - L
        while True:
            cand = np.nonzero(~taken & (l2 >= c2))[0]
            if cand.size == 0:
                break
            cell = (ix[cand] >> sh) * (1 << 31) + (iy[cand] >> sh)
            o = np.lexsort((cand, -l2[cand], cell))          # by cell, then l2 descending, then index
            first = np.ones(cand.size, dtype=bool)
            first[1:] = cell[o][1:] != cell[o][:-1]
            elig = cand[o][first]
            elig = elig[np.lexsort((elig, -l2[elig]))]        # visiting order
            acc, grid = [], {}
            for e in elig:
                gx, gy = int(ix[e] >> sh), int(iy[e] >> sh)
                ok = True
                for ax in range(gx - 2, gx + 3):              # a conflict (distance < c_L) lies
                    for ay in range(gy - 2, gy + 3):          # within one cell; two checked
                        for a in grid.get((ax, ay), ()):
                            dx = x[e, 0] - x[a, 0]
                            dy = x[e, 1] - x[a, 1]
                            if dx * dx + dy * dy < c2:
                                ok = False
                if ok:
                    acc.append(int(e))
                    grid.setdefault((gx, gy), []).append(int(e))
            acc = np.array(acc, dtype=np.int64)
            order.extend(acc.tolist())
            level.extend([L] * acc.size)
            l2sel.extend(l2[acc].tolist())
            taken[acc] = True
            rest = np.nonzero(~taken)[0]
            if rest.size:
                k = min(8, acc.size)
                _, nb = cKDTree(x[acc]).query(x[rest], k=k)
                nb = nb.reshape(rest.size, k)
                for j in range(k):
                    a = acc[nb[:, j]]
                    dx = x[rest, 0] - x[a, 0]
                    dy = x[rest, 1] - x[a, 1]
                    l2[rest] = np.minimum(l2[rest], dx * dx + dy * dy)
    rest = np.nonzero(~taken)[0]
    rest = rest[np.lexsort((rest, -l2[rest]))]
    order.extend(rest.tolist())
    level.extend([31] * rest.size)
    l2sel.extend(l2[rest].tolist())
    return np.array(order, dtype=np.int64), np.array(level, dtype=np.int64), np.array(l2sel)


def knn_prev(x, order, m: int) -> np.ndarray:
    """nbr[i, :] = the min(m, rank(i)) nearest points of smaller rank, by
    (squared distance, rank); -1 padded.  Brute force."""
    x = _f64(x).reshape(-1, 2)
    order = np.ascontiguousarray(order, dtype=np.int64)
    n = x.shape[0]
    out = np.empty((n, m), dtype=np.int64)
    lib().or_knn_prev(n, _p(x), _p(order), int(m), _p(out))
    return out


def bessel_k1(x: float) -> float:
    return lib().or_bessel_k1(float(x))


def bessel_k0(x: float) -> float:
    return lib().or_bessel_k0(float(x))


def matern(nu: float, alpha: float, r) -> np.ndarray:
    r = np.atleast_1d(_f64(r))
    L = lib()
    return np.array([L.or_matern(float(nu), float(alpha), float(v)) for v in r.ravel()]).reshape(r.shape)


def vecchia_factor(x, order, nbr, m: int, nu: float, alpha: float, jitter_base: float = 1e-12):
    """Columns of U~ (Sigma^{-1} ~= U~ U~^T), Eq. (2.19) and Fig. 1.
    Returns (diag, offd, n_jittered)."""
    x = _f64(x).reshape(-1, 2)
    order = np.ascontiguousarray(order, dtype=np.int64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int64)
    n = x.shape[0]
    diag = np.zeros(n)
    offd = np.zeros((n, m))
    nj = lib().or_vecchia_factor(n, _p(x), _p(order), _p(nbr), int(m), float(nu), float(alpha),
                                 float(jitter_base), _p(diag), _p(offd))
    if nj < 0:
        raise RuntimeError("local Cholesky failed")
    return diag, offd, int(nj)


def vecchia_apply(nbr, diag, offd, r) -> np.ndarray:
    """z = U~ (U~^T r)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int64)
    n, m = nbr.shape
    r = _f64(r)
    z = np.empty(n)
    lib().or_vecchia_apply(n, _p(nbr), int(m), _p(_f64(diag)), _p(_f64(offd)), _p(r), _p(z))
    return z


def vecchia_dense(nbr, diag, offd) -> np.ndarray:
    """The dense n x n matrix U~ of Fig. 1 (column i: 1/c at i, -lambda/c at sigma(i))."""
    n, m = nbr.shape
    U = np.zeros((n, n))
    for i in range(n):
        U[i, i] = diag[i]
        for q in range(m):
            if nbr[i, q] >= 0:
                U[nbr[i, q], i] = offd[i, q]
    return U


# --------------------------------------------------------------------------
# preconditioned CG, Sec. 2 (after Eq. 2.5) and Sec. 2.2
def projected_precond(x, deg: int, precond, v, lowrank: bool) -> np.ndarray:
    """Preconditioner of the projected system (Sec. 2.2), applied to v in range(P),
    P = I - Q Q^T.  With S~^{-1} = U~ U~^T the Vecchia approximation of the Matern
    precision (Eq. 2.19, Fig. 1):

    * lowrank = False: z = P S~^{-1} v, i.e. Q_perp^T S~^{-1} Q_perp, the form the
      paper runs (it drops the Schur complement term of the inverse);
    * lowrank = True:  z = S~^{-1} v - S~^{-1} B (B^T S~^{-1} B)^{-1} B^T S~^{-1} v,
      the block-elimination (Schur complement) solution of the saddle-point system
      [S~ B; B^T 0] [z; lam] = [v; 0], i.e. the inverse of Q_perp^T S~ Q_perp on
      range(P) -- the "low-rank update" that Sec. 2.2 mentions and sets aside.

    precond = (nbr, diag, offd)."""
    x = _f64(x).reshape(-1, 2)
    nbr, diag, offd = precond
    t = vecchia_apply(nbr, diag, offd, v)
    B = poly_basis(x, deg)
    if lowrank:
        G = np.stack([vecchia_apply(nbr, diag, offd, B[:, j]) for j in range(B.shape[1])], axis=1)
        return t - G @ np.linalg.solve(B.T @ G, G.T @ v)
    Q, _ = np.linalg.qr(B)
    return t - Q @ (Q.T @ t)


def pcg(x, f, k: int, deg: int, precond=None, tol: float = 1e-10, maxiter: int = 500, atol: float = 0.0,
        lowrank: bool = False):
    """PCG for Q_perp^T M Q_perp u = Q_perp^T f with preconditioner
    ``projected_precond`` (Q_perp^T U~ U~^T Q_perp, or with ``lowrank`` the inverse
    of Q_perp^T S~ Q_perp), run on the iterates w = Q_perp u in R^n using
    Q_perp Q_perp^T = I - Q Q^T (Q from the thin QR of B).  x_0 = 0; stops when
    the recursive residual satisfies ||r_k|| <= max(tol ||Q_perp^T f||, atol).
    The system is multiplied by cpd_sign(k) so that CG sees a positive definite
    operator.  precond = (nbr, diag, offd) or None.  Returns (w, beta, iters, history)."""
    sg = cpd_sign(k)
    x = _f64(x).reshape(-1, 2)
    f = _f64(f)
    B = poly_basis(x, deg)
    Q, R = np.linalg.qr(B)

    def proj(v):
        return v - Q @ (Q.T @ v)

    def mv(v):
        return sg * proj(dense_matvec(x, k, v))

    def prec(v):
        if precond is None:
            return v.copy()
        return projected_precond(x, deg, precond, v, lowrank)

    w = np.zeros_like(f)
    r = sg * proj(f)
    stop = max(tol * np.linalg.norm(r), atol)
    hist = [np.linalg.norm(r)]
    z = prec(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while hist[-1] > stop and it < maxiter:
        q = mv(p)
        a = rz / (p @ q)
        w = w + a * p
        r = r - a * q
        it += 1
        hist.append(np.linalg.norm(r))
        if hist[-1] <= stop:
            break
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    beta = np.linalg.solve(R, Q.T @ (f - dense_matvec(x, k, w)))
    return w, beta, it, np.array(hist)


# --------------------------------------------------------------------------
# GMRES on the kernel matrix alone, Sec. 3.1
def gmres(x, k: int, b, precond=None, tol: float = 1e-8, atol: float = 0.0, restart: int = 50,
          maxiter: int = 500, check_true: bool = True):
    """Right-preconditioned restarted GMRES for M c = b (Sec. 3.1: the kernel matrix of
    Eq. 1.3 alone, no polynomial block), M dense, preconditioner S = U~ U~^T of
    precond = (nbr, diag, offd) (identity if None).  Textbook GMRES(m): Arnoldi with
    modified Gram-Schmidt on A = M S from v_1 = r / ||r||, the Hessenberg least-squares
    problem min ||beta e_1 - H y|| reduced by Givens rotations, c += S V y at the end of a
    cycle and r = b - M c recomputed.  A cycle ends when its least-squares residual
    estimate is <= max(tol ||b||, atol) (or after `restart` iterations); with check_true the
    solve restarts until the RECOMPUTED residual meets the tolerance, without it it stops
    at the first estimate that does (the count a GMRES library reports).  At most maxiter
    iterations.  Returns (c, iterations, cycles, recomputed ||b - M c||)."""
    x = _f64(x).reshape(-1, 2)
    b = _f64(b)
    n = b.size
    M = dense_matrix(x, k)

    def S(v):
        return v.copy() if precond is None else vecchia_apply(*precond, v)

    stop = max(tol * np.linalg.norm(b), atol)
    c = np.zeros(n)
    r = b.copy()
    beta = np.linalg.norm(r)
    it = cycles = 0
    est = beta
    while beta > stop and it < maxiter and (check_true or est > stop):
        cycles += 1
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j = 0
        while j < m and it < maxiter:
            w = M @ S(V[j])
            for q in range(j + 1):           # modified Gram-Schmidt
                H[q, j] = V[q] @ w
                w = w - H[q, j] * V[q]
            H[j + 1, j] = np.linalg.norm(w)
            for q in range(j):               # earlier rotations on the new column
                a = cs[q] * H[q, j] + sn[q] * H[q + 1, j]
                H[q + 1, j] = -sn[q] * H[q, j] + cs[q] * H[q + 1, j]
                H[q, j] = a
            rr = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (H[j, j] / rr, H[j + 1, j] / rr) if rr > 0 else (1.0, 0.0)
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j += 1
            hn = np.linalg.norm(w)
            if abs(g[j]) <= stop or hn == 0.0:
                break
            V[j] = w / hn
        est = abs(g[j])
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        c = c + S(V[:j].T @ y)
        r = b - M @ c
        beta = np.linalg.norm(r)
    return c, it, cycles, beta


# --------------------------------------------------------------------------
# user-frame wrappers
def fit_dense(points, f, k: int, deg: int | None = None, halfwidth: float = 0.25):
    """Exact fit in the normalised frame, weights returned in the caller's frame:
    w_user = rho^k w_norm (Eq. 2.1 generalised to phi = r^k (log r)); beta is
    the coefficient vector of the monomials in the normalised frame."""
    if deg is None:
        deg = min_poly_degree(k)
    xn, c, rho = normalize(points, halfwidth)
    w, beta = solve_augmented(xn, f, k, deg)
    return {"w_norm": w, "w": w * rho ** k, "beta": beta, "center": c, "rho": rho, "xn": xn,
            "k": k, "deg": deg}


def predict(fit: dict, targets) -> np.ndarray:
    yn = (_f64(targets).reshape(-1, 2) - fit["center"]) * fit["rho"]
    return interpolant(fit["xn"], fit["w_norm"], fit["beta"], fit["k"], fit["deg"], yn)


def nu_alpha_default(k: int):
    """Preconditioner parameters: nu = k/2, the Matern whose leading non-analytic
    term is the PHS kernel (Sec. 2.2, Eq. 2.17 for k = 2: nu = 1, alpha ~= 0.35 in
    [-1/4,1/4]^2); alpha = 0.5 in [-1,1]^2 for k >= 4."""
    return (k / 2.0, 0.35) if k <= 3 else (k / 2.0, 0.5)

