"""Pins for the CPU oracle: each test checks it against something other than
itself -- closed forms, published vectors, identities the paper states,
library routines for special cases, and brute force on tiny inputs."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special
from scipy.spatial.distance import cdist

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def _pts(n, seed=0):
    return np.random.default_rng(seed).random((n, 2))


# ---------------------------------------------------------------- phi and M
def test_phi_closed_forms_345_triangle():
    g = _gold("phi_345.json")
    x = np.array(g["points"], dtype=float)
    for k_s, ent in g["entries"].items():
        k = int(k_s)
        M = oracle.dense_matrix(x, k)
        assert np.all(np.diag(M) == 0.0)
        for ij, expr in ent.items():
            i, j = int(ij[0]), int(ij[1])
            want = eval(expr, {"log": math.log})
            assert M[i, j] == pytest.approx(want, rel=1e-15, abs=0)
            assert M[j, i] == M[i, j]


def test_poly_basis_hand_worked_rows():
    """B of Eq. (1.3) against rows worked by hand: the monomial order (graded
    lexicographic), the x/y roles and the powers are fixed independently of the code."""
    g = _gold("poly_basis.json")
    for case in g["rows"]:
        got = oracle.poly_basis(np.array([case["point"]]), case["deg"])[0]
        assert got.tolist() == [float(v) for v in case["row"]], case
    # several points at once: one row each, in input order
    pts = np.array([c["point"] for c in g["rows"] if c["deg"] == 2])
    want = np.array([c["row"] for c in g["rows"] if c["deg"] == 2], dtype=float)
    assert np.array_equal(oracle.poly_basis(pts, 2), want)
    assert oracle.n_poly(2) == 6 and oracle.n_poly(3) == 10


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_dense_matvec_is_symmetric_form(k):
    x = _pts(300, 1)
    rng = np.random.default_rng(2)
    t, s = rng.standard_normal(300), rng.standard_normal(300)
    a = s @ oracle.dense_matvec(x, k, t)
    b = t @ oracle.dense_matvec(x, k, s)
    assert a == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("k", [2, 4])
def test_scale_law_eq21(k):
    """Eq. (2.1), generalised: M(rho) = rho^k M + rho^k log(rho) [r^k]."""
    x = _pts(120, 3)
    rho = 0.37
    Mr = oracle.dense_matrix(rho * x, k)
    M = oracle.dense_matrix(x, k)
    Dk = cdist(x, x) ** k
    want = rho ** k * M + rho ** k * math.log(rho) * Dk
    assert np.max(np.abs(Mr - want)) <= 1e-13 * np.max(np.abs(want))


def _hadamard_factors(x, power):
    """Low-rank factors of [|x_i - x_j|^power] (Sec. 2, after Eq. 2.4), power 2 or 4."""
    a = (x ** 2).sum(1)
    x1, x2 = x[:, 0], x[:, 1]
    one = np.ones_like(a)
    if power == 2:
        U = np.stack([a, one, -2 * x1, -2 * x2], 1)
        V = np.stack([one, a, x1, x2], 1)
    else:
        U = np.stack([a * a, one, 2 * a, -4 * a * x1, -4 * a * x2, -4 * x1, -4 * x2, 4 * x1 * x1, 8 * x1 * x2, 4 * x2 * x2], 1)
        V = np.stack([one, a * a, a, x1, x2, a * x1, a * x2, x1 * x1, x1 * x2, x2 * x2], 1)
    return U, V


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_hadamard_identity_eq26(k):
    """Eq. (2.6): M t = sum_l D_{u_l} M_core D_{v_l} t with M_core = log r (even k)
    or r (odd k) and U V^T = [r^{2m}]."""
    x = _pts(250, 4) - 0.5
    t = np.random.default_rng(5).standard_normal(250)
    R = cdist(x, x)
    np.fill_diagonal(R, 1.0)
    core = np.log(R) if k % 2 == 0 else R.copy()
    np.fill_diagonal(core, 0.0)
    power = k if k % 2 == 0 else k - 1
    U, V = _hadamard_factors(x, power)
    assert np.allclose(U @ V.T, cdist(x, x) ** power, rtol=0, atol=1e-14)
    got = sum(U[:, l] * (core @ (V[:, l] * t)) for l in range(U.shape[1]))
    want = oracle.dense_matvec(x, k, t)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


# ---------------------------------------------------------------- Matern
def test_bessel_k1_against_scipy():
    xs = np.concatenate([np.logspace(-8, 2, 400), [1.999999, 2.0, 2.000001]])
    for v in xs:
        assert oracle.bessel_k1(v) == pytest.approx(scipy.special.k1(v), rel=2e-14)


def test_bessel_k0_against_scipy():
    xs = np.concatenate([np.logspace(-8, 2, 400), [1.999999, 2.0, 2.000001]])
    for v in xs:
        assert oracle.bessel_k0(v) == pytest.approx(scipy.special.k0(v), rel=2e-14)


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.0, 2.5])
def test_matern_against_general_formula(nu):
    alpha = 3.0
    r = np.linspace(1e-3, 4.0, 200)
    a = alpha * r
    want = 2 ** (1 - nu) / scipy.special.gamma(nu) * a ** nu * scipy.special.kv(nu, a)
    got = oracle.matern(nu, alpha, r)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    assert oracle.matern(nu, alpha, 0.0)[0] == 1.0


def test_matern_small_r_tps_link_eq217():
    """Eq. (2.17): a K_1(a) = 1 + c a^2 + (a^2/2) log(a/2) + O(a^4 log a): the
    remainder after removing the log term, divided by a^2, tends to a constant."""
    a = np.array([1e-2, 5e-3, 2.5e-3, 1.25e-3])
    g = (oracle.matern(1.0, 1.0, a) - 1.0 - a ** 2 / 2 * np.log(a / 2)) / a ** 2
    d = np.abs(np.diff(g))
    assert np.all(d[1:] < d[:-1])
    assert d[-1] < 1e-5
    # with the wrong log coefficient the quotient diverges like log a
    g_bad = (oracle.matern(1.0, 1.0, a) - 1.0 - a ** 2 / 4 * np.log(a / 2)) / a ** 2
    assert abs(g_bad[-1] - g_bad[0]) > 0.5


# ---------------------------------------------------------------- augmented system
def _system(n=160, seed=6, k=2):
    x, _, _ = oracle.normalize(_pts(n, seed), 0.25)
    f = np.sin(7 * x[:, 0]) + np.cos(5 * x[:, 1]) + x[:, 0] * x[:, 1]
    return x, f


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_augmented_solvers_agree(k):
    deg = oracle.min_poly_degree(k)
    x, f = _system(k=k)
    w1, b1 = oracle.solve_augmented(x, f, k, deg)
    w2, b2 = oracle.solve_qperp(x, f, k, deg)
    M = oracle.dense_matrix(x, k)
    B = oracle.poly_basis(x, deg)
    S = B.shape[1]
    A = np.block([[M, B], [B.T, np.zeros((S, S))]])
    sol = scipy.linalg.solve(A, np.concatenate([f, np.zeros(S)]), assume_a="sym")
    w3, b3 = sol[: len(f)], sol[len(f):]
    kappa = np.linalg.cond(A)
    tol = max(kappa, 1.0) * 1e-15 * 10
    for w, b in [(w2, b2), (w3, b3)]:
        assert np.linalg.norm(w - w1) <= tol * np.linalg.norm(w1)
        assert np.linalg.norm(b - b1) <= tol * max(np.linalg.norm(b1), 1.0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_interpolation_invariants(k):
    deg = oracle.min_poly_degree(k)
    x, f = _system(k=k)
    w, beta = oracle.solve_augmented(x, f, k, deg)
    B = oracle.poly_basis(x, deg)
    fhat = oracle.interpolant(x, w, beta, k, deg, x)
    assert np.max(np.abs(fhat - f)) <= 1e-9 * np.max(np.abs(f))
    assert np.linalg.norm(B.T @ w) <= 1e-10 * np.linalg.norm(w) * np.linalg.norm(B)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_polynomial_reproduction(k):
    deg = oracle.min_poly_degree(k)
    x, _ = _system(k=k)
    B = oracle.poly_basis(x, deg)
    coef = np.arange(1, B.shape[1] + 1, dtype=float) * np.array([1, -1] * 5)[: B.shape[1]]
    f = B @ coef
    w, beta = oracle.solve_augmented(x, f, k, deg)
    M = oracle.dense_matrix(x, k)
    S = B.shape[1]
    kappa = np.linalg.cond(np.block([[M, B], [B.T, np.zeros((S, S))]]))
    # exact answer: w = 0, beta = coef; the LU solve reaches it to kappa * eps
    assert np.max(np.abs(w)) <= 10 * kappa * 2.2e-16 * np.max(np.abs(f))
    assert np.allclose(beta, coef, rtol=0, atol=10 * kappa * 2.2e-16 * np.max(np.abs(coef)))
    y = np.random.default_rng(1).random((50, 2)) * 0.5 - 0.25
    assert np.allclose(oracle.interpolant(x, w, beta, k, deg, y), oracle.poly_basis(y, deg) @ coef, atol=1e-9)


def test_n_equals_S_gives_zero_weights():
    x = np.array([[0.0, 0.0], [0.2, 0.05], [-0.1, 0.2]])
    f = np.array([1.0, -2.0, 0.5])
    w, beta = oracle.solve_augmented(x, f, 2, 1)
    assert np.max(np.abs(w)) < 1e-14
    assert np.allclose(oracle.poly_basis(x, 1) @ beta, f, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_qperp_projection_is_positive_definite(k):
    deg = oracle.min_poly_degree(k)
    x, _ = _system(n=120, k=k)
    M = oracle.dense_matrix(x, k)
    B = oracle.poly_basis(x, deg)
    Qc, _ = np.linalg.qr(B, mode="complete")
    Qp = Qc[:, B.shape[1]:]
    ev = np.linalg.eigvalsh(Qp.T @ M @ Qp)
    # Sec. 1: Q_perp^T M Q_perp is definite; positive for the thin-plate spline
    assert np.all(oracle.cpd_sign(k) * ev > 0)
    if k == 2:
        assert oracle.cpd_sign(k) == 1


def test_fit_is_scale_invariant():
    """Sec. 2, Eq. (2.1): rescaling the points changes neither the interpolant nor
    the caller-frame weights."""
    w_ = synth.workload("uniform_tps", n=200, n_targets=50)
    a = oracle.fit_dense(w_["points"], w_["f"], 2, halfwidth=0.25)
    b = oracle.fit_dense(w_["points"], w_["f"], 2, halfwidth=1.0)
    assert np.allclose(a["w"], b["w"], rtol=1e-8, atol=1e-8 * np.abs(a["w"]).max())
    fa, fb = oracle.predict(a, w_["targets"]), oracle.predict(b, w_["targets"])
    assert np.max(np.abs(fa - fb)) <= 1e-9 * np.max(np.abs(fa))


# ---------------------------------------------------------------- ordering and neighbours
def test_splitmix64_published_vectors():
    g = _gold("splitmix64.json")
    for i, h in enumerate(g["outputs_hex"]):
        assert oracle.splitmix64(g["seed"], i) == int(h, 16)


def test_random_order_sorted_by_key():
    order = oracle.random_order(1000, 77)
    assert sorted(order.tolist()) == list(range(1000))
    keys = [oracle.splitmix64(77, int(i)) for i in order]
    assert all(keys[i] < keys[i + 1] for i in range(999))


def test_knn_golden_lattice():
    g = _gold("knn_lattice.json")
    x = np.array(g["points"], dtype=float)
    for case in g["cases"]:
        got = oracle.knn_prev(x, np.array(case["order"]), g["m"])
        assert got.tolist() == case["nbr"]


def test_knn_against_independent_brute_force():
    rng = np.random.default_rng(8)
    x = np.round(rng.random((300, 2)) * 16) / 16  # lattice: many exact ties
    order = oracle.random_order(300, 3)
    m = 7
    got = oracle.knn_prev(x, order, m)
    rank = np.empty(300, dtype=np.int64)
    rank[order] = np.arange(300)
    for i in range(300):
        prev = order[: rank[i]]
        d = ((x[prev] - x[i]) ** 2).sum(1)
        sel = prev[np.lexsort((rank[prev], d))][:m]
        want = np.full(m, -1)
        want[: len(sel)] = sel
        assert got[i].tolist() == want.tolist()


def test_maxmin_golden_line():
    g = _gold("maxmin_line.json")
    order, dm = oracle.maxmin_order(np.array(g["points"], dtype=float))
    assert order.tolist() == g["order"]
    assert np.isinf(dm[0]) and dm[1:].tolist() == g["dmin2"][1:]


def test_maxmin_properties():
    x = _pts(400, 9)
    order, dm = oracle.maxmin_order(x)
    assert sorted(order.tolist()) == list(range(400))
    assert np.all(np.diff(dm[1:]) <= 0)
    for r in [1, 7, 50, 399]:
        d = ((x[order[:r]] - x[order[r]]) ** 2).sum(1).min()
        assert d == dm[r]
        rest = order[r:]
        dd = ((x[rest][:, None, :] - x[order[:r]][None, :, :]) ** 2).sum(2).min(1)
        assert dd.max() == dm[r]
    c = (x.min(0) + x.max(0)) / 2
    assert order[0] == np.argmin(((x - c) ** 2).sum(1))


# ---------------------------------------------------------------- Vecchia factor
@pytest.mark.parametrize("nu,alpha", [(1.5, 6.0), (1.0, 4.0)])
def test_vecchia_full_conditioning_is_exact_inverse(nu, alpha):
    """Fig. 1: with sigma(j) = all previous points, U U^T = Sigma^{-1} exactly."""
    n = 120
    x = _pts(n, 10) * 0.5
    order = oracle.random_order(n, 5)
    nbr = oracle.knn_prev(x, order, n - 1)
    diag, offd, nj = oracle.vecchia_factor(x, order, nbr, n - 1, nu, alpha)
    assert nj == 0
    U = oracle.vecchia_dense(nbr, diag, offd)
    with np.errstate(invalid="ignore"):  # the diagonal (0 x inf) is set to K(0) = 1 below
        Sigma = 2 ** (1 - nu) / scipy.special.gamma(nu) * (alpha * cdist(x, x)) ** nu * scipy.special.kv(nu, alpha * cdist(x, x) + 1e-300)
    np.fill_diagonal(Sigma, 1.0)
    Sinv = np.linalg.inv(Sigma)
    assert np.linalg.norm(U @ U.T - Sinv) <= 1e-8 * np.linalg.norm(Sinv)
    # and U is triangular in the enumeration order
    Up = U[np.ix_(order, order)]
    assert np.allclose(Up, np.triu(Up))


def test_vecchia_apply_matches_dense_factor():
    n, m = 200, 10
    x = _pts(n, 11)
    order = oracle.random_order(n, 1)
    nbr = oracle.knn_prev(x, order, m)
    diag, offd, _ = oracle.vecchia_factor(x, order, nbr, m, 1.5, 10.0)
    U = oracle.vecchia_dense(nbr, diag, offd)
    r = np.random.default_rng(0).standard_normal(n)
    assert np.allclose(oracle.vecchia_apply(nbr, diag, offd, r), U @ (U.T @ r), rtol=1e-13, atol=1e-12)


# ---------------------------------------------------------------- projected preconditioner
def _small_factor(n=60, m=8, seed=21, deg=1):
    x = _pts(n, seed) * 0.5
    order = oracle.random_order(n, 3)
    nbr = oracle.knn_prev(x, order, m)
    d, o, _ = oracle.vecchia_factor(x, order, nbr, m, 1.0, 4.0)
    return x, (nbr, d, o)


@pytest.mark.parametrize("deg", [1, 2])
def test_lowrank_precond_solves_the_saddle_point_system(deg):
    """Sec. 2.2's low-rank term: the preconditioned vector is the z-block of the dense
    saddle-point solve [S~ B; B^T 0][z; lam] = [v; 0], with S~ = (U U^T)^{-1} formed and
    the augmented matrix factored directly (no Schur formula)."""
    x, fac = _small_factor(deg=deg)
    n = len(x)
    B = oracle.poly_basis(x, deg)
    S = B.shape[1]
    U = oracle.vecchia_dense(*fac)
    St = np.linalg.inv(U @ U.T)
    v = np.random.default_rng(4).standard_normal(n)
    A = np.block([[St, B], [B.T, np.zeros((S, S))]])
    want = np.linalg.solve(A, np.concatenate([v, np.zeros(S)]))[:n]
    got = oracle.projected_precond(x, deg, fac, v, True)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
    assert np.linalg.norm(B.T @ got) <= 1e-10 * np.linalg.norm(B) * np.linalg.norm(got)


def test_lowrank_precond_inverts_the_projected_matern():
    """On range(P) the low-rank form is the inverse of Q_perp^T S~ Q_perp (checked in
    the coordinates of a complete QR of B); the plain form is Q_perp^T S~^{-1} Q_perp,
    which differs from it (the two agree only when S~^{-1} maps range(B) to itself)."""
    x, fac = _small_factor()
    n = len(x)
    B = oracle.poly_basis(x, 1)
    Qc, _ = np.linalg.qr(B, mode="complete")
    Qp = Qc[:, 3:]
    U = oracle.vecchia_dense(*fac)
    St = np.linalg.inv(U @ U.T)
    u = np.random.default_rng(5).standard_normal(n - 3)
    v = Qp @ u
    z = oracle.projected_precond(x, 1, fac, v, True)
    assert np.linalg.norm(Qp.T @ St @ Qp @ (Qp.T @ z) - u) <= 1e-8 * np.linalg.norm(u)
    assert np.linalg.norm(z - Qp @ (Qp.T @ z)) <= 1e-10 * np.linalg.norm(z)
    zp = oracle.projected_precond(x, 1, fac, v, False)
    assert np.linalg.norm(zp - Qp @ (Qp.T @ (U @ (U.T @ v)))) <= 1e-12 * np.linalg.norm(zp)
    assert np.linalg.norm(zp - z) > 1e-3 * np.linalg.norm(z)


# ---------------------------------------------------------------- PCG
@pytest.mark.parametrize("lowrank", [False, True])
def test_pcg_converges_to_direct_solution_either_form(lowrank):
    """Both preconditioner forms converge to the direct solution; the low-rank form
    needs no more iterations than the plain one."""
    w_ = synth.workload("uniform_tps", n=600, n_targets=10)
    x, c, rho = oracle.normalize(w_["points"], 0.25)
    f = w_["f"]
    order = oracle.hmaxmin_order(x, 1)[0]
    nbr = oracle.knn_prev(x, order, 30)
    d, o, _ = oracle.vecchia_factor(x, order, nbr, 30, 1.0, 0.35)
    w, beta, it, hist = oracle.pcg(x, f, 2, 1, (nbr, d, o), tol=1e-12, maxiter=200, lowrank=lowrank)
    w0, b0 = oracle.solve_augmented(x, f, 2, 1)
    assert hist[-1] <= 1e-12 * hist[0]
    y = (w_["targets"] - c) * rho
    a = oracle.interpolant(x, w, beta, 2, 1, y)
    b = oracle.interpolant(x, w0, b0, 2, 1, y)
    assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))
    _, _, it_plain, _ = oracle.pcg(x, f, 2, 1, (nbr, d, o), tol=1e-12, maxiter=200, lowrank=False)
    assert it <= it_plain


def test_pcg_converges_to_direct_solution():
    """Sec. 2.2 / Sec. 3: the Vecchia-preconditioned CG (nu = 1, alpha = 0.35,
    points in [-1/4,1/4]^2, m = 30, random order) converges in few iterations to
    the direct solution; plain CG needs far more."""
    w_ = synth.workload("uniform_tps", n=600, n_targets=10)
    x, c, rho = oracle.normalize(w_["points"], 0.25)
    f = w_["f"]
    order = oracle.random_order(len(f), 1)
    nbr = oracle.knn_prev(x, order, 30)
    d, o, _ = oracle.vecchia_factor(x, order, nbr, 30, 1.0, 0.35)
    w, beta, it, hist = oracle.pcg(x, f, 2, 1, (nbr, d, o), tol=1e-12, maxiter=200)
    w0, b0 = oracle.solve_augmented(x, f, 2, 1)
    assert hist[-1] <= 1e-12 * hist[0]
    assert it < 25
    y = (w_["targets"] - c) * rho
    a = oracle.interpolant(x, w, beta, 2, 1, y)
    b = oracle.interpolant(x, w0, b0, 2, 1, y)
    assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))
    _, _, it_plain, _ = oracle.pcg(x, f, 2, 1, None, tol=1e-6, maxiter=2000)
    _, _, it_pre, _ = oracle.pcg(x, f, 2, 1, (nbr, d, o), tol=1e-6, maxiter=2000)
    assert it_plain > 5 * it_pre


# ---------------------------------------------------------------- hierarchical maximin
def test_hmaxmin_hand_worked_square():
    """Corners of the unit square plus its centre (E = 1): level 0 picks the centre
    (nearest to (1/2, 1/2)); at level 1 the centre's quadrant (1, 1) inherits it, so the
    other three corners are picked there; the corner (1, 1) shares that quadrant and is
    picked at level 2, where it and the centre fall in different cells ((3, 3) vs (2, 2))."""
    x = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [0.5, 0.5]], dtype=float)
    order, level = oracle.hmaxmin_order(x, 3)
    assert level.tolist() == [1, 1, 1, 2, 0]
    assert order[0] == 4 and sorted(order[1:4].tolist()) == [0, 1, 2] and order[4] == 3
    h = [oracle.splitmix64(3, i) >> 7 for i in (0, 1, 2)]
    assert order[1:4].tolist() == [i for _, i in sorted(zip(h, (0, 1, 2)))]


@pytest.mark.parametrize("clustered", [False, True])
def test_hmaxmin_one_new_point_per_cell_per_level(clustered):
    """Invariant of the definition: the points of level <= L are exactly one per
    non-empty level-L cell, and the level-0 point is the point nearest the centre of
    the bounding square (brute force)."""
    rng = np.random.default_rng(21)
    x = rng.random((2000, 2))
    if clustered:
        x[:600] = 0.3 + 0.01 * rng.standard_normal((600, 2))
    order, level = oracle.hmaxmin_order(x, 5)
    assert np.array_equal(np.sort(order), np.arange(len(x)))
    assert np.all(np.diff(level[order]) >= 0)
    xmin, ymin = x.min(0)
    E = max(np.ptp(x[:, 0]), np.ptp(x[:, 1]))
    ix = np.clip(np.floor((x[:, 0] - xmin) * (2.0 ** 30 / E)), 0, 2 ** 30 - 1).astype(np.int64)
    iy = np.clip(np.floor((x[:, 1] - ymin) * (2.0 ** 30 / E)), 0, 2 ** 30 - 1).astype(np.int64)
    for L in range(0, 31, 3):
        cells = set(zip((ix >> (30 - L)).tolist(), (iy >> (30 - L)).tolist()))
        picked = np.nonzero(level <= L)[0]
        assert len(picked) == len(cells)
        assert len(set(zip((ix[picked] >> (30 - L)).tolist(), (iy[picked] >> (30 - L)).tolist()))) == len(cells)
    c = np.array([xmin + E / 2, ymin + E / 2])
    assert order[0] == np.argmin(((x - c) ** 2).sum(1))


# ---------------------------------------------------------------- dyadic approximate maximin
def _prefix_ratios(x, order):
    """Brute force: for each rank k >= 1, the squared distance of order[k] to the
    points of smaller rank, and the largest such distance over all points of rank >= k."""
    n = len(order)
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    dmin = np.full(n, np.inf)
    got, best = [], []
    for k in range(n):
        p = order[k]
        if k:
            rest = order[k:]
            got.append(dmin[p])
            best.append(dmin[rest].max())
        dmin = np.minimum(dmin, d2[p])
    return np.array(got), np.array(best)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "lattice"])
def test_amaxmin_half_maximin_property(kind):
    """Each point, when appended, is at least half as far from the points before it as
    the farthest point still to come (exact maxmin: equally far); checked by brute
    force, independently of the level/pass bookkeeping."""
    rng = np.random.default_rng(7)
    if kind == "uniform":
        x = rng.random((700, 2))
    elif kind == "clustered":
        c = rng.random((6, 2))
        x = np.concatenate([rng.random((300, 2)), (c[:, None, :] + 0.01 * rng.standard_normal((6, 60, 2))).reshape(-1, 2)])
    else:
        g = np.arange(24) / 23.0
        x = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    order, level, l2 = oracle.amaxmin_order(x)
    assert sorted(order.tolist()) == list(range(len(x)))
    got, best = _prefix_ratios(x, order)
    assert np.all(got >= 0.25 * best * (1 - 1e-12)), np.min(got / best)
    # the recorded selection distance is the one at the start of the point's pass:
    # points accepted before it in the same pass can only be closer
    assert np.all(got <= l2[1:])
    first_of_pass = np.r_[True, (level[2:] != level[1:-1]) | (l2[2:] > l2[1:-1])]
    assert np.array_equal(got[first_of_pass], l2[1:][first_of_pass])
    # levels are non-decreasing along the order, and at level L the selection distance
    # is in [c_L, 2 c_L)
    assert np.all(np.diff(level) >= 0)
    E = max(np.ptp(x[:, 0]), np.ptp(x[:, 1]))
    c = E * 2.0 ** -level[1:].astype(float)
    assert np.all(got >= c * c) and np.all(got < 4 * c * c)


def test_amaxmin_hand_worked_line():
    """Five points on a line, E = 1: the first is 0.5 (nearest the centre (0.5, 0));
    level 0 (c = 1) has no candidate; level 1 (c = 1/2): 0 and 1 are 0.5 away, in
    different cells, accepted in index order (ties); level 2 (c = 1/4): 0.3 is 0.2 from
    0.5 (< 1/4, no), 0.8 is 0.2 from 1 (no): level 3 (c = 1/8): both candidates,
    different cells, 0.3 (l2 = 0.04) and 0.8 (l2 = 0.04) tie, index order."""
    x = np.array([[0.0, 0.0], [0.3, 0.0], [0.5, 0.0], [0.8, 0.0], [1.0, 0.0]])
    order, level, l2 = oracle.amaxmin_order(x)
    assert order.tolist() == [2, 0, 4, 1, 3]
    assert level.tolist() == [-1, 1, 1, 3, 3]


def test_amaxmin_one_eligible_point_per_cell():
    """A = (0.5, 0.5) is first (the centre).  At level 1 (c = 1/2, c^2 = 1/4) B = (0, 0)
    and C = (0.2, 0) share cell (0, 0) and are both candidates (l2 = 0.5 and 0.34); only
    B, the farther, is eligible; D = (1, 1) in cell (1, 1) is accepted in the same pass
    (ties with B on l2 = 0.5, larger index).  C is then 0.2 from B (l2 = 0.04) and is
    first a candidate at level 3 (c^2 = 1/64)."""
    x = np.array([[0.5, 0.5], [0.0, 0.0], [0.2, 0.0], [1.0, 1.0]])
    order, level, _ = oracle.amaxmin_order(x)
    assert order.tolist() == [0, 1, 3, 2]
    assert level.tolist() == [-1, 1, 1, 3]


def test_amaxmin_conflict_between_adjacent_cells():
    """A = (0.5, 0.5) first.  At level 1 the eligible points R = (0, 1), S = (1, 1)
    (l2 = 0.5), P = (0.45, 0) and Q = (0.55, 0) (l2 = 0.2525) sit in four different
    cells and are visited R, S, P, Q; Q is 0.1 from the accepted P (0.01 < c^2 = 1/4),
    so it is rejected, its l2 drops to 0.01 and it waits until level 4 (c^2 = 1/256)."""
    x = np.array([[0.5, 0.5], [0.45, 0.0], [0.55, 0.0], [0.0, 1.0], [1.0, 1.0]])
    order, level, l2 = oracle.amaxmin_order(x)
    assert order.tolist() == [0, 3, 4, 1, 2]
    assert level.tolist() == [-1, 1, 1, 1, 4]
    assert l2[4] == (0.55 - 0.45) ** 2


def test_dense_eval_abs_is_abs_matrix_times_abs_weights():
    """The rounding scale sum_j |w_j phi_ij| equals |M| |w| built from the dense matrix
    (another route), and bounds |dense_eval| with equality for one-signed terms."""
    rng = np.random.default_rng(12)
    x = rng.random((300, 2))
    w = rng.standard_normal(300)
    for k in (1, 2, 3, 4):
        M = oracle.dense_matrix(x, k)
        got = oracle.dense_eval_abs(x, w, k, x[:40])
        assert np.allclose(got, np.abs(M[:40]) @ np.abs(w), rtol=1e-13, atol=0)
        assert np.all(np.abs(oracle.dense_eval(x, w, k, x[:40])) <= got * (1 + 1e-13))
    M = oracle.dense_matrix(x, 3)  # r^3 >= 0: with w >= 0 every term has one sign
    assert np.allclose(oracle.dense_eval_abs(x, np.abs(w), 3, x[:10]), M[:10] @ np.abs(w), rtol=1e-13)


try:
    from hypothesis import given, settings, strategies as hst
    HAVE_HYPOTHESIS = True
except ImportError:  # pragma: no cover
    HAVE_HYPOTHESIS = False

if HAVE_HYPOTHESIS:
    @settings(max_examples=60, deadline=None)
    @given(n=hst.integers(2, 70), seed=hst.integers(0, 2**31 - 1), kind=hst.sampled_from(["uniform", "dups", "grid"]))
    def test_amaxmin_properties_random(n, seed, kind):
        """Random small sets (with coincident points and lattices): the order is a
        permutation, levels never decrease, and every point before the coincident tail
        is at least half as far from its predecessors as the farthest point still to
        come (brute force)."""
        rng = np.random.default_rng(seed)
        if kind == "uniform":
            x = rng.random((n, 2))
        elif kind == "dups":
            x = rng.random((max(1, n // 2), 2))
            x = x[rng.integers(0, len(x), n)]
        else:
            g = int(np.ceil(np.sqrt(n)))
            x = np.stack(np.meshgrid(np.arange(g), np.arange(g)), -1).reshape(-1, 2)[:n] / max(g - 1, 1)
        order, level, _ = oracle.amaxmin_order(x)
        assert sorted(order.tolist()) == list(range(n))
        assert np.all(np.diff(level) >= 0)
        head = int(np.sum(level < 31))
        d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
        dmin = d2[order[0]].copy()
        for k in range(1, head):
            rest = order[k:head]  # coincident tail points (distance 0) are left out
            assert dmin[order[k]] >= 0.25 * dmin[rest].max() * (1 - 1e-12)
            dmin = np.minimum(dmin, d2[order[k]])


# ---------------------------------------------------------------- GMRES on M alone (Sec. 3.1)
def _small_precond(x, m=8, alpha=0.35):
    xn, _, _ = oracle.normalize(x, 0.25)
    order = oracle.random_order(len(x), 3)
    nbr = oracle.knn_prev(xn, order, m)
    d, o, _ = oracle.vecchia_factor(xn, order, nbr, m, 1.0, alpha)
    return nbr, d, o


@pytest.mark.parametrize("j", [1, 2, 3, 5])
def test_gmres_minimal_residual_property(j):
    """After j iterations (one cycle) GMRES's iterate minimises ||b - M c|| over
    c in S K_j(M S, b): checked against a least-squares solve on an explicit, separately
    orthonormalised Krylov basis [b, (M S) b, ..., (M S)^(j-1) b]."""
    x = _pts(60, 21)
    b = np.random.default_rng(22).standard_normal(60)
    pre = _small_precond(x)
    M = oracle.dense_matrix(x, 2)
    S = lambda v: oracle.vecchia_apply(*pre, v)  # noqa: E731
    c, it, cyc, res = oracle.gmres(x, 2, b, pre, tol=1e-300, restart=50, maxiter=j)
    assert it == j and cyc == 1
    K = [b.copy()]
    for _ in range(j - 1):
        K.append(M @ S(K[-1]))
    Qk, _ = np.linalg.qr(np.array(K).T)
    A = np.array([M @ S(Qk[:, i]) for i in range(j)]).T
    y, *_ = np.linalg.lstsq(A, b, rcond=None)
    want = np.linalg.norm(b - A @ y)
    assert res == pytest.approx(want, rel=1e-9, abs=1e-12 * np.linalg.norm(b))


def test_gmres_converges_to_direct_solve():
    """On a small problem GMRES with the Vecchia right preconditioner reaches the dense
    solution of M c = b; without check_true it stops at the first estimate below tol."""
    x = _pts(250, 23)
    b = np.random.default_rng(24).standard_normal(250)
    pre = _small_precond(x, m=20)
    M = oracle.dense_matrix(x, 2)
    c_ref = np.linalg.solve(M, b)
    c, it, cyc, res = oracle.gmres(x, 2, b, pre, tol=1e-11, restart=60, maxiter=400)
    assert res <= 1e-11 * np.linalg.norm(b) and np.linalg.norm(b - M @ c) == pytest.approx(res, rel=1e-6)
    assert np.linalg.norm(c - c_ref) <= 1e-11 * np.linalg.cond(M) * np.linalg.norm(c_ref)
    c2, it2, cyc2, res2 = oracle.gmres(x, 2, b, pre, tol=1e-6, restart=60, maxiter=400, check_true=False)
    assert cyc2 == 1 and it2 <= it
    # without the preconditioner the same problem takes more iterations
    c3, it3, _, _ = oracle.gmres(x, 2, b, None, tol=1e-6, restart=250, maxiter=400, check_true=False)
    assert it3 > it2
