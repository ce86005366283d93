"""The serving engine (phs_server_*): continuous batching of interpolation requests.
A job's result must not depend on the other jobs it shares the GPU with: each request
served in a mix of requests of different sizes and spline orders is compared with the
same request run alone through phs_fit + phs_eval -- the engine runs the same steps with
the same arithmetic, so the results are identical bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402


@pytest.fixture(scope="module")
def phs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_11462_b300 import build
    build.build()
    import paper_2608_11462_b300 as mod
    return mod


def _requests():
    """Mixed sizes, orders and geometries (config-5 style: uniform or clustered points,
    bump-sum fields, minimal polynomial block)."""
    out = []
    rng = np.random.default_rng(500)
    for i, (n, k) in enumerate([(800, 2), (3000, 1), (1500, 3), (12000, 2), (6000, 3), (20000, 2), (2500, 1),
                                (9000, 2), (4000, 3), (16000, 2)]):
        if i % 2:
            pts = rng.random((n, 2))
        else:
            pts = synth.gaussian_mixture(n, 6, 0.02, 0.1, 0.9, rng)
        f = synth.bump_field(rng)(pts)
        tg = rng.random((100, 2))
        out.append((pts, f, tg, k))
    return out


def _alone(phs, pts, f, tg, k, opts):
    plan = phs.Plan(torch.tensor(pts, device="cuda"), k, vecchia_m=20, opts=opts)
    w, beta, info = plan.fit(torch.tensor(f, device="cuda"))
    pred = plan.eval(w, beta, torch.tensor(tg, device="cuda"))
    torch.cuda.synchronize()
    r = (w.cpu().numpy(), beta.cpu().numpy(), pred.cpu().numpy(), info)
    plan.close()
    return r


@pytest.mark.parametrize("max_active", [8, 1])
def test_server_results_identical_alone_and_in_the_mix(phs, max_active):
    reqs = _requests()
    ref = [_alone(phs, p, f, t, k, phs.options(k, maxiter=400)) for p, f, t, k in reqs]
    sv = phs.Server(max_active=max_active, setup_threads=4)
    ids = [sv.submit(p, f, t, k, vecchia_m=20, opts=phs.options(k, maxiter=400)) for p, f, t, k in reqs]
    got = [sv.wait(i) for i in ids]
    st = sv.stats()
    sv.close()
    for (w0, b0, p0, i0), (w1, b1, p1, i1, times) in zip(ref, got):
        assert i1["iters"] == i0["iters"] and i1["converged"] == 1
        assert np.array_equal(w1, w0) and np.array_equal(b1, b0) and np.array_equal(p1, p0)
        assert times[0] <= times[1] <= times[2] <= times[3]
    print("server stats", st)
    assert st["completed"] == len(reqs)
    if max_active > 1:
        assert st["max_concurrent"] > 1  # jobs really shared ticks
    else:
        assert st["max_concurrent"] == 1


def test_server_job_matches_dense_oracle(phs):
    """One served request against the dense FP64 solve of the oracle (Eq. 1.3)."""
    w_ = synth.workload("uniform_tps", n=1200, n_targets=200)
    sv = phs.Server(max_active=4)
    jid = sv.submit(w_["points"], w_["f"], w_["targets"], 2, vecchia_m=10, opts=phs.options(2, tol=1e-10))
    w, beta, pred, info, _ = sv.wait(jid)
    sv.close()
    ref = oracle.fit_dense(w_["points"], w_["f"], 2)
    want = oracle.predict(ref, w_["targets"])
    assert np.max(np.abs(pred - want)) <= 1e-8 * np.max(np.abs(want))


def test_server_admission_respects_memory_budget(phs):
    """With a budget that holds one 60k-point job at a time, the engine runs them one after
    another (never two in a tick) and still completes all of them."""
    rng = np.random.default_rng(9)
    jobs = [(rng.random((60000, 2)), 2) for _ in range(3)]
    budget = 200 * 1024 * 1024
    sv = phs.Server(memory_budget=budget, max_active=8)
    ids = []
    for pts, k in jobs:
        f = np.sin(4 * pts[:, 0]) * np.cos(3 * pts[:, 1])
        ids.append(sv.submit(pts, f, rng.random((50, 2)), k, vecchia_m=20))
    res = [sv.wait(i) for i in ids]
    st = sv.stats()
    sv.close()
    print("budget stats", st)
    assert st["completed"] == 3 and st["max_concurrent"] == 1
    assert all(r[3]["converged"] == 1 for r in res)
    # each job was admitted only after the previous one finished
    t = [r[4] for r in res]
    for a, b in zip(t, t[1:]):
        assert b[1] >= a[3] - 1e-3


def test_batch_of_higher_order_jobs(phs):
    """Config-4 style batch as in Sec. 3.3: k = 4 and 5 (quadratic block), Franke
    function, Sobol points, precision 4 (float-float inside FP64 refinement for k = 4,
    the FP64 operator for k = 5), leaf capacity autotuned (leaf_cap = 0), all jobs
    submitted at once.  Every job converges to 1e-8 and equals the same job run alone
    through phs_fit + phs_eval, and the smallest matches the dense oracle at held-out
    points within 1e-6 relative (the fit stops at 1e-8 of ||P f||; these orders are so
    ill-conditioned that the interpolant's error exceeds the residual's)."""
    jobs = synth.batch_jobs(8, seed=77, n_lo=2000, n_hi=20000, n_targets=60)
    opts = lambda k: phs.options(k, precision=4, leaf_cap=0, tol=1e-8, maxiter=400)  # noqa: E731
    ref = [_alone(phs, j["points"], j["f"], j["targets"], j["k"], opts(j["k"])) for j in jobs]
    sv = phs.Server(max_active=8)
    ids = [sv.submit(j["points"], j["f"], j["targets"], j["k"], vecchia_m=20, opts=opts(j["k"])) for j in jobs]
    got = [sv.wait(i) for i in ids]
    st = sv.stats()
    sv.close()
    print("batch stats", st, [(j["k"], len(j["f"]), g[3]["iters"], g[3]["outer_iters"]) for j, g in zip(jobs, got)])
    for (w0, b0, p0, i0), (w1, b1, p1, i1, _) in zip(ref, got):
        assert i1["converged"] == 1 and i1["iters"] == i0["iters"] and i1["outer_iters"] == i0["outer_iters"]
        assert np.array_equal(w1, w0) and np.array_equal(b1, b0) and np.array_equal(p1, p0)
    small = min(range(len(jobs)), key=lambda i: len(jobs[i]["f"]))
    j = jobs[small]
    dense = oracle.fit_dense(j["points"], j["f"], j["k"], halfwidth=1.0)
    want = oracle.predict(dense, j["targets"])
    err = np.max(np.abs(got[small][2] - want)) / np.max(np.abs(want))
    print("smallest job vs dense oracle", len(j["f"]), j["k"], err)
    assert err <= 1e-6
