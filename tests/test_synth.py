"""CPU checks that the seeded generators produce the workloads the benchmark and the
full-size parity tests are described with (sizes, mixes, bounds, fields, determinism)."""
import numpy as np
import pytest

import synth


def test_tps_1m_recipe():
    w = synth.workload("tps_1m")
    p, f, t = w["points"], w["f"], w["targets"]
    assert p.shape == (1_048_576, 2) and t.shape == (10_000, 2) and w["k"] == 2
    assert p.min() >= 0.0 and p.max() <= 1.0 and t.min() >= 0.0 and t.max() <= 1.0
    # 943,718 uniform points first, then 104,858 clustered ones in 50 equal clusters
    uni, cl = p[:943_718], p[943_718:]
    assert len(cl) == 104_858
    # the clustered tail is far denser than the uniform head: its points have much closer
    # nearest neighbours (sigma = 0.005 against a uniform spacing of ~1e-3)
    from scipy.spatial import cKDTree
    d_uni = cKDTree(uni[:20000]).query(uni[:2000], k=2)[0][:, 1].mean()
    d_cl = cKDTree(cl).query(cl[:2000], k=2)[0][:, 1].mean()
    assert d_cl < 0.3 * d_uni
    x, y = p[:, 0], p[:, 1]
    assert np.array_equal(f, np.exp(-8 * ((x - 0.3) ** 2 + (y - 0.6) ** 2)) + np.sin(10 * x * y))
    # deterministic
    w2 = synth.workload("tps_1m", n=4096)
    w3 = synth.workload("tps_1m", n=4096)
    assert np.array_equal(w2["points"], w3["points"]) and np.array_equal(w2["targets"], w3["targets"])


def test_small_workloads_recipe():
    u = synth.workload("uniform_tps")
    assert u["points"].shape == (1500, 2) and u["targets"].shape == (500, 2) and u["k"] == 2
    x, y = u["points"][:, 0], u["points"][:, 1]
    assert np.array_equal(u["f"], np.sin(4 * x) * np.cos(3 * y) + 0.5 * x ** 2)
    c = synth.workload("cubic_mix", n=20_000)
    assert c["points"].shape == (20_000, 2) and c["k"] == 3
    assert c["points"].min() >= 0.0 and c["points"].max() <= 1.0
    assert synth.workload("cubic_mix")["points"].shape == (100_000, 2)


def test_franke_as_printed():
    """Sec. 3.3's form of the Franke function at hand-checked points: at 9x = c_1 = (2, 2)
    the first term is 0.75 and the others follow from their metrics."""
    import math
    p = np.array([[2 / 9, 2 / 9]])
    want = (0.75 + 0.75 * math.exp(-(3 ** 2) / 49 - (3 ** 2) / 10) + 0.5 * math.exp(-(25 + 1) / 4)
            - 0.2 * math.exp(-4 - 25))
    assert synth.franke(p)[0] == pytest.approx(want, rel=1e-15)


def test_request_streams():
    reqs = synth.serving_requests(40, seed=3)
    assert all(1000 <= len(r["f"]) <= 500_000 and r["k"] in (1, 2, 3) for r in reqs)
    assert {r["k"] for r in reqs} == {1, 2, 3}
    jobs = synth.batch_jobs(20, seed=4, n_hi=20_000)
    assert all(j["k"] in (4, 5) and 2000 <= len(j["f"]) <= 20_000 for j in jobs)
    t = synth.poisson_arrivals(2000, 10.0, seed=1)
    assert np.all(np.diff(t) > 0) and abs(t[-1] / 2000 - 0.1) < 0.01


def test_sobol_points_form_a_net():
    """Scrambled 2D Sobol points (the Sec. 3.3 samples): the first 2^10 form a (0, 10, 2)-net
    in base 2, so every 32 x 32 grid cell (volume 2^-10) holds exactly one point."""
    p = synth.sobol(1024, seed=5)
    assert p.shape == (1024, 2) and np.all((p >= 0) & (p < 1))
    cell = np.floor(p * 32).astype(int)
    counts = np.zeros((32, 32), int)
    np.add.at(counts, (cell[:, 0], cell[:, 1]), 1)
    assert np.all(counts == 1)
