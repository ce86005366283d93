"""phs_dense_matvec_noalloc: the dense PHS product for callers that cannot allocate
device memory (real-time loops that must avoid the implicit synchronisation of
cudaMalloc/cudaFree, applications that own all device memory).  Called through the C ABI and compared with phs_dense_matvec, which
allocates its own scratch, on two calls in a row that reuse the library's fixed
staging array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_11462_b300 import build
    build.build()
    from paper_2608_11462_b300 import _native
    return _native


def _call(native, name, pts, k, t, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    fn = getattr(native.lib(), name)
    code = fn(ctypes.c_void_p(pts.data_ptr()), pts.shape[0], k, ctypes.c_void_p(t.data_ptr()),
              ctypes.c_void_p(out.data_ptr()), stream)
    torch.cuda.synchronize()
    return code


@pytest.mark.parametrize("k", [2, 3])
def test_noalloc_matches_allocating_entry_point_twice(native, k):
    rng = np.random.default_rng(100 + k)
    for n in (5000, 1777):  # second call is smaller: stale staging data must not leak in
        pts = torch.tensor(rng.random((n, 2)), dtype=torch.float64, device="cuda")
        t = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(t)
        got = torch.full_like(t, float("nan"))
        assert _call(native, "phs_dense_matvec", pts, k, t, ref) == 0
        assert _call(native, "phs_dense_matvec_noalloc", pts, k, t, got) == 0
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_noalloc_rejects_sizes_beyond_its_capacity(native):
    n = 65537
    pts = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert _call(native, "phs_dense_matvec_noalloc", pts, 2, t, out) == 1
    assert b"65536" in native.lib().phs_last_error()
