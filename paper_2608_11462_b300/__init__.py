"""B300 (sm_103a) polyharmonic-spline interpolation after Geoga & O'Neil,
"Linear-cost Polyharmonic Spline Interpolation of Arbitrary Degree".

Thin PyTorch-facing binding of the C ABI in include/phs.h: tensors supply
device memory and streams, every step runs in the CUDA library.  Function names
mirror the C entry points; ``Plan`` wraps a plan handle.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import PhsError, PhsFitInfo, PhsOptions, PhsServerConfig, check, lib

__all__ = ["Plan", "PhsError", "PhsOptions", "PhsFitInfo", "options", "phs_dense_matvec", "phs_random_order",
           "phs_maxmin_order", "phs_hmaxmin_order", "phs_amaxmin_order", "phs_knn_prev", "phs_vecchia_factor",
           "phs_fit_predict_host", "phs_tune_alpha", "Server", "lib"]


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype=torch.float64, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.contiguous()


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def options(k: int, **kw) -> PhsOptions:
    """Defaults of phs_options_default(k), overridden by keyword."""
    o = PhsOptions()
    lib().phs_options_default(ctypes.byref(o), int(k))
    for key, v in kw.items():
        if not hasattr(o, key):
            raise KeyError(key)
        setattr(o, key, v)
    return o


class Plan:
    """phs_plan_create / phs_matvec / phs_fit / phs_eval on one point set."""

    def __init__(self, points: torch.Tensor, k: int, poly_degree: int = -1, fmm_order: int = 0,
                 vecchia_m: int = 30, opts: PhsOptions | None = None, stream=None):
        pts = _dev(points, name="points")
        if pts.dim() != 2 or pts.shape[1] != 2:
            raise ValueError("points must be n x 2")
        self.n = pts.shape[0]
        self.k = int(k)
        self.device = pts.device
        self._opts = opts if opts is not None else options(k)
        h = ctypes.c_void_p()
        check(lib().phs_plan_create(_ptr(pts), self.n, self.k, int(poly_degree), int(fmm_order), int(vecchia_m),
                                    ctypes.byref(self._opts), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.m = int(vecchia_m)
        fr, sz = self.frame()
        self.S = int(sz[2])

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().phs_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- hot path
    def matvec(self, t: torch.Tensor, precision: int = 0, stream=None) -> torch.Tensor:
        t = _dev(t, name="t")
        out = torch.empty_like(t)
        check(lib().phs_matvec(self._h, _ptr(t), _ptr(out), int(precision), _stream(stream)))
        return out

    def fit(self, f: torch.Tensor, stream=None, allow_not_converged: bool = False):
        f = _dev(f, name="f")
        w = torch.empty_like(f)
        beta = torch.empty(self.S, dtype=torch.float64, device=f.device)
        info = PhsFitInfo()
        check(lib().phs_fit(self._h, _ptr(f), _ptr(w), _ptr(beta), ctypes.byref(info), _stream(stream)),
              allow=(5,) if allow_not_converged else ())
        return w, beta, info.as_dict()

    def gmres(self, b: torch.Tensor, restart: int = 50, check_true: bool = True, stream=None,
              allow_not_converged: bool = False):
        """phs_gmres: M c = b (kernel matrix alone), Vecchia right preconditioner (Sec. 3.1)."""
        b = _dev(b, name="b")
        c = torch.empty_like(b)
        info = PhsFitInfo()
        check(lib().phs_gmres(self._h, _ptr(b), _ptr(c), int(restart), int(bool(check_true)), ctypes.byref(info),
                              _stream(stream)),
              allow=(5,) if allow_not_converged else ())
        return c, info.as_dict()

    def eval(self, w: torch.Tensor, beta: torch.Tensor, targets: torch.Tensor, stream=None) -> torch.Tensor:
        w = _dev(w, name="w")
        beta = _dev(beta, name="beta")
        tg = _dev(targets, name="targets")
        out = torch.empty(tg.shape[0], dtype=torch.float64, device=tg.device)
        check(lib().phs_eval(self._h, _ptr(w), _ptr(beta), _ptr(tg), tg.shape[0], _ptr(out), _stream(stream)))
        return out

    # ---- inspection
    def frame(self):
        fr = (ctypes.c_double * 4)()
        sz = (ctypes.c_int64 * 8)()
        check(lib().phs_plan_frame(self._h, fr, sz))
        return list(fr), list(sz)

    def vecchia(self):
        import numpy as np
        order = np.empty(self.n, dtype=np.int64)
        nbr = np.empty((self.n, self.m), dtype=np.int64)
        check(lib().phs_plan_vecchia(self._h, order.ctypes.data_as(ctypes.c_void_p),
                                     nbr.ctypes.data_as(ctypes.c_void_p)))
        return order, nbr

    def vecchia_factor(self):
        import numpy as np
        diag = np.empty(self.n)
        offd = np.empty((self.n, self.m))
        check(lib().phs_plan_vecchia_factor(self._h, diag.ctypes.data_as(ctypes.c_void_p),
                                            offd.ctypes.data_as(ctypes.c_void_p)))
        return diag, offd

    def precond(self, r: torch.Tensor, stream=None) -> torch.Tensor:
        r = _dev(r, name="r")
        z = torch.empty_like(r)
        check(lib().phs_plan_precond(self._h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def work(self):
        c = (ctypes.c_int64 * 2)()
        check(lib().phs_plan_work(self._h, c))
        return {"near_pairs": c[0], "m2l_translations": c[1]}

    def kernel_work(self):
        c = (ctypes.c_int64 * 6)()
        check(lib().phs_plan_kernel_work(self._h, c))
        return {"p2p_pairs": c[0], "p2p_column_pairs": c[1], "tc_steps": c[2], "tc_tiles": c[3],
                "tc_mmas_per_step": c[4], "tc_mma_macs": c[5]}

    def memory(self) -> int:
        """phs_plan_memory: device bytes held by the plan."""
        b = ctypes.c_int64()
        check(lib().phs_plan_memory(self._h, ctypes.byref(b)))
        return b.value

    def set_wait_limit(self, ns: int, probe: bool = False):
        """phs_plan_set_wait_limit: main-loop wait limit of the tensor-core M2L (0: 2 s) and
        the probe that makes its first wait expire (a test of the timeout path)."""
        check(lib().phs_plan_set_wait_limit(self._h, int(ns), int(bool(probe))))

    def set_timing(self, enabled: bool):
        check(lib().phs_plan_set_timing(self._h, int(bool(enabled))))

    def timing(self):
        ms = (ctypes.c_double * 8)()
        calls = (ctypes.c_int64 * 8)()
        check(lib().phs_plan_timing(self._h, ms, calls))
        names = ["p2p", "m2l", "upward", "downward", "precond", "vector", "eval", "total"]
        return {nm: (ms[i], calls[i]) for i, nm in enumerate(names)}


# ---- stand-alone building blocks
def phs_dense_matvec(points: torch.Tensor, k: int, t: torch.Tensor, stream=None) -> torch.Tensor:
    pts = _dev(points, name="points")
    t = _dev(t, name="t")
    out = torch.empty_like(t)
    check(lib().phs_dense_matvec(_ptr(pts), pts.shape[0], int(k), _ptr(t), _ptr(out), _stream(stream)))
    return out


def phs_random_order(n: int, seed: int, device="cuda", stream=None) -> torch.Tensor:
    out = torch.empty(int(n), dtype=torch.int64, device=device)
    check(lib().phs_random_order(int(n), ctypes.c_uint64(seed), _ptr(out), _stream(stream)))
    return out


def phs_maxmin_order(points: torch.Tensor, stream=None) -> torch.Tensor:
    pts = _dev(points, name="points")
    out = torch.empty(pts.shape[0], dtype=torch.int64, device=pts.device)
    check(lib().phs_maxmin_order(_ptr(pts), pts.shape[0], _ptr(out), _stream(stream)))
    return out


def phs_hmaxmin_order(points: torch.Tensor, seed: int = 1, stream=None) -> torch.Tensor:
    pts = _dev(points, name="points")
    out = torch.empty(pts.shape[0], dtype=torch.int64, device=pts.device)
    check(lib().phs_hmaxmin_order(_ptr(pts), pts.shape[0], ctypes.c_uint64(seed), _ptr(out), _stream(stream)))
    return out


def phs_amaxmin_order(points: torch.Tensor, stream=None) -> torch.Tensor:
    pts = _dev(points, name="points")
    out = torch.empty(pts.shape[0], dtype=torch.int64, device=pts.device)
    check(lib().phs_amaxmin_order(_ptr(pts), pts.shape[0], _ptr(out), _stream(stream)))
    return out


def phs_knn_prev(points: torch.Tensor, order: torch.Tensor, m: int, stream=None) -> torch.Tensor:
    pts = _dev(points, name="points")
    order = _dev(order, torch.int64, name="order")
    out = torch.empty((pts.shape[0], int(m)), dtype=torch.int64, device=pts.device)
    check(lib().phs_knn_prev(_ptr(pts), pts.shape[0], _ptr(order), int(m), _ptr(out), _stream(stream)))
    return out


def phs_vecchia_factor(points, order, nbr, m: int, nu: float, alpha: float, stream=None):
    pts = _dev(points, name="points")
    order = _dev(order, torch.int64, name="order")
    nbr = _dev(nbr, torch.int64, name="nbr")
    n = pts.shape[0]
    diag = torch.empty(n, dtype=torch.float64, device=pts.device)
    offd = torch.empty((n, int(m)), dtype=torch.float64, device=pts.device)
    nj = ctypes.c_int64()
    check(lib().phs_vecchia_factor(_ptr(pts), n, _ptr(order), _ptr(nbr), int(m), float(nu), float(alpha),
                                   _ptr(diag), _ptr(offd), ctypes.byref(nj), _stream(stream)))
    return diag, offd, nj.value


def phs_tune_alpha(points: torch.Tensor, f: torch.Tensor, k: int, poly_degree: int = -1, fmm_order: int = 0,
                   vecchia_m: int = 30, opts: PhsOptions | None = None, n_sample: int = 32768, stream=None):
    """phs_tune_alpha: the preconditioner's alpha by a search on PCG iterations (Sec. 2.2).
    Returns (alpha, iterations on the subsample)."""
    pts = _dev(points, name="points")
    f = _dev(f, name="f")
    o = opts if opts is not None else options(k)
    a = ctypes.c_double()
    it = ctypes.c_int()
    check(lib().phs_tune_alpha(_ptr(pts), _ptr(f), pts.shape[0], int(k), int(poly_degree), int(fmm_order),
                               int(vecchia_m), ctypes.byref(o), int(n_sample), ctypes.byref(a), ctypes.byref(it),
                               _stream(stream)))
    return a.value, it.value


def phs_fit_predict_host(points, f, targets, k: int, poly_degree: int = -1, fmm_order: int = 0,
                         vecchia_m: int = 30, opts: PhsOptions | None = None, stream=None):
    """End-to-end from host (numpy float64) arrays: returns (w, beta, predictions, info)."""
    import numpy as np
    pts = np.ascontiguousarray(points, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    tg = np.ascontiguousarray(targets, dtype=np.float64)
    n, m = pts.shape[0], tg.shape[0]
    w = np.empty(n)
    beta = np.empty(10)
    pred = np.empty(m)
    info = PhsFitInfo()
    o = opts if opts is not None else options(k)
    P = ctypes.c_void_p
    code = lib().phs_fit_predict_host(pts.ctypes.data_as(P), f.ctypes.data_as(P), n, tg.ctypes.data_as(P), m,
                                      int(k), int(poly_degree), int(fmm_order), int(vecchia_m), ctypes.byref(o),
                                      w.ctypes.data_as(P), beta.ctypes.data_as(P), pred.ctypes.data_as(P),
                                      ctypes.byref(info), _stream(stream))
    check(code)
    S = {0: 1, 1: 3, 2: 6, 3: 10}[poly_degree if poly_degree >= 0 else (k // 2 if k % 2 == 0 else (k - 1) // 2)]
    return w, beta[:S], pred, info.as_dict()


class Server:
    """phs_server_*: continuous batching of interpolation requests on the current device.
    Requests are host (numpy) arrays; results come back as numpy arrays."""

    def __init__(self, memory_budget: int = 0, max_active: int = 32, setup_threads: int = 4):
        cfg = PhsServerConfig(int(memory_budget), int(max_active), int(setup_threads))
        h = ctypes.c_void_p()
        check(lib().phs_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._shape = {}

    def submit(self, points, f, targets, k: int, poly_degree: int = -1, fmm_order: int = 0, vecchia_m: int = 30,
               opts: PhsOptions | None = None) -> int:
        import numpy as np
        pts = np.ascontiguousarray(points, dtype=np.float64)
        fv = np.ascontiguousarray(f, dtype=np.float64)
        tg = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 2)
        o = opts if opts is not None else options(k)
        jid = ctypes.c_int64()
        P = ctypes.c_void_p
        check(lib().phs_server_submit(self._h, pts.ctypes.data_as(P), fv.ctypes.data_as(P), pts.shape[0],
                                      tg.ctypes.data_as(P), tg.shape[0], int(k), int(poly_degree), int(fmm_order),
                                      int(vecchia_m), ctypes.byref(o), ctypes.byref(jid)))
        deg = poly_degree if poly_degree >= 0 else (k // 2 if k % 2 == 0 else (k - 1) // 2)
        self._shape[jid.value] = (pts.shape[0], tg.shape[0], (deg + 1) * (deg + 2) // 2)
        return jid.value

    def wait(self, job_id: int, allow_not_converged: bool = False):
        """(w, beta, predictions, info, times = [submitted, admitted, set up, done] in s)."""
        import numpy as np
        n, m, S = self._shape.pop(job_id)
        w, beta, pred, times = np.empty(n), np.empty(S), np.empty(max(m, 1)), np.empty(4)
        info = PhsFitInfo()
        P = ctypes.c_void_p
        check(lib().phs_server_wait(self._h, int(job_id), w.ctypes.data_as(P), beta.ctypes.data_as(P),
                                    pred.ctypes.data_as(P), ctypes.byref(info), times.ctypes.data_as(P)),
              allow=(5,) if allow_not_converged else ())
        return w, beta, pred[:m], info.as_dict(), times

    def stats(self):
        c = (ctypes.c_int64 * 8)()
        check(lib().phs_server_stats(self._h, c))
        keys = ["ticks", "job_iterations", "max_concurrent", "max_reserved", "budget", "completed", "waiting",
                "reserved"]
        return dict(zip(keys, list(c)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(lib().phs_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
