"""ctypes binding of the C ABI in ``include/tilt.h`` (argument marshalling only: every
step of the method runs in the library's CUDA kernels).

Importing this module loads ``libtilt.so`` from the package directory and raises if it
is missing; there is no fallback.  Device tensors are PyTorch CUDA tensors (PyTorch is
used for device memory only)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

AFFINE = 6
PROJECTIVE = 8

TILT_OK = 0
TILT_PENDING = 1
TILT_E_INVAL = -1
TILT_E_NOMEM = -2
TILT_E_BUSY = -3
TILT_E_CUDA = -4
TILT_E_TIMEOUT = -5
TILT_E_NOTFOUND = -6

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtilt.so")


class TiltError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tilt error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t), ("max_live", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("autotune_cache", ctypes.c_char_p)]


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("eps1", ctypes.c_double), ("eps2", ctypes.c_double),
                ("rho0", ctypes.c_double), ("mu0", ctypes.c_double), ("mu_max", ctypes.c_double),
                ("eps_svd", ctypes.c_double), ("max_inner", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("outer_tol", ctypes.c_double), ("svd_ws", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("p", ctypes.c_int), ("tau", ctypes.c_double * 8),
                ("objective", ctypes.c_double), ("lambda_", ctypes.c_double), ("rank_A", ctypes.c_int),
                ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("svd_sweeps", ctypes.c_int),
                ("svd_warm", ctypes.c_int), ("oob_pixels", ctypes.c_int), ("kkt_residual", ctypes.c_double),
                ("latency_ms", ctypes.c_float), ("phase_cycles", ctypes.c_uint64 * 5),
                ("launch_class", ctypes.c_int), ("svd_reorth", ctypes.c_int), ("svd_cayley", ctypes.c_int)]

    @classmethod
    def from_dict(cls, d: dict) -> "Result":
        r = cls()
        r.status, r.p, r.objective = d["status"], d["p"], d["objective"]
        for k, v in enumerate(d["tau"]):
            r.tau[k] = float(v)
        return r

    def to_dict(self) -> dict:
        return dict(status=self.status, p=self.p, tau=np.array(self.tau[: self.p]), objective=self.objective,
                    lam=self.lambda_, rank=self.rank_A, outer_iters=self.outer_iters,
                    inner_iters=self.inner_iters, svd_sweeps=self.svd_sweeps, svd_warm=self.svd_warm,
                    oob=self.oob_pixels, kkt=self.kkt_residual, latency_ms=self.latency_ms,
                    phase_cycles=list(self.phase_cycles), launch_class=self.launch_class,
                    svd_reorth=self.svd_reorth, svd_cayley=self.svd_cayley)


class RaslResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("svd_sweeps", ctypes.c_int), ("svd_warm", ctypes.c_int), ("svd_reorth", ctypes.c_int),
                ("rank", ctypes.c_int), ("oob_pixels", ctypes.c_int), ("svt_qr", ctypes.c_int),
                ("objective", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("kkt_residual", ctypes.c_double), ("cycles", ctypes.c_uint64 * 5)]

    def to_dict(self) -> dict:
        return dict(status=self.status, outer_iters=self.outer_iters, inner_iters=self.inner_iters,
                    svd_sweeps=self.svd_sweeps, svd_warm=self.svd_warm, svd_reorth=self.svd_reorth,
                    rank=self.rank, oob=self.oob_pixels, svt_qr=self.svt_qr, objective=self.objective,
                    lam=self.lambda_,
                    kkt=self.kkt_residual, phase_cycles=list(self.cycles))


class Problem(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("ld_elems", ctypes.c_size_t),
                ("m", ctypes.c_int), ("n", ctypes.c_int), ("type", ctypes.c_int), ("tau0", ctypes.c_double * 8)]


_P = ctypes.POINTER
_d = ctypes.c_double
_i = ctypes.c_int
_vp = ctypes.c_void_p

# Every exported symbol with its argtypes (also used to check the library exports them all).
SIGNATURES = {
    "tilt_default_params": (None, [_P(Params)]),
    "tilt_create": (_i, [_P(Config), _P(_vp)]),
    "tilt_submit": (_i, [_vp, _vp, _i, _i, ctypes.c_size_t, _i, _i, _i, _P(_d), _i, _P(Params),
                         _P(ctypes.c_uint64)]),
    "tilt_submit_batch": (_i, [_vp, _i, _P(Problem), _i, _P(Params), _P(ctypes.c_uint64)]),
    "tilt_poll": (_i, [_vp, ctypes.c_uint64, _P(Result), _vp, _vp]),
    "tilt_wait": (_i, [_vp, ctypes.c_uint64, _i, _P(Result), _vp, _vp]),
    "tilt_destroy": (_i, [_vp]),
    "tilt_last_error": (ctypes.c_char_p, [_vp]),
    "tilt_kernel_launches": (ctypes.c_uint64, [_vp]),
    "tilt_batch_kernel_ms": (_i, [_vp, _P(ctypes.c_float), _i]),
    "tilt_warp_jacobian": (_i, [_vp, _vp, _i, _i, ctypes.c_size_t, _i, _i, _P(_d), _i, _vp, _vp, _P(_d), _P(_i)]),
    "tilt_gram": (_i, [_vp, _vp, _i, _i, _P(_d), _i, _P(_d), _P(_d), _P(_d)]),
    "tilt_svt": (_i, [_vp, _vp, _i, _i, ctypes.c_float, _vp, _P(ctypes.c_float), _P(_i)]),
    "tilt_inner": (_i, [_vp, _vp, _vp, _i, _i, _P(_d), _i, _P(Params), _d, _vp, _vp, _vp, _P(_i), _P(_d),
                        _P(_d), _P(_d), _P(_d)]),
    "tilt_svt_noalloc": (_i, [_vp, _i, _i, ctypes.c_float, _vp, _vp, _vp]),
    "tilt_step_counters": (_i, [_vp, _P(_i), _P(_i)]),
    "tilt_svd_cayley": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp, _P(_d), _P(_d), _P(_d), _P(_i)]),
    "tilt_svt_warm": (_i, [_vp, _vp, _i, _i, ctypes.c_float, _vp, _vp, _P(ctypes.c_float), _P(_i), _P(_i)]),
    "tilt_inner_adm": (_i, [_vp, _vp, _vp, _i, _i, _i, _P(Params), _d, _vp, _vp, _vp, _P(_i), _P(_d), _P(_d),
                            _P(_i)]),
    "tilt_best_of": (_i, [_P(Result), _i, _i, _P(_i)]),
    "tilt_autotune": (_i, [_vp, _P(_i), _i, _i, _P(_i)]),
    "tilt_rasl": (_i, [_vp, _i, _i, _vp, _i, _i, _i, _i, _i, _i, _P(_d), _P(Params), _P(_d), _vp, _vp, _vp,
                       _P(RaslResult), _P(ctypes.c_float)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_params(**kw) -> Params:
    p = Params()
    lib().tilt_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k in ("lam", "lambda") else k, v)
    return p


def _check(rc: int, ctx=None):
    if rc < 0:
        raise TiltError(rc, lib().tilt_last_error(ctx).decode())
    return rc


def _dptr(t) -> int:
    """Device address of a PyTorch CUDA tensor (contiguous)."""
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def best_of(results: list, starts: int) -> list:
    """Multi-start selection (tilt_best_of): per group of `starts` consecutive results, the
    index of the lowest objective among successful ones (-1 if none)."""
    n = len(results) // starts
    arr = (Result * (n * starts))(*[Result.from_dict(r) for r in results[: n * starts]])
    out = (ctypes.c_int * max(1, n))()
    _check(lib().tilt_best_of(arr, n, starts, out))
    return [out[i] for i in range(n)]


# ------------------------------------------------------------------ layout marshalling
def dims(m: int, n: int):
    return (m, n) if m >= n else (n, m)


def to_long_layout(X: np.ndarray) -> np.ndarray:
    """m x n row-major array -> flat long-side-contiguous storage (see tilt.h)."""
    m, n = X.shape
    return np.ascontiguousarray(X.T if m >= n else X).reshape(-1)


def from_long_layout(flat: np.ndarray, m: int, n: int) -> np.ndarray:
    flat = np.asarray(flat).reshape(-1)
    return flat.reshape(n, m).T.copy() if m >= n else flat.reshape(m, n).copy()


def jacobian_to_rows(Jflat: np.ndarray, m: int, n: int, p: int) -> np.ndarray:
    """p long-layout planes -> (m*n, p) with rows in row-major pixel order (oracle layout)."""
    Jflat = np.asarray(Jflat).reshape(p, m * n)
    return np.stack([from_long_layout(Jflat[k], m, n).reshape(-1) for k in range(p)], axis=1)


def jacobian_from_rows(J: np.ndarray, m: int, n: int) -> np.ndarray:
    p = J.shape[1]
    return np.concatenate([to_long_layout(J[:, k].reshape(m, n)) for k in range(p)])


# ------------------------------------------------------------------ context
class Context:
    """One solver context on one device (``tilt_create`` / ``tilt_destroy``)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_live: int = 0, autotune_cache: str = None,
                 cuda_stream: int = 0):
        """``cuda_stream``: a cudaStream_t handle (e.g. ``torch.cuda.Stream().cuda_stream``) that
        carries the context's grouped launches, copies and steps; 0: the context's own streams."""
        self._cache = autotune_cache.encode() if autotune_cache else None
        cfg = Config(device, hbm_budget_bytes, max_live, cuda_stream or None, self._cache)
        h = _vp()
        _check(lib().tilt_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            _check(lib().tilt_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(lib().tilt_kernel_launches(self.h))

    def autotune(self, shapes, ttype: int = AFFINE) -> list:
        """Tune the Jacobi schedule for the size buckets of the given (m, n) shapes; returns each
        shape's schedule (group width, plus 256 for block-cyclic pair ordering)."""
        shapes = list(shapes)
        arr = (ctypes.c_int * (2 * max(1, len(shapes))))(*[v for mn in shapes for v in mn])
        out = (ctypes.c_int * max(1, len(shapes)))()
        _check(lib().tilt_autotune(self.h, arr, len(shapes), ttype, out), self.h)
        return [out[i] for i in range(len(shapes))]

    def batch_kernel_ms(self) -> list:
        """Device time (ms) of each grouped launch of the last submit_batch (CUDA events)."""
        buf = (ctypes.c_float * 3)()
        n = _check(lib().tilt_batch_kernel_ms(self.h, buf, 3), self.h)
        return [float(buf[i]) for i in range(n)]

    # ---------------------------------------------------------------- serving API
    def submit(self, img, m: int, n: int, tau0, ttype: int, params: Params | None = None) -> int:
        """Queue one problem; ``img`` is a float32 numpy array (host) or CUDA tensor (device)."""
        tau = (ctypes.c_double * 8)(*list(np.asarray(tau0, dtype=np.float64))[:8])
        t = ctypes.c_uint64()
        if isinstance(img, np.ndarray):
            a = np.ascontiguousarray(img, dtype=np.float32)
            H, W = a.shape
            rc = lib().tilt_submit(self.h, a.ctypes.data, H, W, W, 0, m, n, tau, ttype,
                                   ctypes.byref(params) if params else None, ctypes.byref(t))
        else:
            H, W = img.shape
            rc = lib().tilt_submit(self.h, _dptr(img), H, W, img.stride(0), 1, m, n, tau, ttype,
                                   ctypes.byref(params) if params else None, ctypes.byref(t))
        _check(rc, self.h)
        return t.value

    def submit_batch(self, items, params: Params | None = None, on_device: bool = False):
        """Queue a list of (img, m, n, tau0, ttype) as grouped launches; returns tickets."""
        N = len(items)
        arr = (Problem * N)()
        keep = []
        for q, (img, m, n, tau0, ttype) in enumerate(items):
            if on_device:
                ptr, (H, W), ld = _dptr(img), img.shape, img.stride(0)
            elif hasattr(img, "data_ptr"):            # a host (e.g. pinned) PyTorch tensor
                assert not img.is_cuda and img.is_contiguous() and str(img.dtype) == "torch.float32"
                ptr, (H, W), ld = img.data_ptr(), tuple(img.shape), img.stride(0)
            else:
                a = np.ascontiguousarray(img, dtype=np.float32)
                keep.append(a)
                ptr, (H, W), ld = a.ctypes.data, a.shape, a.shape[1]
            arr[q].img = ptr
            arr[q].H, arr[q].W, arr[q].ld_elems = H, W, ld
            arr[q].m, arr[q].n, arr[q].type = m, n, ttype
            for k, v in enumerate(np.asarray(tau0, dtype=np.float64)[:8]):
                arr[q].tau0[k] = float(v)
        tickets = (ctypes.c_uint64 * N)()
        _check(lib().tilt_submit_batch(self.h, N, arr, 1 if on_device else 0,
                                       ctypes.byref(params) if params else None, tickets), self.h)
        return list(tickets)

    def poll(self, ticket: int, with_planes: bool = False, m: int = 0, n: int = 0):
        """None while pending; else the result dict (with 'A', 'E' as m x n arrays when asked)."""
        r = Result()
        A = E = None
        pa = pe = None
        if with_planes:
            A = np.empty((m, n), np.float32)
            E = np.empty((m, n), np.float32)
            pa, pe = A.ctypes.data, E.ctypes.data
        rc = _check(lib().tilt_poll(self.h, ticket, ctypes.byref(r), pa, pe), self.h)
        if rc == TILT_PENDING:
            return None
        d = r.to_dict()
        if with_planes:
            d["A"], d["E"] = A, E
        return d

    def wait(self, ticket: int, timeout_ms: int = 600000, with_planes: bool = False, m: int = 0, n: int = 0):
        r = Result()
        A = E = None
        pa = pe = None
        if with_planes:
            A = np.empty((m, n), np.float32)
            E = np.empty((m, n), np.float32)
            pa, pe = A.ctypes.data, E.ctypes.data
        _check(lib().tilt_wait(self.h, ticket, timeout_ms, ctypes.byref(r), pa, pe), self.h)
        d = r.to_dict()
        if with_planes:
            d["A"], d["E"] = A, E
        return d

    # ---------------------------------------------------------------- step entry points
    def warp_jacobian(self, img_t, m: int, n: int, tau, ttype: int):
        """Returns (Dhat, J) as flat CUDA tensors in long layout, ||D o tau||_F, oob count."""
        import torch
        Dhat = torch.empty(m * n, dtype=torch.float32, device=img_t.device)
        J = torch.empty(ttype * m * n, dtype=torch.float32, device=img_t.device)
        tau_c = (ctypes.c_double * 8)(*list(np.asarray(tau, dtype=np.float64))[:8])
        norm = ctypes.c_double()
        oob = ctypes.c_int()
        H, W = img_t.shape
        _check(lib().tilt_warp_jacobian(self.h, _dptr(img_t), H, W, img_t.stride(0), m, n, tau_c, ttype,
                                        _dptr(Dhat), _dptr(J), ctypes.byref(norm), ctypes.byref(oob)), self.h)
        return Dhat, J, norm.value, oob.value

    def gram(self, J_t, m: int, n: int, tau, ttype: int):
        p = ttype
        tau_c = (ctypes.c_double * 8)(*list(np.asarray(tau, dtype=np.float64))[:8])
        Q = (ctypes.c_double * (3 * p))()
        G = (ctypes.c_double * (p * p))()
        Gi = (ctypes.c_double * (p * p))()
        _check(lib().tilt_gram(self.h, _dptr(J_t), m, n, tau_c, ttype, Q, G, Gi), self.h)
        return (np.array(Q).reshape(3, p), np.array(G).reshape(p, p), np.array(Gi).reshape(p, p))

    def svt(self, M_t, m: int, n: int, eps: float):
        import torch
        A = torch.empty(m * n, dtype=torch.float32, device=M_t.device)
        C = min(m, n)
        sig = (ctypes.c_float * C)()
        sw = ctypes.c_int()
        _check(lib().tilt_svt(self.h, _dptr(M_t), m, n, float(eps), _dptr(A), sig, ctypes.byref(sw)), self.h)
        return A, np.array(sig, dtype=np.float32), sw.value

    def svd_cayley(self, M_t, m: int, n: int, U_t, S_t, V_t) -> dict:
        """tilt_svd_cayley: one Algorithm-2 step; U_t, S_t, V_t (CUDA, column-major) are updated in
        place when the step is accepted."""
        f1, f2, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        acc = ctypes.c_int()
        _check(lib().tilt_svd_cayley(self.h, _dptr(M_t), m, n, _dptr(U_t), _dptr(S_t), _dptr(V_t), ctypes.byref(f1),
                                     ctypes.byref(f2), ctypes.byref(t), ctypes.byref(acc)), self.h)
        return dict(f1=f1.value, f2=f2.value, t=t.value, accepted=bool(acc.value))

    def svt_warm(self, M_t, m: int, n: int, eps: float, V_t):
        """tilt_svt_warm: V_t (CUDA, C x C column-major, C = min(m, n)) is the warm start and
        receives the new right singular vectors; returns (A, sigma, sweeps, reorth)."""
        import torch
        A = torch.empty(m * n, dtype=torch.float32, device=M_t.device)
        C = min(m, n)
        sig = (ctypes.c_float * C)()
        sw, ro = ctypes.c_int(), ctypes.c_int()
        _check(lib().tilt_svt_warm(self.h, _dptr(M_t), m, n, float(eps), _dptr(V_t), _dptr(A), sig, ctypes.byref(sw),
                                   ctypes.byref(ro)), self.h)
        return A, np.array(sig, dtype=np.float32), sw.value, ro.value

    def inner_adm(self, D_t, J_t, m: int, n: int, p: int, params: Params | None, mu0: float = -1.0) -> dict:
        """The ADM baseline (tilt_inner_adm); returns A, E, Y (flat CUDA tensors, long layout),
        iterations, dtau, the last relative residual and the Jacobi sweeps."""
        import torch
        A = torch.empty_like(D_t)
        E = torch.empty_like(D_t)
        Y = torch.empty_like(D_t)
        it, sw = ctypes.c_int(), ctypes.c_int()
        dt = (ctypes.c_double * 8)()
        res = ctypes.c_double()
        _check(lib().tilt_inner_adm(self.h, _dptr(D_t), _dptr(J_t) if p else None, m, n, p,
                                    ctypes.byref(params) if params else None, float(mu0), _dptr(A), _dptr(E),
                                    _dptr(Y), ctypes.byref(it), dt, ctypes.byref(res), ctypes.byref(sw)), self.h)
        return dict(A=A, E=E, Y=Y, iters=it.value, dtau=np.array(dt[:p]), residual=res.value, sweeps=sw.value)

    def rasl(self, imgs, m: int, n: int, tau0, ttype: int, params: Params | None = None,
             planes: bool = False) -> dict:
        """tilt_rasl on a batch of image sets.  ``imgs``: (count, nimg, H, W) float32, a numpy
        array or a contiguous host (e.g. pinned) or CUDA tensor; ``tau0``: (count, nimg, p).
        Returns tau (count, nimg, p), the result records, the launch's kernel time and, when
        ``planes``, A, E and D_hat as (count, m n, nimg) arrays (column c = image c)."""
        if hasattr(imgs, "data_ptr"):
            assert imgs.is_contiguous() and str(imgs.dtype) == "torch.float32"
            count, nimg, H, W = (int(v) for v in imgs.shape)
            ptr, on_dev = imgs.data_ptr(), 1 if imgs.is_cuda else 0
            keep = imgs
        else:
            keep = np.ascontiguousarray(imgs, dtype=np.float32)
            count, nimg, H, W = keep.shape
            ptr, on_dev = keep.ctypes.data, 0
        p = int(ttype)
        t0 = np.ascontiguousarray(np.asarray(tau0, dtype=np.float64).reshape(count, nimg, p))
        tau = np.empty_like(t0)
        res = (RaslResult * max(count, 1))()
        S = m * n * nimg
        A = np.empty((count, S), np.float32) if planes else None
        E = np.empty((count, S), np.float32) if planes else None
        D = np.empty((count, S), np.float32) if planes else None
        ms = ctypes.c_float()
        dp = lambda a: a.ctypes.data if a is not None else None
        _check(lib().tilt_rasl(self.h, count, nimg, ptr, on_dev, H, W, m, n, ttype,
                               t0.ctypes.data_as(_P(_d)), ctypes.byref(params) if params else None,
                               tau.ctypes.data_as(_P(_d)), dp(A), dp(E), dp(D), res, ctypes.byref(ms)), self.h)
        del keep
        out = dict(tau=tau, results=[res[i].to_dict() for i in range(count)], kernel_ms=ms.value)
        if planes:
            shape = (count, nimg, m * n)
            out.update(A=A.reshape(shape).transpose(0, 2, 1), E=E.reshape(shape).transpose(0, 2, 1),
                       Dhat=D.reshape(shape).transpose(0, 2, 1))
        return out

    def inner(self, Dhat_t, J_t, m: int, n: int, tau, ttype: int, params: Params | None, mu0: float,
              A_t, E_t, Y_t) -> dict:
        """tilt_inner; tau = None runs without constraint rows (W^T W = J_perp)."""
        tau_c = (ctypes.c_double * 8)(*list(np.asarray(tau, dtype=np.float64))[:8]) if tau is not None else None
        it = ctypes.c_int()
        dt = (ctypes.c_double * 8)()
        c1, c2, mu = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().tilt_inner(self.h, _dptr(Dhat_t), _dptr(J_t), m, n, tau_c, ttype,
                                ctypes.byref(params) if params else None, float(mu0), _dptr(A_t), _dptr(E_t),
                                _dptr(Y_t), ctypes.byref(it), dt, ctypes.byref(c1), ctypes.byref(c2),
                                ctypes.byref(mu)), self.h)
        sw, cay = ctypes.c_int(), ctypes.c_int()
        _check(lib().tilt_step_counters(self.h, ctypes.byref(sw), ctypes.byref(cay)), self.h)
        return dict(iters=it.value, dtau=np.array(dt[:ttype]), c1=c1.value, c2=c2.value, mu=mu.value,
                    sweeps=sw.value, cayley_steps=cay.value)
