"""Thin ctypes binding of the C-ABI in include/nudft2_hss.h.

Argument marshalling only: every step of the solver runs in the CUDA library.  Tensors are
torch CUDA tensors; complex right-hand sides are complex128 and are passed column major
(a (M, s) tensor is handed over as its (s, M) contiguous transpose with leading dimension M).
If the shared library is missing this module raises at first use; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnudft2_hss.so")

OK, EINVAL, ENOMEM, ECUDA, ERANK, ETIMEOUT, ESTATE, ENOTIMPL = range(8)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ERANK", 5: "ETIMEOUT", 6: "ESTATE", 7: "ENOTIMPL"}
FP64, MIXED = 0, 1
FAST_FWD, FAST_ADJ, EXACT_FWD, EXACT_ADJ, PINV, PINV_ADJ = range(6)


class Opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("levels", ctypes.c_int), ("leaf", ctypes.c_int), ("prec", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("refine_max", ctypes.c_int), ("flags", ctypes.c_uint),
                ("levels_y", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("levels", ctypes.c_int),
                ("prec", ctypes.c_int), ("max_rank", ctypes.c_int), ("level_rank", ctypes.c_int * 16),
                ("t_build_ms", ctypes.c_double), ("t_factor_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("refine_iters", ctypes.c_int), ("refine_relres", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("launches", ctypes.c_int), ("gemm_tuned", ctypes.c_int),
                ("solve_graphs", ctypes.c_int), ("solve_graph_failures", ctypes.c_int), ("solve_replays", ctypes.c_int),
                ("checkpointed_levels", ctypes.c_int)]


class KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("launches", ctypes.c_int)]


FLAG_PROFILE = 1
FLAG_FP64_RESIDUALS = 2
FLAG_FADI = 4


class NudftError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libnudft2_hss.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_2607_00928_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.nudft2_hss_build.argtypes = [vp, vp, i64, ci, ci, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    L.nudft2_hss_factor.argtypes = [vp, vp]
    L.nudft2_hss_solve.argtypes = [vp, vp, i64, ci, vp, i64, vp]
    L.nudft2_hss_apply.argtypes = [vp, ci, vp, i64, ci, vp, i64, vp]
    L.nudft2_hss_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.nudft2_hss_grad.argtypes = [vp, vp, i64, vp, i64, vp, i64, ci, vp, i64, vp, vp, vp]
    L.nudft2_hss_plsqr.argtypes = [vp, vp, i64, ci, vp, i64, ctypes.c_double, ci, ctypes.POINTER(ci),
                                   ctypes.POINTER(ctypes.c_double), vp]
    pp = ctypes.POINTER(vp)
    L.nudft2_hss_build_batched.argtypes = [ci, pp, pp, ctypes.POINTER(i64), ctypes.POINTER(ci), ctypes.POINTER(ci),
                                           ctypes.POINTER(Opts), ci, ci, vp, pp, ctypes.POINTER(ci)]
    L.nudft2_hss_solve_batched.argtypes = [ci, pp, pp, ctypes.POINTER(i64), ctypes.POINTER(ci), pp,
                                           ctypes.POINTER(i64), ci, vp, ctypes.POINTER(ci)]
    L.nudft2_hss_run_batched.argtypes = [ci, pp, pp, ctypes.POINTER(i64), ctypes.POINTER(ci), ctypes.POINTER(ci),
                                         ctypes.POINTER(Opts), pp, ctypes.POINTER(i64), ctypes.POINTER(ci), pp,
                                         ctypes.POINTER(i64), ci, vp, ctypes.POINTER(ci)]
    L.nudft2_hss_free.argtypes = [vp]
    L.nudft2_hss_free.restype = None
    L.nudft2_psi_eval.argtypes = [vp, i64, ci, vp, vp]
    L.nudft2_hss_kstats.argtypes = [vp, ctypes.POINTER(KStat), ci, ctypes.POINTER(ci)]
    L.nudft2_la_tsvd.argtypes = [ci, vp, i64, i64, i64, ctypes.c_double, vp, i64, ctypes.POINTER(ci),
                                 ctypes.POINTER(ctypes.c_double), vp]
    L.nudft2_la_qr.argtypes = [ci, vp, i64, i64, i64, vp, i64, ci, vp]
    L.nudft2_la_qr_apply.argtypes = [ci, vp, i64, i64, i64, vp, i64, i64, ci, ci, vp]
    L.nudft2_hss_save.argtypes = [vp, ctypes.c_char_p]
    L.nudft2_hss_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
    L.nudft2_test_fail_alloc.argtypes = [ctypes.c_longlong]
    L.nudft2_test_fail_alloc.restype = None
    L.nudft2_la_gemm.argtypes = [ci, ci, ci, i64, i64, i64, ctypes.c_double, vp, i64, i64, vp, i64, i64,
                                 ctypes.c_double, vp, i64, i64, ci, vp]
    L.nudft2_exact_apply.argtypes = [vp, vp, i64, ci, ci, ci, vp, i64, ci, vp, i64, vp]
    L.nudft2_exact_fwd_noalloc.argtypes = [vp, vp, i64, ci, ci, vp, i64, ci, vp, i64, vp]
    L.nudft2_peak_fma.argtypes = [ci, ctypes.POINTER(ctypes.c_double), vp]
    L.nudft2_hss_checkpoint.argtypes = [vp, ci, vp]
    pint, pdbl = ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_double)
    L.nudft2_fadi_plan.argtypes = [ci, ci, ci, ctypes.c_double, pint, pint, pint, pdbl, pdbl, pdbl, pdbl]
    L.nudft2_last_error.restype = ctypes.c_char_p
    for f in ("nudft2_hss_build", "nudft2_hss_factor", "nudft2_hss_solve", "nudft2_hss_apply", "nudft2_hss_info",
              "nudft2_hss_grad", "nudft2_hss_build_batched", "nudft2_hss_solve_batched", "nudft2_hss_run_batched", "nudft2_hss_plsqr",
              "nudft2_psi_eval", "nudft2_hss_kstats", "nudft2_la_tsvd", "nudft2_la_qr", "nudft2_la_qr_apply", "nudft2_test_fail_alloc", "nudft2_hss_save", "nudft2_hss_load", "nudft2_la_gemm", "nudft2_exact_apply",
              "nudft2_exact_fwd_noalloc", "nudft2_peak_fma", "nudft2_hss_checkpoint", "nudft2_fadi_plan"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _check(code: int):
    if code != OK:
        raise NudftError(code, lib().nudft2_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor(a: torch.Tensor, rows: int) -> torch.Tensor:
    """(rows,) or (rows, s) complex128 CUDA tensor -> contiguous (s, rows) (= column major)."""
    if a.dim() == 1:
        a = a[:, None]
    assert a.shape[0] == rows, (a.shape, rows)
    return a.to(device="cuda", dtype=torch.complex128).t().contiguous()


def peak_fma(prec: int) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (FP32 FFMA for MIXED, DFMA for FP64)."""
    v = ctypes.c_double()
    _check(lib().nudft2_peak_fma(prec, ctypes.byref(v), _stream()))
    return v.value


def fadi_plan(side: int, d: int, n: int, eps1: float) -> dict:
    """The host-side fADI plan of a node of d columns out of n (nudft2_fadi_plan; no device work)."""
    ne, J, ratio = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    ex = (ctypes.c_int * 65)()
    xa, xb = (ctypes.c_double * 64)(), (ctypes.c_double * 64)()
    C = (ctypes.c_double * (2 * 65 * 65))()
    code = lib().nudft2_fadi_plan(side, d, n, eps1, ctypes.byref(ne), ctypes.byref(J), ex, xa, xb, C,
                                  ctypes.byref(ratio))
    if code != OK:
        raise NudftError(code, "fadi_plan: bad node or eps1 too small for n")
    q = ne.value + J.value
    Cc = [complex(C[2 * e], C[2 * e + 1]) for e in range(q * q)]
    return dict(ex=list(ex[:ne.value]), J=J.value, xa=list(xa[:J.value]), xb=list(xb[:J.value]),
                C=[Cc[j * q:(j + 1) * q] for j in range(q)], ratio=ratio.value)   # C as columns


def psi_eval(x: torch.Tensor, n: int) -> torch.Tensor:
    """Entries Psi(gamma_j, xi_k) of the transformed 1D matrix (M x n complex128)."""
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    out = torch.empty((n, x.numel()), dtype=torch.complex128, device="cuda")
    _check(lib().nudft2_psi_eval(ctypes.c_void_p(x.data_ptr()), x.numel(), n, ctypes.c_void_p(out.data_ptr()),
                                 _stream()))
    return out.t()


def exact_apply(x, y, nx: int, ny: int, op: int, v: torch.Tensor) -> torch.Tensor:
    """Direct FP64 apply of A (op=EXACT_FWD, v: (N,s)) or A^* (op=EXACT_ADJ, v: (M,s)) without an HSS."""
    x = torch.as_tensor(x).to(device="cuda", dtype=torch.float64).contiguous()
    y = torch.as_tensor(y).to(device="cuda", dtype=torch.float64).contiguous()
    M, N = x.numel(), nx * ny
    rows_in, rows_out = (N, M) if op == EXACT_FWD else (M, N)
    squeeze = v.dim() == 1
    vc = _colmajor(v, rows_in)
    s = vc.shape[0]
    out = torch.empty((s, rows_out), dtype=torch.complex128, device="cuda")
    _check(lib().nudft2_exact_apply(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), M, nx, ny, op,
                                    ctypes.c_void_p(vc.data_ptr()), rows_in, s, ctypes.c_void_p(out.data_ptr()),
                                    rows_out, _stream()))
    return out[0] if squeeze else out.t()


def la_tsvd(C: torch.Tensor, eps: float):
    """Truncated SVD of C (r x w) by the library's QR + one-sided Jacobi: (P, sigma)."""
    r, w = C.shape
    dt = C.dtype
    prec = FP64 if dt == torch.complex128 else MIXED
    ct = torch.conj_physical(C).contiguous()        # row-major (r, w) of conj(C) == column-major C^* (w x r)
    p = min(r, w)
    P = torch.zeros((max(p, 1), r), dtype=dt, device="cuda")
    rank = ctypes.c_int()
    sig = (ctypes.c_double * max(p, 1))()
    _check(lib().nudft2_la_tsvd(prec, ctypes.c_void_p(ct.data_ptr()), w, r, max(w, 1), eps,
                                ctypes.c_void_p(P.data_ptr()), r, ctypes.byref(rank), sig, _stream()))
    return P[: rank.value].t(), [sig[i] for i in range(p)]


def la_qr(A: torch.Tensor, grouped: bool = False):
    """Householder QR of A (m x n) by the library: (Q m x m, R m x n)."""
    m, n = A.shape
    dt = A.dtype
    prec = FP64 if dt == torch.complex128 else MIXED
    a = A.t().contiguous()                          # column major
    q = torch.empty((m, m), dtype=dt, device="cuda")
    _check(lib().nudft2_la_qr(prec, ctypes.c_void_p(a.data_ptr()), m, n, m, ctypes.c_void_p(q.data_ptr()), m,
                              int(grouped), _stream()))
    return q.t(), torch.triu(a.t())


def la_qr_apply(A: torch.Tensor, C: torch.Tensor, conj: bool, grouped: bool = False):
    """Householder QR of A (m x n) by the library, then Q^* C (conj) or Q C for C (m x s) by the
    streaming reflector kernels of the solve sweeps: (result m x s, R m x n)."""
    m, n = A.shape
    s = C.shape[1]
    dt = A.dtype
    prec = FP64 if dt == torch.complex128 else MIXED
    a = A.t().contiguous()                          # column major
    c = C.to(dt).t().contiguous()
    _check(lib().nudft2_la_qr_apply(prec, ctypes.c_void_p(a.data_ptr()), m, n, m, ctypes.c_void_p(c.data_ptr()), s,
                                    m, int(conj), int(grouped), _stream()))
    return c.t(), torch.triu(a.t())


_OPS = {"N": 0, "T": 1, "C": 2}


def la_gemm(A: torch.Tensor, B: torch.Tensor, opa: str = "N", opb: str = "N", alpha: float = 1.0,
            beta: float = 0.0, C: torch.Tensor = None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C by the library's batched GEMM; A, B, C are (batch, rows, cols)
    or (rows, cols) complex CUDA tensors (returned C is a new tensor unless C is given)."""
    squeeze = A.dim() == 2
    A3, B3 = (A[None], B[None]) if squeeze else (A, B)
    dt = A3.dtype
    prec = FP64 if dt == torch.complex128 else MIXED
    nb = A3.shape[0]
    m = A3.shape[1] if opa == "N" else A3.shape[2]
    k = A3.shape[2] if opa == "N" else A3.shape[1]
    n = B3.shape[2] if opb == "N" else B3.shape[1]
    a = A3.transpose(1, 2).contiguous()             # column major per batch item
    b = B3.transpose(1, 2).contiguous()
    if C is None:
        c = torch.zeros((nb, n, m), dtype=dt, device=A.device)
    else:
        c = (C[None] if squeeze else C).transpose(1, 2).contiguous()
    _check(lib().nudft2_la_gemm(prec, _OPS[opa], _OPS[opb], m, n, k, float(alpha),
                                ctypes.c_void_p(a.data_ptr()), max(a.shape[2], 1), a.shape[1] * a.shape[2],
                                ctypes.c_void_p(b.data_ptr()), max(b.shape[2], 1), b.shape[1] * b.shape[2], float(beta),
                                ctypes.c_void_p(c.data_ptr()), m, m * n, nb, _stream()))
    out = c.transpose(1, 2)
    return out[0] if squeeze else out


class NudftHSS:
    """Handle of one point set: build (Alg. 1 steps 1-3), factor (step 4), solve (step 5)."""

    def __init__(self, x, y, nx: int, ny: int, eps: float = 1e-10, levels: int = 0, leaf: int = 64,
                 prec: str = "fp64", refine_tol: float = 1e-8, refine_max: int = 8, stream=None,
                 profile: bool = False, fp64_residuals: bool = False, levels_y: int = 0, fadi: bool = False):
        self._h = ctypes.c_void_p()
        self.x = torch.as_tensor(x).to(device="cuda", dtype=torch.float64).contiguous()
        self.y = torch.as_tensor(y).to(device="cuda", dtype=torch.float64).contiguous()
        self.M = self.x.numel()
        self.nx, self.ny, self.N = nx, ny, nx * ny
        self.stream = stream
        o = Opts(eps, levels, leaf, MIXED if prec == "mixed" else FP64, refine_tol, refine_max,
                 (FLAG_PROFILE if profile else 0) | (FLAG_FP64_RESIDUALS if fp64_residuals else 0)
                 | (FLAG_FADI if fadi else 0), levels_y)
        _check(lib().nudft2_hss_build(ctypes.c_void_p(self.x.data_ptr()), ctypes.c_void_p(self.y.data_ptr()),
                                      self.M, nx, ny, ctypes.byref(o), _stream(stream), ctypes.byref(self._h)))

    def factor(self):
        _check(lib().nudft2_hss_factor(self._h, _stream(self.stream)))
        return self

    def save(self, path: str):
        """Write the factored handle (points, generators, URV factors) to `path` (nudft2_hss_save)."""
        _check(lib().nudft2_hss_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, path: str, stream=None) -> "NudftHSS":
        """A factored handle read back from a file written by save() (nudft2_hss_load)."""
        h = cls.__new__(cls)
        h._h = ctypes.c_void_p()
        h.stream = stream
        _check(lib().nudft2_hss_load(str(path).encode(), _stream(stream), ctypes.byref(h._h)))
        i = Info()
        _check(lib().nudft2_hss_info(h._h, ctypes.byref(i)))
        h.M, h.nx, h.ny = int(i.M), int(i.nx), int(i.ny)
        h.N = h.nx * h.ny
        h.x = h.y = None
        return h

    def solve(self, f: torch.Tensor) -> torch.Tensor:
        """c (N, s) = F^{-1} G~_hss^+ f for f (M,) or (M, s); lexicographic ky + kx*ny order."""
        squeeze = f.dim() == 1
        fc = _colmajor(f, self.M)
        s = fc.shape[0]
        c = torch.empty((s, self.N), dtype=torch.complex128, device="cuda")
        _check(lib().nudft2_hss_solve(self._h, ctypes.c_void_p(fc.data_ptr()), self.M, s,
                                      ctypes.c_void_p(c.data_ptr()), self.N, _stream(self.stream)))
        return c[0] if squeeze else c.t()

    def apply(self, op: int, v: torch.Tensor) -> torch.Tensor:
        to_points = op in (FAST_FWD, EXACT_FWD, PINV_ADJ)
        rows_in = self.N if to_points else self.M
        rows_out = self.M if to_points else self.N
        squeeze = v.dim() == 1
        vc = _colmajor(v, rows_in)
        s = vc.shape[0]
        out = torch.empty((s, rows_out), dtype=torch.complex128, device="cuda")
        _check(lib().nudft2_hss_apply(self._h, op, ctypes.c_void_p(vc.data_ptr()), rows_in, s,
                                      ctypes.c_void_p(out.data_ptr()), rows_out, _stream(self.stream)))
        return out[0] if squeeze else out.t()

    def grad(self, f: torch.Tensor, c: torch.Tensor, g: torch.Tensor, points: bool = True):
        """Backward of c = A^+ f for a real loss with gradient g = dL/dRe c + i dL/dIm c (N, s):
        returns (grad_f (M, s), grad_x (M,), grad_y (M,)); grad_x/grad_y are None unless points."""
        squeeze = f.dim() == 1
        fc, cc, gc = _colmajor(f, self.M), _colmajor(c, self.N), _colmajor(g, self.N)
        s = fc.shape[0]
        gf = torch.empty((s, self.M), dtype=torch.complex128, device="cuda")
        gx = torch.empty(self.M, dtype=torch.float64, device="cuda") if points else None
        gy = torch.empty(self.M, dtype=torch.float64, device="cuda") if points else None
        _check(lib().nudft2_hss_grad(self._h, ctypes.c_void_p(fc.data_ptr()), self.M, ctypes.c_void_p(cc.data_ptr()),
                                     self.N, ctypes.c_void_p(gc.data_ptr()), self.N, s, ctypes.c_void_p(gf.data_ptr()),
                                     self.M, ctypes.c_void_p(gx.data_ptr() if points else None),
                                     ctypes.c_void_p(gy.data_ptr() if points else None), _stream(self.stream)))
        return (gf[0] if squeeze else gf.t()), gx, gy

    def plsqr(self, f: torch.Tensor, tol: float = 1e-12, maxit: int = 500):
        """LSQR preconditioned by this factorization (exact FP64 applies of A, A^*): returns
        (c, iterations, relative residual ||f - A c|| / ||f||)."""
        squeeze = f.dim() == 1
        fc = _colmajor(f, self.M)
        s = fc.shape[0]
        c = torch.empty((s, self.N), dtype=torch.complex128, device="cuda")
        it = ctypes.c_int()
        rr = ctypes.c_double()
        _check(lib().nudft2_hss_plsqr(self._h, ctypes.c_void_p(fc.data_ptr()), self.M, s, ctypes.c_void_p(c.data_ptr()),
                                      self.N, float(tol), int(maxit), ctypes.byref(it), ctypes.byref(rr),
                                      _stream(self.stream)))
        return (c[0] if squeeze else c.t()), it.value, rr.value

    def checkpoint(self, levels: int):
        """Hand back the factors of the top `levels` levels (and the root); they are recomputed
        by the next call that needs them."""
        _check(lib().nudft2_hss_checkpoint(self._h, int(levels), _stream(self.stream)))
        return self

    def info(self) -> dict:
        i = Info()
        _check(lib().nudft2_hss_info(self._h, ctypes.byref(i)))
        return {"M": i.M, "nx": i.nx, "ny": i.ny, "levels": i.levels, "prec": i.prec, "max_rank": i.max_rank,
                "level_rank": list(i.level_rank)[: i.levels + 1], "t_build_ms": i.t_build_ms,
                "t_factor_ms": i.t_factor_ms, "t_solve_ms": i.t_solve_ms, "refine_iters": i.refine_iters,
                "refine_relres": i.refine_relres, "device_bytes": i.device_bytes, "launches": i.launches,
                "gemm_tuned": i.gemm_tuned, "solve_graphs": i.solve_graphs,
                "solve_graph_failures": i.solve_graph_failures, "solve_replays": i.solve_replays,
                "checkpointed_levels": i.checkpointed_levels}

    def kstats(self) -> dict:
        """Per kernel class: device ms, algorithmic flops and bytes, launches (profile=True)."""
        arr = (KStat * 16)()
        n = ctypes.c_int()
        _check(lib().nudft2_hss_kstats(self._h, arr, 16, ctypes.byref(n)))
        return {arr[i].name.decode(): {"ms": arr[i].ms, "flops": arr[i].flops, "bytes": arr[i].bytes,
                                       "launches": arr[i].launches} for i in range(n.value)}

    def close(self):
        if self._h:
            lib().nudft2_hss_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(eps=1e-10, levels=0, leaf=64, prec="fp64", refine_tol=1e-8, refine_max=8, profile=False,
          levels_y=0, fadi=False) -> Opts:
    return Opts(eps, levels, leaf, MIXED if prec == "mixed" else FP64, refine_tol, refine_max,
                (FLAG_PROFILE if profile else 0) | (FLAG_FADI if fadi else 0), levels_y)


def build_batched(problems, factor: bool = True, threads: int = 8, stream=None):
    """Build (and factor) many independent problems at once.  problems: list of dicts with x, y
    (M,), nx, ny and optional NudftHSS options (eps, levels, leaf, prec, refine_tol, refine_max).
    The problems run concurrently on their own streams.  Returns a list of NudftHSS handles."""
    n = len(problems)
    xs = [torch.as_tensor(p["x"]).to(device="cuda", dtype=torch.float64).contiguous() for p in problems]
    ys = [torch.as_tensor(p["y"]).to(device="cuda", dtype=torch.float64).contiguous() for p in problems]
    keys = ("eps", "levels", "leaf", "prec", "refine_tol", "refine_max", "levels_y", "fadi")
    opts = (Opts * n)(*[_opts(**{k: p[k] for k in keys if k in p}) for p in problems])
    px = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs])
    py = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ys])
    Ms = (ctypes.c_int64 * n)(*[t.numel() for t in xs])
    nxs = (ctypes.c_int * n)(*[int(p["nx"]) for p in problems])
    nys = (ctypes.c_int * n)(*[int(p["ny"]) for p in problems])
    out = (ctypes.c_void_p * n)()
    st = (ctypes.c_int * n)()
    code = lib().nudft2_hss_build_batched(n, px, py, Ms, nxs, nys, opts, int(factor), threads, _stream(stream),
                                          out, st)
    if code != OK:
        for hp in out:
            if hp:
                lib().nudft2_hss_free(ctypes.c_void_p(hp))
        _check(code)
    hs = []
    for i, p in enumerate(problems):
        h = NudftHSS.__new__(NudftHSS)
        h._h = ctypes.c_void_p(out[i])
        h.x, h.y = xs[i], ys[i]
        h.M = xs[i].numel()
        h.nx, h.ny, h.N = int(p["nx"]), int(p["ny"]), int(p["nx"]) * int(p["ny"])
        h.stream = stream
        hs.append(h)
    return hs


def solve_batched(handles, fs, threads: int = 8, stream=None):
    """Solve problem i of a batch for fs[i] ((M_i,) or (M_i, s_i) complex128 CUDA); returns the list of c."""
    n = len(handles)
    fcs = [_colmajor(f, h.M) for f, h in zip(fs, handles)]
    cs = [torch.empty((fc.shape[0], h.N), dtype=torch.complex128, device="cuda") for fc, h in zip(fcs, handles)]
    hp = (ctypes.c_void_p * n)(*[h._h.value for h in handles])
    pf = (ctypes.c_void_p * n)(*[fc.data_ptr() for fc in fcs])
    pc = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cs])
    ldf = (ctypes.c_int64 * n)(*[h.M for h in handles])
    ldc = (ctypes.c_int64 * n)(*[h.N for h in handles])
    nr = (ctypes.c_int * n)(*[fc.shape[0] for fc in fcs])
    _check(lib().nudft2_hss_solve_batched(n, hp, pf, ldf, nr, pc, ldc, threads, _stream(stream), None))
    return [c[0] if f.dim() == 1 else c.t() for c, f in zip(cs, fs)]


def run_batched(problems, fs, threads: int = 8, stream=None):
    """Build, factor and solve every problem of a batch, each run to completion and freed
    (nudft2_hss_run_batched): at most `threads` factorizations hold device memory at a time.
    problems: dicts as for build_batched; fs[i]: (M_i,) or (M_i, s_i) complex128 CUDA.  Returns
    the list of c (N_i,) or (N_i, s_i)."""
    n = len(problems)
    xs = [torch.as_tensor(p["x"]).to(device="cuda", dtype=torch.float64).contiguous() for p in problems]
    ys = [torch.as_tensor(p["y"]).to(device="cuda", dtype=torch.float64).contiguous() for p in problems]
    keys = ("eps", "levels", "leaf", "prec", "refine_tol", "refine_max", "levels_y", "fadi")
    opts = (Opts * n)(*[_opts(**{k: p[k] for k in keys if k in p}) for p in problems])
    Ns = [int(p["nx"]) * int(p["ny"]) for p in problems]
    fcs = [_colmajor(f, x.numel()) for f, x in zip(fs, xs)]
    cs = [torch.empty((fc.shape[0], N), dtype=torch.complex128, device="cuda") for fc, N in zip(fcs, Ns)]
    vpa = ctypes.c_void_p * n
    _check(lib().nudft2_hss_run_batched(
        n, vpa(*[t.data_ptr() for t in xs]), vpa(*[t.data_ptr() for t in ys]),
        (ctypes.c_int64 * n)(*[t.numel() for t in xs]), (ctypes.c_int * n)(*[int(p["nx"]) for p in problems]),
        (ctypes.c_int * n)(*[int(p["ny"]) for p in problems]), opts, vpa(*[fc.data_ptr() for fc in fcs]),
        (ctypes.c_int64 * n)(*[x.numel() for x in xs]), (ctypes.c_int * n)(*[fc.shape[0] for fc in fcs]),
        vpa(*[c.data_ptr() for c in cs]), (ctypes.c_int64 * n)(*Ns), threads, _stream(stream), None))
    return [c[0] if f.dim() == 1 else c.t() for c, f in zip(cs, fs)]


class _Lstsq(torch.autograd.Function):
    """c = A(x, y)^+ f through the HSS factorization; backward by nudft2_hss_grad (adjoint solve,
    one more solve and the FP64 exact applies of the point derivatives)."""

    @staticmethod
    def forward(ctx, f, x, y, nx, ny, opts):
        opts = dict(opts)
        ck = int(opts.pop("checkpoint_levels", 0))
        h = NudftHSS(x.detach(), y.detach(), nx, ny, **opts).factor()
        c = h.solve(f.detach())
        if ck > 0:
            h.checkpoint(ck)      # the backward pass factors these levels again
        ctx.h = h
        ctx.save_for_backward(f, c)
        return c

    @staticmethod
    def backward(ctx, gc):
        f, c = ctx.saved_tensors
        need_pts = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        gf, gx, gy = ctx.h.grad(f.detach(), c, gc.contiguous(), points=need_pts)
        return (gf if ctx.needs_input_grad[0] else None, gx if ctx.needs_input_grad[1] else None,
                gy if ctx.needs_input_grad[2] else None, None, None, None)


def lstsq(f: torch.Tensor, x: torch.Tensor, y: torch.Tensor, nx: int, ny: int, **opts) -> torch.Tensor:
    """Differentiable c = argmin ||A(x, y) c - f|| (f (M,) or (M, s) complex128 on CUDA; x, y (M,)
    float64).  opts go to NudftHSS (eps, levels, prec, ...); the handle is built per call.
    checkpoint_levels=k hands back the factors of the top k levels between the forward solve and
    the backward pass, which factors them again (less memory held, one partial refactorization)."""
    return _Lstsq.apply(f, x, y, nx, ny, opts)
