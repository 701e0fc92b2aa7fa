"""ctypes binding of the C ABI in include/dwfmm.h (argument marshalling only).

Every function keeps the C name and returns the C status; ``check`` turns a
non-zero status into :class:`DwfmmError`.  The :class:`Plan` helper wraps the
calls for torch tensors (device or host) and numpy arrays.  All numerical
work runs in libdwfmm.so; importing this module without the built library
raises immediately (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdwfmm.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_STATE, \
    ERR_SINGULAR = range(1, 9)
K_EXP, K_MATERN32, K_GAUSS = 0, 1, 2
P_FP64, P_FP32, P_MIXED = 0, 1, 2
W_INV_GAMMA, W_PAPER_LOGRHO, W_EXPLICIT = 0, 1, 2
KERNELS = {"exp": K_EXP, "matern32": K_MATERN32, "gauss": K_GAUSS}
PRECISIONS = {"fp64": P_FP64, "fp32": P_FP32, "mixed": P_MIXED}
WEIGHT_RULES = {"inv_gamma": W_INV_GAMMA, "paper_logrho": W_PAPER_LOGRHO, "explicit": W_EXPLICIT}
I_TOTAL_DEGREE, I_TENSOR = 0, 1
INDEX_SETS = {"total": I_TOTAL_DEGREE, "tensor": I_TENSOR}
PHASES = ("gather", "p2m_m2m", "m2l", "l2l_l2p", "p2p", "scatter", "matvec")

# Every entry point declared in include/dwfmm.h.
EXPORTS = ("dwfmm_plan_create", "dwfmm_plan_set_nodes", "dwfmm_tree_build", "dwfmm_matvec",
           "dwfmm_solve", "dwfmm_plan_destroy", "dwfmm_status_string", "dwfmm_last_error",
           "dwfmm_plan_info", "dwfmm_near_engine", "dwfmm_far_engine", "dwfmm_m2l_engine",
           "dwfmm_plan_set_m2l_engine", "dwfmm_m2l_tune_ms", "dwfmm_plan_export", "dwfmm_tree_export", "dwfmm_lists_export",
           "dwfmm_set_profiling", "dwfmm_phase_times", "dwfmm_direct_sum_noalloc",
           "dwfmm_cg_begin", "dwfmm_cg_step", "dwfmm_cg_poll", "dwfmm_cg_result", "dwfmm_residual",
           "dwfmm_refine",
           "dwfmm_batch_create", "dwfmm_batch_matvec", "dwfmm_batch_info", "dwfmm_batch_shape",
           "dwfmm_batch_cg_step", "dwfmm_batch_engine", "dwfmm_batch_set_engine",
           "dwfmm_batch_destroy",
           "dwfmm_evaluate")


class dwfmm_config(C.Structure):
    _fields_ = [("d", C.c_int32), ("kernel", C.c_int32), ("sigma", C.c_double),
                ("gamma", C.POINTER(C.c_double)), ("weight_rule", C.c_int32),
                ("weights", C.POINTER(C.c_double)), ("q", C.c_double), ("eta", C.c_double),
                ("leaf_size", C.c_int32), ("halton_candidates", C.c_int32),
                ("precision", C.c_int32), ("max_rhs", C.c_int32), ("index_set", C.c_int32)]


class DwfmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dwfmm status {status}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_2402_09531_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    i32, i64, dbl = C.c_int32, C.c_int64, C.c_double
    pd = C.POINTER(C.c_double)
    sig = {
        "dwfmm_plan_create": (i32, [C.POINTER(dwfmm_config), P, C.POINTER(P)]),
        "dwfmm_plan_set_nodes": (i32, [P, P, i64, P]),
        "dwfmm_tree_build": (i32, [P, P, i64, i64, P]),
        "dwfmm_matvec": (i32, [P, P, P, i32, i64, i64, P]),
        "dwfmm_solve": (i32, [P, dbl, P, P, i32, i64, dbl, i32, C.POINTER(i32), pd, P]),
        "dwfmm_plan_destroy": (i32, [P]),
        "dwfmm_status_string": (C.c_char_p, [i32]),
        "dwfmm_last_error": (C.c_char_p, [P]),
        "dwfmm_plan_info": (i32, [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
        "dwfmm_near_engine": (i32, [P, C.POINTER(i32)]),
        "dwfmm_far_engine": (i32, [P, C.POINTER(i32)]),
        "dwfmm_m2l_engine": (i32, [P, C.POINTER(i32)]),
        "dwfmm_plan_set_m2l_engine": (i32, [P, i32]),
        "dwfmm_m2l_tune_ms": (i32, [P, P]),
        "dwfmm_plan_export": (i32, [P, P, P, P, P, P]),
        "dwfmm_tree_export": (i32, [P, P, P, P, P, P]),
        "dwfmm_lists_export": (i32, [P, P, P]),
        "dwfmm_set_profiling": (i32, [P, i32]),
        "dwfmm_phase_times": (i32, [P, P, P, i32]),
        "dwfmm_direct_sum_noalloc": (i32, [i32, dbl, P, i64, i32, i64, P, P, i32, i64, i64, P]),
        "dwfmm_cg_begin": (i32, [P, dbl, P, i32, i64, dbl, P]),
        "dwfmm_cg_step": (i32, [P, i32, P]),
        "dwfmm_cg_poll": (i32, [P, C.POINTER(i32), P, P, P]),
        "dwfmm_cg_result": (i32, [P, P, i64, P]),
        "dwfmm_residual": (i32, [P, dbl, P, P, P, i32, i64, P, P]),
        "dwfmm_refine": (i32, [P, dbl, P, P, P, P, i32, i64, P, P, P]),
        "dwfmm_batch_create": (i32, [P, P, i32, P, C.POINTER(P)]),
        "dwfmm_batch_matvec": (i32, [P, P, P, P]),
        "dwfmm_batch_info": (i32, [P, C.POINTER(i32), P, C.POINTER(i64)]),
        "dwfmm_batch_cg_step": (i32, [P, i32, P]),
        "dwfmm_batch_shape": (i32, [P, P]),
        "dwfmm_batch_engine": (i32, [P, P, P, P]),
        "dwfmm_batch_set_engine": (i32, [P, i32]),
        "dwfmm_batch_destroy": (i32, [P]),
        "dwfmm_evaluate": (i32, [P, P, i64, i64, P, i64, P, i64, i32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(a) -> int | None:
    """Data pointer of a torch tensor or numpy array (None for None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _ld(a, name: str) -> int:
    """Row stride (in elements) of a 2-D float64 array whose rows are
    contiguous: the layout every buffer of the C ABI has.  Anything else
    (another dtype, a strided column, fewer than two dimensions) would be
    misread on the C side, so it raises ValueError here."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {a.dtype}")
        if a.dim() != 2:
            raise ValueError(f"{name} must be 2-D, got shape {tuple(a.shape)}")
        rows, cols = int(a.shape[0]), int(a.shape[1])
        if cols > 1 and a.stride(1) != 1:
            raise ValueError(f"{name} must have contiguous rows (column stride 1)")
        ld = int(a.stride(0))
    else:
        if a.dtype != np.float64:
            raise ValueError(f"{name} must be float64, got {a.dtype}")
        if a.ndim != 2:
            raise ValueError(f"{name} must be 2-D, got shape {a.shape}")
        rows, cols = int(a.shape[0]), int(a.shape[1])
        if cols > 1 and a.strides[1] != 8:
            raise ValueError(f"{name} must have contiguous rows (column stride 8 bytes)")
        if a.strides[0] % 8 != 0:
            raise ValueError(f"{name} row stride must be a multiple of 8 bytes")
        ld = int(a.strides[0] // 8)
    if rows > 1 and ld < cols:
        raise ValueError(f"{name} rows overlap (row stride {ld} < {cols} columns)")
    return max(ld, cols) if rows <= 1 else ld


def _same_layout(ref, ref_name: str, ld: int, *others):
    """Buffers that the C ABI reads with one row stride must share it."""
    for a, name in others:
        if a is None:
            continue
        if tuple(a.shape) != tuple(ref.shape):
            raise ValueError(f"{name} must have the shape of {ref_name} {tuple(ref.shape)}, got {tuple(a.shape)}")
        if _ld(a, name) != ld:
            raise ValueError(f"{name} must have the row stride of {ref_name} ({ld})")


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """One DW-FMM plan: expansion (plan_create), tree (tree_build), matvec, solve."""

    def __init__(self, d: int, kernel: str = "exp", sigma: float = 1.0, gamma=None,
                 weight_rule: str = "inv_gamma", weights=None, q: float = 4.0, eta: float = 1.0,
                 leaf_size: int = 64, halton_candidates: int = 0, precision: str = "fp64",
                 max_rhs: int = 16, stream=None, index_set: str = "total"):
        self._l = lib()
        self.d = int(d)
        self.precision = precision
        self.max_rhs = int(max_rhs)
        g = np.ascontiguousarray(np.ones(d) if gamma is None else np.asarray(gamma, dtype=np.float64))
        w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
        self._keep = (g, w)
        cfg = dwfmm_config(self.d, KERNELS[kernel], float(sigma),
                           g.ctypes.data_as(C.POINTER(C.c_double)),
                           WEIGHT_RULES[weight_rule],
                           w.ctypes.data_as(C.POINTER(C.c_double)) if w is not None else None,
                           float(q), float(eta), int(leaf_size), int(halton_candidates),
                           PRECISIONS[precision], self.max_rhs, INDEX_SETS[index_set])
        h = C.c_void_p()
        st = self._l.dwfmm_plan_create(C.byref(cfg), _stream_handle(stream), C.byref(h))
        if st != OK:
            raise DwfmmError(st, self._l.dwfmm_status_string(st).decode())
        self.h = h
        self.n_x = self.info()[0]

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self._l.dwfmm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cols(self, a, name: str):
        """Once a tree is built, (R, N) buffers must have N columns."""
        n = getattr(self, "n", None)
        if n is not None and int(a.shape[1]) != n:
            raise ValueError(f"{name} must have N = {n} columns, got {int(a.shape[1])}")

    def check(self, st: int):
        if st != OK:
            msg = self._l.dwfmm_last_error(self.h).decode() if self.h else ""
            raise DwfmmError(st, msg or self._l.dwfmm_status_string(st).decode())

    # -- calls ---------------------------------------------------------------
    def set_nodes(self, nodes, stream=None):
        a = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64))
        self.check(self._l.dwfmm_plan_set_nodes(self.h, a.ctypes.data, a.shape[0], _stream_handle(stream)))

    def tree_build(self, pts, stream=None):
        """pts: (N, d) float64, torch (cuda or cpu) or numpy, row-major."""
        n = int(pts.shape[0])
        ld = _ld(pts, "pts") if n else self.d
        if n and int(pts.shape[1]) != self.d:
            raise ValueError(f"pts must have d = {self.d} columns, got {int(pts.shape[1])}")
        self._pts_keep = pts
        self.n = None   # no tree until the build succeeds
        self.check(self._l.dwfmm_tree_build(self.h, _ptr(pts), n, ld, _stream_handle(stream)))
        self.n = n

    def matvec(self, x, y, stream=None):
        """x, y: (R, N) float64 (each row one right-hand side, contiguous)."""
        R = int(x.shape[0])
        ldx, ldy = _ld(x, "x"), _ld(y, "y")
        self._cols(x, "x")
        if tuple(y.shape) != tuple(x.shape):
            raise ValueError(f"y must have the shape of x {tuple(x.shape)}, got {tuple(y.shape)}")
        self.check(self._l.dwfmm_matvec(self.h, _ptr(x), _ptr(y), R, ldx, ldy, _stream_handle(stream)))
        return y

    def solve(self, lam: float, f, c, rtol: float = 1e-6, maxit: int = 1000, stream=None):
        R = int(f.shape[0])
        ld = _ld(f, "f")
        self._cols(f, "f")
        _same_layout(f, "f", ld, (c, "c"))
        it = C.c_int32(0)
        rel = (C.c_double * R)()
        st = self._l.dwfmm_solve(self.h, float(lam), _ptr(f), _ptr(c), R, ld, float(rtol), int(maxit),
                                 C.byref(it), rel, _stream_handle(stream))
        return st, int(it.value), [float(v) for v in rel]

    def evaluate(self, targets, c, out, stream=None):
        """Interpolant at new points: out (R, nt) = sum_j phi(|t - x_j|) c (R, N)."""
        nt = int(targets.shape[0])
        ldt = _ld(targets, "targets") if nt else self.d
        R = int(c.shape[0])
        ldc, ldo = _ld(c, "c"), _ld(out, "out")
        self._cols(c, "c")
        if nt and int(targets.shape[1]) != self.d:
            raise ValueError(f"targets must have d = {self.d} columns, got {int(targets.shape[1])}")
        if tuple(out.shape) != (R, nt):
            raise ValueError(f"out must have shape {(R, nt)}, got {tuple(out.shape)}")
        self.check(self._l.dwfmm_evaluate(self.h, _ptr(targets), nt, ldt, _ptr(c), ldc, _ptr(out), ldo, R,
                                          _stream_handle(stream)))
        return out

    # -- incremental CG (many solves in flight) -----------------------------
    def cg_begin(self, lam: float, f, rtol: float = 1e-6, stream=None):
        """f: (R, N) float64 cuda tensor."""
        ld = _ld(f, "f")
        self._cols(f, "f")
        self._cg_R = int(f.shape[0])
        self._cg_f = f
        self.check(self._l.dwfmm_cg_begin(self.h, float(lam), _ptr(f), self._cg_R, ld,
                                          float(rtol), _stream_handle(stream)))

    def cg_step(self, iters: int, stream=None):
        self.check(self._l.dwfmm_cg_step(self.h, int(iters), _stream_handle(stream)))

    def cg_poll(self):
        """(ready, status[R], iters[R], rr[R]) without blocking."""
        R = self._cg_R
        ready = C.c_int32(0)
        st = np.zeros(R, dtype=np.int32)
        it = np.zeros(R, dtype=np.int32)
        rr = np.zeros(R)
        self.check(self._l.dwfmm_cg_poll(self.h, C.byref(ready), st.ctypes.data, it.ctypes.data, rr.ctypes.data))
        return bool(ready.value), st, it, rr

    def cg_result(self, c, stream=None):
        ld = _ld(c, "c")
        self._cols(c, "c")
        self.check(self._l.dwfmm_cg_result(self.h, _ptr(c), ld, _stream_handle(stream)))
        return c

    def residual(self, lam: float, f, c, r=None, stream=None):
        R = int(f.shape[0])
        ld = _ld(f, "f")
        self._cols(f, "f")
        _same_layout(f, "f", ld, (c, "c"), (r, "r"))
        rel = np.zeros(R)
        self.check(self._l.dwfmm_residual(self.h, float(lam), _ptr(f), _ptr(c), _ptr(r), R, ld,
                                          rel.ctypes.data, _stream_handle(stream)))
        return rel

    def refine(self, lam: float, f, c, delta, r, stream=None):
        """c += alpha delta, r -= alpha (K64 + lam I) delta with a per-column
        alpha that never raises ||r|| (1 where plain refinement lowers it,
        else the minimal-residual length); r must hold f - (K64 + lam I) c.
        c and r are updated in place.  Returns (alpha, relres)."""
        R = int(f.shape[0])
        ld = _ld(f, "f")
        self._cols(f, "f")
        _same_layout(f, "f", ld, (c, "c"), (delta, "delta"), (r, "r"))
        alpha = np.zeros(R)
        rel = np.zeros(R)
        self.check(self._l.dwfmm_refine(self.h, float(lam), _ptr(f), _ptr(c), _ptr(delta), _ptr(r), R, ld,
                                        alpha.ctypes.data, rel.ctypes.data, _stream_handle(stream)))
        return alpha, rel

    def info(self):
        nx, nf, nn, dep = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()
        self.check(self._l.dwfmm_plan_info(self.h, C.byref(nx), C.byref(nf), C.byref(nn), C.byref(dep)))
        return int(nx.value), int(nf.value), int(nn.value), int(dep.value)

    NEAR_ENGINES = {-1: "none", 0: "fp64_list", 1: "fp64_symmetric", 2: "fp32_cuda_cores",
                    3: "mixed_tf32_tensor", 4: "mixed_symmetric_fp16_tensor",
                    5: "mixed_symmetric_fp16_tensor_exponent"}

    def near_engine(self) -> str:
        """Engine that evaluated the near field in the last matvec."""
        e = C.c_int32(-1)
        self.check(self._l.dwfmm_near_engine(self.h, C.byref(e)))
        return self.NEAR_ENGINES.get(int(e.value), str(e.value))

    FAR_ENGINES = {-1: "none", 0: "fp64_cuda_cores", 1: "fp32_cuda_cores", 2: "mixed_fp16_tensor"}

    def far_engine(self) -> str:
        """Engine that ran the expansion phases (P2M/M2M/L2L/L2P) in the last matvec."""
        e = C.c_int32(-1)
        self.check(self._l.dwfmm_far_engine(self.h, C.byref(e)))
        return self.FAR_ENGINES.get(int(e.value), str(e.value))

    M2L_ENGINES = {-1: "none", 0: "fp64_cuda_cores", 1: "fp32_cuda_cores", 2: "mixed_tf32_tensor",
                   3: "mixed_symmetric_fp16_tensor"}

    def m2l_engine(self) -> str:
        """Engine that ran the couplings (M2L) in the last matvec."""
        e = C.c_int32(-1)
        self.check(self._l.dwfmm_m2l_engine(self.h, C.byref(e)))
        return self.M2L_ENGINES.get(int(e.value), str(e.value))

    def set_m2l_engine(self, engine: str = "auto"):
        """M2L engine of MIXED matvecs with 9..16 right-hand sides: "auto"
        (timed once per tree), "mixed_tf32_tensor" or "mixed_symmetric_fp16_tensor"."""
        code = {"auto": -1, "mixed_tf32_tensor": 2, "mixed_symmetric_fp16_tensor": 3}[engine]
        self.check(self._l.dwfmm_plan_set_m2l_engine(self.h, code))

    def m2l_tune_ms(self):
        """(symmetric, ordered) M2L times of the per-tree timing, -1 where not timed."""
        ms = (C.c_double * 2)()
        self.check(self._l.dwfmm_m2l_tune_ms(self.h, ms))
        return float(ms[0]), float(ms[1])

    def export_expansion(self):
        n, d = self.n_x, self.d
        w = np.zeros(d)
        lam = np.zeros((n, d), dtype=np.int32)
        nodes = np.zeros((n, d))
        piv = np.zeros(n, dtype=np.int32)
        vinv = np.zeros((n, n))
        self.check(self._l.dwfmm_plan_export(self.h, w.ctypes.data, lam.ctypes.data, nodes.ctypes.data,
                                             piv.ctypes.data, vinv.ctypes.data))
        return dict(weights=w, lam=lam, nodes=nodes, pivots=piv, vinv=vinv)

    def export_tree(self):
        _, _, _, J = self.info()
        nc = (1 << (J + 1)) - 1
        perm = np.zeros(self.n, dtype=np.int64)
        b = np.zeros(nc, dtype=np.int64)
        e = np.zeros(nc, dtype=np.int64)
        lo = np.zeros((nc, self.d))
        hi = np.zeros((nc, self.d))
        self.check(self._l.dwfmm_tree_export(self.h, perm.ctypes.data, b.ctypes.data, e.ctypes.data,
                                             lo.ctypes.data, hi.ctypes.data))
        return dict(depth=J, perm=perm, begin=b, end=e, lo=lo, hi=hi)

    def export_lists(self):
        _, nf, nn, _ = self.info()
        far = np.zeros((nf, 2), dtype=np.int32)
        near = np.zeros((nn, 2), dtype=np.int32)
        self.check(self._l.dwfmm_lists_export(self.h, far.ctypes.data, near.ctypes.data))
        return far, near

    def set_profiling(self, on: bool, serialize: bool = False):
        self.check(self._l.dwfmm_set_profiling(self.h, (2 if serialize else 1) if on else 0))

    def phase_times(self, reset: bool = True):
        ms = np.zeros(7)
        ln = np.zeros(7, dtype=np.int64)
        self.check(self._l.dwfmm_phase_times(self.h, ms.ctypes.data, ln.ctypes.data, 1 if reset else 0))
        return {p: (float(ms[i]), int(ln[i])) for i, p in enumerate(PHASES)}


class Batch:
    """Many uneven problems (float32 plans with built trees) in one fused matvec."""

    def __init__(self, plans, nrhs, stream=None):
        self._l = lib()
        self.plans = list(plans)
        self.nrhs = [int(r) for r in nrhs]
        hs = (C.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        rs = (C.c_int32 * len(self.plans))(*self.nrhs)
        h = C.c_void_p()
        st = self._l.dwfmm_batch_create(hs, rs, len(self.plans), _stream_handle(stream), C.byref(h))
        if st != OK:
            msg = self._l.dwfmm_last_error(self.plans[0].h).decode()
            raise DwfmmError(st, msg or self._l.dwfmm_status_string(st).decode())
        self.h = h

    def matvec(self, xs, ys, stream=None):
        """xs[i], ys[i]: (nrhs_i, N_i) float64 cuda tensors (contiguous)."""
        if len(xs) != len(self.plans) or len(ys) != len(self.plans):
            raise ValueError(f"one x and one y per problem ({len(self.plans)})")
        for i, (x, y) in enumerate(zip(xs, ys)):
            want = (self.nrhs[i], int(getattr(self.plans[i], "n", -1)))
            for a, name in ((x, f"xs[{i}]"), (y, f"ys[{i}]")):
                if _ld(a, name) != want[1] or tuple(a.shape) != want:
                    raise ValueError(f"{name} must be a contiguous {want} float64 tensor, got {tuple(a.shape)}")
        xp = (C.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        yp = (C.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        st = self._l.dwfmm_batch_matvec(self.h, xp, yp, _stream_handle(stream))
        if st != OK:
            raise DwfmmError(st, self._l.dwfmm_status_string(st).decode())

    def cg_step(self, iters: int, stream=None):
        """`iters` CG iterations of every problem (each begun with
        Plan.cg_begin); one fused batch matvec per iteration."""
        st = self._l.dwfmm_batch_cg_step(self.h, int(iters), _stream_handle(stream))
        if st != OK:
            msg = self._l.dwfmm_last_error(self.plans[0].h).decode() if self.plans else ""
            raise DwfmmError(st, msg or self._l.dwfmm_status_string(st).decode())

    def info(self):
        split = C.c_int32(0)
        tune = (C.c_double * 2)()
        leaves = C.c_int64(0)
        self._l.dwfmm_batch_info(self.h, C.byref(split), tune, C.byref(leaves))
        shape = (C.c_int32 * 4)()
        self._l.dwfmm_batch_shape(self.h, shape)
        return {"split": bool(split.value), "tune_ms": [tune[0], tune[1]], "leaves": int(leaves.value),
                "near_shape": {"per_class": bool(shape[0]), "threads": int(shape[1])},
                "m2l_shape": {"per_class": bool(shape[2]), "threads": int(shape[3])}}

    def engine(self):
        """The matvec engine in use ("graph" or "persistent"), whether the
        persistent one is available, the creation timings (ms) of both and the
        persistent launch's CTAs and group widths."""
        eng = (C.c_int32 * 2)()
        ms = (C.c_double * 2)()
        launch = (C.c_int32 * 3)()
        st = self._l.dwfmm_batch_engine(self.h, eng, ms, launch)
        if st != OK:
            raise DwfmmError(st, self._l.dwfmm_status_string(st).decode())
        return {"engine": "persistent" if eng[0] else "graph", "persistent_available": bool(eng[1]),
                "ms": {"graph": ms[0], "persistent": ms[1]},
                "persistent_launch": {"ctas": int(launch[0]), "near_threads": int(launch[1]),
                                      "m2l_threads": int(launch[2])}}

    def set_engine(self, engine: str):
        """Use "graph" (captured launches) or "persistent" (one cooperative launch)."""
        if engine not in ("graph", "persistent"):
            raise ValueError("engine must be 'graph' or 'persistent'")
        st = self._l.dwfmm_batch_set_engine(self.h, 1 if engine == "persistent" else 0)
        if st != OK:
            msg = self._l.dwfmm_last_error(self.plans[0].h).decode() if self.plans else ""
            raise DwfmmError(st, msg or self._l.dwfmm_status_string(st).decode())

    def close(self):
        if getattr(self, "h", None):
            self._l.dwfmm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
