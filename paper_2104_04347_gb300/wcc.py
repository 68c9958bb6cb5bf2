"""Python binding of the WCC C ABI (include/wcc.h): argument marshalling only.

Every step of the computation runs in libwcc.so's CUDA kernels.  If the
library is missing or no GPU is usable, the calls raise -- there is no CPU
fallback in this package.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwcc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wcc.h")

ADVECTION, BURGERS, EULER = 0, 1, 2
PERIODIC, TRANSMISSIVE = 0, 1
FP64, FP32_MIXED, FP32 = 0, 1, 2

ERRORS = {
    -1: "WCC_E_INVAL", -2: "WCC_E_STATE", -3: "WCC_E_NOMEM", -4: "WCC_E_CUDA",
    -5: "WCC_E_NONFINITE", -6: "WCC_E_POSITIVITY", -7: "WCC_E_CAPACITY", -8: "WCC_E_CFL",
}


class WCCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("adv_speed", ctypes.c_double),
        ("graph_chunk", ctypes.c_int),
        ("tb_depth", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("tb_cfl_growth", ctypes.c_double),
        ("cells_per_block", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class Options2D(ctypes.Structure):
    """Mirror of wcc2d_options (include/wcc2d.h)."""

    _fields_ = [
        ("precision", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("ax", ctypes.c_double),
        ("ay", ctypes.c_double),
        ("rows_per_cta", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
    ]


_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "wcc_default_options": (None, [ctypes.POINTER(Options)]),
    "wcc_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                  _dp, ctypes.c_int, ctypes.POINTER(Options)]),
    "wcc_num_cells": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc_set_initial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wcc_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]),
    "wcc_step_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _dp]),
    "wcc_tb_stats": (ctypes.c_int, [ctypes.c_void_p, _i64p, _i64p, _dp]),
    "wcc_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
    "wcc_step_until": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int64)]),
    "wcc_get_dofs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wcc_get_state": (ctypes.c_int, [ctypes.c_void_p, _dp, _i64p, ctypes.POINTER(ctypes.c_int)]),
    "wcc_get_dt_history": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_int64, _i64p]),
    "wcc_synchronize": (ctypes.c_int, [ctypes.c_void_p]),
    "wcc_device_bytes": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc_launch_count": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc_measure_fp_peak": (ctypes.c_int, [ctypes.c_int, _dp]),
    "wcc_stability_limit": (ctypes.c_int, [ctypes.c_int, _dp]),
    "wcc_default_cfl": (ctypes.c_int, [ctypes.c_int, _dp]),
    "wcc_advance_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp,
                                          ctypes.POINTER(Options), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_double, _dp]),
    "wcc_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64, _i64p,
                                        ctypes.POINTER(ctypes.c_int), _dp, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(Options)]),
    "wcc_batch_dof_count": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc_batch_set_initial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wcc_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]),
    "wcc_batch_get_dofs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wcc_batch_get_times": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_int64]),
    "wcc_batch_get_state": (ctypes.c_int, [ctypes.c_void_p, _i64p, ctypes.POINTER(ctypes.c_int)]),
    "wcc_batch_get_dt_history": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _dp, ctypes.c_int64, _i64p]),
    "wcc_batch_set_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "wcc_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "wcc_batch_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int)]),
    "wcc_batch_tb_stats": (ctypes.c_int, [ctypes.c_void_p, _i64p, _i64p]),
    "wcc_batch_synchronize": (ctypes.c_int, [ctypes.c_void_p]),
    "wcc_batch_launch_count": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc_batch_device_bytes": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "wcc_batch_destroy": (None, [ctypes.c_void_p]),
    "wcc_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "wcc_destroy": (None, [ctypes.c_void_p]),
    "wcc2d_default_options": (None, [ctypes.POINTER(Options2D)]),
    "wcc2d_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int, _dp, ctypes.c_int, ctypes.POINTER(Options2D)]),
    "wcc2d_stage_dims": (ctypes.c_int, [ctypes.c_void_p, _i64p, _i64p]),
    "wcc2d_set_initial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wcc2d_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]),
    "wcc2d_step_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _dp]),
    "wcc2d_step_until": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _i64p]),
    "wcc2d_get_dofs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wcc2d_get_state": (ctypes.c_int, [ctypes.c_void_p, _dp, _i64p, ctypes.POINTER(ctypes.c_int)]),
    "wcc2d_get_dt_history": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_int64, _i64p]),
    "wcc2d_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "wcc2d_synchronize": (ctypes.c_int, [ctypes.c_void_p]),
    "wcc2d_launch_count": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc2d_device_bytes": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
    "wcc2d_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "wcc2d_destroy": (ctypes.c_int, [ctypes.c_void_p]),
}


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions declared in a public header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wcc(?:2d)?_\w+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libwcc.so (building it first if needed).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                from . import build as _build
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not found at {path}; run the build first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def default_options() -> Options:
    o = Options()
    load().wcc_default_options(ctypes.byref(o))
    return o


def measure_fp_peak(precision: int) -> float:
    """FMA throughput of the current device in TFLOP/s (FP64 or FP32)."""
    v = ctypes.c_double()
    rc = load().wcc_measure_fp_peak(int(precision), ctypes.byref(v))
    if rc != 0:
        raise WCCError(rc, "peak measurement failed")
    return v.value


def stability_limit(P: int) -> float:
    """Linear stability limit of degree P (the library's von Neumann scan)."""
    v = ctypes.c_double()
    rc = load().wcc_stability_limit(int(P), ctypes.byref(v))
    if rc != 0:
        raise WCCError(rc, f"no stability limit for P = {P}")
    return v.value


def default_cfl(P: int) -> float:
    """The library's default CFL number of degree P."""
    v = ctypes.c_double()
    rc = load().wcc_default_cfl(int(P), ctypes.byref(v))
    if rc != 0:
        raise WCCError(rc, f"no default CFL number for P = {P}")
    return v.value


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


class Solver:
    """One WCC problem on the GPU (wraps a wcc_handle).

    ``dofs`` arrays are float64 [cells, nv, P+1] of the paper-scaled
    derivatives, as in include/wcc.h.  ``stream`` is a raw cudaStream_t
    handle (e.g. ``torch.cuda.Stream().cuda_stream``) or None."""

    def __init__(self, system: int, N: int, P: int, domain, bc: int, *, precision: int = FP64,
                 limiter: bool = True, alpha: float = 2.0, eps: float = 1e-40, gamma: float = 1.4,
                 adv_speed: float = 1.0, graph_chunk: int = 32, stream: int | None = None, tb_depth: int = 1,
                 tb_cfl_growth: float = 0.1, cells_per_block: int = 0):
        self.lib = load()
        o = default_options()
        o.precision = precision
        o.limiter = 1 if limiter else 0
        o.alpha = alpha
        o.eps = eps
        o.gamma = gamma
        o.adv_speed = adv_speed
        o.graph_chunk = graph_chunk
        o.cuda_stream = stream
        o.tb_depth = tb_depth
        o.tb_cfl_growth = tb_cfl_growth
        o.cells_per_block = cells_per_block
        h = ctypes.c_void_p()
        dom = (ctypes.c_double * 2)(float(domain[0]), float(domain[1]))
        rc = self.lib.wcc_create(ctypes.byref(h), system, int(N), int(P), dom, bc, ctypes.byref(o))
        if rc != 0:
            raise WCCError(rc, self.lib.wcc_last_error(None).decode())
        self.h = h
        self.system, self.N, self.P, self.bc = system, int(N), int(P), bc
        self.nv = 3 if system == EULER else 1
        self.dx = (float(domain[1]) - float(domain[0])) / int(N)

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise WCCError(rc, self.lib.wcc_last_error(self.h).decode())

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.wcc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def num_cells(self) -> int:
        n = ctypes.c_int64()
        self._check(self.lib.wcc_num_cells(self.h, ctypes.byref(n)))
        return n.value

    def set_initial(self, dofs: np.ndarray) -> None:
        a = np.ascontiguousarray(dofs, dtype=np.float64)
        self._check(self.lib.wcc_set_initial(self.h, _ptr(a), a.size))

    def set_initial_ptr(self, host_ptr: int, count: int) -> None:
        """Load from a raw host pointer (e.g. pinned memory)."""
        self._check(self.lib.wcc_set_initial(self.h, ctypes.c_void_p(host_ptr), int(count)))

    def step(self, nsteps: int, cfl: float) -> None:
        self._check(self.lib.wcc_step(self.h, int(nsteps), float(cfl)))

    def step_dt(self, dts) -> None:
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(self.lib.wcc_step_dt(self.h, d.size, d.ctypes.data_as(_dp)))

    def autotune(self, cfl: float):
        """Time the compiled launch configurations on the current stage, keep
        the fastest; returns (cells_per_block, tb_depth)."""
        cpb, tb = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wcc_autotune(self.h, float(cfl), ctypes.byref(cpb), ctypes.byref(tb)))
        return cpb.value, tb.value

    def tb_stats(self):
        """(pairs taken, pairs refused and re-done singly, largest second
        half-step CFL number) of the two-half-step launches."""
        pairs, fb, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.wcc_tb_stats(self.h, ctypes.byref(pairs), ctypes.byref(fb), ctypes.byref(nu)))
        return pairs.value, fb.value, nu.value

    def step_until(self, t_end: float, cfl: float) -> int:
        """Advance to exactly t_end on an integer stage; returns the half-steps taken."""
        n = ctypes.c_int64(0)
        self._check(self.lib.wcc_step_until(self.h, float(t_end), float(cfl), ctypes.byref(n)))
        return int(n.value)

    def get_dofs(self) -> np.ndarray:
        n = self.num_cells()
        out = np.empty((n, self.nv, self.P + 1))
        self._check(self.lib.wcc_get_dofs(self.h, _ptr(out), out.size))
        return out

    def get_dofs_ptr(self, host_ptr: int, count: int) -> None:
        self._check(self.lib.wcc_get_dofs(self.h, ctypes.c_void_p(host_ptr), int(count)))

    def state(self):
        t = ctypes.c_double()
        s = ctypes.c_int64()
        p = ctypes.c_int()
        self._check(self.lib.wcc_get_state(self.h, ctypes.byref(t), ctypes.byref(s), ctypes.byref(p)))
        return t.value, s.value, p.value

    def dt_history(self) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.wcc_get_dt_history(self.h, None, 0, ctypes.byref(n)))
        out = np.empty(n.value)
        self._check(self.lib.wcc_get_dt_history(self.h, out.ctypes.data_as(_dp), out.size, ctypes.byref(n)))
        return out

    def synchronize(self) -> None:
        self._check(self.lib.wcc_synchronize(self.h))

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.wcc_device_bytes(self.h, ctypes.byref(b)))
        return b.value

    def launch_count(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.wcc_launch_count(self.h, ctypes.byref(b)))
        return b.value


class Batch:
    """Many independent problems advanced together (wraps a wcc_batch).

    ``problems`` is a list of objects with system, N, P, x_l, x_r, bc and q0
    (e.g. paper_2104_04347_gb300.inputs.Problem); all share the system.
    Host arrays are the concatenation of the instances' [cells, nv, P+1]."""

    def __init__(self, problems, *, limiter: bool = True, alpha: float = 2.0, eps: float = 1e-40,
                 gamma: float = 1.4, adv_speed: float = 1.0, graph_chunk: int = 32, stream: int | None = None,
                 tb_depth: int = 1, tb_cfl_growth: float = 0.1):
        self.lib = load()
        self.problems = list(problems)
        n = len(self.problems)
        system = self.problems[0].system
        o = default_options()
        o.precision = FP32_MIXED
        o.limiter = 1 if limiter else 0
        o.alpha, o.eps, o.gamma, o.adv_speed = alpha, eps, gamma, adv_speed
        o.graph_chunk = graph_chunk
        o.cuda_stream = stream
        o.tb_depth = tb_depth
        o.tb_cfl_growth = tb_cfl_growth
        Ns = (ctypes.c_int64 * n)(*[p.N for p in self.problems])
        Ps = (ctypes.c_int * n)(*[p.P for p in self.problems])
        doms = (ctypes.c_double * (2 * n))(*[v for p in self.problems for v in (p.x_l, p.x_r)])
        bcs = (ctypes.c_int * n)(*[p.bc for p in self.problems])
        h = ctypes.c_void_p()
        rc = self.lib.wcc_batch_create(ctypes.byref(h), system, n, Ns, Ps, doms, bcs, ctypes.byref(o))
        if rc != 0:
            raise WCCError(rc, self.lib.wcc_batch_last_error(None).decode())
        self.h = h
        self.system = system
        self.nv = 3 if system == EULER else 1
        self.count = n

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise WCCError(rc, self.lib.wcc_batch_last_error(self.h).decode())

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.wcc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def dof_count(self) -> int:
        c = ctypes.c_int64()
        self._check(self.lib.wcc_batch_dof_count(self.h, ctypes.byref(c)))
        return c.value

    def set_initial(self, qs=None) -> None:
        qs = [p.q0 for p in self.problems] if qs is None else qs
        a = np.ascontiguousarray(np.concatenate([np.asarray(q, dtype=np.float64).reshape(-1) for q in qs]))
        self._check(self.lib.wcc_batch_set_initial(self.h, _ptr(a), a.size))

    def set_initial_ptr(self, host_ptr: int, count: int) -> None:
        self._check(self.lib.wcc_batch_set_initial(self.h, ctypes.c_void_p(host_ptr), int(count)))

    def step(self, nsteps: int, cfl: float) -> None:
        self._check(self.lib.wcc_batch_step(self.h, int(nsteps), float(cfl)))

    def state(self):
        s = ctypes.c_int64()
        p = ctypes.c_int()
        self._check(self.lib.wcc_batch_get_state(self.h, ctypes.byref(s), ctypes.byref(p)))
        return s.value, p.value

    def get_dofs(self):
        """List of [cells, nv, P+1] arrays, one per instance."""
        _, parity = self.state()
        flat = np.empty(self.dof_count())
        self._check(self.lib.wcc_batch_get_dofs(self.h, _ptr(flat), flat.size))
        out, off = [], 0
        for p in self.problems:
            cells = p.N if p.bc == PERIODIC else (p.N + 1 if parity == 0 else p.N)
            n = cells * self.nv * (p.P + 1)
            out.append(flat[off:off + n].reshape(cells, self.nv, p.P + 1))
            off += n
        return out

    def get_dofs_ptr(self, host_ptr: int, count: int) -> None:
        self._check(self.lib.wcc_batch_get_dofs(self.h, ctypes.c_void_p(host_ptr), int(count)))

    def times(self) -> np.ndarray:
        t = np.empty(self.count)
        self._check(self.lib.wcc_batch_get_times(self.h, t.ctypes.data_as(_dp), self.count))
        return t

    def dt_history(self, instance: int) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.wcc_batch_get_dt_history(self.h, int(instance), None, 0, ctypes.byref(n)))
        out = np.empty(n.value)
        self._check(self.lib.wcc_batch_get_dt_history(self.h, int(instance), out.ctypes.data_as(_dp), out.size,
                                                      ctypes.byref(n)))
        return out

    def set_grid(self, ctas: int) -> None:
        self._check(self.lib.wcc_batch_set_grid(self.h, int(ctas)))

    def autotune(self, cfl: float) -> int:
        c = ctypes.c_int()
        self._check(self.lib.wcc_batch_autotune(self.h, float(cfl), ctypes.byref(c)))
        return c.value

    def tuning(self):
        """(persistent grid in CTAs, half-steps per launch)."""
        c, d = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wcc_batch_get_tuning(self.h, ctypes.byref(c), ctypes.byref(d)))
        return c.value, d.value

    def tb_stats(self):
        """(pairs taken, pairs refused and re-done as single half-steps)."""
        p, f = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.wcc_batch_tb_stats(self.h, ctypes.byref(p), ctypes.byref(f)))
        return p.value, f.value

    def synchronize(self) -> None:
        self._check(self.lib.wcc_batch_synchronize(self.h))

    def launch_count(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.wcc_batch_launch_count(self.h, ctypes.byref(b)))
        return b.value

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.wcc_batch_device_bytes(self.h, ctypes.byref(b)))
        return b.value


class Solver2D:
    """One 2D WCC problem on the GPU (wraps a wcc2d_handle, include/wcc2d.h).

    ``dofs`` arrays are float64 [rows, cols, nv, nq] of the scaled
    derivatives u_{kx,ly}, nq = (P+1)(P+2)/2, position (k+l)(k+l+1)/2 + l.
    ``domain`` is (x_S, x_E, y_S, y_E).  precision is FP64, FP32_MIXED
    (float arithmetic, float-float cell averages) or FP32."""

    def __init__(self, system: int, nx: int, ny: int, P: int, domain, bc: int, *, precision: int = FP64,
                 limiter: bool = True, alpha: float = 2.0, eps: float = 1e-40, gamma: float = 1.4,
                 ax: float = 1.0, ay: float = 1.0, rows_per_cta: int = 16, stream: int | None = None):
        self.lib = load()
        o = Options2D()
        self.lib.wcc2d_default_options(ctypes.byref(o))
        o.precision = precision
        o.limiter = 1 if limiter else 0
        o.alpha, o.eps, o.gamma, o.ax, o.ay = alpha, eps, gamma, ax, ay
        o.rows_per_cta = rows_per_cta
        o.cuda_stream = stream
        h = ctypes.c_void_p()
        dom = (ctypes.c_double * 4)(*[float(d) for d in domain])
        rc = self.lib.wcc2d_create(ctypes.byref(h), system, int(nx), int(ny), int(P), dom, bc, ctypes.byref(o))
        if rc != 0:
            raise WCCError(rc, self.lib.wcc2d_last_error(None).decode())
        self.h = h
        self.system, self.nx, self.ny, self.P, self.bc = system, int(nx), int(ny), int(P), bc
        self.nv = 4 if system == EULER else 1
        self.nq = (P + 1) * (P + 2) // 2

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise WCCError(rc, self.lib.wcc2d_last_error(self.h).decode())

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.wcc2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stage_dims(self):
        nx, ny = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.wcc2d_stage_dims(self.h, ctypes.byref(nx), ctypes.byref(ny)))
        return nx.value, ny.value

    def set_initial(self, dofs: np.ndarray) -> None:
        a = np.ascontiguousarray(dofs, dtype=np.float64)
        self._check(self.lib.wcc2d_set_initial(self.h, _ptr(a), a.size))

    def step(self, nsteps: int, cfl: float) -> None:
        self._check(self.lib.wcc2d_step(self.h, int(nsteps), float(cfl)))

    def step_dt(self, dts) -> None:
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(self.lib.wcc2d_step_dt(self.h, d.size, d.ctypes.data_as(_dp)))

    def step_until(self, t_end: float, cfl: float) -> int:
        n = ctypes.c_int64(0)
        self._check(self.lib.wcc2d_step_until(self.h, float(t_end), float(cfl), ctypes.byref(n)))
        return int(n.value)

    def get_dofs(self) -> np.ndarray:
        nx, ny = self.stage_dims()
        out = np.empty((ny, nx, self.nv, self.nq))
        self._check(self.lib.wcc2d_get_dofs(self.h, _ptr(out), out.size))
        return out

    def state(self):
        t, s, p = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int()
        self._check(self.lib.wcc2d_get_state(self.h, ctypes.byref(t), ctypes.byref(s), ctypes.byref(p)))
        return t.value, s.value, p.value

    def dt_history(self) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.wcc2d_get_dt_history(self.h, None, 0, ctypes.byref(n)))
        out = np.empty(n.value)
        self._check(self.lib.wcc2d_get_dt_history(self.h, out.ctypes.data_as(_dp), out.size, ctypes.byref(n)))
        return out

    def autotune(self, cfl: float) -> int:
        """Time the strip heights on the current stage, keep the fastest, restore the state."""
        r = ctypes.c_int()
        self._check(self.lib.wcc2d_autotune(self.h, float(cfl), ctypes.byref(r)))
        return r.value

    def synchronize(self) -> None:
        self._check(self.lib.wcc2d_synchronize(self.h))

    def launch_count(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.wcc2d_launch_count(self.h, ctypes.byref(b)))
        return b.value

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        self._check(self.lib.wcc2d_device_bytes(self.h, ctypes.byref(b)))
        return b.value
