"""GB300 (sm_103a) Second Moment TRT hot path: Python binding of libsmtrt.so.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels (``csrc/``), reached through the C ABI of ``include/sm.h``.  PyTorch
supplies device memory and the CUDA stream.  There is no CPU fallback: if the
library has not been built (``python -m paper_2504_21784_gb300.build`` or
``__graft_entry__.build()``) every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmtrt.so")

SM_OK = 0
METHOD_INDEPENDENT, METHOD_CONSISTENT = 0, 1
STATUS = {0: "SM_OK", 1: "SM_ERR_INVALID_ARG", 2: "SM_ERR_CUDA", 3: "SM_ERR_OOM",
          4: "SM_ERR_NO_CONVERGENCE", 5: "SM_ERR_NONPHYSICAL", 6: "SM_ERR_TIMEOUT",
          7: "SM_ERR_UNSUPPORTED"}

#: every symbol declared in include/sm.h and include/sm_debug.h
EXPORTED = ["sm_create_problem", "sm_destroy_problem", "sm_get_info", "sm_set_stream",
            "sm_set_tiling", "sm_get_quadrature", "sm_opacity", "sm_emission", "sm_sweep",
            "sm_closures", "sm_sweep_host", "sm_pack_intensity", "sm_unpack_intensity",
            "sm_synchronize", "sm_autotune", "sm_set_profiling", "sm_get_kernel_times",
            "sm_launch_count", "sm_last_error", "sm_status_string",
            "sm_debug_set_wait_limit_ns", "sm_debug_skip_publish", "sm_debug_withhold_lo_block",
            "sm_debug_set_pcg_form", "sm_debug_get_pcg_form", "sm_debug_exp_neg",
            "sm_debug_set_batch_lo", "sm_set_tail_strips", "sm_debug_set_emission_fp64",
            "sm_sweep_static",
            "sm_default_step_params", "sm_loworder_newton", "sm_step",
            "sm_create_batch", "sm_destroy_batch", "sm_batch_problem", "sm_batch_get_info",
            "sm_batch_set_stream", "sm_batch_set_tiling", "sm_batch_sweep",
            "sm_batch_synchronize", "sm_batch_autotune", "sm_ho_step", "sm_leakage",
            "sm_adjoint_step", "sm_set_quadrant_moments", "sm_batch_step",
            "sm_batch_set_profiling", "sm_batch_get_kernel_times", "sm_batch_tune_slots",
            "sm_set_emission_warps"]


class SMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double), ("n_groups", ctypes.c_int),
                ("group_edges", ctypes.POINTER(ctypes.c_double)), ("n_polar", ctypes.c_int),
                ("n_azim", ctypes.c_int), ("a", ctypes.c_double), ("c", ctypes.c_double),
                ("dt", ctypes.c_double), ("opacity_kind", ctypes.c_int),
                ("opacity_alpha", ctypes.c_double), ("T_bdr", ctypes.c_double * 4),
                ("precision", ctypes.c_int), ("groups_per_warp", ctypes.c_int),
                ("strip_width", ctypes.c_int), ("prefetch_rows", ctypes.c_int)]


class ProblemInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "dim", "nx", "ny", "n_dir", "n_groups", "n_cells", "n_nodes", "n_moments", "n_closures",
        "precision", "dirs_per_quadrant", "groups_per_lane_row", "groups_per_warp",
        "n_groups_padded", "n_warp_tasks", "strip_width", "prefetch_rows", "n_tasks", "n_strips")] + [
        ("intensity_elems", ctypes.c_size_t), ("intensity_bytes", ctypes.c_size_t),
        ("workspace_bytes", ctypes.c_size_t), ("alpha", ctypes.c_double),
        ("emission_warps", ctypes.c_int), ("tail_strips", ctypes.c_int)]


class StepParams(ctypes.Structure):
    """Iteration controls of the low-order solve and the step (sm_step_params)."""
    _fields_ = [("eps_outer", ctypes.c_double), ("eps_inner", ctypes.c_double),
                ("pcg_rtol", ctypes.c_double), ("elim_rtol", ctypes.c_double),
                ("T_floor", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("max_pcg", ctypes.c_int),
                ("max_elim", ctypes.c_int), ("method", ctypes.c_int), ("refine", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "outer_iters", "newton_iters_total", "newton_iters_max", "pcg_iters_total",
        "pcg_iters_max", "pcg_capped", "elim_iters_max", "converged")] + [
        ("last_change", ctypes.c_double), ("refine_corrections", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "n_problems", "n_tasks", "strip_width", "prefetch_rows", "resident_ctas",
        "graphs_cached")] + [("smem_bytes", ctypes.c_size_t), ("updates", ctypes.c_double),
                              ("launches", ctypes.c_int64)]


def step_params(**overrides) -> StepParams:
    """The library's default iteration controls with the given fields replaced."""
    prm = StepParams()
    load().sm_default_step_params(ctypes.byref(prm))
    for k, v in overrides.items():
        if k not in dict(StepParams._fields_):
            raise KeyError(k)
        setattr(prm, k, v)
    return prm


def _stats(st: StepStats) -> dict:
    return {f: getattr(st, f) for f, _ in StepStats._fields_}


_lib = None


def load():
    """Load libsmtrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -m paper_2504_21784_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    PD = ctypes.POINTER(ctypes.c_double)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "sm_create_problem": [ctypes.POINTER(ProblemDesc), P, ctypes.POINTER(P)],
        "sm_destroy_problem": [P],
        "sm_get_info": [P, ctypes.POINTER(ProblemInfo)],
        "sm_set_stream": [P, P],
        "sm_set_tiling": [P, I, I],
        "sm_set_emission_warps": [P, I],
        "sm_get_quadrature": [P, PD, PD, PD],
        "sm_opacity": [P, P, P, P],
        "sm_emission": [P, P, P, P],
        "sm_sweep": [P, P, P, P, P, P, P],
        "sm_closures": [P, P, P, P, P],
        "sm_sweep_host": [P, P, P, P, P, P, P],
        "sm_pack_intensity": [P, P, P],
        "sm_unpack_intensity": [P, P, P],
        "sm_synchronize": [P],
        "sm_autotune": [P, P, P, P, P, I],
        "sm_set_profiling": [P, I],
        "sm_get_kernel_times": [P, PD, ctypes.POINTER(ctypes.c_int)],
        "sm_debug_set_wait_limit_ns": [P, ctypes.c_longlong],
        "sm_debug_skip_publish": [P, I],
        "sm_debug_withhold_lo_block": [P, I],
        "sm_debug_set_pcg_form": [P, I],
        "sm_debug_get_pcg_form": [P, ctypes.POINTER(ctypes.c_int)],
        "sm_debug_exp_neg": [P, P, I, P],
        "sm_debug_set_batch_lo": [P, I],
        "sm_set_tail_strips": [P, I],
        "sm_debug_set_emission_fp64": [P, I],
        "sm_sweep_static": [ctypes.POINTER(ProblemDesc), P, P, P, P, P, P, P],
        "sm_loworder_newton": [P, P, P, P, P, P, P, P, ctypes.POINTER(StepParams),
                               ctypes.POINTER(StepStats)],
        "sm_step": [P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(StepParams),
                    ctypes.POINTER(StepStats)],
        "sm_create_batch": [ctypes.POINTER(ProblemDesc), I, P, ctypes.POINTER(P)],
        "sm_destroy_batch": [P],
        "sm_batch_problem": [P, I, ctypes.POINTER(P)],
        "sm_batch_get_info": [P, ctypes.POINTER(BatchInfo)],
        "sm_batch_set_stream": [P, P],
        "sm_batch_set_tiling": [P, I, I],
        "sm_batch_sweep": [P, PP, PP, PP, PP, PP, PP],
        "sm_batch_synchronize": [P],
        "sm_batch_autotune": [P, PP, PP, PP, PP, I],
        "sm_batch_step": [P, PP, PP, PP, PP, PP, PP, PP, PP, PP, ctypes.POINTER(StepParams),
                          ctypes.POINTER(StepStats)],
        "sm_batch_set_profiling": [P, I],
        "sm_batch_tune_slots": [ctypes.POINTER(ProblemDesc), I, P, I, ctypes.POINTER(ctypes.c_int)],
        "sm_batch_get_kernel_times": [P, PD, ctypes.POINTER(ctypes.c_int)],
        "sm_ho_step": [P, P, P, P, P, P, D, I, ctypes.POINTER(ctypes.c_int)],
        "sm_set_quadrant_moments": [P, P],
        "sm_leakage": [P, P, PD],
        "sm_adjoint_step": [P, P, P, P, P, P, P, P, P, P, P, D, I,
                            ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.sm_default_step_params.argtypes = [ctypes.POINTER(StepParams)]
    lib.sm_default_step_params.restype = None
    lib.sm_launch_count.argtypes = [P]
    lib.sm_launch_count.restype = ctypes.c_int64
    lib.sm_last_error.argtypes = []
    lib.sm_last_error.restype = ctypes.c_char_p
    lib.sm_status_string.argtypes = [ctypes.c_int]
    lib.sm_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code: int):
    if code != SM_OK:
        raise SMError(code, load().sm_last_error().decode())


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _hptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


class Problem:
    """One SM transport problem on the current CUDA device."""

    def __init__(self, dim: int, nx: int, ny: int, extent: Sequence[float], edges,
                 n_polar: int, n_azim: int = 0, a: float = 1.0, c: float = 1.0,
                 dt: float = 0.01, opacity_kind: int = 0, opacity_alpha: float = 0.0,
                 T_bdr: Sequence[float] = (0.0, 0.0, 0.0, 0.0), precision: int = 32,
                 groups_per_warp: int = 0, strip_width: int = 0, prefetch_rows: int = 0,
                 stream=None):
        import torch
        lib = load()
        self._torch = torch
        self._edges = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
        d = ProblemDesc()
        d.dim, d.nx, d.ny = dim, nx, ny
        d.x0, d.x1, d.y0, d.y1 = [float(v) for v in extent]
        d.n_groups = len(self._edges) - 1
        d.group_edges = self._edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_polar, d.n_azim = n_polar, n_azim
        d.a, d.c, d.dt = a, c, dt
        d.opacity_kind, d.opacity_alpha = opacity_kind, opacity_alpha
        for i in range(4):
            d.T_bdr[i] = float(T_bdr[i])
        d.precision = precision
        d.groups_per_warp, d.strip_width, d.prefetch_rows = groups_per_warp, strip_width, prefetch_rows
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.sm_create_problem(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                                     ctypes.byref(h)))
        self._h = h
        self.refresh_info()

    @classmethod
    def from_config(cls, cfg, precision: int = 32, **kw) -> "Problem":
        return cls(cfg.dim, cfg.nx, cfg.ny, cfg.extent, cfg.edges, cfg.n_polar, cfg.n_azim,
                   cfg.a, cfg.c, cfg.dt, cfg.opacity_kind, cfg.opacity_alpha, cfg.T_bdr,
                   precision, **kw)

    # ---------------------------------------------------------------- basics
    def refresh_info(self):
        info = ProblemInfo()
        _check(load().sm_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in ProblemInfo._fields_}
        return self.info

    def close(self):
        if getattr(self, "_h", None):
            load().sm_destroy_problem(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def quadrature(self):
        n = self.info["n_dir"]
        ox, oy, w = np.zeros(n), np.zeros(n), np.zeros(n)
        PD = ctypes.POINTER(ctypes.c_double)
        _check(load().sm_get_quadrature(self._h, ox.ctypes.data_as(PD), oy.ctypes.data_as(PD),
                                        w.ctypes.data_as(PD)))
        return ox, oy, w

    def set_tiling(self, strip_width: int = 0, prefetch_rows: int = 0):
        _check(load().sm_set_tiling(self._h, strip_width, prefetch_rows))
        self.refresh_info()

    def set_emission_warps(self, warps: int):
        """0: the emission runs as its own kernel; 1..4: that many warps per
        sweep CTA compute it inside the sweep kernel (sm_set_emission_warps)."""
        _check(load().sm_set_emission_warps(self._h, int(warps)))
        self.refresh_info()

    def set_emission_fp64(self, on: bool):
        """Test hook (sm_debug_set_emission_fp64): an FP32 problem's sweeps take
        the FP64 Planck evaluation instead of the double-FP32 one."""
        _check(load().sm_debug_set_emission_fp64(self._h, 1 if on else 0))

    def set_tail_strips(self, n: int):
        """n half-width strips at each end of the x range (sm_set_tail_strips;
        0: uniform strips)."""
        _check(load().sm_set_tail_strips(self._h, int(n)))
        self.refresh_info()

    def set_stream(self, stream):
        self._stream = stream
        _check(load().sm_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    # ---------------------------------------------------------------- buffers
    def empty_intensity(self):
        """Device buffer for a packed intensity (I^k or the new I)."""
        dt = self._torch.float32 if self.info["precision"] == 32 else self._torch.float64
        return self._torch.zeros(self.info["intensity_elems"], dtype=dt, device="cuda")

    def pack(self, I_canon):
        out = self.empty_intensity()
        _check(load().sm_pack_intensity(self._h, _ptr(I_canon), _ptr(out)))
        return out

    def unpack(self, I_packed):
        i = self.info
        out = self._torch.zeros((i["n_dir"], i["n_groups"], i["n_cells"], i["n_nodes"]),
                                dtype=self._torch.float64, device="cuda")
        _check(load().sm_unpack_intensity(self._h, _ptr(I_packed), _ptr(out)))
        return out

    # ---------------------------------------------------------------- hot path
    def opacity(self, T, scale, out=None):
        i = self.info
        if out is None:
            out = self._torch.empty((i["n_groups"], i["n_cells"]), dtype=self._torch.float64,
                                    device="cuda")
        _check(load().sm_opacity(self._h, _ptr(T), _ptr(scale), _ptr(out)))
        return out

    def emission(self, T, sigma, want_q: bool = True):
        i = self.info
        q = None
        if want_q:
            q = self._torch.empty((i["n_groups"], i["n_cells"], i["n_nodes"]),
                                  dtype=self._torch.float64, device="cuda")
        _check(load().sm_emission(self._h, _ptr(T), _ptr(sigma), _ptr(q)))
        return q

    def sweep(self, T, sigma, I_prev, I_out, moments=None, closures=None):
        _check(load().sm_sweep(self._h, _ptr(T), _ptr(sigma), _ptr(I_prev), _ptr(I_out),
                               _ptr(moments), _ptr(closures)))

    def new_moments(self):
        i = self.info
        return self._torch.empty((i["n_cells"], i["n_nodes"], i["n_moments"]),
                                 dtype=self._torch.float64, device="cuda")

    def new_closures(self):
        i = self.info
        return self._torch.empty((i["n_cells"], i["n_nodes"], i["n_closures"]),
                                 dtype=self._torch.float64, device="cuda")

    def closures(self, moments, T, sigma, out=None):
        if out is None:
            out = self.new_closures()
        _check(load().sm_closures(self._h, _ptr(moments), _ptr(T), _ptr(sigma), _ptr(out)))
        return out

    def sweep_host(self, T_host: np.ndarray, sigma_host: np.ndarray, I_prev, I_out,
                   moments_host: Optional[np.ndarray], closures_host: Optional[np.ndarray]):
        """End-to-end call with host input/output buffers (copies inside)."""
        mp = _hptr(moments_host) if moments_host is not None else None
        cp = _hptr(closures_host) if closures_host is not None else None
        _check(load().sm_sweep_host(self._h, _hptr(T_host), _hptr(sigma_host), _ptr(I_prev),
                                    _ptr(I_out), mp, cp))

    def synchronize(self):
        _check(load().sm_synchronize(self._h))

    def autotune(self, T, sigma, I_prev, I_out, reps: int = 3):
        _check(load().sm_autotune(self._h, _ptr(T), _ptr(sigma), _ptr(I_prev), _ptr(I_out),
                                  reps))
        self.refresh_info()

    def set_profiling(self, on: bool):
        _check(load().sm_set_profiling(self._h, 1 if on else 0))

    def kernel_times(self):
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_int()
        _check(load().sm_get_kernel_times(self._h, ms, ctypes.byref(n)))
        return {"emission_ms": ms[0], "sweep_ms": ms[1], "reduce_ms": ms[2], "count": n.value}

    # ---------------------------------------------------------------- low order / step
    def new_nodal(self):
        """FP64 [cell][node] device array (T, E, C_v)."""
        i = self.info
        return self._torch.zeros((i["n_cells"], i["n_nodes"]), dtype=self._torch.float64,
                                 device="cuda")

    def new_flux(self):
        i = self.info
        return self._torch.zeros((i["n_cells"], i["n_nodes"], i["dim"]),
                                 dtype=self._torch.float64, device="cuda")

    def loworder_newton(self, closures, T_star, cv, moments_star, T, E, F=None,
                        params: Optional[StepParams] = None) -> dict:
        """Gray low-order Newton solve (sm_loworder_newton); T and E are
        updated in place, F (allocated when None) receives the flux.
        Returns the iteration counts, with the flux under "F"."""
        if F is None:
            F = self.new_flux()
        st = StepStats()
        _check(load().sm_loworder_newton(
            self._h, _ptr(closures), _ptr(T_star), _ptr(cv), _ptr(moments_star), _ptr(T),
            _ptr(E), _ptr(F), ctypes.byref(params) if params is not None else None,
            ctypes.byref(st)))
        out = _stats(st)
        out["F"] = F
        return out

    def step(self, scale, cv, T, E, F, moments, I_prev, I_next, closures=None,
             params: Optional[StepParams] = None) -> dict:
        """One time step of Algorithm 1 (sm_step): T, E, F, moments, I_next
        (and closures, when given) are updated in place."""
        st = StepStats()
        _check(load().sm_step(self._h, _ptr(scale), _ptr(cv), _ptr(T), _ptr(E), _ptr(F),
                              _ptr(moments), _ptr(I_prev), _ptr(I_next), _ptr(closures),
                              ctypes.byref(params) if params is not None else None,
                              ctypes.byref(st)))
        return _stats(st)

    def set_quadrant_moments(self, qmom):
        """Register a [cell][node][4][6] FP64 buffer filled by every later
        sweep with per-quadrant moments (None drops it)."""
        _check(load().sm_set_quadrant_moments(self._h, _ptr(qmom)))

    def new_quadrant_moments(self):
        i = self.info
        return self._torch.zeros((i["n_cells"], i["n_nodes"], 4, 6), dtype=self._torch.float64,
                                 device="cuda")

    # ---------------------------------------------------------------- time steps / adjoint
    def ho_step(self, scale, cv, T, I_prev, I_next, tol: float = 1e-13,
                max_iter: int = 500) -> int:
        """One backward-Euler step of the high-order problem converged by the
        unaccelerated iteration (sm_ho_step); T is updated in place.  Returns
        the number of passes."""
        it = ctypes.c_int()
        _check(load().sm_ho_step(self._h, _ptr(scale), _ptr(cv), _ptr(T), _ptr(I_prev),
                                 _ptr(I_next), float(tol), int(max_iter), ctypes.byref(it)))
        return it.value

    def leakage(self, I) -> float:
        out = ctypes.c_double()
        _check(load().sm_leakage(self._h, _ptr(I), ctypes.byref(out)))
        return out.value

    def adjoint_step(self, scale, cv, T_n, T_np1, I_np1, psi_next, X_next, psi_out, X_out,
                     grad, tol: float = 1e-13, max_iter: int = 500) -> int:
        """One adjoint step (sm_adjoint_step); psi_out, X_out written, grad += dJ/ds."""
        it = ctypes.c_int()
        _check(load().sm_adjoint_step(self._h, _ptr(scale), _ptr(cv), _ptr(T_n), _ptr(T_np1),
                                      _ptr(I_np1), _ptr(psi_next), _ptr(X_next), _ptr(psi_out),
                                      _ptr(X_out), _ptr(grad), float(tol), int(max_iter),
                                      ctypes.byref(it)))
        return it.value

    def launch_count(self) -> int:
        return int(load().sm_launch_count(self._h))

    # ---------------------------------------------------------------- test hooks
    def debug_wait_limit_ns(self, ns: int):
        _check(load().sm_debug_set_wait_limit_ns(self._h, int(ns)))

    def debug_skip_publish(self, on: bool):
        _check(load().sm_debug_skip_publish(self._h, 1 if on else 0))

    def debug_withhold_lo_block(self, on: bool):
        _check(load().sm_debug_withhold_lo_block(self._h, 1 if on else 0))

    #: conjugate-gradient forms of the low-order solve (sm_debug.h)
    PCG_FORMS = {"auto": 0, "textbook": 1, "single": 2, "mixed": 3}

    def debug_set_pcg_form(self, form: str):
        _check(load().sm_debug_set_pcg_form(self._h, self.PCG_FORMS[form]))

    def debug_pcg_form(self) -> str:
        """The form the last low-order solve used ("auto": none yet)."""
        v = ctypes.c_int()
        _check(load().sm_debug_get_pcg_form(self._h, ctypes.byref(v)))
        return {v_: k for k, v_ in self.PCG_FORMS.items()}[v.value]


def _desc_of(cfg, precision: int, keep):
    edges = np.ascontiguousarray(np.asarray(cfg.edges, dtype=np.float64))
    keep.append(edges)
    d = ProblemDesc()
    d.dim, d.nx, d.ny = cfg.dim, cfg.nx, cfg.ny
    d.x0, d.x1, d.y0, d.y1 = [float(v) for v in cfg.extent]
    d.n_groups = len(edges) - 1
    d.group_edges = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_polar, d.n_azim = cfg.n_polar, cfg.n_azim
    d.a, d.c, d.dt = cfg.a, cfg.c, cfg.dt
    d.opacity_kind, d.opacity_alpha = cfg.opacity_kind, cfg.opacity_alpha
    for i in range(4):
        d.T_bdr[i] = float(cfg.T_bdr[i])
    d.precision = precision
    return d


class _Member(Problem):
    """Borrowed handle of a batch member (not destroyed on its own)."""

    def __init__(self, handle, stream):
        import torch
        self._torch = torch
        self._h = handle
        self._stream = stream
        self._edges = None
        self.refresh_info()

    def close(self):
        self._h = None


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _ptr(t) if t is not None else None
    return arr


class Batch:
    """Many independent 2D problems swept in one persistent launch
    (``sm_batch_*``); each pass is recorded once as a CUDA graph per buffer
    set and replayed afterwards."""

    def __init__(self, cfgs, precision: int = 32, stream=None, groups_per_warp=None):
        """groups_per_warp: None (each member's automatic choice) or one value
        per member (e.g. from tune_batch_slots)."""
        import torch
        lib = load()
        self._torch = torch
        keep = []
        descs = (ProblemDesc * len(cfgs))()
        for i, cfg in enumerate(cfgs):
            descs[i] = _desc_of(cfg, precision, keep)
            if groups_per_warp is not None:
                descs[i].groups_per_warp = int(groups_per_warp[i])
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.sm_create_batch(descs, len(cfgs), ctypes.c_void_p(stream.cuda_stream),
                                   ctypes.byref(h)))
        self._h = h
        self.members = []
        for i in range(len(cfgs)):
            ph = ctypes.c_void_p()
            _check(lib.sm_batch_problem(self._h, i, ctypes.byref(ph)))
            self.members.append(_Member(ph, stream))

    def info(self) -> dict:
        bi = BatchInfo()
        _check(load().sm_batch_get_info(self._h, ctypes.byref(bi)))
        return {f: getattr(bi, f) for f, _ in BatchInfo._fields_}

    def set_tiling(self, strip_width: int = 0, prefetch_rows: int = 0):
        _check(load().sm_batch_set_tiling(self._h, strip_width, prefetch_rows))
        for m in self.members:
            m.refresh_info()

    def sweep(self, T, sigma, I_prev, I_out, moments=None, closures=None):
        """Lists of tensors, one per member (I_prev/moments/closures entries may be None)."""
        n = len(self.members)
        Ip = _ptr_array(I_prev if I_prev is not None else [None] * n)
        mo = _ptr_array(moments) if moments is not None else None
        cl = _ptr_array(closures) if closures is not None else None
        self._keep = (_ptr_array(T), _ptr_array(sigma), Ip, _ptr_array(I_out), mo, cl)
        _check(load().sm_batch_sweep(self._h, *self._keep))

    def synchronize(self):
        _check(load().sm_batch_synchronize(self._h))

    def set_profiling(self, on: bool):
        _check(load().sm_batch_set_profiling(self._h, 1 if on else 0))

    def kernel_times(self) -> dict:
        """Summed milliseconds of the timed passes: prologue and emissions,
        the batched sweep kernel, moment sums and closures."""
        ms = (ctypes.c_double * 3)()
        cnt = ctypes.c_int()
        _check(load().sm_batch_get_kernel_times(self._h, ms, ctypes.byref(cnt)))
        return {"emission_ms": ms[0], "sweep_ms": ms[1], "reduce_ms": ms[2], "count": cnt.value}

    def step(self, scale, cv, T, E, F, moments, I_prev, I_next, closures=None,
             params: Optional[StepParams] = None) -> list:
        """One time step of Algorithm 1 for every member (sm_batch_step): lists
        of tensors, one per member, updated in place as by Problem.step.
        Returns the per-member iteration counts."""
        n = len(self.members)
        st = (StepStats * n)()
        cl = _ptr_array(closures) if closures is not None else None
        keep = [_ptr_array(scale), _ptr_array(cv), _ptr_array(T), _ptr_array(E), _ptr_array(F),
                _ptr_array(moments), _ptr_array(I_prev), _ptr_array(I_next), cl]
        _check(load().sm_batch_step(self._h, *keep,
                                    ctypes.byref(params) if params is not None else None, st))
        return [_stats(st[i]) for i in range(n)]

    def set_batched_lo(self, on: bool):
        """Test hook (sm_debug_set_batch_lo): the members' low-order solves of
        Batch.step in one launch (default) or one launch per member."""
        _check(load().sm_debug_set_batch_lo(self._h, 1 if on else 0))

    def autotune(self, T, sigma, I_prev, I_out, reps: int = 2):
        n = len(self.members)
        Ip = _ptr_array(I_prev if I_prev is not None else [None] * n)
        _check(load().sm_batch_autotune(self._h, _ptr_array(T), _ptr_array(sigma), Ip,
                                        _ptr_array(I_out), reps))
        for m in self.members:
            m.refresh_info()

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m.close()
            load().sm_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_batch_slots(cfgs, precision: int = 32, reps: int = 2, stream=None) -> list:
    """Slots per lane for the members of a batch, picked by timing
    (sm_batch_tune_slots); pass the result to Batch(groups_per_warp=...)."""
    import torch
    keep = []
    descs = (ProblemDesc * len(cfgs))()
    for i, cfg in enumerate(cfgs):
        descs[i] = _desc_of(cfg, precision, keep)
    if stream is None:
        stream = torch.cuda.current_stream()
    out = (ctypes.c_int * len(cfgs))()
    _check(load().sm_batch_tune_slots(descs, len(cfgs), ctypes.c_void_p(stream.cuda_stream),
                                      int(reps), out))
    return list(out)


def sweep_static(cfg, precision: int, T, sigma, I_prev, I_out, moments=None, closures=None,
                 groups_per_warp: int = 0, stream=None):
    """Allocation-free pass of the hot path (``sm_sweep_static``) for small 2D
    problems: for callers that cannot allocate device memory.  All tensors are
    caller-owned CUDA tensors in the canonical FP64 layouts (I_prev may be
    None); the library uses its fixed 16 MiB device scratch array."""
    import torch
    edges = np.ascontiguousarray(np.asarray(cfg.edges, dtype=np.float64))
    d = ProblemDesc()
    d.dim, d.nx, d.ny = cfg.dim, cfg.nx, cfg.ny
    d.x0, d.x1, d.y0, d.y1 = [float(v) for v in cfg.extent]
    d.n_groups = len(edges) - 1
    d.group_edges = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_polar, d.n_azim = cfg.n_polar, cfg.n_azim
    d.a, d.c, d.dt = cfg.a, cfg.c, cfg.dt
    d.opacity_kind, d.opacity_alpha = cfg.opacity_kind, cfg.opacity_alpha
    for i in range(4):
        d.T_bdr[i] = float(cfg.T_bdr[i])
    d.precision = precision
    d.groups_per_warp = groups_per_warp
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().sm_sweep_static(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream), _ptr(T),
                                  _ptr(sigma), _ptr(I_prev), _ptr(I_out), _ptr(moments),
                                  _ptr(closures)))
