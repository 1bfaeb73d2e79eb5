"""FP64 CPU oracle for the SM thermal-radiative-transfer hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library under ``paper_2504_21784_gb300`` never imports, links or
executes anything here, and this package imports nothing from the library.

The arithmetic lives in ``sm_oracle.c`` (plain C, FP64, compiled with gcc);
this module is argument marshalling plus a few pure-numpy helpers that restate
definitions (no method arithmetic beyond what each docstring cites).

Functions and the paper passage each follows:

==========================  ===================================================
``gauss_legendre``          GL rule used by the S_N sets (Sec. 6.1, 6.3, 6.4)
``quadrature``              {Omega_d, w_d} (Sec. 2), product set in 2D
``planck_P / rosseland_R``  b_g, r_g integrands (Sec. 2, Eq. planck, r_g def.)
``group_spectra``           b_g(T), r_g(T) with sum = 1 (Sec. 2)
``opacity``                 sigma_g from the cell-mean T (Sec. 3, Rem. opacity)
``emission``                sigma_g B_g(T)/4pi at the nodes (Eq. smm_be_transport)
``inflow``                  B_g(T_bdr)/4pi (Eq. transport, boundary condition)
``sweep`` / ``sweep_pairs`` lumped upwind DG solve (Eqs. upwind, dgsn_transport)
``moments``                 E, F, T, sum sigma_g E_g, sum sigma_g F_g (Sec. 2)
``closures``                sigma_E, sigma_F, sigma_P, additive correction (Sec. 2)
``alpha``                   Eq. alpha with S_N quadrature
==========================  ===================================================

Every function above is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, invariants, textbook or
library routines, or brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sm_oracle.c")
_LIB = os.path.join(_HERE, "libsm_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile ``sm_oracle.c`` into ``libsm_oracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-std=c11", "-Wall", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        sig = {
            "orc_gauss_legendre": (_I, [_I, _PD, _PD]),
            "orc_quadrature_1d": (_I, [_I, _PD, _PD]),
            "orc_quadrature_2d": (_I, [_I, _I, _PD, _PD, _PD]),
            "orc_planck_P": (_D, [_D]),
            "orc_planck_Q": (_D, [_D]),
            "orc_planck_P_head": (_D, [_D]),
            "orc_planck_P_tail": (_D, [_D]),
            "orc_rosseland_R": (_D, [_D]),
            "orc_rosseland_RQ": (_D, [_D]),
            "orc_bernoulli_over_factorial": (_D, [_I]),
            "orc_group_spectra": (None, [_I, _PD, _D, _PD, _PD]),
            "orc_opacity": (None, [_I, _D, _I, _PD, _I, _I, _PD, _PD, _PD]),
            "orc_emission": (None, [_I, _PD, _D, _D, _I, _I, _PD, _PD, _PD]),
            "orc_inflow": (None, [_I, _PD, _D, _D, _PD, _PD]),
            "orc_sweep_pairs": (_I, [_I, _I, _I, _D, _D, _D, _D, _I, _PD, _PD, _I, _PD, _D,
                                     _PD, _PD, _I, _PD, _I, _PI, _PD, _I]),
            "orc_moments": (None, [_I, _I, _I, _PD, _PD, _PD, _I, _PD, _PD, _PD]),
            "orc_closures": (None, [_I, _I, _I, _PD, _D, _PD, _PD, _PD, _PD]),
            "orc_alpha": (_D, [_I, _PD, _PD]),
            "orc_num_threads": (_I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------- quadrature
def gauss_legendre(n: int):
    lib = _load()
    x = np.zeros(n)
    w = np.zeros(n)
    if lib.orc_gauss_legendre(n, _p(x), _p(w)):
        raise ValueError("n must be >= 1")
    return x, w


def quadrature(dim: int, n_polar: int, n_azim: int = 0):
    """Return (omx, omy, w).  1D: n_polar GL points (omy = 0).  2D: 4*np*na."""
    lib = _load()
    if dim == 1:
        omx = np.zeros(n_polar)
        w = np.zeros(n_polar)
        lib.orc_quadrature_1d(n_polar, _p(omx), _p(w))
        return omx, np.zeros(n_polar), w
    nd = 4 * n_polar * n_azim
    omx, omy, w = np.zeros(nd), np.zeros(nd), np.zeros(nd)
    if lib.orc_quadrature_2d(n_polar, n_azim, _p(omx), _p(omy), _p(w)) != nd:
        raise ValueError("bad quadrature")
    return omx, omy, w


def alpha(omx, w) -> float:
    omx, w = _f64(omx), _f64(w)
    return _load().orc_alpha(len(omx), _p(omx), _p(w))


# --------------------------------------------------------------------------- Planck
def planck_P(x: float) -> float:
    return _load().orc_planck_P(float(x))


def planck_Q(x: float) -> float:
    return _load().orc_planck_Q(float(x))


def planck_P_head(x: float) -> float:
    return _load().orc_planck_P_head(float(x))


def planck_P_tail(x: float) -> float:
    return _load().orc_planck_P_tail(float(x))


def rosseland_R(x: float) -> float:
    return _load().orc_rosseland_R(float(x))


def bernoulli_over_factorial(j: int) -> float:
    return _load().orc_bernoulli_over_factorial(int(j))


def group_spectra(edges, T: float):
    edges = _f64(edges)
    G = len(edges) - 1
    b, r = np.zeros(G), np.zeros(G)
    _load().orc_group_spectra(G, _p(edges), float(T), _p(b), _p(r))
    return b, r


# --------------------------------------------------------------------------- materials / sources
def opacity(kind: int, alpha_: float, edges, T_nodal, scale):
    """sigma[g][cell].  kind 0: s_K Tbar^-3; kind 1: s_K alpha (1-e^{-E_g/Tbar})/E_g^3."""
    edges, T_nodal, scale = _f64(edges), _f64(T_nodal), _f64(scale)
    G = len(edges) - 1
    ncell, nnode = T_nodal.shape
    sig = np.zeros((G, ncell))
    _load().orc_opacity(int(kind), float(alpha_), G, _p(edges), ncell, nnode, _p(T_nodal),
                        _p(scale), _p(sig))
    return sig


def emission(edges, a: float, c: float, T_nodal, sigma):
    """q[g][cell][node] = sigma_g a c T^4 b_g(T) / 4pi at every node."""
    edges, T_nodal, sigma = _f64(edges), _f64(T_nodal), _f64(sigma)
    G = len(edges) - 1
    ncell, nnode = T_nodal.shape
    q = np.zeros((G, ncell, nnode))
    _load().orc_emission(G, _p(edges), float(a), float(c), ncell, nnode, _p(T_nodal),
                         _p(sigma), _p(q))
    return q


def inflow(edges, a: float, c: float, T_bdr):
    """inflow[side][g] = a c T^4 b_g(T)/4pi per side (T <= 0: vacuum)."""
    edges, T_bdr = _f64(edges), _f64(T_bdr)
    G = len(edges) - 1
    out = np.zeros((4, G))
    _load().orc_inflow(G, _p(edges), float(a), float(c), _p(T_bdr), _p(out))
    return out


# --------------------------------------------------------------------------- sweep
def sweep_pairs(dim, nx, ny, extent, omx, omy, sigma, inv_cdt, q, I_prev, inflow_, pairs=None,
                nthreads: int = 0):
    """Sweep the listed (d, g) pairs (all when ``pairs`` is None).

    ``I_prev`` is [d][g][cell][node], or [pair][cell][node] for just the listed
    pairs.  Returns I[pair][cell][node] (all: reshaped to [d][g][cell][node])."""
    lib = _load()
    omx, omy, sigma, q, inflow_ = map(_f64, (omx, omy, sigma, q, inflow_))
    G = sigma.shape[0]
    ncell = sigma.shape[1]
    nn = 2 if dim == 1 else 4
    nd = len(omx)
    if pairs is None:
        npair = nd * G
        ppairs = None
    else:
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        npair = pr.shape[0]
        ppairs = pr.ctypes.data_as(_PI)
    per_pair = 0
    if I_prev is not None:
        I_prev = _f64(I_prev)
        if pairs is not None and I_prev.size == npair * ncell * nn:
            per_pair = 1  # I^k given only for the listed pairs
        else:
            assert I_prev.size == nd * G * ncell * nn
        pprev = _p(I_prev)
    else:
        pprev = None
    out = np.zeros((npair, ncell, nn))
    x0, x1, y0, y1 = extent
    rc = lib.orc_sweep_pairs(dim, nx, ny if dim == 2 else 1, x0, x1, y0, y1, nd, _p(omx),
                             _p(omy), G, _p(sigma), float(inv_cdt), _p(q), pprev, per_pair,
                             _p(inflow_), npair, ppairs, _p(out), int(nthreads))
    if rc:
        raise FloatingPointError("singular local system in oracle sweep")
    if pairs is None:
        return out.reshape(nd, G, ncell, nn)
    return out


def sweep(dim, nx, ny, extent, omx, omy, sigma, inv_cdt, q, I_prev, inflow_, nthreads=0):
    return sweep_pairs(dim, nx, ny, extent, omx, omy, sigma, inv_cdt, q, I_prev, inflow_, None,
                       nthreads)


def moments(dim, omx, omy, w, sigma, I):
    """mom[cell][node][m]; 2D m = phi,Fx,Fy,Txx,Txy,Tyy,SE,SFx,SFy; 1D phi,F,T,SE,SF."""
    omx, omy, w, sigma, I = map(_f64, (omx, omy, w, sigma, I))
    G, ncell = sigma.shape
    nd = len(omx)
    nn = 2 if dim == 1 else 4
    nm = 5 if dim == 1 else 9
    assert I.size == nd * G * ncell * nn
    mom = np.zeros((ncell, nn, nm))
    _load().orc_moments(dim, ncell, nd, _p(omx), _p(omy), _p(w), G, _p(sigma), _p(I), _p(mom))
    return mom


def closures(dim, edges, c, sigma, T_nodal, mom):
    """out[cell][node][k]; 2D k = E,Fx,Fy,Txx,Txy,Tyy,sigE,sigF,sigP,Cx,Cy; 1D E,F,T,sigE,sigF,sigP,C."""
    edges, sigma, T_nodal, mom = map(_f64, (edges, sigma, T_nodal, mom))
    G, ncell = sigma.shape
    nn = 2 if dim == 1 else 4
    no = 7 if dim == 1 else 11
    out = np.zeros((ncell, nn, no))
    _load().orc_closures(dim, ncell, G, _p(edges), float(c), _p(sigma), _p(T_nodal), _p(mom),
                         _p(out))
    return out


def num_threads() -> int:
    return _load().orc_num_threads()
