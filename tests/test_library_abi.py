"""CPU checks of the C ABI: the in-tree library builds (nvcc cross-compiles
for sm_103a without a GPU), loads, and exports every function that
include/*.h declares; argument validation happens before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in ("sm.h", "sm_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_21784_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declarations_found():
    names = _declared()
    assert "sm_sweep" in names and "sm_create_problem" in names and len(names) >= 20


def test_every_declared_symbol_is_exported(lib):
    so, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b(sm_\w+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(so, n)


def test_binding_lists_every_declared_symbol():
    import paper_2504_21784_gb300 as sm
    assert sorted(sm.EXPORTED) == _declared()


def test_invalid_descriptors_rejected_before_cuda(lib):
    import numpy as np
    import paper_2504_21784_gb300 as sm
    so = sm.load()
    edges = np.array([0.1, 1.0, 10.0])

    def create(**kw):
        d = sm.ProblemDesc()
        d.dim, d.nx, d.ny = 2, 4, 4
        d.x0, d.x1, d.y0, d.y1 = 0, 1, 0, 1
        d.n_groups = 2
        d.group_edges = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_polar, d.n_azim = 1, 1
        d.a, d.c, d.dt = 1.0, 1.0, 0.1
        d.precision = 32
        for k, v in kw.items():
            setattr(d, k, v)
        h = ctypes.c_void_p()
        rc = so.sm_create_problem(ctypes.byref(d), None, ctypes.byref(h))
        return rc, so.sm_last_error().decode()

    for kw in (dict(nx=0), dict(ny=0), dict(dim=3), dict(n_groups=0), dict(precision=16),
               dict(x1=0.0), dict(n_polar=0), dict(groups_per_warp=3), dict(strip_width=17),
               dict(prefetch_rows=9), dict(a=0.0), dict(opacity_kind=7)):
        rc, msg = create(**kw)
        assert rc == 1, (kw, rc, msg)
        assert msg
    bad = np.array([1.0, 0.5, 2.0])
    d_rc, _ = create(group_edges=bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert d_rc == 1
    # odd 1D order
    rc, _ = create(dim=1, n_polar=5)
    assert rc == 1
    assert so.sm_status_string(6) == b"SM_ERR_TIMEOUT"


def test_null_handles_rejected_before_cuda(lib):
    """Entry points that take a problem or batch handle return
    SM_ERR_INVALID_ARG with a message for a NULL handle, before any CUDA call
    (so this runs without a GPU)."""
    import paper_2504_21784_gb300 as sm
    so = sm.load()
    out = ctypes.c_int()
    calls = {
        "sm_synchronize": lambda: so.sm_synchronize(None),
        "sm_set_profiling": lambda: so.sm_set_profiling(None, 1),
        "sm_debug_set_wait_limit_ns": lambda: so.sm_debug_set_wait_limit_ns(None, 1000),
        "sm_debug_skip_publish": lambda: so.sm_debug_skip_publish(None, 1),
        "sm_debug_withhold_lo_block": lambda: so.sm_debug_withhold_lo_block(None, 1),
        "sm_debug_set_pcg_form": lambda: so.sm_debug_set_pcg_form(None, 1),
        "sm_debug_get_pcg_form": lambda: so.sm_debug_get_pcg_form(None, ctypes.byref(out)),
        "sm_batch_synchronize": lambda: so.sm_batch_synchronize(None),
    }
    for name, call in calls.items():
        rc = call()
        assert rc == 1, (name, rc)
        assert so.sm_last_error(), name
    # the destructors accept NULL as a no-op (include/sm.h)
    assert so.sm_destroy_problem(None) == 0 and so.sm_destroy_batch(None) == 0


def test_static_entry_rejects_bad_descriptors_before_cuda(lib):
    """sm_sweep_static validates its descriptor before any CUDA call: huge
    direction counts whose product would overflow an int, non-finite group
    edges or boundary temperatures, and a mesh beyond 2^30 cells are refused
    with SM_ERR_INVALID_ARG (so this runs without a GPU)."""
    import numpy as np
    import paper_2504_21784_gb300 as sm
    so = sm.load()
    edges = np.array([0.1, 1.0, 10.0])
    inf_edges = np.array([0.1, 1.0, np.inf])
    dummy = ctypes.c_void_p(16)   # never dereferenced: validation comes first

    def call(**kw):
        d = sm.ProblemDesc()
        d.dim, d.nx, d.ny = 2, 4, 4
        d.x0, d.x1, d.y0, d.y1 = 0, 1, 0, 1
        d.n_groups = 2
        d.group_edges = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_polar, d.n_azim = 1, 1
        d.a, d.c, d.dt = 1.0, 1.0, 0.1
        d.precision = 32
        for k, v in kw.items():
            if k == "T_bdr":
                d.T_bdr[0] = v
            else:
                setattr(d, k, v)
        rc = so.sm_sweep_static(ctypes.byref(d), None, dummy, dummy, None, dummy, None, None)
        return rc, so.sm_last_error().decode()

    for kw in (dict(n_polar=65536, n_azim=65536), dict(n_polar=1 << 16, n_azim=1 << 15),
               dict(n_polar=200, n_azim=1), dict(n_polar=12, n_azim=12),
               dict(group_edges=inf_edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               dict(T_bdr=float("nan")), dict(nx=1 << 16, ny=1 << 16), dict(dim=1),
               dict(dt=float("inf"))):
        rc, msg = call(**kw)
        assert rc == 1, (kw, rc, msg)
        assert msg
