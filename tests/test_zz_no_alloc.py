"""The allocation-free entry point sm_sweep_static against sm_sweep.

sm_sweep_static serves callers that cannot call cudaMalloc (and so cannot
create a problem workspace): it keeps every intermediate buffer in one static
device array.  This test calls it through the C ABI twice in a row -- the
second call starting from the first call's intensity, so the shared scratch
is reused with stale contents from the previous call -- and checks both
results against the regular sm_sweep path within the parity tolerance of the
FP32 sweep (1e-5 per field).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W

from _cases import config

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _desc(sm, cfg, precision, edges):
    d = sm.ProblemDesc()
    d.dim, d.nx, d.ny = 2, cfg.nx, cfg.ny
    d.x0, d.x1, d.y0, d.y1 = cfg.extent
    d.n_groups = cfg.n_groups
    d.group_edges = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_polar, d.n_azim = cfg.n_polar, cfg.n_azim
    d.a, d.c, d.dt = cfg.a, cfg.c, cfg.dt
    d.opacity_kind, d.opacity_alpha = cfg.opacity_kind, cfg.opacity_alpha
    for i in range(4):
        d.T_bdr[i] = cfg.T_bdr[i]
    d.precision = precision
    return d


def _field_err(got, ref, axis):
    d = np.abs(got - ref)
    red = tuple(range(axis, d.ndim))
    return float(np.max(d.max(axis=red) / np.maximum(np.abs(ref).max(axis=red), 1e-300)))


def test_static_entry_matches_sm_sweep_twice(gpu_lib):
    import torch
    sm = gpu_lib
    lib = sm.load()
    cfg = config(2, 24, 20, 6, 2, 4, T_bdr=(1.0, 0.0, 0.3, 0.0))
    edges = np.ascontiguousarray(cfg.edges)
    prob = sm.Problem.from_config(cfg, 32)
    T = torch.from_numpy(W.temperature_wave(cfg, seed=4)).cuda()
    sig = torch.from_numpy(O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges,
                                     W.temperature_wave(cfg, seed=4),
                                     W.scale_field(cfg, seed=5))).cuda()
    I0 = torch.from_numpy(W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=6,
                                             scale=0.05)).cuda()
    stream = torch.cuda.current_stream()
    desc = _desc(sm, cfg, 32, edges)

    # regular path: two sweeps in a row
    Ip = prob.pack(I0)
    refs = []
    for _ in range(2):
        Io = prob.empty_intensity()
        mom, clo = prob.new_moments(), prob.new_closures()
        prob.sweep(T, sig, Ip, Io, mom, clo)
        prob.synchronize()
        refs.append((prob.unpack(Io).cpu().numpy(), mom.cpu().numpy(), clo.cpu().numpy()))
        Ip = Io

    # allocation-free path: two calls in a row, canonical layouts
    Iprev = prob.unpack(prob.pack(I0))  # same FP32-rounded start as the regular path
    for k in range(2):
        Iout = torch.empty_like(Iprev)
        mom = torch.empty((cfg.n_cells, 4, 9), dtype=torch.float64, device="cuda")
        clo = torch.empty((cfg.n_cells, 4, 11), dtype=torch.float64, device="cuda")
        rc = lib.sm_sweep_static(ctypes.byref(desc), ctypes.c_void_p(stream.cuda_stream),
                                 T.data_ptr(), sig.data_ptr(), Iprev.data_ptr(), Iout.data_ptr(),
                                 mom.data_ptr(), clo.data_ptr())
        assert rc == 0, lib.sm_last_error().decode()
        I_ref, m_ref, c_ref = refs[k]
        e_I = _field_err(Iout.cpu().numpy(), I_ref, 2)
        m = mom.cpu().numpy()
        e_phi = _field_err(m[..., 0], m_ref[..., 0], 0)
        e_F = float(np.abs(m[..., 1:6] - m_ref[..., 1:6]).max() / np.abs(m_ref[..., 0]).max())
        e_SE = _field_err(m[..., 6], m_ref[..., 6], 0)
        e_E = _field_err(clo.cpu().numpy()[..., 0], c_ref[..., 0], 0)
        print(f"call {k}: I {e_I:.2e} phi {e_phi:.2e} F,T {e_F:.2e} SE {e_SE:.2e} E {e_E:.2e}")
        assert max(e_I, e_phi, e_F, e_SE, e_E) <= RTOL
        Iprev = Iout


def test_static_entry_rejects_oversized_problem(gpu_lib):
    import torch
    sm = gpu_lib
    lib = sm.load()
    cfg = config(2, 256, 256, 64, 4, 8)
    edges = np.ascontiguousarray(cfg.edges)
    desc = _desc(sm, cfg, 32, edges)
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.sm_sweep_static(ctypes.byref(desc), None, dummy.data_ptr(), dummy.data_ptr(), None,
                             dummy.data_ptr(), None, None)
    assert rc == 1
    msg = lib.sm_last_error().decode()
    assert "limited to" in msg and "16777216" in msg
