"""The allocation-free entry point sm_sweep_static against sm_sweep and the
oracle.

sm_sweep_static serves callers that cannot call cudaMalloc (and so cannot
create a problem workspace): it keeps every intermediate buffer in one static
device array.  Each case calls it through the C ABI twice in a row -- the
second call starting from the first call's intensity, so the shared scratch
is reused with stale contents from the previous call -- and checks

* the intensity bit for bit against the regular sm_sweep path with the same
  slots per lane (the same cell solves in the same order), and the moments
  and all eleven closure fields within 1e-12 (FP64) / 2e-6 (FP32) of it (the
  moments are summed with atomics, in another order);
* every output against the FP64 oracle within the parity bars, 1e-11 (FP64)
  and 1e-5 (FP32) per field;
* that a call leaves the device's free memory unchanged (after a first call:
  with lazy module loading the 16 MiB static array itself is placed when the
  library's module is first loaded).

FP32 and FP64 sweeps, with and without a previous intensity.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W

from _cases import config, parity_errors

pytestmark = pytest.mark.gpu

TOL = {64: 1e-11, 32: 1e-5}
SAME = {64: 1e-12, 32: 2e-6}


def _desc(sm, cfg, precision, edges, gw=1):
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
    d.groups_per_warp = gw
    return d


def _field_err(got, ref, axis):
    d = np.abs(got - ref)
    red = tuple(range(axis, d.ndim))
    return float(np.max(d.max(axis=red) / np.maximum(np.abs(ref).max(axis=red), 1e-300)))


@pytest.mark.parametrize("with_prev", [True, False])
@pytest.mark.parametrize("precision", [32, 64])
def test_static_entry_matches_sm_sweep_twice(gpu_lib, precision, with_prev):
    import torch
    sm = gpu_lib
    lib = sm.load()
    cfg = config(2, 24, 20, 6, 2, 4, T_bdr=(1.0, 0.0, 0.3, 0.0))
    edges = np.ascontiguousarray(cfg.edges)
    prob = sm.Problem.from_config(cfg, precision, groups_per_warp=1)
    Tn = W.temperature_wave(cfg, seed=4)
    sig_n = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, Tn,
                      W.scale_field(cfg, seed=5))
    T = torch.from_numpy(Tn).cuda()
    sig = torch.from_numpy(sig_n).cuda()
    I0 = torch.from_numpy(W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=6,
                                             scale=0.05)).cuda()
    stream = torch.cuda.current_stream()
    desc = _desc(sm, cfg, precision, edges)

    # regular path: two sweeps in a row
    Ip = prob.pack(I0) if with_prev else None
    refs = []
    for _ in range(2):
        Io = prob.empty_intensity()
        mom, clo = prob.new_moments(), prob.new_closures()
        prob.sweep(T, sig, Ip, Io, mom, clo)
        prob.synchronize()
        refs.append((prob.unpack(Io).cpu().numpy(), mom.cpu().numpy(), clo.cpu().numpy()))
        Ip = Io

    # allocation-free path: two calls in a row, canonical layouts
    Iprev = prob.unpack(prob.pack(I0)) if with_prev else None  # the same rounded start
    mom = torch.empty((cfg.n_cells, 4, 9), dtype=torch.float64, device="cuda")
    clo = torch.empty((cfg.n_cells, 4, 11), dtype=torch.float64, device="cuda")
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    q = O.emission(cfg.edges, cfg.a, cfg.c, Tn, sig_n)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    # a first call, so that the library's module (with its static array) is
    # loaded before free memory is compared across the calls below
    warm = torch.empty((cfg.n_dir, cfg.n_groups, cfg.n_cells, 4), dtype=torch.float64,
                       device="cuda")
    assert lib.sm_sweep_static(ctypes.byref(desc), ctypes.c_void_p(stream.cuda_stream),
                               T.data_ptr(), sig.data_ptr(), None, warm.data_ptr(), None,
                               None) == 0, lib.sm_last_error().decode()
    del warm
    for k in range(2):
        Iout = torch.empty((cfg.n_dir, cfg.n_groups, cfg.n_cells, 4), dtype=torch.float64,
                           device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = lib.sm_sweep_static(ctypes.byref(desc), ctypes.c_void_p(stream.cuda_stream),
                                 T.data_ptr(), sig.data_ptr(),
                                 Iprev.data_ptr() if Iprev is not None else None,
                                 Iout.data_ptr(), mom.data_ptr(), clo.data_ptr())
        assert rc == 0, lib.sm_last_error().decode()
        free1 = torch.cuda.mem_get_info()[0]
        I_ref, m_ref, c_ref = refs[k]
        Ig, m, c = Iout.cpu().numpy(), mom.cpu().numpy(), clo.cpu().numpy()
        same_I = bool(np.array_equal(Ig, I_ref))
        e_m = max(_field_err(m[..., j], m_ref[..., j], 0) for j in range(9))
        e_c = max(_field_err(c[..., j], c_ref[..., j], 0) for j in range(11))
        # the oracle, from the same (rounded) previous intensity
        Ik = Iprev.cpu().numpy() if Iprev is not None else None
        Ir = O.sweep(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, sig_n, 1.0 / (cfg.c * cfg.dt), q,
                     Ik, infl)
        mr = O.moments(2, omx, omy, w, sig_n, Ir)
        cr = O.closures(2, cfg.edges, cfg.c, sig_n, Tn, mr)
        e = parity_errors(cfg, (Ig, m, c), (Ir, mr, cr), precision, TOL[precision])
        print(f"fp{precision} prev {with_prev} call {k}: intensity identical {same_I}, moments "
              f"{e_m:.2e} closures {e_c:.2e} vs sm_sweep; oracle " +
              "  ".join(f"{n} {v:.2e}" for n, v in e.items()) +
              f"; free memory change {free0 - free1} B")
        assert same_I
        assert e_m <= SAME[precision] and e_c <= SAME[precision]
        bad = {n: v for n, v in e.items() if not v <= TOL[precision]}
        assert not bad, f"parity above {TOL[precision]}: {bad}"
        assert free1 == free0
        Iprev = Iout


def test_static_entry_rejects_oversized_problem(gpu_lib):
    import torch
    sm = gpu_lib
    lib = sm.load()
    cfg = config(2, 256, 256, 64, 4, 8)
    edges = np.ascontiguousarray(cfg.edges)
    desc = _desc(sm, cfg, 32, edges, gw=0)
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.sm_sweep_static(ctypes.byref(desc), None, dummy.data_ptr(), dummy.data_ptr(), None,
                             dummy.data_ptr(), None, None)
    assert rc == 1
    msg = lib.sm_last_error().decode()
    assert "limited to" in msg and "16777216" in msg
