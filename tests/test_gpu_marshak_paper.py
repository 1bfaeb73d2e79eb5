"""The Marshak wave in the paper's units (Sec. 6: [0, 0.05 cm], 2.5 ns,
sigma = 1e12 T^-3 cm^-1 with T in eV, so the opacity spans nine orders of
magnitude as the slab heats; S6; 64 cells, the coarsest time step of the
paper's study, 312 steps) through sm_step with the paper's iteration
controls, independent and consistent closures, FP64 and FP32 sweeps, against
the oracle's run of the same steps: temperature and energy density at 2.5 ns
and the position of the wave front."""
import numpy as np
import pytest

import oracle as O
from oracle import lo as L
from paper_2504_21784_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_ORACLE = {}


def _start(cfg):
    n = cfg.n_cells
    T0 = np.full((n, 2), cfg.T0)
    scale = W.scale_field(cfg)
    cv = np.full((n, 2), cfg.cv)
    mu, omy, w = O.quadrature(1, cfg.n_polar)
    I0 = L.equilibrium_intensity(cfg, T0, mu)
    mom0 = O.moments(1, mu, omy, w, O.opacity(cfg.opacity_kind, 0.0, cfg.edges, T0, scale), I0)
    return T0, scale, cv, I0, mom0


def _oracle_run(cfg, method):
    if method not in _ORACLE:
        T, scale, cv, I, mom = _start(cfg)
        prm = L.StepParams(method=method)
        for _ in range(cfg.steps):
            T, E, F, I, mom, st = L.sm_step(cfg, scale, cv, T, I, mom, prm)
        _ORACLE[method] = (T, E)
    return _ORACLE[method]


def _front(cfg, T):
    """x at which the cell-mean temperature first drops below 500 eV"""
    hot = T.mean(axis=1) > 500.0
    k = int(np.argmin(hot)) if not hot.all() else cfg.nx
    return k * (cfg.extent[1] - cfg.extent[0]) / cfg.nx


@pytest.mark.parametrize("method", ["independent", "consistent"])
@pytest.mark.parametrize("precision", [64, 32])
def test_paper_marshak_wave_matches_oracle(gpu_lib, method, precision):
    import torch
    sm = gpu_lib
    cfg = W.marshak_paper()
    Tr, Er = _oracle_run(cfg, method)
    T0, scale, cv, I0, mom0 = _start(cfg)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    prob = sm.Problem.from_config(cfg, precision)
    T, E, F, mom = cu(T0), prob.new_nodal(), prob.new_flux(), cu(mom0)
    Ip = prob.pack(cu(W.in_precision(I0, precision)))
    mcode = sm.METHOD_CONSISTENT if method == "consistent" else sm.METHOD_INDEPENDENT
    outer = 0
    for _ in range(cfg.steps):
        In = prob.empty_intensity()
        st = prob.step(cu(scale), cu(cv), T, E, F, mom, Ip, In,
                       params=sm.step_params(method=mcode))
        assert st["converged"] == 1
        outer += st["outer_iters"]
        Ip = In
    Tg, Eg = T.cpu().numpy(), E.cpu().numpy()
    eT = float(np.abs(Tg - Tr).max() / np.abs(Tr).max())
    eE = float(np.abs(Eg - Er).max() / np.abs(Er).max())
    fg, fr = _front(cfg, Tg), _front(cfg, Tr)
    print(f"paper Marshak {method} fp{precision}: T {eT:.2e} E {eE:.2e}, front {fg:.5f} cm "
          f"(oracle {fr:.5f}), {outer} outer iterations in {cfg.steps} steps")
    assert eT < 1e-5 and eE < 1e-5
    assert fg == fr
