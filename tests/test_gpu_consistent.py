"""GPU consistent SM method (Sec. 4, consistent): per-quadrant moments from
the sweep, the consistent low-order sources and the consistent step, against
the FP64 oracle (oracle/consistent.py) and against the property that defines
the method: a converged consistent step equals the converged high-order step
(sm_ho_step), while the independent step does not.

Tolerances as in test_gpu_lo.py: 1e-11 per field for FP64 (iterative
solves to 1e-13..1e-15 on both sides), 1e-5 for the FP32 sweep.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from oracle import consistent as OC
from oracle import lo as L
from paper_2504_21784_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cfg(nx=5, ny=4, G=3, npol=2, naz=2, T_bdr=(1.0, 0.3, 0.5, 0.0)):
    return W.Config("cons", 2, nx, ny, (0.0, 1.0, 0.0, 0.7), W.log_edges(G), npol, naz,
                    W.OPACITY_LARSEN, 10.0, T_bdr, a=1.0, c=1.0, dt=0.01)


def _field(a, b, scale=None):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b if scale is None else scale).max())


def _state(cfg, seed=4):
    rng = np.random.default_rng(seed)
    T = 0.1 + 0.8 * rng.random((cfg.n_cells, 4))
    scale = np.exp(0.5 * rng.standard_normal(cfg.n_cells))
    Ik = W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=seed + 1, scale=0.05)
    return T, scale, Ik


def test_quadrant_moments_match_oracle(gpu_lib):
    import torch
    sm = gpu_lib
    cfg = _cfg(7, 5, 4, 2, 4)
    T, scale, Ik = _state(cfg)
    prob = sm.Problem.from_config(cfg, 64)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    Ip = prob.pack(cu(Ik))
    Io = prob.empty_intensity()
    m0 = prob.new_moments()
    prob.sweep(cu(T), cu(sigma), Ip, Io, m0)
    prob.synchronize()
    qm = prob.new_quadrant_moments()
    prob.set_quadrant_moments(qm)
    m1 = prob.new_moments()
    prob.sweep(cu(T), cu(sigma), Ip, Io, m1)
    prob.synchronize()
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    I = O.sweep(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, sigma, 1.0 / (cfg.c * cfg.dt), q, Ik, infl)
    ref = OC.quadrant_moments(omx, omy, w, I)
    got = qm.cpu().numpy()
    for k in range(6):
        assert _field(got[..., k], ref[..., k], scale=ref[..., 0]) < 1e-11
    # registering the per-quadrant moments leaves the ordinary moments unchanged
    assert _field(m1.cpu().numpy(), m0.cpu().numpy(), scale=m0.cpu().numpy()[..., 0]) < 1e-13
    prob.set_quadrant_moments(None)


def _oracle_consistent_lo(cfg, T, scale, Ik, cv):
    """Closures, quadrant moments and the consistent low-order solution of
    the oracle for one sweep at T."""
    m = L.make_mesh(2, cfg.nx, cfg.ny, cfg.extent)
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    alpha = O.alpha(omx, w)
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    I = O.sweep(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, sigma, 1.0 / (cfg.c * cfg.dt), q, Ik, infl)
    mom = O.moments(2, omx, omy, w, sigma, I)
    clo = O.closures(2, cfg.edges, cfg.c, sigma, T, mom)
    momk = O.moments(2, omx, omy, w, sigma, Ik)
    R1, R0 = OC.consistent_sources(m, cfg.c, alpha, clo, omx, omy, w, I, infl.sum(axis=1))
    jin2 = L.boundary_partial_currents(2, omx, omy, w, infl.sum(axis=1))
    Estar = momk[..., 0] / cfg.c
    prm = L.LOParams(eps_inner=1e-13, max_inner=40, elim_rtol=1e-15, max_elim=80)
    Tr, Er, Fr, st = L.lo_newton(m, L.lo_operators(m, cfg.c, alpha), cfg.c, cfg.a, cfg.dt, alpha,
                                 clo, T, cv, Estar, momk[..., 1:3], jin2, T, Estar, prm,
                                 R1=R1, bnd=R0)
    return sigma, clo, momk, Tr, Er, Fr


def test_consistent_loworder_matches_oracle(gpu_lib):
    import torch
    sm = gpu_lib
    cfg = _cfg()
    T, scale, Ik = _state(cfg, seed=6)
    cv = np.full(T.shape, 0.3)
    sigma, clo, momk, Tr, Er, Fr = _oracle_consistent_lo(cfg, T, scale, Ik, cv)
    prob = sm.Problem.from_config(cfg, 64)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    qm = prob.new_quadrant_moments()
    prob.set_quadrant_moments(qm)
    Ip = prob.pack(cu(Ik))
    Io = prob.empty_intensity()
    clo_g = prob.new_closures()
    prob.sweep(cu(T), cu(sigma), Ip, Io, prob.new_moments(), clo_g)
    prob.synchronize()
    Tg, Eg = cu(T), cu(momk[..., 0] / cfg.c)
    st = prob.loworder_newton(clo_g, cu(T), cu(cv), cu(momk), Tg, Eg,
                              params=sm.step_params(eps_inner=1e-13, max_inner=40, pcg_rtol=1e-15,
                                                    elim_rtol=1e-15, max_elim=80,
                                                    method=sm.METHOD_CONSISTENT))
    eT, eE = _field(Tg.cpu().numpy(), Tr), _field(Eg.cpu().numpy(), Er)
    eF = _field(st["F"].cpu().numpy(), Fr, scale=cfg.c * Er)
    print(f"consistent LO: T {eT:.2e} E {eE:.2e} F {eF:.2e}")
    assert eT < 1e-11 and eE < 1e-11 and eF < 1e-11


def _step_inputs(cfg, seed=4):
    rng = np.random.default_rng(seed)
    T0 = 0.1 + 0.8 * rng.random((cfg.n_cells, 4))
    scale = np.exp(0.5 * rng.standard_normal(cfg.n_cells))
    cv = np.full((cfg.n_cells, 4), 0.3)
    pb = OA.Problem(cfg.nx, cfg.ny, cfg.extent, cfg.edges, cfg.n_polar, cfg.n_azim,
                    cfg.opacity_kind, cfg.opacity_alpha, cfg.T_bdr, dt=cfg.dt)
    B4, _ = OA.planck_parts(pb, T0)
    I0 = np.broadcast_to(B4[None], (cfg.n_dir,) + B4.shape).copy()
    return T0, scale, cv, I0, pb


def _gpu_step(sm, cfg, precision, T0, scale, cv, I0, method, tight=True):
    import torch
    prob = sm.Problem.from_config(cfg, precision)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    I0r = W.in_precision(I0, precision)
    Ip = prob.pack(cu(I0r))
    sigma0 = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T0, scale)
    mom = cu(O.moments(2, omx, omy, w, sigma0, I0r))
    T, E, F = cu(T0), prob.new_nodal(), prob.new_flux()
    In = prob.empty_intensity()
    # the FP32 sweep's outer iteration settles at its rounding floor (relative
    # changes ~1e-8, possibly cycling between neighbouring FP32 states), so its
    # stopping tolerance sits above that floor
    kw = dict(eps_outer=1e-14 if precision == 64 else 1e-7, max_outer=400, eps_inner=1e-14,
              max_inner=40, pcg_rtol=1e-15, elim_rtol=1e-15, max_elim=80) if tight else {}
    st = prob.step(cu(scale), cu(cv), T, E, F, mom, Ip, In,
                   params=sm.step_params(method=method, **kw))
    return prob, T.cpu().numpy(), E.cpu().numpy(), mom.cpu().numpy(), In, st, I0r


@pytest.mark.parametrize("precision", [64, 32])
def test_consistent_step_matches_oracle(gpu_lib, precision):
    sm = gpu_lib
    cfg = _cfg(4, 3, 3)
    T0, scale, cv, I0, pb = _step_inputs(cfg)
    prob, Tg, Eg, momg, In, st, I0r = _gpu_step(sm, cfg, precision, T0, scale, cv, I0,
                                                sm.METHOD_CONSISTENT)
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    mom0 = O.moments(2, omx, omy, w, O.opacity(1, 10.0, cfg.edges, T0, scale), I0r)
    prm = L.StepParams(eps_outer=1e-14, max_outer=400, method="consistent",
                       lo=L.LOParams(eps_inner=1e-14, max_inner=40, elim_rtol=1e-15, max_elim=80))
    Tr, Er, Fr, Ir, momr, str_ = L.sm_step(cfg, scale, cv, T0, I0r, mom0, prm)
    tol = 1e-11 if precision == 64 else 1e-5
    eT, eE = _field(Tg, Tr), _field(Eg, Er)
    print(f"consistent step fp{precision}: T {eT:.2e} E {eE:.2e} outer {st['outer_iters']} "
          f"(oracle {str_['outer']})")
    assert st["converged"] == 1
    assert eT < tol and eE < tol


def test_consistent_step_equals_converged_high_order_step(gpu_lib):
    """The defining property, on the GPU alone at a larger size: 24x20 cells,
    6 groups, 32 directions."""
    import torch
    sm = gpu_lib
    cfg = _cfg(24, 20, 6, 2, 4)
    T0, scale, cv, I0, pb = _step_inputs(cfg, seed=9)
    res = {}
    for name, method in (("consistent", sm.METHOD_CONSISTENT), ("independent", sm.METHOD_INDEPENDENT)):
        prob, Tg, Eg, momg, In, st, I0r = _gpu_step(sm, cfg, 64, T0, scale, cv, I0, method)
        res[name] = (Tg, Eg, momg, st)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    prob = sm.Problem.from_config(cfg, 64)
    Th = cu(T0)
    Ih = prob.empty_intensity()
    prob.ho_step(cu(scale), cu(cv), Th, prob.pack(cu(I0)), Ih, 1e-14, 5000)
    Th = Th.cpu().numpy()
    eTc = _field(res["consistent"][0], Th)
    eEc = _field(res["consistent"][1], res["consistent"][2][..., 0] / cfg.c)
    eTi = _field(res["independent"][0], Th)
    print(f"consistent vs HO: T {eTc:.2e}, E_LO vs E_HO {eEc:.2e}; independent vs HO: T {eTi:.2e}")
    assert eTc < 1e-10 and eEc < 1e-10
    assert eTi > 1e-5


# --------------------------------------------------------------------------- 1D slab
def _cfg1d(nx=9, G=3, npol=4, T_bdr=(1.0, 0.3, 0.0, 0.0)):
    return W.Config("cons1d", 1, nx, 1, (0.0, 1.0, 0.0, 1.0), W.log_edges(G), npol, 0,
                    W.OPACITY_LARSEN, 10.0, T_bdr, a=1.0, c=1.0, dt=0.01)


def _state1d(cfg, seed=4):
    rng = np.random.default_rng(seed)
    T = 0.1 + 0.8 * rng.random((cfg.n_cells, 2))
    scale = np.exp(0.5 * rng.standard_normal(cfg.n_cells))
    Ik = W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, 2, seed=seed + 1, scale=0.05)
    return T, scale, Ik


def test_half_moments_1d_match_oracle(gpu_lib):
    import torch
    sm = gpu_lib
    cfg = _cfg1d(13, 5, 6)
    T, scale, Ik = _state1d(cfg)
    prob = sm.Problem.from_config(cfg, 64)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    qm = prob.new_quadrant_moments()
    prob.set_quadrant_moments(qm)
    Io = prob.empty_intensity()
    prob.sweep(cu(T), cu(sigma), prob.pack(cu(Ik)), Io, prob.new_moments())
    prob.synchronize()
    mu, omy, w = O.quadrature(1, cfg.n_polar)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    I = O.sweep(1, cfg.nx, 1, cfg.extent, mu, omy, sigma, 1.0 / (cfg.c * cfg.dt), q, Ik, infl)
    ref = OC.half_moments_1d(mu, w, I)
    got = qm.cpu().numpy()
    for k in range(6):
        assert _field(got[..., k], ref[..., k], scale=ref[..., 0]) < 1e-11
    prob.set_quadrant_moments(None)


def _oracle_consistent_lo_1d(cfg, T, scale, Ik, cv):
    m = L.make_mesh(1, cfg.nx, 1, cfg.extent)
    mu, omy, w = O.quadrature(1, cfg.n_polar)
    alpha = O.alpha(mu, w)
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    I = O.sweep(1, cfg.nx, 1, cfg.extent, mu, omy, sigma, 1.0 / (cfg.c * cfg.dt), q, Ik, infl)
    mom = O.moments(1, mu, omy, w, sigma, I)
    clo = O.closures(1, cfg.edges, cfg.c, sigma, T, mom)
    momk = O.moments(1, mu, omy, w, sigma, Ik)
    R1, R0 = OC.consistent_sources(m, cfg.c, alpha, clo, mu, omy, w, I, infl.sum(axis=1))
    jin2 = L.boundary_partial_currents(1, mu, omy, w, infl.sum(axis=1))
    Estar = momk[..., 0] / cfg.c
    prm = L.LOParams(eps_inner=1e-13, max_inner=40, elim_rtol=1e-15, max_elim=80)
    Tr, Er, Fr, st = L.lo_newton(m, L.lo_operators(m, cfg.c, alpha), cfg.c, cfg.a, cfg.dt, alpha,
                                 clo, T, cv, Estar, momk[..., 1:2], jin2, T, Estar, prm,
                                 R1=R1, bnd=R0)
    return sigma, momk, Tr, Er, Fr


def test_consistent_loworder_matches_oracle_1d(gpu_lib):
    import torch
    sm = gpu_lib
    cfg = _cfg1d()
    T, scale, Ik = _state1d(cfg, seed=6)
    cv = np.full(T.shape, 0.3)
    sigma, momk, Tr, Er, Fr = _oracle_consistent_lo_1d(cfg, T, scale, Ik, cv)
    prob = sm.Problem.from_config(cfg, 64)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    qm = prob.new_quadrant_moments()
    prob.set_quadrant_moments(qm)
    clo_g = prob.new_closures()
    prob.sweep(cu(T), cu(sigma), prob.pack(cu(Ik)), prob.empty_intensity(), prob.new_moments(),
               clo_g)
    prob.synchronize()
    Tg, Eg = cu(T), cu(momk[..., 0] / cfg.c)
    st = prob.loworder_newton(clo_g, cu(T), cu(cv), cu(momk), Tg, Eg,
                              params=sm.step_params(eps_inner=1e-13, max_inner=40, pcg_rtol=1e-15,
                                                    elim_rtol=1e-15, max_elim=80,
                                                    method=sm.METHOD_CONSISTENT))
    eT, eE = _field(Tg.cpu().numpy(), Tr), _field(Eg.cpu().numpy(), Er)
    eF = _field(st["F"].cpu().numpy(), Fr, scale=cfg.c * Er)
    print(f"consistent LO 1D: T {eT:.2e} E {eE:.2e} F {eF:.2e}")
    assert eT < 1e-11 and eE < 1e-11 and eF < 1e-11


@pytest.mark.parametrize("precision", [64, 32])
def test_marshak_consistent_steps_match_oracle(gpu_lib, precision):
    """The 1D Marshak wave (200 cells, S8) over its ten steps with the
    consistent method, converged tightly on both sides."""
    import torch
    sm = gpu_lib
    cfg = W.marshak_1d()
    n = cfg.n_cells
    T0 = np.full((n, 2), cfg.T0)
    scale = W.scale_field(cfg)
    cv = np.full((n, 2), cfg.cv)
    mu, omy, w = O.quadrature(1, cfg.n_polar)
    I0 = L.equilibrium_intensity(cfg, T0, mu)
    mom0 = O.moments(1, mu, omy, w, O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges,
                                               T0, scale), I0)
    prm = L.StepParams(eps_outer=1e-13, max_outer=400, method="consistent",
                       lo=L.LOParams(eps_inner=1e-14, max_inner=60, elim_rtol=1e-15, max_elim=100))
    Tr, Ir, momr = T0, I0, mom0
    for _ in range(cfg.steps):
        Tr, Er, Fr, Ir, momr, _st = L.sm_step(cfg, scale, cv, Tr, Ir, momr, prm)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    prob = sm.Problem.from_config(cfg, precision)
    T, E, F, mom = cu(T0), prob.new_nodal(), prob.new_flux(), cu(mom0)
    Ip = prob.pack(cu(W.in_precision(I0, precision)))
    outer = []
    for _ in range(cfg.steps):
        In = prob.empty_intensity()
        st = prob.step(cu(scale), cu(cv), T, E, F, mom, Ip, In,
                       params=sm.step_params(eps_outer=1e-13 if precision == 64 else 1e-6,
                                             max_outer=400, eps_inner=1e-14, max_inner=60,
                                             pcg_rtol=1e-15, elim_rtol=1e-15, max_elim=100,
                                             method=sm.METHOD_CONSISTENT))
        outer.append((st["outer_iters"], st["converged"], f"{st['last_change']:.1e}"))
        Ip = In
    eT, eE = _field(T.cpu().numpy(), Tr), _field(E.cpu().numpy(), Er)
    print(f"marshak consistent fp{precision}: T {eT:.2e} E {eE:.2e}, outer {outer}")
    tol = 1e-11 if precision == 64 else 1e-5
    assert all(o[1] == 1 for o in outer)
    assert eT < tol and eE < tol
