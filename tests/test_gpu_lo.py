"""GPU low-order solve and full step (Sec. 4 LDG system, Sec. 5 Newton with
nonlinear temperature elimination, Algorithm 1) through the C ABI, against the
FP64 oracle (oracle/lo.py) and against closed forms.

Tolerances.  The oracle solves each linearised system directly; the library
solves the Schur complement by conjugate gradients to a relative residual
pcg_rtol.  With pcg_rtol = 1e-14 and the small, well-conditioned meshes used
here (condition number of S below about 1e3 with dt = 0.01), the low-order
solution differs from the direct solve by at most ~1e-11 relative, measured
per field (T, E against their largest value; F against c times the largest
E, since F vanishes near equilibrium).  A full step with the FP32 sweep
inherits the sweep's 1e-6-level rounding through the closures: 1e-5.

The library has three forms of the conjugate gradients (FP64 with two grid
reductions per iteration, FP64 in the single-reduction form of Chronopoulos and
Gear, and mixed precision: FP32 inner solves refined by FP64 residual updates
to the same FP64 stopping test) and picks one by mesh size; the oracle
comparisons run all three, forced through the sm_debug_set_pcg_form test hook.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lo as L
from paper_2504_21784_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_LO = 1e-11      # FP64 low-order solve vs direct solve
TOL_STEP = {64: 1e-10, 32: 1e-5}


def _field(got, ref, scale=None):
    d = np.abs(np.asarray(got) - np.asarray(ref)).max()
    s = np.abs(ref if scale is None else scale).max()
    return float(d / max(s, 1e-300))


def _cfg(dim, nx, ny, G=3, kind=W.OPACITY_LARSEN, T_bdr=(1.0, 0.0, 0.3, 0.0), dt=0.01):
    edges = W.log_edges(G) if G > 1 else W.GRAY_EDGES.copy()
    return W.Config("lo", dim, nx, ny if dim == 2 else 1, (0.0, 1.0, 0.0, 1.0), edges,
                    4 if dim == 1 else 2, 0 if dim == 1 else 3, kind,
                    10.0 if kind == W.OPACITY_LARSEN else 0.0, T_bdr, a=1.0, c=1.0, dt=dt)


def _lo_inputs(cfg, seed):
    """Closures from one oracle sweep at a random temperature field, the
    previous-step moments of a random intensity, C_v and T*."""
    dim, nx, ny = cfg.dim, cfg.nx, cfg.ny
    m = L.make_mesh(dim, nx, ny, cfg.extent)
    nn = m.nn
    T = W.temperature_random(m.ncell, nn, seed=seed, lo=0.05, hi=1.0)
    scale = np.ones(m.ncell)
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    omx, omy, w = O.quadrature(dim, cfg.n_polar, cfg.n_azim)
    Ik = W.intensity_random(len(w), cfg.n_groups, m.ncell, nn, seed=seed + 1, scale=0.01)
    mom_k = O.moments(dim, omx, omy, w, sigma, Ik)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    I = O.sweep(dim, nx, ny, cfg.extent, omx, omy, sigma, 1.0 / (cfg.c * cfg.dt), q, Ik, infl)
    mom = O.moments(dim, omx, omy, w, sigma, I)
    clo = O.closures(dim, cfg.edges, cfg.c, sigma, T, mom)
    cv = np.full(T.shape, 0.3) * (1.0 + 0.5 * np.random.default_rng(seed + 2).random(T.shape))
    alpha = O.alpha(omx, w)
    jin2 = L.boundary_partial_currents(dim, omx, omy, w, infl.sum(axis=1))
    return m, clo, T, cv, mom_k, alpha, jin2


def _gpu_lo(sm, cfg, clo, Tstar, cv, mom_k, T0, E0, form="auto", **prm):
    import torch
    prob = sm.Problem.from_config(cfg, 64)
    prob.debug_set_pcg_form(form)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    T = cu(T0.copy())
    E = cu(E0.copy())
    st = prob.loworder_newton(cu(clo), cu(Tstar), cu(cv), cu(mom_k), T, E,
                              params=sm.step_params(**prm))
    return T.cpu().numpy(), E.cpu().numpy(), st["F"].cpu().numpy(), st, prob


LO_CASES = {
    "1d_40": (1, 40, 1),
    "1d_single": (1, 1, 1),
    "2d_7x5": (2, 7, 5),
    "2d_1x1": (2, 1, 1),
    "2d_13x3": (2, 13, 3),
}


# the forms of the conjugate gradients (textbook: two grid reductions per
# iteration; single: Chronopoulos-Gear, one; mixed: FP32 inner solves with FP64
# refinement), forced through the test hook
PCG_FORMS = ("textbook", "single", "mixed")


@pytest.mark.parametrize("form", PCG_FORMS)
@pytest.mark.parametrize("name", list(LO_CASES))
def test_loworder_newton_matches_oracle(gpu_lib, name, form):
    dim, nx, ny = LO_CASES[name]
    cfg = _cfg(dim, nx, ny)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=11 + nx)
    Estar = mom_k[..., 0] / cfg.c
    Fstar = mom_k[..., 1:1 + dim]
    ops = L.lo_operators(m, cfg.c, alpha)
    prm = L.LOParams(eps_inner=1e-13, max_inner=40, elim_rtol=1e-15, max_elim=80)
    Tr, Er, Fr, st_r = L.lo_newton(m, ops, cfg.c, cfg.a, cfg.dt, alpha, clo, T, cv, Estar, Fstar,
                                   jin2, T, Estar, prm)
    Tg, Eg, Fg, st_g, prob = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar, form=form,
                                     eps_inner=1e-13, max_inner=40, pcg_rtol=1e-15,
                                     elim_rtol=1e-15, max_elim=80)
    assert prob.debug_pcg_form() == form
    eT, eE = _field(Tg, Tr), _field(Eg, Er)
    eF = _field(Fg, Fr, scale=cfg.c * Er)
    print(f"{name} {form}: T {eT:.2e} E {eE:.2e} F {eF:.2e} newton {st_g['newton_iters_total']} "
          f"(oracle {st_r['newton']}) pcg max {st_g['pcg_iters_max']}")
    assert eT < TOL_LO and eE < TOL_LO and eF < TOL_LO
    assert st_g["pcg_capped"] == 0


def test_pcg_forms_agree_on_a_large_mesh(gpu_lib):
    """200x200 cells: the library's choice is the textbook form (4096 cells
    and up), a small mesh gets the single-reduction form, and the forced
    mixed-precision form gives the textbook form's solve to the accuracy of
    the linear solves, with the same Newton iterations."""
    cfg = _cfg(2, 200, 200)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=17)
    Estar = mom_k[..., 0] / cfg.c
    kw = dict(eps_inner=1e-13, max_inner=40, pcg_rtol=1e-14, elim_rtol=1e-15, max_elim=80)
    Ta, Ea, Fa, sa, pa = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar, form="mixed", **kw)
    Tb, Eb, Fb, sb, pb = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar, **kw)
    assert pa.debug_pcg_form() == "mixed" and pb.debug_pcg_form() == "textbook"
    eT, eE = _field(Tb, Ta), _field(Eb, Ea)
    eF = _field(Fb, Fa, scale=cfg.c * Ea)
    print(f"forms: T {eT:.2e} E {eE:.2e} F {eF:.2e} pcg {sa['pcg_iters_total']} / "
          f"{sb['pcg_iters_total']} newton {sa['newton_iters_total']} / {sb['newton_iters_total']}")
    assert eT < TOL_LO and eE < TOL_LO and eF < TOL_LO
    assert sa["newton_iters_total"] == sb["newton_iters_total"]
    small = _cfg(2, 7, 5)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(small, seed=18)
    *_, ps = _gpu_lo(gpu_lib, small, clo, T, cv, mom_k, T, mom_k[..., 0] / small.c)
    assert ps.debug_pcg_form() == "single"


def test_loworder_default_tolerances_match_oracle(gpu_lib):
    """With the paper's eps = 1e-3 both sides stop after the same Newton
    iteration and agree to the accuracy of the linear solves."""
    cfg = _cfg(2, 9, 8)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=4)
    Estar = mom_k[..., 0] / cfg.c
    ops = L.lo_operators(m, cfg.c, alpha)
    Tr, Er, Fr, st_r = L.lo_newton(m, ops, cfg.c, cfg.a, cfg.dt, alpha, clo, T, cv, Estar,
                                   mom_k[..., 1:3], jin2, T, Estar, L.LOParams())
    Tg, Eg, Fg, st_g, _ = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar)
    assert st_g["newton_iters_total"] == st_r["newton"]
    assert _field(Tg, Tr) < 1e-8 and _field(Eg, Er) < 1e-8


def test_loworder_is_deterministic(gpu_lib):
    cfg = _cfg(2, 11, 6)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=8)
    Estar = mom_k[..., 0] / cfg.c
    a = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar)
    b = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def _energy_residual(m, cfg, cv, Tstar, Estar, T, E, alpha, jin2):
    """sum m [(E - E*) + C_v (T - T*)] / dt + net boundary outflow, and its scale."""
    mass = m.mass()
    vol = mass * np.sum((E - Estar) / cfg.dt + cv * (T - Tstar) / cfg.dt)
    En = E.reshape(-1)
    out = 0.0
    for kind, n, wf, pairs in L.faces(m):
        if kind == "bdr":
            for nb, _ in pairs:
                out += wf * (cfg.c * alpha * En[nb] - jin2[n[2]])
    scale = mass * np.sum(np.abs(E - Estar) / cfg.dt + np.abs(cv * (T - Tstar)) / cfg.dt) + abs(out)
    return vol + out, scale


def test_loworder_conserves_energy(gpu_lib):
    cfg = _cfg(2, 24, 17)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=21)
    Estar = mom_k[..., 0] / cfg.c
    Tg, Eg, Fg, st, _ = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar, eps_inner=1e-14,
                                pcg_rtol=1e-14, elim_rtol=1e-15, max_elim=80)
    res, scale = _energy_residual(m, cfg, cv, T, Estar, Tg, Eg, alpha, jin2)
    assert abs(res) < 1e-11 * scale


def test_pcg_cap_is_reported_not_an_error(gpu_lib):
    cfg = _cfg(2, 16, 16)
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=2)
    Estar = mom_k[..., 0] / cfg.c
    *_, st, _ = _gpu_lo(gpu_lib, cfg, clo, T, cv, mom_k, T, Estar, max_pcg=1, max_inner=2)
    assert st["pcg_capped"] >= 1 and st["pcg_iters_max"] == 1


def test_loworder_rejects_bad_arguments(gpu_lib):
    sm = gpu_lib
    cfg = _cfg(2, 4, 4)
    prob = sm.Problem.from_config(cfg, 64)
    z = prob.new_nodal()
    clo = prob.new_closures()
    mom = prob.new_moments()
    with pytest.raises(sm.SMError, match="INVALID_ARG"):
        prob.loworder_newton(clo, z, z, mom, z.clone(), z.clone(),
                             params=sm.step_params(max_inner=0))
    with pytest.raises(sm.SMError, match="INVALID_ARG"):
        prob.loworder_newton(clo, z, z, mom, z.clone(), z.clone(),
                             params=sm.step_params(pcg_rtol=0.0))
    p0 = sm.Problem.from_config(_cfg(2, 4, 4, dt=0.0), 64)  # steady operator
    with pytest.raises(sm.SMError, match="dt > 0"):
        p0.loworder_newton(p0.new_closures(), z, z, p0.new_moments(), z.clone(), z.clone())


# --------------------------------------------------------------------------- full step
def _zero_d_answer(sig, cv, dt, a, c, T0):
    """Scalar backward Euler: (E - E*)/dt + c sig E = sig a c T^4,
    C_v (T - T*)/dt = c sig E - sig a c T^4, E* = a T0^4, by scalar Newton."""
    Estar = a * T0 ** 4
    T = T0
    for _ in range(200):
        E = (sig * a * c * T ** 4 + Estar / dt) / (1.0 / dt + c * sig)
        dEdT = sig * a * c * 4 * T ** 3 / (1.0 / dt + c * sig)
        f = cv * (T - T0) / dt - (c * sig * E - sig * a * c * T ** 4)
        df = cv / dt - (c * sig * dEdT - 4 * sig * a * c * T ** 3)
        T -= f / df
    E = (sig * a * c * T ** 4 + Estar / dt) / (1.0 / dt + c * sig)
    return T, E


@pytest.mark.parametrize("dim,precision", [(1, 64), (2, 64), (2, 32)])
def test_step_reproduces_infinite_medium(gpu_lib, dim, precision):
    """Uniform gray medium heated by boundary radiation at the answer's own
    radiation temperature: every node follows the scalar backward-Euler pair."""
    import torch
    sm = gpu_lib
    T0, s, cv0, dt, a, c = 0.2, 0.5, 0.3, 0.01, 1.0, 1.0
    sig = s / T0 ** 3
    Tans, Eans = _zero_d_answer(sig, cv0, dt, a, c, T0)
    Tb = (Eans / a) ** 0.25
    nx, ny = (6, 1) if dim == 1 else (5, 4)
    cfg = W.Config("zd", dim, nx, ny, (0.0, 1.0, 0.0, 1.0), W.GRAY_EDGES.copy(),
                   4 if dim == 1 else 2, 0 if dim == 1 else 2, W.OPACITY_POWER, 0.0,
                   (Tb, Tb, Tb if dim == 2 else 0.0, Tb if dim == 2 else 0.0), a=a, c=c, dt=dt)
    prob = sm.Problem.from_config(cfg, precision)
    ncell, nn = cfg.n_cells, cfg.n_nodes
    Tk = np.full((ncell, nn), T0)
    omx, omy, w = O.quadrature(dim, cfg.n_polar, cfg.n_azim)
    Ik = L.equilibrium_intensity(cfg, Tk, omx)
    sigma = O.opacity(0, 0.0, cfg.edges, Tk, np.full(ncell, s))
    mom_k = O.moments(dim, omx, omy, w, sigma, Ik)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    T = cu(Tk)
    E, F = prob.new_nodal(), prob.new_flux()
    mom = cu(mom_k)
    Ip = prob.pack(cu(Ik))
    In = prob.empty_intensity()
    st = prob.step(cu(np.full(ncell, s)), cu(np.full((ncell, nn), cv0)), T, E, F, mom, Ip, In,
                   params=sm.step_params(eps_outer=1e-14 if precision == 64 else 1e-7,
                                         max_outer=200, eps_inner=1e-14,
                                         max_inner=40, pcg_rtol=1e-15, elim_rtol=1e-15,
                                         max_elim=80))
    tol = 1e-11 if precision == 64 else 2e-6
    assert st["converged"] == 1
    assert np.max(np.abs(T.cpu().numpy() - Tans)) < tol * Tans
    assert np.max(np.abs(E.cpu().numpy() - Eans)) < tol * Eans
    assert np.max(np.abs(F.cpu().numpy())) < 10 * tol * c * Eans
    assert np.max(np.abs(mom.cpu().numpy()[..., 0] / c - Eans)) < 10 * tol * Eans


STEP_CASES = {
    "1d_mg": (1, 30, 1, 4, 64),
    "2d_mg_fp64": (2, 6, 5, 3, 64),
    "2d_mg_fp32": (2, 6, 5, 3, 32),
    "2d_gray_fp64": (2, 9, 4, 1, 64),
}


@pytest.mark.parametrize("form", PCG_FORMS)
@pytest.mark.parametrize("name", list(STEP_CASES))
def test_step_matches_oracle(gpu_lib, name, form):
    """A fixed number of outer iterations of Algorithm 1 on both sides."""
    import torch
    sm = gpu_lib
    dim, nx, ny, G, precision = STEP_CASES[name]
    kind = W.OPACITY_POWER if G == 1 else W.OPACITY_LARSEN
    cfg = _cfg(dim, nx, ny, G=G, kind=kind, T_bdr=(1.0, 0.2, 0.6, 0.0))
    prob = sm.Problem.from_config(cfg, precision)
    prob.debug_set_pcg_form(form)
    ncell, nn = cfg.n_cells, cfg.n_nodes
    rng = np.random.default_rng(5 + nx)
    Tk = W.temperature_random(ncell, nn, seed=3 + nx, lo=0.1, hi=0.8)
    scale = W.scale_field(cfg, seed=9) if dim == 2 else 1.0 + rng.random(ncell)
    cv = 0.3 + 0.2 * rng.random((ncell, nn))
    omx, omy, w = O.quadrature(dim, cfg.n_polar, cfg.n_azim)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Ik = W.intensity_random(cfg.n_dir, G, ncell, nn, seed=12, scale=0.05)
    Ik = W.in_precision(Ik, precision)  # what the sweep reads in its precision
    Ip = prob.pack(cu(Ik))
    sigma_k = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, Tk, scale)
    mom_k = O.moments(dim, omx, omy, w, sigma_k, Ik)
    n_outer = 3
    prm_o = L.StepParams(eps_outer=0.0, max_outer=n_outer,
                         lo=L.LOParams(eps_inner=1e-13, max_inner=40, elim_rtol=1e-15,
                                       max_elim=80))
    Tr, Er, Fr, Ir, momr, st_r = L.sm_step(cfg, scale, cv, Tk, Ik, mom_k, prm_o)
    T = cu(Tk)
    E, F = prob.new_nodal(), prob.new_flux()
    mom = cu(mom_k)
    In = prob.empty_intensity()
    st = prob.step(cu(scale), cu(cv), T, E, F, mom, Ip, In,
                   params=sm.step_params(eps_outer=0.0, max_outer=n_outer, eps_inner=1e-13,
                                         max_inner=40, pcg_rtol=1e-15, elim_rtol=1e-15,
                                         max_elim=80))
    assert st["outer_iters"] == st_r["outer"] == n_outer
    Tg, Eg, Fg = T.cpu().numpy(), E.cpu().numpy(), F.cpu().numpy()
    momg, Ig = mom.cpu().numpy(), prob.unpack(In).cpu().numpy()
    errs = {"T": _field(Tg, Tr), "E": _field(Eg, Er), "F": _field(Fg, Fr, scale=cfg.c * Er),
            "phi": _field(momg[..., 0], momr[..., 0]),
            "I": max(_field(Ig[d, g], Ir[d, g]) for d in range(cfg.n_dir) for g in range(G))}
    print(name, {k: f"{v:.2e}" for k, v in errs.items()})
    tol = TOL_STEP[precision]
    assert all(v < tol for v in errs.values()), errs


def test_step_default_params_converges(gpu_lib):
    """The paper's controls on a Marshak-wave-like 1D step: converged, the
    same outer count as the oracle, and agreement to the stopping tolerance."""
    import torch
    sm = gpu_lib
    cfg = W.marshak_1d().resized(nx=60)
    prob = sm.Problem.from_config(cfg, 64)
    ncell, nn = cfg.n_cells, cfg.n_nodes
    Tk = np.full((ncell, nn), cfg.T0)
    omx, omy, w = O.quadrature(1, cfg.n_polar, 0)
    Ik = L.equilibrium_intensity(cfg, Tk, omx)
    scale = np.ones(ncell)
    sigma_k = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, Tk, scale)
    mom_k = O.moments(1, omx, omy, w, sigma_k, Ik)
    cv = np.full((ncell, nn), cfg.cv)
    Tr, Er, Fr, Ir, momr, st_r = L.sm_step(cfg, scale, cv, Tk, Ik, mom_k, L.StepParams())
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    T = cu(Tk)
    E, F = prob.new_nodal(), prob.new_flux()
    mom = cu(mom_k)
    st = prob.step(cu(scale), cu(cv), T, E, F, mom, prob.pack(cu(Ik)), prob.empty_intensity())
    assert st["converged"] == 1 and st["outer_iters"] == st_r["outer"]
    assert _field(T.cpu().numpy(), Tr) < 1e-8
    assert _field(E.cpu().numpy(), Er) < 1e-8


def test_barrier_timeout_reports_status_and_recovers(gpu_lib):
    """The cooperative low-order kernel with one block withheld (a test hook:
    it leaves before its first grid barrier): every other block's bounded
    barrier wait runs out, the solve returns SM_ERR_TIMEOUT without any fault,
    and the next solve of the same problem equals one of a fresh problem."""
    sm = gpu_lib
    cfg = _cfg(2, 40, 36)   # several blocks of cells
    m, clo, T, cv, mom_k, alpha, jin2 = _lo_inputs(cfg, seed=31)
    Estar = mom_k[..., 0] / cfg.c
    ref = _gpu_lo(sm, cfg, clo, T, cv, mom_k, T, Estar)
    import torch
    prob = sm.Problem.from_config(cfg, 64)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prob.debug_wait_limit_ns(50_000_000)  # 50 ms
    prob.debug_withhold_lo_block(True)
    with pytest.raises(sm.SMError) as ei:
        prob.loworder_newton(cu(clo), cu(T), cu(cv), cu(mom_k), cu(T.copy()), cu(Estar.copy()))
    assert ei.value.code == 6  # SM_ERR_TIMEOUT
    prob.debug_withhold_lo_block(False)
    prob.debug_wait_limit_ns(2_000_000_000)
    Tg, Eg = cu(T.copy()), cu(Estar.copy())
    prob.loworder_newton(cu(clo), cu(T), cu(cv), cu(mom_k), Tg, Eg)
    assert np.array_equal(Tg.cpu().numpy(), ref[0]) and np.array_equal(Eg.cpu().numpy(), ref[1])
