"""Parity at the full workload sizes, in the launch configuration the
benchmark times (autotuned tiling), against the FP64 oracle element by
element.  The oracle sweeps one direction (all its groups) at a time and sums
the moments direction by direction (they are linear in the intensity), so the
host never holds more than one direction's intensity; the GPU keeps its whole
unpacked result on the device and hands over one direction at a time.

* 2D multigroup, 256x256 cells, 128 directions, 64 groups: FP32 and FP64
  sweeps (every intensity, moment and closure) and the opacity kernel;
* 2D gray two-material channel, 128x128 cells, 128 directions: the same;
* batched: the 64 uneven problems in one persistent launch (FP32), every
  member against the oracle;
* time steps of Algorithm 1: the 1D Marshak wave (200 cells, S8) over its ten
  steps against the oracle's steps (the 2D steps and the adjoint workload's
  gradient are in test_gpu_steps_fullsize.py);
* a sweep on four times the benchmark mesh, sampled.

The previous intensity is a seeded separable field, exactly representable in
FP32, so both sweep precisions read the same input and one oracle pass serves
both.  Tolerances as in test_gpu_parity.py: 1e-11 (FP64), 1e-5 (FP32), per
field.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W

from _cases import cell_elem_err, elem_bound, parity_errors

pytestmark = pytest.mark.gpu

TOL = {64: 1e-11, 32: 1e-5}


def _cu(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _canonical_on_device(cfg, gen):
    """The whole previous intensity [d][g][cell][node] on the device, filled one
    direction at a time from the host generator."""
    import torch
    canon = torch.empty((cfg.n_dir, cfg.n_groups, cfg.n_cells, cfg.n_nodes),
                        dtype=torch.float64, device="cuda")
    for d in range(cfg.n_dir):
        canon[d].copy_(torch.from_numpy(gen.direction(d)))
    return canon


def _oracle_by_direction(cfg, T, sigma, gen, on_direction):
    """The oracle sweep of every (direction, group), one direction at a time;
    on_direction(d, I_d) sees each direction's [g][cell][node] intensity.
    Returns the oracle's moments and closures."""
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    inv_cdt = 1.0 / (cfg.c * cfg.dt)
    G = cfg.n_groups
    mom = np.zeros((cfg.n_cells, 4, 9))
    for d in range(cfg.n_dir):
        I_d = O.sweep_pairs(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, sigma, inv_cdt, q,
                            gen.direction(d), infl, [(d, g) for g in range(G)])
        mom += O.moments(2, omx[d:d + 1], omy[d:d + 1], w[d:d + 1], sigma, I_d[None])
        on_direction(d, I_d)
    clo = O.closures(2, cfg.edges, cfg.c, sigma, T, mom)
    return mom, clo


class _IntensityErrors:
    """Largest per-(direction, group) field error of each GPU result (keyed
    by sweep precision), and the largest element-wise error against its bound
    (_cases.elem_bound), scaled by the precision's bar."""

    def __init__(self, runs, cfg):
        self.runs = runs                      # {precision: unpacked device intensity}
        self.cfg = cfg
        self.err = {k: 0.0 for k in runs}
        self.elem = {k: 0.0 for k in runs}

    def __call__(self, d, I_d):
        scale = np.maximum(np.abs(I_d).max(axis=(1, 2)), 1e-300)
        for k, Iu in self.runs.items():
            got = Iu[d].cpu().numpy()
            diff = np.abs(got - I_d).max(axis=(1, 2))
            self.err[k] = max(self.err[k], float((diff / scale).max()))
            r, a = elem_bound(self.cfg, k, TOL[k])
            self.elem[k] = max(self.elem[k], TOL[k] * cell_elem_err(got, I_d, r, a))


def _gpu_sweep(sm, cfg, precision, T, sigma, canon, scale=None):
    """One sweep in the benchmark's launch configuration: autotuned tiling,
    previous intensity read, moments and closures fused."""
    prob = sm.Problem.from_config(cfg, precision)
    Td, Sd = _cu(T), _cu(sigma)
    sig_g = prob.opacity(Td, _cu(scale)).cpu().numpy() if scale is not None else None
    Ip = prob.pack(canon)
    Io = prob.empty_intensity()
    prob.autotune(Td, Sd, Ip, Io, reps=1)
    mom, clo = prob.new_moments(), prob.new_closures()
    prob.sweep(Td, Sd, Ip, Io, mom, clo)
    prob.synchronize()
    tiling = {k: prob.info[k] for k in ("strip_width", "prefetch_rows", "groups_per_warp",
                                        "n_tasks")}
    del Ip
    Iu = prob.unpack(Io)
    del Io
    out = (Iu, mom.cpu().numpy(), clo.cpu().numpy(), sig_g, tiling)
    prob.close()
    return out


def _full_sweep_parity(sm, cfg, seed):
    import torch
    T = W.temperature_wave(cfg)
    scale = W.scale_field(cfg)
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    gen = W.SeparableIntensity(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=seed)
    canon = _canonical_on_device(cfg, gen)
    runs, rest = {}, {}
    for prec in (32, 64):
        Iu, mg, cg, sig_g, tiling = _gpu_sweep(sm, cfg, prec, T, sigma, canon, scale)
        runs[prec] = Iu
        rest[prec] = (mg, cg, sig_g, tiling)
    del canon
    torch.cuda.empty_cache()
    ierr = _IntensityErrors(runs, cfg)
    mo, co = _oracle_by_direction(cfg, T, sigma, gen, ierr)
    for prec in (32, 64):
        mg, cg, sig_g, tiling = rest[prec]
        e = parity_errors(cfg, (None, mg, cg), (None, mo, co))
        e["I"] = ierr.err[prec]
        e["I_elem"] = ierr.elem[prec]
        e["opacity"] = float(np.max(np.abs(sig_g - sigma) / sigma))
        print(f"[{cfg.name} fp{prec} {tiling}] " +
              "  ".join(f"{k} {v:.2e}" for k, v in e.items()))
        assert e.pop("opacity") < 1e-13
        bad = {k: v for k, v in e.items() if not v <= TOL[prec]}
        assert not bad, f"fp{prec} parity above {TOL[prec]}: {bad}"
    del runs
    torch.cuda.empty_cache()


def test_multigroup_full_size_parity(gpu_lib):
    """256x256 cells x 128 directions x 64 groups (5.4e8 updates)."""
    _full_sweep_parity(gpu_lib, W.multigroup_2d(), seed=31)


def test_gray_channel_full_size_parity(gpu_lib):
    """128x128 cells x 128 directions, walls 1e4 times thicker than the channel."""
    _full_sweep_parity(gpu_lib, W.gray_channel_2d(), seed=32)


def test_batched_full_size_parity(gpu_lib):
    """The 64 uneven problems (32^2..256^2 cells, 32..128 directions, 8..32
    groups) in one persistent launch with the autotuned batch tiling, FP32;
    every member against the oracle."""
    import torch
    sm = gpu_lib
    members = W.batched_2d()
    cfgs = [m.cfg for m in members]
    b = sm.Batch(cfgs, 32)
    T, S, Ip, Io, M, C, inputs = [], [], [], [], [], [], []
    for i, (mem, h) in enumerate(zip(members, b.members)):
        Tn = W.temperature_wave(mem.cfg)
        sig = O.opacity(mem.cfg.opacity_kind, mem.cfg.opacity_alpha, mem.cfg.edges, Tn, mem.scale)
        gen = W.SeparableIntensity(mem.cfg.n_dir, mem.cfg.n_groups, mem.cfg.n_cells, 4,
                                   seed=200 + i)
        canon = _canonical_on_device(mem.cfg, gen)
        Ip.append(h.pack(canon))
        del canon
        T.append(_cu(Tn))
        S.append(_cu(sig))
        Io.append(h.empty_intensity())
        M.append(h.new_moments())
        C.append(h.new_closures())
        inputs.append((Tn, sig, gen))
    torch.cuda.empty_cache()
    b.autotune(T, S, Ip, Io, reps=1)
    b.sweep(T, S, Ip, Io, M, C)
    b.synchronize()
    info = b.info()
    worst = {}
    for i, (cfg, h) in enumerate(zip(cfgs, b.members)):
        Tn, sig, gen = inputs[i]
        ierr = _IntensityErrors({32: h.unpack(Io[i])}, cfg)
        mo, co = _oracle_by_direction(cfg, Tn, sig, gen, ierr)
        e = parity_errors(cfg, (None, M[i].cpu().numpy(), C[i].cpu().numpy()), (None, mo, co))
        e["I"] = ierr.err[32]
        e["I_elem"] = ierr.elem[32]
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
        bad = {k: v for k, v in e.items() if not v <= TOL[32]}
        assert not bad, f"member {i} ({cfg.name}) parity above {TOL[32]}: {bad}"
        del ierr
        torch.cuda.empty_cache()
    print(f"[batched x{len(cfgs)} strip {info['strip_width']} prefetch {info['prefetch_rows']}] "
          + "  ".join(f"{k} {v:.2e}" for k, v in worst.items()))
    b.close()


def _gpu_steps(sm, cfg, precision, T0, I0, mom0, scale, cv, nsteps, params):
    """nsteps time steps of Algorithm 1 through sm_step; returns T, E and the
    per-step statistics."""
    import torch
    prob = sm.Problem.from_config(cfg, precision)
    T, E, F = _cu(T0), prob.new_nodal(), prob.new_flux()
    mom = _cu(mom0)
    Ip = prob.pack(_cu(W.in_precision(I0, precision)))
    stats = []
    for _ in range(nsteps):
        In = prob.empty_intensity()
        stats.append(prob.step(_cu(scale), _cu(cv), T, E, F, mom, Ip, In,
                               params=sm.step_params(**params)))
        Ip = In
    out = T.cpu().numpy(), E.cpu().numpy(), stats
    prob.close()
    del torch
    return out


def _oracle_steps(cfg, T0, I0, mom0, scale, cv, nsteps, prm):
    from oracle import lo as L
    T, I, mom = T0, I0, mom0
    stats = []
    for _ in range(nsteps):
        T, E, F, I, mom, st = L.sm_step(cfg, scale, cv, T, I, mom, prm)
        stats.append(st)
    return T, E, stats


def _equilibrium_start(cfg):
    from oracle import lo as L
    n, nn = cfg.n_cells, cfg.n_nodes
    T0 = np.full((n, nn), cfg.T0)
    scale = W.scale_field(cfg)
    cv = np.full((n, nn), cfg.cv)
    omx, omy, w = O.quadrature(cfg.dim, cfg.n_polar, cfg.n_azim)
    I0 = L.equilibrium_intensity(cfg, T0, omx)
    sig = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T0, scale)
    return T0, I0, O.moments(cfg.dim, omx, omy, w, sig, I0), scale, cv


@pytest.mark.parametrize("precision", [64, 32])
def test_marshak_ten_steps_match_oracle(gpu_lib, precision):
    """The 1D Marshak-type wave, 200 cells, S8, ten backward-Euler steps from
    T = 0.01 with the inflow at T = 1, every step converged tightly on both
    sides: the temperature and energy after each of the ten steps."""
    from oracle import lo as L
    cfg = W.marshak_1d()
    T0, I0, mom0, scale, cv = _equilibrium_start(cfg)
    tight = dict(eps_outer=1e-13 if precision == 64 else 1e-7, max_outer=400, eps_inner=1e-14,
                 max_inner=60, pcg_rtol=1e-15, elim_rtol=1e-15, max_elim=100)
    prm = L.StepParams(eps_outer=1e-13, max_outer=400,
                       lo=L.LOParams(eps_inner=1e-14, max_inner=60, elim_rtol=1e-15, max_elim=100))
    Tr, Er, str_ = _oracle_steps(cfg, T0, I0, mom0, scale, cv, cfg.steps, prm)
    Tg, Eg, stg = _gpu_steps(gpu_lib, cfg, precision, T0, I0, mom0, scale, cv, cfg.steps, tight)
    eT = float(np.abs(Tg - Tr).max() / np.abs(Tr).max())
    eE = float(np.abs(Eg - Er).max() / np.abs(Er).max())
    front = float(np.mean(Tr > 0.5))
    print(f"marshak fp{precision}: T {eT:.2e} E {eE:.2e}; hot fraction {front:.2f}; outer "
          f"{[s['outer_iters'] for s in stg]} (oracle {[s['outer'] for s in str_]})")
    assert all(s["converged"] == 1 for s in stg)
    tol = TOL[precision]
    assert eT < tol and eE < tol


def test_large_mesh_sampled_parity(gpu_lib):
    """Four times the benchmark mesh, 512x512 cells x 128 directions x 64
    groups (2.1e9 updates, 34 GB per FP32 intensity copy) in the autotuned
    launch configuration: the intensity of one direction per quadrant, all its
    groups, element by element against the oracle's sweeps of those pairs."""
    import torch
    sm = gpu_lib
    torch.cuda.empty_cache()
    cfg = W.multigroup_2d().resized(512)
    T = W.temperature_wave(cfg)
    scale = W.scale_field(cfg)
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    gen = W.SeparableIntensity(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=33)
    canon = _canonical_on_device(cfg, gen)
    prob = sm.Problem.from_config(cfg, 32)
    Td, Sd = _cu(T), _cu(sigma)
    Ip = prob.pack(canon)
    del canon
    torch.cuda.empty_cache()
    Io = prob.empty_intensity()
    prob.autotune(Td, Sd, Ip, Io, reps=1)
    mom = prob.new_moments()
    prob.sweep(Td, Sd, Ip, Io, mom)
    prob.synchronize()
    del Ip
    torch.cuda.empty_cache()
    Iu = prob.unpack(Io)
    del Io
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    nq = cfg.n_dir // 4
    worst = 0.0
    for d in (0, nq + 5, 2 * nq + 17, 4 * nq - 1):   # one direction per quadrant
        Ir = O.sweep_pairs(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, sigma, 1.0 / (cfg.c * cfg.dt),
                           q, gen.direction(d), infl, [(d, g) for g in range(cfg.n_groups)])
        Ig = Iu[d].cpu().numpy()
        e = np.abs(Ig - Ir).max(axis=(1, 2)) / np.maximum(np.abs(Ir).max(axis=(1, 2)), 1e-300)
        worst = max(worst, float(e.max()))
    phi = mom[..., 0]
    print(f"[{cfg.nx}x{cfg.ny}x{cfg.n_dir}x{cfg.n_groups} fp32 strip {prob.info['strip_width']}] "
          f"sampled I {worst:.2e}, "
          f"phi finite and positive: {bool(torch.isfinite(phi).all() and (phi > 0).all())}")
    assert worst < TOL[32]
    assert bool(torch.isfinite(phi).all()) and bool((phi > 0).all())
    del Iu
    prob.close()
    torch.cuda.empty_cache()
