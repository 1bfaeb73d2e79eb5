"""Time steps at the full configuration sizes against the oracle, and the
adjoint workload's gradient against central differences on a fixed cell set.

* 2D gray channel (128x128 cells, 128 directions): all twenty steps of
  Algorithm 1 from the equilibrium start, FP64 and FP32 sweeps;
* 2D multigroup (256x256 cells, 128 directions, 64 groups): one step from the
  equilibrium start, FP64 and FP32 sweeps (the oracle sweeps one direction at a
  time: the previous intensity B_g(T0)/4pi is the same for every direction);
* both: also the FP32 sweeps with FP64 defect correction (sm_step_params.refine,
  FP64 state), held to the FP64 bar;
* adjoint workload (128x128 cells, 64 directions, 16 groups, 20 steps, warm
  start): dJ/ds_K against central differences of the GPU forward on 32 cells
  drawn (seed 21784) from the four cell columns next to the right edge, a set
  fixed before the gradient is computed.

Parity mode (Algorithm 1, Eq. relative_tol): both sides keep the paper's
epsilon = 1e-3 for the outer and Newton iterations, and so take the same
iteration counts (asserted for the FP64 path), while every inner solve runs to
round-off: the oracle solves each linearised system directly and the library
runs conjugate gradients to a relative residual of 1e-15; both eliminate the
temperature to 1e-15.  The two sides then follow the same iterates up to
rounding.  Bars: 1e-11 (FP64 sweep) and 1e-5 (FP32 sweep) relative per field,
the error of every node divided by the field's largest magnitude (T is also
compared node by node).

The oracle's runs take minutes; they start in background workers when the
session starts (conftest.py, _oracle_jobs.py), and this file is collected
after the other GPU tests so that they overlap.
"""
import numpy as np
import pytest

import _oracle_jobs as J
from paper_2504_21784_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {64: 1e-11, 32: 1e-5}

#: the library's side of parity mode (see the module docstring)
PARITY_GPU = dict(eps_outer=J.PARITY_OUTER["eps_outer"], max_outer=J.PARITY_OUTER["max_outer"],
                  eps_inner=J.PARITY_LO["eps_inner"], max_inner=J.PARITY_LO["max_inner"],
                  elim_rtol=J.PARITY_LO["elim_rtol"], max_elim=J.PARITY_LO["max_elim"],
                  pcg_rtol=1e-15, max_pcg=20000)


def _cu(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gpu_steps(sm, cfg, precision, nsteps, state, refine=0):
    """nsteps steps of Algorithm 1 through sm_step from the equilibrium start;
    per step T, E, phi and the statistics (refine = 1: FP64 state, FP32
    correction sweeps)."""
    import torch
    T0, I_dir, mom0, scale, cv = state
    prob = sm.Problem.from_config(cfg, 64 if refine else precision)
    canon = _cu(I_dir)[None].expand(cfg.n_dir, -1, -1, -1).contiguous()
    Ip = prob.pack(canon)
    del canon
    torch.cuda.empty_cache()
    T, E, F, mom = _cu(T0), prob.new_nodal(), prob.new_flux(), _cu(mom0)
    sc, cvd = _cu(scale), _cu(cv)
    prm = sm.step_params(refine=refine, **PARITY_GPU)
    out = []
    for _ in range(nsteps):
        In = prob.empty_intensity()
        st = prob.step(sc, cvd, T, E, F, mom, Ip, In, params=prm)
        out.append({"T": T.cpu().numpy(), "E": E.cpu().numpy(),
                    "phi": mom[..., 0].cpu().numpy(), "stats": st})
        del Ip
        Ip = In
    del Ip
    prob.close()
    torch.cuda.empty_cache()
    return out


def _field(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def _compare(label, gpu, ref, precision):
    e = {"T": _field(gpu["T"], ref["T"]), "E": _field(gpu["E"], ref["E"]),
         "phi": _field(gpu["phi"], ref["phi"])}
    t_node = float(np.max(np.abs(gpu["T"] - ref["T"]) / ref["T"]))
    if precision == 64:
        e["T_node"] = t_node   # FP32: printed only (cold nodes carry the sweep's roundoff)
    st = gpu["stats"]
    same = (st["outer_iters"] == ref["outer"] and
            st["newton_iters_total"] == sum(ref["newton"]))
    extra = "" if "T_node" in e else f"  T_node {t_node:.2e} (printed only)"
    print(f"[{label} fp{precision}] " + "  ".join(f"{k} {v:.2e}" for k, v in e.items()) +
          f"{extra}  outer {st['outer_iters']} newton {st['newton_iters_total']} pcg max "
          f"{st['pcg_iters_max']} capped {st['pcg_capped']} (oracle outer {ref['outer']} "
          f"newton {sum(ref['newton'])})")
    return e, same


def test_adjoint_full_size_matches_central_differences_fixed_cells(gpu_lib):
    """dJ/ds_K of the warm-start adjoint workload (T0 = 0.3, 20 steps,
    checkpoints every sqrt(20) steps) against central differences
    (h = 1e-4 s_K) of the GPU forward, each forward solve converged to a
    relative change of 1e-13, on 32 cells drawn with seed 21784 from the
    columns within four cells of the right edge -- the cells the right-edge
    leakage depends on most, chosen before any gradient is known."""
    import torch
    from paper_2504_21784_gb300 import adjoint as A
    sm = gpu_lib
    cfg = W.adjoint_2d_warm()
    band = np.array([iy * cfg.nx + ix for iy in range(cfg.ny)
                     for ix in range(cfg.nx - 4, cfg.nx)])
    cells = np.random.default_rng(21784).choice(band, 32, replace=False)
    prob = sm.Problem.from_config(cfg, 64)
    T0 = torch.full((cfg.n_cells, 4), cfg.T0, dtype=torch.float64, device="cuda")
    cv = torch.full((cfg.n_cells, 4), cfg.cv, dtype=torch.float64, device="cuda")
    s = _cu(W.scale_field(cfg))
    st = A.LeakageSetup(prob, cv, T0, A.equilibrium_intensity(prob, T0), cfg.steps, 0,
                        tol=1e-13, max_iter=5000, dt=cfg.dt)
    s.requires_grad_(True)
    Jv = A.leakage(s, st)
    Jv.backward()
    g = s.grad.detach().cpu().numpy()
    errs = []
    with torch.no_grad():
        for k in cells:
            h = 1e-4 * s[k].item()
            sp, sm_ = s.detach().clone(), s.detach().clone()
            sp[k] += h
            sm_[k] -= h
            fd = (A.leakage(sp, st).item() - A.leakage(sm_, st).item()) / (2 * h)
            errs.append(abs(fd - g[k]) / abs(g[k]))
    rel_sens = np.abs(g[cells]) * s.detach().cpu().numpy()[cells] / abs(Jv.item())
    print(f"adjoint {cfg.name}: J {Jv.item():.6e}, 32 cells of the right-edge band, relative "
          f"sensitivities {rel_sens.min():.1e}..{rel_sens.max():.1e}, fd rel err max "
          f"{max(errs):.2e} median {np.median(errs):.2e}")
    assert max(errs) < 1e-4
    prob.close()


@pytest.mark.oracle_job("multigroup_1")
def test_multigroup_step_matches_oracle(gpu_lib):
    """One step of the 256x256 x 128 x 64 workload from the equilibrium start,
    FP64 and FP32 sweeps."""
    cfg = W.multigroup_2d()
    state = J.start_state(cfg)
    gpu = {p: _gpu_steps(gpu_lib, cfg, p, 1, state)[0] for p in (64, 32)}
    gpu["refined"] = _gpu_steps(gpu_lib, cfg, 32, 1, state, refine=1)[0]
    ref = J.result("multigroup_1")
    for p in (64, 32, "refined"):
        bar = 64 if p == "refined" else p   # the refined FP32 path is held to the FP64 bar
        e, same = _compare(f"{cfg.name}{' refined' if p == 'refined' else ''}", gpu[p], ref, bar)
        assert gpu[p]["stats"]["converged"] == 1
        if bar == 64:
            assert same, f"{p} path took other iteration counts than the oracle"
        bad = {k: v for k, v in e.items() if not v <= TOL[bar]}
        assert not bad, f"{p} step parity above {TOL[bar]}: {bad}"


@pytest.mark.oracle_job("gray_channel_20")
def test_gray_channel_twenty_steps_match_oracle(gpu_lib):
    """All twenty steps of the 128x128 x 128 gray channel from the equilibrium
    start, FP64 and FP32 sweeps, every step against the oracle's."""
    cfg = W.gray_channel_2d()
    state = J.start_state(cfg)
    gpu = {p: _gpu_steps(gpu_lib, cfg, p, cfg.steps, state) for p in (64, 32)}
    gpu["refined"] = _gpu_steps(gpu_lib, cfg, 32, cfg.steps, state, refine=1)
    ref = J.result("gray_channel_20")
    assert len(ref) == cfg.steps
    paths = (64, 32, "refined")
    worst = {p: {} for p in paths}
    for k in range(cfg.steps):
        for p in paths:
            bar = 64 if p == "refined" else p   # the refined FP32 path: the FP64 bar
            e, same = _compare(f"{cfg.name} step {k + 1}{' refined' if p == 'refined' else ''}",
                               gpu[p][k], ref[k], bar)
            assert gpu[p][k]["stats"]["converged"] == 1
            if bar == 64:
                assert same, f"{p} path took other iteration counts than the oracle at step {k + 1}"
            for n, v in e.items():
                worst[p][n] = max(worst[p].get(n, 0.0), v)
    for p in paths:
        bar = 64 if p == "refined" else p
        print(f"[{cfg.name} 20 steps {p}] worst " +
              "  ".join(f"{n} {v:.2e}" for n, v in worst[p].items()))
        bad = {n: v for n, v in worst[p].items() if not v <= TOL[bar]}
        assert not bad, f"{p} step parity above {TOL[bar]}: {bad}"
