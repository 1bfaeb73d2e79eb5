"""Batched problems in one persistent launch (sm_batch_*): every member's
result equals a single-problem sweep of the same problem (bit-identical
intensity; moments and closures up to the order of their atomic sums), the
FP64 batch matches the oracle per member, graphs are recorded once per buffer
set, and members refuse single-problem sweeps."""
import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cfg(i, n, ny, G, npol, naz, T_bdr=(1.0, 0.0, 0.0, 0.0)):
    return W.Config(f"m{i}", 2, n, ny, (0.0, 1.0, 0.0, 1.0), W.log_edges(G), npol, naz,
                    W.OPACITY_LARSEN, 10.0, T_bdr, seed=i)


MEMBERS = [  # uneven meshes, 32/64/128 directions, group counts giving GW = 2, 4, 8 and padding
    _cfg(0, 13, 9, 5, 2, 4),
    _cfg(1, 24, 31, 12, 4, 4),
    _cfg(2, 17, 17, 9, 4, 8, T_bdr=(1.0, 0.3, 0.5, 0.0)),
    _cfg(3, 40, 7, 3, 2, 4),
    _cfg(4, 8, 21, 20, 4, 8),
    _cfg(5, 1, 1, 2, 2, 4),
]


def _host_inputs(cfg, seed, precision):
    """Seeded host inputs of member `seed`: nodal T, per-cell scale and I^k as
    the sweep of the given precision stores it."""
    T = W.temperature_wave(cfg, seed=seed)
    scale = W.blocky_two_material(cfg.nx, cfg.ny, seed=100 + seed, block=4, thick=50.0)
    Ic = W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=seed + 3, scale=0.05)
    return T, scale, W.in_precision(Ic, precision)


def _inputs(sm, prob, cfg, seed):
    import torch
    T, scale, Ic = _host_inputs(cfg, seed, prob.info["precision"])
    T = torch.from_numpy(T).cuda()
    sigma = prob.opacity(T, torch.from_numpy(scale).cuda())
    Ip = prob.pack(torch.from_numpy(Ic).cuda())
    return T, sigma, Ip


def _run_batch(sm, cfgs, precision, tiling=None):
    b = sm.Batch(cfgs, precision)
    if tiling:
        b.set_tiling(*tiling)
    T, S, Ip, Io, M, C = [], [], [], [], [], []
    for i, (cfg, m) in enumerate(zip(cfgs, b.members)):
        t, s, ip = _inputs(sm, m, cfg, seed=i)
        T.append(t)
        S.append(s)
        Ip.append(ip)
        Io.append(m.empty_intensity())
        M.append(m.new_moments())
        C.append(m.new_closures())
    b.sweep(T, S, Ip, Io, M, C)
    b.synchronize()
    return b, T, S, Ip, Io, M, C


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("precision", [32, 64])
def test_batch_equals_single_sweeps(gpu_lib, precision):
    sm = gpu_lib
    b, T, S, Ip, Io, M, C = _run_batch(sm, MEMBERS, precision, tiling=(4, 3))
    tol = 1e-6 if precision == 32 else 1e-13
    for i, cfg in enumerate(MEMBERS):
        p = sm.Problem.from_config(cfg, precision, strip_width=4, prefetch_rows=3,
                                   groups_per_warp=b.members[i].info["groups_per_warp"])
        assert p.info["groups_per_warp"] == b.members[i].info["groups_per_warp"]
        Io1 = p.empty_intensity()
        m1, c1 = p.new_moments(), p.new_closures()
        p.sweep(T[i], S[i], Ip[i], Io1, m1, c1)
        p.synchronize()
        Ib = b.members[i].unpack(Io[i]).cpu().numpy()
        Is = p.unpack(Io1).cpu().numpy()
        assert np.array_equal(Ib, Is), f"member {i}: intensity differs"
        assert _rel(M[i].cpu().numpy()[..., 0], m1.cpu().numpy()[..., 0]) < tol
        assert _rel(C[i].cpu().numpy()[..., 6], c1.cpu().numpy()[..., 6]) < tol


def test_batch_fp64_matches_oracle(gpu_lib):
    sm = gpu_lib
    cfgs = MEMBERS[:4]
    b, T, S, Ip, Io, M, C = _run_batch(sm, cfgs, 64)
    for i, cfg in enumerate(cfgs):
        Tn, scale, Ipc = _host_inputs(cfg, i, 64)
        Sn = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, Tn, scale)
        omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
        q = O.emission(cfg.edges, cfg.a, cfg.c, Tn, Sn)
        infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
        Ir = O.sweep(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, Sn, 1.0 / (cfg.c * cfg.dt), q, Ipc,
                     infl)
        momr = O.moments(2, omx, omy, w, Sn, Ir)
        Ig = b.members[i].unpack(Io[i]).cpu().numpy()
        eI = max(_rel(Ig[d, g], Ir[d, g]) for d in range(cfg.n_dir) for g in range(cfg.n_groups))
        ephi = _rel(M[i].cpu().numpy()[..., 0], momr[..., 0])
        print(f"member {i}: I {eI:.2e} phi {ephi:.2e}")
        assert eI < 1e-11 and ephi < 1e-11


def test_batch_graphs_recorded_once_per_buffer_set(gpu_lib):
    sm = gpu_lib
    b, T, S, Ip, Io, M, C = _run_batch(sm, MEMBERS[:3], 32)
    assert b.info()["graphs_cached"] == 1
    first = [x.clone() for x in Io]
    b.sweep(T, S, Ip, Io, M, C)          # same buffers: replay
    b.synchronize()
    assert b.info()["graphs_cached"] == 1
    for x, y in zip(first, Io):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
    b.sweep(T, S, Io, Ip, M, C)          # swapped roles: a second graph
    b.synchronize()
    assert b.info()["graphs_cached"] == 2
    launches = b.info()["launches"]
    assert launches == 3 * (2 + 2 * 3)


def test_batch_autotune_keeps_results(gpu_lib):
    sm = gpu_lib
    b, T, S, Ip, Io, M, C = _run_batch(sm, MEMBERS, 32)
    ref = [x.clone() for x in Io]
    b.autotune(T, S, Ip, Io, reps=1)
    info = b.info()
    assert 1 <= info["strip_width"] <= 16 and 2 <= info["prefetch_rows"] <= 4
    b.sweep(T, S, Ip, Io, M, C)
    b.synchronize()
    for m, x, y in zip(b.members, ref, Io):
        assert np.array_equal(m.unpack(x).cpu().numpy(), m.unpack(y).cpu().numpy())


def test_batch_members_refuse_single_sweeps(gpu_lib):
    import torch
    sm = gpu_lib
    b, T, S, Ip, Io, M, C = _run_batch(sm, MEMBERS[:2], 32)
    with pytest.raises(sm.SMError, match="belongs to a batch"):
        b.members[0].sweep(T[0], S[0], Ip[0], Io[0])
    with pytest.raises(sm.SMError, match="belongs to a batch"):
        b.members[0].set_tiling(2, 2)
    one_d = W.Config("d1", 1, 10, 1, (0.0, 1.0, 0.0, 1.0), W.log_edges(3), 4, 0,
                     W.OPACITY_LARSEN, 10.0, (1.0, 0.0, 0.0, 0.0))
    with pytest.raises(sm.SMError, match="2D"):
        sm.Batch([MEMBERS[0], one_d], 32)
    del torch


def test_c5_workload_batch(gpu_lib):
    """The 64-member batched workload: every member's moments are finite and
    positive, and the smallest members match their single-problem sweeps."""
    import torch
    sm = gpu_lib
    members = W.batched_2d()
    cfgs = [m.cfg for m in members]
    b = sm.Batch(cfgs, 32)
    T, S, Io, M = [], [], [], []
    for mem, h in zip(members, b.members):
        t = torch.from_numpy(W.temperature_wave(mem.cfg)).cuda()
        T.append(t)
        S.append(h.opacity(t, torch.from_numpy(mem.scale).cuda()))
        Io.append(h.empty_intensity())
        M.append(h.new_moments())
    b.sweep(T, S, None, Io, M, None)
    b.synchronize()
    for x in M:
        phi = x[..., 0]
        assert bool(torch.isfinite(phi).all()) and bool((phi > 0).all())
    order = np.argsort([c.n_cells * c.n_dir * c.n_groups for c in cfgs])[:3]
    for i in order:
        p = sm.Problem.from_config(cfgs[i], 32, strip_width=b.info()["strip_width"],
                                   prefetch_rows=b.info()["prefetch_rows"],
                                   groups_per_warp=b.members[i].info["groups_per_warp"])
        Io1 = p.empty_intensity()
        p.sweep(T[i], S[i], None, Io1)
        p.synchronize()
        assert np.array_equal(b.members[i].unpack(Io[i]).cpu().numpy(),
                              p.unpack(Io1).cpu().numpy())


def test_problems_sharing_a_kernel_launch_in_any_order(gpu_lib):
    """Two problems with the same slots per lane but different stage sizes
    (32 directions x 32 groups, then 128 directions x 16 groups): the first
    still launches after the second configured the shared kernel."""
    import torch
    sm = gpu_lib
    big = _cfg(10, 12, 10, 32, 2, 4)
    small = _cfg(11, 9, 9, 16, 4, 8)
    pb = sm.Problem.from_config(big, 32, strip_width=8, prefetch_rows=4, groups_per_warp=8)
    ps = sm.Problem.from_config(small, 32, strip_width=2, prefetch_rows=2, groups_per_warp=8)
    assert pb.info["groups_per_warp"] == ps.info["groups_per_warp"] == 8
    for p, cfg in ((pb, big), (ps, small), (pb, big)):
        T, S, Ip = _inputs(sm, p, cfg, seed=1)
        Io = p.empty_intensity()
        p.sweep(T, S, Ip, Io)
        p.synchronize()
        assert bool(torch.isfinite(p.unpack(Io)).all())


# the step's parity mode: the paper's epsilon for the outer and Newton
# iterations (Eq. relative_tol), inner solves to round-off
_STEP_ORACLE = dict(eps_outer=1e-3, max_outer=100)
_STEP_LO = dict(eps_inner=1e-3, max_inner=30, elim_rtol=1e-15, max_elim=100)


@pytest.mark.parametrize("precision,batched_lo", [(64, True), (32, True), (64, False)])
def test_batch_step_matches_oracle(gpu_lib, precision, batched_lo):
    """Two time steps of Algorithm 1 for all six uneven members at once
    (sm_batch_step: one batched pass per outer iteration, FP64 low-order
    solves -- all members' in one cooperative launch, or, through the test
    hook, one launch per member -- and per-member stopping) against the
    oracle's steps of each member: T and E within 1e-11 (FP64 sweep) / 1e-5
    (FP32 sweep) of the field's largest magnitude, and, on the FP64 path, each
    member's own outer and Newton iteration counts.  Members start from
    radiative equilibrium at a seeded non-uniform temperature, with
    two-material opacity maps."""
    import torch
    from oracle import lo as L
    sm = gpu_lib
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    tol = {64: 1e-11, 32: 1e-5}[precision]
    b = sm.Batch(MEMBERS, precision)
    b.set_batched_lo(batched_lo)
    state, ref = [], []
    prm_o = L.StepParams(lo=L.LOParams(**_STEP_LO), **_STEP_ORACLE)
    for i, cfg in enumerate(MEMBERS):
        rng = np.random.default_rng(40 + i)
        T0 = 0.05 + 0.5 * rng.random((cfg.n_cells, 4))
        scale = W.blocky_two_material(cfg.nx, cfg.ny, seed=100 + i, block=4, thick=50.0)
        cv = np.full((cfg.n_cells, 4), 0.3)
        omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
        I0 = W.in_precision(L.equilibrium_intensity(cfg, T0, omx), precision)
        sig0 = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T0, scale)
        mom0 = O.moments(2, omx, omy, w, sig0, I0)
        T, I, mom, steps = T0, I0, mom0, []
        for _ in range(2):
            T, E, F, I, mom, st = L.sm_step(cfg, scale, cv, T, I, mom, prm_o)
            steps.append((T, E, st))
        ref.append(steps)
        m = b.members[i]
        state.append(dict(scale=cu(scale), cv=cu(cv), T=cu(T0), E=m.new_nodal(), F=m.new_flux(),
                          mom=cu(mom0), I=[m.pack(cu(I0)), m.empty_intensity()]))
    prm = sm.step_params(eps_outer=1e-3, eps_inner=1e-3, pcg_rtol=1e-15, max_pcg=20000,
                         elim_rtol=1e-15, max_elim=100)
    worst = {"T": 0.0, "E": 0.0}
    for k in range(2):
        stats = b.step([s["scale"] for s in state], [s["cv"] for s in state],
                       [s["T"] for s in state], [s["E"] for s in state],
                       [s["F"] for s in state], [s["mom"] for s in state],
                       [s["I"][k % 2] for s in state], [s["I"][(k + 1) % 2] for s in state],
                       params=prm)
        outer = []
        for i, s in enumerate(state):
            Tr, Er, st = ref[i][k]
            eT = _rel(s["T"].cpu().numpy(), Tr)
            eE = _rel(s["E"].cpu().numpy(), Er)
            worst["T"] = max(worst["T"], eT)
            worst["E"] = max(worst["E"], eE)
            assert stats[i]["converged"] == 1
            if precision == 64:
                assert stats[i]["outer_iters"] == st["outer"], (i, k, stats[i], st)
                assert stats[i]["newton_iters_total"] == sum(st["newton"]), (i, k)
            outer.append((stats[i]["outer_iters"], st["outer"]))
        print(f"batched step {k + 1} fp{precision} (low-order solves batched {batched_lo}): "
              f"outer (batch, oracle) per member {outer}")
    print(f"batched steps fp{precision} (low-order solves batched {batched_lo}): "
          f"worst T {worst['T']:.2e} E {worst['E']:.2e}")
    assert worst["T"] < tol and worst["E"] < tol
    b.close()


def test_slot_tuner_choices_are_valid_and_sweep_correctly(gpu_lib):
    """sm_batch_tune_slots picks, per member, slots per lane in {1, 2, 4, 8}
    no larger than the member's automatic choice; a batch built with them
    sweeps every member exactly as single-problem sweeps with the same slots."""
    sm = gpu_lib
    gw = sm.tune_batch_slots(MEMBERS, 32, reps=1)
    auto = sm.Batch(MEMBERS, 32)
    auto_gw = [m.info["groups_per_warp"] for m in auto.members]
    auto.close()
    assert all(g in (1, 2, 4, 8) and g <= a for g, a in zip(gw, auto_gw)), (gw, auto_gw)
    b = sm.Batch(MEMBERS, 32, groups_per_warp=gw)
    assert [m.info["groups_per_warp"] for m in b.members] == gw
    T, S, Ip, Io = [], [], [], []
    for i, (cfg, m) in enumerate(zip(MEMBERS, b.members)):
        t, s, ip = _inputs(sm, m, cfg, seed=i)
        T.append(t)
        S.append(s)
        Ip.append(ip)
        Io.append(m.empty_intensity())
    b.sweep(T, S, Ip, Io)
    b.synchronize()
    for i, cfg in enumerate(MEMBERS):
        p = sm.Problem.from_config(cfg, 32, groups_per_warp=gw[i])
        Io1 = p.empty_intensity()
        p.sweep(T[i], S[i], Ip[i], Io1)
        p.synchronize()
        assert bool((p.unpack(Io1) == b.members[i].unpack(Io[i])).all()), i
        p.close()
    print(f"tuned slots per lane {gw} (automatic {auto_gw})")
    b.close()
