"""GPU forward steps and discrete adjoint (sm_ho_step, sm_leakage,
sm_adjoint_step, the checkpointed autograd function) against the FP64 oracle
(oracle/adjoint.py) and against central finite differences of the GPU
forward itself.

Tolerances: forward and adjoint are converged to 1e-13 relative change on
both sides (different iteration paths to the same fixed point), so states,
objective and gradient agree to ~1e-11 relative; central differences with
h = 1e-4 s_K (the spec check) carry O(h^2) truncation, bar 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from paper_2504_21784_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pair(nx=3, ny=2, G=3, npol=1, naz=2, kind=1, seed=1):
    cfg = W.Config("adj", 2, nx, ny, (0.0, 1.0, 0.0, 0.8),
                   W.log_edges(G) if G > 1 else W.GRAY_EDGES.copy(), npol, naz, kind,
                   10.0 if kind == 1 else 0.0, (1.0, 0.0, 0.4, 0.0), dt=0.01)
    pb = OA.Problem(nx, ny, cfg.extent, cfg.edges, npol, naz, kind, cfg.opacity_alpha, cfg.T_bdr,
                    dt=cfg.dt)
    rng = np.random.default_rng(seed)
    ncell = nx * ny
    scale = np.exp(0.5 * rng.standard_normal(ncell))
    cv = np.full((ncell, 4), 0.3)
    T0 = 0.2 + 0.3 * rng.random((ncell, 4))
    omx, omy, w = O.quadrature(2, npol, naz)
    B4, _ = OA.planck_parts(pb, T0)
    I0 = np.broadcast_to(B4[None], (len(w),) + B4.shape).copy()
    return cfg, pb, scale, cv, T0, I0


def _setup(sm, cfg, scale, cv, T0, I0, nsteps, every=0):
    import torch
    from paper_2504_21784_gb300 import adjoint as A
    prob = sm.Problem.from_config(cfg, 64)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    st = A.LeakageSetup(prob, cu(cv), cu(T0), prob.pack(cu(I0)), nsteps, every, tol=1e-13,
                        max_iter=2000, dt=cfg.dt)
    return prob, st, cu(scale)


def test_forward_matches_oracle(gpu_lib):
    import torch
    sm = gpu_lib
    cfg, pb, scale, cv, T0, I0 = _pair()
    J, Ts, Is, _ = OA.forward(pb, scale, cv, T0, I0, 3)
    prob, st, s = _setup(sm, cfg, scale, cv, T0, I0, 3)
    T = st.T0.clone()
    Ic = st.I0
    Jg = 0.0
    for n in range(3):
        In = prob.empty_intensity()
        prob.ho_step(s, st.cv, T, Ic, In, 1e-13, 2000)
        Jg += cfg.dt * prob.leakage(In)
        Ic = In
    eT = np.abs(T.cpu().numpy() - Ts[3]).max() / np.abs(Ts[3]).max()
    eI = np.abs(prob.unpack(Ic).cpu().numpy() - Is[3]).max() / np.abs(Is[3]).max()
    print(f"T {eT:.2e} I {eI:.2e} J {abs(Jg - J) / J:.2e}")
    assert eT < 1e-11 and eI < 1e-11 and abs(Jg - J) < 1e-11 * J
    del torch


@pytest.mark.parametrize("kind,G", [(1, 3), (0, 1)])
def test_adjoint_gradient_matches_oracle(gpu_lib, kind, G):
    from paper_2504_21784_gb300 import adjoint as A
    sm = gpu_lib
    cfg, pb, scale, cv, T0, I0 = _pair(kind=kind, G=G, nx=4, ny=3)
    J, Ts, Is, _ = OA.forward(pb, scale, cv, T0, I0, 3)
    gref = OA.adjoint(pb, scale, cv, Ts, Is)
    prob, st, s = _setup(sm, cfg, scale, cv, T0, I0, 3, every=2)
    s.requires_grad_(True)
    Jg = A.leakage(s, st)
    Jg.backward()
    g = s.grad.cpu().numpy()
    err = np.abs(g - gref).max() / np.abs(gref).max()
    print(f"kind {kind}: J {abs(Jg.item() - J) / J:.2e} grad {err:.2e}")
    assert abs(Jg.item() - J) < 1e-11 * J
    assert err < 1e-11


def test_adjoint_gradient_matches_gpu_finite_differences(gpu_lib):
    """A larger multigroup case than the oracle handles quickly: 12x10 cells,
    6 groups, 32 directions, 3 steps; central differences h = 1e-4 s_K on 6
    cells, the largest gradients included."""
    import torch
    from paper_2504_21784_gb300 import adjoint as A
    sm = gpu_lib
    cfg, pb, scale, cv, T0, I0 = _pair(nx=12, ny=10, G=6, npol=2, naz=4, seed=7)
    prob, st, s = _setup(sm, cfg, scale, cv, T0, I0, 3)
    s.requires_grad_(True)
    J = A.leakage(s, st)
    J.backward()
    g = s.grad.detach().cpu().numpy()
    cells = list(np.argsort(-np.abs(g))[:3]) + list(np.random.default_rng(3).choice(len(g), 3))
    worst = 0.0
    with torch.no_grad():
        for k in cells:
            h = 1e-4 * scale[k]
            sp, sm_ = s.detach().clone(), s.detach().clone()
            sp[k] += h
            sm_[k] -= h
            fd = (A.leakage(sp, st).item() - A.leakage(sm_, st).item()) / (2 * h)
            worst = max(worst, abs(fd - g[k]) / np.abs(g).max())
    print(f"max |grad - fd| / max |grad| = {worst:.2e}")
    assert worst < 1e-4


def test_checkpointing_does_not_change_the_gradient(gpu_lib):
    from paper_2504_21784_gb300 import adjoint as A
    sm = gpu_lib
    cfg, pb, scale, cv, T0, I0 = _pair(nx=6, ny=5, G=4, npol=2, naz=2, seed=11)
    grads = []
    for every in (1, 2, 5):
        prob, st, s = _setup(sm, cfg, scale, cv, T0, I0, 5, every=every)
        s.requires_grad_(True)
        A.leakage(s, st).backward()
        grads.append(s.grad.cpu().numpy())
    for g in grads[1:]:
        assert np.abs(g - grads[0]).max() < 1e-12 * np.abs(grads[0]).max()


def test_forward_and_gradient_are_bit_reproducible(gpu_lib):
    """The convergence norms and the leakage are fixed-order sums, so two runs
    of the forward and of the checkpointed backward give the same bits (the
    central differences of J see no run-to-run summation noise).  480 cells:
    several blocks of the norm and leakage reductions."""
    from paper_2504_21784_gb300 import adjoint as A
    sm = gpu_lib
    cfg, pb, scale, cv, T0, I0 = _pair(nx=24, ny=20, G=4, npol=2, naz=2, seed=5)
    out = []
    for _ in range(2):
        prob, st, s = _setup(sm, cfg, scale, cv, T0, I0, 4, every=2)
        s.requires_grad_(True)
        J = A.leakage(s, st)
        J.backward()
        out.append((J.item(), s.grad.cpu().numpy()))
        prob.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])


def test_adjoint_rejects_bad_arguments(gpu_lib):
    import torch
    sm = gpu_lib
    cfg, pb, scale, cv, T0, I0 = _pair()
    prob, st, s = _setup(sm, cfg, scale, cv, T0, I0, 1)
    a = prob.empty_intensity()
    with pytest.raises(sm.SMError, match="alias"):
        prob.adjoint_step(s, st.cv, st.T0, st.T0, st.I0, a, None, a, st.T0.clone(),
                          torch.zeros_like(s))
    with pytest.raises(sm.SMError, match="tol"):
        prob.ho_step(s, st.cv, st.T0.clone(), st.I0, a, 0.0, 10)
