"""Oracle time steps at the full configuration sizes, run in spawned worker
processes while the GPU tests run.

The oracle takes minutes for these runs (every linearised low-order system is
factorised by sparse LU, every sweep is the plain C oracle), the GPU seconds.
``start`` is called once the test session knows which tests it will run (see
conftest.py), so the oracle works in the background from the first test on;
a test then waits for its job with ``result``.  Workers are spawned, never
forked, so no CUDA state is inherited, and they import the oracle only.

Every job returns what the oracle alone computes from seeded inputs; nothing
here reads a GPU result.

Parity mode (Algorithm 1, Eq. relative_tol): the outer and Newton iterations
keep the paper's epsilon = 1e-3, so that both sides take the same iteration
counts, while every inner solve is driven to round-off (the oracle's linear
solves are direct; its pointwise temperature elimination stops at 1e-15), so
that the two sides follow the same iterates up to rounding.
"""
from __future__ import annotations

import concurrent.futures
import math
import multiprocessing
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

#: the paper's outer / Newton controls, inner solves to round-off
PARITY_LO = dict(eps_inner=1e-3, max_inner=30, elim_rtol=1e-15, max_elim=100)
PARITY_OUTER = dict(eps_outer=1e-3, max_outer=100)

JOBS = ("gray_channel_20", "multigroup_1")

_pool = None
_futures: dict = {}


def _path():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _params():
    from oracle import lo as L
    return L.StepParams(lo=L.LOParams(**PARITY_LO), **PARITY_OUTER)


def equilibrium_group_intensity(cfg):
    """B_g(T0)/4pi at every node of the mesh, [g][cell][node]: the intensity of
    every direction in the equilibrium start (Sec. 6.1, I^0 = B(T0)/4pi)."""
    _path()
    import numpy as np
    import oracle as O
    b, _ = O.group_spectra(cfg.edges, cfg.T0)
    v = cfg.a * cfg.c * cfg.T0 ** 4 * b / (4.0 * math.pi)
    return np.ascontiguousarray(np.broadcast_to(v[:, None, None],
                                                (cfg.n_groups, cfg.n_cells, cfg.n_nodes)))


def equilibrium_moments(cfg, sigma, I_dir):
    """Moments of the equilibrium start, summed direction by direction."""
    _path()
    import numpy as np
    import oracle as O
    omx, omy, w = O.quadrature(cfg.dim, cfg.n_polar, cfg.n_azim)
    mom = np.zeros((cfg.n_cells, cfg.n_nodes, 9 if cfg.dim == 2 else 5))
    for d in range(cfg.n_dir):
        mom += O.moments(cfg.dim, omx[d:d + 1], omy[d:d + 1], w[d:d + 1], sigma, I_dir[None])
    return mom


def start_state(cfg):
    """(T0, I0 of one direction [g][cell][node], mom0, scale, cv) of the
    equilibrium start T = T0 everywhere."""
    _path()
    import numpy as np
    import oracle as O
    from paper_2504_21784_gb300 import workloads as W
    T0 = np.full((cfg.n_cells, cfg.n_nodes), cfg.T0)
    scale = W.scale_field(cfg)
    cv = np.full((cfg.n_cells, cfg.n_nodes), cfg.cv)
    I_dir = equilibrium_group_intensity(cfg)
    sig = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T0, scale)
    return T0, I_dir, equilibrium_moments(cfg, sig, I_dir), scale, cv


def gray_channel_steps(nsteps: int = 20):
    """The 2D gray channel (128x128 cells, 128 directions) over its twenty
    steps from the equilibrium start: per step T, E and the iteration counts."""
    _path()
    import numpy as np
    from oracle import lo as L
    from paper_2504_21784_gb300 import workloads as W
    cfg = W.gray_channel_2d()
    T, I_dir, mom, scale, cv = start_state(cfg)
    I = np.ascontiguousarray(np.broadcast_to(I_dir[None], (cfg.n_dir,) + I_dir.shape))
    out = []
    for _ in range(nsteps):
        T, E, F, I, mom, st = L.sm_step(cfg, scale, cv, T, I, mom, _params())
        out.append({"T": T, "E": E, "phi": mom[..., 0].copy(), "outer": st["outer"],
                    "newton": list(st["newton"])})
    return out


def multigroup_step():
    """One step of the 2D multigroup workload (256x256 cells, 128 directions,
    64 groups) from the equilibrium start; the previous intensity is the same
    for every direction, so each sweep runs one direction at a time."""
    _path()
    from oracle import lo as L
    from paper_2504_21784_gb300 import workloads as W
    cfg = W.multigroup_2d()
    T0, I_dir, mom0, scale, cv = start_state(cfg)
    T, E, F, _, mom, st = L.sm_step(cfg, scale, cv, T0, lambda d: I_dir, mom0, _params())
    return {"T": T, "E": E, "phi": mom[..., 0].copy(), "outer": st["outer"],
            "newton": list(st["newton"])}


_RUN = {"gray_channel_20": gray_channel_steps, "multigroup_1": multigroup_step}


def start(names=JOBS):
    """Submit the named jobs (once each) to a pool of spawned workers."""
    global _pool
    todo = [n for n in names if n not in _futures]
    if not todo:
        return
    if _pool is None:
        _pool = concurrent.futures.ProcessPoolExecutor(
            max_workers=len(JOBS), mp_context=multiprocessing.get_context("spawn"))
    for n in todo:
        _futures[n] = _pool.submit(_RUN[n])


def result(name, timeout=None):
    start([name])
    return _futures[name].result(timeout=timeout)


def shutdown():
    global _pool
    if _pool is not None:
        _pool.shutdown(wait=False, cancel_futures=True)
        _pool = None
    _futures.clear()
