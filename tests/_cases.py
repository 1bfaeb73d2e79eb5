"""Shared helpers for the GPU parity tests: build one case on both sides.

The library gets its inputs as torch tensors; the oracle gets the same values
as numpy arrays.  Nothing here computes any part of the method: the oracle
computes every expected value."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle as O
from paper_2504_21784_gb300 import workloads as W


def config(dim, nx, ny, G, npol, naz=0, kind=W.OPACITY_LARSEN, T_bdr=(1.0, 0.0, 0.0, 0.0),
           dt=0.01, extent=(0.0, 1.0, 0.0, 1.0), name="case") -> W.Config:
    edges = W.log_edges(G) if G > 1 else W.GRAY_EDGES.copy()
    return W.Config(name, dim, nx, ny if dim == 2 else 1, extent, edges, npol, naz, kind,
                    10.0 if kind == W.OPACITY_LARSEN else 0.0, T_bdr, dt=dt)


def rel_err(got, ref, floor_frac):
    """max |got - ref| / (|ref| + floor_frac * max|ref|)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref) + floor_frac * np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref) / scale))


@dataclasses.dataclass
class Case:
    cfg: W.Config
    prob: object
    T: np.ndarray
    scale: np.ndarray
    sigma: np.ndarray        # oracle opacity, fed to both sides
    I_prev: np.ndarray       # canonical, already rounded to the sweep precision
    q: np.ndarray            # oracle emission
    inflow: np.ndarray       # oracle inflow
    omx: np.ndarray
    omy: np.ndarray
    w: np.ndarray


def build_case(sm, cfg: W.Config, precision: int, seed: int = 0, with_prev: bool = True,
               **tiling) -> Case:
    prob = sm.Problem.from_config(cfg, precision, **tiling)
    nn = cfg.n_nodes
    T = W.temperature_wave(cfg, seed=seed + 1)
    scale = W.scale_field(cfg, seed=seed + 7)
    sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, scale)
    omx, omy, w = O.quadrature(cfg.dim, cfg.n_polar, cfg.n_azim)
    I_prev = None
    if with_prev:
        Ic = W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, nn, seed=seed + 3,
                                scale=0.05)
        I_prev = W.in_precision(Ic, precision)  # what the sweep really reads
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    return Case(cfg, prob, T, scale, sigma, I_prev, q, infl, omx, omy, w)


def run_gpu(case: Case, want_closures=True):
    import torch
    prob = case.prob
    Td = torch.from_numpy(case.T).cuda()
    Sd = torch.from_numpy(case.sigma).cuda()
    Ip = None
    if case.I_prev is not None:
        Ip = prob.pack(torch.from_numpy(case.I_prev).cuda())
    Io = prob.empty_intensity()
    mom = prob.new_moments()
    clo = prob.new_closures() if want_closures else None
    prob.sweep(Td, Sd, Ip, Io, mom, clo)
    prob.synchronize()
    I = prob.unpack(Io).cpu().numpy()
    return I, mom.cpu().numpy(), (clo.cpu().numpy() if clo is not None else None), Io


def run_oracle(case: Case):
    cfg = case.cfg
    inv_cdt = 1.0 / (cfg.c * cfg.dt) if cfg.dt > 0 else 0.0
    I = O.sweep(cfg.dim, cfg.nx, cfg.ny, cfg.extent, case.omx, case.omy, case.sigma, inv_cdt,
                case.q, case.I_prev, case.inflow)
    mom = O.moments(cfg.dim, case.omx, case.omy, case.w, case.sigma, I)
    clo = O.closures(cfg.dim, cfg.edges, cfg.c, case.sigma, case.T, mom)
    return I, mom, clo


#: unit roundoff of the sweep precisions
UNIT_ROUNDOFF = {64: 2.0 ** -53, 32: 2.0 ** -24}


def elem_bound(cfg, precision, rel_tol):
    """(relative, cell) coefficients of the element-wise intensity bound
    |got - ref| <= r |ref| + a max|ref over the element's cell|:
    r = max(rel_tol, 2 u (nx + ny)) -- a cell solve errs by a few units of
    roundoff of its inputs and those errors add up along an upwind path of at
    most nx + ny cells (the contraction factor is at most 1) -- and a = 64 u,
    the cancellation inside one lumped cell solve (no positivity fix-up: a
    node can pass through zero while its cell's other nodes set the scale)."""
    u = UNIT_ROUNDOFF[precision]
    path = cfg.nx + (cfg.ny if cfg.dim == 2 else 0)
    return max(rel_tol, 2.0 * u * path), 64.0 * u


def cell_elem_err(got, ref, rel, cell):
    """Element-wise intensity error of [..][cell][node] arrays (leading axes:
    direction, group) against the bound of elem_bound: max |got - ref| /
    (rel |ref| + cell * the largest |ref| at the nodes of the element's cell
    + 1e-30 * the largest |ref| of its slice, which only keeps values below
    the FP32 range out); at most 1 when the bound holds."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    a = np.abs(ref)
    scale = (rel * a + cell * a.max(axis=-1, keepdims=True) +
             1e-30 * a.max(axis=(-2, -1), keepdims=True) + 1e-300)
    return float(np.max(np.abs(got - ref) / scale))


def field_err(got, ref, scale_field=None, axis=None):
    """max |got - ref| / max|scale| (per slice along leading axes when axis given)."""
    sc = ref if scale_field is None else scale_field
    d = np.abs(np.asarray(got) - np.asarray(ref))
    if axis is None:
        return float(d.max() / max(np.abs(sc).max(), 1e-300))
    red = tuple(range(axis, d.ndim))
    return float(np.max(d.max(axis=red) / np.maximum(np.abs(sc).max(axis=red), 1e-300)))


def parity_errors(cfg, gpu, ref, precision=None, rel_tol=None):
    """Per-field relative errors of (intensity, moments, closures); intensity
    None skips its entries.  With precision and rel_tol, "I_elem" is the ratio
    of the largest element-wise intensity error to its bound (elem_bound),
    scaled by rel_tol so that it compares with the same bar as the fields."""
    Ig, mg, cg = gpu
    Io, mo, co = ref
    dim = cfg.dim
    e = {}
    if Ig is not None:
        e["I"] = field_err(Ig, Io, axis=2)  # per (d, g) slice
        if precision is not None:
            r, a = elem_bound(cfg, precision, rel_tol)
            e["I_elem"] = rel_tol * cell_elem_err(Ig, Io, r, a)
    if dim == 2:
        phi, se = 0, 6
        groups = {"phi": [0], "F,T": [1, 2, 3, 4, 5], "SE": [6], "SF": [7, 8]}
        scale_of = {"phi": 0, "F,T": 0, "SE": 6, "SF": 6}
        sE, sF, sP, corr, E_, vec = 6, 7, 8, [9, 10], 0, [1, 2, 3, 4, 5]
    else:
        phi, se = 0, 3
        groups = {"phi": [0], "F,T": [1, 2], "SE": [3], "SF": [4]}
        scale_of = {"phi": 0, "F,T": 0, "SE": 3, "SF": 3}
        sE, sF, sP, corr, E_, vec = 3, 4, 5, [6], 0, [1, 2]
    for name, ms in groups.items():
        e["mom_" + name] = max(field_err(mg[..., m], mo[..., m], mo[..., scale_of[name]])
                               for m in ms)
    e["clo_E"] = field_err(cg[..., E_], co[..., E_])
    e["clo_F,T"] = max(field_err(cg[..., j], co[..., j], co[..., E_] * cfg.c) for j in vec)
    e["clo_sigE"] = field_err(cg[..., sE] * mo[..., phi], co[..., sE] * mo[..., phi],
                               mo[..., se])
    e["clo_sigF,P"] = max(rel_err(cg[..., j], co[..., j], 0.0) for j in (sF, sP))
    e["clo_corr"] = max(field_err(cg[..., j], co[..., j], co[..., sF] * mo[..., phi])
                        for j in corr)
    return e
