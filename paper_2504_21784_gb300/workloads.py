"""Seeded synthetic workloads: problem descriptions and input fields.

This module holds no arithmetic of the method (no Planck integral, no
opacity law, no sweep).  It only states the five problem shapes and draws
the seeded fields that both the CUDA library and the CPU oracle consume:
nodal temperatures, per-cell opacity scale factors (material maps), group
edges, and random non-negative intensities for parity cases.

The shapes follow the paper's workloads (Sec. 6, Table 1): a 1D gray
Marshak-type wave (Sec. 6.1), a 2D gray two-material channel standing in
for the crooked pipe (Sec. 6.3; its geometry is only in a figure, so the
channel here is a fixed bent strip), a 2D multigroup problem with the
opacity form alpha (1 - e^{-nu/T}) / nu^3 of Sec. 6.2, the same at the
adjoint size, and a batch of uneven 2D problems.  Units: a = c = 1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

#: opacity model ids understood by both the library and the oracle
OPACITY_POWER = 0   # sigma = s_K * Tbar^-3 (all groups)
OPACITY_LARSEN = 1  # sigma_g = s_K * alpha (1 - exp(-E_g/Tbar)) / E_g^3


@dataclasses.dataclass
class Config:
    name: str
    dim: int
    nx: int
    ny: int
    extent: Tuple[float, float, float, float]
    edges: np.ndarray            # n_groups + 1 ascending group edges
    n_polar: int                 # 1D: GL order; 2D: polar cosines per octant
    n_azim: int                  # 2D: azimuths per octant
    opacity_kind: int
    opacity_alpha: float
    T_bdr: Tuple[float, float, float, float]   # left, right, bottom, top (<=0: vacuum)
    a: float = 1.0
    c: float = 1.0
    dt: float = 0.01
    cv: float = 0.3
    T0: float = 0.01
    steps: int = 10
    seed: int = 0
    scale_1d: float = 100.0      # 1D: per-cell opacity scale s_K (all cells)

    @property
    def n_groups(self) -> int:
        return len(self.edges) - 1

    @property
    def n_dir(self) -> int:
        return self.n_polar if self.dim == 1 else 4 * self.n_polar * self.n_azim

    @property
    def n_cells(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    @property
    def n_nodes(self) -> int:
        return 2 if self.dim == 1 else 4

    @property
    def updates(self) -> int:
        """cell-direction-group updates per sweep"""
        return self.n_cells * self.n_dir * self.n_groups

    def resized(self, nx: int, ny: Optional[int] = None, n_groups: Optional[int] = None,
                n_polar: Optional[int] = None, n_azim: Optional[int] = None) -> "Config":
        """Same problem family at another size (parity cases)."""
        c = dataclasses.replace(self)
        c.nx = nx
        c.ny = ny if ny is not None else (nx if self.dim == 2 else 1)
        if n_groups is not None and n_groups != self.n_groups:
            c.edges = log_edges(n_groups)
        if n_polar is not None:
            c.n_polar = n_polar
        if n_azim is not None:
            c.n_azim = n_azim
        return c


def log_edges(n_groups: int, lo: float = 1e-2, hi: float = 1e2) -> np.ndarray:
    """n_groups log-spaced groups on [lo, hi] (n_groups + 1 edges)."""
    return np.logspace(math.log10(lo), math.log10(hi), n_groups + 1)


GRAY_EDGES = np.array([1e-2, 1e2])  # one group; its spectrum integrates to 1


def marshak_1d() -> Config:
    """1D slab gray Marshak-type wave: 200 cells on [0,1], S8 Gauss-Legendre,
    sigma = 100 T^-3, c_v = 0.3, T0 = 0.01, Planck inflow at T = 1 on the left,
    vacuum on the right, dt = 0.01, 10 steps."""
    return Config("marshak1d_200x8x1", 1, 200, 1, (0.0, 1.0, 0.0, 1.0), GRAY_EDGES.copy(), 8, 0,
                  OPACITY_POWER, 0.0, (1.0, 0.0, 0.0, 0.0), steps=10)


def gray_channel_2d() -> Config:
    """2D gray two-material layout: 128x128 quads on [0,1]^2, 4 polar x 8
    azimuthal per octant (128 directions), sigma = 0.2 T^-3 in a bent channel
    and 2000 T^-3 in the walls, Planck inflow T = 1 on the left edge, 20 steps."""
    return Config("graychannel2d_128x128x128x1", 2, 128, 128, (0.0, 1.0, 0.0, 1.0),
                  GRAY_EDGES.copy(), 4, 8, OPACITY_POWER, 0.0, (1.0, 0.0, 0.0, 0.0), steps=20)


def multigroup_2d() -> Config:
    """2D multigroup: 256x256 quads, 128 directions, 64 log-spaced groups on
    [0.01, 100], sigma_g = s_K 10 (1 - e^{-E_g/T}) / E_g^3 with a lognormal
    per-cell scale (sigma_ln = 0.5, seed 2504), Planck inflow T = 1 on the left."""
    return Config("multigroup2d_256x256x128x64", 2, 256, 256, (0.0, 1.0, 0.0, 1.0), log_edges(64),
                  4, 8, OPACITY_LARSEN, 10.0, (1.0, 0.0, 0.0, 0.0), steps=10, seed=2504)


def adjoint_2d() -> Config:
    """Adjoint-size problem: 128x128, 64 directions, 16 groups, 20 steps."""
    return Config("adjoint2d_128x128x64x16", 2, 128, 128, (0.0, 1.0, 0.0, 1.0), log_edges(16),
                  4, 4, OPACITY_LARSEN, 10.0, (1.0, 0.0, 0.0, 0.0), steps=20, seed=21784)


def adjoint_2d_warm() -> Config:
    """The adjoint problem from a warm uniform start T0 = 0.3 (the configuration
    leaves the initial state open; from T0 = 0.01 the 20-step right-edge leakage
    depends on a few right-edge cells only, from T0 = 0.3 on ~25 columns)."""
    c = adjoint_2d()
    return dataclasses.replace(c, name="adjoint2d_warm_128x128x64x16", T0=0.3)


# CGS units with temperatures in eV: the radiation constant a = 4 sigma_SB / c
# in erg cm^-3 eV^-4 (7.5657e-15 erg cm^-3 K^-4 at 11604.518 K per eV) and c in
# cm/s
A_RAD_EV = 7.5657e-15 * 11604.518 ** 4
C_CM_S = 2.99792458e10


def marshak_paper(nx: int = 64, dt: float = 8e-12) -> Config:
    """The Marshak wave in the paper's units (Sec. 6, Marshak wave definition):
    [0, 0.05 cm], 2.5 ns, sigma = 1e12 T^-3 cm^-1 (T in eV), c_v = 3e12
    erg cm^-3 eV^-1, equilibrium at 1 eV, a 1 keV Planck source at x = 0
    (vacuum at the right end), Gauss-Legendre S6; dt in seconds (8e-12 s is
    the coarsest step of the paper's time refinement)."""
    steps = int(round(2.5e-9 / dt))
    return Config(f"marshakpaper1d_{nx}x6x1", 1, nx, 1, (0.0, 0.05, 0.0, 1.0), GRAY_EDGES.copy(),
                  6, 0, OPACITY_POWER, 0.0, (1000.0, 0.0, 0.0, 0.0), a=A_RAD_EV, c=C_CM_S, dt=dt,
                  cv=3e12, T0=1.0, steps=steps, scale_1d=1e12)


CONFIGS = {
    "c1": marshak_1d,
    "c2": gray_channel_2d,
    "c3": multigroup_2d,
    "c4": adjoint_2d,
}


# --------------------------------------------------------------------------- fields
def node_coords(cfg: Config) -> Tuple[np.ndarray, np.ndarray]:
    """Physical coordinates of every (cell, node): arrays [cell][node]."""
    x0, x1, y0, y1 = cfg.extent
    hx = (x1 - x0) / cfg.nx
    if cfg.dim == 1:
        ix = np.arange(cfg.nx)
        X = x0 + (ix[:, None] + np.array([0, 1])[None, :]) * hx
        return X, np.zeros_like(X)
    hy = (y1 - y0) / cfg.ny
    iy, ix = np.divmod(np.arange(cfg.nx * cfg.ny), cfg.nx)
    a = np.array([0, 1, 0, 1])
    b = np.array([0, 0, 1, 1])
    X = x0 + (ix[:, None] + a[None, :]) * hx
    Y = y0 + (iy[:, None] + b[None, :]) * hy
    return X, Y


def cell_centres(cfg: Config) -> Tuple[np.ndarray, np.ndarray]:
    X, Y = node_coords(cfg)
    return X.mean(axis=1), Y.mean(axis=1)


def channel_mask(cfg: Config) -> np.ndarray:
    """Bent channel of width 1/8 (union of three rectangles) entering from the
    left edge: True inside the channel (thin material)."""
    xc, yc = cell_centres(cfg)
    x0, x1, y0, y1 = cfg.extent
    u = (xc - x0) / (x1 - x0)
    v = (yc - y0) / (y1 - y0)
    w = 0.125
    leg1 = (u <= 0.5) & (v >= 0.25) & (v <= 0.25 + w)
    riser = (u >= 0.5 - w) & (u <= 0.5) & (v >= 0.25) & (v <= 0.75)
    leg2 = (u >= 0.5 - w) & (v >= 0.75 - w) & (v <= 0.75)
    return leg1 | riser | leg2


def scale_field(cfg: Config, seed: Optional[int] = None) -> np.ndarray:
    """Per-cell opacity scale s_K for the problem's material layout."""
    seed = cfg.seed if seed is None else seed
    if cfg.dim == 1:
        return np.full(cfg.n_cells, cfg.scale_1d)
    if cfg.opacity_kind == OPACITY_POWER:
        return np.where(channel_mask(cfg), 0.2, 2000.0)
    rng = np.random.default_rng(seed)
    return np.exp(0.5 * rng.standard_normal(cfg.n_cells))


def blocky_two_material(nx: int, ny: int, seed: int, block: int = 8, p_thick: float = 0.3,
                        thin: float = 1.0, thick: float = 1000.0) -> np.ndarray:
    """Random two-material map made of block x block cell blocks."""
    rng = np.random.default_rng(seed)
    bx, by = -(-nx // block), -(-ny // block)
    blk = rng.random((by, bx)) < p_thick
    iy, ix = np.divmod(np.arange(nx * ny), nx)
    return np.where(blk[iy // block, ix // block], thick, thin)


def temperature_wave(cfg: Config, seed: int = 1, noise: float = 0.01) -> np.ndarray:
    """Nodal temperature snapshot of a wave entering from the left, in
    [0.01, 1]: hot behind a front near x = 0.3 that wiggles with y, cold
    ahead of it, with small seeded per-node noise.  [cell][node]."""
    X, Y = node_coords(cfg)
    x0, x1, y0, y1 = cfg.extent
    u = (X - x0) / (x1 - x0)
    v = (Y - y0) / (y1 - y0) if cfg.dim == 2 else np.zeros_like(u)
    front = 0.3 + 0.05 * np.sin(2 * np.pi * v)
    T = 0.01 + 0.99 / (1.0 + np.exp((u - front) / 0.05))
    rng = np.random.default_rng(seed)
    T = T * (1.0 + noise * rng.uniform(-1, 1, size=T.shape))
    return np.clip(T, 0.01, 1.0)


def temperature_random(n_cells: int, n_nodes: int, seed: int, lo: float = 0.01,
                       hi: float = 1.0) -> np.ndarray:
    """Log-uniform nodal temperatures on [lo, hi].  [cell][node]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=(n_cells, n_nodes)))


def intensity_random(n_dir: int, n_groups: int, n_cells: int, n_nodes: int, seed: int,
                     scale: float = 1.0) -> np.ndarray:
    """Non-negative random intensities [d][g][cell][node] (lognormal)."""
    rng = np.random.default_rng(seed)
    return scale * np.exp(rng.standard_normal((n_dir, n_groups, n_cells, n_nodes)) - 2.0)


def in_precision(x: np.ndarray, precision: int) -> np.ndarray:
    """x as a sweep of the given precision stores it: rounded to the nearest
    FP32 value for the FP32 sweep, unchanged for FP64 (as float64 either way),
    so that both sides of a comparison read the same previous intensity."""
    x = np.asarray(x, dtype=np.float64)
    return x.astype(np.float32).astype(np.float64) if precision == 32 else x


class SeparableIntensity:
    """A seeded previous intensity I[d][g][cell][node] = s a_d b_g c_{cell,node}
    with lognormal factors, exactly representable in FP32 (so the FP32 and
    FP64 sweeps read the same values), produced one direction at a time so that
    full-size workloads never need the whole array on the host."""

    def __init__(self, n_dir: int, n_groups: int, n_cells: int, n_nodes: int, seed: int,
                 scale: float = 0.05):
        rng = np.random.default_rng(seed)
        self.a = scale * np.exp(0.3 * rng.standard_normal(n_dir))
        self.b = np.exp(0.5 * rng.standard_normal(n_groups))
        self.c = np.exp(0.5 * rng.standard_normal((n_cells, n_nodes)) - 2.0)
        self.n_dir = n_dir

    def direction(self, d: int) -> np.ndarray:
        """[g][cell][node] of direction d."""
        return in_precision(self.a[d] * np.multiply.outer(self.b, self.c), 32)


@dataclasses.dataclass
class BatchMember:
    cfg: Config
    scale: np.ndarray


def batched_2d(n_problems: int = 64) -> List[BatchMember]:
    """64 independent 2D problems with seeded sizes 32^2..256^2 (log-uniform),
    8..32 groups, 32/64/128 directions, blocky two-material layouts
    (8x8-cell blocks, P(thick) = 0.3); problem i uses seed i."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(i)
        n = int(round(math.exp(rng.uniform(math.log(32), math.log(256)))))
        G = int(rng.integers(8, 33))
        npol, naz = [(2, 4), (4, 4), (4, 8)][int(rng.integers(0, 3))]
        cfg = Config(f"batch{i:02d}_{n}x{n}x{4 * npol * naz}x{G}", 2, n, n, (0.0, 1.0, 0.0, 1.0),
                     log_edges(G), npol, naz, OPACITY_LARSEN, 10.0, (1.0, 0.0, 0.0, 0.0),
                     steps=10, seed=i)
        out.append(BatchMember(cfg, blocky_two_material(n, n, seed=1000 + i)))
    return out
