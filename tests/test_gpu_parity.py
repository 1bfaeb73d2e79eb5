"""GPU parity: the CUDA hot path (through the C ABI) against the FP64 oracle,
element by element, on seeded inputs that span several strips, several warp
tasks, padded lanes and groups, and ragged strip tails.

Tolerances (the FP64 bound leaves room for the reordered sums of the fused
moments and the table-driven Planck functions; the FP32 bound for the
rounding of I, q and the cell solve to single precision):
  FP64 sweep:  1e-11 relative      FP32 sweep:  1e-5 relative
"Relative" is taken per field, as the paper reports errors relative to the
magnitude of the reference: every element's error is divided by the largest
magnitude of its field -- one (direction, group) slice of the intensity, one
moment component (F and T are measured against phi, SF against SE, as they
vanish near equilibrium).  The intensity is also bounded element by element
("I_elem"): each node's error against its own magnitude plus 1e-2 of the
largest magnitude at its cell's nodes times 64 units of roundoff (the
lumped-DG solution has no positivity fix-up and can pass through zero inside
a cell, where dividing by the element itself is meaningless), with the
relative part max(bar, 2 u (nx + ny)) -- per-cell roundoff adding up along an
upwind path (_cases.elem_bound) -- so cells far below their slice's maximum
are held to a relative bar too.  sigma_E = SE/phi is compared weighted by
phi for the same reason, the additive correction against sigma_F * phi.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W

from _cases import build_case, config, parity_errors, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = {64: 1e-11, 32: 1e-5}

CASES_2D = {
    # name: (config kwargs, tiling kwargs)
    "ragged_lanes": (dict(nx=37, ny=21, G=5, npol=2, naz=3),
                     dict(strip_width=8, prefetch_rows=2, groups_per_warp=1)),
    "gw2_32dirs": (dict(nx=24, ny=19, G=12, npol=4, naz=8),
                   dict(strip_width=4, prefetch_rows=4, groups_per_warp=2)),
    "gw4_dirblocks": (dict(nx=17, ny=9, G=6, npol=4, naz=16),
                      dict(strip_width=3, prefetch_rows=3, groups_per_warp=4)),
    "gray_channel": (dict(nx=32, ny=32, G=1, npol=4, naz=8, kind=W.OPACITY_POWER),
                     dict(strip_width=8, prefetch_rows=4, groups_per_warp=1)),
    "single_cell": (dict(nx=1, ny=1, G=3, npol=1, naz=2, T_bdr=(1.0, 0.3, 0.5, 0.7)),
                    dict(strip_width=4, prefetch_rows=2, groups_per_warp=1)),
    "steady_allsides": (dict(nx=9, ny=14, G=4, npol=2, naz=4, dt=0.0,
                             T_bdr=(1.0, 0.5, 0.25, 0.8)),
                        dict(strip_width=5, prefetch_rows=6, groups_per_warp=2)),
}

CASES_1D = {
    "marshak_s8": (dict(nx=200, ny=1, G=1, npol=8, kind=W.OPACITY_POWER), dict()),
    "mg_s6_gw2": (dict(nx=53, ny=1, G=11, npol=6, T_bdr=(1.0, 0.4, 0, 0)),
                  dict(groups_per_warp=2)),
}


def _check_all(case, precision, label):
    rtol = TOL[precision]
    Ig, mg, cg, _ = run_gpu(case)
    ref = run_oracle(case)
    e = parity_errors(case.cfg, (Ig, mg, cg), ref, precision, rtol)
    print(f"[{label} fp{precision}] " + "  ".join(f"{k} {v:.2e}" for k, v in e.items()) +
          f"  ({case.prob.info['n_tasks']} tasks, {case.prob.info['n_strips']} strips)")
    bad = {k: v for k, v in e.items() if not v <= rtol}
    assert not bad, f"parity above {rtol}: {bad}"
    return Ig


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(CASES_2D))
def test_sweep_2d_parity(gpu_lib, name, precision):
    ck, tk = CASES_2D[name]
    cfg = config(2, **ck)
    case = build_case(gpu_lib, cfg, precision, seed=sum(map(ord, name)) % 1000, **tk)
    _check_all(case, precision, name)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(CASES_1D))
def test_sweep_1d_parity(gpu_lib, name, precision):
    ck, tk = CASES_1D[name]
    cfg = config(1, **ck)
    case = build_case(gpu_lib, cfg, precision, seed=5, **tk)
    _check_all(case, precision, name)


@pytest.mark.parametrize("precision", [64, 32])
def test_no_previous_intensity(gpu_lib, precision):
    cfg = config(2, 20, 12, 3, 2, 4)
    case = build_case(gpu_lib, cfg, precision, seed=9, with_prev=False, strip_width=8,
                      prefetch_rows=2)
    _check_all(case, precision, "no_prev")


def test_quadrature_matches_oracle(gpu_lib):
    for dim, npol, naz in [(1, 8, 0), (1, 6, 0), (2, 4, 8), (2, 2, 3), (2, 4, 16)]:
        cfg = config(dim, 8, 8, 2, npol, naz)
        prob = gpu_lib.Problem.from_config(cfg, 64)
        ox, oy, w = prob.quadrature()
        rx, ry, rw = O.quadrature(dim, npol, naz)
        assert np.max(np.abs(ox - rx)) < 1e-15
        assert np.max(np.abs(oy - ry)) < 1e-15
        assert np.max(np.abs(w - rw)) < 1e-14
        assert abs(prob.info["alpha"] - O.alpha(rx, rw)) < 1e-15


@pytest.mark.parametrize("kind", [W.OPACITY_POWER, W.OPACITY_LARSEN])
def test_opacity_matches_oracle(gpu_lib, kind):
    import torch
    cfg = config(2, 19, 7, 9, 2, 2, kind=kind)
    prob = gpu_lib.Problem.from_config(cfg, 64)
    T = W.temperature_random(cfg.n_cells, 4, seed=2)
    s = W.scale_field(cfg, seed=3)
    ref = O.opacity(kind, cfg.opacity_alpha, cfg.edges, T, s)
    got = prob.opacity(torch.from_numpy(T).cuda(), torch.from_numpy(s).cuda()).cpu().numpy()
    prob.synchronize()
    assert rel_err(got, ref, 0.0) < 1e-13


@pytest.mark.parametrize("G", [1, 7, 64])
def test_emission_matches_oracle(gpu_lib, G):
    import torch
    cfg = config(2, 13, 11, G, 1, 1)
    prob = gpu_lib.Problem.from_config(cfg, 64)
    T = W.temperature_random(cfg.n_cells, 4, seed=G, lo=0.01, hi=3.0)
    sig = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, np.ones(cfg.n_cells))
    ref = O.emission(cfg.edges, cfg.a, cfg.c, T, sig)
    got = prob.emission(torch.from_numpy(T).cuda(), torch.from_numpy(sig).cuda()).cpu().numpy()
    prob.synchronize()
    e = rel_err(got, ref, 1e-300)
    print(f"emission G={G}: {e:.3e}")
    assert e < 1e-12


def test_emission_at_branch_boundaries(gpu_lib):
    """Nodal temperatures that put one group edge at each switch of the GPU's
    Planck evaluation (head series / Taylor tables / tail series / one-term
    tail / underflow), just below, on and just above it: every group of every
    node against the oracle, elementwise."""
    import torch
    G = 24
    cfg = config(2, 8, 6, G, 1, 1)
    edges = cfg.edges
    xs = [0.5, 0.9999, 1.0, 1.0001, 1.06, 1.9999, 2.0, 2.0001, 11.98, 12.0, 12.03, 36.9999,
          37.0, 37.0001, 100.0, 700.0, 744.0, 746.0]
    rng = np.random.default_rng(5)
    T = np.empty((cfg.n_cells, 4))
    for i in range(T.size):
        x = xs[i % len(xs)]
        e = edges[1 + rng.integers(0, G - 1)]   # an interior edge
        T.flat[i] = e / x
    T = np.clip(T, 1e-3, 1e3)
    prob = gpu_lib.Problem.from_config(cfg, 64)
    sig = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, np.ones(cfg.n_cells))
    ref = O.emission(cfg.edges, cfg.a, cfg.c, T, sig)
    got = prob.emission(torch.from_numpy(T).cuda(), torch.from_numpy(sig).cuda()).cpu().numpy()
    prob.synchronize()
    # relative per element; values below the normal FP64 range (the last
    # groups before the underflow) are compared against a 1e-280 floor
    e = float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-280)))
    print(f"emission at branch switches: {e:.3e}")
    assert e < 1e-12


def test_tiling_does_not_change_intensity(gpu_lib):
    """The per-(d,g) arithmetic is independent of the strip width and of the
    warps per CTA: the intensity is bitwise identical, moments agree to the
    reassociation of their sums."""
    cfg = config(2, 40, 23, 8, 4, 8)
    case = build_case(gpu_lib, cfg, 32, seed=4, strip_width=8, prefetch_rows=2, groups_per_warp=2)
    I1, m1, _, _ = run_gpu(case)
    for sw, pr in [(1, 2), (16, 4), (5, 8)]:
        case.prob.set_tiling(sw, pr)
        I2, m2, _, _ = run_gpu(case)
        assert np.array_equal(I1, I2)
        assert rel_err(m2[..., 0], m1[..., 0], 1e-6) < 1e-6


def test_sweep_host_matches_device(gpu_lib):
    import torch
    cfg = config(2, 21, 17, 6, 2, 4)
    case = build_case(gpu_lib, cfg, 32, seed=8, strip_width=8, prefetch_rows=2)
    Ig, mg, cg, _ = run_gpu(case)
    prob = case.prob
    Ip = prob.pack(torch.from_numpy(case.I_prev).cuda())
    Io = prob.empty_intensity()
    mh = np.zeros((cfg.n_cells, 4, 9))
    ch = np.zeros((cfg.n_cells, 4, 11))
    prob.sweep_host(np.ascontiguousarray(case.T), np.ascontiguousarray(case.sigma), Ip, Io, mh, ch)
    # moments are summed with atomics: equal up to the order of the additions
    assert rel_err(mh[..., 0], mg[..., 0], 1e-6) < 1e-6
    assert rel_err(ch[..., 0], cg[..., 0], 1e-6) < 1e-6
    assert np.array_equal(prob.unpack(Io).cpu().numpy(), Ig)


def test_pack_unpack_roundtrip(gpu_lib):
    import torch
    for prec in (32, 64):
        cfg = config(2, 9, 5, 5, 2, 3)
        prob = gpu_lib.Problem.from_config(cfg, prec, groups_per_warp=2)
        I = W.intensity_random(cfg.n_dir, cfg.n_groups, cfg.n_cells, 4, seed=1)
        back = prob.unpack(prob.pack(torch.from_numpy(I).cuda())).cpu().numpy()
        if prec == 64:
            assert np.array_equal(back, I)
        else:
            assert np.array_equal(back, I.astype(np.float32).astype(np.float64))


def test_autotune_keeps_results(gpu_lib):
    import torch
    cfg = config(2, 48, 40, 8, 4, 8)
    case = build_case(gpu_lib, cfg, 32, seed=6)
    I1, m1, _, _ = run_gpu(case)
    prob = case.prob
    Td = torch.from_numpy(case.T).cuda()
    Sd = torch.from_numpy(case.sigma).cuda()
    Ip = prob.pack(torch.from_numpy(case.I_prev).cuda())
    prob.autotune(Td, Sd, Ip, prob.empty_intensity(), reps=1)
    I2, m2, _, _ = run_gpu(case)
    assert np.array_equal(I1, I2)
    assert rel_err(m2[..., 0], m1[..., 0], 1e-6) < 1e-6


def test_launch_count_and_kernel_times(gpu_lib):
    cfg = config(2, 16, 16, 4, 2, 2)
    case = build_case(gpu_lib, cfg, 32, seed=2)
    n0 = case.prob.launch_count()
    case.prob.set_profiling(True)
    run_gpu(case)
    t = case.prob.kernel_times()
    assert t["count"] == 1 and t["sweep_ms"] > 0
    assert case.prob.launch_count() - n0 >= 3


def test_exp_neg_matches_cuda_exp(gpu_lib):
    """The emission kernels' table-driven e^{-x} (Tang's method, a 2^{-j/64}
    table and a degree-6 polynomial) against CUDA's exp over [0, 708): two
    million uniform and log-uniform points, the table's reduction knots
    k ln2/64 with their floating-point neighbours, and the ends.  Both are
    within about an ulp of e^{-x}, so they differ by at most 2 ulp (and each
    stays within 2 ulp of the host's exp)."""
    import ctypes
    import torch
    rng = np.random.default_rng(708)
    knots = np.arange(0, int(708 * 64 / np.log(2))) * (np.log(2) / 64)
    x = np.concatenate([rng.uniform(0.0, 708.0, 1 << 20),
                        np.exp(rng.uniform(np.log(1e-300), np.log(708.0), 1 << 20)),
                        knots, np.nextafter(knots, 0.0), np.nextafter(knots, 708.0),
                        [0.0, 5e-324, 1e-300, 1e-16, 0.5, 1.0, np.nextafter(708.0, 0.0)]])
    x = x[(x >= 0.0) & (x < 708.0)]
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    lib = gpu_lib.load()
    rc = lib.sm_debug_exp_neg(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                              int(x.size), None)
    assert rc == 0, lib.sm_last_error().decode()
    ref = torch.exp(-xd)                       # CUDA's exp
    torch.cuda.synchronize()
    got, ref = out.cpu().numpy(), ref.cpu().numpy()
    ulp = np.spacing(np.abs(ref))
    e_cuda = float(np.max(np.abs(got - ref) / ulp))
    host = np.exp(-x)
    e_host = float(np.max(np.abs(got - host) / np.spacing(np.abs(host))))
    print(f"exp_neg over {x.size} points: {e_cuda:.2f} ulp from CUDA exp, {e_host:.2f} ulp "
          f"from the host's exp")
    assert e_cuda <= 2.0 and e_host <= 2.0


FUSED = {
    # name: (config kwargs, tiling kwargs, fused emission warps)
    "ragged_lanes": (dict(nx=37, ny=21, G=5, npol=2, naz=3),
                     dict(strip_width=8, prefetch_rows=2, groups_per_warp=1), 2),
    "gw4_dirblocks": (dict(nx=17, ny=9, G=6, npol=4, naz=16),
                      dict(strip_width=3, prefetch_rows=3, groups_per_warp=4), 4),
    "gray_channel": (dict(nx=32, ny=32, G=1, npol=4, naz=8, kind=W.OPACITY_POWER),
                     dict(strip_width=14, prefetch_rows=2, groups_per_warp=1), 2),
    "steady_allsides": (dict(nx=9, ny=14, G=4, npol=2, naz=4, dt=0.0,
                             T_bdr=(1.0, 0.5, 0.25, 0.8)),
                        dict(strip_width=5, prefetch_rows=6, groups_per_warp=2), 1),
    "many_groups": (dict(nx=29, ny=40, G=64, npol=4, naz=8),
                    dict(strip_width=12, prefetch_rows=2, groups_per_warp=4), 2),
}


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(FUSED))
def test_fused_emission_parity(gpu_lib, name, precision):
    """The emission computed inside the sweep kernel (sm_set_emission_warps:
    extra warps per CTA, sweep warps helping while their strip is not ready)
    against the oracle, with ragged strips, padded lanes and groups, and the
    same pass with the emission as its own kernel: intensities within 1e-6
    (FP32, the source records rounded alike) / 1e-13 (FP64) of each other."""
    ck, tk, warps = FUSED[name]
    cfg = config(2, **ck)
    case = build_case(gpu_lib, cfg, precision, seed=sum(map(ord, name)) % 1000 + 17, **tk)
    I_sep, _, _, _ = run_gpu(case)
    case.prob.set_emission_warps(warps)
    assert case.prob.info["emission_warps"] == warps
    Ig = _check_all(case, precision, f"{name} fused x{warps}")
    same = float(np.max(np.abs(Ig - I_sep)) / np.abs(I_sep).max())
    print(f"  fused vs separate emission: {same:.2e}")
    assert same <= (1e-6 if precision == 32 else 1e-13)


TAIL = {
    # name: (config kwargs, tiling kwargs, tail strips at each end)
    "w8_tail1": (dict(nx=40, ny=23, G=8, npol=4, naz=8),
                 dict(strip_width=8, prefetch_rows=2, groups_per_warp=2), 1),
    "w8_tail2_ragged": (dict(nx=37, ny=19, G=5, npol=2, naz=3),
                        dict(strip_width=8, prefetch_rows=3, groups_per_warp=1), 2),
    "w12_tail2_many_groups": (dict(nx=70, ny=31, G=64, npol=4, naz=8),
                              dict(strip_width=12, prefetch_rows=2, groups_per_warp=4), 2),
    "w2_tail1_gray": (dict(nx=9, ny=12, G=1, npol=4, naz=8, kind=W.OPACITY_POWER),
                      dict(strip_width=2, prefetch_rows=2, groups_per_warp=1), 1),
}


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(TAIL))
def test_tail_strips_parity(gpu_lib, name, precision):
    """Half-width strips at both ends of the x range (sm_set_tail_strips),
    with ragged middle strips and one-column strips: every output against
    the oracle, and the intensity bit for bit equal to the uniform layout's
    (the per-(d,g) arithmetic does not depend on the strips), the moments
    within 1e-15 (FP64) / 1e-6 (FP32) of it."""
    ck, tk, tail = TAIL[name]
    cfg = config(2, **ck)
    case = build_case(gpu_lib, cfg, precision, seed=sum(map(ord, name)) % 1000 + 29, **tk)
    I_u, m_u, _, _ = run_gpu(case)
    ns_u = case.prob.info["n_strips"]
    case.prob.set_tail_strips(tail)
    info = case.prob.info
    assert info["tail_strips"] == tail
    W_ = tk["strip_width"]
    mid = cfg.nx - tail * W_
    assert info["n_strips"] == 2 * tail + (mid + W_ - 1) // W_
    Ig = _check_all(case, precision, f"{name} tail {tail}")
    _, m_t, _, _ = run_gpu(case)
    assert np.array_equal(Ig, I_u)
    assert rel_err(m_t[..., 0], m_u[..., 0], 1e-12) <= (1e-15 if precision == 64 else 1e-6)
    print(f"  strips {ns_u} -> {info['n_strips']}")


def test_tail_strips_fall_back_and_refuse_fused_emission(gpu_lib):
    """A layout that does not exist (odd strip width, or no full-width strip
    left in between) falls back to uniform strips; tail strips and fused
    emission warps exclude each other."""
    sm = gpu_lib
    cfg = config(2, 12, 8, 4, 2, 4)
    case = build_case(gpu_lib, cfg, 32, seed=3, strip_width=5, prefetch_rows=2, groups_per_warp=1)
    case.prob.set_tail_strips(1)  # odd width
    assert case.prob.info["tail_strips"] == 0
    case.prob.set_tiling(8, 2)
    case.prob.set_tail_strips(2)  # 12 - 2 * 8 < 8: nothing in between
    assert case.prob.info["tail_strips"] == 0
    case.prob.set_tail_strips(1)  # [4, 8 ragged to 4, 4]: 12 - 8 = 4 < 8 -> falls back too
    assert case.prob.info["tail_strips"] == 0
    case.prob.set_tiling(4, 2)
    case.prob.set_tail_strips(1)  # [2, 4, 4, 2]
    assert case.prob.info["tail_strips"] == 1 and case.prob.info["n_strips"] == 4
    with pytest.raises(sm.SMError):
        case.prob.set_emission_warps(2)
    case.prob.set_tail_strips(0)
    case.prob.set_emission_warps(2)
    with pytest.raises(sm.SMError):
        case.prob.set_tail_strips(1)


def _branch_temperatures(edges, n, seed):
    """Nodal temperatures that put one group edge at each switch of the Planck
    evaluation (head series / Taylor tables / tail series / one-term tail /
    FP32 range / FP64 underflow), just below, on and just above it."""
    xs = [0.5, 0.9999, 1.0, 1.0001, 1.06, 1.9999, 2.0, 2.0001, 11.98, 12.0, 12.03, 36.9999,
          37.0, 37.0001, 86.99, 87.0, 87.01, 100.0, 700.0, 746.0]
    rng = np.random.default_rng(seed)
    G = len(edges) - 1
    T = np.empty(n)
    for i in range(n):
        T[i] = edges[1 + rng.integers(0, G - 1)] / xs[i % len(xs)]
    return np.clip(T, 1e-3, 1e3)


@pytest.mark.parametrize("case_name", ["larsen64_wave", "branch_switches"])
def test_double_fp32_emission_matches_fp64(gpu_lib, case_name):
    """The FP32-sweep path's emission in double-FP32 arithmetic against the
    FP64 evaluation (sm_debug_set_emission_fp64) inside the same sweep: the
    intensities (whose source records are FP32 either way) within 2e-7 of each
    other per (direction, group) slice, and the nodal Planck and Rosseland numerators
    (closure fields sigma_F, sigma_P, FP64) within 1e-13, on a multigroup
    temperature wave and on temperatures that put group edges at every switch
    of the series."""
    import torch
    if case_name == "larsen64_wave":
        cfg = config(2, 21, 17, 64, 2, 4)
        case = build_case(gpu_lib, cfg, 32, seed=11, strip_width=8, prefetch_rows=2)
    else:
        cfg = config(2, 12, 10, 24, 2, 4)
        case = build_case(gpu_lib, cfg, 32, seed=12, strip_width=6, prefetch_rows=2)
        case.T = _branch_temperatures(cfg.edges, cfg.n_cells * 4, 5).reshape(cfg.n_cells, 4)
        case.sigma = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, case.T,
                               case.scale)
    I_df, m_df, c_df, _ = run_gpu(case)
    case.prob.set_emission_fp64(True)
    I_64, m_64, c_64, _ = run_gpu(case)
    case.prob.set_emission_fp64(False)
    red = (2, 3)  # per (direction, group): cells x nodes
    dI = float(np.max(np.abs(I_df - I_64).max(axis=red) /
                      np.maximum(np.abs(I_64).max(axis=red), 1e-300)))
    d_num = max(rel_err(c_df[..., k], c_64[..., k], 0.0) for k in (7, 8))
    print(f"{case_name}: intensity {dI:.2e}, Planck / Rosseland numerators {d_num:.2e}")
    assert dI <= 2e-7
    assert d_num <= 1e-13
