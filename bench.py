"""Benchmark of the SM hot path (rows a1-a4: emission, sweep, fused moments,
closures) on the 2D multigroup workload: 256x256 cells, 128 directions,
64 groups, FP32 sweep arithmetic; the Planck group integrals of the FP32
path in double-FP32 arithmetic (about 48 bits; the FP64 path's in FP64); the
moment sums compensated and finished in FP64.

Prints one JSON line (rank 0).  Metric: cell-direction-group updates/s of
whole hot-path passes, with the intensity resident in HBM (inputs far larger
than L2: 8.6 GB per intensity copy, so no L2 flush is needed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun; the
single-GPU method has no exchange step), timed with a barrier on both sides
and the maximum over ranks.  --impl reference times the FP64 CPU oracle on
the host cores instead (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_FP32 = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiling", default="",
                    help="W,S,E,T: strip width, prefetch rows, fused emission warps and tail "
                         "strips of the main line, set instead of autotuning (profiling runs "
                         "that must not spend launches on the autotuner)")
    ap.add_argument("--groups-per-warp", type=int, default=0,
                    help="(d,g) slots per lane of the main line's problem (0: the library's "
                         "automatic choice; a profiling case otherwise)")
    ap.add_argument("--workload", default="multigroup2d",
                    choices=["multigroup2d", "adjoint2d", "graychannel2d"],
                    help="problem of the main line: the 256^2 x 128 x 64 multigroup workload "
                         "(default), the 128^2 x 64 x 16 adjoint-size problem or the 128^2 x "
                         "128 gray channel (profiling cases; the extra metrics are skipped)")
    ap.add_argument("--nx", type=int, default=0, help="override cells per axis (profiling cases)")
    ap.add_argument("--groups", type=int, default=0, help="override the group count")
    ap.add_argument("--no-step-metric", action="store_true",
                    help="skip the seconds-per-converged-step comparison (FP32 vs FP64 sweep)")
    ap.add_argument("--step-steps", type=int, default=3,
                    help="time steps timed per path in the step comparison (after 1 warm-up step)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched 64-problem measurement")
    ap.add_argument("--no-config-sweeps", action="store_true",
                    help="skip the per-configuration sweep rates (1D slab, gray channel, "
                         "adjoint-size problem)")
    ap.add_argument("--adjoint-fd-cells", type=int, default=32,
                    help="cells of the warm-start adjoint finite-difference check "
                         "(0: skip the adjoint)")
    ap.add_argument("--adjoint-cold-fd-cells", type=int, default=4,
                    help="cells of the configured-start adjoint finite-difference check")
    return ap.parse_args()


def workload(args):
    from paper_2504_21784_gb300 import workloads as W
    cfg = {"multigroup2d": W.multigroup_2d, "adjoint2d": W.adjoint_2d,
           "graychannel2d": W.gray_channel_2d}[args.workload]()
    if args.nx or args.groups:
        cfg = cfg.resized(args.nx or cfg.nx, n_groups=args.groups or None)
        cfg.name = f"{args.workload}_{cfg.nx}x{cfg.ny}x{cfg.n_dir}x{cfg.n_groups}"
    return cfg


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest x over the ranks (x itself without a process group): the
    timed region of a replicated run ends when its slowest rank does."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each process
    units_per_rank units in `seconds` (the max over ranks): weak scaling."""
    return world * units_per_rank / seconds


def algorithmic_bytes(cfg, prec: int) -> dict:
    """Minimal HBM traffic of one sweep-kernel launch: read I^k and write I
    (4 nodes each per update), read the emission (4 nodes) and sigma~, sigma
    once per (cell, group), write the 36 per-cell moment sums once."""
    rs = prec // 8
    upd = cfg.updates
    per_update = 2 * 4 * rs
    src = cfg.n_cells * cfg.n_groups * (4 + 2) * rs
    mom = cfg.n_cells * 36 * rs
    total = upd * per_update + src + mom
    return {"per_update": total / upd, "per_launch": total, "updates": upd}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(prec: int, cfg=None):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"sweep2d_multigroup2d_fp{prec}_traffic.txt")
    src = os.path.join(ROOT, "paper_2504_21784_gb300", "csrc", "sm_sweep.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("sm_sweep_cu_sha256") != h:
        return None
    if cfg is not None and rec.get("workload") not in (None, cfg.name):
        return None
    return rec.get("dram_bytes_per_launch")


def oracle_pass(cfg, n_dirs: int, seed: int = 0, nthreads: int = 0):
    """One bounded hot-path pass of the FP64 oracle, as it stands: emission
    (a1) and closures (a4) on the whole mesh, the sweep (a2) and moments (a3)
    of n_dirs randomly drawn directions with all their groups.  Returns the
    wall time of each part."""
    import numpy as np
    import oracle as O
    from paper_2504_21784_gb300 import workloads as W
    T = W.temperature_wave(cfg)
    s = W.scale_field(cfg)
    sig = O.opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T, s)
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    inv = 1.0 / (cfg.c * cfg.dt)
    dirs = np.sort(np.random.default_rng(seed).choice(cfg.n_dir, n_dirs, replace=False))
    G = cfg.n_groups
    t = {}
    t0 = time.perf_counter()
    q = O.emission(cfg.edges, cfg.a, cfg.c, T, sig)
    t1 = time.perf_counter()
    I = O.sweep_pairs(2, cfg.nx, cfg.ny, cfg.extent, omx, omy, sig, inv, q, None, infl,
                      [(int(d), g) for d in dirs for g in range(G)], nthreads=nthreads)
    t2 = time.perf_counter()
    I = I.reshape(len(dirs), G, cfg.n_cells, 4)
    mom = O.moments(2, omx[dirs], omy[dirs], w[dirs], sig, I)
    t3 = time.perf_counter()
    O.closures(2, cfg.edges, cfg.c, sig, T, mom)
    t4 = time.perf_counter()
    t = {"emission": t1 - t0, "sweep": t2 - t1, "moments": t3 - t2, "closures": t4 - t3}
    return t, len(dirs) * G * cfg.n_cells


def oracle_sample_dirs(cfg, budget_s: float) -> int:
    """Directions per bounded oracle pass so that the pass takes about
    budget_s on this host (a calibration pass of two directions)."""
    t, _ = oracle_pass(cfg, 2, seed=99)
    fixed = t["emission"] + t["closures"]
    per_dir = (t["sweep"] + t["moments"]) / 2
    return int(min(cfg.n_dir, max(2, (budget_s - fixed) / max(per_dir, 1e-4))))


def oracle_summary(cfg, n_dirs: int, times: list, upd: int, cores: int) -> dict:
    """Rate of what ran (the sampled updates over the pass's wall time, the
    whole-mesh emission and closures included), and, stated separately, the
    full pass extrapolated by scaling the sweep and moments to all directions."""
    mean = {k: statistics.mean(t[k] for t in times) for k in times[0]}
    wall = sum(mean.values())
    full = mean["emission"] + mean["closures"] + (mean["sweep"] + mean["moments"]) * \
        cfg.n_dir / n_dirs
    return {"value": upd / wall, "unit": "cell-dir-group updates/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{len(times)} pass(es): emission and closures on the whole "
                      f"{cfg.nx}x{cfg.ny} mesh, sweep and moments of {n_dirs} of {cfg.n_dir} "
                      f"directions x {cfg.n_groups} groups ({upd} updates), "
                      f"{wall:.2f} s per pass, FP64, OpenMP over (direction, group)",
            "s_per_pass": wall, "parts_s": mean,
            "extrapolated_full_pass_s": full,
            "extrapolated_full_pass_rate": cfg.updates / full}


def cpu_baseline(cfg, budget_s: float = 6.0, passes: int = 3):
    """The FP64 oracle, as it stands, on the host cores: `passes` bounded
    a1-a4 passes of the same workload (about budget_s each)."""
    import oracle as O
    n_dirs = oracle_sample_dirs(cfg, budget_s)
    times = []
    for i in range(passes):
        t, upd = oracle_pass(cfg, n_dirs, seed=i)
        times.append(t)
    out = oracle_summary(cfg, n_dirs, times, upd, O.num_threads())
    t1, u1 = oracle_pass(cfg, 1, seed=7, nthreads=1)
    out["value_one_thread_sweep"] = u1 / t1["sweep"]
    return out


def converged_steps(sm, W, cfg, prec: int, n_steps: int, stream, autotune: bool = True,
                    method: int = 0, refine: bool = False, groups_per_warp: int = 0):
    """Seconds per converged time step (Algorithm 1 through sm_step) from the
    equilibrium initial state T = T0, I = B_g(T0)/4pi (whose moments are
    phi = a c T0^4, F = 0), with the paper's iteration controls.  One
    warm-up step (allocates the low-order workspace), then n_steps timed
    steps of the same evolution.  sm_step synchronizes internally, so the
    host clock brackets the device work.  refine: the FP32 sweeps with FP64
    defect correction (an FP64-state problem, sm_step_params.refine = 1).
    groups_per_warp: the problem's slots per lane (0: the library's rule)."""
    import torch
    with torch.cuda.stream(stream):
        prob = sm.Problem.from_config(cfg, prec, stream=stream, groups_per_warp=groups_per_warp)
        nc, nn = cfg.n_cells, cfg.n_nodes
        T = torch.full((nc, nn), cfg.T0, dtype=torch.float64, device="cuda")
        scale = torch.from_numpy(W.scale_field(cfg)).cuda()
        cv = torch.full((nc, nn), cfg.cv, dtype=torch.float64, device="cuda")
        ones = torch.ones((cfg.n_groups, nc), dtype=torch.float64, device="cuda")
        b = prob.emission(T, ones)  # unit opacity: B_g(T0)/4pi per node
        I = [prob.pack(b.unsqueeze(0).expand(cfg.n_dir, -1, -1, -1).contiguous()),
             prob.empty_intensity()]
        del b, ones
        mom = prob.new_moments()
        mom.zero_()
        mom[..., 0] = cfg.a * cfg.c * cfg.T0 ** 4
        E, F = prob.new_nodal(), prob.new_flux()
        if autotune:
            sigma = prob.opacity(T, scale)
            prob.autotune(T, sigma, I[0], I[1], reps=2)
            del sigma
        secs, stats = [], []
        for k in range(1 + n_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = prob.step(scale, cv, T, E, F, mom, I[k % 2], I[(k + 1) % 2],
                           params=sm.step_params(method=method, refine=1 if refine else 0))
            torch.cuda.synchronize()
            if k >= 1:
                secs.append(time.perf_counter() - t0)
                stats.append(st)
        out = {"s_per_step": sum(secs) / len(secs),
               "outer_iters": [s["outer_iters"] for s in stats],
               "newton_iters": [s["newton_iters_total"] for s in stats],
               "pcg_iters": [s["pcg_iters_total"] for s in stats],
               "pcg_capped": sum(s["pcg_capped"] for s in stats),
               "converged": all(s["converged"] for s in stats),
               "tiling": {k: prob.info[k] for k in ("strip_width", "prefetch_rows",
                                                    "groups_per_warp")}}
        if refine:
            out["refine_corrections"] = [s["refine_corrections"] for s in stats]
        Tn = T.cpu().numpy()
        prob.close()
        return out, Tn


def config_sweeps(sm, W, stream, reps: int = 20):
    """Metric 1 on the other single-problem configurations: whole hot-path
    passes (emission + sweep with fused moments + reduction/closures) on the
    1D Marshak slab, the 2D gray channel and the adjoint-size problem, FP32
    and FP64 sweeps, autotuned tiling, one step of history as I^k; updates/s
    of the pass and the sweep kernel's share of the measured copy bandwidth
    (the 1D slab has 1,600 updates per sweep: latency-bound by nature)."""
    import torch
    peak, _ = measured_peaks()
    out = {}
    for cfg in (W.marshak_1d(), W.gray_channel_2d(), W.adjoint_2d()):
        res = {}
        for prec in (32, 64):
            with torch.cuda.stream(stream):
                prob = sm.Problem.from_config(cfg, prec, stream=stream)
                T = torch.from_numpy(W.temperature_wave(cfg)).cuda()
                sigma = prob.opacity(T, torch.from_numpy(W.scale_field(cfg)).cuda())
                I = [prob.empty_intensity(), prob.empty_intensity()]
                mom, clo = prob.new_moments(), prob.new_closures()
                prob.sweep(T, sigma, None, I[0], mom, clo)
                if cfg.dim == 2:
                    prob.autotune(T, sigma, I[0], I[1], reps=2)
                for i in range(3):
                    prob.sweep(T, sigma, I[i % 2], I[(i + 1) % 2], mom, clo)
                prob.synchronize()
                prob.set_profiling(True)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                for i in range(reps):
                    prob.sweep(T, sigma, I[i % 2], I[(i + 1) % 2], mom, clo)
                ev1.record(stream)
                ev1.synchronize()
                prob.synchronize()
                kt = prob.kernel_times()
                prob.set_profiling(False)
                ms = ev0.elapsed_time(ev1) / reps
                sweep_ms = kt["sweep_ms"] / max(kt["count"], 1)
                alg = algorithmic_bytes(cfg, prec) if cfg.dim == 2 else None
                r = {"updates_per_s": cfg.updates / (ms * 1e-3), "ms_per_pass": ms,
                     "sweep_ms": sweep_ms}
                if alg is not None:
                    r["sweep_hbm_frac"] = alg["per_launch"] / (sweep_ms * 1e-3) / 1e9 / peak
                    r["tiling"] = {k: prob.info[k] for k in ("strip_width", "prefetch_rows",
                                                             "groups_per_warp", "tail_strips",
                                                             "emission_warps")}
                res[f"fp{prec}"] = r
                prob.close()
        out[cfg.name] = res
    torch.cuda.empty_cache()
    return out


def marshak_paper_metric(sm, W, stream):
    """The Marshak wave in the paper's units (64 cells, S6, 312 steps of
    8e-12 s to 2.5 ns) through sm_step with the paper's iteration controls:
    wall time of the whole run per closure method and sweep precision, the
    outer iterations, and the wave-front position (first cell-mean T below
    500 eV)."""
    import numpy as np
    import torch
    cfg = W.marshak_paper()
    n = cfg.n_cells
    out = {"workload": f"{cfg.name}, {cfg.steps} steps of {cfg.dt:.0e} s"}
    for method, code in (("independent", sm.METHOD_INDEPENDENT),
                         ("consistent", sm.METHOD_CONSISTENT)):
        for prec in (32, 64):
            with torch.cuda.stream(stream):
                prob = sm.Problem.from_config(cfg, prec, stream=stream)
                T = torch.full((n, 2), cfg.T0, dtype=torch.float64, device="cuda")
                scale = torch.from_numpy(W.scale_field(cfg)).cuda()
                cv = torch.full((n, 2), cfg.cv, dtype=torch.float64, device="cuda")
                ones = torch.ones((cfg.n_groups, n), dtype=torch.float64, device="cuda")
                b = prob.emission(T, ones)  # B(T0)/4pi per node: the equilibrium start
                Ip = prob.pack(b.unsqueeze(0).expand(cfg.n_dir, -1, -1, -1).contiguous())
                mom = prob.new_moments()
                mom.zero_()
                mom[..., 0] = cfg.a * cfg.c * cfg.T0 ** 4
                E, F = prob.new_nodal(), prob.new_flux()
                prm = sm.step_params(method=code)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                outer = 0
                for _ in range(cfg.steps):
                    In = prob.empty_intensity()
                    outer += prob.step(scale, cv, T, E, F, mom, Ip, In, params=prm)["outer_iters"]
                    Ip = In
                torch.cuda.synchronize()
                secs = time.perf_counter() - t0
                Tm = T.cpu().numpy().mean(axis=1)
                hot = Tm > 500.0
                k = int(np.argmin(hot)) if not hot.all() else n
                out[f"{method}_fp{prec}"] = {"s": secs, "outer_iters": outer,
                                             "front_cm": k * 0.05 / n}
                prob.close()
    return out


def step_metric(sm, W, cfgs, n_steps: int, stream):
    """Metric 2: FP32 vs FP64 sweep path, seconds per converged step, with
    the FP32 path's temperature error against the FP64 path after the same
    steps (max |dT| / max |T|)."""
    import numpy as np
    res = {}
    for cfg in cfgs:
        r32, T32 = converged_steps(sm, W, cfg, 32, n_steps, stream)
        r64, T64 = converged_steps(sm, W, cfg, 64, n_steps, stream)
        c32, Tc32 = converged_steps(sm, W, cfg, 32, n_steps, stream, method=sm.METHOD_CONSISTENT)
        # every sweep of the refined path is an FP32 correction sweep, so its
        # FP64-state problem takes the FP32 path's slots per lane
        rr, Trr = converged_steps(sm, W, cfg, 64, n_steps, stream, refine=True,
                                  groups_per_warp=r32["tiling"]["groups_per_warp"])
        res[cfg.name] = {"fp32": r32, "fp64": r64,
                         "fp64_over_fp32_time": r64["s_per_step"] / r32["s_per_step"],
                         "fp32_vs_fp64_T_rel": float(np.abs(T32 - T64).max() / np.abs(T64).max()),
                         "fp32_refined": rr,
                         "fp64_over_refined_time": r64["s_per_step"] / rr["s_per_step"],
                         "refined_vs_fp64_T_rel":
                             float(np.abs(Trr - T64).max() / np.abs(T64).max()),
                         "consistent_fp32": c32,
                         "consistent_vs_independent_T_rel":
                             float(np.abs(Tc32 - T32).max() / np.abs(T32).max()),
                         "steps_timed": n_steps, "warmup_steps": 1,
                         "state": "equilibrium start T0 = %g, steps 2..%d" % (cfg.T0, n_steps + 1)}
    return res


def batched_metric(sm, W, stream, steps: int, warmup: int):
    """The 64-problem batched workload (uneven 32^2..256^2 meshes, 8-32
    groups, 32/64/128 directions, blocky two-material layouts), FP32 sweep:
    whole passes of sm_batch_sweep (prologue, emissions, ONE persistent
    sweep launch with fused moments, moment sums and closures; replayed from
    CUDA graphs, the two intensity buffers alternating) after autotuning the
    batch tiling; the batched sweep kernel's own time from live profiled
    passes (CUDA events) and its share of the measured HBM copy bandwidth;
    the same problems swept one after another through sm_sweep; and seconds
    per batched time step (sm_batch_step, FP32 sweep / FP64 low-order, the
    paper's iteration controls) from the equilibrium start."""
    import torch
    members = W.batched_2d()
    cfgs = [m.cfg for m in members]
    upd = float(sum(c.n_cells * c.n_dir * c.n_groups for c in cfgs))
    alg = sum(algorithmic_bytes(c, 32)["per_launch"] for c in cfgs)
    peak, peak_kind = measured_peaks()
    out = {"workload": "batched2d_64x(32..256)^2x(32..128)x(8..32)", "problems": len(cfgs),
           "updates_per_pass": upd}
    with torch.cuda.stream(stream):
        gw = sm.tune_batch_slots(cfgs, 32, reps=2, stream=stream)  # slots per lane
        b = sm.Batch(cfgs, 32, stream=stream, groups_per_warp=gw)
        out["slots_per_lane"] = {str(v): gw.count(v) for v in sorted(set(gw))}
        T, S, I0, I1, M, C = [], [], [], [], [], []
        for mem, h in zip(members, b.members):
            t = torch.from_numpy(W.temperature_wave(mem.cfg)).cuda()
            T.append(t)
            S.append(h.opacity(t, torch.from_numpy(mem.scale).cuda()))
            I0.append(h.empty_intensity())
            I1.append(h.empty_intensity())
            M.append(h.new_moments())
            C.append(h.new_closures())
        b.sweep(T, S, None, I0, M, C)
        b.synchronize()
        b.autotune(T, S, I0, I1, reps=1)
        bufs = [I0, I1]
        for i in range(warmup):
            b.sweep(T, S, bufs[i % 2], bufs[(i + 1) % 2], M, C)
        b.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(steps):
            b.sweep(T, S, bufs[i % 2], bufs[(i + 1) % 2], M, C)
        ev1.record(stream)
        ev1.synchronize()
        b.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        # the batched sweep kernel alone: live passes with events around it
        b.set_profiling(True)
        for i in range(steps):
            b.sweep(T, S, bufs[i % 2], bufs[(i + 1) % 2], M, C)
        kt = b.kernel_times()
        b.set_profiling(False)
        b.synchronize()
        sweep_ms = kt["sweep_ms"] / max(kt["count"], 1)
        achieved = alg / (sweep_ms * 1e-3) / 1e9
        info = b.info()
        out.update({"value": upd / (ms * 1e-3), "unit": "cell-dir-group updates/s",
                    "ms_per_pass": ms, "pass": "emission + batched sweep with fused moments + "
                    "moment sums and closures (graph replay)",
                    "kernel_ms": {"emission": kt["emission_ms"] / max(kt["count"], 1),
                                  "sweep": sweep_ms,
                                  "reduce_closures": kt["reduce_ms"] / max(kt["count"], 1)},
                    "roofline": {"bound": "hbm", "kernel": "sweep2d_batch_kernel",
                                 "achieved": achieved, "peak": peak, "unit": "GB/s",
                                 "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                                 "algorithmic_bytes": alg},
                    "tiling": {"strip_width": info["strip_width"],
                               "prefetch_rows": info["prefetch_rows"],
                               "resident_ctas": info["resident_ctas"],
                               "queue_items": info["n_tasks"]},
                    "launches_per_pass": 2 + 2 * len(cfgs), "graph": "replayed"})
        del I1
        # the same problems one after another (single-problem sweeps)
        probs = [sm.Problem.from_config(c, 32, stream=stream) for c in cfgs]
        Io = [p.empty_intensity() for p in probs]
        for p, t, s_, io, m_, c_ in zip(probs, T, S, Io, M, C):
            p.sweep(t, s_, None, io, m_, c_)
        torch.cuda.synchronize()
        reps = max(1, steps // 2)
        ev0.record(stream)
        for _ in range(reps):
            for p, t, s_, io, m_, c_ in zip(probs, T, S, Io, M, C):
                p.sweep(t, s_, None, io, m_, c_)
        ev1.record(stream)
        ev1.synchronize()
        ms_seq = ev0.elapsed_time(ev1) / reps
        out["sequential_ms_per_pass"] = ms_seq
        out["batched_speedup"] = ms_seq / ms
        for p in probs:
            p.close()
        del Io, M, C
        torch.cuda.empty_cache()
        out["step"] = batched_step_metric(sm, W, b, members, stream)
        b.close()
    torch.cuda.empty_cache()
    return out


def batched_step_metric(sm, W, b, members, stream, n_steps: int = 3):
    """Seconds per time step of all 64 members through sm_batch_step (FP32
    sweep, FP64 low-order, the paper's iteration controls) from the
    equilibrium start T = T0, I = B_g(T0)/4pi; one warm-up step, then
    n_steps timed steps.  The members' low-order solves run in one
    cooperative launch (the library's default); the same steps with one
    launch per member, from the same start, are timed beside it."""
    res, T1 = _batched_steps(W, b, members, n_steps)
    b.set_batched_lo(False)
    try:
        res["lo_one_launch_per_member"], T2 = _batched_steps(W, b, members, n_steps)
    finally:
        b.set_batched_lo(True)
    # the two launch forms solve the same systems (their grid sums differ in order)
    res["lo_forms_T_rel_diff"] = max(float((a - c).abs().max() / c.abs().max())
                                     for a, c in zip(T1, T2))
    return res


def _batched_steps(W, b, members, n_steps):
    import torch
    st = []
    for mem, h in zip(members, b.members):
        cfg = mem.cfg
        nc = cfg.n_cells
        T = torch.full((nc, 4), cfg.T0, dtype=torch.float64, device="cuda")
        ones = torch.ones((cfg.n_groups, nc), dtype=torch.float64, device="cuda")
        bq = h.emission(T, ones)  # unit opacity: B_g(T0)/4pi per node
        I = [h.pack(bq.unsqueeze(0).expand(cfg.n_dir, -1, -1, -1).contiguous()),
             h.empty_intensity()]
        mom = h.new_moments()
        mom.zero_()
        mom[..., 0] = cfg.a * cfg.c * cfg.T0 ** 4
        st.append(dict(scale=torch.from_numpy(mem.scale).cuda(),
                       cv=torch.full((nc, 4), cfg.cv, dtype=torch.float64, device="cuda"),
                       T=T, E=h.new_nodal(), F=h.new_flux(), mom=mom, I=I))
    secs, outer = [], []
    for k in range(1 + n_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = b.step([s["scale"] for s in st], [s["cv"] for s in st], [s["T"] for s in st],
                       [s["E"] for s in st], [s["F"] for s in st], [s["mom"] for s in st],
                       [s["I"][k % 2] for s in st], [s["I"][(k + 1) % 2] for s in st])
        torch.cuda.synchronize()
        if k >= 1:
            secs.append(time.perf_counter() - t0)
            outer.append(max(x["outer_iters"] for x in stats))
    return {"s_per_step": sum(secs) / len(secs), "members": len(st),
            "outer_iters_max_per_step": outer,
            "converged": all(x["converged"] for x in stats),
            "method": "sm_batch_step: FP32 sweep / FP64 low-order, paper controls",
            "state": "equilibrium start, steps 2..%d" % (n_steps + 1)}, [s["T"] for s in st]


def adjoint_metric(sm, W, fd_cells: int, warm: bool = False):
    """The adjoint workload (128^2 cells, 64 directions, 16 groups, 20
    backward-Euler steps, FP64, each step converged to 1e-13): wall time of
    the forward (with checkpoints every sqrt(20) steps) and of the backward
    (segment recomputation + adjoint steps), and central differences
    (h = 1e-4 s_K) of the time-integrated right-edge leakage on fd_cells
    cells drawn with seed 21784 from a set fixed before the gradient is
    known.  Warm start (T0 = 0.3): cells of the four columns next to the
    right edge, error per cell relative to its own sensitivity.  Configured
    start (T0 = 0.01): the leakage depends on a handful of edge cells only,
    so the cells come from the right-edge column and the error is stated
    relative to the largest sensitivity of all cells (most drawn cells have
    none, which the difference quotients must confirm)."""
    import numpy as np
    import torch
    from paper_2504_21784_gb300 import adjoint as A
    cfg = W.adjoint_2d_warm() if warm else W.adjoint_2d()
    cols = 4 if warm else 1
    band = np.array([iy * cfg.nx + ix for iy in range(cfg.ny)
                     for ix in range(cfg.nx - cols, cfg.nx)])
    cells = np.random.default_rng(21784).choice(band, min(fd_cells, band.size), replace=False)
    prob = sm.Problem.from_config(cfg, 64)
    T0 = torch.full((cfg.n_cells, 4), cfg.T0, dtype=torch.float64, device="cuda")
    cv = torch.full((cfg.n_cells, 4), cfg.cv, dtype=torch.float64, device="cuda")
    s = torch.from_numpy(W.scale_field(cfg)).cuda()
    st = A.LeakageSetup(prob, cv, T0, A.equilibrium_intensity(prob, T0), cfg.steps, 0,
                        tol=1e-13, max_iter=5000, dt=cfg.dt)
    s.requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = A.leakage(s, st)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = s.grad.detach().cpu().numpy()
    out = {"workload": f"{cfg.name}, T0 = {cfg.T0}, {cfg.steps} steps, FP64", "J": J.item(),
           "forward_s": t1 - t0, "backward_s": t2 - t1, "checkpoint_every": st.every(),
           "params": int(g.size), "grad_max_abs": float(np.abs(g).max())}
    if fd_cells > 0:
        fds = []
        with torch.no_grad():
            for k in cells:
                h = 1e-4 * s[k].item()
                sp, sm_ = s.detach().clone(), s.detach().clone()
                sp[k] += h
                sm_[k] -= h
                fds.append((A.leakage(sp, st).item() - A.leakage(sm_, st).item()) / (2 * h))
        fds = np.array(fds)
        gk = g[cells]
        ref = np.abs(gk) if warm else np.full(gk.shape, np.abs(g).max())
        errs = np.abs(fds - gk) / ref
        out.update({"fd_cells": int(len(cells)),
                    "fd_set": f"{cols} column(s) next to the right edge",
                    "fd_h": "1e-4 s_K",
                    "fd_error": "per cell" if warm else "against the largest sensitivity",
                    "fd_max_rel_err": float(errs.max()),
                    "fd_median_rel_err": float(np.median(errs))})
    prob.close()
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    """--impl reference: the oracle on the host cores, same metric and workload.
    Each step is one bounded oracle pass (a1-a4: emission and closures on the
    whole mesh, sweep and moments of a sample of directions, all groups);
    warm-up and timed steps run as stated, ms_per_step is the measured wall
    time of one pass, and value the sampled updates over that time."""
    import oracle as O
    from paper_2504_21784_gb300 import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload(args)
    n_dirs = oracle_sample_dirs(cfg, budget_s=2.0)
    times = []
    for i in range(args.warmup + args.steps):
        t, upd = oracle_pass(cfg, n_dirs, seed=i)
        if i >= args.warmup:
            times.append(t)
    cb = oracle_summary(cfg, n_dirs, times, upd, O.num_threads())
    v = cb["value"]
    line = {"impl": "reference", "metric": "sweep cell-dir-group updates/s", "value": v,
            "unit": "cell-dir-group updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cb["s_per_pass"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg.name,
                       "step": "bounded oracle pass: emission + closures on the whole mesh, "
                               f"sweep + moments of {n_dirs} of {cfg.n_dir} directions"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "cell-dir-group updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def metric2_summary(sm_res: dict) -> dict:
    """Metric 2 in brief (printed last on the line): seconds per converged
    step of the FP32- and FP64-sweep paths and their temperature difference,
    and of the FP32 sweeps with FP64 defect correction."""
    out = {}
    for name, r in sm_res.items():
        out[name] = {"fp32_s_per_step": r["fp32"]["s_per_step"],
                     "fp64_s_per_step": r["fp64"]["s_per_step"],
                     "fp64_over_fp32": r["fp64_over_fp32_time"],
                     "fp32_vs_fp64_T_rel": r["fp32_vs_fp64_T_rel"],
                     "fp32_refined_s_per_step": r["fp32_refined"]["s_per_step"],
                     "refined_vs_fp64_T_rel": r["refined_vs_fp64_T_rel"],
                     "outer_iters_fp32": r["fp32"]["outer_iters"],
                     "outer_iters_fp64": r["fp64"]["outer_iters"],
                     "refine_corrections": r["fp32_refined"]["refine_corrections"]}
    return out


def summary_text(line: dict) -> str:
    """The line's secondary results as one flat string (the last key), for
    readers that keep only the top level of the record."""
    parts = [f"pass {line['value'] / 1e9:.1f} G updates/s"]
    if "roofline" in line:
        parts[0] += f", sweep {line['roofline']['frac']:.3f} of HBM"
    if "e2e" in line:
        parts[0] += f", e2e {line['e2e']['value'] / 1e9:.1f} G"
    for name, r in line.get("metric2", {}).items():
        parts.append(f"{name.split('_')[0]} s/step FP32 {r['fp32_s_per_step'] * 1e3:.2f} ms, "
                     f"FP64 {r['fp64_s_per_step'] * 1e3:.2f} ms, FP32+FP64-correction "
                     f"{r['fp32_refined_s_per_step'] * 1e3:.2f} ms (T vs FP64 "
                     f"{r['refined_vs_fp64_T_rel']:.1e}; FP32 alone {r['fp32_vs_fp64_T_rel']:.1e})")
    b = line.get("batched")
    if b:
        parts.append(f"batched {b['value'] / 1e9:.1f} G updates/s ({b['roofline']['frac']:.3f} of "
                     f"HBM, {b['batched_speedup']:.2f}x one-by-one), batched step "
                     f"{b['step']['s_per_step']:.3f} s")
    for key in ("adjoint", "adjoint_warm"):
        a = line.get(key)
        if a and "fd_max_rel_err" in a:
            parts.append(f"{key} FD {a['fd_cells']} cells max rel err {a['fd_max_rel_err']:.1e}")
    return "; ".join(parts)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import paper_2504_21784_gb300 as sm
    from paper_2504_21784_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = workload(args)
    custom = bool(args.nx or args.groups or args.workload != "multigroup2d" or
                  args.groups_per_warp)
    prec = args.precision
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        prob = sm.Problem.from_config(cfg, prec, stream=stream,
                                      groups_per_warp=args.groups_per_warp)
        T = torch.from_numpy(W.temperature_wave(cfg)).cuda()
        scale = torch.from_numpy(W.scale_field(cfg)).cuda()
        sigma = prob.opacity(T, scale)
        I = [prob.empty_intensity(), prob.empty_intensity()]
        mom = prob.new_moments()
        clo = prob.new_closures()
        prob.sweep(T, sigma, None, I[0], mom, clo)  # realistic I^k: one step of history
        prob.synchronize()
        if args.tiling:
            w_, s_, e_, t_ = (int(v) for v in args.tiling.split(","))
            prob.set_tail_strips(0)
            prob.set_emission_warps(0)
            prob.set_tiling(w_, s_)
            prob.set_emission_warps(e_)
            prob.set_tail_strips(t_)
            prob.sweep(T, sigma, None, I[0], mom, clo)
            prob.synchronize()
        elif not args.no_autotune:  # pick the strip width / prefetch depth (outside timing)
            prob.autotune(T, sigma, I[0], I[1], reps=2)
            prob.sweep(T, sigma, None, I[0], mom, clo)
            prob.synchronize()

        def step(i):
            prob.sweep(T, sigma, I[i % 2], I[(i + 1) % 2], mom, clo)

        for i in range(args.warmup):
            step(i)
        prob.synchronize()
        barrier()
        prob.set_profiling(True)
        n0 = prob.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            time.sleep(0.3)
            ev0.record(stream)
            for i in range(args.steps):
                step(i + args.warmup)
            ev1.record(stream)
            ev1.synchronize()
        prob.synchronize()
        barrier()
        launches = prob.launch_count() - n0
        ktimes = prob.kernel_times()
        prob.set_profiling(False)
        ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist)

        # end to end through the host-buffer entry point
        T_h = torch.from_numpy(W.temperature_wave(cfg)).pin_memory().numpy()
        S_h = sigma.cpu().pin_memory().numpy()
        M_h = torch.zeros(tuple(mom.shape), dtype=torch.float64).pin_memory().numpy()
        C_h = torch.zeros(tuple(clo.shape), dtype=torch.float64).pin_memory().numpy()
        e2e_steps = max(3, args.steps // 2)
        prob.sweep_host(T_h, S_h, I[0], I[1], M_h, C_h)
        barrier()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            prob.sweep_host(T_h, S_h, I[i % 2], I[(i + 1) % 2], M_h, C_h)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    upd = cfg.updates
    value = replica_rate(world, upd, ms * 1e-3)
    alg = algorithmic_bytes(cfg, prec)
    sweep_ms = ktimes["sweep_ms"] / max(ktimes["count"], 1)
    peak, peak_kind = measured_peaks()
    achieved = alg["per_launch"] / (sweep_ms * 1e-3) / 1e9
    clocks = clk.summary()
    line = {
        "metric": "sweep cell-dir-group updates/s",
        "value": value,
        "unit": "cell-dir-group updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == 32 else "f64",
        "data": "synthetic",
        "config": {"workload": cfg.name, "cells": cfg.n_cells, "directions": cfg.n_dir,
                   "groups": cfg.n_groups,
                   "step": ("emission (Planck integrals in double-FP32, about 48 bits)"
                            if prec == 32 else "emission (FP64 Planck)") +
                           " + sweep with fused moments + fixed-order moment reduction "
                           "(FP64 result) + closures",
                   "sweep_precision": f"fp{prec}", "l2": "inputs larger than L2 "
                   f"({prob.info['intensity_bytes'] / 1e9:.1f} GB per intensity copy)",
                   "tiling": {k: prob.info[k] for k in ("strip_width", "prefetch_rows",
                                                        "groups_per_warp", "n_tasks",
                                                        "n_strips", "tail_strips",
                                                        "emission_warps")},
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "kernel_ms": {"emission": ktimes["emission_ms"] / max(ktimes["count"], 1),
                      "sweep": sweep_ms,
                      "reduce_closures": ktimes["reduce_ms"] / max(ktimes["count"], 1)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(prec, cfg),
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_update": alg["per_update"],
                     "kernel": "sweep2d_kernel"},
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": replica_rate(world, upd, e2e_s), "unit": "cell-dir-group updates/s",
                "h2d_bytes_per_step": int(T_h.nbytes + S_h.nbytes),
                "d2h_bytes_per_step": int(M_h.nbytes + C_h.nbytes),
                "api": "sm_sweep_host (host T, sigma in; moments, closures out)"},
    }
    if not args.no_step_metric and not custom:
        del I, mom, clo, sigma, prob
        torch.cuda.empty_cache()
        line["step_metric"] = step_metric(sm, W, [W.multigroup_2d(), W.gray_channel_2d()],
                                          args.step_steps, stream)
    if not args.no_config_sweeps and not custom:
        line["config_sweeps"] = config_sweeps(sm, W, stream)
    if not args.no_step_metric and not custom:
        line["marshak_paper"] = marshak_paper_metric(sm, W, stream)
    if not args.no_batched and not custom:
        line["batched"] = batched_metric(sm, W, stream, max(3, args.steps // 2), 3)
    if args.adjoint_fd_cells > 0 and not custom:
        line["adjoint"] = adjoint_metric(sm, W, args.adjoint_cold_fd_cells)
        line["adjoint_warm"] = adjoint_metric(sm, W, args.adjoint_fd_cells, warm=True)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    if "step_metric" in line:
        line["metric2"] = metric2_summary(line["step_metric"])
    line["summary"] = summary_text(line)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
