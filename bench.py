#!/usr/bin/env python
"""Converged mode-solves/s of the SCVS hot path on one GB300.

Workload (default): the 3D Womersley pipe, radius 1, length 10, a 5-block
O-grid section (8 x 8 core, 6 radial layers) extruded in 71 layers, 6 tets per
hex, 5 % seeded interior jitter: 151,151 P2 velocity nodes, 19,656 P1
pressure nodes, 473,109 complex dofs per mode; 32 modes (omega_k = 2 pi k,
Womersley numbers W_k = 20 k / 31), inlet coefficients |c_k| = k^-2 with
seeded phases, no-slip wall, traction-free outlet.  A step is one pass of the
whole hot path over the batch: CSR pattern + value assembly of the mesh,
Dirichlet lift and preconditioner set-up of the 32 modes, the batched
mixed-precision GMRES(30) solve of all modes to FP64 relative residual 1e-8,
and the 64-sample time reconstruction.  `value` counts converged mode-solves
per second with inputs resident in HBM; `e2e` repeats the step through the
host-pointer entry points (copies inside the timed region).

`--impl reference` times the FP64 CPU oracle (assembly + sparse LU) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import workloads  # noqa: E402

PIPE = dict(n_c=8, n_r=6, n_x=71, n_modes=32, length=10.0)
N_T = 64
SAMPLE_LAYERS = 4  # oracle sample: same section, 4 of the 71 layers, one mode
FULL_DOFS = 473109  # dofs per mode of the 71-layer pipe


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_over_ranks(elapsed, count, device=None):
    """Whole-job figures of a multi-rank run: the slowest rank's time and the
    units all ranks completed (the only collectives of the path; a no-op for
    one rank).  Works with any torch.distributed backend (NCCL with device
    tensors, gloo with CPU tensors)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed), float(count)
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c)
    return float(t.item()), float(c.item())


def shard(items, rank, world):
    """Independent units (meshes of a batch) dealt round-robin to the ranks:
    every unit on exactly one rank, no exchange between ranks."""
    return list(items)[rank::world]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------- oracle

def oracle_sample(mode=1, layers=SAMPLE_LAYERS):
    """One mode of a `layers`-layer slice of the benchmark pipe: assembly + LU (FP64)."""
    from oracle import fem
    L = PIPE["length"] * layers / PIPE["n_x"]
    wl = workloads.pipe_workload(n_c=PIPE["n_c"], n_r=PIPE["n_r"], n_x=layers, n_modes=mode + 1, length=L)
    wl1 = dict(wl, omegas=wl["omegas"][mode:mode + 1], g=wl["g"][mode:mode + 1])
    t = time.perf_counter()
    mats = fem.assemble(wl1["mesh"])
    X = fem.solve_modes(mats, wl1)
    dt = time.perf_counter() - t
    assert np.all(np.isfinite(X))
    return dt, fem.dof_count(mats)


def growth_exponent(small, large):
    """Measured exponent a of t ~ n_dofs^a between two slices (dt, n_dofs)."""
    (t1, n1), (t2, n2) = small, large
    return float(np.log(t2 / t1) / np.log(n2 / n1))


def cpu_baseline_obj(dt, n, small=None):
    """The oracle as measured: `value` is its rate on the SAMPLE_LAYERS slice
    (one mode of a shorter pipe of the same section, timed in full).  Two
    full-size figures are derived and labelled: `value_linear_upper_bound`
    scales the slice time linearly in length (LU cost grows faster than the
    dof count, so this over-states the oracle's full-size rate) and
    `value_extrapolated` scales it by the dof-count exponent measured between
    `small` (a shorter slice) and the sample."""
    scale = PIPE["n_x"] / SAMPLE_LAYERS
    out = {"value": 1.0 / dt, "unit": "mode-solves/s", "cores": 1, "kind": "oracle", "measured_on": "slice",
           "slice_dofs": int(n), "slice_s": round(dt, 3), "value_linear_upper_bound": 1.0 / (dt * scale)}
    grow = ""
    if small is not None:
        a = growth_exponent(small, (dt, n))
        out["growth_exponent"] = round(a, 2)
        out["value_extrapolated"] = 1.0 / (dt * (FULL_DOFS / n) ** a)
        grow = (f"; a {SAMPLE_LAYERS // 2}-layer slice ({small[1]} dofs) took {small[0]:.2f} s, so the cost grows as "
                f"n_dofs^{a:.1f} here, and extrapolated by that exponent to the full pipe's {FULL_DOFS} dofs the rate "
                f"would be {out['value_extrapolated']:.2e} mode-solves/s (value_extrapolated, not measured)")
    out["sample"] = (f"measured: 1 mode (k=1) of a {SAMPLE_LAYERS}-layer slice ({n} dofs) of the same pipe section "
                     f"(assembly + SuperLU, FP64) in {dt:.2f} s, i.e. value = {1.0 / dt:.3g} mode-solves/s on the slice; "
                     f"scaled linearly in length to the 71-layer pipe it would be "
                     f"{out['value_linear_upper_bound']:.2e} mode-solves/s (value_linear_upper_bound, an upper bound "
                     f"on the full-size rate){grow}")
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    times = []
    for _ in range(args.steps):
        dt, n = oracle_sample()
        times.append(dt)
    dt = float(np.mean(times))
    cb = cpu_baseline_obj(dt, n, oracle_sample(layers=SAMPLE_LAYERS // 2))
    cfg = dict(workload_config(), sample=f"one mode of a {SAMPLE_LAYERS}-layer slice ({n} dofs) per step")
    out = {"metric": "converged mode-solves/s at 1e-8 rel. residual", "value": cb["value"],
           "unit": "mode-solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "impl": "reference", "config": cfg, "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "mode-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def workload_config():
    return {"workload": ("3D Womersley pipe R=1 L=10, O-grid 8x8 core + 6 radial x 71 layers, 151,151 P2 nodes, "
                         "473,109 dofs/mode, 32 modes, P2-P1 Taylor-Hood, GMRES(30) FP32-complex + FP64 "
                         "refinement to rel. residual 1e-8, 64-sample reconstruction"),
            "modes": PIPE["n_modes"], "dofs_per_mode": FULL_DOFS, "restart": 30, "tol": 1e-8,
            "l2": "inputs larger than L2 (Krylov basis 3.9 GB, operator blocks 0.24 GB)"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- GPU

PC_NAMES = {0: "block-chebyshev", 1: "block-diagonal", 2: "block-pmg", 3: "triangular-pmg",
            4: "triangular-pmg + coarse Schur correction",
            5: "auto (triangular-pmg + coarse Schur correction)"}


def pc_config(args):
    """The preconditioner entry of a bench line's config (library default: auto)."""
    kind = 5 if args.precond is None else args.precond
    c = {"precond": PC_NAMES.get(kind, str(kind))}
    if getattr(args, "krylov", "fgmres") == "cocr":
        c["krylov"] = "cocr"
    if kind in (4, 5):
        c["schur_agg"] = args.schur_agg or 16
    if kind != 1:
        lap = getattr(args, "lap_size", 0) or 0
        sm = getattr(args, "lap_smooth", 0) or 8
        c["pressure_laplacian"] = ("chebyshev degree %d" % (getattr(args, "cheb_l", 0) or 75) if lap < 0 else
                                   "two-level: aggregates of %d vertices, %d + %d smoothing steps" % (lap or 32, sm, sm))
    return c


def pc_opts(args):
    """Preconditioner and staging options given on the command line (library defaults otherwise)."""
    o = {}
    if getattr(args, "stage", None) is not None:
        o["stage"] = args.stage
    if getattr(args, "krylov", "fgmres") == "cocr":
        o["krylov"] = 1
    if getattr(args, "graphs", False):
        o["graphs"] = 1
    if args.precond is not None:
        o["precond"] = args.precond
    if args.schur_agg:
        o["schur_agg"] = args.schur_agg
    if getattr(args, "lap_size", 0):
        o["lap_size"] = args.lap_size
    if getattr(args, "lap_smooth", 0):
        o["lap_smooth"] = args.lap_smooth
    for k in ("cheb_u", "cheb_m", "cheb_l", "cheb_c"):
        if getattr(args, k, 0):
            o[k] = getattr(args, k)
    return o


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        small = oracle_sample(layers=SAMPLE_LAYERS // 2)
        dt, n = oracle_sample()
        cb = cpu_baseline_obj(dt, n, small)

    wl = workloads.pipe_workload(n_c=PIPE["n_c"], n_r=PIPE["n_r"], n_x=PIPE["n_x"], n_modes=PIPE["n_modes"],
                                 length=PIPE["length"])
    mesh = wl["mesh"]
    N, P, E, d = mesh["xyz"].shape[0], mesh["n_vertices"], mesh["conn"].shape[0], 3
    m = len(wl["omegas"])
    stream = torch.cuda.current_stream(dev)
    opts = dict(stream=stream.cuda_stream, precision=scvs.SCVS_PREC_FP64 if args.precision == "fp64"
                else scvs.SCVS_PREC_MIXED)
    if args.restart:
        opts["restart"] = args.restart
    opts.update(pc_opts(args))
    solver = scvs.Solver(**opts)
    ctx = solver.ctx
    # device-resident inputs
    xyz_d = torch.from_numpy(mesh["xyz"]).to(dev)
    conn_d = torch.from_numpy(mesh["conn"]).to(dev)
    tag_d = torch.from_numpy(mesh["tag"]).to(dev)
    g_d = torch.from_numpy(np.ascontiguousarray(wl["g"])).to(dev)
    u_t = torch.empty((N_T, N, d), dtype=torch.float64, device=dev)
    p_t = torch.empty((N_T, P), dtype=torch.float64, device=dev)

    def step_dev():
        scvs.scvs_clear_meshes(ctx)
        mid = scvs.scvs_set_mesh_dev(ctx, d, N, P, xyz_d.data_ptr(), E, conn_d.data_ptr(), tag_d.data_ptr())
        scvs.scvs_set_physics(ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes_dev(ctx, mid, wl["omegas"], g_d.data_ptr())
        rep = scvs.scvs_solve(ctx, mid, m)
        scvs.scvs_reconstruct_dev(ctx, mid, N_T, wl["period"], u_t.data_ptr(), p_t.data_ptr())
        return rep

    def phases():
        """Host wall time of each call of one step, synchronised after every call
        (a diagnostic step outside the timed region)."""
        out = {}

        def t(name, fn):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            out[name] = round((time.perf_counter() - t0) * 1e3, 2)
            return r
        t("clear_meshes", lambda: scvs.scvs_clear_meshes(ctx))
        mid = t("set_mesh_dev", lambda: scvs.scvs_set_mesh_dev(ctx, d, N, P, xyz_d.data_ptr(), E, conn_d.data_ptr(),
                                                                tag_d.data_ptr()))
        t("set_physics", lambda: scvs.scvs_set_physics(ctx, mid, wl["rho"], wl["mu"]))
        t("set_modes_dev", lambda: scvs.scvs_set_modes_dev(ctx, mid, wl["omegas"], g_d.data_ptr()))
        t("solve", lambda: scvs.scvs_solve(ctx, mid, m))
        t("reconstruct_dev", lambda: scvs.scvs_reconstruct_dev(ctx, mid, N_T, wl["period"], u_t.data_ptr(),
                                                               p_t.data_ptr()))
        return out

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        rep = step_dev()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    scvs.scvs_kernel_timers(ctx, not args.no_timers)
    launches0 = scvs.scvs_launch_count(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for _ in range(args.steps):
        reps.append(step_dev())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    launches = scvs.scvs_launch_count(ctx) - launches0
    ktimes = scvs.scvs_kernel_times(ctx)
    scvs.scvs_kernel_timers(ctx, False)
    conv = sum(1 for rr in reps for r in rr if r["status"] == scvs.SCVS_CONVERGED)
    tuned = scvs.scvs_tuned_shapes(ctx, 0)
    tuned["staged"] = scvs.scvs_staged_info(ctx, 0)
    phase_ms = phases()
    elapsed, conv_total = reduce_over_ranks(elapsed, conv, dev)
    value = conv_total / elapsed

    # ---- end to end through the host-pointer entry points
    e2e = None
    if not args.no_e2e:
        hb = pinned_host_buffers(torch, wl, m, N, P, d)
        for _ in range(1):
            step_host(scvs, ctx, wl, m, N, P, d, hb)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ev0.record(stream)
        conv_e = 0
        for _ in range(args.steps):
            rr, nb_in, nb_out = step_host(scvs, ctx, wl, m, N, P, d, hb)
            conv_e += sum(1 for r in rr if r["status"] == scvs.SCVS_CONVERGED)
        ev1.record(stream)
        torch.cuda.synchronize()
        te = max(ev0.elapsed_time(ev1) / 1e3, time.perf_counter() - t0)
        te, conv_e = reduce_over_ranks(te, conv_e, dev)
        e2e = {"value": conv_e / te, "unit": "mode-solves/s", "h2d_bytes_per_step": nb_in, "d2h_bytes_per_step": nb_out}

    # ---- accuracy and the per-mode FP64 comparison (untimed, rank 0)
    accuracy = fp64_cmp = None
    if rank == 0 and not args.no_fp64_check and args.precision == "mixed":
        accuracy = fp64_error_by_mode(scvs, ctx, wl, m, N, P, d)
        fp64_cmp = fp64_per_mode_rate(scvs, torch, wl, args.fp64_modes)
        fp64_cmp["speedup_of_value"] = value / fp64_cmp["value"]

    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    if args.no_timers:  # no per-class times: the line carries no roofline (placeholder entry below)
        ktimes = dict(ktimes, cheb_fine=(1e-9, 0.0, 1))
    # dominant kernel class by device time inside the timed region
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    ms, by, nl = ktimes[dom]
    achieved = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    traffic = traffic_from_profiles(dom)
    kernel_names = {"cheb_fine": "k_pc_cheb (velocity rows) + k_vel_residual", "arnoldi": "k_arnoldi",
                    "spmm_fp32": "k_saddle<float>", "precond": "k_tri_vel0 + k_prolong + k_pc_step0",
                    "pressure": "k_pressure_solve", "coarse": "k_coarse_solve",
                    "spmm_fp64": "k_saddle<double>"}
    roof = {"bound": "hbm", "kernel": kernel_names.get(dom, dom), "kernel_class": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peak_kind,
            "launches": nl, "avg_launch_us": ms / max(nl, 1) * 1e3,
            "algorithmic_bytes_per_launch": by / max(nl, 1)}
    sp_ms, sp_by, sp_n = ktimes["spmm_fp32"]
    spmm = {"achieved": sp_by / (sp_ms / 1e3) / 1e9 if sp_ms > 0 else 0.0, "unit": "GB/s",
            "frac": (sp_by / (sp_ms / 1e3) / 1e9) / peaks["hbm_gbs"] if sp_ms > 0 else 0.0,
            "launches": sp_n, "avg_launch_us": sp_ms / max(sp_n, 1) * 1e3}
    last = reps[-1]
    out = {"metric": "converged mode-solves/s at 1e-8 rel. residual", "value": value, "unit": "mode-solves/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "c128" if args.precision == "fp64" else "c64+f64", "data": "synthetic",
           "config": dict(workload_config(), **pc_config(args), graphs=bool(args.graphs)),
           "roofline": None if args.no_timers else roof, "spmm": None if args.no_timers else spmm,
           "kernel_ms": {k: round(v[0], 3) for k, v in ktimes.items()},
           "gpu_launches": int(launches), "clocks": clk, "e2e": e2e, "cpu_baseline": cb, "autotune": tuned,
           "phase_ms": phase_ms,
           "solve": {"converged": conv, "modes_per_step": m,
                     "iterations_by_mode": [r["iterations"] for r in last],
                     "iterations_max": max(r["iterations"] for r in last),
                     "iterations_mean": float(np.mean([r["iterations"] for r in last])),
                     "cycles_max": max(r["cycles"] for r in last),
                     "rel_res_max": max(r["rel_res"] for r in last)}}
    if accuracy is not None:
        out["solve"].update(accuracy)
        out["fp64_permode"] = fp64_cmp
    if args.precision == "fp64":
        out["metric_note"] = "all-FP64 GMRES comparison run"
    print(json.dumps(out), flush=True)
    solver.close()


def fp64_error_by_mode(scvs, ctx, wl, m, N, P, d):
    """Relative L2 error of every mode of the last timed (mixed-precision,
    residual 1e-8) solve against an all-FP64 GPU solve of the same modes to a
    1e-12 residual, on the dof vector (u, p)."""
    u, p = scvs.scvs_get_modal(ctx, 0, m, N, d, P)
    X = np.concatenate([u.reshape(m, -1), p], axis=1)
    with scvs.Solver(precision=scvs.SCVS_PREC_FP64, tol=1e-12, max_cycles=2000) as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        rep = scvs.scvs_solve(s.ctx, mid, m)
        u64, p64 = scvs.scvs_get_modal(s.ctx, mid, m, N, d, P)
    X64 = np.concatenate([u64.reshape(m, -1), p64], axis=1)
    err = [float(np.linalg.norm(X[k] - X64[k]) / np.linalg.norm(X64[k])) for k in range(m)]
    return {"err_vs_fp64_by_mode": err, "err_vs_fp64_max": max(err),
            "fp64_reference": ("all-FP64 GPU GMRES of the same modes to rel. residual 1e-12 "
                               f"(max residual {max(r['rel_res'] for r in rep):.1e})")}


def fp64_per_mode_rate(scvs, torch, wl, n_modes):
    """Plain per-mode FP64 GMRES (same block preconditioner, zero guess, one
    mode per solve) on `n_modes` sampled modes of the workload: the rate of
    its solves."""
    modes = [int(k) for k in np.linspace(0, len(wl["omegas"]) - 1, n_modes).round()]
    with scvs.Solver(precision=scvs.SCVS_PREC_FP64) as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        times, its, conv = [], [], 0
        for k in modes:
            scvs.scvs_set_modes(s.ctx, mid, wl["omegas"][k:k + 1], wl["g"][k:k + 1])
            torch.cuda.synchronize()
            t = time.perf_counter()
            rep = scvs.scvs_solve(s.ctx, mid, 1)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
            its.append(rep[0]["iterations"])
            conv += rep[0]["status"] == scvs.SCVS_CONVERGED
    return {"value": conv / sum(times), "unit": "mode-solves/s",
            "method": "plain per-mode FP64 GMRES(30), same preconditioner, zero guess, solve phase only",
            "modes": modes, "iterations": its, "solve_s": [round(t, 4) for t in times]}


def run_kernel_case(args):
    """Launch-light sequence on the full-size pipe for profiler captures:
    assembly, mode set-up, 3 all-modes SpMMs (FP32), 2 preconditioner
    applications and one GMRES(4) cycle (4 Arnoldi steps)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    wl = workloads.pipe_workload(n_c=PIPE["n_c"], n_r=PIPE["n_r"], n_x=PIPE["n_x"], n_modes=PIPE["n_modes"],
                                 length=PIPE["length"])
    mesh = wl["mesh"]
    with scvs.Solver(restart=4, max_cycles=1, **pc_opts(args)) as s:
        mid = scvs.scvs_set_mesh(s.ctx, mesh)
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        n = scvs.scvs_dof_count(s.ctx, mid)
        ld = scvs.scvs_mode_stride(s.ctx, mid)
        x = torch.randn((n, ld), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        torch.cuda.synchronize()
        for _ in range(3):
            scvs.scvs_apply(s.ctx, mid, scvs.SCVS_PREC_MIXED, x.data_ptr(), y.data_ptr())
        for _ in range(2):
            scvs.scvs_apply_precond(s.ctx, mid, x.data_ptr(), y.data_ptr())
        rep = scvs.scvs_solve(s.ctx, mid, len(wl["omegas"]))
        torch.cuda.synchronize()
        log("kernel case done:", scvs.scvs_launch_count(s.ctx), "launches; cycle iterations",
            [r["iterations"] for r in rep][:4])


def run_batch(args):
    """Uneven batch: 48 stenosed pipes (20k-400k P2 nodes, log-uniform), 16
    modes each = 768 independent systems, solved as one mesh of independent
    components (one launch per kernel for all meshes)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    all_parts = workloads.uneven_pipes(n_meshes=args.batch_meshes, n_modes=16, seed=0, scale=args.batch_scale)
    parts = shard(all_parts, rank, world)  # each rank solves its own meshes; no exchange
    U = workloads.union_workload(parts)
    mesh = U["mesh"]
    N, P, E, d = mesh["xyz"].shape[0], mesh["n_vertices"], mesh["conn"].shape[0], 3
    m = len(U["omegas"])
    stream = torch.cuda.current_stream(dev)
    solver = scvs.Solver(stream=stream.cuda_stream, **pc_opts(args))
    ctx = solver.ctx
    xyz_d = torch.from_numpy(mesh["xyz"]).to(dev)
    conn_d = torch.from_numpy(mesh["conn"]).to(dev)
    tag_d = torch.from_numpy(mesh["tag"]).to(dev)
    g_d = torch.from_numpy(np.ascontiguousarray(U["g"])).to(dev)
    u_t = torch.empty((N_T, N, d), dtype=torch.float64, device=dev)
    p_t = torch.empty((N_T, P), dtype=torch.float64, device=dev)

    def step():
        scvs.scvs_clear_meshes(ctx)
        mid = scvs.scvs_set_mesh_dev(ctx, d, N, P, xyz_d.data_ptr(), E, conn_d.data_ptr(), tag_d.data_ptr())
        scvs.scvs_set_components(ctx, mid, U["n_comp"], U["node_comp"])
        scvs.scvs_set_physics(ctx, mid, U["rho"], U["mu"])
        scvs.scvs_set_modes_dev(ctx, mid, U["omegas"], g_d.data_ptr())
        rep = scvs.scvs_solve(ctx, mid, U["n_comp"] * m)
        scvs.scvs_reconstruct_dev(ctx, mid, N_T, U["period"], u_t.data_ptr(), p_t.data_ptr())
        return rep

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    scvs.scvs_kernel_timers(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    el = ev0.elapsed_time(ev1) / 1e3
    kt = scvs.scvs_kernel_times(ctx)
    conv = sum(1 for rr in reps for r in rr if r["status"] == scvs.SCVS_CONVERGED)
    el, conv = reduce_over_ranks(el, conv, dev)
    if rank != 0:
        solver.close()
        return
    sizes = [p["mesh"]["xyz"].shape[0] for p in all_parts]
    out = {"metric": "converged mode-solves/s at 1e-8 rel. residual", "value": conv / el, "unit": "mode-solves/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
           "impl": "batch",
           "config": {"workload": (f"uneven batch: {len(all_parts)} stenosed pipes (R 0.5-1.5, L 5-20, s 0-0.5), "
                                   f"{min(sizes)}-{max(sizes)} P2 nodes (rank 0: {len(parts)} meshes, {N} nodes), "
                                   f"16 modes each = {len(all_parts) * 16} systems, one mesh of independent "
                                   f"components per rank, meshes dealt round-robin to {world} rank(s)"),
                      "systems": len(all_parts) * 16, "nodes_rank0": N, **pc_config(args)},
           "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
           "solve": {"converged": conv, "systems_per_step": len(all_parts) * 16,
                     "iterations_max": max(r["iterations"] for r in reps[-1]),
                     "iterations_mean": float(np.mean([r["iterations"] for r in reps[-1]])),
                     "rel_res_max": max(r["rel_res"] for r in reps[-1])}}
    print(json.dumps(out), flush=True)
    solver.close()


def run_bifurcation(args):
    """Large stenosed bifurcation: parent R = 1 with a 50% cosine stenosis,
    daughters R = 0.7 at +-45 deg, voxel mesh of spacing h (h = 0.038: ~6M P2
    nodes), 16 modes, GMRES(20) FP32 + FP64 refinement."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    t0 = time.perf_counter()
    wl = workloads.bifurcation_workload(h=args.bif_h, n_modes=16)
    t_gen = time.perf_counter() - t0
    mesh = wl["mesh"]
    N, P, E, d = mesh["xyz"].shape[0], mesh["n_vertices"], mesh["conn"].shape[0], 3
    m = len(wl["omegas"])
    stream = torch.cuda.current_stream(dev)
    solver = scvs.Solver(stream=stream.cuda_stream, restart=20, **pc_opts(args))
    ctx = solver.ctx
    xyz_d = torch.from_numpy(mesh["xyz"]).to(dev)
    conn_d = torch.from_numpy(mesh["conn"]).to(dev)
    tag_d = torch.from_numpy(mesh["tag"]).to(dev)
    g_d = torch.from_numpy(np.ascontiguousarray(wl["g"])).to(dev)
    u_t = torch.empty((N_T, N, d), dtype=torch.float64, device=dev)
    p_t = torch.empty((N_T, P), dtype=torch.float64, device=dev)

    def step():
        scvs.scvs_clear_meshes(ctx)
        mid = scvs.scvs_set_mesh_dev(ctx, d, N, P, xyz_d.data_ptr(), E, conn_d.data_ptr(), tag_d.data_ptr())
        scvs.scvs_set_physics(ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes_dev(ctx, mid, wl["omegas"], g_d.data_ptr())
        rep = scvs.scvs_solve(ctx, mid, m)
        scvs.scvs_reconstruct_dev(ctx, mid, N_T, wl["period"], u_t.data_ptr(), p_t.data_ptr())
        return rep

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info(dev)
    scvs.scvs_kernel_timers(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    el = ev0.elapsed_time(ev1) / 1e3
    kt = scvs.scvs_kernel_times(ctx)
    conv = sum(1 for rr in reps for r in rr if r["status"] == scvs.SCVS_CONVERGED)
    out = {"metric": "converged mode-solves/s at 1e-8 rel. residual", "value": conv / el, "unit": "mode-solves/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
           "impl": "bifurcation",
           "config": {"workload": (f"stenosed bifurcation (parent R=1, 50% cosine stenosis, daughters R=0.7 at "
                                   f"+-45 deg), voxel mesh h={args.bif_h}: {N} P2 nodes, {P} vertices, {E} tets, "
                                   f"{3 * N + P} dofs/mode, 16 modes, GMRES(20) FP32 + FP64 refinement"),
                      "nodes": N, "dofs_per_mode": 3 * N + P, "mesh_gen_s": round(t_gen, 1),
                      **pc_config(args)},
           "device_memory_gb": round((total - free) / 1e9, 1),
           "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
           "solve": {"converged": conv, "modes_per_step": m,
                     "iterations_max": max(r["iterations"] for r in reps[-1]),
                     "iterations_mean": float(np.mean([r["iterations"] for r in reps[-1]])),
                     "cycles_max": max(r["cycles"] for r in reps[-1]),
                     "rel_res_max": max(r["rel_res"] for r in reps[-1])}}
    print(json.dumps(out), flush=True)
    solver.close()


def run_spmm(args):
    """All-modes operator y_k = A_hat(omega_k) x_k on the benchmark pipe (32
    modes): CSR SpMM and matrix-free apply, FP32 and FP64, each launch timed on
    the library's stream after an L2 flush (a 512 MB write), algorithmic bytes
    from the library's accounting (every matrix array and the geometry once, x
    read once, y written once)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    wl = workloads.pipe_workload(n_c=PIPE["n_c"], n_r=PIPE["n_r"], n_x=PIPE["n_x"], n_modes=PIPE["n_modes"],
                                 length=PIPE["length"])
    peaks, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream(dev)
    out = {}
    with scvs.Solver(stream=stream.cuda_stream, **pc_opts(args)) as s:
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        staged = scvs.scvs_staged_info(s.ctx, mid)
        n, ld = scvs.scvs_dof_count(s.ctx, mid), scvs.scvs_mode_stride(s.ctx, mid)
        gen = torch.Generator(device=dev).manual_seed(0)
        x64 = torch.randn((n, ld), dtype=torch.complex128, device=dev, generator=gen)
        x32 = x64.to(torch.complex64)
        y64, y32 = torch.empty_like(x64), torch.empty_like(x32)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        cases = [("csr_fp32", scvs.scvs_apply, scvs.SCVS_PREC_MIXED, x32, y32, "spmm_fp32"),
                 ("csr_fp64", scvs.scvs_apply, scvs.SCVS_PREC_FP64, x64, y64, "spmm_fp64"),
                 ("matfree_fp32", scvs.scvs_apply_matfree, scvs.SCVS_PREC_MIXED, x32, y32, "matfree"),
                 ("matfree_fp64", scvs.scvs_apply_matfree, scvs.SCVS_PREC_FP64, x64, y64, "matfree")]
        for name, fn, prec, x, y, cls in cases:
            for _ in range(max(3, args.warmup)):
                fn(s.ctx, mid, prec, x.data_ptr(), y.data_ptr())
            torch.cuda.synchronize()
            scvs.scvs_kernel_timers(s.ctx, True)
            for _ in range(args.steps * 4):
                flush.zero_()
                fn(s.ctx, mid, prec, x.data_ptr(), y.data_ptr())
            torch.cuda.synchronize()
            ms, by, nl = scvs.scvs_kernel_times(s.ctx)[cls]
            scvs.scvs_kernel_timers(s.ctx, False)
            gbs = by / (ms / 1e3) / 1e9
            out[name] = {"us_per_launch": round(ms / nl * 1e3, 1), "algorithmic_mb": round(by / nl / 1e6, 1),
                         "gb_s": round(gbs, 1), "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 3)}
    line = {"metric": "SpMM HBM GB/s (all-modes operator, algorithmic bytes)", "value": out["csr_fp32"]["gb_s"],
            "unit": "GB/s", "n_gpus": 1, "higher_is_better": True, "impl": "spmm", "data": "synthetic",
            "dtype": "c64", "peak": peaks["hbm_gbs"], "peak_source": peak_kind,
            "config": {"workload": "151k-node pipe, 32 modes, 473,109 dofs/mode, L2 flushed before each launch"},
            "cases": out, "staged": staged}
    print(json.dumps(line), flush=True)


def run_guess(args):
    """Learned initial guess on the benchmark pipe family: train on morphs
    (R ~ U[0.5, 1.5], s ~ U[0, 0.5]) of the 151k-node pipe, then solve
    held-out morphs with and without the guess."""
    import torch
    torch.cuda.set_device(0)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    rng = np.random.default_rng(0)

    def morph(i):
        R, st = rng.uniform(0.5, 1.5), rng.uniform(0.0, 0.5)
        wl = workloads.pipe_workload(n_c=PIPE["n_c"], n_r=PIPE["n_r"], n_x=PIPE["n_x"], n_modes=PIPE["n_modes"],
                                     length=PIPE["length"], radius=R, stenosis=st, seed=0)
        c = workloads.phases(PIPE["n_modes"], seed=100 + i)
        wl = dict(wl, coeffs=c, g=wl["g"] / wl["coeffs"][:, None, None] * c[:, None, None])
        f = np.stack([wl["omegas"], c.real, c.imag, np.full(len(c), R), np.full(len(c), st)], axis=1)
        return wl, f

    def solve(s, wl, f):
        scvs.scvs_clear_meshes(s.ctx)
        mid = scvs.scvs_set_mesh(s.ctx, wl["mesh"])
        scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
        scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
        scvs.scvs_guess_set_features(s.ctx, mid, f)
        torch.cuda.synchronize()
        t = time.perf_counter()
        rep = scvs.scvs_solve(s.ctx, mid, len(f))
        return mid, rep, time.perf_counter() - t

    with scvs.Solver(**pc_opts(args)) as s:
        t0 = time.perf_counter()
        for i in range(args.guess_train):
            wl, f = morph(i)
            mid, rep, _ = solve(s, wl, f)
            scvs.scvs_guess_add_snapshots(s.ctx, mid, f)
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        loss = scvs.scvs_train_guess(s.ctx, scvs.scvs_default_train_opts(steps=args.guess_steps))
        t_train = time.perf_counter() - t0
        rows = []
        for i in range(args.guess_test):
            wl, f = morph(10_000 + i)
            res = {}
            for gmode in (scvs.SCVS_GUESS_ZERO, scvs.SCVS_GUESS_MLP):
                s.set_opts(guess=gmode)
                _, rep, dt = solve(s, wl, f)
                res[gmode] = (rep, dt)
            rows.append(res)
        info = scvs.scvs_guess_info(s.ctx)
    it0 = [r["iterations"] for res in rows for r in res[scvs.SCVS_GUESS_ZERO][0]]
    it1 = [r["iterations"] for res in rows for r in res[scvs.SCVS_GUESS_MLP][0]]
    t0s = sum(res[scvs.SCVS_GUESS_ZERO][1] for res in rows)
    t1s = sum(res[scvs.SCVS_GUESS_MLP][1] for res in rows)
    n = len(it0)
    conv1 = sum(1 for res in rows for r in res[scvs.SCVS_GUESS_MLP][0] if r["status"] == scvs.SCVS_CONVERGED)
    out = {"metric": "converged mode-solves/s at 1e-8 rel. residual", "value": conv1 / t1s, "unit": "mode-solves/s",
           "n_gpus": 1, "higher_is_better": True, "impl": "learned-guess", "data": "synthetic", "dtype": "c64+f64",
           "config": {"workload": (f"learned initial guess: {args.guess_train} training morphs x 32 modes of the "
                                   f"151k-node pipe (R 0.5-1.5, s 0-0.5), {args.guess_test} held-out morphs"),
                      "snapshots": info["n_snapshots"], "n_pod": info["n_pod"], "mlp": "5-256-256-256-128 GELU BF16",
                      **pc_config(args)},
           "without_guess": {"value": n / t0s, "iterations_mean": float(np.mean(it0)), "iterations_max": int(max(it0)),
                             "solve_s": t0s},
           "with_guess": {"value": conv1 / t1s, "iterations_mean": float(np.mean(it1)), "iterations_max": int(max(it1)),
                          "solve_s": t1s},
           "training": {"data_s": t_data, "train_s": t_train, "final_loss": loss}}
    print(json.dumps(out), flush=True)


def run_fp64_permode(args):
    """Comparison: plain per-mode FP64 GMRES (same block preconditioner, zero
    guess), one mode per solve, on a sample of the benchmark pipe's modes."""
    import torch
    torch.cuda.set_device(0)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    wl = workloads.pipe_workload(n_c=PIPE["n_c"], n_r=PIPE["n_r"], n_x=PIPE["n_x"], n_modes=PIPE["n_modes"],
                                 length=PIPE["length"])
    r = fp64_per_mode_rate(scvs, torch, wl, args.fp64_modes)
    out = {"metric": "converged mode-solves/s at 1e-8 rel. residual", "value": r["value"], "unit": "mode-solves/s",
           "n_gpus": 1, "impl": "fp64-per-mode GMRES", "dtype": "c128", "data": "synthetic",
           "higher_is_better": True,
           "config": {"workload": ("151k-node pipe, plain per-mode FP64 GMRES(30), same block preconditioner, zero "
                                   f"guess, one mode per solve; sampled modes {r['modes']}")},
           "modes": r["modes"], "iterations": r["iterations"], "solve_s": r["solve_s"]}
    print(json.dumps(out), flush=True)


def run_validation(args):
    """The paper's validation cases on the GPU path (traction inlets, analytic
    solutions): the channel of Sec. 3.2 on the paper's mesh (Table
    channel_err: e(T/4), e(T/2) at W = 0, 2 pi, 10 pi, 20 pi) and the pipe of
    Sec. 3.4 (L/R = 15) on meshes of the QM1-QM4 node counts: e(T/2) at W = 8 pi
    per mesh (Fig. cylinder_msh_elesize) and e(T/2) at W = 0, 8 pi, ..., 80 pi on
    the finest (Fig. cylinder_msh_freq).  The errors use the assembled M_s of
    the library (scvs_get_values) and the time samples of its reconstruction."""
    import torch
    torch.cuda.set_device(0)
    from paper_2009_06725_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2009_06725_gb300 import scvs
    import scipy.sparse as sp
    from synthetic.womersley import channel_profile, pipe_profile

    def solve(wl, tol):
        mesh = wl["mesh"]
        N, P, d, m = mesh["xyz"].shape[0], mesh["n_vertices"], mesh["dim"], len(wl["omegas"])
        with scvs.Solver(tol=tol, max_cycles=2000) as s:
            mid = scvs.scvs_set_mesh(s.ctx, mesh)
            scvs.scvs_set_physics(s.ctx, mid, wl["rho"], wl["mu"])
            scvs.scvs_set_modes(s.ctx, mid, wl["omegas"], wl["g"])
            scvs.scvs_set_neumann(s.ctx, mid, wl["h"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = scvs.scvs_solve(s.ctx, mid, m)
            dt = time.perf_counter() - t0
            u, _ = scvs.scvs_get_modal(s.ctx, mid, m, N, d, P)
            rp, col = scvs.scvs_get_csr(s.ctx, mid, scvs.SCVS_CSR_S)
            vals = scvs.scvs_get_values(s.ctx, mid, scvs.SCVS_CSR_S, d)
        Ms = sp.csr_matrix((vals[0], col, rp), shape=(N, N))
        return u, Ms, rep, dt

    def err_t(Ms, uh, ue, w, t):
        ph = np.exp(1j * w * t)
        a, b = np.real(ue * ph), np.real(uh * ph)
        e, f = a - b, a
        ne = sum(float(e[:, c] @ (Ms @ e[:, c])) for c in range(e.shape[1]))
        nf = sum(float(f[:, c] @ (Ms @ f[:, c])) for c in range(f.shape[1]))
        return float(np.sqrt(ne / nf))

    out = {"metric": "relative L2 error e(t) against the analytic solution (Eq. total_error)", "impl": "validation",
           "n_gpus": 1, "data": "synthetic", "dtype": "c64+f64", "unit": "1", "tol": args.val_tol}
    # channel
    rho, mu, H, L = 1.0, 0.01, 0.5, 5.0
    Ws = [0.0, 2 * np.pi, 10 * np.pi, 20 * np.pi]
    wl = workloads.paper_channel(np.array(Ws) * (mu / rho) / H ** 2, rho=rho, mu=mu, neumann_tag=scvs.SCVS_TAG_NEUMANN)
    u, Ms, rep, dt = solve(wl, args.val_tol)
    y = wl["mesh"]["xyz"][:, 1]
    rows = []
    for k, W in enumerate(Ws):
        w = wl["omegas"][k]
        ex = np.zeros_like(u[k])
        ex[:, 0] = channel_profile(y, w, H, rho, mu, G=1.0 / L)
        T = 2 * np.pi / w if w > 0 else 1.0
        rows.append({"W_over_pi": W / np.pi, "e_T4": err_t(Ms, u[k], ex, w, 0.25 * T),
                     "e_T2": err_t(Ms, u[k], ex, w, 0.5 * T), "iterations": rep[k]["iterations"]})
    out["channel"] = {"mesh": "49 x 9 quads of [0,5] x [-0.5,0.5] in P2 triangles: 882 elements, 1,881 nodes, "
                              "4,262 dofs (the paper's mesh)", "rows": rows, "solve_s": dt,
                      "paper_scvs_percent": {"0": "1.3e-3 (at eps_L 1e-6)", "2pi": [0.01, 0.031],
                                             "10pi": [0.12, 0.46], "20pi": [0.29, 1.8]}}
    # pipe
    rho, mu = 1.0, 1.0
    conv = []
    for (name, target), curved in [(q, cv) for cv in (True, False) for q in
                                   (("QM1", 37469), ("QM2", 70872), ("QM3", 133645), ("QM4", 225610))]:
        wl = workloads.paper_pipe(target, np.array([8 * np.pi * mu / rho]), rho=rho, mu=mu,
                                  neumann_tag=scvs.SCVS_TAG_NEUMANN, curved=curved)
        u, Ms, rep, dt = solve(wl, args.val_tol)
        xyz = wl["mesh"]["xyz"]
        r = np.hypot(xyz[:, 1], xyz[:, 2])
        ex = np.zeros_like(u[0])
        w = wl["omegas"][0]
        ex[:, 0] = pipe_profile(r, w, 1.0, rho, mu, G=1.0 / 15.0)
        n_el = wl["mesh"]["conn"].shape[0]
        h = (np.pi * 15.0 / n_el * 6.0 * np.sqrt(2.0)) ** (1.0 / 3.0)  # edge of a regular tet of the mean volume
        conv.append({"mesh": name + "-sized", "wall": "curved" if curved else "straight",
                     "nodes": int(xyz.shape[0]), "elements": int(n_el), "h_over_R": h,
                     "e_T2": err_t(Ms, u[0], ex, w, np.pi / w), "iterations": rep[0]["iterations"], "solve_s": dt})
    Ws = np.arange(11) * 8 * np.pi
    wl = workloads.paper_pipe(225610, Ws * mu / rho, rho=rho, mu=mu, neumann_tag=scvs.SCVS_TAG_NEUMANN)
    u, Ms, rep, dt = solve(wl, args.val_tol)
    xyz = wl["mesh"]["xyz"]
    r = np.hypot(xyz[:, 1], xyz[:, 2])
    freq = []
    for k, W in enumerate(Ws):
        w = wl["omegas"][k]
        ex = np.zeros_like(u[k])
        ex[:, 0] = pipe_profile(r, w, 1.0, rho, mu, G=1.0 / 15.0)
        T = 2 * np.pi / w if w > 0 else 1.0
        freq.append({"W_over_pi": float(W / np.pi), "e_T2": err_t(Ms, u[k], ex, w, 0.5 * T),
                     "iterations": rep[k]["iterations"]})
    out["pipe"] = {"geometry": ("L/R = 15, R = 1, traction inlet, no-slip wall, traction-free outlet, O-grid tets; "
                                "wall edge nodes on the cylinder (curved, isoparametric) or at chord midpoints"),
                   "convergence_W8pi": conv, "frequency_QM4": freq, "frequency_solve_s": dt,
                   "paper": "QM1-QM4: 37,469-225,610 nodes; e(T/2) at W = 8 pi and its growth with W in "
                            "Figs. cylinder_msh_elesize and cylinder_msh_freq (context only)"}
    print(json.dumps(out), flush=True)


def pinned_host_buffers(torch, wl, m, N, P, d):
    """Inputs copied once into page-locked host memory and page-locked output
    arrays, so the end-to-end step moves its bytes by DMA (set up outside the
    timed region)."""
    def pin(a):
        t = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True)
        v = t.numpy()
        v[...] = a
        return t, v

    mesh = wl["mesh"]
    keep, arrs = [], {}
    for k, a in (("xyz", mesh["xyz"]), ("conn", mesh["conn"]), ("tag", mesh["tag"]), ("g", wl["g"])):
        t, v = pin(np.ascontiguousarray(a))
        keep.append(t)
        arrs[k] = v
    for k, shape, dt in (("u", (m, N, d), torch.complex128), ("p", (m, P), torch.complex128),
                         ("ut", (N_T, N, d), torch.float64), ("pt", (N_T, P), torch.float64)):
        t = torch.empty(shape, dtype=dt, pin_memory=True)
        keep.append(t)
        arrs[k] = t.numpy()
    arrs["mesh"] = dict(mesh, xyz=arrs["xyz"], conn=arrs["conn"], tag=arrs["tag"])
    arrs["_keep"] = keep
    return arrs


def step_host(scvs, ctx, wl, m, N, P, d, hb):
    """One step through the host-array API: inputs from and results to pinned host memory."""
    scvs.scvs_clear_meshes(ctx)
    mid = scvs.scvs_set_mesh(ctx, hb["mesh"])
    scvs.scvs_set_physics(ctx, mid, wl["rho"], wl["mu"])
    scvs.scvs_set_modes(ctx, mid, wl["omegas"], hb["g"])
    rep = scvs.scvs_solve(ctx, mid, m)
    scvs.scvs_get_modal(ctx, mid, m, N, d, P, out_u=hb["u"], out_p=hb["p"])
    scvs.scvs_reconstruct(ctx, mid, N_T, wl["period"], N, d, P, out_u=hb["ut"], out_p=hb["pt"])
    nb_in = sum(hb[k].nbytes for k in ("xyz", "conn", "tag", "g")) + wl["omegas"].nbytes
    nb_out = sum(hb[k].nbytes for k in ("u", "p", "ut", "pt"))
    return rep, int(nb_in), int(nb_out)


def traffic_from_profiles(kernel_class):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it covers it."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(kernel_class)
        return None if e is None else e.get("dram_bytes_per_launch")
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cheb-u", type=int, default=0)
    ap.add_argument("--cheb-m", type=int, default=0)
    ap.add_argument("--cheb-l", type=int, default=0)
    ap.add_argument("--cheb-c", type=int, default=0)
    ap.add_argument("--restart", type=int, default=0)
    ap.add_argument("--precond", type=int, default=None, help="0 BLOCK_CHEB, 1 BLOCK_DIAG, 2 BLOCK_PMG, 3 TRI_PMG, "
                    "4 TRI_PMG_CS (coarse Schur correction), 5 AUTO (default: 4 on the batch and the bifurcation, "
                    "3 on the pipe)")
    ap.add_argument("--schur-agg", type=int, default=0, help="aggregates per component of TRI_PMG_CS (default 96)")
    ap.add_argument("--lap-size", type=int, default=0, help="pressure Laplacian: -1 plain Chebyshev polynomial "
                    "(degree --cheb-l), else vertices per aggregate of its two-level cycle (default 32)")
    ap.add_argument("--lap-smooth", type=int, default=0, help="smoothing steps of the two-level pressure "
                    "Laplacian, each side (default 8)")
    ap.add_argument("--graphs", action="store_true", help="replay the Arnoldi steps from CUDA graphs (needs --no-timers)")
    ap.add_argument("--no-timers", action="store_true", help="time the steps without the per-class kernel timers "
                    "(no roofline entry); the timers disable graph replay")
    ap.add_argument("--krylov", default="fgmres", choices=["fgmres", "cocr"],
                    help="cocr: short-recurrence COCR (with a symmetric, block-diagonal --precond 0/1/2)")
    ap.add_argument("--stage", type=int, default=None, help="staged gathers: 0 autotuned (default), -1 never, "
                    "4/8/16/32 forced mode chunk")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true", help="skip the per-mode FP64 error and comparison")
    ap.add_argument("--kernel-case", action="store_true", help="short kernel sequence for profiler captures")
    ap.add_argument("--workload", default="pipe",
                    choices=["pipe", "batch", "guess", "fp64-permode", "bifurcation", "spmm", "validation"])
    ap.add_argument("--val-tol", type=float, default=1e-10, help="residual tolerance of the validation solves")
    ap.add_argument("--bif-h", type=float, default=0.038, help="voxel spacing of the bifurcation (0.038: ~6M nodes)")
    ap.add_argument("--fp64-modes", type=int, default=4)
    ap.add_argument("--batch-meshes", type=int, default=48)
    ap.add_argument("--batch-scale", type=float, default=1.0, help="scale of the batch's node counts")
    ap.add_argument("--guess-train", type=int, default=16, help="training morphs (x 32 modes)")
    ap.add_argument("--guess-test", type=int, default=3)
    ap.add_argument("--guess-steps", type=int, default=3000)
    args = ap.parse_args()
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.workload == "batch" and args.impl == "gpu":
        run_batch(args)
        return
    if args.workload == "guess" and args.impl == "gpu":
        run_guess(args)
        return
    if args.workload == "spmm" and args.impl == "gpu":
        run_spmm(args)
        return
    if args.workload == "bifurcation" and args.impl == "gpu":
        run_bifurcation(args)
        return
    if args.workload == "validation" and args.impl == "gpu":
        run_validation(args)
        return
    if args.workload == "fp64-permode" and args.impl == "gpu":
        run_fp64_permode(args)
        return
    if args.warmup < 3 and args.impl == "gpu":
        log("note: the timing rules ask for >= 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
