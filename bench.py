"""Benchmark: SU(3) Landau gauge fixing by checkerboard overrelaxation, 32^4.

One step = one complete gauge fixing of a seeded synthetic 32^4 field
(mean plaquette 0.60, Haar-random gauge, seeds 3/4) by the library's public
C ABI: FP32 12-real sweeps until theta < 1e-6, then FP64 sweeps until
theta < 1e-14 (omega = 1.7, theta checked every 25 sweeps).  The field is
restored from a resident pristine copy at the start of each step.

value = site updates per second over the timed steps (V x sweeps / time).
Extra keys: time to theta for mixed, mixed with the learned warm start (stored
parameters), mixed with a double-float finish and all-FP64, |F - F_FP64|, sweep
throughput and achieved HBM bandwidth per storage format, the roofline of the
dominant kernel, the CPU oracle baseline, end-to-end throughput with host
buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Landau OR site-updates/s at 32^4; time to θ<1e-14, mixed/learned vs FP64"
DIMS = (32, 32, 32, 32)
OMEGA = 1.7
THETA_SWITCH = 1e-6
THETA_TARGET = 1e-14
CHECK_EVERY = 25
MAX_ITER = 100_000
SEEDS = (3, 4)
PLAQ = 0.60
# FP64 peak of the FP64-bound sweeps: 152 SMs x 2 FP64 instructions per SM per clock x 2 flop
# (an FMA) x 2.07 GHz, the maximum SM clock (NVIDIA's nominal figure is 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; replicas of the same workload)
# ---------------------------------------------------------------------------
def dist_setup(ngpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def oracle_sample(U_np: np.ndarray, budget_s: float = 12.0):
    import oracle
    oracle.build()
    W = U_np.copy()
    t0 = time.perf_counter()
    oracle.or_sweeps(W, OMEGA, 0, 1)
    one = time.perf_counter() - t0
    n = max(1, min(500, int(budget_s / max(one, 1e-3)) - 1))
    t0 = time.perf_counter()
    oracle.or_sweeps(W, OMEGA, 0, n)
    dt = time.perf_counter() - t0
    V = int(np.prod(DIMS))
    return {"value": V * n / dt, "unit": "site-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} FP64 overrelaxation sweeps (omega {OMEGA}) of the 32^4 Landau field "
                      f"on the host cores, {dt:.1f} s"}


def headline_config(world: int) -> dict:
    """The benchmark's workload, shared by the GPU arm and the reference arm."""
    return {"workload": "landau-or-32^4 mixed: fp32-12 sweeps to theta<1e-6, fp64-18 to theta<1e-14",
            "lattice": list(DIMS), "omega": OMEGA, "plaquette": PLAQ, "seeds": list(SEEDS),
            "check_every": CHECK_EVERY, "theta_switch": THETA_SWITCH,
            "or_variant": "rational 19-flop form of g^omega (Alg. 1)",
            "theta": "(1/3V) sum tr Delta Delta^dagger, Delta = traceless sum_mu [A_mu(x) - A_mu(x-mu)], "
                     "A = (U - U^dagger)/2i",
            "theta_target": THETA_TARGET, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (fp64 field 604 MB, fp32 field 201 MB)"}


def reference_arm(args, rank, world):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_1209_4008_gb300 import synth
    dims = tuple(args.dims) if args.dims else DIMS
    U = synth.as_numpy(synth.make_field(dims, PLAQ, *SEEDS))
    import oracle
    oracle.build()
    W = U.copy()
    V = int(np.prod(dims))
    for _ in range(args.warmup):
        oracle.or_sweeps(W, OMEGA, 0, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.or_sweeps(W, OMEGA, 0, 1)
    dt = time.perf_counter() - t0
    value = V * args.steps / dt
    config = headline_config(world)
    if dims != DIMS:
        config.update(workload=f"landau-or-{'x'.join(map(str, dims))}", lattice=list(dims))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{args.steps} FP64 overrelaxation sweeps (omega {OMEGA}) of the "
                                   f"{'x'.join(map(str, dims))} field, one per step, from the same input; "
                                   f"the rate is per site update, as the GPU arm's"},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def make_ctx(gf, precision):
    c = gf.gf_create(DIMS, gf.GF_LANDAU)
    gf.gf_set_option(c, "precision", precision)
    gf.gf_set_option(c, "theta_switch", THETA_SWITCH)
    gf.gf_set_option(c, "check_every", CHECK_EVERY)
    gf.gf_set_option(c, "storage32", 12)
    gf.gf_set_option(c, "storage64", 18)
    gf.gf_set_option(c, "autotune", 1)
    gf.gf_set_stream(c, torch.cuda.current_stream())
    return c


def sweep_throughput(gf, ctx, field, precision, storage_key, storage, nsweeps=200, warm=20):
    """Average half-sweep kernel time (CUDA events on the launch stream)."""
    gf.gf_set_option(ctx, storage_key, storage)
    gf.gf_upload(ctx, field, precision)
    tps, block = gf.gf_autotune(ctx)
    gf.gf_upload(ctx, field, precision)
    gf.gf_or_sweeps(ctx, OMEGA, warm)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    gf.gf_or_sweeps(ctx, OMEGA, nsweeps)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return ms / (2 * nsweeps), tps, block


def gpu_arm(args, rank, world, local):
    from paper_1209_4008_gb300 import gf, synth
    gf.load()
    dev = torch.device("cuda", local if world > 1 else 0)
    V = int(np.prod(DIMS))
    Vh = V // 2
    pristine = synth.make_field(DIMS, PLAQ, *SEEDS, device=dev)
    work = torch.empty_like(pristine)

    ctx = make_ctx(gf, gf.GF_MIXED)
    gf.gf_set_option(ctx, "kernel_timing", 1)  # events around the sweep kernels, inside the graphs

    def step(c):
        work.copy_(pristine)
        conv, it, F, th = gf.gf_overrelax(c, work, OMEGA, THETA_TARGET, MAX_ITER)
        if not conv:
            raise RuntimeError(f"not converged: theta={th}")
        return it, F, th

    for _ in range(args.warmup):
        step(ctx)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweeps = 0
    checks = 0
    ms32 = ms64 = 0.0
    sw32 = sw64 = 0
    kms = {"fp32": 0.0, "fp64": 0.0}
    kn = {"fp32": 0, "fp64": 0}
    F_mixed = th_mixed = None
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local if world > 1 else 0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            it, F_mixed, th_mixed = step(ctx)
            sweeps += it
            checks += gf.gf_get_stat(ctx, "checks")
            ms32 += gf.gf_get_stat(ctx, "ms_fp32")
            ms64 += gf.gf_get_stat(ctx, "ms_fp64")
            sw32 += int(gf.gf_get_stat(ctx, "sweeps_fp32"))
            sw64 += int(gf.gf_get_stat(ctx, "sweeps_fp64"))
            for ph in ("fp32", "fp64"):
                kms[ph] += gf.gf_get_stat(ctx, f"ms_sweep_kernels_{ph}")
                kn[ph] += int(gf.gf_get_stat(ctx, f"sweep_launches_{ph}"))
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    total_su = world * V * sweeps  # replicas: every rank did the same number of sweeps
    value = total_su / (ms / 1e3)
    # kernels launched per step: 2 per sweep + reductions (2) per check (+1 reunitarise per
    # FP32 check) + encode, identity, apply-gauge, decode + two initial measurements
    fp32_checks = sw32 / CHECK_EVERY
    launches = int(2 * sweeps + 2 * checks + fp32_checks + args.steps * (4 + 4))

    # plaquette of the input and of each leg's result: every sweep is a gauge transformation, so
    # the change measures the rounding drift a leg leaves in the links
    P_in = gf.gf_plaquette(ctx, pristine)
    dP_mixed = abs(gf.gf_plaquette(ctx, work) - P_in)

    # all-FP64 reference solve (time to theta), once, outside the timed steps
    ctx64 = make_ctx(gf, gf.GF_FP64)
    work.copy_(pristine)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv64, it64, F64, th64 = gf.gf_overrelax(ctx64, work, OMEGA, THETA_TARGET, MAX_ITER)
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t0
    dP_fp64 = abs(gf.gf_plaquette(ctx64, work) - P_in)

    # per-format half-sweep kernel times on the same field
    thr = {}
    for name, prec, key, st, nbytes in (("fp32_12", gf.GF_FP32, "storage32", 12, 768),
                                        ("fp32_18", gf.GF_FP32, "storage32", 18, 1152),
                                        ("fp64_12", gf.GF_FP64, "storage64", 12, 1536),
                                        ("fp64_18", gf.GF_FP64, "storage64", 18, 2304),
                                        ("df64_18", gf.GF_FP64, "fp64_arith", 1, 2304)):
        # 200 timed sweeps after 20 warm-up sweeps, for every storage format
        t_half, tps, block = sweep_throughput(gf, ctx64, pristine, prec, key, st, nsweeps=200, warm=20)
        thr[name] = {"ms_per_half_sweep": t_half, "gsu_per_s": Vh / (t_half * 1e-3) / 1e9,
                     "algorithmic_gbs": Vh * nbytes / (t_half * 1e-3) / 1e9,
                     "bytes_per_site_update": nbytes,
                     "threads_per_site": tps, "block": block}
        if key == "fp64_arith":
            gf.gf_set_option(ctx64, "fp64_arith", 0)
    gf.gf_set_option(ctx64, "storage32", 12)
    gf.gf_set_option(ctx64, "storage64", 18)

    # mixed policy with the FP64 phase in double-float arithmetic (FP32 pipe), once
    ctxdf = make_ctx(gf, gf.GF_MIXED)
    gf.gf_set_option(ctxdf, "fp64_arith", 1)
    work.copy_(pristine)
    gf.gf_overrelax(ctxdf, work, OMEGA, THETA_TARGET, MAX_ITER)  # warm-up: autotune, graphs
    work.copy_(pristine)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    convdf, itdf, Fdf, thdf = gf.gf_overrelax(ctxdf, work, OMEGA, THETA_TARGET, MAX_ITER)
    torch.cuda.synchronize()
    t_df = time.perf_counter() - t0
    dP_df = abs(gf.gf_plaquette(ctxdf, work) - P_in)

    # the mixed policy with the learned warm start (stored parameters), once
    learned_row = None
    if os.path.exists(WEIGHTS):
        net = gf.gf_net_create(DIMS)
        gf.gf_net_set_stream(net, torch.cuda.current_stream())
        gf.gf_net_set_params(net, np.load(WEIGHTS).astype(np.float32))
        ctxl = make_ctx(gf, gf.GF_MIXED)
        gf.gf_set_net(ctxl, net)
        gf.gf_set_option(ctxl, "learned_repeat", args.learned_repeat)
        gf.gf_set_option(ctxl, "learned_factor", args.learned_factor)
        work.copy_(pristine)
        gf.gf_overrelax(ctxl, work, OMEGA, THETA_TARGET, MAX_ITER)  # warm-up
        work.copy_(pristine)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        convl, itl, Fl, thl = gf.gf_overrelax(ctxl, work, OMEGA, THETA_TARGET, MAX_ITER)
        torch.cuda.synchronize()
        learned_row = {"learned_s": time.perf_counter() - t0, "sweeps_learned": itl,
                       "sweeps_fp64_phase_learned": gf.gf_get_stat(ctxl, "sweeps_fp64"),
                       "F_learned": Fl, "dF_learned": abs(Fl - F64), "theta_learned": thl,
                       "ms_network": gf.gf_get_stat(ctxl, "ms_learned"),
                       "network_applications": 1 + (gf.gf_get_stat(ctxl, "learned_applications")
                                                    if args.learned_repeat else 0),
                       "weights": os.path.relpath(WEIGHTS, ROOT)}

    # the mixed policy with FP32 restarts (option fp32_restarts), once with a native FP64 finish
    # and once with the double-float finish (fp64_arith 1: the transformation tracked as E = g - 1
    # and applied to the FP64 field in FP64, so the result stays an exact FP64 gauge transform)
    restart_row = {}
    for tag, arith in (("restarts", 0), ("restarts_df64", 1)):
        if args.fp32_restarts <= 0:
            break
        ctxr = make_ctx(gf, gf.GF_MIXED)
        gf.gf_set_option(ctxr, "fp32_restarts", args.fp32_restarts)
        gf.gf_set_option(ctxr, "theta_switch", args.restart_switch)
        gf.gf_set_option(ctxr, "fp64_arith", arith)
        work.copy_(pristine)
        gf.gf_overrelax(ctxr, work, OMEGA, THETA_TARGET, MAX_ITER)  # warm-up
        work.copy_(pristine)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        convr, itr, Fr, thr_ = gf.gf_overrelax(ctxr, work, OMEGA, THETA_TARGET, MAX_ITER)
        torch.cuda.synchronize()
        restart_row.update({
            f"{tag}_s": time.perf_counter() - t0, f"sweeps_{tag}": itr,
            f"sweeps_fp32_{tag}": gf.gf_get_stat(ctxr, "sweeps_fp32"),
            f"sweeps_fp64_phase_{tag}": gf.gf_get_stat(ctxr, "sweeps_fp64"),
            f"theta_after_fp32_stages_{tag}": gf.gf_get_stat(ctxr, "theta_after_restarts"),
            f"F_{tag}": Fr, f"dF_{tag}": abs(Fr - F64), f"dF_vs_exact_{tag}": abs(Fr - Fdf),
            f"theta_{tag}": thr_, f"converged_{tag}": convr,
            f"dP_{tag}": abs(gf.gf_plaquette(ctxr, work) - P_in)})
        if arith:
            restart_row[f"sweeps_df64_{tag}"] = gf.gf_get_stat(ctxr, "sweeps_df64")
    if restart_row:
        restart_row.update({"restarts": args.fp32_restarts, "restart_theta_switch": args.restart_switch})

    # measured FMA peaks (own kernel, CUDA events), clocks sampled meanwhile: the FP64 one is the
    # denominator of the FP64 sweep's roofline
    with ClockSampler(local if world > 1 else 0) as clk_peak:
        fp64_peak, _ = gf.gf_fma_peak(True, 4000)
        fp32_peak, _ = gf.gf_fma_peak(False, 200000)
    peak_clocks = clk_peak.summary()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    host = torch.empty(pristine.shape, dtype=pristine.dtype, pin_memory=True)
    e2e_ms = 0.0
    e2e_sweeps = 0
    for _ in range(max(1, args.steps)):
        host.copy_(pristine.cpu())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, it, _, _ = gf.gf_overrelax(ctx, host.data_ptr(), OMEGA, THETA_TARGET, MAX_ITER)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_sweeps += it
    e2e_ms = max_over_ranks(e2e_ms, world)
    e2e_value = world * V * e2e_sweeps / (e2e_ms / 1e3)

    # DRAM bytes (read + write) per launch of the FP64 phase's half-sweep from ncu captures
    # (profiles/or_half_sweep_fp64_18_32x32x32x32.md): valid for the configurations captured there,
    # the accumulate form near convergence with each register budget at block 128; null for any other
    acc = gf.gf_get_stat(ctx, "accumulate_form") == 1
    traffic64 = {255: 1169.9e6, 168: 1335.4e6, 128: 1495.8e6}.get(
        int(gf.gf_get_stat(ctx, "acc_registers"))) if acc else None
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    # dominant kernel of the step: the half-sweep of the phase whose kernels took longer; its
    # average launch duration comes from the events recorded around the sweep kernels of every
    # check chunk of the timed steps (on the launching stream, inside the graphs)
    ph = "fp64" if kms["fp64"] >= kms["fp32"] else "fp32"
    dom = "fp64_18" if ph == "fp64" else "fp32_12"
    t_launch = kms[ph] / max(1, kn[ph]) * 1e-3  # seconds per half-sweep launch
    gbs = Vh * thr[dom]["bytes_per_site_update"] / t_launch / 1e9
    roof = {"kernel": f"or_half_sweep[{dom}]", "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": (gbs / hbm) if hbm else None, "traffic": None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if hbm else "fallback 6800",
            "launch_ms": t_launch * 1e3, "launches_timed": kn[ph],
            "isolated_launch_ms": thr[dom]["ms_per_half_sweep"]}
    if ph == "fp64":
        flops = Vh * 2253 / t_launch / 1e12
        roof.update({"bound": "alu", "achieved": flops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": flops / fp64_peak,
                     "peak_source": "measured: gf_fma_peak (FP64 FMA chains, 8 blocks per SM, CUDA events), "
                                    f"median SM clock {peak_clocks.get('sm_mhz')} MHz while measured",
                     "derived_peak": FP64_PEAK_TFLOPS,
                     "derived_peak_source": "152 SMs x 2 FP64 instructions per clock (ncu pipe peak) x 2 flop "
                                            "per FMA x 2.07 GHz maximum SM clock",
                     "fp32_fma_peak": fp32_peak,
                     "hbm_gbs": gbs, "hbm_frac": gbs / hbm if hbm else None,
                     "traffic": traffic64, "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "registers_per_thread": int(gf.gf_get_stat(ctx, "acc_registers")) if acc else None,
                     "algorithmic_bytes": Vh * thr[dom]["bytes_per_site_update"]})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(synth.as_numpy(pristine))

    line = {
        "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": headline_config(world),
        "time_to_theta": {"mixed_s": ms / args.steps / 1e3, "fp64_s": t_fp64,
                          "sweeps_mixed": sweeps / args.steps, "sweeps_fp32": sw32 / args.steps,
                          "sweeps_fp64_phase": sw64 / args.steps, "sweeps_all_fp64": it64,
                          "F_mixed": F_mixed, "F_fp64": F64, "dF": abs(F_mixed - F64),
                          "theta_mixed": th_mixed, "theta_fp64": th64,
                          "dP_mixed": dP_mixed, "dP_fp64": dP_fp64,
                          "mixed_df64_s": t_df, "sweeps_mixed_df64": itdf, "F_mixed_df64": Fdf,
                          "dF_mixed_df64": abs(Fdf - F64), "theta_mixed_df64": thdf, "dP_mixed_df64": dP_df,
                          "exact_reference": "F_mixed_df64: the double-float finish applies the tracked "
                                             "transformation to the FP64 field once, in FP64 (no drift)",
                          "phase_ms": {"fp32": ms32 / args.steps, "fp64": ms64 / args.steps},
                          **(learned_row or {}), **(restart_row or {})},
        "sweep_throughput": thr,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "site-updates/s",
                "h2d_bytes_per_step": int(pristine.numel() * 16),
                "d2h_bytes_per_step": int(pristine.numel() * 16)},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


FORMATS = {"fp32_12": (1, "storage32", 12, 768), "fp32_18": (1, "storage32", 18, 1152),
           "fp64_12": (0, "storage64", 12, 1536), "fp64_18": (0, "storage64", 18, 2304),
           "df64_18": (0, "fp64_arith", 1, 2304)}


def kernel_only(args):
    """One storage format's OR half-sweep on the 32^4 field, for profiling:
    warmup sweeps, then timed sweeps; prints the average half-sweep time."""
    from paper_1209_4008_gb300 import gf, synth
    prec_code, key, st, nbytes = FORMATS[args.kernel]
    prec = gf.GF_FP64 if prec_code == 0 else gf.GF_FP32
    dims = tuple(args.dims) if args.dims else DIMS
    field = synth.make_field(dims, PLAQ, *SEEDS, device="cuda")
    c = gf.gf_create(dims, gf.GF_LANDAU)
    gf.gf_set_option(c, key, st)
    if args.tps == 0:
        gf.gf_set_option(c, "variant", 2)  # accumulate form, one thread per site
        if args.acc_regs:
            gf.gf_set_option(c, "acc_registers", args.acc_regs)
    else:
        gf.gf_set_option(c, "variant", 1)
        gf.gf_set_option(c, "threads_per_site", args.tps)
    gf.gf_set_option(c, "block", args.block)
    gf.gf_set_option(c, "use_graphs", 0)
    gf.gf_set_stream(c, torch.cuda.current_stream())
    if args.theta_start:
        # bring the field near convergence first (the state of the FP64 phase of the
        # mixed policy) with the per-subgroup form, so that the profiled launches of
        # the chosen form all come after it
        pre = gf.gf_create(dims, gf.GF_LANDAU)
        gf.gf_set_option(pre, "variant", 1)
        gf.gf_set_option(pre, "threads_per_site", 2)
        gf.gf_set_option(pre, "check_every", CHECK_EVERY)
        gf.gf_set_stream(pre, torch.cuda.current_stream())
        gf.gf_overrelax(pre, field, OMEGA, args.theta_start, MAX_ITER)
    gf.gf_upload(c, field, prec)

    def sweeps(n, first):
        if args.sa_temp is None:
            gf.gf_or_sweeps(c, OMEGA, n)
        else:  # heatbath half-sweeps at the fixed temperature
            for k in range(first, first + n):
                gf.gf_sa_half_sweep(c, 0, args.sa_temp, 9, k)
                gf.gf_sa_half_sweep(c, 1, args.sa_temp, 9, k)

    sweeps(args.warmup, 0)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    sweeps(args.steps, args.warmup)
    e1.record(s)
    torch.cuda.synchronize()
    t_half = e0.elapsed_time(e1) / (2 * args.steps)
    Vh = int(np.prod(dims)) // 2
    print(json.dumps({"kernel": args.kernel + ("" if args.sa_temp is None else f" heatbath T={args.sa_temp}"),
                      "dims": list(dims), "tps": args.tps, "block": args.block, "acc_regs": args.acc_regs,
                      "theta_start": args.theta_start or None,
                      "ms_per_half_sweep": t_half, "gsu_per_s": Vh / (t_half * 1e-3) / 1e9,
                      "algorithmic_gbs": Vh * nbytes / (t_half * 1e-3) / 1e9}), flush=True)


BATCH_SIZES = (8, 12, 16, 24)


def batched(args):
    """64 lattices (16 each of 8^4, 12^4, 16^4, 24^4; seeds 100..163; plaquette
    uniform in [0.55, 0.62] from seed 99), mixed precision, omega 1.7, theta <
    1e-12: one persistent launch per precision phase under a CUDA graph versus a
    loop of single-lattice calls, with the FP64 phase in native FP64 and in
    double-float arithmetic (fp64_arith 1: E = g - 1 tracked, applied in FP64).
    Prints one JSON object (not the headline line)."""
    from paper_1209_4008_gb300 import gf, synth
    dims = [(L, L, L, L) for L in BATCH_SIZES for _ in range(16)]
    plaq = synth.batched_plaquettes(len(dims))
    pristine = [synth.make_field(d, plaq[k], 100 + k, 1100 + k, device="cuda") for k, d in enumerate(dims)]
    work = [p.clone() for p in pristine]
    target, max_iter = 1e-12, 100_000

    def restore():
        for w, p in zip(work, pristine):
            w.copy_(p)

    out = {"workload": "batched-landau 64 lattices (16 each of 8^4,12^4,16^4,24^4), mixed, theta<1e-12",
           "sites": int(sum(np.prod(d) for d in dims))}
    F_native = None
    for arith in (0, 1):
        b = gf.gf_batch_create(dims, gf.GF_LANDAU)
        gf.gf_batch_set_option(b, "precision", gf.GF_MIXED)
        gf.gf_batch_set_option(b, "check_every", CHECK_EVERY)
        gf.gf_batch_set_option(b, "fp64_arith", arith)
        gf.gf_batch_set_stream(b, torch.cuda.current_stream())
        tps, block = gf.gf_batch_autotune(b, work)
        restore()
        gf.gf_batch_overrelax(b, work, OMEGA, target, max_iter)  # warm-up: capture the graph
        restore()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, iters, F, th = gf.gf_batch_overrelax(b, work, OMEGA, target, max_iter)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        su = sum(i * int(np.prod(d)) for i, d in zip(iters, dims))
        stats = {k: gf.gf_batch_get_stat(b, k) for k in ("ms_fp32", "ms_fp64", "grid_fp32", "grid_fp64", "tiles",
                                                          "threads_per_site", "block")}
        if arith:
            stats["grid_df64"] = gf.gf_batch_get_stat(b, "grid_df64")
        gf.gf_batch_destroy(b)
        # per-lattice loop through the single-lattice entry point
        ctxs = []
        for d in dims:
            c = gf.gf_create(d, gf.GF_LANDAU)
            gf.gf_set_option(c, "precision", gf.GF_MIXED)
            gf.gf_set_option(c, "check_every", CHECK_EVERY)
            gf.gf_set_option(c, "autotune", 1)
            gf.gf_set_option(c, "fp64_arith", arith)
            gf.gf_set_stream(c, torch.cuda.current_stream())
            ctxs.append(c)
        restore()
        for c, w in zip(ctxs, work):  # warm-up (autotune, graphs)
            gf.gf_overrelax(c, w, OMEGA, target, max_iter)
        restore()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        su_loop = 0
        for c, w, d in zip(ctxs, work, dims):
            conv, it, _, _ = gf.gf_overrelax(c, w, OMEGA, target, max_iter)
            su_loop += it * int(np.prod(d))
        torch.cuda.synchronize()
        t_loop = time.perf_counter() - t0
        for c in ctxs:
            gf.gf_destroy(c)
        if F_native is None:
            F_native = F
        out["df64" if arith else "native"] = {
            "converged": rc == gf.GF_OK,
            "persistent": {"s": t_batch, "site_updates": su, "su_per_s": su / t_batch,
                           "threads_per_site": tps, "block": block, **stats},
            "loop": {"s": t_loop, "site_updates": su_loop, "su_per_s": su_loop / t_loop},
            "speedup": t_loop / t_batch, "sweeps_min_max": [min(iters), max(iters)],
            "max_dF_vs_native": max(abs(a - c) for a, c in zip(F, F_native))}
    print(json.dumps(out), flush=True)


WEIGHTS = os.path.join(ROOT, "paper_1209_4008_gb300", "weights", "warm_start_16x16x16x16.npy")


def learned(args):
    """Learned warm start: training pairs from the solver on 16^4 fields (seeds
    1000.., plaquette 0.60), GPU training, then fixing fresh 32^4 fields (seeds
    5000..) to theta < 1e-14 with the mixed policy with and without the
    network at the FP32 -> FP64 switch.  Prints one JSON object."""
    from paper_1209_4008_gb300 import gf, learned as L, synth
    t_start = time.perf_counter()
    train_dims = (16, 16, 16, 16)
    t_data = t_train = 0.0
    hist, val = [], None
    if args.weights:
        params = np.load(args.weights).astype(np.float32)
    else:
        ctx = gf.gf_create(train_dims, gf.GF_LANDAU)
        gf.gf_set_option(ctx, "autotune", 1)
        pairs = []
        t0 = time.perf_counter()
        for k in range(args.pairs):
            U = synth.make_field(train_dims, PLAQ, 1000 + k, 3000 + k, device="cuda")
            pairs.append(L.make_pair(ctx, U, theta_switch=THETA_SWITCH, label_theta=1e-12,
                                     check_every=CHECK_EVERY))
        t_data = time.perf_counter() - t0
        nval = max(1, args.pairs // 10)
        train_set, val_set = pairs[nval:], pairs[:nval]
        net = gf.gf_net_create(train_dims)
        gf.gf_net_set_params(net, L.init_params(0))
        t0 = time.perf_counter()
        hist = L.train(net, train_set, epochs=args.epochs, lr=args.lr, lr_decay=args.lr_decay,
                       log=lambda m: print(m, file=sys.stderr, flush=True))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        val = L.validation_loss(net, val_set)
        params = np.zeros(gf.gf_net_param_count(), dtype=np.float32)
        gf.gf_net_get_params(net, params)
    if args.save:
        os.makedirs(os.path.dirname(os.path.abspath(args.save)), exist_ok=True)
        np.save(args.save, params)
    # evaluation on 32^4 fields
    big = gf.gf_net_create(DIMS)
    gf.gf_net_set_params(big, params)
    res = []
    for k in range(args.eval_fields):
        pristine = synth.make_field(DIMS, PLAQ, 5000 + k, 6000 + k, device="cuda")
        row = {}
        for mode in ("mixed", "learned"):
            c = make_ctx(gf, gf.GF_MIXED)
            gf.gf_set_option(c, "fp64_arith", args.eval_arith)
            if mode == "learned":
                gf.gf_set_net(c, big)
                gf.gf_set_option(c, "learned_repeat", args.learned_repeat)
                gf.gf_set_option(c, "learned_factor", args.learned_factor)
            work = pristine.clone()
            gf.gf_overrelax(c, work, OMEGA, THETA_TARGET, MAX_ITER)  # warm-up (autotune, graphs)
            work.copy_(pristine)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            conv, it, F, th = gf.gf_overrelax(c, work, OMEGA, THETA_TARGET, MAX_ITER)
            torch.cuda.synchronize()
            row[mode] = {"s": time.perf_counter() - t1, "sweeps": it, "F": F, "theta": th, "converged": conv,
                         "sweeps_fp64": gf.gf_get_stat(c, "sweeps_fp64")}
            if mode == "learned":
                row[mode]["ms_network"] = gf.gf_get_stat(c, "ms_learned")
                row[mode]["theta_before"] = gf.gf_get_stat(c, "theta_before_learned")
                row[mode]["theta_after"] = gf.gf_get_stat(c, "theta_after_learned")
                row[mode]["applications"] = 1 + (gf.gf_get_stat(c, "learned_applications")
                                                 if args.learned_repeat else 0)
        row["dF"] = abs(row["learned"]["F"] - row["mixed"]["F"])
        res.append(row)
    mean = lambda key, mode: float(np.mean([r[mode][key] for r in res]))

    def mmm(vals):
        return {"min": float(np.min(vals)), "median": float(np.median(vals)), "max": float(np.max(vals))}
    saved_sweeps = [r["mixed"]["sweeps_fp64"] - r["learned"]["sweeps_fp64"] for r in res]
    saved_s = [r["mixed"]["s"] - r["learned"]["s"] for r in res]
    print(json.dumps({
        "workload": (f"learned warm start: stored parameters {args.weights}" if args.weights else
                     f"learned warm start: {args.pairs} solver pairs on 16^4 (plaquette 0.60), "
                     f"{args.epochs} epochs Adam") + f"; test on {args.eval_fields} fresh 32^4 fields, theta<1e-14",
        "data_s": t_data, "train_s": t_train, "train_loss": hist, "val_loss": val,
        "eval": res,
        "mean": {"mixed_s": mean("s", "mixed"), "learned_s": mean("s", "learned"),
                 "mixed_fp64_sweeps": mean("sweeps_fp64", "mixed"),
                 "learned_fp64_sweeps": mean("sweeps_fp64", "learned")},
        "fp64_phase_sweeps_saved": mmm(saved_sweeps), "seconds_saved": mmm(saved_s),
        "time_ratio": mmm([r["learned"]["s"] / r["mixed"]["s"] for r in res]),
        "max_dF": float(max(r["dF"] for r in res)), "all_dF_below_1e-10": all(r["dF"] < 1e-10 for r in res),
        "fp64_arith": args.eval_arith,
        "total_s": time.perf_counter() - t_start}), flush=True)


COULOMB_DIMS = (48, 48, 48, 96)


def coulomb(args):
    """Coulomb gauge on 48^3 x 96 (FP64 links, 6.1 GB), plaquette 0.58, seeds
    7000+k / 8000+k: simulated annealing (heatbath sweeps with T falling
    linearly from 1.45 to 0.01, Philox key 9000+k) then FP64 overrelaxation at
    omega 1.7 to theta < 1e-13; the same start fixed by overrelaxation alone
    for comparison.  Reports the final F of every seed and their distribution.
    Prints one JSON object."""
    from paper_1209_4008_gb300 import gf, synth
    t_start = time.perf_counter()
    target = 1e-13
    ctx = gf.gf_create(COULOMB_DIMS, gf.GF_COULOMB)
    gf.gf_set_option(ctx, "precision", gf.GF_FP64)
    gf.gf_set_option(ctx, "storage64", 18)
    gf.gf_set_option(ctx, "check_every", CHECK_EVERY)
    gf.gf_set_option(ctx, "autotune", 1)
    # --fast: double-float sweeps (E tracked, applied in FP64: exact FP64 gauge transforms) and the
    # FP32 reading of the heatbath draw
    gf.gf_set_option(ctx, "fp64_arith", 1 if args.fast else 0)
    gf.gf_set_option(ctx, "sa_draw", 1 if args.fast else 0)
    gf.gf_set_stream(ctx, torch.cuda.current_stream())
    V = int(np.prod(COULOMB_DIMS))
    rows = []
    for k in range(args.seeds):
        pristine = synth.make_field(COULOMB_DIMS, 0.58, 7000 + k, 8000 + k, device="cuda")
        row = {"seed": k, "plaquette": gf.gf_plaquette(ctx, pristine)}
        for leg in ("sa+or", "or") if k < args.or_seeds else ("sa+or",):
            U = pristine.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if leg == "sa+or":
                rc = gf.gf_anneal(ctx, U, 1.45, 0.01, args.sa_sweeps, 9000 + k, allow_reject=True)
                torch.cuda.synchronize()
                row["sa_s"] = time.perf_counter() - t0
                row["sa_rejects"] = gf.gf_get_stat(ctx, "sa_rejects")
                row["F_after_sa"] = gf.gf_functional(ctx, U)
                t0 = time.perf_counter()
            conv, it, F, th = gf.gf_overrelax(ctx, U, OMEGA, target, MAX_ITER)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            F_t, th_t = gf.gf_measure_timeslices(ctx)
            row[leg] = {"or_s": dt, "sweeps": it, "F": F, "theta": th, "converged": conv,
                        "theta_timeslice_max": float(th_t.max()), "F_timeslice_min_max": [float(F_t.min()),
                                                                                          float(F_t.max())],
                        "su_per_s": V * it / dt, "dplaq": abs(gf.gf_plaquette(ctx, U) - row["plaquette"])}
            del U
        rows.append(row)
        log(json.dumps(row))
    F_sa = [r["sa+or"]["F"] for r in rows]
    F_or = [r["or"]["F"] for r in rows if "or" in r]
    stat = lambda v: {"mean": float(np.mean(v)), "std": float(np.std(v)), "min": float(min(v)), "max": float(max(v))}
    print(json.dumps({
        "workload": f"coulomb 48^3x96 FP64, plaquette 0.58, {args.sa_sweeps} heatbath sweeps T 1.45->0.01, "
                    f"then OR omega 1.7 to theta<1e-13; {args.seeds} seeds"
                    + ("; double-float sweeps (exact FP64 result), FP32 heatbath draw" if args.fast else ""),
        "seeds": rows, "F_sa_or": stat(F_sa), "F_or": stat(F_or) if F_or else None,
        "sa_higher_F": int(sum(r["sa+or"]["F"] > r["or"]["F"] for r in rows if "or" in r)),
        "or_sweeps_saved_by_sa": [r["or"]["sweeps"] - r["sa+or"]["sweeps"] for r in rows if "or" in r],
        "sa_sweeps_per_s": float(np.mean([args.sa_sweeps / r["sa_s"] for r in rows])),
        "total_s": time.perf_counter() - t_start}), flush=True)


def net_kernels(args):
    """The warm-start network's convolutions on one lattice (default 32^4):
    forward and one training step (forward, loss, backward data and weights,
    Adam) on random BF16 inputs, CUDA events on the launch stream; the
    tensor-core rate counts 2 x 81 x C_in x C_out flop per site and layer.
    Prints one JSON object."""
    from paper_1209_4008_gb300 import gf, learned as L
    dims = tuple(args.dims) if args.dims else DIMS
    V = int(np.prod(dims))
    ch = gf.NET_CHANNELS
    layer_flop = [2 * 81 * ch[l] * ch[l + 1] for l in range(4)]
    fwd_flop = V * sum(layer_flop)
    # training: forward, data gradients of layers 2-4, weight gradients of all layers
    train_flop = V * (2 * sum(layer_flop) + sum(layer_flop[1:]))
    net = gf.gf_net_create(dims)
    gf.gf_net_set_stream(net, torch.cuda.current_stream())
    gf.gf_net_set_params(net, L.init_params(0))
    gf.gf_net_set_option(net, "conv_halo", args.conv_halo)
    gen = torch.Generator(device="cuda").manual_seed(7)
    feats = torch.randn(V, ch[0], device="cuda", generator=gen).to(torch.bfloat16)
    target = 0.1 * torch.randn(V, ch[4], device="cuda", generator=gen)
    out = torch.empty(V, ch[4], device="cuda", dtype=torch.float32)
    s = torch.cuda.current_stream()
    res = {}
    for name, fn, flop in (("forward", lambda: gf.gf_net_forward(net, feats, out), fwd_flop),
                           ("train_step", lambda: gf.gf_net_train_step(net, feats, target, 1e-4), train_flop)):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(args.steps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms": ms, "tflops": flop / (ms * 1e-3) / 1e12}
    pk = peaks()
    bf16 = pk.get("bf16_tflops")
    for r in res.values():
        r["frac_of_bf16_peak"] = r["tflops"] / bf16 if bf16 else None
    print(json.dumps({"workload": f"warm-start network {'x'.join(map(str, dims))}, channels {list(ch)}"
                                  + {0: ", per-tap gather convolutions", 1: ", x-line convolutions",
                                     2: ", halo-tile convolutions"}[args.conv_halo],
                      "sites": V, "flop_forward": fwd_flop, "flop_train_step": train_flop,
                      "bf16_peak_tflops": bf16, **res}), flush=True)


def mag(args):
    """Maximally Abelian gauge on the 32^4 field (seeds 3/4, plaquette 0.60):
    overrelaxation omega 1.7 to theta_MAG < 1e-10 with the FP64 and the mixed
    policy (FP32 to 1e-5), per-subgroup site update (autotuned threads per
    site).  Prints one JSON object."""
    from paper_1209_4008_gb300 import gf, synth
    pristine = synth.make_field(DIMS, PLAQ, *SEEDS, device="cuda")
    V = int(np.prod(DIMS))
    out = {"workload": "maximally Abelian gauge 32^4, omega 1.7, theta_MAG < 1e-10"}
    for name, prec in (("fp64", gf.GF_FP64), ("mixed", gf.GF_MIXED)):
        c = gf.gf_create(DIMS, gf.GF_MAG)
        gf.gf_set_option(c, "precision", prec)
        gf.gf_set_option(c, "theta_switch", 1e-5)
        gf.gf_set_option(c, "check_every", CHECK_EVERY)
        gf.gf_set_option(c, "autotune", 1)
        gf.gf_set_option(c, "kernel_timing", 1)
        gf.gf_set_stream(c, torch.cuda.current_stream())
        work = pristine.clone()
        gf.gf_overrelax(c, work, OMEGA, 1e-10, 20_000)  # warm-up: autotune, graphs
        work.copy_(pristine)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, it, F, th = gf.gf_overrelax(c, work, OMEGA, 1e-10, 20_000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        k64 = gf.gf_get_stat(c, "ms_sweep_kernels_fp64") / max(1.0, gf.gf_get_stat(c, "sweep_launches_fp64"))
        out[name] = {"s": dt, "sweeps": it, "F": F, "theta": th, "converged": conv,
                     "su_per_s": V * it / dt, "ms_fp64_half_sweep": k64,
                     "threads_per_site": gf.gf_get_stat(c, "threads_per_site"),
                     "dplaq": abs(gf.gf_plaquette(c, work) - gf.gf_plaquette(c, pristine))}
    out["dF"] = abs(out["fp64"]["F"] - out["mixed"]["F"])
    print(json.dumps(out), flush=True)


def thermal(args):
    """Gauge fixing of a thermalised field: the 32^4 synthetic field (seeds 3/4)
    evolved with the Wilson action at beta = 6.1 (the paper's ensembles, Sec. 5)
    by --therm compound sweeps (one heatbath and 4 overrelaxation sweeps each),
    then fixed to Landau gauge (omega 1.7, theta < 1e-14) with the mixed and the
    all-FP64 policies.  Prints one JSON object."""
    from paper_1209_4008_gb300 import gf, synth
    beta, n_or = 6.1, 4
    U = synth.make_field(DIMS, PLAQ, *SEEDS, device="cuda")
    V = int(np.prod(DIMS))
    g = gf.gf_create(DIMS, gf.GF_LANDAU)
    gf.gf_set_stream(g, torch.cuda.current_stream())
    gf.gf_generate(g, U, beta, 2, n_or, 21, 0)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gf.gf_generate(g, U, beta, args.therm, n_or, 21, 2)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    plaq = gf.gf_plaquette(g, U)
    out = {"workload": f"32^4 Wilson beta={beta}, {args.therm} compound sweeps (1 heatbath + {n_or} OR), "
                       f"then Landau OR omega 1.7 to theta<1e-14",
           "generation": {"s": t_gen, "ms_per_compound_sweep": 1e3 * t_gen / max(1, args.therm),
                          "link_updates_per_s": 4 * V * (1 + n_or) * args.therm / t_gen, "plaquette": plaq}}
    pristine = U.clone()
    for name, prec in (("mixed", gf.GF_MIXED), ("fp64", gf.GF_FP64)):
        c = make_ctx(gf, prec)
        work = pristine.clone()
        gf.gf_overrelax(c, work, OMEGA, THETA_TARGET, MAX_ITER)  # warm-up
        work.copy_(pristine)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, it, F, th = gf.gf_overrelax(c, work, OMEGA, THETA_TARGET, MAX_ITER)
        torch.cuda.synchronize()
        out[name] = {"s": time.perf_counter() - t0, "sweeps": it, "F": F, "theta": th, "converged": conv,
                     "sweeps_fp64": gf.gf_get_stat(c, "sweeps_fp64")}
    out["dF"] = abs(out["mixed"]["F"] - out["fp64"]["F"])
    print(json.dumps(out), flush=True)


def sr_study(args):
    """Overrelaxation against stochastic relaxation (Sec. 1 names both; Sec. 5
    tunes their parameters by the iterations to theta < 1e-12): sweeps and
    time to theta < 1e-12 for omega in --omegas (overrelaxation) and p in
    --probs (stochastic relaxation: the relaxation element, or with
    probability p its square), on the 32^4 synthetic field (seeds 3/4) and on
    that field thermalised at beta = 6.1 (--therm compound sweeps).  FP64
    storage with double-float arithmetic (fp64_arith 1), theta checked every
    25 sweeps.  Prints one JSON object."""
    from paper_1209_4008_gb300 import gf, synth
    target, max_iter = 1e-12, args.sr_max_iter
    base = synth.make_field(DIMS, PLAQ, *SEEDS, device="cuda")
    fields = {"synthetic": base}
    if args.therm > 0:
        g = gf.gf_create(DIMS, gf.GF_LANDAU)
        th = base.clone()
        gf.gf_generate(g, th, 6.1, args.therm, 4, 21, 0)
        fields["beta6.1"] = th
        gf.gf_destroy(g)
    out = {"workload": f"32^4 Landau, theta<{target:g}, FP64 storage, double-float arithmetic, check every 25",
           "therm_sweeps": args.therm, "fields": {}}
    for name, U0 in fields.items():
        rows = []
        runs = [("or", float(w)) for w in args.omegas] + [("sr", float(q)) for q in args.probs]
        for kind, val in runs:
            c = gf.gf_create(DIMS, gf.GF_LANDAU)
            gf.gf_set_stream(c, torch.cuda.current_stream())
            gf.gf_set_option(c, "check_every", CHECK_EVERY)
            gf.gf_set_option(c, "fp64_arith", 1)
            if kind == "sr":
                gf.gf_set_option(c, "stochastic_p", val)
                gf.gf_set_option(c, "sr_seed", 5)
            U = U0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            conv, it, F, thv = gf.gf_overrelax(c, U, val if kind == "or" else 1.0, target, max_iter)
            torch.cuda.synchronize()
            rows.append({"method": kind, "omega" if kind == "or" else "p": val, "sweeps": it, "converged": conv,
                         "s": time.perf_counter() - t0, "F": F, "theta": thv})
            gf.gf_destroy(c)
            log(name, rows[-1])
        pc = gf.gf_create(DIMS, gf.GF_LANDAU)
        out["fields"][name] = {"plaquette": gf.gf_plaquette(pc, U0), "runs": rows}
        gf.gf_destroy(pc)
    print(json.dumps(out), flush=True)


def single_solve(args):
    """One gauge fixing of the seeded synthetic field on --dims (default 32^4)
    with the mixed policy and the given --fp64-arith / --fp32-restarts, twice
    (the second timed); for profiling the kernels of one policy.  Prints one
    JSON object."""
    from paper_1209_4008_gb300 import gf, synth
    dims = tuple(args.dims) if args.dims else DIMS
    U0 = synth.make_field(dims, PLAQ, *SEEDS, device="cuda")
    c = gf.gf_create(dims, gf.GF_LANDAU)
    gf.gf_set_stream(c, torch.cuda.current_stream())
    for k, v in (("precision", gf.GF_MIXED), ("check_every", CHECK_EVERY), ("fp64_arith", args.fp64_arith),
                 ("fp32_restarts", args.fp32_restarts), ("kernel_timing", 1),
                 ("theta_switch", args.restart_switch if args.fp32_restarts else THETA_SWITCH)):
        gf.gf_set_option(c, k, v)
    for rep in range(2):
        U = U0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, it, F, th = gf.gf_overrelax(c, U, OMEGA, THETA_TARGET, MAX_ITER)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    st = {k: gf.gf_get_stat(c, k) for k in ("sweeps_fp32", "sweeps_fp64", "ms_sweep_kernels_fp32",
                                              "sweep_launches_fp32", "ms_sweep_kernels_fp64", "sweep_launches_fp64")}
    print(json.dumps({"dims": dims, "fp64_arith": args.fp64_arith, "fp32_restarts": args.fp32_restarts, "s": t,
                      "sweeps": it, "F": F, "theta": th, "converged": conv,
                      "ms_per_fp64_class_launch": st["ms_sweep_kernels_fp64"] / max(1, st["sweep_launches_fp64"]),
                      "ms_per_fp32_launch": st["ms_sweep_kernels_fp32"] / max(1, st["sweep_launches_fp32"]),
                      **st}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gf", choices=["gf", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--kernel", choices=sorted(FORMATS), help="time one storage format's sweep only")
    ap.add_argument("--tps", type=int, default=1)
    ap.add_argument("--block", type=int, default=64)
    ap.add_argument("--sa-temp", type=float, help="--kernel: time heatbath half-sweeps at this temperature")
    ap.add_argument("--theta-start", type=float, default=0.0,
                    help="--kernel: first overrelax the field (FP64, per-subgroup form) to this theta")
    ap.add_argument("--acc-regs", type=int, default=0, choices=[0, 255, 168, 128],
                    help="--kernel --tps 0: register budget of the accumulate form (FP64 storage)")
    ap.add_argument("--or-seeds", type=int, default=2,
                    help="--coulomb: seeds that are also fixed by overrelaxation alone, for comparison")
    ap.add_argument("--dims", type=int, nargs=4, help="lattice of --kernel and --impl reference (default 32^4)")
    ap.add_argument("--batched", action="store_true", help="the 64-lattice batched workload")
    ap.add_argument("--learned", action="store_true", help="train and evaluate the learned warm start")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-decay", type=float, default=0.7, help="learning-rate factor per epoch")
    ap.add_argument("--learned-repeat", type=int, default=15,
                    help="further applications of the network in the FP64 phase")
    ap.add_argument("--learned-factor", type=float, default=0.316,
                    help="theta falls by this factor between applications")
    ap.add_argument("--eval-fields", type=int, default=4)
    ap.add_argument("--eval-arith", type=int, default=0, choices=[0, 1],
                    help="--learned evaluation: fp64_arith of both legs (1: the exact double-float finish)")
    ap.add_argument("--fp32-restarts", type=int, default=2,
                    help="add a line for the mixed policy with this many FP32 restarts (0: none)")
    ap.add_argument("--restart-switch", type=float, default=1e-30,
                    help="theta_switch of the FP32-restart line (default 1e-30: the first FP32 phase "
                         "runs to its rounding floor)")
    ap.add_argument("--save", nargs="?", const=WEIGHTS, default=None, metavar="PATH",
                    help=f"store the trained parameters (.npy; default path {os.path.relpath(WEIGHTS, ROOT)})")
    ap.add_argument("--weights", metavar="PATH",
                    help="--learned: skip the pairs and training, evaluate these stored parameters")
    ap.add_argument("--coulomb", action="store_true", help="the 48^3x96 Coulomb workload with annealing")
    ap.add_argument("--net", action="store_true", help="time the warm-start network's kernels")
    ap.add_argument("--conv-halo", type=int, default=1, choices=(0, 1, 2),
                    help="--net: convolution kernel, 1 x-line (default), 2 halo-tile, 0 per-tap gather")
    ap.add_argument("--mag", action="store_true", help="the maximally Abelian gauge on the 32^4 field")
    ap.add_argument("--thermal", action="store_true", help="gauge fixing of a field thermalised at beta 6.1")
    ap.add_argument("--solve", action="store_true",
                    help="one mixed-policy solve on --dims with --fp64-arith / --fp32-restarts (profiling)")
    ap.add_argument("--fp64-arith", type=int, default=0, choices=[0, 1])
    ap.add_argument("--sr", action="store_true",
                    help="sweeps to theta<1e-12 against omega (overrelaxation) and p (stochastic relaxation)")
    ap.add_argument("--omegas", type=float, nargs="+", default=[1.5, 1.6, 1.7, 1.8, 1.9])
    ap.add_argument("--probs", type=float, nargs="+", default=[0.5, 0.7, 0.8, 0.9, 0.95])
    ap.add_argument("--sr-max-iter", type=int, default=40000)
    ap.add_argument("--therm", type=int, default=100, help="--thermal: compound sweeps of generation")
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--fast", action="store_true",
                    help="--coulomb: double-float sweeps with the exact FP64 result and the FP32 heatbath draw")
    ap.add_argument("--sa-sweeps", type=int, default=3000)
    args = ap.parse_args()
    if args.learned:
        torch.cuda.set_device(0)
        learned(args)
        return
    if args.batched:
        torch.cuda.set_device(0)
        batched(args)
        return
    if args.coulomb:
        torch.cuda.set_device(0)
        coulomb(args)
        return
    if args.net:
        torch.cuda.set_device(0)
        net_kernels(args)
        return
    if args.mag:
        torch.cuda.set_device(0)
        mag(args)
        return
    if args.thermal:
        torch.cuda.set_device(0)
        thermal(args)
        return
    if args.sr:
        torch.cuda.set_device(0)
        sr_study(args)
        return
    if args.solve:
        torch.cuda.set_device(0)
        single_solve(args)
        return
    if args.kernel:
        torch.cuda.set_device(0)
        kernel_only(args)
        return
    rank, world, local = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            reference_arm(args, rank, world)
        else:
            gpu_arm(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
