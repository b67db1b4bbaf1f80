"""Benchmark of the vortex-field smoothing path on GB300.

One step = the whole path on one synthetic 32^3 x 64 field: load the Z(3)
labels, centrifuge preconditioning (omega = 0.02), 300 annealed over-improved
stout sweeps (eps = -0.25, rho = 0.06) with the vortex-preservation test and
re-unitarisation every 10 sweeps, then the action and the vortex check,
in FP32 with 18-real links.  The input labels come from the library's cooled
hot start (Haar SU(3), 20 MaxReTr cooling sweeps, Z(3) projection; seed 3 +
rank).  The metric is link updates per second (4 V n_sweeps per step).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "link-updates/s at 32^3x64 FP32 vs FP64 at stated error; served p50/p99 latency"
DIMS = (32, 32, 32, 64)
N_SWEEPS = 300
RHO, EPS, U0, OMEGA = 0.06, -0.25, 1.0, 0.02
CENTRIFUGE_SEED = 1234
N_COOL = 20
REUNIT = 10
# algorithmic bytes per link update of one colour-class launch (FP32, 18 reals):
# every link of the field is read once (4 V links for V/4 updates = 16 reads
# per update), the updated link written once, its reference label read once.
BYTES_PER_UPDATE = {(1, 18): 17 * 72 + 1, (1, 12): 17 * 48 + 1, (0, 18): 17 * 144 + 1}
FLOPS_PER_UPDATE_OVERIMPROVED = 65 * 216 + 600
# DRAM bytes (read + write) of one class-update launch of this kernel version,
# from `ncu --set full` on the same command (profiles/k_subsweep_f32_*.md)
NCU_TRAFFIC_PER_LAUNCH = 625.287936e6 + 40.275968e6
# FP32 FMA peak of the GPU: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _dist_init():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        return dist, world, rank, local
    return None, 1, 0, local


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, x, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    dist, world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    from paper_2203_09764_gb300 import vs

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)          # every library call and event runs here
    torch.cuda.set_stream(stream)
    ctx = vs.vs_create(local)
    V = int(np.prod(DIMS))
    n_links = 4 * V
    seed = 3 + rank

    # ---- input: cooled hot start, labels resident on the device ------------
    gen = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18, stream)
    vs.vs_load_cooled(gen, seed, N_COOL)
    labels_dev = torch.empty((4, V), dtype=torch.int8, device=dev)
    vs.vs_read_labels(gen, labels_dev)
    labels_host = torch.empty((4, V), dtype=torch.int8, pin_memory=True)
    labels_host.copy_(labels_dev.cpu())
    vs.vs_field_destroy(gen)

    f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18, stream)

    def step(from_host=False, profile=False, fld=None):
        fld = f if fld is None else fld
        if from_host:
            vs.vs_load_field(fld, labels=labels_host)
        else:
            vs.vs_load_field(fld, labels=labels_dev)
        vs.vs_centrifuge(fld, OMEGA, CENTRIFUGE_SEED)
        vs.vs_set_profiling(fld, profile)
        vs.vs_smooth(fld, args.sweeps, RHO, EPS, U0, reunit_every=REUNIT, vortex_preserve=True)
        S = vs.vs_action(fld)
        chk = vs.vs_vortex_check(fld)
        return S, chk

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # ---- device-resident timed region --------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(dist)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    chain_ms, chain_launches = 0.0, 0
    k0 = vs.vs_kernel_launches()
    for _ in range(args.steps):
        results.append(step(profile=True))
        ms, nl = vs.vs_get_profile(f)
        chain_ms += ms
        chain_launches += nl
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = vs.vs_kernel_launches() - k0
    _barrier(dist)
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    t_ms = _max_over_ranks(dist, t_ms, dev)
    ms_per_step = t_ms / args.steps
    updates_per_step = n_links * args.sweeps
    value = world * updates_per_step * args.steps / (t_ms / 1e3)

    # ---- end to end through the C ABI with host buffers --------------------
    e2e = None
    if not args.no_e2e:
        # Two fields on two streams: the read-back of one step's field (a
        # blocking C call, made from a worker thread) runs while the next step
        # computes on the other field, as a pipelined user would run it.
        from concurrent.futures import ThreadPoolExecutor
        stream2 = torch.cuda.Stream(device=dev)
        f2 = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18, stream2)
        fields = [f, f2]
        outs = [torch.empty((4, V, 3, 3), dtype=torch.complex128, pin_memory=True) for _ in range(2)]
        e2e_steps = max(1, min(args.steps, 3))
        # one untimed pass per field: the first host read-back sizes its staging buffer
        for fld, out in zip(fields, outs):
            step(from_host=True, fld=fld)
            vs.vs_read_field(fld, out)
        _barrier(dist)
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=1) as pool:
            pending = None
            for k in range(e2e_steps):
                step(from_host=True, fld=fields[k % 2])
                if pending is not None:
                    pending.result()
                pending = pool.submit(vs.vs_read_field, fields[k % 2], outs[k % 2])
            pending.result()
        t_e2e = time.perf_counter() - t0
        t_e2e = _max_over_ranks(dist, t_e2e, dev)
        e2e = {"value": world * updates_per_step * e2e_steps / t_e2e, "unit": "link-updates/s",
               "h2d_bytes_per_step": int(labels_host.numel()),
               "d2h_bytes_per_step": int(outs[0].numel() * 16 + 8 + 40), "steps": e2e_steps,
               "pipelining": "two fields on two streams; each step's 1.2 GB FP64 read-back overlaps the "
                             "next step on the other field (the last read-back is not overlapped)"}
        vs.vs_field_destroy(f2)
    vs.vs_field_destroy(f)

    line = {"metric": METRIC, "value": value, "unit": "link-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "32^3x64 cooled hot start (Haar SU(3) seed 3+rank, 20 MaxReTr "
                                   "cooling sweeps, Z(3) projection); centrifuge w=0.02; "
                                   "over-improved stout eps=-0.25 rho=0.06 u0=1, %d annealed sweeps "
                                   "with vortex preservation, re-unitarisation every 10; "
                                   "FP32 18-real links" % args.sweeps,
                       "lattice": list(DIMS), "sweeps": args.sweeps, "precision": "fp32",
                       "storage": "18-real", "parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2: 604 MB field vs 129 MB L2"},
            "clocks": clk, "e2e": e2e,
            "gpu_launches": launches}

    peaks, src = _measured_peaks()
    S_last, chk_last = results[-1]
    line["result"] = {"action": S_last, "n_label_diff": chk_last["n_label_diff"],
                      "n_charge_diff": chk_last["n_charge_diff"],
                      "n_near_boundary": chk_last["n_near_boundary"]}

    # ---- roofline of the dominant kernel (colour-class update) -------------
    per_launch_ms = chain_ms / max(chain_launches, 1)
    units = V // 4
    bpu = BYTES_PER_UPDATE[(1, 18)]
    achieved = units * bpu / (per_launch_ms / 1e3) / 1e9
    tflops = units * FLOPS_PER_UPDATE_OVERIMPROVED / (per_launch_ms / 1e3) / 1e12
    line["roofline"] = {"kernel": "k_subsweep_fused<18,mu> (FP32 over-improved class update)", "bound": "hbm",
                        "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC_PER_LAUNCH,
                        "peak_source": src, "per_launch_ms": per_launch_ms,
                        "bytes_per_update": bpu, "updates_per_launch": units,
                        "achieved_tflops": tflops, "fp32_peak_tflops": FP32_PEAK_TFLOPS,
                        "fp32_frac": tflops / FP32_PEAK_TFLOPS}

    # ---- the same step with 12-real links (rows 1-2 stored, row 3 rebuilt) ----
    if not args.no_fp64:
        try:
            line["fp32_12real"] = storage12(vs, ctx, stream, labels_dev, args, world, dev, peaks)
        except Exception as e:
            line["fp32_12real"] = {"error": repr(e)}

    # ---- FP64 plain path, bounded number of sweeps --------------------------
    if not args.no_fp64:
        try:
            line["fp64_plain"] = fp64_plain(vs, ctx, stream, labels_dev, args, value, world, dev)
        except Exception as e:  # report it, keep the main line
            line["fp64_plain"] = {"error": repr(e)}

    # ---- per-sweep vortex diagnostics of the workload, VP on and off -------
    if not args.no_other:
        try:
            line["vortex_diagnostics"] = vortex_diagnostics(vs, ctx, stream, labels_dev, args)
        except Exception as e:
            line["vortex_diagnostics"] = {"error": repr(e)}

    # ---- the paper's other smoothing paths on the same field ---------------
    if not args.no_other:
        try:
            line["other_paths"] = other_paths(vs, ctx, stream, labels_dev, args, world, dev)
        except Exception as e:
            line["other_paths"] = {"error": repr(e)}

    # ---- serving: continuous batching of a Poisson job mix -----------------
    if not args.no_serve and rank == 0:
        try:
            line["serving"] = run_serving(vs, local, args)
        except Exception as e:
            line["serving"] = {"error": repr(e)}

    if rank == 0 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args, vs, ctx, stream)
        except Exception as e:
            line["cpu_baseline"] = {"error": repr(e)}
        else:
            try:
                line["cpu_baseline"]["single_core"] = oracle_single_core()
            except Exception as e:
                line["cpu_baseline"]["single_core"] = {"error": repr(e)}

    vs.vs_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def storage12(vs, ctx, stream, labels_dev, args, world, dev, peaks):
    """One step of the benchmark workload with 12-real link storage."""
    import torch
    V = int(np.prod(DIMS))
    f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK12, stream)
    vs.vs_load_field(f, labels=labels_dev)
    vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
    vs.vs_smooth(f, 3, RHO, EPS, U0, reunit_every=REUNIT)
    vs.vs_load_field(f, labels=labels_dev)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    vs.vs_load_field(f, labels=labels_dev)
    vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
    vs.vs_set_profiling(f, True)
    vs.vs_smooth(f, args.sweeps, RHO, EPS, U0, reunit_every=REUNIT, vortex_preserve=True)
    vs.vs_action(f)
    chk = vs.vs_vortex_check(f)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    cms, nl = vs.vs_get_profile(f)
    vs.vs_field_destroy(f)
    per = cms / nl
    bpu = BYTES_PER_UPDATE[(1, 12)]
    ach = V / 4 * bpu / (per / 1e3) / 1e9
    return {"value": world * 4 * V * args.sweeps / (ms / 1e3), "unit": "link-updates/s",
            "ms_per_step": ms, "per_launch_ms": per, "bytes_per_update": bpu,
            "achieved_gbs": ach, "hbm_frac": ach / peaks["hbm_gbs"],
            "n_label_diff": chk["n_label_diff"]}


def fp64_plain(vs, ctx, stream, labels_dev, args, value, world, dev):
    """The FP32 ratio over the GPU FP64 plain path on one scope: the same
    sweeps (vs_smooth of --fp64-sweeps annealed over-improved VP sweeps, with
    the FP32 re-unitarisation every 10, from the same centrifuged field after
    one untimed sweep), timed with CUDA events in both precisions."""
    import torch
    n_links = 4 * int(np.prod(DIMS))
    n = args.fp64_sweeps
    ms = {}
    for name, prec in (("fp64", vs.VS_FP64), ("fp32", vs.VS_FP32)):
        f = vs.vs_field_create(ctx, DIMS, prec, vs.VS_LINK18, stream)
        vs.vs_load_field(f, labels=labels_dev)
        vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
        vs.vs_smooth(f, 1, RHO, EPS, U0, reunit_every=REUNIT, vortex_preserve=True)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vs.vs_smooth(f, n, RHO, EPS, U0, reunit_every=REUNIT, vortex_preserve=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms[name] = e0.elapsed_time(e1)
        vs.vs_field_destroy(f)
    v64 = world * n_links * n / (ms["fp64"] / 1e3)
    v32 = world * n_links * n / (ms["fp32"] / 1e3)
    return {"value": v64, "unit": "link-updates/s", "sweeps": n, "ms": ms["fp64"],
            "fp32_same_scope": {"value": v32, "ms": ms["fp32"]}, "fp32_over_fp64": v32 / v64,
            "scope": "vs_smooth sweeps alone in both precisions (class updates, and FP32 "
                     "re-unitarisation every 10 sweeps), same field and sweep count"}


def vortex_diagnostics(vs, ctx, stream, labels_dev, args):
    """The workload's sweeps with and without vortex preservation (Sec. VI),
    per-sweep statistics from the kernels: candidates whose Z(3) label differs
    from the original (without VP: the label differences after the sweep, the
    n_diff of the paper's tables), candidates inside the rounding band of a sector
    edge (with VP the FP32 candidates inside the FP32 band are decided again in
    FP64, and those left within the band of the FP32 link storage are counted),
    the smallest candidate margin, and the action."""
    out = {}
    marks = [k for k in (1, 2, 5, 10, 20, 50, 100, 200, 300) if k <= args.sweeps]
    for vp in (True, False):
        f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18, stream)
        vs.vs_load_field(f, labels=labels_dev)
        vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
        st = vs.vs_smooth(f, args.sweeps, RHO, EPS, U0, reunit_every=REUNIT, vortex_preserve=vp,
                          action_every=1, stats=True)
        chk = vs.vs_vortex_check(f)
        vs.vs_field_destroy(f)
        out["vp_on" if vp else "vp_off"] = {
            "n_label_diff_at_sweep": {str(k): st[k - 1]["n_label_diff"] for k in marks},
            "action_at_sweep": {str(k): st[k - 1]["action"] for k in marks},
            "min_margin_at_sweep": {str(k): st[k - 1]["min_margin"] for k in marks},
            "n_undecidable_total": int(sum(s["n_undecidable"] for s in st)),
            "n_fp64_redecided_total": int(sum(s["n_fp64_redecided"] for s in st)),
            "n_fp64_exp_total": int(sum(s["n_fp64_exp"] for s in st)),
            "after_last_sweep": {"n_label_diff": chk["n_label_diff"], "n_charge_diff": chk["n_charge_diff"]}}
    out["what"] = ("%d sweeps of the workload (FP32 18-real) with per-sweep statistics; with VP the "
                   "candidate label differences are the rejections" % args.sweeps)
    return out


def other_paths(vs, ctx, stream, labels_dev, args, world, dev):
    """The paper's other smoothers on the benchmark field (FP32 18-real,
    centrifuged): time per sweep (RK3: per step of three stages) with CUDA
    events on the field's stream, after one untimed sweep."""
    import torch
    V = int(np.prod(DIMS))
    n = args.other_sweeps
    paths = {
        "euler_wilson_flow": ("annealed stout, eps=1, rho=0.06 (Euler Wilson flow), VP",
                              lambda f, k: vs.vs_smooth(f, k, RHO, 1.0, U0, reunit_every=REUNIT), 1),
        "aus_maxretr": ("AUS, MaxReTr 3 hits, alpha=0.02, eps=-0.25, VP",
                        lambda f, k: vs.vs_smooth_aus(f, k, 0.02, EPS, U0), 1),
        "aus_ucp": ("AUS with unit circle projection, alpha=0.02, eps=-0.25, VP",
                    lambda f, k: vs.vs_smooth_ape(f, k, 0.02, EPS, U0), 1),
        "ape_ucp": ("APE smearing (simultaneous) with unit circle projection, alpha=0.5, eps=-0.25",
                    lambda f, k: vs.vs_smooth_ape(f, k, 0.5, EPS, U0, schedule=vs.VS_SIMULTANEOUS,
                                                  vortex_preserve=False), 1),
        "rk3_wilson_flow": ("Wilson flow, third-order Runge-Kutta, eps=1, step 0.02 (3 stages per step)",
                            lambda f, k: vs.vs_flow_rk3(f, k, 0.02, 1.0, U0), 3),
    }
    out = {}
    for name, (what, run, passes) in paths.items():
        f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18, stream)
        vs.vs_load_field(f, labels=labels_dev)
        vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
        run(f, 1)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(f, n)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        vs.vs_field_destroy(f)
        out[name] = {"what": what, "sweeps": n, "ms_per_sweep": ms / n,
                     "link_updates_per_s": world * 4 * V * passes * n / (ms / 1e3),
                     "sweeps_per_s": world * n / (ms / 1e3)}
    return out


def _serve_run(vs, device, jobs, budget, slots, burst):
    """Submit the job mix at its arrival times (all at once with burst) and
    collect latencies (submit -> result) and the served link updates."""
    ctx = vs.vs_create(device, hbm_budget_bytes=budget, max_slots=slots)
    handles = []
    t_start = time.perf_counter()
    for j in jobs:
        if not burst:
            while time.perf_counter() - t_start < j["arrival_s"]:
                time.sleep(0.0002)
        job = vs.make_job(j["dims"], j["rho"], j["n_sweeps"], epsilon=EPS, seed=j["seed"],
                          n_cool=N_COOL, omega=OMEGA, centrifuge_seed=CENTRIFUGE_SEED)
        handles.append((vs.vs_submit(ctx, job), job, j))
    lat, updates, cool = [], 0, 0
    for t, job, j in handles:
        r = vs.vs_poll(ctx, t, -1)
        assert r["status"] == vs.VS_OK, r
        lat.append(r["t_done_ms"] - r["t_submit_ms"])
        updates += 4 * int(np.prod(j["dims"])) * j["n_sweeps"]
        cool += 4 * int(np.prod(j["dims"])) * N_COOL
    wall = time.perf_counter() - t_start
    st = vs.vs_serve_stats_get(ctx)
    vs.vs_destroy(ctx)
    lat = np.array(lat)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "jobs_per_s": len(jobs) / wall, "link_updates_per_s": updates / wall,
            "link_updates_incl_cooling_per_s": (updates + cool) / wall, "wall_s": wall,
            "peak_bytes_in_use": st["peak_bytes_in_use"]}


def run_serving(vs, device, args):
    """The serving mix (64 jobs, seeds 100-163) three times: all jobs at once,
    which measures the loop's capacity for this mix (jobs/s at saturation),
    then Poisson arrivals (seed 99) at 0.8x and at 1.5x that capacity."""
    import synth
    budget, slots = 512 << 20, 8
    mix = synth.serving_jobs(n_jobs=args.serve_jobs, seed=99, rate_hz=1.0)
    cap = _serve_run(vs, device, mix, budget, slots, burst=True)
    out = {"jobs": len(mix), "hbm_budget_bytes": budget, "max_slots": slots,
           "capacity": dict(cap, what="all jobs submitted at once; jobs/s = jobs / makespan")}
    for tag, f in (("at_0.8x_capacity", 0.8), ("at_1.5x_capacity", 1.5)):
        rate = f * cap["jobs_per_s"]
        jobs = synth.serving_jobs(n_jobs=args.serve_jobs, seed=99, rate_hz=rate)
        out[tag] = dict(_serve_run(vs, device, jobs, budget, slots, burst=False), arrival_rate_hz=rate)
    out["p50_ms"] = out["at_0.8x_capacity"]["p50_ms"]
    out["p99_ms"] = out["at_0.8x_capacity"]["p99_ms"]
    out["mix"] = ("shapes {8^4, 12^3x24, 16^3x32, 24^3x48}, rho U[0.04,0.1], 50-300 sweeps, eps=-0.25, "
                  "w=0.02, VP, FP32 18-real, job seeds 100-163")
    out["latency"] = ("submit to result: queueing, admission, field allocation, the job's input (GPU hot "
                      "start and %d cooling sweeps), centrifuge, the smoothing sweeps, action and vortex "
                      "check; link_updates_per_s counts the smoothing sweeps only" % N_COOL)
    return out


def oracle_input():
    """The benchmark's input built by the oracle (same recipe and seed as the
    GPU arm's vs_load_cooled: Haar SU(3) seed 3, 20 MaxReTr cooling sweeps,
    Z(3) projection), centrifuged; cached on disk after the first build."""
    import oracle as O
    t0 = time.perf_counter()
    lab = O.cooled_labels(DIMS, 3, N_COOL)
    Uc = O.centrifuge(DIMS, lab, OMEGA, CENTRIFUGE_SEED)
    return lab, Uc, time.perf_counter() - t0


def cpu_baseline(args, vs=None, ctx=None, stream=None, sweeps=None, inp=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    `sweeps` annealed sweeps (default --cpu-sweeps) of the 32^3 x 64 cooled
    hot start (8.4M link updates each) after the centrifuge.  Returns
    link-updates/s on the host cores."""
    n_sw = args.cpu_sweeps if sweeps is None else sweeps
    import oracle as O
    V = int(np.prod(DIMS))
    lab, Uc, t_input = inp if inp is not None else oracle_input()
    nt = O.max_threads()
    t0 = time.perf_counter()
    U1, rej = O.smooth(DIMS, Uc, lab, n_sw, RHO, eps=EPS, vp=True, nthreads=nt)
    dt = time.perf_counter() - t0
    out = {"value": 4 * V * n_sw / dt, "unit": "link-updates/s", "cores": nt,
           "kind": "oracle",
           "sample": "%d annealed over-improved sweep(s) of the 32^3x64 cooled hot start (Haar SU(3) "
                     "seed 3, 20 oracle MaxReTr cooling sweeps, Z(3) projection) after the "
                     "centrifuge, FP64, OpenMP over the sites of a colour class" % n_sw,
           "seconds": dt, "input_build_s": t_input}
    if vs is not None:
        # error of the FP32 GPU path against the oracle on the same sample
        f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18, stream)
        vs.vs_load_field(f, labels=lab)
        vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
        st = vs.vs_smooth(f, n_sw, RHO, EPS, U0, vortex_preserve=True, stats=True,
                          reunit_every=REUNIT)
        Ug = vs.vs_read_field(f)
        vs.vs_field_destroy(f)
        out["fp32_max_link_err_vs_oracle"] = float(np.abs(Ug - U1).max())
        out["reject_counts_equal"] = [s["n_reject"] for s in st] == list(rej)
    return out


def oracle_single_core():
    """The FP64 oracle, as it stands, on one host core: one annealed
    over-improved sweep of a 16^3 x 32 field of the same recipe (524,288
    link updates; the cost per link does not depend on the lattice size)."""
    import oracle as O
    import synth
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    lab = synth.iid_labels(dims, 3, p0=1 / 3, p_plus=1 / 3)
    Uc = O.centrifuge(dims, lab, OMEGA, CENTRIFUGE_SEED)
    t0 = time.perf_counter()
    O.smooth(dims, Uc, lab, 1, RHO, eps=EPS, vp=True, nthreads=1)
    dt = time.perf_counter() - t0
    return {"value": 4 * V / dt, "unit": "link-updates/s", "cores": 1,
            "sample": "1 annealed over-improved sweep of a 16^3x32 field from iid uniform Z(3) labels "
                      "(seed 3) after the centrifuge, FP64, one thread", "seconds": dt}


def run_reference(args):
    """The FP64 oracle on the benchmark's workload: each step is a bounded
    sample of it, --ref-sweeps annealed sweeps of the centrifuged cooled
    32^3 x 64 field; ms_per_step is the measured time of those sweeps."""
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if world > 1 and rank != 0:
        return
    t0 = time.perf_counter()
    inp = oracle_input()
    for _ in range(min(args.warmup, 1)):
        cpu_baseline(args, sweeps=args.ref_sweeps, inp=inp)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(args, sweeps=args.ref_sweeps, inp=inp))
    v = statistics.median([x["value"] for x in vals])
    step_ms = statistics.median([x["seconds"] for x in vals]) * 1e3
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "link-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "32^3x64 cooled hot start (Haar SU(3) seed 3, 20 MaxReTr cooling "
                                   "sweeps, Z(3) projection, built by the oracle); centrifuge w=0.02; "
                                   "over-improved stout eps=-0.25 rho=0.06 u0=1, annealed, with vortex "
                                   "preservation; FP64 CPU oracle, each step %d sweep(s) of the "
                                   "workload's %d" % (args.ref_sweeps, args.sweeps),
                       "lattice": list(DIMS), "sweeps": args.ref_sweeps},
            "extrapolated_ms_per_workload_step": {
                "value": 4 * int(np.prod(DIMS)) * args.sweeps / v * 1e3, "sweeps": args.sweeps,
                "note": "not timed: the measured rate applied to the whole %d-sweep step" % args.sweeps},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "link-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "input_build_s": inp[2],
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def _oracle_rate(dims):
    """The FP64 oracle on the host cores: one annealed over-improved VP sweep
    of `dims` from iid uniform Z(3) labels after the centrifuge (its cost per
    link does not depend on the label values)."""
    import oracle as O
    import synth
    V = int(np.prod(dims))
    lab = synth.iid_labels(dims, 5, p0=1 / 3, p_plus=1 / 3)
    Uc = O.centrifuge(dims, lab, OMEGA, CENTRIFUGE_SEED)
    t0 = time.perf_counter()
    O.smooth(dims, Uc, lab, 1, RHO, eps=EPS, vp=True, nthreads=O.max_threads())
    dt = time.perf_counter() - t0
    return {"value": 4 * V / dt, "unit": "link-updates/s", "cores": O.max_threads(), "seconds": dt,
            "sample": "1 annealed over-improved VP sweep from iid uniform labels after the centrifuge"}


def run_scaling(args):
    """Lattice-size sweep (16^3x32 .. 48^3x96): link-updates/s and the roofline
    fraction of the class-update kernel per size, FP32 18- and 12-real, beside
    the FP64 oracle on the host cores (one sweep per size, --no-cpu-baseline
    skips it); one JSON line per size and storage."""
    import torch
    from paper_2203_09764_gb300 import vs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = vs.vs_create(0)
    peaks, src = _measured_peaks()
    for dims in [(16, 16, 16, 32), (24, 24, 24, 48), (32, 32, 32, 64), (40, 40, 40, 80), (48, 48, 48, 96)]:
        orc = None if args.no_cpu_baseline else _oracle_rate(dims)
        for storage, nc in ((vs.VS_LINK18, 18), (vs.VS_LINK12, 12)):
            V = int(np.prod(dims))
            f = vs.vs_field_create(ctx, dims, vs.VS_FP32, storage, stream)
            vs.vs_load_cooled(f, 5, N_COOL)
            vs.vs_centrifuge(f, OMEGA, CENTRIFUGE_SEED)
            vs.vs_smooth(f, 3, RHO, EPS, U0, reunit_every=REUNIT)
            vs.vs_synchronize(f)
            vs.vs_set_profiling(f, True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vs.vs_smooth(f, args.sweeps, RHO, EPS, U0, reunit_every=REUNIT)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            cms, nl = vs.vs_get_profile(f)
            vs.vs_field_destroy(f)
            per = cms / nl
            bpu = BYTES_PER_UPDATE[(1, nc)]
            ach = V / 4 * bpu / (per / 1e3) / 1e9
            rate = 4 * V * args.sweeps / (ms / 1e3)
            print(json.dumps({"lattice": list(dims), "storage": "%d-real" % nc, "sweeps": args.sweeps,
                              "link_updates_per_s": rate,
                              "class_launch_ms": per, "achieved_gbs": ach,
                              "hbm_frac": ach / peaks["hbm_gbs"], "peak_source": src,
                              "field_mb": 4 * nc * 4 * V / 1e6, "oracle_host": orc,
                              "gpu_over_oracle": rate / orc["value"] if orc else None}), flush=True)
    vs.vs_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps", type=int, default=N_SWEEPS)
    ap.add_argument("--fp64-sweeps", type=int, default=10)
    ap.add_argument("--cpu-sweeps", type=int, default=2,
                    help="oracle sweeps in the cpu_baseline leg (about 11 s on 16 Arm cores)")
    ap.add_argument("--ref-sweeps", type=int, default=1,
                    help="oracle sweeps per step of --impl reference")
    ap.add_argument("--serve-jobs", type=int, default=64)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other", action="store_true",
                    help="skip timing the other smoothing paths (AUS, UCP, Runge-Kutta flow)")
    ap.add_argument("--other-sweeps", type=int, default=10)
    ap.add_argument("--scaling", action="store_true",
                    help="lattice-size sweep 16^3x32 .. 48^3x96 instead of the benchmark step")
    ap.add_argument("--lattice", default=None,
                    help="Lx,Ly,Lz,Lt of the workload (default 32,32,32,64), e.g. a small lattice "
                         "for a quick check of the output")
    args = ap.parse_args()
    if args.lattice:
        global DIMS
        DIMS = tuple(int(v) for v in args.lattice.split(","))
        assert len(DIMS) == 4 and all(d > 0 and d % 4 == 0 for d in DIMS), "extents: positive multiples of 4"
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.scaling:
        if args.sweeps == N_SWEEPS:
            args.sweeps = 20
        run_scaling(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
