"""Throughput of the per-timestep PIC cycle on GB300.

Workload: bulk fused silica, 128 x 128 x 512 cells at lambda/40, slab z
128-480 with 8 neutral macroparticles per cell, 5 fs / 2 J cm^-2 pulse, FP32
fields, push and deposit (the 2000-step bulk-silica configuration).  A step
is one full PIC step (gather, Boris, deposit, Yee + polarisation, window,
Keldysh, ionisation, pool maintenance).  The run first advances `--prerun`
untimed steps (default 1700: the pulse has ionised the slab, every material
cell is drawn each step and the pool holds its late-job particle count),
then `--warmup` steps, then times `--steps` steps with CUDA events on the
simulation's stream.  The state (13.9 GB) is far larger than L2, so no
flush is needed between steps.

At one GPU the line also carries, measured the same way:
  mirror  the 20-pair quarter-wave mirror, 256 x 256 x 1024, 3000 steps
          (window after `--mirror-prerun` steps, whole job as e2e, its own
          roofline and oracle baseline);
  scan    the 64-instance fluence scan (batched graph vs one at a time) and
          its time-to-result p50 / p99 (also at the top level).

value   = charged-particle pushes per second (all ranks)
e2e     = the same metric for one whole job through the public API: from the
          host configuration (pic_create copies the layer tables; the
          neutrals are generated on the device from the seed) through all
          2000 steps to FP64 diagnostics and a 64-bin electron spectrum on
          the host; the host<->device bytes are the library's own counters
roofline= the dominant kernel's algorithmic bytes / its CUDA-event time
`--impl reference` times the FP64 CPU oracle on a 4 x 4 column of the same
workload (same z structure, prerun to the same step).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s & cell-updates/s (%HBM roofline); fluence-scan p50/p99 latency"
UNIT = "particle-steps/s"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def kernel_source_hash():
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2502_13695_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, units):
    """DRAM bytes per launch from the committed ncu summary, scaled to the
    units (particles or cells) of this launch; None if the kernel source has
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return e["dram_bytes_per_unit"] * units
    except Exception:
        return None


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        time.sleep(0.2)
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in self.rows for q in range(4)
                          if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": reasons}


def dist_setup(n_gpus, backend="nccl"):
    """(rank, local rank, world size, torch.distributed or None) from the
    torchrun environment; one process per GPU under NCCL (gloo: host only)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if backend == "nccl":
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)
    return rank, local, ws, dist


def allreduce(dist, x, op):
    """All-reduce one float over the ranks (on the GPU under NCCL, on the
    host under gloo); x itself with no process group."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=op)
    return float(t.item())


def replica_seed(seed, rank):
    """Seed of rank's independent replica of the workload."""
    return seed + 7919 * rank


def aggregate(dist, ms, psteps, events):
    """Whole-job totals over the ranks: the slowest rank's time (ms) and the
    particle steps and ionisation events summed; value = particle-steps/s of
    all ranks together."""
    ms_max = allreduce(dist, ms, _op(dist, "max"))
    psteps_all = allreduce(dist, psteps, _op(dist, "sum"))
    events_all = allreduce(dist, events, _op(dist, "sum"))
    return {"ms_max": ms_max, "psteps_all": psteps_all, "events_all": events_all,
            "value": psteps_all / (ms_max / 1e3)}


def emit(line, rank):
    """Rank 0 prints the JSON line; the other ranks print nothing."""
    if rank != 0:
        return False
    print(json.dumps(line), flush=True)
    return True


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def _oracle_column(workload):
    from paper_2502_13695_gb300 import workloads as wl
    cfg = wl.config2() if workload == "silica" else wl.config3()
    return cfg, dict(cfg, nx=4, ny=4, precision="fp64")


def _time_oracle(s, steps):
    psteps = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        psteps += s.np
        s.step(1)
    return psteps, time.perf_counter() - t0


def oracle_sample(prerun, steps, workload="silica", openmp=False):
    """Time the FP64 oracle on a 4 x 4 transverse column of the workload
    (silica: 128x128x512; mirror: 256x256x1024), prerun to the same step;
    returns (particle-steps/s, cell-updates/s, info, state), state being
    what oracle_sample_from_state needs to time the same steps again."""
    import oracle
    oracle.build(openmp=openmp)
    cfg, col = _oracle_column(workload)
    s = oracle.Sim(col, openmp=openmp)
    s.step(prerun)
    n0 = s.np
    state = dict(s.state(), flux=s.flux())
    psteps, dt = _time_oracle(s, steps)
    ncell = col["nx"] * col["ny"] * col["nz"]
    return psteps / dt, ncell * steps / dt, dict(
        sample=f"4x4x{cfg['nz']} column of the {cfg['nx']}x{cfg['ny']}x{cfg['nz']} "
               f"{workload} workload (same z profile), "
               f"steps {prerun}..{prerun + steps}, {n0} charged macroparticles at start",
        seconds=dt, cores=oracle.threads(openmp), workload=cfg["name"],
        grid=[cfg["nx"], cfg["ny"], cfg["nz"]]), state


def oracle_sample_from_state(state, steps, workload="silica"):
    """Time the same sample on the OpenMP build (all host cores) from the
    state oracle_sample started its timed steps from."""
    import oracle
    oracle.build(openmp=True)
    cfg, col = _oracle_column(workload)
    s = oracle.Sim(col, openmp=True)
    sc = state["scalars"]
    s.set_scalars(sc["step"], sc["U_joule"], sc["N_pairs"], sc["U_ion"], sc["n_events"])
    s.set_fields(state["fields"])
    s.set_particles(state["particles"])
    s.set_material(state["material"]["alive"], state["material"]["win"])
    s.set_flux(state["flux"])
    psteps, dt = _time_oracle(s, steps)
    ncell = col["nx"] * col["ny"] * col["nz"]
    return psteps / dt, ncell * steps / dt, oracle.threads(True)


def oracle_samples_async(jobs):
    """Start oracle_sample(prerun, steps, workload) for each job in its own
    spawned process (started before any GPU call), so that the oracle's long
    preruns overlap the GPU measurements; returns (executor, futures)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    ex = ProcessPoolExecutor(max_workers=max(1, len(jobs)), mp_context=mp.get_context("spawn"))
    return ex, [ex.submit(oracle_sample, *j) for j in jobs]


def cpu_baseline_entry(res, steps, workload):
    """cpu_baseline object: the OpenMP build on all host cores, with the
    single-core serial build beside it, over the same sample."""
    ps1, cu1, info, state = res
    psm, cum, cores = oracle_sample_from_state(state, steps, workload)
    return {"value": psm, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": info["sample"] + "; OpenMP build (field, window and Keldysh loops "
                      "parallel; particle and ionisation passes serial)",
            "cell_updates_per_s": cum,
            "single_core": {"value": ps1, "cores": 1, "cell_updates_per_s": cu1}}


def run_reference(args, rank, world, dist):
    if rank != 0:
        return
    steps = max(1, args.steps if args.ref_steps is None else args.ref_steps)
    ps, cu, info, _ = oracle_sample(args.prerun + args.warmup, steps, openmp=True)
    line = {"metric": METRIC, "value": ps, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * info["seconds"] / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": info["workload"], "grid": info["grid"], "ppc": 8,
                       "prerun_steps": args.prerun,
                       "parallelism": f"FP64 oracle, OpenMP build, {info['cores']} host threads"},
            "cell_updates_per_s": cu,
            "cpu_baseline": {"value": ps, "unit": UNIT, "cores": info["cores"],
                             "kind": "oracle", "sample": info["sample"]},
            "e2e": {"value": ps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
# Whole step (per cell, per material cell extra, per charged particle, per
# ionisation event), FP32 and FP64 (8-byte reals, integer words unchanged).
STEP_BYTES = {"fp32": (72.0, 65.0, 60.0, 64.0), "fp64": (144.0, 129.0, 108.0, 112.0)}
ALG_BYTES_F64 = {  # as ALG_BYTES below, with 8-byte reals
    "push": ("particle", 108.0),       # (cell 4 + offset 24 + u 24) x 2 + tag 4
    "fields": ("field point", 144.0),  # + 96 per material point below
    "window": ("material cell", 88.0),  # the 40 B of reals doubled, threshold 8
    "ionize": ("material cell", 16.0),
    "sort": ("particle", 128.0),
    "collide": ("particle", 60.0),
}
ALG_BYTES = {  # FP32 algorithmic bytes per unit of work of each kernel class
    "push": ("particle", 60.0),
    "fields": ("field point", 72.0),  # whole field update; + 48 per material point below
    "window": ("material cell", 48.0),
    "ionize": ("material cell", 16.0),
    "sort": ("particle", 80.0),
    "collide": ("particle", 36.0),  # momentum read + write 24, tag 4, id 8
}
# what bounds each kernel class in practice, as measured (ncu counters and
# timing experiments), where it is not DRAM bandwidth
LIMITER = {
    "push": "L1 sector throughput of the gather loads and current reductions "
            "(~39 + 21 sectors per particle, L1 ~72% busy)",
    "keldysh": "FP32 issue (series of Dawson terms)",
    "ionize": "load latency and integer issue (Philox draws)",
    "collide": "issue rate and lane divergence of the per-pair arithmetic",
}


def measure_workload(cfg, args, rank, local, world, dist, prerun, steps, warmup):
    """Time `steps` full steps of cfg after `prerun + warmup` untimed ones
    (CUDA events on the simulation's stream, clocks sampled meanwhile), then
    up to 200 more steps with every kernel class timed by events (the
    classes then run in order, without the overlap of a plain step, and the
    events add their own cost: a breakdown, not the step time), then one
    whole job of cfg["steps"] steps through the public API (e2e).
    Returns the fields of a bench line for this workload."""
    import torch
    from paper_2502_13695_gb300 import pic
    precision = cfg.get("precision", "fp32")
    sim = pic.Simulation(cfg)
    st = sim.static
    sim.step(prerun + warmup)
    sim.sync()
    stream = sim.stream
    i0, s0 = sim.info(), sim.scalars()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    with Clocks(gpu_index if gpu_index.isdigit() else local) as clk:
        # an NVTX range "timed" marks the timed steps for profilers
        # (ncu --nvtx --nvtx-include "timed/")
        nvtx_push("timed")
        ev0.record(stream)
        sim.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        nvtx_pop()
    ms = ev0.elapsed_time(ev1)
    sim.sync()
    i1, s1 = sim.info(), sim.scalars()
    # the per-class breakdown, from its own profiled steps
    prof_steps = min(steps, 200)
    sim.profile(True)
    sim.step(prof_steps)
    sim.sync()
    prof = sim.profile_read()
    sim.profile(False)
    i2 = sim.info()
    psteps_prof = i2["particle_steps"] - i1["particle_steps"]
    psteps = i1["particle_steps"] - i0["particle_steps"]
    events = s1["n_events"] - s0["n_events"]
    launches = i1["launches"] - i0["launches"]
    agg = aggregate(dist, ms, psteps, events)
    ms_max, psteps_all, events_all = agg["ms_max"], agg["psteps_all"], agg["events_all"]
    t = ms_max / 1e3
    ncell = cfg["nx"] * cfg["ny"] * cfg["nz"]
    cells_all = ncell * steps * world
    b_cell, b_mat, b_part, b_ev = STEP_BYTES[precision]
    alg = (b_cell * ncell + b_mat * st["nmat"]) * steps * world + b_part * psteps_all \
        + b_ev * events_all
    peak, peak_kind = measured_peaks()
    # dominant kernel roofline
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    table = ALG_BYTES_F64 if precision == "fp64" else ALG_BYTES
    limiter = LIMITER.get(dom, "DRAM bandwidth")
    if precision == "fp64" and dom == "push":
        limiter = "the deposit's FP64 atomic additions (up to three per node)"
    elif precision == "fp64" and dom == "keldysh":
        limiter = "FP64 issue (series of Dawson terms)"
    unit_name, per_unit = table.get(dom, ("step", 0.0))
    if dom == "push":
        units = psteps_prof / max(dom_n, 1)
    elif dom in ("sort", "collide"):
        units = (i1["n_particles"] + i0["n_particles"]) / 2
    elif unit_name == "field point":
        units = st["nfield"]
    else:
        units = st["nmat"]
    bytes_launch = per_unit * units
    if dom == "fields":
        bytes_launch += (96.0 if precision == "fp64" else 48.0) * st["nmat"]
    achieved = bytes_launch / (dom_ms / dom_n / 1e3) / 1e9 if dom_n else 0.0
    # end to end: one whole job of the workload through the public API
    sim.close()
    del sim
    torch.cuda.synchronize()
    job_steps = int(cfg["steps"])
    t0 = time.perf_counter()
    job = pic.Simulation(cfg)
    job.step(job_steps)
    jd = job.diagnostics(n_bins=64, e_min_eV=0.0, e_max_eV=100.0)
    e2e_t = time.perf_counter() - t0
    ji = job.info()
    job.close()
    del job
    torch.cuda.empty_cache()
    e2e_t = allreduce(dist, e2e_t, _op(dist, "max"))
    e2e_ps = allreduce(dist, ji["particle_steps"], _op(dist, "sum")) / e2e_t
    return {
        "value": agg["value"], "ms_per_step": ms_max / steps,
        "cell_updates_per_s": cells_all / t,
        "hbm_roofline_frac": alg / t / (peak * 1e9),
        "hbm_alg_bytes_per_step": alg / steps / world,
        "timed_steps": [prerun + warmup, prerun + warmup + steps],
        "charged_particles": [i0["n_particles"], i1["n_particles"]],
        "ionisation_events": events,
        # from the profiled steps after the timed ones (classes in order)
        "per_kernel_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items()},
        "per_kernel_steps": [prerun + warmup + steps, prerun + warmup + steps + prof_steps],
        # a class with no algorithmic bytes (Keldysh) is bound by arithmetic:
        # no HBM fraction is claimed for it
        "roofline": {"kernel": dom, "bound": "hbm" if per_unit else "alu", "limiter": limiter,
                     "achieved": achieved if per_unit else None,
                     "peak": peak if per_unit else None,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if per_unit else None,
                     "bytes_per_launch": bytes_launch,
                     "unit_of_work": unit_name, "per_unit_bytes": per_unit,
                     # the committed ncu capture is of the FP32 kernels
                     "traffic": ncu_traffic(dom, units) if precision == "fp32" else None},
        "e2e": {"value": e2e_ps, "unit": UNIT, "job_steps": job_steps, "job_s": e2e_t,
                "h2d_bytes_per_step": ji["h2d_bytes"] / job_steps,
                "d2h_bytes_per_step": ji["d2h_bytes"] / job_steps,
                "frac_absorbed": jd["frac_absorbed"],
                "frac_reflected": jd["frac_reflected"],
                "frac_absorbed_flux": jd["frac_absorbed_flux"],
                "n_e_peak_m3": jd["n_e_peak"]},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "arena_gb": st["arena_bytes"] / 1e9,
    }


def run_native(args, rank, local, world, dist):
    import torch
    from paper_2502_13695_gb300 import build, workloads as wl
    full = world == 1 and not args.silica_only and args.precision == "fp32" and not args.transverse
    # the oracle's CPU baselines run in spawned processes beside the GPU work
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        jobs = [(args.prerun, args.cpu_steps, "silica")]
        if full:
            jobs.append((args.mirror_prerun, args.cpu_steps, "mirror"))
        cpu = oracle_samples_async(jobs)
    build.build()
    torch.cuda.set_device(local)
    cfg = wl.config2()
    if args.precision == "fp64":
        cfg["precision"] = "fp64"
        cfg["name"] = cfg["name"].replace("fp32", "fp64")
    if args.transverse:
        cfg["nx"] = cfg["ny"] = args.transverse
        cfg["name"] = cfg["name"].replace("128x128", f"{args.transverse}x{args.transverse}")
    cfg["seed"] = replica_seed(cfg["seed"], rank)  # independent replica per rank
    if args.pool_factor is not None:
        cfg["pool_factor"] = args.pool_factor
    if args.coll_every:
        cfg["coll_every"] = args.coll_every
    if args.sort_interval:
        cfg["sort_interval"] = args.sort_interval
    m = measure_workload(cfg, args, rank, local, world, dist, args.prerun, args.steps, args.warmup)
    mirror = scan = None
    if full:
        # the 20-pair multilayer mirror (256 x 256 x 1024, 3000 steps)
        mcfg = wl.config3()
        mm = measure_workload(mcfg, args, rank, local, world, dist, args.mirror_prerun,
                              args.steps, args.warmup)
        mirror = {"workload": mcfg["name"], "grid": [mcfg["nx"], mcfg["ny"], mcfg["nz"]],
                  "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
                  "prerun_steps": args.mirror_prerun,
                  "l2": "state larger than L2 (%.1f GB), no flush" % mm["arena_gb"]}
        mirror.update({k: v for k, v in mm.items() if k != "arena_gb"})
        torch.cuda.empty_cache()
        scan = run_scan(args, emit_line=False)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "grid": [cfg["nx"], cfg["ny"], cfg["nz"]],
                   "ppc": 8, "prerun_steps": args.prerun, "pool_factor": cfg["pool_factor"],
                   "collisions_every": args.coll_every,
                   "sort_interval": args.sort_interval or 16,
                   "l2": "state larger than L2 (%.1f GB), no flush" % m["arena_gb"],
                   "parallelism": f"replicas x{world}"},
    }
    line.update({k: v for k, v in m.items() if k not in ("value", "ms_per_step", "arena_gb")})
    if mirror is not None:
        line["mirror"] = mirror
    if scan is not None:
        line["scan"] = {k: scan[k] for k in ("config", "scan_time_to_result_s", "value",
                                             "cell_updates_per_s", "one_at_a_time",
                                             "batched_total_s", "two_waves_total_s",
                                             "one_launch_per_phase",
                                             "damage_threshold_fluence_J_cm2",
                                             "gpu_launches_per_step", "batch_tuning")}
        line["scan"]["unit"] = UNIT
        line["scan_time_to_result_s"] = scan["scan_time_to_result_s"]
    if cpu is not None:
        ex, futs = cpu
        res = [f.result() for f in futs]
        ex.shutdown()
        line["cpu_baseline"] = cpu_baseline_entry(res[0], args.cpu_steps, "silica")
        if mirror is not None and len(res) > 1:
            mirror["cpu_baseline"] = cpu_baseline_entry(res[1], args.cpu_steps, "mirror")
    emit(line, rank)


def run_scan(args, emit_line=True):
    """Batched fluence scan: 64 instances 64x64x{128..512}, fluence 0.1-3
    J cm^-2 log-spaced, FP32, advanced together from one CUDA graph, against
    the same instances run one at a time on the same GPU.  An instance's
    result is its damage metrics (pic_damage); time-to-result is measured
    from the start of its mode's run to that result on the host.  The line
    also reports, per damage criterion, the lowest fluence of the scan whose
    instance meets it (the scan's damage-threshold estimate)."""
    import torch
    from paper_2502_13695_gb300 import build, pic, workloads as wl
    build.build()
    cfgs = wl.config4(args.scan_instances)
    steps = args.scan_steps
    def batched(one_launch):
        """Every instance on its own stream, one graph per 32-step period
        (each member's own launches, or batch launches); returns the time,
        particle steps, kernel launches, results and tuning record."""
        sims = [pic.Simulation(c, stream=torch.cuda.Stream()) for c in cfgs]
        batch = pic.Batch(sims, one_launch_per_phase=one_launch)
        batch.step(32)  # capture + warm-up
        batch.sync()
        p0 = sum(s.info()["particle_steps"] for s in sims)
        l0 = sum(s.info()["launches"] for s in sims)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.step(steps)
        batch.sync()
        res = [s_.damage() for s_ in sims]
        t = time.perf_counter() - t0
        p = sum(s.info()["particle_steps"] for s in sims) - p0
        nl = sum(s.info()["launches"] for s in sims) - l0
        tu = batch.tuning()
        batch.close()
        for s_ in sims:
            s_.close()
        del sims
        torch.cuda.empty_cache()
        return t, p, nl, res, tu

    t_batch, p_batch, launches, results, _ = batched(False)
    t_one, p_one, launches_one, _, tuning = batched(True)
    cells = sum(c["nx"] * c["ny"] * c["nz"] for c in cfgs) * steps
    # two batched waves, the cheaper half of the instances (fewest cells)
    # first: each wave created and warmed 32 steps outside the clock, as the
    # one-at-a-time runs below are; a result's time counts every wave
    # before its own
    order = sorted(range(len(cfgs)), key=lambda q: cfgs[q]["nx"] * cfgs[q]["ny"] * cfgs[q]["nz"])
    half = len(order) // 2
    lat_w, t_w = [], 0.0
    for wave in (order[:half], order[half:]):
        if not wave:
            continue
        ws = [pic.Simulation(cfgs[q], stream=torch.cuda.Stream()) for q in wave]
        wb = pic.Batch(ws)
        wb.step(32)
        wb.sync()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        wb.step(steps)
        wb.sync()
        for s_ in ws:
            s_.damage()
        t_w += time.perf_counter() - t1
        lat_w += [t_w] * len(wave)
        wb.close()
        for s_ in ws:
            s_.close()
        del ws
        torch.cuda.empty_cache()
    lat_w = sorted(lat_w)
    # one at a time (each instance created, warmed 32 steps, then timed)
    lat, t_seq, p_seq = [], 0.0, 0.0
    for c in cfgs:
        sim = pic.Simulation(c)
        sim.step(32)
        sim.sync()
        q0 = sim.info()["particle_steps"]
        t1 = time.perf_counter()
        sim.step(steps)
        sim.damage()
        t_seq += time.perf_counter() - t1
        lat.append(t_seq)
        p_seq += sim.info()["particle_steps"] - q0
        sim.close()
        del sim
    torch.cuda.empty_cache()
    lat = sorted(lat)

    def pct(v, q):
        return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)]

    # lowest scanned fluence meeting each criterion (any layer)
    names = ["critical_density", "instability_density", "melting", "boiling", "dissociation"]
    lidt = {}
    for bit, name in enumerate(names):
        hit = [c["pulse"]["fluence"] / 1e4 for c, r in zip(cfgs, results)
               if any(ly["flags"] >> bit & 1 for ly in r["layers"])]
        lidt[name] = min(hit) if hit else None

    line = {"metric": METRIC, "value": p_batch / t_batch, "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": 32, "ms_per_step": 1e3 * t_batch / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"fluence scan, {len(cfgs)} instances 64x64x(128..512)",
                       "mode": "batched CUDA graph, each member's own launches"},
            "cell_updates_per_s": cells / t_batch,
            "scan_time_to_result_s": {"batched_p50": t_batch, "batched_p99": t_batch,
                                      "two_waves_p50": pct(lat_w, 0.5),
                                      "two_waves_p99": pct(lat_w, 0.99),
                                      "one_at_a_time_p50": pct(lat, 0.5),
                                      "one_at_a_time_p99": pct(lat, 0.99)},
            "two_waves_total_s": t_w,
            "one_at_a_time": {"particle_steps_per_s": p_seq / t_seq,
                              "cell_updates_per_s": cells / t_seq, "total_s": t_seq},
            "batched_total_s": t_batch,
            "gpu_launches_per_step": launches / steps,
            # the same batch with batch launches (one per phase for all
            # members), its launches per step and the push launch shapes it
            # measured on itself (inside the timed steps: each candidate runs
            # real periods) with its pick
            "one_launch_per_phase": {"total_s": t_one, "particle_steps_per_s": p_one / t_one,
                                     "gpu_launches_per_step": launches_one / steps},
            "batch_tuning": tuning,
            "damage_threshold_fluence_J_cm2": lidt,
            "peak_ne_m3": [max(ly["ne_peak"] for ly in r["layers"]) for r in results],
            "peak_energy_density_J_m3": [max(ly["ed_peak"] for ly in r["layers"]) for r in results]}
    if emit_line:
        print(json.dumps(line), flush=True)
    return line


def run_paper(args):
    """One whole job in the paper's own geometry (Sec. 3): the bulk-silica
    slab or the quarter-wave mirror with the 7 fs sine-squared pulse and its
    4.65 um spot, 24 fs of simulated time, FP32.  Timed from the host
    configuration to the diagnostics and damage metrics on the host; the
    step loop alone is also timed with CUDA events."""
    import torch
    from paper_2502_13695_gb300 import build, pic, workloads as wl
    build.build()
    kw = {} if args.fluence is None else {"fluence_Jcm2": args.fluence}
    if args.coll_every:
        kw["collisions"] = True
    cfg = wl.paper_silica(**kw) if args.workload == "paper-silica" else wl.paper_mirror(**kw)
    if args.coll_every:
        cfg["coll_every"] = args.coll_every
    steps = cfg["steps"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = pic.Simulation(cfg)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    sim.step(steps)
    ev1.record(sim.stream)
    c0 = cfg["nx"] // 2
    # centre of the spot, averaged over 6 x 6 nodes as the paper's profiles
    dmg = sim.damage([c0 - 3, c0 + 3, c0 - 3, c0 + 3])
    # electron spectrum of a (200 nm)^2 column through the first layer at
    # the spot centre (the region of the paper's spectra, Sec. 4.3)
    half = max(1, int(round(100e-9 / cfg["dx"])))
    ly0 = cfg["layers"][0]
    nb, emax = 400, 200.0
    diag = sim.diagnostics(n_bins=nb, e_min_eV=0.0, e_max_eV=emax,
                           region=[c0 - half, c0 + half, c0 - half, c0 + half, ly0["z0"], ly0["z1"]])
    t_job = time.perf_counter() - t0
    import numpy as np
    from paper_2502_13695_gb300.analysis import fit_chi2
    spec = diag["spectrum"]
    fit = fit_chi2(np.linspace(0.0, emax, nb + 1), spec) if spec.sum() > 0 else None
    ms = ev0.elapsed_time(ev1)
    info = sim.info()
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"] * steps
    names = ["critical_density", "instability_density", "melting", "boiling", "dissociation"]
    layers = [{"z": [l["z0"], l["z1"]], "gap_eV": l["gap_eV"],
               "ne_peak_m3": d["ne_peak"], "energy_density_peak_J_m3": d["ed_peak"],
               "intensity_max": d["imax_peak"],
               "criteria_met": [n for b, n in enumerate(names) if d["flags"] >> b & 1]}
              for l, d in zip(cfg["layers"], dmg["layers"])]
    line = {"metric": METRIC, "value": info["particle_steps"] / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": [cfg["nx"], cfg["ny"], cfg["nz"]],
                       "cells_nm": [cfg["dx"] * 1e9, cfg["dy"] * 1e9, cfg["dz"] * 1e9],
                       "fluence_J_cm2": cfg["pulse"]["fluence"] / 1e4,
                       "pulse": "7 fs sine-squared, w0 4.65 um", "collisions_every": cfg.get("coll_every", 0)},
            "cell_updates_per_s": cells / (ms / 1e3), "time_to_result_s": t_job,
            "absorbed_fraction": diag["frac_absorbed"], "U_incident_J": diag["U_incident"],
            "n_crit_m3": dmg["n_crit"], "layers": layers[:6],
            "spectrum_chi2_fit": None if fit is None else
            {"k": fit["k"], "sigma_eV": fit["sigma"], "mean_eV": fit["mean"],
             "region": "(200 nm)^2 x first layer at the spot centre"}}
    print(json.dumps(line), flush=True)
    sim.close()


def run_serve(args):
    """Serving trace: Poisson arrivals (4/s) of silica or 10-pair mirror
    requests on grids 32^3 .. 128x128x512, 500-2000 steps, FP32, admitted
    against a 150 GB budget with continuous batching; compared with serving
    the same trace one request at a time (FIFO, each request's service time
    measured alone on the same GPU)."""
    import torch
    from paper_2502_13695_gb300 import build, pic, serve, workloads as wl
    build.build()
    trace = wl.config5(args.serve_requests)
    reqs = [serve.Request(q, t["cfg"], t["cfg"]["steps"], t["arrival_s"]) for q, t in enumerate(trace)]
    # one at a time: service time of every request alone (create, steps,
    # diagnostics: the whole life of a request, as the server's
    # time-to-result counts it), then FIFO in time
    service = []
    psteps_alone = 0.0
    torch.cuda.synchronize()
    for r in reqs:
        t0 = time.perf_counter()
        sim = pic.Simulation(r.cfg)
        sim.step(r.steps)
        sim.diagnostics()
        service.append(time.perf_counter() - t0)
        psteps_alone += sim.info()["particle_steps"]
        sim.close()
        del sim
    torch.cuda.empty_cache()
    free_at, fifo = 0.0, []
    for r, sv in zip(reqs, service):
        start = max(r.arrival_s, free_at)
        free_at = start + sv
        fifo.append(free_at - r.arrival_s)
    # continuous batching in real time
    srv = serve.Server(budget_bytes=150e9)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    lat = sorted(r.time_to_result_s for r in res)
    fifo = sorted(fifo)
    # how many requests were resident at once (from admit / done times)
    ev = sorted([(r.admit_s, 1) for r in res] + [(r.done_s, -1) for r in res])
    live, peak_live, area = 0, 0, 0.0
    for q, (t, dv) in enumerate(ev):
        if q:
            area += live * (t - ev[q - 1][0])
        live += dv
        peak_live = max(peak_live, live)
    waits = sorted(r.admit_s - r.arrival_s for r in res)

    def pct(v, q):
        return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)]

    line = {"metric": METRIC, "value": psteps_alone / wall, "unit": UNIT, "n_gpus": 1,
            "steps": sum(r.steps for r in reqs), "warmup": 0,
            "ms_per_step": 1e3 * wall / max(1, sum(r.steps for r in reqs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serving trace, {len(reqs)} requests, Poisson 4/s, "
                                   "budget 150 GB", "mode": "continuous batching"},
            "serve_time_to_result_s": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99),
                                       "one_at_a_time_p50": pct(fifo, 0.5),
                                       "one_at_a_time_p99": pct(fifo, 0.99)},
            "serve_wall_s": wall, "one_at_a_time_busy_s": sum(service),
            "last_arrival_s": reqs[-1].arrival_s,
            "resident": {"peak": peak_live, "mean": area / max(ev[-1][0] - ev[0][0], 1e-9)},
            "admission_wait_s": {"p50": pct(waits, 0.5), "p99": pct(waits, 0.99)},
            "one_at_a_time_particle_steps_per_s": psteps_alone / sum(service)}
    print(json.dumps(line), flush=True)


def _op(dist, name):
    if dist is None:
        return None
    return {"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[name]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prerun", type=int, default=1700,
                    help="untimed steps before the silica window (the job has 2000)")
    ap.add_argument("--mirror-prerun", type=int, default=2500,
                    help="untimed steps before the mirror window (the job has 3000)")
    ap.add_argument("--silica-only", action="store_true",
                    help="skip the mirror workload and the fluence scan of the default line")
    ap.add_argument("--transverse", type=int, default=0,
                    help="nx = ny of the silica workload (0: its 128; smaller cases for "
                         "profiling, same z profile)")
    ap.add_argument("--pool-factor", type=float, default=None,
                    help="charged-slot capacity / neutrals (default: the workload's 3.0)")
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-steps", type=int, default=30)
    ap.add_argument("--ref-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="working precision of the bench workload (silica run)")
    ap.add_argument("--sort-interval", type=int, default=0,
                    help="steps between pool sorts (0: the library default)")
    ap.add_argument("--coll-every", type=int, default=0,
                    help="binary-collision pass every N steps (0: none, as the workload defines)")
    ap.add_argument("--workload", choices=["silica", "scan", "serve", "paper-silica", "paper-mirror"],
                    default="silica")
    ap.add_argument("--fluence", type=float, default=None,
                    help="peak fluence (J cm^-2) of the paper-geometry workloads")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--scan-instances", type=int, default=64)
    ap.add_argument("--scan-steps", type=int, default=1000)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        run_reference(args, rank, world, None)
        return
    if args.workload in ("paper-silica", "paper-mirror"):
        return run_paper(args)
    if args.workload == "scan":
        run_scan(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    rank, local, world, dist = dist_setup(args.gpus)
    try:
        run_native(args, rank, local, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
