#!/usr/bin/env python
"""Throughput of the CWTHF single-scale hot path on GB300.

One step = one cwthf_find call on the resident particle set: CIC deposit,
forward FFT, then for each of the workload's wavelet scales the wavelet
multiply + inverse FFT, segmentation and particle assignment with the
per-halo catalogue.  Default workload: 512^3 = 134,217,728 clumped particles
in a 500 Mpc/h box on a 1024^3 grid, scales w = 2, 3, 4 h/Mpc.

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
replica (independent synthetic box, no collective on the data path); the
throughput is the sum over ranks of particles / max-over-ranks step time.
`--impl reference` times the fp64 CPU oracle on a bounded sample of the same
workload instead.

Besides the headline the line carries, each measured outside the timed step:
`e2e` (host buffers and copies every step), `roofline` and `stages` (CUDA
events per launch in separate steps against the algorithmic bytes, DRAM
traffic from profiles/traffic.json), `served` and `batched` (the server and
the graph batch), `cufft` and `stencil` (the library FFT route and the paper's
direct-space CWT beside this path's transform), `multiscale` (the paper's
19-scale loop on a 512^3-particle 50 Mpc/h box, without and with the
self-boundness check, with per-kernel times `kernels_ms` from one more
profiled loop) and `cpu_baseline` (the oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Mparticles/s end-to-end halo ID at 512³/1024³ grid, % HBM roofline; served p50/p99"
UNIT = "Mparticles/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="clumped-512cube-grid1024-L500")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-ng", type=int, default=128)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT (torch.fft) comparison of the transform")
    ap.add_argument("--serve-jobs", type=int, default=200, help="jobs in the served Poisson stream (0: skip)")
    ap.add_argument("--batch-jobs", type=int, default=64, help="uneven subvolumes in the batched graph (0: skip)")
    ap.add_argument("--no-multiscale", action="store_true", help="skip the multi-scale loop on the paper's box")
    return ap.parse_args()


def run_batched(args, dev):
    """64 periodic subvolumes, grids uniform over {32,64,96,128,192}^3, particles
    log-uniform in [1e4, 1e7]: one CUDA-graph launch for the whole batch (jobs on
    8 concurrent slot streams) against back-to-back single cwthf_find calls."""
    import torch
    import paper_2501_10622_gb300 as pkg
    from paper_2501_10622_gb300 import batch, synth
    from paper_2501_10622_gb300 import autotune
    subs = synth.batched_subvolumes(n_jobs=args.batch_jobs, seed=4)
    jobs = [batch.BatchJob(w.positions(dev), w.box, w.ng, [pkg.default_params(2.0)]) for w in subs]
    npart = sum(j.np for j in jobs)
    grids = sorted({j.ng for j in jobs})
    plans = autotune.tune(dev.index or 0, grids, reps=5)

    def graph_ms(fft_plans):
        gb = batch.Batch(jobs, n_slots=8, device=dev, fft_plans=fft_plans)
        try:
            gb.capture()
            for _ in range(2):
                gb.replay()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record(gb.main)
            for _ in range(reps):
                gb.replay()
            e1.record(gb.main)
            torch.cuda.synchronize(dev)
            gb.check()
            return e0.elapsed_time(e1) / reps, [(int(j.n_halo[0]), j.halo_id.clone()) for j in jobs]
        finally:
            gb.close()

    base_ms, base_res = graph_ms(None)
    g_ms, tuned_res = graph_ms(plans)
    same_tuned = all(a[0] == t[0] and bool(torch.equal(a[1], t[1])) for a, t in zip(base_res, tuned_res))
    del base_res
    b = batch.Batch(jobs, n_slots=8, device=dev)
    try:
        sums = [r[0] for r in tuned_res]
        # back to back: one context, one stream, one call per job
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        ctx = b.ctx[0]
        s = torch.cuda.current_stream(dev)
        for j in jobs:
            ctx.find(j.pos, j.box, j.ng, j.params, cat_cap=b.cat_cap, halo_id=j.halo_id, cat=j.cat,
                     n_halo=j.n_halo, stream=s)
        torch.cuda.synchronize(dev)
        e0.record(s)
        for _ in range(reps):
            for j in jobs:
                ctx.find(j.pos, j.box, j.ng, j.params, cat_cap=b.cat_cap, halo_id=j.halo_id, cat=j.cat,
                         n_halo=j.n_halo, stream=s)
        e1.record(s)
        torch.cuda.synchronize(dev)
        ctx.check()
        s_ms = e0.elapsed_time(e1) / reps
        same = sums == [int(j.n_halo[0]) for j in jobs]
    finally:
        b.close()
        del jobs
        torch.cuda.empty_cache()
    return {"jobs": args.batch_jobs, "particles": npart, "grids": grids, "slots": 8,
            "graph_ms": g_ms, "graph_mparticles_per_s": npart / g_ms / 1e3,
            "graph_ms_builtin_fft_plans": base_ms, "fft_plans": {str(k): v for k, v in plans.items()},
            "halo_ids_identical_tuned_vs_builtin": same_tuned,
            "single_calls_ms": s_ms, "single_calls_mparticles_per_s": npart / s_ms / 1e3,
            "identical_halo_counts": same}


def run_multiscale(args, dev):
    """The multi-scale loop (Fig. 1) on the paper's own configuration: 512^3
    clumped particles in a 50 Mpc/h box (SIMBA m50n512's size and particle
    count), Table 1's scales (k_w 0.1 .. 2.5, 19 values, grids Int(400 k_w +
    150) rounded to supported sizes <= 1024).  The paper's single-process CPU
    run of the whole loop (with unbinding) took about 3 hours."""
    import torch
    import paper_2501_10622_gb300 as pkg
    from paper_2501_10622_gb300 import synth
    L, npart = 50.0, 512 ** 3
    pos, vel = synth.clumped_box(npart, L, 200, seed=7, device=dev, velocities=True)
    mp = synth.particle_mass(npart, L)
    kws, ws, ngs = pkg.paper_scales(L)
    ctx = pkg.Context(dev.index or 0, max_ng=max(ngs), max_np=npart, max_scales=2, unbind=True)
    out = {}
    try:
        hid = torch.empty(npart, dtype=torch.int32, device=dev)
        cat = torch.empty((1 << 20, 64), dtype=torch.uint8, device=dev)
        nh = torch.zeros(1, dtype=torch.int64, device=dev)
        s = torch.cuda.current_stream(dev)
        for key, v in (("", None), ("unbind_", vel)):
            run = lambda: ctx.find_multiscale(pos, L, ws, ngs, mass_unit=mp, halo_id=hid, cat=cat, n_halo=nh,
                                              cat_cap=1 << 20, stream=s, vel=v)
            run()
            ctx.check(what="multi-scale warm-up")
            reps = max(1, min(args.steps, 2))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                run()
            e1.record(s)
            torch.cuda.synchronize(dev)
            ctx.check(what="multi-scale")
            ms = e0.elapsed_time(e1) / reps
            # one more loop with CUDA events around every launch, outside the timed
            # region: where the loop's time goes, per kernel
            ctx.profile(True)
            run()
            ctx.check(what="multi-scale profiled loop")
            prof = ctx.profile_read()
            ctx.profile(False)
            top = sorted(prof.items(), key=lambda kv: -kv[1][0])[:12]
            out[key + "kernels_ms"] = {k: [round(v[0], 2), int(v[1])] for k, v in top}
            n = int(nh[0])
            got = pkg.ms_catalogue_to_numpy(cat, min(n, 1 << 20))
            out.update({key + "ms": ms, key + "mparticles_per_s": npart / ms / 1e3, key + "halos": n,
                        key + "halos_per_scale": [int((got["scale"] == j).sum()) for j in range(len(ws))],
                        key + "particles_in_halos": float((hid >= 0).float().mean())})
    finally:
        ctx.close()
        del pos, vel
        torch.cuda.empty_cache()
    return {"workload": "512^3 clumped particles, L = 50 Mpc/h, 200 NFW clumps + 40 % uniform; virial velocities "
                        "for the unbind_ figures (self-boundness check of every scale's kept groups)",
            "k_w": kws, "grids": ngs, **out,
            "paper": "about 3 h for the whole CWTHF catalogue (incl. unbinding) of SIMBA m50n512 on one process "
                     "of a dual Xeon E5-2678 v3 (Appendix A); context only"}


# the served stream's slots per grid class and their HBM budget
SERVED_SLOTS = {96: 6, 192: 4, 288: 3, 384: 2, 512: 2}
SERVED_BUDGET = 120 * 2 ** 30


def run_served(args, dev):
    """A stream of halo-finding jobs with grids 64^3-512^3 (log-uniform,
    2^a 3^b), 8 particles per cell, Poisson arrivals, served by continuous
    batching under a 120 GB HBM budget, against back-to-back single calls.
    Load points: all jobs at once (the served capacity), 0.5x and 0.9x that
    capacity, and the workload's own 200 jobs/s."""
    import math
    import torch
    from paper_2501_10622_gb300 import serve
    rate0 = 200.0
    jobs = serve.poisson_jobs(args.serve_jobs, rate=rate0, lo_ng=64, hi_ng=512, per_cell=8.0, seed=5, device=dev)
    srv = serve.Server(device=dev, budget_bytes=SERVED_BUDGET, slots_per_class=SERVED_SLOTS)
    out = {"jobs": len(jobs), "grid_range": [64, 512], "particles_per_cell": 8, "hbm_budget_gb": 120,
           "distinct_grids": len({j.ng for j in jobs}), "mean_particles_per_job": sum(j.np for j in jobs) / len(jobs)}
    try:
        srv.prepare(jobs)
        warm = list({j.ng: j for j in jobs}.values())  # one job of every size: kernels and caches warm
        srv.run_back_to_back(serve.with_arrivals(warm, [0.0] * len(warm)))
        srv.run(serve.with_arrivals(warm, [0.0] * len(warm)))
        ref = {}

        def point(rate, label):
            js = serve.scaled_load(jobs, rate, rate0)
            served = srv.run(js)
            res = {j.jid: (tuple(j.n_halo), j.checksum) for j in js}
            b2b_js = serve.scaled_load(jobs, rate, rate0)
            b2b = srv.run_back_to_back(b2b_js)
            same = all(res[j.jid] == (tuple(j.n_halo), j.checksum) for j in b2b_js)
            for k, v in res.items():
                same &= ref.setdefault(k, v) == v
            return {"label": label, "arrival_rate_per_s": rate, **served,
                    "back_to_back": {k: b2b[k] for k in ("p50_ms", "p99_ms", "mean_ms", "makespan_s",
                                                         "mparticles_per_s")},
                    "identical_results_alone_vs_mixed": same}

        cap = point(math.inf, "capacity (all jobs at t = 0)")
        mean_np = out["mean_particles_per_job"]
        cap_rate = cap["mparticles_per_s"] * 1e6 / mean_np  # jobs per second at capacity
        points = [cap] + [point(f * cap_rate, f"{f:g} x capacity") for f in (0.5, 0.9)]
        points.append(point(rate0, "the workload's 200 jobs/s"))
        out.update({"slot_memory_gb": srv.used / 2 ** 30, "capacity_jobs_per_s": cap_rate, "loads": points,
                    "identical_results_alone_vs_mixed": all(p["identical_results_alone_vs_mixed"] for p in points),
                    "table_fills_while_serving": sum(p["table_fills"] for p in points)})
    finally:
        srv.close()
        del jobs
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# Algorithmic bytes: what the method itself must move, with u = cells, h = half-spectrum complex values
# ng * ng * (ng/2 + 1), p = particles, k = scales:
#   S1 deposit              12p + 8u        positions in, int64 grid out
#   S2-S4 transform         44u + 24u(k-1)  five passes over the spectrum; each
#                                           extra scale repeats the last three
#   S5-S6 segmentation      8u per scale    CWT in, labels out
#   S7-S8 assignment        20p per scale   positions in, label gather, ids out
# Each kernel is charged its share of those bytes; kernels that move only the
# build's own intermediates (bins, parent codes, slots) are charged nothing.
# ---------------------------------------------------------------------------
STAGES = {
    "S1 deposit": ("k_dep_",),
    "S2-S4 transform": ("k_fft_",),
    "S5-S6 segmentation": ("k_seg_", "k_popc", "k_seed_list"),
    "S7-S8 assignment": ("k_halo_sums", "k_keep", "k_catalogue", "k_rec_halo", "k_finalize", "k_count_cells"),
}


def stage_of(kernel):
    for st, prefixes in STAGES.items():
        if kernel.startswith(prefixes):
            return st
    return "shared (scans)"


def stage_bytes(u):
    cells, npart, k = u["cells"], u["np"], u["scales"]
    return {"S1 deposit": 12 * npart + 8 * cells,
            "S2-S4 transform": 44 * cells + 24 * cells * (k - 1),
            "S5-S6 segmentation": 8 * cells * k,
            "S7-S8 assignment": 20 * npart * k}


def algorithmic_bytes(name, u):
    """The kernel's share of its stage's algorithmic bytes, per launch."""
    cells, half, npart = u["cells"], u["half"], u["np"]
    table = {
        "k_dep_count": 12 * npart,                # positions in
        "k_dep_tile": 8 * cells,                  # int64 grid out
        "k_fft_x_fwd": 8 * cells + 8 * half,      # int64 grid in, half spectrum out
        "k_fft_yz": 2 * 8 * half,                 # half spectrum in and out
        "k_fft_x_inv": 8 * half + 4 * cells,      # half spectrum in, fp32 CWT out
        "k_seg_parent": 4 * cells,                # CWT in
        "k_seg_chase": 4 * cells,                 # labels out
        "k_halo_sums": 12 * npart + 4 * npart,    # positions (as binned records), label gather
        "k_finalize": 4 * npart * u["scales"],    # halo ids out, every scale
    }
    return table.get(name)


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sources_sha(names):
    """Short hash of the kernel sources a stored capture was taken from."""
    h = hashlib.sha256()
    for n in names:
        h.update((ROOT / "paper_2501_10622_gb300" / "csrc" / n).read_bytes())
    return h.hexdigest()[:16]


def stored_traffic(name, u):
    """DRAM bytes per launch from a committed ncu capture (profiles/traffic.json),
    scaled to this workload by its cells, if the kernel's sources are unchanged
    since the capture; else None."""
    f = ROOT / "profiles" / "traffic.json"
    if not f.exists():
        return None
    d = json.loads(f.read_text()).get(name)
    if not d:
        return None
    try:
        if sources_sha(d["sources"]) != d["sources_sha"]:
            return None
    except OSError:
        return None
    return d["dram_bytes_per_launch"] * (u["ng"] / d["ng"]) ** 3


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]) if f[3] not in ("[N/A]", "N/A") else 0.0, f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(wl, sample_ng):
    """Same generator, same cell size and particle density, smaller box."""
    from paper_2501_10622_gb300 import synth
    f = sample_ng / wl.ng
    box = wl.box * f
    npart = int(round(wl.n_particles * f ** 3))
    nclumps = max(1, int(round(wl.n_clumps * f ** 3)))
    pos = synth.clumped_box(npart, box, nclumps, seed=wl.seed).numpy()
    desc = (f"{sample_ng}^3 grid, {npart:,} particles, L={box:g} Mpc/h, {nclumps} clumps (same cell size and "
            f"particle density as the {wl.name} workload), scales {list(wl.scales)}")
    return pos, box, desc


def oracle_step(pos, box, ng, scales):
    import numpy as np
    import oracle
    grid, _ = oracle.cic(pos, box, ng)
    for w in scales:
        C = oracle.cwt(grid, box, w)
        C32 = C.astype(np.float32)
        lab = oracle.segment(C32)
        oracle.assign(pos, box, lab, C32)


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


def cpu_baseline_leg(wl, sample_ng, min_seconds=10.0, max_runs=8):
    """The oracle on one host core, on a bounded sample of the workload: the
    same sample repeated until at least min_seconds of CPU work (at most
    max_runs runs)."""
    spos, sbox, desc = oracle_sample(wl, sample_ng)
    reps, t0 = 0, time.perf_counter()
    while reps < max_runs and (reps == 0 or time.perf_counter() - t0 < min_seconds):
        oracle_step(spos, sbox, sample_ng, wl.scales)
        reps += 1
    t = time.perf_counter() - t0
    return {"value": reps * spos.shape[0] / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{desc}; {reps} runs", "seconds": t, "cpu": cpu_model()}


def run_reference(args, wl, rank):
    if rank != 0:
        return
    pos, box, desc = oracle_sample(wl, args.cpu_sample_ng)
    for _ in range(args.warmup):
        oracle_step(pos, box, args.cpu_sample_ng, wl.scales)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(pos, box, args.cpu_sample_ng, wl.scales)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = pos.shape[0] / t / 1e6
    cores = f"1 of {os.cpu_count()} ({cpu_model()})"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sample": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "cores_note": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    args = parse()
    from paper_2501_10622_gb300 import synth
    wl = synth.WORKLOADS[args.workload]
    from paper_2501_10622_gb300 import replicas
    world, rank, local = replicas.env_ranks()
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import numpy as np
    import torch
    import paper_2501_10622_gb300 as pkg

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    # replicas: each rank finds halos in its own synthetic box (weak scaling)
    pos = synth.clumped_box(wl.n_particles, wl.box, wl.n_clumps, seed=replicas.replica_seed(wl.seed, rank),
                            device=dev)
    npart, ng = pos.shape[0], wl.ng
    params = [pkg.default_params(w) for w in wl.scales]
    ns = len(params)
    cat_cap = 1 << 22
    ctx = pkg.Context(local, max_ng=ng, max_np=npart, max_scales=ns)
    hid = torch.empty((ns, npart), dtype=torch.int32, device=dev)
    cat = torch.empty((ns, cat_cap, 64), dtype=torch.uint8, device=dev)
    nh = torch.zeros(ns, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(p):
        ctx.find(p, wl.box, ng, params, cat_cap=cat_cap, halo_id=hid, cat=cat, n_halo=nh, stream=stream)

    for _ in range(max(args.warmup, 1)):
        step(pos)
    ctx.check(what="warm-up")

    def barrier():
        if dist:
            dist.barrier()

    # ---- device-resident timed region (no per-kernel events inside) ----------
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launch_count()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(pos)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    launches = ctx.launch_count() - launches0
    ctx.check(what="timed steps")
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    value = replicas.whole_job_throughput(npart, world, ms)

    # ---- per-kernel times: a separate pass with CUDA events around every launch
    prof_steps = max(2, min(args.steps, 5))
    ctx.profile(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(prof_steps):
        step(pos)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.check(what="profiled steps")
    prof_ms = p0.elapsed_time(p1) / prof_steps

    # ---- per-kernel and per-stage roofline --------------------------------------
    peak, peak_kind = measured_peaks()
    u = dict(ng=ng, np=npart, cells=ng ** 3, half=ng * ng * (ng // 2 + 1), scales=ns)
    kernels, stage_ms = {}, {}
    for name, (tot, n) in prof.items():
        b = algorithmic_bytes(name, u)
        avg = tot / n
        ent = {"launches_per_step": n / prof_steps, "avg_ms": avg, "ms_per_step": tot / prof_steps,
               "share": tot / prof_steps / prof_ms, "stage": stage_of(name)}
        if b:
            ent["algorithmic_bytes"] = b
            ent["gbs"] = b / (avg / 1e3) / 1e9
            ent["frac"] = ent["gbs"] / peak
        kernels[name] = ent
        stage_ms[ent["stage"]] = stage_ms.get(ent["stage"], 0.0) + tot / prof_steps
    dom = max((k for k in kernels if "gbs" in kernels[k]), key=lambda k: kernels[k]["ms_per_step"])
    d = kernels[dom]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": d["gbs"], "peak": peak, "unit": "GB/s",
                "frac": d["gbs"] / peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy burst)",
                "traffic": stored_traffic(dom, u), "algorithmic_bytes_per_launch": d["algorithmic_bytes"]}
    sb = stage_bytes(u)
    stages = {st: {"algorithmic_bytes": b, "ms_per_step": stage_ms.get(st, 0.0),
                   "gbs": b / (stage_ms[st] / 1e3) / 1e9 if stage_ms.get(st) else None,
                   "frac": b / (stage_ms[st] / 1e3) / 1e9 / peak if stage_ms.get(st) else None}
              for st, b in sb.items()}
    stages["shared (scans)"] = {"ms_per_step": stage_ms.get("shared (scans)", 0.0)}
    step_bytes = sum(sb.values())

    # ---- end to end through host buffers ---------------------------------------
    # Every step copies its positions host -> device and its halo ids and counts
    # device -> host (pinned buffers).  Measured twice: serially on one stream,
    # and pipelined, where step i+1's upload and step i-1's download run on two
    # copy streams beside step i's kernels (double-buffered device inputs and
    # outputs); the pipelined figure is the reported one.
    e2e = None
    if not args.no_e2e:
        pos_h = pos.cpu().pin_memory()
        hid_h = [torch.empty(hid.shape, dtype=hid.dtype).pin_memory() for _ in range(2)]
        nh_h = [torch.empty(nh.shape, dtype=nh.dtype).pin_memory() for _ in range(2)]
        pos_d = [torch.empty_like(pos) for _ in range(2)]
        hid_d = [hid, torch.empty_like(hid)]
        nh_d = [nh, torch.empty_like(nh)]

        def run_find(j):
            ctx.find(pos_d[j], wl.box, ng, params, cat_cap=cat_cap, halo_id=hid_d[j], cat=cat, n_halo=nh_d[j],
                     stream=stream)

        def serial_steps(k):
            for _ in range(k):
                pos_d[0].copy_(pos_h, non_blocking=True)
                run_find(0)
                hid_h[0].copy_(hid_d[0], non_blocking=True)
                nh_h[0].copy_(nh_d[0], non_blocking=True)

        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def pipelined_steps(k):
            def upload(j):
                with torch.cuda.stream(up):
                    if j >= 2:
                        up.wait_event(ev_used[j % 2])  # step j-2 has read this buffer
                    pos_d[j % 2].copy_(pos_h, non_blocking=True)
                    ev_in[j % 2].record(up)
            upload(0)
            for i in range(k):
                if i + 1 < k:
                    upload(i + 1)
                stream.wait_event(ev_in[i % 2])
                if i >= 2:
                    stream.wait_event(ev_out[i % 2])  # step i-2's results are on the host
                run_find(i % 2)
                ev_used[i % 2].record(stream)
                with torch.cuda.stream(down):
                    down.wait_event(ev_used[i % 2])
                    hid_h[i % 2].copy_(hid_d[i % 2], non_blocking=True)
                    nh_h[i % 2].copy_(nh_d[i % 2], non_blocking=True)
                    ev_out[i % 2].record(down)
            stream.wait_stream(down)

        def timed(fn):
            # warm-up: at least two steps, so that both halves of every double
            # buffer (pinned host and device) have been through a copy before
            # the timed steps (the first copy through a pinned buffer runs at
            # about half speed)
            fn(max(2, args.warmup))
            torch.cuda.synchronize(dev)
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            fn(args.steps)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            barrier()
            return replicas.max_over_ranks(f0.elapsed_time(f1) / args.steps, dev)

        sms = timed(serial_steps)
        ems = timed(pipelined_steps)
        ctx.check(what="e2e steps")
        assert torch.equal(hid_h[(args.steps - 1) % 2], hid_d[(args.steps - 1) % 2].cpu())
        e2e = {"value": replicas.whole_job_throughput(npart, world, ems), "unit": UNIT, "ms_per_step": ems,
               "h2d_bytes_per_step": pos.numel() * 4, "d2h_bytes_per_step": hid.numel() * 4 + nh.numel() * 8,
               "copies": "pipelined: step i+1's upload and step i-1's download overlap step i's kernels",
               "serial_value": replicas.whole_job_throughput(npart, world, sms), "serial_ms_per_step": sms}

    # ---- the transform beside cuFFT (rank 0, N = 1) ------------------------------
    # torch.fft (cuFFT) r2c of the fp32 grid once, then per scale a multiply by a
    # precomputed full kernel spectrum and a c2r: the library route to the same
    # convolutions, timed against this path's own FFT kernels (from the profiled
    # pass).  Two formulations, the faster one reported: into preallocated
    # outputs (out=), and with fresh outputs from torch's caching allocator.
    cufft = None
    if rank == 0 and world == 1 and not args.no_cufft:
        ours = sum(v["ms_per_step"] for k, v in kernels.items() if k.startswith("k_fft"))
        g = ctx.deposit(pos, wl.box, ng)
        x = g.to(torch.float32)
        del g
        kspec = torch.randn((ng, ng, ng // 2 + 1), dtype=torch.complex64, device=dev)
        X = torch.empty_like(kspec)
        Y = torch.empty_like(kspec)
        out = torch.empty((ng, ng, ng), dtype=torch.float32, device=dev)

        def preallocated():
            torch.fft.rfftn(x, out=X)
            for _ in wl.scales:
                torch.mul(X, kspec, out=Y)
                torch.fft.irfftn(Y, s=(ng, ng, ng), out=out)

        def fresh():
            Xf = torch.fft.rfftn(x)
            for _ in wl.scales:
                torch.fft.irfftn(Xf * kspec, s=(ng, ng, ng))

        times = {}
        for name, fn in (("preallocated", preallocated), ("fresh", fresh)):
            fn()
            torch.cuda.synchronize(dev)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            for _ in range(args.steps):
                fn()
            c1.record()
            torch.cuda.synchronize(dev)
            times[name] = c0.elapsed_time(c1) / args.steps
        best = min(times, key=times.get)
        cufft = {"ms_per_step": times[best], "formulation": best, "ms_per_step_each": times,
                 "ours_ms_per_step": ours,
                 "what": f"torch.fft rfftn of the fp32 {ng}^3 grid, then per scale ({len(wl.scales)}) a multiply "
                         "by a full precomputed spectrum and irfftn; ours: the k_fft_* kernels of one find step"}
        del x, kspec, X, Y, out
        torch.cuda.empty_cache()

    # ---- the paper's direct-space stencil CWT beside the FFT path (rank 0, N = 1) ----
    # Table 1's stencil is Int(1.5/k_w + 5) cells of the paper's grid
    # Int(400 k_w + 150); the same physical extent on this grid gives R.
    stencil = None
    if rank == 0 and world == 1 and not args.no_cufft:
        g = ctx.deposit(pos, wl.box, ng)
        out = torch.empty((ng, ng, ng), dtype=torch.float32, device=dev)
        per = []
        fft_scale_ms = sum(v["ms_per_step"] for k, v in kernels.items()
                           if k in ("k_fft_yz", "k_fft_x_inv")) / ns - kernels["k_fft_yz"]["avg_ms"] / ns
        for w in wl.scales:
            kw = w * wl.box / 1000.0
            ng_paper = int(400 * kw + 150)
            R = max(1, round(int(1.5 / kw + 5) * ng / ng_paper))
            ctx.transform_stencil(g, wl.box, w, R, cwt=out)
            torch.cuda.synchronize(dev)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(args.steps):
                ctx.transform_stencil(g, wl.box, w, R, cwt=out, stream=stream)
            c1.record(stream)
            torch.cuda.synchronize(dev)
            t = c0.elapsed_time(c1) / args.steps
            b = 44 * ng ** 3
            per.append({"w": w, "k_w": kw, "R": R, "ms": t, "gbs": b / (t / 1e3) / 1e9, "frac": b / (t / 1e3) / 1e9 / peak})
        ctx.check(what="stencil")
        stencil = {"scales": per, "fft_ms_per_extra_scale": fft_scale_ms,
                   "what": "cwthf_transform_stencil (three 1D passes, 44 B/cell) per scale; the FFT path's "
                           "per-scale cost (fused z pass, y inverse, x inverse) beside it"}
        del g, out
        torch.cuda.empty_cache()

    halos = [int(x) for x in nh.cpu()]
    ctx.close()
    del hid, cat
    torch.cuda.empty_cache()

    # ---- served and batched forms (rank 0, N = 1) --------------------------------------
    served = batched = None
    if rank == 0 and world == 1 and args.serve_jobs > 0:
        served = run_served(args, dev)
    if rank == 0 and world == 1 and args.batch_jobs > 0:
        batched = run_batched(args, dev)
    multiscale = None
    if rank == 0 and world == 1 and not args.no_multiscale:
        multiscale = run_multiscale(args, dev)

    # ---- CPU oracle baseline (rank 0, N = 1) ------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(wl, args.cpu_sample_ng)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
                "config": {"workload": wl.name, "n_particles": npart, "ng": ng, "box_mpc_h": wl.box,
                           "scales_h_per_mpc": list(wl.scales), "n_clumps": wl.n_clumps,
                           "l2": "inputs larger than L2 (1.6 GB positions, 8.6 GB grid): no flush",
                           "parallelism": f"replicas x{world}"},
                "grid_cells_per_s": world * ng ** 3 / (ms / 1e3),
                "algorithmic_bytes_per_step": step_bytes,
                "step_roofline_frac": step_bytes / (ms / 1e3) / 1e9 / peak,
                "roofline": roofline, "stages": stages, "kernels": kernels,
                "kernel_table_from": f"{prof_steps} separate steps with CUDA events around every launch "
                                     f"({prof_ms:.2f} ms per step there)",
                "gpu_launches": launches,
                "halos_per_scale": halos,
                "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "served": served, "batched": batched,
                "cufft": cufft, "stencil": stencil, "multiscale": multiscale}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
