"""Throughput of the kinetic Monte Carlo step on GB300 (particle-steps/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--lam L]
                    [--impl ours|reference]

A step is one pass of the whole hot path: closest-candidate search, pairing,
CM scattering, free flight and walls, binning (histogram, scan, counting-sort
scatter) and per-c-bin moments.  Default workload: the 16M-particle FP32 Sod
tube with 2000 c-bins at lambda/L = 1e-3.  The timed region runs K steps
launched kernel by kernel with CUDA events on the library's stream, bracketed
by a barrier and device synchronisation; the state (16M x 64 B x 2 buffers)
is far larger than L2, so no flush is needed between steps.

The reference arm (--impl reference) times the CPU oracle on the host cores,
on a bounded slice of the same workload (central c-bins at full density).
Under torchrun every rank runs its own replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec and HBM GB/s fraction on 1 GB300; batched vs plain at fixed L1 error"
UNIT = "particle-steps/s"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(",") for ln in self.file.read().strip().splitlines() if ln.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


FLOPS_PER_TEST = 25          # binary32 operations per candidate test


def max_over_ranks(values, world, device):
    """Elementwise maximum of per-rank timings over all ranks (the job is as
    slow as its slowest replica); unchanged on one rank."""
    values = [float(v) for v in values]
    if world == 1:
        return values
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_rate(units_per_rank, world, steps, seconds):
    """Whole-job throughput: units of every rank over the slowest rank's time."""
    return units_per_rank * world * steps / seconds


def replica_seed(seed, rank):
    """Independent replicas: rank r draws its state and its scattering with seed + r."""
    return seed + rank


def kernels_per_step(precision):
    """Kernels of one step with moments: search, move, scan, scatter, moments,
    two finalize kernels."""
    return 7
FP32_LANES = 152 * 128       # GB300: SMs x FP32 lanes per SM
FP64_TFLOPS_NOMINAL = 1.25   # GB300 dense binary64 (nominal)
B_ALG_F32 = 72               # algorithmic bytes per particle-step (binary32 state)


def profiled_traffic(kernel, workload, lam):
    """dram bytes per launch of `kernel` from the committed ncu summary, if that
    summary was taken on this workload and the current kernel source (else None)."""
    import hashlib
    if workload != "sod1d_fp32_16M" or lam != 1e-3:
        return None
    path = os.path.join(ROOT, "profiles", f"{kernel}_kernel_sod1d_16M.md")
    src = os.path.join(ROOT, "paper_1210_8084_gb300", "csrc", "kmc_kernels.cuh")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    fields = dict(ln.split(":", 1) for ln in text.splitlines() if ln.startswith(("source_sha256:", "traffic_bytes_per_launch:")))
    if fields.get("source_sha256", "").strip() != sha:
        return None
    try:
        return int(fields["traffic_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


def algorithmic_bytes(n, n_keys, n_bins, frac_paired, phase):
    """Bytes each kernel must move at least (binary32 state), per launch.
    State of a particle: position 12 B + id 4 B, velocity 12 B + instance 4 B."""
    if phase == "search":
        return n * (32 + 8)                    # read own state once, write the partner key
    if phase == "move":                        # own state, partner key, partner's key, B, key, slot, histogram
        return n * (32 + 8 + 8 + 32 + 4 + 4 + 4) + n * frac_paired * 32
    if phase == "moments":                     # read A once, bin sums
        return n * 32 + n_bins * 72 * 2
    if phase == "scan":
        return n_keys * (4 + 4 + 4)            # read count, write start, clear count
    if phase == "scatter":                     # key, slot, start[key], read B, write A, clear key
        return n * (4 + 4 + 4 + 32 + 32 + 8)
    return 0


def make_workload(args):
    from paper_1210_8084_gb300 import inputs
    w = dict(inputs.WORKLOADS[args.workload])
    if args.lam is not None:
        w["lam"] = args.lam
    if args.n is not None:
        w["n"] = args.n
    return w


def ours(args):
    import torch
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    w = make_workload(args)
    n = w["n"]
    pos, vel = inputs.make_state(w, seed=replica_seed(w["seed"], rank))
    dtype = np.float32 if w["precision"] == 32 else np.float64
    pos, vel = inputs.cast_state(pos, vel, dtype, w["lo"], w["hi"], w["bc"])
    stream = torch.cuda.Stream()
    cfg = k.make_config(dim_pos=w["dim_pos"], n_cells=w["n_cells"], lo=w["lo"], hi=w["hi"], bc=w["bc"],
                        lam=w["lam"], dt=w["dt"], seed=replica_seed(w["seed"], rank), precision=w["precision"],
                        stream=stream.cuda_stream, occupancy_target=args.occ)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- device-resident throughput (inputs already in HBM)
    sim = k.Simulation(cfg, pos, vel)
    info = sim.info()
    e_start = sim.moments()[2][0, 1]
    sim.step_profiled(args.warmup, want_moments=1)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    barrier()
    prof = sim.step_profiled(args.steps, want_moments=1)
    barrier()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks([prof["total"]], world, "cuda")[0]
    raw, der, glob = sim.moments()
    pairs = float(glob[0, 6])
    frac_paired = 2 * pairs / n
    energy_drift = float(glob[0, 1] / e_start - 1.0)
    cand = sim.window_size()
    sim.close()

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin_pos = torch.from_numpy(pos).pin_memory()
        pin_vel = torch.from_numpy(vel).pin_memory()
        mom_mask = k.KMC_MOM_RAW | k.KMC_MOM_DERIVED | k.KMC_MOM_GLOBAL
        barrier()
        t0 = time.perf_counter()
        h = k.kmc_init(cfg, n, pin_pos.numpy(), pin_vel.numpy(), k.KMC_WHERE_HOST)
        mom = torch.empty(k.kmc_moments_size(h, mom_mask), dtype=torch.float64).pin_memory()
        for _ in range(args.steps):
            k.kmc_step(h, 1, 1)
            k.kmc_moments(h, mom.numpy(), k.KMC_WHERE_HOST, mom_mask)
        k.kmc_get_state(h, pin_pos.numpy(), pin_vel.numpy(), k.KMC_WHERE_HOST)
        k.kmc_free(h)
        barrier()
        e2e_s = max_over_ranks([time.perf_counter() - t0], world, "cuda")[0]
        state_bytes = pos.nbytes + vel.nbytes
        e2e = {"value": job_rate(n, world, args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(state_bytes / args.steps),
               "d2h_bytes_per_step": int(mom.numel() * 8 + state_bytes / args.steps)}

    if rank != 0:
        return None

    # ---------------- roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    phases = {p: prof[p] / args.steps for p in ("search", "move", "scan", "scatter", "moments", "finalize")}
    dom = max(("search", "move", "scan", "scatter", "moments"), key=lambda p: phases[p])
    t_dom = phases[dom] * 1e-3
    traffic = profiled_traffic(dom, args.workload, w["lam"])
    if dom == "search":
        # arithmetic-bound: 25 binary32 operations per pair test (PoCA test with
        # its early outs).  The window of a particle holds C_p candidates (itself
        # included); binary32 tests every unordered pair once, (C_p - 1) / 2 per
        # particle, binary64 tests all C_p.
        tests = (cand - 1.0) / 2.0 if w["precision"] == 32 else cand
        flops = FLOPS_PER_TEST * tests * n
        if w["precision"] == 32:
            sm_clock = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
            peak = FP32_LANES * 2 * sm_clock / 1e12
            peak_src = "fp32 lanes x 2 x max SM clock (derived)"
        else:
            peak = FP64_TFLOPS_NOMINAL
            peak_src = "nominal GB300 binary64 rate"
        achieved = flops / t_dom / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_src, "ms_per_launch": round(phases[dom], 4),
                "algorithmic_flops_per_launch": int(flops), "candidates_per_particle": round(cand, 3),
                "pair_tests_per_particle": round(tests, 3)}
    else:
        ab = algorithmic_bytes(n, info.n_search_cells, info.n_bins, frac_paired, dom)
        achieved = ab / t_dom / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"{peak_src} hbm_gbs", "ms_per_launch": round(phases[dom], 4),
                "algorithmic_bytes_per_launch": int(ab)}
    step_bytes = B_ALG_F32 * n
    step_hbm = {"algorithmic_bytes_per_step": int(step_bytes),
                "achieved_gbs": round(step_bytes / (elapsed_ms / args.steps * 1e-3) / 1e9, 1),
                "frac_of_measured_hbm": round(step_bytes / (elapsed_ms / args.steps * 1e-3) / 1e9 /
                                              float(peaks.get("hbm_gbs", 6800.0)), 4)}
    value = job_rate(n, world, args.steps, elapsed_ms * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w["precision"] == 32 else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} lambda/L={w['lam']:g}", "n_particles": n,
                   "n_cells": list(w["n_cells"]), "dt": w["dt"], "precision": w["precision"],
                   "search_cells": int(info.n_search_cells), "sub_cells": list(info.sub_cells),
                   "occupancy_target": args.occ,
                   "l2": "no flush: state 2 x %.2f GB > 129 MB L2" % (n * 64 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "phase_ms_per_step": {p: round(v, 4) for p, v in phases.items()},
        "collision_fraction": round(frac_paired, 4),
        "roofline": roof,
        "step_hbm": step_hbm,
        "energy_drift_rel": energy_drift,
        "e2e": e2e,
        "gpu_launches": kernels_per_step(w["precision"]) * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_slice_bins, single_thread_bins=2)
    return out


def batched(args):
    """256 independent Sod instances (log-uniform N and lambda) stepped in one
    launch sequence per step, against the same instances stepped one handle
    at a time.  Per-instance states are identical either way (tested), so both
    runs have the same L1 error; this reports the throughput of each."""
    import torch
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    w = dict(inputs.WORKLOADS["sod1d_batched_256"])
    n_inst = args.instances or w["n_instances"]
    ns, lams = inputs.log_uniform_instances(n_inst, seed=replica_seed(w["seed"], rank), n_range=w["n_range"],
                                            lam_range=w["lam_range"])
    P, V, insts = [], [], []
    for i in range(n_inst):
        p, v = inputs.sod_tube(int(ns[i]), seed=1000 * rank + i)
        p, v = inputs.cast_state(p, v, np.float32, w["lo"], w["hi"], w["bc"])
        P.append(p)
        V.append(v)
        insts.append(dict(n=int(ns[i]), lam=float(lams[i]), dt=w["dt"], seed=1000 * rank + i))
    n_total = int(ns.sum())
    stream = torch.cuda.Stream()
    base = dict(dim_pos=3, n_cells=w["n_cells"], lo=w["lo"], hi=w["hi"], bc=w["bc"], precision=32,
                stream=stream.cuda_stream)

    def timed(h, steps):
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            k.kmc_step(h, steps, 1)
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    cfg = k.make_config(**base, instances=insts)
    pos_all, vel_all = np.concatenate(P), np.concatenate(V)
    # search set-up by measurement (outside the timed region); the plain runs use the same set-up
    tuned, tuned_ms = k.kmc_autotune(cfg, n_total, pos_all, vel_all, k.KMC_WHERE_HOST, 2)
    cfg = tuned
    sim = k.Simulation(cfg, pos_all, vel_all)
    k.kmc_step(sim.h, args.warmup, 1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms_batched = timed(sim.h, args.steps)
    clk = clocks.stop()
    sim.close()
    ms_plain = 0.0
    for i in range(n_inst):
        c = k.make_config(**base, lam=insts[i]["lam"], dt=insts[i]["dt"], seed=insts[i]["seed"],
                          occupancy_target=tuned.occupancy_target, flags=tuned.flags)
        s1 = k.Simulation(c, P[i], V[i])
        k.kmc_step(s1.h, args.warmup, 1)
        torch.cuda.synchronize()
        ms_plain += timed(s1.h, args.steps)
        s1.close()
    ms_batched, ms_plain = max_over_ranks([ms_batched, ms_plain], world, "cuda")
    if rank != 0:
        return None
    value = job_rate(n_total, world, args.steps, ms_batched * 1e-3)
    plain = job_rate(n_total, world, args.steps, ms_plain * 1e-3)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batched / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"sod1d_batched_{n_inst}", "instances": n_inst, "n_particles": n_total,
                   "n_range": list(w["n_range"]), "lambda_range": list(w["lam_range"]),
                   "n_cells_per_instance": list(w["n_cells"]), "dt": w["dt"],
                   "autotuned": {"occupancy_target": tuned.occupancy_target, "flags": tuned.flags,
                                 "ms_per_step_in_tuning": round(tuned_ms, 3)},
                   "l2": "no flush: state %.1f GB > 129 MB L2" % (n_total * 64 / 1e9)},
        "batched_vs_plain": {"batched": value, "plain_sequential": plain, "speedup": value / plain,
                             "ms_per_step_plain": ms_plain / args.steps,
                             "l1_error": "identical (per-instance states bit-identical)"},
        "gpu_launches": kernels_per_step(w["precision"]) * args.steps,
        "clocks": clk,
    }


def oracle_slice(w, n_bins_slice, seed=0):
    """Central c-bins of the workload at full density: the same particles per
    c-bin and per neighbourhood as the full run."""
    from paper_1210_8084_gb300 import inputs
    n, ncx = w["n"], w["n_cells"][0]
    dx = (w["hi"][0] - w["lo"][0]) / ncx
    half = n_bins_slice // 2
    lo = (0.5 - half * dx, w["lo"][1], w["lo"][2])
    hi = (0.5 + half * dx, w["hi"][1], w["hi"][2])
    # particles of the full tube that fall in the slice
    n_l = int(round(n * 8 / 9))
    dens_l = n_l / 0.5
    dens_r = (n - n_l) / 0.5
    n_sl = int(round(dens_l * half * dx))
    n_sr = int(round(dens_r * half * dx))
    pl, vl = inputs.sod_tube(2 * n_sl, seed, lo=lo, hi=hi, rho=(1.0, 1.0), p=(1.0, 1.0))
    pr, vr = inputs.sod_tube(2 * n_sr, seed + 1, lo=lo, hi=hi, rho=(1.0, 1.0), p=(0.8, 0.8))
    pos = np.concatenate([pl[pl[:, 0] < 0.5][:n_sl], pr[pr[:, 0] >= 0.5][:n_sr]])
    vel = np.concatenate([vl[pl[:, 0] < 0.5][:n_sl], vr[pr[:, 0] >= 0.5][:n_sr]])
    return pos, vel, lo, hi


def cpu_baseline(w, n_bins_slice=8, steps=1, single_thread_bins=0):
    """The CPU oracle on the host cores (all OpenMP threads) on a slice of
    central c-bins at full density; optionally also on one thread."""
    import oracle

    def run(nb):
        pos, vel, lo, hi = oracle_slice(w, nb)
        nbar = w["n"] / 1.0
        P = oracle.make_params(w["dim_pos"], (nb, 1, 1), lo, hi, w["bc"],
                               R2=oracle.contact_R2(w["lam"], 0.0, nbar), dt=w["dt"], seed=0,
                               decide32=w["precision"] == 32)
        t0 = time.perf_counter()
        for s in range(steps):
            P.step = s
            pos, vel = oracle.step(P, pos, vel)[:2]
        return pos.shape[0], time.perf_counter() - t0

    cores = oracle.set_threads(0)
    m, el = run(n_bins_slice)
    out = {"value": m * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle", "particles": m,
           "sample": f"{steps} oracle step(s) of the {n_bins_slice} central c-bins at full density: "
                     f"{m} particles with the full run's neighbourhood occupancy, {el:.2f} s"}
    if single_thread_bins > 0:
        oracle.set_threads(1)
        try:
            m1, el1 = run(single_thread_bins)
        finally:
            oracle.set_threads(cores)
        out["single_thread"] = {"value": m1 * steps / el1, "unit": UNIT, "cores": 1, "particles": m1,
                                "sample": f"{steps} oracle step(s) of the {single_thread_bins} central c-bins, "
                                          f"{el1:.2f} s"}
    return out


def reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    w = make_workload(args)
    samples = []
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(w, args.ref_slice_bins)
        if s >= args.warmup:
            samples.append(r)
    value = statistics.median([r["value"] for r in samples])
    n_part = samples[0]["particles"]
    cb = dict(samples[0])
    cb["value"] = value
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_part / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} lambda/L={w['lam']:g}", "n_particles": w["n"],
                   "n_cells": list(w["n_cells"]), "sample_bins": args.ref_slice_bins},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="sod1d_fp32_16M")
    ap.add_argument("--lam", type=float, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--occ", type=float, default=0.0, help="particles per search cell (0: library default)")
    ap.add_argument("--instances", type=int, default=0, help="batched workload: number of instances")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-slice-bins", type=int, default=8)
    ap.add_argument("--ref-slice-bins", type=int, default=2)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        out = reference(args)
    elif args.workload.startswith("sod1d_batched"):
        out = batched(args)
    else:
        out = ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
