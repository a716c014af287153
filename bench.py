"""Throughput of the kinetic Monte Carlo step on GB300 (particle-steps/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--lam L]
                    [--impl ours|reference] [--no-extras] [--no-e2e] [--no-cpu-baseline]

A step is one pass of the whole hot path: closest-candidate search, pairing,
CM scattering, free flight and walls, binning (histogram, scan, counting-sort
scatter into (key, id) order) and per-c-bin moments.

Default workload: the largest single-GPU configuration of the paper's set-ups,
the 3-D Sod tube with 512M particles on 1024 x 64 x 64 c-bins (lambda = 2e-4,
binary32 state).  Its search is arithmetic-bound (about 5,300 candidates per
particle in the 3^D neighbourhood), so the roofline is reported against the
FP32 rate, with the HBM fraction of the step alongside.  The same JSON line
carries, unless --no-extras:
  * sod1d_16M: the 16M-particle slab Sod tube (2000 c-bins, lambda/L = 1e-3)
    with the HBM fraction of its step and its Knudsen sweep (lambda/L = 1e-4 ...
    1);
  * batched_vs_plain: 256 Sod instances (N log-uniform in [50k, 2M],
    lambda/L log-uniform in [1e-4, 1]) in one batched handle against the same
    instances run one after another, with the L1 error of the ensemble against
    the exact Riemann solution at t = 0.1.

The timed region runs K steps launched kernel by kernel with CUDA events on the
library's stream (the per-kernel durations come from those events), bracketed
by a barrier and device synchronisation; every state is far larger than L2, so
no flush is needed between steps.  The reference arm (--impl reference) times
the CPU oracle on the host cores, on a bounded slice of the same workload
(central c-bins at full density).  Under torchrun every rank runs its own
replica (weak scaling, no collective on the data path); rank 0 prints one JSON
line.
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
DEFAULT_WORKLOAD = "sod3d_fp32_512M"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


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


FLOPS_PER_TEST = 25          # binary32 operations per candidate test (the PoCA test with its compares)
FP32_LANES_PER_SM = 128      # Blackwell SM: FP32 lanes
FP64_TFLOPS_NOMINAL = 1.25   # GB300 dense binary64 (nominal)
B_ALG_F32 = 72               # algorithmic bytes per particle-step (binary32 state)


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


def fp32_peak_tflops(n_sm, sm_mhz):
    """FP32 rate from unit counts and clock: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# Source text of each profiled kernel (with the helpers it inlines): a committed
# ncu summary carries the sha256 of this text, so that its DRAM figure is used
# only while the kernel is unchanged.
KERNEL_SEGMENTS = {
    "tile_search": ("// ------------------------------------------------------ tile search",
                    "// Direct search of one particle (global loads)"),
    "tile_pruned": ("// ------------------------------------------------------ pruned tile search (binary32)",
                    "// The plain tile search: one block per c-bin"),
    "search": ("// The PoCA acceptance test of the ordered pair (i, j)",
               "// ------------------------------------------------------ tile search"),
    "move": ("// Unambiguous pairs, CM-frame scattering", "// Counting-sort scatter B -> A in canonical order"),
    "scatter": ("// Counting-sort scatter B -> A in canonical order", "// Index (position in the input arrays"),
    "moments": ("// Moment sums per c-bin of the sorted state A", "// Candidates each particle of A examines"),
}


def kernel_source_sha(kernel):
    import hashlib
    src = open(os.path.join(ROOT, "paper_1210_8084_gb300", "csrc", "kmc_kernels.cuh")).read()
    if kernel not in KERNEL_SEGMENTS:
        return hashlib.sha256(src.encode()).hexdigest()
    a, b = KERNEL_SEGMENTS[kernel]
    i = src.index(a)
    return hashlib.sha256(src[i:src.index(b, i)].encode()).hexdigest()


def profiled_traffic(kernel, workload, n):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of this
    workload, or of its 16M-particle stand-in with the same c-bin occupancy
    (scaled by the particles a launch processes), if the summary was taken on
    the current kernel source; else None."""
    stand_in = {"sod3d_fp32_512M": ("sod3d_16M", 16_000_000), "sod3d_fp32_16M": ("sod3d_16M", 16_000_000),
                "sod1d_fp32_16M": ("sod1d_16M", 16_000_000)}
    if workload not in stand_in:
        return None
    tag, n_prof = stand_in[workload]
    path = os.path.join(ROOT, "profiles", f"{kernel}_kernel_{tag}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    fields = dict(ln.split(":", 1) for ln in text.splitlines()
                  if ln.startswith(("source_sha256:", "traffic_bytes_per_launch:")))
    if fields.get("source_sha256", "").strip() != kernel_source_sha(kernel):
        return None
    try:
        return int(int(fields["traffic_bytes_per_launch"].strip()) * n / n_prof)
    except (KeyError, ValueError):
        return None


def algorithmic_bytes(n, n_keys, n_bins, frac_paired, phase):
    """Bytes each kernel must move at least (binary32 state), per launch.
    State of a particle: position 12 B + id 4 B, velocity 12 B + virial 4 B."""
    if phase in ("search", "tile"):
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


def make_workload(name, lam=None, n=None):
    from paper_1210_8084_gb300 import inputs
    w = dict(inputs.WORKLOADS[name])
    if lam is not None:
        w["lam"] = lam
    if n is not None:
        w["n"] = n
    return w


def nbar_of(w, n=None):
    """Number density N / V of the full workload (Eq. 7's n)."""
    V = float(np.prod([w["hi"][d] - w["lo"][d] for d in range(w["dim_pos"])]))
    return (w["n"] if n is None else n) / V


PHASE_NAMES = ("search", "tile", "move", "scan", "scatter", "moments", "finalize")


def run_device(k, w, seed, steps, warmup, stream, occ=0.0, clocks=None, barrier=None, flags=0, state=None,
               tile=(0, 0, 0)):
    """One handle on a workload: warm-up, then `steps` timed steps launched
    kernel by kernel with events on the handle's stream.  Returns a dict of
    the timings, the handle's description and a few diagnostics."""
    import torch
    from paper_1210_8084_gb300 import inputs
    dtype = np.float32 if w["precision"] == 32 else np.float64
    pos, vel = state if state is not None else inputs.make_state(w, seed=seed, dtype=dtype)
    cfg = k.make_config(dim_pos=w["dim_pos"], n_cells=w["n_cells"], lo=w["lo"], hi=w["hi"], bc=w["bc"],
                        lam=w["lam"], dt=w["dt"], seed=seed, precision=w["precision"], stream=stream.cuda_stream,
                        occupancy_target=occ, flags=flags, tile_threads=tile[0], tile_cap=tile[1],
                        tile_split=tile[2])
    sim = k.Simulation(cfg, pos, vel)
    info = sim.info()
    e_start = sim.moments()[2][0, 1]
    sim.step_profiled(warmup, want_moments=1)
    if barrier:
        barrier()
    tests0 = sim.tile_tests()
    if clocks:
        clocks.start()
    if barrier:
        barrier()
    prof = sim.step_profiled(steps, want_moments=1)
    if barrier:
        barrier()
    clk = clocks.stop() if clocks else None
    tests = (sim.tile_tests() - tests0) / (w["n"] * steps) if info.tile_prune and info.n_search_cells else None
    raw, der, glob = sim.moments()
    out = dict(prof=prof, info=info, clocks=clk, pairs=float(glob[0, 6]), e_start=float(e_start),
               e_end=float(glob[0, 1]), cand=sim.window_size(), cfg=cfg, pos=pos, vel=vel, tile_tests=tests)
    sim.close()
    torch.cuda.synchronize()
    return out


def roofline_of(w, r, steps, n_sm, peaks, peak_src, workload):
    """Roofline object of the dominant kernel of a run (see run_device)."""
    n = w["n"]
    phases = {p: r["prof"][p] / steps for p in PHASE_NAMES}
    dom = max(("search", "tile", "move", "scan", "scatter", "moments"), key=lambda p: phases[p])
    t_dom = phases[dom] * 1e-3
    frac_paired = 2 * r["pairs"] / n
    kernel = {"search": "search", "tile": "tile_pruned" if r.get("tile_tests") is not None else "tile_search"}.get(dom, dom)
    traffic = profiled_traffic(kernel, workload, n)
    if dom in ("search", "tile"):
        # arithmetic-bound: 25 binary32 operations per pair test.  The window of a
        # particle holds C_p candidates (itself included); binary32 tests every
        # unordered pair once, (C_p - 1) / 2 per particle, binary64 all C_p.
        # The algorithmic work is the method's: every candidate pair of the window
        # (25 operations each).  The pruned tile search makes only the tests whose
        # swept boxes meet (counted by the kernel) and skips pairs that provably
        # cannot pass criteria 1-2; its count is reported beside the figure.
        cand = r["cand"]
        plain = (cand - 1.0) / 2.0 if w["precision"] == 32 else cand
        pruned = dom == "tile" and r.get("tile_tests") is not None
        flops = FLOPS_PER_TEST * plain * n
        if w["precision"] == 32:
            sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
            peak = fp32_peak_tflops(n_sm, sm_mhz)
            src = f"{n_sm} SMs (read at run time) x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz ({peak_src} max SM clock)"
        else:
            peak = FP64_TFLOPS_NOMINAL
            src = "nominal GB300 binary64 rate"
        achieved = flops / t_dom / 1e12
        roof = {"bound": "alu", "kernel": kernel + "_kernel", "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": src,
                "ms_per_launch": round(phases[dom], 4), "algorithmic_flops_per_launch": int(flops),
                "candidates_per_particle": round(cand, 3), "pair_tests_per_particle": round(plain, 3),
                "flops_source": f"{FLOPS_PER_TEST} binary32 operations x the window's candidate pairs per particle"}
        if pruned:
            made = r["tile_tests"]
            roof["tests_made_per_particle"] = round(made, 3)
            roof["tests_made_tflops"] = round(FLOPS_PER_TEST * made * n / t_dom / 1e12, 3)
            roof["tests_made_source"] = ("counted by the pruned tile search: (home, candidate) pairs whose swept boxes, "
                                         "widened by R and a rounding margin, meet; the others cannot pass criteria 1-2")
        if traffic is not None:
            roof["traffic_gbs"] = round(traffic / t_dom / 1e9, 1)
    else:
        ab = algorithmic_bytes(n, r["info"].n_search_cells, r["info"].n_bins, frac_paired, dom)
        achieved = ab / t_dom / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "kernel": kernel + "_kernel", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"{peak_src} hbm_gbs", "ms_per_launch": round(phases[dom], 4),
                "algorithmic_bytes_per_launch": int(ab)}
    return roof, phases


def step_hbm_of(n, ms_per_step, peaks):
    b = B_ALG_F32 * n
    gbs = b / (ms_per_step * 1e-3) / 1e9
    return {"algorithmic_bytes_per_step": int(b), "achieved_gbs": round(gbs, 1),
            "frac_of_measured_hbm": round(gbs / float(peaks.get("hbm_gbs", 6800.0)), 4)}


def launches_of(info, steps):
    return (info.kernels_per_step + info.kernels_moments) * steps


def ours(args):
    import torch
    import paper_1210_8084_gb300 as k

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peaks, peak_src = measured_peaks()
    w = make_workload(args.workload, args.lam, args.n)
    n = w["n"]
    seed = replica_seed(w["seed"], rank)
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- device-resident throughput (inputs already in HBM)
    r = run_device(k, w, seed, args.steps, args.warmup, stream, occ=args.occ, clocks=ClockSampler(local),
                   barrier=barrier, tile=(args.tile_threads, args.tile_cap, args.tile_split),
                   flags=(k.KMC_FLAG_NO_TILE_PRUNE if args.no_prune else 0) | args.flags)
    elapsed_ms = max_over_ranks([r["prof"]["total"]], world, "cuda")[0]
    pos, vel, cfg = r.pop("pos"), r.pop("vel"), r["cfg"]

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
               "d2h_bytes_per_step": int(mom.numel() * 8 + state_bytes / args.steps),
               "includes": "kmc_init from pinned host arrays, every step's moments to host, the final state to host"}
        del pin_pos, pin_vel
    del pos, vel

    extras = {}
    if not args.no_extras and args.workload == DEFAULT_WORKLOAD:
        extras["sod1d_16M"] = sod1d_extra(k, args, stream, n_sm, peaks, peak_src, barrier, world, rank)
        extras["batched_vs_plain"] = batched_vs_plain(k, args, stream, rank, world)

    if rank != 0:
        return None

    roof, phases = roofline_of(w, r, args.steps, n_sm, peaks, peak_src, args.workload)
    value = job_rate(n, world, args.steps, elapsed_ms * 1e-3)
    info = r["info"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w["precision"] == 32 else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} lambda={w['lam']:g}", "n_particles": n,
                   "n_cells": list(w["n_cells"]), "box": [list(w["lo"]), list(w["hi"])], "dt": w["dt"],
                   "precision": w["precision"], "search_cells": int(info.n_search_cells),
                   "sub_cells": list(info.sub_cells), "occupancy_target": args.occ,
                   "tile_threads": info.tile_threads, "tile_cap": info.tile_cap, "tile_split": info.tile_split,
                   "tile_prune": info.tile_prune,
                   "l2": "no flush: state 2 x %.2f GB > 129 MB L2" % (n * 32 / 1e9),
                   "parallelism": f"replicas x{world}", "n_sm": n_sm},
        "phase_ms_per_step": {p: round(v, 4) for p, v in phases.items()},
        "collision_fraction": round(2 * r["pairs"] / n, 4),
        "roofline": roof,
        "step_hbm": step_hbm_of(n, elapsed_ms / args.steps, peaks),
        "energy_drift_rel_device": (r["e_end"] - r["e_start"]) / r["e_start"],
        "e2e": e2e,
        "gpu_launches": launches_of(info, args.steps),
        "clocks": r["clocks"],
    }
    if not args.no_cpu_baseline and world == 1:
        cb, drift = cpu_baseline(w, slice_bins(w, args.cpu_slice_bins), single_thread_bins=2, device_check=True)
        out["cpu_baseline"] = cb
        out["energy_fp32_vs_fp64_oracle"] = drift
    out.update(extras)
    return out


def sod1d_extra(k, args, stream, n_sm, peaks, peak_src, barrier, world, rank):
    """The 16M-particle slab Sod tube: step throughput, its HBM fraction, the
    roofline of its dominant kernel, and the Knudsen sweep."""
    name = "sod1d_fp32_16M"
    w = make_workload(name)
    seed = replica_seed(w["seed"], rank)
    steps = max(args.steps, 20)
    r = run_device(k, w, seed, steps, args.warmup, stream, barrier=barrier)
    state = (r.pop("pos"), r.pop("vel"))
    ms = max_over_ranks([r["prof"]["total"]], world, "cuda")[0] / steps
    roof, phases = roofline_of(w, r, steps, n_sm, peaks, peak_src, name)
    sweep = {}
    for lam in w["lam_sweep"]:
        wl = dict(w, lam=lam)
        rs = run_device(k, wl, seed, 10, 3, stream, barrier=barrier, state=state)
        rs.pop("pos"), rs.pop("vel")
        ms_l = max_over_ranks([rs["prof"]["total"]], world, "cuda")[0] / 10
        sweep[f"{lam:g}"] = {"value": job_rate(w["n"], world, 1, ms_l * 1e-3), "ms_per_step": round(ms_l, 4),
                             "candidates_per_particle": round(rs["cand"], 2),
                             "collision_fraction": round(2 * rs["pairs"] / w["n"], 4),
                             "step_hbm_frac": step_hbm_of(w["n"], ms_l, peaks)["frac_of_measured_hbm"]}
    return {"workload": f"{name} lambda/L={w['lam']:g}", "n_particles": w["n"], "steps": steps,
            "value": job_rate(w["n"], world, steps, ms * steps * 1e-3), "unit": UNIT, "ms_per_step": round(ms, 4),
            "phase_ms_per_step": {p: round(v, 4) for p, v in phases.items()},
            "step_hbm": step_hbm_of(w["n"], ms, peaks), "roofline": roof,
            "search_cells": int(r["info"].n_search_cells), "collision_fraction": round(2 * r["pairs"] / w["n"], 4),
            "energy_drift_rel_device": (r["e_end"] - r["e_start"]) / r["e_start"],
            "gpu_launches": launches_of(r["info"], steps), "knudsen_sweep": sweep}


def batched_instances(rank, n_inst=None):
    from paper_1210_8084_gb300 import inputs
    w = dict(inputs.WORKLOADS["sod1d_batched_256"])
    n_inst = n_inst or w["n_instances"]
    ns, lams = inputs.log_uniform_instances(n_inst, seed=replica_seed(w["seed"], rank), n_range=w["n_range"],
                                            lam_range=w["lam_range"])
    P, V, insts = [], [], []
    for i in range(n_inst):
        p, v = inputs.sod_tube(int(ns[i]), seed=1000 * rank + i, dtype=np.float32)
        P.append(p)
        V.append(v)
        insts.append(dict(n=int(ns[i]), lam=float(lams[i]), dt=w["dt"], seed=1000 * rank + i))
    return w, ns, lams, P, V, insts


def l1_of_batch(raw, ns, lams, nc, t, lam_max=1e-3):
    """Relative L1 distance of n, p, T per instance to the exact Riemann solution
    (Sect. "Sod test"; gamma = 5/3), for the instances with lambda/L <= lam_max."""
    from analytic import riemann
    ex = riemann.sod_profile(np.linspace(0, 1, nc + 1), t, 0.5, 1.0, 1.0)
    rows = []
    for i in np.flatnonzero(lams <= lam_max):
        R = raw[nc * i:nc * (i + 1)]
        N = R[:, 0]
        u = R[:, 1] / N
        T = ((R[:, 4] + R[:, 5] + R[:, 6]) / N - (R[:, 1:4] ** 2).sum(1) / N ** 2) / 3.0
        dens = N * nc / (ns[i] * 8 / 9 / 0.5)
        q = (dens, dens * T, T)
        rows.append([float(np.abs(a - b).sum() / np.abs(b).sum()) for a, b in zip(q, (ex[:, 0], ex[:, 2], ex[:, 3]))])
    return np.array(rows)


def batched_vs_plain(k, args, stream, rank, world, n_inst=None):
    """256 independent Sod instances stepped in one launch sequence per step,
    against the same instances stepped one handle at a time with the same
    search set-up.  Per-instance states and moments are identical either way
    (tested bit for bit), so both runs have the same L1 error, reported here
    for the instances with lambda/L <= 1e-3 after the batch is run on to t = 0.1."""
    import torch
    w, ns, lams, P, V, insts = batched_instances(rank, n_inst)
    n_inst = len(ns)
    n_total = int(ns.sum())
    base = dict(dim_pos=3, n_cells=w["n_cells"], lo=w["lo"], hi=w["hi"], bc=w["bc"], precision=32,
                stream=stream.cuda_stream)

    def timed(h, steps):
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
    sim = k.Simulation(tuned, pos_all, vel_all)
    del pos_all, vel_all
    k.kmc_step(sim.h, args.warmup, 1)
    torch.cuda.synchronize()
    steps = args.steps
    ms_batched = timed(sim.h, steps)
    info = sim.info()
    # run on to t = 0.1 for the accuracy of the ensemble
    t_steps = int(round(0.1 / w["dt"]))
    done = args.warmup + steps
    if t_steps > done:
        sim.step(t_steps - done, want_moments=1)
    raw, _, _ = sim.moments()
    sim.close()
    l1 = l1_of_batch(raw, ns, lams, w["n_cells"][0], max(t_steps, done) * w["dt"])
    ms_plain = 0.0
    for i in range(n_inst):
        c = k.make_config(**base, lam=insts[i]["lam"], dt=insts[i]["dt"], seed=insts[i]["seed"],
                          occupancy_target=tuned.occupancy_target, flags=tuned.flags)
        s1 = k.Simulation(c, P[i], V[i])
        k.kmc_step(s1.h, args.warmup, 1)
        torch.cuda.synchronize()
        ms_plain += timed(s1.h, steps)
        s1.close()
    ms_batched, ms_plain = max_over_ranks([ms_batched, ms_plain], world, "cuda")
    value = job_rate(n_total, world, steps, ms_batched * 1e-3)
    plain = job_rate(n_total, world, steps, ms_plain * 1e-3)
    med = np.median(l1, axis=0) if len(l1) else [None] * 3
    return {"workload": f"sod1d_batched_{n_inst}", "instances": n_inst, "n_particles": n_total,
            "n_range": list(w["n_range"]), "lambda_range": list(w["lam_range"]),
            "n_cells_per_instance": list(w["n_cells"]), "dt": w["dt"], "steps": steps,
            "autotuned": {"occupancy_target": tuned.occupancy_target, "flags": tuned.flags,
                          "ms_per_step_in_tuning": round(tuned_ms, 3)},
            "batched": value, "plain_sequential": plain, "speedup": value / plain, "unit": UNIT,
            "ms_per_step_batched": ms_batched / steps, "ms_per_step_plain": ms_plain / steps,
            "gpu_launches_batched": launches_of(info, steps),
            "l1_error": {"at_t": max(t_steps, done) * w["dt"], "instances_lambda_le_1e-3": int(len(l1)),
                         "median_n_p_T": [round(float(x), 4) for x in med],
                         "max_n_p_T": [round(float(x), 4) for x in l1.max(0)] if len(l1) else None,
                         "same_for_plain": "per-instance states and moments bit-identical (tested)"}}


def batched_line(args):
    import torch
    import paper_1210_8084_gb300 as k
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local)
    clocks.start()
    b = batched_vs_plain(k, args, stream, rank, world, args.instances or None)
    clk = clocks.stop()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": b["batched"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step_batched"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "instances": b["instances"], "n_particles": b["n_particles"],
                       "l2": "no flush: state %.1f GB > 129 MB L2" % (b["n_particles"] * 64 / 1e9)},
            "batched_vs_plain": b, "gpu_launches": b["gpu_launches_batched"], "clocks": clk}


def oracle_slice(w, nbx, seed=0):
    """A bounded slice of the workload at full density: nbx c-bins in x
    around the split and, for 3-D c-bin grids, 8 x 8 c-bins in y and z
    (periodic, same c-bin widths), so every particle has the same number of
    candidates as in the full run (the slice's x ends are walls).  Returns
    (pos, vel, lo, hi, n_cells)."""
    from paper_1210_8084_gb300 import inputs
    n, nc = w["n"], w["n_cells"]
    L = [w["hi"][d] - w["lo"][d] for d in range(3)]
    dx = L[0] / nc[0]
    half = nbx // 2
    lo = [0.5 - half * dx, w["lo"][1], w["lo"][2]]
    hi = [0.5 + half * dx, w["hi"][1], w["hi"][2]]
    cells = [nbx, 1, 1]
    for d in (1, 2):
        if nc[d] > 8:
            hi[d] = lo[d] + 8 * L[d] / nc[d]
            cells[d] = 8
    # particles of the full tube that fall in the slice (left density 8/9 of N over half the box)
    V_half = 0.5 * L[0] * L[1] * L[2]
    dens_l = n * 8 / 9 / V_half
    dens_r = n / 9 / V_half
    area = (hi[1] - lo[1]) * (hi[2] - lo[2])
    n_sl = int(round(dens_l * half * dx * area))
    n_sr = int(round(dens_r * half * dx * area))
    pl, vl = inputs.sod_tube(2 * n_sl, seed, lo=lo, hi=hi, rho=(1.0, 1.0), p=(1.0, 1.0))
    pr, vr = inputs.sod_tube(2 * n_sr, seed + 1, lo=lo, hi=hi, rho=(1.0, 1.0), p=(0.8, 0.8))
    pos = np.concatenate([pl[pl[:, 0] < 0.5][:n_sl], pr[pr[:, 0] >= 0.5][:n_sr]])
    vel = np.concatenate([vl[pl[:, 0] < 0.5][:n_sl], vr[pr[:, 0] >= 0.5][:n_sr]])
    if w["precision"] == 32:
        pos, vel = inputs.cast_state(pos, vel, np.float32, lo, hi, w["bc"])
    return pos.astype(np.float64), vel.astype(np.float64), tuple(lo), tuple(hi), tuple(cells)


def cpu_baseline(w, n_bins_slice=8, steps=1, single_thread_bins=0, device_check=False):
    """The CPU oracle on the host cores (all OpenMP threads) on a slice of
    central c-bins at full density; optionally also on one thread.  With
    device_check, the binary32 device path steps the same slice from the same
    state, and the total energies after the step are compared (the FP32 drift
    against the binary64 oracle)."""
    import oracle
    R2 = oracle.contact_R2(w["lam"], 0.0, nbar_of(w))

    def run(nb):
        pos, vel, lo, hi, cells = oracle_slice(w, nb)
        P = oracle.make_params(w["dim_pos"], cells, lo, hi, w["bc"], R2=R2, dt=w["dt"], seed=0,
                               decide32=w["precision"] == 32)
        p, v = pos, vel
        t0 = time.perf_counter()
        for s in range(steps):
            P.step = s
            p, v = oracle.step(P, p, v)[:2]
        return pos, vel, p, v, time.perf_counter() - t0, lo, hi, cells

    cores = oracle.set_threads(0)
    pos, vel, p1, v1, el, lo, hi, cells = run(n_bins_slice)
    m = pos.shape[0]
    out = {"value": m * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle", "particles": m,
           "sample": f"{steps} oracle step(s) of the {n_bins_slice} central x c-bins"
                     f"{' x %d x %d c-bins in y, z' % (cells[1], cells[2]) if cells[1] > 1 else ''} at full "
                     f"density: {m} particles with the full run's neighbourhood occupancy, {el:.2f} s"}
    if single_thread_bins > 0:
        oracle.set_threads(1)
        try:
            pos1, _, _, _, el1, _, _, _ = run(single_thread_bins)
            m1 = pos1.shape[0]
        finally:
            oracle.set_threads(cores)
        out["single_thread"] = {"value": m1 * steps / el1, "unit": UNIT, "cores": 1, "particles": m1,
                                "sample": f"{steps} oracle step(s) of the {single_thread_bins} central x c-bins, "
                                          f"{el1:.2f} s"}
    drift = None
    if device_check:
        import paper_1210_8084_gb300 as k
        dtype = np.float32 if w["precision"] == 32 else np.float64
        cfg = k.make_config(dim_pos=w["dim_pos"], n_cells=cells, lo=lo, hi=hi, bc=w["bc"], sigma=np.pi * R2,
                            dt=w["dt"], seed=0, precision=w["precision"])
        sim = k.Simulation(cfg, pos.astype(dtype), vel.astype(dtype))
        e0 = sim.moments()[2][0, 1]
        sim.step(steps, want_moments=1)
        e_dev = sim.moments()[2][0, 1]
        sim.close()
        e_orc = 0.5 * float((v1 * v1).sum())
        e_in = 0.5 * float((vel * vel).sum())
        drift = {"steps": steps, "particles": m, "e_initial": e_in, "e_device": float(e_dev), "e_oracle": e_orc,
                 "device_vs_oracle_rel": (float(e_dev) - e_orc) / e_orc,
                 "device_drift_rel": (float(e_dev) - float(e0)) / float(e0),
                 "oracle_drift_rel": (e_orc - e_in) / e_in,
                 "sample": "the cpu_baseline slice, stepped by the binary32 device path and the binary64 oracle"}
    return out, drift


def slice_bins(w, asked):
    """x c-bins of the oracle's slice: 8 for slab c-bins (8 x about 8,000
    particles), 16 for 3-D c-bin grids (16 x 8 x 8 c-bins); `asked` > 0
    overrides."""
    if asked > 0:
        return asked
    return 16 if w["dim_pos"] == 3 and w["n_cells"][1] > 1 else 8


def reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    w = make_workload(args.workload, args.lam, args.n)
    samples = []
    for s in range(args.warmup + args.steps):
        r, _ = cpu_baseline(w, slice_bins(w, args.ref_slice_bins))
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
        "config": {"workload": f"{args.workload} lambda={w['lam']:g}", "n_particles": w["n"],
                   "n_cells": list(w["n_cells"]), "sample_x_bins": slice_bins(w, args.ref_slice_bins)},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--lam", type=float, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--occ", type=float, default=0.0, help="particles per search cell (0: library default)")
    ap.add_argument("--instances", type=int, default=0, help="batched workload: number of instances")
    ap.add_argument("--tile-threads", type=int, default=0, help="tile search threads per c-bin block (0: default)")
    ap.add_argument("--tile-cap", type=int, default=0, help="tile search staging capacity (0: default)")
    ap.add_argument("--tile-split", type=int, default=0, help="tile search blocks per c-bin (0: default)")
    ap.add_argument("--no-prune", action="store_true", help="binary32 tile search without cluster pruning")
    ap.add_argument("--flags", type=int, default=0, help="extra KMC_FLAG_* bits of the timed handle")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--cpu-slice-bins", type=int, default=0, help="x c-bins of the oracle slice (0: per workload)")
    ap.add_argument("--ref-slice-bins", type=int, default=0, help="x c-bins of the reference arm's slice (0: same)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        out = reference(args)
    elif args.workload.startswith("sod1d_batched"):
        out = batched_line(args)
    else:
        out = ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
