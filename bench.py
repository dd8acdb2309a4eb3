#!/usr/bin/env python
"""Benchmark of the skip-BF (l,d) motif search on GB300.

One step = the whole hot path over one synthetic workload: window extraction and packing (K0),
the pass-structured search with survivor compaction (K1 steps) and sort/dedup (K2).  The
default workload is the challenge-shaped (15,4) instance: n = 20 sequences of t = 600 bases,
uniform ACGT, one FM-planted instance per sequence (seed 2), all 4^15 candidates.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value   = candidates/s over the whole job (all ranks), inputs resident in HBM, per-step CUDA
          events on the plan's stream, L2 flushed (256 MiB write) before every step outside the
          timed intervals.
e2e     = the same metric through the blocking C-ABI call with host buffers (H2D of the
          characters, D2H of the codes inside the timed region).
roofline= the step kernel against its POPC issue bound (one POPC per canonical unit step).
cpu_baseline / --impl reference = the CPU oracle (C, POSIX threads over all host cores, the
          paper's index-range split) on a bounded sub-range of the same workload.
Multi-GPU (torchrun, --parallelism range, the default): the ranks split the candidate index
space of the one workload into contiguous ranges (Sec. IV.A's per-worker first/last index, by
motif_shard_range); every step each rank searches its range and the accepted codes are
all-gathered over NCCL (counts, then codes padded to the largest count) inside the timed region;
strong scaling, max time over ranks, and the gathered result is checked against the whole-space
search.  --parallelism replicas: every rank searches its own independently seeded instance (weak
scaling, no collective on the data path).
cpu_baseline_1t = the oracle on one thread over a stated sub-range, extrapolated to the whole
          space (the paper's sequential baseline).
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(15,4) candidates/s & window-compares/s vs INT/POPC roofline; serve p50/p99"
CONFIGS = {  # name: (l, d, n, t, seed)
    "l9d2": (9, 2, 20, 600, 1),
    "l15d4": (15, 4, 20, 600, 2),
    "l17d5": (17, 5, 20, 600, 3),
    "l11d4": (11, 4, 28, 859, 7),  # dense: most codes survive (bitmap output, split tiled pass)
}
POPC_PER_SM_CLK = 16.0  # measured by the K4 probe (motif_probe_rate POPC) on GB300
LOP3_PER_SM_CLK = 64.0  # measured by the K4 probe (motif_probe_rate LOP3) on GB300
# Issue slots: each of an SM's 4 sub-partitions issues one warp instruction per clock (the IADD3
# and IMNMX probes reach 128 lanes/clk/SM = 4 warp instructions).
ISSUE_PER_SM_CLK = 4.0
# ncu figures of one launch of the whole-tile tiled pass (tiled_kernel) per workload, from one
# `ncu --set full --clock-control none -k regex:tiled_kernel -c 1` capture of the current kernel
# (MOTIF_NO_GRAPH=1 so that ncu lists it): smsp__inst_executed.sum (warp instructions), DRAM
# bytes read + written, smsp__issue_active and the ALU pipe's share.  Null entries: not captured.
TILED_NCU = {
    "l15d4_n20_t600_seed2": {"inst": 369165171, "dram_bytes": 261888, "issue_active": 0.589,
                             "alu_pipe": 0.633,
                             # sm__inst_executed_pipe_{alu,fma,xu}.sum of the same launch
                             "pipe_inst": {"alu": 200137273, "fma": 59174350, "xu": 18536243}},
    "l17d5_n20_t600_seed3": {"inst": 5007448973, "dram_bytes": 303872, "issue_active": 0.628,
                             "alu_pipe": 0.614,
                             "pipe_inst": {"alu": 2472283262, "fma": 785496564, "xu": 188309451}},
}
# Warp instructions per clock per SM of the pipes the tiled pass loads most, from the K4 probes:
# the ALU pipe (LOP3, 64 lanes/clk), the FMA pipe (IMAD, 64 lanes/clk) and the XU pipe (POPC,
# 16 lanes/clk).  With the pass's per-pipe instruction counts (ncu sm__inst_executed_pipe_*.sum)
# the issue peak for its mix is min(4, rate_p / share_p) over these pipes.
PIPE_PER_SM_CLK = {"alu": 2.0, "fma": 2.0, "xu": 0.5}




@contextlib.contextmanager
def quiet_gc():
    """A host-timed region without the interpreter's cyclic garbage collector: the client's
    objects (results, stats dicts) would otherwise trigger collections that walk every result
    kept so far, pauses of tens of milliseconds that belong to this script, not the library."""
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="l15d4")
    ap.add_argument("--kernel", choices=["auto", "tiled", "group", "cand", "bitslice"],
                    default="auto")
    ap.add_argument("--suffix-bases", type=int, default=0)
    ap.add_argument("--cands-per-thread", type=int, default=0)
    ap.add_argument("--seed", choices=["all", "neighbourhood"], default="all",
                    help="candidates searched: all indices, or (CAND/BITSLICE) only those within d "
                         "of a window of the first sequence")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cand-subrange", type=int, default=1 << 27,
                    help="candidates of the roofline_cand sub-range run (0 = skip)")
    ap.add_argument("--mode", choices=["single", "batch", "serve", "cpu-scaling"], default="single",
                    help="single: one (l,d) search workload, the JSON line; batch: 64 uneven "
                         "jobs batched vs one job per launch; serve: Poisson arrivals, p50/p99 latency per rate")
    ap.add_argument("--rates", default="1,2,5,10,20,50,100,200")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--parallelism", choices=["range", "replicas"], default="range",
                    help="N > 1: split one workload's candidate range over the ranks and gather "
                         "the codes (strong scaling), or one independent instance per rank (weak)")
    ap.add_argument("--cpu-1t-seconds", type=float, default=8.0,
                    help="single-thread oracle sample for cpu_baseline_1t (0 = skip)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch mode: leave the plans on their AUTO choices")
    ap.add_argument("--tune-ms", type=int, default=400,
                    help="batch mode: motif_autotune's time budget per job")
    ap.add_argument("--serve-max-active", type=int, default=128,
                    help="serve mode: jobs resident in the server's table")
    ap.add_argument("--serve-submit", choices=["seqs", "plan"], default="seqs",
                    help="serve mode: submit jobs straight from their rows (motif_submit_seqs) "
                         "or through a plan (create, load, motif_submit, destroy)")
    ap.add_argument("--saturation-only", action="store_true",
                    help="serve mode: only the saturation comparison with the plain path")
    ap.add_argument("--serve-step-tiles", type=int, default=0,
                    help="serve mode: tile budget of one server step over all warps (0 = default)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu() -> dict:
    """The host's processor: model name (from /proc/cpuinfo where it has one) and ISA."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:  # Arm kernels list no model name there; lscpu names the core
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name:"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"cpu_model": model, "isa": platform.machine()}


def cpu_baseline(job, seconds: float, steps: int = 1):
    """Times the oracle (all host cores, the paper's range split) on a bounded sub-range."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    l = job.l
    lo = (4 ** l) // 3
    probe = 1 << 12
    t0 = time.perf_counter()
    oracle.search(job.rows(), l, job.d, lo=lo, hi=lo + probe, threads=cores)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    size = int(min(4 ** l - lo, max(probe, rate * seconds / max(steps, 1))))
    times = []
    for s in range(steps):
        a = lo + s * size
        b = min(4 ** l, a + size)
        t0 = time.perf_counter()
        oracle.search(job.rows(), l, job.d, lo=a, hi=b, threads=cores)
        times.append(time.perf_counter() - t0)
    return size, times, cores, lo


def cpu_baseline_1t(job, seconds: float) -> dict:
    """The oracle on ONE thread (the paper's sequential baseline, Sec. V) over a sub-range sized
    for about `seconds` of work, extrapolated to the whole candidate space."""
    from oracle import oracle
    l = job.l
    lo = (4 ** l) // 3
    probe = 1 << 10
    t0 = time.perf_counter()
    oracle.search(job.rows(), l, job.d, lo=lo, hi=lo + probe, threads=1)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    size = int(min(4 ** l - lo, max(probe, rate * seconds)))
    t0 = time.perf_counter()
    oracle.search(job.rows(), l, job.d, lo=lo, hi=lo + size, threads=1)
    dt = time.perf_counter() - t0
    rate = size / dt
    return dict({"value": rate, "unit": "candidates/s", "cores": 1, "kind": "oracle",
                 "sample": "candidates [%d, %d), %.1f s on one thread" % (lo, lo + size, dt),
                 "full_search_s": 4 ** l / rate,
                 "full_search_s_basis": "extrapolated: 4^%d candidates / the sample's rate" % l},
                **host_cpu())


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from paper_1403_1313_gb300 import fmgen
    l, d, n, t, seed = CONFIGS[args.config]
    job = fmgen.fm_job(n, t, l, d, seed)
    # Warm-up steps, then K timed steps; each step is one bounded sub-range of the workload.
    per_step = max(0.05, min(2.0, 60.0 / max(args.steps + args.warmup, 1)))
    size, times, cores, lo = cpu_baseline(job, per_step * (args.steps + args.warmup),
                                          steps=args.steps + args.warmup)
    timed = times[args.warmup:]
    value = size * len(timed) / sum(timed)
    sample = "candidates [%d, %d) of the (%d,%d) n=%d t=%d seed-%d workload, %d per step" % (
        lo, lo + size * len(times), l, d, n, t, seed, size)
    line = {
        "metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(timed) / len(timed),
        "higher_is_better": True,
        "scaling": "strong" if args.parallelism == "range" else "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "impl": "reference",
        "config": {"workload": "l%dd%d_n%d_t%d_seed%d" % (l, d, n, t, seed), "l": l, "d": d,
                   "n": n, "t": t, "seed": seed, "sample_candidates_per_step": size},
        "cpu_baseline": dict({"value": value, "unit": "candidates/s", "cores": cores,
                              "kind": "oracle", "sample": sample}, **host_cpu()),
        "e2e": {"value": value, "unit": "candidates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import paper_1403_1313_gb300 as m
    from paper_1403_1313_gb300 import fmgen

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    l, d, n, t, seed = CONFIGS[args.config]
    shard = world > 1 and args.parallelism == "range"
    job = fmgen.fm_job(n, t, l, d, seed + (0 if shard or world == 1 else rank * 1000))
    workload = "l%dd%d_n%d_t%d_seed%d" % (l, d, n, t, seed)
    cands = 4 ** l
    # This rank's contiguous share of the candidate space (the whole space at N = 1), in whole
    # 65,536-candidate tiles where there are enough of them (each rank's plan then runs the
    # tiled pass, whose tiles must start on that boundary).
    from paper_1403_1313_gb300.shard import rank_range
    r_lo, r_hi = rank_range(cands, rank, world) if shard else (0, cands)

    stream = torch.cuda.Stream()
    kw = {}
    if args.kernel == "group":
        kw["kernel"] = m.KERNEL_GROUP
    elif args.kernel == "cand":
        kw["kernel"] = m.KERNEL_CAND
    elif args.kernel == "tiled":
        kw["kernel"] = m.KERNEL_TILED
    elif args.kernel == "bitslice":
        kw["kernel"] = m.KERNEL_BITSLICE
    if args.suffix_bases:
        kw["suffix_bases"] = args.suffix_bases
    if args.seed == "neighbourhood":
        kw["seed"] = m.SEED_NEIGHBOURHOOD
    if args.cands_per_thread:
        kw["cands_per_thread"] = args.cands_per_thread
    rkw = dict(kw, range_lo=r_lo, range_hi=r_hi) if shard else dict(kw)
    opts = m.torch_opts(stream=stream, **rkw)
    plan = m.motif_plan_create(n, t, l, d, opts)
    cap = 1 << 16
    with torch.cuda.stream(stream):
        d_chars = torch.from_numpy(job.seqs.copy()).cuda()
        d_out = torch.zeros(cap, dtype=torch.int64, device="cuda")
        d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    if shard:
        from paper_1403_1313_gb300.shard import gather_codes_device

    def step():
        m.motif_load_seqs_device(plan, d_chars)
        m.motif_search_device(plan, d_out, cap, d_cnt)
        if shard:  # the variable-size gather of every rank's codes (counts, then codes)
            return gather_codes_device(d_out, d_cnt)
        return None

    with torch.cuda.stream(stream):  # the gather's collectives follow the search on its stream
        for _ in range(max(args.warmup, 3)):
            step()
    stream.synchronize()
    count = int(d_cnt.item())
    if shard:  # every rank needs room for its own codes
        cnt_all = torch.tensor([count], dtype=torch.int64, device="cuda")
        dist.all_reduce(cnt_all, op=dist.ReduceOp.MAX)
        count_max = int(cnt_all.item())
    else:
        count_max = count
    if count_max > cap:  # a dense result: room for every code, then warm up again
        cap = count_max
        with torch.cuda.stream(stream):
            d_out = torch.zeros(cap, dtype=torch.int64, device="cuda")
            for _ in range(max(args.warmup, 3)):
                step()
        stream.synchronize()
        count = int(d_cnt.item())
    if shard:
        # The gathered result of one step against the whole-space search of this GPU.
        with torch.cuda.stream(stream):
            gathered = step()
        stream.synchronize()
        codes = gathered.cpu().numpy().astype(np.uint64)
        whole = m.motif_plan_create(n, t, l, d, m.torch_opts(stream=stream, **kw))
        m.motif_load_seqs(whole, np.ascontiguousarray(job.seqs))
        ref = m.motif_search(whole)
        m.motif_plan_destroy(whole)
        assert np.array_equal(codes, ref), "gathered result != whole-space search"
    else:
        codes = d_out[:max(count, 0)].cpu().numpy().astype(np.uint64)
    assert codes.size >= 1 and m.motif_encode(job.consensus) in set(codes.tolist()), \
        "result check failed"
    compares, unit_steps = m.motif_count_work(plan)
    st_k = m.motif_stats(plan)
    tiled_units = None
    if st_k["kernel"] == m.KERNEL_TILED:
        try:
            tiled_units = m.motif_count_tiled_work(plan)  # the tiled pass's own work units
        except m.MotifError:  # split into sequence blocks: no whole-tile counts
            tiled_units = None
    if shard:  # the whole job's canonical tally: every rank's range
        cmp_all = torch.tensor([compares, unit_steps], dtype=torch.int64, device="cuda")
        dist.all_reduce(cmp_all)
        compares, unit_steps = (int(x) for x in cmp_all.tolist())
    m.motif_stats(plan)  # resets the summed device times
    st0 = m.motif_stats(plan)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)  # let the sampler come up before the timed region
    launches0 = m.motif_kernel_launches()
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev_s[k].record(stream)
            step()
            ev_e[k].record(stream)
    stream.synchronize()
    clocks = sampler.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in zip(ev_s, ev_e))
    st = m.motif_stats(plan)  # also accounts the step launches run inside the graphs
    launches = m.motif_kernel_launches() - launches0
    if world > 1:
        tt = torch.tensor([t_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        dist.barrier()

    jobs_per_step = 1 if shard else world  # one shared workload, or one instance per rank
    value = jobs_per_step * cands * args.steps / (t_ms / 1e3)
    cps = (1 if shard else world) * compares * args.steps / (t_ms / 1e3)

    # Roofline of the dominant kernel (the step kernel; its launches are bracketed by the plan's
    # events: search_ms_sum over the timed searches), by the per-compare recipe: one algorithmic
    # window compare (the oracle's canonical tally) costs one POPC, so peak = 16 POPC/clk/SM x
    # SMs x max SM clock.  A kernel that factors the compare (GROUP, TILED) resolves many
    # compares per POPC and reads above 1.0 here; the per-candidate kernel (CAND), which pays
    # the full per-compare cost, is timed on a sub-range below as roofline_cand.
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    step_ms = st["search_ms_sum"] / max(st["searches"], 1)
    sort_ms = st["sort_ms_sum"] / max(st["searches"], 1)
    peak = POPC_PER_SM_CLK * sms * max_mhz * 1e6
    kname = {m.KERNEL_GROUP: "GROUP", m.KERNEL_CAND: "CAND", m.KERNEL_TILED: "TILED",
             m.KERNEL_BITSLICE: "BITSLICE"}.get(st["kernel"], "?")
    achieved = compares / (step_ms / 1e3)
    # DRAM traffic per launch of the timed kernel, from an ncu capture of the tiled pass on the
    # default workload (dram__bytes_read.sum + dram__bytes_write.sum of its first step launch);
    # other kernels and workloads were not captured: null.
    traffic = None
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "G window-compares/s (1 POPC each)", "frac": achieved / peak,
            "traffic": traffic,
            "kernel": "step_kernel<%s>" % kname,
            "peak_basis": "16 POPC/clk/SM (K4 probe) x %d SMs x %.0f MHz (max SM clock)" % (sms, max_mhz),
            "step_kernel_ms": step_ms, "sort_ms": sort_ms,
            "algorithmic_compares_per_search": compares,
            "group_prefix_compares_per_search": unit_steps,
            "note": ("frac > 1: the %s kernel factors the Hamming distance over shared candidate "
                     "prefixes, so one POPC or bit test resolves many algorithmic compares; see "
                     "roofline_cand for the per-compare kernel" % kname) if kname != "CAND" else ""}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / (POPC_PER_SM_CLK * sms * clocks["sm_mhz"] * 1e6)
    if kname == "TILED" and tiled_units and not shard:
        # The tiled pass's own roofline: it is bound by instruction issue (integer ALU work,
        # shuffles, shared loads; DRAM traffic is the packed windows once).  achieved = its
        # unit count (tile-sequence visits, counted live by motif_count_tiled_work) x warp
        # instructions per visit (ncu's smsp__inst_executed of one launch / the same visits)
        # / the kernel's event-timed device time; peak = 4 issue slots per SM per clock.
        ncu = TILED_NCU.get(workload, {}) if args.seed == "all" else {}
        peak_i = ISSUE_PER_SM_CLK * sms * max_mhz * 1e6
        per_compare = dict(roof)
        per_compare["note"] = ("the per-compare recipe (one POPC per algorithmic compare): the "
                               "tiled pass resolves a window for a whole tile per filter POPC, "
                               "so this ratio is not a roofline fraction")
        ipv = ncu["inst"] / tiled_units["visits"] if ncu.get("inst") else None
        ach_i = tiled_units["visits"] * ipv / (step_ms / 1e3) if ipv else None
        per_clk, basis = ISSUE_PER_SM_CLK, "4 warp instructions issued per clock per SM (IADD3 probe: 128 lanes/clk/SM)"
        pipes = ncu.get("pipe_inst")
        if pipes and ncu.get("inst"):
            # the instruction mix's own issue peak: the busiest pipe's rate over its share
            lim = {p: PIPE_PER_SM_CLK[p] * ncu["inst"] / pipes[p] for p in PIPE_PER_SM_CLK
                   if pipes.get(p)}
            bind = min(lim, key=lim.get)
            if lim[bind] < per_clk:
                per_clk = lim[bind]
                basis = ("this mix's issue peak: the %s pipe (%.1f warp instructions/clk/SM, K4) "
                         "carries %.1f %% of the pass's instructions, so at most %.2f issue per "
                         "clock per SM" % (bind.upper(), PIPE_PER_SM_CLK[bind],
                                           100.0 * pipes[bind] / ncu["inst"], lim[bind]))
        peak_i = per_clk * sms * max_mhz * 1e6
        roof = {"bound": "alu", "kernel": "tiled_kernel (whole-tile prefix-tiled pass)",
                "bound_detail": "plain integer ALU work, measured against the SM's instruction "
                                "issue rate for this kernel's own mix (per-pipe rates from the "
                                "K4 probes, pipe shares from ncu)",
                "unit": "G warp-instructions/s",
                "achieved": ach_i / 1e9 if ach_i else None, "peak": peak_i / 1e9,
                "frac": ach_i / peak_i if ach_i else None,
                "frac_of_issue_slots": ach_i / (ISSUE_PER_SM_CLK * sms * max_mhz * 1e6)
                                       if ach_i else None,
                "traffic": ncu.get("dram_bytes"),
                "peak_basis": "%s x %d SMs x %.0f MHz (max SM clock)" % (basis, sms, max_mhz),
                "units_per_search": tiled_units, "warp_instructions_per_visit": ipv,
                "warp_instructions_per_search": ncu.get("inst"),
                "ncu": {k: ncu.get(k) for k in ("issue_active", "alu_pipe")},
                "step_kernel_ms": step_ms, "sort_ms": sort_ms,
                "per_compare_popc": per_compare}
        if ach_i and clocks and clocks.get("sm_mhz"):
            roof["frac_at_observed_clock"] = ach_i / (per_clk * sms * clocks["sm_mhz"] * 1e6)
    def per_candidate_leg(kernel, label, cpt):
        """A per-candidate kernel on a sub-range of the same workload (full per-compare work)."""
        o = m.torch_opts(stream=stream, kernel=kernel, cands_per_thread=cpt,
                         range_lo=0, range_hi=min(cands, args.cand_subrange))
        pc = m.motif_plan_create(n, t, l, d, o)
        with torch.cuda.stream(stream):
            m.motif_load_seqs_device(pc, d_chars)
            for _ in range(2):
                m.motif_search_device(pc, d_out, cap, d_cnt)
        stream.synchronize()
        c_cmp = m.motif_count_compares(pc)
        m.motif_stats(pc)
        with torch.cuda.stream(stream):
            for _ in range(5):
                m.motif_search_device(pc, d_out, cap, d_cnt)
        stc = m.motif_stats(pc)
        m.motif_plan_destroy(pc)
        c_ms = stc["search_ms_sum"] / max(stc["searches"], 1)
        c_ach = c_cmp / (c_ms / 1e3)
        return {"bound": "alu", "achieved": c_ach / 1e9, "peak": peak / 1e9,
                "unit": "G window-compares/s (1 POPC each)", "frac": c_ach / peak,
                "kernel": "step_kernel<%s,%d>" % (label, cpt), "step_kernel_ms": c_ms,
                "sample": "candidates [0, %d) of %s" % (min(cands, args.cand_subrange), workload)}

    roof_cand = roof_bitslice = None
    if rank != 0:  # the per-candidate legs are rank 0's alone
        args.cand_subrange = 0
    if kname != "CAND" and args.cand_subrange > 0:
        roof_cand = per_candidate_leg(m.KERNEL_CAND, "CAND", 2)
    if args.cand_subrange > 0 and d <= 7:
        # The bit-sliced compare against both rooflines: the POPC one above and its own, the
        # LOP3 pipe at the counter's LOP3 per 32 compares (11 per three base positions, 5 per
        # position left over; positions past 16 are counted as a second group).
        roof_bitslice = per_candidate_leg(m.KERNEL_BITSLICE, "BITSLICE", 1)
        def counter_lop3(k):  # 15 per 7 positions, 11 per 3, 5 per 1
            return 15 * (k // 7) + 11 * ((k % 7) // 3) + 5 * ((k % 7) % 3)
        lop3 = sum(counter_lop3(k) for k in (max(0, l - 16), min(l, 16)))
        peak_lop3 = LOP3_PER_SM_CLK * sms * max_mhz * 1e6 * 32.0 / lop3
        roof_bitslice.update({
            "peak_lop3": peak_lop3 / 1e9, "frac_lop3": roof_bitslice["achieved"] * 1e9 / peak_lop3,
            "peak_lop3_basis": "64 LOP3/clk/SM (K4 probe) x %d SMs x %.0f MHz x 32 / %d LOP3 "
                               "per 32 compares" % (sms, max_mhz, lop3)})

    # End to end through the blocking C ABI with host buffers (each rank its own range, and the
    # ranks' host codes gathered, in range-shard mode).
    plan2 = m.motif_plan_create(n, t, l, d, m.torch_opts(stream=stream, **rkw))
    host_chars = np.ascontiguousarray(job.seqs)
    m.motif_load_seqs(plan2, host_chars)
    m.motif_search(plan2)
    ne = max(3, args.e2e_steps)
    torch.cuda.synchronize()
    if world > 1:
        from paper_1403_1313_gb300.shard import gather_codes
        dist.barrier()
    with quiet_gc():
        t0 = time.perf_counter()
        for _ in range(ne):
            m.motif_load_seqs(plan2, host_chars)
            got = m.motif_search(plan2)
            d2h = 8 * got.size + 8
            if shard:
                got = gather_codes(got)
        dt = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
    e2e = {"value": jobs_per_step * cands * ne / dt, "unit": "candidates/s",
           "h2d_bytes_per_step": int(n * t), "d2h_bytes_per_step": int(d2h)}
    if shard:
        e2e["note"] = "per rank: its range's codes to the host, then a host-buffer gather"
    m.motif_plan_destroy(plan2)

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True,
            "scaling": "strong" if args.parallelism == "range" else "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload, "l": l, "d": d, "n": n, "t": t, "seed": seed,
                       "candidates": cands, "kernel": roof["kernel"],
                       "candidate_seeding": args.seed,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": ("range shard: %d GPUs, contiguous candidate ranges "
                                       "(motif_shard_range), NCCL gather of the codes inside the "
                                       "timed region" % world) if shard else
                                      ("weak: one independent instance per GPU" if world > 1
                                       else "1 GPU")},
            "window_compares_per_s": cps,
            "algorithmic_compares_per_search": compares,
            "survivors": int(codes.size),
            "roofline": roof,
            "roofline_cand": roof_cand,
            "roofline_bitslice": roof_bitslice,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            size, times, cores, lo = cpu_baseline(job, args.cpu_seconds)
            line["cpu_baseline"] = dict({
                "value": size / times[0], "unit": "candidates/s", "cores": cores, "kind": "oracle",
                "sample": "candidates [%d, %d) of %s (%.1f s wall, all %d cores)" % (
                    lo, lo + size, workload, times[0], cores)}, **host_cpu())
            if args.cpu_1t_seconds > 0:
                line["cpu_baseline_1t"] = cpu_baseline_1t(job, args.cpu_1t_seconds)
        print(json.dumps(line), flush=True)
    m.motif_plan_destroy(plan)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """64 uneven jobs (seed 4): one batched launch sequence vs one job per launch."""
    import numpy as np
    import torch
    import paper_1403_1313_gb300 as m
    from paper_1403_1313_gb300 import fmgen

    torch.cuda.set_device(0)
    jobs = fmgen.batched_jobs(seed=4, count=64)
    out = {}
    runs = [("all_64", lambda j: True, True), ("small_l_le_12", lambda j: j.l <= 12, True)]
    if not args.no_autotune:
        # the AUTO choices too, for comparison, first: the autotuner's choices go to a
        # process-wide cache that later AUTO plans of the same shape would pick up
        runs.insert(0, ("all_64_auto", lambda j: True, False))
    tuned_choice = {}
    for label, sel, tune in runs:
        js = [j for j in jobs if sel(j)]
        plans = []
        t_tune = time.perf_counter()
        for j in js:
            pl = m.motif_plan_create(j.n, j.t, j.l, j.d)
            m.motif_load_seqs(pl, j.seqs)
            if tune and not args.no_autotune:
                # the autotuner times the kernel forms on a sub-range of this job's candidates and
                # keeps the fastest in the plan (and its cache, keyed by the job's shape)
                best = m.motif_autotune(pl, budget_ms=args.tune_ms)
                tuned_choice[(j.l, j.d, j.n, j.t)] = (best.kernel, best.cands_per_thread,
                                                      best.suffix_bases, best.compact_levels)
            plans.append(pl)
        t_tune = time.perf_counter() - t_tune
        compares = sum(m.motif_count_compares(pl) for pl in plans)
        cands = sum(4 ** j.l for j in js)
        plain_res = [m.motif_search(pl) for pl in plans]          # warm-up + reference result
        batch_res = m.motif_batch_search(plans, use_graph=True)
        assert all(np.array_equal(a, b) for a, b in zip(plain_res, batch_res)), "batch != plain"
        reps = max(1, args.steps)
        for _ in range(max(3, args.warmup)):  # untimed: graphs, sort scratch, host buffer pools
            for pl in plans:
                m.motif_search(pl)
            m.motif_batch_search(plans, use_graph=True)
            m.motif_batch_search(plans, use_graph=False)
        torch.cuda.synchronize()
        with quiet_gc():
            t0 = time.perf_counter()
            for _ in range(reps):
                for pl in plans:
                    m.motif_search(pl)
            t_plain = (time.perf_counter() - t0) / reps
        with quiet_gc():
            t0 = time.perf_counter()
            for _ in range(reps):
                m.motif_batch_search(plans, use_graph=True)
            t_batch = (time.perf_counter() - t0) / reps
        with quiet_gc():
            t0 = time.perf_counter()
            for _ in range(reps):
                m.motif_batch_search(plans, use_graph=False)
            t_batch_nograph = (time.perf_counter() - t0) / reps
        survivors = sum(int(r.size) for r in batch_res)
        # Per-job view of both paths (the slowest plain jobs, and the batch's phase split).
        per_job = []
        for j, pl, r in zip(js, plans, plain_res):
            t1 = time.perf_counter()
            m.motif_search(pl)
            dt = time.perf_counter() - t1
            stp = m.motif_stats(pl)
            # work items of its search: 65,536-candidate tiles (tiled pass), else 256-candidate
            # groups per 32 lanes; a job with at least a grid's worth keeps every SM busy alone
            items = (4 ** j.l + 65535) // 65536 if stp["kernel"] == m.KERNEL_TILED else 1 << 40
            per_job.append({"l": j.l, "d": j.d, "n": j.n, "t": j.t, "survivors": int(r.size),
                            "plain_ms": 1e3 * dt, "search_ms": stp["search_ms"],
                            "sort_ms": stp["sort_ms"], "fills_gpu": items >= stp["grid"]})
        # The jobs whose tiles cover the grid alone (they gain little from sharing the GPU)
        full_ms = sum(x["search_ms"] for x in per_job if x["fills_gpu"])
        per_job.sort(key=lambda x: -x["plain_ms"])
        phases = []  # the batch's device phase split: median over a few calls
        for _ in range(5):
            m.motif_batch_search(plans, use_graph=True)
            s0 = m.motif_stats(plans[0])
            phases.append((s0["search_ms"], s0["sort_ms"], s0["queue_ms"]))
        stb = dict(zip(("search_ms", "sort_ms", "queue_ms"),
                       (statistics.median(x) for x in zip(*phases))))
        out[label] = {
            "jobs": len(js), "candidates": cands, "algorithmic_compares": compares,
            "plans": ("autotuned (motif_autotune per job, %.1f s)" % t_tune
                      if tune and not args.no_autotune else "AUTO"),
            "survivors": survivors,
            "plain_ms": 1e3 * t_plain, "batched_ms": 1e3 * t_batch,
            "batched_nograph_ms": 1e3 * t_batch_nograph,
            "plain_jobs_per_s": len(js) / t_plain, "batched_jobs_per_s": len(js) / t_batch,
            "plain_compares_per_s": compares / t_plain, "batched_compares_per_s": compares / t_batch,
            "batched_over_plain": t_plain / t_batch,
            "jobs_filling_gpu": sum(1 for x in per_job if x["fills_gpu"]),
            "filling_jobs_search_ms": full_ms,
            # the ratio if the batch's sorts, copies and host work cost nothing: its step phase
            # (every job's tiles, run side by side) bounds it
            "ratio_bound_steps_only": 1e3 * t_plain / max(stb["search_ms"], 1e-9),
            "batch_device_steps_ms": stb["search_ms"], "batch_device_sort_ms": stb["sort_ms"],
            "batch_copy_to_host_ms": stb["queue_ms"],
            "plain_device_ms": sum(x["search_ms"] + x["sort_ms"] for x in per_job),
            "batched_over_plain_device": sum(x["search_ms"] + x["sort_ms"] for x in per_job)
                                          / max(stb["search_ms"] + stb["sort_ms"], 1e-9),
            "slowest_plain_jobs": per_job[:8],
        }
        for pl in plans:
            m.motif_plan_destroy(pl)
    kinds = {}
    for v in tuned_choice.values():
        kinds[str(v)] = kinds.get(str(v), 0) + 1
    print(json.dumps({"mode": "batch", "workload": "64 jobs, seed 4: l~U{9..15}, d~U{1..4}, "
                      "n~U{5..40}, t~U{200..1000}, FM-planted", "reps": max(1, args.steps),
                      "tuned_choices (kernel, cands_per_thread, suffix_bases, compact_levels)":
                          kinds, "results": out}), flush=True)
    return 0


def run_serve(args):
    """Poisson arrivals at each rate; latency = submit -> result ready, from the library."""
    import numpy as np
    import torch
    import paper_1403_1313_gb300 as m
    from paper_1403_1313_gb300 import fmgen

    torch.cuda.set_device(0)
    rows = []
    for rate in ([] if args.saturation_only else [float(r) for r in args.rates.split(",")]):
        count = int(min(args.serve_jobs, max(20, rate * args.serve_seconds)))
        jobs = fmgen.serving_jobs(rate, count, seed=5)
        m.motif_server_start(max_active=args.serve_max_active, step_tiles=args.serve_step_tiles)
        # warm-up job (graph capture, ball tables, allocator pools)
        wj = fmgen.fm_job(10, 300, 11, 3, 1)
        pl = m.motif_plan_create(wj.n, wj.t, wj.l, wj.d)
        m.motif_load_seqs(pl, wj.seqs)
        m.motif_poll(m.motif_submit(pl), timeout_ms=60000)
        m.motif_plan_destroy(pl)
        with quiet_gc():
            ids = []
            client = ({"submit": 0.0} if args.serve_submit == "seqs" else
                      {"create": 0.0, "load": 0.0, "submit": 0.0, "destroy": 0.0})
            t0 = time.perf_counter()
            for j in jobs:
                delay = t0 + j.arrival_s - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                c0 = time.perf_counter()
                if args.serve_submit == "seqs":
                    ids.append(m.motif_submit_seqs(j.seqs, j.l, j.d))
                    client["submit"] += time.perf_counter() - c0
                    continue
                pl = m.motif_plan_create(j.n, j.t, j.l, j.d)
                c1 = time.perf_counter()
                m.motif_load_seqs(pl, j.seqs)
                c2 = time.perf_counter()
                ids.append(m.motif_submit(pl))
                c3 = time.perf_counter()
                m.motif_plan_destroy(pl)
                c4 = time.perf_counter()
                client["create"] += c1 - c0
                client["load"] += c2 - c1
                client["submit"] += c3 - c2
                client["destroy"] += c4 - c3
            t_submitted = time.perf_counter() - t0
            lat, queue, cands, ok = [], [], 0, 0
            for j, jid in zip(jobs, ids):
                res = m.motif_poll(jid, timeout_ms=600000)
                codes, st = res
                lat.append(st["total_ms"])
                queue.append(st["queue_ms"])
                cands += 4 ** j.l
                c = m.motif_encode(j.consensus)
                pos = int(np.searchsorted(codes, np.uint64(c)))
                ok += int(pos < codes.size and int(codes[pos]) == c)
            wall = time.perf_counter() - t0
        m.motif_server_stop()
        lat = np.array(lat)
        rows.append({"rate_jobs_per_s": rate, "jobs": count, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                     "queue_p50_ms": float(np.percentile(queue, 50)),
                     "queue_p99_ms": float(np.percentile(queue, 99)),
                     "throughput_jobs_per_s": count / wall, "candidates_per_s": cands / wall,
                     "consensus_found": ok,
                     "client_ms_per_job": {k: 1e3 * v / count for k, v in client.items()},
                     "last_arrival_s": jobs[-1].arrival_s, "submitted_all_s": t_submitted,
                     "done_all_s": wall})
        print(json.dumps(rows[-1]), flush=True)
    # Saturation: the same jobs one after another through the blocking path (the plain one-job-
    # per-launch path: plan creation, load, search and release each), then all submitted to the
    # server at once.  Each arm runs the whole job list untimed first (allocator pools, graphs,
    # pinned blocks: once for the plain path, twice for a server), then timed: the plain path
    # once, the server three times (median).
    jobs = fmgen.serving_jobs(1000.0, args.serve_jobs, seed=5)

    def plain_pass():
        codes, dev = [], 0.0
        with quiet_gc():
            t0 = time.perf_counter()
            for j in jobs:
                pl = m.motif_plan_create(j.n, j.t, j.l, j.d)
                m.motif_load_seqs(pl, j.seqs)
                codes.append(m.motif_search(pl))
                stp = m.motif_stats(pl)
                dev += stp["search_ms"] + stp["sort_ms"]
                m.motif_plan_destroy(pl)
            dt = time.perf_counter() - t0
        return codes, dev, dt

    plain_pass()
    plain_codes, dev_ms, t_plain = plain_pass()

    def served_at_once(via, reps, warm=2):
        """Every job submitted at once (through `via`), then every result polled; `reps` timed
        passes after `warm` untimed ones on the same server (a new server's pinned pools fill
        during its first passes)."""
        m.motif_server_start(max_active=args.serve_max_active, step_tiles=args.serve_step_tiles)
        out = []
        for rep in range(reps + warm):
            with quiet_gc():
                t0 = time.perf_counter()
                ids = []
                for j in jobs:
                    if via == "seqs":
                        ids.append(m.motif_submit_seqs(j.seqs, j.l, j.d))
                        continue
                    pl = m.motif_plan_create(j.n, j.t, j.l, j.d)
                    m.motif_load_seqs(pl, j.seqs)
                    ids.append(m.motif_submit(pl))
                    m.motif_plan_destroy(pl)
                t_client = time.perf_counter() - t0
                served = [m.motif_poll(jid, timeout_ms=600000) for jid in ids]
                t_done = time.perf_counter() - t0
            if rep >= warm:
                out.append((t_done, t_client, served))
        m.motif_server_stop()
        out.sort(key=lambda x: x[0])
        return out[len(out) // 2], [x[0] for x in out]

    (t_served_plan, t_client_plan, served_plan), _ = served_at_once("plan", 1)
    (t_served, t_client, served), all_served = served_at_once(args.serve_submit, 3)
    same = all(np.array_equal(a, b[0]) and np.array_equal(a, c[0])
               for a, b, c in zip(plain_codes, served, served_plan))
    lat = np.array([b[1]["total_ms"] for b in served])
    sat = {"jobs": len(jobs), "submit": args.serve_submit, "max_active": args.serve_max_active,
           "plain_jobs_per_s": len(jobs) / t_plain,
           "served_jobs_per_s": len(jobs) / t_served,
           "served_over_plain": t_plain / t_served,
           "served_ms_all_reps": [1e3 * x for x in all_served],
           # the same jobs served through plans (create, load, motif_submit, destroy each)
           "served_via_plans_jobs_per_s": len(jobs) / t_served_plan,
           "served_via_plans_over_plain": t_plain / t_served_plan,
           "served_via_plans_client_loop_ms": 1e3 * t_client_plan,
           # the plain path's summed device time of the searches and sorts: a server that kept
           # the GPU as busy as each job alone does, with no host time at all, would take this
           "plain_device_ms": dev_ms,
           "ratio_bound_device_only": 1e3 * t_plain / max(dev_ms, 1e-9),
           # the client's own loop (the submissions of every job)
           "served_client_loop_ms": 1e3 * t_client,
           "served_equals_plain": bool(same),
           "served_p50_ms": float(np.percentile(lat, 50)),
           "served_p99_ms": float(np.percentile(lat, 99))}
    print(json.dumps({"saturation": sat}), flush=True)
    print(json.dumps({"mode": "serve", "workload": "Poisson arrivals, seed 5: l~U{11..15}, "
                      "d~U{2..4}, n~U{10..30}, t~U{300..800}, GC in {0.4,0.5,0.6}, FM-planted",
                      "submit": args.serve_submit, "rates": rows, "saturation": sat}),
          flush=True)
    return 0


def run_cpu_scaling(args):
    """Speedup of the CPU oracle over its single thread as the thread count grows, on a fixed
    sub-range of each (l,d) workload: the shape of the paper's Fig. 3/4 and Table II (multicore
    speedups over one thread), measured on this machine's host cores."""
    from oracle import oracle
    from paper_1403_1313_gb300 import fmgen
    cores = os.cpu_count() or 1
    threads = sorted({1, 2, 4, 8, 16, 32, 64, cores} & set(range(1, 2 * cores + 1)))
    rows = []
    for (l, d) in ((11, 3), (12, 3), (13, 3), (14, 4), (15, 4)):
        job = fmgen.fm_job(20, 600, l, d, 1000 + l)
        lo = (4 ** l) // 3
        size = 1 << 15
        t0 = time.perf_counter()
        ref, _ = oracle.search(job.rows(), l, d, lo=lo, hi=lo + size, threads=1)
        base = time.perf_counter() - t0
        # size the sample for about one second of single-thread work
        size = int(max(size, size * 1.0 / max(base, 1e-6)))
        t0 = time.perf_counter()
        ref, _ = oracle.search(job.rows(), l, d, lo=lo, hi=lo + size, threads=1)
        base = time.perf_counter() - t0
        sp = {}
        for th in threads:
            t0 = time.perf_counter()
            got, _ = oracle.search(job.rows(), l, d, lo=lo, hi=lo + size, threads=th)
            dt = time.perf_counter() - t0
            assert got.tolist() == ref.tolist()
            sp[th] = base / dt
        rows.append({"l": l, "d": d, "candidates": size, "t1_s": base, "speedup": sp})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"mode": "cpu-scaling", "cores": cores, "rows": rows}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "cpu-scaling":
        return run_cpu_scaling(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
