#!/usr/bin/env python
"""Benchmark of the densest-subgraph hot path on one GB300 (or N replicas).

One step = the whole hot path over one synthetic graph:
  ingest (raw pairs -> canonical CSR, on the device)
  + the Bahmani peel (Algorithm 1) at every eps of the workload
  + core numbers (Algorithm 2, first phase).
Metric: adjacency entries scanned per second (each solve reads every row
once: 2m entries per peel and per core decomposition), bit-exact outputs.

Default workload: Chung-Lu n = 2^24, exponent 2.1, mean degree 32, max
expected degree 100,000, seed 2, 2^28 generated pairs (the largest
single-graph configuration), eps = 1/10.  Inputs are resident in HBM before
the timed region; L2 is flushed (a 512 MiB write) before every timed step.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload instead (the reference arm of this project).
"""
from __future__ import annotations

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

import inputs  # noqa: E402

WORKLOADS = {
    "rmat20": dict(
        desc="R-MAT scale 20 (1,048,576 vertices, 16,777,216 generated pairs, a=.57 b=.19 c=.19, seed 1), "
             "symmetrized, deduped, loops dropped; Bahmani eps in {1/1000, 1/10, 1} + core numbers",
        gen=lambda: inputs.rmat(scale=20, m=1 << 24, a=0.57, b=0.19, c=0.19, seed=1),
        eps=[(1, 1000), (1, 10), (1, 1)]),
    "er1e4": dict(
        desc="Erdos-Renyi G(n=10,000, m=50,000) seed 0 + planted 100-vertex block at p=0.5; "
             "Bahmani eps=1/10 + core numbers",
        gen=lambda: inputs.er_block(n=10_000, m=50_000, k=100, p=0.5, seed=0),
        eps=[(1, 10)]),
    "cl22": dict(
        desc="Chung-Lu n=4,194,304, exponent 2.1, mean degree 32, max expected degree 50,000, seed 2, "
             "2^26 generated pairs (the 2^24-vertex Chung-Lu shape at a quarter of the scale, for profiling); "
             "Bahmani eps=1/10 + core numbers",
        gen=lambda: inputs.chung_lu(n=1 << 22, m_draws=1 << 26, gamma=2.1, mean=32.0, wmax=5e4, seed=2),
        eps=[(1, 10)]),
    "batch": dict(
        desc="4,096 independent graphs (seeds 1000..5095), n log-uniform in [1,000, 1,000,000], even i "
             "Erdos-Renyi mean degree 8, odd i Chung-Lu exponent 2.3 mean degree 16, each with a planted "
             "sqrt(n)-vertex block at p=0.3; Bahmani eps=1/10 for every graph, one persistent launch "
             "(dsg_batch_solve) vs one dsg_bahmani call per graph",
        kind="batch", eps=[(1, 10)]),
    "serve": dict(
        desc="Poisson arrivals at 2,000 requests/s (seed 7) over a pool of pre-generated graphs drawn as in the "
             "batch workload with n log-uniform in [1,000, 2,000,000]; each request asks for Bahmani at eps "
             "1/100 or 1/10 and, with probability 1/2, core numbers; admitted by free HBM, continuous batching",
        kind="serve", eps=[(1, 100), (1, 10)]),
    "onion20": dict(
        desc="nested shells around K_80: every vertex of shell i has 32 edges into shell i-1, each shell "
             "33/32 times the one inside it, 1,078,301 vertices in 191 shells (a long thin tail: one shell "
             "per round); Bahmani eps=1/1000 + core numbers",
        gen=lambda: inputs.onion(n=1 << 20, d=32, core=80),
        eps=[(1, 1000)], lazy_compare=True),
    "cl24": dict(
        desc="Chung-Lu n=16,777,216, exponent 2.1, mean degree 32, max expected degree 100,000, seed 2, "
             "2^28 generated pairs; Bahmani eps=1/10 + core numbers",
        gen=lambda: inputs.chung_lu(n=1 << 24, m_draws=1 << 28, gamma=2.1, mean=32.0, wmax=1e5, seed=2),
        eps=[(1, 10)]),
}

# The serial oracle needs minutes for one whole step of the largest graphs, so
# its timed leg runs on a bounded sample: the same generator at a smaller
# scale (same exponent, mean degree and seed; max expected degree halved per
# factor 4 in n, as between the 2^24 and 2^22 shapes).  Workloads not listed
# here are timed on themselves.
CL_SAMPLE = dict(
    desc="Chung-Lu n=1,048,576, exponent 2.1, mean degree 32, max expected degree 25,000, seed 2, 2^24 "
         "generated pairs (the same generator at 1/16 of the vertices and pairs)",
    gen=lambda: inputs.chung_lu(n=1 << 20, m_draws=1 << 24, gamma=2.1, mean=32.0, wmax=2.5e4, seed=2))
CPU_SAMPLES = {"cl24": CL_SAMPLE, "cl22": CL_SAMPLE}


def cpu_sample(workload: str, raw=None):
    """(raw graph, description) the oracle legs time for `workload`."""
    smp = CPU_SAMPLES.get(workload)
    if smp is None:
        return (raw if raw is not None else WORKLOADS[workload]["gen"]()), "the workload itself"
    return smp["gen"](), smp["desc"]


def workload_config(workload: str, n: int, m_raw: int, world: int) -> dict:
    """The `config` object of a JSON line: what identifies the workload, the
    same for both arms."""
    return {"workload": workload, "desc": WORKLOADS[workload]["desc"], "n": int(n), "m_raw": int(m_raw),
            "l2": "flushed before every timed step (512 MiB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cl24")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cbds", action="store_true", help="skip the densest-core / CBDS-P timing")
    ap.add_argument("--step-api", choices=["separate", "solve"], default="separate",
                    help="device-timed steps: one dsg_bahmani call per eps and one dsg_kcore call (default; "
                         "each kernel bracketed by its own timing events), or one dsg_solve call")
    ap.add_argument("--e2e-api", choices=["separate", "solve"], default="solve",
                    help="end-to-end steps (host buffers, no per-kernel events): dsg_solve (default) or "
                         "separate calls")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-parameter autotuner before warm-up")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--batch-graphs", type=int, default=4096, help="graphs in the batch workload")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: offered requests per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--serve-max-batch", type=int, default=256, help="serve: most graphs per batch launch")
    ap.add_argument("--serve-big-work", type=int, default=0,
                    help="serve: work (2 m_raw + n) above which a request is solved on its own (0: library default)")
    ap.add_argument("--serve-batch-work", type=int, default=0,
                    help="serve: most summed work per batch launch (0: library default)")
    ap.add_argument("--serve-inflight", type=int, default=0,
                    help="serve: batch launches on the device at once (0: library default)")
    ap.add_argument("--serve-ingest-threads", type=int, default=0,
                    help="serve: threads ingesting admitted requests (0: library default)")
    ap.add_argument("--serve-big-threads", type=int, default=0,
                    help="serve: threads solving big requests side by side (0: library default)")
    ap.add_argument("--pool", type=int, default=128, help="serve: distinct pre-generated graphs")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def aggregate_ranks(total_ms: float, units_per_step: int, steps: int, world: int, device=None):
    """Replicas only: every rank ran the same workload.  The job's time is the
    slowest rank's; its throughput counts every rank's units.  Returns
    (max total_ms over ranks, units/s of the whole job)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    value = units_per_step * steps * world / (total_ms / 1e3)
    return total_ms, value


# ----------------------------------------------------- byte model (per launch)
def peel_bytes(n: int, m: int, st: dict) -> int:
    """Algorithmic bytes of one peel launch (alive-list schedule):
    adjacency 8m; two offsets per failed vertex 16n; state mark write 4n;
    per round the alive id + state read 8|S_r| (round 0 reads no id: 4n) and
    the survivor list write 4|S_{r+1}|; per adjacency entry one state read
    (4 B), plus a 4 B write for each decrement of an alive neighbour."""
    sum_S = st["sum_S"]
    sum_S1 = st["sum_S"] - n  # sum over r of |S_{r+1}| = sum_{r>=1} |S_r|
    return (8 * m + 16 * n + 4 * n + 8 * sum_S - 4 * n + 4 * sum_S1 + 4 * 2 * m + 4 * st["decrements"])


def kcore_pkc_atomics(m: int, sum_core: int) -> int:
    """Degree atomics of Algorithm 2's first phase run serially: a neighbour
    above the level loses one degree, and every vertex ends at its core
    number, so the decrements number sum(deg - core) = 2m - sum(core)."""
    return 2 * m - sum_core


def kcore_bytes(n: int, m: int, st: dict, sum_core: int) -> int:
    """Algorithmic bytes of one core-number launch (the method's own traffic):
    adjacency 8m; two offsets per drained vertex 16n; the core number write
    4n; per level the remaining id and degree read 8|R_k| (level 0 reads no
    id); one degree read per adjacency entry 4 * 2m; a read and a write for
    each of the method's decrements 8 * (2m - sum(core))."""
    return (8 * m + 16 * n + 4 * n + 8 * st["rem_scanned"] - 4 * n + 4 * 2 * m
            + 8 * kcore_pkc_atomics(m, sum_core))


def kcore_overhead_bytes(n: int, m: int, st: dict, sum_core: int) -> dict:
    """Traffic the kernel's schedule adds beyond kcore_bytes: the claim
    bitmap (clear n/8, at most a claim word read per scanned vertex, one
    claim atomic per vertex), the remaining-list writes, and the atomics
    above the method's count (a neighbour taken during the level is
    decremented and then undone).  Each adjacency entry's claim-word read
    stands in for the method's degree read, so it adds nothing."""
    extra_atomics = st["atomics"] - kcore_pkc_atomics(m, sum_core)
    return {"extra_atomics": int(extra_atomics), "bytes": int(n // 8 + 4 * st["rem_scanned"] + 8 * n
                                                               + 4 * st["rem_written"] + 8 * extra_atomics)}


KERNEL_SOURCES = {
    "kcore": ["kcore.cu", "kcore_tail.cu"],
    "peel_rounds": ["peel.cu"],
    "cbds_core_hist": ["cbds.cu"],
}

# Roofline units: the peel is one kernel launch; the core numbers are the
# level kernel plus the tail (compaction and the cluster), whose launches
# together compute what the byte model counts.
ROOF_GROUPS = {
    "peel_rounds": lambda name: name == "peel_rounds",
    "kcore": lambda name: name.startswith("kcore_"),
}


def code_only(src: bytes) -> bytes:
    """Source text without // comments, trailing blanks and empty lines: what
    the compiler sees, so a comment edit does not retire a capture."""
    import re
    lines = (re.sub(rb"//.*$", b"", ln).rstrip() for ln in src.splitlines())
    return b"\n".join(ln for ln in lines if ln)


def kernel_source_sha(name: str, read=None) -> str:
    """Hash of the code a kernel is built from (its file and the shared
    headers, comments dropped).  read(file name) -> bytes overrides reading
    the working tree (e.g. to hash a committed version)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2103_00154_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name] + ["dsg_kernels.cuh", "dsg_common.cuh"]:
        if read is not None:
            data = read(f)
        else:
            with open(os.path.join(csrc, f), "rb") as fh:
                data = fh.read()
        h.update(code_only(data))
    return h.hexdigest()[:16]


def dram_traffic(workload: str, name: str):
    """DRAM bytes (read + write) of one launch of `name` from the last ncu
    capture recorded in profiles/dram_traffic.json, or None when there is none
    or the kernel's code (comments aside) changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(workload, {}).get(name)
    except (OSError, ValueError):
        return None
    if not rec or name not in KERNEL_SOURCES or rec.get("source_sha") != kernel_source_sha(name):
        return None
    return rec.get("bytes")


def cbds_hist_bytes(n: int, m: int) -> int:
    """Algorithmic bytes of the densest-core histogram pass: every vertex's
    core number 4n and row start 8n, the adjacency 8m, and the neighbour's
    core number of each edge taken once (u > v) 4m."""
    return 12 * n + 12 * m


def run_cbds_timing(args, g, core_d, set_d, flush, stream, n, m):
    """Densest core + Algorithm 2's second phase on the step's graph, from
    its core numbers (already on the device), timed like the step."""
    import torch
    import paper_2103_00154_gb300 as dsg
    from paper_2103_00154_gb300 import _native as N
    L = dsg.lib()
    for _ in range(3):
        r = g.cbds(core=core_d, out_set=set_d, want_core=False)
    torch.cuda.synchronize()
    L.dsg_profile_reset()
    L.dsg_profile_enable(1)
    ev = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = g.cbds(core=core_d, out_set=set_d, want_core=False)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    L.dsg_profile_enable(0)
    prof = N.profile_report()
    ms = [a.elapsed_time(b) for a, b in ev]
    peak, peak_kind = measured_peaks()
    roof = None
    if "cbds_core_hist" in prof:
        cnt, tot = prof["cbds_core_hist"]
        alg = cbds_hist_bytes(n, m)
        achieved = alg / (tot / cnt * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "cbds_core_hist", "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": dram_traffic(args.workload, "cbds_core_hist"),
                "alg_bytes_per_launch": int(alg), "avg_launch_ms": round(tot / cnt, 4)}
    return {"ms_per_call": round(sum(ms) / len(ms), 4), "kernel_ms": {k: round(v[1] / args.steps, 4)
                                                                     for k, v in prof.items()},
            "roofline": roof, "k_star": r.k_star, "E_core": r.E_core, "V_core": r.V_core, "E": r.E, "V": r.V,
            "n_legit": r.n_legit,
            "note": "dsg_cbds with the step's core numbers supplied on the device (densest core + second phase)"}


def run_lazy_compare(args, wl, dsg, n, src_d, dst_d, flush, stream, m, peel_stats):
    """The peel of the step's first eps with thin-tail lazy rounds on and off
    (same results, checked): launch time (CUDA events, L2 flushed before
    each), rounds, lazy rounds, vertex tests of the threshold passes, and the
    algorithmic bytes of each (the byte model's per-round alive id + state
    reads count the vertices a round actually tests)."""
    import torch
    p, q = wl["eps"][0]
    g = dsg.Graph.from_edges(n, src_d, dst_d, stream=stream)
    res = {}
    for mode in ("on", "off"):
        dsg.set_tuning(peel_lazy=(mode == "on"))
        tr = g.bahmani_trace(p, q)
        ms = []
        for _ in range(max(3, args.steps)):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.bahmani(p, q, want_set=False)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res[mode] = {"ms": round(min(ms), 4), "rounds": int(tr.rounds), "lazy_rounds": int(tr.lazy_rounds),
                     "tested": int(tr.tested), "E": int(tr.E), "V": int(tr.V)}
    dsg.set_tuning()
    g.close()
    on, off = res["on"], res["off"]
    res["same_result"] = (on["E"], on["V"], on["rounds"]) == (off["E"], off["V"], off["rounds"])
    res["speedup"] = round(off["ms"] / on["ms"], 3) if on["ms"] else None
    res["tests_saved"] = off["tested"] - on["tested"]
    return res


# ----------------------------------------------------------------- our arm
def run_ours(args, wl, raw, rank, world):
    import torch
    import paper_2103_00154_gb300 as dsg
    from paper_2103_00154_gb300 import _native as N

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    L = dsg.lib()
    stream = torch.cuda.current_stream()
    n = raw.n
    src_d = torch.from_numpy(raw.src.view(np.int32)).to(dev)
    dst_d = torch.from_numpy(raw.dst.view(np.int32)).to(dev)
    masks = [torch.empty(n, dtype=torch.uint8, device=dev) for _ in wl["eps"]]
    core_d = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    results = {}

    def step():
        g = dsg.Graph.from_edges(n, src_d, dst_d, stream=stream)
        if args.step_api == "separate":
            for i, (p, q) in enumerate(wl["eps"]):
                _, E, V = g.bahmani(p, q, out_set=masks[i])
                results[(p, q)] = (E, V)
            g.kcore(out=core_d)
        else:
            res, _ = g.solve(wl["eps"], out_sets=masks, out_core=core_d)
            for (p, q), (_, E, V) in zip(wl["eps"], res):
                results[(p, q)] = (E, V)
        m = g.m
        g.close()
        return m

    # launch parameters for this graph's size class, picked before warm-up (outside the timed region)
    tuning = None
    if not args.no_autotune:
        g = dsg.Graph.from_edges(n, src_d, dst_d, stream=stream)
        p_t, q_t = wl["eps"][len(wl["eps"]) // 2]
        t0 = time.perf_counter()
        trials = g.autotune(p_t, q_t)
        tuning = {"peel": g.tuning("peel"), "kcore": g.tuning("kcore"), "trials": trials,
                  "tuned_at_eps": f"{p_t}/{q_t}", "seconds": round(time.perf_counter() - t0, 3)}
        g.close()

    for _ in range(max(args.warmup, 0)):
        m = step()
    torch.cuda.synchronize()

    # counters for the byte model, from one traced solve of each kind (outside the timed region)
    g = dsg.Graph.from_edges(n, src_d, dst_d, stream=stream)
    m = g.m
    peel_stats = []
    for (p, q) in wl["eps"]:
        tr = g.bahmani_trace(p, q)
        peel_stats.append({"sum_S": int(tr.hist_S[:-1].sum()), "decrements": int(tr.decrements),
                           "rounds": tr.rounds})
    core_h, kst = g.kcore_counters()
    sum_core = int(core_h.astype(np.int64).sum())
    del core_h
    g.close()

    events = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    L.dsg_profile_reset()
    L.dsg_profile_enable(1)
    launches0 = L.dsg_launch_count()
    with ClockSampler(dev.index) as clk:
        t_wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("dsg_timed_steps")  # lets ncu --nvtx-include pick out the timed launches
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            events.append((a, b))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        t_wall = time.perf_counter() - t_wall0
    launches = L.dsg_launch_count() - launches0
    L.dsg_profile_enable(0)
    prof = N.profile_report()
    step_ms = [a.elapsed_time(b) for a, b in events]
    edges_per_step = 2 * m * (len(wl["eps"]) + 1)
    total_ms, value = aggregate_ranks(sum(step_ms), edges_per_step, args.steps, world, device=dev)

    # roofline of each unit (the peel launch; the core numbers' kernels
    # together); "roofline" is the one with the larger share of timed device time
    peak, peak_kind = measured_peaks()
    by_kernel = {}
    for unit, member in ROOF_GROUPS.items():
        names = sorted(k for k in prof if member(k))
        if not names:
            continue
        ms = sum(prof[k][1] for k in names)
        if unit == "peel_rounds":
            cnt = prof["peel_rounds"][0]
            per_launch = [peel_bytes(n, m, s) for s in peel_stats]
            alg = sum(per_launch) / len(per_launch)
        else:
            cnt = prof["kcore_levels"][0] if "kcore_levels" in prof else prof[names[0]][0]
            alg = kcore_bytes(n, m, kst, sum_core)
        avg_s = ms / cnt / 1e3
        achieved = alg / avg_s / 1e9
        by_kernel[unit] = {"bound": "hbm", "kernel": unit, "achieved": round(achieved, 1), "peak": peak,
                           "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                           "traffic": dram_traffic(args.workload, unit), "alg_bytes_per_launch": int(alg),
                           "avg_launch_ms": round(ms / cnt, 4)}
        if unit == "kcore":
            by_kernel[unit]["kernels"] = names
            by_kernel[unit]["schedule_overhead"] = kcore_overhead_bytes(n, m, kst, sum_core)
            by_kernel[unit]["method_atomics"] = kcore_pkc_atomics(m, sum_core)
    roof = max(by_kernel.values(), key=lambda r: r["avg_launch_ms"]) if by_kernel else None
    shares = {k: round(v[1] / sum(x[1] for x in prof.values()), 4) for k, v in prof.items()} if prof else {}
    out = {
        "ms_per_step": total_ms / args.steps,
        "value": value,
        "m": m,
        "edges_per_step": edges_per_step,
        "results": {f"{p}/{q}": list(v) for (p, q), v in results.items()},
        "roofline": roof,
        "roofline_by_kernel": by_kernel,
        "kernel_share": shares,
        "kernel_ms": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s": t_wall,
        "peel_rounds": [s["rounds"] for s in peel_stats],
        "kcore": dict(kst, sum_core=sum_core),
        "tuning": tuning,
    }

    if wl.get("lazy_compare"):
        out["peel_lazy"] = run_lazy_compare(args, wl, dsg, n, src_d, dst_d, flush, stream, m, peel_stats)
    if not args.no_cbds:
        g = dsg.Graph.from_edges(n, src_d, dst_d, stream=stream)
        g.kcore(out=core_d)
        set_d = torch.empty(n, dtype=torch.uint8, device=dev)
        out["cbds"] = run_cbds_timing(args, g, core_d, set_d, flush, stream, n, m)
        g.close()
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, wl, raw, dev, edges_per_step, world)
    return out


def run_e2e(args, wl, raw, dev, edges_per_step, world):
    """Same metric through the public API with HOST buffers: the raw pairs are
    copied from pinned memory inside the call, results read back to pinned
    host buffers, every step."""
    import torch
    import paper_2103_00154_gb300 as dsg
    n = raw.n
    src_h = torch.from_numpy(raw.src.view(np.int32)).pin_memory()
    dst_h = torch.from_numpy(raw.dst.view(np.int32)).pin_memory()
    masks = [torch.empty(n, dtype=torch.uint8).pin_memory() for _ in wl["eps"]]
    core_h = torch.empty(n, dtype=torch.int32).pin_memory()
    stream = torch.cuda.current_stream()

    def step():
        g = dsg.Graph.from_edges(n, src_h, dst_h, stream=stream)
        if args.e2e_api == "separate":
            for i, (p, q) in enumerate(wl["eps"]):
                g.bahmani(p, q, out_set=masks[i])
            g.kcore(out=core_h)
        else:
            g.solve(wl["eps"], out_sets=masks, out_core=core_h)
        g.close()

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    torch.cuda.synchronize()
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = 8 * raw.m_raw
    d2h = n * len(wl["eps"]) + 4 * n + 16 * len(wl["eps"])
    return {"value": edges_per_step * steps * world / dt, "unit": "edges/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt / steps * 1e3}


# ------------------------------------------------------------ batch workload
def batch_raws(G: int):
    """Generate the batch members on host threads (the generator releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(lambda i: inputs.batch_graph(i, threads=1), range(G)))


def pack_on_device(graphs, dev):
    """Concatenated CSR of resident graphs, assembled on the device."""
    import torch
    import ctypes
    import paper_2103_00154_gb300 as dsg
    ns = [g.n for g in graphs]
    ms = [2 * g.m for g in graphs]
    G = len(graphs)
    vb = np.zeros(G + 1, np.uint64)
    vb[1:] = np.cumsum(ns)
    ab = np.zeros(G + 1, np.uint64)
    ab[1:] = np.cumsum(ms)
    N, A = int(vb[-1]), int(ab[-1])
    off = torch.empty(N + 1, dtype=torch.int64, device=dev)
    adj = torch.empty(max(A, 1), dtype=torch.int32, device=dev)
    L = dsg.lib()
    for g, gr in enumerate(graphs):
        o = off[int(vb[g]):int(vb[g]) + gr.n + 1]
        a = adj[int(ab[g]):int(ab[g]) + 2 * gr.m]
        tmp = torch.empty(gr.n + 1, dtype=torch.int64, device=dev)
        dsg._native.check(L.dsg_graph_csr(gr._h, tmp.data_ptr(), a.data_ptr() if gr.m else None), "graph_csr")
        o.copy_(tmp + int(ab[g]))
    torch.cuda.synchronize()
    return torch.from_numpy(vb.view(np.int64)).to(dev), off, adj, N, A


def run_batch(args, wl, rank, world):
    import torch
    import paper_2103_00154_gb300 as dsg
    from paper_2103_00154_gb300 import _native as N
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    L = dsg.lib()
    G = args.batch_graphs
    t0 = time.perf_counter()
    raws = batch_raws(G)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    graphs = [dsg.Graph.from_edges(r.n, r.src, r.dst) for r in raws]
    t_ingest = time.perf_counter() - t0
    vb, off, adj, Nv, A = pack_on_device(graphs, dev)
    p, q = wl["eps"][0]
    solver = dsg.BatchSolver(vb, off, adj, [(p, q)])
    out_set = torch.empty(max(Nv, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    tuning = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        trials = solver.autotune()
        tuning = {"trials": trials, "seconds": round(time.perf_counter() - t0, 3)}
    for _ in range(max(args.warmup, 1)):
        E, V, R, BR = solver.solve(out_set=out_set, stream=stream)
    # counters of the byte model, from one solve outside the timed region
    bstats = np.zeros(4, np.uint64)
    solver.solve(out_set=out_set, stream=stream, stats=bstats)
    torch.cuda.synchronize()
    L.dsg_profile_reset()
    L.dsg_profile_enable(1)
    launches0 = L.dsg_launch_count()
    ms_steps = []
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.zero_()
            a_ev = torch.cuda.Event(enable_timing=True)
            b_ev = torch.cuda.Event(enable_timing=True)
            a_ev.record(stream)
            E, V, R, BR = solver.solve(out_set=out_set, stream=stream)
            b_ev.record(stream)
            b_ev.synchronize()
            ms_steps.append(a_ev.elapsed_time(b_ev))
    launches = L.dsg_launch_count() - launches0
    L.dsg_profile_enable(0)
    prof = N.profile_report()
    total_ms, value = aggregate_ranks(sum(ms_steps), G, args.steps, world, device=dev)
    # roofline of the block-per-graph launch: the peel byte model summed over its graphs
    roof = None
    if "batch_solve" in prof and int(bstats[3]) == 0:
        cnt, tot = prof["batch_solve"]
        sum_S, dec, entries = int(bstats[0]), int(bstats[1]), int(bstats[2])
        alg = peel_bytes(int(Nv), entries // 2, {"sum_S": sum_S, "decrements": dec})
        peak, peak_kind = measured_peaks()
        achieved = alg / (tot / cnt * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "batch_solve", "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                "alg_bytes_per_launch": int(alg), "avg_launch_ms": round(tot / cnt, 4),
                "model": "sum over the batch's graphs of the single-graph peel byte model"}
    # plain form: one dsg_bahmani per graph on the same resident graphs
    masks = [torch.empty(max(g.n, 1), dtype=torch.uint8, device=dev) for g in graphs]
    for g, m in zip(graphs[:64], masks[:64]):
        g.bahmani(p, q, out_set=m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [g.bahmani(p, q, out_set=m) for g, m in zip(graphs, masks)]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    same = all((int(E[i]), int(V[i])) == (plain[i][1], plain[i][2]) for i in range(G))
    return {"ms_per_step": total_ms / args.steps, "value": value, "edges": A, "N": Nv, "t_gen_s": t_gen,
            "t_ingest_s": t_ingest, "plain_ms": t_plain * 1e3, "plain_graphs_per_s": G / t_plain,
            "batched_equals_plain": bool(same), "gpu_launches": int(launches), "clocks": clk.summary(),
            "rounds_max": int(R.max()), "raws": raws, "E": E, "V": V, "R": R, "BR": BR, "roofline": roof,
            "tuning": tuning, "kernel_ms": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
            "grid_path_graphs": int(bstats[3])}


def _serve_oracle(n, src, dst, eps):
    """Oracle results of one pool graph (runs in a worker process): per eps
    (E, V, rounds, best round, set), and the core numbers."""
    import oracle
    c = oracle.canonical_csr(n, src, dst)
    out = {}
    for p, q in eps:
        w = oracle.bahmani(c, p, q)
        out[(p, q)] = (w.E, w.V, w.rounds, w.best_round, np.asarray(w.mask, np.uint8))
    return out, np.asarray(oracle.kcore_bz(c), np.uint32)


def run_serve(args, wl):
    """Poisson request stream against dsg_serve_*; pool graphs live in pinned
    host memory and are lent to the server (no copy at submit).  Every
    completed request is checked against the oracle's result for its (pool
    graph, eps): (E, V), rounds, best round, the set, and the core numbers when
    asked."""
    import threading
    import multiprocessing as mproc
    import torch
    import paper_2103_00154_gb300 as dsg
    from concurrent.futures import ThreadPoolExecutor
    # the oracle cache first, in spawned processes (no CUDA context in this process yet)
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        pool = list(ex.map(lambda i: inputs.batch_graph(i, seed_base=7_000_000, n_hi=2_000_000, threads=1),
                           range(args.pool)))
    t0 = time.perf_counter()
    with mproc.get_context("spawn").Pool(os.cpu_count() or 1) as pp:
        cache = pp.starmap(_serve_oracle, [(g.n, g.src, g.dst, wl["eps"]) for g in pool])
    t_oracle = time.perf_counter() - t0
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    pinned = [(torch.from_numpy(g.src.view(np.int32)).pin_memory(), torch.from_numpy(g.dst.view(np.int32)).pin_memory())
              for g in pool]
    rng = np.random.default_rng(7)
    n_req = int(args.rate * args.duration)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n_req))
    picks = rng.integers(0, len(pool), n_req)
    eps_i = rng.integers(0, len(wl["eps"]), n_req)
    cores = rng.random(n_req) < 0.5
    # plain form first: one request at a time through the one-graph calls
    # (the first 10 untimed: module load, memory pool growth)
    for i in range(min(n_req, 10)):
        g = pool[picks[i]]
        gr = dsg.Graph.from_edges(g.n, pinned[picks[i]][0], pinned[picks[i]][1])
        gr.bahmani(*wl["eps"][eps_i[i]], want_set=False)
        gr.kcore()
        gr.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_plain = 0
    for i in range(min(n_req, 200)):
        g = pool[picks[i]]
        p, q = wl["eps"][eps_i[i]]
        gr = dsg.Graph.from_edges(g.n, pinned[picks[i]][0], pinned[picks[i]][1])
        gr.bahmani(p, q, want_set=False)
        if cores[i]:
            gr.kcore()
        gr.close()
        n_plain += 1
    plain_gps = n_plain / (time.perf_counter() - t0)
    srv = dsg.Server(max_batch=args.serve_max_batch, big_work=args.serve_big_work,
                     max_batch_work=args.serve_batch_work, max_inflight=args.serve_inflight,
                     big_threads=args.serve_big_threads, ingest_threads=args.serve_ingest_threads)
    tickets = [None] * n_req
    bufs = [None] * n_req
    rejected = 0
    done = threading.Event()
    lat = []
    check = {"checked": 0, "mismatch": 0, "sets": 0, "cores": 0, "bad_status": 0}

    def collector():
        i = 0
        while i < n_req:
            t = tickets[i]
            if t is None:
                if done.is_set() and tickets[i] is None:
                    i += 1
                    continue
                time.sleep(0.0002)
                continue
            if t == -1:
                i += 1
                continue
            r = srv.poll(t, 200_000)
            if r is None:
                continue
            lat.append(r["latency_us"])
            out_set, core = bufs[i]
            want, want_core = cache[int(picks[i])]
            E, V, R, BR, mask = want[tuple(wl["eps"][eps_i[i]])]
            ok = r["status"] == 0 and (r["E"], r["V"], r["rounds"], r["best_round"]) == (E, V, R, BR)
            ok = ok and np.array_equal(out_set, mask)
            check["sets"] += 1
            if core is not None:
                ok = ok and np.array_equal(core, want_core)
                check["cores"] += 1
            check["bad_status"] += r["status"] != 0
            check["checked"] += 1
            check["mismatch"] += not ok
            bufs[i] = None
            i += 1

    th = threading.Thread(target=collector)
    th.start()
    start = time.perf_counter()
    for i in range(n_req):
        delay = start + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        g = pool[picks[i]]
        p, q = wl["eps"][eps_i[i]]
        out_set = np.empty(max(g.n, 1), np.uint8)
        core = np.empty(max(g.n, 1), np.uint32) if cores[i] else None
        bufs[i] = (out_set[:g.n], None if core is None else core[:g.n])
        t = srv.submit(g.n, pinned[picks[i]][0], pinned[picks[i]][1], p, q, bool(cores[i]), out_set, core,
                       borrow=True)
        if t is None:
            rejected += 1
            bufs[i] = None
            tickets[i] = -1
        else:
            tickets[i] = t
    offered_s = time.perf_counter() - start
    done.set()
    th.join()
    wall = time.perf_counter() - start
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    completed = len(lat)
    return {"completed": completed, "rejected": rejected, "offered": n_req, "offered_rate": n_req / offered_s,
            "graphs_per_s": completed / wall, "wall_s": wall,
            "p50_us": float(np.percentile(lat, 50)) if completed else None,
            "p99_us": float(np.percentile(lat, 99)) if completed else None, "batches": st["batches"],
            "plain_graphs_per_s": plain_gps, "all_ok": check["mismatch"] == 0 and check["bad_status"] == 0,
            "checked_vs_oracle": check["checked"], "mismatch_vs_oracle": check["mismatch"],
            "sets_checked": check["sets"], "cores_checked": check["cores"], "oracle_cache_s": round(t_oracle, 1),
            "pool": len(pool), "saturated": completed / wall < 0.95 * args.rate,
            "time_split": {"big_done": st["big_done"], "ingest_busy_s": round(st["ingest_busy_s"], 3),
                           "big_busy_s": round(st["big_busy_s"], 3), "batch_device_s": round(st["batch_device_s"], 3),
                           "wall_s": round(wall, 3),
                           "offered_work_per_s": float(sum(2 * pool[i].m_raw + pool[i].n for i in picks) / offered_s)}}


def batch_cpu_baseline(raws, eps, seconds):
    """The oracle on whole batch members over all host cores (one graph per
    process), until about `seconds` have passed; graphs/s of that sample."""
    import multiprocessing as mproc
    ctx = mproc.get_context("spawn")
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    done, edges = 0, 0
    with ctx.Pool(cores) as pool:
        idx = 0
        while time.perf_counter() - t0 < seconds and idx < len(raws):
            chunk = raws[idx: idx + cores]
            idx += len(chunk)
            for m in pool.starmap(_oracle_one, [(r.n, r.src, r.dst, eps) for r in chunk]):
                done += 1
                edges += 2 * m
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "graphs/s", "cores": cores, "kind": "oracle",
            "edges_per_s": edges / dt,
            "sample": f"first {done} batch members, one per process on {cores} host cores, {dt:.1f} s"}


def _oracle_one(n, src, dst, eps):
    import oracle
    c = oracle.canonical_csr(n, src, dst)
    oracle.bahmani(c, *eps)
    return c.m


# ---------------------------------------------------------------- oracle arm
def oracle_step(raw, eps):
    import oracle
    c = oracle.from_raw(raw)
    for p, q in eps:
        oracle.bahmani(c, p, q)
    oracle.kcore_bz(c)
    return c.m


def run_cpu_baseline(args, wl, raw, seconds):
    """The oracle as it stands, serial on one host core, on whole steps of
    the workload's CPU sample (ingest + the workload's peels + core numbers)
    until about `seconds` of CPU time have passed."""
    smp, smp_desc = cpu_sample(args.workload, raw)
    t0 = time.perf_counter()
    steps = 0
    m = 0
    while True:
        m = oracle_step(smp, wl["eps"])
        steps += 1
        if time.perf_counter() - t0 >= seconds or steps >= 50:
            break
    dt = time.perf_counter() - t0
    eps_step = 2 * m * (len(wl["eps"]) + 1)
    return {"value": eps_step * steps / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} whole step(s) (ingest + {len(wl['eps'])} peel(s) + core numbers) of {smp_desc}, "
                      f"{dt:.1f} s, serial C oracle"}


def run_reference(args, wl):
    """The reference arm: the serial C oracle (there is no reference
    implementation; the paper holds no code) on the host cores, each step one
    whole step of the workload's CPU sample."""
    smp, smp_desc = cpu_sample(args.workload)
    for _ in range(max(args.warmup, 0)):
        oracle_step(inputs.er_block(n=10_000, m=50_000, k=100, p=0.5, seed=0), wl["eps"])
    t0 = time.perf_counter()
    m = 0
    for _ in range(args.steps):
        m = oracle_step(smp, wl["eps"])
    dt = time.perf_counter() - t0
    eps_step = 2 * m * (len(wl["eps"]) + 1)
    value = eps_step * args.steps / dt
    n_full, m_raw_full = workload_size(args.workload)
    return {"impl": "reference", "metric": "edges scanned/s", "value": value, "unit": "edges/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(args.workload, n_full, m_raw_full,
                                                           int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step one whole step (ingest + {len(wl['eps'])} peel(s) + core "
                                       f"numbers) of {smp_desc}; warm-up on the 10^4-vertex case"},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def workload_size(workload: str):
    """(n, generated pairs) of a single-graph workload, without generating it."""
    sizes = {"cl24": (1 << 24, 1 << 28), "cl22": (1 << 22, 1 << 26), "rmat20": (1 << 20, 1 << 24)}
    if workload in sizes:
        return sizes[workload]
    raw = WORKLOADS[workload]["gen"]()
    return raw.n, raw.m_raw


def replica_launch_cmd(argv, gpus: int, port: int):
    """The command that runs this script as `gpus` replica ranks on one node
    (torch.distributed.run, rendezvous on 127.0.0.1), forwarding argv."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]


def main():
    args = parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # asked for N GPUs but started as one process: start the N replica ranks
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        return subprocess.call(replica_launch_cmd(sys.argv[1:], args.gpus, port))
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus and world > 1:
        print(f"bench: --gpus {args.gpus} but {world} ranks were started; the ranks decide", file=sys.stderr)
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        if wl.get("kind"):
            print(json.dumps({"impl": "reference", "unavailable": f"the {args.workload} workload has no oracle "
                              "arm; the single-graph workloads do"}), flush=True)
            return 0
        print(json.dumps(run_reference(args, wl)), flush=True)
        return 0

    import torch
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if wl.get("kind") == "serve":
        res = run_serve(args, wl)
        if rank == 0:
            print(json.dumps({
                "metric": "graphs/s", "value": res["graphs_per_s"], "unit": "graphs/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": res["wall_s"] * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": "serve", "desc": wl["desc"], "rate": args.rate, "duration_s": args.duration,
                           "pool": res["pool"],
                           "server": {"max_batch": args.serve_max_batch, "big_work": args.serve_big_work,
                                      "max_batch_work": args.serve_batch_work, "max_inflight": args.serve_inflight,
                                      "big_threads": args.serve_big_threads,
                                      "ingest_threads": args.serve_ingest_threads, "0": "library default"}},
                "serve": {k: res[k] for k in ("completed", "rejected", "offered", "offered_rate", "p50_us", "p99_us",
                                              "batches", "saturated", "all_ok", "checked_vs_oracle",
                                              "mismatch_vs_oracle", "sets_checked", "cores_checked",
                                              "oracle_cache_s", "time_split")},
                "plain": {"graphs_per_s": res["plain_graphs_per_s"],
                          "form": "one request at a time: ingest + dsg_bahmani (+ dsg_kcore) per request"},
                "served_over_plain": res["graphs_per_s"] / res["plain_graphs_per_s"]}), flush=True)
        return 0
    if wl.get("kind") == "batch":
        res = run_batch(args, wl, rank, world)
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu:
            cpu = batch_cpu_baseline(res["raws"], wl["eps"][0], args.cpu_seconds)
        if rank == 0:
            print(json.dumps({
                "metric": "graphs/s", "value": res["value"], "unit": "graphs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": "batch", "desc": wl["desc"], "graphs": args.batch_graphs,
                           "vertices": res["N"], "adjacency_entries": res["edges"],
                           "l2": "flushed before every timed step (512 MiB write)"},
                "edges_scanned_per_s": res["edges"] * args.steps * world / (res["ms_per_step"] * args.steps / 1e3),
                "plain": {"ms": res["plain_ms"], "graphs_per_s": res["plain_graphs_per_s"],
                          "form": "one dsg_bahmani call per resident graph, same GPU"},
                "batched_over_plain": res["value"] / world / res["plain_graphs_per_s"],
                "batched_equals_plain": res["batched_equals_plain"],
                "cpu_baseline": cpu, "gpu_launches": res["gpu_launches"], "clocks": res["clocks"],
                "roofline": res["roofline"], "kernel_ms_per_step": res["kernel_ms"],
                "run": {"tuning": res["tuning"], "grid_path_graphs": res["grid_path_graphs"]},
                "host_generation_s": res["t_gen_s"], "ingest_s": res["t_ingest_s"],
                "rounds_max": res["rounds_max"]}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    raw = wl["gen"]()
    res = run_ours(args, wl, raw, rank, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_cpu_baseline(args, wl, raw, args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": "edges scanned/s",
            "value": res["value"],
            "unit": "edges/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u32",
            "data": "synthetic",
            "config": workload_config(args.workload, raw.n, raw.m_raw, world),
            "m": res["m"],
            "edges_scanned_per_step": res["edges_per_step"],
            "run": {"step": {"device_timed": "dsg_graph_from_edges, then " + (
                                    "one dsg_bahmani per eps and dsg_kcore, each kernel bracketed by timing events"
                                    if args.step_api == "separate" else
                                    "dsg_solve (peels and core numbers side by side), each kernel bracketed by "
                                    "timing events on its own stream"),
                                "e2e": "host buffers: dsg_graph_from_edges, then " + (
                                    "dsg_solve (peels and core numbers side by side on half the GPU each unless "
                                    "the tuned times say the core numbers dominate)" if args.e2e_api == "solve"
                                    else "one dsg_bahmani per eps and dsg_kcore")},
                       "tuning": res["tuning"]},
            "graphs_per_s": world * args.steps / (res["ms_per_step"] * args.steps / 1e3),
            "roofline": res["roofline"],
            "roofline_by_kernel": res["roofline_by_kernel"],
            "cpu_baseline": cpu,
            "e2e": res.get("e2e"),
            "gpu_launches": res["gpu_launches"],
            "clocks": res["clocks"],
            "kernel_share": res["kernel_share"],
            "kernel_ms_per_step": res["kernel_ms"],
            "peel_rounds": res["peel_rounds"],
            "kcore_counters": res["kcore"],
            "peel_lazy": res.get("peel_lazy"),
            "results": res["results"],
            "cbds": res.get("cbds"),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
