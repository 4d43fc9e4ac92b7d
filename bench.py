"""Benchmark: shots/s and Z[w] term-evals/s of the GB300 per-shot sampler.

Workload (the configuration the headline metric is quoted on): d=5 rotated
surface code, 49 qubits, 5 syndrome rounds, 16 T/T_DAG gates in the injected
rotation, depolarising p in {5e-4, 1e-3, 2e-3}, 10^6 shots per p, detector
sampling with bit-packed uint64 records.  One step = one pass of the whole
hot path (noise, f, detectors, exact marginals, Algorithm 1, records) over
10^6 shots for each of the three p (three launches).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Under torchrun (N > 1) every rank samples its own shot range (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_VALUES = (5e-4, 1e-3, 2e-3)
SHOTS_PER_P = 1_000_000
SEED = 0
METRIC = "shots/sec and Z[w] term-evals/sec, learned+batched vs plain GPU form, bit-exact"
WORKLOADS = {
    "cfg2": "d=5 rotated surface code, 49 qubits, 5 rounds, 16 T/T_DAG, p in {5e-4,1e-3,2e-3}, 1e6 shots per p",
    "cfg3": "d=3 triangular colour-code T-check, 19 qubits, 42 T/T_DAG, 3 check rounds, p=1e-3, postselected, 1e5 shots",
}
WORKLOAD = WORKLOADS["cfg2"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=8.0, help="bound on the oracle baseline's CPU work")
    ap.add_argument("--workload", default="cfg2", choices=sorted(WORKLOADS))
    ap.add_argument("--shots", type=int, default=None, help="shots per program per step")
    ap.add_argument("--profile", action="store_true", help="only run two launches per program (for ncu)")
    args = ap.parse_args()
    global WORKLOAD, SHOTS_PER_P
    WORKLOAD = WORKLOADS[args.workload]
    if args.workload == "cfg3":
        SHOTS_PER_P = 100_000
    if args.shots:
        SHOTS_PER_P = args.shots
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOAD_NAME = "cfg2"


def programs():
    import paper_2604_01059_gb300 as T
    from paper_2604_01059_gb300 import workloads as Wk
    if WORKLOAD_NAME == "cfg3":
        return [T.Program(Wk.config3_circuit(p=1e-3))]
    return [T.Program(Wk.config2_circuit(p=p)) for p in P_VALUES]


def term_evals_per_shot(prog):
    """Sum over the marginals one shot evaluates of their stabilizer terms
    (normalisation of every chain + one table per random output)."""
    return sum(prog.table_terms())


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def int_peak_ops(sm_mhz=None):
    """Integer-issue peak: 152 SMs x 4 SM sub-partitions x 16 INT32 lanes x clock
    (2070 MHz maximum SM clock)."""
    clk = 2070.0
    return 152 * 4 * 16 * clk * 1e6


def oracle_baseline(seconds, impl_line=False):
    """Time the oracle's C evaluator on a bounded sample of the same workload."""
    import tempfile
    from concurrent.futures import ThreadPoolExecutor

    from oracle import evaluator

    evaluator.build()
    cores = os.cpu_count() or 1
    progs = programs()
    paths = []
    tmp = tempfile.mkdtemp()
    for k, p in enumerate(progs):
        path = os.path.join(tmp, f"c2_{k}.prog")
        p.save(path)
        paths.append(path)
    orcs = [evaluator.OracleProgram(pth) for pth in paths]
    # calibrate a sample size that takes about `seconds` on all cores
    n_cal = 4
    while True:
        t0 = time.perf_counter()
        for o in orcs:
            o.sample(SEED, 0, n_cal)
        dt = time.perf_counter() - t0
        if dt > 0.5 or n_cal >= 4096:
            break
        n_cal *= 4
    per_shot = dt / (n_cal * len(orcs))
    chunk = max(1, int(seconds / max(per_shot, 1e-9) / len(orcs)))
    jobs = [(k, r * chunk) for k in range(len(orcs)) for r in range(cores)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda j: orcs[j[0]].sample(SEED, j[1], chunk), jobs))
    dt = time.perf_counter() - t0
    shots = chunk * len(jobs)
    return {"value": shots / dt, "unit": "shots/s", "cores": cores, "kind": "oracle",
            "sample": f"{shots} shots ({chunk} per thread x {cores} threads x {len(orcs)} programs) of "
                      f"the same workload, oracle C evaluator, exact arithmetic"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    base = oracle_baseline(args.cpu_seconds)
    times = []
    for _ in range(args.warmup):
        pass
    for _ in range(args.steps):
        b = oracle_baseline(max(1.0, args.cpu_seconds / max(args.steps, 1)))
        times.append(b["value"])
    val = statistics.median(times) if times else base["value"]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "shots/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "sample": base["sample"], "value": val},
            "e2e": {"value": val, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2604_01059_gb300 as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    progs = programs()
    stream = torch.cuda.current_stream()
    info = progs[0].info
    dw, ow = max(info["det_words"], 1), max(info["obs_words"], 1)
    outs = []
    for _ in progs:
        outs.append((torch.empty((SHOTS_PER_P, dw), dtype=torch.int64, device="cuda"),
                     torch.empty((SHOTS_PER_P, ow), dtype=torch.int64, device="cuda"),
                     torch.empty((SHOTS_PER_P,), dtype=torch.uint8, device="cuda")))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    offset = rank * SHOTS_PER_P

    def step():
        for p, (d, o, a) in zip(progs, outs):
            T.tsim_sample(p.h, SHOTS_PER_P, SEED, offset, None, d, o, a, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    T.tsim_sync(stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    smi_id = ids[local] if local < len(ids) else str(local)
    clocks = ClockSampler(smi_id)
    clocks.start()
    step_ms = []
    per_launch = []
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed iterations
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(progs) + 1)]
        evs[0].record(stream)
        for k, (p, (d, o, a)) in enumerate(zip(progs, outs)):
            T.tsim_sample(p.h, SHOTS_PER_P, SEED, offset, None, d, o, a, stream)
            evs[k + 1].record(stream)
        barrier()
        step_ms.append(evs[0].elapsed_time(evs[-1]))
        per_launch.append([evs[k].elapsed_time(evs[k + 1]) for k in range(len(progs))])
    T.tsim_sync(stream)
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    shots_all = SHOTS_PER_P * len(progs) * args.steps * world
    value = shots_all / (total_ms / 1e3)
    tev = sum(term_evals_per_shot(p) for p in progs) * SHOTS_PER_P * args.steps * world / (total_ms / 1e3)

    # end to end through the host-buffer entry point: copies inside the timed region
    hd = [np.zeros((SHOTS_PER_P, dw), dtype=np.uint64) for _ in progs]
    ho = [np.zeros((SHOTS_PER_P, ow), dtype=np.uint64) for _ in progs]
    ha = [np.zeros(SHOTS_PER_P, dtype=np.uint8) for _ in progs]
    for k, p in enumerate(progs):
        T.tsim_sample_host(p.h, SHOTS_PER_P, SEED, offset, None, hd[k], ho[k], ha[k], stream)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for k, p in enumerate(progs):
            T.tsim_sample_host(p.h, SHOTS_PER_P, SEED, offset, None, hd[k], ho[k], ha[k], stream)
    barrier()
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = SHOTS_PER_P * len(progs) * e2e_steps * world / e2e_s
    d2h = SHOTS_PER_P * len(progs) * (dw * 8 + ow * 8 + 1)

    # roofline of the dominant kernel (the fused sampling kernel)
    avg_launch_ms = statistics.mean(x for row in per_launch for x in row)
    ops = sum(kernel_int_ops(p) for p in progs) / len(progs) * SHOTS_PER_P
    peak = int_peak_ops()
    roof = {"bound": "alu", "achieved": ops / (avg_launch_ms / 1e3) / 1e12, "peak": peak / 1e12,
            "unit": "Tops/s", "frac": ops / (avg_launch_ms / 1e3) / peak, "traffic": None,
            "kernel": "k_sample", "ops_per_shot": ops / SHOTS_PER_P,
            "peak_source": "derived: 152 SMs x 64 INT32 lanes x 2070 MHz",
            "measured_issue_tops": int_peaks_measured()}
    base = oracle_baseline(args.cpu_seconds) if (rank == 0 and world == 1) else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "l2": "flushed between timed steps (256 MiB write)",
                           "shots_per_step": SHOTS_PER_P * len(progs) * world,
                           "terms_per_shot": [term_evals_per_shot(p) for p in progs],
                           "channels": [p.info["num_channels"] for p in progs]},
                "term_evals_per_s": tev,
                "e2e": {"value": e2e, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
                "gpu_launches": len(progs) * args.steps, "roofline": roof, "clocks": clk,
                "cpu_baseline": base}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def kernel_int_ops(prog):
    """Integer operations one shot needs in the fused sampling kernel, counted
    on the packed device tables it actually evaluates:
      noise:   ceil(C/4) Philox4x32-10 calls x 10 rounds x (2 wide multiplies
               + 2 three-input XORs) = 40 per call, plus one compare per channel;
      outputs: 3 per single-bit deterministic output, 60 per Bernoulli decision;
      tables:  per distinct parity 2W+2 (AND, XOR, popcount, insert), per merged
               term 12 (+5 per factor: two bit extracts, index, lookup, add)."""
    i = prog.info
    C = i["num_channels"]
    W = next(p for p in (1, 2, 4, 8, 16, 32) if i["x_words"] <= p)
    ops = 40 * ((C + 3) // 4) + C
    ops += 3 * (i["num_outputs"] - i["num_random"]) + 60 * i["num_random"]
    for t in range(i["num_tables"]):
        classes, factors, parities = prog.device_table_stats(t)
        ops += parities * (2 * W + 2) + 12 * classes + 5 * factors
    return ops


def int_peaks_measured():
    import paper_2604_01059_gb300 as T
    names = ["lop3", "imad", "imad_wide", "popc"]
    return {n: T.tsim_measure_int_peak(k) / 1e12 for k, n in enumerate(names)}


def run_profile():
    """Two launches per program of the chosen workload, nothing else."""
    import torch

    import paper_2604_01059_gb300 as T
    progs = programs()
    for p in progs:
        out = p.sample_torch(SHOTS_PER_P, SEED, 0)
        out = p.sample_torch(SHOTS_PER_P, SEED, 0)
    T.tsim_sync()
    torch.cuda.synchronize()
    print(json.dumps({"profile": WORKLOAD, "shots": SHOTS_PER_P, "programs": len(progs)}))


def main():
    global WORKLOAD_NAME
    args = parse()
    WORKLOAD_NAME = args.workload
    if args.profile:
        run_profile()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
