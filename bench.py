"""Benchmark: shots/s and Z[w] term-evals/s of the GB300 per-shot sampler.

Workload (the configuration the headline metric is quoted on): d=5 rotated
surface code, 49 qubits, 5 syndrome rounds, 16 T/T_DAG gates in the injected
rotation, depolarising p in {5e-4, 1e-3, 2e-3}, 10^6 shots per p, detector
sampling with bit-packed uint64 records.  One step = one pass of the whole
hot path (noise, f, detectors, exact marginals, Algorithm 1, records) over
10^6 shots for each of the three p.

Two forms are timed on the same GPU and must write identical records:
  value  learned + batched: programs compiled with the learned cut order (the
         committed network weights; heuristic order when they are absent), all
         programs in one persistent launch replayed from a CUDA graph;
  plain  heuristic cut order, one tsim_sample launch per program.

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
    "cfg3": "d=3 triangular colour-code T-check, 19 qubits, 42 T/T_DAG, 3 check rounds, p=1e-3, postselected, 1e7 shots",
    "cfg4": "batched launch: 256 seeded random noisy Clifford+T mirror circuits (20-60 qubits, depth 20-100, "
            "8-40 T/T_DAG, 2-qubit density 0.3, p in U[1e-4,3e-3]), shots log-uniform in [1e3,1e6], "
            "one persistent launch replayed from a CUDA graph, autotuned shot block",
}
CFG4_TABLE_BUDGET = 2048     # terms per marginal table
CFG4_PROGRAM_BUDGET = 8192   # terms per program
WORKLOAD = WORKLOADS["cfg2"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: about 0.2 s per form)")
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
        SHOTS_PER_P = 10_000_000
    if args.shots:
        SHOTS_PER_P = args.shots
    if args.steps is None:
        args.steps = {"cfg2": 100, "cfg3": 3, "cfg4": 20}[args.workload]
    return args


def shard_offsets(rank, shots):
    """Weak scaling: rank r samples shots [r n, (r + 1) n) of every program
    (the Philox counter is the global shot index, so the ranks' records
    concatenate to one run over all of them)."""
    return [rank * n for n in shots]


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value over the ranks (timings: the slowest rank decides)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOAD_NAME = "cfg2"
SHOTS_LIST = None


def cut_model():
    """The committed cut-order network weights, or None."""
    from paper_2604_01059_gb300.train_cut_order import load_weights
    return load_weights()


def config4_programs(n=256):
    """Compile the batched workload in parallel host threads; circuits over the
    term budgets are skipped and the next seeds drawn (deterministic order).
    Returns (program, shots, circuit text) triples."""
    from concurrent.futures import ThreadPoolExecutor

    import paper_2604_01059_gb300 as T
    from paper_2604_01059_gb300 import workloads as Wk
    pool = Wk.config4_batch(n=4 * n, seed=0)

    def build(item):
        txt, shots = item
        try:
            p = T.Program(txt, chi_budget=CFG4_TABLE_BUDGET, total_budget=CFG4_PROGRAM_BUDGET)
        except T.TsimError as e:
            if e.code == 3:
                return None
            raise
        return (p, shots, txt) if p.info["total_terms"] <= CFG4_PROGRAM_BUDGET else None

    out = []
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for k in range(0, len(pool), 64):
            for r in ex.map(build, pool[k:k + 64]):
                if r is not None and len(out) < n:
                    out.append(r)
            if len(out) >= n:
                break
    return out


CFG4_TEXTS = None


def programs(decomp=0):
    """The workload's programs.  The batched workload's circuits are selected
    once with the heuristic order; another order compiles the same circuits
    (it never has more terms, so they stay within the budgets)."""
    import paper_2604_01059_gb300 as T
    from paper_2604_01059_gb300 import workloads as Wk
    global SHOTS_LIST, CFG4_TEXTS
    if WORKLOAD_NAME == "cfg3":
        return [T.Program(Wk.config3_circuit(p=1e-3), decomp=decomp)]
    if WORKLOAD_NAME == "cfg4":
        if CFG4_TEXTS is None or decomp == 0:
            pr = config4_programs()
            SHOTS_LIST = [s for _, s, _ in pr]
            CFG4_TEXTS = [t for _, _, t in pr]
            if decomp == 0:
                return [p for p, _, _ in pr]
        return [T.Program(t, chi_budget=CFG4_TABLE_BUDGET, total_budget=CFG4_PROGRAM_BUDGET, decomp=decomp)
                for t in CFG4_TEXTS]
    return [T.Program(Wk.config2_circuit(p=p), decomp=decomp) for p in P_VALUES]


def learned_programs():
    """Programs in the learned cut order, with the order's bookkeeping."""
    import paper_2604_01059_gb300 as T
    w = cut_model()
    if w is None:
        return programs(), {"cut_order": "heuristic (no trained weights)"}
    before = T.tsim_cut_policy_stats()
    T.tsim_cut_model_set(w)
    try:
        progs = programs(decomp=T.DECOMP_LEARNED)
    finally:
        T.tsim_cut_model_set(None)
    after = T.tsim_cut_policy_stats()
    d = [a - b for a, b in zip(after, before)]
    return progs, {"cut_order": "learned (GNN scores, heuristic as fallback and judge)",
                   "scorer_calls": d[0], "scored": d[1], "marginals_learned_kept": d[2],
                   "marginals_heuristic_kept": d[3]}


def shots_of(k):
    return SHOTS_LIST[k] if SHOTS_LIST else SHOTS_PER_P


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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


class OracleBench:
    """The oracle's C evaluator on the host cores, on the programs of the
    workload (at most 16 of them): calibrated once, then timed on bounded
    samples."""

    def __init__(self, progs):
        import tempfile

        from oracle import evaluator

        evaluator.build()
        self.cores = os.cpu_count() or 1
        tmp = tempfile.mkdtemp()
        self.orcs = []
        for k, p in enumerate(progs[:16]):
            path = os.path.join(tmp, f"c2_{k}.prog")
            p.save(path)
            self.orcs.append(evaluator.OracleProgram(path))
        n_cal = 4
        while True:  # per-shot time of one thread
            t0 = time.perf_counter()
            for o in self.orcs:
                o.sample(SEED, 0, n_cal)
            dt = time.perf_counter() - t0
            if dt > 0.5 or n_cal >= 4096:
                break
            n_cal *= 4
        self.per_shot = dt / (n_cal * len(self.orcs))

    def run(self, seconds):
        """About `seconds` of oracle work on all cores; shots per second."""
        from concurrent.futures import ThreadPoolExecutor
        chunk = max(1, int(seconds / max(self.per_shot, 1e-9) / len(self.orcs)))
        jobs = [(k, r * chunk) for k in range(len(self.orcs)) for r in range(self.cores)]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=self.cores) as ex:
            list(ex.map(lambda j: self.orcs[j[0]].sample(SEED, j[1], chunk), jobs))
        dt = time.perf_counter() - t0
        shots = chunk * len(jobs)
        return {"value": shots / dt, "unit": "shots/s", "cores": self.cores, "kind": "oracle",
                "sample": f"{shots} shots ({chunk} per thread x {self.cores} threads x {len(self.orcs)} programs) "
                          f"of the same workload, oracle C evaluator, exact arithmetic"}


def oracle_baseline(seconds, progs=None):
    """Time the oracle's C evaluator on a bounded sample of the same workload."""
    return OracleBench(progs if progs is not None else programs()).run(seconds)


def run_reference(args):
    """The reference arm: the oracle (plain C, exact) on the host cores, on the
    same programs, each step a bounded sample of the workload (the whole run
    about --cpu-seconds of oracle work plus one calibration)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    ob = OracleBench(programs())
    per_step = max(0.05, args.cpu_seconds / max(args.steps, 1))
    for _ in range(args.warmup):
        ob.run(0.02)
    vals = []
    b = None
    for _ in range(args.steps):
        b = ob.run(per_step)
        vals.append(b["value"])
    val = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "shots/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"kind": "oracle", "cores": b["cores"], "sample": b["sample"] + " (per step)",
                             "value": val},
            "e2e": {"value": val, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _outputs(progs, shots):
    import torch
    outs = []
    for p, ns in zip(progs, shots):
        i = p.info
        outs.append((torch.empty((ns, max(i["det_words"], 1)), dtype=torch.int64, device="cuda"),
                     torch.empty((ns, max(i["obs_words"], 1)), dtype=torch.int64, device="cuda"),
                     torch.empty((ns,), dtype=torch.uint8, device="cuda")))
    return outs


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
    plain_progs = programs()
    progs, cut = learned_programs()
    n = len(progs)
    assert n == len(plain_progs)
    shots = [shots_of(k) for k in range(n)]
    offsets = shard_offsets(rank, shots)  # weak scaling: every rank its own shot range
    seeds = [SEED] * n
    stream = torch.cuda.current_stream()
    outs = _outputs(progs, shots)
    plain_outs = _outputs(plain_progs, shots)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def plain_step():
        for k, (p, (d, o, a)) in enumerate(zip(plain_progs, plain_outs)):
            T.tsim_sample(p.h, shots[k], seeds[k], offsets[k], None, d, o, a, stream)

    batch = T.tsim_batch_create([p.h for p in progs], shots, seeds, offsets, None,
                                [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs], autotune=True)
    binfo = T.tsim_batch_info(batch)

    def batch_step():
        T.tsim_batch_launch(batch, stream)

    for _ in range(max(args.warmup, 3)):
        plain_step()
        batch_step()
    T.tsim_sync(stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(step_fn, steps):
        total = 0.0
        for _ in range(steps):
            flush.fill_(1)  # evict L2 between timed iterations
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step_fn()
            e1.record(stream)
            barrier()
            total += e0.elapsed_time(e1)
        T.tsim_sync(stream)
        return max_over_ranks(total, dist, "cuda")

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    clocks = ClockSampler(ids[local] if local < len(ids) else str(local))
    clocks.start()
    batch_ms = timed(batch_step, args.steps)
    plain_ms = timed(plain_step, args.steps)
    clk = clocks.stop()
    T.tsim_batch_free(batch)
    # both forms wrote every record of the step: they must agree bit for bit
    identical = all(torch.equal(a[:, :p.info["det_words"]], b[:, :p.info["det_words"]]) and
                    torch.equal(x[:, :p.info["obs_words"]], y[:, :p.info["obs_words"]]) and torch.equal(u, v)
                    for p, (a, x, u), (b, y, v) in zip(progs, outs, plain_outs))
    shots_step = sum(shots) * world
    value = shots_step * args.steps / (batch_ms / 1e3)
    plain = shots_step * args.steps / (plain_ms / 1e3)
    terms_step = sum(term_evals_per_shot(p) * ns for p, ns in zip(progs, shots)) * world
    plain_terms_step = sum(term_evals_per_shot(p) * ns for p, ns in zip(plain_progs, shots)) * world
    tev = terms_step * args.steps / (batch_ms / 1e3)

    # end to end through the host-buffer entry point: copies inside the timed
    # region, into page-locked host buffers
    def pinned(shape, dtype):
        return torch.zeros(shape, dtype=dtype, pin_memory=True).numpy()

    hbuf = []
    for p, ns in zip(progs, shots):
        i = p.info
        hbuf.append((pinned((ns, max(i["det_words"], 1)), torch.int64).view(np.uint64),
                     pinned((ns, max(i["obs_words"], 1)), torch.int64).view(np.uint64), pinned((ns,), torch.uint8)))

    def e2e_step():
        for k, p in enumerate(progs):
            i = p.info
            d, o, a = hbuf[k]
            T.tsim_sample_host(p.h, shots[k], seeds[k], offsets[k], None, d if i["det_words"] else None,
                               o if i["obs_words"] else None, a, stream)

    e2e_step()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = shots_step * e2e_steps / e2e_s
    d2h = sum(ns * (p.info["det_words"] * 8 + p.info["obs_words"] * 8 + 1) for p, ns in zip(progs, shots))

    # roofline of the dominant kernel: the persistent batched sampling kernel
    ops = sum(kernel_int_ops(p) * ns for p, ns in zip(progs, shots))
    peak = int_peak_ops()
    achieved = ops / (batch_ms / args.steps / 1e3)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": ("k_batch (persistent kernel over all programs, graph replay)" if binfo.get("form", 0) == 0
                       else "k_sample (each program's launch, graph replay)"),
            "ops_per_shot": ops / sum(shots),
            "peak_source": "derived: 152 SMs x 4 sub-partitions x 16 INT32 lanes x 2070 MHz",
            "measured_issue_tops": int_peaks_measured()}
    base = oracle_baseline(args.cpu_seconds, progs) if (rank == 0 and world == 1 and args.cpu_seconds > 0) else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": batch_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "l2": "flushed between timed steps (256 MiB write)",
                           "programs": n, "shots_per_step": shots_step,
                           "terms_per_shot": [term_evals_per_shot(p) for p in progs][:8],
                           "plain_terms_per_shot": [term_evals_per_shot(p) for p in plain_progs][:8],
                           "terms_all_programs": {"learned": sum(term_evals_per_shot(p) for p in progs),
                                                  "heuristic": sum(term_evals_per_shot(p) for p in plain_progs)},
                           "channels": [p.info["num_channels"] for p in progs][:8],
                           "form": "learned cut order + batched persistent launch (CUDA graph)",
                           "cut": cut, "batch": binfo},
                "term_evals_per_s": tev,
                "identical_records": bool(identical),
                "plain": {"value": plain, "unit": "shots/s", "ms_per_step": plain_ms / args.steps,
                          "term_evals_per_s": plain_terms_step * args.steps / (plain_ms / 1e3),
                          "form": "heuristic cut order, one tsim_sample launch per program",
                          "gpu_launches": args.steps * n},
                "speedup_vs_plain": value / plain,
                "e2e": {"value": e2e, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                        "api": "tsim_sample_host (device staging, records copied to page-locked host memory inside the timed region)"},
                "gpu_launches": args.steps * launches_per_step(progs, shots, binfo), "roofline": roof, "clocks": clk,
                "cpu_baseline": base}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def launches_per_step(progs, shots, binfo):
    """Kernel launches one replay of the batch graph makes: one per program in
    the one-launch-per-program form; otherwise one persistent launch per group
    (programs without and with bit-sliced tables)."""
    live = [p for p, n in zip(progs, shots) if n > 0]
    if binfo.get("form", 0) == 1:
        return len(live)
    sliced = [any(p.device_table_layout(t)[0] == 2 for t in range(p.info["num_tables"])) for p in live]
    return int(any(sliced)) + int(not all(sliced))


def kernel_int_ops(prog):
    """Integer operations one shot needs in the fused sampling kernel, counted
    on the packed device tables it actually evaluates:
      noise:   ceil(C/4) Philox4x32-10 calls x 10 rounds x (2 wide multiplies
               + 2 three-input XORs) = 40 per call, plus one compare per channel;
      outputs: 3 per deterministic output outside runs, 6 per run of
               single-bit outputs (+4 per further 64 of its bits), 60 per
               Bernoulli decision;
      tables:  per distinct parity 2W+2 (AND, XOR, popcount, insert), per merged
               term 12 (+5 per factor: two bit extracts, index, lookup, add);
               bit-sliced tables: the lane-operations of one warp for its 32
               shots, as the library counts them, divided by 32."""
    i = prog.info
    C = i["num_channels"]
    W = next(p for p in (1, 2, 4, 8, 16, 32) if i["x_words"] <= p)
    ops = 40 * ((C + 3) // 4) + C
    entries, runs, run_outputs = prog.device_output_stats()
    ops += 3 * (i["num_outputs"] - i["num_random"] - run_outputs) + 60 * i["num_random"]
    ops += 6 * runs + 4 * (run_outputs // 64)  # a run: word extracts, shift, merge
    for t in range(i["num_tables"]):
        layout = prog.device_table_layout(t)
        if layout[0] == 2:  # bit-sliced: the library counts one warp's lane-operations for 32 shots
            ops += layout[4] / 32
            continue
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
    for k, p in enumerate(progs):
        out = p.sample_torch(shots_of(k), SEED, 0)
        out = p.sample_torch(shots_of(k), SEED, 0)
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
