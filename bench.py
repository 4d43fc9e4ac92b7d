"""Benchmark: shots/s and Z[w] term-evals/s of the GB300 per-shot sampler,
learned + batched against the plain GPU form, at identical records.

Headline workload (the line's `value`): the batched launch -- 256 seeded
random noisy Clifford+T mirror circuits of uneven size (20-60 qubits, depth
20-100, 8-40 T/T_DAG, two-qubit density 0.3, depolarising p in U[1e-4,
3e-3]) with shot counts log-uniform in [1e3, 1e6].  One step = one pass of
the whole hot path (noise, f = T e, detectors, exact marginals, Algorithm 1,
records) over every shot of every program.

Two forms are timed on the same GPU and must write identical records:
  value  learned + batched: programs compiled with the learned cut order (the
         committed network weights; heuristic order when they are absent),
         all programs in persistent launches replayed from a CUDA graph, the
         launch shapes picked by the autotuner;
  plain  heuristic cut order, one tsim_sample launch per program.

The same line reports, each with its own timing, roofline and CPU baseline,
the d=5 surface code with two injected logical rotations (3 x 10^6 shots),
the same circuit sampled in measurement mode (every record, long
autoregressive chains), the d=3 colour-code T-check (10^7 shots, the
term-evaluation workload) and the learned-cut-order workload (32 held-out
circuits of the network's training family, 34-46 T/T_DAG, where the learned
order and the heuristic give different programs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--only cfg2|cfg2m|cfg3|cfg4|cfg5] [--profile]

Under torchrun (N > 1) every rank samples its own shot range of every
program (weak scaling, no collective on the data path); timings take the
maximum over ranks and rank 0 prints one JSON line.
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

SEED = 0
METRIC = "shots/sec and Z[w] term-evals/sec, learned+batched vs plain GPU form, bit-exact"
HEADLINE = "cfg4"
WORKLOADS = {
    "cfg2": "d=5 rotated surface code, 49 qubits, 5 rounds, 16 T/T_DAG (two injected logical rotations, the "
            "second by gate teleportation), p in {5e-4,1e-3,2e-3}, 1e6 shots per p",
    "cfg2m": "measurement sampling of the d=5 rotated surface code with two injected logical rotations "
             "(147 measurement records per shot, 37 drawn by Algorithm 1 in 4 chains), p in {5e-4,1e-3,2e-3}, "
             "1e6 shots per p",
    "cfg3": "d=3 triangular colour-code T-check, 19 qubits, 42 T/T_DAG, 3 check rounds, p=1e-3, postselected, "
            "1e7 shots",
    "cfg4": "batched launch: 256 seeded random noisy Clifford+T mirror circuits (20-60 qubits, depth 20-100, "
            "8-40 T/T_DAG, 2-qubit density 0.3, p in U[1e-4,3e-3]), shots log-uniform in [1e3,1e6], "
            "persistent launches replayed from a CUDA graph, autotuned shot block and residency",
    "cfg5": "learned cut order against the heuristic: 32 seeded random Clifford+T circuits of the network's "
            "training family held out from training (3-10 qubits, 34-46 T/T_DAG, CX density 0.4, DEPOLARIZE1 "
            "1e-3 per layer), the first that compile within 8192 terms per marginal and 32768 per program, "
            "measurement sampling, 1e5 shots each",
}
CFG2_P = (5e-4, 1e-3, 2e-3)
CFG4_TABLE_BUDGET = 2048     # terms per marginal table
CFG4_PROGRAM_BUDGET = 8192   # terms per program
CFG5_PROGRAMS = 32
CFG5_T_RANGE = (34, 46)
CFG5_TABLE_BUDGET = 8192     # terms per marginal table
CFG5_PROGRAM_BUDGET = 32768  # terms per program
H2D_NOTE = ("0: a sampling step has no per-step input beyond scalars (seed, shot offset); each program's "
            "tables are uploaded once, before the timed region")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=6.0, help="bound on each oracle baseline's CPU work")
    ap.add_argument("--only", default=None, choices=sorted(WORKLOADS), help="one workload (it becomes the value)")
    ap.add_argument("--profile", action="store_true", help="only two plain launches per program (for ncu)")
    ap.add_argument("--profile-scale", type=float, default=1.0,
                    help="--profile: each program's shots times this factor (at least 32)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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


# ------------------------------------------------------------------ workloads
def cut_model():
    """The committed cut-order network weights, or None."""
    from paper_2604_01059_gb300.train_cut_order import load_weights
    return load_weights()


def config4_programs(n=256, decomp=0, texts=None):
    """The batched workload, compiled in parallel host threads.  Circuits over
    the term budgets are skipped and the next seeds drawn (deterministic
    order); `texts` recompiles a chosen list.  Returns (program, shots, text)."""
    from paper_2604_01059_gb300 import workloads as Wk
    pool = Wk.config4_batch(n=4 * n, seed=0) if texts is None else texts
    return select_programs(pool, n, CFG4_TABLE_BUDGET, CFG4_PROGRAM_BUDGET, 0, decomp)


def config5_programs(n=CFG5_PROGRAMS):
    """The learned-cut-order workload: the first n circuits of the seeded pool
    (training-family circuits, 34-46 T/T_DAG) that compile within the term
    budgets in the heuristic order, measurement mode."""
    import paper_2604_01059_gb300 as T
    from paper_2604_01059_gb300 import workloads as Wk
    pool = Wk.config5_pool(8 * n, t_range=CFG5_T_RANGE)
    return select_programs(pool, n, CFG5_TABLE_BUDGET, CFG5_PROGRAM_BUDGET, T.MODE_MEASUREMENTS, 0)


def select_programs(pool, n, chi_budget, total_budget, mode, decomp):
    """The first n (circuit, shots) items of the pool whose programs fit the
    term budgets, compiled in parallel host threads.  Returns (program, shots,
    text) triples in pool order."""
    from concurrent.futures import ThreadPoolExecutor

    import paper_2604_01059_gb300 as T

    def build(item):
        txt, shots = item
        try:
            p = T.Program(txt, chi_budget=chi_budget, total_budget=total_budget, decomp=decomp, mode=mode)
        except T.TsimError as e:
            if e.code == 3:
                return None
            raise
        return (p, shots, txt) if p.info["total_terms"] <= total_budget else None

    # a sliding window of compilations in pool order: results are taken in
    # order (the first n that fit the budgets), while a slow circuit does not
    # hold up the ones behind it
    out = []
    workers = os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs, nxt = [], 0
        while len(out) < n and (futs or nxt < len(pool)):
            while nxt < len(pool) and len(futs) < 4 * workers:
                futs.append(ex.submit(build, pool[nxt]))
                nxt += 1
            r = futs.pop(0).result()
            if r is not None:
                out.append(r)
        for f in futs:
            f.cancel()
    return out


class Workload:
    """The programs of one configuration, in the plain (heuristic) and the
    learned cut order, and their shot counts."""

    def __init__(self, name):
        import paper_2604_01059_gb300 as T
        from paper_2604_01059_gb300 import workloads as Wk
        self.name = name
        t0 = time.perf_counter()
        if name in ("cfg4", "cfg5"):
            pr = config4_programs() if name == "cfg4" else config5_programs()
            self.plain = [p for p, _, _ in pr]
            self.shots = [s for _, s, _ in pr]
            self.texts = [(t, s) for _, s, t in pr]
        elif name == "cfg3":
            self.texts = [(Wk.config3_circuit(p=1e-3), 10_000_000)]
        else:
            self.texts = [(Wk.config2_circuit(p=p), 1_000_000) for p in CFG2_P]
        self.mode = T.MODE_MEASUREMENTS if name in ("cfg2m", "cfg5") else T.MODE_DETECTORS
        if name not in ("cfg4", "cfg5"):
            self.plain = [T.Program(t, mode=self.mode) for t, _ in self.texts]
            self.shots = [s for _, s in self.texts]
        self.compile_s = {"heuristic": time.perf_counter() - t0}
        t0 = time.perf_counter()
        self.learned, self.cut = self._learned()
        self.compile_s["learned"] = time.perf_counter() - t0

    def _compile(self, decomp):
        """Compile the workload's circuits in parallel host threads, each with
        this rank's GPU current (the cut-order network scores on it)."""
        from concurrent.futures import ThreadPoolExecutor

        import torch

        import paper_2604_01059_gb300 as T
        dev = torch.cuda.current_device() if torch.cuda.is_available() else None

        def one(t):
            if self.name == "cfg4":
                return T.Program(t, chi_budget=CFG4_TABLE_BUDGET, total_budget=CFG4_PROGRAM_BUDGET, decomp=decomp)
            if self.name == "cfg5":
                return T.Program(t, chi_budget=CFG5_TABLE_BUDGET, total_budget=CFG5_PROGRAM_BUDGET, decomp=decomp,
                                 mode=self.mode)
            return T.Program(t, decomp=decomp, mode=self.mode)

        init = (lambda: torch.cuda.set_device(dev)) if dev is not None else None
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1, initializer=init) as ex:
            return list(ex.map(one, [t for t, _ in self.texts]))

    def _learned(self):
        import paper_2604_01059_gb300 as T
        w = cut_model()
        if w is None:
            return self._compile(T.DECOMP_HEURISTIC), {"cut_order": "heuristic (no trained weights)"}
        before = T.tsim_cut_policy_stats()
        T.tsim_cut_model_set(w)
        try:
            progs = self._compile(T.DECOMP_LEARNED)
        finally:
            T.tsim_cut_model_set(None)
        d = [a - b for a, b in zip(T.tsim_cut_policy_stats(), before)]
        return progs, {"cut_order": "learned (GNN scores, heuristic as fallback and judge)", "scorer_calls": d[0],
                       "scored": d[1], "marginals_learned_kept": d[2], "marginals_heuristic_kept": d[3]}


# ------------------------------------------------------------------ counting
def device_terms_per_shot(prog):
    """Terms the device evaluates for one shot: every table a shot evaluates
    (each chain's normalisation and one table per random output), counted
    after terms with equal factor lists are merged into one class (the
    kernel evaluates each class once)."""
    return sum(prog.device_table_stats(t)[0] for t in range(prog.info["num_tables"]))


def premerge_terms_per_shot(prog):
    """Stabilizer terms of the same tables before merging."""
    return sum(prog.table_terms())


def kernel_int_ops(prog, padded=False):
    """Integer operations one shot needs in the fused sampling kernel, counted
    on the packed device tables it evaluates:
      noise, one word per channel: ceil(C/4) Philox4x32-10 calls x 10 rounds x
               (2 wide multiplies + 2 three-input XORs) = 40 per call, plus one
               compare per channel;
      noise, geometric gaps: 10 per word (a quarter Philox call) + 4 (compare,
               table load, branch) for its expected words, + 12 per expected
               candidate (map, threshold walk, signature XOR);
      outputs: 3 per deterministic output outside runs, 6 per run of
               single-bit outputs (+4 per further 64 of its bits), 60 per
               Bernoulli decision;
      tables:  per distinct parity 2W+2 (AND, XOR, popcount, insert), per merged
               term 12 (+5 per factor: two bit extracts, index, lookup, add);
               bit-sliced tables: the lane-operations of one warp for its 32
               shots, as the library counts them, divided by 32: without
               padding (each term's own rows, one batch epilogue per term),
               or with it (padded=True: every row and lane the kernel runs)."""
    i = prog.info
    C = i["num_channels"]
    W = next(p for p in (1, 2, 4, 8, 16, 32) if i["x_words"] <= p)
    nz = prog.noise_info()
    if nz["mode"] == 1:
        words = nz["words_geometric_mode"]
        cand = max(0.0, (words - nz["groups"]) / 2)
        ops = 14 * words + 12 * cand
    else:
        ops = 40 * ((C + 3) // 4) + C
    entries, runs, run_outputs = prog.device_output_stats()
    ops += 3 * (i["num_outputs"] - i["num_random"] - run_outputs) + 60 * i["num_random"]
    ops += 6 * runs + 4 * (run_outputs // 64)
    for t in range(i["num_tables"]):
        layout = prog.device_table_layout(t)
        if layout[0] == 2:
            ops += (layout[4] if padded else layout[5]) / 32
            continue
        classes, factors, parities = prog.device_table_stats(t)
        ops += parities * (2 * W + 2) + 12 * classes + 5 * factors
    return ops


def int_peak(sm_mhz=None):
    """Integer-issue peak of the current GPU: SMs (read from the device) x 4
    sub-partitions x 16 INT32 lanes x the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk = sm_mhz or measured_peaks().get("sm_max_mhz") or 2070.0
    return sms * 4 * 16 * clk * 1e6, sms, clk


def int_peaks_measured():
    import paper_2604_01059_gb300 as T
    names = ["lop3", "imad", "imad_wide", "popc"]
    return {n: T.tsim_measure_int_peak(k) / 1e12 for k, n in enumerate(names)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def launches_per_step(progs, shots, binfo):
    """Kernel launches one replay of the batch graph makes: one per program in
    the one-launch-per-program form; otherwise one persistent launch per group
    (programs without and with bit-sliced tables, by X width)."""
    live = [p for p, n in zip(progs, shots) if n > 0]
    if binfo.get("form", 0) == 1:
        return len(live)
    groups = {(any(p.device_table_layout(t)[0] == 2 for t in range(p.info["num_tables"])),
               next(w for w in (1, 2, 4, 8, 16, 32) if p.info["x_words"] <= w)) for p in live}
    return len(groups)


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


# ------------------------------------------------------------- CPU baseline
class OracleBench:
    """The oracle's C evaluator on the host cores, on the programs of the
    workload (at most 16 of them, spread over the list): calibrated once on
    one thread, then timed on bounded samples on every core."""

    def __init__(self, progs):
        import tempfile

        from oracle import evaluator

        evaluator.build()
        self.cores = os.cpu_count() or 1
        tmp = tempfile.mkdtemp()
        self.orcs = []
        step = max(1, len(progs) // 16)
        for k, p in enumerate(progs[::step][:16]):
            path = os.path.join(tmp, f"w{k}.prog")
            p.save(path)
            self.orcs.append(evaluator.OracleProgram(path))
        n_cal = 1
        while True:  # per-shot time of one thread
            t0 = time.perf_counter()
            for o in self.orcs:
                o.sample(SEED, 0, n_cal)
            dt = time.perf_counter() - t0
            if dt > 0.5 or n_cal >= 4096:
                break
            n_cal *= 4
        self.per_shot = dt / (n_cal * len(self.orcs))
        self.cal_shots = n_cal * len(self.orcs)

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
                "value_1thread": 1.0 / self.per_shot,
                "sample": f"{shots} shots ({chunk} per thread x {self.cores} threads x {len(self.orcs)} programs) "
                          f"of the same workload, oracle C evaluator, exact arithmetic; value_1thread: one thread "
                          f"on {self.cal_shots} shots"}


# ------------------------------------------------------------------ GPU arm
def _outputs(progs, shots):
    """Device record buffers per program: (det, obs, accept, meas or None)."""
    import torch
    outs = []
    for p, ns in zip(progs, shots):
        i = p.info
        meas = (torch.empty((ns, i["meas_words"]), dtype=torch.int64, device="cuda")
                if i["mode"] == 1 and i["meas_words"] else None)
        outs.append((torch.empty((ns, max(i["det_words"], 1)), dtype=torch.int64, device="cuda"),
                     torch.empty((ns, max(i["obs_words"], 1)), dtype=torch.int64, device="cuda"),
                     torch.empty((ns,), dtype=torch.uint8, device="cuda"), meas))
    return outs


def bench_config(wl, steps, args, dist, rank, world, flush, clocks_index):
    """Time one workload in both forms; returns its result dictionary."""
    import numpy as np
    import torch

    import paper_2604_01059_gb300 as T

    progs, plain_progs, shots = wl.learned, wl.plain, wl.shots
    n = len(progs)
    offsets = shard_offsets(rank, shots)
    seeds = [SEED] * n
    stream = torch.cuda.current_stream()
    outs = _outputs(progs, shots)
    plain_outs = _outputs(plain_progs, shots)

    def plain_step():
        for k, (p, (d, o, a, m)) in enumerate(zip(plain_progs, plain_outs)):
            T.tsim_sample(p.h, shots[k], seeds[k], offsets[k], m, d, o, a, stream)

    meas_list = [o[3] for o in outs] if any(o[3] is not None for o in outs) else None
    batch = T.tsim_batch_create([p.h for p in progs], shots, seeds, offsets, meas_list,
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

    def timed(step_fn):
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

    # where the learned order changed programs: the learned programs in the
    # plain form too, to separate the two effects
    differs = any(premerge_terms_per_shot(a) != premerge_terms_per_shot(b) for a, b in zip(progs, plain_progs))
    lp_outs = _outputs(progs, shots) if differs else None

    def learned_plain_step():
        for k, (p, (d, o, a, m)) in enumerate(zip(progs, lp_outs)):
            T.tsim_sample(p.h, shots[k], seeds[k], offsets[k], m, d, o, a, stream)

    if differs:
        for _ in range(max(args.warmup, 3)):
            learned_plain_step()
    clocks = ClockSampler(clocks_index)
    clocks.start()
    batch_ms = timed(batch_step)
    plain_ms = timed(plain_step)
    lp_ms = timed(learned_plain_step) if differs else None
    clk = clocks.stop()
    T.tsim_batch_free(batch)
    def same(set1, set2):
        return all(torch.equal(a[:, :p.info["det_words"]], b[:, :p.info["det_words"]]) and
                   torch.equal(x[:, :p.info["obs_words"]], y[:, :p.info["obs_words"]]) and torch.equal(u, v) and
                   (m1 is None or torch.equal(m1, m2))
                   for p, (a, x, u, m1), (b, y, v, m2) in zip(progs, set1, set2))

    identical = same(outs, plain_outs) and (lp_outs is None or same(lp_outs, plain_outs))
    del outs, plain_outs, lp_outs
    shots_step = sum(shots) * world
    value = shots_step * steps / (batch_ms / 1e3)
    plain = shots_step * steps / (plain_ms / 1e3)
    dev_terms = sum(device_terms_per_shot(p) * ns for p, ns in zip(progs, shots)) * world
    pre_terms = sum(premerge_terms_per_shot(p) * ns for p, ns in zip(progs, shots)) * world
    plain_dev_terms = sum(device_terms_per_shot(p) * ns for p, ns in zip(plain_progs, shots)) * world

    # end to end through the host-buffer entry point: copies inside the timed
    # region, into page-locked host buffers
    def pinned(shape, dtype):
        return torch.zeros(shape, dtype=dtype, pin_memory=True).numpy()

    hbuf = []
    for p, ns in zip(progs, shots):
        i = p.info
        hbuf.append((pinned((ns, max(i["det_words"], 1)), torch.int64).view(np.uint64),
                     pinned((ns, max(i["obs_words"], 1)), torch.int64).view(np.uint64), pinned((ns,), torch.uint8),
                     pinned((ns, i["meas_words"]), torch.int64).view(np.uint64)
                     if i["mode"] == 1 and i["meas_words"] else None))

    def e2e_step():
        for k, p in enumerate(progs):
            i = p.info
            d, o, a, m = hbuf[k]
            T.tsim_sample_host(p.h, shots[k], seeds[k], offsets[k], m, d if i["det_words"] else None,
                               o if i["obs_words"] else None, a, stream)

    e2e_step()
    e2e_steps = max(1, min(steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = shots_step * e2e_steps / e2e_s
    d2h = sum(ns * (p.info["det_words"] * 8 + p.info["obs_words"] * 8 + 1 +
                    (p.info["meas_words"] * 8 if p.info["mode"] == 1 else 0)) for p, ns in zip(progs, shots))
    del hbuf

    # roofline of the dominant kernel (the batched launch's kernels)
    ops = sum(kernel_int_ops(p) * ns for p, ns in zip(progs, shots))
    ops_padded = sum(kernel_int_ops(p, padded=True) * ns for p, ns in zip(progs, shots))
    peak, sms, clk_mhz = int_peak()
    achieved = ops / (batch_ms / steps / 1e3)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": ("k_batch (persistent kernels over all programs, graph replay)" if binfo.get("form", 0) == 0
                       else "k_sample (each program's launch, graph replay)"),
            "ops_per_shot": ops / sum(shots),
            "ops_note": "algorithmic integer operations without padding (bit-sliced rows of each term's own "
                        "factors, one batch epilogue per term)",
            "ops_per_shot_padded": ops_padded / sum(shots),
            "frac_padded": ops_padded / (batch_ms / steps / 1e3) / peak,
            "peak_source": f"derived: {sms} SMs (from the device) x 4 sub-partitions x 16 INT32 lanes x "
                           f"{clk_mhz:.0f} MHz (maximum SM clock)"}
    base = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        base = OracleBench(progs).run(args.cpu_seconds)
    noise = [p.noise_info() for p in progs]
    return {
        "workload": WORKLOADS[wl.name], "value": value, "unit": "shots/s", "ms_per_step": batch_ms / steps,
        "steps": steps, "programs": n, "shots_per_step": shots_step,
        "term_evals_per_s": dev_terms * steps / (batch_ms / 1e3),
        "term_evals_note": "terms the device evaluates: every table of a shot, terms with equal factor lists "
                           "merged into one class",
        "premerge_term_evals_per_s": pre_terms * steps / (batch_ms / 1e3),
        "device_terms_per_shot": dev_terms / max(shots_step, 1),
        "premerge_terms_per_shot": pre_terms / max(shots_step, 1),
        "terms_all_programs": {"learned": sum(premerge_terms_per_shot(p) for p in progs),
                               "heuristic": sum(premerge_terms_per_shot(p) for p in plain_progs)},
        "identical_records": bool(identical),
        "plain": {"value": plain, "unit": "shots/s", "ms_per_step": plain_ms / steps,
                  "term_evals_per_s": plain_dev_terms * steps / (plain_ms / 1e3),
                  "form": "heuristic cut order, one tsim_sample launch per program",
                  "gpu_launches": steps * sum(1 for s in shots if s > 0)},
        "speedup_vs_plain": value / plain,
        "learned_plain": None if lp_ms is None else {
            "value": shots_step * steps / (lp_ms / 1e3), "unit": "shots/s", "ms_per_step": lp_ms / steps,
            "form": "learned cut order, one tsim_sample launch per program",
            "speedup_vs_plain": plain_ms / lp_ms},
        "form": "learned cut order + batched launch (CUDA graph, autotuned)", "batch": binfo, "cut": wl.cut,
        "noise_sampling": {"geometric_programs": sum(1 for z in noise if z["mode"] == 1),
                           "words_per_shot": sum((z["words_geometric_mode"] if z["mode"] == 1 else
                                                  z["words_per_channel_mode"]) * ns
                                                 for z, ns in zip(noise, shots)) / sum(shots)},
        "compile_s": wl.compile_s,
        "e2e": {"value": e2e, "unit": "shots/s", "h2d_bytes_per_step": 0, "h2d_note": H2D_NOTE,
                "d2h_bytes_per_step": d2h,
                "api": "tsim_sample_host (device staging, records copied to page-locked host memory inside the "
                       "timed region)"},
        "gpu_launches": steps * launches_per_step(progs, shots, binfo),
        "roofline": roof, "clocks": clk, "cpu_baseline": base,
    }


def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    clocks_index = ids[local] if local < len(ids) else str(local)
    head = args.only or HEADLINE
    names = [head] + ([] if args.only else [k for k in ("cfg2", "cfg2m", "cfg3", "cfg5") if k != head])
    res = {}
    for name in names:
        wl = Workload(name)
        steps = args.steps if name == head else (min(args.steps, 5) if name == "cfg3" else args.steps)
        res[name] = bench_config(wl, steps, args, dist, rank, world, flush, clocks_index)
        del wl
    h = res[head]
    if rank == 0:
        line = {"metric": METRIC, "value": h["value"], "unit": "shots/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": h["workload"], "l2": "flushed between timed steps (256 MiB write)",
                           "programs": h["programs"], "shots_per_step": h["shots_per_step"],
                           "form": h["form"], "cut": h["cut"], "batch": h["batch"],
                           "terms_all_programs": h["terms_all_programs"], "noise_sampling": h["noise_sampling"],
                           "compile_s": h["compile_s"]},
                "term_evals_per_s": h["term_evals_per_s"], "term_evals_note": h["term_evals_note"],
                "premerge_term_evals_per_s": h["premerge_term_evals_per_s"],
                "identical_records": h["identical_records"], "plain": h["plain"],
                "speedup_vs_plain": h["speedup_vs_plain"], "e2e": h["e2e"], "gpu_launches": h["gpu_launches"],
                "roofline": h["roofline"], "clocks": h["clocks"], "cpu_baseline": h["cpu_baseline"],
                "measured_issue_tops": int_peaks_measured(),
                "configs": {k: v for k, v in res.items() if k != head}}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The reference arm: the oracle (plain C, exact) on the host cores, on the
    headline workload's programs, each step a bounded sample of it (the whole
    run about --cpu-seconds of oracle work plus one calibration)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    head = args.only or HEADLINE
    if head == "cfg4":
        progs = [p for p, _, _ in config4_programs()]
    else:
        import paper_2604_01059_gb300 as T
        from paper_2604_01059_gb300 import workloads as Wk
        progs = ([T.Program(Wk.config3_circuit(p=1e-3))] if head == "cfg3"
                 else [T.Program(Wk.config2_circuit(p=p), mode=1 if head == "cfg2m" else 0) for p in CFG2_P])
    ob = OracleBench(progs)
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
            "config": {"workload": WORKLOADS[head]},
            "cpu_baseline": {"kind": "oracle", "cores": b["cores"], "sample": b["sample"] + " (per step)",
                             "value": val, "value_1thread": b["value_1thread"]},
            "e2e": {"value": val, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(args):
    """For a profiler: two launches of one workload and nothing else -- each
    program's own sampling kernel twice (configs 2 and 3), or the batched
    workload's persistent launches twice (config 4, default launch shape,
    no autotuning runs)."""
    import torch

    import paper_2604_01059_gb300 as T
    name = args.only or "cfg2"

    def scaled(n):
        return max(32, int(round(n * args.profile_scale)))

    if name == "cfg4":
        pr = config4_programs()
        progs, shots = [p for p, _, _ in pr], [scaled(s) for _, s, _ in pr]
        outs = _outputs(progs, shots)
        batch = T.tsim_batch_create([p.h for p in progs], shots, [SEED] * len(progs), None, None,
                                    [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs], autotune=0)
        try:
            for _ in range(2):
                T.tsim_batch_launch(batch)
            T.tsim_sync()
        finally:
            T.tsim_batch_free(batch)
    else:
        wl = Workload(name)
        progs = wl.plain
        for p, ns in zip(wl.plain, wl.shots):
            p.sample_torch(scaled(ns), SEED, 0)
            p.sample_torch(scaled(ns), SEED, 0)
        T.tsim_sync()
    torch.cuda.synchronize()
    print(json.dumps({"profile": WORKLOADS[name], "programs": len(progs), "shots_scale": args.profile_scale}))


def main():
    args = parse()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
