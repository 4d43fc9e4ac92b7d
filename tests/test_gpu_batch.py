"""Batched launch: one persistent kernel over many programs (uneven sizes and
shot counts), replayed from a captured CUDA graph, must write exactly the
records that per-program launches write (which the other GPU tests tie to the
oracle bit for bit); a few programs are also checked against the oracle
directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram
from tests.test_compile_semantics import WORKED_EXAMPLE

pytestmark = pytest.mark.gpu


def _programs(count=12, budget=1024):
    progs, k = [], 0
    while len(progs) < count:
        txt = Wk.random_clifford_t(7000 + k, n=20 + (k % 5) * 4, depth=20 + (k % 7) * 6, t_count=8 + k % 9)
        k += 1
        try:
            progs.append(T.Program(txt, chi_budget=budget))
        except T.TsimError as e:
            if e.code != 3:
                raise
    progs.append(T.Program(Wk.config1_circuit()))
    progs.append(T.Program(WORKED_EXAMPLE, mode=T.MODE_MEASUREMENTS))
    return progs


def _bufs(p, shots):
    i = p.info
    meas = (torch.zeros((shots, i["meas_words"]), dtype=torch.int64, device="cuda")
            if i["mode"] == T.MODE_MEASUREMENTS and i["meas_words"] else None)
    det = torch.zeros((shots, i["det_words"]), dtype=torch.int64, device="cuda") if i["det_words"] else None
    obs = torch.zeros((shots, i["obs_words"]), dtype=torch.int64, device="cuda") if i["obs_words"] else None
    acc = torch.zeros((shots,), dtype=torch.uint8, device="cuda")
    return meas, det, obs, acc


def _np(bufs):
    return [None if t is None else t.cpu().numpy() for t in bufs]


@pytest.mark.parametrize("autotune", [0, 1, 2])  # persistent, autotuned, one launch per program
def test_batch_matches_single_launches(tmp_path, autotune):
    progs = _programs()
    rng = np.random.default_rng(5)
    shots = [int(x) for x in rng.integers(1, 20000, size=len(progs))]
    shots[0] = 1
    seeds = [int(x) for x in rng.integers(0, 2**63, size=len(progs))]
    offs = [int(x) for x in rng.integers(0, 2**40, size=len(progs))]
    want, got = [], []
    for p, n, sd, of in zip(progs, shots, seeds, offs):
        b = _bufs(p, n)
        T.tsim_sample(p.h, n, sd, of, *b)
        want.append(b)
        got.append(_bufs(p, n))
    T.tsim_sync()
    cols = list(zip(*got))
    batch = T.tsim_batch_create([p.h for p in progs], shots, seeds, offs, *[list(c) for c in cols],
                                autotune=autotune)
    try:
        info = T.tsim_batch_info(batch)
        assert info["graph"] == 1 and info["work_items"] >= len(progs)
        assert info["form"] == {0: 0, 2: 1}.get(autotune, info["form"]) and info["form"] in (0, 1)
        for rep in range(2):  # graph replay: the same records every time
            for b in got:
                for t in b:
                    if t is not None:
                        t.zero_()
            T.tsim_batch_launch(batch)
            T.tsim_sync()
            for w, g in zip(want, got):
                for a, c in zip(_np(w), _np(g)):
                    if a is not None:
                        np.testing.assert_array_equal(a, c)
    finally:
        T.tsim_batch_free(batch)
    # direct oracle check of every member, the random programs included: the
    # first 256 shots of each and the last 64 (the ragged end of its items)
    for k in range(len(progs)):
        path = str(tmp_path / f"b{k}.prog")
        progs[k].save(path)
        orc = OracleProgram(path)
        g = _np(got[k])
        n = shots[k]
        for lo, hi in ((0, min(n, 256)), (max(0, n - 64), n)):
            o = orc.sample(seeds[k], offs[k] + lo, hi - lo)
            if g[0] is not None:
                np.testing.assert_array_equal(g[0][lo:hi].view(np.uint64), o["meas"])
            if g[1] is not None:
                np.testing.assert_array_equal(g[1][lo:hi].view(np.uint64), o["det"])
            if g[2] is not None:
                np.testing.assert_array_equal(g[2][lo:hi].view(np.uint64), o["obs"])
            np.testing.assert_array_equal(g[3][lo:hi], o["accept"])


def test_simple_batch_entry_point():
    progs = _programs(count=4)
    shots = [333, 1, 4097, 128, 50, 7]
    seeds = [1, 2, 3, 4, 5, 6]
    want = []
    for p, n, sd in zip(progs, shots, seeds):
        b = _bufs(p, n)
        T.tsim_sample(p.h, n, sd, 0, *b)
        want.append(_np(b))
    T.tsim_sync()
    got = [_bufs(p, n) for p, n in zip(progs, shots)]
    cols = list(zip(*got))
    T.tsim_sample_batch([p.h for p in progs], shots, seeds, None, *[list(c) for c in cols])
    for w, g in zip(want, got):
        for a, c in zip(w, _np(g)):
            if a is not None:
                np.testing.assert_array_equal(a, c)


def test_batch_of_large_sliced_programs():
    # few large programs (colour-code T-check twice, different seeds): the
    # autotuner may keep either launch form; records must equal plain launches
    progs = [T.Program(Wk.config3_circuit()) for _ in range(2)]
    shots, seeds, offs = [20000, 12345], [3, 4], [0, 1 << 32]
    want, got = [], []
    for p, n, sd, of in zip(progs, shots, seeds, offs):
        b = _bufs(p, n)
        T.tsim_sample(p.h, n, sd, of, *b)
        want.append(b)
        got.append(_bufs(p, n))
    T.tsim_sync()
    cols = list(zip(*got))
    for autotune in (1, 2, 0):
        batch = T.tsim_batch_create([p.h for p in progs], shots, seeds, offs, *[list(c) for c in cols],
                                    autotune=autotune)
        try:
            for b in got:
                for t in b:
                    if t is not None:
                        t.zero_()
            T.tsim_batch_launch(batch)
            T.tsim_sync()
            for w, g in zip(want, got):
                for a, c in zip(_np(w), _np(g)):
                    if a is not None:
                        np.testing.assert_array_equal(a, c)
        finally:
            T.tsim_batch_free(batch)
