"""Bit-sliced warp-cooperative table layout: records must not depend on the
device layout of the marginal tables.  Every program is sampled with the
default layout, with the bit-sliced layout forced on every table that
qualifies, and with it disabled; the three record sets must be identical bit
for bit, and the forced-sliced records must equal the oracle's.  Launch sizes
are ragged (not a multiple of the 32 shots a warp evaluates together) and
cross 2^32 in the global shot index."""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram
from tests.test_compile_semantics import PHASED_CHAIN, STEANE_CHECK, WORKED_EXAMPLE, _random_circuit

pytestmark = pytest.mark.gpu


def _records(prog, shots, seed, offset):
    out = prog.sample_torch(shots, seed, offset)
    T.tsim_sync()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _layouts(prog):
    return [prog.device_table_layout(t)[0] for t in range(prog.info["num_tables"])]


def _check_layouts(tmp_path, prog, shots, seed, offset, oracle_shots):
    ref = _records(prog, shots, seed, offset)
    prog.set_table_layout(1, 128)  # rows staged through shared memory by bulk copies
    forced = _layouts(prog)
    sl = _records(prog, shots, seed, offset)
    prog.set_table_layout(1, 0)  # rows read through L1
    _same(_records(prog, shots, seed, offset), sl)
    prog.set_table_layout(-1)
    assert T.TABLE_SLICED not in _layouts(prog)
    off = _records(prog, shots, seed, offset)
    _same(sl, ref)
    _same(off, ref)
    prog.set_table_layout(1)
    path = str(tmp_path / "p.prog")
    prog.save(path)
    o = OracleProgram(path).sample(seed, offset, oracle_shots)
    for k in ("det", "obs", "meas"):
        if k in sl and o.get(k) is not None and sl[k].size:
            np.testing.assert_array_equal(sl[k][:oracle_shots].view(np.uint64), o[k], err_msg=k)
    np.testing.assert_array_equal(sl["accept"][:oracle_shots], o["accept"])
    return forced


SMALL = [
    ("worked_det", WORKED_EXAMPLE, T.MODE_DETECTORS),
    ("worked_meas", WORKED_EXAMPLE, T.MODE_MEASUREMENTS),
    ("cfg1", Wk.config1_circuit(), T.MODE_DETECTORS),
    ("cfg1_meas", Wk.config1_circuit(p=2e-3), T.MODE_MEASUREMENTS),
    ("steane_check", STEANE_CHECK, T.MODE_DETECTORS),
    ("phased_chain", PHASED_CHAIN, T.MODE_DETECTORS),
]


@pytest.mark.parametrize("name,text,mode", SMALL, ids=[c[0] for c in SMALL])
def test_small_programs_every_layout(tmp_path, name, text, mode):
    prog = T.Program(text, mode=mode)
    _check_layouts(tmp_path, prog, 3001, 17, (1 << 32) - 1000, 3001)


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_every_layout(tmp_path, seed):
    rng = random.Random(9100 + seed)
    text = _random_circuit(rng, 5, 30, tcount=8)
    mode = T.MODE_MEASUREMENTS if seed % 2 else T.MODE_DETECTORS
    if mode == T.MODE_DETECTORS:
        text += "\nDETECTOR rec[-1] rec[-2]\nDETECTOR rec[-3]\nOBSERVABLE_INCLUDE(0) rec[-1]\nOBSERVABLE_INCLUDE(1) rec[-2]"
    prog = T.Program(text, mode=mode)
    _check_layouts(tmp_path, prog, 1537, seed, seed * 7919, 1537)


@pytest.mark.parametrize("k", range(4))
def test_random_clifford_t_many_terms(tmp_path, k):
    # mirror circuits with 16-32 T gates: marginals of hundreds of terms
    txt = Wk.random_clifford_t(300 + k, n=20 + 4 * k, depth=30, t_count=16 + 4 * k)
    try:
        prog = T.Program(txt, chi_budget=4096)
    except T.TsimError as e:
        if e.code == 3:
            pytest.skip("over the term budget")
        raise
    forced = _check_layouts(tmp_path, prog, 4099, 5, 1 << 33, 700)
    assert T.TABLE_SLICED in forced or prog.info["max_terms"] < 2


def test_color_code_default_layout_is_sliced(tmp_path):
    # the 16383-term colour-code program: its marginals of 4 terms or more
    # take the sliced layout by default; 97 shots (a ragged warp) checked against the oracle,
    # records identical with the layout disabled
    prog = T.Program(Wk.config3_circuit())
    path = str(tmp_path / "c3.prog")
    prog.save(path)
    shots, seed, offset = 97, 21, (1 << 32) - 40
    g = _records(prog, shots, seed, offset)
    o = OracleProgram(path).sample(seed, offset, shots)
    np.testing.assert_array_equal(g["det"].view(np.uint64), o["det"])
    np.testing.assert_array_equal(g["obs"].view(np.uint64), o["obs"])
    np.testing.assert_array_equal(g["accept"], o["accept"])
    big = _records(prog, 20000, 3, 0)
    for layout in ((4, 128, 2048), (64, 0, 512), (4, 0, 16384), (-1,)):
        prog.set_table_layout(*layout)
        _same(_records(prog, 20000, 3, 0), big)


def test_batch_with_sliced_programs():
    progs = []
    for k in range(6):
        txt = Wk.random_clifford_t(400 + k, n=20 + 2 * k, depth=24, t_count=12 + 2 * k)
        try:
            p = T.Program(txt, chi_budget=2048)
        except T.TsimError as e:
            if e.code == 3:
                continue
            raise
        p.set_table_layout(1 if k % 2 else 4)
        progs.append(p)
    progs.append(T.Program(Wk.config1_circuit()))
    w = T.Program(WORKED_EXAMPLE, mode=T.MODE_MEASUREMENTS)
    w.set_table_layout(1)
    progs.append(w)
    rng = np.random.default_rng(8)
    shots = [int(x) for x in rng.integers(1, 5000, size=len(progs))]
    seeds = [int(x) for x in rng.integers(0, 2**63, size=len(progs))]
    offs = [int(x) for x in rng.integers(0, 2**40, size=len(progs))]

    def bufs(p, n):
        i = p.info
        meas = (torch.zeros((n, i["meas_words"]), dtype=torch.int64, device="cuda")
                if i["mode"] == T.MODE_MEASUREMENTS and i["meas_words"] else None)
        det = torch.zeros((n, i["det_words"]), dtype=torch.int64, device="cuda") if i["det_words"] else None
        obs = torch.zeros((n, i["obs_words"]), dtype=torch.int64, device="cuda") if i["obs_words"] else None
        return meas, det, obs, torch.zeros((n,), dtype=torch.uint8, device="cuda")

    want, got = [], []
    for p, n, sd, of in zip(progs, shots, seeds, offs):
        b = bufs(p, n)
        T.tsim_sample(p.h, n, sd, of, *b)
        want.append(b)
        got.append(bufs(p, n))
    T.tsim_sync()
    T.tsim_sample_batch([p.h for p in progs], shots, seeds, offs, [g[0] for g in got], [g[1] for g in got],
                        [g[2] for g in got], [g[3] for g in got])
    T.tsim_sync()
    for a, b in zip(want, got):
        for x, y in zip(a, b):
            if x is not None:
                assert torch.equal(x, y)
