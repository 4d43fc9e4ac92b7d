"""GPU parity: records from the sm_103a kernels must equal the oracle's
records bit for bit, given identical Philox streams (same program file, seed
and global shot indices).  Sizes span several thread blocks and a ragged
tail; the full-size workload is checked on shots sampled across the launch
that the benchmark times."""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram
from tests.test_compile_semantics import PHASED_CHAIN, REPETITION, STEANE_CHECK, WORKED_EXAMPLE, _random_circuit

pytestmark = pytest.mark.gpu


def _gpu(prog, shots, seed, offset):
    out = prog.sample_torch(shots, seed, offset)
    T.tsim_sync()
    res = {k: (v.cpu().numpy().view(np.uint64) if v is not None and v.dtype == torch.int64 else
               (v.cpu().numpy() if v is not None else None)) for k, v in out.items()}
    return res


def _compare(prog, path, shots, seed, offset):
    g = _gpu(prog, shots, seed, offset)
    o = OracleProgram(path).sample(seed, offset, shots)
    i = prog.info
    if i["det_words"]:
        np.testing.assert_array_equal(g["det"], o["det"])
    if i["obs_words"]:
        np.testing.assert_array_equal(g["obs"], o["obs"])
    if i["mode"] == T.MODE_MEASUREMENTS and i["meas_words"]:
        np.testing.assert_array_equal(g["meas"], o["meas"])
    np.testing.assert_array_equal(g["accept"], o["accept"])
    return g


CASES = [
    ("worked_det", WORKED_EXAMPLE, T.MODE_DETECTORS),
    ("worked_meas", WORKED_EXAMPLE, T.MODE_MEASUREMENTS),
    ("repetition", REPETITION, T.MODE_DETECTORS),
    ("cfg1", Wk.config1_circuit(), T.MODE_DETECTORS),
    ("cfg1_meas", Wk.config1_circuit(p=2e-3), T.MODE_MEASUREMENTS),
    ("steane_check", STEANE_CHECK, T.MODE_DETECTORS),
    ("phased_chain", PHASED_CHAIN, T.MODE_DETECTORS),
]


@pytest.mark.parametrize("noise", [0, 1])  # one word per channel / geometric gaps
@pytest.mark.parametrize("name,text,mode", CASES, ids=[c[0] for c in CASES])
def test_small_programs_bit_exact(tmp_path, name, text, mode, noise):
    prog = T.Program(text, mode=mode)
    prog.set_noise_sampling(noise)
    path = str(tmp_path / "p.prog")
    prog.save(path)
    _compare(prog, path, 3001, seed=11, offset=(1 << 32) - 1000)  # ragged, crosses 2^32


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_bit_exact(tmp_path, seed):
    rng = random.Random(5000 + seed)
    text = _random_circuit(rng, 4, 24, tcount=4)
    mode = T.MODE_MEASUREMENTS if seed % 2 else T.MODE_DETECTORS
    if mode == T.MODE_DETECTORS:
        text += "\nDETECTOR rec[-1] rec[-2]\nDETECTOR rec[-3]\nOBSERVABLE_INCLUDE(0) rec[-1]\nOBSERVABLE_INCLUDE(1) rec[-2]"
    prog = T.Program(text, mode=mode)
    prog.set_noise_sampling(seed % 3 == 0)
    path = str(tmp_path / "p.prog")
    prog.save(path)
    _compare(prog, path, 1537, seed=seed, offset=seed * 7919)


@pytest.mark.parametrize("p,noise", [(5e-4, 1), (1e-3, 1), (2e-3, 1), (2e-3, 0)])
def test_config2_full_size_sampled_shots(tmp_path, p, noise):
    # the benchmark's launch: 10^6 shots per p in one call; check 256 shots
    # spread over the whole launch against the oracle, one shot at a time
    prog = T.Program(Wk.config2_circuit(p=p))
    prog.set_noise_sampling(noise)
    path = str(tmp_path / "c2.prog")
    prog.save(path)
    shots, seed = 1_000_000, 0
    g = _gpu(prog, shots, seed, 0)
    orc = OracleProgram(path)
    rng = random.Random(int(p * 1e7))
    idx = sorted(set([0, shots - 1] + [rng.randrange(shots) for _ in range(254)]))
    for s in idx:
        o = orc.sample(seed, s, 1)
        np.testing.assert_array_equal(g["det"][s], o["det"][0])
        np.testing.assert_array_equal(g["obs"][s], o["obs"][0])
        assert g["accept"][s] == o["accept"][0]


@pytest.mark.parametrize("noise", [1, 0])
def test_config2_measurement_mode_full_size(tmp_path, noise):
    # measurement sampling of the benchmark circuit (147 records per shot, 37
    # drawn by Algorithm 1 in 4 chains: the long autoregressive chains that
    # detector sampling avoids): the full 10^6-shot launch, 256 shots spread
    # over it checked against the oracle one at a time, and a ragged block
    prog = T.Program(Wk.config2_circuit(p=2e-3), mode=T.MODE_MEASUREMENTS)
    prog.set_noise_sampling(noise)
    assert prog.info["num_random"] >= 30 and prog.info["num_chains"] >= 2
    path = str(tmp_path / "c2m.prog")
    prog.save(path)
    shots, seed = 1_000_000, 4
    g = _gpu(prog, shots, seed, 0)
    orc = OracleProgram(path)
    rng = random.Random(77 + noise)
    idx = sorted(set([0, shots - 1] + [rng.randrange(shots) for _ in range(254)]))
    for s in idx:
        o = orc.sample(seed, s, 1)
        np.testing.assert_array_equal(g["meas"][s], o["meas"][0])
        np.testing.assert_array_equal(g["det"][s], o["det"][0])
        np.testing.assert_array_equal(g["obs"][s], o["obs"][0])
        assert g["accept"][s] == o["accept"][0]
    _compare(prog, path, 1025, seed=seed + 1, offset=shots)


def test_config3_color_code_t_check(tmp_path):
    # 19 qubits, 42 T/T_DAG, 3 check rounds (16383 stabilizer terms; the
    # oracle needs ~0.3 s per shot): a ragged two-block launch checked shot
    # by shot, then 32 shots sampled from a 10^6-shot launch
    prog = T.Program(Wk.config3_circuit())
    path = str(tmp_path / "c3.prog")
    prog.save(path)
    _compare(prog, path, 129, seed=9, offset=123456)
    shots, seed = 1_000_000, 0
    g = _gpu(prog, shots, seed, 0)
    orc = OracleProgram(path)
    rng = random.Random(33)
    idx = sorted(set([0, shots - 1] + [rng.randrange(shots) for _ in range(30)]))
    for s in idx:
        o = orc.sample(seed, s, 1)
        np.testing.assert_array_equal(g["det"][s], o["det"][0])
        np.testing.assert_array_equal(g["obs"][s], o["obs"][0])
        assert g["accept"][s] == o["accept"][0]


def test_host_entry_point_matches_device(tmp_path):
    prog = T.Program(Wk.config1_circuit())
    shots = 777
    g = _gpu(prog, shots, 5, 100)
    i = prog.info
    det = np.zeros((shots, i["det_words"]), dtype=np.uint64)
    obs = np.zeros((shots, i["obs_words"]), dtype=np.uint64)
    acc = np.zeros(shots, dtype=np.uint8)
    T.tsim_sample_host(prog.h, shots, 5, 100, None, det, obs, acc)
    np.testing.assert_array_equal(det, g["det"])
    np.testing.assert_array_equal(obs, g["obs"])
    np.testing.assert_array_equal(acc, g["accept"])


@pytest.mark.parametrize("name,text,mode,shots", [
    ("cfg2", Wk.config2_circuit(p=2e-3), T.MODE_DETECTORS, 1_300_001),
    ("cfg1_meas", Wk.config1_circuit(p=2e-3), T.MODE_MEASUREMENTS, (1 << 20) + 3),
])
def test_host_entry_point_in_chunks(name, text, mode, shots):
    # more than 2^19 shots run in chunks whose copies overlap the sampling of
    # the next one (ragged last chunk): the records equal the device path's
    prog = T.Program(text, mode=mode)
    g = _gpu(prog, shots, 9, 12345)
    i = prog.info
    meas = np.zeros((shots, i["meas_words"]), dtype=np.uint64) if mode == T.MODE_MEASUREMENTS else None
    det = np.zeros((shots, i["det_words"]), dtype=np.uint64) if i["det_words"] else None
    obs = np.zeros((shots, i["obs_words"]), dtype=np.uint64) if i["obs_words"] else None
    acc = np.zeros(shots, dtype=np.uint8)
    for rep in range(2):  # the second call reuses the staging buffers
        T.tsim_sample_host(prog.h, shots, 9, 12345, meas, det, obs, acc)
        if meas is not None:
            np.testing.assert_array_equal(meas, g["meas"])
        if det is not None:
            np.testing.assert_array_equal(det, g["det"])
        if obs is not None:
            np.testing.assert_array_equal(obs, g["obs"])
        np.testing.assert_array_equal(acc, g["accept"])


def test_empty_and_invalid_requests():
    prog = T.Program(WORKED_EXAMPLE)
    T.tsim_sample(prog.h, 0, 1, 0)           # zero shots: no launch, no error
    T.tsim_sync()
    bogus = torch.empty((4, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(T.TsimError) as ei:
        T.tsim_sample(prog.h, 4, 1, 0, meas=bogus)  # detector-mode program has no meas record
    assert ei.value.code == 7


def test_shot_ranges_compose(tmp_path):
    # output is a pure function of (program, seed, global shot index)
    prog = T.Program(WORKED_EXAMPLE)
    a = _gpu(prog, 1000, 3, 0)
    b = _gpu(prog, 600, 3, 400)
    np.testing.assert_array_equal(a["obs"][400:], b["obs"][:600])
    np.testing.assert_array_equal(a["det"][400:], b["det"][:600])
