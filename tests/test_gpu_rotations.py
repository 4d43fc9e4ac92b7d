"""GPU parity for circuits with arbitrary rotations (R_X, R_Y, R_Z, U3 at
angles outside the multiples of pi/4).

Their chains are evaluated in double precision on both sides, and the
Bernoulli draw of Algorithm 1 compares U with the FP32-rounded ratio
P_1 / P_prev times 2^32 on both sides, so the records are compared bit for
bit (the two sums differ in order only, which moves a ratio by about 1e-16,
far below an FP32 step).  The complex table values the kernel computed are
compared with the oracle's to 1e-12 relative, through tsim_debug_sample.
"""
import random
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram
from tests import progfile
from tests.test_rotations import PAPER_LISTING, _random_rotation_circuit

pytestmark = pytest.mark.gpu

CASES = [
    ("listing_meas", PAPER_LISTING, T.MODE_MEASUREMENTS),
    ("surface_rz", Wk.surface_code_t_injection(d=3, rounds=3, p=1e-3, rotation=("R_Z(0.125)", "H", "R_Y(0.3)")),
     T.MODE_DETECTORS),
    ("surface_rz_meas", Wk.surface_code_t_injection(d=3, rounds=2, p=2e-3, rotation=("U3(0.3, 0.2, 0.7)",)),
     T.MODE_MEASUREMENTS),
] + [(f"random{k}", _random_rotation_circuit(random.Random(9100 + k), 4, 24, nrot=4), T.MODE_MEASUREMENTS)
     for k in range(4)]


def _gpu(prog, shots, seed, offset):
    out = prog.sample_torch(shots, seed, offset)
    T.tsim_sync()
    return {k: (v.cpu().numpy().view(np.uint64) if v is not None and v.dtype == torch.int64 else
                (v.cpu().numpy() if v is not None else None)) for k, v in out.items()}


@pytest.mark.parametrize("name,text,mode", CASES, ids=[c[0] for c in CASES])
def test_rotation_records_bit_exact(tmp_path, name, text, mode):
    prog = T.Program(text, mode=mode)
    path = str(tmp_path / "r.prog")
    prog.save(path)
    assert any(progfile.read(path)["table_float"])
    shots, seed, off = 20011, 5, (1 << 32) - 3
    g = _gpu(prog, shots, seed, off)
    o = OracleProgram(path).sample(seed, off, shots)
    i = prog.info
    if mode == T.MODE_MEASUREMENTS and i["meas_words"]:
        np.testing.assert_array_equal(g["meas"], o["meas"])
    if i["det_words"]:
        np.testing.assert_array_equal(g["det"], o["det"])
    if i["obs_words"]:
        np.testing.assert_array_equal(g["obs"], o["obs"])
    np.testing.assert_array_equal(g["accept"], o["accept"])


@pytest.mark.parametrize("name,text,mode", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_rotation_values_match_oracle(tmp_path, name, text, mode):
    prog = T.Program(text, mode=mode)
    path = str(tmp_path / "r.prog")
    prog.save(path)
    orc = OracleProgram(path)
    shots = 100_000
    idx = sorted(set([0, 1, 31, 32, shots - 1] + [random.Random(3).randrange(shots) for _ in range(40)]))
    dump = T.tsim_debug_sample(prog.h, shots, 2, 0, idx)
    W = prog.info["x_words"]
    n_float = 0
    for row in dump:
        for r in row:
            X = [int(v) & 0xFFFFFFFFFFFFFFFF for v in r[6:6 + W]]
            t = int(r[0])
            want = orc.eval_table_c(t, X)
            if int(r[5]) == -(1 << 31):
                got = complex(*struct.unpack("<2d", struct.pack("<2q", int(r[1]), int(r[2]))))
                n_float += 1
            else:  # an exact table: (c0 + c1 w + c2 w^2 + c3 w^3) sqrt2^k
                w = complex(np.exp(1j * np.pi / 4))
                got = sum(int(r[1 + j]) * w ** j for j in range(4)) * 2 ** (int(r[5]) / 2)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (t, got, want)
    assert n_float > 0
