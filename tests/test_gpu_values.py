"""GPU parity of the exact marginal values, not only of the records.

A record bit flips only when an error in P_1 moves the Bernoulli threshold
across the shot's uniform word, so a small error in a rare term class could
hide behind equal records.  tsim_debug_sample runs the production kernel on
the full launch and copies out, for chosen shots, every table value the
kernel computed -- the four Z[w] coefficients and the sqrt2 exponent -- with
the X it was evaluated at.  Each is compared exactly with the oracle's own
evaluation of the same table at the same X (Eqs. parities, phase_pair,
scalar_product), and X itself is checked: the noise part against the
oracle's f = T e for that shot (Eq. detector_sampling), the output part
against the records.  Covered: the benchmark surface code at 10^6 shots in
both noise modes, the colour-code T-check in its bit-sliced and its
per-thread table layouts, and small programs forced into the sliced layout.
"""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram
from oracle.zomega import DOmega
from tests import progfile
from tests.test_compile_semantics import PHASED_CHAIN, STEANE_CHECK, WORKED_EXAMPLE

pytestmark = pytest.mark.gpu


def _check_values(prog, path, shots, seed, offset, idx):
    i = prog.info
    det = torch.zeros((shots, max(i["det_words"], 1)), dtype=torch.int64, device="cuda")
    obs = torch.zeros((shots, max(i["obs_words"], 1)), dtype=torch.int64, device="cuda")
    meas = (torch.zeros((shots, i["meas_words"]), dtype=torch.int64, device="cuda")
            if i["mode"] == T.MODE_MEASUREMENTS and i["meas_words"] else None)
    dump = T.tsim_debug_sample(prog.h, shots, seed, offset, idx, meas=meas,
                               det=det if i["det_words"] else None, obs=obs if i["obs_words"] else None)
    det = det.cpu().numpy().view(np.uint64)
    obs = obs.cpu().numpy().view(np.uint64)
    meas = meas.cpu().numpy().view(np.uint64) if meas is not None else None
    orc = OracleProgram(path)
    pf = progfile.read(path)
    W = i["x_words"]
    order = list(pf["chains"]) + [o[3] for o in pf["outputs"] if o[0] == "R"]
    randoms = [(k, o) for k, o in enumerate(pf["outputs"]) if o[0] == "R"]
    checked = 0
    for row, s in enumerate(idx):
        recs = dump[row]
        assert [int(r[0]) for r in recs] == order
        x = orc.noise_x(seed, offset + s)
        # output bits of the shot, from its records
        if i["mode"] == T.MODE_MEASUREMENTS:
            bit = lambda k: int((int(meas[s][k >> 6]) >> (k & 63)) & 1)  # noqa: E731
        else:
            nd = i["num_detectors"]
            bit = lambda k: (int((int(det[s][k >> 6]) >> (k & 63)) & 1) if k < nd else  # noqa: E731
                             int((int(obs[s][(k - nd) >> 6]) >> ((k - nd) & 63)) & 1))
        nch = len(pf["chains"])
        for e, r in enumerate(recs):
            X = [int(v) & 0xFFFFFFFFFFFFFFFF for v in r[6:6 + W]]
            if e < nch:
                want_x = x
            else:
                # the noise X, the earlier random outputs' bits, and this output set to 1
                want_x = list(x)
                for k, o in randoms[:e - nch]:
                    if bit(k):
                        want_x[o[1] >> 6] |= 1 << (o[1] & 63)
                xb = randoms[e - nch][1][1]
                want_x[xb >> 6] |= 1 << (xb & 63)
            assert X == want_x, (s, e)
            got = DOmega([int(v) for v in r[1:5]], -int(r[5]))
            assert got == orc.eval_table(int(r[0]), X), (s, e, int(r[0]))
            checked += 1
    return checked


@pytest.mark.parametrize("noise", [0, 1])
def test_config2_values_full_launch(tmp_path, noise):
    prog = T.Program(Wk.config2_circuit(p=2e-3))
    prog.set_noise_sampling(noise)
    path = str(tmp_path / "c2.prog")
    prog.save(path)
    shots = 1_000_000
    rng = random.Random(noise + 1)
    idx = sorted(set([0, shots - 1] + [rng.randrange(shots) for _ in range(300)]))
    assert _check_values(prog, path, shots, 0, 0, idx) >= 2 * len(idx)


@pytest.mark.parametrize("layout", ["sliced", "per_thread"])
def test_config3_values(tmp_path, layout):
    prog = T.Program(Wk.config3_circuit())
    if layout == "per_thread":
        prog.set_table_layout(-1)
    modes = {prog.device_table_layout(t)[0] for t in range(prog.info["num_tables"])}
    assert (2 in modes) == (layout == "sliced")
    path = str(tmp_path / "c3.prog")
    prog.save(path)
    shots = 200_000 if layout == "sliced" else 20_000
    rng = random.Random(3)
    idx = sorted(set([0, 31, 32, shots - 1] + [rng.randrange(shots) for _ in range(12)]))
    assert _check_values(prog, path, shots, 5, 1 << 32, idx) >= 14 * len(idx)


@pytest.mark.parametrize("name,text,mode", [
    ("worked", WORKED_EXAMPLE, T.MODE_DETECTORS),
    ("worked_meas", WORKED_EXAMPLE, T.MODE_MEASUREMENTS),
    ("steane", STEANE_CHECK, T.MODE_DETECTORS),
    ("phased", PHASED_CHAIN, T.MODE_DETECTORS),
    ("cfg1", Wk.config1_circuit(p=5e-3), T.MODE_DETECTORS),
])
def test_forced_sliced_small_programs_values(tmp_path, name, text, mode):
    prog = T.Program(text, mode=mode)
    prog.set_table_layout(0, 0, 16)  # every qualifying table sliced, 16-word segments
    path = str(tmp_path / "s.prog")
    prog.save(path)
    shots = 4099
    idx = [0, 1, 31, 32, 33, 1000, 2047, 4096, 4098]
    _check_values(prog, path, shots, 17, 12345, idx)
