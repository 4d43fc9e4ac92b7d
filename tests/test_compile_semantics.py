"""Program semantics: the compiled program's marginals must equal the exact
output distribution of the noisy circuit, for every raw noise assignment and
every output pattern (Appendix "Validation": probabilities of bit strings
against a state-vector simulator, here exactly instead of to fp32).

The product compiles the circuit; the oracle's independent state vector gives
P(outputs | e); the oracle's own C evaluator computes every marginal table of
the program file from the phase-pair formulas.  Algorithm 1's chain of
conditionals telescopes, so for every pattern o:
    P_sv(o | e) * prod_chains P_norm  ==  prod_chains P_prev(after o)
exactly, with every deterministic output equal to its parity rule.
"""
import itertools
import random

import pytest

import paper_2604_01059_gb300 as T
from oracle import circuit as ocirc
from oracle import statevector
from oracle.evaluator import OracleProgram
from oracle.zomega import DOmega, compare_real
from tests import progfile

W = DOmega.omega_pow


def check_program(text, mode, tmp_path, max_e=64, seed=0, decomp=T.DECOMP_HEURISTIC, reduction=True):
    h = T.tsim_compile(text, mode=mode, decomp=decomp, channel_reduction=reduction)
    path = str(tmp_path / "p.prog")
    T.tsim_program_save(h, path)
    info = T.tsim_program_info(h)
    T.tsim_program_free(h)
    prog = progfile.read(path)
    oprog = OracleProgram(path)
    circ = ocirc.parse(text)
    E = circ.num_error_bits
    assert info["num_error_bits"] == E
    assert [nb for nb, _, _ in prog["raw"]] == [ch.nbits for ch in circ.channels]
    # raw channel probabilities agree with the oracle's own parse
    for (nb, probs, _), ch in zip(prog["raw"], circ.channels):
        assert probs == pytest.approx([float(p) for p in ch.probs], abs=1e-15)
    rng = random.Random(seed)
    if 2 ** E <= max_e:
        assignments = list(itertools.product((0, 1), repeat=E))
    else:
        assignments = [tuple([0] * E)] + [tuple(rng.randrange(2) if rng.random() < 0.3 else 0
                                                for _ in range(E)) for _ in range(max_e - 1)]
    n_out = len(prog["outputs"])
    modename = "measurements" if mode == T.MODE_MEASUREMENTS else "detectors"
    for e in assignments:
        dist = statevector.output_distribution(circ, list(e), modename)
        x0 = progfile.x_of_raw(prog, e)
        norms = [oprog.eval_table(t, x0) for t in prog["chains"]]
        # a chain's tables share one phase w^j (the scalars its normalisation
        # restores); the normalisation is real and positive after removing it
        phases = []
        for pn in norms:
            js = [j for j in range(8) if (pn * W(-j)).is_real() and (pn * W(-j)).sign() > 0]
            assert len(js) == 1, pn
            phases.append(W(-js[0]))
        for o in itertools.product((0, 1), repeat=n_out):
            x = list(x0)
            pprev = list(norms)
            ok = True
            for i, out in enumerate(prog["outputs"]):
                if out[0] == "D":
                    if progfile.parity(out[1], x) ^ out[2] != o[i]:
                        ok = False
                        break
                else:
                    _, xb, ch, tb = out
                    x[xb >> 6] |= 1 << (xb & 63)
                    p1 = oprog.eval_table(tb, x)
                    p1r, prr = p1 * phases[ch], pprev[ch] * phases[ch]
                    assert p1r.is_real()
                    assert p1r.sign() >= 0 and compare_real(p1r, prr) <= 0
                    if o[i]:
                        pprev[ch] = p1
                    else:
                        pprev[ch] = pprev[ch] - p1
                        x[xb >> 6] &= ~(1 << (xb & 63))
            want = dist.get(tuple(o), DOmega())
            if not ok:
                assert want.is_zero(), (e, o)
                continue
            lhs = want
            for pn in norms:
                lhs = lhs * pn
            rhs = DOmega.from_int(1)
            for pp in pprev:
                rhs = rhs * pp
            assert lhs == rhs, (e, o, float(want))
    return info


T_INTERFERENCE = "RX 0\nT 0\nH 0\nM 0"

BELL_T = """
H 0
CX 0 1
T 1
H 1
M 0 1
"""

# Sec. "Simulation pipeline" worked example: two distance-2 repetition-code
# blocks, a stabilizer round with bit-flip channels, two logical rotations
# (T substituted for the pi/8 labels) separated by a phase-flip channel, a
# transversal CNOT, a second round and terminal measurements; detectors
# compare rounds, two observables come from the terminal measurements.
WORKED_EXAMPLE = """
RX 0 3
CX 0 1 3 4
R 2 5
CX 0 2 1 2 3 5 4 5
X_ERROR(0.01) 0 1 3 4
MR 2 5
DETECTOR rec[-2]
DETECTOR rec[-1]
T 0
Z_ERROR(0.02) 0
T 3
CX 0 3 1 4
CX 0 2 1 2 3 5 4 5
MR 2 5
DETECTOR rec[-2] rec[-4]
DETECTOR rec[-1] rec[-3]
MX 0 1 3 4
OBSERVABLE_INCLUDE(0) rec[-4] rec[-3]
OBSERVABLE_INCLUDE(1) rec[-2] rec[-1]
"""

REPETITION = """
R 0 1 2 3 4
CX 0 3 1 4
DEPOLARIZE2(0.01) 0 3
CX 1 3 2 4
X_ERROR(0.02) 2
MR(0.01) 3 4
DETECTOR rec[-2]
DETECTOR rec[-1]
CX 0 3 1 4
CX 1 3 2 4
MR 3 4
DETECTOR rec[-2] rec[-4]
DETECTOR rec[-1] rec[-3]
M 0 1 2
DETECTOR rec[-3] rec[-2] rec[-5]
OBSERVABLE_INCLUDE(0) rec[-1]
"""


# one transversal T-check on the Steane code: unitary encoder of T_DAG|+>,
# T_DAG on all data, X parity through an ancilla, T on all data, final X
# readout; noise on the injection qubit and on the check ancilla
STEANE_CHECK = """
H 0
T_DAG 0
DEPOLARIZE1(0.02) 0
H 3 5 6
CX 0 1 0 4 3 0 3 1 3 2 5 1 5 2 5 4 6 2 6 3 6 5
T_DAG 0 1 2 3 4 5 6
RX 7
CX 7 0 7 1 7 2 7 3 7 4 7 5 7 6
Z_ERROR(0.01) 7
MX 7
DETECTOR rec[-1]
T 0 1 2 3 4 5 6
X_ERROR(0.01) 2
MX 0 1 2 3 4 5 6
DETECTOR rec[-7] rec[-6] rec[-5] rec[-4]
DETECTOR rec[-6] rec[-5] rec[-3] rec[-2]
DETECTOR rec[-5] rec[-4] rec[-2] rec[-1]
OBSERVABLE_INCLUDE(0) rec[-7] rec[-6] rec[-3]
"""


# a chain whose marginals carry a noise-dependent phase w^j in the program
# (found by delta-debugging a random mirror circuit)
PHASED_CHAIN = """
R 0 1 2 3
H 3
H 1
H 2
H 0
S 3
CZ 0 1
SQRT_X 0
CZ 3 2
H 1
H 3
DEPOLARIZE1(0.003) 0 1 3
T_DAG 1
SQRT_X 0
S 1
S_DAG 3
H 2
CZ 1 3
X_ERROR(0.003) 0 1 2 3
M 0 1 2 3
DETECTOR rec[-4]
DETECTOR rec[-3]
DETECTOR rec[-2]
DETECTOR rec[-1]
OBSERVABLE_INCLUDE(0) rec[-4] rec[-3]
"""


def test_chain_with_noise_dependent_phase(tmp_path):
    check_program(PHASED_CHAIN, T.MODE_DETECTORS, tmp_path, max_e=1024)


def test_steane_t_check(tmp_path):
    # the colour-code T-check: the check and the plaquettes are deterministic
    # without noise; the observable carries the magic state
    check_program(STEANE_CHECK, T.MODE_DETECTORS, tmp_path, max_e=32)


def test_t_interference(tmp_path):
    info = check_program(T_INTERFERENCE, T.MODE_MEASUREMENTS, tmp_path)
    assert info["num_random"] == 1


def test_bell_with_t(tmp_path):
    check_program(BELL_T, T.MODE_MEASUREMENTS, tmp_path)


def test_worked_example_structure_and_values(tmp_path):
    # structure the paper reports: every detector is fixed by one f parity
    # (deterministic output), the observables form one connected component
    info = check_program(WORKED_EXAMPLE, T.MODE_DETECTORS, tmp_path, max_e=32)
    assert info["num_detectors"] == 4 and info["num_observables"] == 2
    assert info["num_random"] >= 1 and info["num_chains"] == 1
    assert info["num_random"] <= 2


def test_worked_example_measurement_mode(tmp_path):
    check_program(WORKED_EXAMPLE, T.MODE_MEASUREMENTS, tmp_path, max_e=8)


def test_clifford_repetition_code_detectors_are_deterministic(tmp_path):
    info = check_program(REPETITION, T.MODE_DETECTORS, tmp_path, max_e=48)
    # Clifford memory: all detectors and the observable are deterministic given e
    assert info["num_random"] == 0 and info["total_terms"] == 0


def test_no_channel_reduction_same_semantics(tmp_path):
    check_program(REPETITION, T.MODE_DETECTORS, tmp_path, max_e=24, reduction=False)


@pytest.mark.parametrize("decomp", [T.DECOMP_SINGLE_T, T.DECOMP_HEURISTIC, T.DECOMP_PAIRS, T.DECOMP_CAT5])
def test_decomposition_policy_invariance(tmp_path, decomp):
    check_program(WORKED_EXAMPLE, T.MODE_DETECTORS, tmp_path, max_e=12, decomp=decomp)


@pytest.mark.parametrize("seed", range(4))
def test_cat5_groups_exact_against_state_vector(tmp_path, seed):
    # three T gates on entangled qubits: six odd spiders in the doubled
    # diagram, so Cat5 (Eq. cat5) takes a group of five; every marginal must
    # still equal the state-vector probability exactly, as with pairs
    rng = random.Random(4000 + seed)
    L = ["RX 0 1 2", "CX 0 1", "CZ 1 2"]
    for q in range(3):
        L.append(f"{rng.choice(['T', 'T_DAG'])} {q}")
        L.append(f"{rng.choice(['H', 'SQRT_X'])} {q}")
    L += ["CX 2 0", "DEPOLARIZE1(0.05) 0 1", "T 1", "H 1", "X_ERROR(0.04) 2", "M 0 1 2"]
    text = "\n".join(L)
    for decomp in (T.DECOMP_CAT5, T.DECOMP_PAIRS):
        check_program(text, T.MODE_MEASUREMENTS, tmp_path, max_e=8, seed=seed, decomp=decomp)


def _random_circuit(rng, nq, depth, tcount):
    lines = [f"RX {q}" if rng.random() < 0.5 else f"R {q}" for q in range(nq)]
    gates1 = ["H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG"]
    placed_t = 0
    for _ in range(depth):
        r = rng.random()
        if r < 0.12 and placed_t < tcount:
            lines.append(f"{rng.choice(['T', 'T_DAG'])} {rng.randrange(nq)}")
            placed_t += 1
        elif r < 0.45:
            lines.append(f"{rng.choice(gates1)} {rng.randrange(nq)}")
        elif r < 0.75:
            a, b = rng.sample(range(nq), 2)
            lines.append(f"{rng.choice(['CX', 'CZ', 'CY', 'SWAP'])} {a} {b}")
        elif r < 0.83:
            q = rng.randrange(nq)
            lines.append(f"{rng.choice(['X_ERROR', 'Z_ERROR', 'Y_ERROR'])}(0.05) {q}")
        elif r < 0.87:
            a, b = rng.sample(range(nq), 2)
            lines.append(f"DEPOLARIZE2(0.03) {a} {b}")
        elif r < 0.9:
            lines.append(f"DEPOLARIZE1(0.03) {rng.randrange(nq)}")
        elif r < 0.95:
            lines.append(f"{rng.choice(['MR', 'M', 'MX'])} {rng.randrange(nq)}")
        else:
            lines.append(f"M(0.02) {rng.randrange(nq)}")
    lines.append("M " + " ".join(str(q) for q in range(nq)))
    return "\n".join(lines)


@pytest.mark.parametrize("seed", range(12))
def test_random_circuits_measurement_mode(tmp_path, seed):
    rng = random.Random(1000 + seed)
    text = _random_circuit(rng, 3, 18, tcount=3)
    c = ocirc.parse(text)
    if c.num_measurements > 7:
        pytest.skip("too many outputs for the exhaustive check")
    check_program(text, T.MODE_MEASUREMENTS, tmp_path, max_e=6, seed=seed)


@pytest.mark.parametrize("seed", range(10))
def test_random_circuits_detector_mode(tmp_path, seed):
    rng = random.Random(2000 + seed)
    text = _random_circuit(rng, 3, 16, tcount=2)
    c = ocirc.parse(text)
    nm = c.num_measurements
    # detectors and observables as random XORs of records
    dets = []
    for _ in range(3):
        k = rng.randrange(1, 3)
        dets.append("DETECTOR " + " ".join(f"rec[-{j}]" for j in rng.sample(range(1, nm + 1), min(k, nm))))
    obs = "OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{j}]" for j in rng.sample(range(1, nm + 1), min(2, nm)))
    text = text + "\n" + "\n".join(dets) + "\n" + obs
    check_program(text, T.MODE_DETECTORS, tmp_path, max_e=6, seed=seed)
