"""Pins for the oracle's program-semantics half: the exact state vector and
the Pauli-frame propagator, each against textbook closed forms, Born-rule
invariants and one another (two independent methods)."""
import itertools
import random

import pytest

from oracle import circuit, frame, statevector
from oracle.zomega import DOmega

W = DOmega.omega_pow
S2 = DOmega.sqrt2_pow


def dist(text, e=None, mode="measurements"):
    c = circuit.parse(text)
    if e is None:
        e = [0] * c.num_error_bits
    return c, statevector.output_distribution(c, e, mode)


def test_bell_state():
    _, d = dist("H 0\nCX 0 1\nM 0 1")
    assert d == {(0, 0): S2(-2), (1, 1): S2(-2)}


def test_t_interference_closed_form():
    # |<0| H T |+>|^2 = |1 + w|^2 / 4 = (2 + sqrt2)/4
    _, d = dist("RX 0\nT 0\nH 0\nM 0")
    assert d[(0,)] == (2 + S2(1)) * S2(-4)
    assert d[(1,)] == (2 - S2(1)) * S2(-4)
    # T T = S: H S |+> measured -> 1/2 each ; T T_DAG = I -> deterministic
    _, d = dist("RX 0\nT 0\nT 0\nH 0\nM 0")
    assert d[(0,)] == S2(-2) and d[(1,)] == S2(-2)
    _, d = dist("RX 0\nT 0\nT_DAG 0\nH 0\nM 0")
    assert d == {(0,): DOmega.from_int(1)}


def test_sqrt_x_and_y_gates():
    # SQRT_X^2 = X ; Y|0> = i|1>
    _, d = dist("SQRT_X 0\nSQRT_X 0\nM 0")
    assert d == {(1,): DOmega.from_int(1)}
    _, d = dist("Y 0\nM 0")
    assert d == {(1,): DOmega.from_int(1)}
    _, d = dist("SQRT_X 0\nSQRT_X_DAG 0\nM 0")
    assert d == {(0,): DOmega.from_int(1)}


def test_noise_bits_insert_paulis():
    text = "X_ERROR(0.25) 0\nM 0"
    c, d0 = dist(text, [0])
    _, d1 = dist(text, [1])
    assert d0 == {(0,): 1} and d1 == {(1,): 1}
    assert c.channels[0].probs == [pytest.approx(0.75), pytest.approx(0.25)]
    # PAULI_CHANNEL_1 encoding: (e_x, e_z) = (1,0) X, (1,1) Y, (0,1) Z
    c = circuit.parse("PAULI_CHANNEL_1(0.1, 0.2, 0.3) 0\nM 0")
    from fractions import Fraction as F
    assert c.channels[0].probs == [F(4, 10), F(1, 10), F(3, 10), F(2, 10)]
    for ex, ez in itertools.product((0, 1), repeat=2):
        _, d = dist("PAULI_CHANNEL_1(0.1, 0.2, 0.3) 0\nM 0", [ex, ez])
        assert d == {(ex,): 1}
        _, d = dist("RX 0\nPAULI_CHANNEL_1(0.1, 0.2, 0.3) 0\nMX 0", [ex, ez])
        assert d == {(ez,): 1}


def test_measurement_flip_and_reset():
    _, d = dist("X 0\nM(0.1) 0\nM 0", [1])
    assert d == {(0, 1): 1}           # record flipped, state not
    _, d = dist("H 0\nMR 0\nM 0")
    assert d == {(0, 0): S2(-2), (1, 0): S2(-2)}
    _, d = dist("H 0\nR 0\nM 0")
    assert d == {(0,): 1}
    _, d = dist("RX 0\nMRX 0\nMX 0")
    assert d == {(0, 0): 1}


def test_classically_controlled_pauli():
    # teleport-like correction: measure half of a Bell pair, fix the other
    _, d = dist("H 0\nCX 0 1\nM 0\nCX rec[-1] 1\nM 1")
    assert d == {(0, 0): S2(-2), (1, 0): S2(-2)}


def _random_circuit(rng, nq, depth, clifford_only, noise=True):
    lines = []
    gates1 = ["H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X"] + ([] if clifford_only else ["T", "T_DAG"])
    for _ in range(depth):
        r = rng.random()
        if r < 0.45:
            lines.append(f"{rng.choice(gates1)} {rng.randrange(nq)}")
        elif r < 0.75:
            a, b = rng.sample(range(nq), 2)
            lines.append(f"{rng.choice(['CX', 'CZ', 'CY'])} {a} {b}")
        elif r < 0.85 and noise:
            q = rng.randrange(nq)
            lines.append(f"{rng.choice(['X_ERROR', 'Z_ERROR', 'Y_ERROR'])}(0.01) {q}")
        elif r < 0.9 and noise:
            a, b = rng.sample(range(nq), 2)
            lines.append(f"DEPOLARIZE2(0.01) {a} {b}")
        else:
            q = rng.randrange(nq)
            lines.append(f"{rng.choice(['M', 'MR', 'MX'])} {q}")
    lines.append("M " + " ".join(str(q) for q in range(nq)))
    return "\n".join(lines)


@pytest.mark.parametrize("seed", range(6))
def test_born_invariants(seed):
    rng = random.Random(seed)
    text = _random_circuit(rng, 3, 14, clifford_only=False)
    c = circuit.parse(text)
    e = [rng.randrange(2) for _ in range(c.num_error_bits)]
    d = statevector.output_distribution(c, e, "measurements")
    total = sum(d.values(), DOmega())
    assert total == 1
    for p in d.values():
        assert p.is_real() and p.sign() > 0
    # marginals are consistent: P(prefix) = P(prefix,0) + P(prefix,1)
    n = c.num_measurements
    for k in range(n):
        for pre in itertools.product((0, 1), repeat=k):
            m = statevector.marginal(d, pre)
            assert m == statevector.marginal(d, pre + (0,)) + statevector.marginal(d, pre + (1,))


def _repetition_code(rounds=2):
    # distance-3 bit-flip repetition code memory, Clifford, deterministic detectors
    L = ["R 0 1 2 3 4"]
    for r in range(rounds):
        L += ["CX 0 3 1 4", "DEPOLARIZE2(0.01) 0 3 1 4", "CX 1 3 2 4",
              "X_ERROR(0.02) 0 1 2", "MR(0.01) 3 4"]
        if r == 0:
            L += ["DETECTOR rec[-2]", "DETECTOR rec[-1]"]
        else:
            L += ["DETECTOR rec[-2] rec[-4]", "DETECTOR rec[-1] rec[-3]"]
    L += ["M 0 1 2", "DETECTOR rec[-3] rec[-2] rec[-5]", "DETECTOR rec[-2] rec[-1] rec[-4]",
          "OBSERVABLE_INCLUDE(0) rec[-1]"]
    return "\n".join(L)


def test_clifford_noiseless_detectors_are_deterministic():
    c = circuit.parse(_repetition_code())
    d = statevector.output_distribution(c, [0] * c.num_error_bits, "detectors")
    assert d == {(0,) * (c.num_detectors + c.num_observables): 1}


@pytest.mark.parametrize("seed", range(4))
def test_frame_flips_match_state_vector(seed):
    # Two independent methods must agree on T's columns (Sec. "Detectors"):
    # flipping one raw error bit changes the (deterministic) detector and
    # observable values exactly as the propagated Pauli says.
    rng = random.Random(100 + seed)
    if seed == 0:
        text = _repetition_code()
    else:
        body = _random_circuit(rng, 3, 12, clifford_only=True)
        # make every measurement deterministic by measuring a fresh copy chain
        text = "R 0 1 2\n" + body.replace("MX", "M")
    c = circuit.parse(text)
    if not c.detectors:
        # declare each final measurement a detector of its own
        text += "\n" + "\n".join(f"DETECTOR rec[-{k}]" for k in range(1, 4))
        c = circuit.parse(text)
    base = statevector.output_distribution(c, [0] * c.num_error_bits, "detectors")
    flips = frame.detector_flips(c)
    for j in range(c.num_error_bits):
        e = [0] * c.num_error_bits
        e[j] = 1
        d = statevector.output_distribution(c, e, "detectors")
        fd, fo = flips[j]
        want = {}
        for key, p in base.items():
            nd = len(fd)
            k2 = tuple(b ^ f for b, f in zip(key, fd + fo))
            want[k2] = p
        assert d == want, (j, flips[j])


@pytest.mark.parametrize("seed", range(3))
def test_frame_flips_through_t_gates_match_state_vector(seed):
    # A Z error that meets T or T_DAG passes unchanged (T Z T^dag = Z), so the
    # frame picture still holds on a non-Clifford circuit where every T sees
    # only Z-type frames: Z_ERROR before the T layer, X_ERROR after it.  The
    # shifted outcome distribution on the exact state vector must match.
    rng = random.Random(300 + seed)
    L = ["RX 0 1 2", "CX 0 1", "Z_ERROR(0.1) 0 1 2"]
    for q in range(3):
        L.append(f"{rng.choice(['T', 'T_DAG'])} {q}")
    L += ["CX 1 2", "H 0", "S 1", "X_ERROR(0.1) 0 2", "CX 2 0", "H 1", "M 0 1 2",
          "DETECTOR rec[-1]", "DETECTOR rec[-2] rec[-3]", "OBSERVABLE_INCLUDE(0) rec[-1] rec[-2]"]
    text = "\n".join(L)
    c = circuit.parse(text)
    base = statevector.output_distribution(c, [0] * c.num_error_bits, "detectors")
    flips = frame.detector_flips(c)
    assert any(any(fd) or any(fo) for fd, fo in flips)
    for j in range(c.num_error_bits):
        e = [0] * c.num_error_bits
        e[j] = 1
        d = statevector.output_distribution(c, e, "detectors")
        fd, fo = flips[j]
        want = {tuple(b ^ f for b, f in zip(key, fd + fo)): p for key, p in base.items()}
        assert d == want, (j, flips[j])
    # an X error in front of a T gate is refused rather than propagated
    with pytest.raises(ValueError):
        frame.detector_flips(circuit.parse("RX 0\nX_ERROR(0.1) 0\nT 0\nH 0\nM 0\nDETECTOR rec[-1]"))
