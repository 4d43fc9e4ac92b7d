"""Arbitrary rotations R_X, R_Y, R_Z and U3 (Sec. "Methods"; angles in units of
pi, as in the paper's listing `R_Z(0.125) 0`).

Pins of the oracle's floating-point state vector against closed forms and
against the exact state vector where the angles are multiples of pi/4; then
the program semantics of compiled rotation circuits: for every raw noise
assignment and every output pattern, the product of the conditionals of
Algorithm 1 computed from the compiled tables (evaluated by the oracle's C
evaluator in complex double, each chain's phase taken from its
normalisation) equals the state-vector probability to 1e-9.
"""
import itertools
import math
import random

import numpy as np
import pytest

import paper_2604_01059_gb300 as T
from oracle import circuit as ocirc
from oracle import statevector, statevector_f
from oracle.evaluator import OracleProgram
from tests import progfile

PAPER_LISTING = """RX 0
R 1
R_Z(0.125) 0
PAULI_CHANNEL_1(0.1, 0.1, 0.2) 0 1
H 0
CNOT 0 1
DEPOLARIZE2(0.01) 0 1
M 0 1
DETECTOR rec[-1] rec[-2]"""


def _fdist(text, e=None, mode="measurements"):
    c = ocirc.parse(text)
    return statevector_f.output_distribution(c, e or [0] * c.num_error_bits, mode)


def test_closed_forms():
    for t in (0.1, 0.37, 1.3):
        d = _fdist(f"R_Y({t}) 0\nM 0")
        assert d[(1,)] == pytest.approx(math.sin(math.pi * t / 2) ** 2, abs=1e-14)
        d = _fdist(f"R_X({t}) 0\nM 0")
        assert d[(1,)] == pytest.approx(math.sin(math.pi * t / 2) ** 2, abs=1e-14)
        # |<+| R_Z(t) |+>|^2 = cos^2(pi t / 2)
        d = _fdist(f"RX 0\nR_Z({t}) 0\nMX 0")
        assert d[(0,)] == pytest.approx(math.cos(math.pi * t / 2) ** 2, abs=1e-14)
    d = _fdist("H 0\nR_Z(0.3) 0\nCX 0 1\nM 0 1")
    assert sum(d.values()) == pytest.approx(1.0, abs=1e-14)
    assert set(d) == {(0, 0), (1, 1)}


def test_multiples_of_quarter_turns_match_the_exact_state_vector():
    # R_Z(1/4) = T, R_Z(1/2) = S, R_X(1/2) = SQRT_X (up to a global phase)
    rng = random.Random(7)
    for _ in range(6):
        L = ["RX 0", "R 1 2"]
        for _ in range(10):
            g = rng.choice(["T", "S", "SQRT_X", "H", "CX"])
            if g == "CX":
                a, b = rng.sample(range(3), 2)
                L.append(f"CX {a} {b}")
            else:
                L.append(f"{g} {rng.randrange(3)}")
        exact = "\n".join(L + ["M 0 1 2"])
        rot = exact.replace("SQRT_X", "R_X(0.5)").replace("T ", "R_Z(0.25) ").replace("S ", "R_Z(0.5) ")
        want = statevector.output_distribution(ocirc.parse(exact), [0] * 0, "measurements")
        got = _fdist(rot)
        for k, p in want.items():
            assert got.get(k, 0.0) == pytest.approx(float(p), abs=1e-12)
        assert sum(got.values()) == pytest.approx(1.0, abs=1e-12)


def test_u3_is_rz_ry_rz():
    for a, b, c in [(0.3, 0.7, 1.1), (1.9, 0.2, 0.45)]:
        d1 = _fdist(f"RX 0\nU3({a}, {b}, {c}) 0\nH 0\nM 0")
        d2 = _fdist(f"RX 0\nR_Z({c}) 0\nR_Y({a}) 0\nR_Z({b}) 0\nH 0\nM 0")
        for k in d1:
            assert d1[k] == pytest.approx(d2[k], abs=1e-12)


def check_float_program(text, mode, tmp_path, max_e=32, seed=0, decomp=T.DECOMP_HEURISTIC):
    prog_h = T.Program(text, mode=mode, decomp=decomp)
    path = str(tmp_path / "p.prog")
    prog_h.save(path)
    prog = progfile.read(path)
    oprog = OracleProgram(path)
    circ = ocirc.parse(text)
    E = circ.num_error_bits
    rng = random.Random(seed)
    if 2 ** E <= max_e:
        assignments = list(itertools.product((0, 1), repeat=E))
    else:
        assignments = [tuple([0] * E)] + [tuple(rng.randrange(2) if rng.random() < 0.3 else 0
                                                for _ in range(E)) for _ in range(max_e - 1)]
    modename = "measurements" if mode == T.MODE_MEASUREMENTS else "detectors"
    n_out = len(prog["outputs"])
    for e in assignments:
        dist = statevector_f.output_distribution(circ, list(e), modename)
        x0 = progfile.x_of_raw(prog, e)
        norms = [oprog.eval_table_c(t, x0) for t in prog["chains"]]
        # the product evaluates the same tables (host, complex double)
        for t, z in zip(prog["chains"], norms):
            assert T.tsim_eval_table_float(prog_h.h, t, x0) == pytest.approx(z, rel=1e-12, abs=1e-12)
        total = 0.0
        for o in itertools.product((0, 1), repeat=n_out):
            x = list(x0)
            pprev = [abs(z) for z in norms]
            ok = True
            for i, out in enumerate(prog["outputs"]):
                if out[0] == "D":
                    if progfile.parity(out[1], x) ^ out[2] != o[i]:
                        ok = False
                        break
                else:
                    _, xb, ch, tb = out
                    x[xb >> 6] |= 1 << (xb & 63)
                    zn = norms[ch]
                    z1 = oprog.eval_table_c(tb, x)
                    p1 = (z1 * zn.conjugate()).real / abs(zn)
                    assert abs((z1 * zn.conjugate()).imag) <= 1e-9 * abs(zn) * (abs(z1) + 1e-300) + 1e-12
                    assert -1e-12 <= p1 <= pprev[ch] * (1 + 1e-12) + 1e-12
                    if o[i]:
                        pprev[ch] = p1
                    else:
                        pprev[ch] -= p1
                        x[xb >> 6] &= ~(1 << (xb & 63))
            want = dist.get(tuple(o), 0.0)
            if not ok:
                assert want == pytest.approx(0.0, abs=1e-12), (e, o)
                continue
            got = 1.0
            for pp, z in zip(pprev, norms):
                got *= pp / abs(z)
            assert got == pytest.approx(want, abs=1e-9), (e, o)
            total += got
        assert total == pytest.approx(1.0, abs=1e-9)
    return prog_h


def test_paper_listing_semantics(tmp_path):
    prog = check_float_program(PAPER_LISTING, T.MODE_MEASUREMENTS, tmp_path, max_e=256)
    assert any(prog.device_table_layout(t)[0] == 3 for t in range(prog.info["num_tables"]))
    check_float_program(PAPER_LISTING, T.MODE_DETECTORS, tmp_path, max_e=256)


def _random_rotation_circuit(rng, nq, depth, nrot):
    lines = [f"RX {q}" if rng.random() < 0.5 else f"R {q}" for q in range(nq)]
    placed = 0
    for _ in range(depth):
        r = rng.random()
        if r < 0.2 and placed < nrot:
            g = rng.choice(["R_X", "R_Y", "R_Z", "U3", "T"])
            if g == "U3":
                lines.append(f"U3({rng.random() * 2:.4f}, {rng.random() * 2:.4f}, {rng.random() * 2:.4f}) "
                             f"{rng.randrange(nq)}")
            elif g == "T":
                lines.append(f"T {rng.randrange(nq)}")
            else:
                lines.append(f"{g}({rng.random() * 2:.4f}) {rng.randrange(nq)}")
            placed += 1
        elif r < 0.45:
            lines.append(f"{rng.choice(['H', 'S', 'SQRT_X', 'X'])} {rng.randrange(nq)}")
        elif r < 0.7:
            a, b = rng.sample(range(nq), 2)
            lines.append(f"{rng.choice(['CX', 'CZ'])} {a} {b}")
        elif r < 0.8:
            lines.append(f"{rng.choice(['X_ERROR', 'Z_ERROR'])}(0.05) {rng.randrange(nq)}")
        elif r < 0.85:
            lines.append(f"DEPOLARIZE1(0.03) {rng.randrange(nq)}")
        elif r < 0.89:
            lines.append(f"{rng.choice(['M', 'MX'])} {rng.randrange(nq)}")
        elif r < 0.92:
            lines.append(f"M(0.02) {rng.randrange(nq)}")
    lines.append("M " + " ".join(str(q) for q in range(nq)))
    return "\n".join(lines)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("decomp", [T.DECOMP_HEURISTIC, T.DECOMP_SINGLE_T])
def test_random_rotation_circuits(tmp_path, seed, decomp):
    rng = random.Random(9000 + seed)
    text = _random_rotation_circuit(rng, 3, 16, nrot=3)
    c = ocirc.parse(text)
    if c.num_measurements > 7:
        pytest.skip("too many outputs for the exhaustive check")
    check_float_program(text, T.MODE_MEASUREMENTS, tmp_path, max_e=8, seed=seed, decomp=decomp)


def test_rotation_program_file_round_trip(tmp_path):
    prog = T.Program(PAPER_LISTING, mode=T.MODE_MEASUREMENTS)
    a = str(tmp_path / "a.prog")
    b = str(tmp_path / "b.prog")
    prog.save(a)
    again = T.Program.load(a)
    again.save(b)
    assert open(a).read() == open(b).read()
    x = [1]
    for t in range(prog.info["num_tables"]):
        assert T.tsim_eval_table_float(again.h, t, x) == T.tsim_eval_table_float(prog.h, t, x)
    flt = progfile.read(a)["table_float"]
    assert any(flt)
    for t, f in enumerate(flt):
        if f:  # the exact form refuses a table with arbitrary phases
            with pytest.raises(T.TsimError):
                T.tsim_eval_table(prog.h, t, x)
        assert np.isfinite(abs(T.tsim_eval_table_float(prog.h, t, x)))
