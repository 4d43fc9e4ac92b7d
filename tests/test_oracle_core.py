"""Pins for the oracle's arithmetic: Philox, Z[w], the factor formulas,
the exact Bernoulli rule and Algorithm 1 on hand-written programs.

Every expected value here comes from a published definition, a closed form
worked by hand, or an independent integer computation -- never from the
code under test.
"""
import math
import os

import pytest

from oracle.zomega import DOmega, compare_real
from tests.progtext import program_text

GOLD = os.path.join(os.path.dirname(__file__), "golden")
W = DOmega.omega_pow


def test_philox_known_answers(oracle_lib):
    n = 0
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert oracle_lib.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])
        n += 1
    assert n == 3


def test_zomega_closed_forms():
    sqrt2 = DOmega.sqrt2_pow(1)
    assert W(8) == W(0) == 1
    assert W(4) == -1
    assert W(2) * W(2) == -1                       # i^2 = -1
    assert sqrt2 * sqrt2 == 2
    assert W(1) + W(7) == sqrt2                    # w + w^-1 = 2 cos(pi/4)
    assert (1 + W(2)) * (1 + W(2)) == 2 * W(2)     # (1+i)^2 = 2i
    one_w = 1 + W(1)
    n = one_w * one_w.conj()                       # |1+w|^2 = 2 + sqrt2
    assert n == 2 + sqrt2 and n.is_real()
    half = DOmega.sqrt2_pow(-2)
    assert half + half == 1
    assert compare_real(sqrt2, DOmega.from_int(1)) == 1
    assert compare_real(DOmega.from_int(3), 2 * sqrt2) == 1      # 3 > 2.828
    assert compare_real(DOmega.from_int(2) * 707, 1000 * sqrt2) == -1  # 1414 < 1414.2
    assert abs(float(n) - (2 + math.sqrt(2))) < 1e-12


def _single_factor_program(tmp_path, kind, alpha, beta):
    # X bit 0 = a, X bit 1 = b ; one table with one factor, c = 1
    txt = program_text(nx=2, nf=2, tables=[[(0, 0, [(kind, alpha, beta, [1], [2])])]])
    p = tmp_path / "f.prog"
    p.write_text(txt)
    return str(p)


def test_phase_pair_formula_matches_hand_table(tmp_path, oracle_lib):
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLD, "phase_pair_clifford.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 16
    for A, B, re_, im_ in rows:
        # choose (alpha, a) and (beta, b) in both ways that give the same A, B
        for a in (0, 1):
            for b in (0, 1):
                alpha, beta = (A - 4 * a) % 8, (B - 4 * b) % 8
                prog = oracle_lib.OracleProgram(_single_factor_program(tmp_path, 0, alpha, beta))
                v = prog.eval_table(0, [a | (b << 1)])
                assert v == re_ + im_ * W(2), (A, B, a, b)


@pytest.mark.parametrize("alpha", range(8))
def test_other_factor_kinds(tmp_path, oracle_lib, alpha):
    # Table "Types of parameterized phase terms": Node 1 + e^{i(alpha + a pi)},
    # Half-pi e^{+-i a pi/2} (generalised to e^{i alpha a pi/4}), pi-pair (-1)^{ab}
    for a in (0, 1):
        for b in (0, 1):
            x = [a | (b << 1)]
            node = oracle_lib.OracleProgram(_single_factor_program(tmp_path, 1, alpha, 0)).eval_table(0, x)
            assert node == 1 + W(alpha + 4 * a)
            ph = oracle_lib.OracleProgram(_single_factor_program(tmp_path, 2, alpha, 0)).eval_table(0, x)
            assert ph == W(alpha * a)
            pp = oracle_lib.OracleProgram(_single_factor_program(tmp_path, 3, 0, 0)).eval_table(0, x)
            assert pp == (-1 if (a and b) else 1)


def test_term_sum_and_scalar(tmp_path, oracle_lib):
    # P = sum_t c^t prod h : c^1 = w^3 / sqrt2, c^2 = sqrt2^3 with a node factor
    txt = program_text(nx=1, nf=1, tables=[[(-1, 3, []), (3, 0, [(1, 2, 0, [1], [0])])]])
    p = tmp_path / "t.prog"
    p.write_text(txt)
    prog = oracle_lib.OracleProgram(str(p))
    s = DOmega.sqrt2_pow
    for a in (0, 1):
        want = W(3) * s(-1) + s(3) * (1 + W(2 + 4 * a))
        assert prog.eval_table(0, [a]) == want


def test_exact_bernoulli_rule(oracle_lib):
    # bit = 1 iff U * P_prev < 2^32 * P_1 ; P = (A + B sqrt2) 2^e
    # P_1 / P_prev = 1/2  ->  threshold exactly 2^31
    assert oracle_lib.decide(2 ** 31 - 1, 1, 0, 0, 1, 0, -1) == 1
    assert oracle_lib.decide(2 ** 31, 1, 0, 0, 1, 0, -1) == 0
    # P_1 = (2 + sqrt2)/4, P_prev = 1: bit = 1 iff 4U < 2^32 (2 + sqrt2)
    t = 2 ** 33 + math.isqrt(2 * 2 ** 64)       # floor(2^32 (2 + sqrt2))
    u_star = (t + 3) // 4                        # smallest U with 4U >= 2^32(2+sqrt2) (irrational: no equality)
    assert oracle_lib.decide(u_star - 1, 1, 0, 0, 2, 1, -2) == 1
    assert oracle_lib.decide(u_star, 1, 0, 0, 2, 1, -2) == 0
    # P_1 = 0 never fires ; P_1 = P_prev always fires
    assert oracle_lib.decide(0, 3, 1, -5, 0, 0, 0) == 0
    assert oracle_lib.decide(2 ** 32 - 1, 3, 1, -5, 3, 1, -5) == 1
    # irrational ratio with negative B: P_1/P_prev = (2 - sqrt2)/2 ~ 0.2929
    t = 2 ** 33 - math.isqrt(2 * 2 ** 64) - 1   # 2^32 (2 - sqrt2) lies in (t, t+1)
    u_star = t // 2 + 1                          # smallest U with 2U > 2^32 (2 - sqrt2)
    assert oracle_lib.decide(u_star - 1, 1, 0, 0, 2, -1, -1) == 1
    assert oracle_lib.decide(u_star, 1, 0, 0, 2, -1, -1) == 0


def _philox_word(oracle_lib, seed, shot, stream, index):
    out = oracle_lib.philox4x32_10((shot & 0xFFFFFFFF, shot >> 32, stream, index >> 2),
                                   (seed & 0xFFFFFFFF, seed >> 32))
    return out[index & 3]


def test_algorithm1_independent_outputs(tmp_path, oracle_lib):
    # Two random outputs in one chain, P = 1, P(m0=1) = 1/2 and
    # P(m0, m1=1) = (1/2)*(2+sqrt2)/4 (independent of m0): Algorithm 1 must
    # reduce to independent Bernoulli draws with the stated rates.
    half = (-2, 0, [])
    t1 = [(-4, 0, []), (-5, 0, [])]                 # (1/2)(1/2 + sqrt2/4)
    txt = program_text(nx=2, nr=2, nobs=2, outputs=[("R", 0, 0, 1), ("R", 1, 0, 2)],
                       chains=[0], tables=[[(0, 0, [])], [half], t1])
    p = tmp_path / "a1.prog"
    p.write_text(txt)
    prog = oracle_lib.OracleProgram(str(p))
    seed, n = 12345, 300
    rec = prog.sample(seed, 1000, n)["obs"][:, 0]
    thr1 = 2 ** 33 + math.isqrt(2 * 2 ** 64)
    for s in range(n):
        shot = 1000 + s
        u0 = _philox_word(oracle_lib, seed, shot, 1, 0)
        u1 = _philox_word(oracle_lib, seed, shot, 1, 1)
        m0 = int(u0 < 2 ** 31)
        m1 = int(4 * u1 <= thr1)   # U < 2^32 (2+sqrt2)/4
        assert int(rec[s]) == m0 | (m1 << 1)


def test_channel_thresholds_and_detector_rule(tmp_path, oracle_lib):
    # one 4-outcome channel; outcome o flips X bit o-1 (o>0); two detector
    # outputs read X bits 0 and 1 (second one complemented)
    thr = [3_000_000_000, 3_500_000_000, 4_000_000_000]
    sigs = [[0], [1], [2], [3]]
    txt = program_text(nx=2, nf=2, ndet=2, outputs=[("D", [1], 0), ("D", [2], 1)],
                       channels=[(thr, sigs)])
    p = tmp_path / "c.prog"
    p.write_text(txt)
    prog = oracle_lib.OracleProgram(str(p))
    seed, n = 7, 400
    out = prog.sample(seed, 0, n)
    for s in range(n):
        U = _philox_word(oracle_lib, seed, s, 0, 0)
        o = next((j for j, t in enumerate(thr) if U < t), 3)
        d0, d1 = o & 1, ((o >> 1) & 1) ^ 1
        assert int(out["det"][s, 0]) == d0 | (d1 << 1)
        assert int(out["accept"][s]) == int(d0 == 0 and d1 == 0)
