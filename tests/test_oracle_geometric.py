"""Pins for the oracle's geometric-gap noise rule (Sec. "Detectors": the gap
between successive firing events is drawn from a geometric distribution).

The rule draws, per group of channels, gaps with P(gap >= k) close to
(Q/2^32)^k, and at a candidate channel maps a word V onto [Q, 2^32) before
the channel's own thresholds decide.  The pins check, through the oracle's
own functions:
  - the gap law against the closed form (Q/2^32)^k, counting the words U
    exactly (the gap is monotone in U, so its breakpoints are found by
    bisection over all 2^32 words);
  - the candidate's outcome law against the conditional distribution of the
    channel given that it is a candidate;
  - end to end on a small program, the per-channel firing rates and their
    independence against the exact product distribution, in both noise
    modes (a dropped offset, a shifted candidate or a wrong mapping moves a
    rate by far more than the sampling error).
"""
from fractions import Fraction

import numpy as np
import pytest

from tests.progtext import program_text

TWO32 = 1 << 32


def _first_word_below(f, k):
    """Smallest U in [0, 2^32] with f(U) < k, for f non-increasing in U
    (2^32 when every word has f(U) >= k): the number of words with f >= k."""
    lo, hi = 0, TWO32
    while lo < hi:
        mid = (lo + hi) // 2
        if f(mid) < k:
            hi = mid
        else:
            lo = mid + 1
    return lo


@pytest.mark.parametrize("Q", [TWO32 - (1 << 22), (9 * TWO32) // 10, TWO32 // 2, 12345, 0])
def test_gap_law_is_geometric(oracle_lib, Q):
    m = 5000
    gap = lambda U: oracle_lib.geo_gap(Q, m, U)  # noqa: E731
    q = Fraction(Q, TWO32)
    assert gap(TWO32 - 1) == 0 or Q == TWO32 - 1
    for k in [1, 2, 3, 7, 50, 1000, 4999]:
        count = _first_word_below(gap, k)  # words U with gap(U) >= k
        exact = q ** k
        # each of the k rounding steps loses less than one unit of 2^-32
        assert abs(Fraction(count, TWO32) - exact) <= Fraction(k, TWO32), (Q, k)
    # the gap never exceeds the channels left, and is 0 with none left
    for U in (0, 1, Q // 2, TWO32 - 1):
        assert 0 <= oracle_lib.geo_gap(Q, 3, U) <= 3
        assert oracle_lib.geo_gap(Q, 0, U) == 0


@pytest.mark.parametrize("Q,thr", [
    (4294000000, [4294500000, 4294700000, 4294900000]),
    (4290000000, [4290000000, 4292000000, 4294900000]),   # Q equal to the outcome-0 threshold
    (2 ** 31, [3 * 2 ** 30, 3 * 2 ** 30 + 5]),
    (0, [100, 2 ** 31]),
])
def test_candidate_outcome_law(oracle_lib, Q, thr):
    n_out = len(thr) + 1
    pick = lambda V: oracle_lib.geo_pick(Q, thr, V)  # noqa: E731
    bounds = [Q] + list(thr) + [TWO32]   # outcome o covers mapped words [bounds[o], bounds[o+1])
    R = TWO32 - Q
    assert pick(0) == next(o for o in range(n_out) if bounds[o + 1] > Q)
    assert pick(TWO32 - 1) == n_out - 1
    prev = 0
    for o in range(n_out):
        # words V whose outcome is <= o: the outcome is non-decreasing in V
        upto = _first_word_below(lambda V: -pick(V), -o)
        cnt = upto - prev
        prev = upto
        want = Fraction(bounds[o + 1] - bounds[o], R)
        assert abs(Fraction(cnt, TWO32) - want) < Fraction(1, TWO32), (o, cnt)
    assert prev == TWO32


def _flip_program(probs, groups):
    """One detector per channel; channel c fires (outcome 1 of 2) with
    probability probs[c] and flips detector c; a last 3-outcome channel
    flips detector 0 (outcome 1) or detectors 0 and 1 (outcome 2)."""
    n = len(probs)
    channels = []
    for c, p in enumerate(probs):
        thr = int(np.floor((1 - p) * TWO32))
        channels.append(([thr], [[0], [1 << c]]))
    channels.append(([int(0.8 * TWO32), int(0.9 * TWO32)], [[0], [1], [3]]))
    outputs = [("D", [1 << c], 0) for c in range(n)]
    return program_text(nx=n, nf=n, ndet=n, outputs=outputs, channels=channels, groups=groups), channels


@pytest.mark.parametrize("geometric", [False, True])
def test_firing_rates_match_product_distribution(tmp_path, oracle_lib, geometric):
    probs = [0.3, 0.2, 0.12, 0.05, 0.3, 0.001]
    n = len(probs)
    _, channels = _flip_program(probs, None)
    groups = None
    if geometric:
        # groups as the compiler would form them (within a factor 2), plus the
        # 3-outcome channel with the first group; Q = lowest outcome-0 threshold
        thr0 = [ch[0][0] for ch in channels]
        members = [[0, 4, 1, n], [2], [3], [5]]
        groups = [(min(thr0[c] for c in m), m) for m in members]
    txt, _ = _flip_program(probs, groups)
    path = tmp_path / "flips.prog"
    path.write_text(txt)
    prog = oracle_lib.OracleProgram(str(path))
    assert prog.noise_mode == (1 if geometric else 0)
    N = 400_000
    det = prog.sample(7, 0, N)["det"][:, 0]
    bits = np.array([(det >> c) & 1 for c in range(n)], dtype=np.float64)
    # exact rates of the quantised channels (2^-32 units) and the extra channel
    pc = [(TWO32 - ch[0][0]) / TWO32 for ch in channels[:n]]
    extra = channels[n][0]
    p1 = (extra[1] - extra[0]) / TWO32
    p2 = (TWO32 - extra[1]) / TWO32
    want = list(pc)
    want[0] = pc[0] * (1 - p1 - p2) + (1 - pc[0]) * (p1 + p2)   # XOR with outcomes 1 and 2
    want[1] = pc[1] * (1 - p2) + (1 - pc[1]) * p2               # XOR with outcome 2
    for c in range(n):
        got = bits[c].mean()
        sd = np.sqrt(want[c] * (1 - want[c]) / N)
        assert abs(got - want[c]) < 5 * sd + 1e-9, (c, got, want[c])
    # independence of channels in one group and across groups
    for a, b in [(0, 4), (1, 4), (2, 4), (3, 4), (2, 3), (4, 5)]:
        joint = (bits[a] * bits[b]).mean()
        w = want[a] * want[b]
        sd = np.sqrt(w * (1 - w) / N)
        assert abs(joint - w) < 5 * sd + 1e-9, (a, b, joint, w)


def test_reader_rejects_inconsistent_groups(tmp_path, oracle_lib):
    probs = [0.3, 0.2]
    _, channels = _flip_program(probs, None)
    bad = [
        [(channels[0][0][0] + 1, [0, 1, 2])],    # Q above a member's outcome-0 threshold
        [(0, [0, 1])],                           # channel 2 in no group
        [(0, [0, 1, 2, 1])],                     # channel 1 twice
    ]
    for groups in bad:
        txt, _ = _flip_program(probs, groups)
        path = tmp_path / "bad.prog"
        path.write_text(txt)
        with pytest.raises(RuntimeError):
            oracle_lib.OracleProgram(str(path))
