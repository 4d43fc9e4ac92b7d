"""Groups of the geometric-gap noise rule, checked on the host.

The rule is exact for any cut of the channels into groups whose Q does not
exceed any member's outcome-0 threshold (Sec. "Detectors"; the oracle's
reader rejects any other).  The compiler cuts the channels, sorted by firing
probability, where the expected random words per shot (one per group, two
per candidate) are fewest.  Checked here: every channel that can fire is in
exactly one group, each group's Q is its most likely member's threshold, and
on programs small enough to enumerate every cut of the sorted channels, no
cut draws fewer expected words than the compiler's."""
import itertools

import pytest

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from tests import progfile

TWO32 = 1 << 32


def _groups(tmp_path, text, mode=T.MODE_DETECTORS):
    prog = T.Program(text, mode=mode)
    prog.set_noise_sampling(1)
    path = str(tmp_path / "p.prog")
    prog.save(path)
    pf = progfile.read(path)
    return pf["channels"], pf["groups"]


def _words(runs, fire):
    # one gap word per group, two per expected candidate
    return sum(1 + 2 * len(r) * fire[r[0]] / TWO32 for r in runs)


@pytest.mark.parametrize("text", [Wk.config1_circuit(p=2e-3), Wk.config2_circuit(p=1e-3), Wk.config3_circuit()],
                         ids=["config1", "config2", "config3"])
def test_groups_partition_the_firing_channels(tmp_path, text):
    channels, groups = _groups(tmp_path, text)
    firing = {c for c, (thr, _) in enumerate(channels) if thr}
    seen = [c for _, members in groups for c in members]
    assert sorted(seen) == sorted(firing)
    for q, members in groups:
        thr0 = [channels[c][0][0] for c in members]
        assert q == min(thr0)  # the most likely member leads
        assert members == sorted(members)


def _small_circuit(seed):
    # a few noisy channels of different strengths on four qubits
    ps = [1e-3, 2e-3, 5e-3, 3e-2, 8e-2][: 2 + seed % 4]
    lines = ["R 0 1 2 3", "H 0", "CX 0 1", "T 1", "CX 1 2", "T_DAG 2", "CX 2 3"]
    for k, p in enumerate(ps):
        lines.append(f"DEPOLARIZE1({p}) {k % 4}")
        lines.append(f"X_ERROR({p / 2}) {(k + 1) % 4}")
    lines.append("M 0 1 2 3")
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("seed", range(6))
def test_cuts_are_the_fewest_words(tmp_path, seed):
    channels, groups = _groups(tmp_path, _small_circuit(seed), T.MODE_MEASUREMENTS)
    fire = {c: TWO32 - thr[0] for c, (thr, _) in enumerate(channels) if thr}
    order = sorted(fire, key=lambda c: -fire[c])
    assert 2 <= len(order) <= 14
    got = sum(1 + 2 * len(m) * (TWO32 - q) / TWO32 for q, m in groups)
    best = min(_words([order[a:b] for a, b in zip((0,) + cuts, cuts + (len(order),))], fire)
               for k in range(len(order))
               for cuts in itertools.combinations(range(1, len(order)), k))
    assert got == pytest.approx(best, rel=1e-12)
