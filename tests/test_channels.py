"""Pins of channel reduction (Appendix "Channel reduction") against closed
forms: independent flips of the same detector merge into one channel whose
flip probability is the XOR convolution p1 (1 - p2) + p2 (1 - p1), error
components that flip nothing vanish, and the stored thresholds are
floor(cdf 2^32)."""
import math

import pytest

import paper_2604_01059_gb300 as T
from tests import progfile


def _channels(tmp_path, text):
    prog = T.Program(text)
    path = str(tmp_path / "c.prog")
    prog.save(path)
    return progfile.read(path)["channels"]


def _thr(p_none):
    return min(2 ** 32 - 1, math.floor(p_none * 2 ** 32))


@pytest.mark.parametrize("p1,p2", [(0.1, 0.2), (1e-3, 3e-3), (0.5, 0.25)])
def test_two_bit_flips_merge(tmp_path, p1, p2):
    chans = _channels(tmp_path, f"X_ERROR({p1}) 0\nX_ERROR({p2}) 0\nM 0\nDETECTOR rec[-1]\n")
    assert len(chans) == 1
    thr, sigs = chans[0]
    assert len(sigs) == 2 and not any(sigs[0])       # outcome 0 flips nothing
    p_none = (1 - p1) * (1 - p2) + p1 * p2            # no flip, or both
    assert abs(thr[0] - _thr(p_none)) <= 1


def test_depolarizing_components_that_flip_nothing_vanish(tmp_path):
    # DEPOLARIZE1(p) before a Z measurement: X and Y flip it (p/3 each), Z
    # does not; with X_ERROR(q) the detector flips with
    # q (1 - 2p/3) + (2p/3)(1 - q)
    p, q = 0.06, 0.01
    chans = _channels(tmp_path, f"X_ERROR({q}) 0\nDEPOLARIZE1({p}) 0\nM 0\nDETECTOR rec[-1]\n")
    assert len(chans) == 1
    thr, sigs = chans[0]
    assert len(sigs) == 2
    f = 2 * p / 3
    assert abs(thr[0] - _thr(1 - (q * (1 - f) + f * (1 - q)))) <= 1


def test_independent_detectors_stay_separate(tmp_path):
    chans = _channels(tmp_path, "X_ERROR(0.1) 0\nX_ERROR(0.2) 1\nM 0 1\nDETECTOR rec[-2]\nDETECTOR rec[-1]\n")
    assert len(chans) == 2
    got = sorted(c[0][0] for c in chans)
    want = sorted([_thr(0.9), _thr(0.8)])
    assert all(abs(a - b) <= 1 for a, b in zip(got, want))
