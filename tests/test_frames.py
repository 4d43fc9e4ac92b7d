"""The compiled T matrix against the oracle's Pauli-frame propagation.

Sec. "Detectors": column j of T (Eq. detector_sampling) lists the detectors
and observables that error bit e_j flips; for Clifford circuits that is the
Tanner graph that propagating a single Pauli through the circuit gives.  The
product's side is tsim_raw_to_x (X = T e for the raw error bits) followed by
each deterministic output's mask; the oracle's side is oracle/frame.py, which
conjugates each error through the gates and shares nothing with the ZX
compiler.  Checked column for column on the benchmark circuits whose T gates
all precede the noise (configs 1 and 2), on Clifford variants of configs 1-3
(S for T), and on surface-code memories of distance 7, 9 and 11.  Every
noiseless detector of these circuits is 0.
"""
import pytest

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle import circuit as ocirc
from oracle import frame
from tests import progfile


def _s_for_t(text):
    out = []
    for line in text.splitlines():
        parts = line.split()
        if parts and parts[0] in ("T", "T_DAG"):
            parts[0] = "S" if parts[0] == "T" else "S_DAG"
        out.append(" ".join(parts))
    return "\n".join(out) + "\n"


CASES = [
    ("cfg1", lambda: Wk.config1_circuit(p=1e-3)),
    ("cfg1_clifford", lambda: _s_for_t(Wk.config1_circuit(p=1e-3))),
    ("cfg2", lambda: Wk.config2_circuit(p=1e-3)),
    ("cfg2_s_for_t", lambda: _s_for_t(Wk.config2_circuit(p=1e-3))),
    ("cfg3_clifford", lambda: Wk.color_code_t_check(rounds=3, p=1e-3, check=False, inject="S_DAG")),
    ("mem_d7", lambda: Wk.surface_code_t_injection(d=7, rounds=3, p=1e-3, rotation=())),
    ("mem_d9", lambda: Wk.surface_code_t_injection(d=9, rounds=2, p=1e-3, rotation=())),
    ("mem_d11", lambda: Wk.surface_code_t_injection(d=11, rounds=2, p=1e-3, rotation=())),
]


def _parity(mask, x):
    v = 0
    for m, w in zip(mask, x):
        v ^= m & w
    return bin(v).count("1") & 1


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_t_matrix_equals_frame_flips(tmp_path, name, make):
    text = make()
    prog = T.Program(text)
    path = str(tmp_path / "p.prog")
    prog.save(path)
    pf = progfile.read(path)
    info = prog.info
    nd, no = info["num_detectors"], info["num_observables"]
    outs = pf["outputs"]
    # every detector is deterministic, and 0 without noise
    for i in range(nd):
        assert outs[i][0] == "D", (name, i)
        assert outs[i][2] == 0, (name, i)
    c = ocirc.parse(text)
    assert c.num_error_bits == info["num_error_bits"]
    flips = frame.detector_flips(c)
    W = info["x_words"]
    compared = 0
    for j in range(c.num_error_bits):
        e = [0] * c.num_error_bits
        e[j] = 1
        x = T.tsim_raw_to_x(prog.h, e, W)
        fd, fo = flips[j]
        want = list(fd) + list(fo)
        for i, o in enumerate(outs):
            if o[0] != "D":
                continue  # a random output (the injected logical): no flip column
            assert _parity(o[1], x) == want[i], (name, j, i)
            compared += 1
    assert compared >= nd * c.num_error_bits
