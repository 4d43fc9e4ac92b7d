"""Seeded synthetic workload generators (Stim-format circuit text).

These stand in for the paper's benchmark circuits (distillation, cultivation
and random exponentiated-Pauli circuits), which are not reproduced here.
Each generator is written from the textbook description of the code it
builds; the module holds no part of the sampling method (no noise sampling,
no GF(2) or Z[w] arithmetic) and is shared by the tests, the benchmark and
the oracle comparisons.
"""
from __future__ import annotations

import math
import random


# --------------------------------------------------------------------------
# rotated surface code
# --------------------------------------------------------------------------
def rotated_surface_layout(d):
    """Data qubits (i, j), 0 <= i, j < d, and stabilizer faces.

    Face (a, b), 0 <= a, b <= d, touches data (a-1, b-1), (a-1, b), (a, b-1),
    (a, b) where they exist; faces alternate X / Z in a checkerboard
    ((a + b) even = X).  Weight-2 faces are kept on the top / bottom edges for
    X type and on the left / right edges for Z type; weight-1 corners are
    dropped.  Logical Z is Z on a row of data qubits, logical X is X on a
    column.  Each face lists its data qubits in the order NW, NE, SW, SE
    (None where absent).
    """
    data = {}
    for i in range(d):
        for j in range(d):
            data[(i, j)] = len(data)
    faces = []
    for a in range(d + 1):
        for b in range(d + 1):
            kind = "X" if (a + b) % 2 == 0 else "Z"
            corners = [(a - 1, b - 1), (a - 1, b), (a, b - 1), (a, b)]
            qs = [data.get(c) for c in corners]
            w = sum(q is not None for q in qs)
            if w < 2:
                continue
            if w == 2:
                top_bottom = a in (0, d)
                if top_bottom and kind != "X":
                    continue
                if not top_bottom and kind != "Z":
                    continue
            faces.append({"kind": kind, "pos": (a, b), "q": qs})
    return data, faces


def _cx_layers(faces, anc):
    """Four CX layers: Z faces visit NW, SW, NE, SE ('N' shape), X faces visit
    NW, NE, SW, SE ('Z' shape), so hook errors run along the logicals."""
    order = {"Z": [0, 2, 1, 3], "X": [0, 1, 2, 3]}
    layers = []
    for step in range(4):
        pairs = []
        for f, a in zip(faces, anc):
            q = f["q"][order[f["kind"]][step]]
            if q is None:
                continue
            pairs.append((a, q) if f["kind"] == "X" else (q, a))
        layers.append(pairs)
    return layers


def surface_code_t_injection(d=3, rounds=3, p=1e-3, rotation=("T",), final_basis="X", teleport=None,
                             teleport_after=None):
    """d x d rotated surface-code memory with a magic state injected at a corner.

    Round 0 prepares a product state (Li-style injection): data qubits above
    the anti-diagonal in |0>, below it in |+>, the rest of the anti-diagonal in
    |0>, and the corner injection qubit (0, d-1) in R |+>, where R is the gate
    sequence `rotation` (default: a single T, so the injected state is T|+>).
    Row 0 (logical Z) then consists of |0> qubits plus the injection qubit and
    column d-1 (logical X) of |+> qubits plus the injection qubit, so the
    logical qubit inherits the injected state.  Each of `rounds` stabilizer
    rounds uses the N-shaped CX order with DEPOLARIZE2(p) after every CX layer
    and X_ERROR(p) before every ancilla measurement; detectors compare
    consecutive rounds (first round: faces deterministic on the product state
    only).  The final data measurement is in `final_basis` with Z_ERROR(p) or
    X_ERROR(p) before it; its faces give the last detectors and the matching
    logical operator is observable 0.
    teleport: a second gate sequence, applied to the logical qubit by gate
    teleportation after round `teleport_after` (default: the middle round):
    a free ancilla m is prepared in teleport |+>, the joint parity Z_L Z_m is
    measured through a second free ancilla (CX from every qubit of the
    logical-Z row and from m), m is measured in X, and the Pauli part of the
    teleportation correction, Z_L conditioned on that X outcome, is applied by
    classically controlled CZ gates (the Clifford part is left out, so the
    logical receives the sequence or its inverse, as the parity says).  The
    parity measurement commutes with every stabilizer, so all detectors stay
    deterministic.  Returns Stim text.
    """
    data, faces = rotated_surface_layout(d)
    nd = len(data)
    anc = [nd + k for k in range(len(faces))]
    L = []
    inj = data[(0, d - 1)]
    plus = [data[(i, j)] for (i, j) in data if i + j > d - 1]
    zero = [data[(i, j)] for (i, j) in data if i + j <= d - 1 and data[(i, j)] != inj]
    L.append("R " + " ".join(map(str, sorted(zero + anc))))
    L.append("RX " + " ".join(map(str, sorted(plus + [inj]))))
    for g in rotation:
        L.append(f"{g} {inj}")
    xa = [a for f, a in zip(faces, anc) if f["kind"] == "X"]
    layers = _cx_layers(faces, anc)
    state = {q: "0" for q in zero}
    state.update({q: "+" for q in plus})
    state[inj] = "T"

    tele_done_after = -2

    def deterministic_first(f):
        want = "+" if f["kind"] == "X" else "0"
        return all(q is None or state[q] == want for q in f["q"])

    nf = len(faces)
    if teleport is not None and teleport_after is None:
        teleport_after = max(0, rounds // 2 - 1)
    for r in range(rounds):
        if xa:
            L.append("H " + " ".join(map(str, xa)))
        for layer in layers:
            flat = [x for pr in layer for x in pr]
            L.append("CX " + " ".join(map(str, flat)))
            L.append(f"DEPOLARIZE2({p}) " + " ".join(map(str, flat)))
        if xa:
            L.append("H " + " ".join(map(str, xa)))
        L.append(f"X_ERROR({p}) " + " ".join(map(str, anc)))
        L.append("MR " + " ".join(map(str, anc)))
        for k, f in enumerate(faces):
            cur = f"rec[-{nf - k}]"
            if r == 0:
                if deterministic_first(f):
                    L.append(f"DETECTOR {cur}")
            elif tele_done_after == r - 1:
                # the teleportation's two measurements sit between the rounds
                L.append(f"DETECTOR {cur} rec[-{2 * nf + 2 - k}]")
            else:
                L.append(f"DETECTOR {cur} rec[-{2 * nf - k}]")
        if teleport is not None and r == teleport_after:
            m, a = anc[0], anc[1]           # free between rounds (reset by MR)
            row0 = [data[(0, j)] for j in range(d)]
            L.append(f"RX {m}")
            for g in teleport:
                L.append(f"{g} {m}")
            L.append(f"DEPOLARIZE1({p}) {m}")
            for q in row0 + [m]:
                L.append(f"CX {q} {a}")
                L.append(f"DEPOLARIZE2({p}) {q} {a}")
            L.append(f"X_ERROR({p}) {a}")
            L.append(f"MR {a}")
            L.append(f"Z_ERROR({p}) {m}")
            L.append(f"MX {m}")
            L.append(f"R {m}")
            for q in row0:
                L.append(f"CZ rec[-1] {q}")
            tele_done_after = r
    flip = "X_ERROR" if final_basis == "Z" else "Z_ERROR"
    L.append(f"{flip}({p}) " + " ".join(map(str, range(nd))))
    L.append(("M " if final_basis == "Z" else "MX ") + " ".join(map(str, range(nd))))
    last_gap = 2 if tele_done_after == rounds - 1 else 0
    for k, f in enumerate(faces):
        if f["kind"] != final_basis:
            continue
        recs = [f"rec[-{nd - q}]" for q in f["q"] if q is not None]
        recs.append(f"rec[-{nd + last_gap + nf - k}]")
        L.append("DETECTOR " + " ".join(recs))
    if final_basis == "Z":
        logical = [data[(0, j)] for j in range(d)]
    else:
        logical = [data[(i, d - 1)] for i in range(d)]
    L.append("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{nd - q}]" for q in logical))
    return "\n".join(L) + "\n"


def t_rotation_sequence(n_t, seed=0):
    """A seeded single-qubit Clifford+T word with n_t T/T_DAG gates, each
    followed by H or SQRT_X so that consecutive T gates do not fuse."""
    rng = random.Random(seed)
    seq = []
    for k in range(n_t):
        seq.append(rng.choice(["T", "T_DAG"]))
        seq.append(rng.choice(["H", "SQRT_X"]) if k + 1 < n_t else "H")
    return tuple(seq)


# --------------------------------------------------------------------------
# d=3 triangular colour code (Steane code) T-check
# --------------------------------------------------------------------------
STEANE_FACES = ([0, 1, 2, 3], [1, 2, 4, 5], [2, 3, 5, 6])
STEANE_LOGICAL = [0, 1, 4]  # X_L = X0 X1 X4, Z_L = Z0 Z1 Z4


def color_code_t_check(rounds=3, p=1e-3, check=True, inject="T_DAG"):
    """d=3 triangular colour code with a T state and transversal T-checks.

    Qubits: data 0-6, syndrome ancillas 7-9 (X plaquettes) and 10-12
    (Z plaquettes), flags 13-18 (one per syndrome ancilla): 19 qubits.
    Encoding: the T state T|+> on data 0 is copied onto the logical-X support
    {0, 1, 4} and the three X plaquette operators are superposed from pivots
    3, 5, 6 (unitary Steane encoder).  Each round: a T-check (T_DAG on all
    data, X-parity of all data measured through ancilla 7 prepared in |+>,
    T on all data: 14 T/T_DAG), then one flagged measurement of the six
    plaquette stabilizers.  DEPOLARIZE1(p) after single-qubit gates,
    DEPOLARIZE2(p) after CX, X_ERROR(p) before measurements.  Detectors:
    check outcomes, flags, first-round stabilizers and round-to-round
    changes; the final data measurement in X gives the X-plaquette detectors
    and observable X_L.  With check=False the T-checks are left out.
    """
    data = list(range(7))
    xa, za = [7, 8, 9], [10, 11, 12]
    fl = list(range(13, 19))
    L = [f"R {' '.join(map(str, range(19)))}", "H 0", f"{inject} 0", f"DEPOLARIZE1({p}) 0"]
    # unitary encoder
    L.append("H 3 5 6")
    L.append(f"DEPOLARIZE1({p}) 3 5 6")
    for c, ts in ((0, [1, 4]), (3, [0, 1, 2]), (5, [1, 2, 4]), (6, [2, 3, 5])):
        for t in ts:
            L.append(f"CX {c} {t}")
            L.append(f"DEPOLARIZE2({p}) {c} {t}")
    nmeas = 0
    stab_rec = {}  # stabilizer key -> measurement index of its last value
    for r in range(rounds):
        if check:
            L.append("T_DAG " + " ".join(map(str, data)))
            L.append(f"DEPOLARIZE1({p}) " + " ".join(map(str, data)))
            L.append("RX 7")
            for d in data:
                L.append(f"CX 7 {d}")
                L.append(f"DEPOLARIZE2({p}) 7 {d}")
            L.append(f"Z_ERROR({p}) 7")
            L.append("MX 7")
            nmeas += 1
            L.append("DETECTOR rec[-1]")
            L.append("T " + " ".join(map(str, data)))
            L.append(f"DEPOLARIZE1({p}) " + " ".join(map(str, data)))
        # flagged stabilizer round
        L.append("R " + " ".join(map(str, za + fl[:3])))
        L.append("RX " + " ".join(map(str, xa + fl[3:])))
        for k, face in enumerate(STEANE_FACES):
            a, f = xa[k], fl[k]          # X plaquette: ancilla |+>, CX anc -> data, flag |0>
            b, g = za[k], fl[3 + k]      # Z plaquette: ancilla |0>, CX data -> anc, flag |+>
            seq = [(a, face[0]), (a, f), (a, face[1]), (a, face[2]), (a, f), (a, face[3])]
            seq += [(face[0], b), (g, b), (face[1], b), (face[2], b), (g, b), (face[3], b)]
            for c, t in seq:
                L.append(f"CX {c} {t}")
                L.append(f"DEPOLARIZE2({p}) {c} {t}")
        L.append(f"Z_ERROR({p}) " + " ".join(map(str, xa + fl[3:])))
        L.append(f"X_ERROR({p}) " + " ".join(map(str, za + fl[:3])))
        order = xa + za + fl
        L.append("MX " + " ".join(map(str, xa)))
        L.append("M " + " ".join(map(str, za)))
        L.append("M " + " ".join(map(str, fl[:3])))
        L.append("MX " + " ".join(map(str, fl[3:])))
        base = nmeas
        nmeas += 12
        idx = {q: base + i for i, q in enumerate(order)}
        for q in fl:
            L.append(f"DETECTOR rec[{idx[q] - nmeas}]")
        for k in range(3):
            for kind, anc in (("X", xa[k]), ("Z", za[k])):
                key = (kind, k)
                cur = f"rec[{idx[anc] - nmeas}]"
                if key in stab_rec:
                    L.append(f"DETECTOR {cur} rec[{stab_rec[key] - nmeas}]")
                else:
                    L.append(f"DETECTOR {cur}")
                stab_rec[key] = idx[anc]
    L.append(f"Z_ERROR({p}) " + " ".join(map(str, data)))
    L.append("MX " + " ".join(map(str, data)))
    nmeas += 7
    for k, face in enumerate(STEANE_FACES):
        recs = [f"rec[{nmeas - 7 + q - nmeas}]" for q in face]
        recs.append(f"rec[{stab_rec[('X', k)] - nmeas}]")
        L.append("DETECTOR " + " ".join(recs))
    L.append("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[{nmeas - 7 + q - nmeas}]" for q in STEANE_LOGICAL))
    return "\n".join(L) + "\n"


# --------------------------------------------------------------------------
# random noisy Clifford+T circuits (batched-launch workload)
# --------------------------------------------------------------------------
_INV = {"H": "H", "S": "S_DAG", "S_DAG": "S", "SQRT_X": "SQRT_X_DAG", "SQRT_X_DAG": "SQRT_X",
        "X": "X", "Z": "Z", "T": "T_DAG", "T_DAG": "T", "CX": "CX", "CZ": "CZ"}


def random_clifford_t(seed, n=None, depth=None, t_count=None, p=None):
    """A seeded random noisy Clifford+T mirror circuit.

    n qubits in U[20, 60], depth in U[20, 100] layers (half a random circuit U,
    half its inverse U^-1, so the noiseless output is all zeros), t_count
    T/T_DAG gates in U[8, 40] (half in U at random positions, mirrored in
    U^-1), a two-qubit gate density of 0.3 per layer (fraction of qubits
    covered by CX/CZ pairs on random partners), random single-qubit Cliffords
    on the other qubits, depolarising p in U[1e-4, 3e-3] after every layer
    and X_ERROR(p) before the final Z measurement of every qubit.  Every
    measurement is a detector; observable 0 is the parity of qubits 0-2.
    """
    rng = random.Random(seed)
    n = n if n is not None else rng.randint(20, 60)
    depth = depth if depth is not None else rng.randint(20, 100)
    t_count = t_count if t_count is not None else rng.randint(8, 40)
    p = p if p is not None else rng.uniform(1e-4, 3e-3)
    half = max(1, depth // 2)
    t_pos = set()
    while len(t_pos) < min(max(1, t_count // 2), n * half):
        t_pos.add((rng.randrange(half), rng.randrange(n)))
    one_q = ["H", "S", "S_DAG", "SQRT_X", "SQRT_X_DAG", "X", "Z"]
    layers = []
    for layer in range(half):
        qs = list(range(n))
        rng.shuffle(qs)
        n_pair = int(round(0.3 * n / 2))
        ops = [(rng.choice(["CX", "CZ"]), (qs[2 * k], qs[2 * k + 1])) for k in range(n_pair)]
        ops += [(rng.choice(one_q), (q,)) for q in qs[2 * n_pair:]]
        ops += [(rng.choice(["T", "T_DAG"]), (q,)) for q in range(n) if (layer, q) in t_pos]
        layers.append(ops)

    def emit(ops, L):
        pairs = [x for g, t in ops if len(t) == 2 for x in t]
        singles = sorted({t[0] for g, t in ops if len(t) == 1})
        for g, t in ops:
            L.append(f"{g} " + " ".join(map(str, t)))
        if pairs:
            L.append(f"DEPOLARIZE2({p:.6g}) " + " ".join(map(str, pairs)))
        if singles:
            L.append(f"DEPOLARIZE1({p:.6g}) " + " ".join(map(str, singles)))

    L = ["R " + " ".join(map(str, range(n)))]
    for ops in layers:
        emit(ops, L)
    for ops in reversed(layers):
        emit([(_INV[g], t) for g, t in reversed(ops)], L)
    L.append(f"X_ERROR({p:.6g}) " + " ".join(map(str, range(n))))
    L.append("M " + " ".join(map(str, range(n))))
    for q in range(n):
        L.append(f"DETECTOR rec[-{n - q}]")
    L.append("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{n - q}]" for q in range(min(3, n))))
    return "\n".join(L) + "\n"


# --------------------------------------------------------------------------
# named configurations
# --------------------------------------------------------------------------
def config1_circuit(p=1e-3):
    """d=3 rotated surface code, 17 qubits, 3 rounds, one injected logical T."""
    return surface_code_t_injection(d=3, rounds=3, p=p, rotation=("T",))


def config2_circuit(p=1e-3, n_t=16, seed=0):
    """d=5 rotated surface code, 49 qubits, 5 rounds, 16 T/T_DAG gates: two
    injected logical rotations of n_t/2 T/T_DAG each, the first by the corner
    injection of round 0, the second by gate teleportation after round 2
    (Pauli corrections by classically controlled CZ)."""
    half = n_t // 2
    return surface_code_t_injection(d=5, rounds=5, p=p, rotation=t_rotation_sequence(half, seed),
                                    teleport=t_rotation_sequence(n_t - half, seed + 1), teleport_after=2)


def config3_circuit(p=1e-3):
    """d=3 triangular colour-code T-check, 19 qubits, 3 check rounds, 42 T/T_DAG."""
    return color_code_t_check(rounds=3, p=p)


def config4_batch(n=256, seed=0):
    """(circuit, shots) pairs of the batched-launch workload: seeded random
    mirror circuits (see random_clifford_t) with shot counts drawn
    log-uniformly from 1e3 to 1e6.  Circuit k uses generator seed
    seed * 100003 + k; the caller may skip circuits it cannot compile and
    draw more with larger k."""
    rng = random.Random(seed)
    out = []
    for k in range(n):
        shots = int(round(10 ** rng.uniform(3, 6)))
        out.append((random_clifford_t(seed * 100003 + k), shots))
    return out


def count_t(text):
    n = 0
    for line in text.splitlines():
        parts = line.split()
        if parts and parts[0] in ("T", "T_DAG"):
            n += len(parts) - 1
    return n


# --------------------------------------------------------------------------
# learned cut order: circuits of the network's training family
# --------------------------------------------------------------------------
def layered_clifford_t(seed, q, t_count, p=1e-3, cx_density=0.4):
    """A seeded random Clifford+T circuit of the family the cut-order network
    is trained on: layers of CX pairs on random partners (cx_density of the
    qubits) and single-qubit gates on the others (T or T_DAG with probability
    1/4, else H, S, S_DAG or SQRT_X) until t_count T/T_DAG gates are placed,
    DEPOLARIZE1(p) after every layer, Z measurement of every qubit.  No
    detectors: it is sampled in measurement mode."""
    rng = random.Random(seed)
    one_q = ["H", "S", "S_DAG", "SQRT_X"]
    L = ["R " + " ".join(map(str, range(q)))]
    placed = 0
    while placed < t_count:
        qs = list(range(q))
        rng.shuffle(qs)
        pairs = int(cx_density * q / 2 + 0.5)
        for k in range(pairs):
            L.append(f"CX {qs[2 * k]} {qs[2 * k + 1]}")
        for qb in qs[2 * pairs:]:
            if rng.random() < 0.25 and placed < t_count:
                L.append(f"{rng.choice(['T', 'T_DAG'])} {qb}")
                placed += 1
            else:
                L.append(f"{rng.choice(one_q)} {qb}")
        L.append(f"DEPOLARIZE1({p:.6g}) " + " ".join(map(str, range(q))))
    L.append("M " + " ".join(map(str, range(q))))
    return "\n".join(L) + "\n"


def config5_pool(n, seed=1, q_range=(3, 10), t_range=(40, 60)):
    """(circuit, shots) pairs for the learned-cut-order comparison: circuits
    of the training family (layered_clifford_t) with config-3-sized T counts
    (40-60 T/T_DAG), drawn from generator seeds the training set does not
    use (seed * 1000003 + k + 7).  1e5 shots each."""
    rng = random.Random(seed)
    out = []
    for k in range(n):
        q = rng.randint(*q_range)
        t = rng.randint(*t_range)
        out.append((layered_clifford_t(seed * 1000003 + k + 7, q, t), 100_000))
    return out
