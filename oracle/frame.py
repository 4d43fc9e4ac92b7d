"""Pauli-frame propagation of single error bits through a Clifford circuit.

Oracle module (test infrastructure only).

Sec. "Detectors": column j of the matrix T (Eq. detector_sampling) lists
the detectors and observables that error bit e_j flips, and that matrix is
the Tanner graph of the detector error model.  For a Clifford circuit the
same columns follow from the textbook rule that a Pauli error is conjugated
through each gate and flips every Z (X) measurement whose qubit carries an X
(Z) component of the propagated Pauli.  This module computes those flip
signatures independently of any ZX rewriting.
"""
from __future__ import annotations

from .circuit import Circuit, channel_bits_to_paulis


def _conj(op, x, z):
    """Update frame bit lists x, z in place for one Clifford op."""
    n = op.name
    t = op.targets
    if n in ("I", "X", "Y", "Z"):
        return
    if n == "H":
        for q in t:
            x[q], z[q] = z[q], x[q]
    elif n in ("S", "S_DAG"):
        for q in t:
            z[q] ^= x[q]
    elif n in ("SQRT_X", "SQRT_X_DAG"):
        for q in t:
            x[q] ^= z[q]
    elif n in ("CX", "CY", "CZ", "SWAP"):
        for a, b in zip(t[::2], t[1::2]):
            if isinstance(a, tuple):
                continue  # classically controlled: handled by the caller
            if n == "CX":
                x[b] ^= x[a]
                z[a] ^= z[b]
            elif n == "CZ":
                z[a] ^= x[b]
                z[b] ^= x[a]
            elif n == "CY":
                # X_c -> X_c Y_t ; X_t -> Z_c X_t ; Z_t -> Z_c Z_t
                z[a] ^= x[b] ^ z[b]
                x[b] ^= x[a]
                z[b] ^= x[a]
            else:
                x[a], x[b] = x[b], x[a]
                z[a], z[b] = z[b], z[a]
    elif n in ("T", "T_DAG"):
        # T commutes with Z (both diagonal), so a frame without an X part on
        # the qubit passes unchanged; an X part would leave the Pauli group
        for q in t:
            if x[q]:
                raise ValueError("an X component reaches a T gate: the frame is not a Pauli")
    else:
        raise ValueError(n)


def error_bit_flips(circ: Circuit):
    """For every raw error bit, the set of measurement records it flips."""
    by_op = {}
    for ch in circ.channels:
        by_op.setdefault(ch.op_index, []).append(ch)
    # measurement index of each (op, target position)
    out = []
    for ch in circ.channels:
        for b in range(ch.nbits):
            out.append(_propagate(circ, ch, 1 << b))
    return out


def _propagate(circ: Circuit, ch, outcome):
    nq = circ.num_qubits
    x = [0] * nq
    z = [0] * nq
    flips = set()
    started = False
    mi = 0
    for idx, op in enumerate(circ.ops):
        n = op.name
        if n in ("M", "MX", "MR", "MRX"):
            for pos, q in enumerate(op.targets):
                if started:
                    f = x[q] if n in ("M", "MR") else z[q]
                    if f:
                        flips ^= {mi}
                    if n in ("M", "MR"):
                        z[q] = 0
                    else:
                        x[q] = 0
                    if n in ("MR", "MRX"):
                        x[q] = z[q] = 0
                if idx == ch.op_index and ch.kind == "MFLIP" and ch.qubits[0] == q and not started:
                    # this noisy measurement's own record flip; only one
                    # channel per target, matched by position in the op
                    if _mflip_pos(circ, ch) == pos and (outcome & 1):
                        flips ^= {mi}
                    started = True
                mi += 1
            continue
        if idx == ch.op_index and ch.kind != "MFLIP":
            for q, xb, zb in channel_bits_to_paulis(ch, outcome):
                x[q] ^= xb
                z[q] ^= zb
            started = True
            continue
        if not started:
            continue
        if n in ("R", "RX"):
            for q in op.targets:
                x[q] = z[q] = 0
        elif n in ("CX", "CY", "CZ") and any(isinstance(a, tuple) for a in op.targets[::2]):
            for a, b in zip(op.targets[::2], op.targets[1::2]):
                if isinstance(a, tuple):
                    if (mi + a[1]) in flips:
                        if n == "CX":
                            x[b] ^= 1
                        elif n == "CZ":
                            z[b] ^= 1
                        else:
                            x[b] ^= 1
                            z[b] ^= 1
                else:
                    _conj(type(op)(n, op.args, [a, b]), x, z)
        elif n in ("DETECTOR", "OBSERVABLE_INCLUDE") or n in (
                "X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "PAULI_CHANNEL_1",
                "DEPOLARIZE2", "PAULI_CHANNEL_2"):
            continue
        else:
            _conj(op, x, z)
    return flips


def _mflip_pos(circ: Circuit, ch):
    """Position, within its op, of the target a measurement-flip channel belongs to."""
    same = [c for c in circ.channels if c.op_index == ch.op_index]
    return same.index(ch)


def detector_flips(circ: Circuit):
    """Per raw error bit: (tuple of flipped detector bits, tuple of observable bits)."""
    res = []
    for flips in error_bit_flips(circ):
        d = tuple(sum(1 for j in det if j in flips) & 1 for det in circ.detectors)
        o = tuple(sum(1 for j in circ.observables[k] if j in flips) & 1
                  for k in range(circ.num_observables))
        res.append((d, o))
    return res
