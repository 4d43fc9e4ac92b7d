"""Stim-subset circuit reader and raw noise-channel enumeration.

Oracle module (test infrastructure only).  Written independently of the
product's C++ parser; both follow the instruction set the paper names
(Sec. "Methods": the Stim circuit format extended with T and T_DAG) and the
noise-bit encoding of Appendix "Pauli noise channels":

* a single-qubit Pauli channel uses two bits (e_x, e_z); outcome (1,0) has
  probability p_x, (1,1) p_y, (0,1) p_z and (0,0) the remainder;
* a two-qubit channel uses four bits (x_a, z_a, x_b, z_b), "constructed
  analogously";
* X_ERROR / Z_ERROR / Y_ERROR use one bit; a noisy measurement M(p) uses one
  bit that flips the recorded outcome.

Raw channels are numbered in circuit order (instruction order, then target
order); raw error bits are numbered channel after channel, bit 0 of a channel
first.  The outcome index of a channel is  sum_i bit_i << i.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
import re

ONE_Q = {"I", "X", "Y", "Z", "H", "S", "S_DAG", "SQRT_X", "SQRT_X_DAG", "T", "T_DAG"}
ROTATIONS = {"R_X", "R_Y", "R_Z", "U3"}  # angles in units of pi (Sec. "Methods")
ALIASES = {"CNOT": "CX", "ZCX": "CX", "ZCZ": "CZ", "ZCY": "CY", "SQRT_Z": "S",
           "SQRT_Z_DAG": "S_DAG", "H_XZ": "H", "MZ": "M", "RZ": "R", "MRZ": "MR"}
TWO_Q = {"CX", "CY", "CZ", "SWAP"}
MEAS = {"M", "MX", "MR", "MRX"}
RESETS = {"R", "RX"}
NOISE1 = {"X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "PAULI_CHANNEL_1"}
NOISE2 = {"DEPOLARIZE2", "PAULI_CHANNEL_2"}
IGNORED = {"TICK", "QUBIT_COORDS", "SHIFT_COORDS"}

# Stim's order of the 15 two-qubit Paulis for PAULI_CHANNEL_2
_PC2_ORDER = ["IX", "IY", "IZ", "XI", "XX", "XY", "XZ", "YI", "YX", "YY", "YZ",
              "ZI", "ZX", "ZY", "ZZ"]
_PAULI_BITS = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}


@dataclass
class Op:
    name: str
    args: list
    targets: list  # ints (qubits) or ("rec", -k)


@dataclass
class RawChannel:
    """One noise channel: its error bits and their joint distribution."""
    kind: str
    qubits: tuple
    nbits: int
    probs: list            # Fraction per outcome index
    op_index: int          # position of the op in the flat op list
    first_bit: int = 0     # global index of bit 0


@dataclass
class Circuit:
    ops: list = field(default_factory=list)
    num_qubits: int = 0
    num_measurements: int = 0
    detectors: list = field(default_factory=list)     # list of lists of measurement indices
    observables: dict = field(default_factory=dict)   # obs index -> list of measurement indices
    channels: list = field(default_factory=list)      # RawChannel in circuit order
    num_error_bits: int = 0

    @property
    def num_detectors(self):
        return len(self.detectors)

    @property
    def num_observables(self):
        return 0 if not self.observables else max(self.observables) + 1


def _frac(x: str) -> Fraction:
    return Fraction(x)


def _tokenize_lines(text):
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if line:
            yield line


_LINE = re.compile(r"^([A-Za-z_0-9]+)(?:\(([^)]*)\))?\s*(.*)$")


def _parse_block(lines, pos, end_brace):
    out = []
    while pos < len(lines):
        line = lines[pos]
        if line == "}":
            if not end_brace:
                raise ValueError("unbalanced }")
            return out, pos + 1
        m = _LINE.match(line)
        if not m:
            raise ValueError(f"cannot parse line: {line!r}")
        name = m.group(1).upper()
        argstr = m.group(2)
        rest = m.group(3).strip()
        if name == "REPEAT":
            if not rest.endswith("{"):
                raise ValueError("REPEAT needs '{'")
            count = int(rest[:-1].strip())
            body, pos = _parse_block(lines, pos + 1, True)
            for _ in range(count):
                out.extend(body)
            continue
        args = [a.strip() for a in argstr.split(",")] if argstr else []
        targets = []
        for tok in rest.split():
            if tok.startswith("rec[") and tok.endswith("]"):
                targets.append(("rec", int(tok[4:-1])))
            else:
                targets.append(int(tok))
        out.append(Op(ALIASES.get(name, name), args, targets))
        pos += 1
    if end_brace:
        raise ValueError("missing }")
    return out, pos


def _pc1_probs(px, py, pz):
    # outcome index = e_x + 2 e_z ; (1,0)->px, (1,1)->py, (0,1)->pz
    p = [Fraction(0)] * 4
    p[1] = px
    p[3] = py
    p[2] = pz
    p[0] = 1 - px - py - pz
    return p


def _pc2_probs(ps):
    p = [Fraction(0)] * 16
    for name, q in zip(_PC2_ORDER, ps):
        xa, za = _PAULI_BITS[name[0]]
        xb, zb = _PAULI_BITS[name[1]]
        p[xa | (za << 1) | (xb << 2) | (zb << 3)] += q
    p[0] = 1 - sum(ps)
    return p


def parse(text: str) -> Circuit:
    """Read a Stim-subset circuit and enumerate its raw noise channels."""
    lines = list(_tokenize_lines(text))
    ops, _ = _parse_block(lines, 0, False)
    c = Circuit()
    nmeas = 0
    bit = 0
    flat = []
    for op in ops:
        n = op.name
        if n in IGNORED:
            continue
        qs = [t for t in op.targets if isinstance(t, int)]
        if qs:
            c.num_qubits = max(c.num_qubits, max(qs) + 1)
        idx = len(flat)
        flat.append(op)
        if n in MEAS:
            p = _frac(op.args[0]) if op.args else Fraction(0)
            for q in op.targets:
                if p > 0:
                    c.channels.append(RawChannel("MFLIP", (q,), 1, [1 - p, p], idx, bit))
                    bit += 1
                nmeas += 1
        elif n in ("X_ERROR", "Y_ERROR", "Z_ERROR"):
            p = _frac(op.args[0])
            for q in op.targets:
                c.channels.append(RawChannel(n, (q,), 1, [1 - p, p], idx, bit))
                bit += 1
        elif n == "DEPOLARIZE1":
            p = _frac(op.args[0])
            for q in op.targets:
                c.channels.append(RawChannel(n, (q,), 2, _pc1_probs(p / 3, p / 3, p / 3), idx, bit))
                bit += 2
        elif n == "PAULI_CHANNEL_1":
            px, py, pz = (_frac(a) for a in op.args)
            for q in op.targets:
                c.channels.append(RawChannel(n, (q,), 2, _pc1_probs(px, py, pz), idx, bit))
                bit += 2
        elif n == "DEPOLARIZE2":
            p = _frac(op.args[0])
            for a, b in zip(op.targets[::2], op.targets[1::2]):
                c.channels.append(RawChannel(n, (a, b), 4, _pc2_probs([p / 15] * 15), idx, bit))
                bit += 4
        elif n == "PAULI_CHANNEL_2":
            ps = [_frac(a) for a in op.args]
            for a, b in zip(op.targets[::2], op.targets[1::2]):
                c.channels.append(RawChannel(n, (a, b), 4, _pc2_probs(ps), idx, bit))
                bit += 4
        elif n == "DETECTOR":
            c.detectors.append([nmeas + t[1] for t in op.targets])
        elif n == "OBSERVABLE_INCLUDE":
            k = int(float(op.args[0]))
            c.observables.setdefault(k, []).extend(nmeas + t[1] for t in op.targets)
        elif n in ONE_Q or n in TWO_Q or n in RESETS:
            pass
        elif n in ROTATIONS:
            if len(op.args) != (3 if n == "U3" else 1):
                raise ValueError(f"{n}: wrong number of angles")
            op.args = [float(a) for a in op.args]
        else:
            raise ValueError(f"unsupported instruction {n}")
    c.ops = flat
    c.num_measurements = nmeas
    c.num_error_bits = bit
    for k in range(c.num_observables):
        c.observables.setdefault(k, [])
    return c


def channel_bits_to_paulis(ch: RawChannel, outcome: int):
    """Paulis (qubit, x, z) applied by a channel for a given outcome index.

    Appendix "Pauli noise channels": bit pairs (e_x, e_z) per qubit.
    For MFLIP the returned list is empty (the record is flipped instead).
    """
    bits = [(outcome >> i) & 1 for i in range(ch.nbits)]
    if ch.kind == "X_ERROR":
        return [(ch.qubits[0], bits[0], 0)]
    if ch.kind == "Z_ERROR":
        return [(ch.qubits[0], 0, bits[0])]
    if ch.kind == "Y_ERROR":
        return [(ch.qubits[0], bits[0], bits[0])]
    if ch.kind in ("DEPOLARIZE1", "PAULI_CHANNEL_1"):
        return [(ch.qubits[0], bits[0], bits[1])]
    if ch.kind in ("DEPOLARIZE2", "PAULI_CHANNEL_2"):
        return [(ch.qubits[0], bits[0], bits[1]), (ch.qubits[1], bits[2], bits[3])]
    if ch.kind == "MFLIP":
        return []
    raise ValueError(ch.kind)
