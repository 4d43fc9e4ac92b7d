"""Floating-point state vector for circuits with arbitrary rotations.

Oracle module (test infrastructure only).  The exact state vector
(statevector.py) works in Z[w, 1/sqrt2], which holds every Clifford+T
amplitude but not those of R_X, R_Y, R_Z and U3 at other angles (Sec.
"Methods": Tsim extends the Stim format with these rotations; angles are
given in units of pi).  This module runs the same circuits in complex double
from the textbook gate matrices:

    R_Z(t) = diag(e^{-i pi t/2}, e^{i pi t/2})
    R_X(t) = [[cos(pi t/2), -i sin(pi t/2)], [-i sin(pi t/2), cos(pi t/2)]]
    R_Y(t) = [[cos(pi t/2), -sin(pi t/2)], [sin(pi t/2), cos(pi t/2)]]
    U3(a, b, c) = [[cos(pi a/2), -e^{i pi c} sin(pi a/2)],
                   [e^{i pi b} sin(pi a/2), e^{i pi (b+c)} cos(pi a/2)]]

with the Pauli noise of a raw assignment e inserted as in the exact module
(Appendix "Pauli noise channels") and every measurement branching into its
two outcomes.  Nothing here is fast.
"""
from __future__ import annotations

import numpy as np

from .circuit import Circuit, channel_bits_to_paulis

_S2 = np.sqrt(0.5)
_FIXED = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "H": np.array([[1, 1], [1, -1]], dtype=complex) * _S2,
    "S": np.diag([1, 1j]).astype(complex),
    "S_DAG": np.diag([1, -1j]).astype(complex),
    "T": np.diag([1, np.exp(1j * np.pi / 4)]),
    "T_DAG": np.diag([1, np.exp(-1j * np.pi / 4)]),
    "SQRT_X": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]]),
    "SQRT_X_DAG": 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]]),
}


def rotation(name, args):
    """2x2 matrix of R_X, R_Y, R_Z or U3 (angles in units of pi)."""
    if name == "R_Z":
        t = float(args[0]) * np.pi / 2
        return np.diag([np.exp(-1j * t), np.exp(1j * t)])
    if name == "R_X":
        t = float(args[0]) * np.pi / 2
        return np.array([[np.cos(t), -1j * np.sin(t)], [-1j * np.sin(t), np.cos(t)]])
    if name == "R_Y":
        t = float(args[0]) * np.pi / 2
        return np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]], dtype=complex)
    if name == "U3":
        a, b, c = (float(x) * np.pi for x in args)
        return np.array([[np.cos(a / 2), -np.exp(1j * c) * np.sin(a / 2)],
                         [np.exp(1j * b) * np.sin(a / 2), np.exp(1j * (b + c)) * np.cos(a / 2)]])
    raise ValueError(name)


class _Branch:
    __slots__ = ("psi", "rec")

    def __init__(self, psi, rec):
        self.psi = psi
        self.rec = rec


class StateVectorF:
    """Unnormalised branches (state, measurement record), complex double."""

    def __init__(self, n):
        self.n = n
        psi = np.zeros(1 << n, dtype=complex)
        psi[0] = 1.0
        self.branches = [_Branch(psi, ())]

    def gate1(self, q, U):
        ax = self.n - 1 - q  # qubit q is bit q of the index
        for b in self.branches:
            t = b.psi.reshape([2] * self.n)
            t = np.moveaxis(np.tensordot(U, t, axes=([1], [ax])), 0, ax)
            b.psi = t.reshape(-1)

    def cx(self, c, t):
        idx = np.arange(1 << self.n)
        src = np.where((idx >> c) & 1, idx ^ (1 << t), idx)
        for b in self.branches:
            b.psi = b.psi[src]

    def cz(self, a, c):
        idx = np.arange(1 << self.n)
        sign = np.where(((idx >> a) & 1) & ((idx >> c) & 1), -1.0, 1.0)
        for b in self.branches:
            b.psi = b.psi * sign

    def swap(self, a, c):
        idx = np.arange(1 << self.n)
        ba, bc = (idx >> a) & 1, (idx >> c) & 1
        src = idx ^ ((ba ^ bc) << a) ^ ((ba ^ bc) << c)
        for b in self.branches:
            b.psi = b.psi[src]

    def measure(self, q, flip=0, record=True):
        """Projective Z measurement: each branch splits by the outcome (an
        unrecorded one keeps the record, so the branches stay a mixture)."""
        idx = np.arange(1 << self.n)
        bit = (idx >> q) & 1
        out = []
        for b in self.branches:
            for m in (0, 1):
                psi = np.where(bit == m, b.psi, 0)
                if np.vdot(psi, psi).real == 0:
                    continue
                out.append(_Branch(psi, b.rec + (m ^ flip,) if record else b.rec))
        self.branches = out

    def reset(self, q):
        """Unrecorded measurement, then X on the branches that found 1."""
        self.measure(q, record=False)
        idx = np.arange(1 << self.n)
        m = 1 << q
        for b in self.branches:
            if np.any(b.psi[((idx >> q) & 1) == 1] != 0):
                b.psi = b.psi[idx ^ m]

    def norm2(self, b):
        return float(np.vdot(b.psi, b.psi).real)


def run(circ: Circuit, e_bits) -> dict:
    """Distribution of the measurement record given raw bits e (floats)."""
    sv = StateVectorF(circ.num_qubits)
    by_op = {}
    for ch in circ.channels:
        by_op.setdefault(ch.op_index, []).append(ch)
    H = _FIXED["H"]
    for idx, op in enumerate(circ.ops):
        n = op.name
        chans = by_op.get(idx, [])
        if n in ("M", "MX", "MR", "MRX"):
            ch_iter = iter(chans)
            for q in op.targets:
                flip = e_bits[next(ch_iter).first_bit] if chans else 0
                if n in ("MX", "MRX"):
                    sv.gate1(q, H)
                sv.measure(q, flip)
                if n in ("MR", "MRX"):
                    sv.reset(q)
                if n in ("MX", "MRX"):
                    sv.gate1(q, H)
            continue
        if n == "R":
            for q in op.targets:
                sv.reset(q)
        elif n == "RX":
            for q in op.targets:
                sv.reset(q)
                sv.gate1(q, H)
        elif n in ("X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "PAULI_CHANNEL_1",
                   "DEPOLARIZE2", "PAULI_CHANNEL_2"):
            for ch in chans:
                o = sum(e_bits[ch.first_bit + i] << i for i in range(ch.nbits))
                for q, xb, zb in channel_bits_to_paulis(ch, o):
                    if zb:
                        sv.gate1(q, _FIXED["Z"])
                    if xb:
                        sv.gate1(q, _FIXED["X"])
        elif n in ("DETECTOR", "OBSERVABLE_INCLUDE"):
            pass
        elif n in _FIXED:
            for q in op.targets:
                sv.gate1(q, _FIXED[n])
        elif n in ("R_X", "R_Y", "R_Z", "U3"):
            U = rotation(n, op.args)
            for q in op.targets:
                sv.gate1(q, U)
        elif n in ("CX", "CY", "CZ", "SWAP"):
            for a, b in zip(op.targets[::2], op.targets[1::2]):
                if isinstance(a, tuple):
                    P = {"CX": _FIXED["X"], "CZ": _FIXED["Z"], "CY": _FIXED["Y"]}[n]
                    for br in sv.branches:
                        if br.rec[len(br.rec) + a[1]]:
                            t = br.psi.reshape([2] * sv.n)
                            ax = sv.n - 1 - b
                            br.psi = np.moveaxis(np.tensordot(P, t, axes=([1], [ax])), 0, ax).reshape(-1)
                    continue
                if n == "CX":
                    sv.cx(a, b)
                elif n == "CZ":
                    sv.cz(a, b)
                elif n == "CY":
                    sv.gate1(b, _FIXED["S_DAG"])
                    sv.cx(a, b)
                    sv.gate1(b, _FIXED["S"])
                else:
                    sv.swap(a, b)
        else:
            raise ValueError(f"unsupported op {n}")
    dist = {}
    for b in sv.branches:
        p = sv.norm2(b)
        if p == 0:
            continue
        dist[b.rec] = dist.get(b.rec, 0.0) + p
    return dist


def output_distribution(circ: Circuit, e_bits, mode: str) -> dict:
    """Distribution of the sampler's outputs given raw bits e: the record
    itself ("measurements"), or detector then observable bits, each the XOR
    of the records it names (Eq. xor)."""
    dist = run(circ, e_bits)
    if mode == "measurements":
        return dist
    out = {}
    for rec, p in dist.items():
        bits = [sum(rec[j] for j in det) & 1 for det in circ.detectors]
        bits += [sum(rec[j] for j in circ.observables[k]) & 1 for k in range(circ.num_observables)]
        key = tuple(bits)
        out[key] = out.get(key, 0.0) + p
    return out
