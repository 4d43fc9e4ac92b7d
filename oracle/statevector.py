"""Exact branching state-vector simulation of a noisy Clifford+T circuit.

Oracle module (test infrastructure only).

For a fixed assignment e of the raw error bits, a noisy Stim circuit is a
pure Clifford+T circuit with Paulis inserted (Appendix "Pauli noise
channels": the error bits select the Pauli that is applied).  Its output
distribution is computed here by the textbook rule: every measurement and
reset branches the (unnormalised) state into its two projections; the
probability of a measurement record is the total squared norm of the
branches that carry it (Born rule).  Amplitudes live in Z[w, 1/sqrt2]
(``zomega``), so every probability is exact.

This is the "plain definition" the compiled sampler must reproduce: the
marginals P(m_0..m_i | e) of Algorithm 1 (Appendix "Sampling from
marginals") and the detector / observable distribution of Sec.
"Detectors", which are XORs of measurement outcomes (Eq. xor).
"""
from __future__ import annotations

from .circuit import Circuit, channel_bits_to_paulis
from .zomega import DOmega, _mul4


def _rot(c, j):
    """Multiply a Z[w] coefficient tuple by w^j."""
    j %= 8
    out = list(c)
    for _ in range(j):
        out = [-out[3], out[0], out[1], out[2]]
    return tuple(out)


_ZERO = (0, 0, 0, 0)


class _Branch:
    __slots__ = ("amp", "rec")

    def __init__(self, amp, rec):
        self.amp = amp      # list of coefficient 4-tuples, index = basis state
        self.rec = rec      # tuple of recorded bits so far


class StateVector:
    """All branches of one noisy run share a common denominator sqrt2^k."""

    def __init__(self, n):
        self.n = n
        amp = [_ZERO] * (1 << n)
        amp[0] = (1, 0, 0, 0)
        self.branches = [_Branch(amp, ())]
        self.k = 0

    # -- single-branch helpers -------------------------------------------
    def _map(self, fn):
        for b in self.branches:
            b.amp = fn(b.amp)

    def phase(self, q, j):
        """diag(1, w^j) on qubit q."""
        m = 1 << q

        def f(a):
            return [_rot(x, j) if (i & m) else x for i, x in enumerate(a)]
        self._map(f)

    def x(self, q):
        m = 1 << q
        self._map(lambda a: [a[i ^ m] for i in range(len(a))])

    def z(self, q):
        self.phase(q, 4)

    def y(self, q):
        # Y = i X Z
        self.z(q)
        self.x(q)
        self._map(lambda a: [_rot(v, 2) for v in a])

    def h(self, q):
        m = 1 << q

        def f(a):
            out = list(a)
            for i in range(len(a)):
                if not (i & m):
                    u, v = a[i], a[i | m]
                    out[i] = tuple(s + t for s, t in zip(u, v))
                    out[i | m] = tuple(s - t for s, t in zip(u, v))
            return out
        self._map(f)
        self.k += 1

    def cx(self, c, t):
        mc, mt = 1 << c, 1 << t
        self._map(lambda a: [a[i ^ mt] if (i & mc) else a[i] for i in range(len(a))])

    def cz(self, a_, b_):
        ma, mb = 1 << a_, 1 << b_

        def f(a):
            return [_rot(x, 4) if (i & ma and i & mb) else x for i, x in enumerate(a)]
        self._map(f)

    def swap(self, a_, b_):
        ma, mb = 1 << a_, 1 << b_

        def perm(i):
            ba, bb = (i & ma) != 0, (i & mb) != 0
            if ba != bb:
                return i ^ ma ^ mb
            return i
        self._map(lambda a: [a[perm(i)] for i in range(len(a))])

    # -- branching -------------------------------------------------------
    def measure(self, q, record=True, flip=0):
        """Projective Z measurement; optionally record outcome XOR flip."""
        m = 1 << q
        out = []
        for b in self.branches:
            for outcome in (0, 1):
                amp = [x if (((i & m) != 0) == bool(outcome)) else _ZERO for i, x in enumerate(b.amp)]
                if all(x == _ZERO for x in amp):
                    continue
                rec = b.rec + ((outcome ^ flip),) if record else b.rec
                out.append(_Branch(amp, rec))
        self.branches = out

    def reset(self, q):
        self.measure(q, record=False)
        m = 1 << q
        for b in self.branches:
            if any(x != _ZERO for i, x in enumerate(b.amp) if i & m):
                b.amp = [b.amp[i ^ m] for i in range(len(b.amp))]

    def norm2(self, b):
        """||branch||^2 as an exact DOmega."""
        tot = [0, 0, 0, 0]
        for x in b.amp:
            if x == _ZERO:
                continue
            c0, c1, c2, c3 = x
            p = _mul4(x, (c0, -c3, -c2, -c1))
            for i in range(4):
                tot[i] += p[i]
        return DOmega(tot, 2 * self.k)


def run(circ: Circuit, e_bits) -> dict:
    """Exact joint distribution of the measurement record given raw bits e.

    Returns {record tuple: DOmega probability}.
    """
    sv = StateVector(circ.num_qubits)
    # channel outcomes in op order
    by_op = {}
    for ch in circ.channels:
        by_op.setdefault(ch.op_index, []).append(ch)
    nrec = 0
    for idx, op in enumerate(circ.ops):
        n = op.name
        chans = by_op.get(idx, [])
        if n in ("M", "MX", "MR", "MRX"):
            # channels appear in target order, one per target when p > 0
            ch_iter = iter(chans)
            for q in op.targets:
                flip = 0
                if chans:
                    ch = next(ch_iter)
                    flip = e_bits[ch.first_bit]
                if n in ("MX", "MRX"):
                    sv.h(q)
                sv.measure(q, True, flip)
                if n in ("MR", "MRX"):
                    # re-initialise to |0> (the outcome is already recorded)
                    m = 1 << q
                    for b in sv.branches:
                        if any(x != _ZERO for i, x in enumerate(b.amp) if i & m):
                            b.amp = [b.amp[i ^ m] for i in range(len(b.amp))]
                if n in ("MX", "MRX"):
                    sv.h(q)
                nrec += 1
            continue
        if n == "R":
            for q in op.targets:
                sv.reset(q)
        elif n == "RX":
            for q in op.targets:
                sv.reset(q)
                sv.h(q)
        elif n in ("X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "PAULI_CHANNEL_1",
                   "DEPOLARIZE2", "PAULI_CHANNEL_2"):
            for ch in chans:
                o = sum(e_bits[ch.first_bit + i] << i for i in range(ch.nbits))
                for q, xb, zb in channel_bits_to_paulis(ch, o):
                    if zb:
                        sv.z(q)
                    if xb:
                        sv.x(q)
        elif n in ("I", "DETECTOR", "OBSERVABLE_INCLUDE"):
            pass
        elif n == "X":
            for q in op.targets:
                sv.x(q)
        elif n == "Y":
            for q in op.targets:
                sv.y(q)
        elif n == "Z":
            for q in op.targets:
                sv.z(q)
        elif n == "H":
            for q in op.targets:
                sv.h(q)
        elif n in ("S", "S_DAG", "T", "T_DAG"):
            j = {"S": 2, "S_DAG": 6, "T": 1, "T_DAG": 7}[n]
            for q in op.targets:
                sv.phase(q, j)
        elif n in ("SQRT_X", "SQRT_X_DAG"):
            j = 2 if n == "SQRT_X" else 6
            for q in op.targets:
                sv.h(q)
                sv.phase(q, j)
                sv.h(q)
        elif n in ("CX", "CY", "CZ", "SWAP"):
            for a, b in zip(op.targets[::2], op.targets[1::2]):
                if isinstance(a, tuple):
                    # classically controlled Pauli on b, per branch record
                    for br in sv.branches:
                        bit = br.rec[len(br.rec) + a[1]]
                        if bit:
                            _apply_pauli_branch(sv, br, n, b)
                    continue
                if n == "CX":
                    sv.cx(a, b)
                elif n == "CZ":
                    sv.cz(a, b)
                elif n == "CY":
                    # CY = (I x S) CX (I x S_DAG)
                    sv.phase(b, 6)
                    sv.cx(a, b)
                    sv.phase(b, 2)
                else:
                    sv.swap(a, b)
        else:
            raise ValueError(f"unsupported op {n}")
    dist = {}
    for b in sv.branches:
        p = sv.norm2(b)
        if p.is_zero():
            continue
        dist[b.rec] = dist.get(b.rec, DOmega()) + p
    return dist


def _apply_pauli_branch(sv, br, gate, q):
    m = 1 << q
    a = br.amp
    if gate == "CX":
        br.amp = [a[i ^ m] for i in range(len(a))]
    elif gate == "CZ":
        br.amp = [_rot(x, 4) if (i & m) else x for i, x in enumerate(a)]
    elif gate == "CY":
        a = [_rot(x, 4) if (i & m) else x for i, x in enumerate(a)]
        a = [a[i ^ m] for i in range(len(a))]
        br.amp = [_rot(x, 2) for x in a]
    else:
        raise ValueError(gate)


def output_distribution(circ: Circuit, e_bits, mode: str) -> dict:
    """Exact distribution of the sampler's outputs given raw bits e.

    mode "measurements": outputs are the measurement record.
    mode "detectors": outputs are the detector bits followed by the
    observable bits, each the XOR of the measurement outcomes it names
    (Eq. xor and Sec. "Sampling detectors and observables").
    """
    dist = run(circ, e_bits)
    if mode == "measurements":
        return dist
    out = {}
    for rec, p in dist.items():
        bits = []
        for det in circ.detectors:
            v = 0
            for j in det:
                v ^= rec[j]
            bits.append(v)
        for k in range(circ.num_observables):
            v = 0
            for j in circ.observables[k]:
                v ^= rec[j]
            bits.append(v)
        key = tuple(bits)
        out[key] = out.get(key, DOmega()) + p
    return out


def marginal(dist: dict, prefix) -> DOmega:
    """P(o_0..o_{i} = prefix) = sum of the joint over the remaining outputs."""
    n = len(prefix)
    tot = DOmega()
    for key, p in dist.items():
        if tuple(key[:n]) == tuple(prefix):
            tot = tot + p
    return tot
