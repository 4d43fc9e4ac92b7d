"""Exact arithmetic in D[w] = Z[w, 1/sqrt2], w = exp(i*pi/4).

Oracle module (test infrastructure only).

Every amplitude of a Clifford+T circuit lies in this ring: the gates H
(entries +-1/sqrt2), S (i = w^2) and T (w) have entries in it, and so do the
phase-pair factors of the paper's parameterised evaluation (Sec. "Parameterized
evaluation of Clifford ZX diagrams", Eq. phase_pair: every term is a sum of
powers of w when the angles are multiples of pi/4).

A value is stored as  (c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^k  with Python
integers c_i and an integer k.  Since w^4 = -1, {1, w, w^2, w^3} is a Z-basis
of Z[w].  Nothing here is fast; everything is exact.
"""
from __future__ import annotations

from fractions import Fraction
import math


def _mul4(a, b):
    """Product of two Z[w] coefficient 4-tuples, reducing with w^4 = -1."""
    out = [0, 0, 0, 0]
    for i in range(4):
        if a[i] == 0:
            continue
        for j in range(4):
            p = a[i] * b[j]
            n = i + j
            if n >= 4:
                out[n - 4] -= p
            else:
                out[n] += p
    return out


# sqrt2 = w - w^3  (w + w^-1 = 2 cos(pi/4) = sqrt2 and w^-1 = -w^3)
_SQRT2 = (0, 1, 0, -1)


class DOmega:
    """Element of Z[w, 1/sqrt2]: (c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^k."""

    __slots__ = ("c", "k")

    def __init__(self, c=(0, 0, 0, 0), k=0):
        self.c = tuple(int(x) for x in c)
        self.k = int(k)

    # -- constructors -----------------------------------------------------
    @staticmethod
    def from_int(n):
        return DOmega((n, 0, 0, 0), 0)

    @staticmethod
    def omega_pow(j):
        """w^j for any integer j (w has order 8)."""
        j %= 8
        c = [0, 0, 0, 0]
        if j < 4:
            c[j] = 1
        else:
            c[j - 4] = -1
        return DOmega(c, 0)

    @staticmethod
    def sqrt2_pow(e):
        """sqrt2^e for any integer e (stored as 1 / sqrt2^(-e))."""
        return DOmega((1, 0, 0, 0), -e)

    # -- ring operations --------------------------------------------------
    def _aligned(self, other):
        """Return coefficient tuples of self and other over a common k."""
        a, b = list(self.c), list(other.c)
        ka, kb = self.k, other.k
        # x / sqrt2^ka = x * sqrt2^(k-ka) / sqrt2^k  with k = max(ka, kb)
        while ka < kb:
            a = _mul4(a, _SQRT2)
            ka += 1
        while kb < ka:
            b = _mul4(b, _SQRT2)
            kb += 1
        return a, b, ka

    def __add__(self, other):
        other = _coerce(other)
        a, b, k = self._aligned(other)
        return DOmega([x + y for x, y in zip(a, b)], k).reduced()

    __radd__ = __add__

    def __neg__(self):
        return DOmega([-x for x in self.c], self.k)

    def __sub__(self, other):
        return self + (-_coerce(other))

    def __rsub__(self, other):
        return _coerce(other) - self

    def __mul__(self, other):
        other = _coerce(other)
        return DOmega(_mul4(self.c, other.c), self.k + other.k).reduced()

    __rmul__ = __mul__

    def conj(self):
        """Complex conjugate: w^j -> w^-j, i.e. (c0, c1, c2, c3) -> (c0, -c3, -c2, -c1)."""
        c0, c1, c2, c3 = self.c
        return DOmega((c0, -c3, -c2, -c1), self.k)

    def is_zero(self):
        return all(x == 0 for x in self.c)

    def reduced(self):
        """Divide numerator and denominator by sqrt2 while it stays integral."""
        c, k = list(self.c), self.k
        if all(x == 0 for x in c):
            return DOmega((0, 0, 0, 0), 0)
        while True:
            # x / sqrt2 = x * sqrt2 / 2
            t = _mul4(c, _SQRT2)
            if all(x % 2 == 0 for x in t):
                c = [x // 2 for x in t]
                k -= 1
            else:
                break
        return DOmega(c, k)

    def __eq__(self, other):
        try:
            other = _coerce(other)
        except TypeError:
            return NotImplemented
        return (self - other).is_zero()

    def __hash__(self):
        r = self.reduced()
        return hash((r.c, r.k))

    # -- real numbers -----------------------------------------------------
    def is_real(self):
        """Im(c0 + c1 w + c2 w^2 + c3 w^3) = c2 + (c1 + c3)/sqrt2 = 0."""
        c0, c1, c2, c3 = self.c
        return c2 == 0 and c1 + c3 == 0

    def real_parts(self):
        """For a real value return (A, B, n) with value = (A + B*sqrt2) / 2^n.

        Re(c0 + c1 w + c2 w^2 + c3 w^3) = c0 + (c1 - c3)/sqrt2
                                         = (2 c0 + (c1 - c3) sqrt2) / 2.
        """
        if not self.is_real():
            raise ValueError("value is not real")
        c0, c1, c2, c3 = self.c
        A, B = 2 * c0, c1 - c3
        k = self.k + 2  # divide by 2 = sqrt2^2
        # (A + B sqrt2)/sqrt2^k ; make k even by multiplying through by sqrt2
        if k % 2:
            A, B = 2 * B, A
            k += 1
        return A, B, k // 2

    def sign(self):
        """Exact sign (-1, 0, 1) of a real value."""
        A, B, _ = self.real_parts()
        return _sign_a_plus_b_sqrt2(A, B)

    def to_complex(self):
        w = complex(math.cos(math.pi / 4), math.sin(math.pi / 4))
        z = sum(self.c[j] * w ** j for j in range(4))
        return z / math.sqrt(2) ** self.k

    def __float__(self):
        return self.to_complex().real

    def __repr__(self):
        return f"DOmega({self.c}, k={self.k})"


def _sign_a_plus_b_sqrt2(A, B):
    """Exact sign of A + B*sqrt2 for integers A, B."""
    if A >= 0 and B >= 0:
        return 0 if (A == 0 and B == 0) else 1
    if A <= 0 and B <= 0:
        return -1
    # opposite signs: compare A^2 with 2 B^2
    if A > 0:  # B < 0
        return 1 if A * A > 2 * B * B else -1
    return 1 if 2 * B * B > A * A else -1


def _coerce(x):
    if isinstance(x, DOmega):
        return x
    if isinstance(x, int):
        return DOmega.from_int(x)
    raise TypeError(f"cannot coerce {type(x)} to DOmega")


def compare_real(x: DOmega, y: DOmega) -> int:
    """Exact comparison of two real elements: sign(x - y)."""
    return (x - y).sign()


def to_fraction_bounds(x: DOmega, digits=40):
    """Rational enclosure of a real value (for printing / golden files)."""
    A, B, n = x.real_parts()
    s = math.isqrt(2 * 10 ** (2 * digits))
    lo = Fraction(A * 10 ** digits + B * s, 10 ** digits * 2 ** n)
    hi = Fraction(A * 10 ** digits + B * (s + 1), 10 ** digits * 2 ** n)
    return (lo, hi) if lo <= hi else (hi, lo)
