"""ctypes wrapper of the oracle program evaluator (``evaluator.c``).

Oracle module (test infrastructure only).  ``build()`` compiles the plain C
file with gcc into ``oracle/_build/liboracle_eval.so``; the wrapper only
marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .zomega import DOmega

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evaluator.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_eval.so")
_lib = None


def build(force=False) -> str:
    """Compile the oracle evaluator (plain C, gcc) if it is missing or stale."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.oracle_load.restype = ctypes.c_void_p
        L.oracle_load.argtypes = [ctypes.c_char_p]
        L.oracle_free.argtypes = [ctypes.c_void_p]
        L.oracle_last_error.restype = ctypes.c_char_p
        L.oracle_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        L.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.oracle_eval_table.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int)]
        L.oracle_sample.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_decide.argtypes = [ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        L.oracle_eval_table_c.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_double)]
        L.oracle_noise_x.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_uint64)]
        L.oracle_geo_gap.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32]
        L.oracle_geo_pick.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int,
                                      ctypes.c_uint32]
    return _lib


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return tuple(o)


def geo_gap(Q, m, U):
    """Geometric gap of the noise rule: non-candidates before the next
    candidate among m channels of a group with parameter Q, for the word U."""
    r = lib().oracle_geo_gap(Q, m, U)
    if r < 0:
        raise RuntimeError(lib().oracle_last_error().decode())
    return r


def geo_pick(Q, thr, V):
    """Outcome of a candidate channel with cumulative thresholds thr (n-1
    values) in a group with parameter Q, for the word V."""
    arr = (ctypes.c_uint32 * len(thr))(*thr)
    r = lib().oracle_geo_pick(Q, arr, len(thr) + 1, V)
    if r < 0:
        raise RuntimeError(lib().oracle_last_error().decode())
    return r


def decide(U, Ap, Bp, ep, A1, B1, e1):
    r = lib().oracle_decide(U, Ap, Bp, ep, A1, B1, e1)
    if r < 0:
        raise RuntimeError(lib().oracle_last_error().decode())
    return r


class OracleProgram:
    """A compiled program as read by the oracle's own reader."""

    def __init__(self, path):
        self._h = lib().oracle_load(path.encode())
        if not self._h:
            raise RuntimeError(lib().oracle_last_error().decode())
        info = (ctypes.c_int64 * 16)()
        lib().oracle_info(self._h, info)
        (self.mode, self.nx, self.words, self.nf, self.nr, self.nmeas, self.ndet,
         self.nobs, self.n_out, self.n_chains, self.n_channels, self.n_tables,
         self.noise_mode, self.n_groups) = info[:14]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_free(h)
            self._h = None

    def eval_table(self, table, xwords) -> DOmega:
        """Exact value of one marginal table at the bit vector X."""
        X = (ctypes.c_uint64 * self.words)(*[int(v) for v in xwords])
        coef = (ctypes.c_int64 * 8)()
        k = ctypes.c_int()
        if lib().oracle_eval_table(self._h, table, X, coef, ctypes.byref(k)) != 0:
            raise RuntimeError(lib().oracle_last_error().decode())
        c = []
        for i in range(4):
            hi, lo = coef[2 * i], coef[2 * i + 1] & 0xFFFFFFFFFFFFFFFF
            c.append((hi << 64) | lo)
        # evaluator stores value * sqrt2^k ; DOmega stores / sqrt2^k
        return DOmega(c, -k.value)

    def eval_table_c(self, table, xwords) -> complex:
        """Value of any table at X in complex double (tables with arbitrary
        phases included)."""
        X = (ctypes.c_uint64 * self.words)(*[int(v) for v in xwords])
        out = (ctypes.c_double * 2)()
        if lib().oracle_eval_table_c(self._h, table, X, out) != 0:
            raise RuntimeError(lib().oracle_last_error().decode())
        return complex(out[0], out[1])

    def noise_x(self, seed, shot):
        """X = T e of one shot after its error mechanisms, before any output."""
        X = (ctypes.c_uint64 * self.words)()
        lib().oracle_noise_x(self._h, seed, shot, X)
        return list(X)

    def sample(self, seed, shot_begin, n):
        wm = (self.nmeas + 63) // 64
        wd = (self.ndet + 63) // 64
        wo = (self.nobs + 63) // 64
        meas = np.zeros((n, max(wm, 1)), dtype=np.uint64)
        det = np.zeros((n, max(wd, 1)), dtype=np.uint64)
        obs = np.zeros((n, max(wo, 1)), dtype=np.uint64)
        acc = np.zeros(n, dtype=np.uint8)
        rc = lib().oracle_sample(self._h, seed, shot_begin, n,
                                 meas.ctypes.data if self.mode == 1 else None,
                                 det.ctypes.data, obs.ctypes.data, acc.ctypes.data)
        if rc != 0:
            raise RuntimeError(lib().oracle_last_error().decode())
        return {"meas": meas[:, :wm], "det": det[:, :wd], "obs": obs[:, :wo], "accept": acc}
