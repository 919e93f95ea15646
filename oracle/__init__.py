"""CPU oracle for the Torontonian -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path (paper_2009_01177_gb300) never does,
and the two share no code: this package wraps `tor_oracle.c`, a plain direct
subset sum (paper Eq. 2, Algorithm 1) in 256-bit fixed point with one global
scaling factor (paper Sec. 5.1-5.3).

Functions
---------
tor(O)            Tor(O) of a 2k x 2k xxpp matrix; returns an OracleResult.
tor_range(O, lo, hi)   the same sum restricted to subset masks in [lo, hi).
tor_exact(O, lo, hi)   the same sums exactly, as Fractions (every bit of the fixed point).
det(O, mask)      det(I - O_Z) for one subset mask (hi, lo).
prob(Ofull, pattern)   click probability of Eq. 1 (hi, lo) plus Tor(O_S).
fx_ops(a, b)      a*b, a+b, a-b, 1/a, 1/sqrt(a) through the fixed-point path.
build()           compile liboracle.so (gcc, OpenMP).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tor_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_FRAC_BITS = 200
ERRORS = {0: "ok", 1: "invalid argument", 2: "not positive definite", 3: "fixed-point overflow"}


def build(force: bool = False) -> str:
    """Compile tor_oracle.c into liboracle.so next to it; returns the path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_tor.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, dp]
            lib.oracle_tor_range.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_uint64, dp]
            lib.oracle_det.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_int, dp]
            lib.oracle_prob.argtypes = [dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_ubyte), ctypes.c_int, ctypes.c_int,
                                        dp]
            lib.oracle_fx_ops.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
            lib.oracle_tor_range_raw.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                                 ctypes.POINTER(ctypes.c_uint64)]
            for f in (lib.oracle_tor, lib.oracle_tor_range, lib.oracle_det, lib.oracle_prob,
                      lib.oracle_fx_ops, lib.oracle_tor_range_raw):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


@dataclasses.dataclass
class OracleResult:
    hi: float
    lo: float
    sum_abs: float
    sum_abs_lo: float

    @property
    def value(self) -> float:
        return self.hi + self.lo

    @property
    def kappa(self) -> float:
        """Condition number of the alternating sum: sum_Z t_Z / |Tor|."""
        return self.sum_abs / abs(self.hi) if self.hi != 0 else float("inf")


def _as_c(O: np.ndarray) -> np.ndarray:
    O = np.ascontiguousarray(O, dtype=np.float64)
    if O.ndim != 2 or O.shape[0] != O.shape[1] or O.shape[0] % 2:
        raise ValueError("O must be a square 2k x 2k float64 matrix")
    return O


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int):
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {ERRORS.get(rc, '?')}")


def tor_range(O: np.ndarray, mask_lo: int, mask_hi: int, frac_bits: int = DEFAULT_FRAC_BITS,
              threads: int = 0, mutation: int = 0) -> OracleResult:
    O = _as_c(O)
    k = O.shape[0] // 2
    out = np.zeros(4)
    _check(_load().oracle_tor_range(_ptr(O), k, max(2 * k, 1), frac_bits, threads, mutation,
                                    mask_lo, mask_hi, _ptr(out)))
    return OracleResult(*map(float, out))


def tor_exact(O: np.ndarray, mask_lo: int = 0, mask_hi: int | None = None,
              frac_bits: int = DEFAULT_FRAC_BITS, threads: int = 0):
    """(Tor, sum_Z t_Z) over the masks in [mask_lo, mask_hi) as exact Fractions of the
    fixed-point sums (frac_bits fraction bits), not rounded to double-double."""
    from fractions import Fraction
    O = _as_c(O)
    k = O.shape[0] // 2
    if mask_hi is None:
        mask_hi = 1 << k
    raw = (ctypes.c_uint64 * 8)()
    _check(_load().oracle_tor_range_raw(_ptr(O), k, max(2 * k, 1), frac_bits, threads, mask_lo,
                                        mask_hi, raw))

    def signed(words):
        v = sum(int(w) << (64 * i) for i, w in enumerate(words))
        return v - (1 << 256) if v >> 255 else v
    return (Fraction(signed(raw[0:4]), 1 << frac_bits), Fraction(signed(raw[4:8]), 1 << frac_bits))


def tor(O: np.ndarray, frac_bits: int = DEFAULT_FRAC_BITS, threads: int = 0,
        mutation: int = 0) -> OracleResult:
    """Tor(O) by the direct subset sum in 256-bit fixed point."""
    O = _as_c(O)
    k = O.shape[0] // 2
    out = np.zeros(4)
    _check(_load().oracle_tor(_ptr(O), k, max(2 * k, 1), frac_bits, threads, mutation, _ptr(out)))
    return OracleResult(*map(float, out))


def det(O: np.ndarray, mask: int, frac_bits: int = DEFAULT_FRAC_BITS):
    """det(I - O_Z) for the subset of modes given by the bits of `mask`, as (hi, lo)."""
    O = _as_c(O)
    k = O.shape[0] // 2
    out = np.zeros(2)
    _check(_load().oracle_det(_ptr(O), k, max(2 * k, 1), mask, frac_bits, _ptr(out)))
    return float(out[0]), float(out[1])


def prob(Ofull: np.ndarray, pattern, frac_bits: int = DEFAULT_FRAC_BITS, threads: int = 0):
    """p(S) of Eq. 1 for a 0/1 pattern of length M: returns (p_hi, p_lo, OracleResult of Tor)."""
    Ofull = _as_c(Ofull)
    M = Ofull.shape[0] // 2
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.uint8))
    if pat.shape != (M,):
        raise ValueError("pattern must have M entries")
    out = np.zeros(6)
    _check(_load().oracle_prob(_ptr(Ofull), M, 2 * M, pat.ctypes.data_as(
        ctypes.POINTER(ctypes.c_ubyte)), frac_bits, threads, _ptr(out)))
    return float(out[0]), float(out[1]), OracleResult(*map(float, out[2:6]))


def fx_ops(a: float, b: float, frac_bits: int = DEFAULT_FRAC_BITS) -> np.ndarray:
    """[a*b, a+b, a-b, 1/a, 1/sqrt(a)] as (hi, lo) pairs through the fixed-point type."""
    out = np.zeros(10)
    _check(_load().oracle_fx_ops(float(a), float(b), frac_bits, _ptr(out)))
    return out.reshape(5, 2)
