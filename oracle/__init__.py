"""CPU oracle for the state-vector hot path (arXiv 2310.17739).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are its only users.  The library path never imports it.

Thin ctypes marshalling over ``oracle.c`` (plain C, complex128, single thread,
sums in index order).  What each function computes, and the passage of the
paper it follows, is stated in ``oracle.c``.  The wrappers here only move
numpy arrays across the C boundary.

Pins (all in ``tests/test_oracle_*.py``): dense Kronecker products of every
gate on <= 6 qubits, scipy ``expm`` for every rotation, GHZ and QFT closed
forms, exp(-i t P) = cos t I - i sin t P for compiled Pauli gadgets, norm and
U-then-U^dagger invariants, Born statistics, the probability-product of the
mid-circuit measurement assertion table, numpy's Philox for the draws, and
numpy's searchsorted on the cumulative Born distribution for final-state shots.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from paper_2310_17739_gb300.workload import GATE_DTYPE, TERM_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, E_INVAL, E_ZEROPROB = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O3, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp, u64, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t
            L.oracle_gate_matrix.argtypes = [dp, dp, dp]
            L.oracle_gate_matrix.restype = ctypes.c_int
            L.oracle_run.argtypes = [dp, ctypes.c_int, dp, sz, dp, u64, dp, ctypes.c_double,
                                     dp, dp, sz, dp]
            L.oracle_run.restype = ctypes.c_int
            L.oracle_prob.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
            L.oracle_measure.argtypes = [dp, ctypes.c_int, ctypes.c_int, u64, u64, ctypes.c_int,
                                         ctypes.c_double, dp, dp]
            L.oracle_measure.restype = ctypes.c_int
            L.oracle_reset.argtypes = [dp, ctypes.c_int, ctypes.c_int, u64, u64, dp, dp]
            L.oracle_reset.restype = ctypes.c_int
            L.oracle_expect.argtypes = [dp, ctypes.c_int, dp, sz, dp]
            L.oracle_philox4x64_10.argtypes = [dp, dp, dp]
            L.oracle_draw.argtypes = [u64, u64]
            L.oracle_draw.restype = ctypes.c_double
            L.oracle_shot_draw.argtypes = [u64, u64]
            L.oracle_shot_draw.restype = ctypes.c_double
            L.oracle_sample.argtypes = [dp, ctypes.c_int, u64, u64, u64, dp]
            L.oracle_sample.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def basis_state(n: int, index: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


def gate_matrix(gate, mats=None) -> np.ndarray:
    g = np.asarray(gate, dtype=GATE_DTYPE).reshape(1)
    mats = np.ascontiguousarray(mats if mats is not None else np.zeros(1), dtype=np.float64)
    out = np.zeros(32, dtype=np.float64)
    d = lib().oracle_gate_matrix(_ptr(g), _ptr(mats), _ptr(out))
    if d < 0:
        raise ValueError("not a unitary gate record")
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


class RunResult:
    def __init__(self, status, outcomes, probs, ordinal):
        self.status = status
        self.outcomes = outcomes
        self.probs = probs
        self.ordinal = ordinal


def run(psi: np.ndarray, n: int, gates: np.ndarray, mats=None, seed: int = 0,
        ordinal: int = 0, thr: float = 0.0, log_cap: int = 4096) -> RunResult:
    """Apply gate records to psi in place (complex128, length 2^n), unfused."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == (1 << n)
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    mats = np.ascontiguousarray(mats if mats is not None else np.zeros(1), dtype=np.float64)
    ordn = np.array([ordinal], dtype=np.uint64)
    outc = np.zeros(max(log_cap, 1), dtype=np.int32)
    probs = np.zeros(max(log_cap, 1), dtype=np.float64)
    nlog = np.zeros(1, dtype=np.uint64)
    st = lib().oracle_run(_ptr(psi), n, _ptr(gates), gates.size, _ptr(mats), seed, _ptr(ordn),
                          thr, _ptr(outc), _ptr(probs), log_cap, _ptr(nlog))
    k = min(int(nlog[0]), log_cap)
    return RunResult(st, outc[:k].copy(), probs[:k].copy(), int(ordn[0]))


def prob(psi: np.ndarray, n: int, q: int):
    p0 = np.zeros(1)
    p1 = np.zeros(1)
    lib().oracle_prob(_ptr(psi), n, q, _ptr(p0), _ptr(p1))
    return float(p0[0]), float(p1[0])


def measure(psi: np.ndarray, n: int, q: int, seed: int, k: int, mode: int = 0, thr: float = 0.0):
    out = np.zeros(1, dtype=np.int32)
    pr = np.zeros(1)
    st = lib().oracle_measure(_ptr(psi), n, q, seed, k, mode, thr, _ptr(out), _ptr(pr))
    return st, int(out[0]), float(pr[0])


def reset(psi: np.ndarray, n: int, q: int, seed: int, k: int):
    out = np.zeros(1, dtype=np.int32)
    pr = np.zeros(1)
    st = lib().oracle_reset(_ptr(psi), n, q, seed, k, _ptr(out), _ptr(pr))
    return st, int(out[0]), float(pr[0])


def expect(psi: np.ndarray, n: int, terms: np.ndarray) -> np.ndarray:
    terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
    out = np.zeros(max(terms.size, 1))
    lib().oracle_expect(_ptr(psi), n, _ptr(terms), terms.size, _ptr(out))
    return out[: terms.size]


def philox_block(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint64).reshape(4).copy()
    k = np.asarray(key, dtype=np.uint64).reshape(2).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed: int, k: int) -> float:
    return float(lib().oracle_draw(seed, k))


def shot_draw(seed: int, s: int) -> float:
    """The uniform draw of final-state shot s (Philox counter (s, 1, 0, 0))."""
    return float(lib().oracle_shot_draw(seed, s))


def sample(psi: np.ndarray, n: int, shots: int, seed: int, mask: int | None = None) -> np.ndarray:
    """Final-state shots from |psi|^2: packed bits of `mask` (default: all qubits)."""
    mask = (1 << n) - 1 if mask is None else mask
    out = np.zeros(max(shots, 1), dtype=np.uint64)
    st = lib().oracle_sample(_ptr(psi), n, mask, shots, seed, _ptr(out))
    if st:
        raise MemoryError("oracle_sample: no memory for the cumulative distribution")
    return out[:shots]
