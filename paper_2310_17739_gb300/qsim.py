"""ctypes binding of libqsim.so (the C ABI declared in include/qsim.h).

Argument marshalling only: every step of gate application, measurement and
expectation runs in the library's sm_103a kernels.  Device memory comes from
PyTorch's caching allocator (through the library's allocator hook) and work is
enqueued on PyTorch's current CUDA stream.  Importing this module raises if the
native library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from .workload import GATE_DTYPE, TERM_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"native library missing: {LIB_PATH} (run __graft_entry__.build() or "
                      "python -m paper_2310_17739_gb300.build)")

_lib = ctypes.CDLL(LIB_PATH)

C64, C128 = 0, 1
PAULI_K = 7  # op-size marker of a Pauli rotation in the compiled op list
OK, E_INVAL, E_OOM, E_CUDA, E_ZEROPROB, E_TIMEOUT, E_STATE, E_CANCELED = range(8)
MEAS_ASSERT = 1
_vp, _sz, _u64, _i32, _dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int, ctypes.c_double


class QsimConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("fusion", ctypes.c_int32), ("k_max", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("chunk_gates", ctypes.c_int32),
                ("lookahead", ctypes.c_int32), ("compile_threads", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("graphs", ctypes.c_int32), ("forced_low", ctypes.c_int32)]


class ProgramInfo(ctypes.Structure):
    _fields_ = [("gates", ctypes.c_uint64), ("fused_ops", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("measurements", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("op_hist", ctypes.c_uint64 * 8)]


class QsimResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_qubits", ctypes.c_int32),
                ("n_meas", ctypes.c_int32), ("pad", ctypes.c_int32), ("outcomes", ctypes.c_uint64),
                ("success", ctypes.c_double), ("z", ctypes.c_double * 32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "qsim_create": ([_i32, _i32, _vp, ALLOC_FN, FREE_FN, _vp, ctypes.POINTER(_vp)], _i32),
    "qsim_destroy": ([_vp], _i32),
    "qsim_set_stream": ([_vp, _vp], _i32),
    "qsim_set_config": ([_vp, ctypes.POINTER(QsimConfig)], _i32),
    "qsim_get_config": ([_vp, ctypes.POINTER(QsimConfig)], _i32),
    "qsim_set_seed": ([_vp, _u64], _i32),
    "qsim_set_assert_threshold": ([_vp, _dbl], _i32),
    "qsim_apply": ([_vp, _vp, _sz, _vp, _sz], _i32),
    "qsim_compile": ([_vp, _vp, _sz, _vp, _sz, ctypes.POINTER(_vp)], _i32),
    "qsim_run": ([_vp, _vp], _i32),
    "qsim_program_get_info": ([_vp, ctypes.POINTER(ProgramInfo)], _i32),
    "qsim_program_free": ([_vp], _i32),
    "qsim_measure": ([_vp, _i32, _u64, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_dbl)], _i32),
    "qsim_prob": ([_vp, _i32, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)], _i32),
    "qsim_outcomes": ([_vp, _vp, _vp, _sz, ctypes.POINTER(_sz)], _i32),
    "qsim_success_prob": ([_vp, ctypes.POINTER(_dbl)], _i32),
    "qsim_expect": ([_vp, _vp, _sz, _vp], _i32),
    "qsim_state": ([_vp, _vp, _sz, _i32], _i32),
    "qsim_set_state": ([_vp, _vp, _sz, _i32], _i32),
    "qsim_reset_state": ([_vp], _i32),
    "qsim_state_ptr": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_sz)], _i32),
    "qsim_sync": ([_vp], _i32),
    "qsim_sync_timeout": ([_vp, _dbl], _i32),
    "qsim_get_draw_ordinal": ([_vp, ctypes.POINTER(_u64)], _i32),
    "qsim_set_draw_ordinal": ([_vp, _u64], _i32),
    "qsim_config_init": ([ctypes.POINTER(QsimConfig)], None),
    "qsim_server_cancel": ([_vp, _u64], _i32),
    "qsim_batch_create": ([_i32, _vp, _i32, _vp, ALLOC_FN, FREE_FN, _vp, ctypes.POINTER(_vp)], _i32),
    "qsim_batch_destroy": ([_vp], _i32),
    "qsim_batch_set_config": ([_vp, ctypes.POINTER(QsimConfig)], _i32),
    "qsim_batch_set_seeds": ([_vp, _vp], _i32),
    "qsim_batch_set_instance_config": ([_vp, _i32, ctypes.POINTER(QsimConfig)], _i32),
    "qsim_batch_compile": ([_vp, _i32, _vp, _sz, _vp, _sz], _i32),
    "qsim_batch_compile_many": ([_vp, _i32, _vp, _vp, _vp, _vp, _vp, _i32], _i32),
    "qsim_batch_run": ([_vp], _i32),
    "qsim_batch_expect": ([_vp, _vp, _vp, _vp], _i32),
    "qsim_batch_state": ([_vp, _i32, _vp, _sz, _i32], _i32),
    "qsim_batch_outcomes": ([_vp, _i32, _vp, _vp, _sz, ctypes.POINTER(_sz)], _i32),
    "qsim_batch_resident_count": ([_vp, ctypes.POINTER(_i32)], _i32),
    "qsim_server_create": ([_i32, _sz, _i32, ctypes.POINTER(QsimConfig), _i32, ctypes.POINTER(_vp)], _i32),
    "qsim_server_destroy": ([_vp], _i32),
    "qsim_server_submit": ([_vp, _i32, _vp, _sz, _vp, _sz, _u64, _dbl, ctypes.POINTER(_u64)], _i32),
    "qsim_server_poll": ([_vp, _vp, _sz, ctypes.POINTER(_sz)], _i32),
    "qsim_server_counts": ([_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                            ctypes.POINTER(_u64), ctypes.POINTER(_u64)], _i32),
    "qsim_server_now": ([_vp], _dbl),
    "qsim_sample": ([_vp, _u64, _u64, _u64, _vp], _i32),
    "qsim_parse_qasm": ([ctypes.c_char_p, _sz, _vp, _sz, ctypes.POINTER(_sz), _vp, _sz, ctypes.POINTER(_sz),
                         ctypes.POINTER(_i32), ctypes.c_char_p, _sz], _i32),
    "qsim_profile_start": ([_vp, _i32], _i32),
    "qsim_profile_read": ([_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_u64), ctypes.POINTER(_dbl),
                           ctypes.POINTER(_dbl), ctypes.POINTER(_u64)], _i32),
    "qsim_last_error": ([_vp], ctypes.c_char_p),
    "qsim_status_string": ([_i32], ctypes.c_char_p),
    "qsim_fuse": ([_i32, _i32, _vp, _sz, _vp, _sz, ctypes.POINTER(QsimConfig), _vp, _vp, _vp, _sz, _vp, _sz,
                   ctypes.POINTER(_sz), ctypes.POINTER(_sz)], _i32),
    "qsim_schedule": ([_i32, _i32, _vp, _sz, _vp, _sz, ctypes.POINTER(QsimConfig), _vp, _vp, _vp, _vp, _sz,
                       ctypes.POINTER(_sz)], _i32),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def lib():
    return _lib


class QsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.qsim_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(st, ctx=None):
    if st != OK:
        msg = _lib.qsim_last_error(ctx).decode(errors="replace")
        raise QsimError(st, msg)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def _gates(g):
    g = np.ascontiguousarray(g, dtype=GATE_DTYPE)
    return g


def _mats(m):
    if m is None:
        return np.zeros(1, dtype=np.float64)
    return np.ascontiguousarray(m, dtype=np.float64).ravel()


def make_config(fusion=1, k_max=2, tile_bits=0, threads=0, chunk_gates=0, lookahead=0,
                compile_threads=0, persistent=0, graphs=0, forced_low=0) -> QsimConfig:
    return QsimConfig(ctypes.sizeof(QsimConfig), fusion, k_max, tile_bits, threads, chunk_gates, lookahead,
                      compile_threads, persistent, graphs, forced_low)


# ----------------------------------------------------------- torch plumbing --
class _TorchAllocator:
    """Device memory through torch's caching allocator (stream-ordered frees)."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            if ptr:
                self.torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Program:
    def __init__(self, sim, handle):
        self.sim = sim
        self.handle = handle

    def info(self) -> dict:
        inf = ProgramInfo()
        _check(_lib.qsim_program_get_info(self.handle, ctypes.byref(inf)))
        return dict(gates=inf.gates, fused_ops=inf.fused_ops, passes=inf.passes,
                    measurements=inf.measurements, device_bytes=inf.device_bytes,
                    op_hist=list(inf.op_hist))

    def free(self):
        if self.handle:
            _lib.qsim_program_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Sim:
    """One state vector of n qubits on the current CUDA device."""

    def __init__(self, n: int, dtype: str = "c64", stream=None, torch_memory: bool = True,
                 config: Optional[dict] = None, seed: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.n = n
        self.dtype = C64 if dtype in ("c64", C64) else C128
        self.np_dtype = np.complex64 if self.dtype == C64 else np.complex128
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._alloc = _TorchAllocator(self.device) if torch_memory else None
        h = ctypes.c_void_p()
        _check(_lib.qsim_create(n, self.dtype, sp,
                                self._alloc.alloc if self._alloc else ALLOC_FN(),
                                self._alloc.free if self._alloc else FREE_FN(),
                                None, ctypes.byref(h)))
        self.h = h
        if config:
            self.set_config(**config)
        if seed:
            self.set_seed(seed)

    # -- configuration
    def set_config(self, **kw):
        cfg = self.get_config()
        cfg.update(kw)
        _check(_lib.qsim_set_config(self.h, ctypes.byref(make_config(**cfg))), self.h)

    def get_config(self) -> dict:
        c = QsimConfig()
        _check(_lib.qsim_get_config(self.h, ctypes.byref(c)), self.h)
        return dict(fusion=c.fusion, k_max=c.k_max, tile_bits=c.tile_bits, threads=c.threads,
                    chunk_gates=c.chunk_gates, lookahead=c.lookahead, compile_threads=c.compile_threads,
                    persistent=c.persistent, graphs=c.graphs, forced_low=c.forced_low)

    def set_seed(self, seed: int):
        _check(_lib.qsim_set_seed(self.h, seed), self.h)

    def set_assert_threshold(self, thr: float):
        _check(_lib.qsim_set_assert_threshold(self.h, thr), self.h)

    # -- gates
    def apply(self, gates, mats=None):
        g = _gates(gates)
        m = _mats(mats)
        _check(_lib.qsim_apply(self.h, _ptr(g), g.size, _ptr(m), m.size), self.h)

    def compile(self, gates, mats=None) -> Program:
        g = _gates(gates)
        m = _mats(mats)
        p = ctypes.c_void_p()
        _check(_lib.qsim_compile(self.h, _ptr(g), g.size, _ptr(m), m.size, ctypes.byref(p)), self.h)
        return Program(self, p)

    def run(self, prog: Program):
        _check(_lib.qsim_run(self.h, prog.handle), self.h)

    # -- measurement
    def measure(self, qubit: int, seed: int, mode: int = 0):
        out = ctypes.c_int()
        pr = ctypes.c_double()
        st = _lib.qsim_measure(self.h, qubit, seed, mode, ctypes.byref(out), ctypes.byref(pr))
        if st == E_ZEROPROB:
            return -1, pr.value, st
        _check(st, self.h)
        return out.value, pr.value, st

    def measure_async(self, qubit: int, seed: int, mode: int = 0):
        _check(_lib.qsim_measure(self.h, qubit, seed, mode, None, None), self.h)

    def prob(self, qubit: int):
        p0, p1 = ctypes.c_double(), ctypes.c_double()
        _check(_lib.qsim_prob(self.h, qubit, ctypes.byref(p0), ctypes.byref(p1)), self.h)
        return p0.value, p1.value

    def outcomes(self, check: bool = True):
        n = ctypes.c_size_t()
        _check(_lib.qsim_outcomes(self.h, None, None, 0, ctypes.byref(n)), self.h)
        k = n.value
        oc = np.zeros(max(k, 1), dtype=np.int32)
        pr = np.zeros(max(k, 1), dtype=np.float64)
        st = _lib.qsim_outcomes(self.h, _ptr(oc), _ptr(pr), k, ctypes.byref(n))
        if check:
            _check(st, self.h)
        return oc[:k].copy(), pr[:k].copy()

    def success_prob(self):
        p = ctypes.c_double()
        st = _lib.qsim_success_prob(self.h, ctypes.byref(p))
        return p.value, st

    # -- expectation
    def expect(self, terms) -> np.ndarray:
        t = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        out = np.zeros(max(t.size, 1), dtype=np.float64)
        _check(_lib.qsim_expect(self.h, _ptr(t), t.size, _ptr(out)), self.h)
        return out[: t.size]

    # -- state
    def state(self) -> np.ndarray:
        a = np.zeros(1 << self.n, dtype=self.np_dtype)
        _check(_lib.qsim_state(self.h, _ptr(a), a.nbytes, 0), self.h)
        return a

    def state_tensor(self):
        """A torch view (no copy) of the device state."""
        import torch
        p = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        _check(_lib.qsim_state_ptr(self.h, ctypes.byref(p), ctypes.byref(nb)), self.h)
        return p.value, nb.value

    def set_state(self, arr):
        a = np.ascontiguousarray(arr, dtype=self.np_dtype)
        _check(_lib.qsim_set_state(self.h, _ptr(a), a.nbytes, 0), self.h)

    def reset(self):
        _check(_lib.qsim_reset_state(self.h), self.h)

    def sync(self):
        return _lib.qsim_sync(self.h)

    def draw_ordinal(self) -> int:
        """Ordinal of the next measurement draw (checkpoint / resume)."""
        k = ctypes.c_uint64()
        _check(_lib.qsim_get_draw_ordinal(self.h, ctypes.byref(k)), self.h)
        return k.value

    def set_draw_ordinal(self, k: int):
        _check(_lib.qsim_set_draw_ordinal(self.h, int(k)), self.h)

    def sync_timeout(self, seconds: float):
        """qsim_sync with a bounded wait: E_TIMEOUT if the work is still running."""
        return _lib.qsim_sync_timeout(self.h, float(seconds))

    # -- sampled kernel timing
    def sample(self, shots: int, seed: int = 0, mask: int | None = None) -> np.ndarray:
        """Final-state shots without collapse (see qsim_sample): packed bits of `mask`
        (default: every qubit) per shot."""
        mask = (1 << self.n) - 1 if mask is None else int(mask)
        out = np.zeros(max(int(shots), 1), dtype=np.uint64)
        _check(_lib.qsim_sample(self.h, mask, int(shots), int(seed), _ptr(out)), self.h)
        return out[: int(shots)]

    def profile_start(self, every: int):
        _check(_lib.qsim_profile_start(self.h, every), self.h)

    def profile_read(self) -> dict:
        ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        ns, nl = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.qsim_profile_read(self.h, ctypes.byref(ms), ctypes.byref(ns), ctypes.byref(fl),
                                      ctypes.byref(by), ctypes.byref(nl)), self.h)
        return dict(ms=ms.value, samples=ns.value, flops=fl.value, bytes=by.value, launches=nl.value)

    def close(self):
        if getattr(self, "h", None):
            _lib.qsim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent states advanced together (see qsim_batch_* in qsim.h)."""

    def __init__(self, n_qubits, dtype: str = "c64", stream=None, torch_memory: bool = True,
                 config: Optional[dict] = None, seeds=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.n = [int(x) for x in n_qubits]
        self.dtype = C64 if dtype in ("c64", C64) else C128
        self.np_dtype = np.complex64 if self.dtype == C64 else np.complex128
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._alloc = _TorchAllocator(self.device) if torch_memory else None
        nq = np.asarray(self.n, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(_lib.qsim_batch_create(len(self.n), _ptr(nq), self.dtype, sp,
                                      self._alloc.alloc if self._alloc else ALLOC_FN(),
                                      self._alloc.free if self._alloc else FREE_FN(), None,
                                      ctypes.byref(h)))
        self.h = h
        if config:
            _check(_lib.qsim_batch_set_config(self.h, ctypes.byref(make_config(**config))))
        if seeds is not None:
            s = np.ascontiguousarray(seeds, dtype=np.uint64)
            _check(_lib.qsim_batch_set_seeds(self.h, _ptr(s)))

    def __len__(self):
        return len(self.n)

    def set_instance_config(self, index: int, **config):
        """Configuration of one instance (applies to its next compile)."""
        _check(_lib.qsim_batch_set_instance_config(self.h, index, ctypes.byref(make_config(**config))))

    def compile(self, index: int, gates, mats=None):
        g = _gates(gates)
        m = _mats(mats)
        _check(_lib.qsim_batch_compile(self.h, index, _ptr(g), g.size, _ptr(m), m.size))

    def compile_many(self, gate_lists, indices=None, mats_lists=None, threads: int = 0):
        """compile(i, gates) for many instances at once (host compilation on
        worker threads); indices default to 0..len(gate_lists)-1."""
        idx = np.arange(len(gate_lists), dtype=np.int32) if indices is None else \
            np.ascontiguousarray(indices, dtype=np.int32)
        gs = [_gates(g) for g in gate_lists]
        ms = [_mats(m) for m in (mats_lists or [None] * len(gs))]
        k = len(gs)
        gp = (ctypes.c_void_p * max(k, 1))(*[g.ctypes.data if g.size else None for g in gs])
        ng = np.array([g.size for g in gs], dtype=np.uint64)
        mp = (ctypes.c_void_p * max(k, 1))(*[m.ctypes.data if m.size else None for m in ms])
        nm = np.array([m.size for m in ms], dtype=np.uint64)
        _check(_lib.qsim_batch_compile_many(self.h, k, _ptr(idx), ctypes.cast(gp, ctypes.c_void_p), _ptr(ng),
                                            ctypes.cast(mp, ctypes.c_void_p), _ptr(nm), threads))

    def run(self):
        _check(_lib.qsim_batch_run(self.h))

    def expect(self, term_lists):
        """term_lists[i]: TERM_DTYPE array for instance i -> list of per-term values."""
        arrs = [np.ascontiguousarray(t, dtype=TERM_DTYPE) for t in term_lists]
        off = np.zeros(len(arrs) + 1, dtype=np.uint64)
        off[1:] = np.cumsum([a.size for a in arrs])
        allt = np.concatenate(arrs) if arrs else np.zeros(0, dtype=TERM_DTYPE)
        out = np.zeros(max(int(off[-1]), 1), dtype=np.float64)
        _check(_lib.qsim_batch_expect(self.h, _ptr(allt), _ptr(off), _ptr(out)))
        return [out[int(off[i]):int(off[i + 1])].copy() for i in range(len(arrs))]

    def state(self, index: int) -> np.ndarray:
        a = np.zeros(1 << self.n[index], dtype=self.np_dtype)
        _check(_lib.qsim_batch_state(self.h, index, _ptr(a), a.nbytes, 0))
        return a

    def outcomes(self, index: int):
        n = ctypes.c_size_t()
        st = _lib.qsim_batch_outcomes(self.h, index, None, None, 0, ctypes.byref(n))
        k = n.value
        oc = np.zeros(max(k, 1), dtype=np.int32)
        pr = np.zeros(max(k, 1), dtype=np.float64)
        st = _lib.qsim_batch_outcomes(self.h, index, _ptr(oc), _ptr(pr), k, ctypes.byref(n))
        return oc[:k].copy(), pr[:k].copy(), st

    def resident_count(self) -> int:
        k = ctypes.c_int()
        _check(_lib.qsim_batch_resident_count(self.h, ctypes.byref(k)))
        return k.value

    def close(self):
        if getattr(self, "h", None):
            _lib.qsim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-admission request loop (see qsim_server_* in qsim.h)."""

    def __init__(self, slots: int = 16, mem_budget: int = 0, dtype: str = "c64",
                 config: Optional[dict] = None, compile_threads: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        torch.cuda.current_device()
        self.dtype = C64 if dtype in ("c64", C64) else C128
        cfg = make_config(**(config or {}))
        h = ctypes.c_void_p()
        _check(_lib.qsim_server_create(slots, mem_budget, self.dtype, ctypes.byref(cfg), compile_threads,
                                       ctypes.byref(h)))
        self.h = h
        self._buf = (QsimResult * 256)()

    def submit(self, n: int, gates, mats=None, seed: int = 0, t_submit: float = -1.0) -> int:
        g = _gates(gates)
        m = _mats(mats)
        rid = ctypes.c_uint64()
        _check(_lib.qsim_server_submit(self.h, n, _ptr(g), g.size, _ptr(m), m.size, seed, t_submit,
                                       ctypes.byref(rid)))
        return rid.value

    def poll(self):
        out = []
        while True:
            k = ctypes.c_size_t()
            _check(_lib.qsim_server_poll(self.h, ctypes.cast(self._buf, ctypes.c_void_p), 256, ctypes.byref(k)))
            for i in range(k.value):
                r = self._buf[i]
                out.append(dict(id=r.id, status=r.status, n=r.n_qubits, n_meas=r.n_meas,
                                outcomes=r.outcomes, success=r.success,
                                z=np.array(r.z[: min(r.n_qubits, 32)]), t_submit=r.t_submit,
                                t_admit=r.t_admit, t_done=r.t_done))
            if k.value < 256:
                return out

    def cancel(self, rid: int) -> int:
        """Cancel a request that has not been admitted (status of the call)."""
        return _lib.qsim_server_cancel(self.h, rid)

    def counts(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(5)]
        _check(_lib.qsim_server_counts(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("submitted", "admitted", "completed", "pending", "running"), (x.value for x in v)))

    def now(self) -> float:
        return _lib.qsim_server_now(self.h)

    def close(self):
        if getattr(self, "h", None):
            _lib.qsim_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------- host-only inspection --
def fuse(n, gates, mats=None, dtype=C64, **cfg):
    """Compiled op list of one chunk: list of (k, qubits, matrix) / ('event', op, q, flags)
    / ('pauli', x, z, theta) for exp(-i theta P) / ('frame', x, z, g) for
    i^g exp(-i pi/2 P), with P = i^{|x & z|} X^x Z^z."""
    g = _gates(gates)
    m = _mats(mats)
    c = make_config(**cfg)
    nops, nmd = ctypes.c_size_t(), ctypes.c_size_t()
    st = _lib.qsim_fuse(n, dtype, _ptr(g), g.size, _ptr(m), m.size, ctypes.byref(c), None, None, None, 0,
                        None, 0, ctypes.byref(nops), ctypes.byref(nmd))
    if st not in (OK, E_INVAL) or (st == E_INVAL and nops.value == 0 and g.size):
        _check(st)
    K = max(nops.value, 1)
    ok = np.zeros(K, dtype=np.uint8)
    oq = np.zeros(6 * K, dtype=np.uint32)
    om = np.zeros(K, dtype=np.uint64)
    md = np.zeros(max(nmd.value, 1), dtype=np.float64)
    _check(_lib.qsim_fuse(n, dtype, _ptr(g), g.size, _ptr(m), m.size, ctypes.byref(c), _ptr(ok), _ptr(oq),
                          _ptr(om), K, _ptr(md), md.size, ctypes.byref(nops), ctypes.byref(nmd)))
    out = []
    for i in range(nops.value):
        k = int(ok[i])
        if k == 0:
            out.append(("event", int(oq[6 * i + 1]), int(oq[6 * i]), int(oq[6 * i + 2])))
        elif k == PAULI_K:
            xm = int(oq[6 * i]) | (int(oq[6 * i + 1]) << 32)
            zm = int(oq[6 * i + 2]) | (int(oq[6 * i + 3]) << 32)
            fl = int(oq[6 * i + 4])
            off = int(om[i])
            if fl & 4:  # Pauli-frame flush: i^g exp(-i pi/2 P)
                out.append(("frame", xm, zm, fl & 3))
            else:
                out.append(("pauli", xm, zm, float(np.arctan2(md[off + 1], md[off]))))
        else:
            d = 1 << k
            off = int(om[i])
            M = md[off: off + 2 * d * d].view(np.complex128).reshape(d, d).copy()
            out.append((k, [int(x) for x in oq[6 * i: 6 * i + k]], M))
    return out


def parse_qasm(text):
    """OpenQASM 2.0 text -> (n_qubits, gate records, matrix doubles); see qsim_parse_qasm."""
    raw = text.encode() if isinstance(text, str) else bytes(text)
    ng, nm, nq = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
    err = ctypes.create_string_buffer(512)
    st = _lib.qsim_parse_qasm(raw, len(raw), None, 0, ctypes.byref(ng), None, 0, ctypes.byref(nm),
                              ctypes.byref(nq), err, 512)
    if st != OK and not (st == E_INVAL and err.value == b"output capacity too small"):
        raise QsimError(st, err.value.decode(errors="replace"))
    g = np.zeros(max(ng.value, 1), dtype=GATE_DTYPE)
    m = np.zeros(max(nm.value, 1), dtype=np.float64)
    st = _lib.qsim_parse_qasm(raw, len(raw), _ptr(g), g.size, ctypes.byref(ng), _ptr(m), m.size,
                              ctypes.byref(nm), ctypes.byref(nq), err, 512)
    if st != OK:
        raise QsimError(st, err.value.decode(errors="replace"))
    return nq.value, g[: ng.value], m


def schedule(n, gates, mats=None, dtype=C64, with_basis=False, **cfg):
    """Pass table of one chunk: list of (pivot_mask, first, count), or with
    with_basis=True (pivot_mask, first, count, basis_vectors)."""
    g = _gates(gates)
    m = _mats(mats)
    c = make_config(**cfg)
    npass = ctypes.c_size_t()
    _lib.qsim_schedule(n, dtype, _ptr(g), g.size, _ptr(m), m.size, ctypes.byref(c), None, None, None, None, 0,
                       ctypes.byref(npass))
    K = max(npass.value, 1)
    t = np.zeros(K, dtype=np.uint64)
    f = np.zeros(K, dtype=np.uint64)
    cnt = np.zeros(K, dtype=np.uint32)
    b = np.zeros(16 * K, dtype=np.uint64)
    _check(_lib.qsim_schedule(n, dtype, _ptr(g), g.size, _ptr(m), m.size, ctypes.byref(c), _ptr(t), _ptr(f),
                              _ptr(cnt), _ptr(b), K, ctypes.byref(npass)))
    if with_basis:
        return [(int(t[i]), int(f[i]), int(cnt[i]), [int(v) for v in b[16 * i: 16 * i + 16] if v])
                for i in range(npass.value)]
    return [(int(t[i]), int(f[i]), int(cnt[i])) for i in range(npass.value)]
