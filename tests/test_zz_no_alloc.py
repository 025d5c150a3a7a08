"""qsim_prob_noalloc: the probability reduction for callers that cannot
allocate device memory (see include/qsim.h).  Collected last on purpose.

It is checked through the C ABI against the allocating entry point qsim_prob
on the same device state, on several calls in a row (the static scratch keeps
the last call's contents, so consecutive calls exercise its reset).  Both
entry points run the same reduction kernel with the same block count and
summation order, so their FP64 results must be identical bit for bit.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
qs = pytest.importorskip("paper_2310_17739_gb300.qsim")
from paper_2310_17739_gb300 import workload as W  # noqa: E402


def noalloc():
    f = qs.lib().qsim_prob_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("dtype,n", [("c128", 12), ("c64", 21), ("c128", 3)])
def test_noalloc_matches_allocating_prob(dtype, n):
    c = W.ucc_circuit(n, seed=31, n_gadgets=30, w_lo=2, w_hi=min(6, n), target_gates=3000)
    sim = qs.Sim(n, dtype)
    sim.apply(c.gates)
    assert sim.sync() == 0
    ptr, nbytes = sim.state_tensor()
    assert nbytes == (8 if dtype == "c64" else 16) << n
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    f = noalloc()
    dt = qs.C64 if dtype == "c64" else qs.C128
    for q in (0, n - 1, n // 2, 0):  # calls in a row, the last one repeats the first qubit
        ref0, ref1 = sim.prob(q)
        a0, a1 = ctypes.c_double(-1), ctypes.c_double(-1)
        st = f(ctypes.c_void_p(ptr), n, dt, q, stream, ctypes.byref(a0), ctypes.byref(a1))
        assert st == qs.OK
        assert a0.value == ref0 and a1.value == ref1
        assert abs(a0.value + a1.value - 1.0) < (1e-12 if dtype == "c128" else 1e-5)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = noalloc()
    sim = qs.Sim(4, "c128")
    ptr, _ = sim.state_tensor()
    a0, a1 = ctypes.c_double(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, q, dt in ((35, 0, qs.C64), (0, 0, qs.C64), (4, 4, qs.C128), (4, 0, 7)):
        assert f(ctypes.c_void_p(ptr), n, dt, q, stream, ctypes.byref(a0), ctypes.byref(a1)) == qs.E_INVAL
    assert f(None, 4, qs.C128, 0, stream, ctypes.byref(a0), ctypes.byref(a1)) == qs.E_INVAL
    # still usable afterwards
    assert f(ctypes.c_void_p(ptr), 4, qs.C128, 1, stream, ctypes.byref(a0), ctypes.byref(a1)) == qs.OK
    assert a0.value == 1.0 and a1.value == 0.0
    sim.close()
