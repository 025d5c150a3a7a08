"""Failure paths of the C ABI, each made on the host: an allocator hook that
returns NULL (QSIM_E_OOM, the context stays usable), a bounded wait that runs
out while legitimate work is still running (QSIM_E_TIMEOUT, nothing is lost),
served requests cancelled before admission (QSIM_E_CANCELED), and admission
held back by the device-memory budget.  No test here makes the GPU fault,
trap or wait on anything that does not finish by itself."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
qs = pytest.importorskip("paper_2310_17739_gb300.qsim")


class SwitchableAllocator:
    """Torch's caching allocator behind the library's hook, with a switch that
    makes every allocation fail (returns NULL) while it is on."""

    def __init__(self):
        self.failing = False
        self.calls = 0
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, user):
            self.calls += 1
            if self.failing:
                return None
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

        def _free(ptr, nbytes, stream, user):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = qs.ALLOC_FN(_alloc)
        self.free = qs.FREE_FN(_free)


def state_of(h, n, dtype):
    out = np.zeros(1 << n, dtype=np.complex64 if dtype == qs.C64 else np.complex128)
    assert qs.lib().qsim_state(h, ctypes.c_void_p(out.ctypes.data), out.nbytes, 0) == qs.OK
    return out


@pytest.mark.parametrize("dtype,n", [(qs.C64, 10), (qs.C128, 16)])
def test_allocator_returning_null_gives_oom_and_the_context_stays_usable(dtype, n):
    lib = qs.lib()
    al = SwitchableAllocator()
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = ctypes.c_void_p()
    al.failing = True
    assert lib.qsim_create(n, dtype, sp, al.alloc, al.free, None, ctypes.byref(h)) == qs.E_OOM
    assert not h.value and al.calls >= 1
    al.failing = False
    assert lib.qsim_create(n, dtype, sp, al.alloc, al.free, None, ctypes.byref(h)) == qs.OK
    c = W.ucc_circuit(n, seed=5, n_gadgets=20, w_lo=2, w_hi=5, target_gates=800, n_meas=2)
    g = np.ascontiguousarray(c.gates)
    # the program upload fails: nothing is enqueued and the state is left as it was
    al.failing = True
    assert lib.qsim_apply(h, ctypes.c_void_p(g.ctypes.data), g.size, None, 0) == qs.E_OOM
    assert b"allocation" in lib.qsim_last_error(h)
    al.failing = False
    assert lib.qsim_sync(h) == qs.OK
    st0 = state_of(h, n, dtype)
    assert st0[0] == 1 and np.count_nonzero(st0) == 1
    # and the same call succeeds once memory is there again
    assert lib.qsim_apply(h, ctypes.c_void_p(g.ctypes.data), g.size, None, 0) == qs.OK
    assert lib.qsim_sync(h) == qs.OK
    ref = oracle.basis_state(n)
    r = oracle.run(ref, n, c.gates)
    got = state_of(h, n, dtype)
    if dtype == qs.C128:
        assert np.abs(got - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, got) <= 1e-5
    outs = np.zeros(8, dtype=np.int32)
    probs = np.zeros(8)
    nt = ctypes.c_size_t()
    assert lib.qsim_outcomes(h, ctypes.c_void_p(outs.ctypes.data), ctypes.c_void_p(probs.ctypes.data), 8,
                             ctypes.byref(nt)) == qs.OK
    assert list(outs[: nt.value]) == list(r.outcomes)
    assert lib.qsim_destroy(h) == qs.OK


def test_bounded_wait_times_out_while_work_runs_and_reports_it_later():
    """22 qubits, paper fusion, every pass launched from the host: the stream
    holds far more than 0.1 ms of work when qsim_apply returns, so a 0.1 ms
    bound expires (QSIM_E_TIMEOUT); the work is not cancelled, and a generous
    bound then returns OK with the state equal, bit for bit, to the same
    stream synchronised without a bound."""
    n = 22
    c = W.ucc_circuit(n, seed=22, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=60_000)
    cfg = dict(fusion=1, graphs=2)
    a = qs.Sim(n, "c64", config=cfg)
    with pytest.raises(qs.QsimError):
        a.set_config(chunk_gates=-1)
    assert qs.lib().qsim_sync_timeout(a.h, -1.0) == qs.E_INVAL
    a.apply(c.gates)
    t0 = time.perf_counter()
    assert a.sync_timeout(1e-4) == qs.E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert b"keeps running" in qs.lib().qsim_last_error(a.h)
    assert a.sync_timeout(120.0) == qs.OK
    assert a.sync_timeout(0.0) == qs.OK          # nothing left to wait for
    b = qs.Sim(n, "c64", config=cfg)
    b.apply(c.gates)
    assert b.sync() == qs.OK
    assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()


def collect(srv, k, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < k and time.time() - t0 < timeout:
        for r in srv.poll():
            got[r["id"]] = r
        time.sleep(0.002)
    assert len(got) == k, srv.counts()
    return got


def test_server_cancels_requests_that_wait_and_keeps_the_order_of_the_rest():
    """One slot: a long request runs while three short ones wait; two of those
    are cancelled (results delivered at once with QSIM_E_CANCELED, never
    admitted), the third still runs and matches the oracle.  Running,
    finished, cancelled and unknown ids cannot be cancelled."""
    srv = qs.Server(slots=1, dtype="c64", config=dict(fusion=2))
    long_c = W.ucc_circuit(22, seed=7, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=1_000_000)
    short = [W.ucc_circuit(10, seed=70 + i, n_gadgets=20, w_lo=2, w_hi=5, target_gates=600, n_meas=2)
             for i in range(3)]
    a = srv.submit(long_c.n, long_c.gates, seed=1)
    ids = [srv.submit(c.n, c.gates, seed=10 + i) for i, c in enumerate(short)]
    assert srv.cancel(ids[0]) == qs.OK
    assert srv.cancel(ids[2]) == qs.OK
    assert srv.cancel(ids[2]) == qs.E_INVAL          # already cancelled
    assert srv.cancel(999_999) == qs.E_INVAL         # unknown
    got = collect(srv, 4, timeout=300.0)
    for i in (0, 2):
        r = got[ids[i]]
        assert r["status"] == qs.E_CANCELED and r["t_admit"] == -1.0 and r["t_done"] >= r["t_submit"]
    assert got[a]["status"] == qs.OK and got[ids[1]]["status"] == qs.OK
    assert got[ids[1]]["t_admit"] >= got[a]["t_done"]   # one slot, arrival order kept
    assert srv.cancel(a) == qs.E_INVAL                  # finished
    ref = oracle.basis_state(10)
    o = oracle.run(ref, 10, short[1].gates, seed=11)
    assert got[ids[1]]["outcomes"] == sum(int(b) << k for k, b in enumerate(o.outcomes))
    assert np.abs(got[ids[1]]["z"] - oracle.expect(ref, 10, W.z_terms(10))).max() <= 2e-5
    cnt = srv.counts()
    assert (cnt["submitted"], cnt["admitted"], cnt["completed"], cnt["pending"], cnt["running"]) == (4, 2, 4, 0, 0)
    srv.close()


def test_server_admits_by_device_memory_budget():
    """Four slots but a budget that holds one 18-qubit request at a time:
    requests wait for memory, not for slots, so their device spans do not
    overlap.  Results match the oracle with that budget and with the default
    one."""
    reqs = [W.ucc_circuit(18, seed=180 + i, n_gadgets=30, w_lo=2, w_hi=6, target_gates=3000, n_meas=1)
            for i in range(4)]
    state_bytes = 8 << 18
    spans = {}
    for budget in (int(1.5 * state_bytes), 0):
        srv = qs.Server(slots=4, mem_budget=budget, dtype="c64", config=dict(fusion=2))
        ids = [srv.submit(c.n, c.gates, seed=30 + i) for i, c in enumerate(reqs)]
        got = collect(srv, len(ids))
        srv.close()
        spans[budget] = sorted((got[i]["t_admit"], got[i]["t_done"]) for i in ids)
        for i, c in zip(ids, reqs):
            ref = oracle.basis_state(c.n)
            oracle.run(ref, c.n, c.gates, seed=30 + ids.index(i))
            assert got[i]["status"] == qs.OK
            assert np.abs(got[i]["z"] - oracle.expect(ref, c.n, W.z_terms(c.n))[:18]).max() <= 2e-5
    tight = spans[int(1.5 * state_bytes)]
    assert all(tight[k + 1][0] >= tight[k][1] for k in range(len(tight) - 1)), tight
