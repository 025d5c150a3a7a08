"""GPU tests of the serving loop (qsim_server_*): every result matches the CPU
oracle, requests overlap on the device, and each result is the same alone and
in the mix."""
import time

import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
qs = pytest.importorskip("paper_2310_17739_gb300.qsim")


def requests(k=24, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(6, 17))
        g = int(rng.integers(300, 3000))
        c = W.ucc_circuit(n, seed=seed * 1000 + i, n_gadgets=None, w_lo=2, w_hi=min(6, n), theta="uniform",
                          target_gates=g, n_meas=int(rng.integers(0, 6)))
        out.append((c, 500 + i))
    return out


def collect(srv, k, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < k and time.time() - t0 < timeout:
        for r in srv.poll():
            got[r["id"]] = r
        time.sleep(0.002)
    assert len(got) == k, srv.counts()
    return got


@pytest.mark.parametrize("slots", [1, 8])
def test_serving_matches_oracle(slots):
    reqs = requests()
    srv = qs.Server(slots=slots, dtype="c64", config=dict(fusion=2))
    ids = [srv.submit(c.n, c.gates, seed=s) for c, s in reqs]
    got = collect(srv, len(reqs))
    for rid, (c, s) in zip(ids, reqs):
        r = got[rid]
        assert r["status"] == 0
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        ref = oracle.basis_state(c.n)
        o = oracle.run(ref, c.n, c.gates, seed=s)
        bits = sum(int(b) << i for i, b in enumerate(o.outcomes))
        assert r["n_meas"] == len(o.outcomes) and r["outcomes"] == bits
        z_ref = oracle.expect(ref, c.n, W.z_terms(c.n))
        assert np.abs(r["z"] - z_ref).max() <= 2e-5
    cnt = srv.counts()
    assert cnt["completed"] == len(reqs) and cnt["running"] == 0
    srv.close()


def test_same_alone_and_in_the_mix():
    reqs = requests(k=16, seed=3)
    mix = qs.Server(slots=8, dtype="c64", config=dict(fusion=2))
    ids = [mix.submit(c.n, c.gates, seed=s) for c, s in reqs]
    got = collect(mix, len(reqs))
    mix.close()
    for j in (0, 5, 11):
        c, s = reqs[j]
        alone = qs.Server(slots=1, dtype="c64", config=dict(fusion=2))
        rid = alone.submit(c.n, c.gates, seed=s)
        r = collect(alone, 1)[rid]
        alone.close()
        m = got[ids[j]]
        assert r["outcomes"] == m["outcomes"] and r["status"] == m["status"]
        assert np.array_equal(r["z"], m["z"])     # bitwise: same kernels, same reduction shape


def test_requests_overlap_and_admit_as_slots_free():
    """More requests than slots: later ones are admitted only as earlier ones
    finish, and with several slots the device runs requests concurrently."""
    reqs = requests(k=12, seed=9)
    srv = qs.Server(slots=4, dtype="c64", config=dict(fusion=2))
    ids = [srv.submit(c.n, c.gates, seed=s) for c, s in reqs]
    got = collect(srv, len(reqs))
    spans = sorted((got[i]["t_admit"], got[i]["t_done"]) for i in ids)
    overlap = any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    assert overlap
    srv.close()


def test_server_rejects_bad_requests():
    srv = qs.Server(slots=2, dtype="c64")
    with pytest.raises(qs.QsimError):
        srv.submit(4, W.records([(W.OP["H"], 4, 0, 0, 0, 0)]))
    with pytest.raises(qs.QsimError):
        srv.submit(40, W.records([]))
    srv.close()
