"""GPU parity of batched execution (qsim_batch_*) against the CPU oracle, and
determinism: every instance's result is the same alone and in the mix."""
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


def mixed_circuits(seed=0):
    widths = [6, 9, 12, 12, 14, 15, 16, 10]
    cs = []
    for i, n in enumerate(widths):
        cs.append(W.ucc_circuit(n, seed=seed + i, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform",
                                target_gates=2500, n_meas=3 if i % 2 else 0))
    return cs


def run_batch(cs, dtype, config, seeds):
    b = qs.Batch([c.n for c in cs], dtype, config=config, seeds=seeds)
    for i, c in enumerate(cs):
        b.compile(i, c.gates, c.mats)
    b.run()
    return b


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("fusion", [1, 2])
def test_batch_matches_oracle(dtype, fusion):
    cs = mixed_circuits()
    seeds = [100 + i for i in range(len(cs))]
    b = run_batch(cs, dtype, dict(fusion=fusion), seeds)
    # widths up to 14 (c64) / 13 (c128) run resident, one block each
    assert b.resident_count() == sum(c.n <= (14 if dtype == "c64" else 13) for c in cs)
    hams = [W.random_hamiltonian(c.n, 40, seed=i) for i, c in enumerate(cs)]
    got_e = b.expect(hams)
    for i, c in enumerate(cs):
        ref = oracle.basis_state(c.n)
        r = oracle.run(ref, c.n, c.gates, seed=seeds[i])
        out, prob, st = b.outcomes(i)
        assert st == 0
        assert np.array_equal(out, r.outcomes), i
        got = b.state(i)
        if dtype == "c128":
            assert np.abs(got - ref).max() <= 1e-10, i
        else:
            assert 1 - H.fidelity(ref, got) <= 1e-5, i
        e_ref = oracle.expect(ref, c.n, hams[i])
        tol = 1e-10 if dtype == "c128" else 2e-5
        assert np.abs(got_e[i] - e_ref).max() <= tol * max(1.0, np.abs(hams[i]["coef"]).max()), i
    b.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_same_alone_and_in_the_mix(dtype):
    cs = mixed_circuits(seed=20)
    seeds = [7 + i for i in range(len(cs))]
    mix = run_batch(cs, dtype, dict(fusion=2), seeds)
    # run 1 was eager, run 2 is captured into a CUDA graph, run 3 replays it:
    # every run restarts from |0...0> and reproduces the same states and outcomes
    first = [mix.state(i) for i in range(len(cs))]
    first_out = [mix.outcomes(i)[0] for i in range(len(cs))]
    for _ in range(2):
        mix.run()
        for i in range(len(cs)):
            assert np.array_equal(mix.state(i), first[i]), i
            out, _, st = mix.outcomes(i)
            assert st == 0 and np.array_equal(out, first_out[i]), i
    for i in (0, 3, 5, 6):
        alone = run_batch([cs[i]], dtype, dict(fusion=2), [seeds[i]])
        assert np.array_equal(alone.state(0), mix.state(i)), i
        assert np.array_equal(alone.outcomes(0)[0], mix.outcomes(i)[0]), i
        alone.close()
    # and the same as the single-context path
    for i in (2, 5):
        sim = qs.Sim(cs[i].n, dtype, seed=seeds[i], config=dict(fusion=2, tile_bits=cs[i].n if cs[i].n <= 14 else 0))
        sim.apply(cs[i].gates)
        a, m = sim.state(), mix.state(i)
        if dtype == "c128":
            assert np.abs(a - m).max() <= 1e-12
        else:
            assert 1 - H.fidelity(a, m) <= 1e-6
    mix.close()


def test_parameter_sets_one_structure():
    cs, hams = W.config_batched(n_param_sets=6, n_uneven=2, gates=3000, n_terms=20, n_set_gadgets=200)
    b = run_batch(cs, "c64", dict(fusion=2), [0] * len(cs))
    vals = b.expect(hams)
    for i in (0, 3, 6, 7):
        ref = oracle.basis_state(cs[i].n)
        oracle.run(ref, cs[i].n, cs[i].gates)
        assert np.abs(vals[i] - oracle.expect(ref, cs[i].n, hams[i])).max() <= 2e-5
    # different angles give different states
    assert not np.allclose(b.state(0), b.state(1))
    # a second run restarts from |0...0> and reproduces the first
    before = b.state(3)
    b.run()
    assert np.array_equal(before, b.state(3))
    b.close()


def test_batch_argument_errors():
    with pytest.raises(qs.QsimError):
        qs.Batch([4, 40], "c64")
    b = qs.Batch([3, 4], "c64")
    with pytest.raises(qs.QsimError):
        b.compile(2, W.records([]))
    with pytest.raises(qs.QsimError):
        b.compile(0, W.records([(W.OP["H"], 3, 0, 0, 0, 0)]))
    with pytest.raises(qs.QsimError):
        b.expect([W.z_terms(4), W.z_terms(4)])   # instance 0 has 3 qubits
    b.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_compile_many_equals_one_by_one(dtype):
    """qsim_batch_compile_many (host compilation on worker threads) gives the
    same programs as qsim_batch_compile per instance: bitwise-equal states and
    outcomes, indices in any order, and an invalid record rejects the call."""
    cs = mixed_circuits(seed=70)
    seeds = [3 + i for i in range(len(cs))]
    cfg = dict(fusion=2)
    ref = run_batch(cs, dtype, cfg, seeds)
    b = qs.Batch([c.n for c in cs], dtype, config=cfg, seeds=seeds)
    order = list(reversed(range(len(cs))))
    b.compile_many([cs[i].gates for i in order], indices=order, mats_lists=[cs[i].mats for i in order],
                   threads=4)
    b.run()
    for i in range(len(cs)):
        assert np.array_equal(b.state(i), ref.state(i))
    bad = cs[0].gates.copy()
    bad["q0"][0] = 99
    with pytest.raises(qs.QsimError):
        b.compile_many([cs[1].gates, bad], indices=[1, 0])
