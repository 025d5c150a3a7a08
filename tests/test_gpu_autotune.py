"""The autotuner through the C ABI: the configuration it picks (single state,
and per width group of a batch) runs the circuit to the oracle's result."""
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
autotune = pytest.importorskip("paper_2310_17739_gb300.autotune")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_tuned_configuration_matches_the_oracle(dtype):
    n = 16
    c = W.ucc_circuit(n, seed=161, n_gadgets=60, w_lo=2, w_hi=6, theta="uniform", target_gates=20_000, n_meas=3)
    best, entry = autotune.tune(n, c.gates, dtype, prefix=8_000, use_cache=False)
    assert best in autotune.candidates(n, dtype)
    assert len(entry["report"]) == len(autotune.candidates(n, dtype))
    assert all(r["gates_per_s"] > 0 for r in entry["report"])
    ref = oracle.basis_state(n)
    r = oracle.run(ref, n, c.gates, seed=3)
    sim = qs.Sim(n, dtype, seed=3, config=best)
    sim.apply(c.gates)
    assert sim.sync() == 0
    out, _ = sim.outcomes()
    assert np.array_equal(out, r.outcomes)
    if dtype == "c128":
        assert np.abs(sim.state() - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, sim.state()) <= 1e-5
    sim.close()


def test_batch_tuned_per_width_group():
    widths = [10, 12, 12, 15, 16]
    cs = [W.ucc_circuit(n, seed=200 + i, n_gadgets=40, w_lo=2, w_hi=6, theta="uniform", target_gates=4000)
          for i, n in enumerate(widths)]
    b = qs.Batch(widths, "c64")
    best = autotune.tune_batch(b, cs, prefix=4000, use_cache=False)
    assert set(best) == set(widths)
    for n, cfg in best.items():
        assert cfg in autotune.candidates(n, "c64")
    b.compile_many([c.gates for c in cs])
    b.run()
    for i, c in enumerate(cs):
        ref = oracle.basis_state(c.n)
        oracle.run(ref, c.n, c.gates)
        assert 1 - H.fidelity(ref, b.state(i)) <= 1e-5, (i, best[c.n])
    b.close()
