"""The measurement assertion (the paper's MMA) end to end on a synthetic
projection filter whose probabilities have a closed form."""
import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import workload as W
from tests import helpers as H
from tests.test_oracle_pins import filter_closed_form

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
qs = pytest.importorskip("paper_2310_17739_gb300.qsim")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_small_filter_matches_the_oracle(dtype):
    c = W.projection_filter(8, seed=3, blocks=6, trotter=5)
    ref = oracle.basis_state(c.n)
    r = oracle.run(ref, c.n, c.gates, seed=0)
    sim = qs.Sim(c.n, dtype, config=dict(fusion=2, tile_bits=6))
    sim.apply(c.gates)
    assert sim.sync() == 0
    out, prob = sim.outcomes()
    assert np.array_equal(out, r.outcomes)
    tol = 1e-10 if dtype == "c128" else 1e-5
    assert np.abs(prob - r.probs).max() <= tol
    if dtype == "c128":
        assert np.abs(sim.state() - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, sim.state()) <= 1e-5


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_deep_filter_at_21_qubits(dtype):
    """20 system qubits + ancilla, 8 filter blocks of 500 Trotter slices
    (80,000 gates per block): every asserted P(0) and their product against the
    closed form."""
    c = W.projection_filter(20, seed=8, blocks=8, trotter=500)
    p0, prod = filter_closed_form(c.meta["thetas"], 8)
    sim = qs.Sim(c.n, dtype, config=dict(fusion=2))
    sim.apply(c.gates)
    assert sim.sync() == 0
    out, prob = sim.outcomes()
    assert np.all(out == 0)
    tol = 1e-9 if dtype == "c128" else 2e-5
    assert np.abs(prob[0::2] - p0).max() <= tol
    succ, st = sim.success_prob()
    assert abs(succ - prod) <= tol
