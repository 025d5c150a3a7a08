"""GPU parity of final-state shots (qsim_sample) against the CPU oracle."""
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


def state_pair(n, dtype, seed, gates=1500, meas=2):
    c = W.ucc_circuit(n, seed=seed, n_gadgets=None, w_lo=2, w_hi=min(6, n), theta="uniform",
                      target_gates=gates, n_meas=meas if n > 2 else 0)
    ref = oracle.basis_state(n)
    oracle.run(ref, n, c.gates, seed=seed)
    sim = qs.Sim(n, dtype, seed=seed, config=dict(fusion=2))
    sim.apply(c.gates)
    assert sim.sync() == 0
    return sim, ref


def near_tie(ref, seed, shots, idx, tol):
    """Shots whose draw lies within tol of a cumulative boundary of the oracle's
    distribution (there either neighbour is a correct answer)."""
    cum = np.cumsum(np.abs(ref) ** 2)
    u = np.array([oracle.shot_draw(seed, int(s)) for s in idx]) * cum[-1]
    d = np.abs(cum[None, :] - u[:, None]).min(axis=1)
    return d <= tol * cum[-1]


@pytest.mark.parametrize("n", [3, 8, 11, 16])
def test_shots_match_the_oracle_complex128(n):
    sim, ref = state_pair(n, "c128", seed=40 + n)
    got = sim.sample(4000, seed=9)
    exp = oracle.sample(ref, n, 4000, seed=9)
    bad = np.nonzero(got != exp)[0]
    assert np.all(near_tie(ref, 9, 4000, bad, 1e-12)), bad[:10]
    for mask in (0b1, (1 << n) - 2, 0b1010101 & ((1 << n) - 1)):
        g = sim.sample(500, seed=5, mask=mask)
        e = oracle.sample(ref, n, 500, seed=5, mask=mask)
        bad = np.nonzero(g != e)[0]
        assert np.all(near_tie(ref, 5, 500, bad, 1e-12))


@pytest.mark.parametrize("n", [9, 14, 18])
def test_shots_are_valid_complex64(n):
    """complex64 amplitudes differ from the oracle's by ~1e-7, so a shot may land
    on either side of a nearby boundary: every shot must lie in the oracle's
    interval of its draw widened by 1e-5, and most must match exactly."""
    sim, ref = state_pair(n, "c64", seed=60 + n)
    shots = 3000
    got = sim.sample(shots, seed=3).astype(np.int64)
    cum = np.cumsum(np.abs(ref) ** 2)
    u = np.array([oracle.shot_draw(3, s) for s in range(shots)]) * cum[-1]
    lo = np.where(got > 0, cum[np.maximum(got - 1, 0)], 0.0)
    hi = cum[got]
    tol = 1e-5 * cum[-1]
    assert np.all((lo - tol <= u) & (u < hi + tol))
    exact = oracle.sample(ref, n, shots, seed=3).astype(np.int64)
    assert np.mean(got == exact) > 0.99


def test_zero_probability_indices_are_never_drawn():
    n = 12
    rows = [(W.OP["H"], 0, 0, 0.0, 0, 0)] + [(W.OP["CX"], 0, q, 0.0, 0, 0) for q in range(1, n)]
    sim = qs.Sim(n, "c64")
    sim.apply(W.records(rows))
    got = sim.sample(20000, seed=1)
    assert set(np.unique(got).tolist()) <= {0, (1 << n) - 1}
    frac = np.mean(got == 0)
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(20000)


def test_full_size_marginals():
    """21 qubits after a 2e6-gate prefix of the benchmark circuit (the benchmark's
    configuration): the frequency of 1 on each qubit over 200,000 shots agrees
    with the FP64 Born probability within 5 sigma, and the state is untouched."""
    c = W.config_large(target_gates=2_000_000, n_meas=0)
    sim = qs.Sim(21, "c64", config=dict(fusion=2, k_max=2, tile_bits=12))
    sim.apply(c.gates)
    assert sim.sync() == 0
    before = sim.state()
    shots = 200_000
    got = sim.sample(shots, seed=77)
    for q in range(21):
        p0, p1 = sim.prob(q)
        p = p1 / (p0 + p1)
        f = np.mean((got >> np.uint64(q)) & np.uint64(1))
        assert abs(f - p) <= 5 * np.sqrt(p * (1 - p) / shots) + 1e-9
    assert np.array_equal(sim.state(), before)
