"""Full-size checks in the benchmark's launch configuration, where the CPU
oracle cannot run the whole circuit: properties that hold at any size, and
oracle parity on a prefix."""
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

# the configuration the benchmark's autotuner picks for the 21-qubit circuit
BENCH_CFG = dict(fusion=2, k_max=2, tile_bits=12)


def test_large_circuit_then_its_inverse_returns_to_zero():
    """21 qubits, the full 1.15e8-gate Trotter circuit (without its measurements,
    which are not invertible) and then its inverse: the complex64 state must come
    back to |0...0> (the inverse of every gadget is the gadget with -theta, so
    both halves run through the same rotation passes)."""
    c = W.config_large(n_meas=0)
    assert c.G >= 115_000_000
    sim = qs.Sim(21, "c64", config=BENCH_CFG)
    sim.apply(c.gates)
    assert sim.sync() == 0
    mid = sim.state()
    # FP32 rounding walks the norm over ~9.4e6 rotations with no measurement to
    # renormalise (about 1e-10 per rotation); fidelity is what the tolerance binds
    norm_mid = float(np.vdot(mid, mid).real)
    assert abs(norm_mid - 1.0) < 1e-2
    assert abs(mid[0]) ** 2 / norm_mid < 0.5          # the circuit did move the state
    sim.apply(H.invert_records(c.gates))
    assert sim.sync() == 0
    st = sim.state()
    norm = float(np.vdot(st, st).real)
    assert abs(norm - 1.0) < 2e-2
    assert 1 - abs(st[0]) ** 2 / norm <= 1e-5


def test_mid_config_full_size():
    """16 qubits, 1e6 gates, 64 mid-circuit measurements (complex64 and complex128):
    the two precisions agree on every outcome and on the final state (infidelity
    <= 1e-5), the state is normalised, and a 60,000-gate prefix matches the
    oracle bit for bit in its outcomes."""
    c = W.config_mid()
    runs = {}
    for dt in ("c128", "c64"):
        sim = qs.Sim(16, dt, seed=1002, config=dict(fusion=2))
        sim.apply(c.gates)
        assert sim.sync() == 0
        runs[dt] = (sim.state(), sim.outcomes())
        sim.close()
    (s128, (o128, p128)), (s64, (o64, p64)) = runs["c128"], runs["c64"]
    assert len(o128) == 64 and np.array_equal(o128, o64)
    assert abs(float(np.vdot(s64, s64).real) - 1.0) < 1e-5
    assert 1 - H.fidelity(s128, s64) <= 1e-5
    # oracle parity on a prefix
    cut = 60_000
    g = c.gates[:cut]
    ref = oracle.basis_state(16)
    r = oracle.run(ref, 16, g, seed=1002)
    sim = qs.Sim(16, "c128", seed=1002, config=dict(fusion=2))
    sim.apply(g)
    assert sim.sync() == 0
    out, prob = sim.outcomes()
    assert np.array_equal(out, r.outcomes)
    assert np.abs(sim.state() - ref).max() <= 1e-10
