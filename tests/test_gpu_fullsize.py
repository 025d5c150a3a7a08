"""Full-size checks in the benchmark's launch configuration: the 16-qubit
1e6-gate circuit against the whole oracle run; where the oracle cannot run the
whole circuit (21 qubits, 1.15e8 gates), the two precisions against each
other and properties that hold at any size; states above L2 size (24 qubits,
oracle parity) and above 2^32 amplitudes (33 qubits, closed forms)."""
import threading

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


def test_large_circuit_with_its_measurements_in_both_precisions():
    """The benchmark's 21-qubit circuit of 1.15e8 gates with its 8 mid-circuit
    measurements, complex64 in the benchmark's configuration and complex128
    (the paper's arithmetic): the same 8 outcomes and final states within
    infidelity 1e-5 (no oracle can run this circuit; the complex128 run is the
    reference the complex64 result is stated against)."""
    c = W.config_large(n_meas=8)
    runs = {}
    for dt, cfg in (("c64", BENCH_CFG), ("c128", dict(fusion=2))):
        sim = qs.Sim(21, dt, seed=1003, config=cfg)
        sim.apply(c.gates)
        assert sim.sync() == 0
        runs[dt] = (sim.state(), sim.outcomes())
        sim.close()
    (s64, (o64, p64)), (s128, (o128, p128)) = runs["c64"], runs["c128"]
    assert len(o128) == 8 and np.array_equal(o64, o128)
    assert np.abs(p64 - p128).max() <= 1e-5
    assert abs(float(np.vdot(s128, s128).real) - 1.0) <= 1e-9
    assert 1 - H.fidelity(s128, s64) <= 1e-5


def test_mid_config_against_the_whole_oracle_run():
    """16 qubits, 1e6 gates, 64 mid-circuit measurements (draws philox(1002, k)):
    the oracle runs the whole circuit (in a thread: the C call releases the
    interpreter lock) while the GPU runs it in complex128 and complex64.
    Outcomes bit-exact, complex128 amplitudes within 1e-10, complex64 within
    infidelity 1e-5."""
    c = W.config_mid()
    ref = oracle.basis_state(16)
    box = {}
    th = threading.Thread(target=lambda: box.update(r=oracle.run(ref, 16, c.gates, seed=1002)))
    th.start()
    runs = {}
    for dt in ("c128", "c64"):
        sim = qs.Sim(16, dt, seed=1002, config=dict(fusion=2))
        sim.apply(c.gates)
        assert sim.sync() == 0
        runs[dt] = (sim.state(), sim.outcomes())
        sim.close()
    th.join()
    r = box["r"]
    assert r.status == 0 and len(r.outcomes) == 64
    (s128, (o128, p128)), (s64, (o64, p64)) = runs["c128"], runs["c64"]
    assert np.array_equal(o128, r.outcomes) and np.array_equal(o64, r.outcomes)
    assert np.abs(p128 - r.probs).max() <= 1e-10
    assert np.abs(s128 - ref).max() <= 1e-10
    assert 1 - H.fidelity(ref, s64) <= 1e-5


@pytest.mark.parametrize("dtype,cfg", [("c64", BENCH_CFG), ("c64", dict(fusion=1)), ("c128", dict(fusion=2))])
def test_state_above_l2_size_against_the_oracle(dtype, cfg):
    """24 qubits (128 MiB complex64, 256 MiB complex128: larger than the 126 MB
    L2, so every pass streams the state from HBM) on a short circuit with 3
    measurements: outcomes and amplitudes against the oracle."""
    n = 24
    c = W.ucc_circuit(n, seed=24, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=400, n_meas=3)
    ref = oracle.basis_state(n)
    r = oracle.run(ref, n, c.gates, seed=9)
    sim = qs.Sim(n, dtype, seed=9, config=cfg)
    sim.apply(c.gates)
    assert sim.sync() == 0
    out, prob = sim.outcomes()
    assert np.array_equal(out, r.outcomes)
    got = sim.state()
    if dtype == "c128":
        assert np.abs(got - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, got) <= 1e-5
    sim.close()


def test_more_than_2_32_amplitudes_ghz_closed_form():
    """33 qubits, complex64 (64 GiB): the GHZ circuit H(0), CX(0,1), ...,
    CX(31,32) gives (|0...0> + |1...1>)/sqrt(2), so every qubit has P(0) = 1/2,
    <Z_0 Z_32> = 1 and <X...X> (all 33 qubits) = 1; a measurement of qubit 32
    then leaves the basis state of its outcome on every qubit.  Checks 64-bit
    amplitude indexing in the tile, reduction, expectation and collapse
    kernels without reading the state back."""
    n = 33
    if torch.cuda.mem_get_info()[0] < (72 << 30):
        pytest.skip("needs 72 GiB of free device memory")
    sim = qs.Sim(n, "c64", seed=4, config=dict(fusion=1))
    sim.apply(W.ghz_circuit(n).gates)
    assert sim.sync() == 0
    for q in (0, 17, 32):
        p0, p1 = sim.prob(q)
        assert abs(p0 - 0.5) < 1e-6 and abs(p1 - 0.5) < 1e-6
    terms = np.zeros(2, dtype=W.TERM_DTYPE)
    terms[0] = (0, (1 << 0) | (1 << 32), 1.0)
    terms[1] = ((1 << n) - 1, 0, 1.0)
    e = sim.expect(terms)
    assert abs(e[0] - 1) < 1e-5 and abs(e[1] - 1) < 1e-5
    out, pr, st = sim.measure(32, 77)
    assert st == 0 and abs(pr - 0.5) < 1e-6
    assert out == (0 if oracle.draw(77, 0) < 0.5 else 1)   # the draw is far from 1/2
    for q in (0, 16, 31):
        p0, p1 = sim.prob(q)
        assert (p0, p1) == ((1.0, 0.0) if out == 0 else (0.0, 1.0))
    sim.close()
