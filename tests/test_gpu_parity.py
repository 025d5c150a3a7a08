"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (written from the arithmetic):
  complex128: max |a_gpu - a_oracle| <= 1e-10 (no phase alignment);
  complex64:  infidelity 1 - |<a_oracle|a_gpu>|^2 / (|a_oracle|^2 |a_gpu|^2) <= 1e-5;
  measurement outcomes: bit-exact, except a logged near-tie |u - P0_oracle| < 1e-12
  (c128) / 1e-5 (c64), which the fixed seeds here must not produce.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import workload as W
from paper_2310_17739_gb300.workload import OP
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
qs = pytest.importorskip("paper_2310_17739_gb300.qsim")

C128_TOL = 1e-10
C64_INFID = 1e-5


def run_oracle(c, seed=0, thr=0.0, psi=None):
    psi = oracle.basis_state(c.n) if psi is None else psi.astype(np.complex128).copy()
    r = oracle.run(psi, c.n, c.gates, c.mats, seed=seed, thr=thr)
    return psi, r


def run_gpu(c, dtype, seed=0, config=None, psi=None, use_compile=False):
    sim = qs.Sim(c.n, dtype, config=config or {}, seed=seed)
    if psi is not None:
        sim.set_state(psi)
    if use_compile:
        p = sim.compile(c.gates, c.mats)
        sim.run(p)
        st = sim.sync()
        p.free()
    else:
        sim.apply(c.gates, c.mats)
        st = sim.sync()
    return sim, st


def check_state(dtype, got, ref):
    if dtype == "c128":
        assert np.abs(got.astype(np.complex128) - ref).max() <= C128_TOL
    else:
        assert 1 - H.fidelity(ref, got) <= C64_INFID


def check_outcomes(dtype, g_out, g_prob, r, seed, ordinal0=0):
    """Outcomes bit-exact against the oracle.  A mismatch whose draw
    u(seed, ordinal) lies within `tie` of the oracle's P0 would be a near-tie
    (both sides right within their precision): it is reported as such, and
    the fixed seeds of these tests must produce none; any other mismatch is
    a failure."""
    o_out, o_prob = r.outcomes, r.probs
    assert len(g_out) == len(o_out)
    tie = 1e-12 if dtype == "c128" else 1e-5
    ptol = 1e-10 if dtype == "c128" else 1e-5
    near = []
    for i, (a, b) in enumerate(zip(g_out, o_out)):
        if a != b:
            p0 = o_prob[i] if b == 0 else 1 - o_prob[i]
            u = oracle.draw(seed, ordinal0 + i)
            if b >= 0 and abs(u - p0) < tie:
                near.append((i, u, p0))
                continue
            pytest.fail(f"outcome {i} differs (gpu {a}, oracle {b}, oracle P0 {p0}, draw {u})")
    assert not near, f"near-ties (draw within {tie} of P0) at fixed seeds: {near}"
    assert np.abs(np.asarray(g_prob) - o_prob).max() <= ptol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,tile_bits", [(3, 0), (7, 0), (10, 0), (12, 8), (13, 10), (14, 12)])
def test_random_gate_mix(dtype, n, tile_bits):
    c = W.random_circuit(n, 600, seed=n, with_generic=False)
    ref, _ = run_oracle(c)
    sim, st = run_gpu(c, dtype, config=dict(tile_bits=tile_bits))
    assert st == 0
    check_state(dtype, sim.state(), ref)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_generic_matrices_non_unitary(dtype):
    n = 9
    c = W.random_circuit(n, 60, seed=4)
    ref, _ = run_oracle(c)
    sim, st = run_gpu(c, dtype, config=dict(tile_bits=7))
    got = sim.state().astype(np.complex128)
    scale = np.abs(ref).max()
    tol = 1e-12 if dtype == "c128" else 3e-5
    assert np.abs(got - ref).max() <= tol * scale


@pytest.mark.parametrize("fusion,k_max", [(0, 2), (1, 2), (1, 3), (1, 4), (1, 5), (2, 2), (2, 4)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fusion_levels(dtype, fusion, k_max):
    n = 15
    c = W.ucc_circuit(n, seed=21, n_gadgets=60, w_lo=2, w_hi=6, target_gates=5000)
    ref, _ = run_oracle(c)
    sim, st = run_gpu(c, dtype, config=dict(fusion=fusion, k_max=k_max, tile_bits=11))
    check_state(dtype, sim.state(), ref)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_small_config_state_and_z(dtype):
    """8 qubits, 40 weight 2-4 gadgets cycled to 2,000 gates, |0..0>: state + <Z_i>."""
    c = W.config_small()
    ref, _ = run_oracle(c)
    sim, _ = run_gpu(c, dtype)
    check_state(dtype, sim.state(), ref)
    zt = W.z_terms(8)
    z_ref = oracle.expect(ref, 8, zt)
    z = sim.expect(zt)
    assert np.abs(z - z_ref).max() <= (1e-12 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("tile_bits", [0, 9])
def test_mid_circuit_measurements_bit_exact(dtype, tile_bits):
    n = 14
    c = W.ucc_circuit(n, seed=2, n_gadgets=None, w_lo=2, w_hi=8, theta="normal0.1",
                      target_gates=20000, n_meas=16)
    ref, r = run_oracle(c, seed=1002)
    sim, st = run_gpu(c, dtype, seed=1002, config=dict(tile_bits=tile_bits))
    assert st == 0
    out, prob = sim.outcomes()
    check_outcomes(dtype, out, prob, r, 1002)
    check_state(dtype, sim.state(), ref)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_measure_api_and_reset(dtype):
    n = 12
    c = W.ucc_circuit(n, seed=8, n_gadgets=20, w_lo=2, w_hi=5, target_gates=600)
    ref, _ = run_oracle(c)
    sim, _ = run_gpu(c, dtype)
    for k, q in enumerate([0, 5, 11, 3]):
        st_o, out_o, pr_o = oracle.measure(ref, n, q, seed=77, k=k)
        out, pr, st = sim.measure(q, 77)
        assert st == 0 and out == out_o
        assert abs(pr - pr_o) < (1e-12 if dtype == "c128" else 1e-6)
    check_state(dtype, sim.state(), ref)
    p0, p1 = sim.prob(7)
    r0, r1 = oracle.prob(ref, n, 7)
    assert abs(p0 - r0) < 1e-6 and abs(p1 - r1) < 1e-6


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,tile_bits,fusion", [(10, 0, 1), (16, 12, 1), (16, 12, 2)])
def test_reset_with_outcome_one(dtype, n, tile_bits, fusion):
    """RESET records whose outcome is 1, so the |1> half is moved onto |0>:
    one drawn (the seed is picked on the oracle so that its first draw gives
    1), one forced (qubit reset, flipped by X, reset again: p0 = 0).  Resident
    (n = 10) and tiled (n = 16) paths, both fusion levels."""
    q1, q2 = 2, n - 1
    body = W.ucc_circuit(n, seed=60 + n, n_gadgets=20, w_lo=2, w_hi=5, target_gates=500).gates
    tail = W.records([(OP["RESET"], q1, 0, 0, 0, 0), (OP["H"], 0, 0, 0, 0, 0), (OP["CX"], 0, q1, 0, 0, 0),
                      (OP["RESET"], q2, 0, 0, 0, 0), (OP["X"], q2, 0, 0, 0, 0),
                      (OP["RESET"], q2, 0, 0, 0, 0), (OP["RY"], q2, 0, 0.7, 0, 0)])
    c = W.Circuit(n, np.concatenate([body, tail]))
    seed = None
    for s in range(200):
        ref, r = run_oracle(c, seed=s)
        if r.status == 0 and r.outcomes[0] == 1:
            seed = s
            break
    assert seed is not None
    assert list(r.outcomes[1:]) == [r.outcomes[1], 1]      # the forced reset gives 1
    sim, st = run_gpu(c, dtype, seed=seed, config=dict(tile_bits=tile_bits, fusion=fusion))
    assert st == 0
    out, prob = sim.outcomes()
    check_outcomes(dtype, out, prob, r, seed)
    check_state(dtype, sim.state(), ref)


@pytest.mark.parametrize("tile_bits", [0, 8])
def test_assertion_mode_and_success_product(tile_bits):
    t = H.load_mma_table("tests/golden/mma_table.txt")
    p0s = t["MMA"][:8]
    n = 10
    rows = [(OP["H"], q, 0, 0.0, 0, 0) for q in range(1, n)]
    for p in p0s:
        th = 2 * math.acos(math.sqrt(p))
        rows += [(OP["RY"], 0, 0, th, 0, 0), (OP["MEASURE"], 0, 0, 0, 0, 0, 1),
                 (OP["BARRIER"], 0, 0, 0, 0, 0), (OP["RESET"], 0, 0, 0, 0, 0)]
    c = W.Circuit(n, W.records(rows))
    ref, r = run_oracle(c)
    sim, st = run_gpu(c, "c128", config=dict(tile_bits=tile_bits))
    assert st == 0
    out, prob = sim.outcomes()
    assert np.array_equal(out, r.outcomes)
    succ, st = sim.success_prob()
    assert abs(succ - np.prod(p0s)) < 1e-12
    assert abs(succ - t["MMA"][8]) < 5e-7
    check_state("c128", sim.state(), ref)


@pytest.mark.parametrize("tile_bits", [0, 8])
def test_assertion_failure_keeps_state(tile_bits):
    n = 10
    rows = [(OP["H"], 3, 0, 0, 0, 0), (OP["X"], 0, 0, 0, 0, 0), (OP["MEASURE"], 0, 0, 0, 0, 0, 1),
            (OP["H"], 5, 0, 0, 0, 0)]
    c = W.Circuit(n, W.records(rows))
    sim = qs.Sim(n, "c128", config=dict(tile_bits=tile_bits))
    sim.apply(c.gates)
    assert sim.sync() == qs.E_ZEROPROB
    ref = oracle.basis_state(n)
    r = oracle.run(ref, n, c.gates)
    assert r.status == oracle.E_ZEROPROB
    check_state("c128", sim.state(), ref)
    # the context refuses further work until reset
    sim.apply(W.records([(OP["X"], 1, 0, 0, 0, 0)]))
    assert sim.sync() == qs.E_ZEROPROB
    sim.reset()
    assert sim.sync() == 0
    st0 = sim.state()
    assert st0[0] == 1 and np.count_nonzero(st0) == 1


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation_random_hamiltonian(dtype):
    n = 12
    c = W.ucc_circuit(n, seed=44, n_gadgets=30, w_lo=2, w_hi=6, target_gates=3000)
    ref, _ = run_oracle(c)
    sim, _ = run_gpu(c, dtype)
    terms = W.random_hamiltonian(n, 200, seed=4)
    e_ref = oracle.expect(ref, n, terms)
    e = sim.expect(terms)
    tol = 1e-11 if dtype == "c128" else 2e-5
    assert np.abs(e - e_ref).max() <= tol * max(1.0, np.abs(terms["coef"]).max())


def test_complex64_expectation_sums_keep_small_terms():
    """complex64 expectation terms are formed in FP32 and summed at FP64
    accuracy.  Use a state whose terms are exact in FP32: real dyadic
    amplitudes with 8-bit mantissas, 256 of them near 2^-6 and the rest near
    2^-21.  The sum then matches the FP64 oracle to 1e-11, and it keeps the
    ~2^-41 terms that a plain FP32 running sum would round away beside the
    ~2^-11 ones.  A per-thread FP32 running sum, in the kernel's thread
    layout, misses by 1.2e-10."""
    n = 14
    N = 1 << n
    rng = np.random.default_rng(7)
    mant = rng.integers(128, 256, size=N).astype(np.float64) * rng.choice([-1.0, 1.0], size=N)
    scale = np.full(N, 2.0 ** -28)
    scale[rng.choice(N, 256, replace=False)] = 2.0 ** -13
    psi = (mant * scale).astype(np.complex128)
    terms = W.random_hamiltonian(n, 60, seed=9)
    z_only = np.zeros(n, dtype=W.TERM_DTYPE)
    for q in range(n):
        z_only[q] = (0, 1 << q, 1.0)
    terms = np.concatenate([terms, z_only])
    e_ref = oracle.expect(psi, n, terms)
    sim = qs.Sim(n, "c64")
    sim.set_state(psi.astype(np.complex64))
    e = sim.expect(terms)
    assert np.abs(e - e_ref).max() <= 1e-11 * max(1.0, np.abs(terms["coef"]).max())
    # the small terms matter at this tolerance: dropping them moves <Z_q> by more
    small = np.where(scale < 2.0 ** -20, np.abs(psi) ** 2, 0.0).sum()
    assert small > 1e-9
    sim.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_compile_run_equals_apply_and_repeats(dtype):
    n = 16
    c = W.ucc_circuit(n, seed=3, n_gadgets=50, w_lo=2, w_hi=6, target_gates=8000, n_meas=3)
    sim_a, _ = run_gpu(c, dtype, seed=5)
    sim_b, _ = run_gpu(c, dtype, seed=5, use_compile=True)
    a, b = sim_a.state(), sim_b.state()
    assert np.array_equal(a, b)
    # chunked compile (small chunks) gives the same physics
    ref, r = run_oracle(c, seed=5)
    sim_c, _ = run_gpu(c, dtype, seed=5, config=dict(chunk_gates=1000, compile_threads=3))
    out, prob = sim_c.outcomes()
    check_outcomes(dtype, out, prob, r, 5)
    check_state(dtype, sim_c.state(), ref)


def test_empty_and_edge_inputs():
    sim = qs.Sim(1, "c128")
    sim.apply(W.records([]))
    assert sim.sync() == 0
    sim.apply(W.records([(OP["H"], 0, 0, 0, 0, 0)]))
    s = sim.state()
    assert abs(s[0] - 1 / math.sqrt(2)) < 1e-15 and abs(s[1] - 1 / math.sqrt(2)) < 1e-15
    with pytest.raises(qs.QsimError):
        sim.apply(W.records([(OP["H"], 1, 0, 0, 0, 0)]))
    with pytest.raises(qs.QsimError):
        qs.Sim(35, "c64")
    sim2 = qs.Sim(2, "c64")
    with pytest.raises(qs.QsimError):
        sim2.set_config(tile_bits=20)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,tile_bits", [(9, 0), (16, 10), (16, 13), (21, 13)])
def test_pauli_rotations_with_measurements(dtype, n, tile_bits):
    """Gadget recognition (fusion=2) with mid-circuit measurements, resident and tiled."""
    gates = 3000 if n < 21 else 1500
    c = W.ucc_circuit(n, seed=40 + n, n_gadgets=None, w_lo=2, w_hi=8 if n > 9 else 6,
                      theta="normal0.1", target_gates=gates, n_meas=6)
    ref, r = run_oracle(c, seed=11)
    sim, st = run_gpu(c, dtype, seed=11, config=dict(fusion=2, tile_bits=tile_bits))
    assert st == 0
    out, prob = sim.outcomes()
    check_outcomes(dtype, out, prob, r, 11)
    check_state(dtype, sim.state(), ref)


def test_program_outlives_its_context():
    """Destroying a context releases its programs' device memory; freeing such an
    orphaned program afterwards (in any order) is safe and running it is refused."""
    c = W.ucc_circuit(12, seed=1, n_gadgets=10, w_lo=2, w_hi=4, target_gates=500)
    sims, progs = [], []
    for fusion in (1, 2):
        s = qs.Sim(12, "c64", config=dict(fusion=fusion, tile_bits=9))
        progs.append(s.compile(c.gates))
        sims.append(s)
    sims[0].close()
    progs[0].free()                    # orphan freed after its context
    progs[1].free()                    # normal order
    sims[1].close()
    s = qs.Sim(12, "c64")
    p = s.compile(c.gates)
    other = qs.Sim(12, "c64")
    with pytest.raises(qs.QsimError):
        other.run(p)                   # a program runs only on its own context
    s.close()
    with pytest.raises(qs.QsimError):
        other.run(p)
    del p


# --------------------------------------- rotation passes over subspace tiles --
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("n,tile_bits", [(16, 10), (16, 12), (21, 11), (21, 12), (21, 13), (21, 14)])
def test_rotation_passes_uniform_angles(n, tile_bits, persistent):
    """complex64 register-segment passes (one block per tile, or resident
    blocks taking tiles from a counter) with angles over the whole circle, so
    the Pauli frame splits about half of the rotations; mid-circuit
    measurements flush it."""
    c = W.ucc_circuit(n, seed=70 + n + tile_bits, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform",
                      target_gates=2500, n_meas=5)
    ref, r = run_oracle(c, seed=13)
    sim, st = run_gpu(c, "c64", seed=13, config=dict(fusion=2, tile_bits=tile_bits, persistent=persistent))
    assert st == 0
    out, prob = sim.outcomes()
    check_outcomes("c64", out, prob, r, 13)
    check_state("c64", sim.state(), ref)


@pytest.mark.parametrize("dtype,n,fusion,tile_bits,forced_low,persistent", [
    ("c64", 15, 2, 12, 3, 0), ("c64", 16, 2, 12, 2, 0), ("c64", 16, 2, 13, 3, 0),
    ("c64", 16, 2, 12, 3, 1), ("c64", 15, 2, 13, 2, 1), ("c64", 15, 1, 12, 2, 0),
    ("c128", 15, 2, 12, 2, 0), ("c128", 16, 1, 12, 2, 0), ("c128", 15, 2, 11, 1, 0)])
def test_fewer_forced_low_qubits(dtype, n, fusion, tile_bits, forced_low, persistent):
    """Tiles with fewer forced low qubits than the default (4 for complex64, 3
    for complex128): shorter contiguous tile rows in the generic pass and the
    register pass, and (persistent = 1) the fallback from resident-block
    passes, which need 4, to one block per tile.  Amplitudes and outcomes
    against the oracle."""
    c = W.ucc_circuit(n, seed=90 + n + forced_low, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform",
                      target_gates=2500, n_meas=4)
    ref, r = run_oracle(c, seed=17)
    cfg = dict(fusion=fusion, tile_bits=tile_bits, forced_low=forced_low, persistent=persistent)
    sim, st = run_gpu(c, dtype, seed=17, config=cfg)
    assert st == 0
    out, prob = sim.outcomes()
    check_outcomes(dtype, out, prob, r, 17)
    check_state(dtype, sim.state(), ref)
    # the same program compiled once and replayed (graph launches on the second run)
    sim2 = qs.Sim(n, dtype, config=cfg, seed=17)
    prog = sim2.compile(c.gates)
    for _ in range(2):
        sim2.reset()
        sim2.run(prog)
        assert sim2.sync() == 0
    check_state(dtype, sim2.state(), ref)
    prog.free()


def test_persistent_passes_replay_and_recover_after_a_failed_assertion():
    """A compiled program replayed several times keeps the tile counter in step;
    a failed assertion makes later persistent passes leave the state alone
    (while still consuming their tile numbers), and after a reset the same
    program runs correctly again."""
    n = 18
    c = W.ucc_circuit(n, seed=5, n_gadgets=200, w_lo=2, w_hi=6, theta="uniform", target_gates=3000)
    cfg = dict(fusion=2, tile_bits=12, persistent=1)
    sim = qs.Sim(n, "c64", config=cfg)
    prog = sim.compile(c.gates)
    ref = oracle.basis_state(n)
    for rep in range(3):
        sim.run(prog)
        assert sim.sync() == 0
        oracle.run(ref, n, c.gates)
        check_state("c64", sim.state(), ref)
    # an assertion that fails: qubit 0 reset, flipped to |1>, then asserted to be |0>
    bad = W.records([(OP["RESET"], 0, 0, 0, 0, 0), (OP["X"], 0, 0, 0, 0, 0),
                     (OP["MEASURE"], 0, 0, 0, 0, 0, 1)])
    sim.apply(bad)
    assert sim.sync() == qs.E_ZEROPROB
    frozen = sim.state()
    sim.run(prog)                      # refused by every pass: the state stays
    assert sim.sync() == qs.E_ZEROPROB
    assert np.array_equal(sim.state(), frozen)
    sim.reset()
    sim.run(prog)
    assert sim.sync() == 0
    ref = oracle.basis_state(n)
    oracle.run(ref, n, c.gates)
    check_state("c64", sim.state(), ref)
    prog.free()


def test_long_run_of_one_rotation_falls_back_to_the_generic_pass():
    """300 repeats of one Pauli rotation whose X mask touches qubit 0 fill a
    register-segment pass beyond its op limit; that pass runs in the generic
    kernel over the row-reduced basis and still matches the oracle."""
    n = 16
    rows = []
    for r in range(300):
        rows += W.gadget_rows([0, 5, 9], "XZY", 0.01 * (r % 17) - 0.08)
    g = W.records([(op, q0, q1, p, 0, 0) for op, q0, q1, p in rows])
    c = W.Circuit(n, np.concatenate([W.ucc_circuit(n, seed=8, n_gadgets=20, w_lo=2, w_hi=5,
                                                   target_gates=400).gates, g]))
    ref, _ = run_oracle(c)
    sim, st = run_gpu(c, "c64", config=dict(fusion=2, tile_bits=12))
    assert st == 0
    check_state("c64", sim.state(), ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_scaled_rotations_stop_before_the_product_of_cosines_underflows(dtype):
    """300 repeats of one Pauli rotation at angles near pi/4 (cos ~ 0.71, so the
    product of 300 cosines is ~1e-45) in one pass: the scaled form a + (W/cos)(...)
    is used only while the product stays >= 2^-40 (the unscaled amplitudes stay
    below 2^40), the rest of the pass runs unscaled; the state must match the
    oracle.  Register and generic tile kernels (complex64), generic (complex128)."""
    n = 16
    rows = []
    for r in range(300):
        rows += W.gadget_rows([1, 6, 11], "XZY", (0.785 if r % 2 else -0.7) + 0.001 * (r % 7))
    g = W.records([(op, q0, q1, p, 0, 0) for op, q0, q1, p in rows])
    c = W.Circuit(n, np.concatenate([W.ucc_circuit(n, seed=9, n_gadgets=20, w_lo=2, w_hi=5,
                                                   target_gates=400).gates, g]))
    ref, _ = run_oracle(c)
    for tb in (12, 10):
        sim, st = run_gpu(c, dtype, config=dict(fusion=2, tile_bits=tb))
        assert st == 0
        got = sim.state()
        assert np.all(np.isfinite(got))
        check_state(dtype, got, ref)
        sim.close()


def test_profile_windows_count_launches_and_bytes():
    """Launch timing windows: every tile-pass launch inside a window is counted
    once with one read and one write of the state; windows close at
    measurements; the sampled time per launch is positive and the whole run's
    launches are counted."""
    n = 18
    c = W.ucc_circuit(n, seed=31, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=6000, n_meas=3)
    sim = qs.Sim(n, "c64", config=dict(fusion=2, tile_bits=12))
    sim.profile_start(4)
    sim.apply(c.gates)
    assert sim.sync() == 0
    prof = sim.profile_read()
    prog = sim.compile(c.gates)
    passes = prog.info()["passes"]          # tile passes (measurements are not counted)
    prog.free()
    assert prof["launches"] == passes
    assert 0 < prof["samples"] <= prof["launches"]
    assert prof["bytes"] == prof["samples"] * 2 * 8 * (1 << n)
    assert prof["ms"] > 0
    sim.profile_start(0)
