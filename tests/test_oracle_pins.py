"""Pins for the CPU oracle against things other than itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a swapped operand, an off-by-one in Eq. (1q-op)/(2q-op), a wrong
Philox constant) fails at least one of them:
  * gate table vs scipy.linalg.expm and textbook identities,
  * every gate on every qubit / ordered qubit pair vs a brute-force 2^n matrix,
  * GHZ and QFT-of-basis-state closed forms,
  * compiled Pauli gadgets vs exp(-i t P) = cos t I - i sin t P,
  * norm and U-then-U^dagger invariants,
  * Born probabilities, collapse, reset and the chi^2 statistics of the draw,
  * the probability-product reading of the paper's assertion table,
  * numpy.random.Philox for the counter-based draw,
  * Pauli expectations vs dense matrices and vs <Z> = p0 - p1.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from paper_2310_17739_gb300 import workload as W
from paper_2310_17739_gb300.workload import OP
from tests import helpers as H

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def one(op, q0=0, q1=1, p=(0.0, 0.0, 0.0)):
    return W.records([(op, q0, q1, p[0], p[1], p[2])])[0]


def expm(a):
    return scipy.linalg.expm(a)


def _np_draw(seed, k):
    """u(seed, k) from numpy.random.Philox alone (the block at counter k is
    numpy's first block when started at counter k - 1)."""
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=(k - 1) % (1 << 256))
    return (int(bg.random_raw(1)[0]) >> 11) * 2.0**-53


# ------------------------------------------------------------ gate table ----
@pytest.mark.parametrize("theta", [0.0, 0.3, -1.7, 2.9])
def test_rotations_match_expm(theta):
    assert np.allclose(oracle.gate_matrix(one(OP["RX"], p=(theta, 0, 0))), expm(-0.5j * theta * H.PX), atol=1e-15)
    assert np.allclose(oracle.gate_matrix(one(OP["RY"], p=(theta, 0, 0))), expm(-0.5j * theta * H.PY), atol=1e-15)
    assert np.allclose(oracle.gate_matrix(one(OP["RZ"], p=(theta, 0, 0))), expm(-0.5j * theta * H.PZ), atol=1e-15)
    XX = np.kron(H.PX, H.PX)
    ZZ = np.kron(H.PZ, H.PZ)
    assert np.allclose(oracle.gate_matrix(one(OP["RXX"], p=(theta, 0, 0))), expm(-0.5j * theta * XX), atol=1e-15)
    assert np.allclose(oracle.gate_matrix(one(OP["RZZ"], p=(theta, 0, 0))), expm(-0.5j * theta * ZZ), atol=1e-15)
    assert np.allclose(oracle.gate_matrix(one(OP["U1"], p=(theta, 0, 0))), np.diag([1, np.exp(1j * theta)]), atol=1e-15)


def test_fixed_gates_identities():
    g = lambda name: oracle.gate_matrix(one(OP[name]))
    assert np.allclose(g("X"), H.PX) and np.allclose(g("Y"), H.PY) and np.allclose(g("Z"), H.PZ)
    assert np.allclose(g("ID"), np.eye(2))
    assert np.allclose(g("H"), (H.PX + H.PZ) / math.sqrt(2), atol=1e-15)
    assert np.allclose(g("S") @ g("S"), H.PZ, atol=1e-15)
    assert np.allclose(g("T") @ g("T"), g("S"), atol=1e-15)
    assert np.allclose(g("SDG"), g("S").conj().T) and np.allclose(g("TDG"), g("T").conj().T)
    assert np.allclose(1j * H.PX @ H.PZ, H.PY)


@pytest.mark.parametrize("seed", range(5))
def test_u3_u2_decompositions(seed):
    rng = np.random.default_rng(seed)
    th, ph, la = rng.uniform(-np.pi, np.pi, size=3)
    u3 = oracle.gate_matrix(one(OP["U3"], p=(th, ph, la)))
    rz = lambda a: expm(-0.5j * a * H.PZ)
    ry = lambda a: expm(-0.5j * a * H.PY)
    # U3(t, p, l) = e^{i(p+l)/2} RZ(p) RY(t) RZ(l)
    assert np.allclose(u3, np.exp(0.5j * (ph + la)) * rz(ph) @ ry(th) @ rz(la), atol=1e-14)
    u2 = oracle.gate_matrix(one(OP["U2"], p=(ph, la, 0.0)))
    assert np.allclose(u2, np.exp(0.5j * (ph + la)) * rz(ph) @ ry(np.pi / 2) @ rz(la), atol=1e-14)


def controlled_local(u):
    """|0><0| on b0 (control, q0) (x) I  +  |1><1| (x) U on b1 (target, q1), in
    the local basis l = b0 + 2 b1, i.e. kron(target_op, control_projector)."""
    P0 = np.diag([1, 0]).astype(np.complex128)
    P1 = np.diag([0, 1]).astype(np.complex128)
    return np.kron(np.eye(2), P0) + np.kron(u, P1)


@pytest.mark.parametrize("seed", range(3))
def test_two_qubit_table(seed):
    rng = np.random.default_rng(seed)
    t, ph, la = rng.uniform(-np.pi, np.pi, size=3)
    g2 = lambda name, p=(0, 0, 0): oracle.gate_matrix(one(OP[name], p=p))
    g1 = lambda name, p=(0, 0, 0): oracle.gate_matrix(one(OP[name], p=p))
    for c2, c1 in [("CX", "X"), ("CY", "Y"), ("CZ", "Z"), ("CH", "H")]:
        assert np.allclose(g2(c2), controlled_local(g1(c1)), atol=1e-15), c2
    for c2, c1 in [("CRX", "RX"), ("CRY", "RY"), ("CRZ", "RZ"), ("CU1", "U1")]:
        assert np.allclose(g2(c2, (t, 0, 0)), controlled_local(g1(c1, (t, 0, 0))), atol=1e-15), c2
    assert np.allclose(g2("CU3", (t, ph, la)), controlled_local(g1("U3", (t, ph, la))), atol=1e-15)
    swap = np.zeros((4, 4))
    for b0 in range(2):
        for b1 in range(2):
            swap[b1 + 2 * b0, b0 + 2 * b1] = 1
    assert np.allclose(g2("SWAP"), swap)


# ------------------------------------------------ Eq. (1q-op) / (2q-op) ----
@pytest.mark.parametrize("n", [1, 3, 5])
def test_every_1q_gate_every_qubit_vs_kronecker(n):
    rng = np.random.default_rng(10 + n)
    ops = W.ONE_QUBIT + [OP["C1"]]
    for q in range(n):
        for op in ops:
            p = rng.uniform(-np.pi, np.pi, size=3)
            mats = (rng.normal(size=8)).astype(np.float64)
            rec = W.records([(op, q, 0, *p)])
            psi = W.random_state(n, seed=int(rng.integers(1 << 30)))
            ref = H.full_1q(n, q, oracle.gate_matrix(rec[0], mats)) @ psi
            r = oracle.run(psi, n, rec, mats)
            assert r.status == 0
            assert np.abs(psi - ref).max() < 1e-14, (op, q)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_every_2q_gate_every_ordered_pair_vs_kronecker(n):
    rng = np.random.default_rng(20 + n)
    ops = W.TWO_QUBIT + [OP["C2"]]
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    for (a, b) in pairs:
        for op in ops if n < 6 else [OP["C2"], OP["CX"], OP["CU3"]]:
            p = rng.uniform(-np.pi, np.pi, size=3)
            mats = rng.normal(size=32)
            rec = W.records([(op, a, b, *p)])
            psi = W.random_state(n, seed=int(rng.integers(1 << 30)))
            ref = H.full_2q(n, a, b, oracle.gate_matrix(rec[0], mats)) @ psi
            r = oracle.run(psi, n, rec, mats)
            assert r.status == 0
            assert np.abs(psi - ref).max() < 1e-14, (op, a, b)


def test_cx_acts_by_definition():
    # CX(c, t) flips bit t exactly where bit c is 1 -- on every basis state.
    n = 4
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            for j in range(1 << n):
                psi = oracle.basis_state(n, j)
                oracle.run(psi, n, W.records([(OP["CX"], c, t, 0, 0, 0)]))
                expect = j ^ (1 << t) if (j >> c) & 1 else j
                assert psi[expect] == 1.0 and np.count_nonzero(psi) == 1


# ------------------------------------------------------------ closed forms ----
@pytest.mark.parametrize("n", [2, 5, 10])
def test_ghz_closed_form(n):
    c = W.ghz_circuit(n)
    psi = oracle.basis_state(n)
    oracle.run(psi, n, c.gates)
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.abs(psi - ref).max() < 1e-15


@pytest.mark.parametrize("n,j", [(3, 5), (6, 0), (6, 37), (8, 201)])
def test_qft_of_basis_state_closed_form(n, j):
    c = W.qft_circuit(n, prep_index=j)
    psi = oracle.basis_state(n)
    oracle.run(psi, n, c.gates)
    N = 1 << n
    ref = np.exp(2j * np.pi * j * np.arange(N) / N) / math.sqrt(N)
    assert np.abs(psi - ref).max() < 1e-13


@pytest.mark.parametrize("seed", range(8))
def test_compiled_gadget_is_exp_minus_i_theta_p(seed):
    rng = np.random.default_rng(seed)
    n = 6
    support, letters = W.random_pauli(rng, n, 1, n)
    theta = float(rng.uniform(-np.pi, np.pi))
    psi = W.random_state(n, seed=seed + 100)
    P = H.pauli_dense(n, dict(zip(support, letters)))
    ref = (math.cos(theta) * np.eye(1 << n) - 1j * math.sin(theta) * P) @ psi
    oracle.run(psi, n, W.gadget(support, letters, theta))
    assert np.abs(psi - ref).max() < 1e-13, (support, letters)


# -------------------------------------------------------------- invariants ----
def test_norm_and_inverse_circuit():
    n = 7
    c = W.ucc_circuit(n, seed=5, n_gadgets=50, w_lo=2, w_hi=5, target_gates=3000)
    psi0 = W.random_state(n, seed=7)
    psi = psi0.copy()
    oracle.run(psi, n, c.gates)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    inv = W.from_columns(*zip(*H.inverse_rows(H.rows_of(c.gates))))
    oracle.run(psi, n, inv)
    assert np.abs(psi - psi0).max() < 1e-12


def test_random_gate_mix_unitarity():
    n = 5
    c = W.random_circuit(n, 400, seed=3, with_generic=False)
    psi = W.random_state(n, seed=1)
    oracle.run(psi, n, c.gates)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_invalid_records_rejected():
    n = 3
    psi = oracle.basis_state(n)
    assert oracle.run(psi, n, W.records([(OP["H"], 3, 0, 0, 0, 0)])).status == oracle.E_INVAL
    assert oracle.run(psi, n, W.records([(OP["CX"], 1, 1, 0, 0, 0)])).status == oracle.E_INVAL
    assert oracle.run(psi, n, W.records([(99, 0, 0, 0, 0, 0)])).status == oracle.E_INVAL
    assert np.array_equal(psi, oracle.basis_state(n))


# ------------------------------------------------------------------ Philox ----
@pytest.mark.parametrize("seed,k", [(0, 0), (1, 0), (5, 3), (1002, 63), (2**63 + 7, 2**40 + 1),
                                    (123456789, 2**64 - 1)])
def test_philox_matches_numpy(seed, k):
    # numpy advances its counter before producing a block, so the block at
    # counter k is numpy's first block when started at counter k-1 (mod 2^256).
    # (The key goes in as a uint64 array: a Python list of big ints loses bits.)
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=(k - 1) % (1 << 256))
    ref = bg.random_raw(4)
    assert np.array_equal(oracle.philox_block([k, 0, 0, 0], [seed, 0]), ref)
    u_ref = (int(ref[0]) >> 11) * 2.0**-53
    assert oracle.draw(seed, k) == u_ref


def test_philox_counter_carry_matches_numpy():
    ctr = [2**64 - 1, 5, 0, 0]
    c_int = ctr[0] + (ctr[1] << 64)
    bg = np.random.Philox(key=np.array([9, 11], dtype=np.uint64), counter=c_int - 1)
    assert np.array_equal(oracle.philox_block(ctr, [9, 11]), bg.random_raw(4))


# ------------------------------------------------------------- measurement ----
def test_probabilities_collapse_and_norm():
    n = 6
    rng = np.random.default_rng(0)
    for q in range(n):
        psi = W.random_state(n, seed=int(rng.integers(1 << 30)))
        bits = (np.arange(1 << n) >> q) & 1
        w = np.abs(psi) ** 2
        p0, p1 = oracle.prob(psi, n, q)
        assert abs(p0 - w[bits == 0].sum()) < 1e-15 and abs(p1 - w[bits == 1].sum()) < 1e-15
        before = psi.copy()
        st, out, pr = oracle.measure(psi, n, q, seed=77, k=q)
        u = oracle.draw(77, q)
        assert st == 0 and out == (0 if u < p0 / (p0 + p1) else 1)
        assert abs(pr - (p0 if out == 0 else p1)) < 1e-15
        assert np.all(psi[bits != out] == 0)
        assert abs(np.linalg.norm(psi) - 1) < 1e-14
        kept = before[bits == out] / math.sqrt(p0 if out == 0 else p1)
        assert np.abs(psi[bits == out] - kept).max() < 1e-15


def test_outcome_rule_edges():
    n = 2
    psi = oracle.basis_state(n, 0b10)          # qubit 1 is surely 1: p0 = 0
    st, out, pr = oracle.measure(psi, n, 1, seed=0, k=0)
    assert (st, out, pr) == (0, 1, 1.0)
    psi = oracle.basis_state(n, 0b00)          # p1 = 0: always 0, for any draw
    for k in range(50):
        st, out, pr = oracle.measure(psi, n, 0, seed=3, k=k)
        assert (st, out, pr) == (0, 0, 1.0)


def test_assertion_mode_zero_probability_leaves_state():
    n = 3
    psi = oracle.basis_state(n, 0b001)
    before = psi.copy()
    st, out, pr = oracle.measure(psi, n, 0, seed=0, k=0, mode=W.MEAS_ASSERT)
    assert st == oracle.E_ZEROPROB and pr == 0.0
    assert np.array_equal(psi, before)
    r = oracle.run(psi, n, W.records([(OP["H"], 1, 0, 0, 0, 0), (OP["MEASURE"], 0, 0, 0, 0, 0, 1),
                                      (OP["H"], 2, 0, 0, 0, 0)]))
    assert r.status == oracle.E_ZEROPROB and r.ordinal == 0
    # processing stopped at the failed assertion: the H on qubit 2 never ran
    assert abs(psi[0b011] - 1 / math.sqrt(2)) < 1e-15 and np.count_nonzero(psi) == 2


def test_reset_moves_one_half():
    n = 3
    psi = W.random_state(n, seed=4)
    st, out, pr = oracle.reset(psi, n, 1, seed=8, k=0)
    bits = (np.arange(1 << n) >> 1) & 1
    assert st == 0 and np.all(psi[bits == 1] == 0)
    assert abs(np.linalg.norm(psi) - 1) < 1e-14


def _reset_one_expected(before, n, q):
    """RESET with outcome 1, written out with numpy: amplitude i (bit q set)
    lands on i with bit q cleared, scaled by 1/sqrt(p1) with p1 the raw (not
    normalised) weight of the |1> half; the |1> half becomes zero."""
    idx = np.arange(1 << n)
    one = ((idx >> q) & 1) == 1
    p1 = float(np.sum(np.abs(before[one]) ** 2))
    want = np.zeros_like(before)
    want[idx[one] & ~(1 << q)] = before[one] / math.sqrt(p1)
    return want


@pytest.mark.parametrize("q", [0, 1, 3])
def test_reset_outcome_one_forced_by_zero_p0(q):
    """p0 = 0 on qubit q makes the draw give 1 for every u in [0, 1) (strict
    u < P0), so the move branch must run.  The state is left unnormalised
    (norm^2 = 0.37) so that a missing or wrong 1/sqrt(p1) scale shows."""
    n = 4
    psi = W.random_state(n, seed=40 + q)
    one = ((np.arange(1 << n) >> q) & 1) == 1
    psi[~one] = 0
    psi *= math.sqrt(0.37) / np.linalg.norm(psi)
    before = psi.copy()
    st, out, pr = oracle.reset(psi, n, q, seed=8, k=3)
    assert (st, out) == (0, 1) and abs(pr - 1.0) < 1e-15
    want = _reset_one_expected(before, n, q)
    assert np.allclose(psi, want, rtol=1e-14, atol=1e-17)
    assert np.all(psi[one] == 0)
    assert abs(np.linalg.norm(psi) - 1) < 1e-14


def test_reset_outcome_one_drawn_on_a_generic_state():
    """Both halves populated; the (seed, k) pair is chosen with numpy's Philox
    (independent of the oracle's) so that u >= P0, i.e. the draw gives 1."""
    n, q = 5, 2
    psi = W.random_state(n, seed=9)
    psi *= math.sqrt(0.61) / np.linalg.norm(psi)
    one = ((np.arange(1 << n) >> q) & 1) == 1
    P0 = float(np.sum(np.abs(psi[~one]) ** 2) / np.sum(np.abs(psi) ** 2))
    seed = 21
    k = next(k for k in range(1000) if _np_draw(seed, k) >= P0 + 1e-9)
    before = psi.copy()
    st, out, pr = oracle.reset(psi, n, q, seed=seed, k=k)
    assert (st, out) == (0, 1)
    assert abs(pr - (1 - P0)) < 1e-14
    want = _reset_one_expected(before, n, q)
    assert np.allclose(psi, want, rtol=1e-14, atol=1e-17)
    assert np.all(psi[one] == 0)
    # and a (seed, k) pair whose draw gives 0 leaves the kept half in place
    k0 = next(k for k in range(1000) if _np_draw(seed, k) < P0 - 1e-9)
    psi0 = before.copy()
    st, out, pr = oracle.reset(psi0, n, q, seed=seed, k=k0)
    assert (st, out) == (0, 0)
    p0 = float(np.sum(np.abs(before[~one]) ** 2))
    assert np.allclose(psi0[~one], before[~one] / math.sqrt(p0), rtol=1e-14, atol=1e-17)
    assert np.all(psi0[one] == 0)


def test_born_statistics_chi2():
    n = 2
    theta = 1.1
    p0_true = math.cos(theta / 2) ** 2
    counts = [0, 0]
    trials = 10000
    for k in range(trials):
        psi = oracle.basis_state(n)
        r = oracle.run(psi, n, W.records([(OP["RY"], 0, 0, theta, 0, 0), (OP["H"], 1, 0, 0, 0, 0),
                                          (OP["MEASURE"], 0, 0, 0, 0, 0)]), seed=2024, ordinal=k)
        counts[int(r.outcomes[0])] += 1
    exp = [trials * p0_true, trials * (1 - p0_true)]
    chi2 = sum((c - e) ** 2 / e for c, e in zip(counts, exp))
    assert scipy.stats.chi2.sf(chi2, df=1) > 1e-3, (counts, exp)


# ------------------------------------ the paper's assertion table (Table mma) ----
def test_mma_table_success_is_product_of_p0():
    t = H.load_mma_table("tests/golden/mma_table.txt")
    p0 = t["MMA"][:8]
    assert abs(np.prod(p0) - t["MMA"][8]) < 5e-7   # printed to 6 decimals
    # Each case's rows account for all 1024 shots.
    for case in ("Case-1", "Case-2", "Case-3"):
        assert sum(t[case][:9]) == 1024


def test_mma_rejections_consistent_with_p0():
    """The expected rejections at M_k are (survivors before M_k) * (1 - P0_k);
    the three printed cases must be consistent with it (chi^2 over M1..M8 and success)."""
    t = H.load_mma_table("tests/golden/mma_table.txt")
    p0 = np.array(t["MMA"][:8])
    surv = 1024 * np.concatenate([[1.0], np.cumprod(p0)])
    exp = np.concatenate([surv[:-1] * (1 - p0), [surv[-1]]])
    for case in ("Case-1", "Case-2", "Case-3"):
        obs = np.array(t[case][:9])
        chi2 = float(((obs - exp) ** 2 / exp).sum())
        assert scipy.stats.chi2.sf(chi2, df=8) > 1e-3, (case, chi2)


def ancilla_filter_circuit(p0s, mode, extra_qubits=2):
    """Ancilla q0 rotated so that P(0) = p0_k before the k-th measurement, with a
    reset after each one; spectator qubits in superposition."""
    rows = [(OP["H"], q, 0, 0.0, 0, 0) for q in range(1, 1 + extra_qubits)]
    for p in p0s:
        theta = 2 * math.acos(math.sqrt(p))
        rows += [(OP["RY"], 0, 0, theta, 0, 0), (OP["MEASURE"], 0, 0, 0, 0, 0, mode),
                 (OP["BARRIER"], 0, 0, 0, 0, 0), (OP["RESET"], 0, 0, 0, 0, 0),
                 (OP["BARRIER"], 0, 0, 0, 0, 0)]
    return W.records(rows)


def test_assertion_mode_tracks_table_probabilities():
    t = H.load_mma_table("tests/golden/mma_table.txt")
    p0 = t["MMA"][:8]
    n = 3
    psi = oracle.basis_state(n)
    r = oracle.run(psi, n, ancilla_filter_circuit(p0, W.MEAS_ASSERT))
    assert r.status == 0
    meas = r.probs[0::2]                    # MEASURE records; RESET records interleave
    assert np.allclose(meas, p0, atol=1e-14)
    assert np.all(r.outcomes == 0)
    assert abs(np.prod(meas) - t["MMA"][8]) < 5e-7


def test_sequential_shots_reproduce_table_statistics():
    """Plain draws, 1024 shots each run to the first rejection: the rejection
    counts follow the same law as the table's three cases."""
    t = H.load_mma_table("tests/golden/mma_table.txt")
    p0 = t["MMA"][:8]
    n = 1
    circ = ancilla_filter_circuit(p0, 0, extra_qubits=0)
    rej = np.zeros(9)
    for shot in range(1024):
        psi = oracle.basis_state(n)
        r = oracle.run(psi, n, circ, seed=4242, ordinal=shot * 16)
        m = r.outcomes[0::2]
        first = np.flatnonzero(m == 1)
        rej[first[0] if first.size else 8] += 1
    surv = 1024 * np.concatenate([[1.0], np.cumprod(p0)])
    exp = np.concatenate([surv[:-1] * (1 - np.array(p0)), [surv[-1]]])
    chi2 = float(((rej - exp) ** 2 / exp).sum())
    assert scipy.stats.chi2.sf(chi2, df=8) > 1e-3, (rej, exp)


# -------------------------------------------------------------- expectation ----
@pytest.mark.parametrize("n", [1, 4, 6])
def test_expectation_vs_dense(n):
    terms = W.random_hamiltonian(n, 30, seed=n)
    psi = W.random_state(n, seed=n + 50)
    got = oracle.expect(psi, n, terms)
    for t, g in zip(terms, got):
        P = H.term_dense(n, int(t["x"]), int(t["z"]))
        ref = t["coef"] * np.vdot(psi, P @ psi)
        assert abs(ref.imag) < 1e-13
        assert abs(g - ref.real) < 1e-13


def test_z_expectation_is_p0_minus_p1():
    n = 8
    c = W.config_small()
    psi = oracle.basis_state(n)
    oracle.run(psi, n, c.gates)
    z = oracle.expect(psi, n, W.z_terms(n))
    for q in range(n):
        p0, p1 = oracle.prob(psi, n, q)
        assert abs(z[q] - (p0 - p1)) < 1e-13


# ------------------------------------------------------- final-state shots ----
@pytest.mark.parametrize("seed,s", [(0, 0), (7, 1), (1003, 999), (2**63 + 1, 2**33)])
def test_shot_draw_matches_numpy(seed, s):
    """Shot s draws from the Philox block at counter (s, 1, 0, 0)."""
    c_int = s + (1 << 64)
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=c_int - 1)
    ref = bg.random_raw(4)
    assert oracle.shot_draw(seed, s) == (int(ref[0]) >> 11) * 2.0**-53


def test_sample_is_the_inverse_cumulative_distribution():
    """Every shot is numpy.searchsorted of its draw on the cumulative Born
    distribution (the smallest index whose cumulative probability exceeds
    draw * total), with the masked bits packed in ascending order."""
    n = 9
    psi = W.random_state(n, seed=21)
    psi[::3] = 0                      # zero-probability indices must never be drawn
    cum = np.cumsum(np.abs(psi) ** 2)
    shots = oracle.sample(psi, n, 3000, seed=17)
    u = np.array([oracle.shot_draw(17, s) for s in range(3000)])
    x = np.searchsorted(cum, u * cum[-1], side="right")
    assert np.array_equal(shots, x)
    assert not np.any(shots % 3 == 0)
    mask = 0b101010010
    packed = oracle.sample(psi, n, 3000, seed=17, mask=mask)
    bits = [b for b in range(n) if (mask >> b) & 1]
    ref = sum(((x >> b) & 1) << j for j, b in enumerate(bits))
    assert np.array_equal(packed, ref)


def test_sample_born_statistics_and_special_states():
    n = 4
    psi = W.random_state(n, seed=5)
    p = np.abs(psi) ** 2
    shots = oracle.sample(psi, n, 40000, seed=3)
    counts = np.bincount(shots.astype(np.int64), minlength=1 << n)
    chi2, pval = scipy.stats.chisquare(counts, p * 40000)
    assert pval > 1e-4
    # a basis state always gives its own index; a uniform superposition is uniform
    e = np.zeros(1 << n, dtype=np.complex128)
    e[11] = 1
    assert np.all(oracle.sample(e, n, 100, seed=1) == 11)
    u = np.full(1 << n, 0.25, dtype=np.complex128)
    counts = np.bincount(oracle.sample(u, n, 32000, seed=2).astype(np.int64), minlength=16)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


# --------------------------------------------- projection filter (assertions) --
def filter_closed_form(thetas, blocks):
    """P(0) of each filter block and their product, from the system's uniform
    superposition: the controlled phase on |x> is phi_x = 2 sum_j theta_j s_j
    (s_j = +-1), block k keeps the weight cos^2(phi_x / 2) once more."""
    n = thetas.size
    x = np.arange(1 << n)
    s = 1.0 - 2.0 * ((x[:, None] >> np.arange(n)[None, :]) & 1)
    phi = 2.0 * (s * thetas[None, :]).sum(axis=1)
    c2 = np.cos(phi / 2) ** 2
    m = [np.mean(c2 ** k) for k in range(blocks + 1)]
    return np.array([m[k] / m[k - 1] for k in range(1, blocks + 1)]), m[blocks]


def test_projection_filter_assertions_follow_the_closed_form():
    c = W.projection_filter(7, seed=11, blocks=5, trotter=3)
    psi = oracle.basis_state(c.n)
    r = oracle.run(psi, c.n, c.gates, seed=0)
    assert r.status == 0
    p0, prod = filter_closed_form(c.meta["thetas"], 5)
    assert np.all(r.outcomes == 0)
    assert np.abs(r.probs[0::2] - p0).max() < 1e-12       # the asserted P(0) of each block
    assert np.all(r.probs[1::2] == 1.0)                    # the resets after an assertion
    assert abs(np.prod(r.probs[0::2]) - prod) < 1e-12
