"""The synthetic input recipes (host only): gate counts, two-qubit fraction,
measurement placement and the batched / serving structures that stand in for
the paper's circuits."""
import numpy as np

from paper_2310_17739_gb300 import workload as W
from paper_2310_17739_gb300.workload import OP

TWO_Q = {OP[k] for k in ("CX", "CY", "CZ", "CH", "SWAP", "CRX", "CRY", "CRZ", "CU1", "CU3", "RXX", "RZZ", "C2")}


def two_qubit_fraction(g):
    ops = g["op"]
    unitary = ~np.isin(ops, [OP["MEASURE"], OP["RESET"], OP["BARRIER"]])
    return np.isin(ops[unitary], list(TWO_Q)).mean()


def test_gate_count_is_authoritative_and_cut_at_a_gadget_end():
    """Cycled Trotter steps stop at the end of the gadget that crosses the
    target; the overshoot is shorter than the longest gadget."""
    for target in (5_000, 12_345, 40_000):
        c = W.ucc_circuit(21, seed=3, n_gadgets=200, w_lo=2, w_hi=6, target_gates=target)
        # longest gadget of weight 6: a basis gate on each side of 6 X/Y
        # qubits, 2 x 5 CX and the RZ
        assert target <= c.G < target + 4 * 6 - 1
        assert c.meta["steps"] == c.G / W.ucc_circuit(21, seed=3, n_gadgets=200, w_lo=2, w_hi=6).G


def test_large_recipe_two_qubit_fraction_and_measurements():
    """The benchmark's recipe (21 qubits, 2,000 gadgets of weight 2-6 per step,
    8 measurements) on a 200,000-gate prefix: about half of the gates are
    two-qubit CX (the paper's circuits: ~60 %), 8 MEASURE records, each at a
    gadget boundary."""
    c = W.ucc_circuit(21, seed=3, n_gadgets=2000, w_lo=2, w_hi=6, target_gates=200_000, n_meas=8)
    assert 0.45 <= two_qubit_fraction(c.gates) <= 0.55
    ops = c.gates["op"]
    meas = np.flatnonzero(ops == OP["MEASURE"])
    assert meas.size == 8
    # the same stream without the MEASURE records, whose insertion points must
    # be gadget boundaries
    bare = W.ucc_circuit(21, seed=3, n_gadgets=2000, w_lo=2, w_hi=6, target_gates=200_000)
    assert bare.G == c.G - 8
    keep = np.ones(c.G, dtype=bool)
    keep[meas] = False
    assert np.array_equal(c.gates[keep], bare.gates)
    # gadget boundaries from the step's gadgets, cycled
    lens = [W.gadget_rows(s, letters, t) for s, letters, t in c.meta["paulis"]]
    lens = np.array([len(r) for r in lens])
    step = int(lens.sum())
    bounds = (np.cumsum(lens)[None, :] + step * np.arange(bare.G // step + 1)[:, None]).ravel()
    pos = meas - np.arange(meas.size)          # insertion points in the bare stream
    assert np.all(np.isin(pos, bounds))


def test_batched_recipe_structure():
    """The batched recipe at reduced sizes: the parameter sets share one
    12-qubit structure (only RZ angles differ), the uneven part spans widths
    10..18, every instance reaches its gate count and has its Hamiltonian."""
    cs, hams = W.config_batched(n_param_sets=8, n_uneven=16, gates=2_000, n_terms=20, n_set_gadgets=40)
    sets, uneven = cs[:8], cs[8:]
    ref = sets[0].gates
    for c in sets[1:]:
        assert c.n == 12
        assert np.array_equal(c.gates["op"], ref["op"]) and np.array_equal(c.gates["q0"], ref["q0"])
        diff = np.flatnonzero(np.any(c.gates["p"] != ref["p"], axis=1))
        assert diff.size and np.all(c.gates["op"][diff] == OP["RZ"])
    assert all(10 <= c.n <= 18 for c in uneven) and len({c.n for c in uneven}) > 3
    assert all(c.G >= 2_000 for c in cs)
    assert len(hams) == len(cs) and all(len(h) == 20 for h in hams)
