"""Host-side tests of the native library (no GPU): exported symbols, the fusion
compiler (fused == unfused on the oracle), the pass schedule's invariants and
argument validation."""
import re

import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import workload as W
from paper_2310_17739_gb300.workload import OP
from tests import helpers as H

qs = pytest.importorskip("paper_2310_17739_gb300.qsim")


def header_symbols():
    txt = open("include/qsim.h").read()
    return sorted(set(re.findall(r"QSIM_API\s+[\w\s\*]*?\b(qsim_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(qs.lib(), s), s


def fused_to_records(ops):
    """Express compiled ops (k <= 2) as C1/C2/MEASURE/RESET gate records + mats."""
    rows, mats = [], []
    off = 0
    for o in ops:
        if o[0] == "event":
            _, op, q, flags = o
            rows.append((op, q, 0, 0.0, 0.0, 0.0, flags))
            continue
        k, qubits, M = o
        assert k <= 2
        rows.append((OP["C1"] if k == 1 else OP["C2"], qubits[0], qubits[1] if k == 2 else 0,
                     0.0, 0.0, 0.0, 0, off))
        flat = np.ascontiguousarray(M, dtype=np.complex128).view(np.float64).ravel()
        mats.append(flat)
        off += flat.size
    return W.records(rows), (np.concatenate(mats) if mats else np.zeros(1))


def apply_block(psi, n, qubits, M):
    """Dense k-qubit block on psi (numpy reshape; bit j of the local index = qubits[j])."""
    k = len(qubits)
    t = psi.reshape([2] * n)  # axis a <-> qubit n-1-a
    axes = [n - 1 - q for q in reversed(qubits)]  # local index bits high..low
    t = np.moveaxis(t, axes, list(range(k)))
    shp = t.shape
    t = (M @ t.reshape(1 << k, -1)).reshape(shp)
    t = np.moveaxis(t, list(range(k)), axes)
    return np.ascontiguousarray(t).reshape(-1)


@pytest.mark.parametrize("fusion", [0, 1])
@pytest.mark.parametrize("n,seed", [(2, 0), (4, 1), (6, 2), (9, 3)])
def test_fused_equals_unfused_on_oracle(fusion, n, seed):
    c = W.random_circuit(n, 300, seed=seed)
    ops = qs.fuse(n, c.gates, c.mats, dtype=qs.C128, fusion=fusion)
    recs, mats = fused_to_records(ops)
    a = W.random_state(n, seed=seed + 9)
    b = a.copy()
    oracle.run(a, n, c.gates, c.mats)
    oracle.run(b, n, recs, mats)
    # the generic C1/C2 records are not unitary: compare relative to the state's scale
    assert np.abs(a - b).max() < 1e-13 * max(1.0, np.abs(a).max())
    if fusion == 0:
        assert sum(1 for o in ops if o[0] != "event") == c.G


@pytest.mark.parametrize("tile_bits", [0, 6, 8])
def test_fusion_with_measurements_matches_oracle_outcomes(tile_bits):
    n = 10
    c = W.ucc_circuit(n, seed=11, n_gadgets=30, w_lo=2, w_hi=6, target_gates=4000, n_meas=12,
                      meas_reset=True)
    ops = qs.fuse(n, c.gates, c.mats, dtype=qs.C128, tile_bits=tile_bits)
    recs, mats = fused_to_records(ops)
    a = oracle.basis_state(n)
    b = oracle.basis_state(n)
    ra = oracle.run(a, n, c.gates, c.mats, seed=99)
    rb = oracle.run(b, n, recs, mats, seed=99)
    assert ra.status == rb.status == 0
    assert np.array_equal(ra.outcomes, rb.outcomes)
    assert np.abs(ra.probs - rb.probs).max() < 1e-12
    assert np.abs(a - b).max() < 1e-12


def test_no_gate_crosses_a_failed_assertion():
    """Gates pending on other qubits must be applied before a measurement, so the
    state left by a failed assertion equals the unfused stream's."""
    n = 6
    rows = [(OP["H"], 3, 0, 0, 0, 0), (OP["RY"], 4, 0, 0.3, 0, 0), (OP["CX"], 1, 2, 0, 0, 0),
            (OP["X"], 0, 0, 0, 0, 0), (OP["MEASURE"], 0, 0, 0, 0, 0, 1), (OP["H"], 5, 0, 0, 0, 0),
            (OP["RZ"], 3, 0, 0.2, 0, 0)]
    g = W.records(rows)
    for tile_bits in (0, 6):
        ops = qs.fuse(n, g, dtype=qs.C128, tile_bits=tile_bits)
        recs, mats = fused_to_records(ops)
        a = W.random_state(n, seed=1)
        a[1::2] = 0  # qubit 0 surely 0 ...
        a /= np.linalg.norm(a)
        b = a.copy()
        ra = oracle.run(a, n, g)           # ... X makes it surely 1: the assertion fails
        rb = oracle.run(b, n, recs, mats)
        assert ra.status == rb.status == oracle.E_ZEROPROB
        assert np.abs(a - b).max() < 1e-14


@pytest.mark.parametrize("k_max", [3, 4, 5])
@pytest.mark.parametrize("dtype", [0, 1])
def test_k_qubit_blocks_equal_unfused(k_max, dtype):
    n = 11
    c = W.ucc_circuit(n, seed=5, n_gadgets=40, w_lo=2, w_hi=6, target_gates=2500)
    ops = qs.fuse(n, c.gates, c.mats, dtype=dtype, k_max=k_max, tile_bits=8)
    assert max(o[0] for o in ops) <= k_max
    assert any(o[0] > 2 for o in ops)
    psi = W.random_state(n, seed=3)
    ref = psi.copy()
    oracle.run(ref, n, c.gates)
    for k, qubits, M in ops:
        psi = apply_block(psi, n, qubits, M)
    assert np.abs(psi - ref).max() < 1e-11


def test_apply_block_helper_is_the_kronecker_product():
    n = 4
    rng = np.random.default_rng(0)
    M = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    psi = W.random_state(n, seed=1)
    assert np.allclose(apply_block(psi, n, [3, 1], M), H.full_2q(n, 3, 1, M) @ psi)


def test_fusion_reduces_ucc_op_count():
    n = 13
    c = W.ucc_circuit(n, seed=7, n_gadgets=200, w_lo=2, w_hi=6, target_gates=20000)
    ops = qs.fuse(n, c.gates, dtype=qs.C64)
    n_ops = sum(1 for o in ops if o[0] != "event")
    # the paper reports 1.98-2.32x on its circuits; UCC gadgets fuse at least as well
    assert c.G / n_ops > 1.8


@pytest.mark.parametrize("dtype,tile_bits", [(0, 0), (0, 9), (1, 8), (1, 0)])
def test_schedule_invariants(dtype, tile_bits):
    n = 16
    c = W.ucc_circuit(n, seed=9, n_gadgets=100, w_lo=2, w_hi=8, target_gates=6000, n_meas=5)
    ops = qs.fuse(n, c.gates, dtype=dtype, tile_bits=tile_bits)
    passes = qs.schedule(n, c.gates, dtype=dtype, tile_bits=tile_bits)
    L = 4 if dtype == 0 else 3
    covered = 0
    m_seen = set()
    for tile, first, count in passes:
        assert first == covered
        covered += count
        if tile == 0:
            assert count == 1 and ops[first][0] == "event"
            continue
        m_seen.add(bin(tile).count("1"))
        assert tile & ((1 << L) - 1) == (1 << L) - 1
        for o in ops[first: first + count]:
            assert o[0] != "event"
            for q in o[1]:
                assert (tile >> q) & 1
    assert covered == len(ops)
    assert len(m_seen) == 1


def test_invalid_records_rejected_on_host():
    n = 4
    bad = [W.records([(OP["H"], 4, 0, 0, 0, 0)]), W.records([(OP["CX"], 2, 2, 0, 0, 0)]),
           W.records([(200, 0, 0, 0, 0, 0)]), W.records([(OP["C2"], 0, 1, 0, 0, 0, 0, 100)]),
           W.records([(OP["RX"], 0, 0, float("nan"), 0, 0)])]
    for g in bad:
        with pytest.raises(qs.QsimError) as e:
            qs.fuse(n, g, np.zeros(8))
        assert e.value.status == qs.E_INVAL
