"""Replay of compiled programs as CUDA graphs (qsim_config.graphs) against
stream launches and the oracle.

Graph replay launches the same kernels with the same arguments in the same
order, so the states are compared bit for bit with the launch-by-launch
replay; the oracle check uses the complex64 tolerance of the parity tests
(infidelity <= 1e-5) and bit-exact outcomes.
"""
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


def replay(c, graphs, runs, fusion=2, tile_bits=12, dtype="c64", chunk_gates=0):
    sim = qs.Sim(c.n, dtype, seed=9, config=dict(fusion=fusion, tile_bits=tile_bits, graphs=graphs,
                                                 chunk_gates=chunk_gates))
    prog = sim.compile(c.gates, c.mats)
    for _ in range(runs):
        sim.run(prog)
    assert sim.sync() == 0
    psi = sim.state()
    out, probs = sim.outcomes()
    prog.free()
    sim.close()
    return psi, out, probs


@pytest.mark.parametrize("fusion,dtype", [(2, "c64"), (1, "c64"), (1, "c128")])
def test_graph_replay_matches_stream_launches_and_oracle(fusion, dtype):
    """Three replays of a program with measurements (chunks of 1,500 gates, so
    several chunks and graph runs): stream launches, graphs from the second
    run, graphs from the first run — identical states and outcomes; the same
    against the oracle running the circuit three times in a row (measurement
    ordinals continue across replays)."""
    n = 16
    c = W.ucc_circuit(n, seed=41, n_gadgets=None, w_lo=2, w_hi=5, theta="uniform", target_gates=5000, n_meas=3)
    ref = [replay(c, 2, 3, fusion=fusion, dtype=dtype, chunk_gates=1500)]
    for mode in (0, 1):
        ref.append(replay(c, mode, 3, fusion=fusion, dtype=dtype, chunk_gates=1500))
    for psi, out, probs in ref[1:]:
        assert np.array_equal(psi, ref[0][0])
        assert np.array_equal(out, ref[0][1])
        assert np.array_equal(probs, ref[0][2])
    psi_o = oracle.basis_state(n)
    gates3 = np.concatenate([c.gates] * 3)
    r = oracle.run(psi_o, n, gates3, c.mats, seed=9)
    assert r.status == 0
    assert np.array_equal(ref[0][1], r.outcomes)
    assert 1 - H.fidelity(psi_o, ref[0][0]) <= 1e-5


def test_graphs_rebuilt_after_set_config_and_disabled_by_persistent():
    """A config change between replays rebuilds (or drops) the program's graphs;
    every combination reaches the same state as plain launches."""
    n = 15
    c = W.ucc_circuit(n, seed=43, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=4000, n_meas=2)
    ref, _, _ = replay(c, 2, 4)
    sim = qs.Sim(n, "c64", seed=9, config=dict(fusion=2, tile_bits=12, graphs=1))
    prog = sim.compile(c.gates, c.mats)
    sim.run(prog)
    sim.set_config(graphs=0)           # rebuilt at the next run
    sim.run(prog)
    sim.set_config(persistent=1)       # resident blocks: launched pass by pass
    sim.run(prog)
    sim.set_config(persistent=0, graphs=1)
    sim.run(prog)
    assert sim.sync() == 0
    got = sim.state()
    prog.free()
    sim.close()
    assert 1 - H.fidelity(ref, got) <= 1e-6


def test_graph_profile_windows_span_one_graph_launch():
    """With sampling on, each graph launch is one timing window counting all of
    its tile passes once, with one read and one write of the state each."""
    n = 18
    c = W.ucc_circuit(n, seed=31, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=6000, n_meas=3)
    sim = qs.Sim(n, "c64", config=dict(fusion=2, tile_bits=12, graphs=1))
    prog = sim.compile(c.gates)
    passes = prog.info()["passes"]
    sim.profile_start(4)
    sim.run(prog)
    assert sim.sync() == 0
    prof = sim.profile_read()
    assert prof["launches"] == passes
    assert prof["samples"] == passes       # every graph launch is a window
    assert prof["bytes"] == passes * 2 * 8 * (1 << n)
    assert prof["ms"] > 0
    sim.profile_start(0)
    prog.free()
    sim.close()


def test_program_freed_after_graph_replay_and_context_destroyed_first():
    """Graphs are released with their program, and with their context when the
    context goes first (the program becomes an orphan)."""
    n = 14
    c = W.ucc_circuit(n, seed=47, n_gadgets=None, w_lo=2, w_hi=5, theta="uniform", target_gates=2000, n_meas=1)
    sim = qs.Sim(n, "c64", config=dict(fusion=2, tile_bits=12, graphs=1))
    p1 = sim.compile(c.gates)
    p2 = sim.compile(c.gates)
    sim.run(p1)
    sim.run(p2)
    assert sim.sync() == 0
    p1.free()
    sim.close()
    p2.free()


def test_apply_long_chunks_as_graphs_matches_stream_launches():
    """qsim_apply runs a chunk of >= 256 tile passes as graph launches (the
    graphs released once their launches complete): same state and outcomes as
    launching every pass, and the oracle's outcomes."""
    n = 16
    c = W.ucc_circuit(n, seed=53, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=40000, n_meas=4)
    res = []
    for graphs in (2, 0):
        sim = qs.Sim(n, "c64", seed=5, config=dict(fusion=2, tile_bits=12, graphs=graphs))
        prog = sim.compile(c.gates)
        passes = prog.info()["passes"]
        prog.free()
        sim.apply(c.gates, c.mats)
        assert sim.sync() == 0
        res.append((sim.state(), sim.outcomes()[0]))
        sim.close()
    assert passes >= 256
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    psi = oracle.basis_state(n)
    r = oracle.run(psi, n, c.gates, c.mats, seed=5)
    assert np.array_equal(res[1][1], r.outcomes)
    assert 1 - H.fidelity(psi, res[1][0]) <= 1e-5
