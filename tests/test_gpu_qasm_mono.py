"""GPU parity for two input forms: an OpenQASM 2.0 program with the paper's
multi-qubit gates (parsed on the host, run through the C ABI), and streams of
diagonal and permutation gates, which the packer turns into monomial ops
(one complex multiply per amplitude) in the tile and resident kernels."""
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

QASM = """OPENQASM 2.0;
include "qelib1.inc";
qreg a[6];
qreg b[6];
creg c[4];
gate layer(t) x, y, z { ry(t) x; cx x, y; rzz(t/2) y, z; ccx x, y, z; }
h a;
ry(0.3) b;
layer(0.7) a[0], a[1], b[2];
c3x a[0], a[1], a[2], b[0];
rccx b[1], b[2], a[3];
c4x a[1], b[1], a[4], b[4], a[5];
rc3x a[2], b[3], b[5], a[0];
c3sqrtx b[0], a[3], b[2], a[1];
cswap a[5], b[4], b[5];
measure a[2] -> c[0];
sx b;
layer(-1.1) b[3], a[5], a[4];
barrier a, b;
u3(0.4, 1.2, -0.3) a;
crz(0.9) a[1], b[1];
reset b[0];
cu1(2.2) b[2], a[2];
measure b[4] -> c[1];
"""


@pytest.mark.parametrize("dtype,cfg", [("c128", dict(fusion=1)), ("c64", dict(fusion=2)),
                                       ("c128", dict(fusion=0, tile_bits=8)), ("c64", dict(fusion=1, tile_bits=9))])
def test_parsed_qasm_program_against_the_oracle(dtype, cfg):
    n, g, m = qs.parse_qasm(QASM)
    assert n == 12
    ref = oracle.basis_state(n)
    r = oracle.run(ref, n, g, m, seed=21)
    assert r.status == 0 and len(r.outcomes) == 3
    sim = qs.Sim(n, dtype, seed=21, config=cfg)
    sim.apply(g, m)
    assert sim.sync() == 0
    out, _ = sim.outcomes()
    assert np.array_equal(out, r.outcomes)
    got = sim.state()
    if dtype == "c128":
        assert np.abs(got - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, got) <= 1e-5


def diag_perm_stream(n, G, seed):
    """Random diagonal (Z, S, T, RZ, U1, CZ, CU1, CRZ, RZZ) and permutation (X, CX,
    SWAP) gates after an H layer, so that every amplitude is populated."""
    rng = np.random.default_rng(seed)
    one = ["Z", "S", "SDG", "T", "TDG", "RZ", "U1", "X"]
    two = ["CZ", "CU1", "CRZ", "RZZ", "CX", "SWAP"]
    rows = [(OP["H"], q, 0, 0.0, 0.0, 0.0) for q in range(n)]
    for _ in range(G):
        if rng.random() < 0.5:
            rows.append((OP[one[rng.integers(len(one))]], int(rng.integers(n)), 0, float(rng.uniform(-3, 3)), 0, 0))
        else:
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            rows.append((OP[two[rng.integers(len(two))]], a, b, float(rng.uniform(-3, 3)), 0, 0))
    return W.Circuit(n, W.records(rows))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,tile_bits,fusion", [(9, 0, 0), (9, 0, 1), (16, 12, 0), (16, 11, 1), (15, 10, 1)])
def test_diagonal_and_permutation_streams(dtype, n, tile_bits, fusion):
    c = diag_perm_stream(n, 1500, seed=n + 3 * fusion)
    ref = oracle.basis_state(n)
    oracle.run(ref, n, c.gates)
    sim = qs.Sim(n, dtype, config=dict(tile_bits=tile_bits, fusion=fusion))
    sim.apply(c.gates)
    assert sim.sync() == 0
    got = sim.state()
    if dtype == "c128":
        assert np.abs(got - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, got) <= 1e-5
