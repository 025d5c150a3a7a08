"""OpenQASM 2.0 reader (qsim_parse_qasm, host only): records, broadcasting,
user gates, the decompositions of ccx / cswap / sx / c3x / c4x / c3sqrtx /
rccx / rc3x against the oracle and dense matrices, errors."""
import math

import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import qsim as qs
from paper_2310_17739_gb300 import workload as W
from paper_2310_17739_gb300.workload import OP


def recs(g):
    return [(int(r["op"]), int(r["q0"]), int(r["q1"]), tuple(float(x) for x in r["p"])) for r in g]


def test_basic_program():
    text = """OPENQASM 2.0;
include "qelib1.inc";
// a comment
qreg q[3];
creg c[3];
h q[0];
cx q[0], q[1];
rz(pi/4) q[2];
u3(0.1, -pi/2, 2*pi/3) q[1];
u2(0, pi) q[0];
crz(-(1.5 + 0.5)^2) q[2], q[0];
barrier q;
measure q[1] -> c[1];
reset q[2];
"""
    n, g, m = qs.parse_qasm(text)
    assert n == 3
    assert recs(g) == [
        (OP["H"], 0, 0, (0.0, 0.0, 0.0)),
        (OP["CX"], 0, 1, (0.0, 0.0, 0.0)),
        (OP["RZ"], 2, 0, (math.pi / 4, 0.0, 0.0)),
        (OP["U3"], 1, 0, (0.1, -math.pi / 2, 2 * math.pi / 3)),
        (OP["U2"], 0, 0, (0.0, math.pi, 0.0)),
        (OP["CRZ"], 2, 0, (-4.0, 0.0, 0.0)),
        (OP["BARRIER"], 0, 0, (0.0, 0.0, 0.0)),
        (OP["MEASURE"], 1, 0, (0.0, 0.0, 0.0)),
        (OP["RESET"], 2, 0, (0.0, 0.0, 0.0)),
    ]


def test_registers_broadcast_and_offsets():
    text = "OPENQASM 2.0; qreg a[3]; qreg b[3]; creg c[6]; h a; cx a, b; rx(0.5) b[2]; measure a -> c;"
    n, g, _ = qs.parse_qasm(text)
    assert n == 6
    r = recs(g)
    assert r[:3] == [(OP["H"], k, 0, (0.0, 0.0, 0.0)) for k in range(3)]
    assert r[3:6] == [(OP["CX"], k, 3 + k, (0.0, 0.0, 0.0)) for k in range(3)]
    assert r[6] == (OP["RX"], 5, 0, (0.5, 0.0, 0.0))
    assert [x[:2] for x in r[7:]] == [(OP["MEASURE"], k) for k in range(3)]


def test_user_gate_definitions_expand_with_parameters():
    text = """OPENQASM 2.0; include "qelib1.inc"; qreg q[2];
gate half(theta) a, b { rz(theta/2) a; cx a, b; ry(-theta) b; }
gate twice(t) a, b { half(t) a, b; half(2*t) b, a; }
twice(0.3) q[1], q[0];
"""
    _, g, _ = qs.parse_qasm(text)
    assert recs(g) == [
        (OP["RZ"], 1, 0, (0.15, 0.0, 0.0)), (OP["CX"], 1, 0, (0.0, 0.0, 0.0)), (OP["RY"], 0, 0, (-0.3, 0.0, 0.0)),
        (OP["RZ"], 0, 0, (0.3, 0.0, 0.0)), (OP["CX"], 0, 1, (0.0, 0.0, 0.0)), (OP["RY"], 1, 0, (-0.6, 0.0, 0.0)),
    ]


def run_qasm(text, psi):
    n, g, m = qs.parse_qasm(text)
    out = psi.copy()
    oracle.run(out, n, g, m)
    return out


def test_ccx_and_cswap_are_exact():
    """The decompositions equal the Toffoli and Fredkin permutations exactly
    (phases included), on every basis state and on a random state."""
    n = 3
    for gate, perm in (("ccx q[0], q[1], q[2];", lambda x: x ^ 4 if (x & 3) == 3 else x),
                       ("cswap q[0], q[1], q[2];",
                        lambda x: (x & 1) | ((x >> 2) & 1) << 1 | ((x >> 1) & 1) << 2 if x & 1 else x)):
        text = "OPENQASM 2.0; qreg q[3]; " + gate
        for x in range(8):
            e = np.zeros(8, dtype=np.complex128)
            e[x] = 1
            out = run_qasm(text, e)
            ref = np.zeros(8, dtype=np.complex128)
            ref[perm(x)] = 1
            assert np.abs(out - ref).max() < 1e-12, (gate, x)
        psi = W.random_state(n, seed=1)
        ref = np.zeros_like(psi)
        for x in range(8):
            ref[perm(x)] = psi[x]
        assert np.abs(run_qasm(text, psi) - ref).max() < 1e-12


def dense_of(text, n):
    """The 2^n x 2^n matrix a program applies, column by column on the oracle."""
    N = 1 << n
    U = np.zeros((N, N), dtype=np.complex128)
    for x in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[x] = 1
        U[:, x] = run_qasm(text, e)
    return U


def controlled_dense(n, controls, target, u):
    """|x> -> |x> unless every control bit is 1; then u acts on the target bit
    (matrix written entry by entry from that definition)."""
    N = 1 << n
    M = np.zeros((N, N), dtype=np.complex128)
    cm = sum(1 << c for c in controls)
    for x in range(N):
        if x & cm != cm:
            M[x, x] = 1
            continue
        b = (x >> target) & 1
        for r in range(2):
            M[(x & ~(1 << target)) | (r << target), x] = u[r, b]
    return M


SQRT_X = np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]]) / 2
PAULI_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)


@pytest.mark.parametrize("gate,n,controls,target,u", [
    ("c3x q[0], q[1], q[2], q[3];", 4, [0, 1, 2], 3, PAULI_X),
    ("c3x q[3], q[0], q[2], q[1];", 4, [3, 0, 2], 1, PAULI_X),
    ("c4x q[0], q[1], q[2], q[3], q[4];", 5, [0, 1, 2, 3], 4, PAULI_X),
    ("c4x q[4], q[2], q[0], q[3], q[1];", 5, [4, 2, 0, 3], 1, PAULI_X),
    ("c3sqrtx q[0], q[1], q[2], q[3];", 4, [0, 1, 2], 3, SQRT_X),
    ("c3sqrtx q[2], q[3], q[1], q[0];", 4, [2, 3, 1], 0, SQRT_X),
])
def test_multi_controlled_gates_are_exact(gate, n, controls, target, u):
    """The paper's gate table: C3X, C4X (X controlled by 3 / 4 qubits) and
    C3XSQRTX (sqrt(X) = the matrix of `sx`, controlled by 3 qubits), exactly,
    global phase included, against the matrix of their definition."""
    U = dense_of(f"OPENQASM 2.0; qreg q[{n}]; " + gate, n)
    assert np.abs(U - controlled_dense(n, controls, target, u)).max() < 1e-12
    # c3sqrtx applied twice is c3x
    if "sqrtx" in gate:
        U2 = dense_of(f"OPENQASM 2.0; qreg q[{n}]; " + gate + gate, n)
        assert np.abs(U2 - controlled_dense(n, controls, target, PAULI_X)).max() < 1e-12


def test_relative_phase_toffolis():
    """RCCX and RC3X (the paper's gate table: relative-phase CCX and 3-controlled
    X) equal CCX / C3X followed by a diagonal of unit phases (the defining
    property), with the phases of the OpenQASM 2.0 standard header: for rccx a, b, c
    -i on |c b a> = |011>, +i on |111>, -1 on |101> after the Toffoli (index bit
    q = qubit q); for rc3x a, b, c, d +i on |d c b a> = |0011>, -i on |1011>, -1 on
    |1111> after the C3X."""
    U = dense_of("OPENQASM 2.0; qreg q[3]; rccx q[0], q[1], q[2];", 3)
    D = U @ controlled_dense(3, [0, 1], 2, PAULI_X).conj().T
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12
    want = np.ones(8, dtype=np.complex128)
    want[0b011], want[0b111], want[0b101] = -1j, 1j, -1
    assert np.abs(np.diag(D) - want).max() < 1e-12
    U = dense_of("OPENQASM 2.0; qreg q[4]; rc3x q[0], q[1], q[2], q[3];", 4)
    D = U @ controlled_dense(4, [0, 1, 2], 3, PAULI_X).conj().T
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12
    want = np.ones(16, dtype=np.complex128)
    want[0b0011], want[0b1011], want[0b1111] = 1j, -1j, -1
    assert np.abs(np.diag(D) - want).max() < 1e-12
    # on other qubits and broadcast-free operands too
    U = dense_of("OPENQASM 2.0; qreg q[4]; rccx q[3], q[1], q[0];", 4)
    D = U @ controlled_dense(4, [3, 1], 0, PAULI_X).conj().T
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12
    assert np.allclose(np.abs(np.diag(D)), 1)


def test_sx_squares_to_x_and_sxdg_undoes_it():
    psi = W.random_state(2, seed=4)
    out = run_qasm("OPENQASM 2.0; qreg q[2]; sx q[1]; sx q[1];", psi)
    ref = psi.reshape(2, 2)[::-1, :].reshape(-1)   # X on qubit 1 (the high index bit)
    assert np.abs(out - ref).max() < 1e-12
    assert np.abs(run_qasm("OPENQASM 2.0; qreg q[2]; sx q[0]; sxdg q[0];", psi) - psi).max() < 1e-12


def to_qasm(n, g):
    """Gate records of the named qelib1 gates as OpenQASM 2.0 text (test helper)."""
    names = {OP["H"]: "h", OP["X"]: "x", OP["Y"]: "y", OP["Z"]: "z", OP["S"]: "s", OP["SDG"]: "sdg",
             OP["T"]: "t", OP["TDG"]: "tdg", OP["RX"]: "rx", OP["RY"]: "ry", OP["RZ"]: "rz", OP["U1"]: "u1",
             OP["U2"]: "u2", OP["U3"]: "u3", OP["CX"]: "cx", OP["CY"]: "cy", OP["CZ"]: "cz", OP["CH"]: "ch",
             OP["SWAP"]: "swap", OP["CRX"]: "crx", OP["CRY"]: "cry", OP["CRZ"]: "crz", OP["CU1"]: "cu1",
             OP["CU3"]: "cu3", OP["RXX"]: "rxx", OP["RZZ"]: "rzz", OP["ID"]: "id"}
    npar = {"rx": 1, "ry": 1, "rz": 1, "u1": 1, "u2": 2, "u3": 3, "crx": 1, "cry": 1, "crz": 1, "cu1": 1,
            "cu3": 3, "rxx": 1, "rzz": 1}
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{n}];"]
    for r in g:
        nm = names[int(r["op"])]
        par = "(" + ", ".join(repr(float(x)) for x in r["p"][: npar[nm]]) + ")" if nm in npar else ""
        qa = f"q[{int(r['q0'])}]" + (f", q[{int(r['q1'])}]" if int(r["op"]) >= 32 else "")
        lines.append(f"{nm}{par} {qa};")
    return "\n".join(lines) + "\n"


def test_round_trip_of_a_random_circuit_and_its_state():
    n = 6
    c = W.random_circuit(n, 400, seed=9, with_generic=False)
    n2, g, m = qs.parse_qasm(to_qasm(n, c.gates))
    assert n2 == n
    keep = [(op, q0, q1 if op >= 32 else 0) for op, q0, q1, _ in recs(c.gates)]
    assert [x[:3] for x in recs(g)] == keep          # the angles are checked through the state
    psi = W.random_state(n, seed=2)
    a, b = psi.copy(), psi.copy()
    oracle.run(a, n, c.gates)
    oracle.run(b, n, g, m)
    assert np.abs(a - b).max() < 1e-12


@pytest.mark.parametrize("text,where", [
    ("OPENQASM 2.0; qreg q[2]; foo q[0];", "line 1: unknown gate 'foo'"),
    ("OPENQASM 2.0;\nqreg q[2];\nh q[2];", "line 3: index out of range"),
    ("OPENQASM 2.0;\nqreg q[2];\nrx q[0];", "line 3: 'rx' takes 1 parameter"),
    ("OPENQASM 2.0;\nqreg q[2];\ncx q[0], q[0];", "line 3: 'cx' on a repeated qubit"),
    ("OPENQASM 2.0;\nqreg q[2];\nh q[0]\nh q[1];", "line 4: expected ';'"),
    ("OPENQASM 2.0; qreg q[1]; creg c[1]; if (c==1) x q[0];", "'if' is not supported"),
    ("OPENQASM 3.0; qubit q;", "only OpenQASM 2.x"),
])
def test_errors_name_the_line(text, where):
    with pytest.raises(qs.QsimError) as e:
        qs.parse_qasm(text)
    assert e.value.status == qs.E_INVAL and where in str(e.value)


def test_expression_functions_numbers_and_precedence():
    """Parameter expressions: unary functions, exponent notation, leading-dot
    numbers, right-associative ^, and ^ binding tighter than unary minus
    (-2^2 = -4)."""
    text = """OPENQASM 2.0; qreg q[1];
rz(sin(pi/6) + cos(0)) q[0];
rz(sqrt(16) * exp(0) - ln(1)) q[0];
rz(tan(pi/4)) q[0];
rz(1e-3 + .5 + 2.5E1) q[0];
rz(2^3^2) q[0];
rz(-2^2) q[0];
rz((1 - 3) * -2 / 4) q[0];
"""
    _, g, _ = qs.parse_qasm(text)
    got = [float(r["p"][0]) for r in g]
    want = [1.5, 4.0, 1.0, 25.501, 512.0, -4.0, 1.0]
    assert np.allclose(got, want, rtol=0, atol=1e-12), got


def test_builtin_u_cx_and_nested_user_gates():
    """U and CX (the language's built-ins) and a user gate calling another one
    with expressions of its parameters, against the oracle."""
    text = """OPENQASM 2.0; qreg q[3];
gate inner(a) x, y { U(a, 0, 0) x; CX x, y; }
gate outer(b, c) x, y, z { inner(b / 2) x, y; inner(-c) y, z; rz(b + c) z; }
outer(0.8, 0.3) q[0], q[1], q[2];
"""
    n, g, m = qs.parse_qasm(text)
    assert n == 3
    ops = [int(r["op"]) for r in g]
    assert ops == [OP["U3"], OP["CX"], OP["U3"], OP["CX"], OP["RZ"]]
    ref = W.records([(OP["U3"], 0, 0, 0.4, 0.0, 0.0, 0, 0), (OP["CX"], 0, 1, 0, 0, 0, 0, 0),
                     (OP["U3"], 1, 0, -0.3, 0.0, 0.0, 0, 0), (OP["CX"], 1, 2, 0, 0, 0, 0, 0),
                     (OP["RZ"], 2, 0, 1.1, 0.0, 0.0, 0, 0)])
    psi = W.random_state(n, seed=4)
    a, b = psi.copy(), psi.copy()
    oracle.run(a, n, g, m)
    oracle.run(b, n, ref)
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("text,where", [
    ("OPENQASM 2.0; qreg a[2]; qreg b[3]; cx a, b;", "registers of different sizes"),
    ("OPENQASM 2.0; qreg q[1]; opaque g q;", "'opaque' is not supported"),
    ("OPENQASM 2.0; qreg q[1]; rz(foo) q[0];", "foo"),
])
def test_more_errors(text, where):
    with pytest.raises(qs.QsimError) as e:
        qs.parse_qasm(text)
    assert e.value.status == qs.E_INVAL and where in str(e.value)
