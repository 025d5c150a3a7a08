"""Brute-force numpy constructions used to pin the oracle (test-only).

Everything here is built a different way from the oracle: full 2^n x 2^n
matrices from Kronecker products or from explicit index comparison, Pauli
strings from Kronecker products of 2x2 Pauli matrices.
"""
import math

import numpy as np

from paper_2310_17739_gb300 import workload as W

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}


def kron_all(mats):
    out = np.ones((1, 1), dtype=np.complex128)
    for m in mats:
        out = np.kron(out, m)
    return out


def full_1q(n, q, u):
    """I_{2^{n-q-1}} (x) U (x) I_{2^q}: qubit q is index bit q (little-endian)."""
    return kron_all([np.eye(1 << (n - q - 1)), u, np.eye(1 << q)])


def full_2q(n, q0, q1, m):
    """Full matrix of a 4x4 operator in local basis l = b_q0 + 2 b_q1, built by
    comparing every pair of basis indices (no index formula shared with the oracle)."""
    N = 1 << n
    F = np.zeros((N, N), dtype=np.complex128)
    other = ~((1 << q0) | (1 << q1))
    for i in range(N):
        li = ((i >> q0) & 1) + 2 * ((i >> q1) & 1)
        for j in range(N):
            if (i & other) != (j & other):
                continue
            lj = ((j >> q0) & 1) + 2 * ((j >> q1) & 1)
            F[i, j] = m[li, lj]
    return F


def pauli_dense(n, letters_by_qubit):
    """letters_by_qubit: dict q -> 'X'|'Y'|'Z'.  Returns the 2^n matrix."""
    mats = [PAULI[letters_by_qubit.get(q, "I")] for q in reversed(range(n))]
    return kron_all(mats)


def term_dense(n, x, z):
    letters = {}
    for q in range(n):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        if xb and zb:
            letters[q] = "Y"
        elif xb:
            letters[q] = "X"
        elif zb:
            letters[q] = "Z"
    return pauli_dense(n, letters)


def inverse_rows(rows):
    """Adjoint of a list of named-gate rows (op, q0, q1, p0): reversed order,
    rotation angles negated, S<->SDG and T<->TDG; self-inverse gates kept."""
    from paper_2310_17739_gb300.workload import OP
    neg = {OP["RX"], OP["RY"], OP["RZ"], OP["U1"], OP["CRX"], OP["CRY"], OP["CRZ"], OP["CU1"],
           OP["RXX"], OP["RZZ"]}
    flip = {OP["S"]: OP["SDG"], OP["SDG"]: OP["S"], OP["T"]: OP["TDG"], OP["TDG"]: OP["T"]}
    selfinv = {OP["ID"], OP["X"], OP["Y"], OP["Z"], OP["H"], OP["CX"], OP["CY"], OP["CZ"],
               OP["CH"], OP["SWAP"]}
    out = []
    for r in reversed(list(rows)):
        op = int(r[0])
        if op in neg:
            out.append((op, int(r[1]), int(r[2]), -float(r[3])))
        elif op in flip:
            out.append((flip[op], int(r[1]), int(r[2]), float(r[3])))
        elif op in selfinv:
            out.append((op, int(r[1]), int(r[2]), float(r[3])))
        else:
            raise ValueError(f"no named inverse for op {op}")
    return out


def rows_of(gates):
    return [(int(g["op"]), int(g["q0"]), int(g["q1"]), float(g["p"][0])) for g in gates]


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def load_mma_table(path):
    rows = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[parts[0]] = [float(v) for v in parts[1:]]
    return rows


SELF_INVERSE = {"ID", "X", "Y", "Z", "H", "CX", "CY", "CZ", "SWAP", "BARRIER"}
NEGATE_ANGLE = {"RX", "RY", "RZ", "U1", "CRX", "CRY", "CRZ", "CU1", "RXX", "RZZ"}


def invert_records(g):
    """Gate records of the inverse circuit (reversed order, each gate inverted),
    for the gates whose inverse is the gate itself or its negated angle."""
    inv = g[::-1].copy()
    names = {v: k for k, v in W.OP.items()}
    orig = inv["op"].copy()          # rules select on the original op codes
    for op in np.unique(orig):
        name = names[int(op)]
        sel = orig == op
        if name in NEGATE_ANGLE:
            inv["p"][sel, 0] = -inv["p"][sel, 0]
        elif name == "S":
            inv["op"][sel] = W.OP["SDG"]
        elif name == "SDG":
            inv["op"][sel] = W.OP["S"]
        elif name == "T":
            inv["op"][sel] = W.OP["TDG"]
        elif name == "TDG":
            inv["op"][sel] = W.OP["T"]
        elif name not in SELF_INVERSE:
            raise ValueError(f"no inverse rule for {name}")
    return inv
