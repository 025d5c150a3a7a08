"""Seeded synthetic inputs: gate-record streams and Pauli-term lists.

This module holds no simulation arithmetic.  It only builds input records
(which gates, on which qubits, with which angles) and is shared by the GPU
library's tests and benchmark and by the CPU oracle's tests.

The paper's own workloads (Table "Problem circuits": nuclear projection-filter
circuits of 7/13/21 qubits and 1.2e4 to 1.15e8 gates, ~60% of them 2-qubit,
with one ancilla measured and reset after every filtering block) are not
available.  Seeded UCC-style circuits of the same widths, gate counts, 2-qubit
fraction and measurement pattern stand in for them.  A UCC-style circuit is a
sequence of Pauli-string exponentials exp(-i theta P), each written in
elementary gates:

    basis change  H on X letters, RX(pi/2) on Y letters, nothing on Z
    CNOT ladder   CX(q1->q2), CX(q2->q3), ..., CX(q_{w-1}->q_w)
    rotation      RZ(2 theta) on q_w
    uncompute     the ladder reversed, then H / RX(-pi/2)

With RZ(t) = exp(-i t Z/2) the block equals exp(-i theta P) exactly.
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------- records ----
# One gate record, 40 bytes, little-endian:
#   op u16 | flags u16 | q0 u32 | q1 u32 | mat u32 | p f64[3]
# q0 is the first operand (the control of controlled gates); for 2-qubit
# matrices the local basis index is b_q0 + 2*b_q1.  mat is the offset, in
# doubles, of a C1 (8 doubles) or C2 (32 doubles) row-major complex matrix in
# the companion mats array.  MEASURE flags bit 0 selects the assertion mode.
GATE_DTYPE = np.dtype({
    "names": ["op", "flags", "q0", "q1", "mat", "p"],
    "formats": ["<u2", "<u2", "<u4", "<u4", "<u4", ("<f8", (3,))],
    "offsets": [0, 2, 4, 8, 12, 16],
    "itemsize": 40,
})
# Pauli term: x = qubits with X or Y, z = qubits with Z or Y, coef real.
TERM_DTYPE = np.dtype({
    "names": ["x", "z", "coef"],
    "formats": ["<u8", "<u8", "<f8"],
    "offsets": [0, 8, 16],
    "itemsize": 24,
})

OP = dict(
    ID=0, X=1, Y=2, Z=3, H=4, S=5, SDG=6, T=7, TDG=8, RX=9, RY=10, RZ=11, U1=12, U2=13,
    U3=14, C1=15,
    CX=32, CY=33, CZ=34, CH=35, SWAP=36, CRX=37, CRY=38, CRZ=39, CU1=40, CU3=41, RXX=42,
    RZZ=43, C2=44,
    MEASURE=64, RESET=65, BARRIER=66,
)
OP_NAME = {v: k for k, v in OP.items()}
ONE_QUBIT = [OP[k] for k in ("ID", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "RX", "RY",
                             "RZ", "U1", "U2", "U3")]
TWO_QUBIT = [OP[k] for k in ("CX", "CY", "CZ", "CH", "SWAP", "CRX", "CRY", "CRZ", "CU1", "CU3",
                             "RXX", "RZZ")]
N_PARAMS = {OP["RX"]: 1, OP["RY"]: 1, OP["RZ"]: 1, OP["U1"]: 1, OP["U2"]: 2, OP["U3"]: 3,
            OP["CRX"]: 1, OP["CRY"]: 1, OP["CRZ"]: 1, OP["CU1"]: 1, OP["CU3"]: 3,
            OP["RXX"]: 1, OP["RZZ"]: 1}
MEAS_ASSERT = 1


def records(rows) -> np.ndarray:
    """rows: iterable of (op, q0, q1, p0, p1, p2[, flags[, mat]]) -> gate records."""
    rows = list(rows)
    g = np.zeros(len(rows), dtype=GATE_DTYPE)
    for i, r in enumerate(rows):
        g[i]["op"] = r[0]
        g[i]["q0"] = r[1]
        g[i]["q1"] = r[2]
        g[i]["p"] = (r[3], r[4], r[5])
        if len(r) > 6:
            g[i]["flags"] = r[6]
        if len(r) > 7:
            g[i]["mat"] = r[7]
    return g


def from_columns(op, q0, q1, p0, flags=None) -> np.ndarray:
    g = np.zeros(len(op), dtype=GATE_DTYPE)
    g["op"] = op
    g["q0"] = q0
    g["q1"] = q1
    g["p"][:, 0] = p0
    if flags is not None:
        g["flags"] = flags
    return g


# ---------------------------------------------------------- Pauli gadgets ----
def gadget_rows(support, letters, theta):
    """Gate rows of exp(-i theta P) for P = prod letters[j] on support[j]."""
    rows = []
    for q, L in zip(support, letters):
        if L == "X":
            rows.append((OP["H"], q, 0, 0.0))
        elif L == "Y":
            rows.append((OP["RX"], q, 0, math.pi / 2))
    for a, b in zip(support[:-1], support[1:]):
        rows.append((OP["CX"], a, b, 0.0))
    rows.append((OP["RZ"], support[-1], 0, 2.0 * theta))
    for a, b in reversed(list(zip(support[:-1], support[1:]))):
        rows.append((OP["CX"], a, b, 0.0))
    for q, L in zip(support, letters):
        if L == "X":
            rows.append((OP["H"], q, 0, 0.0))
        elif L == "Y":
            rows.append((OP["RX"], q, 0, -math.pi / 2))
    return rows


def gadget(support, letters, theta) -> np.ndarray:
    rows = gadget_rows(support, letters, theta)
    return from_columns([r[0] for r in rows], [r[1] for r in rows], [r[2] for r in rows],
                        [r[3] for r in rows])


def pauli_masks(support, letters):
    x = z = 0
    for q, L in zip(support, letters):
        if L in "XY":
            x |= 1 << q
        if L in "ZY":
            z |= 1 << q
    return x, z


def random_pauli(rng, n, w_lo, w_hi):
    w = int(rng.integers(w_lo, w_hi + 1))
    w = min(w, n)
    support = sorted(int(q) for q in rng.choice(n, size=w, replace=False))
    letters = "".join("XYZ"[int(i)] for i in rng.integers(0, 3, size=w))
    return support, letters


def _theta(rng, dist, size=None):
    if dist == "uniform":
        return rng.uniform(-math.pi, math.pi, size=size)
    if dist == "normal0.1":
        return rng.normal(0.0, 0.1, size=size)
    raise ValueError(dist)


class Circuit:
    """Gate records plus what the generator knows about them."""

    def __init__(self, n, gates, mats=None, **meta):
        self.n = n
        self.gates = gates
        self.mats = np.zeros(1) if mats is None else mats
        self.meta = meta

    @property
    def G(self):
        return int(self.gates.size)


def ucc_circuit(n, *, seed, n_gadgets=None, w_lo=2, w_hi=4, theta="uniform",
                target_gates=None, n_meas=0, meas_mode=0, meas_reset=False,
                meas_qubit=None, thetas=None) -> Circuit:
    """Seeded UCC-style circuit.

    n_gadgets given: that many random gadgets form one Trotter step, repeated
    (same angles) until target_gates is reached; the stream stops at the end of
    the gadget that crosses the target (the gate count is the authoritative
    size; the step count is recorded).  n_gadgets None: fresh gadgets are drawn
    until target_gates is reached.  n_meas MEASURE records are placed at gadget
    boundaries drawn uniformly without replacement, on uniform qubits (or on
    meas_qubit), each optionally followed by a RESET of the same qubit.
    thetas overrides the drawn angles of the gadget set (parameter sweeps over
    one circuit structure).
    """
    rng = np.random.default_rng(seed)
    ops, q0s, q1s, ps, bounds = [], [], [], [], []
    paulis = []

    def emit(support, letters, th):
        for r in gadget_rows(support, letters, th):
            ops.append(r[0]); q0s.append(r[1]); q1s.append(r[2]); ps.append(r[3])
        bounds.append(len(ops))

    if n_gadgets is not None:
        set_paulis = [random_pauli(rng, n, w_lo, w_hi) for _ in range(n_gadgets)]
        th = _theta(rng, theta, size=n_gadgets)
        if thetas is not None:
            th = np.asarray(thetas, dtype=np.float64)
        for (s, L), t in zip(set_paulis, th):
            emit(s, L, float(t))
            paulis.append((s, L, float(t)))
        step = from_columns(ops, q0s, q1s, ps)
        step_bounds = np.asarray(bounds, dtype=np.int64)
        if target_gates is None or target_gates <= step.size:
            reps = 1
        else:
            reps = -(-target_gates // step.size)
        gates = np.tile(step, reps)
        all_bounds = (step_bounds[None, :] + step.size * np.arange(reps)[:, None]).ravel()
        if target_gates is not None and target_gates < gates.size:
            cut_idx = int(np.searchsorted(all_bounds, target_gates))
            cut = int(all_bounds[min(cut_idx, all_bounds.size - 1)])
            gates = gates[:cut]
            all_bounds = all_bounds[: cut_idx + 1]
        steps = gates.size / step.size
    else:
        assert target_gates is not None
        while len(ops) < target_gates:
            s, L = random_pauli(rng, n, w_lo, w_hi)
            t = float(_theta(rng, theta))
            emit(s, L, t)
            paulis.append((s, L, t))
        gates = from_columns(ops, q0s, q1s, ps)
        all_bounds = np.asarray(bounds, dtype=np.int64)
        steps = 1.0

    meas_pos = np.zeros(0, dtype=np.int64)
    meas_q = np.zeros(0, dtype=np.int64)
    if n_meas:
        mrng = np.random.default_rng(seed + 1_000_003)
        inner = all_bounds[:-1] if all_bounds.size > 1 else all_bounds
        meas_pos = np.sort(mrng.choice(inner, size=min(n_meas, inner.size), replace=False))
        if meas_qubit is None:
            meas_q = mrng.integers(0, n, size=meas_pos.size)
        else:
            meas_q = np.full(meas_pos.size, meas_qubit)
        recs = [np.zeros(1, dtype=GATE_DTYPE) for _ in range(meas_pos.size)]
        ins = []
        for i, (pos, q) in enumerate(zip(meas_pos, meas_q)):
            m = np.zeros(2 if meas_reset else 1, dtype=GATE_DTYPE)
            m[0]["op"] = OP["MEASURE"]
            m[0]["q0"] = q
            m[0]["flags"] = meas_mode
            if meas_reset:
                m[1]["op"] = OP["RESET"]
                m[1]["q0"] = q
            recs[i] = m
            ins.append(pos)
        pieces, prev = [], 0
        for pos, m in zip(ins, recs):
            pieces.append(gates[prev:pos])
            pieces.append(m)
            prev = pos
        pieces.append(gates[prev:])
        gates = np.concatenate(pieces)

    return Circuit(n, gates, None, seed=seed, steps=steps, n_meas=int(meas_pos.size),
                   meas_qubits=meas_q.tolist(), paulis=paulis if len(paulis) < 5000 else None,
                   n_gadgets_total=int(all_bounds.size))


# ------------------------------------------------------ closed-form cases ----
def ghz_circuit(n) -> Circuit:
    rows = [(OP["H"], 0, 0, 0.0)] + [(OP["CX"], i, i + 1, 0.0) for i in range(n - 1)]
    return Circuit(n, from_columns(*zip(*rows)))


def qft_circuit(n, prep_index=0) -> Circuit:
    """X gates preparing |prep_index>, then the textbook QFT with the final
    qubit-reversal swaps: H on the highest qubit first, controlled phases
    CU1(pi/2^k), ..., then SWAP(i, n-1-i)."""
    rows = [(OP["X"], q, 0, 0.0) for q in range(n) if (prep_index >> q) & 1]
    for j in reversed(range(n)):
        rows.append((OP["H"], j, 0, 0.0))
        for k in reversed(range(j)):
            rows.append((OP["CU1"], k, j, math.pi / (1 << (j - k))))
    for i in range(n // 2):
        rows.append((OP["SWAP"], i, n - 1 - i, 0.0))
    return Circuit(n, from_columns(*zip(*rows)))


def random_circuit(n, G, *, seed, ops=None, with_generic=True) -> Circuit:
    """Random gates of every kind in the gate table (and generic C1/C2 records
    with random complex matrices) on random qubits; angles U(-pi, pi)."""
    rng = np.random.default_rng(seed)
    pool = list(ops) if ops is not None else ONE_QUBIT + (TWO_QUBIT if n >= 2 else [])
    if with_generic and ops is None:
        pool = pool + [OP["C1"]] + ([OP["C2"]] if n >= 2 else [])
    g = np.zeros(G, dtype=GATE_DTYPE)
    mats = []
    off = 0
    for i in range(G):
        op = int(pool[rng.integers(0, len(pool))])
        g[i]["op"] = op
        if op in TWO_QUBIT or op == OP["C2"]:
            a, b = rng.choice(n, size=2, replace=False)
            g[i]["q0"], g[i]["q1"] = int(a), int(b)
        else:
            g[i]["q0"] = int(rng.integers(0, n))
        g[i]["p"] = rng.uniform(-math.pi, math.pi, size=3)
        if op in (OP["C1"], OP["C2"]):
            d = 2 if op == OP["C1"] else 4
            m = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
            m /= np.sqrt(d)
            mats.append(m.astype(np.complex128).view(np.float64).ravel())
            g[i]["mat"] = off
            off += 2 * d * d
    mats_arr = np.concatenate(mats) if mats else np.zeros(1)
    return Circuit(n, g, mats_arr)


# ----------------------------------------------------------- Hamiltonians ----
def random_hamiltonian(n, n_terms, *, seed) -> np.ndarray:
    """n_terms Pauli strings, each letter uniform over {I,X,Y,Z} (the all-identity
    string redrawn), coef ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    t = np.zeros(n_terms, dtype=TERM_DTYPE)
    for i in range(n_terms):
        while True:
            letters = rng.integers(0, 4, size=n)
            if letters.any():
                break
        x = z = 0
        for q, L in enumerate(letters):
            if L in (1, 2):
                x |= 1 << q
            if L in (2, 3):
                z |= 1 << q
        t[i]["x"], t[i]["z"] = x, z
        t[i]["coef"] = rng.normal()
    return t


def z_terms(n) -> np.ndarray:
    t = np.zeros(n, dtype=TERM_DTYPE)
    for q in range(n):
        t[q]["z"] = 1 << q
        t[q]["coef"] = 1.0
    return t


def random_state(n, *, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


# ------------------------------------------------ the five workload shapes ----
def config_small(seed=1) -> Circuit:
    """8 qubits, 40 gadgets of weight 2-4, theta ~ U(-pi, pi), cycled to 2,000 gates."""
    return ucc_circuit(8, seed=seed, n_gadgets=40, w_lo=2, w_hi=4, theta="uniform",
                       target_gates=2000)


def config_mid(seed=2, n_meas=64, target_gates=1_000_000) -> Circuit:
    """16 qubits, 1e6 gates of fresh weight 2-8 gadgets, theta ~ N(0, 0.1), 64 measurements."""
    return ucc_circuit(16, seed=seed, n_gadgets=None, w_lo=2, w_hi=8, theta="normal0.1",
                       target_gates=target_gates, n_meas=n_meas)


def config_large(seed=3, target_gates=115_000_000, n_meas=8) -> Circuit:
    """21 qubits, one Trotter step of 2,000 weight 2-6 gadgets with theta ~ U(-pi, pi),
    cycled to 1.15e8 gates, with n_meas mid-circuit measurements (the paper's 21-qubit
    circuits carry 8 filtering measurements)."""
    return ucc_circuit(21, seed=seed, n_gadgets=2000, w_lo=2, w_hi=6, theta="uniform",
                       target_gates=target_gates, n_meas=n_meas)


def projection_filter(n_sys, *, seed, blocks=8, trotter=4, theta_scale=0.4) -> Circuit:
    """A synthetic projection filter in the shape of the paper's circuits: the
    system qubits 0..n_sys-1 start in the uniform superposition (H on each);
    each of `blocks` filter blocks puts the ancilla (qubit n_sys) in |+>, applies
    the controlled evolution exp(2i sum_j theta_j Z_j) on ancilla |1> as
    `trotter` slices of exp(-i (theta_j / trotter) Z_a Z_j) gadgets and
    RZ(-2 theta_j / trotter) on qubit j, closes with H on the ancilla, asserts
    the ancilla in |0> (assertion-mode measurement) and resets it.  The angles
    theta_j ~ theta_scale * U(-1, 1) are in meta["thetas"]."""
    rng = np.random.default_rng(seed)
    thetas = theta_scale * rng.uniform(-1.0, 1.0, size=n_sys)
    a = n_sys
    rows = [(OP["H"], q, 0, 0.0) for q in range(n_sys)]
    recs = [from_columns([r[0] for r in rows], [r[1] for r in rows], [r[2] for r in rows],
                         [r[3] for r in rows])]
    for _ in range(blocks):
        rows = [(OP["H"], a, 0, 0.0)]
        for _ in range(trotter):
            for j in range(n_sys):
                t = float(thetas[j]) / trotter
                rows += gadget_rows(sorted([j, a]), "ZZ", t)
                rows.append((OP["RZ"], j, 0, -2.0 * t))
        rows.append((OP["H"], a, 0, 0.0))
        recs.append(from_columns([r[0] for r in rows], [r[1] for r in rows], [r[2] for r in rows],
                                 [r[3] for r in rows]))
        m = np.zeros(2, dtype=GATE_DTYPE)
        m[0]["op"], m[0]["q0"], m[0]["flags"] = OP["MEASURE"], a, 1
        m[1]["op"], m[1]["q0"] = OP["RESET"], a
        recs.append(m)
    return Circuit(n_sys + 1, np.concatenate(recs), None, seed=seed, thetas=thetas, blocks=blocks,
                   trotter=trotter)


def config_batched(seed=4, n_param_sets=512, n_uneven=256, gates=20_000, n_terms=200,
                   n_set_gadgets=1600):
    """(i) n_param_sets parameter sets (theta ~ U(-pi, pi), set i drawn with seed
    seed + i) of one 12-qubit UCC-style circuit structure (n_set_gadgets weight
    2-6 gadgets, cycled to `gates`); (ii) n_uneven circuits of width uniform in
    10..18 with `gates` gates each.  One random n_terms-term Hamiltonian per
    instance (seed 10_000 + instance).  Returns (circuits, hamiltonians)."""
    circuits = []
    base = ucc_circuit(12, seed=seed, n_gadgets=n_set_gadgets, w_lo=2, w_hi=6, target_gates=gates)
    rz = np.flatnonzero(base.gates["op"] == OP["RZ"])  # one RZ(2 theta) per gadget, in order
    gadget_of_rz = np.arange(rz.size) % n_set_gadgets
    for i in range(n_param_sets):
        th = np.random.default_rng(seed + i).uniform(-math.pi, math.pi, size=n_set_gadgets)
        g = base.gates.copy()
        g["p"][rz, 0] = 2.0 * th[gadget_of_rz]
        circuits.append(Circuit(12, g, None, seed=seed, param_set=i))
    wrng = np.random.default_rng(seed + 77_777)
    widths = wrng.integers(10, 19, size=n_uneven)
    for j, n in enumerate(widths):
        circuits.append(ucc_circuit(int(n), seed=seed + 100_000 + j, n_gadgets=None, w_lo=2, w_hi=6,
                                    theta="uniform", target_gates=gates))
    hams = [random_hamiltonian(c.n, n_terms, seed=10_000 + k) for k, c in enumerate(circuits)]
    return circuits, hams
