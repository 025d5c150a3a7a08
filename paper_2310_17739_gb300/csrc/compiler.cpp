// compiler.cpp -- host compiler: gate matrices, fusion (paper, Section "Gate
// Fusion"), pass scheduling into shared-memory tiles, k-qubit block merging.
//
// Fusion follows the paper's four stages, realised in one streaming pass over
// the gate records (every merge is exact algebra, so the grouping only changes
// rounding):
//   stage 1  consecutive 1-qubit gates on one qubit are multiplied into one
//            pending 2x2 (C1);
//   stage 2  a 2-qubit gate absorbs the pending C1 of both its qubits
//            (backward absorption); a C1 left pending at a measurement, reset
//            or barrier (on any qubit), or at the end of the stream, is
//            absorbed forward into the last 2-qubit op on that qubit if no
//            other op touched the qubit since, else emitted as a C1;
//   stage 3  every 2-qubit matrix is expressed with its lower qubit as local
//            bit 0 (U(b,a) -> SWAP U(a,b) SWAP, done as a basis permutation of
//            the 4x4 rather than two extra SWAP gates);
//   stage 4  a 2-qubit gate whose two qubits were last touched by the same C2
//            (same pair, nothing in between on either wire) is multiplied into
//            it -- this also merges CX gates with control and target swapped.
#include "compiler.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace qsim {

namespace {

const double kPi = 3.14159265358979323846;

inline cd expi(double a) { return cd(std::cos(a), std::sin(a)); }

bool is_1q(int op) { return op >= QSIM_OP_ID && op <= QSIM_OP_C1; }
bool is_2q(int op) { return op >= QSIM_OP_CX && op <= QSIM_OP_C2; }
bool is_event(int op) {
    return op == QSIM_OP_MEASURE || op == QSIM_OP_RESET || op == QSIM_OP_BARRIER;
}

// 2x2 of the named one-qubit gates, row-major.
bool named_1q(int op, const double *p, cd *u) {
    const cd I(0, 1);
    const double r = std::sqrt(0.5);
    auto set = [&](cd a, cd b, cd c, cd d) { u[0] = a; u[1] = b; u[2] = c; u[3] = d; };
    switch (op) {
        case QSIM_OP_ID: set(1, 0, 0, 1); return true;
        case QSIM_OP_X: set(0, 1, 1, 0); return true;
        case QSIM_OP_Y: set(0, -I, I, 0); return true;
        case QSIM_OP_Z: set(1, 0, 0, -1); return true;
        case QSIM_OP_H: set(r, r, r, -r); return true;
        case QSIM_OP_S: set(1, 0, 0, I); return true;
        case QSIM_OP_SDG: set(1, 0, 0, -I); return true;
        case QSIM_OP_T: set(1, 0, 0, expi(kPi / 4)); return true;
        case QSIM_OP_TDG: set(1, 0, 0, expi(-kPi / 4)); return true;
        case QSIM_OP_RX: {
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            set(c, cd(0, -s), cd(0, -s), c);
            return true;
        }
        case QSIM_OP_RY: {
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            set(c, -s, s, c);
            return true;
        }
        case QSIM_OP_RZ: set(expi(-p[0] / 2), 0, 0, expi(p[0] / 2)); return true;
        case QSIM_OP_U1: set(1, 0, 0, expi(p[0])); return true;
        case QSIM_OP_U2:
        case QSIM_OP_U3: {
            double t = op == QSIM_OP_U2 ? kPi / 2 : p[0];
            double ph = op == QSIM_OP_U2 ? p[0] : p[1];
            double la = op == QSIM_OP_U2 ? p[1] : p[2];
            double c = std::cos(t / 2), s = std::sin(t / 2);
            set(c, -expi(la) * s, expi(ph) * s, expi(ph + la) * c);
            return true;
        }
        default: return false;
    }
}

// 4x4 of the named two-qubit gates in basis l = b_q0 + 2 b_q1.
bool named_2q(int op, const double *p, cd *m) {
    for (int i = 0; i < 16; i++) m[i] = 0;
    int target_op = -1;
    switch (op) {
        case QSIM_OP_CX: target_op = QSIM_OP_X; break;
        case QSIM_OP_CY: target_op = QSIM_OP_Y; break;
        case QSIM_OP_CZ: target_op = QSIM_OP_Z; break;
        case QSIM_OP_CH: target_op = QSIM_OP_H; break;
        case QSIM_OP_CRX: target_op = QSIM_OP_RX; break;
        case QSIM_OP_CRY: target_op = QSIM_OP_RY; break;
        case QSIM_OP_CRZ: target_op = QSIM_OP_RZ; break;
        case QSIM_OP_CU1: target_op = QSIM_OP_U1; break;
        case QSIM_OP_CU3: target_op = QSIM_OP_U3; break;
        default: break;
    }
    if (target_op >= 0) {
        cd u[4];
        named_1q(target_op, p, u);
        // control = local bit 0; control 0 -> identity on the target bit.
        m[0 * 4 + 0] = 1;
        m[2 * 4 + 2] = 1;
        m[1 * 4 + 1] = u[0];
        m[1 * 4 + 3] = u[1];
        m[3 * 4 + 1] = u[2];
        m[3 * 4 + 3] = u[3];
        return true;
    }
    switch (op) {
        case QSIM_OP_SWAP:
            m[0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[15] = 1;
            return true;
        case QSIM_OP_RXX: {
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            for (int l = 0; l < 4; l++) {
                m[l * 4 + l] = c;
                m[l * 4 + (3 - l)] = cd(0, -s);
            }
            return true;
        }
        case QSIM_OP_RZZ:
            m[0] = expi(-p[0] / 2);
            m[5] = expi(p[0] / 2);
            m[10] = expi(p[0] / 2);
            m[15] = expi(-p[0] / 2);
            return true;
        default: return false;
    }
}

// Matrix helpers on row-major 2^k x 2^k arrays.
// Left-multiply by U (2x2) acting on local bit j: M <- (U on bit j) * M.
void left_1q(cd *M, int k, int j, const cd *U) {
    const int D = 1 << k, b = 1 << j;
    for (int r0 = 0; r0 < D; r0++) {
        if (r0 & b) continue;
        const int r1 = r0 | b;
        for (int c = 0; c < D; c++) {
            cd x0 = M[r0 * D + c], x1 = M[r1 * D + c];
            M[r0 * D + c] = U[0] * x0 + U[1] * x1;
            M[r1 * D + c] = U[2] * x0 + U[3] * x1;
        }
    }
}
// Right-multiply by U acting on local bit j: M <- M * (U on bit j).
void right_1q(cd *M, int k, int j, const cd *U) {
    const int D = 1 << k, b = 1 << j;
    for (int r = 0; r < D; r++) {
        for (int c0 = 0; c0 < D; c0++) {
            if (c0 & b) continue;
            const int c1 = c0 | b;
            cd y0 = M[r * D + c0], y1 = M[r * D + c1];
            M[r * D + c0] = y0 * U[0] + y1 * U[2];
            M[r * D + c1] = y0 * U[1] + y1 * U[3];
        }
    }
}
void matmul(const cd *A, const cd *B, cd *C, int D) {  // C = A * B
    for (int r = 0; r < D; r++)
        for (int c = 0; c < D; c++) {
            cd s = 0;
            for (int t = 0; t < D; t++) s += A[r * D + t] * B[t * D + c];
            C[r * D + c] = s;
        }
}
// Swap local bits 0 and 1 of a 4x4 (basis permutation P M P).
void swap_bits_4(cd *M) {
    static const int perm[4] = {0, 2, 1, 3};
    cd T[16];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) T[perm[r] * 4 + perm[c]] = M[r * 4 + c];
    std::memcpy(static_cast<void *>(M), T, sizeof(T));
}

// Expand a k-qubit matrix (qubits qs) into the u-qubit space us (qs subset of us).
void expand(const cd *M, int k, const uint32_t *qs, int u, const uint32_t *us, cd *E) {
    int pos[kMaxK];
    for (int j = 0; j < k; j++)
        for (int t = 0; t < u; t++)
            if (us[t] == qs[j]) pos[j] = t;
    uint32_t inmask = 0;
    for (int j = 0; j < k; j++) inmask |= 1u << pos[j];
    const int D = 1 << u, d = 1 << k;
    for (int r = 0; r < D; r++) {
        int lr = 0;
        for (int j = 0; j < k; j++) lr |= ((r >> pos[j]) & 1) << j;
        for (int c = 0; c < D; c++) {
            if ((r & ~inmask) != (c & ~inmask)) {
                E[r * D + c] = 0;
                continue;
            }
            int lc = 0;
            for (int j = 0; j < k; j++) lc |= ((c >> pos[j]) & 1) << j;
            E[r * D + c] = M[lr * d + lc];
        }
    }
}
// E (u-qubit, 2^u x 2^u) <- B(op on qubits qb) * E
void left_apply(cd *E, int u, const uint32_t *us, const cd *B, int kb, const uint32_t *qb) {
    int pos[kMaxK];
    for (int j = 0; j < kb; j++)
        for (int t = 0; t < u; t++)
            if (us[t] == qb[j]) pos[j] = t;
    uint32_t bmask = 0;
    for (int j = 0; j < kb; j++) bmask |= 1u << pos[j];
    const int D = 1 << u, d = 1 << kb;
    cd x[1 << kMaxK], y[1 << kMaxK];
    int off[1 << kMaxK];
    for (int l = 0; l < d; l++) {
        int o = 0;
        for (int j = 0; j < kb; j++) o |= ((l >> j) & 1) << pos[j];
        off[l] = o;
    }
    for (int c = 0; c < D; c++) {
        for (int r0 = 0; r0 < D; r0++) {
            if (r0 & bmask) continue;
            for (int l = 0; l < d; l++) x[l] = E[(r0 | off[l]) * D + c];
            for (int a = 0; a < d; a++) {
                cd s = 0;
                for (int b = 0; b < d; b++) s += B[a * d + b] * x[b];
                y[a] = s;
            }
            for (int l = 0; l < d; l++) E[(r0 | off[l]) * D + c] = y[l];
        }
    }
}

int popc(uint64_t x) { return __builtin_popcountll(x); }

// ---------------------------------------------------- Pauli-gadget blocks --
// A block  B_q (1-qubit gates per qubit) ; F (CX network) ; RZ(phi) on t ;
// F reversed ; B_q^dagger  equals  B^dag F^dag exp(-i phi/2 Z_t) F B
// = exp(-i phi/2 * B^dag Z_S B)  with S the set of qubits whose bits F XORs
// into t (F^dag Z_t F = Z_S for a CX network).  Each B_q^dag Z B_q must be a
// signed Pauli; the product of the signs goes into the angle.
struct Gadget {
    size_t len = 0;
    uint64_t xm = 0, zm = 0;
    double theta = 0;
};

bool is_basis_gate(const qsim_gate &g) {
    switch (g.op) {
        case QSIM_OP_H: case QSIM_OP_S: case QSIM_OP_SDG: case QSIM_OP_X: case QSIM_OP_Y:
        case QSIM_OP_Z: case QSIM_OP_RX: case QSIM_OP_RY: case QSIM_OP_U2: case QSIM_OP_U3:
            return true;
        default: return false;
    }
}

// |z| > tol, decided as std::abs(z) > tol is (std::abs rounds faithfully),
// without its square root in the clear cases: |z| >= max(|re|, |im|), and
// |z| <= |re| + |im|, which is below tol when that sum is at most tol / 2.
inline bool exceeds(cd z, double tol) {
    const double a = std::fabs(z.real()), b = std::fabs(z.imag());
    if (a > tol || b > tol) return true;
    if (a + b <= 0.5 * tol) return false;
    return std::abs(z) > tol;
}

// Which signed Pauli U^dag Z U is: 1=X, 2=Y, 3=Z (sign in *sgn), 0 = none.
int conj_z(const cd *U, int *sgn) {
    // V = U^dag Z U
    cd V[4];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) V[r * 2 + c] = std::conj(U[0 * 2 + r]) * U[0 * 2 + c] - std::conj(U[1 * 2 + r]) * U[1 * 2 + c];
    const double tol = 1e-12;
    auto near = [&](const cd *P, double s) {
        for (int i = 0; i < 4; i++)
            if (exceeds(V[i] - s * P[i], tol)) return false;
        return true;
    };
    static const cd X[4] = {0, 1, 1, 0}, Y[4] = {0, cd(0, -1), cd(0, 1), 0}, Z[4] = {1, 0, 0, -1};
    const cd *P[3] = {X, Y, Z};
    for (int p = 0; p < 3; p++)
        for (int s = -1; s <= 1; s += 2)
            if (near(P[p], s)) {
                *sgn = s;
                return p + 1;
            }
    return 0;
}

// A basis change of a gadget on one qubit: its leading product U_lead and
// trailing product U_trail.  undone: U_trail U_lead == I (within 1e-12);
// letter, sign: U_lead^dag Z U_lead as conj_z gives them.
struct BasisChange {
    bool undone = false;
    int letter = 0, sign = 1;
};

void eval_basis_change(const cd *B, const cd *A, BasisChange &bc) {  // B = U_lead, A = U_trail
    cd P[4] = {A[0] * B[0] + A[1] * B[2], A[0] * B[1] + A[1] * B[3],
               A[2] * B[0] + A[3] * B[2], A[2] * B[1] + A[3] * B[3]};
    bc.undone = !(exceeds(P[0] - 1.0, 1e-12) || exceeds(P[1], 1e-12) || exceeds(P[2], 1e-12) ||
                  exceeds(P[3] - 1.0, 1e-12));
    bc.sign = 1;
    bc.letter = conj_z(B, &bc.sign);
}

// The product of the 1-qubit gates idx[0..cnt) that act on qubit q, later
// gates on the left; false if one has no 2x2 matrix.
bool gate_product(const qsim_gate *g, const size_t *idx, size_t cnt, uint32_t q, const double *mats,
                  size_t nm, cd *U) {
    bool first = true;
    for (size_t e = 0; e < cnt; e++) {
        if (g[idx[e]].q0 != q) continue;
        cd m[16];
        if (gate_matrix(g[idx[e]], mats, nm, m) != 2) return false;
        if (first) {
            for (int k = 0; k < 4; k++) U[k] = m[k];
            first = false;
        } else {
            cd r[4] = {m[0] * U[0] + m[1] * U[2], m[0] * U[1] + m[1] * U[3],
                       m[2] * U[0] + m[3] * U[2], m[2] * U[1] + m[3] * U[3]};
            for (int k = 0; k < 4; k++) U[k] = r[k];
        }
    }
    return true;
}

// BasisChange of one leading and one trailing named gate.  Gadgets repeat a
// few such pairs (H ... H, RX(pi/2) ... RX(-pi/2)), so each thread keeps the
// results of recent pairs, keyed by the two records' op codes and parameters
// (the matrices depend on nothing else); false if a gate has no 2x2 matrix.
bool basis_change(const qsim_gate &lead, const qsim_gate &trail, const double *mats, size_t nm,
                  BasisChange &bc) {
    struct Entry {
        bool used = false;
        uint16_t lop = 0, top = 0;
        double lp[3], tp[3];
        BasisChange bc;
    };
    if (lead.op == QSIM_OP_C1 || trail.op == QSIM_OP_C1) {  // a matrix from `mats`: not keyed by the record
        cd Ul[16], Ut[16];
        if (gate_matrix(lead, mats, nm, Ul) != 2 || gate_matrix(trail, mats, nm, Ut) != 2) return false;
        eval_basis_change(Ul, Ut, bc);
        return true;
    }
    constexpr int kEntries = 64;
    thread_local Entry memo[kEntries];
    uint64_t h = (uint64_t)lead.op * 0x9E3779B97F4A7C15ull ^ (uint64_t)trail.op * 0xC2B2AE3D27D4EB4Full;
    for (int k = 0; k < 3; k++) {
        uint64_t a, b;
        std::memcpy(&a, &lead.p[k], 8);
        std::memcpy(&b, &trail.p[k], 8);
        h = (h ^ a) * 0x100000001B3ull;
        h = (h ^ b) * 0x100000001B3ull;
    }
    Entry &e = memo[(h >> 32) % kEntries];
    if (e.used && e.lop == lead.op && e.top == trail.op && std::memcmp(e.lp, lead.p, sizeof(e.lp)) == 0 &&
        std::memcmp(e.tp, trail.p, sizeof(e.tp)) == 0) {
        bc = e.bc;
        return true;
    }
    cd Ul[16], Ut[16];
    if (gate_matrix(lead, mats, nm, Ul) != 2 || gate_matrix(trail, mats, nm, Ut) != 2) return false;
    eval_basis_change(Ul, Ut, bc);
    e.used = true;
    e.lop = lead.op;
    e.top = trail.op;
    std::memcpy(e.lp, lead.p, sizeof(e.lp));
    std::memcpy(e.tp, trail.p, sizeof(e.tp));
    e.bc = bc;
    return true;
}

bool match_gadget(int n, const qsim_gate *g, size_t i, size_t end, const double *mats, size_t nm,
                  Gadget &out) {
    (void)n;
    constexpr size_t kMaxLead = 16;
    size_t j = i;
    uint64_t lead_mask = 0;
    size_t lead[kMaxLead];  // gate indices of the leading 1-qubit gates
    size_t nl = 0;
    while (j < end && nl < kMaxLead && is_basis_gate(g[j])) {
        lead[nl++] = j;
        lead_mask |= 1ull << g[j].q0;
        j++;
    }
    // CX network
    const size_t f0 = j;
    while (j < end && g[j].op == QSIM_OP_CX) j++;
    const size_t f1 = j;
    if (f1 == f0 || j >= end || g[j].op != QSIM_OP_RZ) return false;
    const uint32_t t = g[j].q0;
    const double phi = g[j].p[0];
    j++;
    const size_t nf = f1 - f0;
    if (j + nf > end) return false;
    for (size_t k = 0; k < nf; k++) {
        const qsim_gate &a = g[f1 - 1 - k], &b = g[j + k];
        if (b.op != QSIM_OP_CX || b.q0 != a.q0 || b.q1 != a.q1) return false;
    }
    j += nf;
    // parity set: bits XORed into t by the network
    uint64_t rowmask[64];  // only the touched qubits' entries are read
    uint64_t touched = 1ull << t;
    for (size_t k = f0; k < f1; k++) touched |= (1ull << g[k].q0) | (1ull << g[k].q1);
    for (uint64_t r = touched; r; r &= r - 1) rowmask[__builtin_ctzll(r)] = r & -r;
    for (size_t k = f0; k < f1; k++) rowmask[g[k].q1] ^= rowmask[g[k].q0];
    const uint64_t S = rowmask[t];
    if (popc(S) < 2) return false;
    // one slot per basis-changed qubit (at most kMaxLead), with its leading
    // and trailing gates (their matrices are formed only when needed)
    int8_t slot[64];
    std::memset(slot, -1, sizeof(slot));
    int nlead[kMaxLead] = {0}, ntrail[kMaxLead] = {0};
    size_t first_lead[kMaxLead], first_trail[kMaxLead];
    int n_slots = 0;
    for (size_t e0 = 0; e0 < nl; e0++) {
        const uint32_t q = g[lead[e0]].q0;
        if (slot[q] < 0) {
            slot[q] = (int8_t)n_slots;
            first_lead[n_slots++] = lead[e0];
        }
        nlead[slot[q]]++;
    }
    // trailing: as many 1-qubit gates per qubit as the lead had, undoing it
    size_t trail[kMaxLead];
    size_t nt = 0, need = nl;
    while (need > 0) {
        if (j >= end || !is_basis_gate(g[j])) return false;
        const uint32_t q = g[j].q0;
        if (!((lead_mask >> q) & 1)) return false;
        const int sq = slot[q];
        if (ntrail[sq] >= nlead[sq]) return false;
        if (ntrail[sq] == 0) first_trail[sq] = j;
        trail[nt++] = j;
        ntrail[sq]++;
        need--;
        j++;
    }
    // trail * lead == I on every basis-changed qubit, letters from U^dag Z U
    uint64_t xm = 0, zm = 0;
    int sign = 1;
    for (uint64_t r = lead_mask | S; r; r &= r - 1) {
        const int q = __builtin_ctzll(r);
        const bool inS = (S >> q) & 1;
        const int sq = slot[q];
        int letter = 3, s = 1;
        if (sq >= 0) {
            BasisChange bc;
            if (nlead[sq] == 1) {
                if (!basis_change(g[first_lead[sq]], g[first_trail[sq]], mats, nm, bc)) return false;
            } else {
                cd Ul[4], Ut[4];
                if (!gate_product(g, lead, nl, (uint32_t)q, mats, nm, Ul) ||
                    !gate_product(g, trail, nt, (uint32_t)q, mats, nm, Ut))
                    return false;
                eval_basis_change(Ul, Ut, bc);
            }
            if (!bc.undone) return false;
            letter = bc.letter;
            s = bc.sign;
        }
        if (!inS) continue;
        if (!letter) return false;
        sign *= s;
        if (letter == 1 || letter == 2) xm |= 1ull << q;
        if (letter == 2 || letter == 3) zm |= 1ull << q;
    }
    out.len = j - i;
    out.xm = xm;
    out.zm = zm;
    out.theta = sign * phi / 2;
    return true;
}

}  // namespace

// ------------------------------------------------------------------ config --
Config config_from(const qsim_config *c) {
    Config k;
    if (!c) return k;
    k.fusion = c->fusion;
    k.k_max = c->k_max;
    k.tile_bits = c->tile_bits;
    k.threads = c->threads;
    k.chunk_gates = c->chunk_gates;
    k.lookahead = c->lookahead;
    k.compile_threads = c->compile_threads;
    k.persistent = c->persistent;
    k.graphs = c->graphs;
    k.forced_low = c->forced_low;
    return k;
}

void config_to(const Config &c, qsim_config *o) {
    std::memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(qsim_config);
    o->fusion = c.fusion;
    o->k_max = c.k_max;
    o->tile_bits = c.tile_bits;
    o->threads = c.threads;
    o->chunk_gates = c.chunk_gates;
    o->lookahead = c.lookahead;
    o->compile_threads = c.compile_threads;
    o->persistent = c.persistent;
    o->graphs = c.graphs;
    o->forced_low = c.forced_low;
}

static int max_tile_bits(qsim_dtype dt) { return dt == QSIM_C64 ? 14 : 13; }

int tile_bits_for(const Config &cfg, int n, qsim_dtype dtype) {
    const int mx = max_tile_bits(dtype);
    int m = cfg.tile_bits;
    if (m <= 0) {
        // Resident (whole state in one block) for small states.  Complex64
        // rotation passes (register segments) run fastest on 12-dimensional
        // tiles from 16 qubits up (measured on one GB300 for 12-22 qubits:
        // 16q 18.2 vs 13.8 M gates/s at m = 10, 21q 12.0 vs 11.4 at m = 13,
        // 22q 7.1 vs 5.5 at m = 14) and on 10-11-dimensional ones below;
        // complex128 rotation passes at most 12 (two blocks per SM: 1.30 vs 1.21
        // M gates/s at 21q, m = 12 vs 13); other passes take the largest tile
        // that still leaves >= 256 tiles to spread over 152 SMs.
        if (n <= 10) return n;
        if (dtype == QSIM_C64 && cfg.fusion == 2) m = std::max(10, std::min(12, n - 4));
        else if (cfg.fusion == 2) m = std::max(10, std::min(12, n - 8));
        else m = std::max(10, std::min(mx, n - 8));
    }
    m = std::min(m, mx);
    m = std::min(m, n);
    return std::max(m, 1);
}

int forced_low_bits(qsim_dtype dtype, int m, int requested) {
    int L = requested > 0 ? requested : (dtype == QSIM_C64 ? 4 : 3);  // 16 x 8 B or 8 x 16 B
    L = std::max(L, m - 10);
    return std::min(L, m);
}

// ------------------------------------------------------------------ matrices --
int gate_matrix(const qsim_gate &g, const double *mats, size_t n_mats, cd *out) {
    if (g.op == QSIM_OP_C1 || g.op == QSIM_OP_C2) {
        const int d = g.op == QSIM_OP_C1 ? 2 : 4;
        if (!mats || (size_t)g.mat + 2 * d * d > n_mats) return -1;
        for (int i = 0; i < d * d; i++) out[i] = cd(mats[g.mat + 2 * i], mats[g.mat + 2 * i + 1]);
        return d;
    }
    if (is_1q(g.op)) return named_1q(g.op, g.p, out) ? 2 : -1;
    if (is_2q(g.op)) return named_2q(g.op, g.p, out) ? 4 : -1;
    if (is_event(g.op)) return 0;
    return -1;
}

bool validate(int n, const qsim_gate *g, size_t n_gates, const double *mats, size_t n_mats,
              std::string &err) {
    for (size_t i = 0; i < n_gates; i++) {
        const qsim_gate &x = g[i];
        const int op = x.op;
        bool ok = true;
        if (is_1q(op) || op == QSIM_OP_MEASURE || op == QSIM_OP_RESET) {
            ok = x.q0 < (uint32_t)n;
        } else if (is_2q(op)) {
            ok = x.q0 < (uint32_t)n && x.q1 < (uint32_t)n && x.q0 != x.q1;
        } else if (op != QSIM_OP_BARRIER) {
            ok = false;
        }
        if (ok && (op == QSIM_OP_C1 || op == QSIM_OP_C2)) {
            const size_t need = op == QSIM_OP_C1 ? 8 : 32;
            ok = mats != nullptr && (size_t)x.mat + need <= n_mats;
        }
        if (ok && !is_event(op)) {
            for (int j = 0; j < 3; j++) ok = ok && std::isfinite(x.p[j]);
        }
        if (!ok) {
            err = "malformed gate record " + std::to_string(i) + " (op " + std::to_string(op) +
                  ", q0 " + std::to_string(x.q0) + ", q1 " + std::to_string(x.q1) + ")";
            return false;
        }
    }
    return true;
}

// -------------------------------------------------------------------- fusion --
void fuse(int n, const qsim_gate *g, size_t n_gates, const double *mats, size_t n_mats,
          int fusion, std::vector<FOp> &ops, std::vector<cd> &pool, uint64_t *n_meas,
          int max_rotation_qubits) {
    ops.clear();
    pool.clear();
    ops.reserve(n_gates / 2 + 16);
    pool.reserve(n_gates * 8 + 64);
    uint64_t meas = 0;
    std::vector<cd> pend(4 * (size_t)n);
    std::vector<char> has_pend(n, 0);
    std::vector<int64_t> open2(n, -1);  // last op on the qubit, if a C2 that can still absorb
    cd m[16], t[16];

    auto emit_mat = [&](int k, const uint32_t *qs, const cd *M) -> int64_t {
        FOp o;
        o.k = (uint8_t)k;
        for (int j = 0; j < k; j++) o.q[j] = qs[j];
        o.mat = pool.size();
        pool.insert(pool.end(), M, M + (1 << (2 * k)));
        ops.push_back(o);
        return (int64_t)ops.size() - 1;
    };
    auto flush = [&](int q) {
        if (!has_pend[q]) return;
        cd *U = &pend[4 * (size_t)q];
        const int64_t idx = open2[q];
        if (idx >= 0) {  // forward absorption into the last C2 on q
            FOp &o = ops[idx];
            const int j = o.q[0] == (uint32_t)q ? 0 : 1;
            left_1q(&pool[o.mat], 2, j, U);
        } else {
            uint32_t qs[1] = {(uint32_t)q};
            emit_mat(1, qs, U);
        }
        has_pend[q] = 0;
    };

    for (size_t i = 0; i < n_gates; i++) {
        const qsim_gate &x = g[i];
        const int op = x.op;
        if (fusion == 2 && (op == QSIM_OP_CX || is_basis_gate(x))) {
            Gadget gd;
            if (match_gadget(n, g, i, n_gates, mats, n_mats, gd) &&
                popc(gd.xm | gd.zm) <= max_rotation_qubits) {
                // gates pending on the rotation's qubits run before it; nothing
                // after it may be absorbed into an op before it
                const uint64_t sup = gd.xm | gd.zm;
                for (int q = 0; q < n; q++)
                    if ((sup >> q) & 1) {
                        flush(q);
                        open2[q] = -1;
                    }
                FOp o;
                o.k = kPauli;
                o.xm = gd.xm;
                o.zm = gd.zm;
                o.mat = pool.size();
                pool.push_back(cd(std::cos(gd.theta), std::sin(gd.theta)));
                ops.push_back(o);
                i += gd.len - 1;
                continue;
            }
        }
        if (is_event(op)) {
            FOp e;
            e.k = 0;
            e.ev = op == QSIM_OP_MEASURE ? EV_MEASURE : op == QSIM_OP_RESET ? EV_RESET : EV_BARRIER;
            e.flags = x.flags;
            e.q[0] = x.q0;
            // Every event is a fusion barrier on all qubits: no gate crosses a
            // measurement, so the state an event sees (and the state left by a
            // failed assertion) is the state of the unfused stream at that point.
            if (fusion) {
                for (int q = 0; q < n; q++) {
                    flush(q);
                    open2[q] = -1;
                }
            }
            if (op != QSIM_OP_BARRIER) meas++;
            ops.push_back(e);
            continue;
        }
        const int d = gate_matrix(x, mats, n_mats, m);
        if (d == 2) {
            const int q = (int)x.q0;
            if (!fusion) {
                uint32_t qs[1] = {(uint32_t)q};
                emit_mat(1, qs, m);
                continue;
            }
            cd *U = &pend[4 * (size_t)q];
            if (has_pend[q]) {  // stage 1: U <- m * U
                cd r[4] = {m[0] * U[0] + m[1] * U[2], m[0] * U[1] + m[1] * U[3],
                           m[2] * U[0] + m[3] * U[2], m[2] * U[1] + m[3] * U[3]};
                for (int j = 0; j < 4; j++) U[j] = r[j];
            } else {
                for (int j = 0; j < 4; j++) U[j] = m[j];
                has_pend[q] = 1;
            }
            continue;
        }
        // two-qubit gate; stage 3: lower qubit becomes local bit 0
        uint32_t p = x.q0, q = x.q1;
        if (p > q) {
            swap_bits_4(m);
            std::swap(p, q);
        }
        if (!fusion) {
            uint32_t qs[2] = {p, q};
            emit_mat(2, qs, m);
            continue;
        }
        // stage 2 (backward): absorb pending C1 on p (bit 0) and q (bit 1)
        if (has_pend[p]) { right_1q(m, 2, 0, &pend[4 * (size_t)p]); has_pend[p] = 0; }
        if (has_pend[q]) { right_1q(m, 2, 1, &pend[4 * (size_t)q]); has_pend[q] = 0; }
        const int64_t a = open2[p], b = open2[q];
        if (a >= 0 && a == b) {  // stage 4: same pair, nothing in between
            cd *M = &pool[ops[a].mat];
            matmul(m, M, t, 4);
            std::memcpy(static_cast<void *>(M), t, sizeof(t));
        } else {
            uint32_t qs[2] = {p, q};
            const int64_t idx = emit_mat(2, qs, m);
            open2[p] = open2[q] = idx;
        }
    }
    if (fusion)
        for (int q = 0; q < n; q++) flush(q);
    if (n_meas) *n_meas = meas;
}

// --------------------------------------------------------- k-qubit merging --
namespace {

double merge_cost(int k, qsim_dtype dt) {
    // Per-amplitude cost of one op in a shared-memory tile: one read+write
    // sweep (~16 FMA-equivalents of shared-memory bandwidth for c64) plus
    // 4 * 2^k FMAs (2^k complex multiply-adds).  FP64 FMAs are far slower than
    // FP32 ones on this part, so for c128 the arithmetic term dominates.
    const double alu = 4.0 * (1 << k);
    return dt == QSIM_C64 ? 16.0 + alu : 16.0 + 16.0 * alu;
}

size_t mat_entries(const FOp &o) { return o.pauli() ? 1 : ((size_t)1 << (2 * o.k)); }

void merge_pass(std::vector<FOp> &ops, std::vector<cd> &pool, size_t first, size_t count,
                int k_max, qsim_dtype dt, std::vector<FOp> &out) {
    if (count == 0) return;
    FOp cur = ops[first];
    std::vector<cd> curM(pool.begin() + cur.mat, pool.begin() + cur.mat + mat_entries(cur));
    std::vector<cd> E;
    auto flush = [&]() {
        cur.mat = pool.size();
        pool.insert(pool.end(), curM.begin(), curM.end());
        out.push_back(cur);
    };
    for (size_t i = first + 1; i < first + count; i++) {
        const FOp &o = ops[i];
        const uint64_t um = cur.mask() | o.mask();
        const int u = popc(um);
        // Pauli rotations are already cheaper than any dense block: never merged
        if (!cur.pauli() && !o.pauli() && u <= k_max &&
            merge_cost(u, dt) <= merge_cost(cur.k, dt) + merge_cost(o.k, dt)) {
            uint32_t us[kMaxK];
            int t = 0;
            for (int b = 0; b < 64; b++)
                if ((um >> b) & 1) us[t++] = (uint32_t)b;
            E.assign((size_t)1 << (2 * u), cd(0));
            expand(curM.data(), cur.k, cur.q, u, us, E.data());
            left_apply(E.data(), u, us, &pool[o.mat], o.k, o.q);
            cur.k = (uint8_t)u;
            for (int j = 0; j < u; j++) cur.q[j] = us[j];
            curM.swap(E);
        } else {
            flush();
            cur = o;
            curM.assign(pool.begin() + o.mat, pool.begin() + o.mat + mat_entries(o));
        }
    }
    flush();
}

}  // namespace

// ---------------------------------------------------------------- schedule --
namespace {

// Whether op o fits the tile subspace V within m dimensions (see Pass).
bool fits(const Subspace &V, const FOp &o, int m) {
    if (o.pauli()) return V.d < m || V.contains(o.xm);
    uint64_t r[kMaxK];
    int rank = 0;
    for (int j = 0; j < o.k; j++) {
        uint64_t v = V.reduce_unit((int)o.q[j]);
        for (int i = 0; i < rank; i++)
            if ((v >> __builtin_ctzll(r[i])) & 1) v ^= r[i];
        if (v) r[rank++] = v;
    }
    return V.d + rank <= m;
}

void take(Subspace &V, const FOp &o) {
    if (o.pauli()) {
        V.add(o.xm);
    } else {
        for (int j = 0; j < o.k; j++) V.add(1ull << o.q[j]);
    }
}

}  // namespace

void compile(int n, qsim_dtype dtype, const Config &cfg, const qsim_gate *g, size_t n_gates,
             const double *mats, size_t n_mats, HostProgram &out) {
    out = HostProgram();
    out.n = n;
    out.gates = n_gates;
    std::vector<FOp> ops;
    std::vector<cd> pool;
    const int m = tile_bits_for(cfg, n, dtype);
    // a rotation needs one tile dimension for its X mask, whatever its weight
    fuse(n, g, n_gates, mats, n_mats, cfg.fusion, ops, pool, &out.measurements, 64);

    out.m = m;
    out.resident = (m == n);
    const int L = forced_low_bits(dtype, m, cfg.forced_low);
    const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1);
    const size_t W = cfg.lookahead > 0 ? (size_t)cfg.lookahead : 64;
    const bool reg_candidate = dtype == QSIM_C64 && !out.resident && m >= 10 && m <= 14;
    const int k_max = std::max(2, std::min(cfg.k_max > 0 ? cfg.k_max : 2, std::min(5, m)));

    // Doubly linked list over not-yet-scheduled ops (in stream order).
    const size_t N = ops.size();
    std::vector<int64_t> nxt(N + 1), prv(N + 1);
    const int64_t HEAD = (int64_t)N;  // sentinel
    for (size_t i = 0; i < N; i++) {
        nxt[i] = (int64_t)i + 1 < (int64_t)N ? (int64_t)i + 1 : HEAD;
        prv[i] = i == 0 ? HEAD : (int64_t)i - 1;
    }
    nxt[HEAD] = N ? 0 : HEAD;
    prv[HEAD] = N ? (int64_t)N - 1 : HEAD;
    auto unlink = [&](int64_t i) {
        nxt[prv[i]] = nxt[i];
        prv[nxt[i]] = prv[i];
    };

    std::vector<FOp> sched;
    sched.reserve(N);
    std::vector<cd> spool;
    spool.reserve(pool.size());
    std::vector<size_t> taken;
    // the Pauli rotations skipped so far in a pass: support, X and Z masks
    struct SkippedPauli {
        uint64_t sup, x, z;
    };
    std::vector<SkippedPauli> skipped_pauli;

    // Pauli frame.  The state on the device is F^dagger times the circuit's
    // state, F = i^k X^x Z^z.  A rotation exp(-i theta P) reaches the device
    // as exp(-i s theta P), s = -1 when P anticommutes with F; one with
    // |cos theta| < |sin theta| is split as exp(-i (theta -+ pi/2) P) (-+ i P)
    // and the Pauli factor joins the frame (F <- F (-+ i P)), so every
    // rotation on the device has |cos| >= 1/sqrt(2).  A dense op U reaches it
    // as F^dagger U F (F restricted to its qubits).  Before a measurement or
    // reset, and at the end of the program, a flush op applies F to the state
    // (F = i^{k - y + 1} exp(-i pi/2 P_F), P_F = i^y X^x Z^z, y = |x & z|).
    struct Frame {
        uint64_t x = 0, z = 0;
        int k = 0;
        bool trivial() const { return !x && !z && !(k & 3); }
    } F;
    auto frame_apply = [&](FOp &c) {
        cd *M = &spool[c.mat];
        if (c.pauli()) {
            double cs = M[0].real(), sn = M[0].imag();
            if ((popc(F.x & c.zm) + popc(F.z & c.xm)) & 1) sn = -sn;
            if (std::fabs(cs) < std::fabs(sn)) {
                const int y = popc(c.xm & c.zm);
                int qk;
                if (sn > 0) {  // theta' = theta - pi/2, factor -iP = i^{3+y} X Z
                    const double t = cs;
                    cs = sn;
                    sn = -t;
                    qk = 3 + y;
                } else {       // theta' = theta + pi/2, factor iP = i^{1+y} X Z
                    const double t = cs;
                    cs = -sn;
                    sn = t;
                    qk = 1 + y;
                }
                F.k = (F.k + qk + 2 * popc(F.z & c.xm)) & 3;
                F.x ^= c.xm;
                F.z ^= c.zm;
            }
            M[0] = cd(cs, sn);
            return;
        }
        uint32_t a = 0, b = 0;
        for (int j = 0; j < c.k; j++) {
            a |= (uint32_t)((F.x >> c.q[j]) & 1) << j;
            b |= (uint32_t)((F.z >> c.q[j]) & 1) << j;
        }
        if (!a && !b) return;
        const int D = 1 << c.k;
        std::vector<cd> T(M, M + (size_t)D * D);
        for (int r = 0; r < D; r++)
            for (int q = 0; q < D; q++) {
                const cd v = T[(size_t)(r ^ a) * D + (q ^ a)];
                M[(size_t)r * D + q] = ((popc(b & r) + popc(b & q)) & 1) ? -v : v;
            }
    };
    auto frame_flush = [&]() {
        if (F.trivial()) return;
        FOp o;
        o.k = kPauli;
        o.xm = F.x;
        o.zm = F.z;
        o.flags = (uint16_t)(((F.k - popc(F.x & F.z) + 1) & 3) | kFrameFlush);
        Pass p;
        p.first = sched.size();
        p.count = 1;
        p.mat_first = spool.size();
        p.mat_count = 1;
        p.fpa = 8;
        p.basis = (uint32_t)out.bvec.size();
        if (out.resident) {
            p.tile = all;
            for (int b = 0; b < n; b++) out.bvec.push_back(1ull << b);
        } else {
            Subspace V;
            if (L < m)
                for (int b = 0; b < L; b++) V.add(1ull << b);
            if (F.x) V.add(F.x);
            for (int b = 0; b < n && V.d < m; b++) V.add(1ull << b);
            for (uint64_t b = V.pivots; b; b &= b - 1) out.bvec.push_back(V.vec[V.at[__builtin_ctzll(b)]]);
            p.tile = V.pivots;
        }
        o.mat = spool.size();
        spool.push_back(cd(0.0, 1.0));
        sched.push_back(o);
        out.passes.push_back(p);
        F = Frame();
    };

    while (nxt[HEAD] != HEAD) {
        const int64_t f = nxt[HEAD];
        if (ops[f].k == 0) {  // event: its own pass, never reordered
            unlink(f);
            if (ops[f].ev != EV_BARRIER) {
                frame_flush();
                Pass p;
                p.first = sched.size();
                p.count = 1;
                p.ev = ops[f].ev;
                p.flags = ops[f].flags;
                p.q = ops[f].q[0];
                sched.push_back(ops[f]);
                out.passes.push_back(p);
            }
            continue;
        }
        // An op may join the pass if the tile's subspace V can take it (see
        // Pass) within m dimensions and it commutes with every op skipped so
        // far (disjoint qubits, or two commuting Pauli rotations), so pulling
        // it ahead of them changes nothing.  V starts with the forced low
        // qubits (coalesced tile rows) unless the pass's first op would not
        // fit beside them.  A resident program's tile is the whole state.
        Subspace V;
        if (!out.resident) {
            for (int b = 0; b < L; b++) V.add(1ull << b);
            if (!fits(V, ops[f], m)) V = Subspace();
        }
        bool only_rot = true;
        uint64_t blocked_np = 0, blocked_p = 0;
        size_t skipped = 0, n_mats = 0;
        taken.clear();
        skipped_pauli.clear();
        for (int64_t i = f; i != HEAD && skipped < W;) {
            const int64_t ni = nxt[i];
            const FOp &o = ops[i];
            if (o.k == 0) break;  // events bound the scan
            // the tile kernel holds a pass's ops and coefficients in shared memory
            if (taken.size() >= (size_t)kTilePassOps ||
                n_mats + mat_entries(o) > (size_t)kTilePassMats)
                break;
            const uint64_t Q = o.mask();
            bool ok = (out.resident || fits(V, o, m)) && !(Q & blocked_np);
            // a complex64 rotation-only pass runs as register segments, which
            // hold a rotation whose tile coordinates span at most 5 bits: a
            // wider one (an X mask already in the span) waits for a later pass
            // (the pass's first op is always taken, so every pass makes progress)
            if (ok && i != f && reg_candidate && only_rot && o.pauli() && V.contains(o.xm) &&
                popc(V.coords(o.xm)) > 5)
                ok = false;
            if (ok && (Q & blocked_p)) {
                if (!o.pauli()) ok = false;
                else
                    for (const SkippedPauli &sp : skipped_pauli)  // as ops_commute
                        if ((Q & sp.sup) && ((popc(o.xm & sp.z) + popc(o.zm & sp.x)) & 1)) {
                            ok = false;
                            break;
                        }
            }
            if (ok) {
                if (!out.resident) take(V, o);
                only_rot = only_rot && o.pauli();
                taken.push_back((size_t)i);
                n_mats += mat_entries(o);
                unlink(i);
            } else {
                if (o.pauli()) {
                    blocked_p |= Q;
                    skipped_pauli.push_back({Q, o.xm, o.zm});
                } else {
                    blocked_np |= Q;
                }
                skipped++;
                if (popc(blocked_np) >= n) break;
            }
            i = ni;
        }
        // Pad V to exactly m dimensions with the lowest free unit vectors, and
        // record the basis: a rotation-only pass keeps the vectors in the
        // order they were added (each new rotation's X mask is one tile bit),
        // any other pass the row-echelon basis by ascending pivot (then a
        // qubit in V is the tile bit of its rank among the pivots).
        uint64_t T;
        const uint32_t bfirst = (uint32_t)out.bvec.size();
        if (out.resident) {
            T = all;
            for (int b = 0; b < n; b++) out.bvec.push_back(1ull << b);
        } else {
            for (int b = 0; b < n && V.d < m; b++) V.add(1ull << b);
            T = V.pivots;
            if (only_rot) {
                for (int j = 0; j < V.d; j++) out.bvec.push_back(V.added[j]);
            } else {
                // by ascending pivot
                for (uint64_t b = V.pivots; b; b &= b - 1) out.bvec.push_back(V.vec[V.at[__builtin_ctzll(b)]]);
            }
        }
        std::vector<FOp> body;
        body.reserve(taken.size());
        if (cfg.k_max > 2) {
            // merge in the pass's order into <= k_max-qubit dense blocks
            std::vector<FOp> tmp;
            tmp.reserve(taken.size());
            for (size_t t : taken) tmp.push_back(ops[t]);
            merge_pass(tmp, pool, 0, tmp.size(), k_max, dtype, body);
        } else {
            for (size_t t : taken) body.push_back(ops[t]);
        }
        // Emit as one pass, or as several consecutive passes over the same
        // tile when merged blocks exceed the per-pass coefficient budget.
        Pass p;
        auto open_pass = [&]() {
            p = Pass();
            p.tile = T;
            p.basis = bfirst;
            p.gadget = (uint8_t)(!out.resident && only_rot);
            p.first = sched.size();
            p.mat_first = spool.size();
        };
        auto close_pass = [&]() {
            p.count = (uint32_t)(sched.size() - p.first);
            p.mat_count = (uint32_t)(spool.size() - p.mat_first);
            for (size_t i = p.first; i < sched.size(); i++)
                p.fpa += sched[i].pauli() ? 8u : (8u << sched[i].k);  // a Pauli rotation: 2 complex MACs
            if (p.count) out.passes.push_back(p);
        };
        open_pass();
        for (const FOp &o : body) {
            const size_t e = mat_entries(o);
            if (sched.size() - p.first >= (size_t)kTilePassOps ||
                spool.size() - p.mat_first + e > (size_t)kTilePassMats) {
                close_pass();
                open_pass();
            }
            FOp c = o;
            c.mat = spool.size();
            spool.insert(spool.end(), pool.begin() + o.mat, pool.begin() + o.mat + e);
            frame_apply(c);
            sched.push_back(c);
        }
        close_pass();
    }
    frame_flush();
    for (const FOp &o : sched)
        if (o.k) out.hist[o.k]++;
    out.ops.swap(sched);
    out.pool.swap(spool);
}

}  // namespace qsim
