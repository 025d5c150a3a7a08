// compiler.h -- host-side gate-stream compiler: gate matrices, the four fusion
// stages of the paper's Section "Gate Fusion", k-qubit block merging, and the
// shared-memory pass schedule consumed by the sm_103a kernels.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {

using cd = std::complex<double>;

constexpr int kMaxK = 6;         // largest dense block (qubits)
constexpr int kMaxTileBits = 15; // largest shared-memory tile (qubits)

enum : uint8_t { EV_NONE = 0, EV_MEASURE = 1, EV_RESET = 2, EV_BARRIER = 3 };

// One fused operation.  k > 0: dense 2^k x 2^k matrix at pool[mat], bit j of
// the local matrix index <-> qubit q[j].  k == 0: an event (measure, reset,
// barrier) on qubit q[0] (barrier: all qubits).
//
// k == kPauli: a Pauli rotation exp(-i theta P) with P = i^{#Y} X^xm Z^zm on the
// qubits of xm | zm (Y = bit in both); pool[mat] = (cos theta, sin theta).
constexpr uint8_t kPauli = 7;
// FOp::flags of a Pauli op: bits 0-1 = g, the op is i^g exp(-i theta P) (g != 0
// only for a frame flush, whose cos theta is 0); bit 2 = frame flush.
constexpr uint16_t kPhaseMask = 3;
constexpr uint16_t kFrameFlush = 4;

struct FOp {
    uint8_t k = 0;
    uint8_t ev = EV_NONE;
    uint16_t flags = 0;
    uint32_t q[kMaxK] = {0, 0, 0, 0, 0, 0};
    uint64_t mat = 0;
    uint64_t xm = 0, zm = 0;  // Pauli rotations only
    bool pauli() const { return k == kPauli; }
    uint64_t mask() const {
        if (k == kPauli) return xm | zm;
        uint64_t m = 0;
        for (int j = 0; j < k; j++) m |= 1ull << q[j];
        return m;
    }
};

// Two ops may be reordered iff they act on disjoint qubits, or both are Pauli
// rotations whose Paulis commute (even symplectic product).
inline bool ops_commute(const FOp &a, const FOp &b) {
    if (!(a.mask() & b.mask())) return true;
    if (a.pauli() && b.pauli())
        return ((__builtin_popcountll(a.xm & b.zm) + __builtin_popcountll(a.zm & b.xm)) & 1) == 0;
    return false;
}

// A linear subspace of GF(2)^n (bit q <-> qubit q) in reduced row-echelon
// form: vec[i] has its lowest set bit at piv[i] and a zero at every other
// pivot, so v is in the subspace iff reduce(v) == 0, and the coordinates of a
// member are read off its pivot bits.  combo[i] is vec[i] written in the basis
// of the vectors that add() accepted, in their order (bit j = the j-th).
struct Subspace {
    static constexpr int kCap = 16;
    int d = 0;
    uint64_t pivots = 0;
    uint64_t vec[kCap];
    uint32_t combo[kCap];
    uint8_t piv[kCap];
    uint64_t added[kCap];  // the accepted vectors, in order
    uint8_t at[64];        // at[p]: the vector whose pivot is p (p in pivots)

    // Since every vector has a zero at every other vector's pivot, the
    // vectors v meets while it is reduced are fixed by v's own pivot bits:
    // XORing one of them clears its pivot bit and touches no other.
    uint64_t reduce(uint64_t v) const {
        for (uint64_t b = v & pivots; b; b &= b - 1) v ^= vec[at[__builtin_ctzll(b)]];
        return v;
    }
    bool contains(uint64_t v) const { return reduce(v) == 0; }
    // reduce(2^q): at most the vector whose pivot is q.
    uint64_t reduce_unit(int q) const {
        const uint64_t v = 1ull << q;
        return (pivots & v) ? v ^ vec[at[q]] : v;
    }
    // Adds v; returns false (and changes nothing) if v is already a member or
    // the capacity is reached.
    bool add(uint64_t v) {
        if (d >= kCap) return false;
        uint64_t r = v;
        uint32_t c = 1u << d;
        for (uint64_t b = v & pivots; b; b &= b - 1) {
            const int i = at[__builtin_ctzll(b)];
            r ^= vec[i];
            c ^= combo[i];
        }
        if (!r) return false;
        const int p = __builtin_ctzll(r);
        for (int i = 0; i < d; i++)
            if ((vec[i] >> p) & 1) {
                vec[i] ^= r;
                combo[i] ^= c;
            }
        vec[d] = r;
        combo[d] = c;
        piv[d] = (uint8_t)p;
        at[p] = (uint8_t)d;
        added[d] = v;
        pivots |= 1ull << p;
        d++;
        return true;
    }
    // Coordinates of a member v in the basis added[0..d): bit j <-> added[j].
    uint32_t coords(uint64_t v) const {
        uint32_t c = 0;
        for (uint64_t b = v & pivots; b; b &= b - 1) c ^= combo[at[__builtin_ctzll(b)]];
        return c;
    }
};

// A pass: full-state sweep over tiles applying ops [first, first+count) in
// order; or an event pass (tile == 0, count == 1).  A tile is a coset
// x0 + V of an m-dimensional subspace V: tile element t (m bits) is amplitude
// x0 ^ (XOR of basis[j] over the set bits j of t), with the tile's own x0
// spread over the positions that are not pivots of V.  A dense op needs the
// unit vector of each of its qubits in V (then that vector is a basis vector
// and the qubit is one tile bit); a Pauli rotation needs only its X mask in V
// (its Z part becomes a parity of the tile index and of x0).
struct Pass {
    uint64_t tile = 0;    // pivot positions of V (for unit-vector bases: the tile qubits)
    uint64_t first = 0;
    uint32_t count = 0;
    uint8_t ev = EV_NONE;
    uint8_t reg = 0;      // register segments (set when packed for the device): 1 rotations only,
                          // 2 with dense ops (RegDense)
    uint16_t flags = 0;   // event flags (bit 0: assertion mode)
    uint32_t q = 0;       // event qubit
    uint32_t fpa = 0;     // algorithmic real flops per amplitude of the pass (8 * 2^k per op)
    uint64_t mat_first = 0;  // the pass's coefficients: pool[mat_first, mat_first + mat_count)
    uint32_t mat_count = 0;
    uint32_t basis = 0;   // the pass's m basis vectors: bvec[basis, basis + m) of its program
    uint8_t gadget = 0;   // basis = X masks of its rotations in order (rotation-only pass);
                          // otherwise the reduced row-echelon basis, ascending pivots
    float scale = 1.0f;   // register-segment passes: product of the rotations' cosines
    double gscale = 1.0;  // generic passes: product of the cosines of the rotations in scaled form
};

// Per-pass limits of the tile kernel (its ops and coefficients are copied
// into shared memory next to the tile): ops, and complex coefficient values.
constexpr int kTilePassOps = 256;
constexpr int kTilePassMats = 1024;

struct Config {
    int fusion = 1;
    int k_max = 2;
    int tile_bits = 0;
    int threads = 0;
    int chunk_gates = 0;
    int lookahead = 0;
    int compile_threads = 0;
    int persistent = 0;
    int graphs = 0;
    int forced_low = 0;
};

Config config_from(const qsim_config *c);
void config_to(const Config &c, qsim_config *out);

// Tile size (qubits) used for an n-qubit state of this dtype.
int tile_bits_for(const Config &cfg, int n, qsim_dtype dtype);
// Qubits always kept in every tile so that tile rows are contiguous runs
// (default 128 bytes: 4 for complex64, 3 for complex128; `requested` > 0
// overrides), never fewer than m - 10 (the generic pass tabulates at most
// 1,024 row offsets).
int forced_low_bits(qsim_dtype dtype, int m, int requested = 0);

// Compiled host program: fused ops (with FP64 matrices) in execution order and
// the pass schedule over them.
struct HostProgram {
    int n = 0;
    int m = 0;                 // tile bits
    bool resident = false;     // whole state is one tile
    std::vector<FOp> ops;
    std::vector<cd> pool;
    std::vector<Pass> passes;
    std::vector<uint64_t> bvec;  // tile bases of the passes (m per non-event pass)
    uint64_t gates = 0;
    uint64_t measurements = 0;
    uint64_t hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// Matrix of one gate record (dim 2 or 4, row-major, 2q basis l = b_q0 + 2 b_q1).
// Returns the dimension, or 0 for a non-unitary record, -1 for an unknown op.
int gate_matrix(const qsim_gate &g, const double *mats, size_t n_mats, cd *out);

// Validates records; on error returns false and fills err.
bool validate(int n, const qsim_gate *g, size_t n_gates, const double *mats, size_t n_mats,
              std::string &err);

// Stages 1-4 of the paper (fusion=1) or one op per gate (fusion=0); fusion=2
// additionally replaces every recognised Pauli-gadget block (basis change,
// CX network computing a parity, RZ, the network reversed, the basis change
// undone) by one Pauli rotation before the four stages run on the rest.
// Rotations on more than max_rotation_qubits qubits are left as gates.
void fuse(int n, const qsim_gate *g, size_t n_gates, const double *mats, size_t n_mats,
          int fusion, std::vector<FOp> &ops, std::vector<cd> &pool, uint64_t *n_meas,
          int max_rotation_qubits);

// Full compile of one stream (fusion + schedule + k-merge) for n qubits.
void compile(int n, qsim_dtype dtype, const Config &cfg, const qsim_gate *g, size_t n_gates,
             const double *mats, size_t n_mats, HostProgram &out);

}  // namespace qsim
