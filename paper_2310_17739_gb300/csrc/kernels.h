// kernels.h -- internal launch interface between the host runtime (capi.cpp)
// and the sm_103a kernels (kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace qsim {

// One instruction of a device program (16 bytes).  k > 0: dense 2^k x 2^k
// complex matrix at mats[mat] (row-major), bit j of the local matrix index
// <-> tile position lq[j].  k == 0: event `ev` (1 measure, 2 reset) on global
// qubit lq[0], flags bit 0 = assertion mode.  k == 7: Pauli rotation in tile
// coordinates: X mask lq[0..1], Z mask lq[2..3], lq[4] bit 0 = odd (the pair
// factor is i W rather than W), Z parity mask over the tile origin's bits in
// flags | pad << 16, coefficient (cos theta, W) at mats[mat]:
//   a'_j = cos a_j + W (odd ? i : 1) (-1)^{parity(k & z) ^ parity(zc & tile)} a_k,  k = j ^ x.
// lq[4] bit 1 = scaled: the coefficient is (cos theta, t = W / cos theta) and
// the op computes a'_j = a_j + t (odd ? i : 1) (...) a_k, the missing cosine
// being part of the pass's write-back factor (TileArgs::wscale).
// Inside a register segment a rotation is a RegRot instead.
struct DevOp {
    uint8_t k;
    uint8_t ev;
    uint16_t flags;
    uint8_t lq[6];
    uint16_t pad;
    uint32_t mat;
};
static_assert(sizeof(DevOp) == 16, "DevOp layout");

// Measurement control block of one state (device memory).
struct MeasCtl {
    int32_t status;       // sticky: 0 or QSIM_E_ZEROPROB
    int32_t outcome;      // last outcome (for the collapse kernel)
    double scale;         // 1/sqrt(p_outcome) of the last measurement
    double success;       // product of asserted P(0)
    uint32_t arrive;      // block arrival counter of the grid reduction
    uint32_t pad;
    double p0, p1;        // raw sums of the last measurement
    uint64_t fail_log;    // log index of the measurement that failed
};

struct MeasRec {
    int32_t outcome;
    int32_t pad;
    double prob;
};

// A state run resident in one block's shared memory.
struct Instance {
    void *state;
    const DevOp *ops;
    const void *mats;
    uint64_t n_ops;
    uint64_t seed;
    uint64_t ordinal0;     // draw ordinal of the first event
    uint64_t log0;         // log index of the first event
    uint64_t log_cap;
    MeasCtl *ctl;
    MeasRec *log;
    double thr;
    int32_t n;
    uint32_t flags;        // kInstInit: start from |0...0> and a cleared control block
};
constexpr uint32_t kInstInit = 1;

// One batched expectation job: terms (x, z, coef bits) of one state.
struct ExpectJob {
    const void *state;
    const uint64_t *terms;
    double *out;
    uint32_t n_terms;
    int32_t n;
};

struct MeasArgs {
    int q;
    int mode;       // bit 0 assertion
    int reset;      // 1: RESET (draw, then move |1> onto |0>)
    int pad;
    uint64_t seed;
    uint64_t ordinal;
    uint64_t log_idx;
    uint64_t log_cap;
    double thr;
};

// dtype: 0 = complex64, 1 = complex128 (values of qsim_dtype).
cudaError_t setup_kernels();
size_t resident_smem_bytes(int dtype, int n);
int max_resident_bits(int dtype);

// One tile pass: its op slice ops[0, n_ops) and coefficient slice (mat_count
// complex values starting at element mat_first of the pool; op.mat relative to
// mat_first) are copied into shared memory together with the tile.
struct TileArgs {
    void *state;
    const DevOp *ops;
    const void *mats;
    const MeasCtl *ctl;
    uint32_t n_ops;
    uint32_t mat_first;
    uint32_t mat_count;
    int n;
    int m;
    int L;
    uint32_t cta_first;  // multi-state launches: first block of this state's pass
    uint32_t pad;
    float scale;         // register-segment passes: factor applied when the tile is written back
    uint32_t pad2;
    double wscale;       // generic passes: factor applied when the tile is written back (the
                         // product of the cosines of its scaled rotations; 1 = none)
    uint64_t bv[16];     // tile basis: tile bit j <-> amplitude-index XOR bv[j] (m entries)
    uint8_t ntq[48];     // non-pivot qubits, ascending (n - m entries): the tile origin's bits
};
// Fill a TileArgs for a pass whose tile subspace has pivot positions
// `pivots` and basis vectors basis[0..m) (returns false if it cannot run).
bool make_tile_args(int dtype, void *state, int n, int m, uint64_t pivots, const uint64_t *basis,
                    const DevOp *ops, uint32_t n_ops, const void *mats, uint32_t mat_first,
                    uint32_t mat_count, const MeasCtl *ctl, TileArgs *out);
// Whether the generic tile pass (k_tile_pass, k_tile_pass_multi) can run a
// tile: it tabulates the offsets of the 2^(m-L) tile rows in a fixed shared
// array of 1024 entries.
bool generic_tile_ok(const TileArgs &a);
// A complex64 pass laid out in register segments (see kSegMarker): 2^(m-5)
// threads, 32 amplitudes each; 10 <= m <= 14, n <= 32.  Its rotations carry
// (cos, t = W / cos) and run as a' = a + t (...) with the cosines' product
// `scale` applied when the tile is written back.  dense: the pass also holds
// RegDense ops (a separate build of the kernel; rotation-only passes keep the
// build without them).
cudaError_t launch_rot_pass(void *state, int n, int m, uint64_t pivots, const uint64_t *basis,
                            const DevOp *ops, uint32_t n_ops, const void *mats, uint32_t mat_first,
                            uint32_t mat_count, float scale, bool dense, const MeasCtl *ctl, cudaStream_t s);
// Register-segment passes of several states in one launch: descs[0..n_desc)
// in device memory with increasing cta_first, each made by make_tile_args
// (with its scale) for a register-segment pass of tile size m (all equal);
// dense as for launch_rot_pass (any of them holds RegDense ops).
cudaError_t launch_rot_pass_multi(const TileArgs *d_descs, int n_desc, uint32_t total_ctas, int m, bool dense,
                                  cudaStream_t s);
// The same pass with resident blocks taking tiles from the device counter
// *ctr (numbers base .. base + 2^(n-m) - 1 are this pass's tiles), each
// prefetching its next tile while it computes the current one.  A launch
// advances the counter by exactly 2^(n-m) + *grid_used.  10 <= m <= 13,
// n <= 32, and the basis must start with the unit vectors of qubits 0..3.
cudaError_t launch_rot_pipe(void *state, int n, int m, uint64_t pivots, const uint64_t *basis,
                            const DevOp *ops, uint32_t n_ops, const void *mats, uint32_t mat_first,
                            uint32_t mat_count, float scale, const MeasCtl *ctl, unsigned long long *ctr,
                            unsigned long long base, uint32_t *grid_used, cudaStream_t s);
// Op-size marker of a register segment: lq[0..4] = the 5 tile positions held
// in registers, flags = number of rotations that follow in the segment.
constexpr uint8_t kSegMarker = 8;
// Monomial 1- and 2-qubit ops (at most one nonzero entry per row: diagonal
// gates, permutations such as X, CX, SWAP, and their products with phases):
// as a dense op of k = 1 / 2 qubits (lq, mat), but only the entry of each row
// r in column perm[r] = (flags >> 2r) & 3 is used (a row without a nonzero
// names column 0, whose entry is then zero):
//   out_r = M[r][perm[r]] * in_{perm[r]}.
constexpr uint8_t kMono1 = 9;
constexpr uint8_t kMono2 = 10;
// A rotation inside a register segment (the 16 bytes of a DevOp slot).  sel =
// xr << 1 | odd, xr its X mask over the segment's 5 register slots; zt its
// tile-local Z mask; zc as in DevOp; tab = offset (in floats, a multiple of
// 4) of its coefficient table in the pass's coefficient slice.  The table
// lists u_p = t (-1)^{parity(j_p & zr)}, t = W / cos theta, zr the Z mask over
// the register slots, for the pairs p = 0..15 (j_p = p with a zero inserted
// at xr's top bit; for xr = 0, the 32 slots), followed by the same values
// negated; a thread takes the negated half when parity(zt & tb) ^
// parity(zc & tile) = 1.  Then, for the pairs (j, k = j ^ xr):
//   odd:  a'_j = a_j + i u a_k,  a'_k = a_k + i u a_j
//   even: a'_j = a_j - u a_k,    a'_k = a_k + u a_j
// (xr = 0: a'_j = (1 + u (odd ? i : 1)) a_j), and the cosines multiply the
// tile when it is written back.
struct RegRot {
    uint8_t k;  // kPauli
    uint8_t sel;
    uint16_t zt;
    uint32_t tab;
    uint32_t zc;
    uint32_t pad;
};
static_assert(sizeof(RegRot) == sizeof(DevOp), "RegRot layout");
// A dense 1- or 2-qubit op inside a register segment (the 16 bytes of a
// DevOp slot), k = kDenseReg.  sel names the kind and the register slots:
//   0..4    C1 on slot s = sel
//   5..14   C2 on the slot pair number sel - 5 of (0,1) (0,2) (0,3) (0,4) (1,2)
//           (1,3) (1,4) (2,3) (2,4) (3,4)
//   15..19  monomial C1 on slot sel - 15
//   20..49  monomial C2 on the slot pair number (sel - 20) % 10 whose row r
//           uses column col_r of pattern (sel - 20) / 10: 0 diagonal
//           (0,1,2,3), 1 (0,3,2,1), 2 (0,1,3,2); a monomial C2 of another
//           pattern is emitted as a dense C2
// Its 2^k x 2^k complex matrix (row-major, bit 0 of the local index <-> the
// lower slot) is at float offset tab (a multiple of 4) of the pass's
// coefficient slice; a monomial C1 uses only the entry in column
// perm[r] = (perm >> 2r) & 3 of each row r (as kMono1), a monomial C2 only
// the entries its pattern names.
constexpr uint8_t kDenseReg = 11;
struct RegDense {
    uint8_t k;  // kDenseReg
    uint8_t sel;
    uint16_t perm;
    uint32_t tab;
    uint32_t pad0;
    uint32_t pad1;
};
static_assert(sizeof(RegDense) == sizeof(DevOp), "RegDense layout");
// Several states' passes in one launch: descs[0..n_desc) in device memory with
// increasing cta_first; total_ctas blocks; max_m the largest tile among them.
cudaError_t launch_tile_pass_multi(int dtype, int threads, int kmax, const TileArgs *d_descs,
                                   int n_desc, uint32_t total_ctas, int max_m, cudaStream_t s);

// Per-pass limits of the tile kernel: the pass's ops and coefficients are
// copied into shared memory next to the tile.
constexpr int kPassOps = 256;
constexpr int kPassMats = 1024;  // complex values (one 5-qubit block, or 64 C2)
size_t tile_smem_bytes(int dtype, int m);

// One tile pass over ops[0, n_ops) whose coefficients are mats[mat_first,
// mat_first + mat_count) (op.mat relative to mat_first).  kmax: largest dense
// op (qubits); <= 2 selects the register-lean build without k >= 3 paths.
cudaError_t launch_tile_pass(int dtype, int threads, int kmax, void *state, int n, int m,
                             uint64_t pivots, const uint64_t *basis, const DevOp *ops, uint32_t n_ops,
                             const void *mats, uint32_t mat_first, uint32_t mat_count, double wscale,
                             const MeasCtl *ctl, cudaStream_t s);
// Resident whole-state interpreter; kmax as for launch_tile_pass.  The batch
// form runs one block per instance, shared memory sized for max_n qubits.
cudaError_t launch_resident(int dtype, int kmax, const Instance &inst, cudaStream_t s);
cudaError_t launch_resident_batch(int dtype, int kmax, const Instance *d_insts, int count,
                                  int max_n, cudaStream_t s);
// Grid size (blocks) the probability reduction uses for an n-qubit state;
// partials must hold that many double2.
int prob_blocks(int n);
cudaError_t launch_measure(int dtype, void *state, int n, const MeasArgs &a, double *partials,
                           MeasCtl *ctl, MeasRec *log, cudaStream_t s);
// Born probabilities only (no draw, no collapse): writes ctl->p0, ctl->p1.
cudaError_t launch_prob_only(int dtype, const void *state, int n, int q, double *partials,
                             MeasCtl *ctl, cudaStream_t s);
// One block per job (states of <= 14 qubits): every term of the job in turn.
cudaError_t launch_expect_batch(int dtype, const ExpectJob *d_jobs, int count, cudaStream_t s);
int expect_blocks(int n);
cudaError_t launch_expect(int dtype, const void *state, int n, const uint64_t *d_terms,
                          size_t n_terms, double *partials, double *d_out, cudaStream_t s);
cudaError_t launch_set_basis(int dtype, void *state, int n, uint64_t index, cudaStream_t s);
// Final-state shots (see qsim_sample): chunks of sample_chunk(n) consecutive
// amplitudes; partials holds 2^n / chunk doubles, offsets one more, d_out
// `shots` words.
int sample_chunk(int n);
cudaError_t launch_sample(int dtype, const void *state, int n, uint64_t mask, uint64_t shots, uint64_t seed,
                          double *partials, double *offsets, uint64_t *d_out, cudaStream_t s);

}  // namespace qsim
